// step_table.cu -- model dispatch of the step kernels.
//
// The bounds-checked build (LBM_DEBUG, liblbm_debug.so) holds three models:
// BGK-W2 and TRT (with their FP64 integer / double-float collisions and the
// staged AA steps) and the cumulant model (the moment-space path); the other
// models are not built there and report LBM_ERR_UNSUPPORTED.
#include "batch.cuh"
#include "internal.h"
#include "kernels.cuh"

#ifdef LBM_DEBUG
#define LBM_FULL_ONLY(...)
#else
#define LBM_FULL_ONLY(...) __VA_ARGS__
#endif

namespace lbm {
StepFn step_fn_bgk_w2(int, int, int, int);
StepFn step_fn_bgk_nw4(int, int, int, int);
StepFn step_fn_trt(int, int, int, int);
StepFn step_fn_reg(int, int, int, int);
StepFn step_fn_rr(int, int, int, int);
StepFn step_fn_rm(int, int, int, int);
StepFn step_fn_hm(int, int, int, int);
StepFn step_fn_cm(int, int, int, int);
StepFn step_fn_chm(int, int, int, int);
StepFn step_fn_k(int, int, int, int);
StepFn step_fn_bgk_w2_loop(int, int, int, int);
StepFn step_fn_bgk_w2_edu(int, int, int, int);

BatchFn batch_fn_bgk_w2(int, int);
BatchFn batch_fn_bgk_nw4(int, int);
BatchFn batch_fn_trt(int, int);
BatchFn batch_fn_reg(int, int);
BatchFn batch_fn_rr(int, int);
BatchFn batch_fn_rm(int, int);
BatchFn batch_fn_hm(int, int);
BatchFn batch_fn_cm(int, int);
BatchFn batch_fn_chm(int, int);
BatchFn batch_fn_k(int, int);
BatchFn batch_fn_bgk_w2_loop(int, int);
BatchFn batch_fn_bgk_w2_edu(int, int);

StepSumFn step_sum_fn_bgk_w2(int, int, int, int);
StepSumFn step_sum_fn_bgk_nw4(int, int, int, int);
StepSumFn step_sum_fn_trt(int, int, int, int);
StepSumFn step_sum_fn_reg(int, int, int, int);
StepSumFn step_sum_fn_rr(int, int, int, int);
StepSumFn step_sum_fn_rm(int, int, int, int);
StepSumFn step_sum_fn_hm(int, int, int, int);
StepSumFn step_sum_fn_cm(int, int, int, int);
StepSumFn step_sum_fn_chm(int, int, int, int);
StepSumFn step_sum_fn_k(int, int, int, int);
StepSumFn step_sum_fn_bgk_w2_loop(int, int, int, int);
StepSumFn step_sum_fn_bgk_w2_edu(int, int, int, int);
StagedFn staged_fn_bgk_w2(int, int, int);
StagedFn staged_fn_bgk_nw4(int, int, int);
StagedFn staged_fn_trt(int, int, int);
StagedFn staged_fn_reg(int, int, int);
StagedFn staged_fn_rr(int, int, int);
StagedFn staged_fn_rm(int, int, int);
StagedFn staged_fn_hm(int, int, int);
StagedFn staged_fn_cm(int, int, int);
StagedFn staged_fn_chm(int, int, int);
StagedFn staged_fn_k(int, int, int);
StagedFn staged_fn_bgk_w2_loop(int, int, int);
StagedFn staged_fn_bgk_w2_edu(int, int, int);

CurvedFn curved_fn_bgk_nw4(int, int, int, int);
CurvedFn curved_fn_bgk_w2(int, int, int, int);
CurvedFn curved_fn_bgk_w2_edu(int, int, int, int);
CurvedFn curved_fn_bgk_w2_loop(int, int, int, int);
CurvedFn curved_fn_chm(int, int, int, int);
CurvedFn curved_fn_cm(int, int, int, int);
CurvedFn curved_fn_hm(int, int, int, int);
CurvedFn curved_fn_k(int, int, int, int);
CurvedFn curved_fn_reg(int, int, int, int);
CurvedFn curved_fn_rm(int, int, int, int);
CurvedFn curved_fn_rr(int, int, int, int);
CurvedFn curved_fn_trt(int, int, int, int);

StepFn step_fn(int model, int Q, int P, int L, int SK) {
  switch (model) {
    case BGK_W2: return step_fn_bgk_w2(Q, P, L, SK);
    LBM_FULL_ONLY(case BGK_NW4: return step_fn_bgk_nw4(Q, P, L, SK);)
    case TRT: return step_fn_trt(Q, P, L, SK);
    LBM_FULL_ONLY(case REG: return step_fn_reg(Q, P, L, SK);)
    LBM_FULL_ONLY(case RR: return step_fn_rr(Q, P, L, SK);)
    LBM_FULL_ONLY(case RM: return step_fn_rm(Q, P, L, SK);)
    LBM_FULL_ONLY(case HM: return step_fn_hm(Q, P, L, SK);)
    LBM_FULL_ONLY(case CM: return step_fn_cm(Q, P, L, SK);)
    LBM_FULL_ONLY(case CHM: return step_fn_chm(Q, P, L, SK);)
    case KUM: return step_fn_k(Q, P, L, SK);
    LBM_FULL_ONLY(case BGK_W2_LOOP: return step_fn_bgk_w2_loop(Q, P, L, SK);)
    LBM_FULL_ONLY(case BGK_W2_EDU: return step_fn_bgk_w2_edu(Q, P, L, SK);)
    default: return nullptr;
  }
}

CurvedFn curved_fn(int model, int Q, int P, int L, int SK) {
  switch (model) {
    case BGK_W2: return curved_fn_bgk_w2(Q, P, L, SK);
    LBM_FULL_ONLY(case BGK_NW4: return curved_fn_bgk_nw4(Q, P, L, SK);)
    case TRT: return curved_fn_trt(Q, P, L, SK);
    LBM_FULL_ONLY(case REG: return curved_fn_reg(Q, P, L, SK);)
    LBM_FULL_ONLY(case RR: return curved_fn_rr(Q, P, L, SK);)
    LBM_FULL_ONLY(case RM: return curved_fn_rm(Q, P, L, SK);)
    LBM_FULL_ONLY(case HM: return curved_fn_hm(Q, P, L, SK);)
    LBM_FULL_ONLY(case CM: return curved_fn_cm(Q, P, L, SK);)
    LBM_FULL_ONLY(case CHM: return curved_fn_chm(Q, P, L, SK);)
    case KUM: return curved_fn_k(Q, P, L, SK);
    LBM_FULL_ONLY(case BGK_W2_LOOP: return curved_fn_bgk_w2_loop(Q, P, L, SK);)
    LBM_FULL_ONLY(case BGK_W2_EDU: return curved_fn_bgk_w2_edu(Q, P, L, SK);)
    default: return nullptr;
  }
}
BatchFn batch_fn(int model, int Q, int P) {
  switch (model) {
    case BGK_W2: return batch_fn_bgk_w2(Q, P);
    LBM_FULL_ONLY(case BGK_NW4: return batch_fn_bgk_nw4(Q, P);)
    case TRT: return batch_fn_trt(Q, P);
    LBM_FULL_ONLY(case REG: return batch_fn_reg(Q, P);)
    LBM_FULL_ONLY(case RR: return batch_fn_rr(Q, P);)
    LBM_FULL_ONLY(case RM: return batch_fn_rm(Q, P);)
    LBM_FULL_ONLY(case HM: return batch_fn_hm(Q, P);)
    LBM_FULL_ONLY(case CM: return batch_fn_cm(Q, P);)
    LBM_FULL_ONLY(case CHM: return batch_fn_chm(Q, P);)
    case KUM: return batch_fn_k(Q, P);
    LBM_FULL_ONLY(case BGK_W2_LOOP: return batch_fn_bgk_w2_loop(Q, P);)
    LBM_FULL_ONLY(case BGK_W2_EDU: return batch_fn_bgk_w2_edu(Q, P);)
    default: return nullptr;
  }
}
StagedFn staged_fn(int model, int Q, int P, int SK) {
  switch (model) {
    case BGK_W2: return staged_fn_bgk_w2(Q, P, SK);
    LBM_FULL_ONLY(case BGK_NW4: return staged_fn_bgk_nw4(Q, P, SK);)
    case TRT: return staged_fn_trt(Q, P, SK);
    LBM_FULL_ONLY(case REG: return staged_fn_reg(Q, P, SK);)
    LBM_FULL_ONLY(case RR: return staged_fn_rr(Q, P, SK);)
    LBM_FULL_ONLY(case RM: return staged_fn_rm(Q, P, SK);)
    LBM_FULL_ONLY(case HM: return staged_fn_hm(Q, P, SK);)
    LBM_FULL_ONLY(case CM: return staged_fn_cm(Q, P, SK);)
    LBM_FULL_ONLY(case CHM: return staged_fn_chm(Q, P, SK);)
    case KUM: return staged_fn_k(Q, P, SK);
    LBM_FULL_ONLY(case BGK_W2_LOOP: return staged_fn_bgk_w2_loop(Q, P, SK);)
    LBM_FULL_ONLY(case BGK_W2_EDU: return staged_fn_bgk_w2_edu(Q, P, SK);)
    default: return nullptr;
  }
}
StepSumFn step_sum_fn(int model, int Q, int P, int L, int SK) {
  switch (model) {
    case BGK_W2: return step_sum_fn_bgk_w2(Q, P, L, SK);
    LBM_FULL_ONLY(case BGK_NW4: return step_sum_fn_bgk_nw4(Q, P, L, SK);)
    case TRT: return step_sum_fn_trt(Q, P, L, SK);
    LBM_FULL_ONLY(case REG: return step_sum_fn_reg(Q, P, L, SK);)
    LBM_FULL_ONLY(case RR: return step_sum_fn_rr(Q, P, L, SK);)
    LBM_FULL_ONLY(case RM: return step_sum_fn_rm(Q, P, L, SK);)
    LBM_FULL_ONLY(case HM: return step_sum_fn_hm(Q, P, L, SK);)
    LBM_FULL_ONLY(case CM: return step_sum_fn_cm(Q, P, L, SK);)
    LBM_FULL_ONLY(case CHM: return step_sum_fn_chm(Q, P, L, SK);)
    case KUM: return step_sum_fn_k(Q, P, L, SK);
    LBM_FULL_ONLY(case BGK_W2_LOOP: return step_sum_fn_bgk_w2_loop(Q, P, L, SK);)
    LBM_FULL_ONLY(case BGK_W2_EDU: return step_sum_fn_bgk_w2_edu(Q, P, L, SK);)
    default: return nullptr;
  }
}
}  // namespace lbm
