// model_bgk_w2.cu -- step kernels of the BGK_W2 collision model for every lattice,
// storage precision, layout and step kind, and its batched (many-lattice)
// kernels (one translation unit per model so that the build parallelises).
#include "batch.cuh"
#include "internal.h"
#include "kernels.cuh"
#include "staged.cuh"

namespace lbm {
StepFn step_fn_bgk_w2(int Q, int P, int L, int SK) { return step_fn_for_model<BGK_W2>(Q, P, L, SK); }
BatchFn batch_fn_bgk_w2(int Q, int P) { return batch_fn_for_model<BGK_W2>(Q, P); }
StagedFn staged_fn_bgk_w2(int Q, int P, int SK) { return staged_fn_for_model<BGK_W2>(Q, P, SK); }
StepSumFn step_sum_fn_bgk_w2(int Q, int P, int L, int SK) { return step_sum_fn_for_model<BGK_W2>(Q, P, L, SK); }
CurvedFn curved_fn_bgk_w2(int Q, int P, int L, int SK) { return curved_fn_for_model<BGK_W2>(Q, P, L, SK); }
}  // namespace lbm
