"""Compiler resource report (nvcc -Xptxas -v) of the kernels of BGK-W2 and the cumulant model: no
stack frame and no spills in the FP64 and FP32 batch kernels (the serving mix), none in the FP64
D3Q19 single-lattice and summing step kernels (the headline step and lbm_step_sums), and at most a
few spilled words in the FP64 D3Q27 ones -- in the narrow range of the FP64 BGK-W2 fast path,
which flows near the weights run; the wide-range instantiations are held to a few words.

A batch block takes its member's relaxation rates from the member table.  When they ended up in
per-thread local memory instead of registers or shared memory, every cell's collision re-read
them from there and the FP64 BGK-W2 batch ran 20 times slower than the same lattice stepped alone,
while every result stayed bit-identical; only the resource report shows it without a GPU.  The
FP64 D3Q27 BGK-W2 step kernels hold 27 populations beside the integer and double-float state of
their collision and the route that reloads a cell (at most 128 registers): a handful of spilled
words is the measured price of keeping two blocks per SM.
"""
import os
import re
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_2010_11751_b300 import build as B

F64, F32 = 0, 1
# spilled bytes allowed in the wide-range FP64 BGK-W2 step kernels (fx64.cuh)
WIDE_LIMIT = 32
MODELS = {"model_bgk_w2.cu": 0, "model_k.cu": 9}  # the serving form's collision models


def _report(src):
    with tempfile.TemporaryDirectory() as tmp:
        cmd = [B._nvcc()] + B.FLAGS + B.ARCH + ["-Xptxas", "-v", "-c", os.path.join(B.CSRC, src),
                                                "-o", os.path.join(tmp, "x.o")]
        r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stderr


@pytest.fixture(scope="module")
def reports():
    if not os.path.exists(B._nvcc()):
        pytest.skip("nvcc not available")
    with ThreadPoolExecutor(len(MODELS)) as ex:
        return dict(zip(MODELS, ex.map(_report, MODELS)))


def _batch_kernels(text):
    out = []
    for blk in text.split("Compiling entry function")[1:]:
        name = blk.split("'")[1]
        m = re.search(r"batch_aa_kernelILi(\d+)ELi(\d+)ELi(\d+)ELi(\d+)E", name)
        if not m:
            continue
        q, model, prec, sk = map(int, m.groups())
        frame = int(re.search(r"(\d+) bytes stack frame", blk).group(1))
        spill = int(re.search(r"(\d+) bytes spill stores", blk).group(1))
        out.append((q, model, prec, sk, frame, spill))
    return out


@pytest.mark.parametrize("src", sorted(MODELS))
def test_batch_kernels_keep_rates_out_of_local_memory(reports, src):
    ks = [k for k in _batch_kernels(reports[src]) if k[2] in (F64, F32)]
    # D3Q19 and D3Q27, FP64 and FP32, even and odd AA steps
    assert len(ks) == 8 and {k[1] for k in ks} == {MODELS[src]}, ks
    bad = [k for k in ks if k[4] or k[5]]
    assert not bad, f"(Q, model, precision, step kind, stack frame, spill bytes): {bad}"


def _step_kernels(text):
    out = []
    for blk in text.split("Compiling entry function")[1:]:
        name = blk.split("'")[1]
        m = re.search(r"(step_kernel|step_sum_kernel)ILi(\d+)ELi(\d+)ELi(\d+)ELi(\d+)ELi(\d+)ELb([01])E", name)
        if not m:
            continue
        q, model, prec, layout, sk, wide = map(int, m.groups()[1:])
        frame = int(re.search(r"(\d+) bytes stack frame", blk).group(1))
        spill = int(re.search(r"(\d+) bytes spill stores", blk).group(1))
        out.append((m.group(1), q, model, prec, layout, sk, frame, spill, wide))
    return out


@pytest.mark.parametrize("src", sorted(MODELS))
def test_fp64_step_kernels_keep_everything_in_registers(reports, src):
    """The FP64 single-lattice and summing step kernels (the headline step and the first step of
    lbm_step_sums) are bound by the FP64 pipe; local-memory traffic would come on top of it."""
    ks = [k for k in _step_kernels(reports[src]) if k[3] == F64]
    # step kernels: D3Q19/D3Q27 x SoA/AoS x 4 step kinds; summing kernels: SoA only; BGK-W2 has
    # them in both ranges of its fast path
    ranges = 2 if MODELS[src] == 0 else 1
    assert len([k for k in ks if k[0] == "step_kernel"]) == 16 * ranges, ks
    assert len([k for k in ks if k[0] == "step_sum_kernel"]) == 8 * ranges, ks
    limit = {(19, 0): 0, (27, 0): 16, (19, 1): WIDE_LIMIT, (27, 1): WIDE_LIMIT}
    bad = [k for k in ks if k[6] > limit[k[1], k[8]] or k[7] > limit[k[1], k[8]]]
    assert not bad, f"(kernel, Q, model, precision, layout, step kind, stack frame, spill bytes, wide): {bad}"
