"""The allocation-free conserved-sums entry point, lbm_conserved_sums_static.

Some callers cannot let a library allocate device memory. Examples are an application that
hands out every buffer from its own pool, or a loop that cannot take the implicit
synchronisation of cudaMalloc/cudaFree. They pass their own populations, flags and output
buffer, and the library uses a fixed scratch array. These tests check, through the C ABI,
that it returns the same FP64 sums as the handle-based lbm_reduce on two calls in a row
(the second call reuses the scratch left by the first), and that it rejects what it cannot
handle before any kernel runs.
"""
import numpy as np
import pytest

from gpu_helpers import case, gpu_lattice, prm
from paper_2010_11751_b300 import inputs as I
from paper_2010_11751_b300 import lbm as L

pytestmark = pytest.mark.gpu

MAX_CELLS = 33554432


def _static_sums(torch, Q, N, f_dev, flags_dev):
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    L.lbm_conserved_sums_static(Q, N, f_dev, flags_dev, out)
    torch.cuda.synchronize()
    m, e = out.cpu().tolist()
    return m, e


@pytest.mark.parametrize("Q", [19, 27])
def test_matches_lbm_reduce_on_two_consecutive_calls(Q):
    torch = pytest.importorskip("torch")
    dims = (20, 18, 24)  # 8640 cells: five 2048-cell blocks, the last one ragged
    N = dims[0] * dims[1] * dims[2]
    flags, f0 = case(Q, dims, seed=81)
    flags_dev = torch.from_numpy(flags.copy()).cuda()
    f_dev = torch.empty(Q * N, dtype=torch.float64, device="cuda")
    results = []
    with gpu_lattice(Q, dims, flags, "TRT", prm(), "aa") as g:
        g.set_populations(f0)
        for _ in range(2):
            g.step(3)
            m_ref, e_ref = g.reduce()
            g.get_populations(f_dev)
            torch.cuda.synchronize()
            m, e = _static_sums(torch, Q, N, f_dev, flags_dev)
            assert abs(m - m_ref) <= 1e-13 * m_ref
            assert abs(e - e_ref) <= 1e-10 * e_ref
            results.append((m, e))
    assert results[0][1] != results[1][1]  # the second call saw a different state


def test_matches_lbm_reduce_at_256_cubed():
    torch = pytest.importorskip("torch")
    n, Q = 256, 19
    N = n ** 3
    flags = I.cavity_flags(n, n, n)
    rho, u = I.taylor_green_fields(n, n, n, 0.02)
    flags_dev = torch.from_numpy(flags).cuda()
    f_dev = torch.empty(Q * N, dtype=torch.float64, device="cuda")
    with L.Lattice(Q, n, n, n, "aa", "BGK_W2", 1.9, flags, wall_velocities={I.LID: (0.02, 0.0, 0.0)}) as g:
        g.init_equilibrium(rho, u.ravel())
        for _ in range(2):
            g.step(1)
            m_ref, e_ref = g.reduce()
            g.get_populations(f_dev)
            torch.cuda.synchronize()
            m, e = _static_sums(torch, Q, N, f_dev, flags_dev)
            assert abs(m - m_ref) <= 1e-13 * m_ref
            assert abs(e - e_ref) <= 1e-10 * e_ref


def test_rejects_sizes_and_host_pointers_without_launching():
    torch = pytest.importorskip("torch")
    Q = 19
    f_dev = torch.zeros(Q * 64, dtype=torch.float64, device="cuda")
    flags_dev = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for bad_n in (0, -5, MAX_CELLS + 1):
        with pytest.raises(L.LBMError) as ei:
            L.lbm_conserved_sums_static(Q, bad_n, f_dev, flags_dev, out)
        assert ei.value.code == L.ERR_INVALID_ARG
        assert "33554432" in str(ei.value) or bad_n < 1
    with pytest.raises(L.LBMError) as ei:
        L.lbm_conserved_sums_static(21, 64, f_dev, flags_dev, out)
    assert ei.value.code == L.ERR_INVALID_ARG
    host_f = np.zeros(Q * 64)
    with pytest.raises(L.LBMError) as ei:
        L.lbm_conserved_sums_static(Q, 64, host_f, flags_dev, out)
    assert ei.value.code == L.ERR_INVALID_ARG
    torch.cuda.synchronize()


def test_rejects_wrong_dtype_and_short_buffers():
    """Bad buffers are refused before the C call can launch anything: a float32 f, an f or
    out with too few elements, and flags of the wrong type."""
    torch = pytest.importorskip("torch")
    Q, N = 19, 64
    f_dev = torch.zeros(Q * N, dtype=torch.float64, device="cuda")
    flags_dev = torch.zeros(N, dtype=torch.uint8, device="cuda")
    out = torch.full((2,), -7.0, dtype=torch.float64, device="cuda")
    bad = [(f_dev.float(), flags_dev, out), (f_dev[: Q * N - 1], flags_dev, out), (f_dev, flags_dev.int(), out),
           (f_dev, flags_dev[: N - 3], out), (f_dev, flags_dev, out[:1])]
    for f, fl, o in bad:
        with pytest.raises(L.LBMError) as ei:
            L.lbm_conserved_sums_static(Q, N, f, fl, o)
        assert ei.value.code == L.ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert out.tolist() == [-7.0, -7.0]  # nothing was launched


def test_no_device_memory_is_taken():
    """After a first call (which may load the library's device code), further calls leave
    the device's free memory unchanged: the scratch is the library's fixed array."""
    torch = pytest.importorskip("torch")
    Q, N = 27, 40000
    f_dev = torch.rand(Q * N, dtype=torch.float64, device="cuda") + 0.01
    flags_dev = torch.zeros(N, dtype=torch.uint8, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    L.lbm_conserved_sums_static(Q, N, f_dev, flags_dev, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        L.lbm_conserved_sums_static(Q, N, f_dev, flags_dev, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert abs(out[0].item() - f_dev.sum().item()) <= 1e-12 * f_dev.sum().item()
