"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle.

* every collision model on D3Q19 and D3Q27, two-population SoA FP64, element by element,
  within 1e-12 relative per population, on a lattice that spans several thread blocks with a
  ragged tail, random walls of three kinds and periodic wrap;
* every scheme (swap, AA, esoteric twist) and the AoS layout bit-identical to the
  two-population scheme after odd and even step counts (the six strategies of Section 2.3
  compute the same map);
* macroscopic fields, conserved sums and the equilibrium initialisation against the oracle;
* the 32^3 cavity (BGK-W2, two-population SoA, Re 100, 100 steps) element by element;
* degenerate sizes, checkpoint/resume across parities, host and device buffers.
"""
import numpy as np
import pytest

from gpu_helpers import MODELS, RTOL_F64, SCHEMES, WALLS, case, gpu_lattice, gpu_run, oracle_run, prm, rel_err
from oracle import oracle as O
from paper_2010_11751_b300 import inputs as I
from paper_2010_11751_b300 import lbm as L

pytestmark = pytest.mark.gpu

DIMS = (10, 9, 12)  # 1080 cells: five 256-thread blocks, the last one ragged


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", MODELS)
def test_twopop_matches_oracle(Q, model):
    p = prm()
    flags, f0 = case(Q, DIMS, seed=11, model=model)
    ref = oracle_run(Q, DIMS, flags, model, p, f0, 6)
    got = gpu_run(Q, DIMS, flags, model, p, f0, 6)
    assert rel_err(got, ref.f, flags) <= RTOL_F64
    assert np.all(got[:, flags != 0] == 0.0)


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", MODELS)
def test_schemes_and_layouts_bit_identical(Q, model):
    p = prm()
    flags, f0 = case(Q, DIMS, seed=21, model=model)
    for steps in (5, 6):
        base = gpu_run(Q, DIMS, flags, model, p, f0, steps)
        for name in ("swap", "aa", "esotwist"):
            for layout in (L.SOA, L.AOS):
                got = gpu_run(Q, DIMS, flags, model, p, f0, steps, scheme=name, layout=layout)
                assert np.array_equal(got, base), (name, layout, steps)
        got = gpu_run(Q, DIMS, flags, model, p, f0, steps, scheme="twopop", layout=L.AOS)
        assert np.array_equal(got, base)


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_macroscopic_and_conserved_sums(Q, scheme):
    p = prm()
    flags, f0 = case(Q, DIMS, seed=31)
    for steps in (3, 4):
        ref = oracle_run(Q, DIMS, flags, "TRT", p, f0, steps)
        rho_o, u_o = ref.macroscopic()
        m_o, e_o = ref.conserved()
        with gpu_lattice(Q, DIMS, flags, "TRT", p, scheme) as g:
            g.set_populations(f0)
            g.step(steps)
            rho, u = g.macroscopic()
            m, e = g.reduce()
        assert np.max(np.abs(rho - rho_o) / rho_o) < 1e-13
        assert np.max(np.abs(u - u_o)) < 1e-13
        assert abs(m - m_o) <= 1e-13 * m_o
        assert abs(e - e_o) <= 1e-10 * e_o


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", ["BGK_W2", "BGK_NW4", "K"])
@pytest.mark.parametrize("scheme", ["twopop", "esotwist"])
def test_init_equilibrium(Q, model, scheme):
    nx, ny, nz = DIMS
    flags = I.random_obstacle_flags(nx, ny, nz, 0.1, seed=41)
    rho, u = I.smooth_random_fields(nx, ny, nz, amp=0.05, seed=42)
    ref = O.Lattice(Q, nx, ny, nz, flags, model, O.params(1.0), WALLS)
    ref.init_equilibrium(rho, u)
    with gpu_lattice(Q, DIMS, flags, model, prm(), scheme) as g:
        g.init_equilibrium(np.ascontiguousarray(rho), np.ascontiguousarray(u))
        got = g.get_populations()
    assert rel_err(got, ref.f, flags) < 1e-14


def test_cavity_32_bgk_twopop_100_steps():
    n = 32
    flags = I.cavity_flags(n, n, n)
    nu = I.cavity_nu(0.02, n, 100.0)
    omega = 1.0 / (3.0 * nu + 0.5)
    ref = O.Lattice(19, n, n, n, flags, "BGK_W2", O.params(omega), {I.LID: (0.02, 0.0, 0.0)})
    ref.init_equilibrium(1.0, np.zeros((3, n ** 3)))
    ref.step(100)
    with L.Lattice(19, n, n, n, "twopop", "BGK_W2", omega, flags, wall_velocities={I.LID: (0.02, 0.0, 0.0)}) as g:
        g.init_equilibrium()
        g.step(100)
        got = g.get_populations()
        m, _ = g.reduce()
    assert rel_err(got, ref.f, flags) <= RTOL_F64
    m0 = float((flags == 0).sum())
    assert abs(m - m0) <= 1e-12 * m0


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 5, 7), (2, 3, 4), (3, 3, 3), (5, 1, 2), (7, 6, 5)])
@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_degenerate_and_tiny_sizes(dims, scheme):
    Q, model, p = 19, "K", prm()
    nx, ny, nz = dims
    flags = I.random_obstacle_flags(nx, ny, nz, 0.2 if nx * ny * nz > 8 else 0.0, seed=51)
    rho, u = I.smooth_random_fields(nx, ny, nz, seed=52)
    ref0 = O.Lattice(Q, nx, ny, nz, flags, model, O.params(1.0), WALLS)
    ref0.init_equilibrium(rho, u)
    f0 = ref0.f * I.noise(ref0.f.shape, 0.05, seed=53)
    ref = oracle_run(Q, dims, flags, model, p, f0, 5)
    got = gpu_run(Q, dims, flags, model, p, f0, 5, scheme=scheme)
    if (flags == 0).any():
        assert rel_err(got, ref.f, flags) <= RTOL_F64


@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_all_solid_lattice(scheme):
    flags = np.ones(4 * 4 * 4, np.uint8)
    with L.Lattice(27, 4, 4, 4, scheme, "BGK_W2", 1.2, flags) as g:
        g.init_equilibrium()
        g.step(3)
        m, e = g.reduce()
        rho, u = g.macroscopic()
    assert m == 0.0 and e == 0.0
    assert np.all(rho == 1.0) and np.all(u == 0.0)


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_checkpoint_resume_bit_identical(Q, scheme):
    p = prm()
    flags, f0 = case(Q, DIMS, seed=61)
    full = gpu_run(Q, DIMS, flags, "RR", p, f0, 7, scheme=scheme)
    with gpu_lattice(Q, DIMS, flags, "RR", p, scheme) as g:
        g.set_populations(f0)
        g.step(3)  # odd parity for AA and the esoteric twist
        mid = g.get_populations().copy()
    resumed = gpu_run(Q, DIMS, flags, "RR", p, mid, 4, scheme=scheme)
    assert np.array_equal(full, resumed)


def test_host_and_device_buffers_agree():
    torch = pytest.importorskip("torch")
    Q, p = 19, prm()
    flags, f0 = case(Q, DIMS, seed=71)
    with gpu_lattice(Q, DIMS, flags, "CM", p, "aa") as g:
        g.set_populations(torch.from_numpy(f0.ravel().copy()).cuda())
        g.step(3)
        fd = torch.empty(Q * g.N, dtype=torch.float64, device="cuda")
        g.get_populations(fd)
        rd = torch.empty(g.N, dtype=torch.float64, device="cuda")
        ud = torch.empty(3 * g.N, dtype=torch.float64, device="cuda")
        g.macroscopic(rd, ud)
        torch.cuda.synchronize()
        fh = g.get_populations()
        rh, uh = g.macroscopic()
    assert np.array_equal(fd.cpu().numpy().reshape(Q, -1), fh)
    assert np.array_equal(rd.cpu().numpy(), rh) and np.array_equal(ud.cpu().numpy().reshape(3, -1), uh)
    ref = oracle_run(Q, DIMS, flags, "CM", p, f0, 3)
    assert rel_err(fh, ref.f, flags) <= RTOL_F64


def test_state_errors():
    flags = np.zeros(27, np.uint8)
    with L.Lattice(19, 3, 3, 3, "aa", "BGK_W2", 1.0, flags) as g:
        with pytest.raises(L.LBMError) as ei:
            g.macroscopic()
        assert ei.value.code == L.ERR_STATE
        g.step(1)  # implicit rest equilibrium
        with pytest.raises(L.LBMError) as ei:
            L.lbm_set_precision(g.h, L.F32)
        assert ei.value.code == L.ERR_STATE
        with pytest.raises(L.LBMError) as ei:
            g.step(-1)
        assert ei.value.code == L.ERR_INVALID_ARG
        m, _ = g.reduce()
        assert abs(m - 27.0) < 1e-12
    with L.Lattice(19, 3, 3, 3, "aa", "BGK_W2", 1.0, flags) as g:
        with pytest.raises(L.LBMError) as ei:
            L.lbm_set_layout(g.h, L.AOS) or L.lbm_set_precision(g.h, L.F32)
        assert ei.value.code == L.ERR_UNSUPPORTED


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", ["RM", "HM", "CM", "CHM", "K"])
@pytest.mark.parametrize("omega_bulk", [None, 1.1])
def test_omega_high_one_path_matches_oracle(Q, model, omega_bulk):
    """With omega_high = 1 (the default) the moment models skip the high-order moments
    altogether (they relax to equilibrium); the result must still match the oracle."""
    p = prm(omega=1.45, omega_bulk=1.45 if omega_bulk is None else omega_bulk, omega_high=1.0)
    flags, f0 = case(Q, DIMS, seed=131, model=model)
    ref = oracle_run(Q, DIMS, flags, model, p, f0, 6)
    got = gpu_run(Q, DIMS, flags, model, p, f0, 6, scheme="aa")
    assert rel_err(got, ref.f, flags) <= RTOL_F64


@pytest.mark.parametrize("scheme", ["twopop", "aa"])
def test_divergence_is_reported(scheme):
    """A non-finite population (injected through the host input, no device fault) spreads
    through the collision and is reported by the FP64 conserved sums as LBM_ERR_DIVERGED."""
    Q = 19
    flags, f0 = case(Q, DIMS, seed=141)
    bad = f0.copy()
    i = int(np.flatnonzero(flags == 0)[7])
    bad[3, i] = np.nan
    with gpu_lattice(Q, DIMS, flags, "BGK_W2", prm(), scheme) as g:
        g.set_populations(bad)
        g.step(2)
        with pytest.raises(L.LBMError) as ei:
            g.reduce()
        assert ei.value.code == L.ERR_DIVERGED
    with gpu_lattice(Q, DIMS, flags, "BGK_W2", prm(), scheme) as g:
        g.set_populations(f0)
        g.step(2)
        g.reduce()  # finite state: no error


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("scheme", list(SCHEMES))
@pytest.mark.parametrize("model", ["BGK_W2", "TRT", "REG", "RR", "K"])
def test_step_sums_is_reduce_then_step(Q, scheme, model):
    """lbm_step_sums(n): the FP64 sums of the starting state (as lbm_reduce gives them, up to
    summation order) and the same populations as lbm_step(n), bit for bit, at both parities."""
    p = prm()
    flags, f0 = case(Q, DIMS, seed=151, model=model)
    for pre in (0, 1):
        with gpu_lattice(Q, DIMS, flags, model, p, scheme) as g:
            g.set_populations(f0)
            g.step(pre)
            m0, e0 = g.reduce()
            g.step(3)
            want = g.get_populations().copy()
        with gpu_lattice(Q, DIMS, flags, model, p, scheme) as g:
            g.set_populations(f0)
            g.step(pre)
            m, e = g.step_sums(3)
            got = g.get_populations().copy()
        assert np.array_equal(got, want), (scheme, pre)
        assert abs(m - m0) <= 1e-13 * m0 and abs(e - e0) <= 1e-12 * e0, (m, m0, e, e0)


def test_step_sums_fallback_and_zero_steps():
    """AoS has no summing kernel: lbm_step_sums runs the reduction, then the steps; n = 0 is
    lbm_reduce."""
    Q, p = 19, prm()
    flags, f0 = case(Q, DIMS, seed=161)
    with gpu_lattice(Q, DIMS, flags, "TRT", p, "aa", layout=L.AOS) as g:
        g.set_populations(f0)
        m0, e0 = g.reduce()
        assert g.step_sums(0) == (m0, e0)
        assert g.step_sums(2) == (m0, e0)  # the same reduction kernel: identical sums
        assert g.steps_done == 2
        m2, e2 = g.reduce()
    with gpu_lattice(Q, DIMS, flags, "TRT", p, "aa") as g:
        g.set_populations(f0)
        g.step(2)
        assert g.reduce() == (m2, e2)


@pytest.mark.parametrize("scheme", list(SCHEMES))
@pytest.mark.parametrize("model", ["BGK_W2", "K"])
def test_step_sums_async_equals_step_sums(scheme, model):
    """lbm_step_sums_async enqueues the work of lbm_step_sums: the same sums, bit for bit, into
    pinned host or device memory, with one call kept in flight while the previous call's sums
    are read; the same populations afterwards.  Pageable host memory is refused."""
    torch = pytest.importorskip("torch")
    Q, p = 19, prm()
    flags, f0 = case(Q, DIMS, seed=171, model=model)
    with gpu_lattice(Q, DIMS, flags, model, p, scheme) as g:
        g.set_populations(f0)
        sync = [g.step_sums(1) for _ in range(5)]
        f_sync = g.get_populations().copy()
    host = torch.empty((5, 2), dtype=torch.float64).pin_memory()
    dev = torch.empty((5, 2), dtype=torch.float64, device="cuda")
    for out in (host, dev):
        with gpu_lattice(Q, DIMS, flags, model, p, scheme) as g:
            g.set_populations(f0)
            for i in range(5):
                g.step_sums_async(out[i])
            torch.cuda.synchronize()
            assert [tuple(r) for r in out.cpu().tolist()] == sync
            assert np.array_equal(g.get_populations(), f_sync)
    with gpu_lattice(Q, DIMS, flags, model, p, scheme) as g:
        g.set_populations(f0)
        with pytest.raises(L.LBMError) as ei:
            g.step_sums_async(np.zeros(2))
        assert ei.value.code == L.ERR_INVALID_ARG
        with pytest.raises(L.LBMError) as ei:
            g.step_sums_async(host[0], n=0)
        assert ei.value.code == L.ERR_INVALID_ARG
        assert g.steps_done == 0


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", ["BGK_W2_EDU", "BGK_W2_LOOP"])
@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_educational_bgk_matches_oracle(Q, model, scheme):
    """BGK-W2 in the educational form of Section 2.6 (loops over the directions, tabulated c_k
    and t_k) computes the oracle's BGK-W2 within the FP64 tolerance in every scheme."""
    p = prm()
    flags, f0 = case(Q, DIMS, seed=181, model="BGK_W2")
    ref = oracle_run(Q, DIMS, flags, "BGK_W2", p, f0, 5)
    got = gpu_run(Q, DIMS, flags, model, p, f0, 5, scheme=scheme)
    assert rel_err(got, ref.f, flags) <= RTOL_F64
    assert np.all(got[:, flags != 0] == 0.0)


def test_out_of_device_memory_is_reported():
    """A lattice whose populations cannot fit in device memory (D3Q27 FP64, 1200^3 cells:
    373 GB) is created (flags and masks fit), and the first call that writes populations reports
    LBM_ERR_OOM without allocating them; the handle stays usable for destroy."""
    n = 1200
    flags = np.zeros(n ** 3, np.uint8)
    g = L.Lattice(27, n, n, n, "aa", "BGK_W2", 1.2, flags)
    try:
        with pytest.raises(L.LBMError) as ei:
            g.init_equilibrium()
        assert ei.value.code == L.ERR_OOM
        with pytest.raises(L.LBMError) as ei:
            g.step(1)  # implicit initialisation: the same pre-flight check
        assert ei.value.code == L.ERR_OOM
    finally:
        g.close()
