"""GPU parity at the sizes the benchmark and the precision form run, against the FP64 oracle.

* D3Q19 lid-driven cavity 256^3, Re 1000, AA pattern, SoA, FP64, BGK-W2 -- the benchmark's
  headline workload and launch configuration -- started from rest with 5 % multiplicative
  noise on every population (so that every cell is out of equilibrium), 6 steps (three even
  and three odd AA kernels), compared with the oracle population by population within
  1e-12; once through lbm_step and once through lbm_step_sums, whose per-step FP64 mass
  and energy are checked against correctly rounded sums of the oracle's per-cell density and
  velocity of the same states.
* The same cavity with TRT in FP16 shifted storage: the staged AA step (persistent grid of
  two blocks per SM walking ~55 tiles each, plus the listed-cell kernel), 6 steps, within
  the FP16 short-run budget.
* D3Q27 cavity 256^3 FP64 BGK-W2, AA (the staged step with three blocks per SM), 4 steps,
  within 1e-12 (the bench line's D3Q27 form); D3Q19 256^3 RR (the matrix's size), 4 steps.
* D3Q19 512^3 (the precision form's size) in FP64, FP32 and FP16, Taylor-Green (u0 = 0.05:
  in FP64 the wide range of the BGK-W2 fast path) and noisy cavity:
  the oracle is too slow for whole 512^3 steps, so it steps windows of 24^3 cells cut from
  the GPU's state; after one step every cell at least one cell inside the window depends
  only on populations inside it (streaming moves one cell per step), so those cells are
  compared with the GPU's own next state.  Both an even and an odd AA step are checked.

The oracle uses every host core (OpenMP); whole-lattice comparisons go one population at a
time to bound host memory.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_11751_b300 import inputs as I
from paper_2010_11751_b300 import lbm as L

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1
LID = {I.LID: (0.02, 0.0, 0.0)}


def _cavity(n, model, seed, Q=19):
    flags = I.cavity_flags(n, n, n)
    omega = 1.0 / (3.0 * I.cavity_nu(0.02, n, 1000.0) + 0.5)
    ref = O.Lattice(Q, n, n, n, flags, model, O.params(omega), LID)
    ref.init_equilibrium()
    ref.f *= I.noise(ref.f.shape, 0.05, seed=seed)
    ref.f[:, flags != 0] = 0.0
    return flags, omega, ref


def _max_rel(got, ref, fluid):
    err = 0.0
    for k in range(ref.shape[0]):
        err = max(err, float(np.max(np.abs(got[k, fluid] - ref[k, fluid]) / np.abs(ref[k, fluid]))))
    return err


def _exact_sums(ref, fluid):
    """Mass and energy of the oracle's state, from its per-cell rho and u, each summed with
    math.fsum (correctly rounded): at 16.8M cells a plain sequential sum is itself off by
    ~1e-13, more than the GPU's tree sum."""
    rho, u = ref.macroscopic()
    ke = 0.5 * rho * (u * u).sum(0)
    return math.fsum(rho[fluid]), math.fsum(ke[fluid])


@pytest.fixture(scope="module")
def cavity256_bgk():
    """The oracle's 6 steps of the noisy 256^3 cavity, with its sums before every step."""
    n = 256
    flags, omega, ref = _cavity(n, "BGK_W2", seed=2561)
    f0 = ref.f.copy()
    sums = []
    for _ in range(6):
        sums.append(_exact_sums(ref, flags == 0))
        ref.step(1, nthreads=THREADS)
    return dict(n=n, flags=flags, omega=omega, f0=f0, f6=ref.f, sums=sums)


@pytest.mark.parametrize("entry", ["lbm_step", "lbm_step_sums"])
def test_headline_cavity256_fp64_aa_matches_oracle(cavity256_bgk, entry):
    c = cavity256_bgk
    n, flags = c["n"], c["flags"]
    with L.Lattice(19, n, n, n, "aa", "BGK_W2", c["omega"], flags, wall_velocities=LID) as g:
        g.set_populations(c["f0"])
        if entry == "lbm_step":
            g.step(6)
        else:
            for s in range(6):
                m, e = g.step_sums(1)
                m_o, e_o = c["sums"][s]
                assert abs(m - m_o) <= 1e-13 * m_o, (s, m, m_o)
                assert abs(e - e_o) <= 1e-10 * e_o, (s, e, e_o)
        got = g.get_populations()
    assert _max_rel(got, c["f6"], flags == 0) <= 1e-12
    assert not got[:, flags != 0].any()


def test_cavity256_fp16_staged_aa_matches_oracle():
    n = 256
    flags, omega, ref = _cavity(n, "TRT", seed=2562)
    with L.Lattice(19, n, n, n, "aa", "TRT", omega, flags, precision=L.F16, wall_velocities=LID) as g:
        assert L.lbm_kernels_per_step(g.h) == 2  # staged bulk kernel + listed-cell kernel
        g.set_populations(ref.f)
        g.step(6)
        got = g.get_populations()
        m, e = g.reduce()  # LBM_ERR_TIMEOUT here if a staged wait had given up
    ref.step(6, nthreads=THREADS)
    assert np.isfinite(m) and np.isfinite(e)
    assert _max_rel(got, ref.f, flags == 0) <= 3e-3


def test_cavity256_d3q27_fp64_staged_aa_matches_oracle():
    n = 256
    flags, omega, ref = _cavity(n, "BGK_W2", seed=2563, Q=27)
    with L.Lattice(27, n, n, n, "aa", "BGK_W2", omega, flags, wall_velocities=LID) as g:
        assert L.lbm_kernels_per_step(g.h) == 2  # staged bulk kernel + listed-cell kernel
        g.set_populations(ref.f)
        g.step(4)
        got = g.get_populations()
    ref.step(4, nthreads=THREADS)
    assert _max_rel(got, ref.f, flags == 0) <= 1e-12


def test_cavity256_rr_fp64_matches_oracle():
    """The recursive-regularized collision at the matrix's size: D3Q19 256^3 noisy cavity, AA
    (its one-thread-per-cell kernels, the integer / double-float route for most cells), 4 steps,
    within 1e-12."""
    n = 256
    flags, omega, ref = _cavity(n, "RR", seed=2564)
    with L.Lattice(19, n, n, n, "aa", "RR", omega, flags, wall_velocities=LID) as g:
        g.set_populations(ref.f)
        g.step(4)
        got = g.get_populations()
    ref.step(4, nthreads=THREADS)
    assert _max_rel(got, ref.f, flags == 0) <= 1e-12


def _window(f_dev, flags, n, corner, w):
    x0, y0, z0 = corner
    fw = f_dev.view(19, n, n, n)[:, x0:x0 + w, y0:y0 + w, z0:z0 + w].cpu().numpy().reshape(19, -1)
    fl = flags.reshape(n, n, n)[x0:x0 + w, y0:y0 + w, z0:z0 + w].reshape(-1).copy()
    return np.ascontiguousarray(fw), fl


@pytest.mark.parametrize("precision,workload,tol", [("f64", "taylor_green", 1e-12), ("f64", "cavity", 1e-12),
                                                    ("f32", "taylor_green", 2e-6), ("f32", "cavity", 2e-6),
                                                    ("f16", "taylor_green", 1e-3), ("f16", "cavity", 1e-3)])
def test_512_windows_one_step_against_oracle(precision, workload, tol):
    import torch

    n, w = 512, 24
    if workload == "taylor_green":
        u0, model = 0.05, "BGK_W2"
        flags, walls = I.periodic_flags(n, n, n), {}
        omega = 1.0 / (3.0 * (u0 * n / 1000.0) + 0.5)
        rho, u = I.taylor_green_fields_torch(n, n, n, u0)
        corners = [(0, 0, 0), (200, 311, 77), (n - w, n - w, n - w)]
    else:
        model = "TRT"
        flags, walls = I.cavity_flags(n, n, n), LID
        omega = 1.0 / (3.0 * I.cavity_nu(0.02, n, 1000.0) + 0.5)
        rho = u = None
        corners = [(0, 0, n - w), (n - w, 100, n - w), (0, n - w, 0), (250, 260, 270)]
    with L.Lattice(19, n, n, n, "aa", model, omega, flags, precision=L.PRECISIONS[precision],
                   wall_velocities=walls) as g:
        g.init_equilibrium(rho, u)
        g.step(3)
        del rho, u
        f_dev = torch.empty(19 * n ** 3, dtype=torch.float64, device="cuda")
        g.get_populations(f_dev)
        torch.cuda.synchronize()
        before = [_window(f_dev, flags, n, c, w) for c in corners]
        for parity in range(2):  # step 4 (odd AA kernel), then step 5 (even)
            g.step(1)
            g.get_populations(f_dev)
            torch.cuda.synchronize()
            after = [_window(f_dev, flags, n, c, w)[0] for c in corners]
            for (fw, fl), fa in zip(before, after):
                lat = O.Lattice(19, w, w, w, fl, model, O.params(omega), walls)
                lat.f = fw.copy()
                lat.step(1)
                inner = np.zeros((w, w, w), bool)
                inner[1:-1, 1:-1, 1:-1] = True
                fluid = inner.reshape(-1) & (fl == 0)
                assert fluid.sum() > 0
                err = _max_rel(fa, lat.f, fluid)
                assert err <= tol, (parity, err)
            before = [_window(f_dev, flags, n, c, w) for c in corners]
        m, e = g.reduce()
        assert np.isfinite(m) and np.isfinite(e)
        del f_dev
        torch.cuda.empty_cache()
