"""The routes of the FP64 BGK-W2 and TRT collisions, against the FP64 oracle.

The FP64 collisions of these models take their density and momentum as exact integer sums and
their equilibrium in double-float arithmetic when every population of a cell lies in the
binade of its lattice weight (narrow range, LBM_PARAM_FX_RANGE = 1) or also in one of the two
next to it (wide range, 2); a cell with a population outside the range takes the plain FP64
operator.  The relaxed equilibrium w E_k is assembled on the bit pattern of W_c = w t_c; a cell
whose value leaves W_c's binade is recomputed by the FP64 operator from its reloaded
populations, except in the wide range on D3Q27, where a value in a binade next to W_c's is
moved there (rounded to nearest above, exact below).  The lattice here mixes five kinds of
cell inside every warp (they alternate along z, the fastest index), with walls of three kinds
and periodic wrap, and checks, in both ranges and in the automatic choice:

* that each kind meets the condition of its route (classified on the host from the oracle's own
  equilibrium);
* one step and five steps of the CUDA path against the oracle, within 1e-12 per population,
  and the AA, swap and esoteric-twist results bit-identical to the two-population ones
  (Section 2.3, Table 1: every scheme computes the same map).  These states are far from
  equilibrium and w = 1.94 over-relaxes them, so a few populations pass close to zero in
  later steps; there a relative error means nothing, and populations below 0.1 t_k are held to
  1e-12 t_k in absolute terms instead.
"""
import numpy as np
import pytest

from gpu_helpers import RTOL_F64, WALLS
from oracle import oracle as O
from paper_2010_11751_b300 import inputs as I

pytestmark = pytest.mark.gpu

DIMS = (8, 7, 65)  # 3640 cells, rows of 65 along z: every warp holds every kind
OMEGA = 1.94  # close to the 256^3 cavity's: w t_c sits high (D3Q19) or low (D3Q27) in its binade


def _exponent(x):
    return np.frexp(x)[1]


KINDS = 5


def _mixed_state(Q, seed):
    """Cells cycle along z through:
    0. near equilibrium (small u, 1 % noise): populations in their weights' binades;
    1. flow with |u_i| up to 0.08: some populations in the binades next to their weights';
    2. populations t_k (1 + 0.11 s_k), s_k the sign of c_k . (1, 1, 0): every population in its
       weight's binade, but a momentum that takes some w E_k out of the binade of w t_k;
    3. near equilibrium with population 0 times four: outside the three binades;
    4. populations t_k (1 + a s_k), a = 0.6 (D3Q19) or 0.55 (D3Q27): inside the three
       binades, with a momentum (|u| ~ 0.2) whose w E_k are out of reach of the integer
       assembly."""
    nx, ny, nz = DIMS
    c, t, _ = O.lattice(Q)
    flags = I.random_obstacle_flags(nx, ny, nz, 0.05, seed=seed)
    rng = I.rng(seed + 1)
    N = nx * ny * nz
    f = np.zeros((Q, N))
    kind = np.arange(N) % nz % KINDS
    s = np.sign(c @ np.array([1, 1, 0]))
    for i in range(N):
        if flags[i] != 0:
            continue
        if kind[i] in (0, 3):
            u = rng.uniform(-0.01, 0.01, 3)
            f[:, i] = O.model_equilibrium(Q, "BGK_W2", 1.0 + rng.uniform(-0.01, 0.01), u)
            f[:, i] *= 1.0 + rng.uniform(-0.01, 0.01, Q)
            if kind[i] == 3:
                f[0, i] *= 4.0
        elif kind[i] == 1:
            u = rng.uniform(-0.08, 0.08, 3)
            f[:, i] = O.model_equilibrium(Q, "BGK_W2", 1.0, u) * (1.0 + rng.uniform(-0.01, 0.01, Q))
        else:
            a = 0.11 if kind[i] == 2 else (0.6 if Q == 19 else 0.55)
            f[:, i] = t * (1.0 + a * s) * (1.0 + rng.uniform(-1e-3, 1e-3, Q))
    return flags, kind, f, c, t


def _classify(Q, flags, f, c, t):
    """Per fluid cell, for BGK-W2: every population positive and at most one binade away from
    its weight's; every population in its weight's binade; every w E_k at most one binade away
    from w t_k's; every w E_k in the binade of w t_k."""
    fluid = np.flatnonzero(flags == 0)
    ef = _exponent(f[:, fluid]) - _exponent(t)[:, None]
    in_reach = np.all((f[:, fluid] > 0) & (np.abs(ef) <= 1), axis=0)
    in_binade = np.all(ef == 0, axis=0)
    w_reach = np.zeros(fluid.size, bool)
    w_binade = np.zeros(fluid.size, bool)
    W = OMEGA * t
    for n, i in enumerate(fluid):
        rho = f[:, i].sum()
        u = (c.T @ f[:, i]) / rho
        ew = _exponent(OMEGA * O.model_equilibrium(Q, "BGK_W2", rho, u)) - _exponent(W)
        w_reach[n] = np.all(np.abs(ew) <= 1)
        w_binade[n] = np.all(ew == 0)
    return in_reach, in_binade, w_reach, w_binade


def _run(Q, dims, flags, model, p, f0, steps, fx_range, scheme="twopop"):
    from paper_2010_11751_b300 import lbm as L

    with L.Lattice(Q, *dims, scheme, model, p["omega"], flags, wall_velocities=WALLS, omega_bulk=p["omega_bulk"],
                   omega_high=p["omega_high"], trt_lambda=p["trt_lambda"]) as g:
        g.set_param(L.PARAM_FX_RANGE, fx_range)
        g.set_populations(f0)
        g.step(steps)
        return g.get_populations().copy()


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", ["BGK_W2", "TRT"])
@pytest.mark.parametrize("fx_range", [1, 2, 0])
def test_fx_routes_match_oracle(Q, model, fx_range):
    flags, kind, f0, c, t = _mixed_state(Q, seed=1907 + Q)
    in_reach, in_binade, w_reach, w_binade = _classify(Q, flags, f0, c, t)
    k = kind[flags == 0]
    # each kind meets the condition of its route
    assert np.all(in_binade[k == 0] & w_binade[k == 0])
    assert np.all(in_reach[k == 1]) and np.mean(in_binade[k == 1]) < 0.1 and np.all(w_reach[k == 1])
    assert np.all(in_binade[k == 2] & w_reach[k == 2]) and not np.all(w_binade[k == 2])
    assert not np.any(in_reach[k == 3])
    assert np.all(in_reach[k == 4]) and (Q == 27 or not np.all(w_reach[k == 4]))
    p = dict(omega=OMEGA, omega_bulk=OMEGA, omega_high=1.0, trt_lambda=0.25)
    for steps in (1, 5):
        lat = O.Lattice(Q, *DIMS, flags, model, O.params(OMEGA, OMEGA, 1.0, 0.25), WALLS)
        lat.f = f0.copy()
        lat.step(steps)
        base = _run(Q, DIMS, flags, model, p, f0, steps, fx_range)
        fluid = flags == 0
        ref, got = lat.f[:, fluid], base[:, fluid]
        small = np.abs(ref) < 0.1 * t[:, None]
        scale = np.where(small, t[:, None], np.abs(ref))
        assert np.max(np.abs(got - ref) / scale) <= RTOL_F64, steps
        for scheme in ("aa", "swap", "esotwist"):
            got = _run(Q, DIMS, flags, model, p, f0, steps, fx_range, scheme=scheme)
            assert np.array_equal(got, base), (scheme, steps)
        if fx_range == 0:
            # more than 1 % of the cells have populations outside their weights' binades:
            # the automatic choice is the wide range
            assert np.array_equal(base, _run(Q, DIMS, flags, model, p, f0, steps, 2))


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", ["BGK_W2", "TRT"])
def test_fast_taylor_green_matches_oracle(Q, model):
    """A periodic Taylor-Green vortex at u0 = 0.1 (48^3, k = 2 pi / 48): most cells have
    populations in the binades next to their weights', and the AA steps run the staged kernels;
    four steps against the oracle within 1e-12 in the automatic choice (the wide range) and the
    narrow range, AA bit-identical to two-population; a cavity at rest picks the narrow range."""
    from paper_2010_11751_b300 import lbm as L

    n, u0, omega = 48, 0.1, 1.9
    flags = np.zeros(n ** 3, np.uint8)
    rho, u = I.taylor_green_fields(n, n, n, u0)
    c, t, _ = O.lattice(Q)
    ref = O.Lattice(Q, n, n, n, flags, model, O.params(omega, omega, 1.0, 0.25), {})
    ref.init_equilibrium(rho, u)
    assert np.mean(np.any(_exponent(ref.f) != _exponent(t)[:, None], axis=0)) > 0.3
    ref.step(4)
    got = {}
    for fx_range in (0, 1, 2):
        for scheme in ("aa", "twopop"):
            with L.Lattice(Q, n, n, n, scheme, model, omega, flags, omega_bulk=omega, trt_lambda=0.25) as g:
                g.set_param(L.PARAM_FX_RANGE, fx_range)
                g.init_equilibrium(rho, u.ravel())
                g.step(4)
                got[scheme, fx_range] = g.get_populations()
        assert np.max(np.abs(got["aa", fx_range] - ref.f) / np.abs(ref.f)) <= RTOL_F64, fx_range
        assert np.array_equal(got["aa", fx_range], got["twopop", fx_range]), fx_range
    assert np.array_equal(got["aa", 0], got["aa", 2])
    assert not np.array_equal(got["aa", 1], got["aa", 2])  # the ranges round differently
    # a cavity at rest: the automatic choice is the narrow range
    cflags = I.cavity_flags(24, 24, 24)
    cav = {}
    for fx_range in (0, 1):
        with L.Lattice(Q, 24, 24, 24, "aa", model, 1.9, cflags, wall_velocities={I.LID: (0.02, 0.0, 0.0)}) as g:
            g.set_param(L.PARAM_FX_RANGE, fx_range)
            g.init_equilibrium()
            g.step(30)
            cav[fx_range] = g.get_populations()
    assert np.array_equal(cav[0], cav[1])


@pytest.mark.parametrize("Q", [19, 27])
def test_rr_routes_match_oracle(Q):
    """The recursive-regularized collision in FP64 takes the same integer / double-float route
    (fx_rr.cuh) for cells whose populations lie in their weights' binades, and the FP64 operator
    for the others (and for cells whose new populations would leave them): the five kinds of cell
    above, mixed in every warp, against the oracle within 1e-12 after one and five steps, every
    scheme bit-identical to the two-population one."""
    flags, kind, f0, c, t = _mixed_state(Q, seed=2907 + Q)
    in_reach, in_binade, _, _ = _classify(Q, flags, f0, c, t)
    k = kind[flags == 0]
    assert np.all(in_binade[k == 0]) and not np.any(in_binade[k == 3])
    p = dict(omega=OMEGA, omega_bulk=1.2, omega_high=1.0, trt_lambda=0.25)
    for steps in (1, 5):
        lat = O.Lattice(Q, *DIMS, flags, "RR", O.params(OMEGA, 1.2, 1.0, 0.25), WALLS)
        lat.f = f0.copy()
        lat.step(steps)
        base = _run(Q, DIMS, flags, "RR", p, f0, steps, 0)
        fluid = flags == 0
        ref, got = lat.f[:, fluid], base[:, fluid]
        small = np.abs(ref) < 0.1 * t[:, None]
        scale = np.where(small, t[:, None], np.abs(ref))
        assert np.max(np.abs(got - ref) / scale) <= RTOL_F64, steps
        for scheme in ("aa", "swap", "esotwist"):
            got = _run(Q, DIMS, flags, "RR", p, f0, steps, 0, scheme=scheme)
            assert np.array_equal(got, base), (scheme, steps)


@pytest.mark.parametrize("Q", [19, 27])
def test_rr_cavity_near_rest_takes_the_fast_route(Q):
    """A cavity near rest: every cell stays in its weights' binades, the RR update is the
    integer / double-float one; 20 steps of a 20^3 cavity at Re 100 against the oracle."""
    n = 20
    flags = I.cavity_flags(n, n, n)
    omega = 1.0 / (3.0 * I.cavity_nu(0.02, n, 100.0) + 0.5)
    lid = {I.LID: (0.02, 0.0, 0.0)}
    ref = O.Lattice(Q, n, n, n, flags, "RR", O.params(omega), lid)
    ref.init_equilibrium()
    ref.step(20)
    from paper_2010_11751_b300 import lbm as L

    with L.Lattice(Q, n, n, n, "aa", "RR", omega, flags, wall_velocities=lid) as g:
        g.init_equilibrium()
        g.step(20)
        got = g.get_populations()
    fluid = flags == 0
    assert np.max(np.abs(got[:, fluid] - ref.f[:, fluid]) / np.abs(ref.f[:, fluid])) <= RTOL_F64
