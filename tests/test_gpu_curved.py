"""Walls at a fraction of their links (lbm_set_link_fractions) on the GPU, against the oracle's
orc_step_curved (the curved-wall extension of link-wise bounce-back the paper points to in
Section 1, pinned in tests/test_oracle_curved.py).

* Random obstacles of three wall kinds (two moving) with a random fraction on every wall link
  (some exactly 1/2), random out-of-equilibrium states: the two-population FP64 path against the
  oracle within 1e-12 per population, and every other scheme (swap, AA -- staged for FP64 BGK-W2
  and TRT -- esoteric twist) and the AoS layout bit-identical to it (Section 2.3, Table 1: every
  scheme computes the same map), for several collision models on D3Q19 and D3Q27.
* FP32 and FP16 shifted storage: schemes bit-identical, and the oracle within the short-run
  budgets of the precision form.
* All fractions 1/2 give the halfway bounce-back bit for bit; removing the fractions restores it.
* lbm_step_sums: the same populations as lbm_step, sums against lbm_reduce.
* Fractions outside (0, 1] on a wall link are refused; such a handle cannot join a batch.
"""
import numpy as np
import pytest

from gpu_helpers import RTOL_F64, SCHEMES, WALLS, case, gpu_lattice, prm, rel_err
from oracle import oracle as O
from paper_2010_11751_b300 import lbm as L

pytestmark = pytest.mark.gpu

DIMS = (11, 9, 13)  # 1287 cells: several blocks, a ragged tail, walls next to faces


def _fractions(Q, dims, flags, seed):
    """A fraction in (0, 1] on every link of a fluid cell that meets a wall (a quarter of them
    exactly 1/2), 1/2 elsewhere."""
    rng = np.random.default_rng(seed)
    N = int(np.prod(dims))
    q = rng.uniform(0.05, 1.0, size=(Q, N))
    q[rng.uniform(size=(Q, N)) < 0.25] = 0.5
    return q


def _oracle(Q, dims, flags, model, p, f0, q, steps):
    lat = O.Lattice(Q, *dims, flags, model, O.params(p["omega"], p["omega_bulk"], p["omega_high"], p["trt_lambda"]),
                    WALLS)
    lat.f = f0.copy()
    lat.qfrac = q
    lat.step(steps)
    return lat.f


def _gpu(Q, dims, flags, model, p, f0, q, steps, scheme="twopop", layout=L.SOA, precision=L.F64):
    with gpu_lattice(Q, dims, flags, model, p, scheme, layout, precision) as g:
        g.set_link_fractions(q)
        g.set_populations(f0)
        g.step(steps)
        return g.get_populations().copy()


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", ["BGK_W2", "TRT", "REG", "RR", "K"])
def test_fp64_matches_oracle_and_schemes_agree(Q, model):
    p = prm()
    flags, f0 = case(Q, DIMS, seed=301, model=model)
    q = _fractions(Q, DIMS, flags, seed=302)
    for steps in (1, 5):
        ref = _oracle(Q, DIMS, flags, model, p, f0, q, steps)
        base = _gpu(Q, DIMS, flags, model, p, f0, q, steps)
        assert rel_err(base, ref, flags) <= RTOL_F64, steps
        for scheme in ("swap", "aa", "esotwist"):
            for layout in (L.SOA, L.AOS):
                got = _gpu(Q, DIMS, flags, model, p, f0, q, steps, scheme=scheme, layout=layout)
                assert np.array_equal(got, base), (scheme, layout, steps)


@pytest.mark.parametrize("precision,rtol", [(L.F32, 2e-5), (L.F16, 3e-3)])
@pytest.mark.parametrize("model", ["BGK_W2", "TRT", "K"])
def test_shifted_storage(precision, rtol, model):
    Q, p = 19, prm()
    flags, f0 = case(Q, DIMS, seed=311, model=model)
    q = _fractions(Q, DIMS, flags, seed=312)
    ref = _oracle(Q, DIMS, flags, model, p, f0, q, 4)
    base = _gpu(Q, DIMS, flags, model, p, f0, q, 4, precision=precision)
    assert rel_err(base, ref, flags) <= rtol
    for scheme in ("swap", "aa", "esotwist"):
        got = _gpu(Q, DIMS, flags, model, p, f0, q, 4, scheme=scheme, precision=precision)
        assert np.array_equal(got, base), scheme


def test_half_fractions_are_the_halfway_bounce_back():
    Q, p = 19, prm()
    flags, f0 = case(Q, DIMS, seed=321)
    plain = {}
    for scheme in SCHEMES:
        with gpu_lattice(Q, DIMS, flags, "TRT", p, scheme) as g:
            g.set_populations(f0)
            g.step(4)
            plain[scheme] = g.get_populations().copy()
            b0 = L.lbm_device_bytes(g.h)
            g.set_link_fractions(np.full((Q, g.N), 0.5))  # no link away from 1/2: no tables
            assert L.lbm_device_bytes(g.h) == b0
        half = _gpu(Q, DIMS, flags, "TRT", p, f0, np.full((Q, int(np.prod(DIMS))), 0.5), 4, scheme=scheme)
        assert np.array_equal(half, plain[scheme])
    q = _fractions(Q, DIMS, flags, seed=322)
    with gpu_lattice(Q, DIMS, flags, "TRT", p, "aa") as g:
        g.set_link_fractions(q)
        g.set_link_fractions(None)  # removed again before any step
        g.set_populations(f0)
        g.step(4)
        assert np.array_equal(g.get_populations(), plain["aa"])


@pytest.mark.parametrize("scheme", ["twopop", "aa", "esotwist"])
def test_step_sums(scheme):
    Q, p = 19, prm()
    flags, f0 = case(Q, DIMS, seed=331)
    q = _fractions(Q, DIMS, flags, seed=332)
    base = _gpu(Q, DIMS, flags, "BGK_W2", p, f0, q, 3, scheme=scheme)
    with gpu_lattice(Q, DIMS, flags, "BGK_W2", p, scheme) as g:
        g.set_link_fractions(q)
        g.set_populations(f0)
        sums = []
        for _ in range(3):
            m_ref, e_ref = g.reduce()
            m, e = g.step_sums(1)
            assert abs(m - m_ref) <= 1e-13 * m_ref and abs(e - e_ref) <= 1e-10 * e_ref
            sums.append((m, e))
        assert np.array_equal(g.get_populations(), base)


def test_refused_fractions_and_batches():
    Q, p = 19, prm()
    flags, f0 = case(Q, DIMS, seed=341)
    N = int(np.prod(DIMS))
    with gpu_lattice(Q, DIMS, flags, "BGK_W2", p, "aa") as g:
        for bad in (0.0, -0.2, 1.5, np.nan):
            q = np.full((Q, N), bad)
            with pytest.raises(L.LBMError) as e:
                g.set_link_fractions(q)
            assert e.value.code == L.ERR_INVALID_ARG
        with pytest.raises(L.LBMError):
            g.set_link_fractions(np.full((Q, N - 1), 0.5))
        g.set_link_fractions(_fractions(Q, DIMS, flags, seed=342))
        with L.Batch() as b:
            with pytest.raises(L.LBMError) as e:
                b.add(g)
            assert e.value.code == L.ERR_UNSUPPORTED
