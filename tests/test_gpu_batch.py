"""Batching form: many uneven lattices advanced by one launch per time step.

A batched step must be bit-identical to stepping each member alone (same per-cell code),
with members of different sizes, relaxation rates, wall velocities and step parities,
with and without CUDA-graph replay and for every launch shape the autotuner may pick; one
member is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

from gpu_helpers import RTOL_F64, WALLS, case, oracle_run, prm, rel_err
from paper_2010_11751_b300 import inputs as I
from paper_2010_11751_b300 import lbm as L

pytestmark = pytest.mark.gpu

SIZES = [(5, 7, 9), (12, 3, 8), (16, 16, 16), (7, 11, 4), (20, 9, 13), (3, 3, 3)]


def _members(Q, model, precision, seed):
    out = []
    for m, dims in enumerate(SIZES):
        flags, f0 = case(Q, dims, seed=seed + m, model=model)
        p = prm(omega=1.2 + 0.1 * m, omega_bulk=1.0 + 0.05 * m)
        pre = m % 2  # odd members start at odd parity
        out.append((dims, flags, f0, p, pre))
    return out


def _make(Q, model, precision, dims, flags, p):
    return L.Lattice(Q, *dims, "aa", model, p["omega"], flags, precision=precision, wall_velocities=WALLS,
                     omega_bulk=p["omega_bulk"], omega_high=p["omega_high"], trt_lambda=p["trt_lambda"])


@pytest.mark.parametrize("Q,model,precision", [(19, "TRT", L.F32), (19, "BGK_W2", L.F64), (27, "K", L.F64),
                                               (27, "BGK_W2", L.F32), (19, "K", L.F32), (19, "RR", L.F16)])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_equals_individual(Q, model, precision, use_graph):
    mem = _members(Q, model, precision, seed=200)
    alone, batched = [], []
    for dims, flags, f0, p, pre in mem:
        with _make(Q, model, precision, dims, flags, p) as g:
            g.set_populations(f0)
            g.step(pre + 8)
            alone.append(g.get_populations().copy())
    lats = []
    for dims, flags, f0, p, pre in mem:
        g = _make(Q, model, precision, dims, flags, p)
        g.set_populations(f0)
        g.step(pre)
        lats.append(g)
    with L.Batch(lats) as b:
        b.set_launch(128, 2)
        b.step(3, use_graph=use_graph)
        b.step(3, use_graph=use_graph)  # replays the captured graph
        b.set_launch(64, 4)
        b.step(1, use_graph=use_graph)
        b.set_launch(32, 1)
        b.step(1, use_graph=use_graph)
        b.sync()
        for g, ref, (_, _, _, _, pre) in zip(lats, alone, mem):
            assert g.steps_done == pre + 8
            assert np.array_equal(g.get_populations(), ref)
    for g in lats:
        g.close()


def test_batched_member_matches_oracle():
    Q, model = 19, "RR"
    dims = (14, 11, 9)
    flags, f0 = case(Q, dims, seed=300, model=model)
    p = prm()
    ref = oracle_run(Q, dims, flags, model, p, f0, 8)
    others = [_make(Q, model, L.F64, d, I.periodic_flags(*d), p) for d in [(8, 8, 8), (5, 6, 7)]]
    for g in others:
        g.init_equilibrium()
    g = _make(Q, model, L.F64, dims, flags, p)
    g.set_populations(f0)
    with L.Batch(others + [g]) as b:
        b.step(8)
        b.sync()
        got = g.get_populations()
    assert rel_err(got, ref.f, flags) <= RTOL_F64
    for h in others + [g]:
        h.close()


def test_autotune_keeps_results():
    Q, model, precision = 19, "TRT", L.F32
    mem = _members(Q, model, precision, seed=400)
    lats_a, lats_b = [], []
    for dims, flags, f0, p, pre in mem:
        for lst in (lats_a, lats_b):
            g = _make(Q, model, precision, dims, flags, p)
            g.set_populations(f0)
            lst.append(g)
    with L.Batch(lats_a) as ba, L.Batch(lats_b) as bb:
        t, c = ba.autotune()
        assert t in (32, 64, 128, 256) and c in (1, 2, 4)
        steps = lats_a[0].steps_done
        bb.step(steps, use_graph=False)
        ba.step(5)
        bb.step(5)
        ba.sync()
        bb.sync()
        for x, y in zip(lats_a, lats_b):
            assert np.array_equal(x.get_populations(), y.get_populations())
        assert ba.autotune() == (t, c)  # cached
    for g in lats_a + lats_b:
        g.close()


def test_batch_rejects_mismatched_members():
    f = I.periodic_flags(4, 4, 4)
    with L.Lattice(19, 4, 4, 4, "aa", "TRT", 1.2, f) as a, \
            L.Lattice(19, 4, 4, 4, "aa", "BGK_W2", 1.2, f) as b, \
            L.Lattice(19, 4, 4, 4, "esotwist", "TRT", 1.2, f) as c, \
            L.Lattice(27, 4, 4, 4, "aa", "TRT", 1.2, f) as d:
        with L.Batch([a]) as bt:
            for other in (b, c, d):
                with pytest.raises(L.LBMError) as ei:
                    bt.add(other)
                assert ei.value.code == L.ERR_INVALID_ARG
            with pytest.raises(L.LBMError):
                bt.add(a)
            assert bt.size == (1, 64)
            bt.remove(a)
            assert bt.size == (1 - 1, 0)


def test_batch_on_a_caller_stream_waits_for_member_set_up():
    """A batch stepped on a caller's non-blocking stream (which does not order with the legacy
    default stream) must still see its members' initialisation, enqueued on the legacy default
    stream just before, and must wait for its own earlier steps when the stream is switched."""
    import torch

    n = 96
    rho, u = I.taylor_green_fields_torch(n, n, n, 0.03)
    ref = L.Lattice(19, n, n, n, "aa", "TRT", 1.7, I.periodic_flags(n, n, n), precision=L.F32)
    ref.init_equilibrium(rho, u)
    ref.step(6)
    want = ref.get_populations()
    ref.close()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream(priority=-64)
    g = L.Lattice(19, n, n, n, "aa", "TRT", 1.7, I.periodic_flags(n, n, n), precision=L.F32)
    with L.Batch() as b:
        b.set_stream(s1.cuda_stream)
        g.init_equilibrium(rho, u)  # legacy default stream, asynchronous
        b.add(g)
        b.step(3, use_graph=False)
        b.set_stream(s2.cuda_stream)
        b.step(3, use_graph=False)
        b.sync()
        b.remove(g)
    assert np.array_equal(g.get_populations(), want)
    g.close()
