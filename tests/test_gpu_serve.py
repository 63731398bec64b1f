"""Serving form on the GPU: requests of mixed lattice, workload, collision and precision run
concurrently through the continuous-batching scheduler (arrival order and least-work-first
admission, fixed and timed ticks); every result must equal the same request run alone (FP32:
bitwise, the same per-cell kernel code; FP64: within 1e-12), and match the FP64 oracle run on
the same request: FP64 centre-line profiles and masses within 1e-12, FP32 profiles within the
FP32 cavity budget (1e-4 of the lid or Taylor-Green velocity)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_11751_b300 import inputs as I
from paper_2010_11751_b300.serve import GpuBackend, Request, Scheduler, summarize

pytestmark = pytest.mark.gpu


def _trace():
    g = np.random.default_rng(77)
    out = []
    for i in range(12):
        out.append(Request(i, 0.004 * i, int(g.choice([19, 27])), str(g.choice(["cavity", "taylor_green"])),
                           str(g.choice(["BGK_W2", "K"])), str(g.choice(["f32", "f64"])), int(g.integers(10, 25)),
                           int(g.integers(15, 70))))
    return out


def _oracle_result(req):
    """The oracle's run of a served request (same lattice set-up as GpuBackend.make_lattice)."""
    n = req.side
    if req.workload == "cavity":
        nu = I.cavity_nu(GpuBackend.U_LID, n, req.reynolds)
        flags, walls = I.cavity_flags(n, n, n), {I.LID: (GpuBackend.U_LID, 0.0, 0.0)}
        rho = u = None
    else:
        nu = GpuBackend.U0_TG * n / req.reynolds
        flags, walls = I.periodic_flags(n, n, n), {}
        rho, u = I.taylor_green_fields(n, n, n, GpuBackend.U0_TG)
    lat = O.Lattice(req.lattice, n, n, n, flags, req.collision, O.params(1.0 / (3.0 * nu + 0.5)), walls)
    lat.init_equilibrium(rho, u)
    lat.step(req.steps)
    _, uu = lat.macroscopic()
    m, _ = lat.conserved()
    return uu[0].reshape(n, n, n)[n // 2, n // 2, :], m


@pytest.mark.parametrize("policy,tick_seconds", [("fifo", None), ("shortest", 0.002)])
def test_mixed_results_equal_alone(policy, tick_seconds):
    trace = _trace()
    be = GpuBackend()
    sched = Scheduler(be, tick_steps=16, policy=policy, tick_seconds=tick_seconds)
    res = sched.run(trace, time_scale=0.05)  # arrivals 0.2 ms apart: requests overlap
    be.close()
    assert all(r.error is None for r in res)
    assert sched.ticks > 1 and sched.max_active > 1
    alone = GpuBackend()
    for req, r in zip(trace, res):
        g = alone.make_lattice(req)
        g.step(req.steps)
        ref = alone.read_result(g)
        g.close()
        if req.precision == "f32":
            assert np.array_equal(r.profile, ref["profile"]), req
            assert r.mass == ref["mass"] and r.energy == ref["energy"]
        else:
            assert np.allclose(r.profile, ref["profile"], rtol=1e-12, atol=1e-15), req
            assert abs(r.mass - ref["mass"]) <= 1e-12 * ref["mass"]
    s = summarize(res, wall_s=max(r.finished_s for r in res))
    assert s["completed"] == len(trace)


def test_served_results_match_oracle():
    trace = _trace()
    be = GpuBackend()
    res = Scheduler(be, tick_steps=16, policy="shortest", tick_seconds=0.002).run(trace, time_scale=0.05)
    be.close()
    for req, r in zip(trace, res):
        prof, m = _oracle_result(req)
        if req.precision == "f64":
            assert np.allclose(r.profile, prof, rtol=1e-12, atol=1e-15), req
            assert abs(r.mass - m) <= 1e-12 * m, req
        else:
            # relative to the flow's velocity scale (the Taylor-Green centre line has u_x = 0)
            scale = GpuBackend.U_LID if req.workload == "cavity" else GpuBackend.U0_TG
            err = np.max(np.abs(r.profile - prof)) / scale
            assert err <= 1e-4, (req, err)
