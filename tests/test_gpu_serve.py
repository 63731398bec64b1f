"""Serving form on the GPU: requests of mixed lattice, workload, collision and precision run
concurrently through the continuous-batching scheduler; every result must equal the same
request run alone (FP32: bitwise, the same per-cell kernel code; FP64: within 1e-12)."""
import numpy as np
import pytest

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


def test_mixed_results_equal_alone():
    trace = _trace()
    be = GpuBackend()
    sched = Scheduler(be, tick_steps=16)
    res = sched.run(trace, time_scale=1.0)
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
