"""The bounded waits of the staged FP16 AA step, made to give up on purpose.

The staged kernel's copy pipeline waits on mbarriers (consumers for a stage's copies, the
producer for a stage's release).  Each wait is bounded; LBM_PARAM_WAIT_CYCLES shrinks the
bound to a single clock cycle, far below a copy's latency, so the waits give up.  The
kernel must then record the timeout in its error word, let every block drain its own bulk
copies before it exits, and leave the GPU context usable: lbm_reduce and the host
lbm_get_populations report LBM_ERR_TIMEOUT, and a fresh handle with the default bound steps
cleanly and bit-identically to the one-thread-per-cell kernels.
"""
import numpy as np
import pytest

from paper_2010_11751_b300 import inputs as I
from paper_2010_11751_b300 import lbm as L

pytestmark = pytest.mark.gpu

N = 128
LID = {I.LID: (0.02, 0.0, 0.0)}


def _lattice(scheme, **kw):
    omega = 1.0 / (3.0 * I.cavity_nu(0.02, N, 1000.0) + 0.5)
    return L.Lattice(19, N, N, N, scheme, "BGK_W2", omega, I.cavity_flags(N, N, N), precision=L.F16,
                     wall_velocities=LID, **kw)


def test_staged_wait_timeout_is_reported_and_the_context_survives():
    with _lattice("aa") as g:
        g.init_equilibrium()
        g.step(2)
        g.reduce()  # default bound: clean
        g.set_param(L.PARAM_WAIT_CYCLES, 1)
        g.step(4)
        with pytest.raises(L.LBMError) as e:
            g.reduce()
        assert e.value.code == L.ERR_TIMEOUT
        with pytest.raises(L.LBMError) as e:
            g.get_populations()
        assert e.value.code == L.ERR_TIMEOUT
    # the context is intact: a fresh handle with the default bound runs cleanly, and its
    # staged steps still match the two-population kernels bit for bit
    out = {}
    for scheme in ("aa", "twopop"):
        with _lattice(scheme) as g:
            g.init_equilibrium()
            g.step(7)
            m, e = g.reduce()
            assert np.isfinite(m) and np.isfinite(e)
            out[scheme] = g.get_populations().copy()
    assert np.array_equal(out["aa"], out["twopop"])


def test_wait_cycles_range_is_checked():
    with _lattice("aa") as g:
        for bad in (0.0, -5.0, 2.0 ** 41, float("nan")):
            with pytest.raises(L.LBMError) as e:
                g.set_param(L.PARAM_WAIT_CYCLES, bad)
            assert e.value.code == L.ERR_INVALID_ARG
        g.set_param(L.PARAM_WAIT_CYCLES, 2.0 ** 32)
