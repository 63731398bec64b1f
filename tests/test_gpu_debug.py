"""The bounds-checked build, liblbm_debug.so (kernels compiled with -DLBM_DEBUG), on the tiny
and ragged parity cases.

Every kernel of that build checks each population load and store, each own and neighbour cell
index, each flag and solid-neighbour mask read, each bulk copy of the staged AA steps (against
the array plus its 128 bytes of padding) and each read of a staged run against its extent, and
records the first failure per handle; the padding holds canary bytes.  These tests run the
paths that touch memory -- every scheme and layout, FP64 / FP32 / FP16 storage, the staged AA
steps (FP16, and FP64 BGK-W2 / TRT) over many tiles with ragged last tiles, the listed-cell
and curved-wall kernels, the summing steps, the state kernels and a batch -- through that
build, check that no fault was recorded and no canary was touched, and that the results still
match the FP64 oracle (the checks are in-bounds no-ops when nothing is wrong).
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import RTOL_F64, SCHEMES, WALLS, case, gpu_lattice, oracle_run, prm, rel_err
from oracle import oracle as O
from paper_2010_11751_b300 import build as B
from paper_2010_11751_b300 import inputs as I
from paper_2010_11751_b300 import lbm as L

pytestmark = pytest.mark.gpu

# the debug build holds these collision models
DEBUG_MODELS = ["BGK_W2", "TRT", "K"]
TINY = [(1, 1, 1), (1, 5, 7), (2, 3, 4), (3, 3, 3), (5, 1, 2), (7, 6, 5)]
# many staged tiles (1024 / 512 cells FP16, 128 FP64) with a ragged last one, and a z extent
# whose rows straddle 128-byte boundaries
RAGGED = (13, 11, 17)
# short-run budgets of shifted storage against the FP64 oracle (as in the curved-wall tests)
RTOL = {L.F64: RTOL_F64, L.F32: 2e-5, L.F16: 3e-3}


@pytest.fixture(scope="module", autouse=True)
def debug_lib():
    B.build(debug=True)
    with L.debug_library():
        yield


def _run(Q, dims, flags, model, p, f0, steps, scheme="twopop", layout=L.SOA, precision=L.F64, q=None):
    with gpu_lattice(Q, dims, flags, model, p, scheme, layout, precision) as g:
        if q is not None:
            g.set_link_fractions(q)
        g.set_populations(f0)
        g.step(steps)
        got = g.get_populations().copy()
        g.macroscopic()
        g.reduce()
        fault = g.debug_check()
    assert fault == 0, (hex(fault), L.DEBUG_FAULTS.get(fault >> 56))
    return got


def test_release_library_has_no_checks():
    release = L._load(L.LIBRARY)
    h = ctypes.c_void_p()
    flags = np.zeros(27, np.uint8)
    assert release.lbm_create(ctypes.byref(h), 19, 3, 3, 3, L.AA, L.BGK_W2, 1.2, flags.ctypes.data) == L.OK
    try:
        w = ctypes.c_ulonglong(7)
        assert release.lbm_debug_check(h, ctypes.byref(w)) == L.ERR_UNSUPPORTED
        assert w.value == 0
    finally:
        release.lbm_destroy(h)


def test_models_outside_the_debug_build_are_refused():
    flags = np.zeros(27, np.uint8)
    with pytest.raises(L.LBMError) as ei:
        L.Lattice(19, 3, 3, 3, "aa", "RR", 1.2, flags)
    assert ei.value.code == L.ERR_UNSUPPORTED


@pytest.mark.parametrize("dims", TINY)
@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_tiny_sizes_every_scheme(dims, scheme):
    Q, model, p = 19, "K", prm()
    nx, ny, nz = dims
    flags = I.random_obstacle_flags(nx, ny, nz, 0.2 if nx * ny * nz > 8 else 0.0, seed=51)
    rho, u = I.smooth_random_fields(nx, ny, nz, seed=52)
    ref0 = O.Lattice(Q, nx, ny, nz, flags, model, O.params(1.0), WALLS)
    ref0.init_equilibrium(rho, u)
    f0 = ref0.f * I.noise(ref0.f.shape, 0.05, seed=53)
    ref = oracle_run(Q, dims, flags, model, p, f0, 5)
    for layout in (L.SOA, L.AOS):
        got = _run(Q, dims, flags, model, p, f0, 5, scheme=scheme, layout=layout)
        if (flags == 0).any():
            assert rel_err(got, ref.f, flags) <= RTOL_F64


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", DEBUG_MODELS)
@pytest.mark.parametrize("precision", [L.F64, L.F32, L.F16])
def test_ragged_lattice_every_scheme_and_precision(Q, model, precision):
    """AA in FP16 (every model) and FP64 (BGK-W2, TRT) runs the staged step and its listed-cell
    kernel; odd and even step counts end on either AA kernel."""
    p = prm()
    flags, f0 = case(Q, RAGGED, seed=611, model=model)
    for steps in (5, 6):
        ref = oracle_run(Q, RAGGED, flags, model, p, f0, steps)
        for scheme in SCHEMES:
            got = _run(Q, RAGGED, flags, model, p, f0, steps, scheme=scheme, precision=precision)
            assert rel_err(got, ref.f, flags) <= RTOL[precision], (scheme, steps)


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 4), (3, 3, 40), (5, 7, 33)])
@pytest.mark.parametrize("precision", [L.F64, L.F16])
def test_staged_steps_on_degenerate_sizes(dims, precision):
    """A single cell, lattices smaller than one tile, and z rows that are not a multiple of the
    128-byte copy unit: the widened copies stay inside the padding."""
    Q, model, p = 27, "TRT", prm()
    flags, f0 = case(Q, dims, seed=621, model=model, solid=0.1 if np.prod(dims) > 8 else 0.0)
    ref = oracle_run(Q, dims, flags, model, p, f0, 7)
    got = _run(Q, dims, flags, model, p, f0, 7, scheme="aa", precision=precision)
    if (flags == 0).any():
        assert rel_err(got, ref.f, flags) <= RTOL[precision]


@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_curved_walls_and_step_sums(scheme):
    Q, model, p = 19, "TRT", prm()
    flags, f0 = case(Q, RAGGED, seed=631, model=model)
    rng = np.random.default_rng(632)
    q = rng.uniform(0.05, 1.0, size=(Q, int(np.prod(RAGGED))))
    with gpu_lattice(Q, RAGGED, flags, model, p, scheme) as g:
        g.set_link_fractions(q)
        g.set_populations(f0)
        g.step_sums(3)
        g.step(2)
        g.step_sums(1)
        assert g.debug_check() == 0


def test_batch_members():
    Q, model, p = 19, "TRT", prm()
    lats = []
    try:
        for s, dims in enumerate([(9, 8, 7), (16, 5, 11), (3, 3, 3)]):
            flags, f0 = case(Q, dims, seed=640 + s, model=model)
            g = L.Lattice(Q, *dims, "aa", model, p["omega"], flags, precision=L.F32, wall_velocities=WALLS,
                          omega_bulk=p["omega_bulk"], trt_lambda=p["trt_lambda"])
            g.set_populations(f0)
            g.step(s)  # members of both step parities
            lats.append(g)
        with L.Batch(lats) as b:
            for threads, cpt in ((128, 2), (32, 4), (256, 1)):
                b.set_launch(threads, cpt)
                b.step(3, use_graph=False)
            b.sync()
        for g in lats:
            assert g.debug_check() == 0
    finally:
        for g in lats:
            g.close()
