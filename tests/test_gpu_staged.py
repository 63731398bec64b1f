"""Staged AA steps -- FP16 for every model, FP64 for BGK-W2, TRT and D3Q27 RR -- (bulk cells from
shared-memory tiles filled by bulk asynchronous copies, the other fluid cells by a listed-cell
kernel) against the one-thread-per-cell kernels.

Both update every cell with the same loads, collision and stores, so the AA pattern through
the staged kernels must be bit-identical to the two-population scheme (which never stages) in
the same storage precision, for every collision model, on lattices that span many tiles with a
ragged last tile, walls of three kinds next to bulk cells, periodic faces, and degenerate
sizes down to a single cell.  The FP16 result is also held to its budget against the FP64
oracle, the FP64 one to 1e-12, and the staged kernels' error word must stay clear (lbm_reduce
would report LBM_ERR_TIMEOUT otherwise).
"""
import numpy as np
import pytest

from gpu_helpers import MODELS, RTOL_F64, case, gpu_lattice, gpu_run, oracle_run, prm, rel_err
from paper_2010_11751_b300 import inputs as I
from paper_2010_11751_b300 import lbm as L

pytestmark = pytest.mark.gpu

DIMS = (41, 23, 37)  # 34,891 cells: 34 tiles of 1024 (D3Q19) or 69 of 512 (D3Q27), ragged last


def listed_cells(flags, dims, Q):
    """Fluid cells that the staged step leaves to the listed-cell kernel: on a domain face, or
    with a solid neighbour along one of the Q - 1 lattice links (periodic box)."""
    nx, ny, nz = dims
    solid = (flags.reshape(nx, ny, nz) & 7) != 0
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    face = (x == 0) | (x == nx - 1) | (y == 0) | (y == ny - 1) | (z == 0) | (z == nz - 1)
    near = np.zeros_like(solid)
    for c in np.ndindex(3, 3, 3):
        c = np.array(c) - 1
        n2 = int((c * c).sum())
        if n2 == 0 or (Q == 19 and n2 == 3):
            continue
        near |= np.roll(solid, shift=tuple(-c), axis=(0, 1, 2))
    return int(((~solid) & (face | near)).sum())


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", MODELS)
def test_staged_aa_bit_identical_to_twopop(Q, model):
    p = prm()
    flags, f0 = case(Q, DIMS, seed=171, model=model)
    for steps in (5, 6):
        base = gpu_run(Q, DIMS, flags, model, p, f0, steps, precision=L.F16)
        got = gpu_run(Q, DIMS, flags, model, p, f0, steps, scheme="aa", precision=L.F16)
        assert np.array_equal(got, base), steps


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", ["BGK_W2", "TRT", "RR"])
def test_staged_fp64_bit_identical_to_twopop_and_oracle(Q, model):
    """FP64 staged tiles (256 cells for D3Q19, 128 for D3Q27) over many tiles with a ragged last
    one; the two-population scheme never stages."""
    p = prm()
    flags, f0 = case(Q, DIMS, seed=173, model=model)
    for steps in (5, 6):
        base = gpu_run(Q, DIMS, flags, model, p, f0, steps)
        with gpu_lattice(Q, DIMS, flags, model, p, "aa") as g:
            # staged kernel + listed-cell kernel (D3Q19 RR keeps the one-thread-per-cell kernel)
            assert L.lbm_kernels_per_step(g.h) == (1 if (model == "RR" and Q == 19) else 2)
            g.set_populations(f0)
            g.step(steps)
            got = g.get_populations().copy()
            m, e = g.reduce()
        assert np.isfinite(m) and np.isfinite(e)
        assert np.array_equal(got, base), steps
    ref = oracle_run(Q, DIMS, flags, model, p, f0, 6)
    assert rel_err(got, ref.f, flags) <= RTOL_F64


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1, 17), (2, 3, 5), (3, 1, 40), (16, 16, 16), (1, 64, 64),
                                  (5, 7, 333)])
@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("precision", [L.F16, L.F64])
def test_staged_degenerate_and_ragged_sizes(dims, Q, precision):
    p = prm()
    nx, ny, nz = dims
    solid = 0.15 if nx * ny * nz > 8 else 0.0
    flags, f0 = case(Q, dims, seed=181, solid=solid, model="TRT")
    for steps in (3, 4):
        base = gpu_run(Q, dims, flags, "TRT", p, f0, steps, precision=precision)
        got = gpu_run(Q, dims, flags, "TRT", p, f0, steps, scheme="aa", precision=precision)
        assert np.array_equal(got, base), (dims, steps)


def test_staged_periodic_and_cavity_bulk():
    # periodic box: the only listed cells are the domain faces (periodic wrap)
    n, nz = 48, 40
    flags = I.periodic_flags(n, n, nz)
    rho, u = I.taylor_green_fields(n, n, nz, 0.05)
    omega = 1.0 / (3.0 * (0.05 * n / 1000.0) + 0.5)
    out = {}
    for scheme in ("twopop", "aa"):
        with L.Lattice(19, n, n, nz, scheme, "BGK_W2", omega, flags, precision=L.F16) as g:
            g.init_equilibrium(rho, u.ravel())
            g.step(7)
            out[scheme] = g.get_populations().copy()
            m, e = g.reduce()
            assert np.isfinite(m) and np.isfinite(e)
    assert np.array_equal(out["aa"], out["twopop"])
    # cavity: walls on five faces, the lid on the sixth; listed cells line every wall
    n = 40
    flags = I.cavity_flags(n, n, n)
    omega = 1.0 / (3.0 * I.cavity_nu(0.02, n, 1000.0) + 0.5)
    for scheme in ("twopop", "aa"):
        with L.Lattice(19, n, n, n, scheme, "TRT", omega, flags, precision=L.F16,
                       wall_velocities={I.LID: (0.02, 0.0, 0.0)}) as g:
            g.init_equilibrium()
            g.step(9)
            out[scheme] = g.get_populations().copy()
    assert np.array_equal(out["aa"], out["twopop"])


@pytest.mark.parametrize("Q,model", [(19, "BGK_W2"), (27, "K")])
def test_staged_fp16_against_oracle(Q, model):
    p = prm()
    flags, f0 = case(Q, DIMS, seed=191, model=model)
    ref = oracle_run(Q, DIMS, flags, model, p, f0, 6)
    got = gpu_run(Q, DIMS, flags, model, p, f0, 6, scheme="aa", precision=L.F16)
    fluid = flags == 0
    err = np.max(np.abs(got[:, fluid] - ref.f[:, fluid]) / np.abs(ref.f[:, fluid]))
    assert err <= 3e-3, err


def test_staged_handle_reuse_and_accounting():
    """The listed cells and their records are built once, on the first staged step, and counted
    in lbm_device_bytes; stepping on after a read-back continues bit-identically."""
    Q, p = 19, prm()
    flags, f0 = case(Q, DIMS, seed=201, model="REG")
    full = gpu_run(Q, DIMS, flags, "REG", p, f0, 9, scheme="aa", precision=L.F16)
    with gpu_lattice(Q, DIMS, flags, "REG", p, "aa", precision=L.F16) as g:
        g.set_populations(f0)
        b0 = L.lbm_device_bytes(g.h)
        g.step(4)
        b1 = L.lbm_device_bytes(g.h)
        g.get_populations()
        g.step(5)
        got = g.get_populations().copy()
    # per listed cell: index, solid mask and two words of wall kinds
    assert b1 - b0 == 24 * listed_cells(flags, DIMS, Q)
    assert np.array_equal(got, full)


def test_kernels_per_step_reports_the_launches():
    flags = I.cavity_flags(12, 10, 9)
    cases = [("aa", L.F16, flags, 2), ("aa", L.F32, flags, 1), ("aa", L.F64, flags, 2), ("swap", L.F16, flags, 2),
             ("twopop", L.F16, flags, 1), ("esotwist", L.F16, flags, 1),
             ("aa", L.F16, np.ones(12 * 10 * 9, np.uint8), 1)]  # all solid: no listed cells
    for scheme, prec, fl, want in cases:
        with L.Lattice(19, 12, 10, 9, scheme, "BGK_W2", 1.3, fl, precision=prec) as g:
            assert L.lbm_kernels_per_step(g.h) == want, (scheme, prec)
            g.step(2)  # and the step still runs after the query built the list
