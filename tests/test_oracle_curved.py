"""Pins of the oracle's walls at a fraction of their links (orc_step_curved), the extension of
link-wise bounce-back to curved walls that the paper points to (Section 1: link-based and
entirely local), read as the linear interpolation of Bouzidi, Firdaouss & Lallemand (2001) with
the population that streamed into the cell standing for the neighbour's post-collision value.

* q = 1/2 on every link is the halfway bounce-back of Section 2.1: bit for bit the plain step,
  on random obstacles with moving walls, for several collision models and both lattices.
* Couette flow between a resting and a moving wall placed off the lattice (q from 0.1 to 0.95,
  on both sides of 1/2): the steady profile is the straight line through the true wall
  positions, to round-off, for BGK-W2 and TRT at two viscosities (a linear interpolation of a
  linear profile is exact).  A wrong population, index or wall-term weight in either branch
  breaks it.
* Poiseuille flow driven by a body force between off-lattice walls: second-order convergence
  (error ratio ~4 per doubling of the channel) against the parabola through the true walls.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_11751_b300 import inputs as I


def _wall_fractions(Q, ny, q_bottom, q_top):
    """q for the links of the first and last fluid rows of a 1 x ny x 1 channel crossing the
    walls at y = 0 and y = ny - 1 (every such link meets the plane at the same fraction)."""
    c, _, _ = O.lattice(Q)
    q = np.full((Q, ny), 0.5)
    for k in range(Q):
        if c[k][1] == -1:
            q[k, 1] = q_bottom
        if c[k][1] == 1:
            q[k, ny - 2] = q_top
    return q


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", ["BGK_W2", "TRT", "RR", "K"])
def test_half_link_walls_are_the_plain_bounce_back(Q, model):
    dims = (7, 6, 9)
    flags = I.random_obstacle_flags(*dims, 0.2, seed=41)
    walls = {2: (0.03, -0.01, 0.02), 3: (-0.02, 0.01, 0.0)}
    rho, u = I.smooth_random_fields(*dims, amp=0.03, seed=42)
    a = O.Lattice(Q, *dims, flags, model, O.params(1.4, 1.1, 0.9, 0.3), walls)
    a.init_equilibrium(rho, u)
    a.f *= I.noise(a.f.shape, 0.05, seed=43)
    a.f[:, flags != 0] = 0.0
    b = O.Lattice(Q, *dims, flags, model, O.params(1.4, 1.1, 0.9, 0.3), walls)
    b.f = a.f.copy()
    b.qfrac = np.full((Q, a.N), 0.5)
    a.step(3)
    b.step(3)
    assert np.array_equal(a.f, b.f)


def _couette(Q, model, q_b, q_t, omega, ny_fluid=8, U=0.01, steps=20000):
    ny = ny_fluid + 2
    flags = np.zeros(ny, np.uint8)
    flags[0], flags[-1] = 1, 2
    lat = O.Lattice(Q, 1, ny, 1, flags, model, O.params(omega), {2: (U, 0.0, 0.0)})
    lat.init_equilibrium()
    lat.qfrac = _wall_fractions(Q, ny, q_b, q_t)
    lat.step(steps)
    _, u = lat.macroscopic()
    y = np.arange(ny, dtype=float)
    yb, yt = 1 - q_b, (ny - 2) + q_t
    exact = U * (y - yb) / (yt - yb)
    fluid = flags == 0
    return np.max(np.abs(u[0][fluid] - exact[fluid])) / U, np.max(np.abs(u[1:, fluid]))


@pytest.mark.parametrize("model", ["BGK_W2", "TRT"])
@pytest.mark.parametrize("q_b,q_t", [(0.25, 0.7), (0.8, 0.3), (0.1, 0.95), (0.5, 0.5)])
@pytest.mark.parametrize("omega", [1.0, 1.6])
def test_couette_between_off_lattice_walls_is_exact(model, q_b, q_t, omega):
    err, cross = _couette(19, model, q_b, q_t, omega)
    assert err <= 1e-10, err
    assert cross <= 1e-14


def _poiseuille(q_b, q_t, omega, ny_fluid, g=1e-6):
    ny = ny_fluid + 2
    flags = np.zeros(ny, np.uint8)
    flags[0] = flags[-1] = 1
    lat = O.Lattice(19, 1, ny, 1, flags, "BGK_W2", O.params(omega))
    lat.init_equilibrium()
    lat.qfrac = _wall_fractions(19, ny, q_b, q_t)
    nu = (1.0 / omega - 0.5) / 3.0
    H = ny_fluid - 1 + q_b + q_t
    lat.step(int(8 * H * H / nu) + 2000, force=[g, 0.0, 0.0])
    _, u = lat.macroscopic()
    y = np.arange(ny, dtype=float)
    yb, yt = 1 - q_b, (ny - 2) + q_t
    exact = g / (2.0 * nu) * (y - yb) * (yt - y)
    ux = u[0] + 0.5 * g  # the force is added after collision: half a step of it in the velocity
    fluid = flags == 0
    return np.sqrt(np.sum((ux[fluid] - exact[fluid]) ** 2) / np.sum(exact[fluid] ** 2))


@pytest.mark.parametrize("q_b,q_t", [(0.3, 0.7), (0.8, 0.25)])
def test_poiseuille_between_off_lattice_walls_converges_at_second_order(q_b, q_t):
    e1, e2 = _poiseuille(q_b, q_t, 1.2, 6), _poiseuille(q_b, q_t, 1.2, 12)
    assert e1 < 0.05
    assert 3.5 <= e1 / e2 <= 4.5, (e1, e2)
