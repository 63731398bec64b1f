"""Pins of the oracle's full stream-and-collide iteration against closed forms.

* Couette flow between bounce-back walls (one moving): linear profile with the walls
  half-way, exact to round-off (momentum-exchange term of Section 2.1).
* Body-force driven Poiseuille flow with TRT at Lambda = 3/16: exact parabola with the walls
  half-way (a published TRT property); BGK within the known viscosity-dependent slip error.
* Taylor-Green vortex: amplitude decays as exp(-2 nu k^2 t), nu = (1/omega - 1/2) c_s^2
  (Section 2.6), with second-order convergence of the decay rate.
* Order independence of the traversal (the thread-safety criterion of Section 2.3).
* Mass conservation of the closed lid-driven cavity with a full-plane tangential lid.
* Brute-force streaming on tiny lattices: each destination population pulled by hand.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_11751_b300 import inputs as I


def omega_of(nu):
    return 1.0 / (3.0 * nu + 0.5)


@pytest.mark.parametrize("model", ["BGK_W2", "TRT", "RR", "K", "CM", "REG"])
def test_couette_exact(model):
    nx, ny, nz, U = 1, 10, 1, 0.01
    for omega in (0.7, 1.6):
        lat = O.Lattice(19, nx, ny, nz, I.channel_flags(nx, ny, nz, moving_top=True), model, O.params(omega),
                        {I.LID: (U, 0, 0)})
        lat.init_equilibrium(1.0, np.zeros((3, nx * ny * nz)))
        lat.step(12000)
        _, u = lat.macroscopic()
        y = np.arange(1, ny - 1)
        ux = u[0].reshape(nx, ny, nz)[0, 1:-1, 0]
        assert np.abs(ux - U * (y - 0.5) / (ny - 2)).max() < 1e-9 * U


def _poiseuille(model, omega, lam):
    nx, ny, nz, g = 1, 10, 1, 1e-6
    lat = O.Lattice(19, nx, ny, nz, I.channel_flags(nx, ny, nz), model, O.params(omega, trt_lambda=lam))
    lat.init_equilibrium(1.0, np.zeros((3, nx * ny * nz)))
    lat.step(25000, force=np.array([g, 0.0, 0.0]))
    rho, u = lat.macroscopic()
    y = np.arange(1, ny - 1)
    nu = (1.0 / omega - 0.5) / 3.0
    exact = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    ux = u[0].reshape(nx, ny, nz)[0, 1:-1, 0] + 0.5 * g / rho.reshape(nx, ny, nz)[0, 1:-1, 0]
    return np.abs(ux - exact).max() / exact.max()


@pytest.mark.parametrize("omega", [0.8, 1.3, 1.7])
def test_poiseuille_trt_magic_exact(omega):
    assert _poiseuille("TRT", omega, 3.0 / 16.0) < 1e-9


def test_poiseuille_bgk_slip_error():
    err = _poiseuille("BGK_W2", 1.3, 0.25)
    assert 1e-4 < err < 5e-2  # second-order wall-slip error, viscosity dependent


def _tg_rate_error(model, N, Q=19, nu=0.05, u0=1e-3):
    nx, ny, nz = N, N, 1
    rho, u = I.taylor_green_fields(nx, ny, nz, u0)
    lat = O.Lattice(Q, nx, ny, nz, I.periodic_flags(nx, ny, nz), model, O.params(omega_of(nu)))
    lat.init_equilibrium(rho, u)
    k = 2 * np.pi / N
    T = int(0.5 / (2 * nu * k * k))
    mode = I.taylor_green_mode(nx, ny, nz)
    lat.step(T // 5)
    ts, amps = [], []
    for i in range(5):
        _, uu = lat.macroscopic()
        ts.append(T // 5 * (i + 1))
        amps.append((uu[0] * mode).sum() / (mode * mode).sum())
        lat.step(T // 5)
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    return abs(rate - 2 * nu * k * k) / (2 * nu * k * k)


@pytest.mark.parametrize("model", ["BGK_W2", "TRT", "REG"])
def test_taylor_green_second_order(model):
    e32, e64 = _tg_rate_error(model, 32), _tg_rate_error(model, 64)
    assert e64 < 1e-3
    assert 3.0 < e32 / e64 < 5.5


@pytest.mark.parametrize("Q,model", [(19, "BGK_NW4"), (19, "RR"), (19, "RM"), (19, "HM"), (19, "CM"), (19, "CHM"),
                                     (19, "K"), (27, "BGK_W2"), (27, "K"), (27, "RR")])
def test_taylor_green_viscosity(Q, model):
    assert _tg_rate_error(model, 32, Q=Q) < 2e-3


@pytest.mark.parametrize("Q,model", [(19, "BGK_W2"), (19, "K"), (27, "TRT"), (27, "CHM")])
def test_order_independence(Q, model):
    nx, ny, nz = 5, 4, 6
    N = nx * ny * nz
    flags = I.random_obstacle_flags(nx, ny, nz, 0.15, seed=3)
    rho, u = I.smooth_random_fields(nx, ny, nz, seed=4)
    prm = O.params(1.5, 1.2, 0.9)
    runs = []
    for perm in (None, np.arange(N)[::-1].copy(), np.random.default_rng(6).permutation(N)):
        lat = O.Lattice(Q, nx, ny, nz, flags, model, prm, {2: (0.02, -0.01, 0.0), 3: (0.0, 0.01, 0.03)})
        lat.init_equilibrium(rho, u)
        lat.f *= I.noise(lat.f.shape, 0.05, seed=7)
        lat.f[:, flags != 0] = 0.0
        lat.step(3, perm=perm)
        runs.append(lat.f.copy())
    assert np.array_equal(runs[0], runs[1])
    assert np.array_equal(runs[0], runs[2])


@pytest.mark.parametrize("Q,model", [(19, "BGK_W2"), (27, "K"), (19, "RR")])
def test_cavity_mass_conservation(Q, model):
    n = 12
    flags = I.cavity_flags(n, n, n)
    lat = O.Lattice(Q, n, n, n, flags, model, O.params(omega_of(I.cavity_nu(0.02, n, 100.0))),
                    {I.LID: (0.02, 0, 0)})
    lat.init_equilibrium(1.0, np.zeros((3, n ** 3)))
    m0, _ = lat.conserved()
    lat.step(100)
    m1, e1 = lat.conserved()
    assert abs(m1 - m0) <= 1e-12 * m0
    assert e1 > 0  # the lid has set the fluid in motion


def _pull_by_hand(Q, nx, ny, nz, flags, wall_u, f):
    """Identity collision: each destination population taken from where it comes from."""
    c, t, opp = O.lattice(Q)
    N = nx * ny * nz
    out = np.zeros_like(f)
    for x in range(nx):
        for y in range(ny):
            for z in range(nz):
                i = (x * ny + y) * nz + z
                if flags[i]:
                    continue
                for k in range(Q):
                    xs, ys, zs = (x - c[k, 0]) % nx, (y - c[k, 1]) % ny, (z - c[k, 2]) % nz
                    src = (xs * ny + ys) * nz + zs
                    if flags[src] == 0:
                        out[k, i] = f[k, src]
                    else:  # population k arrives by reflection of opp[k] leaving i towards src
                        kb = opp[k]
                        out[k, i] = f[kb, i] - 6 * t[kb] * (c[kb] @ wall_u[flags[src]])
    return out


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("dims", [(3, 3, 3), (4, 5, 3)])
def test_streaming_brute_force(Q, dims):
    nx, ny, nz = dims
    N = nx * ny * nz
    c, t, _ = O.lattice(Q)
    flags = np.zeros(N, np.uint8)
    flags[(1 * ny + 1) * nz + 1] = 1
    flags[(2 * ny + 0) * nz + 2] = 2
    wall = {2: (0.03, -0.02, 0.01)}
    lat = O.Lattice(Q, nx, ny, nz, flags, "BGK_W2", O.params(0.0), wall)
    f = np.where(flags[None, :] == 0, t[:, None] * I.noise((Q, N), 0.2, seed=8), 0.0)
    lat.f = f.copy()
    lat.step(1)
    assert np.array_equal(lat.f, _pull_by_hand(Q, nx, ny, nz, flags, lat.wall_u, f))


@pytest.mark.parametrize("Q,model", [(19, "BGK_W2"), (27, "BGK_NW4"), (19, "K")])
def test_conserved_sums_of_known_fields(Q, model):
    """The oracle's FP64 sums against their definitions (fluid cells only):
    mass = sum rho and energy = sum rho |u|^2 / 2.  A uniform flow of known rho and u gives
    N_fluid rho and N_fluid rho |u|^2 / 2; a smooth random field gives the same sums formed
    here in numpy from the (rho, u) it was built from, since every model's equilibrium
    reproduces its own rho and u."""
    nx, ny, nz = 6, 5, 4
    N = nx * ny * nz
    flags = np.zeros(N, np.uint8)
    flags[[3, 17, 60, 99]] = [1, 2, 1, 3]
    fluid = flags == 0
    rho0, u0 = 1.03, np.array([0.03, -0.02, 0.011])
    lat = O.Lattice(Q, nx, ny, nz, flags, model, O.params(1.2))
    lat.init_equilibrium(np.full(N, rho0), np.repeat(u0[:, None], N, axis=1))
    m, e = lat.conserved()
    nf = int(fluid.sum())
    assert abs(m - nf * rho0) <= 1e-14 * nf
    assert abs(e - nf * 0.5 * rho0 * float(u0 @ u0)) <= 1e-12 * nf * 0.5 * rho0 * float(u0 @ u0)
    g = np.random.default_rng(31)
    rho = 1.0 + 0.02 * g.standard_normal(N)
    u = 0.04 * g.standard_normal((3, N))
    lat.init_equilibrium(rho, u)
    m, e = lat.conserved()
    want_m = rho[fluid].sum()
    want_e = (0.5 * rho * (u * u).sum(0))[fluid].sum()
    assert abs(m - want_m) <= 1e-13 * want_m
    assert abs(e - want_e) <= 1e-12 * want_e
