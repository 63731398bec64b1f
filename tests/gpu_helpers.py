"""Shared set-up of the GPU parity tests: the same seeded inputs go to the oracle and to the
CUDA library; expected values always come from the oracle."""
import numpy as np

from oracle import oracle as O
from paper_2010_11751_b300 import inputs as I
from paper_2010_11751_b300 import lbm as L

WALLS = {2: (0.03, -0.01, 0.02), 3: (-0.02, 0.01, 0.0)}
MODELS = list(O.MODELS)
SCHEMES = {"twopop": L.TWOPOP, "swap": L.SWAP, "aa": L.AA, "esotwist": L.ESOTWIST}

# relative per-population tolerance of the FP64 path against the FP64 oracle
RTOL_F64 = 1e-12


def prm(omega=1.55, omega_bulk=1.2, omega_high=0.9, trt_lambda=0.3):
    return dict(omega=omega, omega_bulk=omega_bulk, omega_high=omega_high, trt_lambda=trt_lambda)


def case(Q, dims, seed=1, solid=0.12, model="BGK_W2", amp=0.04):
    """Random obstacles of three wall kinds, smooth random (rho, u), the model's equilibrium
    perturbed by multiplicative noise (so every moment is out of equilibrium)."""
    nx, ny, nz = dims
    flags = I.random_obstacle_flags(nx, ny, nz, solid, seed=seed)
    rho, u = I.smooth_random_fields(nx, ny, nz, amp=amp, seed=seed + 1)
    ref = O.Lattice(Q, nx, ny, nz, flags, model, O.params(1.0), WALLS)
    ref.init_equilibrium(rho, u)
    f0 = ref.f * I.noise(ref.f.shape, 0.05, seed=seed + 2)
    f0[:, flags != 0] = 0.0
    return flags, f0


def oracle_run(Q, dims, flags, model, p, f0, steps):
    nx, ny, nz = dims
    lat = O.Lattice(Q, nx, ny, nz, flags, model,
                    O.params(p["omega"], p["omega_bulk"], p["omega_high"], p["trt_lambda"]), WALLS)
    lat.f = f0.copy()
    lat.step(steps)
    return lat


def gpu_lattice(Q, dims, flags, model, p, scheme="twopop", layout=L.SOA, precision=L.F64):
    nx, ny, nz = dims
    return L.Lattice(Q, nx, ny, nz, scheme, model, p["omega"], flags, layout=layout, precision=precision,
                     wall_velocities=WALLS, omega_bulk=p["omega_bulk"], omega_high=p["omega_high"],
                     trt_lambda=p["trt_lambda"])


def gpu_run(Q, dims, flags, model, p, f0, steps, scheme="twopop", layout=L.SOA, precision=L.F64):
    with gpu_lattice(Q, dims, flags, model, p, scheme, layout, precision) as g:
        g.set_populations(f0)
        g.step(steps)
        return g.get_populations().copy()


def rel_err(got, ref, flags):
    fluid = flags == 0
    return np.max(np.abs(got[:, fluid] - ref[:, fluid]) / np.abs(ref[:, fluid]))
