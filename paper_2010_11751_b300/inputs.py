"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds only workload geometry and analytic initial fields: flag
fields, the Taylor-Green velocity/density field, random perturbations, the
batch of uneven cavities and the serving request trace.  It contains none of
the lattice Boltzmann arithmetic (no equilibria, no collision, no streaming),
so that the CUDA library and the CPU oracle can both consume its output
without sharing method code.

Flag values: 0 fluid, 1 resting bounce-back wall, 2..7 moving walls whose
velocities are set separately.  Cell index i = (x*ny + y)*nz + z.
"""
from __future__ import annotations

import numpy as np

SEED = 20101175
FLUID, WALL, LID = 0, 1, 2


def rng(seed: int | None = None) -> np.random.Generator:
    return np.random.default_rng(SEED if seed is None else seed)


def periodic_flags(nx: int, ny: int, nz: int) -> np.ndarray:
    return np.zeros(nx * ny * nz, dtype=np.uint8)


def cavity_flags(nx: int, ny: int, nz: int) -> np.ndarray:
    """Lid-driven cavity: one wall layer on every face; the whole plane z = nz-1
    (edges and corners included) carries the lid flag."""
    f = np.zeros((nx, ny, nz), dtype=np.uint8)
    f[0, :, :] = WALL
    f[-1, :, :] = WALL
    f[:, 0, :] = WALL
    f[:, -1, :] = WALL
    f[:, :, 0] = WALL
    f[:, :, -1] = LID
    return f.reshape(-1)


def channel_flags(nx: int, ny: int, nz: int, moving_top: bool = False) -> np.ndarray:
    """Walls on the planes y = 0 and y = ny-1, periodic in x and z."""
    f = np.zeros((nx, ny, nz), dtype=np.uint8)
    f[:, 0, :] = WALL
    f[:, -1, :] = LID if moving_top else WALL
    return f.reshape(-1)


def random_obstacle_flags(nx: int, ny: int, nz: int, solid_fraction: float = 0.1, seed: int | None = None,
                          wall_kinds=(WALL, LID, 3)) -> np.ndarray:
    """Periodic box with randomly placed solid cells of several wall kinds."""
    g = rng(seed)
    solid = g.random(nx * ny * nz) < solid_fraction
    kinds = g.choice(np.asarray(wall_kinds, dtype=np.uint8), size=nx * ny * nz)
    return np.where(solid, kinds, FLUID).astype(np.uint8)


def taylor_green_fields(nx: int, ny: int, nz: int, u0: float, kx: float | None = None, ky: float | None = None):
    """Analytic z-invariant Taylor-Green vortex: returns rho[N], u[3][N]."""
    kx = 2.0 * np.pi / nx if kx is None else kx
    ky = 2.0 * np.pi / ny if ky is None else ky
    x, y, _ = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ux = u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = -u0 * np.sin(kx * x) * np.cos(ky * y)
    rho = 1.0 - 0.75 * u0 * u0 * (np.cos(2 * kx * x) + np.cos(2 * ky * y))
    u = np.stack([ux.ravel(), uy.ravel(), np.zeros(nx * ny * nz)])
    return rho.ravel().astype(np.float64), u.astype(np.float64)


def taylor_green_fields_torch(nx: int, ny: int, nz: int, u0: float, device: str = "cuda"):
    """The same analytic Taylor-Green field as taylor_green_fields, built with torch on a device
    (contiguous float64 rho[N] and u[3*N])."""
    import torch

    kx, ky = 2.0 * np.pi / nx, 2.0 * np.pi / ny
    x = torch.arange(nx, dtype=torch.float64, device=device).view(nx, 1, 1).expand(nx, ny, nz)
    y = torch.arange(ny, dtype=torch.float64, device=device).view(1, ny, 1).expand(nx, ny, nz)
    ux = u0 * torch.cos(kx * x) * torch.sin(ky * y)
    uy = -u0 * torch.sin(kx * x) * torch.cos(ky * y)
    rho = 1.0 - 0.75 * u0 * u0 * (torch.cos(2 * kx * x) + torch.cos(2 * ky * y))
    u = torch.stack([ux.reshape(-1), uy.reshape(-1), torch.zeros(nx * ny * nz, dtype=torch.float64, device=device)])
    return rho.reshape(-1).contiguous(), u.reshape(-1).contiguous()


def taylor_green_mode(nx: int, ny: int, nz: int, kx: float | None = None, ky: float | None = None) -> np.ndarray:
    """The spatial shape cos(kx x) sin(ky y) of the x-velocity, for amplitude fits."""
    kx = 2.0 * np.pi / nx if kx is None else kx
    ky = 2.0 * np.pi / ny if ky is None else ky
    x, y, _ = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return (np.cos(kx * x) * np.sin(ky * y)).ravel()


def smooth_random_fields(nx: int, ny: int, nz: int, amp: float = 0.03, seed: int | None = None):
    """A random smooth (few Fourier modes) density/velocity field for parity tests."""
    g = rng(seed)
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    rho = np.ones((nx, ny, nz))
    u = np.zeros((3, nx, ny, nz))
    for _ in range(3):
        kx, ky, kz = (2 * np.pi * g.integers(0, 3, 3) / np.array([nx, ny, nz]))
        ph = g.random(4) * 2 * np.pi
        rho += 0.3 * amp * np.sin(kx * x + ky * y + kz * z + ph[0])
        for d in range(3):
            u[d] += amp * g.standard_normal() * np.sin(kx * x + ky * y + kz * z + ph[d + 1])
    return rho.ravel(), u.reshape(3, -1)


def noise(shape, amp: float, seed: int | None = None) -> np.ndarray:
    """Multiplicative perturbation factors 1 + amp * U(-1, 1)."""
    return 1.0 + amp * (2.0 * rng(seed).random(shape) - 1.0)


def cavity_nu(u_lid: float, n: int, reynolds: float) -> float:
    """Kinematic viscosity of a cavity workload: nu = u * N / Re."""
    return u_lid * n / reynolds


def batch_cavities(count: int = 256, lo: int = 16, hi: int = 96, re_lo: float = 100.0, re_hi: float = 1000.0,
                   seed: int | None = None):
    """Uneven independent cavities: per-lattice (nx, ny, nz, Re), sides uniform in [lo, hi]."""
    g = rng(seed)
    dims = g.integers(lo, hi + 1, size=(count, 3))
    re = g.uniform(re_lo, re_hi, size=count)
    return [(int(a), int(b), int(c), float(r)) for (a, b, c), r in zip(dims, re)]


def serving_trace(count: int = 500, rate_hz: float = 50.0, side_lo: int = 32, side_hi: int = 192,
                  steps_lo: int = 100, steps_hi: int = 2000, seed: int | None = None):
    """Poisson request stream: arrival time, lattice, workload, collision, precision, side, steps."""
    g = rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate_hz, size=count))
    out = []
    for i in range(count):
        out.append({
            "id": i,
            "arrival_s": float(t[i]),
            "lattice": int(g.choice([19, 27])),
            "workload": str(g.choice(["cavity", "taylor_green"])),
            "collision": str(g.choice(["BGK_W2", "K"])),
            "precision": str(g.choice(["f32", "f64"])),
            "side": int(g.integers(side_lo, side_hi + 1)),
            "steps": int(g.integers(steps_lo, steps_hi + 1)),
        })
    return out
