"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  The CUDA library never imports it, and it never imports the CUDA
library.  Arrays are numpy float64 in SoA order [Q][N] with the cell index
i = (x*ny + y)*nz + z (the index map of Section 2.5 of the paper).
"""
import ctypes
import os

import numpy as np

from . import build as _build

MODELS = {"BGK_W2": 0, "BGK_NW4": 1, "TRT": 2, "REG": 3, "RR": 4, "RM": 5, "HM": 6, "CM": 7, "CHM": 8, "K": 9}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.orc_lattice.argtypes = [ctypes.c_int, ip, dp, ip]
        L.orc_moment_basis.argtypes = [ctypes.c_int, ip, dp]
        L.orc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_model_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_collide.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_cumulants.argtypes = [ctypes.c_int, dp, dp]
        L.orc_step.argtypes = [ctypes.c_int] * 4 + [u8p, dp, ctypes.c_int, dp, dp, i64p, ctypes.c_int, dp, dp]
        L.orc_run.argtypes = [ctypes.c_int] * 4 + [u8p, dp, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, dp]
        L.orc_step_curved.argtypes = [ctypes.c_int] * 4 + [u8p, dp, ctypes.c_int, dp, dp, dp, ctypes.c_int, dp, dp]
        L.orc_macroscopic.argtypes = [ctypes.c_int, ctypes.c_int64, u8p, dp, dp, dp, dp]
        L.orc_conserved.argtypes = [ctypes.c_int, ctypes.c_int64, u8p, dp, dp, dp]
        L.orc_init_equilibrium_field.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, u8p, dp, dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def lattice(Q):
    """Velocities c[Q,3], weights t[Q], opposite index opp[Q]."""
    c = np.zeros((Q, 3), dtype=np.int32)
    t = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    rc = lib().orc_lattice(Q, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(t),
                           opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != Q:
        raise ValueError(f"unsupported lattice Q={Q}")
    return c.astype(np.int64), t, opp.astype(np.int64)


def moment_basis(Q):
    """Monomial exponents pqr[Q,3] and the exact inverse of the moment matrix (rows = populations)."""
    pqr = np.zeros((Q, 3), dtype=np.int32)
    Tinv = np.zeros((Q, Q))
    _check(lib().orc_moment_basis(Q, pqr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(Tinv)), "basis")
    return pqr.astype(np.int64), Tinv


def equilibrium(Q, kind, rho, u):
    feq = np.zeros(Q)
    _check(lib().orc_equilibrium(Q, kind, float(rho), _dp(_c64(u)), _dp(feq)), "equilibrium")
    return feq


def model_equilibrium(Q, model, rho, u):
    feq = np.zeros(Q)
    _check(lib().orc_model_equilibrium(Q, MODELS[model], float(rho), _dp(_c64(u)), _dp(feq)), "equilibrium")
    return feq


def params(omega, omega_bulk=None, omega_high=1.0, trt_lambda=0.25):
    return np.array([omega, omega if omega_bulk is None else omega_bulk, omega_high, trt_lambda], dtype=np.float64)


def collide(Q, model, prm, f):
    f = _c64(f)
    out = np.zeros(Q)
    _check(lib().orc_collide(Q, MODELS[model], _dp(_c64(prm)), _dp(f), _dp(out)), "collide")
    return out


def cumulants(Q, f):
    out = np.zeros(Q)
    _check(lib().orc_cumulants(Q, _dp(_c64(f)), _dp(out)), "cumulants")
    return out


def wall_table(wall_velocities=None):
    """8x3 table indexed by flag value; flag 1 is the resting wall."""
    W = np.zeros((8, 3))
    for fl, v in (wall_velocities or {}).items():
        W[int(fl)] = v
    return W


class Lattice:
    """A periodic box of nx*ny*nz cells with a flag field, stepped by the oracle."""

    def __init__(self, Q, nx, ny, nz, flags, model, prm, wall_velocities=None):
        self.Q, self.nx, self.ny, self.nz = Q, nx, ny, nz
        self.N = nx * ny * nz
        self.flags = np.ascontiguousarray(flags, dtype=np.uint8).reshape(self.N)
        self.model = model
        self.prm = _c64(prm)
        self.wall_u = _c64(wall_table(wall_velocities))
        self.f = np.zeros((Q, self.N))
        # walls at a fraction of their links: [Q][N] (see orc_step_curved), or None (halfway)
        self.qfrac = None

    def init_equilibrium(self, rho=None, u=None):
        """f = the model's own equilibrium of per-cell rho[N], u[3][N] (None: rho = 1, u = 0);
        solid cells get 0."""
        rp = up = None
        if rho is not None:
            rho = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, dtype=np.float64), (self.N,)))
            rp = _dp(rho)
        if u is not None:
            u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3, self.N))
            up = _dp(u)
        _check(lib().orc_init_equilibrium_field(self.Q, MODELS[self.model], self.N,
                                                self.flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                                rp, up, _dp(self.f)), "init_equilibrium")

    def step(self, n=1, force=None, perm=None, nthreads=1):
        L = lib()
        fl = self.flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        fp = None if force is None else _dp(_c64(force))
        if self.qfrac is not None:
            if perm is not None:
                raise ValueError("traversal permutations are not combined with curved walls")
            q = np.ascontiguousarray(np.asarray(self.qfrac, dtype=np.float64).reshape(self.Q, self.N))
            for _ in range(n):
                new = np.zeros_like(self.f)
                _check(L.orc_step_curved(self.Q, self.nx, self.ny, self.nz, fl, _dp(self.wall_u),
                                         MODELS[self.model], _dp(self.prm), fp, _dp(q), nthreads, _dp(self.f),
                                         _dp(new)), "step_curved")
                self.f = new
            return
        if perm is None and n > 1:
            _check(L.orc_run(self.Q, self.nx, self.ny, self.nz, fl, _dp(self.wall_u), MODELS[self.model],
                             _dp(self.prm), fp, n, nthreads, _dp(self.f)), "run")
            return
        pp = None
        if perm is not None:
            perm = np.ascontiguousarray(perm, dtype=np.int64)
            pp = perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        for _ in range(n):
            new = np.zeros_like(self.f)
            _check(L.orc_step(self.Q, self.nx, self.ny, self.nz, fl, _dp(self.wall_u), MODELS[self.model],
                              _dp(self.prm), fp, pp, nthreads, _dp(self.f), _dp(new)), "step")
            self.f = new

    def macroscopic(self):
        rho = np.zeros(self.N)
        u = np.zeros((3, self.N))
        _check(lib().orc_macroscopic(self.Q, self.N, self.flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                     _dp(self.wall_u), _dp(self.f), _dp(rho), _dp(u)), "macroscopic")
        return rho, u

    def conserved(self):
        m = ctypes.c_double()
        e = ctypes.c_double()
        _check(lib().orc_conserved(self.Q, self.N, self.flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                   _dp(self.f), ctypes.byref(m), ctypes.byref(e)), "conserved")
        return m.value, e.value


def library_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblbm_oracle.so")
