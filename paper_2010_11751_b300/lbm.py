"""Thin ctypes binding of liblbm.so (the C ABI of include/lbm.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Module-level functions carry the C names (``lbm_create``,
``lbm_step``, ...) and raise ``LBMError`` on a non-zero status.  Arrays may be
numpy arrays (host) or torch tensors (host or CUDA); they must be contiguous
float64 (populations, fields) or uint8 (flags).  There is no fallback: if the
library is missing, loading raises.
"""
from __future__ import annotations

import contextlib
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY = os.path.join(_HERE, "liblbm.so")
# the bounds-checked build of the same sources (three collision models; see build.py)
LIBRARY_DEBUG = os.path.join(_HERE, "liblbm_debug.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_STATE, ERR_DIVERGED, ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
D3Q19, D3Q27 = 19, 27
TWOPOP, SWAP, AA, ESOTWIST = 0, 1, 2, 3
SCHEMES = {"twopop": TWOPOP, "swap": SWAP, "aa": AA, "esotwist": ESOTWIST}
BGK_W2, BGK_NW4, TRT, REG, RR, RM, HM, CM, CHM, K, BGK_W2_EDU, BGK_W2_LOOP = range(12)
MODELS = {"BGK_W2": BGK_W2, "BGK_NW4": BGK_NW4, "TRT": TRT, "REG": REG, "RR": RR, "RM": RM, "HM": HM, "CM": CM,
          "CHM": CHM, "K": K, "BGK_W2_EDU": BGK_W2_EDU, "BGK_W2_LOOP": BGK_W2_LOOP}
SOA, AOS = 0, 1
F64, F32, F16 = 0, 1, 2
PRECISIONS = {"f64": F64, "f32": F32, "f16": F16}
PARAM_OMEGA, PARAM_OMEGA_BULK, PARAM_OMEGA_HIGH, PARAM_TRT_LAMBDA, PARAM_WAIT_CYCLES, PARAM_FX_RANGE = 0, 1, 2, 3, 4, 5
FX_AUTO, FX_NARROW, FX_WIDE = 0, 1, 2


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


_lib = None
_loaded = {}


def lib() -> ctypes.CDLL:
    """The library every call of this module goes to: liblbm.so, or liblbm_debug.so inside a
    ``debug_library()`` block (raises if it has not been built)."""
    global _lib
    if _lib is None:
        _lib = _load(LIBRARY)
    return _lib


@contextlib.contextmanager
def debug_library():
    """Route every call of this module to liblbm_debug.so, the bounds-checked build, for the
    duration of the block.  Handles made inside belong to that library and must be destroyed
    inside the block."""
    global _lib
    prev = lib()
    _lib = _load(LIBRARY_DEBUG)
    try:
        yield _lib
    finally:
        _lib = prev


def _load(path) -> ctypes.CDLL:
    if path in _loaded:
        return _loaded[path]
    if not os.path.exists(path):
        raise LBMError(ERR_STATE, f"{path} is missing; build it with paper_2010_11751_b300.build.build()")
    L = ctypes.CDLL(path)
    vp, dp, u8p = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
    i, d = ctypes.c_int, ctypes.c_double
    sigs = {
        "lbm_create": [ctypes.POINTER(vp), i, i, i, i, i, i, d, u8p],
        "lbm_set_layout": [vp, i],
        "lbm_set_precision": [vp, i],
        "lbm_set_wall_velocity": [vp, i, d, d, d],
        "lbm_set_link_fractions": [vp, dp],
        "lbm_set_param": [vp, i, d],
        "lbm_set_stream": [vp, vp],
        "lbm_init_equilibrium": [vp, dp, dp],
        "lbm_step": [vp, i],
        "lbm_macroscopic": [vp, dp, dp],
        "lbm_get_populations": [vp, dp],
        "lbm_set_populations": [vp, dp],
        "lbm_reduce": [vp, ctypes.POINTER(d), ctypes.POINTER(d)],
        "lbm_steps_done": [vp, ctypes.POINTER(ctypes.c_longlong)],
        "lbm_device_bytes": [vp, ctypes.POINTER(ctypes.c_size_t)],
        "lbm_bytes_per_cell_update": [vp, ctypes.POINTER(d)],
        "lbm_kernels_per_step": [vp, ctypes.POINTER(i)],
        "lbm_step_sums": [vp, i, ctypes.POINTER(d), ctypes.POINTER(d)],
        "lbm_step_sums_async": [vp, i, dp],
        "lbm_destroy": [vp],
        "lbm_supported": [i, i, i, i, i],
        "lbm_conserved_sums_static": [i, i, dp, u8p, dp, vp],
        "lbm_batch_create": [ctypes.POINTER(vp)],
        "lbm_batch_add": [vp, vp],
        "lbm_batch_remove": [vp, vp],
        "lbm_batch_set_launch": [vp, i, i],
        "lbm_batch_autotune": [vp, ctypes.POINTER(i), ctypes.POINTER(i)],
        "lbm_batch_step": [vp, i, i],
        "lbm_batch_set_stream": [vp, vp],
        "lbm_batch_sync": [vp],
        "lbm_batch_size": [vp, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)],
        "lbm_batch_destroy": [vp],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.lbm_debug_check.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong)]
    L.lbm_debug_check.restype = ctypes.c_int
    L.lbm_last_error.argtypes = []
    L.lbm_last_error.restype = ctypes.c_char_p
    _loaded[path] = L
    return L


def _check(rc):
    if rc != OK:
        raise LBMError(rc, lib().lbm_last_error().decode())
    return rc


def ptr(a):
    """Raw address of a numpy array / torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported buffer type {type(a)}")


# ---- C names, marshalling only ----
def lbm_create(lattice, nx, ny, nz, scheme, collision, omega, flags):
    h = ctypes.c_void_p()
    fl = np.ascontiguousarray(flags, dtype=np.uint8)
    _check(lib().lbm_create(ctypes.byref(h), lattice, nx, ny, nz, scheme, collision, omega, fl.ctypes.data))
    return h


def lbm_set_layout(h, layout):
    return _check(lib().lbm_set_layout(h, layout))


def lbm_set_precision(h, precision):
    return _check(lib().lbm_set_precision(h, precision))


def lbm_set_wall_velocity(h, flag, ux, uy, uz):
    return _check(lib().lbm_set_wall_velocity(h, flag, ux, uy, uz))


def lbm_set_link_fractions(h, q):
    """q: None, or host FP64 [Q][N] wall fractions of the links that meet a wall."""
    if q is not None:
        q = np.ascontiguousarray(q, dtype=np.float64)
    return _check(lib().lbm_set_link_fractions(h, ptr(q)))


def lbm_set_param(h, key, value):
    return _check(lib().lbm_set_param(h, key, value))


def lbm_set_stream(h, stream):
    return _check(lib().lbm_set_stream(h, stream))


def lbm_init_equilibrium(h, rho=None, u=None):
    return _check(lib().lbm_init_equilibrium(h, ptr(rho), ptr(u)))


def lbm_step(h, n):
    return _check(lib().lbm_step(h, n))


def lbm_macroscopic(h, rho, u):
    return _check(lib().lbm_macroscopic(h, ptr(rho), ptr(u)))


def lbm_get_populations(h, f):
    return _check(lib().lbm_get_populations(h, ptr(f)))


def lbm_set_populations(h, f):
    return _check(lib().lbm_set_populations(h, ptr(f)))


def lbm_reduce(h):
    m, e = ctypes.c_double(), ctypes.c_double()
    _check(lib().lbm_reduce(h, ctypes.byref(m), ctypes.byref(e)))
    return m.value, e.value


def lbm_steps_done(h):
    v = ctypes.c_longlong()
    _check(lib().lbm_steps_done(h, ctypes.byref(v)))
    return v.value


def lbm_device_bytes(h):
    v = ctypes.c_size_t()
    _check(lib().lbm_device_bytes(h, ctypes.byref(v)))
    return v.value


def lbm_bytes_per_cell_update(h):
    v = ctypes.c_double()
    _check(lib().lbm_bytes_per_cell_update(h, ctypes.byref(v)))
    return v.value


def lbm_step_sums_async(h, n, out):
    """Enqueue lbm_step_sums' work; out (2 doubles, a device tensor or pinned host tensor)
    receives {mass, energy} when the stream gets there."""
    return _check(lib().lbm_step_sums_async(h, n, ptr(out)))


# kinds of the fault word of lbm_debug_check (bits 56..63)
DEBUG_FAULTS = {1: "population load", 2: "population store", 3: "cell index", 4: "flag read",
                5: "solid-neighbour mask read", 6: "staged population copy", 7: "staged flag copy",
                8: "staged run read", 9: "link-fraction row", 10: "padding canary"}


def lbm_debug_check(h):
    """First bounds fault the handle's kernels recorded since the last check (0: none), and the
    padding canaries; only liblbm_debug.so has the checks (liblbm.so raises ERR_UNSUPPORTED)."""
    w = ctypes.c_ulonglong()
    _check(lib().lbm_debug_check(h, ctypes.byref(w)))
    return w.value


def lbm_step_sums(h, n):
    m, e = ctypes.c_double(), ctypes.c_double()
    _check(lib().lbm_step_sums(h, n, ctypes.byref(m), ctypes.byref(e)))
    return m.value, e.value


def lbm_kernels_per_step(h):
    v = ctypes.c_int()
    _check(lib().lbm_kernels_per_step(h, ctypes.byref(v)))
    return v.value


def lbm_destroy(h):
    return _check(lib().lbm_destroy(h))


def lbm_supported(lattice, scheme, collision, layout, precision):
    return bool(lib().lbm_supported(lattice, scheme, collision, layout, precision))


def _check_static_buffers(lattice, N, f, flags, out):
    """Sizes, types and device of torch tensors handed to lbm_conserved_sums_static (the C
    side sees bare pointers and cannot check sizes)."""
    if not 1 <= int(N) <= 33554432:
        return  # the C call rejects the size itself, with its limit in the message
    want = (("f", f, "float64", lattice * int(N)), ("flags", flags, "uint8", int(N)), ("out", out, "float64", 2))
    for name, t, dtype, numel in want:
        if not hasattr(t, "data_ptr"):
            continue
        if str(t.dtype) != "torch." + dtype:
            raise LBMError(ERR_INVALID_ARG, f"{name} must be a {dtype} tensor, got {t.dtype}")
        if t.numel() < numel:
            raise LBMError(ERR_INVALID_ARG, f"{name} holds {t.numel()} elements, needs {numel}")
        if t.device.type == "cuda":
            import torch
            if t.device.index != torch.cuda.current_device():
                raise LBMError(ERR_INVALID_ARG, f"{name} is on {t.device}, not the current device")


def lbm_conserved_sums_static(lattice, N, f, flags, out, stream=None):
    """FP64 {sum rho, sum rho|u|^2/2} of canonical device populations into device out[2];
    allocates nothing (fixed library scratch; see include/lbm.h)."""
    _check_static_buffers(lattice, N, f, flags, out)
    return _check(lib().lbm_conserved_sums_static(lattice, N, ptr(f), ptr(flags), ptr(out), stream))


def lbm_batch_create():
    b = ctypes.c_void_p()
    _check(lib().lbm_batch_create(ctypes.byref(b)))
    return b


def lbm_batch_add(b, h):
    return _check(lib().lbm_batch_add(b, h))


def lbm_batch_remove(b, h):
    return _check(lib().lbm_batch_remove(b, h))


def lbm_batch_set_launch(b, threads, cells_per_thread):
    return _check(lib().lbm_batch_set_launch(b, threads, cells_per_thread))


def lbm_batch_autotune(b):
    t, c = ctypes.c_int(), ctypes.c_int()
    _check(lib().lbm_batch_autotune(b, ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


def lbm_batch_step(b, n, use_graph=True):
    return _check(lib().lbm_batch_step(b, n, 1 if use_graph else 0))


def lbm_batch_set_stream(b, stream):
    return _check(lib().lbm_batch_set_stream(b, stream))


def lbm_batch_sync(b):
    return _check(lib().lbm_batch_sync(b))


def lbm_batch_size(b):
    m, c = ctypes.c_int(), ctypes.c_longlong()
    _check(lib().lbm_batch_size(b, ctypes.byref(m), ctypes.byref(c)))
    return m.value, c.value


def lbm_batch_destroy(b):
    return _check(lib().lbm_batch_destroy(b))


def lbm_last_error():
    return lib().lbm_last_error().decode()


def _enum(v, table):
    return table[v] if isinstance(v, str) else int(v)


class Lattice:
    """One lattice on the GPU: a handle plus host-side bookkeeping of its sizes."""

    def __init__(self, lattice, nx, ny, nz, scheme, collision, omega, flags, layout=SOA, precision=F64,
                 wall_velocities=None, omega_bulk=None, omega_high=None, trt_lambda=None, stream=None):
        self.Q, self.nx, self.ny, self.nz = int(lattice), int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.h = lbm_create(self.Q, self.nx, self.ny, self.nz, _enum(scheme, SCHEMES), _enum(collision, MODELS),
                            float(omega), flags)
        try:
            if layout != SOA:
                lbm_set_layout(self.h, layout)
            if precision != F64:
                lbm_set_precision(self.h, _enum(precision, PRECISIONS))
            for fl, v in (wall_velocities or {}).items():
                lbm_set_wall_velocity(self.h, int(fl), *map(float, v))
            if omega_bulk is not None:
                lbm_set_param(self.h, PARAM_OMEGA_BULK, omega_bulk)
            if omega_high is not None:
                lbm_set_param(self.h, PARAM_OMEGA_HIGH, omega_high)
            if trt_lambda is not None:
                lbm_set_param(self.h, PARAM_TRT_LAMBDA, trt_lambda)
            if stream is not None:
                lbm_set_stream(self.h, stream)
        except Exception:
            self.close()
            raise

    def init_equilibrium(self, rho=None, u=None):
        lbm_init_equilibrium(self.h, rho, u)

    def step(self, n=1):
        lbm_step(self.h, n)

    def macroscopic(self, rho=None, u=None):
        """Fills the given buffers (host or device); allocates host numpy arrays if none given."""
        if rho is None and u is None:
            rho, u = np.empty(self.N), np.empty(3 * self.N)
            lbm_macroscopic(self.h, rho, u)
            return rho, u.reshape(3, self.N)
        lbm_macroscopic(self.h, rho, u)
        return rho, u

    def get_populations(self, out=None):
        if out is None:
            out = np.empty(self.Q * self.N)
            lbm_get_populations(self.h, out)
            return out.reshape(self.Q, self.N)
        lbm_get_populations(self.h, out)
        return out

    def set_populations(self, f):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
        lbm_set_populations(self.h, f)

    def step_sums(self, n=1):
        """(mass, energy) of the current state, then n steps: lbm_step_sums."""
        return lbm_step_sums(self.h, n)

    def step_sums_async(self, out, n=1):
        """lbm_step_sums_async: enqueue n steps; out receives the sums of the current state."""
        lbm_step_sums_async(self.h, n, out)

    def reduce(self):
        return lbm_reduce(self.h)

    def debug_check(self):
        """lbm_debug_check: the first recorded bounds fault (0: none); liblbm_debug.so only."""
        return lbm_debug_check(self.h)

    def set_link_fractions(self, q):
        """Walls at a fraction q of their links ([Q][N] FP64, or None for halfway walls)."""
        if q is not None:
            q = np.asarray(q, dtype=np.float64)
            if q.size != self.Q * self.N:
                raise LBMError(ERR_INVALID_ARG, f"link fractions need {self.Q} x {self.N} values")
        lbm_set_link_fractions(self.h, q)

    def set_param(self, key, value):
        lbm_set_param(self.h, key, value)

    @property
    def steps_done(self):
        return lbm_steps_done(self.h)

    @property
    def bytes_per_cell_update(self):
        return lbm_bytes_per_cell_update(self.h)

    @property
    def device_bytes(self):
        return lbm_device_bytes(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many lattices advanced by one launch per time step (members share lattice, model, precision)."""

    def __init__(self, lattices=()):
        self.b = lbm_batch_create()
        self.members = []
        for lat in lattices:
            self.add(lat)

    def add(self, lat):
        lbm_batch_add(self.b, lat.h)
        self.members.append(lat)

    def remove(self, lat):
        lbm_batch_remove(self.b, lat.h)
        self.members.remove(lat)

    def set_launch(self, threads=0, cells_per_thread=0):
        lbm_batch_set_launch(self.b, threads, cells_per_thread)

    def autotune(self):
        return lbm_batch_autotune(self.b)

    def step(self, n=1, use_graph=True):
        lbm_batch_step(self.b, n, use_graph)

    def set_stream(self, stream):
        """Launch on a caller's CUDA stream (a raw cudaStream_t value)."""
        lbm_batch_set_stream(self.b, stream)

    def sync(self):
        lbm_batch_sync(self.b)

    @property
    def size(self):
        return lbm_batch_size(self.b)

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
