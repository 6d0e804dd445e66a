"""Python binding of the GB300 ENO-AO library (``libenoao.so``, include/enoao.h).

Argument marshalling only: every step of the scheme runs in the library's
CUDA kernels.  There is no CPU fallback -- if the library is missing, or no
GPU is present, the calls raise.

States are float64 arrays shaped ``(nv, nz, ny, nx)`` (structure of arrays,
x fastest): numpy arrays are host buffers, CUDA torch tensors are device
buffers (``on_device`` in the C interface).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import inputs  # noqa: F401  (seeded workload generators)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libenoao.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "enoao.h")

SCALAR_ADVECTION, EULER = 0, 1
PERIODIC, TRANSMISSIVE = 0, 1
FP64, FP32_BULK = 0, 1
ALPHA_PER_STEP, ALPHA_PER_STAGE, ALPHA_PER_FIELD = 0, 1, 2
REDECIDE_AUTO, REDECIDE_IN_SWEEP, REDECIDE_GRID = 0, 1, 2

STATUS = {0: "ENOAO_OK", 1: "ENOAO_EINVAL", 2: "ENOAO_ENOMEM", 3: "ENOAO_ECUDA",
          4: "ENOAO_ENONPHYS", 5: "ENOAO_ETIMEOUT"}


class EnoaoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("system", ctypes.c_int), ("order", ctypes.c_int),
        ("precision", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3), ("bc", ctypes.c_int * 3), ("alpha_mode", ctypes.c_int),
        ("adv_speed", ctypes.c_double), ("gamma", ctypes.c_double),
        ("delta", ctypes.c_double), ("tie_rel", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("steps", ctypes.c_int64), ("alpha", ctypes.c_double * 3),
        ("dt", ctypes.c_double), ("fp64_fallbacks", ctypes.c_uint64),
        ("decisions", ctypes.c_uint64),
    ]


_lib = None


def header_symbols():
    """Entry points declared in include/enoao.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"\b(enoao_\w+)\s*\(", text)))


def load():
    """Load libenoao.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, D, I64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
    C = ctypes.POINTER(Config)
    sig = {
        "enoao_config_default": (None, [C]),
        "enoao_create": (ctypes.c_int, [C, P, ctypes.POINTER(P)]),
        "enoao_batch_create": (ctypes.c_int, [C, ctypes.c_int, ctypes.POINTER(I64), D, D, P,
                                              ctypes.POINTER(P)]),
        "enoao_destroy": (None, [P]),
        "enoao_batch_problem_stats": (ctypes.c_int, [P, ctypes.c_int, D, D, D]),
        "enoao_create_subdomain": (ctypes.c_int, [C, I64, I64, P, ctypes.POINTER(P)]),
        "enoao_halo_export": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int]),
        "enoao_halo_import": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int]),
        "enoao_halo_fill_transmissive": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int]),
        "enoao_local_alpha": (ctypes.c_int, [P, D]),
        "enoao_set_step_alpha": (ctypes.c_int, [P, D]),
        "enoao_last_error": (ctypes.c_char_p, [P]),
        "enoao_init_state": (ctypes.c_int, [P, P, ctypes.c_int]),
        "enoao_get_state": (ctypes.c_int, [P, P, ctypes.c_int]),
        "enoao_get_stage_state": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int]),
        "enoao_reconstruct_fluxes": (ctypes.c_int, [P, ctypes.c_int, P, P, ctypes.c_int]),
        "enoao_rk_stage": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_double]),
        "enoao_advance": (ctypes.c_int, [P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         I64, D, ctypes.POINTER(I64)]),
        "enoao_advance_steps": (ctypes.c_int, [P, I64, ctypes.c_double]),
        "enoao_advance_steps_async": (ctypes.c_int, [P, I64, ctypes.c_double]),
        "enoao_sync": (ctypes.c_int, [P]),
        "enoao_get_stats": (ctypes.c_int, [P, ctypes.POINTER(Stats)]),
        "enoao_launches_per_step": (ctypes.c_int, [P]),
        "enoao_set_tiles": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "enoao_set_redecide": (ctypes.c_int, [P, ctypes.c_int]),
        "enoao_uses_grid_redecide": (ctypes.c_int, [P]),
        "enoao_set_redecide_pass_limit": (ctypes.c_int, [P, ctypes.c_int]),
        "enoao_set_tma": (ctypes.c_int, [P, ctypes.c_int]),
        "enoao_set_fused_stage": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int]),
        "enoao_get_tiles": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
        "enoao_autotune": (ctypes.c_int, [P]),
        "enoao_time_sweep": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_float)]),
        "enoao_step_noalloc": (ctypes.c_int, [C, P, P, ctypes.c_double, P]),
        "enoao_measure_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P,
                                                  ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_float)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, nbytes=None):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if _is_torch(x):
        assert x.is_contiguous(), "tensor must be contiguous"
        return ctypes.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return ctypes.c_void_p(x.ctypes.data), 0


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_config(shape, lo, hi, system=EULER, order=5, precision=FP64, bc=TRANSMISSIVE,
                adv_speed=1.0, gamma=1.4, delta=1e-5, tie_rel=1e-3,
                alpha_mode=0) -> Config:
    lib = load()
    cfg = Config()
    lib.enoao_config_default(ctypes.byref(cfg))
    ndim = len(shape)
    cfg.ndim, cfg.system, cfg.order, cfg.precision = ndim, system, order, precision
    bcs = bc if isinstance(bc, (list, tuple)) else [bc] * ndim
    for d in range(3):
        if d < ndim:
            cfg.n[d], cfg.lo[d], cfg.hi[d], cfg.bc[d] = int(shape[d]), lo[d], hi[d], int(bcs[d])
    cfg.adv_speed, cfg.gamma, cfg.delta, cfg.tie_rel = adv_speed, gamma, delta, tie_rel
    cfg.alpha_mode = alpha_mode
    return cfg


def step_noalloc(cfg, U_in, U_out, dt, stream=None):
    """One Runge-Kutta step of a 1D problem through enoao_step_noalloc.

    U_in / U_out are CUDA tensors shaped (nv, n) or (nv, 1, 1, n); the library
    allocates nothing for the step (its stage states live in a fixed device
    array of at most 2^18 cells)."""
    nv = 3 if cfg.system == EULER else 1
    n = int(cfg.n[0])
    for name, U in (("U_in", U_in), ("U_out", U_out)):
        # the C side reads and writes nv * n doubles through these pointers:
        # check everything it cannot see before any device call
        if not _is_torch(U):
            raise ValueError(f"{name} must be a CUDA torch tensor")
        if tuple(U.shape) not in ((nv, n), (nv, 1, 1, n)):
            raise ValueError(f"{name} has shape {tuple(U.shape)}; expected ({nv}, {n})")
        if str(U.dtype) != "torch.float64":
            raise ValueError(f"{name} has dtype {U.dtype}; expected torch.float64")
        if not U.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if not U.is_cuda:
            raise ValueError(f"{name} must be on the GPU (enoao_step_noalloc takes device buffers)")
        import torch
        if U.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on cuda:{U.device.index}, not the current device "
                             f"cuda:{torch.cuda.current_device()}")
    lib = load()
    pi, _ = _ptr(U_in)
    po, _ = _ptr(U_out)
    st = lib.enoao_step_noalloc(ctypes.byref(cfg), pi, po, dt, _stream_handle(stream))
    if st:
        raise EnoaoError(st, lib.enoao_last_error(None).decode())


PEAK_FP32, PEAK_FP32X2, PEAK_FP64 = 0, 1, 2


def measure_fma_peak(kind, trips=1000, stream=None):
    """(TFLOP/s, ms) of the multiply-add microbenchmark of the given kind."""
    lib = load()
    tf, ms = ctypes.c_double(), ctypes.c_float()
    st = lib.enoao_measure_fma_peak(kind, trips, _stream_handle(stream), ctypes.byref(tf),
                                    ctypes.byref(ms))
    if st:
        raise EnoaoError(st, "enoao_measure_fma_peak failed")
    return tf.value, ms.value


class Solver:
    """One ENO-AO problem on the GPU (enoao_create); shape = (nx,), (nx, ny) or (nx, ny, nz)."""

    def __init__(self, shape, lo, hi, stream=None, **kw):
        self._lib = load()
        self.cfg = make_config(shape, lo, hi, **kw)
        self.shape = tuple(int(s) for s in shape)
        self.nv = len(shape) + 2 if self.cfg.system == EULER else 1
        full = list(self.shape) + [1] * (3 - len(self.shape))
        self.state_shape = (self.nv, full[2], full[1], full[0])
        self._h = ctypes.c_void_p()
        st = self._lib.enoao_create(ctypes.byref(self.cfg), _stream_handle(stream),
                                    ctypes.byref(self._h))
        if st:
            raise EnoaoError(st, self._lib.enoao_last_error(None).decode())

    # -- plumbing
    def _check(self, st):
        if st:
            raise EnoaoError(st, self._lib.enoao_last_error(self._h).decode())

    def close(self):
        if self._h:
            self._lib.enoao_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- C-ABI mirrors
    def init_state(self, U):
        if not _is_torch(U):
            U = np.ascontiguousarray(U, dtype=np.float64)
        assert tuple(U.shape) == self.state_shape, (tuple(U.shape), self.state_shape)
        p, dev = _ptr(U)
        self._check(self._lib.enoao_init_state(self._h, p, dev))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.state_shape)
        p, dev = _ptr(out)
        self._check(self._lib.enoao_get_state(self._h, p, dev))
        return out

    def get_stage_state(self, k, out=None):
        """Runge-Kutta stage state k (0: U^n, 1: U^(1), 2: U^(2)) as last written."""
        if out is None:
            out = np.empty(self.state_shape)
        p, dev = _ptr(out)
        self._check(self._lib.enoao_get_stage_state(self._h, k, p, dev))
        return out

    def face_shape(self, d):
        s = list(self.state_shape)
        s[3 - d] += 1
        return tuple(s)

    def reconstruct_fluxes(self, d, want_idx=False, out=None, idx_out=None):
        fs = self.face_shape(d)
        F = np.empty(fs) if out is None else out
        idx = None
        if want_idx:
            idx = np.empty((fs[0], 2) + fs[1:], dtype=np.int8) if idx_out is None else idx_out
        pF, dev = _ptr(F)
        pI = _ptr(idx)[0] if idx is not None else None
        self._check(self._lib.enoao_reconstruct_fluxes(self._h, d, pF, pI, dev))
        return F, idx

    def rk_stage(self, stage, dt):
        self._check(self._lib.enoao_rk_stage(self._h, stage, dt))

    def advance(self, t_end, cfl=0.5, dt_fixed=0.0, max_steps=0):
        t = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self._lib.enoao_advance(self._h, t_end, cfl, dt_fixed, max_steps,
                                            ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value

    def advance_steps(self, nsteps, cfl=0.5):
        self._check(self._lib.enoao_advance_steps(self._h, nsteps, cfl))

    def advance_steps_async(self, nsteps, cfl=0.5):
        self._check(self._lib.enoao_advance_steps_async(self._h, nsteps, cfl))

    def sync(self):
        self._check(self._lib.enoao_sync(self._h))

    def stats(self) -> Stats:
        s = Stats()
        self._check(self._lib.enoao_get_stats(self._h, ctypes.byref(s)))
        return s

    def launches_per_step(self):
        return self._lib.enoao_launches_per_step(self._h)

    def set_tiles(self, d, ta, ts):
        self._check(self._lib.enoao_set_tiles(self._h, d, ta, ts))

    def set_redecide(self, mode):
        """Where FP32-bulk near-ties are re-decided in FP64: REDECIDE_AUTO,
        REDECIDE_IN_SWEEP or REDECIDE_GRID (the grid-wide pass after each sweep)."""
        self._check(self._lib.enoao_set_redecide(self._h, mode))

    def set_tma(self, on):
        """FP32 bulk: stage raw tiles by TMA (True) or load them directly (False, default)."""
        self._check(self._lib.enoao_set_tma(self._h, 1 if on else 0))

    def set_fused_stage(self, on, tiles=(0, 0, 0, 0)):
        """2D: one launch per Runge-Kutta stage for both axes (True) or one per
        axis (False, default); tiles = (x_lines, x_cells, y_lines, y_cells), all
        0 to keep the current ones."""
        self._check(self._lib.enoao_set_fused_stage(self._h, 1 if on else 0, *[int(t) for t in tiles]))

    def set_redecide_pass_limit(self, passes):
        """Test knob: bound on the in-sweep FP64 re-decision passes (-1: default)."""
        self._check(self._lib.enoao_set_redecide_pass_limit(self._h, passes))

    def uses_grid_redecide(self):
        return bool(self._lib.enoao_uses_grid_redecide(self._h))

    def get_tiles(self, d):
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.enoao_get_tiles(self._h, d, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def time_sweep(self, d, nrep=10):
        """Mean duration (ms) of one sweep-kernel launch along axis d (CUDA events)."""
        ms = ctypes.c_float()
        self._check(self._lib.enoao_time_sweep(self._h, d, nrep, ctypes.byref(ms)))
        return ms.value

    def autotune(self):
        self._check(self._lib.enoao_autotune(self._h))


class SubDomain(Solver):
    """Layers [offset, offset + n_local) of the last axis of a 2D/3D problem
    (enoao_create_subdomain); shape, lo, hi describe the global grid."""

    def __init__(self, shape, lo, hi, offset, n_local, stream=None, **kw):
        self._lib = load()
        self.cfg = make_config(shape, lo, hi, **kw)
        self.global_shape = tuple(int(s) for s in shape)
        local = list(self.global_shape)
        local[-1] = int(n_local)
        self.shape = tuple(local)
        self.offset, self.n_local = int(offset), int(n_local)
        self.nv = len(shape) + 2 if self.cfg.system == EULER else 1
        full = list(self.shape) + [1] * (3 - len(self.shape))
        self.state_shape = (self.nv, full[2], full[1], full[0])
        self.G = self.cfg.order // 2 + 2
        self.plane = int(np.prod(self.shape[:-1]))
        self.halo_shape = (self.nv, self.G, self.plane)
        self._h = ctypes.c_void_p()
        st = self._lib.enoao_create_subdomain(ctypes.byref(self.cfg), self.offset, self.n_local,
                                              _stream_handle(stream), ctypes.byref(self._h))
        if st:
            raise EnoaoError(st, self._lib.enoao_last_error(None).decode())

    def halo_export(self, k, side, out=None):
        if out is None:
            out = np.empty(self.halo_shape)
        p, dev = _ptr(out)
        self._check(self._lib.enoao_halo_export(self._h, k, side, p, dev))
        return out

    def halo_import(self, k, side, buf):
        p, dev = _ptr(buf)
        self._check(self._lib.enoao_halo_import(self._h, k, side, p, dev))

    def halo_fill_transmissive(self, k, side):
        self._check(self._lib.enoao_halo_fill_transmissive(self._h, k, side))

    def local_alpha(self):
        a = np.zeros(3)
        self._check(self._lib.enoao_local_alpha(self._h, a.ctypes.data_as(
            ctypes.POINTER(ctypes.c_double))))
        return a

    def set_step_alpha(self, alpha):
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        self._check(self._lib.enoao_set_step_alpha(self._h, a.ctypes.data_as(
            ctypes.POINTER(ctypes.c_double))))


class Batch(Solver):
    """Independent 1D problems of uneven lengths (enoao_batch_create)."""

    def __init__(self, sizes, lo, hi, stream=None, **kw):
        self._lib = load()
        sizes = np.ascontiguousarray(sizes, dtype=np.int64)
        lo = np.ascontiguousarray(np.broadcast_to(lo, sizes.shape), dtype=np.float64)
        hi = np.ascontiguousarray(np.broadcast_to(hi, sizes.shape), dtype=np.float64)
        self.cfg = make_config((int(sizes.max()),), (0.0,), (1.0,), **kw)
        self.sizes = sizes
        self.nv = 3 if self.cfg.system == EULER else 1
        self.state_shape = (self.nv, int(sizes.sum()))
        self._h = ctypes.c_void_p()
        D = ctypes.POINTER(ctypes.c_double)
        st = self._lib.enoao_batch_create(
            ctypes.byref(self.cfg), len(sizes), sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            lo.ctypes.data_as(D), hi.ctypes.data_as(D), _stream_handle(stream), ctypes.byref(self._h))
        if st:
            raise EnoaoError(st, self._lib.enoao_last_error(None).decode())

    def problem_stats(self, p):
        """(t, alpha of the last step, last dt) of problem p."""
        t, a, dt = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.enoao_batch_problem_stats(self._h, p, ctypes.byref(t),
                                                        ctypes.byref(a), ctypes.byref(dt)))
        return t.value, a.value, dt.value
