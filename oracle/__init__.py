"""TEST INFRASTRUCTURE ONLY: ctypes wrapper around the plain FP64 C oracle.

The oracle restates the ENO-AO method of Shen (arXiv 2108.12742) on the CPU,
operation by operation, so that the CUDA library can be checked against it.
Only the test-suite, ``__graft_entry__.smoke`` and the CPU-baseline leg of
``bench.py`` may import this module; the library itself never does.

State arrays are C-contiguous float64 numpy arrays shaped ``(nv, nz, ny, nx)``
(structure of arrays, x fastest), with nv = 1 for scalar advection and
nv = ndim + 2 for the Euler equations (rho, momenta, total energy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "enoao_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SCALAR, EULER = 0, 1
PERIODIC, TRANSMISSIVE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -ffp-contract=off)."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
            _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class Problem(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("system", ctypes.c_int), ("order", ctypes.c_int),
        ("nthreads", ctypes.c_int), ("n", ctypes.c_long * 3),
        ("dx", ctypes.c_double * 3), ("bc", ctypes.c_int * 3), ("alpha_per_stage", ctypes.c_int),
        ("alpha_per_field", ctypes.c_int),
        ("adv_speed", ctypes.c_double), ("gamma", ctypes.c_double),
        ("delta", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            P = ctypes.POINTER(Problem)
            lib.or_face_value.restype = ctypes.c_double
            lib.or_face_value.argtypes = [D, ctypes.c_int, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_int), D, D]
            lib.or_candidate_deltas.argtypes = [D, ctypes.c_int, D, D]
            lib.or_candidate_flux.restype = ctypes.c_double
            lib.or_candidate_flux.argtypes = [D, ctypes.c_int]
            lib.or_euler_eigen.argtypes = [ctypes.c_int, ctypes.c_double, D,
                                           ctypes.c_double, D, D]
            lib.or_roe_average.argtypes = [D, D, ctypes.c_int, ctypes.c_double, D, D]
            lib.or_alpha.argtypes = [P, D, D]
            lib.or_alpha_fields.argtypes = [P, D, D]
            lib.or_fluxes_fields.argtypes = [P, D, ctypes.c_int, D, D,
                                             ctypes.POINTER(ctypes.c_byte), D]
            lib.or_rhs_fields.argtypes = [P, D, D, D]
            lib.or_step_alpha_fields.argtypes = [P, D, ctypes.c_double, D]
            lib.or_fluxes.argtypes = [P, D, ctypes.c_int, D, D,
                                      ctypes.POINTER(ctypes.c_byte), D]
            lib.or_rhs.argtypes = [P, D, D, D]
            lib.or_step.argtypes = [P, D, ctypes.c_double]
            lib.or_step_alpha.argtypes = [P, D, ctypes.c_double, D]
            lib.or_advance.argtypes = [P, D, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_long,
                                       D, ctypes.POINTER(ctypes.c_long)]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_problem(shape, lo, hi, system=EULER, order=5, bc=TRANSMISSIVE,
                 adv_speed=1.0, gamma=1.4, delta=1e-5, nthreads=0,
                 alpha_per_stage=False, alpha_per_field=False) -> Problem:
    """shape = (nx,) / (nx, ny) / (nx, ny, nz); lo/hi per axis; bc scalar or per axis;
    alpha_per_stage: each Runge-Kutta stage splits with the alpha of its own input state;
    alpha_per_field: each characteristic field k splits with max |lambda_k| (Euler).
    With alpha_per_field the alpha arguments below are the (3, 5) per-field arrays
    of ``alpha_fields``."""
    ndim = len(shape)
    P = Problem()
    P.ndim, P.system, P.order, P.nthreads = ndim, system, order, nthreads
    bcs = bc if isinstance(bc, (list, tuple)) else [bc] * ndim
    for d in range(3):
        if d < ndim:
            P.n[d] = int(shape[d])
            P.dx[d] = (hi[d] - lo[d]) / shape[d]
            P.bc[d] = int(bcs[d])
        else:
            P.n[d], P.dx[d], P.bc[d] = 1, 1.0, PERIODIC
    P.adv_speed, P.gamma, P.delta = adv_speed, gamma, delta
    P.alpha_per_stage = int(bool(alpha_per_stage))
    P.alpha_per_field = int(bool(alpha_per_field))
    return P


def nvars(P: Problem) -> int:
    return P.ndim + 2 if P.system == EULER else 1


def _state(P, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.size == nvars(P) * P.n[0] * P.n[1] * P.n[2]
    return U


def face_value(window9, order=5, delta=1e-5):
    """window9[k] = f_{j+k-4}; returns (value, index, IS[9], gap_rel)."""
    w = np.ascontiguousarray(window9, dtype=np.float64)
    assert w.size == 9
    lib = _load()
    idx = ctypes.c_int()
    IS = np.zeros(9)
    gap = ctypes.c_double()
    centre = _centre(w)
    v = lib.or_face_value(centre, order, delta, ctypes.byref(idx), _dp(IS),
                          ctypes.cast(ctypes.byref(gap), ctypes.POINTER(ctypes.c_double)))
    return v, idx.value, IS, gap.value


def _centre(w):
    return ctypes.cast(w.ctypes.data + 4 * 8, ctypes.POINTER(ctypes.c_double))


def candidate_deltas(window9, c):
    w = np.ascontiguousarray(window9, dtype=np.float64)
    dl, dr = ctypes.c_double(), ctypes.c_double()
    _load().or_candidate_deltas(_centre(w), c,
                                ctypes.cast(ctypes.byref(dl), ctypes.POINTER(ctypes.c_double)),
                                ctypes.cast(ctypes.byref(dr), ctypes.POINTER(ctypes.c_double)))
    return dl.value, dr.value


def candidate_flux(window9, c):
    w = np.ascontiguousarray(window9, dtype=np.float64)
    return _load().or_candidate_flux(_centre(w), c)


def euler_eigen(ndim, gamma, vel, H):
    nv = ndim + 2
    R = np.zeros((nv, nv))
    L = np.zeros((nv, nv))
    v = np.ascontiguousarray(vel, dtype=np.float64)
    _load().or_euler_eigen(ndim, gamma, _dp(v), H, _dp(R), _dp(L))
    return R, L


def roe_average(ndim, gamma, ql, qr):
    """Roe-averaged (velocity[ndim], H) of two conserved Euler states."""
    ql = np.ascontiguousarray(ql, dtype=np.float64)
    qr = np.ascontiguousarray(qr, dtype=np.float64)
    assert ql.shape == qr.shape == (ndim + 2,)
    vel = np.zeros(ndim)
    H = ctypes.c_double()
    _load().or_roe_average(_dp(ql), _dp(qr), ndim, gamma, _dp(vel), ctypes.byref(H))
    return vel, H.value


def alpha(P, U):
    U = _state(P, U)
    a = np.zeros(3)
    st = _load().or_alpha(ctypes.byref(P), _dp(U), _dp(a))
    if st:
        raise FloatingPointError("oracle: non-physical state")
    return a


def alpha_fields(P, U):
    """Per-field splitting constants, shape (3, 5): [d, k] = max |lambda_k| along d."""
    U = _state(P, U)
    a = np.zeros(15)
    st = _load().or_alpha_fields(ctypes.byref(P), _dp(U), _dp(a))
    if st:
        raise FloatingPointError("oracle: non-physical state")
    return a.reshape(3, 5)


def _per_field(P):
    return bool(P.alpha_per_field) and P.system == EULER


def _alpha_arg(P, U, alpha_vec):
    if _per_field(P):
        a = alpha_fields(P, U) if alpha_vec is None else alpha_vec
        return np.ascontiguousarray(a, dtype=np.float64).reshape(15)
    return alpha(P, U) if alpha_vec is None else np.ascontiguousarray(alpha_vec, dtype=np.float64)


def face_shape(P, d):
    nv = nvars(P)
    n = [P.n[0], P.n[1], P.n[2]]
    n[d] += 1
    return (nv, n[2], n[1], n[0])


def fluxes(P, U, d, alpha_vec=None, want_idx=False):
    """Interface fluxes along axis d: (Fhat, idx, gap) with face-major layout."""
    U = _state(P, U)
    a = _alpha_arg(P, U, alpha_vec)
    shp = face_shape(P, d)
    F = np.zeros(shp)
    idx = np.zeros((shp[0], 2) + shp[1:], dtype=np.int8) if want_idx else None
    gap = np.zeros((shp[0], 2) + shp[1:]) if want_idx else None
    fn = _load().or_fluxes_fields if _per_field(P) else _load().or_fluxes
    st = fn(ctypes.byref(P), _dp(U), d, _dp(a), _dp(F),
                           idx.ctypes.data_as(ctypes.POINTER(ctypes.c_byte)) if want_idx else None,
                           _dp(gap) if want_idx else None)
    assert st == 0
    return F, idx, gap


def rhs(P, U, alpha_vec=None):
    U = _state(P, U)
    a = _alpha_arg(P, U, alpha_vec)
    out = np.zeros_like(U)
    fn = _load().or_rhs_fields if _per_field(P) else _load().or_rhs
    fn(ctypes.byref(P), _dp(U), _dp(a), _dp(out))
    return out


def step(P, U, dt):
    U = _state(P, U).copy()
    st = _load().or_step(ctypes.byref(P), _dp(U), dt)
    if st:
        raise FloatingPointError("oracle: non-physical state")
    return U


def step_alpha(P, U, dt, alpha_vec):
    """One step with the splitting constants of the full mesh given."""
    U = _state(P, U).copy()
    a = _alpha_arg(P, U, alpha_vec)
    fn = _load().or_step_alpha_fields if _per_field(P) else _load().or_step_alpha
    fn(ctypes.byref(P), _dp(U), dt, _dp(a))
    return U


def advance(P, U, t_end, cfl=0.5, dt_fixed=0.0, max_steps=0):
    """Returns (U_final, t, steps)."""
    U = _state(P, U).copy()
    t = ctypes.c_double()
    n = ctypes.c_long()
    st = _load().or_advance(ctypes.byref(P), _dp(U), t_end, cfl, dt_fixed, max_steps,
                            ctypes.cast(ctypes.byref(t), ctypes.POINTER(ctypes.c_double)),
                            ctypes.byref(n))
    if st:
        raise FloatingPointError("oracle: non-physical state")
    return U, t.value, n.value
