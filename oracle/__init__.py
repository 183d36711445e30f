"""CPU oracle (test infrastructure only).

A plain, slow FP64 C implementation of one multiple-shooting objective + gradient
evaluation, written from the paper (see the header of ``msqoc_oracle.c`` for the equations
it follows).  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product path never does.

Complex arrays cross this boundary interleaved (re, im) as float64.  Helpers below convert
to numpy complex matrices: an N x E column-major matrix is ``x.view(complex).reshape(E, N).T``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msqoc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmsqoc_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/ (plain -O2, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fcx-limited-range", "-o", tmp, _SRC,
               "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int), ("L", ctypes.c_int), ("ness", ctypes.c_int),
        ("xi", ctypes.c_void_p), ("xi_cross", ctypes.c_void_p), ("detune", ctypes.c_void_p),
        ("jx", ctypes.c_void_p), ("nf", ctypes.c_void_p), ("omega", ctypes.c_void_p),
        ("d1", ctypes.c_int), ("T", ctypes.c_double), ("nsteps", ctypes.c_int64),
        ("M", ctypes.c_int), ("mu", ctypes.c_double), ("target", ctypes.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER(_Problem)
            vp, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            sig = {
                "oracle_dims": (ci, [P, vp, vp, vp]),
                "oracle_window_range": (None, [P, ci, vp, vp]),
                "oracle_bspline": (cd, [cd]),
                "oracle_controls": (None, [P, vp, cd, vp]),
                "oracle_system_hamiltonian": (ci, [P, vp]),
                "oracle_hamiltonian": (ci, [P, vp, cd, vp]),
                "oracle_lowering": (ci, [P, ci, vp]),
                "oracle_target": (ci, [P, vp]),
                "oracle_identity_state": (ci, [P, vp]),
                "oracle_infidelity": (cd, [P, vp]),
                "oracle_propagate": (ci, [P, vp, i64, i64, vp, vp, ci]),
                "oracle_propagate_adjoint": (ci, [P, vp, i64, i64, vp, vp, ci]),
                "oracle_rollout": (ci, [P, vp, vp]),
                "oracle_regularization": (cd, [P, vp, cd, cd, vp]),
                "oracle_eval_windows": (ci, [P, vp, vp, ci, ci, ci, vp, vp, vp, vp, vp, vp, vp]),
                "oracle_eval": (ci, [P, vp, vp, ci, vp, vp, vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


class Problem:
    """ctypes view of a ProblemSpec; keeps the parameter arrays alive."""

    def __init__(self, spec, target: Optional[np.ndarray] = None):
        self.spec = spec
        q = spec.q
        self._xi = np.ascontiguousarray(spec.xi, dtype=np.float64)
        self._xc = np.ascontiguousarray(np.asarray(spec.xi_cross, dtype=np.float64).reshape(q, q))
        self._det = None if spec.detune is None else np.ascontiguousarray(spec.detune, dtype=np.float64)
        self._jx = None if spec.jx is None else np.ascontiguousarray(np.asarray(spec.jx, dtype=np.float64).reshape(q, q))
        self._nf = np.ascontiguousarray([len(w) for w in spec.omega], dtype=np.int32)
        self._om = np.ascontiguousarray([x for w in spec.omega for x in w], dtype=np.float64)
        self._tgt = None if target is None else np.ascontiguousarray(target, dtype=np.float64)
        self.c = _Problem(q, spec.L, spec.ness, _ptr(self._xi), _ptr(self._xc), _ptr(self._det), _ptr(self._jx),
                          _ptr(self._nf), _ptr(self._om), spec.d1, float(spec.T), int(spec.nsteps), spec.M,
                          float(spec.mu), _ptr(self._tgt))
        N, E, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        if lib().oracle_dims(ctypes.byref(self.c), ctypes.byref(N), ctypes.byref(E), ctypes.byref(d)) != 0:
            raise ValueError("invalid problem description")
        self.N, self.E, self.d = N.value, E.value, d.value

    @property
    def ref(self):
        return ctypes.byref(self.c)


def _as_problem(spec_or_problem, target=None) -> Problem:
    return spec_or_problem if isinstance(spec_or_problem, Problem) else Problem(spec_or_problem, target)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def cplx_to_f64(z: np.ndarray) -> np.ndarray:
    """N x ncols complex matrix -> column-major interleaved doubles."""
    z = np.asarray(z, dtype=np.complex128)
    return np.ascontiguousarray(z.T).view(np.float64).ravel().copy()


def f64_to_cplx(x: np.ndarray, nrows: int) -> np.ndarray:
    """column-major interleaved doubles -> nrows x ncols complex matrix."""
    z = np.ascontiguousarray(x, dtype=np.float64).view(np.complex128)
    return z.reshape(-1, nrows).T.copy()


def dims(spec):
    p = _as_problem(spec)
    return p.N, p.E, p.d


def window_range(spec, m: int):
    p = _as_problem(spec)
    n0, n1 = ctypes.c_int64(), ctypes.c_int64()
    lib().oracle_window_range(p.ref, m, ctypes.byref(n0), ctypes.byref(n1))
    return n0.value, n1.value


def bspline(tau: float) -> float:
    return lib().oracle_bspline(float(tau))


def controls(spec, alpha, t: float) -> np.ndarray:
    p = _as_problem(spec)
    out = np.zeros(2 * p.spec.q)
    a = _f64(alpha)
    lib().oracle_controls(p.ref, _ptr(a), float(t), _ptr(out))
    return out.view(np.complex128).copy()


def system_hamiltonian(spec) -> np.ndarray:
    p = _as_problem(spec)
    out = np.zeros(2 * p.N * p.N)
    if lib().oracle_system_hamiltonian(p.ref, _ptr(out)):
        raise ValueError
    return f64_to_cplx(out, p.N)


def hamiltonian(spec, alpha, t: float) -> np.ndarray:
    p = _as_problem(spec)
    out = np.zeros(2 * p.N * p.N)
    a = _f64(alpha)
    if lib().oracle_hamiltonian(p.ref, _ptr(a), float(t), _ptr(out)):
        raise ValueError
    return f64_to_cplx(out, p.N)


def lowering(spec, k: int) -> np.ndarray:
    p = _as_problem(spec)
    out = np.zeros(2 * p.N * p.N)
    if lib().oracle_lowering(p.ref, k, _ptr(out)):
        raise ValueError
    return f64_to_cplx(out, p.N)


def target(spec, target=None) -> np.ndarray:
    p = _as_problem(spec, target)
    out = np.zeros(2 * p.N * p.E)
    if lib().oracle_target(p.ref, _ptr(out)):
        raise ValueError
    return f64_to_cplx(out, p.N)


def identity_state(spec) -> np.ndarray:
    p = _as_problem(spec)
    out = np.zeros(2 * p.N * p.E)
    if lib().oracle_identity_state(p.ref, _ptr(out)):
        raise ValueError
    return f64_to_cplx(out, p.N)


def infidelity(spec, U: np.ndarray, target=None) -> float:
    p = _as_problem(spec, target)
    u = cplx_to_f64(U)
    return lib().oracle_infidelity(p.ref, _ptr(u))


def propagate(spec, alpha, n0: int, n1: int, U: np.ndarray) -> np.ndarray:
    p = _as_problem(spec)
    U = np.asarray(U, dtype=np.complex128)
    u = cplx_to_f64(U)
    out = np.zeros_like(u)
    a = _f64(alpha)
    if lib().oracle_propagate(p.ref, _ptr(a), int(n0), int(n1), _ptr(u), _ptr(out), U.shape[1]):
        raise RuntimeError("oracle_propagate failed")
    return f64_to_cplx(out, p.N)


def propagate_adjoint(spec, alpha, n0: int, n1: int, Lam: np.ndarray) -> np.ndarray:
    p = _as_problem(spec)
    Lam = np.asarray(Lam, dtype=np.complex128)
    x = cplx_to_f64(Lam)
    out = np.zeros_like(x)
    a = _f64(alpha)
    if lib().oracle_propagate_adjoint(p.ref, _ptr(a), int(n0), int(n1), _ptr(x), _ptr(out), Lam.shape[1]):
        raise RuntimeError("oracle_propagate_adjoint failed")
    return f64_to_cplx(out, p.N)


def rollout(spec, alpha) -> np.ndarray:
    """W^1..W^{M-1} of the single-shooting roll-out, as the flat [M-1][E][N] interleaved vector."""
    p = _as_problem(spec)
    out = np.zeros(2 * p.N * p.E * max(p.spec.M - 1, 0))
    a = _f64(alpha)
    if lib().oracle_rollout(p.ref, _ptr(a), _ptr(out)):
        raise RuntimeError("oracle_rollout failed")
    return out


def regularization(spec, alpha, gamma_tik: float, gamma_energy: float):
    """(R, dR/dalpha): (gamma_tik/2)||alpha||^2 + gamma_energy * the midpoint-rule time average
    (1/T) int_0^T sum_k |d_k(t)|^2 dt (Sec. 5 regularization)."""
    p = _as_problem(spec)
    a = _f64(alpha)
    g = np.zeros(a.size)
    R = lib().oracle_regularization(p.ref, _ptr(a), float(gamma_tik), float(gamma_energy), _ptr(g))
    return R, g


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def evaluate(spec, alpha, W, *, grad: bool = True, nthreads: Optional[int] = None, windows=None,
             per_window: bool = False, target=None) -> dict:
    """Objective (and gradient) of the multiple-shooting problem.

    windows=(lo, hi) restricts the work to windows lo..hi (1-based, inclusive); then P is the
    sum of those windows' terms and grad_W is valid only for m with m and m+1 in range.
    """
    p = _as_problem(spec, target)
    M = p.spec.M
    lo, hi = (1, M) if windows is None else windows
    a = _f64(alpha)
    w = _f64(W) if M > 1 else np.zeros(2)
    P, J = ctypes.c_double(), ctypes.c_double(np.nan)
    pen = np.zeros(max(M - 1, 1))
    ga = np.zeros(p.d) if grad else None
    gW = np.zeros(max(2 * p.N * p.E * (M - 1), 1)) if grad else None
    ne2 = 2 * p.N * p.E
    Uend = np.zeros(ne2 * M) if per_window else None
    Lam0 = np.zeros(ne2 * M) if (per_window and grad) else None
    rc = lib().oracle_eval_windows(p.ref, _ptr(a), _ptr(w), lo, hi, nthreads or default_threads(),
                                   ctypes.byref(P), ctypes.byref(J), _ptr(pen), _ptr(ga), _ptr(gW),
                                   _ptr(Uend), _ptr(Lam0))
    if rc != 0:
        raise RuntimeError(f"oracle_eval_windows failed ({rc})")
    out = {"P": P.value, "J": J.value if hi == M else float("nan"), "pen": pen[: M - 1].copy()}
    if grad:
        out["grad_alpha"] = ga
        out["grad_W"] = gW[: 2 * p.N * p.E * (M - 1)]
    if per_window:
        out["Uend"] = Uend
        if grad:
            out["Lam0"] = Lam0
    return out
