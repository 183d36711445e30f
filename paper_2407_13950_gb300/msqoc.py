"""ctypes binding of libmsqoc (include/msqoc.h): argument marshalling only.

Every step of an evaluation runs in the CUDA library; this module converts Python arguments
(numpy arrays in host memory, or torch tensors on the GPU or host) into the pointers and sizes
of the C ABI and raises ``MsqocError`` on any non-zero status.  The names follow the C ABI:
``create_problem``, ``eval_objective``, ``eval_gradient``, ``query``, ``destroy_problem``.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

MSQOC_OK = 0
STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OUT_OF_MEMORY", -3: "NOT_ADMITTED", -4: "CUDA_ERROR",
                -5: "TIMEOUT", -6: "UNSUPPORTED", -7: "INTERNAL"}
SOLVER_DEFAULT, SOLVER_FP64, SOLVER_MIXED = 0, 1, 2
LAYOUT_AUTO, LAYOUT_FIBER, LAYOUT_PAIR, LAYOUT_QUAD, LAYOUT_FIBER_LEAN = 0, 1, 2, 3, 4

EXPORTED = ["msqoc_create_problem", "msqoc_query", "msqoc_query_layout", "msqoc_eval_objective", "msqoc_eval_gradient",
            "msqoc_destroy_problem", "msqoc_last_error", "msqoc_version", "msqoc_kernel_times",
            "msqoc_measure_fp64_peak", "msqoc_eval_objective_noalloc", "msqoc_batch_create",
            "msqoc_batch_eval_objective", "msqoc_batch_eval_gradient", "msqoc_batch_destroy", "msqoc_set_inputs",
            "msqoc_get_objective", "msqoc_get_gradient", "msqoc_batch_eval_subset", "msqoc_autotune",
            "msqoc_rollout", "msqoc_rollout_estimate", "msqoc_eval_regularization", "msqoc_lbfgs_direction",
            "msqoc_lbfgs_trial", "msqoc_lbfgs_update", "msqoc_selftest_bounded_wait",
            "msqoc_selftest_split", "msqoc_selftest_dot", "msqoc_selftest_carry"]
BATCH_GRADIENT, BATCH_GRAPH = 1, 2
KERNEL_NAMES = ["controls", "forward", "terminal", "adjoint", "finalize"]


class MsqocError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"msqoc {STATUS_NAMES.get(status, status)} ({status}): {message}")
        self.status = status


class Hamiltonian(ctypes.Structure):
    _fields_ = [("nqubits", ctypes.c_int32), ("nlevels", ctypes.c_int32), ("ness", ctypes.c_int32),
                ("xi", ctypes.c_void_p), ("xi_cross", ctypes.c_void_p), ("detune", ctypes.c_void_p),
                ("jx", ctypes.c_void_p)]


class Controls(ctypes.Structure):
    _fields_ = [("ncarriers", ctypes.c_void_p), ("carriers", ctypes.c_void_p), ("nsplines", ctypes.c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int32), ("col_block", ctypes.c_int32), ("ckpt_interval", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("layout", ctypes.c_int32), ("window_first", ctypes.c_int32),
                ("window_last", ctypes.c_int32), ("steps_per_sync", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmsqoc.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise MsqocError(-7, f"{path} is missing: build it with paper_2407_13950_gb300.build.build()")
        lib = ctypes.CDLL(path)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        sigs = {
            "msqoc_create_problem": (i32, [vp, vp, vp, ctypes.c_double, i64, i32, ctypes.c_double, vp, vp]),
            "msqoc_query": (i32, [vp, vp, vp, vp]),
            "msqoc_query_layout": (i32, [vp, vp, vp, vp, vp, vp, vp]),
            "msqoc_eval_objective": (i32, [vp, vp, vp, vp, vp, vp, vp]),
            "msqoc_eval_gradient": (i32, [vp, vp, vp, vp, vp, vp, vp]),
            "msqoc_destroy_problem": (i32, [vp]),
            "msqoc_last_error": (i32, [vp, sz]),
            "msqoc_version": (i32, []),
            "msqoc_kernel_times": (i32, [vp, vp]),
            "msqoc_measure_fp64_peak": (i32, [vp]),
            "msqoc_selftest_bounded_wait": (i32, [ctypes.c_int64, i32, vp]),
            "msqoc_selftest_split": (i32, [vp, i64, i32, i32, vp, vp]),
            "msqoc_selftest_dot": (i32, [vp, vp, i64, i32, i32, i32, vp]),
            "msqoc_selftest_carry": (i32, [vp, vp, vp, i64, i32, i32, vp]),
            "msqoc_eval_objective_noalloc": (i32, [vp, vp, vp, ctypes.c_double, i64, i32, ctypes.c_double, i32,
                                                   vp, vp, vp, vp, vp, vp]),
            "msqoc_batch_create": (i32, [vp, i32, i32, vp]),
            "msqoc_batch_eval_objective": (i32, [vp, vp]),
            "msqoc_batch_eval_gradient": (i32, [vp, vp]),
            "msqoc_batch_destroy": (i32, [vp]),
            "msqoc_set_inputs": (i32, [vp, vp, vp, vp]),
            "msqoc_get_objective": (i32, [vp, vp, vp, vp, vp]),
            "msqoc_get_gradient": (i32, [vp, vp, vp, vp, vp]),
            "msqoc_batch_eval_subset": (i32, [vp, vp, i32, i32, i32, vp]),
            "msqoc_rollout": (i32, [vp, vp, vp, vp]),
            "msqoc_rollout_estimate": (i32, [vp, vp, vp]),
            "msqoc_eval_regularization": (i32, [vp, vp, ctypes.c_double, ctypes.c_double, vp, vp, vp]),
            "msqoc_lbfgs_direction": (i32, [i64, i64, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp]),
            "msqoc_lbfgs_trial": (i32, [i64, i64, vp, vp, ctypes.c_double, vp, vp, vp, vp, vp]),
            "msqoc_lbfgs_update": (i32, [i64, vp, vp, vp, vp, vp, vp, vp, vp]),
            "msqoc_autotune": (i32, [vp, vp, ctypes.c_double, i64, i32, ctypes.c_double, vp, vp, i32, vp, vp, vp, vp,
                                     vp, vp, vp, i32, vp]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def last_error() -> str:
    lib = load()
    buf = ctypes.create_string_buffer(1024)
    lib.msqoc_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(status: int):
    if status != MSQOC_OK:
        raise MsqocError(status, last_error())


def _ptr(x) -> Optional[int]:
    """Data pointer of a numpy array or torch tensor (must be contiguous float64)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be contiguous float64")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):  # torch.Tensor
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class _Description:
    """The msqoc_hamiltonian / msqoc_controls structs of a problem spec, with the host arrays
    they point to kept alive."""

    def __init__(self, spec, target: Optional[np.ndarray] = None):
        q = spec.q
        self._xi = np.ascontiguousarray(spec.xi, dtype=np.float64)
        self._xc = np.ascontiguousarray(np.asarray(spec.xi_cross, dtype=np.float64).reshape(q, q))
        self._det = None if spec.detune is None else np.ascontiguousarray(spec.detune, dtype=np.float64)
        self._jx = None if spec.jx is None else np.ascontiguousarray(np.asarray(spec.jx, dtype=np.float64).reshape(q, q))
        self._nf = np.ascontiguousarray([len(w) for w in spec.omega], dtype=np.int32)
        self._om = np.ascontiguousarray([x for w in spec.omega for x in w], dtype=np.float64)
        self._tgt = None if target is None else np.ascontiguousarray(target, dtype=np.float64)
        self.H = Hamiltonian(q, spec.L, spec.ness, self._xi.ctypes.data, self._xc.ctypes.data,
                             None if self._det is None else self._det.ctypes.data,
                             None if self._jx is None else self._jx.ctypes.data)
        self.C = Controls(self._nf.ctypes.data, self._om.ctypes.data, spec.d1)
        self.target_ptr = None if self._tgt is None else self._tgt.ctypes.data


class Problem:
    """One multiple-shooting problem living on the current CUDA device.

    solver: SOLVER_MIXED (default: FP64 residual, FP32 corrections) or SOLVER_FP64; col_block:
    columns per sweep tile (0: the library's model); ckpt_interval: K (0: automatic); layout:
    LAYOUT_FIBER, LAYOUT_PAIR, LAYOUT_QUAD (2-level subsystems) or LAYOUT_FIBER_LEAN (one thread
    per fiber, 168 registers: 12 warps an SM) to force a sweep kernel family
    (LAYOUT_AUTO: the model's choice); steps_per_sync: time steps per synchronisation of a tile
    with the midpoint history (0: one); windows: (first, last), 1-based, to create the shard of
    windows first..last of the spec's M-window problem (its W input and grad_W output are the
    window states W^max(first-1,1) .. W^min(last,M-1); see `shard_w_range`).  After creation
    .col_block, .tiles, .threads, .ckpt_interval, .layout and .steps_per_sync report what the
    library chose, .nW the doubles of W and .npen the penalty terms the problem owns."""

    def __init__(self, spec, target: Optional[np.ndarray] = None, solver: int = SOLVER_DEFAULT,
                 col_block: int = 0, ckpt_interval: int = 0, profile: bool = False, layout: int = 0,
                 windows: Optional[tuple] = None, steps_per_sync: int = 0):
        lib = load()
        self.spec = spec
        self._desc = _Description(spec, target)
        first, last = windows if windows is not None else (0, 0)
        self.windows = (first, last) if windows is not None else (1, spec.M)
        O = Options(solver, col_block, ckpt_interval, 1 if profile else 0, layout, int(first), int(last),
                    int(steps_per_sync))
        h = ctypes.c_void_p()
        _check(lib.msqoc_create_problem(ctypes.byref(self._desc.H), ctypes.byref(self._desc.C), self._desc.target_ptr,
                                        float(spec.T), int(spec.nsteps), int(spec.M), float(spec.mu),
                                        ctypes.byref(O), ctypes.byref(h)))
        self.handle = h
        cb, nt, th, K = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        lay, sps = ctypes.c_int32(), ctypes.c_int32()
        _check(lib.msqoc_query_layout(h, ctypes.byref(cb), ctypes.byref(nt), ctypes.byref(th), ctypes.byref(K),
                                      ctypes.byref(lay), ctypes.byref(sps)))
        self.col_block, self.tiles, self.threads, self.ckpt_interval = cb.value, nt.value, th.value, K.value
        self.layout, self.steps_per_sync = lay.value, sps.value
        d, nW, nbytes = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        _check(lib.msqoc_query(h, ctypes.byref(d), ctypes.byref(nW), ctypes.byref(nbytes)))
        self.d, self.nW, self.device_bytes = d.value, nW.value, nbytes.value
        a, b = self.windows
        self.npen = (b - a + 1) - (1 if b == spec.M else 0)

    def close(self):
        if getattr(self, "handle", None):
            load().msqoc_destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def kernel_times(self) -> dict:
        """Device ms of each kernel of the last evaluation (problem created with profile=True)."""
        ms = (ctypes.c_float * 5)()
        _check(load().msqoc_kernel_times(self.handle, ms))
        return dict(zip(KERNEL_NAMES, [float(x) for x in ms]))

    # ---- host-array convenience API (numpy in, numpy out; synchronous)
    def eval_objective(self, alpha, W=None, stream=None) -> dict:
        P, J = np.zeros(1), np.zeros(1)
        pen = np.zeros(max(self.npen, 1))
        w = W if self.nW > 0 else None
        _check(load().msqoc_eval_objective(self.handle, _ptr(alpha), _ptr(w), _ptr(P), _ptr(J),
                                           _ptr(pen) if self.npen > 0 else None, _stream_handle(stream)))
        return {"P": float(P[0]), "J": float(J[0]), "pen": pen[:self.npen].copy()}

    def eval_gradient(self, alpha, W=None, stream=None) -> dict:
        P = np.zeros(1)
        ga = np.zeros(self.d)
        gW = np.zeros(max(self.nW, 1))
        w = W if self.nW > 0 else None
        _check(load().msqoc_eval_gradient(self.handle, _ptr(alpha), _ptr(w), _ptr(P), _ptr(ga),
                                          _ptr(gW) if self.nW > 0 else None, _stream_handle(stream)))
        return {"P": float(P[0]), "grad_alpha": ga, "grad_W": gW[:self.nW].copy()}

    def rollout(self, alpha, stream=None) -> np.ndarray:
        """Window states from a sequential roll-out of the identity under alpha (W^m = U(t_m))."""
        W = np.zeros(max(self.nW, 1))
        _check(load().msqoc_rollout(self.handle, _ptr(alpha), _ptr(W) if self.spec.M > 1 else None,
                                    _stream_handle(stream)))
        return W[:self.nW].copy()

    def rollout_estimate(self, stream=None) -> float:
        """Roll-out infidelity estimate from the last evaluation (objective or gradient)."""
        est = np.zeros(1)
        _check(load().msqoc_rollout_estimate(self.handle, _ptr(est), _stream_handle(stream)))
        return float(est[0])

    def eval_regularization(self, alpha, gamma_tik: float, gamma_energy: float, stream=None) -> dict:
        """Tikhonov + time-averaged control-energy regularization (Sec. 5) and its alpha-gradient."""
        R = np.zeros(1)
        g = np.zeros(self.d)
        _check(load().msqoc_eval_regularization(self.handle, _ptr(alpha), float(gamma_tik), float(gamma_energy),
                                                _ptr(R), _ptr(g), _stream_handle(stream)))
        return {"R": float(R[0]), "grad_alpha": g}

    # ---- pointer-level API (device tensors; asynchronous on the stream)
    def eval_regularization_into(self, alpha, gamma_tik: float, gamma_energy: float, R_out, grad_alpha,
                                 stream=None):
        _check(load().msqoc_eval_regularization(self.handle, _ptr(alpha), float(gamma_tik), float(gamma_energy),
                                                _ptr(R_out), _ptr(grad_alpha), _stream_handle(stream)))

    def eval_gradient_into(self, alpha, W, P_out, grad_alpha, grad_W, stream=None):
        _check(load().msqoc_eval_gradient(self.handle, _ptr(alpha), _ptr(W), _ptr(P_out), _ptr(grad_alpha),
                                          _ptr(grad_W), _stream_handle(stream)))

    def eval_objective_into(self, alpha, W, P_out, J_out=None, pen_out=None, stream=None):
        _check(load().msqoc_eval_objective(self.handle, _ptr(alpha), _ptr(W), _ptr(P_out), _ptr(J_out),
                                           _ptr(pen_out), _stream_handle(stream)))


def shard_w_range(M: int, first: int, last: int):
    """Window states W^k (k, 1-based) a shard of windows first..last of an M-window problem
    reads, and whose dP/dW terms it returns: (k_first, k_last), empty when k_last < k_first."""
    return max(first - 1, 1), min(last, M - 1)


# C-ABI-named functions
def create_problem(spec, target=None, **kw) -> Problem:
    return Problem(spec, target, **kw)


def eval_objective(problem: Problem, alpha, W=None, stream=None) -> dict:
    return problem.eval_objective(alpha, W, stream)


def eval_gradient(problem: Problem, alpha, W=None, stream=None) -> dict:
    return problem.eval_gradient(alpha, W, stream)


def query(problem: Problem):
    return problem.d, problem.nW, problem.device_bytes


def destroy_problem(problem: Problem):
    problem.close()


def measure_fp64_peak() -> float:
    """FP64 TFLOP/s of the current device (FMA microbenchmark in the library)."""
    t = ctypes.c_double()
    _check(load().msqoc_measure_fp64_peak(ctypes.byref(t)))
    return t.value


def selftest_bounded_wait(spins: int, arrive: bool = False) -> float:
    """The sweeps' bounded mbarrier wait on a phase that completes (arrive) or never does: raises
    MsqocError with status TIMEOUT (-5) when the wait gave up; returns the launch's seconds."""
    t = ctypes.c_double()
    _check(load().msqoc_selftest_bounded_wait(int(spins), 1 if arrive else 0, ctypes.byref(t)))
    return t.value


def selftest_split(x, sh: int = 0, device: bool = False):
    """(hi, lo) float32 arrays with x 2^-sh = hi + lo to 2^-48 (the mixed solver's split of the
    midpoint states for the gradient products), computed on the host or on the device."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    hi = np.empty(x.shape, np.float32)
    lo = np.empty(x.shape, np.float32)
    _check(load().msqoc_selftest_split(x.ctypes.data, x.size, int(sh), 1 if device else 0, hi.ctypes.data,
                                       lo.ctypes.data))
    return hi, lo


def selftest_dot(x, y, shx: int = 0, shy: int = 0, device: bool = False) -> float:
    """sum x_i y_i formed the way the mixed solver's adjoint forms its gradient products
    (split operands, compensated FP32 accumulation, one double)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if x.shape != y.shape:
        raise ValueError("x and y differ in shape")
    out = ctypes.c_double()
    _check(load().msqoc_selftest_dot(x.ctypes.data, y.ctypes.data, x.size, int(shx), int(shy), 1 if device else 0,
                                     ctypes.byref(out)))
    return out.value


def selftest_carry(u0, P, d, sh: int = 0, device: bool = False) -> complex:
    """n steps of the mixed solver's compensated implicit-midpoint state update on one entry:
    U_{j+1} = R U_j + 2 d_j with R = 2P - 1 (msqoc_selftest_carry); returns the final state."""
    u = np.array([complex(u0).real, complex(u0).imag])
    p = np.array([complex(P).real, complex(P).imag])
    dd = np.ascontiguousarray(np.asarray(d, dtype=np.complex128).reshape(-1)).view(np.float64)
    out = np.zeros(2)
    _check(load().msqoc_selftest_carry(u.ctypes.data, p.ctypes.data, dd.ctypes.data, dd.size // 2, int(sh),
                                       1 if device else 0, out.ctypes.data))
    return complex(out[0], out[1])


NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024   # MSQOC_NOALLOC_SCRATCH_BYTES


def eval_objective_noalloc(spec, alpha, W=None, target=None, solver: int = SOLVER_DEFAULT, stream=None,
                           P_out=None, J_out=None, pen_out=None) -> dict:
    """Objective of ``spec`` through msqoc_eval_objective_noalloc: no problem handle and no
    device allocation by the library (for callers that cannot allocate device memory).
    Outputs default to host arrays; device tensors may be passed instead.  Synchronous."""
    M = spec.M
    P = np.zeros(1) if P_out is None else P_out
    J = np.zeros(1) if J_out is None else J_out
    pen = np.zeros(max(M - 1, 1)) if pen_out is None else pen_out
    desc = _Description(spec, target)
    _check(load().msqoc_eval_objective_noalloc(ctypes.byref(desc.H), ctypes.byref(desc.C), desc.target_ptr,
                                               float(spec.T), int(spec.nsteps), int(M), float(spec.mu), int(solver),
                                               _ptr(alpha), _ptr(W if M > 1 else None), _ptr(P), _ptr(J),
                                               _ptr(pen) if M > 1 else None, _stream_handle(stream)))
    if P_out is not None:
        return {"P": P_out, "J": J_out, "pen": pen_out}
    return {"P": float(P[0]), "J": float(J[0]), "pen": pen[:M - 1].copy()}


class Batch:
    """Problems evaluated together (msqoc_batch_*): one sweep launch per shape for all of them,
    optionally replayed as a CUDA graph.  The problems must outlive the batch."""

    def __init__(self, problems, gradient: bool = True, graph: bool = False):
        lib = load()
        self.problems = list(problems)
        arr = (ctypes.c_void_p * len(self.problems))(*[p.handle.value for p in self.problems])
        flags = (BATCH_GRADIENT if gradient else 0) | (BATCH_GRAPH if graph else 0)
        h = ctypes.c_void_p()
        _check(lib.msqoc_batch_create(arr, len(self.problems), flags, ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().msqoc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_inputs(self, i: int, alpha, W=None, stream=None):
        p = self.problems[i]
        _check(load().msqoc_set_inputs(p.handle, _ptr(alpha), _ptr(W if p.spec.M > 1 else None),
                                       _stream_handle(stream)))

    def eval_gradient(self, stream=None):
        _check(load().msqoc_batch_eval_gradient(self.handle, _stream_handle(stream)))

    def eval_objective(self, stream=None):
        _check(load().msqoc_batch_eval_objective(self.handle, _stream_handle(stream)))

    def eval_subset(self, members, gradient: bool = True, slot: int = 0, stream=None):
        """Evaluate only the listed problems (indices into the batch) in shared launches."""
        arr = (ctypes.c_int32 * len(members))(*[int(m) for m in members])
        _check(load().msqoc_batch_eval_subset(self.handle, arr, len(members), 1 if gradient else 0, int(slot),
                                              _stream_handle(stream)))

    def get_gradient(self, i: int, stream=None) -> dict:
        p = self.problems[i]
        P = np.zeros(1)
        ga = np.zeros(p.d)
        gW = np.zeros(max(p.nW, 1))
        _check(load().msqoc_get_gradient(p.handle, _ptr(P), _ptr(ga), _ptr(gW) if p.spec.M > 1 else None,
                                         _stream_handle(stream)))
        return {"P": float(P[0]), "grad_alpha": ga, "grad_W": gW[:p.nW].copy()}

    def get_objective(self, i: int, stream=None) -> dict:
        p = self.problems[i]
        P, J = np.zeros(1), np.zeros(1)
        pen = np.zeros(max(p.spec.M - 1, 1))
        _check(load().msqoc_get_objective(p.handle, _ptr(P), _ptr(J), _ptr(pen) if p.spec.M > 1 else None,
                                          _stream_handle(stream)))
        return {"P": float(P[0]), "J": float(J[0]), "pen": pen[:p.spec.M - 1].copy()}


# ---- L-BFGS steps (device arrays; asynchronous on the stream)
LBFGS_MAXMEM = 64


def lbfgs_direction(n, nb, x, g, lim, S, Y, rho, yy, cap, m, head, d_out, slope_out, stream=None):
    """d_out = -H pg by the two-loop recursion over the m newest ring slots (msqoc_lbfgs_direction)."""
    _check(load().msqoc_lbfgs_direction(int(n), int(nb), _ptr(x), _ptr(g), _ptr(lim), _ptr(S), _ptr(Y), _ptr(rho),
                                        _ptr(yy), int(cap), int(m), int(head), _ptr(d_out), _ptr(slope_out),
                                        _stream_handle(stream)))


def lbfgs_trial(n, nb, x, d, step, lim, g, x_new, dec_out, stream=None):
    """x_new = box projection of x + step d, dec_out = <g, x_new - x> (msqoc_lbfgs_trial)."""
    _check(load().msqoc_lbfgs_trial(int(n), int(nb), _ptr(x), _ptr(d), float(step), _ptr(lim), _ptr(g), _ptr(x_new),
                                    _ptr(dec_out), _stream_handle(stream)))


def lbfgs_update(n, x, x_new, g, g_new, s_out, y_out, sy_yy_out, stream=None):
    """s_out = x_new - x, y_out = g_new - g, sy_yy_out = (<s, y>, <y, y>) (msqoc_lbfgs_update)."""
    _check(load().msqoc_lbfgs_update(int(n), _ptr(x), _ptr(x_new), _ptr(g), _ptr(g_new), _ptr(s_out), _ptr(y_out),
                                     _ptr(sy_yy_out), _stream_handle(stream)))


def autotune(spec, alpha=None, probe_steps: int = 64, solver: int = SOLVER_DEFAULT, ckpt_interval: int = 0,
             layout: int = LAYOUT_AUTO, steps_per_sync: int = 0):
    """Kernel family, columns per sweep tile and steps per history synchronisation by measurement
    (msqoc_autotune): returns (best width, best layout, best steps per sync,
    {(layout, width, steps per sync): ms per probe evaluation})."""
    lib = load()
    desc = _Description(spec)
    O = Options(solver, 0, ckpt_interval, 0, layout, 0, 0, steps_per_sync)
    a = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64)
    best, best_layout, best_sps = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    widths = (ctypes.c_int32 * 128)()
    layouts = (ctypes.c_int32 * 128)()
    depths = (ctypes.c_int32 * 128)()
    ms = (ctypes.c_float * 128)()
    n = ctypes.c_int32()
    _check(lib.msqoc_autotune(ctypes.byref(desc.H), ctypes.byref(desc.C), float(spec.T), int(spec.nsteps),
                              int(spec.M), float(spec.mu), ctypes.byref(O), None if a is None else a.ctypes.data,
                              int(probe_steps), ctypes.byref(best), ctypes.byref(best_layout), ctypes.byref(best_sps),
                              widths, layouts, depths, ms, 128, ctypes.byref(n)))
    return best.value, best_layout.value, best_sps.value, {
        (int(layouts[i]), int(widths[i]), int(depths[i])): float(ms[i]) for i in range(n.value)}
