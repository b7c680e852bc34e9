"""Python binding of liblrs.so (include/lrs.h), by ctypes.

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Host arrays are numpy arrays; device arrays are torch CUDA
tensors (PyTorch supplies device memory and streams).  The functions carry
the C names; `Solver` is a small convenience wrapper over them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblrs.so")

LRS_OK, LRS_ERR_ARG, LRS_ERR_STATE, LRS_ERR_OOM, LRS_ERR_CUDA, LRS_ERR_NUMERICAL, \
    LRS_ERR_TIMEOUT, LRS_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["LRS_OK", "LRS_ERR_ARG", "LRS_ERR_STATE", "LRS_ERR_OOM", "LRS_ERR_CUDA",
                "LRS_ERR_NUMERICAL", "LRS_ERR_TIMEOUT", "LRS_ERR_UNSUPPORTED"]
LRS_OP_GAUSSIAN, LRS_OP_DFT2D_MASK = 0, 1
LRS_A_FP32, LRS_A_BF16, LRS_A_FP8_HI, LRS_A_FP8_HILO = 0, 1, 2, 3


class LrsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


LRS_REDUCER = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                               ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_float), ctypes.c_int32)


class lrs_options(ctypes.Structure):
    _fields_ = [("tau0", ctypes.c_int32), ("tau", ctypes.c_int32), ("T", ctypes.c_int32),
                ("c_eta", ctypes.c_double), ("rho_max", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("a_dtype", ctypes.c_int32),
                ("refine_every", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("power_iters", ctypes.c_int32), ("power_tol", ctypes.c_double),
                ("use_graph", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("seed", ctypes.c_uint64), ("profile", ctypes.c_int32),
                ("slab_mode", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("engine", ctypes.c_int32), ("inflight", ctypes.c_int32),
                ("task_kib", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("wait_ms", ctypes.c_int32), ("grad_block", ctypes.c_int32),
                ("reduce", LRS_REDUCER), ("reduce_ctx", ctypes.c_void_p),
                ("reduce_cap", ctypes.c_int32), ("test_withhold", ctypes.c_int32)]


class lrs_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("q", ctypes.c_int64),
                ("r", ctypes.c_int32), ("rho", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("opt", lrs_options), ("y", ctypes.c_void_p), ("A_or_mask", ctypes.c_void_p),
                ("mem_kind", ctypes.c_int32), ("U", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("S_idx", ctypes.c_void_p), ("S_val", ctypes.c_void_p),
                ("out_mem_kind", ctypes.c_int32), ("user", ctypes.c_void_p)]


class lrs_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("message", ctypes.c_char * 256),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("end_s", ctypes.c_double), ("footprint", ctypes.c_size_t),
                ("worker", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("admitted", ctypes.c_int64), ("group", ctypes.c_int64),
                ("group_size", ctypes.c_int32)]


LRS_RUNNER = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(lrs_request),
                              ctypes.c_int32, ctypes.c_int32)


class lrs_server_options(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("slots", ctypes.c_int32),
                ("sms", ctypes.c_int32), ("runner", LRS_RUNNER), ("runner_ctx", ctypes.c_void_p),
                ("batch", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p


def lib():
    """Load liblrs.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2311_03824_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "lrs_create": [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                           ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(lrs_options),
                           ctypes.POINTER(_P)],
            "lrs_set_measurements": [_P, _P, _P, ctypes.c_int32],
            "lrs_init": [_P],
            "lrs_estimate_rank": [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_int32), _P,
                                  ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)],
            "lrs_iterate": [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)],
            "lrs_solve": [_P],
            "lrs_iterate_batch": [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32],
            "lrs_get": [_P, _P, _P, _P, _P, ctypes.c_int32],
            "lrs_get_x": [_P, _P, ctypes.c_int32],
            "lrs_set_state": [_P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_double,
                              ctypes.c_int32],
            "lrs_get_progress": [_P, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_int32)],
            "lrs_set_reference": [_P, _P, ctypes.c_int32],
            "lrs_phase_times": [_P, ctypes.POINTER(ctypes.c_double)],
            "lrs_describe": [_P, ctypes.c_char_p, ctypes.c_int32],
            "lrs_sweep_trace": [_P, _P, ctypes.c_int64],
            "lrs_orthonormalize": [_P, _P, ctypes.c_int64, ctypes.c_int32, _P],
            "lrs_autotune": [_P, ctypes.c_int32, ctypes.c_char_p, ctypes.c_int32],
            "lrs_orthonormalize_noalloc": [_P, _P, ctypes.c_int64, ctypes.c_int32, _P],
            "lrs_destroy": [_P],
            "lrs_server_create": [ctypes.POINTER(lrs_server_options), ctypes.POINTER(_P)],
            "lrs_server_submit": [_P, ctypes.POINTER(lrs_request), ctypes.POINTER(ctypes.c_uint64)],
            "lrs_server_wait": [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(lrs_result)],
            "lrs_server_destroy": [_P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.lrs_last_error.argtypes = []
        L.lrs_last_error.restype = ctypes.c_char_p
        L.lrs_noalloc_last_error.argtypes = []
        L.lrs_noalloc_last_error.restype = ctypes.c_char_p
        L.lrs_server_last_error.argtypes = []
        L.lrs_server_last_error.restype = ctypes.c_char_p
        L.lrs_request_footprint.argtypes = [ctypes.POINTER(lrs_request)]
        L.lrs_request_footprint.restype = ctypes.c_size_t
        _lib = L
    return _lib


def _check(st):
    if st != LRS_OK:
        raise LrsError(st, lib().lrs_last_error().decode())


def _ptr(x):
    """(pointer, mem_kind) of a numpy array (host, 0) or torch CUDA tensor (1)."""
    if x is None:
        return None, 0
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return x.ctypes.data_as(_P), 0
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        if not x.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return _P(x.data_ptr()), 1
    raise TypeError(f"unsupported buffer type {type(x)}")


def _same_kind(*bufs):
    kinds = {_ptr(b)[1] for b in bufs if b is not None}
    if len(kinds) > 1:
        raise ValueError("mix of host and device buffers in one call")
    return kinds.pop() if kinds else 0


def make_options(**kw):
    o = lrs_options()
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream           # torch.cuda.Stream
        setattr(o, k, v if v is not None else 0)
    return o


# ----------------------------------------------------------- C-name calls --

def lrs_create(n, m, q, r, rho, kind=LRS_OP_GAUSSIAN, options=None):
    h = _P()
    _check(lib().lrs_create(n, m, q, r, rho, kind,
                            ctypes.byref(options) if options is not None else None,
                            ctypes.byref(h)))
    return h


def lrs_set_measurements(h, y, A_or_mask):
    mk = _same_kind(y, A_or_mask)
    _check(lib().lrs_set_measurements(h, _ptr(y)[0], _ptr(A_or_mask)[0], mk))


def lrs_init(h):
    _check(lib().lrs_init(h))


def lrs_estimate_rank(h, energy=0.65):
    """(r, singular values used) of the automatic rank (lrs_estimate_rank)."""
    r, nsv = ctypes.c_int32(0), ctypes.c_int32(0)
    sv = np.zeros(64, np.float64)
    _check(lib().lrs_estimate_rank(h, energy, ctypes.byref(r), sv.ctypes.data, len(sv),
                                   ctypes.byref(nsv)))
    return int(r.value), sv[:nsv.value].copy()


def lrs_iterate(h, iters, err_log=None):
    buf = None
    if err_log is not None:
        buf = (ctypes.c_double * iters)()
    _check(lib().lrs_iterate(h, iters, buf))
    if err_log is not None:
        err_log[:] = list(buf)


def lrs_iterate_batch(handles, iters):
    """lrs_iterate_batch over the handles (lrs_t values)."""
    arr = (_P * len(handles))(*handles)
    _check(lib().lrs_iterate_batch(arr, len(handles), iters))


def lrs_solve(h):
    _check(lib().lrs_solve(h))


def lrs_get(h, U=None, B=None, S_idx=None, S_val=None):
    mk = _same_kind(U, B, S_idx, S_val)
    _check(lib().lrs_get(h, _ptr(U)[0], _ptr(B)[0], _ptr(S_idx)[0], _ptr(S_val)[0], mk))


def lrs_get_x(h, X):
    """X = U B + S of the current iterate (n x q column-major: a (q, n) array)."""
    _check(lib().lrs_get_x(h, _ptr(X)[0], _ptr(X)[1]))


def lrs_set_state(h, U, B, S_idx, S_val, t, eta):
    mk = _same_kind(U, B, S_idx, S_val)
    _check(lib().lrs_set_state(h, _ptr(U)[0], _ptr(B)[0], _ptr(S_idx)[0], _ptr(S_val)[0],
                               t, eta, mk))


def lrs_get_progress(h):
    eta = ctypes.c_double()
    t = ctypes.c_int32()
    _check(lib().lrs_get_progress(h, ctypes.byref(eta), ctypes.byref(t)))
    return eta.value, t.value


def lrs_set_reference(h, Xref):
    _check(lib().lrs_set_reference(h, _ptr(Xref)[0], _ptr(Xref)[1]))


def lrs_phase_times(h):
    out = (ctypes.c_double * 4)()
    _check(lib().lrs_phase_times(h, out))
    return {"sweep_ms": out[0], "grad_ms": out[1], "qr_ms": out[2], "iters": int(out[3])}


TRACE_PHASES = ["setup", "w_pass", "As_exchange", "proj_u", "col_pass", "Ag_exchange",
                "proj_norm", "hard_threshold", "final_As", "ls_residual", "final_col_pass",
                "output"]


TASK_PROF = ["wait_task", "w_tasks", "at_tasks", "wait_pieces", "step_w", "step_iht",
             "step_final", "producer_wait_ticket", "n_tasks", "n_steps", "iht_load", "iht_mu",
             "iht_ht", "iht_next", "iht_publish"]


def lrs_sweep_trace(h, q):
    out = np.zeros(q * len(TRACE_PHASES), np.uint64)
    _check(lib().lrs_sweep_trace(h, out.ctypes.data_as(_P), out.size))
    return out.reshape(q, len(TRACE_PHASES))


RES_PROF = ["load", "w_pass", "wait", "gram", "proj_at", "agg", "mu", "ht_local", "merge",
            "as_update", "final", "n_columns", "n_exchanges", "n_support_changes", "n_sweeps"]


def lrs_resident_profile(h):
    """Resident-engine counters (handle created with engine=3, profile=2)."""
    out = np.zeros(len(RES_PROF), np.uint64)
    _check(lib().lrs_sweep_trace(h, out.ctypes.data_as(_P), out.size))
    return dict(zip(RES_PROF, (int(v) for v in out)))


def lrs_task_profile(h):
    """Task-engine counters (handle created with engine=2, profile=2)."""
    out = np.zeros(len(TASK_PROF), np.uint64)
    _check(lib().lrs_sweep_trace(h, out.ctypes.data_as(_P), out.size))
    return dict(zip(TASK_PROF, (int(v) for v in out)))


FOURIER_PROF = ["setup_gram", "sparse_dft", "norms_updates", "fft", "hard_threshold", "final",
                "proj_solve", "proj_apply"]


def lrs_fourier_profile(h):
    """DFT sweep counters: thread-0 cycles of every CTA per phase (handle
    created with profile=2)."""
    out = np.zeros(len(FOURIER_PROF), np.uint64)
    _check(lib().lrs_sweep_trace(h, out.ctypes.data_as(_P), out.size))
    return dict(zip(FOURIER_PROF, (int(v) for v in out)))


def lrs_describe(h):
    buf = ctypes.create_string_buffer(512)
    _check(lib().lrs_describe(h, buf, 512))
    import json
    return json.loads(buf.value.decode())


def lrs_autotune(h, trial_iters=2):
    """Time candidate task-engine shapes from the current iterate; returns the
    trials and the chosen shape (cached for later handles of this shape)."""
    buf = ctypes.create_string_buffer(4096)
    _check(lib().lrs_autotune(h, trial_iters, buf, 4096))
    import json
    return json.loads(buf.value.decode())


def lrs_orthonormalize(Z, Q, stream=None):
    """Q = Cholesky-QR2 orthonormalisation of Z (torch CUDA float32, n x r)."""
    n, r = Z.shape
    st = None if stream is None else _P(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    _check(lib().lrs_orthonormalize(_P(Z.data_ptr()), _P(Q.data_ptr()), n, r, st))


def lrs_orthonormalize_noalloc(Z, Q, stream=None):
    """lrs_orthonormalize with no device allocation (fixed scratch; n <= 65536)."""
    n, r = Z.shape
    st = None if stream is None else _P(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    status = lib().lrs_orthonormalize_noalloc(_P(Z.data_ptr()), _P(Q.data_ptr()), n, r, st)
    if status != LRS_OK:
        raise LrsError(status, lib().lrs_noalloc_last_error().decode())


def _check_srv(st):
    if st != LRS_OK:
        raise LrsError(st, lib().lrs_server_last_error().decode())


def lrs_server_create(hbm_budget=0, slots=0, sms=0, runner=None, batch=0):
    """Native request server (lrs_server_*).  runner: None (the library's
    solver) or a Python callable (request, grid, worker) -> status used in
    its place; the ctypes callback object is kept on the returned handle's
    side by the caller (see serve.Server)."""
    o = lrs_server_options()
    o.hbm_budget = int(hbm_budget)
    o.slots = int(slots)
    o.sms = int(sms)
    o.batch = int(batch)
    cb = None
    if runner is not None:
        cb = LRS_RUNNER(lambda ctx, req, grid, worker: int(runner(req.contents, grid, worker)))
        o.runner = cb
    h = _P()
    _check_srv(lib().lrs_server_create(ctypes.byref(o), ctypes.byref(h)))
    return h, cb


def lrs_server_submit(srv, req):
    t = ctypes.c_uint64()
    _check_srv(lib().lrs_server_submit(srv, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def lrs_server_wait(srv, ticket, timeout_ms=-1):
    res = lrs_result()
    _check_srv(lib().lrs_server_wait(srv, ticket, timeout_ms, ctypes.byref(res)))
    return res


def lrs_server_destroy(srv):
    _check_srv(lib().lrs_server_destroy(srv))


def lrs_request_footprint(req):
    return int(lib().lrs_request_footprint(ctypes.byref(req)))


def lrs_destroy(h):
    _check(lib().lrs_destroy(h))


def lrs_last_error():
    return lib().lrs_last_error().decode()


# --------------------------------------------------------------- wrapper --

class Solver:
    """One problem.  Gaussian: A (q, m, n) float32, Y (q, m) float32.  DFT
    (kind=LRS_OP_DFT2D_MASK, nx=.., ny=..): masks (q, m) int32, Y (q, m)
    complex64.  Rows of A / Y / masks are the columns k of the problem."""

    def __init__(self, n, m, q, r, rho, kind=LRS_OP_GAUSSIAN, **opts):
        self.n, self.m, self.q, self.r = n, m, q, r
        self.kind = kind
        self.dtype = np.complex64 if kind == LRS_OP_DFT2D_MASK else np.float32
        self.opts = make_options(**opts)
        self.rho = self.opts.rho_max or rho
        self.h = lrs_create(n, m, q, r, rho, kind, self.opts)

    def set_measurements(self, Y, A):
        lrs_set_measurements(self.h, Y, A)

    def init(self):
        lrs_init(self.h)

    def estimate_rank(self, energy=0.65):
        """Automatic rank from L0 (before init): (r, singular values used)."""
        return lrs_estimate_rank(self.h, energy)

    def iterate(self, iters=1, err_log=None):
        lrs_iterate(self.h, iters, err_log)

    def get(self):
        """Host copies: U (n, r), B (r, q), S_idx (q, rho), S_val (q, rho)."""
        U = np.empty((self.r, self.n), self.dtype)      # n x r column-major
        B = np.empty((self.q, self.r), self.dtype)      # r x q column-major
        S_idx = np.empty((self.q, max(self.rho, 1)), np.int32)
        S_val = np.empty((self.q, max(self.rho, 1)), self.dtype)
        lrs_get(self.h, U, B, S_idx if self.rho else None, S_val if self.rho else None)
        return U.T.copy(), B.T.copy(), S_idx[:, :self.rho], S_val[:, :self.rho]

    def X(self):
        """X = U B + S (n, q), assembled by the library (lrs_get_x)."""
        X = np.empty((self.q, self.n), self.dtype)      # n x q column-major
        lrs_get_x(self.h, X)
        return X.T.copy()

    def progress(self):
        return lrs_get_progress(self.h)

    def close(self):
        if self.h:
            lrs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
