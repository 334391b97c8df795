"""Thin ctypes binding of the BLWS C ABI (``include/blws.h``).

Argument marshalling only: every step of the path runs in the CUDA library
``_lib/libblws.so``.  There is no fallback: if the library is missing the
calls raise.  Arrays are torch tensors on the GPU holding FP64 data in
column-major (LAPACK) order; ``colmajor(x)`` makes such a tensor from any
(m, n) tensor, and results come back as column-major views of shape (m, n).
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libblws.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ENONFINITE, ETIMEOUT, ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
PREC_FP64, PREC_MIXED, PREC_FP64_TC = 0, 1, 2

# every symbol include/blws.h declares
EXPORTS = ("blws_config_default", "blws_create", "blws_destroy", "blws_status_str",
           "blws_last_error", "blws_launch_count", "blws_graph_stats", "blws_tune_count", "blws_apply", "blws_apply_noalloc",
           "blws_svt", "blws_evd", "rpca_params_default", "rpca_solve", "mc_params_default", "mc_solve",
           "blws_server_config_default", "blws_server_create", "blws_request_bytes",
           "blws_server_submit", "blws_server_wait", "blws_server_stats_get", "blws_server_destroy",
           "blws_csc_mirror", "blws_gemm", "blws_wait_probe", "blws_timing_start", "blws_timing_stop",
           "blws_timing_records")


class BlwsConfig(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("k_cold", ctypes.c_int), ("precision", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("device", ctypes.c_int), ("start", ctypes.c_int),
                ("warm", ctypes.c_int), ("grid_sms", ctypes.c_int), ("graphs", ctypes.c_int),
                ("tune", ctypes.c_int), ("guard", ctypes.c_double)]


class BlwsOp(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("W", ctypes.c_void_p),
                ("ldw", ctypes.c_int), ("nnz", ctypes.c_int), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("val", ctypes.c_void_p), ("rl", ctypes.c_int),
                ("Ul", ctypes.c_void_p), ("sl", ctypes.c_void_p), ("Vl", ctypes.c_void_p),
                ("colptr", ctypes.c_void_p), ("rowidx", ctypes.c_void_p), ("perm", ctypes.c_void_p)]


class RpcaParams(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("rho", ctypes.c_double), ("mu0", ctypes.c_double), ("mu_bar_ratio", ctypes.c_double),
                ("sv0", ctypes.c_int), ("trace", ctypes.POINTER(ctypes.c_double)),
                ("trace_len", ctypes.c_int), ("mixed_tol", ctypes.c_double)]


class RpcaInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rank", ctypes.c_int), ("nnzE", ctypes.c_int64),
                ("residual", ctypes.c_double), ("norm_two", ctypes.c_double),
                ("status", ctypes.c_int), ("mixed_iters", ctypes.c_int), ("restarts", ctypes.c_int)]


class McParams(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("tau", ctypes.c_double), ("delta", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("incr", ctypes.c_int),
                ("eta", ctypes.c_double), ("tau_min_rel", ctypes.c_double),
                ("xtol", ctypes.c_double)]


class McInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rank", ctypes.c_int), ("residual", ctypes.c_double),
                ("norm_two", ctypes.c_double), ("status", ctypes.c_int), ("restarts", ctypes.c_int)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int), ("hbm_budget", ctypes.c_size_t), ("cfg", BlwsConfig)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("D", ctypes.c_void_p), ("m", ctypes.c_int), ("n", ctypes.c_int),
                ("ld", ctypes.c_int), ("rpca", RpcaParams), ("A", ctypes.c_void_p), ("E", ctypes.c_void_p),
                ("nnz", ctypes.c_int), ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p),
                ("vals", ctypes.c_void_p), ("mc", McParams), ("max_rank", ctypes.c_int),
                ("U", ctypes.c_void_p), ("theta", ctypes.c_void_p), ("V", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("rpca", RpcaInfo), ("mc", McInfo)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("budget", ctypes.c_size_t), ("in_use", ctypes.c_size_t),
                ("peak_in_use", ctypes.c_size_t), ("peak_running", ctypes.c_int)]


REQ_RPCA, REQ_MC = 0, 1

_lib = None


def load():
    """Open the library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("BLWS CUDA library not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.blws_config_default.argtypes = [ctypes.POINTER(BlwsConfig)]
    lib.blws_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(BlwsConfig)]
    lib.blws_destroy.argtypes = [vp]
    lib.blws_status_str.argtypes = [ci]
    lib.blws_status_str.restype = ctypes.c_char_p
    lib.blws_last_error.argtypes = [vp]
    lib.blws_last_error.restype = ctypes.c_char_p
    lib.blws_svt.argtypes = [vp, ctypes.POINTER(BlwsOp), cd, ci, vp, vp, ci, vp, ci, vp, vp, vp,
                             ctypes.POINTER(ci), vp]
    lib.blws_evd.argtypes = [vp, vp, ci, ci, cd, ci, vp, ci, vp, ci, vp, vp, ctypes.POINTER(ci), vp]
    lib.blws_apply.argtypes = [vp, ctypes.POINTER(BlwsOp), vp, ci, ci, vp, ci, vp]
    lib.blws_apply_noalloc.argtypes = [vp, ci, ci, ci, vp, ci, ci, vp, ci, vp]
    lib.rpca_params_default.argtypes = [ctypes.POINTER(RpcaParams)]
    lib.rpca_solve.argtypes = [vp, vp, ci, ci, ci, ctypes.POINTER(RpcaParams), vp, vp,
                               ctypes.POINTER(RpcaInfo), vp]
    lib.mc_params_default.argtypes = [ctypes.POINTER(McParams)]
    lib.mc_solve.argtypes = [vp, ci, ci, ci, vp, vp, vp, ctypes.POINTER(McParams), ci, vp, vp, vp,
                             ctypes.POINTER(McInfo), vp]
    lib.blws_launch_count.argtypes = [vp]
    lib.blws_graph_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    lib.blws_graph_stats.restype = ctypes.c_int
    lib.blws_server_config_default.argtypes = [ctypes.POINTER(ServerConfig)]
    lib.blws_server_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ServerConfig)]
    lib.blws_request_bytes.argtypes = [ctypes.POINTER(Request), ci]
    lib.blws_server_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    lib.blws_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result)]
    lib.blws_server_stats_get.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.blws_server_destroy.argtypes = [vp]
    lib.blws_csc_mirror.argtypes = [vp, ci, ci, ci, vp, vp, vp, vp, vp, vp]
    lib.blws_gemm.argtypes = [vp, ci, ci, ci, ci, ci, cd, vp, ci, vp, ci, cd, vp, ci, ci, vp]
    lib.blws_wait_probe.argtypes = [vp, ctypes.c_uint, vp]
    lib.blws_timing_start.argtypes = [vp]
    lib.blws_timing_stop.argtypes = [vp, ctypes.POINTER(cd), ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(cd)]
    lib.blws_timing_records.argtypes = [vp, ctypes.c_size_t, ctypes.POINTER(cd), ctypes.POINTER(cd),
                                        ctypes.POINTER(ctypes.c_int)]
    for f in EXPORTS:
        if f not in ("blws_status_str", "blws_last_error"):
            getattr(lib, f).restype = ci
    lib.blws_launch_count.restype = ctypes.c_uint64
    lib.blws_tune_count.argtypes = []
    lib.blws_tune_count.restype = ctypes.c_size_t
    lib.blws_request_bytes.restype = ctypes.c_size_t
    lib.blws_timing_records.restype = ctypes.c_size_t
    _lib = lib
    return lib


class BlwsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (load().blws_status_str(status).decode(), status, msg))
        self.status = status


def _torch():
    import torch
    return torch


def colmajor(x):
    """A column-major FP64 CUDA copy of the (m, n) tensor x (view of shape (m, n))."""
    torch = _torch()
    x = x.to(device="cuda", dtype=torch.float64) if x.device.type != "cuda" or x.dtype != torch.float64 else x
    return x.t().contiguous().t()


def empty_colmajor(m, n, device="cuda"):
    torch = _torch()
    return torch.empty((n, m), dtype=torch.float64, device=device).t()


def _check_colmajor(x, m, n, name):
    torch = _torch()
    if x.dtype != torch.float64 or x.device.type != "cuda":
        raise ValueError("%s must be a float64 CUDA tensor" % name)
    if tuple(x.shape) != (m, n) or (n > 1 and x.stride(1) != m) or (m > 1 and x.stride(0) != 1):
        raise ValueError("%s must be a column-major (%d, %d) tensor" % (name, m, n))


def _ptr(x):
    return ctypes.c_void_p(0 if x is None else x.data_ptr())


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def apply_noalloc(W, X, P, stream=None):
    """P = [W X_v; W^T X_u] through blws_apply_noalloc (no context, no
    allocation; P must be a preallocated column-major (m+n, b) tensor).
    Returns the status code."""
    m, n = W.shape
    b = X.shape[1]
    _check_colmajor(W, m, n, "W")
    _check_colmajor(X, m + n, b, "X")
    _check_colmajor(P, m + n, b, "P")
    return load().blws_apply_noalloc(_ptr(W), m, n, m, _ptr(X), m + n, b, _ptr(P), m + n,
                                     _stream(stream))


class Context:
    """Owns a blws_ctx (workspace, generator state) bound to one device."""

    def __init__(self, k=3, k_cold=4, seed=0x5EED, device=0, precision=0, start=0, warm=1,
                 grid_sms=0, graphs=1, tune=0, guard=0.0):
        lib = load()
        cfg = BlwsConfig()
        lib.blws_config_default(ctypes.byref(cfg))
        cfg.k, cfg.k_cold, cfg.seed, cfg.device = k, k_cold, seed, device
        cfg.precision, cfg.start, cfg.warm, cfg.grid_sms = precision, start, warm, grid_sms
        cfg.graphs, cfg.tune, cfg.guard = graphs, tune, guard
        h = ctypes.c_void_p()
        st = lib.blws_create(ctypes.byref(h), ctypes.byref(cfg))
        if st != OK:
            raise BlwsError(st, "blws_create")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            load().blws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self):
        """Kernels launched through this context so far."""
        return int(load().blws_launch_count(self._h))

    @staticmethod
    def tune_count():
        """Size buckets the product autotuner holds in this process."""
        return int(load().blws_tune_count())

    def graph_stats(self):
        """(phases captured, phase replays) of this context's CUDA graphs."""
        c, r = ctypes.c_uint64(), ctypes.c_uint64()
        st = load().blws_graph_stats(self._h, ctypes.byref(c), ctypes.byref(r))
        if st != OK:
            raise BlwsError(st, "blws_graph_stats")
        return int(c.value), int(r.value)

    def _raise(self, st, what):
        raise BlwsError(st, "%s: %s" % (what, load().blws_last_error(self._h).decode()))

    # ------------------------------------------------------------------ SVT --
    def blws_evd(self, W, eps, r, U0=None, G=None, stream=None):
        """Partial EVD of a symmetric W (column-major (m, m) FP64 CUDA tensor)
        by block Lanczos warm-started from U0 (m, w).  Returns (U (m, r),
        lam (r,) decreasing, count = #{lam > eps})."""
        torch = _torch()
        m = W.shape[0]
        _check_colmajor(W, m, m, "W")
        w = 0 if U0 is None else U0.shape[1]
        if w:
            _check_colmajor(U0, m, w, "U0")
        g = 0 if G is None else G.shape[1]
        if g:
            _check_colmajor(G, m, g, "G")
        U = empty_colmajor(m, r)
        lam = torch.empty(r, dtype=torch.float64, device="cuda")
        cnt = ctypes.c_int(0)
        st = load().blws_evd(self._h, _ptr(W), m, m, float(eps), int(r), _ptr(U0), w, _ptr(G), g,
                             _ptr(U), _ptr(lam), ctypes.byref(cnt), _stream(stream))
        if st != OK:
            self._raise(st, "blws_evd")
        return U, lam, cnt.value

    def blws_svt(self, W, eps, r, U0=None, V0=None, G=None, stream=None, sparse=None):
        """One SVT evaluation by BLWS.  W: column-major (m, n) FP64 CUDA tensor,
        or None with sparse=(m, n, rowptr, colidx, val[, Ul, sl, Vl]).
        Returns (U (m, r), V (n, r), sigma (r,), count)."""
        torch = _torch()
        op = BlwsOp()
        if W is not None:
            m, n = W.shape
            _check_colmajor(W, m, n, "W")
            op.m, op.n, op.W, op.ldw = m, n, W.data_ptr(), m
        else:
            m, n, rowptr, colidx, val = sparse[:5]
            op.m, op.n, op.W, op.ldw = m, n, None, m
            op.nnz, op.rowptr, op.colidx, op.val = int(val.numel()), rowptr.data_ptr(), colidx.data_ptr(), val.data_ptr()
            if len(sparse) > 5:
                Ul, sl, Vl = sparse[5:8]
                op.rl, op.Ul, op.sl, op.Vl = int(sl.numel()), Ul.data_ptr(), sl.data_ptr(), Vl.data_ptr()
        w = 0 if U0 is None else U0.shape[1]
        if w:
            _check_colmajor(U0, m, w, "U0")
            _check_colmajor(V0, n, w, "V0")
        g = 0 if G is None else G.shape[1]
        if g:
            _check_colmajor(G, m + n, g, "G")
        U = empty_colmajor(m, r)
        V = empty_colmajor(n, r)
        sigma = torch.empty(r, dtype=torch.float64, device="cuda")
        cnt = ctypes.c_int(0)
        st = load().blws_svt(self._h, ctypes.byref(op), float(eps), int(r), _ptr(U0), _ptr(V0), w,
                             _ptr(G), g, _ptr(U), _ptr(V), _ptr(sigma), ctypes.byref(cnt),
                             _stream(stream))
        if st != OK:
            self._raise(st, "blws_svt")
        return U, V, sigma, cnt.value

    def apply(self, W, X, P=None, stream=None):
        """P = [W X_v; W^T X_u] (one product with the augmented matrix).
        W column-major (m, n); X column-major (m+n, b).  Does not synchronise."""
        m, n = W.shape
        _check_colmajor(W, m, n, "W")
        b = X.shape[1]
        _check_colmajor(X, m + n, b, "X")
        P = empty_colmajor(m + n, b) if P is None else P
        op = BlwsOp()
        op.m, op.n, op.W, op.ldw = m, n, W.data_ptr(), m
        st = load().blws_apply(self._h, ctypes.byref(op), _ptr(X), m + n, b, _ptr(P), m + n,
                               _stream(stream))
        if st != OK:
            self._raise(st, "blws_apply")
        return P

    def gemm(self, A, B, C, alpha=1.0, beta=0.0, ta=False, tb=False, sym=False, stream=None):
        """C = alpha op(A) op(B) + beta C with the context's block-product
        arithmetic (blws_gemm).  A, B, C column-major FP64 CUDA tensors; op(X)
        is X^T when ta / tb.  Synchronises.  Returns C."""
        M, N = C.shape
        K = A.shape[0] if ta else A.shape[1]
        _check_colmajor(A, A.shape[0], A.shape[1], "A")
        _check_colmajor(B, B.shape[0], B.shape[1], "B")
        _check_colmajor(C, M, N, "C")
        if (A.shape[1] if ta else A.shape[0]) != M or (B.shape[1] if tb else B.shape[0]) != K or \
                (B.shape[0] if tb else B.shape[1]) != N:
            raise ValueError("gemm: shapes do not match")
        st = load().blws_gemm(self._h, int(ta), int(tb), M, N, K, float(alpha), _ptr(A), A.shape[0],
                              _ptr(B), B.shape[0], float(beta), _ptr(C), M, int(sym), _stream(stream))
        if st != OK:
            self._raise(st, "blws_gemm")
        return C

    def timing_start(self):
        """Start timing the products with the augmented matrix (step a2)."""
        st = load().blws_timing_start(self._h)
        if st != OK:
            self._raise(st, "blws_timing_start")

    def timing_stop(self):
        """Stop timing; returns (device ms, products, multiply-adds)."""
        ms, n, work = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_double()
        st = load().blws_timing_stop(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(work))
        if st != OK:
            self._raise(st, "blws_timing_stop")
        return ms.value, int(n.value), work.value

    # kernel kinds of the timed products
    KIND_FP64, KIND_TF32, KIND_DIGITS = 0, 1, 2

    def timing_records(self):
        """Per-product (device ms, multiply-adds, kernel kind) of the last timing_stop."""
        k = int(load().blws_timing_records(self._h, 0, None, None, None))
        ms, w = (ctypes.c_double * max(k, 1))(), (ctypes.c_double * max(k, 1))()
        kd = (ctypes.c_int * max(k, 1))()
        load().blws_timing_records(self._h, k, ms, w, kd)
        return [(ms[i], w[i], kd[i]) for i in range(k)]

    def wait_probe(self, polls=256, stream=None):
        """Run the bounded-wait self-test; returns its status (ETIMEOUT expected)."""
        return load().blws_wait_probe(self._h, int(polls), _stream(stream))

    def csc_mirror(self, m, n, rowptr, colidx, stream=None):
        """(colptr, rowidx, perm): the column-major mirror of a CSR pattern (int32 tensors)."""
        torch = _torch()
        nnz = int(colidx.numel())
        colptr = torch.empty(n + 1, dtype=torch.int32, device="cuda")
        rowidx = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        perm = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        st = load().blws_csc_mirror(self._h, m, n, nnz, rowptr.data_ptr(), colidx.data_ptr(),
                                    colptr.data_ptr(), rowidx.data_ptr(), perm.data_ptr(), _stream(stream))
        if st != OK:
            self._raise(st, "blws_csc_mirror")
        return colptr, rowidx, perm

    def apply_sparse(self, m, n, rowptr, colidx, vals, X, P=None, stream=None, mirror=None):
        """P = [S X_v; S^T X_u] for the CSR matrix S (int32 rowptr/colidx, FP64 vals):
        the matrix-completion product.  mirror: (colptr, rowidx, perm) from
        csc_mirror, else the call builds one."""
        b = X.shape[1]
        _check_colmajor(X, m + n, b, "X")
        P = empty_colmajor(m + n, b) if P is None else P
        op = BlwsOp()
        op.m, op.n, op.W, op.ldw = m, n, None, m
        op.nnz, op.rowptr, op.colidx, op.val = int(vals.numel()), rowptr.data_ptr(), colidx.data_ptr(), vals.data_ptr()
        if mirror is not None:
            op.colptr, op.rowidx, op.perm = (t.data_ptr() for t in mirror)
        st = load().blws_apply(self._h, ctypes.byref(op), _ptr(X), m + n, b, _ptr(P), m + n,
                               _stream(stream))
        if st != OK:
            self._raise(st, "blws_apply")
        return P

    # ----------------------------------------------------------------- RPCA --
    def rpca_solve(self, D, lam=0.0, tol=1e-7, max_iter=1000, rho=1.5, sv0=10, mu0=0.0,
                   mu_bar_ratio=1e7, A=None, E=None, stream=None, allow_noconv=False, trace=0,
                   mixed_tol=1e-5):
        """Robust PCA by inexact ALM with BLWS.  D: column-major (m, n) FP64.
        Returns (A, E, info dict); with trace=T the dict also holds the first T
        iterations' (residual, count above eps, predicted rank)."""
        m, n = D.shape
        _check_colmajor(D, m, n, "D")
        A = empty_colmajor(m, n) if A is None else A
        E = empty_colmajor(m, n) if E is None else E
        p = RpcaParams()
        load().rpca_params_default(ctypes.byref(p))
        p.lambda_, p.tol, p.max_iter, p.rho, p.sv0, p.mu0, p.mu_bar_ratio = lam, tol, max_iter, rho, sv0, mu0, mu_bar_ratio
        p.mixed_tol = mixed_tol
        tr = None
        if trace:
            tr = (ctypes.c_double * (3 * trace))()
            p.trace, p.trace_len = ctypes.cast(tr, ctypes.POINTER(ctypes.c_double)), trace
        info = RpcaInfo()
        st = load().rpca_solve(self._h, _ptr(D), m, n, m, ctypes.byref(p), _ptr(A), _ptr(E),
                               ctypes.byref(info), _stream(stream))
        if st != OK and not (st == ENOCONV and allow_noconv):
            self._raise(st, "rpca_solve")
        out = {"iters": info.iters, "rank": info.rank, "nnzE": info.nnzE,
               "residual": info.residual, "norm_two": info.norm_two, "status": info.status,
               "mixed_iters": info.mixed_iters, "restarts": info.restarts}
        if tr is not None:
            k = min(trace, info.iters)
            out["trace"] = [(tr[3 * i], int(tr[3 * i + 1]), int(tr[3 * i + 2])) for i in range(k)]
        return A, E, out

    # ------------------------------------------------------------------- MC --
    def mc_solve(self, m, n, rowptr, colidx, vals, max_rank, variant=0, tau=0.0, delta=0.0,
                 tol=1e-4, max_iter=500, incr=5, eta=0.25, tau_min_rel=1e-4, xtol=1e-3,
                 stream=None, allow_noconv=False):
        """Matrix completion (variant 0: SVT, 1: proximal/FPC).  rowptr/colidx
        int32 CUDA tensors (CSR), vals FP64.  Returns (U, theta, V, info)."""
        torch = _torch()
        U = empty_colmajor(m, max_rank)
        V = empty_colmajor(n, max_rank)
        th = torch.empty(max_rank, dtype=torch.float64, device="cuda")
        p = McParams()
        load().mc_params_default(ctypes.byref(p))
        p.variant, p.tau, p.delta, p.tol, p.max_iter, p.incr = variant, tau, delta, tol, max_iter, incr
        p.eta, p.tau_min_rel, p.xtol = eta, tau_min_rel, xtol
        info = McInfo()
        st = load().mc_solve(self._h, m, n, int(vals.numel()), _ptr(rowptr), _ptr(colidx), _ptr(vals),
                             ctypes.byref(p), int(max_rank), _ptr(U), _ptr(th), _ptr(V),
                             ctypes.byref(info), _stream(stream))
        if st != OK and not (st == ENOCONV and allow_noconv):
            self._raise(st, "mc_solve")
        r = info.rank
        return U[:, :r], th[:r], V[:, :r], {"iters": info.iters, "rank": r,
                                            "residual": info.residual, "norm_two": info.norm_two,
                                            "status": info.status, "restarts": info.restarts}


class Server:
    """The library's request server (include/blws.h, "Serving and batching"):
    `workers` concurrent solves, each on its own context and stream, admitted
    in arrival order while their estimated device memory fits `hbm_budget`
    (0: 70% of the free memory).  Tensors handed to submit_* are kept alive
    here until wait() returns their result."""

    def __init__(self, workers=8, hbm_budget=0, k=3, k_cold=4, seed=0x5EED, device=0, precision=0,
                 grid_sms=0, graphs=1, tune=0, guard=0.0):
        lib = load()
        cfg = ServerConfig()
        lib.blws_server_config_default(ctypes.byref(cfg))
        cfg.workers, cfg.hbm_budget = workers, hbm_budget
        cfg.cfg.k, cfg.cfg.k_cold, cfg.cfg.seed, cfg.cfg.device, cfg.cfg.precision = k, k_cold, seed, device, precision
        cfg.cfg.grid_sms, cfg.cfg.graphs, cfg.cfg.tune, cfg.cfg.guard = grid_sms, graphs, tune, guard
        h = ctypes.c_void_p()
        st = lib.blws_server_create(ctypes.byref(h), ctypes.byref(cfg))
        if st != OK:
            raise BlwsError(st, "blws_server_create")
        self._h = h
        self._keep = {}
        self.precision = precision

    def close(self):
        if getattr(self, "_h", None):
            load().blws_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _submit(self, req, keep):
        t = ctypes.c_uint64(0)
        st = load().blws_server_submit(self._h, ctypes.byref(req), ctypes.byref(t))
        if st != OK:
            raise BlwsError(st, "blws_server_submit")
        self._keep[t.value] = keep
        return t.value

    def submit_rpca(self, D, tol=1e-7, max_iter=1000, sv0=10, lam=0.0, mixed_tol=1e-5):
        """Queue a Robust PCA solve of the column-major (m, n) FP64 CUDA tensor D."""
        m, n = D.shape
        _check_colmajor(D, m, n, "D")
        A, E = empty_colmajor(m, n), empty_colmajor(m, n)
        req = Request()
        req.kind, req.D, req.m, req.n, req.ld = REQ_RPCA, D.data_ptr(), m, n, m
        load().rpca_params_default(ctypes.byref(req.rpca))
        req.rpca.tol, req.rpca.max_iter, req.rpca.sv0, req.rpca.lambda_ = tol, max_iter, sv0, lam
        req.rpca.mixed_tol = mixed_tol
        req.A, req.E = A.data_ptr(), E.data_ptr()
        return self._submit(req, ("rpca", D, A, E))

    def submit_mc(self, m, n, rowptr, colidx, vals, max_rank, variant=0, tol=1e-4, max_iter=500):
        """Queue a matrix completion solve (CSR int32 pattern, FP64 values, CUDA tensors)."""
        torch = _torch()
        U, V = empty_colmajor(m, max_rank), empty_colmajor(n, max_rank)
        th = torch.empty(max_rank, dtype=torch.float64, device="cuda")
        req = Request()
        req.kind, req.m, req.n = REQ_MC, m, n
        req.nnz, req.rowptr, req.colidx, req.vals = int(vals.numel()), rowptr.data_ptr(), colidx.data_ptr(), vals.data_ptr()
        load().mc_params_default(ctypes.byref(req.mc))
        req.mc.variant, req.mc.tol, req.mc.max_iter = variant, tol, max_iter
        req.max_rank, req.U, req.theta, req.V = max_rank, U.data_ptr(), th.data_ptr(), V.data_ptr()
        return self._submit(req, ("mc", rowptr, colidx, vals, U, th, V))

    def wait(self, ticket):
        """Block until the ticket's solve finished.  RPCA: (A, E, info); MC: (U, theta, V, info)."""
        res = Result()
        st = load().blws_server_wait(self._h, ctypes.c_uint64(ticket), ctypes.byref(res))
        if st != OK:
            raise BlwsError(st, "blws_server_wait")
        keep = self._keep.pop(ticket)
        info = {"status": res.status, "queue_ms": res.queue_ms, "run_ms": res.run_ms}
        if keep[0] == "rpca":
            r = res.rpca
            info.update(iters=r.iters, rank=r.rank, nnzE=r.nnzE, residual=r.residual, mixed_iters=r.mixed_iters)
            return keep[2], keep[3], info
        r = res.mc
        info.update(iters=r.iters, rank=r.rank, residual=r.residual)
        return keep[4][:, :r.rank], keep[5][:r.rank], keep[6][:, :r.rank], info

    def stats(self):
        s = ServerStats()
        load().blws_server_stats_get(self._h, ctypes.byref(s))
        return {"submitted": s.submitted, "completed": s.completed, "budget": s.budget,
                "in_use": s.in_use, "peak_in_use": s.peak_in_use, "peak_running": s.peak_running}
