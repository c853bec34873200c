"""ctypes declarations of include/vl.h and thin handle wrappers."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))

COV_EXPONENTIAL, COV_MATERN15 = 0, 1
LIK_BERNOULLI_LOGIT, LIK_POISSON_LOG, LIK_GAMMA_LOG = 0, 1, 2
PREC_VADU, PREC_LVA, PREC_LRAC = 0, 1, 2
FP64, FP32_REFINE = 0, 1
OP_A, OP_PINV, OP_B, OP_BT, OP_BINV, OP_BTINV, OP_SIGMA, OP_A2 = range(8)
SOLVE_AUTO, SOLVE_SHARED, SOLVE_CLUSTER, SOLVE_GRID, SOLVE_GRID_ALL, SOLVE_TILE = range(6)

_STATUS = {0: "VL_OK", 1: "VL_ERR_INVALID_ARG", 2: "VL_ERR_OOM", 3: "VL_ERR_NOT_SPD",
           4: "VL_ERR_NOT_CONVERGED", 5: "VL_ERR_TIMEOUT", 6: "VL_ERR_CUDA", 7: "VL_ERR_STATE"}


class VLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("precond", C.c_int), ("t", C.c_int), ("k", C.c_int),
                ("s", C.c_int), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int),
                ("newton_tol", C.c_double), ("newton_max_iter", C.c_int), ("nugget", C.c_double),
                ("seed", C.c_uint64), ("lik_shape", C.c_double), ("newton_eta_max", C.c_double)]

    @classmethod
    def make(cls, **kw) -> "Opts":
        o = cls()
        library().vl_opts_default(C.byref(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise AttributeError(k)
            setattr(o, k, v)
        return o


class Stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("cg_calls", C.c_int), ("cg_iters_max", C.c_int),
                ("cg_iters_total", C.c_int), ("cg_relres_max", C.c_double), ("refine_steps", C.c_int),
                ("true_relres_max", C.c_double), ("slq_mean", C.c_double), ("slq_stderr", C.c_double),
                ("logdet", C.c_double), ("ms_total", C.c_double), ("probe_relres_max", C.c_double),
                ("probe_refine_steps", C.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_live = []   # weak references to open handles, closed children-first at exit


def _track(obj):
    import weakref
    _live.append(weakref.ref(obj))


def _close_all():
    for kind in (State, Batch, Factor, Context):
        for r in list(_live):
            o = r()
            if isinstance(o, kind):
                try:
                    o.close()
                except Exception:
                    pass


import atexit  # noqa: E402

atexit.register(_close_all)


def lib_path() -> str:
    return os.path.join(_HERE, "_build", "libvl.so")


def library():
    """The loaded libvl; raises if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = lib_path()
    if not os.path.exists(p):
        raise ImportError(f"libvl.so not found at {p}: run paper_2310_12000_gb300.build.build() "
                          "(the CUDA library is required; there is no CPU fallback)")
    L = C.CDLL(p)
    vp, i64, i32, d, st = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_int
    sig = {
        "vl_version": (C.c_char_p, []),
        "vl_opts_default": (None, [vp]),
        "vl_ctx_create": (st, [i32, vp, vp, C.c_size_t, vp]),
        "vl_ctx_destroy": (None, [vp]),
        "vl_last_error": (C.c_char_p, [vp]),
        "vl_ctx_synchronize": (st, [vp]),
        "vl_ctx_mem": (st, [vp, vp, vp]),
        "vl_ctx_set_solve_form": (st, [vp, i32]),
        "vl_ctx_set_wait_limit": (st, [vp, C.c_longlong]),
        "vl_ctx_set_autotune": (st, [vp, i32]),
        "vl_tune_report": (C.c_size_t, [vp, C.c_size_t]),
        "vl_tune_reset": (None, []),
        "vl_ctx_wait_probe": (st, [vp]),
        "vl_profile_enable": (st, [vp, i32]),
        "vl_profile_read": (st, [vp, C.c_char_p, i32, vp, vp, i32]),
        "vl_profile_trace": (st, [vp, C.c_char_p, i32, vp, i32, vp, vp, vp]),
        "vl_build_factor": (st, [vp, vp, i64, vp, i32, d, d, i32, vp, vp]),
        "vl_factor_refit": (st, [vp, d, d, vp]),
        "vl_factor_export": (st, [vp, vp, vp, vp, vp, vp]),
        "vl_factor_info": (st, [vp, vp, vp, vp, vp]),
        "vl_factor_destroy": (None, [vp]),
        "vl_find_mode": (st, [vp, i32, vp, vp, vp, vp, vp]),
        "vl_state_destroy": (None, [vp]),
        "vl_state_stats": (st, [vp, vp]),
        "vl_log_marglik": (st, [vp, vp, vp, vp, vp]),
        "vl_slq_gammas": (st, [vp, vp, i32]),
        "vl_pred_var": (st, [vp, vp, i64, vp, vp, vp, vp, vp]),
        "vl_knn_prev": (st, [vp, vp, i64, i32, vp]),
        "vl_knn_cross": (st, [vp, vp, i64, vp, i64, i32, vp]),
        "vl_apply": (st, [vp, i32, vp, i32, vp, vp]),
        "vl_pcg_solve": (st, [vp, vp, i32, vp, vp, i32, vp, vp, vp, vp]),
        "vl_apply_A_noalloc": (st, [vp, vp, i32, vp]),
        "vl_lrac_export": (st, [vp, i32, vp, vp]),
        "vl_lml_grad": (st, [vp, vp, vp, vp, vp]),
        "vl_pred_var_lanczos": (st, [vp, vp, i64, vp, i32, i32, vp, vp, vp]),
        "vl_batch_create": (st, [vp, i32, vp, vp]),
        "vl_batch_refresh": (st, [vp]),
        "vl_batch_info": (st, [vp, vp, vp, vp]),
        "vl_batch_find_mode": (st, [vp, vp, vp, vp, vp, vp, vp]),
        "vl_batch_log_marglik": (st, [vp, vp, vp, vp, vp]),
        "vl_batch_gammas": (st, [vp, vp, i32]),
        "vl_batch_pred_var": (st, [vp, vp, vp, vp, vp, vp, vp]),
        "vl_batch_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(a, dtype) -> int:
    """Pointer of a contiguous numpy array or torch tensor of the given dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
        return a.ctypes.data
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        tmap = {np.float64: torch.float64, np.int32: torch.int32}
        if a.dtype != tmap[np.dtype(dtype).type] or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {np.dtype(dtype)} tensor")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _host(a, dtype):
    if a is None or not isinstance(a, np.ndarray):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def _numel(a):
    if isinstance(a, np.ndarray):
        return a.size
    numel = getattr(a, "numel", None)         # torch tensors
    return int(numel()) if callable(numel) else None


def _need(a, count: int, name: str):
    """The C ABI takes bare pointers: refuse an array that does not hold exactly `count`
    elements before the library reads or writes past its end."""
    k = None if a is None else _numel(a)
    if k is not None and k != count:
        raise ValueError(f"{name}: expected {count} elements, got {k}")


def _check_permutation(order, n: int):
    """order must be a permutation of 0..n-1 (the library gathers through it unchecked).
    Host arrays are checked here; a device tensor is the caller's responsibility."""
    if order is None:
        return
    if not isinstance(order, np.ndarray):
        if getattr(order, "is_cuda", False):
            return
        order = np.asarray(order)
    o = order.astype(np.int64, copy=False).ravel()
    if o.size and (o.min() < 0 or o.max() >= n or np.bincount(o, minlength=n).max() != 1):
        raise ValueError("order: expected a permutation of 0..n-1")


def _points(a, name: str) -> int:
    """Number of rows of an (n, 2) location array (numpy or torch)."""
    shape = tuple(getattr(a, "shape", ()))
    if len(shape) != 2 or shape[1] != 2:
        raise ValueError(f"{name}: expected an (n, 2) array of locations, got shape {shape}")
    return int(shape[0])


class Context:
    """A libvl context on one CUDA device: a stream and a workspace.

    ws_bytes sizes the workspace every handle of this context sub-allocates from.
    With torch available the workspace is a torch CUDA buffer owned by this object
    (PyTorch as the device-memory provider); otherwise the library allocates it."""

    def __init__(self, device: int = 0, ws_bytes: int = 1 << 30, stream=None, use_torch: bool = True):
        self.lib = library()
        self._ws = None
        ws_ptr = None
        sptr = None
        if use_torch:
            try:
                import torch
                if torch.cuda.is_available():
                    self._ws = torch.empty(int(ws_bytes), dtype=torch.uint8, device=f"cuda:{device}")
                    ws_ptr = self._ws.data_ptr()
                    if stream is None:
                        stream = torch.cuda.current_stream(device)
                    sptr = stream.cuda_stream
            except ImportError:
                pass
        if stream is not None and sptr is None:
            sptr = int(stream)
        h = C.c_void_p()
        s = self.lib.vl_ctx_create(device, sptr, ws_ptr, int(ws_bytes), C.byref(h))
        if s != 0:
            raise VLError(s, "vl_ctx_create failed")
        self.h = h
        self.device = device
        _track(self)

    def check(self, status: int):
        if status != 0:
            raise VLError(status, self.lib.vl_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            for r in list(_live):          # children first: they reference this context
                o = r()
                if o is not None and o is not self and getattr(o, "ctx", None) is self:
                    o.close()
            self.lib.vl_ctx_destroy(self.h)
            self.h = None
            self._ws = None                # every handle is gone: the workspace can go back to PyTorch

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        self.check(self.lib.vl_ctx_synchronize(self.h))

    def mem(self):
        a, b = C.c_size_t(), C.c_size_t()
        self.check(self.lib.vl_ctx_mem(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_solve_form(self, form: int):
        """Force the triangular-solve form (SOLVE_AUTO, SOLVE_SHARED, SOLVE_CLUSTER,
        SOLVE_GRID, SOLVE_GRID_ALL, SOLVE_TILE) of every later solve on this context; SOLVE_AUTO restores
        the per-solve choice."""
        self.check(self.lib.vl_ctx_set_solve_form(self.h, int(form)))

    def set_wait_limit(self, cycles: int):
        """Cycle limit of every bounded device-side wait on this context (0: the default,
        about 2 s); a wait that runs out makes the call fail with VL_ERR_TIMEOUT."""
        self.check(self.lib.vl_ctx_set_wait_limit(self.h, int(cycles)))

    def set_autotune(self, enable: bool):
        """Tune result-neutral launch parameters at first use (default on)."""
        self.check(self.lib.vl_ctx_set_autotune(self.h, 1 if enable else 0))

    def wait_probe(self):
        """One bounded wait on a flag nothing sets: raises VLError(VL_ERR_TIMEOUT)."""
        self.check(self.lib.vl_ctx_wait_probe(self.h))

    def profile(self, enable=True):
        """enable: False/0 off, True/1 kernel timing, 2 also per-level solve traces."""
        self.check(self.lib.vl_profile_enable(self.h, int(enable)))

    def profile_trace(self, cls: str, t: int):
        cap = 1 << 16
        buf = np.zeros(cap, np.int64)
        ln, lh, lt = C.c_int(), C.c_int(), C.c_int()
        self.check(self.lib.vl_profile_trace(self.h, cls.encode(), t, buf.ctypes.data, cap, C.byref(ln),
                                             C.byref(lh), C.byref(lt)))
        return buf[:ln.value].copy(), lh.value, lt.value

    def profile_read(self, cls: str, t: int = 0, reset: bool = False):
        ms, cnt = C.c_double(), C.c_int64()
        self.check(self.lib.vl_profile_read(self.h, cls.encode(), t, C.byref(ms), C.byref(cnt), 1 if reset else 0))
        return ms.value, cnt.value

    # ---------------------------------------------------------------- calls
    def build_factor(self, locs, order, cov: int, sigma2: float, rho: float, m: int,
                     opts: Opts | None = None) -> "Factor":
        locs = _host(locs, np.float64)
        order = _host(order, np.int32)
        n = _points(locs, "locs")
        _need(order, n, "order")
        _check_permutation(order, n)
        opts = opts or Opts.make()
        h = C.c_void_p()
        self.check(self.lib.vl_build_factor(self.h, _ptr(locs, np.float64), n, _ptr(order, np.int32), cov,
                                            sigma2, rho, m, C.byref(opts), C.byref(h)))
        return Factor(self, h, n, m)

    def knn_prev(self, locs, m: int, out=None):
        locs = _host(locs, np.float64)
        n = _points(locs, "locs")
        out = np.empty((n, m), np.int32) if out is None else out
        _need(out, n * m, "out")
        self.check(self.lib.vl_knn_prev(self.h, _ptr(locs, np.float64), n, m, _ptr(out, np.int32)))
        return out

    def knn_cross(self, train, test, m: int, out=None):
        train, test = _host(train, np.float64), _host(test, np.float64)
        _points(train, "train")
        n_p = _points(test, "test")
        out = np.empty((n_p, m), np.int32) if out is None else out
        _need(out, n_p * m, "out")
        self.check(self.lib.vl_knn_cross(self.h, _ptr(train, np.float64), train.shape[0], _ptr(test, np.float64),
                                         test.shape[0], m, _ptr(out, np.int32)))
        return out


class Factor:
    def __init__(self, ctx: Context, h, n: int, m: int):
        self.ctx, self.h, self.n, self.m = ctx, h, n, m
        _track(self)

    def close(self):
        if self.h:
            self.ctx.lib.vl_factor_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refit(self, sigma2: float, rho: float, opts: Opts | None = None):
        opts = opts or Opts.make()
        self.ctx.check(self.ctx.lib.vl_factor_refit(self.h, sigma2, rho, C.byref(opts)))

    def info(self):
        n, m, a, b = C.c_int64(), C.c_int(), C.c_int(), C.c_int()
        self.ctx.check(self.ctx.lib.vl_factor_info(self.h, C.byref(n), C.byref(m), C.byref(a), C.byref(b)))
        return {"n": n.value, "m": m.value, "nlev_fwd": a.value, "nlev_bwd": b.value}

    def export(self):
        n, m = self.n, self.m
        N = np.empty((n, m), np.int32)
        A = np.empty((n, m))
        D = np.empty(n)
        lf = np.empty(n, np.int32)
        lb = np.empty(n, np.int32)
        self.ctx.check(self.ctx.lib.vl_factor_export(self.h, N.ctypes.data, A.ctypes.data, D.ctypes.data,
                                                     lf.ctypes.data, lb.ctypes.data))
        return {"N": N, "A": A, "D": D, "lev_fwd": lf, "lev_bwd": lb}

    def lrac_export(self, k: int, with_L: bool = True):
        """(pivots as Vecchia indices, L_k as n x k in caller order or None)."""
        piv = np.empty(k, np.int32)
        L = np.empty((self.n, k)) if with_L else None
        self.ctx.check(self.ctx.lib.vl_lrac_export(self.h, k, piv.ctypes.data, _ptr(L, np.float64)))
        return piv, L

    def find_mode(self, lik: int, y, F=None, opts: Opts | None = None, mode_out=None, allow_unconverged=False):
        y = _host(y, np.float64)
        F = _host(F, np.float64)
        _need(y, self.n, "y")
        _need(F, self.n, "F")
        _need(mode_out, self.n, "mode_out")
        opts = opts or Opts.make()
        mode = np.empty(self.n) if mode_out is None else mode_out
        h = C.c_void_p()
        s = self.ctx.lib.vl_find_mode(self.h, lik, _ptr(y, np.float64), _ptr(F, np.float64), C.byref(opts),
                                      _ptr(mode, np.float64), C.byref(h))
        if s != 0 and not (allow_unconverged and s == 4 and h.value):
            if h.value:
                self.ctx.lib.vl_state_destroy(h)
            self.ctx.check(s)
        return State(self, h, mode)


class State:
    def __init__(self, fac: Factor, h, mode):
        self.fac, self.ctx, self.h, self.mode = fac, fac.ctx, h, mode
        _track(self)

    def close(self):
        if self.h:
            self.ctx.lib.vl_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def mode_stats(self) -> dict:
        st = Stats()
        self.ctx.check(self.ctx.lib.vl_state_stats(self.h, C.byref(st)))
        return st.as_dict()

    def log_marglik(self, opts: Opts | None = None, with_stats: bool = False):
        opts = opts or Opts.make()
        lml, ld = C.c_double(), C.c_double()
        st = Stats()
        self.ctx.check(self.ctx.lib.vl_log_marglik(self.h, C.byref(opts), C.byref(lml), C.byref(ld), C.byref(st)))
        return (lml.value, st.as_dict()) if with_stats else lml.value

    def lml_grad(self, opts: Opts | None = None, with_stats: bool = False, offset: bool = False):
        """(dL/dsigma2, dL/drange) by stochastic trace estimation on the SLQ probes; with
        offset=True also dL/dF (caller order) as a second result."""
        opts = opts or Opts.make()
        g = np.zeros(2)
        dF = np.zeros(self.fac.n) if offset else None
        st = Stats()
        self.ctx.check(self.ctx.lib.vl_lml_grad(self.h, C.byref(opts), g.ctypes.data, _ptr(dF, np.float64),
                                                C.byref(st)))
        out = (g, dF) if offset else g
        return (out, st.as_dict()) if with_stats else out

    def slq_gammas(self, t: int):
        g = np.empty(t)
        self.ctx.check(self.ctx.lib.vl_slq_gammas(self.h, g.ctypes.data, t))
        return g

    def pred_var(self, test_locs, Fp=None, opts: Opts | None = None, mean_out=None, var_out=None,
                 with_stats: bool = False):
        test_locs = _host(test_locs, np.float64)
        Fp = _host(Fp, np.float64)
        opts = opts or Opts.make()
        n_p = _points(test_locs, "test_locs")
        _need(Fp, n_p, "Fp")
        _need(mean_out, n_p, "mean_out")
        _need(var_out, n_p, "var_out")
        mean = np.empty(n_p) if mean_out is None else mean_out
        var = np.empty(n_p) if var_out is None else var_out
        st = Stats()
        self.ctx.check(self.ctx.lib.vl_pred_var(self.h, _ptr(test_locs, np.float64), n_p, _ptr(Fp, np.float64),
                                                C.byref(opts), _ptr(mean, np.float64), _ptr(var, np.float64),
                                                C.byref(st)))
        return (mean, var, st.as_dict()) if with_stats else (mean, var)

    def pred_var_lanczos(self, test_locs, k: int, Fp=None, precond_l: int = 1, with_stats: bool = False):
        """Predictive mean and variance with rank-k preconditioned Lanczos variances (P_L1)."""
        test_locs = _host(test_locs, np.float64)
        Fp = _host(Fp, np.float64)
        n_p = _points(test_locs, "test_locs")
        _need(Fp, n_p, "Fp")
        mean = np.empty(n_p)
        var = np.empty(n_p)
        st = Stats()
        self.ctx.check(self.ctx.lib.vl_pred_var_lanczos(self.h, _ptr(test_locs, np.float64), n_p,
                                                        _ptr(Fp, np.float64), int(k), int(precond_l),
                                                        mean.ctypes.data, var.ctypes.data, C.byref(st)))
        return (mean, var, st.as_dict()) if with_stats else (mean, var)

    def apply(self, op: int, X, opts: Opts | None = None):
        X = np.ascontiguousarray(X, dtype=np.float64)
        if X.ndim == 1:
            X = X[:, None]
        if X.ndim != 2 or X.shape[0] != self.fac.n:
            raise ValueError(f"X: expected {self.fac.n} rows, got shape {X.shape}")
        opts = opts or Opts.make()
        Y = np.empty_like(X)
        self.ctx.check(self.ctx.lib.vl_apply(self.h, op, X.ctypes.data, X.shape[1], C.byref(opts), Y.ctypes.data))
        return Y

    def apply_A_noalloc(self, X_dev, Y_dev):
        """(W + B^T D^{-1} B) X for device tensors X, Y (n x t float64) without
        allocating; see vl_apply_A_noalloc in include/vl.h."""
        t = 1 if len(X_dev.shape) == 1 else X_dev.shape[1]
        _need(X_dev, self.fac.n * t, "X")
        _need(Y_dev, self.fac.n * t, "Y")
        self.ctx.check(self.ctx.lib.vl_apply_A_noalloc(self.h, _ptr(X_dev, np.float64), t, _ptr(Y_dev, np.float64)))
        return Y_dev

    def pcg_solve(self, RHS, opts: Opts | None = None, lmax: int = 0):
        R = np.ascontiguousarray(RHS, dtype=np.float64)
        if R.ndim == 1:
            R = R[:, None]
        if R.ndim != 2 or R.shape[0] != self.fac.n:
            raise ValueError(f"RHS: expected {self.fac.n} rows, got shape {R.shape}")
        t = R.shape[1]
        opts = opts or Opts.make()
        U = np.empty_like(R)
        Td = np.zeros((t, max(lmax, 1)))
        To = np.zeros((t, max(lmax, 1)))
        it = np.zeros(t, np.int32)
        rel = np.zeros(t)
        self.ctx.check(self.ctx.lib.vl_pcg_solve(self.h, R.ctypes.data, t, C.byref(opts), U.ctypes.data, lmax,
                                                 Td.ctypes.data if lmax else None, To.ctypes.data if lmax else None,
                                                 it.ctypes.data, rel.ctypes.data))
        return U, Td, To, it, rel


class Batch:
    """Independent problems merged into one block-diagonal system (vl_batch_* in include/vl.h):
    one launch of every kernel serves all problems, each following its own Newton iteration
    and PCG stopping rule. Vectors are lists, one array per problem in its caller order."""

    def __init__(self, ctx: Context, factors):
        self.ctx, self.factors = ctx, list(factors)
        arr = (C.c_void_p * len(self.factors))(*[f.h.value for f in self.factors])
        h = C.c_void_p()
        ctx.check(ctx.lib.vl_batch_create(ctx.h, len(self.factors), arr, C.byref(h)))
        self.h = h
        self.sizes = [f.n for f in self.factors]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        _track(self)

    def close(self):
        if self.h:
            self.ctx.lib.vl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refresh(self):
        """Copy the members' factor values again (after Factor.refit of any of them)."""
        self.ctx.check(self.ctx.lib.vl_batch_refresh(self.h))

    def info(self):
        n, a, b = C.c_int64(), C.c_int(), C.c_int()
        self.ctx.check(self.ctx.lib.vl_batch_info(self.h, C.byref(n), C.byref(a), C.byref(b)))
        return {"n": n.value, "nlev_fwd": a.value, "nlev_bwd": b.value}

    def _split(self, flat):
        return [flat[self.offsets[k]:self.offsets[k + 1]] for k in range(len(self.sizes))]

    def find_mode(self, liks, ys, Fs=None, opts: Opts | None = None, with_stats: bool = False):
        """Modes of every problem (a list of arrays); raises if any problem does not converge."""
        P = len(self.sizes)
        if len(ys) != P or len(liks) != P or (Fs is not None and len(Fs) != P):
            raise ValueError(f"expected {P} problems")
        for k, y in enumerate(ys):
            _need(y, self.sizes[k], f"y[{k}]")
        y = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float64) for v in ys]))
        F = None
        if Fs is not None:
            for k, v in enumerate(Fs):
                _need(v, self.sizes[k], f"F[{k}]")
            F = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float64) for v in Fs]))
        lik = np.ascontiguousarray(np.asarray(liks, np.int32))
        opts = opts or Opts.make()
        mode = np.empty(int(self.offsets[-1]))
        st = (Stats * P)()
        self.ctx.check(self.ctx.lib.vl_batch_find_mode(self.h, lik.ctypes.data, y.ctypes.data, _ptr(F, np.float64),
                                                       C.byref(opts), mode.ctypes.data, st))
        modes = self._split(mode)
        return (modes, [x.as_dict() for x in st]) if with_stats else modes

    def log_marglik(self, opts: Opts | None = None, with_stats: bool = False):
        """L^VLA of every problem at its mode (an array of nprob values)."""
        P = len(self.sizes)
        opts = opts or Opts.make()
        lml = np.empty(P)
        ld = np.empty(P)
        st = (Stats * P)()
        self.ctx.check(self.ctx.lib.vl_batch_log_marglik(self.h, C.byref(opts), lml.ctypes.data, ld.ctypes.data, st))
        return (lml, [x.as_dict() for x in st]) if with_stats else lml

    def pred_var(self, test_locs, Fps=None, opts: Opts | None = None):
        """Predictive means and simulated variances per problem (lists of arrays): test_locs is a
        list of (np_k, 2) arrays, Fps a list of offsets or None."""
        P = len(self.sizes)
        if len(test_locs) != P or (Fps is not None and len(Fps) != P):
            raise ValueError(f"expected {P} problems")
        counts = np.array([_points(np.asarray(q, np.float64), f"test_locs[{k}]") for k, q in enumerate(test_locs)],
                          np.int64)
        q = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float64).reshape(-1, 2) for v in test_locs]))
        Fp = None
        if Fps is not None:
            for k, v in enumerate(Fps):
                _need(v, int(counts[k]), f"Fp[{k}]")
            Fp = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float64) for v in Fps]))
        opts = opts or Opts.make()
        tot = int(counts.sum())
        mean = np.empty(tot)
        var = np.empty(tot)
        self.ctx.check(self.ctx.lib.vl_batch_pred_var(self.h, counts.ctypes.data, q.ctypes.data, _ptr(Fp, np.float64),
                                                      C.byref(opts), mean.ctypes.data, var.ctypes.data))
        off = np.concatenate([[0], np.cumsum(counts)])
        return ([mean[off[k]:off[k + 1]] for k in range(P)], [var[off[k]:off[k + 1]] for k in range(P)])

    def gammas(self, t: int):
        g = np.empty(len(self.sizes) * t)
        self.ctx.check(self.ctx.lib.vl_batch_gammas(self.h, g.ctypes.data, t))
        return g.reshape(len(self.sizes), t)


def tune_reset():
    """Forget the launch tuner's choices (vl_tune_reset)."""
    library().vl_tune_reset()


def tune_report() -> list:
    """The launch tuner's choices so far (vl_tune_report)."""
    import json
    L = library()
    need = L.vl_tune_report(None, 0)
    buf = C.create_string_buffer(int(need))
    L.vl_tune_report(buf, need)
    return json.loads(buf.value.decode() or "[]")
