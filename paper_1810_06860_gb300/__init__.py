"""GB300 fast-SVT matrix completion (Feng, Yu & Li, arXiv 1810.06860).

Python binding of libmc.so: the same entry points as ``include/mc.h`` with
argument marshalling only -- every step of the computation runs in the CUDA
kernels of the library.  Arrays may be NumPy arrays (host) or CUDA torch
tensors (device); outputs are NumPy arrays unless ``device=True``.

The library needs a CUDA GPU; there is no CPU path.  When torch is available
its caching allocator is handed to the library as the device allocator.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native
from ._native import McIterInfo, McParams

__all__ = ["Handle", "Server", "McError", "params", "omega", "eig_sym", "gram", "load", "lib_path"]

load = _native.load
lib_path = _native.lib_path


class McError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(st: int, what: str):
    if st != _native.MC_OK:
        lib = load()
        raise McError(st, f"{what}: {lib.mc_status_str(st).decode()}: {lib.mc_last_error().decode()}")


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, keepalive) for a host NumPy array or a torch tensor (CUDA or host)."""
    if a is None:
        return None, None
    if _is_torch(a):
        if not a.is_contiguous():
            a = a.contiguous()
        return C.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), arr


def _out(shape, dtype, device: bool):
    if device:
        import torch

        tdt = {np.float32: torch.float32, np.uint32: torch.int32, np.int64: torch.int64}[dtype]
        return torch.empty(shape, dtype=tdt, device="cuda")
    return np.empty(shape, dtype=dtype)


def params(**kw) -> McParams:
    """Alg. 6 parameters with the paper's defaults (mc_params_default)."""
    p = McParams()
    load().mc_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _info(i: McIterInfo) -> dict:
    return {f: getattr(i, f) for f, _ in McIterInfo._fields_ if f != "reserved"}


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self):
        import torch

        self._torch = torch
        self.alloc_cb = _native.ALLOC_FN(self._alloc)
        self.free_cb = _native.FREE_FN(self._free)
        self.struct = _native.McAllocator(None, self.alloc_cb, self.free_cb)

    def _alloc(self, ctx, nbytes, stream):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(self, ctx, ptr, nbytes, stream):
        self._torch.cuda.caching_allocator_delete(int(ptr))


class Handle:
    """One completion problem: the observed entries P_Phi(M) in CSR form."""

    def __init__(self, m: int, n: int, row_ptr, col, val, stream=None, torch_alloc: bool = True):
        lib = load()
        self._lib = lib
        self.m, self.n = int(m), int(n)
        rp, k1 = _ptr(row_ptr, np.int64)
        ci, k2 = _ptr(col, np.int32)
        vv, k3 = _ptr(val, np.float32)
        self.nnz = int(len(col))
        self._alloc = None
        alloc_p = None
        if torch_alloc:
            try:
                import torch

                if torch.cuda.is_available():
                    self._alloc = _TorchAllocator()
                    alloc_p = C.byref(self._alloc.struct)
            except ImportError:
                pass
        st_ptr = None
        if stream is not None:
            st_ptr = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        h = C.c_void_p()
        _check(lib.mc_create(C.byref(h), self.m, self.n, self.nnz, rp, ci, vv, st_ptr, alloc_p), "mc_create")
        self._h = h

    @classmethod
    def from_observed(cls, obs, **kw):
        return cls(obs.m, obs.n, obs.row_ptr, obs.col, obs.val, **kw)

    @classmethod
    def from_coo(cls, m: int, n: int, rows, cols, vals, stream=None):
        """Observed entries as coordinates in any order (mc_create_coo)."""
        self = cls.__new__(cls)
        lib = load()
        self._lib = lib
        self.m, self.n = int(m), int(n)
        r, k1 = _ptr(rows, np.int64)
        c, k2 = _ptr(cols, np.int32)
        v, k3 = _ptr(vals, np.float32)
        self.nnz = int(len(cols))
        self._alloc = None
        st_ptr = None
        if stream is not None:
            st_ptr = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        h = C.c_void_p()
        _check(lib.mc_create_coo(C.byref(h), self.m, self.n, self.nnz, r, c, v, st_ptr, None), "mc_create_coo")
        self._h = h
        return self

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_precision(self, precision: int):
        """0: plain float32; 1: bf16 panels in the Krylov products (mixed form)."""
        _check(self._lib.mc_set_precision(self._h, int(precision)), "mc_set_precision")

    # ---- randomized SVDs -------------------------------------------------
    def _rsvd(self, fn, k, s, p, seed, call_id, device):
        U = _out((self.m, k), np.float32, device)
        S = _out((k,), np.float32, device)
        V = _out((self.n, k), np.float32, device)
        ko = C.c_int(0)
        pu, _ = _ptr(U, np.float32)
        ps, _ = _ptr(S, np.float32)
        pv, _ = _ptr(V, np.float32)
        _check(fn(self._h, k, s, p, seed, call_id, pu, ps, pv, C.byref(ko)), fn.__name__)
        kk = ko.value
        # the library writes m x k_out and n x k_out densely at the buffers' start
        return (U.reshape(-1)[:self.m * kk].reshape(self.m, kk), S[:kk],
                V.reshape(-1)[:self.n * kk].reshape(self.n, kk))

    def rsvd_bki(self, k: int, s: int = 10, p: int = 3, seed: int = 0, call_id: int = 0, device: bool = False):
        """Alg. 5: rank-k SVD (U, S descending, V) of the current iterate."""
        return self._rsvd(self._lib.mc_rsvd_bki, k, s, p, seed, call_id, device)

    def rsvd_pi(self, k: int, s: int = 10, p: int = 3, seed: int = 0, call_id: int = 0, device: bool = False):
        """Alg. 4: rank-k SVD of the current iterate by power iteration."""
        return self._rsvd(self._lib.mc_rsvd_pi, k, s, p, seed, call_id, device)

    # ---- SVT ---------------------------------------------------------------
    def rsvd_basic(self, k: int, s: int = 10, p: int = 3, seed: int = 0, call_id: int = 0, device: bool = False):
        """Basic rSVD with power iteration (Alg. 1): (U, S, V)."""
        return self._rsvd(self._lib.mc_rsvd_basic, k, s, p, seed, call_id, device)

    def svt_step(self, prm: McParams | None = None) -> dict:
        info = McIterInfo()
        _check(self._lib.mc_svt_step(self._h, C.byref(prm) if prm is not None else None, C.byref(info)),
               "mc_svt_step")
        return _info(info)

    def svt_reset(self):
        _check(self._lib.mc_svt_reset(self._h), "mc_svt_reset")

    def svt_solve(self, prm: McParams) -> dict:
        info = McIterInfo()
        st = self._lib.mc_svt_solve(self._h, C.byref(prm), C.byref(info))
        if st not in (_native.MC_OK, _native.MC_ENOTCONVERGED):
            _check(st, "mc_svt_solve")
        return _info(info)

    def factors(self, device: bool = False):
        r = C.c_int(0)
        _check(self._lib.mc_svt_factors(self._h, 0, None, None, None, C.byref(r)), "mc_svt_factors")
        r = r.value
        Us = _out((self.m, r), np.float32, device)
        V = _out((self.n, r), np.float32, device)
        sg = _out((r,), np.float32, device)
        pu, _ = _ptr(Us, np.float32)
        pv, _ = _ptr(V, np.float32)
        ps, _ = _ptr(sg, np.float32)
        rr = C.c_int(0)
        _check(self._lib.mc_svt_factors(self._h, r, pu, pv, ps, C.byref(rr)), "mc_svt_factors")
        return Us, V, sg

    def factors_into(self, Us, V, sigma) -> int:
        """Copy the factors of the current estimate into caller buffers of
        capacity max_r = Us.shape[1] columns (Us: m x r, V: n x r and sigma: r
        written densely at the start of each buffer); returns r."""
        cap = int(Us.shape[1])
        pu, _ = _ptr(Us, np.float32)
        pv, _ = _ptr(V, np.float32)
        ps, _ = _ptr(sigma, np.float32)
        r = C.c_int(0)
        _check(self._lib.mc_svt_factors(self._h, cap, pu, pv, ps, C.byref(r)), "mc_svt_factors")
        return r.value

    def sample(self, rows, cols, device: bool = False):
        rows = rows if _is_torch(rows) else np.ascontiguousarray(rows, np.int64)
        cols = cols if _is_torch(cols) else np.ascontiguousarray(cols, np.int64)
        out = _out((len(rows),), np.float32, device)
        pr, _ = _ptr(rows, np.int64)
        pc, _ = _ptr(cols, np.int64)
        po, _ = _ptr(out, np.float32)
        _check(self._lib.mc_svt_sample(self._h, len(rows), pr, pc, po), "mc_svt_sample")
        return out

    def get_values(self, device: bool = False):
        out = _out((self.nnz,), np.float32, device)
        po, _ = _ptr(out, np.float32)
        _check(self._lib.mc_get_values(self._h, po), "mc_get_values")
        return out

    def set_values(self, val):
        pv, keep = _ptr(val, np.float32)
        _check(self._lib.mc_set_values(self._h, pv), "mc_set_values")

    def join(self):
        """Order the handle's stream after its second stream (mc_join)."""
        _check(self._lib.mc_join(self._h), "mc_join")

    def timing_enable(self, on=True):
        """True / 1: every kernel class; 2: the sparse products only; False / 0: off."""
        mode = on if isinstance(on, int) and not isinstance(on, bool) else (1 if on else 0)
        _check(self._lib.mc_timing_enable(self._h, mode), "mc_timing_enable")

    def timing_read(self) -> dict:
        arr = (_native.McTiming * len(_native.TIMING_NAMES))()
        _check(self._lib.mc_timing_read(self._h, arr), "mc_timing_read")
        return {name: dict(ms=t.ms, bytes=t.bytes, flops=t.flops, launches=t.launches)
                for name, t in zip(_native.TIMING_NAMES, arr)}

    def gather_rate(self, k: int, trans: bool = False, reps: int = 10) -> float:
        """GB/s at which the sparse products' panel-row gathers alone run
        (mc_gather_rate)."""
        g = C.c_double(0.0)
        _check(self._lib.mc_gather_rate(self._h, 1 if trans else 0, k, reps, C.byref(g)), "mc_gather_rate")
        return g.value

    def spmm(self, X, trans: bool = False, device: bool = False):
        """Y X (trans=False, X: n x k) or Y^T X (trans=True, X: m x k)."""
        k = X.shape[1]
        out = _out((self.n if trans else self.m, k), np.float32, device)
        px, keep = _ptr(X, np.float32)
        po, _ = _ptr(out, np.float32)
        _check(self._lib.mc_spmm(self._h, 1 if trans else 0, k, px, po), "mc_spmm")
        return out


def omega(n: int, k: int, seed: int, call_id: int = 0, col0: int = 0, words: bool = False):
    """Philox Gaussian Omega (n x k, float32) and optionally the raw (x0, x1) words."""
    lib = load()
    out = np.empty((n, k), np.float32)
    w = np.empty((n, k, 2), np.uint32) if words else None
    _check(lib.mc_omega(n, k, seed, call_id, col0, out.ctypes.data_as(C.c_void_p),
                        w.ctypes.data_as(C.c_void_p) if words else None), "mc_omega")
    return (out, w) if words else out


def eig_sym(A, kw: int):
    """kw largest eigenpairs (descending) of the symmetric matrix A (float32)."""
    lib = load()
    A = np.ascontiguousarray(A, np.float32)
    K = A.shape[0]
    lam = np.empty(kw, np.float32)
    W = np.empty((K, kw), np.float32)
    _check(lib.mc_eig_sym(K, kw, A.ctypes.data_as(C.c_void_p), lam.ctypes.data_as(C.c_void_p),
                          W.ctypes.data_as(C.c_void_p)), "mc_eig_sym")
    return lam, W


def gram(X, tensor_cores: bool = False):
    """X^T X of a tall float32 matrix (SIMT, or tcgen05 tensor cores for K <= 256)."""
    lib = load()
    px, keep = _ptr(X, np.float32)
    G = np.empty((X.shape[1], X.shape[1]), np.float32)
    fn = lib.mc_gram_tc if tensor_cores else lib.mc_gram
    _check(fn(X.shape[0], X.shape[1], px, G.ctypes.data_as(C.c_void_p)), fn.__name__)
    return G


def panel_gemm(X, W, tensor_cores: bool = True):
    """Z = X W of a tall float32 X (R x K) and a small W (K x N) (mc_panel_gemm)."""
    lib = load()
    X = np.ascontiguousarray(X, np.float32)
    W = np.ascontiguousarray(W, np.float32)
    R, K = X.shape
    N = W.shape[1]
    Z = np.empty((R, N), np.float32)
    _check(lib.mc_panel_gemm(R, K, N, X.ctypes.data_as(C.c_void_p), W.ctypes.data_as(C.c_void_p),
                             Z.ctypes.data_as(C.c_void_p), 1 if tensor_cores else 0), "mc_panel_gemm")
    return Z


def panel_gram(X1, X2, tensor_cores: bool = True):
    """C = X1^T X2 of two tall float32 panels with the same row count (mc_panel_gram)."""
    lib = load()
    X1 = np.ascontiguousarray(X1, np.float32)
    X2 = np.ascontiguousarray(X2, np.float32)
    R, K1 = X1.shape
    K2 = X2.shape[1]
    Cm = np.empty((K1, K2), np.float32)
    _check(lib.mc_panel_gram(R, K1, K2, X1.ctypes.data_as(C.c_void_p), X2.ctypes.data_as(C.c_void_p),
                             Cm.ctypes.data_as(C.c_void_p), 1 if tensor_cores else 0), "mc_panel_gram")
    return Cm


def orth_block(X, Qp=None, stream=None):
    """Orthonormal basis of (I - Qp Qp^T) X for CUDA float32 tensors X (R x K)
    and Qp (R x cols), K and cols multiples of 4 (mc_orth_block).  X is
    overwritten; returns a new R x K tensor."""
    import torch

    lib = load()
    if X.dtype != torch.float32 or not X.is_cuda or not X.is_contiguous():
        raise McError(1, "orth_block: X must be a contiguous CUDA float32 tensor")
    R, K = X.shape
    out = torch.empty_like(X)
    cols, pq, ldq = 0, None, 0
    if Qp is not None and Qp.shape[1] > 0:
        if Qp.dtype != torch.float32 or not Qp.is_cuda or not Qp.is_contiguous() or Qp.shape[0] != R:
            raise McError(1, "orth_block: Qp must be a contiguous CUDA float32 tensor with R rows")
        cols, pq, ldq = Qp.shape[1], C.c_void_p(Qp.data_ptr()), Qp.shape[1]
    st = C.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    _check(lib.mc_orth_block(R, K, C.c_void_p(X.data_ptr()), K, pq, ldq, cols, C.c_void_p(out.data_ptr()), K, st),
           "mc_orth_block")
    return out


class Server:
    """Serving form: whole SVT solves of many jobs on one GPU (mc_server_*).

    Jobs are admitted in arrival order as slots and the device-memory budget
    allow; each runs on its own stream, so jobs overlap on the GPU."""

    def __init__(self, budget_bytes: int = 0, max_active: int = 8, device: int = 0, simulate: bool = False):
        self._lib = load()
        s = C.c_void_p()
        _check(self._lib.mc_server_create(C.byref(s), int(budget_bytes), int(max_active), int(device),
                                          1 if simulate else 0), "mc_server_create")
        self._s = s

    def close(self):
        if getattr(self, "_s", None):
            self._lib.mc_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, m: int, n: int, row_ptr, col, val, prm: McParams) -> int:
        rp = np.ascontiguousarray(row_ptr, np.int64)
        ci = np.ascontiguousarray(col, np.int32)
        vv = np.ascontiguousarray(val, np.float32)
        d = _native.McJobDesc(int(m), int(n), int(len(ci)), rp.ctypes.data, ci.ctypes.data, vv.ctypes.data, prm)
        jid = C.c_uint64(0)
        _check(self._lib.mc_submit(self._s, C.byref(d), C.byref(jid)), "mc_submit")
        return int(jid.value)

    def submit_observed(self, obs, prm: McParams) -> int:
        return self.submit(obs.m, obs.n, obs.row_ptr, obs.col, obs.val, prm)

    def poll(self, job_id: int, factors: bool = True):
        """None while the job is queued or running, else its result (a dict)."""
        res = _native.McResult()
        st = self._lib.mc_poll(self._s, C.c_uint64(job_id), C.byref(res))
        if st == _native.MC_PENDING:
            return None
        if st not in (_native.MC_OK, _native.MC_ECANCELLED):
            _check(st, "mc_poll")
        out = {f: getattr(res, f) for f, _ in _native.McResult._fields_ if f not in ("Us", "V", "sigma", "message")}
        out["message"] = (res.message or b"").decode(errors="replace")
        r = res.r
        if factors and r > 0 and res.Us:
            out["Us"] = np.ctypeslib.as_array(res.Us, shape=(res.m, r)).copy()
            out["V"] = np.ctypeslib.as_array(res.V, shape=(res.n, r)).copy()
            out["sigma"] = np.ctypeslib.as_array(res.sigma, shape=(r,)).copy()
        return out

    def wait(self, job_id: int, timeout_s: float = 3600.0):
        st = self._lib.mc_wait(self._s, C.c_uint64(job_id), float(timeout_s))
        _check(st, "mc_wait")
        return self.poll(job_id)

    def cancel(self, job_id: int):
        _check(self._lib.mc_cancel(self._s, C.c_uint64(job_id)), "mc_cancel")

    def release(self, job_id: int):
        _check(self._lib.mc_result_release(self._s, C.c_uint64(job_id)), "mc_result_release")

    def stats(self) -> dict:
        info = _native.McServerInfo()
        _check(self._lib.mc_server_stats(self._s, C.byref(info)), "mc_server_stats")
        return {f: getattr(info, f) for f, _ in _native.McServerInfo._fields_}

    def admit_order(self):
        n = self._lib.mc_server_admit_order(self._s, None, 0)
        buf = (C.c_uint64 * max(n, 1))()
        n = self._lib.mc_server_admit_order(self._s, buf, n)
        return [int(buf[i]) for i in range(n)]
