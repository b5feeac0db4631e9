"""Thin ctypes binding of libdcf.so (the C ABI of include/dcf.h).

The module-level functions carry the C names and only marshal arguments;
:class:`Solver` wraps a handle for convenience.  Host data are numpy arrays,
device data are torch CUDA tensors (their ``data_ptr()`` is passed with
``where=1``).  The library is loaded on first use; when it is missing the
call raises :class:`DcfError` -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB = None
_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdcf.so")

DCF_OK, DCF_EINVAL, DCF_ENOMEM, DCF_ECUDA, DCF_ENONFINITE, DCF_ETIMEOUT, DCF_ENOTCONV, \
    DCF_EPRIVATE, DCF_ESTATE = range(9)
STATUS_NAMES = {0: "DCF_OK", 1: "DCF_EINVAL", 2: "DCF_ENOMEM", 3: "DCF_ECUDA",
                4: "DCF_ENONFINITE", 5: "DCF_ETIMEOUT", 6: "DCF_ENOTCONV",
                7: "DCF_EPRIVATE", 8: "DCF_ESTATE"}


class DcfError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class dcf_params(C.Structure):
    _fields_ = [("m", C.c_int64), ("E", C.c_int), ("n_i", C.POINTER(C.c_int64)),
                ("r", C.c_int), ("rho", C.c_double), ("lambda_", C.c_double),
                ("max_iter", C.c_int), ("tol", C.c_double), ("u_mode", C.c_int),
                ("local_steps", C.c_int), ("eta0", C.c_double), ("seed", C.c_uint64),
                ("path", C.c_int)]


class dcf_problem(C.Structure):
    _fields_ = [("m", C.c_int64), ("E", C.c_int), ("n_i", C.POINTER(C.c_int64)),
                ("r", C.c_int), ("rho", C.c_double), ("lambda_", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_SIGS = {
    "dcf_set_allocator": (None, [ALLOC_FN, FREE_FN, C.c_void_p]),
    "dcf_create": (C.c_int, [C.POINTER(dcf_params), C.POINTER(C.c_void_p)]),
    "dcf_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dcf_get_path": (C.c_int, [C.c_void_p]),
    "dcf_kernels_per_iteration": (C.c_int, [C.c_void_p]),
    "dcf_load_blocks": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                  C.c_int, C.c_int]),
    "dcf_reload_blocks": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                    C.c_int]),
    "dcf_reload_blocks_async": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p),
                                          C.POINTER(C.c_int64), C.c_int]),
    "dcf_load_init": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p), C.c_int]),
    "dcf_step": (C.c_int, [C.c_void_p, C.c_int]),
    "dcf_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "dcf_get_factors": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p), C.c_int]),
    "dcf_get_LS": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "dcf_set_private": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "dcf_get_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                C.POINTER(C.c_int)]),
    "dcf_get_conditioning": (C.c_int, [C.c_void_p, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int)]),
    "dcf_set_truth": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "dcf_rel_err": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "dcf_singular_values": (C.c_int, [C.c_void_p, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "dcf_last_error": (C.c_char_p, [C.c_void_p]),
    "dcf_destroy": (None, [C.c_void_p]),
    "dcf_version": (C.c_char_p, []),
    "dcf_profile_phases": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int]),
    "dcf_profile_step": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "dcf_tc_selftest": (C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "dcf_unrolled_forward": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]),
    "dcf_unrolled_backward": (C.c_int, [C.c_void_p, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.c_void_p, C.POINTER(C.c_void_p), C.c_int]),
    "dcf_batch_create": (C.c_int, [C.POINTER(dcf_problem), C.c_int, C.c_int, C.c_double,
                                   C.c_uint64, C.POINTER(C.c_void_p)]),
    "dcf_batch_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dcf_batch_load": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p),
                                 C.POINTER(C.c_int64), C.c_int]),
    "dcf_batch_load_init": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_void_p),
                                      C.c_int]),
    "dcf_batch_tune": (C.c_int, [C.c_void_p, C.c_int, C.c_char_p, C.c_int]),
    "dcf_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "dcf_batch_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "dcf_batch_get_factors": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_void_p),
                                        C.c_int]),
    "dcf_batch_get_stats": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "dcf_batch_profile_step": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_int]),
    "dcf_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "dcf_batch_destroy": (None, [C.c_void_p]),
    "dcf_iterate_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_double,
                                      C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p]),
}


def lib():
    """Load libdcf.so (raises DcfError when it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise DcfError(DCF_ESTATE, f"{LIB_PATH} is missing; run paper_2207_11669_gb300.build")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def exported_symbols():
    return list(_SIGS)


# ---------------------------------------------------------------------------
# argument helpers
# ---------------------------------------------------------------------------
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr_where(x):
    """(pointer, where) for a numpy array (host) or a torch CUDA tensor (device)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0
    a = np.asarray(x)
    return C.c_void_p(a.ctypes.data), 0


def _check(h, status):
    if status != DCF_OK:
        msg = lib().dcf_last_error(h).decode() if h else ""
        raise DcfError(status, msg)


# ---------------------------------------------------------------------------
# C-named entry points (marshalling only)
# ---------------------------------------------------------------------------
_alloc_keep = []


def dcf_set_allocator(alloc=None, release=None):
    """Route the library's device allocations through Python callables
    ``alloc(nbytes) -> int`` and ``release(ptr)``; None restores cudaMalloc."""
    if alloc is None:
        lib().dcf_set_allocator(ALLOC_FN(), FREE_FN(), None)
        _alloc_keep.clear()
        return
    fa = ALLOC_FN(lambda n, ctx: alloc(int(n)))
    ff = FREE_FN(lambda p, ctx: release(int(p)))
    _alloc_keep[:] = [fa, ff]
    lib().dcf_set_allocator(fa, ff, None)


def use_torch_allocator():
    """Allocate the library's device buffers from torch's caching allocator."""
    import torch

    def alloc(n):
        try:
            return torch.cuda.caching_allocator_alloc(n)
        except RuntimeError:
            return 0

    def release(p):
        torch.cuda.caching_allocator_delete(p)

    dcf_set_allocator(alloc, release)


PATH_AUTO, PATH_GENERAL, PATH_FUSED, PATH_TC2, PATH_SMALL = 0, 1, 2, 3, 4


def dcf_create(m, n_i, r, rho, lam, max_iter=100, tol=1e-6, u_mode=0, local_steps=1,
               eta0=0.0, seed=0, path=PATH_AUTO):
    n_arr = (C.c_int64 * len(n_i))(*[int(x) for x in n_i])
    p = dcf_params(int(m), len(n_i), n_arr, int(r), float(rho), float(lam), int(max_iter),
                   float(tol), int(u_mode), int(local_steps), float(eta0), int(seed), int(path))
    h = C.c_void_p()
    st = lib().dcf_create(C.byref(p), C.byref(h))
    if st != DCF_OK:
        raise DcfError(st, "dcf_create rejected the parameters")
    return h


def dcf_kernels_per_iteration(h):
    return lib().dcf_kernels_per_iteration(h)


def dcf_get_path(h):
    return lib().dcf_get_path(h)


def dcf_set_stream(h, stream_ptr):
    _check(h, lib().dcf_set_stream(h, C.c_void_p(stream_ptr)))


def dcf_load_blocks(h, blocks, ld=None, borrow=False):
    ptrs, wheres = zip(*[_ptr_where(b) for b in blocks])
    where = wheres[0]
    arr = (C.c_void_p * len(ptrs))(*[p.value for p in ptrs])
    ld_arr = None if ld is None else (C.c_int64 * len(ld))(*[int(x) for x in ld])
    _check(h, lib().dcf_load_blocks(h, arr, ld_arr, where, 1 if borrow else 0))


def dcf_reload_blocks(h, blocks, ld=None):
    ptrs, wheres = zip(*[_ptr_where(b) for b in blocks])
    arr = (C.c_void_p * len(ptrs))(*[p.value for p in ptrs])
    ld_arr = None if ld is None else (C.c_int64 * len(ld))(*[int(x) for x in ld])
    _check(h, lib().dcf_reload_blocks(h, arr, ld_arr, wheres[0]))


def dcf_reload_blocks_async(h, blocks, ld=None):
    ptrs, wheres = zip(*[_ptr_where(b) for b in blocks])
    arr = (C.c_void_p * len(ptrs))(*[p.value for p in ptrs])
    ld_arr = None if ld is None else (C.c_int64 * len(ld))(*[int(x) for x in ld])
    _check(h, lib().dcf_reload_blocks_async(h, arr, ld_arr, wheres[0]))


def dcf_load_init(h, U0, V0_blocks=None):
    pu, where = _ptr_where(U0)
    varr = None
    if V0_blocks is not None:
        vp = [_ptr_where(v)[0].value for v in V0_blocks]
        varr = (C.c_void_p * len(vp))(*vp)
    _check(h, lib().dcf_load_init(h, pu, varr, where))


def dcf_step(h, n_steps=1):
    _check(h, lib().dcf_step(h, int(n_steps)))


def dcf_solve(h):
    it = C.c_int()
    d = C.c_double()
    st = lib().dcf_solve(h, C.byref(it), C.byref(d))
    if st not in (DCF_OK, DCF_ENOTCONV):
        _check(h, st)
    return it.value, d.value, st == DCF_OK


def dcf_get_factors(h, U_out, V_outs=None):
    pu, where = _ptr_where(U_out)
    varr = None
    if V_outs is not None:
        vp = [_ptr_where(v)[0].value for v in V_outs]
        varr = (C.c_void_p * len(vp))(*vp)
    _check(h, lib().dcf_get_factors(h, pu, varr, where))


def dcf_get_LS(h, i, L_out=None, S_out=None):
    pl, wl = _ptr_where(L_out)
    ps, ws = _ptr_where(S_out)
    where = wl if L_out is not None else ws
    _check(h, lib().dcf_get_LS(h, int(i), pl, ps, where))


def dcf_set_private(h, i, is_private=True):
    _check(h, lib().dcf_set_private(h, int(i), 1 if is_private else 0))


def dcf_get_stats(h):
    o, d, it = C.c_double(), C.c_double(), C.c_int()
    _check(h, lib().dcf_get_stats(h, C.byref(o), C.byref(d), C.byref(it)))
    return o.value, d.value, it.value


def dcf_get_conditioning(h, routes=False):
    g, q, rg, rq = C.c_double(), C.c_double(), C.c_int(), C.c_int()
    _check(h, lib().dcf_get_conditioning(h, C.byref(g), C.byref(q), C.byref(rg), C.byref(rq)))
    return (g.value, q.value, rg.value, rq.value) if routes else (g.value, q.value)


def dcf_set_truth(h, A, B):
    pa, where = _ptr_where(A)
    pb, _ = _ptr_where(B)
    _check(h, lib().dcf_set_truth(h, pa, pb, int(A.shape[1]), where))


def dcf_rel_err(h):
    e = C.c_double()
    _check(h, lib().dcf_rel_err(h, C.byref(e)))
    return e.value


def dcf_singular_values(h, r, k=0):
    """(sigma (r,), sigma0 (k,) or None, err or None): singular values of the
    current L = U V^T, and with k > 0 those of the registered truth and the
    relative singular-value error of Table 1."""
    sig = (C.c_double * r)()
    if k > 0:
        sig0 = (C.c_double * k)()
        err = C.c_double()
        _check(h, lib().dcf_singular_values(h, sig, sig0, C.byref(err)))
        return np.array(sig[:]), np.array(sig0[:]), float(err.value)
    _check(h, lib().dcf_singular_values(h, sig, None, None))
    return np.array(sig[:]), None, None


def dcf_last_error(h):
    return lib().dcf_last_error(h).decode()


def dcf_destroy(h):
    if h:
        lib().dcf_destroy(h)


def dcf_profile_phases(h):
    buf = C.create_string_buffer(1024)
    n = lib().dcf_profile_phases(h, buf, 1024)
    return buf.value.decode().split(",")[:n]


def dcf_profile_step(h, n_steps):
    names = dcf_profile_phases(h)
    ms = (C.c_double * len(names))()
    _check(h, lib().dcf_profile_step(h, int(n_steps), ms))
    return dict(zip(names, list(ms)))


def dcf_tc_selftest(cfg):
    """Run the tensor-core layout self-test; returns the 128 x 256 accumulator dump."""
    arr = (C.c_int * 12)(*[int(x) for x in cfg])
    out = np.zeros((128, 256), np.float32)
    st = lib().dcf_tc_selftest(arr, out.ctypes.data_as(C.POINTER(C.c_float)))
    if st != DCF_OK:
        raise DcfError(st, "dcf_tc_selftest")
    return out


def dcf_iterate_noalloc(M, m, n, r, rho, lam, U_in, V_in, U_out, V_out, stream=0):
    """One allocation-free iteration on device tensors (see include/dcf.h);
    returns the status code (0 on success) without raising."""
    def ptr(t):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("dcf_iterate_noalloc takes contiguous CUDA tensors")
        return C.c_void_p(t.data_ptr())
    return lib().dcf_iterate_noalloc(ptr(M), int(m), int(n), int(r), float(rho), float(lam),
                                     ptr(U_in), ptr(V_in), ptr(U_out), ptr(V_out),
                                     C.c_void_p(stream))


def _dvec(x, K):
    if x is None:
        return None
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    if a.size != K:
        raise ValueError(f"expected {K} values, got {a.size}")
    return a


def dcf_unrolled_forward(h, a, b, c, weights=None, want_loss=True):
    """Forward pass of the learned network; returns (total_loss, per-step losses)
    or (None, None) when want_loss is False."""
    K = len(a)
    av, bv, cv = _dvec(a, K), _dvec(b, K), _dvec(c, K)
    wv = _dvec(weights, K)
    dp = lambda v: None if v is None else v.ctypes.data_as(C.POINTER(C.c_double))
    terms = np.zeros(K) if want_loss else None
    tot = C.c_double()
    _check(h, lib().dcf_unrolled_forward(h, int(K), dp(av), dp(bv), dp(cv), dp(wv), dp(terms),
                                         C.byref(tot) if want_loss else None))
    return (tot.value, terms) if want_loss else (None, None)


def dcf_unrolled_backward(h, K, grad_U0=None, grad_V0_blocks=None):
    """Reverse pass of the last forward: returns (grad_a, grad_b, grad_c); the
    start-point gradients go into grad_U0 / grad_V0_blocks when given."""
    ga, gb, gc = np.zeros(K), np.zeros(K), np.zeros(K)
    dp = lambda v: v.ctypes.data_as(C.POINTER(C.c_double))
    pu, where = _ptr_where(grad_U0)
    varr = None
    if grad_V0_blocks is not None:
        vp = [_ptr_where(v)[0].value for v in grad_V0_blocks]
        where = _ptr_where(grad_V0_blocks[0])[1]
        varr = (C.c_void_p * len(vp))(*vp)
    _check(h, lib().dcf_unrolled_backward(h, dp(ga), dp(gb), dp(gc), pu, varr, where))
    return ga, gb, gc


def dcf_version():
    return lib().dcf_version().decode()


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class Solver:
    """One DCF-PCA problem on the current CUDA device.

    ``M`` is an m x n float32 matrix in column-major order: a numpy array
    with ``order='F'`` (copied to the device) or a torch CUDA tensor holding
    M^T in row-major order, i.e. shape (n, m) (borrowed in place).
    """

    def __init__(self, m, n_i, r, rho, lam, max_iter=100, tol=1e-6, u_mode=0, eta0=0.0,
                 seed=0, stream=None, path=PATH_AUTO, local_steps=1):
        self.m, self.n_i, self.r = int(m), [int(x) for x in n_i], int(r)
        self.n = int(sum(self.n_i))
        self.h = dcf_create(m, n_i, r, rho, lam, max_iter, tol, u_mode, local_steps, eta0, seed,
                            path)
        if stream is not None:
            dcf_set_stream(self.h, stream)
        self._keep = None

    def close(self):
        if self.h:
            dcf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def blocks_of(self, M):
        off = np.concatenate([[0], np.cumsum(self.n_i)])
        if _is_torch(M):
            return [M[off[i]:off[i + 1]] for i in range(len(self.n_i))]
        M = np.asfortranarray(M, dtype=np.float32)
        return [M[:, off[i]:off[i + 1]] for i in range(len(self.n_i))]

    def load(self, M, borrow=None):
        blocks = self.blocks_of(M)
        if borrow is None:
            borrow = _is_torch(M)
        self._keep = (M, blocks)
        dcf_load_blocks(self.h, blocks, borrow=borrow)

    def reload(self, M):
        """New values of M (same shape), copied into the loaded buffer; the
        iterate carries over (dcf_reload_blocks).  The copy has completed on
        return, so M need not outlive the call."""
        dcf_reload_blocks(self.h, self.blocks_of(M))

    def reload_async(self, M):
        """dcf_reload_blocks_async: M's copy overlaps the work already enqueued;
        the next step reads it.  M must stay unchanged until a later call that
        returns host data (factors, stats) has returned; the Solver keeps the
        two most recent such matrices referenced."""
        self._async_keep = (getattr(self, "_async_keep", (None, None))[1], M)
        dcf_reload_blocks_async(self.h, self.blocks_of(M))

    def load_init(self, U0, V0=None):
        U0 = self._as_factor(U0)
        Vb = None
        if V0 is not None:
            V0 = self._as_factor(V0)
            off = np.concatenate([[0], np.cumsum(self.n_i)])
            Vb = [V0[off[i]:off[i + 1]] for i in range(len(self.n_i))]
        self._keep_init = (U0, V0, Vb)
        dcf_load_init(self.h, U0, Vb)

    @staticmethod
    def _as_factor(x):
        if _is_torch(x):
            return x.contiguous()
        return np.ascontiguousarray(x, dtype=np.float32)

    @property
    def path(self):
        return dcf_get_path(self.h)

    def step(self, n=1):
        dcf_step(self.h, n)

    def solve(self):
        return dcf_solve(self.h)

    def factors(self):
        U = np.empty((self.m, self.r), np.float32)
        Vs = [np.empty((ni, self.r), np.float32) for ni in self.n_i]
        dcf_get_factors(self.h, U, Vs)
        return U, np.concatenate(Vs, axis=0)

    def LS(self, i):
        L = np.empty((self.n_i[i], self.m), np.float32)   # column-major m x n_i
        S = np.empty((self.n_i[i], self.m), np.float32)
        dcf_get_LS(self.h, i, L, S)
        return L.T, S.T

    def stats(self):
        return dcf_get_stats(self.h)

    def conditioning(self, routes=False):
        """(kappa of U^T U + rho I, kappa of V^T V + rho I) of the last iteration,
        and with routes=True how their inverses were formed (0 FP32 route,
        1 double-float)."""
        return dcf_get_conditioning(self.h, routes)

    def set_truth(self, A, B):
        self._truth = (np.ascontiguousarray(A, np.float32), np.ascontiguousarray(B, np.float32))
        dcf_set_truth(self.h, *self._truth)

    def rel_err(self):
        return dcf_rel_err(self.h)

    def singular_values(self, with_truth=False):
        """dcf_singular_values: sigma of U V^T, and (with_truth) sigma of the
        registered truth plus the relative singular-value error of Table 1."""
        k = self._truth[0].shape[1] if with_truth else 0
        return dcf_singular_values(self.h, self.r, k)

    def unrolled_forward(self, a, b, c, weights=None, want_loss=True):
        return dcf_unrolled_forward(self.h, a, b, c, weights, want_loss)

    def unrolled_backward(self, K, start_grads=False):
        """(grad_a, grad_b, grad_c), plus (grad_U0, grad_V0) when start_grads."""
        if not start_grads:
            return dcf_unrolled_backward(self.h, K)
        gU = np.empty((self.m, self.r), np.float32)
        gVs = [np.empty((ni, self.r), np.float32) for ni in self.n_i]
        g = dcf_unrolled_backward(self.h, K, gU, gVs)
        return g + (gU, np.concatenate(gVs, axis=0))


# ---------------------------------------------------------------------------
# batches of independent problems
# ---------------------------------------------------------------------------
def _bcheck(b, status):
    if status != DCF_OK:
        msg = lib().dcf_batch_last_error(b).decode() if b else ""
        raise DcfError(status, msg)


class Batch:
    """Independent problems advanced together (dcf_batch_* of include/dcf.h).

    ``problems`` is a list of dicts with keys m, n_i, r, rho, lam.
    """

    def __init__(self, problems, max_iter=100, tol=1e-6, seed=0, stream=None):
        self.problems = [dict(m=int(p["m"]), n_i=[int(x) for x in p["n_i"]], r=int(p["r"]),
                              rho=float(p["rho"]), lam=float(p["lam"])) for p in problems]
        keep = []
        arr = (dcf_problem * len(problems))()
        for q, p in enumerate(self.problems):
            ni = (C.c_int64 * len(p["n_i"]))(*p["n_i"])
            keep.append(ni)
            arr[q] = dcf_problem(p["m"], len(p["n_i"]), ni, p["r"], p["rho"], p["lam"])
        h = C.c_void_p()
        st = lib().dcf_batch_create(arr, len(problems), int(max_iter), float(tol), int(seed),
                                    C.byref(h))
        if st != DCF_OK:
            raise DcfError(st, "dcf_batch_create rejected the problems")
        self.h = h
        self._keep = []
        if stream is not None:
            _bcheck(self.h, lib().dcf_batch_set_stream(self.h, C.c_void_p(stream)))

    def close(self):
        if self.h:
            lib().dcf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, i, M):
        """M: m x n float32, numpy (column-major copy) or torch CUDA tensor of shape (n, m)."""
        if not 0 <= i < len(self.problems):
            _bcheck(self.h, lib().dcf_batch_load(self.h, int(i), None, None, 0))
        p = self.problems[i]
        off = np.concatenate([[0], np.cumsum(p["n_i"])])
        if _is_torch(M):
            blocks = [M[off[k]:off[k + 1]] for k in range(len(p["n_i"]))]
        else:
            M = np.asfortranarray(M, dtype=np.float32)
            blocks = [M[:, off[k]:off[k + 1]] for k in range(len(p["n_i"]))]
        ptrs, wheres = zip(*[_ptr_where(b) for b in blocks])
        arr = (C.c_void_p * len(ptrs))(*[q.value for q in ptrs])
        _bcheck(self.h, lib().dcf_batch_load(self.h, int(i), arr, None, wheres[0]))
        self._keep.append((M, blocks))

    def load_init(self, i, U0, V0=None):
        p = self.problems[i]
        U0 = np.ascontiguousarray(U0, np.float32)
        varr = None
        if V0 is not None:
            V0 = np.ascontiguousarray(V0, np.float32)
            off = np.concatenate([[0], np.cumsum(p["n_i"])])
            vb = [np.ascontiguousarray(V0[off[k]:off[k + 1]]) for k in range(len(p["n_i"]))]
            self._keep.append(vb)
            varr = (C.c_void_p * len(vb))(*[v.ctypes.data for v in vb])
        self._keep.append(U0)
        _bcheck(self.h, lib().dcf_batch_load_init(self.h, int(i), C.c_void_p(U0.ctypes.data),
                                                  varr, 0))

    def tune(self, reps=3):
        buf = C.create_string_buffer(8192)
        _bcheck(self.h, lib().dcf_batch_tune(self.h, int(reps), buf, 8192))
        return buf.value.decode()

    def step(self, n=1):
        _bcheck(self.h, lib().dcf_batch_step(self.h, int(n)))

    def solve(self):
        its = (C.c_int * len(self.problems))()
        nc = C.c_int()
        st = lib().dcf_batch_solve(self.h, its, C.byref(nc))
        if st not in (DCF_OK, DCF_ENOTCONV):
            _bcheck(self.h, st)
        return list(its), nc.value

    def factors(self, i):
        p = self.problems[i]
        U = np.empty((p["m"], p["r"]), np.float32)
        Vs = [np.empty((ni, p["r"]), np.float32) for ni in p["n_i"]]
        varr = (C.c_void_p * len(Vs))(*[v.ctypes.data for v in Vs])
        _bcheck(self.h, lib().dcf_batch_get_factors(self.h, int(i), C.c_void_p(U.ctypes.data),
                                                    varr, 0))
        return U, np.concatenate(Vs, axis=0)

    BATCH_PHASES = ["make_w", "pass1_vstep", "pass2_pstep", "gram_v", "reduce_q", "rows_ustep",
                    "reduce_g"]

    def profile_step(self, n):
        ms = (C.c_double * 7)()
        _bcheck(self.h, lib().dcf_batch_profile_step(self.h, int(n), ms, 7))
        return dict(zip(self.BATCH_PHASES, list(ms)))

    def stats(self, i):
        o, d, it = C.c_double(), C.c_double(), C.c_int()
        _bcheck(self.h, lib().dcf_batch_get_stats(self.h, int(i), C.byref(o), C.byref(d),
                                                  C.byref(it)))
        return o.value, d.value, it.value
