"""ctypes binding of the C ABI in include/hs.h (argument marshalling only).

Every computation happens in libhs.so.  Loading fails loudly when the library
has not been built (``python -m paper_1611_03189_gb300.build`` or
``__graft_entry__.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhs.so")

HS_OK = 0
HS_ERR_INVALID = 1
HS_ERR_NOT_SPD = 2
HS_ERR_CAPACITY = 3
HS_ERR_OOM = 4
HS_ERR_NO_CONVERGENCE = 5
HS_ERR_TIMEOUT = 6
HS_ERR_CUDA = 7

HS_LORASP = 0
HS_GC_CONSTANT = 1
HS_GC_USER = 2
HS_GC_PROJ = 3
HS_MAX_PHI = 4

HS_PREC_F64 = 0
HS_PREC_F32 = 1
HS_PREC_TF32 = 2
HS_PREC_BF16 = 3
HS_PREC_TF32X3 = 4

HS_ORDER_WAVES = 0
HS_ORDER_SEQUENTIAL = 1

STATUS_NAMES = {
    0: "HS_OK", 1: "HS_ERR_INVALID", 2: "HS_ERR_NOT_SPD", 3: "HS_ERR_CAPACITY", 4: "HS_ERR_OOM",
    5: "HS_ERR_NO_CONVERGENCE", 6: "HS_ERR_TIMEOUT", 7: "HS_ERR_CUDA",
}

# every symbol include/hs.h declares
EXPORTS = [
    "hs_factor_create", "hs_factor_refactor", "hs_factor_create_batch", "hs_factor_refactor_batch",
    "hs_launch_count", "hs_profile_phases", "hs_abi_sizes", "hs_apply", "hs_apply_static", "hs_pcg", "hs_gmres", "hs_factor_info", "hs_factor_ranks",
    "hs_factor_destroy", "hs_last_error", "hs_plan_create", "hs_plan_level_waves",
    "hs_plan_super_lists", "hs_plan_destroy", "hs_gemm_tc", "hs_gemm_tune_report", "hs_test_wait_probe",
]


class HsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class HsCsr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class HsClustering(C.Structure):
    _fields_ = [("perm", C.c_void_p), ("leaf_ptr", C.c_void_p), ("nleaf", C.c_int32), ("nbr_dist", C.c_int32)]


class HsOpts(C.Structure):
    _fields_ = [("eps", C.c_double), ("variant", C.c_int32), ("factor_prec", C.c_int32),
                ("phi", C.c_void_p), ("eps_level", C.c_void_p), ("n_eps_level", C.c_int32),
                ("n_phi", C.c_int32), ("eps1", C.c_double), ("scale", C.c_int32),
                ("timeout_cycles", C.c_int64), ("order_mode", C.c_int32), ("max_rank_ratio", C.c_double),
                ("allocator", C.c_void_p), ("rank_f64", C.c_int32)]


# hs_allocator: alloc(bytes, device, stream, ctx) -> device pointer or NULL;
# free(ptr, device, stream, ctx)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_uint64, C.c_int32, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p)


class HsAllocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class DeviceAllocator:
    """A device-memory hook (hs_opts.allocator) that takes the handle's
    memory from PyTorch's caching allocator and counts it: `held` is the bytes
    the handles using this hook hold right now, `peak` the most they held at
    once.  With `limit` set, a request that would take `held` past it gets no
    memory (the library call then fails with HS_ERR_OOM), which is how a
    serving loop caps what one factorization may take.

    One object may serve several handles; it must outlive them (Factor keeps a
    reference).  The callbacks run on the thread that called the library.
    """

    def __init__(self, limit: int | None = None):
        import threading

        self.limit = limit
        self.held = 0
        self.peak = 0
        self.calls = 0
        self.blocks: dict[int, int] = {}
        self.errors: list[str] = []   # exceptions the callbacks caught (they cannot raise into C)
        self._mu = threading.Lock()
        self._alloc = ALLOC_FN(self._on_alloc)
        self._free = FREE_FN(self._on_free)
        self.struct = HsAllocator(self._alloc, self._free, None)

    def _on_alloc(self, nbytes, device, stream, ctx):
        try:
            import torch

            nbytes = int(nbytes)
            with self._mu:
                if self.limit is not None and self.held + nbytes > self.limit:
                    return None
            p = int(torch.cuda.caching_allocator_alloc(nbytes, device=int(device), stream=int(stream or 0)))
            with self._mu:
                self.blocks[p] = nbytes
                self.held += nbytes
                self.peak = max(self.peak, self.held)
                self.calls += 1
            return p
        except Exception as ex:
            self.errors.append(f"alloc({int(nbytes)}): {ex!r}")
            return None   # the library reports HS_ERR_OOM

    def _on_free(self, ptr, device, stream, ctx):
        try:
            import torch

            p = int(ptr)
            with self._mu:
                nbytes = self.blocks.pop(p)
                self.held -= nbytes
            torch.cuda.caching_allocator_delete(p)
        except Exception as ex:
            self.errors.append(f"free({int(ptr or 0):#x}): {ex!r}")

    def ptr(self) -> int:
        return C.addressof(self.struct)


def _phi_block(phi):
    """Preserved vectors as hs_opts wants them: an n-vector, or an n x p array
    (one vector per column) -> (p x n C-contiguous float64, p)."""
    a = np.asarray(phi, dtype=np.float64)
    if a.ndim == 1:
        return np.ascontiguousarray(a), 1
    return np.ascontiguousarray(a.T), int(a.shape[1])


class HsInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("levels", C.c_int32), ("waves", C.c_int32),
                ("super_nodes", C.c_int32), ("root_size", C.c_int32), ("max_rank", C.c_int32),
                ("max_super", C.c_int32), ("device_bytes", C.c_int64), ("factor_bytes", C.c_int64),
                ("factor_flops", C.c_double), ("eig_flops", C.c_double), ("factor_ms", C.c_double),
                ("trunc_big_ms", C.c_double), ("trunc_big_flops", C.c_double), ("trunc_big_launches", C.c_int32),
                ("host_ms", C.c_double), ("wait_ms", C.c_double), ("phase_ms", C.c_double * 16),
                ("alg_flops", C.c_double), ("tc_flops", C.c_double), ("tc_ms", C.c_double),
                ("tc_launches", C.c_int64)]

    PHASES = ("merge", "gather", "chol_Ass", "gram", "trunc_small", "trunc_large", "cholqr_large",
              "extension", "schur", "root", "grid_prepare", "grid_tridiag_steps", "grid_qtz",
              "grid_eigvec_T", "grid_qy", "unused")

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "phase_ms"}
        d["phase_ms"] = dict(zip(self.PHASES, list(self.phase_ms)))
        return d


_lib = None


def lib():
    """The loaded libhs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libhs.so not built at {LIB_PATH}; run paper_1611_03189_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.hs_factor_create.argtypes = [C.POINTER(HsCsr), C.POINTER(HsClustering), C.POINTER(HsOpts), vp,
                                       C.POINTER(vp)]
        L.hs_factor_refactor.argtypes = [vp, vp, vp]
        L.hs_factor_create_batch.argtypes = [i32, C.POINTER(HsCsr), C.POINTER(HsClustering), C.POINTER(HsOpts),
                                             vp, vp, C.POINTER(vp), vp]
        L.hs_factor_refactor_batch.argtypes = [i32, C.POINTER(vp), vp, vp, vp]
        L.hs_launch_count.argtypes = []
        L.hs_profile_phases.argtypes = [i32]
        L.hs_abi_sizes.argtypes = [vp, i32]
        L.hs_apply.argtypes = [vp, vp, vp, i32, i64, vp]
        L.hs_apply_static.argtypes = [vp, vp, vp, i32, i64, vp]
        L.hs_pcg.argtypes = [vp, vp, vp, i32, i64, dbl, i32, vp, vp, vp]
        L.hs_gmres.argtypes = [vp, vp, vp, dbl, i32, i32, vp, vp, vp]
        L.hs_factor_info.argtypes = [vp, C.POINTER(HsInfo)]
        L.hs_factor_ranks.argtypes = [vp, i32, vp, i32, C.POINTER(i32)]
        L.hs_factor_destroy.argtypes = [vp]
        L.hs_last_error.restype = C.c_char_p
        L.hs_plan_create.argtypes = [i64, vp, vp, C.POINTER(HsClustering), C.POINTER(vp)]
        L.hs_plan_level_waves.argtypes = [vp, i32, vp, i32, C.POINTER(i32)]
        L.hs_plan_super_lists.argtypes = [vp, i32, i32, vp, vp, i32, C.POINTER(i32), C.POINTER(i32)]
        L.hs_plan_destroy.argtypes = [vp]
        flt = C.c_float
        L.hs_gemm_tc.argtypes = [i32, i32, i32, i32, flt, vp, i64, i32, vp, i64, i32, flt, vp, i64, i32, vp]
        L.hs_gemm_tune_report.argtypes = [i32, vp, vp, i32]
        L.hs_test_wait_probe.argtypes = [i32]
        for name in EXPORTS:
            if name not in ("hs_last_error", "hs_launch_count"):
                getattr(L, name).restype = C.c_int
        L.hs_launch_count.restype = C.c_int64
        _lib = L
    return _lib


def launch_count() -> int:
    """Kernels launched by libhs.so in this process so far."""
    return int(lib().hs_launch_count())


def check(code: int):
    if code != HS_OK:
        raise HsError(code, lib().hs_last_error().decode())
    return code


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---------------------------------------------------------------------------
# planner (host only)
# ---------------------------------------------------------------------------

class Plan:
    """Symbolic planner of the library (host only)."""

    def __init__(self, n, rowptr, col, perm, leaf_ptr, nbr_dist=1):
        self._keep = [np.ascontiguousarray(x, dtype=np.int32) for x in (rowptr, col, perm, leaf_ptr)]
        rp, ci, pe, lp = self._keep
        cl = HsClustering(_ptr(pe), _ptr(lp), len(lp) - 1, int(nbr_dist))
        h = C.c_void_p()
        check(lib().hs_plan_create(int(n), _ptr(rp), _ptr(ci), C.byref(cl), C.byref(h)))
        self._h = h
        self.L = int(round(np.log2(len(lp) - 1)))

    def waves(self, level: int) -> np.ndarray:
        ns = 2 ** (level - 1)
        out = np.empty(ns, dtype=np.int32)
        nw = C.c_int32()
        check(lib().hs_plan_level_waves(self._h, level, _ptr(out), ns, C.byref(nw)))
        return out

    def lists(self, level: int, s: int):
        cap = 4096
        nb = np.empty(cap, dtype=np.int32)
        ws = np.empty(cap, dtype=np.int32)
        nn, nw = C.c_int32(), C.c_int32()
        check(lib().hs_plan_super_lists(self._h, level, s, _ptr(nb), _ptr(ws), cap, C.byref(nn),
                                        C.byref(nw)))
        return nb[: nn.value].tolist(), ws[: nw.value].tolist()

    def close(self):
        if self._h:
            lib().hs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# factorization handle (device)
# ---------------------------------------------------------------------------

def _stream_ptr(stream):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Factor:
    """hs_factor_create / hs_apply / hs_pcg on torch CUDA tensors.

    rowptr, col: int32 CUDA tensors; val: float64 CUDA tensor (original order).
    perm, leaf_ptr: host int32 arrays (clustering).  phi: host float64, an
    n-vector or n x p (p <= HS_MAX_PHI vectors), for HS_GC_USER / HS_GC_PROJ.
    eps1: HS_GC_PROJ's first tolerance.  nbr_dist: neighbour rule (1: joined by
    an edge; 2: also nodes sharing a neighbour).
    """

    def __init__(self, rowptr, col, val, perm, leaf_ptr, eps, variant=HS_GC_CONSTANT,
                 prec=HS_PREC_F64, phi=None, stream=None, eps_level=None, eps1=0.0, nbr_dist=1, scale=False,
                 timeout_cycles=0, order_mode=HS_ORDER_WAVES, max_rank_ratio=0.0, allocator=None,
                 rank_f64=False):
        import torch

        assert rowptr.is_cuda and col.is_cuda and val.is_cuda
        assert rowptr.dtype == torch.int32 and col.dtype == torch.int32 and val.dtype == torch.float64
        self.n = int(rowptr.numel() - 1)
        self._perm = np.ascontiguousarray(perm, dtype=np.int32)
        self._lp = np.ascontiguousarray(leaf_ptr, dtype=np.int32)
        self._phi, nphi = (None, 0) if phi is None else _phi_block(phi)
        A = HsCsr(self.n, int(col.numel()), rowptr.data_ptr(), col.data_ptr(), val.data_ptr())
        cl = HsClustering(_ptr(self._perm), _ptr(self._lp), len(self._lp) - 1, int(nbr_dist))
        self._epsl = None if eps_level is None else np.ascontiguousarray(eps_level, dtype=np.float64)
        o = HsOpts(float(eps), int(variant), int(prec), None if self._phi is None else _ptr(self._phi),
                   None if self._epsl is None else _ptr(self._epsl), 0 if self._epsl is None else len(self._epsl),
                   nphi, float(eps1), int(bool(scale)), int(timeout_cycles), int(order_mode),
                   float(max_rank_ratio), None if allocator is None else allocator.ptr(), int(bool(rank_f64)))
        h = C.c_void_p()
        self._h = None
        self._alloc = allocator   # the hook must outlive the handle
        check(lib().hs_factor_create(C.byref(A), C.byref(cl), C.byref(o), _stream_ptr(stream), C.byref(h)))
        self._h = h

    def refactor(self, val, stream=None):
        """Factor new values (float64 CUDA tensor, nnz) of the same pattern."""
        import torch

        assert val.is_cuda and val.dtype == torch.float64 and val.is_contiguous()
        check(lib().hs_factor_refactor(self._h, val.data_ptr(), _stream_ptr(stream)))

    def apply(self, r, z=None, stream=None):
        """z = A_H^-1 r; r is (n,) or (nrhs, n) float64 CUDA (each row one rhs)."""
        import torch

        r = r.contiguous()
        nrhs = 1 if r.dim() == 1 else r.shape[0]
        if z is None:
            z = torch.empty_like(r)
        check(lib().hs_apply(self._h, r.data_ptr(), z.data_ptr(), nrhs, self.n, _stream_ptr(stream)))
        return z

    def pcg(self, b, rtol=1e-10, maxit=500, x=None, stream=None, raise_on_fail=True):
        """x, iters, relres, status for A x = b; b is (n,) or (nrhs, n) float64 CUDA."""
        import torch

        b = b.contiguous()
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        if x is None:
            x = torch.empty_like(b)
        it = np.zeros(nrhs, dtype=np.int32)
        rr = np.zeros(nrhs, dtype=np.float64)
        code = lib().hs_pcg(self._h, b.data_ptr(), x.data_ptr(), nrhs, self.n, float(rtol), int(maxit),
                            _ptr(it), _ptr(rr), _stream_ptr(stream))
        if code not in (HS_OK, HS_ERR_NO_CONVERGENCE) or (raise_on_fail and code != HS_OK):
            check(code)
        return x, it, rr, code

    def gmres(self, b, rtol=1e-10, maxit=300, restart=0, x=None, stream=None, raise_on_fail=True):
        """x, iters, relres, status of right-preconditioned GMRES for A x = b;
        b is (n,) float64 CUDA; restart = 0 runs without restarts."""
        import torch

        b = b.contiguous()
        if x is None:
            x = torch.empty_like(b)
        it = C.c_int32()
        rr = C.c_double()
        code = lib().hs_gmres(self._h, b.data_ptr(), x.data_ptr(), float(rtol), int(maxit), int(restart),
                              C.byref(it), C.byref(rr), _stream_ptr(stream))
        if code not in (HS_OK, HS_ERR_NO_CONVERGENCE) or (raise_on_fail and code != HS_OK):
            check(code)
        return x, int(it.value), float(rr.value), code

    def info(self) -> dict:
        inf = HsInfo()
        check(lib().hs_factor_info(self._h, C.byref(inf)))
        return inf.as_dict()

    def ranks(self, level: int) -> np.ndarray:
        ns = 2 ** (level - 1)
        out = np.empty(ns, dtype=np.int32)
        cnt = C.c_int32()
        check(lib().hs_factor_ranks(self._h, level, _ptr(out), ns, C.byref(cnt)))
        return out

    def close(self):
        if self._h:
            lib().hs_factor_destroy(self._h)
            self._h = None
        self._alloc = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def factor_batch(problems, eps, variant=HS_GC_CONSTANT, prec=HS_PREC_F64, phis=None, stream=None,
                 eps_level=None, eps1=0.0, nbr_dist=1, scale=False, allocator=None, rank_f64=False):
    """hs_factor_create_batch over `problems`: a list of (rowptr, col, val,
    perm, leaf_ptr) with rowptr/col int32 and val float64 CUDA tensors and
    perm/leaf_ptr host arrays.  Returns (factors, status): one Factor per
    problem (None where its status is HS_ERR_NOT_SPD) and the status array."""
    import torch

    k = len(problems)
    A = (HsCsr * k)()
    cl = (HsClustering * k)()
    keep = []
    for p, (rp, ci, va, perm, lp) in enumerate(problems):
        assert rp.is_cuda and ci.is_cuda and va.is_cuda
        assert rp.dtype == torch.int32 and ci.dtype == torch.int32 and va.dtype == torch.float64
        pe = np.ascontiguousarray(perm, dtype=np.int32)
        lpa = np.ascontiguousarray(lp, dtype=np.int32)
        keep += [pe, lpa]
        A[p] = HsCsr(int(rp.numel() - 1), int(ci.numel()), rp.data_ptr(), ci.data_ptr(), va.data_ptr())
        cl[p] = HsClustering(_ptr(pe), _ptr(lpa), len(lpa) - 1, int(nbr_dist))
    phi_arr = None
    nphi = 0
    if phis is not None:
        blocks = [_phi_block(x) for x in phis]
        nphi = blocks[0][1]
        assert all(b[1] == nphi for b in blocks), "every problem needs the same number of vectors"
        ph = [b[0] for b in blocks]
        keep += ph
        phi_arr = (C.c_void_p * k)(*[_ptr(x) for x in ph])
    epsl = None if eps_level is None else np.ascontiguousarray(eps_level, dtype=np.float64)
    keep.append(epsl)
    o = HsOpts(float(eps), int(variant), int(prec), None, None if epsl is None else _ptr(epsl),
               0 if epsl is None else len(epsl), nphi, float(eps1), int(bool(scale)), 0, HS_ORDER_WAVES, 0.0,
               None if allocator is None else allocator.ptr(), int(bool(rank_f64)))
    out = (C.c_void_p * k)()
    status = np.zeros(k, dtype=np.int32)
    code = lib().hs_factor_create_batch(k, A, cl, C.byref(o), phi_arr, _stream_ptr(stream), out, _ptr(status))
    if code not in (HS_OK, HS_ERR_NOT_SPD):
        check(code)
    fs = []
    for p, (rp, ci, va, perm, lp) in enumerate(problems):
        if status[p] != HS_OK:
            fs.append(None)
            continue
        f = Factor.__new__(Factor)
        f.n = int(rp.numel() - 1)
        f._perm = keep[2 * p]
        f._lp = keep[2 * p + 1]
        f._phi = None
        f._alloc = allocator
        f._h = C.c_void_p(out[p])
        fs.append(f)
    return fs, status


def refactor_batch(factors, vals, stream=None):
    """hs_factor_refactor_batch: new values (float64 CUDA tensors) for each
    handle.  Returns the per-problem status array (HS_OK or HS_ERR_NOT_SPD)."""
    k = len(factors)
    hs = (C.c_void_p * k)(*[f._h.value for f in factors])
    vs = (C.c_void_p * k)(*[v.data_ptr() for v in vals])
    status = np.zeros(k, dtype=np.int32)
    code = lib().hs_factor_refactor_batch(k, hs, vs, _stream_ptr(stream), _ptr(status))
    if code not in (HS_OK, HS_ERR_NOT_SPD):
        check(code)
    return status


def gemm_tc(prec, A, B, C, alpha=1.0, beta=0.0, ta=False, tb=False, bn=0, stream=None):
    """C = alpha op(A) op(B) + beta C through the tensor-core GEMM (hs_gemm_tc).
    A, B, C: 2-D float32 CUDA tensors, row-major with unit column stride
    (their row strides are the leading dimensions); op(X) = X.T when the
    flag is set.  C is updated in place."""
    for X in (A, B, C):
        if X.dim() != 2 or X.stride(1) != 1 or str(X.dtype) != "torch.float32":
            raise ValueError("A, B, C must be 2-D float32 tensors with unit column stride")
    M, N = C.shape
    K = A.shape[0] if ta else A.shape[1]

    def ld(X):
        return max(X.stride(0), X.shape[1], 1)

    check(lib().hs_gemm_tc(int(prec), M, N, K, float(alpha), A.data_ptr(), ld(A), int(bool(ta)),
                           B.data_ptr(), ld(B), int(bool(tb)), float(beta), C.data_ptr(), ld(C),
                           int(bn), _stream_ptr(stream)))
    return C


def gemm_tune_report(prec) -> list:
    """The GEMM autotuner's table for operand precision `prec` on the current
    device: one dict per shape class (hs_gemm_tune_report)."""
    cap = 32
    ms = np.zeros(3 * cap, dtype=np.float32)
    route = np.zeros(cap, dtype=np.int32)
    n = int(lib().hs_gemm_tune_report(int(prec), _ptr(ms), _ptr(route), cap))
    if n < 0:
        check(-n)
    mn = ("<=32", "<=64", "<=128", "<=256", ">256")
    kk = ("<=32", "<=128", "<=512", ">512")
    return [{"max_mn": mn[c // 4], "k": kk[c % 4], "ms_simt": float(ms[3 * c]), "ms_tc64": float(ms[3 * c + 1]),
             "ms_tc128": float(ms[3 * c + 2]), "route": int(route[c])} for c in range(min(n, cap))]


def profile_phases(on: bool) -> None:
    """hs_profile_phases: per-phase device times of later factorizations."""
    check(lib().hs_profile_phases(1 if on else 0))
