"""Host-side checks of the C ABI library: it loads, exports every entry point
of include/hs.h, and its symbolic planner reproduces the oracle's canonical
waves and neighbour / well-separated lists exactly (integers, bit for bit)."""
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import hsolver as H
from paper_1611_03189_gb300 import _lib
from paper_1611_03189_gb300 import problems as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1611_03189_gb300.build import build

    build()
    return _lib.lib()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "hs.h")).read()
    declared = set(re.findall(r"^\s*(?:int|int64_t|const char \*)\s*(hs_\w+)\s*\(", hdr, flags=re.M))
    assert declared == set(_lib.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(hs_\w+)\b", out))
    assert declared <= exported
    for name in declared:
        assert hasattr(lib, name)


def test_binding_structs_match_the_compiled_abi(lib):
    """The ctypes mirrors of hs_csr, hs_clustering, hs_opts and hs_info have the
    sizes the library was compiled with (a field added on one side only would
    shift every later field)."""
    import ctypes as C

    sizes = np.zeros(5, dtype=np.int64)
    assert lib.hs_abi_sizes(sizes.ctypes.data, 5) == 5
    mine = [C.sizeof(_lib.HsCsr), C.sizeof(_lib.HsClustering), C.sizeof(_lib.HsOpts), C.sizeof(_lib.HsInfo),
            C.sizeof(_lib.HsAllocator)]
    assert sizes.tolist() == mine


PLAN_CASES = [
    ("poisson2d 32 leaf8", lambda: P.poisson2d(32, leaf_size=8)),
    ("poisson2d 64 leaf16", lambda: P.poisson2d(64, leaf_size=16)),
    ("rect 24x20 leaf4", lambda: P.make_problem((24, 20), P.coef_constant((24, 20)), 4)),
    ("poisson3d 12 leaf8", lambda: P.poisson3d(12, leaf_size=8)),
    ("diffusion 40 leaf4", lambda: P.diffusion2d(40, 1.0, 0, leaf_size=4)),
]


@pytest.mark.parametrize("name,maker", PLAN_CASES, ids=[c[0] for c in PLAN_CASES])
@pytest.mark.parametrize("nbr_dist", [1, 2])
def test_planner_matches_oracle_waves_and_lists(lib, name, maker, nbr_dist):
    pb = maker()
    F = H.factor(pb.n, pb.rowptr, pb.col, pb.val, pb.perm, pb.leaf_ptr, 0.3, H.LORASP, nbr_dist=nbr_dist)
    plan = _lib.Plan(pb.n, pb.rowptr, pb.col, pb.perm, pb.leaf_ptr, nbr_dist=nbr_dist)
    try:
        for lv in F.levels:
            wo = plan.waves(lv.level)
            expect = np.full(lv.nsup, -1, dtype=np.int32)
            for wi, w in enumerate(lv.waves):
                expect[w] = wi
            assert np.array_equal(wo, expect), f"level {lv.level}"
            for rec in lv.supers:
                nb, ws = plan.lists(lv.level, rec.key)
                assert nb == rec.nbrs and ws == rec.wsep, f"level {lv.level} super {rec.key}"
    finally:
        plan.close()


def test_planner_rejects_bad_inputs(lib):
    pb = P.poisson2d(8, leaf_size=4)
    bad_perm = pb.perm.copy()
    bad_perm[0] = bad_perm[1]
    with pytest.raises(_lib.HsError) as e:
        _lib.Plan(pb.n, pb.rowptr, pb.col, bad_perm, pb.leaf_ptr)
    assert e.value.code == _lib.HS_ERR_INVALID and "permutation" in str(e.value)
    lp3 = np.array([0, 20, 40, 64], dtype=np.int32)
    with pytest.raises(_lib.HsError) as e:
        _lib.Plan(pb.n, pb.rowptr, pb.col, pb.perm, lp3)
    assert "power of two" in str(e.value)
    # structurally unsymmetric pattern
    rp = np.array([0, 2, 3], dtype=np.int32)
    ci = np.array([0, 1, 1], dtype=np.int32)
    with pytest.raises(_lib.HsError) as e:
        _lib.Plan(2, rp, ci, np.array([0, 1], np.int32), np.array([0, 1, 2], np.int32))
    assert "symmetric" in str(e.value)
    for d in (-1, 3):
        with pytest.raises(_lib.HsError) as e:
            _lib.Plan(pb.n, pb.rowptr, pb.col, pb.perm, pb.leaf_ptr, nbr_dist=d)
        assert "nbr_dist" in str(e.value)


def test_library_does_not_fall_back_without_a_device(lib):
    """With no CUDA device the compute entry points fail; nothing runs on the CPU."""
    import ctypes as C

    import torch

    if torch.cuda.is_available():
        pytest.skip("a device is present")
    pb = P.poisson2d(8, leaf_size=4)
    rp, ci, pe, lp = (np.ascontiguousarray(x, np.int32) for x in (pb.rowptr, pb.col, pb.perm, pb.leaf_ptr))
    val = np.ascontiguousarray(pb.val)
    A = _lib.HsCsr(pb.n, pb.nnz, rp.ctypes.data, ci.ctypes.data, val.ctypes.data)
    cl = _lib.HsClustering(pe.ctypes.data, lp.ctypes.data, len(lp) - 1)
    o = _lib.HsOpts(0.1, _lib.HS_GC_CONSTANT, _lib.HS_PREC_F64, None)
    h = C.c_void_p()
    code = lib.hs_factor_create(C.byref(A), C.byref(cl), C.byref(o), None, C.byref(h))
    assert code == _lib.HS_ERR_CUDA and not h.value


def test_options_are_validated_before_any_device_work(lib):
    import ctypes as C

    A = _lib.HsCsr(4, 4, 1, 1, 1)
    cl = _lib.HsClustering(1, 1, 1)
    h = C.c_void_p()
    for eps, var, prec in ((-1.0, 1, 0), (1e-8, 1, 0), (0.1, 7, 0), (0.1, 1, 5), (0.1, 2, 0)):
        o = _lib.HsOpts(eps, var, prec, None)
        assert lib.hs_factor_create(C.byref(A), C.byref(cl), C.byref(o), None, C.byref(h)) == _lib.HS_ERR_INVALID
    # GMRES: tolerance, step counts and the Krylov basis limit come first
    it, rr = C.c_int32(), C.c_double()
    for rtol, maxit, restart in ((0.0, 10, 0), (1e-10, 0, 0), (1e-10, 10, -1), (1e-10, 2000, 0), (1e-10, 5000, 1001)):
        assert lib.hs_gmres(C.c_void_p(8), 8, 8, rtol, maxit, restart, C.byref(it), C.byref(rr), None) == _lib.HS_ERR_INVALID
    # several vectors and the Appendix B projection: n_phi in range, only for the
    # variants that take vectors, eps1 finite and >= 0, phi present
    phi = np.ones(8)
    P_ = phi.ctypes.data
    for var, ptr, nphi, eps1 in ((_lib.HS_GC_USER, P_, 5, 0.0), (_lib.HS_GC_USER, P_, -1, 0.0),
                                 (_lib.HS_GC_CONSTANT, None, 2, 0.0), (_lib.HS_LORASP, None, 2, 0.0),
                                 (_lib.HS_GC_PROJ, P_, 1, -1.0), (_lib.HS_GC_PROJ, P_, 1, float("nan")),
                                 (_lib.HS_GC_PROJ, None, 1, 0.1)):
        o = _lib.HsOpts(0.1, var, 0, ptr, None, 0, nphi, eps1)
        assert lib.hs_factor_create(C.byref(A), C.byref(cl), C.byref(o), None, C.byref(h)) == _lib.HS_ERR_INVALID


def test_allocator_hook_is_validated_before_any_device_work(lib):
    """hs_opts.allocator needs both functions; a half-set hook is refused
    before the device is touched (no GPU needed)."""
    import ctypes as C

    A = _lib.HsCsr(4, 4, 1, 1, 1)
    cl = _lib.HsClustering(1, 1, 1)
    h = C.c_void_p()
    hook = _lib.DeviceAllocator()
    half = _lib.HsAllocator(hook.struct.alloc, _lib.FREE_FN(), None)
    o = _lib.HsOpts(0.1, _lib.HS_GC_CONSTANT, 0, None)
    o.allocator = C.addressof(half)
    assert lib.hs_factor_create(C.byref(A), C.byref(cl), C.byref(o), None, C.byref(h)) == _lib.HS_ERR_INVALID
    assert "both alloc and free" in lib.hs_last_error().decode()
    # the binding's hook: every field set, and its counters start at zero
    assert hook.struct.alloc and hook.struct.free and hook.held == 0 and hook.peak == 0


def test_rank_f64_option_is_validated_before_any_device_work(lib):
    import ctypes as C

    A = _lib.HsCsr(4, 4, 1, 1, 1)
    cl = _lib.HsClustering(1, 1, 1)
    h = C.c_void_p()
    o = _lib.HsOpts(0.1, _lib.HS_GC_CONSTANT, _lib.HS_PREC_F32, None)
    o.rank_f64 = 2
    assert lib.hs_factor_create(C.byref(A), C.byref(cl), C.byref(o), None, C.byref(h)) == _lib.HS_ERR_INVALID
    assert "rank_f64" in lib.hs_last_error().decode()


def test_hook_is_not_called_without_a_device(lib):
    """With no CUDA device the create fails before any allocation: the hook
    sees no call and holds nothing."""
    import ctypes as C

    import torch

    if torch.cuda.is_available():
        pytest.skip("a device is present")
    pb = P.poisson2d(8, leaf_size=4)
    rp, ci, pe, lp = (np.ascontiguousarray(x, np.int32) for x in (pb.rowptr, pb.col, pb.perm, pb.leaf_ptr))
    val = np.ascontiguousarray(pb.val)
    A = _lib.HsCsr(pb.n, pb.nnz, rp.ctypes.data, ci.ctypes.data, val.ctypes.data)
    cl = _lib.HsClustering(pe.ctypes.data, lp.ctypes.data, len(lp) - 1)
    hook = _lib.DeviceAllocator()
    o = _lib.HsOpts(0.1, _lib.HS_GC_CONSTANT, _lib.HS_PREC_F32, None)
    o.allocator = hook.ptr()
    h = C.c_void_p()
    assert lib.hs_factor_create(C.byref(A), C.byref(cl), C.byref(o), None, C.byref(h)) == _lib.HS_ERR_CUDA
    assert not h.value and hook.calls == 0 and hook.held == 0 and not hook.errors


def test_device_allocator_bookkeeping_without_a_device():
    """The binding's hook: a request past its limit gets NULL and is not an
    error; a request the backing allocator cannot serve gets NULL and is kept
    in `errors`; freeing an unknown pointer is recorded, not raised into C."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a device is present")
    hook = _lib.DeviceAllocator(limit=100)
    assert hook._on_alloc(200, 0, None, None) is None and not hook.errors and hook.held == 0
    assert hook._on_alloc(50, 0, None, None) is None and len(hook.errors) == 1   # no CUDA here
    hook._on_free(0x1234, 0, None, None)
    assert len(hook.errors) == 2 and hook.held == 0 and hook.calls == 0
