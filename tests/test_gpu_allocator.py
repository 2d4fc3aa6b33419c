"""The device-memory hook (hs_opts.allocator) on the GPU.

A caller that keeps its own account of device memory -- the serving loop,
which admits work against a byte budget, or a framework with a caching
allocator -- hands the handle an hs_allocator and the handle takes every
device block it holds from it.  The hook changes where the memory comes from
and nothing else, so:
* results are those of the default handle, bit for bit (apply, PCG,
  refactor), in FP64 and FP32;
* every block taken is given back at destroy, and what the hook holds covers
  the factor arenas the handle reports in device_bytes;
* a hook without memory fails the call with HS_ERR_OOM after every block that
  call took is back, and the handle or device stays usable.
"""
import numpy as np
import pytest

from paper_1611_03189_gb300 import _lib
from paper_1611_03189_gb300 import problems as P

from gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu


def _factor(pb, prec, allocator=None):
    rp, ci, va = to_dev(pb)
    return _lib.Factor(rp, ci, va, pb.perm, pb.leaf_ptr, 1e-2, _lib.HS_GC_CONSTANT, prec, allocator=allocator)


@pytest.mark.parametrize("prec", [_lib.HS_PREC_F64, _lib.HS_PREC_F32])
def test_hooked_handle_matches_default_bitwise_and_returns_every_block(prec):
    torch = need_gpu()
    pb = P.diffusion2d(64, 1.0, 3, leaf_size=8)
    hook = _lib.DeviceAllocator()
    G0 = _factor(pb, prec)
    G1 = _factor(pb, prec, hook)
    held_after_factor = hook.held
    assert hook.calls > 0 and held_after_factor > 0
    assert held_after_factor >= G1.info()["device_bytes"]
    B = torch.as_tensor(P.rhs(pb.n, 7, nrhs=3).T.copy(), device="cuda")
    assert torch.equal(G0.apply(B), G1.apply(B))
    x0, it0, rr0, _ = G0.pcg(B, rtol=1e-10, maxit=500)
    x1, it1, rr1, _ = G1.pcg(B, rtol=1e-10, maxit=500)
    assert np.array_equal(it0, it1) and np.array_equal(rr0, rr1)
    assert torch.equal(x0, x1)
    # the solve workspaces came from the hook too
    assert hook.held > held_after_factor
    # new values of the same pattern
    pb2 = P.diffusion2d(64, 1.0, 4, leaf_size=8)
    v2 = torch.as_tensor(pb2.val, device="cuda")
    G0.refactor(v2)
    G1.refactor(v2)
    assert torch.equal(G0.apply(B), G1.apply(B))
    G1.close()
    torch.cuda.synchronize()
    assert hook.held == 0 and not hook.blocks and not hook.errors
    G0.close()


def test_hook_without_memory_fails_with_oom_and_leaks_nothing():
    torch = need_gpu()
    pb = P.diffusion2d(48, 1.0, 5, leaf_size=8)
    # too little for the factor arenas: the create fails and returns what it took
    small = _lib.DeviceAllocator(limit=1 << 20)
    with pytest.raises(_lib.HsError) as ei:
        _factor(pb, _lib.HS_PREC_F32, small)
    assert ei.value.code == _lib.HS_ERR_OOM
    assert "allocator hook" in str(ei.value)
    torch.cuda.synchronize()
    assert small.held == 0 and not small.blocks
    # no room left for the PCG workspace after the factorization: the solve
    # fails, and succeeds once the hook has memory again
    hook = _lib.DeviceAllocator()
    G = _factor(pb, _lib.HS_PREC_F32, hook)
    hook.limit = hook.held
    b = torch.as_tensor(P.rhs(pb.n, 9), device="cuda")
    with pytest.raises(_lib.HsError) as ei:
        G.pcg(b, rtol=1e-10, maxit=500)
    assert ei.value.code == _lib.HS_ERR_OOM
    hook.limit = None
    x, it, rr, code = G.pcg(b, rtol=1e-10, maxit=500)
    assert code == _lib.HS_OK and rr[0] <= 1e-10
    ref = _factor(pb, _lib.HS_PREC_F32)
    xr, itr, _, _ = ref.pcg(b, rtol=1e-10, maxit=500)
    assert torch.equal(x, xr) and np.array_equal(it, itr)
    G.close()
    ref.close()
    torch.cuda.synchronize()
    assert hook.held == 0 and not hook.blocks


def test_batched_handles_share_one_hook():
    torch = need_gpu()
    pbs = [P.diffusion2d(side, 1.0, 10 + side, leaf_size=8) for side in (32, 48, 40)]
    hook = _lib.DeviceAllocator()
    probs = [(*to_dev(pb), pb.perm, pb.leaf_ptr) for pb in pbs]
    fs, status = _lib.factor_batch(probs, 1e-2, _lib.HS_GC_CONSTANT, _lib.HS_PREC_F32, allocator=hook)
    assert list(status) == [0, 0, 0]
    assert hook.held > 0
    for pb, f in zip(pbs, fs):
        b = torch.as_tensor(P.rhs(pb.n, 2), device="cuda")
        alone = _factor(pb, _lib.HS_PREC_F32)
        assert torch.equal(f.apply(b), alone.apply(b))
        alone.close()
    for f in fs:
        f.close()
    torch.cuda.synchronize()
    assert hook.held == 0 and not hook.blocks


def test_serving_charges_the_bytes_the_hooks_count():
    """The serving loop charges each resident factorization what its handle's
    hook counts (exact), plus a reservation that covers the solve workspaces
    at the largest right-hand-side batch; every block is back after the run."""
    torch = need_gpu()
    from paper_1611_03189_gb300 import serving as S

    hooks = []

    class Recording(S.CudaBackend):
        def factor(self, stream, pb):
            f, nbytes = super().factor(stream, pb)
            hooks.append((f._alloc, nbytes))
            return f, nbytes

    reqs = S.poisson_stream(16, rate=400.0, seed=5, sides=(10, 16), s=2.0, leaf=64, p_factor=0.25)
    srv = S.Server(8 << 30, slots=2, max_rhs=16, backend=Recording())
    res = srv.run(reqs, realtime=False)
    assert all(r.status == _lib.HS_OK for r in res), [r.error for r in res if r.status]
    assert hooks and all(nb > 0 for _, nb in hooks)
    assert srv.overgrown == 0
    torch.cuda.synchronize()
    assert all(h.held == 0 and not h.blocks for h, _ in hooks)
