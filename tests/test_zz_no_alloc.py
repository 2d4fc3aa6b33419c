"""hs_apply_static, the allocation-free apply, against hs_apply.

Some callers cannot allocate device memory at the moment they solve -- a
service whose device footprint is fixed at start-up, or code running where a
cudaMalloc could block behind other work or is not permitted; they apply the
preconditioner through hs_apply_static, whose workspace is a static device
array inside the library.  It runs the same kernels in the same order as
hs_apply, so its result must equal hs_apply's bit for bit on the same
factorization, call after call, and requests that do not fit the array must be
refused with HS_ERR_CAPACITY.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1611_03189_gb300 import _lib
from paper_1611_03189_gb300 import problems as P

from gpu_util import gpu_factor, need_gpu

pytestmark = pytest.mark.gpu


def _apply_static(G, r, torch):
    r = r.contiguous()
    nrhs = 1 if r.dim() == 1 else r.shape[0]
    z = torch.empty_like(r)
    code = _lib.lib().hs_apply_static(G._h, r.data_ptr(), z.data_ptr(), nrhs, G.n,
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, z


@pytest.mark.parametrize("prec", [_lib.HS_PREC_F64, _lib.HS_PREC_F32])
def test_static_apply_matches_apply_on_two_calls_in_a_row(prec):
    torch = need_gpu()
    pb = P.diffusion2d(48, 1.0, 2, leaf_size=8)
    G = gpu_factor(pb, 1e-2, _lib.HS_GC_CONSTANT, prec=prec)
    # first call: three right-hand sides; second call: one, so stale workspace
    # contents of the first call would show up in the second result
    for seed, nrhs in ((11, 3), (12, 1)):
        b = P.rhs(pb.n, seed, nrhs=nrhs)
        r = torch.as_tensor(b.T.copy() if nrhs > 1 else b, device="cuda")
        z_ref = G.apply(r).cpu().numpy()
        code, z = _apply_static(G, r, torch)
        torch.cuda.synchronize()
        assert code == _lib.HS_OK, _lib.lib().hs_last_error().decode()
        assert torch.equal(z.cpu(), torch.as_tensor(z_ref))


def test_static_apply_refuses_requests_beyond_its_buffer():
    torch = need_gpu()
    pb = P.poisson2d(192, leaf_size=16)   # n = 36864: 64 rhs need > 18 MB of workspace
    G = gpu_factor(pb, 1e-2, _lib.HS_GC_CONSTANT, prec=_lib.HS_PREC_F64)
    r = torch.as_tensor(P.rhs(pb.n, 3, nrhs=64).T.copy(), device="cuda")
    code, _ = _apply_static(G, r, torch)
    assert code == _lib.HS_ERR_CAPACITY
    assert "static buffer holds" in _lib.lib().hs_last_error().decode()
    # a request that fits still works afterwards
    code, z = _apply_static(G, r[0].contiguous(), torch)
    assert code == _lib.HS_OK
    assert torch.equal(z, G.apply(r[0].contiguous()))
