"""GMRES on the GPU (hs_gmres), the outer solver of the paper's experiments
(Sec. 7, Tables 2-5), against the oracle's GMRES on the same inputs.

Bars: Arnoldi step counts within +-1 of the oracle; true relative residual
<= 2e-10 (the stopping test uses the least-squares estimate at 1e-10); x
within 1e-8 of the oracle's when the counts agree; no more steps than PCG
(both search the same Krylov space, GMRES minimises the residual)."""
import numpy as np
import pytest

from oracle import hsolver as H
from paper_1611_03189_gb300 import _lib
from paper_1611_03189_gb300 import problems as P

from gpu_util import gpu_factor, need_gpu, oracle_factor, rel

pytestmark = pytest.mark.gpu

CASES = [
    ("poisson2d 32 leaf8", lambda: P.poisson2d(32, leaf_size=8)),
    ("diffusion2d 64 s1", lambda: P.diffusion2d(64, 1.0, 0, leaf_size=16)),
    ("poisson3d 16 leaf64", lambda: P.poisson3d(16, leaf_size=64)),
]


@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("variant", [H.LORASP, H.GC_CONSTANT])
def test_gmres_matches_oracle(name, maker, variant):
    torch = need_gpu()
    pb = maker()
    F = oracle_factor(pb, 0.1, variant)
    G = gpu_factor(pb, 0.1, variant)
    b = P.rhs(pb.n, 3)
    xo, ito, _ = H.gmres_solve(F, pb.rowptr, pb.col, pb.val, b)
    xg, itg, rr, code = G.gmres(torch.as_tensor(b, device="cuda"))
    assert code == _lib.HS_OK and rr <= 2e-10
    assert abs(itg - ito) <= 1
    if itg == ito:
        assert rel(xg.cpu().numpy(), xo) <= 1e-8
    _, itc, _, _ = G.pcg(torch.as_tensor(b, device="cuda"))
    assert itg <= int(itc[0]) + 1
    G.close()


def test_gmres_fp32_factor_and_restarts():
    torch = need_gpu()
    pb = P.diffusion2d(64, 1.0, 1, leaf_size=16)
    G = gpu_factor(pb, 1e-2, H.GC_CONSTANT, prec=1)
    b = torch.as_tensor(P.rhs(pb.n, 4), device="cuda")
    x0, it0, rr0, code = G.gmres(b)
    assert code == _lib.HS_OK and rr0 <= 2e-10
    # a restart length beyond the step count changes nothing
    x1, it1, rr1, _ = G.gmres(b, restart=it0 + 3)
    assert it1 == it0 and np.array_equal(x1.cpu().numpy(), x0.cpu().numpy())
    # short cycles still converge, in more steps
    x2, it2, rr2, code2 = G.gmres(b, restart=4, maxit=400)
    assert code2 == _lib.HS_OK and rr2 <= 2e-10 and it2 >= it0
    assert rel(x2.cpu().numpy(), x0.cpu().numpy()) <= 1e-7
    G.close()


def test_gmres_exact_preconditioner_and_no_convergence():
    torch = need_gpu()
    pb = P.poisson2d(32, leaf_size=8)
    G = gpu_factor(pb, 0.0, H.GC_CONSTANT)
    b = torch.as_tensor(P.rhs(pb.n, 6), device="cuda")
    x, it, rr, code = G.gmres(b)
    assert code == _lib.HS_OK and it == 1 and rr <= 1e-11
    G.close()
    G = gpu_factor(pb, 0.3, H.LORASP)
    x, it, rr, code = G.gmres(b, maxit=2, raise_on_fail=False)
    assert code == _lib.HS_ERR_NO_CONVERGENCE and it == 2 and rr > 1e-10
    # a zero right-hand side returns x = 0 at once
    x, it, rr, code = G.gmres(torch.zeros(pb.n, dtype=torch.float64, device="cuda"))
    assert code == _lib.HS_OK and it == 0 and float(x.abs().max()) == 0.0
    G.close()
