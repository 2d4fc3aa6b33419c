"""Parity at the benchmark's full size: 512 x 512 diffusion, s = 1, leaves of
16, eps = 1e-2, GC-constant -- the configuration bench.py times -- against the
whole FP64 oracle factorization of the same matrix (about 25 s on one core).

* FP64 factor: the rank of every super node of every level equals the
  oracle's, except where a singular value lies within 1e-10 relative of the
  truncation threshold (Sec. 3.2; the exemption north of the rank rule);
  the apply matches element by element within 1e-10 per right-hand side
  (Algorithm 2); PCG takes the oracle's iteration count +-1 and its solution
  is within 1e-10 of the oracle's iterate after the same number of
  iterations (Sec. 7: relative residual 1e-10).
* Properties that hold at any size: PCG reaches 1e-10 with the FP32 factor
  too and its solution agrees with the FP64 one; the FP64 preconditioner is
  symmetric and positive and keeps the constant vector (Sec. 6).

Collected after the other parity tests (only the allocation-free apply's
file comes later), so that a failure here skips none of them.
"""
import numpy as np
import pytest

from oracle import hsolver as H
from paper_1611_03189_gb300 import _lib
from paper_1611_03189_gb300 import problems as P

from gpu_util import elem, gpu_factor, need_gpu, rel

pytestmark = pytest.mark.gpu

EPS = 1e-2


@pytest.fixture(scope="module")
def workload():
    need_gpu()
    pb = P.diffusion2d(512, 1.0, 0, leaf_size=16)
    F = H.factor(pb.n, pb.rowptr, pb.col, pb.val, pb.perm, pb.leaf_ptr, EPS, H.GC_CONSTANT)
    G = gpu_factor(pb, EPS, H.GC_CONSTANT, prec=_lib.HS_PREC_F64)
    yield pb, F, G
    G.close()


def test_all_levels_ranks_match_oracle(workload):
    pb, F, G = workload
    bad, exempt, total = [], 0, 0
    for lv in F.levels:
        g = G.ranks(lv.level)
        for rec in lv.supers:
            want = rec.k if rec.wsep else -1
            total += 1
            if g[rec.key] != want:
                if rec.margin < 1e-10:
                    exempt += 1
                else:
                    bad.append((lv.level, rec.key, want, int(g[rec.key]), rec.margin))
    assert total > 16000
    assert bad == [], bad[:5]


def test_apply_elementwise_matches_oracle(workload):
    import torch

    pb, F, G = workload
    B = P.rhs(pb.n, 21, nrhs=2)
    zg = G.apply(torch.as_tensor(B.T.copy(), device="cuda")).cpu().numpy().T
    assert elem(zg, H.apply(F, B)) <= 1e-10


def test_pcg_matches_oracle(workload):
    import torch

    pb, F, G = workload
    b = P.rhs(pb.n, 1000)
    xo, ito, rro = H.pcg(F, pb.rowptr, pb.col, pb.val, b)
    x, it, rr, code = G.pcg(torch.as_tensor(b, device="cuda"), rtol=1e-10, maxit=500)
    assert code == _lib.HS_OK and rr[0] <= 1e-10
    its = int(it[0])
    assert abs(its - ito) <= 1
    if its != ito:
        xo, done, _ = H.pcg(F, pb.rowptr, pb.col, pb.val, b, rtol=1e-300, maxit=its)
        assert done == its
    assert rel(x.cpu().numpy(), xo) <= 1e-10


def test_bench_configuration_properties(workload):
    import torch

    pb, _, G64 = workload
    b = torch.as_tensor(P.rhs(pb.n, 1000), device="cuda")
    G32 = gpu_factor(pb, EPS, H.GC_CONSTANT, prec=_lib.HS_PREC_F32)
    x32, it32, rr32, _ = G32.pcg(b)
    x64, it64, rr64, _ = G64.pcg(b)
    assert rr32[0] <= 1e-10 and rr64[0] <= 1e-10
    assert int(it32[0]) <= 60 and abs(int(it32[0]) - int(it64[0])) <= 2
    # both meet the residual bar; their difference is bounded by kappa(A) x 2e-10
    # (kappa ~ 1e5 here), and is far below it in practice
    assert rel(x32.cpu().numpy(), x64.cpu().numpy()) <= 1e-6
    # GC-constant keeps the constant vector: A_H^-1 (A 1) = 1 (FP64 factor)
    A = pb.to_scipy()
    one = np.ones(pb.n)
    z = G64.apply(torch.as_tensor(A @ one, device="cuda")).cpu().numpy()
    assert elem(z, one) <= 1e-8
    # symmetric and positive definite, on random vectors
    rng = np.random.default_rng(5)
    U = rng.standard_normal((4, pb.n))
    Z = G64.apply(torch.as_tensor(U, device="cuda")).cpu().numpy()
    Q = U @ Z.T
    d = np.sqrt(np.outer(np.diag(Q), np.diag(Q)))
    assert np.all(np.diag(Q) > 0)
    # rounding of an apply is about u ||A_H^-1|| ||u||^2 times the depth, while
    # u^T A_H^-1 u is about ||u||^2 times the mean eigenvalue of A_H^-1
    assert np.max(np.abs(Q - Q.T) / d) <= 1e-8
    G32.close()
