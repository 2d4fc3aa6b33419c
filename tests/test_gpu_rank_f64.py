"""The FP64 rank decision of the mixed-precision factors (hs_opts.rank_f64).

With rank_f64 an FP32 / TF32 / BF16 factor forms each node's Gram matrix
A_sw A_sw^T in FP64 from FP64 copies of its FP32 blocks, eigen-decomposes it
in FP64 and decides the rank there (Sec. 3.2 threshold sigma > eps ||A_sw||;
Sec. 6 for GC); only the elimination stays in the factor precision.

What bounds the agreement with the FP64 oracle is then the FP32 storage of the
blocks, not the FP32 eigen-solve.  A first-level A_sw is a fill block made by
one FP32 Schur update over an m x m pivot, so its entries carry a relative
error of order m u_32, and a singular value moves by that much of ||A_sw||:
a rank can differ from the oracle's only where the oracle's margin (the
distance of the nearest singular value from the threshold, relative to it) is
below delta = 64 m u_32 / eps.  The plain FP32 factor's own eigen-solve
resolves only delta_32 = (w + m) u_32 / eps^2, which at eps = 1e-3 exempts
every node.  Above the first level the blocks also carry the rounding of the
earlier levels; there, as for the plain FP32 factor, at most 2% of the super
nodes may differ.  Every factor must still take FP64 PCG to 1e-10.
"""
import numpy as np
import pytest

from oracle import hsolver as H
from paper_1611_03189_gb300 import _lib
from paper_1611_03189_gb300 import problems as P

from gpu_util import need_gpu, oracle_factor, to_dev

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24

CASES = [
    ("poisson2d 32 leaf8", lambda: P.poisson2d(32, leaf_size=8)),
    ("diffusion2d 64 s1", lambda: P.diffusion2d(64, 1.0, 0, leaf_size=16)),
    ("poisson3d 16 leaf64", lambda: P.poisson3d(16, leaf_size=64)),
]


def _factor(pb, eps, variant, prec, rank_f64):
    rp, ci, va = to_dev(pb)
    return _lib.Factor(rp, ci, va, pb.perm, pb.leaf_ptr, eps, variant, prec, rank_f64=rank_f64)


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3])
def test_fp64_rank_decision_of_the_fp32_factor_matches_the_oracle(eps):
    need_gpu()
    total = bad_all = 0
    for name, maker in CASES:
        pb = maker()
        for variant in (H.LORASP, H.GC_CONSTANT):
            F = oracle_factor(pb, eps, variant)
            G = _factor(pb, eps, variant, _lib.HS_PREC_F32, True)
            first = F.levels[0]
            for lv in F.levels:
                g = G.ranks(lv.level)
                for rec in lv.supers:
                    want = rec.k if rec.wsep else -1
                    total += 1
                    if g[rec.key] == want:
                        continue
                    bad_all += 1
                    if lv is first:
                        delta = 64 * rec.m * U32 / eps
                        assert rec.margin < delta, (name, variant, lv.level, rec.key, want, int(g[rec.key]),
                                                    rec.margin, delta)
            G.close()
    assert bad_all <= 0.02 * total, (bad_all, total)


@pytest.mark.parametrize("prec", [_lib.HS_PREC_F32, _lib.HS_PREC_TF32, _lib.HS_PREC_BF16])
@pytest.mark.parametrize("name,maker", [CASES[1], CASES[2]], ids=[CASES[1][0], CASES[2][0]])
def test_mixed_factors_with_fp64_ranks_reach_fp64_accuracy_under_pcg(name, maker, prec):
    torch = need_gpu()
    pb = maker()
    F = oracle_factor(pb, 1e-2, H.GC_CONSTANT)
    G = _factor(pb, 1e-2, H.GC_CONSTANT, prec, True)
    b = P.rhs(pb.n, 4)
    x, it, rr, code = G.pcg(torch.as_tensor(b, device="cuda"), rtol=1e-10, maxit=500)
    _, ito, _ = H.pcg(F, pb.rowptr, pb.col, pb.val, b)
    assert code == _lib.HS_OK and rr[0] <= 1e-10
    extra = {_lib.HS_PREC_F32: 5, _lib.HS_PREC_TF32: 4, _lib.HS_PREC_BF16: 8}[prec]
    assert int(it[0]) <= ito + extra, (int(it[0]), ito)
    x = x.cpu().numpy()
    true_rr = np.linalg.norm(b - pb.to_scipy() @ x) / np.linalg.norm(b)
    assert true_rr <= 1e-10, true_rr
    G.close()


def test_fp64_rank_decision_is_deterministic_and_off_for_the_fp64_factor():
    """Two factorizations with rank_f64 give the same bits; the FP64 factor
    ignores the option (it decides in FP64 anyway)."""
    torch = need_gpu()
    pb = CASES[1][1]()
    b = torch.as_tensor(P.rhs(pb.n, 6), device="cuda")
    G1 = _factor(pb, 1e-2, H.GC_CONSTANT, _lib.HS_PREC_F32, True)
    G2 = _factor(pb, 1e-2, H.GC_CONSTANT, _lib.HS_PREC_F32, True)
    assert torch.equal(G1.apply(b), G2.apply(b))
    D0 = _factor(pb, 1e-2, H.GC_CONSTANT, _lib.HS_PREC_F64, False)
    D1 = _factor(pb, 1e-2, H.GC_CONSTANT, _lib.HS_PREC_F64, True)
    assert torch.equal(D0.apply(b), D1.apply(b))
    for G in (G1, G2, D0, D1):
        G.close()
