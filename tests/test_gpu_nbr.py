"""The distance-2 neighbour rule (hs_clustering.nbr_dist = 2, the algebraic
stand-in for the geometric rule of the paper's experiments) on the GPU,
against the oracle: equal ranks, FP64 apply within 1e-10, PCG to 1e-10."""
import numpy as np
import pytest

from oracle import hsolver as H
from paper_1611_03189_gb300 import _lib
from paper_1611_03189_gb300 import problems as P

from gpu_util import elem, need_gpu, rel, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    ("poisson2d 32 leaf8", lambda: P.poisson2d(32, leaf_size=8)),
    ("diffusion2d 64 s1", lambda: P.diffusion2d(64, 1.0, 0, leaf_size=16)),
    ("poisson3d 16 leaf64", lambda: P.poisson3d(16, leaf_size=64)),
]


@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("variant", [H.LORASP, H.GC_CONSTANT])
def test_distance2_rule_matches_oracle(name, maker, variant):
    torch = need_gpu()
    pb = maker()
    F = H.factor(pb.n, pb.rowptr, pb.col, pb.val, pb.perm, pb.leaf_ptr, 0.1, variant, nbr_dist=2)
    rp, ci, va = to_dev(pb)
    G = _lib.Factor(rp, ci, va, pb.perm, pb.leaf_ptr, 0.1, variant, _lib.HS_PREC_F64, nbr_dist=2)
    for lv in F.levels:
        g = G.ranks(lv.level)
        for rec in lv.supers:
            assert g[rec.key] == (rec.k if rec.wsep else -1), (lv.level, rec.key)
    B = P.rhs(pb.n, 7, nrhs=2)
    zg = G.apply(torch.as_tensor(B.T.copy(), device="cuda")).cpu().numpy().T
    assert elem(zg, H.apply(F, B)) <= 1e-10
    x, it, rr, _ = G.pcg(torch.as_tensor(B[:, 0].copy(), device="cuda"))
    xo, ito, _ = H.pcg(F, pb.rowptr, pb.col, pb.val, B[:, 0])
    assert rr[0] <= 1e-10 and abs(int(it[0]) - ito) <= 1
    G.close()
