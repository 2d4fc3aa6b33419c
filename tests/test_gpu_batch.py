"""Batched factorization: independent problems of different sizes factored in
lock step (one launch per kernel kind and step for all of them) give each
problem the factorization it gets alone, bit for bit; a problem that fails
leaves the batch without disturbing the others."""
import numpy as np
import pytest

from oracle import hsolver as H
from paper_1611_03189_gb300 import _lib
from paper_1611_03189_gb300 import problems as P

from gpu_util import elem, gpu_factor, need_gpu, oracle_factor, rel, to_dev

pytestmark = pytest.mark.gpu


def _problems():
    # uneven sizes and depths: 2D sides 20..72 (levels 5..9) and one 3D grid
    pbs = [P.diffusion2d(side, 1.0, seed, leaf_size=16) for seed, side in enumerate((20, 72, 33, 48, 64))]
    pbs.append(P.poisson3d(12, leaf_size=64))
    return pbs


def _batch_args(pbs):
    return [to_dev(pb) + (pb.perm, pb.leaf_ptr) for pb in pbs]


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
def test_batch_equals_each_problem_alone(prec):
    torch = need_gpu()
    pbs = _problems()
    fs, status = _lib.factor_batch(_batch_args(pbs), 1e-2, H.GC_CONSTANT, prec)
    assert list(status) == [0] * len(pbs)
    for pb, f in zip(pbs, fs):
        g = gpu_factor(pb, 1e-2, H.GC_CONSTANT, prec=prec)
        B = torch.as_tensor(P.rhs(pb.n, 9, nrhs=2).T.copy(), device="cuda")
        assert np.array_equal(f.apply(B).cpu().numpy(), g.apply(B).cpu().numpy())
        for lv in range(2, int(np.log2(len(pb.leaf_ptr) - 1)) + 1):
            assert np.array_equal(f.ranks(lv), g.ranks(lv))
        x, it, rr, _ = f.pcg(B[0].clone(), rtol=1e-10, maxit=300)
        assert rr[0] <= 1e-10
        g.close()
        f.close()


def test_batch_matches_oracle_fp64():
    torch = need_gpu()
    pbs = _problems()[:3]
    fs, status = _lib.factor_batch(_batch_args(pbs), 1e-2, H.GC_CONSTANT, 0)
    for pb, f in zip(pbs, fs):
        F = oracle_factor(pb, 1e-2, H.GC_CONSTANT)
        B = P.rhs(pb.n, 4, nrhs=2)
        zg = f.apply(torch.as_tensor(B.T.copy(), device="cuda")).cpu().numpy().T
        assert elem(zg, H.apply(F, B)) <= 1e-10
        f.close()


def test_refactor_batch_equals_fresh_batch():
    torch = need_gpu()
    pbs = _problems()[:4]
    new = [P.diffusion2d(int(round(np.sqrt(pb.n))), 1.0, 50 + i, leaf_size=16) for i, pb in enumerate(pbs)]
    fs, _ = _lib.factor_batch(_batch_args(pbs), 1e-2, H.GC_CONSTANT, 1)
    status = _lib.refactor_batch(fs, [torch.as_tensor(pb.val, device="cuda") for pb in new])
    assert list(status) == [0] * 4
    fresh, _ = _lib.factor_batch(_batch_args(new), 1e-2, H.GC_CONSTANT, 1)
    for pb, a, b in zip(new, fs, fresh):
        r = torch.as_tensor(P.rhs(pb.n, 1), device="cuda")
        assert np.array_equal(a.apply(r).cpu().numpy(), b.apply(r).cpu().numpy())
        a.close()
        b.close()


def test_failed_problem_leaves_the_batch():
    """A 16 x 16 diffusion field with s = 3 is not SPD under GC at eps = 0.1 (a
    property of the method, confirmed by the dense emulator in the oracle
    tests); its neighbours in the batch still factor correctly."""
    torch = need_gpu()
    bad = P.diffusion2d(16, 3.0, 2, leaf_size=8)
    with pytest.raises(H.NotSPD):
        oracle_factor(bad, 1e-1, H.GC_CONSTANT)
    good = _problems()[:2]
    pbs = [good[0], bad, good[1]]
    fs, status = _lib.factor_batch(_batch_args(pbs), 1e-1, H.GC_CONSTANT, 0)
    assert list(status) == [0, _lib.HS_ERR_NOT_SPD, 0]
    assert fs[1] is None
    for pb, f in ((good[0], fs[0]), (good[1], fs[2])):
        g = gpu_factor(pb, 1e-1, H.GC_CONSTANT)
        r = torch.as_tensor(P.rhs(pb.n, 2), device="cuda")
        assert np.array_equal(f.apply(r).cpu().numpy(), g.apply(r).cpu().numpy())
        f.close()
        g.close()
