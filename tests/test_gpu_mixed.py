"""The mixed-precision factorizations against the FP64 oracle.

HS_PREC_TF32 and HS_PREC_BF16 keep blocks and records in FP32 and run the
elimination's contractions (L^-1 U and its CholQR, L^-1 A_sN, M_ss, P_ss,
A_Nr, A_rr, the Schur update; Sec. 3.2, Appendix A) on the tensor cores, each
task through the variant the GEMM autotuner picked for its shape.  The outer
FP64 PCG acts as iterative refinement (Sec. 7 stopping rule), so:

* PCG reaches a true relative residual <= 1e-10 and its solution agrees with
  the oracle's to within kappa(A) x 2e-10 (both meet the residual bar; 1e-8
  covers kappa(A) <= 5e7, far above these problems' ~1e4);
* TF32 needs at most two iterations more than the oracle; BF16 (unit
  roundoff 2^-8) at most six more on these problems;
* the apply itself differs from the FP64 A_H^-1 r by the operand rounding
  (TF32 unit roundoff 2^-11) amplified by the pivot blocks' conditioning:
  within 0.1 element by element (measured <= 3.3e-2); with the 3xTF32 split
  (HS_PREC_TF32X3, near-FP32 products) within 5e-3, the FP32 factor's level
  (measured <= 2.5e-3), and at most one iteration more than the oracle.
HS_GEMM_ROUTE forces every task onto one kernel, so that the tensor-core
kernel itself is exercised on these small problems (the autotuner sends most
of their tiny tasks to the CUDA-core kernel).
"""
import os
import subprocess
import sys

import pytest

from paper_1611_03189_gb300 import _lib

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))

CODE = """
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
sys.path.insert(0, {here!r})
from gpu_util import elem, gpu_factor, oracle_factor, rel
from oracle import hsolver as H
from paper_1611_03189_gb300 import problems as P, _lib
cases = [("poisson2d 64 leaf16", lambda: P.poisson2d(64, leaf_size=16)),
         ("diffusion2d 64 s1", lambda: P.diffusion2d(64, 1.0, 0, leaf_size=16)),
         ("poisson3d 16 leaf64", lambda: P.poisson3d(16, leaf_size=64))]
prec = {prec}
for name, maker in cases:
    pb = maker()
    for variant in (H.LORASP, H.GC_CONSTANT):
        for eps in (1e-1, 1e-2):
            F = oracle_factor(pb, eps, variant)
            G = gpu_factor(pb, eps, variant, prec=prec)
            info = G.info()
            assert info["tc_launches"] > 0 or {route!r} in ("simt", "auto"), (name, info["tc_launches"])
            b = P.rhs(pb.n, 0)
            xo, ito, _ = H.pcg(F, pb.rowptr, pb.col, pb.val, b)
            x, it, rr, code = G.pcg(torch.as_tensor(b, device="cuda"), rtol=1e-10, maxit=500)
            x = x.cpu().numpy()
            true_rr = np.linalg.norm(b - pb.to_scipy() @ x) / np.linalg.norm(b)
            assert code == 0 and true_rr <= 1e-10, (name, variant, eps, code, true_rr)
            assert int(it[0]) <= ito + {extra_it}, (name, variant, eps, int(it[0]), ito)
            assert rel(x, xo) <= 1e-8, (name, variant, eps, rel(x, xo))
            if prec in (_lib.HS_PREC_TF32, _lib.HS_PREC_TF32X3):
                B = P.rhs(pb.n, 7, nrhs=2)
                zg = G.apply(torch.as_tensor(B.T.copy(), device="cuda")).cpu().numpy().T
                e = elem(zg, H.apply(F, B))
                assert e <= (0.1 if prec == _lib.HS_PREC_TF32 else 5e-3), (name, variant, eps, e)
            G.close()
print("ok")
"""


def _run(prec, route, extra_it):
    need_gpu()
    env = dict(os.environ)
    env.pop("HS_GEMM_ROUTE", None)
    if route != "auto":
        env["HS_GEMM_ROUTE"] = route
    code = CODE.format(root=os.path.dirname(HERE), here=HERE, prec=prec, route=route, extra_it=extra_it)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]


@pytest.mark.parametrize("route", ["auto", "tc64", "tc128"])
def test_tf32_factor_meets_the_fp64_bar_under_pcg(route):
    _run(_lib.HS_PREC_TF32, route, 2)


@pytest.mark.parametrize("route", ["tc64", "tc128"])
def test_tf32x3_factor_meets_the_fp64_bar_under_pcg(route):
    _run(_lib.HS_PREC_TF32X3, route, 1)


def test_bf16_factor_meets_the_fp64_bar_under_pcg():
    _run(_lib.HS_PREC_BF16, "tc64", 6)


def test_autotuner_table():
    need_gpu()
    for prec in (_lib.HS_PREC_TF32, _lib.HS_PREC_BF16, _lib.HS_PREC_TF32X3):
        rows = _lib.gemm_tune_report(prec)
        assert len(rows) == 20
        for r in rows:
            assert r["route"] in (0, 64, 128)
            # the choice is the fastest, with a 15% handicap on the tensor-core variants
            eff = {0: r["ms_simt"], 64: 1.15 * r["ms_tc64"], 128: 1.15 * r["ms_tc128"]}
            assert min(eff.values()) > 0
            assert eff[r["route"]] <= min(eff.values()) * (1 + 1e-6)


def test_wait_that_runs_out_returns_timeout_and_the_device_stays_usable():
    """hs_opts.timeout_cycles bounds every wait of the tensor-core GEMM on its
    mbarriers.  With hs_test_wait_probe on, each launch first waits on a
    barrier that nothing arrives at: the factorization must fail with
    HS_ERR_TIMEOUT (no tensor-core work was issued; the kernel frees its
    tensor memory and returns), and with the probe off the next factorization
    and solve on the same device must work."""
    need_gpu()
    code = f"""
import sys, numpy as np, torch
sys.path.insert(0, {os.path.dirname(HERE)!r})
sys.path.insert(0, {HERE!r})
from gpu_util import to_dev
from paper_1611_03189_gb300 import problems as P, _lib
pb = P.poisson2d(64, leaf_size=16)
rp, ci, va = to_dev(pb)
_lib.lib().hs_test_wait_probe(1)
try:
    try:
        _lib.Factor(rp, ci, va, pb.perm, pb.leaf_ptr, 1e-2, _lib.HS_GC_CONSTANT, _lib.HS_PREC_TF32,
                    timeout_cycles=100000)
        raise SystemExit("no timeout")
    except _lib.HsError as e:
        assert e.code == _lib.HS_ERR_TIMEOUT, e
finally:
    _lib.lib().hs_test_wait_probe(0)
G = _lib.Factor(rp, ci, va, pb.perm, pb.leaf_ptr, 1e-2, _lib.HS_GC_CONSTANT, _lib.HS_PREC_TF32)
b = torch.as_tensor(P.rhs(pb.n, 0), device="cuda")
x, it, rr, code = G.pcg(b)
assert code == 0 and rr[0] <= 1e-10
print("ok")
"""
    env = dict(os.environ, HS_GEMM_ROUTE="tc64")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]
