"""The persistent apply (HS_APPLY_PERSISTENT=1): Algorithm 2's wave steps in
one cooperative launch per right-hand-side chunk, with bounded grid barriers.

* It runs the per-step kernels' arithmetic in the same order, so its result
  equals the default (graph of per-step launches) bit for bit, FP64 and FP32,
  one and several right-hand sides; and it is within 1e-10 of the oracle
  element by element (FP64).
* A barrier that runs out (hs_test_wait_probe) makes hs_pcg return
  HS_ERR_TIMEOUT; the next solve on the same handle works.
The switch is read once per process, so each case runs in a child process.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = """
import sys, numpy as np, torch
sys.path.insert(0, {root!r}); sys.path.insert(0, {here!r})
from gpu_util import to_dev
from paper_1611_03189_gb300 import problems as P, _lib
out = {{}}
for prec in (_lib.HS_PREC_F64, _lib.HS_PREC_F32):
    for name, pb in (("d64", P.diffusion2d(64, 1.0, 0, leaf_size=16)), ("p16", P.poisson3d(16, leaf_size=64))):
        rp, ci, va = to_dev(pb)
        G = _lib.Factor(rp, ci, va, pb.perm, pb.leaf_ptr, 1e-2, _lib.HS_GC_CONSTANT, prec)
        for nrhs in (1, 5):
            B = torch.as_tensor(P.rhs(pb.n, 3, nrhs=nrhs).T.copy(), device="cuda")
            out["%s_%d_%d" % (name, prec, nrhs)] = G.apply(B).cpu().numpy()
        x, it, rr, code = G.pcg(torch.as_tensor(P.rhs(pb.n, 1), device="cuda"))
        out["%s_%d_pcg" % (name, prec)] = x.cpu().numpy()
        out["%s_%d_it" % (name, prec)] = np.array([int(it[0]), code])
        G.close()
np.savez({path!r}, **out)
print("ok")
"""


def _child(path, persistent):
    env = dict(os.environ)
    env.pop("HS_APPLY_PERSISTENT", None)
    if persistent:
        env["HS_APPLY_PERSISTENT"] = "1"
    code = CHILD.format(root=ROOT, here=HERE, path=path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]
    return np.load(path)


def test_persistent_apply_equals_the_step_launches_bit_for_bit(tmp_path):
    need_gpu()
    a = _child(str(tmp_path / "steps.npz"), False)
    b = _child(str(tmp_path / "pers.npz"), True)
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k


def test_persistent_apply_matches_the_oracle():
    need_gpu()
    code = f"""
import sys, numpy as np, torch
sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {HERE!r})
from gpu_util import elem, gpu_factor, oracle_factor
from oracle import hsolver as H
from paper_1611_03189_gb300 import problems as P, _lib
pb = P.diffusion2d(64, 1.0, 0, leaf_size=16)
for variant in (H.LORASP, H.GC_CONSTANT):
    F = oracle_factor(pb, 1e-2, variant)
    G = gpu_factor(pb, 1e-2, variant)
    B = P.rhs(pb.n, 5, nrhs=3)
    zg = G.apply(torch.as_tensor(B.T.copy(), device="cuda")).cpu().numpy().T
    e = elem(zg, H.apply(F, B))
    assert e <= 1e-10, (variant, e)
    G.close()
print("ok")
"""
    env = dict(os.environ, HS_APPLY_PERSISTENT="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]


def test_persistent_barrier_that_runs_out_returns_timeout():
    need_gpu()
    code = f"""
import sys, numpy as np, torch
sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {HERE!r})
from gpu_util import to_dev
from paper_1611_03189_gb300 import problems as P, _lib
pb = P.poisson2d(64, leaf_size=16)
rp, ci, va = to_dev(pb)
# about 10 ms of SM clocks: far above a real barrier's wait, short for the probe's
G = _lib.Factor(rp, ci, va, pb.perm, pb.leaf_ptr, 1e-2, _lib.HS_GC_CONSTANT, _lib.HS_PREC_F32,
                timeout_cycles=20000000)
b = torch.as_tensor(P.rhs(pb.n, 0), device="cuda")
_lib.lib().hs_test_wait_probe(1)
try:
    try:
        G.pcg(b, maxit=3)
        raise SystemExit("no timeout")
    except _lib.HsError as e:
        assert e.code == _lib.HS_ERR_TIMEOUT, e
finally:
    _lib.lib().hs_test_wait_probe(0)
x, it, rr, code = G.pcg(b)
assert code == 0 and rr[0] <= 1e-10, (code, rr)
print("ok")
"""
    env = dict(os.environ, HS_APPLY_PERSISTENT="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]
