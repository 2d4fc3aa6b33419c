"""The solve's recorded CUDA graphs replay exactly the launches they replace,
and a right-hand side's result does not depend on its batch.

hs_apply and each PCG iteration after the first run as recorded graphs by
default; HS_APPLY_GRAPH=0 selects direct launches.  The kernels, launch shapes
and order are the same either way, so the results must agree bit for bit.
The direct run happens in a child process, because the switch is read once per
process.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1611_03189_gb300 import problems as P

from gpu_util import gpu_factor, need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
from paper_1611_03189_gb300 import problems as P
from gpu_util import gpu_factor
pb = P.diffusion2d(64, 1.0, 3, leaf_size=16)
out = {{}}
for prec in (0, 1):
    G = gpu_factor(pb, 1e-2, 1, prec=prec)
    B = torch.as_tensor(P.rhs(pb.n, 5, nrhs=3).T.copy(), device="cuda")
    z = G.apply(B).cpu().numpy()
    x, it, rr, _ = G.pcg(B[:2].clone(), rtol=1e-10, maxit=500)
    out[str(prec)] = {{"z": z.tobytes().hex(), "x": x.cpu().numpy().tobytes().hex(), "it": it.tolist()}}
    G.close()
print(json.dumps(out))
"""


def _run(pb, prec, torch):
    G = gpu_factor(pb, 1e-2, 1, prec=prec)
    B = torch.as_tensor(P.rhs(pb.n, 5, nrhs=3).T.copy(), device="cuda")
    z = G.apply(B).cpu().numpy()
    z2 = G.apply(B).cpu().numpy()          # second replay of the same graph
    x, it, rr, _ = G.pcg(B[:2].clone(), rtol=1e-10, maxit=500)
    G.close()
    return z, z2, x.cpu().numpy(), it.tolist()


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
def test_graph_replay_is_bitwise_equal_to_direct_launches(prec):
    torch = need_gpu()
    pb = P.diffusion2d(64, 1.0, 3, leaf_size=16)
    z, z2, x, it = _run(pb, prec, torch)
    assert np.array_equal(z, z2)
    env = dict(os.environ, HS_APPLY_GRAPH="0")
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])[str(prec)]
    assert bytes.fromhex(d["z"]) == z.tobytes()
    assert bytes.fromhex(d["x"]) == x.tobytes()
    assert d["it"] == it


def test_graphs_follow_a_refactor():
    """A refactor changes ranks and record pointers; the recorded graphs must
    be dropped, so the apply after it equals a fresh factor's apply."""
    torch = need_gpu()
    pa = P.diffusion2d(64, 1.0, 0, leaf_size=16)
    pb = P.diffusion2d(64, 2.0, 1, leaf_size=16)
    B = torch.as_tensor(P.rhs(pa.n, 2).T.copy(), device="cuda").squeeze(0)
    G = gpu_factor(pa, 1e-2, 1, prec=1)
    G.apply(B)
    G.pcg(B, rtol=1e-10, maxit=500)
    G.refactor(torch.as_tensor(pb.val, device="cuda"))
    z_re = G.apply(B).cpu().numpy()
    x_re, it_re, _, _ = G.pcg(B, rtol=1e-10, maxit=500)
    F = gpu_factor(pb, 1e-2, 1, prec=1)
    z_fresh = F.apply(B).cpu().numpy()
    x_fresh, it_fresh, _, _ = F.pcg(B, rtol=1e-10, maxit=500)
    assert np.array_equal(z_re, z_fresh)
    assert np.array_equal(x_re.cpu().numpy(), x_fresh.cpu().numpy())
    assert it_re.tolist() == it_fresh.tolist()
    G.close()
    F.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
def test_batched_rhs_bitwise_equal_to_solo_solves(prec):
    """A right-hand side's PCG result does not depend on which others share
    its batch: the apply is column-wise and every PCG reduction visits rows in
    an order that depends on n alone."""
    torch = need_gpu()
    pb = P.diffusion2d(64, 2.0, 4, leaf_size=16)
    G = gpu_factor(pb, 1e-2, 1, prec=prec)
    B = torch.as_tensor(P.rhs(pb.n, 11, nrhs=5).T.copy(), device="cuda")
    X, its, rrs, _ = G.pcg(B.clone(), rtol=1e-10, maxit=500)
    X = X.cpu().numpy()
    for j in range(5):
        x, it, rr, _ = G.pcg(B[j].clone(), rtol=1e-10, maxit=500)
        assert np.array_equal(x.cpu().numpy().reshape(-1), X[j]), j
        assert int(it[0]) == int(its[j])
    G.close()
