"""Benchmark of the GB300 hierarchical solver (factor + FP64 PCG to rel-res 1e-10).

Workload (default "diffusion2d_512"): 2D variable-coefficient diffusion,
5-point, 512 x 512 grid (n = 262144), a = exp(s g) with s = 1 and g a Gaussian
random field of length scale 8 cells, recursive-bisection leaves of 16
unknowns, truncation tolerance 1e-2, GC-constant compression, PCG to relative
residual 1e-10, b ~ N(0,1).  A step is one whole pass of the hot path: the
numeric factorization of a new matrix (same pattern, the field drawn from a new
seed) followed by one PCG solve with `--nrhs` right-hand sides.  The symbolic
plan is built once per pattern, before timing.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(rank 0 only), on a bounded sample of the same recipe.
"""
from __future__ import annotations

import argparse
import json
import math
import numpy as np
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (dimension, grid side, s, eps, leaf size); s = 0 is the constant-coefficient Poisson problem
    "diffusion2d_512": (2, 512, 1.0, 1e-2, 16),
    "diffusion2d_256": (2, 256, 1.0, 1e-2, 16),
    "poisson2d_64": (2, 64, 0.0, 1e-2, 16),
    "poisson3d_64": (3, 64, 0.0, 1e-2, 64),
    "poisson3d_32": (3, 32, 0.0, 1e-2, 64),
    "poisson3d_24": (3, 24, 0.0, 1e-2, 64),
}
# Workloads whose one-step oracle run exceeds a few minutes of one core are
# timed on a smaller grid of the same recipe and scaled by the unknown count
# (the 3D ones: the ranks grow with the grid there, so the scaled figure
# flatters the oracle and is labelled an estimate).  The 2D workloads are
# timed on the workload itself.
CPU_SAMPLE = {"poisson3d_64": "poisson3d_24", "poisson3d_32": "poisson3d_24"}
METRIC = "solves/s to rel-res 1e-10 (factor + PCG solve; mixed vs FP64 factor)"
# factor precisions by name (values of HS_PREC_*)
PRECS = {"f64": 0, "f32": 1, "tf32": 2, "bf16": 3, "tf32x3": 4}
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch unit
# of the roofline entries, from one ncu capture of the same bench command:
# "apply" per application (all its launches), "trunc" per launch group of the
# large-node truncation.  Each figure names the profiles/ summary that holds
# the capture and its command; a kernel changed since its capture has no
# entry here (traffic null).
TRAFFIC = {
    # profiles/traffic_diffusion2d_512_f32.md: one application = 181 launches
    # (455.6 MB read, 0.01 MB written); the large-node truncation of one
    # factorization = 193.5 MB over its 46 launch groups
    ("diffusion2d_512", "f32"): {"apply": 455.62e6, "trunc": 193.48e6 / 46},
}


def make_problem(name: str, seed: int):
    from paper_1611_03189_gb300 import problems as P

    dim, side, s, eps, leaf = WORKLOADS[name]
    if dim == 3:
        if s == 0.0:
            return P.poisson3d(side, leaf_size=leaf), eps
        return P.diffusion3d(side, s, seed, leaf_size=leaf), eps
    if s == 0.0:
        return P.poisson2d(side, leaf_size=leaf), eps
    return P.diffusion2d(side, s, seed, leaf_size=leaf), eps


def replica_seed(rank: int, k: int) -> int:
    """Coefficient-field seed of step k on replica `rank`: replicas solve
    different systems (the path has no data exchange; weak scaling)."""
    return rank * 1000 + k


def max_over_ranks(ms: float, dist, device=None) -> float:
    """The slowest rank's time: every rank contributes its own, all get the max."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, nrhs: int, ms: float) -> float:
    """Solves per second of the whole job: all replicas' solves over the slowest time."""
    return world * steps * nrhs / (ms / 1000.0)


def sample_for(name: str):
    """(sample workload, unknowns of the workload / unknowns of the sample)."""
    sample = CPU_SAMPLE.get(name, name)
    d, side, *_ = WORKLOADS[name]
    _, sside, *_ = WORKLOADS[sample]
    return sample, (side / sside) ** d


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out.name)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# the oracle (CPU baseline / reference arm): run in a child process with one thread
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import hsolver as H
import bench
times = []
iters = []
for k in range({reps}):
    pb, eps = bench.make_problem({name!r}, {seed0} + k)
    from paper_1611_03189_gb300 import problems as P
    b = P.rhs(pb.n, 1000 + k)
    t0 = time.perf_counter()
    F = H.factor(pb.n, pb.rowptr, pb.col, pb.val, pb.perm, pb.leaf_ptr, eps, H.GC_CONSTANT)
    x, it, rr = H.pcg(F, pb.rowptr, pb.col, pb.val, b, rtol=1e-10, maxit=1000)
    times.append(time.perf_counter() - t0)
    iters.append(it)
print(json.dumps({{"times": times, "iters": iters}}))
"""


def tensor_peak_for(prec: str, peaks: dict):
    """Dense tensor-core peak (TFLOP/s) for the operand type of a factor
    precision: the measured sustained BF16 figure (the GEMM runs inside a long
    step), times the nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s) for TF32."""
    bf16 = peaks.get("bf16_tflops_sustained")
    src = "measured sustained bf16 (MEASURED_PEAKS.json)"
    if not bf16:
        bf16, src = 1700.0, "fallback sustained bf16"
    if prec == "tf32":
        return bf16 * 1.1 / 2.25, src + " x nominal tf32/bf16 ratio 1.1/2.25"
    if prec == "tf32x3":
        return bf16 * 1.1 / 2.25 / 3, src + " x nominal tf32/bf16 ratio 1.1/2.25 / 3 (three MMAs per product)"
    if prec in ("f32", "f64"):
        return bf16, src + " (the contractions' peak if they ran as bf16 on tensor cores)"
    return bf16, src


def run_oracle(name: str, reps: int, seed0: int = 0) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, reps=reps, name=name, seed0=seed0)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(workload: str) -> dict:
    sample, scale = sample_for(workload)
    res = run_oracle(sample, 1, seed0=0)
    t = res["times"][0]
    if scale == 1.0:
        what = (f"one step of the workload itself ({workload}: factor of the seed-0 field + PCG solve of "
                f"1 rhs, {res['iters'][0]} iterations, {t:.1f} s), measured")
    else:
        what = (f"one factor + PCG solve (1 rhs) of the same recipe on the smaller grid {sample} "
                f"({t:.2f} s, {res['iters'][0]} iterations), scaled by the unknown count x{scale:g}: an estimate")
    return {"value": (1.0 / t) / scale, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": what,
            "sample_seconds": t, "measured": scale == 1.0}


def reference_arm(args) -> None:
    """The oracle (FP64, one core, in a child process) on the bench's own
    workload.  Each oracle step of the 2D workload takes about half a minute
    of one core, so min(steps, 2) steps are timed and no warm-up is run (the
    oracle has nothing to warm up); the line says so."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sample, scale = sample_for(args.workload)
    nsteps = max(1, min(args.steps, 2))
    res = run_oracle(sample, nsteps, seed0=0)
    times = res["times"]
    per = sum(times) / len(times)
    value = (1.0 / per) / scale
    measured = scale == 1.0
    sample_txt = (f"each step one factor + PCG solve (1 rhs) of the workload itself, {nsteps} steps timed "
                  f"(no warm-up: the oracle has none)" if measured else
                  f"each step one factor + PCG solve of the recipe on the smaller grid {sample}, "
                  f"scaled by the unknown count x{scale:g} (an estimate)")
    line = {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": nsteps, "warmup": 0,
        "requested": {"steps": args.steps, "warmup": args.warmup},
        "ms_per_step": per * 1000 * scale, "ms_per_step_measured": measured,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "nrhs": 1, "sample": sample, "factor_prec": "f64 (oracle)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample_txt},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "iterations": res["iters"],
        "step_seconds": times,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched: many independent 2D diffusion problems factored in lock step
# ---------------------------------------------------------------------------
def batched_arm(args) -> None:
    """Each step: the numeric factorization of all problems in lock step
    (hs_factor_refactor_batch: one launch per kernel kind and wave step for all
    of them), then a 4-RHS FP64 PCG solve of every problem, the solves spread
    over CUDA streams.  Compared with the same problems factored one by one."""
    import concurrent.futures as cf

    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03189_gb300 import _lib
    from paper_1611_03189_gb300 import problems as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    count, nrhs = args.batch_count, 4
    t_gen = time.perf_counter()
    sides = P.batched_sides(count, seed=3, lo=32, hi=256)
    pbs = [P.diffusion2d(side, 2.0, 7000 + i, leaf_size=16) for i, side in enumerate(sides)]
    t_gen = time.perf_counter() - t_gen
    devs = [(torch.as_tensor(pb.rowptr, device=dev), torch.as_tensor(pb.col, device=dev),
             torch.as_tensor(pb.val, device=dev)) for pb in pbs]
    rhs = [torch.as_tensor(P.rhs(pb.n, 100 + i, nrhs=nrhs).T.copy(), device=dev) for i, pb in enumerate(pbs)]
    prec = PRECS[args.prec]
    fs, status = _lib.factor_batch([d + (pb.perm, pb.leaf_ptr) for d, pb in zip(devs, pbs)], 1e-2,
                                   _lib.HS_GC_CONSTANT, prec, scale=args.scale)
    live = [i for i in range(count) if status[i] == _lib.HS_OK]
    streams = [torch.cuda.Stream(device=dev) for _ in range(8)]
    pool = cf.ThreadPoolExecutor(max_workers=len(streams))

    def solve_one(j):
        i = live[j]
        s = streams[j % len(streams)]
        with torch.cuda.stream(s):
            x, it, rr, code = fs[i].pcg(rhs[i], rtol=1e-10, maxit=1000, stream=s, raise_on_fail=False)
            s.synchronize()
        return int(it.max()), float(np.max(rr)), code

    def step():
        st = _lib.refactor_batch([fs[i] for i in live], [devs[i][2] for i in live])
        if any(int(c) != _lib.HS_OK for c in st):
            raise RuntimeError("a refactor in the batch failed")
        torch.cuda.synchronize()
        return list(pool.map(solve_one, range(len(live))))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = _lib.launch_count()
    w0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    res = []
    for _ in range(args.steps):
        res = step()
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    launches = _lib.launch_count() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # the factor part alone: batched vs one problem at a time
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _lib.refactor_batch([fs[i] for i in live], [devs[i][2] for i in live])
    torch.cuda.synchronize()
    batched_factor_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    for i in live:
        fs[i].refactor(devs[i][2])
    torch.cuda.synchronize()
    single_factor_ms = (time.perf_counter() - t0) * 1e3
    solves = len(live) * nrhs * args.steps
    line = {
        "metric": "solves/s to rel-res 1e-10 (batched factor + PCG, 4 rhs per problem)",
        "value": solves / (ms / 1000.0), "unit": "rhs solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.prec == "f64" else f"{args.prec}+f64", "data": "synthetic",
        "config": {"workload": f"batched_{count}", "problems": count, "sides": "log-uniform [32, 256]",
                   "s": 2.0, "leaf": 16, "eps": 1e-2, "variant": "GC-constant", "nrhs": nrhs,
                   "factor_prec": args.prec, "unknowns_total": int(sum(pb.n for pb in pbs)),
                   "diagonal_scaling": bool(args.scale),
                   "generation_s": t_gen, "pcg_streams": len(streams),
                   "l2": "inputs larger than L2 (factor records > 129 MB)"},
        "problems_not_spd": int(count - len(live)),
        "systems_per_s": len(live) * args.steps / (ms / 1000.0),
        "factor_batched_ms": batched_factor_ms, "factor_one_by_one_ms": single_factor_ms,
        "max_pcg_iterations": max(r[0] for r in res), "max_relres": max(r[1] for r in res),
        "gpu_launches": launches, "clocks": clk, "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    pool.shutdown()
    for f in fs:
        if f is not None:
            f.close()


# ---------------------------------------------------------------------------
# serving: a Poisson stream of 3D diffusion factor / solve requests
# ---------------------------------------------------------------------------
def gmres_table_arm(args) -> None:
    """The paper's headline experiment on the GPU (Sec. 7.1, Table 2): GMRES
    iterations to relative residual 1e-10 preconditioned by LoRaSp,
    GC-constant and GC-eigenvector (the smallest Laplacian eigenvector) at
    eps = 0.1, 0.2, 0.3, on the 2D constant-coefficient Poisson problem with
    leaves of 8 unknowns, for growing grids.  PCG iterations of the same
    factors are reported beside them.  One JSON line."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03189_gb300 import _lib
    from paper_1611_03189_gb300 import problems as P

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    prec = _lib.HS_PREC_F32 if args.table_prec == "f32" else _lib.HS_PREC_F64
    rows = []
    t0 = time.perf_counter()
    for side in (int(v) for v in args.table_sides.split(",")):
        pb = P.poisson2d(side, leaf_size=8)
        rp = torch.as_tensor(pb.rowptr, dtype=torch.int32, device=dev)
        ci = torch.as_tensor(pb.col, dtype=torch.int32, device=dev)
        va = torch.as_tensor(pb.val, dtype=torch.float64, device=dev)
        b = torch.as_tensor(P.rhs(pb.n, 0), device=dev)
        phi = P.laplacian_eigvec_2d(side, side)
        row = {"side": side, "n": pb.n, "depth": int(round(math.log2(len(pb.leaf_ptr) - 1)))}
        worst = 0.0
        for key, var, ph in (("lorasp", _lib.HS_LORASP, None), ("gc_constant", _lib.HS_GC_CONSTANT, None),
                             ("gc_eigenvector", _lib.HS_GC_USER, phi)):
            gm, cg = [], []
            for eps in (0.1, 0.2, 0.3):
                try:
                    G = _lib.Factor(rp, ci, va, pb.perm, pb.leaf_ptr, eps, var, prec, phi=ph, nbr_dist=args.table_nbr)
                except RuntimeError as e:   # a factorization that fails is reported, not fatal
                    gm.append(None)
                    cg.append(None)
                    row.setdefault("errors", []).append(f"{key} eps={eps}: {e}")
                    continue
                _, it, rr, _ = G.gmres(b, rtol=1e-10, maxit=400, raise_on_fail=False)
                _, itc, rrc, _ = G.pcg(b, rtol=1e-10, maxit=400, raise_on_fail=False)
                gm.append(it)
                cg.append(int(itc[0]))
                worst = max(worst, rr, float(rrc[0]))
                G.close()
            row[key] = gm
            row[key + "_pcg"] = cg
        row["max_relres"] = worst
        rows.append(row)
        print(json.dumps({"row": row}), flush=True)
    print(json.dumps({"table": "GMRES iterations to relative residual 1e-10, 2D constant-coefficient Poisson, "
                               "leaves of 8 (Sec. 7.1, Table 2); columns eps = 0.1, 0.2, 0.3",
                      "factor_prec": args.table_prec, "nbr_dist": args.table_nbr, "solver": "hs_gmres (flexible, no restart); hs_pcg beside it",
                      "rhs": "standard normal, seed 0", "rows": rows,
                      "seconds": round(time.perf_counter() - t0, 1)}), flush=True)


def sweep_arm(args) -> None:
    """The 2D variable-coefficient workload over its parameter grid: contrast
    s in {1, 2, 3} x tolerance eps in {1e-1, 1e-2, 1e-3}, each with and without
    the symmetric diagonal scaling, in the factor precision --prec.  Per point:
    one warm-up and --steps timed factor + PCG solves (fields of seeds 0, 1,
    ...), PCG iterations, the largest relative residual, or the failure
    (HS_ERR_NOT_SPD when GC-constant loses definiteness).  One JSON line."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03189_gb300 import _lib
    from paper_1611_03189_gb300 import problems as P

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    side = WORKLOADS[args.workload][1]
    prec = PRECS[args.prec]
    rows = []
    t0 = time.perf_counter()
    nst = max(args.steps, 1)
    for s_ in (1.0, 2.0, 3.0):
        pbs = [P.diffusion2d(side, s_, k, leaf_size=16) for k in range(nst + 1)]
        rp = torch.as_tensor(pbs[0].rowptr, device=dev)
        ci = torch.as_tensor(pbs[0].col, device=dev)
        vals = [torch.as_tensor(pb.val, device=dev) for pb in pbs]
        bs = [torch.as_tensor(P.rhs(pbs[0].n, 1000 + k), device=dev) for k in range(nst + 1)]
        for eps in (1e-1, 1e-2, 1e-3):
            for scale in (False, True):
                row = {"s": s_, "eps": eps, "scale": scale}
                try:
                    G = _lib.Factor(rp, ci, vals[0], pbs[0].perm, pbs[0].leaf_ptr, eps, _lib.HS_GC_CONSTANT, prec,
                                    scale=scale)
                except _lib.HsError as e:
                    row["failed"] = str(e)[:160]
                    rows.append(row)
                    print(json.dumps({"point": row}), flush=True)
                    continue
                its, rrs, fails = [], [], 0
                torch.cuda.synchronize()
                ms = 0.0
                for k in range(nst + 1):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    try:
                        if k > 0:
                            G.refactor(vals[k])
                        _, it, rr, code = G.pcg(bs[k], rtol=1e-10, maxit=1000, raise_on_fail=False)
                    except _lib.HsError:
                        fails += 1
                        continue
                    e1.record()
                    torch.cuda.synchronize()
                    if k > 0:
                        ms += e0.elapsed_time(e1)
                        its.append(int(it[0]))
                        rrs.append(float(rr[0]))
                timed = len(its)
                row.update({"solves_per_s": timed / (ms / 1000.0) if ms > 0 else None, "iterations": its,
                            "max_relres": max(rrs) if rrs else None, "not_spd_fields": fails,
                            "fields": nst + 1, "factor_bytes": G.info()["factor_bytes"]})
                G.close()
                rows.append(row)
                print(json.dumps({"point": row}), flush=True)
    print(json.dumps({"sweep": f"2D diffusion {side}x{side}, leaves of 16, GC-constant, PCG to 1e-10",
                      "factor_prec": args.prec, "rows": rows, "seconds": round(time.perf_counter() - t0, 1)}),
          flush=True)


def gemm_arm(args) -> None:
    """The tensor-core GEMM alone (hs_gemm_tc): C = A B with M = N = K =
    --gemm-size, FP32 operands rounded to --prec (tf32 or bf16), FP32
    accumulation; each of --steps timed calls after --warmup, CUDA events on
    the launching stream.  TFLOP/s against the measured bf16 burst peak (times
    the nominal tf32/bf16 ratio for tf32).  One JSON line."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03189_gb300 import _lib

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    n = args.gemm_size
    prec = PRECS[args.prec]
    if prec not in (_lib.HS_PREC_TF32, _lib.HS_PREC_BF16, _lib.HS_PREC_TF32X3):
        raise SystemExit("--gemm needs --prec tf32, tf32x3 or bf16")
    g = torch.Generator(device=dev).manual_seed(0)
    A = torch.randn((n, n), generator=g, device=dev, dtype=torch.float32)
    B = torch.randn((n, n), generator=g, device=dev, dtype=torch.float32)
    C = torch.zeros((n, n), device=dev, dtype=torch.float32)
    res = {}
    for bn in (64, 128):
        for _ in range(max(args.warmup, 1)):
            _lib.gemm_tc(prec, A, B, C, bn=bn)
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(args.steps, 1)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _lib.gemm_tc(prec, A, B, C, bn=bn)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        res[bn] = min(ts)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    bf16 = peaks.get("bf16_tflops", 1900.0)
    # 3xTF32 issues three TF32 MMAs per product: its useful rate peaks at a third of TF32's
    peak = bf16 * {"tf32": 1.1 / 2.25, "tf32x3": 1.1 / 2.25 / 3}.get(args.prec, 1.0)
    flops = 2.0 * n ** 3
    best = min(res, key=res.get)
    ach = flops / (res[best] / 1000.0) / 1e12
    print(json.dumps({"metric": "tensor-core GEMM TFLOP/s (hs_gemm_tc)", "value": ach, "unit": "TFLOP/s",
                      "prec": args.prec, "m_n_k": n, "ms": res, "best_tile_n": best,
                      "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                   "frac": ach / peak,
                                   "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)" +
                                                  {"tf32": " x nominal tf32/bf16 ratio 1.1/2.25",
                                                   "tf32x3": " x nominal tf32/bf16 ratio 1.1/2.25 / 3 MMAs"}.get(
                                                      args.prec, "")}}), flush=True)


# The short serving stream of the step benchmark's line: the serving recipe
# (3D diffusion requests, s = 2, leaves of 64, 20 % factor requests, 1-16
# right-hand sides, Poisson arrivals), at grid sides 16-32 and 60 requests so
# that it stays within seconds; `--serve` runs the full recipe (sides 32-96).
SERVE_LEG = {"requests": 60, "rate": 40.0, "sides": (16, 32), "budget_gb": 16, "slots": 4, "limit_s": 120}


def serve_leg(prec: int) -> dict:
    """Served latency (p50/p99 over all requests, arrival to result) and solve
    requests/s of the continuous-batching loop on the short stream, with the
    step benchmark's factor precision and diagonal scaling (every 3D matrix of
    the recipe then factors)."""
    from paper_1611_03189_gb300 import serving as S

    c = SERVE_LEG
    warm = S.poisson_stream(8, 1000.0, seed=12, sides=(c["sides"][0], c["sides"][0]), s=2.0, leaf=64)
    reqs = S.poisson_stream(c["requests"], c["rate"], seed=11, sides=c["sides"], s=2.0, leaf=64)
    srv = S.Server(int(c["budget_gb"]) << 30, slots=c["slots"], max_rhs=16, prec=prec, scale=True)
    srv.run(warm, realtime=False)
    # bounded: the stream normally takes seconds; a run still going after
    # c["limit_s"] is reported as such and left to the daemon worker threads
    box = {}

    def serve():
        box["res"] = srv.run(reqs, realtime=True)

    w0 = time.perf_counter()
    th = threading.Thread(target=serve, daemon=True)
    th.start()
    th.join(c["limit_s"])
    wall = time.perf_counter() - w0
    if "res" not in box:
        return {"error": f"the serving stream did not finish within {c['limit_s']} s"}
    res = box["res"]
    summ = S.summarize(res, wall)
    rr = [float(np.max(r.relres)) for r in res if r.kind == "solve" and r.relres is not None]
    return {"p50_ms": summ["p50_ms"], "p99_ms": summ["p99_ms"], "solve_p50_ms": summ["solve_p50_ms"],
            "solve_p99_ms": summ["solve_p99_ms"], "solve_requests_per_s": summ["solves_per_s"],
            "rhs_per_s": summ["rhs_per_s"], "requests": summ["requests"], "failed": summ["failed"],
            "mean_batch": summ["mean_batch"], "max_relres": max(rr) if rr else None, "wall_s": wall,
            "peak_charged_gb": srv.peak_used / 2**30,
            "config": {"workload": "serving_diffusion3d_short", "sides": list(c["sides"]), "s": 2.0, "leaf": 64,
                       "eps": 1e-2, "p_factor": 0.2, "nrhs": [1, 16], "rate_per_s": c["rate"],
                       "slots": c["slots"], "budget_gb": c["budget_gb"], "diagonal_scaling": True}}


def serve_arm(args) -> None:
    """Served latency (p50/p99) and throughput of the continuous-batching loop,
    mixed (FP32) factor against the plain FP64 factor on the same stream."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03189_gb300 import _lib
    from paper_1611_03189_gb300 import serving as S

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lo, hi = (int(v) for v in args.serve_sides.split(","))
    t_gen = time.perf_counter()
    reqs = S.poisson_stream(args.serve_requests, args.serve_rate, seed=11, sides=(lo, hi), s=2.0, leaf=64)
    t_gen = time.perf_counter() - t_gen
    budget = int(args.serve_budget_gb * (1 << 30))
    # warm-up: kernels loaded, graphs and allocator primed on a few small requests
    warm = S.poisson_stream(8, 1000.0, seed=12, sides=(lo, lo), s=2.0, leaf=64)
    out = {}
    for name, prec in (("mixed_f32", _lib.HS_PREC_F32), ("f64", _lib.HS_PREC_F64)):
        if name == "f64" and args.no_f64_arm:
            continue
        srv = S.Server(budget, slots=args.serve_slots, max_rhs=16, prec=prec, scale=args.scale)
        srv.run(warm, realtime=False)
        clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        clocks.start()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        res = srv.run(reqs, realtime=True)
        wall = time.perf_counter() - w0
        clk = clocks.stop()
        summ = S.summarize(res, wall)
        summ["clocks"] = clk
        summ["peak_charged_gb"] = srv.peak_used / 2**30
        rr = [float(np.max(r.relres)) for r in res if r.kind == "solve" and r.relres is not None]
        summ["max_relres"] = max(rr) if rr else None
        out[name] = summ
    m = out["mixed_f32"]
    line = {
        "metric": "served p50/p99 latency and solves/s (continuous batching; mixed vs FP64 factor)",
        "value": m["solves_per_s"], "unit": "solve requests/s", "n_gpus": 1, "steps": args.serve_requests,
        "warmup": len(warm), "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "serving_diffusion3d", "sides": [lo, hi], "s": 2.0, "leaf": 64, "eps": 1e-2,
                   "p_factor": 0.2, "nrhs": [1, 16], "rate_per_s": args.serve_rate,
                   "budget_gb": args.serve_budget_gb, "slots": args.serve_slots, "max_batch_rhs": 16,
                   "diagonal_scaling": bool(args.scale),
                   "requests": args.serve_requests, "generation_s": t_gen},
        "p50_ms": m["p50_ms"], "p99_ms": m["p99_ms"],
        "serving": out,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="diffusion2d_512", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="f32", choices=["f32", "tf32", "tf32x3", "bf16", "f64"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--scale", action="store_true", help="factor the diagonally scaled D^-1/2 A D^-1/2")
    ap.add_argument("--rank-f64", action="store_true",
                    help="mixed factors: truncation (Gram, eigen-solve, rank decision) in FP64 (hs_opts.rank_f64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve-leg", action="store_true",
                    help="skip the short serving stream (served p50/p99) of the step benchmark's line")
    ap.add_argument("--no-f64-arm", action="store_true", help="skip the FP64-factor comparison")
    ap.add_argument("--profile", action="store_true", help="print a phase breakdown to stderr")
    ap.add_argument("--batched", action="store_true", help="run the batched many-problem benchmark")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--serve", action="store_true", help="run the serving stream instead of the step benchmark")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-rate", type=float, default=20.0, help="mean arrivals per second")
    ap.add_argument("--serve-sides", default="32,96", help="grid side range of the 3D requests")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--gemm", action="store_true", help="time the tensor-core GEMM alone (one JSON line)")
    ap.add_argument("--gemm-size", type=int, default=4096)
    ap.add_argument("--sweep", action="store_true",
                    help="2D diffusion parameter grid: s x eps x scaling (no oracle, one JSON line)")
    ap.add_argument("--gmres-table", action="store_true",
                    help="GMRES iteration table of the paper's Table 2 (no timing)")
    ap.add_argument("--table-sides", default="32,64,128,256,512,1024")
    ap.add_argument("--table-prec", default="f32", choices=["f32", "f64"])
    ap.add_argument("--table-nbr", type=int, default=1, choices=[1, 2],
                    help="neighbour rule: 1 edge-joined clusters, 2 also clusters sharing a neighbour")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.batched:
        batched_arm(args)
        return
    if args.serve:
        serve_arm(args)
        return
    if args.gmres_table:
        gmres_table_arm(args)
        return
    if args.sweep:
        sweep_arm(args)
        return
    if args.gemm:
        gemm_arm(args)
        return

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03189_gb300 import _lib
    from paper_1611_03189_gb300 import problems as P

    dev = torch.device("cuda", local)
    prec = PRECS[args.prec]
    nsteps = args.warmup + args.steps
    # inputs resident in HBM: one matrix (new coefficient field) and rhs block per step
    pbs = []
    for k in range(nsteps):
        pb, eps = make_problem(args.workload, seed=replica_seed(rank, k))
        pbs.append(pb)
    pb0 = pbs[0]
    rp = torch.as_tensor(pb0.rowptr, device=dev)
    ci = torch.as_tensor(pb0.col, device=dev)
    vals = [torch.as_tensor(pb.val, device=dev) for pb in pbs]
    bs = [torch.as_tensor(P.rhs(pb0.n, 1000 + k, nrhs=args.nrhs).T.copy(), device=dev).squeeze(0)
          for k in range(nsteps)]
    stream = torch.cuda.current_stream()
    t_plan = time.perf_counter()
    G = _lib.Factor(rp, ci, vals[0], pb0.perm, pb0.leaf_ptr, eps, _lib.HS_GC_CONSTANT, prec, scale=args.scale,
                    rank_f64=args.rank_f64)
    t_plan = time.perf_counter() - t_plan

    iters_seen = []

    def step(k):
        G.refactor(vals[k])
        x, it, rr, code = G.pcg(bs[k], rtol=1e-10, maxit=1000, raise_on_fail=False)
        if code != _lib.HS_OK:
            raise RuntimeError(f"PCG did not converge: iters {it}, relres {rr}")
        iters_seen.append(int(it.max()))
        return rr

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    # ---- timed region: K steps, device events on the launching stream ----
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = _lib.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    e0.record(stream)
    rrs = []
    for k in range(args.warmup, nsteps):
        rrs.append(float(np.max(step(k))))
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    launches = _lib.launch_count() - l0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    ms_per_step = ms / args.steps
    value = whole_job_rate(world, args.steps, args.nrhs, ms)
    info = G.info()

    # ---- factor-only and solve-only splits (resident factor), for context ----
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    G.refactor(vals[args.warmup])
    e3.record(stream)
    torch.cuda.synchronize()
    factor_ms = e2.elapsed_time(e3)
    # one more refactor with the library's per-phase device timing (event pairs)
    _lib.profile_phases(True)
    G.refactor(vals[args.warmup])
    torch.cuda.synchronize()
    _lib.profile_phases(False)
    phase_ms = G.info()["phase_ms"]
    e2.record(stream)
    _, it1, _, _ = G.pcg(bs[args.warmup], rtol=1e-10, maxit=1000)
    e3.record(stream)
    torch.cuda.synchronize()
    solve_ms = e2.elapsed_time(e3)

    # ---- dominant kernel class of the solve: the apply (Algorithm 2), HBM-bound ----
    napply = 20
    r = bs[args.warmup]
    G.apply(r)
    torch.cuda.synchronize()
    e2.record(stream)
    for _ in range(napply):
        G.apply(r)
    e3.record(stream)
    torch.cuda.synchronize()
    apply_ms = e2.elapsed_time(e3) / napply
    n = pb0.n
    vec_bytes = 8 * n * args.nrhs * 4     # r in, z out, workspace in/out per level-L unknown
    apply_bytes = info["factor_bytes"] + vec_bytes
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    achieved = apply_bytes / (apply_ms / 1000.0) / 1e9

    # ---- the plain FP64 factor at the same accuracy (same inputs, same steps) ----
    f64 = None
    if prec != _lib.HS_PREC_F64 and not args.no_f64_arm:
        x_mixed, _, _, _ = G.pcg(bs[args.warmup], rtol=1e-10, maxit=1000)
        G64 = _lib.Factor(rp, ci, vals[0], pb0.perm, pb0.leaf_ptr, eps, _lib.HS_GC_CONSTANT, _lib.HS_PREC_F64,
                          scale=args.scale)
        it64, rr64 = [], []
        for k in range(args.warmup):
            G64.refactor(vals[k])
            G64.pcg(bs[k], rtol=1e-10, maxit=1000)
        torch.cuda.synchronize()
        e2.record(stream)
        for k in range(args.warmup, nsteps):
            G64.refactor(vals[k])
            x64, it, rr, code = G64.pcg(bs[k], rtol=1e-10, maxit=1000, raise_on_fail=False)
            if code != _lib.HS_OK:
                raise RuntimeError(f"FP64-factor PCG did not converge: iters {it}, relres {rr}")
            it64.append(int(it.max()))
            rr64.append(float(np.max(rr)))
        e3.record(stream)
        torch.cuda.synchronize()
        ms64 = e2.elapsed_time(e3)
        e2.record(stream)
        G64.refactor(vals[args.warmup])
        e3.record(stream)
        torch.cuda.synchronize()
        f64_factor_ms = e2.elapsed_time(e3)
        x64, _, _, _ = G64.pcg(bs[args.warmup], rtol=1e-10, maxit=1000)
        diff = float(torch.linalg.norm(x_mixed - x64) / torch.linalg.norm(x64))
        f64 = {"value": args.steps * args.nrhs / (ms64 / 1000.0), "unit": "solves/s", "ms_per_step": ms64 / args.steps,
               "factor_ms": f64_factor_ms, "iterations_timed": it64, "max_relres": max(rr64),
               "x_rel_diff_mixed_vs_f64": diff, "factor_bytes": G64.info()["factor_bytes"]}
        G64.close()

    # ---- end to end through the C ABI with host buffers (H2D values + rhs, D2H x) ----
    hv = [torch.empty(pb0.nnz, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    hb = [torch.empty(bs[0].shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    hx = [torch.empty(bs[0].shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    for j in range(2):
        hv[j].copy_(vals[args.warmup + j % args.steps].cpu())
        hb[j].copy_(bs[args.warmup + j % args.steps].cpu())
    dv = torch.empty(pb0.nnz, dtype=torch.float64, device=dev)
    db = torch.empty(bs[0].shape, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2.record(stream)
    for k in range(args.steps):
        dv.copy_(hv[k % 2], non_blocking=True)
        db.copy_(hb[k % 2], non_blocking=True)
        G.refactor(dv)
        x, it, rr, code = G.pcg(db, rtol=1e-10, maxit=1000)
        hx[k % 2].copy_(x, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e2.elapsed_time(e3), dist, dev)
    e2e_val = whole_job_rate(world, args.steps, args.nrhs, e2e_ms)

    if args.profile and rank == 0:
        print(json.dumps({"plan_and_first_factor_s": t_plan, "factor_ms": factor_ms, "solve_ms": solve_ms,
                          "apply_ms": apply_ms, "iters": int(it1.max()), "info": info,
                          "apply_GBps": achieved, "wall_timed_s": wall}), file=sys.stderr, flush=True)

    # ---- served latency on a short stream of the serving recipe ----
    served = None
    if world == 1 and not args.no_serve_leg:
        try:
            served = serve_leg(prec)
        except Exception as ex:  # the serving figures must not hide the step's number
            served = {"error": str(ex)[:300]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(args.workload)
        except Exception as ex:  # the baseline must not hide the GPU number
            cpu = {"error": str(ex)[:200]}

    # ---- the large-node truncation (tridiagonal eigen path): plain FP32/FP64 ALU work ----
    # nominal eigen-solve flops (4/3 m^3 + 2 m^2 k per node) over the device time
    # of its launches (CUDA events on the factor stream, inside the library)
    info_f = G.info()
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    if args.prec != "f64":
        alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12      # FP32 FMA lanes x 2 flops x clock
        alu_src = f"derived: 152 SMs x 128 FP32 lanes x 2 flops x {sm_mhz:.0f} MHz"
    else:
        alu_peak = 1.25                                   # nominal GB300 FP64 rate
        alu_src = "nominal GB300 FP64 (1.25 TFLOP/s)"
    tb_ms = info_f["trunc_big_ms"]
    tb_launches = max(info_f["trunc_big_launches"], 1)
    tb_ach = info_f["trunc_big_flops"] / (tb_ms / 1000.0) / 1e12 if tb_ms > 0 else 0.0
    roof_trunc = {"bound": "alu", "kernel": "k_trunc_big (large-node truncation: tridiagonalisation, "
                  "bisection, inverse iteration, back-transformation)",
                  "achieved": tb_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": tb_ach / alu_peak,
                  "peak_source": alu_src, "traffic": TRAFFIC.get((args.workload, args.prec), {}).get("trunc"),
                  "algorithmic_flops_per_launch": info_f["trunc_big_flops"] / tb_launches,
                  "launch_ms": tb_ms / tb_launches, "launches_per_factor": info_f["trunc_big_launches"],
                  "share_of_step": tb_ms / ms_per_step}
    roof_apply = {"bound": "hbm", "kernel": "apply (Algorithm 2: k_f1, k_f2, k_b1, k_b2, k_root)",
                  "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                  "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback",
                  "traffic": TRAFFIC.get((args.workload, args.prec), {}).get("apply"),
                  "algorithmic_bytes": apply_bytes, "launch_ms": apply_ms,
                  "share_of_step": apply_ms * int(it1.max()) / ms_per_step}
    # ---- the tensor-core GEMM of the mixed factors (tcgen05), against the tensor peak ----
    # flops it executes (2MNK per task) over the device time of its launches
    # (an event pair around each launch on the factor stream, inside the library)
    tensor_peak, tensor_src = tensor_peak_for(args.prec, peaks)
    roofs = [roof_trunc, roof_apply]
    if info_f["tc_launches"] > 0 and info_f["tc_ms"] > 0:
        tc_ach = info_f["tc_flops"] / (info_f["tc_ms"] / 1000.0) / 1e12
        roofs.append({"bound": "tensor", "kernel": f"k_gemm_tc ({args.prec.upper()} operands, FP32 accumulate in TMEM)",
                      "achieved": tc_ach, "peak": tensor_peak, "unit": "TFLOP/s", "frac": tc_ach / tensor_peak,
                      "peak_source": tensor_src, "traffic": None,
                      "algorithmic_flops_per_launch": info_f["tc_flops"] / info_f["tc_launches"],
                      "launch_ms": info_f["tc_ms"] / info_f["tc_launches"],
                      "launches_per_factor": info_f["tc_launches"], "share_of_step": info_f["tc_ms"] / ms_per_step})
    # the dominant kernel of the step is the one with the largest share of its time
    roofs.sort(key=lambda r: -r["share_of_step"])
    dominant, others = roofs[0], roofs[1:]
    # the factorization's algorithmic work (per-node count of the hot-path
    # table: Gram, R^T, Cholesky, Y, S, G, H, Schur, M_ss / P_ss) over its device
    # time, against the tensor peak its contractions would run at
    factor_alg = {"alg_flops": info_f["alg_flops"], "factor_ms": factor_ms,
                  "achieved_tflops": info_f["alg_flops"] / (factor_ms / 1000.0) / 1e12,
                  "peak_tflops": tensor_peak, "peak_source": tensor_src,
                  "frac": info_f["alg_flops"] / (factor_ms / 1000.0) / 1e12 / tensor_peak,
                  "executed_flops": info_f["factor_flops"], "eig_flops_nominal": info_f["eig_flops"]}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.prec == "f64" else f"{args.prec}+f64", "data": "synthetic",
            "config": {"workload": args.workload, "dim": WORKLOADS[args.workload][0],
                       "grid": WORKLOADS[args.workload][1], "n": n,
                       "s": WORKLOADS[args.workload][2], "eps": WORKLOADS[args.workload][3],
                       "leaf": WORKLOADS[args.workload][4], "variant": "GC-constant",
                       "factor_prec": args.prec, "pcg": "fp64", "rtol": 1e-10, "nrhs": args.nrhs,
                       "diagonal_scaling": bool(args.scale),
                       "rank_decision": ("fp64" if args.prec == "f64" or args.rank_f64
                                         else "fp32 eigen-solve, fp64 comparison"),
                       "l2": "inputs larger than L2 (factor records > 129 MB)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": dominant,
            "roofline_other": others,
            "factor_algorithmic": factor_alg,
            "gemm_autotune": ([{k: r[k] for k in ("max_mn", "k", "route")} for r in _lib.gemm_tune_report(prec)]
                              if args.prec in ("tf32", "tf32x3", "bf16") else None),
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": 8 * (pb0.nnz + n * args.nrhs),
                    "d2h_bytes_per_step": 8 * n * args.nrhs},
            "fp64_factor": f64,
            "served": served,
            "gpu_launches": launches,
            "launches_before_timed": l0,
            "clocks": clk,
            "factor_ms": factor_ms, "solve_ms": solve_ms, "pcg_iterations": int(it1.max()),
            "factor_host_ms": info_f["host_ms"], "factor_wait_ms": info_f["wait_ms"],
            "factor_phase_ms": phase_ms,
            "iterations_timed": iters_seen[args.warmup:], "max_relres": max(rrs),
            "factor_info": {k: info[k] for k in ("levels", "waves", "super_nodes", "root_size", "max_rank",
                                                 "max_super", "factor_bytes", "device_bytes", "factor_flops")},
        }
        print(json.dumps(line), flush=True)
    G.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
