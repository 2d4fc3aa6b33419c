"""A serving loop over the C ABI: continuous batching of factor and solve
requests on one GPU.

The paper states a solver, not a service; this module is the request loop
that a solver service needs on a GPU.

Requests
  * factor: a new matrix (CSR pattern and values, clustering) to factor and
    keep resident;
  * solve: 1..16 right-hand sides against a matrix factored earlier.
They arrive over time, for example as a Poisson process.

Scheduling
  * Slots: the server runs ``slots`` worker threads, each with its own CUDA
    stream. A request that arrives while others are on the GPU starts as soon
    as a slot and enough of the device-memory budget are free, so work of
    different requests overlaps on the device. The library calls release the
    Python GIL (ctypes), and every call runs on its slot's stream.
  * Memory admission: a factor request is admitted only when its estimated
    device bytes fit in the budget. If they do not, idle resident
    factorizations are evicted, least recently used first. The estimate per
    unknown is calibrated by the factorizations done so far; an admitted
    factor is then charged its measured bytes. ``CudaBackend`` measures them
    exactly: every handle takes its device memory through a counting
    allocator hook (``_lib.DeviceAllocator``, hs_opts.allocator) backed by
    PyTorch's caching allocator, so a factor is charged the bytes it holds,
    plus a reservation for its solve workspaces; when the workspaces outgrow
    that reservation, the charge follows the bytes held.
  * Right-hand-side batching: solve requests waiting for the same resident
    factorization are merged in arrival order into one ``hs_pcg`` call of at
    most ``max_rhs`` columns.

Identity of results
  * The library computes every right-hand side column by column. PCG
    reductions visit rows in an order that depends on n alone, and the
    factorization is deterministic.
  * So a request's solution has the same bits alone as in any mix or batch.
    ``run_alone`` replays a request list one request at a time, which lets a
    test check this.

Solves for a matrix that was evicted refactor it first, from the host copy
kept with its factor request, and are reported as such.

The work itself goes through a backend (``CudaBackend``: the C ABI on the
slot's stream); tests of the host logic substitute a fake one.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Optional

import numpy as np

from . import _lib


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                      # "factor" or "solve"
    matrix: int                    # matrix id (a factor request defines it)
    arrival: float                 # seconds after the start of the stream
    problem: object = None         # factor: problems.Problem (host CSR, clustering)
    rhs: Optional[np.ndarray] = None   # solve: (nrhs, n) float64

    @property
    def nrhs(self) -> int:
        return 0 if self.rhs is None else int(self.rhs.shape[0])


@dataclasses.dataclass
class Result:
    rid: int
    kind: str
    matrix: int
    arrival: float
    start: float = 0.0
    finish: float = 0.0
    x: Optional[np.ndarray] = None
    iters: Optional[np.ndarray] = None
    relres: Optional[np.ndarray] = None
    batch: int = 1                 # requests that shared the library call
    refactored: bool = False       # a solve that had to refactor an evicted matrix
    status: int = _lib.HS_OK
    error: str = ""

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


class _Resident:
    def __init__(self, matrix: int, n: int):
        self.matrix = matrix
        self.n = n
        self.factor = None
        self.bytes = 0
        self.busy = False
        self.ready = False         # factored and usable
        self.reserved = 0          # bytes reserved by the running job
        self.last_use = 0.0


class CudaBackend:
    """Runs the work of a slot through the C ABI on the slot's CUDA stream."""

    def __init__(self, device: int = 0, eps: float = 1e-2, variant: int = _lib.HS_GC_CONSTANT,
                 prec: int = _lib.HS_PREC_F32, rtol: float = 1e-10, maxit: int = 1000, scale: bool = False,
                 exact_memory: bool = True):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the serving loop needs a CUDA device")
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.eps, self.variant, self.prec = eps, variant, prec
        self.rtol, self.maxit = rtol, maxit
        self.scale = scale   # factor D^-1/2 A D^-1/2 (hs_opts.scale)
        # each handle's device memory through its own counting allocator hook
        self.exact_memory = exact_memory

    def clone(self):
        return CudaBackend(self.device.index or 0, self.eps, self.variant, self.prec, self.rtol, self.maxit,
                           self.scale, self.exact_memory)

    def slot(self):
        """Per-worker state: a CUDA stream of its own."""
        self.torch.cuda.set_device(self.device)
        return self.torch.cuda.Stream(device=self.device)

    def factor(self, stream, pb):
        """Factor problem pb; returns (handle, device bytes of the handle)."""
        torch = self.torch
        d = self.device
        with torch.cuda.stream(stream):
            rp = torch.as_tensor(pb.rowptr, dtype=torch.int32).pin_memory().to(d, non_blocking=True)
            ci = torch.as_tensor(pb.col, dtype=torch.int32).pin_memory().to(d, non_blocking=True)
            va = torch.as_tensor(pb.val, dtype=torch.float64).pin_memory().to(d, non_blocking=True)
            hook = _lib.DeviceAllocator() if self.exact_memory else None
            f = _lib.Factor(rp, ci, va, pb.perm, pb.leaf_ptr, self.eps, self.variant, self.prec, stream=stream,
                            scale=self.scale, allocator=hook)
            stream.synchronize()
        if hook is not None:
            return f, hook.held   # every device byte the handle holds
        # factor arenas + permuted CSR and maps
        return f, int(f.info()["device_bytes"]) + 16 * (pb.n + 1 + 2 * len(pb.col))

    def held(self, f):
        """Device bytes handle f holds now (None when not counted)."""
        hook = getattr(f, "_alloc", None)
        return None if hook is None else hook.held

    def solve(self, stream, f, B: np.ndarray):
        """PCG on the rows of B (nrhs, n); returns (X, iters, relres, status)."""
        torch = self.torch
        with torch.cuda.stream(stream):
            hb = torch.from_numpy(np.ascontiguousarray(B)).pin_memory()
            db = hb.to(self.device, non_blocking=True)
            x, it, rr, code = f.pcg(db, rtol=self.rtol, maxit=self.maxit, stream=stream, raise_on_fail=False)
            hx = torch.empty(x.shape, dtype=torch.float64, pin_memory=True)
            hx.copy_(x, non_blocking=True)
            stream.synchronize()
        return hx.numpy().reshape(B.shape), it, rr, code

    def release(self, f):
        f.close()


class Server:
    """Continuous-batching solver service on one GPU (see module docstring)."""

    def __init__(self, budget_bytes: int, slots: int = 4, max_rhs: int = 16, batching: bool = True,
                 backend=None, **backend_opts):
        self.backend = backend if backend is not None else CudaBackend(**backend_opts)
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.max_rhs = int(max_rhs)
        self.batching = batching
        self.bytes_per_unknown = 24_000.0          # first guess, replaced by measurements
        self._measured = []                        # (n, bytes)
        self.peak_used = 0                         # largest charged total seen
        self.overgrown = 0                         # solves whose workspaces outgrew the reservation
        self.final_used = 0                        # charged total when the last request finished

    # ---- memory model -------------------------------------------------------
    def _solve_bytes(self, n: int) -> int:
        """Solve buffers of a handle at max_rhs columns: 7 FP64 PCG vectors and
        the apply workspace and scratch (about 5 more), rounded up."""
        np2 = 1
        while np2 < self.max_rhs:
            np2 *= 2
        return 8 * n * np2 * 12

    def _estimate(self, n: int) -> int:
        return int(self.bytes_per_unknown * n) + self._solve_bytes(n) + 16 * 7 * n

    def _calibrate(self, n: int, used: int):
        """Bytes per unknown of the factorizations seen so far (the largest
        ratio, with a 15% margin): the admission estimate."""
        used -= self._solve_bytes(n)
        self._measured.append((n, used))
        self.bytes_per_unknown = max(1.15 * max(b / max(a, 1) for a, b in self._measured), 1000.0)

    # ---- the loop ------------------------------------------------------------
    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Serve `requests`.  With realtime, each request is released at its
        arrival time; otherwise all are available at once."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        results = {r.rid: Result(r.rid, r.kind, r.matrix, r.arrival) for r in reqs}
        problems = {r.matrix: r.problem for r in reqs if r.kind == "factor"}
        residents: dict[int, _Resident] = {}
        used = [0]
        cv = threading.Condition()
        pending: collections.deque = collections.deque()
        jobs: collections.deque = collections.deque()
        state = {"done": 0, "stop": False}
        be = self.backend
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731

        def charge(delta: int):
            used[0] += delta
            self.peak_used = max(self.peak_used, used[0])

        def worker():
            stream = be.slot()
            while True:
                with cv:
                    while not jobs and not state["stop"]:
                        cv.wait()
                    if state["stop"] and not jobs:
                        return
                    kind, rs, reqlist = jobs.popleft()
                start = now()
                for q in reqlist:
                    results[q.rid].start = start
                did_factor = kind == "factor" or not rs.ready
                err = None
                grow = [0]   # solve workspaces beyond the charge of the factor
                try:
                    if did_factor:
                        if rs.factor is not None:
                            be.release(rs.factor)
                            rs.factor = None
                        rs.ready = False
                        rs.factor, fbytes = be.factor(stream, problems[rs.matrix])
                        rs.bytes = fbytes + self._solve_bytes(rs.n)
                        rs.ready = True
                    if kind == "solve":
                        B = np.concatenate([q.rhs for q in reqlist], axis=0)
                        X, it, rr, code = be.solve(stream, rs.factor, B)
                        held = getattr(be, "held", None)
                        now_held = held(rs.factor) if held is not None else None
                        if now_held is not None and now_held > rs.bytes:
                            grow[0] = now_held - rs.bytes   # charged below, under the lock
                        c = 0
                        for q in reqlist:
                            r = results[q.rid]
                            r.x = X[c:c + q.nrhs].copy()
                            r.iters = np.asarray(it[c:c + q.nrhs]).copy()
                            r.relres = np.asarray(rr[c:c + q.nrhs]).copy()
                            r.status = code
                            c += q.nrhs
                except Exception as ex:  # reported per request, the loop goes on
                    err = ex
                fin = now()
                with cv:
                    for q in reqlist:
                        r = results[q.rid]
                        r.finish = fin
                        r.batch = len(reqlist)
                        r.refactored = kind == "solve" and did_factor
                        if err is not None:
                            r.status = getattr(err, "code", _lib.HS_ERR_INVALID)
                            r.error = str(err)[:300]
                    # the reservation becomes the measured footprint
                    charge(-rs.reserved)
                    rs.reserved = 0
                    if did_factor:
                        if rs.ready:
                            charge(rs.bytes)
                            self._calibrate(rs.n, rs.bytes)
                        else:
                            rs.bytes = 0
                    if grow[0] > 0 and rs.ready:
                        rs.bytes += grow[0]
                        charge(grow[0])
                        self.overgrown += 1
                    rs.busy = False
                    rs.last_use = fin
                    state["done"] += len(reqlist)
                    cv.notify_all()

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.slots)]
        for t in threads:
            t.start()

        def evict_for(need: int) -> bool:
            """Make room for `need` bytes: evict idle factorizations, least
            recently used first -- those no waiting request refers to, then
            (so that a waiting factor request cannot starve) the others."""
            if used[0] + need <= self.budget:
                return True
            idle = [r for r in residents.values() if r.ready and not r.busy]
            wanted = {q.matrix for q in pending}
            order = sorted(idle, key=lambda r: (r.matrix in wanted, r.last_use))
            if used[0] - sum(r.bytes for r in order) + need > self.budget:
                return False        # evicting everything idle would not be enough: evict nothing
            for r in order:
                if used[0] + need <= self.budget:
                    break
                be.release(r.factor)
                r.factor = None
                r.ready = False
                charge(-r.bytes)
                r.bytes = 0
            return True

        def dispatch():
            """Move admissible pending requests to the job queue (cv held)."""
            busy_slots = sum(1 for r in residents.values() if r.busy)
            taken = set()
            blocked = False     # a factor request waits for memory
            i = 0
            while i < len(pending) and busy_slots < self.slots:
                q = pending[i]
                if q.kind == "factor":
                    if blocked:
                        # factor requests keep their order: none may take the
                        # memory an earlier one waits for
                        i += 1
                        continue
                    rs = residents.setdefault(q.matrix, _Resident(q.matrix, q.problem.n))
                    if rs.busy:
                        i += 1
                        continue
                    need = self._estimate(q.problem.n)
                    if not evict_for(need):
                        blocked = True
                        i += 1
                        continue
                    rs.busy = True
                    rs.reserved = need
                    charge(need)
                    del pending[i]
                    jobs.append(("factor", rs, [q]))
                    busy_slots += 1
                    continue
                rs = residents.get(q.matrix)
                if rs is None or rs.busy or q.matrix in taken:
                    i += 1
                    continue
                if not rs.ready:
                    # an evicted matrix is refactored first; that takes memory,
                    # so it waits behind a blocked factor request too
                    if blocked or any(p.kind == "factor" and p.matrix == q.matrix for p in pending):
                        i += 1
                        continue
                    need = self._estimate(rs.n)
                    if not evict_for(need):
                        i += 1
                        continue
                    rs.reserved = need
                    charge(need)
                # merge the waiting solves of this matrix, in arrival order
                batch, cols = [q], q.nrhs
                if self.batching:
                    for p in list(pending)[i + 1:]:
                        if p.kind == "solve" and p.matrix == q.matrix and cols + p.nrhs <= self.max_rhs:
                            batch.append(p)
                            cols += p.nrhs
                for p in batch:
                    pending.remove(p)
                rs.busy = True
                taken.add(q.matrix)
                jobs.append(("solve", rs, batch))
                busy_slots += 1
            cv.notify_all()

        nxt = 0
        total = len(reqs)
        with cv:
            while state["done"] < total:
                t = now()
                while nxt < total and (not realtime or reqs[nxt].arrival <= t):
                    pending.append(reqs[nxt])
                    nxt += 1
                dispatch()
                wait = 0.05
                if realtime and nxt < total:
                    wait = max(0.0, min(wait, reqs[nxt].arrival - now()))
                if state["done"] < total:
                    cv.wait(timeout=wait if wait > 0 else 0.0005)
            state["stop"] = True
            cv.notify_all()
        for t in threads:
            t.join()
        self.final_used = used[0]   # charged bytes of the residents left at the end
        for rs in residents.values():
            if rs.factor is not None:
                be.release(rs.factor)
                rs.factor = None
        return [results[r.rid] for r in reqs]

    def run_alone(self, requests: list[Request]) -> list[Result]:
        """Each request by itself, one after another, in arrival order: one
        slot, no batching, no overlap (the reference for identity checks)."""
        solo = Server(self.budget, slots=1, max_rhs=self.max_rhs, batching=False, backend=self.backend.clone())
        return solo.run(requests, realtime=False)


# ---------------------------------------------------------------------------
# workload: a Poisson-arrival stream of 3D diffusion requests
# ---------------------------------------------------------------------------
def poisson_stream(count: int, rate: float, seed: int, sides=(32, 96), s: float = 2.0, leaf: int = 64,
                   p_factor: float = 0.2, rhs_range=(1, 16), recent: int = 8) -> list[Request]:
    """`count` requests with exponential inter-arrival times of mean 1/rate.
    A fraction p_factor are factor requests for a new 3D diffusion matrix
    (side uniform in `sides`, a = exp(s g)); the rest are solves with nrhs
    uniform in `rhs_range` against one of the `recent` latest matrices."""
    from . import problems as P

    rng = np.random.default_rng(seed)
    reqs: list[Request] = []
    t = 0.0
    mats: list[tuple[int, int]] = []      # (matrix id, n)
    for rid in range(count):
        t += rng.exponential(1.0 / rate)
        if not mats or rng.random() < p_factor:
            side = int(rng.integers(sides[0], sides[1] + 1))
            mid = len(mats)
            pb = P.diffusion3d(side, s, seed * 100003 + mid, leaf_size=leaf)
            mats.append((mid, pb.n))
            reqs.append(Request(rid, "factor", mid, t, problem=pb))
        else:
            mid, n = mats[int(rng.integers(max(0, len(mats) - recent), len(mats)))]
            k = int(rng.integers(rhs_range[0], rhs_range[1] + 1))
            reqs.append(Request(rid, "solve", mid, t, rhs=rng.standard_normal((k, n))))
    return reqs


def summarize(results: list[Result], wall: float) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    solves = [r for r in results if r.kind == "solve"]
    fac = [r for r in results if r.kind == "factor"]
    rhs = sum(0 if r.x is None else r.x.shape[0] for r in solves)

    def pct(a, p):
        return float(np.percentile(a, p)) if len(a) else None

    ls = np.array([r.latency for r in solves]) * 1e3
    lf = np.array([r.latency for r in fac]) * 1e3
    return {
        "requests": len(results), "factor_requests": len(fac), "solve_requests": len(solves),
        "rhs_solved": int(rhs), "wall_s": wall,
        "solves_per_s": len(solves) / wall if wall > 0 else None,
        "rhs_per_s": rhs / wall if wall > 0 else None,
        "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
        "solve_p50_ms": pct(ls, 50), "solve_p99_ms": pct(ls, 99),
        "factor_p50_ms": pct(lf, 50), "factor_p99_ms": pct(lf, 99),
        "mean_batch": float(np.mean([r.batch for r in solves])) if solves else None,
        "refactored": sum(1 for r in solves if r.refactored),
        "failed": sum(1 for r in results if r.status != _lib.HS_OK),
    }
