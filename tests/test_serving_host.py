"""Host logic of the serving loop (admission, eviction, batching, result
routing), with a fake backend in place of the GPU: no CUDA needed."""
import threading
import time
import types

import numpy as np
import pytest

from paper_1611_03189_gb300.serving import Request, Server, summarize


class FakeHandle:
    def __init__(self, matrix_n):
        self.n = matrix_n
        self.closed = False


class FakeBackend:
    """Sleeps instead of computing; x = 2 b so that routing can be checked."""

    def __init__(self, bytes_per_unknown=1000):
        self.bpu = bytes_per_unknown
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.log = []          # (event, matrix n, tag or columns, time)

    def clone(self):
        return FakeBackend(self.bpu)

    def slot(self):
        return None

    def _enter(self):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)

    def _leave(self):
        with self.lock:
            self.active -= 1

    def factor(self, stream, pb):
        self._enter()
        self.log.append(("factor", pb.n, pb.tag, time.perf_counter()))
        time.sleep(0.002 + pb.n * 1e-6)
        self._leave()
        return FakeHandle(pb.n), self.bpu * pb.n

    def solve(self, stream, f, B):
        assert not f.closed
        self._enter()
        self.log.append(("solve", f.n, B.shape[0], time.perf_counter()))
        time.sleep(0.001)
        self._leave()
        k = B.shape[0]
        return 2.0 * B, np.full(k, 7, np.int32), np.full(k, 1e-11), 0

    def release(self, f):
        f.closed = True


def _pb(n, tag):
    return types.SimpleNamespace(n=n, col=np.zeros(5 * n, np.int32), tag=tag)


def _stream(count, seed, sizes=(1000, 4000), p_factor=0.25, rate=2000.0):
    rng = np.random.default_rng(seed)
    reqs, mats, t = [], [], 0.0
    for rid in range(count):
        t += rng.exponential(1.0 / rate)
        if not mats or rng.random() < p_factor:
            n = int(rng.integers(*sizes))
            reqs.append(Request(rid, "factor", len(mats), t, problem=_pb(n, len(mats))))
            mats.append(n)
        else:
            m = int(rng.integers(max(0, len(mats) - 6), len(mats)))
            k = int(rng.integers(1, 17))
            reqs.append(Request(rid, "solve", m, t, rhs=rng.standard_normal((k, mats[m]))))
    return reqs


def _check_results(reqs, res):
    by = {r.rid: r for r in res}
    for q in reqs:
        r = by[q.rid]
        assert r.status == 0, r.error
        assert r.finish >= r.start >= 0.0
        if q.kind == "solve":
            assert np.array_equal(r.x, 2.0 * q.rhs)      # each request gets its own rows back
            assert r.iters.shape == (q.nrhs,)


@pytest.mark.parametrize("realtime", [False, True])
def test_all_requests_served_and_routed(realtime):
    reqs = _stream(120, 0)
    be = FakeBackend()
    srv = Server(10**12, slots=4, max_rhs=16, backend=be)
    res = srv.run(reqs, realtime=realtime)
    assert len(res) == len(reqs)
    _check_results(reqs, res)
    assert 1 < be.max_active <= 4
    s = summarize(res, max(r.finish for r in res))
    assert s["failed"] == 0 and s["requests"] == 120
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_batches_respect_max_rhs_and_matrix():
    reqs = _stream(150, 1, rate=1e6)                # everything arrives at once
    be = FakeBackend()
    srv = Server(10**12, slots=2, max_rhs=16, backend=be)
    res = srv.run(reqs, realtime=False)
    _check_results(reqs, res)
    for ev, n, cols, _ in be.log:
        if ev == "solve":
            assert 1 <= cols <= 16
    solves = [r for r in res if r.kind == "solve"]
    assert max(r.batch for r in solves) > 1           # batching happened
    # requests that shared a call are of one matrix and finished together
    groups = {}
    for r in solves:
        groups.setdefault((r.start, r.finish), []).append(r)
    for g in groups.values():
        if len(g) > 1:
            assert len({x.matrix for x in g}) == 1
            assert all(x.batch == len(g) for x in g)


def test_no_batching_means_one_request_per_call():
    reqs = _stream(60, 2, rate=1e6)
    be = FakeBackend()
    res = Server(10**12, slots=3, batching=False, backend=be).run(reqs, realtime=False)
    _check_results(reqs, res)
    assert all(r.batch == 1 for r in res)
    nsolve = sum(1 for q in reqs if q.kind == "solve")
    assert sum(1 for e in be.log if e[0] == "solve") == nsolve


def test_budget_forces_eviction_and_refactor_without_exceeding_it():
    reqs = _stream(200, 3, sizes=(2000, 2001), p_factor=0.3)
    be = FakeBackend(bytes_per_unknown=1000)
    probe = Server(10**12, slots=3, max_rhs=16, backend=be)
    # room for about three resident factorizations
    srv = Server(int(3.5 * 1000 * 2000 * 1.2 + 3 * probe._solve_bytes(2000)), slots=3, max_rhs=16,
                 backend=be)
    srv.bytes_per_unknown = 1000 * 1.15            # a calibrated estimate
    res = srv.run(reqs, realtime=False)
    _check_results(reqs, res)
    assert srv.peak_used <= srv.budget
    assert any(r.refactored for r in res)           # evicted matrices came back


def test_factor_requests_start_in_arrival_order():
    reqs = _stream(100, 4, p_factor=0.5, rate=1e6)
    be = FakeBackend()
    srv = Server(10**12, slots=4, backend=be)
    srv.run(reqs, realtime=False)
    tags = [tag for ev, n, tag, t in sorted(be.log, key=lambda e: e[3]) if ev == "factor"]
    # first factorizations of each matrix follow matrix-id (= arrival) order
    first = []
    for t in tags:
        if t not in first:
            first.append(t)
    assert first == sorted(first)


def test_failed_request_reports_error_and_loop_continues():
    class Failing(FakeBackend):
        def factor(self, stream, pb):
            if pb.tag == 1:
                raise RuntimeError("factor failed on purpose")
            return super().factor(stream, pb)

    reqs = _stream(80, 5)
    res = Server(10**12, slots=2, backend=Failing()).run(reqs, realtime=False)
    bad = [r for r in res if r.matrix == 1]
    good = [r for r in res if r.matrix != 1]
    assert bad and all(r.status != 0 and "on purpose" in r.error for r in bad)
    assert all(r.status == 0 for r in good)


class CountingBackend(FakeBackend):
    """As FakeBackend, with held(f): the bytes a handle holds as an allocator
    hook counts them -- its factor bytes, then its solve workspaces, which
    appear with its first solve and here grow past the server's reservation."""

    def __init__(self, extra):
        super().__init__()
        self.extra = extra
        self.held_bytes = {}

    def clone(self):
        return CountingBackend(self.extra)

    def factor(self, stream, pb):
        f, nbytes = super().factor(stream, pb)
        self.held_bytes[id(f)] = nbytes
        return f, nbytes

    def solve(self, stream, f, B):
        out = super().solve(stream, f, B)
        self.held_bytes[id(f)] = self.bpu * f.n + self.extra * f.n
        return out

    def held(self, f):
        return self.held_bytes.get(id(f))


@pytest.mark.parametrize("extra,grows", [(10, False), (10_000, True)])
def test_charge_follows_the_bytes_a_handle_holds(extra, grows):
    """A resident's charge is its counted factor bytes plus the solve
    reservation; when the counted bytes after a solve exceed that, the charge
    moves up to them (and stays within the budget accounting)."""
    reqs = [Request(0, "factor", 0, 0.0, problem=_pb(1000, 0)),
            Request(1, "solve", 0, 0.001, rhs=np.ones((2, 1000)))]
    be = CountingBackend(extra)
    srv = Server(budget_bytes=1 << 40, slots=1, backend=be)
    res = srv.run(reqs, realtime=False)
    assert all(r.status == 0 for r in res)
    reserved = 1000 * 1000 + srv._solve_bytes(1000)
    held = 1000 * 1000 + extra * 1000
    assert srv.overgrown == (1 if grows else 0)
    assert srv.final_used == (held if grows else reserved)
    assert srv.peak_used >= srv.final_used
