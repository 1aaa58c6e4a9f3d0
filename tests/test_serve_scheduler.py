"""Host logic of the continuous-batching server, with a host-only backend (no GPU)."""
import threading
import time

import numpy as np
import pytest

from paper_2009_08500_gb300.serve import AdmissionError, Backend, Server, ServeRequest


class FakeBackend(Backend):
    """Completes a request `dur` seconds after launch; tracks concurrency and memory."""

    def __init__(self, dur=0.02, fail_on=None):
        self.dur = dur
        self.fail_on = fail_on
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.mem = 0
        self.max_mem = 0
        self.order = []

    def nbytes(self, req):
        return int(req.params.shape[0] * 100)

    def launch(self, req, slot):
        if self.fail_on is not None and req.fit == self.fail_on:
            raise RuntimeError("injected launch failure")
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.mem += req.nbytes
            self.max_mem = max(self.max_mem, self.mem)
            self.order.append(req.id)
        dur = self.dur if np.isscalar(self.dur) else self.dur[req.fit]
        return [time.perf_counter() + dur, req, False]

    def done(self, handle):
        return time.perf_counter() >= handle[0]

    def finish(self, handle):
        req = handle[1]
        with self.lock:
            self.running -= 1
            self.mem -= req.nbytes
        return float(req.params.sum())


def _req(fit, npv=4, npt=10, **kw):
    return ServeRequest(fit=fit, times=np.zeros(npt), params=np.full((npv, 9), float(fit)), **kw)


def test_results_slots_and_memory_budget():
    be = FakeBackend(dur=0.01)
    with Server(be, slots=3, mem_budget=1000) as srv:
        futs = [srv.submit(_req(i, npv=2 + i % 4)) for i in range(30)]
        res = [f.result(timeout=10) for f in futs]
    assert res == [float(np.full((2 + i % 4, 9), float(i)).sum()) for i in range(30)]
    assert be.max_running <= 3 and be.max_mem <= 1000
    assert be.max_running == 3                      # requests did overlap
    assert be.order == sorted(be.order)             # admitted in arrival order


def test_memory_admission_holds_back_then_admits():
    be = FakeBackend(dur=0.03)
    with Server(be, slots=8, mem_budget=1000) as srv:
        big = [srv.submit(_req(0, npv=6)) for _ in range(3)]     # 600 bytes each: one at a time
        for f in big:
            f.result(timeout=10)
    assert be.max_running == 1 and be.max_mem <= 1000


def test_oversize_request_is_rejected_at_submit():
    with Server(FakeBackend(), slots=2, mem_budget=500) as srv:
        with pytest.raises(AdmissionError):
            srv.submit(_req(0, npv=10))


def test_continuous_admission_while_others_run():
    # a long request occupies one slot; short requests submitted later are
    # admitted and finish while it is still running
    be = FakeBackend(dur={0: 0.3, 1: 0.01})
    with Server(be, slots=2, mem_budget=10_000) as srv:
        long_f = srv.submit(_req(0))
        time.sleep(0.02)
        short = [srv.submit(_req(1)) for _ in range(10)]
        for f in short:
            f.result(timeout=10)
        assert not long_f.done()
        long_f.result(timeout=10)
        done = {r.id: r for r in srv.completed}
    assert max(done[i].t_finish for i in range(1, 11)) < done[0].t_finish


def test_cancellation_and_deadline_before_admission():
    be = FakeBackend(dur=0.2)
    with Server(be, slots=1, mem_budget=10_000) as srv:
        first = srv.submit(_req(0))
        time.sleep(0.01)
        cancelled = srv.submit(_req(1))
        expired = srv.submit(_req(2, deadline_s=0.05))
        assert cancelled.cancel()
        first.result(timeout=10)
        with pytest.raises(TimeoutError):
            expired.result(timeout=10)
    assert cancelled.cancelled()
    assert 1 not in be.order and 2 not in be.order


def test_launch_failure_is_reported_and_releases_resources():
    be = FakeBackend(dur=0.01, fail_on=5)
    with Server(be, slots=2, mem_budget=10_000) as srv:
        bad = srv.submit(_req(5))
        good = srv.submit(_req(6))
        with pytest.raises(RuntimeError, match="injected"):
            bad.result(timeout=10)
        assert good.result(timeout=10) == float(np.full((4, 9), 6.0).sum())


def test_many_client_threads():
    be = FakeBackend(dur=0.002)
    results = {}
    with Server(be, slots=4, mem_budget=100_000) as srv:
        def client(c):
            for k in range(20):
                results[(c, k)] = srv.submit(_req(c * 100 + k)).result(timeout=30)
        ths = [threading.Thread(target=client, args=(c,)) for c in range(8)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        st = srv.stats()
    assert len(results) == 160 and st["requests"] == 160
    assert all(v == float(np.full((4, 9), float(key[0] * 100 + key[1])).sum()) for key, v in results.items())
    assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0


def test_latency_counts_from_the_intended_arrival():
    be = FakeBackend(dur=0.005)
    with Server(be, slots=2, mem_budget=10_000) as srv:
        late = _req(1, t_intended=time.perf_counter() - 0.05)    # submitted 50 ms after it was due
        srv.submit(late).result(timeout=10)
        st = srv.stats()
    assert st["latency_clock"].startswith("scheduler thread")
    assert st["latency_p50_ms"] >= 50 and st["client_latency_p50_ms"] >= 50


def test_request_is_not_admitted_before_its_arrival():
    be = FakeBackend(dur=0.001)
    with Server(be, slots=2, mem_budget=10_000) as srv:
        t_due = time.perf_counter() + 0.08
        early = _req(1, t_intended=t_due)
        fut = srv.submit(early)
        time.sleep(0.03)
        assert not fut.done()
        fut.result(timeout=10)
        st = srv.stats()
    rec = srv.completed[0]
    assert rec.t_admit >= t_due and st["latency_p50_ms"] < 60


@pytest.mark.parametrize("ss,npb", [(None, 1), ((3,), 1), ((1, 5, 2), 3), ((4, 4, 4, 4), 4)])
def test_request_points_is_the_sample_count(ss, npb):
    """points = npv x the sum over times of the supersampling factor of each time's passband,
    counted by brute force here; a caller-given count is used as it is."""
    rng = np.random.default_rng(npb)
    npv, npt = 7, 1001
    pb = rng.integers(0, npb, npt).astype(np.int32)
    r = ServeRequest(fit=0, times=np.zeros(npt), params=np.zeros((npv, 9)), pb_index=pb,
                     supersampling=None if ss is None else np.array(ss, np.int32))
    brute = npv * sum(1 if ss is None else ss[b] for b in pb)
    assert r.points == brute
    assert ServeRequest(fit=0, times=np.zeros(npt), params=np.zeros((npv, 9)), npoints=12).points == 12


def test_request_shapes_are_checked():
    from paper_2009_08500_gb300.serve import _check_shapes
    ok = ServeRequest(fit=0, times=np.zeros(10), params=np.zeros((3, 9)), pb_index=np.zeros(10, np.int32),
                      grad_flux=np.zeros((3, 10)))
    _check_shapes(ok, 9)
    with pytest.raises(ValueError, match="params"):
        _check_shapes(ok, 11)
    with pytest.raises(ValueError, match="pb_index"):
        _check_shapes(ServeRequest(fit=0, times=np.zeros(10), params=np.zeros((3, 9)), pb_index=np.zeros(9)), 9)
    with pytest.raises(ValueError, match="grad_flux"):
        _check_shapes(ServeRequest(fit=0, times=np.zeros(10), params=np.zeros((3, 9)), grad_flux=np.zeros((3, 9))), 9)
