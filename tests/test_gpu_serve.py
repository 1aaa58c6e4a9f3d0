"""Serving on the GPU: each result is the same alone and in the mix."""
import threading

import numpy as np
import pytest

from paper_2009_08500_gb300 import workloads as W
from paper_2009_08500_gb300.serve import CudaBackend, NativeServer, Server, ServeRequest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fits():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2009_08500_gb300 import rr
    out = {}
    for name, ld in [("a", "quadratic"), ("b", "nonlinear"), ("c", "tabulated"), ("d", "quadratic_tri")]:
        wl = W.make_small(ld, npv=1, npt=8, seed=ord(name))
        out[name] = (rr.model_for(wl), wl)
    return out


def _requests(fits, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    names = sorted(fits)
    for i in range(n):
        name = names[int(rng.integers(0, len(names)))]
        tmpl = fits[name][1]
        wl = W.make_small(tmpl.ld_model, npv=int(rng.integers(1, 48)), npt=int(rng.integers(500, 6000)),
                          seed=int(rng.integers(0, 2 ** 31)), ss=(int(rng.choice([1, 3, 7])),), exptime=(0.01,))
        gbar = rng.normal(size=(wl.npv, wl.npt)).astype(np.float32) if i % 3 == 0 else None
        reqs.append(ServeRequest(fit=name, times=wl.times, params=wl.params, pb_index=wl.pb_index,
                                 supersampling=wl.supersampling, exptime=wl.exptime, grad_flux=gbar))
    return reqs


def _alone(fits, req):
    import torch
    m = fits[req.fit][0]
    dev = m.device
    t = torch.as_tensor(req.times, dtype=torch.float64, device=dev)
    p = torch.as_tensor(req.params, dtype=torch.float64, device=dev)
    pb = torch.as_tensor(req.pb_index, dtype=torch.int32, device=dev)
    f = m.evaluate(t, p, pb, req.supersampling, req.exptime).cpu().numpy()
    g = None
    if req.grad_flux is not None:
        g = m.evaluate_grad(t, p, torch.as_tensor(req.grad_flux, device=dev), pb, req.supersampling,
                            req.exptime).cpu().numpy()
    return f, g


@pytest.mark.parametrize("budget", [8 << 30, 40 << 20])
def test_results_identical_alone_and_in_the_mix(fits, budget):
    reqs = _requests(fits, 36, seed=budget % 97)
    backend = CudaBackend({k: v[0] for k, v in fits.items()}, slots=6)
    futs = {}
    with Server(backend, slots=6, mem_budget=budget) as srv:
        def client(part):
            for r in part:
                futs[id(r)] = srv.submit(r)
        ths = [threading.Thread(target=client, args=(reqs[c::3],)) for c in range(3)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        res = {k: f.result(timeout=120) for k, f in futs.items()}
        stats = srv.stats()
    for r in reqs:
        out = res[id(r)]
        f, g = _alone(fits, r)
        assert np.array_equal(out["flux"], f)
        assert not out["pv_status"].any()
        if g is not None:
            assert np.array_equal(out["grad"], g)
    assert stats["requests"] == len(reqs)
    if budget > (1 << 30):
        assert stats["max_inflight"] > 1      # requests overlapped on the device


def test_served_flux_matches_oracle(fits):
    from oracle import model as om
    reqs = _requests(fits, 4, seed=5)
    backend = CudaBackend({k: v[0] for k, v in fits.items()}, slots=2)
    with Server(backend, slots=2) as srv:
        outs = [srv.submit(r).result(timeout=120) for r in reqs]
    for r, o in zip(reqs, outs):
        tmpl = fits[r.fit][1]
        s = om.build(tmpl.grid, tmpl.ld_model, 1, False, tmpl.profiles)
        ref = om.evaluate(s, r.times, r.pb_index, r.params, r.supersampling, r.exptime)
        assert np.abs(o["flux"] - ref).max() <= 1e-6


@pytest.mark.parametrize("budget", [8 << 30, 40 << 20])
def test_native_server_results_identical_alone_and_in_the_mix(fits, budget):
    reqs = _requests(fits, 36, seed=budget % 89 + 1)
    futs = {}
    with NativeServer({k: v[0] for k, v in fits.items()}, slots=6, mem_budget=budget) as srv:
        def client(part):
            for r in part:
                futs[id(r)] = srv.submit(r)
        ths = [threading.Thread(target=client, args=(reqs[c::3],)) for c in range(3)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        res = {k: f.result(timeout=120) for k, f in futs.items()}
        srv.drain()
        stats = srv.stats()
    for r in reqs:
        out = res[id(r)]
        f, g = _alone(fits, r)
        assert np.array_equal(out["flux"], f)
        assert not out["pv_status"].any()
        if g is not None:
            assert np.array_equal(out["grad"], g)
    assert stats["requests"] == len(reqs)
    assert stats["latency_p99_ms"] >= stats["latency_p50_ms"] > 0
    # latency on the library's clock: never longer than the same requests seen by the client
    assert stats["latency_clock"].startswith("library")
    assert stats["client_latency_p99_ms"] >= stats["latency_p50_ms"]


def test_native_server_writes_caller_result_buffers(fits):
    """Results land in the caller's pinned buffers when it passes them; a buffer of the wrong
    shape or not pinned is refused at submit."""
    import torch
    reqs = _requests(fits, 4, seed=23)
    with NativeServer({k: v[0] for k, v in fits.items()}, slots=2, mem_budget=8 << 30) as srv:
        for r in reqs:
            m = fits[r.fit][0]
            r.out = {"flux": torch.full((r.npv, r.npt), -3.0, dtype=torch.float32).pin_memory(),
                     "status": torch.full((r.npv,), -1, dtype=torch.int32).pin_memory()}
            if r.grad_flux is not None:
                r.out["grad"] = torch.zeros((r.npv, m.nparam), dtype=torch.float64).pin_memory()
            out = srv.submit(r).result(timeout=60)
            assert out["flux"].ctypes.data == r.out["flux"].data_ptr()
            f, g = _alone(fits, r)
            assert np.array_equal(r.out["flux"].numpy(), f) and not r.out["status"].any()
            if g is not None:
                assert np.array_equal(r.out["grad"].numpy(), g)
        bad = _requests(fits, 1, seed=24)[0]
        bad.out = {"flux": torch.empty((bad.npv, bad.npt + 1), dtype=torch.float32).pin_memory()}
        with pytest.raises(ValueError):
            srv.submit(bad)
        bad.out = {"flux": torch.empty((bad.npv, bad.npt), dtype=torch.float32)}
        with pytest.raises(ValueError):
            srv.submit(bad)


def test_native_server_checks_that_host_buffers_are_page_locked(fits):
    """The library refuses pageable host buffers (RR_EPAGEABLE, checked at both ends of each); the
    Python server then copies them into pinned memory, so pageable torch inputs still give the
    results of the model alone."""
    import torch
    r = _requests(fits, 1, seed=29)[0]
    m = fits[r.fit][0]
    t, p = torch.from_numpy(np.ascontiguousarray(r.times)), torch.from_numpy(np.ascontiguousarray(r.params))
    pb = torch.from_numpy(np.ascontiguousarray(r.pb_index, np.int32))
    with NativeServer({k: v[0] for k, v in fits.items()}, slots=2, mem_budget=8 << 30) as srv:
        ss = srv._small(r.supersampling, m.npb, np.int32, 1)
        ex = srv._small(r.exptime, m.npb, np.float64, 0.0)
        flux = torch.empty((r.npv, r.npt), dtype=torch.float32).pin_memory()
        status = torch.empty(r.npv, dtype=torch.int32).pin_memory()
        h = {"t": t, "p": p.pin_memory(), "pb": pb.pin_memory(), "g": None, "flux": flux, "status": status,
             "grad": None}
        assert srv._submit_c(r, m, h, ss, ex, 0) == -7           # times pageable
        # the same times inside a larger pinned block are accepted
        big = torch.zeros(8 << 20, dtype=torch.float64).pin_memory()
        big[: r.npt] = t
        r._host = dict(h, t=big[: r.npt])
        assert srv._submit_c(r, m, r._host, ss, ex, 0) >= 0
        srv.drain()
        req = ServeRequest(fit=r.fit, times=t, params=p, pb_index=pb, supersampling=r.supersampling,
                           exptime=r.exptime, grad_flux=r.grad_flux)
        out = srv.submit(req).result(timeout=60)
    f, _ = _alone(fits, r)
    assert np.array_equal(out["flux"], f)


def test_native_server_rejects_oversize_requests(fits):
    from paper_2009_08500_gb300.serve import AdmissionError
    reqs = _requests(fits, 2, seed=3)
    with NativeServer({k: v[0] for k, v in fits.items()}, slots=2, mem_budget=1 << 10) as srv:
        with pytest.raises(AdmissionError):
            srv.submit(reqs[0])


def test_native_server_release_time(fits):
    """A request submitted ahead of its arrival is admitted no earlier; its
    latency counts from the arrival; a late one counts its lateness."""
    import time
    reqs = _requests(fits, 3, seed=17)
    with NativeServer({k: v[0] for k, v in fits.items()}, slots=2, mem_budget=8 << 30) as srv:
        t_due = time.perf_counter() + 0.08
        reqs[0].t_intended = t_due
        f0 = srv.submit(reqs[0])
        time.sleep(0.03)
        assert not f0.done()
        out0 = f0.result(timeout=60)
        reqs[1].t_intended = time.perf_counter() - 0.05       # already 50 ms late
        out1 = srv.submit(reqs[1]).result(timeout=60)
        srv.drain()
        recs = {r.id: r for r in srv.completed}
        stats = srv.stats()
    r0, r1 = recs[reqs[0].id], recs[reqs[1].id]
    off = srv._clock_off
    # the library's arrival time is the intended one (clocks mapped to within a millisecond)
    assert abs((r0.server_ns[0] - off) * 1e-9 - t_due) < 1e-3
    assert r0.server_ns[1] >= r0.server_ns[0] and r0.t_admit >= t_due - 1e-3
    assert (r1.server_ns[2] - r1.server_ns[0]) * 1e-9 >= 0.05
    assert stats["requests"] == 2
    for r, out in ((reqs[0], out0), (reqs[1], out1)):
        f, g = _alone(fits, r)
        assert np.array_equal(out["flux"], f)


def test_a_device_wait_that_gave_up_is_reported_by_the_request(fits):
    """A bounded device wait that runs out (the failure self-test's queue-slot wait, on a flag that
    nothing sets) sets the fit's error word; the next request of that fit through the server
    reports RR_ETIMEOUT, and the word is cleared for the one after it."""
    import torch
    from paper_2009_08500_gb300 import rr
    m, tmpl = fits["a"]
    m.selftest_wait(1)
    torch.cuda.synchronize()
    wl = W.make_small(tmpl.ld_model, npv=3, npt=900, seed=5)

    def req():
        return ServeRequest(fit="a", times=wl.times, params=wl.params, pb_index=wl.pb_index,
                            supersampling=wl.supersampling, exptime=wl.exptime)

    with NativeServer({"a": m}, slots=2, mem_budget=1 << 30, device=m.device.index or 0) as srv:
        with pytest.raises(rr.RRError) as ei:
            srv.submit(req()).result(timeout=60)
        assert ei.value.status == 6
        out = srv.submit(req()).result(timeout=60)
    assert out["flux"].shape == (3, 900) and np.all(out["pv_status"] == 0)
