"""Continuous-batching evaluation server for many concurrent fits.

Requests (a parameter batch for one fit's light curve, optionally with a
cotangent for the gradient) arrive from many fitting loops at once.  The
server keeps every fit's model context -- its LD profiles and (k, g) tables
-- resident on the device, and:

* admits queued requests in arrival order whenever a stream slot and enough
  device memory (inputs + outputs + workspace, counted exactly) are free;
* runs every admitted request on its own CUDA stream, so the work of
  requests admitted at different times overlaps on the device;
* completes a request's future as soon as its stream has finished (event
  polling), releasing its memory and slot for the next admission;
* records arrival / admission / launch / finish times, points and bytes of
  every request (p50 / p99 latency and points/s come from these).

Results do not depend on what else is in flight: each request runs the same
kernels with the same tiling as it would alone (the adjoint's summation
order depends on the request's own number of times only).

The scheduling logic is backend-agnostic (``Backend``); ``CudaBackend`` runs
requests through the library, tests may plug in a host-only backend.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field
from typing import Any, Callable, Deque, Dict, List, Optional

import numpy as np


class AdmissionError(RuntimeError):
    """The request can never be admitted (larger than the memory budget)."""


@dataclass
class ServeRequest:
    fit: Any
    times: np.ndarray
    params: np.ndarray
    pb_index: Optional[np.ndarray] = None
    supersampling: Optional[np.ndarray] = None
    exptime: Optional[np.ndarray] = None
    grad_flux: Optional[np.ndarray] = None      # cotangent: the request also wants d/d(params)
    deadline_s: Optional[float] = None          # seconds after arrival; expired requests are not admitted
    # time.perf_counter() at which the request arrives (an open-loop client's
    # schedule): it is not admitted earlier, and its latency counts from then
    # even when the submit call comes later
    t_intended: Optional[float] = None
    # caller-owned pinned host result buffers {"flux", "status"[, "grad"]} of the request's
    # shapes and types, written instead of buffers allocated on submit (a client that reuses its
    # buffers); the caller leaves them alone until the future is done
    out: Optional[dict] = None
    # light-curve samples of the request, when the caller knows them; else counted on first use
    npoints: Optional[int] = None
    # filled by the server
    id: int = -1
    nbytes: int = 0
    t_arrival: float = 0.0
    t_admit: float = 0.0
    t_launch: float = 0.0
    t_finish: float = 0.0
    server_ns: Optional[tuple] = None           # library clock: submitted, admitted, finished (ns)
    future: Future = field(default_factory=Future)

    @property
    def npv(self) -> int:
        return int(self.params.shape[0])

    @property
    def npt(self) -> int:
        return int(self.times.shape[0])

    @property
    def points(self) -> int:
        """npv x the sum over times of the supersampling factor of each time's passband (counted
        once, and without a pass over the times when every passband has the same factor)."""
        if self.npoints is None:
            if self.supersampling is None:
                per_pv = self.npt
            else:
                ss = np.asarray(self.supersampling, dtype=np.int64).reshape(-1)
                if self.pb_index is None or ss.size == 1 or np.all(ss == ss[0]):
                    per_pv = self.npt * int(ss[0])
                else:
                    counts = np.bincount(np.asarray(self.pb_index).reshape(-1), minlength=ss.size)
                    per_pv = int(counts[:ss.size] @ ss)
            self.npoints = self.npv * per_pv
        return self.npoints


@dataclass
class Done:
    """What the server keeps of a finished request (its buffers belong to the caller)."""
    id: int
    points: int
    ok: bool
    t_arrival: float
    t_admit: float
    t_finish: float
    t_intended: float
    server_ns: Optional[tuple] = None


def _check_shapes(req: ServeRequest, nparam: int) -> None:
    """The array shapes a model's request must have (its rows are read with these strides)."""
    ps = req.params.shape
    if len(ps) != 2 or ps[1] != nparam:
        raise ValueError(f"params must have shape (npv, {nparam})")
    npt = req.times.shape[0]
    pb = req.pb_index
    if pb is not None and (len(pb.shape) != 1 or pb.shape[0] != npt):
        raise ValueError("pb_index must have one entry per time")
    g = req.grad_flux
    if g is not None and (len(g.shape) != 2 or g.shape[0] != ps[0] or g.shape[1] != npt):
        raise ValueError(f"grad_flux must have shape ({ps[0]}, {npt})")


def _done_record(req: ServeRequest, ok: bool) -> Done:
    t_int = req.t_arrival if req.t_intended is None else req.t_intended
    return Done(req.id, req.points, ok, req.t_arrival, req.t_admit, req.t_finish, t_int, req.server_ns)


class Backend:
    """What the scheduler needs from an executor."""

    def nbytes(self, req: ServeRequest) -> int:
        raise NotImplementedError

    def prepare(self, req: ServeRequest) -> None:
        """Host-side preparation, run on the submitting thread (optional)."""

    def launch(self, req: ServeRequest, slot: int) -> Any:
        """Enqueue the request on stream `slot`; return a handle for `done` / `finish`."""
        raise NotImplementedError

    def done(self, handle: Any) -> bool:
        raise NotImplementedError

    def finish(self, handle: Any) -> Any:
        """Result of a completed request (releases its resources)."""
        raise NotImplementedError


class Server:
    """Continuous-batching scheduler.

    slots       requests that may be in flight at once (one stream each)
    mem_budget  device bytes that in-flight requests may hold together
    """

    def __init__(self, backend: Backend, slots: int = 8, mem_budget: int = 8 << 30, poll_s: float = 50e-6):
        self.backend = backend
        self.slots = slots
        self.mem_budget = mem_budget
        self.poll_s = poll_s
        self._queue: Deque[ServeRequest] = collections.deque()
        self._inflight: Dict[int, tuple] = {}        # slot -> (request, handle)
        self._free_slots = list(range(slots))[::-1]
        self._mem_used = 0
        self._lock = threading.Condition()
        self._next_id = 0
        self._stop = False
        self.completed: List[Done] = []
        self.max_inflight_seen = 0
        self._thread = threading.Thread(target=self._run, name="rr-serve", daemon=True)
        self._thread.start()

    # -- client side ------------------------------------------------------------
    def submit(self, req: ServeRequest) -> Future:
        req.nbytes = self.backend.nbytes(req)
        if req.nbytes > self.mem_budget:
            raise AdmissionError(f"request needs {req.nbytes} bytes, more than the {self.mem_budget}-byte budget")
        req.points
        self.backend.prepare(req)
        with self._lock:
            if self._stop:
                raise RuntimeError("server is stopped")
            req.id = self._next_id
            self._next_id += 1
            req.t_arrival = time.perf_counter()
            self._queue.append(req)
            self._lock.notify()
        return req.future

    def close(self, wait: bool = True):
        with self._lock:
            self._stop = True
            self._lock.notify()
        if wait:
            self._thread.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def drain(self, timeout_s: float = 600.0):
        """Wait until nothing is queued or in flight."""
        t0 = time.perf_counter()
        while True:
            with self._lock:
                if not self._queue and not self._inflight:
                    return
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain")
            time.sleep(1e-3)

    # -- scheduler --------------------------------------------------------------
    def _admit(self):
        """Admit queued requests in order while a slot and memory are free (lock held)."""
        now = time.perf_counter()
        while self._queue and self._free_slots:
            req = self._queue[0]
            if req.future.cancelled():
                self._queue.popleft()
                continue
            if req.t_intended is not None and req.t_intended > now:
                break                                   # in order: not released yet
            if req.deadline_s is not None and now - req.t_arrival > req.deadline_s:
                self._queue.popleft()
                req.future.set_exception(TimeoutError(f"request {req.id} expired before admission"))
                continue
            if self._mem_used + req.nbytes > self.mem_budget:
                break                                   # in order: wait for memory to free up
            self._queue.popleft()
            if not req.future.set_running_or_notify_cancel():
                continue
            slot = self._free_slots.pop()
            self._mem_used += req.nbytes
            req.t_admit = time.perf_counter()
            try:
                handle = self.backend.launch(req, slot)
            except Exception as exc:                  # launch failed: report it, release resources
                self._mem_used -= req.nbytes
                self._free_slots.append(slot)
                req.future.set_exception(exc)
                continue
            req.t_launch = time.perf_counter()
            self._inflight[slot] = (req, handle)
            self.max_inflight_seen = max(self.max_inflight_seen, len(self._inflight))

    def _reap(self):
        """Complete finished requests (lock held)."""
        for slot in list(self._inflight):
            req, handle = self._inflight[slot]
            exc = None
            try:
                if not self.backend.done(handle):
                    continue
                result = self.backend.finish(handle)
            except Exception as e:
                exc = e
            req.t_finish = time.perf_counter()
            del self._inflight[slot]
            self._free_slots.append(slot)
            self._mem_used -= req.nbytes
            req._host = None
            # the record first: a caller that sees the future done also sees it in the stats
            self.completed.append(_done_record(req, exc is None))
            if exc is None:
                req.future.set_result(result)
            else:
                req.future.set_exception(exc)

    def _run(self):
        while True:
            with self._lock:
                self._reap()
                self._admit()
                if self._stop and not self._queue and not self._inflight:
                    return
                if not self._inflight and not self._queue:
                    self._lock.wait(timeout=0.05)
                    continue
            time.sleep(self.poll_s)

    # -- metrics ----------------------------------------------------------------
    def stats(self) -> dict:
        """Throughput and latency of the finished requests.

        A request arrives at its intended time (ServeRequest.t_intended: the
        schedule of an open-loop client), else at its submit call.
        latency_*: the scheduler's own clock, from arrival to completion -- for
        the native server the library's steady clock (arrival until the
        request's stream passed it), so a pause of the Python poller does not
        stretch it, while a client that submits late has its lateness counted.
        client_latency_*: from arrival until the poller completed the future.
        """
        done = [r for r in self.completed if r.ok]
        if not done:
            return {"requests": 0}
        if all(r.server_ns is not None for r in done):
            lat = np.array([(r.server_ns[2] - r.server_ns[0]) * 1e-9 for r in done])
            wait = np.array([(r.server_ns[1] - r.server_ns[0]) * 1e-9 for r in done])
            clock = "library steady clock (rr_server_submit to stream completion)"
        else:
            lat = np.array([r.t_finish - r.t_intended for r in done])
            wait = np.array([r.t_admit - r.t_intended for r in done])
            clock = "scheduler thread (arrival to completion)"
        client = np.array([r.t_finish - r.t_intended for r in done])
        t0 = min(min(r.t_arrival, r.t_intended) for r in done)
        t1 = max(r.t_finish for r in done)
        pts = sum(r.points for r in done)
        return {"requests": len(done), "points": pts, "points_per_s": pts / (t1 - t0),
                "latency_p50_ms": float(np.percentile(lat, 50) * 1e3),
                "latency_p99_ms": float(np.percentile(lat, 99) * 1e3),
                "queue_wait_p50_ms": float(np.percentile(wait, 50) * 1e3),
                "queue_wait_p99_ms": float(np.percentile(wait, 99) * 1e3),
                "client_latency_p50_ms": float(np.percentile(client, 50) * 1e3),
                "client_latency_p99_ms": float(np.percentile(client, 99) * 1e3),
                "latency_clock": clock,
                "max_inflight": self.max_inflight_seen, "wall_s": t1 - t0}


class CudaBackend(Backend):
    """Runs requests through librr: one CUDA stream per slot, device-resident fit contexts.

    fits: {fit id: rr.Model} (built); requests carry host arrays (pinned when submitted).
    """

    def __init__(self, fits: Dict[Any, Any], slots: int, device: int = 0):
        import torch
        self.torch = torch
        self.fits = fits
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]

    def nbytes(self, req: ServeRequest) -> int:
        """Device bytes of the request: its scratch for rr_enqueue_host (inputs, outputs, workspace)."""
        m = self.fits[req.fit]
        _check_shapes(req, m.nparam)
        return m.request_bytes(req.npv, req.npt, req.grad_flux is not None)

    def prepare(self, req: ServeRequest) -> None:
        """Pinned host inputs and pinned result buffers (submitting thread).  Inputs
        that are already pinned CPU tensors of the right type are used as they are."""
        torch = self.torch
        m = self.fits[req.fit]
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32}

        def pin(a, dt):
            if isinstance(a, torch.Tensor) and a.device.type == "cpu":
                t = a.to(tdt[dt]).contiguous()
                return t if t.is_pinned() else t.pin_memory()
            return torch.from_numpy(np.ascontiguousarray(a, dt)).pin_memory()

        given = req.out or {}

        def result(name, shape, dt):
            b = given.get(name)
            if b is None:
                return torch.empty(shape, dtype=dt, pin_memory=True)
            if not (isinstance(b, torch.Tensor) and b.dtype == dt and tuple(b.shape) == shape
                    and b.is_contiguous() and b.is_pinned()):
                raise ValueError(f"out[{name!r}] must be a pinned contiguous {dt} tensor of shape {shape}")
            return b

        h = {"t": pin(req.times, np.float64), "p": pin(req.params, np.float64),
             "pb": None if req.pb_index is None else pin(req.pb_index, np.int32),
             "flux": result("flux", (req.npv, req.npt), m.dtype),
             "status": result("status", (req.npv,), torch.int32), "g": None, "grad": None}
        if req.grad_flux is not None:
            h["g"] = pin(req.grad_flux, np.float32 if m.precision == "mixed" else np.float64)
            h["grad"] = result("grad", (req.npv, m.nparam), torch.float64)
        req._host = h

    def launch(self, req: ServeRequest, slot: int):
        """One library call enqueues the copies in, the kernels and the copies out on the slot's stream."""
        torch = self.torch
        m = self.fits[req.fit]
        s = self.streams[slot]
        h = req._host
        with torch.cuda.stream(s):
            # allocated on the slot's stream: the caching allocator reuses it only after that stream's work
            scratch = torch.empty(max(req.nbytes, 256), dtype=torch.uint8, device=self.device)
        m.enqueue_host(h["t"], h["p"], h["pb"], req.supersampling, req.exptime, h["g"], h["flux"], h["grad"],
                       h["status"], scratch, s)
        ev = torch.cuda.Event()
        ev.record(s)
        # the scratch stays referenced by the handle until the event has completed
        return (ev, h, scratch)

    def done(self, handle) -> bool:
        return handle[0].query()

    def finish(self, handle):
        _, h, _ = handle
        out = {"flux": h["flux"].numpy(), "pv_status": h["status"].numpy()}
        if h["grad"] is not None:
            out["grad"] = h["grad"].numpy()
        return out


class NativeServer:
    """Continuous batching in the library's worker thread (rr_server_*).

    The library admits requests in arrival order by stream slots and device
    memory, enqueues each on its own stream and reports completion; this
    class only prepares pinned host buffers on submit and completes the
    futures from one poller thread.  fits: {fit id: rr.Model} (built); while
    the server runs, only the server may use those models.
    """

    def __init__(self, fits: Dict[Any, Any], slots: int = 8, mem_budget: int = 8 << 30, device: int = 0):
        import ctypes

        import torch

        from . import rr
        self.torch, self.ctypes, self.rr = torch, ctypes, rr
        self.fits = fits
        self.lib = rr.load_library()
        h = ctypes.c_void_p()
        st = self.lib.rr_server_create(device, slots, mem_budget, ctypes.byref(h))
        if st != 0:
            raise rr.RRError(st, "rr_server_create failed")
        self._h = h
        self.mem_budget = mem_budget
        self._clock_off = self._clock_offset()
        self._backend = CudaBackend.__new__(CudaBackend)   # reuse its host-buffer preparation
        self._backend.torch, self._backend.fits = torch, fits
        self._lock = threading.Lock()
        self._inflight: Dict[int, ServeRequest] = {}
        self._stop = False
        self.completed: List[ServeRequest] = []
        self.max_inflight_seen = 0
        self._poller = threading.Thread(target=self._poll, name="rr-native-serve-poll", daemon=True)
        self._poller.start()

    def _clock_offset(self) -> int:
        """library steady clock - time.perf_counter_ns(), from the tightest of a few readings."""
        best = None
        for _ in range(7):
            a = time.perf_counter_ns()
            n = self.lib.held.rr_server_now_ns()
            b = time.perf_counter_ns()
            if best is None or b - a < best[0]:
                best = (b - a, n - (a + b) // 2)
        return best[1]

    def submit(self, req: ServeRequest) -> Future:
        """Queue a request.  With req.t_intended (time.perf_counter() seconds) the
        request arrives then: the library does not admit it earlier, and its
        latency counts from that time even when the submit call comes later."""
        rr = self.rr
        m = self.fits[req.fit]
        _check_shapes(req, m.nparam)
        req.t_arrival = time.perf_counter()
        release = 0 if req.t_intended is None else max(1, int(req.t_intended * 1e9) + self._clock_off)
        req.points
        ss = self._small(req.supersampling, m.npb, np.int32, 1)
        ex = self._small(req.exptime, m.npb, np.float64, 0.0)
        req._ssex = (ss, ex)
        # torch CPU tensors of the right type and layout go to the library as they are (it checks that
        # they are page-locked); anything else, or a buffer the library finds pageable, is copied into
        # pinned memory first
        h = self._as_given(req, m)
        rid = -7 if h is None else self._submit_c(req, m, h, ss, ex, release)
        if rid == -7:
            self._backend.prepare(req)
            h = req._host
            rid = self._submit_c(req, m, h, ss, ex, release)
        if rid < 0:
            if -rid == 2:
                raise AdmissionError(f"request larger than the {self.mem_budget}-byte budget")
            raise rr.RRError(-rid, "rr_server_submit rejected the request")
        return req.future

    @staticmethod
    def _small(x, n, dtype, default):
        if type(x) is np.ndarray and x.dtype == dtype and x.shape == (n,) and x.flags.c_contiguous:
            return x
        return np.ascontiguousarray(np.broadcast_to(np.asarray(default if x is None else x, dtype=dtype), (n,)))

    def _as_given(self, req, m):
        """The request's host buffers without conversion, or None when one needs converting."""
        torch = self.torch
        T = torch.Tensor

        def ok(a, dt, shape):
            return (type(a) is T and a.dtype == dt and a.device.type == "cpu" and a.is_contiguous()
                    and tuple(a.shape) == shape)

        npv, npt = req.npv, req.npt
        out = req.out or {}
        h = {"t": req.times, "p": req.params, "pb": req.pb_index, "g": req.grad_flux,
             "flux": out.get("flux"), "status": out.get("status"), "grad": out.get("grad")}
        if not (ok(h["t"], torch.float64, (npt,)) and ok(h["p"], torch.float64, (npv, m.nparam))
                and (h["pb"] is None or ok(h["pb"], torch.int32, (npt,)))
                and ok(h["flux"], m.dtype, (npv, npt)) and ok(h["status"], torch.int32, (npv,))):
            return None
        if req.grad_flux is None:
            h["grad"] = None
        elif not (ok(h["g"], m.dtype, (npv, npt)) and ok(h["grad"], torch.float64, (npv, m.nparam))):
            return None
        req._host = h
        return h

    def _submit_c(self, req, m, h, ss, ex, release):
        ctypes, rr = self.ctypes, self.rr
        with self._lock:
            if self._stop:
                raise RuntimeError("server is stopped")
            rid = self.lib.held.rr_server_submit_at(self._h, m._h, rr._ptr(h["t"]), rr._ptr(h["pb"]), req.npt,
                                                    rr._ptr(h["p"]), req.npv,
                                                    ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                    ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                    rr._ptr(h["g"]), rr._ptr(h["flux"]), rr._ptr(h["grad"]),
                                                    rr._ptr(h["status"]), release)
            if rid >= 0:
                req.id = int(rid)
                self._inflight[req.id] = req
                self.max_inflight_seen = max(self.max_inflight_seen, len(self._inflight))
        return rid

    def _poll(self):
        ctypes = self.ctypes
        n = 64
        ids = (ctypes.c_int64 * n)()
        sts = (ctypes.c_int32 * n)()
        tms = (ctypes.c_int64 * (3 * n))()
        while True:
            got = self.lib.rr_server_poll(self._h, ids, sts, tms, n, 20000)
            now = time.perf_counter()
            with self._lock:
                reqs = [self._inflight.pop(int(ids[i])) for i in range(max(got, 0))]
            for i, req in enumerate(reqs):
                req.t_finish = now
                req.server_ns = (int(tms[3 * i]), int(tms[3 * i + 1]), int(tms[3 * i + 2]))
                req.t_admit = (tms[3 * i + 1] - self._clock_off) * 1e-9
                h = req._host
                req._host = None
                # the record first: a caller that sees the future done also sees it in the stats
                self.completed.append(_done_record(req, sts[i] == 0))
                if sts[i] != 0:
                    req.future.set_exception(self.rr.RRError(int(sts[i]), "request failed in the server"))
                else:
                    out = {"flux": h["flux"].numpy(), "pv_status": h["status"].numpy()}
                    if h["grad"] is not None:
                        out["grad"] = h["grad"].numpy()
                    req.future.set_result(out)
            with self._lock:
                if self._stop and not self._inflight:
                    return

    def reset_stats(self):
        """Forget the finished requests (a new measurement window on a running server)."""
        with self._lock:
            self.completed = []
            self.max_inflight_seen = len(self._inflight)

    def drain(self, timeout_s: float = 600.0):
        t0 = time.perf_counter()
        while True:
            with self._lock:
                if not self._inflight:
                    return
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain")
            time.sleep(1e-3)

    def close(self):
        with self._lock:
            self._stop = True
        self._poller.join()
        if self._h:
            self.lib.rr_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    stats = Server.stats

