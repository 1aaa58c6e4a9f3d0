"""Python binding of librr (argument marshalling only).

Every numerical step runs in the library's CUDA kernels; this module checks
tensor placement and dtypes, passes raw pointers and the current CUDA stream
through the C ABI of ``include/rr.h``, and wraps the adjoint in a
``torch.autograd.Function``.  There is no CPU fallback: without a built
``librr.so`` or a CUDA device every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librr.so")

LD_MODELS = {"uniform": 0, "quadratic": 1, "quadratic_tri": 2, "nonlinear": 3, "tabulated": 4, "linear": 5,
             "general": 6, "logarithmic": 7, "exponential": 8, "power2": 9, "power2_pm": 10}
PRECISIONS = {"fp64": 0, "mixed": 1}
STATUS = {0: "RR_OK", 1: "RR_EINVAL", 2: "RR_ENOMEM", 3: "RR_ECUDA", 4: "RR_ESTATE", 5: "RR_EDOMAIN",
          6: "RR_ETIMEOUT", 7: "RR_EPAGEABLE"}
TABLES = {"ze": 0, "zm": 1, "mu": 2, "weights": 3, "basis": 4, "istar": 5, "proj": 6}

PV_K_RANGE, PV_E_RANGE, PV_B_RANGE, PV_P_RANGE = 1, 2, 4, 8
PV_NONFINITE, PV_LD_INVALID, PV_A_RANGE, PV_KEPLER = 16, 32, 64, 128

#: every exported entry point of include/rr.h
EXPORTS = ["rr_create", "rr_destroy", "rr_set_ld_profile", "rr_build_weights", "rr_nparam",
           "rr_workspace_bytes", "rr_evaluate", "rr_evaluate_grad", "rr_read_table",
           "rr_sync_status", "rr_last_error", "rr_launch_count", "rr_profile", "rr_profile_read",
           "rr_evaluate_noalloc", "rr_prepare", "rr_evaluate_prepared", "rr_evaluate_grad_prepared",
           "rr_evaluate_host", "rr_request_bytes", "rr_enqueue_host", "rr_server_create", "rr_server_destroy",
           "rr_server_submit", "rr_server_submit_at", "rr_server_now_ns", "rr_server_poll", "rr_server_pending", "rr_exact_flux", "rr_choose_grid",
           "rr_selftest_wait", "rr_count_samples", "rr_count_read", "rr_host_path", "rr_evaluate_both_prepared"]
KERNELS = {"ld_basis": 0, "weights": 1, "pv_setup": 2, "flux": 3, "grad": 4, "grad_reduce": 5, "points": 6,
           "direct": 7}
#: sample counters of the counting form (include/rr.h RR_COUNT_*)
COUNTS = ["cand", "samples", "orbit", "circular", "newton", "transit", "refined", "lens"]


class RRConfig(ctypes.Structure):
    _fields_ = [("zcut", ctypes.c_double), ("nzin", ctypes.c_int32), ("nzlimb", ctypes.c_int32),
                ("ng", ctypes.c_int32), ("nk", ctypes.c_int32), ("k0", ctypes.c_double),
                ("k1", ctypes.c_double), ("npb", ctypes.c_int32), ("ld_model", ctypes.c_int32),
                ("chromatic", ctypes.c_int32), ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("ncoef", ctypes.c_int32), ("direct", ctypes.c_int32), ("shared_weights", ctypes.c_int32),
                ("k_small", ctypes.c_double)]


class RRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librr.so and declare the C signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2009_08500_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, sz, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)
    L.rr_create.argtypes = [ctypes.POINTER(RRConfig), ctypes.POINTER(vp)]
    L.rr_destroy.argtypes = [vp]
    L.rr_set_ld_profile.argtypes = [vp, i32, dp, dp, i32]
    L.rr_build_weights.argtypes = [vp, vp]
    L.rr_nparam.argtypes = [vp]
    L.rr_nparam.restype = i32
    L.rr_workspace_bytes.argtypes = [vp, i32, i32, i32]
    L.rr_workspace_bytes.restype = sz
    L.rr_evaluate.argtypes = [vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, vp, sz, vp]
    L.rr_evaluate_grad.argtypes = [vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, vp, vp, sz, vp]
    L.rr_evaluate_noalloc.argtypes = [vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, vp]
    L.rr_prepare.argtypes = [vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, sz, vp]
    L.rr_evaluate_prepared.argtypes = [vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, vp, sz, vp]
    L.rr_evaluate_grad_prepared.argtypes = [vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, vp, vp, sz,
                                            vp]
    L.rr_evaluate_host.argtypes = [vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, vp, vp, i32]
    L.rr_evaluate_both_prepared.argtypes = [vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, vp, vp, vp,
                                            sz, vp]
    L.rr_request_bytes.argtypes = [vp, i32, i32, i32]
    L.rr_request_bytes.restype = sz
    L.rr_enqueue_host.argtypes = [vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, vp, vp, vp, sz, vp]
    L.rr_server_create.argtypes = [i32, i32, sz, ctypes.POINTER(vp)]
    L.rr_server_create.restype = ctypes.c_int
    L.rr_server_destroy.argtypes = [vp]
    L.rr_server_destroy.restype = ctypes.c_int
    L.rr_server_submit.argtypes = [vp, vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, vp, vp]
    L.rr_server_submit.restype = i64
    L.rr_server_submit_at.argtypes = [vp, vp, vp, vp, i32, vp, i32, ctypes.POINTER(i32), dp, vp, vp, vp, vp, i64]
    L.rr_server_submit_at.restype = i64
    L.rr_server_now_ns.argtypes = []
    L.rr_server_now_ns.restype = i64
    L.rr_server_poll.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i64), i32, i32]
    L.rr_server_poll.restype = i32
    L.rr_server_pending.argtypes = [vp]
    L.rr_server_pending.restype = i32
    # the server's submission and clock through a handle that keeps the GIL during the call:
    # they take microseconds and never block for long, and releasing and retaking the GIL
    # around them costs more than the call when other Python threads are busy
    H = ctypes.PyDLL(path)
    H.rr_server_submit_at.argtypes = L.rr_server_submit_at.argtypes
    H.rr_server_submit_at.restype = i64
    H.rr_server_now_ns.argtypes = []
    H.rr_server_now_ns.restype = i64
    L.held = H
    L.rr_read_table.argtypes = [vp, i32, dp, i64]
    L.rr_read_table.restype = i64
    L.rr_sync_status.argtypes = [vp, vp]
    L.rr_last_error.argtypes = [vp]
    L.rr_last_error.restype = ctypes.c_char_p
    L.rr_launch_count.argtypes = [vp]
    L.rr_launch_count.restype = i64
    L.rr_profile.argtypes = [vp, i32]
    L.rr_profile_read.argtypes = [vp, i32, dp, ctypes.POINTER(i64), i32]
    L.rr_exact_flux.argtypes = [vp, vp, vp, i32, dp, i32, vp, vp]
    L.rr_selftest_wait.argtypes = [vp, i32, vp]
    L.rr_count_samples.argtypes = [vp, i32]
    L.rr_count_read.argtypes = [vp, i32, ctypes.POINTER(i64), i32]
    L.rr_host_path.argtypes = [vp]
    L.rr_host_path.restype = i32
    L.rr_choose_grid.argtypes = [ctypes.POINTER(RRConfig), dp, i32, dp, dp, dp, i32, ctypes.c_double, dp]
    for name in ("rr_exact_flux", "rr_choose_grid", "rr_selftest_wait", "rr_create", "rr_destroy", "rr_set_ld_profile", "rr_build_weights", "rr_evaluate",
                 "rr_evaluate_grad", "rr_sync_status", "rr_profile", "rr_profile_read", "rr_evaluate_noalloc",
                 "rr_prepare", "rr_evaluate_prepared", "rr_evaluate_grad_prepared", "rr_evaluate_host",
                 "rr_enqueue_host", "rr_count_samples", "rr_count_read", "rr_evaluate_both_prepared"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def _host_array(x, n, dtype, default):
    if x is None:
        x = [default] * n
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=dtype), (n,)))
    return a


class Model:
    """A RoadRunner model context: radial grid, LD profiles and (k, g) tables on one GPU.

    ld_model   'uniform' | 'quadratic' | 'quadratic_tri' | 'nonlinear' | 'tabulated' | 'linear' |
               'general' | 'logarithmic' | 'exponential'
    npb        passbands; chromatic: one radius ratio per passband
    precision  'mixed' (FP32 bulk, float flux) or 'fp64' (double flux)
    grid       dict(zcut, nzin, nzlimb, ng, nk, k0, k1)
    n_general  terms of the general law (1..4)
    direct     the direct model: weights for each k computed per call, interpolation in g
               only, any 0 < k < 1 (the grid's nk, k0, k1 are then unused)
    shared_weights  with chromatic k: one weight array per pv at the mean of its radius ratios
               (transmission spectroscopy); area and g keep each passband's k
    k_small    small-planet approximation below this radius ratio (0 = off): the profile at the
               planet's centre instead of the weighted average
    """

    def __init__(self, ld_model: str = "quadratic", npb: int = 1, chromatic: bool = False,
                 precision: str = "mixed", grid: Optional[dict] = None, device: int = 0, n_general: int = 0,
                 direct: bool = False, shared_weights: bool = False, k_small: float = 0.0):
        from .workloads import GRID
        g = dict(GRID if grid is None else grid)
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = torch.device("cuda", device)
        self.ld_model, self.npb, self.chromatic, self.precision = ld_model, npb, chromatic, precision
        self.direct = bool(direct)
        self.shared_weights = bool(shared_weights)
        self.k_small = float(k_small)
        self.grid = g
        cfg = RRConfig(g["zcut"], g["nzin"], g["nzlimb"], g["ng"], g["nk"], g["k0"], g["k1"], npb,
                       LD_MODELS[ld_model], int(chromatic), PRECISIONS[precision], device,
                       int(n_general) if ld_model == "general" else 0, int(bool(direct)),
                       int(bool(shared_weights)), float(k_small))
        h = ctypes.c_void_p()
        st = self.lib.rr_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise RRError(st, self.lib.rr_last_error(None).decode())
        self._h = h
        self.dtype = torch.float64 if precision == "fp64" else torch.float32

    # -- plumbing -------------------------------------------------------------
    def _check(self, st: int):
        if st != 0:
            raise RRError(st, self.lib.rr_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.lib.rr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nparam(self) -> int:
        return int(self.lib.rr_nparam(self._h))

    @property
    def launch_count(self) -> int:
        return int(self.lib.rr_launch_count(self._h))

    def workspace_bytes(self, npv: int, npt: int, grad: bool = False) -> int:
        return int(self.lib.rr_workspace_bytes(self._h, npv, npt, int(grad)))

    def workspace(self, npv: int, npt: int, grad: bool = False) -> torch.Tensor:
        return torch.empty(max(self.workspace_bytes(npv, npt, grad), 256), dtype=torch.uint8,
                           device=self.device)

    # -- set-up ---------------------------------------------------------------
    def set_ld_profile(self, pb: int, mu: Sequence[float], intensity: Sequence[float]):
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        it = np.ascontiguousarray(intensity, dtype=np.float64)
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.rr_set_ld_profile(self._h, pb, mu.ctypes.data_as(dp), it.ctypes.data_as(dp),
                                               int(mu.size)))

    def build(self, stream=None):
        self._check(self.lib.rr_build_weights(self._h, _stream_handle(stream)))
        return self

    def read_table(self, which: str) -> np.ndarray:
        n = self.lib.rr_read_table(self._h, TABLES[which], None, 0)
        if n < 0:
            raise RRError(4, self.lib.rr_last_error(self._h).decode())
        out = np.empty(n, np.float64)
        r = self.lib.rr_read_table(self._h, TABLES[which], out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
        if r < 0:
            raise RRError(4, self.lib.rr_last_error(self._h).decode())
        return out

    def exact_flux(self, z, k, ldc=(), pb: int = 0, stream=None) -> torch.Tensor:
        """Exact flux (radial integral, no grid) at distances z and radius ratios k (float64 tensors
        or arrays; a float32 input keeps its float32 rounding)."""
        z = torch.as_tensor(z, dtype=torch.float64, device=self.device).contiguous()
        k = torch.as_tensor(k, dtype=torch.float64, device=self.device).contiguous()
        out = torch.empty_like(z)
        c = np.ascontiguousarray(np.asarray(ldc, np.float64).reshape(-1))
        cp = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if c.size else None
        self._check(self.lib.rr_exact_flux(self._h, _ptr(z), _ptr(k), int(z.numel()), cp, int(pb), _ptr(out),
                                           _stream_handle(stream)))
        return out

    def profile(self, enable: bool = True):
        """Bracket every kernel launch with CUDA events on its stream (measurement aid)."""
        self._check(self.lib.rr_profile(self._h, int(enable)))

    def profile_read(self, reset: bool = False) -> dict:
        """{kernel: (total_ms, launches)} of the launches timed so far."""
        out = {}
        for name, kind in KERNELS.items():
            ms, n = ctypes.c_double(), ctypes.c_int64()
            self._check(self.lib.rr_profile_read(self._h, kind, ctypes.byref(ms), ctypes.byref(n), 0))
            out[name] = (ms.value, n.value)
        if reset:
            self._check(self.lib.rr_profile_read(self._h, 0, None, None, 1))
        return out

    def count_samples(self, enable: bool = True):
        """Run the flux and adjoint kernels in their counting form (measurement aid)."""
        self._check(self.lib.rr_count_samples(self._h, int(enable)))

    def count_read(self, kind: str, reset: bool = False) -> dict:
        """{counter: value} of kernel kind 'flux' or 'grad' (include/rr.h RR_COUNT_*)."""
        buf = (ctypes.c_int64 * len(COUNTS))()
        self._check(self.lib.rr_count_read(self._h, KERNELS[kind], buf, int(reset)))
        return dict(zip(COUNTS, buf))

    @property
    def host_path(self) -> str:
        """How the last evaluate_host / enqueue_host call ran: 'in place', 'staged' or 'none'."""
        return {1: "in place", 2: "staged"}.get(int(self.lib.rr_host_path(self._h)), "none")

    def sync_status(self, stream=None):
        self._check(self.lib.rr_sync_status(self._h, _stream_handle(stream)))

    def selftest_wait(self, which: int, stream=None):
        """Enqueue a bounded device wait that runs out on purpose (0: mbarrier, 1: work queue);
        the next sync_status raises RR_ETIMEOUT."""
        self._check(self.lib.rr_selftest_wait(self._h, int(which), _stream_handle(stream)))

    # -- evaluation -----------------------------------------------------------
    def _inputs(self, times, params, pb_index):
        dev = self.device
        for name, t, dt in (("times", times, torch.float64), ("params", params, torch.float64)):
            if not (isinstance(t, torch.Tensor) and t.device == dev and t.dtype == dt and t.is_contiguous()):
                raise TypeError(f"{name} must be a contiguous {dt} tensor on {dev}")
        if params.dim() != 2 or params.shape[1] != self.nparam:
            raise ValueError(f"params must have shape (npv, {self.nparam})")
        if pb_index is not None and not (pb_index.device == dev and pb_index.dtype == torch.int32
                                         and pb_index.is_contiguous() and pb_index.numel() == times.numel()):
            raise TypeError("pb_index must be a contiguous int32 tensor with one entry per time")
        return times.numel(), params.shape[0]

    def prepare(self, times: torch.Tensor, params: torch.Tensor, pb_index: Optional[torch.Tensor] = None,
                supersampling=None, exptime=None, pv_status: Optional[torch.Tensor] = None,
                workspace: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Shared set-up of a batch for :meth:`evaluate` and :meth:`evaluate_grad` (rr_prepare).

        Returns the workspace that holds the prepared batch; pass it as
        ``prepared=`` to both calls, with the same inputs."""
        npt, npv = self._inputs(times, params, pb_index)
        ss = _host_array(supersampling, self.npb, np.int32, 1)
        ex = _host_array(exptime, self.npb, np.float64, 0.0)
        if workspace is None:
            workspace = self.workspace(npv, npt, True)
        st = self.lib.rr_prepare(self._h, _ptr(times), _ptr(pb_index), npt, _ptr(params), npv,
                                 ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(pv_status),
                                 _ptr(workspace), workspace.numel(), _stream_handle(stream))
        self._check(st)
        return workspace

    def evaluate(self, times: torch.Tensor, params: torch.Tensor, pb_index: Optional[torch.Tensor] = None,
                 supersampling=None, exptime=None, out: Optional[torch.Tensor] = None,
                 pv_status: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                 stream=None, prepared: Optional[torch.Tensor] = None) -> torch.Tensor:
        """flux[npv, npt] (float32 in 'mixed', float64 in 'fp64'), enqueued on the current stream.

        prepared: a workspace filled by :meth:`prepare` with the same inputs."""
        npt, npv = self._inputs(times, params, pb_index)
        ss = _host_array(supersampling, self.npb, np.int32, 1)
        ex = _host_array(exptime, self.npb, np.float64, 0.0)
        if out is None:
            out = torch.empty((npv, npt), dtype=self.dtype, device=self.device)
        fn = self.lib.rr_evaluate
        if prepared is not None:
            fn, workspace = self.lib.rr_evaluate_prepared, prepared
        elif workspace is None:
            workspace = self.workspace(npv, npt, False)
        st = fn(self._h, _ptr(times), _ptr(pb_index), npt, _ptr(params), npv,
                ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                _ptr(out), _ptr(pv_status), _ptr(workspace), workspace.numel(), _stream_handle(stream))
        self._check(st)
        return out

    def evaluate_noalloc(self, times: torch.Tensor, params: torch.Tensor, pb_index: Optional[torch.Tensor] = None,
                         supersampling=None, exptime=None, out: Optional[torch.Tensor] = None,
                         pv_status: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """As :meth:`evaluate`, with the library's fixed scratch instead of a workspace (see rr.h)."""
        npt, npv = self._inputs(times, params, pb_index)
        ss = _host_array(supersampling, self.npb, np.int32, 1)
        ex = _host_array(exptime, self.npb, np.float64, 0.0)
        if out is None:
            out = torch.empty((npv, npt), dtype=self.dtype, device=self.device)
        st = self.lib.rr_evaluate_noalloc(self._h, _ptr(times), _ptr(pb_index), npt, _ptr(params), npv,
                                          ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(out),
                                          _ptr(pv_status), _stream_handle(stream))
        self._check(st)
        return out

    def evaluate_grad(self, times: torch.Tensor, params: torch.Tensor, grad_flux: torch.Tensor,
                      pb_index: Optional[torch.Tensor] = None, supersampling=None, exptime=None,
                      out: Optional[torch.Tensor] = None, pv_status: Optional[torch.Tensor] = None,
                      workspace: Optional[torch.Tensor] = None, stream=None,
                      prepared: Optional[torch.Tensor] = None) -> torch.Tensor:
        """grad_params[npv, nparam] = sum_t grad_flux[pv, t] d flux[pv, t] / d params[pv, :].

        prepared: a workspace filled by :meth:`prepare` with the same inputs."""
        npt, npv = self._inputs(times, params, pb_index)
        if not (grad_flux.dtype == self.dtype and grad_flux.is_contiguous() and grad_flux.shape == (npv, npt)):
            raise TypeError(f"grad_flux must be a contiguous {self.dtype} tensor of shape ({npv}, {npt})")
        ss = _host_array(supersampling, self.npb, np.int32, 1)
        ex = _host_array(exptime, self.npb, np.float64, 0.0)
        if out is None:
            out = torch.empty((npv, self.nparam), dtype=torch.float64, device=self.device)
        fn = self.lib.rr_evaluate_grad
        if prepared is not None:
            fn, workspace = self.lib.rr_evaluate_grad_prepared, prepared
        elif workspace is None:
            workspace = self.workspace(npv, npt, True)
        st = fn(self._h, _ptr(times), _ptr(pb_index), npt, _ptr(params), npv,
                ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                _ptr(grad_flux), _ptr(out), _ptr(pv_status), _ptr(workspace), workspace.numel(),
                _stream_handle(stream))
        self._check(st)
        return out

    def evaluate_both(self, times: torch.Tensor, params: torch.Tensor, grad_flux: torch.Tensor,
                      prepared: torch.Tensor, pb_index: Optional[torch.Tensor] = None, supersampling=None,
                      exptime=None, out: Optional[torch.Tensor] = None, grad_out: Optional[torch.Tensor] = None,
                      pv_status: Optional[torch.Tensor] = None, stream=None):
        """(flux, grad_params) of a batch prepared by :meth:`prepare`, for a cotangent known in advance
        (rr_evaluate_both_prepared): the adjoint on a second stream of the context, beside the
        forward kernel; bitwise :meth:`evaluate` and :meth:`evaluate_grad` with ``prepared``."""
        npt, npv = self._inputs(times, params, pb_index)
        if not (grad_flux.dtype == self.dtype and grad_flux.is_contiguous() and grad_flux.shape == (npv, npt)):
            raise TypeError(f"grad_flux must be a contiguous {self.dtype} tensor of shape ({npv}, {npt})")
        ss = _host_array(supersampling, self.npb, np.int32, 1)
        ex = _host_array(exptime, self.npb, np.float64, 0.0)
        if out is None:
            out = torch.empty((npv, npt), dtype=self.dtype, device=self.device)
        if grad_out is None:
            grad_out = torch.empty((npv, self.nparam), dtype=torch.float64, device=self.device)
        st = self.lib.rr_evaluate_both_prepared(self._h, _ptr(times), _ptr(pb_index), npt, _ptr(params), npv,
                                                ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                _ptr(grad_flux), _ptr(out), _ptr(grad_out), _ptr(pv_status),
                                                _ptr(prepared), prepared.numel(), _stream_handle(stream))
        self._check(st)
        return out, grad_out

    def evaluate_host(self, times, params, pb_index=None, supersampling=None, exptime=None, grad_flux=None,
                      chunk_pvs: Optional[int] = None, out=None, grad_out=None, status_out=None):
        """Host arrays in, host arrays out: (flux, grad_params or None, pv_status) (rr_evaluate_host).

        Inputs not in pinned memory are first copied to pinned memory, and the
        kernels then read and write the pinned buffers in place over the
        host-device link (the library's staged path, chunks of pvs with copies
        overlapped on three streams, serves other host memory through the C
        ABI).  Results are bitwise those of one :meth:`evaluate` /
        :meth:`evaluate_grad` call on the whole batch.  out / grad_out /
        status_out are optional pinned CPU tensors for the results.
        """
        def pinned(x, dt):
            t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))
            t = t.to(dt).contiguous()
            return t if t.is_pinned() else t.pin_memory()

        def result(buf, shape, dt):
            if buf is None:
                return torch.empty(shape, dtype=dt, pin_memory=True)
            if not (buf.device.type == "cpu" and buf.dtype == dt and tuple(buf.shape) == shape
                    and buf.is_contiguous()):
                raise TypeError(f"result buffer must be a contiguous CPU {dt} tensor of shape {shape}")
            return buf

        t_h = pinned(times, torch.float64)
        p_h = pinned(params, torch.float64)
        pb_h = None if pb_index is None else pinned(pb_index, torch.int32)
        g_h = None if grad_flux is None else pinned(grad_flux, self.dtype)
        nparam = self.nparam
        if p_h.dim() != 2 or p_h.shape[1] != nparam:
            raise ValueError(f"params must have shape (npv, {nparam})")
        npv, npt = p_h.shape[0], t_h.numel()
        if g_h is not None and tuple(g_h.shape) != (npv, npt):
            raise ValueError(f"grad_flux must have shape ({npv}, {npt})")
        if pb_h is not None and pb_h.numel() != npt:
            raise ValueError("pb_index must have one entry per time")
        f_h = result(out, (npv, npt), self.dtype)
        go_h = result(grad_out, (npv, nparam), torch.float64) if g_h is not None else None
        st_h = result(status_out, (npv,), torch.int32)
        ss = _host_array(supersampling, self.npb, np.int32, 1)
        ex = _host_array(exptime, self.npb, np.float64, 0.0)
        with torch.cuda.device(self.device):
            st = self.lib.rr_evaluate_host(self._h, _ptr(t_h), _ptr(pb_h), npt, _ptr(p_h), npv,
                                           ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(g_h), _ptr(f_h),
                                           _ptr(go_h), _ptr(st_h), int(chunk_pvs or 0))
        self._check(st)
        return f_h, go_h, st_h

    def request_bytes(self, npv: int, npt: int, grad: bool = False) -> int:
        """Device scratch of one :meth:`enqueue_host` request (rr_request_bytes)."""
        return int(self.lib.rr_request_bytes(self._h, npv, npt, int(grad)))

    def enqueue_host(self, times, params, pb_index, supersampling, exptime, grad_flux, out, grad_out, status_out,
                     scratch: torch.Tensor, stream) -> None:
        """One request from pinned CPU tensors, enqueued on `stream` (rr_enqueue_host).

        All host tensors must be contiguous pinned CPU tensors of the model's
        types and stay untouched until the stream has passed the request."""
        npv, npt = int(params.shape[0]), int(times.numel())
        ss = _host_array(supersampling, self.npb, np.int32, 1)
        ex = _host_array(exptime, self.npb, np.float64, 0.0)
        self._check(self.lib.rr_enqueue_host(self._h, _ptr(times), _ptr(pb_index), npt, _ptr(params), npv,
                                             ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                             ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(grad_flux),
                                             _ptr(out), _ptr(grad_out), _ptr(status_out), _ptr(scratch),
                                             scratch.numel(), _stream_handle(stream)))

    def flux(self, times, params, pb_index=None, supersampling=None, exptime=None) -> torch.Tensor:
        """Differentiable light curves (gradient w.r.t. ``params`` through the adjoint kernel)."""
        return _RRFlux.apply(self, times, pb_index, params, supersampling, exptime)


class _RRFlux(torch.autograd.Function):
    @staticmethod
    def forward(ctx, model: Model, times, pb_index, params, supersampling, exptime):
        ctx.model = model
        ctx.meta = (supersampling, exptime)
        p = params.detach()
        ctx.save_for_backward(times, pb_index, p)
        # one set-up for the forward and the backward pass, when a gradient is wanted
        ctx.prepared = model.prepare(times, p, pb_index, supersampling, exptime) if params.requires_grad else None
        return model.evaluate(times, p, pb_index, supersampling, exptime, prepared=ctx.prepared)

    @staticmethod
    def backward(ctx, gflux):
        times, pb_index, params = ctx.saved_tensors
        ss, ex = ctx.meta
        g = ctx.model.evaluate_grad(times, params, gflux.contiguous().to(ctx.model.dtype), pb_index, ss, ex,
                                    prepared=ctx.prepared)
        ctx.prepared = None
        return None, None, None, g.to(params.dtype), None, None


def model_for(wl, device: int = 0) -> Model:
    """Model context for a :class:`workloads.Workload`, with profiles set and tables built."""
    m = Model(wl.ld_model, wl.npb, wl.chromatic, wl.precision, wl.grid, device, getattr(wl, "n_general", 0),
              getattr(wl, "direct", False), getattr(wl, "shared_weights", False), getattr(wl, "k_small", 0.0))
    if wl.ld_model == "tabulated":
        for pb, (mu, it) in enumerate(wl.profiles):
            m.set_ld_profile(pb, mu, it)
    return m.build()


def choose_grid(ld_model: str, k, ldc=(), target: float = 1e-6, profile=None, n_general: int = 0,
                device: int = 0) -> dict:
    """Cheapest grid (zcut, nzin, nzlimb, ng) whose flux stays within `target` of the exact
    integral for the radius ratios `k` and LD coefficients `ldc` (or the tabulated `profile`)."""
    lib = load_library()
    cfg = RRConfig(0.7, 8, 8, 20, 2, 0.005, 0.3, 1, LD_MODELS[ld_model], 0, PRECISIONS["fp64"], device,
                   int(n_general) if ld_model == "general" else 0, 1, 0, 0.0)
    ks = np.ascontiguousarray(np.atleast_1d(np.asarray(k, np.float64)))
    c = np.ascontiguousarray(np.asarray(ldc, np.float64).reshape(-1))
    dp = ctypes.POINTER(ctypes.c_double)
    if profile is not None:
        mu = np.ascontiguousarray(profile[0], np.float64)
        it = np.ascontiguousarray(profile[1], np.float64)
        mup, itp, nt = mu.ctypes.data_as(dp), it.ctypes.data_as(dp), mu.size
    else:
        mup = itp = None
        nt = 0
    err = ctypes.c_double(np.nan)
    st = lib.rr_choose_grid(ctypes.byref(cfg), ks.ctypes.data_as(dp), ks.size, c.ctypes.data_as(dp) if c.size else None,
                            mup, itp, nt, float(target), ctypes.byref(err))
    if st not in (0, 5):
        raise RRError(st, "rr_choose_grid failed")
    return {"zcut": cfg.zcut, "nzin": cfg.nzin, "nzlimb": cfg.nzlimb, "ng": cfg.ng, "max_error": err.value,
            "met": st == 0}


def to_device(wl, device: int = 0):
    """times, pb_index, params of a workload as device tensors."""
    dev = torch.device("cuda", device)
    return (torch.as_tensor(wl.times, dtype=torch.float64, device=dev),
            torch.as_tensor(wl.pb_index, dtype=torch.int32, device=dev),
            torch.as_tensor(wl.params, dtype=torch.float64, device=dev))
