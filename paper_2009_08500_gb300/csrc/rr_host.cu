// Host-buffer evaluation (rr_evaluate_host, rr_enqueue_host).
//
// In place: when every caller buffer is page-locked host memory mapped for
// the device (cudaHostAlloc, or registered memory, on a unified address
// space), the kernels read the times, parameters and cotangent and write the
// light curves, validity words and gradient where they are, over the
// host-device link (NVLink-C2C on a Grace host): no staging copies, and the
// adjoint reads only the cotangent rows of the (pv, group) items that may
// transit.  The kernels keep the bulk asynchronous copy engine to device
// memory and reach host memory with plain loads and stores.
//
// Staged (any other host memory): the batch is cut into chunks of
// parameter vectors; chunk c's inputs are copied to the device on one stream
// while chunk c-1 is evaluated on a second and chunk c-2's results are copied
// back on a third, with three device slots per array, so both copy
// directions and the kernels overlap.  Each chunk goes through the public
// device entry points (one shared set-up when the adjoint is wanted), so the
// results are those of one device call on the whole batch: a pv's flux and
// gradient do not depend on the other pvs of the launch.
#include <algorithm>
#include <cstring>

#include "rr_internal.h"

using namespace rr;

namespace {

constexpr int kSlots = 3;

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

rr_status pipe_fail(rr_ctx* c, cudaError_t e, const char* what) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return RR_ECUDA;
}

cudaError_t ensure_pipe(rr_ctx* c, size_t bytes) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        if (!c->pipe.s[i]) e = cudaStreamCreateWithFlags(&c->pipe.s[i], cudaStreamNonBlocking);
    for (int b = 0; b < kSlots && e == cudaSuccess; ++b)
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            if (!c->pipe.ev[b][k]) e = cudaEventCreateWithFlags(&c->pipe.ev[b][k], cudaEventDisableTiming);
    if (e != cudaSuccess || c->pipe.bytes >= bytes) return e;
    // the previous call finished (it synchronised before returning): the old buffer is idle
    if (c->pipe.buf) cudaFree(c->pipe.buf);
    c->pipe.buf = nullptr;
    c->pipe.bytes = 0;
    if ((e = cudaMalloc(&c->pipe.buf, bytes)) == cudaSuccess) c->pipe.bytes = bytes;
    return e;
}

}  // namespace

namespace rr {
const void* mapped_host(const void* p, size_t bytes) {
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a, b;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
        cudaPointerGetAttributes(&b, (const char*)p + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if ((const char*)b.devicePointer - (const char*)a.devicePointer != (ptrdiff_t)(bytes - 1)) return nullptr;
    return a.devicePointer;
}
}  // namespace rr

namespace {

}  // namespace

namespace rr {
InPlace map_in_place(const rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt,
                     const double* params, int32_t npv, const void* grad_flux, void* flux, double* grad_params,
                     int32_t* pv_status) {
    InPlace m;
    if (npt <= 0 || npv <= 0) return m;
    const size_t es = c->cfg.precision == RR_PREC_FP64 ? sizeof(double) : sizeof(float);
    const size_t np = (size_t)c->nparam, pts = (size_t)npv * npt;
    if (!(m.t = (const double*)mapped_host(times, (size_t)npt * 8))) return m;
    if (pb_index && !(m.pb = (const int32_t*)mapped_host(pb_index, (size_t)npt * 4))) return m;
    if (!(m.p = (const double*)mapped_host(params, (size_t)npv * np * 8))) return m;
    if (!(m.f = (void*)mapped_host(flux, pts * es))) return m;
    if (pv_status && !(m.st = (int32_t*)mapped_host(pv_status, (size_t)npv * 4))) return m;
    if (grad_flux) {
        if (!(m.g = mapped_host(grad_flux, pts * es))) return m;
        if (!(m.go = (double*)mapped_host(grad_params, (size_t)npv * np * 8))) return m;
    }
    m.ok = true;
    return m;
}

// One evaluation (and adjoint) on the mapped buffers, enqueued on s.
rr_status run_in_place(rr_ctx* c, const InPlace& m, int32_t npt, int32_t npv, const int32_t* ss,
                       const double* exptime, void* ws, size_t ws_bytes, cudaStream_t s, bool overlap) {
    if (!m.g) return rr_evaluate(c, m.t, m.pb, npt, m.p, npv, ss, exptime, m.f, m.st, ws, ws_bytes, s);
    rr_status st = rr_prepare(c, m.t, m.pb, npt, m.p, npv, ss, exptime, m.st, ws, ws_bytes, s);
    if (st == RR_OK && overlap)
        return rr_evaluate_both_prepared(c, m.t, m.pb, npt, m.p, npv, ss, exptime, m.g, m.f, m.go, m.st, ws, ws_bytes,
                                         s);
    if (st == RR_OK) st = rr_evaluate_prepared(c, m.t, m.pb, npt, m.p, npv, ss, exptime, m.f, m.st, ws, ws_bytes, s);
    if (st == RR_OK)
        st = rr_evaluate_grad_prepared(c, m.t, m.pb, npt, m.p, npv, ss, exptime, m.g, m.go, m.st, ws, ws_bytes, s);
    return st;
}

void release_host_pipe(rr_ctx* c) {
    for (int i = 0; i < 3; ++i)
        if (c->pipe.s[i]) cudaStreamDestroy(c->pipe.s[i]);
    for (int b = 0; b < kSlots; ++b)
        for (int k = 0; k < 4; ++k)
            if (c->pipe.ev[b][k]) cudaEventDestroy(c->pipe.ev[b][k]);
    if (c->pipe.buf) cudaFree(c->pipe.buf);
    c->pipe = rr_ctx::HostPipe{};
}
}  // namespace rr

extern "C" rr_status rr_evaluate_host(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt,
                                      const double* params, int32_t npv, const int32_t* ss, const double* exptime,
                                      const void* grad_flux, void* flux, double* grad_params, int32_t* pv_status,
                                      int32_t chunk_pvs) {
    NvtxRange nvtx_range("rr_evaluate_host");
    if (!c) return RR_EINVAL;
    if (npt < 0 || npv < 0 || chunk_pvs < 0) {
        c->err = "npt, npv and chunk_pvs must be >= 0";
        return RR_EINVAL;
    }
    if (npv == 0) return RR_OK;
    const bool grad = grad_flux != nullptr;
    if (!params || (npt > 0 && (!times || !flux)) || (grad && !grad_params) || (c->cfg.npb > 1 && npt > 0 && !pb_index)) {
        c->err = "rr_evaluate_host: a required host array is null";
        return RR_EINVAL;
    }
    const bool f64 = c->cfg.precision == RR_PREC_FP64;
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    const int np = c->nparam;
    {
        cudaError_t e = cudaSetDevice(c->cfg.device);
        if (e != cudaSuccess) return pipe_fail(c, e, "rr_evaluate_host set-up");
        const InPlace m = map_in_place(c, times, pb_index, npt, params, npv, grad_flux, flux, grad_params, pv_status);
        c->host_path = m.ok ? RR_HOST_IN_PLACE : RR_HOST_STAGED;
        if (m.ok) {
            const size_t wsb = up256(rr_workspace_bytes(c, npv, npt, grad ? 1 : 0));
            if ((e = ensure_pipe(c, wsb)) != cudaSuccess) return pipe_fail(c, e, "rr_evaluate_host set-up");
            cudaStream_t s = c->pipe.s[1];
            const rr_status st = run_in_place(c, m, npt, npv, ss, exptime, c->pipe.buf, wsb, s, true);
            e = cudaStreamSynchronize(s);
            if (st != RR_OK) return st;
            if (e != cudaSuccess) return pipe_fail(c, e, "rr_evaluate_host");
            return rr_sync_status(c, s);
        }
    }
    // default: 8 chunks, each large enough to fill the GPU on its own (small chunks
    // leave the kernels short of parallelism and pay the per-chunk launches)
    const int cp = chunk_pvs > 0 ? std::min(chunk_pvs, npv) : std::max(std::min(512, npv), (npv + 7) / 8);
    const size_t ws_bytes = up256(rr_workspace_bytes(c, cp, npt, grad ? 1 : 0));
    // device layout: times, passbands, then per slot params | flux | status | workspace | [gbar | grad]
    const size_t o_t = 0, o_pb = up256((size_t)npt * 8);
    const size_t o_slot = o_pb + up256((size_t)npt * 4);
    const size_t s_p = up256((size_t)cp * np * 8), s_f = up256((size_t)cp * npt * es), s_st = up256((size_t)cp * 4);
    const size_t s_g = grad ? s_f : 0, s_go = grad ? s_p : 0;
    const size_t slot = s_p + s_f + s_st + ws_bytes + s_g + s_go;
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e == cudaSuccess) e = ensure_pipe(c, o_slot + kSlots * slot);
    if (e != cudaSuccess) return pipe_fail(c, e, "rr_evaluate_host set-up");
    char* base = (char*)c->pipe.buf;
    cudaStream_t s_in = c->pipe.s[0], s_run = c->pipe.s[1], s_out = c->pipe.s[2];
    double* d_t = (double*)(base + o_t);
    int32_t* d_pb = pb_index ? (int32_t*)(base + o_pb) : nullptr;
    if (npt > 0) e = cudaMemcpyAsync(d_t, times, (size_t)npt * 8, cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess && d_pb && npt > 0)
        e = cudaMemcpyAsync(d_pb, pb_index, (size_t)npt * 4, cudaMemcpyHostToDevice, s_in);
    rr_status st = e == cudaSuccess ? RR_OK : pipe_fail(c, e, "rr_evaluate_host copy of the times");
    const int nchunks = (npv + cp - 1) / cp;
    for (int k = 0; k < nchunks && st == RR_OK; ++k) {
        e = cudaSuccess;
        const int c0 = k * cp, n = std::min(cp, npv - c0), b = k % kSlots;
        char* sb = base + o_slot + (size_t)b * slot;
        double* d_p = (double*)sb;
        char* d_f = sb + s_p;
        int32_t* d_st = (int32_t*)(sb + s_p + s_f);
        void* d_ws = sb + s_p + s_f + s_st;
        char* d_g = sb + s_p + s_f + s_st + ws_bytes;
        double* d_go = (double*)(d_g + s_g);
        cudaEvent_t* ev = c->pipe.ev[b];
        const size_t rowb = (size_t)npt * es;
        if (k >= kSlots) e = cudaStreamWaitEvent(s_in, ev[2], 0);   // slot free: its results are copied out
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_p, params + (size_t)c0 * np, (size_t)n * np * 8, cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess && grad && npt > 0)
            e = cudaMemcpyAsync(d_g, (const char*)grad_flux + (size_t)c0 * rowb, (size_t)n * rowb,
                                cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_run, ev[0], 0);
        if (e != cudaSuccess) {
            st = pipe_fail(c, e, "rr_evaluate_host copy-in");
            break;
        }
        // the light curves go out as soon as the forward kernel is done (with a
        // gradient, their copy runs beside the adjoint, which does not write them)
        bool flux_out = false;
        if (grad) {
            st = rr_prepare(c, d_t, d_pb, npt, d_p, n, ss, exptime, d_st, d_ws, ws_bytes, s_run);
            if (st == RR_OK)
                st = rr_evaluate_prepared(c, d_t, d_pb, npt, d_p, n, ss, exptime, d_f, d_st, d_ws, ws_bytes, s_run);
            if (st == RR_OK && npt > 0) {
                e = cudaEventRecord(ev[3], s_run);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev[3], 0);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync((char*)flux + (size_t)c0 * rowb, d_f, (size_t)n * rowb,
                                        cudaMemcpyDeviceToHost, s_out);
                if (e != cudaSuccess) {
                    st = pipe_fail(c, e, "rr_evaluate_host copy-out");
                    break;
                }
                flux_out = true;
            }
            if (st == RR_OK)
                st = rr_evaluate_grad_prepared(c, d_t, d_pb, npt, d_p, n, ss, exptime, d_g, d_go, d_st, d_ws, ws_bytes,
                                               s_run);
        } else {
            st = rr_evaluate(c, d_t, d_pb, npt, d_p, n, ss, exptime, d_f, d_st, d_ws, ws_bytes, s_run);
        }
        if (st != RR_OK) break;
        e = cudaEventRecord(ev[1], s_run);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev[1], 0);
        if (e == cudaSuccess && npt > 0 && !flux_out)
            e = cudaMemcpyAsync((char*)flux + (size_t)c0 * rowb, d_f, (size_t)n * rowb, cudaMemcpyDeviceToHost, s_out);
        if (e == cudaSuccess && pv_status)
            e = cudaMemcpyAsync(pv_status + c0, d_st, (size_t)n * 4, cudaMemcpyDeviceToHost, s_out);
        if (e == cudaSuccess && grad)
            e = cudaMemcpyAsync(grad_params + (size_t)c0 * np, d_go, (size_t)n * np * 8, cudaMemcpyDeviceToHost,
                                s_out);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], s_out);
        if (e != cudaSuccess) {
            st = pipe_fail(c, e, "rr_evaluate_host copy-out");
            break;
        }
    }
    // wait for everything enqueued (also after an error, so that the slots are idle)
    cudaError_t e1 = cudaStreamSynchronize(s_in), e2 = cudaStreamSynchronize(s_run), e3 = cudaStreamSynchronize(s_out);
    if (st != RR_OK) return st;
    e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
    if (e != cudaSuccess) return pipe_fail(c, e, "rr_evaluate_host");
    return rr_sync_status(c, s_out);
}

// ---------------------------------------------------------------------------
// One request from host buffers, enqueued on a stream (serving): layout of the
// caller's device scratch, then copy-in, evaluation (and adjoint), copy-out.
namespace {

struct ReqLayout {
    size_t t, pb, p, f, st, ws, g, go, total, ws_bytes;
};

ReqLayout req_layout(const rr_ctx* c, int npv, int npt, bool grad) {
    const size_t es = c->cfg.precision == RR_PREC_FP64 ? sizeof(double) : sizeof(float);
    ReqLayout L;
    L.t = 0;
    L.pb = up256((size_t)npt * 8);
    L.p = L.pb + up256((size_t)npt * 4);
    L.f = L.p + up256((size_t)npv * c->nparam * 8);
    L.st = L.f + up256((size_t)npv * npt * es);
    L.ws = L.st + up256((size_t)npv * 4);
    L.ws_bytes = up256(rr_workspace_bytes(c, npv, npt, grad ? 1 : 0));
    L.g = L.ws + L.ws_bytes;
    L.go = L.g + (grad ? up256((size_t)npv * npt * es) : 0);
    L.total = L.go + (grad ? up256((size_t)npv * c->nparam * 8) : 0);
    return L;
}

}  // namespace

extern "C" size_t rr_request_bytes(const rr_ctx* c, int32_t npv, int32_t npt, int32_t with_grad) {
    if (!c || npv < 0 || npt < 0) return 0;
    return req_layout(c, npv, npt, with_grad != 0).total;
}

extern "C" int32_t rr_host_path(const rr_ctx* c) { return c ? c->host_path : 0; }

namespace rr {
size_t request_bytes_in_place(const rr_ctx* c, int npv, int npt, bool grad) {
    return npv > 0 && npt > 0 ? req_layout(c, npv, npt, grad).ws_bytes : req_layout(c, npv, npt, grad).total;
}
}  // namespace rr

extern "C" rr_status rr_enqueue_host(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt,
                                     const double* params, int32_t npv, const int32_t* ss, const double* exptime,
                                     const void* grad_flux, void* flux, double* grad_params, int32_t* pv_status,
                                     void* scratch, size_t scratch_bytes, void* stream) {
    NvtxRange nvtx_range("rr_enqueue_host");
    if (!c) return RR_EINVAL;
    if (npt < 0 || npv < 0) {
        c->err = "npt and npv must be >= 0";
        return RR_EINVAL;
    }
    if (npv == 0) return RR_OK;
    const bool grad = grad_flux != nullptr;
    if (!params || (npt > 0 && (!times || !flux)) || (grad && !grad_params) || (c->cfg.npb > 1 && npt > 0 && !pb_index)) {
        c->err = "rr_enqueue_host: a required host array is null";
        return RR_EINVAL;
    }
    const ReqLayout L = req_layout(c, npv, npt, grad);
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e != cudaSuccess) return pipe_fail(c, e, "rr_enqueue_host");
    const InPlace m = map_in_place(c, times, pb_index, npt, params, npv, grad_flux, flux, grad_params, pv_status);
    // in place, the scratch holds the workspace only
    if (!scratch || scratch_bytes < (m.ok ? L.ws_bytes : L.total) || ((uintptr_t)scratch & 255u)) {
        c->err = "rr_enqueue_host: scratch too small or not 256-byte aligned";
        return RR_EINVAL;
    }
    c->host_path = m.ok ? RR_HOST_IN_PLACE : RR_HOST_STAGED;
    if (m.ok) return run_in_place(c, m, npt, npv, ss, exptime, scratch, L.ws_bytes, (cudaStream_t)stream, false);
    const size_t es = c->cfg.precision == RR_PREC_FP64 ? sizeof(double) : sizeof(float);
    const int np = c->nparam;
    char* b = (char*)scratch;
    double* d_t = (double*)(b + L.t);
    int32_t* d_pb = pb_index ? (int32_t*)(b + L.pb) : nullptr;
    double* d_p = (double*)(b + L.p);
    void* d_f = b + L.f;
    int32_t* d_st = (int32_t*)(b + L.st);
    void* d_ws = b + L.ws;
    void* d_g = b + L.g;
    double* d_go = (double*)(b + L.go);
    cudaStream_t s = (cudaStream_t)stream;
    if (npt > 0) e = cudaMemcpyAsync(d_t, times, (size_t)npt * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && d_pb && npt > 0) e = cudaMemcpyAsync(d_pb, pb_index, (size_t)npt * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_p, params, (size_t)npv * np * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && grad && npt > 0)
        e = cudaMemcpyAsync(d_g, grad_flux, (size_t)npv * npt * es, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return pipe_fail(c, e, "rr_enqueue_host copy-in");
    rr_status st;
    if (grad) {
        st = rr_prepare(c, d_t, d_pb, npt, d_p, npv, ss, exptime, d_st, d_ws, L.ws_bytes, s);
        if (st == RR_OK) st = rr_evaluate_prepared(c, d_t, d_pb, npt, d_p, npv, ss, exptime, d_f, d_st, d_ws, L.ws_bytes, s);
        if (st == RR_OK)
            st = rr_evaluate_grad_prepared(c, d_t, d_pb, npt, d_p, npv, ss, exptime, d_g, d_go, d_st, d_ws, L.ws_bytes, s);
    } else {
        st = rr_evaluate(c, d_t, d_pb, npt, d_p, npv, ss, exptime, d_f, d_st, d_ws, L.ws_bytes, s);
    }
    if (st != RR_OK) return st;
    if (npt > 0) e = cudaMemcpyAsync(flux, d_f, (size_t)npv * npt * es, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && pv_status) e = cudaMemcpyAsync(pv_status, d_st, (size_t)npv * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad_params, d_go, (size_t)npv * np * 8, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return pipe_fail(c, e, "rr_enqueue_host copy-out");
    return RR_OK;
}
