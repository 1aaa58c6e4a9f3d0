// Host implementation of the C ABI declared in include/rr.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "rr_internal.h"

using namespace rr;

namespace {

thread_local std::string g_create_err;

rr_status fail(rr_ctx* c, rr_status st, const std::string& msg) {
    if (c) c->err = msg; else g_create_err = msg;
    return st;
}

rr_status cuda_fail(rr_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, RR_ECUDA, m);
}

int ncoef(int model, int n_general) {
    switch (model) {
        case RR_LD_QUADRATIC:
        case RR_LD_QUADRATIC_TRI:
        case RR_LD_LOGARITHMIC:
        case RR_LD_EXPONENTIAL:
        case RR_LD_POWER2:
        case RR_LD_POWER2_PM: return 2;
        case RR_LD_NONLINEAR: return 4;
        case RR_LD_LINEAR: return 1;
        case RR_LD_GENERAL: return n_general;
        default: return 0;
    }
}

// Radial grid of Sect. 3.1.1: constant dz on [0, zcut] (nzin annuli),
// constant dmu from mu(zcut) to 0 (nzlimb annuli); zm = bin midpoints,
// mu = sqrt(1 - zm^2).
void make_grid(double zcut, int nzin, int nzlimb, std::vector<double>& ze, std::vector<double>& zm,
               std::vector<double>& mu) {
    const int nz = nzin + nzlimb;
    ze.assign(nz + 1, 0.0);
    for (int j = 0; j <= nzin; ++j) ze[j] = j * zcut / nzin;
    const double mucut = std::sqrt(1.0 - zcut * zcut);
    for (int m = 1; m <= nzlimb; ++m) {
        const double mm = mucut * (1.0 - (double)m / nzlimb);
        ze[nzin + m] = std::sqrt(1.0 - mm * mm);
    }
    zm.resize(nz);
    mu.resize(nz);
    for (int j = 0; j < nz; ++j) {
        zm[j] = 0.5 * (ze[j] + ze[j + 1]);
        mu[j] = std::sqrt(1.0 - zm[j] * zm[j]);
    }
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
}

void free_all(rr_ctx* c) {
    release_host_pipe(c);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    c->aux = nullptr;
    c->ev_fork = c->ev_join = nullptr;
    for (auto& t : c->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    c->timed.clear();
    c->ev_pool.clear();
    cudaFree(c->d_ze);
    cudaFree(c->d_mu);
    cudaFree(c->d_w);
    cudaFree(c->d_basis);
    cudaFree(c->d_istar);
    cudaFree(c->d_T64);
    cudaFree(c->d_T32);
    cudaFree(c->d_DT32);
    cudaFree(c->d_tab);
    cudaFree(c->d_tab_off);
    cudaFree(c->d_err);
    cudaFree(c->d_svtab);
    cudaFree(c->d_counts);
    cudaFree(c->d_zef);
    cudaFree(c->d_basisf);
    cudaFree(c->d_pre64);
    cudaFree(c->d_pref);
    cudaFree(c->d_gl);
    cudaFree(c->d_lnmu);
    cudaFree(c->d_lnmuf);
}

// Per-kernel timing: when enabled, every launch is bracketed by two CUDA
// events recorded on the launching stream; rr_profile_read resolves them.
cudaEvent_t take_event(rr_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

template <typename F>
cudaError_t timed(rr_ctx* c, int kind, cudaStream_t s, F&& launch) {
    if (!c->profiling) return launch();
    cudaEvent_t a = take_event(c), b = take_event(c);
    cudaEventRecord(a, s);
    cudaError_t e = launch();
    cudaEventRecord(b, s);
    c->timed.push_back({kind, a, b});
    return e;
}

void resolve_timing(rr_ctx* c) {
    for (auto& t : c->timed) {
        float ms = 0.f;
        cudaEventSynchronize(t.b);
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            c->prof_ms[t.kind] += ms;
            c->prof_n[t.kind] += 1;
        }
        c->ev_pool.push_back(t.a);
        c->ev_pool.push_back(t.b);
    }
    c->timed.clear();
}

// Checks shared by rr_evaluate and rr_evaluate_grad; fills the passband constants.
rr_status check_eval(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt, const double* params,
                     int32_t npv, const int32_t* ss, const double* exptime, const void* out, void* ws,
                     size_t ws_bytes, bool grad, PbParams& pbp) {
    if (!c) return fail(nullptr, RR_EINVAL, "null context");
    if (!c->tables_built) return fail(c, RR_ESTATE, "rr_build_weights has not been called since the last change");
    if (npt < 0 || npv < 0) return fail(c, RR_EINVAL, "npt and npv must be >= 0");
    if (!ss || !exptime) return fail(c, RR_EINVAL, "supersampling and exptime (host arrays) are required");
    std::memset(&pbp, 0, sizeof(pbp));
    pbp.npb = c->cfg.npb;
    for (int pb = 0; pb < c->cfg.npb; ++pb) {
        if (ss[pb] < 1 || ss[pb] > 1024) return fail(c, RR_EINVAL, "supersampling must be in [1, 1024]");
        if (!std::isfinite(exptime[pb]) || exptime[pb] < 0.0)
            return fail(c, RR_EINVAL, "exptime must be finite and >= 0");
        pbp.ss[pb] = ss[pb];
        pbp.exptime[pb] = ss[pb] > 1 ? exptime[pb] : 0.0;
        const double step = ss[pb] > 1 ? exptime[pb] / ss[pb] : 0.0;
        const double first = ss[pb] > 1 ? -0.5 * exptime[pb] + 0.5 * step : 0.0;
        pbp.step[pb] = (float)step;
        pbp.first[pb] = (float)first;
        pbp.step_lo[pb] = (float)(step - (double)pbp.step[pb]);
        pbp.first_lo[pb] = (float)(first - (double)pbp.first[pb]);
        pbp.inv_ss[pb] = (float)(1.0 / ss[pb]);
    }
    if (npt == 0 || npv == 0) return RR_OK;
    if (!times || !params || !out) return fail(c, RR_EINVAL, "times, params and the output must be non-null");
    if (c->cfg.npb > 1 && !pb_index) return fail(c, RR_EINVAL, "pb_index is required when npb > 1");
    const size_t need = rr_workspace_bytes(c, npv, npt, grad ? 1 : 0);
    if (!ws || ws_bytes < need) {
        char b[160];
        std::snprintf(b, sizeof b, "workspace too small: %zu bytes given, %zu needed", ws ? ws_bytes : (size_t)0, need);
        return fail(c, RR_EINVAL, b);
    }
    if (((uintptr_t)ws & 255u) != 0) return fail(c, RR_EINVAL, "workspace must be 256-byte aligned");
    if (((uintptr_t)times & 7u) != 0 || ((uintptr_t)params & 7u) != 0)
        return fail(c, RR_EINVAL, "times and params must be 8-byte aligned");
    return RR_OK;
}

}  // namespace

namespace rr {
size_t records_bytes(const rr_ctx* c, int npv, bool grad) {
    const RecLayout L = c->cfg.precision == RR_PREC_FP64 ? make_layout<double>(c->cfg.npb, c->cfg.ng, c->nldc, grad)
                                                         : make_layout<float>(c->cfg.npb, c->cfg.ng, c->nldc, grad);
    return rows_offset(L, npv) + (size_t)npv * L.rows_bytes;
}

WsLayout ws_layout(const rr_ctx* c, int npv, int npt, bool grad) {
    WsLayout w;
    w.rec = 0;
    size_t off = align256(records_bytes(c, npv, grad));
    w.dir = off;
    if (c->cfg.direct) off += align256(direct_bytes(c, npv, grad));
    w.pts_dt = off;
    if (c->cfg.precision == RR_PREC_MIXED) off += align256((size_t)npt * 8);
    w.pts_pb = off;
    if (c->cfg.precision == RR_PREC_MIXED) off += align256((size_t)npt * 4);
    w.pts_grp = off;
    if (c->cfg.precision == RR_PREC_MIXED) off += align256((size_t)((npt + kWarpPts - 1) / kWarpPts) * sizeof(GroupInfo));
    w.pts_ord = off;
    if (c->cfg.precision == RR_PREC_MIXED && c->cfg.npb > 1)
        off += align256((size_t)time_chunks(npt, groups_per_cta(npt)) * sizeof(int));
    w.part = off;
    if (grad) off += align256(partials_bytes(c, npv, npt));
    w.total = off > 0 ? off : 256;
    return w;
}
}  // namespace rr

namespace {

// Per-pv set-up and per-time preparation (the first two kernels of every evaluation).
// The direct model's per-call projections (before the set-up kernel that reads them).
cudaError_t run_direct(rr_ctx* c, const double* params, int npv, bool grad, void* ws, cudaStream_t s) {
    if (!c->cfg.direct) return cudaSuccess;
    const WsLayout W = ws_layout(c, npv, 0, grad);
    const DirectTables D = direct_view(c, (char*)ws + W.dir, npv, grad);
    return timed(c, RR_KERNEL_DIRECT, s, [&] { return launch_direct_tables(c, params, npv, grad, D, s); });
}

cudaError_t run_setup(rr_ctx* c, const double* times, const int32_t* pb_index, int npt, const double* params,
                      int npv, const PbParams& pbp, bool grad, int32_t* pv_status, void* ws, cudaStream_t s) {
    cudaError_t e = run_direct(c, params, npv, grad, ws, s);
    if (e != cudaSuccess) return e;
    // the per-pv set-up and (mixed form) the per-time preparation in one launch (measured: the
    // preparation then costs nothing on the population workload; with 8 passbands the set-up
    // grows by 1.5 us and the step saves 4 us against a launch of its own); with several
    // passbands the chunk ordering follows
    const WsLayout W = ws_layout(c, npv, npt, grad);
    char* wb = (char*)ws;
    e = timed(c, RR_KERNEL_PV_SETUP, s, [&] {
        return launch_pv_setup(c, params, npv, pbp, grad, ws, pv_status, s, times, pb_index, npt,
                               wb + W.pts_dt, wb + W.pts_pb, wb + W.pts_grp);
    });
    if (e != cudaSuccess || c->cfg.npb == 1 || c->cfg.precision != RR_PREC_MIXED || npt == 0) return e;
    return timed(c, RR_KERNEL_POINTS, s,
                 [&] { return launch_chunk_order(c, npt, wb + W.pts_grp, wb + W.pts_ord, s); });
}

// Validity words only (npt == 0 with a pv_status array): the set-up kernel alone.
rr_status status_only(rr_ctx* c, const double* params, int npv, const PbParams& pbp, bool grad,
                      int32_t* pv_status, void* ws, size_t ws_bytes, cudaStream_t s, const char* what) {
    if (!params) return fail(c, RR_EINVAL, "params must be non-null");
    if (!ws || ws_bytes < rr_workspace_bytes(c, npv, 0, grad ? 1 : 0) || ((uintptr_t)ws & 255u))
        return fail(c, RR_EINVAL, "workspace too small or misaligned");
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e == cudaSuccess) e = run_direct(c, params, npv, grad, ws, s);
    if (e == cudaSuccess)
        e = timed(c, RR_KERNEL_PV_SETUP, s, [&] { return launch_pv_setup(c, params, npv, pbp, grad, ws, pv_status, s); });
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return RR_OK;
}

rr_status evaluate_impl(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt, const double* params,
                        int32_t npv, const int32_t* ss, const double* exptime, void* flux, int32_t* pv_status,
                        void* ws, size_t ws_bytes, bool prepared, void* stream) {
    PbParams pbp;
    rr_status st = check_eval(c, times, pb_index, npt, params, npv, ss, exptime, flux, ws, ws_bytes, prepared, pbp);
    cudaStream_t s = (cudaStream_t)stream;
    if (st != RR_OK || npt == 0 || npv == 0) {
        // nothing to evaluate, but report the validity of every pv
        if (st == RR_OK && npv > 0 && pv_status && npt == 0 && !prepared)
            return status_only(c, params, npv, pbp, false, pv_status, ws, ws_bytes, s, "rr_evaluate");
        return st;
    }
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    if (!prepared && (e = run_setup(c, times, pb_index, npt, params, npv, pbp, false, pv_status, ws, s)) != cudaSuccess)
        return cuda_fail(c, e, "set-up kernels");
    const WsLayout W = ws_layout(c, npv, npt, prepared);
    char* wb = (char*)ws;
    if ((e = timed(c, RR_KERNEL_FLUX, s, [&] {
             return launch_flux(c, times, pb_index, wb + W.pts_dt, wb + W.pts_pb, wb + W.pts_grp,
                                c->cfg.npb > 1 ? wb + W.pts_ord : nullptr, npt, npv, pbp, ws, flux, pv_status,
                                prepared, s);
         })) != cudaSuccess)
        return cuda_fail(c, e, "flux kernel");
    return RR_OK;
}

rr_status evaluate_grad_impl(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt,
                             const double* params, int32_t npv, const int32_t* ss, const double* exptime,
                             const void* grad_flux, double* grad_params, int32_t* pv_status, void* ws,
                             size_t ws_bytes, bool prepared, void* stream) {
    PbParams pbp;
    rr_status st = check_eval(c, times, pb_index, npt, params, npv, ss, exptime, grad_params, ws, ws_bytes, true, pbp);
    if (st != RR_OK) return st;
    if (npv == 0) return RR_OK;
    if (npt > 0 && !grad_flux) return fail(c, RR_EINVAL, "grad_flux must be non-null");
    if (!grad_params || !params) return fail(c, RR_EINVAL, "params and grad_params must be non-null");
    if (c->nparam > 64) return fail(c, RR_EINVAL, "the adjoint supports at most 64 parameters per vector");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    if (npt == 0) {
        if ((e = cudaMemsetAsync(grad_params, 0, (size_t)npv * c->nparam * sizeof(double), s)) != cudaSuccess)
            return cuda_fail(c, e, "rr_evaluate_grad");
        return RR_OK;
    }
    if (!prepared && (e = run_setup(c, times, pb_index, npt, params, npv, pbp, true, pv_status, ws, s)) != cudaSuccess)
        return cuda_fail(c, e, "set-up kernels");
    const WsLayout W = ws_layout(c, npv, npt, true);
    char* wb = (char*)ws;
    void* partials = wb + W.part;
    if ((e = timed(c, RR_KERNEL_GRAD, s, [&] {
             return launch_grad(c, times, pb_index, wb + W.pts_dt, wb + W.pts_pb, wb + W.pts_grp,
                                c->cfg.npb > 1 ? wb + W.pts_ord : nullptr, npt, npv, pbp, ws, grad_flux, partials,
                                pv_status, s);
         })) != cudaSuccess)
        return cuda_fail(c, e, "adjoint kernel");
    if ((e = timed(c, RR_KERNEL_GRAD_REDUCE, s, [&] {
             return launch_grad_reduce(c, npt, params, npv, ws, partials, grad_params, s);
         })) != cudaSuccess)
        return cuda_fail(c, e, "adjoint reduction kernel");
    return RR_OK;
}

}  // namespace

extern "C" {

rr_status rr_create(const rr_config* cfg, rr_ctx** out) {
    if (!out) return fail(nullptr, RR_EINVAL, "out is null");
    *out = nullptr;
    if (!cfg) return fail(nullptr, RR_EINVAL, "cfg is null");
    const rr_config& k = *cfg;
    if (!(k.zcut > 0.0 && k.zcut < 1.0)) return fail(nullptr, RR_EINVAL, "zcut must be in (0, 1)");
    if (k.nzin < 1 || k.nzlimb < 1 || k.nzin + k.nzlimb > kMaxNz)
        return fail(nullptr, RR_EINVAL, "need nzin >= 1, nzlimb >= 1, nzin + nzlimb <= 4096");
    if (k.ng < 2 || k.ng > 4096) return fail(nullptr, RR_EINVAL, "ng must be in [2, 4096]");
    if (k.direct != 0 && k.direct != 1) return fail(nullptr, RR_EINVAL, "direct must be 0 or 1");
    if (k.shared_weights != 0 && k.shared_weights != 1)
        return fail(nullptr, RR_EINVAL, "shared_weights must be 0 or 1");
    if (!(k.k_small >= 0.0 && k.k_small < 1.0)) return fail(nullptr, RR_EINVAL, "k_small must be in [0, 1)");
    if (!k.direct) {
        if (k.nk < 2 || k.nk > 4096) return fail(nullptr, RR_EINVAL, "nk must be in [2, 4096]");
        if (!(k.k0 > 0.0 && k.k0 < k.k1 && k.k1 < 1.0)) return fail(nullptr, RR_EINVAL, "need 0 < k0 < k1 < 1");
    }
    if (k.npb < 1 || k.npb > RR_MAX_PB) return fail(nullptr, RR_EINVAL, "npb must be in [1, 32]");
    if (k.ld_model < RR_LD_UNIFORM || k.ld_model > RR_LD_POWER2_PM) return fail(nullptr, RR_EINVAL, "unknown ld_model");
    if ((k.ld_model == RR_LD_POWER2 || k.ld_model == RR_LD_POWER2_PM) && (k.direct != 1 || k.k_small != 0.0))
        return fail(nullptr, RR_EINVAL, "the power-2 laws need the direct model (direct = 1) and k_small = 0");
    if (k.ld_model == RR_LD_GENERAL ? (k.ncoef < 1 || k.ncoef > 4) : k.ncoef != 0)
        return fail(nullptr, RR_EINVAL, "ncoef must be 1..4 for RR_LD_GENERAL and 0 otherwise");
    if (k.precision != RR_PREC_FP64 && k.precision != RR_PREC_MIXED) return fail(nullptr, RR_EINVAL, "unknown precision");
    if (k.chromatic != 0 && k.chromatic != 1) return fail(nullptr, RR_EINVAL, "chromatic must be 0 or 1");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
    if (k.device < 0 || k.device >= ndev) return fail(nullptr, RR_EINVAL, "no such CUDA device");
    if ((e = cudaSetDevice(k.device)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");

    rr_ctx* c = new (std::nothrow) rr_ctx();
    if (!c) return fail(nullptr, RR_ENOMEM, "host allocation failed");
    c->cfg = k;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, k.device);
    c->nz = k.nzin + k.nzlimb;
    c->nldc = ncoef(k.ld_model, k.ncoef);
    const bool p2 = k.ld_model == RR_LD_POWER2 || k.ld_model == RR_LD_POWER2_PM;
    c->nbasis = k.ld_model == RR_LD_TABULATED ? k.npb : (p2 ? 1 : 1 + c->nldc);
    c->nkp = k.chromatic ? k.npb : 1;
    c->nparam = 6 + c->nkp + k.npb * c->nldc;
    c->dk = k.direct ? 1.0 : (k.k1 - k.k0) / (k.nk - 1);
    c->dg = 1.0 / (k.ng - 1);
    make_grid(k.zcut, k.nzin, k.nzlimb, c->ze, c->zm, c->mu);
    c->tab_mu.resize(k.npb);
    c->tab_I.resize(k.npb);
    // the (k, g) projections (interpolated model) or the running sums of the direct model
    const size_t nT = k.direct ? 0 : (size_t)c->nbasis * k.nk * k.ng;
    const size_t nP = k.direct ? (size_t)c->nbasis * (c->nz + 1) : 0;
    if (dalloc(&c->d_ze, c->nz + 1) || dalloc(&c->d_mu, c->nz) || dalloc(&c->d_basis, (size_t)c->nbasis * c->nz) ||
        dalloc(&c->d_istar, c->nbasis) || dalloc(&c->d_T64, nT) || dalloc(&c->d_T32, nT) || dalloc(&c->d_DT32, nT) ||
        dalloc(&c->d_tab_off, k.npb + 1) || dalloc(&c->d_err, 1) ||
        (k.precision == RR_PREC_MIXED && dalloc(&c->d_svtab, kSvTabLen)) ||
        (k.direct && (dalloc(&c->d_zef, c->nz + 1) || dalloc(&c->d_basisf, (size_t)c->nbasis * c->nz) ||
                      dalloc(&c->d_pre64, nP) || dalloc(&c->d_pref, 2 * nP))) ||
        (p2 && (dalloc(&c->d_lnmu, c->nz) || dalloc(&c->d_lnmuf, c->nz)))) {
        free_all(c);
        delete c;
        cudaGetLastError();
        return fail(nullptr, RR_ENOMEM, "device allocation failed");
    }
    if (p2) {
        std::vector<double> lm(c->nz);
        std::vector<float> lmf(c->nz);
        for (int j = 0; j < c->nz; ++j) {
            lm[j] = std::log(c->mu[j]);
            lmf[j] = (float)lm[j];
        }
        if ((e = cudaMemcpy(c->d_lnmu, lm.data(), c->nz * sizeof(double), cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(c->d_lnmuf, lmf.data(), c->nz * sizeof(float), cudaMemcpyHostToDevice))) {
            free_all(c);
            delete c;
            return cuda_fail(nullptr, e, "upload of ln mu");
        }
    }
    if (c->d_svtab) {
        // sin x0 and 1 - cos x0 = 2 sin^2(x0 / 2) in FP64 on the host, as float pairs
        std::vector<float4> tab(kSvTabLen);
        for (int j = 0; j < kSvTabLen; ++j) {
            const double x0 = (double)(j - kSvTabRes) / kSvTabRes;
            const double S = std::sin(x0), h = std::sin(0.5 * x0), V = 2.0 * h * h;
            const float Sh = (float)S, Vh = (float)V;
            tab[j] = make_float4(Sh, (float)(S - (double)Sh), Vh, (float)(V - (double)Vh));
        }
        if ((e = cudaMemcpy(c->d_svtab, tab.data(), kSvTabLen * sizeof(float4), cudaMemcpyHostToDevice))) {
            free_all(c);
            delete c;
            return cuda_fail(nullptr, e, "upload of the sine table");
        }
    }
    if ((e = cudaMemcpy(c->d_ze, c->ze.data(), (c->nz + 1) * sizeof(double), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->d_mu, c->mu.data(), c->nz * sizeof(double), cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(c->d_err, 0, sizeof(int)))) {
        free_all(c);
        delete c;
        return cuda_fail(nullptr, e, "upload of the radial grid");
    }
    *out = c;
    return RR_OK;
}

rr_status rr_destroy(rr_ctx* c) {
    if (!c) return RR_OK;
    cudaSetDevice(c->cfg.device);
    free_all(c);
    delete c;
    return RR_OK;
}

rr_status rr_set_ld_profile(rr_ctx* c, int32_t pb, const double* mu, const double* I, int32_t n) {
    if (!c) return fail(nullptr, RR_EINVAL, "null context");
    if (c->cfg.ld_model != RR_LD_TABULATED) return fail(c, RR_ESTATE, "rr_set_ld_profile needs RR_LD_TABULATED");
    if (pb < 0 || pb >= c->cfg.npb) return fail(c, RR_EINVAL, "passband index out of range");
    if (!mu || !I || n < 2) return fail(c, RR_EINVAL, "need mu, intensity and n >= 2");
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(mu[i]) || !std::isfinite(I[i])) return fail(c, RR_EINVAL, "non-finite profile value");
        if (mu[i] < 0.0 || mu[i] > 1.0) return fail(c, RR_EINVAL, "mu must lie in [0, 1]");
        if (i > 0 && !(mu[i] > mu[i - 1])) return fail(c, RR_EINVAL, "mu must be strictly increasing");
    }
    c->tab_mu[pb].assign(mu, mu + n);
    c->tab_I[pb].assign(I, I + n);
    c->tables_built = false;
    return RR_OK;
}

rr_status rr_build_weights(rr_ctx* c, void* stream) {
    NvtxRange nvtx_range("rr_build_weights");
    if (!c) return fail(nullptr, RR_EINVAL, "null context");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    if (c->cfg.ld_model == RR_LD_TABULATED) {
        std::vector<int> off(c->cfg.npb + 1, 0);
        for (int pb = 0; pb < c->cfg.npb; ++pb) {
            if (c->tab_mu[pb].empty()) return fail(c, RR_ESTATE, "a tabulated passband profile has not been set");
            off[pb + 1] = off[pb] + (int)c->tab_mu[pb].size();
        }
        std::vector<double> buf;
        buf.reserve(2 * (size_t)off.back());
        for (int pb = 0; pb < c->cfg.npb; ++pb) {
            buf.insert(buf.end(), c->tab_mu[pb].begin(), c->tab_mu[pb].end());
            buf.insert(buf.end(), c->tab_I[pb].begin(), c->tab_I[pb].end());
        }
        cudaFree(c->d_tab);
        c->d_tab = nullptr;
        if (dalloc(&c->d_tab, buf.size())) return fail(c, RR_ENOMEM, "device allocation failed");
        if ((e = cudaMemcpy(c->d_tab, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(c->d_tab_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice)))
            return cuda_fail(c, e, "upload of the tabulated profiles");
    }
    if (!c->d_w && !c->cfg.direct) {
        if (dalloc(&c->d_w, (size_t)c->cfg.nk * c->cfg.ng * c->nz)) {
            cudaGetLastError();
            return fail(c, RR_ENOMEM, "device allocation of the weight table failed");
        }
    }
    if ((e = timed(c, RR_KERNEL_LD_BASIS, s, [&] { return launch_ld_basis(c, s); })) != cudaSuccess)
        return cuda_fail(c, e, "LD profile kernel");
    if (c->cfg.direct) {
        // no (k, g) table: the running sums over wholly covered annuli
        if ((e = timed(c, RR_KERNEL_WEIGHTS, s, [&] { return launch_direct_prefix(c, s); })) != cudaSuccess)
            return cuda_fail(c, e, "direct-model set-up kernel");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "rr_build_weights");
        c->tables_built = true;
        return RR_OK;
    }
    const bool need_w = !c->weights_built;
    if ((e = timed(c, RR_KERNEL_WEIGHTS, s, [&] { return launch_weights(c, need_w, s); })) != cudaSuccess)
        return cuda_fail(c, e, "weight table kernel");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "rr_build_weights");
    c->weights_built = true;
    c->tables_built = true;
    return RR_OK;
}

int32_t rr_nparam(const rr_ctx* c) { return c ? c->nparam : -1; }

size_t rr_workspace_bytes(const rr_ctx* c, int32_t npv, int32_t npt, int32_t with_grad) {
    if (!c || npv < 0 || npt < 0) return 0;
    return ws_layout(c, npv, npt, with_grad != 0).total;
}


rr_status rr_evaluate(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt, const double* params,
                      int32_t npv, const int32_t* ss, const double* exptime, void* flux, int32_t* pv_status,
                      void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("rr_evaluate");
    return evaluate_impl(c, times, pb_index, npt, params, npv, ss, exptime, flux, pv_status, ws, ws_bytes, false,
                         stream);
}

rr_status rr_evaluate_grad(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt,
                           const double* params, int32_t npv, const int32_t* ss, const double* exptime,
                           const void* grad_flux, double* grad_params, int32_t* pv_status, void* ws,
                           size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("rr_evaluate_grad");
    return evaluate_grad_impl(c, times, pb_index, npt, params, npv, ss, exptime, grad_flux, grad_params, pv_status,
                              ws, ws_bytes, false, stream);
}

rr_status rr_prepare(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt, const double* params,
                     int32_t npv, const int32_t* ss, const double* exptime, int32_t* pv_status, void* ws,
                     size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("rr_prepare");
    PbParams pbp;
    // the workspace stands in for the output pointer: rr_prepare writes only the workspace
    rr_status st = check_eval(c, times, pb_index, npt, params, npv, ss, exptime, ws, ws, ws_bytes, true, pbp);
    cudaStream_t s = (cudaStream_t)stream;
    if (st != RR_OK || npv == 0) return st;
    if (npt == 0)
        return pv_status ? status_only(c, params, npv, pbp, true, pv_status, ws, ws_bytes, s, "rr_prepare") : RR_OK;
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    if ((e = run_setup(c, times, pb_index, npt, params, npv, pbp, true, pv_status, ws, s)) != cudaSuccess)
        return cuda_fail(c, e, "set-up kernels");
    return RR_OK;
}

rr_status rr_evaluate_prepared(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt,
                               const double* params, int32_t npv, const int32_t* ss, const double* exptime,
                               void* flux, int32_t* pv_status, const void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("rr_evaluate_prepared");
    return evaluate_impl(c, times, pb_index, npt, params, npv, ss, exptime, flux, pv_status, const_cast<void*>(ws),
                         ws_bytes, true, stream);
}

rr_status rr_evaluate_grad_prepared(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt,
                                    const double* params, int32_t npv, const int32_t* ss, const double* exptime,
                                    const void* grad_flux, double* grad_params, int32_t* pv_status, const void* ws,
                                    size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("rr_evaluate_grad_prepared");
    return evaluate_grad_impl(c, times, pb_index, npt, params, npv, ss, exptime, grad_flux, grad_params, pv_status,
                              const_cast<void*>(ws), ws_bytes, true, stream);
}

rr_status rr_evaluate_both_prepared(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt,
                                    const double* params, int32_t npv, const int32_t* ss, const double* exptime,
                                    const void* grad_flux, void* flux, double* grad_params, int32_t* pv_status,
                                    const void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("rr_evaluate_both_prepared");
    if (!c) return fail(nullptr, RR_EINVAL, "null context");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e == cudaSuccess && !c->aux) e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->ev_fork) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !c->ev_join) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    // the adjoint (and its finish kernel) on the second stream, after everything before on s
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "rr_evaluate_both_prepared");
    // the adjoint first: it is the longer of the two, and the forward kernel's CTAs fill in
    rr_status st = evaluate_grad_impl(c, times, pb_index, npt, params, npv, ss, exptime, grad_flux, grad_params,
                                      pv_status, const_cast<void*>(ws), ws_bytes, true, c->aux);
    const rr_status st2 = st == RR_OK ? evaluate_impl(c, times, pb_index, npt, params, npv, ss, exptime, flux,
                                                      pv_status, const_cast<void*>(ws), ws_bytes, true, stream)
                                      : st;
    // s waits for the second stream whatever happened, so that nothing of this call is left behind it
    e = cudaEventRecord(c->ev_join, c->aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join, 0);
    if (st != RR_OK) return st;
    if (st2 != RR_OK) return st2;
    if (e != cudaSuccess) return cuda_fail(c, e, "rr_evaluate_both_prepared");
    return RR_OK;
}

int64_t rr_read_table(rr_ctx* c, int32_t which, double* out, int64_t capacity) {
    if (!c) return -1;
    const int nk = c->cfg.nk, ng = c->cfg.ng, nz = c->nz, nb = c->nbasis;
    const double* src = nullptr;
    const double* hsrc = nullptr;
    int64_t n = 0;
    switch (which) {
        case RR_TABLE_ZE: hsrc = c->ze.data(); n = nz + 1; break;
        case RR_TABLE_ZM: hsrc = c->zm.data(); n = nz; break;
        case RR_TABLE_MU: hsrc = c->mu.data(); n = nz; break;
        case RR_TABLE_WEIGHTS: src = c->d_w; n = (int64_t)nk * ng * nz; break;
        case RR_TABLE_BASIS: src = c->d_basis; n = (int64_t)nb * nz; break;
        case RR_TABLE_ISTAR: src = c->d_istar; n = nb; break;
        case RR_TABLE_PROJ: src = c->d_T64; n = (int64_t)nb * nk * ng; break;
        default: fail(c, RR_EINVAL, "unknown table"); return -1;
    }
    if (c->cfg.direct && (which == RR_TABLE_WEIGHTS || which == RR_TABLE_PROJ)) {
        fail(c, RR_ESTATE, "the direct model has no (k, g) table");
        return -1;
    }
    if (!out) return n;
    const int64_t m = capacity < n ? capacity : n;
    if (m <= 0) return n;
    if (hsrc) {
        std::memcpy(out, hsrc, (size_t)m * sizeof(double));
        return n;
    }
    if (!c->tables_built || !src) {
        fail(c, RR_ESTATE, "tables are not built");
        return -1;
    }
    cudaSetDevice(c->cfg.device);
    cudaError_t e = cudaMemcpy(out, src, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cuda_fail(c, e, "rr_read_table");
        return -1;
    }
    return n;
}

rr_status rr_sync_status(rr_ctx* c, void* stream) {
    if (!c) return fail(nullptr, RR_EINVAL, "null context");
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "rr_sync_status");
    int w = 0;
    if ((e = cudaMemcpy(&w, c->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(c, e, "rr_sync_status");
    if (w != 0) {
        cudaMemset(c->d_err, 0, sizeof(int));
        return fail(c, RR_ETIMEOUT, w == kErrQueueTimeout ? "a kernel gave up waiting for its shared work queue"
                                                           : "a kernel gave up waiting for its shared-memory staging copy");
    }
    return RR_OK;
}

rr_status rr_selftest_wait(rr_ctx* c, int32_t which, void* stream) {
    if (!c) return fail(nullptr, RR_EINVAL, "null context");
    if (which != 0 && which != 1) return fail(c, RR_EINVAL, "which must be 0 (mbarrier) or 1 (work queue)");
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e == cudaSuccess) e = launch_selftest(c, which, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "rr_selftest_wait");
    return RR_OK;
}

const char* rr_last_error(const rr_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

int64_t rr_launch_count(const rr_ctx* c) { return c ? c->launches : 0; }

rr_status rr_count_samples(rr_ctx* c, int32_t enable) {
    if (!c) return fail(nullptr, RR_EINVAL, "null context");
    cudaSetDevice(c->cfg.device);
    if (enable && !c->d_counts) {
        const size_t n = (size_t)RR_KERNEL_KINDS * RR_COUNT_KINDS;
        cudaError_t e = cudaMalloc((void**)&c->d_counts, n * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(c, e, "allocation of the sample counters");
        if ((e = cudaMemset(c->d_counts, 0, n * sizeof(unsigned long long))) != cudaSuccess)
            return cuda_fail(c, e, "clearing the sample counters");
    }
    c->counting = enable != 0;
    return RR_OK;
}

rr_status rr_count_read(rr_ctx* c, int32_t kind, int64_t* counts, int32_t reset) {
    if (!c || !counts) return fail(c, RR_EINVAL, "null argument");
    if (kind != RR_KERNEL_FLUX && kind != RR_KERNEL_GRAD) return fail(c, RR_EINVAL, "counted kinds: flux, grad");
    for (int j = 0; j < RR_COUNT_KINDS; ++j) counts[j] = 0;
    if (!c->d_counts) return RR_OK;
    cudaSetDevice(c->cfg.device);
    unsigned long long h[(size_t)RR_KERNEL_KINDS * RR_COUNT_KINDS];
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, c->d_counts, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the sample counters");
    for (int j = 0; j < RR_COUNT_KINDS; ++j) counts[j] = (int64_t)h[(size_t)kind * RR_COUNT_KINDS + j];
    if (reset && (e = cudaMemset(c->d_counts, 0, sizeof h)) != cudaSuccess)
        return cuda_fail(c, e, "clearing the sample counters");
    return RR_OK;
}

rr_status rr_profile(rr_ctx* c, int32_t enable) {
    if (!c) return fail(nullptr, RR_EINVAL, "null context");
    c->profiling = enable != 0;
    return RR_OK;
}

rr_status rr_profile_read(rr_ctx* c, int32_t kind, double* total_ms, int64_t* count, int32_t reset) {
    if (!c) return fail(nullptr, RR_EINVAL, "null context");
    if (kind < 0 || kind >= RR_KERNEL_KINDS) return fail(c, RR_EINVAL, "unknown kernel kind");
    cudaSetDevice(c->cfg.device);
    resolve_timing(c);
    if (total_ms) *total_ms = c->prof_ms[kind];
    if (count) *count = c->prof_n[kind];
    if (reset) {
        for (int k = 0; k < RR_KERNEL_KINDS; ++k) { c->prof_ms[k] = 0.0; c->prof_n[k] = 0; }
    }
    return RR_OK;
}

}  // extern "C"
