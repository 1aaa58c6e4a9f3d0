// Internal layout shared by the host code and the kernels of librr.
//
// Per-call data flow (all stream-ordered, no host synchronisation):
//   rr_direct_table_kernel  (direct model only) per (pv, k slot) and g node the
//                        weight projections for the pv's own k -> workspace
//   rr_pv_setup_kernel   params -> one record per parameter vector in the
//                        caller's workspace (orbit constants, transit window,
//                        profile rows divided by I_star: interpolated in k, the
//                        pv's direct projections, or below k_small the profile at
//                        the planet's centre); in the same launch (mixed form)
//                        the per-time float-float offsets, passband and 128-time
//                        group summaries; with several passbands then
//                        rr_chunk_order_kernel (time chunks heaviest first)
//   rr_flux_mixed_kernel / rr_flux_fp64_kernel: records of a pv tile -> shared
//                        memory (one bulk async copy), flux[pv][t] for the tile
//   rr_grad_mixed_kernel / rr_grad_fp64_kernel: same tiling; per-(pv, chunk)
//                        partial sums of the vector-Jacobian product -> workspace
//   rr_grad_finish_kernel  partial sums -> grad_params (fixed order), chain rules
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/rr.h"

namespace rr {

constexpr int kBlock = 256;               // threads per CTA in the per-point kernels
constexpr int kPPT = 4;                   // points per thread
constexpr int kPtTile = kBlock * kPPT;    // points per CTA
constexpr int kMaxPvTile = 32;            // parameter vectors per CTA (upper bound)
constexpr int kSmemTarget = 32 * 1024;    // record bytes per CTA the tiler aims for
constexpr int kMaxNz = 4096;
constexpr size_t kMaxSmem = 227 * 1024;   // dynamic shared memory per CTA on sm_103a
constexpr int kMaxBasis = RR_MAX_PB + 4;  // profile bases: 1 + nldc (named) or npb (tabulated)
constexpr double kESwitch = 0.8;          // above this eccentricity Kepler is solved in FP64
constexpr float kContactBand = 5e-3f;     // mixed adjoint: samples with min(1 + k - z, |z - (1 - k)|) below
                                          // this get z and the contact factors in float-float (adjoint_sample)
constexpr float kContactBandGrazing = 1e-2f;  // the same for a grazing (pv, passband): z at conjunction above
                                              // 1 - k, every in-transit sample near the outer contact
constexpr float kNodeBand = 1e-4f;        // ... and so do samples within this of a g-node (in units of cells)
constexpr int kWarpPts = 4 * 32;          // times per group: one warp, 4 consecutive times per lane

// Per 128-time group, written once per call by points_group (mixed form):
// the range and largest magnitude of the float offsets of its times from the
// group's first time t_g, whether all 128 times exist with a valid passband,
// t_g - t_0 (t_0 = the first time of the call) as a float pair, and the
// group's weight: its exposure sub-samples (the sum of ss over its times).
struct alignas(16) GroupInfo {
    float wlo, whi, maxdt;
    int32_t full;                 // 1: 128 times, every passband index valid
    float toff_h, toff_l;
    float weight;
    float pad;
};

static_assert(sizeof(GroupInfo) % 16 == 0, "group summaries are copied with bulk asynchronous copies");

// device error word values (ctx->d_err)
constexpr int kErrBarrierTimeout = 1;
constexpr int kErrQueueTimeout = 2;

enum PvFlags : int32_t { kPvCircular = 1, kPvKepler64 = 2, kPvNoWindow = 4 };

// Fixed part of a per-pv record.  R = float (mixed) or double (FP64).
// Derived quantities of the Keplerian orbit written in the offset-from-
// conjunction form used by the kernels (x = E - E0):
//   P_x = ax1 V + ax2 S,  P_y = rho0 + ay1 V + ay2 S,  V = 1 - cos x, S = sin x
//   z^2 = a^2 P_x^2 + b^2 P_y^2, in front iff P_y > 0
//   Kepler: x - ecE0 S + esE0 V = dM,  dM = M - M0 = n (t - T0) reduced
template <typename R>
struct alignas(16) PvHead {
    double T0, P, invP;            // FP64 epoch and period (phase reduction)
    double ecE0d, esE0d, inv_den0d;  // FP64 Kepler constants (e > kESwitch fallback)
    float wmax_c;                  // largest point window over the passbands, cycles
    float kep2, kep3;              // FP32 Kepler start: x = y + kep2 y^2 + kep3 y^3, y = dM / (1 - e cos E0)
    float kepC;                    // bound of |f'' / (2 f')| of the offset Kepler function (convergence test)
    R a, b, a2, b2;
    R e, ecE0, esE0, inv_den0;     // inv_den0 = 1 / (1 - e cos E0)
    R ax1, ax2, ay1, ay2;
    R rho0, n, Bh, Bl;             // n = 2 pi / P; Bh + Bl = 1 / P (float-float)
    R dM0de, dM0dw, se, cw;        // dM0/de, dM0/dw, sqrt(1 - e^2), cos w
    R sw, cE0, sE0, inv_se;        // sin w, cos E0, sin E0, 1 / sqrt(1 - e^2)
    int32_t flags, status, pad3, pad4;
};

// Per-(pv, passband) constants.
template <typename R>
struct alignas(16) PvPb {
    R k, inv1pk;      // radius ratio, 1 / (1 + k)
    R win_s;          // |dM| bound of a possible transit for one sample [rad]
    R win_p;          // same, widened by the passband's exposure half-span [rad]
    float win_pc;     // win_p in cycles (phase units of the FP32 point check)
    float cband;      // the mixed adjoint's contact band: kContactBand, or kContactBandGrazing
    float pad[2];
};

// Arguments of the per-time preparation carried by the set-up launch (its
// first npoints CTAs; none when npt == 0).
struct PointsArgs {
    const double* times;
    const int32_t* pb_index;
    int32_t npt, ngroups, npoints, pad_;
    float2* dt;
    int32_t* pbw;
    GroupInfo* grp;
};

// Orbit constants of a pv as float pairs (hi + lo of the FP64 value) for the
// mixed adjoint's contact refinement (mixed form, adjoint layout only): a
// block at the end of the pv's header (staged into shared memory with it),
// followed by one PvContactFF per passband.
// Read only for the few samples within kContactBand of a contact point, where
// the derivative of the covered area behaves like sqrt(1 + k - z) and the FP32
// rounding of z (~1e-7) would reach the gradient with a large factor (see
// adjoint_sample).
struct alignas(16) PvOrbitFF {
    float ax1[2], ax2[2], ay1[2], ay2[2];   // P_x = ax1 V + ax2 S, P_y = rho0 + ay1 V + ay2 S (as in PvHead)
    float rho0[2], a2[2], b2[2];            // z^2 = a2 P_x^2 + b2 P_y^2
    float ecE0[2], esE0[2];                 // Kepler: x - ecE0 S + esE0 V = dM
    float pad[2];
};
struct alignas(16) PvContactFF {
    float opk[2], omk[2];                   // 1 + k and 1 - k of the passband's radius ratio
    float gsc[2], pad[2];                   // (ng - 1) / (1 + k): g-node coordinate per unit of z
};

// Table of sin x0 and 1 - cos x0 (float pairs: S hi, S lo, V hi, V lo) at
// x0 = j / kSvTabRes, j = -kSvTabRes .. kSvTabRes (the float-float sine of the
// mixed adjoint's contact refinement).
constexpr int kSvTabRes = 64;
constexpr int kSvTabLen = 2 * kSvTabRes + 1;
// Per-pv records live in two regions of the workspace: the headers (PvHead +
// one PvPb per passband; staged into shared memory by the kernels) and the
// profile rows (read through the cache hierarchy where a transit needs them).
struct RecLayout {
    int32_t npb, ng, ng_pad, rows_per_pb;  // rows: 1 (flux) or 3 + nldc (adjoint)
    int32_t nldc, off_pb;                  // byte offset of the PvPb array in a header
    int32_t head_bytes, rows_bytes;        // per-pv strides of the two regions (multiples of 16)
    int32_t kbar_slot;                     // adjoint accumulator of the shared weights' mean k, else -1
    int32_t orb_off;                       // byte offset of the PvOrbitFF block in a header, else -1
};

template <typename R>
inline RecLayout make_layout(int npb, int ng, int nldc, bool grad) {
    RecLayout L;
    L.npb = npb;
    L.ng = ng;
    L.ng_pad = (ng + 3) & ~3;
    L.nldc = nldc;
    L.rows_per_pb = grad ? 3 + nldc : 1;
    L.off_pb = (int32_t)sizeof(PvHead<R>);
    size_t head = ((size_t)L.off_pb + npb * sizeof(PvPb<R>) + 15) & ~(size_t)15;
    L.orb_off = -1;
    if (grad && sizeof(R) == sizeof(float)) {
        L.orb_off = (int32_t)head;
        head += sizeof(PvOrbitFF) + (size_t)npb * sizeof(PvContactFF);
    }
    L.head_bytes = (int32_t)head;
    L.rows_bytes = (int32_t)(((size_t)npb * L.rows_per_pb * L.ng_pad * sizeof(R) + 15) & ~(size_t)15);
    L.kbar_slot = -1;
    return L;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Start of the rows region after npv headers.
__host__ __device__ inline size_t rows_offset(const RecLayout& L, int npv) {
    return ((size_t)npv * L.head_bytes + 255) & ~(size_t)255;
}

// Passband sampling constants, passed by value.
struct PbParams {
    int32_t npb;
    int32_t ss[RR_MAX_PB];
    double exptime[RR_MAX_PB];
    float first[RR_MAX_PB];     // offset of sub-sample s = first + s * step [days]
    float step[RR_MAX_PB];
    float inv_ss[RR_MAX_PB];
    float first_lo[RR_MAX_PB];  // FP64 first and step minus their floats (first + first_lo, step + step_lo)
    float step_lo[RR_MAX_PB];
};

// Model constants for the kernels (by value).
struct ModelParams {
    int32_t ld_model, npb, chromatic, nldc, nparam, nk, ng, nbasis;
    int32_t direct, nz;   // direct model (per-call weights for each k); radial bins
    int32_t shared, pad_;  // one weight array per pv at the mean of its per-passband k
    double k0, k1, dk;
    double inv_dk;   // 1 / dk (host FP64)
    double exp_c;    // int_0^1 mu / (e^mu - 1) dmu (disk integral of the exponential law's second term)
    double dg;       // 1 / (ng - 1)
    double k_small;  // small-planet approximation threshold (0 = off)
    double mu_min;   // mu of the outermost bin mean (the small-planet approximation's limb clamp)
    const double* tab;   // tabulated profiles (device): per passband mu nodes then intensities
    const int* tab_off;  // node offsets of the passbands in tab (npb + 1)
};

// Per-call projections of the direct model (the workspace region after the
// records): for every (pv, k slot) row = pv * nkp + slot, basis b and g node,
// T[b][row][ig] = sum_j w_j(k_row, g) l_b[j] (R = float: hi + lo float
// pair; R = double: hi only) and, for the adjoint, dT/dk at fixed g.
struct DirectTables {
    void* hi;      // R[nbasis][nrows][ng]
    float* lo;     // float[nbasis][nrows][ng] (mixed form), else null
    void* dk;      // R[nbasis][nrows][ng] (adjoint layout), else null
    int32_t nrows;
};

}  // namespace rr

// The context (opaque to users).
struct rr_ctx {
    rr_config cfg;
    int nz = 0, nldc = 0, nbasis = 0, nparam = 0, nkp = 0;
    double dk = 0, dg = 0;
    std::vector<double> ze, zm, mu;
    std::vector<std::vector<double>> tab_mu, tab_I;
    double* d_ze = nullptr;
    double* d_mu = nullptr;
    double* d_w = nullptr;       // nk * ng * nz
    double* d_basis = nullptr;   // nbasis * nz
    double* d_istar = nullptr;   // nbasis
    double* d_T64 = nullptr;     // nbasis * nk * ng
    float* d_T32 = nullptr;      // nbasis * nk * ng
    float* d_DT32 = nullptr;     // nbasis * nk * ng: T[.][.][ig+1] - T[.][.][ig] (FP64 difference, FP32 stored)
    double* d_tab = nullptr;     // tabulated profiles, concatenated (mu then I per passband)
    int* d_tab_off = nullptr;    // npb + 1 offsets (in nodes)
    int* d_err = nullptr;        // device error word
    float4* d_svtab = nullptr;   // kSvTabLen entries (mixed form): sin and 1 - cos as float pairs
    unsigned long long* d_counts = nullptr;   // RR_KERNEL_KINDS x RR_COUNT_KINDS sample counters
    bool counting = false;
    int host_path = 0;   // RR_HOST_IN_PLACE / RR_HOST_STAGED of the last host-buffer call
    // direct model: FP32 copies of the edges and profiles, and per basis the
    // running sums P[b][m] = sum_{j<m} pi (ze[j+1]^2 - ze[j]^2) l_b[j]
    float* d_zef = nullptr;      // nz + 1
    float* d_basisf = nullptr;   // nbasis * nz
    double* d_pre64 = nullptr;   // nbasis * (nz + 1)
    float* d_pref = nullptr;     // 2 * nbasis * (nz + 1): FP32 hi, then lo
    double* d_gl = nullptr;      // Gauss-Legendre nodes and weights of rr_exact_flux (on first use)
    double* d_lnmu = nullptr;    // ln mu of the bin means (power-2 laws, direct model)
    float* d_lnmuf = nullptr;    // the same in FP32
    int num_sms = 0;
    bool weights_built = false;
    bool tables_built = false;
    std::string err;
    long long launches = 0;
    // optional per-kernel timing with CUDA events on the launching stream
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Timed { int kind; cudaEvent_t a, b; };
    std::vector<Timed> timed;
    double prof_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long prof_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // second stream of rr_evaluate_both_prepared (the adjoint beside the forward kernel) and its
    // fork and join events, created on first use
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // host-buffer pipeline (rr_evaluate_host): copy-in, compute and copy-out
    // streams, per-slot events, one grow-only device buffer
    struct HostPipe {
        cudaStream_t s[3] = {nullptr, nullptr, nullptr};
        cudaEvent_t ev[3][4] = {};   // [slot][inputs copied, computed, results copied, flux computed]
        void* buf = nullptr;
        size_t bytes = 0;
    } pipe;
};

namespace rr {
// An NVTX range over a C-ABI call (visible in Nsight timelines; a no-op without a tool).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// shared weights in effect: one weight array per pv for several per-passband k
inline bool shared_weights(const rr_ctx* c) { return c->cfg.shared_weights && c->cfg.chromatic && c->cfg.npb > 1; }
// rows of the direct model's per-call projections per pv
inline int direct_rows_per_pv(const rr_ctx* c) { return shared_weights(c) ? 1 : c->nkp; }
// power-2 laws: the profile is formed per pv inside the direct model's weight pass
inline bool power2_law(const rr_ctx* c) {
    return c->cfg.ld_model == RR_LD_POWER2 || c->cfg.ld_model == RR_LD_POWER2_PM;
}
// columns of the direct model's projections per row: the profile bases, or for the power-2
// laws 1 and, per passband the row serves, mu^alpha and mu^alpha ln mu
inline int direct_cols(const rr_ctx* c) {
    if (!power2_law(c)) return c->nbasis;
    return (c->cfg.chromatic && !shared_weights(c)) ? 3 : 1 + 2 * c->cfg.npb;
}
// adjoint accumulators per pv: the parameters, plus the mean k with shared weights
inline int grad_nacc(const rr_ctx* c) { return c->nparam + (shared_weights(c) ? 1 : 0); }

// launchers (defined in the .cu files); all return cudaGetLastError() after launch
cudaError_t launch_ld_basis(rr_ctx* c, cudaStream_t s);
cudaError_t launch_weights(rr_ctx* c, bool need_w, cudaStream_t s);
// direct model: the running sums at build time, the per-call projections
cudaError_t launch_direct_prefix(rr_ctx* c, cudaStream_t s);
cudaError_t launch_direct_tables(rr_ctx* c, const double* params, int npv, bool grad, const DirectTables& D,
                                 cudaStream_t s);
size_t direct_bytes(const rr_ctx* c, int npv, bool grad);
DirectTables direct_view(const rr_ctx* c, void* base, int npv, bool grad);
cudaError_t launch_selftest(rr_ctx* c, int which, cudaStream_t s);
// with several passbands also the order of the CTA time chunks, heaviest first (ws_ord)
// records: the workspace (the direct model's projections follow the records).  With times
// (mixed form, npt > 0) the same launch also writes the per-time inputs of the FP32 kernels
// (float-float offsets, passband, 128-time group summaries) into pts_dt, pts_pb, pts_grp.
cudaError_t launch_pv_setup(rr_ctx* c, const double* params, int npv, const PbParams& pbp,
                            bool grad, void* records, int32_t* pv_status, cudaStream_t s,
                            const double* times = nullptr, const int32_t* pb_index = nullptr, int npt = 0,
                            void* pts_dt = nullptr, void* pts_pb = nullptr, void* pts_grp = nullptr);
// grad_layout: the records were written in the adjoint's layout (rr_prepare)
// pts_ord: the order of the time chunks (several passbands), or null (in index order)
cudaError_t launch_flux(rr_ctx* c, const double* times, const int32_t* pb_index, const void* pts_dt,
                        const void* pts_pb, const void* pts_grp, const void* pts_ord, int npt, int npv,
                        const PbParams& pbp, const void* records,
                        void* flux, int32_t* pv_status, bool grad_layout, cudaStream_t s);
cudaError_t launch_grad(rr_ctx* c, const double* times, const int32_t* pb_index, const void* pts_dt,
                        const void* pts_pb, const void* pts_grp, const void* pts_ord, int npt, int npv,
                        const PbParams& pbp, const void* records,
                        const void* grad_flux, void* partials, int32_t* pv_status, cudaStream_t s);
cudaError_t launch_chunk_order(rr_ctx* c, int npt, void* ws_grp, void* ws_ord, cudaStream_t s);
// time chunks of the FP32 per-point kernels
inline int time_chunks(int npt, int gpc) { return ((npt + kWarpPts - 1) / kWarpPts + gpc - 1) / gpc; }
// Whether p is device memory.  A caller's buffer may also be page-locked host memory, which the
// kernels reach in place over the host link with plain loads and stores; the bulk asynchronous
// copy engine (stores from shared memory, L2 prefetches) is used on device memory only.
// The device address of a caller's buffer [p, p + bytes) when it is page-locked host memory
// that kernels on the current device can reach in place (both ends mapped, in one mapping);
// nullptr otherwise.
const void* mapped_host(const void* p, size_t bytes);
// Device scratch of one request whose host buffers are all mapped page-locked memory (the
// workspace alone; rr_request_bytes is the staged figure).
size_t request_bytes_in_place(const rr_ctx* c, int npv, int npt, bool grad);
// Device addresses of every caller buffer of one evaluation, when all of them are mapped
// page-locked memory (ok; looked up for the current device); a batch with no times or no pvs
// is staged.
struct InPlace {
    const double* t = nullptr;
    const int32_t* pb = nullptr;
    const double* p = nullptr;
    const void* g = nullptr;
    void* f = nullptr;
    double* go = nullptr;
    int32_t* st = nullptr;
    bool ok = false;
};
InPlace map_in_place(const rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt,
                     const double* params, int32_t npv, const void* grad_flux, void* flux, double* grad_params,
                     int32_t* pv_status);
// One evaluation (with the adjoint when m.g is set) on mapped buffers, enqueued on s; ws is a
// device workspace of ws_bytes >= rr_workspace_bytes.  overlap: the forward and adjoint kernels
// on s and the context's second stream (rr_evaluate_both_prepared).
rr_status run_in_place(rr_ctx* c, const InPlace& m, int32_t npt, int32_t npv, const int32_t* ss,
                       const double* exptime, void* ws, size_t ws_bytes, cudaStream_t s, bool overlap);
inline bool in_device_memory(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice;
}
cudaError_t launch_grad_reduce(rr_ctx* c, int npt, const double* params, int npv, const void* records,
                               const void* partials, double* grad_params, cudaStream_t s);
size_t records_bytes(const rr_ctx* c, int npv, bool grad);
size_t partials_bytes(const rr_ctx* c, int npv, int npt);
// workspace layout: [records | direct-model projections | per-point float-float times + passband,
//                    per-group summaries (mixed form) | partial sums]
struct WsLayout {
    size_t rec, dir, pts_dt, pts_pb, pts_grp, pts_ord, part, total;
};
WsLayout ws_layout(const rr_ctx* c, int npv, int npt, bool grad);

ModelParams model_params(const rr_ctx* c);
int pv_tile_for(int rec_bytes);
void release_host_pipe(rr_ctx* c);
int groups_per_cta(int npt);
}  // namespace rr
