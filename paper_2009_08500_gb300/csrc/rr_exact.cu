// The exact occulted flux (the radial integral the model discretises, with
// neither the radial grid nor the weights) and the automatic choice of the
// grid resolution against it (Sect. 3.1.1 and 3.3 note that z_cut and the two
// radial resolutions can be tuned automatically for a limb-darkening law and
// an error threshold; the g resolution is tuned here as well).
//
// Occulted flux of a planet of radius k at distance c (Eq. 1 in radial form):
//   F(c) = int_0^1 I(mu(r)) 2 r theta(r) dr,  mu = sqrt(1 - r^2),
// theta(r) = the half-angle of the radius-r circle inside the planet: pi for
// r <= k - c (the planet covers the disk's centre), the lens angle
// atan2(K, r^2 + c^2 - k^2) for |c - k| < r < c + k, 0 beyond.  flux =
// 1 - F / I_star.  Each piece [a, b] is integrated by Gauss-Legendre in phi
// with r = a + (b - a)(1 - cos phi) / 2, phi in [0, pi]: the substitution
// absorbs the square-root behaviour of theta at the contacts and of mu at the
// limb, so a fixed rule converges fast: to FP64 round-off for the polynomial
// laws in mu, ~1e-11 for the laws with mu^(1/2), mu ln mu or 1/(1 - e^mu)
// terms (not smooth at the limb after the substitution), ~1e-8 for a table
// (kinks at its nodes; 512 nodes).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "rr_device.cuh"

namespace rr {
namespace {

constexpr int kGL = 96;       // Gauss-Legendre nodes per piece (named laws)
constexpr int kGLTab = 512;   // for a table: its profile has a kink at every node, which a rule
                              // of n nodes resolves to O(n^-2)

// Nodes and weights of the n-point Gauss-Legendre rule on [-1, 1]: the roots
// of P_n by Newton's method on the three-term recurrence
// j P_j = (2j - 1) x P_{j-1} - (j - 1) P_{j-2}, and w = 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p0 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double pm = p0;
                p0 = p1;
                p1 = ((2.0 * j - 1.0) * z * p0 - (j - 1.0) * pm) / j;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-15) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

struct ExactLaw {
    double ud[5];   // weights of the profile bases: 1, then the coefficients
    int b0, nc;     // first basis (the passband's for a table), coefficient count
    int pb;         // passband (its disk integral for a table)
};

// Profile at radius r (r <= 1).
__device__ __forceinline__ double profile_at(const ModelParams& mp, const ExactLaw& lw, double r,
                                             const double* tab, const int* tab_off) {
    const double m = sqrt(fmax(1.0 - r * r, 0.0));
    double v = 0.0, d;
    for (int c = 0; c <= lw.nc; ++c) v += lw.ud[c] * ld_basis_mu(mp, lw.b0 + c, fmax(m, 1e-300), tab, tab_off, d);
    return v;
}

// One warp per point; lanes take every 32nd node of each piece; the sum over
// lanes is a fixed shuffle tree.
__global__ void __launch_bounds__(256) rr_exact_kernel(ModelParams mp, ExactLaw lw, const double* __restrict__ z,
                                                       const double* __restrict__ kk, int n,
                                                       const double* __restrict__ gl, int ngl,
                                                       const double* __restrict__ istar,
                                                       const double* __restrict__ tab,
                                                       const int* __restrict__ tab_off, double* __restrict__ out) {
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double c = z[warp], k = kk[warp];
    double Is = mp.ld_model == RR_LD_TABULATED ? istar[lw.pb] : istar[0];
    if (mp.ld_model != RR_LD_TABULATED)
        for (int j = 0; j < lw.nc; ++j) Is += lw.ud[1 + j] * istar[1 + j];
    double F = 0.0;
    if (c < 1.0 + k && k > 0.0) {
        const double pi = CUDART_PI;
        // piece A: wholly covered circles, r in [0, min(k - c, 1)]
        if (c < k) {
            const double a = 0.0, b = fmin(k - c, 1.0);
            for (int i = lane; i < ngl; i += 32) {
                const double phi = 0.5 * pi * (gl[i] + 1.0);
                const double r = a + 0.5 * (b - a) * (1.0 - cos(phi));
                const double jac = 0.5 * (b - a) * sin(phi) * 0.5 * pi;
                F += gl[ngl + i] * jac * profile_at(mp, lw, r, tab, tab_off) * 2.0 * pi * r;
            }
        }
        // piece B: the lens, r in [|c - k|, min(c + k, 1)]
        const double a = fabs(c - k), b = fmin(c + k, 1.0);
        if (a < b) {
            for (int i = lane; i < ngl; i += 32) {
                const double phi = 0.5 * pi * (gl[i] + 1.0);
                const double r = a + 0.5 * (b - a) * (1.0 - cos(phi));
                const double jac = 0.5 * (b - a) * sin(phi) * 0.5 * pi;
                const double h = ((r + k) - c) * (c + (k - r)) * (c + (r - k)) * (c + r + k);
                const double theta = atan2(sqrt(fmax(h, 0.0)), r * r + (c - k) * (c + k));
                F += gl[ngl + i] * jac * profile_at(mp, lw, r, tab, tab_off) * 2.0 * r * theta;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) F += __shfl_xor_sync(0xffffffffu, F, o);
    if (lane == 0) out[warp] = 1.0 - F / Is;
}

}  // namespace
}  // namespace rr

using namespace rr;

namespace {

// Coefficients of one passband as basis weights (the Kipping map applied).
rr_status exact_law(const rr_ctx* c, const double* ldc, int pb, ExactLaw& lw) {
    std::memset(&lw, 0, sizeof(lw));
    lw.ud[0] = 1.0;
    lw.pb = pb;
    const bool named = c->cfg.ld_model != RR_LD_TABULATED;
    lw.b0 = named ? 0 : pb;
    lw.nc = named ? c->nldc : 0;
    if (!named) return RR_OK;
    if (c->nldc > 0 && !ldc) return RR_EINVAL;
    if (c->cfg.ld_model == RR_LD_QUADRATIC_TRI) {
        const double sq = std::sqrt(std::max(ldc[0], 0.0));
        lw.ud[1] = 2.0 * sq * ldc[1];
        lw.ud[2] = sq * (1.0 - 2.0 * ldc[1]);
    } else {
        for (int j = 0; j < c->nldc; ++j) lw.ud[1 + j] = ldc[j];
    }
    return RR_OK;
}

}  // namespace

extern "C" rr_status rr_exact_flux(rr_ctx* c, const double* z, const double* k, int32_t n, const double* ldc,
                                   int32_t pb, double* out, void* stream) {
    if (!c) return RR_EINVAL;
    if (n < 0 || pb < 0 || pb >= c->cfg.npb) {
        c->err = "rr_exact_flux: n must be >= 0 and pb a passband of the context";
        return RR_EINVAL;
    }
    if (!c->tables_built) {
        c->err = "rr_exact_flux: rr_build_weights has not been called since the last change";
        return RR_ESTATE;
    }
    if (n == 0) return RR_OK;
    if (!z || !k || !out) {
        c->err = "rr_exact_flux: z, k and out must be non-null";
        return RR_EINVAL;
    }
    ExactLaw lw;
    if (exact_law(c, ldc, pb, lw) != RR_OK) {
        c->err = "rr_exact_flux: ldc must hold the law's coefficients";
        return RR_EINVAL;
    }
    cudaError_t e = cudaSetDevice(c->cfg.device);
    const int ngl = c->cfg.ld_model == RR_LD_TABULATED ? kGLTab : kGL;
    if (e == cudaSuccess && !c->d_gl) {
        // nodes then weights of the rule
        std::vector<double> x, w;
        gauss_legendre(ngl, x, w);
        x.insert(x.end(), w.begin(), w.end());
        e = cudaMalloc((void**)&c->d_gl, x.size() * sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(c->d_gl, x.data(), x.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        const ModelParams mp = model_params(c);
        const unsigned blocks = (unsigned)(((size_t)n * 32 + 255) / 256);
        rr_exact_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(mp, lw, z, k, n, c->d_gl, ngl, c->d_istar, c->d_tab,
                                                                  c->d_tab_off, out);
        c->launches++;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        c->err = std::string("rr_exact_flux: ") + cudaGetErrorName(e);
        return RR_ECUDA;
    }
    return RR_OK;
}

namespace {

// Resolution ladders of the search.
const int kNzLadder[] = {4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048};
const int kNgLadder[] = {10, 15, 20, 30, 40, 60, 80, 120, 160, 240, 320, 480, 640, 960, 1280, 1920, 2560, 3840};
const double kZcut[] = {0.5, 0.6, 0.7, 0.8, 0.9};
constexpr int kNNz = sizeof(kNzLadder) / sizeof(int), kNNg = sizeof(kNgLadder) / sizeof(int), kNZc = 5;

struct Cand {
    int zc, in, lb, g;   // ladder indices
    bool operator==(const Cand& o) const { return zc == o.zc && in == o.in && lb == o.lb && g == o.g; }
};

// Test batch: one circular, central orbit per radius ratio (a = 1000, P = 1,
// T0 = 0, b = 0) and, per radius ratio, times at which z = g (1 + k) for a
// fixed low-discrepancy set of g in [0, 1) (golden-ratio sequence, and 0).
struct Probe {
    int npv = 0, npt = 0, nldc = 0;
    std::vector<double> times, params, zs, ks, exact;
    double *d_times = nullptr, *d_params = nullptr, *d_flux = nullptr, *d_z = nullptr, *d_k = nullptr;
    double* d_exact = nullptr;
    void* d_ws = nullptr;
    size_t ws_bytes = 0;
    void release() {
        cudaFree(d_times); cudaFree(d_params); cudaFree(d_flux); cudaFree(d_z); cudaFree(d_k); cudaFree(d_exact);
        cudaFree(d_ws);
        d_times = d_params = d_flux = d_z = d_k = d_exact = nullptr;
        d_ws = nullptr;
    }
};

constexpr int kProbeG = 400;
constexpr double kProbeA = 1000.0;

rr_config cand_config(const rr_config& base, const Cand& q) {
    rr_config c = base;
    c.zcut = kZcut[q.zc];
    c.nzin = kNzLadder[q.in];
    c.nzlimb = kNzLadder[q.lb];
    c.ng = kNgLadder[q.g];
    return c;
}

// Largest |model - exact| of a candidate grid over the probe (direct model, FP64); -1 on failure.
double cand_error(const rr_config& base, const Cand& q, const double* mu_tab, const double* I_tab, int ntab,
                  Probe& pr, std::string& err) {
    rr_config cfg = cand_config(base, q);
    if (cfg.nzin + cfg.nzlimb > 4096) return -1.0;
    rr_ctx* ctx = nullptr;
    if (rr_create(&cfg, &ctx) != RR_OK) {
        err = rr_last_error(nullptr);
        return -1.0;
    }
    double worst = -1.0;
    do {
        if (cfg.ld_model == RR_LD_TABULATED && rr_set_ld_profile(ctx, 0, mu_tab, I_tab, ntab) != RR_OK) break;
        if (rr_build_weights(ctx, nullptr) != RR_OK) break;
        if (!pr.d_exact) {
            // the reference: the exact integral (independent of the grid)
            if (cudaMalloc((void**)&pr.d_exact, pr.zs.size() * sizeof(double)) != cudaSuccess) break;
            if (rr_exact_flux(ctx, pr.d_z, pr.d_k, (int)pr.zs.size(), pr.nldc ? pr.params.data() + 7 : nullptr, 0,
                              pr.d_exact, nullptr) != RR_OK)
                break;
            pr.exact.resize(pr.zs.size());
            if (cudaMemcpy(pr.exact.data(), pr.d_exact, pr.exact.size() * sizeof(double), cudaMemcpyDeviceToHost) !=
                cudaSuccess)
                break;
        }
        const size_t need = rr_workspace_bytes(ctx, pr.npv, pr.npt, 0);
        if (need > pr.ws_bytes) {
            cudaFree(pr.d_ws);
            pr.d_ws = nullptr;
            pr.ws_bytes = 0;
            if (cudaMalloc(&pr.d_ws, need) != cudaSuccess) break;
            pr.ws_bytes = need;
        }
        const int32_t ss = 1;
        const double ex = 0.0;
        if (rr_evaluate(ctx, pr.d_times, nullptr, pr.npt, pr.d_params, pr.npv, &ss, &ex, pr.d_flux, nullptr, pr.d_ws,
                        pr.ws_bytes, nullptr) != RR_OK)
            break;
        std::vector<double> f((size_t)pr.npv * pr.npt);
        if (cudaMemcpy(f.data(), pr.d_flux, f.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) break;
        // pv p holds the points of radius ratio p at columns p * kProbeG .. (p + 1) * kProbeG
        double m = 0.0;
        for (int p = 0; p < pr.npv; ++p)
            for (int j = 0; j < kProbeG; ++j) {
                const size_t col = (size_t)p * kProbeG + j;
                m = std::max(m, std::fabs(f[(size_t)p * pr.npt + col] - pr.exact[col]));
            }
        worst = m;
    } while (false);
    if (worst < 0.0 && err.empty()) err = rr_last_error(ctx);
    rr_destroy(ctx);
    return worst;
}

}  // namespace

extern "C" rr_status rr_choose_grid(rr_config* cfg, const double* k, int32_t nk, const double* ldc,
                                    const double* mu_tab, const double* I_tab, int32_t ntab, double target,
                                    double* max_err) {
    if (!cfg || !k || nk < 1 || nk > 64 || !(target > 0.0)) return RR_EINVAL;
    if (cfg->ld_model == RR_LD_TABULATED && (!mu_tab || !I_tab || ntab < 2)) return RR_EINVAL;
    for (int i = 0; i < nk; ++i)
        if (!(k[i] > 0.0 && k[i] < 1.0)) return RR_EINVAL;
    rr_config base = *cfg;
    base.direct = 1;
    base.shared_weights = 0;
    base.k_small = 0.0;
    base.npb = 1;
    base.chromatic = 0;
    base.precision = RR_PREC_FP64;
    // the probe: one pv per radius ratio
    Probe pr;
    pr.npv = nk;
    pr.npt = nk * kProbeG;
    int nldc = 0;
    switch (base.ld_model) {
        case RR_LD_QUADRATIC: case RR_LD_QUADRATIC_TRI: case RR_LD_LOGARITHMIC: case RR_LD_EXPONENTIAL: nldc = 2; break;
        case RR_LD_NONLINEAR: nldc = 4; break;
        case RR_LD_LINEAR: nldc = 1; break;
        case RR_LD_GENERAL: nldc = base.ncoef; break;
        default: nldc = 0;
    }
    if (nldc > 0 && !ldc) return RR_EINVAL;
    pr.nldc = nldc;
    const int nparam = 7 + nldc;
    pr.params.assign((size_t)nk * nparam, 0.0);
    for (int p = 0; p < nk; ++p) {
        double* row = pr.params.data() + (size_t)p * nparam;
        row[1] = 1.0;            // P
        row[2] = kProbeA;        // a
        row[6] = k[p];
        for (int j = 0; j < nldc; ++j) row[7 + j] = ldc[j];
    }
    for (int p = 0; p < nk; ++p)
        for (int j = 0; j < kProbeG; ++j) {
            const double g = j == 0 ? 0.0 : std::fmod(j * 0.6180339887498949, 1.0) * 0.999;
            const double zz = g * (1.0 + k[p]);
            // circular, b = 0: z = a |sin(2 pi t / P)| near t = 0
            pr.times.push_back(std::asin(zz / kProbeA) / (2.0 * 3.14159265358979323846));
            pr.zs.push_back(zz);
            pr.ks.push_back(k[p]);
        }
    // the model evaluates its own z from the times; the exact integral is taken at those z
    // (both in FP64; they differ from zs by rounding only)
    cudaError_t e = cudaSetDevice(base.device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&pr.d_times, pr.times.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&pr.d_params, pr.params.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&pr.d_flux, (size_t)pr.npv * pr.npt * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&pr.d_z, pr.zs.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&pr.d_k, pr.ks.size() * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpy(pr.d_times, pr.times.data(), pr.times.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(pr.d_params, pr.params.data(), pr.params.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pr.d_z, pr.zs.data(), pr.zs.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pr.d_k, pr.ks.data(), pr.ks.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pr.release();
        return RR_ECUDA;
    }
    std::string err;
    auto cost = [](const Cand& q) { return (double)(kNzLadder[q.in] + kNzLadder[q.lb]) * kNgLadder[q.g]; };
    auto eval = [&](const Cand& q) { return cand_error(base, q, mu_tab, I_tab, ntab, pr, err); };
    // Greedy search: from a coarse grid, take the refinement (one ladder step of nzin, nzlimb or
    // ng, or a move of zcut) with the largest error reduction per unit of added cost until the
    // error meets the target; then coarsen any dimension that can be coarsened within the target.
    Cand cur{2, 2, 2, 2};
    double ecur = eval(cur);
    rr_status st = ecur < 0.0 ? RR_ECUDA : RR_OK;
    int steps = 0;
    while (st == RR_OK && ecur > target && steps++ < 120) {
        Cand best = cur;
        double best_score = -1e300, best_err = ecur;
        Cand moves[5] = {cur, cur, cur, cur, cur};
        moves[0].in++; moves[1].lb++; moves[2].g++; moves[3].zc--; moves[4].zc++;
        for (const Cand& m : moves) {
            if (m.in >= kNNz || m.lb >= kNNz || m.g >= kNNg || m.zc < 0 || m.zc >= kNZc) continue;
            const double em = eval(m);
            if (em < 0.0) continue;
            const double dc = std::log(cost(m) / cost(cur));
            const double de = std::log(std::max(ecur, 1e-300) / std::max(em, 1e-300));
            const double score = dc > 0.0 ? de / dc : (de > 0.0 ? 1e30 * de : -1e300);
            if (score > best_score) { best_score = score; best = m; best_err = em; }
        }
        if (best == cur) break;
        cur = best;
        ecur = best_err;
    }
    if (st == RR_OK && ecur <= target) {
        bool changed = true;
        while (changed) {
            changed = false;
            Cand moves[3] = {cur, cur, cur};
            moves[0].in--; moves[1].lb--; moves[2].g--;
            for (const Cand& m : moves) {
                if (m.in < 0 || m.lb < 0 || m.g < 0) continue;
                const double em = eval(m);
                if (em >= 0.0 && em <= target) { cur = m; ecur = em; changed = true; break; }
            }
        }
    }
    pr.release();
    if (st != RR_OK) return st;
    const rr_config found = cand_config(base, cur);
    cfg->zcut = found.zcut;
    cfg->nzin = found.nzin;
    cfg->nzlimb = found.nzlimb;
    cfg->ng = found.ng;
    if (max_err) *max_err = ecur;
    return ecur <= target ? RR_OK : RR_EDOMAIN;
}
