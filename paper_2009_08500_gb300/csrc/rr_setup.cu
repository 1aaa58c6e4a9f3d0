// Set-up kernels: LD profile bases and disk integrals, the (k, g) weight table
// with its projections, the direct model's per-call weight projections, the
// small-planet rows, and the per-call, per-parameter-vector records.
#include <cmath>

#include "rr_device.cuh"

namespace rr {

// ---------------------------------------------------------------------------
// LD profile bases at the bin means and their disk integrals (Sect. 3.2, Eq. 2)
//
// Every supported law is affine in its coefficients,
//   I(mu) = beta_0(mu) + sum_c u_c beta_c(mu),
// so the mean covered brightness w . l (Sect. 2) and I_star are the same
// combination of per-basis values.  Bases:
//   uniform                 beta_0 = 1
//   quadratic (and q1, q2)  beta_0 = 1, beta_1 = -(1 - mu), beta_2 = -(1 - mu)^2
//   nonlinear               beta_0 = 1, beta_n = -(1 - mu^(n/2)), n = 1..4
//   tabulated               one basis per passband: the table interpolated at mu
// I_star of a basis is 2 pi int_0^1 mu beta(mu) dmu: closed forms for the
// named bases, and for a table the exact integral of its piecewise-linear
// interpolant (constant outside the nodes).
// ---------------------------------------------------------------------------
__device__ double block_sum_f64(double v, double* red) {
    // deterministic tree over a power-of-two block
    const int t = threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) red[t] += red[t + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) rr_ld_basis_kernel(ModelParams mp, const double* __restrict__ mu,
                                                          int nz, const double* __restrict__ tab,
                                                          const int* __restrict__ tab_off,
                                                          double* __restrict__ basis,
                                                          double* __restrict__ istar) {
    __shared__ double red[256];
    const int b = blockIdx.x;
    double* out = basis + (size_t)b * nz;
    if (mp.ld_model != RR_LD_TABULATED) {
        for (int j = threadIdx.x; j < nz; j += blockDim.x) {
            const double m = mu[j];
            double v = 1.0;
            if (b > 0) {
                switch (mp.ld_model) {
                    case RR_LD_NONLINEAR: v = -(1.0 - pow(m, 0.5 * b)); break;
                    case RR_LD_GENERAL: v = -pow(1.0 - m, (double)b); break;
                    case RR_LD_LOGARITHMIC: v = b == 1 ? -(1.0 - m) : -m * log(m); break;
                    case RR_LD_EXPONENTIAL: v = b == 1 ? -(1.0 - m) : -1.0 / (1.0 - exp(m)); break;
                    default: v = (b == 1) ? -(1.0 - m) : -(1.0 - m) * (1.0 - m);   // linear, quadratic
                }
            }
            out[j] = v;
        }
        if (threadIdx.x == 0) {
            // 2 pi int_0^1 mu basis(mu) dmu, closed forms
            double I;
            if (b == 0)
                I = CUDART_PI;
            else if (mp.ld_model == RR_LD_NONLINEAR)
                I = -CUDART_PI * b / (b + 4.0);
            else if (mp.ld_model == RR_LD_GENERAL)
                I = -2.0 * CUDART_PI / ((b + 1.0) * (b + 2.0));
            else if (b == 1)
                I = -CUDART_PI / 3.0;
            else if (mp.ld_model == RR_LD_LOGARITHMIC)
                I = 2.0 * CUDART_PI / 9.0;
            else if (mp.ld_model == RR_LD_EXPONENTIAL)
                I = 2.0 * CUDART_PI * mp.exp_c;
            else
                I = -CUDART_PI / 6.0;
            istar[b] = I;
        }
        return;
    }
    // tabulated profile of passband b: nodes tmu[0..n), tI[0..n)
    const int o0 = tab_off[b], n = tab_off[b + 1] - o0;
    const double* tmu = tab + 2 * o0;
    const double* tI = tmu + n;
    for (int j = threadIdx.x; j < nz; j += blockDim.x) {
        const double m = mu[j];
        double v;
        if (m <= tmu[0]) {
            v = tI[0];
        } else if (m >= tmu[n - 1]) {
            v = tI[n - 1];
        } else {
            int lo = 0, hi = n - 1;  // tmu[lo] < m < tmu[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (tmu[mid] <= m) lo = mid; else hi = mid;
            }
            const double t = (m - tmu[lo]) / (tmu[lo + 1] - tmu[lo]);
            v = tI[lo] + t * (tI[lo + 1] - tI[lo]);
        }
        out[j] = v;
    }
    // 2 pi int mu I dmu of the interpolant: segment [m0, m1] contributes
    // (m1 - m0)/6 [I0 (2 m0 + m1) + I1 (m0 + 2 m1)]; constant ends
    double s = 0.0;
    for (int i = threadIdx.x; i < n - 1; i += blockDim.x) {
        const double m0 = tmu[i], m1 = tmu[i + 1];
        s += (m1 - m0) / 6.0 * (tI[i] * (2.0 * m0 + m1) + tI[i + 1] * (m0 + 2.0 * m1));
    }
    if (threadIdx.x == 0) s += 0.5 * tI[0] * tmu[0] * tmu[0] + 0.5 * tI[n - 1] * (1.0 - tmu[n - 1] * tmu[n - 1]);
    const double tot = block_sum_f64(s, red);
    if (threadIdx.x == 0) istar[b] = 2.0 * CUDART_PI * tot;
}

// ---------------------------------------------------------------------------
// Weight table (Sect. 2 below Eq. 4; Sect. 3.1, 3.1.2) and its projections
//   w[ik][ig][j] = (a(ze[j+1]) - a(ze[j])) / a(1),   c = g_ig (1 + k_ik)
//   T[b][ik][ig] = sum_j w[ik][ig][j] beta_b[j]
// a(r) = area common to the radius-r disk and the planet; at g = 1 (covered
// area 0) the row is its limit, all weight in the outermost annulus.
// One CTA per (ik, ig) row, FP64.
// ---------------------------------------------------------------------------
__device__ double lens_area_f64(double r, double k, double c) {
    if (c >= r + k) return 0.0;
    if (c <= fabs(r - k)) {
        const double m = r < k ? r : k;
        return CUDART_PI * m * m;
    }
    double h = ((r + k) - c) * (c + (r - k)) * (c - (r - k)) * (c + (r + k));
    h = h > 0.0 ? h : 0.0;
    const double K = sqrt(h);
    const double kap0 = atan2(K, c * c + (r * r - k * k));
    const double kap1 = atan2(K, c * c + (k * k - r * r));
    return r * r * kap0 + k * k * kap1 - 0.5 * K;
}

__global__ void __launch_bounds__(256) rr_weights_kernel(ModelParams mp, const double* __restrict__ ze,
                                                         int nz, const double* __restrict__ basis,
                                                         int write_w, double* __restrict__ w,
                                                         double* __restrict__ T64,
                                                         float* __restrict__ T32) {
    extern __shared__ double sh[];   // nz + 1 edge areas, then nz weights
    double* ea = sh;
    double* ws = sh + nz + 1;
    const int ig = blockIdx.x, ik = blockIdx.y;
    const double k = mp.k0 + ik * mp.dk;
    const double g = ig * (1.0 / (mp.ng - 1));
    const double c = g * (1.0 + k);
    const double atot = lens_area_f64(1.0, k, c);
    const bool limb = (c >= 1.0 + k) || !(atot > 0.0);
    if (!limb)
        for (int j = threadIdx.x; j <= nz; j += blockDim.x) ea[j] = lens_area_f64(ze[j], k, c);
    __syncthreads();
    double* wrow = w + ((size_t)ik * mp.ng + ig) * nz;
    for (int j = threadIdx.x; j < nz; j += blockDim.x) {
        const double v = limb ? (j == nz - 1 ? 1.0 : 0.0) : (ea[j + 1] - ea[j]) / atot;
        ws[j] = v;
        if (write_w) wrow[j] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = warp; b < mp.nbasis; b += blockDim.x >> 5) {
        const double* bb = basis + (size_t)b * nz;
        double s = 0.0;
        for (int j = lane; j < nz; j += 32) s += ws[j] * bb[j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const size_t idx = ((size_t)b * mp.nk + ik) * mp.ng + ig;
            T64[idx] = s;
            T32[idx] = (float)s;
        }
    }
}

// Differences of neighbouring g nodes of every projection, formed in FP64 and
// stored in FP32, so that in-cell slopes keep full FP32 relative precision.
__global__ void rr_diff_table_kernel(const double* __restrict__ T64, float* __restrict__ DT32, int ng,
                                     size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ig = (int)(i % ng);
    DT32[i] = ig < ng - 1 ? (float)(T64[i + 1] - T64[i]) : 0.0f;
}

// ---------------------------------------------------------------------------
// Direct model (Sect. 3.1.2 without the k interpolation): per call, the
// weights of every g node for each parameter vector's own k, projected onto
// the profile bases, T[b][row][ig] = sum_j w_j l_b[j] with
// w_j = (a(ze[j+1]) - a(ze[j])) / a(1), and for the adjoint their
// k-derivative at fixed g (c = g (1 + k)):
//   d a / d k |_g = d a / d k + g d a / d c,
//   d w_j / d k = (a'(ze[j+1]) - a'(ze[j])) / a(1) - w_j a'(1) / a(1).
// Only the edges inside the planet's band |c - k| < r < c + k need the lens
// formula: below it the disk is either wholly covered (c < k; those annuli
// come from running sums P[b][m] built once) or untouched, and above it the
// covered area is the whole planet, so those annuli get no weight.
// ---------------------------------------------------------------------------

// Small-angle part of a circular segment: phi(x) = x - sin x cos x =
// (2x - sin 2x) / 2 for x < 0.75, where that difference cancels, from the
// Taylor series of sin (t = 2x):
//   phi = t^3 / 12 (1 - t^2/20 + t^4/840 - t^6/60480 + t^8/6652800 - t^10/1037836800),
// whose first omitted term is below 1e-9 of the sum there.
__device__ __forceinline__ float seg_phi_small(float x) {
    const float t = 2.0f * x, t2 = t * t;
    float p = -1.0f / 1037836800.0f;
    p = fmaf(p, t2, 1.0f / 6652800.0f);
    p = fmaf(p, t2, -1.0f / 60480.0f);
    p = fmaf(p, t2, 1.0f / 840.0f);
    p = fmaf(p, t2, -1.0f / 20.0f);
    p = fmaf(p, t2, 1.0f);
    return t * t2 * (1.0f / 12.0f) * p;
}

// x + y - z where x + y is close to z: the rounding error of x + y is added
// back (error-free sum), so the result keeps its relative accuracy.
__device__ __forceinline__ float sum3_small(float x, float y, float z) {
    const float s = __fadd_rn(x, y);
    const float bb = __fsub_rn(s, x);
    const float e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(y, bb));
    return __fadd_rn(__fsub_rn(s, z), e);
}

// Area common to the radius-r disk and the planet (radius k, centre at
// distance c) with its partials d a / d k (the planet's rim inside the disk,
// 2 k kappa_1) and d a / d c (minus the common chord, -K / c); inv_c = 1 / c
// and inv4c2 = 1 / (4 c^2) are the caller's.
// FP32: the lens is the sum of two circular segments, r^2 phi(kappa_0) +
// k^2 phi(kappa_1), phi(x) = x - sin x cos x, each non-negative, so that the
// area keeps a few ulp of relative accuracy when k << r (the textbook form
// r^2 kappa_0 + k^2 kappa_1 - K / 2 cancels there).  With K = 2 c h (h the
// half chord) and x_0 = 2 c r cos kappa_0, x_1 = 2 c k cos kappa_1,
// r^2 sin kappa_0 cos kappa_0 = K x_0 / (4 c^2) and k^2 sin kappa_1 cos kappa_1
// = K x_1 / (4 c^2), so no sine is evaluated.  Heron's factors that vanish at
// a contact (r + k - c, c + k - r, c + r - k) are formed by sum3_small, and
// their signs decide disjoint and nested circles.  Each cosine numerator is
// a sum of a square and a difference of squares, taken with the pair of radii
// or distances that is closest (that difference is then exact): it vanishes
// without cancellation error when r ~ k at small c.
// far = (c >= 2 k): every edge that reaches the lens has c/2 <= r <= 2c, so
// r - c is exact and the factors need no compensation.
__device__ __forceinline__ float edge_area(float r, float k, float c, float inv_c, float inv4c2, bool far,
                                           float& dk, float& dc) {
    float p1, p2, s2;
    if (far) {
        const float dr = r - c;
        p1 = k + dr;                // r + k - c
        p2 = k - dr;                // c + k - r
        s2 = (c + r) - k;           // c + r - k >= 2 k here
    } else {
        p1 = sum3_small(r, k, c);
        p2 = sum3_small(c, k, r);
        s2 = sum3_small(c, r, k);
    }
    // branch-free: the lens formula is evaluated for every edge (finite or
    // NaN garbage outside the lens) and the closed forms of disjoint and
    // nested circles are selected afterwards
    const float s1 = r + k + c;
    const float P = (p1 * p2) * (s1 * s2);
    const float K = P > 1e-30f ? P * rsqrtf(P) : 0.0f;              // 2 c x (half chord)
    const float r2 = r * r, k2 = k * k, c2 = c * c;
    // 2 c r cos(kappa_0) = c^2 + r^2 - k^2, 2 c k cos(kappa_1) = c^2 + k^2 - r^2
    const float drk = r - k;
    const float x0 = fabsf(drk) < fabsf(c - k) ? fmaf(drk, r + k, c2) : fmaf(c - k, c + k, r2);
    const float x1 = fabsf(drk) < fabsf(c - r) ? fmaf(-drk, r + k, c2) : fmaf(c - r, c + r, k2);
    const float kap0 = atan2_upper(K, x0), kap1 = atan2_upper(K, x1);
    const float q = K * inv4c2;
    const float seg0 = kap0 < 0.75f ? r2 * seg_phi_small(kap0) : fmaf(r2, kap0, -q * x0);
    const float seg1 = kap1 < 0.75f ? k2 * seg_phi_small(kap1) : fmaf(k2, kap1, -q * x1);
    float a = seg0 + seg1;
    float ddk = 2.0f * k * kap1, ddc = -K * inv_c;
    if (s2 <= 0.0f) { a = CUDART_PI_F * r2; ddk = 0.0f; ddc = 0.0f; }                    // disk inside the planet
    if (p2 <= 0.0f) { a = CUDART_PI_F * k2; ddk = 2.0f * CUDART_PI_F * k; ddc = 0.0f; }  // planet inside the disk
    if (p1 <= 0.0f) { a = 0.0f; ddk = 0.0f; ddc = 0.0f; }                                 // disjoint
    dk = ddk;
    dc = ddc;
    return a;
}

// FP64: the textbook form (its cancellation for k << r costs r / k ulp of FP64).
__device__ __forceinline__ double edge_area(double r, double k, double c, double, double, bool, double& dk,
                                            double& dc) {
    if (c >= r + k) { dk = 0.0; dc = 0.0; return 0.0; }
    if (c <= fabs(r - k)) {
        dc = 0.0;
        if (k < r) { dk = 2.0 * CUDART_PI * k; return CUDART_PI * k * k; }
        dk = 0.0;
        return CUDART_PI * r * r;
    }
    double h = ((r + k) - c) * (c + (r - k)) * (c - (r - k)) * (c + (r + k));
    h = h > 0.0 ? h : 0.0;
    const double K = sqrt(h);
    const double kap0 = atan2(K, c * c + (r * r - k * k));
    const double kap1 = atan2(K, c * c + (k * k - r * r));
    dk = 2.0 * k * kap1;
    dc = -K / c;
    return r * r * kap0 + k * k * kap1 - 0.5 * K;
}

// Sums of products for the projections.  FP32: compensated (Kahan) sums
// kept as an unevaluated float pair (h, l), with rounding-exact intrinsics
// that the compiler does not contract, so that neighbouring g nodes differ by
// their true difference (the products' own roundings are far below the
// areas' few-ulp errors); FP64: plain sums.
template <typename A> struct DirSum;
template <> struct DirSum<float> {
    float h = 0.0f, l = 0.0f;
    __device__ __forceinline__ void add_prod(float x, float y) {
        const float y2 = __fadd_rn(__fmul_rn(x, y), l);
        const float t = __fadd_rn(h, y2);
        l = __fsub_rn(y2, __fsub_rn(t, h));
        h = t;
    }
    __device__ __forceinline__ void add(float h2, float l2) {
        const float s = __fadd_rn(h, h2);
        const float bb = __fsub_rn(s, h);
        const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
        h = s;
        l = __fadd_rn(l, __fadd_rn(l2, e));
    }
    // (h + l) / d as a normalised pair
    __device__ __forceinline__ void div(float d, float& qh, float& ql) const {
        const float q = __fdiv_rn(h, d);
        const float r = __fadd_rn(fmaf(-q, d, h), l);   // h - q d is exact
        const float q2 = __fdiv_rn(r, d);
        qh = __fadd_rn(q, q2);
        ql = __fsub_rn(q2, __fsub_rn(qh, q));
    }
};
template <> struct DirSum<double> {
    double h = 0.0;
    __device__ __forceinline__ void add_prod(double x, double y) { h = fma(x, y, h); }
    __device__ __forceinline__ void add(double h2, float) { h += h2; }
    __device__ __forceinline__ void div(double d, double& qh, float& ql) const { qh = h / d; ql = 0.0f; }
};

// Build time: FP32 copies of the edges and profiles, and the running sums
// P[b][m] = sum_{j<m} pi (ze[j+1] - ze[j]) (ze[j+1] + ze[j]) l_b[j] in FP64
// (stored as FP64 and as an FP32 pair).  One CTA per basis.
__global__ void rr_direct_prefix_kernel(ModelParams mp, const double* __restrict__ ze,
                                        const double* __restrict__ basis, float* __restrict__ zef,
                                        float* __restrict__ basisf, double* __restrict__ pre64,
                                        float* __restrict__ pref) {
    const int b = blockIdx.x, nz = mp.nz;
    const double* lb = basis + (size_t)b * nz;
    for (int j = threadIdx.x; j < nz; j += blockDim.x) basisf[(size_t)b * nz + j] = (float)lb[j];
    if (b == 0)
        for (int j = threadIdx.x; j <= nz; j += blockDim.x) zef[j] = (float)ze[j];
    if (threadIdx.x != 0) return;
    double* P = pre64 + (size_t)b * (nz + 1);
    float* Ph = pref + (size_t)b * (nz + 1);
    float* Pl = pref + (size_t)mp.nbasis * (nz + 1) + (size_t)b * (nz + 1);
    double acc = 0.0;
    P[0] = 0.0; Ph[0] = 0.0f; Pl[0] = 0.0f;
    for (int m = 0; m < nz; ++m) {
        acc += CUDART_PI * (ze[m + 1] - ze[m]) * (ze[m + 1] + ze[m]) * lb[m];
        P[m + 1] = acc;
        const float hi = (float)acc;
        Ph[m + 1] = hi;
        Pl[m + 1] = (float)(acc - (double)hi);
    }
}

// Per call: one thread per (row, g node), rows being (pv, k slot) pairs and
// the 32 lanes of a warp neighbouring g nodes of one row (their bands
// overlap, so the edges and profiles they read are shared through L1).  Each
// thread finds its band's edges by bisection, walks them once (the area of
// an edge serves both bins it bounds) and sums the bins' projections, bases
// kDirBases at a time.  The FP32 form takes c = g (1 + k) rounded to FP32 and
// adds the first-order effect of that rounding, (d a / d c) c_lo, to every
// area, so the nodes' positions are exact to FP32 working accuracy.
constexpr int kDirWarps = 8;
constexpr int kDirBases = 5;

template <typename A, bool P2>
__global__ void __launch_bounds__(kDirWarps * 32) rr_direct_table_kernel(
        ModelParams mp, const double* __restrict__ params, const A* __restrict__ ze,
        const A* __restrict__ basis, const double* __restrict__ basis64, const A* __restrict__ pre,
        const float* __restrict__ pre_lo, const A* __restrict__ lnmu, const double* __restrict__ mu64,
        DirectTables D, int grad) {
    const int ng = mp.ng, nz = mp.nz;
    const int wpr = (ng + 31) >> 5;   // warps per row
    const long long w = (long long)blockIdx.x * kDirWarps + (threadIdx.x >> 5);
    if (w >= (long long)D.nrows * wpr) return;
    const int row = (int)(w / wpr);
    const int ig = (int)(w - (long long)row * wpr) * 32 + (threadIdx.x & 31);
    if (ig >= ng) return;
    const int nkp = mp.chromatic ? mp.npb : 1;
    const int rpp = mp.shared ? 1 : nkp;   // rows per pv
    const int pv = row / rpp, slot = row - pv * rpp;
    double kd;
    if (mp.shared) {
        // shared weights: the mean of the pv's per-passband radius ratios (invalid if any is)
        kd = 0.0;
        bool ok = true;
        for (int j = 0; j < nkp; ++j) {
            const double kj = params[(size_t)pv * mp.nparam + 6 + j];
            ok = ok && kj > 0.0 && kj < 1.0;
            kd += kj;
        }
        kd = ok ? kd / nkp : -1.0;
    } else {
        kd = params[(size_t)pv * mp.nparam + 6 + slot];
    }
    // bases of the row: every named basis; tabulated, the passband's own
    // profile when the row is one passband's, else every passband's.  The
    // power-2 laws: column 0 the constant, then per passband q the row serves
    // mu^alpha_q and mu^alpha_q ln mu (the latter for the adjoint)
    constexpr bool p2 = P2;                          // a power-2 law (instantiated apart)
    const bool p2own = mp.chromatic && !mp.shared;   // a power-2 row serves its own passband only
    int b_lo = 0, b_hi = p2 ? (p2own ? 3 : 1 + 2 * mp.npb) : mp.nbasis;
    if (mp.ld_model == RR_LD_TABULATED && mp.chromatic && !mp.shared) { b_lo = slot; b_hi = slot + 1; }
    // power-2 exponent of a column's passband
    auto p2_alpha = [&](int b) -> double {
        const int pb = p2own ? slot : (b - 1) >> 1;
        const double* cf = params + (size_t)pv * mp.nparam + 6 + nkp + pb * 2;
        if (mp.ld_model == RR_LD_POWER2) return cf[1];
        const double cc = 1.0 - cf[0] + cf[1];
        return cc > 0.0 && cf[1] > 0.0 ? log2(cc / cf[1]) : 1.0;   // invalid: flagged by the set-up kernel
    };
    A* Thi = reinterpret_cast<A*>(D.hi);
    A* Tdk = reinterpret_cast<A*>(D.dk);
    const size_t bstride = (size_t)D.nrows * ng;
    const size_t o = (size_t)row * ng + ig;
    // rows of small-planet passbands are not read (their rows come from the profile directly)
    const bool valid = kd > 0.0 && kd < 1.0 && !(kd < mp.k_small);
    const A k = (A)kd;
    const double gd = ig * mp.dg;
    const double cd = gd * (1.0 + (double)k);
    const A c = (A)cd, c_lo = (A)(cd - (double)c), g = (A)gd;
    const A inv_c = A(1) / c, inv4c2 = A(0.25) * inv_c * inv_c;
    const bool far = c >= A(2) * k;
    A tk = 0, tc = 0;
    A atot = valid ? edge_area(A(1), k, c, inv_c, inv4c2, far, tk, tc) : A(0);
    atot += tc * c_lo;
    if (!valid || ig == ng - 1 || !(atot > A(0))) {
        // g = 1 (no covered area): the row's limit, all weight in the outermost
        // annulus; rows of invalid k are zero (never read)
        for (int b = b_lo; b < b_hi; ++b) {
            double v = 0.0;
            if (valid) {
                if (!p2 || b == 0) {
                    v = p2 ? 1.0 : basis64[(size_t)b * nz + nz - 1];
                } else {
                    const double lm = log(mu64[nz - 1]);
                    v = exp(p2_alpha(b) * lm) * (((b - 1) & 1) ? lm : 1.0);
                }
            }
            Thi[b * bstride + o] = (A)v;
            if (D.lo) D.lo[b * bstride + o] = (float)(v - (double)(A)v);
            if (grad) Tdk[b * bstride + o] = A(0);
        }
        return;
    }
    const A lo_r = c > k ? c - k : k - c, hi_r = c + k;
    // e0: last edge with ze <= |c - k| (ze[0] = 0); e1: first edge with ze >= c + k, else nz
    int L = 0, H = nz + 1;
    while (H - L > 1) {
        const int m = (L + H) >> 1;
        if (ze[m] <= lo_r) L = m; else H = m;
    }
    int e0 = L;
    L = e0; H = nz;
    while (H - L > 1) {
        const int m = (L + H) >> 1;
        if (ze[m] >= hi_r) H = m; else L = m;
    }
    const int e1 = H;
    // the disk's centre is covered: annuli below e0 count whole, from the running sums; the
    // power-2 profiles differ per pv, so there the walk starts at the centre instead
    const bool centre = c < k && !p2;
    if (c < k && p2) e0 = 0;
    const A dtot = tk + g * tc;
    for (int bg = b_lo; bg < b_hi; bg += kDirBases) {
        const int nb = min(kDirBases, b_hi - bg);
        DirSum<A> S[kDirBases];
        A dS[kDirBases];
        #pragma unroll
        for (int q = 0; q < kDirBases; ++q) dS[q] = A(0);
        // power-2 columns: exponent and kind (0: 1, 1: mu^alpha, 2: mu^alpha ln mu)
        A alpha[kDirBases];
        int kind[kDirBases];
        #pragma unroll
        for (int q = 0; q < kDirBases; ++q) {
            const int b = bg + q;
            kind[q] = (!p2 || b == 0 || q >= nb) ? 0 : 1 + ((b - 1) & 1);
            alpha[q] = kind[q] ? (A)p2_alpha(b) : A(0);
        }
        A ak, ac;
        A a0 = edge_area(ze[e0], k, c, inv_c, inv4c2, far, ak, ac);
        a0 += ac * c_lo;
        A da0 = ak + g * ac;
        #pragma unroll 1
        for (int j = e0; j < e1; ++j) {
            A a1 = edge_area(ze[j + 1], k, c, inv_c, inv4c2, far, ak, ac);
            a1 += ac * c_lo;
            const A da1 = ak + g * ac;
            const A d = a1 - a0, dd = da1 - da0;
            #pragma unroll
            for (int q = 0; q < kDirBases; ++q) {
                if (q < nb) {
                    A lbj;
                    if (!p2) {
                        lbj = basis[(size_t)(bg + q) * nz + j];
                    } else if (kind[q] == 0) {
                        lbj = A(1);
                    } else {
                        const A lm = lnmu[j];
                        lbj = exp(alpha[q] * lm);
                        if (kind[q] == 2) lbj *= lm;
                    }
                    S[q].add_prod(d, lbj);
                    if (grad) dS[q] += dd * lbj;
                }
            }
            a0 = a1;
            da0 = da1;
        }
        #pragma unroll
        for (int q = 0; q < kDirBases; ++q) {
            if (q >= nb) continue;
            const int b = bg + q;
            if (centre) S[q].add(pre[(size_t)b * (nz + 1) + e0], pre_lo ? pre_lo[(size_t)b * (nz + 1) + e0] : 0.0f);
            A th;
            float tl;
            S[q].div(atot, th, tl);
            Thi[b * bstride + o] = th;
            if (D.lo) D.lo[b * bstride + o] = tl;
            if (grad) Tdk[b * bstride + o] = (dS[q] - th * dtot) / atot;
        }
    }
}

// ---------------------------------------------------------------------------
// Per-call parameter-vector records.  Validation, orbit constants and
// windows in FP64 (rounded to R); profile rows in R (FP32 in the mixed form).
//
// Validates the row (the RR_PV_* bits), derives the orbit constants of the
// offset-from-conjunction form (see PvHead), the transit window, and for
// every passband the profile row interpolated in k (Sect. 3.1.2, the
// (1 - ak) dot(w[ik], l) + ak dot(w[ik+1], l) of the paper, evaluated as the
// same combination of the precomputed projections T) divided by I_star.
// With `grad`, each passband also gets the differences of neighbouring row
// entries (in-cell slopes), d(row)/dk and, per LD coefficient c,
// Q_c = (T_c - row I_star_c) / I_star, the derivative of row / I_star
// with respect to u_c.
//
// Transit window: z >= r |cos(w + f)| >= a (1 - e) |cos(w + f)|, so a
// transit needs |cos(w + f)| < q = (1 + k) / (a (1 - e)) with the planet in
// front, i.e. f within asin(q) (pi/2 if q >= 1) of the conjunction anomaly
// f0 = pi/2 - w.  Mapped to mean anomaly this gives |M - M0| <= win.
// ---------------------------------------------------------------------------
__device__ double wrap_2pi(double x) {
    const double tp = 2.0 * CUDART_PI;
    x = fmod(x, tp);
    return x < 0.0 ? x + tp : x;
}

__device__ double mean_anomaly_of_true(double f, double e) {
    const double E = 2.0 * atan2(sqrt(1.0 - e) * sin(0.5 * f), sqrt(1.0 + e) * cos(0.5 * f));
    return E - e * sin(E);
}

// Math in the record's precision R (FP32 scalar set-up for the mixed form;
// its window margins absorb FP32 rounding).
__device__ __forceinline__ float r_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double r_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float r_asin(float x) { return asinf(x); }
__device__ __forceinline__ double r_asin(double x) { return asin(x); }
__device__ __forceinline__ float r_fmod(float x, float y) { return fmodf(x, y); }
__device__ __forceinline__ double r_fmod(double x, double y) { return fmod(x, y); }
__device__ __forceinline__ float r_max(float x, float y) { return fmaxf(x, y); }
__device__ __forceinline__ double r_max(double x, double y) { return fmax(x, y); }

template <typename R>
__device__ R wrap_2pi_r(R x) {
    const R tp = R(2) * Tr<R>::pi();
    x = r_fmod(x, tp);
    return x < R(0) ? x + tp : x;
}

template <typename R>
__device__ R mean_anomaly_of_true_r(R f, R e) {
    R sh, ch;
    d_sincos(R(0.5) * f, &sh, &ch);
    const R E = R(2) * r_atan2(d_sqrt(R(1) - e) * sh, d_sqrt(R(1) + e) * ch);
    R sE, cE;
    d_sincos(E, &sE, &cE);
    return E - e * sE;
}

// Small-planet approximation (Sect. 3.4): the rows of the (pv, passband)
// pairs whose weights' radius ratio k_w is below k_small, written by the
// set-up kernel in place of the interpolated rows.  At g node i the row holds
// the profile at the planet's centre, mu = sqrt(1 - min(c, 1)^2) with
// c = g_i (1 + k_w), clamped below to mu_min, divided by I_star; with the
// adjoint also the in-cell difference, d/dk (through mu; 0 where clamped) and
// the coefficient rows (basis_c - row I_star_c) / I_star.
struct SmallPlanetRow {
    double kw;
    double ud[5];   // weights of the bases: 1, then the coefficients
    int b0, nc;
    // FP32 copies for the FP32 rows, converted once per row (FP64 issues at a small
    // fraction of the FP32 rate on GB300, conversions included)
    float kw1f;     // 1 + kw
    float udf[5];
    float mu_minf, dgf;
};

__device__ double small_planet_node(const ModelParams& mp, const SmallPlanetRow& sp, const double* tab,
                                    const int* tab_off, int i, double* vb, double& dk) {
    const double gi = i * mp.dg, cc = gi * (1.0 + sp.kw);
    const double cm = fmin(cc, 1.0);
    const double m0 = sqrt(fmax(1.0 - cm * cm, 0.0));
    const bool free = cc < 1.0 && m0 > mp.mu_min;
    const double m = free ? m0 : mp.mu_min;
    const double dmdk = free ? -cc * gi / m : 0.0;
    double v = 0.0, dv = 0.0;
    for (int c = 0; c <= sp.nc; ++c) {
        double dd;
        const double bv = ld_basis_mu(mp, sp.b0 + c, m, tab, tab_off, dd);
        vb[c] = bv;
        v += sp.ud[c] * bv;
        dv += sp.ud[c] * dd;
    }
    dk = dv * dmdk;
    return v;
}

// FP32 twins of ld_basis_mu and small_planet_node, for rows stored in FP32 (the mixed form):
// FP64 issues at a small fraction of the FP32 rate on GB300, and the rows keep 24 bits.
// 1 - c^2 as (1 - c)(1 + c), and the exponential law's 1 - e^mu as -expm1(mu), keep the
// relative precision at the limb.
__device__ __forceinline__ float ld_basis_mu_f(const ModelParams& mp, int b, float m, const double* __restrict__ tab,
                                               const int* __restrict__ tab_off, float& d) {
    if (mp.ld_model == RR_LD_TABULATED) {
        const int o0 = tab_off[b], n = tab_off[b + 1] - o0;
        const double* tmu = tab + 2 * o0;
        const double* tI = tmu + n;
        if (m < (float)tmu[0]) { d = 0.0f; return (float)tI[0]; }
        if (m >= (float)tmu[n - 1]) { d = 0.0f; return (float)tI[n - 1]; }
        int lo = 0, hi = n - 1;   // tmu[lo] <= m < tmu[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if ((float)tmu[mid] <= m) lo = mid; else hi = mid;
        }
        const float m0 = (float)tmu[lo], i0 = (float)tI[lo];
        d = ((float)tI[lo + 1] - i0) / ((float)tmu[lo + 1] - m0);
        return i0 + d * (m - m0);
    }
    if (b == 0) { d = 0.0f; return 1.0f; }
    const float q = 1.0f - m;
    switch (mp.ld_model) {
        case RR_LD_NONLINEAR: {
            const float sq = sqrtf(m);
            const float p = b == 1 ? sq : (b == 2 ? m : (b == 3 ? m * sq : m * m));
            d = b == 1 ? 0.5f / sq : (b == 2 ? 1.0f : (b == 3 ? 1.5f * sq : 2.0f * m));
            return -(1.0f - p);
        }
        case RR_LD_GENERAL: {
            float p = 1.0f;
            for (int j = 1; j < b; ++j) p *= q;
            d = b * p;
            return -p * q;
        }
        case RR_LD_LOGARITHMIC:
            if (b == 1) { d = 1.0f; return -q; }
            d = -(logf(m) + 1.0f);
            return -m * logf(m);
        case RR_LD_EXPONENTIAL:
            if (b == 1) { d = 1.0f; return -q; }
            {
                const float em1 = expm1f(m), r = -1.0f / em1;   // 1 / (1 - e^mu)
                d = -(em1 + 1.0f) * r * r;
                return -r;
            }
        default:
            if (b == 1) { d = 1.0f; return -q; }
            d = 2.0f * q;
            return -q * q;
    }
}

__device__ __forceinline__ float small_planet_node_f(const ModelParams& mp, const SmallPlanetRow& sp,
                                                     const double* tab, const int* tab_off, int i, float* vb,
                                                     float& dk) {
    const float gi = (float)i * sp.dgf, cc = gi * sp.kw1f;
    const float cm = fminf(cc, 1.0f);
    const float m0 = sqrtf(fmaxf((1.0f - cm) * (1.0f + cm), 0.0f));
    const bool free = cc < 1.0f && m0 > sp.mu_minf;
    const float m = free ? m0 : sp.mu_minf;
    const float dmdk = free ? -cc * gi / m : 0.0f;
    float v = 0.0f, dv = 0.0f;
    for (int c = 0; c <= sp.nc; ++c) {
        float dd;
        const float bv = ld_basis_mu_f(mp, sp.b0 + c, m, tab, tab_off, dd);
        vb[c] = bv;
        v += sp.udf[c] * bv;
        dv += sp.udf[c] * dd;
    }
    dk = dv * dmdk;
    return v;
}

// A small-planet node in the arithmetic of the rows: FP32 for the mixed form, FP64 otherwise.
template <typename R>
__device__ __forceinline__ R small_planet_node_r(const ModelParams& mp, const SmallPlanetRow& sp, int i, R* vb, R& dk) {
    if constexpr (sizeof(R) == sizeof(float)) {
        return small_planet_node_f(mp, sp, mp.tab, mp.tab_off, i, vb, dk);
    } else {
        return small_planet_node(mp, sp, mp.tab, mp.tab_off, i, vb, dk);
    }
}

// Pvs per CTA of the set-up kernel: few, so that the launch has several
// CTAs per SM and the per-pv scalar chains of many CTAs overlap; the rows
// and windows are spread over the whole CTA.  At most N; fewer with more
// passbands (each pv then has that many rows), so that the launch spreads
// over the SMs (8 passbands: 2 per CTA, measured 49.7 -> 39.6 us for 2,048
// pvs; 1 per CTA was slower again).
template <typename R> struct SetupPvs { static constexpr int N = 8; };
__host__ __device__ inline int setup_pvs_per_cta(int npb) { return npb >= 4 ? 2 : (npb >= 2 ? 4 : 8); }

template <typename R>
__global__ void __launch_bounds__(256, 4) rr_pv_setup_kernel(ModelParams mp, PbParams pbp,
                                                          const double* __restrict__ params, int npv,
                                                          const R* __restrict__ T, const float* __restrict__ DT,
                                                          const double* __restrict__ istar,
                                                          RecLayout L, int grad, char* __restrict__ records,
                                                          int32_t* __restrict__ pv_status, DirectTables D,
                                                          PointsArgs pa) {
    if ((int)blockIdx.x < pa.npoints) {
        // the per-time inputs of the FP32 kernels, two 128-time groups per CTA, in the same
        // launch as the per-pv set-up (the two are independent); these short CTAs come first
        __shared__ float pred[2][4][kWarpPts / 32];
        __shared__ int predf[2][kWarpPts / 32];
        __shared__ int ss_s[RR_MAX_PB];
        const int half = threadIdx.x / kWarpPts;
        for (int j = threadIdx.x; j < mp.npb; j += blockDim.x) ss_s[j] = pbp.ss[j];
        __syncthreads();
        points_group(pa.times, pa.pb_index, pa.npt, mp.npb, pa.dt, pa.pbw, pa.grp, (int)blockIdx.x * 2 + half,
                     pa.ngroups, threadIdx.x % kWarpPts, pred[half], predf[half], mp.npb > 1 ? ss_s : nullptr);
        return;
    }
    const int sblock = (int)blockIdx.x - pa.npoints;   // this CTA's index among the set-up CTAs
    constexpr int NP = SetupPvs<R>::N;
    __shared__ R u_s[NP][RR_MAX_PB][4];
    __shared__ R invIs_s[NP][RR_MAX_PB];
    __shared__ R ak_s[NP][RR_MAX_PB];
    __shared__ int ik_s[NP][RR_MAX_PB];       // k cell or direct row; -1: small-planet approximation
                                              // (ak_s then holds the weights' radius ratio)
    __shared__ int st_s[NP];       // validity after (1): LD coefficients, I_star, k
    __shared__ int st2_s[NP];      // full validity after (2a)
    __shared__ int rows_next;
    __shared__ int wmax_s[NP];     // largest point window over the passbands (float bits, -1 = none)
    __shared__ int flags_s[NP];
    __shared__ R orb_s[NP][7];     // a, b, e, f0, M0, n, z at conjunction (b r0 / a)
    const int ppc = setup_pvs_per_cta(mp.npb);
    const int pv0 = sblock * ppc;
    const int nloc = min(ppc, npv - pv0);
    const int nkp = mp.chromatic ? mp.npb : 1;
    const int tid = threadIdx.x;
    if (tid < NP) st_s[tid] = 0;
    if (tid == 0) rows_next = 0;
    __syncthreads();

    // (1) per (pv, passband): validity, LD coefficients, I_star, k cell
    for (int t = tid; t < nloc * mp.npb; t += blockDim.x) {
        const int lp = t / mp.npb, pb = t % mp.npb;
        const double* row = params + (size_t)(pv0 + lp) * mp.nparam;
        int st = 0;
        const double* c = row + 6 + nkp + pb * mp.nldc;
        double u[4] = {0, 0, 0, 0};
        if (mp.ld_model == RR_LD_QUADRATIC_TRI) {
            const double q1 = c[0], q2 = c[1];
            if (!(q1 >= 0.0 && q1 <= 1.0 && q2 >= 0.0 && q2 <= 1.0)) st |= RR_PV_LD_INVALID;
            const double sq = sqrt(fmax(q1, 0.0));
            u[0] = 2.0 * sq * q2;
            u[1] = sq * (1.0 - 2.0 * q2);
        } else if (mp.ld_model == RR_LD_POWER2 || mp.ld_model == RR_LD_POWER2_PM) {
            // (c, alpha); from (h1, h2): c = 1 - h1 + h2, alpha = log2(c / h2)
            const double cc = mp.ld_model == RR_LD_POWER2 ? c[0] : 1.0 - c[0] + c[1];
            const double al = mp.ld_model == RR_LD_POWER2 ? c[1] : (cc > 0.0 && c[1] > 0.0 ? log2(cc / c[1]) : -1.0);
            if (!(al > 0.0)) st |= RR_PV_LD_INVALID;
            u[0] = cc;
            u[1] = al;
        } else {
            for (int j = 0; j < mp.nldc; ++j) u[j] = c[j];
        }
        double Is;
        if (mp.ld_model == RR_LD_TABULATED) {
            Is = istar[pb];
        } else if (mp.ld_model == RR_LD_POWER2 || mp.ld_model == RR_LD_POWER2_PM) {
            Is = CUDART_PI * (1.0 - u[0] * u[1] / (u[1] + 2.0));
        } else {
            Is = istar[0];
            for (int j = 0; j < mp.nldc; ++j) Is += u[j] * istar[1 + j];
        }
        if (!(Is > 0.0)) st |= RR_PV_LD_INVALID;
        const double k = row[6 + (mp.chromatic ? pb : 0)];
        // the weights' radius ratio: the passband's own, or the mean over the pv's passbands
        double kw = k;
        if (mp.shared) {
            kw = 0.0;
            for (int j = 0; j < nkp; ++j) kw += row[6 + j];
            kw /= nkp;
        }
        // every radius ratio in (0, 1); the interpolated model also needs the weights' radius
        // ratio inside the k table unless the small-planet approximation replaces the weights
        const bool small = kw < mp.k_small;
        if (!(k > 0.0 && k < 1.0)) st |= RR_PV_K_RANGE;
        else if (!mp.direct && !small && !(kw >= mp.k0 && kw <= mp.k1)) st |= RR_PV_K_RANGE;
        int ik;
        double ak;
        if (small) {
            ik = -1;
            ak = kw;   // the small-planet rows' radius ratio
        } else if (mp.direct) {
            // the row of this (pv, k slot) in the per-call projections
            ik = mp.shared ? pv0 + lp : (pv0 + lp) * nkp + (mp.chromatic ? pb : 0);
            ak = 0.0;
        } else {
            const double x = (kw - mp.k0) / mp.dk;
            ik = (int)floor(x);
            ik = ik < 0 ? 0 : (ik > mp.nk - 2 ? mp.nk - 2 : ik);
            ak = x - ik;
        }
        for (int j = 0; j < 4; ++j) u_s[lp][pb][j] = (R)u[j];
        invIs_s[lp][pb] = (R)(1.0 / Is);
        ik_s[lp][pb] = ik;
        ak_s[lp][pb] = (R)ak;
        if (st) atomicOr(&st_s[lp], st);
    }
    __syncthreads();

    // From here warp 0 computes the orbit constants and transit windows
    // (2a-2c) while the other warps build the profile rows (3), which need only
    // (1); warp 0 joins the rows when it is done.
    const int warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
    // (2a) per pv, one lane each: orbit constants
    if (tid < nloc) {
        const int pv = pv0 + tid;
        const double* row = params + (size_t)pv * mp.nparam;
        char* rec = records + (size_t)pv * L.head_bytes;
        PvHead<R>* H = reinterpret_cast<PvHead<R>*>(rec);
        const double T0 = row[0], P = row[1], ad = row[2], bd = row[3], ed = row[4], wd = row[5];
        bool finite = true;
        for (int j = 0; j < mp.nparam; ++j) finite = finite && isfinite(row[j]);
        int st = st_s[tid];
        if (!finite) {
            st = RR_PV_NONFINITE;
        } else {
            if (!(ed >= 0.0 && ed < 1.0)) st |= RR_PV_E_RANGE;
            if (!(P > 0.0)) st |= RR_PV_P_RANGE;
            if (!(ad > 1.0)) st |= RR_PV_A_RANGE;
            if (!(bd >= 0.0 && bd <= ad)) st |= RR_PV_B_RANGE;
        }
        st2_s[tid] = st;
        H->status = st;
        if (pv_status) pv_status[pv] = st;
        H->flags = 0;
        H->wmax_c = 0.0f;
        H->pad3 = 0;
        H->pad4 = 0;
        wmax_s[tid] = __float_as_int(-1.0f);
        flags_s[tid] = 0;
        if (st == 0) {
            const R a = (R)ad, b = (R)bd, e = (R)ed;
            const R pi = Tr<R>::pi();
            const R f0 = R(0.5) * pi - (R)wd;
            // One FP64 sincos: the conjunction's true anomaly f0 = pi/2 - w has
            // sin f0 = cos w and cos f0 = sin w, and its eccentric anomaly E0
            // cos E0 = (e + cos f0) / (1 + e cos f0), sin E0 = sqrt(1 - e^2) sin f0 / (1 + e cos f0),
            // with 1 - e cos E0 = (1 - e^2) / (1 + e cos f0) (no cancellation).
            double swd, cwd;
            sincos(wd, &swd, &cwd);
            const double sed = sqrt(1.0 - ed * ed);
            const double qd = 1.0 / (1.0 + ed * swd);
            const double cE0d = (ed + swd) * qd, sE0d = sed * cwd * qd, den0d = (1.0 - ed * ed) * qd;
            const R sE0 = (R)sE0d, cE0 = (R)cE0d, sw = (R)swd, cw = (R)cwd;
            const R se = (R)sed;
            const R den0 = (R)den0d;
            // M0 serves the (FP32) transit windows only
            const float M0 = atan2f((float)sE0d, (float)cE0d) - (float)ed * (float)sE0d;
            const double invP = 1.0 / P;
            const R n = (R)(2.0 * CUDART_PI * invP);
            R ax1, ax2, ay1, ay2, rho0;
            if (ed == 0.0) {
                ax1 = R(0); ax2 = R(-1); ay1 = R(-1); ay2 = R(0); rho0 = R(1);
            } else {
                ax1 = -cw * cE0 + sw * se * sE0;
                ax2 = -cw * sE0 - sw * se * cE0;
                ay1 = -sw * cE0 - cw * se * sE0;
                ay2 = -sw * sE0 + cw * se * cE0;
                rho0 = den0;
            }
            H->T0 = T0; H->P = P; H->invP = invP;
            // FP64 Kepler constants (the FP64 form, and e > kESwitch in the mixed form)
            H->ecE0d = ed * cE0d;
            H->esE0d = ed * sE0d;
            H->inv_den0d = (1.0 + ed * swd) / (1.0 - ed * ed);
            {
                // third-order inversion of d0 x + (e sin E0 / 2) x^2 + (e cos E0 / 6) x^3 = dM
                const float sy = (float)(e * sE0 / den0), cy = (float)(e * cE0 / den0);
                H->kep2 = -0.5f * sy;
                H->kep3 = 0.5f * sy * sy - cy * (1.0f / 6.0f);
                const float ef = (float)e;
                H->kepC = fmaxf(0.5f * ef / (1.0f - fminf(ef, 0.999f)), 0.5f);
            }
            H->a = a; H->b = b; H->a2 = a * a; H->b2 = b * b;
            H->e = e; H->ecE0 = (R)(ed * cE0d); H->esE0 = (R)(ed * sE0d); H->inv_den0 = (R)H->inv_den0d;
            H->ax1 = ax1; H->ax2 = ax2; H->ay1 = ay1; H->ay2 = ay2;
            H->rho0 = rho0; H->n = n;
            const float Bh = (float)invP;
            H->Bh = (R)Bh; H->Bl = (R)(float)(invP - (double)Bh);
            H->dM0de = -den0 * sE0 / (R(1) - e * e) - sE0;
            H->dM0dw = -den0 * den0 / se;
            H->se = se; H->cw = cw; H->sw = sw; H->cE0 = cE0; H->sE0 = sE0; H->inv_se = R(1) / se;
            int flags = 0;
            if (ed == 0.0) flags |= kPvCircular;
            if (ed > kESwitch) flags |= kPvKepler64;
            flags_s[tid] = flags;
            orb_s[tid][0] = a; orb_s[tid][1] = b; orb_s[tid][2] = e; orb_s[tid][3] = f0;
            orb_s[tid][4] = M0; orb_s[tid][5] = n; orb_s[tid][6] = b * rho0;
        }
    }
    __syncwarp();

    // (2b) per (pv, passband), one lane each: transit window
    for (int t = lane; t < nloc * mp.npb; t += 32) {
        const int lp = t / mp.npb, pb = t % mp.npb;
        if (st2_s[lp] != 0) continue;
        const int pv = pv0 + lp;
        const double* row = params + (size_t)pv * mp.nparam;
        PvPb<R>* PB = reinterpret_cast<PvPb<R>*>(records + (size_t)pv * L.head_bytes + L.off_pb);
        // the window is a conservative bound with explicit margins: FP32 in both
        // forms (dependent FP64 transcendentals are slow on GB300)
        using W = float;
        const W a = (W)orb_s[lp][0], b = (W)orb_s[lp][1], e = (W)orb_s[lp][2], f0 = (W)orb_s[lp][3];
        const W M0 = (W)orb_s[lp][4], n = (W)orb_s[lp][5];
        const W pi = Tr<W>::pi();
        const W ra = a * (W(1) - e);
        // conjunction anomaly wrapped to (-pi, pi] (periastron at 0)
        const W fc = f0 - W(2) * pi * floorf((f0 + pi) / (W(2) * pi));
        const R k = (R)row[6 + (mp.chromatic ? pb : 0)];
        const W kw = (W)k;
        // Transit window in true anomaly, |f - f0| <= d.  A transit needs
        // X^2 + Y^2 < (1 + k)^2 with |X| = r |sin(f - f0)|, |Y| = r cos(f - f0) b / a
        // (planet in front: |f - f0| < pi/2).  Start from r >= a (1 - e); then, with
        // r_min and the smallest |Y| over the current window, |sin(f - f0)| <=
        // sqrt((1 + k)^2 - Y_min^2) / r_min gives a window that still holds every
        // transit point.  Safety factors absorb the FP32 rounding.
        const W lim = W(1) + kw;
        const W q = lim / ra;
        W d = q >= W(1) ? W(0.5) * pi : r_asin(q);
        bool none = false;
        for (int it = 0; it < 5 && !none; ++it) {
            const W mc = fabsf(fc) <= d ? W(1) : r_max(cosf(fc - d), cosf(fc + d));
            const W rmin = a * (W(1) - e * e) / (W(1) + e * mc);
            const W ymin = rmin * cosf(d) * (b / a) * W(1 - 4e-6);
            const W x2 = lim * lim * W(1 + 4e-6) - ymin * ymin;
            if (!(x2 > W(0))) { none = true; break; }
            const W sx = d_sqrt(x2) / rmin;
            const W dn = sx >= W(1) ? W(0.5) * pi : r_asin(sx);
            d = dn < d ? dn : d;
        }
        PB[pb].k = k;
        PB[pb].inv1pk = R(1) / (R(1) + k);
        PB[pb].pad[0] = PB[pb].pad[1] = 0.0f;
        // grazing: the planet never wholly on the disk, every in-transit sample near the
        // outer contact (where the adjoint's z rounding is amplified): a wider band
        PB[pb].cband = (float)orb_s[lp][6] > 1.0f - (float)kw ? kContactBandGrazing : kContactBand;
        if (none) {            // the orbit never brings the planet over the disk
            PB[pb].win_s = R(-1);
            PB[pb].win_p = R(-1);
            PB[pb].win_pc = -1.0f;
            continue;
        }
        const W hi = wrap_2pi_r(mean_anomaly_of_true_r(f0 + d, e) - M0);
        const W lo = wrap_2pi_r(M0 - mean_anomaly_of_true_r(f0 - d, e));
        W win = r_max(hi, lo);
        win += W(1e-5) * (W(1) + win);
        const int ss = pbp.ss[pb];
        const W half = W(0.5) * (W)pbp.exptime[pb] * (W(1) - W(1) / W(ss));
        W winp = win + n * (ss > 1 ? half : W(0)) * W(1.000001);
        if (win >= pi) { win = W(1e30); atomicOr(&flags_s[lp], (int)kPvNoWindow); }
        if (winp >= pi) winp = W(1e30);
        PB[pb].win_s = (R)win;
        PB[pb].win_p = (R)winp;
        const float wc = winp * (W(0.5) / pi);
        PB[pb].win_pc = wc;
        atomicMax(&wmax_s[lp], __float_as_int(wc));   // non-negative floats order as their bits
    }
    __syncwarp();

    // (2c) the per-pv summary of the windows
    if (tid < nloc && st2_s[tid] == 0) {
        PvHead<R>* H = reinterpret_cast<PvHead<R>*>(records + (size_t)(pv0 + tid) * L.head_bytes);
        H->wmax_c = __int_as_float(wmax_s[tid]);
        H->flags = flags_s[tid];
    }
    }   // warp 0

    if (warp == 1 && L.orb_off >= 0 && lane < nloc) {
        // the orbit constants and radius ratios of the mixed adjoint's contact refinement as
        // float pairs (FP64 arithmetic: here, beside warp 0's orbit and window work, rather than
        // on its path; pvs that (2a) finds invalid get values that are never read)
        const int pv = pv0 + lane;
        const double* row = params + (size_t)pv * mp.nparam;
        const double ad = row[2], bd = row[3], ed = row[4], wd = row[5];
        double swd, cwd;
        sincos(wd, &swd, &cwd);
        const double sed = sqrt(fmax(1.0 - ed * ed, 0.0));
        const double qd = 1.0 / (1.0 + ed * swd);
        const double cE0d = (ed + swd) * qd, sE0d = sed * cwd * qd, den0d = (1.0 - ed * ed) * qd;
        char* blk = records + (size_t)pv * L.head_bytes + L.orb_off;
        PvOrbitFF* O = reinterpret_cast<PvOrbitFF*>(blk);
        auto split = [](float* d, double v) {
            d[0] = (float)v;
            d[1] = (float)(v - (double)d[0]);
        };
        const bool circ = ed == 0.0;
        split(O->ax1, circ ? 0.0 : -cwd * cE0d + swd * sed * sE0d);
        split(O->ax2, circ ? -1.0 : -cwd * sE0d - swd * sed * cE0d);
        split(O->ay1, circ ? -1.0 : -swd * cE0d - cwd * sed * sE0d);
        split(O->ay2, circ ? 0.0 : -swd * sE0d + cwd * sed * cE0d);
        split(O->rho0, circ ? 1.0 : den0d);
        split(O->a2, ad * ad);
        split(O->b2, bd * bd);
        split(O->ecE0, ed * cE0d);
        split(O->esE0, ed * sE0d);
        O->pad[0] = O->pad[1] = 0.0f;
        PvContactFF* C = reinterpret_cast<PvContactFF*>(O + 1);
        for (int pb = 0; pb < mp.npb; ++pb) {
            const double k = row[6 + (mp.chromatic ? pb : 0)];
            split(C[pb].opk, 1.0 + k);
            split(C[pb].omk, 1.0 - k);
            split(C[pb].gsc, (double)(mp.ng - 1) / (1.0 + k));
            C[pb].pad[0] = C[pb].pad[1] = 0.0f;
        }
    }

    // (3) profile rows of all pvs of the CTA: the k-interpolated combination of
    // the basis projections times 1 / I_star (arithmetic in R)
    const size_t kstride = (size_t)mp.ng;
    const size_t bstride = (size_t)mp.nk * mp.ng;
    const R inv_dk = (R)mp.inv_dk;
    char* rows_region = records + rows_offset(L, npv);
    const bool named = mp.ld_model != RR_LD_TABULATED;
    const int nc = named ? mp.nldc : 0;
    // work units of 64 g nodes of one (pv, passband) row block, taken by the
    // warps from a shared counter; lanes walk the nodes.  Rows of pvs that
    // (2a) finds invalid are built too and never read.
    const int nchunk = (L.ng_pad + 63) / 64;
    const int nunits = nloc * mp.npb * nchunk;
    #pragma unroll 1
    while (true) {
        int w = 0;
        if (lane == 0) w = atomicAdd(&rows_next, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= nunits) break;
        const int rw = w / nchunk, ch = w - rw * nchunk;
        const int lp = rw / mp.npb, pb = rw - lp * mp.npb;
        if (st_s[lp] != 0) continue;
        R* r0 = reinterpret_cast<R*>(rows_region + (size_t)(pv0 + lp) * L.rows_bytes) +
                (size_t)pb * L.rows_per_pb * L.ng_pad;
        const int ik = ik_s[lp][pb];
        const R ak = ak_s[lp][pb], bk = R(1) - ak;
        const R invIs = invIs_s[lp][pb];
        R uc[4];
        #pragma unroll
        for (int c = 0; c < 4; ++c) uc[c] = c < nc ? u_s[lp][pb][c] : R(0);
        R Ic[4];   // basis disk integrals, converted once per row
        // (the power-2 laws have no coefficient bases: their I_star partials are formed per pv)
        const bool p2law = mp.ld_model == RR_LD_POWER2 || mp.ld_model == RR_LD_POWER2_PM;
        #pragma unroll
        for (int c = 0; c < 4; ++c) Ic[c] = (grad && c < nc && !p2law) ? (R)istar[1 + c] : R(0);
        const int b0 = named ? 0 : pb;
        if (ik < 0) {
            // small-planet approximation (Sect. 3.4): the profile at the planet's centre at each
            // g node (small_planet_node), in the rows' arithmetic R
            SmallPlanetRow sp;
            sp.kw = (double)ak;
            sp.b0 = b0;
            sp.nc = nc;
            sp.ud[0] = 1.0;
            #pragma unroll
            for (int c = 0; c < 4; ++c) sp.ud[1 + c] = (double)uc[c];
            sp.kw1f = 1.0f + (float)ak;
            #pragma unroll
            for (int c = 0; c < 5; ++c) sp.udf[c] = (float)sp.ud[c];
            sp.mu_minf = (float)mp.mu_min;
            sp.dgf = (float)mp.dg;
            const int ig_end = min(L.ng_pad, 64 * ch + 64);
            for (int ig = 64 * ch + lane; ig < ig_end; ig += 32) {
                if (ig >= mp.ng) {
                    for (int r = 0; r < L.rows_per_pb; ++r) r0[(size_t)r * L.ng_pad + ig] = (R)0;
                    continue;
                }
                R vb[5] = {R(0), R(0), R(0), R(0), R(0)}, dk = R(0), vb1[5], dk1;
                const R v = small_planet_node_r<R>(mp, sp, ig, vb, dk) * invIs;
                r0[ig] = v;
                if (!grad) continue;
                const R vn = ig < mp.ng - 1 ? small_planet_node_r<R>(mp, sp, ig + 1, vb1, dk1) * invIs : v;
                r0[L.ng_pad + ig] = vn - v;
                r0[2 * L.ng_pad + ig] = dk * invIs;
                for (int j = 0; j < nc; ++j) r0[(size_t)(3 + j) * L.ng_pad + ig] = (vb[1 + j] - v * Ic[j]) * invIs;
            }
            continue;
        }
        if (mp.direct && (mp.ld_model == RR_LD_POWER2 || mp.ld_model == RR_LD_POWER2_PM)) {
            // power-2 laws: row = ((1 - c) T0 + c T1) / I_star with T0 = w . 1 and T1 = w . mu^alpha
            // of this passband; adjoint rows in (c, alpha) with T2 = w . mu^alpha ln mu = dT1/dalpha,
            // then for (h1, h2) the chain rule through c = 1 - h1 + h2, alpha = log2(c / h2)
            const size_t ds = (size_t)D.nrows * mp.ng;
            const int q = (mp.chromatic && !mp.shared) ? 0 : pb;
            const size_t o0 = (size_t)ik * mp.ng;
            const R* Hp = reinterpret_cast<const R*>(D.hi) + o0;
            const float* Lp = D.lo ? D.lo + o0 : nullptr;
            const R* Kp = grad ? reinterpret_cast<const R*>(D.dk) + o0 : nullptr;
            const int cl[3] = {0, 1 + 2 * q, 2 + 2 * q};
            const R cc = uc[0], al = uc[1];
            // d I_star / d c and d I_star / d alpha
            const R Ic_c = -Tr<R>::pi() * al / (al + R(2));
            const R Ic_a = -R(2) * Tr<R>::pi() * cc / ((al + R(2)) * (al + R(2)));
            auto val = [&](int col, int i) -> R {
                return Hp[cl[col] * ds + i] + (Lp ? (R)Lp[cl[col] * ds + i] : R(0));
            };
            const int ig_end = min(L.ng_pad, 64 * ch + 64);
            for (int ig = 64 * ch + lane; ig < ig_end; ig += 32) {
                if (ig >= mp.ng) {
                    for (int r = 0; r < L.rows_per_pb; ++r) r0[(size_t)r * L.ng_pad + ig] = (R)0;
                    continue;
                }
                const R t0 = val(0, ig), t1 = val(1, ig);
                const R ldw_n = ((R(1) - cc) * t0 + cc * t1) * invIs;
                r0[ig] = ldw_n;
                if (!grad) continue;
                R dv = 0;
                if (ig < mp.ng - 1) {
                    R d0 = Hp[cl[0] * ds + ig + 1] - Hp[cl[0] * ds + ig];
                    R d1 = Hp[cl[1] * ds + ig + 1] - Hp[cl[1] * ds + ig];
                    if (Lp) {
                        d0 += (R)(Lp[cl[0] * ds + ig + 1] - Lp[cl[0] * ds + ig]);
                        d1 += (R)(Lp[cl[1] * ds + ig + 1] - Lp[cl[1] * ds + ig]);
                    }
                    dv = (R(1) - cc) * d0 + cc * d1;
                }
                r0[L.ng_pad + ig] = dv * invIs;
                r0[2 * L.ng_pad + ig] = ((R(1) - cc) * Kp[cl[0] * ds + ig] + cc * Kp[cl[1] * ds + ig]) * invIs;
                const R t2 = val(2, ig);
                R Qc = ((t1 - t0) - ldw_n * Ic_c) * invIs;
                R Qa = (cc * t2 - ldw_n * Ic_a) * invIs;
                if (mp.ld_model == RR_LD_POWER2_PM) {
                    // h2 = c 2^-alpha; dc/dh1 = -1, dalpha/dh1 = -1 / (c ln 2),
                    // dc/dh2 = 1, dalpha/dh2 = (1/c - 1/h2) / ln 2
                    const R inv_ln2 = R(1.4426950408889634);
                    const R inv_h2 = exp2(al) / cc;
                    const R Qh1 = -Qc - Qa * inv_ln2 / cc;
                    const R Qh2 = Qc + Qa * (R(1) / cc - inv_h2) * inv_ln2;
                    Qc = Qh1;
                    Qa = Qh2;
                }
                r0[3 * L.ng_pad + ig] = Qc;
                r0[4 * L.ng_pad + ig] = Qa;
            }
            continue;
        }
        if (mp.direct) {
            // direct model: the pv's own projections (no k interpolation); the
            // in-cell slopes come from the differences of the FP32 pairs
            const size_t ds = (size_t)D.nrows * mp.ng;
            const size_t o0 = (size_t)b0 * ds + (size_t)ik * mp.ng;
            const R* Hp = reinterpret_cast<const R*>(D.hi) + o0;
            const float* Lp = D.lo ? D.lo + o0 : nullptr;
            const R* Kp = grad ? reinterpret_cast<const R*>(D.dk) + o0 : nullptr;
            const int ig_end = min(L.ng_pad, 64 * ch + 64);
            for (int ig = 64 * ch + lane; ig < ig_end; ig += 32) {
                if (ig >= mp.ng) {
                    for (int r = 0; r < L.rows_per_pb; ++r) r0[(size_t)r * L.ng_pad + ig] = (R)0;
                    continue;
                }
                R vb[5];
                #pragma unroll
                for (int c = 0; c < 5; ++c)
                    vb[c] = (c == 0 || c <= nc) ? Hp[c * ds + ig] + (Lp ? (R)Lp[c * ds + ig] : R(0)) : R(0);
                R v = vb[0];
                #pragma unroll
                for (int c = 0; c < 4; ++c) v += uc[c] * vb[1 + c];
                const R ldw_n = v * invIs;
                r0[ig] = ldw_n;
                if (!grad) continue;
                R dv = 0, kv = 0;
                #pragma unroll
                for (int c = 0; c < 5; ++c) {
                    if (c == 0 || c <= nc) {
                        const R w = c == 0 ? R(1) : uc[c - 1];
                        if (ig < mp.ng - 1) {
                            R dd = Hp[c * ds + ig + 1] - Hp[c * ds + ig];
                            if (Lp) dd += (R)(Lp[c * ds + ig + 1] - Lp[c * ds + ig]);
                            dv += w * dd;
                        }
                        kv += w * Kp[c * ds + ig];
                    }
                }
                r0[L.ng_pad + ig] = dv * invIs;
                r0[2 * L.ng_pad + ig] = kv * invIs;
                #pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (c < nc) r0[(size_t)(3 + c) * L.ng_pad + ig] = (vb[1 + c] - ldw_n * Ic[c]) * invIs;
            }
            continue;
        }
        const R* T0p = T + (size_t)b0 * bstride + (size_t)ik * kstride;
        const float* D0p = DT + (size_t)b0 * bstride + (size_t)ik * kstride;
        const int ig_end = min(L.ng_pad, 64 * ch + 64);
        for (int ig = 64 * ch + lane; ig < ig_end; ig += 32) {
            if (ig >= mp.ng) {
                for (int r = 0; r < L.rows_per_pb; ++r) r0[(size_t)r * L.ng_pad + ig] = (R)0;
                continue;
            }
            R lo = T0p[ig], hi = T0p[kstride + ig];
            #pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c < nc) {
                    const R* Tc = T0p + (size_t)(1 + c) * bstride;
                    lo += uc[c] * Tc[ig];
                    hi += uc[c] * Tc[kstride + ig];
                }
            }
            const R ldw_n = (bk * lo + ak * hi) * invIs;
            r0[ig] = ldw_n;
            if (!grad) continue;
            // row 1: ldw_n[ig+1] - ldw_n[ig], from differences that keep full relative precision
            R dlo = 0, dhi = 0;
            if (ig < mp.ng - 1) {
                #pragma unroll
                for (int c = 0; c < 5; ++c) {
                    if (c == 0 || c <= nc) {
                        const R w = c == 0 ? R(1) : uc[c - 1];
                        if (sizeof(R) == sizeof(double)) {
                            const R* Tc = T0p + (size_t)c * bstride;
                            dlo += w * (Tc[ig + 1] - Tc[ig]);
                            dhi += w * (Tc[kstride + ig + 1] - Tc[kstride + ig]);
                        } else {
                            const float* Dc = D0p + (size_t)c * bstride;
                            dlo += w * (R)Dc[ig];
                            dhi += w * (R)Dc[kstride + ig];
                        }
                    }
                }
            }
            r0[L.ng_pad + ig] = (bk * dlo + ak * dhi) * invIs;
            r0[2 * L.ng_pad + ig] = (hi - lo) * (inv_dk * invIs);
            #pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c < nc) {
                    const R* Tc = T0p + (size_t)(1 + c) * bstride;
                    const R Rc = bk * Tc[ig] + ak * Tc[kstride + ig];
                    r0[(size_t)(3 + c) * L.ng_pad + ig] = (Rc - ldw_n * Ic[c]) * invIs;
                }
            }
        }
    }
}

ModelParams model_params(const rr_ctx* c) {
    ModelParams mp;
    mp.ld_model = c->cfg.ld_model;
    mp.npb = c->cfg.npb;
    mp.chromatic = c->cfg.chromatic;
    mp.nldc = c->nldc;
    mp.nparam = c->nparam;
    mp.nk = c->cfg.nk;
    mp.ng = c->cfg.ng;
    mp.nbasis = c->nbasis;
    mp.k0 = c->cfg.k0;
    mp.k1 = c->cfg.k1;
    mp.dk = c->dk;
    mp.inv_dk = 1.0 / c->dk;
    mp.direct = c->cfg.direct;
    mp.dg = 1.0 / (c->cfg.ng - 1);
    mp.shared = shared_weights(c) ? 1 : 0;
    mp.pad_ = 0;
    mp.k_small = c->cfg.k_small;
    mp.mu_min = c->mu.empty() ? 0.0 : c->mu.back();
    mp.nz = c->nz;
    mp.tab = c->d_tab;
    mp.tab_off = c->d_tab_off;
    // int_0^1 mu / (e^mu - 1) dmu = pi^2/6 - Li2(1/e) + ln(1 - 1/e) (expand 1/(e^mu - 1) = sum_k e^(-k mu));
    // Li2(1/e) = sum_k e^(-k) / k^2, 40 terms below 1e-18
    double li2 = 0.0, p = 1.0;
    for (int j = 1; j <= 40; ++j) {
        p *= std::exp(-1.0);
        li2 += p / ((double)j * j);
    }
    mp.exp_c = CUDART_PI * CUDART_PI / 6.0 - li2 + std::log(1.0 - std::exp(-1.0));
    return mp;
}

cudaError_t launch_ld_basis(rr_ctx* c, cudaStream_t s) {
    ModelParams mp = model_params(c);
    rr_ld_basis_kernel<<<c->nbasis, 256, 0, s>>>(mp, c->d_mu, c->nz, c->d_tab, c->d_tab_off, c->d_basis,
                                                 c->d_istar);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_weights(rr_ctx* c, bool need_w, cudaStream_t s) {
    ModelParams mp = model_params(c);
    const size_t smem = (size_t)(2 * c->nz + 1) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(rr_weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(c->cfg.ng, c->cfg.nk);
    rr_weights_kernel<<<grid, 256, smem, s>>>(mp, c->d_ze, c->nz, c->d_basis, need_w ? 1 : 0, c->d_w,
                                              c->d_T64, c->d_T32);
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t n = (size_t)c->nbasis * c->cfg.nk * c->cfg.ng;
    rr_diff_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->d_T64, c->d_DT32, c->cfg.ng, n);
    c->launches++;
    return cudaGetLastError();
}

size_t direct_bytes(const rr_ctx* c, int npv, bool grad) {
    const size_t n = (size_t)direct_cols(c) * npv * direct_rows_per_pv(c) * c->cfg.ng;
    const size_t rb = c->cfg.precision == RR_PREC_FP64 ? sizeof(double) : sizeof(float);
    size_t b = align256(n * rb);
    if (c->cfg.precision == RR_PREC_MIXED) b += align256(n * sizeof(float));
    if (grad) b += align256(n * rb);
    return b;
}

DirectTables direct_view(const rr_ctx* c, void* base, int npv, bool grad) {
    DirectTables D;
    const size_t n = (size_t)direct_cols(c) * npv * direct_rows_per_pv(c) * c->cfg.ng;
    const size_t rb = c->cfg.precision == RR_PREC_FP64 ? sizeof(double) : sizeof(float);
    char* p = (char*)base;
    D.hi = p;
    p += align256(n * rb);
    D.lo = nullptr;
    if (c->cfg.precision == RR_PREC_MIXED) {
        D.lo = (float*)p;
        p += align256(n * sizeof(float));
    }
    D.dk = grad ? p : nullptr;
    D.nrows = npv * direct_rows_per_pv(c);
    return D;
}

cudaError_t launch_direct_prefix(rr_ctx* c, cudaStream_t s) {
    ModelParams mp = model_params(c);
    rr_direct_prefix_kernel<<<c->nbasis, 256, 0, s>>>(mp, c->d_ze, c->d_basis, c->d_zef, c->d_basisf, c->d_pre64,
                                                      c->d_pref);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_direct_tables(rr_ctx* c, const double* params, int npv, bool grad, const DirectTables& D,
                                 cudaStream_t s) {
    if (npv == 0) return cudaSuccess;
    ModelParams mp = model_params(c);
    const long long warps = (long long)npv * direct_rows_per_pv(c) * ((c->cfg.ng + 31) / 32);
    const unsigned grid = (unsigned)((warps + kDirWarps - 1) / kDirWarps);
    const bool p2 = power2_law(c);
    if (c->cfg.precision == RR_PREC_FP64) {
        auto kern = p2 ? rr_direct_table_kernel<double, true> : rr_direct_table_kernel<double, false>;
        kern<<<grid, kDirWarps * 32, 0, s>>>(mp, params, c->d_ze, c->d_basis, c->d_basis, c->d_pre64, nullptr,
                                             c->d_lnmu, c->d_mu, D, grad ? 1 : 0);
    } else {
        auto kern = p2 ? rr_direct_table_kernel<float, true> : rr_direct_table_kernel<float, false>;
        kern<<<grid, kDirWarps * 32, 0, s>>>(mp, params, c->d_zef, c->d_basisf, c->d_basis, c->d_pref,
                                             c->d_pref + (size_t)c->nbasis * (c->nz + 1), c->d_lnmuf, c->d_mu, D,
                                             grad ? 1 : 0);
    }
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_pv_setup(rr_ctx* c, const double* params, int npv, const PbParams& pbp, bool grad,
                            void* records, int32_t* pv_status, cudaStream_t s, const double* times,
                            const int32_t* pb_index, int npt, void* pts_dt, void* pts_pb, void* pts_grp) {
    ModelParams mp = model_params(c);
    DirectTables D = {nullptr, nullptr, nullptr, 0};
    if (c->cfg.direct) D = direct_view(c, (char*)records + align256(records_bytes(c, npv, grad)), npv, grad);
    const int ppc = setup_pvs_per_cta(c->cfg.npb);
    PointsArgs pa = {};
    int blocks = (npv + ppc - 1) / ppc;
    if (c->cfg.precision == RR_PREC_MIXED && npt > 0 && times) {
        // the per-time preparation rides in the same launch: two groups per CTA
        pa.times = times;
        pa.pb_index = pb_index;
        pa.npt = npt;
        pa.ngroups = (npt + kWarpPts - 1) / kWarpPts;
        pa.dt = (float2*)pts_dt;
        pa.pbw = (int32_t*)pts_pb;
        pa.grp = (GroupInfo*)pts_grp;
        pa.npoints = (pa.ngroups + 1) / 2;
        blocks += pa.npoints;
    }
    if (c->cfg.precision == RR_PREC_FP64) {
        RecLayout L = make_layout<double>(c->cfg.npb, c->cfg.ng, c->nldc, grad);
        rr_pv_setup_kernel<double><<<blocks, 256, 0, s>>>(mp, pbp, params, npv, c->d_T64, c->d_DT32, c->d_istar, L,
                                                          grad ? 1 : 0, (char*)records, pv_status, D, pa);
    } else {
        RecLayout L = make_layout<float>(c->cfg.npb, c->cfg.ng, c->nldc, grad);
        rr_pv_setup_kernel<float><<<blocks, 256, 0, s>>>(mp, pbp, params, npv, c->d_T32, c->d_DT32, c->d_istar, L,
                                                         grad ? 1 : 0, (char*)records, pv_status, D, pa);
    }
    c->launches++;
    return cudaGetLastError();
}

}  // namespace rr
