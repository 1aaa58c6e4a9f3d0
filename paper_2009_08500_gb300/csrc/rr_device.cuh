// Device-side building blocks of the per-point kernels.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "rr_internal.h"

namespace rr {

template <typename R> struct Tr;
template <> struct Tr<float> {
    static __device__ __forceinline__ float pi() { return CUDART_PI_F; }
    static __device__ __forceinline__ float two_pi() { return 2.0f * CUDART_PI_F; }
};
template <> struct Tr<double> {
    static __device__ __forceinline__ double pi() { return CUDART_PI; }
    static __device__ __forceinline__ double two_pi() { return 2.0 * CUDART_PI; }
};

// Angle of the point (x, y), y >= 0, in [0, pi] (atan2 for the upper half
// plane): folded onto t = min(y, |x|) / max(y, |x|) in [0, 1], where
// atan(t) = t P(t^2) with P(u) = 1 + c1 u + ... + c8 u^8.  The coefficients
// minimise the largest relative error over [0, 1] (1.67e-8 in exact
// arithmetic): Lawson's iteration (least squares on 2,000 Chebyshev nodes,
// each weight multiplied by its node's error every round, which converges to
// the minimax polynomial), in FP64, rounded to FP32 -- a CPU test repeats the
// fit and compares.  Evaluated in FP32 the result is within 1.4 ulp of atan,
// 4 ulp with the fast quotient.  Then atan = pi/2 - atan(1/t) above the
// diagonal and pi - angle for x < 0.
__device__ __forceinline__ float atan2_upper(float y, float x) {
    const float ax = fabsf(x);
    const float mx = fmaxf(y, ax), mn = fminf(y, ax);
    const float t = mx > 1e-30f ? __fdividef(mn, mx) : 0.0f;
    const float u = t * t;
    float p = 2.920693019e-03f;
    p = fmaf(p, u, -1.636793092e-02f);
    p = fmaf(p, u, 4.321186617e-02f);
    p = fmaf(p, u, -7.552214712e-02f);
    p = fmaf(p, u, 1.066600457e-01f);
    p = fmaf(p, u, -1.421105564e-01f);
    p = fmaf(p, u, 1.999377310e-01f);
    p = fmaf(p, u, -3.333315253e-01f);
    p = fmaf(p, u, 1.0f);
    float a = t * p;
    if (y > ax) a = CUDART_PIO2_F - a;
    if (x < 0.0f) a = CUDART_PI_F - a;
    return a;
}

// FP32 square root by the approximate instruction (relative error of order
// 2^-23, against half an ulp for the rounding-exact sqrtf, whose special-case
// handling costs issue slots on every sample): z and the lens chord K carry
// several ulp of orbit rounding already.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
// the forward kernel's per-sample square roots (z, the lens chord): approximate in FP32
__device__ __forceinline__ float d_sqrt_sample(float x) { return sqrt_approx(x); }
__device__ __forceinline__ double d_sqrt_sample(double x) { return sqrt(x); }
// the covered area's half-angles: the upper-half-plane arctangent (y = K >= 0)
__device__ __forceinline__ float d_atan2(float y, float x) { return atan2_upper(y, x); }
__device__ __forceinline__ double d_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ void d_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void d_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float d_rint(float x) { return rintf(x); }
__device__ __forceinline__ double d_rint(double x) { return rint(x); }
// Reciprocal: the approximate instruction in FP32 (within about an ulp; the
// adjoint's per-sample 1 / z and 1 / (1 - e cos E), far from zero and from
// the FP32 range limits, where the rounding-exact form's special-case handling
// costs issue slots), an exact IEEE division in FP64.
__device__ __forceinline__ float d_rcp(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double d_rcp(double x) { return 1.0 / x; }

// Area covered by a planet of radius k at centre distance z on a unit stellar
// disk (the a(c, k) of Eq. 5), for z < 1 + k, with its partial derivatives.
// Lens case: A = kappa0 + k^2 kappa1 - K/2 with K = sqrt of Heron's product
// of the triangle (1, k, z) built from differences, and the half-angles as
// atan2(K, .) -- accurate near both contact points.  dA/dz = -K/z (minus the
// common chord), dA/dk = 2 k kappa1 (planet rim inside the star).
// The contact factors f1 = 1 + k - z (outer contact) and f3 = z - (1 - k)
// (inner contact) are arguments: the mixed adjoint passes them from FP64 near
// the contacts, where K ~ sqrt(f1 f3) amplifies their rounding.
template <typename R, bool GRAD>
__device__ __forceinline__ R covered_area_f13(R k, R z, R f1, R f3, R& dAdz, R& dAdk) {
    const R one = R(1);
    if (z <= fabs(one - k)) {
        if (GRAD) dAdz = R(0);
        if (k < one) {
            if (GRAD) dAdk = R(2) * Tr<R>::pi() * k;
            return Tr<R>::pi() * k * k;
        }
        if (GRAD) dAdk = R(0);
        return Tr<R>::pi();
    }
    const R f2 = z + (one - k);
    const R f4 = z + (one + k);
    R h = (f1 * f2) * (f3 * f4);
    h = h > R(0) ? h : R(0);
    const R K = GRAD ? d_sqrt(h) : d_sqrt_sample(h);   // the adjoint keeps the rounding-exact root
    const R zz = z * z, kk = k * k;
    const R kap0 = d_atan2(K, zz + (one - kk));
    const R kap1 = d_atan2(K, zz + (kk - one));
    if (GRAD) {
        dAdz = -K * d_rcp(z);
        dAdk = R(2) * k * kap1;
    }
    return kap0 + kk * kap1 - R(0.5) * K;
}

template <typename R, bool GRAD>
__device__ __forceinline__ R covered_area(R k, R z, R& dAdz, R& dAdk) {
    return covered_area_f13<R, GRAD>(k, z, (R(1) + k) - z, z - (R(1) - k), dAdz, dAdk);
}

// Linear interpolation of a profile row over the g nodes g_i = i / (ng - 1):
// the cell is floor(g (ng - 1)), clamped to ng - 2.  Returns the value and
// the in-cell slope d/dg.
template <typename R>
__device__ __forceinline__ R lerp_row(const R* row, int ng, R g, R& slope_cell, int& cell) {
    const R x = g * R(ng - 1);
    int i = (int)x;                       // x >= 0: truncation is floor
    i = i < ng - 2 ? i : ng - 2;
    const R al = x - R(i);
    // plain loads: `row` may point to shared memory (staged rows) or to global memory
    const R l0 = row[i], l1 = row[i + 1];
    slope_cell = (l1 - l0);
    cell = i;
    return l0 + al * (l1 - l0);
}

// S = sin x and V = 1 - cos x for |x| <= 1 from their Taylor series in x^2
// (through x^9 and x^10: truncation below 3e-8 of S and 5e-9 of V), V
// without cancellation; larger |x| from the half angle.
__device__ __forceinline__ void half_angle_SV(float x, float& S, float& V) {
    if (fabsf(x) <= 1.0f) {
        const float x2 = x * x;
        float ps = fmaf(x2, 2.7557319e-6f, -1.9841270e-4f);    // 1/9!, -1/7!
        ps = fmaf(x2, ps, 8.3333333e-3f);                       // 1/5!
        ps = fmaf(x2, ps, -1.6666667e-1f);                      // -1/3!
        S = fmaf(x * x2, ps, x);
        float pv = fmaf(x2, 2.7557319e-7f, -2.4801587e-5f);    // 1/10!, -1/8!
        pv = fmaf(x2, pv, 1.3888889e-3f);                       // 1/6!
        pv = fmaf(x2, pv, -4.1666668e-2f);                      // -1/4!
        pv = fmaf(x2, pv, 0.5f);                                // 1/2!
        V = x2 * pv;
    } else {
        float hs, hc;
        sincosf(0.5f * x, &hs, &hc);
        S = 2.0f * hs * hc;
        V = 2.0f * hs * hs;
    }
}

// Offset-form Kepler solve in FP32 for x = E - E0 given dM = M - M0
// (Newton, f(x) = x - ecE0 sin x + esE0 (1 - cos x) - dM, f' = 1 - e cos E).
// Start: the series inversion through third order (kep2, kep3 per pv).  A
// Newton step dx leaves an error of at most kepC dx^2 (kepC >= |f''/(2 f')|),
// so the loop stops once that is below FP32 resolution of x; S and V follow x
// by a first-order rotation, whose error dx^2 / 2 is below the same bound.
// On return S = sin x, V = 1 - cos x.  Returns false if not converged.
__device__ __forceinline__ bool kepler_offset_f32(float dM, float ecE0, float esE0, float inv_den0, float kep2,
                                                  float kep3, float kepC, float& x, float& S, float& V, int& iters) {
    const float y = dM * inv_den0;
    x = fmaf(fmaf(kep3, y, kep2), y * y, y);
    #pragma unroll 1
    for (int it = 0; it < 24; ++it) {
        half_angle_SV(x, S, V);
        const float fx = (x - dM) - ecE0 * S + esE0 * V;
        const float fp = (1.0f - ecE0) + ecE0 * V + esE0 * S;
        const float dx = __fdividef(fx, fp);
        x -= dx;
        const float S_old = S;
        S -= dx * (1.0f - V);
        V -= dx * S_old;
        iters = it + 1;
        if (kepC * dx * dx <= 1.5e-8f * fabsf(x) + 1e-37f) return true;
    }
    return false;
}

// FP64 offset-form Kepler solve (used for e > kESwitch and by the FP64 path).
__device__ __forceinline__ bool kepler_offset_f64(double dM, double ecE0, double esE0,
                                                  double inv_den0, double& x, double& S,
                                                  double& V) {
    x = dM * inv_den0;
    #pragma unroll 1
    for (int it = 0; it < 100; ++it) {
        double hs, hc;
        sincos(0.5 * x, &hs, &hc);
        S = 2.0 * hs * hc;
        V = 2.0 * hs * hs;
        const double fx = (x - dM) - ecE0 * S + esE0 * V;
        const double fp = (1.0 - ecE0) + ecE0 * V + esE0 * S;
        const double dx = fx / fp;
        x -= dx;
        const double S_old = S;
        S -= dx * (1.0 - V);
        V -= dx * S_old;
        // after a step this small the quadratic convergence has left only round-off
        if (fabs(dx) <= 1e-12 * fabs(x) + 1e-300) return true;
    }
    return false;
}

// ---- bulk asynchronous copy global -> shared with an mbarrier (TMA engine) ----

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// dst, src 16-byte aligned; bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bulk asynchronous copy shared -> global (TMA engine, bulk-group completion).
// Both addresses 16-byte aligned, size a multiple of 16 bytes.
// The L2 policy marks the written lines evict-first (a streamed output, as
// st.global.cs does for ordinary stores).
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void bulk_s2g(void* gdst, const void* ssrc, uint32_t bytes, uint64_t pol) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(
                     __cvta_generic_to_global(gdst)),
                 "r"(smem_u32(ssrc)), "r"(bytes), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Start fetching [gsrc, gsrc + bytes) of global memory into L2 (a hint: nothing
// waits for it).  gsrc 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* gsrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(gsrc)), "r"(bytes)
                 : "memory");
}
// Wait until every bulk group this thread committed has completed (writes done).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Make this thread's generic-proxy writes to shared memory visible to the async proxy.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: at most 2^21 polls and about one second
// (try_wait may suspend the thread for a system-dependent time per poll, so
// the clock bounds the total).  false when it gave up.
constexpr uint64_t kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    #pragma unroll 1
    for (int i = 0; i < (1 << 21); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(64);
        if ((i & 255) == 255 && global_ns() - t0 > kWaitLimitNs) break;
    }
    return false;
}

// Stage `bytes` (multiple of 16) from global memory into shared memory with
// one elected thread issuing the copy; every thread waits (bounded).  On a
// timeout the device error word is set, the wait is retried once more
// (bounded) and false is returned: the CTA then leaves.  The copies are at
// most 64 KB each from global memory, which a working GPU completes in
// microseconds, so a copy still in flight after two waits of about a second
// each means a device that has stopped making progress; the retry only gives
// a slow copy its chance to land before the CTA's shared memory is released.
__device__ __forceinline__ bool stage_to_smem(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar, int* err) {
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, bytes);
        // the copy engine limits one bulk copy's size; split into chunks
        const uint32_t chunk = 1u << 16;
        for (uint32_t off = 0; off < bytes; off += chunk) {
            const uint32_t n = bytes - off < chunk ? bytes - off : chunk;
            bulk_g2s((char*)dst + off, (const char*)src + off, n, bar);
        }
    }
    __syncthreads();
    bool ok = mbar_wait_bounded(bar, 0);
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, kErrBarrierTimeout);
        mbar_wait_bounded(bar, 0);
    }
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// ---- phase and orbit (offset-from-conjunction form) ----

struct Phase32 {
    float fr_h, fr_l;   // reduced phase in cycles, fr_h + fr_l, |.| <~ 0.5
    float m;            // integer cycles removed by the reduction
};

// Round to the nearest integer (ties to even) for |x| < 2^22 with two FP32
// additions: adding 1.5 * 2^23 leaves no fraction bits in the sum.
__device__ __forceinline__ float round_nearest(float x) {
    return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
}

// Precise phase (cycles) of a time relative to the nearest conjunction:
// psi = A + dt / P with dt = dh + dl, A = Ah + Al, 1 / P = Bh + Bl.
__device__ __forceinline__ Phase32 precise_phase(float dh, float dl, float Ah, float Al, float Bh,
                                                 float Bl) {
    const float p = dh * Bh;
    float e = fmaf(dh, Bh, -p);          // exact low part of dh * Bh
    e = fmaf(dh, Bl, e);
    e = fmaf(dl, Bh, e);
    const float s = p + Ah;              // two-sum of p and Ah
    const float bb = s - p;
    const float err = (p - (s - bb)) + (Ah - bb);
    const float m = round_nearest(s);
    Phase32 r;
    r.fr_h = s - m;                      // exact (m is the nearest integer to s)
    r.fr_l = err + (Al + e);
    r.m = m;
    return r;
}

struct Orbit32 {
    float z, Px, Py, S, V;
    float x;            // eccentric-anomaly offset E - E0 (= dM on a circular orbit)
    bool front, ok;
};

// Projected distance from the mean-anomaly offset dM = M - M0 (radians).
// dMd: the same offset in FP64, used when e > kESwitch.  iters: the Newton
// iterations of the FP32 Kepler solve (0 otherwise).
// The FP32 header's per-sample constants sit in aligned quadruples, each read
// with one 16-byte load (the header is 16-byte aligned in shared or global
// memory: records are multiples of 16 bytes from a 16-byte aligned base).
static_assert(offsetof(PvHead<float>, wmax_c) % 16 == 0 && offsetof(PvHead<float>, kepC) == offsetof(PvHead<float>, wmax_c) + 12,
              "wmax_c, kep2, kep3, kepC: one quadruple");
static_assert(offsetof(PvHead<float>, a) % 16 == 0 && offsetof(PvHead<float>, b2) == offsetof(PvHead<float>, a) + 12,
              "a, b, a2, b2: one quadruple");
static_assert(offsetof(PvHead<float>, e) % 16 == 0 && offsetof(PvHead<float>, inv_den0) == offsetof(PvHead<float>, e) + 12,
              "e, ecE0, esE0, inv_den0: one quadruple");
static_assert(offsetof(PvHead<float>, ax1) % 16 == 0 && offsetof(PvHead<float>, ay2) == offsetof(PvHead<float>, ax1) + 12,
              "ax1, ax2, ay1, ay2: one quadruple");
static_assert(offsetof(PvHead<float>, rho0) % 16 == 0 && offsetof(PvHead<float>, Bl) == offsetof(PvHead<float>, rho0) + 12,
              "rho0, n, Bh, Bl: one quadruple");
static_assert(sizeof(PvHead<float>) % 16 == 0 && alignof(PvHead<float>) == 16, "16-byte header");
static_assert(offsetof(PvPb<float>, k) == 0 && offsetof(PvPb<float>, win_p) == 12 && alignof(PvPb<float>) == 16,
              "k, inv1pk, win_s, win_p: one quadruple");
__device__ __forceinline__ float4 quad(const float& first) { return *reinterpret_cast<const float4*>(&first); }

// APPROX_Z: z by the approximate square root (the forward kernel, where z's
// rounding reaches the flux with a factor below 1); the adjoint takes the
// rounding-exact one, since near a contact point its z-derivative amplifies
// z's rounding by 1 / (2 (1 + k - z)).
template <bool APPROX_Z = true>
__device__ __forceinline__ Orbit32 orbit32(const PvHead<float>& H, float dM, double dMd, int& iters) {
    Orbit32 o;
    o.ok = true;
    iters = 0;
    float x;
    const int flags = H.flags;
    if (flags & kPvCircular) {
        half_angle_SV(dM, o.S, o.V);
        x = dM;
    } else if (flags & kPvKepler64) {
        double xd, Sd, Vd;
        o.ok = kepler_offset_f64(dMd, H.ecE0d, H.esE0d, H.inv_den0d, xd, Sd, Vd);
        o.S = (float)Sd;
        o.V = (float)Vd;
        x = (float)xd;
    } else {
        const float4 ke = quad(H.e);        // e, ecE0, esE0, inv_den0
        const float4 ks = quad(H.wmax_c);   // wmax_c, kep2, kep3, kepC
        o.ok = kepler_offset_f32(dM, ke.y, ke.z, ke.w, ks.y, ks.z, ks.w, x, o.S, o.V, iters);
    }
    o.x = x;
    const float4 ax = quad(H.ax1);          // ax1, ax2, ay1, ay2
    const float4 ab = quad(H.a);            // a, b, a2, b2
    const float rho0 = H.rho0;
    o.Px = fmaf(ax.x, o.V, ax.y * o.S);
    o.Py = rho0 + fmaf(ax.z, o.V, ax.w * o.S);
    const float z2 = fmaf(ab.z * o.Px, o.Px, ab.w * o.Py * o.Py);
    o.z = APPROX_Z ? sqrt_approx(z2) : sqrtf(z2);
    o.front = o.Py > 0.0f;
    return o;
}

struct Orbit64 {
    double z, Px, Py, S, V, x;
    bool front, ok;
};

__device__ __forceinline__ Orbit64 orbit64(const PvHead<double>& H, double dM) {
    Orbit64 o;
    o.ok = true;
    if (H.flags & kPvCircular) {
        double hs, hc;
        sincos(0.5 * dM, &hs, &hc);
        o.S = 2.0 * hs * hc;
        o.V = 2.0 * hs * hs;
        o.x = dM;
    } else {
        o.ok = kepler_offset_f64(dM, H.ecE0d, H.esE0d, H.inv_den0d, o.x, o.S, o.V);
    }
    o.Px = fma(H.ax1, o.V, H.ax2 * o.S);
    o.Py = H.rho0 + fma(H.ay1, o.V, H.ay2 * o.S);
    o.z = sqrt(fma(H.a2 * o.Px, o.Px, H.b2 * o.Py * o.Py));
    o.front = o.Py > 0.0;
    return o;
}

// ---- float-float arithmetic: a value as the unevaluated sum h + l of two
// floats (about 48 significant bits), from the error-free transformations of
// Knuth (two-sum), Dekker (fast two-sum) and the FMA product error.  The
// intrinsics keep the compiler from fusing or reassociating them. ----
struct FF {
    float h, l;
};

// s + e == a + b exactly
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// s + e == a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const FF s = ff_two_sum(a.h, b.h);
    return ff_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, FF{-b.h, -b.l}); }
__device__ __forceinline__ FF ff_add_f(FF a, float b) {
    const FF s = ff_two_sum(a.h, b);
    return ff_fast_two_sum(s.h, __fadd_rn(s.l, a.l));
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ FF ff_mul_f(FF a, float b) {
    const float p = __fmul_rn(a.h, b);
    return ff_fast_two_sum(p, fmaf(a.l, b, fmaf(a.h, b, -p)));
}
__device__ __forceinline__ FF ff_ld(const float* v) { return FF{v[0], v[1]}; }

// A rational constant as a float pair: hi = the nearest float, lo = the rest.
struct FFConst {
    float h, l;
};
constexpr FFConst ff_const(double v) { return FFConst{(float)v, (float)(v - (double)(float)v)}; }
__device__ __forceinline__ FF ff_c(FFConst c) { return FF{c.h, c.l}; }

// S = sin x and V = 1 - cos x as float pairs for a float |x| <= 1: x = x0 +
// d with x0 = j / kSvTabRes the nearest table node (d exact, |d| <= 1/128),
//   sin x = S0 (1 - Vd) + (1 - V0) Sd,  1 - cos x = V0 + (1 - V0) Vd + S0 Sd,
// Sd = d - d^3/6 + d^5/120 and Vd = d^2/2 - d^4/24 + d^6/720 (d^2 exact as a
// pair, the rest in FP32: below 8e-8, truncation below 2e-16).  Absolute
// error ~1e-13.
__device__ __forceinline__ void ff_sin_vers(float x, const float4* __restrict__ tab, FF& S, FF& V) {
    const int j = __float2int_rn(x * (float)kSvTabRes);
    const float4 t = tab[j + kSvTabRes];   // a generic load: the table may be in shared or global memory
    const float d = x - (float)j * (1.0f / (float)kSvTabRes);   // exact
    const float d2 = __fmul_rn(d, d);
    const FF Sd = ff_fast_two_sum(d, d * d2 * fmaf(d2, 1.0f / 120.0f, -1.0f / 6.0f));
    const FF Vd = ff_add_f(FF{0.5f * d2, 0.5f * fmaf(d, d, -d2)}, d2 * d2 * fmaf(d2, 1.0f / 720.0f, -1.0f / 24.0f));
    const FF S0{t.x, t.y}, V0{t.z, t.w};
    const FF C0 = ff_sub(FF{1.0f, 0.0f}, V0);
    S = ff_add(ff_sub(S0, ff_mul(S0, Vd)), ff_mul(C0, Sd));
    V = ff_add(V0, ff_add(ff_mul(C0, Vd), ff_mul(S0, Sd)));
}

// Projected distance as a float pair for a sample near a contact point (the
// mixed adjoint).  xc: the sample's phase from the conjunction in cycles as a
// float pair; x32: the FP32 orbit's eccentric-anomaly offset, |x32| <= 1.
// S and V are evaluated at x32 and turned by the Newton correction dx of the
// float-float Kepler residual (one step: the FP32 x is within ~1e-7 relative,
// so ~1e-14 remains; S(x + dx) = S + dx (1 - V) and V(x + dx) = V + dx S to
// first order, dx^2 ~ 1e-15); on a circular orbit x = dM, evaluated at its
// high part and turned by its low part.  Error of z ~1e-12.
__device__ __forceinline__ FF contact_z_ff(const PvOrbitFF& O, const float4* __restrict__ svtab, bool circular, FF xc,
                                          float x32) {
    constexpr FFConst two_pi = ff_const(6.283185307179586476925);
    const FF dM = ff_mul(ff_c(two_pi), xc);
    const float xe = circular ? dM.h : x32;
    FF S, V;
    ff_sin_vers(xe, svtab, S, V);
    float dx;
    if (circular) {
        dx = dM.l;
    } else {
        // f(x) = x - dM - ecE0 S + esE0 V, f'(x) = 1 - ecE0 (1 - V) + esE0 S
        const FF ec = ff_ld(O.ecE0), es = ff_ld(O.esE0);
        const FF fx = ff_sub(ff_add(ff_add_f(FF{-dM.h, -dM.l}, xe), ff_mul(es, V)), ff_mul(ec, S));
        const float fp = fmaf(ec.h, V.h - 1.0f, 1.0f) + es.h * S.h;
        dx = -__fdividef(fx.h + fx.l, fp);
    }
    const float Sh = S.h, Vh = V.h;
    S = ff_add_f(S, dx * (1.0f - Vh));
    V = ff_add_f(V, dx * Sh);
    const FF Px = ff_add(ff_mul(ff_ld(O.ax1), V), ff_mul(ff_ld(O.ax2), S));
    const FF Py = ff_add(ff_ld(O.rho0), ff_add(ff_mul(ff_ld(O.ay1), V), ff_mul(ff_ld(O.ay2), S)));
    const FF z2 = ff_add(ff_mul(ff_ld(O.a2), ff_mul(Px, Px)), ff_mul(ff_ld(O.b2), ff_mul(Py, Py)));
    // square root: the FP32 root and one Newton correction (z2 - zf^2) / (2 zf)
    const float zf = sqrtf(z2.h);
    const float p = __fmul_rn(zf, zf);
    const float r = (__fsub_rn(z2.h, p) - fmaf(zf, zf, -p)) + z2.l;
    return ff_fast_two_sum(zf, r * (0.5f / zf));
}

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__device__ __forceinline__ T sel4(const T (&v)[4], int q) {
    return q == 0 ? v[0] : (q == 1 ? v[1] : (q == 2 ? v[2] : v[3]));
}

// Thread t of a CTA owns the 4 consecutive times pt0 + 4t .. pt0 + 4t + 3.
__device__ __forceinline__ void load_points(const float2* __restrict__ pdt, const int32_t* __restrict__ ppb,
                                            int p0, int npt, float (&dh)[4], float (&dl)[4], int (&pbv)[4]) {
    if (p0 + 3 < npt) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(pdt + p0));
        const float4 b = __ldg(reinterpret_cast<const float4*>(pdt + p0 + 2));
        const int4 c = __ldg(reinterpret_cast<const int4*>(ppb + p0));
        dh[0] = a.x; dl[0] = a.y; dh[1] = a.z; dl[1] = a.w;
        dh[2] = b.x; dl[2] = b.y; dh[3] = b.z; dl[3] = b.w;
        pbv[0] = c.x; pbv[1] = c.y; pbv[2] = c.z; pbv[3] = c.w;
    } else {
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int p = p0 + q;
            dh[q] = dl[q] = 0.0f;
            pbv[q] = -1;
            if (p < npt) {
                const float2 v = __ldg(pdt + p);
                dh[q] = v.x;
                dl[q] = v.y;
                pbv[q] = __ldg(ppb + p);
            }
        }
    }
}



// ---- per-warp compaction of transit candidates -------------------------------
//
// A warp owns 128 consecutive times (4 per lane).  For one pv, the times
// whose exposure may overlap the transit are listed in shared memory with
// their sub-exposure counts; the warp then walks the flattened list of
// (time, sub-exposure) pairs 32 at a time, so every lane does useful work
// regardless of where the transit falls or how many sub-exposures a
// passband has.

struct WarpList {
    float4 cand[kWarpPts];   // fr_h, fr_l (precise phase, cycles), m (cycles removed), gb (cotangent / -ss)
    int pb[kWarpPts];
    int soff[kWarpPts + 1];  // first flattened sample of each candidate; soff[nc] = total
    float pacc[kWarpPts];    // per-candidate sum over its sub-exposures
};

__device__ __forceinline__ int warp_excl_scan(int v, int& total) {
    const int lane = threadIdx.x & 31;
    int x = v;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Walk the flattened samples of a candidate list 32 at a time.  For the
// chunk starting at sample e0, candidate jf holds e0; the candidates that
// start inside the chunk are marked in a 32-bit mask (one OR-reduction over
// the warp), so lane l's candidate is jf + (starts at positions 1..l).
struct ChunkWalk {
    int jf;   // candidate holding the chunk's first sample (warp-uniform)
};

__device__ __forceinline__ int chunk_cand(ChunkWalk& cw, const int* soff, int nc, int e0) {
    const int lane = threadIdx.x & 31;
    if (cw.jf + 1 < nc && soff[cw.jf + 1] <= e0) ++cw.jf;   // warp-uniform
    const int jn = cw.jf + 1 + lane;
    unsigned bit = 0u;
    if (jn < nc) {
        const int pos = soff[jn] - e0;
        if (pos > 0 && pos < 32) bit = 1u << pos;
    }
    const unsigned starts = __reduce_or_sync(0xffffffffu, bit);
    const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    const int j = cw.jf + __popc(starts & upto);
    cw.jf = __shfl_sync(0xffffffffu, j, 31);   // holds e0 + 31: the next chunk starts there or one later
    return j;
}

// Passband constants staged in shared memory (indexing the by-value kernel
// argument with a runtime passband would place it in local memory).
struct PbShared {
    int ss[RR_MAX_PB];
    float first[RR_MAX_PB], step[RR_MAX_PB], inv_ss[RR_MAX_PB];
    float first_lo[RR_MAX_PB], step_lo[RR_MAX_PB];   // low parts (the mixed adjoint's contact refinement)
};

__device__ __forceinline__ void stage_pb(const PbParams& pbp, PbShared* ps) {
    for (int j = threadIdx.x; j < pbp.npb; j += blockDim.x) {
        ps->ss[j] = pbp.ss[j];
        ps->first[j] = pbp.first[j];
        ps->step[j] = pbp.step[j];
        ps->inv_ss[j] = pbp.inv_ss[j];
        ps->first_lo[j] = pbp.first_lo[j];
        ps->step_lo[j] = pbp.step_lo[j];
    }
}

// Build the candidate list of this warp for one pv.  cand: 4-bit mask of the
// lane's candidate times; gb[q]: per-time weights stored with the entries.
// Returns the number of flattened samples (warp-uniform); nc gets the
// number of candidates, base the lane's first entry.
__device__ __forceinline__ int build_list(WarpList* wl, unsigned cand, const float (&dh)[4], const float (&dl)[4],
                                          const int (&pbv)[4], const float (&gbq)[4], float Ah, float Al, float Bh,
                                          float Bl, const PbShared* ps, int& nc, int& base) {
    const int lane = threadIdx.x & 31;
    int ns_l = 0;
    #pragma unroll
    for (int q = 0; q < 4; ++q)
        if (cand & (1u << q)) ns_l += ps->ss[pbv[q]];
    base = warp_excl_scan(__popc(cand), nc);
    int ns;
    int soff = warp_excl_scan(ns_l, ns);
    int j = base;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (cand & (1u << q)) {
            const Phase32 ph = precise_phase(dh[q], dl[q], Ah, Al, Bh, Bl);
            wl->cand[j] = make_float4(ph.fr_h, ph.fr_l, ph.m, gbq[q]);
            wl->pb[j] = pbv[q];
            wl->soff[j] = soff;
            wl->pacc[j] = 0.0f;
            soff += ps->ss[pbv[q]];
            ++j;
        }
    }
    if (lane == 0) wl->soff[nc] = ns;
    __syncwarp();
    return ns;
}

// Candidate list when every passband has one sample per time: a candidate
// is a sample, so the list is built from one ballot per time slot of the
// lanes (no scans) and holds the raw offsets (dh, dl), the passband and the
// per-time weight gbq; the precise phase is formed where a sample is
// evaluated.  The list keeps time order (lane-major), so that a chunk of 32
// samples is a contiguous stretch of the transit and takes the same branches.
// bq[q] gets the list index of the lane's time q.  Returns the number of
// candidates (warp-uniform).
__device__ __forceinline__ int build_list_ss1(WarpList* wl, unsigned cand, const float (&dh)[4],
                                              const float (&dl)[4], const int (&pbv)[4], const float (&gbq)[4],
                                              int (&bq)[4]) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int total = 0, before = 0;     // candidates of the whole warp / of the lanes below this one
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned bal = __ballot_sync(0xffffffffu, (cand >> q) & 1u);
        before += __popc(bal & below);
        total += __popc(bal);
    }
    #pragma unroll
    for (int q = 0; q < 4; ++q) bq[q] = before + __popc(cand & ((1u << q) - 1u));
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        if ((cand >> q) & 1u) {
            wl->cand[bq[q]] = make_float4(dh[q], dl[q], 0.0f, gbq[q]);
            wl->pb[bq[q]] = pbv[q];
        }
    }
    __syncwarp();
    return total;
}

// The same list for the adjoint, which needs neither the per-candidate sums
// nor the sub-exposure offsets: one float4 per candidate (dh, dl, passband
// index as int bits, gbq), 2 KB per warp instead of 3.6 KB, so that four CTAs
// fit on an SM.
__device__ __forceinline__ int build_list_ss1_packed(float4* wl, unsigned cand, const float (&dh)[4],
                                                     const float (&dl)[4], const int (&pbv)[4],
                                                     const float (&gbq)[4]) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int total = 0, before = 0;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned bal = __ballot_sync(0xffffffffu, (cand >> q) & 1u);
        before += __popc(bal & below);
        total += __popc(bal);
    }
    #pragma unroll
    for (int q = 0; q < 4; ++q)
        if ((cand >> q) & 1u)
            wl[before + __popc(cand & ((1u << q) - 1u))] = make_float4(dh[q], dl[q], __int_as_float(pbv[q]), gbq[q]);
    __syncwarp();
    return total;
}

// The forward kernel's per-warp candidate list, 16 bytes per candidate so that
// four CTAs fit on an SM: the candidate's phase pair (with supersampling the
// precise phase fr_h, fr_l in cycles; with one sample per time the raw offsets
// dh, dl), its passband and first flattened sample packed as (soff << 5) | pb
// (pb < RR_MAX_PB = 32; ps[nc] = ns << 5), and its sum over sub-exposures.
struct FluxList {
    float2 cand[kWarpPts];
    int ps[kWarpPts + 1];
    float pacc[kWarpPts];
};

__device__ __forceinline__ int chunk_cand_ps(ChunkWalk& cw, const int* ps, int nc, int e0) {
    const int lane = threadIdx.x & 31;
    if (cw.jf + 1 < nc && (ps[cw.jf + 1] >> 5) <= e0) ++cw.jf;   // warp-uniform
    const int jn = cw.jf + 1 + lane;
    unsigned bit = 0u;
    if (jn < nc) {
        const int pos = (ps[jn] >> 5) - e0;
        if (pos > 0 && pos < 32) bit = 1u << pos;
    }
    const unsigned starts = __reduce_or_sync(0xffffffffu, bit);
    const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    const int j = cw.jf + __popc(starts & upto);
    cw.jf = __shfl_sync(0xffffffffu, j, 31);
    return j;
}

// build_list for the forward kernel (FluxList; returns the flattened sample count).
__device__ __forceinline__ int build_list_flux(FluxList* fl, unsigned cand, const float (&dh)[4], const float (&dl)[4],
                                               const int (&pbv)[4], float Ah, float Al, float Bh, float Bl,
                                               const PbShared* ps, int& nc, int& base) {
    const int lane = threadIdx.x & 31;
    int ns_l = 0;
    #pragma unroll
    for (int q = 0; q < 4; ++q)
        if (cand & (1u << q)) ns_l += ps->ss[pbv[q]];
    base = warp_excl_scan(__popc(cand), nc);
    int ns;
    int soff = warp_excl_scan(ns_l, ns);
    int j = base;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (cand & (1u << q)) {
            const Phase32 ph = precise_phase(dh[q], dl[q], Ah, Al, Bh, Bl);
            fl->cand[j] = make_float2(ph.fr_h, ph.fr_l);
            fl->ps[j] = (soff << 5) | pbv[q];
            fl->pacc[j] = 0.0f;
            soff += ps->ss[pbv[q]];
            ++j;
        }
    }
    if (lane == 0) fl->ps[nc] = ns << 5;
    __syncwarp();
    return ns;
}

// build_list_ss1 for the forward kernel (FluxList: ps[j] = passband).
__device__ __forceinline__ int build_list_ss1_flux(FluxList* fl, unsigned cand, const float (&dh)[4],
                                                   const float (&dl)[4], const int (&pbv)[4], int (&bq)[4]) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int total = 0, before = 0;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned bal = __ballot_sync(0xffffffffu, (cand >> q) & 1u);
        before += __popc(bal & below);
        total += __popc(bal);
    }
    #pragma unroll
    for (int q = 0; q < 4; ++q) bq[q] = before + __popc(cand & ((1u << q) - 1u));
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        if ((cand >> q) & 1u) {
            fl->cand[bq[q]] = make_float2(dh[q], dl[q]);
            fl->ps[bq[q]] = pbv[q];
        }
    }
    __syncwarp();
    return total;
}

// Shared-memory layout common to the FP32 per-point kernels:
//   [mbarrier 16][reduction 64][per-pv tile constants 16 x kMaxPvTile]
//   [passband constants][one candidate list per warp][pv records ...]
constexpr size_t kOffRed = 16;
constexpr size_t kOffCta = kOffRed + 64;
constexpr size_t kOffPb = kOffCta + 16 * kMaxPvTile;
constexpr size_t kOffWl = kOffPb + ((sizeof(PbShared) + 15) / 16) * 16;
constexpr size_t kWlBytes = ((sizeof(WarpList) + 15) / 16) * 16;
constexpr size_t kOffRecs32 = kOffWl + (kBlock / 32) * kWlBytes;
// the forward kernel: FluxList
constexpr size_t kFlBytes = ((sizeof(FluxList) + 15) / 16) * 16;
constexpr size_t kOffRecsFlux = kOffWl + (kBlock / 32) * kFlBytes;
// the adjoint with one sample per time keeps only the packed list (float4 per candidate)
constexpr size_t kWlBytesPacked = kWarpPts * sizeof(float4);
constexpr size_t kOffRecs32Packed = kOffWl + (kBlock / 32) * kWlBytesPacked;

// Per-thread sample counts of the counting form of the FP32 kernels (indices
// RR_COUNT_*); added into the context's counters when the kernel ends.
struct Tally {
    unsigned n[RR_COUNT_KINDS];
};

__device__ __forceinline__ void tally_flush(const Tally& t, unsigned long long* counts) {
    #pragma unroll
    for (int j = 0; j < RR_COUNT_KINDS; ++j) {
        const unsigned v = __reduce_add_sync(0xffffffffu, t.n[j]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(counts + j, (unsigned long long)v);
    }
}

// One sub-exposure of one (pv, time): delta = A Ib (Eq. 5 without the 1 -),
// 0 outside the transit.  Kepler failure: bad = true, NaN.  COUNT: add the
// sample's work to `tl`.
template <bool COUNT = false>
__device__ __forceinline__ float delta32(const PvHead<float>& H, const PvPb<float>& pbc, const float* __restrict__ row,
                                         int ng, float fr_h, float fr_l, float s, float first, float step, bool& bad,
                                         Tally* tl = nullptr) {
    if (COUNT) ++tl->n[RR_COUNT_SAMPLES];
    const float off = fmaf(s, step, first) * H.Bh;   // sub-exposure s (exact integer), offset in cycles
    float x = (fr_h + off) + fr_l;
    x -= round_nearest(x);
    const float dM = 6.28318530717958647692f * x;
    if (fabsf(dM) > pbc.win_s) return 0.0f;
    double dMd = 0.0;
    if (H.flags & kPvKepler64) {
        double xd = ((double)fr_h + (double)off) + (double)fr_l;
        xd -= rint(xd);
        dMd = 6.283185307179586476925 * xd;
    }
    int iters;
    const Orbit32 o = orbit32(H, dM, dMd, iters);
    if (COUNT) {
        ++tl->n[RR_COUNT_ORBIT];
        if (H.flags & kPvCircular) ++tl->n[RR_COUNT_CIRCULAR];
        tl->n[RR_COUNT_NEWTON] += iters;
    }
    if (!o.ok) {
        bad = true;
        return __int_as_float(0x7fc00000);
    }
    const float2 pq = *reinterpret_cast<const float2*>(&pbc.k);   // k, inv1pk
    const float g = o.z * pq.y;
    if (!o.front || g >= 1.0f) return 0.0f;
    if (COUNT) {
        ++tl->n[RR_COUNT_TRANSIT];
        if (o.z > fabsf(1.0f - pq.x)) ++tl->n[RR_COUNT_LENS];
    }
    float d0, d1, sl;
    int cell;
    const float A = covered_area<float, false>(pq.x, o.z, d0, d1);
    return A * lerp_row<float>(row, ng, g, sl, cell);
}


// Per-warp group state of the FP32 kernels.  A group is kWarpPts = 128
// consecutive times, 4 per lane; its float-float times are relative to the
// group's first time t_g.  The group's summary comes from points_group;
// lane l also holds the phase constants of pv l of the CTA's tile at t_g:
// A = frac((t_g - T0) / P) as a float pair and the removed integer cycles m.
struct GroupState {
    float wlo, whi, maxdt;   // warp-uniform: range of dh and largest |dh| over the group's times
    int full;                // all 128 times present with valid passbands
    float Ah, Al, m;         // phase constants of pv `lane`
};

// Phase constants of the tile's pvs at the CTA's first group g0 (the only FP64
// of the per-point kernels, once per CTA): cta_ph[i] = (A0h, A0l, m0, 0).
__device__ __forceinline__ void cta_phase(float4* cta_ph, const double* __restrict__ times, int g0,
                                          const char* recs, int rec_bytes, int npv_t) {
    for (int i = threadIdx.x; i < npv_t; i += blockDim.x) {
        const PvHead<float>& H = *reinterpret_cast<const PvHead<float>*>(recs + (size_t)i * rec_bytes);
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (H.status == 0) {
            const double psi = (__ldg(times + (size_t)g0 * kWarpPts) - H.T0) * H.invP;
            const double m = rint(psi);
            const double A = psi - m;
            v.x = (float)A;
            v.y = (float)(A - (double)v.x);
            v.z = (float)m;
        }
        cta_ph[i] = v;
    }
}

// Difference of two float pairs, (ah + al) - (bh + bl), as a float pair.
__device__ __forceinline__ void ff_sub(float ah, float al, float bh, float bl, float& rh, float& rl) {
    const float s = ah - bh;
    const float v = s - ah;
    const float e = (ah - (s - v)) - (bh + v);   // exact error of s
    rh = s;
    rl = e + (al - bl);
}

// sg: the CTA's copy in shared memory of the summaries of its groups (sg[j]
// for group gbeg + j, copied with the records); group gbeg is the phase
// reference of cta_phase.  Plain loads (shared memory).
__device__ __forceinline__ void group_load(GroupState& gs, const GroupInfo* sg, int j, const float4* cta_ph,
                                           const char* recs, int rec_bytes, int npv_t) {
    const int lane = threadIdx.x & 31;
    const float4 s0 = *reinterpret_cast<const float4*>(sg + j);
    const float2 tg = reinterpret_cast<const float2*>(sg + j)[2];
    const float2 t0 = reinterpret_cast<const float2*>(sg)[2];
    gs.wlo = s0.x;
    gs.whi = s0.y;
    gs.maxdt = s0.z;
    gs.full = __float_as_int(s0.w);
    gs.Ah = gs.Al = gs.m = 0.0f;
    if (lane < npv_t) {
        const PvHead<float>& H = *reinterpret_cast<const PvHead<float>*>(recs + (size_t)lane * rec_bytes);
        if (H.status == 0) {
            // phase at t_g = phase at t_g0 + (t_g - t_g0) / P, in float-float
            float dh, dl;
            ff_sub(tg.x, tg.y, t0.x, t0.y, dh, dl);
            const float4 a0 = cta_ph[lane];
            const Phase32 ph = precise_phase(dh, dl, a0.x, a0.y, H.Bh, H.Bl);
            gs.Ah = ph.fr_h;
            gs.Al = ph.fr_l;
            gs.m = a0.z + ph.m;
        }
    }
}

// Passband indices of the lane's 4 times (-1 beyond npt).
__device__ __forceinline__ void load_pb(const int32_t* __restrict__ ppb, int p0, int npt, int (&pbv)[4]) {
    if (p0 + 3 < npt) {
        const int4 c = __ldg(reinterpret_cast<const int4*>(ppb + p0));
        pbv[0] = c.x; pbv[1] = c.y; pbv[2] = c.z; pbv[3] = c.w;
    } else {
        #pragma unroll
        for (int q = 0; q < 4; ++q) pbv[q] = p0 + q < npt ? __ldg(ppb + p0 + q) : -1;
    }
}

// Can any of the warp's times be in transit for this pv?  The warp's phase
// interval [A + wlo/P, A + whi/P], widened by the pv's largest window and the
// rounding bound, must contain an integer (a conjunction).  Warp-uniform.
__device__ __forceinline__ bool warp_may_transit(const PvHead<float>& H, float4 c, float wlo, float whi) {
    if (!(wlo <= whi)) return false;
    const float W = H.wmax_c + 2.0f * c.w;
    const float plo = fmaf(wlo, H.Bh, c.x) - W;
    const float phi = fmaf(whi, H.Bh, c.x) + W;
    return ceilf(plo) <= phi;
}

// ---- scheduling of the FP32 kernels ----------------------------------------
//
// Warps take 128-time groups from a shared counter.  For a group, lane l
// decides for pv l of the tile whether the group's phase interval can hold a
// transit; a ballot gives the warp the tile's mask.  Pvs outside the mask need
// no arithmetic (flux exactly 1) and are stored at once; the others become
// work items (pv, group) in a shared-memory queue.  In the adjoint, warps
// claim queued items between groups and after the last one.  In the flux
// kernel a set of stream warps takes all the groups first while the other
// warps evaluate the items as they appear (with supersampling every warp
// streams first), so the output stream overlaps the in-transit arithmetic.
// Either way the in-transit work of the CTA is spread over all its warps
// whatever groups it falls in.
//
// Queue protocol: a producer reserves slots (atomicAdd on nitems), writes the
// item, then publishes it by writing its key (slots start at -1).  Consumers
// claim only reserved slots (compare-and-swap on next_item) and wait, a few
// instructions at most, for the key.  A warp that has no group left
// decrements `producers`; when that count is 0 and nothing is claimable the
// queue is finished.  Every wait is bounded.

// Shared counters.
struct TileCounters {
    int next_group, nitems, next_item, producers;
    unsigned rows_pf;   // pvs of the tile whose rows an L2 prefetch has been issued for (adjoint)
};

// Work item: phase constants of the pv at the group start (Ah, Al, m, rounding
// bound in cycles) and key = (group << 5) | pv-in-tile.
struct ItemQueue {
    float4* c;
    int* gi;
};

// Queue bytes for `cap` items (16-byte multiple).
__host__ __device__ inline size_t queue_bytes(int cap) { return ((size_t)cap * 20 + 15) & ~(size_t)15; }

__device__ __forceinline__ ItemQueue queue_at(char* base, int cap) {
    ItemQueue q;
    q.c = reinterpret_cast<float4*>(base);
    q.gi = reinterpret_cast<int*>(base + (size_t)cap * 16);
    return q;
}

// Before the CTA's first barrier: counters and empty slots.
__device__ __forceinline__ void queue_init(ItemQueue q, TileCounters* tc, int cap, int g0) {
    for (int j = threadIdx.x; j < cap; j += blockDim.x) q.gi[j] = -1;
    if (threadIdx.x == 0) {
        tc->next_group = g0;
        tc->nitems = 0;
        tc->next_item = 0;
        tc->producers = blockDim.x >> 5;
        tc->rows_pf = 0u;
    }
}

// Lane l: transit decision for pv l of the tile at this group.  Returns the
// warp's mask of pvs that may transit; `bad` gets the mask of invalid pvs and
// `cl` lane l's phase constants (x, y, z = Ah, Al, m; w = rounding bound).
__device__ __forceinline__ unsigned group_decide(const GroupState& gs, const char* recs, int rec_bytes, int npv_t,
                                                 unsigned& bad, float4& cl) {
    const int lane = threadIdx.x & 31;
    bool may = false, inval = false;
    cl = make_float4(gs.Ah, gs.Al, gs.m, 0.0f);
    if (lane < npv_t) {
        const PvHead<float>& H = *reinterpret_cast<const PvHead<float>*>(recs + (size_t)lane * rec_bytes);
        inval = H.status != 0;
        cl.w = 2.4e-7f * (gs.maxdt * H.Bh + 1.0f);
        may = !inval && warp_may_transit(H, cl, gs.wlo, gs.whi);
    }
    bad = __ballot_sync(0xffffffffu, inval);
    return __ballot_sync(0xffffffffu, may);
}

// Append the warp's items (one per set bit of `may`) and publish them.
__device__ __forceinline__ void queue_push(ItemQueue q, TileCounters* tc, unsigned may, int g, float4 cl) {
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0) base = atomicAdd(&tc->nitems, __popc(may));
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((may >> lane) & 1u) {
        const int pos = base + __popc(may & ((1u << lane) - 1u));
        q.c[pos] = cl;
        __threadfence_block();
        *reinterpret_cast<volatile int*>(q.gi + pos) = (g << 5) | lane;
    }
}

// This warp takes no more groups.
__device__ __forceinline__ void queue_producer_done(TileCounters* tc) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        __threadfence_block();
        atomicSub(&tc->producers, 1);
    }
}

// Claim one reserved item for the warp (warp-uniform result), or -1 if every
// reserved item is claimed.
__device__ __forceinline__ int queue_claim(TileCounters* tc) {
    int it = -1;
    if ((threadIdx.x & 31) == 0) {
        volatile int* vn = &tc->nitems;
        int cur = *reinterpret_cast<volatile int*>(&tc->next_item);
        for (int tries = 0; tries < 64 && cur < *vn; ++tries) {
            const int prev = atomicCAS(&tc->next_item, cur, cur + 1);
            if (prev == cur) {
                it = cur;
                break;
            }
            cur = prev;
        }
    }
    return __shfl_sync(0xffffffffu, it, 0);
}

// Key of claimed item `it` once its producer has published it; -1 if the
// bounded wait gives up.
__device__ __forceinline__ int queue_key(ItemQueue q, int it) {
    int key = -1;
    if ((threadIdx.x & 31) == 0) {
        volatile int* vk = q.gi + it;
        for (int i = 0; i < (1 << 20); ++i) {
            key = *vk;
            if (key >= 0) break;
            __nanosleep(32);
        }
        __threadfence_block();
    }
    return __shfl_sync(0xffffffffu, key, 0);
}

// No group left for this warp and nothing claimable: true when no producer
// remains (the queue is then final).
__device__ __forceinline__ bool queue_finished(TileCounters* tc) {
    int done = 0;
    if ((threadIdx.x & 31) == 0) {
        done = *reinterpret_cast<volatile int*>(&tc->producers) == 0;
        __threadfence_block();
    }
    return __shfl_sync(0xffffffffu, done, 0) != 0;
}
// Value and mu-derivative of profile basis b at an arbitrary mu (the bases of
// rr_ld_basis_kernel; tabulated: passband b's table interpolated at mu, the
// slope of the segment holding mu, 0 outside the nodes).  FP64; mu > 0.
__device__ __forceinline__ double ld_basis_mu(const ModelParams& mp, int b, double m, const double* __restrict__ tab,
                              const int* __restrict__ tab_off, double& d) {
    if (mp.ld_model == RR_LD_TABULATED) {
        const int o0 = tab_off[b], n = tab_off[b + 1] - o0;
        const double* tmu = tab + 2 * o0;
        const double* tI = tmu + n;
        if (m < tmu[0]) { d = 0.0; return tI[0]; }
        if (m >= tmu[n - 1]) { d = 0.0; return tI[n - 1]; }
        int lo = 0, hi = n - 1;   // tmu[lo] <= m < tmu[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tmu[mid] <= m) lo = mid; else hi = mid;
        }
        d = (tI[lo + 1] - tI[lo]) / (tmu[lo + 1] - tmu[lo]);
        return tI[lo] + d * (m - tmu[lo]);
    }
    if (b == 0) { d = 0.0; return 1.0; }
    const double q = 1.0 - m;
    switch (mp.ld_model) {
        case RR_LD_NONLINEAR: {
            // -(1 - mu^(b/2)) and (b/2) mu^(b/2 - 1) through sqrt(mu)
            const double sq = sqrt(m);
            const double p = b == 1 ? sq : (b == 2 ? m : (b == 3 ? m * sq : m * m));
            d = b == 1 ? 0.5 / sq : (b == 2 ? 1.0 : (b == 3 ? 1.5 * sq : 2.0 * m));
            return -(1.0 - p);
        }
        case RR_LD_GENERAL: {
            double p = 1.0;
            for (int j = 1; j < b; ++j) p *= q;   // q^(b-1)
            d = b * p;
            return -p * q;
        }
        case RR_LD_LOGARITHMIC:
            if (b == 1) { d = 1.0; return -q; }
            d = -(log(m) + 1.0);
            return -m * log(m);
        case RR_LD_EXPONENTIAL:
            if (b == 1) { d = 1.0; return -q; }
            {
                const double e = exp(m), r = 1.0 / (1.0 - e);
                d = -e * r * r;
                return -r;
            }
        default:   // linear, quadratic (and q1, q2)
            if (b == 1) { d = 1.0; return -q; }
            d = 2.0 * q;
            return -q * q;
    }
}

// Per-point inputs of the FP32 kernels, once per call, for one 128-time group
// g (thread t = 0..127 of the group): dt = t - t_g as a float pair, t_g = the
// group's first time (FP64 here, so that the per-(pv, point) work is FP32
// only), and the passband index with out-of-range values mapped to npb; the
// group's summary (GroupInfo): the range and largest magnitude of its float
// offsets, whether it is full with valid passbands, t_g - t_0, and its weight
// (the sum over its times of ss[passband], ss in shared memory, or the count
// of valid times when ss is null).  Every thread of the block calls (one
// barrier); groups g >= ngroups only take part in the barrier.  red, redf:
// the group's reduction slots in shared memory.
__device__ __forceinline__ void points_group(const double* __restrict__ times, const int32_t* __restrict__ pb_index,
                                             int npt, int npb, float2* __restrict__ dt, int32_t* __restrict__ pbw,
                                             GroupInfo* __restrict__ grp, int g, int ngroups, int t,
                                             float (*red)[kWarpPts / 32], int* redf, const int* ss) {
    const int lane = t & 31, warp = t >> 5;
    const bool live = g < ngroups;
    const int p = g * kWarpPts + t;
    float lo = INFINITY, hi = -INFINITY, mx = 0.0f, wt = 0.0f;
    int ok = 0;
    double tg = 0.0;
    if (live) tg = times[(size_t)g * kWarpPts];
    if (live && p < npt) {
        const double d = times[p] - tg;
        const float h = (float)d;
        dt[p] = make_float2(h, (float)(d - (double)h));
        const int pb = pb_index ? pb_index[p] : 0;
        const int v = (pb >= 0 && pb < npb) ? pb : npb;
        pbw[p] = v;
        lo = hi = h;
        mx = fabsf(h);
        ok = v < npb;
        if (ok) wt = ss ? (float)ss[v] : 1.0f;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        wt += __shfl_xor_sync(0xffffffffu, wt, o);
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
        red[0][warp] = lo;
        red[1][warp] = hi;
        red[2][warp] = mx;
        red[3][warp] = wt;
        redf[warp] = ok;
    }
    __syncthreads();
    if (t == 0 && live) {
        GroupInfo gi;
        gi.wlo = red[0][0];
        gi.whi = red[1][0];
        gi.maxdt = red[2][0];
        gi.full = redf[0];
        gi.weight = red[3][0];
        for (int w = 1; w < kWarpPts / 32; ++w) {
            gi.wlo = fminf(gi.wlo, red[0][w]);
            gi.whi = fmaxf(gi.whi, red[1][w]);
            gi.maxdt = fmaxf(gi.maxdt, red[2][w]);
            gi.weight += red[3][w];
            gi.full &= redf[w];
        }
        const double d0 = tg - times[0];
        gi.toff_h = (float)d0;
        gi.toff_l = (float)(d0 - (double)gi.toff_h);
        gi.pad = 0.0f;
        grp[g] = gi;
    }
}

}  // namespace rr
