// Hand-written adjoint of the light-curve kernels (vector-Jacobian product).
//
// For every (pv, time) with a non-zero cotangent gbar and an exposure that
// overlaps the transit window, every sub-exposure is recomputed in
// registers and differentiated by the chain rule:
//   flux = 1 - (1/ss) sum_s delta_s,  delta = A(z, k) * Ib(g, k),  g = z / (1 + k)
//   Ib   = row / I_star interpolated in g (row interpolated in k, Sect. 3.1.2)
//   dA/dz = -K / z, dA/dk = 2 k kappa1   (covered_area)
//   dIb/dg = in-cell slope, dIb/dk = in-cell lerp of d(row)/dk / I_star,
//   dIb/du_c = in-cell lerp of Q_c (profile coefficient rows)
//   z(T0, P, a, b, e, w) through Kepler's equation in the offset form:
//     z^2 = a^2 P_x^2 + b^2 P_y^2,  P_x, P_y functions of (E, e, w)
//     dE = (dM + sin E de) / (1 - e cos E),
//     dM/dT0 = -n, dM/dP = -n (t - T0) / P, dM/de = dM0/de, dM/dw = dM0/dw.
// Per-thread sums -> warp shuffles -> fixed-order sum over warps (FP64) ->
// one partial per (pv, time tile) in the workspace -> rr_grad_reduce sums the
// tiles in order.  The result for a pv is therefore independent of which
// other pvs share the launch.
#include "rr_device.cuh"

namespace rr {

template <typename R>
struct GradAcc {
    R o[6];     // T0, P, a, b, e, w
    R k;
    R u[4];
};

// Contribution of one sub-exposure; gb = -gbar / ss.
template <typename R, bool DEP>
__device__ __forceinline__ void grad_sample(const PvHead<R>& H, const PvPb<R>& pbc,
                                            const R* __restrict__ rowblk, const RecLayout& L, R z,
                                            R Px, R Py, R S, R V, R psi_tot, R gb, GradAcc<R>& acc,
                                            R* dep, int kslot, int uslot) {
    const R one = R(1);
    R dAdz, dAdk;
    const R A = covered_area<R, true>(pbc.k, z, dAdz, dAdk);
    const R g = z * pbc.inv1pk;
    R sl;
    int i;
    const R Ib = lerp_row<R>(rowblk, L.ng, g, sl, i);
    const R al = g * R(L.ng - 1) - R(i);
    const R dIdg = sl * R(L.ng - 1);
    const R* rk = rowblk + L.ng_pad;
    const R Ik = rk[i] + al * (rk[i + 1] - rk[i]);
    const R ddz = dAdz * Ib + A * dIdg * pbc.inv1pk;
    const R ddk = dAdk * Ib + A * (Ik - dIdg * z * pbc.inv1pk * pbc.inv1pk);

    // orbit partials.  With den = r / a = 1 - e cos E and u = w + f the sky
    // coordinates are P_x = den cos u, P_y = den sin u.  The e and w
    // derivatives are written so that every small factor is formed directly
    // (differences from conjunction: dsinE = sin E - sin E0, dden = den -
    // den0), since at conjunction dP_x/de and dP/dw vanish identically and a
    // difference of O(1) terms would lose all FP32 digits there:
    //   dE/de  = (dsinE - den0 sE0 / (1 - e^2)) / den
    //   du/de  = [(den0 dsinE + dden sin E) / se + se dsinE] / den^2
    //   dE/dw  = dM0/dw / den = -den0^2 / (se den)
    //   du/dw  = dden (den + den0) / den^2
    //   d den  = -cos E de + e sin E dE
    //   dP_x = d den P_x / den - P_y du,  dP_y = d den P_y / den + P_x du
    const R omV = one - V;
    const R dden = H.ecE0 * V + H.esE0 * S;
    const R den0 = one - H.ecE0;
    const R den = den0 + dden;
    const R invden = one / den;
    const R dsinE = H.cE0 * S - H.sE0 * V;
    const R sinE = H.sE0 + dsinE;
    const R cosE = H.cE0 * omV - H.sE0 * S;
    const R dPxdE = H.ax1 * S + H.ax2 * omV;
    const R dPydE = H.ay1 * S + H.ay2 * omV;
    const R invz = one / z;
    const R zE = (H.a2 * Px * dPxdE + H.b2 * Py * dPydE) * invz;
    const R inv_se = H.inv_se;
    const R ce = -(H.dM0de + H.sE0);                    // den0 sE0 / (1 - e^2)
    const R dEde = (dsinE - ce) * invden;
    const R ddende = -cosE + H.e * sinE * dEde;
    const R dude = ((den0 * dsinE + dden * sinE) * inv_se + H.se * dsinE) * invden * invden;
    const R dPxde = ddende * Px * invden - Py * dude;
    const R dPyde = ddende * Py * invden + Px * dude;
    const R dEdw = H.dM0dw * invden;
    const R ddendw = H.e * sinE * dEdw;
    const R dudw = dden * (den + den0) * invden * invden;
    const R dPxdw = ddendw * Px * invden - Py * dudw;
    const R dPydw = ddendw * Py * invden + Px * dudw;
    const R c = gb * ddz;
    acc.o[0] += c * (zE * (-H.n * invden));
    acc.o[1] += c * (zE * (-H.n * psi_tot * invden));
    acc.o[2] += c * (H.a * Px * Px * invz);
    acc.o[3] += c * (H.b * Py * Py * invz);
    acc.o[4] += c * ((H.a2 * Px * dPxde + H.b2 * Py * dPyde) * invz);
    acc.o[5] += c * ((H.a2 * Px * dPxdw + H.b2 * Py * dPydw) * invz);
    const R gk = gb * ddk;
    if (DEP) dep[(kslot - 6) * kBlock] += gk; else acc.k += gk;
    #pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        if (cc < L.nldc) {
            const R* rq = rowblk + (size_t)(2 + cc) * L.ng_pad;
            const R Q = rq[i] + al * (rq[i + 1] - rq[i]);
            if (DEP) dep[(uslot + cc - 6) * kBlock] += gb * A * Q; else acc.u[cc] += gb * A * Q;
        }
    }
}

// Sum one value per thread over the CTA (deterministic order): warp
// shuffles, then warps in index order in FP64.  All threads must call.
template <typename R>
__device__ __forceinline__ void block_partials(const GradAcc<R>& acc, const R* dep, int nacc, bool DEP,
                                               double* wred, double* out) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // register slots (compile-time indices)
    #pragma unroll
    for (int j = 0; j < 11; ++j) {
        if (j < nacc && (j < 6 || !DEP)) {
            R v = j < 6 ? acc.o[j < 6 ? j : 0] : (j == 6 ? acc.k : acc.u[j >= 7 ? j - 7 : 0]);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) wred[warp * nacc + j] = (double)v;
        }
    }
    if (DEP) {
        for (int j = 6; j < nacc; ++j) {
            R v = dep[(j - 6) * kBlock];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) wred[warp * nacc + j] = (double)v;
        }
    }
    __syncthreads();
    if (tid < nacc) {
        double s = 0.0;
        for (int w = 0; w < (kBlock >> 5); ++w) s += wred[w * nacc + tid];
        out[tid] = s;
    }
    __syncthreads();
}

template <bool DEP>
__global__ void __launch_bounds__(kBlock) rr_grad_mixed_kernel(
    const double* __restrict__ times, const int32_t* __restrict__ pb_index, int npt, int npv,
    PbParams pbp, RecLayout L, int pv_tile, const char* __restrict__ records,
    const float* __restrict__ gflux, double* __restrict__ partials, int nacc, int chromatic,
    int32_t* __restrict__ pv_status, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    float* red = reinterpret_cast<float*>(smem + 16);
    float4* cta = reinterpret_cast<float4*>(smem + 16 + 16 * 4);
    char* recs = reinterpret_cast<char*>(smem + 16 + 16 * 4 + 16 * kMaxPvTile);
    double* wred = reinterpret_cast<double*>(recs + (size_t)pv_tile * L.bytes);
    float* depcols = reinterpret_cast<float*>(wred + (kBlock >> 5) * nacc);

    const int tid = threadIdx.x;
    const int tile = blockIdx.x, ntiles = gridDim.x;
    const int pt0 = tile * kPtTile;
    const int pv0 = blockIdx.y * pv_tile;
    const int npv_t = min(pv_tile, npv - pv0);
    const uint32_t bytes = (uint32_t)npv_t * (uint32_t)L.bytes;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, bytes);
        const char* src = records + (size_t)pv0 * L.bytes;
        for (uint32_t off = 0; off < bytes; off += 65536u) {
            const uint32_t n = bytes - off < 65536u ? bytes - off : 65536u;
            bulk_g2s(recs + off, src + off, n, bar);
        }
    }
    const double t_ref = times[pt0];
    float dh[kPPT], dl[kPPT];
    int pbv[kPPT];
    float maxdt = 0.0f;
    #pragma unroll
    for (int j = 0; j < kPPT; ++j) {
        const int p = pt0 + j * kBlock + tid;
        pbv[j] = -1;
        dh[j] = 0.0f;
        dl[j] = 0.0f;
        if (p < npt) {
            const double dt = __ldg(times + p) - t_ref;
            dh[j] = (float)dt;
            dl[j] = (float)(dt - (double)dh[j]);
            const int pb = pb_index ? __ldg(pb_index + p) : 0;
            pbv[j] = (pb >= 0 && pb < L.npb) ? pb : -1;
            maxdt = fmaxf(maxdt, fabsf(dh[j]));
        }
    }
    maxdt = warp_max(maxdt);
    if ((tid & 31) == 0) red[tid >> 5] = maxdt;
    __syncthreads();
    if (tid < 32) {
        float v = tid < (kBlock >> 5) ? red[tid] : 0.0f;
        v = warp_max(v);
        if (tid == 0) red[0] = v;
    }
    bool ok = mbar_wait_bounded(bar, 0);
    if (!ok) {
        if (tid == 0) atomicExch(err, kErrBarrierTimeout);
        mbar_wait_bounded(bar, 0);
    }
    if (__syncthreads_or(ok ? 0 : 1)) return;
    maxdt = red[0];
    if (tid < npv_t) {
        const PvHead<float>& H = *reinterpret_cast<const PvHead<float>*>(recs + (size_t)tid * L.bytes);
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (H.status == 0) {
            const double psi = (t_ref - H.T0) * H.invP;
            const double m = rint(psi);
            const double A = psi - m;
            c.x = (float)A;
            c.y = (float)(A - (double)c.x);
            c.z = (float)m;
            c.w = 1.5e-6f * (maxdt * H.Bh + 1.0f);
        }
        cta[tid] = c;
    }
    __syncthreads();

    const float two_pi = 6.28318530717958647692f;
    const int nkp = chromatic ? L.npb : 1;
    float* dep = DEP ? depcols + tid : nullptr;
    #pragma unroll 1
    for (int i = 0; i < npv_t; ++i) {
        const char* rec = recs + (size_t)i * L.bytes;
        const PvHead<float>& H = *reinterpret_cast<const PvHead<float>*>(rec);
        if (H.status != 0) continue;   // uniform over the CTA
        const PvPb<float>* PB = reinterpret_cast<const PvPb<float>*>(rec + L.off_pb);
        const float* rows = reinterpret_cast<const float*>(rec + L.off_rows);
        const float4 c = cta[i];
        const float* gf = gflux + (size_t)(pv0 + i) * npt;
        GradAcc<float> acc;
        #pragma unroll
        for (int j = 0; j < 6; ++j) acc.o[j] = 0.0f;
        acc.k = 0.0f;
        #pragma unroll
        for (int j = 0; j < 4; ++j) acc.u[j] = 0.0f;
        if (DEP)
            for (int j = 6; j < nacc; ++j) dep[(j - 6) * kBlock] = 0.0f;
        bool bad = false;
        #pragma unroll 1
        for (int j = 0; j < kPPT; ++j) {
            const int pb = pbv[j];
            if (pb < 0) continue;
            const PvPb<float> pbc = PB[pb];
            const float psi = fmaf(dh[j], H.Bh, c.x);
            const float phi = two_pi * (psi - rintf(psi));
            if (fabsf(phi) > pbc.win_p + c.w) continue;
            const int p = pt0 + j * kBlock + tid;
            const float gb = -__ldg(gf + p) * pbp.inv_ss[pb];
            if (gb == 0.0f) continue;
            const float* rowblk = rows + (size_t)pb * L.rows_per_pb * L.ng_pad;
            const int kslot = 6 + (chromatic ? pb : 0);
            const int uslot = 6 + nkp + pb * L.nldc;
            const Phase32 ph = precise_phase(dh[j], dl[j], c.x, c.y, H.Bh, H.Bl);
            const int ss = pbp.ss[pb];
            #pragma unroll 1
            for (int s = 0; s < ss; ++s) {
                const float off = fmaf((float)s, pbp.step[pb], pbp.first[pb]) * H.Bh;
                const float xr = (ph.fr_h + off) + ph.fr_l;
                const float r = rintf(xr);
                const float x = xr - r;
                const float dM = two_pi * x;
                if (fabsf(dM) > pbc.win_s) continue;
                double dMd = 0.0;
                if (H.flags & kPvKepler64) {
                    double xd = ((double)ph.fr_h + (double)off) + (double)ph.fr_l;
                    xd -= rint(xd);
                    dMd = 6.283185307179586476925 * xd;
                }
                const Orbit32 o = orbit32(H, dM, dMd);
                if (!o.ok) { bad = true; continue; }
                const float g = o.z * pbc.inv1pk;
                if (!o.front || g >= 1.0f) continue;
                const float psi_tot = ((c.z + ph.m) + r) + x;   // (t_s - T0) / P
                grad_sample<float, DEP>(H, pbc, rowblk, L, o.z, o.Px, o.Py, o.S, o.V, psi_tot, gb, acc, dep,
                                        kslot, uslot);
            }
        }
        if (bad) {
            acc.o[0] = __int_as_float(0x7fc00000);
            if (pv_status) atomicOr(pv_status + pv0 + i, RR_PV_KEPLER);
        }
        block_partials<float>(acc, dep, nacc, DEP, wred, partials + ((size_t)(pv0 + i) * ntiles + tile) * nacc);
    }
}

template <bool DEP>
__global__ void __launch_bounds__(kBlock) rr_grad_fp64_kernel(
    const double* __restrict__ times, const int32_t* __restrict__ pb_index, int npt, int npv,
    PbParams pbp, RecLayout L, int pv_tile, const char* __restrict__ records,
    const double* __restrict__ gflux, double* __restrict__ partials, int nacc, int chromatic,
    int32_t* __restrict__ pv_status, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    char* recs = reinterpret_cast<char*>(smem + 16 + 16 * 4 + 16 * kMaxPvTile);
    double* wred = reinterpret_cast<double*>(recs + (size_t)pv_tile * L.bytes);
    double* depcols = wred + (kBlock >> 5) * nacc;
    const int tid = threadIdx.x;
    const int tile = blockIdx.x, ntiles = gridDim.x;
    const int pt0 = tile * kPtTile;
    const int pv0 = blockIdx.y * pv_tile;
    const int npv_t = min(pv_tile, npv - pv0);
    if (!stage_to_smem(recs, records + (size_t)pv0 * L.bytes, (uint32_t)npv_t * (uint32_t)L.bytes, bar, err))
        return;
    double tv[kPPT];
    int pbv[kPPT];
    #pragma unroll
    for (int j = 0; j < kPPT; ++j) {
        const int p = pt0 + j * kBlock + tid;
        pbv[j] = -1;
        tv[j] = 0.0;
        if (p < npt) {
            tv[j] = __ldg(times + p);
            const int pb = pb_index ? __ldg(pb_index + p) : 0;
            pbv[j] = (pb >= 0 && pb < L.npb) ? pb : -1;
        }
    }
    const int nkp = chromatic ? L.npb : 1;
    double* dep = DEP ? depcols + tid : nullptr;
    #pragma unroll 1
    for (int i = 0; i < npv_t; ++i) {
        const char* rec = recs + (size_t)i * L.bytes;
        const PvHead<double>& H = *reinterpret_cast<const PvHead<double>*>(rec);
        if (H.status != 0) continue;
        const PvPb<double>* PB = reinterpret_cast<const PvPb<double>*>(rec + L.off_pb);
        const double* rows = reinterpret_cast<const double*>(rec + L.off_rows);
        const double* gf = gflux + (size_t)(pv0 + i) * npt;
        GradAcc<double> acc;
        for (int j = 0; j < 6; ++j) acc.o[j] = 0.0;
        acc.k = 0.0;
        for (int j = 0; j < 4; ++j) acc.u[j] = 0.0;
        if (DEP)
            for (int j = 6; j < nacc; ++j) dep[(j - 6) * kBlock] = 0.0;
        bool bad = false;
        #pragma unroll 1
        for (int j = 0; j < kPPT; ++j) {
            const int pb = pbv[j];
            if (pb < 0) continue;
            const PvPb<double> pbc = PB[pb];
            double tau0 = tv[j] - H.T0;
            tau0 = fma(-rint(tau0 * H.invP), H.P, tau0);
            if (fabs(H.n * tau0) > pbc.win_p + 1e-9) continue;
            const int p = pt0 + j * kBlock + tid;
            const int ss = pbp.ss[pb];
            const double gb = -__ldg(gf + p) / ss;
            if (gb == 0.0) continue;
            const double* rowblk = rows + (size_t)pb * L.rows_per_pb * L.ng_pad;
            const int kslot = 6 + (chromatic ? pb : 0);
            const int uslot = 6 + nkp + pb * L.nldc;
            #pragma unroll 1
            for (int s = 0; s < ss; ++s) {
                const double ts = tv[j] + pbp.exptime[pb] * ((s + 0.5) / ss - 0.5);
                const double tau = ts - H.T0;
                const double m = rint(tau * H.invP);
                const double tr = fma(-m, H.P, tau);
                const double dM = H.n * tr;
                if (fabs(dM) > pbc.win_s) continue;
                const Orbit64 o = orbit64(H, dM);
                if (!o.ok) { bad = true; continue; }
                const double g = o.z * pbc.inv1pk;
                if (!o.front || g >= 1.0) continue;
                const double psi_tot = m + tr * H.invP;
                grad_sample<double, DEP>(H, pbc, rowblk, L, o.z, o.Px, o.Py, o.S, o.V, psi_tot, gb, acc, dep,
                                         kslot, uslot);
            }
        }
        if (bad) {
            acc.o[0] = __longlong_as_double(0x7ff8000000000000ll);
            if (pv_status) atomicOr(pv_status + pv0 + i, RR_PV_KEPLER);
        }
        block_partials<double>(acc, dep, nacc, DEP, wred, partials + ((size_t)(pv0 + i) * ntiles + tile) * nacc);
    }
}

// Sum the per-tile partials of each pv in tile order; map the quadratic
// coefficients (u1, u2) to Kipping's (q1, q2) where that law is used:
//   d/dq1 = d/du1 q2 / sqrt(q1) + d/du2 (1 - 2 q2) / (2 sqrt(q1))
//   d/dq2 = d/du1 2 sqrt(q1) - d/du2 2 sqrt(q1)
// Invalid pvs get NaN rows.
template <typename R>
__global__ void rr_grad_reduce_kernel(const double* __restrict__ partials, int ntiles, int nacc, int npv,
                                      const char* __restrict__ records, int rec_bytes,
                                      const double* __restrict__ params, int nparam, int ld_model, int npb,
                                      int nkp, double* __restrict__ grad) {
    const int pv = blockIdx.x * blockDim.y + threadIdx.y;
    if (pv >= npv) return;
    const PvHead<R>& H = *reinterpret_cast<const PvHead<R>*>(records + (size_t)pv * rec_bytes);
    double* out = grad + (size_t)pv * nparam;
    const double nan_ = __longlong_as_double(0x7ff8000000000000ll);
    for (int j = threadIdx.x; j < nacc; j += blockDim.x) {
        double s = 0.0;
        const double* pp = partials + (size_t)pv * ntiles * nacc + j;
        for (int t = 0; t < ntiles; ++t) s += pp[(size_t)t * nacc];
        out[j] = H.status != 0 ? nan_ : s;
    }
    __syncwarp();
    if (ld_model == RR_LD_QUADRATIC_TRI && threadIdx.x == 0 && H.status == 0) {
        const double* row = params + (size_t)pv * nparam;
        for (int pb = 0; pb < npb; ++pb) {
            const int o = 6 + nkp + 2 * pb;
            const double q1 = row[o], q2 = row[o + 1];
            const double sq = sqrt(q1);
            const double g1 = out[o], g2 = out[o + 1];
            out[o] = g1 * q2 / sq + g2 * (1.0 - 2.0 * q2) / (2.0 * sq);
            out[o + 1] = g1 * 2.0 * sq - g2 * 2.0 * sq;
        }
    }
}

static size_t grad_smem(int pv_tile, const RecLayout& L, int nacc, bool dep, size_t rsize) {
    size_t s = 16 + 16 * 4 + 16 * kMaxPvTile + (size_t)pv_tile * L.bytes + (size_t)(kBlock >> 5) * nacc * 8;
    if (dep) s += (size_t)(nacc - 6) * kBlock * rsize;
    return s;
}

size_t partials_bytes(const rr_ctx* c, int npv, int npt) {
    const size_t ntiles = ((size_t)npt + kPtTile - 1) / kPtTile;
    return (size_t)npv * ntiles * (size_t)c->nparam * sizeof(double);
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_grad(rr_ctx* c, const double* times, const int32_t* pb_index, int npt, int npv,
                        const PbParams& pbp, const void* records, const void* grad_flux, double* partials,
                        int32_t* pv_status, cudaStream_t s) {
    const bool f64 = c->cfg.precision == RR_PREC_FP64;
    RecLayout L = f64 ? make_layout<double>(c->cfg.npb, c->cfg.ng, c->nldc, true)
                      : make_layout<float>(c->cfg.npb, c->cfg.ng, c->nldc, true);
    const int nacc = c->nparam;
    const bool dep = nacc > 11 || (c->cfg.npb > 1 && (c->cfg.chromatic || c->nldc > 0));
    const int pv_tile = pv_tile_for(L.bytes);
    const size_t smem = grad_smem(pv_tile, L, nacc, dep, f64 ? 8 : 4);
    const int ntiles = (npt + kPtTile - 1) / kPtTile;
    dim3 grid(ntiles, (npv + pv_tile - 1) / pv_tile);
    if (smem > kMaxSmem || grid.y > 65535u) return cudaErrorInvalidConfiguration;
    cudaError_t e;
#define RR_LAUNCH_GRAD(KERNEL, GT)                                                                          \
    do {                                                                                                    \
        e = set_smem(KERNEL, smem);                                                                         \
        if (e != cudaSuccess) return e;                                                                     \
        KERNEL<<<grid, kBlock, smem, s>>>(times, pb_index, npt, npv, pbp, L, pv_tile, (const char*)records, \
                                          (const GT*)grad_flux, partials, nacc, c->cfg.chromatic,          \
                                          pv_status, c->d_err);                                             \
    } while (0)
    if (f64) {
        if (dep) RR_LAUNCH_GRAD(rr_grad_fp64_kernel<true>, double);
        else RR_LAUNCH_GRAD(rr_grad_fp64_kernel<false>, double);
    } else {
        if (dep) RR_LAUNCH_GRAD(rr_grad_mixed_kernel<true>, float);
        else RR_LAUNCH_GRAD(rr_grad_mixed_kernel<false>, float);
    }
#undef RR_LAUNCH_GRAD
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_grad_reduce(rr_ctx* c, int npt, const double* params, int npv, const void* records,
                               const double* partials, double* grad_params, cudaStream_t s) {
    const bool f64 = c->cfg.precision == RR_PREC_FP64;
    RecLayout L = f64 ? make_layout<double>(c->cfg.npb, c->cfg.ng, c->nldc, true)
                      : make_layout<float>(c->cfg.npb, c->cfg.ng, c->nldc, true);
    const int nacc = c->nparam;
    const int ntiles = (npt + kPtTile - 1) / kPtTile;
    dim3 rb(32, 4);
    const int nkp = c->cfg.chromatic ? c->cfg.npb : 1;
    if (f64)
        rr_grad_reduce_kernel<double><<<(npv + 3) / 4, rb, 0, s>>>(partials, ntiles, nacc, npv, (const char*)records,
                                                                   L.bytes, params, c->nparam, c->cfg.ld_model,
                                                                   c->cfg.npb, nkp, grad_params);
    else
        rr_grad_reduce_kernel<float><<<(npv + 3) / 4, rb, 0, s>>>(partials, ntiles, nacc, npv, (const char*)records,
                                                                  L.bytes, params, c->nparam, c->cfg.ld_model,
                                                                  c->cfg.npb, nkp, grad_params);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace rr
