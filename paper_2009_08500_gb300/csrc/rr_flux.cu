// Fused light-curve kernels: time -> phase -> z -> Eq. 5 -> mean over
// sub-exposures, for a tile of parameter vectors x a tile of times.
//
// Tiling: a CTA of kBlock threads owns kPtTile consecutive times (kPPT per
// thread, strided by kBlock so that each store of a warp covers 32
// consecutive floats) and `pv_tile` consecutive parameter vectors.  The pv
// records of the tile are staged into shared memory by one bulk async copy
// (TMA engine, mbarrier completion); every thread then loops over the
// tile's pvs, reusing its times from registers.
//
// Mixed precision (FP32 bulk):
//  * per time, once per CTA: dt = t - t_ref in FP64, kept as a float pair
//    (dh, dl) -- t_ref is the first time of the tile;
//  * per (CTA, pv), FP64: A = frac((t_ref - T0) / P) as a float pair;
//  * per (pv, time): coarse phase psi = A + dh / P with one FMA.  If the
//    whole exposure lies outside the pv's transit window the point is 1
//    exactly and nothing else is computed.  Otherwise the phase is formed in
//    float-float (error ~1e-9 of a cycle) and every sub-exposure goes
//    through Kepler (FP32 Newton in the offset form, FP64 above e = 0.8),
//    the projected distance, the covered area and the profile row lookup.
// FP64 form: the same structure with every step in FP64 and the phase
// reduced per sub-exposure as tau = t_s - T0 - P rint((t_s - T0) / P).
#include "rr_device.cuh"

namespace rr {

// Mean of Eq. 5 over the sub-exposures of one (pv, time); called only for
// points whose exposure overlaps the transit window.
__device__ __noinline__ float flux_point32(const PvHead<float>& H, const PvPb<float>& pbc,
                                           const float* __restrict__ row, int ng, float dh, float dl,
                                           float Ah, float Al, int ss, float first, float step,
                                           float inv_ss, bool& bad) {
    const Phase32 ph = precise_phase(dh, dl, Ah, Al, H.Bh, H.Bl);
    const float two_pi = 6.28318530717958647692f;
    float acc = 0.0f;
    #pragma unroll 1
    for (int s = 0; s < ss; ++s) {
        const float off = fmaf((float)s, step, first) * H.Bh;   // sub-exposure offset, cycles
        float x = (ph.fr_h + off) + ph.fr_l;
        x -= rintf(x);
        const float dM = two_pi * x;
        if (fabsf(dM) > pbc.win_s) continue;
        double dMd = 0.0;
        if (H.flags & kPvKepler64) {
            double xd = ((double)ph.fr_h + (double)off) + (double)ph.fr_l;
            xd -= rint(xd);
            dMd = 6.283185307179586476925 * xd;
        }
        const Orbit32 o = orbit32(H, dM, dMd);
        if (!o.ok) {
            bad = true;
            return __int_as_float(0x7fc00000);
        }
        const float g = o.z * pbc.inv1pk;
        if (!o.front || g >= 1.0f) continue;
        float d0, d1, sl;
        int cell;
        const float A = covered_area<float, false>(pbc.k, o.z, d0, d1);
        const float Ib = lerp_row<float>(row, ng, g, sl, cell);
        acc = fmaf(A, Ib, acc);
    }
    return 1.0f - acc * inv_ss;
}

__global__ void __launch_bounds__(kBlock) rr_flux_mixed_kernel(const double* __restrict__ times,
                                                               const int32_t* __restrict__ pb_index,
                                                               int npt, int npv, PbParams pbp, RecLayout L,
                                                               int pv_tile, const char* __restrict__ records,
                                                               float* __restrict__ flux,
                                                               int32_t* __restrict__ pv_status, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    float* red = reinterpret_cast<float*>(smem + 16);                  // kBlock / 32 floats
    float4* cta = reinterpret_cast<float4*>(smem + 16 + 16 * 4);      // per pv: Ah, Al, mref, margin
    char* recs = reinterpret_cast<char*>(smem + 16 + 16 * 4 + 16 * kMaxPvTile);

    const int tid = threadIdx.x;
    const int pt0 = blockIdx.x * kPtTile;
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
    // times of this tile (FP64 difference to the tile's first time, kept as a float pair)
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
            pbv[j] = (pb >= 0 && pb < L.npb) ? pb : L.npb;   // L.npb marks an invalid index (NaN)
            maxdt = fmaxf(maxdt, fabsf(dh[j]));
        }
    }
    maxdt = warp_max(maxdt);
    if ((tid & 31) == 0) red[tid >> 5] = maxdt;
    __syncthreads();   // also publishes the barrier initialisation
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
            // coarse-phase error bound (FMA of a rounded dh and 1/P), radians
            c.w = 1.5e-6f * (maxdt * H.Bh + 1.0f);
        }
        cta[tid] = c;
    }
    __syncthreads();

    const float nanf_ = __int_as_float(0x7fc00000);
    const float two_pi = 6.28318530717958647692f;
    #pragma unroll 1
    for (int i = 0; i < npv_t; ++i) {
        const char* rec = recs + (size_t)i * L.bytes;
        const PvHead<float>& H = *reinterpret_cast<const PvHead<float>*>(rec);
        const PvPb<float>* PB = reinterpret_cast<const PvPb<float>*>(rec + L.off_pb);
        const float* rows = reinterpret_cast<const float*>(rec + L.off_rows);
        float* out = flux + (size_t)(pv0 + i) * npt;
        if (H.status != 0) {
            #pragma unroll
            for (int j = 0; j < kPPT; ++j)
                if (pbv[j] >= 0) __stcs(out + pt0 + j * kBlock + tid, nanf_);
            continue;
        }
        const float4 c = cta[i];
        const float Bh = H.Bh;
        bool bad = false;
        #pragma unroll
        for (int j = 0; j < kPPT; ++j) {
            const int pb = pbv[j];
            if (pb < 0) continue;
            float f;
            if (pb >= L.npb) {
                f = nanf_;
            } else {
                const PvPb<float> pbc = PB[pb];
                const float psi = fmaf(dh[j], Bh, c.x);
                const float phi = two_pi * (psi - rintf(psi));
                f = 1.0f;
                if (fabsf(phi) <= pbc.win_p + c.w)
                    f = flux_point32(H, pbc, rows + (size_t)pb * L.rows_per_pb * L.ng_pad, L.ng, dh[j],
                                     dl[j], c.x, c.y, pbp.ss[pb], pbp.first[pb], pbp.step[pb],
                                     pbp.inv_ss[pb], bad);
            }
            __stcs(out + pt0 + j * kBlock + tid, f);
        }
        if (bad && pv_status) atomicOr(pv_status + pv0 + i, RR_PV_KEPLER);
    }
}

// ----------------------------- FP64 form -----------------------------------

__device__ __noinline__ double flux_point64(const PvHead<double>& H, const PvPb<double>& pbc,
                                            const double* __restrict__ row, int ng, double t, int ss,
                                            double exptime, bool& bad) {
    double acc = 0.0;
    #pragma unroll 1
    for (int s = 0; s < ss; ++s) {
        const double ts = t + exptime * ((s + 0.5) / ss - 0.5);
        double tau = ts - H.T0;
        tau = fma(-rint(tau * H.invP), H.P, tau);
        const double dM = H.n * tau;
        if (fabs(dM) > pbc.win_s) continue;
        const Orbit64 o = orbit64(H, dM);
        if (!o.ok) {
            bad = true;
            return __longlong_as_double(0x7ff8000000000000ll);
        }
        const double g = o.z * pbc.inv1pk;
        if (!o.front || g >= 1.0) continue;
        double d0, d1, sl;
        int cell;
        const double A = covered_area<double, false>(pbc.k, o.z, d0, d1);
        const double Ib = lerp_row<double>(row, ng, g, sl, cell);
        acc += A * Ib;
    }
    return 1.0 - acc / ss;
}

__global__ void __launch_bounds__(kBlock) rr_flux_fp64_kernel(const double* __restrict__ times,
                                                              const int32_t* __restrict__ pb_index,
                                                              int npt, int npv, PbParams pbp, RecLayout L,
                                                              int pv_tile, const char* __restrict__ records,
                                                              double* __restrict__ flux,
                                                              int32_t* __restrict__ pv_status, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    char* recs = reinterpret_cast<char*>(smem + 16 + 16 * 4 + 16 * kMaxPvTile);
    const int tid = threadIdx.x;
    const int pt0 = blockIdx.x * kPtTile;
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
            pbv[j] = (pb >= 0 && pb < L.npb) ? pb : L.npb;   // L.npb marks an invalid index (NaN)
        }
    }
    const double nan_ = __longlong_as_double(0x7ff8000000000000ll);
    #pragma unroll 1
    for (int i = 0; i < npv_t; ++i) {
        const char* rec = recs + (size_t)i * L.bytes;
        const PvHead<double>& H = *reinterpret_cast<const PvHead<double>*>(rec);
        const PvPb<double>* PB = reinterpret_cast<const PvPb<double>*>(rec + L.off_pb);
        const double* rows = reinterpret_cast<const double*>(rec + L.off_rows);
        double* out = flux + (size_t)(pv0 + i) * npt;
        bool bad = false;
        #pragma unroll
        for (int j = 0; j < kPPT; ++j) {
            const int pb = pbv[j];
            if (pb < 0) continue;
            double f;
            if (H.status != 0 || pb >= L.npb) {
                f = nan_;
            } else {
                const PvPb<double> pbc = PB[pb];
                double tau = tv[j] - H.T0;
                tau = fma(-rint(tau * H.invP), H.P, tau);
                f = 1.0;
                if (fabs(H.n * tau) <= pbc.win_p + 1e-9)
                    f = flux_point64(H, pbc, rows + (size_t)pb * L.rows_per_pb * L.ng_pad, L.ng, tv[j],
                                     pbp.ss[pb], pbp.exptime[pb], bad);
            }
            __stcs(out + pt0 + j * kBlock + tid, f);
        }
        if (bad && pv_status) atomicOr(pv_status + pv0 + i, RR_PV_KEPLER);
    }
}

static size_t flux_smem(int pv_tile, int rec_bytes) {
    return 16 + 16 * 4 + 16 * kMaxPvTile + (size_t)pv_tile * rec_bytes;
}

int pv_tile_for(int rec_bytes) {
    int t = kSmemTarget / rec_bytes;
    if (t < 1) t = 1;
    if (t > kMaxPvTile) t = kMaxPvTile;
    return t;
}

cudaError_t launch_flux(rr_ctx* c, const double* times, const int32_t* pb_index, int npt, int npv,
                        const PbParams& pbp, const void* records, void* flux, int32_t* pv_status,
                        cudaStream_t s) {
    const bool f64 = c->cfg.precision == RR_PREC_FP64;
    RecLayout L = f64 ? make_layout<double>(c->cfg.npb, c->cfg.ng, c->nldc, false)
                      : make_layout<float>(c->cfg.npb, c->cfg.ng, c->nldc, false);
    const int pv_tile = pv_tile_for(L.bytes);
    const size_t smem = flux_smem(pv_tile, L.bytes);
    dim3 grid((npt + kPtTile - 1) / kPtTile, (npv + pv_tile - 1) / pv_tile);
    if (smem > kMaxSmem || grid.y > 65535u) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if (f64) {
        e = cudaFuncSetAttribute(rr_flux_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        rr_flux_fp64_kernel<<<grid, kBlock, smem, s>>>(times, pb_index, npt, npv, pbp, L, pv_tile,
                                                       (const char*)records, (double*)flux, pv_status,
                                                       c->d_err);
    } else {
        e = cudaFuncSetAttribute(rr_flux_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        rr_flux_mixed_kernel<<<grid, kBlock, smem, s>>>(times, pb_index, npt, npv, pbp, L, pv_tile,
                                                        (const char*)records, (float*)flux, pv_status,
                                                        c->d_err);
    }
    c->launches++;
    return cudaGetLastError();
}

}  // namespace rr
