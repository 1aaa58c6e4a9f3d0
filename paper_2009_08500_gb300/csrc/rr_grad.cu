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
// The FP32 kernel takes the flux kernel's groups and work items (every warp
// alternates between deciding a group and evaluating an item).  Sums: per
// lane over an item's samples -> a warp reduce-scatter in a fixed order ->
// one slot per (pv, group) in shared memory -> per (pv, CTA chunk) in the
// workspace -> rr_grad_finish_kernel sums the chunks in order in FP64 (and
// applies the Kipping chain rule).  The chunking depends on npt only, so the
// result for a pv is independent of which other pvs share the launch and of
// which warp took which item.
#include "rr_device.cuh"

namespace rr {

template <typename R>
struct GradAcc {
    R o[6];     // T0, P, a, b, e, w
    R k;
    R u[4];
};

// Contribution of one sub-exposure; gb = -gbar / ss.  rowblk points to
// global memory (read through the read-only data path).
// f1 = 1 + k - z and f3 = z - (1 - k): the contact factors of the covered
// area; i and al: the g cell of the sample (the lower cell on a node, clamped
// to ng - 2) and its position in the cell (both from float-float near the
// contacts and the cell edges in the mixed adjoint).
template <typename R, bool DEP>
__device__ __forceinline__ void grad_sample(const PvHead<R>& H, const PvPb<R>& pbc,
                                            const R* __restrict__ rowblk, const RecLayout& L, R z, R f1, R f3,
                                            int i, R al, R Px, R Py, R S, R V, R psi_tot, R gb, GradAcc<R>& acc,
                                            R* dep, int kslot, int uslot) {
    const R one = R(1);
    R dAdz, dAdk;
    const R A = covered_area_f13<R, true>(pbc.k, z, f1, f3, dAdz, dAdk);
    const R d = __ldg(rowblk + L.ng_pad + i);         // row[i+1] - row[i]
    const R Ib = __ldg(rowblk + i) + al * d;
    const R dIdg = d * R(L.ng - 1);
    const R* rk = rowblk + 2 * L.ng_pad;
    const R rk0 = __ldg(rk + i);
    const R Ik = rk0 + al * (__ldg(rk + i + 1) - rk0);
    const R ddz = dAdz * Ib + A * dIdg * pbc.inv1pk;
    // k enters through the area and g (own k) and through the row (the weights' k)
    const R kown = dAdk * Ib - A * dIdg * z * pbc.inv1pk * pbc.inv1pk;
    const R krow = A * Ik;

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
    const R invden = d_rcp(den);
    const R dsinE = H.cE0 * S - H.sE0 * V;
    const R sinE = H.sE0 + dsinE;
    const R cosE = H.cE0 * omV - H.sE0 * S;
    const R dPxdE = H.ax1 * S + H.ax2 * omV;
    const R dPydE = H.ay1 * S + H.ay2 * omV;
    const R invz = d_rcp(z);
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
    if (DEP) {
        if (L.kbar_slot >= 0) {
            // shared weights: the row's part belongs to the mean k (spread over every k later)
            dep[(kslot - 6) * kBlock] += gb * kown;
            dep[(L.kbar_slot - 6) * kBlock] += gb * krow;
        } else {
            dep[(kslot - 6) * kBlock] += gb * (kown + krow);
        }
    } else {
        acc.k += gb * (kown + krow);
    }
    #pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        if (cc < L.nldc) {
            const R* rq = rowblk + (size_t)(3 + cc) * L.ng_pad;
            const R q0 = __ldg(rq + i);
            const R Q = q0 + al * (__ldg(rq + i + 1) - q0);
            if (DEP) dep[(uslot + cc - 6) * kBlock] += gb * A * Q; else acc.u[cc] += gb * A * Q;
        }
    }
}

// Sum one accumulator set over a warp (shuffles, fixed order) and store it
// in the warp's slot of the CTA's partial-sum table.  Skipped (zeros) when
// no lane of the warp contributed.  All lanes of the warp must call.
template <typename R, bool DEP>
__device__ __forceinline__ void warp_partials(const GradAcc<R>& acc, const R* dep, int nacc, bool any,
                                              R* slot /* [nacc] of this warp */) {
    const int lane = threadIdx.x & 31;
    if (!__any_sync(0xffffffffu, any)) {
        for (int j = lane; j < nacc; j += 32) slot[j] = R(0);
        return;
    }
    #pragma unroll
    for (int j = 0; j < 11; ++j) {
        if (j < nacc && (j < 6 || !DEP)) {
            R v = j < 6 ? acc.o[j < 6 ? j : 0] : (j == 6 ? acc.k : acc.u[j >= 7 ? j - 7 : 0]);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) slot[j] = v;
        }
    }
    if (DEP) {
        for (int j = 6; j < nacc; ++j) {
            R v = dep[(j - 6) * kBlock];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) slot[j] = v;
        }
    }
}

// Sum of 16 per-lane values over the warp by recursive halving (reduce-
// scatter): each step exchanges half of the remaining values with the partner
// lane and keeps the other half, so that lane l ends with the warp total of
// value idx(l) (held by lanes 2m and 2m + 1): 16 shuffles instead of 5 per
// value.  The order of the additions is fixed.
__device__ __forceinline__ float warp_reduce_scatter16(const float (&v)[16], int& idx) {
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
    float a[8], b[4], c[2];
    #pragma unroll
    for (int i = 0; i < 8; ++i)
        a[i] = (h16 ? v[i + 8] : v[i]) + __shfl_xor_sync(0xffffffffu, h16 ? v[i] : v[i + 8], 16);
    #pragma unroll
    for (int i = 0; i < 4; ++i)
        b[i] = (h8 ? a[i + 4] : a[i]) + __shfl_xor_sync(0xffffffffu, h8 ? a[i] : a[i + 4], 8);
    #pragma unroll
    for (int i = 0; i < 2; ++i)
        c[i] = (h4 ? b[i + 2] : b[i]) + __shfl_xor_sync(0xffffffffu, h4 ? b[i] : b[i + 2], 4);
    float d = (h2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h2 ? c[0] : c[1], 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    idx = (h16 ? 8 : 0) + (h8 ? 4 : 0) + (h4 ? 2 : 0) + (h2 ? 1 : 0);
    return d;
}

// Add one accumulator set, summed over the warp (fixed order), to the warp's
// running slot: lane 2j adds value j.
template <typename R, bool DEP>
__device__ __forceinline__ void warp_accumulate(const GradAcc<R>& acc, const R* dep, int nacc, bool any, R* slot) {
    const int lane = threadIdx.x & 31;
    if (!__any_sync(0xffffffffu, any)) return;
    if constexpr (!DEP && sizeof(R) == sizeof(float)) {
        const float v[16] = {acc.o[0], acc.o[1], acc.o[2], acc.o[3], acc.o[4], acc.o[5], acc.k, acc.u[0],
                             acc.u[1], acc.u[2], acc.u[3], 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        int idx;
        const float sum = warp_reduce_scatter16(v, idx);
        if ((lane & 1) == 0 && idx < nacc) slot[idx] += sum;
        return;
    }
    #pragma unroll
    for (int j = 0; j < 11; ++j) {
        if (j < nacc && (j < 6 || !DEP)) {
            R v = j < 6 ? acc.o[j < 6 ? j : 0] : (j == 6 ? acc.k : acc.u[j >= 7 ? j - 7 : 0]);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) slot[j] += v;
        }
    }
    if (DEP) {
        for (int j = 6; j < nacc; ++j) {
            R v = dep[(j - 6) * kBlock];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) slot[j] += v;
        }
    }
}

// After the pv loop: partial[pv][tile][j] = sum over warps (index order) of the
// warp slots, for every valid pv of the tile.
template <typename R>
__device__ __forceinline__ void cta_partials(const R* wpart, const char* recs, int rec_bytes, int npv_t, int nacc,
                                             int pv0, int tile, int ntiles, R* partials) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < npv_t * nacc; idx += blockDim.x) {
        const int i = idx / nacc, j = idx % nacc;
        if (reinterpret_cast<const PvHead<R>*>(recs + (size_t)i * rec_bytes)->status != 0) continue;
        R s = R(0);
        for (int w = 0; w < (kBlock >> 5); ++w) s += wpart[((size_t)i * (kBlock >> 5) + w) * nacc + j];
        partials[((size_t)(pv0 + i) * ntiles + tile) * nacc + j] = s;
    }
}

// After the group loop: partial[pv][chunk][j] = sum over the CTA's groups (index order).
__device__ __forceinline__ void cta_partials_groups(const float* gacc, const char* recs, int rec_bytes, int npv_t,
                                                    int nacc, int gpc, int pv0, int chunk, int nchunks,
                                                    float* partials) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < npv_t * nacc; idx += blockDim.x) {
        const int i = idx / nacc, j = idx % nacc;
        if (reinterpret_cast<const PvHead<float>*>(recs + (size_t)i * rec_bytes)->status != 0) continue;
        float s = 0.0f;
        for (int g = 0; g < gpc; ++g) s += gacc[((size_t)i * gpc + g) * nacc + j];
        partials[((size_t)(pv0 + i) * nchunks + chunk) * nacc + j] = s;
    }
}

// One sample of the FP32 adjoint: the phase fr_h + fr_l cycles from the
// conjunction m + mg cycles after the group's epoch (mg: the pv's cycles at
// the group start), shifted by the sub-exposure offset `off` (cycles; sub-
// exposure s of passband pb); gb is the cotangent weight.  Adds to `acc`;
// returns whether the sample is in transit; sets `bad` on a Kepler failure.
//
// Refinement: within the contact band of a contact point (kContactBand; for
// a grazing transit, whose samples are all near the outer contact,
// kContactBandGrazing) the area's z-derivative
// -K/z varies like sqrt(1 + k - z) (or sqrt(z - 1 + k)), so the ~1e-7 FP32
// rounding of z moves the per-sample derivative by ~1e-7 / (2 (1 + k - z))
// relative (5e-5 at 1e-3 from contact): the largest share of the FP32
// adjoint's error against the FP64 chain rule.  And within kNodeBand of a
// g-node the rounding of g can put the sample in the neighbouring cell,
// whose slope (the derivative of the piecewise-linear profile) differs.  For
// those samples (about 2% of in-transit samples on the population workload)
// z, the contact factors 1 + k - z, z - (1 - k) and the g cell are recomputed
// in float-float (contact_z_ff) from the pv's orbit block `orb` (float pairs
// at the end of its header, in shared memory), on the FP32 pipe: FP64 issues at 1/64 of the FP32 rate
// here, and a lane takes the branch alone.  Orbits whose near-contact
// samples lie more than 1 rad of eccentric anomaly from conjunction
// (a (1 - e) below about 1.2 (1 + k)) keep the FP32 values.
template <bool DEP, bool COUNT>
__device__ __forceinline__ bool adjoint_sample(const PvHead<float>& H, const PvPb<float>& pbr,
                                               const float* __restrict__ rowblk,
                                               const PvOrbitFF* __restrict__ orb,
                                               const float4* __restrict__ svtab, int pb, int s,
                                               const PbShared* ps, const RecLayout& L, float fr_h,
                                               float fr_l, float m, float off, float mg, float gb, GradAcc<float>& acc,
                                               float* dep, int kslot, int uslot, bool& bad, Tally& tl) {
    if (COUNT) ++tl.n[RR_COUNT_SAMPLES];
    const PvPb<float> pbc = pbr;
    const float xr = (fr_h + off) + fr_l;
    const float r = round_nearest(xr);
    const float x = xr - r;
    const float dM = 6.28318530717958647692f * x;
    if (fabsf(dM) > pbc.win_s) return false;
    double dMd = 0.0;
    if (H.flags & kPvKepler64) {
        double xd = ((double)fr_h + (double)off) + (double)fr_l;
        xd -= rint(xd);
        dMd = 6.283185307179586476925 * xd;
    }
    int iters;
    const Orbit32 o = orbit32<false>(H, dM, dMd, iters);
    if (COUNT) {
        ++tl.n[RR_COUNT_ORBIT];
        if (H.flags & kPvCircular) ++tl.n[RR_COUNT_CIRCULAR];
        tl.n[RR_COUNT_NEWTON] += iters;
    }
    if (!o.ok) {
        bad = true;
        return false;
    }
    const float gz = o.z * pbc.inv1pk;
    if (!o.front || gz >= 1.0f) return false;
    if (COUNT) ++tl.n[RR_COUNT_TRANSIT];
    float z = o.z;
    float f1 = (1.0f + pbc.k) - z, f3 = z - (1.0f - pbc.k);
    float xg = gz * (float)(L.ng - 1);
    int cell = min((int)xg, L.ng - 2);
    float al = xg - (float)cell;
    if (orb != nullptr && (fminf(f1, fabsf(f3)) < pbc.cband || fabsf(xg - rintf(xg)) < kNodeBand) &&
        fabsf(o.x) <= 1.0f) {
        if (COUNT) ++tl.n[RR_COUNT_REFINED];
        // the sample's phase from the conjunction (cycles) as a float pair, with the exact
        // sub-exposure offset (first + s step) / P
        FF xc = ff_two_sum(fr_h - r, fr_l);
        if (ps->ss[pb] > 1) {
            const FF step{ps->step[pb], ps->step_lo[pb]};
            const FF od = ff_add(FF{ps->first[pb], ps->first_lo[pb]}, ff_mul_f(step, (float)s));
            xc = ff_add(xc, ff_mul(od, FF{H.Bh, H.Bl}));
        }
        const FF zz = contact_z_ff(*orb, svtab, (H.flags & kPvCircular) != 0, xc, o.x);
        const PvContactFF kc = reinterpret_cast<const PvContactFF*>(orb + 1)[pb];
        const FF d1 = ff_sub(ff_ld(kc.opk), zz), d3 = ff_sub(zz, ff_ld(kc.omk));
        z = zz.h;
        f1 = d1.h + d1.l;
        f3 = d3.h + d3.l;
        // the g cell from g (ng - 1) = z (ng - 1) / (1 + k) as a float pair: its high part is
        // an integer with a negative low part just below a node
        const FF xf = ff_mul(zz, ff_ld(kc.gsc));
        int c = (int)floorf(xf.h);
        if (xf.h == (float)c && xf.l < 0.0f) --c;
        cell = min(c, L.ng - 2);
        al = (xf.h - (float)cell) + xf.l;
    }
    if (COUNT && z > fabsf(1.0f - pbc.k)) ++tl.n[RR_COUNT_LENS];
    const float psi_tot = ((mg + m) + r) + x;   // (t_s - T0) / P
    grad_sample<float, DEP>(H, pbc, rowblk, L, z, f1, f3, cell, al, o.Px, o.Py, o.S, o.V, psi_tot, gb, acc, dep,
                            kslot, uslot);
    return true;
}

template <bool DEP, bool SS1, bool COUNT>
__global__ void __launch_bounds__(kBlock, 3) rr_grad_mixed_kernel(
    const double* __restrict__ times, const float2* __restrict__ pdt, const int32_t* __restrict__ ppb,
    const GroupInfo* __restrict__ grp, int npt,
    int npv, PbParams pbp, RecLayout L, int pv_tile, int groups_per_cta, const char* __restrict__ records,
    const char* __restrict__ rowsg, const float* __restrict__ gflux, float* __restrict__ partials, int nacc,
    int chromatic, int vec_g, const float4* __restrict__ svtab, unsigned long long* counts,
    const int* __restrict__ chunk_order, int32_t* __restrict__ pv_status, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    PbShared* ps = reinterpret_cast<PbShared*>(smem + kOffPb);
    // one sample per time: the packed candidate list (2 KB per warp) and the records after it
    constexpr size_t kRecsOff = SS1 ? kOffRecs32Packed : kOffRecs32;
    char* recs = reinterpret_cast<char*>(smem + kRecsOff);
    float* gacc = reinterpret_cast<float*>(recs + (size_t)pv_tile * L.head_bytes);   // [pv][group][nacc]
    float* depcols = gacc + (size_t)pv_tile * groups_per_cta * nacc;
    char* qbase = reinterpret_cast<char*>(depcols + (DEP ? (size_t)(nacc - 6) * kBlock : 0));
    const ItemQueue queue = queue_at(qbase, pv_tile * groups_per_cta);
    // the summaries of the CTA's groups, copied with the records, then the sine table of the
    // refinement (read by a lane alone, where an L2 read would hold its warp)
    GroupInfo* sgrp = reinterpret_cast<GroupInfo*>(qbase + queue_bytes(pv_tile * groups_per_cta));
    float4* ssv = reinterpret_cast<float4*>(sgrp + groups_per_cta);
    TileCounters* tc = reinterpret_cast<TileCounters*>(smem + kOffRed);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    WarpList* wl = reinterpret_cast<WarpList*>(smem + kOffWl + warp * kWlBytes);
    float4* wlp = reinterpret_cast<float4*>(smem + kOffWl + warp * kWlBytesPacked);
    const int ngroups = (npt + kWarpPts - 1) / kWarpPts;
    // grid: x = pv tile, y = time chunk (in launch order; chunk_order: heaviest first)
    const int chunk = chunk_order ? __ldg(chunk_order + blockIdx.y) : (int)blockIdx.y;
    const int gbeg = chunk * groups_per_cta;
    const int gend = min(ngroups, gbeg + groups_per_cta);
    const int pv0 = blockIdx.x * pv_tile;
    const int npv_t = min(pv_tile, npv - pv0);
    const uint32_t bytes = (uint32_t)npv_t * (uint32_t)L.head_bytes;
    const uint32_t gbytes = (uint32_t)(gend - gbeg) * (uint32_t)sizeof(GroupInfo);
    queue_init(queue, tc, pv_tile * groups_per_cta, gbeg);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, bytes + gbytes);
        bulk_g2s(sgrp, grp + gbeg, gbytes, bar);
        const char* src = records + (size_t)pv0 * L.head_bytes;
        for (uint32_t off = 0; off < bytes; off += 65536u) {
            const uint32_t n = bytes - off < 65536u ? bytes - off : 65536u;
            bulk_g2s(recs + off, src + off, n, bar);
        }
    }
    stage_pb(pbp, ps);
    for (int j = tid; j < pv_tile * groups_per_cta * nacc; j += kBlock) gacc[j] = 0.0f;
    if (L.orb_off >= 0)
        for (int j = tid; j < kSvTabLen; j += kBlock) ssv[j] = __ldg(svtab + j);
    __syncthreads();
    bool ok = mbar_wait_bounded(bar, 0);
    if (!ok) {
        if (tid == 0) atomicExch(err, kErrBarrierTimeout);
        mbar_wait_bounded(bar, 0);
    }
    if (__syncthreads_or(ok ? 0 : 1)) return;
    float4* cta_ph = reinterpret_cast<float4*>(smem + kOffCta);
    cta_phase(cta_ph, times, gbeg, recs, L.head_bytes, npv_t);
    __syncthreads();

    // a group: the tile's transit mask -> work items
    auto do_group = [&](int g) {
        GroupState gs;
        group_load(gs, sgrp, g - gbeg, cta_ph, recs, L.head_bytes, npv_t);
        unsigned bad;
        float4 cl;
        const unsigned may = group_decide(gs, recs, L.head_bytes, npv_t, bad, cl);
        if (may) {
            queue_push(queue, tc, may, g, cl);
            if ((may >> lane) & 1u) {
                // the items of this group read pv `lane`'s rows and cotangent segment, which the
                // forward pass's output stream has usually evicted from L2: start fetching them
                // now (rows once per CTA), well before a warp claims the item
                if (!((atomicOr(&tc->rows_pf, 1u << lane) >> lane) & 1u))
                    bulk_prefetch_l2(rowsg + (size_t)(pv0 + lane) * L.rows_bytes, (uint32_t)L.rows_bytes);
                if ((vec_g & 2) && gs.full)
                    bulk_prefetch_l2(gflux + (size_t)(pv0 + lane) * npt + (size_t)g * kWarpPts,
                                     kWarpPts * (uint32_t)sizeof(float));
            }
        }
    };

    // an item: its sums go to its own (pv, group) slot, so the result does not
    // depend on which warp took which item
    const int nkp = chromatic ? L.npb : 1;
    float* dep = DEP ? depcols + tid : nullptr;
    Tally tl{};   // the counting form's per-thread sample counts
    auto do_item = [&](int it, int key) {
        const float4 c = queue.c[it];
        const int g = key >> 5, i = key & 31;
        const int p0 = g * kWarpPts + 4 * lane;
        float dh[4], dl[4];
        int pbv[4];
        load_points(pdt, ppb, p0, npt, dh, dl, pbv);
        const char* rec = recs + (size_t)i * L.head_bytes;
        const PvHead<float>& H = *reinterpret_cast<const PvHead<float>*>(rec);
        const PvPb<float>* PB = reinterpret_cast<const PvPb<float>*>(rec + L.off_pb);
        const float* rows = reinterpret_cast<const float*>(rowsg + (size_t)(pv0 + i) * L.rows_bytes);
        const PvOrbitFF* orb = L.orb_off >= 0 ? reinterpret_cast<const PvOrbitFF*>(rec + L.orb_off) : nullptr;
        const float* gf = gflux + (size_t)(pv0 + i) * npt + p0;
        unsigned cand = 0;
        float gbq[4], gv[4];
        if ((vec_g & 1) && p0 + 3 < npt) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(gf));
            gv[0] = v.x; gv[1] = v.y; gv[2] = v.z; gv[3] = v.w;
        } else {
            #pragma unroll
            for (int q = 0; q < 4; ++q) gv[q] = p0 + q < npt ? __ldg(gf + q) : 0.0f;
        }
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            gbq[q] = 0.0f;
            const int pb = pbv[q];
            if (pb < 0 || pb >= L.npb) continue;
            const float psi = fmaf(dh[q], H.Bh, c.x);
            const float d = psi - round_nearest(psi);
            if (fabsf(d) <= PB[pb].win_pc + c.w) {
                gbq[q] = -gv[q] * ps->inv_ss[pb];
                if (gbq[q] != 0.0f) cand |= 1u << q;
            }
        }
        if (!__any_sync(0xffffffffu, cand != 0)) return;
        GradAcc<float> acc;
        #pragma unroll
        for (int j = 0; j < 6; ++j) acc.o[j] = 0.0f;
        acc.k = 0.0f;
        #pragma unroll
        for (int j = 0; j < 4; ++j) acc.u[j] = 0.0f;
        if (DEP)
            for (int j = 6; j < nacc; ++j) dep[(j - 6) * kBlock] = 0.0f;
        bool any = false, bad = false;
        if constexpr (SS1) {
            // one sample per time: the candidates are the samples
            const int nc = build_list_ss1_packed(wlp, cand, dh, dl, pbv, gbq);
            #pragma unroll 1
            for (int e0 = 0; e0 < nc; e0 += 32) {
                const int j = e0 + lane;
                if (j >= nc) continue;
                const float4 cd = wlp[j];
                const int pb = __float_as_int(cd.z);
                const Phase32 ph = precise_phase(cd.x, cd.y, c.x, c.y, H.Bh, H.Bl);
                if (COUNT) ++tl.n[RR_COUNT_TIMES];
                any |= adjoint_sample<DEP, COUNT>(H, PB[pb], rows + (size_t)pb * L.rows_per_pb * L.ng_pad, orb, ssv, pb, 0,
                                           ps, L, ph.fr_h, ph.fr_l, ph.m, 0.0f, c.z, cd.w, acc, dep,
                                           6 + (chromatic ? pb : 0), 6 + nkp + pb * L.nldc, bad, tl);
            }
        } else {
            int nc, base;
            const int ns = build_list(wl, cand, dh, dl, pbv, gbq, c.x, c.y, H.Bh, H.Bl, ps, nc, base);
            if (COUNT && lane == 0) tl.n[RR_COUNT_TIMES] += nc;
            ChunkWalk cw{0};
            #pragma unroll 1
            for (int e0 = 0; e0 < ns; e0 += 32) {
                const int e = e0 + lane;
                const int j = chunk_cand(cw, wl->soff, nc, e0);
                if (e >= ns) continue;
                const int pb = wl->pb[j];
                const float4 cd = wl->cand[j];
                const int sub = e - wl->soff[j];
                const float off = fmaf((float)sub, ps->step[pb], ps->first[pb]) * H.Bh;
                any |= adjoint_sample<DEP, COUNT>(H, PB[pb], rows + (size_t)pb * L.rows_per_pb * L.ng_pad, orb, ssv, pb, sub,
                                           ps, L, cd.x, cd.y, cd.z, off, c.z, cd.w, acc, dep, 6 + (chromatic ? pb : 0),
                                           6 + nkp + pb * L.nldc, bad, tl);
            }
        }
        __syncwarp();
        if (bad) {
            acc.o[0] = __int_as_float(0x7fc00000);
            any = true;
            if (pv_status) atomicOr(pv_status + pv0 + i, RR_PV_KEPLER);
        }
        warp_accumulate<float, DEP>(acc, dep, nacc, any, gacc + ((size_t)i * groups_per_cta + (g - gbeg)) * nacc);
    };

    bool groups_left = true;
    int idle = 0;
    #pragma unroll 1
    while (true) {
        if (groups_left) {
            int g = 0;
            if (lane == 0) g = atomicAdd(&tc->next_group, 1);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g < gend) do_group(g);
            else { groups_left = false; queue_producer_done(tc); }
        }
        const int it = queue_claim(tc);
        if (it >= 0) {
            const int key = queue_key(queue, it);
            if (key < 0) {
                if (lane == 0) atomicExch(err, kErrQueueTimeout);
                break;
            }
            do_item(it, key);
            continue;
        }
        if (groups_left) continue;
        if (queue_finished(tc)) {
            // no producer left: the queue is final; drain what is still claimable
            const int last = queue_claim(tc);
            if (last < 0) break;
            const int key = queue_key(queue, last);
            if (key < 0) {
                if (lane == 0) atomicExch(err, kErrQueueTimeout);
                break;
            }
            do_item(last, key);
            continue;
        }
        // other warps still take groups: wait for their items (bounded)
        if (++idle > (1 << 22)) {
            if (lane == 0) atomicExch(err, kErrQueueTimeout);
            break;
        }
        __nanosleep(64);
    }
    if (COUNT) tally_flush(tl, counts);
    cta_partials_groups(gacc, recs, L.head_bytes, npv_t, nacc, groups_per_cta, pv0, chunk, gridDim.y, partials);
}

template <bool DEP>
__global__ void __launch_bounds__(kBlock) rr_grad_fp64_kernel(
    const double* __restrict__ times, const int32_t* __restrict__ pb_index, int npt, int npv,
    PbParams pbp, RecLayout L, int pv_tile, const char* __restrict__ records, const char* __restrict__ rowsg,
    const double* __restrict__ gflux, double* __restrict__ partials, int nacc, int chromatic,
    int32_t* __restrict__ pv_status, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    char* recs = reinterpret_cast<char*>(smem + 16 + 16 * 4 + 16 * kMaxPvTile);
    double* wpart = reinterpret_cast<double*>(recs + (size_t)pv_tile * L.head_bytes);
    double* depcols = wpart + (size_t)pv_tile * (kBlock >> 5) * nacc;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tile = blockIdx.x, ntiles = gridDim.x;
    const int pt0 = tile * kPtTile;
    const int pv0 = blockIdx.y * pv_tile;
    const int npv_t = min(pv_tile, npv - pv0);
    if (!stage_to_smem(recs, records + (size_t)pv0 * L.head_bytes, (uint32_t)npv_t * (uint32_t)L.head_bytes, bar,
                       err))
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
        const char* rec = recs + (size_t)i * L.head_bytes;
        const PvHead<double>& H = *reinterpret_cast<const PvHead<double>*>(rec);
        if (H.status != 0) continue;
        const PvPb<double>* PB = reinterpret_cast<const PvPb<double>*>(rec + L.off_pb);
        const double* rows = reinterpret_cast<const double*>(rowsg + (size_t)(pv0 + i) * L.rows_bytes);
        const double* gf = gflux + (size_t)(pv0 + i) * npt;
        GradAcc<double> acc;
        for (int j = 0; j < 6; ++j) acc.o[j] = 0.0;
        acc.k = 0.0;
        for (int j = 0; j < 4; ++j) acc.u[j] = 0.0;
        if (DEP)
            for (int j = 6; j < nacc; ++j) dep[(j - 6) * kBlock] = 0.0;
        bool any = false, bad = false;
        #pragma unroll
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
                const double xg = g * (double)(L.ng - 1);
                const int cell = min((int)xg, L.ng - 2);
                grad_sample<double, DEP>(H, pbc, rowblk, L, o.z, (1.0 + pbc.k) - o.z, o.z - (1.0 - pbc.k), cell,
                                         xg - (double)cell, o.Px, o.Py, o.S, o.V, psi_tot, gb, acc, dep, kslot,
                                         uslot);
                any = true;
            }
        }
        if (bad) {
            acc.o[0] = __longlong_as_double(0x7ff8000000000000ll);
            any = true;
            if (pv_status) atomicOr(pv_status + pv0 + i, RR_PV_KEPLER);
        }
        warp_partials<double, DEP>(acc, dep, nacc, any, wpart + ((size_t)i * (kBlock >> 5) + warp) * nacc);
    }
    cta_partials<double>(wpart, recs, L.head_bytes, npv_t, nacc, pv0, tile, ntiles, partials);
}

// Sum the partial sums of each pv over its chunks in chunk order (FP64),
// one lane per (pv, parameter).  Invalid pvs get NaN rows.
// grad[pv][j] = sum over the pv's partial-sum chunks (chunk order, FP64); then,
// for the (q1, q2) parametrisation, the chain rule through u1 = 2 sqrt(q1) q2,
// u2 = sqrt(q1) (1 - 2 q2).  A block takes kFinishPvs pvs: one thread per
// (pv, parameter) for the sums, then one per (pv, passband) for the chain rule.
constexpr int kFinishThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kFinishThreads) rr_grad_finish_kernel(
    const R* __restrict__ partials, int nchunks, int nacc, int nparam, int npv, int pvs_per_block,
    const char* __restrict__ heads, int head_bytes, const double* __restrict__ params, int kipping, int shared,
    int npb, int nkp, double* __restrict__ grad) {
    extern __shared__ double sg[];                 // [pvs_per_block][nacc]
    const int pv0 = blockIdx.x * pvs_per_block;
    const int nloc = min(pvs_per_block, npv - pv0);
    for (int t = threadIdx.x; t < nloc * nacc; t += blockDim.x) {
        const int lp = t / nacc, j = t - lp * nacc;
        const R* pp = partials + (size_t)(pv0 + lp) * nchunks * nacc + j;
        double s = 0.0;
        int c = 0;
        for (; c + 4 <= nchunks; c += 4) {
            const R v0 = pp[(size_t)c * nacc], v1 = pp[(size_t)(c + 1) * nacc];
            const R v2 = pp[(size_t)(c + 2) * nacc], v3 = pp[(size_t)(c + 3) * nacc];
            s += (double)v0;
            s += (double)v1;
            s += (double)v2;
            s += (double)v3;
        }
        for (; c < nchunks; ++c) s += (double)pp[(size_t)c * nacc];
        const bool bad = reinterpret_cast<const PvHead<R>*>(heads + (size_t)(pv0 + lp) * head_bytes)->status != 0;
        s = bad ? __longlong_as_double(0x7ff8000000000000ll) : s;
        sg[t] = s;
        if (j < nparam) grad[(size_t)(pv0 + lp) * nparam + j] = s;
    }
    if (!kipping && !shared) return;               // block-uniform
    __syncthreads();
    if (shared) {
        // shared weights: d kbar / d k_j = 1 / nkp for every per-passband radius ratio
        for (int t = threadIdx.x; t < nloc * nkp; t += blockDim.x) {
            const int lp = t / nkp, j = t - lp * nkp;
            grad[(size_t)(pv0 + lp) * nparam + 6 + j] = sg[lp * nacc + 6 + j] + sg[lp * nacc + nparam] / nkp;
        }
    }
    if (!kipping) return;
    for (int t = threadIdx.x; t < nloc * npb; t += blockDim.x) {
        const int lp = t / npb, pb = t - lp * npb;
        const int o = 6 + nkp + 2 * pb;
        const double* row = params + (size_t)(pv0 + lp) * nparam;
        const double g1 = sg[lp * nacc + o], g2 = sg[lp * nacc + o + 1];
        if (g1 != g1) continue;                    // invalid pv: NaN row stays
        const double sq = sqrt(row[o]), q2 = row[o + 1];
        const double isq = 1.0 / sq;
        double* out = grad + (size_t)(pv0 + lp) * nparam;
        out[o] = g1 * q2 * isq + g2 * (1.0 - 2.0 * q2) * (0.5 * isq);
        out[o + 1] = 2.0 * sq * (g1 - g2);
    }
}

static size_t grad_smem(int pv_tile, const RecLayout& L, int nacc, bool dep, size_t rsize, int slots, bool ss1) {
    size_t s = (rsize == 8 ? 16 + 16 * 4 + 16 * kMaxPvTile : (ss1 ? kOffRecs32Packed : kOffRecs32)) +
               (size_t)pv_tile * L.head_bytes +
               (size_t)pv_tile * slots * nacc * rsize;
    if (dep) s += (size_t)(nacc - 6) * kBlock * rsize;
    // FP32 kernel: item queue, then the summaries of the CTA's groups and the sine table
    if (rsize == 4)
        s = ((s + 15) & ~(size_t)15) + queue_bytes(pv_tile * slots) + (size_t)slots * sizeof(GroupInfo) +
            (size_t)kSvTabLen * sizeof(float4);
    return s;
}

// Partial sums per pv: one per 1024-time tile (FP64 kernel) or per CTA
// chunk of 128-time groups (FP32 kernel); depends on npt only.
static int grad_chunks(const rr_ctx* c, int npt) {
    if (c->cfg.precision == RR_PREC_FP64) return (npt + kPtTile - 1) / kPtTile;
    const int ngroups = (npt + kWarpPts - 1) / kWarpPts;
    const int gpc = groups_per_cta(npt);
    return (ngroups + gpc - 1) / gpc;
}

size_t partials_bytes(const rr_ctx* c, int npv, int npt) {
    const size_t rsize = c->cfg.precision == RR_PREC_FP64 ? sizeof(double) : sizeof(float);
    return (size_t)npv * (size_t)grad_chunks(c, npt) * (size_t)grad_nacc(c) * rsize;
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

static bool grad_dep(const rr_ctx* c) {
    return c->nparam > 11 || (c->cfg.npb > 1 && (c->cfg.chromatic || c->nldc > 0)) || shared_weights(c);
}

cudaError_t launch_grad(rr_ctx* c, const double* times, const int32_t* pb_index, const void* pts_dt,
                        const void* pts_pb, const void* pts_grp, const void* pts_ord, int npt, int npv,
                        const PbParams& pbp, const void* records,
                        const void* grad_flux, void* partials, int32_t* pv_status, cudaStream_t s) {
    const bool f64 = c->cfg.precision == RR_PREC_FP64;
    RecLayout L = f64 ? make_layout<double>(c->cfg.npb, c->cfg.ng, c->nldc, true)
                      : make_layout<float>(c->cfg.npb, c->cfg.ng, c->nldc, true);
    const int nacc = grad_nacc(c);
    if (shared_weights(c)) L.kbar_slot = c->nparam;
    const bool dep = grad_dep(c);
    const size_t rsize = f64 ? 8 : 4;
    // pv tile: records plus the per-warp partial sums within the shared-memory target
    const int slots = f64 ? (kBlock >> 5) : groups_per_cta(npt);   // partial-sum slots per pv in the CTA
    const size_t per_pv = (size_t)L.head_bytes + (size_t)slots * nacc * rsize;
    int pv_tile = (int)(kSmemTarget / per_pv);
    pv_tile = pv_tile < 1 ? 1 : (pv_tile > kMaxPvTile ? kMaxPvTile : pv_tile);
    bool ss1 = true;
    for (int pb = 0; pb < pbp.npb; ++pb) ss1 = ss1 && pbp.ss[pb] == 1;
    const size_t smem = grad_smem(pv_tile, L, nacc, dep, rsize, slots, ss1);
    const char* rowsg = (const char*)records + rows_offset(L, npv);
    const int npvt = (npv + pv_tile - 1) / pv_tile;
    const int gpc = groups_per_cta(npt);
    dim3 grid = f64 ? dim3(grad_chunks(c, npt), npvt) : dim3(npvt, grad_chunks(c, npt));
    if (smem > kMaxSmem || grid.y > 65535u) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if (f64) {
#define RR_LAUNCH_GRAD64(KERNEL)                                                                              \
    do {                                                                                                      \
        e = set_smem(KERNEL, smem);                                                                           \
        if (e != cudaSuccess) return e;                                                                       \
        KERNEL<<<grid, kBlock, smem, s>>>(times, pb_index, npt, npv, pbp, L, pv_tile, (const char*)records,   \
                                          rowsg, (const double*)grad_flux, (double*)partials, nacc,           \
                                          c->cfg.chromatic,                                                   \
                                          pv_status, c->d_err);                                               \
    } while (0)
        if (dep) RR_LAUNCH_GRAD64(rr_grad_fp64_kernel<true>);
        else RR_LAUNCH_GRAD64(rr_grad_fp64_kernel<false>);
#undef RR_LAUNCH_GRAD64
    } else {
#define RR_LAUNCH_GRAD32(KERNEL)                                                                             \
    do {                                                                                                     \
        e = set_smem(KERNEL, smem);                                                                          \
        if (e != cudaSuccess) return e;                                                                      \
        KERNEL<<<grid, kBlock, smem, s>>>(times, (const float2*)pts_dt, (const int32_t*)pts_pb,                \
                                          (const GroupInfo*)pts_grp, npt, npv, pbp,                           \
                                          L, pv_tile, gpc, (const char*)records, rowsg,                       \
                                          (const float*)grad_flux, (float*)partials, nacc, c->cfg.chromatic,  \
                                          vec_g, c->d_svtab, counts, (const int*)pts_ord,                     \
                                          pv_status, c->d_err);                                               \
    } while (0)
        // bit 0: 16-byte loads; bit 1: L2 prefetches of cotangent rows (grad_flux in device memory)
        const int vec_g = (npt % 4 == 0) && (((uintptr_t)grad_flux & 15u) == 0)
                              ? (in_device_memory(grad_flux) ? 3 : 1) : 0;
        unsigned long long* counts = c->d_counts ? c->d_counts + (size_t)RR_KERNEL_GRAD * RR_COUNT_KINDS : nullptr;
        if (c->counting) {
            if (dep) {
                if (ss1) RR_LAUNCH_GRAD32((rr_grad_mixed_kernel<true, true, true>));
                else RR_LAUNCH_GRAD32((rr_grad_mixed_kernel<true, false, true>));
            } else {
                if (ss1) RR_LAUNCH_GRAD32((rr_grad_mixed_kernel<false, true, true>));
                else RR_LAUNCH_GRAD32((rr_grad_mixed_kernel<false, false, true>));
            }
        } else if (dep) {
            if (ss1) RR_LAUNCH_GRAD32((rr_grad_mixed_kernel<true, true, false>));
            else RR_LAUNCH_GRAD32((rr_grad_mixed_kernel<true, false, false>));
        } else {
            if (ss1) RR_LAUNCH_GRAD32((rr_grad_mixed_kernel<false, true, false>));
            else RR_LAUNCH_GRAD32((rr_grad_mixed_kernel<false, false, false>));
        }
#undef RR_LAUNCH_GRAD32
    }
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_grad_reduce(rr_ctx* c, int npt, const double* params, int npv, const void* records,
                               const void* partials, double* grad_params, cudaStream_t s) {
    const bool f64 = c->cfg.precision == RR_PREC_FP64;
    RecLayout L = f64 ? make_layout<double>(c->cfg.npb, c->cfg.ng, c->nldc, true)
                      : make_layout<float>(c->cfg.npb, c->cfg.ng, c->nldc, true);
    const int nacc = grad_nacc(c);
    const int shared = shared_weights(c) ? 1 : 0;
    const int nchunks = grad_chunks(c, npt);
    const int nkp = c->cfg.chromatic ? c->cfg.npb : 1;
    const int kip = c->cfg.ld_model == RR_LD_QUADRATIC_TRI ? 1 : 0;
    const int per_block = kFinishThreads / nacc > 0 ? kFinishThreads / nacc : 1;
    const unsigned blocks = (unsigned)((npv + per_block - 1) / per_block);
    const size_t smem = (size_t)per_block * nacc * sizeof(double);
    if (f64)
        rr_grad_finish_kernel<double><<<blocks, kFinishThreads, smem, s>>>(
            (const double*)partials, nchunks, nacc, c->nparam, npv, per_block, (const char*)records, L.head_bytes,
            params, kip, shared, c->cfg.npb, nkp, grad_params);
    else
        rr_grad_finish_kernel<float><<<blocks, kFinishThreads, smem, s>>>(
            (const float*)partials, nchunks, nacc, c->nparam, npv, per_block, (const char*)records, L.head_bytes,
            params, kip, shared, c->cfg.npb, nkp, grad_params);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace rr
