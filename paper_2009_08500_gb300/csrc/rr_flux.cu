// Fused light-curve kernels: time -> phase -> z -> Eq. 5 -> mean over
// sub-exposures, for a tile of parameter vectors x a tile of times.
//
// FP32 kernel.  A CTA owns a chunk of consecutive 128-time groups (4
// consecutive times per lane of a warp) and a tile of up to 32 parameter
// vectors (lane i of a warp speaks for pv i).  One bulk asynchronous copy
// (TMA engine, mbarrier completion, bounded wait) stages the tile's pv
// records and the chunk's group summaries into shared memory.  Stream warps
// then take the groups: per group one transit test per pv, whole 512-byte
// row segments of exactly 1 for the pvs outside their windows (bulk
// asynchronous stores from a constant shared-memory row), and a work item
// (pv, group) in a shared-memory queue for the others; the remaining warps
// evaluate the items as they appear (candidate samples compacted per warp,
// 32 at a time).  FP64 kernel: a tile of kPtTile times strided by kBlock
// and the same pv tile, every sample in FP64.
//
// Mixed precision (FP32 bulk):
//  * per time, once per call (points_group): dt = t - t_g in FP64, kept as
//    a float pair (dh, dl) -- t_g is the first time of the time's group;
//  * per (CTA, pv), FP64: A = frac((t_ref - T0) / P) as a float pair at the
//    CTA's first group, carried to each group in float-float;
//  * per (pv, time): coarse phase psi = A + dh / P with one FMA, rounded
//    with two additions (no FP64, no conversion per point).  If the
//    whole exposure lies outside the pv's transit window the point is 1
//    exactly and nothing else is computed.  Otherwise the phase is formed in
//    float-float (error ~1e-9 of a cycle) and every sub-exposure goes
//    through Kepler (FP32 Newton in the offset form, FP64 above e = 0.8),
//    the projected distance, the covered area and the profile row lookup.
// FP64 form: the same structure with every step in FP64 and the phase
// reduced per sub-exposure as tau = t_s - T0 - P rint((t_s - T0) / P).
#include "rr_device.cuh"

namespace rr {

// Order of the time chunks of the FP32 per-point kernels, heaviest first (one
// CTA): chunk i (groups i gpc .. i gpc + gpc - 1) weighs the exposure
// sub-samples of its groups; order[rank] = i, ties in index order.  With
// passbands of different supersampling the chunks' work differs several-fold
// (a chunk of 30-sub-exposure times against one of single samples), and the
// heaviest CTAs are best started first: the last wave then holds light ones.
// More than 1024 chunks: index order.
__global__ void __launch_bounds__(1024) rr_chunk_order_kernel(const GroupInfo* __restrict__ grp, int ngroups,
                                                              int gpc, int nchunks, int* __restrict__ order) {
    __shared__ float w[1024];
    const int i = threadIdx.x;
    if (nchunks > 1024) {
        for (int j = i; j < nchunks; j += blockDim.x) order[j] = j;
        return;
    }
    if (i < nchunks) {
        float s = 0.0f;
        const int g1 = min(ngroups, (i + 1) * gpc);
        for (int g = i * gpc; g < g1; ++g) s += grp[g].weight;
        w[i] = s;
    }
    __syncthreads();
    if (i < nchunks) {
        const float wi = w[i];
        int rank = 0;
        for (int j = 0; j < nchunks; ++j) rank += (w[j] > wi) || (w[j] == wi && j < i);
        order[rank] = i;
    }
}

cudaError_t launch_chunk_order(rr_ctx* c, int npt, void* ws_grp, void* ws_ord, cudaStream_t s) {
    const int ngroups = (npt + kWarpPts - 1) / kWarpPts;
    const int gpc = groups_per_cta(npt);
    rr_chunk_order_kernel<<<1, 1024, 0, s>>>((const GroupInfo*)ws_grp, ngroups, gpc, time_chunks(npt, gpc),
                                             (int*)ws_ord);
    c->launches++;
    return cudaGetLastError();
}

// Stores the 4 outputs of a lane (one 16-byte store when the row is vector-aligned).
__device__ __forceinline__ void store4(float* out, const float (&f)[4], const int (&pbv)[4], bool full) {
    if (full) {
        __stcs(reinterpret_cast<float4*>(out), make_float4(f[0], f[1], f[2], f[3]));
    } else {
        #pragma unroll
        for (int q = 0; q < 4; ++q)
            if (pbv[q] >= 0) __stcs(out + q, f[q]);
    }
}

template <bool STAGE_ROWS, bool SS1, bool COUNT>
__global__ void __launch_bounds__(kBlock, 4) rr_flux_mixed_kernel(const double* __restrict__ times,
                                                               const float2* __restrict__ pdt,
                                                               const int32_t* __restrict__ ppb,
                                                               const GroupInfo* __restrict__ grp,
                                                               int npt, int npv, PbParams pbp, RecLayout L,
                                                               int pv_tile, int groups_per_cta,
                                                               const char* __restrict__ records,
                                                               const char* __restrict__ rowsg,
                                                               float* __restrict__ flux,
                                                               int32_t* __restrict__ pv_status, int vec_store,
                                                               int stream_warps, unsigned long long* counts,
                                                               const int* __restrict__ chunk_order, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    PbShared* ps = reinterpret_cast<PbShared*>(smem + kOffPb);
    char* recs = reinterpret_cast<char*>(smem + kOffRecsFlux);
    TileCounters* tc = reinterpret_cast<TileCounters*>(smem + kOffRed);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    FluxList* wl = reinterpret_cast<FluxList*>(smem + kOffWl + warp * kFlBytes);
    const int ngroups = (npt + kWarpPts - 1) / kWarpPts;
    // grid: x = pv tile, y = time chunk (in launch order; chunk_order: heaviest first)
    const int chunk = chunk_order ? __ldg(chunk_order + blockIdx.y) : (int)blockIdx.y;
    const int gbeg = chunk * groups_per_cta;
    const int gend = min(ngroups, gbeg + groups_per_cta);
    const int pv0 = blockIdx.x * pv_tile;
    const int npv_t = min(pv_tile, npv - pv0);
    // staged: headers of the tile, then (STAGE_ROWS) their profile rows, then the item queue
    char* srows = recs + (size_t)pv_tile * L.head_bytes;
    char* qbase = srows + (STAGE_ROWS ? (size_t)pv_tile * L.rows_bytes : 0);
    const ItemQueue queue = queue_at(qbase, pv_tile * groups_per_cta);
    // constant output rows of one group (1 and NaN), sources of the bulk stores
    float* rows1 = reinterpret_cast<float*>(qbase + queue_bytes(pv_tile * groups_per_cta));
    float* rowsnan = rows1 + kWarpPts;
    // the summaries of the CTA's groups, copied with the records
    GroupInfo* sgrp = reinterpret_cast<GroupInfo*>(rowsnan + kWarpPts);
    const uint32_t hbytes = (uint32_t)npv_t * (uint32_t)L.head_bytes;
    const uint32_t rbytes = STAGE_ROWS ? (uint32_t)npv_t * (uint32_t)L.rows_bytes : 0u;
    const uint32_t gbytes = (uint32_t)(gend - gbeg) * (uint32_t)sizeof(GroupInfo);
    queue_init(queue, tc, pv_tile * groups_per_cta, gbeg);
    for (int j = tid; j < kWarpPts; j += blockDim.x) {
        rows1[j] = 1.0f;
        rowsnan[j] = __int_as_float(0x7fc00000);
    }
    fence_proxy_async_smem();   // the bulk stores read these through the async proxy
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, hbytes + rbytes + gbytes);
        bulk_g2s(sgrp, grp + gbeg, gbytes, bar);
        const char* src = records + (size_t)pv0 * L.head_bytes;
        for (uint32_t off = 0; off < hbytes; off += 65536u) {
            const uint32_t n = hbytes - off < 65536u ? hbytes - off : 65536u;
            bulk_g2s(recs + off, src + off, n, bar);
        }
        const char* rsrc = rowsg + (size_t)pv0 * L.rows_bytes;
        for (uint32_t off = 0; off < rbytes; off += 65536u) {
            const uint32_t n = rbytes - off < 65536u ? rbytes - off : 65536u;
            bulk_g2s(srows + off, rsrc + off, n, bar);
        }
    }
    stage_pb(pbp, ps);
    __syncthreads();   // publishes the barrier initialisation, the counters and the passband table
    bool ok = mbar_wait_bounded(bar, 0);
    if (!ok) {
        if (tid == 0) atomicExch(err, kErrBarrierTimeout);
        mbar_wait_bounded(bar, 0);
    }
    if (__syncthreads_or(ok ? 0 : 1)) return;
    float4* cta_ph = reinterpret_cast<float4*>(smem + kOffCta);
    cta_phase(cta_ph, times, gbeg, recs, L.head_bytes, npv_t);
    __syncthreads();

    const float nanf_ = __int_as_float(0x7fc00000);
    const uint64_t l2_pol = l2_evict_first_policy();
    Tally tl{};   // the counting form's per-thread sample counts

    // a group: the tile's transit mask; every pv outside it is 1 (NaN for an
    // invalid pv or passband index) without arithmetic, the others are queued
    auto do_group = [&](int g) {
        const int p0 = g * kWarpPts + 4 * lane;
        GroupState gs;
        group_load(gs, sgrp, g - gbeg, cta_ph, recs, L.head_bytes, npv_t);
        unsigned bad;
        float4 cl;
        const unsigned may = group_decide(gs, recs, L.head_bytes, npv_t, bad, cl);
        if (may) queue_push(queue, tc, may, g, cl);
        int pbv[4] = {0, 0, 0, 0};
        if (!gs.full) load_pb(ppb, p0, npt, pbv);    // a partial group or invalid passbands
        float fb[4];
        #pragma unroll
        for (int q = 0; q < 4; ++q) fb[q] = pbv[q] < L.npb ? 1.0f : nanf_;
        const bool full = (vec_store & 1) && (p0 + 3 < npt);
        float* out = flux + (size_t)pv0 * npt + p0;
        // the pvs of the tile that need no arithmetic
        unsigned rest = (npv_t >= 32 ? 0xffffffffu : ((1u << npv_t) - 1u)) & ~may;
        if ((vec_store & 2) && gs.full) {
            // a whole 512-byte row segment per pv from a constant row in shared
            // memory, one bulk asynchronous store per lane (lane i: pv i); the
            // addresses are 16-byte aligned (npt % 4 == 0, aligned flux in device memory)
            if ((rest >> lane) & 1u) {
                bulk_s2g(flux + (size_t)(pv0 + lane) * npt + (size_t)g * kWarpPts,
                         ((bad >> lane) & 1u) ? rowsnan : rows1, kWarpPts * sizeof(float), l2_pol);
                bulk_commit();
            }
            rest = 0u;
        }
        #pragma unroll 1
        while (rest) {
            const int i = __ffs(rest) - 1;
            rest &= rest - 1u;
            const bool inval = (bad >> i) & 1u;
            const float f[4] = {inval ? nanf_ : fb[0], inval ? nanf_ : fb[1], inval ? nanf_ : fb[2],
                                inval ? nanf_ : fb[3]};
            store4(out + (size_t)i * npt, f, pbv, full);
        }
    };

    // an item: every time of the group for one pv that may transit
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
        const float* rows = STAGE_ROWS ? reinterpret_cast<const float*>(srows + (size_t)i * L.rows_bytes)
                                       : reinterpret_cast<const float*>(rowsg + (size_t)(pv0 + i) * L.rows_bytes);
        float f[4];
        unsigned cand = 0;
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int pb = pbv[q];
            f[q] = pb < L.npb ? 1.0f : nanf_;
            if (pb < 0 || pb >= L.npb) continue;
            const float psi = fmaf(dh[q], H.Bh, c.x);
            const float d = psi - round_nearest(psi);
            if (fabsf(d) <= PB[pb].win_pc + c.w) cand |= 1u << q;
        }
        bool bad = false;
        if constexpr (SS1) {
          if (__any_sync(0xffffffffu, cand != 0)) {
            // one sample per time: the candidates are the samples
            int bq[4];
            const int nc = build_list_ss1_flux(wl, cand, dh, dl, pbv, bq);
            #pragma unroll 1
            for (int e0 = 0; e0 < nc; e0 += 32) {
                const int j = e0 + lane;
                if (j < nc) {
                    const int pb = wl->ps[j];
                    const float2 cd = wl->cand[j];
                    const Phase32 ph = precise_phase(cd.x, cd.y, c.x, c.y, H.Bh, H.Bl);
                    if (COUNT) ++tl.n[RR_COUNT_TIMES];
                    wl->pacc[j] = delta32<COUNT>(H, PB[pb], rows + (size_t)pb * L.rows_per_pb * L.ng_pad, L.ng,
                                                 ph.fr_h, ph.fr_l, 0.0f, 0.0f, 0.0f, bad, &tl);
                }
            }
            __syncwarp();
            #pragma unroll
            for (int q = 0; q < 4; ++q)
                if ((cand >> q) & 1u) f[q] = 1.0f - wl->pacc[bq[q]];
            __syncwarp();
          }
        } else if (__any_sync(0xffffffffu, cand != 0)) {
            int nc, base;
            const int ns = build_list_flux(wl, cand, dh, dl, pbv, c.x, c.y, H.Bh, H.Bl, ps, nc, base);
            if (COUNT && lane == 0) tl.n[RR_COUNT_TIMES] += nc;
            // The item's flattened samples [0, ns) in 32 contiguous runs of run = ceil(ns / 32),
            // one per lane.  A lane walks its run in order, summing the sub-exposures of the
            // candidate at hand: the sum of a candidate that starts and ends inside the run is
            // final; the candidate at the run's start (head) and the one at its end (tail) may
            // go on in the neighbouring runs, and are combined once per item, in lane order.
            const int run = (ns + 31) >> 5;
            const int e_beg = min(lane * run, ns), e_end = min(e_beg + run, ns);
            int jh = -1, jt = -1;          // head and tail candidates of the run (-1: none)
            float ph = 0.0f, pt = 0.0f;    // their partial sums over the run
            if (e_beg < e_end) {
                // the candidate holding sample e_beg: the last j with soff(j) <= e_beg
                int lo = 0, hi = nc - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if ((wl->ps[mid] >> 5) <= e_beg) lo = mid; else hi = mid - 1;
                }
                int j = lo;
                int pw = wl->ps[j];
                int next = wl->ps[j + 1] >> 5;     // first sample of candidate j + 1 (ps[nc] = ns << 5)
                // the candidate's passband: its constants, profile row and sub-exposure spacing,
                // looked up once per candidate rather than per sample
                int pb = pw & 31;
                float2 cd = wl->cand[j];
                float sub = (float)(e_beg - (pw >> 5));
                float part = 0.0f;
                jh = j;
                #pragma unroll 1
                for (int e = e_beg; e < e_end; ++e) {
                    if (e == next) {
                        // candidate j ends inside the run: the head's sum, or a final one
                        if (j == jh) ph = part; else wl->pacc[j] = part;
                        ++j;
                        pw = wl->ps[j];
                        next = wl->ps[j + 1] >> 5;
                        pb = pw & 31;
                        cd = wl->cand[j];
                        sub = 0.0f;
                        part = 0.0f;
                    }
                    part += delta32<COUNT>(H, PB[pb], rows + (size_t)pb * L.rows_per_pb * L.ng_pad, L.ng, cd.x, cd.y,
                                           sub, ps->first[pb], ps->step[pb], bad, &tl);
                    sub += 1.0f;
                }
                if (j == jh) ph = part; else { jt = j; pt = part; }
            }
            // a tail that goes on into the next run is added in front of that run's head
            const int tprev_j = __shfl_up_sync(0xffffffffu, jt, 1);
            const float tprev_p = __shfl_up_sync(0xffffffffu, pt, 1);
            if (lane > 0 && jh >= 0 && tprev_j == jh) ph = tprev_p + ph;
            const int hnext_j = __shfl_down_sync(0xffffffffu, jh, 1);
            if (jt >= 0 && (lane == 31 || hnext_j != jt)) wl->pacc[jt] = pt;   // the tail ends with the run
            // heads: segmented inclusive scan over the lanes by candidate (fixed order); the last
            // lane of each segment holds the candidate's sum
            float v = ph;
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, v, o);
                const int ky = __shfl_up_sync(0xffffffffu, jh, o);
                if (lane >= o && ky == jh) v = y + v;
            }
            if (jh >= 0 && (lane == 31 || hnext_j != jh)) wl->pacc[jh] = v;
            __syncwarp();
            int jj = base;
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (cand & (1u << q)) {
                    f[q] = 1.0f - wl->pacc[jj] * ps->inv_ss[pbv[q]];
                    ++jj;
                }
            }
            __syncwarp();
        }
        if (bad && pv_status) atomicOr(pv_status + pv0 + i, RR_PV_KEPLER);
        store4(flux + (size_t)(pv0 + i) * npt + p0, f, pbv, (vec_store & 1) && (p0 + 3 < npt));
    };

    // Warps below stream_warps first take the groups (the output stream) and
    // produce the items; the others start on the items at once.  Every warp
    // then drains the items.
    if (warp < stream_warps) {
        #pragma unroll 1
        while (true) {
            int g = 0;
            if (lane == 0) g = atomicAdd(&tc->next_group, 1);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= gend) break;
            do_group(g);
        }
    }
    queue_producer_done(tc);
    int idle = 0;
    #pragma unroll 1
    while (true) {
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
    bulk_wait_all();   // the bulk stores read shared memory that ends with the CTA
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
                                                              const char* __restrict__ rowsg,
                                                              double* __restrict__ flux,
                                                              int32_t* __restrict__ pv_status, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    char* recs = reinterpret_cast<char*>(smem + 16 + 16 * 4 + 16 * kMaxPvTile);
    const int tid = threadIdx.x;
    const int pt0 = blockIdx.x * kPtTile;
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
            pbv[j] = (pb >= 0 && pb < L.npb) ? pb : L.npb;   // L.npb marks an invalid index (NaN)
        }
    }
    const double nan_ = __longlong_as_double(0x7ff8000000000000ll);
    #pragma unroll 1
    for (int i = 0; i < npv_t; ++i) {
        const char* rec = recs + (size_t)i * L.head_bytes;
        const PvHead<double>& H = *reinterpret_cast<const PvHead<double>*>(rec);
        const PvPb<double>* PB = reinterpret_cast<const PvPb<double>*>(rec + L.off_pb);
        const double* rows = reinterpret_cast<const double*>(rowsg + (size_t)(pv0 + i) * L.rows_bytes);
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

static size_t flux_smem(int pv_tile, int rec_bytes, bool f64, int gpc) {
    if (f64) return 16 + 16 * 4 + 16 * kMaxPvTile + (size_t)pv_tile * rec_bytes;
    // + two constant rows (1 and NaN) for the bulk stores + the group summaries
    return kOffRecsFlux + (size_t)pv_tile * rec_bytes + queue_bytes(pv_tile * gpc) + 2 * kWarpPts * sizeof(float) +
           (size_t)gpc * sizeof(GroupInfo);
}
static_assert(kOffRecs32 % 16 == 0 && kOffRecs32Packed % 16 == 0 && kOffRecsFlux % 16 == 0,
              "shared-memory regions must stay 16-byte aligned");

// 128-time groups per CTA of the FP32 kernels.  A function of npt only, so
// the adjoint's summation order for a pv never depends on the other pvs in
// the launch: between 1 and 16 groups per warp, about one eighth of the
// point range per CTA.
int groups_per_cta(int npt) {
    const int ntiles = (npt + kPtTile - 1) / kPtTile;
    int t = ntiles / 8;
    t = t < 1 ? 1 : (t > 16 ? 16 : t);
    return t * (kBlock / 32);
}

int pv_tile_for(int rec_bytes) {
    int t = kSmemTarget / rec_bytes;
    if (t < 1) t = 1;
    if (t > kMaxPvTile) t = kMaxPvTile;
    return t;
}

// Failure-detection self-test: one bounded wait that nothing completes (see
// rr_selftest_wait); the expiry is recorded in the error word like any other.
__global__ void rr_selftest_kernel(int which, int* err) {
    __shared__ uint64_t bar;
    __shared__ int slot[1];
    __shared__ float4 slot_c[1];
    if (which == 0) {
        if (threadIdx.x != 0) return;
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, 16);   // this thread arrives; the 16 bytes of transaction never come
        if (!mbar_wait_bounded(&bar, 0)) atomicExch(err, kErrBarrierTimeout);
        return;
    }
    // a claimed slot whose producer never publishes it; the whole warp takes part
    // (the claim wait ends in a warp shuffle)
    if (threadIdx.x == 0) slot[0] = -1;
    __syncwarp();
    ItemQueue q;
    q.c = slot_c;
    q.gi = slot;
    if (queue_key(q, 0) < 0 && threadIdx.x == 0) atomicExch(err, kErrQueueTimeout);
}

cudaError_t launch_selftest(rr_ctx* c, int which, cudaStream_t s) {
    rr_selftest_kernel<<<1, 32, 0, s>>>(which, c->d_err);
    c->launches++;
    return cudaGetLastError();
}

// Warps of a flux CTA that take the 128-time groups before any item.  With
// one sample per time the items are light: two warps keep the output stream
// going while six evaluate the transits beside it (population workload: flux
// kernel 80.8 -> 75.1 us).  With supersampling the items dominate and every
// warp streams its groups first (heterogeneous workload: 835 -> 792 us).
constexpr int kStreamWarpsSS1 = 2;

cudaError_t launch_flux(rr_ctx* c, const double* times, const int32_t* pb_index, const void* pts_dt,
                        const void* pts_pb, const void* pts_grp, const void* pts_ord, int npt, int npv,
                        const PbParams& pbp, const void* records,
                        void* flux, int32_t* pv_status, bool grad_layout, cudaStream_t s) {
    const bool f64 = c->cfg.precision == RR_PREC_FP64;
    RecLayout L = f64 ? make_layout<double>(c->cfg.npb, c->cfg.ng, c->nldc, grad_layout)
                      : make_layout<float>(c->cfg.npb, c->cfg.ng, c->nldc, grad_layout);
    // FP32 kernel with several passbands: headers and rows of the tile in
    // shared memory (the rows of many passbands do not stay in L1); one
    // passband, the adjoint's record layout (rows 3 + nldc times larger) and
    // the FP64 kernel: headers only, rows through L1/L2
    const bool stage_rows = !f64 && c->cfg.npb > 1 && !grad_layout;
    const int per_pv = stage_rows ? L.head_bytes + L.rows_bytes : L.head_bytes;
    const int pv_tile = pv_tile_for(per_pv);
    const int gpc = groups_per_cta(npt);
    const size_t smem = flux_smem(pv_tile, per_pv, f64, gpc);
    const char* rowsg = (const char*)records + rows_offset(L, npv);
    const int npvt = (npv + pv_tile - 1) / pv_tile;
    const int ngroups = (npt + kWarpPts - 1) / kWarpPts;
    dim3 grid = f64 ? dim3((npt + kPtTile - 1) / kPtTile, npvt) : dim3(npvt, (ngroups + gpc - 1) / gpc);
    if (smem > kMaxSmem || grid.y > 65535u) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if (f64) {
        e = cudaFuncSetAttribute(rr_flux_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        rr_flux_fp64_kernel<<<grid, kBlock, smem, s>>>(times, pb_index, npt, npv, pbp, L, pv_tile,
                                                       (const char*)records, rowsg, (double*)flux, pv_status,
                                                       c->d_err);
    } else {
        bool ss1 = true;
        for (int pb = 0; pb < pbp.npb; ++pb) ss1 = ss1 && pbp.ss[pb] == 1;
        auto kern = c->counting
                        ? (stage_rows ? (ss1 ? rr_flux_mixed_kernel<true, true, true>
                                             : rr_flux_mixed_kernel<true, false, true>)
                                      : (ss1 ? rr_flux_mixed_kernel<false, true, true>
                                             : rr_flux_mixed_kernel<false, false, true>))
                        : (stage_rows ? (ss1 ? rr_flux_mixed_kernel<true, true, false>
                                             : rr_flux_mixed_kernel<true, false, false>)
                                      : (ss1 ? rr_flux_mixed_kernel<false, true, false>
                                             : rr_flux_mixed_kernel<false, false, false>));
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // bit 0: 16-byte stores; bit 1: bulk stores of constant rows (flux in device memory)
        const int vec = (npt % 4 == 0) && (((uintptr_t)flux & 15u) == 0) ? (in_device_memory(flux) ? 3 : 1) : 0;
        kern<<<grid, kBlock, smem, s>>>(times, (const float2*)pts_dt, (const int32_t*)pts_pb,
                                        (const GroupInfo*)pts_grp, npt, npv, pbp, L,
                                        pv_tile, gpc, (const char*)records, rowsg, (float*)flux, pv_status, vec,
                                        ss1 ? kStreamWarpsSS1 : (kBlock >> 5),
                                        c->d_counts ? c->d_counts + (size_t)RR_KERNEL_FLUX * RR_COUNT_KINDS : nullptr,
                                        (const int*)pts_ord, c->d_err);
    }
    c->launches++;
    return cudaGetLastError();
}

}  // namespace rr
