// Bucket walk: the temporal filter and the detector links, one CTA per bucket of 2^LB
// consecutive 2x2 tiles (LB <= 9).
//
// The radix sort orders the batch by bucket only (the tile id's high bits), stably, so
// a bucket's events are contiguous and in arrival order.  The CTA loads them into shared
// memory in pieces of BW_PIECE events and sorts each piece stably by the tile id's low
// bits (warp multisplit ranking): each tile's events are then a contiguous segment in
// arrival order.  Per piece:
//   - links, one event per thread: one 16-byte record per event in the event ring,
//     {dP, dT, nP, nT} = distance to the previous / next event of the same pixel and of
//     the same tile (0xFFFFFFFF: none), from the event's neighbours in its tile segment
//     (same pixel: the nearest with the same sub-pixel); the first event of a pixel /
//     tile in the piece links to the last one before it (an earlier piece or batch),
//     whose next-link it patches in place;
//   - temporal filter, one thread per tile walking its segment in arrival order with
//     the four pixels' state in registers (Sec. 4.1): Eq. 7 (EMA of the increment
//     C_p p), Eq. 6 with the updated average, Eq. 10; FP32 state.
// The active event queue of Sec. 4.2 is the index window [h, k]; with these links a
// push activates a pixel iff dP > k - h, and popping event j deactivates it iff
// nP(j) > k - j (likewise for tiles), so the detector never touches a per-pixel counter.
// S1 additionally writes, per pixel, the list of its batch events and L after each
// (without this batch's blurs), grouped by pixel inside the bucket.
#include "fibar_internal.cuh"

namespace fibar {

constexpr int BW_THREADS = 512;  // = max tiles per bucket
constexpr int BW_PIECE = 2048;
constexpr int BW_WARPS = BW_THREADS / 32;
constexpr int BW_PER_WARP = BW_PIECE / BW_WARPS;  // 256 events ranked by each warp

struct BwSmem {
    unsigned long long key[BW_PIECE];
    unsigned long long out[BW_PIECE];
    unsigned long long plast[4 * BW_THREADS];  // per pixel: its last event before the piece
    unsigned long long tlast[BW_THREADS];      // per tile: its last event before the piece
    unsigned short rank[BW_PIECE];
    unsigned whist[BW_WARPS][BW_THREADS];
    unsigned tstart[BW_THREADS];
    unsigned tcnt[BW_THREADS];
    unsigned warp[BW_WARPS];
    unsigned bucket;
};

__device__ __forceinline__ unsigned sat_dist2(unsigned long long later, unsigned long long earlier)
{
    const unsigned long long d = later - earlier;
    return d >= SAT ? SAT : (unsigned)d;
}

// exclusive scan over the block (BW_THREADS values); returns the total in *tot
__device__ __forceinline__ unsigned bw_scan(unsigned v, unsigned *s_warp, unsigned *tot)
{
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned t = lane < BW_WARPS ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < BW_WARPS) s_warp[lane] = t;  // inclusive
    }
    __syncthreads();
    const unsigned wex = w ? s_warp[w - 1] : 0u;
    *tot = s_warp[BW_WARPS - 1];
    const unsigned r = wex + x - v;
    __syncthreads();
    return r;
}

template <bool kLinks, bool kS1, bool kGain>
__global__ void __launch_bounds__(BW_THREADS, 2)
k_bwalk(KParams kp, Bufs b, const unsigned long long *srt)
{
    PDL_ENTRY();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwSmem &S = *reinterpret_cast<BwSmem *>(smem_raw);
    Ctrl *ctrl = b.ctrl;
    const unsigned m = ctrl->m;
    const unsigned long long base = ctrl->base;
    const int batch_no = (int)ctrl->batch_no;
    const unsigned LB = kp.lb;
    const unsigned lmask = (1u << LB) - 1u;
    const unsigned nbuckets = kp.nbuckets;
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned long long live_lo = base > kp.live ? base - kp.live : 0ull;
    unsigned *ring_u = reinterpret_cast<unsigned *>(b.ring4);

    for (;;) {
        if (threadIdx.x == 0) S.bucket = atomicAdd(&ctrl->walk_ticket, 1u);
        __syncthreads();
        if (S.bucket >= nbuckets) break;
        // largest buckets first when the decode ordered them (fewer CTAs idle at the end)
        const unsigned bk = b.bucket_order ? b.bucket_order[S.bucket] : S.bucket;
        const unsigned bs = b.bucket_start[bk];
        const unsigned be = bk + 1 < nbuckets ? b.bucket_start[bk + 1] : m;
        if (bs >= be) {
            __syncthreads();
            continue;
        }
        // this thread's tile and its four pixels
        const unsigned tile = (bk << LB) + threadIdx.x;
        const bool has_tile = threadIdx.x <= lmask && tile < kp.ntiles;
        const unsigned tx = has_tile ? tile % kp.tiles_w : 0u, ty = has_tile ? tile / kp.tiles_w : 0u;
        unsigned pix[4];
        bool ok[4];
        float pb[4], lv[4], l0[4];
        float gq[4];  // (1 + beta) / 2, times the pixel's gain on Eq. 6 (Sec. 5.2) if set
        unsigned long long lp0[4];
        unsigned ord[4], soff[4], seen = 0;  // seen: sub-pixels with an event in the bucket
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const unsigned x = 2 * tx + (s & 1), y = 2 * ty + (s >> 1);
            ok[s] = has_tile && x < kp.W && y < kp.H;
            pix[s] = ok[s] ? y * kp.W + x : 0u;
            pb[s] = ok[s] ? b.pbar[pix[s]] : 0.f;
            lv[s] = ok[s] ? b.L[pix[s]] : 0.f;
            l0[s] = lv[s];
            gq[s] = kGain ? (ok[s] ? kp.g * b.gain[pix[s]] : 0.f) : kp.g;
            lp0[s] = ok[s] ? b.last_pix[pix[s]] : NONE64;
            S.plast[4 * threadIdx.x + s] = lp0[s];
            ord[s] = 0;
            soff[s] = 0;
        }
        S.tlast[threadIdx.x] = has_tile ? b.last_tile[tile] : NONE64;

        if (kS1) {
            // per (tile, sub-pixel) counts over the whole bucket -> list offsets
            unsigned *cnt4 = &S.whist[0][0];  // 4 * BW_THREADS counters
            for (unsigned i = threadIdx.x; i < 4u * BW_THREADS; i += BW_THREADS) cnt4[i] = 0;
            __syncthreads();
            for (unsigned i = bs + threadIdx.x; i < be; i += BW_THREADS) {
                const unsigned long long r = srt[i];
                const unsigned lt = (unsigned)(r >> 32) & lmask;
                atomicAdd(&cnt4[lt * 4 + ((unsigned)(r >> 1) & 3u)], 1u);
            }
            __syncthreads();
            const unsigned c0 = cnt4[threadIdx.x * 4], c1 = cnt4[threadIdx.x * 4 + 1];
            const unsigned c2 = cnt4[threadIdx.x * 4 + 2], c3 = cnt4[threadIdx.x * 4 + 3];
            unsigned tot;
            const unsigned ex = bw_scan(c0 + c1 + c2 + c3, S.warp, &tot);
            soff[0] = bs + ex;
            soff[1] = soff[0] + c0;
            soff[2] = soff[1] + c1;
            soff[3] = soff[2] + c2;
        }

        for (unsigned p0 = bs; p0 < be; p0 += BW_PIECE) {
            const unsigned n = min((unsigned)BW_PIECE, be - p0);
            for (unsigned i = threadIdx.x; i < BW_PIECE; i += BW_THREADS) {
                S.key[i] = i < n ? srt[p0 + i] : ~0ull;
            }
            for (unsigned i = threadIdx.x; i < BW_WARPS * BW_THREADS; i += BW_THREADS) (&S.whist[0][0])[i] = 0;
            __syncthreads();
            // stable rank within (warp range, local tile)
            for (int q = 0; q < BW_PER_WARP / 32; ++q) {
                const unsigned r = w * BW_PER_WARP + q * 32 + lane;
                const bool valid = r < n;
                const unsigned d = valid ? (unsigned)(S.key[r] >> 32) & lmask : BW_THREADS;
                const unsigned peers = warp_peers<10>(d);  // local tile < 512, or 512 (none)
                const unsigned rk = __popc(peers & lt_mask);
                if (valid) S.rank[r] = (unsigned short)(S.whist[w][d] + rk);
                __syncwarp();
                if (valid && rk == 0) S.whist[w][d] += __popc(peers);
                __syncwarp();
            }
            __syncthreads();
            // per local tile: exclusive offsets of each warp, the tile's count, its start
            unsigned run = 0;
            for (int ww = 0; ww < BW_WARPS; ++ww) {
                const unsigned c = S.whist[ww][threadIdx.x];
                S.whist[ww][threadIdx.x] = run;
                run += c;
            }
            unsigned tot;
            const unsigned my_start = bw_scan(run, S.warp, &tot);
            S.tstart[threadIdx.x] = my_start;
            S.tcnt[threadIdx.x] = run;
            __syncthreads();
            for (unsigned i = threadIdx.x; i < n; i += BW_THREADS) {
                const unsigned long long kk = S.key[i];
                const unsigned d = (unsigned)(kk >> 32) & lmask;
                S.out[S.tstart[d] + S.whist[i / BW_PER_WARP][d] + S.rank[i]] = kk;
            }
            __syncthreads();
            if (kLinks) {
                // links, one event per thread (reads the last events before the piece)
                for (unsigned i = threadIdx.x; i < n; i += BW_THREADS) {
                    const unsigned long long r = S.out[i];
                    const unsigned d = (unsigned)(r >> 32) & lmask;
                    const unsigned ts = S.tstart[d], te = ts + S.tcnt[d];
                    const unsigned k = (unsigned)(r >> 3) & 0x1FFFFFFFu, s = (unsigned)(r >> 1) & 3u;
                    const unsigned long long g = base + k;
                    unsigned dT, nT = SAT, dP = SAT, nP = SAT;
                    if (i > ts) {
                        dT = k - ((unsigned)(S.out[i - 1] >> 3) & 0x1FFFFFFFu);
                    } else {
                        const unsigned long long tl = S.tlast[d];
                        dT = tl == NONE64 ? SAT : sat_dist2(g, tl);
                        // the tile's previous event (an earlier piece or batch) learns its next
                        if (tl != NONE64 && tl >= live_lo) ring_u[4 * (tl & kp.ring_mask) + 3] = dT;
                    }
                    if (i + 1 < te) nT = ((unsigned)(S.out[i + 1] >> 3) & 0x1FFFFFFFu) - k;
                    // the same pixel: nearest earlier / later event of the segment with sub-pixel s
                    bool found = false;
                    for (unsigned j = i; j > ts && !found; --j) {
                        const unsigned long long rj = S.out[j - 1];
                        if (((unsigned)(rj >> 1) & 3u) == s) {
                            dP = k - ((unsigned)(rj >> 3) & 0x1FFFFFFFu);
                            found = true;
                        }
                    }
                    if (!found) {
                        const unsigned long long pl = S.plast[4 * d + s];
                        dP = pl == NONE64 ? SAT : sat_dist2(g, pl);
                        if (pl != NONE64 && pl >= live_lo) ring_u[4 * (pl & kp.ring_mask) + 2] = dP;
                    }
                    for (unsigned j = i + 1; j < te; ++j) {
                        const unsigned long long rj = S.out[j];
                        if (((unsigned)(rj >> 1) & 3u) == s) {
                            nP = ((unsigned)(rj >> 3) & 0x1FFFFFFFu) - k;
                            break;
                        }
                    }
                    b.ring4[g & kp.ring_mask] = make_uint4(dP, dT, nP, nT);
                }
                __syncthreads();
            }
            // temporal filter: this thread's tile, in arrival order
            const unsigned e0 = my_start, e1 = my_start + run;
            unsigned long long lastg[4] = {NONE64, NONE64, NONE64, NONE64};
            for (unsigned i = e0; i < e1; ++i) {
                const unsigned long long r = S.out[i];
                const unsigned k = (unsigned)(r >> 3) & 0x1FFFFFFFu;
                const int s = (int)(r >> 1) & 3;
                const bool off_ev = r & 1u;
                float pbs = pb[0], lvs = lv[0], gs = gq[0];
#pragma unroll
                for (int qq = 1; qq < 4; ++qq)
                    if (qq == s) { pbs = pb[qq]; lvs = lv[qq]; gs = gq[qq]; }
                if (!kGain) gs = kp.g;
                // Eqs. 2-3: increment C_p p; Eq. 7 then Eq. 6 (updated average, times the
                // pixel's gain when one is set) and Eq. 10
                const float inc = off_ev ? -kp.c_off : kp.c_on;
                pbs = kp.a * pbs + kp.oma * inc;
                lvs = kp.b * lvs + gs * (inc - pbs);
                if (kS1) {
                    unsigned os = ord[0], ps0 = soff[0];
#pragma unroll
                    for (int qq = 1; qq < 4; ++qq)
                        if (qq == s) { os = ord[qq]; ps0 = soff[qq]; }
                    b.plist[ps0 + os] = k;
                    b.plnb[ps0 + os] = lvs;
                    b.epos[k] = os;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) ord[qq] += (qq == s);
                }
#pragma unroll
                for (int qq = 0; qq < 4; ++qq)
                    if (qq == s) { pb[qq] = pbs; lv[qq] = lvs; lastg[qq] = base + k; }
            }
            // the tile's and its pixels' last events for the next piece
            if (run) {
                S.tlast[threadIdx.x] = base + ((S.out[e1 - 1] >> 3) & 0x1FFFFFFFull);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq)
                    if (lastg[qq] != NONE64) {
                        S.plast[4 * threadIdx.x + qq] = lastg[qq];
                        seen |= 1u << qq;
                    }
            }
            __syncthreads();
        }
        // write back the tile's state
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!ok[s] || !(seen >> s & 1u)) continue;
            b.pbar[pix[s]] = pb[s];
            b.L[pix[s]] = lv[s];
            b.last_pix[pix[s]] = S.plast[4 * threadIdx.x + s];
            if (kS1) {
                long long prev = -0x7FFFFFFFll - 1;  // no earlier event
                if (lp0[s] != NONE64) {
                    const long long rel = (long long)(lp0[s] - base);
                    prev = rel < -0x40000000ll ? -0x40000000ll : rel;
                }
                b.s1_info[pix[s]] = make_int4(batch_no, (int)soff[s], (int)ord[s], (int)prev);
                b.s1_linit[pix[s]] = l0[s];
            }
        }
        if (has_tile && seen) b.last_tile[tile] = S.tlast[threadIdx.x];
        __syncthreads();
    }
}

size_t bwalk_smem() { return sizeof(BwSmem); }

template <bool kLinks, bool kS1, bool kGain>
static cudaError_t walk_variant(const KParams &kp, const Bufs &b, const unsigned long long *sorted, cudaStream_t s)
{
    static std::atomic<unsigned long long> attr_done{0};
    const size_t smem = sizeof(BwSmem);
    if (cudaError_t e = smem_attr_once(attr_done, k_bwalk<kLinks, kS1, kGain>, smem)) return e;
    return launch_pdl(k_bwalk<kLinks, kS1, kGain>, grid_for(2), BW_THREADS, smem, s, kp, b, sorted);
}

cudaError_t launch_walk(const KParams &kp, const Bufs &b_in, const unsigned long long *sorted, unsigned sort_passes,
                        cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    Bufs b = b_in;
    if (sort_passes != 1) b.bucket_order = nullptr;  // only a one-pass sort's decode orders them
    const bool gain = b.gain != nullptr;
    cudaError_t e;
    if (kp.spatial && kp.blur_mode == 0)
        e = gain ? walk_variant<true, true, true>(kp, b, sorted, s) : walk_variant<true, true, false>(kp, b, sorted, s);
    else if (kp.spatial)
        e = gain ? walk_variant<true, false, true>(kp, b, sorted, s) : walk_variant<true, false, false>(kp, b, sorted, s);
    else
        e = gain ? walk_variant<false, false, true>(kp, b, sorted, s) : walk_variant<false, false, false>(kp, b, sorted, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace fibar
