// Bucket walk: the temporal filter and the detector links, one CTA per bucket of 2^LB
// consecutive 2x2 tiles (LB <= 9).
//
// The radix sort orders the batch by bucket only (the tile id's high bits), stably, so
// a bucket's events are contiguous and in arrival order.  The CTA loads them into shared
// memory in pieces of BW_PIECE events and sorts each piece stably by the tile id's low
// bits (warp multisplit ranking): each tile's events are then a contiguous segment in
// arrival order.  A block-wide segmented scan of packed per-sub-pixel counts then splits
// every tile segment stably by sub-pixel ("pixel order": each pixel's events of the
// piece contiguous, in arrival order).  Per piece:
//   - links, one event per thread: one 16-byte record per event in the event ring,
//     {dP, dT, nP, nT} = distance to the previous / next event of the same pixel and of
//     the same tile (0xFFFFFFFF: none): the tile links from the event's neighbours in its
//     tile segment, the pixel links from its neighbours in pixel order; the first event
//     of a pixel / tile in the piece links to the last one before it (an earlier piece or
//     batch), whose next-link it patches in place;
//   - temporal filter (Sec. 4.1: Eq. 7, the EMA of the increment C_p p, then Eq. 6 with
//     the updated average and Eq. 10; FP32 state), by one of two schedules chosen per
//     piece from its longest tile chain (KParams::chain_policy):
//       walk: one thread per tile walks its segment in arrival order with the four
//             pixels' state in registers;
//       scan: per event, Eqs. 7, 6, 10 are one affine map of the pixel's (p_bar, L),
//               M = [[alpha, 0], [-g alpha, beta]],  u = [(1 - alpha) C_p p, g alpha C_p p],
//             g = (1 + beta) / 2 (times the pixel's Sec. 5.2 gain); a block-wide
//             segmented scan composes the maps of each pixel's events in pixel order
//             (segments = pixels), so a chain of any length costs the same few levels.
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
constexpr int BW_PER_THREAD = BW_PIECE / BW_THREADS;  // events per thread in the block scans
// chain_policy 0 (auto): a piece whose longest tile segment is longer than this is
// filtered by the scan (the walk's cost grows with the longest segment, the scan's not)
constexpr unsigned BW_SCAN_RUN = 64;

// x' = [[a, 0], [c, b]] x + [u1, u2] on a pixel's state x = (p_bar, L)
struct Aff {
    float a, c, b, u1, u2;
};

// pixel state tables of a bucket (scan schedule), overlaid on BwSmem::whist
struct BwTables {
    float pb[4 * BW_THREADS], lv[4 * BW_THREADS];  // per pixel slot 4 * local tile + sub-pixel
    unsigned lbase[4 * BW_THREADS];                // S1: list offset + events listed so far
    unsigned ord[4 * BW_THREADS];                  // S1: events listed so far
};

struct BwSmem {
    unsigned long long key[BW_PIECE];          // loaded piece; then packed sub-pixel ranks
    unsigned long long out[BW_PIECE];          // piece in tile order
    unsigned long long plast[4 * BW_THREADS];  // per pixel: its last event before the piece
    unsigned long long tlast[BW_THREADS];      // per tile: its last event before the piece
    unsigned long long subofs[BW_THREADS];     // per tile: 4 x 16-bit sub-pixel offsets in pixel order
    unsigned long long sagg[BW_WARPS];         // block scan: warp aggregates (counts)
    Aff aagg[BW_WARPS];                        // block scan: warp aggregates (affine maps)
    unsigned short rank[BW_PIECE];
    unsigned short pinv[BW_PIECE];             // pixel order -> tile-order position
    unsigned whist[BW_WARPS][BW_THREADS];
    unsigned tstart[BW_THREADS];
    unsigned tcnt[BW_THREADS];
    unsigned warp[BW_WARPS];
    unsigned sflag[BW_WARPS];
    unsigned bucket;
};
static_assert(sizeof(BwTables) <= sizeof(unsigned) * BW_WARPS * BW_THREADS, "tables overlay whist");

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

__device__ __forceinline__ unsigned kof(unsigned long long r) { return (unsigned)(r >> 3) & 0x1FFFFFFFu; }

// g after f
__device__ __forceinline__ Aff aff_then(const Aff &f, const Aff &g)
{
    Aff r;
    r.a = g.a * f.a;
    r.c = g.c * f.a + g.b * f.c;
    r.b = g.b * f.b;
    r.u1 = g.a * f.u1 + g.u1;
    r.u2 = g.c * f.u1 + g.b * f.u2 + g.u2;
    return r;
}

__device__ __forceinline__ Aff aff_shfl_up(const Aff &v, int o)
{
    Aff r;
    r.a = __shfl_up_sync(0xFFFFFFFFu, v.a, o);
    r.c = __shfl_up_sync(0xFFFFFFFFu, v.c, o);
    r.b = __shfl_up_sync(0xFFFFFFFFu, v.b, o);
    r.u1 = __shfl_up_sync(0xFFFFFFFFu, v.u1, o);
    r.u2 = __shfl_up_sync(0xFFFFFFFFu, v.u2, o);
    return r;
}

struct CountOps {
    using T = unsigned long long;
    static __device__ __forceinline__ T ident() { return 0ull; }
    static __device__ __forceinline__ T then(T earlier, T later) { return earlier + later; }
    static __device__ __forceinline__ T shfl_up(T v, int o) { return __shfl_up_sync(0xFFFFFFFFu, v, o); }
    static __device__ __forceinline__ T *agg(BwSmem &S) { return S.sagg; }
};

struct AffOps {
    using T = Aff;
    static __device__ __forceinline__ T ident() { return Aff{1.f, 0.f, 1.f, 0.f, 0.f}; }
    static __device__ __forceinline__ T then(const T &earlier, const T &later) { return aff_then(earlier, later); }
    static __device__ __forceinline__ T shfl_up(const T &v, int o) { return aff_shfl_up(v, o); }
    static __device__ __forceinline__ T *agg(BwSmem &S) { return S.aagg; }
};

// Block-wide exclusive segmented scan: each thread brings the aggregate of its elements
// since its last segment head (`head`: it has one).  Returns the combination of all
// elements from the segment head before the thread's first element up to that element
// (identity where the thread's first element is itself a head, or nothing precedes it).
template <class Ops>
__device__ __forceinline__ typename Ops::T bw_seg_scan(typename Ops::T x, bool head, BwSmem &S)
{
    using T = typename Ops::T;
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    bool f = head;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = Ops::shfl_up(x, o);
        const bool fy = __shfl_up_sync(0xFFFFFFFFu, f, o);
        if (lane >= (unsigned)o) {
            if (!f) x = Ops::then(y, x);
            f = f || fy;
        }
    }
    T ex = Ops::shfl_up(x, 1);
    bool fe = __shfl_up_sync(0xFFFFFFFFu, f, 1);
    if (lane == 0) {
        ex = Ops::ident();
        fe = false;
    }
    T *agg = Ops::agg(S);
    if (lane == 31) {
        agg[w] = x;
        S.sflag[w] = f;
    }
    __syncthreads();
    if (w == 0) {
        // exclusive scan of the warp aggregates
        T v = lane < BW_WARPS ? agg[lane] : Ops::ident();
        bool vf = lane < BW_WARPS ? S.sflag[lane] != 0 : false;
#pragma unroll
        for (int o = 1; o < BW_WARPS; o <<= 1) {
            const T y = Ops::shfl_up(v, o);
            const bool fy = __shfl_up_sync(0xFFFFFFFFu, vf, o);
            if (lane >= (unsigned)o) {
                if (!vf) v = Ops::then(y, v);
                vf = vf || fy;
            }
        }
        T pv = Ops::shfl_up(v, 1);
        if (lane == 0) pv = Ops::ident();
        __syncwarp();
        if (lane < BW_WARPS) agg[lane] = pv;
    }
    __syncthreads();
    if (!fe) ex = Ops::then(agg[w], ex);
    __syncthreads();
    return ex;
}

__device__ __forceinline__ unsigned sub16(unsigned long long packed, unsigned s)
{
    return (unsigned)(packed >> (16 * s)) & 0xFFFFu;
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
        // (the pixels' values at the bucket start stay in memory until the write-back)
        float pb[4], lv[4];
        float gq[4];  // (1 + beta) / 2, times the pixel's gain on Eq. 6 (Sec. 5.2) if set
        unsigned ord[4], soff[4], seen = 0;  // seen: sub-pixels with an event in the bucket
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const unsigned x = 2 * tx + (s & 1), y = 2 * ty + (s >> 1);
            const bool ok = has_tile && x < kp.W && y < kp.H;
            const unsigned pix = ok ? y * kp.W + x : 0u;
            pb[s] = ok ? b.pbar[pix] : 0.f;
            lv[s] = ok ? b.L[pix] : 0.f;
            gq[s] = kGain ? (ok ? kp.g * b.gain[pix] : 0.f) : kp.g;
            S.plast[4 * threadIdx.x + s] = ok ? b.last_pix[pix] : NONE64;
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
            // schedule of the temporal filter for this piece (uniform over the block)
            const bool long_chain = __syncthreads_or(run > BW_SCAN_RUN) != 0;
            const bool scan = kp.chain_policy == 2 || (kp.chain_policy == 0 && long_chain);
            if (threadIdx.x == 0) atomicAdd(scan ? &ctrl->scan_pieces : &ctrl->walk_pieces, 1ull);
            if (kLinks || scan) {
                // pixel order: per event of the tile-ordered piece, its rank among the
                // earlier events of its tile with the same sub-pixel (four 16-bit counters
                // in one word, segmented scan with heads at the tile starts)
                unsigned long long oh[BW_PER_THREAD];
                bool hd[BW_PER_THREAD];
                unsigned long long agg = 0;
                bool any_head = false;
#pragma unroll
                for (int j = 0; j < BW_PER_THREAD; ++j) {
                    const unsigned i = BW_PER_THREAD * threadIdx.x + j;
                    if (i < n) {
                        const unsigned long long r = S.out[i];
                        const unsigned d = (unsigned)(r >> 32) & lmask;
                        oh[j] = 1ull << (16 * ((unsigned)(r >> 1) & 3u));
                        hd[j] = i == S.tstart[d];
                    } else {
                        oh[j] = 0;
                        hd[j] = true;
                    }
                    agg = hd[j] ? oh[j] : agg + oh[j];
                    any_head = any_head || hd[j];
                }
                unsigned long long cur = bw_seg_scan<CountOps>(agg, any_head, S);
#pragma unroll
                for (int j = 0; j < BW_PER_THREAD; ++j) {
                    if (hd[j]) cur = 0;
                    S.key[BW_PER_THREAD * threadIdx.x + j] = cur;  // exclusive ranks
                    cur += oh[j];
                }
                __syncthreads();
                if (run) {
                    const unsigned long long r = S.out[my_start + run - 1];
                    const unsigned long long tot = S.key[my_start + run - 1] + (1ull << (16 * ((unsigned)(r >> 1) & 3u)));
                    const unsigned c0 = sub16(tot, 0), c1 = sub16(tot, 1), c2 = sub16(tot, 2);
                    S.subofs[threadIdx.x] = ((unsigned long long)(c0 + c1 + c2) << 48) |
                                            ((unsigned long long)(c0 + c1) << 32) | ((unsigned long long)c0 << 16);
                }
                __syncthreads();
                for (unsigned i = threadIdx.x; i < n; i += BW_THREADS) {
                    const unsigned long long r = S.out[i];
                    const unsigned d = (unsigned)(r >> 32) & lmask, sp = (unsigned)(r >> 1) & 3u;
                    S.pinv[S.tstart[d] + sub16(S.subofs[d], sp) + sub16(S.key[i], sp)] = (unsigned short)i;
                }
                __syncthreads();
            }
            if (kLinks) {
                // links, one event per thread (reads the last events before the piece)
                for (unsigned i = threadIdx.x; i < n; i += BW_THREADS) {
                    const unsigned long long r = S.out[i];
                    const unsigned d = (unsigned)(r >> 32) & lmask;
                    const unsigned ts = S.tstart[d], te = ts + S.tcnt[d];
                    const unsigned k = kof(r), sp = (unsigned)(r >> 1) & 3u;
                    const unsigned long long g = base + k;
                    unsigned dT, nT = SAT, dP, nP = SAT;
                    if (i > ts) {
                        dT = k - kof(S.out[i - 1]);
                    } else {
                        const unsigned long long tl = S.tlast[d];
                        dT = tl == NONE64 ? SAT : sat_dist2(g, tl);
                        // the tile's previous event (an earlier piece or batch) learns its next
                        if (tl != NONE64 && tl >= live_lo) ring_u[4 * (tl & kp.ring_mask) + 3] = dT;
                    }
                    if (i + 1 < te) nT = kof(S.out[i + 1]) - k;
                    // the same pixel: neighbours in pixel order
                    const unsigned so = sub16(S.subofs[d], sp);
                    const unsigned se = sp < 3 ? sub16(S.subofs[d], sp + 1) : S.tcnt[d];
                    const unsigned rk = sub16(S.key[i], sp);
                    const unsigned pos = ts + so + rk;
                    if (rk > 0) {
                        dP = k - kof(S.out[S.pinv[pos - 1]]);
                    } else {
                        const unsigned long long pl = S.plast[4 * d + sp];
                        dP = pl == NONE64 ? SAT : sat_dist2(g, pl);
                        if (pl != NONE64 && pl >= live_lo) ring_u[4 * (pl & kp.ring_mask) + 2] = dP;
                    }
                    if (so + rk + 1 < se) nP = kof(S.out[S.pinv[pos + 1]]) - k;
                    b.ring4[g & kp.ring_mask] = make_uint4(dP, dT, nP, nT);
                }
                __syncthreads();
            }
            if (!scan) {
                // walk: this thread's tile, in arrival order
                const unsigned e0 = my_start, e1 = my_start + run;
                unsigned long long lastg[4] = {NONE64, NONE64, NONE64, NONE64};
                for (unsigned i = e0; i < e1; ++i) {
                    const unsigned long long r = S.out[i];
                    const unsigned k = kof(r);
                    const int sp = (int)(r >> 1) & 3;
                    const bool off_ev = r & 1u;
                    float pbs = pb[0], lvs = lv[0], gs = gq[0];
#pragma unroll
                    for (int qq = 1; qq < 4; ++qq)
                        if (qq == sp) { pbs = pb[qq]; lvs = lv[qq]; gs = gq[qq]; }
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
                            if (qq == sp) { os = ord[qq]; ps0 = soff[qq]; }
                        b.plist[ps0 + os] = k;
                        b.plnb[ps0 + os] = lvs;
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) ord[qq] += (qq == sp);
                    }
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq)
                        if (qq == sp) { pb[qq] = pbs; lv[qq] = lvs; lastg[qq] = base + k; }
                }
                // the tile's and its pixels' last events for the next piece
                if (run) {
                    S.tlast[threadIdx.x] = base + kof(S.out[e1 - 1]);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq)
                        if (lastg[qq] != NONE64) {
                            S.plast[4 * threadIdx.x + qq] = lastg[qq];
                            seen |= 1u << qq;
                        }
                }
            } else {
                // scan: the tile's pixel states go to shared memory, every event is an
                // affine map of its pixel's state, composed along the pixel order.  A run's
                // first event folds the pixel's state at the piece start into its map (a
                // constant map), so every composed map is constant: its u1, u2 are the
                // state after that event.  Only run heads read the state table, before the
                // scan's barriers; only run ends write it, after them.
                BwTables &T = *reinterpret_cast<BwTables *>(&S.whist[0][0]);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    T.pb[4 * threadIdx.x + qq] = pb[qq];
                    T.lv[4 * threadIdx.x + qq] = lv[qq];
                    if (kS1) {
                        T.lbase[4 * threadIdx.x + qq] = soff[qq] + ord[qq];
                        T.ord[4 * threadIdx.x + qq] = ord[qq];
                    }
                }
                __syncthreads();
                float2 *hstate = reinterpret_cast<float2 *>(S.key);  // per pixel-order position
                const unsigned e_begin = BW_PER_THREAD * threadIdx.x;
                // the affine map of the event at pixel-order position e (e < n), its slot
                auto event_map = [&](unsigned e, unsigned &slot_out, unsigned &k_out) {
                    const unsigned long long r = S.out[S.pinv[e]];
                    const unsigned d = (unsigned)(r >> 32) & lmask, sp = (unsigned)(r >> 1) & 3u;
                    slot_out = 4 * d + sp;
                    k_out = kof(r);
                    float gs = kp.g;
                    if (kGain) {
                        const unsigned tl = (bk << LB) + d;
                        const unsigned x = 2 * (tl % kp.tiles_w) + (sp & 1u), y = 2 * (tl / kp.tiles_w) + (sp >> 1);
                        gs = kp.g * b.gain[y * kp.W + x];
                    }
                    // Eqs. 2-3, 7, 6, 10 as one affine map of (p_bar, L)
                    const float inc = (r & 1u) ? -kp.c_off : kp.c_on;
                    const float ga = gs * kp.a;
                    return Aff{kp.a, -ga, kp.b, kp.oma * inc, ga * inc};
                };
                unsigned prev_slot = ~0u;
                if (e_begin > 0 && e_begin < n) {
                    const unsigned long long rp = S.out[S.pinv[e_begin - 1]];
                    prev_slot = 4 * ((unsigned)(rp >> 32) & lmask) + ((unsigned)(rp >> 1) & 3u);
                }
                const unsigned first_slot = prev_slot;
                Aff agg = AffOps::ident();
                bool any_head = false;
#pragma unroll
                for (int j = 0; j < BW_PER_THREAD; ++j) {
                    const unsigned e = e_begin + j;
                    if (e >= n) break;
                    unsigned sl, k;
                    Aff m = event_map(e, sl, k);
                    if (sl != prev_slot) {
                        // run head: the state after it, from the state at the piece start
                        const float p0 = T.pb[sl], v0 = T.lv[sl];
                        const float p1 = m.a * p0 + m.u1;
                        const float v1 = m.c * p0 + m.b * v0 + m.u2;
                        hstate[e] = make_float2(p1, v1);
                        agg = Aff{0.f, 0.f, 0.f, p1, v1};
                        any_head = true;
                    } else {
                        agg = aff_then(agg, m);
                    }
                    prev_slot = sl;
                }
                Aff cur = bw_seg_scan<AffOps>(agg, any_head, S);
                prev_slot = first_slot;
#pragma unroll
                for (int j = 0; j < BW_PER_THREAD; ++j) {
                    const unsigned e = e_begin + j;
                    if (e >= n) break;
                    unsigned sl, k;
                    const Aff m = event_map(e, sl, k);
                    if (sl != prev_slot) {
                        const float2 hs = hstate[e];
                        cur = Aff{0.f, 0.f, 0.f, hs.x, hs.y};
                    } else {
                        cur = aff_then(cur, m);
                    }
                    prev_slot = sl;
                    if (kS1) {
                        const unsigned d = sl >> 2, sp = sl & 3u;
                        const unsigned rk = e - S.tstart[d] - sub16(S.subofs[d], sp);
                        b.plist[T.lbase[sl] + rk] = k;
                        b.plnb[T.lbase[sl] + rk] = cur.u2;
                    }
                    // the last event of each pixel's run stores the pixel's new state
                    bool last = e + 1 >= n;
                    if (!last) {
                        const unsigned long long rn = S.out[S.pinv[e + 1]];
                        last = 4 * ((unsigned)(rn >> 32) & lmask) + ((unsigned)(rn >> 1) & 3u) != sl;
                    }
                    if (last) {
                        T.pb[sl] = cur.u1;
                        T.lv[sl] = cur.u2;
                    }
                }
                __syncthreads();
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    pb[qq] = T.pb[4 * threadIdx.x + qq];
                    lv[qq] = T.lv[4 * threadIdx.x + qq];
                }
                // the tile's and its pixels' last events, and the S1 list positions
                if (run) {
                    S.tlast[threadIdx.x] = base + kof(S.out[my_start + run - 1]);
                    const unsigned long long so = S.subofs[threadIdx.x];
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        const unsigned lo = sub16(so, qq), hi = qq < 3 ? sub16(so, qq + 1) : run;
                        if (hi > lo) {
                            S.plast[4 * threadIdx.x + qq] = base + kof(S.out[S.pinv[my_start + hi - 1]]);
                            seen |= 1u << qq;
                            if (kS1) ord[qq] += hi - lo;
                        }
                    }
                }
            }
            __syncthreads();
        }
        // write back the tile's state
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!(seen >> s & 1u)) continue;  // only pixels inside the sensor have events
            const unsigned pix = (2 * ty + (s >> 1)) * kp.W + 2 * tx + (s & 1);
            if (kS1) {
                const unsigned long long lp0 = b.last_pix[pix];  // before this batch
                long long prev = -0x7FFFFFFFll - 1;  // no earlier event
                if (lp0 != NONE64) {
                    const long long rel = (long long)(lp0 - base);
                    prev = rel < -0x40000000ll ? -0x40000000ll : rel;
                }
                b.s1_info[pix] = make_int4(batch_no, (int)soff[s], (int)ord[s], (int)prev);
                b.s1_linit[pix] = b.L[pix];  // L at the batch start
            }
            b.pbar[pix] = pb[s];
            b.L[pix] = lv[s];
            b.last_pix[pix] = S.plast[4 * threadIdx.x + s];
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
    return launch_pdl(k_bwalk<kLinks, kS1, kGain>, grid_for(kp, 2), BW_THREADS, smem, s, kp, b, sorted);
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
