// Stale-pixel detector (Sec. 4.2 steps 2-3, Eqs. 19-20), evaluated exactly for every
// event, in parallel by speculation over chunks of CHUNK events.
//
// State after step k: the window [h, k] of queued events.  The distinct pixel and tile
// counts N_ap, N_at and therefore q_targ_{k+1} (Eq. 20) are functions of the window, so
// two runs that reach the same h at the same k agree from then on.  One step:
//   push k:  N_ap += dP(k) > k - h   (the pixel had no queued event), same for tiles;
//   pop:     while q = k - h + 1 exceeds q_targ_k: event j = h leaves; N_ap -= nP(j) > k - j;
//            h += 1.  A pixel whose last queued event leaves is stale from this step on;
//   Eq. 20:  q_targ_{k+1} = clamp(floor(q * fill_num * 4 * N_at / (fill_den * N_ap))),
//            kept as the ratio X / Y: "q > q_targ" is tested as q > q_min and
//            (q > q_max or q * Y > X), which needs no division.
//
// Pass 1: chunk c starts from a guessed window slightly longer than the true one: the
//         shortest chunk-aligned window that the regulator would shrink, plus a margin
//         (k_det_hist, k_det_init); its exact distinct counts come from per-chunk suffix
//         histograms.  A too-long window pops down to its target in the first steps and
//         then coincides with the true trajectory; each chunk also warms up over the
//         previous chunk.
// Pass 2: chunk c restarts from pass 1's exit state of chunk c-1 and runs until its
//         queue length equals pass 1's at the same step (the trajectories merged).
// Fixup:  if some chunk did not merge, one thread walks the chunks in order and re-runs
//         exactly those whose entry state was wrong.  The result is exact in all cases.
#include "fibar_internal.cuh"

namespace fibar {

struct Geo {
    unsigned long long base;
    unsigned m, S, nchunks, Gold;
};

// Chunk length S: at least CHUNK, at most DET_MAX_CHUNKS chunks per batch, and DET_G
// chunks must cover twice the queue length at the batch start.
__device__ __forceinline__ Geo geometry(const KParams &kp, const Ctrl *ctrl)
{
    Geo g;
    g.base = ctrl->base;
    g.m = ctrl->m;
    const unsigned long long qprev = g.base - (unsigned long long)ctrl->det.h;
    unsigned long long S = (2ull * qprev + 4ull * CHUNK + DET_G - 1) / DET_G;
    S = max(S, ((unsigned long long)g.m + DET_MAX_CHUNKS - 1) / DET_MAX_CHUNKS);
    S = (S + 15) / 16 * 16;
    g.S = (unsigned)max((unsigned long long)CHUNK, S);
    g.nchunks = (g.m + g.S - 1) / g.S;
    const unsigned long long old_chunks = (g.base + g.S - 1) / g.S;
    g.Gold = (unsigned)min((unsigned long long)DET_G, old_chunks);
    return g;
}

// the two halves of an event's ring record: {dP, dT} (previous) and {nP, nT} (next)
__device__ __forceinline__ uint2 prv_of(const uint4 *ring, unsigned long long slot)
{
    return reinterpret_cast<const uint2 *>(ring)[2 * slot];
}
__device__ __forceinline__ uint2 nxt_of(const uint4 *ring, unsigned long long slot)
{
    return reinterpret_cast<const uint2 *>(ring)[2 * slot + 1];
}

__device__ __forceinline__ unsigned warp_sum(unsigned v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Chunk of a batch-relative index (indices below -Gold*S are never asked for).
__device__ __forceinline__ long long chunk_of(long long x, unsigned S, unsigned Gold)
{
    return (x + (long long)Gold * S) / S - Gold;
}

// Suffix histograms, stored transposed: for chunk c' (old chunks -Gold..-1 and the
// batch's chunks) and distance g = 1..DET_G,
//   Mt[t][g][c' + Gold] = #{j in c' : next(j) >= (c'+g) S}      (t = 0 pixels, 1 tiles)
// i.e. the events of c' still last of their pixel / tile at the start of chunk c'+g.
// The distinct counts of the aligned window [(c-g)S, cS) are then
// N(c, g) = sum_{g'=1..g} Mt[g'][c - g'], which lanes handling consecutive chunks read
// with coalesced loads.  A block handles HB_CHUNKS consecutive chunks: each warp builds
// one chunk's histogram in shared memory, the block writes the rows out per distance.
constexpr int HB_CHUNKS = 32;

struct HistSmem {
    unsigned hist[8][DET_G + 1];
    unsigned short tile[HB_CHUNKS][DET_G + 1];
};

__global__ void __launch_bounds__(256)
k_det_hist(KParams kp, Ctrl *ctrl, const uint4 *ring, unsigned short *Mt, size_t mt_stride)
{
    PDL_ENTRY();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HistSmem &H = *reinterpret_cast<HistSmem *>(smem_raw);
    const Geo g = geometry(kp, ctrl);
    const unsigned lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const unsigned nwork = g.nchunks + g.Gold;
    const unsigned nblk = (nwork + HB_CHUNKS - 1) / HB_CHUNKS;
    const long long lo_exist = -(long long)g.base;
    for (unsigned blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        for (int t = 0; t < 2; ++t) {  // pixels, then tiles
            for (unsigned cc = wl; cc < HB_CHUNKS; cc += 8) {
                const unsigned wi = blk * HB_CHUNKS + cc;
                unsigned *hp = H.hist[wl];
                for (unsigned i = lane; i <= DET_G; i += 32) hp[i] = 0;
                __syncwarp();
                if (wi < nwork) {
                    const long long c = (long long)wi - (long long)g.Gold;
                    const long long lo = c * g.S;
                    for (unsigned r = lane; r < g.S; r += 32) {
                        const long long j = lo + r;
                        if (j < lo_exist || j >= (long long)g.m) continue;
                        const uint2 n = nxt_of(ring, (g.base + (unsigned long long)j) & kp.ring_mask);
                        const unsigned nv = t ? n.y : n.x;
                        const long long d = nv == SAT ? DET_G : min((long long)DET_G, chunk_of(j + nv, g.S, g.Gold) - c);
                        atomicAdd(&hp[d], 1u);
                    }
                }
                __syncwarp();
                // suffix sums over d; lane owns d in [lane*BPL, lane*BPL+BPL)
                constexpr int BPL = (DET_G + 1) / 32;
                unsigned sp = 0;
#pragma unroll 8
                for (int i = 0; i < BPL; ++i) sp += hp[lane * BPL + i];
                unsigned xp = sp;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned yp = __shfl_down_sync(0xFFFFFFFFu, xp, o);
                    if (lane + o < 32) xp += yp;
                }
                unsigned rp = xp - sp;  // counts of d above this lane's range
#pragma unroll 8
                for (int i = BPL - 1; i >= 0; --i) {
                    const unsigned d = lane * BPL + i;
                    rp += hp[d];
                    H.tile[cc][d] = (unsigned short)rp;
                }
                __syncwarp();
            }
            __syncthreads();
            // write out transposed: row g holds the chunks' values contiguously
            unsigned short *base_t = Mt + (size_t)t * (DET_G + 1) * mt_stride;
            const unsigned c_first = blk * HB_CHUNKS;
            for (unsigned gg = wl + 1; gg <= DET_G; gg += 8) {
                if (c_first + lane < nwork) base_t[(size_t)gg * mt_stride + c_first + lane] = H.tile[lane][gg];
            }
            __syncthreads();
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->S = g.S;
        ctrl->nchunks = g.nchunks;
        ctrl->G = DET_G;
        ctrl->Gold = g.Gold;
    }
}

// Speculative start of chunk c (c >= 1).  Lanes handle 32 consecutive chunks and scan the
// aligned windows g = 1..DET_G ending just before their chunk (coalesced rows of Mt),
// keeping the shortest one that the regulator would shrink at the next event (its length
// is at the equilibrium of Eq. 20, to within one chunk) plus DET_MARGIN chunks: a slight
// overestimate of the true queue, which merges with the true trajectory within a few
// tens of events.  Then, chunk by chunk, the warp applies the chunk's first event exactly,
// popping the excess in parallel.
__global__ void __launch_bounds__(256)
k_det_init(KParams kp, const Ctrl *ctrl, const uint4 *ring, const unsigned short *Mt, size_t mt_stride,
           unsigned *qout, DetState *E0)
{
    PDL_ENTRY();
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long base = ctrl->base;
    const unsigned S = ctrl->S, nch = ctrl->nchunks, Gold = ctrl->Gold;
    const unsigned warps_total = gridDim.x * (blockDim.x >> 5);
    const unsigned short *MP = Mt, *MT = Mt + (size_t)(DET_G + 1) * mt_stride;
    for (unsigned cb = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; cb < nch; cb += warps_total * 32) {
        const unsigned c = cb + lane;
        const bool real = c >= 1 && c < nch;
        const unsigned long long reach = (unsigned long long)c * S + base;  // events before the chunk
        unsigned np = 0, nt = 0, gsel = 0, snp = 0, snt = 0, found = 0;
        for (unsigned g0 = 1; g0 <= DET_G; g0 += 8) {
            // the next 8 distances' counts, all loads in flight together
            unsigned short vp[8], vt[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const unsigned gg = g0 + u;
                const long long cw = (long long)c - gg;  // chunk entering the window
                vp[u] = vt[u] = 0;
                if (real && gg <= DET_G && cw >= -(long long)Gold) {
                    const size_t col = (size_t)(cw + Gold);
                    vp[u] = MP[(size_t)gg * mt_stride + col];
                    vt[u] = MT[(size_t)gg * mt_stride + col];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const unsigned gg = g0 + u;
                if (gg > DET_G) break;
                np += vp[u];
                nt += vt[u];
                if (real && !found) {
                    const unsigned long long L = min((unsigned long long)gg * S, reach);
                    const unsigned long long X = L * kp.numA * nt, Y = (unsigned long long)kp.den * np;
                    const unsigned long long q = L + 1;
                    if (np > 0 && q > kp.q_min && (q > kp.q_max || q * Y > X)) found = gg;
                }
                if (real && gsel == 0 && (found ? gg == min(found + DET_MARGIN, (unsigned)DET_G) : gg == DET_G)) {
                    gsel = gg;
                    snp = np;
                    snt = nt;
                }
            }
            if (!__any_sync(0xFFFFFFFFu, real && gsel == 0)) break;  // every lane has its window
        }
        // chunk by chunk: the first event of the chunk, pops counted by the whole warp
        const unsigned todo = __ballot_sync(0xFFFFFFFFu, real);
        for (unsigned bits = todo; bits; bits &= bits - 1) {
            const int src = __ffs(bits) - 1;
            const unsigned cc = cb + src;
            const unsigned gs = __shfl_sync(0xFFFFFFFFu, gsel, src);
            const unsigned nap0 = __shfl_sync(0xFFFFFFFFu, snp, src);
            const unsigned nat0 = __shfl_sync(0xFFFFFFFFu, snt, src);
            const long long k0 = (long long)cc * S;
            const long long hs = max(k0 - (long long)gs * S, -(long long)base);
            const unsigned long long L = (unsigned long long)(k0 - hs);
            unsigned long long X = L * kp.numA * nat0, Y = (unsigned long long)kp.den * nap0;
            if (nap0 == 0) { X = kp.q_min; Y = 1; }
            const uint2 d = prv_of(ring, (base + (unsigned long long)k0) & kp.ring_mask);
            const unsigned nap = nap0 + ((long long)d.x > (long long)L);
            const unsigned nat = nat0 + ((long long)d.y > (long long)L);
            const unsigned long long q = L + 1;
            unsigned long long qt = X / Y;
            qt = min(qt, (unsigned long long)kp.q_max);
            qt = max(qt, (unsigned long long)kp.q_min);
            const unsigned long long npop = q > qt ? q - qt : 0ull;
            unsigned dp = 0, dtt = 0;
            for (unsigned long long i = lane; i < npop; i += 32) {
                const long long j = hs + (long long)i;
                const uint2 nn = nxt_of(ring, (base + (unsigned long long)j) & kp.ring_mask);
                dp += (long long)nn.x > k0 - j;
                dtt += (long long)nn.y > k0 - j;
            }
            dp = warp_sum(dp);
            dtt = warp_sum(dtt);
            if (lane == 0) {
                DetState st0;
                const unsigned long long qa = q - npop;
                st0.h = hs + (long long)npop;
                st0.nap = nap - dp;
                st0.nat = nat - dtt;
                st0.X = qa * kp.numA * st0.nat;
                st0.Y = (unsigned long long)kp.den * st0.nap;
                E0[cc] = st0;
                qout[k0] = (unsigned)qa;
            }
        }
    }
}

// Run the detector over chunks with groups of GW lanes, 32/GW chunks per warp.  All lanes
// of a group hold the same state of their chunk.  Per step, lane j of a group tests
// whether the (j+1)-th pop of this step happens: the pop condition q > q_targ is
// monotone in q, so the group's ballot bits are a prefix whose population count is the
// number of pops (another round while some group pops GW events).  Lane j also holds the
// ring links of event h + j, so the deactivations of the popped events are two more
// ballots.  The sequential streams dpt (read) and qout (written, or compared in merge
// mode) move in blocks of GW steps.  Groups whose chunk is finished stay in the warp's
// collective operations with no effect.
// kMerge = false: write every step's queue length to qout.
// kMerge = true : compare with qout; a group stops at the first equal step (merged),
//                 having overwritten the differing entries before it.
template <int GW, bool kMerge>
__device__ __forceinline__ bool group_run(const KParams &kp, unsigned long long base,
                                          const uint4 *__restrict__ ring,
                                          unsigned *qout, unsigned k0, unsigned k1, DetState &st,
                                          unsigned *err, unsigned *nsteps = nullptr, unsigned kw = 0)
{
    static_assert(GW == 8 || GW == 16 || GW == 32, "group width");
    const unsigned lane = threadIdx.x & 31;
    const unsigned gl = lane % GW;               // lane within the group
    const unsigned gshift = lane - gl;           // first lane of the group
    const unsigned gbits = GW == 32 ? 0xFFFFFFFFu : ((1u << GW) - 1u);
    const unsigned ring_mask32 = (unsigned)kp.ring_mask;
    const unsigned base32 = (unsigned)base;
    int h = (int)st.h;
    unsigned nap = st.nap, nat = st.nat;
    unsigned long long X = st.X;
    unsigned Y = (unsigned)st.Y;
    bool merged = false, bad = false;
    unsigned done = k1 > k0 ? k1 - k0 : 0u;
    // the warp iterates over the longest chunk of its groups
    unsigned span = k1 > k0 ? k1 - k0 : 0u;
    for (int o = 16; o >= GW; o >>= 1) span = max(span, __shfl_xor_sync(0xFFFFFFFFu, span, o));
    bool active = k0 < k1;
    // register window of the ring's next-links ahead of the queue front: lane gl holds
    // the links of events hb + gl (wa) and hb + GW + gl (wb); h - hb stays in [0, GW)
    int hb = h;
    uint2 wa = nxt_of(ring, (base32 + (unsigned)(hb + (int)gl)) & ring_mask32);
    uint2 wb = nxt_of(ring, (base32 + (unsigned)(hb + GW + (int)gl)) & ring_mask32);
    // push stream, double buffered by blocks of GW steps
    uint2 dnext = active && k0 + gl < k1 ? prv_of(ring, (base32 + k0 + gl) & ring_mask32) : make_uint2(0u, 0u);
    unsigned qnext = 0;
    if (kMerge) qnext = active && k0 + gl < k1 ? qout[k0 + gl] : 0u;
    for (unsigned off = 0; off < span; off += GW) {
        if (!__any_sync(0xFFFFFFFFu, active)) break;  // every group of the warp is done
        const unsigned kb = k0 + off;
        const uint2 dblk = dnext;
        const unsigned qold = qnext;
        {
            const unsigned kn = kb + GW + gl;
            const bool nb = active && kn < k1;
            dnext = nb ? prv_of(ring, (base32 + kn) & ring_mask32) : make_uint2(0u, 0u);
            if (kMerge) qnext = nb ? qout[kn] : 0u;
        }
        unsigned qmine = 0, nwrite = 0;
        for (unsigned i = 0; i < GW; ++i) {
            const unsigned k = kb + i;
            const bool act = active && k < k1;
            const unsigned dx = __shfl_sync(0xFFFFFFFFu, dblk.x, i, GW);
            const unsigned dy = __shfl_sync(0xFFFFFFFFu, dblk.y, i, GW);
            const int dist = (int)k - h;
            if (act && dist < 0) {  // impossible for a consistent state; never loop on a bad one
                if (gl == 0) atomicOr(err, ERR_BAD_STATE);
                bad = true;
            }
            const bool go = act && !bad;
            if (go) {
                nap += dx > (unsigned)dist;
                nat += dy > (unsigned)dist;
            }
            unsigned q = go ? (unsigned)dist + 1u : 0u;
            bool popping = go;
            for (;;) {
                // links of event h + gl from the window
                const unsigned src = (unsigned)(h - hb) + gl;
                const unsigned ax = __shfl_sync(0xFFFFFFFFu, wa.x, src & (GW - 1), GW);
                const unsigned ay = __shfl_sync(0xFFFFFFFFu, wa.y, src & (GW - 1), GW);
                const unsigned bx = __shfl_sync(0xFFFFFFFFu, wb.x, src & (GW - 1), GW);
                const unsigned by = __shfl_sync(0xFFFFFFFFu, wb.y, src & (GW - 1), GW);
                const unsigned rx = src < GW ? ax : bx, ry = src < GW ? ay : by;
                const unsigned v = q - gl;  // queue length before pop number gl+1
                const bool pop = popping && gl < q && v > kp.q_min &&
                                 (v > kp.q_max || (unsigned long long)v * Y > X);
                const unsigned c = __popc((__ballot_sync(0xFFFFFFFFu, pop) >> gshift) & gbits);
                const int dj = (int)k - (h + (int)gl);
                const bool offP = gl < c && rx > (unsigned)dj;
                const bool offT = gl < c && ry > (unsigned)dj;
                nap -= __popc((__ballot_sync(0xFFFFFFFFu, offP) >> gshift) & gbits);
                nat -= __popc((__ballot_sync(0xFFFFFFFFu, offT) >> gshift) & gbits);
                h += (int)c;
                q -= c;
                // keep h - hb in [0, GW): slide the window (the new upper half is loaded
                // about GW pops before it is needed)
                while (h - hb >= GW) {
                    hb += GW;
                    wa = wb;
                    wb = nxt_of(ring, (base32 + (unsigned)(hb + GW + (int)gl)) & ring_mask32);
                }
                const bool more = c == (unsigned)GW;
                if (!__any_sync(0xFFFFFFFFu, more)) break;
                if (!more) popping = false;  // this group is done: no candidates in further rounds
            }
            const unsigned qo = kMerge ? __shfl_sync(0xFFFFFFFFu, qold, i, GW) : 0u;
            if (go) {
                X = (unsigned long long)q * kp.numA * nat;
                Y = kp.den * nap;
                if (gl == i) qmine = q;
                nwrite = i + 1;
                if (kMerge && qo == q) {
                    merged = true;
                    done = k + 1 - k0;
                    nwrite = i;  // the equal entry is already right
                    active = false;
                }
            }
            if (bad) active = false;
        }
        if (gl < nwrite && kb + gl >= kw) qout[kb + gl] = qmine;
    }
    if (nsteps) *nsteps = done;
    st.h = h; st.nap = nap; st.nat = nat; st.X = X; st.Y = Y;
    return merged;
}

constexpr int DET_GW = 8;  // lanes per chunk in the parallel passes

// Pass 1, groups of DET_GW lanes per chunk.  Chunk c >= 1 warms up over the previous
// chunk: it starts from the speculative state of chunk c-1's first event (E0[c-1]) and
// records the queue lengths of its own chunk only, so its trajectory has had a whole
// chunk to merge with the true one by the time its own chunk starts.
__global__ void __launch_bounds__(128)
k_det_pass1(KParams kp, Ctrl *ctrl, const uint4 *ring, unsigned *qout,
            const DetState *E0, DetState *E1)
{
    PDL_ENTRY();
    const unsigned long long base = ctrl->base;
    const unsigned m = ctrl->m, S = ctrl->S, nch = ctrl->nchunks;
    const unsigned lane = threadIdx.x & 31;
    constexpr unsigned CPW = 32 / DET_GW;  // chunks per warp
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned wb = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * CPW; wb < nch; wb += warps * CPW) {
        const unsigned c = wb + lane / DET_GW;
        DetState st{0, 0, 0, 0, 1};
        unsigned k0 = 0, k1 = 0, kw = 0;
        if (c < nch) {
            kw = c * S;
            k1 = min(m, (c + 1) * S);
            if (c <= 1) {  // from the true state at the batch start
                st = ctrl->det;
                st.h = (long long)((unsigned long long)st.h - base);
                k0 = 0;
            } else {
                st = E0[c - 1];
                k0 = (c - 1) * S + 1;  // chunk c-1's first event was applied by k_det_init
            }
        }
        group_run<DET_GW, false>(kp, base, ring, qout, k0, k1, st, &ctrl->error, nullptr, kw);
        if (c < nch && lane % DET_GW == 0) E1[c] = st;
    }
}

__global__ void __launch_bounds__(128)
k_det_pass2(KParams kp, Ctrl *ctrl, const uint4 *ring, unsigned *qout,
            const DetState *E1, DetState *E2, unsigned char *merged, unsigned *unm_bits)
{
    PDL_ENTRY();
    const unsigned long long base = ctrl->base;
    const unsigned m = ctrl->m, S = ctrl->S, nch = ctrl->nchunks;
    const unsigned lane = threadIdx.x & 31;
    constexpr unsigned CPW = 32 / DET_GW;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned wb = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * CPW; wb < nch; wb += warps * CPW) {
        const unsigned c = wb + lane / DET_GW;
        const bool real = c >= 1 && c < nch;
        DetState st{0, 0, 0, 0, 1};
        unsigned k0 = 0, k1 = 0;
        if (real) {
            st = E1[c - 1];
            k0 = c * S;
            k1 = min(m, (c + 1) * S);
        }
        unsigned steps = 0;
        const bool mg = group_run<DET_GW, true>(kp, base, ring, qout, k0, k1, st, &ctrl->error, &steps);
        if (real && lane % DET_GW == 0) {
            merged[c] = mg;
            atomicAdd(&ctrl->pass2_steps, (unsigned long long)steps);
            if (!mg) {
                E2[c] = st;
                atomicAdd(&ctrl->unmerged, 1u);
                atomicAdd(&ctrl->unmerged_total, 1ull);
                atomicOr(&unm_bits[c >> 5], 1u << (c & 31));
            }
        }
    }
}

__device__ __forceinline__ bool same_state(const DetState &a, const DetState &b)
{
    return a.h == b.h && a.nap == b.nap && a.nat == b.nat && a.X == b.X && a.Y == b.Y;
}

// Serial fixup, one warp.  Pass 2 ran chunk c from E1[c-1]; that run is exact when
// E1[c-1] is the exact exit of chunk c-1.  Chunks that merged in pass 2 end on E1[c], so
// exactness can only break right after a chunk that did not merge (its exact exit is
// E2[c]).  The warp jumps from one unmerged chunk to the next with a bitmap, and re-runs
// chunks only while the entry they were run from differs from the exact one.  The
// bitmap is cleared on the way.
__global__ void k_det_fix(KParams kp, Ctrl *ctrl, const uint4 *ring, unsigned *qout,
                          const DetState *E1, const DetState *E2, const unsigned char *merged,
                          unsigned *unm_bits)
{
    PDL_ENTRY();
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const unsigned lane = threadIdx.x;
    const unsigned long long base = ctrl->base;
    const unsigned m = ctrl->m, S = ctrl->S, nch = ctrl->nchunks;
    if (m == 0) {
        if (lane == 0) ctrl->h_prev = ctrl->det.h;
        return;
    }
    DetState fin;
    if (ctrl->unmerged == 0) {
        fin = E1[nch - 1];
    } else {
        if (lane == 0) ctrl->fixups += 1;
        const unsigned nwords = (nch + 31) / 32;
        unsigned c = 1;  // chunks < c are exact and chunk c's pass-2 entry E1[c-1] is exact
        DetState exit_c;
        bool have_exit = false;  // exit of chunk c-1 if it differs from E1[c-1]
        while (c < nch) {
            if (!have_exit) {
                // next unmerged chunk >= c
                unsigned w = c >> 5, found = nch;
                for (unsigned wb = w; wb < nwords && found == nch; wb += 32) {
                    const unsigned wi = wb + lane;
                    unsigned bits = wi < nwords ? unm_bits[wi] : 0u;
                    if (wi == w) bits &= ~0u << (c & 31);
                    const unsigned any = __ballot_sync(0xFFFFFFFFu, bits != 0u);
                    if (any) {
                        const unsigned src = __ffs(any) - 1;
                        const unsigned b = __shfl_sync(0xFFFFFFFFu, bits, src);
                        found = (wb + src) * 32 + __ffs(b) - 1;
                    }
                }
                if (found >= nch) { c = nch; break; }
                // chunk `found` has an exact entry and did not merge: its exact exit is E2
                exit_c = E2[found];
                c = found + 1;
                have_exit = true;
                continue;
            }
            // chunk c was run from E1[c-1]; the exact entry is exit_c
            if (same_state(E1[c - 1], exit_c)) { have_exit = false; continue; }
            DetState st = exit_c;
            unsigned steps = 0;
            const bool mg = group_run<32, true>(kp, base, ring, qout, c * S, min(m, (c + 1) * S), st,
                                           &ctrl->error, &steps);
            if (lane == 0) ctrl->fix_steps += steps;
            exit_c = mg ? (merged[c] ? E1[c] : E2[c]) : st;
            ++c;
            have_exit = true;
        }
        fin = have_exit ? exit_c : E1[nch - 1];
        for (unsigned wi = lane; wi < nwords; wi += 32) unm_bits[wi] = 0u;
    }
    __syncwarp();
    if (lane == 0) {
        fin.h = (long long)(base + (unsigned long long)fin.h);
        ctrl->h_prev = ctrl->det.h;
        ctrl->det = fin;
    }
}

cudaError_t launch_det_counts(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 2;
    static bool attr_set = false;
    const size_t smem = sizeof(HistSmem);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_det_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (cudaError_t e_ = launch_pdl(k_det_hist, grid_for(2), 256, smem, s, kp, b.ctrl, b.ring4, b.dMt, b.mt_stride))
        return e_;
    if (cudaError_t e_ = launch_pdl(k_det_init, grid_for(2), 256, 0, s, kp, b.ctrl, b.ring4, b.dMt, b.mt_stride,
                                    b.qout, b.E0))
        return e_;
    return cudaGetLastError();
}

cudaError_t launch_det_pass1(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    if (cudaError_t e_ = launch_pdl(k_det_pass1, grid_for(8), 128, 0, s, kp, b.ctrl, b.ring4, b.qout, b.E0, b.E1)) return e_;
    return cudaGetLastError();
}

cudaError_t launch_det_pass2(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    if (cudaError_t e_ = launch_pdl(k_det_pass2, grid_for(8), 128, 0, s, kp, b.ctrl, b.ring4, b.qout, b.E1, b.E2, b.merged,
                                           b.unm_bits)) return e_;
    return cudaGetLastError();
}

cudaError_t launch_det_fix(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    if (cudaError_t e_ = launch_pdl(k_det_fix, 1, 32, 0, s, kp, b.ctrl, b.ring4, b.qout, b.E1, b.E2, b.merged, b.unm_bits)) return e_;
    return cudaGetLastError();
}

}  // namespace fibar
