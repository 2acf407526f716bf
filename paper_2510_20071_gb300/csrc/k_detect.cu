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
//         shortest of 8 candidate window lengths (ratio sqrt 2) that the regulator would
//         shrink (k_det_counts, k_det_init); the exact distinct counts of the candidate
//         windows of every chunk come from sliding-window recurrences over per-chunk
//         counts.  A too-long window pops down to its target in the first steps and then
//         coincides with the true trajectory.
// Pass 2: chunk c restarts from pass 1's exit state of chunk c-1 and runs until its
//         queue length equals pass 1's at the same step (the trajectories merged).
// Fixup:  if some chunk did not merge, one thread walks the chunks in order and re-runs
//         exactly those whose entry state was wrong.  The result is exact in all cases.
#include "fibar_internal.cuh"

namespace fibar {

struct Geo {
    unsigned long long base;
    unsigned m, S, nchunks, Gold;
    unsigned gtop;              // reach of the longest candidate window, in chunks
};

// Chunk length S (the batch is cut into at most DET_MAX_CHUNKS chunks of at least CHUNK
// events) and the candidate window lengths: NCAND lengths in chunks, ratio sqrt(2),
// the longest about 2.5x the queue length at the batch start (for a young stream, whose
// queue is still growing, the whole sensor).
__device__ __forceinline__ Geo geometry(const KParams &kp, const Ctrl *ctrl)
{
    Geo g;
    g.base = ctrl->base;
    g.m = ctrl->m;
    unsigned long long S = ((unsigned long long)g.m + DET_MAX_CHUNKS - 1) / DET_MAX_CHUNKS;
    S = (S + 15) / 16 * 16;
    g.S = (unsigned)max((unsigned long long)CHUNK, S);
    g.nchunks = (g.m + g.S - 1) / g.S;
    const unsigned long long qprev = g.base - (unsigned long long)ctrl->det.h;
    unsigned long long reach;
    if (g.base < kp.q_max) reach = kp.q_max;
    else reach = min((unsigned long long)kp.q_max, (5ull * qprev) / 2 + 4ull * g.S);
    g.gtop = (unsigned)((reach + g.S - 1) / g.S) + 1;
    const unsigned long long old_chunks = (g.base + g.S - 1) / g.S;
    g.Gold = (unsigned)min((unsigned long long)g.gtop, old_chunks);
    return g;
}

// candidate i (0 = longest) in chunks
__device__ __forceinline__ unsigned cand_g(unsigned gtop, int i)
{
    // gtop * 2^(-i/2), at least 1
    const float f = exp2f(-0.5f * (float)i);
    return max(1u, (unsigned)((float)gtop * f + 0.5f));
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

// Exact distinct pixel / tile counts of the candidate windows W_i(c) = [(c-g_i)S, cS)
// (clipped at the stream start) of every chunk c, by sliding-window recurrences:
//   N_i(c+1) = N_i(c) + A(c) - B_i(c) - E_i(c - g_i)
//   A(c)   = #{j in chunk c : next(j) >= (c+1)S}         (last of its pixel at the chunk end)
//   B_i(c) = #{j in chunk c : prev(j) in W_i(c)}          (its predecessor stops being last)
//   E_i(c) = #{j in chunk c : next(j) >= (c+g_i+1)S}      (last events leaving the window)
//   N_i(0) = #{j in W_i(0) : next(j) >= 0}.
// One warp per chunk (old chunks -Gold..-1 and the batch's chunks); the last block scans
// the increments into init[c][i] = {N_ap, N_at}.
__global__ void __launch_bounds__(256)
k_det_counts(KParams kp, Ctrl *ctrl, const uint4 *ring, unsigned *cA, unsigned *cB, unsigned *cE,
             uint2 *init, size_t max_chunks)
{
    PDL_ENTRY();
    const Geo g = geometry(kp, ctrl);
    const unsigned lane = threadIdx.x & 31;
    const unsigned nwork = g.nchunks + g.Gold;
    const unsigned warps_total = gridDim.x * (blockDim.x >> 5);
    const long long lo_exist = -(long long)g.base;
    unsigned gc[NCAND];
#pragma unroll
    for (int i = 0; i < NCAND; ++i) gc[i] = cand_g(g.gtop, i);
    for (unsigned wi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wi < nwork; wi += warps_total) {
        const long long c = (long long)wi - (long long)g.Gold;
        const long long lo = c * g.S;
        unsigned aP = 0, aT = 0;
        unsigned bP[NCAND], bT[NCAND], eP[NCAND], eT[NCAND];
#pragma unroll
        for (int i = 0; i < NCAND; ++i) bP[i] = bT[i] = eP[i] = eT[i] = 0;
        for (unsigned r = lane; r < g.S; r += 32) {
            const long long j = lo + r;
            if (j < lo_exist || j >= (long long)g.m) continue;
            const unsigned long long slot = (g.base + (unsigned long long)j) & kp.ring_mask;
            const uint2 n = nxt_of(ring, slot);
            const long long np = n.x == SAT ? 0x7FFFFFFFFFFFFFFFll : j + (long long)n.x;
            const long long nt = n.y == SAT ? 0x7FFFFFFFFFFFFFFFll : j + (long long)n.y;
            if (c < 0) {
                // only E (old chunks leave the windows), and N_i(0) contributions
#pragma unroll
                for (int i = 0; i < NCAND; ++i) {
                    const long long eth = (c + (long long)gc[i] + 1) * (long long)g.S;
                    eP[i] += np >= eth;
                    eT[i] += nt >= eth;
                    const bool inw = j >= -(long long)gc[i] * g.S;
                    bP[i] += inw && np >= 0;  // reused as N_i(0) partials for old chunks
                    bT[i] += inw && nt >= 0;
                }
            } else {
                const long long ath = (c + 1) * (long long)g.S;
                aP += np >= ath;
                aT += nt >= ath;
                const uint2 d = prv_of(ring, slot);
                const long long pp = d.x == SAT ? -0x7FFFFFFFFFFFFFFFll : j - (long long)d.x;
                const long long pt = d.y == SAT ? -0x7FFFFFFFFFFFFFFFll : j - (long long)d.y;
#pragma unroll
                for (int i = 0; i < NCAND; ++i) {
                    const long long eth = (c + (long long)gc[i] + 1) * (long long)g.S;
                    eP[i] += np >= eth;
                    eT[i] += nt >= eth;
                    const long long wlo = (c - (long long)gc[i]) * (long long)g.S;
                    bP[i] += pp >= wlo && pp < lo;
                    bT[i] += pt >= wlo && pt < lo;
                }
            }
        }
        aP = warp_sum(aP);
        aT = warp_sum(aT);
#pragma unroll
        for (int i = 0; i < NCAND; ++i) {
            bP[i] = warp_sum(bP[i]); bT[i] = warp_sum(bT[i]);
            eP[i] = warp_sum(eP[i]); eT[i] = warp_sum(eT[i]);
        }
        if (lane == 0) {
            const size_t ei = (size_t)(c + g.Gold);
#pragma unroll
            for (int i = 0; i < NCAND; ++i) {
                cE[(ei * NCAND + i) * 2] = eP[i];
                cE[(ei * NCAND + i) * 2 + 1] = eT[i];
            }
            if (c >= 0) {
                cA[c * 2] = aP;
                cA[c * 2 + 1] = aT;
#pragma unroll
                for (int i = 0; i < NCAND; ++i) {
                    cB[((size_t)c * NCAND + i) * 2] = bP[i];
                    cB[((size_t)c * NCAND + i) * 2 + 1] = bT[i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < NCAND; ++i) {
                    if (bP[i]) atomicAdd(&ctrl->N0[i][0], bP[i]);
                    if (bT[i]) atomicAdd(&ctrl->N0[i][1], bT[i]);
                }
            }
        }
    }
    __threadfence();
    __syncthreads();
    __shared__ bool s_last;
    __shared__ int s_tot[2 * NCAND][256];
    if (threadIdx.x == 0) s_last = atomicAdd(&ctrl->cnt_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // 2*NCAND scans over the chunks: each thread owns a contiguous range of chunks
    const unsigned n = g.nchunks;
    const unsigned per = (n + 255) / 256;
    const unsigned c0 = threadIdx.x * per, c1 = min(n, c0 + per);
    const long long eloc = -(long long)g.Gold;
    int tot[2 * NCAND];
#pragma unroll
    for (int q = 0; q < 2 * NCAND; ++q) tot[q] = 0;
    for (unsigned c = c0; c < c1; ++c) {
        const int a0 = (int)__ldcg(&cA[c * 2]), a1 = (int)__ldcg(&cA[c * 2 + 1]);
#pragma unroll
        for (int i = 0; i < NCAND; ++i) {
            const long long ce = (long long)c - gc[i];
            int e0 = 0, e1 = 0;
            if (ce >= eloc) {
                const size_t ei = (size_t)(ce + g.Gold);
                e0 = (int)__ldcg(&cE[(ei * NCAND + i) * 2]);
                e1 = (int)__ldcg(&cE[(ei * NCAND + i) * 2 + 1]);
            }
            tot[2 * i] += a0 - (int)__ldcg(&cB[((size_t)c * NCAND + i) * 2]) - e0;
            tot[2 * i + 1] += a1 - (int)__ldcg(&cB[((size_t)c * NCAND + i) * 2 + 1]) - e1;
        }
    }
#pragma unroll
    for (int q = 0; q < 2 * NCAND; ++q) s_tot[q][threadIdx.x] = tot[q];
    __syncthreads();
    if (threadIdx.x < 2 * NCAND) {  // serial scan over the 256 partial sums of one sequence
        const int q = threadIdx.x;
        int run = (int)atomicAdd(&ctrl->N0[q / 2][q & 1], 0u);
        for (int i = 0; i < 256; ++i) {
            const int v = s_tot[q][i];
            s_tot[q][i] = run;
            run += v;
        }
    }
    __syncthreads();
    int r[2 * NCAND];
#pragma unroll
    for (int q = 0; q < 2 * NCAND; ++q) r[q] = s_tot[q][threadIdx.x];
    for (unsigned c = c0; c < c1; ++c) {
        const int a0 = (int)__ldcg(&cA[c * 2]), a1 = (int)__ldcg(&cA[c * 2 + 1]);
#pragma unroll
        for (int i = 0; i < NCAND; ++i) {
            init[(size_t)c * NCAND + i] = make_uint2((unsigned)r[2 * i], (unsigned)r[2 * i + 1]);
            const long long ce = (long long)c - gc[i];
            int e0 = 0, e1 = 0;
            if (ce >= eloc) {
                const size_t ei = (size_t)(ce + g.Gold);
                e0 = (int)__ldcg(&cE[(ei * NCAND + i) * 2]);
                e1 = (int)__ldcg(&cE[(ei * NCAND + i) * 2 + 1]);
            }
            r[2 * i] += a0 - (int)__ldcg(&cB[((size_t)c * NCAND + i) * 2]) - e0;
            r[2 * i + 1] += a1 - (int)__ldcg(&cB[((size_t)c * NCAND + i) * 2 + 1]) - e1;
        }
    }
    if (threadIdx.x == 0) {
        ctrl->S = g.S;
        ctrl->nchunks = g.nchunks;
        ctrl->G = g.gtop;
        ctrl->Gold = g.Gold;
        ctrl->cnt_done = 0;
    }
}

// Speculative start of chunk c (c >= 1), one warp per chunk: among the candidate
// windows ending just before the chunk, take the shortest one that the regulator would
// shrink at the next event (its length is at or past the equilibrium of Eq. 20; the
// next candidate is sqrt(2) shorter), i.e. a slight overestimate of the true queue, which
// merges with the true trajectory within a few tens of events.  The warp then applies
// the chunk's first event exactly, popping the excess in parallel.
__global__ void __launch_bounds__(256)
k_det_init(KParams kp, const Ctrl *ctrl, const uint4 *ring, const uint2 *init, unsigned *qout,
           DetState *E0)
{
    PDL_ENTRY();
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long base = ctrl->base;
    const unsigned S = ctrl->S, nch = ctrl->nchunks, gtop = ctrl->G;
    const unsigned warps_total = gridDim.x * (blockDim.x >> 5);
    for (unsigned c = 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nch; c += warps_total) {
        const long long k0 = (long long)c * S;
        // lane i < NCAND evaluates candidate i
        bool shrink = false;
        uint2 cnt = make_uint2(0u, 0u);
        if (lane < NCAND) {
            const long long hs = max(k0 - (long long)cand_g(gtop, lane) * S, -(long long)base);
            const unsigned long long L = (unsigned long long)(k0 - hs);
            cnt = init[(size_t)c * NCAND + lane];
            const unsigned long long X = L * kp.numA * cnt.y, Y = (unsigned long long)kp.den * cnt.x;
            const unsigned long long q = L + 1;
            shrink = cnt.x > 0 && q > kp.q_min && (q > kp.q_max || q * Y > X);
        }
        // candidates are longest first: the shortest shrinking one is the highest lane set
        const unsigned sb = __ballot_sync(0xFFFFFFFFu, shrink);
        const int sel = sb ? 31 - __clz(sb) : 0;
        const unsigned nap0 = __shfl_sync(0xFFFFFFFFu, cnt.x, sel);
        const unsigned nat0 = __shfl_sync(0xFFFFFFFFu, cnt.y, sel);
        const long long hs = max(k0 - (long long)cand_g(gtop, sel) * S, -(long long)base);
        const unsigned long long L = (unsigned long long)(k0 - hs);
        unsigned long long X = L * kp.numA * nat0, Y = (unsigned long long)kp.den * nap0;
        if (nap0 == 0) { X = kp.q_min; Y = 1; }
        // step k0: push, then pop down to q_targ = clamp(floor(X / Y))
        const uint2 d = prv_of(ring, (base + (unsigned long long)k0) & kp.ring_mask);
        unsigned nap = nap0 + ((long long)d.x > (long long)L);
        unsigned nat = nat0 + ((long long)d.y > (long long)L);
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
            E0[c] = st0;
            qout[k0] = (unsigned)qa;
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
                                          unsigned *err, unsigned *nsteps = nullptr)
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
        if (gl < nwrite) qout[kb + gl] = qmine;
    }
    if (nsteps) *nsteps = done;
    st.h = h; st.nap = nap; st.nat = nat; st.X = X; st.Y = Y;
    return merged;
}

constexpr int DET_GW = 8;  // lanes per chunk in the parallel passes

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
        unsigned k0 = 0, k1 = 0;
        if (c < nch) {
            k0 = c * S;
            k1 = min(m, (c + 1) * S);
            if (c == 0) {
                st = ctrl->det;
                st.h = (long long)((unsigned long long)st.h - base);
            } else {
                st = E0[c];
                k0 += 1;  // the chunk's first event was applied by k_det_init
            }
        }
        group_run<DET_GW, false>(kp, base, ring, qout, k0, k1, st, &ctrl->error);
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
    if (cudaError_t e_ = launch_pdl(k_det_counts, grid_for(8), 256, 0, s, kp, b.ctrl, b.ring4, b.cA, b.cB, b.cE,
                                    b.cinit, b.max_chunks))
        return e_;
    if (cudaError_t e_ = launch_pdl(k_det_init, grid_for(4), 256, 0, s, kp, b.ctrl, b.ring4, b.cinit, b.qout, b.E0))
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
