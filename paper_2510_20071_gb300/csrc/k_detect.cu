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
//         shortest chunk-aligned window that the regulator would shrink, plus one chunk
//         (k_det_hist, k_det_init); its exact distinct counts come from per-chunk suffix
//         histograms.  A too-long window pops down to its target in the first steps and
//         then coincides with the true trajectory.
// Pass 2: chunk c restarts from pass 1's exit state of chunk c-1 and runs until its
//         queue length equals pass 1's at the same step (the trajectories merged).
// Fixup:  if some chunk did not merge, one thread walks the chunks in order and re-runs
//         exactly those whose entry state was wrong.  The result is exact in all cases.
#include "fibar_internal.cuh"

namespace fibar {

struct Geo {
    unsigned long long base;
    unsigned m, S, nchunks, G, Gold;
};

// Chunk length S and the reach G (in chunks) of the guessed windows: G * S covers
// about twice the queue length at the batch start, with at most DET_G chunks.
__device__ __forceinline__ Geo geometry(const KParams &kp, const Ctrl *ctrl)
{
    Geo g;
    g.base = ctrl->base;
    g.m = ctrl->m;
    const unsigned long long qprev = g.base - (unsigned long long)ctrl->det.h;
    const unsigned long long want = 2ull * qprev + 4ull * CHUNK;
    unsigned long long S = (want + DET_G - 1) / DET_G;
    S = (S + 31) / 32 * 32;
    g.S = (unsigned)max((unsigned long long)CHUNK, S);
    g.nchunks = (g.m + g.S - 1) / g.S;
    g.G = DET_G;
    const unsigned long long old_chunks = (g.base + g.S - 1) / g.S;
    g.Gold = (unsigned)min((unsigned long long)g.G, old_chunks);
    return g;
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

// Suffix histograms: for chunk c' (old chunks -Gold..-1 and the batch's chunks),
//   M[c'][g] = #{j in c' : next(j) >= (c'+g) S}     (g = 1..G, pixels and tiles)
// i.e. the events of c' that are still the last of their pixel / tile at the start of
// chunk c'+g.  The distinct counts of any chunk-aligned window [(c-g)S, cS) are then
// N(c, g) = sum_{g'=1..g} M[c-g'][g'].
__global__ void __launch_bounds__(256)
k_det_hist(KParams kp, Ctrl *ctrl, const uint2 *ring, unsigned short *M)
{
    PDL_ENTRY();
    __shared__ unsigned hist[8][2][DET_G + 1];
    const Geo g = geometry(kp, ctrl);
    const unsigned lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const unsigned nwork = g.nchunks + g.Gold;
    const unsigned warps_total = gridDim.x * (blockDim.x >> 5);
    const long long lo_exist = -(long long)g.base;
    unsigned *hP = hist[wl][0], *hT = hist[wl][1];
    for (unsigned wi = blockIdx.x * (blockDim.x >> 5) + wl; wi < nwork; wi += warps_total) {
        const long long c = (long long)wi - (long long)g.Gold;
        for (unsigned i = lane; i <= DET_G; i += 32) { hP[i] = 0; hT[i] = 0; }
        __syncwarp();
        const long long lo = c * g.S;
        for (unsigned r = lane; r < g.S; r += 32) {
            const long long j = lo + r;
            if (j < lo_exist || j >= (long long)g.m) continue;
            const uint2 n = ring[(g.base + (unsigned long long)j) & kp.ring_mask];
            const long long dp = n.x == SAT ? DET_G : min((long long)DET_G, chunk_of(j + n.x, g.S, g.Gold) - c);
            const long long dt = n.y == SAT ? DET_G : min((long long)DET_G, chunk_of(j + n.y, g.S, g.Gold) - c);
            atomicAdd(&hP[dp], 1u);
            atomicAdd(&hT[dt], 1u);
        }
        __syncwarp();
        // suffix sums over d: lane owns d in [lane*8, lane*8+8)
        unsigned sp = 0, st = 0, vp[8], vt[8];
#pragma unroll
        for (int i = 7; i >= 0; --i) {
            const unsigned d = lane * 8 + i;
            sp += d <= DET_G ? hP[d] : 0u;
            st += d <= DET_G ? hT[d] : 0u;
            vp[i] = sp;
            vt[i] = st;
        }
        // add the totals of the lanes above (exclusive suffix over lanes)
        unsigned xp = sp, xt = st;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned yp = __shfl_down_sync(0xFFFFFFFFu, xp, o);
            const unsigned yt = __shfl_down_sync(0xFFFFFFFFu, xt, o);
            if (lane + o < 32) { xp += yp; xt += yt; }
        }
        const unsigned above_p = xp - sp, above_t = xt - st;
        unsigned short *row = M + (size_t)(c + g.Gold) * 2 * (DET_G + 1);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const unsigned d = lane * 8 + i;
            if (d <= DET_G) {
                row[d] = (unsigned short)(vp[i] + above_p);
                row[DET_G + 1 + d] = (unsigned short)(vt[i] + above_t);
            }
        }
        __syncwarp();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->S = g.S;
        ctrl->nchunks = g.nchunks;
        ctrl->G = g.G;
        ctrl->Gold = g.Gold;
    }
}

// Speculative start of chunk c (c >= 1), one warp per chunk.  Among the windows of
// g = 1..G whole chunks ending just before the chunk, take the shortest one that the
// regulator would shrink at the next event (its length is at or past the equilibrium
// of Eq. 20), plus one chunk: a slight overestimate of the true queue, which merges
// with the true trajectory within a few tens of events.  The warp then applies the
// chunk's first event exactly, popping the excess in parallel.
__global__ void __launch_bounds__(256)
k_det_init(KParams kp, const Ctrl *ctrl, const uint2 *dpt, const uint2 *ring,
           const unsigned short *M, unsigned *qout, DetState *E0)
{
    PDL_ENTRY();
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long base = ctrl->base;
    const unsigned m = ctrl->m, S = ctrl->S, nch = ctrl->nchunks, Gold = ctrl->Gold;
    const unsigned warps_total = gridDim.x * (blockDim.x >> 5);
    for (unsigned c = 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nch; c += warps_total) {
        // M[c-g][g] for g = lane*8+1 .. lane*8+8
        unsigned np8[8], nt8[8], sp = 0, st = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const unsigned gg = lane * 8 + i + 1;
            unsigned vp = 0, vt = 0;
            if (gg <= DET_G && (long long)c - gg >= -(long long)Gold) {
                const unsigned short *row = M + (size_t)((long long)c - gg + Gold) * 2 * (DET_G + 1);
                vp = row[gg];
                vt = row[DET_G + 1 + gg];
            }
            sp += vp;
            st += vt;
            np8[i] = sp;
            nt8[i] = st;
        }
        unsigned xp = sp, xt = st;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned yp = __shfl_up_sync(0xFFFFFFFFu, xp, o);
            const unsigned yt = __shfl_up_sync(0xFFFFFFFFu, xt, o);
            if (lane >= o) { xp += yp; xt += yt; }
        }
        const unsigned below_p = xp - sp, below_t = xt - st;
        const unsigned long long reach = (unsigned long long)c * S + base;  // events before the chunk
        int first = 0;
#pragma unroll
        for (int i = 0; i < 8 && !first; ++i) {
            const unsigned gg = lane * 8 + i + 1;
            if (gg > DET_G) break;
            const unsigned long long L = min((unsigned long long)gg * S, reach);
            const unsigned long long nap = np8[i] + below_p, nat = nt8[i] + below_t;
            const unsigned long long X = L * kp.numA * nat, Y = (unsigned long long)kp.den * nap;
            const unsigned long long q = L + 1;
            if (nap > 0 && q > kp.q_min && (q > kp.q_max || q * Y > X)) first = (int)gg;
        }
        const unsigned any = __ballot_sync(0xFFFFFFFFu, first != 0);
        unsigned gsel = DET_G;
        if (any) gsel = min((unsigned)DET_G, (unsigned)__shfl_sync(0xFFFFFFFFu, first, __ffs(any) - 1) + 1u);
        // counts of the chosen window: lane holding gsel broadcasts
        const unsigned src = (gsel - 1) / 8, idx = (gsel - 1) % 8;
        unsigned mynp = 0, mynt = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i == (int)idx) { mynp = np8[i] + below_p; mynt = nt8[i] + below_t; }
        unsigned nap = __shfl_sync(0xFFFFFFFFu, mynp, src);
        unsigned nat = __shfl_sync(0xFFFFFFFFu, mynt, src);
        const long long k0 = (long long)c * S;
        const long long hs = max(k0 - (long long)gsel * S, -(long long)base);
        unsigned long long L = (unsigned long long)(k0 - hs);
        unsigned long long X = L * kp.numA * nat, Y = (unsigned long long)kp.den * nap;
        if (nap == 0) { X = kp.q_min; Y = 1; }
        // step k0: push, then pop down to q_targ = clamp(floor(X / Y))
        const uint2 d = dpt[k0];
        nap += (long long)d.x > (long long)L;
        nat += (long long)d.y > (long long)L;
        const unsigned long long q = L + 1;
        unsigned long long qt = X / Y;
        qt = min(qt, (unsigned long long)kp.q_max);
        qt = max(qt, (unsigned long long)kp.q_min);
        const unsigned long long npop = q > qt ? q - qt : 0ull;
        unsigned dp = 0, dtt = 0;
        for (unsigned long long i = lane; i < npop; i += 32) {
            const long long j = hs + (long long)i;
            const uint2 n = ring[(base + (unsigned long long)j) & kp.ring_mask];
            dp += (long long)n.x > k0 - j;
            dtt += (long long)n.y > k0 - j;
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

// Run the detector over steps [k0, k1) from state st (h batch-relative) with one warp.
// All lanes hold the same state.  Per step, lane j tests whether the (j+1)-th pop of
// this step happens: the pop condition q > q_targ is monotone in q, so the ballot of
// lanes 0..31 is a prefix whose population count is the number of pops (another round
// if all 32 pop).  Lane j also holds the ring links of event h + j, so the deactivations
// of the popped events are two more ballots.  The sequential streams dpt (read) and
// qout (written, or compared in merge mode) move in coalesced blocks of 32 steps.
// kMerge = false: write every step's queue length to qout.
// kMerge = true : compare with qout; stop (return true) at the first equal step,
//                 overwriting the differing entries before it.
template <bool kMerge>
__device__ __forceinline__ bool warp_run(const KParams &kp, unsigned long long base,
                                         const uint2 *__restrict__ dpt, const uint2 *__restrict__ ring,
                                         unsigned *qout, unsigned k0, unsigned k1, DetState &st,
                                         unsigned *err, unsigned *nsteps = nullptr)
{
    const unsigned lane = threadIdx.x & 31;
    long long h = st.h;
    unsigned nap = st.nap, nat = st.nat;
    unsigned long long X = st.X;
    unsigned long long Y = st.Y;
    bool merged = false;
    unsigned done = k1 - k0;
    for (unsigned kb = k0; kb < k1; kb += 32) {
        const unsigned nb = min(32u, k1 - kb);
        const uint2 dblk = lane < nb ? dpt[kb + lane] : make_uint2(0u, 0u);
        unsigned qold = 0;
        if (kMerge) qold = lane < nb ? qout[kb + lane] : 0u;
        unsigned qmine = 0;
        unsigned i = 0;
        bool bad = false;
        for (; i < nb; ++i) {
            const unsigned k = kb + i;
            uint2 rn = ring[(base + (unsigned long long)(h + lane)) & kp.ring_mask];
            const unsigned dx = __shfl_sync(0xFFFFFFFFu, dblk.x, i);
            const unsigned dy = __shfl_sync(0xFFFFFFFFu, dblk.y, i);
            const long long dist = (long long)k - h;
            if (dist < 0) {  // impossible for a consistent state; never loop on a bad one
                if (lane == 0) atomicOr(err, ERR_BAD_STATE);
                bad = true;
                break;
            }
            nap += (long long)dx > dist;
            nat += (long long)dy > dist;
            unsigned long long q = (unsigned long long)dist + 1;
            for (;;) {
                const unsigned long long v = q - lane;  // queue length before pop number lane+1
                const bool pop = lane < q && v > kp.q_min && (v > kp.q_max || v * Y > X);
                const unsigned c = __popc(__ballot_sync(0xFFFFFFFFu, pop));
                const long long dj = (long long)k - (h + lane);
                const bool offP = lane < c && (long long)rn.x > dj;
                const bool offT = lane < c && (long long)rn.y > dj;
                nap -= __popc(__ballot_sync(0xFFFFFFFFu, offP));
                nat -= __popc(__ballot_sync(0xFFFFFFFFu, offT));
                h += c;
                q -= c;
                if (c < 32) break;
                rn = ring[(base + (unsigned long long)(h + lane)) & kp.ring_mask];
            }
            X = q * kp.numA * nat;
            Y = (unsigned long long)kp.den * nap;
            if (lane == i) qmine = (unsigned)q;
            if (kMerge) {
                const unsigned qo = __shfl_sync(0xFFFFFFFFu, qold, i);
                if (qo == (unsigned)q) {
                    merged = true;
                    done = k + 1 - k0;
                    break;
                }
            }
        }
        // this block's queue lengths (in merge mode the equal one at i is not rewritten)
        if (lane < i) qout[kb + lane] = qmine;
        if (merged || bad) break;
    }
    if (nsteps) *nsteps = done;
    st.h = h; st.nap = nap; st.nat = nat; st.X = X; st.Y = Y;
    return merged;
}

__global__ void __launch_bounds__(128)
k_det_pass1(KParams kp, Ctrl *ctrl, const uint2 *dpt, const uint2 *ring, unsigned *qout,
            const DetState *E0, DetState *E1)
{
    PDL_ENTRY();
    const unsigned long long base = ctrl->base;
    const unsigned m = ctrl->m, S = ctrl->S, nch = ctrl->nchunks;
    const unsigned lane = threadIdx.x & 31;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nch; c += warps) {
        DetState st;
        unsigned k0 = c * S;
        if (c == 0) {
            st = ctrl->det;
            st.h = (long long)((unsigned long long)st.h - base);
        } else {
            st = E0[c];
            k0 += 1;  // the chunk's first event was applied by k_det_init
        }
        warp_run<false>(kp, base, dpt, ring, qout, k0, min(m, (c + 1) * S), st, &ctrl->error);
        if (lane == 0) E1[c] = st;
    }
}

__global__ void __launch_bounds__(128)
k_det_pass2(KParams kp, Ctrl *ctrl, const uint2 *dpt, const uint2 *ring, unsigned *qout,
            const DetState *E1, DetState *E2, unsigned char *merged, unsigned *unm_bits)
{
    PDL_ENTRY();
    const unsigned long long base = ctrl->base;
    const unsigned m = ctrl->m, S = ctrl->S, nch = ctrl->nchunks;
    const unsigned lane = threadIdx.x & 31;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned c = 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nch; c += warps) {
        DetState st = E1[c - 1];
        unsigned steps = 0;
        const bool mg = warp_run<true>(kp, base, dpt, ring, qout, c * S, min(m, (c + 1) * S), st,
                                       &ctrl->error, &steps);
        if (lane == 0) {
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
__global__ void k_det_fix(KParams kp, Ctrl *ctrl, const uint2 *dpt, const uint2 *ring, unsigned *qout,
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
            const bool mg = warp_run<true>(kp, base, dpt, ring, qout, c * S, min(m, (c + 1) * S), st,
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
    if (cudaError_t e_ = launch_pdl(k_det_hist, grid_for(4), 256, 0, s, kp, b.ctrl, b.ring_npt, b.dM)) return e_;
    if (cudaError_t e_ = launch_pdl(k_det_init, grid_for(4), 256, 0, s, kp, b.ctrl, b.dpt, b.ring_npt, b.dM, b.qout, b.E0)) return e_;
    return cudaGetLastError();
}

cudaError_t launch_det_pass1(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    if (cudaError_t e_ = launch_pdl(k_det_pass1, grid_for(8), 128, 0, s, kp, b.ctrl, b.dpt, b.ring_npt, b.qout, b.E0, b.E1)) return e_;
    return cudaGetLastError();
}

cudaError_t launch_det_pass2(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    if (cudaError_t e_ = launch_pdl(k_det_pass2, grid_for(8), 128, 0, s, kp, b.ctrl, b.dpt, b.ring_npt, b.qout, b.E1, b.E2, b.merged,
                                           b.unm_bits)) return e_;
    return cudaGetLastError();
}

cudaError_t launch_det_fix(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    if (cudaError_t e_ = launch_pdl(k_det_fix, 1, 32, 0, s, kp, b.ctrl, b.dpt, b.ring_npt, b.qout, b.E1, b.E2, b.merged, b.unm_bits)) return e_;
    return cudaGetLastError();
}

}  // namespace fibar
