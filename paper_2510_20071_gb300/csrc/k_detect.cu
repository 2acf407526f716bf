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
// Guess:  chunk c's window before its first step is guessed as the shortest window that
//         the regulator would shrink (k_det_hist, k_det_init): first to the chunk, from
//         per-chunk suffix histograms of the distance to each event's next occurrence,
//         then to the event inside the chunk where it starts.  k_det_init applies step cS
//         to it; the trajectory then coincides with the true one within a few tens of
//         steps (most often fewer than 16).
// Pass 1: each chunk runs from its guess.
// Pass 2: chunk c restarts from pass 1's exit state of chunk c-1 and runs until its
//         queue length equals pass 1's at the same step (the trajectories merged):
//         one chunk per lane for the first steps, then one chunk per warp for the few
//         that take longer.
// Fixup:  if some chunk did not merge, one warp walks the chunks in order and re-runs
//         exactly those whose entry state was wrong.  The result is exact in all cases.
// One chunk per lane is lane_run, one chunk per warp is group_run.
#include "fibar_internal.cuh"

namespace fibar {

// The window table holds, per target chunk c, a band of DET_BAND distances
// [g_lo(c), g_lo(c) + DET_BAND) centred on the chunk's expected window; distances below
// g_lo(c) enter only through their sum N(c, g_lo(c) - 1).  First build: the expected
// queue length starts at the batch's q and, if the queue grew (or shrank) by more than an
// eighth over the previous batch, drifts at that rate.  The same pass stores the whole
// column of distances 1..639 of every DET_SAMPLE-th chunk (about 16 columns in a short
// batch), from which k_det_center finds the regulator's window there;
// if a sampled window falls outside its band (a queue that fills after a stream starts,
// or jumps with the scene), the table is built a second time with bands centred on the
// sampled windows, interpolated between samples.  A window that still leaves its band
// only makes that chunk's guess wrong, which pass 2 and the fixup correct.  While the
// queue is short S is raised so that the band reaches npix / 16 events (npix / 3 in a
// stream's first batch, which starts from an empty queue).
constexpr unsigned DET_BAND = 256;
constexpr int HB_BINS = 640;  // histogram bins: chunk distances 0..639
constexpr unsigned GROW_MIN_EVENTS = 2048;  // shorter batches give no growth estimate
constexpr unsigned BAND_MARGIN = 16;        // sampled windows this close to a band's edge rebuild

struct Geo {
    unsigned long long base;
    unsigned m, S, nchunks, Gold;
    unsigned mid0;      // first build: band centre at chunk 0 (chunks) ...
    int slope;          //   ... drifting per chunk, 16.16 fixed point
    unsigned g_lo_min, g_hi_max;  // union of the first build's bands
};

__device__ __forceinline__ unsigned band_clamp(long long mid)
{
    return (unsigned)max(1ll, min((long long)(HB_BINS - DET_BAND), mid - (long long)(DET_BAND / 2)));
}

// First distance of chunk c's band in the first build.
__device__ __forceinline__ unsigned band_lo_lin(unsigned mid0, int slope, long long c)
{
    return band_clamp((long long)mid0 + ((long long)slope * c) / 65536);
}

// Chunks between sampled windows: DET_SAMPLE, or fewer in a short batch so that it still
// has about 16 samples.
__device__ __forceinline__ unsigned sample_step(unsigned nchunks)
{
    return nchunks >= 16 * DET_SAMPLE ? DET_SAMPLE : max(1u, nchunks / 16);
}
__device__ __forceinline__ unsigned n_samples_of(unsigned nchunks)
{
    return nchunks > 0 ? (nchunks - 1) / sample_step(nchunks) : 0u;
}

// First distance of chunk c's band in the second build: the sampled windows at chunks
// step * s (s = 1..ns), linear in between, constant beyond the ends.
__device__ __forceinline__ unsigned band_lo_tab(const unsigned short *ctr, unsigned ns, unsigned step, long long c)
{
    const long long s0 = c / step;
    if (s0 < 1) return band_clamp(ctr[1]);
    if (s0 >= (long long)ns) return band_clamp(ctr[ns]);
    const long long a = ctr[s0], b = ctr[s0 + 1], r = c - s0 * step;
    return band_clamp(a + (b - a) * r / (long long)step);
}

// Chunk length S: at least CHUNK, at most DET_MAX_CHUNKS chunks per batch, and DET_G
// chunks must cover twice the longest queue expected in the batch.
__device__ __forceinline__ Geo geometry(const KParams &kp, const Ctrl *ctrl)
{
    Geo g;
    g.base = ctrl->base;
    g.m = ctrl->m;
    const unsigned long long qprev = g.base - (unsigned long long)ctrl->det.h;
    // growth per event over the previous batch, within [-1, 1] (16.16)
    long long rate = 0;
    if (ctrl->grow_den >= GROW_MIN_EVENTS) {
        rate = ctrl->grow_num * 65536 / (long long)ctrl->grow_den;
        rate = max(-65536ll, min(65536ll, rate));
    }
    // the band drifts at that rate only when the queue changed by more than an eighth over
    // the previous batch (a stream filling up); a queue that only wanders keeps a flat
    // band, and the sampled windows catch the rest
    const long long dq = ctrl->grow_num < 0 ? -ctrl->grow_num : ctrl->grow_num;
    const long long slope = dq * 8 > (long long)qprev ? rate : 0;
    // the table reaches 1.25 times the queue at the batch start (639 of DET_G / 2
    // chunks); a queue expected to grow beyond 1.2 times it sizes the chunks instead
    const long long q_end = max((long long)kp.q_min,
                                min((long long)kp.q_max, (long long)qprev + rate * (long long)g.m / 65536));
    const unsigned long long q_hi = (unsigned long long)q_end * 5 > qprev * 6 ? (unsigned long long)q_end : qprev;
    unsigned long long S = (2ull * q_hi + 4ull * CHUNK + DET_G - 1) / DET_G;
    S = max(S, ((unsigned long long)g.m + DET_MAX_CHUNKS - 1) / DET_MAX_CHUNKS);
    if (qprev < kp.npix / 32) {
        // a short queue: the band must reach npix / 16 events, or npix / 3 in a stream's
        // first batch (no growth measured yet, and the queue may fill a third of the sensor)
        const unsigned long long reach = ctrl->grow_den == 0 ? 3ull : 16ull;
        S = max(S, ((unsigned long long)kp.npix + reach * DET_BAND - 1) / (reach * DET_BAND));
    }
    S = (S + 15) / 16 * 16;
    g.S = (unsigned)max((unsigned long long)CHUNK, S);
    g.nchunks = (g.m + g.S - 1) / g.S;
    g.mid0 = (unsigned)(qprev / g.S);  // <= 511 by the choice of S
    g.slope = (int)slope;
    const unsigned a = band_lo_lin(g.mid0, g.slope, 0), b = band_lo_lin(g.mid0, g.slope, g.nchunks);
    g.g_lo_min = min(a, b);
    g.g_hi_max = max(a, b) + DET_BAND - 1;
    // old chunks as far back as the sampled columns reach
    const unsigned long long old_chunks = (g.base + g.S - 1) / g.S;
    g.Gold = (unsigned)min((unsigned long long)(HB_BINS - 1), old_chunks);
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

// Suffix histograms by target chunk: for a batch chunk c and distance g,
//   M(c, g) = #{j in chunk c-g : next(j) >= cS}          (per t = 0 pixels, 1 tiles)
// i.e. the events of chunk c-g still last of their pixel / tile at the start of chunk c
// (source chunks reach back to -Gold).  The distinct counts of the aligned window
// [(c-g)S, cS) are N(c, g) = sum_{g'=1..g} M(c, g').  Stored per target chunk c, with
// its band [g_lo(c), g_hi(c)]:
//   base[t][c]             = N(c, g_lo(c) - 1)                (accumulated with atomics)
//   Mt[t][c][g - g_lo(c)]  = M(c, g) for g in [g_lo(c), g_hi(c)]  (a contiguous row)
// A block handles HB_CHUNKS consecutive source chunks and both t: the histograms of chunk
// distances in shared memory (one word of padding per 32 bins and a row pitch of 2 mod
// 32 words, so that a lane's run of 32 bins and the diagonal reads both spread over the
// banks), suffix sums in registers, then per target the sum of its distances below the
// band and, per target row, a run of HB_CHUNKS consecutive band distances.
constexpr int HB_CHUNKS = 12;
constexpr int HB_BLOCKS_PER_SM = 3;  // resident table-build blocks per SM (shared memory)
constexpr int HB_PITCH = 674;   // >= HB_BINS + HB_BINS / 32 words with padding, = 2 (mod 32)
constexpr int MT_PITCH = DET_BAND;  // u16 per target row (512 B: 16-byte aligned rows)


__device__ __forceinline__ int hb_slot(int d) { return d + (d >> 5); }

struct HistSmem {
    unsigned h[2][HB_CHUNKS][HB_PITCH];  // [pixel, tile][source chunk][distance]
    short gl[HB_CHUNKS + HB_BINS];  // first band distance of target c_lo + D (0: no target)
};

// floor(n / S) for the histogram's small quotients (n < 640 S): a single-precision
// estimate from a reciprocal, then made exact with integer products (the estimate is
// within one of the quotient since n / S < 2^10 and n is converted with 24 bits).
struct ChunkDiv {
    unsigned S;
    float r;
    __device__ explicit ChunkDiv(unsigned S_) : S(S_), r(1.0f / (float)S_) {}
    __device__ __forceinline__ unsigned operator()(unsigned n) const
    {
        unsigned q = (unsigned)((float)n * r);
        if (q * S > n) --q;
        if ((q + 1) * S <= n) ++q;
        return q;
    }
};

// kBuild 0: first build, bands from (mid0, slope), plus the sampled columns.
// kBuild 1: second build, only when k_det_center asked for it (band_mode), bands from the
//           sampled windows; its below-band sums go to the second set of counters.
template <int kBuild>
__global__ void __launch_bounds__(256)
k_det_hist(KParams kp, Ctrl *ctrl, const uint4 *ring, unsigned short *Mt, size_t mt_rows, unsigned *base_cnt,
           unsigned short *prof, size_t n_samples, const unsigned short *ctr)
{
    PDL_ENTRY();
    if (kBuild == 1 && ctrl->band_mode == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HistSmem &H = *reinterpret_cast<HistSmem *>(smem_raw);
    const Geo g = geometry(kp, ctrl);
    const unsigned ns = n_samples_of(g.nchunks), sstep = sample_step(g.nchunks);
    const unsigned tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
    const unsigned nwork = g.nchunks + g.Gold;
    const unsigned nunits = (nwork + HB_CHUNKS - 1) / HB_CHUNKS;
    const long long lo_exist = -(long long)g.base;
    // distances whose band entries some target may need
    const int D0 = kBuild ? 1 : (int)g.g_lo_min;
    const int g_hi_all = kBuild ? HB_BINS - 1 : (int)g.g_hi_max;
    unsigned *bc = base_cnt + (size_t)kBuild * 2 * mt_rows;
    auto band_of = [&](long long ct) -> int {
        return kBuild ? (int)band_lo_tab(ctr, ns, sstep, ct) : (int)band_lo_lin(g.mid0, g.slope, ct);
    };
    const ChunkDiv div_S(g.S);
    for (unsigned unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
        const long long c_lo = (long long)(unit * HB_CHUNKS) - (long long)g.Gold;  // first source chunk
        uint4 *hw = reinterpret_cast<uint4 *>(&H.h[0][0][0]);
        for (unsigned i = tid; i < 2 * HB_CHUNKS * HB_PITCH / 4; i += 256) hw[i] = make_uint4(0u, 0u, 0u, 0u);
        for (unsigned D = tid; D < HB_CHUNKS + HB_BINS; D += 256) {
            const long long ct = c_lo + D;
            H.gl[D] = (short)(ct >= 1 && ct < (long long)g.nchunks ? band_of(ct) : 0);
        }
        __syncthreads();
        // histograms of the chunk distance to the next event of the same pixel and of the
        // same tile (distances beyond the table counted at its last one)
        const long long j_lo = c_lo * g.S;
        const unsigned n_hi = (unsigned)min((long long)HB_CHUNKS * g.S, (long long)g.m - j_lo);
        const unsigned n_lo = (unsigned)max(0ll, lo_exist - j_lo);
        const unsigned long long lim = (unsigned long long)(HB_BINS - 1) * g.S;
        for (unsigned i = n_lo + tid; i < n_hi; i += 256) {
            const unsigned long long j = g.base + (unsigned long long)(j_lo + i);
            const uint2 n = nxt_of(ring, j & kp.ring_mask);
            const unsigned cc = div_S(i), r = i - cc * g.S;
            // distances from the start of chunk cc, in chunks
            const unsigned long long rp = (unsigned long long)r + n.x, rt = (unsigned long long)r + n.y;
            const unsigned dp = (n.x == SAT || rp >= lim) ? (unsigned)(HB_BINS - 1) : div_S((unsigned)rp);
            const unsigned dt = (n.y == SAT || rt >= lim) ? (unsigned)(HB_BINS - 1) : div_S((unsigned)rt);
            atomicAdd(&H.h[0][cc][hb_slot((int)dp)], 1u);
            atomicAdd(&H.h[1][cc][hb_slot((int)dt)], 1u);
        }
        __syncthreads();
        // suffix sums over d: warp per (type, chunk) row, lane l owns bins 32l .. 32l+31
        for (unsigned rw = wl; rw < 2 * HB_CHUNKS; rw += 8) {
            const bool own = lane < HB_BINS / 32;
            unsigned *row = &H.h[rw / HB_CHUNKS][rw % HB_CHUNKS][33 * (own ? lane : 0)];
            unsigned v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = own ? row[i] : 0u;
#pragma unroll
            for (int i = 30; i >= 0; --i) v[i] += v[i + 1];
            unsigned x = v[0];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_down_sync(0xFFFFFFFFu, x, o);
                if (lane + o < 32) x += y;
            }
            const unsigned carry = x - v[0];  // bins above this lane's run
            if (own) {
#pragma unroll
                for (int i = 0; i < 32; ++i) row[i] = v[i] + carry;
            }
        }
        __syncthreads();
        // below the band: target c_lo + D gets sum_{cc} M at distance D - cc in [1, g_lo)
        for (int D = 1 + (int)tid; D < HB_CHUNKS + g_hi_all - (int)DET_BAND; D += 256) {
            const long long ct = c_lo + D;
            const int gl = H.gl[D];
            if (gl == 0) continue;
            unsigned acc0 = 0, acc1 = 0;
#pragma unroll
            for (int cc = 0; cc < HB_CHUNKS; ++cc) {
                const int d = D - cc;
                if (d >= 1 && d < gl) {
                    acc0 += H.h[0][cc][hb_slot(d)];
                    acc1 += H.h[1][cc][hb_slot(d)];
                }
            }
            if (acc0) atomicAdd(&bc[ct], acc0);
            if (acc1) atomicAdd(&bc[mt_rows + ct], acc1);
        }
        // the bands: target row c_lo + D receives distances D-15 .. D from the block's
        // sources; HB_CHUNKS threads write one row's run (both types)
        const int D1 = g_hi_all + HB_CHUNKS - 1;  // targets with some band distance
        for (unsigned i = tid; i < (unsigned)(D1 - D0 + 1) * HB_CHUNKS; i += 256) {
            const int D = D0 + (int)(i / HB_CHUNKS), u = (int)(i % HB_CHUNKS);
            const int cc = HB_CHUNKS - 1 - u, d = D - cc;
            const long long ct = c_lo + D;  // target chunk
            const int gl = H.gl[D];
            if (gl != 0 && d >= gl && d < gl + (int)DET_BAND) {
                const size_t at = (size_t)ct * MT_PITCH + (d - gl);
                Mt[at] = (unsigned short)H.h[0][cc][hb_slot(d)];
                Mt[(size_t)mt_rows * MT_PITCH + at] = (unsigned short)H.h[1][cc][hb_slot(d)];
            }
        }
        if (kBuild == 0 && ns > 0) {
            // columns of the sampled targets sstep * s within reach of the sources:
            // prof[t][s][d] = M(sstep * s, d), d in 1..639 (HB_CHUNKS threads write the
            // consecutive distances one sample takes from the block's sources)
            const int t_lo = (int)c_lo + 1, t_hi = (int)c_lo + HB_CHUNKS - 1 + (HB_BINS - 1);
            const int st = (int)sstep;
            const int s_lo = t_lo <= st ? 1 : (t_lo + st - 1) / st;
            const int s_hi = min((int)ns, t_hi / st);
            for (int i = (int)tid; i < (s_hi - s_lo + 1) * HB_CHUNKS; i += 256) {
                const int sidx = s_lo + i / HB_CHUNKS, cc = i % HB_CHUNKS;
                const int d = sidx * st - ((int)c_lo + cc);
                if (d >= 1 && d <= HB_BINS - 1) {
                    prof[(size_t)sidx * HB_BINS + d] = (unsigned short)H.h[0][cc][hb_slot(d)];
                    prof[((size_t)n_samples + sidx) * HB_BINS + d] = (unsigned short)H.h[1][cc][hb_slot(d)];
                }
            }
        }
        __syncthreads();
    }
    if (kBuild == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->S = g.S;
        ctrl->nchunks = g.nchunks;
        ctrl->band_mid0 = g.mid0;
        ctrl->band_slope = g.slope;
        ctrl->Gold = g.Gold;
    }
}

// The regulator's window at every sampled chunk c = step * s (one warp each): the
// shortest aligned window of the column prof[.][s][1..639] that the regulator would
// shrink (the test of k_det_init), or the longest one that exists.  If one of them lies
// outside (or within BAND_MARGIN of the edge of) the first build's band, band_mode asks
// for the second build.
__global__ void __launch_bounds__(256)
k_det_center(KParams kp, Ctrl *ctrl, const unsigned short *prof, size_t n_samples, unsigned short *ctr)
{
    PDL_ENTRY();
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long base = ctrl->base;
    const unsigned S = ctrl->S, nch = ctrl->nchunks, Gold = ctrl->Gold;
    const unsigned mid0 = ctrl->band_mid0;
    const int slope = ctrl->band_slope;
    const unsigned ns = n_samples_of(nch), sstep = sample_step(nch);
    const unsigned warps_total = gridDim.x * (blockDim.x >> 5);
    constexpr int PER = HB_BINS / 32;  // distances per lane
    bool out = false;
    for (unsigned s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) + 1; s <= ns; s += warps_total) {
        const unsigned c = s * sstep;
        const unsigned gmax = min((unsigned)(HB_BINS - 1), c + Gold);  // sources that exist
        const unsigned long long reach = (unsigned long long)c * S + base;
        const unsigned short *pp = prof + (size_t)s * HB_BINS;
        const unsigned short *pt = prof + ((size_t)n_samples + s) * HB_BINS;
        unsigned ap[PER], at[PER], sp = 0, st = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const unsigned gg = lane * PER + u;  // distance 0 is not a window
            const bool ok = gg >= 1 && gg <= gmax;
            sp += ok ? pp[gg] : 0u;
            st += ok ? pt[gg] : 0u;
            ap[u] = sp;
            at[u] = st;
        }
        unsigned ip = sp, it = st;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned yp = __shfl_up_sync(0xFFFFFFFFu, ip, o), yt = __shfl_up_sync(0xFFFFFFFFu, it, o);
            if (lane >= (unsigned)o) { ip += yp; it += yt; }
        }
        const unsigned op = ip - sp, ot = it - st;
        unsigned mine = 0;
#pragma unroll
        for (int u = PER - 1; u >= 0; --u) {
            const unsigned gg = lane * PER + u;
            const unsigned long long np = op + ap[u], nt = ot + at[u];
            const unsigned long long L = min((unsigned long long)gg * S, reach), q = L + 1;
            if (gg >= 1 && gg <= gmax && np > 0 && q > kp.q_min &&
                (q > kp.q_max || q * kp.den * np > L * kp.numA * nt))
                mine = gg;
        }
        const unsigned any = __ballot_sync(0xFFFFFFFFu, mine != 0);
        const unsigned w = any ? __shfl_sync(0xFFFFFFFFu, mine, __ffs(any) - 1) : gmax;
        if (lane == 0) {
            ctr[s] = (unsigned short)w;
            const unsigned gl = band_lo_lin(mid0, slope, c);
            out |= (w < gl + BAND_MARGIN || w + BAND_MARGIN > gl + DET_BAND - 1) && band_clamp(w) != gl;
        }
    }
    if (out) {
        if (atomicOr(&ctrl->band_mode, 1u) == 0u) atomicAdd(&ctrl->recenters, 1ull);
    }
}

// q_targ = max(q_min, min(q_max, floor(X / Y))) (Eq. 20 as the ratio X / Y, Y = 0 when
// N_ap = 0): a single-precision quotient, then corrected with exact 64-bit products so
// that the result is the exact floor.
__device__ __forceinline__ unsigned q_target(const KParams &kp, unsigned long long X, unsigned Y)
{
    if (Y == 0) return max(kp.q_min, kp.q_max);
    // X as a float from its 32-bit halves (a 64-bit conversion is slow)
    const float xf = fmaf(__uint2float_rn((unsigned)(X >> 32)), 4294967296.0f, __uint2float_rn((unsigned)X));
    const float r = __fdividef(xf, __uint2float_rn(Y));
    unsigned t = r >= (float)kp.q_max ? kp.q_max + 1u : (unsigned)r;
    while (t > 0 && (unsigned long long)t * Y > X) --t;                     // t <= X / Y
    while (t <= kp.q_max && (unsigned long long)(t + 1) * Y <= X) ++t;      // t = floor, or above q_max
    return max(kp.q_min, min(kp.q_max, t));
}

// Speculative start of chunk c >= 1, one warp per chunk.
// (1) The window: among the aligned windows of g in the chunk's band [g_lo, g_hi] of
//     chunks ending at cS (N(c, g_lo - 1) plus a prefix sum of one band row: 8 distances per lane, one
//     16-byte load per lane and type), the first that the regulator would shrink at the
//     next event (Eq. 20); then, inside the chunk where that window starts, the shortest
//     window, to the event, that would still be shrunk.  Its length is where the
//     regulator holds the queue.
// (2) Step cS applied to it.  All pops of a step test against the ratio X / Y of the
//     previous step, so their number is q - q_targ at once; the warp counts the pixels
//     and tiles whose last queued event is among the popped ones.
__device__ __forceinline__ unsigned pick8(const unsigned (&a)[8], unsigned u)
{
    unsigned r = a[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) r = u == (unsigned)i ? a[i] : r;
    return r;
}

// kMode: the table build in use (0: bands from (mid0, slope); 1: from the sampled
// windows, below-band counts in the second set).  One copy of the body per build keeps
// the loads at the top of each chunk independent of the mode.
template <int kMode>
__device__ __forceinline__ void init_chunks(const KParams &kp, const Ctrl *ctrl, const uint4 *ring,
                                            const unsigned short *Mt, size_t mt_rows, unsigned *base_cnt,
                                            const unsigned short *ctr, DetState *E0, unsigned *qout)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long base = ctrl->base;
    const unsigned S = ctrl->S, nch = ctrl->nchunks, Gold = ctrl->Gold;
    const unsigned mid0 = ctrl->band_mid0;
    const int slope = ctrl->band_slope;
    const unsigned ns = n_samples_of(nch), sstep = sample_step(nch);
    unsigned *bc = base_cnt + (size_t)kMode * 2 * mt_rows;
    const unsigned warps_total = gridDim.x * (blockDim.x >> 5);
    for (unsigned c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) + 1; c < nch; c += warps_total) {
        const unsigned g_lo = kMode ? band_lo_tab(ctr, ns, sstep, c) : band_lo_lin(mid0, slope, c);
        const unsigned g_hi = g_lo + DET_BAND - 1;
        const unsigned short *rp = Mt + (size_t)c * MT_PITCH;
        const unsigned short *rt = Mt + (mt_rows + c) * MT_PITCH;
        const unsigned gmax = min(g_hi, c + Gold);  // sources that exist in the table
        const unsigned long long reach = (unsigned long long)c * S + base;  // events before the chunk
        // N(c, g_lo - 1), then cleared for the next batch's accumulation
        const unsigned bp = bc[c], bt = bc[mt_rows + c];
        unsigned found = 0, snp = 0, snt = 0, fp1 = bp, ft1 = bt;
        const uint4 wp = *reinterpret_cast<const uint4 *>(rp + 8 * lane);
        const uint4 wt = *reinterpret_cast<const uint4 *>(rt + 8 * lane);
        __syncwarp();
        if (lane == 0) {
            bc[c] = 0;
            bc[mt_rows + c] = 0;
            if (kMode) {  // the first build's counters too
                base_cnt[c] = 0;
                base_cnt[mt_rows + c] = 0;
            }
        }
        const unsigned xp[4] = {wp.x, wp.y, wp.z, wp.w}, xt[4] = {wt.x, wt.y, wt.z, wt.w};
        unsigned pp[8], pt[8];
        unsigned sp = 0, st = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const unsigned gg = g_lo + 8 * lane + u;
            const bool ok = gg <= gmax;
            sp += ok ? (xp[u >> 1] >> (16 * (u & 1))) & 0xFFFFu : 0u;
            st += ok ? (xt[u >> 1] >> (16 * (u & 1))) & 0xFFFFu : 0u;
            pp[u] = sp;
            pt[u] = st;
        }
        // exclusive prefix of the lanes' sums
        unsigned ip = sp, it = st;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned yp = __shfl_up_sync(0xFFFFFFFFu, ip, o), yt = __shfl_up_sync(0xFFFFFFFFu, it, o);
            if (lane >= (unsigned)o) { ip += yp; it += yt; }
        }
        const unsigned op = bp + ip - sp, ot = bt + it - st;
        unsigned mine = 0;
#pragma unroll
        for (int u = 7; u >= 0; --u) {
            const unsigned gg = g_lo + 8 * lane + u;
            const unsigned long long np = op + pp[u], nt = ot + pt[u];
            const unsigned long long L = min((unsigned long long)gg * S, reach), q = L + 1;
            if (np > 0 && q > kp.q_min && (q > kp.q_max || q * kp.den * np > L * kp.numA * nt)) mine = gg;
        }
        const unsigned any = __ballot_sync(0xFFFFFFFFu, mine != 0);
        if (any) {
            found = __shfl_sync(0xFFFFFFFFu, mine, __ffs(any) - 1);
            // N(c, found - 1): the base when found is the band's first distance
            if (found > g_lo) {
                const unsigned g1 = found - 1 - g_lo, owner = g1 >> 3, u = g1 & 7;
                fp1 = __shfl_sync(0xFFFFFFFFu, op + pick8(pp, u), owner);
                ft1 = __shfl_sync(0xFFFFFFFFu, ot + pick8(pt, u), owner);
            }
        }
        const unsigned carry_p = bp + __shfl_sync(0xFFFFFFFFu, ip, 31);  // N(c, g_hi)
        const unsigned carry_t = bt + __shfl_sync(0xFFFFFFFFu, it, 31);
        const long long k0 = (long long)c * S;
        long long h;
        if (found && (unsigned long long)found * S <= reach) {
            // The window starts in chunk c - found: take the shortest one, to the event, that
            // the regulator would still shrink.  Its counts are N(c, found - 1) plus the
            // events from its start to the end of that chunk that are the last of their
            // pixel / tile before k0 (suffix sums of those flags, 32 events per round from
            // the chunk's end).
            const long long j0 = k0 - (long long)found * S;
            unsigned cfp = 0, cft = 0, best = 0;
            bool got = false;
            for (int blk = (int)((S - 1) / 32); blk >= 0 && !got; --blk) {
                const unsigned y = (unsigned)blk * 32 + lane;
                unsigned fp = 0, ft = 0;
                if (y < S) {
                    const long long j = j0 + y;
                    const uint2 n = nxt_of(ring, (base + (unsigned long long)j) & kp.ring_mask);
                    const unsigned long long dj = (unsigned long long)(k0 - j);
                    fp = n.x == SAT || n.x >= dj;
                    ft = n.y == SAT || n.y >= dj;
                }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned yp = __shfl_down_sync(0xFFFFFFFFu, fp, o), yt = __shfl_down_sync(0xFFFFFFFFu, ft, o);
                    if (lane + o < 32) { fp += yp; ft += yt; }
                }
                const unsigned long long np = fp1 + cfp + fp, nt = ft1 + cft + ft;
                const unsigned long long L = (unsigned long long)found * S - y, q = L + 1;
                const bool shr = y < S && np > 0 && q > kp.q_min && (q > kp.q_max || q * kp.den * np > L * kp.numA * nt);
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, shr);
                if (bal) {
                    const unsigned top = 31 - __clz(bal);
                    best = (unsigned)blk * 32 + top;
                    snp = __shfl_sync(0xFFFFFFFFu, (unsigned)np, top);
                    snt = __shfl_sync(0xFFFFFFFFu, (unsigned)nt, top);
                    got = true;
                }
                cfp += __shfl_sync(0xFFFFFFFFu, fp, 0);
                cft += __shfl_sync(0xFFFFFFFFu, ft, 0);
            }
            h = j0 + best;  // y = 0 always shrinks (the aligned window of `found` chunks)
        } else {
            // no shrinking window within g_hi chunks (then all of them), or the window
            // reaches back to the stream start (then the whole history): the counts
            // accumulated over the scanned distances
            h = max(k0 - (long long)(found ? found : g_hi) * S, -(long long)base);
            snp = carry_p;
            snt = carry_t;
        }
        const unsigned long long ql = (unsigned long long)(k0 - h);
        const unsigned long long X = ql * kp.numA * snt, Y = (unsigned long long)kp.den * snp;
        // step k0
        const uint2 d = prv_of(ring, (base + (unsigned long long)k0) & kp.ring_mask);
        unsigned nap = snp + (d.x > ql ? 1u : 0u);
        unsigned nat = snt + (d.y > ql ? 1u : 0u);
        const unsigned long long q = ql + 1;
        const unsigned thr = q_target(kp, X, (unsigned)Y);
        const unsigned P = q > thr ? (unsigned)(q - thr) : 0u;
        unsigned offp = 0, offt = 0;
#pragma unroll 4
        for (unsigned u = lane; u < P; u += 32) {
            const long long j = h + u;
            const uint2 n = nxt_of(ring, (base + (unsigned long long)j) & kp.ring_mask);
            const unsigned long long dj = (unsigned long long)(k0 - j);
            offp += n.x > dj;
            offt += n.y > dj;
        }
        nap -= warp_sum(offp);
        nat -= warp_sum(offt);
        if (lane == 0) {
            const unsigned long long qn = q - P;
            DetState st0;
            st0.h = h + P;
            st0.nap = nap;
            st0.nat = nat;
            st0.X = qn * kp.numA * nat;
            st0.Y = (unsigned long long)kp.den * nap;
            E0[c] = st0;
            qout[k0] = (unsigned)qn;
        }
    }
}

__global__ void __launch_bounds__(256)
k_det_init(KParams kp, const Ctrl *ctrl, const uint4 *ring, const unsigned short *Mt, size_t mt_rows,
           unsigned *base_cnt, const unsigned short *ctr, DetState *E0, unsigned *qout)
{
    PDL_ENTRY();
    if (ctrl->band_mode)
        init_chunks<1>(kp, ctrl, ring, Mt, mt_rows, base_cnt, ctr, E0, qout);
    else
        init_chunks<0>(kp, ctrl, ring, Mt, mt_rows, base_cnt, ctr, E0, qout);
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

// ---------------------------------------------------------------------------------------
// Lane engine for the parallel passes: lane j of a warp runs chunk j's steps one after
// the other (32 chunks per warp).  Each lane stages the links its next steps need in
// shared memory with asynchronous copies, one block of LR_B steps ahead:
//   push: {dP, dT} of the block's events, double buffered;
//   pop:  {nP, nT} of the events from the queue front h on, a ring of LR_R entries kept
//         full; pops past the landed entries read the ring buffer in global memory;
//   ref:  (merge mode) the queue lengths already in qout, to detect the merge.
// A step counts its pops first (the pop test needs only q and the ratio of the previous
// step), then reads the popped events' links.  A lane with more than LR_BIG pops in a
// step (after a bad start) has them counted by the whole warp with coalesced loads, and
// its ring refilled.
constexpr int LR_B = 16;      // steps per staged block
constexpr int LR_R = 128;     // pop-link ring entries per lane (power of two)
constexpr int LR_BIG = 64;    // pops per step handled by the lane alone
constexpr int LR_WARPS = 2;   // warps per block

struct LaneSmem {
    uint2 push[2][32][LR_B + 1];
    uint2 pop[32][LR_R + 1];
    unsigned ref[2][32][LR_B + 1];
};

__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}
// n 8-byte copies from a source with a 16-byte stride to consecutive shared slots (a
// shared address and a global pointer walked by plain increments)
__device__ __forceinline__ void cp_async8_run(unsigned dst_s, const uint2 *src, int n)
{
    const char *p = reinterpret_cast<const char *>(src);
    for (int u = 0; u < n; ++u, dst_s += 8, p += 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst_s), "l"(p) : "memory");
}
__device__ __forceinline__ const uint2 *nxt_ptr(const uint4 *ring, unsigned base32, unsigned mask32, int e)
{
    return reinterpret_cast<const uint2 *>(ring) + 2 * ((base32 + (unsigned)e) & mask32) + 1;
}

// Lane j runs its chunk's steps [k0, k1) from st, writing the queue lengths of steps
// k >= kw to qout.  kMerge: stop before the first step whose queue length equals qout's
// (the entry is already right) and return whether that happened; *nsteps counts the steps
// up to and including the merge.
template <bool kMerge>
__device__ bool lane_run(const KParams &kp, unsigned long long base, const uint4 *__restrict__ ring,
                         unsigned *qout, unsigned k0, unsigned k1, unsigned kw, DetState &st,
                         LaneSmem &sm, Ctrl *ctrl, unsigned *nsteps)
{
    unsigned *err = &ctrl->error;
    unsigned n_big = 0, n_miss = 0;
    const unsigned lane = threadIdx.x & 31;
    const unsigned mask32 = (unsigned)kp.ring_mask, base32 = (unsigned)base;
    const uint2 *ring2 = reinterpret_cast<const uint2 *>(ring);
    const uint2 *rg = sm.pop[lane];
    int h = (int)st.h;
    unsigned nap = st.nap, nat = st.nat;
    unsigned long long X = st.X;
    unsigned Y = (unsigned)st.Y;
    bool active = k0 < k1, merged = false;
    unsigned done = 0;
    unsigned span = active ? k1 - k0 : 0u;
#pragma unroll
    for (int o = 16; o; o >>= 1) span = max(span, __shfl_xor_sync(0xFFFFFFFFu, span, o));
    const unsigned nblk = (span + LR_B - 1) / LR_B;
    // pop links [h, v) have landed, [v, f) are in flight; a short run stages fewer
    const int ring_fill = (int)min((unsigned)LR_R, 4u * span + 16u);
    int f = h, v = h;
    // copy the pop links of events [e, e + n) into the lane's ring (n <= LR_R), walking
    // source and destination pointers through at most two wraps of each ring
    auto copy_links = [&](int e, int n) {
        while (n > 0) {
            const unsigned gs = (base32 + (unsigned)e) & mask32;          // global slot
            const unsigned ss = (unsigned)e & (LR_R - 1);                // ring slot
            const int run = min(n, (int)min(mask32 + 1 - gs, (unsigned)LR_R - ss));
            cp_async8_run((unsigned)__cvta_generic_to_shared(&sm.pop[lane][ss]), ring2 + 2 * (size_t)gs + 1, run);
            e += run;
            n -= run;
        }
    };
    auto fill_pop = [&]() {
        if (f < h) f = h;
        const int want = active ? h + ring_fill - f : 0;
        copy_links(f, want);
        if (want > 0) f = h + ring_fill;
    };
    auto stage = [&](int buf, unsigned b) {
        const unsigned kb = k0 + b * LR_B;
        const int n = active ? (int)min((unsigned)LR_B, k1 > kb ? k1 - kb : 0u) : 0;
        const unsigned gs = (base32 + kb) & mask32;
        const int run = min(n, (int)(mask32 + 1 - gs));
        const unsigned dst_s = (unsigned)__cvta_generic_to_shared(&sm.push[buf][lane][0]);
        cp_async8_run(dst_s, ring2 + 2 * (size_t)gs, run);
        cp_async8_run(dst_s + 8u * (unsigned)run, ring2, n - run);
        if (kMerge)
            for (int u = 0; u < n; ++u) cp_async4(&sm.ref[buf][lane][u], qout + kb + u);
    };
    fill_pop();
    stage(0, 0);
    cp_async_wait_all();
    v = f;
    __syncwarp();
    for (unsigned b = 0; b < nblk; ++b) {
        if (!__any_sync(0xFFFFFFFFu, active)) break;
        const int buf = b & 1;
        if (b + 1 < nblk) stage(buf ^ 1, b + 1);
        fill_pop();
        for (unsigned i = 0; i < LR_B; ++i) {
            const unsigned k = k0 + b * LR_B + i;
            bool act = active && k < k1;
            const int dist = (int)k - h;
            if (act && dist < 0) {  // impossible for a consistent state; never loop on a bad one
                atomicOr(err, ERR_BAD_STATE);
                active = act = false;
            }
            // push
            const uint2 d = sm.push[buf][lane][i];
            const unsigned ud = (unsigned)dist;
            if (act) {
                nap += d.x > ud;
                nat += d.y > ud;
            }
            unsigned q = ud + 1u;
            // pops of this step: the test "q > q_targ" is monotone in q
            unsigned P = 0;
            if (act) {
                const unsigned T = q_target(kp, X, Y);
                P = q > T ? q - T : 0u;
            }
            if (__any_sync(0xFFFFFFFFu, P > LR_BIG)) {
                // the warp counts the big pops with coalesced loads and refills those
                // lanes' rings; in-flight copies land first so that no ring slot races
                unsigned big = __ballot_sync(0xFFFFFFFFu, P > LR_BIG);
                cp_async_wait_all();
                __syncwarp();
                if (f > v) v = f;
                while (big) {
                    const unsigned j = __ffs(big) - 1;
                    big &= big - 1;
                    const int hj = __shfl_sync(0xFFFFFFFFu, h, j);
                    const unsigned Pj = __shfl_sync(0xFFFFFFFFu, P, j), kj = __shfl_sync(0xFFFFFFFFu, k, j);
                    unsigned op = 0, ot = 0;
#pragma unroll 4
                    for (unsigned u = lane; u < Pj; u += 32) {
                        const uint2 n = *nxt_ptr(ring, base32, mask32, hj + (int)u);
                        const unsigned dj = kj - (unsigned)(hj + (int)u);
                        op += n.x > dj;
                        ot += n.y > dj;
                    }
                    op = warp_sum(op);
                    ot = warp_sum(ot);
                    const int hn = hj + (int)Pj;
                    for (unsigned u = lane; u < LR_R; u += 32)
                        sm.pop[j][(hn + (int)u) & (LR_R - 1)] = *nxt_ptr(ring, base32, mask32, hn + (int)u);
                    if (lane == j) {
                        ++n_big;
                        nap -= op;
                        nat -= ot;
                        h = hn;
                        q -= Pj;
                        P = 0;
                        f = v = hn + LR_R;
                    }
                }
                __syncwarp();
            }
            // the lane's own pops, links from its ring, four per iteration (from global
            // memory past the landed entries: rare, a separate loop)
            if (!__any_sync(0xFFFFFFFFu, h + (int)P > v)) {
                const unsigned hu = (unsigned)h, kh = k - hu;  // k - e = kh - u for e = h + u
                for (unsigned u = 0; u < P; u += 4) {
                    // four pops per iteration: the four ring loads in flight together
                    const uint2 n0 = rg[(hu + u) & (LR_R - 1)];
                    const uint2 n1 = rg[(hu + u + 1) & (LR_R - 1)];
                    const uint2 n2 = rg[(hu + u + 2) & (LR_R - 1)];
                    const uint2 n3 = rg[(hu + u + 3) & (LR_R - 1)];
                    const unsigned r = P - u;  // pops left (>= 1)
                    const unsigned d0 = kh - u;
                    nap -= (n0.x > d0) + (r > 1 && n1.x > d0 - 1) + (r > 2 && n2.x > d0 - 2) + (r > 3 && n3.x > d0 - 3);
                    nat -= (n0.y > d0) + (r > 1 && n1.y > d0 - 1) + (r > 2 && n2.y > d0 - 2) + (r > 3 && n3.y > d0 - 3);
                }
                h += (int)P;
            } else {
                for (unsigned u = 0; u < P; ++u) {
                    n_miss += h >= v;
                    const uint2 n = h < v ? sm.pop[lane][h & (LR_R - 1)] : *nxt_ptr(ring, base32, mask32, h);
                    const unsigned dj = k - (unsigned)h;
                    nap -= n.x > dj;
                    nat -= n.y > dj;
                    ++h;
                }
            }
            q -= P;
            if (act) {
                X = (unsigned long long)q * kp.numA * nat;
                Y = kp.den * nap;
                if (kMerge && sm.ref[buf][lane][i] == q) {
                    merged = true;
                    active = false;
                    done = k + 1 - k0;
                } else if (k >= kw) {
                    qout[k] = q;
                }
            }
        }
        cp_async_wait_all();
        v = f;
        __syncwarp();
    }
    if (!kMerge || !merged) done = k1 > k0 ? k1 - k0 : 0u;
    if (nsteps) *nsteps = done;
    n_big = warp_sum(n_big);
    n_miss = warp_sum(n_miss);
    if (lane == 0 && (n_big | n_miss)) {
        atomicAdd(&ctrl->big_pops, (unsigned long long)n_big);
        atomicAdd(&ctrl->ring_misses, (unsigned long long)n_miss);
    }
    st.h = h; st.nap = nap; st.nat = nat; st.X = X; st.Y = Y;
    return merged;
}

// Chunk c's own steps (its queue lengths are pass 1's and its exit is E1[c]) are
// [own_begin(c), own_begin(c + 1)); for c >= 1 they start DET_WARM steps after its
// speculative start at cS, which pass 1 uses to converge.  The last chunk keeps at
// least its last event.
__device__ __forceinline__ unsigned own_begin(unsigned c, unsigned S, unsigned m)
{
    return c == 0 ? 0u : min(c * S + DET_WARM, m - 1);
}
__device__ __forceinline__ unsigned own_end(unsigned c, unsigned S, unsigned m, unsigned nch)
{
    return c + 1 < nch ? own_begin(c + 1, S, m) : m;
}

// Pass 1: chunk c >= 1 runs from its speculative start E0[c] (the state after step cS)
// to the end of its own steps, recording those; chunk 0 starts from the true state at the
// batch start.
__global__ void __launch_bounds__(32 * LR_WARPS, 1)
k_det_pass1(KParams kp, Ctrl *ctrl, const uint4 *ring, unsigned *qout,
            const DetState *E0, DetState *E1)
{
    PDL_ENTRY();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LaneSmem &sm = reinterpret_cast<LaneSmem *>(smem_raw)[threadIdx.x >> 5];
    const unsigned long long base = ctrl->base;
    const unsigned m = ctrl->m, S = ctrl->S, nch = ctrl->nchunks;
    const unsigned lane = threadIdx.x & 31;
    const unsigned warps = gridDim.x * LR_WARPS;
    for (unsigned wb = (blockIdx.x * LR_WARPS + (threadIdx.x >> 5)) * 32; wb < nch; wb += warps * 32) {
        const unsigned c = wb + lane;
        DetState st{0, 0, 0, 0, 1};
        unsigned k0 = 0, k1 = 0, kw = 0;
        if (c < nch) {
            k1 = own_end(c, S, m, nch);
            kw = own_begin(c, S, m);
            if (c == 0) {
                st = ctrl->det;
                st.h = (long long)((unsigned long long)st.h - base);
                k0 = 0;
            } else {
                st = E0[c];
                k0 = c * S + 1;
            }
        }
        lane_run<false>(kp, base, ring, qout, k0, k1, kw, st, sm, ctrl, nullptr);
        if (c < nch) E1[c] = st;
    }
}

// Pass 2: chunk c >= 1 re-runs from pass 1's exit of chunk c-1 until it merges with
// pass 1's trajectory of its own chunk.  Most chunks merge within a few steps, a few
// need tens: the lane stage (k_det_pass2) runs every chunk for at most P2_LANE_STEPS
// steps and lists the ones still running, which k_det_pass2w continues one warp per
// chunk (a step costs a warp there, but the chains of the slow chunks run side by side).
constexpr unsigned P2_LANE_STEPS = 4;

__device__ __forceinline__ void p2_unmerged(Ctrl *ctrl, const DetState &st, unsigned c, DetState *E2,
                                            unsigned *unm_bits)
{
    E2[c] = st;
    atomicAdd(&ctrl->unmerged, 1u);
    atomicAdd(&ctrl->unmerged_total, 1ull);
    atomicOr(&unm_bits[c >> 5], 1u << (c & 31));
}

__global__ void __launch_bounds__(32 * LR_WARPS, 1)
k_det_pass2(KParams kp, Ctrl *ctrl, const uint4 *ring, unsigned *qout,
            const DetState *E1, DetState *E2, unsigned char *merged, unsigned *unm_bits, unsigned *p2_ids)
{
    PDL_ENTRY();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LaneSmem &sm = reinterpret_cast<LaneSmem *>(smem_raw)[threadIdx.x >> 5];
    const unsigned long long base = ctrl->base;
    const unsigned m = ctrl->m, S = ctrl->S, nch = ctrl->nchunks;
    const unsigned lane = threadIdx.x & 31;
    const unsigned warps = gridDim.x * LR_WARPS;
    for (unsigned wb = (blockIdx.x * LR_WARPS + (threadIdx.x >> 5)) * 32; wb < nch; wb += warps * 32) {
        const unsigned c = wb + lane;
        const bool real = c >= 1 && c < nch;
        DetState st{0, 0, 0, 0, 1};
        unsigned k0 = 0, kend = 0, k1 = 0;
        if (real) {
            st = E1[c - 1];
            k0 = own_begin(c, S, m);
            kend = own_end(c, S, m, nch);
            k1 = min(kend, k0 + P2_LANE_STEPS);
        }
        unsigned steps = 0;
        const bool mg = lane_run<true>(kp, base, ring, qout, k0, k1, k0, st, sm, ctrl, &steps);
        // one atomic per warp for the step count and for the list of continuing chunks
        const unsigned wsteps = warp_sum(real ? steps : 0u);
        const bool cont = real && !mg && k1 < kend;  // continues in k_det_pass2w from k1
        const unsigned cb = __ballot_sync(0xFFFFFFFFu, cont);
        unsigned slot0 = 0;
        if (lane == 0) {
            if (wsteps) atomicAdd(&ctrl->pass2_steps, (unsigned long long)wsteps);
            if (cb) slot0 = atomicAdd(&ctrl->p2_count, (unsigned)__popc(cb));
        }
        slot0 = __shfl_sync(0xFFFFFFFFu, slot0, 0);
        if (real) {
            merged[c] = mg;
            if (cont) {
                E2[c] = st;
                p2_ids[slot0 + __popc(cb & ((1u << lane) - 1u))] = c;
            } else if (!mg) {
                p2_unmerged(ctrl, st, c, E2, unm_bits);
            }
        }
    }
}

__global__ void __launch_bounds__(256)
k_det_pass2w(KParams kp, Ctrl *ctrl, const uint4 *ring, unsigned *qout,
             DetState *E2, unsigned char *merged, unsigned *unm_bits, const unsigned *p2_ids)
{
    PDL_ENTRY();
    const unsigned long long base = ctrl->base;
    const unsigned m = ctrl->m, S = ctrl->S, n = ctrl->p2_count, nch = ctrl->nchunks;
    const unsigned lane = threadIdx.x & 31;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const unsigned c = p2_ids[i];
        DetState st = E2[c];
        const unsigned k0 = own_begin(c, S, m) + P2_LANE_STEPS, k1 = own_end(c, S, m, nch);
        unsigned steps = 0;
        const bool mg = group_run<32, true>(kp, base, ring, qout, k0, k1, st, &ctrl->error, &steps);
        if (lane == 0) {
            atomicAdd(&ctrl->pass2_steps, (unsigned long long)steps);
            if (mg) merged[c] = 1;
            else p2_unmerged(ctrl, st, c, E2, unm_bits);
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
        // the bitmap in shared memory first: all its loads in flight at once
        __shared__ unsigned s_bits[DET_MAX_CHUNKS / 32 + 1];
#pragma unroll 8
        for (unsigned wi = lane; wi < nwords; wi += 32) s_bits[wi] = unm_bits[wi];
        __syncwarp();
        unsigned c = 1;  // chunks < c are exact and chunk c's pass-2 entry E1[c-1] is exact
        DetState exit_c;
        bool have_exit = false;  // exit of chunk c-1 if it differs from E1[c-1]
        while (c < nch) {
            if (!have_exit) {
                // next unmerged chunk >= c
                unsigned w = c >> 5, found = nch;
                for (unsigned wb = w; wb < nwords && found == nch; wb += 32) {
                    const unsigned wi = wb + lane;
                    unsigned bits = wi < nwords ? s_bits[wi] : 0u;
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
            const bool mg = group_run<32, true>(kp, base, ring, qout, own_begin(c, S, m), own_end(c, S, m, nch), st,
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
    nl += 4;
    static std::atomic<unsigned long long> attr_done0{0}, attr_done1{0};
    const size_t smem = sizeof(HistSmem);
    if (cudaError_t e = smem_attr_once(attr_done0, k_det_hist<0>, smem)) return e;
    if (cudaError_t e = smem_attr_once(attr_done1, k_det_hist<1>, smem)) return e;
    if (cudaError_t e_ = launch_pdl(k_det_hist<0>, grid_for(kp, HB_BLOCKS_PER_SM), 256, smem, s, kp, b.ctrl, b.ring4, b.dMt, b.mt_rows,
                                    b.det_base, b.det_prof, b.n_samples, (const unsigned short *)b.band_ctr))
        return e_;
    if (cudaError_t e_ = launch_pdl(k_det_center, grid_for(kp, 2), 256, 0, s, kp, b.ctrl, (const unsigned short *)b.det_prof,
                                    b.n_samples, b.band_ctr))
        return e_;
    if (cudaError_t e_ = launch_pdl(k_det_hist<1>, grid_for(kp, HB_BLOCKS_PER_SM), 256, smem, s, kp, b.ctrl, b.ring4, b.dMt, b.mt_rows,
                                    b.det_base, b.det_prof, b.n_samples, (const unsigned short *)b.band_ctr))
        return e_;
    if (cudaError_t e_ = launch_pdl(k_det_init, grid_for(kp, 8), 256, 0, s, kp, b.ctrl, b.ring4, b.dMt, b.mt_rows,
                                    b.det_base, (const unsigned short *)b.band_ctr, b.E0, b.qout))
        return e_;
    return cudaGetLastError();
}

static cudaError_t lane_smem_attr()
{
    static std::atomic<unsigned long long> done1{0}, done2{0};
    const size_t smem = sizeof(LaneSmem) * LR_WARPS;
    if (cudaError_t e = smem_attr_once(done1, k_det_pass1, smem)) return e;
    return smem_attr_once(done2, k_det_pass2, smem);
}

cudaError_t launch_det_pass1(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    if (cudaError_t e = lane_smem_attr()) return e;
    if (cudaError_t e_ = launch_pdl(k_det_pass1, grid_for(kp, 2), 32 * LR_WARPS, sizeof(LaneSmem) * LR_WARPS, s, kp,
                                    b.ctrl, b.ring4, b.qout, b.E0, b.E1))
        return e_;
    return cudaGetLastError();
}

cudaError_t launch_det_pass2(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 2;
    if (cudaError_t e = lane_smem_attr()) return e;
    if (cudaError_t e_ = launch_pdl(k_det_pass2, grid_for(kp, 2), 32 * LR_WARPS, sizeof(LaneSmem) * LR_WARPS, s, kp,
                                    b.ctrl, b.ring4, b.qout, b.E1, b.E2, b.merged, b.unm_bits, b.p2_ids))
        return e_;
    if (cudaError_t e_ = launch_pdl(k_det_pass2w, grid_for(kp, 8), 256, 0, s, kp, b.ctrl, b.ring4, b.qout, b.E2,
                                    b.merged, b.unm_bits, b.p2_ids))
        return e_;
    return cudaGetLastError();
}

cudaError_t launch_det_fix(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    if (cudaError_t e_ = launch_pdl(k_det_fix, 1, 32, 0, s, kp, b.ctrl, b.ring4, b.qout, b.E1, b.E2, b.merged, b.unm_bits)) return e_;
    return cudaGetLastError();
}

}  // namespace fibar
