// S1: the paper's spatial filter (Sec. 4.2) - when the last queued event of a pixel
// leaves the active event queue, that pixel's L is replaced once by the 3x3 Gaussian of
// the current L around it, and later events of the pixel continue from the blurred
// value (the blur touches L only, never p_bar).
//
// Every blur reads its neighbours at its own step, so blurs depend on earlier blurs.
// The batch is evaluated exactly in five kernels:
//   k_s1_pops   - from the per-event queue lengths, the step at which every popped event
//                 left the queue, and whether its pixel went stale (no later event of the
//                 pixel by then: nP(j) > k - j);
//   k_s1_select - ordered compaction of the stale pops into the blur list, in pop order
//                 (increasing event index = increasing step, Gauss-Seidel within a step);
//   k_s1_lb     - per pixel, the latest blur attached to each of its batch events;
//   k_s1_blur   - dataflow: warps take blurs in list order; a blur waits (bounded) only
//                 for the earlier blurs it reads, then publishes D = B - L_nb, where L_nb
//                 is the pixel's L without this batch's blurs.  A neighbour's L at step k
//                 is L_nb(k) + beta^m D_b, with b its latest earlier blur and m its events
//                 since (the filter is affine with factor beta per event on L);
//   k_s1_apply  - final L of every pixel whose L a blur of this batch changed.
#include "fibar_internal.cuh"

namespace fibar {

constexpr unsigned NOBLUR = 0xFFFFFFFFu;
constexpr int SEL_THREADS = 256, SEL_PER_THREAD = 16, SEL_TILE = SEL_THREADS * SEL_PER_THREAD;

// beta^m: a per-handle table for m < 64 (filled once on the host in double), exp2 beyond
__device__ __forceinline__ float beta_pow(const KParams &kp, const float *tab, int m)
{
    if (m < 64) return __ldg(tab + m);
    return exp2f(kp.log2b * (float)m);
}

// Words that carry their whole message (a tag and a value or count in 64 bits): relaxed
// single-copy-atomic loads and stores suffice, no ordering with other memory is needed.
__device__ __forceinline__ unsigned long long ld_relaxed_u64b(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64b(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

struct S1Geo {
    unsigned long long base;
    long long hs, he;  // batch-relative queue front before / after the batch
    unsigned m;
    unsigned batch_no;
};

__device__ __forceinline__ S1Geo s1_geo(const Ctrl *ctrl)
{
    S1Geo g;
    g.base = ctrl->base;
    g.m = ctrl->m;
    g.hs = (long long)((unsigned long long)ctrl->h_prev - g.base);
    g.he = (long long)((unsigned long long)ctrl->det.h - g.base);
    g.batch_no = ctrl->batch_no;
    return g;
}

// pop step of every event popped in this batch, and whether its pixel went stale
__global__ void __launch_bounds__(256) k_s1_pops(KParams kp, Bufs b)
{
    PDL_ENTRY();
    const S1Geo g = s1_geo(b.ctrl);
    const unsigned *ring_u = reinterpret_cast<const unsigned *>(b.ring4);
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < g.m; k += gridDim.x * blockDim.x) {
        const long long h0 = k == 0 ? g.hs : (long long)k - (long long)b.qout[k - 1];
        const long long h1 = (long long)k + 1 - (long long)b.qout[k];
        for (long long j = h0; j < h1; ++j) {
            const unsigned np = ring_u[4 * ((g.base + (unsigned long long)j) & kp.ring_mask) + 2];
            const bool stale = (long long)np > (long long)k - j;
            b.popk[j - g.hs] = k | (stale ? 0x80000000u : 0u);
        }
    }
}

// ordered compaction of the stale pops (decoupled look-back over tiles)
__global__ void __launch_bounds__(SEL_THREADS) k_s1_select(KParams kp, Bufs b)
{
    PDL_ENTRY();
    __shared__ unsigned s_warp[16];
    __shared__ unsigned s_tile, s_pre;
    Ctrl *ctrl = b.ctrl;
    const S1Geo g = s1_geo(ctrl);
    const unsigned n = (unsigned)(g.he - g.hs);
    const unsigned ntiles = (n + SEL_TILE - 1) / SEL_TILE;
    const unsigned long long tag = (unsigned long long)(g.batch_no + 1u) << 32;
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctrl->sel_ticket, 1u);
        __syncthreads();
        const unsigned tile = s_tile;
        if (tile >= ntiles) break;
        const unsigned i0 = tile * SEL_TILE + threadIdx.x * SEL_PER_THREAD;
        unsigned flags = 0, cnt = 0;
#pragma unroll
        for (int q = 0; q < SEL_PER_THREAD; ++q) {
            const unsigned i = i0 + q;
            if (i < n && (b.popk[i] >> 31)) { flags |= 1u << q; ++cnt; }
        }
        // block exclusive scan of cnt
        unsigned x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned t = threadIdx.x < 8 ? s_warp[threadIdx.x] : 0u;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xFFFFFFFFu, t, o);
                if (lane >= o) t += y;
            }
            if (threadIdx.x < 8) s_warp[8 + threadIdx.x] = t;
        }
        __syncthreads();
        const unsigned excl = (w ? s_warp[8 + w - 1] : 0u) + x - cnt;
        const unsigned tile_cnt = s_warp[15];
        // publish this tile's count; sum all predecessors' counts (no look-back chain)
        unsigned long long *st = b.sel_status;
        // (the status word is the whole message: tag, flag and count)
        if (threadIdx.x == 0) st_relaxed_u64b(&st[tile], tag | (1ull << 30) | tile_cnt);
        unsigned part = 0;
        for (unsigned tp = threadIdx.x; tp < tile; tp += SEL_THREADS) {
            unsigned long long v = ld_relaxed_u64b(&st[tp]);
            unsigned spins = 0;
            while ((v >> 32) != (tag >> 32) || ((v >> 30) & 3ull) == 0ull) {
                if (++spins > SPIN_LIMIT) { atomicOr(&ctrl->error, ERR_SORT_WAIT); break; }
                __nanosleep(64);
                v = ld_relaxed_u64b(&st[tp]);
            }
            part += (unsigned)v & 0x3FFFFFFFu;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        if (lane == 0) s_warp[w] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned pre = 0;
            for (int i = 0; i < SEL_THREADS / 32; ++i) pre += s_warp[i];
            s_pre = pre;
            if (tile == ntiles - 1) ctrl->nblur = pre + tile_cnt;
        }
        __syncthreads();
        unsigned o = s_pre + excl;
#pragma unroll
        for (int q = 0; q < SEL_PER_THREAD; ++q) {
            const unsigned i = i0 + q;
            if (i >= n) break;
            if (flags >> q & 1u) {
                const long long j = g.hs + (long long)i;
                b.blur_ord[i] = o;
                b.bk[o] = b.popk[i] & 0x7FFFFFFFu;
                b.bj[o] = (int)j;
                b.bpix[o] = b.ring_pix[(g.base + (unsigned long long)j) & kp.ring_mask];
                ++o;
            } else {
                b.blur_ord[i] = NOBLUR;
            }
        }
        __syncthreads();
    }
}

// blur ordinal attached to a popped event of this batch (NOBLUR if none)
__device__ __forceinline__ unsigned blur_of(const Bufs &b, const S1Geo &g, long long j)
{
    if (j < g.hs || j >= g.he) return NOBLUR;
    return b.blur_ord[j - g.hs];
}

// per pixel list: latest blur attached to events at positions <= p.  Each pixel with
// batch events owns the list plist[info.y .. info.y + info.z); a thread starting at the
// list's first position walks it.
__global__ void __launch_bounds__(256) k_s1_lb(KParams kp, Bufs b)
{
    PDL_ENTRY();
    const S1Geo g = s1_geo(b.ctrl);
    for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < g.m; p += gridDim.x * blockDim.x) {
        const unsigned pix = b.ring_pix[(g.base + b.plist[p]) & kp.ring_mask];
        const int4 info = b.s1_info[pix];
        if ((unsigned)info.y != p) continue;
        unsigned run = info.w > -0x40000000 ? blur_of(b, g, info.w) : NOBLUR;
        int run_ord = -1;  // the blur of the event before the batch
        for (int q = info.y; q < info.y + info.z; ++q) {
            const unsigned bo = blur_of(b, g, (long long)b.plist[q]);
            if (bo != NOBLUR) {
                run = bo;
                run_ord = q - info.y;
            }
            b.lbl[q] = run;
            b.lbo[q] = run_ord;
        }
    }
}

struct Tap {
    float lnb;   // L of the pixel without this batch's blurs, at the blur's step
    unsigned bl; // latest earlier blur of the pixel in this batch (NOBLUR if none)
    int m;       // events of the pixel since that blur
};

__device__ __forceinline__ Tap resolve(const KParams &kp, const Bufs &b, const S1Geo &g, unsigned n,
                                       unsigned ks, unsigned s)
{
    Tap t;
    t.bl = NOBLUR;
    t.m = 0;
    int ord_e = -1;
    int ord_b = -1;  // ordinal of the tap's blur event in its pixel's list (-1: before the batch)
    long long prev;
    const int4 info = b.s1_info[n];
    bool found = false;
    if ((unsigned)info.x == g.batch_no) {
        int lo = 0, hi = info.z - 1, f = -1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            if (b.plist[info.y + mid] <= ks) { f = mid; lo = mid + 1; }
            else hi = mid - 1;
        }
        prev = info.w;
        if (f >= 0) {
            found = true;
            const int p = info.y + f;
            const long long e = (long long)b.plist[p];
            t.lnb = b.plnb[p];
            ord_e = f;
            const unsigned own = blur_of(b, g, e);
            if (own != NOBLUR && own < s) {
                t.bl = own;
                ord_b = f;
            } else if (f > 0) {
                t.bl = b.lbl[p - 1];
                ord_b = b.lbo[p - 1];
            } else {
                t.bl = prev > -0x40000000 ? blur_of(b, g, prev) : NOBLUR;
            }
        } else {
            t.lnb = b.s1_linit[n];
        }
    } else {
        const unsigned long long lp = b.last_pix[n];
        prev = lp == NONE64 ? -0x7FFFFFFFll - 1 : (long long)(lp - g.base);
        t.lnb = b.L[n];
    }
    if (!found && prev > -0x40000000) {
        const unsigned own = blur_of(b, g, prev);
        if (own != NOBLUR && own < s) t.bl = own;
    }
    if (t.bl != NOBLUR) t.m = ord_e - ord_b;
    return t;
}

__global__ void __launch_bounds__(128) k_s1_blur(KParams kp, Bufs b)
{
    PDL_ENTRY();
    Ctrl *ctrl = b.ctrl;
    const S1Geo g = s1_geo(ctrl);
    const unsigned nb = ctrl->nblur;
    const unsigned lane = threadIdx.x & 31;
    const float wt[3] = {1.f, 2.f, 1.f};
    for (;;) {
        unsigned s0 = 0;
        if (lane == 0) s0 = atomicAdd(&ctrl->blur_ticket, 32u);
        s0 = __shfl_sync(0xFFFFFFFFu, s0, 0);
        if (s0 >= nb) break;
        const unsigned s = s0 + lane;
        const bool active = s < nb;
        Tap tp[9];
        float wsum = 0.f, lself = 0.f;
        if (active) {
            const unsigned ks = b.bk[s];
            const unsigned p = b.bpix[s];
            const int x = (int)(p % kp.W), y = (int)(p / kp.W);
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int dx = t % 3 - 1, dy = t / 3 - 1;
                const int xx = x + dx, yy = y + dy;
                if (xx < 0 || yy < 0 || xx >= (int)kp.W || yy >= (int)kp.H) {
                    tp[t].lnb = 0.f; tp[t].bl = NOBLUR; tp[t].m = -1;  // m = -1: outside
                    continue;
                }
                tp[t] = resolve(kp, b, g, (unsigned)(yy * (int)kp.W + xx), ks, s);
                wsum += wt[dx + 1] * wt[dy + 1];
            }
            lself = tp[4].lnb;
        }
        bool done = !active;
        unsigned spins = 0;
        float dv[9];  // published D of each tap's blur (the value and its flag in one word)
        float cm[9];  // beta^m of each tap's blur, ready before the wait
        unsigned pending = 0;  // taps whose blur has not been seen published yet
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            dv[t] = 0.f;
            cm[t] = 0.f;
            if (active && tp[t].bl != NOBLUR) {  // (the taps of a lane without a blur are unset)
                pending |= 1u << t;
                cm[t] = beta_pow(kp, b.beta_pow, tp[t].m);
            }
        }
        while (__any_sync(0xFFFFFFFFu, !done)) {
            if (!done) {
                // every pending tap at once (independent relaxed loads, one round trip):
                // a published word holds its tag and its value and never changes
#pragma unroll
                for (int t = 0; t < 9; ++t)
                    if (pending >> t & 1u) {
                        const unsigned long long v = ld_relaxed_u64b(&b.bval[tp[t].bl]);
                        if ((unsigned)(v >> 32) == g.batch_no) {
                            dv[t] = __uint_as_float((unsigned)v);
                            pending &= ~(1u << t);
                        }
                    }
                const bool ready = pending == 0;
                if (ready) {
                    float acc = 0.f;
#pragma unroll
                    for (int t = 0; t < 9; ++t) {
                        const int dx = t % 3 - 1, dy = t / 3 - 1;
                        // taps outside the sensor hold lnb = 0 and no blur: they add 0
                        float v = tp[t].lnb;
                        if (tp[t].bl != NOBLUR) v += cm[t] * dv[t];
                        acc += wt[dx + 1] * wt[dy + 1] * v;
                    }
                    const float D = acc / wsum - lself;
                    // the word is the whole message (readers take tag and value from it):
                    // no ordering with other stores is needed
                    st_relaxed_u64b(&b.bval[s], ((unsigned long long)g.batch_no << 32) | __float_as_uint(D));
                    done = true;
                } else if (++spins > SPIN_LIMIT) {
                    atomicOr(&ctrl->error, ERR_S1_WAIT);
                    done = true;
                } else {
                    __nanosleep(32);  // back off: polls compete with the stores they wait for
                }
            }
        }
    }
}

// final L of the pixels a blur of this batch changed
__global__ void __launch_bounds__(256) k_s1_apply(KParams kp, Bufs b)
{
    PDL_ENTRY();
    const S1Geo g = s1_geo(b.ctrl);
    const unsigned nb = b.ctrl->nblur;
    for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < g.m; p += gridDim.x * blockDim.x) {
        const unsigned pix = b.ring_pix[(g.base + b.plist[p]) & kp.ring_mask];
        const int4 info = b.s1_info[pix];
        if ((unsigned)info.y != p) continue;
        const int last = info.y + info.z - 1;
        const unsigned bl = b.lbl[last];
        if (bl == NOBLUR) continue;
        const int ord_b = b.lbo[last];
        b.L[pix] = b.plnb[last] + beta_pow(kp, b.beta_pow, info.z - 1 - ord_b) * __uint_as_float((unsigned)__ldcg(&b.bval[bl]));
    }
    // pixels without events in this batch whose previous event was popped (and blurred) now
    for (unsigned s = blockIdx.x * blockDim.x + threadIdx.x; s < nb; s += gridDim.x * blockDim.x) {
        if (b.bj[s] >= 0) continue;
        const unsigned pix = b.bpix[s];
        if ((unsigned)b.s1_info[pix].x == g.batch_no) continue;
        b.L[pix] += __uint_as_float((unsigned)__ldcg(&b.bval[s]));
    }
}

cudaError_t launch_s1(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 5;
    if (cudaError_t e_ = launch_pdl(k_s1_pops, grid_for(kp, 4), 256, 0, s, kp, b)) return e_;
    if (cudaError_t e_ = launch_pdl(k_s1_select, grid_for(kp, 2), SEL_THREADS, 0, s, kp, b)) return e_;
    if (cudaError_t e_ = launch_pdl(k_s1_lb, grid_for(kp, 4), 256, 0, s, kp, b)) return e_;
    // as many blur warps as 64 registers a thread allow (32 per SM): more blurs in flight
    if (cudaError_t e_ = launch_pdl(k_s1_blur, grid_for(kp, 8), 128, 0, s, kp, b)) return e_;
    if (cudaError_t e_ = launch_pdl(k_s1_apply, grid_for(kp, 4), 256, 0, s, kp, b)) return e_;
    return cudaGetLastError();
}

}  // namespace fibar
