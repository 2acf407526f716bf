// Ingest: decode packed events, cut the read-out prefix, compact, and sort by tile.
//
// k_decode  - one pass over the pending records (a carry buffer of records left
//             pending by the previous read-out, then the pushed packets in order).
//             Each record is read once with a 16-byte load.  Tiles of 4096 records
//             publish (events kept, position of the first record whose time stamp is
//             later than the read-out time); each tile reduces its predecessors' values
//             in order to find its output offset and whether it lies past the cut: the applied
//             set is the longest prefix with t <= t_read (Eq. 4's t_k <= t), minus
//             out-of-range records, which are counted and skipped.  Kept events get
//             consecutive batch indices k and a 64-bit sort record
//             (tile id << 32 | k << 3 | sub-pixel << 1 | OFF).  Records after the
//             cut are copied to the other carry buffer.
// k_sort_*  - stable LSD radix sort of the records by tile id, digits of up to 9 bits
//             (one histogram kernel for all digits, then one kernel per digit whose tiles
//             publish their digit counts; tile prefixes come from group totals of 32
//             tiles plus the earlier tiles of the own group, with no look-back chains),
//             so that every 2x2 tile's events end up contiguous and in arrival order.
#include "fibar_internal.cuh"

namespace fibar {

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Bulk asynchronous copies (TMA) into shared memory, completing on an mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned phase)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(phase)
                 : "memory");
    return ok != 0;
}
// Bounded wait for an mbarrier phase; false (and the error flag) if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned phase, Ctrl *ctrl, unsigned flag)
{
    unsigned spins = 0;
    while (!mbar_try_wait(bar, phase)) {
        if (++spins > TMA_SPIN_LIMIT) {
            atomicOr(&ctrl->error, flag);
            return false;
        }
    }
    return true;
}

// Block-wide exclusive scan of one value per thread (blockDim.x == 256).
__device__ __forceinline__ unsigned block_excl_scan256(unsigned v, unsigned *s_warp, unsigned *total)
{
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned t = threadIdx.x < 8 ? s_warp[threadIdx.x] : 0u;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            unsigned y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        if (threadIdx.x < 8) s_warp[threadIdx.x + 8] = t;  // inclusive warp prefix
    }
    __syncthreads();
    unsigned warp_excl = w ? s_warp[8 + w - 1] : 0u;
    *total = s_warp[15];
    unsigned r = warp_excl + x - v;
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------------
// decode
// ---------------------------------------------------------------------------------
constexpr unsigned S_NONE = 0x7FFFFFFFu;
constexpr unsigned NOREC = 0xFFFFFFFFu;

struct DAgg {
    unsigned s;  // absolute position of the first late record, S_NONE if none
    unsigned c;  // kept events, counted only before any late record
};

__device__ __forceinline__ DAgg dcombine(DAgg a, DAgg b)  // a precedes b
{
    if (a.s != S_NONE) return a;
    return DAgg{b.s, a.c + b.c};
}

__device__ __forceinline__ unsigned long long dpack(unsigned flag, DAgg a)
{
    return ((unsigned long long)flag << 62) | ((unsigned long long)a.s << 31) | a.c;
}

// Segment holding record pos (pos >= carry_n): the last segment starting at or before it.
__device__ __forceinline__ int seg_of(unsigned nseg, const unsigned *s_start, unsigned pos)
{
    int lo = 0, hi = (int)nseg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s_start[mid] <= pos) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Shared-memory index of tile position r: one word of padding per DEC_PER_THREAD, so that
// a thread's run of consecutive positions (thread t at DEC_PER_THREAD t) and a warp's 32
// consecutive positions both fall in distinct banks.
__device__ __forceinline__ unsigned dpad(unsigned r) { return r + r / DEC_PER_THREAD; }

// With a one-pass sort the decode also counts the kept records per bucket (the sort's
// only digit) and the block that completes the last tile turns the counts into the
// sort's digit offsets and the walk's bucket starts (otherwise k_sort_hist does).
struct DecHist {
    unsigned *ghist, *gbase, *bucket_start;  // ghist == nullptr: off
    unsigned *order;                         // buckets by decreasing size, for the walk
    unsigned nbuckets, lb;
};

__global__ void __launch_bounds__(DEC_THREADS)
k_decode(KParams kp, const __grid_constant__ SegTable T, const SegTable *Tdev, Ctrl *ctrl,
         unsigned long long *status, unsigned long long *rec_out, unsigned *ring_pix, DecHist dh)
{
    PDL_ENTRY();
    // the read-out's packets: the launch's own table, or (a captured read-out chain) the
    // table written to device memory before the chain runs
    const SegTable &TS = Tdev ? *Tdev : T;
    const unsigned nseg = TS.nseg, carry_slot = TS.carry_slot;
    const int4 *const carry = TS.carry;
    int4 *const carry_out = TS.carry_out;
    const unsigned long long t_read = TS.t_read;
    extern __shared__ __align__(128) int4 s_rec[];  // the tile's records (DEC_TILE)
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ unsigned s_start[MAXSEG + 1];
    __shared__ const int4 *s_ptr[MAXSEG];
    __shared__ unsigned s_info[DEC_TILE + DEC_TILE / DEC_PER_THREAD];  // indexed by dpad()
    __shared__ unsigned s_pix[DEC_TILE + DEC_TILE / DEC_PER_THREAD];
    __shared__ unsigned s_warp[16];
    __shared__ unsigned s_tile, s_vmin, s_pre_s, s_pre_c, s_drop;
    __shared__ unsigned s_red_s[DEC_THREADS / 32], s_red_c[DEC_THREADS / 32];
    __shared__ unsigned s_hb[RADIX];  // kept records per bucket (this tile)
    __shared__ bool s_hlast;

    const unsigned carry_n = ctrl->carry_n[carry_slot];
    if (threadIdx.x == 0) {
        unsigned acc = carry_n;
        for (unsigned i = 0; i < nseg; ++i) {
            s_start[i] = acc;
            s_ptr[i] = TS.ptr[i];
            acc += TS.n[i];
        }
        s_start[nseg] = acc;
        mbar_init(&s_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const unsigned total = s_start[nseg];
    const unsigned ntiles = (total + DEC_TILE - 1) / DEC_TILE;
    unsigned phase = 0;
    const bool hist = dh.ghist != nullptr;
    // digit offsets and bucket starts of the last tile's block (all zero without tiles)
    auto hist_finish = [&]() {
        const unsigned d0 = 2 * threadIdx.x;
        const unsigned v0 = atomicExch(&dh.ghist[d0], 0u), v1 = atomicExch(&dh.ghist[d0 + 1], 0u);
        unsigned tot;
        const unsigned ex = block_excl_scan256(v0 + v1, s_warp, &tot);
        dh.gbase[d0] = ex;
        dh.gbase[d0 + 1] = ex + v0;
        const bool ok0 = d0 < dh.nbuckets, ok1 = d0 + 1 < dh.nbuckets;
        if (ok0) dh.bucket_start[d0] = ex;
        if (ok1) dh.bucket_start[d0 + 1] = ex + v0;
        // the walk's order: buckets by decreasing size, in 64 size classes (a counting
        // sort; the order within a class does not matter, the buckets are independent)
        __syncthreads();
        if (threadIdx.x < 65) s_hb[threadIdx.x] = 0u;
        __syncthreads();
        const unsigned c0 = ok0 ? v0 : 0u, c1 = ok1 ? v1 : 0u;
        const unsigned wmax = __reduce_max_sync(0xFFFFFFFFu, max(c0, c1));
        if ((threadIdx.x & 31) == 0) atomicMax(&s_hb[64], wmax);
        __syncthreads();
        const unsigned mx = max(1u, s_hb[64]);
        const unsigned k0 = 63u - (unsigned)((unsigned long long)c0 * 63u / mx);
        const unsigned k1 = 63u - (unsigned)((unsigned long long)c1 * 63u / mx);
        if (ok0) atomicAdd(&s_hb[k0], 1u);
        if (ok1) atomicAdd(&s_hb[k1], 1u);
        __syncthreads();
        if (threadIdx.x < 32) {
            const unsigned a = s_hb[2 * threadIdx.x], bb = s_hb[2 * threadIdx.x + 1];
            unsigned x = a + bb;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (threadIdx.x >= (unsigned)o) x += y;
            }
            const unsigned excl = x - a - bb;
            s_hb[2 * threadIdx.x] = excl;
            s_hb[2 * threadIdx.x + 1] = excl + a;
        }
        __syncthreads();
        if (ok0) dh.order[atomicAdd(&s_hb[k0], 1u)] = d0;
        if (ok1) dh.order[atomicAdd(&s_hb[k1], 1u)] = d0 + 1;
    };
    if (hist && ntiles == 0) {
        if (blockIdx.x == 0) hist_finish();
        return;
    }

    for (;;) {
        if (threadIdx.x == 0) {
            s_tile = atomicAdd(&ctrl->dec_ticket, 1u);
            s_vmin = S_NONE;
            s_drop = 0;
        }
        if (hist)
            for (unsigned i = threadIdx.x; i < RADIX; i += DEC_THREADS) s_hb[i] = 0u;
        __syncthreads();
        const unsigned tile = s_tile;
        if (tile >= ntiles) break;
        const unsigned pos0 = tile * DEC_TILE;

        // the tile's records into shared memory with bulk copies (TMA), one per contiguous
        // piece of the carry buffer and the packets (16-byte records, 16-byte aligned)
        const unsigned pos1 = min(pos0 + DEC_TILE, total);
        if (threadIdx.x == 0) {
            mbar_expect_tx(&s_bar, (pos1 - pos0) * 16u);
            unsigned p = pos0;
            if (p < carry_n) {
                const unsigned e = min(pos1, carry_n);
                bulk_g2s(s_rec, carry + p, (e - p) * 16u, &s_bar);
                p = e;
            }
            if (p < pos1) {
                int sg = seg_of(nseg, s_start, p);
                while (p < pos1) {
                    while (sg + 1 < (int)nseg && s_start[sg + 1] <= p) ++sg;
                    const unsigned e = min(pos1, s_start[sg + 1]);
                    bulk_g2s(s_rec + (p - pos0), s_ptr[sg] + (p - s_start[sg]), (e - p) * 16u, &s_bar);
                    p = e;
                }
            }
        }
        if (!mbar_wait(&s_bar, phase, ctrl, ERR_DEC_WAIT)) mbar_wait(&s_bar, phase, ctrl, ERR_DEC_WAIT);
        phase ^= 1u;
        unsigned vloc = S_NONE;
#pragma unroll
        for (int i = 0; i < DEC_PER_THREAD; ++i) {
            const unsigned r = i * DEC_THREADS + threadIdx.x;
            const unsigned pos = pos0 + r;
            unsigned info = NOREC;
            if (pos < total) {
                const int4 e = s_rec[r];
                const unsigned x = (unsigned)e.x & 0xFFFFu, y = (unsigned)e.x >> 16;
                const int p = (int)(signed char)(e.y & 0xFF);
                const unsigned long long t =
                    ((unsigned long long)(unsigned)e.w << 32) | (unsigned)e.z;
                if (t > t_read) vloc = min(vloc, r);
                const bool valid = x < kp.W && y < kp.H;
                const unsigned tid_ = valid ? (y >> 1) * kp.tiles_w + (x >> 1) : 0u;
                const unsigned sub = valid ? (((y & 1u) << 1) | (x & 1u)) : 0u;
                info = (valid ? 0x80000000u : 0u) | (tid_ << 3) | (sub << 1) | (p > 0 ? 0u : 1u);
                s_pix[dpad(r)] = valid ? y * kp.W + x : 0u;
            }
            s_info[dpad(r)] = info;
        }
        if (vloc != S_NONE) atomicMin(&s_vmin, vloc);
        __syncthreads();
        const unsigned vfirst = s_vmin;

        // DEC_PER_THREAD contiguous records per thread, in arrival order
        unsigned cnt = 0, drop = 0, keep = 0;
#pragma unroll
        for (int j = 0; j < DEC_PER_THREAD; ++j) {
            const unsigned r = threadIdx.x * DEC_PER_THREAD + j;
            const unsigned info = s_info[dpad(r)];
            if (info != NOREC && r < vfirst) {
                if (info >> 31) { ++cnt; keep |= 1u << j; }
                else ++drop;
            }
        }
        unsigned tile_cnt;
        const unsigned excl = block_excl_scan256(cnt, s_warp, &tile_cnt);
        if (drop) atomicAdd(&s_drop, drop);

        // publish this tile's aggregate, then reduce all predecessors' aggregates in
        // order (each thread a contiguous range, then an ordered tree): no chains
        const DAgg own{vfirst != S_NONE ? pos0 + vfirst : S_NONE, tile_cnt};
        if (threadIdx.x == 0) st_release(&status[tile], dpack(1u, own));
        DAgg acc{S_NONE, 0u};
        {
            const unsigned per = (tile + DEC_THREADS - 1) / DEC_THREADS;
            const unsigned t0 = threadIdx.x * per, t1 = min(tile, t0 + per);
            for (unsigned tp = t0; tp < t1; ++tp) {
                unsigned long long v = ld_relaxed(&status[tp]);
                unsigned spins = 0;
                while ((v >> 62) == 0ull) {
                    if (++spins > SPIN_LIMIT) { atomicOr(&ctrl->error, ERR_DEC_WAIT); break; }
                    __nanosleep(64);  // back off: the polls would compete with the loads awaited
                    v = ld_relaxed(&status[tp]);
                }
                acc = dcombine(acc, DAgg{(unsigned)(v >> 31) & 0x7FFFFFFFu, (unsigned)v & 0x7FFFFFFFu});
            }
        }
        // ordered reduction across the block
        {
            const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned os = __shfl_down_sync(0xFFFFFFFFu, acc.s, o);
                const unsigned oc = __shfl_down_sync(0xFFFFFFFFu, acc.c, o);
                if (lane + o < 32 && (lane & (2 * o - 1)) == 0) acc = dcombine(acc, DAgg{os, oc});
            }
            if (lane == 0) { s_red_s[w] = acc.s; s_red_c[w] = acc.c; }
            __syncthreads();
            if (threadIdx.x == 0) {
                DAgg pre{S_NONE, 0u};
                for (int i = 0; i < DEC_THREADS / 32; ++i) pre = dcombine(pre, DAgg{s_red_s[i], s_red_c[i]});
                s_pre_s = pre.s;
                s_pre_c = pre.c;
                if (tile == ntiles - 1) {
                    const DAgg inc = dcombine(pre, own);
                    const unsigned s = inc.s == S_NONE ? total : inc.s;
                    ctrl->m = inc.c;
                    ctrl->consumed = s;
                    ctrl->carry_n[1 - carry_slot] = total - s;
                }
            }
        }
        __syncthreads();
        const unsigned pre_s = s_pre_s, pre_c = s_pre_c;
        if (pre_s == S_NONE) {
            const unsigned long long base = ctrl->base;
            // compact the kept records in shared memory (each thread moves its own, in
            // order, after all have read theirs), then write them out coalesced
            unsigned my_info[DEC_PER_THREAD], my_pix[DEC_PER_THREAD];
#pragma unroll
            for (int j = 0; j < DEC_PER_THREAD; ++j) {
                my_info[j] = s_info[dpad(threadIdx.x * DEC_PER_THREAD + j)];
                my_pix[j] = s_pix[dpad(threadIdx.x * DEC_PER_THREAD + j)];
            }
            __syncthreads();
            unsigned li = excl;
#pragma unroll
            for (int j = 0; j < DEC_PER_THREAD; ++j) {
                if (keep >> j & 1u) {
                    s_info[dpad(li)] = my_info[j];
                    s_pix[dpad(li)] = my_pix[j];
                    ++li;
                }
            }
            __syncthreads();
            for (unsigned i = threadIdx.x; i < tile_cnt; i += DEC_THREADS) {
                const unsigned k = pre_c + i, info = s_info[dpad(i)];
                rec_out[k] = ((unsigned long long)((info >> 3) & 0x0FFFFFFFu) << 32) |
                             ((unsigned long long)k << 3) | (info & 7u);
                if (hist) atomicAdd(&s_hb[((info >> 3) & 0x0FFFFFFFu) >> dh.lb], 1u);
                if (ring_pix) ring_pix[(base + k) & kp.ring_mask] = s_pix[dpad(i)];
            }
            if (threadIdx.x == 0 && s_drop) atomicAdd(&ctrl->dropped, (unsigned long long)s_drop);
            if (vfirst != S_NONE) {
                const unsigned s = pos0 + vfirst;
                for (int i = 0; i < DEC_PER_THREAD; ++i) {
                    const unsigned r = i * DEC_THREADS + threadIdx.x;
                    const unsigned pos = pos0 + r;
                    if (r >= vfirst && pos < total) carry_out[pos - s] = s_rec[r];
                }
            }
        } else {
            for (int i = 0; i < DEC_PER_THREAD; ++i) {
                const unsigned r = i * DEC_THREADS + threadIdx.x;
                const unsigned pos = pos0 + r;
                if (pos < total) carry_out[pos - pre_s] = s_rec[r];
            }
        }
        if (hist) {
            __syncthreads();
            for (unsigned d = threadIdx.x; d < dh.nbuckets; d += DEC_THREADS)
                if (s_hb[d]) atomicAdd(&dh.ghist[d], s_hb[d]);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) s_hlast = atomicAdd(&ctrl->hist_done, 1u) == ntiles - 1;
            __syncthreads();
            if (s_hlast) {
                __threadfence();
                hist_finish();
                if (threadIdx.x == 0) ctrl->hist_done = 0;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------
// radix sort by tile id (stable)
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_sort_hist(Ctrl *ctrl, const unsigned long long *rec, unsigned passes, unsigned dbits, unsigned lb,
            unsigned nbuckets, unsigned *ghist, unsigned *gbase, unsigned *bcnt, unsigned *bucket_start)
{
    PDL_ENTRY();
    __shared__ unsigned h[SORT_MAX_PASSES][RADIX];
    __shared__ unsigned hb[MAX_BUCKETS];
    __shared__ unsigned s_warp[16];
    __shared__ bool s_last;
    for (unsigned i = threadIdx.x; i < SORT_MAX_PASSES * RADIX; i += blockDim.x) (&h[0][0])[i] = 0;
    for (unsigned i = threadIdx.x; i < nbuckets; i += blockDim.x) hb[i] = 0;
    __syncthreads();
    const unsigned m = ctrl->m;
    const unsigned dmask = (1u << dbits) - 1u;
    // eight records per thread and round, all loads in flight before the counting
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += 8 * stride) {
        unsigned key[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const unsigned i = i0 + u * stride;
            key[u] = i < m ? (unsigned)(rec[i] >> 32) >> lb : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (key[u] == 0xFFFFFFFFu) continue;
            for (unsigned p = 0; p < passes; ++p) atomicAdd(&h[p][(key[u] >> (dbits * p)) & dmask], 1u);
            atomicAdd(&hb[key[u]], 1u);
        }
    }
    __syncthreads();
    for (unsigned p = 0; p < passes; ++p)
        for (unsigned d = threadIdx.x; d < RADIX; d += 256) {
            const unsigned v = h[p][d];
            if (v) atomicAdd(&ghist[p * RADIX + d], v);
        }
    for (unsigned d = threadIdx.x; d < nbuckets; d += 256) {
        const unsigned v = hb[d];
        if (v) atomicAdd(&bcnt[d], v);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctrl->hist_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (unsigned p = 0; p < passes; ++p) {
        // two digits per thread
        const unsigned d0 = 2 * threadIdx.x;
        const unsigned v0 = atomicExch(&ghist[p * RADIX + d0], 0u);
        const unsigned v1 = atomicExch(&ghist[p * RADIX + d0 + 1], 0u);
        unsigned tot;
        const unsigned ex = block_excl_scan256(v0 + v1, s_warp, &tot);
        gbase[p * RADIX + d0] = ex;
        gbase[p * RADIX + d0 + 1] = ex + v0;
    }
    // bucket starts: each thread a contiguous run of buckets
    {
        const unsigned per = (nbuckets + 255) / 256;
        const unsigned b0 = threadIdx.x * per, b1 = min(nbuckets, b0 + per);
        unsigned sum = 0;
        for (unsigned bb = b0; bb < b1; ++bb) sum += __ldcg(&bcnt[bb]);
        unsigned tot;
        unsigned run = block_excl_scan256(sum, s_warp, &tot);
        for (unsigned bb = b0; bb < b1; ++bb) {
            const unsigned v = atomicExch(&bcnt[bb], 0u);
            bucket_start[bb] = run;
            run += v;
        }
    }
    if (threadIdx.x == 0) ctrl->hist_done = 0;
}

__device__ __forceinline__ unsigned ld_acq_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_rel_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// wait (bounded) until *flag == epoch
__device__ __forceinline__ void wait_flag(const unsigned *flag, unsigned epoch, Ctrl *ctrl)
{
    unsigned spins = 0;
    while (ld_acq_u32(flag) != epoch) {
        if (++spins > SPIN_LIMIT) { atomicOr(&ctrl->error, ERR_SORT_WAIT); return; }
        __nanosleep(64);
    }
}

// dynamic shared memory layout of k_sort_pass
struct SortSmem {
    unsigned long long key[SORT_TILE];
    unsigned glast;
    unsigned long long out[SORT_TILE];
    unsigned short rank[SORT_TILE];
    unsigned whist[8][RADIX];
    unsigned tdig[RADIX];
    unsigned gpos[RADIX];
    unsigned warp[16];
    unsigned tile;
};

__global__ void __launch_bounds__(SORT_THREADS)
k_sort_pass(Ctrl *ctrl, const unsigned long long *in, unsigned long long *out, unsigned pass,
            unsigned dbits, unsigned lb, const unsigned *gbase, unsigned *rows, unsigned *rowflag,
            unsigned *gtot, unsigned *gflag, unsigned *gcount)
{
    PDL_ENTRY();
    // flag value of this pass: distinct for every pass of every read-out (the commit
    // counter starts at 1), so that no flag needs clearing between read-outs
    const unsigned epoch = (ctrl->batch_no - 1u) * SORT_MAX_PASSES + 1u + pass;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &S = *reinterpret_cast<SortSmem *>(smem_raw);
    const unsigned m = ctrl->m;
    const unsigned ntiles = (m + SORT_TILE - 1) / SORT_TILE;
    const unsigned shift = 32 + lb + dbits * pass;
    const unsigned dmask = (1u << dbits) - 1u;
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;

    for (;;) {
        if (threadIdx.x == 0) S.tile = atomicAdd(&ctrl->sort_ticket[pass], 1u);
        for (unsigned i = threadIdx.x; i < 8 * RADIX; i += SORT_THREADS) (&S.whist[0][0])[i] = 0;
        __syncthreads();
        const unsigned tile = S.tile;
        if (tile >= ntiles) break;
        const unsigned base = tile * SORT_TILE;
        const unsigned n_here = min((unsigned)SORT_TILE, m - base);
        // asynchronous copies: the whole tile in flight at once
#pragma unroll
        for (int i = 0; i < SORT_PER_THREAD; ++i) {
            const unsigned r = i * SORT_THREADS + threadIdx.x;
            if (r < n_here) {
                const unsigned d = (unsigned)__cvta_generic_to_shared(&S.key[r]);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(in + base + r) : "memory");
            } else {
                S.key[r] = ~0ull;
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
        // stable rank within (warp range, digit): warp w owns records
        // [w * SORT_WARP_RANGE, (w + 1) * SORT_WARP_RANGE)
        for (int q = 0; q < SORT_WARP_RANGE / 32; ++q) {
            const unsigned r = w * SORT_WARP_RANGE + q * 32 + lane;
            const bool valid = r < n_here;
            const unsigned d = valid ? (unsigned)(S.key[r] >> shift) & dmask : RADIX;
            const unsigned peers = warp_peers<10>(d);  // digit < 512, or RADIX (none)
            const unsigned rank = __popc(peers & lt_mask);
            if (valid) S.rank[r] = (unsigned short)(S.whist[w][d] + rank);
            __syncwarp();
            if (valid && rank == 0) S.whist[w][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per-digit exclusive offsets of each warp, the tile's digit counts (2 digits per thread)
        const unsigned d0 = 2 * threadIdx.x;
        unsigned run0 = 0, run1 = 0;
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) {
            const unsigned c0 = S.whist[ww][d0], c1 = S.whist[ww][d0 + 1];
            S.whist[ww][d0] = run0;
            S.whist[ww][d0 + 1] = run1;
            run0 += c0;
            run1 += c1;
        }
        unsigned tot;
        const unsigned tdig = block_excl_scan256(run0 + run1, S.warp, &tot);
        S.tdig[d0] = tdig;
        S.tdig[d0 + 1] = tdig + run0;
        // tile prefix per digit: publish this tile's digit counts; the last tile of each
        // group of LB_GROUP tiles to arrive publishes the group's totals; a tile adds the
        // totals of earlier groups and the counts of earlier tiles of its own group
        unsigned *row = rows + (size_t)tile * RADIX;
        row[d0] = run0;
        row[d0 + 1] = run1;
        __syncthreads();
        const unsigned g = tile / LB_GROUP;
        if (threadIdx.x == 0) {
            __threadfence();
            st_rel_u32(&rowflag[tile], epoch);
            const unsigned gsize = min((unsigned)LB_GROUP, ntiles - g * LB_GROUP);
            const unsigned old = atomicAdd(&gcount[g], 1u);
            S.glast = old == gsize - 1;
            if (S.glast) gcount[g] = 0;
        }
        __syncthreads();
        if (S.glast) {
            // every member has published (it counted itself in after publishing)
            const unsigned gsize = min((unsigned)LB_GROUP, ntiles - g * LB_GROUP);
            unsigned a0 = 0, a1 = 0;
#pragma unroll 8
            for (unsigned t = g * LB_GROUP; t < g * LB_GROUP + gsize; ++t) {
                a0 += __ldcg(&rows[(size_t)t * RADIX + d0]);
                a1 += __ldcg(&rows[(size_t)t * RADIX + d0 + 1]);
            }
            gtot[(size_t)g * RADIX + d0] = a0;
            gtot[(size_t)g * RADIX + d0 + 1] = a1;
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                st_rel_u32(&gflag[g], epoch);
            }
        }
        // wait until the earlier groups' totals and the earlier tiles of this group are
        // published: thread i watches one flag, the block polls them together
        {
            const unsigned nt = tile - g * LB_GROUP;  // earlier tiles of this group (< 32)
            const unsigned *flag = nullptr;
            if (threadIdx.x < nt) flag = &rowflag[g * LB_GROUP + threadIdx.x];
            else if (threadIdx.x >= 32 && threadIdx.x - 32 < g) flag = &gflag[threadIdx.x - 32];
            unsigned spins = 0;
            bool ok = flag == nullptr || ld_acq_u32(flag) == epoch;
            while (!__syncthreads_and(ok)) {
                if (++spins > SPIN_LIMIT) {
                    if (threadIdx.x == 0) atomicOr(&ctrl->error, ERR_SORT_WAIT);
                    break;
                }
                if (!ok) ok = ld_acq_u32(flag) == epoch;
            }
        }
        unsigned pre0 = 0, pre1 = 0;
#pragma unroll 8
        for (unsigned gg = 0; gg < g; ++gg) {
            pre0 += __ldcg(&gtot[(size_t)gg * RADIX + d0]);
            pre1 += __ldcg(&gtot[(size_t)gg * RADIX + d0 + 1]);
        }
#pragma unroll 8
        for (unsigned t = g * LB_GROUP; t < tile; ++t) {
            pre0 += __ldcg(&rows[(size_t)t * RADIX + d0]);
            pre1 += __ldcg(&rows[(size_t)t * RADIX + d0 + 1]);
        }
        S.gpos[d0] = gbase[pass * RADIX + d0] + pre0;
        S.gpos[d0 + 1] = gbase[pass * RADIX + d0 + 1] + pre1;
        __syncthreads();
        // reorder the tile by digit in shared memory
#pragma unroll 4
        for (int i = 0; i < SORT_PER_THREAD; ++i) {
            const unsigned r = i * SORT_THREADS + threadIdx.x;
            if (r < n_here) {
                const unsigned long long k = S.key[r];
                const unsigned dd = (unsigned)(k >> shift) & dmask;
                const unsigned ww = r / SORT_WARP_RANGE;
                S.out[S.tdig[dd] + S.whist[ww][dd] + S.rank[r]] = k;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int i = 0; i < SORT_PER_THREAD; ++i) {
            const unsigned lp = i * SORT_THREADS + threadIdx.x;
            if (lp < n_here) {
                const unsigned long long k = S.out[lp];
                const unsigned dd = (unsigned)(k >> shift) & dmask;
                out[S.gpos[dd] + (lp - S.tdig[dd])] = k;
            }
        }
        __syncthreads();
    }
}

// SM count of each device (0: not looked up yet), for grid sizes in whole waves
static std::atomic<int> g_sms[64];

int grid_for(int mult)
{
    int dev = 0;
    cudaGetDevice(&dev);
    int n = dev >= 0 && dev < 64 ? g_sms[dev].load(std::memory_order_relaxed) : 0;
    if (n <= 0) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
        if (dev >= 0 && dev < 64) g_sms[dev].store(n, std::memory_order_relaxed);
    }
    return n * mult;
}

int grid_for(const KParams &kp, int mult)
{
    const int all = grid_for(1);
    const int sms = kp.grid_sms ? std::min((int)kp.grid_sms, all) : all;
    return sms * mult;
}

cudaError_t launch_decode(const KParams &kp, const Bufs &b, const SegTable &t, unsigned sort_passes,
                          cudaStream_t s, unsigned long long &nl, const SegTable *tdev)
{
    nl += 1;
    static std::atomic<unsigned long long> attr_done{0};
    const int smem = DEC_TILE * (int)sizeof(int4);
    if (cudaError_t e = smem_attr_once(attr_done, k_decode, (size_t)smem)) return e;
    DecHist dh{nullptr, nullptr, nullptr, nullptr, kp.nbuckets, kp.lb};
    if (sort_passes == 1) {
        dh.ghist = b.sort_hist;
        dh.gbase = b.sort_base;
        dh.bucket_start = b.bucket_start;
        dh.order = b.bucket_order;
    }
    if (cudaError_t e_ = launch_pdl(k_decode, grid_for(kp, DEC_BLOCKS_PER_SM), DEC_THREADS, smem, s, kp, t, tdev, b.ctrl, b.dec_status, b.rec[0],
                                    kp.spatial ? b.ring_pix : nullptr, dh)) return e_;
    return cudaGetLastError();
}

cudaError_t launch_sort(const KParams &kp, const Bufs &b, unsigned passes, cudaStream_t s, unsigned long long &nl)
{
    nl += (passes == 1 ? 0 : 1) + passes;  // one pass: the decode counted the digits
    static std::atomic<unsigned long long> attr_done{0};
    const size_t smem = sizeof(SortSmem);
    if (cudaError_t e = smem_attr_once(attr_done, k_sort_pass, smem)) return e;
    const unsigned bucket_bits = kp.key_bits - kp.lb;
    const unsigned dbits = passes ? (bucket_bits + passes - 1) / passes : 1u;
    if (passes != 1)
        if (cudaError_t e_ = launch_pdl(k_sort_hist, grid_for(kp, 2), 256, 0, s, b.ctrl, b.rec[0], passes, dbits, kp.lb,
                                        kp.nbuckets, b.sort_hist, b.sort_base, b.bucket_cnt, b.bucket_start))
            return e_;
    for (unsigned p = 0; p < passes; ++p) {
        if (cudaError_t e_ = launch_pdl(k_sort_pass, grid_for(kp, SORT_BLOCKS_PER_SM), SORT_THREADS, smem, s, b.ctrl, b.rec[p & 1],
                                        b.rec[(p + 1) & 1], p, dbits, kp.lb, b.sort_base, b.sort_rows,
                                        b.sort_rowflag, b.sort_gtot, b.sort_gflag, b.sort_gcount))
            return e_;
    }
    return cudaGetLastError();
}

}  // namespace fibar
