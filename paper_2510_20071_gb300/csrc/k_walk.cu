// Tile walk: one thread per 2x2 tile that has events in the batch.
//
// After the stable sort by tile id, each tile's events are contiguous and in arrival
// order.  The thread owning a tile keeps the four pixels' state in registers and walks
// the tile's events once:
//   - temporal filter of the event's pixel (Sec. 4.1): Eq. 7 (EMA of the increment
//     C_p p), Eq. 6 with the updated average, Eq. 10; FP32 state;
//   - links for the stale-pixel detector: distance to the previous event of the same
//     pixel (dP) and of the same tile (dT) for this event, and, in the event ring, the
//     distance to the next one (nP, nT) for the previous event, including events of
//     earlier batches that are still inside the live part of the ring.
// The active event queue of Sec. 4.2 is the index window [h, k]; with these links a
// push activates a pixel iff dP > k - h, and popping event j deactivates it iff
// nP(j) > k - j (likewise for tiles with dT, nT), so the detector never touches a
// per-pixel counter.
#include "fibar_internal.cuh"

namespace fibar {

__device__ __forceinline__ unsigned sat_dist(unsigned long long later, unsigned long long earlier)
{
    const unsigned long long d = later - earlier;
    return d >= SAT ? SAT : (unsigned)d;
}

template <bool kLinks, bool kS1>
__global__ void __launch_bounds__(256)
k_walk(KParams kp, Bufs b, const unsigned long long *srt)
{
    PDL_ENTRY();
    Ctrl *ctrl = b.ctrl;
    unsigned *ring_np = (unsigned *)b.ring_npt;
    const unsigned m = ctrl->m;
    const unsigned long long base = ctrl->base;
    const int batch_no = (int)ctrl->batch_no;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const unsigned long long r0 = srt[i];
        const unsigned key = (unsigned)(r0 >> 32);
        if (i > 0 && (unsigned)(srt[i - 1] >> 32) == key) continue;

        const unsigned tx = key % kp.tiles_w, ty = key / kp.tiles_w;
        const unsigned x0 = 2 * tx, y0 = 2 * ty;
        unsigned pix[4];
        bool ok[4];
        float pb[4], lv[4], l0[4];
        unsigned long long lp[4], lp0[4];
        bool hit[4];
        unsigned off[4], ord[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const unsigned x = x0 + (s & 1), y = y0 + (s >> 1);
            ok[s] = x < kp.W && y < kp.H;
            pix[s] = ok[s] ? y * kp.W + x : 0u;
            pb[s] = ok[s] ? b.pbar[pix[s]] : 0.f;
            lv[s] = ok[s] ? b.L[pix[s]] : 0.f;
            l0[s] = lv[s];
            lp[s] = ok[s] ? b.last_pix[pix[s]] : NONE64;
            lp0[s] = lp[s];
            hit[s] = false;
            off[s] = 0;
            ord[s] = 0;
        }
        if (kS1) {
            // per-pixel lists inside the tile's range [i, end): pixel s first, in order
            unsigned cnt[4] = {0, 0, 0, 0};
            for (unsigned j = i; j < m; ++j) {
                const unsigned long long r = j == i ? r0 : srt[j];
                if ((unsigned)(r >> 32) != key) break;
                const int s = (int)(r >> 1) & 3;
#pragma unroll
                for (int q = 0; q < 4; ++q) cnt[q] += (q == s);
            }
            off[0] = i;
            off[1] = i + cnt[0];
            off[2] = off[1] + cnt[1];
            off[3] = off[2] + cnt[2];
        }
        unsigned long long lt = b.last_tile[key];
        const unsigned long long live_lo = base > kp.live ? base - kp.live : 0ull;

        for (unsigned j = i; j < m; ++j) {
            const unsigned long long r = j == i ? r0 : srt[j];
            if ((unsigned)(r >> 32) != key) break;
            const unsigned k = (unsigned)(r >> 3) & 0x1FFFFFFFu;
            const int s = (int)(r >> 1) & 3;
            const bool off_ev = r & 1u;
            const unsigned long long g = base + k;
            // the four pixels' values live in registers: select by s without local memory
            unsigned long long lps = lp[0];
            float pbs = pb[0], lvs = lv[0];
#pragma unroll
            for (int q = 1; q < 4; ++q)
                if (q == s) { lps = lp[q]; pbs = pb[q]; lvs = lv[q]; }
            if (kLinks) {
                unsigned dP = SAT, dT = SAT;
                if (lps != NONE64) {
                    dP = sat_dist(g, lps);
                    if (lps >= live_lo) ring_np[2 * (lps & kp.ring_mask)] = dP;
                }
                if (lt != NONE64) {
                    dT = sat_dist(g, lt);
                    if (lt >= live_lo) ring_np[2 * (lt & kp.ring_mask) + 1] = dT;
                }
                b.dpt[k] = make_uint2(dP, dT);
                unsigned ps = pix[0];
#pragma unroll
                for (int q = 1; q < 4; ++q)
                    if (q == s) ps = pix[q];
                b.ring_pix[g & kp.ring_mask] = ps;
            }
            lt = g;
            // Eqs. 2-3: increment C_p p; Eq. 7 then Eq. 6 (updated average) and Eq. 10
            const float inc = off_ev ? -kp.c_off : kp.c_on;
            pbs = kp.a * pbs + kp.oma * inc;
            lvs = kp.b * lvs + kp.g * (inc - pbs);
            if (kS1) {
                unsigned os = ord[0], ps0 = off[0];
#pragma unroll
                for (int q = 1; q < 4; ++q)
                    if (q == s) { os = ord[q]; ps0 = off[q]; }
                b.plist[ps0 + os] = k;
                b.plnb[ps0 + os] = lvs;
                b.epos[k] = os;
#pragma unroll
                for (int q = 0; q < 4; ++q) ord[q] += (q == s);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q == s) { lp[q] = g; pb[q] = pbs; lv[q] = lvs; hit[q] = true; }
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!hit[s]) continue;
            b.pbar[pix[s]] = pb[s];
            b.L[pix[s]] = lv[s];
            b.last_pix[pix[s]] = lp[s];
            if (kLinks) ring_np[2 * (lp[s] & kp.ring_mask)] = SAT;
            if (kS1) {
                long long prev = -0x7FFFFFFFll - 1;  // no earlier event
                if (lp0[s] != NONE64) {
                    const long long rel = (long long)(lp0[s] - base);
                    prev = rel < -0x40000000ll ? -0x40000000ll : rel;
                }
                b.s1_info[pix[s]] = make_int4(batch_no, (int)off[s], (int)ord[s], (int)prev);
                b.s1_linit[pix[s]] = l0[s];
            }
        }
        b.last_tile[key] = lt;
        if (kLinks) ring_np[2 * (lt & kp.ring_mask) + 1] = SAT;
    }
}

cudaError_t launch_walk(const KParams &kp, const Bufs &b, const unsigned long long *sorted,
                        cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    cudaError_t e;
    if (kp.spatial && kp.blur_mode == 0)
        e = launch_pdl(k_walk<true, true>, grid_for(8), 256, 0, s, kp, b, sorted);
    else if (kp.spatial)
        e = launch_pdl(k_walk<true, false>, grid_for(8), 256, 0, s, kp, b, sorted);
    else
        e = launch_pdl(k_walk<false, false>, grid_for(8), 256, 0, s, kp, b, sorted);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace fibar
