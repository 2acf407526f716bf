// Read-out, batch commit and small bookkeeping kernels.
//
// k_readout_s2 - masked separable 3x3 Gaussian ([1,2,1] x [1,2,1] / 16, weights of taps
//   outside the sensor dropped and the rest renormalised, Sec. 4.2's 3x3 Gaussian):
//   out_i = blur(L)_i where pixel i is stale (had an event, none queued: last_pix < h),
//   L_i elsewhere.  Each block stages a (32+2) x (32+2) halo of L in shared memory and
//   applies the horizontal then the vertical [1,2,1] pass; a thread owns four rows.
// k_commit     - advances the batch base and resets the per-read-out counters.
#include "fibar_internal.cuh"

namespace fibar {

constexpr int RB_X = 32, RB_Y = 8;  // threads per block
constexpr int RB_ROWS = 4;          // rows per thread: a block covers 32 x 32 pixels
constexpr int RB_TY = RB_Y * RB_ROWS;

__global__ void __launch_bounds__(RB_X *RB_Y)
k_readout_s2(KParams kp, const Ctrl *ctrl, const float *__restrict__ L,
             const unsigned long long *__restrict__ last_pix, float *out_arg, float *const *outp)
{
    PDL_ENTRY();
    float *__restrict__ out = outp ? *outp : out_arg;  // outp: a captured chain's descriptor
    __shared__ float t[RB_TY + 2][RB_X + 2];
    __shared__ float hs[RB_TY + 2][RB_X];
    const int x0 = blockIdx.x * RB_X, y0 = blockIdx.y * RB_TY;
    const int W = (int)kp.W, H = (int)kp.H;
    const int lx = threadIdx.x % RB_X, ly = threadIdx.x / RB_X;
    const int x = x0 + lx;
    // the mask inputs first, so that their loads overlap the halo's
    const unsigned long long h = (unsigned long long)ctrl->det.h;
    unsigned long long lp[RB_ROWS];
#pragma unroll
    for (int r = 0; r < RB_ROWS; ++r) {
        const int y = y0 + ly + r * RB_Y;
        lp[r] = (x < W && y < H) ? last_pix[(size_t)y * W + x] : NONE64;
    }
    for (int i = threadIdx.x; i < (RB_TY + 2) * (RB_X + 2); i += RB_X * RB_Y) {
        const int ty = i / (RB_X + 2), tx = i % (RB_X + 2);
        const int gx = x0 + tx - 1, gy = y0 + ty - 1;
        t[ty][tx] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? L[(size_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (RB_TY + 2) * RB_X; i += RB_X * RB_Y) {
        const int ty = i / RB_X, tx = i % RB_X;
        hs[ty][tx] = t[ty][tx] + 2.f * t[ty][tx + 1] + t[ty][tx + 2];
    }
    __syncthreads();
    if (x >= W) return;
    const float wx = 4.f - (x == 0 ? 1.f : 0.f) - (x == W - 1 ? 1.f : 0.f);
#pragma unroll
    for (int r = 0; r < RB_ROWS; ++r) {
        const int ty = ly + r * RB_Y, y = y0 + ty;
        if (y >= H) break;
        const bool stale = lp[r] != NONE64 && lp[r] < h;
        float v = t[ty + 1][lx + 1];
        if (stale) {
            const float wy = 4.f - (y == 0 ? 1.f : 0.f) - (y == H - 1 ? 1.f : 0.f);
            v = (hs[ty][lx] + 2.f * hs[ty + 1][lx] + hs[ty + 2][lx]) / (wx * wy);
        }
        out[(size_t)y * W + x] = v;
    }
}

__global__ void k_copy(const float4 *__restrict__ in, float4 *out_arg, size_t n4,
                       const float *__restrict__ in1, float *out1_arg, size_t n, float *const *outp)
{
    PDL_ENTRY();
    float4 *__restrict__ out = outp ? reinterpret_cast<float4 *>(*outp) : out_arg;
    float *__restrict__ out1 = outp ? *outp : out1_arg;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
        out[i] = in[i];
    const size_t tail = n4 * 4;
    if (blockIdx.x == 0 && threadIdx.x < n - tail) out1[tail + threadIdx.x] = in1[tail + threadIdx.x];
}

// After the last kernel of a read-out: base += m, reset tickets and look-back status.
__global__ void k_commit(Ctrl *ctrl, unsigned long long *dec_status, size_t n_status, int next_carry_slot,
                         unsigned *snap, const ReadDesc *d)
{
    PDL_ENTRY();
    // a captured chain: the slot follows from the descriptor's table
    if (d) next_carry_slot = 1 - (int)d->t.carry_slot;
    for (size_t i = threadIdx.x; i < n_status; i += blockDim.x) dec_status[i] = 0ull;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (ctrl->m > 0) {
            // the queue's growth over this batch (the detector ran: h_prev is the h at
            // the batch start), from which the next batch's window band drifts
            const long long q0 = (long long)(ctrl->base - (unsigned long long)ctrl->h_prev);
            const long long q1 = (long long)(ctrl->base + ctrl->m - (unsigned long long)ctrl->det.h);
            ctrl->grow_num = q1 - q0;
            ctrl->grow_den = ctrl->m;
        }
        ctrl->base += ctrl->m;
        ctrl->m = 0;
        ctrl->band_mode = 0;
        ctrl->dec_ticket = 0;
        for (int p = 0; p < SORT_MAX_PASSES; ++p) ctrl->sort_ticket[p] = 0;
        ctrl->unmerged = 0;
        ctrl->s1_blurs += ctrl->nblur;
        ctrl->nblur = 0;
        ctrl->blur_ticket = 0;
        ctrl->sel_ticket = 0;
        ctrl->walk_ticket = 0;
        ctrl->p2_count = 0;
        ctrl->batch_no += 1;
        // the carry slot just consumed becomes the output slot of the next decode
        ctrl->carry_n[1 - next_carry_slot] = 0;
        // for the host: the records left pending and the error flags, then (ordered after
        // them) this commit's number
        snap[0] = ctrl->carry_n[next_carry_slot];
        snap[2] = ctrl->error;
        __threadfence_system();
        *(volatile unsigned *)&snap[1] = ctrl->batch_no - 1u;
        if (d && d->stamp) {
            unsigned long long ns;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
            *(volatile unsigned long long *)d->stamp = ns;
        }
    }
}

// The bounded wait of the pipeline's look-back and dataflow kernels, on a flag that
// nothing sets: after max_spins polls (with the same back-off) it records ERR_PROBE_WAIT
// in the error flags and returns, as a wait that gives up does.
__global__ void k_probe_wait(Ctrl *ctrl, const unsigned *flag, unsigned max_spins)
{
    if (threadIdx.x != 0) return;
    unsigned spins = 0;
    while (*(volatile const unsigned *)flag == 0u) {
        if (++spins > max_spins) {
            atomicOr(&ctrl->error, ERR_PROBE_WAIT);
            return;
        }
        __nanosleep(64);
    }
}

__global__ void k_init(KParams kp, Ctrl *ctrl)
{
    PDL_ENTRY();
    if (threadIdx.x != 0) return;
    ctrl->base = 0;
    ctrl->dropped = 0;
    ctrl->m = 0;
    ctrl->consumed = 0;
    ctrl->carry_n[0] = ctrl->carry_n[1] = 0;
    ctrl->dec_ticket = 0;
    for (int p = 0; p < SORT_MAX_PASSES; ++p) ctrl->sort_ticket[p] = 0;
    ctrl->hist_done = 0;
    ctrl->cnt_done = 0;
    ctrl->error = 0;
    ctrl->unmerged = 0;
    ctrl->fixups = 0;
    ctrl->unmerged_total = ctrl->pass2_steps = ctrl->fix_steps = ctrl->s1_blurs = 0;
    ctrl->big_pops = ctrl->ring_misses = 0;
    ctrl->walk_pieces = ctrl->scan_pieces = 0;
    ctrl->p2_count = 0;
    ctrl->batch_no = 1;
    ctrl->h_prev = 0;
    ctrl->grow_num = 0;
    ctrl->grow_den = 0;
    ctrl->band_mode = 0;
    ctrl->recenters = 0;
    ctrl->nblur = 0;
    ctrl->blur_ticket = 0;
    ctrl->sel_ticket = 0;
    ctrl->walk_ticket = 0;
    ctrl->det.h = 0;
    ctrl->det.nap = 0;
    ctrl->det.nat = 0;
    ctrl->det.X = kp.q_min;  // overwritten by the host with q_init
    ctrl->det.Y = 1;
}

// Debug: per-pixel count of queued events, cnt[pix(j)] += 1 for j in [h, base).
__global__ void k_debug_counts(KParams kp, const Ctrl *ctrl, const unsigned *ring_pix, unsigned *cnt)
{
    PDL_ENTRY();
    const unsigned long long h = (unsigned long long)ctrl->det.h, k = ctrl->base;
    for (unsigned long long j = h + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ring_pix[j & kp.ring_mask]], 1u);
}

cudaError_t launch_init(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl)
{
    nl += 1;
    if (cudaError_t e_ = launch_pdl(k_init, 1, 32, 0, s, kp, b.ctrl)) return e_;
    return cudaGetLastError();
}

cudaError_t launch_readout(const KParams &kp, const Bufs &b, float *out, cudaStream_t s,
                           unsigned long long &nl, float *const *outp)
{
    nl += 1;
    if (kp.spatial && kp.blur_mode >= 1) {  // S2, and the learned fill's Gaussian fallback
        dim3 grid((kp.W + RB_X - 1) / RB_X, (kp.H + RB_TY - 1) / RB_TY);
        if (cudaError_t e_ = launch_pdl(k_readout_s2, grid, RB_X * RB_Y, 0, s, kp, b.ctrl, b.L, b.last_pix, out, outp))
            return e_;
    } else {
        const size_t n = kp.npix;
        // a captured chain's output (outp) is 16-byte aligned by contract
        const bool aligned = outp || ((uintptr_t)out & 15) == 0;
        if (aligned) {
            const size_t n4 = n / 4;
            if (cudaError_t e_ = launch_pdl(k_copy, grid_for(kp, 4), 256, 0, s, (const float4 *)b.L, (float4 *)out, n4,
                                            b.L, out, n, outp))
                return e_;
        } else {
            nl -= 1;
            return cudaMemcpyAsync(out, b.L, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_probe_wait(const Bufs &b, const unsigned *flag, unsigned max_spins, cudaStream_t s,
                              unsigned long long &nl)
{
    nl += 1;
    k_probe_wait<<<1, 32, 0, s>>>(b.ctrl, flag, max_spins);
    return cudaGetLastError();
}

cudaError_t launch_commit(const KParams &kp, const Bufs &b, int next_carry_slot, cudaStream_t s,
                          unsigned long long &nl, const ReadDesc *d)
{
    nl += 1;
    (void)kp;
    if (cudaError_t e_ = launch_pdl(k_commit, 1, 256, 0, s, b.ctrl, b.dec_status, b.max_dec_tiles, next_carry_slot,
                                    b.snap, d)) return e_;
    return cudaGetLastError();
}

cudaError_t launch_debug_counts(const KParams &kp, const Bufs &b, unsigned int *cnt, cudaStream_t s,
                                unsigned long long &nl)
{
    nl += 1;
    if (cudaError_t e_ = launch_pdl(k_debug_counts, grid_for(kp, 2), 256, 0, s, kp, b.ctrl, b.ring_pix, cnt)) return e_;
    return cudaGetLastError();
}

}  // namespace fibar
