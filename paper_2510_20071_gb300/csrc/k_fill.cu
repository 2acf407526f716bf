// Learned stale-pixel fill: a 3-layer 3x3 convolutional network replaces the 3x3
// Gaussian at stale pixels (the read-out's masked fill).  The paper fills a pixel that
// went stale with an isotropic 3x3 Gaussian (Sec. 4.2) and, in its limitations section,
// names what that blur ignores (the gradient's magnitude and direction) and leaves more
// elaborate fills to GPUs; this is one such fill.
//
// Network (inputs per pixel: x0 = L, the filter output of Eq. 10, and x1 = the activity
// age min(4, (k - last) / q), k the events applied, last the pixel's last event, q the
// queue length; the queue of Sec. 4.2 is the window [k - q, k)):
//   a1 = relu(b1 + W1 * bf16(x))   2 -> 16 channels
//   a2 = relu(b2 + W2 * bf16(a1))  16 -> 16
//   y  = b3 + W3 * bf16(a2)        16 -> 1
//   out = y at stale pixels (had an event, none queued), L elsewhere
// ("*" a 3x3 cross-correlation with zero padding at the image border).  Every layer is a
// tcgen05.mma kind::f16 contraction: BF16 weights and inputs, FP32 accumulation in TMEM.
//
// Inference kernel (k_fill): persistent, one CTA of 512 threads per SM, units of 8 output
// rows x 124 output columns, so that every layer's rows are 128 pixels (the MMA's M).  Per
// unit: the inputs of 14 x 130 pixels go to shared memory as BF16 in the tensor cores'
// canonical K-major layout without swizzle (one 16-byte row per pixel: L, age and six
// zeros; the second K half of every input row is a shared block of zeros); each layer is
// 9 MMAs of 128 x 16 x 16 per output row (tap (dy, dx): the input row r + dy read from
// pixel dx on, i.e. the descriptor's start moved by dx rows), 108 + 90 + 72 per unit, issued
// tap by tap across the rows (consecutive MMAs never share an accumulator) by one thread
// into its own TMEM columns and completed through tcgen05.commit on an
// mbarrier (bounded wait); the epilogues read TMEM with tcgen05.ld (lane = pixel), add the
// bias, apply ReLU and store the next layer's BF16 tile (zero outside the image); the last
// one writes the image.  conv3 has one real output: its B operand is padded to N = 16.
//
// Training (k_fill_train, k_fill_adam): one CTA per 24 x 24 crop runs the forward pass,
// the loss gradient over the crop's interior stale pixels (the 7 x 7 receptive field
// inside the crop) and the backward pass in shared memory on CUDA cores (FP32), and
// adds its weight gradients to a global sum; the Adam step divides by the number of
// loss pixels and updates the FP32 master weights.
#include <math.h>
#include <string.h>

#include "fibar_internal.cuh"

namespace fibar {

constexpr int FL_R = 8;            // output rows per unit
constexpr int FL_OC = 124;         // output columns per unit
constexpr int FL_M = 128;          // pixels per MMA (M): a1 columns, and a2 / output columns with halo
constexpr int FL_C = FL_M + 2;     // allocated columns of every tile (an MMA reads pixels dx .. dx + 127)
constexpr int FL_A2R = FL_R + 2;   // a2 rows
constexpr int FL_A1R = FL_R + 4;   // a1 rows
constexpr int FL_XR = FL_R + 6;    // input rows
constexpr int FL_THREADS = 512;
constexpr int FL_XN = FL_XR * FL_C;                         // input positions per unit
constexpr int FL_XITER = (FL_XN + FL_THREADS - 1) / FL_THREADS;
constexpr unsigned FL_TMEM_COLS = 512;                      // one CTA per SM (shared memory)
// Each MMA multiplies one input row (shifted by dx) by the three dy taps at once (N = 48):
// its three 16-column blocks are the accumulators of output rows j - 2, j - 1 and j, so
// output row r's accumulator sits at column t0 + 16 (r + 2) (rows -2 and -1 and the last
// two are scratch).  TMEM columns: conv1 16 x 16 = 256, conv2 14 x 16 = 224; conv3 (12 x 16)
// reuses conv1's, which its epilogue has read by then.
constexpr unsigned FL_T1 = 0, FL_T2 = 256, FL_T3 = 0;
constexpr unsigned FL_PLANE = FL_C * 16;                    // one K half (8 channels) of a tile row
constexpr unsigned FL_ROW2 = 2 * FL_PLANE;                  // a1 / a2 row: both K halves
constexpr float FL_AGE_MAX = 4.f;
constexpr unsigned FL_SPIN_LIMIT = 1u << 20;
constexpr unsigned ERR_FILL_WAIT = 32u;                     // Ctrl::error bit

struct FillSmem {
    unsigned char x[FL_XR * FL_PLANE];    // inputs: channels (L, age, 0 x 6) as BF16, one K half
    unsigned char zero[FL_M * 16];        // the inputs' second K half: zeros
    unsigned char a1[FL_A1R * FL_ROW2];   // canonical K-major layout, no swizzle
    unsigned char a2[FL_A2R * FL_ROW2];
    uint4 w[3][9 * 32];                   // B operands of the three layers
    float lout[FL_R][FL_OC];              // L of the output pixels (FP32: written where not stale)
    unsigned char stale[FL_R][FL_OC];
    unsigned long long bar;
    unsigned tmem;
};
static_assert(sizeof(FillSmem) < 227 * 1024, "fill tile");

// Where the inputs come from: a handle's state (read-out) or explicit images.
struct FillIO {
    int from_handle;
    const Ctrl *ctrl;                      // handle: k = base + m, h = det.h
    const float *L;                        // handle: filter output
    const unsigned long long *last_pix;    // handle: global index of each pixel's last event
    const float *x;                        // explicit: [2][H][W]
    const unsigned char *stale;            // explicit: [H][W] (1 = fill)
    float *out;                            // [H][W]
    float *const *outp;                    // if set: where to find out (a captured chain's descriptor)
    unsigned *err;                         // error word (bit ERR_FILL_WAIT)
    unsigned W, H;
};

__device__ __forceinline__ unsigned fl_smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned short fl_bf16_bits(float v)
{
    // round to nearest even (v is finite and >= 0 here: a ReLU output)
    const unsigned u = __float_as_uint(v);
    return (unsigned short)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

// round to nearest even for any finite value (inputs may be negative)
__device__ __forceinline__ unsigned short fl_bf16_bits_any(float v)
{
    const unsigned u = __float_as_uint(v);
    return (unsigned short)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance of
// the two 8-element K halves, sbo = byte distance of 8-row groups.
__device__ __forceinline__ unsigned long long fl_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    return (unsigned long long)((saddr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = 48
constexpr unsigned FL_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((48u >> 3) << 17) | ((128u >> 4) << 24);
constexpr unsigned FL_BDX = 1536;   // bytes of one dx block of a layer's B operand (48 rows x 32 B)

__device__ __forceinline__ void fl_mma(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d_tmem), "l"(a), "l"(b), "r"(FL_IDESC), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ bool fl_wait(unsigned long long *bar, unsigned phase)
{
    for (unsigned spins = 0; spins < FL_SPIN_LIMIT; ++spins) {
        unsigned ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(fl_smem_u32(bar)), "r"(phase)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fl_tmem_ld16(unsigned taddr, float (&v)[16])
{
    unsigned r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                 "%12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// tcgen05.ld of 16 columns without the wait: several loads in flight, then fl_tmem_wait
__device__ __forceinline__ void fl_tmem_ld16_async(unsigned taddr, unsigned (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                 "%12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

__device__ __forceinline__ void fl_tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 columns of zeros into the warp's TMEM lanes
__device__ __forceinline__ void fl_tmem_zero16(unsigned taddr)
{
    const unsigned z = 0u;
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
                 "%1, %1, %1, %1};" ::"r"(taddr), "r"(z) : "memory");
}

__device__ __forceinline__ float fl_tmem_ld1(unsigned taddr)
{
    unsigned r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return __uint_as_float(r);
}

// A layer (run_layer in k_fill): for each of its output rows r, 9 MMAs (taps dy, dx) of
// 128 pixels x 16 channels x 16 inputs into TMEM columns t0 + 16 r.  The A operand of tap
// (dy, dx) is the input tile's row r + dy from pixel dx on (the descriptor's start moves by
// dx rows of 16 bytes); its second K half lies `lbo` bytes after the start: the next plane
// of the tile, or for the 2-channel inputs a block of zeros.  One thread issues them.
__global__ void __launch_bounds__(FL_THREADS, 1) k_fill(FillParams fp, FillIO io)
{
    PDL_ENTRY();
    extern __shared__ __align__(1024) unsigned char fl_smem_raw[];
    FillSmem &S = *reinterpret_cast<FillSmem *>(fl_smem_raw);
    const int W = (int)io.W, H = (int)io.H;
    float *const fout = io.outp ? *io.outp : io.out;
    const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nseg = (W + FL_OC - 1) / FL_OC, nstrip = (H + FL_R - 1) / FL_R;
    const int units = nseg * nstrip;

    unsigned long long k_now = 0, h = 0, q = 1;
    if (io.from_handle) {
        k_now = io.ctrl->base + io.ctrl->m;
        h = (unsigned long long)io.ctrl->det.h;
        q = k_now > h ? k_now - h : 1ull;
    }
    for (int i = threadIdx.x; i < 9 * 32; i += FL_THREADS) {
        S.w[0][i] = fp.w1[i];
        S.w[1][i] = fp.w2[i];
        S.w[2][i] = fp.w3[i];
    }
    for (int i = threadIdx.x; i < FL_M; i += FL_THREADS) reinterpret_cast<uint4 *>(S.zero)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fl_smem_u32(&S.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(fl_smem_u32(&S.tmem)), "r"(FL_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = S.tmem;
    const unsigned bar = fl_smem_u32(&S.bar);
    const unsigned x_base = fl_smem_u32(S.x), z_base = fl_smem_u32(S.zero);
    const unsigned a1_base = fl_smem_u32(S.a1), a2_base = fl_smem_u32(S.a2);
    const unsigned w_base = fl_smem_u32(S.w[0]);
    unsigned phase = 0;
    bool failed = false;
    // make the threads' shared-memory writes visible to the tensor cores, wait for every
    // thread, and (thread 0) issue a layer; then everyone waits for its completion
    auto run_layer = [&](unsigned in_base, unsigned row_bytes, bool lbo_to_zero, unsigned wsel, unsigned t0,
                         int in_rows) {
        // zero the layer's accumulators (every MMA adds to three of them)
        for (int c = (int)(warp >> 2); c < in_rows + 2; c += FL_THREADS / 128)
            fl_tmem_zero16(tmem + ((32u * (warp & 3)) << 16) + t0 + 16u * c);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (threadIdx.x == 0) {
            // descriptors of input row 0, dx 0; a row or dx moves the start address (low
            // field, in 16-byte units) and, for the inputs, the distance to the zero block
            // the other way (the LBO field)
            const unsigned long long a0 = fl_desc(in_base, lbo_to_zero ? z_base - in_base : FL_PLANE, 128);
            const unsigned long long b0 = fl_desc(w_base + wsel * 3 * FL_BDX, FL_BDX / 2, 128);
            const unsigned long long step_unit = lbo_to_zero ? (1ull - (1ull << 16)) : 1ull;
            // rows in steps of three: consecutive MMAs write disjoint accumulators
            for (int dx = 0; dx < 3; ++dx)
                for (int j0 = 0; j0 < 3; ++j0)
                    for (int j = j0; j < in_rows; j += 3) {
                        const unsigned off = (j * row_bytes + dx * 16) >> 4;
                        fl_mma(tmem + t0 + 16 * j, a0 + step_unit * off, b0 + (unsigned long long)(dx * (FL_BDX >> 4)), 1u);
                    }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                         : "memory");
        }
        // one warp polls the barrier, the others wait at the block barrier
        bool ok = warp == 0 ? fl_wait(&S.bar, phase) : true;
        phase ^= 1u;
        if (!ok && threadIdx.x == 0) atomicOr(io.err, ERR_FILL_WAIT);
        failed = __syncthreads_or(!ok) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };
    // epilogue of conv1 / conv2: TMEM -> bias, ReLU -> BF16 tile rows (zero outside the image)
    auto epilogue = [&](unsigned t0, int rows, const float *bias, unsigned char *dst, int gy0, int gx0) {
        constexpr int RSTEP = FL_THREADS / 128;                      // rows a warp handles apart
        constexpr int RMAX = (FL_A1R + RSTEP - 1) / RSTEP;           // rows per warp at most
        const int px = 32 * (warp & 3) + lane;
        const int gx = gx0 + px;
        const int r0 = (int)(warp >> 2);
        // all of the warp's TMEM loads first, one wait
        unsigned raw[RMAX][16];
#pragma unroll
        for (int j = 0; j < RMAX; ++j)
            if (r0 + j * RSTEP < rows)
                fl_tmem_ld16_async(tmem + ((32u * (warp & 3)) << 16) + t0 + 16u * (r0 + j * RSTEP + 2), raw[j]);
        fl_tmem_wait();
#pragma unroll
        for (int j = 0; j < RMAX; ++j) {
            const int r = r0 + j * RSTEP;
            if (r >= rows) break;
            const int gy = gy0 + r;
            const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
            unsigned pk[8];
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const unsigned lo = in ? fl_bf16_bits(fmaxf(__uint_as_float(raw[j][2 * o]) + bias[2 * o], 0.f)) : 0u;
                const unsigned hi = in ? fl_bf16_bits(fmaxf(__uint_as_float(raw[j][2 * o + 1]) + bias[2 * o + 1], 0.f)) : 0u;
                pk[o] = lo | (hi << 16);
            }
            uint4 *row = reinterpret_cast<uint4 *>(dst + r * FL_ROW2);
            row[px] = make_uint4(pk[0], pk[1], pk[2], pk[3]);            // channels 0-7
            row[FL_C + px] = make_uint4(pk[4], pk[5], pk[6], pk[7]);     // channels 8-15
        }
    };

    // a unit's global inputs, one thread's share, loaded into registers: the next unit's are
    // requested right after the current unit's have been stored, so that they arrive
    // while the tensor cores run the current unit
    float v0[FL_XITER], v1x[FL_XITER];
    unsigned long long lp[FL_XITER];
    unsigned char sx[FL_XITER];
    auto load_inputs = [&](int u) {
        const int y0 = (u / nseg) * FL_R, x0 = (u % nseg) * FL_OC;
#pragma unroll
        for (int it = 0; it < FL_XITER; ++it) {
            const int i = threadIdx.x + it * FL_THREADS;
            const int r = i / FL_C, c = i % FL_C;
            const int gy = y0 - 3 + r, gx = x0 - 3 + c;
            const bool in = u < units && i < FL_XN && gy >= 0 && gy < H && gx >= 0 && gx < W;
            const size_t p = in ? (size_t)gy * W + gx : 0;
            v0[it] = 0.f;
            v1x[it] = 0.f;
            lp[it] = NONE64;
            sx[it] = 0;
            if (in) {
                if (io.from_handle) {
                    v0[it] = io.L[p];
                    lp[it] = io.last_pix[p];
                } else {
                    v0[it] = io.x[p];
                    v1x[it] = io.x[(size_t)W * H + p];
                    sx[it] = io.stale[p];
                }
            }
        }
    };
    load_inputs(blockIdx.x);

    for (int u = blockIdx.x; u < units && !failed; u += gridDim.x) {
        const int y0 = (u / nseg) * FL_R, x0 = (u % nseg) * FL_OC;
        // inputs: rows y0-3 .. y0+10, columns x0-3 .. x0+126 (zero outside the image), as
        // BF16 channels (L, age); the output pixels' L in FP32 and their stale flags
        {
#pragma unroll
            for (int it = 0; it < FL_XITER; ++it) {
                const int i = threadIdx.x + it * FL_THREADS;
                if (i >= FL_XN) break;
                const int r = i / FL_C, c = i % FL_C;
                const int gy = y0 - 3 + r, gx = x0 - 3 + c;
                const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
                float v1 = v1x[it];
                unsigned char st = sx[it];
                if (in && io.from_handle) {
                    if (lp[it] == NONE64) {
                        v1 = FL_AGE_MAX;
                    } else {
                        const unsigned long long gap = k_now - lp[it];
                        v1 = gap >= 4ull * q ? FL_AGE_MAX : (float)gap / (float)q;
                    }
                    st = (lp[it] != NONE64 && lp[it] < h) ? 1 : 0;
                }
                const int orow = gy - y0, ocol = gx - x0;
                if (in && orow >= 0 && orow < FL_R && ocol >= 0 && ocol < FL_OC) {
                    S.stale[orow][ocol] = st;
                    S.lout[orow][ocol] = v0[it];
                }
                const unsigned b0 = in ? fl_bf16_bits_any(v0[it]) : 0u;
                const unsigned b1 = in ? fl_bf16_bits_any(v1) : 0u;
                reinterpret_cast<uint4 *>(S.x + r * FL_PLANE)[c] = make_uint4(b0 | (b1 << 16), 0u, 0u, 0u);
            }
        }
        load_inputs(u + (int)gridDim.x);
        // conv1: a1 rows (global y0-2 ..), pixels x0-2 .. x0+125
        run_layer(x_base, FL_PLANE, true, 0, FL_T1, FL_XR);
        if (failed) break;
        epilogue(FL_T1, FL_A1R, fp.b1, S.a1, y0 - 2, x0 - 2);
        // conv2: a2 rows (global y0-1 ..), pixels x0-1 .. x0+126
        run_layer(a1_base, FL_ROW2, false, 1, FL_T2, FL_A1R);
        if (failed) break;
        epilogue(FL_T2, FL_A2R, fp.b2, S.a2, y0 - 1, x0 - 1);
        // conv3: output rows y0 .., pixels x0 .. x0+127 (the first 124 kept)
        run_layer(a2_base, FL_ROW2, false, 2, FL_T3, FL_A2R);
        if (failed) break;
        {
            const int px = 32 * (warp & 3) + lane;
            const int gx = x0 + px;
            for (int o = (int)(warp >> 2); o < FL_R; o += FL_THREADS / 128) {
                const float y = fl_tmem_ld1(tmem + ((32u * (warp & 3)) << 16) + FL_T3 + 16u * (o + 2)) + fp.b3;
                const int gy = y0 + o;
                if (px < FL_OC && gx < W && gy < H) fout[(size_t)gy * W + gx] = S.stale[o][px] ? y : S.lout[o][px];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FL_TMEM_COLS) : "memory");
}

// The network's inputs from a handle's state: x [2][H][W] (L, age) and the stale mask.
__global__ void k_fill_features(const Ctrl *ctrl, const float *L, const unsigned long long *last_pix,
                                unsigned W, unsigned H, float *x, unsigned char *stale)
{
    const unsigned long long k_now = ctrl->base + ctrl->m, h = (unsigned long long)ctrl->det.h;
    const unsigned long long q = k_now > h ? k_now - h : 1ull;
    const size_t n = (size_t)W * H;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long lp = last_pix[p];
        float a = FL_AGE_MAX;
        if (lp != NONE64) {
            const unsigned long long gap = k_now - lp;
            a = gap >= 4ull * q ? FL_AGE_MAX : (float)gap / (float)q;
        }
        x[p] = L[p];
        x[n + p] = a;
        if (stale) stale[p] = (lp != NONE64 && lp < h) ? 1 : 0;
    }
}

// ---- training --------------------------------------------------------------------

constexpr int FT_S = 24;                 // crop side
constexpr int FT_P = FT_S * FT_S;
constexpr int FT_THREADS = 256;
constexpr int FT_MARGIN = 3;             // loss only where the 7 x 7 receptive field is inside

struct TrainSmem {
    float x[2][FT_P];
    float z1[16][FT_P];     // z1, then dz1
    float z2[16][FT_P];     // z2, then dz2
    float g[FT_P];          // y, then the loss gradient gy
    float th[FILL_NPARAMS];
    float red[FT_THREADS / 32];
};

// parameter offsets in theta (W1, b1, W2, b2, W3, b3)
constexpr int OW1 = 0, OB1 = 288, OW2 = 304, OB2 = 2608, OW3 = 2624, OB3 = 2768;

__device__ __forceinline__ float fl_bf16_round(float v)
{
    const unsigned u = __float_as_uint(v);
    return __uint_as_float(((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16) << 16);
}

__device__ __forceinline__ float crop_at(const float *a, int y, int x)
{
    return (y >= 0 && y < FT_S && x >= 0 && x < FT_S) ? a[y * FT_S + x] : 0.f;
}

__device__ __forceinline__ float block_sum_ft(float v, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x < 32) {
        t = threadIdx.x < FT_THREADS / 32 ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    }
    return t;  // valid in thread 0
}

// One CTA per crop: forward, loss gradient, backward; unnormalised gradient sums into
// grad[0 .. FILL_NPARAMS), the loss sum into acc[0] and the loss pixel count into acc[1].
__global__ void __launch_bounds__(FT_THREADS, 2)
k_fill_train(const float *X, const float *T, const unsigned char *M, unsigned W, unsigned H, unsigned F,
             const int *crops, const float *theta, float *grad, double *acc)
{
    extern __shared__ __align__(16) unsigned char ft_smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(ft_smem_raw);
    const int f = crops[3 * blockIdx.x], cy = crops[3 * blockIdx.x + 1], cx = crops[3 * blockIdx.x + 2];
    // a crop outside the frames contributes nothing (counted in acc[2])
    if (f < 0 || f >= (int)F || cy < 0 || cx < 0 || cy + FT_S > (int)H || cx + FT_S > (int)W) {
        if (threadIdx.x == 0) atomicAdd(&acc[2], 1.0);
        return;
    }
    const size_t plane = (size_t)W * H;
    const float *Xf = X + (size_t)f * 2 * plane;
    for (int i = threadIdx.x; i < FILL_NPARAMS; i += FT_THREADS) {
        const float v = theta[i];
        // the forward pass uses BF16 weights (biases stay FP32)
        const bool is_w = i < OB1 || (i >= OW2 && i < OB2) || (i >= OW3 && i < OB3);
        S.th[i] = is_w ? fl_bf16_round(v) : v;
    }
    for (int p = threadIdx.x; p < FT_P; p += FT_THREADS) {
        // every layer's input enters as BF16 (the read-out's tensor-core operands)
        const size_t g = (size_t)(cy + p / FT_S) * W + cx + p % FT_S;
        S.x[0][p] = fl_bf16_round(Xf[g]);
        S.x[1][p] = fl_bf16_round(Xf[plane + g]);
    }
    __syncthreads();
    // forward: z1, z2 (pre-activations), y
    for (int i = threadIdx.x; i < 16 * FT_P; i += FT_THREADS) {
        const int o = i / FT_P, p = i % FT_P, py = p / FT_S, px = p % FT_S;
        float a = S.th[OB1 + o];
        for (int ci = 0; ci < 2; ++ci)
            for (int t = 0; t < 9; ++t)
                a = fmaf(S.th[OW1 + o * 18 + ci * 9 + t], crop_at(S.x[ci], py + t / 3 - 1, px + t % 3 - 1), a);
        S.z1[o][p] = a;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 16 * FT_P; i += FT_THREADS) {
        const int o = i / FT_P, p = i % FT_P, py = p / FT_S, px = p % FT_S;
        float a = S.th[OB2 + o];
        for (int ci = 0; ci < 16; ++ci)
            for (int t = 0; t < 9; ++t) {
                const int yy = py + t / 3 - 1, xx = px + t % 3 - 1;
                const float v = (yy >= 0 && yy < FT_S && xx >= 0 && xx < FT_S) ? fl_bf16_round(fmaxf(S.z1[ci][yy * FT_S + xx], 0.f)) : 0.f;
                a = fmaf(S.th[OW2 + (o * 16 + ci) * 9 + t], v, a);
            }
        S.z2[o][p] = a;
    }
    __syncthreads();
    float lsum = 0.f, lcnt = 0.f;
    for (int p = threadIdx.x; p < FT_P; p += FT_THREADS) {
        const int py = p / FT_S, px = p % FT_S;
        float a = S.th[OB3];
        for (int ci = 0; ci < 16; ++ci)
            for (int t = 0; t < 9; ++t)
                a = fmaf(S.th[OW3 + ci * 9 + t],
                         fl_bf16_round(fmaxf(crop_at(S.z2[ci], py + t / 3 - 1, px + t % 3 - 1), 0.f)), a);
        const bool inner = py >= FT_MARGIN && py < FT_S - FT_MARGIN && px >= FT_MARGIN && px < FT_S - FT_MARGIN;
        const size_t g = (size_t)f * plane + (size_t)(cy + py) * W + cx + px;
        float gy = 0.f;
        if (inner && M[g]) {
            const float r = a - T[g];
            gy = 2.f * r;
            lsum += r * r;
            lcnt += 1.f;
        }
        S.g[p] = gy;
    }
    __syncthreads();
    {
        const float ls = block_sum_ft(lsum, S.red);
        const float lc = block_sum_ft(lcnt, S.red);
        if (threadIdx.x == 0) {
            atomicAdd(&acc[0], (double)ls);
            atomicAdd(&acc[1], (double)lc);
        }
    }
    // conv3 weights and bias
    for (int i = threadIdx.x; i < 16 * 9 + 1; i += FT_THREADS) {
        float s = 0.f;
        if (i < 144) {
            const int ci = i / 9, t = i % 9;
            for (int p = 0; p < FT_P; ++p)
                s = fmaf(S.g[p], fl_bf16_round(fmaxf(crop_at(S.z2[ci], p / FT_S + t / 3 - 1, p % FT_S + t % 3 - 1), 0.f)), s);
            atomicAdd(&grad[OW3 + i], s);
        } else {
            for (int p = 0; p < FT_P; ++p) s += S.g[p];
            atomicAdd(&grad[OB3], s);
        }
    }
    __syncthreads();
    // dz2 = (conv3 transposed applied to gy) where z2 > 0, in place of z2
    for (int i = threadIdx.x; i < 16 * FT_P; i += FT_THREADS) {
        const int c = i / FT_P, p = i % FT_P, py = p / FT_S, px = p % FT_S;
        float d = 0.f;
        if (S.z2[c][p] > 0.f)
            for (int t = 0; t < 9; ++t) d = fmaf(S.th[OW3 + c * 9 + t], crop_at(S.g, py - (t / 3 - 1), px - (t % 3 - 1)), d);
        S.z2[c][p] = d;
    }
    __syncthreads();
    // conv2 weights and biases: sum over pixels of dz2 x bf16(a1) shifted
    for (int i = threadIdx.x; i < 16 * 16 * 9 + 16; i += FT_THREADS) {
        float s = 0.f;
        if (i < 2304) {
            const int o = i / 144, ci = (i / 9) % 16, t = i % 9;
            for (int p = 0; p < FT_P; ++p) {
                const int yy = p / FT_S + t / 3 - 1, xx = p % FT_S + t % 3 - 1;
                const float a1 = (yy >= 0 && yy < FT_S && xx >= 0 && xx < FT_S) ? fl_bf16_round(fmaxf(S.z1[ci][yy * FT_S + xx], 0.f)) : 0.f;
                s = fmaf(S.z2[o][p], a1, s);
            }
            atomicAdd(&grad[OW2 + i], s);
        } else {
            const int o = i - 2304;
            for (int p = 0; p < FT_P; ++p) s += S.z2[o][p];
            atomicAdd(&grad[OB2 + o], s);
        }
    }
    __syncthreads();
    // dz1 = (conv2 transposed applied to dz2) where z1 > 0, in place of z1
    for (int i = threadIdx.x; i < 16 * FT_P; i += FT_THREADS) {
        const int ci = i / FT_P, p = i % FT_P, py = p / FT_S, px = p % FT_S;
        float d = 0.f;
        if (S.z1[ci][p] > 0.f)
            for (int o = 0; o < 16; ++o)
                for (int t = 0; t < 9; ++t)
                    d = fmaf(S.th[OW2 + (o * 16 + ci) * 9 + t], crop_at(S.z2[o], py - (t / 3 - 1), px - (t % 3 - 1)), d);
        S.z1[ci][p] = d;
    }
    __syncthreads();
    // conv1 weights and biases
    for (int i = threadIdx.x; i < 16 * 2 * 9 + 16; i += FT_THREADS) {
        float s = 0.f;
        if (i < 288) {
            const int o = i / 18, ci = (i / 9) % 2, t = i % 9;
            for (int p = 0; p < FT_P; ++p)
                s = fmaf(S.z1[o][p], crop_at(S.x[ci], p / FT_S + t / 3 - 1, p % FT_S + t % 3 - 1), s);
            atomicAdd(&grad[OW1 + i], s);
        } else {
            const int o = i - 288;
            for (int p = 0; p < FT_P; ++p) s += S.z1[o][p];
            atomicAdd(&grad[OB1 + o], s);
        }
    }
}

// Adam on the FP32 master weights with the gradient sums divided by the loss pixels;
// grad is left holding the mean gradient.
__global__ void k_fill_adam(float *theta, float *m, float *v, float *grad, const double *acc, unsigned step,
                            float lr, float b1, float b2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= FILL_NPARAMS) return;
    const double n = acc[1];
    const float g = n > 0.0 ? (float)((double)grad[i] / n) : 0.f;
    grad[i] = g;
    if (lr <= 0.f) return;
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)step));
    const float vh = vi / (1.f - powf(b2, (float)step));
    theta[i] -= lr * mh / (sqrtf(vh) + eps);
}

cudaError_t launch_fill(const FillParams &fp, const FillIO &io, cudaStream_t s, unsigned long long &nl, int max_ctas = 0);

cudaError_t launch_fill_readout(const FillParams &fp, const KParams &kp, const Bufs &b, float *out, cudaStream_t s,
                                unsigned long long &nl, float *const *outp)
{
    FillIO io{};
    io.from_handle = 1;
    io.ctrl = b.ctrl;
    io.L = b.L;
    io.last_pix = b.last_pix;
    io.out = out;
    io.outp = outp;
    io.err = &b.ctrl->error;
    io.W = kp.W;
    io.H = kp.H;
    return launch_fill(fp, io, s, nl, grid_for(kp, 1));
}

size_t fill_smem_bytes() { return sizeof(FillSmem); }
size_t fill_train_smem_bytes() { return sizeof(TrainSmem); }

cudaError_t launch_fill(const FillParams &fp, const FillIO &io, cudaStream_t s, unsigned long long &nl, int max_ctas)
{
    nl += 1;
    static std::atomic<unsigned long long> attr_done{0};
    if (cudaError_t e = smem_attr_once(attr_done, k_fill, sizeof(FillSmem))) return e;
    const int units = ((int)((io.W + FL_OC - 1) / FL_OC)) * ((int)((io.H + FL_R - 1) / FL_R));
    const int grid = std::min(max_ctas > 0 ? max_ctas : grid_for(1), units);
    if (cudaError_t e = launch_pdl(k_fill, grid, FL_THREADS, sizeof(FillSmem), s, fp, io)) return e;
    return cudaGetLastError();
}

}  // namespace fibar

using namespace fibar;

namespace {

unsigned short host_bf16_bits(float v)
{
    unsigned u;
    memcpy(&u, &v, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (unsigned short)(u >> 16);  // inf / nan: truncate
    return (unsigned short)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}


}  // namespace

namespace fibar {

// Kernel parameters of the network from theta (W1, b1, W2, b2, W3, b3; FP32): weights
// rounded to BF16, W2 packed as the per-tap B operands.
int pack_fill_params(const float *theta, FillParams *fp)
{
    for (int i = 0; i < FILL_NPARAMS; ++i)
        if (!isfinite(theta[i])) return FIBAR_EINVAL;
    memset(fp, 0, sizeof(*fp));
    for (int i = 0; i < 16; ++i) fp->b1[i] = theta[OB1 + i];
    for (int i = 0; i < 16; ++i) fp->b2[i] = theta[OB2 + i];
    fp->b3 = theta[OB3];
    // tap (dy, dx), output channel co, input channel k: dx block of 48 rows n = 16 (2 - dy) + co,
    // byte dx * 1536 + (k / 8) * 768 + n * 16 + (k % 8) * 2
    auto put = [](uint4 *ops, int t, int co, int k, float v) {
        const int dy = t / 3, dx = t % 3, n = 16 * (2 - dy) + co;
        unsigned short *w = reinterpret_cast<unsigned short *>(ops);
        w[((size_t)dx * 1536 + (k / 8) * 768 + n * 16 + (k % 8) * 2) / 2] = host_bf16_bits(v);
    };
    for (int t = 0; t < 9; ++t)
        for (int co = 0; co < 16; ++co) {
            for (int ci = 0; ci < 2; ++ci) put(fp->w1, t, co, ci, theta[OW1 + (co * 2 + ci) * 9 + t]);
            for (int ci = 0; ci < 16; ++ci) put(fp->w2, t, co, ci, theta[OW2 + (co * 16 + ci) * 9 + t]);
        }
    for (int t = 0; t < 9; ++t)
        for (int ci = 0; ci < 16; ++ci) put(fp->w3, t, 0, ci, theta[OW3 + ci * 9 + t]);
    return FIBAR_OK;
}

}  // namespace fibar

extern "C" int fibar_fill_set_weights(fibar_t *h, const float *theta, size_t n)
{
    if (!h) return FIBAR_EINVAL;
    h->config_version += 1;  // a captured read-out chain holds the weights by value
    if (!theta) {
        delete h->fill;
        h->fill = nullptr;
        return FIBAR_OK;
    }
    if (n != (size_t)FILL_NPARAMS) {
        h->err = "fill_set_weights: expected " + std::to_string(FILL_NPARAMS) + " parameters";
        return FIBAR_EINVAL;
    }
    FillParams fp;
    if (pack_fill_params(theta, &fp) != FIBAR_OK) {
        h->err = "fill_set_weights: every parameter must be finite";
        return FIBAR_EINVAL;
    }
    if (!h->fill) h->fill = new (std::nothrow) FillParams;
    if (!h->fill) return FIBAR_ENOMEM;
    *h->fill = fp;
    return FIBAR_OK;
}

extern "C" int fibar_fill_features(fibar_t *h, float *x, uint8_t *stale, void *cuda_stream)
{
    if (!h || !x) return FIBAR_EINVAL;
    if (((uintptr_t)x & 3) != 0) {
        h->err = "fill_features: misaligned output";
        return FIBAR_EINVAL;
    }
    if (!h->kp.spatial) {
        h->err = "fill_features: the handle has no stale-pixel detector (spatial_filter = 0)";
        return FIBAR_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_fill_features<<<grid_for(h->kp, 4), 256, 0, s>>>(h->b.ctrl, h->b.L, h->b.last_pix, h->W, h->H, x, stale);
    h->launches += 1;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->err = std::string("fill_features: ") + cudaGetErrorString(e);
        return FIBAR_ECUDA;
    }
    return FIBAR_OK;
}

extern "C" int fibar_fill_forward(const float *theta, const float *x, const uint8_t *stale, uint32_t W, uint32_t H,
                                  float *out, void *cuda_stream)
{
    if (!theta || !x || !stale || !out || W == 0 || H == 0 || (unsigned long long)W * H > (1ull << 24))
        return FIBAR_EINVAL;
    if (((uintptr_t)x & 3) != 0 || ((uintptr_t)out & 3) != 0) return FIBAR_EINVAL;
    FillParams fp;
    if (pack_fill_params(theta, &fp) != FIBAR_OK) return FIBAR_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned *err = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&err, sizeof(unsigned), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FIBAR_ENOMEM;
    }
    e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
    FillIO io{};
    io.from_handle = 0;
    io.x = x;
    io.stale = stale;
    io.out = out;
    io.err = err;
    io.W = W;
    io.H = H;
    unsigned long long nl = 0;
    if (e == cudaSuccess) e = launch_fill(fp, io, s, nl);
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(err, s);
    if (e != cudaSuccess) return FIBAR_ECUDA;
    return herr ? FIBAR_ETIMEOUT : FIBAR_OK;
}

extern "C" int fibar_fill_train_step(const float *X, const float *T, const uint8_t *M, uint32_t W, uint32_t H,
                                     uint32_t n_frames, const int32_t *crops, uint32_t n_crops, float *theta,
                                     float *m, float *v, float *grad, uint32_t step, float lr, double *loss_acc,
                                     void *cuda_stream)
{
    if (!X || !T || !M || !crops || !theta || !m || !v || !grad || !loss_acc || W < FT_S || H < FT_S ||
        n_frames == 0 || n_crops == 0 || n_crops > 65535 || step == 0)
        return FIBAR_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    static std::atomic<unsigned long long> attr_done{0};
    if (cudaError_t e = smem_attr_once(attr_done, k_fill_train, sizeof(TrainSmem))) return FIBAR_ECUDA;
    cudaError_t e = cudaMemsetAsync(grad, 0, FILL_NPARAMS * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss_acc, 0, 3 * sizeof(double), s);
    if (e != cudaSuccess) return FIBAR_ECUDA;
    k_fill_train<<<n_crops, FT_THREADS, sizeof(TrainSmem), s>>>(X, T, M, W, H, n_frames, crops, theta, grad, loss_acc);
    k_fill_adam<<<(FILL_NPARAMS + 255) / 256, 256, 0, s>>>(theta, m, v, grad, loss_acc, step, lr, 0.9f, 0.999f, 1e-8f);
    e = cudaGetLastError();
    return e == cudaSuccess ? FIBAR_OK : FIBAR_ECUDA;
}
