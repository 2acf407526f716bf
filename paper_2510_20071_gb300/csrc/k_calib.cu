// fibar_relative_thresholds: relative contrast thresholds of every pixel from a
// calibration recording (the paper's appendix on relative contrast thresholds).
//
// Under a spatially uniform, stationary signal every pixel sees the same total brightness
// travel |dL| upwards and downwards, so N_on,i C_on,i = N_off,i C_off,i = |dL|.  With
// C_i the harmonic mean of C_on,i and C_off,i, C the harmonic mean of the C_i over all
// pixels and Nbar the mean event count per pixel:
//   C'_on,i = C_on,i / C = Nbar / (2 N_on,i),  C'_off,i = Nbar / (2 N_off,i),
//   C'_i    = C_i / C    = Nbar / (N_on,i + N_off,i).
// C'_i is the per-pixel factor that Sec. 5.2 applies to the right-hand side of Eq. 6
// (fibar_set_pixel_gain).
//
// Two kernels: per-pixel ON / OFF counts with global atomics (four 16-byte records per
// thread and iteration in flight, the total per block reduced in shared memory), then
// one thread per pixel for the three quotients.
#include "fibar_internal.cuh"

namespace fibar {
namespace {

constexpr size_t CAL_CHUNK = size_t(1) << 22;  // host events staged per copy (64 MiB)

__global__ void __launch_bounds__(256) k_calib_count(const int4 *__restrict__ ev, size_t n, unsigned W, unsigned H,
                                                     unsigned *n_on, unsigned *n_off, unsigned long long *total)
{
    __shared__ unsigned s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    unsigned mine = 0;
    auto count = [&](const int4 r) {
        const unsigned x = (unsigned)r.x & 0xFFFFu, y = (unsigned)r.x >> 16;
        const int p = (int)(signed char)(r.y & 0xFF);
        if (x < W && y < H) {
            atomicAdd(p > 0 ? &n_on[y * W + x] : &n_off[y * W + x], 1u);
            ++mine;
        }
    };
    // four records in flight per thread (read once: not kept in L2)
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (; k + 3 * stride < n; k += 4 * stride) {
        const int4 r0 = __ldcs(&ev[k]), r1 = __ldcs(&ev[k + stride]);
        const int4 r2 = __ldcs(&ev[k + 2 * stride]), r3 = __ldcs(&ev[k + 3 * stride]);
        count(r0);
        count(r1);
        count(r2);
        count(r3);
    }
    for (; k < n; k += stride) count(__ldcs(&ev[k]));
    // block total of the counted records
#pragma unroll
    for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xFFFFFFFFu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(total, (unsigned long long)s_cnt);
}

__global__ void __launch_bounds__(256) k_calib_finish(size_t npix, const unsigned *n_on, const unsigned *n_off,
                                                      const unsigned long long *total, float *c_on, float *c_off,
                                                      float *c)
{
    const double nbar = (double)*total / (double)npix;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npix; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned a = n_on[i], b = n_off[i];
        c_on[i] = a ? (float)(nbar / (2.0 * a)) : __int_as_float(0x7FC00000);
        c_off[i] = b ? (float)(nbar / (2.0 * b)) : __int_as_float(0x7FC00000);
        c[i] = a + b ? (float)(nbar / ((double)a + (double)b)) : __int_as_float(0x7FC00000);
    }
}

}  // namespace
}  // namespace fibar

using namespace fibar;

extern "C" int fibar_relative_thresholds(const fibar_event_t *ev, size_t n, uint32_t W, uint32_t H, int on_device,
                                         float *c_on, float *c_off, float *c, void *cuda_stream)
{
    const size_t npix = (size_t)W * H;
    if (W == 0 || H == 0 || npix > (size_t(1) << 24) || (n && !ev) || !c_on || !c_off || !c) return FIBAR_EINVAL;
    if (on_device && n && ((uintptr_t)ev & 15) != 0) return FIBAR_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // workspace: counts, total, host-event staging, host-output staging
    const size_t stage_n = on_device ? 0 : std::min(n, CAL_CHUNK);
    const size_t off_total = 2 * npix * sizeof(unsigned);
    const size_t off_stage = (off_total + sizeof(unsigned long long) + 15) & ~size_t(15);
    const size_t off_out = off_stage + stage_n * sizeof(int4);
    const size_t bytes = off_out + (on_device ? 0 : 3 * npix * sizeof(float));
    char *ws = nullptr;
    if (cudaMallocAsync((void **)&ws, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return FIBAR_ENOMEM;
    }
    unsigned *n_on = reinterpret_cast<unsigned *>(ws), *n_off = n_on + npix;
    unsigned long long *total = reinterpret_cast<unsigned long long *>(ws + off_total);
    int4 *stage = reinterpret_cast<int4 *>(ws + off_stage);
    float *o_on = on_device ? c_on : reinterpret_cast<float *>(ws + off_out);
    float *o_off = on_device ? c_off : o_on + npix;
    float *o_c = on_device ? c : o_on + 2 * npix;
    cudaError_t e = cudaMemsetAsync(ws, 0, off_total + sizeof(unsigned long long), s);
    if (on_device) {
        if (e == cudaSuccess && n)
            k_calib_count<<<grid_for(8), 256, 0, s>>>(reinterpret_cast<const int4 *>(ev), n, W, H, n_on, n_off, total);
    } else {
        for (size_t off = 0; off < n && e == cudaSuccess; off += CAL_CHUNK) {
            const size_t cnt = std::min(CAL_CHUNK, n - off);
            e = cudaMemcpyAsync(stage, ev + off, cnt * sizeof(int4), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) k_calib_count<<<grid_for(8), 256, 0, s>>>(stage, cnt, W, H, n_on, n_off, total);
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) k_calib_finish<<<grid_for(4), 256, 0, s>>>(npix, n_on, n_off, total, o_on, o_off, o_c);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (!on_device && e == cudaSuccess) {
        e = cudaMemcpyAsync(c_on, o_on, npix * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c_off, o_off, npix * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c, o_c, npix * sizeof(float), cudaMemcpyDeviceToHost, s);
    }
    const cudaError_t ef = cudaFreeAsync(ws, s);
    if (e == cudaSuccess) e = ef;
    if (!on_device && e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FIBAR_ECUDA;
    }
    return FIBAR_OK;
}
