// fibar_queue_counts_noalloc: the per-pixel queued-event counts of fibar_debug_state,
// computed without allocating memory.
//
// fibar_debug_state counts into a device buffer that it allocates on first use.  This
// entry point counts into a fixed buffer compiled into the library instead (a file-scope
// __device__ array of NOALLOC_MAX_PIXELS 32-bit counters, 4 MiB), so a caller that must
// not allocate device memory once it is running can still read the counts.
//
// Set-up: every call looks up the buffer's device address with cudaGetSymbolAddress
// while the handle's device is current (this allocates nothing).  The first lookup in a
// process may load the library's device code on that device; make the first call before
// any stream capture.  Looking the address up again on each call keeps it valid after a
// context has been torn down and re-created (the module then reloads at a new address).
// Zeroing: the counters must start at zero; every call clears the first W*H of them on
// its stream before counting.
// Sharing: the buffer is one per device for the whole process.  Calls that overlap in
// time (other streams, other threads, other handles on the same device) race on it and
// may return wrong counts; calls issued on one stream are ordered and safe.
#include <stdio.h>

#include "fibar_internal.cuh"

namespace fibar {
namespace {

constexpr size_t NOALLOC_MAX_PIXELS = size_t(1) << 20;  // 4 MiB of counters
static __device__ __align__(256) unsigned g_count_scratch[NOALLOC_MAX_PIXELS];

// Device address of the scratch array on the current device.
cudaError_t scratch_address(unsigned **ptr)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_count_scratch);
    if (e != cudaSuccess) return e;
    *ptr = static_cast<unsigned *>(p);
    return cudaSuccess;
}

// One count per queued event: the window [h, k) of global event indices (its pixel ids
// are in the ring), the same count as the debug read-out's kernel.
__global__ void k_queue_counts_scratch(KParams kp, const Ctrl *ctrl, const unsigned *ring_pix, unsigned *cnt)
{
    const unsigned long long h = (unsigned long long)ctrl->det.h, k = ctrl->base;
    for (unsigned long long j = h + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ring_pix[j & kp.ring_mask]], 1u);
}

int fail_msg(fibar_t *h, int code, const std::string &msg)
{
    h->err = msg;
    return code;
}

}  // namespace
}  // namespace fibar

using namespace fibar;

extern "C" int fibar_queue_counts_noalloc(fibar_t *h, uint32_t *cnt, int on_device, void *cuda_stream)
{
    if (!h || !cnt) return FIBAR_EINVAL;
    const size_t npix = h->kp.npix;
    if (npix > NOALLOC_MAX_PIXELS)
        return fail_msg(h, FIBAR_EINVAL,
                        "fibar_queue_counts_noalloc: W*H = " + std::to_string(npix) +
                            " pixels exceeds its fixed buffer of " + std::to_string(NOALLOC_MAX_PIXELS) +
                            " counters; use fibar_debug_state");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_msg(h, FIBAR_ECUDA, std::string("fibar_queue_counts_noalloc: ") + cudaGetErrorString(e));
    if (dev != h->device)
        return fail_msg(h, FIBAR_EINVAL, "fibar_queue_counts_noalloc: the handle's device must be current");
    unsigned *scratch = nullptr;
    e = scratch_address(&scratch);
    if (e != cudaSuccess)
        return fail_msg(h, FIBAR_ECUDA, std::string("fibar_queue_counts_noalloc set-up: ") + cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    e = cudaMemsetAsync(scratch, 0, npix * sizeof(unsigned), s);
    if (e == cudaSuccess && h->kp.spatial) {
        k_queue_counts_scratch<<<grid_for(h->kp, 2), 256, 0, s>>>(h->kp, h->b.ctrl, h->b.ring_pix, scratch);
        e = cudaGetLastError();
        h->launches += 1;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cnt, scratch, npix * sizeof(unsigned),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    // host output: after the synchronisation, the pipeline's error word says whether a
    // bounded device wait gave up (the queue window may then be inconsistent); it is
    // read into a stack variable, which allocates nothing
    unsigned err = 0;
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(&err, &h->b.ctrl->error, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_msg(h, FIBAR_ECUDA, std::string("fibar_queue_counts_noalloc: ") + cudaGetErrorString(e));
    if (err) {
        char msg[96];
        snprintf(msg, sizeof msg, "fibar_queue_counts_noalloc: a bounded device wait gave up (flags 0x%x)", err);
        return fail_msg(h, FIBAR_ETIMEOUT, msg);
    }
    return FIBAR_OK;
}
