// fibar_readout_batch: read-outs of many handles (streams of different sensors) with
// their pipelines running side by side on the device.
//
// One handle's read-out is a chain of kernels that must run in order; the read-outs of
// different handles share nothing.  A small sensor's read-out leaves most of the 152 SMs
// idle, so the handles of a batch are spread over a pool of internal CUDA streams: the
// GPU runs the chains of several handles at once, and a short chain does not wait
// behind a long one.
//
// Assignment: largest pending work first, each handle to the pool stream with the least
// assigned work (longest-processing-time-first list scheduling); a handle's work is its
// bound on pending events plus a fixed cost for the launches of one read-out.
// Ordering: the pool streams wait for an event recorded on the caller's stream before
// the first handle's work, and the caller's stream waits for an event recorded on each
// pool stream after its last handle's work.
#include <algorithm>
#include <mutex>
#include <vector>

#include "fibar_internal.cuh"

namespace fibar {
namespace {

constexpr int BATCH_STREAMS = 16;
constexpr size_t BATCH_MAX = 4096;
constexpr int BATCH_MAX_DEVICES = 64;
// the cost of one read-out's launch chain, in events of work
constexpr unsigned long long READOUT_FIXED_COST = 32768;

struct StreamPool {
    bool ready = false;
    cudaStream_t s[BATCH_STREAMS] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[BATCH_STREAMS] = {};
};

std::mutex g_batch_mutex;
StreamPool g_pool[BATCH_MAX_DEVICES];

// Create the pool of the current device (called with g_batch_mutex held).
cudaError_t pool_ready(int dev, StreamPool **out)
{
    StreamPool &p = g_pool[dev];
    if (!p.ready) {
        cudaError_t e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming);
        for (int j = 0; j < BATCH_STREAMS && e == cudaSuccess; ++j) {
            e = cudaStreamCreateWithFlags(&p.s[j], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.join[j], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            for (int j = 0; j < BATCH_STREAMS; ++j) {
                if (p.s[j]) cudaStreamDestroy(p.s[j]);
                if (p.join[j]) cudaEventDestroy(p.join[j]);
                p.s[j] = nullptr;
                p.join[j] = nullptr;
            }
            if (p.fork) cudaEventDestroy(p.fork);
            p.fork = nullptr;
            return e;
        }
        p.ready = true;
    }
    *out = &p;
    return cudaSuccess;
}

}  // namespace
}  // namespace fibar

using namespace fibar;

extern "C" int fibar_readout_batch(fibar_t *const *hs, const uint64_t *t_us, float *const *outs, size_t n,
                                   void *const *done_events, int *status, void *cuda_stream)
{
    if (n == 0) return FIBAR_OK;
    if (!hs || !t_us || !outs || n > BATCH_MAX) return FIBAR_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= BATCH_MAX_DEVICES) return FIBAR_EINVAL;
    std::vector<fibar_t *> sorted(hs, hs + n);
    for (fibar_t *h : sorted)
        if (!h || h->device != dev) return FIBAR_EINVAL;
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return FIBAR_EINVAL;

    std::lock_guard<std::mutex> lock(g_batch_mutex);
    StreamPool *pool = nullptr;
    cudaError_t e = pool_ready(dev, &pool);
    if (e != cudaSuccess) return FIBAR_ECUDA;

    // longest-processing-time-first assignment to the pool streams
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return hs[a]->pending_upper > hs[b]->pending_upper; });
    unsigned long long load[BATCH_STREAMS] = {};
    std::vector<int> lane(n);
    for (size_t i : order) {
        int j = (int)(std::min_element(load, load + BATCH_STREAMS) - load);
        lane[i] = j;
        load[j] += hs[i]->pending_upper + READOUT_FIXED_COST;
    }

    cudaStream_t caller = (cudaStream_t)cuda_stream;
    e = cudaEventRecord(pool->fork, caller);
    bool used[BATCH_STREAMS] = {};
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
        const int j = lane[i];
        if (!used[j]) {
            e = cudaStreamWaitEvent(pool->s[j], pool->fork, 0);
            used[j] = true;
        }
    }
    if (e != cudaSuccess) {
        if (status)
            for (size_t i = 0; i < n; ++i) status[i] = FIBAR_ECUDA;
        return FIBAR_ECUDA;
    }

    std::vector<int> rcs(n, FIBAR_OK);
    for (size_t i : order) {
        cudaStream_t s = pool->s[lane[i]];
        int rc = fibar_readout(hs[i], t_us[i], outs[i], 1, s);
        if (rc == FIBAR_OK && done_events && done_events[i]) {
            if (cudaEventRecord((cudaEvent_t)done_events[i], s) != cudaSuccess) {
                hs[i]->err = "readout_batch: recording the completion event failed";
                rc = FIBAR_ECUDA;
            }
        }
        rcs[i] = rc;
    }
    // join: the caller's stream waits for every pool stream used
    for (int j = 0; j < BATCH_STREAMS; ++j) {
        if (!used[j]) continue;
        cudaError_t ej = cudaEventRecord(pool->join[j], pool->s[j]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(caller, pool->join[j], 0);
        if (ej != cudaSuccess && e == cudaSuccess) e = ej;
    }
    int first = FIBAR_OK;
    for (size_t i = 0; i < n; ++i) {
        if (status) status[i] = rcs[i];
        if (rcs[i] != FIBAR_OK && first == FIBAR_OK) first = rcs[i];
    }
    if (first == FIBAR_OK && e != cudaSuccess) first = FIBAR_ECUDA;
    return first;
}
