// fibar_group: read-outs of a fixed set of handles, each member's read-out one launch of
// a CUDA graph captured once.
//
// A handle's read-out is a chain of about a dozen dependent kernels (decode, sort, walk,
// detector, blur, image, commit).  Issued from the host one launch at a time, the chains
// of many small streams leave the GPU waiting on the host's launch calls, and chains
// that each take a short batch are bound by their own latency, not by the device.  A
// group therefore
//   - captures each member's chain once into a graph, with the parts that change between
//     read-outs (the packets to decode, the read-out time, the image pointer, the carry
//     slot) read by the kernels from the member's descriptor in device memory;
//   - gives each member its own CUDA stream, so that the chains of different members -
//     of the same call and of consecutive calls - run side by side, while one member's
//     read-outs stay in order.
// The descriptor of a member's c-th commit (read-out or flush) is written by the host
// into slot c mod DESC_RING of a ring in mapped page-locked memory; the chain's first
// kernel (k_desc_fetch) copies slot (commits so far) mod DESC_RING, which the device
// knows from its own commit counter, into device memory.  A call costs the host one
// graph launch and one stream wait per member, whatever the chain's length.
//
// Latency: k_desc_fetch and the commit kernel stamp the GPU's global timer into mapped
// memory; an image's latency is its commit stamp minus the earliest fetch stamp of its
// call.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fibar_internal.cuh"

using namespace fibar;

namespace {

constexpr unsigned DESC_RING = 16;        // descriptor slots per member
constexpr unsigned GROUP_TICKETS = 4096;  // calls whose latency stamps are kept
constexpr size_t GROUP_MAX = 1024;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long ns;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
    return ns;
}

// Copy the descriptor of this read-out (the slot of the handle's commit number) from the
// mapped host ring into device memory, and stamp the chain's start.
__global__ void __launch_bounds__(256) k_desc_fetch(const Ctrl *ctrl, const ReadDesc *ring, ReadDesc *dst)
{
    const unsigned slot = (ctrl->batch_no - 1u) % DESC_RING;
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(ring + slot);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
    constexpr unsigned WORDS = sizeof(ReadDesc) / 8;
    for (unsigned i = threadIdx.x; i < WORDS; i += blockDim.x) d[i] = src[i];
    if (threadIdx.x == 0) {
        unsigned long long *b = ring[slot].stamp_begin;
        if (b) *(volatile unsigned long long *)b = global_ns();
    }
}
static_assert(sizeof(ReadDesc) % 8 == 0, "descriptor copied in 8-byte words");

struct Member {
    fibar_t *h = nullptr;
    cudaStream_t s = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long version = 0;
    unsigned long long chain_launches = 0;  // kernels per read-out (k_desc_fetch included)
    bool pdl = false;                       // captured with programmatic edges
    bool used_since_join = false;
};

}  // namespace

struct fibar_group_s {
    std::vector<Member> mem;
    int device = -1;
    ReadDesc *d_desc = nullptr;                      // one device descriptor per member
    ReadDesc *h_ring = nullptr, *hd_ring = nullptr;  // n x DESC_RING, host / device view
    unsigned long long *h_stamps = nullptr, *d_stamps = nullptr;  // GROUP_TICKETS x n x 2
    std::vector<std::vector<uint32_t>> ticket_members;
    unsigned long long next_ticket = 0;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    unsigned long long launches = 0, builds = 0;
    std::string err;
};

namespace {

int gfail(fibar_group_t *g, int code, const std::string &msg)
{
    g->err = msg;
    return code;
}

int gcuda(fibar_group_t *g, cudaError_t e, const char *where)
{
    g->err = std::string(where) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return FIBAR_ECUDA;
}

// Capture member i's chain (k_desc_fetch, then the read-out's kernels) into a graph.
int capture_member(fibar_group_t *g, size_t i, bool pdl, cudaGraphExec_t *exec_out, unsigned long long *nk_out)
{
    Member &mb = g->mem[i];
    fibar_t *h = mb.h;
    cudaStream_t cap = mb.s;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return gcuda(g, e, "group: begin capture");
    const unsigned long long l0 = h->launches;
    k_desc_fetch<<<1, 256, 0, cap>>>(h->b.ctrl, g->hd_ring + i * DESC_RING, g->d_desc + i);
    e = cudaGetLastError();
    SegTable dummy;
    memset(&dummy, 0, sizeof(dummy));
    pdl_enabled = pdl;
    const int rc = e == cudaSuccess ? enqueue_readout_chain(h, dummy, nullptr, g->d_desc + i, cap, false) : FIBAR_OK;
    pdl_enabled = true;
    *nk_out = h->launches - l0 + 1;
    h->launches = l0;
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cap, &graph);
    if (e != cudaSuccess || rc != FIBAR_OK || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return gcuda(g, e, "group: descriptor fetch");
        if (rc != FIBAR_OK) return gfail(g, rc, "group: capturing member " + std::to_string(i) + ": " + h->err);
        return gcuda(g, ee, "group: end capture");
    }
    e = cudaGraphInstantiate(exec_out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return gcuda(g, e, "group: instantiate");
    return FIBAR_OK;
}

// (Re)build member i's graph.  Launches of the previous graph still queued on the
// member's stream keep it alive until they complete.  Programmatic edges first, plain
// edges if the driver refuses them.
int build_member(fibar_group_t *g, size_t i)
{
    Member &mb = g->mem[i];
    cudaGraphExec_t ex = nullptr;
    unsigned long long nk = 0;
    bool pdl = true;
    int rc = capture_member(g, i, true, &ex, &nk);
    if (rc != FIBAR_OK) {
        pdl = false;
        rc = capture_member(g, i, false, &ex, &nk);
    }
    if (rc != FIBAR_OK) return rc;
    if (mb.exec) cudaGraphExecDestroy(mb.exec);
    mb.exec = ex;
    mb.chain_launches = nk;
    mb.pdl = pdl;
    mb.version = mb.h->config_version;
    g->builds += 1;
    return FIBAR_OK;
}

}  // namespace

extern "C" void fibar_group_destroy(fibar_group_t *g)
{
    if (!g) return;
    if (g->device >= 0) cudaSetDevice(g->device);
    for (Member &mb : g->mem) {
        if (mb.s) cudaStreamSynchronize(mb.s);
        if (mb.exec) cudaGraphExecDestroy(mb.exec);
        if (mb.s) cudaStreamDestroy(mb.s);
    }
    for (cudaEvent_t ev : g->ev_join)
        if (ev) cudaEventDestroy(ev);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->d_desc) cudaFree(g->d_desc);
    if (g->h_ring) cudaFreeHost(g->h_ring);
    if (g->h_stamps) cudaFreeHost(g->h_stamps);
    delete g;
}

extern "C" int fibar_group_create(fibar_t *const *hs, size_t n, fibar_group_t **out)
{
    if (!out) return FIBAR_EINVAL;
    *out = nullptr;
    if (!hs || n == 0 || n > GROUP_MAX) return FIBAR_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FIBAR_ECUDA;
    std::vector<fibar_t *> sorted(hs, hs + n);
    for (fibar_t *h : sorted)
        if (!h || h->device != dev) return FIBAR_EINVAL;
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return FIBAR_EINVAL;

    fibar_group_t *g = new (std::nothrow) fibar_group_s();
    if (!g) return FIBAR_ENOMEM;
    g->mem.resize(n);
    g->ev_join.assign(n, nullptr);
    g->ticket_members.resize(GROUP_TICKETS);
    g->device = dev;
    const size_t ring_bytes = n * DESC_RING * sizeof(ReadDesc);
    const size_t stamp_bytes = (size_t)GROUP_TICKETS * n * 2 * sizeof(unsigned long long);
    cudaError_t e = cudaMalloc((void **)&g->d_desc, n * sizeof(ReadDesc));
    if (e == cudaSuccess) e = cudaMemset(g->d_desc, 0, n * sizeof(ReadDesc));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&g->h_ring, ring_bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&g->hd_ring, g->h_ring, 0);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&g->h_stamps, stamp_bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&g->d_stamps, g->h_stamps, 0);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming);
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
        g->mem[i].h = hs[i];
        e = cudaStreamCreateWithFlags(&g->mem[i].s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        fibar_group_destroy(g);
        return e == cudaErrorMemoryAllocation ? FIBAR_ENOMEM : FIBAR_ECUDA;
    }
    memset(g->h_ring, 0, ring_bytes);
    memset(g->h_stamps, 0, stamp_bytes);
    for (size_t i = 0; i < n; ++i)
        if (build_member(g, i) != FIBAR_OK) {
            fibar_group_destroy(g);
            return FIBAR_ECUDA;
        }
    *out = g;
    return FIBAR_OK;
}

extern "C" int fibar_group_readout(fibar_group_t *g, const uint32_t *members, const uint64_t *t_us,
                                   float *const *outs, size_t m, int *status, uint64_t *ticket, void *cuda_stream)
{
    if (!g) return FIBAR_EINVAL;
    if (m == 0) return FIBAR_OK;
    const size_t n = g->mem.size();
    if (!members || !t_us || !outs || m > n) return gfail(g, FIBAR_EINVAL, "group_readout: bad arguments");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device)
        return gfail(g, FIBAR_EINVAL, "group_readout: not the group's device");
    // every check before anything is enqueued: a failing entry leaves all members untouched
    std::vector<unsigned char> seen(n, 0);
    int first = FIBAR_OK;
    for (size_t k = 0; k < m; ++k) {
        int rc = FIBAR_OK;
        const uint32_t i = members[k];
        if (i >= n || seen[i]) {
            rc = FIBAR_EINVAL;
        } else {
            seen[i] = 1;
            fibar_t *h = g->mem[i].h;
            if (!outs[k] || ((uintptr_t)outs[k] & 15) != 0)
                rc = FIBAR_EINVAL, h->err = "group_readout: output null or not 16-byte aligned";
            else if (h->have_readout && t_us[k] < h->last_readout)
                rc = FIBAR_EORDER, h->err = "readout: time earlier than the previous read-out";
        }
        if (status) status[k] = rc;
        if (rc != FIBAR_OK && first == FIBAR_OK) first = rc;
    }
    if (first != FIBAR_OK) return gfail(g, first, "group_readout: an entry failed its checks (see status)");
    for (size_t k = 0; k < m; ++k) {
        const uint32_t i = members[k];
        if (g->mem[i].h->config_version != g->mem[i].version) {
            const int rc = build_member(g, i);
            if (rc != FIBAR_OK) return rc;
        }
    }

    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the members' work starts after what the caller queued so far (its packets)
    cudaError_t e = cudaEventRecord(g->ev_fork, s);
    if (e != cudaSuccess) return gcuda(g, e, "group_readout: fork event");
    const unsigned long long tk = g->next_ticket;
    const unsigned ts = (unsigned)(tk % GROUP_TICKETS);
    unsigned long long *stamps = g->d_stamps + (size_t)ts * n * 2;
    for (size_t k = 0; k < m; ++k) {
        const uint32_t i = members[k];
        Member &mb = g->mem[i];
        fibar_t *h = mb.h;
        // this commit's descriptor slot was last read by commit c - DESC_RING
        const unsigned long long c = h->commits;
        if (c >= DESC_RING &&
            (unsigned long long)__atomic_load_n(&h->snap_host[1], __ATOMIC_ACQUIRE) + DESC_RING < c + 1) {
            e = cudaStreamSynchronize(mb.s);
            if (e != cudaSuccess) return gcuda(g, e, "group_readout: descriptor ring");
        }
        ReadDesc &d = g->h_ring[i * DESC_RING + c % DESC_RING];
        fill_segtable(h, t_us[k], d.t);
        d.out = outs[k];
        d.stamp_begin = stamps + 2 * i;
        d.stamp = stamps + 2 * i + 1;
        e = cudaStreamWaitEvent(mb.s, g->ev_fork, 0);
        const bool host_packets = h->copy_pending;
        if (e == cudaSuccess && host_packets) {
            // host packets of this member: the copy stream's work comes first
            e = cudaEventRecord(h->ev_copied, h->copy_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(mb.s, h->ev_copied, 0);
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(mb.exec, mb.s);
        if (e == cudaSuccess && host_packets) {
            // the staging buffer is free once this read-out has run
            e = cudaEventRecord(h->ev_free[h->staging_cur], mb.s);
            h->staging_cur ^= 1;
            h->copy_pending = false;
        }
        if (e != cudaSuccess) return gcuda(g, e, "group_readout: launch");
        mb.used_since_join = true;
        readout_committed(h);
        h->have_readout = true;
        h->last_readout = t_us[k];
        h->readouts += 1;
        h->launches += mb.chain_launches;
    }
    g->next_ticket = tk + 1;
    g->launches += 1;
    g->ticket_members[ts].assign(members, members + m);
    if (ticket) *ticket = tk;
    return FIBAR_OK;
}

extern "C" int fibar_group_join(fibar_group_t *g, void *cuda_stream)
{
    if (!g) return FIBAR_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    for (size_t i = 0; i < g->mem.size(); ++i) {
        Member &mb = g->mem[i];
        if (!mb.used_since_join) continue;
        cudaError_t e = cudaEventRecord(g->ev_join[i], mb.s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g->ev_join[i], 0);
        if (e != cudaSuccess) return gcuda(g, e, "group_join");
        mb.used_since_join = false;
    }
    return FIBAR_OK;
}

extern "C" int fibar_group_latency(fibar_group_t *g, uint64_t ticket, float *ms, size_t m)
{
    if (!g) return FIBAR_EINVAL;
    if (ticket >= g->next_ticket || g->next_ticket - ticket > GROUP_TICKETS)
        return gfail(g, FIBAR_EINVAL, "group_latency: unknown or expired ticket");
    const unsigned ts = (unsigned)(ticket % GROUP_TICKETS);
    const std::vector<uint32_t> &mem = g->ticket_members[ts];
    if (!ms || m != mem.size()) return gfail(g, FIBAR_EINVAL, "group_latency: one value per member read out");
    for (uint32_t i : mem) {
        const cudaError_t e = cudaStreamSynchronize(g->mem[i].s);
        if (e != cudaSuccess) return gcuda(g, e, "group_latency: sync");
    }
    const size_t n = g->mem.size();
    const volatile unsigned long long *st = g->h_stamps + (size_t)ts * n * 2;
    unsigned long long t0 = ~0ull;
    for (uint32_t i : mem) t0 = std::min(t0, (unsigned long long)st[2 * i]);
    for (size_t k = 0; k < m; ++k) {
        const unsigned long long t1 = st[2 * mem[k] + 1];
        ms[k] = t1 >= t0 ? (float)((double)(t1 - t0) * 1e-6) : 0.f;
    }
    return FIBAR_OK;
}

extern "C" int fibar_group_stats(fibar_group_t *g, fibar_group_stats_t *st)
{
    if (!g || !st) return FIBAR_EINVAL;
    st->members = g->mem.size();
    st->graph_launches = g->launches;
    st->builds = g->builds;
    unsigned long long k = 0;
    int pdl = 1;
    for (const Member &mb : g->mem) {
        k += mb.chain_launches;
        pdl &= mb.pdl ? 1 : 0;
    }
    st->graph_kernels = k;
    st->programmatic_edges = pdl;
    return FIBAR_OK;
}

extern "C" const char *fibar_group_last_error(fibar_group_t *g)
{
    return g ? g->err.c_str() : "null group";
}
