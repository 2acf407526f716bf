// fibar_group: read-outs of a fixed set of handles as one CUDA graph launch.
//
// A handle's read-out is a chain of about a dozen dependent kernels (decode, sort, walk,
// detector, blur, image, commit).  Issued from the host one launch at a time, the chains
// of many small streams leave the GPU waiting on the host's launch calls.  A group
// captures each member's chain once into one graph, with the parts that change between
// read-outs - the packets to decode (its segment table), the image pointer and the carry
// slot - read by the kernels from a per-member descriptor in device memory:
//
//   k_group_begin -> IF(active[0]) { chain of member 0 }
//                 -> IF(active[1]) { chain of member 1 }
//                 -> ...                                   (all side by side)
//
// One conditional node per member.  A read-out of any subset of the members is then one
// host-to-device copy of the descriptors (from a ring of pinned host slots) and one graph
// launch; k_group_begin sets each member's condition from the copied flags, and the
// chains of the members read out run concurrently.  Each chain's commit kernel stamps
// the GPU's global timer into mapped host memory, which gives every image's latency
// from the launch's start without an event per member.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fibar_internal.cuh"

using namespace fibar;

namespace {

constexpr unsigned GROUP_RING = 8;       // pinned descriptor slots (copies in flight)
constexpr unsigned GROUP_TICKETS = 256;  // launches whose latency stamps are kept
constexpr size_t GROUP_MAX = 1024;

struct GroupHead {
    unsigned long long *start_stamp;  // %globaltimer at the launch's start
    unsigned n;
    unsigned pad;
};

__global__ void k_group_begin(const GroupHead *head, const unsigned *active,
                              const cudaGraphConditionalHandle *cond, unsigned n)
{
    if (threadIdx.x == 0) {
        unsigned long long ns;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
        *(volatile unsigned long long *)head->start_stamp = ns;
    }
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) cudaGraphSetConditional(cond[i], active[i] ? 1u : 0u);
}

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

}  // namespace

struct fibar_group_s {
    std::vector<fibar_t *> hs;
    std::vector<unsigned long long> versions;        // members' config_version at capture
    std::vector<unsigned long long> chain_launches;  // kernels in each member's chain
    int device = -1;
    size_t off_active = 0, off_desc = 0, blk_bytes = 0;
    unsigned char *d_blk = nullptr;   // descriptors on the device
    unsigned char *h_ring = nullptr;  // GROUP_RING pinned slots of blk_bytes
    cudaEvent_t ev_slot[GROUP_RING] = {};
    unsigned long long slot_uses = 0;
    cudaGraphConditionalHandle *d_cond = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    bool pdl = false;                   // chains captured with programmatic edges
    unsigned long long *h_stamps = nullptr, *d_stamps = nullptr;  // GROUP_TICKETS x (1 + n)
    cudaEvent_t ev_ticket[GROUP_TICKETS] = {};
    std::vector<std::vector<uint32_t>> ticket_members;
    unsigned long long next_ticket = 0;
    cudaStream_t last_stream = nullptr;
    bool have_last = false;
    unsigned long long launches = 0, rebuilds = 0, kernels = 0;
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

void drop_graph(fibar_group_t *g)
{
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->exec = nullptr;
    g->graph = nullptr;
}

// Capture every member's chain under one conditional node each and instantiate.
int build_graph(fibar_group_t *g, bool pdl)
{
    drop_graph(g);
    const size_t n = g->hs.size();
    cudaError_t e = cudaGraphCreate(&g->graph, 0);
    if (e != cudaSuccess) return gcuda(g, e, "group: graph");
    std::vector<cudaGraphConditionalHandle> cond(n);
    for (size_t i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaGraphConditionalHandleCreate(&cond[i], g->graph, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_cond, cond.data(), n * sizeof(cudaGraphConditionalHandle), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return gcuda(g, e, "group: conditional handles");

    const GroupHead *head = reinterpret_cast<const GroupHead *>(g->d_blk);
    const unsigned *active = reinterpret_cast<const unsigned *>(g->d_blk + g->off_active);
    const cudaGraphConditionalHandle *dc = g->d_cond;
    unsigned nn = (unsigned)n;
    void *args[] = {(void *)&head, (void *)&active, (void *)&dc, (void *)&nn};
    cudaKernelNodeParams kn = {};
    kn.func = (void *)k_group_begin;
    kn.gridDim = dim3(1);
    kn.blockDim = dim3(256);
    kn.kernelParams = args;
    cudaGraphNode_t root = nullptr;
    e = cudaGraphAddKernelNode(&root, g->graph, nullptr, 0, &kn);
    if (e != cudaSuccess) return gcuda(g, e, "group: root node");

    ReadDesc *desc = reinterpret_cast<ReadDesc *>(g->d_blk + g->off_desc);
    SegTable dummy;
    memset(&dummy, 0, sizeof(dummy));
    g->kernels = 1;
    for (size_t i = 0; i < n; ++i) {
        fibar_t *h = g->hs[i];
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond[i];
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        e = cudaGraphAddNode(&node, g->graph, &root, nullptr, 1, &np);
        if (e != cudaSuccess) return gcuda(g, e, "group: conditional node");
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(g->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return gcuda(g, e, "group: begin capture");
        const unsigned long long l0 = h->launches;
        pdl_enabled = pdl;
        const int rc = enqueue_readout_chain(h, dummy, nullptr, desc + i, g->cap, false);
        pdl_enabled = true;
        g->chain_launches[i] = h->launches - l0;
        h->launches = l0;
        cudaGraph_t got = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(g->cap, &got);
        if (rc != FIBAR_OK) return gfail(g, rc, "group: capturing member " + std::to_string(i) + ": " + h->err);
        if (ee != cudaSuccess) return gcuda(g, ee, "group: end capture");
        g->kernels += g->chain_launches[i];
        g->versions[i] = h->config_version;
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) return gcuda(g, e, "group: instantiate");
    g->pdl = pdl;
    return FIBAR_OK;
}

// Programmatic edges first; a driver that refuses them inside conditional bodies gets
// plain edges.
int build(fibar_group_t *g)
{
    int rc = build_graph(g, true);
    if (rc != FIBAR_OK) rc = build_graph(g, false);
    if (rc == FIBAR_OK) g->rebuilds += 1;
    return rc;
}

}  // namespace

extern "C" void fibar_group_destroy(fibar_group_t *g)
{
    if (!g) return;
    if (g->device >= 0) cudaSetDevice(g->device);
    // a launch still in flight keeps its graph alive until it completes
    drop_graph(g);
    for (cudaEvent_t &ev : g->ev_slot)
        if (ev) cudaEventSynchronize(ev), cudaEventDestroy(ev);
    for (cudaEvent_t &ev : g->ev_ticket)
        if (ev) cudaEventSynchronize(ev), cudaEventDestroy(ev);
    if (g->cap) cudaStreamDestroy(g->cap);
    if (g->d_blk) cudaFree(g->d_blk);
    if (g->d_cond) cudaFree(g->d_cond);
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
    g->hs.assign(hs, hs + n);
    g->versions.assign(n, 0);
    g->chain_launches.assign(n, 0);
    g->ticket_members.resize(GROUP_TICKETS);
    g->device = dev;
    g->off_active = align16(sizeof(GroupHead));
    g->off_desc = g->off_active + align16(n * sizeof(unsigned));
    g->blk_bytes = g->off_desc + n * sizeof(ReadDesc);
    cudaError_t e = cudaMalloc((void **)&g->d_blk, g->blk_bytes);
    if (e == cudaSuccess) e = cudaMemset(g->d_blk, 0, g->blk_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->d_cond, n * sizeof(cudaGraphConditionalHandle));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&g->h_ring, GROUP_RING * g->blk_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&g->h_stamps, GROUP_TICKETS * (n + 1) * sizeof(unsigned long long),
                          cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&g->d_stamps, g->h_stamps, 0);
    for (unsigned i = 0; i < GROUP_RING && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&g->ev_slot[i], cudaEventDisableTiming);
    for (unsigned i = 0; i < GROUP_TICKETS && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&g->ev_ticket[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fibar_group_destroy(g);
        return e == cudaErrorMemoryAllocation ? FIBAR_ENOMEM : FIBAR_ECUDA;
    }
    memset(g->h_ring, 0, GROUP_RING * g->blk_bytes);
    memset(g->h_stamps, 0, GROUP_TICKETS * (n + 1) * sizeof(unsigned long long));
    if (build(g) != FIBAR_OK) {
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
    const size_t n = g->hs.size();
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
            fibar_t *h = g->hs[i];
            if (!outs[k] || ((uintptr_t)outs[k] & 15) != 0)
                rc = FIBAR_EINVAL, h->err = "group_readout: output null or not 16-byte aligned";
            else if (h->have_readout && t_us[k] < h->last_readout)
                rc = FIBAR_EORDER, h->err = "readout: time earlier than the previous read-out";
        }
        if (status) status[k] = rc;
        if (rc != FIBAR_OK && first == FIBAR_OK) first = rc;
    }
    if (first != FIBAR_OK) return gfail(g, first, "group_readout: an entry failed its checks (see status)");

    for (size_t i = 0; i < n; ++i)
        if (g->hs[i]->config_version != g->versions[i]) {
            const int rc = build(g);
            if (rc != FIBAR_OK) return rc;
            break;
        }

    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSuccess;
    // the previous launch read the device descriptors: order after it
    const unsigned long long tk = g->next_ticket;
    if (g->have_last && g->last_stream != s)
        e = cudaStreamWaitEvent(s, g->ev_ticket[(tk + GROUP_TICKETS - 1) % GROUP_TICKETS], 0);
    if (e != cudaSuccess) return gcuda(g, e, "group_readout: order after the previous launch");

    const unsigned j = (unsigned)(g->slot_uses % GROUP_RING);
    e = cudaEventSynchronize(g->ev_slot[j]);  // the copy out of this slot has run
    if (e != cudaSuccess) return gcuda(g, e, "group_readout: descriptor slot");
    unsigned char *blk = g->h_ring + (size_t)j * g->blk_bytes;
    const unsigned ts = (unsigned)(tk % GROUP_TICKETS);
    unsigned long long *stamps = g->d_stamps + (size_t)ts * (n + 1);
    GroupHead *head = reinterpret_cast<GroupHead *>(blk);
    head->start_stamp = stamps;
    head->n = (unsigned)n;
    unsigned *active = reinterpret_cast<unsigned *>(blk + g->off_active);
    memset(active, 0, n * sizeof(unsigned));
    ReadDesc *desc = reinterpret_cast<ReadDesc *>(blk + g->off_desc);
    size_t top = 0;
    for (size_t k = 0; k < m; ++k) {
        const uint32_t i = members[k];
        fibar_t *h = g->hs[i];
        active[i] = 1;
        fill_segtable(h, t_us[k], desc[i].t);
        desc[i].out = outs[k];
        desc[i].stamp = stamps + 1 + i;
        top = std::max(top, (size_t)i + 1);
        if (h->copy_pending) {
            // host packets of this member: the copy stream's work comes first
            e = cudaEventRecord(h->ev_copied, h->copy_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_copied, 0);
            if (e != cudaSuccess) return gcuda(g, e, "group_readout: wait for host packets");
        }
    }
    e = cudaMemcpyAsync(g->d_blk, blk, g->off_desc + top * sizeof(ReadDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev_slot[j], s);
    g->slot_uses += 1;
    if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev_ticket[ts], s);
    if (e != cudaSuccess) return gcuda(g, e, "group_readout: launch");
    g->next_ticket = tk + 1;
    g->have_last = true;
    g->last_stream = s;
    g->launches += 1;
    g->ticket_members[ts].assign(members, members + m);
    for (size_t k = 0; k < m; ++k) {
        fibar_t *h = g->hs[members[k]];
        if (h->copy_pending) {
            // the staging buffer is free once this launch has run
            e = cudaEventRecord(h->ev_free[h->staging_cur], s);
            if (e != cudaSuccess) return gcuda(g, e, "group_readout: staging event");
            h->staging_cur ^= 1;
            h->copy_pending = false;
        }
        readout_committed(h);
        h->have_readout = true;
        h->last_readout = t_us[k];
        h->readouts += 1;
        h->launches += g->chain_launches[members[k]];
    }
    if (ticket) *ticket = tk;
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
    const cudaError_t e = cudaEventSynchronize(g->ev_ticket[ts]);
    if (e != cudaSuccess) return gcuda(g, e, "group_latency: sync");
    const size_t n = g->hs.size();
    const volatile unsigned long long *st = g->h_stamps + (size_t)ts * (n + 1);
    const unsigned long long t0 = st[0];
    for (size_t k = 0; k < m; ++k) {
        const unsigned long long t1 = st[1 + mem[k]];
        ms[k] = t1 >= t0 ? (float)((double)(t1 - t0) * 1e-6) : 0.f;
    }
    return FIBAR_OK;
}

extern "C" int fibar_group_stats(fibar_group_t *g, fibar_group_stats_t *st)
{
    if (!g || !st) return FIBAR_EINVAL;
    st->members = g->hs.size();
    st->graph_launches = g->launches;
    st->builds = g->rebuilds;
    st->graph_kernels = g->kernels;
    st->programmatic_edges = g->pdl ? 1 : 0;
    return FIBAR_OK;
}

extern "C" const char *fibar_group_last_error(fibar_group_t *g)
{
    return g ? g->err.c_str() : "null group";
}
