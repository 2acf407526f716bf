// Host side of the C ABI declared in include/fibar.h.
//
// A read-out (or flush) enqueues, on the caller's stream and without host
// synchronisation:
//   decode -> radix sort by tile -> tile walk (links + IIR) -> detector (counts, pass 1,
//   pass 2, fixup) -> read-out image -> commit.
// Batch sizes live in device memory; every kernel sizes its loop from there, so the host
// never needs to know how many of the pending records a read-out applied.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "fibar_internal.cuh"

using namespace fibar;

namespace {

int fail(fibar_t *h, int code, const char *msg)
{
    if (h) h->err = msg;
    return code;
}

int cuda_fail(fibar_t *h, cudaError_t e, const char *where)
{
    if (h) {
        h->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return FIBAR_ECUDA;
}

unsigned long long next_pow2(unsigned long long v)
{
    unsigned long long p = 1;
    while (p < v) p <<= 1;
    return p;
}

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc((void **)p, std::max<size_t>(count, 1) * sizeof(T));
}

void free_all(fibar_t *h)
{
    Bufs &b = h->b;
    void *ptrs[] = {b.ctrl, b.pbar, b.L, b.last_pix, b.last_tile, b.staging, b.carry[0], b.carry[1],
                    b.dec_status, b.rec[0], b.rec[1], b.sort_hist, b.sort_base, b.sort_rows, b.sort_rowflag, b.sort_gtot, b.sort_gflag, b.sort_gcount,
                    b.qout, b.ring4, b.ring_pix, b.bucket_start, b.bucket_cnt, b.bucket_order, b.dMt, b.det_base, b.det_prof, b.band_ctr, b.E0, b.E1, b.E2, b.p2_ids, b.merged, b.unm_bits,
                    b.out_staging, b.dbg_cnt, b.plist, b.plnb, b.lbl, b.lbo, b.s1_info, b.s1_linit,
                    b.popk, b.blur_ord, b.bk, b.bpix, b.bj, b.bval, b.sel_status, b.beta_pow};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->snap_host) cudaFreeHost(h->snap_host);
    h->snap_host = nullptr;
    if (h->gain_buf) cudaFree(h->gain_buf);
    h->gain_buf = nullptr;
    memset(&h->b, 0, sizeof(h->b));
}

}  // namespace

extern "C" void fibar_default_params(fibar_params_t *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->t_cut = 40.0;
    p->fill_num = 1;
    p->fill_den = 2;
    p->q_min = 0;
    p->q_init = 0;
    p->c_on = 1.0f;
    p->c_off = 1.0f;
    p->spatial_filter = 1;
    p->blur_mode = 0;
    p->chain_policy = 0;
    p->max_pending = 0;
}

namespace {

// The handle's derived constants: the filter coefficients (Eqs. 16-18), the kernel
// parameters and the buffer capacities.  Shared by fibar_create and fibar_memory_bytes.
struct Layout {
    fibar_params_t p;
    KParams kp;
    Bufs b;  // capacities only (no pointers)
    double alpha, beta;
    unsigned long long R;
    uint32_t sort_passes;
};

int derive_layout(uint32_t W, uint32_t H, const fibar_params_t *pp, Layout &lo)
{
    fibar_params_t p;
    if (pp) p = *pp; else fibar_default_params(&p);
    const unsigned long long npix = (unsigned long long)W * H;
    if (W == 0 || H == 0 || npix > (1ull << 24)) return FIBAR_EINVAL;
    if (!(p.t_cut > 4.0)) return FIBAR_EINVAL;
    if (p.fill_num == 0 || p.fill_den == 0 || p.fill_num > 255 || p.fill_den > 255) return FIBAR_EINVAL;
    if (!(p.c_on > 0.f) || !(p.c_off > 0.f) || !isfinite(p.c_on) || !isfinite(p.c_off)) return FIBAR_EINVAL;
    if (p.spatial_filter != 0 && p.spatial_filter != 1) return FIBAR_EINVAL;
    if (p.blur_mode < 0 || p.blur_mode > 2) return FIBAR_EINVAL;
    if (p.chain_policy < 0 || p.chain_policy > 2) return FIBAR_EINVAL;
    const unsigned long long qmin = p.q_min ? p.q_min : std::max(1ull, (npix + 1023) / 1024);
    const unsigned long long qinit = p.q_init ? p.q_init : qmin;
    if (qmin > npix || qinit < qmin || qinit > npix) return FIBAR_EINVAL;
    const unsigned long long maxp = p.max_pending ? p.max_pending : (8ull << 20);
    if (maxp > (1ull << 27)) return FIBAR_EINVAL;
    p.max_pending = (uint32_t)maxp;
    p.q_init = (uint32_t)qinit;
    lo.p = p;

    // Eqs. 16-18 in double, then rounded once to the FP32 filter coefficients
    const double w = 2.0 * M_PI / p.t_cut;
    const double c = cos(w);
    lo.alpha = (1.0 - sin(w)) / c;
    lo.beta = (2.0 - c) - sqrt((2.0 - c) * (2.0 - c) - 1.0);

    KParams &kp = lo.kp;
    memset(&kp, 0, sizeof(kp));
    kp.W = W;
    kp.H = H;
    kp.tiles_w = (W + 1) / 2;
    kp.tiles_h = (H + 1) / 2;
    kp.npix = (uint32_t)npix;
    kp.ntiles = kp.tiles_w * kp.tiles_h;
    kp.a = (float)lo.alpha;
    kp.oma = (float)(1.0 - lo.alpha);
    kp.b = (float)lo.beta;
    kp.g = (float)(0.5 * (1.0 + lo.beta));
    kp.log2b = (float)log2(lo.beta);
    kp.c_on = p.c_on;
    kp.c_off = p.c_off;
    kp.q_min = (uint32_t)qmin;
    kp.q_max = (uint32_t)npix;
    kp.numA = p.fill_num * 4u;
    kp.den = p.fill_den;
    kp.max_pending = (uint32_t)maxp;
    unsigned bits = 1;
    while ((1ull << bits) < kp.ntiles) ++bits;
    kp.key_bits = bits;
    // buckets of 2^lb consecutive tiles: the radix sort orders by bucket only, the bucket
    // walk sorts each bucket by the low lb bits in shared memory
    kp.lb = std::min<unsigned>(9u, bits);
    kp.nbuckets = (kp.ntiles + (1u << kp.lb) - 1) >> kp.lb;
    lo.sort_passes = (bits - kp.lb + RADIX_BITS - 1) / RADIX_BITS;
    kp.spatial = p.spatial_filter;
    kp.blur_mode = p.blur_mode;
    kp.chain_policy = p.chain_policy;
    // event ring: the batch plus everything a window (or a guessed window) can reach back
    lo.R = next_pow2(maxp + npix + 8ull * 256);
    kp.ring_mask = lo.R - 1;
    kp.live = lo.R - maxp;

    Bufs &b = lo.b;
    memset(&b, 0, sizeof(b));
    b.max_dec_tiles = (maxp + DEC_TILE - 1) / DEC_TILE + 1;
    b.max_sort_tiles = (maxp + SORT_TILE - 1) / SORT_TILE + 1;
    b.max_chunks = std::min<unsigned long long>((maxp + CHUNK - 1) / CHUNK, DET_MAX_CHUNKS) + 1;
    b.mt_rows = b.max_chunks;
    b.n_samples = b.max_chunks / DET_SAMPLE + 18;  // short batches take up to 16 samples
    b.max_pops = maxp + npix + 8;
    b.max_sel_tiles = (b.max_pops + 4095) / 4096 + 1;
    return FIBAR_OK;
}

// Every device buffer of a handle with layout lo, as f(pointer, element count).
template <class F>
void for_each_buffer(const Layout &lo, Bufs &b, F &&f)
{
    const unsigned long long npix = lo.kp.npix, maxp = lo.kp.max_pending, R = lo.R;
    const KParams &kp = lo.kp;
    f(b.ctrl, 1);
    f(b.pbar, npix);
    f(b.L, npix);
    f(b.last_pix, npix);
    f(b.last_tile, kp.ntiles);
    f(b.staging, maxp);
    f(b.carry[0], maxp);
    f(b.carry[1], maxp);
    f(b.dec_status, b.max_dec_tiles);
    f(b.rec[0], maxp);
    f(b.rec[1], maxp);
    f(b.sort_hist, SORT_MAX_PASSES * RADIX);
    f(b.sort_base, SORT_MAX_PASSES * RADIX);
    f(b.sort_rows, b.max_sort_tiles * RADIX);
    f(b.sort_rowflag, b.max_sort_tiles);
    f(b.sort_gtot, (b.max_sort_tiles / LB_GROUP + 1) * RADIX);
    f(b.sort_gflag, b.max_sort_tiles / LB_GROUP + 1);
    f(b.sort_gcount, b.max_sort_tiles / LB_GROUP + 1);
    f(b.out_staging, npix);
    f(b.bucket_start, kp.nbuckets);
    f(b.bucket_cnt, kp.nbuckets);
    f(b.bucket_order, kp.nbuckets);
    if (lo.p.spatial_filter) {
        f(b.qout, maxp);
        f(b.ring4, R);
        f(b.ring_pix, R);
        f(b.dMt, 2 * b.mt_rows * 256);
        f(b.det_base, 4 * b.mt_rows);
        f(b.det_prof, 2 * b.n_samples * 640);
        f(b.band_ctr, b.n_samples);
        f(b.E0, b.max_chunks);
        f(b.E1, b.max_chunks);
        f(b.E2, b.max_chunks);
        f(b.p2_ids, b.max_chunks);
        f(b.merged, b.max_chunks);
        f(b.unm_bits, b.max_chunks / 32 + 2);
    }
    if (lo.p.spatial_filter && lo.p.blur_mode == 0) {
        f(b.plist, maxp);
        f(b.plnb, maxp);
        f(b.lbl, maxp);
        f(b.lbo, maxp);
        f(b.s1_info, npix);
        f(b.s1_linit, npix);
        f(b.popk, b.max_pops);
        f(b.blur_ord, b.max_pops);
        f(b.bk, b.max_pops);
        f(b.bpix, b.max_pops);
        f(b.bj, b.max_pops);
        f(b.bval, b.max_pops);
        f(b.sel_status, b.max_sel_tiles);
        f(b.beta_pow, 64);
    }
}

}  // namespace

extern "C" int fibar_memory_bytes(uint32_t W, uint32_t H, const fibar_params_t *p, uint64_t *bytes)
{
    if (!bytes) return FIBAR_EINVAL;
    Layout lo;
    const int rc = derive_layout(W, H, p, lo);
    if (rc) return rc;
    Bufs b = lo.b;
    uint64_t total = 0;
    for_each_buffer(lo, b, [&](auto *ptr, unsigned long long n) {
        // cudaMalloc hands out whole 512-byte blocks (at least one per buffer)
        const uint64_t sz = (uint64_t)std::max<unsigned long long>(n, 1) * sizeof(*ptr);
        total += (sz + 511) & ~uint64_t(511);
    });
    *bytes = total;
    return FIBAR_OK;
}

extern "C" int fibar_create(uint32_t W, uint32_t H, const fibar_params_t *pp, fibar_t **out)
{
    if (!out) return FIBAR_EINVAL;
    *out = nullptr;
    Layout lo;
    if (derive_layout(W, H, pp, lo) != FIBAR_OK) return FIBAR_EINVAL;
    const fibar_params_t &p = lo.p;
    const unsigned long long npix = (unsigned long long)W * H;
    const unsigned long long qinit = p.q_init;

    fibar_t *h = new (std::nothrow) fibar_s();
    if (!h) return FIBAR_ENOMEM;
    h->params = p;
    h->W = W;
    h->H = H;
    cudaGetDevice(&h->device);
    h->alpha = lo.alpha;
    h->beta = lo.beta;
    h->kp = lo.kp;
    const KParams &kp = h->kp;
    h->sort_passes = lo.sort_passes;
    h->R = lo.R;
    h->b = lo.b;
    Bufs &b = h->b;

    cudaError_t e = cudaSuccess;
    for_each_buffer(lo, b, [&](auto *&ptr, unsigned long long n) {
        if (e == cudaSuccess) e = dalloc(&ptr, n);
    });
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&h->snap_host, 4 * sizeof(unsigned), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        h->snap_host[0] = 0u;
        h->snap_host[1] = 0u;
        h->snap_host[2] = 0u;
        e = cudaHostGetDevicePointer((void **)&b.snap, h->snap_host, 0);
    }
    if (e != cudaSuccess) {
        free_all(h);
        cudaGetLastError();
        delete h;
        return FIBAR_ENOMEM;
    }
    cudaStream_t s = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(b.pbar, 0, npix * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.L, 0, npix * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.last_pix, 0xFF, npix * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.last_tile, 0xFF, kp.ntiles * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.dec_status, 0, b.max_dec_tiles * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.sort_hist, 0, SORT_MAX_PASSES * RADIX * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.sort_rowflag, 0, b.max_sort_tiles * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.sort_gflag, 0, (b.max_sort_tiles / LB_GROUP + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.sort_gcount, 0, (b.max_sort_tiles / LB_GROUP + 1) * 4, s);
    if (e == cudaSuccess && p.spatial_filter) e = cudaMemsetAsync(b.ring4, 0xFF, h->R * 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.bucket_start, 0, (size_t)kp.nbuckets * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.bucket_cnt, 0, (size_t)kp.nbuckets * 4, s);
    if (e == cudaSuccess && p.spatial_filter) e = cudaMemsetAsync(b.ring_pix, 0, h->R * 4, s);
    if (e == cudaSuccess && b.unm_bits) e = cudaMemsetAsync(b.unm_bits, 0, (b.max_chunks / 32 + 2) * 4, s);
    if (e == cudaSuccess && b.det_base) e = cudaMemsetAsync(b.det_base, 0, 4 * b.mt_rows * 4, s);
    if (e == cudaSuccess && b.s1_info) e = cudaMemsetAsync(b.s1_info, 0, npix * sizeof(int4), s);
    if (e == cudaSuccess && b.bval) e = cudaMemsetAsync(b.bval, 0, b.max_pops * 8, s);
    if (e == cudaSuccess && b.sel_status) e = cudaMemsetAsync(b.sel_status, 0, b.max_sel_tiles * 8, s);
    if (e == cudaSuccess && b.beta_pow) {
        float tab[64];
        double v = 1.0;
        for (int i = 0; i < 64; ++i) {
            tab[i] = (float)v;
            v *= h->beta;
        }
        e = cudaMemcpy(b.beta_pow, tab, sizeof(tab), cudaMemcpyHostToDevice);
    }
    h->launches = 0;
    if (e == cudaSuccess) e = launch_init(kp, b, s, h->launches);
    if (e == cudaSuccess) {
        // q_targ_0 = q_init as the ratio q_init / 1
        DetState d0{0, 0, 0, qinit, 1};
        e = cudaMemcpyAsync(&b.ctrl->det, &d0, sizeof(d0), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free_all(h);
        delete h;
        return FIBAR_ECUDA;
    }
    h->staging_used = 0;
    h->pending_upper = 0;
    h->commits = 0;
    h->pushed_since = 0;
    h->carry_slot = 0;
    h->have_readout = false;
    h->last_readout = 0;
    h->pushed = 0;
    h->readouts = 0;
    h->timing = false;
    h->ev_used = 0;
    memset(h->stage_ms, 0, sizeof(h->stage_ms));
    h->stage_calls = 0;
    *out = h;
    return FIBAR_OK;
}

extern "C" int fibar_debug_wait_timeout(fibar_t *h, uint32_t max_spins, void *cuda_stream)
{
    if (!h || max_spins == 0 || max_spins > (1u << 20)) return FIBAR_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned *flag = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&flag, sizeof(unsigned), s);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(h, FIBAR_ENOMEM, "debug_wait_timeout: allocation"); }
    e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = launch_probe_wait(h->b, flag, max_spins, s, h->launches);
    unsigned err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &h->b.ctrl->error, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    // clear this probe's flag again (the pipeline's own flags stay as they were)
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && (err & ERR_PROBE_WAIT)) {
        const unsigned keep = err & ~ERR_PROBE_WAIT;
        e = cudaMemcpyAsync(&h->b.ctrl->error, &keep, sizeof(unsigned), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFreeAsync(flag, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "debug_wait_timeout");
    if (err & ERR_PROBE_WAIT) {
        char msg[128];
        snprintf(msg, sizeof msg, "a bounded device wait gave up after %u polls (flags 0x%x)", max_spins, err);
        return fail(h, FIBAR_ETIMEOUT, msg);
    }
    return FIBAR_OK;
}

extern "C" int fibar_set_grid_share(fibar_t *h, uint32_t sms)
{
    if (!h) return FIBAR_EINVAL;
    if (h->kp.grid_sms != sms) h->config_version += 1;
    h->kp.grid_sms = sms;
    return FIBAR_OK;
}

extern "C" int fibar_set_pixel_gain(fibar_t *h, const float *gain, int on_device, void *cuda_stream)
{
    if (!h) return FIBAR_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!gain) {
        if (h->b.gain) h->config_version += 1;
        h->b.gain = nullptr;
        return FIBAR_OK;
    }
    const size_t npix = h->kp.npix;
    if (!on_device) {
        for (size_t i = 0; i < npix; ++i)
            if (!(gain[i] > 0.f) || !isfinite(gain[i]))
                return fail(h, FIBAR_EINVAL, "set_pixel_gain: every gain must be finite and > 0");
    } else if (((uintptr_t)gain & 3) != 0) {
        return fail(h, FIBAR_EINVAL, "set_pixel_gain: misaligned device array");
    }
    if (!h->gain_buf) {
        cudaError_t e = cudaMalloc((void **)&h->gain_buf, npix * sizeof(float));
        if (e != cudaSuccess) {
            h->gain_buf = nullptr;
            cudaGetLastError();
            return fail(h, FIBAR_ENOMEM, "set_pixel_gain: device allocation failed");
        }
    }
    cudaError_t e = cudaMemcpyAsync(h->gain_buf, gain, npix * sizeof(float),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_pixel_gain: copy");
    if (h->b.gain != h->gain_buf) h->config_version += 1;
    h->b.gain = h->gain_buf;
    return FIBAR_OK;
}

extern "C" void fibar_destroy(fibar_t *h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->copy_stream) {
        cudaStreamDestroy(h->copy_stream);
        cudaEventDestroy(h->ev_free[0]);
        cudaEventDestroy(h->ev_free[1]);
        cudaEventDestroy(h->ev_copied);
        cudaFree(h->staging2);
    }
    free_all(h);
    delete h->fill;
    delete h;
}

extern "C" const char *fibar_last_error(fibar_t *h)
{
    return h ? h->err.c_str() : "null handle";
}

extern "C" int fibar_push_events(fibar_t *h, const fibar_event_t *ev, size_t n, int on_device,
                                 void *cuda_stream)
{
    if (!h) return FIBAR_EINVAL;
    if (n == 0) return FIBAR_OK;
    if (!ev) return fail(h, FIBAR_EINVAL, "push: null event pointer");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (h->pending_upper + n > h->params.max_pending && h->commits &&
        __atomic_load_n(&h->snap_host[1], __ATOMIC_ACQUIRE) == (unsigned)h->commits) {
        // the last commit has run: its count of records left pending is current
        h->pending_upper = h->snap_host[0] + h->pushed_since;
    }
    if (h->pending_upper + n > h->params.max_pending) {
        // the bound may be stale: learn the true carry count before refusing
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "push: sync");
        unsigned carry = 0;
        e = cudaMemcpy(&carry, &h->b.ctrl->carry_n[h->carry_slot], 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "push: carry count");
        unsigned long long segs = 0;
        for (unsigned v : h->seg_n) segs += v;
        h->pending_upper = carry + segs;
        if (h->pending_upper + n > h->params.max_pending)
            return fail(h, FIBAR_ENOMEM, "push: pending capacity exceeded; read out or flush first");
    }
    if (on_device) {
        if (((uintptr_t)ev & 15) != 0) return fail(h, FIBAR_EINVAL, "push: device packet not 16-byte aligned");
        if (h->seg_ptr.size() >= (size_t)MAXSEG)
            return fail(h, FIBAR_ENOMEM, "push: too many pending device packets; read out or flush first");
        h->seg_ptr.push_back((const int4 *)ev);
        h->seg_n.push_back((unsigned)n);
    } else {
        if (h->staging_used + n > h->params.max_pending)
            return fail(h, FIBAR_ENOMEM, "push: host staging full; read out or flush first");
        if (!h->copy_stream) {
            cudaError_t e = cudaMalloc((void **)&h->staging2, (size_t)h->params.max_pending * sizeof(int4));
            if (e != cudaSuccess) {
                h->staging2 = nullptr;
                cudaGetLastError();
                return fail(h, FIBAR_ENOMEM, "push: second host staging buffer");
            }
            e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_free[0], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_free[1], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_copied, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(h, e, "push: copy stream");
        }
        int4 *buf = h->staging_cur ? h->staging2 : h->b.staging;
        if (!h->copy_pending) {
            // the decode that last read this buffer must have run
            cudaError_t e = cudaStreamWaitEvent(h->copy_stream, h->ev_free[h->staging_cur], 0);
            if (e != cudaSuccess) return cuda_fail(h, e, "push: wait for the staging buffer");
            h->copy_pending = true;
        }
        int4 *dst = buf + h->staging_used;
        cudaError_t e = cudaMemcpyAsync(dst, ev, n * sizeof(fibar_event_t), cudaMemcpyHostToDevice, h->copy_stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "push: host-to-device copy");
        if (!h->seg_ptr.empty() && h->seg_ptr.back() + h->seg_n.back() == dst) {
            h->seg_n.back() += (unsigned)n;
        } else {
            if (h->seg_ptr.size() >= (size_t)MAXSEG)
                return fail(h, FIBAR_ENOMEM, "push: too many pending packets; read out or flush first");
            h->seg_ptr.push_back(dst);
            h->seg_n.push_back((unsigned)n);
        }
        h->staging_used += n;
    }
    h->pending_upper += n;
    h->pushed_since += n;
    h->pushed += n;
    return FIBAR_OK;
}

extern "C" int fibar_push_batch(fibar_t *const *hs, const fibar_event_t *const *evs, const size_t *ns, size_t count,
                                int on_device, int *status, void *cuda_stream)
{
    if (count == 0) return FIBAR_OK;
    if (!hs || !evs || !ns) return FIBAR_EINVAL;
    int first = FIBAR_OK;
    for (size_t k = 0; k < count; ++k) {
        const int rc = hs[k] ? fibar_push_events(hs[k], evs[k], ns[k], on_device, cuda_stream) : FIBAR_EINVAL;
        if (status) status[k] = rc;
        if (rc != FIBAR_OK && first == FIBAR_OK) first = rc;
    }
    return first;
}

extern "C" int fibar_push_events_many(fibar_t *h, const fibar_event_t *const *evs, const size_t *ns, size_t count,
                                      int on_device, void *cuda_stream)
{
    if (!h) return FIBAR_EINVAL;
    if (count == 0) return FIBAR_OK;
    if (!evs || !ns) return fail(h, FIBAR_EINVAL, "push_many: null array");
    // runs of packets that follow each other in memory go in as one packet
    size_t i = 0;
    while (i < count) {
        const fibar_event_t *p = evs[i];
        size_t n = ns[i];
        size_t j = i + 1;
        while (j < count && p && evs[j] == p + n) n += ns[j++];
        const int rc = fibar_push_events(h, p, n, on_device, cuda_stream);
        if (rc != FIBAR_OK) return rc;
        i = j;
    }
    return FIBAR_OK;
}

namespace {

constexpr unsigned EV_SETS = 4096;  // read-outs whose stage events are kept

// Fold recorded stage events into the accumulated times (synchronises on them).
void fold_stage_events(fibar_t *h)
{
    for (unsigned i = 0; i < h->ev_used; ++i) {
        cudaEvent_t *e = &h->ev_pool[(size_t)i * (FIBAR_NSTAGES + 1)];
        cudaEventSynchronize(e[FIBAR_NSTAGES]);
        for (int st = 0; st < FIBAR_NSTAGES; ++st) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, e[st], e[st + 1]) == cudaSuccess) h->stage_ms[st] += ms;
        }
        h->stage_calls += 1;
    }
    h->ev_used = 0;
}

struct StageMarks {
    fibar_t *h;
    cudaStream_t s;
    cudaEvent_t *e;
    StageMarks(fibar_t *h_, cudaStream_t s_, bool on) : h(h_), s(s_), e(nullptr)
    {
        if (!on || !h->timing) return;
        if (h->ev_used == EV_SETS) fold_stage_events(h);
        e = &h->ev_pool[(size_t)h->ev_used * (FIBAR_NSTAGES + 1)];
        h->ev_used += 1;
    }
    void mark(int boundary)
    {
        if (e) cudaEventRecord(e[boundary], s);
    }
};

}  // namespace

namespace fibar {

// The pending packets of the next read-out, as its decode takes them.
void fill_segtable(const fibar_t *h, unsigned long long t_read, SegTable &T)
{
    memset(&T, 0, sizeof(T));
    T.nseg = (unsigned)h->seg_ptr.size();
    for (unsigned i = 0; i < T.nseg; ++i) {
        T.ptr[i] = h->seg_ptr[i];
        T.n[i] = h->seg_n[i];
    }
    T.carry_slot = (unsigned)h->carry_slot;
    T.carry = h->b.carry[h->carry_slot];
    T.carry_out = h->b.carry[1 - h->carry_slot];
    T.t_read = t_read;
}

// The kernels of one read-out, in order (out == nullptr: apply only, a flush).  With a
// descriptor d (a chain captured into a group's graph) the decode, the image and the
// commit take the read-out's table, image pointer and carry slot from device memory
// instead of T and out; nothing else of a read-out changes from call to call.
int enqueue_readout_chain(fibar_t *h, const SegTable &T, float *out, const ReadDesc *d, cudaStream_t s,
                          bool stage_marks)
{
    const KParams &kp = h->kp;
    const Bufs &b = h->b;
    unsigned long long &nl = h->launches;
    StageMarks mk(h, stage_marks ? s : nullptr, stage_marks);
    const SegTable *tdev = d ? &d->t : nullptr;
    float *const *outp = d ? &d->out : nullptr;

    mk.mark(FIBAR_STAGE_DECODE);
    cudaError_t e = launch_decode(kp, b, T, h->sort_passes, s, nl, tdev);
    if (e != cudaSuccess) return cuda_fail(h, e, "decode");
    if (h->copy_pending && !d) {
        // the staging buffer is free again once the decode has run; the next host packets
        // go to the other one
        e = cudaEventRecord(h->ev_free[h->staging_cur], s);
        if (e != cudaSuccess) return cuda_fail(h, e, "staging event");
        h->staging_cur ^= 1;
        h->copy_pending = false;
    }
    mk.mark(FIBAR_STAGE_SORT);
    e = launch_sort(kp, b, h->sort_passes, s, nl);
    if (e != cudaSuccess) return cuda_fail(h, e, "sort");
    const unsigned long long *sorted = b.rec[h->sort_passes & 1];
    mk.mark(FIBAR_STAGE_WALK);
    e = launch_walk(kp, b, sorted, h->sort_passes, s, nl);
    if (e != cudaSuccess) return cuda_fail(h, e, "walk");
    mk.mark(FIBAR_STAGE_DET_COUNTS);
    if (kp.spatial) e = launch_det_counts(kp, b, s, nl);
    mk.mark(FIBAR_STAGE_DET_PASS1);
    if (kp.spatial && e == cudaSuccess) e = launch_det_pass1(kp, b, s, nl);
    mk.mark(FIBAR_STAGE_DET_PASS2);
    if (kp.spatial && e == cudaSuccess) e = launch_det_pass2(kp, b, s, nl);
    mk.mark(FIBAR_STAGE_DET_FIX);
    if (kp.spatial && e == cudaSuccess) e = launch_det_fix(kp, b, s, nl);
    if (e != cudaSuccess) return cuda_fail(h, e, "detector");
    mk.mark(FIBAR_STAGE_S1);
    if (kp.spatial && kp.blur_mode == 0) {
        e = launch_s1(kp, b, s, nl);
        if (e != cudaSuccess) return cuda_fail(h, e, "S1 blur");
    }
    mk.mark(FIBAR_STAGE_READOUT);
    if (out || d) {
        if (kp.spatial && kp.blur_mode == 2 && h->fill)
            e = launch_fill_readout(*h->fill, kp, b, out, s, nl, outp);
        else
            e = launch_readout(kp, b, out, s, nl, outp);
        if (e != cudaSuccess) return cuda_fail(h, e, "readout");
    }
    mk.mark(FIBAR_STAGE_COMMIT);
    e = launch_commit(kp, b, 1 - (int)T.carry_slot, s, nl, d);
    if (e != cudaSuccess) return cuda_fail(h, e, "commit");
    mk.mark(FIBAR_NSTAGES);
    return FIBAR_OK;
}

// Host bookkeeping once a read-out's (or flush's) kernels are enqueued.
void readout_committed(fibar_t *h)
{
    h->carry_slot = 1 - h->carry_slot;
    h->seg_ptr.clear();
    h->seg_n.clear();
    h->staging_used = 0;
    h->commits += 1;
    h->pushed_since = 0;
}

}  // namespace fibar

namespace {

// Enqueue the whole per-read-out pipeline.  out == nullptr: apply only (flush).
int process(fibar_t *h, unsigned long long t_read, float *out, cudaStream_t s)
{
    SegTable T;
    fill_segtable(h, t_read, T);
    if (h->copy_pending) {
        // the read-out's host packets, copied on the internal stream
        cudaError_t e = cudaEventRecord(h->ev_copied, h->copy_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_copied, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "wait for the host packets");
    }
    const int rc = enqueue_readout_chain(h, T, out, nullptr, s, true);
    if (rc) return rc;
    readout_committed(h);
    return FIBAR_OK;
}

// After a synchronisation that covered the last commit: its copy of the error flags
// (mapped host memory, no device round trip).
int check_device_error(fibar_t *h)
{
    const unsigned err = __atomic_load_n(&h->snap_host[2], __ATOMIC_ACQUIRE);
    if (err) {
        char msg[128];
        snprintf(msg, sizeof msg, "a bounded device wait gave up (flags 0x%x)", err);
        return fail(h, FIBAR_ETIMEOUT, msg);
    }
    return FIBAR_OK;
}

}  // namespace

extern "C" int fibar_readout(fibar_t *h, uint64_t t_us, float *out, int on_device, void *cuda_stream)
{
    if (!h) return FIBAR_EINVAL;
    if (!out) return fail(h, FIBAR_EINVAL, "readout: null output");
    if (h->have_readout && t_us < h->last_readout)
        return fail(h, FIBAR_EORDER, "readout: time earlier than the previous read-out");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (on_device && ((uintptr_t)out & 3) != 0) return fail(h, FIBAR_EINVAL, "readout: misaligned output");
    float *dst = on_device ? out : h->b.out_staging;
    int rc = process(h, t_us, dst, s);
    if (rc) return rc;
    h->have_readout = true;
    h->last_readout = t_us;
    h->readouts += 1;
    if (!on_device) {
        cudaError_t e = cudaMemcpyAsync(out, h->b.out_staging, (size_t)h->kp.npix * sizeof(float),
                                        cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "readout: device-to-host copy");
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "readout: sync");
        return check_device_error(h);
    }
    return FIBAR_OK;
}

extern "C" int fibar_readout_host_async(fibar_t *h, uint64_t t_us, float *out, void *cuda_stream)
{
    if (!h) return FIBAR_EINVAL;
    if (!out) return fail(h, FIBAR_EINVAL, "readout_host_async: null output");
    if (h->have_readout && t_us < h->last_readout)
        return fail(h, FIBAR_EORDER, "readout: time earlier than the previous read-out");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int rc = process(h, t_us, h->b.out_staging, s);
    if (rc) return rc;
    h->have_readout = true;
    h->last_readout = t_us;
    h->readouts += 1;
    cudaError_t e = cudaMemcpyAsync(out, h->b.out_staging, (size_t)h->kp.npix * sizeof(float),
                                    cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "readout_host_async: device-to-host copy");
    return FIBAR_OK;
}

extern "C" int fibar_wait(fibar_t *h, void *cuda_stream)
{
    if (!h) return FIBAR_EINVAL;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "wait: sync");
    return h->commits ? check_device_error(h) : FIBAR_OK;
}

extern "C" int fibar_flush(fibar_t *h, void *cuda_stream)
{
    if (!h) return FIBAR_EINVAL;
    int rc = process(h, ~0ull, nullptr, (cudaStream_t)cuda_stream);
    if (rc) return rc;
    h->pending_upper = 0;
    return FIBAR_OK;
}

namespace {

int read_ctrl(fibar_t *h, Ctrl *c, cudaStream_t s)
{
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "sync");
    e = cudaMemcpy(c, h->b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "control block");
    unsigned long long segs = 0;
    for (unsigned v : h->seg_n) segs += v;
    h->pending_upper = c->carry_n[h->carry_slot] + segs;
    if (c->error) {
        char msg[128];
        snprintf(msg, sizeof msg, "a bounded device wait gave up (flags 0x%x)", c->error);
        return fail(h, FIBAR_ETIMEOUT, msg);
    }
    return FIBAR_OK;
}

unsigned long long q_targ_of(const fibar_t *h, const DetState &d)
{
    unsigned long long q = d.Y ? d.X / d.Y : h->kp.q_min;
    q = std::min<unsigned long long>(q, h->kp.q_max);
    q = std::max<unsigned long long>(q, h->kp.q_min);
    return q;
}

}  // namespace

extern "C" int fibar_stats(fibar_t *h, fibar_stats_t *st, void *cuda_stream)
{
    if (!h || !st) return FIBAR_EINVAL;
    Ctrl c;
    int rc = read_ctrl(h, &c, (cudaStream_t)cuda_stream);
    memset(st, 0, sizeof(*st));
    st->events_pushed = h->pushed;
    st->events_applied = c.base;
    st->events_dropped = c.dropped;
    st->events_pending = h->pending_upper;
    st->readouts = h->readouts;
    if (h->kp.spatial) {
        st->q = c.base - (unsigned long long)c.det.h;
        st->q_targ = q_targ_of(h, c.det);
        st->n_ap = c.det.nap;
        st->n_at = c.det.nat;
    }
    st->detector_fixups = c.fixups;
    st->kernel_launches = h->launches;
    st->detector_unmerged = c.unmerged_total;
    st->detector_pass2_steps = c.pass2_steps;
    st->detector_fix_steps = c.fix_steps;
    st->s1_blurs = c.s1_blurs;
    st->detector_big_pops = c.big_pops;
    st->detector_ring_misses = c.ring_misses;
    st->detector_recenters = c.recenters;
    st->iir_walk_pieces = c.walk_pieces;
    st->iir_scan_pieces = c.scan_pieces;
    return rc;
}

extern "C" int fibar_set_timing(fibar_t *h, int enable)
{
    if (!h) return FIBAR_EINVAL;
    if (enable && h->ev_pool.empty()) {
        h->ev_pool.resize((size_t)EV_SETS * (FIBAR_NSTAGES + 1));
        for (cudaEvent_t &e : h->ev_pool) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_fail(h, r, "set_timing: event");
        }
    }
    h->timing = enable != 0;
    return FIBAR_OK;
}

extern "C" int fibar_stage_times(fibar_t *h, fibar_stage_times_t *t, int reset, void *cuda_stream)
{
    if (!h || !t) return FIBAR_EINVAL;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stage_times: sync");
    fold_stage_events(h);
    for (int i = 0; i < FIBAR_NSTAGES; ++i) t->ms[i] = h->stage_ms[i];
    t->calls = h->stage_calls;
    if (reset) {
        memset(h->stage_ms, 0, sizeof(h->stage_ms));
        h->stage_calls = 0;
    }
    return FIBAR_OK;
}

extern "C" int fibar_debug_state(fibar_t *h, fibar_state_view_t *v, void *cuda_stream)
{
    if (!h || !v) return FIBAR_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Ctrl c;
    int rc = read_ctrl(h, &c, s);
    if (rc) return rc;
    const size_t npix = h->kp.npix;
    cudaError_t e = cudaSuccess;
    if (v->pbar) e = cudaMemcpy(v->pbar, h->b.pbar, npix * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v->L) e = cudaMemcpy(v->L, h->b.L, npix * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v->last_idx) e = cudaMemcpy(v->last_idx, h->b.last_pix, npix * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "debug_state copy");
    v->k = c.base;
    if (h->kp.spatial) {
        v->h = (unsigned long long)c.det.h;
        v->q = c.base - v->h;
        v->q_targ = q_targ_of(h, c.det);
        v->n_ap = c.det.nap;
        v->n_at = c.det.nat;
    } else {
        v->h = c.base;
        v->q = 0;
        v->q_targ = 0;
        v->n_ap = v->n_at = 0;
    }
    const bool want_cnt = v->cnt || v->tcnt || v->stale;
    if (want_cnt) {
        std::vector<uint32_t> cnt(npix, 0);
        if (h->kp.spatial && v->q > 0) {
            if (!h->b.dbg_cnt) {
                e = cudaMalloc((void **)&h->b.dbg_cnt, npix * 4);
                if (e != cudaSuccess) return cuda_fail(h, e, "debug_state alloc");
            }
            e = cudaMemsetAsync(h->b.dbg_cnt, 0, npix * 4, s);
            if (e == cudaSuccess) e = launch_debug_counts(h->kp, h->b, h->b.dbg_cnt, s, h->launches);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e == cudaSuccess) e = cudaMemcpy(cnt.data(), h->b.dbg_cnt, npix * 4, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(h, e, "debug_state counts");
        }
        if (v->cnt) memcpy(v->cnt, cnt.data(), npix * 4);
        if (v->tcnt) {
            memset(v->tcnt, 0, h->kp.ntiles);
            for (size_t i = 0; i < npix; ++i) {
                const size_t x = i % h->W, y = i / h->W;
                if (cnt[i]) v->tcnt[(y / 2) * h->kp.tiles_w + x / 2] += 1;
            }
        }
        if (v->stale) {
            std::vector<unsigned long long> last(npix);
            e = cudaMemcpy(last.data(), h->b.last_pix, npix * 8, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(h, e, "debug_state last");
            for (size_t i = 0; i < npix; ++i)
                v->stale[i] = (h->kp.spatial && last[i] != NONE64 && cnt[i] == 0) ? 1 : 0;
        }
    }
    return FIBAR_OK;
}
