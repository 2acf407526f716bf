// Internal declarations shared by the FIBAR CUDA translation units.
//
// Device data layout (one handle = one sensor stream):
//   per pixel  : pbar f32, L f32 (row-major), last_pix u64 (global index of the pixel's
//                last applied event, ~0 = none)
//   per tile   : last_tile u64 (2x2 tiles aligned at (0,0))
//   event ring : for global event index g, slot g & ring_mask holds
//                ring4 = {dP, dT, nP, nT}: distance to the previous / next event of the
//                same pixel and of the same tile (0xFFFFFFFF = none, or >= 2^32-1), and
//                ring_pix = pixel id.
//                The active event queue (Sec. 4.2) is always the index window [h, k].
//   batch      : qout[k] = queue length after the pops of step k (window [k+1-q, k]),
//                k the batch-relative event index (0 .. m-1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "../../include/fibar.h"

namespace fibar {

constexpr uint32_t SAT = 0xFFFFFFFFu;          // saturated / absent distance
constexpr unsigned long long NONE64 = ~0ull;   // "no event yet"
constexpr unsigned TMA_SPIN_LIMIT = 1u << 16;    // bounded waits on bulk-copy barriers (each try blocks a while)
constexpr int DEC_THREADS = 256;
constexpr int DEC_PER_THREAD = 16;
constexpr int DEC_TILE = DEC_THREADS * DEC_PER_THREAD;   // records per decode tile
constexpr int SORT_THREADS = 256;
constexpr int SORT_PER_THREAD = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_PER_THREAD;
constexpr int SORT_WARP_RANGE = SORT_TILE / (SORT_THREADS / 32);  // records ranked by one warp
constexpr int SORT_BLOCKS_PER_SM = 2;
constexpr int DEC_BLOCKS_PER_SM = 2;
constexpr int SORT_MAX_PASSES = 4;
constexpr int RADIX_BITS = 9;                  // sort digit width (max)
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int MAX_BUCKETS = 8192;              // buckets of <= 512 tiles (W*H <= 2^24)
constexpr int MAXSEG = 192;                    // pending device packets per read-out
constexpr uint32_t CHUNK = 64;                 // minimum detector chunk length (events)
constexpr unsigned DET_G = 1023;               // reach of the guessed windows, in chunks
constexpr unsigned DET_WARM = 32;              // steps a chunk runs from its guess before its own steps
constexpr unsigned DET_MAX_CHUNKS = 32768;     // chunks per batch at most (S grows beyond)
constexpr unsigned DET_SAMPLE = 64;            // chunks between sampled regulator windows
constexpr int LB_WIN = 8;                      // look-back window (predecessor tiles per load round)
constexpr int LB_GROUP = 32;                   // sort tiles per published group total
constexpr unsigned SPIN_LIMIT = 1u << 20;      // bounded device waits (~1 s)

// error bits in Ctrl::error
constexpr unsigned ERR_DEC_WAIT = 1u;
constexpr unsigned ERR_SORT_WAIT = 2u;
constexpr unsigned ERR_BAD_STATE = 4u;
constexpr unsigned ERR_S1_WAIT = 8u;
constexpr unsigned ERR_PROBE_WAIT = 16u;  // fibar_debug_wait_timeout

// Detector state after some step: window [h, k] (h batch-relative or global, see use),
// distinct pixels / tiles in the window, and q_targ for the next step as the ratio
// X / Y (Eq. 20 before the floor and the clamp).
struct DetState {
    long long h;
    unsigned int nap, nat;
    unsigned long long X, Y;
};

struct Ctrl {
    unsigned long long base;     // global index of the first event of the current batch
    unsigned long long dropped;  // out-of-range records skipped so far
    unsigned int m;              // valid events in the current batch
    unsigned int consumed;       // pending records consumed by the last decode
    unsigned int carry_n[2];     // records left pending in carry buffer 0 / 1
    unsigned int dec_ticket;
    unsigned int sort_ticket[SORT_MAX_PASSES];
    unsigned int hist_done;
    unsigned int cnt_done;
    unsigned int error;
    unsigned int unmerged;       // chunks whose second detector pass did not merge
    unsigned int fixups;         // batches that needed the serial detector fixup
    unsigned int S, nchunks, Gold;  // detector geometry of the batch (k_det_hist)
    unsigned int band_mid0;       // window band: centre at the batch start, in chunks,
    int band_slope;               //   and its drift per chunk (16.16 fixed point)
    unsigned int band_mode;       // 0: bands from (mid0, slope); 1: from the sampled centres
    unsigned long long recenters; // batches whose bands were rebuilt from the samples
    long long grow_num;           // queue growth over the last batch (events) ...
    unsigned int grow_den;        //   ... and that batch's length (0: none yet)
    unsigned int batch_no;       // read-outs/flushes committed (epoch of S1 flags)
    DetState det;                // detector state at the batch start (h global)
    long long h_prev;            // global h before the current batch (set by the fixup)
    unsigned int nblur;          // S1: stale pixels (blurs) in the current batch
    unsigned int blur_ticket;    // S1: dataflow work counter
    unsigned int sel_ticket;     // S1: stale-list compaction tile counter
    unsigned int walk_ticket;    // bucket walk work counter
    unsigned int p2_count;       // chunks that pass 2 hands on to its warp-per-chunk stage
    unsigned long long unmerged_total;  // diagnostics, cumulative
    unsigned long long pass2_steps;
    unsigned long long fix_steps;
    unsigned long long s1_blurs;
    unsigned long long big_pops, ring_misses;
    unsigned long long walk_pieces, scan_pieces;  // temporal filter schedules (cumulative)
};

// Constant per-handle parameters passed to kernels by value.
struct KParams {
    uint32_t W, H, tiles_w, tiles_h;
    uint32_t npix, ntiles;
    float a, oma, b, g;          // alpha, 1 - alpha, beta, (1 + beta) / 2
    float log2b;                 // log2(beta) (S1: beta^m for long gaps)
    float c_on, c_off;
    uint32_t q_min, q_max;
    uint32_t numA, den;          // fill_num * 4, fill_den  (Eq. 20 with A = 4)
    unsigned long long ring_mask;
    unsigned long long live;     // ring slots that stay valid behind the batch start
    uint32_t max_pending;
    uint32_t key_bits;           // bits of the tile id
    uint32_t lb;                 // low tile-id bits handled inside a bucket (<= 9)
    uint32_t nbuckets;           // buckets of 2^lb consecutive tiles
    int spatial, blur_mode;
    int chain_policy;            // temporal filter schedule: 0 auto (per piece), 1 walk, 2 scan
    uint32_t grid_sms;           // SMs the handle's grids are sized for (0: all of the device)
};

struct SegTable {
    const int4 *ptr[MAXSEG];
    unsigned int n[MAXSEG];
    unsigned int nseg;
    unsigned int carry_slot;     // ctrl->carry_n[carry_slot] = records in `carry`
    const int4 *carry;
    int4 *carry_out;
    unsigned long long t_read;
};

// One read-out of a handle as a captured read-out chain sees it: what changes from one
// read-out to the next, in device memory, written before the chain runs.
struct ReadDesc {
    SegTable t;
    float *out;                        // the image (16-byte aligned)
    unsigned long long *stamp_begin;   // if set: %globaltimer (ns) when the chain starts
    unsigned long long *stamp;         // if set: %globaltimer (ns) once the read-out has committed
};

struct Bufs {
    Ctrl *ctrl;
    float *pbar, *L;
    unsigned long long *last_pix, *last_tile;
    int4 *staging;
    int4 *carry[2];
    unsigned long long *dec_status;
    unsigned long long *rec[2];
    unsigned int *sort_hist;     // [SORT_MAX_PASSES][RADIX]
    unsigned int *sort_base;     // [SORT_MAX_PASSES][RADIX]
    unsigned *sort_rows, *sort_rowflag, *sort_gtot, *sort_gflag, *sort_gcount;
    unsigned int *qout;
    uint4 *ring4;                // {dP, dT, nP, nT} per global event index (ring)
    unsigned int *ring_pix;
    unsigned int *bucket_start;  // [nbuckets] first sorted position of each bucket
    unsigned int *bucket_cnt;    // [nbuckets] scratch histogram
    unsigned int *bucket_order;  // [nbuckets] walk order, largest buckets first (one-pass sorts)
    // detector chunk data
    unsigned short *dMt;         // [2][mt_rows][256] band of suffix histograms by target chunk
    unsigned int *det_base;      // [2 builds][2][mt_rows] window counts below the band (zero between batches)
    unsigned short *det_prof;    // [2][n_samples][640] window table columns of the sampled chunks
    unsigned short *band_ctr;    // [n_samples] regulator window (chunks) at the sampled chunks
    size_t n_samples;
    size_t mt_rows;              // chunk rows per table of dMt
    DetState *E0, *E1, *E2;
    unsigned int *p2_ids;        // [max_chunks] chunks continued by the warp-per-chunk pass 2
    unsigned int *snap;          // mapped host memory: {records left pending, commits, error flags} after a commit
    unsigned char *merged;
    unsigned *unm_bits;          // [chunks / 32] chunks that did not merge in pass 2
    float *out_staging;
    float *gain;                 // [npix] factor on Eq. 6 per pixel (Sec. 5.2), nullptr = none
    unsigned int *dbg_cnt;
    // S1 (blur in place when a pixel goes stale)
    unsigned int *plist;         // [maxp] batch events grouped by pixel (tile-major), in order
    float *plnb;                 // [maxp] L without this batch's blurs after that event
    unsigned int *lbl;           // [maxp] latest blur attached to the pixel's events <= position
    int *lbo;                    // [maxp] ordinal of that blur's event in the pixel's list (-1: before the batch)
    int4 *s1_info;               // [npix] {batch_no, list start, list length, previous event - base}
    float *s1_linit;             // [npix] L at the batch start (pixels with batch events)
    unsigned int *popk;          // [maxp + npix] pop step | stale << 31 of each popped event
    unsigned int *blur_ord;      // [maxp + npix] blur ordinal of each popped event (or ~0)
    unsigned int *bk, *bpix;     // [maxp + npix] step and pixel of each blur
    int *bj;                     // [maxp + npix] popped event (batch-relative) of each blur
    unsigned long long *bval;    // [maxp + npix] batch_no << 32 | bits of D (blurred value
                                 // minus L-without-blurs), published in one store
    unsigned long long *sel_status;
    float *beta_pow;             // [64] beta^m
    size_t max_pops, max_sel_tiles;
    size_t max_chunks, max_dec_tiles, max_sort_tiles;
};

// Learned stale-pixel fill (k_fill.cu): network parameters as a kernel parameter.
constexpr int FILL_NPARAMS = 2769;  // W1 16x2x3x3, b1 16, W2 16x16x3x3, b2 16, W3 1x16x3x3, b3 1
struct FillParams {
    // B operands per dx: 48 (n) x 16 (k) BF16, K-major, no swizzle, n = 16 (2 - dy) + output
    // channel: row n at 16 B, the second K half at +768 B, 1536 B per dx
    uint4 w1[9 * 32];      // conv1: k = input channel (only 0, 1 used)
    uint4 w2[9 * 32];      // conv2
    uint4 w3[9 * 32];      // conv3: output channel 0 only (the other rows zero)
    float b1[16], b2[16];
    float b3;
};

}  // namespace fibar

struct fibar_s {
    fibar::KParams kp;
    fibar_params_t params;
    double alpha, beta;
    uint32_t W, H;
    uint32_t sort_passes;
    unsigned long long R;
    fibar::Bufs b;
    // pending (host view)
    std::vector<const int4 *> seg_ptr;
    std::vector<unsigned int> seg_n;
    unsigned long long staging_used;
    unsigned long long pending_upper;   // upper bound of records not yet applied
    unsigned int *snap_host;            // host view of Bufs::snap (written by k_commit)
    float *gain_buf;                    // per-pixel gains, allocated by the first fibar_set_pixel_gain
    fibar::FillParams *fill;            // learned-fill network (blur_mode 2), nullptr = Gaussian
    // host packets: copied on an internal stream into one of two staging buffers, so that
    // the copy for the next read-out overlaps the current one (created by the first host push)
    int4 *staging2;                     // second staging buffer (b.staging is the first)
    int staging_cur;                    // buffer the pending host packets go to
    cudaStream_t copy_stream;
    cudaEvent_t ev_free[2];             // recorded after the decode that read buffer i
    cudaEvent_t ev_copied;              // the pending read-out's host packets have arrived
    bool copy_pending;                  // host packets queued since the last read-out
    unsigned long long commits;         // read-outs and flushes launched
    unsigned long long pushed_since;    // records pushed since the last read-out or flush
    int carry_slot;
    bool have_readout;
    unsigned long long last_readout;
    unsigned long long pushed, readouts;
    int device;
    std::string err;
    unsigned long long launches;
    // per-stage timing: events[i][0..FIBAR_NSTAGES] bracket the stages of read-out i
    bool timing;
    std::vector<cudaEvent_t> ev_pool;
    unsigned ev_used;            // read-outs recorded in ev_pool
    double stage_ms[FIBAR_NSTAGES];
    unsigned long long stage_calls;
    // bumped by every change of what a read-out chain launches (grid share, gains, fill
    // weights), so that a group's captured chains can be rebuilt
    unsigned long long config_version;
};

namespace fibar {
// Programmatic dependent launch: every kernel of the pipeline is launched with
// programmatic stream serialization and starts with PDL_ENTRY(), which lets the next
// kernel's blocks become resident early and then waits until the previous grid has
// completed and its memory is visible.  This hides most of the launch gap between the
// dependent kernels of a read-out.
#define PDL_ENTRY()                                              \
    do {                                                         \
        asm volatile("griddepcontrol.wait;" ::: "memory");       \
        asm volatile("griddepcontrol.launch_dependents;" :::);   \
    } while (0)

// Launches of this thread carry the PDL attribute (cleared while a chain is captured
// into a graph whose edges may not take it).
inline thread_local bool pdl_enabled = true;

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Lanes of the warp holding the same value as this lane, for values below 2^BITS: one
// ballot per bit (a warp multisplit), much cheaper than a general match.
template <int BITS>
__device__ __forceinline__ unsigned warp_peers(unsigned v)
{
    unsigned peers = 0xFFFFFFFFu;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const bool bit = (v >> b) & 1u;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// One-time set-up per device, safe under concurrent callers: `done` holds one bit per
// device ordinal (< 64) whose set-up succeeded; devices beyond 63 redo it every call.
// Two threads may both run `setup` for the same device; it must be idempotent.
template <class F>
inline cudaError_t once_per_device(std::atomic<unsigned long long> &done, F &&setup)
{
    int dev = 0;
    if (cudaError_t e = cudaGetDevice(&dev)) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    const cudaError_t e = setup();
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// Raise a kernel's dynamic shared memory limit once per device.
template <typename... KArgs>
inline cudaError_t smem_attr_once(std::atomic<unsigned long long> &done, void (*kern)(KArgs...), size_t smem)
{
    return once_per_device(done, [&] {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
}

// launchers (kernels live in their own translation units); `nl` counts kernel launches
cudaError_t launch_init(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl);
cudaError_t launch_probe_wait(const Bufs &b, const unsigned *flag, unsigned max_spins, cudaStream_t s,
                              unsigned long long &nl);
// tdev / outp / d (captured chains): the read-out's table, image pointer and descriptor
// in device memory, used instead of t / out
cudaError_t launch_decode(const KParams &kp, const Bufs &b, const SegTable &t, unsigned sort_passes, cudaStream_t s,
                          unsigned long long &nl, const SegTable *tdev = nullptr);
cudaError_t launch_sort(const KParams &kp, const Bufs &b, unsigned passes, cudaStream_t s, unsigned long long &nl);
cudaError_t launch_walk(const KParams &kp, const Bufs &b, const unsigned long long *sorted, unsigned sort_passes,
                        cudaStream_t s, unsigned long long &nl);
cudaError_t launch_det_counts(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl);
cudaError_t launch_det_pass1(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl);
cudaError_t launch_det_pass2(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl);
cudaError_t launch_det_fix(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl);
cudaError_t launch_readout(const KParams &kp, const Bufs &b, float *out, cudaStream_t s,
                           unsigned long long &nl, float *const *outp = nullptr);
cudaError_t launch_commit(const KParams &kp, const Bufs &b, int next_carry_slot, cudaStream_t s,
                          unsigned long long &nl, const ReadDesc *d = nullptr);
cudaError_t launch_s1(const KParams &kp, const Bufs &b, cudaStream_t s, unsigned long long &nl);
cudaError_t launch_debug_counts(const KParams &kp, const Bufs &b, unsigned int *cnt,
                                cudaStream_t s, unsigned long long &nl);
int grid_for(int sms_mult);
int grid_for(const KParams &kp, int sms_mult);  // the handle's share of the SMs
// learned fill read-out of a handle (k_fill.cu)
cudaError_t launch_fill_readout(const FillParams &fp, const KParams &kp, const Bufs &b, float *out, cudaStream_t s,
                                unsigned long long &nl, float *const *outp = nullptr);
// the kernels of one read-out (fibar_api.cu); d != nullptr: a chain captured for a group
int enqueue_readout_chain(fibar_t *h, const SegTable &T, float *out, const ReadDesc *d, cudaStream_t s,
                          bool stage_marks);
void fill_segtable(const fibar_t *h, unsigned long long t_read, SegTable &T);
void readout_committed(fibar_t *h);
}  // namespace fibar
