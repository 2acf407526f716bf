/*
 * fibar.h - C ABI of the GB300 (sm_103a) FIBAR event-to-image reconstruction library.
 *
 * FIBAR ("Filter-Based Reconstruction of Images from Events", arXiv 2510.20071)
 * turns a stream of event-camera events into a brightness image that can be read out
 * at any time (abstract; Sec. 1):
 *   - every event drives its pixel's temporal IIR filter (Sec. 4.1, Eqs. 6, 7, 10 with
 *     coefficients from Eqs. 16-18);
 *   - a global FIFO "active event queue" whose target length is regulated every event
 *     by the 2x2-tile fill ratio (Sec. 4.2 steps 1-3, Eqs. 19-20) decides when a pixel
 *     goes stale;
 *   - stale pixels are filled with a 3x3 Gaussian (Sec. 4.2).
 * All compute runs in hand-written CUDA kernels on the device; there is no CPU path.
 *
 * Conventions
 *   - Every function returns FIBAR_OK (0) or a negative FIBAR_E* code; the message of
 *     the last failure of a handle is available from fibar_last_error().
 *   - A handle is not thread safe.  All calls on one handle must be ordered: issue
 *     them on one CUDA stream (or synchronise between streams).  Separate handles are
 *     independent.
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Device memory is owned by the handle and released by fibar_destroy().
 */
#ifndef FIBAR_H
#define FIBAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FIBAR_OK 0
#define FIBAR_EINVAL (-1)   /* bad argument or parameter */
#define FIBAR_ENOMEM (-2)   /* device allocation failed, or pending capacity exceeded */
#define FIBAR_EORDER (-3)   /* read-out time earlier than the previous read-out time */
#define FIBAR_ECUDA (-4)    /* a CUDA runtime call failed */
#define FIBAR_ETIMEOUT (-5) /* a bounded device-side wait gave up (state is unreliable) */

/* One event, 16 bytes, little endian.  p > 0 is an ON event (brightness increased by
 * the ON threshold), otherwise OFF (Sec. 3, Eqs. 1-3).  t_us is the sensor time stamp
 * in microseconds; FIBAR itself ignores time stamps (Sec. 4.1: each pixel runs on its
 * own event clock) except to decide which events a read-out includes (Eq. 4, t_k <= t). */
typedef struct {
    uint16_t x, y;
    int8_t p;
    uint8_t pad[3];
    uint64_t t_us;
} fibar_event_t;

/* Parameters.  Fill with fibar_default_params() and override fields. */
typedef struct {
    double t_cut;            /* cutoff period in events (Eq. 16); default 40 (Sec. 5.1).
                                omega_cut = 2 pi / t_cut, alpha by Eq. 17, beta by Eq. 18.
                                Must be > 4; +inf gives alpha = beta = 1 (plain sum, Eq. 5) */
    uint32_t fill_num;       /* target fill ratio r_fill = fill_num / fill_den (Eq. 20);  */
    uint32_t fill_den;       /*   default 1/2 (Sec. 4.2).  Each in 1..255                 */
    uint32_t q_min;          /* lower bound of the target queue length (Sec. 4.2 requires
                                one but gives no value); 0 = max(1, ceil(W*H/1024))      */
    uint32_t q_init;         /* initial target queue length; 0 = q_min                    */
    float c_on, c_off;       /* contrast scales multiplying ON (+1) / OFF (-1) polarities
                                before Eqs. 7 and 6 (Eqs. 2-3); 1, 1 = the paper's units  */
    int32_t spatial_filter;  /* 1 = stale detection + Gaussian fill; 0 = FIBAR-NSF (Tab. 2) */
    int32_t blur_mode;       /* 0 = "S1": blur the pixel's L in place when it goes stale
                                   (Sec. 4.2, the paper's method; read-out copies L);
                                1 = "S2": never modify L; at read-out, output the 3x3 blur
                                   of L at stale pixels (had an event, none queued) and L
                                   elsewhere;
                                2 = learned fill: as S2, with the stale pixels filled by
                                   the network set by fibar_fill_set_weights (the Gaussian
                                   of S2 until weights are set)                           */
    int32_t chain_policy;    /* schedule of the temporal filter (same results up to FP32
                                rounding; the paper runs it event by event):
                                0 = auto: per piece of <= 2048 events of 512 tiles, the scan
                                    when one tile has more than 64 events in it, else the walk;
                                1 = walk: one thread per 2x2 tile, events in arrival order;
                                2 = scan: segmented scan of the per-event affine maps of
                                    Eqs. 7, 6, 10 along each pixel's events               */
    uint32_t max_pending;    /* capacity, in events, of pushed-but-unapplied events and of
                                one processing batch; 0 = 8 Mi events                     */
} fibar_params_t;

typedef struct fibar_s fibar_t;

/* Host-side counters.  Filled by fibar_stats(), which synchronises the stream. */
typedef struct {
    uint64_t events_pushed;   /* records handed to fibar_push_events                      */
    uint64_t events_applied;  /* valid events applied to the state                       */
    uint64_t events_dropped;  /* out-of-range records skipped (counted, not applied)      */
    uint64_t events_pending;  /* pushed records not yet applied                          */
    uint64_t readouts;
    uint64_t q;               /* current queue length (events in the active window)      */
    uint64_t q_targ;          /* target length for the next event (Eq. 20)               */
    uint64_t n_ap, n_at;      /* active pixels / active 2x2 tiles (Eq. 19)               */
    uint64_t detector_fixups; /* batches whose speculative detector needed a serial fixup */
    uint64_t kernel_launches; /* CUDA kernels this handle has launched                    */
    uint64_t detector_unmerged;    /* speculative chunks that did not merge (cumulative)  */
    uint64_t detector_pass2_steps; /* events re-run by the merging pass (cumulative)       */
    uint64_t detector_fix_steps;   /* events re-run serially by the fixup (cumulative)     */
    uint64_t s1_blurs;             /* S1 in-place blurs applied (cumulative)               */
    uint64_t detector_big_pops;    /* detector steps whose many pops a whole warp counted  */
    uint64_t detector_ring_misses; /* popped-event links read past the staged ring         */
    uint64_t detector_recenters;   /* batches whose window bands were rebuilt from samples */
    uint64_t iir_walk_pieces;      /* pieces (<= 2048 events of one bucket of 512 tiles) whose
                                      temporal filter ran as a walk per tile (cumulative)   */
    uint64_t iir_scan_pieces;      /* pieces whose temporal filter ran as a segmented scan  */
} fibar_stats_t;

/* Stages of one read-out, in launch order (fibar_stage_times). */
enum {
    FIBAR_STAGE_DECODE = 0,  /* decode + read-out cut + compaction (one pass over records)  */
    FIBAR_STAGE_SORT,        /* stable radix sort by 2x2 tile                               */
    FIBAR_STAGE_WALK,        /* per-tile walk: temporal filter (Eqs. 6, 7, 10) + links        */
    FIBAR_STAGE_DET_COUNTS,  /* detector: per-chunk window counts + scan                     */
    FIBAR_STAGE_DET_PASS1,   /* detector: speculative pass over all chunks                   */
    FIBAR_STAGE_DET_PASS2,   /* detector: re-run from predecessors until trajectories merge  */
    FIBAR_STAGE_DET_FIX,     /* detector: serial fixup (no-op when every chunk merged)       */
    FIBAR_STAGE_S1,          /* S1 only: ordered in-place blurs of pixels going stale        */
    FIBAR_STAGE_READOUT,     /* output image (copy of L, or S2 masked blur)                  */
    FIBAR_STAGE_COMMIT,      /* batch bookkeeping                                            */
    FIBAR_NSTAGES
};

/* Accumulated device time per stage, measured with CUDA events recorded on the
 * caller's stream around each stage of every read-out/flush while timing is on. */
typedef struct {
    double ms[FIBAR_NSTAGES];
    uint64_t calls;           /* read-outs/flushes measured */
} fibar_stage_times_t;

/* Debug copy of the device state.  Each array pointer is a caller-owned HOST buffer
 * or NULL (skipped).  Arrays are row-major, pixel i = y * W + x; tiles are 2x2 blocks
 * aligned at (0,0), tile j = (y/2) * ceil(W/2) + (x/2). */
typedef struct {
    float *pbar;        /* [W*H] detrending average p_bar (Eq. 7)                         */
    float *L;           /* [W*H] filter output L (Eq. 10), including S1 blurs             */
    uint32_t *cnt;      /* [W*H] events of each pixel in the active event queue           */
    uint8_t *tcnt;      /* [tiles] active pixels of each 2x2 tile                         */
    uint8_t *stale;     /* [W*H] 1 = pixel had an event and has none queued               */
    uint64_t *last_idx; /* [W*H] global index of the pixel's last applied event, or
                           UINT64_MAX if it never had one                                 */
    /* scalars, always written */
    uint64_t k;         /* events applied so far (global index of the next event)        */
    uint64_t h;         /* global index of the oldest queued event                        */
    uint64_t q, q_targ, n_ap, n_at;
} fibar_state_view_t;

/* Fill *p with the defaults above. */
void fibar_default_params(fibar_params_t *p);

/* Create a stream reconstructor for a W x H sensor on the current CUDA device.
 * p may be NULL (defaults).  Allocates all device memory up front (state, rings,
 * batch buffers sized by max_pending).  Errors: EINVAL (W or H = 0, W*H > 2^24,
 * max_pending > 2^27, bad parameter), ENOMEM, ECUDA.  On success *out owns the
 * handle. */
int fibar_create(uint32_t W, uint32_t H, const fibar_params_t *p, fibar_t **out);

/* Queue n events for the next read-out (Sec. 1: events arrive in packets).
 *   on_device = 0: `ev` is host memory; it is copied to the device on an internal copy
 *                  stream of the handle, into one of two staging buffers (the next
 *                  read-out's packets go to the other one, so their copy overlaps the
 *                  current read-out); the next read-out or flush on `cuda_stream` waits
 *                  for the copy.  Pageable buffers may be reused on return; page-locked
 *                  buffers once that read-out has completed.  The first host push
 *                  allocates the second staging buffer (16 bytes x max_pending).
 *   on_device = 1: `ev` is device memory (16-byte aligned) read in place by the next
 *                  fibar_readout() or fibar_flush(); it must stay valid and unchanged
 *                  until that call's work has completed on the stream.
 * Nothing is applied here.  Records with x >= W or y >= H are dropped and counted
 * when applied.  Errors: EINVAL, ENOMEM (more than max_pending events or 192 device
 * packets pending: read out or flush first), ECUDA. */
int fibar_push_events(fibar_t *h, const fibar_event_t *ev, size_t n, int on_device,
                      void *cuda_stream);

/* Queue several packets in one call: for i < count, what fibar_push_events(h, evs[i],
 * ns[i], on_device, cuda_stream) does, in order.  Packets that follow each other in
 * memory (evs[i] + ns[i] == evs[i + 1]) are queued as one: one host-to-device copy for
 * host packets, one pending segment for device packets.  The paper has no counterpart;
 * this saves a call and a copy per packet for callers that receive packets in bursts.
 * Stops at the first run that fails (the earlier ones stay queued) and returns its error
 * (as fibar_push_events). */
int fibar_push_events_many(fibar_t *h, const fibar_event_t *const *evs, const size_t *ns, size_t count,
                           int on_device, void *cuda_stream);

/* Queue packets for several handles in one call: for k < count, what
 * fibar_push_events(hs[k], evs[k], ns[k], on_device, cuda_stream) does, in order (a
 * handle may appear more than once).  The paper has no counterpart; a server that
 * receives one packet per stream per tick makes one call instead of one per stream.
 * status: NULL, or count ints with each entry's code.  Every entry is attempted; returns
 * the first non-zero code (EINVAL for a NULL handle), else FIBAR_OK. */
int fibar_push_batch(fibar_t *const *hs, const fibar_event_t *const *evs, const size_t *ns, size_t count,
                     int on_device, int *status, void *cuda_stream);

/* Apply the longest prefix of pending events whose time stamps are all <= t_us
 * (Eq. 4's t_k <= t, in push order), then write the W*H float image (row-major) to
 * `out`: L for S1 and NSF (Sec. 1: no work at read-out), or the masked 3x3 blur of
 * L for S2.  Pending events after the prefix stay queued.
 *   on_device = 1: out is device memory; the call returns without waiting.
 *   on_device = 0: out is host memory; the call waits for the result.
 * Errors: EINVAL, EORDER (t_us < previous read-out time), ECUDA, ETIMEOUT. */
int fibar_readout(fibar_t *h, uint64_t t_us, float *out, int on_device, void *cuda_stream);

/* fibar_readout into a HOST buffer without waiting: queues the read-out and the
 * device-to-host copy of the image into `out` (W*H floats; page-locked memory makes the
 * copy asynchronous) on cuda_stream and returns.  The image is in `out` once the stream
 * has passed the copy (fibar_wait, or an event recorded on the stream after this call).
 * The paper has no counterpart; this lets a caller overlap the next packets' upload and
 * read-out with the current one.  Errors: EINVAL, EORDER, ECUDA (bounded device waits
 * that gave up are reported by fibar_wait). */
int fibar_readout_host_async(fibar_t *h, uint64_t t_us, float *out, void *cuda_stream);

/* Wait for the work queued on cuda_stream (synchronises it); ETIMEOUT if a bounded device
 * wait of the last committed read-out or flush gave up.  Errors: EINVAL, ECUDA, ETIMEOUT. */
int fibar_wait(fibar_t *h, void *cuda_stream);

/* Read out n handles together: for every i, what fibar_readout(hs[i], t_us[i], outs[i],
 * 1, ...) does, with the work of different handles running concurrently on the device.
 * The paper reconstructs one stream; this serves many streams of different sensors at
 * once.  Each handle's pipeline goes to one of the library's internal CUDA streams
 * (16 per device, created on the first call): the handles are dealt out by their
 * pending event counts, largest first, each to the internal stream with the least work
 * so far.  The work of all handles starts after the work already queued on
 * `cuda_stream`, and work queued on `cuda_stream` after the call starts after all of it,
 * so calls on one caller stream stay ordered.
 *   hs[n], t_us[n], outs[n]: handles, read-out times, device images of W_i*H_i floats.
 *   done_events: NULL, or n cudaEvent_t (passed as void*, NULL entries skipped); entry
 *                i is recorded when handle i's image is complete.
 *   status:      NULL, or n ints that receive each handle's code as fibar_readout's.
 * Returns FIBAR_OK, or the first non-zero status in index order (the other handles are
 * still read out), or EINVAL before any work is queued when an array is NULL, n > 4096,
 * a handle appears twice, or a handle belongs to a device that is not current.  Batch
 * calls on one device from several host threads are serialised by the library. */
int fibar_readout_batch(fibar_t *const *hs, const uint64_t *t_us, float *const *outs, size_t n,
                        void *const *done_events, int *status, void *cuda_stream);

/* Device memory in bytes that fibar_create(W, H, p) allocates (the sum of its buffers,
 * each rounded up to 512 bytes; the CUDA context and the driver's page granularity are
 * not included).  Host arithmetic only: needs no device.  The paper has no counterpart;
 * a server uses it to admit streams by memory.  Errors: EINVAL (bytes NULL, or arguments
 * that fibar_create rejects as EINVAL). */
int fibar_memory_bytes(uint32_t W, uint32_t H, const fibar_params_t *p, uint64_t *bytes);

/* Relative contrast thresholds of every pixel from a calibration recording (the paper's
 * appendix on relative contrast thresholds): with N_on,i and N_off,i the pixel's ON and
 * OFF event counts and Nbar the mean of N_on,i + N_off,i over all W*H pixels,
 *   c_on[i] = Nbar / (2 N_on,i),  c_off[i] = Nbar / (2 N_off,i),  c[i] = Nbar / (N_on,i + N_off,i)
 * (row-major W*H floats each; NaN where the count in the denominator is 0).  These are
 * C_on,i / C, C_off,i / C and C_i / C, C_i being the harmonic mean of a pixel's two
 * thresholds and C the harmonic mean of the C_i, when the recording is of a spatially
 * uniform, stationary signal.  Records outside the sensor are skipped.
 *   on_device = 1: ev and the outputs are device memory (ev 16-byte aligned); the call
 *                  returns without waiting.
 *   on_device = 0: host memory; events are copied in chunks of 4 Mi records; the call
 *                  returns after the results are in place.
 * Workspace (8 bytes per pixel, plus staging for host data) is allocated and released on
 * `cuda_stream` (stream-ordered allocation).  Needs no handle.  The paper has no code
 * for this; it derives the formulas.  Errors: EINVAL (W or H = 0, W*H > 2^24, a NULL
 * pointer, misaligned device events), ENOMEM, ECUDA. */
int fibar_relative_thresholds(const fibar_event_t *ev, size_t n, uint32_t W, uint32_t H, int on_device,
                              float *c_on, float *c_off, float *c, void *cuda_stream);

/* Sec. 5.2 threshold correction: from the next read-out on, the right-hand side of
 * Eq. 6 (the detrended increment p_k - pbar_k) of pixel i is multiplied by gain[i]
 * (Sec. 5.2 uses the relative threshold c[i] of fibar_relative_thresholds).  gain: W*H
 * floats, row-major, copied into the handle (the first call allocates W*H*4 bytes);
 * NULL removes the correction.  on_device = 0: host memory, every value must be finite
 * and > 0 (else EINVAL, nothing changes); on_device = 1: device memory, copied on
 * `cuda_stream` without checking.  Errors: EINVAL, ENOMEM, ECUDA. */
int fibar_set_pixel_gain(fibar_t *h, const float *gain, int on_device, void *cuda_stream);

/* Apply every pending event (as a read-out at t = +inf without output; does not
 * change the read-out time order). */
int fibar_flush(fibar_t *h, void *cuda_stream);

/* Synchronise and copy the state (see fibar_state_view_t). */
int fibar_debug_state(fibar_t *h, fibar_state_view_t *v, void *cuda_stream);

/* The number of queued events of every pixel (the per-pixel queued-event count that
 * fibar_debug_state reports as cnt; a pixel whose count is zero after it had an event is
 * stale), written to cnt[W*H] in row-major order: device memory when on_device is
 * non-zero (asynchronous on cuda_stream), else host memory (returns after the copy).
 * The paper has no counterpart; this exists for callers that must not allocate device
 * memory once they run (a process sharing the GPU under a fixed memory budget, where an
 * allocation can fail, or a latency-bound loop that cannot afford the implicit device
 * synchronisation an allocation may cause).  fibar_debug_state allocates its counter
 * buffer on first use; this call counts into a fixed buffer of 1,048,576 32-bit counters
 * (4 MiB) built into the library, one per device, cleared by every call before it counts.
 * Errors: EINVAL (h or cnt NULL, W*H > 1,048,576, or the handle's device not current),
 * ECUDA, and, with host output only, ETIMEOUT when a bounded device wait of the pipeline
 * gave up (with device output, fibar_stats reports that flag).  Every call looks up the
 * buffer's device address (no allocation); the first call in a process may load the
 * library's device code, so make it before any stream capture.  Calls that overlap in
 * time on other streams or threads, with this or another handle on the same device,
 * share the buffer and race; calls on one stream are ordered. */
int fibar_queue_counts_noalloc(fibar_t *h, uint32_t *cnt, int on_device, void *cuda_stream);

/* ---- Learned stale-pixel fill ---------------------------------------------------------
 * The paper fills a pixel that goes stale with an isotropic 3x3 Gaussian (Sec. 4.2); its
 * limitations section names what that blur ignores (the gradient's magnitude and
 * direction) and leaves more elaborate fills to GPUs.  The learned fill is a 3-layer 3x3
 * convolutional network (2 -> 16 -> 16 -> 1 channels, ReLU, zero padding; BF16 weights,
 * FP32 accumulation; the 16 -> 16 layer on the tensor cores) whose inputs per pixel are
 * L (Eq. 10) and the activity age min(4, (k - last) / q) (k the events applied, last the
 * pixel's last event, q the queue length); its output replaces L at the stale pixels.
 * Parameters theta: FIBAR_FILL_NPARAMS floats, in order W1 [16][2][3][3], b1 [16],
 * W2 [16][16][3][3], b2 [16], W3 [1][16][3][3], b3 [1] (weights are rounded to BF16).  */
#define FIBAR_FILL_NPARAMS 2769

/* Set (theta != NULL, n = FIBAR_FILL_NPARAMS host floats, copied) or remove (theta = NULL)
 * the network a blur_mode = 2 handle fills with from its next read-out on.
 * Errors: EINVAL (h NULL, wrong n, a non-finite parameter), ENOMEM. */
int fibar_fill_set_weights(fibar_t *h, const float *theta, size_t n);

/* The network's inputs for the handle's current state (after its last read-out or flush),
 * for training and evaluation: x = device float [2][H][W] (L, then the age), stale = device
 * uint8 [H][W] (1 = had an event, none queued) or NULL.  Asynchronous on cuda_stream.
 * Errors: EINVAL (NULL h or x, misaligned x, a handle with spatial_filter = 0), ECUDA. */
int fibar_fill_features(fibar_t *h, float *x, uint8_t *stale, void *cuda_stream);

/* The fill image of explicit inputs with the read-out's kernel: out[i] = the network's
 * output where stale[i] != 0, x[0][i] elsewhere.  theta: host floats (as above); x, stale,
 * out: device memory (x, out 4-byte aligned).  Synchronises cuda_stream.  Needs no handle
 * (a 4-byte status word is allocated on the stream).  Errors: EINVAL (NULL pointer, W or
 * H = 0, W*H > 2^24, a non-finite parameter), ENOMEM, ECUDA, ETIMEOUT (the tensor-core
 * completion wait gave up). */
int fibar_fill_forward(const float *theta, const float *x, const uint8_t *stale, uint32_t W, uint32_t H,
                       float *out, void *cuda_stream);

/* One training step of the fill network (all pointers device memory):
 *   X [F][2][H][W] inputs, T [F][H][W] targets, M [F][H][W] loss mask (uint8), F = n_frames;
 *   crops [n_crops][3] = (frame, y0, x0) of 24 x 24 crops inside a frame (a crop that is not
 *   is skipped and counted in loss_acc[2]); the loss is the
 *   mean squared error of the network (evaluated on each crop with zero padding at its
 *   border, BF16 weights) against T over the masked pixels at least 3 pixels inside a crop;
 *   theta, m, v: FIBAR_FILL_NPARAMS FP32 master weights and Adam moments, updated in place
 *   with step number `step` (>= 1) and learning rate lr (beta1 0.9, beta2 0.999, eps 1e-8;
 *   lr <= 0: gradient only); grad receives the mean gradient; loss_acc[3] receives (sum of
 *   squared errors, number of loss pixels, skipped crops) in double.  Asynchronous on cuda_stream.
 * Errors: EINVAL (NULL pointer, W or H < 24, n_frames = 0, n_crops = 0 or > 65535,
 * step = 0), ECUDA. */
int fibar_fill_train_step(const float *X, const float *T, const uint8_t *M, uint32_t W, uint32_t H,
                          uint32_t n_frames, const int32_t *crops, uint32_t n_crops, float *theta, float *m,
                          float *v, float *grad, uint32_t step, float lr, double *loss_acc, void *cuda_stream);

/* Failure-detection check (no counterpart in the paper): runs, on the device, the bounded
 * wait that the pipeline's look-back and dataflow kernels use, on a flag that nothing
 * sets, with a limit of max_spins polls (1..2^20, each followed by a ~64 ns back-off).
 * The wait gives up, records its flag in the handle's error word and returns; this call
 * synchronises, clears that flag again (the handle stays usable) and returns ETIMEOUT,
 * with a message.  Errors: EINVAL, ENOMEM, ECUDA. */
int fibar_debug_wait_timeout(fibar_t *h, uint32_t max_spins, void *cuda_stream);

/* Synchronise and fill counters.  Reports ETIMEOUT if a device wait gave up. */
int fibar_stats(fibar_t *h, fibar_stats_t *s, void *cuda_stream);

/* Turn per-stage timing on (1) or off (0).  While on, each read-out/flush records 10
 * CUDA events on its stream (up to 4096 read-outs are kept; older ones are folded in
 * when fibar_stage_times is called). */
int fibar_set_timing(fibar_t *h, int enable);

/* Synchronise and return the accumulated per-stage times; reset = 1 clears them. */
int fibar_stage_times(fibar_t *h, fibar_stage_times_t *t, int reset, void *cuda_stream);

/* Message of the last failed call on this handle ("" if none).  Owned by the handle. */
const char *fibar_last_error(fibar_t *h);

/* Size the handle's kernel grids for `sms` streaming multiprocessors from its next
 * read-out on (0, or more than the device has: all of them; the default).  Results do not
 * change (every kernel distributes its work by tickets or strided loops).  The paper has
 * no counterpart; when many small streams are read out concurrently
 * (fibar_readout_batch), a share below the whole device lets their pipelines run side by
 * side instead of each one's grids filling the GPU in turn.  Errors: EINVAL. */
int fibar_set_grid_share(fibar_t *h, uint32_t sms);

/* ---- groups: read-outs of a fixed set of handles, one graph launch per member -------
 * The paper reconstructs one stream and has no counterpart.  A read-out is a chain of
 * about a dozen dependent kernels; issued one launch at a time (fibar_readout_batch),
 * the chains of many small streams leave the device waiting on the host, and each short
 * chain is bound by its own latency.  A group captures every member's chain once into a
 * CUDA graph, and gives every member its own internal CUDA stream: what changes between
 * read-outs (the packets pushed, the read-out time, the image pointer, the carry slot) is
 * written by the host into a ring of descriptors in mapped page-locked memory, which the
 * graph's first kernel copies to the device.  A read-out of a member is then one graph
 * launch on its stream, and the chains of different members - of one call and of
 * consecutive calls - run side by side, each member's read-outs in order.
 * Results are those of fibar_readout on each member (same kernels, same order per
 * member).  A member's change of grid share, pixel gains or fill weights is picked up by
 * re-capturing its graph at its next group read-out.  A group's calls are not
 * thread-safe; work on a member's own handle (push, fibar_readout, flush) must not be
 * queued while its group read-outs are in flight (join first); destroy the group before
 * its members.  Per-stage timing (fibar_set_timing) does not cover group read-outs. */
typedef struct fibar_group_s fibar_group_t;

typedef struct {
    uint64_t members;         /* handles in the group */
    uint64_t graph_launches;  /* fibar_group_readout calls that launched work */
    uint64_t builds;          /* member graph captures (one per member + re-captures) */
    uint64_t graph_kernels;   /* kernel nodes in the members' graphs (all members) */
    int32_t programmatic_edges;  /* 1: every chain captured with programmatic
                                    (early-launch) edges; 0: some with plain edges */
} fibar_group_stats_t;

/* Create a group over hs[0..n) (n <= 1024, distinct handles of the current device) and
 * capture each member's graph.  *out receives the group.  Errors: EINVAL, ENOMEM, ECUDA. */
int fibar_group_create(fibar_t *const *hs, size_t n, fibar_group_t **out);

/* Read out members[k] (indices into the group's hs, distinct) at t_us[k] into outs[k]
 * (device images of W*H floats, 16-byte aligned), k < m: what fibar_readout(hs[members[k]],
 * t_us[k], outs[k], 1, ...) does for each, as one graph launch per member on the member's
 * own stream.  The launches start after the work already queued on cuda_stream (the
 * packets); work queued on cuda_stream later does NOT wait for them: call
 * fibar_group_join (or fibar_group_latency, which waits) before using the images there.
 * ticket: NULL, or receives the call's number for fibar_group_latency.  status: NULL, or
 * m ints with each entry's check result.  Every entry is checked before anything is
 * queued: if one fails (EINVAL: index out of range or repeated, output NULL or
 * misaligned; EORDER: time earlier than the member's previous read-out), nothing is
 * queued and the first failing code is returned.  Errors also: ECUDA. */
int fibar_group_readout(fibar_group_t *g, const uint32_t *members, const uint64_t *t_us, float *const *outs,
                        size_t m, int *status, uint64_t *ticket, void *cuda_stream);

/* Make work queued on cuda_stream from now on wait for every group read-out queued so
 * far.  Errors: EINVAL, ECUDA. */
int fibar_group_join(fibar_group_t *g, void *cuda_stream);

/* Device time in ms from the start of call `ticket` (the first of its members' chains to
 * start) to each of its images being complete (that member's read-out committed),
 * ms[k] for the k-th entry of that call; m must equal that call's m.  Waits for the
 * call's members.  Tickets of the last 4096 calls are kept.  Errors: EINVAL (unknown or
 * expired ticket, m mismatch), ECUDA. */
int fibar_group_latency(fibar_group_t *g, uint64_t ticket, float *ms, size_t m);

/* Counters of the group.  Errors: EINVAL. */
int fibar_group_stats(fibar_group_t *g, fibar_group_stats_t *st);

/* Message of the last failed group call ("" if none).  Owned by the group. */
const char *fibar_group_last_error(fibar_group_t *g);

/* Release the group (waits for its work in flight); its members stay valid. */
void fibar_group_destroy(fibar_group_t *g);

/* Release the handle and its device memory (waits for its outstanding work). */
void fibar_destroy(fibar_t *h);

#ifdef __cplusplus
}
#endif
#endif /* FIBAR_H */
