/*
 * FIBAR FP64 oracle - TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, event-by-event CPU restatement of "Filter-Based Reconstruction of
 * Images from Events" (FIBAR, arXiv 2510.20071), in double precision, processing
 * events strictly in arrival order with an explicit FIFO queue and explicit per-pixel
 * and per-tile counters.  It exists to check the CUDA library; nothing in the product
 * path may link, load or call it (only tests, the smoke check and the benchmark's CPU
 * baseline do).  It shares no code or header with the CUDA library.
 *
 * Passages followed (paper sections / equations):
 *   Sec. 3, Eqs. 2-3 : event increment  dL = C_p * p      (here C_p = c_on or c_off)
 *   Sec. 4.1, Eq. 7  : p_bar_k = alpha p_bar_{k-1} + (1 - alpha) p_k
 *   Sec. 4.1, Eq. 6  : dL_det_k = p_k - p_bar_k  (with the UPDATED p_bar_k)
 *   Sec. 4.1, Eq. 10 : L_k = beta L_{k-1} + (1 + beta)/2 * dL_det_k
 *   Sec. 4.1, Eqs. 16-18: omega_cut = 2 pi / T_cut, alpha_cut, beta_cut
 *   Sec. 4.2 steps 1-3: update the pixel, push the event to the back of the active
 *                       event queue (per-pixel counter ++), pop from the front while
 *                       the queue is longer than q_targ (counter --, a pixel whose
 *                       counter reaches zero is inactive and gets a one-time 3x3
 *                       Gaussian blur).
 *   Sec. 4.2, Eq. 19 : r_k = N_ap / (N_at * A), 2x2 tiles, A = 4
 *   Sec. 4.2, Eq. 20 : q_targ_{k+1} = floor(q_k * r_fill / r_k), in integers from
 *                      N_ap and N_at, bounded below.
 *   Sec. 5.2         : inter-pixel threshold correction - the right-hand side of Eq. 6
 *                      multiplied by the pixel's relative threshold C'_i (an optional
 *                      per-pixel gain, 1 when unset).
 *   Appendix (relative contrast thresholds): from a recording of a stationary signal,
 *                      N_on,i C_on,i = N_off,i C_off,i = |dL|; C_i is the harmonic mean
 *                      of C_on,i and C_off,i and C the harmonic mean of the C_i, so with
 *                      Nbar the mean of N_on,i + N_off,i over all pixels
 *                      C'_on,i = Nbar / (2 N_on,i), C'_off,i = Nbar / (2 N_off,i),
 *                      C'_i = Nbar / (N_on,i + N_off,i).
 *
 * Readings of points the paper leaves open (each one is a parameter or a fixed rule):
 *   - the queue is FIFO (push back, pop front), although the text once calls it LIFO;
 *   - q_targ is updated after every event, right after that event's pops; q_k is the
 *     queue length after the pops;
 *   - Eq. 20 is evaluated as floor(q * fill_num * A * N_at / (fill_den * N_ap)) with
 *     64-bit integers and clamped to [q_min, q_max], q_max = W*H (queue capped at the
 *     number of pixels), q_min default max(1, ceil(W*H/1024)), initial q_targ = q_init
 *     (default q_min);
 *   - counters are 32-bit (a 16-bit counter can overflow);
 *   - the Gaussian is the binomial [1,2,1] x [1,2,1] / 16; at the border the weights
 *     of the taps that fall inside the sensor are renormalised; all nine taps read the
 *     current L whatever the neighbour's state;
 *   - several pixels going stale in one step are blurred one after the other in pop
 *     order, each reading values already blurred in this step;
 *   - the blur changes L only, never p_bar;
 *   - c_on / c_off scale the +1 / -1 polarity before it enters Eq. 7 and Eq. 6
 *     (1, 1 = the paper's units);
 *   - read-out at time t applies the longest prefix of pushed events whose time
 *     stamps are all <= t; read-out times must not decrease;
 *   - a relative threshold whose count is zero (no ON, no OFF or no events at the
 *     pixel) is undefined and returned as NaN;
 *   - blur_mode 0 ("S1") blurs in place when the pixel goes stale (the paper);
 *     blur_mode 1 ("S2") never changes L and instead replaces, in the read-out image
 *     only, every pixel that has had an event and has no event in the queue by the
 *     3x3 blur of the unblurred L.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define REF_OK 0
#define REF_INVAL (-1)
#define REF_NOMEM (-2)
#define REF_ORDER (-3)

typedef struct {
    uint16_t x, y;
    int8_t p;
    uint8_t pad[3];
    uint64_t t_us;
} ref_event_t;

typedef struct {
    double t_cut;
    uint32_t fill_num, fill_den;
    uint32_t q_min, q_init;
    float c_on, c_off;
    int32_t spatial_filter;
    int32_t blur_mode;
    int32_t chain_policy; /* ignored by the oracle */
} ref_params_t;

/* optional per-event trace, written while events are applied */
typedef struct {
    uint64_t cap;          /* capacity of the per-event arrays */
    uint64_t *h;           /* global index of the queue front after the pops of event k */
    uint64_t *q_targ;      /* q_targ_{k+1}, computed at the end of step k */
    uint64_t *n_ap;        /* N_ap after step k */
    uint64_t *n_at;        /* N_at after step k */
    uint64_t stale_cap;
    uint64_t *stale_k;     /* step at which a pixel went stale */
    uint32_t *stale_pix;   /* which pixel, in pop order */
    uint64_t n_stale;      /* number of stale records produced (may exceed stale_cap) */
    uint64_t k0;           /* global index of trace entry 0 */
} ref_trace_t;

typedef struct {
    uint32_t W, H;
    uint64_t npix, ntiles, tiles_w;
    double alpha, beta;
    double c_on, c_off;
    int spatial_filter, blur_mode;
    uint64_t fill_num, fill_den, q_min, q_max, q_init;
    /* per-pixel state */
    double *pbar, *L;
    double *gain;          /* Sec. 5.2 per-pixel factor on Eq. 6, NULL = 1 */
    uint32_t *cnt;
    uint8_t *ever;
    uint64_t *last;        /* global index of the pixel's last event, UINT64_MAX if none */
    uint8_t *tcnt;         /* active pixels per 2x2 tile (0..4) */
    /* active event queue: FIFO of pixel ids, ring of capacity q_max + 1 */
    uint32_t *queue;
    uint64_t qcap, qhead, qlen;
    uint64_t n_ap, n_at, q_targ;
    uint64_t k;            /* events applied so far (global index of the next event) */
    /* pushed but not yet applied events */
    ref_event_t *pend;
    uint64_t pend_head, pend_len, pend_cap;
    uint64_t last_readout;
    int have_readout;
    uint64_t dropped, readouts;
    ref_trace_t *trace;
} ref_t;

/* Eqs. 16-18: cutoff frequency and the two filter coefficients. */
void fibar_ref_coefficients(double t_cut, double *alpha, double *beta)
{
    double w = 2.0 * M_PI / t_cut;
    double c = cos(w);
    *alpha = (1.0 - sin(w)) / c;                           /* Eq. 17 */
    *beta = (2.0 - c) - sqrt((2.0 - c) * (2.0 - c) - 1.0); /* Eq. 18 */
}

void fibar_ref_default_params(ref_params_t *p)
{
    memset(p, 0, sizeof(*p));
    p->t_cut = 40.0;      /* Sec. 5.1 choice */
    p->fill_num = 1;      /* r_fill = 0.5, Sec. 4.2 */
    p->fill_den = 2;
    p->q_min = 0;         /* 0 = max(1, ceil(W*H/1024)) */
    p->q_init = 0;        /* 0 = q_min */
    p->c_on = 1.0f;
    p->c_off = 1.0f;
    p->spatial_filter = 1;
    p->blur_mode = 0;
}

int fibar_ref_create(uint32_t W, uint32_t H, const ref_params_t *pp, ref_t **out)
{
    ref_params_t p;
    ref_t *o;
    if (!out) return REF_INVAL;
    *out = NULL;
    if (pp) p = *pp; else fibar_ref_default_params(&p);
    uint64_t npix = (uint64_t)W * (uint64_t)H;
    if (W == 0 || H == 0 || npix >= (1ull << 31)) return REF_INVAL;
    if (!(p.t_cut > 4.0)) return REF_INVAL;
    if (p.fill_num == 0 || p.fill_den == 0 || p.fill_num > 255 || p.fill_den > 255) return REF_INVAL;
    if (!(p.c_on > 0.0f) || !(p.c_off > 0.0f)) return REF_INVAL;
    if (p.spatial_filter != 0 && p.spatial_filter != 1) return REF_INVAL;
    if (p.blur_mode != 0 && p.blur_mode != 1) return REF_INVAL;
    uint64_t q_min = p.q_min ? p.q_min : ((npix + 1023) / 1024 > 1 ? (npix + 1023) / 1024 : 1);
    uint64_t q_max = npix;
    uint64_t q_init = p.q_init ? p.q_init : q_min;
    if (q_min > q_max || q_init < q_min || q_init > q_max) return REF_INVAL;

    o = (ref_t *)calloc(1, sizeof(ref_t));
    if (!o) return REF_NOMEM;
    o->W = W; o->H = H; o->npix = npix;
    o->tiles_w = (W + 1) / 2;
    o->ntiles = o->tiles_w * ((H + 1) / 2);
    fibar_ref_coefficients(p.t_cut, &o->alpha, &o->beta);
    o->c_on = p.c_on; o->c_off = p.c_off;
    o->spatial_filter = p.spatial_filter; o->blur_mode = p.blur_mode;
    o->fill_num = p.fill_num; o->fill_den = p.fill_den;
    o->q_min = q_min; o->q_max = q_max; o->q_init = q_init;
    o->pbar = (double *)calloc(npix, sizeof(double));
    o->L = (double *)calloc(npix, sizeof(double));
    o->cnt = (uint32_t *)calloc(npix, sizeof(uint32_t));
    o->ever = (uint8_t *)calloc(npix, 1);
    o->last = (uint64_t *)malloc(npix * sizeof(uint64_t));
    o->tcnt = (uint8_t *)calloc(o->ntiles, 1);
    o->qcap = q_max + 1;
    o->queue = (uint32_t *)malloc(o->qcap * sizeof(uint32_t));
    if (!o->pbar || !o->L || !o->cnt || !o->ever || !o->last || !o->tcnt || !o->queue) {
        free(o->pbar); free(o->L); free(o->cnt); free(o->ever); free(o->last);
        free(o->tcnt); free(o->queue); free(o);
        return REF_NOMEM;
    }
    for (uint64_t i = 0; i < npix; i++) o->last[i] = UINT64_MAX;
    o->q_targ = q_init;
    *out = o;
    return REF_OK;
}

void fibar_ref_destroy(ref_t *o)
{
    if (!o) return;
    free(o->pbar); free(o->L); free(o->cnt); free(o->ever); free(o->last);
    free(o->tcnt); free(o->queue); free(o->pend); free(o->gain); free(o);
}

/* Sec. 5.2: multiply the right-hand side of Eq. 6 of pixel i by gain[i] for every later
 * event (gain NULL: back to 1). */
int fibar_ref_set_gain(ref_t *o, const double *gain)
{
    if (!gain) {
        free(o->gain);
        o->gain = NULL;
        return REF_OK;
    }
    if (!o->gain) o->gain = (double *)malloc(o->npix * sizeof(double));
    if (!o->gain) return REF_NOMEM;
    memcpy(o->gain, gain, o->npix * sizeof(double));
    return REF_OK;
}

/* Appendix (relative contrast thresholds): per-pixel ON / OFF counts of a recording and
 * the relative thresholds they give.  Records outside the sensor are skipped. */
int fibar_ref_relative_thresholds(uint32_t W, uint32_t H, const ref_event_t *ev, uint64_t n,
                                  double *c_on, double *c_off, double *c)
{
    uint64_t npix = (uint64_t)W * H;
    if (W == 0 || H == 0) return REF_INVAL;
    uint64_t *n_on = (uint64_t *)calloc(npix, sizeof(uint64_t));
    uint64_t *n_off = (uint64_t *)calloc(npix, sizeof(uint64_t));
    if (!n_on || !n_off) { free(n_on); free(n_off); return REF_NOMEM; }
    uint64_t total = 0;
    for (uint64_t k = 0; k < n; k++) {
        if (ev[k].x >= W || ev[k].y >= H) continue;
        uint64_t i = (uint64_t)ev[k].y * W + ev[k].x;
        if (ev[k].p > 0) n_on[i]++; else n_off[i]++;
        total++;
    }
    /* Nbar: the mean number of events per pixel, over all W*H pixels */
    double nbar = (double)total / (double)npix;
    for (uint64_t i = 0; i < npix; i++) {
        c_on[i] = n_on[i] ? nbar / (2.0 * (double)n_on[i]) : NAN;
        c_off[i] = n_off[i] ? nbar / (2.0 * (double)n_off[i]) : NAN;
        c[i] = n_on[i] + n_off[i] ? nbar / (double)(n_on[i] + n_off[i]) : NAN;
    }
    free(n_on); free(n_off);
    return REF_OK;
}

void fibar_ref_set_trace(ref_t *o, ref_trace_t *tr)
{
    o->trace = tr;
    if (tr) { tr->n_stale = 0; tr->k0 = o->k; }
}

static uint64_t tile_of(const ref_t *o, uint64_t pix)
{
    uint64_t x = pix % o->W, y = pix / o->W;
    return (y / 2) * o->tiles_w + (x / 2);
}

/* 3x3 Gaussian [1,2,1] x [1,2,1] at pixel i over the current values of `img`,
 * renormalised over the taps that lie inside the sensor. */
static double blur3x3(const ref_t *o, const double *img, uint64_t i)
{
    static const double w[3] = {1.0, 2.0, 1.0};
    int64_t x = (int64_t)(i % o->W), y = (int64_t)(i / o->W);
    double acc = 0.0, wsum = 0.0;
    for (int dy = -1; dy <= 1; dy++) {
        int64_t yy = y + dy;
        if (yy < 0 || yy >= (int64_t)o->H) continue;
        for (int dx = -1; dx <= 1; dx++) {
            int64_t xx = x + dx;
            if (xx < 0 || xx >= (int64_t)o->W) continue;
            double wt = w[dy + 1] * w[dx + 1];
            acc += wt * img[(uint64_t)yy * o->W + (uint64_t)xx];
            wsum += wt;
        }
    }
    return acc / wsum;
}

/* Apply one event (pixel i, polarity p) as the paper's per-event procedure. */
static void apply_event(ref_t *o, uint64_t i, int p)
{
    /* Eqs. 2-3: polarity-dependent increment (C = c_on or c_off) */
    double s = p > 0 ? o->c_on : -o->c_off;

    /* Step 1: temporal filter. Eq. 7 (EMA of the increments), then Eq. 6 with the
     * updated average, then Eq. 10. */
    o->pbar[i] = o->alpha * o->pbar[i] + (1.0 - o->alpha) * s;
    double dl_det = s - o->pbar[i];
    if (o->gain) dl_det *= o->gain[i];  /* Sec. 5.2 */
    o->L[i] = o->beta * o->L[i] + 0.5 * (1.0 + o->beta) * dl_det;
    o->ever[i] = 1;

    uint64_t k = o->k;
    if (o->spatial_filter) {
        /* Step 2: push to the back of the active event queue */
        o->queue[(o->qhead + o->qlen) % o->qcap] = (uint32_t)i;
        o->qlen++;
        if (o->cnt[i]++ == 0) {
            o->n_ap++;
            if (o->tcnt[tile_of(o, i)]++ == 0) o->n_at++;
        }
        /* Step 3: pop from the front until the queue has reached q_targ */
        while (o->qlen > o->q_targ) {
            uint64_t j = o->queue[o->qhead];
            o->qhead = (o->qhead + 1) % o->qcap;
            o->qlen--;
            if (--o->cnt[j] == 0) {
                o->n_ap--;
                if (--o->tcnt[tile_of(o, j)] == 0) o->n_at--;
                if (o->blur_mode == 0) o->L[j] = blur3x3(o, o->L, j);
                if (o->trace) {
                    ref_trace_t *tr = o->trace;
                    if (tr->n_stale < tr->stale_cap) {
                        tr->stale_k[tr->n_stale] = k;
                        tr->stale_pix[tr->n_stale] = (uint32_t)j;
                    }
                    tr->n_stale++;
                }
            }
        }
        /* Eq. 20 with Eq. 19 substituted: q_targ = floor(q * r_fill / r_k)
         * = floor(q * fill_num * A * N_at / (fill_den * N_ap)), A = 4. */
        uint64_t q = o->qlen;
        unsigned __int128 num = (unsigned __int128)q * o->fill_num * 4u * o->n_at;
        unsigned __int128 den = (unsigned __int128)o->fill_den * o->n_ap;
        unsigned __int128 qt128 = num / den;
        uint64_t qt = qt128 > o->q_max ? o->q_max : (uint64_t)qt128;
        if (qt > o->q_max) qt = o->q_max;
        if (qt < o->q_min) qt = o->q_min;
        o->q_targ = qt;
    }
    o->last[i] = k;
    if (o->trace && k - o->trace->k0 < o->trace->cap) {
        ref_trace_t *tr = o->trace;
        uint64_t e = k - tr->k0;
        tr->h[e] = k + 1 - o->qlen;
        tr->q_targ[e] = o->q_targ;
        tr->n_ap[e] = o->n_ap;
        tr->n_at[e] = o->n_at;
    }
    o->k = k + 1;
}

int fibar_ref_push_events(ref_t *o, const ref_event_t *ev, uint64_t n)
{
    if (!o || (!ev && n)) return REF_INVAL;
    if (o->pend_head + o->pend_len + n > o->pend_cap) {
        /* compact, then grow */
        if (o->pend_head) {
            memmove(o->pend, o->pend + o->pend_head, o->pend_len * sizeof(ref_event_t));
            o->pend_head = 0;
        }
        if (o->pend_len + n > o->pend_cap) {
            uint64_t cap = o->pend_cap ? o->pend_cap : 1024;
            while (cap < o->pend_len + n) cap *= 2;
            ref_event_t *np = (ref_event_t *)realloc(o->pend, cap * sizeof(ref_event_t));
            if (!np) return REF_NOMEM;
            o->pend = np;
            o->pend_cap = cap;
        }
    }
    memcpy(o->pend + o->pend_head + o->pend_len, ev, n * sizeof(ref_event_t));
    o->pend_len += n;
    return REF_OK;
}

/* Apply the longest pending prefix whose time stamps are <= t_us. */
static void apply_until(ref_t *o, uint64_t t_us, int all)
{
    while (o->pend_len) {
        const ref_event_t *e = &o->pend[o->pend_head];
        if (!all && e->t_us > t_us) break;
        if (e->x >= o->W || e->y >= o->H) {
            o->dropped++;
        } else {
            apply_event(o, (uint64_t)e->y * o->W + e->x, e->p > 0 ? 1 : -1);
        }
        o->pend_head++;
        o->pend_len--;
    }
}

int fibar_ref_flush(ref_t *o)
{
    if (!o) return REF_INVAL;
    apply_until(o, 0, 1);
    return REF_OK;
}

/* Read-out at time t_us into out[W*H] (row-major, double). */
int fibar_ref_readout(ref_t *o, uint64_t t_us, double *out)
{
    if (!o || !out) return REF_INVAL;
    if (o->have_readout && t_us < o->last_readout) return REF_ORDER;
    o->have_readout = 1;
    o->last_readout = t_us;
    apply_until(o, t_us, 0);
    o->readouts++;
    if (o->spatial_filter && o->blur_mode == 1) {
        for (uint64_t i = 0; i < o->npix; i++) {
            int stale = o->ever[i] && o->cnt[i] == 0;
            out[i] = stale ? blur3x3(o, o->L, i) : o->L[i];
        }
    } else {
        memcpy(out, o->L, o->npix * sizeof(double));
    }
    return REF_OK;
}

/* State dump. Any pointer may be NULL. `last` uses UINT64_MAX for "no event yet". */
int fibar_ref_state(const ref_t *o, double *pbar, double *L, uint32_t *cnt, uint8_t *tcnt,
                    uint8_t *ever, uint64_t *last, uint64_t *scalars /* [8] */)
{
    if (!o) return REF_INVAL;
    if (pbar) memcpy(pbar, o->pbar, o->npix * sizeof(double));
    if (L) memcpy(L, o->L, o->npix * sizeof(double));
    if (cnt) memcpy(cnt, o->cnt, o->npix * sizeof(uint32_t));
    if (tcnt) memcpy(tcnt, o->tcnt, o->ntiles);
    if (ever) memcpy(ever, o->ever, o->npix);
    if (last) memcpy(last, o->last, o->npix * sizeof(uint64_t));
    if (scalars) {
        scalars[0] = o->k;                 /* events applied */
        scalars[1] = o->k - o->qlen;       /* h: global index of the queue front */
        scalars[2] = o->qlen;              /* q */
        scalars[3] = o->q_targ;            /* q_targ for the next event */
        scalars[4] = o->n_ap;
        scalars[5] = o->n_at;
        scalars[6] = o->dropped;
        scalars[7] = o->pend_len;          /* pushed, not yet applied */
    }
    return REF_OK;
}

/* Read-only accessors for the tests. */
void fibar_ref_info(const ref_t *o, double *alpha_beta, uint64_t *qbounds /* [3] */)
{
    alpha_beta[0] = o->alpha;
    alpha_beta[1] = o->beta;
    qbounds[0] = o->q_min;
    qbounds[1] = o->q_max;
    qbounds[2] = o->q_init;
}

/* The 3x3 blur rule on its own, applied to an arbitrary image (for the blur pins). */
void fibar_ref_blur_image(uint32_t W, uint32_t H, const double *img, double *out)
{
    ref_t tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.W = W; tmp.H = H;
    for (uint64_t i = 0; i < (uint64_t)W * H; i++) out[i] = blur3x3(&tmp, img, i);
}
