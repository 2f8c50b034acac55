/*
 * Seeded synthetic grayscale images that stand in for the paper's CK+ face
 * crops (Sec. 3.1).  This module holds none of the LDP/LBP arithmetic: it only
 * produces uint8 pixels, and both the CPU oracle and the CUDA library are fed
 * the very same bytes.
 *
 * Recipe (one independent SplitMix64 stream per image seed):
 *   draws 0,1         : image height / width when a size range is requested
 *   draws 2 .. 2+HW-1 : uniform [0,255) base noise, row-major
 *   next HW draws     : Box-Muller pairs -> N(0,1), scaled to std 8
 *   base noise -> separable Gaussian blur (double, radius ceil(4 sigma),
 *   mirror borders) -> min-max rescale to [0,255] -> + noise -> round half to
 *   even -> clip to [0,255].
 *
 * SplitMix64 is counter based (output n = mix(seed + (n+1)*gamma)), so any
 * draw can be computed directly; that is what lets rows of one large image be
 * generated by several threads with identical results.
 *
 * Build: gcc -O3 -ffp-contract=off -fPIC -shared -pthread gen.c -lm
 * (-ffp-contract=off keeps the arithmetic free of FMA contraction, so x86 and
 * Arm builds differ at most through libm's exp/log/cos/sin).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SM_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number n (0-based) of the SplitMix64 stream started at `seed`. */
uint64_t synth_draw(uint64_t seed, uint64_t n) { return sm_mix(seed + (n + 1) * SM_GAMMA); }

static inline double u53(uint64_t d) { return (double)(d >> 11) * 0x1.0p-53; } /* [0,1) */

/* Height and width uniform on the integers [lo, hi], from draws 0 and 1. */
void synth_sizes(uint64_t seed, int lo, int hi, int *H, int *W) {
    double span = (double)(hi - lo + 1);
    int h = lo + (int)(u53(synth_draw(seed, 0)) * span);
    int w = lo + (int)(u53(synth_draw(seed, 1)) * span);
    *H = h > hi ? hi : h;
    *W = w > hi ? hi : w;
}

static inline int mirror(int i, int n) {
    if (n == 1) return 0;
    for (;;) {
        if (i < 0) i = -i;
        else if (i >= n) i = 2 * (n - 1) - i;
        else return i;
    }
}

typedef struct {
    uint64_t seed;
    int H, W, pitch, radius;
    const double *wts; /* 2*radius+1 normalised Gaussian weights */
    double *a, *b;     /* H*W scratch */
    uint8_t *out;
    double lo, scale;  /* rescale parameters (final pass) */
    int r0, r1;        /* row range of this worker */
    double mn, mx;     /* per-worker min / max of the blurred image */
} img_job;

/* pass 1: base noise + horizontal blur, rows [r0,r1) into b */
static void pass_hblur(img_job *j) {
    const int W = j->W, R = j->radius;
    double *row = (double *)malloc(sizeof(double) * (size_t)W);
    for (int r = j->r0; r < j->r1; ++r) {
        for (int c = 0; c < W; ++c)
            row[c] = 255.0 * u53(synth_draw(j->seed, 2 + (uint64_t)r * W + c));
        double *dst = j->b + (size_t)r * W;
        for (int c = 0; c < W; ++c) {
            double s = 0.0;
            if (c >= R && c + R < W) {
                const double *src = row + c - R;
                for (int t = 0; t <= 2 * R; ++t) s += j->wts[t] * src[t];
            } else {
                for (int t = -R; t <= R; ++t) s += j->wts[t + R] * row[mirror(c + t, W)];
            }
            dst[c] = s;
        }
    }
    free(row);
}

/* pass 2: vertical blur of b into a for rows [r0,r1), tracking min / max */
static void pass_vblur(img_job *j) {
    const int W = j->W, H = j->H, R = j->radius;
    double mn = INFINITY, mx = -INFINITY;
    for (int r = j->r0; r < j->r1; ++r) {
        double *dst = j->a + (size_t)r * W;
        for (int c = 0; c < W; ++c) dst[c] = 0.0;
        for (int t = -R; t <= R; ++t) {
            const double w = j->wts[t + R];
            const double *src = j->b + (size_t)mirror(r + t, H) * W;
            for (int c = 0; c < W; ++c) dst[c] += w * src[c];
        }
        for (int c = 0; c < W; ++c) {
            if (dst[c] < mn) mn = dst[c];
            if (dst[c] > mx) mx = dst[c];
        }
    }
    j->mn = mn;
    j->mx = mx;
}

/* pass 3: rescale, add N(0, 8^2) noise, round half to even, clip */
static void pass_final(img_job *j) {
    const int W = j->W;
    const uint64_t HW = (uint64_t)j->H * (uint64_t)W;
    const double two_pi = 6.283185307179586476925286766559;
    for (int r = j->r0; r < j->r1; ++r) {
        const double *src = j->a + (size_t)r * W;
        uint8_t *dst = j->out + (size_t)r * (size_t)j->pitch;
        for (int c = 0; c < W; ++c) {
            uint64_t p = (uint64_t)r * W + c, q = p >> 1;
            double u1 = ((double)(synth_draw(j->seed, 2 + HW + 2 * q) >> 11) + 1.0) * 0x1.0p-53;
            double u2 = u53(synth_draw(j->seed, 2 + HW + 2 * q + 1));
            double rad = sqrt(-2.0 * log(u1));
            double z = (p & 1) ? rad * sin(two_pi * u2) : rad * cos(two_pi * u2);
            double v = (src[c] - j->lo) * j->scale + 8.0 * z;
            v = nearbyint(v);
            if (v < 0.0) v = 0.0;
            if (v > 255.0) v = 255.0;
            dst[c] = (uint8_t)v;
        }
    }
}

typedef void (*pass_fn)(img_job *);
typedef struct { img_job *job; pass_fn fn; } thr_arg;
static void *thr_main(void *p) {
    thr_arg *a = (thr_arg *)p;
    a->fn(a->job);
    return NULL;
}

static void run_rows(img_job *proto, int nthreads, pass_fn fn, img_job *jobs) {
    pthread_t tid[256];
    thr_arg args[256];
    int H = proto->H;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *proto;
        jobs[t].r0 = (int)((int64_t)H * t / nthreads);
        jobs[t].r1 = (int)((int64_t)H * (t + 1) / nthreads);
        args[t].job = &jobs[t];
        args[t].fn = fn;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&tid[t], NULL, thr_main, &args[t]);
    thr_main(&args[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(tid[t], NULL);
}

/* One image into out (row pitch `pitch` >= W); rows split over nthreads. */
int synth_image(uint64_t seed, int H, int W, double sigma, uint8_t *out, int pitch, int nthreads) {
    if (H < 1 || W < 1 || pitch < W || sigma <= 0.0 || !out) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > H) nthreads = H;
    int R = (int)ceil(4.0 * sigma);
    double *wts = (double *)malloc(sizeof(double) * (size_t)(2 * R + 1));
    double sum = 0.0;
    for (int t = -R; t <= R; ++t) sum += (wts[t + R] = exp(-(double)(t * t) / (2.0 * sigma * sigma)));
    for (int t = 0; t <= 2 * R; ++t) wts[t] /= sum;
    size_t n = (size_t)H * (size_t)W;
    double *a = (double *)malloc(sizeof(double) * n), *b = (double *)malloc(sizeof(double) * n);
    if (!a || !b) { free(a); free(b); free(wts); return 2; }
    img_job proto;
    memset(&proto, 0, sizeof proto);
    proto.seed = seed; proto.H = H; proto.W = W; proto.pitch = pitch; proto.radius = R;
    proto.wts = wts; proto.a = a; proto.b = b; proto.out = out;
    img_job jobs[256];
    run_rows(&proto, nthreads, pass_hblur, jobs);
    run_rows(&proto, nthreads, pass_vblur, jobs);
    double mn = INFINITY, mx = -INFINITY;
    for (int t = 0; t < nthreads; ++t) {
        if (jobs[t].r1 > jobs[t].r0) {
            if (jobs[t].mn < mn) mn = jobs[t].mn;
            if (jobs[t].mx > mx) mx = jobs[t].mx;
        }
    }
    proto.lo = mn;
    proto.scale = (mx > mn) ? 255.0 / (mx - mn) : 0.0;
    run_rows(&proto, nthreads, pass_final, jobs);
    free(a); free(b); free(wts);
    return 0;
}

/* ---- batch: images distributed over threads, one image per thread at a time ---- */
typedef struct {
    int n;
    const uint64_t *seeds;
    const int *H, *W, *pitch;
    const int64_t *offset;
    double sigma;
    uint8_t *base;
    int next; /* shared work counter */
    int err;
} batch_job;

static void *batch_worker(void *p) {
    batch_job *b = (batch_job *)p;
    for (;;) {
        int i = __atomic_fetch_add(&b->next, 1, __ATOMIC_RELAXED);
        if (i >= b->n) break;
        if (synth_image(b->seeds[i], b->H[i], b->W[i], b->sigma, b->base + b->offset[i], b->pitch[i], 1))
            __atomic_store_n(&b->err, 1, __ATOMIC_RELAXED);
    }
    return NULL;
}

/* n images; image i is written at base + offset[i] with row pitch pitch[i]. */
int synth_batch(int n, const uint64_t *seeds, const int *H, const int *W, const int *pitch,
                const int64_t *offset, double sigma, uint8_t *base, int nthreads) {
    if (n < 0 || !base) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    batch_job job = {n, seeds, H, W, pitch, offset, sigma, base, 0, 0};
    pthread_t tid[256];
    for (int t = 1; t < nthreads; ++t) pthread_create(&tid[t], NULL, batch_worker, &job);
    batch_worker(&job);
    for (int t = 1; t < nthreads; ++t) pthread_join(tid[t], NULL);
    return job.err;
}
