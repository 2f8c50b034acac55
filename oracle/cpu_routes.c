/*
 * CPU ORACLE companion (test and CPU-baseline infrastructure only): LDP codes
 * and region histograms of a batch of images along one of three response
 * routes, on host threads, for the timed CPU baselines of bench.py.
 *
 *   route 0: the eight Kirsch masks applied literally (Eq. 1), as the oracle;
 *   route 1: the paper's accelerated scheme, fifteen column sums combined
 *            three at a time (Sec. 2.3, Eqs. 7-29, aldp_responses);
 *   route 2: the ring-sum identity m_i = 8 S3_i - 3 S8 (ringsum_responses).
 *
 * Every route ends in the same code step (Eqs. 2-3, the oracle's stable
 * sort by |m_i|) and the same region histograms (Eqs. 4-6), so a timing
 * ratio between routes isolates the response computation, the part the
 * paper accelerates (Sec. 2.3.3: LDP time = responses + histogram).
 */
#include <pthread.h>
#include <stdlib.h>

#include "oracle_ldp.h"

typedef struct {
    int route, n, H, W, pitch, k, R, C, nbins_k;
    const uint8_t *base;
    const int64_t *off;
    uint32_t *hist;
    int hist_len;
    int next, err;
} routes_ctx;

static int route_codes(int route, const uint8_t *img, int H, int W, int pitch, int k, uint8_t *codes) {
    const int cp = W - 2;
    for (int x = 1; x < H - 1; ++x)
        for (int y = 1; y < W - 1; ++y) {
            int32_t m[8];
            if (route == 0)
                oracle_responses(img, H, W, pitch, x, y, m);
            else if (route == 1)
                aldp_responses(img, H, W, pitch, x, y, m);
            else
                ringsum_responses(img, H, W, pitch, x, y, m);
            codes[(size_t)(x - 1) * cp + (size_t)(y - 1)] = (uint8_t)oracle_code_from_responses(m, k);
        }
    return 0;
}

static void *routes_worker(void *arg) {
    routes_ctx *c = (routes_ctx *)arg;
    uint8_t *codes = (uint8_t *)malloc((size_t)(c->H - 2) * (size_t)(c->W - 2));
    if (!codes) {
        __atomic_store_n(&c->err, 1, __ATOMIC_RELAXED);
        return NULL;
    }
    for (;;) {
        const int i = __atomic_fetch_add(&c->next, 1, __ATOMIC_RELAXED);
        if (i >= c->n) break;
        route_codes(c->route, c->base + c->off[i], c->H, c->W, c->pitch, c->k, codes);
        if (oracle_region_hist(codes, c->H, c->W, c->W - 2, c->R, c->C, c->nbins_k,
                               c->hist + (size_t)i * (size_t)c->hist_len))
            __atomic_store_n(&c->err, 1, __ATOMIC_RELAXED);
    }
    free(codes);
    return NULL;
}

/* The responses alone (the R part of Sec. 2.3.3), for timing the routes
 * without the shared code step: the sum over the n images of sum_i |m_i|
 * over every interior pixel (a checksum that keeps the work observable). */
int64_t route_response_sum(int route, int n, const uint8_t *base, const int64_t *off, int H, int W, int pitch) {
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        const uint8_t *img = base + off[i];
        for (int x = 1; x < H - 1; ++x)
            for (int y = 1; y < W - 1; ++y) {
                int32_t m[8];
                if (route == 0)
                    oracle_responses(img, H, W, pitch, x, y, m);
                else if (route == 1)
                    aldp_responses(img, H, W, pitch, x, y, m);
                else
                    ringsum_responses(img, H, W, pitch, x, y, m);
                for (int j = 0; j < 8; ++j) total += m[j] < 0 ? -m[j] : m[j];
            }
    }
    return total;
}

/* n images of H x W (row pitch `pitch`) at base + off[i]; histograms of an
 * R x C region grid (compact: C(8,k) bins per region, else 256 raw bins) to
 * hist + i * R*C*bins.  Returns 0, or -1 for bad arguments / an allocation
 * failure. */
int route_extract_batch(int route, int n, const uint8_t *base, const int64_t *off, int H, int W, int pitch,
                        int k, int R, int C, int compact, uint32_t *hist, int nthreads) {
    if (route < 0 || route > 2 || n < 0 || !base || !off || !hist || H < 3 || W < 3 || pitch < W || k < 1 ||
        k > 7 || R < 1 || C < 1)
        return -1;
    int nb = 256;
    if (compact) {
        nb = 1;
        for (int i = 1; i <= k; ++i) nb = nb * (8 - k + i) / i;
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    routes_ctx ctx = {route, n, H, W, pitch, k, R, C, compact ? k : 0, base, off, hist, R * C * nb, 0, 0};
    pthread_t tid[256];
    int started = 1;
    for (int t = 1; t < nthreads; ++t, ++started)
        if (pthread_create(&tid[t], NULL, routes_worker, &ctx)) break;
    routes_worker(&ctx);
    for (int t = 1; t < started; ++t) pthread_join(tid[t], NULL);
    return ctx.err ? -1 : 0;
}
