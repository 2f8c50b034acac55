/*
 * CPU ORACLE (test infrastructure only) -- literal LDP / LBP extraction.
 * See oracle_ldp.h for the readings of the paper this file follows.
 * Nothing here is blocked, fused or reordered: every pixel applies the eight
 * masks of Sec. 2.2.1 one by one (Eq. 1), sorts the responses (Eq. 2-3), and
 * histograms are counted from the finished code map (Eq. 4-6).
 */
#include "oracle_ldp.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/*
 * Kirsch compass masks (Sec. 2.2.1, Fig. 1; the figure is missing from the
 * text, the orientation is fixed by Eqs. 22-29): three 5s on consecutive ring
 * positions, -3 on the other five, 0 in the centre.  Rows top to bottom.
 */
static const int32_t KIRSCH[8][3][3] = {
    {{-3, -3, 5}, {-3, 0, 5}, {-3, -3, 5}},    /* M0  East       */
    {{-3, 5, 5}, {-3, 0, 5}, {-3, -3, -3}},    /* M1  North-East */
    {{5, 5, 5}, {-3, 0, -3}, {-3, -3, -3}},    /* M2  North      */
    {{5, 5, -3}, {5, 0, -3}, {-3, -3, -3}},    /* M3  North-West */
    {{5, -3, -3}, {5, 0, -3}, {5, -3, -3}},    /* M4  West       */
    {{-3, -3, -3}, {5, 0, -3}, {5, 5, -3}},    /* M5  South-West */
    {{-3, -3, -3}, {-3, 0, -3}, {5, 5, 5}},    /* M6  South      */
    {{-3, -3, -3}, {-3, 0, 5}, {-3, 5, 5}},    /* M7  South-East */
};

void oracle_kirsch_mask(int i, int32_t out3x3[9]) {
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) out3x3[a * 3 + b] = KIRSCH[i & 7][a][b];
}

static inline int32_t px(const uint8_t *img, int pitch, int x, int y) {
    return (int32_t)img[(size_t)x * (size_t)pitch + (size_t)y];
}

/* Eq. 1: m_i = sum_{k,l in {-1,0,1}} M_i(k+1, l+1) * I(x+k, y+l). */
void oracle_responses(const uint8_t *img, int H, int W, int pitch, int x, int y, int32_t m[8]) {
    (void)H;
    (void)W;
    for (int i = 0; i < 8; ++i) {
        int32_t s = 0;
        for (int k = -1; k <= 1; ++k)
            for (int l = -1; l <= 1; ++l) s += KIRSCH[i][k + 1][l + 1] * px(img, pitch, x + k, y + l);
        m[i] = s;
    }
}

static inline int32_t iabs32(int32_t v) { return v < 0 ? -v : v; }

/* Eq. 2-3 with |m_i| ranking: a stable insertion sort of the direction
 * indices by |m_i| descending (so equal magnitudes keep ascending index
 * order), then bit i = 1 for the first k indices of the sorted order. */
int oracle_code_from_responses(const int32_t m[8], int k) {
    int order[8];
    for (int i = 0; i < 8; ++i) order[i] = i;
    for (int i = 1; i < 8; ++i) {
        int v = order[i], j = i - 1;
        while (j >= 0 && iabs32(m[order[j]]) < iabs32(m[v])) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = v;
    }
    int code = 0;
    for (int r = 0; r < k && r < 8; ++r) code |= 1 << order[r];
    return code;
}

/* Eq. 2-3 under each reading of the printed formula.  The ranking value v_i
 * is |m_i| (variants 0, 2) or the signed response m_i (variants 1, 3).
 * Variants 0 / 1 set the first k indices of a stable sort by v descending
 * (exactly k bits, ties to the lower index); variants 2 / 3 apply s(x >= 0)
 * of Eq. 3 literally against the k-th index of that order, so every
 * response tied with it is set as well (k or more bits). */
int oracle_code_variant(const int32_t m[8], int k, int variant) {
    int32_t v[8];
    int order[8];
    for (int i = 0; i < 8; ++i) {
        v[i] = (variant & 1) ? m[i] : iabs32(m[i]);
        order[i] = i;
    }
    for (int i = 1; i < 8; ++i) {
        int o = order[i], j = i - 1;
        while (j >= 0 && v[order[j]] < v[o]) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = o;
    }
    int code = 0;
    if (variant < 2) {
        for (int r = 0; r < k && r < 8; ++r) code |= 1 << order[r];
    } else {
        const int32_t t = v[order[k - 1]];
        for (int i = 0; i < 8; ++i)
            if (v[i] - t >= 0) code |= 1 << i;
    }
    return code;
}

/* Sec. 2.1: threshold the 8-neighbourhood at the centre value; neighbour j
 * taken counter-clockwise from East, like the mask numbering. */
int oracle_lbp_code(const uint8_t *img, int H, int W, int pitch, int x, int y) {
    static const int dx[8] = {0, -1, -1, -1, 0, 1, 1, 1};
    static const int dy[8] = {1, 1, 0, -1, -1, -1, 0, 1};
    (void)H;
    (void)W;
    int32_t c = px(img, pitch, x, y), code = 0;
    for (int j = 0; j < 8; ++j)
        if (px(img, pitch, x + dx[j], y + dy[j]) >= c) code |= 1 << j;
    return code;
}

int oracle_codes_rect(const uint8_t *img, int H, int W, int pitch, int mode, int k, int x0, int x1,
                      int y0, int y1, uint8_t *codes, int code_pitch) {
    if (!img || !codes || H < 3 || W < 3 || pitch < W) return -1;
    if (x0 < 1 || y0 < 1 || x1 > H - 1 || y1 > W - 1 || x0 > x1 || y0 > y1) return -1;
    if (mode < 0 || mode > 4) return -1;
    if (mode != 1 && (k < 1 || k > 7)) return -1;
    for (int x = x0; x < x1; ++x)
        for (int y = y0; y < y1; ++y) {
            int code;
            if (mode == 0) {
                int32_t m[8];
                oracle_responses(img, H, W, pitch, x, y, m);
                code = oracle_code_from_responses(m, k);
            } else if (mode >= 2) {
                int32_t m[8];
                oracle_responses(img, H, W, pitch, x, y, m);
                code = oracle_code_variant(m, k, mode - 1);
            } else {
                code = oracle_lbp_code(img, H, W, pitch, x, y);
            }
            codes[(size_t)(x - x0) * (size_t)code_pitch + (size_t)(y - y0)] = (uint8_t)code;
        }
    return 0;
}

static int popcount8(int v) {
    int c = 0;
    for (int b = 0; b < 8; ++b) c += (v >> b) & 1;
    return c;
}

/* Eq. 6: the C(8,k) admissible codes, in ascending numeric order, found by
 * scanning all 256 byte values. */
int oracle_compact_codes(int k, int *list) {
    int n = 0;
    for (int v = 0; v < 256; ++v)
        if (popcount8(v) == k) {
            if (list) list[n] = v;
            ++n;
        }
    return n;
}

int oracle_bin_of_code(int code, int k) {
    int n = 0;
    for (int v = 0; v < 256; ++v)
        if (popcount8(v) == k) {
            if (v == code) return n;
            ++n;
        }
    return -1;
}

void oracle_band(int n, int nb, int b, int *lo, int *hi) {
    *lo = (int)(((int64_t)b * n) / nb);
    *hi = (int)(((int64_t)(b + 1) * n) / nb);
}

/* Eq. 4-5 per region: H_b = number of interior pixels of the region whose
 * code equals bin b's pattern. */
int oracle_region_hist(const uint8_t *codes, int H, int W, int code_pitch, int R, int C,
                       int nbins_k, uint32_t *hist) {
    if (!codes || !hist || H < 3 || W < 3 || R < 1 || C < 1 || nbins_k < 0 || nbins_k > 7) return -1;
    int nbins = nbins_k ? oracle_compact_codes(nbins_k, NULL) : 256;
    int bin_of[256];
    for (int v = 0; v < 256; ++v) bin_of[v] = nbins_k ? oracle_bin_of_code(v, nbins_k) : v;
    memset(hist, 0, sizeof(uint32_t) * (size_t)R * (size_t)C * (size_t)nbins);
    for (int ri = 0; ri < R; ++ri) {
        int xlo, xhi;
        oracle_band(H, R, ri, &xlo, &xhi);
        if (xlo < 1) xlo = 1;
        if (xhi > H - 1) xhi = H - 1;
        for (int rj = 0; rj < C; ++rj) {
            int ylo, yhi;
            oracle_band(W, C, rj, &ylo, &yhi);
            if (ylo < 1) ylo = 1;
            if (yhi > W - 1) yhi = W - 1;
            uint32_t *h = hist + ((size_t)ri * C + rj) * (size_t)nbins;
            for (int x = xlo; x < xhi; ++x)
                for (int y = ylo; y < yhi; ++y) {
                    int b = bin_of[codes[(size_t)(x - 1) * code_pitch + (size_t)(y - 1)]];
                    if (b >= 0) h[b] += 1;
                }
        }
    }
    return 0;
}

int oracle_window_count(int n, int w, int s) {
    if (w < 1 || s < 1 || n < 0) return -1;
    if (n <= w) return 1;
    return (n - w + s - 1) / s + 1;
}

int oracle_window_hist(const uint8_t *codes, int H, int W, int code_pitch, int wh, int ww, int sh,
                       int sw, int nbins_k, uint32_t *hist) {
    if (!codes || !hist || H < 3 || W < 3 || nbins_k < 0 || nbins_k > 7) return -1;
    int nr = oracle_window_count(H, wh, sh), nc = oracle_window_count(W, ww, sw);
    if (nr < 1 || nc < 1) return -1;
    int nbins = nbins_k ? oracle_compact_codes(nbins_k, NULL) : 256;
    int bin_of[256];
    for (int v = 0; v < 256; ++v) bin_of[v] = nbins_k ? oracle_bin_of_code(v, nbins_k) : v;
    memset(hist, 0, sizeof(uint32_t) * (size_t)nr * (size_t)nc * (size_t)nbins);
    for (int a = 0; a < nr; ++a) {
        int xlo = a * sh, xhi = a * sh + wh;
        if (xhi > H) xhi = H;
        if (xlo < 1) xlo = 1;
        if (xhi > H - 1) xhi = H - 1;
        for (int b = 0; b < nc; ++b) {
            int ylo = b * sw, yhi = b * sw + ww;
            if (yhi > W) yhi = W;
            if (ylo < 1) ylo = 1;
            if (yhi > W - 1) yhi = W - 1;
            uint32_t *h = hist + ((size_t)a * nc + b) * (size_t)nbins;
            for (int x = xlo; x < xhi; ++x)
                for (int y = ylo; y < yhi; ++y) {
                    int bin = bin_of[codes[(size_t)(x - 1) * code_pitch + (size_t)(y - 1)]];
                    if (bin >= 0) h[bin] += 1;
                }
        }
    }
    return 0;
}

/* Sample position of output index i: y = ((2i + 1) n_src - n_dst) / (2 n_dst)
 * exactly; i0 = floor(y), w1 = round((y - i0) * 2048) with halves up;
 * y < 0 clamps to (0, 0) and y >= n_src - 1 to (n_src - 1, 0). */
void oracle_resize_coord(int i, int n_src, int n_dst, int *i0, int *w1) {
    const long long num = (2LL * i + 1) * (long long)n_src - (long long)n_dst;  /* y * 2 n_dst */
    const long long den = 2LL * n_dst;
    if (num <= 0) {
        *i0 = 0;
        *w1 = 0;
        return;
    }
    long long q = num / den, r = num - q * den;
    long long w = (r * 2048 + den / 2) / den;  /* round half up (den is even) */
    if (w == 2048) {
        q += 1;
        w = 0;
    }
    if (q >= n_src - 1) {
        *i0 = n_src - 1;
        *w1 = 0;
        return;
    }
    *i0 = (int)q;
    *w1 = (int)w;
}

int oracle_resize_bilinear(const uint8_t *src, int H, int W, int pitch, int cy, int cx, int ch, int cw,
                           uint8_t *dst, int OH, int OW, int dst_pitch) {
    if (!src || !dst || H < 1 || W < 1 || pitch < W || ch < 1 || cw < 1 || OH < 1 || OW < 1 || dst_pitch < OW)
        return -1;
    if (cy < 0 || cx < 0 || cy + ch > H || cx + cw > W) return -1;
    for (int i = 0; i < OH; ++i) {
        int y0, wy1;
        oracle_resize_coord(i, ch, OH, &y0, &wy1);
        const int y1 = (y0 + 1 < ch) ? y0 + 1 : y0, wy0 = 2048 - wy1;
        for (int j = 0; j < OW; ++j) {
            int x0, wx1;
            oracle_resize_coord(j, cw, OW, &x0, &wx1);
            const int x1 = (x0 + 1 < cw) ? x0 + 1 : x0, wx0 = 2048 - wx1;
            const long long p00 = src[(size_t)(cy + y0) * pitch + (size_t)(cx + x0)];
            const long long p01 = src[(size_t)(cy + y0) * pitch + (size_t)(cx + x1)];
            const long long p10 = src[(size_t)(cy + y1) * pitch + (size_t)(cx + x0)];
            const long long p11 = src[(size_t)(cy + y1) * pitch + (size_t)(cx + x1)];
            const long long v = wy0 * (wx0 * p00 + wx1 * p01) + wy1 * (wx0 * p10 + wx1 * p11);
            dst[(size_t)i * dst_pitch + (size_t)j] = (uint8_t)((v + (1LL << 21)) >> 22);
        }
    }
    return 0;
}

int oracle_hist_distance(const uint32_t *q, int nq, int ldq, const uint32_t *g, int ng, int ldg, int D,
                         int metric, void *out, int ldo) {
    if (!q || !g || !out || nq < 1 || ng < 1 || D < 1 || ldq < D || ldg < D || ldo < ng) return -1;
    if (metric < 0 || metric > 2) return -1;
    for (int a = 0; a < nq; ++a)
        for (int b = 0; b < ng; ++b) {
            const uint32_t *x = q + (size_t)a * ldq, *y = g + (size_t)b * ldg;
            uint64_t acc = 0;
            double chi = 0.0;
            for (int d = 0; d < D; ++d) {
                const uint64_t u = x[d], v = y[d];
                if (metric == 0) acc += u > v ? u - v : v - u;
                else if (metric == 1) acc += u < v ? u : v;
                else if (u + v > 0) chi += ((double)u - (double)v) * ((double)u - (double)v) / ((double)u + (double)v);
            }
            if (metric == 2) ((double *)out)[(size_t)a * ldo + b] = chi;
            else ((uint64_t *)out)[(size_t)a * ldo + b] = acc;
        }
    return 0;
}

int oracle_extract(const uint8_t *img, int H, int W, int pitch, int mode, int k, int R, int C,
                   int compact, uint32_t *hist, uint8_t *codes, int code_pitch) {
    if (!img || H < 3 || W < 3 || pitch < W) return -1;
    if (mode < 0 || mode > 4) return -1;
    if (mode != 1 && (k < 1 || k > 7)) return -1;
    int own = 0;
    if (!codes) {
        code_pitch = W - 2;
        codes = (uint8_t *)malloc((size_t)(H - 2) * (size_t)(W - 2));
        if (!codes) return -1;
        own = 1;
    }
    int rc = oracle_codes_rect(img, H, W, pitch, mode, k, 1, H - 1, 1, W - 1, codes, code_pitch);
    if (rc == 0 && hist)
        rc = oracle_region_hist(codes, H, W, code_pitch, R, C, ((mode == 0 || mode == 2) && compact) ? k : 0,
                                hist);
    if (own) free(codes);
    return rc;
}

typedef struct {
    int n;
    const uint8_t *img_base;
    const int64_t *img_off;
    const int *H, *W, *pitch;
    int mode, k, R, C, compact;
    uint32_t *hist_base;
    const int64_t *hist_off;
    uint8_t *codes_base;
    const int64_t *code_off;
    const int *code_pitch;
    int next, err;
} batch_ctx;

static void *batch_worker(void *p) {
    batch_ctx *b = (batch_ctx *)p;
    for (;;) {
        int i = __atomic_fetch_add(&b->next, 1, __ATOMIC_RELAXED);
        if (i >= b->n) break;
        uint8_t *codes = b->codes_base ? b->codes_base + b->code_off[i] : NULL;
        int cp = b->codes_base ? b->code_pitch[i] : 0;
        uint32_t *hist = b->hist_base ? b->hist_base + b->hist_off[i] : NULL;
        if (oracle_extract(b->img_base + b->img_off[i], b->H[i], b->W[i], b->pitch[i], b->mode, b->k,
                           b->R, b->C, b->compact, hist, codes, cp))
            __atomic_store_n(&b->err, 1, __ATOMIC_RELAXED);
    }
    return NULL;
}

int oracle_extract_batch(int n, const uint8_t *img_base, const int64_t *img_off, const int *H,
                         const int *W, const int *pitch, int mode, int k, int R, int C, int compact,
                         uint32_t *hist_base, const int64_t *hist_off, uint8_t *codes_base,
                         const int64_t *code_off, const int *code_pitch, int nthreads) {
    if (n < 0 || !img_base) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    batch_ctx ctx = {n, img_base, img_off, H, W, pitch, mode, k, R, C, compact,
                     hist_base, hist_off, codes_base, code_off, code_pitch, 0, 0};
    pthread_t tid[256];
    int started = 1;
    for (int t = 1; t < nthreads; ++t, ++started)
        if (pthread_create(&tid[t], NULL, batch_worker, &ctx)) break;
    batch_worker(&ctx);
    for (int t = 1; t < started; ++t) pthread_join(tid[t], NULL);
    return ctx.err ? -1 : 0;
}
