/*
 * CPU ORACLE for Local Directional Pattern (LDP) and Local Binary Pattern (LBP)
 * extraction -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, literal restatement of the method of "An Acceleration Scheme
 * to the Local Directional Pattern" (Ayami & Shabat, arXiv:1810.11518):
 *   Sec. 2.1          LBP codes, 256-bin histograms
 *   Sec. 2.2.1, Eq. 1 eight Kirsch compass responses (3x3 correlation)
 *   Sec. 2.2.2, Eq. 2-3 LDP code: bits of the k most outstanding responses
 *   Sec. 2.2.3, Eq. 4-6 code histograms / feature vector
 *   Sec. 2.3, Eq. 7-29  the paper's ALDP column-sum scheme (aldp.c)
 * It shares no code, header, table or helper with the CUDA library; only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may call it.
 *
 * Readings taken where the paper is silent or garbled:
 *   - x is the row, y the column; Eq. 1 is a correlation with mask M_i
 *     (the printed "M_1" is read as M_i).
 *   - M_0 is East and the masks run counter-clockwise (M_1 = NE, M_2 = N, ...,
 *     M_7 = SE); this orientation is the one Eqs. 22-29 reproduce.
 *   - "most outstanding" = largest |m_i|; exactly k bits are set, ties in
 *     |m_i| go to the lower direction index.
 *   - Only interior pixels (1 <= x <= H-2, 1 <= y <= W-2) get a code and are
 *     counted; the compact histogram orders the C(8,k) codes by value.
 *   - Regions: row band ri covers [floor(ri*H/R), floor((ri+1)*H/R)), column
 *     band rj covers [floor(rj*W/C), floor((rj+1)*W/C)), in image
 *     coordinates; region (ri, rj) is stored at (ri*C + rj) * nbins.
 *   - LBP: bit j is set when neighbour p_j >= centre, p_0..p_7 taken
 *     counter-clockwise from East like the masks.
 *   - Sliding windows (Sec. 3.2): windows start at multiples of the stride
 *     and are clipped at the image edge; with stride = size this reproduces
 *     every window count of Table 3 for a 280-pixel side.
 * All counters are uint32.
 */
#ifndef ORACLE_LDP_H
#define ORACLE_LDP_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The eight masks, M_i(row, col), rows top to bottom (Sec. 2.2.1). */
void oracle_kirsch_mask(int i, int32_t out3x3[9]);

/* m_0..m_7 at interior pixel (x, y) by Eq. 1. */
void oracle_responses(const uint8_t *img, int H, int W, int pitch, int x, int y, int32_t m[8]);

/* Eq. 2-3: stable sort of 0..7 by |m_i| descending, first k indices set. */
int oracle_code_from_responses(const int32_t m[8], int k);

/* Eq. 2-3 under each reading of the printed formula: ranking value |m_i|
 * (variant 0, 2) or m_i (1, 3); exactly k bits with ties to the lower index
 * (0, 1) or every bit with v_i >= v of the k-th ranked index (2, 3).
 * Variant 0 equals oracle_code_from_responses. */
int oracle_code_variant(const int32_t m[8], int k, int variant);

/* LBP label at interior pixel (x, y) (Sec. 2.1). */
int oracle_lbp_code(const uint8_t *img, int H, int W, int pitch, int x, int y);

/* Codes for interior pixels x in [x0,x1), y in [y0,y1) (image coordinates).
 * Code of (x, y) goes to codes[(x - x0) * code_pitch + (y - y0)].
 * mode: 0 = LDP with this k, 1 = LBP (k ignored), 2 / 3 / 4 = LDP code
 * variants 1 / 2 / 3 of oracle_code_variant.  Returns 0 or -1. */
int oracle_codes_rect(const uint8_t *img, int H, int W, int pitch, int mode, int k,
                      int x0, int x1, int y0, int y1, uint8_t *codes, int code_pitch);

/* Number of compact bins C(8,k), and the ascending list of codes with
 * popcount k (Eq. 6 ordering).  list may be NULL. */
int oracle_compact_codes(int k, int *list);

/* Position of `code` in the compact list for k, or -1. */
int oracle_bin_of_code(int code, int k);

/* Region bounds [lo, hi) of band b among nb bands over n pixels. */
void oracle_band(int n, int nb, int b, int *lo, int *hi);

/* Region histograms from a full interior code map (code of (x,y) at
 * codes[(x-1)*code_pitch + (y-1)]).  nbins_k = 0: 256 raw bins per region;
 * 1..7: compact C(8,k) bins.  hist is overwritten (R*C*nbins uint32). */
int oracle_region_hist(const uint8_t *codes, int H, int W, int code_pitch, int R, int C,
                       int nbins_k, uint32_t *hist);

/* Sliding windows along one axis of n pixels (Sec. 3.2, Table 3): window j
 * of size w at stride s covers [j*s, min(j*s + w, n)); there are 1 window
 * when n <= w, else ceil((n - w) / s) + 1 (the last one is clipped to n).
 * Returns -1 for w < 1 or s < 1. */
int oracle_window_count(int n, int w, int s);

/* Window histograms from a full interior code map (as oracle_region_hist):
 * window (a, b) covers image rows [a*sh, min(a*sh + wh, H)) and columns
 * [b*sw, min(b*sw + ww, W)), intersected with the interior, and is stored at
 * (a * nwc + b) * nbins with nwc = oracle_window_count(W, ww, sw).  hist is
 * overwritten. */
int oracle_window_hist(const uint8_t *codes, int H, int W, int code_pitch, int wh, int ww, int sh,
                       int sw, int nbins_k, uint32_t *hist);

/* Crop-and-resize front end (Sec. 3.1: faces resized to 260 x 260).
 * Bilinear resampling of the crop rectangle (rows cy..cy+ch-1, columns
 * cx..cx+cw-1 of the source) to OH x OW with half-pixel centres: output
 * pixel (i, j) samples the crop at y = (i + 1/2) * ch / OH - 1/2,
 * x = (j + 1/2) * cw / OW - 1/2, clamped to [0, ch-1] x [0, cw-1].  The
 * fraction of each coordinate is quantised to an 11-bit weight w1 =
 * round(frac * 2048) (halves up), w0 = 2048 - w1, all in exact integer
 * arithmetic on the rational coordinate, and
 *   out = (wy0 (wx0 p00 + wx1 p01) + wy1 (wx0 p10 + wx1 p11) + 2^21) >> 22.
 * Returns -1 on invalid arguments. */
int oracle_resize_bilinear(const uint8_t *src, int H, int W, int pitch, int cy, int cx, int ch, int cw,
                           uint8_t *dst, int OH, int OW, int dst_pitch);

/* The integer sampling position of output index i along an axis (the rule
 * above): first source index and the 11-bit weight of the next one. */
void oracle_resize_coord(int i, int n_src, int n_dst, int *i0, int *w1);

/* Distances between LDP descriptors (histograms used as feature vectors,
 * Sec. 3.2-3.3): for query rows q_a (nq x D, row stride ldq) and gallery rows
 * g_b (ng x D, row stride ldg),
 *   metric 0 (L1):            sum_d |q - g|
 *   metric 1 (intersection):  sum_d min(q, g)
 *   metric 2 (chi-square):    sum over d with q + g > 0 of (q - g)^2 / (q + g)
 * out[a * ldo + b]: uint64 for metrics 0 and 1, double for metric 2.
 * Returns -1 on invalid arguments. */
int oracle_hist_distance(const uint32_t *q, int nq, int ldq, const uint32_t *g, int ng, int ldg, int D,
                         int metric, void *out, int ldo);

/* Whole path for one image: codes (optional, may be NULL) + region hists.
 * mode as oracle_codes_rect; compact selects C(8,k) bins for the exact-k
 * LDP modes 0 and 2 (the threshold modes always count 256 raw bins). */
int oracle_extract(const uint8_t *img, int H, int W, int pitch, int mode, int k, int R, int C,
                   int compact, uint32_t *hist, uint8_t *codes, int code_pitch);

/* The same for n images, spread over nthreads host threads (one image per
 * thread at a time).  Image i: img_base + img_off[i], (H[i], W[i], pitch[i]);
 * hist at hist_base + hist_off[i] (uint32 elements); codes at
 * codes_base + code_off[i] with code_pitch[i] when codes_base != NULL. */
int oracle_extract_batch(int n, const uint8_t *img_base, const int64_t *img_off, const int *H,
                         const int *W, const int *pitch, int mode, int k, int R, int C, int compact,
                         uint32_t *hist_base, const int64_t *hist_off, uint8_t *codes_base,
                         const int64_t *code_off, const int *code_pitch, int nthreads);

/* ---- the paper's accelerated scheme (aldp.c) ---- */

/* m_0..m_7 at (x, y) from the fifteen column sums A0..A14 (Eqs. 7-29). */
void aldp_responses(const uint8_t *img, int H, int W, int pitch, int x, int y, int32_t m[8]);

/* m_i = 8*S3_i - 3*S8 from ring sums (the identity the GPU path uses). */
void ringsum_responses(const uint8_t *img, int H, int W, int pitch, int x, int y, int32_t m[8]);

/* Eq. 2 by rank counting: bit i set iff fewer than k indices j beat i
 * (|m_j| > |m_i|, or equal with j < i). */
int rank_code_from_responses(const int32_t m[8], int k);

/* Full-image LDP codes via ALDP responses + rank counting (CPU baseline). */
int aldp_codes(const uint8_t *img, int H, int W, int pitch, int k, uint8_t *codes, int code_pitch);

#ifdef __cplusplus
}
#endif
#endif
