/*
 * libldp -- Local Directional Pattern (LDP) and Local Binary Pattern (LBP)
 * feature extraction on NVIDIA GB300 (sm_103a).
 *
 * Method: Ayami & Shabat, "An Acceleration Scheme to the Local Directional
 * Pattern", arXiv:1810.11518.
 *   Sec. 2.2.1, Eq. 1   eight Kirsch compass responses m_0..m_7 per pixel
 *   Sec. 2.2.2, Eq. 2-3 LDP code: bits of the k most outstanding responses
 *   Sec. 2.2.3, Eq. 4-6 code histograms (feature vectors), here per region
 *   Sec. 2.1            LBP codes and 256-bin histograms (the comparison)
 *   Sec. 3.2            windowed extraction, here an R x C grid of regions
 *
 * Conventions fixed by this library (the paper leaves them open):
 *   - Images are uint8, row-major, H rows x W columns, row pitch >= W bytes.
 *     x is the row, y the column; M_0 is East and the masks run
 *     counter-clockwise (M_1 = NE, M_2 = N, ..., M_7 = SE); code bit i
 *     belongs to mask i.  Eq. 1 is a correlation.
 *   - Ranking is by |m_i|, exactly k bits are set, and equal |m_i| are
 *     ranked by lower direction index first.
 *   - Only interior pixels (1 <= x <= H-2, 1 <= y <= W-2) have a code and
 *     are counted.  The code of (x, y) is stored at
 *     codes[(x-1)*code_pitch + (y-1)]; code_pitch >= W-2.
 *   - Region (ri, rj) of an R x C grid holds rows
 *     [floor(ri*H/R), floor((ri+1)*H/R)) and columns
 *     [floor(rj*W/C), floor((rj+1)*W/C)) of the image; its histogram is
 *     stored at hist[(ri*C + rj)*nbins ...].  nbins is 256 (raw code
 *     values) or, for LDP with compact = 1, C(8,k) bins ordered by ascending
 *     code value (Eq. 6).  Counters are uint32.
 *   - LBP bit j is set when neighbour p_j >= centre, p_0 = East,
 *     counter-clockwise; 256 bins.
 *
 * Memory and streams: every image, code and histogram buffer is a device
 * pointer owned by the caller.  Calls are asynchronous and ordered on the
 * CUDA stream passed as `stream` (a cudaStream_t; NULL = legacy default
 * stream); the caller synchronises before reading results.  Histogram
 * buffers are overwritten (zeroed on the stream first).  The library owns
 * only opaque batch plans.
 *
 * Errors: every entry point returns an ldp_status and never aborts or traps.
 * LDP_EINVAL rejects bad arguments before anything is launched; CUDA launch
 * or runtime errors give LDP_ECUDA.  ldp_last_error() returns a message for
 * the calling thread's most recent failure.
 *
 * Alignment: any pointer and pitch are accepted.  16-byte aligned image and
 * code buffers with pitches that are multiples of 16 take the fast path;
 * other layouts are processed correctly by a slower byte-wise path.  There
 * is no CPU fallback: the work always runs on the GPU.
 */
#ifndef LDP_H
#define LDP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LDP_API __attribute__((visibility("default")))
#else
#define LDP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LDP_OK = 0,
    LDP_EINVAL = 1,   /* invalid argument, nothing launched */
    LDP_ECUDA = 2,    /* CUDA runtime / launch error */
    LDP_ENOMEM = 3,   /* device or host allocation failed */
    LDP_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    LDP_ENOTIMPL = 5  /* combination not supported */
} ldp_status;

/* R x C grid of regions (Sec. 3.2 windows); compact = 1 selects the C(8,k)
 * bins of Eq. 6 for LDP, 0 the 256 raw code values.  R, C >= 1. */
typedef struct {
    int32_t R, C;
    int32_t compact;
} ldp_region_spec;

/* One image of a batch, resident in device memory.  codes may be NULL (no
 * code map for that image).  hist_offset counts uint32 elements from the
 * d_hist pointer given to the batch run.  40 bytes, 8-byte aligned. */
typedef struct {
    const uint8_t *img;
    int32_t H, W, pitch, code_pitch;
    uint8_t *codes;
    uint64_t hist_offset;
} ldp_image_desc;

/* ---- single image ---- */

/* LDP codes (Eq. 1-3) of the interior of one image.
 * d_img: H x W, row pitch `pitch` bytes.  k in [1,7].
 * d_codes: (H-2) x (W-2), row pitch code_pitch >= W-2.
 * EINVAL: NULL pointer, H < 3, W < 3, pitch < W, code_pitch < W-2, k out
 * of range, H or W > 1<<20. */
LDP_API int ldp_codes(const uint8_t *d_img, int H, int W, int pitch, int k, uint8_t *d_codes,
              int code_pitch, void *stream);

/* LDP codes fused with region histograms (Eq. 1-6): one launch computes
 * the codes, optionally stores them (d_codes_or_null), and accumulates the
 * R x C region histograms into d_hist (R*C*nbins uint32, overwritten).
 * EINVAL as ldp_codes, plus R < 1, C < 1, compact not 0/1, d_hist NULL. */
LDP_API int ldp_region_hist(const uint8_t *d_img, int H, int W, int pitch, int k, ldp_region_spec rs,
                    uint32_t *d_hist, uint8_t *d_codes_or_null, int code_pitch, void *stream);

/* LBP codes (Sec. 2.1) of the interior of one image; layout as ldp_codes. */
LDP_API int lbp_codes(const uint8_t *d_img, int H, int W, int pitch, uint8_t *d_codes, int code_pitch,
              void *stream);

/* LBP codes fused with 256-bin region histograms (R x C regions). */
LDP_API int lbp_region_hist(const uint8_t *d_img, int H, int W, int pitch, int R, int C, uint32_t *d_hist,
                    uint8_t *d_codes_or_null, int code_pitch, void *stream);

/* ---- crop-and-resize front end (Sec. 3.1) ---- */

/* One crop of a batch: rows cy..cy+ch-1, columns cx..cx+cw-1 of the source
 * image (H x W, row pitch `pitch`), resized into dst (row pitch dst_pitch).
 * 48 bytes, 8-byte aligned. */
typedef struct {
    const uint8_t *src;
    uint8_t *dst;
    int32_t H, W, pitch;
    int32_t cy, cx, ch, cw;
    int32_t dst_pitch;
} ldp_crop_desc;

/* Bilinear crop-and-resize (the paper resizes detected faces to 260 x 260
 * before extraction; detection itself is not part of the library): output
 * pixel (i, j) samples the crop at ((i + 1/2) ch / OH - 1/2,
 * (j + 1/2) cw / OW - 1/2), clamped to the crop; the fractions become 11-bit
 * weights (round half up) computed in exact integer arithmetic, and the
 * result is (sum of weight products x pixels + 2^21) >> 22.  d_dst: OH x OW,
 * row pitch dst_pitch >= OW.  EINVAL: NULL pointers, the crop outside the
 * image, sizes < 1, pitch < W, dst_pitch < OW, OH or OW > 1<<16. */
LDP_API int ldp_resize(const uint8_t *d_src, int H, int W, int pitch, int cy, int cx, int ch, int cw,
                       uint8_t *d_dst, int OH, int OW, int dst_pitch, void *stream);

/* Every crop of d_descs[0..count) (device memory, count a host value) to
 * OH x OW in one launch.  A descriptor that fails the checks of ldp_resize
 * is skipped and sets bit 3 of the device status word (ldp_device_status). */
LDP_API int ldp_batch_resize(const ldp_crop_desc *d_descs, int count, int OH, int OW, void *stream);

/* ---- distances between descriptors (matching LDP feature vectors) ---- */

#define LDP_DIST_L1 0        /* sum |q - g|, uint64 out */
#define LDP_DIST_INTERSECT 1 /* sum min(q, g), uint64 out */
#define LDP_DIST_CHI2 2      /* sum over q + g > 0 of (q - g)^2 / (q + g), float out */

/* Distance of every query row (d_q: nq x D uint32, row stride ldq) to every
 * gallery row (d_g: ng x D, row stride ldg), e.g. region or window
 * histograms of images: d_out[a * ldo + b] (uint64 for L1 / intersection,
 * float for chi-square).  Integer metrics are exact for counts below 2^27;
 * chi-square runs in fp32 (counts exact below 2^24): relative error at most
 * (D + 5) * 2^-24 (every term is non-negative).  EINVAL: NULL pointers,
 * nq, ng or D < 1, ldq < D, ldg < D, ldo < ng, unknown metric. */
LDP_API int ldp_hist_distance(const uint32_t *d_q, int nq, int ldq, const uint32_t *d_g, int ng, int ldg, int D,
                              int metric, void *d_out, int ldo, void *stream);

/* ---- readings of Eq. 2-3 (code modes) ----
 * Eq. 2 sets s(m_i - m_k) for the k-th "most outstanding" response; the
 * printed formula leaves the ranking (|m_i| or m_i) and the treatment of ties
 * open.  LDP_CODE_ABS is the default everywhere else in this API. */
#define LDP_CODE_ABS 0        /* the k largest |m_i|, exactly k bits, ties to the lower index */
#define LDP_CODE_RAW 1        /* the k largest signed m_i, exactly k bits, ties to the lower index */
#define LDP_CODE_ABS_THRESH 2 /* every i with |m_i| >= the k-th largest |m| (k or more bits) */
#define LDP_CODE_RAW_THRESH 3 /* every i with m_i >= the k-th largest m (k or more bits) */

/* ldp_codes with a code mode (LDP_CODE_*).  EINVAL as ldp_codes, plus
 * code_mode out of range. */
LDP_API int ldp_codes_ex(const uint8_t *d_img, int H, int W, int pitch, int k, int code_mode, uint8_t *d_codes,
                         int code_pitch, void *stream);

/* ldp_region_hist with a code mode.  The threshold modes produce codes of k
 * or more bits, so they count 256 raw bins: rs.compact must be 0 (EINVAL
 * otherwise). */
LDP_API int ldp_region_hist_ex(const uint8_t *d_img, int H, int W, int pitch, int k, int code_mode,
                               ldp_region_spec rs, uint32_t *d_hist, uint8_t *d_codes_or_null, int code_pitch,
                               void *stream);

/* ---- sliding windows (Sec. 3.2, Table 3) ---- */

/* Windows of wh x ww pixels whose origins step by (sh, sw): window (a, b)
 * covers image rows [a*sh, min(a*sh + wh, H)) and columns
 * [b*sw, min(b*sw + ww, W)), interior pixels only (windows overlap when the
 * stride is below the size, leave gaps when above).  compact as in
 * ldp_region_spec.  All five fields >= 1 except compact (0 or 1). */
typedef struct {
    int32_t wh, ww;
    int32_t sh, sw;
    int32_t compact;
} ldp_window_spec;

/* Windows along one axis of n pixels: 1 when n <= w, else
 * ceil((n - w) / s) + 1 (the last one clipped at n).  -1 when w < 1 or
 * s < 1.  With s = w this is ceil(n / w): Table 3's counts for n = 280. */
LDP_API int ldp_window_count(int n, int w, int s);

/* Device scratch bytes ldp_window_hist / lbp_window_hist need for an H x W
 * image (k = 0: LBP or raw bins): a code map of (H-2) x (W-2) bytes unless
 * codes_given, plus the cell histograms (cells of gcd(size, stride) pixels)
 * when the windows overlap or leave gaps and cannot take the single fused
 * pass -- which needs the column stride to divide the window width, windows
 * of at most 65535 pixels (the pass counts in 16-bit halves) and the
 * window's rows of cells to fit in shared memory.  0 on invalid arguments. */
LDP_API uint64_t ldp_window_scratch_bytes(int H, int W, int k, ldp_window_spec ws, int codes_given);

/* LDP codes of one image (Eq. 1-3), then the histogram of every sliding
 * window (Eq. 4-6 per window, Sec. 3.2) into d_hist: nwr x nwc x nbins
 * uint32 (every element written), nwr = ldp_window_count(H, wh, sh),
 * nwc = ldp_window_count(W, ww, sw).  Codes go to d_codes_or_null
 * (code_pitch) or to the scratch.  d_scratch: at least
 * ldp_window_scratch_bytes(H, W, k, ws, d_codes_or_null != NULL) bytes,
 * 256-byte aligned, owned by the caller (NULL when that is 0).  EINVAL as
 * ldp_region_hist, plus a bad window spec or short scratch. */
LDP_API int ldp_window_hist(const uint8_t *d_img, int H, int W, int pitch, int k, ldp_window_spec ws,
                            uint32_t *d_hist, uint8_t *d_codes_or_null, int code_pitch, void *d_scratch,
                            uint64_t scratch_bytes, void *stream);

/* The same with LBP codes (Sec. 2.1) and 256 raw bins (ws.compact must be 0). */
LDP_API int lbp_window_hist(const uint8_t *d_img, int H, int W, int pitch, ldp_window_spec ws, uint32_t *d_hist,
                            uint8_t *d_codes_or_null, int code_pitch, void *d_scratch, uint64_t scratch_bytes,
                            void *stream);

/* Scratch bytes of ldp_batch_window_hist: count x (cell words of a
 * max_H x max_W image) x 4, or 0 when no cell scratch is needed (stride =
 * size, or the fused pass of ldp_window_scratch_bytes applies). */
LDP_API uint64_t ldp_batch_window_scratch_bytes(int count, int max_H, int max_W, int k, ldp_window_spec ws);

/* Window histograms of `count` images (host value) from code maps already
 * in device memory, e.g. stored by ldp_batch_run: image i is d_descs[i]
 * (codes, code_pitch, H, W; img unused), its windows go to
 * d_hist + hist_offset.  Every image must satisfy 3 <= H <= max_H,
 * 3 <= W <= max_W and code_pitch >= W - 2: one that does not is skipped
 * and sets bit 0 of the device status word (ldp_device_status); images with
 * codes == NULL are skipped.  k >= 1 with ws.compact = 1: C(8,k) bins; else
 * 256 raw bins (k = 0 for LBP maps). */
LDP_API int ldp_batch_window_hist(const ldp_image_desc *d_descs, int count, int max_H, int max_W, int k,
                                  ldp_window_spec ws, uint32_t *d_hist, void *d_scratch, uint64_t scratch_bytes,
                                  void *stream);

/* ---- batches of images of any sizes: one persistent launch ---- */

typedef struct ldp_batch_plan ldp_batch_plan;

#define LDP_PLAN_LBP 1u       /* plan runs LBP (k ignored, 256 bins) */
#define LDP_PLAN_NO_GRAPH 2u  /* launch kernels directly instead of replaying a CUDA graph */
/* code mode of an LDP plan (LDP_CODE_*, default LDP_CODE_ABS); plans of the
 * other modes run one fixed tile shape (ldp_batch_plan_set_config keeps the
 * CTAs per SM only) */
#define LDP_PLAN_CODE_MODE(m) (((unsigned)(m) & 3u) << 2)

/* Creates a plan for batches of up to max_images images holding up to
 * max_pixels pixels in total.  The plan owns its device work-list scratch
 * (allocated here, sized for the tile height of variant 0: at most
 * max_pixels (TH + 129) / (384 TH) + max_images + 1 tiles of TH rows x 128
 * columns, enough for any batch within the two bounds) and a CUDA graph of
 * its launches (built on first run).  A batch whose descriptors hold more
 * than max_pixels pixels is clamped on the device and sets bit 1 of the
 * device status word; the checked build reports it as LDP_EINVAL.
 * EINVAL: out NULL, max_images < 1, bad k / rs; ENOMEM on allocation
 * failure. */
LDP_API int ldp_batch_plan_create(ldp_batch_plan **out, int max_images, uint64_t max_pixels, int k,
                          ldp_region_spec rs, unsigned flags);

/* Runs the plan: the image count is read from device memory (*d_count,
 * clamped to max_images), descriptors from d_descs[0..count), so one
 * captured graph serves any count.  Each image's histogram
 * (R*C*nbins uint32 at d_hist + hist_offset) is zeroed and accumulated;
 * its codes are stored when desc.codes != NULL.  Images whose descriptor
 * is invalid (H < 3, W < 3, pitch < W, NULL img, or codes with
 * code_pitch < W-2) are skipped and flagged in the device status word.
 * Stream-ordered; d_descs, d_count and d_hist must stay valid until the
 * work completes.  ldp_batch_run requires an LDP plan, lbp_batch_run an
 * LBP plan (EINVAL otherwise). */
LDP_API int ldp_batch_run(ldp_batch_plan *plan, const ldp_image_desc *d_descs, const int *d_count,
                  uint32_t *d_hist, void *stream);
LDP_API int lbp_batch_run(ldp_batch_plan *plan, const ldp_image_desc *d_descs, const int *d_count,
                  uint32_t *d_hist, void *stream);

/* Kernel timing: after enable_timing(plan, capacity), each of the next
 * `capacity` runs records a pair of CUDA events around its persistent
 * kernel (inside the CUDA graph too, by updating the graph's event-record
 * nodes).  kernel_times() waits for the recorded events, writes the
 * elapsed milliseconds of up to `capacity` runs (in run order) to ms,
 * stores their number in *count, and starts a new recording. */
LDP_API int ldp_batch_plan_enable_timing(ldp_batch_plan *plan, int capacity);
LDP_API int ldp_batch_plan_kernel_times(ldp_batch_plan *plan, float *ms, int capacity, int *count);

/* Frees the plan's device scratch, events and graph (synchronises the device). */
LDP_API int ldp_batch_plan_destroy(ldp_batch_plan *plan);

/* Kernel configuration (tile shape / CTAs per SM) a plan uses; set by the
 * autotuner.  variant in [0, ldp_num_variants()), ctas_per_sm 0 = as many
 * as fit.  A variant of shorter tiles than the plan's work list was sized
 * for reallocates the work list (synchronising the device); on failure
 * (ENOMEM, or EINVAL when the list would exceed 1.5e9 tiles) the plan keeps
 * its previous configuration. */
LDP_API int ldp_batch_plan_set_config(ldp_batch_plan *plan, int variant, int ctas_per_sm);
LDP_API int ldp_num_variants(void);
/* Short description of a variant, static storage: "r<rows per warp tile>
 * w<warps per CTA> b<min CTAs per SM> t<1: rows staged by the bulk-copy
 * engine>" and a trailing "s" when a tile narrower than 64 columns shares
 * its rows among lane groups, or "f" when the shared histogram slots hold
 * the current region row only and are flushed at each region-row boundary
 * (e.g. "r128w4b7t0", "r64w4b7t0s", "r128w4b6t0f"). */
LDP_API const char *ldp_variant_name(int variant);
/* Variant used by the single-image entry points; -1 (the default) chooses
 * by image size: short warp tiles for images of few 64-row tiles (their
 * latency is that of one tile: 4-row tiles while the image has fewer 8-row
 * tiles than the GPU has warp schedulers, then 8 and 16 rows), 64-row
 * tiles for large images. */
LDP_API int ldp_set_plain_variant(int variant);

/* ---- host-to-host pipeline: copies and compute overlapped ---- */

/* Extraction of images that live in host memory: the batch is cut into
 * chunks of consecutive images (at most chunk_images images and chunk_pixels
 * pixels each); chunk c goes through device buffer c % nbuf -- images copied
 * in, codes and histograms computed by that buffer's batch plan (k, rs and
 * flags as ldp_batch_plan_create), results copied back -- on the buffer's
 * own stream, so copy-in, kernels and copy-out of different chunks overlap.
 * The pipeline owns nbuf device buffers (grown on first use), plans and
 * streams.  EINVAL: bad sizes, nbuf outside [1, 8], LDP_PLAN_NO_GRAPH;
 * ENOMEM on allocation failure. */
typedef struct ldp_pipeline ldp_pipeline;
LDP_API int ldp_pipeline_create(ldp_pipeline **out, int chunk_images, uint64_t chunk_pixels, int k,
                                ldp_region_spec rs, int nbuf, unsigned flags);

/* Runs `count` images: image i at h_img + img_off[i] (H[i] x W[i], row
 * pitch[i]; offsets non-decreasing), its codes to h_codes + code_off[i] with
 * code_pitch[i] (h_codes NULL: no codes), its histograms to
 * h_hist + i * (R*C*nbins).  Host buffers should be pinned; they must stay
 * valid until `stream` has passed the run: the pipeline starts after work
 * already queued on `stream`, and `stream` waits for the whole run, so
 * synchronising it means every result is in place.  The host arrays are read
 * before the call returns. */
LDP_API int ldp_pipeline_run(ldp_pipeline *p, int count, const uint8_t *h_img, const int64_t *img_off,
                             const int *H, const int *W, const int *pitch, uint8_t *h_codes,
                             const int64_t *code_off, const int *code_pitch, uint32_t *h_hist, void *stream);

/* Tile variant and CTAs per SM of every plan of the pipeline (as
 * ldp_batch_plan_set_config). */
LDP_API int ldp_pipeline_set_config(ldp_pipeline *p, int variant, int ctas_per_sm);

/* Waits for the pipeline's work and frees everything it owns.  NULL is a no-op. */
LDP_API int ldp_pipeline_destroy(ldp_pipeline *p);

/* ---- serving: continuous batching of single-image requests ---- */

/* A request runtime: images submitted one by one from host memory are
 * admitted into a resident device arena when their buffers fit (admission by
 * free device memory), gathered into batches as they arrive, and run by the
 * batched kernel on `streams` concurrent streams, so batches overlap on the
 * device (one copying in while another computes or copies out).  Results go
 * back to the caller's host buffers; completions are collected with
 * ldp_server_poll.  Each request gets exactly the codes and histograms that
 * ldp_region_hist gives for the same image (LDP, k and rs of the config). */
typedef struct ldp_server ldp_server;

typedef struct {
    int32_t max_batch;     /* requests per batch launch, >= 1 */
    int32_t streams;       /* batches in flight, 1..16 */
    uint64_t arena_bytes;  /* device memory for resident request buffers */
    int32_t k;             /* LDP k, 1..7 */
    ldp_region_spec rs;    /* region histograms of every request */
    int32_t variant;       /* tile variant (-1: default) */
    int32_t ctas_per_sm;   /* 0: as many as fit */
} ldp_server_config;

typedef struct {
    uint64_t tag;          /* the caller's tag from ldp_server_submit */
    uint64_t t_submit_ns;  /* steady-clock times: submitted, */
    uint64_t t_start_ns;   /* admitted into a batch, */
    uint64_t t_done_ns;    /* results in the caller's buffers */
} ldp_completion;

typedef struct {
    uint64_t completed, pixels, batches, pending, arena_used, arena_bytes;
} ldp_server_stats_t;

/* Creates the runtime (allocates the arena and per-stream buffers, runs each
 * stream's batch plans once on an empty batch so that their kernels are
 * loaded and their CUDA graphs captured before the first request, starts a
 * dispatcher and a completion thread).  EINVAL on a bad config, ENOMEM when
 * an allocation fails, ECUDA when the warm-up fails. */
LDP_API int ldp_server_create(ldp_server **out, const ldp_server_config *cfg);

/* Queues one request.  host_img (H x W, row pitch `pitch`) must stay valid
 * and unchanged until the request completes (pinned memory lets the copy run
 * asynchronously).  host_codes ((H-2) x (W-2), row pitch code_pitch) may be
 * NULL; host_hist (R*C*nbins uint32) may be NULL.  Never blocks on the GPU.
 * EINVAL for a bad shape or an image larger than the arena; ECUDA once the
 * runtime has hit a CUDA error (the message says which). */
LDP_API int ldp_server_submit(ldp_server *s, const uint8_t *host_img, int H, int W, int pitch,
                              uint8_t *host_codes, int code_pitch, uint32_t *host_hist, uint64_t tag);

/* Moves up to `max` completed requests (completion order) into out; *n_out
 * is their number. */
LDP_API int ldp_server_poll(ldp_server *s, ldp_completion *out, int max, int *n_out);

/* Counters since creation. */
LDP_API int ldp_server_stats(ldp_server *s, ldp_server_stats_t *out);

/* Completes every submitted request, stops the threads and frees
 * everything. */
LDP_API int ldp_server_destroy(ldp_server *s);

/* Batch run that allocates nothing, for callers that cannot call
 * cudaMalloc / cudaFree while they run (device memory budgeted once at
 * start-up, memory owned by another allocator's pool, or loops that must
 * not risk an allocation failure or the device-wide synchronisation
 * cudaFree can cause).  The paper has no counterpart: it is a deployment
 * variant of ldp_batch_run.
 *
 * Same work as an LDP plan run (codes when desc.codes != NULL, region
 * histograms zeroed and accumulated in d_hist when d_hist != NULL), but:
 *   - count (number of descriptors in d_descs) is a host value;
 *   - no plan and no CUDA graph: four direct kernel launches on `stream`;
 *   - the work list lives in one static device array of 2^21 ints (8 MiB)
 *     that every GPU loading the library keeps until the process exits.
 *     The caller bounds the batch by max_pixels (sum of H*W) and max_side
 *     (largest H or W); the call returns LDP_EINVAL, with the sizes in
 *     ldp_last_error(), when
 *       3 + (count+1) + max_pixels/8192 + 1 + count*(max_side/64 + max_side/128 + 3)
 *     exceeds 2^21.  (4096 images of 640x490 fit with room to spare.)
 *     A batch that breaks its own bounds is clamped on the device and
 *     flagged in the device status word (bit 1).
 *   - the first call on each device looks up the array's address
 *     (cudaGetSymbolAddress) with that device current: make it before any
 *     stream capture.
 *   - every call shares the array, which keeps the last call's contents;
 *     each call rewrites what it reads first.  Calls that overlap on the GPU
 *     (other streams or host threads) race on it: serialise them.
 * EINVAL also for count < 0, NULL d_descs with count > 0, bad k or rs,
 * max_side outside [3, 1<<20]. */
LDP_API int ldp_batch_run_noalloc(const ldp_image_desc *d_descs, int count, uint64_t max_pixels,
                                  int max_side, int k, ldp_region_spec rs, uint32_t *d_hist,
                                  void *stream);

/* ---- helpers ---- */

/* Compact bins for k (Eq. 6): C(8,k), or -1 when k is outside [0,8]. */
LDP_API int ldp_hist_bins(int k);

/* Compact bin of an 8-bit code for k (its colex rank among the codes with
 * popcount k, i.e. its position in ascending code order), or -1. */
LDP_API int ldp_bin_of_code(int code, int k);

/* Message for the calling thread's most recent failing call ("" if none). */
LDP_API const char *ldp_last_error(void);

/* Reads and clears the device status word (bit 0: a batch descriptor was
 * rejected on the device; bit 1: a batch needed more tiles than its plan
 * holds; bit 2: a bounded wait for staged input gave up; bit 3: a crop
 * descriptor was rejected; bit 4, checked build: an index outside its
 * buffer was skipped).  Synchronises `stream`.  The checked build also
 * waits at the end of every batch and single-image run and returns
 * LDP_EINVAL for bit 1 and LDP_ETIMEOUT for bit 2 (without clearing them). */
LDP_API int ldp_device_status(void *stream, int *out);

/* ---- fault injection (tests of the error paths; the paper has no
 * counterpart) ----
 * Makes later calls fail on the host, the way a real failure would, so that
 * tests can check the error codes and the clean shutdown without faulting a
 * GPU.  After `after` more operations of the kind succeed, the next `count`
 * fail:
 *   LDP_FAULT_DEVICE_ALLOC: device allocations of batch plans and of the
 *     serving runtime fail as if the device were out of memory
 *     (ldp_batch_plan_create, ldp_batch_plan_set_config and
 *     ldp_server_create then return LDP_ENOMEM and free what they had);
 *   LDP_FAULT_SERVER_LAUNCH: serving batches fail to launch as if the launch
 *     had returned a CUDA error, without queueing any work: the runtime
 *     records the error, gives the batch's arena space back, later
 *     ldp_server_submit / ldp_server_poll calls return LDP_ECUDA and
 *     ldp_server_destroy still shuts down;
 *   LDP_FAULT_STAGE_WAIT (checked build only, LDP_ENOTIMPL otherwise; after
 *     must be 0): the staged tile variants stop filling input-stage group
 *     `count` of every tile (0 turns it off) and give up waiting for it
 *     after a few polls, with no copy in flight for that stage; the run sets
 *     bit 2 of the device status word and returns LDP_ETIMEOUT.
 *     Synchronises `stream`.
 * count = 0 clears pending faults of the kind.  EINVAL for an unknown kind
 * or a negative after / count. */
#define LDP_FAULT_DEVICE_ALLOC 0
#define LDP_FAULT_SERVER_LAUNCH 1
#define LDP_FAULT_STAGE_WAIT 2
LDP_API int ldp_test_inject_fault(int kind, int after, int count, void *stream);

/* Library version (major*10000 + minor*100 + patch). */
LDP_API int ldp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LDP_H */
