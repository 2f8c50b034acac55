// C-ABI of libldp (declared in include/ldp.h): argument validation, error
// reporting, single-image launches (codes and region histograms in every code
// mode), batch plans with CUDA-graph replay.  The entry points of sliding
// windows, crop-and-resize and distances sit beside their kernels
// (ldp_windows.cu, ldp_resize.cu, ldp_distance.cu).
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ldp_launch.h"

namespace {

thread_local std::string t_err;
std::atomic<int> g_plain_variant{-1};  // -1: chosen per image size

int check_regions(int R, int C) {
    if (R < 1 || C < 1) return ldp::report_error(LDP_EINVAL, "region grid must be at least 1x1");
    if ((int64_t)R * (int64_t)C > (1 << 22))
        return ldp::report_error(LDP_EINVAL, "region grid larger than 1<<22 regions");
    return LDP_OK;
}

// Tile variant of a single-image launch: an image of few 64-row tiles keeps
// most SMs idle and its latency is that of one tile, so smaller images take
// shorter warp tiles (more tiles in flight; 4-row tiles while the image has
// fewer 8-row tiles than the GPU has warp schedulers); large images keep
// 64-row tiles (less flush overhead per pixel).  The first non-staged
// variant of each height is used.
struct PlainChoice {
    int v4 = -1, v8 = 0, v16 = 0, sms = 132;
};

// the short-tile variants and the SM count, found once (thread-safe static)
const PlainChoice& plain_choice() {
    static const PlainChoice c = [] {
        PlainChoice r;
        bool f8 = false, f16 = false;
        for (int v = 0; v < ldp::num_variants(); ++v) {
            const char* name = ldp::variant_name(v);
            const int th = ldp::variant_tile_h(v);
            const bool staged = name[0] && name[strlen(name) - 1] == '1';
            if (!staged && th == 4 && r.v4 < 0) r.v4 = v;
            if (!staged && th == 8 && !f8) r.v8 = v, f8 = true;
            if (!staged && th == 16 && !f16) r.v16 = v, f16 = true;
        }
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            r.sms = sms;
        return r;
    }();
    return c;
}

int plain_variant(int H, int W) {
    const int fixed = g_plain_variant.load();
    if (fixed >= 0) return fixed;
    const PlainChoice& c = plain_choice();
    const long long tiles64 = (long long)((H - 2 + 63) / 64) * (long long)((W - 2 + 127) / 128);
    const long long tiles8 = (long long)((H - 2 + 7) / 8) * (long long)((W - 2 + 127) / 128);
    if (c.v4 >= 0 && tiles8 < 4LL * c.sms) return c.v4;  // fewer 8-row tiles than warp schedulers
    if (tiles64 < 2LL * c.sms) return c.v8;
    if (tiles64 < 8LL * c.sms) return c.v16;
    return 0;
}

}  // namespace

namespace ldp {

int report_error(int code, const char* msg) {
    t_err = msg;
    return code;
}

int report_cuda(cudaError_t e, const char* where) {
    t_err = std::string(where) + ": " + cudaGetErrorName(e) + ": " + cudaGetErrorString(e);
    return LDP_ECUDA;
}

int binom8(int r) {
    if (r < 0 || r > 8) return -1;
    int c = 1;
    for (int i = 1; i <= r; ++i) c = c * (8 - r + i) / i;
    return c;
}

int check_image(const void* img, int H, int W, int pitch) {
    if (!img) return report_error(LDP_EINVAL, "image pointer is NULL");
    if (H < 3 || W < 3) return report_error(LDP_EINVAL, "image must be at least 3x3");
    if (H > (1 << 20) || W > (1 << 20)) return report_error(LDP_EINVAL, "image side larger than 1<<20");
    if (pitch < W) return report_error(LDP_EINVAL, "pitch < W");
    return LDP_OK;
}

int check_codes(const void* codes, int W, int code_pitch, bool required) {
    if (!codes) return required ? report_error(LDP_EINVAL, "codes pointer is NULL") : LDP_OK;
    if (code_pitch < W - 2) return report_error(LDP_EINVAL, "code_pitch < W-2");
    return LDP_OK;
}

int run_plain(int mode, const uint8_t* img, int H, int W, int pitch, int k, int R, int C, int compact,
              uint32_t* hist, uint8_t* codes, int code_pitch, void* stream) {
    Range range("ldp.single_image");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    JobArgs jb{img, H, W, pitch, codes, code_pitch, hist, status_word()};
    HistArgs hc{R, C, 256, 0};
    if (hist) {
        const bool exact = mode == kLDP || mode == kLDPRaw;  // codes of exactly k bits
        hc.nbins = (exact && compact) ? binom8(k) : 256;
        hc.compact = (exact && compact) ? 1 : 0;
        const size_t bytes = (size_t)R * (size_t)C * (size_t)hc.nbins * sizeof(uint32_t);
        cudaError_t e = cudaMemsetAsync(hist, 0, bytes, s);
        if (e != cudaSuccess) return report_cuda(e, "zeroing the histogram");
    }
    cudaError_t e = launch_plain(mode, k, hist != nullptr, plain_variant(H, W), jb, hc, s);
    if (e != cudaSuccess) return report_cuda(e, "kernel launch");
#ifdef LDP_CHECKED
    // checked builds wait for the launch and report a bounded wait that gave up
    int st = 0;
    e = peek_status(s, &st);
    if (e != cudaSuccess) return report_cuda(e, "reading the device status");
    if (st & kStatusWaitTimeout) return report_error(LDP_ETIMEOUT, "a bounded wait for staged input gave up");
#endif
    return LDP_OK;
}

}  // namespace ldp

using ldp::binom8;
using ldp::check_codes;
using ldp::check_image;
using ldp::run_plain;

namespace {
int fail(int code, const char* msg) { return ldp::report_error(code, msg); }
int cuda_fail(cudaError_t e, const char* where) { return ldp::report_cuda(e, where); }
}  // namespace

struct ldp_batch_plan {
    int mode = 0, k = 3;
    ldp_region_spec rs{1, 1, 0};
    unsigned flags = 0;
    int max_images = 0, max_tiles = 0;
    int cap_th = 0;  // tile height the work list is sized for
    uint64_t max_pixels = 0;
    int variant = 0, ctas_per_sm = 0;
    int device = 0, num_sms = 0;
    void* scratch = nullptr;
    ldp::BatchScratch scr{};
    cudaStream_t cap_stream = nullptr;
    // graph cache
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;  // kept alive: its event-record nodes address the exec's nodes
    const void *g_descs = nullptr, *g_count = nullptr, *g_hist = nullptr;
    int g_variant = -1, g_grid = 0;
    // timing: event-record nodes around the persistent kernel
    cudaEvent_t ph_start = nullptr, ph_end = nullptr;  // events the graph was captured with
    cudaGraphNode_t node_start = nullptr, node_end = nullptr;
    std::vector<cudaEvent_t> ev_start, ev_end;
    int nrec = 0;
};

namespace {

// Upper bound on the warp tiles (TH rows x 128 columns) of any batch of at
// most n images holding at most P pixels.  An H x W image (H, W >= 3) has
// ceil(h/TH) * ceil(w/128) tiles, h = H-2, w = W-2, at most
// (h + TH-1)(w + 127) / (128 TH) = (hw + 127 h + (TH-1) w + 127 (TH-1)) / (128 TH);
// with hw <= HW and h, w <= HW/3 (the other side is at least 3) that is
// below HW (TH + 129) / (384 TH) + 1.  Summed over the images:
double tile_capacity(uint64_t P, int n, int TH) {
    return (double)P * (double)(TH + 129) / (384.0 * (double)TH) + (double)n + 1.0;
}

// (Re)allocates the plan's work list (counter, total, prefix, tile map) for
// tiles of TH rows.  On failure the plan keeps its previous work list.  The
// old list may be in use by queued work and by the captured graph: the
// device is synchronised and the graph dropped before it is freed.
int plan_size_work_list(ldp_batch_plan* p, int TH) {
    const double bound = tile_capacity(p->max_pixels, p->max_images, TH);
    if (bound > 1.5e9) return fail(LDP_EINVAL, "max_pixels too large for a plan of this tile height");
    const int max_tiles = (int)bound;
    const size_t n_ints = (size_t)(p->max_images + 1) + (size_t)max_tiles + 2;
    void* mem = nullptr;
    cudaError_t e = ldp::device_malloc(&mem, n_ints * sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LDP_ENOMEM, "device allocation of the plan's work list failed");
    }
    if (p->scratch) {
        cudaDeviceSynchronize();
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        p->exec = nullptr;
        p->graph = nullptr;
        cudaFree(p->scratch);
    }
    p->scratch = mem;
    p->max_tiles = max_tiles;
    p->cap_th = TH;
    int* base = static_cast<int*>(mem);
    p->scr.counter = base;
    p->scr.total = base + 1;
    p->scr.prefix = base + 2;
    p->scr.tile_img = base + 2 + (p->max_images + 1);
    return LDP_OK;
}

}  // namespace

extern "C" {

int ldp_version(void) { return 100; }

const char* ldp_last_error(void) { return t_err.c_str(); }

int ldp_hist_bins(int k) { return binom8(k); }

int ldp_bin_of_code(int code, int k) {
    if (code < 0 || code > 255 || k < 0 || k > 8) return -1;
    if (__builtin_popcount((unsigned)code) != k) return -1;
    // colex rank: sum over set bits b_1 < ... < b_k of C(b_j, j)
    int r = 0, j = 0;
    for (int b = 0; b < 8; ++b)
        if (code >> b & 1) {
            ++j;
            int c = 1;
            for (int i = 1; i <= j; ++i) c = c * (b - j + i) / i;
            r += (j <= b) ? c : 0;
        }
    return r;
}

int ldp_num_variants(void) { return ldp::num_variants(); }

const char* ldp_variant_name(int variant) { return ldp::variant_name(variant); }

int ldp_set_plain_variant(int variant) {
    if (variant < -1 || variant >= ldp::num_variants()) return fail(LDP_EINVAL, "variant out of range");
    g_plain_variant.store(variant);
    return LDP_OK;
}

int ldp_codes(const uint8_t* d_img, int H, int W, int pitch, int k, uint8_t* d_codes, int code_pitch,
              void* stream) {
    int rc;
    if ((rc = check_image(d_img, H, W, pitch))) return rc;
    if ((rc = check_codes(d_codes, W, code_pitch, true))) return rc;
    if (k < 1 || k > 7) return fail(LDP_EINVAL, "k must be in [1,7]");
    return run_plain(0, d_img, H, W, pitch, k, 1, 1, 0, nullptr, d_codes, code_pitch, stream);
}

int ldp_region_hist(const uint8_t* d_img, int H, int W, int pitch, int k, ldp_region_spec rs,
                    uint32_t* d_hist, uint8_t* d_codes_or_null, int code_pitch, void* stream) {
    int rc;
    if ((rc = check_image(d_img, H, W, pitch))) return rc;
    if ((rc = check_codes(d_codes_or_null, W, code_pitch, false))) return rc;
    if (k < 1 || k > 7) return fail(LDP_EINVAL, "k must be in [1,7]");
    if ((rc = check_regions(rs.R, rs.C))) return rc;
    if (rs.compact != 0 && rs.compact != 1) return fail(LDP_EINVAL, "compact must be 0 or 1");
    if (!d_hist) return fail(LDP_EINVAL, "histogram pointer is NULL");
    return run_plain(0, d_img, H, W, pitch, k, rs.R, rs.C, rs.compact, d_hist, d_codes_or_null, code_pitch,
                     stream);
}

int lbp_codes(const uint8_t* d_img, int H, int W, int pitch, uint8_t* d_codes, int code_pitch, void* stream) {
    int rc;
    if ((rc = check_image(d_img, H, W, pitch))) return rc;
    if ((rc = check_codes(d_codes, W, code_pitch, true))) return rc;
    return run_plain(1, d_img, H, W, pitch, 1, 1, 1, 0, nullptr, d_codes, code_pitch, stream);
}

int lbp_region_hist(const uint8_t* d_img, int H, int W, int pitch, int R, int C, uint32_t* d_hist,
                    uint8_t* d_codes_or_null, int code_pitch, void* stream) {
    int rc;
    if ((rc = check_image(d_img, H, W, pitch))) return rc;
    if ((rc = check_codes(d_codes_or_null, W, code_pitch, false))) return rc;
    if ((rc = check_regions(R, C))) return rc;
    if (!d_hist) return fail(LDP_EINVAL, "histogram pointer is NULL");
    return run_plain(1, d_img, H, W, pitch, 1, R, C, 0, d_hist, d_codes_or_null, code_pitch, stream);
}

namespace {
// LDP_CODE_* -> kernel mode
int code_mode_kernel(int code_mode) {
    switch (code_mode) {
        case LDP_CODE_ABS: return ldp::kLDP;
        case LDP_CODE_RAW: return ldp::kLDPRaw;
        case LDP_CODE_ABS_THRESH: return ldp::kLDPThresh;
        case LDP_CODE_RAW_THRESH: return ldp::kLDPRawThresh;
        default: return -1;
    }
}
}  // namespace

int ldp_codes_ex(const uint8_t* d_img, int H, int W, int pitch, int k, int code_mode, uint8_t* d_codes,
                 int code_pitch, void* stream) {
    int rc;
    if ((rc = check_image(d_img, H, W, pitch))) return rc;
    if ((rc = check_codes(d_codes, W, code_pitch, true))) return rc;
    if (k < 1 || k > 7) return fail(LDP_EINVAL, "k must be in [1,7]");
    const int mode = code_mode_kernel(code_mode);
    if (mode < 0) return fail(LDP_EINVAL, "code_mode must be one of LDP_CODE_*");
    return run_plain(mode, d_img, H, W, pitch, k, 1, 1, 0, nullptr, d_codes, code_pitch, stream);
}

int ldp_region_hist_ex(const uint8_t* d_img, int H, int W, int pitch, int k, int code_mode, ldp_region_spec rs,
                       uint32_t* d_hist, uint8_t* d_codes_or_null, int code_pitch, void* stream) {
    int rc;
    if ((rc = check_image(d_img, H, W, pitch))) return rc;
    if ((rc = check_codes(d_codes_or_null, W, code_pitch, false))) return rc;
    if (k < 1 || k > 7) return fail(LDP_EINVAL, "k must be in [1,7]");
    const int mode = code_mode_kernel(code_mode);
    if (mode < 0) return fail(LDP_EINVAL, "code_mode must be one of LDP_CODE_*");
    if ((rc = check_regions(rs.R, rs.C))) return rc;
    if (rs.compact != 0 && rs.compact != 1) return fail(LDP_EINVAL, "compact must be 0 or 1");
    if (rs.compact && (mode == ldp::kLDPThresh || mode == ldp::kLDPRawThresh))
        return fail(LDP_EINVAL, "threshold code modes count 256 raw bins (compact = 0)");
    if (!d_hist) return fail(LDP_EINVAL, "histogram pointer is NULL");
    return run_plain(mode, d_img, H, W, pitch, k, rs.R, rs.C, rs.compact, d_hist, d_codes_or_null, code_pitch,
                     stream);
}

int ldp_batch_plan_create(ldp_batch_plan** out, int max_images, uint64_t max_pixels, int k, ldp_region_spec rs,
                          unsigned flags) {
    if (!out) return fail(LDP_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_images < 1 || max_images > (1 << 24)) return fail(LDP_EINVAL, "max_images must be in [1, 1<<24]");
    if (max_pixels < 9) return fail(LDP_EINVAL, "max_pixels must be at least 9");
    const int cmode = (int)((flags >> 2) & 3u);
    if ((flags & LDP_PLAN_LBP) && cmode) return fail(LDP_EINVAL, "code modes apply to LDP plans only");
    const int mode = (flags & LDP_PLAN_LBP) ? 1 : code_mode_kernel(cmode);
    if (mode != 1 && (k < 1 || k > 7)) return fail(LDP_EINVAL, "k must be in [1,7]");
    int rc;
    if ((rc = check_regions(rs.R, rs.C))) return rc;
    if (rs.compact != 0 && rs.compact != 1) return fail(LDP_EINVAL, "compact must be 0 or 1");
    if (rs.compact && (mode == ldp::kLDPThresh || mode == ldp::kLDPRawThresh))
        return fail(LDP_EINVAL, "threshold code modes count 256 raw bins (compact = 0)");
    const int th0 = ldp::variant_tile_h(0);
    if (tile_capacity(max_pixels, max_images, th0) > 1.5e9) return fail(LDP_EINVAL, "max_pixels too large for one plan");
    ldp_batch_plan* p = new (std::nothrow) ldp_batch_plan();
    if (!p) return fail(LDP_ENOMEM, "host allocation failed");
    p->mode = mode;
    p->k = mode != 1 ? k : 1;
    p->rs = rs;
    if (mode == 1) p->rs.compact = 0;
    p->flags = flags;
    p->max_images = max_images;
    p->max_pixels = max_pixels;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "querying the device");
    }
    if ((rc = plan_size_work_list(p, th0)) != LDP_OK) {
        delete p;
        return rc;
    }
    *out = p;
    return LDP_OK;
}

int ldp_batch_plan_set_config(ldp_batch_plan* plan, int variant, int ctas_per_sm) {
    if (!plan) return fail(LDP_EINVAL, "plan is NULL");
    if (variant < 0 || variant >= ldp::num_variants()) return fail(LDP_EINVAL, "variant out of range");
    if (ctas_per_sm < 0 || ctas_per_sm > 64) return fail(LDP_EINVAL, "ctas_per_sm out of range");
    // a variant of shorter tiles than the work list was sized for needs a
    // larger one (code-mode plans always run the tile shape of kCodeModeVariant)
    const int th = ldp::variant_tile_h(plan->mode >= 2 ? ldp::kCodeModeVariant : variant);
    if (th < plan->cap_th) {
        const int rc = plan_size_work_list(plan, th);
        if (rc != LDP_OK) return rc;  // the plan keeps its previous configuration
    }
    plan->variant = variant;
    plan->ctas_per_sm = ctas_per_sm;
    return LDP_OK;
}

static int batch_launch(ldp_batch_plan* plan, int mode, const ldp_image_desc* d_descs, const int* d_count,
                        uint32_t* d_hist, void* stream) {
    ldp::Range range("ldp.batch_run");
    if (!plan) return fail(LDP_EINVAL, "plan is NULL");
    if ((plan->mode == 1) != (mode == 1))
        return fail(LDP_EINVAL, "plan was created for the other descriptor (LDP vs LBP)");
    mode = plan->mode;  // LDP plans carry their code mode
    // the code-mode kernels have one tile shape (the one of kCodeModeVariant)
    const int variant = mode >= 2 ? ldp::kCodeModeVariant : plan->variant;
    if (!d_descs || !d_count) return fail(LDP_EINVAL, "descriptor or count pointer is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ldp::BatchArgs a{};
    a.descs = d_descs;
    a.count = d_count;
    a.hist = d_hist;
    a.max_images = plan->max_images;
    a.max_tiles = plan->max_tiles;
    a.scr = plan->scr;
    a.hc.R = plan->rs.R;
    a.hc.C = plan->rs.C;
    a.hc.compact = ((mode == ldp::kLDP || mode == ldp::kLDPRaw) && plan->rs.compact) ? 1 : 0;
    a.hc.nbins = a.hc.compact ? binom8(plan->k) : 256;
    a.status = ldp::status_word();
    if (!a.status) return fail(LDP_ECUDA, "device status word not found");
    int occ = 0;
    cudaError_t e = ldp::batch_occupancy(mode, plan->k, d_hist != nullptr, variant, &occ);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (occ < 1) return fail(LDP_ENOTIMPL, "persistent kernel does not fit on an SM");
    const int per_sm = plan->ctas_per_sm > 0 ? (plan->ctas_per_sm < occ ? plan->ctas_per_sm : occ) : occ;
    const int grid = plan->num_sms * per_sm;
    const bool hist = d_hist != nullptr;
    const bool timed = plan->nrec < (int)plan->ev_start.size();
    if (!plan->ph_start) {
        e = cudaEventCreate(&plan->ph_start);
        if (e == cudaSuccess) e = cudaEventCreate(&plan->ph_end);
        if (e != cudaSuccess) return cuda_fail(e, "creating timing events");
    }
    if (plan->flags & LDP_PLAN_NO_GRAPH) {
        e = ldp::launch_batch_prep(variant, a, s);
        if (e != cudaSuccess) return cuda_fail(e, "batch preparation launch");
        if (timed) cudaEventRecord(plan->ev_start[plan->nrec], s);
        e = ldp::launch_batch_main(mode, plan->k, hist, variant, grid, a, s);
        if (e != cudaSuccess) return cuda_fail(e, "persistent kernel launch");
        if (timed) {
            e = cudaEventRecord(plan->ev_end[plan->nrec], s);
            if (e != cudaSuccess) return cuda_fail(e, "recording a timing event");
            ++plan->nrec;
        }
        return LDP_OK;
    }
    if (!plan->exec || plan->g_descs != d_descs || plan->g_count != d_count || plan->g_hist != d_hist ||
        plan->g_variant != variant || plan->g_grid != grid) {
        if (plan->exec) {
            cudaGraphExecDestroy(plan->exec);
            plan->exec = nullptr;
        }
        if (plan->graph) {
            cudaGraphDestroy(plan->graph);
            plan->graph = nullptr;
        }
        if (!plan->cap_stream) {
            e = cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "creating the capture stream");
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "beginning graph capture");
        cudaError_t e1 = ldp::launch_batch_prep(variant, a, plan->cap_stream);
        // external event records become event-record nodes of the captured graph
        if (e1 == cudaSuccess) e1 = cudaEventRecordWithFlags(plan->ph_start, plan->cap_stream, cudaEventRecordExternal);
        cudaError_t e2 = e1 == cudaSuccess
                             ? ldp::launch_batch_main(mode, plan->k, hist, variant, grid, a, plan->cap_stream)
                             : e1;
        if (e2 == cudaSuccess) e2 = cudaEventRecordWithFlags(plan->ph_end, plan->cap_stream, cudaEventRecordExternal);
        e = cudaStreamEndCapture(plan->cap_stream, &g);
        if (e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(e2, "capturing the batch launches");
        }
        if (e != cudaSuccess) return cuda_fail(e, "ending graph capture");
        // find the two event-record nodes (start / end of the persistent kernel)
        plan->node_start = plan->node_end = nullptr;
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev = nullptr;
            cudaGraphEventRecordNodeGetEvent(nd, &ev);
            if (ev == plan->ph_start) plan->node_start = nd;
            if (ev == plan->ph_end) plan->node_end = nd;
        }
        e = cudaGraphInstantiate(&plan->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            plan->exec = nullptr;
            return cuda_fail(e, "instantiating the batch graph");
        }
        plan->graph = g;
        if (!plan->node_start || !plan->node_end) return fail(LDP_ECUDA, "timing nodes missing from the graph");
        plan->g_descs = d_descs;
        plan->g_count = d_count;
        plan->g_hist = d_hist;
        plan->g_variant = variant;
        plan->g_grid = grid;
    }
    cudaEvent_t es = timed ? plan->ev_start[plan->nrec] : plan->ph_start;
    cudaEvent_t ee = timed ? plan->ev_end[plan->nrec] : plan->ph_end;
    e = cudaGraphExecEventRecordNodeSetEvent(plan->exec, plan->node_start, es);
    if (e == cudaSuccess) e = cudaGraphExecEventRecordNodeSetEvent(plan->exec, plan->node_end, ee);
    if (e != cudaSuccess) return cuda_fail(e, "setting the graph's timing events");
    e = cudaGraphLaunch(plan->exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    if (timed) ++plan->nrec;
    return LDP_OK;
}

// Checked builds wait for the work just queued on `stream` and turn the
// status bits a caller can cause into errors: a batch with more tiles than
// its work list holds (its descriptors exceed the plan's max_pixels) and a
// bounded wait that gave up.  Release builds stay asynchronous; the bits
// are read with ldp_device_status.
static int checked_status(void* stream) {
#ifdef LDP_CHECKED
    int st = 0;
    const cudaError_t e = ldp::peek_status(static_cast<cudaStream_t>(stream), &st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device status");
    if (st & ldp::kStatusTooManyTiles)
        return fail(LDP_EINVAL, "the batch needed more tiles than the plan holds (pixels beyond max_pixels)");
    if (st & ldp::kStatusWaitTimeout) return fail(LDP_ETIMEOUT, "a bounded wait for staged input gave up");
#else
    (void)stream;
#endif
    return LDP_OK;
}

static int batch_run(ldp_batch_plan* plan, int mode, const ldp_image_desc* d_descs, const int* d_count,
                     uint32_t* d_hist, void* stream) {
    const int rc = batch_launch(plan, mode, d_descs, d_count, d_hist, stream);
    return rc != LDP_OK ? rc : checked_status(stream);
}

int ldp_batch_plan_enable_timing(ldp_batch_plan* plan, int capacity) {
    if (!plan) return fail(LDP_EINVAL, "plan is NULL");
    if (capacity < 0 || capacity > (1 << 20)) return fail(LDP_EINVAL, "capacity out of range");
    while ((int)plan->ev_start.size() < capacity) {
        cudaEvent_t a = nullptr, b = nullptr;
        cudaError_t e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        if (e != cudaSuccess) {
            if (a) cudaEventDestroy(a);
            return cuda_fail(e, "creating timing events");
        }
        plan->ev_start.push_back(a);
        plan->ev_end.push_back(b);
    }
    plan->nrec = 0;
    return LDP_OK;
}

int ldp_batch_plan_kernel_times(ldp_batch_plan* plan, float* ms, int capacity, int* count) {
    if (!plan || !count || (capacity > 0 && !ms)) return fail(LDP_EINVAL, "NULL argument");
    const int n = plan->nrec < capacity ? plan->nrec : capacity;
    for (int i = 0; i < n; ++i) {
        cudaError_t e = cudaEventSynchronize(plan->ev_end[i]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[i], plan->ev_start[i], plan->ev_end[i]);
        if (e != cudaSuccess) return cuda_fail(e, "reading timing events");
    }
    *count = n;
    plan->nrec = 0;
    return LDP_OK;
}

int ldp_batch_run(ldp_batch_plan* plan, const ldp_image_desc* d_descs, const int* d_count, uint32_t* d_hist,
                  void* stream) {
    return batch_run(plan, 0, d_descs, d_count, d_hist, stream);
}

int lbp_batch_run(ldp_batch_plan* plan, const ldp_image_desc* d_descs, const int* d_count, uint32_t* d_hist,
                  void* stream) {
    return batch_run(plan, 1, d_descs, d_count, d_hist, stream);
}

int ldp_batch_plan_destroy(ldp_batch_plan* plan) {
    if (!plan) return LDP_OK;
    cudaDeviceSynchronize();
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
    for (cudaEvent_t ev : plan->ev_start) cudaEventDestroy(ev);
    for (cudaEvent_t ev : plan->ev_end) cudaEventDestroy(ev);
    if (plan->ph_start) cudaEventDestroy(plan->ph_start);
    if (plan->ph_end) cudaEventDestroy(plan->ph_end);
    if (plan->scratch) cudaFree(plan->scratch);
    delete plan;
    return LDP_OK;
}

int ldp_test_inject_fault(int kind, int after, int count, void* stream) {
    if (count < 0 || after < 0) return fail(LDP_EINVAL, "after and count must be >= 0");
    switch (kind) {
        case LDP_FAULT_DEVICE_ALLOC:
        case LDP_FAULT_SERVER_LAUNCH: ldp::set_faults(kind, after, count); return LDP_OK;
        case LDP_FAULT_STAGE_WAIT: {
            if (after != 0) return fail(LDP_EINVAL, "the stage-wait fault takes after = 0");
#ifdef LDP_CHECKED
            const cudaError_t e = ldp::set_wait_fault(count, static_cast<cudaStream_t>(stream));
            if (e != cudaSuccess) return cuda_fail(e, "setting the stage-wait fault");
            return LDP_OK;
#else
            (void)stream;
            return fail(LDP_ENOTIMPL, "the stage-wait fault exists in the checked build only");
#endif
        }
        default: return fail(LDP_EINVAL, "unknown fault kind");
    }
}

int ldp_device_status(void* stream, int* out) {
    if (!out) return fail(LDP_EINVAL, "out is NULL");
    cudaError_t e = ldp::read_clear_status(static_cast<cudaStream_t>(stream), out);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device status");
    return LDP_OK;
}

}  // extern "C"
