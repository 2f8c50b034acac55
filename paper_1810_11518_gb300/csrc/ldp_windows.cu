// Sliding-window code histograms (Sec. 3.2): windows of wh x ww pixels at
// stride (sh, sw) over the image, window (a, b) covering image rows
// [a*sh, min(a*sh + wh, H)) and columns [b*sw, min(b*sw + ww, W)), interior
// pixels only.  Every window is a union of cells of the grid with cell size
// (gcd(wh, sh), gcd(ww, sw)), so the work is
//   k_cell_hist:   one pass over the code map; a CTA owns a row of cells (a
//                  chunk of it for wide images) -- or, when all of an
//                  image's cells fit in shared memory, the whole image
//                  (k_cell_hist_image) -- and counts its codes there, four
//                  codes per lane and load, then stores the cells'
//                  histograms (no global atomics: every cell belongs to
//                  exactly one CTA);
//   k_window_sum:  each window histogram is the sum of its cells' (skipped
//                  when stride = size: the cells are the windows).
// Images come from ldp_image_desc records (batches) or one record passed by
// value (single image).
#include <cuda_runtime.h>

#include <cstdint>

#include "ldp_device.cuh"
#include "ldp_launch.h"

namespace ldp {

namespace {

constexpr int kCellThreads = 256;
constexpr int kCellSmemWords = 12160;  // counters at most: with the 512-byte table, 48 KB of shared memory

struct CellArgs {
    const ldp_image_desc* descs;  // nullptr: the single image `one`
    ldp_image_desc one;
    int ch, cw;        // cell size in pixels
    int nbins, k;      // k >= 1 with compact bins: C(8,k) bins; else 256 raw bins
    int chunk;         // cells per CTA along a row
    int direct;        // 1: cells are the windows, stored at hist + hist_offset
    uint32_t* hist;    // window histograms (direct) ...
    uint32_t* cells;   // ... or cell histograms, image i at cells + i * cell_stride
    uint64_t cell_stride;
};

__device__ __forceinline__ ldp_image_desc desc_of(const CellArgs& a, int i) {
    return a.descs ? a.descs[i] : a.one;
}

// Cell of column y: y / cw, from a float estimate corrected by one step
// either way (exact for y < 2^21; image sides are at most 2^20).
__device__ __forceinline__ int cell_of(int y, int cw, float inv_cw) {
    int q = (int)((float)y * inv_cw);
    if (q * cw > y) --q;
    if ((q + 1) * cw <= y) ++q;
    return q;
}

// CTA work item p = (image, cell row) pairs, strided over the grid; the
// grid's y index picks the chunk of cells along the row.  Warps take the
// item's rows, lanes four consecutive columns (one 32-bit load of codes when
// the row is 4-byte aligned), blocks of 128 columns at a time; the four
// columns' cells are found once per block and reused for every row.
__global__ void __launch_bounds__(kCellThreads) k_cell_hist(CellArgs a, int count, int ncr_max) {
    extern __shared__ uint32_t cnt[];  // a.chunk * a.nbins counters (sized at launch)
    __shared__ int16_t lut[256];
    for (int c = threadIdx.x; c < 256; c += blockDim.x)
        lut[c] = (a.k >= 1) ? __ldg(&g_bin_table.bin[a.k][c]) : (int16_t)c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const float inv_cw = 1.0f / (float)a.cw;
    const uint64_t pairs = (uint64_t)count * (uint64_t)ncr_max;
    for (uint64_t p = blockIdx.x; p < pairs; p += gridDim.x) {
        const int img = (int)(p / (uint64_t)ncr_max), i = (int)(p % (uint64_t)ncr_max);
        const ldp_image_desc d = desc_of(a, img);
        const int H = d.H, W = d.W;
        const int ncr = (H + a.ch - 1) / a.ch, ncc = (W + a.cw - 1) / a.cw;
        const int j0 = blockIdx.y * a.chunk;
        if (i >= ncr || j0 >= ncc || d.codes == nullptr) continue;  // uniform over the CTA
        const int j1 = min(j0 + a.chunk, ncc);
        const int words = (j1 - j0) * a.nbins;
        __syncthreads();  // lut ready; the previous item's counters are stored
        for (int e = threadIdx.x; e < words; e += blockDim.x) cnt[e] = 0;
        __syncthreads();
        // interior pixels of cell row i, cells j0..j1-1 (code (x, y) at codes[(x-1)*Pc + y-1])
        const int x0 = max(i * a.ch, 1), x1 = min((i + 1) * a.ch, H - 1);
        const int y0 = max(j0 * a.cw, 1), y1 = min(j1 * a.cw, W - 1);
        const bool al = (((uintptr_t)d.codes | (uintptr_t)d.code_pitch) & 3u) == 0;
        for (int yb = y0; yb < y1; yb += 128) {
            // this lane's four columns: yq .. yq+3 (code columns yq-1 .. yq+2)
            const int yq = yb + 4 * lane;
            int off[4];
            bool in[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                in[t] = yq + t < y1;
                off[t] = in[t] ? (cell_of(yq + t, a.cw, inv_cw) - j0) * a.nbins : 0;
            }
            const bool vec = al && in[3] && ((yq - 1) & 3) == 0;
#pragma unroll 4
            for (int x = x0 + warp; x < x1; x += nwarps) {
                const uint8_t* cp = d.codes + (size_t)(x - 1) * (size_t)d.code_pitch + (yq - 1);
                uint32_t w4 = 0;
                if (vec) {
                    w4 = __ldg(reinterpret_cast<const unsigned int*>(cp));
                } else {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (in[t]) w4 |= (uint32_t)__ldg(cp + t) << (8 * t);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int b = lut[(w4 >> (8 * t)) & 0xFFu];
                    if (in[t] && b >= 0) atomicAdd(&cnt[off[t] + b], 1u);
                }
            }
        }
        __syncthreads();
        uint32_t* out = a.direct ? a.hist + d.hist_offset : a.cells + (uint64_t)img * a.cell_stride;
        out += ((size_t)i * (size_t)ncc + (size_t)j0) * (size_t)a.nbins;
        for (int e = threadIdx.x; e < words; e += blockDim.x) out[e] = cnt[e];
    }
}

// Whole-image items, for images whose every cell fits in shared memory (the
// face-sized crops): one CTA per image, counters zeroed and stored once,
// warps over rows, lanes over four consecutive columns whose cells are found
// once for all rows.
__global__ void __launch_bounds__(kCellThreads) k_cell_hist_image(CellArgs a, int count) {
    extern __shared__ uint32_t cnt[];  // ncr * ncc * nbins counters of the largest image
    __shared__ int16_t lut[256];
    for (int c = threadIdx.x; c < 256; c += blockDim.x)
        lut[c] = (a.k >= 1) ? __ldg(&g_bin_table.bin[a.k][c]) : (int16_t)c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const float inv_cw = 1.0f / (float)a.cw, inv_ch = 1.0f / (float)a.ch;
    for (int img = blockIdx.x; img < count; img += gridDim.x) {
        const ldp_image_desc d = desc_of(a, img);
        if (d.codes == nullptr) continue;  // uniform over the CTA
        const int H = d.H, W = d.W;
        const int ncc = (W + a.cw - 1) / a.cw;
        const int words = ((H + a.ch - 1) / a.ch) * ncc * a.nbins;
        __syncthreads();  // lut ready; the previous image's counters are stored
        for (int e = threadIdx.x; e < words; e += blockDim.x) cnt[e] = 0;
        __syncthreads();
        const bool al = (((uintptr_t)d.codes | (uintptr_t)d.code_pitch) & 3u) == 0;
        for (int yb = 1; yb < W - 1; yb += 128) {
            const int yq = yb + 4 * lane;  // columns yq .. yq+3 (code columns yq-1 .. yq+2)
            int off[4];
            bool in[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                in[t] = yq + t < W - 1;
                off[t] = in[t] ? cell_of(yq + t, a.cw, inv_cw) * a.nbins : 0;
            }
            const bool vec = al && in[3];  // yq - 1 is a multiple of 4
#pragma unroll 4
            for (int x = 1 + warp; x < H - 1; x += nwarps) {
                const int rbase = cell_of(x, a.ch, inv_ch) * ncc * a.nbins;
                const uint8_t* cp = d.codes + (size_t)(x - 1) * (size_t)d.code_pitch + (yq - 1);
                uint32_t w4 = 0;
                if (vec) {
                    w4 = __ldg(reinterpret_cast<const unsigned int*>(cp));
                } else {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (in[t]) w4 |= (uint32_t)__ldg(cp + t) << (8 * t);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int b = lut[(w4 >> (8 * t)) & 0xFFu];
                    if (in[t] && b >= 0) atomicAdd(&cnt[rbase + off[t] + b], 1u);
                }
            }
        }
        __syncthreads();
        uint32_t* out = a.direct ? a.hist + d.hist_offset : a.cells + (uint64_t)img * a.cell_stride;
        for (int e = threadIdx.x; e < words; e += blockDim.x) out[e] = cnt[e];
    }
}

struct SumArgs {
    const ldp_image_desc* descs;
    ldp_image_desc one;
    int ch, cw, wh_c, ww_c, sh_c, sw_c;  // window size and stride in cells
    int wh, ww, sh, sw;                  // in pixels (window counts)
    int nbins;
    const uint32_t* cells;
    uint64_t cell_stride;
    uint32_t* hist;
};

__device__ __forceinline__ int win_count(int n, int w, int s) { return n <= w ? 1 : (n - w + s - 1) / s + 1; }

// One CTA per (window row, image) item, strided over the grid: warps take
// the row's windows, lanes the bins (consecutive bins: coalesced loads and
// stores, no division in the loop).
__global__ void __launch_bounds__(256) k_window_sum(SumArgs a, int count, int nwr_max) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint64_t items = (uint64_t)count * (uint64_t)nwr_max;
    for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int img = (int)(it / (uint64_t)nwr_max), wa = (int)(it % (uint64_t)nwr_max);
        const ldp_image_desc d = a.descs ? a.descs[img] : a.one;
        const int H = d.H, W = d.W;
        const int nwr = win_count(H, a.wh, a.sh);
        if (wa >= nwr) continue;
        const int ncr = (H + a.ch - 1) / a.ch, ncc = (W + a.cw - 1) / a.cw;
        const int nwc = win_count(W, a.ww, a.sw);
        const uint32_t* cells = a.cells + (uint64_t)img * a.cell_stride;
        uint32_t* out = a.hist + d.hist_offset + (uint64_t)wa * (uint64_t)nwc * (uint64_t)a.nbins;
        const int i0 = wa * a.sh_c, i1 = min(i0 + a.wh_c, ncr);
        for (int wb = warp; wb < nwc; wb += nwarps) {
            const int j0 = wb * a.sw_c, j1 = min(j0 + a.ww_c, ncc);
            for (int bin = lane; bin < a.nbins; bin += 32) {
                uint32_t s = 0;
                for (int ci = i0; ci < i1; ++ci) {
                    const uint32_t* row = cells + ((size_t)ci * (size_t)ncc) * (size_t)a.nbins + bin;
                    for (int cj = j0; cj < j1; ++cj) s += __ldg(row + (size_t)cj * (size_t)a.nbins);
                }
                out[(size_t)wb * (size_t)a.nbins + bin] = s;
            }
        }
    }
}

int gcd_int(int a, int b) {
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace

uint64_t window_cell_words(int H, int W, const WindowGeom& g) {
    const int ch = gcd_int(g.wh, g.sh), cw = gcd_int(g.ww, g.sw);
    return (uint64_t)((H + ch - 1) / ch) * (uint64_t)((W + cw - 1) / cw) * (uint64_t)g.nbins;
}

bool window_direct(const WindowGeom& g) { return g.wh == g.sh && g.ww == g.sw; }

cudaError_t launch_windows(const ldp_image_desc* d_descs, const ldp_image_desc* one, int count, int max_H,
                           int max_W, const WindowGeom& g, uint32_t* hist, uint32_t* cells,
                           uint64_t cell_stride, cudaStream_t s) {
    const int ch = gcd_int(g.wh, g.sh), cw = gcd_int(g.ww, g.sw);
    const bool direct = window_direct(g);
    CellArgs ca{};
    ca.descs = d_descs;
    if (one) ca.one = *one;
    ca.ch = ch;
    ca.cw = cw;
    ca.nbins = g.nbins;
    ca.k = g.compact ? g.k : 0;
    const int ncc_max = (max_W + cw - 1) / cw;
    ca.chunk = kCellSmemWords / g.nbins;
    if (ca.chunk > ncc_max) ca.chunk = ncc_max;  // shared memory sized to what a row of cells needs
    ca.direct = direct ? 1 : 0;
    ca.hist = hist;
    ca.cells = cells;
    ca.cell_stride = cell_stride;
    const int ncr = (max_H + ch - 1) / ch;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t image_words = (uint64_t)ncr * (uint64_t)ncc_max * (uint64_t)g.nbins;
    if (image_words <= (uint64_t)kCellSmemWords) {
        // every cell of an image fits: one CTA per image
        const unsigned grid = (unsigned)(count < sms * 16 ? count : sms * 16);
        k_cell_hist_image<<<grid, kCellThreads, sizeof(uint32_t) * (size_t)image_words, s>>>(ca, count);
    } else {
        // CTAs loop over (image, cell row) items: a few waves of the GPU
        const uint64_t pairs = (uint64_t)count * (uint64_t)ncr;
        const uint64_t cap = (uint64_t)sms * 32;
        dim3 grid((unsigned)(pairs < cap ? pairs : cap), (ncc_max + ca.chunk - 1) / ca.chunk);
        k_cell_hist<<<grid, kCellThreads, sizeof(uint32_t) * (size_t)ca.chunk * (size_t)g.nbins, s>>>(ca, count,
                                                                                                    ncr);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || direct) return e;
    SumArgs sa{};
    sa.descs = d_descs;
    if (one) sa.one = *one;
    sa.ch = ch;
    sa.cw = cw;
    sa.wh_c = g.wh / ch;
    sa.ww_c = g.ww / cw;
    sa.sh_c = g.sh / ch;
    sa.sw_c = g.sw / cw;
    sa.wh = g.wh;
    sa.ww = g.ww;
    sa.sh = g.sh;
    sa.sw = g.sw;
    sa.nbins = g.nbins;
    sa.cells = cells;
    sa.cell_stride = cell_stride;
    sa.hist = hist;
    const int nwr_max = (max_H <= g.wh) ? 1 : (max_H - g.wh + g.sh - 1) / g.sh + 1;
    const uint64_t items = (uint64_t)count * (uint64_t)nwr_max;
    k_window_sum<<<(unsigned)(items < (1u << 20) ? items : (1u << 20)), 256, 0, s>>>(sa, count, nwr_max);
    return cudaGetLastError();
}

}  // namespace ldp

// C-ABI entry points (include/ldp.h): argument checks, scratch sizes, the
// code pass of single images (run_plain) followed by the window kernels.
extern "C" {

int ldp_window_count(int n, int w, int s) {
    if (w < 1 || s < 1 || n < 0) return -1;
    return n <= w ? 1 : (n - w + s - 1) / s + 1;
}

namespace {

int check_windows(const ldp_window_spec& ws, int k) {
    if (ws.wh < 1 || ws.ww < 1 || ws.sh < 1 || ws.sw < 1)
        return ldp::report_error(LDP_EINVAL, "window size and stride must be at least 1");
    if (ws.compact != 0 && ws.compact != 1) return ldp::report_error(LDP_EINVAL, "compact must be 0 or 1");
    if (ws.compact && (k < 1 || k > 7)) return ldp::report_error(LDP_EINVAL, "compact bins need k in [1,7]");
    return LDP_OK;
}

ldp::WindowGeom window_geom(const ldp_window_spec& ws, int k) {
    ldp::WindowGeom g{ws.wh, ws.ww, ws.sh, ws.sw, 256, k, ws.compact};
    if (ws.compact) g.nbins = ldp::binom8(k);
    return g;
}

uint64_t align256(uint64_t b) { return (b + 255u) & ~(uint64_t)255u; }

uint64_t window_scratch(int H, int W, int k, const ldp_window_spec& ws, bool codes_given) {
    const ldp::WindowGeom g = window_geom(ws, k);
    uint64_t b = codes_given ? 0 : align256((uint64_t)(H - 2) * (uint64_t)(W - 2));
    if (!ldp::window_direct(g)) b += ldp::window_cell_words(H, W, g) * sizeof(uint32_t);
    return b;
}

int run_windows(int mode, const uint8_t* d_img, int H, int W, int pitch, int k, const ldp_window_spec& ws,
                uint32_t* d_hist, uint8_t* d_codes, int code_pitch, void* d_scratch, uint64_t scratch_bytes,
                void* stream) {
    ldp::Range range("ldp.window_hist");
    int rc;
    if ((rc = ldp::check_image(d_img, H, W, pitch))) return rc;
    if ((rc = ldp::check_codes(d_codes, W, code_pitch, false))) return rc;
    if ((rc = check_windows(ws, k))) return rc;
    if (!d_hist) return ldp::report_error(LDP_EINVAL, "histogram pointer is NULL");
    const int nwr = ldp_window_count(H, ws.wh, ws.sh), nwc = ldp_window_count(W, ws.ww, ws.sw);
    if ((int64_t)nwr * (int64_t)nwc > (1 << 22)) return ldp::report_error(LDP_EINVAL, "more than 1<<22 windows");
    const uint64_t need = window_scratch(H, W, k, ws, d_codes != nullptr);
    if (need && (!d_scratch || scratch_bytes < need)) return ldp::report_error(LDP_EINVAL, "scratch missing or too small");
    if (((uintptr_t)d_scratch & 255u) != 0) return ldp::report_error(LDP_EINVAL, "scratch must be 256-byte aligned");
    uint8_t* sp = static_cast<uint8_t*>(d_scratch);
    if (!d_codes) {
        d_codes = sp;
        code_pitch = W - 2;
        sp += align256((uint64_t)(H - 2) * (uint64_t)(W - 2));
    }
    if ((rc = ldp::run_plain(mode, d_img, H, W, pitch, k < 1 ? 1 : k, 1, 1, 0, nullptr, d_codes, code_pitch, stream)))
        return rc;
    ldp_image_desc one{d_img, H, W, pitch, code_pitch, d_codes, 0};
    cudaError_t e = ldp::launch_windows(nullptr, &one, 1, H, W, window_geom(ws, k), d_hist,
                                        reinterpret_cast<uint32_t*>(sp), 0, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return ldp::report_cuda(e, "window kernels");
    return LDP_OK;
}

}  // namespace

uint64_t ldp_window_scratch_bytes(int H, int W, int k, ldp_window_spec ws, int codes_given) {
    if (H < 3 || W < 3 || k < 0 || k > 7 || ws.wh < 1 || ws.ww < 1 || ws.sh < 1 || ws.sw < 1) return 0;
    if (ws.compact && k < 1) return 0;
    return window_scratch(H, W, k, ws, codes_given != 0);
}

int ldp_window_hist(const uint8_t* d_img, int H, int W, int pitch, int k, ldp_window_spec ws, uint32_t* d_hist,
                    uint8_t* d_codes_or_null, int code_pitch, void* d_scratch, uint64_t scratch_bytes,
                    void* stream) {
    if (k < 1 || k > 7) return ldp::report_error(LDP_EINVAL, "k must be in [1,7]");
    return run_windows(0, d_img, H, W, pitch, k, ws, d_hist, d_codes_or_null, code_pitch, d_scratch,
                       scratch_bytes, stream);
}

int lbp_window_hist(const uint8_t* d_img, int H, int W, int pitch, ldp_window_spec ws, uint32_t* d_hist,
                    uint8_t* d_codes_or_null, int code_pitch, void* d_scratch, uint64_t scratch_bytes,
                    void* stream) {
    if (ws.compact) return ldp::report_error(LDP_EINVAL, "LBP windows use 256 raw bins (compact = 0)");
    return run_windows(1, d_img, H, W, pitch, 0, ws, d_hist, d_codes_or_null, code_pitch, d_scratch,
                       scratch_bytes, stream);
}

uint64_t ldp_batch_window_scratch_bytes(int count, int max_H, int max_W, int k, ldp_window_spec ws) {
    if (count < 1 || max_H < 3 || max_W < 3 || k < 0 || k > 7 || ws.wh < 1 || ws.ww < 1 || ws.sh < 1 ||
        ws.sw < 1 || (ws.compact && k < 1))
        return 0;
    const ldp::WindowGeom g = window_geom(ws, k);
    if (ldp::window_direct(g)) return 0;
    return (uint64_t)count * ldp::window_cell_words(max_H, max_W, g) * sizeof(uint32_t);
}

int ldp_batch_window_hist(const ldp_image_desc* d_descs, int count, int max_H, int max_W, int k,
                          ldp_window_spec ws, uint32_t* d_hist, void* d_scratch, uint64_t scratch_bytes,
                          void* stream) {
    int rc;
    if (!d_descs) return ldp::report_error(LDP_EINVAL, "descriptor pointer is NULL");
    if (count < 1 || count > (1 << 24)) return ldp::report_error(LDP_EINVAL, "count must be in [1, 1<<24]");
    if (max_H < 3 || max_W < 3 || max_H > (1 << 20) || max_W > (1 << 20))
        return ldp::report_error(LDP_EINVAL, "max_H / max_W must be in [3, 1<<20]");
    if (k < 0 || k > 7) return ldp::report_error(LDP_EINVAL, "k must be in [0,7]");
    if ((rc = check_windows(ws, k))) return rc;
    if (!d_hist) return ldp::report_error(LDP_EINVAL, "histogram pointer is NULL");
    ldp::Range range("ldp.batch_window_hist");
    const ldp::WindowGeom g = window_geom(ws, k);
    const uint64_t words = ldp::window_direct(g) ? 0 : ldp::window_cell_words(max_H, max_W, g);
    if (words && (!d_scratch || scratch_bytes < (uint64_t)count * words * sizeof(uint32_t)))
        return ldp::report_error(LDP_EINVAL, "scratch missing or too small");
    cudaError_t e = ldp::launch_windows(d_descs, nullptr, count, max_H, max_W, g, d_hist,
                                        static_cast<uint32_t*>(d_scratch), words, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return ldp::report_cuda(e, "window kernels");
    return LDP_OK;
}

}  // extern "C"
