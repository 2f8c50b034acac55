// Sliding-window code histograms (Sec. 3.2): windows of wh x ww pixels at
// stride (sh, sw) over the image, window (a, b) covering image rows
// [a*sh, min(a*sh + wh, H)) and columns [b*sw, min(b*sw + ww, W)), interior
// pixels only.  Every window is a union of cells of the grid with cell size
// (gcd(wh, sh), gcd(ww, sw)), so the work is
//   k_cell_hist:   one pass over the code map; a CTA owns a row of cells (a
//                  chunk of it for wide images) -- or, when all of an
//                  image's cells fit in shared memory, the whole image
//                  (k_cell_hist_image; k_cell_hist_thread, a thread per
//                  cell over 16-bit counters, when the cells also fit the
//                  CTA's threads) -- and counts its codes there, then
//                  stores the cells' histograms (no global atomics: every
//                  cell belongs to exactly one CTA);
//   k_window_sum:  each window histogram is the sum of its cells' (skipped
//                  when stride = size: the cells are the windows).
// When the column stride divides the window width (cells as wide as the
// stride) and qh rows of cells fit in shared memory, k_window_fused does both
// in one pass instead: a CTA walks an image's window rows top to bottom in
// groups, counts each cell row once into a shared-memory ring that holds the
// cell rows of the current group (16-bit counters, one lane per cell, so
// the reductions of a warp never meet), and sums the group's window rows
// from the ring into a staging copy that the bulk-copy engine sends to HBM
// -- the cell histograms never reach HBM.
// Images come from ldp_image_desc records (batches) or one record passed by
// value (single image).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "ldp_device.cuh"
#include "ldp_launch.h"

namespace ldp {

namespace {

constexpr int kCellThreads = 256;
constexpr int kCellSmemWords = 12156;  // counters at most: with 4 junk words and the 512-byte table, 48 KB
constexpr int kCellThreadSmemBytes = 45056;  // thread-per-cell counters at most (44 KB)

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
    int max_H, max_W;  // bounds of the images' sizes
    int* status;       // device status word
    int junk;          // shared word past the counters: columns past the image, codes without a bin
};

__device__ __forceinline__ ldp_image_desc desc_of(const CellArgs& a, int i) {
    return a.descs ? a.descs[i] : a.one;
}

// An image outside the call's size bounds (or without interior pixels, or
// with a short code pitch) is skipped and sets bit 0 of the status word.
__device__ __forceinline__ bool win_desc_ok(const ldp_image_desc& d, int max_H, int max_W, int* status) {
    const bool ok = d.H >= 3 && d.W >= 3 && d.H <= max_H && d.W <= max_W && d.code_pitch >= d.W - 2;
    if (!ok && threadIdx.x == 0) atomicOr(status, kStatusBadDesc);
    return ok;
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
    extern __shared__ uint32_t cnt[];  // a.chunk * a.nbins counters (sized at launch), then the junk word
    __shared__ int16_t lut[256];
    for (int c = threadIdx.x; c < 256; c += blockDim.x)
        lut[c] = (a.k >= 1) ? __ldg(&g_bin_table.bin[a.k][c]) : (int16_t)c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const float inv_cw = 1.0f / (float)a.cw;
    const uint64_t pairs = (uint64_t)count * (uint64_t)ncr_max;
    for (uint64_t p = blockIdx.x; p < pairs; p += gridDim.x) {
        const int img = (int)(p / (uint64_t)ncr_max), i = (int)(p % (uint64_t)ncr_max);
        const ldp_image_desc d = desc_of(a, img);
        if (d.codes == nullptr || !win_desc_ok(d, a.max_H, a.max_W, a.status)) continue;  // uniform over the CTA
        const int H = d.H, W = d.W;
        const int ncr = (H + a.ch - 1) / a.ch, ncc = (W + a.cw - 1) / a.cw;
        const int j0 = blockIdx.y * a.chunk;
        if (i >= ncr || j0 >= ncc) continue;  // uniform over the CTA
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
                    const int ix = (in[t] && b >= 0) ? off[t] + b : a.junk;
                    if (index_ok(ix <= a.junk, a.status)) atomicAdd(&cnt[ix], 1u);
                }
            }
        }
        __syncthreads();
        uint32_t* out = a.direct ? a.hist + d.hist_offset : a.cells + (uint64_t)img * a.cell_stride;
        const uint64_t first = ((uint64_t)i * (uint64_t)ncc + (uint64_t)j0) * (uint64_t)a.nbins;
        out += first;
        if (a.direct || index_ok(first + (uint64_t)words <= a.cell_stride, a.status))
            for (int e = threadIdx.x; e < words; e += blockDim.x) out[e] = cnt[e];
    }
}

// Whole-image items, for images whose every cell fits in shared memory (the
// face-sized crops): one CTA per image, counters zeroed and stored once,
// warps over rows, lanes over four consecutive columns whose cells are found
// once for all rows (several rows per warp step in a narrow last block).
__global__ void __launch_bounds__(kCellThreads) k_cell_hist_image(CellArgs a, int count) {
    extern __shared__ uint32_t cnt[];  // ncr * ncc * nbins counters of the largest image, then the junk word
    __shared__ int16_t lut[256];
    for (int c = threadIdx.x; c < 256; c += blockDim.x)
        lut[c] = (a.k >= 1) ? __ldg(&g_bin_table.bin[a.k][c]) : (int16_t)c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const float inv_cw = 1.0f / (float)a.cw, inv_ch = 1.0f / (float)a.ch;
    for (int img = blockIdx.x; img < count; img += gridDim.x) {
        const ldp_image_desc d = desc_of(a, img);
        if (d.codes == nullptr || !win_desc_ok(d, a.max_H, a.max_W, a.status)) continue;  // uniform over the CTA
        const int H = d.H, W = d.W;
        const int ncc = (W + a.cw - 1) / a.cw;
        const int words = ((H + a.ch - 1) / a.ch) * ncc * a.nbins;
        __syncthreads();  // lut ready; the previous image's counters are stored
        for (int e = threadIdx.x; e < words; e += blockDim.x) cnt[e] = 0;
        __syncthreads();
        const bool al = (((uintptr_t)d.codes | (uintptr_t)d.code_pitch) & 3u) == 0;
        for (int yb = 1; yb < W - 1; yb += 128) {
            // a block narrower than 128 columns (the image's last) takes
            // several rows per warp step: lp lanes per row (a power of two
            // covering its columns), 32 / lp rows at once
            const int ng = (min(128, W - 1 - yb) + 3) / 4;  // four-column groups of the block
            const int lp = ng > 16 ? 32 : ng > 8 ? 16 : ng > 4 ? 8 : ng > 2 ? 4 : ng > 1 ? 2 : 1;
            const int rows = 32 / lp;
            const int yq = yb + 4 * (lane % lp);  // columns yq .. yq+3 (code columns yq-1 .. yq+2)
            int off[4];
            bool in[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                in[t] = yq + t < W - 1;
                off[t] = in[t] ? cell_of(yq + t, a.cw, inv_cw) * a.nbins : 0;
            }
            const bool vec = al && in[3];  // yq - 1 is a multiple of 4
#pragma unroll 4
            for (int x = 1 + warp * rows + lane / lp; x < H - 1; x += nwarps * rows) {
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
                    const int ix = (in[t] && b >= 0) ? rbase + off[t] + b : a.junk;
                    if (index_ok(ix <= a.junk, a.status)) atomicAdd(&cnt[ix], 1u);
                }
            }
        }
        __syncthreads();
        uint32_t* out = a.direct ? a.hist + d.hist_offset : a.cells + (uint64_t)img * a.cell_stride;
        if (a.direct || index_ok((uint64_t)words <= a.cell_stride, a.status))
            for (int e = threadIdx.x; e < words; e += blockDim.x) out[e] = cnt[e];
    }
}

// Whole-image items with a thread per cell, for images whose cells fit one
// CTA's threads and whose counters fit shared memory (the face-sized crops):
// counters are 16 bits, two bins to a word, pair-major with the cell index
// fastest -- bin j of cell c is half j & 1 of word (j >> 1) * P + c, P a
// multiple of 32 -- so the 32 reductions of a warp (32 consecutive cells)
// hit 32 different banks whatever the codes.  A cell holds at most 65535
// pixels.  Each thread walks its cell's rows: cells of CW columns read
// aligned words one row ahead (rows above the image's last code row may be
// read into their pitch and the next row) and cut them into bytes with a
// funnel shift, positions past the cell masked to code 0 (no compact bin:
// the spare pair row); other cell widths, unaligned code maps and the last
// code row read byte by byte.  The counters then leave as the cells'
// histograms, four bins per 16-byte store where the output allows.
template <int CW>
__device__ __forceinline__ void count_cell(const ldp_image_desc& d, const CellArgs& a, int cell, int ncc, int P,
                                           uint32_t cnt_addr, uint32_t cnt_bytes, const uint16_t* lut,
                                           uint32_t junk_e, bool al) {
    const int H = d.H, W = d.W;
    const int cr = cell / ncc, cc = cell - cr * ncc;
    const int xlo = max(cr * a.ch, 1), xhi = min(cr * a.ch + a.ch, H - 1);  // image rows with codes
    const int ylo = max(cc * a.cw, 1), yhi = min(cc * a.cw + a.cw, W - 1);
    const int s0 = ylo - 1, n = max(yhi - ylo, 0);                          // code columns s0 .. s0+n-1
    const uint32_t rb = cnt_addr + 4u * (uint32_t)cell;
    auto one = [&](uint32_t code, bool ok) {
        uint32_t e = lut[code];
        if (!ok) e = junk_e;
        uint32_t inc;
        asm("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(inc) : "r"(0u), "r"(1u), "r"(e));
        const uint32_t addr = rb + (e & ~31u);
        if (index_ok(addr - cnt_addr < cnt_bytes, a.status)) asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(inc));
    };
    const uint8_t* rp = d.codes + (size_t)(xlo - 1) * (size_t)d.code_pitch;
    constexpr int NW = CW > 0 ? (CW + 6) / 4 : 1;  // words holding CW bytes from any byte offset
    if constexpr (CW > 0) {
        const int base = s0 & ~3;
        const uint32_t sh = 8u * (uint32_t)(s0 & 3);
        const bool words = al && W - 2 >= 4 * NW;  // uniform over the image
        const bool compact = a.k >= 1;             // code 0 has no bin
        constexpr int NA = (CW + 3) / 4;
        for (int x = xlo; x < xhi; ++x, rp += d.code_pitch) {
            uint32_t w[NW];
            if (words && x < H - 2) {
#pragma unroll
                for (int i = 0; i < NW; ++i) w[i] = __ldg(reinterpret_cast<const unsigned int*>(rp + base) + i);
            } else {
#pragma unroll
                for (int i = 0; i < NW; ++i) {
                    w[i] = 0;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int col = base + 4 * i + t;
                        if (col >= s0 && col < s0 + n) w[i] |= (uint32_t)__ldg(rp + col) << (8 * t);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                uint32_t av = __funnelshift_r(w[i], i + 1 < NW ? w[i + 1] : 0u, sh);
                const int m = min(max(n - 4 * i, 0), 4);  // positions below n in this word
                if (compact) av &= m == 4 ? 0xFFFFFFFFu : (1u << (8 * m)) - 1u;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (4 * i + t < CW) one(prmt(av, 0u, 0x4440u | (uint32_t)t), compact || 4 * i + t < n);
            }
        }
    } else {
        for (int x = xlo; x < xhi; ++x, rp += d.code_pitch)
            for (int j = 0; j < n; ++j) one(__ldg(rp + s0 + j), true);
    }
}

__global__ void __launch_bounds__(kCellThreads) k_cell_hist_thread(CellArgs a, int count, int P) {
    extern __shared__ uint4 cnt4[];  // (nbins / 2 + 1) x P words
    uint32_t* cnt = reinterpret_cast<uint32_t*>(cnt4);
    const int npr = a.nbins / 2 + 1;
    const uint32_t cnt_addr = (uint32_t)__cvta_generic_to_shared(cnt);
    const uint32_t cnt_bytes = 4u * (uint32_t)(npr * P);
    // per code: byte offset of its bin pair's row + 16 x (bin & 1) (codes
    // without a compact bin: pair row nbins / 2, lower half)
    __shared__ uint16_t lut[256];
    for (int c = threadIdx.x; c < 256; c += blockDim.x) {
        int b = (a.k >= 1) ? (int)__ldg(&g_bin_table.bin[a.k][c]) : c;
        if (b < 0) b = a.nbins;
        lut[c] = (uint16_t)((uint32_t)(b >> 1) * 4u * (uint32_t)P + 16u * (uint32_t)(b & 1));
    }
    const uint32_t junk_e = (uint32_t)(a.nbins >> 1) * 4u * (uint32_t)P;
    for (int img = blockIdx.x; img < count; img += gridDim.x) {
        const ldp_image_desc d = desc_of(a, img);
        if (d.codes == nullptr || !win_desc_ok(d, a.max_H, a.max_W, a.status)) continue;  // uniform over the CTA
        const int ncc = (d.W + a.cw - 1) / a.cw, ncells = ((d.H + a.ch - 1) / a.ch) * ncc;
        __syncthreads();  // table ready; the previous image's counters are stored
        for (int e = threadIdx.x; e < npr * P / 4; e += blockDim.x) cnt4[e] = make_uint4(0, 0, 0, 0);
        __syncthreads();
        const bool al = (((uintptr_t)d.codes | (uintptr_t)d.code_pitch) & 3u) == 0;
        for (int cell = threadIdx.x; cell < ncells; cell += blockDim.x) {
            if (a.cw == 20) count_cell<20>(d, a, cell, ncc, P, cnt_addr, cnt_bytes, lut, junk_e, al);
            else if (a.cw == 10) count_cell<10>(d, a, cell, ncc, P, cnt_addr, cnt_bytes, lut, junk_e, al);
            else if (a.cw == 25) count_cell<25>(d, a, cell, ncc, P, cnt_addr, cnt_bytes, lut, junk_e, al);
            else count_cell<0>(d, a, cell, ncc, P, cnt_addr, cnt_bytes, lut, junk_e, al);
        }
        asm volatile("" ::: "memory");
        __syncthreads();
        // cell c's histogram: words c * nbins .. of its output; thread per
        // (cell, group of four bins), cells fastest (conflict-free reads)
        uint32_t* out = a.direct ? a.hist + d.hist_offset : a.cells + (uint64_t)img * a.cell_stride;
        const int words = ncells * a.nbins;
        if (!a.direct && !index_ok((uint64_t)words <= a.cell_stride, a.status)) continue;
        const bool vec = (a.nbins & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
        if (vec) {
            for (int q = 0; q < a.nbins / 4; ++q)
                for (int c = threadIdx.x; c < ncells; c += blockDim.x) {
                    const uint32_t lo = cnt[(2 * q) * P + c], hi = cnt[(2 * q + 1) * P + c];
                    __stcs(reinterpret_cast<uint4*>(out + (size_t)c * a.nbins + 4 * q),
                           make_uint4(lo & 0xFFFFu, lo >> 16, hi & 0xFFFFu, hi >> 16));
                }
        } else {
            for (int p = 0; p < a.nbins / 2; ++p)
                for (int c = threadIdx.x; c < ncells; c += blockDim.x) {
                    const uint32_t v = cnt[p * P + c];
                    out[(size_t)c * a.nbins + 2 * p] = v & 0xFFFFu;
                    out[(size_t)c * a.nbins + 2 * p + 1] = v >> 16;
                }
        }
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
    int max_H, max_W;
    int* status;
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
        // images without codes have no cells (the counting pass skipped them)
        if (d.codes == nullptr || !win_desc_ok(d, a.max_H, a.max_W, a.status)) continue;
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
                    for (int cj = j0; cj < j1; ++cj)
                        if (index_ok(((uint64_t)ci * (uint64_t)ncc + (uint64_t)cj) * (uint64_t)a.nbins + (uint64_t)bin <
                                         a.cell_stride,
                                     a.status))
                            s += __ldg(row + (size_t)cj * (size_t)a.nbins);
                }
                out[(size_t)wb * (size_t)a.nbins + bin] = s;
            }
        }
    }
}

constexpr int kFusedThreads = 256;
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int kFusedSmemWords = 40960;    // ring + staging at most (160 KB)
constexpr int kFusedGroupWords = 14080;   // ring + staging up to which window rows are grouped (55 KB: 4 CTAs per SM)
constexpr int kFusedMaxGroup = 8;         // window rows per group at most

// 32-bit load from shared memory at byte address a.
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

struct FusedArgs {
    const ldp_image_desc* descs;  // nullptr: the single image `one`
    ldp_image_desc one;
    int ch, cw;          // cell size in pixels; cw is the column stride
    int qh, qw;          // window size in cells
    int ph;              // row stride in cells
    int wh, ww, sh, sw;  // window size and stride in pixels (window counts)
    int nbins, k;        // as in CellArgs (nbins even)
    int ncp;             // cells per ring row: a multiple of 32 covering the widest image's cells and windows
    int row_stride;      // ring words per cell row: (nbins / 2 + 1) x ncp (bin pairs, pair nbins / 2 takes codes without a bin)
    int stage_words;     // staging words per window row: the widest image's windows x nbins
    int group;           // window rows per group (G)
    int nslots;          // ring rows: (G - 1) * ph + qh
    int rows_per_band;   // window rows per work item
    int bands;           // work items per image
    uint32_t* hist;
    int max_H, max_W;    // bounds of the images' sizes (the ring is sized for max_W)
    int* status;
};

// Work item = (image, band of window rows).  The band is walked in groups of
// G window rows.  Per group: the cell rows the group covers that are not yet
// in the ring are zeroed and counted (ring slot = cell row mod nslots; the
// nslots = (G-1) ph + qh rows of a group are distinct mod nslots, rows past
// the image stay out), then each output word (window b, bin) of the G window
// rows is the sum over the window's qh x qw cells of their ring counters,
// written to a shared staging copy of the G window rows, laid out as in HBM,
// which one thread hands to the bulk-copy engine as one contiguous block
// while the next group is zeroed and counted (the threads copy it word by
// word when the histograms are not 16-byte aligned or not whole quads of
// bins).  Three barriers per group.
// Counters are 16 bits, two bins to a word: bin j of cell c is half j & 1 of
// word (j >> 1) * ncp + c of its ring row (ncp a multiple of 32), so a cell
// of at most 65535 pixels cannot carry into the other half, and sums of such
// words over a window of at most 65535 pixels stay exact in each half.
// Counting gives each lane one cell: units (image row, block of 32 cells) are
// split evenly over the warps, and lane l counts the row's pixels of cell
// 32 * block + l, so the 32 reductions of one instruction hit 32 different
// words in 32 different banks, whatever the codes.  The code table holds
// one byte per code, its bin b: the reduction adds 1 << (16 (b & 1)) to the
// word of pair row b >> 1.  Output items (a block of 32 windows and four
// bins -- two pair rows -- or, when nbins is not a multiple of four, two
// bins) go to the warps in turn, a lane per window: a warp reads 32
// consecutive cells of a pair row per load, and each cell row of a pair of
// window rows once.

__global__ void __launch_bounds__(kFusedThreads, 4) k_window_fused(FusedArgs a, int count) {
    extern __shared__ uint4 smem4[];  // ring (nslots x row_stride words), then staging (group x stage_words)
    uint32_t* ring = reinterpret_cast<uint32_t*>(smem4);
    const int rs = a.row_stride, ns = a.nslots, ncp = a.ncp;
    const uint32_t b4 = 4u * (uint32_t)ncp;  // bytes between the pair rows of a ring row
    // bin of each code (compact bins: nbins for codes without one); one byte
    // an entry, so a lookup meets at most two words in a bank
    __shared__ uint8_t lut[256];
    for (int c = threadIdx.x; c < 256; c += kFusedThreads) {
        int b = (a.k >= 1) ? (int)__ldg(&g_bin_table.bin[a.k][c]) : c;
        if (b < 0) b = a.nbins;
        lut[c] = (uint8_t)b;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ring_addr = (uint32_t)__cvta_generic_to_shared(ring);
    const uint32_t ring_bytes = 4u * (uint32_t)(ns * rs);
    const uint32_t stage_addr = ring_addr + ring_bytes;
    const uint32_t stage_bytes = 4u * (uint32_t)(a.group * a.stage_words);  // (checked builds)
    const unsigned items = (unsigned)count * (unsigned)a.bands;  // below 2^31 (checked at launch)
    for (unsigned it = blockIdx.x; it < items; it += gridDim.x) {
        const int img = (int)(it / (unsigned)a.bands), band = (int)(it - (unsigned)img * (unsigned)a.bands);
        const ldp_image_desc d = a.descs ? a.descs[img] : a.one;
        if (d.codes == nullptr || !win_desc_ok(d, a.max_H, a.max_W, a.status)) continue;  // uniform over the CTA
        const int H = d.H, W = d.W;
        const int nwr = win_count(H, a.wh, a.sh), nwc = win_count(W, a.ww, a.sw);
        const int a0 = band * a.rows_per_band, a1 = min(a0 + a.rows_per_band, nwr);
        if (a0 >= a1) continue;
        const int ncr = (H + a.ch - 1) / a.ch;
        const int ncc = (W - 2) / a.cw + 1;  // cells holding interior columns
        const int nblk = (ncc + 31) / 32;
        const int words = nwc * a.nbins;
        uint32_t* out_img = a.hist + d.hist_offset;
        // the staged window rows leave in 16-byte stores when the image's
        // histograms start on a 16-byte boundary and every window is whole
        // quads of bins (the staging copy is read by windows)
        const bool vec = (a.nbins & 3) == 0 && (reinterpret_cast<uintptr_t>(out_img) & 15u) == 0;

        const bool al = ((reinterpret_cast<uintptr_t>(d.codes) | (uintptr_t)d.code_pitch) & 3u) == 0;
        int n0 = 0, sn0 = 0;  // first cell row counted by the current group, its ring slot
        // count image rows [xa, xb) of cell block cb: lane l takes cell
        // 32 cb + l (code columns s0 .. s0+n-1 of each row), each code one
        // reduction into the ring row of its cell row.  COMPACT (k >= 1):
        // code 0 has no bin, so positions past the cell's columns are zeroed
        // and count into the spare bin row through the table; raw bins test
        // the position instead.
        auto count_rows = [&](int cb, int xa, int xb, auto cw_c, auto compact_c) {
            constexpr int CW = decltype(cw_c)::value;  // a.cw when it is at most 13, else 0
            constexpr bool COMPACT = decltype(compact_c)::value;
            const int c = cb * 32 + lane;
            const int s0 = max(c * a.cw - 1, 0), e0 = min(c * a.cw + a.cw - 1, W - 2);
            const int n = c < ncc ? max(e0 - s0, 0) : 0;
            const int r = (int)((unsigned)xa / (unsigned)a.ch);  // cell row of image row xa (>= n0)
            int s = sn0 + (r - n0), nb = (r + 1) * a.ch;
            if (s >= ns) s -= ns;
            uint32_t rb = ring_addr + 4u * (uint32_t)(s * rs + c);
            // one code (byte 0 of `code`): its table entry e, one reduction
            // of 1 << (e mod 32) -- 1 or 1 << 16 -- at rb + (e rounded down to 32)
            auto one = [&](uint32_t code, bool ok) {
                uint32_t bin = lut[code];
                if (!COMPACT && !ok) bin = (uint32_t)a.nbins;
                uint32_t inc;
                asm("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(inc) : "r"(0u), "r"(1u), "r"(bin << 4));
                const uint32_t addr = rb + (bin >> 1) * b4;
                if (index_ok(addr - ring_addr < ring_bytes, a.status))
                    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(inc));
            };
            auto next_row = [&](int x) {
                if (x >= nb) {  // into the next cell row
                    nb += a.ch;
                    if (++s == ns) s = 0;
                    rb = ring_addr + 4u * (uint32_t)(s * rs + c);
                }
            };
            if constexpr (CW > 0) {
                // the cell's bytes, at positions 0 .. CW-1 from column s0,
                // come from four aligned words at `base` (one row ahead).  With
                // whole words (aligned code map, W - 2 >= 16) a row is read up
                // to 16 bytes from base: past its last code into its pitch and
                // the next row, never past the image's last code row, which
                // (like every row without whole words) is read byte by byte,
                // its bytes outside the cell zero
                const int lastw = (W - 3) & ~3;             // the word holding a row's last code
                const int base = min(s0 & ~3, lastw);       // clamped for cells past the image
                const uint32_t sh = 8u * (uint32_t)(s0 & 3);
                const bool words = al && W - 2 >= 16;       // uniform over the image
                const int xlast = H - 2;                     // image row of the last code row
                constexpr int NA = (CW + 3) / 4;
                uint32_t msk[NA];                            // bytes of positions below n
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    const int m = min(max(n - 4 * i, 0), 4);
                    msk[i] = m == 4 ? 0xFFFFFFFFu : (1u << (8 * m)) - 1u;
                }
                const uint8_t* rp = d.codes + (size_t)(xa - 1) * (size_t)d.code_pitch + base;
                auto fetch = [&](const uint8_t* row, int x, uint32_t(&w)[4]) {
                    if (words && x < xlast) {  // uniform over the warp
#pragma unroll
                        for (int i = 0; i < 4; ++i) w[i] = __ldg(reinterpret_cast<const unsigned int*>(row) + i);
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            w[i] = 0;
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                const int col = base + 4 * i + t;
                                if (col >= s0 && col < s0 + n) w[i] |= (uint32_t)__ldg(row + 4 * i + t) << (8 * t);
                            }
                        }
                    }
                };
                uint32_t w[4], nx[4];
                if (xa < xb) fetch(rp, xa, nx);
                for (int x = xa; x < xb; ++x) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) w[i] = nx[i];
                    rp += d.code_pitch;
                    if (x + 1 < xb) fetch(rp, x + 1, nx);
                    next_row(x);
                    // positions 4i .. 4i+3 in av[i]
                    uint32_t av[NA];
#pragma unroll
                    for (int i = 0; i < NA; ++i) {
                        av[i] = __funnelshift_r(w[i], i + 1 < 4 ? w[i + 1] : 0u, sh);
                        if constexpr (COMPACT) av[i] &= msk[i];
                    }
#pragma unroll
                    for (int j = 0; j < CW; ++j) one(prmt(av[j >> 2], 0u, 0x4440u | (uint32_t)(j & 3)), j < n);
                }
            } else {
                const uint8_t* rp = d.codes + (size_t)(xa - 1) * (size_t)d.code_pitch + s0;
                for (int x = xa; x < xb; ++x, rp += d.code_pitch) {
                    next_row(x);
                    for (int j = 0; j < n; ++j) one(__ldg(rp + j), true);
                }
            }
            asm volatile("" ::: "memory");  // the reductions come before the barrier that follows
        };


        // ring slots: cell row r lives in slot r mod ns, tracked without
        // divisions from the slot of the group's first new cell row (sn0)
        const int ph2_ns = (2 * a.ph) % ns;
        // output items (bin group q, block of 32 windows) go to the warps in
        // turn: item = q * nbw + bb, stepped by the warp count
        const bool quad = (a.nbins & 3) == 0;           // items of four bins (two pair rows), else two
        const int nq = quad ? a.nbins >> 2 : a.nbins >> 1;
        const int nbw = (nwc + 31) >> 5;
        const int dbb = kFusedWarps % nbw, dq = kFusedWarps / nbw;
        const int q_first = warp / nbw, bb_first = warp % nbw;

        // the staged window rows of the previous group -> HBM
        uint32_t* pend_dst = nullptr;
        int pend_n = 0;  // words
        // The staging copy is laid out like the rows in HBM.  With 16-byte
        // alignment one thread hands the block to the bulk-copy engine
        // (cp.async.bulk, shared -> global) and the CTA goes on; the copy has
        // read the staging before it is written again (the wait before the
        // output phase's barrier).  Otherwise the threads copy it word by word.
        auto copy_out = [&]() {
            if (pend_n <= 0) return;
            if (vec) {
                if (threadIdx.x == 0 && index_ok(4u * (uint32_t)pend_n <= stage_bytes, a.status)) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile(
                        "{\n\t.reg .u64 g;\n\tcvta.to.global.u64 g, %0;\n\t"
                        "cp.async.bulk.global.shared::cta.bulk_group [g], [%1], %2;\n\t}" ::"l"(pend_dst),
                        "r"(stage_addr), "r"(4u * (uint32_t)pend_n)
                        : "memory");
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
            } else {
                for (int e = threadIdx.x; e < pend_n; e += kFusedThreads) {
                    const uint32_t sa = stage_addr + 4u * (uint32_t)e;
                    if (index_ok(sa - stage_addr < stage_bytes, a.status)) pend_dst[e] = lds32(sa);
                }
            }
            pend_n = 0;
        };
        auto staging_free = [&]() {  // the bulk copies have read the staging
            if (vec && threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        };

        // window rows wa and (two) wa + 1 of the group starting at g0 into the
        // staging copy; sw: ring slot of the first cell row of window row wa.
        // The cell rows of both are read once, [wa * ph, wa * ph + ph + qh):
        // the rows they share (ph < qh) count into both.
        // QW: qw when it is a small constant (unrolled), else 0 (a loop)
        auto emit = [&](auto qw_c, auto quad_c, int wa, bool two, int g0, int sw) {
            constexpr int QW = decltype(qw_c)::value;
            constexpr bool QUAD = decltype(quad_c)::value;
            const int qwn = QW ? QW : a.qw;
            const int nrow = min(two ? a.ph + a.qh : a.qh, ncr - wa * a.ph);
            const uint32_t rs4 = 4u * (uint32_t)rs, so0 = rs4 * (uint32_t)sw;
            const uint32_t srow = 4u * (uint32_t)words;  // staging bytes per window row
            const uint32_t st0 = stage_addr + srow * (uint32_t)(wa - g0), st1 = st0 + srow;
            for (int q = q_first, bb = bb_first; q < nq;) {
                const int b = bb * 32 + lane;  // lane l takes window 32 * block + l
                bb += dbb;
                const int qi = q;
                q += dq;
                if (bb >= nbw) {
                    bb -= nbw;
                    ++q;
                }
                if (b >= nwc) continue;
                // pair rows (QUAD ? 2qi, 2qi+1 : qi) of cell b at p0 (p1) + so
                const uint32_t pq = ring_addr + (QUAD ? 2u : 1u) * b4 * (uint32_t)qi + 4u * (uint32_t)b;
                uint32_t ax = 0, ay = 0, bx = 0, by = 0;  // packed bin pairs of window rows wa, wa + 1
                uint32_t so = so0;
                for (int ri = 0; ri < nrow; ++ri) {
                    const uint32_t p0 = pq + so, p1 = p0 + b4;
                    uint32_t x = 0, y = 0;
                    if (index_ok((QUAD ? p1 : p0) + 4u * (uint32_t)(qwn - 1) - ring_addr < ring_bytes, a.status)) {
#pragma unroll
                        for (int c = 0; c < qwn; ++c) {
                            x += lds32(p0 + 4u * c);
                            if constexpr (QUAD) y += lds32(p1 + 4u * c);
                        }
                    }
                    if (ri < a.qh) {
                        ax += x;
                        ay += y;
                    }
                    if (two && ri >= a.ph) {
                        bx += x;
                        by += y;
                    }
                    so += rs4;
                    if (so == ring_bytes) so = 0;
                }
                const uint32_t o = 4u * (uint32_t)(b * a.nbins + (QUAD ? 4 : 2) * qi);
                for (int h = 0; h < (two ? 2 : 1); ++h) {
                    const uint32_t sa = (h ? st1 : st0) + o, u = h ? bx : ax, v = h ? by : ay;
                    if (!index_ok(sa + (QUAD ? 16u : 8u) - stage_addr <= stage_bytes, a.status)) continue;
                    if constexpr (QUAD)
                        asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(sa), "r"(u & 0xFFFFu),
                                     "r"(u >> 16), "r"(v & 0xFFFFu), "r"(v >> 16)
                                     : "memory");
                    else
                        asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(sa), "r"(u & 0xFFFFu), "r"(u >> 16)
                                     : "memory");
                }
            }
        };
        auto emit_pair = [&](int wa, bool two, int g0, int sw) {
            auto go = [&](auto quad_c) {
                if (a.qw == 1) emit(std::integral_constant<int, 1>{}, quad_c, wa, two, g0, sw);
                else if (a.qw == 2) emit(std::integral_constant<int, 2>{}, quad_c, wa, two, g0, sw);
                else if (a.qw == 3) emit(std::integral_constant<int, 3>{}, quad_c, wa, two, g0, sw);
                else if (a.qw == 4) emit(std::integral_constant<int, 4>{}, quad_c, wa, two, g0, sw);
                else emit(std::integral_constant<int, 0>{}, quad_c, wa, two, g0, sw);
            };
            if (quad) go(std::true_type{});
            else go(std::false_type{});
        };

        int next = a0 * a.ph;  // first cell row not in the ring
        for (int g0 = a0; g0 < a1; g0 += a.group) {
            const int g1 = min(g0 + a.group, a1);  // window rows [g0, g1)
            n0 = max(next, g0 * a.ph);
            const int n1 = min((g1 - 1) * a.ph + a.qh, ncr);  // cell rows to count: [n0, n1)
            sn0 = n0 % ns;
            __syncthreads();  // the previous group's reads of the ring and writes of the staging are done
            copy_out();
            for (int r = n0, sl = sn0; r < n1; ++r) {
                uint4* row = reinterpret_cast<uint4*>(ring + sl * rs);
                for (int e = threadIdx.x; e < rs / 4; e += kFusedThreads) row[e] = make_uint4(0, 0, 0, 0);
                if (++sl == ns) sl = 0;
            }
            __syncthreads();
            if (n0 < n1) {
                // units (cell block, image row) of cell rows [n0, n1), block-major,
                // an equal share of consecutive units per warp
                const int x0 = max(n0 * a.ch, 1), x1 = min(n1 * a.ch, H - 1);
                const int R = x1 - x0;
                if (R > 0) {
                    const int T = R * nblk;
                    const int t1 = (T * (warp + 1)) / kFusedWarps;
                    for (int t = (T * warp) / kFusedWarps; t < t1;) {
                        const int cb = (int)((unsigned)t / (unsigned)R), r0 = t - cb * R, r1 = min(R, r0 + (t1 - t));
                        const int xa = x0 + r0, xb = x0 + r1;
                        if (a.k >= 1) {
                            const std::true_type cp;
                            if (a.cw == 10) count_rows(cb, xa, xb, std::integral_constant<int, 10>{}, cp);
                            else if (a.cw <= 13) count_rows(cb, xa, xb, std::integral_constant<int, 13>{}, cp);
                            else count_rows(cb, xa, xb, std::integral_constant<int, 0>{}, cp);
                        } else {
                            const std::false_type cp;
                            if (a.cw <= 13) count_rows(cb, xa, xb, std::integral_constant<int, 13>{}, cp);
                            else count_rows(cb, xa, xb, std::integral_constant<int, 0>{}, cp);
                        }
                        t += r1 - r0;
                    }
                }
            }
            next = max(next, n1);
            staging_free();
            __syncthreads();
            int sw = (g0 * a.ph) % ns;  // slot of the first cell row of window row wa
            for (int wa = g0; wa < g1; wa += 2) {
                emit_pair(wa, wa + 1 < g1, g0, sw);
                sw += ph2_ns;
                if (sw >= ns) sw -= ns;
            }
            // the staging writes, seen by the bulk-copy engine's reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            pend_dst = out_img + (size_t)g0 * (size_t)words;
            pend_n = (g1 - g0) * words;
        }
        __syncthreads();
        copy_out();  // the next item's output waits for it (staging_free)
    }
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // every copy done
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

bool window_direct(const WindowGeom& g) { return g.wh == g.sh && g.ww == g.sw; }

namespace {
struct FusedPlan {
    uint64_t rs = 0;
    int ncp = 0, group = 1, nslots = 1, stage_words = 0;
};

// The fused pass for images up to max_W wide: ring row words (rs), staging
// words per window row, window rows per group (G) and ring rows (nslots);
// rs = 0 when the pass does not apply (stride = size, a column stride that
// does not divide the width, windows of more than 65535 pixels -- their sums
// would not fit a 16-bit half --, or rows of cells too wide for shared
// memory).  Groups take as many window rows as keep the
// ring and the staging within kFusedGroupWords (up to kFusedMaxGroup); rows of
// windows with gaps between them (row stride above the height) are not
// grouped.
FusedPlan fused_plan(int max_W, const WindowGeom& g) {
    FusedPlan p;
    if (window_direct(g) || g.ww % g.sw != 0 || (g.nbins & 1) != 0) return p;
    if ((int64_t)g.wh * (int64_t)g.ww > 65535) return p;
    const int ch = gcd_int(g.wh, g.sh), qh = g.wh / ch, qw = g.ww / g.sw, ph = g.sh / ch;
    // cells of a ring row: those a window row reads (the last window of the
    // widest image starts in cell nwc - 1 and spans qw cells) and those
    // holding interior columns
    const int nwc = max_W <= g.ww ? 1 : (max_W - g.ww + g.sw - 1) / g.sw + 1;
    const int ncells = std::max(nwc + qw - 1, (max_W - 2) / g.sw + 1);
    const int ncp = (ncells + 31) / 32 * 32;
    const uint64_t rs = (uint64_t)(g.nbins / 2 + 1) * (uint64_t)ncp;
    const uint64_t stage = (uint64_t)nwc * (uint64_t)g.nbins;  // staging words per window row
    if ((uint64_t)qh * rs + stage > (uint64_t)kFusedSmemWords) return p;
    p.rs = rs;
    p.ncp = ncp;
    p.nslots = qh;
    p.stage_words = (int)stage;
    if (ph <= qh)
        for (int G = 2; G <= kFusedMaxGroup; ++G) {
            const int ns = (G - 1) * ph + qh;
            if ((uint64_t)ns * rs + (uint64_t)G * stage > (uint64_t)kFusedGroupWords) break;
            p.group = G;
            p.nslots = ns;
        }
    return p;
}
}  // namespace

uint64_t window_cell_words(int H, int W, const WindowGeom& g) {
    if (window_direct(g) || fused_plan(W, g).rs) return 0;
    const int ch = gcd_int(g.wh, g.sh), cw = gcd_int(g.ww, g.sw);
    return (uint64_t)((H + ch - 1) / ch) * (uint64_t)((W + cw - 1) / cw) * (uint64_t)g.nbins;
}

cudaError_t launch_windows(const ldp_image_desc* d_descs, const ldp_image_desc* one, int count, int max_H,
                           int max_W, const WindowGeom& g, uint32_t* hist, uint32_t* cells,
                           uint64_t cell_stride, cudaStream_t s) {
    const int ch = gcd_int(g.wh, g.sh), cw = gcd_int(g.ww, g.sw);
    const bool direct = window_direct(g);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int* status = status_word();
    if (!status) return cudaErrorInvalidSymbol;
    if (const FusedPlan fp = fused_plan(max_W, g); fp.rs) {
        cudaError_t e = cudaFuncSetAttribute(k_window_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kFusedSmemWords * sizeof(uint32_t)));
        if (e != cudaSuccess) return e;
        FusedArgs fa{};
        fa.descs = d_descs;
        if (one) fa.one = *one;
        fa.ch = ch;
        fa.cw = cw;
        fa.qh = g.wh / ch;
        fa.qw = g.ww / cw;
        fa.ph = g.sh / ch;
        fa.wh = g.wh;
        fa.ww = g.ww;
        fa.sh = g.sh;
        fa.sw = g.sw;
        fa.nbins = g.nbins;
        fa.k = g.compact ? g.k : 0;
        fa.row_stride = (int)fp.rs;
        fa.stage_words = fp.stage_words;
        fa.ncp = fp.ncp;
        fa.group = fp.group;
        fa.nslots = fp.nslots;
        fa.hist = hist;
        fa.max_H = max_H;
        fa.max_W = max_W;
        fa.status = status;
        const size_t smem =
            sizeof(uint32_t) * ((size_t)fp.rs * (size_t)fp.nslots + (size_t)fp.group * (size_t)fp.stage_words);
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_window_fused, kFusedThreads, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
        // bands of window rows: enough work items for two waves of the GPU,
        // each band at least one group long
        const int nwr_max = (max_H <= g.wh) ? 1 : (max_H - g.wh + g.sh - 1) / g.sh + 1;
        const int64_t want = 2LL * sms * occ;
        int bands = (int)((want + count - 1) / count);
        const int max_bands = (nwr_max + fp.group - 1) / fp.group;
        if (bands > max_bands) bands = max_bands;
        if (bands < 1) bands = 1;
        if ((int64_t)count * bands > (int64_t)INT32_MAX) bands = 1;  // work items stay below 2^31
        fa.rows_per_band = (nwr_max + bands - 1) / bands;
        fa.bands = (nwr_max + fa.rows_per_band - 1) / fa.rows_per_band;
        const uint64_t items = (uint64_t)count * (uint64_t)fa.bands;
        const unsigned grid = (unsigned)(items < (1u << 20) ? items : (1u << 20));
        k_window_fused<<<grid, kFusedThreads, smem, s>>>(fa, count);
        return cudaGetLastError();
    }
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
    ca.max_H = max_H;
    ca.max_W = max_W;
    ca.status = status;
    const int ncr = (max_H + ch - 1) / ch;
    const uint64_t image_words = (uint64_t)ncr * (uint64_t)ncc_max * (uint64_t)g.nbins;
    const uint64_t ncells_max = (uint64_t)ncr * (uint64_t)ncc_max;
    const uint64_t P = (ncells_max + 31) / 32 * 32;
    const uint64_t tw = (uint64_t)(g.nbins / 2 + 1) * P;  // words of the thread-per-cell counters
    if (ncells_max <= (uint64_t)kCellThreads && (g.nbins & 1) == 0 && (uint64_t)ch * (uint64_t)cw <= 65535u &&
        tw * 4u <= (uint64_t)kCellThreadSmemBytes && (uint64_t)(g.nbins / 2) * 4u * P + 16u <= 65535u) {
        // a thread per cell, one CTA per image
        const unsigned grid = (unsigned)(count < sms * 16 ? count : sms * 16);
        const unsigned threads = (unsigned)P;
        k_cell_hist_thread<<<grid, threads, sizeof(uint32_t) * (size_t)tw, s>>>(ca, count, (int)P);
    } else if (image_words <= (uint64_t)kCellSmemWords) {
        // every cell of an image fits: one CTA per image
        const unsigned grid = (unsigned)(count < sms * 16 ? count : sms * 16);
        ca.junk = (int)image_words;
        k_cell_hist_image<<<grid, kCellThreads, sizeof(uint32_t) * ((size_t)image_words + 4), s>>>(ca, count);
    } else {
        // CTAs loop over (image, cell row) items: a few waves of the GPU
        const uint64_t pairs = (uint64_t)count * (uint64_t)ncr;
        const uint64_t cap = (uint64_t)sms * 32;
        dim3 grid((unsigned)(pairs < cap ? pairs : cap), (ncc_max + ca.chunk - 1) / ca.chunk);
        ca.junk = ca.chunk * g.nbins;
        k_cell_hist<<<grid, kCellThreads, sizeof(uint32_t) * ((size_t)ca.junk + 4), s>>>(ca, count, ncr);
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
    sa.max_H = max_H;
    sa.max_W = max_W;
    sa.status = status;
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
    b += ldp::window_cell_words(H, W, g) * sizeof(uint32_t);
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
    const ldp::WindowGeom g = window_geom(ws, k);
    // one image: the cell stride is the image's own cell words (the bound a
    // checked build tests the cell reads against)
    cudaError_t e = ldp::launch_windows(nullptr, &one, 1, H, W, g, d_hist, reinterpret_cast<uint32_t*>(sp),
                                        ldp::window_cell_words(H, W, g), static_cast<cudaStream_t>(stream));
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
    const uint64_t words = ldp::window_cell_words(max_H, max_W, g);
    if (words && (!d_scratch || scratch_bytes < (uint64_t)count * words * sizeof(uint32_t)))
        return ldp::report_error(LDP_EINVAL, "scratch missing or too small");
    cudaError_t e = ldp::launch_windows(d_descs, nullptr, count, max_H, max_W, g, d_hist,
                                        static_cast<uint32_t*>(d_scratch), words, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return ldp::report_cuda(e, "window kernels");
    return LDP_OK;
}

}  // extern "C"
