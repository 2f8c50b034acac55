// Crop-and-resize front end (Sec. 3.1: detected faces are resized to
// 260 x 260 before extraction).  Bilinear resampling with half-pixel centres:
// output index i of an axis samples the source at
//     y = ((2i + 1) n_src - n_dst) / (2 n_dst),
// clamped to [0, n_src - 1]; the fraction becomes an 11-bit weight
// w1 = round(frac * 2048) (halves up), w0 = 2048 - w1, all in exact integer
// arithmetic, and
//     out = (wy0 (wx0 p00 + wx1 p01) + wy1 (wx0 p10 + wx1 p11) + 2^21) >> 22
// (at most 2048 * 2048 * 255 + 2^21 < 2^32).  A CTA owns kRows output rows of
// one image: the rows' coordinates and source row addresses, and (for output
// widths up to kMaxCols) every column's coordinate, are computed once into
// shared memory, in 32-bit arithmetic whenever the numbers fit.  Threads then
// take groups of four output columns of the rows in turn (the CTA's work
// spread evenly whatever the width) and store the four results as one
// 32-bit word where the destination allows.  With aligned source rows (and
// outputs up to kMaxFastCols wide) a group whose source bytes lie within 16
// bytes of an aligned word reads four words of each of its two source rows,
// picks its eight left and right neighbours with byte permutes and forms each
// row's weighted sum with one dp2a (two 16-bit weights times two bytes); other
// groups, and rows that are the image's last, gather the sixteen bytes one by
// one.  Wider outputs compute their column coordinates per thread instead.
#include <cuda_runtime.h>

#include <cstdint>

#include "ldp_device.cuh"
#include "ldp_launch.h"

namespace ldp {

namespace {

constexpr int kRows = 64;
constexpr int kThreads = 256;
constexpr int kMaxCols = 4096;     // output widths whose column table fits in shared memory
constexpr int kMaxFastCols = 2048;  // output widths with the per-group word tables

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// a.lo * b.byte0 + a.hi * b.byte1 + c (16-bit weights, 8-bit pixels)
__device__ __forceinline__ uint32_t dp2a_lo(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("dp2a.lo.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Bytes o_t (t = 0..3, each below 16) of the 16 bytes w[0..3], one per byte
// lane: selector nibble t = o_t mod 8 picks from w[0..1] and from w[2..3],
// the byte mask m (0xFF in lane t where o_t >= 8) chooses between them.
__device__ __forceinline__ uint32_t pick16(const uint32_t (&w)[4], uint32_t sel, uint32_t m) {
    const uint32_t lo = prmt(w[0], w[1], sel), hi = prmt(w[2], w[3], sel);
    return (lo & ~m) | (hi & m);
}

__device__ __forceinline__ void coord(int i, int n_src, int n_dst, int& i0, int& w1) {
    // y = num / den with num = (2i + 1) n_src - n_dst, den = 2 n_dst
    if ((2LL * i + 1) * (long long)n_src < (1LL << 31) && 2LL * n_dst * 2048 < (1LL << 31)) {
        const int num = (2 * i + 1) * n_src - n_dst, den = 2 * n_dst;
        if (num <= 0) {
            i0 = 0;
            w1 = 0;
            return;
        }
        int q = (int)((unsigned)num / (unsigned)den);
        const int r = num - q * den;
        int w = (int)((unsigned)(r * 2048 + den / 2) / (unsigned)den);
        if (w == 2048) {
            q += 1;
            w = 0;
        }
        if (q >= n_src - 1) {
            i0 = n_src - 1;
            w1 = 0;
            return;
        }
        i0 = q;
        w1 = w;
        return;
    }
    const long long num = (2LL * i + 1) * (long long)n_src - (long long)n_dst;
    const long long den = 2LL * n_dst;
    if (num <= 0) {
        i0 = 0;
        w1 = 0;
        return;
    }
    long long q = num / den;
    const long long r = num - q * den;
    long long w = (r * 2048 + den / 2) / den;
    if (w == 2048) {
        q += 1;
        w = 0;
    }
    if (q >= n_src - 1) {
        i0 = n_src - 1;
        w1 = 0;
        return;
    }
    i0 = (int)q;
    w1 = (int)w;
}

struct ResizeArgs {
    const ldp_crop_desc* descs;  // nullptr: the single crop `one`
    ldp_crop_desc one;
    int count, OH, OW;
    int* status;
};

__global__ void __launch_bounds__(kThreads) k_resize(ResizeArgs a) {
    __shared__ const uint8_t* s_pa[kRows];
    __shared__ const uint8_t* s_pb[kRows];
    __shared__ uint32_t s_wy1[kRows];
    __shared__ uint32_t s_col[kMaxCols];  // x0 << 12 | wx1 of each output column (OW <= kMaxCols)
    // OW <= kMaxFastCols: per column wx0 | wx1 << 16; per group of four
    // columns: source column B of the aligned word the group's bytes start
    // in (bit 31: they end within 16 bytes of it), the byte selectors of the
    // four left (low half) and right (high half) neighbours, their masks
    __shared__ uint32_t s_wp[kMaxFastCols];
    __shared__ uint32_t s_grp[kMaxFastCols];
    const int r0 = blockIdx.x * kRows;
    const bool table = a.OW <= kMaxCols;
    for (int img = blockIdx.y; img < a.count; img += gridDim.y) {
        const ldp_crop_desc d = a.descs ? a.descs[img] : a.one;
        const bool ok = d.src && d.dst && d.ch >= 1 && d.cw >= 1 && d.cy >= 0 && d.cx >= 0 &&
                        d.cy + d.ch <= d.H && d.cx + d.cw <= d.W && d.pitch >= d.W && d.dst_pitch >= a.OW;
        if (!ok) {  // uniform over the CTA
            if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(a.status, kStatusBadCrop);
            continue;
        }
        // word path: aligned source rows of at least 16 bytes; a group reads
        // the 16 bytes from its aligned start B, which may run past W into
        // the row's pitch and the next row, so rows that are the image's last
        // take the byte gathers
        const bool fast = a.OW <= kMaxFastCols && (((uintptr_t)d.src | (uintptr_t)d.pitch) & 3u) == 0 && d.W >= 16;
        __syncthreads();  // the previous image's tables are no longer read
        if (threadIdx.x < kRows && r0 + (int)threadIdx.x < a.OH) {
            int y0, w;
            coord(r0 + threadIdx.x, d.ch, a.OH, y0, w);
            const int y1 = y0 + 1 < d.ch ? y0 + 1 : y0;
            s_pa[threadIdx.x] = d.src + (size_t)(d.cy + y0) * (size_t)d.pitch + d.cx;
            s_pb[threadIdx.x] = d.src + (size_t)(d.cy + y1) * (size_t)d.pitch + d.cx;
            s_wy1[threadIdx.x] = (uint32_t)w | (fast && d.cy + y1 < d.H - 1 ? 0x80000000u : 0u);
        }
        if (fast)
            for (int g = threadIdx.x; 4 * g < a.OW; g += blockDim.x) {
                int x0[4], xb[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int j = min(4 * g + t, a.OW - 1);
                    int wx1;
                    coord(j, d.cw, a.OW, x0[t], wx1);
                    xb[t] = x0[t] + 1 < d.cw ? x0[t] + 1 : x0[t];
                    if (4 * g + t < a.OW) {
                        s_col[j] = ((uint32_t)x0[t] << 12) | (uint32_t)wx1;
                        s_wp[j] = (2048u - (uint32_t)wx1) | ((uint32_t)wx1 << 16);
                    }
                }
                const int B = (d.cx + x0[0]) & ~3;
                uint32_t sel = 0, mL = 0, mR = 0;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int oL = min(d.cx + x0[t] - B, 15), oR = min(d.cx + xb[t] - B, 15);
                    sel |= ((uint32_t)(oL & 7) << (4 * t)) | ((uint32_t)(oR & 7) << (16 + 4 * t));
                    mL |= (oL >= 8 ? 0xFFu : 0u) << (8 * t);
                    mR |= (oR >= 8 ? 0xFFu : 0u) << (8 * t);
                }
                s_grp[4 * (g & 511)] = (uint32_t)B | (d.cx + xb[3] - B < 16 ? 0x80000000u : 0u);
                s_grp[4 * (g & 511) + 1] = sel;
                s_grp[4 * (g & 511) + 2] = mL;
                s_grp[4 * (g & 511) + 3] = mR;
            }
        else if (table)
            for (int j = threadIdx.x; j < a.OW; j += blockDim.x) {
                int x0, wx1;
                coord(j, d.cw, a.OW, x0, wx1);
                s_col[j] = ((uint32_t)x0 << 12) | (uint32_t)wx1;  // x0 < 2^20, wx1 <= 2047
            }
        __syncthreads();
        const int nr = min(kRows, a.OH - r0);
        uint8_t* drow = d.dst + (size_t)r0 * (size_t)d.dst_pitch;
        if (table) {
            // bilinear value of output column j from source rows pa / pb
            auto pixel = [&](const uint8_t* pa, const uint8_t* pb, uint32_t wy1, int j) -> uint32_t {
                const uint32_t c = s_col[j];
                const int x0 = (int)(c >> 12);
                const uint32_t wx1 = c & 0xFFFu, wx0 = 2048u - wx1;
                const int xb = x0 + 1 < d.cw ? x0 + 1 : x0;
                if (!index_ok(j < kMaxCols && x0 < d.cw, a.status)) return 0u;
                const uint32_t top = wx0 * __ldg(pa + x0) + wx1 * __ldg(pa + xb);
                const uint32_t bot = wx0 * __ldg(pb + x0) + wx1 * __ldg(pb + xb);
                return ((2048u - wy1) * top + wy1 * bot + (1u << 21)) >> 22;
            };
            const int ncg = (a.OW + 3) / 4;  // groups of four columns
            const bool words = (((uintptr_t)d.dst | (uintptr_t)d.dst_pitch) & 3u) == 0;
            // items (row, group) = threadIdx.x + k * blockDim.x, stepped without a division
            const int dr = (int)blockDim.x / ncg, dc = (int)blockDim.x % ncg;
            int r = (int)threadIdx.x / ncg, cg = (int)threadIdx.x % ncg;
            for (; r < nr;) {
                const uint8_t* pa = s_pa[r];
                const uint8_t* pb = s_pb[r];
                const uint32_t wyf = s_wy1[r], wy1 = wyf & 0xFFFu;
                const int j0 = 4 * cg;
                uint8_t* dp = drow + (size_t)r * (size_t)d.dst_pitch + j0;
                if (j0 + 4 <= a.OW) {
                    uint32_t v0, v1, v2, v3;
                    const uint32_t gB = fast ? s_grp[4 * (cg & 511)] : 0u;
                    if ((wyf & gB) >> 31) {
                        // the group's source bytes lie in four aligned words
                        // of each row: gather them with byte permutes, one
                        // dp2a per row and pixel
                        const int B = (int)(gB & 0x7FFFFFFFu);
                        const uint32_t sel = s_grp[4 * (cg & 511) + 1], mL = s_grp[4 * (cg & 511) + 2],
                                       mR = s_grp[4 * (cg & 511) + 3];
                        const unsigned int* qa = reinterpret_cast<const unsigned int*>(pa - d.cx + B);
                        const unsigned int* qb = reinterpret_cast<const unsigned int*>(pb - d.cx + B);
                        uint32_t wa[4], wb[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            wa[i] = __ldg(qa + i);
                            wb[i] = __ldg(qb + i);
                        }
                        const uint32_t la = pick16(wa, sel & 0xFFFFu, mL), ra = pick16(wa, sel >> 16, mR);
                        const uint32_t lb = pick16(wb, sel & 0xFFFFu, mL), rb = pick16(wb, sel >> 16, mR);
                        uint32_t v[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const uint32_t wp = s_wp[j0 + t], ps = (uint32_t)t | ((uint32_t)(4 + t) << 4);
                            const uint32_t top = dp2a_lo(wp, prmt(la, ra, ps), 0u);
                            const uint32_t bot = dp2a_lo(wp, prmt(lb, rb, ps), 0u);
                            v[t] = ((2048u - wy1) * top + wy1 * bot + (1u << 21)) >> 22;
                        }
                        v0 = v[0];
                        v1 = v[1];
                        v2 = v[2];
                        v3 = v[3];
                    } else {
                        v0 = pixel(pa, pb, wy1, j0);
                        v1 = pixel(pa, pb, wy1, j0 + 1);
                        v2 = pixel(pa, pb, wy1, j0 + 2);
                        v3 = pixel(pa, pb, wy1, j0 + 3);
                    }
                    if (words) {
                        *reinterpret_cast<uint32_t*>(dp) = v0 | (v1 << 8) | (v2 << 16) | (v3 << 24);
                    } else {
                        dp[0] = (uint8_t)v0;
                        dp[1] = (uint8_t)v1;
                        dp[2] = (uint8_t)v2;
                        dp[3] = (uint8_t)v3;
                    }
                } else {
                    for (int j = j0; j < a.OW; ++j) dp[j - j0] = (uint8_t)pixel(pa, pb, wy1, j);
                }
                cg += dc;
                r += dr;
                if (cg >= ncg) {
                    cg -= ncg;
                    ++r;
                }
            }
        } else {
            for (int j = threadIdx.x; j < a.OW; j += blockDim.x) {
                int x0, wx1;
                coord(j, d.cw, a.OW, x0, wx1);
                const int xb = x0 + 1 < d.cw ? x0 + 1 : x0;
                const uint32_t wx0 = 2048u - (uint32_t)wx1;
                uint8_t* dp = drow + j;
                for (int rr = 0; rr < nr; ++rr, dp += d.dst_pitch) {
                    const uint8_t* pa = s_pa[rr];
                    const uint8_t* pb = s_pb[rr];
                    const uint32_t top = wx0 * __ldg(pa + x0) + (uint32_t)wx1 * __ldg(pa + xb);
                    const uint32_t bot = wx0 * __ldg(pb + x0) + (uint32_t)wx1 * __ldg(pb + xb);
                    const uint32_t wy1 = s_wy1[rr] & 0xFFFu;
                    const uint32_t v = (2048u - wy1) * top + wy1 * bot;
                    *dp = (uint8_t)((v + (1u << 21)) >> 22);
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_resize(const ldp_crop_desc* d_descs, const ldp_crop_desc* one, int count, int OH, int OW,
                          int* status, cudaStream_t s) {
    ResizeArgs a{};
    a.descs = d_descs;
    if (one) a.one = *one;
    a.count = count;
    a.OH = OH;
    a.OW = OW;
    a.status = status;
    dim3 grid((OH + kRows - 1) / kRows, count < 65535 ? count : 65535);
    k_resize<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ldp

// C-ABI entry points (include/ldp.h).
extern "C" {

int ldp_resize(const uint8_t* d_src, int H, int W, int pitch, int cy, int cx, int ch, int cw, uint8_t* d_dst,
               int OH, int OW, int dst_pitch, void* stream) {
    if (!d_src || !d_dst) return ldp::report_error(LDP_EINVAL, "image pointer is NULL");
    if (H < 1 || W < 1 || pitch < W) return ldp::report_error(LDP_EINVAL, "bad source size or pitch");
    if (H > (1 << 20) || W > (1 << 20)) return ldp::report_error(LDP_EINVAL, "image side larger than 1<<20");
    if (ch < 1 || cw < 1 || cy < 0 || cx < 0 || cy + ch > H || cx + cw > W)
        return ldp::report_error(LDP_EINVAL, "crop outside the image");
    if (OH < 1 || OW < 1 || OH > (1 << 16) || OW > (1 << 16)) return ldp::report_error(LDP_EINVAL, "output size out of range");
    if (dst_pitch < OW) return ldp::report_error(LDP_EINVAL, "dst_pitch < OW");
    int* status = ldp::status_word();
    if (!status) return ldp::report_error(LDP_ECUDA, "device status word not found");
    ldp::Range range("ldp.resize");
    ldp_crop_desc one{d_src, d_dst, H, W, pitch, cy, cx, ch, cw, dst_pitch};
    cudaError_t e = ldp::launch_resize(nullptr, &one, 1, OH, OW, status, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return ldp::report_cuda(e, "resize kernel");
    return LDP_OK;
}

int ldp_batch_resize(const ldp_crop_desc* d_descs, int count, int OH, int OW, void* stream) {
    if (!d_descs) return ldp::report_error(LDP_EINVAL, "descriptor pointer is NULL");
    if (count < 1 || count > (1 << 24)) return ldp::report_error(LDP_EINVAL, "count must be in [1, 1<<24]");
    if (OH < 1 || OW < 1 || OH > (1 << 16) || OW > (1 << 16)) return ldp::report_error(LDP_EINVAL, "output size out of range");
    int* status = ldp::status_word();
    if (!status) return ldp::report_error(LDP_ECUDA, "device status word not found");
    ldp::Range range("ldp.batch_resize");
    cudaError_t e = ldp::launch_resize(d_descs, nullptr, count, OH, OW, status, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return ldp::report_cuda(e, "resize kernel");
    return LDP_OK;
}

}  // extern "C"
