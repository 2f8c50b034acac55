// Device building blocks for LDP / LBP extraction on sm_103a.
//
// Per pixel (Sec. 2.2.1-2.2.2, Eq. 1-3): every Kirsch mask weighs three
// consecutive ring neighbours by 5 and the other five by -3, so
//     m_i = 8*S3_i - 3*S8,   S3_i = p_{i-1} + p_i + p_{i+1},  S8 = sum_j p_j
// (ring p_0..p_7 counter-clockwise from East).  The eight S3_i and S8 are
// built from column and row three-sums shared between neighbouring pixels.
//
// Ranking: with D_i = 256*m_i = 2048*S3_i - 768*S8 (low 8 bits zero) the key
//     key_i = 2^20 - |D_i| + 2^i
// is unique per direction, orders by |m_i| descending, and breaks ties toward
// the lower index (smaller 2^i).  The k smallest keys are the k most
// outstanding responses, and because the low bytes of the keys are distinct
// one-hot bits, the low byte of the sum of the k winners IS the LDP code.
#pragma once

#include <cstdint>

namespace ldp {

constexpr int kTileW = 128;           // output columns per tile: 32 lanes x 4 columns
constexpr int kMaxSlots = 16;         // regions a tile may touch and still count in smem
constexpr uint32_t kKeyBase = 1u << 20;  // > 256 * max|m_i| = 979200

enum Mode { kLDP = 0, kLBP = 1 };

// One image of work, as the kernels see it.
struct Job {
    const uint8_t* img;
    int H, W, P;
    uint8_t* codes;  // nullptr: no code map
    int Pc;
    uint32_t* hist;  // R*C*nbins counters of this image, nullptr: no histogram
};

struct HistCfg {
    int R, C, nbins, compact;
};

__device__ __forceinline__ void cswap(uint32_t& a, uint32_t& b) {
    uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Sum of the K smallest of eight distinct keys.
template <int K>
__device__ __forceinline__ uint32_t sum_k_smallest(uint32_t (&k)[8]) {
    if constexpr (K == 3) {
        // pairs -> sorted lowest three of each half -> bitonic half-cleaner
        cswap(k[0], k[1]);
        cswap(k[2], k[3]);
        cswap(k[4], k[5]);
        cswap(k[6], k[7]);
        uint32_t e0 = min(k[0], k[2]), ex = max(k[0], k[2]), ey = min(k[1], k[3]);
        uint32_t e1 = min(ex, ey), e2 = max(ex, ey);
        uint32_t f0 = min(k[4], k[6]), fx = max(k[4], k[6]), fy = min(k[5], k[7]);
        uint32_t f1 = min(fx, fy), f2 = max(fx, fy);
        return min(e0, f2) + min(e1, f1) + min(e2, f0);
    } else {
        // Batcher odd-even merge sort of 8; unused comparator halves are
        // removed by the compiler.
        cswap(k[0], k[1]); cswap(k[2], k[3]); cswap(k[4], k[5]); cswap(k[6], k[7]);
        cswap(k[0], k[2]); cswap(k[1], k[3]); cswap(k[4], k[6]); cswap(k[5], k[7]);
        cswap(k[1], k[2]); cswap(k[5], k[6]);
        cswap(k[0], k[4]); cswap(k[1], k[5]); cswap(k[2], k[6]); cswap(k[3], k[7]);
        cswap(k[2], k[4]); cswap(k[3], k[5]);
        cswap(k[1], k[2]); cswap(k[3], k[4]); cswap(k[5], k[6]);
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) s += k[i];
        return s;
    }
}

// LDP code of one pixel from its three-sums (Eq. 1-3).
template <int K>
__device__ __forceinline__ uint32_t ldp_code(const int (&s3)[8], int s8) {
    const int nb = s8 * -768;
    uint32_t key[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) key[i] = (kKeyBase + (1u << i)) - (uint32_t)abs(s3[i] * 2048 + nb);
    return sum_k_smallest<K>(key) & 0xFFu;
}

// Bytes at columns v..v+5 of one image row as ints (zero past column W-1).
__device__ __forceinline__ void load_row6(const uint8_t* __restrict__ row, int v, int W, bool fast,
                                          int (&b)[6]) {
    if (fast) {
        uint32_t w0 = __ldg(reinterpret_cast<const unsigned int*>(row + v));
        uint32_t w1 = __ldg(reinterpret_cast<const unsigned short*>(row + v + 4));
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = (int)__byte_perm(w0, 0u, 0x4440u + j);
        b[4] = (int)(w1 & 0xFFu);
        b[5] = (int)(w1 >> 8);
    } else {
#pragma unroll
        for (int j = 0; j < 6; ++j) b[j] = (v + j < W) ? (int)__ldg(row + v + j) : 0;
    }
}

__device__ __forceinline__ int band_of(int x, int n, int nb) {
    // index of the band [floor(b*n/nb), floor((b+1)*n/nb)) holding x: floor((nb*x + nb - 1) / n)
    uint64_t num = (uint64_t)nb * (uint64_t)x + (uint64_t)(nb - 1);
    if (num < 0xFFFFFFFFull) return (int)((uint32_t)num / (uint32_t)n);
    return (int)(num / (uint64_t)n);
}

__device__ __forceinline__ int binom_small(int n, int r) {
    // C(n, r) for 0 <= n < 8, computed exactly
    if (r < 0 || r > n) return 0;
    int c = 1;
    for (int i = 1; i <= r; ++i) c = c * (n - r + i) / i;
    return c;
}

// Position of a code among the codes with the same popcount, ascending:
// its colex rank sum_j C(b_j, j) over set bits b_1 < ... < b_k.
__device__ __forceinline__ int colex_rank(int code) {
    int r = 0, j = 0;
    for (int b = 0; b < 8; ++b)
        if (code >> b & 1) {
            ++j;
            r += binom_small(b, j);
        }
    return r;
}

__device__ __forceinline__ int bin_of(int code, const HistCfg& hc) {
    return hc.compact ? colex_rank(code) : code;
}

// Shared memory of one CTA.
template <int TH>
struct Smem {
    uint32_t hist[kMaxSlots * 256];
    int col[kTileW];  // per tile column: slot offset (smem) or rj (global)
    int row[TH];      // per tile row: slot offset (smem) or ri*C (global)
    int geo[8];       // ri_lo, rj_lo, ncs, nslots, use_smem
    Job job;          // persistent kernel: current image
    int tile_u0, tile_v0, next;
};

// Processes one TH x 128 output tile at (u0, v0) of image `jb`.
// All threads of the CTA must call it (it synchronises).
template <int MODE, int K, int RPW, int NWARPS, bool HIST>
__device__ __forceinline__ void process_tile(const Job& jb, const HistCfg& hc, int u0, int v0,
                                             Smem<RPW * NWARPS>& sm) {
    constexpr int TH = RPW * NWARPS;
    constexpr int NT = NWARPS * 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int H = jb.H, W = jb.W;

    bool use_smem = true;
    if constexpr (HIST) {
        if (tid == 0) {
            const int x_last = min(u0 + TH, H - 2), y_last = min(v0 + kTileW, W - 2);
            const int ri_lo = band_of(u0 + 1, H, hc.R), ri_hi = band_of(x_last, H, hc.R);
            const int rj_lo = band_of(v0 + 1, W, hc.C), rj_hi = band_of(y_last, W, hc.C);
            const int ncs = rj_hi - rj_lo + 1, nslots = (ri_hi - ri_lo + 1) * ncs;
            sm.geo[0] = ri_lo;
            sm.geo[1] = rj_lo;
            sm.geo[2] = ncs;
            sm.geo[3] = nslots;
            sm.geo[4] = nslots <= kMaxSlots;
        }
        __syncthreads();
        const int ri_lo = sm.geo[0], rj_lo = sm.geo[1], ncs = sm.geo[2], nslots = sm.geo[3];
        use_smem = sm.geo[4] != 0;
        for (int j = tid; j < kTileW; j += NT) {
            const int y = v0 + 1 + j;
            int val;
            if (y <= W - 2) {
                const int rj = band_of(y, W, hc.C);
                val = use_smem ? (rj - rj_lo) * 256 : rj;
            } else {
                val = 0;  // column past the interior: never counted
            }
            sm.col[j] = val;
        }
        for (int i = tid; i < TH; i += NT) {
            const int x = u0 + 1 + i;
            int val = 0;
            if (x <= H - 2) {
                const int ri = band_of(x, H, hc.R);
                val = use_smem ? (ri - ri_lo) * ncs * 256 : ri * hc.C;
            }
            sm.row[i] = val;
        }
        if (use_smem)
            for (int e = tid; e < nslots * 256; e += NT) sm.hist[e] = 0;
        __syncthreads();
    }

    const int v = v0 + 4 * lane;
    const int ub = u0 + warp * RPW;
    const int ue = min(ub + RPW, H - 2);
    if (v < W - 2 && ub < ue) {
        const bool img_al = ((reinterpret_cast<uintptr_t>(jb.img) | (uintptr_t)jb.P) & 3u) == 0;
        const bool fast_ld = img_al && (v + 6 <= W);
        const bool cod_al = jb.codes != nullptr &&
                            ((reinterpret_cast<uintptr_t>(jb.codes) | (uintptr_t)jb.Pc) & 3u) == 0;
        const bool fast_st = cod_al && (v + 4 <= W - 2);
        const int nvalid = min(4, W - 2 - v);
        bool valid[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) valid[t] = t < nvalid;
        int colb[4];
        if constexpr (HIST) {
#pragma unroll
            for (int t = 0; t < 4; ++t) colb[t] = sm.col[4 * lane + t];
        }
        const uint8_t* rp = jb.img + (size_t)ub * (size_t)jb.P;
        int A[6], B[6], Cc[6];
        load_row6(rp, v, W, fast_ld, A);
        load_row6(rp + jb.P, v, W, fast_ld, B);
        // row three-sums X[t] + X[t+1] + X[t+2] of the top and middle rows
        int hsA[4], hsB[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            hsA[t] = A[t] + A[t + 1] + A[t + 2];
            hsB[t] = B[t] + B[t + 1] + B[t + 2];
        }
        rp += 2 * (size_t)jb.P;
#pragma unroll 2
        for (int u = ub; u < ue; ++u, rp += jb.P) {
            load_row6(rp, v, W, fast_ld, Cc);
            int hsC[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) hsC[t] = Cc[t] + Cc[t + 1] + Cc[t + 2];
            uint32_t code[4];
            if constexpr (MODE == kLDP) {
                int V[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) V[j] = A[j] + B[j] + Cc[j];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    int s3[8];
                    s3[0] = V[t + 2];
                    s3[1] = B[t + 2] + A[t + 2] + A[t + 1];
                    s3[2] = hsA[t];
                    s3[3] = A[t + 1] + A[t] + B[t];
                    s3[4] = V[t];
                    s3[5] = B[t] + Cc[t] + Cc[t + 1];
                    s3[6] = hsC[t];
                    s3[7] = Cc[t + 1] + Cc[t + 2] + B[t + 2];
                    const int s8 = V[t] + V[t + 2] + A[t + 1] + Cc[t + 1];
                    code[t] = ldp_code<K>(s3, s8);
                }
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int c = B[t + 1];
                    code[t] = (uint32_t)(B[t + 2] >= c) | ((uint32_t)(A[t + 2] >= c) << 1) |
                              ((uint32_t)(A[t + 1] >= c) << 2) | ((uint32_t)(A[t] >= c) << 3) |
                              ((uint32_t)(B[t] >= c) << 4) | ((uint32_t)(Cc[t] >= c) << 5) |
                              ((uint32_t)(Cc[t + 1] >= c) << 6) | ((uint32_t)(Cc[t + 2] >= c) << 7);
                }
            }
            if (jb.codes) {
                uint8_t* cp = jb.codes + (size_t)u * (size_t)jb.Pc + v;
                if (fast_st) {
                    const uint32_t p01 = __byte_perm(code[0], code[1], 0x0040u);
                    const uint32_t p23 = __byte_perm(code[2], code[3], 0x0040u);
                    *reinterpret_cast<uint32_t*>(cp) = __byte_perm(p01, p23, 0x5410u);
                } else {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (valid[t]) cp[t] = (uint8_t)code[t];
                }
            }
            if constexpr (HIST) {
                const int rowb = sm.row[u - u0];
                if (use_smem) {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (valid[t]) atomicAdd(&sm.hist[rowb + colb[t] + (int)code[t]], 1u);
                } else {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (valid[t])
                            atomicAdd(&jb.hist[(size_t)(rowb + colb[t]) * hc.nbins + bin_of((int)code[t], hc)], 1u);
                }
            }
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                A[j] = B[j];
                B[j] = Cc[j];
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                hsA[t] = hsB[t];
                hsB[t] = hsC[t];
            }
        }
    }

    if constexpr (HIST) {
        __syncthreads();
        if (use_smem) {
            const int ri_lo = sm.geo[0], rj_lo = sm.geo[1], ncs = sm.geo[2], nslots = sm.geo[3];
            for (int e = tid; e < nslots * 256; e += NT) {
                const uint32_t c = sm.hist[e];
                if (c) {
                    const int slot = e >> 8, code = e & 255;
                    const int ri = ri_lo + slot / ncs, rj = rj_lo + slot % ncs;
                    atomicAdd(&jb.hist[(size_t)(ri * hc.C + rj) * hc.nbins + bin_of(code, hc)], c);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace ldp
