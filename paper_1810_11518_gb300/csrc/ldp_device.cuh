// Device building blocks for LDP / LBP extraction on sm_103a.
//
// Per pixel (Sec. 2.2.1-2.2.2, Eq. 1-3): every Kirsch mask weighs three
// consecutive ring neighbours by 5 and the other five by -3, so
//     m_i = 8*S3_i - 3*S8,   S3_i = p_{i-1} + p_i + p_{i+1},  S8 = sum_j p_j
// (ring p_0..p_7 counter-clockwise from East).  The eight S3_i and S8 are
// built from column and row sums shared between neighbouring pixels.
//
// LDP arithmetic is exact integer arithmetic on two pixels at once: every
// 32-bit word holds two 16-bit lanes (pixel columns y and y+2), the sums are
// plain 32-bit adds of such words and the selection is 16x2 SIMD min/max.
// With p = S8 mod 2 (all m_i share the parity of S8) and C = 3824 + p,
//     a_i = 8C - 8 m_i,   b_i = 8C + 8 m_i,   key_i = min(a_i, b_i) + i
//         = 8 (C - |m_i|) + i
// lies in [0, 30607]; a_i and b_i stay in [0, 61200], so neither ever leaves
// its 16-bit lane, and the words are exact although intermediate terms may
// carry between the lanes (everything before the min is linear mod 2^32).
// Keys order like |m_i| descending with ties to the lower index, bits 0..2
// hold i and bit 3 is 0 (C - |m_i| is even).  The k smallest keys are the k
// most outstanding responses; a byte_perm with the keys' low bytes as its
// selector turns each winner's index into the one-hot bit 2^i.
#pragma once

#include <cstdint>
#include <type_traits>

#include "ldp_modes.h"

namespace ldp {

constexpr int kTileW = 128;           // output columns per tile: 32 lanes x 4 columns
constexpr int kMaxSlots = 16;         // regions a tile may touch and still count in smem



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

// 16x2 SIMD min / max of two words of 16-bit lanes.
__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// byte_perm with the hardware's full selector semantics: a selector nibble
// with bit 3 set replicates the sign of the chosen byte.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// The M best of eight keys per lane (SMALL: the M smallest, else the M
// largest), unordered, in w[0..M-1].  Each half of four is reduced to its M
// best in order; a bitonic half-cleaner then keeps the M best of both.
template <int M, bool SMALL>
__device__ __forceinline__ void select_best(const uint32_t (&k)[8], uint32_t (&w)[4]) {
    auto lo = [](uint32_t a, uint32_t b) { return SMALL ? vmin2(a, b) : vmax2(a, b); };
    auto hi = [](uint32_t a, uint32_t b) { return SMALL ? vmax2(a, b) : vmin2(a, b); };
    if constexpr (M == 1) {
        w[0] = lo(lo(lo(k[0], k[1]), lo(k[2], k[3])), lo(lo(k[4], k[5]), lo(k[6], k[7])));
    } else {
        uint32_t e[4], f[4];
        auto half = [&](const uint32_t* x, uint32_t(&o)[4]) {
            const uint32_t a0 = lo(x[0], x[1]), a1 = hi(x[0], x[1]);
            const uint32_t a2 = lo(x[2], x[3]), a3 = hi(x[2], x[3]);
            o[0] = lo(a0, a2);
            const uint32_t ex = hi(a0, a2), ey = lo(a1, a3);
            o[1] = lo(ex, ey);
            o[2] = hi(ex, ey);
            o[3] = hi(a1, a3);
        };
        half(k, e);
        half(k + 4, f);
#pragma unroll
        for (int i = 0; i < M; ++i) w[i] = lo(e[i], f[M - 1 - i]);
    }
}

// Codes of the two pixels of a pair of 16-bit lanes from their M best keys:
// bytes 0 and 2 of the result (bytes 1 and 3 are don't-care).
template <int K>
__device__ __forceinline__ uint32_t code_pair(const uint32_t (&key)[8]) {
    constexpr bool kSmall = K <= 4;
    constexpr int M = kSmall ? K : 8 - K;
    uint32_t w[4];
    select_best<M, kSmall>(key, w);
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        // selector nibble 0 = lane 0's index, nibble 2 = lane 1's (bit 3 of
        // both is 0); the table bytes are 1, 2, 4, ..., 128
        const uint32_t sel = prmt(w[j], 0u, 0x3120u);
        acc |= prmt(0x08040201u, 0x80402010u, sel);
    }
    return kSmall ? acc : ~acc;  // for k >= 5 the M largest keys are the losers
}

// The six bytes v..v+5 of one image row a thread needs: w0 = bytes v..v+3,
// w1 = bytes v+4, v+5 in its low half.  Columns past W-1 read as 0.
struct Raw {
    uint32_t w0, w1;
};

__device__ __forceinline__ Raw load_raw(const uint8_t* __restrict__ row, int v, int W, bool fast) {
    Raw r;
    if (fast) {
        r.w0 = __ldg(reinterpret_cast<const unsigned int*>(row + v));
        r.w1 = __ldg(reinterpret_cast<const unsigned short*>(row + v + 4));
    } else {
        uint32_t b[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) b[j] = (v + j < W) ? (uint32_t)__ldg(row + v + j) : 0u;
        r.w0 = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
        r.w1 = b[4] | (b[5] << 8);
    }
    return r;
}

// Threshold reading of Eq. 2-3 for a pair of lanes: t = the K-th smallest
// key (Batcher's odd-even merge sort of eight, pruned to what s[K-1] needs);
// every direction whose key is at most t | 7 -- the same ranking value as
// the K-th or a better one, whatever its index -- is set.  Bytes 0 and 2.
template <int K>
__device__ __forceinline__ uint32_t code_thresh(const uint32_t (&key)[8]) {
    uint32_t s[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] = key[i];
    auto cs = [](uint32_t& a, uint32_t& b) {
        const uint32_t lo = vmin2(a, b), hi = vmax2(a, b);
        a = lo;
        b = hi;
    };
    cs(s[0], s[1]); cs(s[2], s[3]); cs(s[4], s[5]); cs(s[6], s[7]);
    cs(s[0], s[2]); cs(s[1], s[3]); cs(s[4], s[6]); cs(s[5], s[7]);
    cs(s[1], s[2]); cs(s[5], s[6]);
    cs(s[0], s[4]); cs(s[1], s[5]); cs(s[2], s[6]); cs(s[3], s[7]);
    cs(s[2], s[4]); cs(s[3], s[5]);
    cs(s[1], s[2]); cs(s[3], s[4]); cs(s[5], s[6]);
    const uint32_t t = s[K - 1] | 0x00070007u;
    const uint32_t t0 = t & 0xFFFFu, t1 = t >> 16;
    uint32_t c0 = 0, c1 = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        c0 |= (uint32_t)((key[i] & 0xFFFFu) <= t0) << i;
        c1 |= (uint32_t)((key[i] >> 16) <= t1) << i;
    }
    return c0 | (c1 << 16);
}

// One image row restricted to the six columns v..v+5 a thread needs, in
// pairs of 16-bit lanes: P[j] = (byte v+j, byte v+j+2), j = 0..3, and the row
// three-sums T[c] = P[c] + P[c+1] + P[c+2], centred on columns v+1+c, v+3+c.
struct SRow {
    uint32_t P[4], T[2];
};

__device__ __forceinline__ void unpack_srow(const Raw& w, SRow& r) {
    // source bytes 0..3 = columns v..v+3 (w0), 4..5 = v+4, v+5 (w1), 6..7 = 0
    r.P[0] = __byte_perm(w.w0, w.w1, 0x6260u);
    r.P[1] = __byte_perm(w.w0, w.w1, 0x6361u);
    r.P[2] = __byte_perm(w.w0, w.w1, 0x6462u);
    r.P[3] = __byte_perm(w.w0, w.w1, 0x6563u);
    r.T[0] = r.P[0] + r.P[1] + r.P[2];
    r.T[1] = r.P[1] + r.P[2] + r.P[3];
}

// LBP row in byte-SIMD form: s[d] holds bytes v+d..v+d+3 (d = 0, 1, 2), i.e.
// the row's pixel at column offset d for the four output pixels.
struct BRow {
    uint32_t s[3];
};

__device__ __forceinline__ void unpack_brow(const Raw& w, BRow& r) {
    r.s[0] = w.w0;
    r.s[1] = __byte_perm(w.w0, w.w1, 0x4321u);
    r.s[2] = __byte_perm(w.w0, w.w1, 0x5432u);
}

// Per byte lane: bit 7 set iff x >= y (unsigned).  (x | 0x80) - (y & 0x7f)
// never borrows across lanes and its bit 7 is [x_low7 >= y_low7]; where the
// top bits of x and y differ, x's top bit decides instead.
__device__ __forceinline__ uint32_t bytes_ge(uint32_t x, uint32_t y_low7) {
    return (x | 0x80808080u) - y_low7;
}

// LBP codes of four pixels (Sec. 2.1), one per byte lane.
__device__ __forceinline__ uint32_t lbp_row4(const BRow& A, const BRow& B, const BRow& C) {
    const uint32_t c = B.s[1];  // centres
    const uint32_t cl = c & 0x7F7F7F7Fu;
    const uint32_t nb[8] = {B.s[2], A.s[2], A.s[1], A.s[0], B.s[0], C.s[0], C.s[1], C.s[2]};  // p_0..p_7
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // bit j inserted at bit 7, then shifted down 7-j times
        const uint32_t x = nb[j];
        const uint32_t t = bytes_ge(x, cl);
        // bit 7 of each lane: x and c agree in bit 7 ? t : x
        const uint32_t ge = (((x ^ c) & x) | (~(x ^ c) & t)) & 0x80808080u;
        // shift the lanes' bits so far down by one and insert bit j at bit 7
        acc = ((acc >> 1) & 0x7F7F7F7Fu) | ge;
    }
    return acc;
}

// Codes of the two pixels of lane pair c (c = 0: columns v+1, v+3; c = 1:
// columns v+2, v+4) of one output row, from rows A (x-1), B (x), C (x+1) and
// the column three-sums V; bytes 0 and 2 of the result.
template <int K, int MODE, int c>
__device__ __forceinline__ uint32_t ldp_pair(const SRow& A, const SRow& B, const SRow& C, const uint32_t (&V)[4]) {
    constexpr bool kRaw = MODE == kLDPRaw || MODE == kLDPRawThresh;
    constexpr int L = c, M = c + 1, R = c + 2;  // west, centre and east columns of the pair
    const uint32_t S3[8] = {
        V[R],                       // E : p7 + p0 + p1
        B.P[R] + A.P[R] + A.P[M],   // NE: p0 + p1 + p2
        A.T[c],                     // N : p1 + p2 + p3
        A.P[M] + A.P[L] + B.P[L],   // NW: p2 + p3 + p4
        V[L],                       // W : p3 + p4 + p5
        B.P[L] + C.P[L] + C.P[M],   // SW: p4 + p5 + p6
        C.T[c],                     // S : p5 + p6 + p7
        C.P[M] + C.P[R] + B.P[R]};  // SE: p6 + p7 + p0
    const uint32_t S8 = A.T[c] + C.T[c] + B.P[L] + B.P[R];
    const uint32_t Q = (S8 & 0x00010001u) * 8u + 30592u * 0x00010001u;  // 8C per lane, C = 3824 + p
    const uint32_t Za = Q + S8 * 24u, Zb = Q - S8 * 24u;               // 8C + 24 S8, 8C - 24 S8
    uint32_t key[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        // a = 8C - 8 m_i, b = 8C + 8 m_i: one multiply-add each (FMA pipe),
        // the min and the tie index i on the ALU.  Ranking the signed m_i
        // (kRaw) the key is a + i = 8 (C - m_i) + i, in [0, 61207].
        uint32_t a, b;
        asm("mad.lo.u32 %0, %1, -64, %2;" : "=r"(a) : "r"(S3[i]), "r"(Za));
        if constexpr (kRaw) {
            key[i] = a + (uint32_t)i * 0x00010001u;
        } else {
            asm("mad.lo.u32 %0, %1, 64, %2;" : "=r"(b) : "r"(S3[i]), "r"(Zb));
            key[i] = vmin2(a, b) + (uint32_t)i * 0x00010001u;
        }
    }
    if constexpr (exact_k(MODE))
        return code_pair<K>(key);
    else
        return code_thresh<K>(key);
}

// Codes of the four pixels of one output row (byte t = column v+t).
template <int K, int MODE>
__device__ __forceinline__ uint32_t ldp_row4(const SRow& A, const SRow& B, const SRow& C) {
    uint32_t V[4];  // column three-sums
#pragma unroll
    for (int j = 0; j < 4; ++j) V[j] = A.P[j] + B.P[j] + C.P[j];
    const uint32_t c02 = ldp_pair<K, MODE, 0>(A, B, C, V), c13 = ldp_pair<K, MODE, 1>(A, B, C, V);
    return __byte_perm(c02, c13, 0x6240u);
}

// Band b of nb bands over n pixels covers [floor(b*n/nb), floor((b+1)*n/nb));
// pixel x lies in band floor((nb*x + nb - 1) / n).
__device__ __forceinline__ int band_of(int x, int n, int nb) {
    uint64_t num = (uint64_t)nb * (uint64_t)x + (uint64_t)(nb - 1);
    if (num < 0xFFFFFFFFull) return (int)((uint32_t)num / (uint32_t)n);
    return (int)(num / (uint64_t)n);
}

// Compact bin of every code, per k (Eq. 6: ascending code value among the
// C(8,k) codes with popcount k); -1 for other popcounts.  Built at compile
// time as the colex rank sum_j C(b_j, j) over set bits b_1 < ... < b_k.
struct BinTable {
    int16_t bin[9][256];
};

__host__ __device__ constexpr int binom_ce(int n, int r) {
    if (r < 0 || r > n) return 0;
    int c = 1;
    for (int i = 1; i <= r; ++i) c = c * (n - r + i) / i;
    return c;
}

constexpr BinTable make_bin_table() {
    BinTable t{};
    for (int k = 0; k < 9; ++k)
        for (int code = 0; code < 256; ++code) {
            int pop = 0, r = 0;
            for (int b = 0; b < 8; ++b)
                if (code >> b & 1) {
                    ++pop;
                    r += binom_ce(b, pop);
                }
            t.bin[k][code] = (int16_t)(pop == k ? r : -1);
        }
    return t;
}

static __device__ const BinTable g_bin_table = make_bin_table();

// The C(8,k) codes with popcount k in ascending order (Eq. 6), per k.
struct CodeList {
    uint8_t code[9][70];
};

constexpr CodeList make_code_list() {
    CodeList l{};
    for (int k = 0; k < 9; ++k) {
        int n = 0;
        for (int code = 0; code < 256; ++code) {
            int pop = 0;
            for (int b = 0; b < 8; ++b) pop += (code >> b) & 1;
            if (pop == k) l.code[k][n++] = (uint8_t)code;
        }
    }
    return l;
}

static __device__ const CodeList g_code_list = make_code_list();

__device__ __forceinline__ int bin_of(int code, const HistCfg& hc, int k) {
    return hc.compact ? (int)__ldg(&g_bin_table.bin[k][code]) : code;
}

constexpr int kWarpSlots = 6;  // region slots a warp tile may touch and still count in smem
// shared 256-bin slots of a warp's histogram: LBP adds a junk slot that takes
// the counts of columns past the interior (LBP produces every code, so no
// bin of a counted slot is free for them)
template <int MODE>
__host__ __device__ constexpr int warp_hist_slots() { return is_ldp(MODE) ? kWarpSlots : kWarpSlots + 1; }

// Staged input (bulk-copy engine): per warp a ring of kStages stages of
// kStageRows image rows, kRowBytes bytes each (the 130 bytes a 128-column
// tile reads, rounded up to 16), filled by cp.async.bulk and completed on one
// mbarrier per stage.
constexpr int kStageRows = 8, kStages = 3, kRowBytes = 144;
constexpr int kSpinLimit = 1 << 22;  // bounded mbarrier waits
constexpr int kTestSpinLimit = 256;  // checked builds: the wait of a withheld stage (test hook)

// Checked builds (-DLDP_CHECKED) test every shared- and global-memory index
// of the tile loop (and of the window and resize kernels) against its buffer;
// a violation sets kStatusBounds in the device status word and the access is
// skipped (nothing traps).  In normal builds the test is compiled away.
__device__ __forceinline__ bool index_ok(bool ok, int* status) {
#ifdef LDP_CHECKED
    if (!ok) atomicOr(status, kStatusBounds);
    return ok;
#else
    (void)status;
    (void)ok;
    return true;
#endif
}

struct WarpRing {
    alignas(128) uint8_t row[kStages][kStageRows][kRowBytes];
    alignas(8) unsigned long long bar[kStages];
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Lane 0 of each warp initialises the warp's ring barriers (once per kernel).
__device__ __forceinline__ void ring_init(WarpRing* ring) {
    if ((threadIdx.x & 31) == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&ring->bar[s], 1);
        mbar_fence_init();
    }
    __syncwarp();
}

// Lower bound of band b: floor(b*n/nb).
__device__ __forceinline__ int band_lo(int b, int n, int nb) {
    return (int)(((uint64_t)b * (uint64_t)n) / (uint64_t)nb);
}

// Flush of a warp's shared histogram slots [0, nsl): slot sl holds region
// row ri_first + sl / ncs, region column rj_lo + sl % ncs.  Every non-zero
// bin of a code that can occur is added to the global histogram and reset
// (the C(8,k) codes with popcount k for the exact-k LDP modes, bin = position
// in the code list when compact, the code itself when raw; every code but 0
// for the LDP threshold modes, whose code 0 holds the skipped columns; all
// 256 for LBP).  Warp-collective.
template <int MODE, int K>
__device__ __forceinline__ void flush_slots(const Job& jb, const HistCfg& hc, uint32_t* wh, int ri_first,
                                            int rj_lo, int ncs, int nsl, int* status) {
    const int lane = threadIdx.x & 31;
    asm volatile("" ::: "memory");  // the reductions into wh come first
    __syncwarp();
    constexpr int NC = exact_k(MODE) ? binom_ce(8, K) : 256;
    constexpr int NI = (NC + 31) / 32;
    int code_of[NI];
#pragma unroll
    for (int m = 0; m < NI; ++m) {
        const int idx = lane + 32 * m;
        code_of[m] = exact_k(MODE) ? (idx < NC ? (int)__ldg(&g_code_list.code[K][idx]) : -1)
                                   : ((is_ldp(MODE) && idx == 0) ? -1 : idx);
    }
    for (int sl = 0; sl < nsl; ++sl) {
        const int hbase = ((ri_first + sl / ncs) * hc.C + rj_lo + sl % ncs) * hc.nbins;
        uint32_t* hs = wh + sl * 256;
#pragma unroll
        for (int m = 0; m < NI; ++m) {
            const int code = code_of[m];
            if (code >= 0) {
                const uint32_t c = hs[code];
                if (c) {
                    const int bin = (exact_k(MODE) && hc.compact) ? lane + 32 * m : code;
                    if (index_ok(hbase + bin < hc.R * hc.C * hc.nbins, status)) atomicAdd(&jb.hist[hbase + bin], c);
                    hs[code] = 0;
                }
            }
        }
    }
    __syncwarp();
}

// One warp processes one tile of RW output rows x 128 output columns at
// (u0, v0): lane l owns columns v0+4l .. v0+4l+3 and walks down the rows.
// Input rows come either from per-lane global loads one row ahead, or
// (STAGED, for 16-byte aligned images) from the warp's bulk-copy ring, two
// stages ahead.  With HIST the codes are counted in the warp's private shared
// histogram `wh` (kWarpSlots x 256 raw bins, one slot per region the counts
// go to; every bin the flush reads is zero on entry and on exit): the flush
// adds every non-zero bin to the global histogram and resets it.  A slot per
// (region row, region column) of the tile is kept until the tile ends; with
// RSLOTS (per-lane loads, neither STAGED nor SPLIT) the slots hold the
// region columns of the current region row only: the rows are walked in
// segments that end at region-row boundaries and the slots are flushed
// there, so a tile that crosses many region rows of a small image still
// counts in shared memory.  In the LDP modes bin 0 of a slot (code 0, which
// they never produce) takes the counts of columns past the interior and is
// never read; LBP has a junk slot for them.
// Region grids too fine for kWarpSlots slots count straight into global
// memory.  `ph` holds the ring's per-stage wait parities across tiles.
template <int MODE, int K, int RW, bool HIST, bool STAGED, bool SPLIT, bool RSLOTS>
__device__ __forceinline__ void warp_tile(const Job& jb, const HistCfg& hc, int u0, int v0, uint32_t* wh,
                                          WarpRing* ring, uint32_t& ph, int* status) {
    const int lane = threadIdx.x & 31;
    const int H = jb.H, W = jb.W;
    const int ue = min(u0 + RW, H - 2);  // output rows [u0, ue) = image rows [u0+1, ue]
    // SPLIT: a tile narrower than 64 columns (an image's last column tile)
    // shares its rows between lane groups: lp lanes per row (a power of two
    // covering its four-column groups), 32 / lp groups of consecutive rows.
    // This lane's output rows are [ul, uh); otherwise all of the tile's.
    int ul = u0, uh = ue, lc = lane;
    if constexpr (SPLIT && !STAGED) {
        const int ng = (min(kTileW, W - 2 - v0) + 3) / 4;
        if (ng <= 16) {
            const int lp = ng > 8 ? 16 : ng > 4 ? 8 : ng > 2 ? 4 : ng > 1 ? 2 : 1;
            const int groups = 32 / lp, len = (ue - u0 + groups - 1) / groups;
            ul = min(u0 + (lane / lp) * len, ue);
            uh = min(ul + len, ue);
            lc = lane % lp;
        }
    }
    const int v = v0 + 4 * lc;
    // slots per region column of the current region row, flushed at each
    // region-row boundary (else: per region of the tile, flushed at its end)
    constexpr bool kRowSlots = RSLOTS && !STAGED && !SPLIT;

    // region slots of the tile (uniform across the warp)
    int ri_lo = 0, rj_lo = 0, ncs = 1, nslots = 1;
    bool use_smem = true;
    if constexpr (HIST) {
        ri_lo = band_of(u0 + 1, H, hc.R);
        rj_lo = band_of(v0 + 1, W, hc.C);
        ncs = band_of(min(v0 + kTileW, W - 2), W, hc.C) - rj_lo + 1;
        nslots = kRowSlots ? ncs : (band_of(ue, H, hc.R) - ri_lo + 1) * ncs;
        use_smem = nslots <= kWarpSlots;
    }

    const size_t P = (size_t)jb.P;
    // the ring holds bytes v0 .. v0+nbytes of every input row; the bulk-copy
    // engine fills rows when the image is 16-byte aligned, except the last
    // image row when it would read past W (no pitch padding is guaranteed
    // there); such rows are copied by the warp with plain loads
    const int nbytes = min(kRowBytes, (W - v0 + 15) & ~15);
    const bool bulk_img = ((reinterpret_cast<uintptr_t>(jb.img) | P) & 15u) == 0;
    constexpr bool staged = STAGED;

    const bool img_al = ((reinterpret_cast<uintptr_t>(jb.img) | P) & 3u) == 0;
    const bool fast_ld = img_al && (v + 6 <= W);
    const bool cod_al =
        jb.codes != nullptr && ((reinterpret_cast<uintptr_t>(jb.codes) | (uintptr_t)jb.Pc) & 3u) == 0;
    const bool fast_st = cod_al && (v + 4 <= W - 2);
    bool valid[4];
    int colb[4];  // per column: slot offset (smem) or region column (global)
    // byte_perm selector of column t's code for the shared histogram; a
    // column past the interior reads a zero byte instead: code 0 never occurs
    // in the LDP modes (at least one bit is set), so its bin is never flushed
    // and the count needs no branch
    uint32_t csel[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        valid[t] = v + t < W - 2;
        csel[t] = valid[t] ? (0x4440u | (uint32_t)t) : 0x4444u;
        colb[t] = 0;
        if (HIST && valid[t]) {
            const int rj = band_of(v + t + 1, W, hc.C);
            colb[t] = use_smem ? (rj - rj_lo) * 256 : rj;
        }
    }
    // region row of image row x = u + 1, advanced as the rows go down
    int ri = ri_lo, next_b = 0, rowb = 0;
    if constexpr (HIST && SPLIT && !STAGED) ri = band_of(ul + 1, H, hc.R);
    // shared-memory byte address of bin 0 of each column's current slot
    uint32_t sbase[4] = {0u, 0u, 0u, 0u};
    const uint32_t wh_addr = HIST && use_smem && is_ldp(MODE) ? smem_addr(wh) : 0u;
    // LBP: word index of bin 0 of each column's current slot (the junk slot
    // for columns past the interior)
    int lbase[4] = {0, 0, 0, 0};
    auto set_sbase = [&]() {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if constexpr (is_ldp(MODE))
                sbase[t] = wh_addr + 4u * (uint32_t)(rowb + colb[t]);
            else
                lbase[t] = valid[t] ? rowb + colb[t] : kWarpSlots * 256;
        }
    };
    if constexpr (HIST) {
        next_b = band_lo(ri + 1, H, hc.R);
        if constexpr (SPLIT && !STAGED)
            rowb = use_smem ? (ri - ri_lo) * ncs * 256 : ri * hc.C;
        else
            rowb = use_smem ? 0 : ri * hc.C;
        if (use_smem) set_sbase();
    }

    // codes of output row u (byte t of `packed` = column v+t) -> code map and histogram
    auto emit = [&](int u, uint32_t packed) {
        if (jb.codes && index_ok(u >= 0 && u < H - 2, status)) {
            uint8_t* cp = jb.codes + (size_t)u * (size_t)jb.Pc + v;
            if (fast_st) {
                if (index_ok(v + 3 < W - 2, status)) *reinterpret_cast<uint32_t*>(cp) = packed;
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (valid[t]) cp[t] = (uint8_t)(packed >> (8 * t));
            }
        }
        if constexpr (HIST && !kRowSlots) {
            while (u + 1 >= next_b) {  // crossed into the next region row
                ++ri;
                next_b = band_lo(ri + 1, H, hc.R);
                rowb = use_smem ? (ri - ri_lo) * ncs * 256 : ri * hc.C;
                if (use_smem) set_sbase();
            }
        }
        if constexpr (HIST) {
            if (use_smem && is_ldp(MODE)) {
                // LDP codes spread over the bins: one byte extract, one
                // multiply-add for the address, one reduction per pixel
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint32_t code = prmt(packed, 0u, csel[t]);
                    uint32_t addr;
                    asm("mad.lo.u32 %0, %1, 4, %2;" : "=r"(addr) : "r"(code), "r"(sbase[t]));
                    if (index_ok(addr - wh_addr < 4u * kWarpSlots * 256u, status))
                        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
                }
            } else if (use_smem) {
                // LBP: neighbouring lanes often share a code (flat areas give
                // 255); the compiler's shared atomicAdd is faster there
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int idx = lbase[t] + (int)((packed >> (8 * t)) & 0xFFu);
                    if (index_ok(idx < warp_hist_slots<MODE>() * 256, status)) atomicAdd(&wh[idx], 1u);
                }
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (valid[t]) {
                        const int code = (int)((packed >> (8 * t)) & 0xFFu);
                        const int bin = bin_of(code, hc, K);
                        if (index_ok(rowb + colb[t] < hc.R * hc.C && bin >= 0 && bin < hc.nbins, status))
                            atomicAdd(&jb.hist[(size_t)(rowb + colb[t]) * hc.nbins + bin], 1u);
                    }
            }
        }
    };
    auto codes_of_row = [&](const auto& A, const auto& B, const auto& C) -> uint32_t {
        if constexpr (is_ldp(MODE))
            return ldp_row4<K, MODE>(A, B, C);
        else
            return lbp_row4(A, B, C);
    };
    using Row = std::conditional_t<is_ldp(MODE), SRow, BRow>;
    auto unpack = [&](const Raw& w, Row& r) {
        if constexpr (is_ldp(MODE))
            unpack_srow(w, r);
        else
            unpack_brow(w, r);
    };

    if constexpr (staged) {
        // all lanes run the ring protocol; lanes past the interior compute
        // nothing that is stored or counted (valid[] is false)
        const int nrows = ue - u0 + 2;  // input rows u0 .. ue+1
        const uint8_t* base = jb.img + (size_t)u0 * P + v0;
        uint32_t pend = 0;  // stages filled and not yet waited
        bool ok = true;
#ifdef LDP_CHECKED
        // test hook (word 1 of the status word): stage group `withheld` is
        // never filled, so its bounded wait runs out with no copy in flight
        const int withheld = status[1];
#else
        constexpr int withheld = 0;
#endif
        auto fill = [&](int g) {
            const int r0 = g * kStageRows, n = min(kStageRows, nrows - r0);
            if (n <= 0 || (withheld > 0 && g == withheld)) return;
            const int sidx = g % kStages;
            // rows [r0, r0 + nb) go through the bulk-copy engine
            int nb = bulk_img ? n : 0;
            if (nb > 0 && u0 + r0 + nb - 1 == H - 1 && v0 + nbytes > W) --nb;
            __syncwarp();
            if (lane == 0) {
                fence_proxy_async();
                mbar_expect_tx(&ring->bar[sidx], (uint32_t)(nb * nbytes));  // 0 bytes: the phase completes now
            }
            __syncwarp();
            if (lane < nb) {
                fence_proxy_async();
                bulk_g2s(ring->row[sidx][lane], base + (size_t)(r0 + lane) * P, (uint32_t)nbytes, &ring->bar[sidx]);
            }
            for (int r = nb; r < n; ++r) {  // plain copies, zero past column W-1
                const uint8_t* src = base + (size_t)(r0 + r) * P;
                uint8_t* dst = ring->row[sidx][r];
                for (int b = lane; b < kRowBytes; b += 32) dst[b] = (v0 + b < W) ? __ldg(src + b) : (uint8_t)0;
            }
            __syncwarp();
            pend |= 1u << sidx;
        };
        auto wait = [&](int g) {
            const int sidx = g % kStages;
            const uint32_t par = (ph >> sidx) & 1u;
            const int limit = (withheld > 0 && g == withheld) ? kTestSpinLimit : kSpinLimit;
            bool done = false;
            for (int i = 0; i < limit && !done; ++i) done = mbar_try_wait(&ring->bar[sidx], par);
            if (done) {
                ph ^= 1u << sidx;
                pend &= ~(1u << sidx);
            } else {
                ok = false;
            }
        };
        auto read = [&](int ir) {
            const uint8_t* q = ring->row[(ir / kStageRows) % kStages][ir % kStageRows] + 4 * lane;
            Raw r;
            r.w0 = *reinterpret_cast<const uint32_t*>(q);
            r.w1 = *reinterpret_cast<const uint16_t*>(q + 4);
            return r;
        };
        for (int g = 0; g < kStages; ++g) fill(g);
        wait(0);
        Row r0, r1, r2;
        if (ok) {
            unpack(read(0), r0);
            unpack(read(1), r1);
        }
        auto step = [&](const Row& A, const Row& B, Row& C, int ou) {
            const int ir = ou + 2;  // input row that becomes C
            if (ir % kStageRows == 0) wait(ir / kStageRows);
            if (!ok) return;
            unpack(read(ir), C);
            if (ir % kStageRows == kStageRows - 1) fill(ir / kStageRows + kStages);  // stage fully read
            emit(u0 + ou, codes_of_row(A, B, C));
        };
        const int nout = ue - u0;
        int ou = 0;
        for (; ou + 3 <= nout && ok; ou += 3) {
            step(r0, r1, r2, ou);
            step(r1, r2, r0, ou + 1);
            step(r2, r0, r1, ou + 2);
        }
        if (ok && ou < nout) step(r0, r1, r2, ou);
        if (ok && ou + 1 < nout) step(r1, r2, r0, ou + 1);
        // every filled stage is consumed on the way; after a timeout, give the
        // copies still in flight a bounded chance to land before returning
        if (!ok || pend) {
            if (lane == 0) atomicOr(status, kStatusWaitTimeout);
            for (int sidx = 0; sidx < kStages; ++sidx)
                if (pend >> sidx & 1u) {
                    const uint32_t par = (ph >> sidx) & 1u;
                    bool done = false;
                    for (int i = 0; i < kSpinLimit && !done; ++i) done = mbar_try_wait(&ring->bar[sidx], par);
                    if (done) ph ^= 1u << sidx;
                }
        }
    } else if constexpr (kRowSlots) {  // per-lane global loads, one row ahead, in region-row segments
        // every lane walks the rows (lanes past the interior count into
        // bins the flush never reads), in segments of one region row
        const uint8_t* rp = jb.img + (size_t)u0 * P;
        const uint8_t* pf = rp + 3 * P;  // next input row to prefetch (one row ahead)
        Raw nx = load_raw(rp + 2 * P, v, W, fast_ld);
        // LBP does far less arithmetic per row than LDP: its input rows come
        // two ahead, the second one clamped to the image's last row (a spare
        // load there instead of a test)
        constexpr bool kTwoAhead = !is_ldp(MODE);
        const uint8_t* const last_row = jb.img + (size_t)(H - 1) * P;
        Raw nx2{};
        if constexpr (kTwoAhead) {
            nx2 = load_raw(u0 + 3 < H ? pf : last_row, v, W, fast_ld);
            pf += P;  // input row u0 + 4
        }
        Row r0, r1, r2;
        unpack(load_raw(rp, v, W, fast_ld), r0);
        unpack(load_raw(rp + P, v, W, fast_ld), r1);
        // ALWAYS: the next output row exists, so the prefetch needs no test
        auto step = [&](const Row& A, const Row& B, Row& C, int u, auto always) {
            unpack(nx, C);
            if constexpr (kTwoAhead) {
                nx = nx2;
                nx2 = load_raw(u + 4 < H ? pf : last_row, v, W, fast_ld);
            } else if (decltype(always)::value ? index_ok(u + 3 < H, status)
                                               : (u + 1 < ue && index_ok(u + 3 < H, status))) {
                nx = load_raw(pf, v, W, fast_ld);
            }
            pf += P;
            emit(u, codes_of_row(A, B, C));
        };
        const std::true_type yes;
        const std::false_type no;
        int u = u0;
        for (;;) {
            // rows [u, se) are image rows u+1 .. se of region row ri
            const int se = HIST ? min(ue, next_b - 1) : ue;
            for (const int lim = min(se, ue - 1); u + 3 <= lim; u += 3) {
                step(r0, r1, r2, u, yes);
                step(r1, r2, r0, u + 1, yes);
                step(r2, r0, r1, u + 2, yes);
            }
            // zero to three rows left in the segment
            int j = 0;
            if (u < se) {
                step(r0, r1, r2, u, no);
                j = 1;
                if (u + 1 < se) {
                    step(r1, r2, r0, u + 1, no);
                    j = 2;
                    if (u + 2 < se) {
                        step(r2, r0, r1, u + 2, no);
                        j = 3;
                    }
                }
            }
            u += j;
            if (u >= ue) break;
            // region-row boundary: flush the finished region row, move to
            // the one holding image row u+1, and bring the next two input
            // rows back to r0, r1
            if constexpr (HIST) {
                if (use_smem) flush_slots<MODE, K>(jb, hc, wh, ri, rj_lo, ncs, ncs, status);
            }
            while (u + 1 >= next_b) {
                ++ri;
                next_b = band_lo(ri + 1, H, hc.R);
            }
            if (!use_smem) rowb = ri * hc.C;
            if (j == 1) {
                r0 = r1;
                r1 = r2;
            } else if (j == 2) {
                const Row t = r0;
                r0 = r2;
                r1 = t;
            }
        }
    } else if (v < W - 2 && (!SPLIT || ul < uh)) {  // per-lane global loads, one row ahead
        const uint8_t* rp = jb.img + (size_t)ul * P;
        const uint8_t* pf = rp + 3 * P;  // next input row to prefetch (one row ahead)
        Raw nx = load_raw(rp + 2 * P, v, W, fast_ld);
        Row r0, r1, r2;
        unpack(load_raw(rp, v, W, fast_ld), r0);
        unpack(load_raw(rp + P, v, W, fast_ld), r1);
        // ALWAYS: the next output row exists, so the prefetch needs no test
        auto step = [&](const Row& A, const Row& B, Row& C, int u, auto always) {
            unpack(nx, C);
            if (decltype(always)::value ? index_ok(u + 3 < H, status)
                                        : (u + 1 < uh && index_ok(u + 3 < H, status)))
                nx = load_raw(pf, v, W, fast_ld);
            pf += P;
            emit(u, codes_of_row(A, B, C));
        };
        const std::true_type yes;
        const std::false_type no;
        int u = ul;
        for (; u + 4 <= uh; u += 3) {
            step(r0, r1, r2, u, yes);
            step(r1, r2, r0, u + 1, yes);
            step(r2, r0, r1, u + 2, yes);
        }
        // one to three rows left
        if (u < uh) step(r0, r1, r2, u, no);
        if (u + 1 < uh) step(r1, r2, r0, u + 1, no);
        if (u + 2 < uh) step(r2, r0, r1, u + 2, no);
    }

    if constexpr (HIST) {
        if (use_smem) {
            if constexpr (kRowSlots) {
                flush_slots<MODE, K>(jb, hc, wh, ri, rj_lo, ncs, ncs, status);
            } else {
                __syncwarp();
                // Only codes that can occur are scanned: the C(8,k) codes with
                // popcount k for the exact-k LDP modes (bin = position in the
                // list when compact, the code itself when raw), all 256 for LBP
                // and the threshold modes.
                constexpr int NC = exact_k(MODE) ? binom_ce(8, K) : 256;
                constexpr int NI = (NC + 31) / 32;
                int code_of[NI];
#pragma unroll
                for (int m = 0; m < NI; ++m) {
                    const int idx = lane + 32 * m;
                    // (code 0 of the LDP threshold modes holds the skipped columns)
                    code_of[m] = exact_k(MODE) ? (idx < NC ? (int)__ldg(&g_code_list.code[K][idx]) : -1)
                                               : ((is_ldp(MODE) && idx == 0) ? -1 : idx);
                }
                for (int sl = 0; sl < nslots; ++sl) {
                    const int hbase = ((ri_lo + sl / ncs) * hc.C + rj_lo + sl % ncs) * hc.nbins;
                    uint32_t* hs = wh + sl * 256;
#pragma unroll
                    for (int m = 0; m < NI; ++m) {
                        const int code = code_of[m];
                        if (code >= 0) {
                            const uint32_t c = hs[code];
                            if (c) {
                                const int bin = (exact_k(MODE) && hc.compact) ? lane + 32 * m : code;
                                if (index_ok(hbase + bin < hc.R * hc.C * hc.nbins, status))
                                    atomicAdd(&jb.hist[hbase + bin], c);
                                hs[code] = 0;
                            }
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
}

}  // namespace ldp
