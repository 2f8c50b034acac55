// Kernels of libldp for ONE tile variant (rows per warp tile x warps per CTA), compiled
// once per variant with -DLDP_VAR_ID=<n> -DLDP_VAR_RPW=<rows> -DLDP_VAR_NW=<warps>
// -DLDP_VAR_MB=<min CTAs per SM> -DLDP_VAR_ST=<1: rows staged through the bulk-copy engine>
// -DLDP_VAR_SP=<1: narrow tiles split their rows between lane groups, 2: shared
// histogram slots per region column of the current region row>:
// the single-image fused kernel and the persistent batch kernel for every
// (mode, k, histogram) combination, plus their launchers.  Built once more
// per other reading of Eq. 2-3 with -DLDP_CODE_MODES=<kernel mode> (raw-m
// ranking, thresholds; namespaces varcm2..varcm4), in the tile shape of
// variant 0.
#include <cuda_runtime.h>

#include "ldp_device.cuh"
#include "ldp_launch.h"

#ifndef LDP_VAR_ID
#error "compile with -DLDP_VAR_ID, -DLDP_VAR_RPW, -DLDP_VAR_NW, -DLDP_VAR_MB, -DLDP_VAR_ST and -DLDP_VAR_SP"
#endif
#define LDP_CAT2(a, b) a##b
#define LDP_CAT(a, b) LDP_CAT2(a, b)
#define LDP_VNS LDP_CAT(var, LDP_VAR_ID)

namespace ldp {
namespace LDP_VNS {

struct VAR {
    // RPW: rows of a warp tile, NW: warps per CTA, MB: min CTAs per SM,
    // ST: input rows staged through the bulk-copy ring
    static constexpr int RPW = LDP_VAR_RPW, NW = LDP_VAR_NW, MB = LDP_VAR_MB;
    static constexpr bool ST = LDP_VAR_ST != 0;
    static constexpr bool SP = LDP_VAR_SP == 1;  // narrow tiles split their rows between lane groups
    static constexpr bool RS = LDP_VAR_SP == 2;  // shared slots per region column of the current region row
};


__device__ __forceinline__ Job to_job(const JobArgs& a) {
    Job j;
    j.img = a.img;
    j.H = a.H;
    j.W = a.W;
    j.P = a.P;
    j.codes = a.codes;
    j.Pc = a.Pc;
    j.hist = a.hist;
    return j;
}

__device__ __forceinline__ HistCfg to_hc(const HistArgs& h) {
    HistCfg c;
    c.R = h.R;
    c.C = h.C;
    c.nbins = h.nbins;
    c.compact = h.compact;
    return c;
}

// Shared memory of a CTA: per warp a private histogram of SLOTS x 256 bins
// (with HIST) and, in the staged variants, a bulk-copy ring.
template <class V, bool HIST, int SLOTS, bool ST = V::ST>
struct WarpSmem {
    uint32_t h[HIST ? V::NW : 1][HIST ? SLOTS * 256 : 1];
    WarpRing ring[V::NW];
};
template <class V, bool HIST, int SLOTS>
struct WarpSmem<V, HIST, SLOTS, false> {
    uint32_t h[HIST ? V::NW : 1][HIST ? SLOTS * 256 : 1];
};

// The warp's ring (staged variants) and histogram, whose counted slots are
// zeroed (a junk slot is never read).
template <class V, bool HIST, int SLOTS>
__device__ __forceinline__ uint32_t* warp_setup(WarpSmem<V, HIST, SLOTS>& s, WarpRing** ring) {
    const int w = threadIdx.x >> 5;
    *ring = nullptr;
    if constexpr (V::ST) {
        *ring = &s.ring[w];
        ring_init(*ring);
    }
    if constexpr (!HIST) return nullptr;
    uint32_t* wh = s.h[w];
    for (int e = threadIdx.x & 31; e < kWarpSlots * 256; e += 32) wh[e] = 0;
    __syncwarp();
    return wh;
}

// ---------------- single image: one warp per tile ----------------
template <int MODE, int K, class V, bool HIST>
__global__ void __launch_bounds__(V::NW * 32, V::MB) k_plain(JobArgs ja, HistArgs ha) {
    __shared__ WarpSmem<V, HIST, warp_hist_slots<MODE>()> sh;
    const Job jb = to_job(ja);
    const int ntx = (jb.W - 2 + kTileW - 1) / kTileW;
    const int nty = (jb.H - 2 + V::RPW - 1) / V::RPW;
    const int w = blockIdx.x * V::NW + (threadIdx.x >> 5);
    if (w >= ntx * nty) return;  // whole warp
    WarpRing* ring;
    uint32_t* wh = warp_setup(sh, &ring);
    uint32_t ph = 0;
    warp_tile<MODE, K, V::RPW, HIST, V::ST, V::SP, V::RS>(jb, to_hc(ha), (w / ntx) * V::RPW, (w % ntx) * kTileW, wh, ring,
                                                   ph, ja.status);
}

// ---------------- persistent batch kernel: warps take tiles independently ----------------
// Each warp takes tiles from an atomic counter: lane 0 takes the index and
// the tile's image, lanes 0..10 load the image descriptor and its first tile
// index together, and shuffles hand them to the whole warp.  No CTA-wide
// barrier is ever needed.
template <int MODE, int K, class V, bool HIST>
__global__ void __launch_bounds__(V::NW * 32, V::MB) k_batch(BatchArgs a) {
    __shared__ WarpSmem<V, HIST, warp_hist_slots<MODE>()> sh;
    const HistCfg hc = to_hc(a.hc);
    const int lane = threadIdx.x & 31;
    const int total = *a.scr.total;
    WarpRing* ring;
    uint32_t* wh = warp_setup(sh, &ring);
    uint32_t ph = 0;
    for (;;) {
        int t = 0, img = 0;
        if (lane == 0) {
            t = atomicAdd(a.scr.counter, 1);
            if (t < total) img = a.scr.tile_img[t];
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        img = __shfl_sync(0xffffffffu, img, 0);
        // descriptor words 0..9 (40 bytes) and the image's first tile index
        uint32_t word = 0;
        if (lane < 10) word = __ldg(reinterpret_cast<const unsigned int*>(a.descs + img) + lane);
        else if (lane == 10) word = (uint32_t)__ldg(a.scr.prefix + img);
        auto wd = [&](int i) { return __shfl_sync(0xffffffffu, word, i); };
        Job jb;
        jb.img = reinterpret_cast<const uint8_t*>((uint64_t)wd(0) | ((uint64_t)wd(1) << 32));
        jb.H = (int)wd(2);
        jb.W = (int)wd(3);
        jb.P = (int)wd(4);
        jb.Pc = (int)wd(5);
        jb.codes = reinterpret_cast<uint8_t*>((uint64_t)wd(6) | ((uint64_t)wd(7) << 32));
        const uint64_t hoff = (uint64_t)wd(8) | ((uint64_t)wd(9) << 32);
        jb.hist = a.hist ? a.hist + hoff : nullptr;
        const int lt = t - (int)wd(10);
        const int ntx = (jb.W - 2 + kTileW - 1) / kTileW;
        warp_tile<MODE, K, V::RPW, HIST, V::ST, V::SP, V::RS>(jb, hc, (lt / ntx) * V::RPW, (lt % ntx) * kTileW, wh, ring,
                                                       ph, a.status);
    }
}

// ---------------- dispatch ----------------
#define LDP_KCASES(X, M)     \
    case 1: X(M, 1); break; \
    case 2: X(M, 2); break; \
    case 3: X(M, 3); break; \
    case 4: X(M, 4); break; \
    case 5: X(M, 5); break; \
    case 6: X(M, 6); break; \
    case 7: X(M, 7); break; \
    default: return cudaErrorInvalidValue;

cudaError_t launch_plain(int mode, int k, bool hist, const JobArgs& jb, const HistArgs& hc, cudaStream_t s) {
    const int tiles = ((jb.W - 2 + kTileW - 1) / kTileW) * ((jb.H - 2 + VAR::RPW - 1) / VAR::RPW);
    dim3 grid((tiles + VAR::NW - 1) / VAR::NW);
    dim3 block(VAR::NW * 32);
#define LDP_PLAIN(M, KK)                                                        \
    do {                                                                        \
        if (hist) k_plain<M, KK, VAR, true><<<grid, block, 0, s>>>(jb, hc);     \
        else k_plain<M, KK, VAR, false><<<grid, block, 0, s>>>(jb, hc);         \
    } while (0)
    switch (mode) {
#ifdef LDP_CODE_MODES
        case LDP_CODE_MODES: switch (k) { LDP_KCASES(LDP_PLAIN, LDP_CODE_MODES) } break;
#else
        case kLBP: LDP_PLAIN(kLBP, 1); break;
        case kLDP: switch (k) { LDP_KCASES(LDP_PLAIN, kLDP) } break;
#endif
        default: return cudaErrorInvalidValue;
    }
#undef LDP_PLAIN
    return cudaGetLastError();
}

template <int M>
static const void* batch_fn_k(int k, bool hist) {
#define LDP_BFN(KK) (hist ? (const void*)k_batch<M, KK, VAR, true> : (const void*)k_batch<M, KK, VAR, false>)
    switch (k) {
        case 1: return LDP_BFN(1);
        case 2: return LDP_BFN(2);
        case 3: return LDP_BFN(3);
        case 4: return LDP_BFN(4);
        case 5: return LDP_BFN(5);
        case 6: return LDP_BFN(6);
        case 7: return LDP_BFN(7);
        default: return nullptr;
    }
#undef LDP_BFN
}

static const void* batch_fn(int mode, int k, bool hist) {
    switch (mode) {
#ifdef LDP_CODE_MODES
        case LDP_CODE_MODES: return batch_fn_k<LDP_CODE_MODES>(k, hist);
#else
        case kLBP: return hist ? (const void*)k_batch<kLBP, 1, VAR, true> : (const void*)k_batch<kLBP, 1, VAR, false>;
        case kLDP: return batch_fn_k<kLDP>(k, hist);
#endif
        default: return nullptr;
    }
}

cudaError_t launch_batch_main(int mode, int k, bool hist, int grid, const BatchArgs& a, cudaStream_t s) {
    const void* fn = batch_fn(mode, k, hist);
    if (!fn) return cudaErrorInvalidValue;
    BatchArgs arg = a;
    void* params[] = {&arg};
    return cudaLaunchKernel(fn, dim3(grid), dim3(VAR::NW * 32), params, 0, s);
}

cudaError_t batch_occupancy(int mode, int k, bool hist, int* blocks_per_sm) {
    const void* fn = batch_fn(mode, k, hist);
    if (!fn) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, VAR::NW * 32, 0);
}

}  // namespace LDP_VNS
}  // namespace ldp
