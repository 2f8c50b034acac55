// Kernels of libldp for ONE tile variant (rows per warp x warps), compiled
// once per variant with -DLDP_VAR_ID=<n> -DLDP_VAR_RPW=<rows> -DLDP_VAR_NW=<warps>
// -DLDP_VAR_MB=<min CTAs per SM of the persistent kernel>:
// the single-image fused kernel and the persistent batch kernel for every
// (mode, k, histogram) combination, plus their launchers.
#include <cuda_runtime.h>

#include "ldp_device.cuh"
#include "ldp_launch.h"

#ifndef LDP_VAR_ID
#error "compile with -DLDP_VAR_ID, -DLDP_VAR_RPW, -DLDP_VAR_NW and -DLDP_VAR_MB"
#endif
#define LDP_CAT2(a, b) a##b
#define LDP_CAT(a, b) LDP_CAT2(a, b)
#define LDP_VNS LDP_CAT(var, LDP_VAR_ID)

namespace ldp {
namespace LDP_VNS {

struct VAR {
    static constexpr int RPW = LDP_VAR_RPW, NW = LDP_VAR_NW, TH = LDP_VAR_RPW * LDP_VAR_NW, MB = LDP_VAR_MB;
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

// ---------------- single image: one CTA per tile ----------------
template <int MODE, int K, class V, bool HIST>
__global__ void __launch_bounds__(V::NW * 32, V::MB) k_plain(JobArgs ja, HistArgs ha) {
    __shared__ Smem<V::TH> sm;
    const Job jb = to_job(ja);
    const HistCfg hc = to_hc(ha);
    const int u0 = blockIdx.y * V::TH, v0 = blockIdx.x * kTileW;
    TileGeo geo{0, 0, 1, 1, 1};
    if (HIST) geo = tile_geo(jb.H, jb.W, hc, u0, v0, V::TH);  // uniform: every thread computes it
    process_tile<MODE, K, V::RPW, V::NW, HIST>(jb, hc, u0, v0, geo, sm);
}

// ---------------- persistent batch kernel ----------------
// Asynchronous global -> shared copies.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Tiles come from an atomic counter (dynamic load balance across uneven
// images).  Thread 0 takes the next tile, copies its descriptor into shared
// memory asynchronously and publishes it at a barrier.
template <int MODE, int K, class V, bool HIST>
__global__ void __launch_bounds__(V::NW * 32, V::MB) k_batch(BatchArgs a) {
    __shared__ Smem<V::TH> sm;
    const HistCfg hc = to_hc(a.hc);
    const int total = *a.scr.total;
    for (;;) {
        if (threadIdx.x == 0) {
            TileSlot& sl = sm.tile[0];
            const int t = atomicAdd(a.scr.counter, 1);
            if (t >= total) {
                sl.u0 = -1;
            } else {
                const int img = a.scr.tile_img[t];
                const uint64_t* src = reinterpret_cast<const uint64_t*>(a.descs + img);
#pragma unroll
                for (int w = 0; w < 5; ++w) cp_async8(&sm.stage[w], src + w);
                cp_async4(&sm.stage[5], a.scr.prefix + img);
                cp_async_wait_all();
                const ldp_image_desc& d = *reinterpret_cast<const ldp_image_desc*>(&sm.stage[0]);
                const int lt = t - (int)(sm.stage[5] & 0xFFFFFFFFu);
                const int ntx = (d.W - 2 + kTileW - 1) / kTileW;
                sl.u0 = (lt / ntx) * V::TH;
                sl.v0 = (lt % ntx) * kTileW;
                sl.job.img = d.img;
                sl.job.H = d.H;
                sl.job.W = d.W;
                sl.job.P = d.pitch;
                sl.job.codes = d.codes;
                sl.job.Pc = d.code_pitch;
                sl.job.hist = a.hist ? a.hist + d.hist_offset : nullptr;
                if (HIST) sl.geo = tile_geo(d.H, d.W, hc, sl.u0, sl.v0, V::TH);
            }
        }
        __syncthreads();
        const TileSlot& cur = sm.tile[0];
        if (cur.u0 < 0) break;
        const Job jb = cur.job;
        const TileGeo geo = cur.geo;
        process_tile<MODE, K, V::RPW, V::NW, HIST>(jb, hc, cur.u0, cur.v0, geo, sm);
        __syncthreads();
    }
}

// ---------------- dispatch ----------------
cudaError_t launch_plain(int mode, int k, bool hist, const JobArgs& jb, const HistArgs& hc, cudaStream_t s) {
    dim3 grid((jb.W - 2 + kTileW - 1) / kTileW, (jb.H - 2 + VAR::TH - 1) / VAR::TH);
    dim3 block(VAR::NW * 32);
#define LDP_PLAIN(M, KK)                                                        \
    do {                                                                        \
        if (hist) k_plain<M, KK, VAR, true><<<grid, block, 0, s>>>(jb, hc);     \
        else k_plain<M, KK, VAR, false><<<grid, block, 0, s>>>(jb, hc);         \
    } while (0)
    if (mode == kLBP) {
        LDP_PLAIN(kLBP, 1);
    } else {
        switch (k) {
            case 1: LDP_PLAIN(kLDP, 1); break;
            case 2: LDP_PLAIN(kLDP, 2); break;
            case 3: LDP_PLAIN(kLDP, 3); break;
            case 4: LDP_PLAIN(kLDP, 4); break;
            case 5: LDP_PLAIN(kLDP, 5); break;
            case 6: LDP_PLAIN(kLDP, 6); break;
            case 7: LDP_PLAIN(kLDP, 7); break;
            default: return cudaErrorInvalidValue;
        }
    }
#undef LDP_PLAIN
    return cudaGetLastError();
}

static const void* batch_fn(int mode, int k, bool hist) {
#define LDP_BFN(M, KK) (hist ? (const void*)k_batch<M, KK, VAR, true> : (const void*)k_batch<M, KK, VAR, false>)
    if (mode == kLBP) return LDP_BFN(kLBP, 1);
    switch (k) {
        case 1: return LDP_BFN(kLDP, 1);
        case 2: return LDP_BFN(kLDP, 2);
        case 3: return LDP_BFN(kLDP, 3);
        case 4: return LDP_BFN(kLDP, 4);
        case 5: return LDP_BFN(kLDP, 5);
        case 6: return LDP_BFN(kLDP, 6);
        case 7: return LDP_BFN(kLDP, 7);
        default: return nullptr;
    }
#undef LDP_BFN
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
