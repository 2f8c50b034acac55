// Variant-independent kernels and dispatch of libldp: batch preparation
// (tile scan, tile -> image map, histogram zeroing), the device status word,
// and the switch from a runtime tile variant to its translation unit.
#include <cuda_runtime.h>

#include "ldp_device.cuh"
#include "ldp_launch.h"

#include <atomic>
#include <mutex>

namespace ldp {

// Device status word (word 0): the kStatus* bits of ldp_modes.h.  Word 1
// is read by the staged tile loop of checked builds: an input-stage group
// to withhold (0: none), set by the wait-fault test hook.
__device__ int g_status[2];

int* status_word() {
    static std::mutex mu;
    static int* addr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;  // word 0
        addr[dev] = static_cast<int*>(p);
    }
    return addr[dev];
}

#define LDP_NAME(ID, RPW, NW, MB, ST, SP)                                \
    (SP == 1   ? "r" #RPW "w" #NW "b" #MB "t" #ST "s"                   \
     : SP == 2 ? "r" #RPW "w" #NW "b" #MB "t" #ST "f"                   \
               : "r" #RPW "w" #NW "b" #MB "t" #ST),
#define LDP_TH(ID, RPW, NW, MB, ST, SP) (RPW),
#define LDP_COUNT(ID, RPW, NW, MB, ST, SP) +1
static const char* kVariantNames[] = {LDP_VARIANTS(LDP_NAME)};
static const int kVariantTH[] = {LDP_VARIANTS(LDP_TH)};
constexpr int kNumVariants = 0 LDP_VARIANTS(LDP_COUNT);
#undef LDP_NAME
#undef LDP_TH
#undef LDP_COUNT

int num_variants() { return kNumVariants; }
const char* variant_name(int v) { return (v >= 0 && v < kNumVariants) ? kVariantNames[v] : ""; }
int variant_tile_h(int v) { return (v >= 0 && v < kNumVariants) ? kVariantTH[v] : 0; }

__device__ __forceinline__ bool desc_ok(const ldp_image_desc& d) {
    return d.img != nullptr && d.H >= 3 && d.W >= 3 && d.H <= (1 << 20) && d.W <= (1 << 20) &&
           d.pitch >= d.W && (d.codes == nullptr || d.code_pitch >= d.W - 2);
}

// One CTA: tiles per image (tile = TH rows x 128 columns, one warp each), exclusive scan
// into prefix[0..n], total, and the tile counter reset.
__global__ void __launch_bounds__(1024) k_batch_scan(BatchArgs a, int TH) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    const int n = max(0, min(*a.count, a.max_images));
    const int tid = threadIdx.x;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    int bad = 0;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + tid;
        int t = 0;
        if (i < n) {
            const ldp_image_desc d = a.descs[i];
            if (desc_ok(d)) {
                t = ((d.W - 2 + kTileW - 1) / kTileW) * ((d.H - 2 + TH - 1) / TH);
            } else {
                bad = 1;
            }
        }
        int incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((tid & 31) >= o) incl += y;
        }
        if ((tid & 31) == 31) s_warp[tid >> 5] = incl;
        __syncthreads();
        if (tid < 32) {
            int w = s_warp[tid];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (tid >= o) w += y;
            }
            s_warp[tid] = w;  // inclusive over warps
        }
        __syncthreads();
        const int warp_excl = (tid >> 5) ? s_warp[(tid >> 5) - 1] : 0;
        const int carry = s_carry;
        if (i < n) a.scr.prefix[i] = carry + warp_excl + incl - t;
        __syncthreads();
        if (tid == 1023) s_carry = carry + warp_excl + incl;
        __syncthreads();
    }
    if (bad) atomicOr(&g_status[0], kStatusBadDesc);
    if (tid == 0) {
        int total = s_carry;
        if (total > a.max_tiles) {
            atomicOr(&g_status[0], kStatusTooManyTiles);
            total = a.max_tiles;
        }
        a.scr.prefix[n] = s_carry;
        *a.scr.total = total;
        *a.scr.counter = 0;
    }
}

// Grid-stride over images: zero each histogram, write the tile -> image map.
__global__ void __launch_bounds__(256) k_batch_fill(BatchArgs a) {
    const int n = max(0, min(*a.count, a.max_images));
    const int L = a.hc.R * a.hc.C * a.hc.nbins;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        if (a.hist) {
            uint32_t* h = a.hist + a.descs[i].hist_offset;
            for (int e = threadIdx.x; e < L; e += blockDim.x) h[e] = 0;
        }
        const int t0 = min(a.scr.prefix[i], a.max_tiles), t1 = min(a.scr.prefix[i + 1], a.max_tiles);
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) a.scr.tile_img[t] = i;
    }
}

cudaError_t launch_batch_prep(int variant, const BatchArgs& a, cudaStream_t s) {
    if (variant < 0 || variant >= kNumVariants) return cudaErrorInvalidValue;
    k_batch_scan<<<1, 1024, 0, s>>>(a, kVariantTH[variant]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int grid = a.max_images < 2048 ? a.max_images : 2048;
    k_batch_fill<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_plain(int mode, int k, bool hist, int variant, const JobArgs& jb, const HistArgs& hc,
                         cudaStream_t s) {
    if (mode == kLDPRaw) return varcm2::launch_plain(mode, k, hist, jb, hc, s);
    if (mode == kLDPThresh) return varcm3::launch_plain(mode, k, hist, jb, hc, s);
    if (mode == kLDPRawThresh) return varcm4::launch_plain(mode, k, hist, jb, hc, s);
    switch (variant) {
#define LDP_CASE(ID, RPW, NW, MB, ST, SP) \
    case ID: return var##ID::launch_plain(mode, k, hist, jb, hc, s);
        LDP_VARIANTS(LDP_CASE)
#undef LDP_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_main(int mode, int k, bool hist, int variant, int grid, const BatchArgs& a,
                              cudaStream_t s) {
    if (mode == kLDPRaw) return varcm2::launch_batch_main(mode, k, hist, grid, a, s);
    if (mode == kLDPThresh) return varcm3::launch_batch_main(mode, k, hist, grid, a, s);
    if (mode == kLDPRawThresh) return varcm4::launch_batch_main(mode, k, hist, grid, a, s);
    switch (variant) {
#define LDP_CASE(ID, RPW, NW, MB, ST, SP) \
    case ID: return var##ID::launch_batch_main(mode, k, hist, grid, a, s);
        LDP_VARIANTS(LDP_CASE)
#undef LDP_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t batch_occupancy(int mode, int k, bool hist, int variant, int* blocks_per_sm) {
    if (mode == kLDPRaw) return varcm2::batch_occupancy(mode, k, hist, blocks_per_sm);
    if (mode == kLDPThresh) return varcm3::batch_occupancy(mode, k, hist, blocks_per_sm);
    if (mode == kLDPRawThresh) return varcm4::batch_occupancy(mode, k, hist, blocks_per_sm);
    switch (variant) {
#define LDP_CASE(ID, RPW, NW, MB, ST, SP) \
    case ID: return var##ID::batch_occupancy(mode, k, hist, blocks_per_sm);
        LDP_VARIANTS(LDP_CASE)
#undef LDP_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t peek_status(cudaStream_t s, int* out) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

// ---------------- fault injection for tests (ldp_test_inject_fault) ----------------
// Per kind: operations still allowed to succeed, then operations to fail.
static std::mutex g_fault_mu;
static int g_fault_after[kFaultKinds], g_fault_count[kFaultKinds];

bool take_fault(int kind) {
    if (kind < 0 || kind >= kFaultKinds) return false;
    std::lock_guard<std::mutex> lk(g_fault_mu);
    if (g_fault_count[kind] <= 0) return false;
    if (g_fault_after[kind] > 0) {
        --g_fault_after[kind];
        return false;
    }
    --g_fault_count[kind];
    return true;
}

void set_faults(int kind, int after, int count) {
    if (kind < 0 || kind >= kFaultKinds) return;
    std::lock_guard<std::mutex> lk(g_fault_mu);
    g_fault_after[kind] = after > 0 ? after : 0;
    g_fault_count[kind] = count > 0 ? count : 0;
}

cudaError_t device_malloc(void** p, size_t bytes) {
    if (take_fault(kFaultDeviceAlloc)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

#ifdef LDP_CHECKED
// Checked builds: the staged tile loop skips the fill of input-stage group
// `group` (when >= 1) and waits for it only kTestSpinLimit polls, so that
// bounded wait gives up with no copy in flight for the stage.
cudaError_t set_wait_fault(int group, cudaStream_t s) {
    cudaError_t e =
        cudaMemcpyToSymbolAsync(g_status, &group, sizeof(int), sizeof(int), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}
#endif

cudaError_t read_clear_status(cudaStream_t s, int* out) {
    static const int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbolAsync(g_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace ldp
