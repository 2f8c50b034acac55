// ldp_batch_run_noalloc: the batched LDP run for callers that cannot
// allocate device memory.
//
// Who needs it: a caller whose device memory is budgeted once at start-up
// (a real-time or serving loop, or a process whose memory is owned by
// another allocator's pool) cannot call cudaMalloc/cudaFree per batch:
// those calls can fail under memory pressure at run time, and cudaFree can
// synchronise the whole device, stalling unrelated streams.  The regular
// batch path allocates its work list in ldp_batch_plan_create; this entry
// point keeps that work list in a fixed static device array instead, so it
// allocates nothing.
//
// The array (kNoAllocInts ints, 8 MiB) lives in every GPU that loads the
// library until the process exits.  Its device address is looked up once
// per device with cudaGetSymbolAddress, by the first call made on that
// device; make that first call before any stream capture begins.  All
// calls share the array and it keeps the last call's contents; every call
// rewrites the parts it reads (count, tile counter, prefix, tile map)
// before reading them.  Calls that overlap on the GPU (different streams,
// or several host threads) race on the array: serialise them.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "ldp_device.cuh"
#include "ldp_launch.h"

namespace {

constexpr int kNoAllocInts = 1 << 21;  // 8 MiB of work list
constexpr int kMaxDevices = 64;
constexpr int kTileCols = ldp::kTileW;  // output columns per warp tile

// [0] tile counter, [1] total tiles, [2] image count, [3..count+3] prefix,
// then the tile -> image map.
static __device__ __align__(256) int g_noalloc_scratch[kNoAllocInts];

std::mutex g_setup_mutex;
int* g_scratch_addr[kMaxDevices] = {};

__global__ void k_noalloc_set_count(int n) { g_noalloc_scratch[2] = n; }

thread_local char t_msg[256];

}  // namespace

// The thread-local error text behind ldp_last_error() lives in ldp_abi.cu.
namespace ldp {
int report_error(int code, const char* msg);
}

extern "C" LDP_API int ldp_batch_run_noalloc(const ldp_image_desc* d_descs, int count, uint64_t max_pixels,
                                            int max_side, int k, ldp_region_spec rs, uint32_t* d_hist,
                                            void* stream) {
    if (!d_descs && count > 0) return ldp::report_error(LDP_EINVAL, "descriptor pointer is NULL");
    if (count < 0) return ldp::report_error(LDP_EINVAL, "count < 0");
    if (k < 1 || k > 7) return ldp::report_error(LDP_EINVAL, "k must be in [1,7]");
    if (rs.R < 1 || rs.C < 1 || (int64_t)rs.R * rs.C > (1 << 22))
        return ldp::report_error(LDP_EINVAL, "region grid must be 1x1 .. 1<<22 regions");
    if (rs.compact != 0 && rs.compact != 1) return ldp::report_error(LDP_EINVAL, "compact must be 0 or 1");
    if (max_side < 3 || max_side > (1 << 20)) return ldp::report_error(LDP_EINVAL, "max_side must be in [3, 1<<20]");
    // the run uses tile variant 0 (tiles of TH rows x 128 columns);
    // ceil(a)*ceil(b) <= ab + a + b + 1 with a = (H-2)/TH, b = (W-2)/128, so an
    // image has at most H*W/(128 TH) + floor(max_side/TH) + floor(max_side/128) + 3 tiles
    const int kTileRows = ldp::variant_tile_h(0);
    if (kTileRows < 1) return ldp::report_error(LDP_ENOTIMPL, "tile variant 0 missing");
    const uint64_t tile_bound = max_pixels / (uint64_t)(kTileRows * kTileCols) + 1 +
                                (uint64_t)count * (uint64_t)(max_side / kTileRows + max_side / kTileCols + 3);
    const uint64_t need = 3 + (uint64_t)count + 1 + tile_bound;
    if (need > (uint64_t)kNoAllocInts) {
        snprintf(t_msg, sizeof t_msg,
                 "batch too large for the static work list: needs %llu ints (count %d, max_pixels %llu, "
                 "max_side %d), the maximum is %d ints",
                 (unsigned long long)need, count, (unsigned long long)max_pixels, max_side, kNoAllocInts);
        return ldp::report_error(LDP_EINVAL, t_msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ldp::report_error(LDP_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return ldp::report_error(LDP_ENOTIMPL, "device index beyond 63");
    int* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // device `dev` is current
            if (e != cudaSuccess || !p) {
                snprintf(t_msg, sizeof t_msg, "cudaGetSymbolAddress of the static work list failed: %s",
                         cudaGetErrorString(e));
                return ldp::report_error(LDP_ECUDA, t_msg);
            }
            g_scratch_addr[dev] = static_cast<int*>(p);
        }
        base = g_scratch_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ldp::BatchArgs a{};
    a.descs = d_descs;
    a.count = base + 2;
    a.hist = d_hist;
    a.max_images = count > 0 ? count : 1;
    a.max_tiles = (int)tile_bound;
    a.scr.counter = base;
    a.scr.total = base + 1;
    a.scr.prefix = base + 3;
    a.scr.tile_img = base + 3 + (count + 1);
    a.status = ldp::status_word();
    a.hc.R = rs.R;
    a.hc.C = rs.C;
    a.hc.compact = rs.compact;
    a.hc.nbins = 256;
    if (rs.compact) {
        int c = 1;
        for (int i = 1; i <= k; ++i) c = c * (8 - k + i) / i;
        a.hc.nbins = c;
    }
    int occ = 0;
    e = ldp::batch_occupancy(0, k, d_hist != nullptr, 0, &occ);
    if (e != cudaSuccess) return ldp::report_error(LDP_ECUDA, cudaGetErrorString(e));
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return ldp::report_error(LDP_ECUDA, cudaGetErrorString(e));
    k_noalloc_set_count<<<1, 1, 0, s>>>(count);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = ldp::launch_batch_prep(0, a, s);
    if (e == cudaSuccess) e = ldp::launch_batch_main(0, k, d_hist != nullptr, 0, nsm * (occ > 0 ? occ : 1), a, s);
    if (e != cudaSuccess) return ldp::report_error(LDP_ECUDA, cudaGetErrorString(e));
    return LDP_OK;
}
