// Internal interface between the C-ABI files (ldp_abi.cu and the entry points
// of the feature files) and the kernel translation units.  Not part of the
// public ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>

#include "ldp.h"
#include "ldp_modes.h"

namespace ldp {

// NVTX range around a host-side call (a named span in profiler timelines; a
// no-op unless a tool is attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

struct JobArgs {
    const uint8_t* img;
    int H, W, P;
    uint8_t* codes;
    int Pc;
    uint32_t* hist;
    int* status;  // device status word
};

struct HistArgs {
    int R, C, nbins, compact;
};

// Device scratch of a batch plan (owned by the plan).
struct BatchScratch {
    int* prefix;    // [max_images + 1] exclusive scan of tiles per image
    int* tile_img;  // [max_tiles] image of each tile
    int* counter;   // next tile to hand out
    int* total;     // tiles of this run
};

struct BatchArgs {
    const ldp_image_desc* descs;
    const int* count;
    uint32_t* hist;
    int max_images;
    int max_tiles;
    BatchScratch scr;
    HistArgs hc;
    int* status;  // device status word
};

// Tile variants X(id, rows per tile, warps per CTA, min CTAs per SM, staged,
// split): each warp owns a tile of 128 columns x rows; MB caps registers;
// staged = 1 feeds the rows through the bulk-copy (TMA) engine into a shared
// ring; split = 1 lets a tile narrower than 64 columns (an image's last) share
// its rows between lane groups (for batches of narrow images); split = 2
// keeps shared histogram slots for the current region row only, flushed at
// each region-row boundary (small images, whose tiles cross many regions).
// ldp_kernels.cu is compiled once per entry (the build script reads this list).
#define LDP_VARIANTS(X)                                                                                      \
    X(0, 64, 4, 5, 0, 0) X(1, 64, 4, 6, 0, 0) X(2, 64, 8, 3, 0, 0) X(3, 64, 4, 4, 1, 0) X(4, 128, 4, 4, 1, 0) \
    X(5, 64, 4, 7, 0, 0) X(6, 64, 8, 4, 0, 0) X(7, 16, 4, 6, 0, 0) X(8, 8, 4, 6, 0, 0) X(9, 64, 4, 7, 0, 1)   \
    X(10, 128, 4, 7, 0, 0) X(11, 128, 4, 6, 0, 2) X(12, 128, 4, 7, 0, 2) X(13, 4, 4, 6, 0, 0)

#define LDP_DECLARE_VARIANT(ID, RPW, NW, MB, ST, SP)                                                          \
    namespace var##ID {                                                                                   \
    cudaError_t launch_plain(int mode, int k, bool hist, const JobArgs& jb, const HistArgs& hc,           \
                             cudaStream_t s);                                                             \
    cudaError_t launch_batch_main(int mode, int k, bool hist, int grid, const BatchArgs& a, cudaStream_t s); \
    cudaError_t batch_occupancy(int mode, int k, bool hist, int* blocks_per_sm);                          \
    }
LDP_VARIANTS(LDP_DECLARE_VARIANT)
// the code-variant modes kLDPRaw, kLDPThresh, kLDPRawThresh (one unit each),
// in the tile shape of variant 0
LDP_DECLARE_VARIANT(cm2, 64, 4, 5, 0, 0)
LDP_DECLARE_VARIANT(cm3, 64, 4, 5, 0, 0)
LDP_DECLARE_VARIANT(cm4, 64, 4, 5, 0, 0)
#undef LDP_DECLARE_VARIANT
constexpr int kCodeModeVariant = 0;  // variant whose tile shape varcm2..4 use

int num_variants();
const char* variant_name(int v);
int variant_tile_h(int v);

// mode: 0 = LDP, 1 = LBP.  hist = fused region histograms.
cudaError_t launch_plain(int mode, int k, bool hist, int variant, const JobArgs& jb, const HistArgs& hc,
                         cudaStream_t s);

// Prep (scan + tile map + histogram zeroing) and the persistent kernel.
cudaError_t launch_batch_prep(int variant, const BatchArgs& a, cudaStream_t s);
cudaError_t launch_batch_main(int mode, int k, bool hist, int variant, int grid, const BatchArgs& a,
                              cudaStream_t s);
// Resident CTAs per SM of the persistent kernel.
cudaError_t batch_occupancy(int mode, int k, bool hist, int variant, int* blocks_per_sm);

// Sliding windows (ldp_windows.cu): wh x ww pixels at stride (sh, sw); bins
// are C(8,k) compact codes when compact (k >= 1), else the 256 raw codes.
struct WindowGeom {
    int wh, ww, sh, sw;
    int nbins, k, compact;
};
// uint32 words of the cell histograms of one H x W image: 0 when no cell
// scratch is needed (stride = size, or the fused single pass applies)
uint64_t window_cell_words(int H, int W, const WindowGeom& g);
// stride = size: the cells are the windows (no cell scratch, no sum pass)
bool window_direct(const WindowGeom& g);
// Window histograms of `count` images from their code maps: descriptors in
// device memory (d_descs) or one by value (one, count = 1); max_H / max_W
// bound the images' sizes; cells: scratch of cell_stride words per image
// (unused when window_cell_words is 0).
cudaError_t launch_windows(const ldp_image_desc* d_descs, const ldp_image_desc* one, int count, int max_H,
                           int max_W, const WindowGeom& g, uint32_t* hist, uint32_t* cells,
                           uint64_t cell_stride, cudaStream_t s);

// Crop-and-resize (ldp_resize.cu): descriptors in device memory (d_descs) or
// one by value (one, count = 1); rejected crops set status bit 3.
cudaError_t launch_resize(const ldp_crop_desc* d_descs, const ldp_crop_desc* one, int count, int OH, int OW,
                          int* status, cudaStream_t s);

// Descriptor distances (ldp_distance.cu), metric LDP_DIST_*.
cudaError_t launch_distance(const uint32_t* q, int nq, int ldq, const uint32_t* g, int ng, int ldg, int D,
                            int metric, void* out, int ldo, cudaStream_t s);

cudaError_t read_clear_status(cudaStream_t s, int* out);
// Reads the device status word without clearing it (synchronises s).
cudaError_t peek_status(cudaStream_t s, int* out);

// Fault injection for tests (ldp_test_inject_fault): after `after` more
// operations of a kind, take_fault(kind) is true (and uses one up) for the
// next `count` ones.
constexpr int kFaultDeviceAlloc = LDP_FAULT_DEVICE_ALLOC;  // device allocations of plans and the server
constexpr int kFaultServerLaunch = LDP_FAULT_SERVER_LAUNCH;  // a serving batch fails to launch
constexpr int kFaultKinds = 3;
bool take_fault(int kind);
void set_faults(int kind, int after, int count);
// cudaMalloc, or cudaErrorMemoryAllocation while a device-allocation fault is pending
cudaError_t device_malloc(void** p, size_t bytes);
#ifdef LDP_CHECKED
// Makes the staged tile loop withhold input-stage group `group` (0: off).
cudaError_t set_wait_fault(int group, cudaStream_t s);
#endif
// Device address of the status word on the current device (looked up once per device).
int* status_word();

// Host side of the C-ABI (defined in ldp_abi.cu, used by every file that
// exports entry points).
// Records msg as the calling thread's ldp_last_error() text; returns code.
int report_error(int code, const char* msg);
// Records "where: <CUDA error name>: <text>"; returns LDP_ECUDA.
int report_cuda(cudaError_t e, const char* where);
// C(8, r) for r in [0, 8], else -1: the number of compact bins of k = r.
int binom8(int r);
// Argument checks of an image / a code map (required: a NULL map is an
// error); LDP_OK or LDP_EINVAL with the reason recorded.
int check_image(const void* img, int H, int W, int pitch);
int check_codes(const void* codes, int W, int code_pitch, bool required);
// One single-image launch of kernel mode `mode` (validated arguments): zeroes
// the R x C histogram (when hist is given) and runs the plain kernel in the
// tile variant chosen for the image's size.
int run_plain(int mode, const uint8_t* img, int H, int W, int pitch, int k, int R, int C, int compact,
              uint32_t* hist, uint8_t* codes, int code_pitch, void* stream);

}  // namespace ldp
