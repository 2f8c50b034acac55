// Host-to-host batched extraction with copies and compute overlapped.
//
// A batch of images in host memory is cut into chunks of consecutive images
// (at most chunk_images images and chunk_pixels pixels each).  Chunk c uses
// device buffer c % nbuf: its images are copied in with one cudaMemcpyAsync
// (the host layout of the chunk's images is kept, so the copy is one range),
// its descriptors and count with another, the buffer's batch plan extracts
// codes and histograms, and the codes and histograms are copied back to the
// caller's host buffers -- all on the buffer's own stream.  With nbuf >= 3
// the copy-in of one chunk, the kernels of the next and the copy-out of a
// third overlap (host->device and device->host copies run on separate copy
// engines).  The caller's stream orders the whole run: the pipeline streams
// wait for it before the first copy, and it waits for every pipeline stream
// at the end, so synchronising that stream means the results are in place.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "ldp_launch.h"

struct ldp_pipeline {
    int chunk_images = 0, nbuf = 0, k = 3;
    uint64_t chunk_pixels = 0;
    ldp_region_spec rs{1, 1, 0};
    unsigned flags = 0;
    int hist_len = 0;
    struct Buf {
        cudaStream_t stream = nullptr;
        ldp_batch_plan* plan = nullptr;
        uint8_t* d_img = nullptr;
        uint64_t img_cap = 0;
        uint8_t* d_codes = nullptr;
        uint64_t code_cap = 0;
        uint32_t* d_hist = nullptr;
        uint8_t* d_meta = nullptr;  // [count, pad, descriptors ...]
        uint8_t* h_meta = nullptr;  // pinned staging of the same
        cudaEvent_t meta_done = nullptr;  // the descriptor staging of the last chunk has been copied
        cudaEvent_t done = nullptr;       // the buffer's last chunk is back in host memory
        bool used = false;
    };
    std::vector<Buf> bufs;
    cudaEvent_t start = nullptr;
};

namespace {

constexpr size_t kMetaHead = 16;  // count (int32) + padding, keeps the descriptors 8-byte aligned

int pfail(int code, const char* msg) { return ldp::report_error(code, msg); }

int pcuda(cudaError_t e, const char* where) { return ldp::report_cuda(e, where); }

void destroy_bufs(ldp_pipeline* p) {
    for (auto& b : p->bufs) {
        if (b.stream) cudaStreamSynchronize(b.stream);
        if (b.plan) ldp_batch_plan_destroy(b.plan);
        cudaFree(b.d_img);
        cudaFree(b.d_codes);
        cudaFree(b.d_hist);
        cudaFree(b.d_meta);
        if (b.h_meta) cudaFreeHost(b.h_meta);
        if (b.done) cudaEventDestroy(b.done);
        if (b.meta_done) cudaEventDestroy(b.meta_done);
        if (b.stream) cudaStreamDestroy(b.stream);
    }
    p->bufs.clear();
    if (p->start) cudaEventDestroy(p->start);
    p->start = nullptr;
}

// grows a device buffer (cudaFree waits for the device, so work still queued
// on the old buffer finishes first; this happens on the first runs only)
int ensure(uint8_t** ptr, uint64_t* cap, uint64_t need) {
    if (need <= *cap) return LDP_OK;
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    const uint64_t sz = need + need / 8 + 4096;
    if (cudaMalloc(ptr, sz) != cudaSuccess) {
        cudaGetLastError();
        return pfail(LDP_ENOMEM, "device allocation of a pipeline buffer failed");
    }
    *cap = sz;
    return LDP_OK;
}

}  // namespace

int ldp_pipeline_create(ldp_pipeline** out, int chunk_images, uint64_t chunk_pixels, int k, ldp_region_spec rs,
                        int nbuf, unsigned flags) {
    if (!out) return pfail(LDP_EINVAL, "out is NULL");
    *out = nullptr;
    if (chunk_images < 1 || chunk_images > (1 << 20)) return pfail(LDP_EINVAL, "chunk_images must be in [1, 1<<20]");
    if (chunk_pixels < 9) return pfail(LDP_EINVAL, "chunk_pixels must be at least 9");
    if (nbuf < 1 || nbuf > 8) return pfail(LDP_EINVAL, "nbuf must be in [1, 8]");
    if (flags & LDP_PLAN_NO_GRAPH) return pfail(LDP_EINVAL, "pipelines always replay graphs");
    ldp_pipeline* p = new (std::nothrow) ldp_pipeline();
    if (!p) return pfail(LDP_ENOMEM, "host allocation failed");
    p->chunk_images = chunk_images;
    p->chunk_pixels = chunk_pixels;
    p->k = k;
    p->rs = rs;
    p->flags = flags;
    p->nbuf = nbuf;
    const bool lbp = (flags & LDP_PLAN_LBP) != 0;
    const int cmode = (int)((flags >> 2) & 3u);
    const bool compact = rs.compact && !lbp && (cmode == LDP_CODE_ABS || cmode == LDP_CODE_RAW);
    p->hist_len = rs.R * rs.C * (compact ? ldp_hist_bins(k) : 256);
    p->bufs.resize(nbuf);
    cudaError_t e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
    for (auto& b : p->bufs) {
        if (e != cudaSuccess) break;
        int rc = ldp_batch_plan_create(&b.plan, chunk_images, chunk_pixels, k, rs, flags);
        if (rc) {
            destroy_bufs(p);
            delete p;
            return rc;  // the plan reported the reason
        }
        e = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.meta_done, cudaEventDisableTiming);
        const size_t meta = kMetaHead + sizeof(ldp_image_desc) * (size_t)chunk_images;
        if (e == cudaSuccess) e = cudaMalloc(&b.d_meta, meta);
        if (e == cudaSuccess) e = cudaMallocHost(&b.h_meta, meta);
        if (e == cudaSuccess) e = cudaMalloc(&b.d_hist, sizeof(uint32_t) * (size_t)p->hist_len * chunk_images);
    }
    if (e != cudaSuccess) {
        destroy_bufs(p);
        delete p;
        cudaGetLastError();
        return pfail(LDP_ENOMEM, "pipeline allocation failed");
    }
    *out = p;
    return LDP_OK;
}

int ldp_pipeline_run(ldp_pipeline* p, int count, const uint8_t* h_img, const int64_t* img_off, const int* H,
                     const int* W, const int* pitch, uint8_t* h_codes, const int64_t* code_off, const int* code_pitch,
                     uint32_t* h_hist, void* stream) {
    if (!p) return pfail(LDP_EINVAL, "pipeline is NULL");
    if (count < 0) return pfail(LDP_EINVAL, "count < 0");
    if (count == 0) return LDP_OK;
    if (!h_img || !img_off || !H || !W || !pitch || !h_hist) return pfail(LDP_EINVAL, "NULL host array");
    if (h_codes && (!code_off || !code_pitch)) return pfail(LDP_EINVAL, "codes need offsets and pitches");
    for (int i = 0; i < count; ++i) {
        if (H[i] < 3 || W[i] < 3 || pitch[i] < W[i] || img_off[i] < 0)
            return pfail(LDP_EINVAL, "bad image size, pitch or offset");
        if ((uint64_t)H[i] * (uint64_t)W[i] > p->chunk_pixels) return pfail(LDP_EINVAL, "image larger than a chunk");
        if (i && img_off[i] < img_off[i - 1]) return pfail(LDP_EINVAL, "image offsets must not decrease");
        if (h_codes) {
            if (code_pitch[i] < W[i] - 2 || code_off[i] < 0) return pfail(LDP_EINVAL, "bad code pitch or offset");
            if (i && code_off[i] < code_off[i - 1]) return pfail(LDP_EINVAL, "code offsets must not decrease");
        }
    }
    ldp::Range range("ldp.pipeline_run");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaEventRecord(p->start, cs);
    if (e != cudaSuccess) return pcuda(e, "recording the start event");
    for (auto& b : p->bufs) {
        e = cudaStreamWaitEvent(b.stream, p->start, 0);
        if (e != cudaSuccess) return pcuda(e, "ordering the pipeline after the caller's stream");
    }
    int first = 0, chunk = 0;
    while (first < count) {
        // the next chunk: consecutive images within the image and pixel limits
        int last = first;
        uint64_t px = (uint64_t)H[first] * (uint64_t)W[first];
        while (last + 1 < count && last + 1 - first < p->chunk_images &&
               px + (uint64_t)H[last + 1] * (uint64_t)W[last + 1] <= p->chunk_pixels) {
            ++last;
            px += (uint64_t)H[last] * (uint64_t)W[last];
        }
        const int n = last - first + 1;
        ldp_pipeline::Buf& b = p->bufs[chunk % p->nbuf];
        // the host rewrites the buffer's descriptor staging: its previous copy
        // must be done (device buffers are reused in stream order)
        if (b.used) {
            e = cudaEventSynchronize(b.meta_done);
            if (e != cudaSuccess) return pcuda(e, "waiting for a pipeline buffer");
        }
        const int64_t i0 = img_off[first];
        const uint64_t img_bytes = (uint64_t)(img_off[last] - i0) + (uint64_t)(H[last] - 1) * pitch[last] + W[last];
        int rc = ensure(&b.d_img, &b.img_cap, img_bytes);
        if (rc) return rc;
        int64_t c0 = 0;
        uint64_t code_bytes = 0;
        if (h_codes) {
            c0 = code_off[first];
            code_bytes = (uint64_t)(code_off[last] - c0) + (uint64_t)(H[last] - 3) * code_pitch[last] + (W[last] - 2);
            rc = ensure(&b.d_codes, &b.code_cap, code_bytes);
            if (rc) return rc;
        }
        // descriptors of the chunk, pointing into the buffer's staging
        int32_t* hc = reinterpret_cast<int32_t*>(b.h_meta);
        hc[0] = n;
        ldp_image_desc* hd = reinterpret_cast<ldp_image_desc*>(b.h_meta + kMetaHead);
        for (int j = 0; j < n; ++j) {
            const int i = first + j;
            hd[j].img = b.d_img + (img_off[i] - i0);
            hd[j].H = H[i];
            hd[j].W = W[i];
            hd[j].pitch = pitch[i];
            hd[j].code_pitch = h_codes ? code_pitch[i] : W[i] - 2;
            hd[j].codes = h_codes ? b.d_codes + (code_off[i] - c0) : nullptr;
            hd[j].hist_offset = (uint64_t)j * (uint64_t)p->hist_len;
        }
        const size_t meta = kMetaHead + sizeof(ldp_image_desc) * (size_t)n;
        e = cudaMemcpyAsync(b.d_img, h_img + i0, img_bytes, cudaMemcpyHostToDevice, b.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.d_meta, b.h_meta, meta, cudaMemcpyHostToDevice, b.stream);
        if (e == cudaSuccess) e = cudaEventRecord(b.meta_done, b.stream);
        if (e != cudaSuccess) return pcuda(e, "copying a chunk to the device");
        rc = ((p->flags & LDP_PLAN_LBP) ? lbp_batch_run : ldp_batch_run)(
            b.plan, reinterpret_cast<const ldp_image_desc*>(b.d_meta + kMetaHead), reinterpret_cast<int*>(b.d_meta),
            b.d_hist, b.stream);
        if (rc) return rc;
        if (h_codes) e = cudaMemcpyAsync(h_codes + c0, b.d_codes, code_bytes, cudaMemcpyDeviceToHost, b.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_hist + (uint64_t)first * (uint64_t)p->hist_len, b.d_hist,
                                sizeof(uint32_t) * (size_t)n * (size_t)p->hist_len, cudaMemcpyDeviceToHost, b.stream);
        if (e == cudaSuccess) e = cudaEventRecord(b.done, b.stream);
        if (e != cudaSuccess) return pcuda(e, "copying a chunk back");
        b.used = true;
        first = last + 1;
        ++chunk;
    }
    for (auto& b : p->bufs) {
        if (!b.used) continue;
        e = cudaStreamWaitEvent(cs, b.done, 0);
        if (e != cudaSuccess) return pcuda(e, "ordering the caller's stream after the pipeline");
    }
    return LDP_OK;
}

int ldp_pipeline_set_config(ldp_pipeline* p, int variant, int ctas_per_sm) {
    if (!p) return pfail(LDP_EINVAL, "pipeline is NULL");
    for (auto& b : p->bufs) {
        const int rc = ldp_batch_plan_set_config(b.plan, variant, ctas_per_sm);
        if (rc) return rc;
    }
    return LDP_OK;
}

int ldp_pipeline_destroy(ldp_pipeline* p) {
    if (!p) return LDP_OK;
    destroy_bufs(p);
    delete p;
    return LDP_OK;
}
