// ldp_server: continuous-batching request runtime over the batched LDP path.
//
// Requests (one host image each) are admitted into a resident device arena
// when their buffers fit (admission by free device memory), gathered into
// batches by a dispatcher thread as they arrive, and run through one batch
// plan per stream slot, so a batch that is copying in can overlap another
// that is computing or copying out.  A completion thread waits for each
// batch, hands results back (codes straight into the caller's buffer,
// histograms from a pinned staging buffer), frees the arena space and time
// stamps the requests.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ldp_launch.h"

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr uint64_t kAlign = 256;
uint64_t align_up(uint64_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size) with coalescing frees.
class Arena {
   public:
    explicit Arena(uint64_t size) : size_(size) { free_[0] = size; }
    bool alloc(uint64_t n, uint64_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const uint64_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t n) {
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    uint64_t used() const { return used_; }
    uint64_t size() const { return size_; }

   private:
    uint64_t size_, used_ = 0;
    std::map<uint64_t, uint64_t> free_;
};

struct Request {
    const uint8_t* img;
    int H, W, pitch;
    uint8_t* codes;
    int code_pitch;
    uint32_t* hist;
    uint64_t tag;
    uint64_t t_submit = 0, t_start = 0, t_done = 0;
    uint64_t off = 0, bytes = 0;  // arena range
    uint64_t img_off = 0, code_off = 0;
    int dpitch = 0, dcpitch = 0;
};

struct Slot {  // one stream with its own plans and staging buffers
    cudaStream_t stream = nullptr;
    ldp_batch_plan* plan = nullptr;        // the configured tile variant
    ldp_batch_plan* plan_short = nullptr;  // short warp tiles, for batches of few 64-row tiles
    ldp_image_desc* h_desc = nullptr;  // pinned
    int* h_count = nullptr;            // pinned
    ldp_image_desc* d_desc = nullptr;
    int* d_count = nullptr;
    uint32_t* d_hist = nullptr;        // max_batch * hist_len
    uint32_t* h_hist = nullptr;        // pinned copy
    cudaEvent_t done = nullptr;
    std::vector<Request> reqs;
    bool busy = false;
};

}  // namespace

struct ldp_server {
    ldp_server_config cfg{};
    int hist_len = 0;
    int num_sms = 1;
    uint8_t* d_arena = nullptr;
    Arena* arena = nullptr;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_dispatch, cv_complete;
    std::deque<Request> pending;   // submitted, not yet admitted
    std::deque<int> ready_slots;   // launched, waiting for completion (in launch order)
    std::deque<Request> finished;  // completed, not yet polled
    std::atomic<bool> stop{false};
    std::thread dispatcher, completer;
    int device = 0;
    std::string error;
    uint64_t n_done = 0, pixels_done = 0, batches = 0;
};

namespace {

void set_error(ldp_server* s, const std::string& msg) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error.empty()) s->error = msg;
}

// Launches one batch on slot `si` from the admitted requests in s->slots[si].reqs.
bool launch_batch(ldp_server* s, int si) {
    ldp::Range range("ldp.server.batch");
    Slot& sl = s->slots[si];
    if (ldp::take_fault(ldp::kFaultServerLaunch)) {  // test hook: fail before queueing anything
        set_error(s, std::string("server batch launch (injected): ") + cudaGetErrorString(cudaErrorLaunchFailure));
        return false;
    }
    cudaError_t e = cudaSuccess;
    const int n = (int)sl.reqs.size();
    for (int i = 0; i < n; ++i) {
        Request& r = sl.reqs[i];
        ldp_image_desc& d = sl.h_desc[i];
        d.img = s->d_arena + r.img_off;
        d.H = r.H;
        d.W = r.W;
        d.pitch = r.dpitch;
        d.code_pitch = r.dcpitch;
        d.codes = r.codes ? s->d_arena + r.code_off : nullptr;
        d.hist_offset = (uint64_t)i * (uint64_t)s->hist_len;
        if (e == cudaSuccess) {
            if (r.dpitch == r.pitch)  // same layout on both sides: one linear copy
                e = cudaMemcpyAsync(s->d_arena + r.img_off, r.img, (size_t)r.pitch * (r.H - 1) + r.W,
                                    cudaMemcpyHostToDevice, sl.stream);
            else
                e = cudaMemcpy2DAsync(s->d_arena + r.img_off, r.dpitch, r.img, r.pitch, r.W, r.H,
                                      cudaMemcpyHostToDevice, sl.stream);
        }
    }
    *sl.h_count = n;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.d_desc, sl.h_desc, sizeof(ldp_image_desc) * n, cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_count, sl.h_count, sizeof(int), cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) {
        set_error(s, std::string("server H2D: ") + cudaGetErrorString(e));
        return false;
    }
    // a batch of few 64-row tiles leaves most SMs idle and its latency is that
    // of one tile: such batches run with short warp tiles (more tiles in flight)
    long long tiles64 = 0;
    for (int i = 0; i < n; ++i)
        tiles64 += (long long)((sl.reqs[i].H - 2 + 63) / 64) * (long long)((sl.reqs[i].W - 2 + 127) / 128);
    ldp_batch_plan* plan = (sl.plan_short && tiles64 < 2LL * s->num_sms) ? sl.plan_short : sl.plan;
    if (ldp_batch_run(plan, sl.d_desc, sl.d_count, s->hist_len ? sl.d_hist : nullptr, sl.stream) != LDP_OK) {
        set_error(s, std::string("server batch run: ") + ldp_last_error());
        return false;
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        Request& r = sl.reqs[i];
        if (r.codes) {
            if (r.dcpitch == r.code_pitch && r.code_pitch == r.W - 2)  // unpadded rows: one linear copy
                e = cudaMemcpyAsync(r.codes, s->d_arena + r.code_off, (size_t)r.code_pitch * (r.H - 2),
                                    cudaMemcpyDeviceToHost, sl.stream);
            else
                e = cudaMemcpy2DAsync(r.codes, r.code_pitch, s->d_arena + r.code_off, r.dcpitch, r.W - 2, r.H - 2,
                                      cudaMemcpyDeviceToHost, sl.stream);
        }
    }
    if (e == cudaSuccess && s->hist_len)
        e = cudaMemcpyAsync(sl.h_hist, sl.d_hist, sizeof(uint32_t) * s->hist_len * n, cudaMemcpyDeviceToHost,
                            sl.stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
    if (e != cudaSuccess) {
        set_error(s, std::string("server D2H: ") + cudaGetErrorString(e));
        return false;
    }
    return true;
}

void dispatcher_main(ldp_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop.load()) {
        // a free slot and at least one admissible request
        int si = -1;
        for (int i = 0; i < (int)s->slots.size(); ++i)
            if (!s->slots[i].busy) {
                si = i;
                break;
            }
        if (si < 0 || s->pending.empty()) {
            s->cv_dispatch.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        Slot& sl = s->slots[si];
        sl.reqs.clear();
        // admit in arrival order while the arena has room (continuous batching)
        while (!s->pending.empty() && (int)sl.reqs.size() < s->cfg.max_batch) {
            Request& r = s->pending.front();
            uint64_t off;
            if (!s->arena->alloc(r.bytes, &off)) break;
            r.off = off;
            r.img_off = off;
            r.code_off = off + align_up((uint64_t)r.dpitch * r.H);
            r.t_start = now_ns();
            sl.reqs.push_back(r);
            s->pending.pop_front();
        }
        if (sl.reqs.empty()) {  // nothing fits until a batch completes
            s->cv_dispatch.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        sl.busy = true;
        lk.unlock();
        const bool ok = launch_batch(s, si);
        lk.lock();
        if (!ok) {
            // copies already queued on the slot's stream may still read or
            // write the batch's arena ranges: let them finish first
            lk.unlock();
            cudaStreamSynchronize(sl.stream);
            lk.lock();
            for (Request& r : sl.reqs) s->arena->release(r.off, r.bytes);
            sl.reqs.clear();
            sl.busy = false;
            continue;
        }
        s->ready_slots.push_back(si);
        s->cv_complete.notify_one();
    }
}

void completer_main(ldp_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        if (s->ready_slots.empty()) {
            if (s->stop.load()) break;
            s->cv_complete.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        const int si = s->ready_slots.front();
        s->ready_slots.pop_front();
        Slot& sl = s->slots[si];
        lk.unlock();
        cudaError_t e = cudaEventSynchronize(sl.done);
        const uint64_t t = now_ns();
        if (e == cudaSuccess && s->hist_len)
            for (size_t i = 0; i < sl.reqs.size(); ++i)
                if (sl.reqs[i].hist)
                    std::memcpy(sl.reqs[i].hist, sl.h_hist + i * s->hist_len, sizeof(uint32_t) * s->hist_len);
        lk.lock();
        if (e != cudaSuccess && s->error.empty()) s->error = std::string("server batch: ") + cudaGetErrorString(e);
        for (Request& r : sl.reqs) {
            s->arena->release(r.off, r.bytes);
            r.t_done = t;
            s->pixels_done += (uint64_t)r.H * r.W;
            s->finished.push_back(r);
        }
        s->n_done += sl.reqs.size();
        s->batches += 1;
        sl.reqs.clear();
        sl.busy = false;
        s->cv_dispatch.notify_one();
    }
}

void destroy_resources(ldp_server* s) {
    for (Slot& sl : s->slots) {
        if (sl.plan) ldp_batch_plan_destroy(sl.plan);
        if (sl.plan_short) ldp_batch_plan_destroy(sl.plan_short);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
        if (sl.h_count) cudaFreeHost(sl.h_count);
        if (sl.h_hist) cudaFreeHost(sl.h_hist);
        if (sl.d_desc) cudaFree(sl.d_desc);
        if (sl.d_count) cudaFree(sl.d_count);
        if (sl.d_hist) cudaFree(sl.d_hist);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (s->d_arena) cudaFree(s->d_arena);
    delete s->arena;
}

}  // namespace

extern "C" {

int ldp_server_create(ldp_server** out, const ldp_server_config* cfg) {
    if (!out || !cfg) return ldp::report_error(LDP_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->max_batch < 1 || cfg->max_batch > (1 << 16)) return ldp::report_error(LDP_EINVAL, "max_batch out of range");
    if (cfg->streams < 1 || cfg->streams > 16) return ldp::report_error(LDP_EINVAL, "streams must be in [1,16]");
    if (cfg->arena_bytes < (1u << 20)) return ldp::report_error(LDP_EINVAL, "arena_bytes below 1 MiB");
    if (cfg->k < 1 || cfg->k > 7) return ldp::report_error(LDP_EINVAL, "k must be in [1,7]");
    if (cfg->rs.R < 1 || cfg->rs.C < 1 || (int64_t)cfg->rs.R * cfg->rs.C > (1 << 16))
        return ldp::report_error(LDP_EINVAL, "region grid must be 1x1 .. 65536 regions");
    if (cfg->rs.compact != 0 && cfg->rs.compact != 1) return ldp::report_error(LDP_EINVAL, "compact must be 0 or 1");
    ldp_server* s = new (std::nothrow) ldp_server();
    if (!s) return ldp::report_error(LDP_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    s->hist_len = cfg->rs.R * cfg->rs.C * (cfg->rs.compact ? ldp_hist_bins(cfg->k) : 256);
    cudaGetDevice(&s->device);
    void* arena_mem = nullptr;
    cudaError_t e = ldp::device_malloc(&arena_mem, cfg->arena_bytes);
    s->d_arena = static_cast<uint8_t*>(arena_mem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return ldp::report_error(LDP_ENOMEM, "device arena allocation failed");
    }
    s->arena = new Arena(cfg->arena_bytes);
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    s->slots.resize(cfg->streams);
    const uint64_t max_pixels = cfg->arena_bytes;  // pixels in flight never exceed arena bytes
    for (Slot& sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_desc, sizeof(ldp_image_desc) * cfg->max_batch);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_count, sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_hist, sizeof(uint32_t) * (size_t)s->hist_len * cfg->max_batch);
        if (e == cudaSuccess)
            e = ldp::device_malloc(reinterpret_cast<void**>(&sl.d_desc), sizeof(ldp_image_desc) * cfg->max_batch);
        if (e == cudaSuccess) e = ldp::device_malloc(reinterpret_cast<void**>(&sl.d_count), sizeof(int));
        if (e == cudaSuccess)
            e = ldp::device_malloc(reinterpret_cast<void**>(&sl.d_hist),
                                   sizeof(uint32_t) * (size_t)s->hist_len * cfg->max_batch);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            if (ldp_batch_plan_create(&sl.plan, cfg->max_batch, max_pixels, cfg->k, cfg->rs, 0) != LDP_OK ||
                (cfg->variant >= 0 && ldp_batch_plan_set_config(sl.plan, cfg->variant, cfg->ctas_per_sm) != LDP_OK)) {
                const std::string why = ldp_last_error();
                destroy_resources(s);
                delete s;
                cudaGetLastError();
                return ldp::report_error(LDP_ENOMEM, ("server batch plan: " + why).c_str());
            }
            // short tiles: the first non-staged variant of 8-row tiles, unless a variant was fixed
            int vshort = -1;
            for (int v = 0; v < ldp::num_variants() && cfg->variant < 0; ++v) {
                const char* name = ldp::variant_name(v);
                if (ldp::variant_tile_h(v) == 8 && name[0] && name[strlen(name) - 1] == '0') {
                    vshort = v;
                    break;
                }
            }
            // it only runs batches of fewer than 2 x #SMs 64-row tiles; such a
            // tile covers at most 66 x 130 input pixels, which bounds the
            // pixels of those batches (and so the short plan's work list)
            const uint64_t short_pixels = std::min<uint64_t>(max_pixels, 2ull * (uint64_t)s->num_sms * 66u * 130u);
            if (vshort >= 0 &&
                (ldp_batch_plan_create(&sl.plan_short, cfg->max_batch, short_pixels, cfg->k, cfg->rs, 0) != LDP_OK ||
                 ldp_batch_plan_set_config(sl.plan_short, vshort, cfg->ctas_per_sm) != LDP_OK)) {
                const std::string why = ldp_last_error();
                destroy_resources(s);
                delete s;
                cudaGetLastError();
                return ldp::report_error(LDP_ENOMEM, ("server short-tile plan: " + why).c_str());
            }
        }
    }
    if (e != cudaSuccess) {
        destroy_resources(s);
        delete s;
        cudaGetLastError();
        return ldp::report_error(LDP_ENOMEM, "server buffer allocation failed");
    }
    // warm every plan up with an empty batch: its kernels' modules load and
    // its CUDA graph is captured now, not inside the first request that
    // happens to need it (that costs milliseconds)
    for (Slot& sl : s->slots) {
        e = cudaMemsetAsync(sl.d_count, 0, sizeof(int), sl.stream);
        for (ldp_batch_plan* pl : {sl.plan, sl.plan_short})
            if (e == cudaSuccess && pl &&
                ldp_batch_run(pl, sl.d_desc, sl.d_count, s->hist_len ? sl.d_hist : nullptr, sl.stream) != LDP_OK)
                e = cudaErrorUnknown;
        if (e == cudaSuccess) e = cudaStreamSynchronize(sl.stream);
        if (e != cudaSuccess) {
            const std::string why = std::string("server warm-up: ") + ldp_last_error();
            destroy_resources(s);
            delete s;
            cudaGetLastError();
            return ldp::report_error(LDP_ECUDA, why.c_str());
        }
    }
    s->dispatcher = std::thread(dispatcher_main, s);
    s->completer = std::thread(completer_main, s);
    *out = s;
    return LDP_OK;
}

int ldp_server_submit(ldp_server* s, const uint8_t* host_img, int H, int W, int pitch, uint8_t* host_codes,
                      int code_pitch, uint32_t* host_hist, uint64_t tag) {
    if (!s || !host_img) return ldp::report_error(LDP_EINVAL, "NULL argument");
    if (H < 3 || W < 3 || H > (1 << 20) || W > (1 << 20) || pitch < W)
        return ldp::report_error(LDP_EINVAL, "bad image shape");
    if (host_codes && code_pitch < W - 2) return ldp::report_error(LDP_EINVAL, "code_pitch < W-2");
    Request r;
    r.img = host_img;
    r.H = H;
    r.W = W;
    r.pitch = pitch;
    r.codes = host_codes;
    r.code_pitch = code_pitch;
    r.hist = host_hist;
    r.tag = tag;
    // device pitches: the caller's when 16-byte multiples (one linear copy
    // each way), else W and W-2 rounded up to 16 (fast kernel loads/stores)
    r.dpitch = (pitch % 16 == 0) ? pitch : (int)((W + 15) & ~15);
    r.dcpitch = (host_codes && code_pitch % 16 == 0) ? code_pitch : (int)((W - 2 + 15) & ~15);
    r.bytes = align_up((uint64_t)r.dpitch * H) + (host_codes ? align_up((uint64_t)r.dcpitch * (H - 2)) : 0);
    if (r.bytes > s->arena->size()) return ldp::report_error(LDP_EINVAL, "image larger than the server's device arena");
    r.t_submit = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->error.empty()) return ldp::report_error(LDP_ECUDA, s->error.c_str());
        s->pending.push_back(r);
    }
    s->cv_dispatch.notify_one();
    return LDP_OK;
}

int ldp_server_poll(ldp_server* s, ldp_completion* out, int max, int* n_out) {
    if (!s || !n_out || (max > 0 && !out)) return ldp::report_error(LDP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    int n = 0;
    while (n < max && !s->finished.empty()) {
        const Request& r = s->finished.front();
        out[n].tag = r.tag;
        out[n].t_submit_ns = r.t_submit;
        out[n].t_start_ns = r.t_start;
        out[n].t_done_ns = r.t_done;
        ++n;
        s->finished.pop_front();
    }
    *n_out = n;
    if (!s->error.empty()) return ldp::report_error(LDP_ECUDA, s->error.c_str());
    return LDP_OK;
}

int ldp_server_stats(ldp_server* s, ldp_server_stats_t* st) {
    if (!s || !st) return ldp::report_error(LDP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    st->completed = s->n_done;
    st->pixels = s->pixels_done;
    st->batches = s->batches;
    st->pending = s->pending.size();
    st->arena_used = s->arena->used();
    st->arena_bytes = s->arena->size();
    return LDP_OK;
}

int ldp_server_destroy(ldp_server* s) {
    if (!s) return LDP_OK;
    // finish what was submitted, then stop
    for (;;) {
        std::unique_lock<std::mutex> lk(s->mu);
        bool idle = s->pending.empty() && s->ready_slots.empty();
        for (const Slot& sl : s->slots) idle = idle && !sl.busy;
        if (idle || !s->error.empty()) break;
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    s->stop.store(true);
    s->cv_dispatch.notify_all();
    s->cv_complete.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    if (s->completer.joinable()) s->completer.join();
    cudaDeviceSynchronize();
    destroy_resources(s);
    delete s;
    return LDP_OK;
}

}  // extern "C"
