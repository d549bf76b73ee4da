// wsm_server.cu -- a quantization server: continuous batching of requests
// over the batched path (wsm_quantize_batch) with admission by device-memory
// footprint.  Host code only.
//
// Lanes: each lane owns a stream, a library handle limited to its share of
// the SMs (wsm_set_grid_limit) and up to slots_per_lane images per batch, so
// the persistent launches of different lanes run side by side.  A scheduler
// thread repeats:
//   1. completions: a busy lane whose completion event has fired hands its
//      requests their results (N', iterations, MSE; the index image and
//      palette were copied into the caller's buffers on the lane's stream),
//      and frees their device buffers;
//   2. admission: an idle lane takes requests from the head of the queue
//      (first come, first served) while it has slots, they share the head's
//      iteration settings, and their buffers fit in the device arena; then
//      it enqueues the copies in, the whole path and the copies out, and
//      records its completion event.
// Requests that arrive while other lanes are busy are admitted as soon as a
// lane and memory are free, and their work overlaps the other lanes' on the
// device.  Every result is exactly what wsm_quantize_batch gives the image on
// its own (the per-image computation does not depend on the batch).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wsm_arena.h"
#include "wsm_internal.cuh"

namespace wsm {

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// One device allocation; the placement of the requests' blocks in it is
// ArenaBook's (wsm_arena.h).
class Arena {
  public:
    int init(size_t bytes) {
        const size_t total = ArenaBook::round_up(bytes);
        cudaError_t e = cudaMalloc(&base_, total);
        if (e != cudaSuccess) return cuda_fail(e, "server arena");
        book_.reset(total);
        return WSM_OK;
    }
    ~Arena() {
        if (base_) cudaFree(base_);
    }
    size_t capacity() const { return book_.capacity(); }
    size_t used() const { return book_.used(); }
    // offset of a block of `bytes`, or SIZE_MAX if none is free
    size_t alloc(size_t bytes) { return book_.alloc(bytes); }
    void release(size_t off, size_t bytes) { book_.release(off, bytes); }
    unsigned char* at(size_t off) const { return static_cast<unsigned char*>(base_) + off; }

  private:
    void* base_ = nullptr;
    ArenaBook book_;
};

struct Req {
    uint64_t id;
    wsm_request r;
    size_t off = 0, bytes = 0;      // arena block
    wsm_result res{};
    bool done = false;
};

// Device bytes of one request: pixels, colors, counts, labels, index, centers.
static size_t footprint(const wsm_request& r) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t n = (size_t)r.n_pixels;
    return up(n * r.pixel_stride) + 2 * up(4 * n) + 2 * up(n) + up(16 * (size_t)r.K);
}

struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    wsm_handle* h = nullptr;
    std::vector<Req*> batch;
    int64_t* d_nu = nullptr;        // [slots] per-batch outputs (device)
    int* d_it = nullptr;
    double* d_mse = nullptr;
    int64_t* h_nu = nullptr;        // pinned mirrors
    int* h_it = nullptr;
    double* h_mse = nullptr;
};

}  // namespace wsm

struct wsm_server {
    wsm_server_config cfg{};
    int device = -1;
    wsm::Arena arena;
    std::vector<wsm::Lane> lanes;
    std::mutex mu;                  // queue, request table, stats, stop flag
    std::condition_variable cv_sched, cv_done;
    std::deque<wsm::Req*> pending;
    std::unordered_map<uint64_t, wsm::Req*> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread thread;
    wsm_server_stats stats{};
};

namespace wsm {

// Status bits of a lane's handle (read and cleared; the stream is idle).
static unsigned take_status(Lane& L) {
    unsigned st = 0;
    cudaMemcpyAsync(&L.h->host_ctrl->status, &L.h->ctrl->status, sizeof(unsigned),
                    cudaMemcpyDeviceToHost, L.stream);
    cudaMemsetAsync(&L.h->ctrl->status, 0, sizeof(unsigned), L.stream);
    if (cudaStreamSynchronize(L.stream) == cudaSuccess) st = L.h->host_ctrl->status;
    return st;
}

static void finish(wsm_server* S, Lane& L) {
    const unsigned st = take_status(L);
    const double t = now_s();
    std::lock_guard<std::mutex> lock(S->mu);
    for (size_t i = 0; i < L.batch.size(); ++i) {
        Req* q = L.batch[i];
        q->res.n_unique = L.h_nu[i];
        q->res.iters = L.h_it[i];
        q->res.mse = L.h_mse[i];
        q->res.t_done = t;
        if (st & ST_TIMEOUT) q->res.status = WSM_E_TIMEOUT;
        else if (q->res.n_unique < q->r.K) q->res.status = WSM_E_INVAL;   // skipped: N' < K
        else if (st & (ST_BAD_LABEL | ST_CAPACITY)) q->res.status = WSM_E_CUDA;
        else q->res.status = WSM_OK;
        S->arena.release(q->off, q->bytes);
        q->done = true;
        S->stats.completed += 1;
        if (q->res.status != WSM_OK) S->stats.failed += 1;
    }
    S->stats.in_flight -= (int64_t)L.batch.size();
    S->stats.arena_used = S->arena.used();
    L.batch.clear();
    S->cv_done.notify_all();
}

// Take requests for an idle lane (caller holds S->mu).
static void admit(wsm_server* S, Lane& L) {
    const int slots = S->cfg.slots_per_lane;
    while (!S->pending.empty() && (int)L.batch.size() < slots) {
        Req* q = S->pending.front();
        if (!L.batch.empty() && (q->r.max_iter != L.batch[0]->r.max_iter ||
                                 q->r.eps != L.batch[0]->r.eps))
            break;                                    // next batch: other settings
        const size_t off = S->arena.alloc(q->bytes);
        if (off == SIZE_MAX) break;                   // wait for memory, in order
        q->off = off;
        q->res.t_admit = now_s();
        S->pending.pop_front();
        L.batch.push_back(q);
    }
    S->stats.in_flight += (int64_t)L.batch.size();
    S->stats.arena_used = S->arena.used();
    S->stats.max_in_flight = std::max(S->stats.max_in_flight, S->stats.in_flight);
    S->stats.arena_peak = std::max(S->stats.arena_peak, (int64_t)S->arena.used());
}

// Enqueue the copies in, the path and the copies out of a lane's batch.
static int launch(wsm_server* S, Lane& L) {
    const int n = (int)L.batch.size();
    std::vector<wsm_item> items(n);
    std::vector<uint64_t> seeds(n);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        Req* q = L.batch[i];
        const size_t np = (size_t)q->r.n_pixels;
        auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
        unsigned char* p = S->arena.at(q->off);
        wsm_item& it = items[i];
        it.d_rgb = p;
        p += up(np * q->r.pixel_stride);
        it.d_colors = reinterpret_cast<uint32_t*>(p);
        p += up(4 * np);
        it.d_counts = reinterpret_cast<uint32_t*>(p);
        p += up(4 * np);
        it.d_labels = p;
        p += up(np);
        it.d_index = p;
        p += up(np);
        it.d_centers = reinterpret_cast<float*>(p);
        it.n_pixels = q->r.n_pixels;
        it.pixel_stride = q->r.pixel_stride;
        it.K = q->r.K;
        it.n_unique = 0;
        seeds[i] = q->r.seed;
        e = cudaMemcpyAsync(const_cast<uint8_t*>(it.d_rgb), q->r.rgb, np * q->r.pixel_stride,
                            cudaMemcpyHostToDevice, L.stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "server input copy");
    int rc = wsm_quantize_batch(L.h, items.data(), n, seeds.data(), L.batch[0]->r.max_iter,
                                L.batch[0]->r.eps, L.d_nu, L.d_it, L.d_mse, L.stream);
    if (rc != WSM_OK) return rc;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        Req* q = L.batch[i];
        if (q->r.index_out)
            e = cudaMemcpyAsync(q->r.index_out, items[i].d_index, (size_t)q->r.n_pixels,
                                cudaMemcpyDeviceToHost, L.stream);
        if (e == cudaSuccess && q->r.palette_out)
            e = cudaMemcpyAsync(q->r.palette_out, items[i].d_centers, 16 * (size_t)q->r.K,
                                cudaMemcpyDeviceToHost, L.stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.h_nu, L.d_nu, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, L.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.h_it, L.d_it, sizeof(int) * n, cudaMemcpyDeviceToHost, L.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.h_mse, L.d_mse, sizeof(double) * n, cudaMemcpyDeviceToHost, L.stream);
    if (e == cudaSuccess) e = cudaEventRecord(L.done, L.stream);
    if (e != cudaSuccess) return cuda_fail(e, "server output copy");
    return WSM_OK;
}

static void fail_batch(wsm_server* S, Lane& L, int rc) {
    std::lock_guard<std::mutex> lock(S->mu);
    const double t = now_s();
    for (Req* q : L.batch) {
        q->res.status = rc;
        q->res.t_done = t;
        S->arena.release(q->off, q->bytes);
        q->done = true;
        S->stats.completed += 1;
        S->stats.failed += 1;
    }
    S->stats.in_flight -= (int64_t)L.batch.size();
    L.batch.clear();
    S->cv_done.notify_all();
}

static void scheduler(wsm_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        bool progress = false;
        for (Lane& L : S->lanes) {
            if (!L.batch.empty() && cudaEventQuery(L.done) == cudaSuccess) {
                finish(S, L);
                progress = true;
            }
        }
        for (Lane& L : S->lanes) {
            if (!L.batch.empty()) continue;
            {
                std::lock_guard<std::mutex> lock(S->mu);
                admit(S, L);
                if (!L.batch.empty()) S->stats.batches += 1;
            }
            if (L.batch.empty()) continue;
            progress = true;
            const int rc = launch(S, L);
            if (rc != WSM_OK) {
                cudaStreamSynchronize(L.stream);
                take_status(L);
                fail_batch(S, L, rc);
            }
        }
        std::unique_lock<std::mutex> lock(S->mu);
        bool busy = false;
        for (Lane& L : S->lanes) busy |= !L.batch.empty();
        if (S->stop && S->pending.empty() && !busy) break;
        if (!progress) {
            // busy lanes are polled every 20 us; an idle server sleeps until a submission
            if (busy) S->cv_sched.wait_for(lock, std::chrono::microseconds(20));
            else S->cv_sched.wait_for(lock, std::chrono::milliseconds(5));
        }
    }
}

static void destroy_lanes(wsm_server* S) {
    for (Lane& L : S->lanes) {
        if (L.h) wsm_destroy(L.h);
        if (L.d_nu) cudaFree(L.d_nu);
        if (L.d_it) cudaFree(L.d_it);
        if (L.d_mse) cudaFree(L.d_mse);
        if (L.h_nu) cudaFreeHost(L.h_nu);
        if (L.h_it) cudaFreeHost(L.h_it);
        if (L.h_mse) cudaFreeHost(L.h_mse);
        if (L.done) cudaEventDestroy(L.done);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    S->lanes.clear();
}

}  // namespace wsm

using namespace wsm;

extern "C" int wsm_server_create(wsm_server** out, const wsm_server_config* cfg) {
    if (!out || !cfg) return fail(WSM_E_INVAL, "null argument");
    *out = nullptr;
    if (cfg->max_K < 1 || cfg->max_K > WSM_MAX_K)
        return fail(WSM_E_INVAL, "max_K must be in [1, 256]");
    if (cfg->max_pixels < 1 || cfg->max_pixels > WSM_MAX_PIXELS)
        return fail(WSM_E_INVAL, "max_pixels must be in [1, 2^24]");
    if (cfg->lanes < 1 || cfg->lanes > 8) return fail(WSM_E_INVAL, "lanes must be in [1, 8]");
    if (cfg->slots_per_lane < 1 || cfg->slots_per_lane > kMaxBatch)
        return fail(WSM_E_INVAL, "slots_per_lane must be in [1, 64]");
    if (cfg->arena_bytes < ((int64_t)1 << 20)) return fail(WSM_E_INVAL, "arena_bytes below 1 MiB");
    wsm_server* S = new (std::nothrow) wsm_server();
    if (!S) return fail(WSM_E_NOMEM, "host allocation failed");
    S->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "cudaGetDevice");
    }
    int rc = S->arena.init((size_t)cfg->arena_bytes);
    S->lanes.resize(cfg->lanes);
    for (int l = 0; l < cfg->lanes && rc == WSM_OK; ++l) {
        Lane& L = S->lanes[l];
        const size_t ns = (size_t)cfg->slots_per_lane;
        rc = wsm_create(&L.h, cfg->max_K, cfg->max_pixels, cfg->max_pixels);
        if (rc == WSM_OK) rc = wsm_reserve_batch(L.h, cfg->slots_per_lane);
        if (rc == WSM_OK && cfg->lanes > 1) {
            int blocks = 0;
            wsm_launch_shape(L.h, -1, nullptr, &blocks, nullptr);
            const int share = std::max(kMaxBatch, blocks * L.h->sms / cfg->lanes);
            rc = wsm_set_grid_limit(L.h, share);
        }
        if (rc != WSM_OK) break;
        e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&L.d_nu, sizeof(int64_t) * ns);
        if (e == cudaSuccess) e = cudaMalloc(&L.d_it, sizeof(int) * ns);
        if (e == cudaSuccess) e = cudaMalloc(&L.d_mse, sizeof(double) * ns);
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_nu, sizeof(int64_t) * ns);
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_it, sizeof(int) * ns);
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_mse, sizeof(double) * ns);
        if (e != cudaSuccess) rc = cuda_fail(e, "server lane");
    }
    if (rc != WSM_OK) {
        destroy_lanes(S);
        delete S;
        return rc;
    }
    S->stats.arena_bytes = (int64_t)S->arena.capacity();
    S->thread = std::thread(scheduler, S);
    *out = S;
    return WSM_OK;
}

extern "C" int wsm_server_submit(wsm_server* S, const wsm_request* r, uint64_t* id) {
    if (!S || !r || !id) return fail(WSM_E_INVAL, "null argument");
    if (r->pixel_stride != 3 && r->pixel_stride != 4)
        return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
    if (r->n_pixels < 1 || r->n_pixels > S->cfg.max_pixels)
        return fail(WSM_E_INVAL, "n_pixels must be in [1, max_pixels]");
    if (r->K < 1 || r->K > S->cfg.max_K) return fail(WSM_E_INVAL, "K out of [1, max_K]");
    if (r->max_iter < 0 || r->max_iter > kMaxTrace)
        return fail(WSM_E_INVAL, "max_iter must be in [0, 4096]");
    if (!r->rgb) return fail(WSM_E_INVAL, "null pixel pointer");
    Req* q = new (std::nothrow) Req();
    if (!q) return fail(WSM_E_NOMEM, "host allocation failed");
    q->r = *r;
    q->bytes = footprint(*r);
    if (q->bytes > S->arena.capacity()) {
        delete q;
        return fail(WSM_E_CAPACITY, "the request needs more device memory than the arena holds");
    }
    q->res.t_submit = now_s();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop) {
            delete q;
            return fail(WSM_E_STATE, "the server is shutting down");
        }
        q->id = S->next_id++;
        S->reqs[q->id] = q;
        S->pending.push_back(q);
        S->stats.submitted += 1;
    }
    S->cv_sched.notify_one();
    *id = q->id;
    return WSM_OK;
}

extern "C" int wsm_server_wait(wsm_server* S, uint64_t id, double timeout_s, wsm_result* res) {
    if (!S || !res) return fail(WSM_E_INVAL, "null argument");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return fail(WSM_E_INVAL, "unknown request id");
    Req* q = it->second;
    const auto pred = [q] { return q->done; };
    if (timeout_s < 0) S->cv_done.wait(lock, pred);
    else if (!S->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), pred))
        return fail(WSM_E_TIMEOUT, "the request is not done yet");
    *res = q->res;
    S->reqs.erase(it);
    delete q;
    if (res->status != WSM_OK)
        return fail(res->status, res->status == WSM_E_INVAL
                                     ? "the image has fewer unique colors than K"
                                     : "the request failed on the device");
    return WSM_OK;
}

extern "C" int wsm_server_stats_get(wsm_server* S, wsm_server_stats* st) {
    if (!S || !st) return fail(WSM_E_INVAL, "null argument");
    std::lock_guard<std::mutex> lock(S->mu);
    *st = S->stats;
    st->queued = (int64_t)S->pending.size();
    return WSM_OK;
}

extern "C" int wsm_server_destroy(wsm_server* S) {
    if (!S) return WSM_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_sched.notify_all();
    if (S->thread.joinable()) S->thread.join();
    destroy_lanes(S);
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
    return WSM_OK;
}
