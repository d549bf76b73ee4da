// wsm_pipeline.cu -- the whole path for a batch of images with no host
// synchronisation, and the autotuner of the persistent kernel's launch shape.
//
// wsm_quantize_batch runs unique colors (Sec. 2) -> initialisation
// (Algorithm 2, first step) -> the Sort-Means iterations with the Sec. 3.2
// stop rule -> final assignment and pixel mapping (Sec. 1) -> MSE (Eq. 2,
// from the final assignment's squared distances) for every image,
// stream-ordered.  The number of unique colors N' of each
// image stays on the device: the initialisation draws its Floyd sample from
// it there, and the persistent launches split their blocks from it there
// (k_plan), so the host never waits and the whole sequence can be captured
// into a CUDA graph and replayed on new pixels.
//
// wsm_autotune_batch times every resident launch shape (threads per block x
// blocks per SM) of the persistent kernel on a batch and keeps the fastest
// for the handle; every shape gives the same results bit for bit (the
// reductions are exact), so the choice is about time only.
#include <algorithm>
#include <vector>

#include "wsm_internal.cuh"

namespace wsm {

// Eq. 2 of image i from its final assignment: MSE = map_sse * 2^-20 / n.
// The assignment summed, over the unique colors, count * (squared distance
// to the assigned center truncated to 2^-20 units), with the distances the
// per-pixel MSE computes, so this equals that MSE bit for bit.
struct MapMse {
    int n_items;
    int64_t n[kMaxBatch];
};

__global__ void k_mse_from_map(const __grid_constant__ MapMse M, const Ctrl* __restrict__ ctrl,
                               double* __restrict__ out, double* __restrict__ user) {
    for (int i = threadIdx.x; i < M.n_items; i += blockDim.x) {
        const double m = (double)ctrl[i].map_sse * (1.0 / 1048576.0) / (double)M.n[i];
        out[i] = m;
        if (user) user[i] = m;
    }
}

static int mse_from_map(wsm_handle* h, const wsm_item* items, int n_items, double* d_mse,
                        cudaStream_t s) {
    for (int i0 = 0; i0 < n_items; i0 += kMaxBatch) {
        MapMse M;
        M.n_items = std::min(kMaxBatch, n_items - i0);
        for (int q = 0; q < M.n_items; ++q) M.n[q] = items[i0 + q].n_pixels;
        k_mse_from_map<<<1, 64, 0, s>>>(M, h->slot_ctrl + i0, h->batch_mse + i0,
                                        d_mse ? d_mse + i0 : nullptr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "MSE launch");
    }
    return WSM_OK;
}

static int check_batch(wsm_handle* h, const wsm_item* items, int n_items, const uint64_t* seeds,
                       int max_iter) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (n_items < 0 || (n_items > 0 && (!items || !seeds)))
        return fail(WSM_E_INVAL, "bad item list");
    if (n_items > h->slots)
        return fail(WSM_E_INVAL, "more items than reserved slots (wsm_reserve_batch)");
    if (max_iter < 0 || max_iter > kMaxTrace)
        return fail(WSM_E_INVAL, "max_iter must be in [0, 4096]");
    for (int i = 0; i < n_items; ++i) {
        const wsm_item& it = items[i];
        rc = check_pixels(h, it);
        if (rc != WSM_OK) return rc;
        if (it.K < 1 || it.K > h->max_K) return fail(WSM_E_INVAL, "K out of [1, max_K]");
        if (!it.d_colors || !it.d_counts || !it.d_centers || !it.d_labels || !it.d_index)
            return fail(WSM_E_INVAL, "null device pointer");
        if ((uintptr_t)it.d_centers & 15)
            return fail(WSM_E_INVAL, "centers must be 16-byte aligned");
    }
    return WSM_OK;
}

// Two blocks meet at a barrier that waits for three: the wait can only run
// out (the failure the persistent kernel's barriers guard against).
__global__ void k_barrier_timeout(unsigned* counter, unsigned* status,
                                  unsigned long long limit_ns) {
    grid_sync(counter, status, gridDim.x + 1, limit_ns);
}

// Independent FMA chains (kFmaChains per thread, no memory traffic in the
// loop); the sum is stored only if it equals a value it cannot take, so the
// chains stay live.
constexpr int kFmaChains = 16;

__global__ void __launch_bounds__(256) k_ffma(float b, float c, int iters, float* sink) {
    float a[kFmaChains];
#pragma unroll
    for (int q = 0; q < kFmaChains; ++q) a[q] = (float)(threadIdx.x + q) * 1e-3f;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < kFmaChains; ++q) a[q] = fmaf(a[q], b, c);
    }
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < kFmaChains; ++q) sum += a[q];
    if (sum == -1.0f) *sink = sum;
}

}  // namespace wsm

using namespace wsm;

extern "C" int wsm_selftest_barrier_timeout(wsm_handle* h, int limit_ms, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (limit_ms < 1 || limit_ms > 2000) return fail(WSM_E_INVAL, "limit_ms must be in [1, 2000]");
    cudaStream_t s = (cudaStream_t)stream;
    // slot 0's barrier counter, cleared before and after (the next launch clears it too)
    cudaError_t e = cudaMemsetAsync(&h->slot_ctrl[0].bar_count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "self-test set-up");
    k_barrier_timeout<<<2, 32, 0, s>>>(&h->slot_ctrl[0].bar_count, &h->ctrl->status,
                                       (unsigned long long)limit_ms * 1000000ull);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(&h->slot_ctrl[0].bar_count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
    return read_status(h, s);
}

extern "C" int wsm_quantize_batch_stages(wsm_handle* h, const wsm_item* items, int n_items,
                                         const uint64_t* seeds, int max_iter, double eps,
                                         int64_t* d_n_unique, int* d_iters, double* d_mse,
                                         unsigned stages, wsm_stream stream) {
    int rc = check_batch(h, items, n_items, seeds, max_iter);
    if (rc != WSM_OK) return rc;
    if (stages & ~(unsigned)WSM_STAGE_ALL) return fail(WSM_E_INVAL, "unknown stage bits");
    if (n_items == 0) return WSM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (stages & WSM_STAGE_REDUCE) rc = reduce_items(h, items, n_items, s);
    if (rc == WSM_OK && (stages & WSM_STAGE_INIT)) rc = init_items_dev(h, items, n_items, seeds, s);
    if (rc == WSM_OK && (stages & WSM_STAGE_ITERATE)) {
        // the persistent kernel writes N' and the iterations run of every image
        rc = iterate_items(h, items, n_items, max_iter, eps, h->batch_nu, s, d_n_unique,
                           d_iters);
    }
    if (rc == WSM_OK && (stages & WSM_STAGE_MAP))
        rc = map_items(h, items, n_items, h->batch_nu, true, s);
    if (rc == WSM_OK && (stages & WSM_STAGE_INDEX))
        rc = pixel_items(h, items, n_items, true, nullptr, h->batch_nu, s);
    if (rc == WSM_OK && (stages & WSM_STAGE_DISTORTION))
        rc = mse_from_map(h, items, n_items, d_mse, s);
    return rc;
}

extern "C" int wsm_quantize_batch(wsm_handle* h, const wsm_item* items, int n_items,
                                  const uint64_t* seeds, int max_iter, double eps,
                                  int64_t* d_n_unique, int* d_iters, double* d_mse,
                                  wsm_stream stream) {
    return wsm_quantize_batch_stages(h, items, n_items, seeds, max_iter, eps, d_n_unique, d_iters,
                                     d_mse, WSM_STAGE_ALL, stream);
}

extern "C" int wsm_batch_stats(wsm_handle* h, int n_items, int64_t* evaluated, int* iters,
                               wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (n_items < 0 || n_items > h->slots) return fail(WSM_E_INVAL, "n_items out of [0, slots]");
    if (n_items == 0) return WSM_OK;
    rc = read_status(h, (cudaStream_t)stream);
    if (rc != WSM_OK) return rc;
    std::vector<Ctrl> c(n_items);
    cudaError_t e = cudaMemcpy(c.data(), h->slot_ctrl, sizeof(Ctrl) * n_items,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats copy");
    for (int i = 0; i < n_items; ++i) {
        if (evaluated) evaluated[i] = (int64_t)c[i].evaluated;
        if (iters) iters[i] = c[i].iters_done;
    }
    return WSM_OK;
}

extern "C" int wsm_set_grid_limit(wsm_handle* h, int blocks) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (blocks != 0 && blocks < kMaxBatch)
        return fail(WSM_E_INVAL, "a grid limit must be 0 (none) or at least 48 blocks");
    h->grid_limit = blocks;
    return WSM_OK;
}

extern "C" int wsm_set_first_pass_start(wsm_handle* h, int candidate) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    h->cand_start = candidate != 0;
    return WSM_OK;
}

extern "C" int wsm_set_launch_shape(wsm_handle* h, int shape) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (shape < 0 || shape >= kNumIterShapes) return fail(WSM_E_INVAL, "shape out of range");
    if (!h->shape_ok[shape])
        return fail(WSM_E_INVAL, "that launch shape cannot be resident at this handle's max_K");
    h->iter_shape = shape;
    return WSM_OK;
}

extern "C" int wsm_launch_shape(wsm_handle* h, int shape, int* threads, int* blocks_per_sm,
                                int* resident) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (shape < 0) shape = h->iter_shape;
    if (shape >= kNumIterShapes) return fail(WSM_E_INVAL, "shape out of range");
    if (threads) *threads = kIterShapes[shape].threads;
    if (blocks_per_sm) *blocks_per_sm = kIterShapes[shape].blocks_per_sm;
    if (resident) *resident = h->shape_ok[shape] ? 1 : 0;
    return shape;
}

// Work weights of the images for the device-side block split (k_plan).  The
// split gives each image blocks in proportion to its unique colors, but the
// cost per color differs between images (visit lengths), and the launch
// ends with its slowest image group.  kWeighRounds rounds: run the iterations with
// the current weights, read each group's time from the globaltimer stamps in
// its control block, multiply each image's weight by its time over the mean
// time (a slower group gets more blocks), and rescale so that the weighted
// demand keeps its unweighted total.  Weights only move blocks between
// images; every split gives the same results bit for bit.
// Rounds of the weighing: a group's time has a part that more blocks do not
// shorten (barriers, centers, rows), so each round moves the weights only part
// of the way; six rounds measured faster than three on the 8-image step
// (iterations 0.413-0.416 vs 0.421-0.422 ms over three runs each).
constexpr int kWeighRounds = 6;

int calibrate_weights(wsm_handle* h, const wsm_item* items, int n_items, const uint64_t* seeds,
                      int max_iter, double eps, cudaStream_t s) {
    std::vector<double> w(n_items, 1.0);
    cudaError_t e = cudaMemsetAsync(h->slot_weight, 0, sizeof(int) * n_items, s);
    if (e != cudaSuccess) return cuda_fail(e, "weights reset");
    if (n_items < 2) return WSM_OK;
    std::vector<Ctrl> ctrl(n_items);
    std::vector<int> wi(n_items);
    std::vector<int64_t> nu(n_items);
    for (int round = 0; round < kWeighRounds; ++round) {
        int rc = init_items_dev(h, items, n_items, seeds, s);
        if (rc == WSM_OK) rc = iterate_items(h, items, n_items, max_iter, eps, h->batch_nu, s);
        if (rc != WSM_OK) return rc;
        e = cudaMemcpyAsync(ctrl.data(), h->slot_ctrl, sizeof(Ctrl) * n_items,
                            cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(nu.data(), h->batch_nu, sizeof(int64_t) * n_items,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "weights timing copy");
        rc = read_status(h, s);
        if (rc != WSM_OK) return rc;
        double mean = 0.0;
        int timed = 0;
        for (int i = 0; i < n_items; ++i)
            if (ctrl[i].t_end > ctrl[i].t_start) {
                mean += (double)(ctrl[i].t_end - ctrl[i].t_start);
                ++timed;
            }
        if (timed < 2) return WSM_OK;
        mean /= timed;
        double sum_old = 0.0, sum_new = 0.0;
        for (int i = 0; i < n_items; ++i) {
            const double base = (double)std::max<int64_t>(nu[i], 1);   // the demand's scale
            sum_old += base;
            if (ctrl[i].t_end > ctrl[i].t_start)
                w[i] *= (double)(ctrl[i].t_end - ctrl[i].t_start) / mean;
            w[i] = std::min(16.0, std::max(1.0 / 16.0, w[i]));
            sum_new += base * w[i];
        }
        for (int i = 0; i < n_items; ++i) {
            const double v = w[i] * sum_old / sum_new;
            wi[i] = (int)std::min(16384.0, std::max(64.0, v * 1024.0 + 0.5));
        }
        e = cudaMemcpyAsync(h->slot_weight, wi.data(), sizeof(int) * n_items,
                            cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "weights copy");
    }
    return WSM_OK;
}

extern "C" int wsm_weigh_batch(wsm_handle* h, const wsm_item* items, int n_items,
                               const uint64_t* seeds, int max_iter, double eps,
                               wsm_stream stream) {
    int rc = check_batch(h, items, n_items, seeds, max_iter);
    if (rc != WSM_OK) return rc;
    if (n_items == 0) return WSM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    rc = reduce_items(h, items, n_items, s);
    if (rc != WSM_OK) return rc;
    return calibrate_weights(h, items, n_items, seeds, max_iter, eps, s);
}

extern "C" int wsm_autotune_batch(wsm_handle* h, const wsm_item* items, int n_items,
                                  const uint64_t* seeds, int max_iter, double eps, int repeats,
                                  float* times_ms, wsm_stream stream) {
    int rc = check_batch(h, items, n_items, seeds, max_iter);
    if (rc != WSM_OK) return rc;
    if (n_items == 0) return h->iter_shape;
    if (repeats < 1 || repeats > 100) return fail(WSM_E_INVAL, "repeats must be in [1, 100]");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return cuda_fail(e, "autotune events");
    }
    const int saved = h->iter_shape;
    int best = -1;
    float best_ms = 0.f;
    rc = reduce_items(h, items, n_items, s);
    for (int q = 0; q < kNumIterShapes && rc == WSM_OK; ++q) {
        float t_min = -1.f;
        if (h->shape_ok[q]) {
            h->iter_shape = q;
            for (int r = 0; r < repeats && rc == WSM_OK; ++r) {
                // the initialisation restores the starting centers and labels
                rc = init_items_dev(h, items, n_items, seeds, s);
                if (rc != WSM_OK) break;
                e = cudaEventRecord(a, s);
                if (e == cudaSuccess) {
                    rc = iterate_items(h, items, n_items, max_iter, eps, h->batch_nu, s);
                    if (rc != WSM_OK) break;
                    e = cudaEventRecord(b, s);
                }
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "autotune timing");
                    break;
                }
                if (t_min < 0.f || ms < t_min) t_min = ms;
            }
            if (rc == WSM_OK && (best < 0 || t_min < best_ms)) {
                best = q;
                best_ms = t_min;
            }
        }
        if (times_ms) times_ms[q] = t_min;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc == WSM_OK) rc = read_status(h, s);
    if (rc != WSM_OK || best < 0) {
        h->iter_shape = saved;
        return rc != WSM_OK ? rc : fail(WSM_E_CUDA, "no launch shape could be timed");
    }
    h->iter_shape = best;
    rc = calibrate_weights(h, items, n_items, seeds, max_iter, eps, s);
    if (rc != WSM_OK) return rc;
    return best;
}

extern "C" int wsm_measure_fp32(wsm_handle* h, int repeats, double* tflops, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (repeats < 1 || repeats > 20) return fail(WSM_E_INVAL, "repeats must be in [1, 20]");
    if (!tflops) return fail(WSM_E_INVAL, "null output");
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = 8 * h->sms, threads = 256, iters = 32768;
    float* sink = reinterpret_cast<float*>(h->mse_part);   // never written in practice
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = -1.f;
    for (int r = 0; r <= repeats && e == cudaSuccess; ++r) {
        e = cudaEventRecord(a, s);
        if (e == cudaSuccess) {
            k_ffma<<<blocks, threads, 0, s>>>(0.999999f, 1e-6f, iters, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && r > 0 && (best < 0.f || ms < best)) best = ms;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "FP32 measurement");
    const double flop = 2.0 * kFmaChains * (double)iters * threads * blocks;
    *tflops = flop / (best * 1e-3) / 1e12;
    return WSM_OK;
}
