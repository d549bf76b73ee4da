// wsm_api.cu -- handle lifetime, error reporting, the status word, and the
// initialisation step (Algorithm 2, first step; Sec. 3.2).
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "wsm_internal.cuh"

namespace wsm {

static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }

int fail(int code, const std::string& msg) {
    t_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(WSM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int check_handle(wsm_handle* h) {
    if (!h) return fail(WSM_E_INVAL, "null handle");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != h->device)
        return fail(WSM_E_STATE, "handle belongs to device " + std::to_string(h->device) +
                                     " but device " + std::to_string(dev) + " is current");
    return WSM_OK;
}

// Synchronise the stream, fetch the status word, clear it, and map it to a
// return code.
int read_status(wsm_handle* h, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(&h->host_ctrl->status, &h->ctrl->status, sizeof(unsigned),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&h->ctrl->status, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    unsigned st = h->host_ctrl->status;
    if (st & ST_TIMEOUT) return fail(WSM_E_TIMEOUT, "a device-side grid barrier timed out");
    if (st & ST_CAPACITY)
        return fail(WSM_E_CAPACITY, "more unique colors than the output capacity");
    if (st & ST_FEW_COLORS)
        return fail(WSM_E_INVAL, "an image has fewer unique colors than K (it was skipped)");
    if (st & ST_BAD_LABEL) return fail(WSM_E_INVAL, "a membership or palette index was >= K");
    return WSM_OK;
}

// splitmix64 (Steele, Lea, Flood 2014): draw r of the stream seeded with
// `seed` is the state seed + (r+1) * golden-gamma passed through the mixer.
__host__ __device__ static inline uint64_t splitmix_draw(uint64_t seed, uint64_t r) {
    uint64_t s = seed + 0x9E3779B97F4A7C15ull * (r + 1ull);
    s ^= s >> 30;
    s *= 0xBF58476D1CE4E5B9ull;
    s ^= s >> 27;
    s *= 0x94D049BB133111EBull;
    s ^= s >> 31;
    return s;
}

// Floyd's sampling (Bentley & Floyd, "A sample of brilliance", CACM 1987):
// K distinct integers from [0, n), each K-subset equally likely; returned
// in ascending order.
static std::vector<int64_t> floyd_sample(int64_t n, int K, uint64_t seed) {
    std::vector<int64_t> pick;
    pick.reserve(K);
    uint64_t r = 0;
    for (int64_t top = n - K; top < n; ++top) {
        int64_t t = (int64_t)(splitmix_draw(seed, r++) % (uint64_t)(top + 1));
        bool seen = std::find(pick.begin(), pick.end(), t) != pick.end();
        pick.push_back(seen ? top : t);
    }
    std::sort(pick.begin(), pick.end());
    return pick;
}

struct InitPick {
    uint32_t idx[WSM_MAX_K_WIDE];
};

// Memberships start at 0 (uint8 or uint16: bytes of zero either way).
__device__ __forceinline__ void zero_labels(void* labels, int64_t n, int label_bytes, int64_t t,
                                            int64_t nt) {
    uint8_t* p = static_cast<uint8_t*>(labels);
    for (int64_t q = t; q < n * label_bytes; q += nt) p[q] = 0;
}

__global__ void k_init(const uint32_t* __restrict__ colors, int64_t n_unique, int K,
                       const __grid_constant__ InitPick pick, float4* __restrict__ centers,
                       void* __restrict__ labels, int label_bytes) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = tid; k < K; k += nt) {
        const uint32_t c = colors[pick.idx[k]];
        centers[k] = make_float4((float)((c >> 16) & 255u), (float)((c >> 8) & 255u),
                                 (float)(c & 255u), 0.f);
    }
    zero_labels(labels, n_unique, label_bytes, tid, nt);
}

// The images of one initialisation launch: image i owns the blocks
// [first_blk[i], first_blk[i+1]) and reads its K sampled indices at
// pick + i * pick_stride.
struct InitItems {
    int n_items;
    int first_blk[kMaxBatch + 1];
    const uint32_t* colors[kMaxBatch];
    int64_t n_unique[kMaxBatch];
    int K[kMaxBatch];
    float4* centers[kMaxBatch];
    void* labels[kMaxBatch];
    const uint32_t* pick;
    int pick_stride;
    int label_bytes;
};

__global__ void k_init_batch(const __grid_constant__ InitItems B) {
    const int i = item_of_block(B.first_blk, B.n_items, blockIdx.x);
    const int G = B.first_blk[i + 1] - B.first_blk[i];
    const int64_t tid = (int64_t)(blockIdx.x - B.first_blk[i]) * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)G * blockDim.x;
    for (int64_t k = tid; k < B.K[i]; k += nt) {
        const uint32_t c = B.colors[i][B.pick[(size_t)i * B.pick_stride + k]];
        B.centers[i][k] = make_float4((float)((c >> 16) & 255u), (float)((c >> 8) & 255u),
                                      (float)(c & 255u), 0.f);
    }
    zero_labels(B.labels[i], B.n_unique[i], B.label_bytes, tid, nt);
}

// The initialisation of a batch whose N' values are on the device (written
// by the reduction): image i owns blocks [i * kInitBlocks, (i+1) * kInitBlocks)
// which zero its labels; the first of them also draws the K indices exactly
// as floyd_sample does on the host (the splitmix64 draws in parallel, the
// Floyd steps in order with a warp checking the earlier picks), sorts them
// and gathers the centers.  An image with N' < K gets ST_FEW_COLORS.
constexpr int kInitBlocks = 8;

struct InitDevItems {
    int n_items;
    const int64_t* n_dev;           // N' of item i at n_dev[i]
    const uint32_t* colors[kMaxBatch];
    int K[kMaxBatch];
    float4* centers[kMaxBatch];
    void* labels[kMaxBatch];
    uint64_t seed[kMaxBatch];
    unsigned* status;
    int label_bytes;
};

__global__ void __launch_bounds__(256) k_init_dev(const __grid_constant__ InitDevItems B) {
    __shared__ uint64_t s_draw[WSM_MAX_K_WIDE];
    __shared__ uint32_t s_pick[WSM_MAX_K_WIDE];
    __shared__ uint32_t s_sorted[WSM_MAX_K_WIDE];
    const int i = blockIdx.x / kInitBlocks, j = blockIdx.x % kInitBlocks;
    const int tid = threadIdx.x;
    const int64_t n = B.n_dev[i];
    const int K = B.K[i];
    if (n < K) {                                    // skipped: zero centers, flagged
        if (j == 0) {
            for (int k = tid; k < K; k += blockDim.x)
                B.centers[i][k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (tid == 0) atomicOr(B.status, ST_FEW_COLORS);
        }
        return;
    }
    zero_labels(B.labels[i], n, B.label_bytes, (int64_t)j * blockDim.x + tid,
                (int64_t)kInitBlocks * blockDim.x);
    if (j != 0) return;
    // Floyd step r draws t_r = draw_r mod (top_r + 1), top_r = n - K + r, and
    // takes t_r unless it is already taken, else top_r.  t_r is taken before
    // step r exactly when an earlier draw had the same value (that value was
    // taken then, as itself or already before), or when t_r = top_q for an
    // earlier step q that took top_q.  The first test needs no order (all
    // pairs at once).  The second links step r to the one earlier step
    // q = t_r - (n - K), so "took top" is the OR of the first test along a
    // chain of such links: pointer jumping resolves every chain in
    // ceil(log2 K) rounds, each OR-ing the value at the end of a pointer and
    // doubling the pointer's reach (s_sorted holds the pointers meanwhile).
    for (int r = tid; r < K; r += blockDim.x)
        s_draw[r] = splitmix_draw(B.seed[i], (uint64_t)r) % (uint64_t)(n - K + r + 1);
    __syncthreads();
    constexpr uint32_t kNone = 0xFFFFFFFFu;
    const int64_t base = n - K;
    for (int r = tid; r < K; r += blockDim.x) {
        const uint64_t t = s_draw[r];
        bool seen = false;
        for (int q = 0; q < r; ++q) seen |= s_draw[q] == t;
        s_pick[r] = seen ? 1u : 0u;                  // for now: t_r equals an earlier draw
        const int64_t q = (int64_t)t - base;
        s_sorted[r] = (q >= 0 && q < r) ? (uint32_t)q : kNone;
    }
    __syncthreads();
    constexpr int kPer = WSM_MAX_K_WIDE / 256;       // steps per thread (256 threads)
    for (int reach = 1; reach < K; reach <<= 1) {
        uint32_t v[kPer], pp[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int r = tid + u * 256;
            v[u] = 0u;
            pp[u] = kNone;
            if (r < K) {
                v[u] = s_pick[r];
                pp[u] = s_sorted[r];
                if (pp[u] != kNone) {
                    v[u] |= s_pick[pp[u]];
                    pp[u] = s_sorted[pp[u]];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int r = tid + u * 256;
            if (r < K) {
                s_pick[r] = v[u];
                s_sorted[r] = pp[u];
            }
        }
        __syncthreads();
    }
    for (int r = tid; r < K; r += blockDim.x)
        s_pick[r] = s_pick[r] ? (uint32_t)(n - K + r) : (uint32_t)s_draw[r];
    __syncthreads();
    for (int r = tid; r < K; r += blockDim.x) {     // the picks are distinct: rank = position
        const uint32_t v = s_pick[r];
        int rank = 0;
        for (int q = 0; q < K; ++q) rank += s_pick[q] < v;
        s_sorted[rank] = v;
    }
    __syncthreads();
    for (int k = tid; k < K; k += blockDim.x) {
        const uint32_t c = B.colors[i][s_sorted[k]];
        B.centers[i][k] = make_float4((float)((c >> 16) & 255u), (float)((c >> 8) & 255u),
                                      (float)(c & 255u), 0.f);
    }
}

int init_items_dev(wsm_handle* h, const wsm_item* items, int n_items, const uint64_t* seeds,
                   cudaStream_t s) {
    for (int i0 = 0; i0 < n_items; i0 += kMaxBatch) {
        InitDevItems B;
        B.n_items = std::min(kMaxBatch, n_items - i0);
        B.n_dev = h->batch_nu + i0;
        B.status = &h->ctrl->status;
        B.label_bytes = h->label_bytes;
        for (int q = 0; q < B.n_items; ++q) {
            const wsm_item& it = items[i0 + q];
            B.colors[q] = it.d_colors;
            B.K[q] = it.K;
            B.centers[q] = reinterpret_cast<float4*>(it.d_centers);
            B.labels[q] = it.d_labels;
            B.seed[q] = seeds[i0 + q];
        }
        k_init_dev<<<B.n_items * kInitBlocks, 256, 0, s>>>(B);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "init launch");
    }
    return WSM_OK;
}

int iterate_kernel_setup(wsm_handle* h);   // wsm_iterate.cu

void free_slots(wsm_handle* h) {
    void* ptrs[] = {h->tab,   h->tab_nb, h->sums,      h->sums64,   h->acc,       h->trace,
                    h->lut,   h->slot_ctrl, h->hist,   h->bitmap,   h->blk_total, h->batch_nu,
                    h->batch_mse, h->pick, h->plan, h->grid, h->bkt_count, h->bkt_cursor,
                    h->keys16, h->bkt_work, h->bkt_nwork, h->slot_weight};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    void* host_ptrs[] = {h->host_nu, h->host_mse, h->host_pick};
    for (void* p : host_ptrs)
        if (p) cudaFreeHost(p);
    h->hist = nullptr;
    h->bitmap = nullptr;
    h->blk_total = nullptr;
    h->bkt_count = nullptr;
    h->bkt_cursor = nullptr;
    h->keys16 = nullptr;
    h->bkt_work = nullptr;
    h->bkt_nwork = nullptr;
    h->batch_nu = nullptr;
    h->batch_mse = nullptr;
    h->pick = nullptr;
    h->plan = nullptr;
    h->slot_weight = nullptr;
    h->grid = nullptr;
    h->host_nu = nullptr;
    h->host_mse = nullptr;
    h->host_pick = nullptr;
    h->rslots = 0;
    h->tab = nullptr;
    h->tab_nb = nullptr;
    h->sums = nullptr;
    h->sums64 = nullptr;
    h->acc = nullptr;
    h->trace = nullptr;
    h->lut = nullptr;
    h->slot_ctrl = nullptr;
    h->slots = 0;
}

// Per-image scratch for `slots` images (replaces any previous slots), and
// unique-color reduction scratch for min(slots, kReduceSlots) images.
int alloc_slots(wsm_handle* h, int slots) {
    free_slots(h);
    const size_t kk = (size_t)h->max_K * h->max_K, n = (size_t)slots;
    const size_t r = (size_t)std::min(slots, kReduceSlots);
    struct {
        void** p;
        size_t bytes;
    } allocs[] = {
        {(void**)&h->tab, sizeof(float4) * kk * n},
        {(void**)&h->tab_nb, kk * n * h->label_bytes},
        {(void**)&h->sums, sizeof(unsigned) * 2 * kCopies * 5 * (size_t)h->max_K * n},
        {(void**)&h->sums64, sizeof(unsigned long long) * 2 * kCopies * 4 * n},
        {(void**)&h->acc, sizeof(unsigned long long) * 4 * (size_t)h->max_K * n},
        {(void**)&h->trace, sizeof(double) * kMaxTrace * n},
        {(void**)&h->lut, (size_t)kHistBins * n * h->label_bytes},
        {(void**)&h->slot_ctrl, sizeof(Ctrl) * n},
        {(void**)&h->hist, sizeof(uint32_t) * kHistBins * r},
        {(void**)&h->bitmap, sizeof(uint32_t) * kMapWords * r},
        {(void**)&h->blk_total, sizeof(uint32_t) * kScanBlocks * r},
        {(void**)&h->bkt_count, sizeof(uint32_t) * kBuckets * r},
        {(void**)&h->bkt_cursor, sizeof(uint32_t) * kBuckets * r},
        {(void**)&h->keys16, sizeof(uint16_t) * keys_stride(h) * r},
        {(void**)&h->bkt_work, sizeof(uint4) * (size_t)bkt_max_work(h->max_pixels) * r},
        {(void**)&h->bkt_nwork, sizeof(int) * r},
        {(void**)&h->batch_nu, sizeof(int64_t) * n},
        {(void**)&h->batch_mse, sizeof(double) * n},
        {(void**)&h->pick, sizeof(uint32_t) * (size_t)h->max_K * n},
        {(void**)&h->plan, sizeof(int) * (n / kMaxBatch + 1) * (kMaxBatch + 1)},
        {(void**)&h->slot_weight, sizeof(int) * n},
        {(void**)&h->grid, (size_t)kGridCells * n * h->label_bytes},
    };
    for (auto& a : allocs) {
        cudaError_t e = cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            free_slots(h);
            return fail(WSM_E_NOMEM, std::string("cudaMalloc (image slots): ") +
                                         cudaGetErrorString(e));
        }
    }
    struct {
        void** p;
        size_t bytes;
    } host_allocs[] = {
        {(void**)&h->host_nu, sizeof(int64_t) * n},
        {(void**)&h->host_mse, sizeof(double) * n},
        {(void**)&h->host_pick, sizeof(uint32_t) * (size_t)h->max_K * n},
    };
    for (auto& a : host_allocs) {
        cudaError_t e = cudaMallocHost(a.p, a.bytes);
        if (e != cudaSuccess) {
            free_slots(h);
            return fail(WSM_E_NOMEM, std::string("cudaMallocHost (image slots): ") +
                                         cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaMemset(h->slot_ctrl, 0, sizeof(Ctrl) * n);
    if (e == cudaSuccess) e = cudaMemset(h->hist, 0, sizeof(uint32_t) * kHistBins * r);
    if (e == cudaSuccess) e = cudaMemset(h->bitmap, 0, sizeof(uint32_t) * kMapWords * r);
    if (e == cudaSuccess) e = cudaMemset(h->bkt_count, 0, sizeof(uint32_t) * kBuckets * r);
    if (e == cudaSuccess) e = cudaMemset(h->slot_weight, 0, sizeof(int) * n);
    if (e == cudaSuccess)
        e = cudaMemset(h->acc, 0, sizeof(unsigned long long) * 4 * (size_t)h->max_K * n);
    if (e != cudaSuccess) {
        free_slots(h);
        return cuda_fail(e, "slot initialisation");
    }
    h->slots = slots;
    h->rslots = (int)r;
    return WSM_OK;
}

}  // namespace wsm

using namespace wsm;

extern "C" const char* wsm_last_error(void) { return t_last_error.c_str(); }

extern "C" int wsm_create(wsm_handle** out, int max_K, int64_t max_pixels, int64_t max_unique) {
    if (!out) return fail(WSM_E_INVAL, "null output pointer");
    *out = nullptr;
    if (max_K < 1 || max_K > WSM_MAX_K_WIDE)
        return fail(WSM_E_INVAL, "max_K must be in [1, 1024]");
    if (max_pixels < 1 || max_pixels > WSM_MAX_PIXELS)
        return fail(WSM_E_INVAL, "max_pixels must be in [1, 2^24]");
    if (max_unique < 1 || max_unique > max_pixels)
        return fail(WSM_E_INVAL, "max_unique must be in [1, max_pixels]");
    wsm_handle* h = new (std::nothrow) wsm_handle();
    if (!h) return fail(WSM_E_NOMEM, "host allocation failed");
    h->max_K = max_K;
    h->label_bytes = max_K > WSM_MAX_K ? 2 : 1;
    h->max_pixels = max_pixels;
    h->max_unique = max_unique;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount,
                                                      h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "device query");
    }
    int rc = iterate_kernel_setup(h);
    if (rc != WSM_OK) {
        delete h;
        return rc;
    }
    const int gk = std::min(max_K, WSM_MAX_K);
    struct {
        void** p;
        size_t bytes;
    } allocs[] = {
        {(void**)&h->mse_part, sizeof(double) * 1032},   // 1024 partials + result
        {(void**)&h->ctrl, sizeof(Ctrl)},
        // the gradient calls take palettes of at most 256 colors
        {(void**)&h->grad_tab, sizeof(float4) * (size_t)gk * gk},
        {(void**)&h->grad_nb, (size_t)gk * gk},
        {(void**)&h->grad_part, sizeof(float4) * (size_t)grad_blocks(h) * (gk + 1)},
    };
    for (auto& a : allocs) {
        e = cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            wsm_destroy(h);
            return fail(WSM_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    rc = alloc_slots(h, 1);
    if (rc != WSM_OK) {
        wsm_destroy(h);
        return rc;
    }
    e = cudaMallocHost((void**)&h->host_ctrl, sizeof(Ctrl));
    if (e != cudaSuccess) {
        wsm_destroy(h);
        return fail(WSM_E_NOMEM, "cudaMallocHost failed");
    }
    e = cudaEventCreateWithFlags(&h->pick_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(h->ctrl, 0, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        wsm_destroy(h);
        return cuda_fail(e, "scratch initialisation");
    }
    *out = h;
    return WSM_OK;
}

extern "C" int wsm_destroy(wsm_handle* h) {
    if (!h) return WSM_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (h->device >= 0 && prev != h->device) cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    free_slots(h);
    void* dev_ptrs[] = {h->mse_part, h->ctrl, h->grad_tab, h->grad_nb, h->grad_part};
    for (void* p : dev_ptrs)
        if (p) cudaFree(p);
    if (h->host_ctrl) cudaFreeHost(h->host_ctrl);
    if (h->pick_ready) cudaEventDestroy(h->pick_ready);
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    delete h;
    return WSM_OK;
}

extern "C" int wsm_reserve_batch(wsm_handle* h, int max_items) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (max_items < 1 || max_items > 4096)
        return fail(WSM_E_INVAL, "max_items must be in [1, 4096]");
    if (max_items <= h->slots) return WSM_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "device sync");
    rc = alloc_slots(h, max_items);
    if (rc != WSM_OK) {
        int rc1 = alloc_slots(h, 1);   // keep the handle usable for single images
        (void)rc1;
        return rc;
    }
    return WSM_OK;
}

extern "C" int wsm_sync_status(wsm_handle* h, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    return read_status(h, (cudaStream_t)stream);
}

extern "C" int wsm_init(wsm_handle* h, const uint32_t* d_colors, int64_t n_unique, int K,
                        uint64_t seed, float* d_centers, void* d_labels, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (K < 1 || K > h->max_K) return fail(WSM_E_INVAL, "K out of [1, max_K]");
    if (n_unique < K || n_unique > h->max_unique)
        return fail(WSM_E_INVAL, "n_unique must be in [K, max_unique]");
    if (!d_colors || !d_centers || !d_labels) return fail(WSM_E_INVAL, "null device pointer");
    std::vector<int64_t> pick = floyd_sample(n_unique, K, seed);
    InitPick p;
    for (int k = 0; k < K; ++k) p.idx[k] = (uint32_t)pick[k];
    int threads = 256;
    int64_t want = (n_unique + threads - 1) / threads;
    int blocks = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)h->sms * 8);
    k_init<<<blocks, threads, 0, (cudaStream_t)stream>>>(d_colors, n_unique, K, p,
                                                          (float4*)d_centers, d_labels,
                                                          h->label_bytes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_init launch");
    return WSM_OK;
}

extern "C" int wsm_init_batch(wsm_handle* h, const wsm_item* items, int n_items,
                              const uint64_t* seeds, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (n_items < 0 || (n_items > 0 && (!items || !seeds)))
        return fail(WSM_E_INVAL, "bad item list");
    if (n_items > h->slots)
        return fail(WSM_E_INVAL, "more items than reserved slots (wsm_reserve_batch)");
    for (int i = 0; i < n_items; ++i) {
        const wsm_item& it = items[i];
        if (it.K < 1 || it.K > h->max_K) return fail(WSM_E_INVAL, "K out of [1, max_K]");
        if (it.n_unique < it.K || it.n_unique > h->max_unique)
            return fail(WSM_E_INVAL, "n_unique must be in [K, max_unique]");
        if (!it.d_colors || !it.d_centers || !it.d_labels)
            return fail(WSM_E_INVAL, "null device pointer");
        if ((uintptr_t)it.d_centers & 15)
            return fail(WSM_E_INVAL, "centers must be 16-byte aligned");
    }
    if (n_items == 0) return WSM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // the previous call's copy out of the staging buffer must be done
    cudaError_t e = cudaEventSynchronize(h->pick_ready);
    if (e != cudaSuccess) return cuda_fail(e, "staging buffer wait");
    for (int i = 0; i < n_items; ++i) {
        std::vector<int64_t> pick = floyd_sample(items[i].n_unique, items[i].K, seeds[i]);
        for (int k = 0; k < items[i].K; ++k)
            h->host_pick[(size_t)i * h->max_K + k] = (uint32_t)pick[k];
    }
    e = cudaMemcpyAsync(h->pick, h->host_pick, sizeof(uint32_t) * (size_t)h->max_K * n_items,
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(h->pick_ready, s);
    if (e != cudaSuccess) return cuda_fail(e, "initial index copy");
    for (int i0 = 0; i0 < n_items; i0 += kMaxBatch) {
        InitItems B;
        B.n_items = std::min(kMaxBatch, n_items - i0);
        B.pick = h->pick + (size_t)i0 * h->max_K;
        B.pick_stride = h->max_K;
        B.label_bytes = h->label_bytes;
        B.first_blk[0] = 0;
        for (int q = 0; q < B.n_items; ++q) {
            const wsm_item& it = items[i0 + q];
            B.colors[q] = it.d_colors;
            B.n_unique[q] = it.n_unique;
            B.K[q] = it.K;
            B.centers[q] = reinterpret_cast<float4*>(it.d_centers);
            B.labels[q] = it.d_labels;
            const int64_t want = (it.n_unique + 255) / 256;   // >= 1 block, covers K <= N'
            B.first_blk[q + 1] = B.first_blk[q] + (int)std::min<int64_t>(want, 64);
        }
        k_init_batch<<<B.first_blk[B.n_items], 256, 0, s>>>(B);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "init launch");
    }
    return WSM_OK;
}
