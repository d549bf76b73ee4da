// wsm_iterate.cu -- the Sort-Means loop of Algorithm 2 (Sec. 2) as one
// persistent cooperative kernel, used both for the iterations (wsm_iterate)
// and for the final assignment before pixel mapping (wsm_map).
//
// One launch runs every iteration.  Per iteration:
//   phase A (all blocks)  new centers c_k = S_k / W_k from the integer sums
//                         of the previous pass (correctly rounded to FP32,
//                         an empty cluster keeps its center), SSE of the
//                         previous pass and the Sec. 3.2 stop test (every
//                         block computes the same values in the same order,
//                         so all take the same decision); then block b builds
//                         rows p = b, b+G, ... of the sorted center table.
//   grid barrier
//   phase B (all blocks)  the pruned nearest-center search for a contiguous
//                         chunk of the unique colors, with the cluster sums
//                         accumulated in shared memory and flushed to global
//                         int64 once per block, plus the block's SSE partial.
//   grid barrier
// Row p of the table holds, nearest first, (d[p][t] / 4, c_t) for every
// center t: the stop test d[p][t] >= 4 prev_dist becomes row[j].x >= prev
// (scaling by 4 is exact), and the visited center's coordinates come with
// the same 16-byte load.  The center index of an entry is only read when a
// visited center becomes the new minimum.
#include <algorithm>
#include <mutex>

#include "wsm_internal.cuh"

namespace wsm {

struct SortMeansParams {
    const uint32_t* colors;
    const uint32_t* counts;
    int64_t n;
    int K;
    float4* centers;       // [K] in/out (read-only in the map mode)
    uint8_t* labels;       // [n] in/out
    int max_iter;
    double eps;
    float4* tab;           // [K*K] rows of (d/4, c.x, c.y, c.z), nearest first
    uint8_t* tab_nb;       // [K*K] center index of each entry
    unsigned long long* acc;   // [2][K][4]
    double* sse_part;      // [2][gridDim.x]
    double* trace;         // [kMaxTrace]
    uint8_t* lut;          // map mode: [2^24] color -> label
    Ctrl* ctrl;
};

// fl32(S / W) rounded to nearest-even, for 0 <= S < 2^32 and 1 <= W < 2^25,
// from exact integer arithmetic: a 64-bit quotient carrying at least 26
// significant bits, then rounding on the dropped bits and the remainder.
__device__ __forceinline__ float div_rn_u32(unsigned long long S, unsigned long long W) {
    if (S == 0) return 0.f;
    int ls = 63 - __clzll((long long)S);
    int lw = 63 - __clzll((long long)W);
    int k = min(max(26 - ls + lw, 0), 63 - ls); // S * 2^k / W lies in [2^25, 2^27)
    unsigned long long num = S << k;
    unsigned long long q = num / W;
    bool sticky = (num - q * W) != 0;
    int nb = 64 - __clzll((long long)q);
    int shift = max(nb - 24, 1);                // keep 24 significant bits
    unsigned long long m = q >> shift;
    unsigned long long rest = q & ((1ull << shift) - 1);
    unsigned long long half = 1ull << (shift - 1);
    if (rest > half || (rest == half && (sticky || (m & 1)))) m += 1;
    return ldexpf((float)m, shift - k);
}

template <bool kMap>
__global__ void __launch_bounds__(kIterThreads) k_sortmeans(SortMeansParams P) {
    extern __shared__ float4 smem[];
    const int K = P.K;
    float4* s_c = smem;                                       // [K] centers
    unsigned* s_acc = reinterpret_cast<unsigned*>(s_c + K);   // [K][4] block sums
    float* s_row = reinterpret_cast<float*>(s_acc + 4 * K);   // [K] one table row
    __shared__ double s_red[kIterThreads / 32];
    __shared__ unsigned long long s_ev[kIterThreads / 32];
    __shared__ int s_stop;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    for (int k = tid; k < K; k += blockDim.x) s_c[k] = P.centers[k];
    __syncthreads();

    double prev_sse = 0.0;
    unsigned long long evaluated = 0;
    int it = 0;
    for (;;) {
        // ---------------- phase A ----------------
        if (!kMap) {
            if (it > 0) {
                const unsigned long long* A = P.acc + (size_t)((it - 1) & 1) * 4 * K;
                for (int k = tid; k < K; k += blockDim.x) {
                    unsigned long long W = A[4 * k + 3];
                    if (W) {
                        s_c[k] = make_float4(div_rn_u32(A[4 * k + 0], W),
                                             div_rn_u32(A[4 * k + 1], W),
                                             div_rn_u32(A[4 * k + 2], W), 0.f);
                    }
                }
                if (wid == 0) {
                    const double* part = P.sse_part + (size_t)((it - 1) & 1) * G;
                    double s = 0.0;
                    for (int i = lane; i < G; i += 32) s += part[i];
                    unsigned long long Nw = 0;
                    for (int k = lane; k < K; k += 32) Nw += A[4 * k + 3];
                    for (int o = 16; o > 0; o >>= 1) {
                        s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
                        Nw += __shfl_xor_sync(0xFFFFFFFFu, Nw, o);
                    }
                    if (lane == 0) {
                        double sse = Nw ? s / (double)Nw : 0.0;
                        if (b == 0 && it - 1 < kMaxTrace) P.trace[it - 1] = sse;
                        bool stop = it >= P.max_iter;
                        if (P.eps > 0.0) {
                            if (sse == 0.0) stop = true;
                            else if (it >= 2 && (prev_sse - sse) / sse <= P.eps) stop = true;
                        }
                        s_stop = stop;
                        prev_sse = sse;
                    }
                }
                __syncthreads();
                if (s_stop) break;
            } else if (P.max_iter <= 0) {
                break;
            }
            if (b == 0) {
                unsigned long long* A = P.acc + (size_t)(it & 1) * 4 * K;
                for (int j = tid; j < 4 * K; j += blockDim.x) A[j] = 0ull;
            }
        }
        // sorted center table rows owned by this block
        for (int p = b; p < K; p += G) {
            float4 cp = s_c[p];
            float dj = 0.f;
            if (tid < K) {
                float4 cj = s_c[tid];
                dj = sq3(cp.x, cp.y, cp.z, cj.x, cj.y, cj.z);
                s_row[tid] = dj;
            }
            __syncthreads();
            if (tid < K) {
                const int oj = (tid == p) ? -1 : tid;
                int rank = 0;
                for (int k = 0; k < K; ++k) {
                    float dk = s_row[k];
                    int ok = (k == p) ? -1 : k;
                    rank += (dk < dj) || (dk == dj && ok < oj);
                }
                float4 cj = s_c[tid];
                P.tab[(size_t)p * K + rank] = make_float4(dj * 0.25f, cj.x, cj.y, cj.z);
                P.tab_nb[(size_t)p * K + rank] = (uint8_t)tid;
            }
            __syncthreads();
        }
        if (!grid_sync(P.ctrl, G)) return;

        // ---------------- phase B ----------------
        if (!kMap) {
            for (int j = tid; j < 4 * K; j += blockDim.x) s_acc[j] = 0u;
            __syncthreads();
        }
        const int64_t chunk = (P.n + G - 1) / G;
        const int64_t begin = (int64_t)b * chunk;
        const int64_t end = min(P.n, begin + chunk);
        double sse = 0.0;
        bool bad = false;
        for (int64_t i = begin + tid; i < end; i += blockDim.x) {
            const uint32_t col = __ldg(P.colors + i);
            const int p0 = P.labels[i];
            int p = p0;
            if (p >= K) {                         // invalid input membership
                bad = true;
                p = 0;
            }
            const float x = (float)((col >> 16) & 255u);
            const float y = (float)((col >> 8) & 255u);
            const float z = (float)(col & 255u);
            const float4 cp = s_c[p];
            const float prev = sq3(x, y, z, cp.x, cp.y, cp.z);
            float mn = prev;
            int lab = p;
            const float4* row = P.tab + (size_t)p * K;
            int j = 1;
            for (; j < K; ++j) {
                const float4 e = row[j];
                if (e.x >= prev) break;           // d[p][t] >= 4 prev_dist: stop
                const float dist = sq3(x, y, z, e.y, e.z, e.w);
                if (dist <= mn) {                 // last of equal distances wins
                    mn = dist;
                    lab = P.tab_nb[(size_t)p * K + j];
                }
            }
            evaluated += (unsigned long long)j;   // c_p plus the j-1 visited centers
            if (lab != p0) P.labels[i] = (uint8_t)lab;
            if (kMap) {
                P.lut[col & 0xFFFFFFu] = (uint8_t)lab;
            } else {
                const unsigned n = __ldg(P.counts + i);
                atomicAdd(s_acc + 4 * lab + 0, n * ((col >> 16) & 255u));
                atomicAdd(s_acc + 4 * lab + 1, n * ((col >> 8) & 255u));
                atomicAdd(s_acc + 4 * lab + 2, n * (col & 255u));
                atomicAdd(s_acc + 4 * lab + 3, n);
                sse += (double)n * (double)mn;
            }
        }
        if (bad) atomicOr(&P.ctrl->status, ST_BAD_LABEL);
        if (kMap) break;
        __syncthreads();
        {
            unsigned long long* A = P.acc + (size_t)(it & 1) * 4 * K;
            for (int j = tid; j < 4 * K; j += blockDim.x) {
                unsigned v = s_acc[j];
                if (v) atomicAdd(A + j, (unsigned long long)v);
            }
        }
        for (int o = 16; o > 0; o >>= 1) sse += __shfl_xor_sync(0xFFFFFFFFu, sse, o);
        if (lane == 0) s_red[wid] = sse;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
            P.sse_part[(size_t)(it & 1) * G + b] = t;
        }
        if (!grid_sync(P.ctrl, G)) return;
        ++it;
    }

    // epilogue: centers after the last update, iteration count, distance count
    if (!kMap && b == 0) {
        for (int k = tid; k < K; k += blockDim.x) P.centers[k] = s_c[k];
        if (tid == 0) P.ctrl->iters_done = it;
    }
    for (int o = 16; o > 0; o >>= 1) evaluated += __shfl_xor_sync(0xFFFFFFFFu, evaluated, o);
    if (lane == 0) s_ev[wid] = evaluated;
    __syncthreads();
    if (tid == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_ev[w];
        if (t) atomicAdd(&P.ctrl->evaluated, t);
    }
}

static size_t sortmeans_smem(int K) { return (size_t)K * (16 + 16 + 4); }

// Co-residency of the persistent kernel: blocks per SM for the largest K.
int iterate_kernel_setup(wsm_handle* h) {
    int occ_it = 0, occ_map = 0;
    size_t smem = sortmeans_smem(h->max_K);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ_it, k_sortmeans<false>, kIterThreads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_map, k_sortmeans<true>,
                                                          kIterThreads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    int occ = std::min(occ_it, occ_map);
    if (occ < 1) return fail(WSM_E_CUDA, "persistent kernel cannot be resident");
    h->iter_blocks_per_sm = std::min(occ, 2);
    h->iter_grid = h->iter_blocks_per_sm * h->sms;
    return WSM_OK;
}

// Blocks for n colors: enough for every thread to hold at least one color,
// at most the co-resident grid.
static int sortmeans_grid(wsm_handle* h, int64_t n) {
    int64_t want = (n + kIterThreads - 1) / kIterThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, h->iter_grid));
}

int launch_sortmeans(wsm_handle* h, bool map_mode, const uint32_t* colors, const uint32_t* counts,
                     int64_t n, int K, float* centers, uint8_t* labels, int max_iter, double eps,
                     cudaStream_t s) {
    SortMeansParams P;
    P.colors = colors;
    P.counts = counts;
    P.n = n;
    P.K = K;
    P.centers = reinterpret_cast<float4*>(centers);
    P.labels = labels;
    P.max_iter = max_iter;
    P.eps = eps;
    P.tab = h->tab;
    P.tab_nb = h->tab_nb;
    P.acc = h->acc;
    P.sse_part = h->sse_part;
    P.trace = h->trace;
    P.lut = h->lut;
    P.ctrl = h->ctrl;
    int grid = sortmeans_grid(h, n);
    void* args[] = {&P};
    void* fn = map_mode ? (void*)k_sortmeans<true> : (void*)k_sortmeans<false>;
    cudaError_t e = cudaMemsetAsync(h->ctrl, 0, kLaunchResetBytes, s);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel(fn, grid, kIterThreads, args, sortmeans_smem(K), s);
    if (e != cudaSuccess) return cuda_fail(e, "sort-means launch");
    return WSM_OK;
}

}  // namespace wsm

using namespace wsm;

extern "C" int wsm_iterate(wsm_handle* h, const uint32_t* d_colors, const uint32_t* d_counts,
                           int64_t n_unique, int K, float* d_centers, uint8_t* d_labels,
                           int max_iter, double eps, int* iters_done, double* sse_trace,
                           wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (K < 1 || K > h->max_K) return fail(WSM_E_INVAL, "K out of [1, max_K]");
    if (n_unique < 1 || n_unique > h->max_unique)
        return fail(WSM_E_INVAL, "n_unique must be in [1, max_unique]");
    if (max_iter < 0 || max_iter > kMaxTrace)
        return fail(WSM_E_INVAL, "max_iter must be in [0, 4096]");
    if (!d_colors || !d_counts || !d_centers || !d_labels)
        return fail(WSM_E_INVAL, "null device pointer");
    if ((uintptr_t)d_centers & 15) return fail(WSM_E_INVAL, "centers must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    rc = launch_sortmeans(h, false, d_colors, d_counts, n_unique, K, d_centers, d_labels,
                          max_iter, eps, s);
    if (rc != WSM_OK) return rc;
    if (iters_done || sse_trace) {
        cudaError_t e = cudaMemcpyAsync(&h->host_ctrl->iters_done, &h->ctrl->iters_done,
                                        sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "iteration count copy");
        rc = read_status(h, s);
        if (rc != WSM_OK) return rc;
        int it = h->host_ctrl->iters_done;
        if (iters_done) *iters_done = it;
        if (sse_trace && it > 0) {
            e = cudaMemcpy(sse_trace, h->trace, sizeof(double) * std::min(it, max_iter),
                           cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "SSE trace copy");
        }
    }
    return WSM_OK;
}

extern "C" int wsm_iterate_stats(wsm_handle* h, int K, int64_t* evaluated, int64_t* S, int64_t* W,
                                 wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (K < 1 || K > h->max_K) return fail(WSM_E_INVAL, "K out of [1, max_K]");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream sync");
    Ctrl c;
    e = cudaMemcpy(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats copy");
    if (evaluated) *evaluated = (int64_t)c.evaluated;
    if (S || W) {
        // the sums of the last pass sit in buffer (iters_done - 1) & 1
        if (c.iters_done < 1) return fail(WSM_E_STATE, "no completed iteration");
        int slot = (c.iters_done - 1) & 1;
        unsigned long long buf[4 * WSM_MAX_K];
        e = cudaMemcpy(buf, h->acc + (size_t)slot * 4 * K, sizeof(unsigned long long) * 4 * K,
                       cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "sums copy");
        for (int k = 0; k < K; ++k) {
            if (S)
                for (int ch = 0; ch < 3; ++ch) S[3 * k + ch] = (int64_t)buf[4 * k + ch];
            if (W) W[k] = (int64_t)buf[4 * k + 3];
        }
    }
    return WSM_OK;
}

// ---------------------------------------------------------------------------
// wsm_iterate_noalloc: the same Sort-Means iterations for callers that may
// not allocate device memory (see include/wsm.h).  All scratch lives in the
// file-scope array below, which every GPU that loads this library holds
// until the process exits.
// ---------------------------------------------------------------------------
namespace wsm {

constexpr int kStaticMaxK = WSM_MAX_K;
constexpr int kStaticMaxGrid = 1024;
constexpr size_t kStaticTabBytes = sizeof(float4) * kStaticMaxK * kStaticMaxK;   // 1 MiB
constexpr size_t kStaticNbBytes = (size_t)kStaticMaxK * kStaticMaxK;            // 64 KiB
constexpr size_t kStaticAccBytes = sizeof(unsigned long long) * 2 * 4 * kStaticMaxK;
constexpr size_t kStaticSseBytes = sizeof(double) * 2 * kStaticMaxGrid;
constexpr size_t kStaticTraceBytes = sizeof(double) * kMaxTrace;
constexpr size_t kStaticOffNb = kStaticTabBytes;
constexpr size_t kStaticOffAcc = kStaticOffNb + kStaticNbBytes;
constexpr size_t kStaticOffSse = kStaticOffAcc + kStaticAccBytes;
constexpr size_t kStaticOffTrace = kStaticOffSse + kStaticSseBytes;
constexpr size_t kStaticOffCtrl = kStaticOffTrace + kStaticTraceBytes;
constexpr size_t kStaticBytes = kStaticOffCtrl + 256;           // about 1.13 MiB in total

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct StaticSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;   // device address of g_static_scratch
    int grid = 0;
};
static std::mutex g_static_mutex;
static StaticSetup g_static_setup[64];

// Once per device, with that device current: the device address of the
// scratch array and the co-resident grid of the persistent kernel.
static int static_setup(int dev, StaticSetup** out) {
    if (dev < 0 || dev >= 64) return fail(WSM_E_STATE, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_static_mutex);
    StaticSetup& st = g_static_setup[dev];
    if (!st.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        int sms = 0, occ = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &occ, k_sortmeans<false>, kIterThreads, sortmeans_smem(kStaticMaxK));
        if (e != cudaSuccess) return cuda_fail(e, "static set-up query");
        if (occ < 1) return fail(WSM_E_CUDA, "persistent kernel cannot be resident");
        st.scratch = static_cast<unsigned char*>(p);
        st.grid = std::min(std::min(occ, 2) * sms, kStaticMaxGrid);
        st.ready = true;
    }
    *out = &st;
    return WSM_OK;
}

}  // namespace wsm

extern "C" int wsm_iterate_noalloc(const uint32_t* d_colors, const uint32_t* d_counts,
                                   int64_t n_unique, int K, float* d_centers, uint8_t* d_labels,
                                   int max_iter, double eps, int* iters_done, double* sse_trace,
                                   wsm_stream stream) {
    if (K < 1 || K > kStaticMaxK)
        return fail(WSM_E_INVAL, "wsm_iterate_noalloc: K must be in [1, 256] (the static "
                                 "scratch holds 256 x 256 sorted center tables)");
    if (n_unique < 1 || n_unique > WSM_MAX_PIXELS)
        return fail(WSM_E_INVAL, "wsm_iterate_noalloc: n_unique must be in [1, 2^24]");
    if (max_iter < 0 || max_iter > kMaxTrace)
        return fail(WSM_E_INVAL, "wsm_iterate_noalloc: max_iter must be in [0, 4096]");
    if (!d_colors || !d_counts || !d_centers || !d_labels)
        return fail(WSM_E_INVAL, "null device pointer");
    if ((uintptr_t)d_centers & 15) return fail(WSM_E_INVAL, "centers must be 16-byte aligned");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    StaticSetup* st = nullptr;
    int rc = static_setup(dev, &st);
    if (rc != WSM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = st->scratch;
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(base + kStaticOffCtrl);
    SortMeansParams P;
    P.colors = d_colors;
    P.counts = d_counts;
    P.n = n_unique;
    P.K = K;
    P.centers = reinterpret_cast<float4*>(d_centers);
    P.labels = d_labels;
    P.max_iter = max_iter;
    P.eps = eps;
    P.tab = reinterpret_cast<float4*>(base);
    P.tab_nb = base + kStaticOffNb;
    P.acc = reinterpret_cast<unsigned long long*>(base + kStaticOffAcc);
    P.sse_part = reinterpret_cast<double*>(base + kStaticOffSse);
    P.trace = reinterpret_cast<double*>(base + kStaticOffTrace);
    P.lut = nullptr;
    P.ctrl = ctrl;
    int64_t want = (n_unique + kIterThreads - 1) / kIterThreads;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, st->grid));
    void* args[] = {&P};
    // the barrier words, counters and status word start at zero on every call
    e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((void*)k_sortmeans<false>, grid, kIterThreads, args,
                                        sortmeans_smem(K), s);
    if (e != cudaSuccess) return cuda_fail(e, "wsm_iterate_noalloc launch");
    if (iters_done || sse_trace) {
        Ctrl host;
        e = cudaMemcpyAsync(&host, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "wsm_iterate_noalloc result copy");
        if (host.status & ST_TIMEOUT) return fail(WSM_E_TIMEOUT, "a device-side grid barrier timed out");
        if (host.status & ST_BAD_LABEL) return fail(WSM_E_INVAL, "a membership was >= K");
        if (iters_done) *iters_done = host.iters_done;
        if (sse_trace && host.iters_done > 0) {
            e = cudaMemcpyAsync(sse_trace, P.trace, sizeof(double) * std::min(host.iters_done, max_iter),
                                cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "wsm_iterate_noalloc trace copy");
        }
    }
    return WSM_OK;
}
