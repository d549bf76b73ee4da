// wsm_internal.cuh -- shared definitions of libwsm's translation units:
// the handle, status bits, bounded device-side waits and the grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "wsm.h"

namespace wsm {

// Device status word bits (kernel-side failures, reported on the next sync).
enum : unsigned {
    ST_TIMEOUT = 1u,    // a grid barrier wait ran past its limit
    ST_BAD_LABEL = 2u,  // an input membership or palette index was >= K
    ST_CAPACITY = 4u,   // more unique colors than the output capacity
    ST_FEW_COLORS = 8u, // an image of a device-sized batch has fewer unique colors than K
};

// A grid barrier waits at most this long (globaltimer ns) before giving up.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

constexpr int kHistBins = 1 << 24;           // one bin per 24-bit color
constexpr int kMapWords = kHistBins / 32;    // occupancy bitmap words
constexpr int kScanWordsPerThread = 4;       // bitmap words per thread in the compaction
constexpr int kScanThreads = 512;
constexpr int kScanWordsPerBlock = kScanWordsPerThread * kScanThreads;   // 2048
constexpr int kScanBlocks = kMapWords / kScanWordsPerBlock;             // 256
constexpr int kMaxTrace = 4096;              // SSE values kept per wsm_iterate call
constexpr int kCopies = 1;                   // copies of the global accumulators
constexpr int kChunk = 32;                   // colors per warp chunk (one per lane)
constexpr int kMaxBatch = 64;                // images per persistent launch
constexpr int kReduceSlots = 16;             // images per unique-color reduction launch
constexpr int kGridCells = 4096;             // 16^3 cells of the first pass's candidate grid
// Bucketed unique-color reduction (large images): buckets by the top 10 bits
// of the 24-bit key, each with a 2^14-bin histogram that fits shared memory.
constexpr int kBktBits = 10;
constexpr int kBuckets = 1 << kBktBits;      // buckets per image
constexpr int kBktBins = 1 << (24 - kBktBits);   // colors per bucket (16384)
constexpr int kBktChunk = 16384;             // keys per bucket-histogram work item
// work items of one image: one per nonempty bucket plus one per further chunk
__host__ __device__ constexpr int64_t bkt_max_work(int64_t max_pixels) {
    return (max_pixels + kBktChunk - 1) / kBktChunk + kBuckets;
}

// A launch shape of the persistent sort-means kernel.
struct IterShape {
    int threads;         // per block: 256, 512 or 1024
    int blocks_per_sm;   // co-resident blocks per SM
};
constexpr int kNumIterShapes = 5;
extern const IterShape kIterShapes[kNumIterShapes];

// Control words in device memory: one for the handle (status word, N', MSE
// mirror) and one per image slot (barrier counter, iteration and distance
// counts, chunk tickets), the latter cleared before every persistent launch
// so that a barrier abandoned after a timeout cannot confuse the next one.
struct Ctrl {
    unsigned bar_count;        // grid barrier: monotonic arrival counter
    int iters_done;            // iterations completed by the last wsm_iterate
    unsigned long long evaluated;  // distances computed by the last persistent launch
    unsigned status;           // ST_* bits (cleared only when read by the host)
    unsigned ticket[2];        // chunks handed out in the assignment pass, by pass parity
    int64_t n_unique;          // N' of the last wsm_reduce
    double mse;                // host mirror slot of the last wsm_distortion
    unsigned long long map_sse;    // sum over colors of count * ||x - c||^2 in units of
                                   // 2^-20 (each term truncated) of the last final assignment
    unsigned long long t_start;    // globaltimer at the start and the end of the slot's
    unsigned long long t_end;      //   group in the last persistent launch of iterations
};

}  // namespace wsm

struct wsm_handle {
    int device = -1;
    int sms = 0;
    int max_K = 0;
    int label_bytes = 1;         // 1 (max_K <= 256) or 2: memberships, indices, table entries
    int64_t max_pixels = 0;
    int64_t max_unique = 0;
    int iter_shape = 0;          // index into kIterShapes used by the persistent launches
    int grid_limit = 0;          // > 0: at most this many blocks per persistent launch
    bool cand_start = true;      // see wsm_set_first_pass_start
    int reduce_path = 0;         // see wsm_set_reduce_path: 0 by size, 1 direct, 2 bucketed
    bool shape_ok[wsm::kNumIterShapes] = {};   // shapes whose blocks can all be resident
    // scratch (device)
    double* mse_part = nullptr;  // [1024] block partials + [1] result
    wsm::Ctrl* ctrl = nullptr;   // status word, N', MSE mirror
    wsm::Ctrl* host_ctrl = nullptr;  // pinned mirror for status reads
    cudaEvent_t pick_ready = nullptr;  // host_pick may be rewritten once this has fired
    // differentiable distortion scratch
    float4* grad_tab = nullptr;  // [max_K^2] full sorted rows of the palette
    uint8_t* grad_nb = nullptr;  // [max_K^2]
    float4* grad_part = nullptr; // [grad_blocks][max_K + 1] block partials
    // unique-color reduction scratch, one slot per image of a reduction launch
    int rslots = 0;
    uint32_t* hist = nullptr;    // [rslots][2^24] zero between calls
    uint32_t* bitmap = nullptr;  // [rslots][2^19] zero between calls
    uint32_t* blk_total = nullptr;   // [rslots][kScanBlocks]
    uint32_t* bkt_count = nullptr;   // [rslots][kBuckets] pixels per bucket, zero between calls
    uint32_t* bkt_cursor = nullptr;  // [rslots][kBuckets] next free key position per bucket
    uint16_t* keys16 = nullptr;      // [rslots][max_pixels] low 14 bits of the keys, by bucket
    uint4* bkt_work = nullptr;       // [rslots][bkt_max_work] (bucket, start, length, shared)
    int* bkt_nwork = nullptr;        // [rslots] work items of the last planned launch
    // per-image scratch of the persistent kernel, one slot per image of a batch
    int slots = 0;
    float4* tab = nullptr;       // [slots][max_K^2] sorted rows: (d/4, c.x, c.y, c.z)
    uint8_t* tab_nb = nullptr;   // [slots][max_K^2] center index of each row entry (label_bytes)
    unsigned* sums = nullptr;    // [slots][2][kCopies][5 max_K] replicated sums and maxima
    unsigned long long* sums64 = nullptr;  // [slots][2][kCopies][4] SSE, distances, pixels, nonzero
    unsigned long long* acc = nullptr;     // [slots][4 max_K] S_k (3) and W_k of the last pass
    double* trace = nullptr;     // [slots][kMaxTrace]
    uint8_t* lut = nullptr;      // [slots][2^24] color -> label (label_bytes each)
    uint8_t* grid = nullptr;     // [slots][kGridCells] candidate center per RGB cell (idem)
    wsm::Ctrl* slot_ctrl = nullptr;  // [slots] barrier counter, iterations, distances
    int64_t* batch_nu = nullptr;     // [slots] N' of each image of the last wsm_reduce_batch
    double* batch_mse = nullptr;     // [slots] MSE of each image of the last wsm_distortion_batch
    uint32_t* pick = nullptr;        // [slots][max_K] initial center indices (wsm_init_batch)
    int* plan = nullptr;             // [slots / kMaxBatch + 1][kMaxBatch + 1] block splits
    int* slot_weight = nullptr;      // [slots] work weight of each image in the device-side
                                     //   split, 1/1024 units (0: 1), set by the autotuner
    int64_t* host_nu = nullptr;      // pinned mirrors of the three arrays above
    double* host_mse = nullptr;
    uint32_t* host_pick = nullptr;
};

namespace wsm {

// Keys of one reduction slot in the bucketed path: max_pixels rounded up to
// a multiple of 8 (16-byte rows of uint16).
inline size_t keys_stride(const wsm_handle* h) { return ((size_t)h->max_pixels + 7) & ~(size_t)7; }

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
int check_handle(wsm_handle* h);
int read_status(wsm_handle* h, cudaStream_t s);
int alloc_slots(wsm_handle* h, int slots);
int grad_blocks(wsm_handle* h);
int iter_grid(const wsm_handle* h);
// Raise (never lower) a kernel's dynamic shared-memory limit on the current
// device; the limit is shared by every handle.
cudaError_t raise_smem_limit(const void* fn, size_t bytes);

// Stream-ordered pieces of the batch calls (no checks, no synchronisation);
// item i of a call uses image slot i.  With n_dev, N' of item i is read on
// the device from n_dev[i] (written by reduce_items into batch_nu).
int check_item(wsm_handle* h, const wsm_item& it, bool need_pixels, bool need_counts);
int check_pixels(wsm_handle* h, const wsm_item& it);
int reduce_items(wsm_handle* h, const wsm_item* items, int n_items, cudaStream_t s);
int init_items_dev(wsm_handle* h, const wsm_item* items, int n_items, const uint64_t* seeds,
                   cudaStream_t s);
int iterate_items(wsm_handle* h, const wsm_item* items, int n_items, int max_iter, double eps,
                  const int64_t* n_dev, cudaStream_t s, int64_t* d_n_unique = nullptr,
                  int* d_iters = nullptr);
int launch_sortmeans(wsm_handle* h, bool map_mode, const uint32_t* colors, const uint32_t* counts,
                     int64_t n, int K, float* centers, void* labels, int max_iter, double eps,
                     cudaStream_t s);
int launch_map_items(wsm_handle* h, const wsm_item* items, int n_items, int slot0,
                     const int64_t* n_dev, bool sse, cudaStream_t s);
int map_items(wsm_handle* h, const wsm_item* items, int n_items, const int64_t* n_dev, bool sse,
              cudaStream_t s);
int pixel_items(wsm_handle* h, const wsm_item* items, int n_items, bool gather, double* d_mse,
                const int64_t* n_dev, cudaStream_t s);
void free_slots(wsm_handle* h);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned add_release(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Barrier over `nblocks` co-resident blocks (a whole cooperative grid, or one
// image's group of it).  Thread 0 of each block adds 1 to a counter that only
// grows (release), and waits (acquire) until it reaches the next multiple of
// nblocks, i.e. until every block has arrived at this barrier.  The wait has
// a time limit (limit_ns): past it *status gets ST_TIMEOUT and the function
// returns false in every thread of the block.  Memory written before the barrier by any of
// the blocks is visible to all of them after it.
__device__ __forceinline__ bool grid_sync(unsigned* counter, unsigned* status, unsigned nblocks,
                                          unsigned long long limit_ns = kWaitLimitNs) {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned old = add_release(counter, 1u);
        unsigned target = (old / nblocks + 1u) * nblocks;
        unsigned ok = 1u;
        if ((int)(ld_acquire(counter) - target) < 0) {
            unsigned long long t0 = global_ns();
            while ((int)(ld_acquire(counter) - target) < 0) {
                if (global_ns() - t0 > limit_ns) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0u;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Packed key 0x00RRGGBB of pixel p of an image stored as [n][stride] bytes
// (R, G, B first; a fourth byte per pixel is ignored).
__device__ __forceinline__ uint32_t pixel_key(const uint8_t* __restrict__ rgb, int64_t p,
                                              int stride) {
    if (stride == 4) {
        uint32_t v = __ldg(reinterpret_cast<const uint32_t*>(rgb) + p);
        return ((v & 0xFFu) << 16) | (v & 0xFF00u) | ((v >> 16) & 0xFFu);
    }
    const uint8_t* q = rgb + 3 * p;
    return ((uint32_t)__ldg(q) << 16) | ((uint32_t)__ldg(q + 1) << 8) | (uint32_t)__ldg(q + 2);
}

// Index of the item that owns block `blk` when item i owns the blocks
// [first[i], first[i+1]) (ranges may be empty).
__device__ __forceinline__ int item_of_block(const int* first, int n_items, int blk) {
    int i = 0;
    while (i + 1 < n_items && blk >= first[i + 1]) ++i;
    return i;
}

// Squared distance in the difference form with one fixed rounding order
// (no contraction choices left to the compiler), so that every call site --
// center table, previous-center distance, visited entries -- rounds alike.
__device__ __forceinline__ float sq3(float ax, float ay, float az, float bx, float by, float bz) {
    const float ex = __fsub_rn(ax, bx), ey = __fsub_rn(ay, by), ez = __fsub_rn(az, bz);
    return __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
}

// The table M of Algorithm 2 (Sec. 2): row p lists the centers by their
// distance d[p][t] from c_p, nearest first, as entries (d[p][t] / 4, c_t)
// with the center index t in a parallel byte array.

// Row-sort key of center t in row p: the bits of d (>= 0, so they order like
// the values) above the tie order (t != p, t).
__device__ __forceinline__ unsigned long long row_key(float d, int t, int p) {
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)(t == p ? 0 : t + 1);
}

// Compare-exchange of a bitonic network step for the element held here
// (index i) and its partner (index i ^ h, value o): the lower index of an
// ascending block ((i & k) == 0) keeps the smaller key, of a descending one
// the larger.
__device__ __forceinline__ unsigned long long bitonic_keep(unsigned long long a,
                                                           unsigned long long o, int i, int h,
                                                           int k) {
    const bool lower = (i & h) == 0, up = (i & k) == 0;
    return (lower == up) ? (a < o ? a : o) : (a < o ? o : a);
}

// One step of the network between slots HS apart in the same lane (partners
// 32 * HS elements apart): each pair once, from its lower slot.
template <int HS, int S>
__device__ __forceinline__ void bitonic_slots(unsigned long long (&v)[S], int lane, int k) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if (s & HS) continue;
        const int t = s | HS;
        const unsigned long long a = v[s], c = v[t];
        const bool up = ((lane + 32 * s) & k) == 0;
        const unsigned long long lo = a < c ? a : c, hi = a < c ? c : a;
        v[s] = up ? lo : hi;
        v[t] = up ? hi : lo;
    }
}

// Sorts the 32 S keys (S = 4 or 8) that one warp holds in registers,
// element lane + 32 s in v[s], ascending (bitonic network; partners 32 or
// more apart are in the same lane, nearer ones in lane ^ h).
template <int S>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&v)[S], int lane) {
    for (int k = 2; k <= 32 * S; k <<= 1) {
        for (int h = k >> 1; h > 0; h >>= 1) {
            if constexpr (S == 8) {
                if (h == 128) {
                    bitonic_slots<4, 8>(v, lane, k);
                    continue;
                }
            }
            if (h == 64) {
                bitonic_slots<2, S>(v, lane, k);
            } else if (h == 32) {
                bitonic_slots<1, S>(v, lane, k);
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, v[s], h);
                    v[s] = bitonic_keep(v[s], o, lane + 32 * s, h, k);
                }
            }
        }
    }
}

// The L (<= 32 S) kept keys of row p, from shared memory, sorted by one warp
// in registers and written as the row's entries, then its four sentinels.
template <int S, typename Label>
__device__ __forceinline__ void sort_row_in_registers(const unsigned long long* key, int L, int p,
                                                      int K, int lane, const float4* s_c,
                                                      float4* row, Label* row_nb) {
    unsigned long long v[S];
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const int j = lane + 32 * q;
        v[q] = j < L ? key[j] : ~0ull;
    }
    warp_bitonic<S>(v, lane);
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const int j = lane + 32 * q;
        if (j < L) {
            const unsigned lo = (unsigned)v[q];
            const int c = lo ? (int)lo - 1 : p;
            const float4 ct = s_c[c];
            const float d4 = __uint_as_float((unsigned)(v[q] >> 32)) * 0.25f;
            row[j] = make_float4(d4, ct.x, ct.y, ct.z);
            row_nb[j] = (Label)c;
        }
    }
    if (lane < 4 && L + lane < K)
        row[L + lane] = make_float4(__int_as_float(0x7f800000), 0.f, 0.f, 0.f);
}

// Barrier of the ts warps of team m (ts a power of two; a named barrier
// 1 + m when ts > 1, so at most 15 teams of several warps per block).
__device__ __forceinline__ void team_sync(int m, int ts) {
    if (ts == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(m + 1), "r"(ts * 32) : "memory");
}

// Warps per row-building team: the largest power of two ts <= WPB that
// still leaves at least K teams over the image's G blocks (one row each),
// counting only team sizes that give at most 8 teams per block; 1 (one warp
// per row, several rows per warp) when even single warps are fewer than K.
// Launches sized for palettes of more than 256 colors (KM > 256) always use
// whole blocks: their key buffer in shared memory holds one row per block.
__device__ __forceinline__ int row_team_size(int K, int KM, int G, int WPB) {
    if (KM > WSM_MAX_K) return WPB;
    int ts = 1;
    for (int c = 2; c <= WPB; c *= 2)
        if (WPB / c <= 8 && (long long)G * (WPB / c) >= K) ts = c;
    return ts;
}

// The rows of one image's table, built by teams of ts warps: team m of
// block b is team number m * G + b of the image and builds rows team,
// team + (number of teams), ...  Row p keeps the centers t with
// d[p][t] < thr[p] (p itself always); the rank of a key among the kept keys
// (keys are distinct, so the order in which they were collected does not
// matter) is its entry position.  The team's threads split the comparisons
// of a rank when there are more of them than kept keys; a row of more than
// 64 kept keys built by a single warp is sorted in registers by a bitonic
// network instead (the same order).  Four entries with an infinite bound
// follow the kept ones.
template <typename Label>
__device__ __forceinline__ void build_rows(int K, int KM, int G, int b, const float4* s_c,
                                           const float* s_thr, unsigned long long* s_wkey,
                                           float4* tab, Label* tab_nb) {
    __shared__ int s_len[32];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, WPB = blockDim.x >> 5;
    const int ts = row_team_size(K, KM, G, WPB), TT = ts * 32;
    const int m = wid / ts, r = threadIdx.x - m * TT;          // team, thread in team
    const int teams = G * (WPB / ts);
    unsigned long long* key = s_wkey + (size_t)m * ts * K;     // the team's buffer: ts * K
    int* rank_part = reinterpret_cast<int*>(key + K);           // [K] when ts > 1
    const unsigned below = (1u << lane) - 1u;
    for (int p = m * G + b; p < K; p += teams) {
        const float4 cp = s_c[p];
        const float bound = s_thr[p];
        if (r == 0) s_len[m] = 0;
        team_sync(m, ts);
        for (int t0 = 0; t0 < K; t0 += TT) {
            const int t = t0 + r;
            float d = 0.f;
            bool keep = false;
            if (t < K) {
                const float4 ct = s_c[t];
                d = sq3(cp.x, cp.y, cp.z, ct.x, ct.y, ct.z);
                keep = d < bound || t == p;
            }
            const unsigned vote = __ballot_sync(0xFFFFFFFFu, keep);
            int base = 0;
            if (lane == 0 && vote) base = atomicAdd(&s_len[m], __popc(vote));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (keep) key[base + __popc(vote & below)] = row_key(d, t, p);
        }
        team_sync(m, ts);
        const int L = s_len[m];
        float4* row = tab + (size_t)p * K;
        Label* row_nb = tab_nb + (size_t)p * K;
        if (ts == 1 && L > 64) {
            // a long row kept by a single warp: sorted in registers by a
            // bitonic network (the same order as the ranks below, keys being
            // distinct), padded to 128 or 256 with keys above every real one
            if (L > 128) sort_row_in_registers<8>(key, L, p, K, lane, s_c, row, row_nb);
            else sort_row_in_registers<4>(key, L, p, K, lane, s_c, row, row_nb);
            team_sync(m, ts);
            continue;
        }
        const int H = ts > 1 ? max(1, TT / L) : 1;               // threads per kept key
        if (H > 1) {
            for (int j = r; j < L; j += TT) rank_part[j] = 0;
            team_sync(m, ts);
            const int span = (L + H - 1) / H;
            for (int u = r; u < L * H; u += TT) {
                const int j = u % L, h = u / L;
                const unsigned long long kj = key[j];
                int cnt = 0;
                const int k1 = min(L, (h + 1) * span);
                for (int k = h * span; k < k1; ++k) cnt += key[k] < kj;
                if (cnt) atomicAdd(rank_part + j, cnt);
            }
            team_sync(m, ts);
        }
        for (int j = r; j < L; j += TT) {
            const unsigned long long kj = key[j];
            int rank = 0;
            if (H > 1) {
                rank = rank_part[j];
            } else {
#pragma unroll 8
                for (int k = 0; k < L; ++k) rank += key[k] < kj;
            }
            const unsigned lo = (unsigned)kj;
            const int c = lo ? (int)lo - 1 : p;
            const float4 ct = s_c[c];
            const float d4 = __uint_as_float((unsigned)(kj >> 32)) * 0.25f;
            row[rank] = make_float4(d4, ct.x, ct.y, ct.z);
            row_nb[rank] = (Label)c;
        }
        if (r < 4 && L + r < K)
            row[L + r] = make_float4(__int_as_float(0x7f800000), 0.f, 0.f, 0.f);
        team_sync(m, ts);
    }
}

}  // namespace wsm
