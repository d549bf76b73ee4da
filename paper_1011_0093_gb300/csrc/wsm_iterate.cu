// wsm_iterate.cu -- the Sort-Means loop of Algorithm 2 (Sec. 2) as one
// persistent cooperative kernel, used both for the iterations (wsm_iterate)
// and for the final assignment before pixel mapping (wsm_map).
//
// One launch runs every iteration, as two phases separated by grid barriers:
//   A  every block turns the cluster sums of the previous pass into the new
//      centers c_k = S_k / W_k (correctly rounded to FP32; an empty cluster
//      keeps its center), measures that pass's SSE and applies the Sec. 3.2
//      stop rule (all blocks compute the same values, so all decide alike),
//      then sorts rows p = b, b+G, ... of the center table: row p lists,
//      nearest first, the entries (d[p][t] / 4, c_t) for the centers t, ties
//      ordered by (t != p, t), so entry 0 is p itself.  In the first pass of
//      a launch a row holds every center; later a row holds only the centers
//      below a bound that no visit of that row can pass (see the row bound
//      below), followed by entries with an infinite bound -- the entries a
//      visit reads, and their order, are the same as with the full row.
//   B  the pruned nearest-center search, one lane per unique color; warp w
//      of block b takes the chunks of 32 consecutive colors numbered
//      b * WPB + w + k * G * WPB (spreading costly regions of color space over
//      all blocks) and loads the next chunk's records while it searches the
//      current one.  A color starts at its previous center p with
//      prev = ||x - c_p||^2 and visits row p from entry 1 on; the visit stops
//      at the first entry with d[p][t] / 4 >= prev (the paper's
//      d[p][t] >= 4 prev_dist; scaling by 4 is exact), and a visited center
//      replaces the current one when its distance is <= the running
//      minimum, so among equal distances the one visited last wins.  Entries
//      are loaded four at a time; since a row is sorted, the four are all
//      visited when the last one is below the bound.  Cluster sums are
//      accumulated per block in shared memory (uint32, exact because an
//      image has at most 2^24 pixels) and added into one of kCopies
//      replicated global accumulators (integer atomics, so the totals are
//      exact and independent of the order).
// The SSE is accumulated as an integer in units of 2^-20 (each color's
// n_i * min_dist_i truncated to that grid), so every reduction is exact and
// the results do not depend on the grid or on the order of the additions.
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
    unsigned* sums;        // [2][kCopies][5K] cluster sums (4K) and the largest squared
                           //   distance of a member to its center (K, FP32 bits),
                           //   double-buffered by pass parity
    unsigned long long* sums64;  // [2][kCopies][4] SSE (2^-20 units), distances, pixels,
                                 //   colors with a nonzero minimum
    unsigned long long* acc;     // [K][4] cluster sums of the last pass
    double* trace;         // [kMaxTrace]
    uint8_t* lut;          // map mode: [2^24] color -> label
    Ctrl* ctrl;
};

// floor(t / W) for t < 128 W (or t < 2^32 with a quotient below 2^8) and
// 1 <= W <= 2^24: an FP32 estimate from the reciprocal, off by at most one,
// then corrected with exact integer arithmetic.
__device__ __forceinline__ unsigned small_quotient(unsigned t, unsigned W, float rcp) {
    unsigned q = __float2uint_rz(__fmul_rn((float)t, rcp));
    long long r = (long long)t - (long long)q * W;
    if (r < 0) { --q; r += W; }
    if (r >= (long long)W) ++q;
    return q;
}

// fl32(S / W) rounded to nearest-even, for 0 <= S < 2^32 and 1 <= W <= 2^24
// (S <= 255 W), by exact long division: the integer part, then seven fraction
// bits per step until at least 26 significant bits are known, then rounding
// on the dropped bits and the remainder.
__device__ __forceinline__ float div_rn_u32(unsigned S, unsigned W, float rcp) {
    if (S == 0) return 0.f;
    unsigned q = small_quotient(S, W, rcp);
    unsigned rem = S - q * W;                   // < W <= 2^24, so rem << 7 fits
    unsigned long long m = q;
    int e = 0;                                  // S / W = (m + rem / W) * 2^-e
    for (int step = 0; step < 10 && m < (1ull << 26); ++step) {
        const unsigned t = rem << 7;
        const unsigned d = small_quotient(t, W, rcp);
        rem = t - d * W;
        m = (m << 7) | d;
        e += 7;
    }
    const int nb = 64 - __clzll((long long)m);
    const int shift = max(nb - 24, 1);          // keep 24 significant bits (3..9 here)
    unsigned long long mant = m >> shift;
    const unsigned long long rest = m & ((1ull << shift) - 1);
    const unsigned long long half = 1ull << (shift - 1);
    if (rest > half || (rest == half && (rem != 0 || (mant & 1)))) mant += 1;
    return ldexpf((float)mant, shift - e);
}

// n * v * 2^20 truncated toward zero, for v >= 0 finite below 2^18, from the
// FP32 bits of v (exact integer arithmetic).
__device__ __forceinline__ unsigned long long sse_fixed(unsigned n, float v) {
    unsigned bits = __float_as_uint(v);
    int e = (bits >> 23) & 255;
    unsigned long long m = bits & 0x7FFFFFu;
    if (e) m |= 0x800000u;
    else e = 1;
    unsigned long long prod = (unsigned long long)n * m;   // < 2^48
    int sh = e - 150 + 20;                                 // v = m * 2^(e-150)
    if (sh >= 0) return prod << min(sh, 15);
    if (sh <= -63) return 0ull;
    return prod >> (-sh);
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Row-sort key of center t in row p: the bits of d (>= 0, so they order like
// the values) above the tie order (t != p, t).
__device__ __forceinline__ unsigned long long row_key(float d, int t, int p) {
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)(t == p ? 0 : t + 1);
}

// This block's rows of the sorted center table.  Row p keeps the centers t
// with d[p][t] < thr[p] (p itself always), sorted by rank: the rank of a key
// among the kept keys (keys are distinct) is its entry position, S threads
// share one key's comparisons.  Four entries with an infinite bound follow
// the kept ones, so every visit stops there (the scan reads four entries per
// step).  thr = NULL keeps every center.
__device__ __forceinline__ void build_rows(const SortMeansParams& P, const float4* s_c,
                                           const float* thr, unsigned long long* s_key,
                                           int* s_rank, int* s_cnt) {
    const int K = P.K, tid = threadIdx.x, T = blockDim.x, lane = tid & 31, wid = tid >> 5;
    for (int p = blockIdx.x; p < K; p += gridDim.x) {
        const float4 cp = s_c[p];
        const float bound = thr ? thr[p] : __int_as_float(0x7f800000);
        // kept centers, compacted in index order (K <= 256 <= T: one round)
        {
            const int t = tid;
            float d = 0.f;
            bool keep = false;
            if (t < K) {
                const float4 ct = s_c[t];
                d = sq3(cp.x, cp.y, cp.z, ct.x, ct.y, ct.z);
                keep = d < bound || t == p;
            }
            const unsigned vote = __ballot_sync(0xFFFFFFFFu, keep);
            if (lane == 0) s_cnt[wid] = __popc(vote);
            __syncthreads();
            if (tid == 0) {
                int run = 0;
                for (int w = 0; w < (T >> 5); ++w) {
                    const int c = s_cnt[w];
                    s_cnt[w] = run;
                    run += c;
                }
                s_cnt[32] = run;
            }
            __syncthreads();
            if (keep) s_key[s_cnt[wid] + __popc(vote & ((1u << lane) - 1u))] = row_key(d, t, p);
            if (tid < K) s_rank[tid] = 0;
            __syncthreads();
        }
        const int L = s_cnt[32];
        const int S = max(1, T / L);
        const int span = (L + S - 1) / S;
        for (int t = tid; t < S * L; t += T) {
            const int j = t % L, h = t / L;
            const unsigned long long kj = s_key[j];
            const int lo = h * span, hi = min(L, lo + span);
            int rank = 0;
#pragma unroll 8
            for (int k = lo; k < hi; ++k) rank += s_key[k] < kj;
            if (S == 1) s_rank[j] = rank;
            else if (rank) atomicAdd(s_rank + j, rank);
        }
        __syncthreads();
        for (int t = tid; t < L; t += T) {
            const unsigned long long key = s_key[t];
            const unsigned lo = (unsigned)key;
            const int c = lo ? (int)lo - 1 : p;
            const float4 ct = s_c[c];
            const int r = s_rank[t];
            P.tab[(size_t)p * K + r] =
                make_float4(__uint_as_float((unsigned)(key >> 32)) * 0.25f, ct.x, ct.y, ct.z);
            P.tab_nb[(size_t)p * K + r] = (uint8_t)c;
        }
        if (tid < 4 && L + tid < K)
            P.tab[(size_t)p * K + L + tid] = make_float4(__int_as_float(0x7f800000), 0.f, 0.f, 0.f);
        __syncthreads();
    }
}

// One visited entry: distance, and the update with the later entry winning ties.
#define WSM_VISIT(e, jj)                                        \
    {                                                           \
        const float dist_ = sq3(x, y, z, (e).y, (e).z, (e).w);  \
        if (dist_ <= mn) {                                      \
            mn = dist_;                                         \
            mpos = (jj);                                        \
        }                                                       \
    }

template <bool kMap>
__global__ void __launch_bounds__(kIterThreads, 2) k_sortmeans(SortMeansParams P) {
    extern __shared__ float4 smem[];
    const int K = P.K;
    float4* s_c = smem;                                                       // [K] centers
    float4* s_cn = s_c + K;                                                   // [K] new centers
    unsigned long long* s_key = reinterpret_cast<unsigned long long*>(s_cn + K);  // [K]
    unsigned* s_acc = reinterpret_cast<unsigned*>(s_key + K);                 // [5K] sums, max
    float* s_thr = reinterpret_cast<float*>(s_acc + 5 * K);                   // [K] row bounds
    int* s_rank = reinterpret_cast<int*>(s_thr + K);                          // [K]
    __shared__ unsigned long long s_red[4][kIterThreads / 32];
    __shared__ int s_cnt[33];
    __shared__ int s_stop;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int T = blockDim.x, WPB = T >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    const int copy = b % kCopies;
    const int64_t n = P.n;
    if (!kMap && P.max_iter <= 0) return;

    for (int k = tid; k < K; k += T) s_c[k] = P.centers[k];
    if (!kMap && b == 0) {
        for (int j = tid; j < kCopies * 5 * K; j += T) P.sums[j] = 0u;
        if (tid < 4 * kCopies) P.sums64[tid] = 0ull;
    }
    __syncthreads();
    build_rows(P, s_c, nullptr, s_key, s_rank, s_cnt);
    if (!grid_sync(P.ctrl, G)) return;

    unsigned long long prev_fx = 0;        // SSE of the previous pass, in thread 0 only
    for (int it = 0;; ++it) {
        // ---------------- phase B: assignment ----------------
        const int buf = it & 1;
        if (!kMap)
            for (int j = tid; j < 5 * K; j += T) s_acc[j] = 0u;
        __syncthreads();
        unsigned long long sse_fx = 0, ev = 0, npix = 0, nonzero = 0;
        bool bad = false;
        // Chunks of kChunk consecutive colors, one color per lane: warp w of
        // block b takes chunks c = b * WPB + w, then c + G * WPB, ...  The next
        // chunk's records are loaded while the current one is searched.
#ifdef WSM_CONTIGUOUS
        const int64_t per_block = (n + G - 1) / G;
        const int64_t blk_lo = min(n, (int64_t)b * per_block), blk_hi = min(n, blk_lo + per_block);
        int64_t cur = blk_lo + (int64_t)wid * kChunk;
        const int64_t stride = (int64_t)WPB * kChunk, lim = blk_hi;
#else
        int64_t cur = ((int64_t)b * WPB + wid) * kChunk;
        const int64_t stride = (int64_t)G * WPB * kChunk, lim = n;
#endif
        uint32_t col_n = 0, cnt_n = 0;
        int lab_n = 0;
        if (cur + lane < lim) {
            col_n = __ldg(P.colors + cur + lane);
            lab_n = P.labels[cur + lane];
            if (!kMap) cnt_n = __ldg(P.counts + cur + lane);
        }
        for (; cur < lim; cur += stride) {
            const int64_t nxt = cur + stride;
            const int64_t i = cur + lane;
            const bool active = i < lim;
            const uint32_t col = col_n;
            const unsigned cnt = cnt_n;
            const int p0 = lab_n;
            if (nxt + lane < lim) {
                col_n = __ldg(P.colors + nxt + lane);
                lab_n = P.labels[nxt + lane];
                if (!kMap) cnt_n = __ldg(P.counts + nxt + lane);
            }
            int p = p0;
            if (p >= K) {                          // invalid input membership
                bad = true;
                p = 0;
            }
            const float x = (float)((col >> 16) & 255u);
            const float y = (float)((col >> 8) & 255u);
            const float z = (float)(col & 255u);
            const float4 cp = s_c[p];
            const float prev = sq3(x, y, z, cp.x, cp.y, cp.z);
            float mn = prev;
            int mpos = 0;
            int j = 1;
            if (active) {
                const float4* row = P.tab + (size_t)p * K;
                bool more = true;
                // four entries per step; the row is sorted, so when the last
                // of them is below the bound, all four are visited
                for (; more && j + 3 < K; j += 4) {
                    const float4 e0 = row[j], e1 = row[j + 1], e2 = row[j + 2], e3 = row[j + 3];
                    if (e3.x < prev) {
                        WSM_VISIT(e0, j);
                        WSM_VISIT(e1, j + 1);
                        WSM_VISIT(e2, j + 2);
                        WSM_VISIT(e3, j + 3);
                    } else {
                        more = false;
                        if (e0.x < prev) {
                            WSM_VISIT(e0, j);
                            if (e1.x < prev) {
                                WSM_VISIT(e1, j + 1);
                                if (e2.x < prev) {
                                    WSM_VISIT(e2, j + 2);
                                    j += 3;
                                } else {
                                    j += 2;
                                }
                            } else {
                                j += 1;
                            }
                        }
                        break;
                    }
                }
                for (; more && j < K; ++j) {
                    const float4 e = row[j];
                    if (e.x >= prev) break;        // d[p][t] >= 4 prev_dist: stop
                    WSM_VISIT(e, j);
                }
                ev += (unsigned long long)j;       // c_p plus the j - 1 visited centers
                const int lab = mpos ? P.tab_nb[(size_t)p * K + mpos] : p;
                if (lab != p0) P.labels[i] = (uint8_t)lab;
                if (kMap) {
                    P.lut[col & 0xFFFFFFu] = (uint8_t)lab;
                } else {
                    atomicAdd(s_acc + 4 * lab + 0, cnt * ((col >> 16) & 255u));
                    atomicAdd(s_acc + 4 * lab + 1, cnt * ((col >> 8) & 255u));
                    atomicAdd(s_acc + 4 * lab + 2, cnt * (col & 255u));
                    atomicAdd(s_acc + 4 * lab + 3, cnt);
                    atomicMax(s_acc + 4 * K + lab, __float_as_uint(mn));
                    sse_fx += sse_fixed(cnt, mn);
                    npix += cnt;
                    nonzero += mn > 0.f;
                }
            }
        }
        if (bad) atomicOr(&P.ctrl->status, ST_BAD_LABEL);
        sse_fx = warp_sum_u64(sse_fx);
        ev = warp_sum_u64(ev);
        npix = warp_sum_u64(npix);
        nonzero = warp_sum_u64(nonzero);
        if (lane == 0) {
            s_red[0][wid] = sse_fx;
            s_red[1][wid] = ev;
            s_red[2][wid] = npix;
            s_red[3][wid] = nonzero;
        }
        __syncthreads();
        if (tid < 4) {
            unsigned long long t = 0;
            for (int w = 0; w < WPB; ++w) t += s_red[tid][w];
            if (kMap) {
                if (tid == 1 && t) atomicAdd(&P.ctrl->evaluated, t);
            } else if (t) {
                atomicAdd(P.sums64 + (size_t)(buf * kCopies + copy) * 4 + tid, t);
            }
        }
        if (kMap) break;
        {
            unsigned* dst = P.sums + (size_t)(buf * kCopies + copy) * 5 * K;
            for (int j = tid; j < 5 * K; j += T) {
                const unsigned v = s_acc[j];
                if (v) {
                    if (j < 4 * K) atomicAdd(dst + j, v);
                    else atomicMax(dst + j, v);
                }
            }
        }
        if (!grid_sync(P.ctrl, G)) return;

        // ---------------- phase A: totals, centers, stop rule, next table ----------------
        {
            const unsigned* src = P.sums + (size_t)buf * kCopies * 5 * K;
            for (int j = tid; j < 5 * K; j += T) {
                unsigned v[kCopies];
#pragma unroll
                for (int c = 0; c < kCopies; ++c) v[c] = src[(size_t)c * 5 * K + j];
                unsigned t = 0;
                if (j < 4 * K) {
#pragma unroll
                    for (int c = 0; c < kCopies; ++c) t += v[c];
                } else {
#pragma unroll
                    for (int c = 0; c < kCopies; ++c) t = max(t, v[c]);
                }
                s_acc[j] = t;
            }
        }
        if (wid == 0) {
            const unsigned long long* s64 = P.sums64 + (size_t)buf * kCopies * 4;
            unsigned long long fx = 0, evt = 0, N = 0, nz = 0;
            if (lane < kCopies) {
                fx = s64[lane * 4 + 0];
                evt = s64[lane * 4 + 1];
                N = s64[lane * 4 + 2];
                nz = s64[lane * 4 + 3];
            }
            fx = warp_sum_u64(fx);
            evt = warp_sum_u64(evt);
            N = warp_sum_u64(N);
            nz = warp_sum_u64(nz);
            if (lane == 0) {
                // Sec. 3.2: stop once (SSE_{i-1} - SSE_i) / SSE_i <= eps, i >= 2, or
                // SSE_i = 0; the common factor 2^-20 / N cancels in the ratio
                const int done = it + 1;
                bool stop = done >= P.max_iter;
                if (P.eps > 0.0) {
                    if (nz == 0) stop = true;
                    else if (done >= 2 && (double)((long long)(prev_fx - fx)) <= P.eps * (double)fx)
                        stop = true;
                }
                prev_fx = fx;
                s_stop = stop;
                if (b == 0) {
                    if (it < kMaxTrace)
                        P.trace[it] = N ? (double)fx * (1.0 / 1048576.0) / (double)N : 0.0;
                    P.ctrl->iters_done = done;
                    P.ctrl->evaluated += evt;
                }
            }
        }
        if (b == 0) {   // clear the accumulators of the next pass (read last two barriers ago)
            unsigned* nxt = P.sums + (size_t)(buf ^ 1) * kCopies * 5 * K;
            for (int j = tid; j < kCopies * 5 * K; j += T) nxt[j] = 0u;
            if (tid < 4 * kCopies) P.sums64[(size_t)(buf ^ 1) * kCopies * 4 + tid] = 0ull;
        }
        __syncthreads();
        {
            const float* s_cf = reinterpret_cast<const float*>(s_c);
            float* s_cnf = reinterpret_cast<float*>(s_cn);
            for (int u = tid; u < 3 * K; u += T) {
                const int k = u / 3, ch = u - 3 * k;
                const unsigned w = s_acc[4 * k + 3];
                s_cnf[4 * k + ch] = w ? div_rn_u32(s_acc[4 * k + ch], w, __frcp_rn((float)w))
                                      : s_cf[4 * k + ch];
            }
            if (b == 0)
                for (int j = tid; j < 4 * K; j += T) P.acc[j] = s_acc[j];
        }
        __syncthreads();
        // Row bound for the next pass: a member x of cluster k had
        // ||x - c_k|| <= sqrt(max_k) against the old center, so against the new
        // one prev <= (sqrt(max_k) + ||c_k,new - c_k,old||)^2 (triangle
        // inequality); a visit of row k never goes past 4 prev.  The margin
        // (x 1.001, + 1e-3) covers the FP32 rounding of these bounds.
        for (int k = tid; k < K; k += T) {
            const float4 o = s_c[k], c = s_cn[k];
            const float r = sqrtf(__uint_as_float(s_acc[4 * K + k])) +
                            sqrtf(sq3(o.x, o.y, o.z, c.x, c.y, c.z));
            s_thr[k] = 4.f * (r * r * 1.001f + 1e-3f);
            s_c[k] = make_float4(c.x, c.y, c.z, 0.f);
        }
        __syncthreads();
        if (s_stop) break;
        build_rows(P, s_c, s_thr, s_key, s_rank, s_cnt);
        if (!grid_sync(P.ctrl, G)) return;
    }

    // centers after the last update
    if (!kMap && b == 0)
        for (int k = tid; k < K; k += T) P.centers[k] = s_c[k];
}
#undef WSM_VISIT

static size_t sortmeans_smem(int K) { return (size_t)K * (16 + 16 + 8 + 20 + 4 + 4); }

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
// at most `cap` (the co-resident grid).
static int sortmeans_grid(int cap, int64_t n) {
    int64_t want = (n + kIterThreads - 1) / kIterThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

static int launch_with(bool map_mode, const uint32_t* colors, const uint32_t* counts, int64_t n,
                       int K, float* centers, uint8_t* labels, int max_iter, double eps,
                       float4* tab, uint8_t* tab_nb, unsigned* sums,
                       unsigned long long* sums64, unsigned long long* acc, double* trace,
                       uint8_t* lut, Ctrl* ctrl, int grid, cudaStream_t s) {
    SortMeansParams P;
    P.colors = colors;
    P.counts = counts;
    P.n = n;
    P.K = K;
    P.centers = reinterpret_cast<float4*>(centers);
    P.labels = labels;
    P.max_iter = max_iter;
    P.eps = eps;
    P.tab = tab;
    P.tab_nb = tab_nb;
    P.sums = sums;
    P.sums64 = sums64;
    P.acc = acc;
    P.trace = trace;
    P.lut = lut;
    P.ctrl = ctrl;
    void* args[] = {&P};
    void* fn = map_mode ? (void*)k_sortmeans<true> : (void*)k_sortmeans<false>;
    cudaError_t e = cudaMemsetAsync(ctrl, 0, kLaunchResetBytes, s);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel(fn, grid, kIterThreads, args, sortmeans_smem(K), s);
    if (e != cudaSuccess) return cuda_fail(e, "sort-means launch");
    return WSM_OK;
}

int launch_sortmeans(wsm_handle* h, bool map_mode, const uint32_t* colors, const uint32_t* counts,
                     int64_t n, int K, float* centers, uint8_t* labels, int max_iter, double eps,
                     cudaStream_t s) {
    return launch_with(map_mode, colors, counts, n, K, centers, labels, max_iter, eps,
                       h->tab, h->tab_nb, h->sums, h->sums64,
                       h->acc, h->trace, h->lut, h->ctrl, sortmeans_grid(h->iter_grid, n), s);
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
        if (c.iters_done < 1) return fail(WSM_E_STATE, "no completed iteration");
        unsigned long long buf[4 * WSM_MAX_K];
        e = cudaMemcpy(buf, h->acc, sizeof(unsigned long long) * 4 * K, cudaMemcpyDeviceToHost);
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
constexpr int kStaticMaxGrid = 1024;           // co-resident blocks used at most
constexpr size_t kStaticTabBytes = sizeof(float4) * kStaticMaxK * kStaticMaxK;   // 1 MiB
constexpr size_t kStaticNbBytes = (size_t)kStaticMaxK * kStaticMaxK;            // 64 KiB
constexpr size_t kStaticSumsBytes = sizeof(unsigned) * 2 * kCopies * 5 * kStaticMaxK;
constexpr size_t kStaticSums64Bytes = sizeof(unsigned long long) * 2 * kCopies * 4;
constexpr size_t kStaticAccBytes = sizeof(unsigned long long) * 4 * kStaticMaxK;
constexpr size_t kStaticTraceBytes = sizeof(double) * kMaxTrace;
constexpr size_t kStaticOffNb = kStaticTabBytes;
constexpr size_t kStaticOffSums = kStaticOffNb + kStaticNbBytes;
constexpr size_t kStaticOffSums64 = kStaticOffSums + kStaticSumsBytes;
constexpr size_t kStaticOffAcc = kStaticOffSums64 + kStaticSums64Bytes;
constexpr size_t kStaticOffTrace = kStaticOffAcc + kStaticAccBytes;
constexpr size_t kStaticOffCtrl = kStaticOffTrace + kStaticTraceBytes;
constexpr size_t kStaticBytes = kStaticOffCtrl + 256;           // about 1.2 MiB in total
static_assert(kStaticOffSums % 16 == 0 && kStaticOffCtrl % 16 == 0, "scratch alignment");

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
    double* trace = reinterpret_cast<double*>(base + kStaticOffTrace);
    // the status word starts at zero on every call (the launch clears the rest)
    e = cudaMemsetAsync(&ctrl->status, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "wsm_iterate_noalloc status clear");
    rc = launch_with(false, d_colors, d_counts, n_unique, K, d_centers, d_labels, max_iter, eps,
                     reinterpret_cast<float4*>(base), base + kStaticOffNb,
                     reinterpret_cast<unsigned*>(base + kStaticOffSums),
                     reinterpret_cast<unsigned long long*>(base + kStaticOffSums64),
                     reinterpret_cast<unsigned long long*>(base + kStaticOffAcc), trace, nullptr,
                     ctrl, sortmeans_grid(st->grid, n_unique), s);
    if (rc != WSM_OK) return rc;
    if (iters_done || sse_trace) {
        Ctrl host;
        e = cudaMemcpyAsync(&host, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "wsm_iterate_noalloc result copy");
        if (host.status & ST_TIMEOUT) return fail(WSM_E_TIMEOUT, "a device-side grid barrier timed out");
        if (host.status & ST_BAD_LABEL) return fail(WSM_E_INVAL, "a membership was >= K");
        if (iters_done) *iters_done = host.iters_done;
        if (sse_trace && host.iters_done > 0) {
            e = cudaMemcpyAsync(sse_trace, trace, sizeof(double) * std::min(host.iters_done, max_iter),
                                cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "wsm_iterate_noalloc trace copy");
        }
    }
    return WSM_OK;
}
