// wsm_iterate.cu -- the Sort-Means loop of Algorithm 2 (Sec. 2) as one
// persistent cooperative kernel over a batch of images, used for the
// iterations (wsm_iterate, wsm_iterate_batch) and for the final assignment
// before pixel mapping (wsm_map, wsm_map_batch).
//
// The blocks of a launch are split into one group per image (sized by the
// image's unique colors and palette); a group runs its image on its own, with
// a grid barrier of its own, so images of different sizes and iteration
// counts share one launch.  Within a group:
//   0  bound pass: every color's squared distance to its current center,
//      prev = ||x - c_p||^2, raises the largest prev of cluster p;
//   A  every block of the group turns the cluster sums of the previous pass
//      into the new centers c_k = S_k / W_k, one thread per center
//      (correctly rounded to FP32; an empty cluster keeps its center),
//      measures that pass's SSE and applies the Sec. 3.2 stop rule (all
//      blocks compute the same values, so all decide alike); then teams of
//      warps of the group's blocks
//      build the rows of the center table: row p lists, nearest first, the
//      entries (d[p][t] / 4, c_t), ties ordered by (t != p, t), so entry 0
//      is p.
//      A row keeps only the centers t with d[p][t] below four times a bound
//      on the prev of any member of cluster p -- no visit of row p goes
//      further (Sec. 2: the visit stops at d[p][t] >= 4 prev) -- followed by
//      four entries with an infinite bound; the entries a visit reads, and
//      their order, are those of the full row.  The bound is the largest
//      prev of the bound pass for the first table, and afterwards
//      (sqrt(largest min_dist of the pass) + ||c_p,new - c_p,old||)^2 by the
//      triangle inequality, with a margin for FP32 rounding.
//   B  the pruned nearest-center search, one lane per unique color; warp w
//      of block b takes the chunks of 32 consecutive colors numbered
//      b * WPB + w + k * G * WPB and loads the next chunk's records while it
//      searches the current one.  A color starts at its previous center p
//      and visits row p from entry 1 on; the visit stops at the first entry
//      with d[p][t] / 4 >= prev (the paper's d[p][t] >= 4 prev_dist; scaling
//      by 4 is exact), and a visited center replaces the current one when its
//      distance is <= the running minimum, so among equal distances the one
//      visited last wins.  Entries are loaded four at a time and all four
//      distances computed; a row is sorted, so the entries below the bound
//      are a prefix of it, and only those take part in the update, in row
//      order.  Cluster sums (uint32, exact because an image has at most
//      2^24 pixels) are accumulated per block in shared memory and added into
//      the global accumulators (kCopies copies; integer atomics: the
//      totals are exact and independent of the order).  The first pass of a
//      launch sums every color; later passes keep the totals and move only
//      the colors whose membership changed from their old cluster to their
//      new one.
// The SSE is accumulated as an integer in units of 2^-20 (each color's
// n_i * min_dist_i truncated to that grid), so every reduction is exact and
// the results do not depend on the grid, the grouping or the order.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "wsm_internal.cuh"
#include "wsm_split.h"

namespace wsm {

// One image of a launch.
struct ItemDesc {
    const uint32_t* colors;    // [n] ascending 0xRRGGBB
    const uint32_t* counts;    // [n]
    void* labels;              // [n] in/out, uint8 or uint16 (the handle's label width)
    float4* centers;           // [K] in/out (read-only in the map mode)
    int64_t n;
    int K;
    int slot;                  // scratch slot
    int64_t* nu_out = nullptr;     // iterations: N' and the iterations run, written by the
    int* iters_out = nullptr;      //   group's first block at its exit (may be null)
};

// Per-image scratch: slot s of each array starts at base + s * (its slot size).
struct Scratch {
    float4* tab;               // [max_K^2] rows of (d/4, c.x, c.y, c.z), nearest first
    void* tab_nb;              // [max_K^2] center index of each entry (label width)
    unsigned* sums;            // [2][kCopies][5 max_K] by pass parity: the largest prev /
                               //   min_dist of a member (last K words, FP32 bits); the
                               //   first 4K words of parity 0 hold the running cluster
                               //   sums of the launch (those of parity 1 are unused)
    unsigned long long* sums64;    // [2][kCopies][4] SSE (2^-20 units), distances, pixels,
                                   //   colors with a nonzero minimum
    unsigned long long* acc;   // [4 max_K] cluster sums of the last pass
    double* trace;             // [kMaxTrace]
    void* lut;                 // [2^24] color -> label (map mode; label width)
    void* grid;                // [kGridCells] a nearby center for each 16^3 cell of the RGB
                               //   cube (label width)
    Ctrl* ctrl;                // barrier counter, iterations, distances
    int max_K;
    int label_bytes;           // 1: uint8 memberships and entries; 2: uint16
};

struct BatchParams {
    Scratch sc;
    unsigned* status;          // ST_* bits for the whole call
    int n_items;
    int max_iter;
    double eps;
    const int64_t* n_dev;      // if set, image i has n_dev[item[i].slot] colors (written by an
                               //   earlier kernel) and the split is first_dev (k_plan)
    const int* first_dev;
    const int* weight;         // with n_dev: per-slot work weights for the split (may be null)
    int cand_start;            // first pass of an iterate launch starts at the grid candidate
    int first_blk[kMaxBatch + 1];  // image i owns blocks [first_blk[i], first_blk[i+1])
    ItemDesc item[kMaxBatch];
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

// Before a launch whose image sizes are on the device: the words the
// persistent kernel needs at zero (the slots' control blocks and both
// parities of their accumulators, `nz` 32-bit words in three ranges) are
// cleared by all threads, and the block split is written to first_dev by
// thread 0 of block 0.
struct ClearRanges {
    unsigned* p[3];
    size_t n[3];
};

__global__ void k_plan(const __grid_constant__ BatchParams P, int threads, int grid,
                       int* first_dev, const __grid_constant__ ClearRanges Z) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nt = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < 3; ++r)
        for (size_t q = t; q < Z.n[r]; q += nt) Z.p[r][q] = 0u;
    if (t != 0) return;
    int64_t want[kMaxBatch];
    for (int i = 0; i < P.n_items; ++i) {
        // a measured work weight (1/1024 units) scales the image's share
        want[i] = weighted_want(group_want(P.n_dev[P.item[i].slot], P.item[i].K, threads),
                                P.weight ? P.weight[P.item[i].slot] : 0);
    }
    split_groups(want, P.n_items, grid, first_dev);
}

// Cell of the 16^3 grid over the RGB cube that holds color 0x00RRGGBB.
__device__ __forceinline__ int grid_cell(uint32_t col) {
    return (int)(((col >> 12) & 0xF00u) | ((col >> 8) & 0xF0u) | ((col >> 4) & 0xFu));
}

// Sort key of center t in row p, exactly as build_rows computes it.
__device__ __forceinline__ unsigned long long key_in_row(const float4* s_c, int p, int t) {
    const float4 a = s_c[p], c = s_c[t];
    return row_key(sq3(a.x, a.y, a.z, c.x, c.y, c.z), t, p);
}

struct CandResult {
    int best;      // the winner, or -1 if row p must be visited after all
    float mn;      // its squared distance
    int visits;    // distances computed
};

// The first-pass search of color x (membership p, prev = ||x - c_p||^2) from
// the grid candidate q != p: visits row q up to the bound dq = ||x - c_q||^2
// (no center past it is nearer than c_q), keeping the nearest center with
// ties to the one latest in row p, and returns it if Algorithm 2's visit of
// row p would meet it (d[p][t] / 4 < prev, or t = p).
template <typename Label>
__device__ __forceinline__ CandResult candidate_search(float x, float y, float z, int p, int q,
                                                    float prev, int K, const float4* s_c,
                                                    const float4* tab, const Label* tab_nb) {
    const float4 cq = s_c[q];
    const float dq = sq3(x, y, z, cq.x, cq.y, cq.z);
    const float4* rq = tab + q * K;
    const Label* nq = tab_nb + q * K;
    int bpos = -1;                 // the best so far: c_p (-1), c_q (0) or entry bpos of row q
    float bmn = prev;
    if (dq <= prev) {              // c_q is later than c_p in row p
        bpos = 0;
        bmn = dq;
    }
    int v = 2;
    const auto center_at = [&](int pos) { return pos < 0 ? p : pos == 0 ? q : (int)nq[pos]; };
    // entry e at position pos of row q, when `in` (it is within the bound)
    const auto visit = [&](const float4& e, int pos, bool in) {
        const float d = sq3(x, y, z, e.y, e.z, e.w);
        v += (int)in;
        if (in && d < bmn) {
            bmn = d;
            bpos = pos;
        } else if (in && d == bmn &&
                   key_in_row(s_c, p, center_at(pos)) > key_in_row(s_c, p, center_at(bpos))) {
            bpos = pos;
        }
    };
    // rounds of four entries, the entries up to the bound being a prefix of
    // the sorted row (as in the assignment pass)
    int j = 1;
    bool go = true;
    for (; go && j + 3 < K; j += 4) {
        const float4 e0 = rq[j], e1 = rq[j + 1], e2 = rq[j + 2], e3 = rq[j + 3];
        const bool v0 = e0.x <= dq, v1 = e1.x <= dq, v2 = e2.x <= dq, v3 = e3.x <= dq;
        visit(e0, j, v0);
        visit(e1, j + 1, v1);
        visit(e2, j + 2, v2);
        visit(e3, j + 3, v3);
        go = v3;
    }
    for (; go && j < K; ++j) {
        const float4 e = rq[j];
        if (e.x > dq) break;
        visit(e, j, true);
    }
    const int best = center_at(bpos);
    const float4 cp = s_c[p], cb = s_c[best];
    CandResult r;
    r.best = (best == p || sq3(cp.x, cp.y, cp.z, cb.x, cb.y, cb.z) * 0.25f < prev) ? best : -1;
    r.mn = bmn;
    r.visits = v;
    return r;
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
// The same for an entry of a round when `v` (the entry is below the bound).
#define WSM_VISIT_IF(e, jj, v)                                  \
    {                                                           \
        const float dist_ = sq3(x, y, z, (e).y, (e).z, (e).w);  \
        if ((v) && dist_ <= mn) {                               \
            mn = dist_;                                         \
            mpos = (jj);                                        \
        }                                                       \
    }

// One assignment pass over an image's colors by one warp (phase B of
// k_sortmeans): the warp's chunks of 32 colors, one color per lane, each
// color's pruned visit of its row, and the per-block sums.  kCand: the first
// pass of an iterate launch, whose search starts at the grid candidate.
// kDelta: the cluster sums of the previous pass are kept, so only a color
// whose membership changes adds its terms, to its new cluster, and takes
// them from its old one (the totals stay exact: integer sums).
// Raises the shared word *a to v; a plain read first skips the atomic when the
// word is already at least v (words only grow within a pass, so a stale read
// can only cost an atomic, never lose a maximum).
__device__ __forceinline__ void smem_max_u32(unsigned* a, unsigned v) {
    if (v > *reinterpret_cast<volatile unsigned*>(a)) atomicMax(a, v);
}

template <bool kMap, bool kCand, bool kDelta, typename Label>
__device__ __forceinline__ void assign_pass(const ItemDesc& I, int n, int K, int G, int b,
                                            int WPB, int lane, int wid, unsigned* ticket,
                                            const float4* s_c, unsigned* s_acc, const float4* tab,
                                            const Label* tab_nb, const Label* grid, Label* lut,
                                            unsigned long long& sse_fx, unsigned long long& ev,
                                            unsigned long long& npix, unsigned long long& nonzero,
                                            bool& bad) {
    // Chunks: warp w of block b starts with chunk b * WPB + w, then takes
    // chunks G * WPB + t in the order of the tickets t it draws from the
    // slot's counter (each ticket drawn one chunk ahead), so the warps of
    // the group finish together whatever the cost of their colors.
    // per-lane counts of this pass fit 32 bits (at most 2^24 pixels per image)
    unsigned ev32 = 0, npix32 = 0, nz32 = 0;
    int cur = (b * WPB + wid) * kChunk;                 // colors: at most 2^24
    int nxt = n;
    {
        unsigned t = 0;
        if (lane == 0 && cur < n) t = atomicAdd(ticket, 1u);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        if (cur < n) nxt = (G * WPB + (int)t) * kChunk;
    }
    Label* const labels = static_cast<Label*>(I.labels);
    uint32_t col_n = 0, cnt_n = 0;
    int lab_n = 0;
    if (cur + lane < n) {
        col_n = __ldg(I.colors + cur + lane);
        lab_n = labels[cur + lane];
        if (!kMap || I.counts) cnt_n = __ldg(I.counts + cur + lane);
    }
    while (cur < n) {
        const int i = cur + lane;
        const bool active = i < n;
        const uint32_t col = col_n;
        const unsigned cnt = cnt_n;
        const int p0 = lab_n;
        unsigned t_after = 0;
        if (nxt < n) {
            if (nxt + lane < n) {
                col_n = __ldg(I.colors + nxt + lane);
                lab_n = labels[nxt + lane];
                if (!kMap || I.counts) cnt_n = __ldg(I.counts + nxt + lane);
            }
            if (lane == 0) t_after = atomicAdd(ticket, 1u);   // used after this chunk
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
        int lab = p;
        bool scan_p = active;
        if (kCand && active) {
            // First pass of the launch, where the memberships may be far
            // off (all 0 after the initialisation): the same outcome as the
            // visit of row p from a nearer start.  With q the grid
            // candidate and dq = ||x - c_q||^2, every center at least as
            // near as c_q has d[q][t] <= 4 dq, so visiting row q up to that
            // bound meets every nearest center; among equal distances the
            // one latest in row p wins (the later visit wins in row p).
            // If the winner would not be visited in row p (d[p][t] >=
            // 4 prev, which the triangle inequality rules out but for
            // rounding at the bound), row p is visited as usual.
            const int q = grid[grid_cell(col)];
            if (q != p) {
                const CandResult r =
                    candidate_search<Label>(x, y, z, p, q, prev, K, s_c, tab, tab_nb);
                if (r.best >= 0) {
                    scan_p = false;
                    lab = r.best;
                    mn = r.mn;
                    ev32 += (unsigned)r.visits;
                }
            }
        }
        if (scan_p) {
            const float4* row = tab + p * K;
            bool more = true;
            // Rounds of four entries.  A row is sorted, so the entries below the
            // bound are a prefix of it: the visit stops within the first round
            // whose last entry is not below it.  Every entry of a round has its
            // distance computed and only those below the bound take part in the
            // update, in row order, so a warp runs one path through a round.
            for (; more && j + 3 < K; j += 4) {
                const float4 e0 = row[j], e1 = row[j + 1], e2 = row[j + 2], e3 = row[j + 3];
                const bool v0 = e0.x < prev, v1 = e1.x < prev, v2 = e2.x < prev, v3 = e3.x < prev;
                WSM_VISIT_IF(e0, j, v0);
                WSM_VISIT_IF(e1, j + 1, v1);
                WSM_VISIT_IF(e2, j + 2, v2);
                WSM_VISIT_IF(e3, j + 3, v3);
                if (!v3) {                     // d[p][t] >= 4 prev_dist within this round: stop
                    j += (int)v0 + (int)v1 + (int)v2;
                    more = false;
                    break;
                }
            }
            for (; more && j < K; ++j) {
                const float4 e = row[j];
                if (e.x >= prev) break;        // d[p][t] >= 4 prev_dist: stop
                WSM_VISIT(e, j);
            }
            ev32 += (unsigned)j;               // c_p plus the j - 1 visited centers
            lab = mpos ? tab_nb[p * K + mpos] : p;
        }
        if (active) {
            if (lab != p0) labels[i] = (Label)lab;
            if (kMap) {
                lut[col & 0xFFFFFFu] = (Label)lab;
                // Eq. 2 over the pixels of this color, each pixel's squared
                // distance truncated to 2^-20 units as the per-pixel MSE does
                sse_fx += (unsigned long long)cnt * sse_fixed(1u, mn);
            } else {
                if (!kDelta || lab != p) {
                    const unsigned sr = cnt * ((col >> 16) & 255u), sg = cnt * ((col >> 8) & 255u),
                                   sb = cnt * (col & 255u);
                    atomicAdd(s_acc + 4 * lab + 0, sr);
                    atomicAdd(s_acc + 4 * lab + 1, sg);
                    atomicAdd(s_acc + 4 * lab + 2, sb);
                    atomicAdd(s_acc + 4 * lab + 3, cnt);
                    if (kDelta) {              // modulo 2^32: the totals are below 2^32
                        atomicSub(s_acc + 4 * p + 0, sr);
                        atomicSub(s_acc + 4 * p + 1, sg);
                        atomicSub(s_acc + 4 * p + 2, sb);
                        atomicSub(s_acc + 4 * p + 3, cnt);
                    }
                }
                smem_max_u32(s_acc + 4 * K + lab, __float_as_uint(mn));
                sse_fx += sse_fixed(cnt, mn);
                npix32 += cnt;
                nz32 += mn > 0.f;
            }
        }
        const unsigned t = __shfl_sync(0xFFFFFFFFu, t_after, 0);
        cur = nxt;
        nxt = cur < n ? (G * WPB + (int)t) * kChunk : n;
    }
    ev += ev32;
    npix += npix32;
    nonzero += nz32;
}

template <bool kMap, int kThreads, typename Label>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads)
    k_sortmeans(const __grid_constant__ BatchParams P) {
    // ---- this block's image and group
    const int* first_blk = P.first_dev ? P.first_dev : P.first_blk;
    if ((int)blockIdx.x >= first_blk[P.n_items]) return;   // not needed by any image
    const int ii = item_of_block(first_blk, P.n_items, blockIdx.x);
    const ItemDesc I = P.item[ii];
    const int G = first_blk[ii + 1] - first_blk[ii];
    const int b = blockIdx.x - first_blk[ii];
    const int K = I.K;
    const int64_t n = P.n_dev ? P.n_dev[I.slot] : I.n;
    // sizes from the device were checked by the initialisation, which flagged
    // an image with fewer unique colors than K; such an image is skipped
    // the caller's copies of N' and of the iterations run, at every exit
    Ctrl* const gctrl = P.sc.ctrl + I.slot;
    if (!kMap && b == 0 && threadIdx.x == 0) gctrl->t_start = global_ns();
    const auto outputs = [&](int iters) {
        if (!kMap && b == 0 && threadIdx.x == 0) {
            if (I.nu_out) *I.nu_out = n;
            if (I.iters_out) *I.iters_out = iters;
            gctrl->t_end = global_ns();
        }
    };
    if (P.n_dev && n < K) {
        outputs(0);
        return;
    }
    const size_t kk = (size_t)P.sc.max_K * P.sc.max_K, s5 = (size_t)5 * P.sc.max_K;
    float4* const tab = P.sc.tab + (size_t)I.slot * kk;
    Label* const tab_nb = static_cast<Label*>(P.sc.tab_nb) + (size_t)I.slot * kk;
    unsigned* const sums = P.sc.sums + (size_t)I.slot * 2 * kCopies * s5;
    unsigned long long* const sums64 = P.sc.sums64 + (size_t)I.slot * 2 * kCopies * 4;
    unsigned long long* const acc = P.sc.acc + (size_t)I.slot * 4 * P.sc.max_K;
    double* const trace = P.sc.trace + (size_t)I.slot * kMaxTrace;
    Label* const lut = kMap ? static_cast<Label*>(P.sc.lut) + (size_t)I.slot * kHistBins : nullptr;
    Ctrl* const ctrl = P.sc.ctrl + I.slot;

    extern __shared__ float4 smem[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int T = blockDim.x, WPB = T >> 5;
    const int KM = P.sc.max_K;                  // smem arrays are sized for the batch's largest K
    float4* s_c = smem;                                                       // [KM] centers
    unsigned* s_acc = reinterpret_cast<unsigned*>(s_c + KM);                  // [5KM] sums, max
    float* s_thr = reinterpret_cast<float*>(s_acc + 5 * KM);                  // [KM] row bounds
    unsigned long long* s_wkey = reinterpret_cast<unsigned long long*>(s_thr + KM);
    // row keys: [WPB][KM], or [2 KM] for palettes of more than 256 colors
    Label* const s_grid =                                     // [kGridCells] candidate grid
        reinterpret_cast<Label*>(s_wkey + (KM > WSM_MAX_K ? 2 * KM : WPB * KM));
    __shared__ unsigned long long s_red[4][kThreads / 32];
    __shared__ int s_stop;

    const int copy = b % kCopies;
    if (!kMap && P.max_iter <= 0) {
        outputs(0);
        return;
    }

    // the slot's accumulators (both parities) were cleared before the launch
    for (int k = tid; k < K; k += T) s_c[k] = I.centers[k];
    for (int j = tid; j < 5 * K; j += T) s_acc[j] = 0u;
    __syncthreads();

    // The candidate grid (iterations only): for every 16^3 cell of the RGB
    // cube the center nearest to the cell's middle, where the first pass of
    // the launch starts each color's search (see there).
    Label* const grid = static_cast<Label*>(P.sc.grid) + (size_t)I.slot * kGridCells;
    const bool cand = !kMap && P.cand_start;
    if (cand) {
        const int nt = G * T;
        if (nt >= 2 * kGridCells) {
            // `sub` consecutive lanes (2, 4 or 8) share a cell and scan every
            // sub-th center; the reduction keeps the smaller distance and,
            // between equal ones, the lower index, as the one-lane scan does.
            // Every lane runs the shuffles (cells fill whole warps).
            int sub = 2;
            while (sub < 8 && nt >= 2 * sub * kGridCells) sub *= 2;
            const int gt = b * T + tid, c = gt / sub, part = gt % sub;
            float bd = __int_as_float(0x7f800000);
            int bt = 0;
            if (c < kGridCells) {
                const float gx = (float)((c >> 8) * 16 + 8), gy = (float)(((c >> 4) & 15) * 16 + 8),
                            gz = (float)((c & 15) * 16 + 8);
                for (int k = part; k < K; k += sub) {
                    const float4 ck = s_c[k];
                    const float d = sq3(gx, gy, gz, ck.x, ck.y, ck.z);
                    if (d < bd) {
                        bd = d;
                        bt = k;
                    }
                }
            }
            for (int o = 1; o < sub; o <<= 1) {
                const float od = __shfl_xor_sync(0xFFFFFFFFu, bd, o);
                const int ot = __shfl_xor_sync(0xFFFFFFFFu, bt, o);
                if (od < bd || (od == bd && ot < bt)) {
                    bd = od;
                    bt = ot;
                }
            }
            if (c < kGridCells && part == 0) grid[c] = (Label)bt;
        } else {
            for (int c = b * T + tid; c < kGridCells; c += nt) {
                const float gx = (float)((c >> 8) * 16 + 8), gy = (float)(((c >> 4) & 15) * 16 + 8),
                            gz = (float)((c & 15) * 16 + 8);
                float bd = __int_as_float(0x7f800000);
                int bt = 0;
                for (int k = 0; k < K; ++k) {
                    const float4 ck = s_c[k];
                    const float d = sq3(gx, gy, gz, ck.x, ck.y, ck.z);
                    if (d < bd) {
                        bd = d;
                        bt = k;
                    }
                }
                grid[c] = (Label)bt;
            }
        }
        if (!grid_sync(&ctrl->bar_count, P.status, G)) return;
        // every block keeps a copy in shared memory for the first pass
        for (int c = tid; c < kGridCells; c += T) s_grid[c] = grid[c];
        __syncthreads();
    }

    // Colors of this block: chunks of kChunk, one per lane, warp w of block b
    // takes chunks b * WPB + w + m * G * WPB.
    const int64_t first = ((int64_t)b * WPB + wid) * kChunk;
    const int64_t stride = (int64_t)G * WPB * kChunk;

    // ---------------- bound pass ----------------
    {
        bool bad = false;
        for (int64_t cur = first; cur < n; cur += stride) {
            const int64_t i = cur + lane;
            if (i < n) {
                const uint32_t col = __ldg(I.colors + i);
                int p = static_cast<const Label*>(I.labels)[i];
                if (p >= K) {
                    bad = true;
                    p = 0;
                }
                const float x = (float)((col >> 16) & 255u), y = (float)((col >> 8) & 255u),
                            z = (float)(col & 255u);
                const float4 cp = s_c[p];
                const float prev = sq3(x, y, z, cp.x, cp.y, cp.z);
                smem_max_u32(s_acc + 4 * K + p, __float_as_uint(prev));
                if (cand) {                        // the first pass also reads row q
                    const int q = s_grid[grid_cell(col)];
                    if (q != p) {
                        const float4 cq = s_c[q];
                        const float dq = sq3(x, y, z, cq.x, cq.y, cq.z);
                        smem_max_u32(s_acc + 4 * K + q, __float_as_uint(dq));
                    }
                }
            }
        }
        if (bad) atomicOr(P.status, ST_BAD_LABEL);
        __syncthreads();
        unsigned* dst = sums + (size_t)(kCopies + copy) * s5;   // parity 1, zeroed above
        for (int k = tid; k < K; k += T) {
            const unsigned v = s_acc[4 * K + k];
            if (v) atomicMax(dst + 4 * K + k, v);
        }
        if (!grid_sync(&ctrl->bar_count, P.status, G)) return;
        for (int k = tid; k < K; k += T) {
            unsigned m = 0;
#pragma unroll
            for (int c = 0; c < kCopies; ++c)
                m = max(m, sums[(size_t)(kCopies + c) * s5 + 4 * K + k]);
            s_thr[k] = 4.f * (__uint_as_float(m) * 1.001f + 1e-3f);
        }
        __syncthreads();
        build_rows<Label>(K, KM, G, b, s_c, s_thr, s_wkey, tab, tab_nb);
        if (!grid_sync(&ctrl->bar_count, P.status, G)) return;
    }

    unsigned long long prev_fx = 0;        // SSE of the previous pass, in the stop-rule lane only
    // The stop rule runs in the block's last warp: with fewer centers than
    // threads it has no center of its own in phase A, so the rule stays off
    // the path of the centers (iterations 0.413-0.414 -> 0.410-0.413 ms with
    // the prefetch below).
    const int w_stop = WPB - 1;
    for (int it = 0;; ++it) {
        // ---------------- phase B: assignment ----------------
        const int buf = it & 1;
        for (int j = tid; j < 5 * K; j += T) s_acc[j] = 0u;
        __syncthreads();
        unsigned long long sse_fx = 0, ev = 0, npix = 0, nonzero = 0;
        bool bad = false;
        unsigned* const ticket = &ctrl->ticket[buf];
        if constexpr (!kMap) {
            if (it > 0)                        // the totals of the previous pass are kept
                assign_pass<false, false, true, Label>(I, (int)n, K, G, b, WPB, lane, wid, ticket,
                                                       s_c, s_acc, tab, tab_nb, s_grid, lut, sse_fx,
                                                       ev, npix, nonzero, bad);
            else if (cand)
                assign_pass<false, true, false, Label>(I, (int)n, K, G, b, WPB, lane, wid, ticket,
                                                       s_c, s_acc, tab, tab_nb, s_grid, lut, sse_fx,
                                                       ev, npix, nonzero, bad);
            else
                assign_pass<false, false, false, Label>(I, (int)n, K, G, b, WPB, lane, wid, ticket,
                                                        s_c, s_acc, tab, tab_nb, s_grid, lut, sse_fx,
                                                        ev, npix, nonzero, bad);
        } else {
            assign_pass<true, false, false, Label>(I, (int)n, K, G, b, WPB, lane, wid, ticket, s_c,
                                                   s_acc, tab, tab_nb, s_grid, lut, sse_fx, ev,
                                                   npix, nonzero, bad);
        }
        if (bad) atomicOr(P.status, ST_BAD_LABEL);
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
                if (tid == 0 && t) atomicAdd(&ctrl->map_sse, t);
                if (tid == 1 && t) atomicAdd(&ctrl->evaluated, t);
            } else if (t) {
                atomicAdd(sums64 + (size_t)(buf * kCopies + copy) * 4 + tid, t);
            }
        }
        if (kMap) break;
        {
            // the block's changes of the running totals (parity 0 of its copy) and
            // its maxima of the pass (this parity)
            unsigned* tot = sums + (size_t)copy * s5;
            unsigned* dst = sums + (size_t)(buf * kCopies + copy) * s5;
            for (int j = tid; j < 5 * K; j += T) {
                const unsigned v = s_acc[j];
                if (v) {
                    if (j < 4 * K) atomicAdd(tot + j, v);
                    else atomicMax(dst + j, v);
                }
            }
        }
        if (!grid_sync(&ctrl->bar_count, P.status, G)) return;

        // ---------------- phase A: totals, centers, stop rule, next table ----------------
        // Every load of the totals a thread needs is issued before any is
        // used: right after the barrier they come from L2 lines that all
        // blocks of the group have just updated, and a chain of dependent
        // rounds of loads costs microseconds.  The block's threads read the
        // totals of their centers directly, so one block barrier ends the phase.
        unsigned long long fx = 0, evt = 0, N = 0, nz = 0;
        if (wid == w_stop && lane < kCopies) {
            const unsigned long long* s64 = sums64 + (size_t)buf * kCopies * 4;
            fx = s64[lane * 4 + 0];
            evt = s64[lane * 4 + 1];
            N = s64[lane * 4 + 2];
            nz = s64[lane * 4 + 3];
        }
        if (b == 0) {   // clear the maxima of the next pass (read two barriers ago)
            unsigned* nxt = sums + (size_t)(buf ^ 1) * kCopies * s5;
            for (int j = tid; j < kCopies * K; j += T) {
                const int c = j / K, r = j - c * K;
                nxt[(size_t)c * s5 + 4 * K + r] = 0u;
            }
            if (tid < 4 * kCopies) sums64[(size_t)(buf ^ 1) * kCopies * 4 + tid] = 0ull;
            if (tid == 0) ctrl->ticket[buf ^ 1] = 0u;   // drawn from two barriers ago
        }
        // One thread per center: its totals (the running sums and this pass's
        // largest member distance), the new center c_k = S_k / W_k (an empty
        // cluster keeps its center) and the bound of its next row.  A member x
        // of cluster k had ||x - c_k|| <= sqrt(max_k) against the old center,
        // so against the new one prev <= (sqrt(max_k) + ||c_k,new - c_k,old||)^2
        // (triangle inequality); a visit of row k never goes past 4 prev.  The
        // margin (x 1.001, + 1e-3) covers the FP32 rounding of these bounds.
        {
            const unsigned* mx = sums + (size_t)buf * kCopies * s5 + 4 * K;
            for (int k = tid; k < K; k += T) {
                unsigned v[5][kCopies];
#pragma unroll
                for (int c = 0; c < kCopies; ++c) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q][c] = sums[(size_t)c * s5 + 4 * k + q];
                    v[4][c] = mx[(size_t)c * s5 + k];
                }
                unsigned S[4] = {0u, 0u, 0u, 0u}, M = 0u;
#pragma unroll
                for (int c = 0; c < kCopies; ++c) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) S[q] += v[q][c];
                    M = max(M, v[4][c]);
                }
                const float4 o = s_c[k];
                float4 cn = make_float4(o.x, o.y, o.z, 0.f);
                if (S[3]) {
                    const float rcp = __frcp_rn((float)S[3]);
                    cn.x = div_rn_u32(S[0], S[3], rcp);
                    cn.y = div_rn_u32(S[1], S[3], rcp);
                    cn.z = div_rn_u32(S[2], S[3], rcp);
                }
                const float r = sqrtf(__uint_as_float(M)) + sqrtf(sq3(o.x, o.y, o.z, cn.x, cn.y, cn.z));
                s_thr[k] = 4.f * (r * r * 1.001f + 1e-3f);
                s_c[k] = cn;
                if (b == 0) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[4 * k + q] = S[q];
                }
            }
        }
        if (wid == w_stop) {
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
                        trace[it] = N ? (double)fx * (1.0 / 1048576.0) / (double)N : 0.0;
                    ctrl->iters_done = done;
                    ctrl->evaluated += evt;
                }
            }
        }
        __syncthreads();
        if (s_stop) break;
        if (!kMap) {
            // the records of this warp's first chunk of the next pass into L1
            // (the memberships of this pass are final): their loads then do
            // not start cold after the barrier
            const int64_t i0 = first + lane;
            if (i0 < n) {
                asm volatile("prefetch.global.L1 [%0];" ::"l"(I.colors + i0));
                asm volatile("prefetch.global.L1 [%0];" ::"l"(I.counts + i0));
                asm volatile("prefetch.global.L1 [%0];" ::"l"(static_cast<const Label*>(I.labels) + i0));
            }
        }
        build_rows<Label>(K, KM, G, b, s_c, s_thr, s_wkey, tab, tab_nb);
        if (!grid_sync(&ctrl->bar_count, P.status, G)) return;
    }

    // centers after the last update
    if (!kMap && b == 0)
        for (int k = tid; k < K; k += T) I.centers[k] = s_c[k];
    outputs(ctrl->iters_done);          // written by this thread in phase A
}
#undef WSM_VISIT
#undef WSM_VISIT_IF

// Dynamic shared memory of k_sortmeans for palettes of up to KM colors.
static size_t sortmeans_smem(int KM, int threads, bool map_mode) {
    const size_t keys = KM > WSM_MAX_K ? (size_t)2 * KM : (size_t)(threads / 32) * KM;
    // the candidate grid of the first pass (iterations only)
    const size_t grid = map_mode ? 0 : (size_t)kGridCells * (KM > WSM_MAX_K ? 2 : 1);
    return (size_t)KM * (16 + 20 + 4) + keys * 8 + grid;
}

// The launch shapes of the persistent kernel: threads per block and blocks
// per SM (the grid is that many blocks on every SM, all co-resident).
const IterShape kIterShapes[kNumIterShapes] = {{512, 2}, {256, 4}, {1024, 1}, {256, 2}, {512, 1}};

// The kernel for a launch; uint16 memberships only with 512 threads per
// block (nullptr for the other shapes).
static void* sortmeans_fn(bool map_mode, int threads, int label_bytes) {
    if (label_bytes == 2) {
        if (threads != 512) return nullptr;
        return map_mode ? (void*)k_sortmeans<true, 512, uint16_t>
                        : (void*)k_sortmeans<false, 512, uint16_t>;
    }
    switch (threads) {
        case 256:
            return map_mode ? (void*)k_sortmeans<true, 256, uint8_t>
                            : (void*)k_sortmeans<false, 256, uint8_t>;
        case 1024:
            return map_mode ? (void*)k_sortmeans<true, 1024, uint8_t>
                            : (void*)k_sortmeans<false, 1024, uint8_t>;
        default:
            return map_mode ? (void*)k_sortmeans<true, 512, uint8_t>
                            : (void*)k_sortmeans<false, 512, uint8_t>;
    }
}

// The dynamic shared-memory limit of a kernel belongs to the function on the
// current device, not to a handle: every handle and wsm_iterate_noalloc share
// it.  It is only ever raised, to the largest size any caller on that device
// has asked for, so that creating a handle for a small palette never takes
// the room away from a launch sized for a larger one.
cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
    static std::mutex mutex;
    static std::map<std::pair<int, const void*>, size_t> limits;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mutex);
    size_t& cur = limits[{dev, fn}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// Residency of each launch shape for palettes of up to max_K colors; the
// handle starts with the first shape that fits.
int iterate_kernel_setup(wsm_handle* h) {
    h->iter_shape = -1;
    for (int q = 0; q < kNumIterShapes; ++q) {
        const IterShape& sh = kIterShapes[q];
        const size_t smem = sortmeans_smem(h->max_K, sh.threads, false);   // the larger
        int occ = 1 << 30;
        for (int m = 0; m < 2; ++m) {
            void* fn = sortmeans_fn(m == 1, sh.threads, h->label_bytes);
            if (!fn) {
                occ = 0;
                break;
            }
            int o = 0;
            cudaError_t e = raise_smem_limit(fn, smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, sh.threads, smem);
            if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
            occ = std::min(occ, o);
        }
        h->shape_ok[q] = occ >= sh.blocks_per_sm;
        if (h->shape_ok[q] && h->iter_shape < 0) h->iter_shape = q;
    }
    if (h->iter_shape < 0) return fail(WSM_E_CUDA, "persistent kernel cannot be resident");
    return WSM_OK;
}

// Blocks of the persistent launches: the shape's full co-resident grid, or
// fewer if the handle is limited to a share of the GPU.
int iter_grid(const wsm_handle* h) {
    const int full = kIterShapes[h->iter_shape].blocks_per_sm * h->sms;
    return h->grid_limit > 0 ? std::min(full, h->grid_limit) : full;
}

static Scratch handle_scratch(wsm_handle* h) {
    Scratch sc;
    sc.tab = h->tab;
    sc.tab_nb = h->tab_nb;
    sc.sums = h->sums;
    sc.sums64 = h->sums64;
    sc.acc = h->acc;
    sc.trace = h->trace;
    sc.lut = h->lut;
    sc.grid = h->grid;
    sc.ctrl = h->slot_ctrl;
    sc.max_K = h->max_K;
    sc.label_bytes = h->label_bytes;
    return sc;
}

// One cooperative launch over n_items <= kMaxBatch images (item i in the
// slot it names) with `threads` per block on at most grid_cap blocks.  With
// n_dev the image sizes are read on the device (n_dev[slot]), k_plan writes
// the split to first_dev ([kMaxBatch + 1]) and the whole grid_cap is
// launched; otherwise the host splits the blocks.
int launch_batch(const Scratch& sc, unsigned* status, bool map_mode, const ItemDesc* items,
                 int n_items, int max_iter, double eps, int threads, int grid_cap,
                 const int64_t* n_dev, int* first_dev, bool cand_start, cudaStream_t s,
                 const int* weight = nullptr) {
    BatchParams P;
    P.sc = sc;
    P.status = status;
    P.n_items = n_items;
    P.max_iter = max_iter;
    P.eps = eps;
    P.n_dev = n_dev;
    P.first_dev = n_dev ? first_dev : nullptr;
    P.weight = n_dev ? weight : nullptr;
    P.cand_start = cand_start ? 1 : 0;
    int64_t want[kMaxBatch];
    for (int i = 0; i < n_items; ++i) {
        P.item[i] = items[i];
        want[i] = group_want(items[i].n, items[i].K, threads);
    }
    const int grid = n_dev ? grid_cap : split_groups(want, n_items, grid_cap, P.first_blk);
    void* args[] = {&P};
    // Clear the barrier counters and the accumulators of the slots used.  The
    // items of a launch use consecutive slots, so one memset per array does.
    int lo = items[0].slot, hi = items[0].slot;
    for (int i = 1; i < n_items; ++i) {
        lo = std::min(lo, items[i].slot);
        hi = std::max(hi, items[i].slot);
    }
    const size_t nsl = (size_t)(hi - lo + 1), s5 = (size_t)5 * sc.max_K;
    static_assert(sizeof(Ctrl) % 4 == 0, "control blocks are cleared as 32-bit words");
    ClearRanges Z;
    Z.p[0] = reinterpret_cast<unsigned*>(sc.ctrl + lo);
    Z.n[0] = sizeof(Ctrl) / 4 * nsl;
    Z.p[1] = sc.sums + (size_t)lo * 2 * kCopies * s5;
    Z.n[1] = 2 * kCopies * s5 * nsl;
    Z.p[2] = reinterpret_cast<unsigned*>(sc.sums64 + (size_t)lo * 2 * kCopies * 4);
    Z.n[2] = 2 * (2 * kCopies * 4 * nsl);
    cudaError_t e = cudaSuccess;
    if (n_dev) {
        // one kernel clears and plans (fewer nodes in a captured graph)
        k_plan<<<std::min<int>(64, (int)((Z.n[1] + 255) / 256) + 1), 256, 0, s>>>(
            P, threads, grid, first_dev, Z);
        e = cudaGetLastError();
    } else {
        for (int r = 0; r < 3 && e == cudaSuccess; ++r)
            e = cudaMemsetAsync(Z.p[r], 0, sizeof(unsigned) * Z.n[r], s);
    }
    void* fn = sortmeans_fn(map_mode, threads, sc.label_bytes);
    if (!fn) return fail(WSM_E_INVAL, "16-bit memberships need 512 threads per block");
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel(fn, grid, threads, args,
                                        sortmeans_smem(sc.max_K, threads, map_mode),
                                        s);
    if (e != cudaSuccess) return cuda_fail(e, "sort-means launch");
    return WSM_OK;
}

int launch_sortmeans(wsm_handle* h, bool map_mode, const uint32_t* colors, const uint32_t* counts,
                     int64_t n, int K, float* centers, void* labels, int max_iter, double eps,
                     cudaStream_t s) {
    ItemDesc it;
    it.colors = colors;
    it.counts = counts;
    it.labels = labels;
    it.centers = reinterpret_cast<float4*>(centers);
    it.n = n;
    it.K = K;
    it.slot = 0;
    return launch_batch(handle_scratch(h), &h->ctrl->status, map_mode, &it, 1, max_iter, eps,
                        kIterShapes[h->iter_shape].threads, iter_grid(h), nullptr, nullptr,
                        h->cand_start, s);
}

// The final assignment of n_items images (slots slot0, slot0 + 1, ...) in
// one persistent launch in map mode; with sse, each slot's map_sse also gets
// the image's squared-error sum (from the items' counts).
int launch_map_items(wsm_handle* h, const wsm_item* items, int n_items, int slot0,
                     const int64_t* n_dev, bool sse, cudaStream_t s) {
    ItemDesc d[kMaxBatch];
    for (int q = 0; q < n_items; ++q) {
        d[q].colors = items[q].d_colors;
        d[q].counts = sse ? items[q].d_counts : nullptr;
        d[q].labels = items[q].d_labels;
        d[q].centers = reinterpret_cast<float4*>(items[q].d_centers);
        d[q].n = n_dev ? items[q].n_pixels : items[q].n_unique;
        d[q].K = items[q].K;
        d[q].slot = slot0 + q;
    }
    return launch_batch(handle_scratch(h), &h->ctrl->status, true, d, n_items, 1, 0.0,
                        kIterShapes[h->iter_shape].threads, iter_grid(h), n_dev,
                        h->plan + (size_t)(slot0 / kMaxBatch) * (kMaxBatch + 1), false, s);
}

// The iterations of n_items images (item i in slot i), one persistent launch
// per kMaxBatch images; with n_dev the sizes are read on the device.
int iterate_items(wsm_handle* h, const wsm_item* items, int n_items, int max_iter, double eps,
                  const int64_t* n_dev, cudaStream_t s, int64_t* d_n_unique, int* d_iters) {
    for (int i0 = 0; i0 < n_items; i0 += kMaxBatch) {
        const int m = std::min(kMaxBatch, n_items - i0);
        ItemDesc d[kMaxBatch];
        for (int q = 0; q < m; ++q) {
            const wsm_item& it = items[i0 + q];
            d[q].colors = it.d_colors;
            d[q].counts = it.d_counts;
            d[q].labels = it.d_labels;
            d[q].centers = reinterpret_cast<float4*>(it.d_centers);
            d[q].n = n_dev ? it.n_pixels : it.n_unique;   // an upper bound in device mode
            d[q].K = it.K;
            d[q].slot = i0 + q;
            d[q].nu_out = d_n_unique ? d_n_unique + i0 + q : nullptr;
            d[q].iters_out = d_iters ? d_iters + i0 + q : nullptr;
        }
        int rc = launch_batch(handle_scratch(h), &h->ctrl->status, false, d, m, max_iter, eps,
                              kIterShapes[h->iter_shape].threads, iter_grid(h), n_dev,
                              h->plan + (size_t)(i0 / kMaxBatch) * (kMaxBatch + 1),
                              h->cand_start, s, h->slot_weight);
        if (rc != WSM_OK) return rc;
    }
    return WSM_OK;
}

// Checks of one batch item shared by the iterate and map entry points.
int check_item(wsm_handle* h, const wsm_item& it, bool need_pixels, bool need_counts) {
    if (it.K < 1 || it.K > h->max_K) return fail(WSM_E_INVAL, "K out of [1, max_K]");
    if (it.n_unique < 1 || it.n_unique > h->max_unique)
        return fail(WSM_E_INVAL, "n_unique must be in [1, max_unique]");
    if (!it.d_colors || !it.d_centers || !it.d_labels || (need_counts && !it.d_counts))
        return fail(WSM_E_INVAL, "null device pointer");
    if ((uintptr_t)it.d_centers & 15) return fail(WSM_E_INVAL, "centers must be 16-byte aligned");
    if (need_pixels) {
        if (it.pixel_stride != 3 && it.pixel_stride != 4)
            return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
        if (it.n_pixels < 1 || it.n_pixels > h->max_pixels || it.n_unique > it.n_pixels)
            return fail(WSM_E_INVAL, "n_pixels must be in [max(1, n_unique), max_pixels]");
        if (!it.d_rgb || !it.d_index) return fail(WSM_E_INVAL, "null pixel or index pointer");
        if (it.pixel_stride == 4 && ((uintptr_t)it.d_rgb & 3))
            return fail(WSM_E_INVAL, "4-byte pixels must be 4-byte aligned");
    }
    return WSM_OK;
}

}  // namespace wsm

using namespace wsm;

extern "C" int wsm_iterate(wsm_handle* h, const uint32_t* d_colors, const uint32_t* d_counts,
                           int64_t n_unique, int K, float* d_centers, void* d_labels,
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
        cudaError_t e = cudaMemcpyAsync(&h->host_ctrl->iters_done, &h->slot_ctrl[0].iters_done,
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

extern "C" int wsm_iterate_batch(wsm_handle* h, const wsm_item* items, int n_items, int max_iter,
                                 double eps, int* iters_done, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (n_items < 0 || (n_items > 0 && !items)) return fail(WSM_E_INVAL, "bad item list");
    if (n_items > h->slots)
        return fail(WSM_E_INVAL, "more items than reserved slots (wsm_reserve_batch)");
    if (max_iter < 0 || max_iter > kMaxTrace)
        return fail(WSM_E_INVAL, "max_iter must be in [0, 4096]");
    for (int i = 0; i < n_items; ++i) {
        rc = check_item(h, items[i], false, true);
        if (rc != WSM_OK) return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rc = iterate_items(h, items, n_items, max_iter, eps, nullptr, s);
    if (rc != WSM_OK) return rc;
    if (iters_done && n_items > 0) {
        rc = read_status(h, s);
        if (rc != WSM_OK) return rc;
        for (int i = 0; i < n_items; ++i) {
            cudaError_t e = cudaMemcpy(&iters_done[i], &h->slot_ctrl[i].iters_done, sizeof(int),
                                       cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "iteration count copy");
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
    e = cudaMemcpy(&c, &h->slot_ctrl[0], sizeof(Ctrl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats copy");
    if (evaluated) *evaluated = (int64_t)c.evaluated;
    if (S || W) {
        if (c.iters_done < 1) return fail(WSM_E_STATE, "no completed iteration");
        std::vector<unsigned long long> buf((size_t)4 * K);
        e = cudaMemcpy(buf.data(), h->acc, sizeof(unsigned long long) * 4 * K,
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
constexpr int kStaticThreads = 512;
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
constexpr size_t kStaticOffGrid = kStaticOffTrace + kStaticTraceBytes;
constexpr size_t kStaticOffCtrl = kStaticOffGrid + kGridCells;
constexpr size_t kStaticOffStatus = kStaticOffCtrl + 256;       // outside the cleared Ctrl
constexpr size_t kStaticBytes = kStaticOffStatus + 256;         // about 1.2 MiB in total
static_assert(kStaticOffSums % 16 == 0 && kStaticOffCtrl % 16 == 0, "scratch alignment");
static_assert(sizeof(Ctrl) <= kStaticOffStatus - kStaticOffCtrl,
              "the control block must fit the room kept for it");

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
            e = raise_smem_limit((const void*)k_sortmeans<false, kStaticThreads, uint8_t>,
                                 sortmeans_smem(kStaticMaxK, kStaticThreads, false));
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &occ, k_sortmeans<false, kStaticThreads, uint8_t>, kStaticThreads,
                sortmeans_smem(kStaticMaxK, kStaticThreads, false));
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
    // The status word lies outside the control block that every launch
    // clears: a failure of a call that did not synchronise stays recorded
    // until a later call reads it (and only then clears it).
    unsigned* status = reinterpret_cast<unsigned*>(base + kStaticOffStatus);
    Scratch sc;
    sc.tab = reinterpret_cast<float4*>(base);
    sc.tab_nb = base + kStaticOffNb;
    sc.sums = reinterpret_cast<unsigned*>(base + kStaticOffSums);
    sc.sums64 = reinterpret_cast<unsigned long long*>(base + kStaticOffSums64);
    sc.acc = reinterpret_cast<unsigned long long*>(base + kStaticOffAcc);
    sc.trace = trace;
    sc.lut = nullptr;
    sc.grid = base + kStaticOffGrid;
    sc.ctrl = ctrl;
    sc.max_K = kStaticMaxK;
    sc.label_bytes = 1;
    ItemDesc it;
    it.colors = d_colors;
    it.counts = d_counts;
    it.labels = d_labels;
    it.centers = reinterpret_cast<float4*>(d_centers);
    it.n = n_unique;
    it.K = K;
    it.slot = 0;
    rc = launch_batch(sc, status, false, &it, 1, max_iter, eps, kStaticThreads, st->grid,
                      nullptr, nullptr, true, s);
    if (rc != WSM_OK) return rc;
    if (iters_done || sse_trace) {
        Ctrl host;
        unsigned st_bits = 0;
        e = cudaMemcpyAsync(&host, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&st_bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "wsm_iterate_noalloc result copy");
        if (st_bits) {
            e = cudaMemsetAsync(status, 0, sizeof(unsigned), s);
            if (e != cudaSuccess) return cuda_fail(e, "wsm_iterate_noalloc status clear");
        }
        if (st_bits & ST_TIMEOUT)
            return fail(WSM_E_TIMEOUT, "a device-side grid barrier timed out");
        if (st_bits & ST_BAD_LABEL) return fail(WSM_E_INVAL, "a membership was >= K");
        if (iters_done) *iters_done = host.iters_done;
        if (sse_trace && host.iters_done > 0) {
            e = cudaMemcpyAsync(sse_trace, trace,
                                sizeof(double) * std::min(host.iters_done, max_iter),
                                cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "wsm_iterate_noalloc trace copy");
        }
    }
    return WSM_OK;
}
