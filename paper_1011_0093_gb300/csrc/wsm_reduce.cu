// wsm_reduce.cu -- unique colors and their frequencies (Sec. 2, data
// sampling and sample weighting).
//
// The paper collects the distinct colors with a chained hash table.  Here the
// counts end up in a 2^24-bin uint32 histogram (one bin per 24-bit color)
// with a 2^24-bit occupancy map beside it.  A two-kernel prefix scan over the
// occupancy map then writes (color, count) for every set bit, in ascending
// color order, and clears the bins and bits it read, so the scratch is zero
// again for the next image without a 64 MiB memset.
//
// Two ways fill the histogram, with identical results (every count is an
// exact integer sum):
//   direct    every pixel adds one to its bin with a global atomic (lanes of a
//             warp holding the same color add together), the first pixel of a
//             color sets its bit.  Few launches; the cost is one L2 atomic on
//             a random bin per pixel, so it suits small images.
//   bucketed  (large images) the pixels are first grouped by bucket, the top
//             10 bits of their key: one pass counts the pixels of each bucket,
//             a plan kernel turns the counts into bucket offsets and a work
//             list, a second pass writes each pixel's low 14 bits into its
//             bucket's run (staged in shared memory so that every run is
//             written contiguously), and then each work item -- one bucket, or
//             a chunk of a large one -- counts its keys in a 2^14-bin
//             shared-memory histogram and flushes the nonzero bins into the
//             global histogram and occupancy map (plain stores when the bucket
//             is one item, atomics when several items share it).  Global
//             atomics drop from one per pixel to about one per distinct color.
#include <algorithm>

#include "wsm_internal.cuh"
#include "wsm_pixels.cuh"

namespace wsm {

// The images of one reduction launch: image i uses reduction slot i (its own
// histogram, occupancy map and block totals), owns the histogram blocks
// [first_blk[i], first_blk[i+1]) and the compaction blocks
// [i * kScanBlocks, (i+1) * kScanBlocks).
struct ReduceItems {
    int n_items;
    int first_blk[kReduceSlots + 1];
    const uint8_t* rgb[kReduceSlots];
    int64_t n[kReduceSlots];
    int stride[kReduceSlots];
    uint32_t* colors[kReduceSlots];
    uint32_t* counts[kReduceSlots];
    int64_t capacity[kReduceSlots];
    int64_t* n_out[kReduceSlots];    // N' (device), always written
    int64_t* n_user[kReduceSlots];   // N' (device), a caller's copy, may be null
    uint32_t* hist;                  // slot i at hist + i * 2^24
    uint32_t* bitmap;                // slot i at bitmap + i * 2^19
    uint32_t* blk_total;             // slot i at blk_total + i * kScanBlocks
    unsigned* status;
    // bucketed path
    uint32_t* bkt_count;             // slot i at bkt_count + i * kBuckets
    uint32_t* bkt_cursor;            // slot i at bkt_cursor + i * kBuckets
    uint16_t* keys16;                // slot i at keys16 + i * keys_stride
    uint4* work;                     // slot i at work + i * work_stride
    int* n_work;                     // [slot]
    int64_t keys_stride;
    int64_t work_stride;
};

// Histogram with warp aggregation: lanes holding the same color elect one
// leader, which adds the group's size with a single atomic.
__global__ void __launch_bounds__(256) k_hist24(const __grid_constant__ ReduceItems R) {
    const int i = item_of_block(R.first_blk, R.n_items, blockIdx.x);
    const int g = blockIdx.x - R.first_blk[i], G = R.first_blk[i + 1] - R.first_blk[i];
    const uint8_t* rgb = R.rgb[i];
    const int64_t n = R.n[i];
    const int stride = R.stride[i];
    uint32_t* hist = R.hist + (size_t)i * kHistBins;
    uint32_t* bitmap = R.bitmap + (size_t)i * kMapWords;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)g * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = ((int64_t)G * blockDim.x) >> 5;
    for (int64_t base = warp * 32; base < n; base += warps * 32) {
        int64_t p = base + lane;
        bool valid = p < n;
        uint32_t key = valid ? pixel_key(rgb, p, stride) : 0xFFFFFFFFu;
        unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
        if (valid && lane == __ffs(peers) - 1) {
            unsigned old = atomicAdd(hist + key, (unsigned)__popc(peers));
            if (old == 0) atomicOr(bitmap + (key >> 5), 1u << (key & 31));
        }
    }
}

// ---- bucketed path -------------------------------------------------------------

// The pixels of block g (of G) of image i, 16 consecutive pixels per thread
// and step: calls f(key) for each (the vector path for 16-byte aligned
// images, one pixel at a time for the rest and the last n % 16 pixels).
template <typename F>
__device__ __forceinline__ void for_pixels(const uint8_t* __restrict__ rgb, int64_t n, int stride,
                                           int64_t t, int64_t nt, F&& f) {
    int64_t done = 0;
    if (vector_ok(rgb, nullptr)) {
        const int64_t ng = n / kGroup;
        for (int64_t gr = t; gr < ng; gr += nt) {
            uint32_t key[kGroup];
            pixel_keys16(rgb, gr, stride, key);
#pragma unroll
            for (int j = 0; j < kGroup; ++j) f(key[j]);
        }
        done = ng * kGroup;
    }
    for (int64_t p = done + t; p < n; p += nt) f(pixel_key(rgb, p, stride));
}

// Shared-memory slot of bucket b (= R << 2 | G >> 6): R in the low bits, so
// that the buckets of nearby colors (a noisy region spans a few dozen
// consecutive R values) fall in different banks.
__device__ __forceinline__ unsigned bslot(unsigned b) { return ((b & 3u) << 8) | (b >> 2); }

// Pass A: the number of pixels of each bucket.  A thread adds a run of equal
// buckets among its consecutive pixels with one shared-memory atomic; each
// block adds its nonzero counts to the image's.
__global__ void __launch_bounds__(256) k_bkt_count(const __grid_constant__ ReduceItems R) {
    __shared__ unsigned s_cnt[kBuckets];
    const int i = item_of_block(R.first_blk, R.n_items, blockIdx.x);
    const int g = blockIdx.x - R.first_blk[i], G = R.first_blk[i + 1] - R.first_blk[i];
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) s_cnt[b] = 0u;
    __syncthreads();
    unsigned run_b = 0xFFFFFFFFu, run_n = 0;
    for_pixels(R.rgb[i], R.n[i], R.stride[i], (int64_t)g * blockDim.x + threadIdx.x,
               (int64_t)G * blockDim.x, [&](uint32_t key) {
                   const unsigned b = key >> (24 - kBktBits);
                   if (b != run_b) {
                       if (run_n) atomicAdd(&s_cnt[bslot(run_b)], run_n);
                       run_b = b;
                       run_n = 0;
                   }
                   ++run_n;
               });
    if (run_n) atomicAdd(&s_cnt[bslot(run_b)], run_n);
    __syncthreads();
    uint32_t* cnt = R.bkt_count + (size_t)i * kBuckets;
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) {
        const unsigned c = s_cnt[bslot(b)];
        if (c) atomicAdd(cnt + b, c);
    }
}

// Block-wide exclusive scan of one value per thread (kBuckets threads);
// returns the thread's exclusive prefix and writes the total to *total.
__device__ __forceinline__ unsigned scan_buckets(unsigned v, unsigned* s_w, unsigned* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned w = lane < kBuckets / 32 ? s_w[lane] : 0u;
        unsigned wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < kBuckets / 32) s_w[lane] = wi - w;     // exclusive per warp
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    const unsigned r = s_w[wid] + incl - v;
    __syncthreads();
    return r;
}

// Plan (one block of kBuckets threads per image): bucket b's keys go to
// [off_b, off_b + n_b) of the image's key array (the cursor starts at off_b);
// its work items are chunks of at most kBktChunk keys, flagged shared when
// there are several.  The bucket counts are cleared for the next call.
__global__ void __launch_bounds__(kBuckets) k_bkt_plan(const __grid_constant__ ReduceItems R) {
    __shared__ unsigned s_w[kBuckets / 32];
    __shared__ unsigned s_off[kBuckets + 1];      // first key of each bucket, then N
    __shared__ unsigned s_item0[kBuckets + 1];    // first work item of each bucket, then all
    __shared__ unsigned s_total;
    const int i = blockIdx.x, b = threadIdx.x;
    uint32_t* cnt = R.bkt_count + (size_t)i * kBuckets;
    const unsigned nb = cnt[b];
    cnt[b] = 0u;
    const unsigned off = scan_buckets(nb, s_w, &s_total);
    const unsigned n_all = s_total;
    s_off[b] = off;
    R.bkt_cursor[(size_t)i * kBuckets + b] = off;
    const unsigned first = scan_buckets((nb + kBktChunk - 1) / kBktChunk, s_w, &s_total);
    s_item0[b] = first;
    if (b == 0) {
        s_off[kBuckets] = n_all;
        s_item0[kBuckets] = s_total;
    }
    __syncthreads();
    const unsigned n_items = s_item0[kBuckets];
    uint4* work = R.work + (size_t)i * R.work_stride;
    for (unsigned t = threadIdx.x; t < n_items; t += blockDim.x) {
        // the bucket of item t: the last q with s_item0[q] <= t (a nonempty one)
        int lo = 0, hi = kBuckets - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_item0[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const unsigned c = t - s_item0[lo];
        const unsigned nq = s_item0[lo + 1] - s_item0[lo];
        const unsigned start = s_off[lo] + c * kBktChunk;
        const unsigned len = min((unsigned)kBktChunk, s_off[lo + 1] - start);
        work[t] = make_uint4((unsigned)lo, start, len, nq > 1 ? 1u : 0u);
    }
    if (threadIdx.x == 0) R.n_work[i] = (int)n_items;
}

// Pass B: each block takes tiles of kScatterPix pixels (16 consecutive pixels
// per thread); every pixel gets its rank among the tile's pixels of its
// bucket (a thread's run of equal buckets takes one shared-memory atomic),
// the tile's pixels are placed in shared memory in bucket order, each
// nonempty bucket of the tile claims a range of its run in the image's key
// array with one global atomic, and the threads write the staged keys' low
// 14 bits to consecutive positions of those ranges.  The per-bucket tables
// are indexed by bslot.
constexpr int kScatterThreads = 512;    // tiles of 8192 pixels: 0.409 -> 0.400 ms for
                                          // 4 x 4096^2 against 4096 (16384: 0.411)
constexpr int kScatterPerSM = 1024 / kScatterThreads;      // resident blocks per SM
constexpr int kScatterPix = kScatterThreads * kGroup;      // pixels per tile
constexpr int kScatterPer = kBuckets / kScatterThreads;    // buckets per thread in the scan
static_assert(kBuckets % kScatterThreads == 0, "the tile scan splits the buckets evenly");

__global__ void __launch_bounds__(kScatterThreads, kScatterPerSM)
    k_bkt_scatter(const __grid_constant__ ReduceItems R) {
    __shared__ unsigned s_cnt[kBuckets];      // pixels of each bucket in the tile
    __shared__ unsigned s_base[kBuckets];     // their offset within the tile
    __shared__ unsigned s_gpos[kBuckets];     // their first position in the key array
    __shared__ unsigned s_w[kScatterThreads / 32];
    __shared__ unsigned s_total;
    extern __shared__ uint32_t s_key[];       // [kScatterPix] the tile's keys in bucket order
    const int i = item_of_block(R.first_blk, R.n_items, blockIdx.x);
    const int g = blockIdx.x - R.first_blk[i], G = R.first_blk[i + 1] - R.first_blk[i];
    const uint8_t* rgb = R.rgb[i];
    const int64_t n = R.n[i];
    const int stride = R.stride[i];
    const bool vec = vector_ok(rgb, nullptr);
    uint32_t* cursor = R.bkt_cursor + (size_t)i * kBuckets;
    uint16_t* keys = R.keys16 + (size_t)i * R.keys_stride;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int b = tid; b < kBuckets; b += kScatterThreads) s_cnt[b] = 0u;
    __syncthreads();
    for (int64_t t0 = (int64_t)g * kScatterPix; t0 < n; t0 += (int64_t)G * kScatterPix) {
        const int64_t p0 = t0 + (int64_t)tid * kGroup;       // this thread's 16 pixels
        uint32_t key[kGroup];
        int m = 0;                                            // how many are in the image
        if (vec && p0 + kGroup <= n) {
            pixel_keys16(rgb, p0 / kGroup, stride, key);
            m = kGroup;
        } else {
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                key[j] = p0 + j < n ? pixel_key(rgb, p0 + j, stride) : 0u;
                if (p0 + j < n) m = j + 1;
            }
        }
        // rank of each pixel among the tile's pixels of its bucket: walking
        // back, each run of equal buckets takes one atomic at its last pixel
        unsigned rank[kGroup];
        {
            // position of each pixel in its run, 4 bits per pixel
            unsigned long long pos = 0;
            unsigned p = 0;
#pragma unroll
            for (int j = 1; j < kGroup; ++j) {
                p = (key[j] >> (24 - kBktBits)) == (key[j - 1] >> (24 - kBktBits)) ? p + 1u : 0u;
                pos |= (unsigned long long)p << (4 * j);
            }
            unsigned base = 0;
#pragma unroll
            for (int j = kGroup - 1; j >= 0; --j) {
                if (j < m) {
                    const unsigned b = key[j] >> (24 - kBktBits);
                    const unsigned pj = (unsigned)(pos >> (4 * j)) & 15u;
                    const bool last = j == m - 1 ||
                                      (j + 1 < kGroup && (key[j + 1] >> (24 - kBktBits)) != b);
                    if (last) base = atomicAdd(&s_cnt[bslot(b)], pj + 1u);
                    rank[j] = base + pj;
                }
            }
        }
        __syncthreads();
        // tile offsets of the buckets in bucket order: thread t scans buckets
        // kScatterPer t .. kScatterPer t + kScatterPer - 1
        unsigned c[kScatterPer], sum = 0;
#pragma unroll
        for (int q = 0; q < kScatterPer; ++q) {
            c[q] = s_cnt[bslot(kScatterPer * tid + q)];
            sum += c[q];
        }
        unsigned incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            constexpr int kW = kScatterThreads / 32;
            const unsigned w = lane < kW ? s_w[lane] : 0u;
            unsigned wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned u = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= o) wi += u;
            }
            if (lane < kW) s_w[lane] = wi - w;
            if (lane == 31) s_total = wi;
        }
        __syncthreads();
        unsigned ex = s_w[wid] + incl - sum;
#pragma unroll
        for (int q = 0; q < kScatterPer; ++q) {
            const unsigned b = kScatterPer * tid + q, sl = bslot(b);
            s_base[sl] = ex;
            s_gpos[sl] = c[q] ? atomicAdd(cursor + b, c[q]) : 0u;
            ex += c[q];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kGroup; ++j)
            if (j < m) s_key[s_base[bslot(key[j] >> (24 - kBktBits))] + rank[j]] = key[j];
        __syncthreads();
        const unsigned tile_n = s_total;
        for (unsigned q = tid; q < tile_n; q += kScatterThreads) {
            const uint32_t k = s_key[q];
            const unsigned sl = bslot(k >> (24 - kBktBits));
            keys[s_gpos[sl] + (q - s_base[sl])] = (uint16_t)(k & (kBktBins - 1));
        }
#pragma unroll
        for (int q = 0; q < kScatterPer; ++q) s_cnt[bslot(kScatterPer * tid + q)] = 0u;
        __syncthreads();
    }
}

// Pass C: work item (bucket b, start, length, shared) of image i counts its
// keys in a 2^14-bin shared-memory histogram, then writes the nonzero bins
// into the image's histogram and occupancy map: plain stores when it is the
// bucket's only item (no other item touches those bins and words), atomics
// when the bucket is shared.  The blocks of the launch take the items of all
// images in turn.
constexpr int kBktHistThreads = 512;

__global__ void __launch_bounds__(kBktHistThreads, 3)
    k_bkt_hist(const __grid_constant__ ReduceItems R, int max_items) {
    extern __shared__ unsigned s_h[];                      // [kBktBins]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t total = (int64_t)R.n_items * max_items;
    for (int64_t v = blockIdx.x; v < total; v += gridDim.x) {
        const int i = (int)(v / max_items), t = (int)(v % max_items);
        if (t >= R.n_work[i]) continue;                    // uniform over the block
        const uint4 w = R.work[(size_t)i * R.work_stride + t];
        const unsigned b = w.x, start = w.y, len = w.z;
        const bool shared = w.w != 0u;
        const uint16_t* keys = R.keys16 + (size_t)i * R.keys_stride;
        // the item's keys: a ragged head up to an 8-key boundary, 16-byte
        // loads of 8 keys (at most kVec per thread, all issued before the
        // histogram is cleared), a ragged tail
        constexpr int kVec = kBktChunk / 8 / kBktHistThreads;
        const unsigned a0 = min(len, (8u - (start & 7u)) & 7u);
        const unsigned nv = (len - a0) / 8u;
        const uint4* kv = reinterpret_cast<const uint4*>(keys + start + a0);
        uint4 u[kVec];
#pragma unroll
        for (int r = 0; r < kVec; ++r) {
            const unsigned q = tid + r * kBktHistThreads;
            u[r] = q < nv ? __ldg(kv + q) : make_uint4(0u, 0u, 0u, 0u);
        }
        const unsigned head = tid < (int)a0 ? keys[start + tid] : 0u;
        const unsigned tq = a0 + nv * 8u + tid;
        const unsigned tail = tq < len ? keys[start + tq] : 0u;
        for (int q = tid; q < kBktBins / 4; q += kBktHistThreads)
            reinterpret_cast<uint4*>(s_h)[q] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        if (tid < (int)a0) atomicAdd(&s_h[head], 1u);
        if (tq < len) atomicAdd(&s_h[tail], 1u);
#pragma unroll
        for (int r = 0; r < kVec; ++r) {
            if (tid + r * kBktHistThreads < nv) {
                const unsigned ws[4] = {u[r].x, u[r].y, u[r].z, u[r].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    atomicAdd(&s_h[ws[e] & 0xFFFFu], 1u);
                    atomicAdd(&s_h[ws[e] >> 16], 1u);
                }
            }
        }
        __syncthreads();
        uint32_t* hist = R.hist + (size_t)i * kHistBins + (size_t)b * kBktBins;
        uint32_t* bitmap = R.bitmap + (size_t)i * kMapWords + (size_t)b * (kBktBins / 32);
        for (int wd = wid; wd < kBktBins / 32; wd += kBktHistThreads / 32) {
            const unsigned c = s_h[wd * 32 + lane];
            const unsigned m = __ballot_sync(0xFFFFFFFFu, c != 0u);
            if (!m) continue;
            if (shared) {
                if (c) atomicAdd(hist + wd * 32 + lane, c);
                if (lane == 0) atomicOr(bitmap + wd, m);
            } else {
                if (c) hist[wd * 32 + lane] = c;
                if (lane == 0) bitmap[wd] = m;
            }
        }
        __syncthreads();
    }
}

// Pass 1 of the compaction: the number of set bits in each block's 2048 words.
__global__ void __launch_bounds__(kScanThreads)
    k_scan_count(const __grid_constant__ ReduceItems R) {
    const int i = blockIdx.x / kScanBlocks, b = blockIdx.x % kScanBlocks;
    const uint32_t* bitmap = R.bitmap + (size_t)i * kMapWords;
    const uint4 a = reinterpret_cast<const uint4*>(bitmap)[
        ((size_t)b * kScanWordsPerBlock + threadIdx.x * kScanWordsPerThread) / 4];
    unsigned c = __popc(a.x) + __popc(a.y) + __popc(a.z) + __popc(a.w);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    __shared__ unsigned s_w[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += s_w[w];
        R.blk_total[(size_t)i * kScanBlocks + b] = t;
    }
}

// Pass 2: each block finds its output offset from the totals of the blocks
// before it and scans its words into output offsets, listing the nonzero
// words in order (one scan of the packed per-thread counts of set bits and
// of nonzero words); then the warps take the listed words, kEmitBatch in
// flight per warp, one word at a time with lane l handling bit l (so the 32
// bins of a word are read and cleared with one coalesced access), and emit
// (color, count) for every set bit.  Empty words cost nothing past the scan.
// Output order is ascending color order.
__global__ void __launch_bounds__(kScanThreads) k_scan_emit(const __grid_constant__ ReduceItems R) {
    __shared__ uint32_t s_word[kScanWordsPerBlock];     // the block's nonzero words, in order
    __shared__ uint32_t s_off[kScanWordsPerBlock];      // output offset of each (within the block)
    __shared__ uint16_t s_idx[kScanWordsPerBlock];      // word index within the block
    __shared__ unsigned s_w[kScanThreads / 32];
    __shared__ unsigned long long s_base;
    const int item = blockIdx.x / kScanBlocks, b = blockIdx.x % kScanBlocks;
    uint32_t* bitmap = R.bitmap + (size_t)item * kMapWords;
    uint32_t* hist = R.hist + (size_t)item * kHistBins;
    const uint32_t* blk_total = R.blk_total + (size_t)item * kScanBlocks;
    uint32_t* colors = R.colors[item];
    uint32_t* counts = R.counts[item];
    const int64_t capacity = R.capacity[item];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // offset of this block: sum of the totals of blocks [0, b)
    unsigned long long before = 0;
    for (int q = tid; q < b; q += kScanThreads) before += blk_total[q];
    for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xFFFFFFFFu, before, o);
    if (tid == 0) s_base = 0;
    __syncthreads();
    if (lane == 0 && before) atomicAdd(&s_base, before);
    const size_t w0 = (size_t)b * kScanWordsPerBlock;
    uint4* wv = reinterpret_cast<uint4*>(bitmap + w0) + tid;
    const uint4 a = wv[0];
    const uint32_t words[4] = {a.x, a.y, a.z, a.w};
    // packed per-thread counts: nonzero words << 20 | set bits (block totals fit:
    // at most 2048 words and 65536 bits)
    unsigned mine = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) mine += (words[q] ? (1u << 20) : 0u) + __popc(words[q]);
    unsigned incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    unsigned warp_off = 0;
    for (int q = 0; q < wid; ++q) warp_off += s_w[q];
    unsigned off = warp_off + (incl - mine);                 // packed exclusive prefix
    unsigned total = 0;
    for (int q = 0; q < kScanThreads / 32; ++q) total += s_w[q];
    unsigned slot = off >> 20, bits = off & 0xFFFFFu;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (words[q]) {
            s_word[slot] = words[q];
            s_off[slot] = bits;
            s_idx[slot] = (uint16_t)(4 * tid + q);
            ++slot;
            bits += __popc(words[q]);
        }
    }
    if (a.x | a.y | a.z | a.w) wv[0] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const int64_t base = (int64_t)s_base;
    const int nnz = (int)(total >> 20);
    const unsigned below = (1u << lane) - 1u;
    constexpr int kEmitBatch = 16;
    constexpr int kWarps = kScanThreads / 32;
    for (int k0 = wid * kEmitBatch; k0 < nnz; k0 += kWarps * kEmitBatch) {
        uint32_t wd[kEmitBatch], cnt[kEmitBatch];
#pragma unroll
        for (int u = 0; u < kEmitBatch; ++u) {
            wd[u] = k0 + u < nnz ? s_word[k0 + u] : 0u;
            cnt[u] = 0;
            if ((wd[u] >> lane) & 1u) cnt[u] = hist[((w0 + s_idx[k0 + u]) << 5) | lane];
        }
#pragma unroll
        for (int u = 0; u < kEmitBatch; ++u) {
            if ((wd[u] >> lane) & 1u) {
                const uint32_t key = (uint32_t)((w0 + s_idx[k0 + u]) << 5) | (uint32_t)lane;
                const int64_t pos = base + s_off[k0 + u] + __popc(wd[u] & below);
                hist[key] = 0;
                if (pos < capacity) {
                    colors[pos] = key;
                    counts[pos] = cnt[u];
                }
            }
        }
    }
    if (b == kScanBlocks - 1 && tid == 0) {
        const int64_t all = base + (total & 0xFFFFFu);      // N': the last block ends at it
        *R.n_out[item] = all;
        if (R.n_user[item]) *R.n_user[item] = all;
        if (all > capacity) atomicOr(R.status, ST_CAPACITY);
    }
}

// The bucketed path is used for launches of at least kBktMinPixels pixels in
// all and kBktMinMeanPixels per image on average: below that the direct
// histogram's atomics stay in L2 and it is faster (measured on one GB300:
// one 2048^2 image 0.067 vs 0.091 ms, one 2896^2 image equal, one 4096^2
// image 0.15 vs 0.14 ms, 4 x 4096^2 0.58 vs 0.41 ms).
constexpr int64_t kBktMinPixels = 1 << 24;
constexpr int64_t kBktMinMeanPixels = 1 << 21;

// Blocks of a pass over the pixels: at most `budget` blocks in all, split in
// proportion to the images' pixels, at most `want(n)` for an image of n.
template <typename Want>
static void split_pixels(ReduceItems& R, int64_t budget, Want want) {
    int64_t total = 0;
    for (int i = 0; i < R.n_items; ++i) total += R.n[i];
    R.first_blk[0] = 0;
    for (int i = 0; i < R.n_items; ++i) {
        const int64_t share = std::max<int64_t>(1, budget * R.n[i] / std::max<int64_t>(total, 1));
        R.first_blk[i + 1] = R.first_blk[i] + (int)(R.n[i] > 0 ? std::min(want(R.n[i]), share) : 0);
    }
}

// Launch the reduction kernels for R.n_items images whose per-image fields
// are filled in; sets the scratch pointers and the blocks of each pass.
static int launch_reduce(wsm_handle* h, ReduceItems& R, cudaStream_t s) {
    R.hist = h->hist;
    R.bitmap = h->bitmap;
    R.blk_total = h->blk_total;
    R.status = &h->ctrl->status;
    R.bkt_count = h->bkt_count;
    R.bkt_cursor = h->bkt_cursor;
    R.keys16 = h->keys16;
    R.work = h->bkt_work;
    R.n_work = h->bkt_nwork;
    R.keys_stride = (int64_t)keys_stride(h);
    R.work_stride = bkt_max_work(h->max_pixels);
    int64_t total = 0, nmax = 0;
    for (int i = 0; i < R.n_items; ++i) {
        total += R.n[i];
        nmax = std::max(nmax, R.n[i]);
    }
    const bool bucketed = h->reduce_path == 2 ||
                          (h->reduce_path == 0 && total >= kBktMinPixels &&
                           total >= kBktMinMeanPixels * R.n_items);
    if (bucketed && R.n_items > 0) {
        static_assert(kBktBins * sizeof(unsigned) <= 64 * 1024, "bucket histogram size");
        cudaError_t e = raise_smem_limit((const void*)k_bkt_hist, kBktBins * sizeof(unsigned));
        if (e != cudaSuccess) return cuda_fail(e, "bucket histogram set-up");
        // counting pass: at most 8 blocks of 256 per SM in all, 16 pixels a thread
        split_pixels(R, (int64_t)h->sms * 8, [](int64_t n) { return (n + 4095) / 4096; });
        if (R.first_blk[R.n_items] > 0) k_bkt_count<<<R.first_blk[R.n_items], 256, 0, s>>>(R);
        k_bkt_plan<<<R.n_items, kBuckets, 0, s>>>(R);
        // scatter pass: the resident blocks of every SM at most, tiles of kScatterPix pixels
        e = raise_smem_limit((const void*)k_bkt_scatter, kScatterPix * sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_fail(e, "scatter set-up");
        split_pixels(R, (int64_t)h->sms * kScatterPerSM,
                     [](int64_t n) { return (n + kScatterPix - 1) / kScatterPix; });
        if (R.first_blk[R.n_items] > 0)
            k_bkt_scatter<<<R.first_blk[R.n_items], kScatterThreads,
                            kScatterPix * sizeof(uint32_t), s>>>(R);
        k_bkt_hist<<<h->sms * 3, kBktHistThreads, kBktBins * sizeof(unsigned), s>>>(
            R, (int)bkt_max_work(nmax));
    } else {
        // at most 8 blocks of 256 per SM in all, one pixel a thread and step
        split_pixels(R, (int64_t)h->sms * 8, [](int64_t n) { return (n + 255) / 256; });
        if (R.first_blk[R.n_items] > 0) k_hist24<<<R.first_blk[R.n_items], 256, 0, s>>>(R);
    }
    k_scan_count<<<kScanBlocks * R.n_items, kScanThreads, 0, s>>>(R);
    k_scan_emit<<<kScanBlocks * R.n_items, kScanThreads, 0, s>>>(R);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "reduce launch");
    return WSM_OK;
}

// Unique colors of n_items images (item i's N' to batch_nu[i]), one launch of
// each reduction kernel per h->rslots images; colors and counts of item i
// have room for its n_pixels entries.
int reduce_items(wsm_handle* h, const wsm_item* items, int n_items, cudaStream_t s) {
    for (int i0 = 0; i0 < n_items; i0 += h->rslots) {
        ReduceItems R;
        R.n_items = std::min(h->rslots, n_items - i0);
        for (int q = 0; q < R.n_items; ++q) {
            const wsm_item& it = items[i0 + q];
            R.rgb[q] = it.d_rgb;
            R.n[q] = it.n_pixels;
            R.stride[q] = it.pixel_stride;
            R.colors[q] = it.d_colors;
            R.counts[q] = it.d_counts;
            R.capacity[q] = it.n_pixels;
            R.n_out[q] = h->batch_nu + i0 + q;
            R.n_user[q] = nullptr;
        }
        int rc = launch_reduce(h, R, s);
        if (rc != WSM_OK) return rc;
    }
    return WSM_OK;
}

// Checks of the pixel fields of a batch item (reduction, mapping, distortion).
int check_pixels(wsm_handle* h, const wsm_item& it) {
    if (it.pixel_stride != 3 && it.pixel_stride != 4)
        return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
    if (it.n_pixels < 1 || it.n_pixels > h->max_pixels)
        return fail(WSM_E_INVAL, "n_pixels must be in [1, max_pixels]");
    if (!it.d_rgb) return fail(WSM_E_INVAL, "null pixel pointer");
    if (it.pixel_stride == 4 && ((uintptr_t)it.d_rgb & 3))
        return fail(WSM_E_INVAL, "4-byte pixels must be 4-byte aligned");
    return WSM_OK;
}

}  // namespace wsm

using namespace wsm;

extern "C" int wsm_reduce(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels, int pixel_stride,
                          uint32_t* d_colors, uint32_t* d_counts, int64_t capacity,
                          int64_t* d_n_unique, int64_t* n_unique, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (pixel_stride != 3 && pixel_stride != 4)
        return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
    if (n_pixels < 0 || n_pixels > h->max_pixels)
        return fail(WSM_E_INVAL, "n_pixels must be in [0, max_pixels]");
    if (capacity < 0) return fail(WSM_E_INVAL, "negative capacity");
    if (n_pixels > 0 && !d_rgb) return fail(WSM_E_INVAL, "null pixel pointer");
    if (capacity > 0 && (!d_colors || !d_counts)) return fail(WSM_E_INVAL, "null output pointer");
    if (pixel_stride == 4 && ((uintptr_t)d_rgb & 3))
        return fail(WSM_E_INVAL, "4-byte pixels must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    ReduceItems R;
    R.n_items = 1;
    R.rgb[0] = d_rgb;
    R.n[0] = n_pixels;
    R.stride[0] = pixel_stride;
    R.colors[0] = d_colors;
    R.counts[0] = d_counts;
    R.capacity[0] = capacity;
    R.n_out[0] = &h->ctrl->n_unique;
    R.n_user[0] = d_n_unique;
    rc = launch_reduce(h, R, s);
    if (rc != WSM_OK) return rc;
    cudaError_t e;
    if (n_unique) {
        e = cudaMemcpyAsync(&h->host_ctrl->n_unique, &h->ctrl->n_unique, sizeof(int64_t),
                            cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "n_unique copy");
        rc = read_status(h, s);
        *n_unique = h->host_ctrl->n_unique;
        if (rc != WSM_OK) return rc;
    }
    return WSM_OK;
}

extern "C" int wsm_reduce_batch(wsm_handle* h, wsm_item* items, int n_items, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (n_items < 0 || (n_items > 0 && !items)) return fail(WSM_E_INVAL, "bad item list");
    if (n_items > h->slots)
        return fail(WSM_E_INVAL, "more items than reserved slots (wsm_reserve_batch)");
    for (int i = 0; i < n_items; ++i) {
        rc = check_pixels(h, items[i]);
        if (rc != WSM_OK) return rc;
        if (!items[i].d_colors || !items[i].d_counts)
            return fail(WSM_E_INVAL, "null device pointer");
    }
    cudaStream_t s = (cudaStream_t)stream;
    rc = reduce_items(h, items, n_items, s);
    if (rc != WSM_OK) return rc;
    if (n_items == 0) return WSM_OK;
    cudaError_t e = cudaMemcpyAsync(h->host_nu, h->batch_nu, sizeof(int64_t) * n_items,
                                    cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "n_unique copy");
    rc = read_status(h, s);
    if (rc != WSM_OK) return rc;
    for (int i = 0; i < n_items; ++i) items[i].n_unique = h->host_nu[i];
    return WSM_OK;
}

extern "C" int wsm_set_reduce_path(wsm_handle* h, int path) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (path < 0 || path > 2) return fail(WSM_E_INVAL, "path must be 0, 1 or 2");
    h->reduce_path = path;
    return WSM_OK;
}
