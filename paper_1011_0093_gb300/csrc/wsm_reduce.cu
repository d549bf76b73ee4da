// wsm_reduce.cu -- unique colors and their frequencies (Sec. 2, data
// sampling and sample weighting).
//
// The paper collects the distinct colors with a chained hash table.  Here
// every pixel adds one to its bin of a 2^24-bin uint32 histogram (one bin per
// 24-bit color) and, when it is the first pixel of that color, sets the
// color's bit in a 2^24-bit occupancy map.  A two-kernel prefix scan over the
// occupancy map then writes (color, count) for every set bit, in ascending
// color order, and clears the bins and bits it read, so the scratch is zero
// again for the next image without a 64 MiB memset.
#include <algorithm>

#include "wsm_internal.cuh"

namespace wsm {

// Packed key 0x00RRGGBB of pixel p.
__device__ __forceinline__ uint32_t pixel_key(const uint8_t* __restrict__ rgb, int64_t p,
                                              int stride) {
    if (stride == 4) {
        uint32_t v = __ldg(reinterpret_cast<const uint32_t*>(rgb) + p);
        return ((v & 0xFFu) << 16) | (v & 0xFF00u) | ((v >> 16) & 0xFFu);
    }
    const uint8_t* q = rgb + 3 * p;
    return ((uint32_t)__ldg(q) << 16) | ((uint32_t)__ldg(q + 1) << 8) | (uint32_t)__ldg(q + 2);
}

// Histogram with warp aggregation: lanes holding the same color elect one
// leader, which adds the group's size with a single atomic.
__global__ void __launch_bounds__(256) k_hist24(const uint8_t* __restrict__ rgb, int64_t n,
                                                int stride, uint32_t* __restrict__ hist,
                                                uint32_t* __restrict__ bitmap) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
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

// Pass 1 of the compaction: the number of set bits in each block's 2048 words.
__global__ void __launch_bounds__(kScanThreads) k_scan_count(const uint32_t* __restrict__ bitmap,
                                                             uint32_t* __restrict__ blk_total) {
    const uint4 a = reinterpret_cast<const uint4*>(bitmap)[
        ((size_t)blockIdx.x * kScanWordsPerBlock + threadIdx.x * kScanWordsPerThread) / 4];
    unsigned c = __popc(a.x) + __popc(a.y) + __popc(a.z) + __popc(a.w);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    __shared__ unsigned s_w[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int i = 0; i < kScanThreads / 32; ++i) t += s_w[i];
        blk_total[blockIdx.x] = t;
    }
}

// Pass 2: each block finds its output offset from the totals of the blocks
// before it, scans its words' bit counts into per-word output offsets, and
// then emits (color, count) for every set bit: a warp takes one word at a
// time, lane l handles bit l (so the 32 bins of a word are read and cleared
// with one coalesced access), kEmitBatch words in flight per warp.  Output
// order is ascending color order.
__global__ void __launch_bounds__(kScanThreads) k_scan_emit(
    uint32_t* __restrict__ bitmap, uint32_t* __restrict__ hist,
    const uint32_t* __restrict__ blk_total, uint32_t* __restrict__ colors,
    uint32_t* __restrict__ counts, int64_t capacity, int64_t* __restrict__ d_n_unique,
    Ctrl* __restrict__ ctrl) {
    __shared__ uint32_t s_word[kScanWordsPerBlock];
    __shared__ uint32_t s_off[kScanWordsPerBlock];
    __shared__ unsigned s_w[kScanThreads / 32];
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // offset of this block: sum of the totals of blocks [0, blockIdx.x)
    unsigned long long before = 0;
    for (int i = tid; i < (int)blockIdx.x; i += kScanThreads) before += blk_total[i];
    for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xFFFFFFFFu, before, o);
    if (tid == 0) s_base = 0;
    __syncthreads();
    if (lane == 0 && before) atomicAdd(&s_base, before);
    const size_t w0 = (size_t)blockIdx.x * kScanWordsPerBlock;
    uint4* wv = reinterpret_cast<uint4*>(bitmap + w0) + tid;
    const uint4 a = wv[0];
    const uint32_t words[4] = {a.x, a.y, a.z, a.w};
    unsigned mine = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) mine += __popc(words[i]);
    // block-wide exclusive scan of `mine`
    unsigned incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    unsigned warp_off = 0;
    for (int i = 0; i < wid; ++i) warp_off += s_w[i];
    unsigned off = warp_off + (incl - mine);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        s_word[4 * tid + i] = words[i];
        s_off[4 * tid + i] = off;
        off += __popc(words[i]);
    }
    if (a.x | a.y | a.z | a.w) wv[0] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const int64_t base = (int64_t)s_base;
    const unsigned below = (1u << lane) - 1u;
    constexpr int kWordsPerWarp = kScanWordsPerBlock / (kScanThreads / 32);
    constexpr int kEmitBatch = 16;
    static_assert(kWordsPerWarp % kEmitBatch == 0, "emit batches");
    for (int q = wid * kWordsPerWarp; q < (wid + 1) * kWordsPerWarp; q += kEmitBatch) {
        uint32_t wd[kEmitBatch], cnt[kEmitBatch];
#pragma unroll
        for (int u = 0; u < kEmitBatch; ++u) {
            wd[u] = s_word[q + u];
            cnt[u] = 0;
            if ((wd[u] >> lane) & 1u) cnt[u] = hist[((w0 + q + u) << 5) | lane];
        }
#pragma unroll
        for (int u = 0; u < kEmitBatch; ++u) {
            if ((wd[u] >> lane) & 1u) {
                const uint32_t key = (uint32_t)((w0 + q + u) << 5) | (uint32_t)lane;
                const int64_t pos = base + s_off[q + u] + __popc(wd[u] & below);
                hist[key] = 0;
                if (pos < capacity) {
                    colors[pos] = key;
                    counts[pos] = cnt[u];
                }
            }
        }
    }
    if (blockIdx.x == gridDim.x - 1 && tid == kScanThreads - 1) {
        const int64_t total = base + off;   // the last thread of the last block ends at N'
        ctrl->n_unique = total;
        if (d_n_unique) *d_n_unique = total;
        if (total > capacity) atomicOr(&ctrl->status, ST_CAPACITY);
    }
}

}  // namespace wsm

using namespace wsm;

extern "C" int wsm_reduce(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels, int pixel_stride,
                          uint32_t* d_colors, uint32_t* d_counts, int64_t capacity,
                          int64_t* d_n_unique, int64_t* n_unique, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (pixel_stride != 3 && pixel_stride != 4) return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
    if (n_pixels < 0 || n_pixels > h->max_pixels)
        return fail(WSM_E_INVAL, "n_pixels must be in [0, max_pixels]");
    if (capacity < 0) return fail(WSM_E_INVAL, "negative capacity");
    if (n_pixels > 0 && !d_rgb) return fail(WSM_E_INVAL, "null pixel pointer");
    if (capacity > 0 && (!d_colors || !d_counts)) return fail(WSM_E_INVAL, "null output pointer");
    if (pixel_stride == 4 && ((uintptr_t)d_rgb & 3))
        return fail(WSM_E_INVAL, "4-byte pixels must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (n_pixels > 0) {
        int64_t warps_needed = (n_pixels + 31) / 32;
        int64_t blocks = (warps_needed + 7) / 8;
        int grid = (int)std::min<int64_t>(blocks, (int64_t)h->sms * 8);
        k_hist24<<<grid, 256, 0, s>>>(d_rgb, n_pixels, pixel_stride, h->hist, h->bitmap);
    }
    k_scan_count<<<kScanBlocks, kScanThreads, 0, s>>>(h->bitmap, h->blk_total);
    k_scan_emit<<<kScanBlocks, kScanThreads, 0, s>>>(h->bitmap, h->hist, h->blk_total, d_colors,
                                                    d_counts, capacity, d_n_unique, h->ctrl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "reduce launch");
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
