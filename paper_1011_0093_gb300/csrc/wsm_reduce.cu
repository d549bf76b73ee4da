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

// Launch the three reduction kernels for R.n_items images whose per-image
// fields are filled in; sets the scratch pointers and the histogram blocks.
static int launch_reduce(wsm_handle* h, ReduceItems& R, cudaStream_t s) {
    R.hist = h->hist;
    R.bitmap = h->bitmap;
    R.blk_total = h->blk_total;
    R.status = &h->ctrl->status;
    int64_t total = 0;
    for (int i = 0; i < R.n_items; ++i) total += R.n[i];
    // at most 8 blocks of 256 per SM in all, split in proportion to pixels
    const int64_t budget = (int64_t)h->sms * 8;
    R.first_blk[0] = 0;
    for (int i = 0; i < R.n_items; ++i) {
        const int64_t want = (R.n[i] + 255) / 256;
        const int64_t share = std::max<int64_t>(1, budget * R.n[i] / std::max<int64_t>(total, 1));
        R.first_blk[i + 1] = R.first_blk[i] + (int)(R.n[i] > 0 ? std::min(want, share) : 0);
    }
    if (R.first_blk[R.n_items] > 0) k_hist24<<<R.first_blk[R.n_items], 256, 0, s>>>(R);
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
