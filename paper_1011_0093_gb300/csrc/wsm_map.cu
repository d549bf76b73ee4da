// wsm_map.cu -- pixel mapping (Sec. 1: every pixel takes the palette entry of
// its cluster) and the mean squared error of Eq. 2 (Sec. 3.1).
//
// Mapping: one more pruned assignment of the unique colors against the final
// centers (the persistent sort-means kernel in map mode) scatters each
// color's membership into a 2^24-entry uint8 color->label table; a gather
// kernel then reads the table at every pixel's 24-bit color.  Only the N'
// entries of this image are written, and every pixel's color is one of them.
#include <algorithm>

#include "wsm_internal.cuh"

namespace wsm {


__global__ void __launch_bounds__(256) k_gather(const uint8_t* __restrict__ rgb, int64_t n,
                                                int stride, const uint8_t* __restrict__ lut,
                                                uint8_t* __restrict__ index) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        index[p] = lut[pixel_key(rgb, p, stride)];
}

// The gather of a batch: image i owns blocks [first_blk[i], first_blk[i+1])
// and reads the color->label table of its slot.
struct GatherBatch {
    int n_items;
    int first_blk[kMaxBatch + 1];
    const uint8_t* rgb[kMaxBatch];
    uint8_t* index[kMaxBatch];
    int64_t n[kMaxBatch];
    int stride[kMaxBatch];
    int slot[kMaxBatch];
    int K[kMaxBatch];
    const uint8_t* lut;        // slot s at lut + s * 2^24
    const int64_t* n_dev;      // if set: an image with n_dev[slot] < K was skipped (index 0)
};

__global__ void __launch_bounds__(256) k_gather_batch(const __grid_constant__ GatherBatch B) {
    const int i = item_of_block(B.first_blk, B.n_items, blockIdx.x);
    const int g0 = B.first_blk[i], G = B.first_blk[i + 1] - g0;
    const uint8_t* lut = B.lut + (size_t)B.slot[i] * kHistBins;
    const int64_t n = B.n[i];
    const bool skipped = B.n_dev && B.n_dev[B.slot[i]] < B.K[i];
    for (int64_t p = (int64_t)(blockIdx.x - g0) * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)G * blockDim.x)
        B.index[i][p] = skipped ? 0 : lut[pixel_key(B.rgb[i], p, B.stride[i])];
}

constexpr int kMseThreads = 256;
constexpr int kMseMaxBlocks = 1024;

// v * 2^20 truncated toward zero, for v >= 0 finite below 2^18, from the FP32
// bits of v (exact integer arithmetic).
__device__ __forceinline__ unsigned long long to_fixed20(float v) {
    const unsigned bits = __float_as_uint(v);
    int e = (bits >> 23) & 255;
    unsigned long long m = bits & 0x7FFFFFu;
    if (e) m |= 0x800000u;
    else e = 1;
    const int sh = e - 150 + 20;                // v = m * 2^(e-150)
    if (sh >= 0) return m << min(sh, 40);
    if (sh <= -63) return 0ull;
    return m >> (-sh);
}

// Per-block sums of ||x_p - c_{index_p}||^2, each pixel's FP32 squared
// distance truncated to units of 2^-20 and added as an integer, so the total
// does not depend on the order of the additions.
__global__ void __launch_bounds__(kMseThreads) k_mse_partial(
    const uint8_t* __restrict__ rgb, int64_t n, int stride, const float4* __restrict__ centers,
    int K, const uint8_t* __restrict__ index, unsigned long long* __restrict__ part, Ctrl* ctrl) {
    __shared__ float4 s_c[WSM_MAX_K];
    __shared__ unsigned long long s_red[kMseThreads / 32];
    for (int k = threadIdx.x; k < K; k += blockDim.x) s_c[k] = centers[k];
    __syncthreads();
    unsigned long long acc = 0;
    bool bad = false;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int k = index[p];
        if (k >= K) {
            bad = true;
            continue;
        }
        const uint32_t key = pixel_key(rgb, p, stride);
        const float4 c = s_c[k];
        acc += to_fixed20(sq3((float)((key >> 16) & 255u), (float)((key >> 8) & 255u),
                              (float)(key & 255u), c.x, c.y, c.z));
    }
    if (bad) atomicOr(&ctrl->status, ST_BAD_LABEL);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kMseThreads / 32; ++w) t += s_red[w];
        part[blockIdx.x] = t;
    }
}

// One warp adds the block sums and writes MSE = total * 2^-20 / N.
__global__ void k_mse_final(const unsigned long long* __restrict__ part, int nparts, int64_t n,
                            double* __restrict__ out, double* __restrict__ out2) {
    unsigned long long t = 0;
    for (int i = threadIdx.x; i < nparts; i += 32) t += part[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if (threadIdx.x == 0) {
        const double m = n > 0 ? (double)t * (1.0 / 1048576.0) / (double)n : 0.0;
        *out = m;
        if (out2) *out2 = m;
    }
}

// The images of one distortion launch: image i owns the partial-sum blocks
// [first_blk[i], first_blk[i+1]).
struct MseItems {
    int n_items;
    int first_blk[kMaxBatch + 1];
    const uint8_t* rgb[kMaxBatch];
    int64_t n[kMaxBatch];
    int stride[kMaxBatch];
    const float4* centers[kMaxBatch];
    int K[kMaxBatch];
    const uint8_t* index[kMaxBatch];
    double* out[kMaxBatch];     // MSE (device), always written
    double* user[kMaxBatch];    // MSE (device), a caller's copy, may be null
    unsigned long long* part;   // one partial sum per block of the launch
    unsigned* status;
    const int64_t* n_dev;       // if set: an image with n_dev[i] < K[i] was skipped (MSE 0)
};

// Per-block fixed-point sums as in k_mse_partial, for the image owning the block.
__global__ void __launch_bounds__(kMseThreads)
    k_mse_partial_batch(const __grid_constant__ MseItems B) {
    __shared__ float4 s_c[WSM_MAX_K];
    __shared__ unsigned long long s_red[kMseThreads / 32];
    const int i = item_of_block(B.first_blk, B.n_items, blockIdx.x);
    const int g = blockIdx.x - B.first_blk[i], G = B.first_blk[i + 1] - B.first_blk[i];
    const int K = B.K[i];
    const uint8_t* rgb = B.rgb[i];
    const uint8_t* index = B.index[i];
    const int64_t n = B.n[i];
    const int stride = B.stride[i];
    const bool skipped = B.n_dev && B.n_dev[i] < K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) s_c[k] = B.centers[i][k];
    __syncthreads();
    unsigned long long acc = 0;
    bool bad = false;
    for (int64_t p = (int64_t)g * blockDim.x + threadIdx.x; !skipped && p < n;
         p += (int64_t)G * blockDim.x) {
        const int k = index[p];
        if (k >= K) {
            bad = true;
            continue;
        }
        const uint32_t key = pixel_key(rgb, p, stride);
        const float4 c = s_c[k];
        acc += to_fixed20(sq3((float)((key >> 16) & 255u), (float)((key >> 8) & 255u),
                              (float)(key & 255u), c.x, c.y, c.z));
    }
    if (bad) atomicOr(B.status, ST_BAD_LABEL);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kMseThreads / 32; ++w) t += s_red[w];
        B.part[blockIdx.x] = t;
    }
}

// One warp per image adds its blocks' sums and writes MSE = total * 2^-20 / N.
__global__ void k_mse_final_batch(const __grid_constant__ MseItems B) {
    const int i = blockIdx.x;
    unsigned long long t = 0;
    for (int q = B.first_blk[i] + threadIdx.x; q < B.first_blk[i + 1]; q += 32) t += B.part[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if (threadIdx.x == 0) {
        const double m = (double)t * (1.0 / 1048576.0) / (double)B.n[i];
        *B.out[i] = m;
        if (B.user[i]) *B.user[i] = m;
    }
}

// The final assignment and the gather of n_items images (item i in slot i):
// per kMaxBatch images one persistent launch in map mode and one gather.
int map_items(wsm_handle* h, const wsm_item* items, int n_items, const int64_t* n_dev,
              cudaStream_t s) {
    for (int i0 = 0; i0 < n_items; i0 += kMaxBatch) {
        const int m = std::min(kMaxBatch, n_items - i0);
        int rc = launch_map_items(h, items + i0, m, i0, n_dev, s);
        if (rc != WSM_OK) return rc;
        GatherBatch B;
        B.n_items = m;
        B.lut = h->lut;
        B.n_dev = n_dev;
        int64_t total = 0;
        for (int q = 0; q < m; ++q) total += items[i0 + q].n_pixels;
        const int64_t budget = (int64_t)h->sms * 16;
        B.first_blk[0] = 0;
        for (int q = 0; q < m; ++q) {
            const wsm_item& it = items[i0 + q];
            B.rgb[q] = it.d_rgb;
            B.index[q] = it.d_index;
            B.n[q] = it.n_pixels;
            B.stride[q] = it.pixel_stride;
            B.slot[q] = i0 + q;
            B.K[q] = it.K;
            const int64_t want = (it.n_pixels + 255) / 256;
            const int64_t share =
                std::max<int64_t>(1, budget * it.n_pixels / std::max<int64_t>(total, 1));
            B.first_blk[q + 1] = B.first_blk[q] + (int)std::min(want, share);
        }
        k_gather_batch<<<B.first_blk[m], 256, 0, s>>>(B);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "gather launch");
    }
    return WSM_OK;
}

// Eq. 2 for n_items images (item i's MSE to batch_mse[i] and, if d_mse is
// given, d_mse[i]): per kMaxBatch images one pair of launches.  With n_dev,
// an image skipped for N' < K gets MSE 0.
int distortion_items(wsm_handle* h, const wsm_item* items, int n_items, double* d_mse,
                     const int64_t* n_dev, cudaStream_t s) {
    for (int i0 = 0; i0 < n_items; i0 += kMaxBatch) {
        MseItems B;
        B.n_items = std::min(kMaxBatch, n_items - i0);
        B.n_dev = n_dev ? n_dev + i0 : nullptr;
        B.part = reinterpret_cast<unsigned long long*>(h->mse_part);
        B.status = &h->ctrl->status;
        int64_t total = 0;
        for (int q = 0; q < B.n_items; ++q) total += items[i0 + q].n_pixels;
        // at most 4 blocks per SM in all (and no more than the partial-sum
        // buffer holds), split in proportion to pixels, >= 1 block per image
        const int64_t budget = std::min<int64_t>(kMseMaxBlocks - kMaxBatch, 4 * (int64_t)h->sms);
        B.first_blk[0] = 0;
        for (int q = 0; q < B.n_items; ++q) {
            const wsm_item& it = items[i0 + q];
            B.rgb[q] = it.d_rgb;
            B.n[q] = it.n_pixels;
            B.stride[q] = it.pixel_stride;
            B.centers[q] = reinterpret_cast<const float4*>(it.d_centers);
            B.K[q] = it.K;
            B.index[q] = it.d_index;
            B.out[q] = h->batch_mse + i0 + q;
            B.user[q] = d_mse ? d_mse + i0 + q : nullptr;
            const int64_t want = (it.n_pixels + 4 * kMseThreads - 1) / (4 * kMseThreads);
            const int64_t share = std::max<int64_t>(1, budget * it.n_pixels / total);
            B.first_blk[q + 1] = B.first_blk[q] + (int)std::min(want, share);
        }
        k_mse_partial_batch<<<B.first_blk[B.n_items], kMseThreads, 0, s>>>(B);
        k_mse_final_batch<<<B.n_items, 32, 0, s>>>(B);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "distortion launch");
    }
    return WSM_OK;
}

}  // namespace wsm

using namespace wsm;

extern "C" int wsm_map(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels, int pixel_stride,
                       const uint32_t* d_colors, int64_t n_unique, const float* d_centers, int K,
                       uint8_t* d_labels, uint8_t* d_index, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (pixel_stride != 3 && pixel_stride != 4)
        return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
    if (n_pixels < 1 || n_pixels > h->max_pixels)
        return fail(WSM_E_INVAL, "n_pixels must be in [1, max_pixels]");
    if (n_unique < 1 || n_unique > h->max_unique || n_unique > n_pixels)
        return fail(WSM_E_INVAL, "n_unique must be in [1, min(max_unique, n_pixels)]");
    if (K < 1 || K > h->max_K) return fail(WSM_E_INVAL, "K out of [1, max_K]");
    if (!d_rgb || !d_colors || !d_centers || !d_labels || !d_index)
        return fail(WSM_E_INVAL, "null device pointer");
    if ((uintptr_t)d_centers & 15) return fail(WSM_E_INVAL, "centers must be 16-byte aligned");
    if (pixel_stride == 4 && ((uintptr_t)d_rgb & 3))
        return fail(WSM_E_INVAL, "4-byte pixels must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    rc = launch_sortmeans(h, true, d_colors, nullptr, n_unique, K, const_cast<float*>(d_centers),
                          d_labels, 1, 0.0, s);
    if (rc != WSM_OK) return rc;
    int64_t blocks = (n_pixels + 255) / 256;
    int grid = (int)std::min<int64_t>(blocks, (int64_t)h->sms * 16);
    k_gather<<<grid, 256, 0, s>>>(d_rgb, n_pixels, pixel_stride, h->lut, d_index);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gather launch");
    return WSM_OK;
}

extern "C" int wsm_map_batch(wsm_handle* h, const wsm_item* items, int n_items,
                             wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (n_items < 0 || (n_items > 0 && !items)) return fail(WSM_E_INVAL, "bad item list");
    if (n_items > h->slots)
        return fail(WSM_E_INVAL, "more items than reserved slots (wsm_reserve_batch)");
    for (int i = 0; i < n_items; ++i) {
        rc = check_item(h, items[i], true, false);
        if (rc != WSM_OK) return rc;
    }
    return map_items(h, items, n_items, nullptr, (cudaStream_t)stream);
}

extern "C" int wsm_distortion(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels,
                              int pixel_stride, const float* d_centers, int K,
                              const uint8_t* d_index, double* d_mse, double* mse,
                              wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (pixel_stride != 3 && pixel_stride != 4)
        return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
    if (n_pixels < 0 || n_pixels > h->max_pixels)
        return fail(WSM_E_INVAL, "n_pixels must be in [0, max_pixels]");
    if (K < 1 || K > WSM_MAX_K) return fail(WSM_E_INVAL, "K out of [1, 256]");
    if (n_pixels > 0 && (!d_rgb || !d_index)) return fail(WSM_E_INVAL, "null device pointer");
    if (!d_centers) return fail(WSM_E_INVAL, "null centers");
    if ((uintptr_t)d_centers & 15) return fail(WSM_E_INVAL, "centers must be 16-byte aligned");
    if (pixel_stride == 4 && ((uintptr_t)d_rgb & 3))
        return fail(WSM_E_INVAL, "4-byte pixels must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t want = (n_pixels + 4 * kMseThreads - 1) / (4 * kMseThreads);
    int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>(want, std::min(kMseMaxBlocks, 4 * h->sms)));
    unsigned long long* part = reinterpret_cast<unsigned long long*>(h->mse_part);
    k_mse_partial<<<grid, kMseThreads, 0, s>>>(d_rgb, n_pixels, pixel_stride,
                                                reinterpret_cast<const float4*>(d_centers), K,
                                                d_index, part, h->ctrl);
    k_mse_final<<<1, 32, 0, s>>>(part, grid, n_pixels, h->mse_part + kMseMaxBlocks, d_mse);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "distortion launch");
    if (mse) {
        e = cudaMemcpyAsync(&h->host_ctrl->mse, h->mse_part + kMseMaxBlocks, sizeof(double),
                            cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "mse copy");
        rc = read_status(h, s);
        *mse = h->host_ctrl->mse;
        if (rc != WSM_OK) return rc;
    }
    return WSM_OK;
}

extern "C" int wsm_distortion_batch(wsm_handle* h, const wsm_item* items, int n_items,
                                    double* d_mse, double* mse, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (n_items < 0 || (n_items > 0 && !items)) return fail(WSM_E_INVAL, "bad item list");
    if (n_items > h->slots)
        return fail(WSM_E_INVAL, "more items than reserved slots (wsm_reserve_batch)");
    for (int i = 0; i < n_items; ++i) {
        const wsm_item& it = items[i];
        if (it.pixel_stride != 3 && it.pixel_stride != 4)
            return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
        if (it.n_pixels < 1 || it.n_pixels > h->max_pixels)
            return fail(WSM_E_INVAL, "n_pixels must be in [1, max_pixels]");
        if (it.K < 1 || it.K > WSM_MAX_K) return fail(WSM_E_INVAL, "K out of [1, 256]");
        if (!it.d_rgb || !it.d_index || !it.d_centers)
            return fail(WSM_E_INVAL, "null device pointer");
        if ((uintptr_t)it.d_centers & 15)
            return fail(WSM_E_INVAL, "centers must be 16-byte aligned");
        if (it.pixel_stride == 4 && ((uintptr_t)it.d_rgb & 3))
            return fail(WSM_E_INVAL, "4-byte pixels must be 4-byte aligned");
    }
    if (n_items == 0) return WSM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    rc = distortion_items(h, items, n_items, d_mse, nullptr, s);
    if (rc != WSM_OK) return rc;
    if (mse) {
        cudaError_t e = cudaMemcpyAsync(h->host_mse, h->batch_mse, sizeof(double) * n_items,
                                        cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "mse copy");
        rc = read_status(h, s);
        if (rc != WSM_OK) return rc;
        for (int i = 0; i < n_items; ++i) mse[i] = h->host_mse[i];
    }
    return WSM_OK;
}
