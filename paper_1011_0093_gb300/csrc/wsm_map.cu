// wsm_map.cu -- pixel mapping (Sec. 1: every pixel takes the palette entry of
// its cluster) and the mean squared error of Eq. 2 (Sec. 3.1).
//
// Mapping: one more pruned assignment of the unique colors against the final
// centers (the persistent sort-means kernel in map mode) scatters each
// color's membership into a 2^24-entry color->label table (uint8, or uint16
// for a wide handle); a gather kernel then reads the table at every pixel's
// 24-bit color.  Only the N' entries of this image are written, and every
// pixel's color is one of them.  The per-pixel MSE reads the pixels and the
// index image; the batch pipeline's MSE comes from the final assignment
// instead (wsm_pipeline.cu).
#include <algorithm>

#include "wsm_pixels.cuh"

namespace wsm {


constexpr int kPixThreads = 256;
constexpr int kMseMaxBlocks = 1024;   // partial sums the handle's buffer holds

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

// ||x - c_k||^2 of a pixel key in units of 2^-20 (truncated), or a flag for
// a label outside the palette.
struct MseSum {
    unsigned long long acc;
    bool bad;
};

__device__ __forceinline__ void mse_add(MseSum& m, uint32_t key, int k, int K,
                                        const float4* s_c) {
    if (k >= K) {
        m.bad = true;
        return;
    }
    const float4 c = s_c[k];
    m.acc += to_fixed20(sq3((float)(key >> 16), (float)((key >> 8) & 255u), (float)(key & 255u),
                            c.x, c.y, c.z));
}

// One pass over the pixels of one image that thread t of nt handles.
//   kGather: index[p] = lut[color of p] (0 for a skipped image);
//   kMse:    the sum of ||x_p - c_{label_p}||^2, label_p the gathered label
//            (kGather) or index[p], each pixel's FP32 squared distance
//            truncated to units of 2^-20 and added as an integer, so that the
//            total does not depend on the order of the additions.
// Groups of 16 pixels go with vector loads (and 16-byte index stores or
// loads: one for uint8 labels, two for uint16) when the pixels and the index
// image are 16-byte aligned, then the last n % 16 pixels (or all of an
// unaligned image) one at a time.
template <bool kGather, bool kMse, typename Label>
__device__ __forceinline__ MseSum pixel_pass(const uint8_t* __restrict__ rgb, int64_t n,
                                             int stride, const Label* __restrict__ lut,
                                             Label* __restrict__ index, const float4* s_c,
                                             int K, bool skipped, int64_t t, int64_t nt) {
    constexpr int kB = (int)sizeof(Label);              // bytes per label
    constexpr uint32_t kMask = kB == 1 ? 0xFFu : 0xFFFFu;
    MseSum m = {0ull, false};
    if (skipped && !kGather) return m;
    int64_t done = 0;
    if (vector_ok(rgb, index)) {
        const int64_t ng = n / kGroup;
        for (int64_t g = t; g < ng; g += nt) {
            uint32_t lab[4 * kB] = {};                  // the group's labels, packed
            if (!skipped) {
                uint32_t key[kGroup];
                pixel_keys16(rgb, g, stride, key);
                if (kGather) {
#pragma unroll
                    for (int j = 0; j < kGroup; ++j)
                        lab[(j * kB) >> 2] |= (uint32_t)__ldg(lut + key[j]) << (8 * ((j * kB) & 3));
                } else {
#pragma unroll
                    for (int v = 0; v < kB; ++v) {
                        const uint4 w = __ldg(reinterpret_cast<const uint4*>(index) + g * kB + v);
                        lab[4 * v + 0] = w.x;
                        lab[4 * v + 1] = w.y;
                        lab[4 * v + 2] = w.z;
                        lab[4 * v + 3] = w.w;
                    }
                }
                if (kMse) {
#pragma unroll
                    for (int j = 0; j < kGroup; ++j)
                        mse_add(m, key[j], (lab[(j * kB) >> 2] >> (8 * ((j * kB) & 3))) & kMask,
                                K, s_c);
                }
            }
            if (kGather) {
#pragma unroll
                for (int v = 0; v < kB; ++v)
                    reinterpret_cast<uint4*>(index)[g * kB + v] =
                        make_uint4(lab[4 * v], lab[4 * v + 1], lab[4 * v + 2], lab[4 * v + 3]);
            }
        }
        done = ng * kGroup;
    }
    for (int64_t p = done + t; p < n; p += nt) {
        if (skipped) {
            index[p] = 0;   // kGather only
            continue;
        }
        const uint32_t key = pixel_key(rgb, p, stride);
        const int k = kGather ? (int)__ldg(lut + key) : (int)index[p];
        if (kGather) index[p] = (Label)k;
        if (kMse) mse_add(m, key, k, K, s_c);
    }
    return m;
}

// Palette entries a block stages in shared memory for the MSE.
template <typename Label>
struct PalMax {
    static constexpr int value = sizeof(Label) == 1 ? WSM_MAX_K : WSM_MAX_K_WIDE;
};

// The block's sum of acc over its threads (thread 0 returns it).
__device__ __forceinline__ unsigned long long block_sum(unsigned long long acc) {
    __shared__ unsigned long long s_red[kPixThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kPixThreads / 32; ++w) t += s_red[w];
    return t;
}

template <typename Label>
__global__ void __launch_bounds__(kPixThreads) k_gather(const uint8_t* __restrict__ rgb,
                                                        int64_t n, int stride,
                                                        const Label* __restrict__ lut,
                                                        Label* __restrict__ index) {
    pixel_pass<true, false, Label>(rgb, n, stride, lut, index, nullptr, 0, false,
                                   (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                   (int64_t)gridDim.x * blockDim.x);
}

// Per-block sums of the squared errors of one image's pixels.
template <typename Label>
__global__ void __launch_bounds__(kPixThreads) k_mse_partial(
    const uint8_t* __restrict__ rgb, int64_t n, int stride, const float4* __restrict__ centers,
    int K, const Label* __restrict__ index, unsigned long long* __restrict__ part, Ctrl* ctrl) {
    __shared__ float4 s_c[PalMax<Label>::value];
    for (int k = threadIdx.x; k < K; k += blockDim.x) s_c[k] = centers[k];
    __syncthreads();
    const MseSum m = pixel_pass<false, true, Label>(
        rgb, n, stride, nullptr, const_cast<Label*>(index), s_c, K, false,
        (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
    if (m.bad) atomicOr(&ctrl->status, ST_BAD_LABEL);
    const unsigned long long t = block_sum(m.acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
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

// The images of one pixel pass over a batch (gather or MSE): image i owns
// the blocks [first_blk[i], first_blk[i+1]).
struct PixelItems {
    int n_items;
    int first_blk[kMaxBatch + 1];
    const uint8_t* rgb[kMaxBatch];
    void* index[kMaxBatch];             // uint8 or uint16 labels (the handle's width)
    int64_t n[kMaxBatch];
    int stride[kMaxBatch];
    int K[kMaxBatch];
    const void* lut[kMaxBatch];         // the image's color->label table (gather)
    const float4* centers[kMaxBatch];   // (MSE)
    double* out[kMaxBatch];             // MSE (device), always written
    double* user[kMaxBatch];            // MSE (device), a caller's copy, may be null
    unsigned long long* part;           // one partial sum per block of the launch
    unsigned* status;
    const int64_t* n_dev;   // [n_items] or null: an image with N' < K was skipped
                            // (index 0, MSE 0)
};

template <bool kGather, bool kMse, typename Label>
__global__ void __launch_bounds__(kPixThreads)
    k_pixels_batch(const __grid_constant__ PixelItems B) {
    __shared__ float4 s_c[kMse ? PalMax<Label>::value : 1];
    const int i = item_of_block(B.first_blk, B.n_items, blockIdx.x);
    const int g = blockIdx.x - B.first_blk[i], G = B.first_blk[i + 1] - B.first_blk[i];
    const int K = B.K[i];
    const bool skipped = B.n_dev && B.n_dev[i] < K;
    if (kMse) {
        for (int k = threadIdx.x; k < K; k += blockDim.x) s_c[k] = B.centers[i][k];
        __syncthreads();
    }
    const MseSum m = pixel_pass<kGather, kMse, Label>(
        B.rgb[i], B.n[i], B.stride[i], static_cast<const Label*>(B.lut[i]),
        static_cast<Label*>(B.index[i]), s_c, K, skipped, (int64_t)g * blockDim.x + threadIdx.x,
        (int64_t)G * blockDim.x);
    if (kMse) {
        if (m.bad) atomicOr(B.status, ST_BAD_LABEL);
        const unsigned long long t = block_sum(m.acc);
        if (threadIdx.x == 0) B.part[blockIdx.x] = t;
    }
}

// One warp per image adds its blocks' sums and writes MSE = total * 2^-20 / N.
__global__ void k_mse_final_batch(const __grid_constant__ PixelItems B) {
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

// The final assignment of n_items images (item i in slot i): labels of the
// unique colors and the slot's color->label table (and, with sse, the
// slot's squared-error sum), per kMaxBatch images one persistent launch in
// map mode.
int map_items(wsm_handle* h, const wsm_item* items, int n_items, const int64_t* n_dev, bool sse,
              cudaStream_t s) {
    for (int i0 = 0; i0 < n_items; i0 += kMaxBatch) {
        const int m = std::min(kMaxBatch, n_items - i0);
        int rc = launch_map_items(h, items + i0, m, i0, n_dev, sse, s);
        if (rc != WSM_OK) return rc;
    }
    return WSM_OK;
}

// A pass over the pixels of n_items images (item i in slot i), per kMaxBatch
// images one launch: the index images through the slots' tables (gather,
// after map_items), or Eq. 2 from the index images (item i's MSE to
// batch_mse[i] and, if d_mse is given, d_mse[i]; plus one launch of the
// final sums).
int pixel_items(wsm_handle* h, const wsm_item* items, int n_items, bool gather, double* d_mse,
                const int64_t* n_dev, cudaStream_t s) {
    for (int i0 = 0; i0 < n_items; i0 += kMaxBatch) {
        PixelItems B;
        B.n_items = std::min(kMaxBatch, n_items - i0);
        B.n_dev = n_dev ? n_dev + i0 : nullptr;
        B.part = reinterpret_cast<unsigned long long*>(h->mse_part);
        B.status = &h->ctrl->status;
        int64_t total = 0;
        for (int q = 0; q < B.n_items; ++q) total += items[i0 + q].n_pixels;
        // at most 6 blocks of 256 per SM in all (and no more partial sums than
        // the buffer holds), split in proportion to pixels, >= 1 block per
        // image, one 16-pixel group per thread
        const int64_t budget = std::min<int64_t>(kMseMaxBlocks - kMaxBatch, 6 * (int64_t)h->sms);
        B.first_blk[0] = 0;
        for (int q = 0; q < B.n_items; ++q) {
            const wsm_item& it = items[i0 + q];
            B.rgb[q] = it.d_rgb;
            B.index[q] = it.d_index;
            B.n[q] = it.n_pixels;
            B.stride[q] = it.pixel_stride;
            B.K[q] = it.K;
            B.lut[q] = h->lut + (size_t)(i0 + q) * kHistBins * h->label_bytes;
            B.centers[q] = reinterpret_cast<const float4*>(it.d_centers);
            B.out[q] = h->batch_mse + i0 + q;
            B.user[q] = d_mse ? d_mse + i0 + q : nullptr;
            const int64_t want = (it.n_pixels + kGroup * kPixThreads - 1) / (kGroup * kPixThreads);
            const int64_t share = std::max<int64_t>(1, budget * it.n_pixels / total);
            B.first_blk[q + 1] = B.first_blk[q] + (int)std::min(want, share);
        }
        const int grid = B.first_blk[B.n_items];
        const bool wide = h->label_bytes == 2;
        if (gather) {
            if (wide) k_pixels_batch<true, false, uint16_t><<<grid, kPixThreads, 0, s>>>(B);
            else k_pixels_batch<true, false, uint8_t><<<grid, kPixThreads, 0, s>>>(B);
        } else {
            if (wide) k_pixels_batch<false, true, uint16_t><<<grid, kPixThreads, 0, s>>>(B);
            else k_pixels_batch<false, true, uint8_t><<<grid, kPixThreads, 0, s>>>(B);
            k_mse_final_batch<<<B.n_items, 32, 0, s>>>(B);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "pixel pass launch");
    }
    return WSM_OK;
}

// The palette as 8-bit colors: each coordinate rounded to the nearest
// integer (rintf: ties to even in the default rounding mode), clamped.
__global__ void k_round_palette(const float4* __restrict__ centers, int K,
                                uchar4* __restrict__ palette, float4* __restrict__ rounded) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        const float4 c = centers[k];
        const float r = fminf(fmaxf(rintf(c.x), 0.f), 255.f);
        const float g = fminf(fmaxf(rintf(c.y), 0.f), 255.f);
        const float b = fminf(fmaxf(rintf(c.z), 0.f), 255.f);
        if (palette) palette[k] = make_uchar4((unsigned char)r, (unsigned char)g,
                                              (unsigned char)b, 0);
        if (rounded) rounded[k] = make_float4(r, g, b, 0.f);
    }
}

// Largest palette the per-pixel calls take with this handle's labels: 256
// for uint8 labels, 1024 for uint16.
static int palette_limit(const wsm_handle* h) {
    return h->label_bytes == 2 ? WSM_MAX_K_WIDE : WSM_MAX_K;
}

}  // namespace wsm

using namespace wsm;

extern "C" int wsm_map(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels, int pixel_stride,
                       const uint32_t* d_colors, int64_t n_unique, const float* d_centers, int K,
                       void* d_labels, void* d_index, wsm_stream stream) {
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
    int64_t blocks = (n_pixels + 256 * kGroup - 1) / (256 * kGroup);
    int grid = (int)std::min<int64_t>(blocks, (int64_t)h->sms * 8);
    if (h->label_bytes == 2)
        k_gather<uint16_t><<<grid, 256, 0, s>>>(d_rgb, n_pixels, pixel_stride,
                                                reinterpret_cast<const uint16_t*>(h->lut),
                                                static_cast<uint16_t*>(d_index));
    else
        k_gather<uint8_t><<<grid, 256, 0, s>>>(d_rgb, n_pixels, pixel_stride, h->lut,
                                               static_cast<uint8_t*>(d_index));
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
    rc = map_items(h, items, n_items, nullptr, false, (cudaStream_t)stream);
    if (rc != WSM_OK) return rc;
    return pixel_items(h, items, n_items, true, nullptr, nullptr, (cudaStream_t)stream);
}

extern "C" int wsm_distortion(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels,
                              int pixel_stride, const float* d_centers, int K,
                              const void* d_index, double* d_mse, double* mse,
                              wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (pixel_stride != 3 && pixel_stride != 4)
        return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
    if (n_pixels < 0 || n_pixels > h->max_pixels)
        return fail(WSM_E_INVAL, "n_pixels must be in [0, max_pixels]");
    if (K < 1 || K > palette_limit(h)) return fail(WSM_E_INVAL, "K out of [1, palette limit]");
    if (n_pixels > 0 && (!d_rgb || !d_index)) return fail(WSM_E_INVAL, "null device pointer");
    if (!d_centers) return fail(WSM_E_INVAL, "null centers");
    if ((uintptr_t)d_centers & 15) return fail(WSM_E_INVAL, "centers must be 16-byte aligned");
    if (pixel_stride == 4 && ((uintptr_t)d_rgb & 3))
        return fail(WSM_E_INVAL, "4-byte pixels must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t want = (n_pixels + kGroup * kPixThreads - 1) / (kGroup * kPixThreads);
    int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>(want, std::min(kMseMaxBlocks, 6 * h->sms)));
    unsigned long long* part = reinterpret_cast<unsigned long long*>(h->mse_part);
    const float4* c4 = reinterpret_cast<const float4*>(d_centers);
    if (h->label_bytes == 2)
        k_mse_partial<uint16_t><<<grid, kPixThreads, 0, s>>>(
            d_rgb, n_pixels, pixel_stride, c4, K, static_cast<const uint16_t*>(d_index), part,
            h->ctrl);
    else
        k_mse_partial<uint8_t><<<grid, kPixThreads, 0, s>>>(
            d_rgb, n_pixels, pixel_stride, c4, K, static_cast<const uint8_t*>(d_index), part,
            h->ctrl);
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
        if (it.K < 1 || it.K > palette_limit(h))
            return fail(WSM_E_INVAL, "K out of [1, palette limit]");
        if (!it.d_rgb || !it.d_index || !it.d_centers)
            return fail(WSM_E_INVAL, "null device pointer");
        if ((uintptr_t)it.d_centers & 15)
            return fail(WSM_E_INVAL, "centers must be 16-byte aligned");
        if (it.pixel_stride == 4 && ((uintptr_t)it.d_rgb & 3))
            return fail(WSM_E_INVAL, "4-byte pixels must be 4-byte aligned");
    }
    if (n_items == 0) return WSM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    rc = pixel_items(h, items, n_items, false, d_mse, nullptr, s);
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

extern "C" int wsm_round_palette(wsm_handle* h, const float* d_centers, int K, uint8_t* d_palette,
                                 float* d_rounded, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (K < 1 || K > palette_limit(h)) return fail(WSM_E_INVAL, "K out of [1, palette limit]");
    if (!d_centers) return fail(WSM_E_INVAL, "null centers");
    if (((uintptr_t)d_centers & 15) || ((uintptr_t)d_rounded & 15) || ((uintptr_t)d_palette & 3))
        return fail(WSM_E_INVAL, "centers/rounded must be 16-byte, palette 4-byte aligned");
    k_round_palette<<<(K + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(d_centers), K, reinterpret_cast<uchar4*>(d_palette),
        reinterpret_cast<float4*>(d_rounded));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "palette launch");
    return WSM_OK;
}
