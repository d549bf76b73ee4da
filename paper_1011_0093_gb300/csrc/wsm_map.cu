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

int launch_sortmeans(wsm_handle* h, bool map_mode, const uint32_t* colors, const uint32_t* counts,
                     int64_t n, int K, float* centers, uint8_t* labels, int max_iter, double eps,
                     cudaStream_t s);

__device__ __forceinline__ uint32_t key_of(const uint8_t* __restrict__ rgb, int64_t p, int stride) {
    if (stride == 4) {
        uint32_t v = __ldg(reinterpret_cast<const uint32_t*>(rgb) + p);
        return ((v & 0xFFu) << 16) | (v & 0xFF00u) | ((v >> 16) & 0xFFu);
    }
    const uint8_t* q = rgb + 3 * p;
    return ((uint32_t)__ldg(q) << 16) | ((uint32_t)__ldg(q + 1) << 8) | (uint32_t)__ldg(q + 2);
}

__global__ void __launch_bounds__(256) k_gather(const uint8_t* __restrict__ rgb, int64_t n,
                                                int stride, const uint8_t* __restrict__ lut,
                                                uint8_t* __restrict__ index) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        index[p] = lut[key_of(rgb, p, stride)];
}

constexpr int kMseThreads = 256;
constexpr int kMseMaxBlocks = 1024;

// Per-block FP64 partial sums of ||x_p - c_{index_p}||^2, each block over a
// fixed contiguous range, reduced in a fixed order (deterministic).
__global__ void __launch_bounds__(kMseThreads) k_mse_partial(
    const uint8_t* __restrict__ rgb, int64_t n, int stride, const float4* __restrict__ centers,
    int K, const uint8_t* __restrict__ index, double* __restrict__ part, Ctrl* ctrl) {
    __shared__ float4 s_c[WSM_MAX_K];
    __shared__ double s_red[kMseThreads / 32];
    for (int k = threadIdx.x; k < K; k += blockDim.x) s_c[k] = centers[k];
    __syncthreads();
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t begin = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(n, begin + chunk);
    double acc = 0.0;
    bool bad = false;
    for (int64_t p = begin + threadIdx.x; p < end; p += blockDim.x) {
        int k = index[p];
        if (k >= K) {
            bad = true;
            continue;
        }
        uint32_t key = key_of(rgb, p, stride);
        float4 c = s_c[k];
        acc += (double)sq3((float)((key >> 16) & 255u), (float)((key >> 8) & 255u),
                           (float)(key & 255u), c.x, c.y, c.z);
    }
    if (bad) atomicOr(&ctrl->status, ST_BAD_LABEL);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kMseThreads / 32; ++w) t += s_red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_mse_final(const double* __restrict__ part, int nparts, int64_t n,
                            double* __restrict__ out, double* __restrict__ out2) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nparts; ++i) t += part[i];
        double m = n > 0 ? t / (double)n : 0.0;
        *out = m;
        if (out2) *out2 = m;
    }
}

}  // namespace wsm

using namespace wsm;

extern "C" int wsm_map(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels, int pixel_stride,
                       const uint32_t* d_colors, int64_t n_unique, const float* d_centers, int K,
                       uint8_t* d_labels, uint8_t* d_index, wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (pixel_stride != 3 && pixel_stride != 4) return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
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

extern "C" int wsm_distortion(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels,
                              int pixel_stride, const float* d_centers, int K,
                              const uint8_t* d_index, double* d_mse, double* mse,
                              wsm_stream stream) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (pixel_stride != 3 && pixel_stride != 4) return fail(WSM_E_INVAL, "pixel_stride must be 3 or 4");
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
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, kMseMaxBlocks));
    k_mse_partial<<<grid, kMseThreads, 0, s>>>(d_rgb, n_pixels, pixel_stride,
                                                reinterpret_cast<const float4*>(d_centers), K,
                                                d_index, h->mse_part, h->ctrl);
    k_mse_final<<<1, 32, 0, s>>>(h->mse_part, grid, n_pixels, h->mse_part + kMseMaxBlocks, d_mse);
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
