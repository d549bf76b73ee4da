// wsm_grad.cu -- the weighted distortion as a differentiable function of the
// palette and of the points (Eq. 1, the k-means objective, with the sample
// weights of Sec. 2):
//
//   D(C, X) = sum_i w_i min_k ||x_i - c_k||^2
//   dD/dc_k = -2 sum_{i : m_i = k} w_i (x_i - c_k)       (m_i: nearest center)
//   dD/dx_i =  2 w_i (x_i - c_{m_i})
//
// away from ties, where D is differentiable (it is piecewise quadratic).
// The forward pass finds m_i with the pruned search of Algorithm 2 (Sec. 2)
// from a starting center (the previous call's m_i when the caller keeps it,
// so a slowly moving palette costs few visits per point), over a table of
// full sorted rows.  It returns D and, per cluster, R_k = sum w_i (x_i - c_k)
// and sum w_i, which is all the backward pass needs for dD/dC.
//
// Sums are FP32 in a fixed order (each lane over its points, a warp's points
// into per-warp cluster slots in lane order, warps in order, blocks in a
// fixed tree), so results are identical run to run; R_k accumulates the
// small residuals x_i - c_k rather than sum w_i x_i, so the gradient keeps
// its accuracy near a Lloyd fixed point, where it vanishes.
#include <algorithm>

#include "wsm_internal.cuh"

namespace wsm {

constexpr int kGradThreads = 256;
constexpr int kGradWarps = kGradThreads / 32;
constexpr int kGradBlocksPerSM = 4;

// Full sorted rows of the K centers (no bound: every center is kept).
__global__ void __launch_bounds__(kGradThreads) k_grad_rows(const float* __restrict__ c, int cs,
                                                            int K, float4* __restrict__ tab,
                                                            uint8_t* __restrict__ tab_nb) {
    __shared__ float4 s_c[WSM_MAX_K];
    __shared__ float s_thr[WSM_MAX_K];
    __shared__ unsigned long long s_wkey[kGradWarps * WSM_MAX_K];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        s_c[k] = make_float4(c[(size_t)k * cs], c[(size_t)k * cs + 1], c[(size_t)k * cs + 2], 0.f);
        s_thr[k] = __int_as_float(0x7f800000);
    }
    __syncthreads();
    build_rows<uint8_t>(K, K, gridDim.x, blockIdx.x, s_c, s_thr, s_wkey, tab, tab_nb);
}

struct GradFwd {
    const float* x;
    int xs;
    const float* w;        // null: every weight is w_uniform
    float w_uniform;
    int64_t n;
    int K;
    uint8_t* assign;
    int warm;              // start each search at assign[i] (else at center 0)
    const float4* tab;
    const uint8_t* nb;
    float4* part;          // [gridDim.x][K + 1]: R_k and sum w per cluster, then (D, 0, 0, 0)
    unsigned* status;
};

__global__ void __launch_bounds__(kGradThreads) k_grad_fwd(const __grid_constant__ GradFwd A) {
    extern __shared__ float4 s_acc[];                // [kGradWarps][K]
    __shared__ float s_d[kGradWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, K = A.K;
    float4* acc = s_acc + (size_t)wid * K;
    for (int k = lane; k < K; k += 32) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    float dsum = 0.f;
    bool bad = false;
    const int64_t step = (int64_t)gridDim.x * kGradWarps * 32;
    for (int64_t base = ((int64_t)blockIdx.x * kGradWarps + wid) * 32; base < A.n; base += step) {
        const int64_t i = base + lane;
        int m = -1;
        float rx = 0.f, ry = 0.f, rz = 0.f, wi = 0.f;
        if (i < A.n) {
            const float* xi = A.x + i * A.xs;
            const float x = xi[0], y = xi[1], z = xi[2];
            wi = A.w ? A.w[i] : A.w_uniform;
            int p = A.warm ? A.assign[i] : 0;
            if (p >= K) {
                bad = true;
                p = 0;
            }
            const float4* row = A.tab + (size_t)p * K;
            float4 best = row[0];                    // entry 0 of row p is c_p
            const float prev = sq3(x, y, z, best.y, best.z, best.w);
            float mn = prev;
            int mpos = 0;
            for (int j = 1; j < K; ++j) {
                const float4 e = row[j];
                if (e.x >= prev) break;              // d[p][t] / 4 >= prev: none nearer further on
                const float d = sq3(x, y, z, e.y, e.z, e.w);
                if (d <= mn) {                       // the later of equal distances wins
                    mn = d;
                    mpos = j;
                    best = e;
                }
            }
            m = A.nb[(size_t)p * K + mpos];
            A.assign[i] = (uint8_t)m;
            dsum = __fmaf_rn(wi, mn, dsum);
            rx = __fmul_rn(wi, __fsub_rn(x, best.y));
            ry = __fmul_rn(wi, __fsub_rn(y, best.z));
            rz = __fmul_rn(wi, __fsub_rn(z, best.w));
        }
        // lane k % 32 owns cluster k's slot; the warp's points are added in lane order
        for (int t = 0; t < 32; ++t) {
            const int mt = __shfl_sync(0xFFFFFFFFu, m, t);
            const float ax = __shfl_sync(0xFFFFFFFFu, rx, t);
            const float ay = __shfl_sync(0xFFFFFFFFu, ry, t);
            const float az = __shfl_sync(0xFFFFFFFFu, rz, t);
            const float aw = __shfl_sync(0xFFFFFFFFu, wi, t);
            if (mt >= 0 && (mt & 31) == lane) {
                float4 v = acc[mt];
                v.x = __fadd_rn(v.x, ax);
                v.y = __fadd_rn(v.y, ay);
                v.z = __fadd_rn(v.z, az);
                v.w = __fadd_rn(v.w, aw);
                acc[mt] = v;
            }
        }
    }
    if (bad) atomicOr(A.status, ST_BAD_LABEL);
    for (int o = 16; o > 0; o >>= 1) dsum = __fadd_rn(dsum, __shfl_xor_sync(0xFFFFFFFFu, dsum, o));
    if (lane == 0) s_d[wid] = dsum;
    __syncthreads();
    float4* out = A.part + (size_t)blockIdx.x * (K + 1);
    for (int k = threadIdx.x; k < K; k += kGradThreads) {
        float4 v = s_acc[k];
        for (int q = 1; q < kGradWarps; ++q) {
            const float4 u = s_acc[(size_t)q * K + k];
            v.x = __fadd_rn(v.x, u.x);
            v.y = __fadd_rn(v.y, u.y);
            v.z = __fadd_rn(v.z, u.z);
            v.w = __fadd_rn(v.w, u.w);
        }
        out[k] = v;
    }
    if (threadIdx.x == 0) {
        float d = s_d[0];
        for (int q = 1; q < kGradWarps; ++q) d = __fadd_rn(d, s_d[q]);
        out[K] = make_float4(d, 0.f, 0.f, 0.f);
    }
}

// One warp per output row r of the block partials (r < K: cluster r, r = K:
// D), summed over the nparts blocks in a fixed order.
__global__ void k_grad_reduce(const float4* __restrict__ part, int nparts, int K,
                              float4* __restrict__ resid, float* __restrict__ D) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r > K) return;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int b = lane; b < nparts; b += 32) {
        const float4 u = part[(size_t)b * (K + 1) + r];
        v.x = __fadd_rn(v.x, u.x);
        v.y = __fadd_rn(v.y, u.y);
        v.z = __fadd_rn(v.z, u.z);
        v.w = __fadd_rn(v.w, u.w);
    }
    for (int o = 16; o > 0; o >>= 1) {
        v.x = __fadd_rn(v.x, __shfl_xor_sync(0xFFFFFFFFu, v.x, o));
        v.y = __fadd_rn(v.y, __shfl_xor_sync(0xFFFFFFFFu, v.y, o));
        v.z = __fadd_rn(v.z, __shfl_xor_sync(0xFFFFFFFFu, v.z, o));
        v.w = __fadd_rn(v.w, __shfl_xor_sync(0xFFFFFFFFu, v.w, o));
    }
    if (lane == 0) {
        if (r < K) resid[r] = v;
        else *D = v.x;
    }
}

struct GradBwd {
    const float* x;
    int xs;
    const float* w;
    float w_uniform;
    int64_t n;
    const float* c;
    int cs;
    int K;
    const uint8_t* assign;
    const float4* resid;
    const float* gD;       // dL/dD (device scalar)
    float* gC;             // [K][cs] or null
    float* gX;             // [n][xs] or null
    unsigned* status;
};

__global__ void __launch_bounds__(kGradThreads) k_grad_bwd(const __grid_constant__ GradBwd A) {
    __shared__ float4 s_c[WSM_MAX_K];
    const int K = A.K;
    const float g2 = __fmul_rn(2.f, *A.gD);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const float* ck = A.c + (size_t)k * A.cs;
        s_c[k] = make_float4(ck[0], ck[1], ck[2], 0.f);
        if (blockIdx.x == 0 && A.gC) {
            const float4 r = A.resid[k];
            float* gk = A.gC + (size_t)k * A.cs;
            gk[0] = -__fmul_rn(g2, r.x);
            gk[1] = -__fmul_rn(g2, r.y);
            gk[2] = -__fmul_rn(g2, r.z);
            if (A.cs == 4) gk[3] = 0.f;
        }
    }
    __syncthreads();
    if (!A.gX) return;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int m = A.assign[i];
        float* gi = A.gX + i * A.xs;
        if (m >= K) {
            bad = true;
            continue;
        }
        const float* xi = A.x + i * A.xs;
        const float s = __fmul_rn(g2, A.w ? A.w[i] : A.w_uniform);
        const float4 c = s_c[m];
        gi[0] = __fmul_rn(s, __fsub_rn(xi[0], c.x));
        gi[1] = __fmul_rn(s, __fsub_rn(xi[1], c.y));
        gi[2] = __fmul_rn(s, __fsub_rn(xi[2], c.z));
        if (A.xs == 4) gi[3] = 0.f;
    }
    if (bad) atomicOr(A.status, ST_BAD_LABEL);
}

static int check_grad_args(wsm_handle* h, const float* d_x, int x_stride, int64_t n,
                           const float* d_centers, int c_stride, int K) {
    int rc = check_handle(h);
    if (rc != WSM_OK) return rc;
    if (x_stride != 3 && x_stride != 4) return fail(WSM_E_INVAL, "x_stride must be 3 or 4");
    if (c_stride != 3 && c_stride != 4) return fail(WSM_E_INVAL, "c_stride must be 3 or 4");
    if (n < 0 || n > ((int64_t)1 << 31)) return fail(WSM_E_INVAL, "n must be in [0, 2^31]");
    if (K < 1 || K > std::min(h->max_K, WSM_MAX_K))
        return fail(WSM_E_INVAL, "K out of [1, min(max_K, 256)]");
    if (n > 0 && !d_x) return fail(WSM_E_INVAL, "null point pointer");
    if (!d_centers) return fail(WSM_E_INVAL, "null centers");
    return WSM_OK;
}

int grad_blocks(wsm_handle* h) { return kGradBlocksPerSM * h->sms; }

}  // namespace wsm

using namespace wsm;

extern "C" int wsm_distortion_fwd(wsm_handle* h, const float* d_x, int x_stride, const float* d_w,
                                  int64_t n, const float* d_centers, int c_stride, int K,
                                  uint8_t* d_assign, int warm_start, float* d_D, float* d_resid,
                                  wsm_stream stream) {
    int rc = check_grad_args(h, d_x, x_stride, n, d_centers, c_stride, K);
    if (rc != WSM_OK) return rc;
    if (!d_D || !d_resid) return fail(WSM_E_INVAL, "null output pointer");
    if ((uintptr_t)d_resid & 15) return fail(WSM_E_INVAL, "resid must be 16-byte aligned");
    if (n > 0 && !d_assign) return fail(WSM_E_INVAL, "null assignment pointer");
    cudaStream_t s = (cudaStream_t)stream;
    k_grad_rows<<<(K + kGradWarps - 1) / kGradWarps, kGradThreads, 0, s>>>(
        d_centers, c_stride, K, h->grad_tab, h->grad_nb);
    int grid = 0;
    if (n > 0) {
        grid = (int)std::min<int64_t>((n + kGradThreads - 1) / kGradThreads, grad_blocks(h));
        GradFwd A;
        A.x = d_x;
        A.xs = x_stride;
        A.w = d_w;
        A.w_uniform = 1.0f / (float)n;
        A.n = n;
        A.K = K;
        A.assign = d_assign;
        A.warm = warm_start ? 1 : 0;
        A.tab = h->grad_tab;
        A.nb = h->grad_nb;
        A.part = h->grad_part;
        A.status = &h->ctrl->status;
        k_grad_fwd<<<grid, kGradThreads, sizeof(float4) * kGradWarps * K, s>>>(A);
    }
    const int rows_per_block = 256 / 32;
    k_grad_reduce<<<(K + 1 + rows_per_block - 1) / rows_per_block, 256, 0, s>>>(
        h->grad_part, grid, K, reinterpret_cast<float4*>(d_resid), d_D);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "distortion forward launch");
    return WSM_OK;
}

extern "C" int wsm_distortion_bwd(wsm_handle* h, const float* d_x, int x_stride, const float* d_w,
                                  int64_t n, const float* d_centers, int c_stride, int K,
                                  const uint8_t* d_assign, const float* d_resid, const float* d_gD,
                                  float* d_gC, float* d_gX, wsm_stream stream) {
    int rc = check_grad_args(h, d_x, x_stride, n, d_centers, c_stride, K);
    if (rc != WSM_OK) return rc;
    if (!d_resid || !d_gD) return fail(WSM_E_INVAL, "null resid or upstream gradient");
    if ((uintptr_t)d_resid & 15) return fail(WSM_E_INVAL, "resid must be 16-byte aligned");
    if (d_gX && n > 0 && !d_assign) return fail(WSM_E_INVAL, "null assignment pointer");
    if (!d_gC && !d_gX) return WSM_OK;
    GradBwd A;
    A.x = d_x;
    A.xs = x_stride;
    A.w = d_w;
    A.w_uniform = n > 0 ? 1.0f / (float)n : 0.f;
    A.n = n;
    A.c = d_centers;
    A.cs = c_stride;
    A.K = K;
    A.assign = d_assign;
    A.resid = reinterpret_cast<const float4*>(d_resid);
    A.gD = d_gD;
    A.gC = d_gC;
    A.gX = n > 0 ? d_gX : nullptr;
    A.status = &h->ctrl->status;
    const int grid = A.gX ? (int)std::max<int64_t>(1, std::min<int64_t>(
                                (n + kGradThreads - 1) / kGradThreads, 8 * (int64_t)h->sms))
                          : 1;
    k_grad_bwd<<<grid, kGradThreads, 0, (cudaStream_t)stream>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "distortion backward launch");
    return WSM_OK;
}
