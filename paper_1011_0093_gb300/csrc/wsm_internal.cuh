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
};

// A grid barrier waits at most this long (globaltimer ns) before giving up.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

constexpr int kHistBins = 1 << 24;           // one bin per 24-bit color
constexpr int kMapWords = kHistBins / 32;    // occupancy bitmap words
constexpr int kScanWordsPerThread = 8;       // bitmap words per thread in the compaction
constexpr int kScanThreads = 256;
constexpr int kScanWordsPerBlock = kScanWordsPerThread * kScanThreads;   // 2048
constexpr int kScanBlocks = kMapWords / kScanWordsPerBlock;             // 256
constexpr int kIterThreads = 512;            // threads per block of the persistent kernel
constexpr int kMaxTrace = 4096;              // SSE values kept per wsm_iterate call

// Control words in device memory (one block per handle).
// The first kLaunchResetBytes bytes are cleared before every persistent
// launch, so a barrier abandoned after a timeout cannot confuse the next one.
struct Ctrl {
    unsigned bar_count;        // grid barrier: arrivals
    unsigned bar_gen;          // grid barrier: generation
    int iters_done;            // iterations completed by the last wsm_iterate
    unsigned reserved;
    unsigned long long evaluated;  // distances computed by the last persistent launch
    unsigned status;           // ST_* bits (cleared only when read by the host)
    unsigned reserved2;
    int64_t n_unique;          // N' of the last wsm_reduce
    double mse;                // host mirror slot of the last wsm_distortion
};
constexpr size_t kLaunchResetBytes = 24;
static_assert(offsetof(Ctrl, status) == kLaunchResetBytes, "Ctrl layout");

}  // namespace wsm

struct wsm_handle {
    int device = -1;
    int sms = 0;
    int max_K = 0;
    int64_t max_pixels = 0;
    int64_t max_unique = 0;
    int iter_grid = 0;           // co-resident blocks of the persistent kernel
    int iter_blocks_per_sm = 0;
    // scratch (device)
    uint32_t* hist = nullptr;    // [2^24] zero between calls
    uint32_t* bitmap = nullptr;  // [2^19] zero between calls
    uint32_t* blk_total = nullptr;   // [kScanBlocks]
    uint8_t* lut = nullptr;      // [2^24] color -> label
    float4* tab = nullptr;       // [max_K * max_K] sorted rows: (d/4, c.x, c.y, c.z)
    uint8_t* tab_nb = nullptr;   // [max_K * max_K] center index of each row entry
    unsigned long long* acc = nullptr;  // [2][max_K][4]: S_k (3) and W_k
    double* sse_part = nullptr;  // [2][iter_grid]
    double* trace = nullptr;     // [kMaxTrace]
    double* mse_part = nullptr;  // [1024] block partials + [1] result
    wsm::Ctrl* ctrl = nullptr;
    wsm::Ctrl* host_ctrl = nullptr;  // pinned mirror for status reads
};

namespace wsm {

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
int check_handle(wsm_handle* h);
int read_status(wsm_handle* h, cudaStream_t s);

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

// Grid-wide barrier for a cooperative launch of `nblocks` co-resident
// blocks.  Thread 0 of each block arrives on a counter; the last arrival
// resets it and advances the generation word; the others spin on the
// generation with a time limit.  On a timeout the status word gets
// ST_TIMEOUT and the function returns false in every thread of the block
// (also when another block recorded a failure).  Memory written before the
// barrier by any block is visible to every block after it.
__device__ __forceinline__ bool grid_sync(Ctrl* ctrl, unsigned nblocks) {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned gen = ld_acquire(&ctrl->bar_gen);
        __threadfence();
        unsigned arrived = atomicAdd(&ctrl->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&ctrl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctrl->bar_gen, 1u);
        } else {
            unsigned long long t0 = global_ns();
            while (ld_acquire(&ctrl->bar_gen) == gen) {
                if (global_ns() - t0 > kWaitLimitNs) {
                    atomicOr(&ctrl->status, ST_TIMEOUT);
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        s_ok = (ld_acquire(&ctrl->status) & ST_TIMEOUT) ? 0u : 1u;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ float sq3(float ax, float ay, float az, float bx, float by, float bz) {
    float ex = ax - bx, ey = ay - by, ez = az - bz;
    return ex * ex + ey * ey + ez * ez;
}

}  // namespace wsm
