// wsm_pixels.cuh -- vector reads of packed 8-bit pixels for the kernels that
// stream whole images (unique-color histogram, gather, MSE).
//
// Sixteen consecutive pixels occupy 48 bytes (R, G, B) or 64 bytes (R, G, B,
// pad): three or four 16-byte loads instead of one load per byte.  A group
// starts at a pixel index that is a multiple of 16, so its first byte is
// 16-byte aligned whenever the image base is; callers take the vector path
// only for such bases and finish the last n % 16 pixels one at a time with
// pixel_key.
#pragma once

#include "wsm_internal.cuh"

namespace wsm {

constexpr int kGroup = 16;   // pixels per vector group

// Keys 0x00RRGGBB of pixels 16 g .. 16 g + 15 (stride 3 or 4 bytes per pixel;
// rgb 16-byte aligned).
__device__ __forceinline__ void pixel_keys16(const uint8_t* __restrict__ rgb, int64_t g,
                                             int stride, uint32_t (&key)[kGroup]) {
    if (stride == 4) {
        const uint4* q = reinterpret_cast<const uint4*>(rgb) + 4 * g;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const uint4 w = __ldg(q + v);
            // bytes (R, G, B, pad) -> 0x00RRGGBB; selector nibble 4 takes a zero byte
            key[4 * v + 0] = __byte_perm(w.x, 0u, 0x4012);
            key[4 * v + 1] = __byte_perm(w.y, 0u, 0x4012);
            key[4 * v + 2] = __byte_perm(w.z, 0u, 0x4012);
            key[4 * v + 3] = __byte_perm(w.w, 0u, 0x4012);
        }
        return;
    }
    const uint4* q = reinterpret_cast<const uint4*>(rgb) + 3 * g;
    uint32_t w[12];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const uint4 t = __ldg(q + v);
        w[4 * v + 0] = t.x;
        w[4 * v + 1] = t.y;
        w[4 * v + 2] = t.z;
        w[4 * v + 3] = t.w;
    }
#pragma unroll
    for (int j = 0; j < kGroup; ++j) {
        // pixel j is bytes 3j .. 3j+2 of the group: word a = 3j / 4 from byte s
        const int a = (3 * j) >> 2, s = (3 * j) & 3;
        const uint32_t hi = w[a + 1 < 12 ? a + 1 : 11];
        key[j] = __byte_perm(w[a], hi, (unsigned)((s + 2) | ((s + 1) << 4) | (s << 8))) &
                 0xFFFFFFu;
    }
}

// Whether an image can take the vector path: base (and, if given, a second
// per-pixel byte array) 16-byte aligned.
__host__ __device__ __forceinline__ bool vector_ok(const void* rgb, const void* other) {
    return (((uintptr_t)rgb | (uintptr_t)other) & 15) == 0;
}

}  // namespace wsm
