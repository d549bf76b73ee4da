// wsm_split.h -- how the persistent Sort-Means launch divides its blocks
// between the images of a batch.  Shared by the host (launches whose sizes
// it knows) and the device (k_plan, from the device's N' values), and plain
// enough for the host C++ compiler, so that both derive the same split and
// the CPU tests can check it.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define WSM_HD __host__ __device__
#else
#define WSM_HD
#endif

namespace wsm {

constexpr int64_t kGroupFloor = 16;   // blocks an image's group gets before the split

// Blocks of one image's group: enough for every lane to hold a color and for
// every warp to hold a table row.
WSM_HD inline int64_t group_want(int64_t n, int K, int threads) {
    const int64_t warps = threads / 32;
    const int64_t for_colors = (n + threads - 1) / threads;
    const int64_t for_rows = (K + warps - 1) / warps;
    const int64_t w = for_colors > for_rows ? for_colors : for_rows;
    return w > 1 ? w : 1;
}

// An image's demand scaled by its work weight (1/1024 units; 0 leaves it
// as it is), at least one block.
WSM_HD inline int64_t weighted_want(int64_t want, int weight) {
    if (weight <= 0) return want;
    const int64_t v = want * weight / 1024;
    return v > 1 ? v : 1;
}

// Split `grid` blocks into one group per image: min(want, floor) each, the
// floor at most kGroupFloor and at most half of the grid over the images,
// the rest in proportion to each image's want beyond that (every image gets
// at least one; grid >= n_items), integer arithmetic only so that host and
// device derive the same split.  Returns the number of blocks used.
WSM_HD inline int split_groups(const int64_t* want, int n_items, int grid, int* first_blk) {
    int64_t total = 0;
    for (int i = 0; i < n_items; ++i) total += want[i];
    first_blk[0] = 0;
    if (total <= grid) {
        for (int i = 0; i < n_items; ++i) first_blk[i + 1] = first_blk[i] + (int)want[i];
        return first_blk[n_items];
    }
    // every image first gets min(want, floor) blocks: a small image's group
    // still has the warps for its row build and for the tail of its visits;
    // the floors take at most half of the grid, so that with many images the
    // large ones still get their share
    const int64_t half = (int64_t)grid / (2 * n_items) > 1 ? (int64_t)grid / (2 * n_items) : 1;
    const int64_t floor = half < kGroupFloor ? half : kGroupFloor;
    int64_t fixed = 0;
    for (int i = 0; i < n_items; ++i) fixed += want[i] < floor ? want[i] : floor;
    const int64_t left = grid - fixed, excess = total - fixed;
    int used = 0;
    for (int i = 0; i < n_items; ++i) {
        const int64_t f = want[i] < floor ? want[i] : floor;
        first_blk[i + 1] = (int)(f + left * (want[i] - f) / excess);   // g_i, for now
        used += first_blk[i + 1];
    }
    for (int i = 0; i < n_items && used < grid; ++i)   // the rounding remainder, in order
        if (first_blk[i + 1] < want[i]) {
            ++first_blk[i + 1];
            ++used;
        }
    for (int i = 0; i < n_items; ++i) first_blk[i + 1] += first_blk[i];
    return first_blk[n_items];
}

}  // namespace wsm
