/*
 * wsm.h -- C ABI of libwsm, a GB300 (sm_103a) implementation of Weighted
 * Sort-Means (WSM) color quantization (M. E. Celebi, "Fast Color
 * Quantization Using Weighted Sort-Means Clustering", arXiv:1011.0093).
 *
 * Problem (Sec. 1): an image of N pixels of 24-bit RGB is reduced to a
 * palette of K colors plus an index image.  The path is
 *   wsm_reduce      unique colors and their frequencies   (Sec. 2, data
 *                   sampling and sample weighting)
 *   wsm_init        K random unique colors as centers     (Algorithm 2,
 *                   first step; Sec. 3.2 random initialisation)
 *   wsm_iterate     the Sort-Means loop with weighted means and the
 *                   termination rule                      (Algorithm 2,
 *                   Sec. 3.2)
 *   wsm_map         final assignment and pixel mapping    (Sec. 1)
 *   wsm_distortion  mean squared error of the mapping     (Sec. 3.1, Eq. 2)
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: WSM_OK (0) or a negative
 *     WSM_E_* code.  No function aborts the process.  wsm_last_error()
 *     returns a message for the calling thread's last failure.
 *   - Pointers named d_* are device pointers to memory owned by the caller;
 *     the library never frees them and keeps no reference after a call
 *     returns.  Pointers without the prefix are host pointers.
 *   - A wsm_handle owns library scratch memory on the device that was
 *     current at wsm_create; every later call on it must run with that
 *     device current.  One handle serves one stream at a time: calls that
 *     share a handle must be ordered on the same stream (or synchronised).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *     are asynchronous on it unless they return a host value (documented
 *     per function), in which case they synchronise the stream.
 *   - Kernel-side failures (a grid barrier that waited too long, a label or
 *     palette index >= K in the input, more unique colors than the output
 *     can hold) are recorded in a per-handle status word; the next call that
 *     synchronises reports them (WSM_E_TIMEOUT, WSM_E_INVAL, WSM_E_CAPACITY)
 *     and clears the word.  wsm_sync_status() does so explicitly.
 *
 * Data layouts:
 *   pixels   uint8 [N][pixel_stride], pixel_stride 3 (R,G,B) or 4 (R,G,B,x;
 *            the fourth byte is ignored).
 *   colors   uint32 [N'] packed 0x00RRGGBB, strictly ascending.
 *   counts   uint32 [N'] pixel frequency of each color (w_i = n_i / N).
 *   centers  float32 [K][4] = (R, G, B, unused), the palette c_1..c_K.
 *   labels   uint8 [N'] membership m[i] in [0, K) of each unique color.
 *   index    uint8 [N] palette index of each pixel.
 * Limits: 1 <= K <= 256 (uint8 labels); N <= 2^24 pixels per image, which
 * keeps every per-cluster sum of n_i * x_i below 2^32.
 */
#ifndef WSM_H
#define WSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define WSM_API __attribute__((visibility("default")))
#else
#define WSM_API
#endif

typedef struct wsm_handle wsm_handle;
typedef struct CUstream_st* wsm_stream; /* same type as cudaStream_t */

enum {
    WSM_OK = 0,
    WSM_E_INVAL = -1,    /* bad argument, or a label / index >= K found on the device */
    WSM_E_NOMEM = -2,    /* device or host allocation failed */
    WSM_E_CUDA = -3,     /* a CUDA runtime call failed; see wsm_last_error() */
    WSM_E_TIMEOUT = -4,  /* a device-side wait gave up (bounded spin) */
    WSM_E_STATE = -5,    /* handle used on the wrong device, or destroyed */
    WSM_E_CAPACITY = -6  /* more unique colors than the output arrays hold */
};

#define WSM_MAX_K 256          /* largest palette with 8-bit memberships */
#define WSM_MAX_K_WIDE 1024    /* largest palette of a wide handle (16-bit memberships) */
#define WSM_MAX_PIXELS (1ll << 24)

/* Message describing the calling thread's most recent failure ("" if none).
 * The string stays valid until the thread's next libwsm call. */
WSM_API const char* wsm_last_error(void);

/* Create a handle for images of at most max_pixels pixels, at most
 * max_unique unique colors and palettes of at most max_K colors, on the
 * current device.  Allocates the scratch: a 2^24-bin uint32 color histogram
 * (64 MiB) with a one-bit-per-bin occupancy map (2 MiB), a 2^24-entry
 * color->label table (16 MiB), the max_K x max_K sorted center tables and
 * the reduction and barrier words.
 * Label width: with max_K <= 256 (WSM_MAX_K) every membership (d_labels),
 * palette index (d_index) and table entry is a uint8; a handle with
 * 256 < max_K <= 1024 (WSM_MAX_K_WIDE) is wide: they are uint16, and the
 * calls that take d_labels or d_index read and write uint16 arrays (the
 * pointer types below are void* for that reason).  The gradient calls, the
 * server and wsm_iterate_noalloc keep palettes of at most 256 colors.
 * Errors: WSM_E_INVAL (limits out of range), WSM_E_NOMEM, WSM_E_CUDA.  *h
 * is NULL on failure. */
WSM_API int wsm_create(wsm_handle** h, int max_K, int64_t max_pixels, int64_t max_unique);

/* Free the handle and its scratch (synchronises the device first).
 * NULL is accepted.  Errors: none (always WSM_OK); a handle must be freed
 * once. */
WSM_API int wsm_destroy(wsm_handle* h);

/* Read, report and clear the handle's device status word (synchronises
 * `stream`).  Returns WSM_OK if no kernel-side failure was recorded.
 * Errors: the recorded failure -- WSM_E_TIMEOUT (a grid barrier gave up),
 * WSM_E_CAPACITY (more unique colors than the outputs hold), WSM_E_INVAL
 * (an image with N' < K was skipped, or a membership / index >= K was
 * found); WSM_E_INVAL (NULL handle), WSM_E_STATE (wrong device),
 * WSM_E_CUDA (the read failed). */
WSM_API int wsm_sync_status(wsm_handle* h, wsm_stream stream);

/* Sec. 2, data sampling + sample weighting.  The unique colors of the
 * image and their pixel counts: d_colors[0..N') ascending, d_counts[i] the
 * number of pixels of color d_colors[i].  The paper uses a chained hash
 * table; this builds a 2^24-bin count histogram with warp-aggregated atomics
 * and compacts it with a prefix scan over the occupancy map, which yields
 * the same set already in ascending order, and leaves the histogram zeroed
 * for the next image.
 *   d_rgb        [n_pixels][pixel_stride] uint8, 0 <= n_pixels <= max_pixels
 *   d_colors,
 *   d_counts     [capacity] each; capacity >= N' or WSM_E_CAPACITY
 *   d_n_unique   device int64, receives N' (may be NULL)
 *   n_unique     host int64, receives N' (may be NULL; if given, the call
 *                synchronises `stream`; otherwise it is asynchronous)
 * Errors: WSM_E_INVAL (sizes, stride), WSM_E_CAPACITY (N' > capacity: the
 * first `capacity` colors are written, the histogram is still cleared). */
WSM_API int wsm_reduce(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels, int pixel_stride,
               uint32_t* d_colors, uint32_t* d_counts, int64_t capacity,
               int64_t* d_n_unique, int64_t* n_unique, wsm_stream stream);

/* Algorithm 2, first step: the initial centers are K distinct unique
 * colors chosen at random (Sec. 3.2 uses random initialisation).  The
 * indices are drawn on the host with Floyd's sampling algorithm (Bentley &
 * Floyd 1987) from the counter-based splitmix64 stream of `seed` (draw r =
 * mix(seed + (r+1) * 0x9E3779B97F4A7C15), Steele et al. 2014; draw r picks
 * t uniformly in [0, j] by t = draw mod (j+1)), sorted ascending, and
 * gathered on the device: d_centers[k] = unpack(d_colors[idx_k]).  Every
 * membership starts at 0: d_labels[i] = 0.  Asynchronous.
 *   d_colors   [n_unique]; d_centers [K][4] out; d_labels [n_unique] out
 * Errors: WSM_E_INVAL (K < 1, K > max_K, K > n_unique). */
WSM_API int wsm_init(wsm_handle* h, const uint32_t* d_colors, int64_t n_unique, int K,
                     uint64_t seed, float* d_centers, void* d_labels, wsm_stream stream);

/* Algorithm 2 with the Sec. 3.2 termination rule, in one persistent
 * cooperative launch.  Each iteration: the K x K squared center distances
 * d[p][j] and, per row p, the centers sorted by (d[p][j], j != p, j); then
 * the pruned nearest-center search of every unique color starting from its
 * previous membership p, which stops at the first center t of row p with
 * d[p][t] >= 4 ||x_i - c_p||^2 and moves to a visited center when its
 * distance is <= the running minimum; then the weighted means
 * c_k = sum n_i x_i / sum n_i over m[i] = k, with exact integer sums and an
 * empty cluster keeping its center.  SSE_i = sum_i (n_i / N) min_dist_i is
 * taken in the assignment step of iteration i.
 *   max_iter   >= 0 iterations at most
 *   eps        > 0: WSM-C, stop after iteration i >= 2 once
 *              (SSE_{i-1} - SSE_i) / SSE_i <= eps, or when SSE_i = 0;
 *              <= 0: WSM, exactly max_iter iterations
 *   d_centers  [K][4] in: current centers, out: centers after the last update
 *   d_labels   [n_unique] in: memberships (each < K), out: the last assignment
 *   iters_done host int (may be NULL), sse_trace host double [max_iter]
 *              (may be NULL); if either is given the call synchronises.
 * Distances are FP32 on CUDA cores in difference form; sums are integers.
 * Errors: WSM_E_INVAL (K, sizes; label >= K found), WSM_E_TIMEOUT. */
WSM_API int wsm_iterate(wsm_handle* h, const uint32_t* d_colors, const uint32_t* d_counts,
                int64_t n_unique, int K, float* d_centers, void* d_labels, int max_iter,
                double eps, int* iters_done, double* sse_trace, wsm_stream stream);

/* Diagnostics of the last wsm_iterate on this handle, valid until the next
 * wsm_iterate or wsm_map on it (synchronises):
 * evaluated = number of distances ||x_i - c_k||^2 computed, summed over all
 * colors and iterations (one per color for the previous center plus one per
 * visited center); S [K][3] and W [K] (may be NULL) = the integer sums
 * sum n_i x_i and sum n_i of the last update.
 * evaluated may be NULL too.  Errors: WSM_E_INVAL (K out of [1, max_K]),
 * WSM_E_STATE (S or W asked for before any completed iteration, wrong
 * device), WSM_E_CUDA. */
WSM_API int wsm_iterate_stats(wsm_handle* h, int K, int64_t* evaluated, int64_t* S, int64_t* W,
                      wsm_stream stream);

/* One image of a batch call; fields as for the single-image calls.  Which
 * fields each batch call reads (r) or writes (w):
 *   wsm_reduce_batch      d_rgb n_pixels pixel_stride (r); d_colors d_counts
 *                         (w, device memory of n_pixels entries each);
 *                         n_unique (w, host)
 *   wsm_init_batch        K d_colors n_unique (r); d_centers d_labels (w)
 *   wsm_iterate_batch     K d_colors d_counts n_unique (r); d_centers d_labels (rw)
 *   wsm_map_batch         every field but d_counts (r); d_labels d_index (w)
 *   wsm_distortion_batch  d_rgb n_pixels pixel_stride K d_centers d_index (r) */
typedef struct {
    const uint8_t* d_rgb;       /* [n_pixels][pixel_stride] */
    int64_t n_pixels;
    int pixel_stride;           /* 3 or 4 */
    int K;                      /* 1 <= K <= max_K */
    uint32_t* d_colors;         /* [n_unique] ascending (written by wsm_reduce_batch) */
    uint32_t* d_counts;         /* [n_unique] (written by wsm_reduce_batch) */
    int64_t n_unique;
    float* d_centers;           /* [K][4], 16-byte aligned */
    void* d_labels;             /* [n_unique] uint8 (uint16 with a wide handle) */
    void* d_index;              /* [n_pixels] uint8 (uint16 with a wide handle) */
} wsm_item;

/* Reserve per-image scratch for batches of up to max_items images (about
 * 17.2 MiB each at max_K = 256, dominated by the color->label table), plus
 * the unique-color reduction scratch of min(max_items, 16) images (66 MiB
 * each: the 2^24-bin histogram and its occupancy map).  Synchronises the
 * device.  A new handle has one slot.
 * Errors: WSM_E_INVAL, WSM_E_NOMEM (the handle keeps one slot). */
WSM_API int wsm_reserve_batch(wsm_handle* h, int max_items);

/* Algorithm 2 with the Sec. 3.2 termination rule for n_items independent
 * images in one persistent cooperative launch per 64 images: the blocks are
 * split into one group per image (in proportion to its unique colors and
 * palette size), each group iterating its image exactly as wsm_iterate would
 * (same results, bit for bit) with a barrier of its own, so images of
 * different sizes and iteration counts share the launch.  Each item needs
 * d_colors, d_counts, n_unique, K, d_centers, d_labels.
 *   iters_done  host int [n_items] (may be NULL; if given, synchronises)
 * Errors: WSM_E_INVAL (item sizes, more items than reserved slots),
 * WSM_E_TIMEOUT. */
WSM_API int wsm_iterate_batch(wsm_handle* h, const wsm_item* items, int n_items, int max_iter,
                              double eps, int* iters_done, wsm_stream stream);

/* Sec. 2, unique colors and their counts for n_items images, as wsm_reduce
 * gives them one by one (same output), in one launch of each reduction
 * kernel per 16 images and one device synchronisation for the whole batch.
 * On success items[i].n_unique holds N' of image i; its d_colors and
 * d_counts hold N' entries (ascending colors) and must have room for
 * n_pixels.  1 <= n_pixels <= max_pixels.
 * Errors: WSM_E_INVAL (sizes, pointers, more items than reserved slots). */
WSM_API int wsm_reduce_batch(wsm_handle* h, wsm_item* items, int n_items, wsm_stream stream);

/* Algorithm 2, first step, for n_items images, as wsm_init would do them
 * one by one with seeds[i] (same centers and labels): the host draws every
 * image's K indices (Floyd sampling of splitmix64 draws), one copy moves
 * them to the device and one launch per 64 images gathers the centers and
 * zeroes the labels.  seeds: host uint64 [n_items].  Waits, on the host,
 * only for the previous call's index copy.
 * Errors: WSM_E_INVAL (K, n_unique < K, pointers, more items than slots). */
WSM_API int wsm_init_batch(wsm_handle* h, const wsm_item* items, int n_items,
                           const uint64_t* seeds, wsm_stream stream);

/* Eq. 2 for n_items images, as wsm_distortion gives them one by one (same
 * values: the sum is exact in 2^-20 units whatever the block split), in one
 * pair of launches per 64 images.
 *   d_mse  device double [n_items] (may be NULL)
 *   mse    host double [n_items] (may be NULL; if given, synchronises and
 *          reports a palette index >= K as WSM_E_INVAL)
 * Errors: WSM_E_INVAL (sizes, pointers, more items than reserved slots). */
WSM_API int wsm_distortion_batch(wsm_handle* h, const wsm_item* items, int n_items,
                                 double* d_mse, double* mse, wsm_stream stream);

/* Sec. 1, pixel mapping for n_items images: one final pruned assignment per
 * image in one persistent launch (as wsm_map), then one gather launch over
 * all images' pixels.  Each item needs every field but d_counts.
 * Errors: as wsm_map. */
WSM_API int wsm_map_batch(wsm_handle* h, const wsm_item* items, int n_items, wsm_stream stream);

/* Allocation-free variant of wsm_iterate.  The paper has no counterpart:
 * it exists for callers that cannot call cudaMalloc -- a plugin inside a
 * host program that owns every device byte through its own pool, a process
 * whose device memory is already fully reserved by another framework's
 * caching allocator, or a latency-critical loop that cannot afford the
 * implicit device synchronisation of an allocation.  It needs no handle and
 * allocates nothing: the caller passes the inputs and outputs exactly as for
 * wsm_iterate (same meaning, layout and results), and the kernel's scratch
 * (sorted center tables, cluster sums, SSE partials and trace, barrier
 * words) lives in one file-scope device array of about 1.2 MiB that every
 * GPU which loads libwsm keeps until the process exits.
 *   - Limits: 1 <= K <= 256, 1 <= n_unique <= 2^24, 0 <= max_iter <= 4096;
 *     larger sizes are rejected with WSM_E_INVAL and a message.
 *   - The first call on each device looks up the array's device address and
 *     the kernel's co-resident grid for that device (with that device
 *     current); make that first call before any stream capture begins.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; each call clears the words that must start at zero.  Calls
 *     whose executions overlap on the GPU (other streams, other host
 *     threads) race on the array and give wrong results: order them.
 *   - iters_done / sse_trace as for wsm_iterate.  If either is given, the
 *     call synchronises and reports device-side failures (a barrier timeout,
 *     a label >= K).  If neither is given, the call is asynchronous and
 *     reports none: the failure stays recorded in the array and the next
 *     call on this device that passes iters_done or sse_trace reports it
 *     (and clears the record).
 *   - Handles created or destroyed before or after a call (of any palette
 *     size) do not affect it: the kernel's shared-memory limit on a device
 *     is only ever raised.
 * Errors: WSM_E_INVAL (limits above, NULL pointers, centers not 16-byte
 * aligned, a label >= K found), WSM_E_TIMEOUT, WSM_E_CUDA. */
WSM_API int wsm_iterate_noalloc(const uint32_t* d_colors, const uint32_t* d_counts,
                                int64_t n_unique, int K, float* d_centers, uint8_t* d_labels,
                                int max_iter, double eps, int* iters_done, double* sse_trace,
                                wsm_stream stream);

/* Sec. 1, pixel mapping.  One more pruned assignment of the unique colors
 * against d_centers (starting from d_labels, which it updates), a scatter
 * of the memberships into the handle's 2^24-entry color->label table, and
 * a gather d_index[p] = table[color of pixel p].  d_colors must be the
 * unique colors of these same pixels.  Asynchronous.
 * Errors: WSM_E_INVAL (sizes, K; label >= K found), WSM_E_TIMEOUT. */
WSM_API int wsm_map(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels, int pixel_stride,
            const uint32_t* d_colors, int64_t n_unique, const float* d_centers, int K,
            void* d_labels, void* d_index, wsm_stream stream);

/* Sec. 3.1, Eq. 2: MSE = (1/N) sum_p ||x_p - c_{index_p}||^2 over the three
 * channels.  Each pixel's squared distance (FP32, difference form) is
 * truncated to units of 2^-20 and summed as an integer, so the result does
 * not depend on the order of the additions (deterministic).  K may be up to
 * 256 (1024 with a wide handle, whose d_index is uint16), whatever max_K.
 *   d_mse  device double (may be NULL); mse host double (may be NULL; if
 *          given, the call synchronises).
 * Errors: WSM_E_INVAL (sizes, K; index >= K found). */
WSM_API int wsm_distortion(wsm_handle* h, const uint8_t* d_rgb, int64_t n_pixels, int pixel_stride,
                   const float* d_centers, int K, const void* d_index, double* d_mse,
                   double* mse, wsm_stream stream);

/* Sec. 3.1: the palette as 8-bit colors.  Every FP32 center coordinate is
 * rounded to the nearest integer, ties to even, and clamped to [0, 255].
 * A quantized image stores such colors; the paper does not say whether its
 * MSE uses them, so wsm_distortion on the FP32 centers gives the primary
 * MSE and wsm_distortion on d_rounded the MSE of the 8-bit palette.
 *   d_centers  device float [K][4] (x, y, z, unused), 16-byte aligned
 *   d_palette  device uint8 [K][4] out (R, G, B, 0), may be NULL
 *   d_rounded  device float [K][4] out (the same colors as floats, 4th 0),
 *              16-byte aligned, may be NULL
 * Asynchronous.  Errors: WSM_E_INVAL (K out of [1, 256], or [1, 1024] with a
 * wide handle; null or unaligned pointers). */
WSM_API int wsm_round_palette(wsm_handle* h, const float* d_centers, int K, uint8_t* d_palette,
                              float* d_rounded, wsm_stream stream);

/* Measured FP32 throughput of this GPU, for the roofline of the assignment
 * kernel (not part of the method): a kernel of independent FMA chains, 8
 * blocks of 256 threads per SM, timed with CUDA events (best of `repeats`
 * after one untimed launch).  Synchronises the stream.
 *   tflops  host out: FP32 TFLOP/s (one FMA = 2 FLOP)
 * Errors: WSM_E_INVAL (repeats out of [1, 20]), WSM_E_CUDA. */
WSM_API int wsm_measure_fp32(wsm_handle* h, int repeats, double* tflops, wsm_stream stream);

/* The whole path -- Sec. 2 unique colors, Algorithm 2 (initialisation,
 * Sort-Means iterations with the Sec. 3.2 stop rule), Sec. 1 final
 * assignment and pixel mapping, Eq. 2 MSE -- for n_items images, with no
 * host synchronisation: N' of each image stays on the device (the
 * initialisation draws its Floyd sample there, the persistent launches split
 * their blocks there).  The call only enqueues work, so it can be captured
 * into a CUDA graph (cudaStreamBeginCapture on `stream`) and replayed.
 * Results equal those of wsm_reduce, wsm_init(seeds[i]), wsm_iterate,
 * wsm_map and wsm_distortion image by image, bit for bit.
 * Each item needs d_rgb, n_pixels, pixel_stride, K and device buffers with
 * room for n_pixels entries in d_colors, d_counts and d_labels, [K][4]
 * d_centers and [n_pixels] d_index; n_unique is not read.
 *   seeds       host uint64 [n_items]
 *   d_n_unique  device int64 [n_items] (may be NULL): N'
 *   d_iters     device int [n_items] (may be NULL): iterations run
 *   d_mse       device double [n_items] (may be NULL): MSE
 * An image with N' < K is skipped and reported (WSM_E_INVAL) at the next
 * synchronising call, e.g. wsm_sync_status.
 * Errors: WSM_E_INVAL (sizes, pointers, more items than reserved slots). */
WSM_API int wsm_quantize_batch(wsm_handle* h, const wsm_item* items, int n_items,
                               const uint64_t* seeds, int max_iter, double eps,
                               int64_t* d_n_unique, int* d_iters, double* d_mse,
                               wsm_stream stream);

/* The stages of wsm_quantize_batch, for wsm_quantize_batch_stages. */
enum {
    WSM_STAGE_REDUCE = 1,      /* Sec. 2 unique colors (writes N' on the device) */
    WSM_STAGE_INIT = 2,        /* Algorithm 2 initialisation (needs REDUCE before) */
    WSM_STAGE_ITERATE = 4,     /* Sort-Means iterations, Sec. 3.2 stop rule; d_n_unique, d_iters */
    WSM_STAGE_MAP = 8,         /* final assignment: unique colors' labels, color->label table */
    WSM_STAGE_INDEX = 32,      /* pixel mapping: the index image (needs MAP before) */
    WSM_STAGE_DISTORTION = 16, /* Eq. 2 MSE from the final assignment; d_mse (needs MAP) */
    WSM_STAGE_ALL = 63
};

/* The stages of wsm_quantize_batch named by the `stages` bits, in the order
 * listed above (INDEX before DISTORTION), on the device state the earlier
 * stages left (the handle's N' values, the items' buffers, the squared-error
 * sum of the last final assignment).  Running the stages in several calls,
 * e.g. to time them or to capture each into its own CUDA graph, gives
 * exactly the results of one wsm_quantize_batch call.  DISTORTION reads no
 * pixels: the final assignment (MAP) sums, over the unique colors,
 * count x squared distance to the assigned center with each pixel's term
 * truncated to 2^-20 as wsm_distortion truncates it, so the MSE equals
 * wsm_distortion's on the index image bit for bit.
 * Errors: as wsm_quantize_batch; WSM_E_INVAL for unknown stage bits. */
WSM_API int wsm_quantize_batch_stages(wsm_handle* h, const wsm_item* items, int n_items,
                                      const uint64_t* seeds, int max_iter, double eps,
                                      int64_t* d_n_unique, int* d_iters, double* d_mse,
                                      unsigned stages, wsm_stream stream);

/* Counters of the last persistent launch over image slots 0..n_items-1
 * (an iterate launch, or the final assignment of a mapping, which resets
 * them): distances evaluated (1 + visited row entries per color and pass)
 * and iterations run.  Synchronises the stream.
 *   evaluated  host int64 [n_items] (may be NULL); iters host int [n_items]
 *              (may be NULL)
 * Errors: WSM_E_INVAL (n_items > reserved slots), or a pending device error. */
WSM_API int wsm_batch_stats(wsm_handle* h, int n_items, int64_t* evaluated, int* iters,
                            wsm_stream stream);

/* Self-test of failure detection: two blocks wait at a device barrier that
 * waits for three, so the wait runs out after limit_ms (1..2000); the
 * kernel records the timeout in the status word and returns, as the
 * persistent kernel's barriers do (their limit is 2 s).  Synchronises.
 * Returns WSM_E_TIMEOUT when the detection works; the handle stays usable.
 * Errors: WSM_E_INVAL (limit), WSM_E_CUDA. */
WSM_API int wsm_selftest_barrier_timeout(wsm_handle* h, int limit_ms, wsm_stream stream);

/* Launch shapes of the persistent Sort-Means kernel (no counterpart in the
 * paper: a GPU launch parameter).  Shape s = (threads per block, blocks per
 * SM); the persistent launches of the handle use its current shape.  Every
 * shape gives the same results bit for bit.
 * wsm_launch_shape: shape s (or, for s < 0, the current one) -> *threads,
 * *blocks_per_sm, *resident (1 if all its blocks fit on the GPU at this
 * handle's max_K); returns s (>= 0) or an error code.
 * wsm_set_launch_shape: makes s current.  Errors: WSM_E_INVAL (out of range,
 * not resident). */
WSM_API int wsm_launch_shape(wsm_handle* h, int shape, int* threads, int* blocks_per_sm,
                             int* resident);
WSM_API int wsm_set_launch_shape(wsm_handle* h, int shape);

/* How the first pass of each iterate launch searches (no counterpart in the
 * paper: it changes the work, not the outcome).  candidate = 1 (default):
 * each color's search starts at the center nearest to its 16^3 cell of the
 * RGB cube (found once per launch) and visits that center's row up to the
 * triangle-inequality bound; the winner is the one Algorithm 2's visit of
 * row m[i] would keep (equal distances: the latest in that row), and the
 * visit of row m[i] itself is made whenever that winner would not be on it.
 * The memberships, sums and SSE are those of Algorithm 2; far fewer
 * distances are computed when the memberships are far off (all 0 after the
 * initialisation).  candidate = 0: every pass visits row m[i] as Algorithm 2
 * does (the distance counts of wsm_iterate_stats are then Algorithm 2's).
 * Errors: WSM_E_STATE (wrong device). */
WSM_API int wsm_set_first_pass_start(wsm_handle* h, int candidate);

/* How the handle's unique-color reductions fill their histogram (Sec. 2,
 * data sampling; both give the same colors and counts bit for bit):
 *   0  by size (default): bucketed when a launch has at least 2^24 pixels
 *      in all and 2^21 per image on average, direct otherwise;
 *   1  direct: one global atomic per pixel into the 2^24-bin histogram (lanes
 *      of a warp with the same color combined);
 *   2  bucketed: pixels grouped by the top 10 bits of their color, then each
 *      group counted in a shared-memory histogram and flushed once.
 * Errors: WSM_E_INVAL (path not 0, 1 or 2), WSM_E_STATE (wrong device). */
WSM_API int wsm_set_reduce_path(wsm_handle* h, int path);

/* Limits every persistent launch of the handle to `blocks` blocks (0: the
 * whole co-resident grid of its shape), so that several handles on several
 * streams can run their persistent launches side by side on one GPU.
 * Errors: WSM_E_INVAL (0 < blocks < 48). */
WSM_API int wsm_set_grid_limit(wsm_handle* h, int blocks);

/* Autotuner: runs the unique-color reduction of the batch once, then for
 * every resident shape `repeats` times the initialisation (untimed) and the
 * Sort-Means iterations (timed with CUDA events on `stream`), and makes the
 * fastest shape current.  Then, with that shape, it runs the iterations
 * six more times to weigh the images: each image's group of blocks is
 * timed on the device, and the image's share of the persistent launch's
 * blocks is scaled by its time over the mean time, so that the groups end
 * together.  The weights stay with the handle's image slots and apply to
 * its later device-sized launches of the iterations (wsm_quantize_batch and
 * its stages); they only move blocks between images, and every split gives
 * the same results bit for bit.  Synchronises.  Items as for
 * wsm_quantize_batch; their centers and labels end as one complete run
 * leaves them.
 *   times_ms  host float [5] (may be NULL): best time of each shape, -1 if
 *             not resident
 * Returns the chosen shape (>= 0; with n_items = 0 the current one, nothing
 * run) or an error code: WSM_E_INVAL (repeats out of [1, 100], items as for
 * wsm_quantize_batch), WSM_E_TIMEOUT, WSM_E_CUDA. */
WSM_API int wsm_autotune_batch(wsm_handle* h, const wsm_item* items, int n_items,
                               const uint64_t* seeds, int max_iter, double eps, int repeats,
                               float* times_ms, wsm_stream stream);

/* The second half of wsm_autotune_batch alone: with the handle's current
 * launch shape (wsm_set_launch_shape), run the reduction once and the
 * iterations six times, and set the images' work weights from the timed
 * groups.  For a caller that fixes the shape itself.  Synchronises.  Items
 * as for wsm_quantize_batch; their centers and labels end as one complete
 * run leaves them.
 * Errors: WSM_E_INVAL (items as for wsm_quantize_batch), WSM_E_TIMEOUT,
 * WSM_E_CUDA. */
WSM_API int wsm_weigh_batch(wsm_handle* h, const wsm_item* items, int n_items,
                            const uint64_t* seeds, int max_iter, double eps, wsm_stream stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of quantization requests (no counterpart in
 * the paper, which quantizes one image at a time).  A server owns `lanes`
 * lanes -- each a stream, a handle limited to 1/lanes of the SMs and up to
 * slots_per_lane images per batch -- and a device arena of arena_bytes for
 * the requests' buffers.  A scheduler thread admits queued requests first
 * come, first served, into idle lanes while slots and arena memory allow
 * (a request needs about 14 bytes per pixel, see wsm_server_submit), runs
 * each lane's batch as wsm_quantize_batch with the copies in and out on the
 * lane's stream, and completes the requests when the lane's event fires.
 * Lanes overlap on the device; a request's results are the same alone and
 * in any mix (the per-image computation does not depend on the batch).
 * ------------------------------------------------------------------------- */
typedef struct wsm_server wsm_server;

typedef struct {
    int max_K;               /* 1..256 */
    int64_t max_pixels;      /* per request, 1..2^24 */
    int lanes;               /* 1..8 */
    int slots_per_lane;      /* 1..64 */
    int64_t arena_bytes;     /* device memory for the requests' buffers */
} wsm_server_config;

typedef struct {
    const uint8_t* rgb;      /* host [n_pixels][pixel_stride]; page-locked for overlap */
    int64_t n_pixels;
    int pixel_stride;        /* 3 or 4 */
    int K;
    uint64_t seed;           /* initialisation seed (as wsm_init) */
    int max_iter;            /* requests with other (max_iter, eps) go to other batches */
    double eps;
    uint8_t* index_out;      /* host [n_pixels] (may be NULL); page-locked for overlap */
    float* palette_out;      /* host [K][4] (may be NULL); page-locked for overlap */
} wsm_request;

typedef struct {
    int status;              /* WSM_OK, or the request's error (N' < K: WSM_E_INVAL) */
    int iters;
    int64_t n_unique;
    double mse;
    double t_submit, t_admit, t_done;   /* steady-clock seconds */
} wsm_result;

typedef struct {
    int64_t submitted, completed, failed, batches;
    int64_t in_flight, max_in_flight, queued;
    int64_t arena_bytes, arena_used, arena_peak;
} wsm_server_stats;

/* Creates the lanes, the arena and the scheduler thread on the current
 * device.  Errors: WSM_E_INVAL (config), WSM_E_NOMEM, WSM_E_CUDA. */
WSM_API int wsm_server_create(wsm_server** out, const wsm_server_config* cfg);

/* Queues a request (thread-safe, does not block).  The host buffers must
 * stay valid until wsm_server_wait returns for it.  Footprint in the arena:
 * the pixels, 4 + 4 bytes per pixel for colors and counts, 1 + 1 for labels
 * and index, 16 K for the palette, each rounded up to 256 bytes.
 * Errors: WSM_E_INVAL (sizes), WSM_E_CAPACITY (footprint > arena),
 * WSM_E_STATE (shutting down). */
WSM_API int wsm_server_submit(wsm_server* s, const wsm_request* r, uint64_t* id);

/* Waits for request `id` (timeout_s < 0: no limit) and returns its result;
 * the id is then forgotten.  The index image and palette are in the
 * request's output buffers.  Returns the request's status, WSM_E_TIMEOUT if
 * it is not done in time (it stays queued), WSM_E_INVAL for an unknown id. */
WSM_API int wsm_server_wait(wsm_server* s, uint64_t id, double timeout_s, wsm_result* res);

/* Counters of the server since its creation (a consistent snapshot).
 * Errors: WSM_E_INVAL (NULL argument). */
WSM_API int wsm_server_stats_get(wsm_server* s, wsm_server_stats* st);

/* Completes every queued request, then frees the server.  NULL is accepted.
 * Errors: none (always WSM_OK). */
WSM_API int wsm_server_destroy(wsm_server* s);

/* The weighted distortion of Eq. 1 (the k-means objective) with the sample
 * weights of Sec. 2, as a differentiable function of the palette C and of
 * the points X:  D(C, X) = sum_i w_i min_k ||x_i - c_k||^2.  Forward pass:
 * each point's nearest center m_i by the pruned search of Algorithm 2
 * (Sec. 2), starting at d_assign[i] if warm_start (else at center 0), over
 * full sorted rows of C; among equal distances the center visited last wins.
 *   d_x       device float [n][x_stride] (x_stride 3 or 4; a 4th value is ignored)
 *   d_w       device float [n] weights, or NULL for w_i = 1/n
 *   d_centers device float [K][c_stride] (c_stride 3 or 4), 1 <= K <= max_K
 *   d_assign  device uint8 [n]: in, the starting centers (if warm_start,
 *             each < K); out, m_i
 *   d_D       device float [1]: D
 *   d_resid   device float [K][4], 16-byte aligned: (R_k, W_k) with
 *             R_k = sum_{m_i = k} w_i (x_i - c_k), W_k = sum_{m_i = k} w_i;
 *             the input of wsm_distortion_bwd
 * All sums are FP32 in a fixed order (identical results run to run).  n may
 * be 0 (D = 0).  Asynchronous.  Uses the handle's gradient scratch: calls on
 * one handle must be ordered on one stream.
 * Errors: WSM_E_INVAL (strides, K, n > 2^31, pointers; a starting center
 * >= K is reported at the next synchronising call). */
WSM_API int wsm_distortion_fwd(wsm_handle* h, const float* d_x, int x_stride, const float* d_w,
                               int64_t n, const float* d_centers, int c_stride, int K,
                               uint8_t* d_assign, int warm_start, float* d_D, float* d_resid,
                               wsm_stream stream);

/* Backward pass of wsm_distortion_fwd for the upstream gradient g = *d_gD
 * (device float [1]), away from ties (where D is differentiable):
 *   d_gC  device float [K][c_stride] (may be NULL): -2 g R_k (0 in a 4th column)
 *   d_gX  device float [n][x_stride] (may be NULL): 2 g w_i (x_i - c_{m_i})
 * with d_assign and d_resid from the forward pass on the same d_x, d_w and
 * d_centers.  Asynchronous.
 * Errors: as wsm_distortion_fwd. */
WSM_API int wsm_distortion_bwd(wsm_handle* h, const float* d_x, int x_stride, const float* d_w,
                               int64_t n, const float* d_centers, int c_stride, int K,
                               const uint8_t* d_assign, const float* d_resid, const float* d_gD,
                               float* d_gC, float* d_gX, wsm_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* WSM_H */
