/*
 * wsm_oracle.c -- plain, slow, single-threaded FP64 reference of Weighted
 * Sort-Means (WSM) color quantization, written from M. E. Celebi, "Fast Color
 * Quantization Using Weighted Sort-Means Clustering" (arXiv:1011.0093).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  It shares no code,
 * header, table or helper with the CUDA library, and the library never calls
 * it.  Every function follows the paper's steps in the paper's order and
 * notation; the section, algorithm or equation it follows is named above it.
 *
 * Readings where the paper is silent (each stated below):
 *   R1  init: the random initial centers are K distinct indices into the
 *       unique color list, drawn with Floyd's sampling algorithm (Bentley & Floyd,
 *       CACM 1987) from a counter-based splitmix64 stream (Steele et al.,
 *       2014), then sorted ascending; initial memberships m[i] = 0.
 *   R2  the row sort of M breaks ties by the key (d, j != p, j): row p starts
 *       with p itself, equal distances follow in index order.
 *   R3  an empty cluster keeps its previous center.
 *   R4  SSE_i is the weighted distortion sum_i w_i min_dist_i measured in the
 *       assignment step of iteration i; WSM-C stops after iteration i >= 2
 *       when (SSE_{i-1} - SSE_i) / SSE_i <= eps, or when SSE_i = 0.
 *   R5  the final palette is the float centers; pixels are mapped after one
 *       more pruned assignment against them.
 *   R6  Algorithm 1's argmin resolves ties to the lowest center index.
 *
 * Build: cc -std=c11 -O2 -ffp-contract=off -shared -fPIC (no fused
 * multiply-add, so x86 and Arm hosts give identical results).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Sec. 2 "Data sampling": only the pixels with unique colors are sampled.  */
/* The paper finds them with a chained hash table; the set it produces is   */
/* the same as sorting the packed 24-bit keys and collapsing equal runs,    */
/* which is what this plain version does.  "Sample weighting": the weight   */
/* of a color is proportional to its frequency, so the run length (the      */
/* number of pixels with that color) is returned with it.                   */
/* ------------------------------------------------------------------------ */
static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

int64_t wsmo_unique(const uint8_t* rgb, int64_t n_pixels, int stride,
                    uint32_t* colors, uint32_t* counts) {
    if (n_pixels < 0 || (stride != 3 && stride != 4)) return -1;
    if (n_pixels == 0) return 0;
    uint32_t* keys = (uint32_t*)malloc((size_t)n_pixels * sizeof(uint32_t));
    if (!keys) return -2;
    for (int64_t p = 0; p < n_pixels; ++p) {
        const uint8_t* px = rgb + p * stride;
        keys[p] = ((uint32_t)px[0] << 16) | ((uint32_t)px[1] << 8) | (uint32_t)px[2];
    }
    qsort(keys, (size_t)n_pixels, sizeof(uint32_t), cmp_u32);
    int64_t n_unique = 0;
    for (int64_t p = 0; p < n_pixels; ++p) {
        if (p == 0 || keys[p] != keys[p - 1]) {
            colors[n_unique] = keys[p];
            counts[n_unique] = 1;
            ++n_unique;
        } else {
            counts[n_unique - 1] += 1;
        }
    }
    free(keys);
    return n_unique;
}

/* Color x_i of the unique list as a point of R^3 (R, G, B). */
static void unpack(uint32_t c, double x[3]) {
    x[0] = (double)((c >> 16) & 255u);
    x[1] = (double)((c >> 8) & 255u);
    x[2] = (double)(c & 255u);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, first step: the initial centers are K of the unique colors */
/* chosen at random (reading R1).                                           */
/* ------------------------------------------------------------------------ */

/* splitmix64 draw number i (0-based) of the stream seeded with `seed`:
 * the generator adds the golden-ratio increment to its state once per draw
 * and returns the state passed through its mixing function. */
uint64_t wsmo_splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* Floyd's algorithm: for j = N'-K .. N'-1 draw t uniformly in [0, j]; take t
 * unless it was taken already, in which case take j.  Draw number r is used
 * for the r-th step.  Every K-subset is equally likely. */
int wsmo_init_indices(int64_t n_unique, int K, uint64_t seed, int64_t* idx) {
    if (K < 1 || (int64_t)K > n_unique) return -1;
    int taken = 0;
    for (int64_t j = n_unique - K; j < n_unique; ++j) {
        uint64_t t = wsmo_splitmix64(seed, (uint64_t)taken) % (uint64_t)(j + 1);
        int dup = 0;
        for (int q = 0; q < taken; ++q)
            if (idx[q] == (int64_t)t) { dup = 1; break; }
        idx[taken++] = dup ? j : (int64_t)t;
    }
    qsort(idx, (size_t)K, sizeof(int64_t), cmp_i64);
    return 0;
}

/* c_k = x_{idx_k}; m[i] = 0 for every i (reading R1). */
void wsmo_init_centers(const uint32_t* colors, int64_t n_unique, const int64_t* idx,
                       int K, double* centers, int32_t* labels) {
    for (int k = 0; k < K; ++k) unpack(colors[idx[k]], centers + 3 * k);
    for (int64_t i = 0; i < n_unique; ++i) labels[i] = 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, loop body.                                                  */
/* ------------------------------------------------------------------------ */

static double sqdist(const double a[3], const double b[3]) {
    double e0 = a[0] - b[0], e1 = a[1] - b[1], e2 = a[2] - b[2];
    return e0 * e0 + e1 * e1 + e2 * e2;
}

/* Algorithm 2, start of each pass: the symmetric table of squared
 * center-to-center distances d[i][j] = ||c_i - c_j||^2, filled from the
 * upper triangle, zero on the diagonal. */
void wsmo_center_distances(const double* centers, int K, double* d) {
    for (int i = 0; i < K; ++i) d[i * K + i] = 0.0;
    for (int i = 0; i < K; ++i)
        for (int j = i + 1; j < K; ++j) {
            double v = sqdist(centers + 3 * i, centers + 3 * j);
            d[i * K + j] = v;
            d[j * K + i] = v;
        }
}

/* true when center a comes before center b in row p of M (reading R2). */
static int row_before(const double* drow, int p, int a, int b) {
    if (drow[a] != drow[b]) return drow[a] < drow[b];
    int ca = (a != p), cb = (b != p);
    if (ca != cb) return ca < cb;
    return a < b;
}

/* Algorithm 2: M[p] lists all K center indices ordered by their distance
 * from c_p, nearest first (ties as in reading R2).  Plain insertion sort of
 * every row; indices are 0-based. */
void wsmo_sort_rows(const double* d, int K, int32_t* M) {
    for (int p = 0; p < K; ++p) {
        const double* drow = d + (size_t)p * K;
        int32_t* row = M + (size_t)p * K;
        for (int j = 0; j < K; ++j) {
            int v = j, q = j;
            while (q > 0 && row_before(drow, p, v, row[q - 1])) {
                row[q] = row[q - 1];
                --q;
            }
            row[q] = v;
        }
    }
}

/* Algorithm 2, assignment (Sec. 2, sort-means): color x_i starts from the
 * center p it held after the previous pass; prev_dist, its squared distance
 * to c_p, is also the running minimum.  The other centers are visited in the
 * order of row p of M.  By the triangle inequality a center c_t with
 * ||c_p - c_t|| >= 2 ||x_i - c_p|| cannot be nearer than c_p, and since the
 * row is sorted neither can any later one, so the visit stops at the first
 * such t (squared: d[p][t] >= 4 prev_dist; note that the bound uses the
 * distance to c_p, not the running minimum).  A visited center replaces the
 * current one when its distance is less than or equal to the running
 * minimum, so among equal distances the one visited last wins.
 * Writes each color's final minimum to out_min (if not NULL) and returns
 * the number of distances ||x_i - c_k||^2 computed over all colors. */
int64_t wsmo_assign(const uint32_t* colors, int64_t n_unique, const double* centers, int K,
                    const double* d, const int32_t* M, int32_t* labels, double* out_min) {
    int64_t evaluated = 0;
    for (int64_t i = 0; i < n_unique; ++i) {
        double x[3];
        unpack(colors[i], x);
        int p = labels[i];
        double prev_dist = sqdist(x, centers + 3 * p);
        double min_dist = prev_dist;
        evaluated += 1;
        for (int j = 1; j < K; ++j) {           /* 0-based: j = 1 is the paper's j = 2 */
            int t = M[(size_t)p * K + j];
            if (d[(size_t)p * K + t] >= 4.0 * prev_dist) break;
            double dist = sqdist(x, centers + 3 * t);
            evaluated += 1;
            if (dist <= min_dist) {
                min_dist = dist;
                labels[i] = t;
            }
        }
        if (out_min) out_min[i] = min_dist;
    }
    return evaluated;
}

/* Algorithm 2, update: every center moves to the weighted mean of the
 * colors assigned to it, c_k = (sum_{m[i]=k} w_i x_i) / (sum_{m[i]=k} w_i)
 * with w_i = n_i / N.  The normalisation by N cancels in
 * the ratio, so the numerator and denominator are accumulated exactly as the
 * integers S_k = sum n_i x_i and W_k = sum n_i and divided once in FP64.
 * An empty cluster keeps its center (reading R3).  S is [K][3], W is [K]. */
void wsmo_update(const uint32_t* colors, const uint32_t* counts, int64_t n_unique,
                 const int32_t* labels, int K, double* centers, int64_t* S, int64_t* W) {
    memset(S, 0, sizeof(int64_t) * 3 * (size_t)K);
    memset(W, 0, sizeof(int64_t) * (size_t)K);
    for (int64_t i = 0; i < n_unique; ++i) {
        int k = labels[i];
        int64_t n = counts[i];
        S[3 * k + 0] += n * (int64_t)((colors[i] >> 16) & 255u);
        S[3 * k + 1] += n * (int64_t)((colors[i] >> 8) & 255u);
        S[3 * k + 2] += n * (int64_t)(colors[i] & 255u);
        W[k] += n;
    }
    for (int k = 0; k < K; ++k)
        if (W[k] > 0)
            for (int c = 0; c < 3; ++c) centers[3 * k + c] = (double)S[3 * k + c] / (double)W[k];
}

/* The same update written literally with normalised FP64 weights
 * w_i = n_i / N ("Sample weighting"); used to check that the normalisation
 * indeed cancels. */
void wsmo_update_normalised(const uint32_t* colors, const uint32_t* counts, int64_t n_unique,
                            const int32_t* labels, int K, double* centers) {
    double N = 0.0;
    for (int64_t i = 0; i < n_unique; ++i) N += (double)counts[i];
    double* num = (double*)calloc((size_t)K * 4, sizeof(double));
    if (!num) return;
    for (int64_t i = 0; i < n_unique; ++i) {
        double x[3], w = (double)counts[i] / N;
        unpack(colors[i], x);
        int k = labels[i];
        for (int c = 0; c < 3; ++c) num[4 * k + c] += w * x[c];
        num[4 * k + 3] += w;
    }
    for (int k = 0; k < K; ++k)
        if (num[4 * k + 3] > 0.0)
            for (int c = 0; c < 3; ++c) centers[3 * k + c] = num[4 * k + c] / num[4 * k + 3];
    free(num);
}

/* One pass of the main loop of Algorithm 2: distances between centers, the
 * sorted matrix M, the pruned assignment and the weighted means.  Returns
 * SSE_i = sum_i w_i min_dist_i of the assignment step (reading R4); S and W
 * (may be NULL) receive the integer sums of the update. */
double wsmo_iteration(const uint32_t* colors, const uint32_t* counts, int64_t n_unique, int K,
                      double* centers, int32_t* labels, int64_t* S, int64_t* W,
                      int64_t* evaluated) {
    double* d = (double*)malloc(sizeof(double) * (size_t)K * K);
    int32_t* M = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * K);
    double* mind = (double*)malloc(sizeof(double) * (size_t)(n_unique > 0 ? n_unique : 1));
    int64_t* S_ = S ? S : (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)K);
    int64_t* W_ = W ? W : (int64_t*)malloc(sizeof(int64_t) * (size_t)K);
    double sse = -1.0;
    if (d && M && mind && S_ && W_) {
        wsmo_center_distances(centers, K, d);
        wsmo_sort_rows(d, K, M);
        int64_t ev = wsmo_assign(colors, n_unique, centers, K, d, M, labels, mind);
        if (evaluated) *evaluated = ev;
        double N = 0.0;
        for (int64_t i = 0; i < n_unique; ++i) N += (double)counts[i];
        sse = 0.0;
        for (int64_t i = 0; i < n_unique; ++i) sse += ((double)counts[i] / N) * mind[i];
        wsmo_update(colors, counts, n_unique, labels, K, centers, S_, W_);
    }
    free(d);
    free(M);
    free(mind);
    if (!S) free(S_);
    if (!W) free(W_);
    return sse;
}

/* Algorithm 2 with the termination rule of Sec. 3.2: the fixed-iteration
 * variant (WSM) runs max_iter iterations when eps <= 0; the convergent
 * variant (WSM-C) stops as in reading R4, capped at max_iter.  sse_trace
 * (length max_iter, may be NULL) receives SSE_1..SSE_i.  Returns the number
 * of iterations run, or -1 on bad arguments. */
int wsmo_run(const uint32_t* colors, const uint32_t* counts, int64_t n_unique, int K,
             double* centers, int32_t* labels, int max_iter, double eps,
             double* sse_trace, int64_t* evaluated_total) {
    if (K < 1 || n_unique < 1 || max_iter < 0) return -1;
    double prev_sse = 0.0;
    int64_t total = 0;
    int it = 0;
    while (it < max_iter) {
        int64_t ev = 0;
        double sse = wsmo_iteration(colors, counts, n_unique, K, centers, labels, NULL, NULL, &ev);
        if (sse < 0.0) return -1;
        total += ev;
        if (sse_trace) sse_trace[it] = sse;
        ++it;
        if (eps > 0.0) {
            if (sse == 0.0) break;
            if (it >= 2 && (prev_sse - sse) / sse <= eps) break;
        }
        prev_sse = sse;
    }
    if (evaluated_total) *evaluated_total = total;
    return it;
}

/* ------------------------------------------------------------------------ */
/* Checkers that do not prune.                                              */
/* ------------------------------------------------------------------------ */

/* For every color: the smallest and second smallest ||x_i - c_k||^2 over all
 * K centers, and the lowest index attaining the smallest (reading R6). */
void wsmo_exhaustive(const uint32_t* colors, int64_t n_unique, const double* centers, int K,
                     double* best, double* second, int32_t* argmin) {
    for (int64_t i = 0; i < n_unique; ++i) {
        double x[3];
        unpack(colors[i], x);
        double b = INFINITY, s = INFINITY;
        int a = -1;
        for (int k = 0; k < K; ++k) {
            double v = sqdist(x, centers + 3 * k);
            if (v < b) { s = b; b = v; a = k; }
            else if (v < s) { s = v; }
        }
        if (best) best[i] = b;
        if (second) second[i] = s;
        if (argmin) argmin[i] = a;
    }
}

/* One iteration of Algorithm 1 (conventional batch k-means) over all pixels:
 * m[p] = argmin_k ||x_p - c_k||^2 (reading R6), then c_k = mean of the pixels
 * in S_k (empty cluster keeps its center, reading R3).  Returns the mean
 * squared distance of the assignment step. */
double wsmo_kmeans_pixels_iteration(const uint8_t* rgb, int64_t n_pixels, int stride, int K,
                                    double* centers, int32_t* labels) {
    double* sum = (double*)calloc((size_t)K * 4, sizeof(double));
    if (!sum) return -1.0;
    double sse = 0.0;
    for (int64_t p = 0; p < n_pixels; ++p) {
        double x[3] = {rgb[p * stride], rgb[p * stride + 1], rgb[p * stride + 2]};
        double b = INFINITY;
        int a = 0;
        for (int k = 0; k < K; ++k) {
            double v = sqdist(x, centers + 3 * k);
            if (v < b) { b = v; a = k; }
        }
        labels[p] = a;
        sse += b;
        for (int c = 0; c < 3; ++c) sum[4 * a + c] += x[c];
        sum[4 * a + 3] += 1.0;
    }
    for (int k = 0; k < K; ++k)
        if (sum[4 * k + 3] > 0.0)
            for (int c = 0; c < 3; ++c) centers[3 * k + c] = sum[4 * k + c] / sum[4 * k + 3];
    free(sum);
    return sse / (double)n_pixels;
}

/* ------------------------------------------------------------------------ */
/* Sec. 1: pixel mapping (each pixel takes the palette entry of its color)  */
/* and Sec. 3.1: MSE (Eq. 2) and PSNR (Eq. 3).                              */
/* ------------------------------------------------------------------------ */

/* index[p] = m[i] where x_i is the color of pixel p, found by binary search
 * in the ascending unique list.  Returns -1 if a color is missing. */
int wsmo_map(const uint8_t* rgb, int64_t n_pixels, int stride, const uint32_t* colors,
             const int32_t* labels, int64_t n_unique, int32_t* index) {
    for (int64_t p = 0; p < n_pixels; ++p) {
        const uint8_t* px = rgb + p * stride;
        uint32_t key = ((uint32_t)px[0] << 16) | ((uint32_t)px[1] << 8) | (uint32_t)px[2];
        int64_t lo = 0, hi = n_unique - 1, at = -1;
        while (lo <= hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (colors[mid] == key) { at = mid; break; }
            if (colors[mid] < key) lo = mid + 1; else hi = mid - 1;
        }
        if (at < 0) return -1;
        index[p] = labels[at];
    }
    return 0;
}

/* Eq. 2: MSE = (1/HW) sum_{h,w} ||x(h,w) - xhat(h,w)||^2 with xhat the
 * palette color of the pixel's index (full squared norm over the three
 * channels, divided by the number of pixels only). */
double wsmo_mse(const uint8_t* rgb, int64_t n_pixels, int stride, const double* palette, int K,
                const int32_t* index) {
    double acc = 0.0;
    for (int64_t p = 0; p < n_pixels; ++p) {
        int k = index[p];
        if (k < 0 || k >= K) return -1.0;
        double x[3] = {rgb[p * stride], rgb[p * stride + 1], rgb[p * stride + 2]};
        acc += sqdist(x, palette + 3 * k);
    }
    return n_pixels > 0 ? acc / (double)n_pixels : 0.0;
}

/* Eq. 3: PSNR = 20 log10(255 / sqrt(MSE)). */
double wsmo_psnr(double mse) { return 20.0 * log10(255.0 / sqrt(mse)); }

/* ------------------------------------------------------------------------ */
/* Weighted distortion as a function of the palette and of the colors,     */
/* D(C, X) = sum_i w_i min_k ||x_i - c_k||^2, and its gradient away from    */
/* ties: dD/dc_k = 2 sum_{m(i)=k} w_i (c_k - x_i), dD/dx_i = 2 w_i (x_i -   */
/* c_{m(i)}), with m(i) the exhaustive nearest center (reading R6).  The    */
/* colors are real-valued here (X is [n][3] doubles) so that the gradient   */
/* with respect to them can be checked by finite differences.               */
/* ------------------------------------------------------------------------ */
double wsmo_distortion_grad(const double* X, const double* w, int64_t n, const double* centers,
                            int K, double* dC, double* dX, int32_t* assign) {
    double D = 0.0;
    if (dC) memset(dC, 0, sizeof(double) * 3 * (size_t)K);
    for (int64_t i = 0; i < n; ++i) {
        double b = INFINITY;
        int a = 0;
        for (int k = 0; k < K; ++k) {
            double v = sqdist(X + 3 * i, centers + 3 * k);
            if (v < b) { b = v; a = k; }
        }
        D += w[i] * b;
        if (assign) assign[i] = a;
        for (int c = 0; c < 3; ++c) {
            double diff = X[3 * i + c] - centers[3 * a + c];
            if (dC) dC[3 * a + c] += -2.0 * w[i] * diff;
            if (dX) dX[3 * i + c] = 2.0 * w[i] * diff;
        }
    }
    return D;
}
