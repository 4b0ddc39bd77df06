// Downstream analyses of a fitted model: the personalised subtype matrix of patient profiles
// (Sec. 3.3) and k-means stratification of the patient factor's rows (Sec. 3.1.1).
//
// Subtype matrix of a profile u (J1): S = G x1 u (J2 x J3), S[q][r] = sum_p g_pqr u_p; the
// weight of gene-mode subtype q is ||S[q][:]||, the weight of platform k is the norm of column
// k of S x3 U3 (J2 x I3), (S x3 U3)[q][k] = sum_r S[q][r] U3[k][r].  A batch of profiles runs
// in one launch: each CTA stages G once and takes profiles in turn.
//
// k-means: Lloyd's iterations on the rows of U1 with squared Euclidean distances, from the
// caller's initial centroids.  A pass assigns every row to its nearest centroid (ties to the
// lower index) and counts the rows whose cluster changed; if none did the run has converged,
// else every centroid with rows moves to their mean (a centroid without rows stays).  The
// assignment is an integer decision, so it is taken in FP64 with one fixed operation order --
// per centroid, over the coordinates in order, a separately rounded subtract, multiply and add
// (no fused multiply-add) -- and every centroid coordinate is a sum over the rows in ascending
// order divided by the count.  The FP32 rows convert to FP64 exactly, so the distances, the
// assignments and the centroids are the same numbers a sequential FP64 program with that order
// computes.  After each pass a stable radix sort of (cluster, row) pairs lists every cluster's
// rows in ascending order, so each (cluster, coordinate) thread of the update adds only its own
// rows, in that order.  Iterations are queued in chunks; a device flag set by the update step when a pass
// changed nothing turns the remaining launches of the chunk into no-ops, and the host reads it
// between chunks.
#include <math.h>

#include <cub/cub.cuh>

#include "common.cuh"

namespace snect {

namespace {

constexpr int kMaxClusters = 128;   // centroids staged in shared memory: 128 x 32 doubles
constexpr int kKmChunk = 8;         // Lloyd passes queued between two host checks

__global__ void __launch_bounds__(256)
    k_subtype(const float *__restrict__ u, int64_t n, const float *__restrict__ G, const float *__restrict__ U3,
              int32_t J1, int32_t J2, int32_t J3, int32_t I3, float *__restrict__ S, float *__restrict__ row_norm,
              float *__restrict__ plat_norm) {
    extern __shared__ float sm[];
    const int PI = J1 * J2 * J3, Q = J2 * J3;
    float *sG = sm;             // PI
    float *sS = sG + PI;        // J2 x J3
    float *su = sS + Q;         // J1
    for (int t = threadIdx.x; t < PI; t += blockDim.x) sG[t] = G[t];
    for (int64_t qn = blockIdx.x; qn < n; qn += gridDim.x) {
        __syncthreads();  // sG staged; the previous profile's sS and su consumed
        for (int p = threadIdx.x; p < J1; p += blockDim.x) su[p] = u[qn * J1 + p];
        __syncthreads();
        for (int s = threadIdx.x; s < Q; s += blockDim.x) {
            float acc = 0.f;
            for (int p = 0; p < J1; ++p) acc = fmaf(sG[p * Q + s], su[p], acc);
            sS[s] = acc;
            if (S) S[qn * Q + s] = acc;
        }
        __syncthreads();
        if (row_norm)
            for (int q = threadIdx.x; q < J2; q += blockDim.x) {
                float acc = 0.f;
                for (int r = 0; r < J3; ++r) acc = fmaf(sS[q * J3 + r], sS[q * J3 + r], acc);
                row_norm[qn * J2 + q] = sqrtf(acc);
            }
        if (plat_norm)
            for (int k = threadIdx.x; k < I3; k += blockDim.x) {
                const float *c = U3 + (int64_t)k * J3;
                float acc = 0.f;
                for (int q = 0; q < J2; ++q) {
                    float t = 0.f;
                    for (int r = 0; r < J3; ++r) t = fmaf(sS[q * J3 + r], c[r], t);
                    acc = fmaf(t, t, acc);
                }
                plat_norm[qn * I3 + k] = sqrtf(acc);
            }
    }
}

// squared distance of row x (d FP32 values) to centroid c (FP64), coordinates in order, each
// subtract, multiply and add rounded on its own
__device__ __forceinline__ double km_dist(const float *__restrict__ x, const double *c, int d) {
    double s = 0.0;
    for (int p = 0; p < d; ++p) {
        const double t = __dsub_rn((double)x[p], c[p]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// one thread per row: nearest centroid (ties to the lower index); counts changed rows
__global__ void __launch_bounds__(256)
    k_km_assign(const float *__restrict__ X, int64_t n, int32_t d, int32_t k, const double *__restrict__ cent,
                int32_t *__restrict__ assign, int32_t *__restrict__ changed, const int32_t *__restrict__ done) {
    __shared__ double sc[kMaxClusters * kMaxRank];
    if (*done) return;
    for (int t = threadIdx.x; t < k * d; t += blockDim.x) sc[t] = cent[t];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *x = X + i * d;
    int best = 0;
    double bd = 0.0;
    for (int c = 0; c < k; ++c) {
        const double dist = km_dist(x, sc + c * d, d);
        if (c == 0 || dist < bd) {
            bd = dist;
            best = c;
        }
    }
    if (assign[i] != best) {
        atomicAdd(changed, 1);
        assign[i] = best;
    }
}

// first position in the sorted cluster ids at which the id is >= c
__device__ __forceinline__ int64_t km_lower(const int32_t *__restrict__ keys, int64_t n, int32_t c) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// one thread per (centroid, coordinate): the mean of the centroid's rows, summed in ascending
// row order (keys: the cluster ids sorted stably, rows: the row of each sorted position)
__global__ void __launch_bounds__(256)
    k_km_update(const float *__restrict__ X, int64_t n, int32_t d, int32_t k, double *__restrict__ cent,
                const int32_t *__restrict__ keys, const int32_t *__restrict__ rows,
                const int32_t *__restrict__ changed, int32_t *__restrict__ done, int32_t *__restrict__ updates) {
    if (*done) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (*changed == 0) {  // the pass changed nothing: converged, the centroids stay
        if (t == 0) *done = 1;
        return;
    }
    if (t == 0) *updates += 1;
    if (t >= k * d) return;
    const int c = t / d, p = t % d;
    const int64_t lo = km_lower(keys, n, c), hi = km_lower(keys, n, c + 1);
    double s = 0.0;
    for (int64_t q = lo; q < hi; ++q) s = __dadd_rn(s, (double)X[(int64_t)rows[q] * d + p]);
    if (hi > lo) cent[t] = __ddiv_rn(s, (double)(hi - lo));
}

__global__ void k_iota(int32_t *__restrict__ v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

__global__ void __launch_bounds__(256)
    k_km_inertia(const float *__restrict__ X, int64_t n, int32_t d, const double *__restrict__ cent,
                 const int32_t *__restrict__ assign, double *__restrict__ inertia) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < n) v = km_dist(X + i * d, cent + (int64_t)assign[i] * d, d);
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(inertia, v);
}

}  // namespace

int run_subtype(Ctx *c, const float *u, int64_t n, float *S, float *row_norm, float *plat_norm) {
    const Dims &d = c->d;
    const int64_t Q = (int64_t)d.J2 * d.J3;
    float *du = nullptr, *dS = nullptr, *drn = nullptr, *dpn = nullptr;
    int rc = SNECT_OK;
    auto cleanup = [&]() {
        for (float *p : {du, dS, drn, dpn})
            if (p) cudaFreeAsync(p, c->stream);
    };
    cudaError_t e = scratch_alloc(c, &du, sizeof(float) * n * d.J1);
    if (e == cudaSuccess && S) e = scratch_alloc(c, &dS, sizeof(float) * n * Q);
    if (e == cudaSuccess && row_norm) e = scratch_alloc(c, &drn, sizeof(float) * n * d.J2);
    if (e == cudaSuccess && plat_norm) e = scratch_alloc(c, &dpn, sizeof(float) * n * d.I3);
    if (e == cudaSuccess) e = cudaMemcpyAsync(du, u, sizeof(float) * n * d.J1, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        const int grid = (int)std::min<int64_t>(n, 4 * (int64_t)std::max(sms, 1));
        const size_t smem = sizeof(float) * ((size_t)c->PI + Q + d.J1);
        k_subtype<<<grid, 256, smem, c->stream>>>(du, n, c->G, c->U[2], d.J1, d.J2, d.J3, d.I3, dS, drn, dpn);
        c->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && S) e = cudaMemcpyAsync(S, dS, sizeof(float) * n * Q, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && row_norm)
        e = cudaMemcpyAsync(row_norm, drn, sizeof(float) * n * d.J2, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && plat_norm)
        e = cudaMemcpyAsync(plat_norm, dpn, sizeof(float) * n * d.I3, cudaMemcpyDefault, c->stream);
    cleanup();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = fail(c, SNECT_ECUDA, std::string("subtype: ") + cudaGetErrorString(e));
    return rc;
}

int run_kmeans(Ctx *c, int32_t k, const double *init, int32_t max_iter, int32_t *assign, double *centroids,
               int32_t *n_updates, double *inertia) {
    const Dims &d = c->d;
    const int64_t n = d.I1;
    double *cent = nullptr, *dinert = nullptr;
    int32_t *dassign = nullptr, *words = nullptr;  // words: changed, done, updates
    int32_t *keys = nullptr, *rows_in = nullptr, *rows = nullptr;  // the stable (cluster, row) sort
    void *sort_tmp = nullptr;
    size_t sort_bytes = 0;
    int end_bit = 1;
    while (end_bit < 31 && (k >> end_bit)) ++end_bit;
    cudaError_t e = scratch_alloc(c, &cent, sizeof(double) * k * d.J1);
    if (e == cudaSuccess) e = scratch_alloc(c, &dinert, sizeof(double));
    if (e == cudaSuccess) e = scratch_alloc(c, &dassign, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = scratch_alloc(c, &words, sizeof(int32_t) * 3);
    if (e == cudaSuccess) e = scratch_alloc(c, &keys, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = scratch_alloc(c, &rows_in, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = scratch_alloc(c, &rows, sizeof(int32_t) * n);
    if (e == cudaSuccess)
        e = cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, dassign, keys, rows_in, rows, n, 0, end_bit,
                                            c->stream);
    if (e == cudaSuccess) e = scratch_alloc(c, &sort_tmp, std::max<size_t>(sort_bytes, 16));
    if (e == cudaSuccess) {
        k_iota<<<ceil_div(n, 256), 256, 0, c->stream>>>(rows_in, n);
        c->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(cent, init, sizeof(double) * k * d.J1, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dassign, 0xff, sizeof(int32_t) * n, c->stream);  // -1: none yet
    if (e == cudaSuccess) e = cudaMemsetAsync(words, 0, sizeof(int32_t) * 3, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dinert, 0, sizeof(double), c->stream);
    const int grid_rows = ceil_div(n, 256), grid_upd = ceil_div((int64_t)k * d.J1, 256);
    int32_t done = 0;
    for (int32_t it = 0; it < max_iter && e == cudaSuccess && !done; it += kKmChunk) {
        for (int32_t j = it; j < std::min(max_iter, it + kKmChunk) && e == cudaSuccess; ++j) {
            e = cudaMemsetAsync(words, 0, sizeof(int32_t), c->stream);
            if (e != cudaSuccess) break;
            k_km_assign<<<grid_rows, 256, 0, c->stream>>>(c->U[0], n, d.J1, k, cent, dassign, words, words + 1);
            e = cudaGetLastError();
            if (e == cudaSuccess)  // each cluster's rows, in ascending order (a stable sort)
                e = cub::DeviceRadixSort::SortPairs(sort_tmp, sort_bytes, dassign, keys, rows_in, rows, n, 0,
                                                    end_bit, c->stream);
            if (e != cudaSuccess) break;
            k_km_update<<<grid_upd, 256, 0, c->stream>>>(c->U[0], n, d.J1, k, cent, keys, rows, words, words + 1,
                                                         words + 2);
            c->launches += 3;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&done, words + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e == cudaSuccess) {
        k_km_inertia<<<grid_rows, 256, 0, c->stream>>>(c->U[0], n, d.J1, cent, dassign, dinert);
        c->launches++;
        e = cudaGetLastError();
    }
    int32_t upd = 0;
    double in = 0.0;
    if (e == cudaSuccess && assign) e = cudaMemcpyAsync(assign, dassign, sizeof(int32_t) * n, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && centroids)
        e = cudaMemcpyAsync(centroids, cent, sizeof(double) * k * d.J1, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&upd, words + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&in, dinert, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    for (void *p : {(void *)cent, (void *)dinert, (void *)dassign, (void *)words, (void *)keys, (void *)rows_in,
                    (void *)rows, sort_tmp})
        if (p) cudaFreeAsync(p, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SNECT_ECUDA, std::string("kmeans: ") + cudaGetErrorString(e));
    if (n_updates) *n_updates = upd;
    if (inertia) *inertia = in;
    return SNECT_OK;
}

int kmeans_max_clusters() { return kMaxClusters; }

}  // namespace snect
