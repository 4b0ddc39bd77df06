// Network term pass over the gene factor U2 (Alg. 1 line 10; graph regulariser f_g of
// Sec. 2.3.1; its per-edge gradient lambda_g y (u_k1 - u_k2) in the gradient equation).
//
// Every edge updates both endpoints.  Each gene row k owns its updates and applies them
// neighbour by neighbour in ascending neighbour order against the snapshot s of U2 taken
// when the pass starts:
//   u_k <- (1 - a_j) u_k + a_j s_j,   a_j = lr * lambda_g * y_kj
// Columns of a row evolve independently.
//   light rows (degree <= kHeavyDegree): one thread per (row, column) walks the row's CSR
//                      list (reads of s for consecutive columns are coalesced);
//   hub rows           one CTA each: the walk is a composition of affine maps
//                      u -> (1 - a) u + a s, so each thread folds a contiguous chunk of the
//                      list into (P, S) with P = prod (1 - a), S the chunk's walk from 0, and
//                      the chunks are then applied to u in list order.
// The two touch disjoint rows and read only the snapshot, so one launch (k_edge_pass_all)
// runs both: the hub CTAs first (their walks are the longest), the light rows' CTAs beside
// them.  The batched form launches them separately over all problems.
#include "common.cuh"

namespace snect {

namespace {

// one (row, column) of a light row: the row's walk over its CSR list
__device__ __forceinline__ void light_walk(const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                           const float *__restrict__ cw, const float *__restrict__ snap,
                                           float *__restrict__ U2, int32_t I2, int32_t J2, float step, int64_t t) {
    if (t >= (int64_t)I2 * J2) return;
    const int32_t k = (int32_t)(t / J2), q = (int32_t)(t % J2);
    const int32_t s0 = ptr[k], s1 = ptr[k + 1];
    if (s0 == s1 || s1 - s0 > kHeavyDegree) return;
    float u = U2[t];
    for (int32_t s = s0; s < s1; ++s) {
        const float st = step * cw[s];
        u = u - st * (u - snap[(int64_t)col[s] * J2 + q]);
    }
    U2[t] = u;
}

constexpr int kHeavyThreads = 512;

// one hub row k by one CTA: thread (chunk, q) folds its chunk of the list for column q into
// (P, S); then the first J2 threads apply the chunks to u_k in list order
__device__ __forceinline__ void heavy_walk(int32_t k, const int32_t *__restrict__ ptr,
                                           const int32_t *__restrict__ col, const float *__restrict__ cw,
                                           const float *__restrict__ snap, float *__restrict__ U2, int32_t J2,
                                           float step, float *sP, float *sS) {
    const int nch = kHeavyThreads / J2;  // chunks (J2 <= 32: at least 16)
    const int q = threadIdx.x % J2, ch = threadIdx.x / J2;
    const int32_t s0 = ptr[k], s1 = ptr[k + 1];
    const int32_t L = (s1 - s0 + nch - 1) / nch;
    if (ch < nch) {
        const int32_t c0 = s0 + ch * L, c1 = min(s1, c0 + L);
        float P = 1.f, S = 0.f;
        for (int32_t s = c0; s < c1; ++s) {
            const float a = step * cw[s];
            P *= 1.f - a;
            S = S - a * (S - snap[(int64_t)col[s] * J2 + q]);
        }
        if (q == 0) sP[ch] = P;
        sS[ch * J2 + q] = S;
    }
    __syncthreads();
    if ((int)threadIdx.x < J2) {
        float u = U2[(int64_t)k * J2 + q];
        for (int t = 0; t < nch; ++t) u = fmaf(sP[t], u, sS[t * J2 + q]);
        U2[(int64_t)k * J2 + q] = u;
    }
}

__global__ void __launch_bounds__(kHeavyThreads)
    k_edge_pass_all(const int32_t *__restrict__ rows, int32_t n_heavy, const int32_t *__restrict__ ptr,
                    const int32_t *__restrict__ col, const float *__restrict__ cw, const float *__restrict__ snap,
                    float *__restrict__ U2, int32_t I2, int32_t J2, float step) {
    __shared__ float sP[kHeavyThreads];
    __shared__ float sS[kHeavyThreads];
    if ((int)blockIdx.x < n_heavy) {
        heavy_walk(rows[blockIdx.x], ptr, col, cw, snap, U2, J2, step, sP, sS);
        return;
    }
    light_walk(ptr, col, cw, snap, U2, I2, J2, step,
               (int64_t)(blockIdx.x - n_heavy) * kHeavyThreads + threadIdx.x);
}

// batched: blockIdx.y selects the problem
__global__ void k_batch_snap(const EdgeArgs *__restrict__ E) {
    const EdgeArgs &e = E[blockIdx.y];
    const int64_t n = (int64_t)e.I2 * e.J2;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        e.snap[t] = e.U2[t];
}

__global__ void k_batch_edge(const EdgeArgs *__restrict__ E) {
    const EdgeArgs &e = E[blockIdx.y];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)e.I2 * e.J2;
         t += (int64_t)gridDim.x * blockDim.x)
        light_walk(e.ptr, e.col, e.w, e.snap, e.U2, e.I2, e.J2, e.step, t);
}

__global__ void __launch_bounds__(kHeavyThreads) k_batch_edge_heavy(const EdgeArgs *__restrict__ E) {
    __shared__ float sP[kHeavyThreads];
    __shared__ float sS[kHeavyThreads];
    const EdgeArgs &e = E[blockIdx.y];
    if ((int64_t)blockIdx.x >= e.n_heavy) return;
    heavy_walk(e.heavy[blockIdx.x], e.ptr, e.col, e.w, e.snap, e.U2, e.J2, e.step, sP, sS);
}

}  // namespace

cudaError_t launch_edge_pass(Ctx *c) {
    if (c->m == 0 || c->cfg.lambda_g == 0.f) return cudaSuccess;
    const int64_t n = (int64_t)c->d.I2 * c->d.J2;
    cudaError_t e = cudaMemcpyAsync(c->snap, c->U[1], sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                    c->stream);
    if (e != cudaSuccess) return e;
    const float step = c->cfg.lr * c->cfg.lambda_g;
    const int32_t nh = (int32_t)c->n_heavy;
    k_edge_pass_all<<<(unsigned)(ceil_div(n, kHeavyThreads) + nh), kHeavyThreads, 0, c->stream>>>(
        c->heavy_rows, nh, c->csr_ptr, c->csr_col, c->csr_w, c->snap, c->U[1], c->d.I2, c->d.J2, step);
    c->launches++;
    return cudaGetLastError();
}

EdgeArgs make_edge_args(const Ctx *c) {
    EdgeArgs e;
    e.ptr = c->csr_ptr;
    e.col = c->csr_col;
    e.w = c->csr_w;
    e.snap = c->snap;
    e.U2 = c->U[1];
    e.I2 = c->d.I2;
    e.J2 = c->d.J2;
    e.step = c->cfg.lr * c->cfg.lambda_g;
    e.heavy = c->heavy_rows;
    // a problem without a network pass gets no rows: its light and hub walks are empty
    const bool on = c->m > 0 && c->cfg.lambda_g != 0.f;
    e.I2 = on ? c->d.I2 : 0;
    e.n_heavy = on ? c->n_heavy : 0;
    return e;
}

cudaError_t launch_batch_edge_pass(const EdgeArgs *d_args, int32_t P, int64_t max_cells, int64_t max_heavy,
                                   cudaStream_t st, int64_t *launches) {
    if (P <= 0 || max_cells <= 0) return cudaSuccess;
    const unsigned gx = (unsigned)std::min<int64_t>(ceil_div(max_cells, 256), 4096);
    k_batch_snap<<<dim3(gx, (unsigned)P), 256, 0, st>>>(d_args);
    k_batch_edge<<<dim3(gx, (unsigned)P), 256, 0, st>>>(d_args);
    *launches += 2;
    if (max_heavy > 0) {
        k_batch_edge_heavy<<<dim3((unsigned)max_heavy, (unsigned)P), kHeavyThreads, 0, st>>>(d_args);
        *launches += 1;
    }
    return cudaGetLastError();
}

}  // namespace snect
