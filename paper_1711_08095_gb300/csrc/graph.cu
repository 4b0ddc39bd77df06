// Network term pass over the gene factor U2 (Alg. 1 line 10; graph regulariser f_g of
// Sec. 2.3.1; its per-edge gradient lambda_g y (u_k1 - u_k2) in the gradient equation).
//
// Every edge updates both endpoints.  Each gene row k owns its updates and applies them
// neighbour by neighbour in ascending neighbour order against the snapshot s of U2 taken
// when the pass starts:
//   u_k <- (1 - a_j) u_k + a_j s_j,   a_j = lr * lambda_g * y_kj
// Columns of a row evolve independently.
//   k_edge_pass        rows of degree <= kHeavyDegree: one thread per (row, column) walks the
//                      row's CSR list (reads of s for consecutive columns are coalesced);
//   k_edge_pass_heavy  hub rows, one CTA each: the walk is a composition of affine maps
//                      u -> (1 - a) u + a s, so each thread folds a contiguous chunk of the
//                      list into (P, S) with P = prod (1 - a), S the chunk's walk from 0, and
//                      the chunks are then applied to u in list order.
#include "common.cuh"

namespace snect {

namespace {

__global__ void k_edge_pass(const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            const float *__restrict__ cw, const float *__restrict__ snap,
                            float *__restrict__ U2, int32_t I2, int32_t J2, float step) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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

constexpr int kHeavyThreads = 256;

__global__ void __launch_bounds__(kHeavyThreads)
    k_edge_pass_heavy(const int32_t *__restrict__ rows, const int32_t *__restrict__ ptr,
                      const int32_t *__restrict__ col, const float *__restrict__ cw,
                      const float *__restrict__ snap, float *__restrict__ U2, int32_t J2, float step) {
    __shared__ float sP[kHeavyThreads];
    __shared__ float sS[kHeavyThreads * kMaxRank];
    const int32_t k = rows[blockIdx.x];
    const int32_t s0 = ptr[k], s1 = ptr[k + 1];
    const int32_t deg = s1 - s0;
    const int32_t L = (deg + kHeavyThreads - 1) / kHeavyThreads;
    const int32_t c0 = s0 + threadIdx.x * L, c1 = min(s1, c0 + L);
    float P = 1.f;
    float S[kMaxRank];
    for (int q = 0; q < J2; ++q) S[q] = 0.f;
    for (int32_t s = c0; s < c1; ++s) {
        const float a = step * cw[s];
        const float *sj = snap + (int64_t)col[s] * J2;
        P *= 1.f - a;
        for (int q = 0; q < J2; ++q) S[q] = S[q] - a * (S[q] - sj[q]);
    }
    sP[threadIdx.x] = P;
    for (int q = 0; q < J2; ++q) sS[threadIdx.x * kMaxRank + q] = S[q];
    __syncthreads();
    if (threadIdx.x < J2) {
        const int q = threadIdx.x;
        float u = U2[(int64_t)k * J2 + q];
        for (int t = 0; t < kHeavyThreads; ++t) u = fmaf(sP[t], u, sS[t * kMaxRank + q]);
        U2[(int64_t)k * J2 + q] = u;
    }
}

}  // namespace

cudaError_t launch_edge_pass(Ctx *c) {
    if (c->m == 0 || c->cfg.lambda_g == 0.f) return cudaSuccess;
    const int64_t n = (int64_t)c->d.I2 * c->d.J2;
    cudaError_t e = cudaMemcpyAsync(c->snap, c->U[1], sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                    c->stream);
    if (e != cudaSuccess) return e;
    const float step = c->cfg.lr * c->cfg.lambda_g;
    k_edge_pass<<<ceil_div(n, 256), 256, 0, c->stream>>>(c->csr_ptr, c->csr_col, c->csr_w, c->snap,
                                                         c->U[1], c->d.I2, c->d.J2, step);
    c->launches++;
    if (c->n_heavy) {
        k_edge_pass_heavy<<<(unsigned)c->n_heavy, kHeavyThreads, 0, c->stream>>>(
            c->heavy_rows, c->csr_ptr, c->csr_col, c->csr_w, c->snap, c->U[1], c->d.J2, step);
        c->launches++;
    }
    return cudaGetLastError();
}

}  // namespace snect
