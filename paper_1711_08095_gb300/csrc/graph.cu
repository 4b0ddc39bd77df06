// Network term pass over the gene factor U2 (Alg. 1 line 10; graph regulariser f_g of
// Sec. 2.3.1; its per-edge gradient lambda_g y (u_k1 - u_k2) in the gradient equation).
//
// Every edge updates both endpoints.  Each gene row k owns its updates and applies them
// neighbour by neighbour in ascending neighbour order against the snapshot s of U2 taken
// when the pass starts:
//   u_k <- u_k - lr * lambda_g * y_kj * (u_k - s_j)
// Columns of a row evolve independently, so one thread handles one (row, column) pair and
// walks the row's CSR neighbour list; reads of s for consecutive columns are coalesced.
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
    if (s0 == s1) return;
    float u = U2[t];
    for (int32_t s = s0; s < s1; ++s) {
        const float st = step * cw[s];
        u = u - st * (u - snap[(int64_t)col[s] * J2 + q]);
    }
    U2[t] = u;
}

}  // namespace

cudaError_t launch_edge_pass(Ctx *c) {
    if (c->m == 0 || c->cfg.lambda_g == 0.f) return cudaSuccess;
    const int64_t n = (int64_t)c->d.I2 * c->d.J2;
    cudaError_t e = cudaMemcpyAsync(c->snap, c->U[1], sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                    c->stream);
    if (e != cudaSuccess) return e;
    k_edge_pass<<<ceil_div(n, 256), 256, 0, c->stream>>>(c->csr_ptr, c->csr_col, c->csr_w, c->snap,
                                                         c->U[1], c->d.I2, c->d.J2,
                                                         c->cfg.lr * c->cfg.lambda_g);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace snect
