// Objective terms (Eq. 3 in the per-entry L2 form of Sec. 2.3.2, graph regulariser f_g,
// f_opt = f + lambda_g f_g) and RMSE.  Predictions are FP32 contractions; squares and all
// sums are FP64 (block reductions, then one FP64 atomic per block).
//   acc[0] sum (x - x~)^2 over the training entries
//   acc[1] sum (x - x~)^2 over the test entries
//   acc[2] ||G||^2 + sum_n sum_{i: |Omega^{n,i}| > 0} ||u_i^(n)||^2
//   acc[3] sum_edges y ||u^(2)_k1 - u^(2)_k2||^2
#include "contract.cuh"

namespace snect {

namespace {

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

template <int CJ1, int CJ2, int CJ3>
__global__ void __launch_bounds__(256)
    k_loss_entries(const Rec *__restrict__ rec, int64_t n, Dims d, const float *__restrict__ Gg,
                   const float *__restrict__ U1, const float *__restrict__ U2,
                   const float *__restrict__ U3, double *acc) {
    const int J1 = CJ1 ? CJ1 : d.J1, J2 = CJ2 ? CJ2 : d.J2, J3 = CJ3 ? CJ3 : d.J3;
    const int PI = J1 * J2 * J3;
    extern __shared__ float sG[];
    __shared__ double red[8];
    for (int t = threadIdx.x; t < PI; t += blockDim.x) sG[t] = Gg[t];
    __syncthreads();
    double local = 0.0;
    // one entry per thread: a grid-stride loop would let the compiler keep all of G in
    // registers across iterations
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) {
        const Rec r = rec[e];
        float a[RankCap<CJ1>::value], b[RankCap<CJ2>::value], c[RankCap<CJ3>::value];
#pragma unroll
        for (int p = 0; p < J1; ++p)
            a[p] = U1[(int64_t)r.i * J1 + p];
#pragma unroll
        for (int q = 0; q < J2; ++q)
            b[q] = U2[(int64_t)r.j * J2 + q];
#pragma unroll
        for (int s = 0; s < J3; ++s)
            c[s] = U3[(int64_t)r.k * J3 + s];
        const float xt = predict_entry<CJ1, CJ2, CJ3>(sG, J1, J2, J3, a, b, c);
        const double res = (double)r.x - (double)xt;
        local += res * res;
    }
    const double s = block_sum(local, red);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

__global__ void __launch_bounds__(256)
    k_loss_reg(const float *__restrict__ G, int32_t PI, const float *__restrict__ U1,
               const float *__restrict__ U2, const float *__restrict__ U3,
               const int32_t *__restrict__ c1, const int32_t *__restrict__ c2,
               const int32_t *__restrict__ c3, Dims d, double *acc) {
    __shared__ double red[8];
    const int64_t n1 = (int64_t)d.I1 * d.J1, n2 = (int64_t)d.I2 * d.J2, n3 = (int64_t)d.I3 * d.J3;
    const int64_t total = PI + n1 + n2 + n3;
    double local = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        double x = 0.0;
        if (t < PI) {
            x = G[t];
        } else if (t < PI + n1) {
            const int64_t u = t - PI;
            if (c1[u / d.J1] > 0) x = U1[u];
        } else if (t < PI + n1 + n2) {
            const int64_t u = t - PI - n1;
            if (c2[u / d.J2] > 0) x = U2[u];
        } else {
            const int64_t u = t - PI - n1 - n2;
            if (c3[u / d.J3] > 0) x = U3[u];
        }
        local += x * x;
    }
    const double s = block_sum(local, red);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

__global__ void __launch_bounds__(256)
    k_loss_graph(const int2 *__restrict__ edges, const float *__restrict__ w, int64_t m,
                 const float *__restrict__ U2, int32_t J2, double *acc) {
    __shared__ double red[8];
    double local = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = edges[t];
        double d2 = 0.0;
        for (int q = 0; q < J2; ++q) {
            const double df = (double)U2[(int64_t)e.x * J2 + q] - (double)U2[(int64_t)e.y * J2 + q];
            d2 += df * df;
        }
        local += (double)w[t] * d2;
    }
    const double s = block_sum(local, red);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

int loss_grid(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(ceil_div(n, 256), 1), 4096); }

// The same squared residuals through Gc_k = G x3 c_k of every platform, formed once per CTA in
// shared memory (when I3 J1 J2 floats fit): x~ = a^T Gc_k b, J1 J2 products per entry instead
// of the full contraction.  A grid-stride loop amortises the set-up over many entries.
constexpr int kLossGcMax = 12288;  // floats of Gc in shared memory (48 KB)

template <int CJ1, int CJ2>
__global__ void __launch_bounds__(256)
    k_loss_entries_gc(const Rec *__restrict__ rec, int64_t n, Dims d, const float *__restrict__ Gg,
                      const float *__restrict__ U1, const float *__restrict__ U2,
                      const float *__restrict__ U3, double *acc) {
    constexpr int J1 = CJ1, J2 = CJ2, Q = CJ1 * CJ2;
    const int J3 = d.J3, I3 = d.I3;
    extern __shared__ float sGc[];  // I3 x J1 x J2
    __shared__ double red[8];
    for (int s = threadIdx.x; s < I3 * Q; s += blockDim.x) {
        const int k = s / Q, pq = s % Q;
        float g = 0.f;
        for (int r = 0; r < J3; ++r) g = fmaf(Gg[pq * J3 + r], U3[(int64_t)k * J3 + r], g);
        sGc[s] = g;
    }
    __syncthreads();
    double local = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const Rec r = rec[e];
        float b[J2];
#pragma unroll
        for (int q = 0; q < J2; ++q) b[q] = __ldg(U2 + (int64_t)r.j * J2 + q);
        const float *gc = sGc + r.k * Q;
        float xt = 0.f;
#pragma unroll
        for (int p = 0; p < J1; ++p) {
            float vp = 0.f;
#pragma unroll
            for (int q = 0; q < J2; ++q) vp = fmaf(gc[p * J2 + q], b[q], vp);
            xt = fmaf(__ldg(U1 + (int64_t)r.i * J1 + p), vp, xt);
        }
        const double res = (double)r.x - (double)xt;
        local += res * res;
    }
    const double s = block_sum(local, red);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t run_loss(Ctx *c, const Rec *recs, int64_t n, int which) {
    if constexpr (CJ1 > 0 && CJ2 > 0) {
        const int64_t gcf = (int64_t)c->d.I3 * CJ1 * CJ2;
        if (gcf <= kLossGcMax) {
            const int grid = (int)std::min<int64_t>(ceil_div(n, 256), 8 * 152);
            k_loss_entries_gc<CJ1, CJ2><<<grid, 256, sizeof(float) * gcf, c->stream>>>(
                recs, n, c->d, c->G, c->U[0], c->U[1], c->U[2], c->lacc + which);
            c->launches++;
            return cudaGetLastError();
        }
    }
    const size_t smem = sizeof(float) * c->PI;
    k_loss_entries<CJ1, CJ2, CJ3><<<ceil_div(n, 256), 256, smem, c->stream>>>(
        recs, n, c->d, c->G, c->U[0], c->U[1], c->U[2], c->lacc + which);
    c->launches++;
    return cudaGetLastError();
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t set_loss_attr(Ctx *) {
    return cudaFuncSetAttribute(k_loss_entries<CJ1, CJ2, CJ3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                64 * 1024);
}

}  // namespace

cudaError_t loss_init_attrs(Ctx *c) {
    return SNECT_DISPATCH_RANKS(c->d.J1, c->d.J2, c->d.J3, set_loss_attr, c);
}

cudaError_t launch_loss(Ctx *c, const Rec *recs, int64_t n, int which) {
    if (n == 0) return cudaSuccess;
    return SNECT_DISPATCH_RANKS(c->d.J1, c->d.J2, c->d.J3, run_loss, c, recs, n, which);
}

cudaError_t launch_loss_reg_graph(Ctx *c) {
    const int64_t total = c->PI + (int64_t)c->d.I1 * c->d.J1 + (int64_t)c->d.I2 * c->d.J2 +
                          (int64_t)c->d.I3 * c->d.J3;
    k_loss_reg<<<loss_grid(total), 256, 0, c->stream>>>(c->G, c->PI, c->U[0], c->U[1], c->U[2],
                                                         c->cnt[0], c->cnt[1], c->cnt[2], c->d,
                                                         c->lacc + 2);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || c->m == 0) return e;
    k_loss_graph<<<loss_grid(c->m), 256, 0, c->stream>>>(c->edges, c->ew, c->m, c->U[1], c->d.J2,
                                                         c->lacc + 3);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace snect
