// Deterministic mini-batch sweep (Alg. 1 lines 4-8 with fixed-order mini-batches).
//
// A batch is a run of consecutive entries of the visit order.  Every gradient of the batch
// is evaluated at the parameters the batch starts from, and the contributions are summed:
//   u_i <- u_i - lr * sum_{e in batch, i_e = i} ( r_e * (G x_{m!=n} u_m) + lambda/|Omega^{n,i}| u_i )
//   G   <- G   - lr * sum_{e in batch} ( r_e * a_e o b_e o c_e + lambda/|Omega| G )
// with r_e = x~_e - x_e (gradient equation, Sec. 2.3.2).  A batch of one entry is the
// per-entry step of Alg. 1.
//
// Two kernels per batch:
//   k_det_grad   one thread per entry: contraction, residual, the three row gradients into
//                a scratch buffer (entry-major), and each CTA's core partial sum
//                sum_e (r_e a_e) o b_e o c_e over its entries, in entry order;
//   k_det_apply  one thread per row segment (entries of a batch that share a row, in entry
//                order, grouped at set-up) sums its gradients in entry order and updates the
//                row; one thread per core element sums the CTA partials in CTA order.
// Every sum has a fixed order, so the result is the same on every run.
#include "contract.cuh"

namespace snect {

namespace {

constexpr int kGradThreads = 128;
constexpr int kApplyThreads = 256;

template <int CJ1, int CJ2, int CJ3>
__global__ void __launch_bounds__(kGradThreads)
    k_det_grad(const Rec *__restrict__ rec, int64_t first, int32_t len, Dims d,
               const float *__restrict__ Gg, const float *__restrict__ U1,
               const float *__restrict__ U2, const float *__restrict__ U3,
               const int32_t *__restrict__ cnt1, const int32_t *__restrict__ cnt2,
               const int32_t *__restrict__ cnt3, float lam, float *__restrict__ gbuf,
               float *__restrict__ part) {
    const int J1 = CJ1 ? CJ1 : d.J1, J2 = CJ2 ? CJ2 : d.J2, J3 = CJ3 ? CJ3 : d.J3;
    const int PI = J1 * J2 * J3, SJ = J1 + J2 + J3;
    extern __shared__ float sm[];
    float *sG = sm;                         // PI
    float *sRA = sG + PI;                   // kGradThreads * J1 : r * a
    float *sB = sRA + kGradThreads * J1;    // kGradThreads * J2
    float *sC = sB + kGradThreads * J2;     // kGradThreads * J3
    for (int t = threadIdx.x; t < PI; t += blockDim.x) sG[t] = Gg[t];
    __syncthreads();

    const int64_t el = (int64_t)blockIdx.x * kGradThreads + threadIdx.x;
    const int tl = threadIdx.x;
    float a[RankCap<CJ1>::value], b[RankCap<CJ2>::value], c[RankCap<CJ3>::value];
    float v[RankCap<CJ1>::value], w2[RankCap<CJ2>::value], w3[RankCap<CJ3>::value];
    if (el < len) {
        const Rec e = rec[first + el];
#pragma unroll
        for (int p = 0; p < J1; ++p)
            a[p] = U1[(int64_t)e.i * J1 + p];
#pragma unroll
        for (int q = 0; q < J2; ++q)
            b[q] = U2[(int64_t)e.j * J2 + q];
#pragma unroll
        for (int r = 0; r < J3; ++r)
            c[r] = U3[(int64_t)e.k * J3 + r];
        const float xt = contract_entry<CJ1, CJ2, CJ3>(sG, J1, J2, J3, a, b, c, v, w2, w3);
        const float res = xt - e.x;
        const float la = lam / (float)cnt1[e.i], lb = lam / (float)cnt2[e.j], lc = lam / (float)cnt3[e.k];
        float *g = gbuf + el * SJ;
#pragma unroll
        for (int p = 0; p < J1; ++p)
            {
                g[p] = fmaf(res, v[p], la * a[p]);
                sRA[tl * J1 + p] = res * a[p];
            }
#pragma unroll
        for (int q = 0; q < J2; ++q)
            {
                g[J1 + q] = fmaf(res, w2[q], lb * b[q]);
                sB[tl * J2 + q] = b[q];
            }
#pragma unroll
        for (int r = 0; r < J3; ++r)
            {
                g[J1 + J2 + r] = fmaf(res, w3[r], lc * c[r]);
                sC[tl * J3 + r] = c[r];
            }
    }
    __syncthreads();
    // core partial of this CTA: sum over its entries, in entry order
    const int64_t left = len - (int64_t)blockIdx.x * kGradThreads;
    const int n_here = left < kGradThreads ? (int)left : kGradThreads;
    for (int s = threadIdx.x; s < PI; s += blockDim.x) {
        const int p = s / (J2 * J3), q = (s / J3) % J2, r = s % J3;
        float acc = 0.f;
        for (int t = 0; t < n_here; ++t) acc = fmaf(sRA[t * J1 + p] * sB[t * J2 + q], sC[t * J3 + r], acc);
        part[(int64_t)blockIdx.x * PI + s] = acc;
    }
}

__global__ void __launch_bounds__(kApplyThreads)
    k_det_apply(const Rec *__restrict__ rec, int64_t first, int32_t len, Dims d,
                const int32_t *__restrict__ pos0, const int32_t *__restrict__ pos1,
                const int32_t *__restrict__ pos2, const uint8_t *__restrict__ head0,
                const uint8_t *__restrict__ head1, const uint8_t *__restrict__ head2,
                const float *__restrict__ gbuf, const float *__restrict__ part, int32_t n_part,
                float lr, float lam_core, float *__restrict__ G, float *__restrict__ U1,
                float *__restrict__ U2, float *__restrict__ U3) {
    const int mode = blockIdx.y;
    const int SJ = d.J1 + d.J2 + d.J3;
    if (mode < 3) {
        const int64_t sl = (int64_t)blockIdx.x * kApplyThreads + threadIdx.x;
        if (sl >= len) return;
        const int32_t *pos = mode == 0 ? pos0 : (mode == 1 ? pos1 : pos2);
        const uint8_t *head = mode == 0 ? head0 : (mode == 1 ? head1 : head2);
        const int64_t s = first + sl;
        if (!head[s]) return;
        int64_t end = s + 1;
        while (end < first + len && !head[end]) ++end;
        const Rec e = rec[pos[s]];
        const int row = mode == 0 ? e.i : (mode == 1 ? e.j : e.k);
        const int Jn = mode == 0 ? d.J1 : (mode == 1 ? d.J2 : d.J3);
        const int off = mode == 0 ? 0 : (mode == 1 ? d.J1 : d.J1 + d.J2);
        float *U = mode == 0 ? U1 : (mode == 1 ? U2 : U3);
        for (int q = 0; q < Jn; ++q) {
            float acc = 0.f;
            for (int64_t t = s; t < end; ++t) acc += gbuf[(int64_t)(pos[t] - first) * SJ + off + q];
            U[(int64_t)row * Jn + q] -= lr * acc;
        }
    } else {
        const int PI = d.J1 * d.J2 * d.J3;
        const int s = blockIdx.x * kApplyThreads + threadIdx.x;
        if (s >= PI) return;
        float acc = 0.f;
        for (int t = 0; t < n_part; ++t) acc += part[(int64_t)t * PI + s];
        const float g = G[s];
        G[s] = g - lr * fmaf((float)len * lam_core, g, acc);
    }
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t run_grad(Ctx *c, int64_t first, int64_t len) {
    const int blocks = ceil_div(len, kGradThreads);
    const size_t smem = sizeof(float) * (c->PI + (size_t)kGradThreads * c->SJ);
    k_det_grad<CJ1, CJ2, CJ3><<<blocks, kGradThreads, smem, c->stream>>>(
        c->rec, first, (int32_t)len, c->d, c->G, c->U[0], c->U[1], c->U[2], c->cnt[0], c->cnt[1],
        c->cnt[2], c->cfg.lambda, c->gbuf, c->part);
    c->launches++;
    return cudaGetLastError();
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t set_grad_attr(Ctx *) {
    return cudaFuncSetAttribute(k_det_grad<CJ1, CJ2, CJ3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
}

}  // namespace

cudaError_t det_init_attrs(Ctx *c) {
    return SNECT_DISPATCH_RANKS(c->d.J1, c->d.J2, c->d.J3, set_grad_attr, c);
}

cudaError_t launch_det_grad(Ctx *c, int64_t first, int64_t len) {
    return SNECT_DISPATCH_RANKS(c->d.J1, c->d.J2, c->d.J3, run_grad, c, first, len);
}

cudaError_t launch_det_apply(Ctx *c, int64_t first, int64_t len) {
    const int n_part = ceil_div(len, kGradThreads);
    const int bx = (int)std::max<int64_t>(ceil_div(len, kApplyThreads), ceil_div(c->PI, kApplyThreads));
    dim3 grid(bx, 4);
    k_det_apply<<<grid, kApplyThreads, 0, c->stream>>>(
        c->rec, first, (int32_t)len, c->d, c->grp_pos[0], c->grp_pos[1], c->grp_pos[2],
        c->grp_head[0], c->grp_head[1], c->grp_head[2], c->gbuf, c->part, n_part, c->cfg.lr,
        c->cfg.lambda / (float)c->nnz, c->G, c->U[0], c->U[1], c->U[2]);
    c->launches++;
    return cudaGetLastError();
}

int det_scratch_floats(const Ctx *c, int64_t *gbuf_floats, int64_t *part_floats) {
    *gbuf_floats = (int64_t)c->cfg.batch * c->SJ;
    *part_floats = (int64_t)ceil_div(c->cfg.batch, kGradThreads) * c->PI;
    return 0;
}

}  // namespace snect
