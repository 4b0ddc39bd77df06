// The lock-free form of Alg. 1 as the paper states it (Sec. 2.3.3), for comparison with the
// wave-synchronous fast mode.
//
// P workers share one interleaved order of entries and network edges; worker t takes items
// t, t + P, t + 2P, ... one after another.  An entry item reads its three factor rows and the
// core as they are at that moment, forms the per-entry gradients of Sec. 2.3.2 and subtracts
// lr times them from the three rows with atomic adds (lock-free: no update is lost, none is
// waited for); the core is stepped by worker 0 alone, with step lr * P, on the entries worker 0
// visits (Alg. 1 line 8: "executed by only one core").  An edge item (k1, k2, y) reads both
// gene rows and moves each towards the other by lr lambda_g y (u_k1 - u_k2) (line 10).  With
// P = 1 this is Alg. 1 with one worker, item by item in the given order.
//
// Rows and core are read through L2 (ld.global.cg) because other workers change them during
// the launch.  One launch per epoch; P threads.
#include "contract.cuh"

namespace snect {

namespace {

struct HogArgs {
    const Rec *rec;
    const int2 *edges;
    const float *ew;
    const int32_t *order;
    int64_t n_items, nnz;
    int32_t P;
    float *G, *U1, *U2, *U3;
    const int32_t *cnt1, *cnt2, *cnt3;
    Dims d;
    float lam, lam_g, lr, lam_core;
};

template <int CJ1, int CJ2, int CJ3>
__global__ void __launch_bounds__(128) k_hogwild(HogArgs A) {
    const int J1 = CJ1 ? CJ1 : A.d.J1, J2 = CJ2 ? CJ2 : A.d.J2, J3 = CJ3 ? CJ3 : A.d.J3;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.P) return;
    const bool core_writer = t == 0;
    const float core_step = A.lr * (float)A.P;
    float a[RankCap<CJ1>::value], b[RankCap<CJ2>::value], c[RankCap<CJ3>::value];
    float v[RankCap<CJ1>::value], w2[RankCap<CJ2>::value], w3[RankCap<CJ3>::value];
    for (int64_t s = t; s < A.n_items; s += A.P) {
        const int32_t it = A.order[s];
        if (it < A.nnz) {
            const Rec e = A.rec[it];
            float *ua = A.U1 + (int64_t)e.i * J1, *ub = A.U2 + (int64_t)e.j * J2, *uc = A.U3 + (int64_t)e.k * J3;
#pragma unroll
            for (int p = 0; p < J1; ++p) a[p] = __ldcg(ua + p);
#pragma unroll
            for (int q = 0; q < J2; ++q) b[q] = __ldcg(ub + q);
#pragma unroll
            for (int r = 0; r < J3; ++r) c[r] = __ldcg(uc + r);
            // v = G x2 b x3 c, w2 = G x1 a x3 c, w3 = G x1 a x2 b, x~ = a . v; G read from L2
#pragma unroll
            for (int q = 0; q < J2; ++q) w2[q] = 0.f;
#pragma unroll
            for (int r = 0; r < J3; ++r) w3[r] = 0.f;
#pragma unroll
            for (int p = 0; p < J1; ++p) {
                float vp = 0.f;
#pragma unroll
                for (int q = 0; q < J2; ++q) {
                    const float *g = A.G + (p * J2 + q) * J3;
                    const float ab = a[p] * b[q];
                    float tq = 0.f;
#pragma unroll
                    for (int r = 0; r < J3; ++r) {
                        const float gr = __ldcg(g + r);
                        tq = fmaf(gr, c[r], tq);
                        w3[r] = fmaf(ab, gr, w3[r]);
                    }
                    vp = fmaf(tq, b[q], vp);
                    w2[q] = fmaf(a[p], tq, w2[q]);
                }
                v[p] = vp;
            }
            float xt = 0.f;
#pragma unroll
            for (int p = 0; p < J1; ++p) xt = fmaf(a[p], v[p], xt);
            const float r = xt - e.x;
            const float la = A.lam / (float)A.cnt1[e.i], lb = A.lam / (float)A.cnt2[e.j],
                        lc = A.lam / (float)A.cnt3[e.k];
#pragma unroll
            for (int p = 0; p < J1; ++p) atomicAdd(ua + p, -A.lr * fmaf(r, v[p], la * a[p]));
#pragma unroll
            for (int q = 0; q < J2; ++q) atomicAdd(ub + q, -A.lr * fmaf(r, w2[q], lb * b[q]));
#pragma unroll
            for (int rr = 0; rr < J3; ++rr) atomicAdd(uc + rr, -A.lr * fmaf(r, w3[rr], lc * c[rr]));
            if (core_writer) {  // the single writer of the core: step lr * P
#pragma unroll
                for (int p = 0; p < J1; ++p)
#pragma unroll
                    for (int q = 0; q < J2; ++q) {
                        float *g = A.G + (p * J2 + q) * J3;
                        const float rab = r * a[p] * b[q];
#pragma unroll
                        for (int rr = 0; rr < J3; ++rr) {
                            const float gr = __ldcg(g + rr);
                            __stcg(g + rr, gr - core_step * fmaf(rab, c[rr], A.lam_core * gr));
                        }
                    }
            }
        } else {
            const int64_t ed = it - A.nnz;
            const int2 kk = A.edges[ed];
            float *u = A.U2 + (int64_t)kk.x * J2, *x = A.U2 + (int64_t)kk.y * J2;
            const float st = A.lr * A.lam_g * A.ew[ed];
#pragma unroll
            for (int q = 0; q < J2; ++q) b[q] = __ldcg(u + q) - __ldcg(x + q);
#pragma unroll
            for (int q = 0; q < J2; ++q) {
                atomicAdd(u + q, -st * b[q]);
                atomicAdd(x + q, st * b[q]);
            }
        }
    }
}

__global__ void k_check_items(const int32_t *__restrict__ order, int64_t n, int64_t n_total, int32_t *flag) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n && (order[s] < 0 || order[s] >= n_total)) atomicOr(flag, 1);
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t launch_hogwild(Ctx *c, const HogArgs &A) {
    k_hogwild<CJ1, CJ2, CJ3><<<ceil_div(A.P, 128), 128, 0, c->stream>>>(A);
    return cudaGetLastError();
}

}  // namespace

int run_hogwild(Ctx *c, const int32_t *order, int64_t n_items, int32_t P, int32_t n_epochs) {
    int32_t *dord = nullptr;
    SNECT_CUDA(c, scratch_alloc(c, &dord, sizeof(int32_t) * n_items));
    cudaError_t e = cudaMemcpyAsync(dord, order, sizeof(int32_t) * n_items, cudaMemcpyDefault, c->stream);
    // every item in range (the copy may come from device memory, so it is checked there)
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream);
    if (e == cudaSuccess && n_items > 0) {
        k_check_items<<<ceil_div(n_items, 256), 256, 0, c->stream>>>(dord, n_items, c->nnz + c->m, c->flag);
        c->launches++;
        e = cudaGetLastError();
    }
    int32_t bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, c->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && !bad) {
        HogArgs A;
        A.rec = c->rec;
        A.edges = c->edges;
        A.ew = c->ew;
        A.order = dord;
        A.n_items = n_items;
        A.nnz = c->nnz;
        A.P = P;
        A.G = c->G;
        A.U1 = c->U[0];
        A.U2 = c->U[1];
        A.U3 = c->U[2];
        A.cnt1 = c->cnt[0];
        A.cnt2 = c->cnt[1];
        A.cnt3 = c->cnt[2];
        A.d = c->d;
        A.lam = c->cfg.lambda;
        A.lam_g = c->cfg.lambda_g;
        A.lr = c->cfg.lr;
        A.lam_core = c->nnz ? c->cfg.lambda / (float)c->nnz : 0.f;
        for (int32_t ep = 0; ep < n_epochs && e == cudaSuccess; ++ep) {
            e = SNECT_DISPATCH_RANKS(c->d.J1, c->d.J2, c->d.J3, launch_hogwild, c, A);
            c->launches++;
        }
    }
    cudaFreeAsync(dord, c->stream);
    if (e != cudaSuccess) return fail(c, SNECT_ECUDA, std::string("hogwild: ") + cudaGetErrorString(e));
    if (bad) return fail(c, SNECT_EINVAL, "order holds an item outside [0, nnz + m)");
    c->param_version++;
    return SNECT_OK;
}

}  // namespace snect
