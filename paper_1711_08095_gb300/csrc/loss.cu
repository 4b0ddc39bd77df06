// Objective terms (Eq. 3 in the per-entry L2 form of Sec. 2.3.2, graph regulariser f_g,
// f_opt = f + lambda_g f_g) and RMSE.  Predictions are FP32 contractions.  Each thread sums
// its squared residuals in FP32 with Neumaier's compensation (about two units of roundoff
// whatever the count, all terms being non-negative), so the FP64 pipe, a small fraction of
// the FP32 rate on this part, is used once per thread; block reductions and the one atomic
// per block are FP64.
//   acc[0] sum (x - x~)^2 over the training entries
//   acc[1] sum (x - x~)^2 over the test entries
//   acc[2] ||G||^2 + sum_n sum_{i: |Omega^{n,i}| > 0} ||u_i^(n)||^2
//   acc[3] sum_edges y ||u^(2)_k1 - u^(2)_k2||^2
#include "contract.cuh"

namespace snect {

namespace {

// a running sum of non-negative FP32 terms with Neumaier's compensation
struct Sum32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

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

// Where the entry-loss kernels read the entries: packed records, or the caller's arrays
// (idx n x 3 int32, val n float) checked on the way: an index outside the tensor sets bit 1
// of *flag and leaves the entry out, a non-finite value sets bit 2.
struct EntrySrc {
    const Rec *rec;
    const int32_t *idx;
    const float *val;
    int32_t I1, I2, I3;
    int32_t *flag;
    __device__ __forceinline__ bool load(int64_t e, Rec &r) const {
        if (rec) {
            r = rec[e];
            return true;
        }
        r.i = idx[3 * e];
        r.j = idx[3 * e + 1];
        r.k = idx[3 * e + 2];
        r.x = val[e];
        if (!isfinite(r.x)) atomicOr(flag, 2);
        if (r.i < 0 || r.i >= I1 || r.j < 0 || r.j >= I2 || r.k < 0 || r.k >= I3) {
            atomicOr(flag, 1);
            return false;
        }
        return true;
    }
};

template <int CJ1, int CJ2, int CJ3>
__global__ void __launch_bounds__(256)
    k_loss_entries(EntrySrc src, int64_t n, Dims d, const float *__restrict__ Gg,
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
    Rec r;
    if (e < n && src.load(e, r)) {
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
        const float res = r.x - predict_entry<CJ1, CJ2, CJ3>(sG, J1, J2, J3, a, b, c);
        local = (double)(res * res);
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
    Sum32 local;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = edges[t];
        float d2 = 0.f;
        for (int q = 0; q < J2; ++q) {
            const float df = U2[(int64_t)e.x * J2 + q] - U2[(int64_t)e.y * J2 + q];
            d2 = fmaf(df, df, d2);
        }
        local.add(w[t] * d2);
    }
    const double s = block_sum(local.value(), red);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

int loss_grid(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(ceil_div(n, 256), 1), 4096); }

// The same squared residuals through Gc_k = G x3 c_k of every platform, formed once per CTA in
// shared memory (when I3 J1 J2 floats fit): x~ = w^T b with w = Gc_k^T a.  Entries are taken
// by lane groups: L = J2 / VEC lanes per entry, each lane holding VEC components of w and
// reading VEC components of the gene row b in one vector load, the group's partial sums
// meeting by shuffles; E = 32 / L entries per warp step.  Each warp walks one contiguous
// range of entries in batches of up to 32, and a group keeps its w while the (platform,
// patient) key stays the same:
// the fast mode keeps each wave's entries grouped by platform and patient, so w is formed
// about once per run there, and once per entry for entries in visit order.
constexpr int kLossGcMax = 12288;  // floats of Gc in shared memory (48 KB)

template <int VEC>
__device__ __forceinline__ void load_vec(const float *p, float *out, bool global) {
    if constexpr (VEC == 4) {
        const float4 t = global ? __ldg(reinterpret_cast<const float4 *>(p)) : *reinterpret_cast<const float4 *>(p);
        out[0] = t.x, out[1] = t.y, out[2] = t.z, out[3] = t.w;
    } else if constexpr (VEC == 2) {
        const float2 t = global ? __ldg(reinterpret_cast<const float2 *>(p)) : *reinterpret_cast<const float2 *>(p);
        out[0] = t.x, out[1] = t.y;
    } else {
        out[0] = global ? __ldg(p) : *p;
    }
}

template <int CJ1, int CJ2>
__global__ void __launch_bounds__(256)
    k_loss_entries_gc(EntrySrc src, int64_t n, Dims d, const float *__restrict__ Gg,
                      const float *__restrict__ U1, const float *__restrict__ U2,
                      const float *__restrict__ U3, double *acc) {
    constexpr int J1 = CJ1, J2 = CJ2, Q = CJ1 * CJ2;
    constexpr int VEC = J2 % 4 == 0 ? 4 : (J2 % 2 == 0 ? 2 : 1), L = J2 / VEC, E = 32 / L;
    static_assert(L <= 32, "lane groups");
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
    // a batch is K steps of E entries: lane l < B holds entry base + l of it, loaded in one
    // coalesced access while the previous batch is worked on; every step's gene rows are
    // requested before any is used
    constexpr int K = 32 / E, B = E * K;
    const int lane = threadIdx.x & 31, grp = lane / L, m = lane % L;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t per = (n + warps - 1) / warps;
    const int64_t r0 = min(n, wid * per), r1 = min(n, r0 + per);
    Sum32 local;
    unsigned long long ckey = ~0ull;  // the key w belongs to
    float w[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) w[v] = 0.f;
    Rec nxt;
    nxt.i = nxt.j = nxt.k = 0;
    nxt.x = 0.f;
    int nok = lane < B && r0 + lane < r1 && src.load(r0 + lane, nxt);
    for (int64_t base = r0; base < r1; base += B) {  // uniform across the warp
        const Rec cur = nxt;
        const int cok = nok;
        nok = lane < B && base + B + lane < r1 && src.load(base + B + lane, nxt);
        const int g = grp < E ? grp : 0;
        float bv[K][VEC];
#pragma unroll
        for (int t = 0; t < K; ++t) {
            // every lane takes part in every shuffle (idle lanes too)
            const int j = __shfl_sync(0xffffffffu, cur.j, t * E + g);
            const int sok = __shfl_sync(0xffffffffu, cok, t * E + g);
            if (grp < E && sok) {
                load_vec<VEC>(U2 + (int64_t)j * J2 + VEC * m, bv[t], true);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) bv[t][v] = 0.f;
            }
        }
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int sl = t * E + g;
            const int ri = __shfl_sync(0xffffffffu, cur.i, sl), rk = __shfl_sync(0xffffffffu, cur.k, sl);
            const float rx = __shfl_sync(0xffffffffu, cur.x, sl);
            const int sok = __shfl_sync(0xffffffffu, cok, sl);
            const bool ok = grp < E && sok;
            float part = 0.f;
            if (ok) {
                const unsigned long long key = ((unsigned long long)(uint32_t)rk << 32) | (uint32_t)ri;
                if (key != ckey) {  // w_q = sum_p a_p Gc_k[p][q] for this lane's q
                    ckey = key;
                    const float *gc = sGc + rk * Q + VEC * m;
#pragma unroll
                    for (int v = 0; v < VEC; ++v) w[v] = 0.f;
#pragma unroll
                    for (int p = 0; p < J1; ++p) {
                        const float ap = __ldg(U1 + (int64_t)ri * J1 + p);
                        float gv[VEC];
                        load_vec<VEC>(gc + p * J2, gv, false);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) w[v] = fmaf(ap, gv[v], w[v]);
                    }
                }
#pragma unroll
                for (int v = 0; v < VEC; ++v) part = fmaf(w[v], bv[t][v], part);
            }
#pragma unroll
            for (int off = 1; off < L; off <<= 1) {  // lane m gathers [m, m + 2 off) of its group
                const float o = __shfl_down_sync(0xffffffffu, part, off);
                if (m + off < L) part += o;
            }
            if (ok && m == 0) {
                const float res = rx - part;
                local.add(res * res);
            }
        }
    }
    const double s = block_sum(local.value(), red);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

// W[i][k] = Gc_k^T a_i for every (patient, platform), one thread per element:
// W[i][k][q] = sum_p a_p sum_r G[p][q][r] c_k[r]
__global__ void k_loss_rows(const float *__restrict__ Gg, const float *__restrict__ U1,
                            const float *__restrict__ U3, Dims d, float *__restrict__ W) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int J1 = d.J1, J2 = d.J2, J3 = d.J3;
    if (t >= (int64_t)d.I1 * d.I3 * J2) return;
    const int q = (int)(t % J2);
    const int64_t ik = t / J2, i = ik / d.I3, k = ik % d.I3;
    float w = 0.f;
    for (int p = 0; p < J1; ++p) {
        float g = 0.f;
        for (int r = 0; r < J3; ++r) g = fmaf(Gg[(p * J2 + q) * J3 + r], U3[k * J3 + r], g);
        w = fmaf(U1[i * J1 + p], g, w);
    }
    W[t] = w;
}

// The squared residuals through W: x~ = W[i][k] . b_j, a J2-term product of two gathered
// rows.  L = J2 / VEC lanes per entry, each reading VEC components of both rows in one
// vector load each, the group's partial sums meeting by shuffles; E = 32 / L entries per
// step and K steps per iteration, all their loads issued before any is used.  Each warp
// walks one contiguous range of entries.
template <int CJ2>
__global__ void __launch_bounds__(256)
    k_loss_entries_w(EntrySrc src, int64_t n, const float *__restrict__ W, int32_t I3,
                     const float *__restrict__ U2, double *acc) {
    constexpr int J2 = CJ2, VEC = J2 % 4 == 0 ? 4 : (J2 % 2 == 0 ? 2 : 1), L = J2 / VEC, E = 32 / L, K = 4;
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, grp = lane / L, m = lane % L;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t per = (n + warps - 1) / warps;
    const int64_t r0 = min(n, wid * per), r1 = min(n, r0 + per);
    Sum32 local;
    for (int64_t base = r0; base < r1; base += K * E) {  // uniform across the warp
        Rec r[K];
        bool ok[K];
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int64_t e = base + t * E + grp;
            r[t].i = r[t].j = r[t].k = 0;
            r[t].x = 0.f;
            ok[t] = grp < E && e < r1 && src.load(e, r[t]);
        }
        float wv[K][VEC], bv[K][VEC];
#pragma unroll
        for (int t = 0; t < K; ++t) {
            if (ok[t]) {
                load_vec<VEC>(W + ((int64_t)r[t].i * I3 + r[t].k) * J2 + VEC * m, wv[t], true);
                load_vec<VEC>(U2 + (int64_t)r[t].j * J2 + VEC * m, bv[t], true);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) wv[t][v] = bv[t][v] = 0.f;
            }
        }
#pragma unroll
        for (int t = 0; t < K; ++t) {
            float part = 0.f;
#pragma unroll
            for (int v = 0; v < VEC; ++v) part = fmaf(wv[t][v], bv[t][v], part);
#pragma unroll
            for (int off = 1; off < L; off <<= 1) {  // lane m gathers [m, m + 2 off) of its group
                const float o = __shfl_down_sync(0xffffffffu, part, off);
                if (m + off < L) part += o;
            }
            if (ok[t] && m == 0) {
                const float res = r[t].x - part;
                local.add(res * res);
            }
        }
    }
    const double s = block_sum(local.value(), red);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t run_loss(Ctx *c, EntrySrc src, int64_t n, int which, const float *W) {
    if constexpr (CJ2 > 0) {
        if (W) {
            const int grid = (int)std::min<int64_t>(ceil_div(n, 256), 8 * 152);
            k_loss_entries_w<CJ2><<<grid, 256, 0, c->stream>>>(src, n, W, c->d.I3, c->U[1], c->lacc + which);
            c->launches++;
            return cudaGetLastError();
        }
    }
    if constexpr (CJ1 > 0 && CJ2 > 0) {
        const int64_t gcf = (int64_t)c->d.I3 * CJ1 * CJ2;
        if (gcf <= kLossGcMax) {
            const int grid = (int)std::min<int64_t>(ceil_div(n, 256), 8 * 152);
            k_loss_entries_gc<CJ1, CJ2><<<grid, 256, sizeof(float) * gcf, c->stream>>>(
                src, n, c->d, c->G, c->U[0], c->U[1], c->U[2], c->lacc + which);
            c->launches++;
            return cudaGetLastError();
        }
    }
    const size_t smem = sizeof(float) * c->PI;
    k_loss_entries<CJ1, CJ2, CJ3><<<ceil_div(n, 256), 256, smem, c->stream>>>(
        src, n, c->d, c->G, c->U[0], c->U[1], c->U[2], c->lacc + which);
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

cudaError_t loss_rows(Ctx *c, float **W) {
    *W = nullptr;
    const int64_t rows = (int64_t)c->d.I1 * c->d.I3;
    if (rows > std::max<int64_t>(c->nnz, 1)) return cudaSuccess;  // more rows than entries
    const int64_t cells = rows * c->d.J2;
    cudaError_t e = scratch_alloc(c, W, sizeof(float) * (size_t)cells);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *W = nullptr;
        return cudaSuccess;  // the loss kernels work without it
    }
    k_loss_rows<<<ceil_div(cells, 256), 256, 0, c->stream>>>(c->G, c->U[0], c->U[2], c->d, *W);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_loss(Ctx *c, const Rec *recs, int64_t n, int which, const float *W) {
    if (n == 0) return cudaSuccess;
    const EntrySrc src{recs, nullptr, nullptr, c->d.I1, c->d.I2, c->d.I3, nullptr};
    return SNECT_DISPATCH_RANKS(c->d.J1, c->d.J2, c->d.J3, run_loss, c, src, n, which, W);
}

cudaError_t launch_loss_checked(Ctx *c, const int32_t *idx, const float *val, int64_t n, int which,
                                int32_t *flag, const float *W) {
    if (n == 0) return cudaSuccess;
    const EntrySrc src{nullptr, idx, val, c->d.I1, c->d.I2, c->d.I3, flag};
    return SNECT_DISPATCH_RANKS(c->d.J1, c->d.J2, c->d.J3, run_loss, c, src, n, which, W);
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
