// Fold-in of a new patient (Eq. 9) and top-k patient search (Sec. 3.2.1).
//
// Fold-in holds G, U2, U3 fixed and solves for the patient row u:
//   min_u 1/2 sum_{(j,k) observed} (x_jk - u . w_jk)^2 + lambda/2 ||u||^2,
//   w_jk = G x2 u2_j x3 u3_k  (length J1)
// i.e. (sum w w^T + lambda I) u = sum x w.  The lambda/2 ||u||^2 term is what the per-entry
// L2 terms of Sec. 2.3.2 add up to for one row.
//   k_wtable         w_jk for every (gene, platform) pair once the factors are fixed
//                    (I2*I3 rows of J1 floats; L2-resident at the paper's sizes);
//   k_foldin_partial each CTA checks a fixed run of the query's cells and sums w w^T and x w
//                    over it, in cell order (one thread per Gram element), into its own partial;
//   k_foldin_solve   one CTA adds the partials in CTA order, adds lambda I, and solves by an
//                    FP64 Cholesky factorisation.
// The partition into CTAs depends only on the query's size, so the result of a query is the
// same whether it runs alone or beside others.
//
// Top-k: cos(u, u1_i) for every patient row, then k rounds of a block-wide arg-max
// (largest score, lower index on ties); a zero-norm row or query scores 0.
#include "common.cuh"
#include "serve.cuh"

namespace snect {

namespace {

__global__ void k_wtable(const float *__restrict__ G, const float *__restrict__ U2,
                         const float *__restrict__ U3, int32_t I2, int32_t I3, int32_t J1,
                         int32_t J2, int32_t J3, float *__restrict__ table) {
    extern __shared__ float sG[];
    const int PI = J1 * J2 * J3;
    for (int t = threadIdx.x; t < PI; t += blockDim.x) sG[t] = G[t];
    __syncthreads();
    const int64_t jk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (jk >= (int64_t)I2 * I3) return;
    const int64_t j = jk / I3, k = jk % I3;
    const float *b = U2 + j * J2;
    const float *c = U3 + k * J3;
    float cr[kMaxRank];
    for (int r = 0; r < J3; ++r) cr[r] = c[r];
    for (int p = 0; p < J1; ++p) {
        float s = 0.f;
        for (int q = 0; q < J2; ++q) {
            float t = 0.f;
            const float *g = sG + (p * J2 + q) * J3;
            for (int r = 0; r < J3; ++r) t = fmaf(g[r], cr[r], t);
            s = fmaf(t, b[q], s);
        }
        table[jk * J1 + p] = s;
    }
}

// cells [blockIdx.x * chunk, ...) of one query; part: (J1*J1 + J1) floats per CTA.  Each
// cell is checked as it is staged: one outside the I2 x I3 table is read as (0, 0) and ORs 1
// into *flag, a value that is not finite ORs 2 (the query is then rejected)
__global__ void __launch_bounds__(kFoldThreads)
    k_foldin_partial(const int2 *__restrict__ jk, const float *__restrict__ val, int64_t n,
                     int64_t chunk, const float *__restrict__ table, int32_t I2, int32_t I3, int32_t J1,
                     float *__restrict__ part, int32_t *__restrict__ flag) {
    __shared__ float sw[kFoldTile * kMaxRank];
    __shared__ float sx[kFoldTile];
    const int64_t c0 = (int64_t)blockIdx.x * chunk;
    const int64_t c1 = min(n, c0 + chunk);
    const int nG = J1 * J1;
    float acc[kFoldPerThread];
#pragma unroll
    for (int t = 0; t < kFoldPerThread; ++t) acc[t] = 0.f;
    float accx = 0.f;
    for (int64_t base = c0; base < c1; base += kFoldTile) {
        const int len = (c1 - base) < kFoldTile ? (int)(c1 - base) : kFoldTile;
        __syncthreads();
        for (int t = threadIdx.x; t < len * J1; t += blockDim.x) {
            const int e = t / J1, p = t % J1;
            int2 cell = jk[base + e];
            if (cell.x < 0 || cell.x >= I2 || cell.y < 0 || cell.y >= I3) {
                cell = make_int2(0, 0);
                if (p == 0) atomicOr(flag, 1);
            }
            sw[e * J1 + p] = table[((int64_t)cell.x * I3 + cell.y) * J1 + p];
        }
        for (int t = threadIdx.x; t < len; t += blockDim.x) {
            const float x = val[base + t];
            if (!isfinite(x)) atomicOr(flag, 2);
            sx[t] = x;
        }
        __syncthreads();
        // four independent sums over the cells (e mod 4), added in a fixed order at the end
#pragma unroll
        for (int t = 0; t < kFoldPerThread; ++t) {
            const int s = threadIdx.x + t * kFoldThreads;
            if (s < nG) {
                const int p = s / J1, q = s % J1;
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
                int e = 0;
                for (; e + 4 <= len; e += 4) {
                    a0 = fmaf(sw[e * J1 + p], sw[e * J1 + q], a0);
                    a1 = fmaf(sw[(e + 1) * J1 + p], sw[(e + 1) * J1 + q], a1);
                    a2 = fmaf(sw[(e + 2) * J1 + p], sw[(e + 2) * J1 + q], a2);
                    a3 = fmaf(sw[(e + 3) * J1 + p], sw[(e + 3) * J1 + q], a3);
                }
                for (; e < len; ++e) a0 = fmaf(sw[e * J1 + p], sw[e * J1 + q], a0);
                acc[t] += (a0 + a1) + (a2 + a3);
            }
        }
        if (threadIdx.x < J1) {
            const int p = threadIdx.x;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            int e = 0;
            for (; e + 4 <= len; e += 4) {
                a0 = fmaf(sx[e], sw[e * J1 + p], a0);
                a1 = fmaf(sx[e + 1], sw[(e + 1) * J1 + p], a1);
                a2 = fmaf(sx[e + 2], sw[(e + 2) * J1 + p], a2);
                a3 = fmaf(sx[e + 3], sw[(e + 3) * J1 + p], a3);
            }
            for (; e < len; ++e) a0 = fmaf(sx[e], sw[e * J1 + p], a0);
            accx += (a0 + a1) + (a2 + a3);
        }
    }
    float *out = part + (int64_t)blockIdx.x * (nG + J1);
#pragma unroll
    for (int t = 0; t < kFoldPerThread; ++t) {
        const int s = threadIdx.x + t * kFoldThreads;
        if (s < nG) out[s] = acc[t];
    }
    if (threadIdx.x < J1) out[nG + threadIdx.x] = accx;
}

// flag_out, if given, receives the partials' cell flag, which is zeroed for the next query
// of the stream (every partial CTA has finished when this kernel starts)
__global__ void __launch_bounds__(kFoldThreads)
    k_foldin_solve(const float *__restrict__ part, int32_t n_part, int32_t J1, float ridge,
                   float *__restrict__ u_out, int32_t *__restrict__ status, int32_t *__restrict__ flag,
                   int32_t *__restrict__ flag_out) {
    __shared__ double M[kMaxRank * kMaxRank];
    __shared__ double rhs[kMaxRank];
    __shared__ double dinv[kMaxRank];  // 1 / L[j][j]
    if (flag_out && threadIdx.x == 0) {
        *flag_out = *flag;
        *flag = 0;
    }
    const int nG = J1 * J1;
    for (int s = threadIdx.x; s < nG + J1; s += blockDim.x) {
        float a = 0.f;
        for (int t = 0; t < n_part; ++t) a += part[(int64_t)t * (nG + J1) + s];
        if (s < nG) {
            M[s] = (double)a + ((s / J1 == s % J1) ? (double)ridge : 0.0);
        } else {
            rhs[s - nG] = (double)a;
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    // Cholesky M = L L^T (right-looking, lower triangle in place) by one warp: lane i owns row
    // i; then the two triangular solves, one column at a time
    const int lane = threadIdx.x;
    constexpr unsigned FULL = 0xffffffffu;
    for (int j = 0; j < J1; ++j) {
        const double dj = M[j * J1 + j];
        if (!(dj > 0.0)) {  // the same value in every lane
            if (lane < J1) u_out[lane] = 0.f;
            if (lane == 0) *status = 1;
            return;
        }
        // 1/sqrt(dj) from the FP32 estimate and two Newton-Raphson steps r <- r (3 - dj r^2) / 2
        // (each squares the relative error: 2^-22 -> 2^-43 -> below FP64 rounding), then
        // sqrt(dj) = dj r; pivots outside the FP32 normal range take the FP64 square root
        double inv, d;
        const float jf = (float)dj;
        if (jf >= 1.1754944e-38f && jf <= 3.4e38f) {
            double r = (double)rsqrtf(jf);
            r = r * (1.5 - 0.5 * dj * r * r);
            r = r * (1.5 - 0.5 * dj * r * r);
            inv = r;
            d = dj * r;
        } else {
            d = sqrt(dj);
            inv = 1.0 / d;
        }
        __syncwarp(FULL);
        if (lane == j) {
            M[j * J1 + j] = d;
            dinv[j] = inv;
        }
        if (lane > j && lane < J1) M[lane * J1 + j] *= inv;
        __syncwarp(FULL);
        if (lane > j && lane < J1) {
            const double lij = M[lane * J1 + j];
            for (int m = j + 1; m <= lane; ++m) M[lane * J1 + m] -= lij * M[m * J1 + j];
        }
        __syncwarp(FULL);
    }
    for (int i = 0; i < J1; ++i) {  // L y = rhs
        const double yi = rhs[i] * dinv[i];
        __syncwarp(FULL);
        if (lane == i) rhs[i] = yi;
        if (lane > i && lane < J1) rhs[lane] -= M[lane * J1 + i] * yi;
        __syncwarp(FULL);
    }
    for (int i = J1 - 1; i >= 0; --i) {  // L^T u = y
        const double ui = rhs[i] * dinv[i];
        __syncwarp(FULL);
        if (lane == i) rhs[i] = ui;
        if (lane < i) rhs[lane] -= M[i * J1 + lane] * ui;
        __syncwarp(FULL);
    }
    if (lane < J1) u_out[lane] = (float)rhs[lane];
    if (lane == 0) *status = 0;
}

__global__ void k_cosine(const float *__restrict__ U1, int32_t I1, int32_t J1,
                         const float *__restrict__ u, float *__restrict__ score) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I1) return;
    float nu = 0.f, d = 0.f, nr = 0.f;
    for (int p = 0; p < J1; ++p) {
        const float x = U1[(int64_t)i * J1 + p], y = u[p];
        d = fmaf(x, y, d);
        nr = fmaf(x, x, nr);
        nu = fmaf(y, y, nu);
    }
    score[i] = (nr > 0.f && nu > 0.f) ? d / (sqrtf(nr) * sqrtf(nu)) : 0.f;
}

// one CTA: k rounds of (largest score, lowest index) over the unpicked rows
__global__ void __launch_bounds__(1024)
    k_topk(const float *__restrict__ score, int32_t I1, int32_t k, int32_t *__restrict__ idx_out,
           float *__restrict__ score_out, uint8_t *__restrict__ taken) {
    __shared__ float ws[32];
    __shared__ int32_t wi[32];
    for (int32_t i = threadIdx.x; i < I1; i += blockDim.x) taken[i] = 0;
    __syncthreads();
    for (int32_t round = 0; round < k; ++round) {
        float bs = -INFINITY;
        int32_t bi = INT32_MAX;
        for (int32_t i = threadIdx.x; i < I1; i += blockDim.x) {
            if (taken[i]) continue;
            const float s = score[i];
            if (s > bs || (s == bs && i < bi)) {
                bs = s;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, bs, o);
            const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (os > bs || (os == bs && oi < bi)) {
                bs = os;
                bi = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            ws[threadIdx.x >> 5] = bs;
            wi[threadIdx.x >> 5] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float b = -INFINITY;
            int32_t ix = INT32_MAX;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (ws[w] > b || (ws[w] == b && wi[w] < ix)) {
                    b = ws[w];
                    ix = wi[w];
                }
            idx_out[round] = ix;
            score_out[round] = b;
            taken[ix] = 1;
        }
        __syncthreads();
    }
}

}  // namespace

int64_t foldin_parts(int64_t n) { return std::max<int64_t>(1, ceil_div(n, kFoldChunk)); }

cudaError_t launch_wtable(Ctx *c, float *table) {
    const int64_t rows = (int64_t)c->d.I2 * c->d.I3;
    k_wtable<<<ceil_div(rows, 128), 128, sizeof(float) * c->PI, c->stream>>>(
        c->G, c->U[1], c->U[2], c->d.I2, c->d.I3, c->d.J1, c->d.J2, c->d.J3, table);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_foldin(Ctx *c, cudaStream_t st, const int2 *jk, const float *val, int64_t n,
                          const float *table, float *part, float *u_out, int32_t *status, int32_t *flag,
                          int32_t *flag_out) {
    const int64_t np = foldin_parts(n);
    k_foldin_partial<<<(unsigned)np, kFoldThreads, 0, st>>>(jk, val, n, kFoldChunk, table, c->d.I2, c->d.I3,
                                                            c->d.J1, part, flag);
    k_foldin_solve<<<1, kFoldThreads, 0, st>>>(part, (int32_t)np, c->d.J1, c->cfg.lambda, u_out, status, flag,
                                               flag_out);
    c->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_topk(Ctx *c, cudaStream_t st, const float *u, int32_t k, float *score,
                        uint8_t *taken, int32_t *idx_out, float *score_out) {
    k_cosine<<<ceil_div(c->d.I1, 256), 256, 0, st>>>(c->U[0], c->d.I1, c->d.J1, u, score);
    k_topk<<<1, 1024, 0, st>>>(score, c->d.I1, k, idx_out, score_out, taken);
    c->launches += 2;
    return cudaGetLastError();
}

}  // namespace snect
