// Fast sweep of Alg. 1 for large problems: wave-synchronous proximal updates.
//
// Alg. 1 updates rows and core per entry, lock-free, with a few dozen CPU workers.  A GPU
// keeps 10^4 - 10^5 entries in flight; summing that many per-entry steps on one row (a hot
// gene is in every (patient, platform) pair) or on the core (every entry) diverges.  So the
// visit order is cut into waves; inside a wave every gradient is evaluated at the wave-start
// parameters (no entry waits for another, nothing is locked), and at the end of the wave
// each parameter block takes one proximal (implicit) step
//     theta <- theta - (H + I/lr)^{-1} g,
// g = the summed gradient of the wave's entries, H = a bound of their curvature:
//   * patient / gene row: H ~ h I with h = sum_e (||v_e||^2 + lambda/|Omega^{n,i}|), the trace
//     of the row's Gauss-Newton matrix (an upper bound of its top eigenvalue);
//   * platform row k: H = n_k G_(3) (Ma kron Mb) G_(3)^T + n_k lambda/|Omega^{3,k}| I, a J3 x J3
//     Cholesky solve (Ma, Mb: second moments of the patient and gene rows over the entries);
//   * core: H ~ lambda_max(sum_k n_k c_k c_k^T) lambda_max(Ma) lambda_max(Mb) I.
// With few entries per wave (lr * h << 1) the step is the summed per-entry step of Alg. 1;
// with many it tends to the Newton step of the wave's quadratic, so it stays stable for any
// wave size.
//
// Inside a wave the entries are grouped by platform, so within a tile c_k is fixed and the
// contraction uses Gc = G x3 c_k (J1 x J2):
//   v  = Gc b,  w2 = Gc^T a,  x~ = a . v,  r = x~ - x
//   g(u^(1)_i) += r v + lambda/|Omega^{1,i}| a,   g(u^(2)_j) += r w2 + lambda/|Omega^{2,j}| b
// and both dense gradients come from one J1 x J2 matrix per platform,
//   M_k = sum_{entries of platform k} r a b^T:
//   dG_pqr = sum_k M_k[p,q] c_k[r] + n lambda/|Omega| g_pqr
//   dc_k[r] = sum_pq g_pqr M_k[p,q] + n_k lambda/|Omega^{3,k}| c_k[r].
// M_k is accumulated per CTA in registers over staged tiles (one thread per 2 x 2 block and
// entry slice) and merged into global memory once per platform change.
#include "contract.cuh"

namespace snect {

namespace {

constexpr int kFastThreads = kFastTile;  // one entry per thread per tile
constexpr int kGramRows = 128;

__host__ __device__ constexpr int even_up(int x) { return (x + 1) & ~1; }
__host__ __device__ constexpr int align4(int x) { return (x + 3) & ~3; }

struct FastArgs {
    const Rec *rec;
    const int32_t *tile_start, *tile_len, *tile_k;
    int32_t n_tiles;
    int32_t *ctr;
    Dims d;
    const float *G;
    const float *U1, *U2, *U3;
    const int32_t *cnt1, *cnt2;
    float lam;
    float *macc;
    float *gA, *gB;  // per row: J_n gradient sums + 1 curvature sum
};

template <int CJ1, int CJ2, int CJ3>
__global__ void __launch_bounds__(kFastThreads) k_fast_sweep(FastArgs A) {
    const int J1 = CJ1 ? CJ1 : A.d.J1, J2 = CJ2 ? CJ2 : A.d.J2, J3 = CJ3 ? CJ3 : A.d.J3;
    const int J1P = even_up(J1), J2P = even_up(J2);
    const int PI = J1 * J2 * J3;
    extern __shared__ __align__(16) float sm[];
    float *sG = sm;                            // PI
    float *sGc = sG + align4(PI);              // J1*J2 (G x3 c_k)
    float *sRA = sGc + align4(J1 * J2);        // kFastThreads * J1P : r a  (8-byte aligned rows)
    float *sB = sRA + kFastThreads * J1P;      // kFastThreads * J2P : b
    float *sRed = sB + kFastThreads * J2P;     // kFastThreads * 4
    __shared__ int sTile;
    const int tid = threadIdx.x;
    for (int t = tid; t < PI; t += kFastThreads) sG[t] = A.G[t];

    // M_k accumulation layout: 2x2 blocks of (p, q), entry slices
    const int nbq = J2P / 2, NB = (J1P / 2) * nbq;
    const int S = NB >= kFastThreads ? 1 : kFastThreads / NB;
    const int L = (kFastThreads + S - 1) / S;
    const int my_b = tid % NB, my_s = tid / NB;
    const bool active = my_s < S;
    const int bp = (my_b / nbq) * 2, bq = (my_b % nbq) * 2;
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;

    int cur_k = -1;
    for (;;) {
        __syncthreads();  // previous tile fully consumed (sTile, sRA, sB, sGc)
        if (tid == 0) sTile = atomicAdd(A.ctr, 1);
        __syncthreads();
        const int t = sTile;
        const bool done = t >= A.n_tiles;
        const int k = done ? -1 : A.tile_k[t];
        if (k != cur_k) {
            if (cur_k >= 0) {  // merge this CTA's M_k
                if (active) {
                    float *o = sRed + (my_s * NB + my_b) * 4;
                    o[0] = acc0;
                    o[1] = acc1;
                    o[2] = acc2;
                    o[3] = acc3;
                }
                __syncthreads();
                for (int s = tid; s < NB * 4; s += kFastThreads) {
                    const int b = s >> 2, i = s & 3;
                    const int p = (b / nbq) * 2 + (i >> 1), q = (b % nbq) * 2 + (i & 1);
                    if (p < J1 && q < J2) {
                        float sum = 0.f;
                        for (int sl = 0; sl < S; ++sl) sum += sRed[(sl * NB + b) * 4 + i];
                        atomicAdd(A.macc + ((int64_t)cur_k * J1 + p) * J2 + q, sum);
                    }
                }
                acc0 = acc1 = acc2 = acc3 = 0.f;
            }
            if (done) break;
            const float *ck = A.U3 + (int64_t)k * J3;
            for (int s = tid; s < J1 * J2; s += kFastThreads) {
                float g = 0.f;
                for (int r = 0; r < J3; ++r) g = fmaf(sG[s * J3 + r], ck[r], g);
                sGc[s] = g;
            }
            cur_k = k;
            __syncthreads();
        }
        const int n_e = A.tile_len[t];
        float *ra = sRA + tid * J1P;
        float *bb = sB + tid * J2P;
        if (tid < n_e) {
            const Rec e = A.rec[A.tile_start[t] + tid];
            float a[RankCap<CJ1>::value], b[RankCap<CJ2>::value];
            float v[RankCap<CJ1>::value], w2[RankCap<CJ2>::value];
            const float *ua = A.U1 + (int64_t)e.i * J1;
            const float *ub = A.U2 + (int64_t)e.j * J2;
#pragma unroll
            for (int p = 0; p < J1; ++p) a[p] = __ldcg(ua + p);
#pragma unroll
            for (int q = 0; q < J2; ++q) {
                b[q] = __ldcg(ub + q);
                w2[q] = 0.f;
            }
#pragma unroll
            for (int p = 0; p < J1; ++p) {
                float vp = 0.f;
#pragma unroll
                for (int q = 0; q < J2; ++q) {
                    const float g = sGc[p * J2 + q];
                    vp = fmaf(g, b[q], vp);
                    w2[q] = fmaf(a[p], g, w2[q]);
                }
                v[p] = vp;
            }
            float xt = 0.f;
#pragma unroll
            for (int p = 0; p < J1; ++p) xt = fmaf(a[p], v[p], xt);
            const float r = xt - e.x;
            const float la = A.lam / (float)A.cnt1[e.i], lb = A.lam / (float)A.cnt2[e.j];
            // row accumulators: [gradient (J), curvature, zero padding] in float4 groups
            constexpr int RA = (RankCap<CJ1>::value + 4) & ~3, RB = (RankCap<CJ2>::value + 4) & ~3;
            const int RS1 = (J1 + 4) & ~3, RS2 = (J2 + 4) & ~3;
            float gva[RA], gvb[RB];
            float hv = la, hw = lb;
#pragma unroll
            for (int p = 0; p < J1; ++p) {
                gva[p] = fmaf(r, v[p], la * a[p]);
                hv = fmaf(v[p], v[p], hv);
                ra[p] = r * a[p];
            }
            gva[J1] = hv;
#pragma unroll
            for (int p = J1 + 1; p < RS1; ++p) gva[p] = 0.f;
#pragma unroll
            for (int q = 0; q < J2; ++q) {
                gvb[q] = fmaf(r, w2[q], lb * b[q]);
                hw = fmaf(w2[q], w2[q], hw);
                bb[q] = b[q];
            }
            gvb[J2] = hw;
#pragma unroll
            for (int q = J2 + 1; q < RS2; ++q) gvb[q] = 0.f;
            float4 *ga = reinterpret_cast<float4 *>(A.gA + (int64_t)e.i * RS1);
            float4 *gb = reinterpret_cast<float4 *>(A.gB + (int64_t)e.j * RS2);
#pragma unroll
            for (int t = 0; t < RS1 / 4; ++t)
                atomicAdd(ga + t, make_float4(gva[4 * t], gva[4 * t + 1], gva[4 * t + 2], gva[4 * t + 3]));
#pragma unroll
            for (int t = 0; t < RS2 / 4; ++t)
                atomicAdd(gb + t, make_float4(gvb[4 * t], gvb[4 * t + 1], gvb[4 * t + 2], gvb[4 * t + 3]));
            if (J1P != J1) ra[J1] = 0.f;
            if (J2P != J2) bb[J2] = 0.f;
        } else {
            for (int p = 0; p < J1P; ++p) ra[p] = 0.f;
            for (int q = 0; q < J2P; ++q) bb[q] = 0.f;
        }
        __syncthreads();
        if (active) {
            const int e1 = min(kFastThreads, (my_s + 1) * L);
            for (int e = my_s * L; e < e1; ++e) {
                const float2 x = *reinterpret_cast<const float2 *>(sRA + e * J1P + bp);
                const float2 y = *reinterpret_cast<const float2 *>(sB + e * J2P + bq);
                acc0 = fmaf(x.x, y.x, acc0);
                acc1 = fmaf(x.x, y.y, acc1);
                acc2 = fmaf(x.y, y.x, acc2);
                acc3 = fmaf(x.y, y.y, acc3);
            }
        }
    }
}

// Patient / gene rows at the end of a wave: u <- u - g / (1/lr + h), accumulators cleared;
// then the count-weighted second moments of the updated rows into gram_out:
// [0 .. J1^2) = sum_i cnt1_i/n a_i a_i^T, [J1^2 .. J1^2 + J2^2) = sum_j cnt2_j/n b_j b_j^T.
__device__ void wave_rows(int blk, float *__restrict__ U1, float *__restrict__ U2, float *__restrict__ gA,
                          float *__restrict__ gB, const int32_t *__restrict__ cnt1,
                          const int32_t *__restrict__ cnt2, const Dims &d, float inv_lr, float inv_n,
                          int32_t nb1, float *__restrict__ gram_out, float *rows, float *wts) {
    const bool first = blk < nb1;
    const int J = first ? d.J1 : d.J2;
    const int RS = (J + 4) & ~3;
    const int I = first ? d.I1 : d.I2;
    float *U = first ? U1 : U2;
    float *g = first ? gA : gB;
    const int32_t *cnt = first ? cnt1 : cnt2;
    const int64_t r0 = (int64_t)(first ? blk : blk - nb1) * kGramRows;
    const int64_t left = (int64_t)I - r0;
    const int nr = left < kGramRows ? (int)left : kGramRows;
    if (nr <= 0) return;
    for (int t = threadIdx.x; t < nr * J; t += blockDim.x) {
        const int i = t / J, q = t % J;
        const int64_t row = r0 + i;
        float *gr = g + row * RS;
        const float h = gr[J];
        float u = U[row * J + q];
        if (h > 0.f) {
            u -= gr[q] / (inv_lr + h);
            U[row * J + q] = u;
        }
        gr[q] = 0.f;
        rows[t] = u;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
        g[(r0 + t) * RS + J] = 0.f;
        wts[t] = (float)cnt[r0 + t] * inv_n;
    }
    __syncthreads();
    float *out = gram_out + (first ? 0 : d.J1 * d.J1);
    for (int s = threadIdx.x; s < J * J; s += blockDim.x) {
        const int p = s / J, q = s % J;
        float acc = 0.f;
        for (int i = 0; i < nr; ++i) acc = fmaf(wts[i] * rows[i * J + p], rows[i * J + q], acc);
        atomicAdd(out + s, acc);
    }
}

// largest eigenvalue of a symmetric PSD n x n matrix (n <= 32) by power iteration, one warp,
// warm-started from the vector of the previous wave (vec, n floats, kept in global memory)
__device__ float warp_top_eig(const float *M, int n, float *vec) {
    const int lane = threadIdx.x & 31;
    float v = lane < n ? vec[lane] : 0.f;
    float v2 = v * v;
#pragma unroll
    for (int o = 16; o; o >>= 1) v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    if (!(v2 > 0.f)) {
        v = lane < n ? rsqrtf((float)n) : 0.f;
    } else {
        v *= rsqrtf(v2);
    }
    float lam = 0.f;
    for (int it = 0; it < 12; ++it) {
        float y = 0.f;
        for (int q = 0; q < n; ++q) {
            const float vq = __shfl_sync(0xffffffffu, v, q);
            if (lane < n) y = fmaf(M[lane * n + q], vq, y);
        }
        float nn = y * y;
#pragma unroll
        for (int o = 16; o; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
        const float norm = sqrtf(nn);
        if (!(norm > 0.f)) return 0.f;
        lam = norm;
        v = y / norm;
    }
    if (lane < n) vec[lane] = v;
    // with a few iterations |Mv| can sit slightly below the top eigenvalue; 5% headroom keeps
    // the core step on the safe side
    return 1.05f * lam;
}

struct DenseArgs {
    Dims d;
    float *G, *U3;
    const int32_t *cnt3;
    float *macc;
    float *gram_in;   // moments used for the curvature (cleared after use)
    float *eigvec;    // 3 * kMaxRank warm-start vectors
    const float *nk;  // entries of this wave per platform
    float n_wave, lam, lr, lam_core;
};

// The proximal step of the core and the platform rows after a wave (one CTA).
__device__ void wave_dense(const DenseArgs &A, float *sm) {
    const Dims &d = A.d;
    const int J1 = d.J1, J2 = d.J2, J3 = d.J3, I3 = d.I3, PI = J1 * J2 * J3, Q = J1 * J2;
    float *sG = sm;                  // PI
    float *sX = sG + PI;             // PI: X[r][p][q'] = sum_p' Ma[p][p'] g(p', q', r)
    float *sT = sX + PI;             // PI: T[r][p][q] = (Ma G_r Mb)[p][q]
    float *sC = sT + PI;             // I3*J3
    float *sCn = sC + I3 * J3;       // J3*J3
    float *sH = sCn + J3 * J3;       // J3*J3
    float *sGk = sH + J3 * J3;       // I3*J3 platform gradients
    float *sDel = sGk + I3 * J3;     // I3*J3 platform steps
    float *sMa = sDel + I3 * J3;     // J1*J1
    float *sMb = sMa + J1 * J1;      // J2*J2
    float *sEig = sMb + J2 * J2;     // 3
    const int tid = threadIdx.x;
    for (int s = tid; s < PI; s += blockDim.x) sG[s] = A.G[s];
    for (int s = tid; s < I3 * J3; s += blockDim.x) sC[s] = A.U3[s];
    for (int s = tid; s < J1 * J1; s += blockDim.x) sMa[s] = A.gram_in[s];
    for (int s = tid; s < J2 * J2; s += blockDim.x) sMb[s] = A.gram_in[J1 * J1 + s];
    __syncthreads();
    for (int s = tid; s < J3 * J3; s += blockDim.x) {
        const int r = s / J3, t = s % J3;
        float a = 0.f;
        for (int k = 0; k < I3; ++k) a = fmaf(A.nk[k] * sC[k * J3 + r], sC[k * J3 + t], a);
        sCn[s] = a;
    }
    for (int s = tid; s < PI; s += blockDim.x) {  // s = (r, p, q')
        const int r = s / Q, p = (s / J2) % J1, q = s % J2;
        float a = 0.f;
        for (int pp = 0; pp < J1; ++pp) a = fmaf(sMa[p * J1 + pp], sG[(pp * J2 + q) * J3 + r], a);
        sX[s] = a;
    }
    for (int s = tid; s < I3 * J3; s += blockDim.x) {
        const int k = s / J3, r = s % J3;
        float a = 0.f;
        const float *M = A.macc + (int64_t)k * Q;
        for (int pq = 0; pq < Q; ++pq) a = fmaf(sG[pq * J3 + r], M[pq], a);
        const float reg = A.cnt3[k] > 0 ? A.nk[k] * A.lam / (float)A.cnt3[k] : 0.f;
        sGk[s] = fmaf(reg, sC[s], a);
    }
    __syncthreads();
    const int warp = tid >> 5;
    if (warp < 3) {
        const float *M = warp == 0 ? sMa : (warp == 1 ? sMb : sCn);
        const int n = warp == 0 ? J1 : (warp == 1 ? J2 : J3);
        const float e = warp_top_eig(M, n, A.eigvec + warp * kMaxRank);
        if ((tid & 31) == 0) sEig[warp] = e;
    }
    for (int s = tid; s < PI; s += blockDim.x) {  // T[r][p][q] = sum_q' X[r][p][q'] Mb[q'][q]
        const int r = s / Q, p = (s / J2) % J1, q = s % J2;
        float a = 0.f;
        for (int qq = 0; qq < J2; ++qq) a = fmaf(sX[(r * J1 + p) * J2 + qq], sMb[qq * J2 + q], a);
        sT[s] = a;
    }
    __syncthreads();
    for (int s = tid; s < J3 * J3; s += blockDim.x) {  // H[r][t] = sum_pq g(p,q,r) T[t][p][q]
        const int r = s / J3, t = s % J3;
        float a = 0.f;
        for (int pq = 0; pq < Q; ++pq) a = fmaf(sG[pq * J3 + r], sT[t * Q + pq], a);
        sH[s] = a;
    }
    __syncthreads();
    if (tid < I3) {  // platform row k: (nk H + (nk lambda/cnt3 + 1/lr) I) delta = g_k, Cholesky
        const int k = tid;
        float *del = sDel + k * J3;
        const float nk = A.nk[k];
        if (nk > 0.f) {
            float Ak[kMaxRank * kMaxRank];  // J3 <= 32; only I3 threads hold one
            const float reg = A.cnt3[k] > 0 ? nk * A.lam / (float)A.cnt3[k] : 0.f;
            for (int r = 0; r < J3; ++r)
                for (int t = 0; t < J3; ++t)
                    Ak[r * J3 + t] = nk * sH[r * J3 + t] + (r == t ? reg + 1.f / A.lr : 0.f);
            bool ok = true;
            for (int j = 0; j < J3 && ok; ++j) {
                float dd = Ak[j * J3 + j];
                for (int q = 0; q < j; ++q) dd -= Ak[j * J3 + q] * Ak[j * J3 + q];
                if (!(dd > 0.f)) {
                    ok = false;
                    break;
                }
                dd = sqrtf(dd);
                Ak[j * J3 + j] = dd;
                for (int i = j + 1; i < J3; ++i) {
                    float x = Ak[i * J3 + j];
                    for (int q = 0; q < j; ++q) x -= Ak[i * J3 + q] * Ak[j * J3 + q];
                    Ak[i * J3 + j] = x / dd;
                }
            }
            for (int i = 0; i < J3; ++i) del[i] = sGk[k * J3 + i];
            if (ok) {
                for (int i = 0; i < J3; ++i) {
                    float x = del[i];
                    for (int q = 0; q < i; ++q) x -= Ak[i * J3 + q] * del[q];
                    del[i] = x / Ak[i * J3 + i];
                }
                for (int i = J3 - 1; i >= 0; --i) {
                    float x = del[i];
                    for (int q = i + 1; q < J3; ++q) x -= Ak[q * J3 + i] * del[q];
                    del[i] = x / Ak[i * J3 + i];
                }
            } else {  // not reached for an SPD matrix; the plain summed step
                for (int i = 0; i < J3; ++i) del[i] *= A.lr;
            }
        } else {
            for (int i = 0; i < J3; ++i) del[i] = 0.f;
        }
    }
    __syncthreads();
    const float curv = sEig[0] * sEig[1] * sEig[2];
    const float eta = 1.f / (1.f / A.lr + curv);
    for (int s = tid; s < PI; s += blockDim.x) {
        const int pq = s / J3, r = s % J3;
        float a = 0.f;
        for (int k = 0; k < I3; ++k) a = fmaf(A.macc[(int64_t)k * Q + pq], sC[k * J3 + r], a);
        A.G[s] = sG[s] - eta * fmaf(A.n_wave * A.lam_core, sG[s], a);
    }
    for (int s = tid; s < I3 * J3; s += blockDim.x) A.U3[s] = sC[s] - sDel[s];
    __syncthreads();
    for (int s = tid; s < I3 * Q; s += blockDim.x) A.macc[s] = 0.f;
    for (int s = tid; s < J1 * J1 + J2 * J2; s += blockDim.x) A.gram_in[s] = 0.f;
}

// End of a wave: CTA 0 takes the proximal step of the core and platform rows (curvature from
// the previous wave's moments, gram_prev); CTAs 1.. update the patient and gene rows and
// accumulate the new moments into gram_next.  With do_dense = 0 only the moments are formed
// (set-up: every accumulator is zero, so no row moves).
__global__ void __launch_bounds__(256)
    k_fast_wave_end(DenseArgs A, int do_dense, float *__restrict__ U1, float *__restrict__ U2,
                    float *__restrict__ gA, float *__restrict__ gB, const int32_t *__restrict__ cnt1,
                    const int32_t *__restrict__ cnt2, float inv_n, int32_t nb1,
                    float *__restrict__ gram_next) {
    extern __shared__ __align__(16) float smw[];
    if (blockIdx.x == 0) {
        if (do_dense) wave_dense(A, smw);
        return;
    }
    wave_rows(blockIdx.x - 1, U1, U2, gA, gB, cnt1, cnt2, A.d, 1.f / A.lr, inv_n, nb1, gram_next, smw,
              smw + kGramRows * kMaxRank);
}

template <int CJ1, int CJ2, int CJ3>
size_t sweep_smem(const Ctx *c) {
    const int J1P = even_up(c->d.J1), J2P = even_up(c->d.J2);
    return sizeof(float) * ((size_t)align4(c->PI) + align4(c->d.J1 * c->d.J2) +
                            (size_t)kFastThreads * (J1P + J2P + 4));
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t init_sweep(Ctx *c) {
    const size_t smem = sweep_smem<CJ1, CJ2, CJ3>(c);
    cudaError_t e = cudaFuncSetAttribute(k_fast_sweep<CJ1, CJ2, CJ3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fast_sweep<CJ1, CJ2, CJ3>, kFastThreads, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return e;
    c->fast_grid = std::max(1, per_sm) * sms;
    return cudaSuccess;
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t run_sweep(Ctx *c, int64_t w) {
    const int64_t t0 = c->wave_tile[w], nt = c->wave_tile[w + 1] - t0;
    FastArgs A;
    A.rec = c->rec;
    A.tile_start = c->tile_start + t0;
    A.tile_len = c->tile_len + t0;
    A.tile_k = c->tile_k + t0;
    A.n_tiles = (int32_t)nt;
    A.ctr = c->tile_ctr + w;
    A.d = c->d;
    A.G = c->G;
    A.U1 = c->U[0];
    A.U2 = c->U[1];
    A.U3 = c->U[2];
    A.cnt1 = c->cnt[0];
    A.cnt2 = c->cnt[1];
    A.lam = c->cfg.lambda;
    A.macc = c->macc;
    A.gA = c->gacc[0];
    A.gB = c->gacc[1];
    if (nt == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>(c->fast_grid, nt);
    k_fast_sweep<CJ1, CJ2, CJ3><<<grid, kFastThreads, sweep_smem<CJ1, CJ2, CJ3>(c), c->stream>>>(A);
    c->launches++;
    return cudaGetLastError();
}

size_t wave_end_smem(const Ctx *c) {
    const Dims &d = c->d;
    const size_t dense = 3 * (size_t)c->PI + 3 * d.I3 * d.J3 + 2 * d.J3 * d.J3 + d.J1 * d.J1 + d.J2 * d.J2 + 4;
    const size_t rows = (size_t)kGramRows * kMaxRank + kGramRows;
    return sizeof(float) * std::max(dense, rows);
}

DenseArgs dense_args(Ctx *c, int64_t w, int parity) {
    DenseArgs A;
    A.d = c->d;
    A.G = c->G;
    A.U3 = c->U[2];
    A.cnt3 = c->cnt[2];
    A.macc = c->macc;
    A.gram_in = c->gram + (size_t)(parity ^ 1) * c->gram_stride;
    A.eigvec = c->gram + 2 * (size_t)c->gram_stride;
    A.nk = c->wave_nk + (w >= 0 ? w : 0) * c->d.I3;
    A.n_wave = w >= 0 ? (float)c->wave_len[w] : 0.f;
    A.lam = c->cfg.lambda;
    A.lr = c->cfg.lr;
    A.lam_core = c->nnz ? c->cfg.lambda / (float)c->nnz : 0.f;
    return A;
}

cudaError_t launch_wave_end(Ctx *c, int64_t w, int parity, int do_dense) {
    const Dims &d = c->d;
    const int nb1 = ceil_div(d.I1, kGramRows), nb2 = ceil_div(d.I2, kGramRows);
    k_fast_wave_end<<<1 + nb1 + nb2, 256, wave_end_smem(c), c->stream>>>(
        dense_args(c, w, parity), do_dense, c->U[0], c->U[1], c->gacc[0], c->gacc[1], c->cnt[0], c->cnt[1],
        c->nnz ? 1.f / (float)c->nnz : 0.f, nb1, c->gram + (size_t)parity * c->gram_stride);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace

int init_fast(Ctx *c) {
    const Dims &d = c->d;
    SNECT_CUDA(c, cudaMalloc((void **)&c->tile_ctr, sizeof(int32_t) * std::max<int64_t>(1, c->n_waves)));
    SNECT_CUDA(c, cudaMalloc((void **)&c->macc, sizeof(float) * d.I3 * d.J1 * d.J2));
    SNECT_CUDA(c, cudaMemsetAsync(c->macc, 0, sizeof(float) * d.I3 * d.J1 * d.J2, c->stream));
    // moments: two buffers (this wave's, the previous wave's) + 3 eigenvector warm starts
    c->gram_stride = ((int64_t)d.J1 * d.J1 + d.J2 * d.J2 + 3) & ~3;
    const int64_t gf = 2 * c->gram_stride + 3 * kMaxRank;
    SNECT_CUDA(c, cudaMalloc((void **)&c->gram, sizeof(float) * gf));
    SNECT_CUDA(c, cudaMemsetAsync(c->gram, 0, sizeof(float) * gf, c->stream));
    for (int n = 0; n < 2; ++n) {
        const int64_t nf = (int64_t)(n ? d.I2 : d.I1) * ((((n ? d.J2 : d.J1) + 4)) & ~3);
        SNECT_CUDA(c, cudaMalloc((void **)&c->gacc[n], sizeof(float) * nf));
        SNECT_CUDA(c, cudaMemsetAsync(c->gacc[n], 0, sizeof(float) * nf, c->stream));
    }
    SNECT_CUDA(c, SNECT_DISPATCH_RANKS(d.J1, d.J2, d.J3, init_sweep, c));
    SNECT_CUDA(c, cudaFuncSetAttribute(k_fast_wave_end, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)wave_end_smem(c)));
    // the first wave's curvature: moments of the initial rows into the odd buffer
    SNECT_CUDA(c, launch_wave_end(c, -1, 1, 0));
    return timing_events(c, c->n_waves);
}

int enqueue_fast_epoch(Ctx *c) {
    if (c->n_waves == 0) return SNECT_OK;
    const Dims &d = c->d;
    SNECT_CUDA(c, cudaMemsetAsync(c->tile_ctr, 0, sizeof(int32_t) * c->n_waves, c->stream));
    // n_waves is even, so wave w's parity (w % 2) continues across epochs
    for (int64_t w = 0; w < c->n_waves; ++w) {
        SNECT_CUDA(c, cudaEventRecordWithFlags(c->ev_begin[w], c->stream, cudaEventRecordExternal));
        SNECT_CUDA(c, SNECT_DISPATCH_RANKS(d.J1, d.J2, d.J3, run_sweep, c, w));
        SNECT_CUDA(c, cudaEventRecordWithFlags(c->ev_end[w], c->stream, cudaEventRecordExternal));
        SNECT_CUDA(c, launch_wave_end(c, w, (int)(w & 1), 1));
    }
    return SNECT_OK;
}

void free_fast(Ctx *c) {
    auto f = [](auto *&p) {
        if (p) cudaFree(p);
        p = nullptr;
    };
    f(c->tile_start);
    f(c->tile_len);
    f(c->tile_k);
    f(c->tile_ctr);
    f(c->wave_nk);
    f(c->macc);
    f(c->gram);
    f(c->gacc[0]);
    f(c->gacc[1]);
}

}  // namespace snect
