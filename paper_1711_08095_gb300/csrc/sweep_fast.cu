// Fast sweep of Alg. 1 for large problems: wave-synchronous proximal updates.
//
// Alg. 1 updates rows and core per entry, lock-free, with a few dozen CPU workers.  A GPU
// keeps 10^4 - 10^5 entries in flight; summing that many per-entry steps on one row (a hot
// gene is in every (patient, platform) pair) or on the core (every entry) diverges.  So the
// visit order is cut into waves; inside a wave every gradient is evaluated at the wave-start
// parameters (no entry waits for another, nothing is locked), and at the end of the wave
// each parameter block takes one proximal (implicit) step
//     theta <- theta - (H + I/lr)^{-1} g,
// g = the summed gradient of the wave's entries, H their Gauss-Newton curvature, with the
// rows of one entry's other modes replaced by their second moments over the training entries
// (Ma = E[a a^T], Mb = E[b b^T]):
//   * patient row i:  H = sum_k n_ik Gc_k Mb Gc_k^T + n_i lambda/|Omega^{1,i}| I   (J1 x J1)
//   * gene row j:     H = sum_k n_jk Gc_k^T Ma Gc_k + n_j lambda/|Omega^{2,j}| I   (J2 x J2)
//     (n_ik: the row's entries of platform k in the wave; Cholesky, one thread per row for
//     compile-time ranks up to 16, else one warp per row)
//   * platform row k: H = n_k G_(3) (Ma kron Mb) G_(3)^T + n_k lambda/|Omega^{3,k}| I
//   * core:           H = Cn kron Mb kron Ma + n lambda/|Omega| I, Cn = sum_k n_k c_k c_k^T,
//     solved in the eigenbases of Ma, Mb, Cn (one-warp Jacobi, warm-started per wave).
// A direction of small curvature moves by lr * g, like the summed per-entry steps of Alg. 1;
// one of large curvature moves by the Newton step of the wave's quadratic.  Every wave size
// is stable.
//
// Inside a wave the entries are grouped by platform, so within a tile c_k is fixed and the
// contraction uses Gc = G x3 c_k (J1 x J2):
//   v  = Gc b,  w2 = Gc^T a,  x~ = a . v,  r = x~ - x
//   g(u^(1)_i) += r v,   g(u^(2)_j) += r w2   (the data term; a row's L2 term, the same for
//   each of its n entries in the wave, is added once at the wave end as n lambda/|Omega| u)
// and both dense gradients come from one J1 x J2 matrix per platform,
//   M_k = sum_{entries of platform k} r a b^T:
//   dG_pqr = sum_k M_k[p,q] c_k[r] + n lambda/|Omega| g_pqr
//   dc_k[r] = sum_pq g_pqr M_k[p,q] + n_k lambda/|Omega^{3,k}| c_k[r].
// M_k is accumulated per CTA in registers over staged tiles (one thread per 2 x 2 block and
// entry slice) and merged into global memory once per platform change.
#include <stdlib.h>
#include <string.h>

#include <type_traits>

#include "contract.cuh"
#include "tc.cuh"

namespace snect {

namespace {

constexpr int kFastThreads = kFastTile;  // one entry per thread per tile

__host__ __device__ constexpr int even_up(int x) { return (x + 1) & ~1; }
__host__ __device__ constexpr int align4(int x) { return (x + 3) & ~3; }

constexpr int kMaccStage = 8192;   // a wave's M_k staged in shared memory up to this size

struct DenseArgs {
    Dims d;
    float *G, *U3;
    const int32_t *cnt3;
    float *macc;
    float *gram_in;   // moments of the rows formed at the previous wave end (cleared after use)
    float *eigv;      // eigenvectors of Ma, Mb, Cn (J1^2 + J2^2 + J3^2), also the next warm start
    float *eigval;    // their eigenvalues (J1 + J2 + J3)
    float *ainv;      // inverses of the platform rows' systems (I3 x J3 x J3)
    int32_t *wave_counter;  // dense steps taken so far (selects the waves that re-decompose)
    float *curv;      // platform curvatures for this wave's row steps (I3 J1^2 + I3 J2^2)
    const float *nk;  // entries of this wave per platform
    float n_wave, lam, lr, lam_core;
};

// eigen tiles: row stride n_max + 1; the round tables of the Jacobi need 64 floats of scratch
__host__ __device__ inline int eig_ld(const Dims &d) {
    const int n = d.J1 > d.J2 ? d.J1 : d.J2;
    return (n > d.J3 ? n : d.J3) + 1;
}
__host__ __device__ inline int eig_tile(const Dims &d) {
    const int t = (eig_ld(d) - 1) * eig_ld(d);
    return t < 64 ? 64 : ((t + 3) & ~3);
}

// floats of shared memory of the two halves of the dense step
__host__ __device__ inline int64_t dense_pre_floats(const Dims &d) {
    const int64_t PI = (int64_t)d.J1 * d.J2 * d.J3;
    return 3 * PI + (int64_t)d.I3 * d.J3 + 2 * d.J3 * d.J3 + d.J1 * d.J1 + d.J2 * d.J2 + 9 * (int64_t)eig_tile(d) +
           (int64_t)d.I3 * d.J3 * d.J3;
}
__host__ __device__ inline int64_t dense_post_floats(const Dims &d) {
    const int64_t PI = (int64_t)d.J1 * d.J2 * d.J3, Q = (int64_t)d.J1 * d.J2;
    const int64_t stage = (int64_t)d.I3 * Q <= kMaccStage ? (int64_t)d.I3 * Q : 0;
    return 3 * PI + 3 * (int64_t)d.I3 * d.J3 + (int64_t)(d.J1 + d.J2 + d.J3) * (eig_ld(d) + 1) +
           (int64_t)d.I3 * d.J3 * d.J3 + 2 * (int64_t)d.I3 + stage;
}

struct FastArgs {
    const Rec *rec;
    const int32_t *tile_start, *tile_len, *tile_k;
    int32_t n_tiles;
    int32_t *ctr;
    Dims d;
    const float *G;
    const float *U1, *U2, *U3;
    float *macc;
    // per row: data-term gradient sums (J_n, padded to 4), then entries per platform (written
    // only when count_atomics is set)
    float *gA, *gB;
    int32_t rs1, rs2;  // row strides of gA, gB
    int32_t *err;      // set when a tensor-core wait gives up
    DenseArgs pre;     // the wave's dense pre-work (the first CTAs of the launch)
    int32_t count_atomics;  // 1: count each row's entries per platform with atomics (no table)
    int64_t e_first, e_count;  // the wave's entries: positions [e_first, e_first + e_count) of rec
    const __nv_bfloat16 *U2h;  // BF16 copy of the gene factor (the BF16-gather sweep)
};

// The wave-independent half of the dense step; part 0, 1, 2 split it over three CTAs, -1
// runs all of it in one.
template <int CJ1 = 0, int CJ2 = 0, int CJ3 = 0>
__device__ void dense_pre(const DenseArgs &A, float *sm, int part = -1);
constexpr int kPreCtas = 3;  // CTAs of a fast-sweep launch that take the dense pre-work

// Adds each run of equal patient indices in a warp to its patient row once.  The entries of a
// tile are sorted by patient within their wave and platform, so a patient's entries sit next
// to each other: segmented suffix sums by shuffles leave each run's total in its first lane,
// which adds it and the run's length (entries of platform k) to the row accumulator.  iv < 0
// marks a lane without an entry.  Every lane of the warp calls this.
template <int RA>
__device__ __forceinline__ void add_patient_runs(float (&g)[RA], int J, int iv, float *__restrict__ gA, int32_t rs,
                                                 int k, bool count) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int inext = __shfl_down_sync(FULL, iv, 1);
    if (__any_sync(FULL, lane < 31 && iv >= 0 && inext == iv)) {
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int io = __shfl_down_sync(FULL, iv, off);
            const bool same = lane + off < 32 && io == iv;
#pragma unroll
            for (int p = 0; p < RA; ++p) {
                if (p < J) {
                    const float o = __shfl_down_sync(FULL, g[p], off);
                    if (same) g[p] += o;
                }
            }
        }
    }
    const int iprev = __shfl_up_sync(FULL, iv, 1);
    const unsigned run = __match_any_sync(FULL, iv);
    if (iv >= 0 && (lane == 0 || iprev != iv)) {
        float *ga = gA + (int64_t)iv * rs;
        const int JA = (J + 3) & ~3;
#pragma unroll
        for (int t = 0; t < RA / 4; ++t)
            if (4 * t < JA)
                atomicAdd(reinterpret_cast<float4 *>(ga) + t, make_float4(g[4 * t], g[4 * t + 1], g[4 * t + 2], g[4 * t + 3]));
        if (count) atomicAdd(ga + JA + k, (float)__popc(run));
    }
}

// This thread's entry of a tile of platform k (valid: the tile has an entry for this thread);
// every thread of the CTA calls this.
// Gathers a, b (read-only during the sweep: cached loads), v = Gc b, w2 = Gc^T a, the
// residual, the row gradients (patient rows by runs, gene rows one atomic per entry), and
// stages r a and b in shared memory (ra, bb: this thread's rows) for the M_k accumulation.
template <int CJ1, int CJ2, int CJ3>
__device__ __forceinline__ void tile_entries(const FastArgs &A, const Rec &e, bool valid, int k,
                                             const float *__restrict__ sGc, float *ra, float *bb) {
    const int J1 = CJ1 ? CJ1 : A.d.J1, J2 = CJ2 ? CJ2 : A.d.J2;
    const int J1P = even_up(J1), J2P = even_up(J2);
    constexpr int RA = (RankCap<CJ1>::value + 3) & ~3, RB = (RankCap<CJ2>::value + 3) & ~3;
    const int JB = (J2 + 3) & ~3;
    float gva[RA];
#pragma unroll
    for (int p = 0; p < RA; ++p) gva[p] = 0.f;
    int iv = -1;
    if (valid) {
        iv = e.i;
        float a[RankCap<CJ1>::value], b[RankCap<CJ2>::value];
        float v[RankCap<CJ1>::value], w2[RankCap<CJ2>::value];
        const float *ua = A.U1 + (int64_t)e.i * J1;
        const float *ub = A.U2 + (int64_t)e.j * J2;
        // rows of even compile-time length load as float2 (row starts are 8-byte aligned)
        if constexpr (CJ1 > 0 && CJ1 % 2 == 0) {
#pragma unroll
            for (int p = 0; p < CJ1; p += 2) {
                const float2 t2 = __ldg(reinterpret_cast<const float2 *>(ua + p));
                a[p] = t2.x;
                a[p + 1] = t2.y;
            }
        } else {
#pragma unroll
            for (int p = 0; p < J1; ++p) a[p] = __ldg(ua + p);
        }
        if constexpr (CJ2 > 0 && CJ2 % 2 == 0) {
#pragma unroll
            for (int q = 0; q < CJ2; q += 2) {
                const float2 t2 = __ldg(reinterpret_cast<const float2 *>(ub + q));
                b[q] = t2.x;
                b[q + 1] = t2.y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < J2; ++q) b[q] = __ldg(ub + q);
        }
#pragma unroll
        for (int q = 0; q < J2; ++q) w2[q] = 0.f;
        if constexpr (CJ2 > 0 && CJ2 % 2 == 0) {  // Gc read as float2 pairs (broadcast)
#pragma unroll
            for (int p = 0; p < CJ1; ++p) {
                float vp = 0.f;
#pragma unroll
                for (int q = 0; q < CJ2; q += 2) {
                    const float2 g = *reinterpret_cast<const float2 *>(sGc + p * CJ2 + q);
                    vp = fmaf(g.x, b[q], vp);
                    vp = fmaf(g.y, b[q + 1], vp);
                    w2[q] = fmaf(a[p], g.x, w2[q]);
                    w2[q + 1] = fmaf(a[p], g.y, w2[q + 1]);
                }
                v[p] = vp;
            }
        } else {
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
        }
        float xt = 0.f;
#pragma unroll
        for (int p = 0; p < J1; ++p) xt = fmaf(a[p], v[p], xt);
        const float r = xt - e.x;
        // row accumulators: [data-term gradient (J, padded to 4), entries per platform (I3,
        // padded)]; the L2 term n lambda/|Omega| u of a row is added by the wave end
        float gvb[RB];
#pragma unroll
        for (int p = 0; p < J1; ++p) {
            gva[p] = r * v[p];
            ra[p] = r * a[p];
        }
#pragma unroll
        for (int q = 0; q < J2; ++q) {
            gvb[q] = r * w2[q];
            bb[q] = b[q];
        }
#pragma unroll
        for (int q = J2; q < JB; ++q) gvb[q] = 0.f;
        float *gb = A.gB + (int64_t)e.j * A.rs2;
#pragma unroll
        for (int t4 = 0; t4 < RB / 4; ++t4)
            if (4 * t4 < JB)
                atomicAdd(reinterpret_cast<float4 *>(gb) + t4,
                          make_float4(gvb[4 * t4], gvb[4 * t4 + 1], gvb[4 * t4 + 2], gvb[4 * t4 + 3]));
        if (A.count_atomics) atomicAdd(gb + JB + k, 1.f);
        if (J1P != J1) ra[J1] = 0.f;
        if (J2P != J2) bb[J2] = 0.f;
    } else {
        for (int p = 0; p < J1P; ++p) ra[p] = 0.f;
        for (int q = 0; q < J2P; ++q) bb[q] = 0.f;
    }
    add_patient_runs<RA>(gva, J1, iv, A.gA, A.rs1, k, A.count_atomics);
}

// M_k accumulation layout: 2 x 2 blocks of (p, q) and slices of the tile's entries.
struct MLayout {
    int nbq, NB, S, L, my_b, my_s, bp, bq;
    bool active;
    __device__ MLayout(int J1P, int J2P) {
        nbq = J2P / 2;
        NB = (J1P / 2) * nbq;
        S = NB >= kFastThreads ? 1 : kFastThreads / NB;
        L = (kFastThreads + S - 1) / S;
        my_b = threadIdx.x % NB;
        my_s = threadIdx.x / NB;
        active = my_s < S;
        bp = (my_b / nbq) * 2;
        bq = (my_b % nbq) * 2;
    }
};

// this thread's 2 x 2 block of M_k over its slice of the staged tile
__device__ __forceinline__ void m_accumulate(const MLayout &ml, const float *sRA, const float *sB, int J1P, int J2P,
                                             float &acc0, float &acc1, float &acc2, float &acc3) {
    if (!ml.active) return;
    const int e1 = min(kFastThreads, (ml.my_s + 1) * ml.L);
    for (int e = ml.my_s * ml.L; e < e1; ++e) {
        const float2 x = *reinterpret_cast<const float2 *>(sRA + e * J1P + ml.bp);
        const float2 y = *reinterpret_cast<const float2 *>(sB + e * J2P + ml.bq);
        acc0 = fmaf(x.x, y.x, acc0);
        acc1 = fmaf(x.x, y.y, acc1);
        acc2 = fmaf(x.y, y.x, acc2);
        acc3 = fmaf(x.y, y.y, acc3);
    }
}

// merges the CTA's M_k partial (2 x 2 blocks x slices, staged through sRed) into macc
__device__ __forceinline__ void m_merge(const MLayout &ml, float *sRed, float *__restrict__ macc, int J1, int J2,
                                        float &acc0, float &acc1, float &acc2, float &acc3) {
    if (ml.active) {
        float *o = sRed + (ml.my_s * ml.NB + ml.my_b) * 4;
        o[0] = acc0;
        o[1] = acc1;
        o[2] = acc2;
        o[3] = acc3;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < ml.NB * 4; s += kFastThreads) {
        const int b = s >> 2, i = s & 3;
        const int p = (b / ml.nbq) * 2 + (i >> 1), q = (b % ml.nbq) * 2 + (i & 1);
        if (p < J1 && q < J2) {
            float sum = 0.f;
            for (int sl = 0; sl < ml.S; ++sl) sum += sRed[(sl * ml.NB + b) * 4 + i];
            atomicAdd(macc + (p * J2 + q), sum);
        }
    }
    acc0 = acc1 = acc2 = acc3 = 0.f;
}

// Gc = G x3 c_k into shared memory
__device__ __forceinline__ void form_gc(const float *sG, const float *__restrict__ ck, float *sGc, int J1, int J2,
                                        int J3) {
    for (int s = threadIdx.x; s < J1 * J2; s += kFastThreads) {
        float g = 0.f;
        for (int r = 0; r < J3; ++r) g = fmaf(sG[s * J3 + r], ck[r], g);
        sGc[s] = g;
    }
}

// a tile's platform and this thread's record (fetched one tile ahead)
struct TileFetch {
    Rec e;
    int k;
    bool valid;
};

__device__ __forceinline__ TileFetch fetch_tile(const FastArgs &A, int t) {
    TileFetch f;
    f.k = -1;
    f.valid = false;
    f.e.i = f.e.j = f.e.k = 0;
    f.e.x = 0.f;
    if (t < A.n_tiles) {
        f.k = A.tile_k[t];
        f.valid = (int)threadIdx.x < A.tile_len[t];
        if (f.valid) {  // streamed once per epoch: evict-first
            const int4 v = __ldcs(reinterpret_cast<const int4 *>(A.rec + A.tile_start[t] + threadIdx.x));
            f.e.i = v.x;
            f.e.j = v.y;
            f.e.k = v.z;
            f.e.x = __int_as_float(v.w);
        }
    }
    return f;
}

// ---------------------------------------------------------------------------------------
// Per-patient factoring of a tile's contraction (compile-time J1, J2 <= 16).
//
// The entries of a tile share the platform k, and inside a wave and platform they are sorted
// by patient, so a warp's 32 entries fall into a few runs of one patient i each (a_i fixed).
// For a run the contraction factors through a_i:
//   w2 = Gc^T a_i (once per run),  x~_e = a_i^T Gc b_e = w2 . b_e,  r_e = x~_e - x_e
//   gene rows:    g(b_e) += r_e w2                                    (per entry)
//   s = sum_e r_e b_e                                                  (run sum)
//   patient row:  g(a_i) += Gc s                                      (= sum_e r_e Gc b_e)
//   M_k += a_i s^T                                                     (= sum_e r_e a_i b_e^T)
// (the rows' L2 terms are added at the wave end)
// so the per-entry work is O(J2) and the J1 x J2 products are paid once per run.  Vectors of
// the run are spread over the warp (lane l holds component l / 2) by recursive-halving
// reductions.

template <int CJ1, int CJ2>
__host__ __device__ constexpr bool runs_path() { return CJ1 > 0 && CJ2 > 0 && CJ1 <= 16 && CJ2 <= 16; }

// the statically partitioned sweep keeps Gc_k and M_k of every platform in shared memory
constexpr int kGcAll = 4096;

// sum over the 32 lanes of v[0..16): lane l returns the total of component l >> 1
__device__ __forceinline__ float reduce_scatter16(const float (&v)[16]) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float h8[8], h4[4], h2[2];
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
    for (int i = 0; i < 8; ++i) h8[i] = (b4 ? v[i + 8] : v[i]) + __shfl_xor_sync(FULL, b4 ? v[i] : v[i + 8], 16);
#pragma unroll
    for (int i = 0; i < 4; ++i) h4[i] = (b3 ? h8[i + 4] : h8[i]) + __shfl_xor_sync(FULL, b3 ? h8[i] : h8[i + 4], 8);
#pragma unroll
    for (int i = 0; i < 2; ++i) h2[i] = (b2 ? h4[i + 2] : h4[i]) + __shfl_xor_sync(FULL, b2 ? h4[i] : h4[i + 2], 4);
    float h = (b1 ? h2[1] : h2[0]) + __shfl_xor_sync(FULL, b1 ? h2[0] : h2[1], 2);
    return h + __shfl_xor_sync(FULL, h, 1);
}

// rows of M_k one lane accumulates: column l / 2, rows of parity l % 2
template <int CJ1>
struct MRows {
    static constexpr int n = (CJ1 + 1) / 2;
};

// This warp's entries of a tile of platform k (e, valid: the lane's entry), run by run.  Every
// lane of the warp calls this.  mreg: the lane's share of the CTA's M_k.
template <int CJ1, int CJ2, bool CNT = true>
__device__ __forceinline__ void warp_runs(const FastArgs &A, const Rec &e, bool valid, int k,
                                          const float *__restrict__ sGc, float (&mreg)[MRows<CJ1>::n]) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int J1 = CJ1, J2 = CJ2;
    constexpr int JA = (J1 + 3) & ~3, JB = (J2 + 3) & ~3;
    const int lane = threadIdx.x & 31;
    const int q = lane >> 1;      // this lane's component of the spread vectors
    const int par = lane & 1;     // parity of the M_k rows this lane accumulates
    // per warp: w2 (floats 0-15) and s (16-31) of the current run, shared by the lanes
    __shared__ __align__(16) float sWv[kFastThreads / 32][32];
    float *wv = sWv[threadIdx.x >> 5];
    float b[J2];
    float x = 0.f;
    int ej = 0;
    if (valid) {
        ej = e.j;
        x = e.x;
        const float *ub = A.U2 + (int64_t)e.j * J2;
        if constexpr (J2 % 2 == 0) {
#pragma unroll
            for (int qq = 0; qq < J2; qq += 2) {
                const float2 t2 = __ldg(reinterpret_cast<const float2 *>(ub + qq));
                b[qq] = t2.x;
                b[qq + 1] = t2.y;
            }
        } else {
#pragma unroll
            for (int qq = 0; qq < J2; ++qq) b[qq] = __ldg(ub + qq);
        }
    } else {
#pragma unroll
        for (int qq = 0; qq < J2; ++qq) b[qq] = 0.f;
    }
    const int iv = valid ? e.i : -1;
    unsigned rem = __ballot_sync(FULL, valid);
    while (rem) {  // warp-uniform: one run (one patient) per pass
        const int ih = __shfl_sync(FULL, iv, __ffs(rem) - 1);
        const unsigned run = __ballot_sync(FULL, iv == ih);
        rem &= ~run;
        const bool mine = (run >> lane) & 1u;
        // the run's patient row: one address for the whole warp
        float a[J1];
        const float *ua = A.U1 + (int64_t)ih * J1;
        if constexpr (J1 % 2 == 0) {
#pragma unroll
            for (int p = 0; p < J1; p += 2) {
                const float2 t2 = __ldg(reinterpret_cast<const float2 *>(ua + p));
                a[p] = t2.x;
                a[p + 1] = t2.y;
            }
        } else {
#pragma unroll
            for (int p = 0; p < J1; ++p) a[p] = __ldg(ua + p);
        }
        // w2 = Gc^T a: component q in lanes 2q, 2q + 1, then read by every lane from shared
        // memory (broadcast float4 loads)
        float wq = 0.f;
        if (q < J2) {
#pragma unroll
            for (int p = 0; p < J1; ++p) wq = fmaf(sGc[p * J2 + q], a[p], wq);
        }
        __syncwarp();  // every lane is done with the previous run's w2 and s
        if (!par && q < J2) wv[q] = wq;
        __syncwarp();
        float w2[JB];
#pragma unroll
        for (int t4 = 0; t4 < JB / 4; ++t4) {
            const float4 v = reinterpret_cast<const float4 *>(wv)[t4];
            w2[4 * t4] = v.x;
            w2[4 * t4 + 1] = v.y;
            w2[4 * t4 + 2] = v.z;
            w2[4 * t4 + 3] = v.w;
        }
        // the lane's entry, if it is in this run: residual and gene-row gradient
        float r = 0.f;
        if (mine) {
            float xt = 0.f;
#pragma unroll
            for (int qq = 0; qq < J2; ++qq) xt = fmaf(w2[qq], b[qq], xt);
            r = xt - x;
            float gvb[JB];
#pragma unroll
            for (int qq = 0; qq < JB; ++qq) gvb[qq] = qq < J2 ? r * w2[qq] : 0.f;
            float *gb = A.gB + (int64_t)ej * A.rs2;
#pragma unroll
            for (int t4 = 0; t4 < JB / 4; ++t4)
                atomicAdd(reinterpret_cast<float4 *>(gb) + t4,
                          make_float4(gvb[4 * t4], gvb[4 * t4 + 1], gvb[4 * t4 + 2], gvb[4 * t4 + 3]));
            if (CNT && A.count_atomics) atomicAdd(gb + JB + k, 1.f);
        }
        // s = sum over the run of r_e b_e (lanes outside the run give 0): lane l gets s[l / 2]
        float u[16];
#pragma unroll
        for (int qq = 0; qq < 16; ++qq) u[qq] = qq < J2 ? r * b[qq] : 0.f;
        const float s_q = reduce_scatter16(u);
        // M_k += a s^T: rows p = par, par + 2, ... of column q
        if (q < J2) {
#pragma unroll
            for (int t = 0; t < MRows<CJ1>::n; ++t) {
                const float ap = par ? (2 * t + 1 < J1 ? a[2 * t + 1 < J1 ? 2 * t + 1 : 0] : 0.f) : a[2 * t];
                mreg[t] = fmaf(ap, s_q, mreg[t]);
            }
        }
        // patient gradient Gc s: s goes to shared memory, and lane 2p forms
        // (Gc s)[p] = sum_q Gc[p][q] s[q] from row p of Gc
        if (!par && q < J2) wv[16 + q] = s_q;
        __syncwarp();
        if (!par && q < J1) {
            float sv[JB];
#pragma unroll
            for (int t4 = 0; t4 < JB / 4; ++t4) {
                const float4 v = reinterpret_cast<const float4 *>(wv + 16)[t4];
                sv[4 * t4] = v.x;
                sv[4 * t4 + 1] = v.y;
                sv[4 * t4 + 2] = v.z;
                sv[4 * t4 + 3] = v.w;
            }
            float gcs = 0.f;
#pragma unroll
            for (int qq = 0; qq < J2; ++qq) gcs = fmaf(sGc[q * J2 + qq], sv[qq], gcs);
            float *ga = A.gA + (int64_t)ih * A.rs1;
            atomicAdd(ga + q, gcs);
            if (CNT && lane == 0 && A.count_atomics) atomicAdd(ga + JA + k, (float)__popc(run));
        }
    }
}

// merges the warps' shares of M_k (staged through sMw, one J1 x J2 block per warp) into macc
template <int CJ1, int CJ2>
__device__ __forceinline__ void runs_merge(float (&mreg)[MRows<CJ1>::n], float *sMw, float *__restrict__ macc) {
    constexpr int J1 = CJ1, J2 = CJ2, Q = J1 * J2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane >> 1, par = lane & 1;
    if (q < J2) {
#pragma unroll
        for (int t = 0; t < MRows<CJ1>::n; ++t) {
            const int p = 2 * t + par;
            if (p < J1) sMw[warp * Q + p * J2 + q] = mreg[t];
            mreg[t] = 0.f;
        }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < Q; s += kFastThreads) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < kFastThreads / 32; ++w) sum += sMw[w * Q + s];
        atomicAdd(macc + s, sum);
    }
}

// a 32-entry unit u of the wave (unit p of tile u / 8): platform (-1: no entry in the unit)
// and this lane's record; u >= the wave's units gives an empty unit
__device__ __forceinline__ TileFetch fetch_unit(const FastArgs &A, int64_t u, int lane) {
    TileFetch f;
    f.k = -1;
    f.valid = false;
    f.e.i = f.e.j = f.e.k = 0;
    f.e.x = 0.f;
    const int64_t t = u / (kFastTile / 32);
    if (t < A.n_tiles) {
        const int off = (int)(u % (kFastTile / 32)) * 32;
        const int len = A.tile_len[t];
        if (off < len) {
            f.k = A.tile_k[t];
            f.valid = off + lane < len;
            if (f.valid) {
                const int4 v = __ldcs(reinterpret_cast<const int4 *>(A.rec + A.tile_start[t] + off + lane));
                f.e.i = v.x;
                f.e.j = v.y;
                f.e.k = v.z;
                f.e.x = __int_as_float(v.w);
            }
        }
    }
    return f;
}

// CTAs per SM the register budget is cut for (more entries in flight hide the gathers)
template <int CJ1, int CJ2>
constexpr int sweep_min_blocks() {
    return (CJ1 > 0 && CJ2 > 0 && CJ1 * CJ2 <= 100) ? 4 : (CJ1 == 16 && CJ2 == 16) ? 2 : 1;
}

// CNT: the sweep counts each row's entries per platform with atomics (no set-up table)
template <int CJ1, int CJ2, int CJ3, bool CNT>
__global__ void __launch_bounds__(kFastThreads, sweep_min_blocks<CJ1, CJ2>()) k_fast_sweep(FastArgs A) {
    const int J1 = CJ1 ? CJ1 : A.d.J1, J2 = CJ2 ? CJ2 : A.d.J2, J3 = CJ3 ? CJ3 : A.d.J3;
    const int J1P = even_up(J1), J2P = even_up(J2);
    const int PI = J1 * J2 * J3;
    extern __shared__ __align__(16) float sm[];
    // CTAs 0-2 (dispatched first, so they run beside the tile CTAs): the wave's dense
    // pre-work, split into its three independent parts
    if (blockIdx.x < kPreCtas) {
        dense_pre<CJ1, CJ2, CJ3>(A.pre, sm, (int)blockIdx.x);
        return;
    }
    float *sG = sm;                            // PI
    float *sGc = sG + align4(PI);              // J1*J2 (G x3 c_k)
    float *sRA = sGc + align4(J1 * J2);        // kFastThreads * J1P : r a  (8-byte aligned rows)
    float *sB = sRA + kFastThreads * J1P;      // kFastThreads * J2P : b
    float *sRed = sB + kFastThreads * J2P;     // kFastThreads * 4
    __shared__ int sTile[2];
    const int tid = threadIdx.x;
    for (int s = tid; s < PI; s += kFastThreads) sG[s] = A.G[s];
    if constexpr (runs_path<CJ1, CJ2>()) {
      if (A.d.I3 * J1 * J2 <= kGcAll) {
        // Static partition: the wave's tiles are cut into 32-entry units (8 per tile) and each
        // warp takes a contiguous range of them, so no CTA barrier and no tile claim sit in the
        // loop.  Gc_k for every platform is formed once per CTA; a warp's M_k shares go to a
        // per-CTA M (shared atomics) when its platform changes, and that to macc at the end.
        const int I3 = A.d.I3, Q = J1 * J2;
        float *sGcAll = sG + align4(PI);       // I3 x J1*J2
        float *sMacc = sGcAll + I3 * Q;        // I3 x J1*J2
        __syncthreads();  // sG
        for (int s = tid; s < I3 * Q; s += kFastThreads) {
            const int kk = s / Q, pq = s % Q;
            float g = 0.f;
            for (int r = 0; r < J3; ++r) g = fmaf(sG[pq * J3 + r], A.U3[(int64_t)kk * J3 + r], g);
            sGcAll[s] = g;
            sMacc[s] = 0.f;
        }
        __syncthreads();
        const int lane = tid & 31;
        const int64_t W = (int64_t)(gridDim.x - kPreCtas) * (kFastThreads / 32);
        const int64_t w = (int64_t)(blockIdx.x - kPreCtas) * (kFastThreads / 32) + (tid >> 5);
        const int64_t U = (int64_t)A.n_tiles * (kFastTile / 32);
        const int64_t u0 = w * U / W, u1 = (w + 1) * U / W;
        float mreg[MRows<CJ1>::n];
#pragma unroll
        for (int i = 0; i < MRows<CJ1>::n; ++i) mreg[i] = 0.f;
        int cur_k = -1;
        auto flush = [&]() {  // this warp's M_k shares into the CTA's M
            const int q = lane >> 1, par = lane & 1;
            if (q < J2) {
#pragma unroll
                for (int i = 0; i < MRows<CJ1>::n; ++i) {
                    const int pp = 2 * i + par;
                    if (pp < J1 && mreg[i] != 0.f) atomicAdd(sMacc + cur_k * Q + pp * J2 + q, mreg[i]);
                    mreg[i] = 0.f;
                }
            }
        };
        TileFetch f = fetch_unit(A, u0 < u1 ? u0 : U, lane);
        for (int64_t u = u0; u < u1; ++u) {
            const TileFetch cur = f;
            f = fetch_unit(A, u + 1 < u1 ? u + 1 : U, lane);  // one unit ahead
            if (cur.k < 0) continue;                          // an empty unit of a short tile
            if (cur.k != cur_k) {
                if (cur_k >= 0) flush();
                cur_k = cur.k;
            }
            warp_runs<CJ1, CJ2, CNT>(A, cur.e, cur.valid, cur.k, sGcAll + cur.k * Q, mreg);
        }
        if (cur_k >= 0) flush();
        __syncthreads();
        for (int s = tid; s < I3 * Q; s += kFastThreads)
            if (sMacc[s] != 0.f) atomicAdd(A.macc + s, sMacc[s]);
        return;
      }
    }
    if constexpr (runs_path<CJ1, CJ2>()) {  // per-patient-run factoring; M_k shares in registers
        float *sMw = sGc + align4(J1 * J2);    // (kFastThreads / 32) x J1*J2: the M_k merge
        float mreg[MRows<CJ1>::n];
#pragma unroll
        for (int t = 0; t < MRows<CJ1>::n; ++t) mreg[t] = 0.f;
        if (tid == 0) sTile[0] = atomicAdd(A.ctr, 1);
        __syncthreads();
        int t = sTile[0], par = 0;
        TileFetch f = fetch_tile(A, t);
        int cur_k = -1;
        for (;;) {
            const bool done = t >= A.n_tiles;
            if (tid == 0 && !done) sTile[par ^ 1] = atomicAdd(A.ctr, 1);
            if (f.k != cur_k || done) {
                if (cur_k >= 0) runs_merge<CJ1, CJ2>(mreg, sMw, A.macc + (int64_t)cur_k * J1 * J2);
                if (done) break;
                form_gc(sG, A.U3 + (int64_t)f.k * J3, sGc, J1, J2, J3);
                cur_k = f.k;
                __syncthreads();
            }
            warp_runs<CJ1, CJ2, CNT>(A, f.e, f.valid, f.k, sGc, mreg);
            __syncthreads();  // the next claim is visible; sGc and sMw free for reuse
            t = sTile[par ^ 1];
            par ^= 1;
            f = fetch_tile(A, t);
        }
    } else {
    const MLayout ml(J1P, J2P);
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;

    // software pipeline: the next tile is claimed, and its records fetched, before the M_k
    // accumulation of the current one
    if (tid == 0) sTile[0] = atomicAdd(A.ctr, 1);
    __syncthreads();
    int t = sTile[0], par = 0;
    TileFetch f = fetch_tile(A, t);
    int cur_k = -1;
    for (;;) {
        const bool done = t >= A.n_tiles;
        if (tid == 0 && !done) sTile[par ^ 1] = atomicAdd(A.ctr, 1);
        if (f.k != cur_k || done) {  // (a CTA that finds no tile at its first claim leaves too)
            if (cur_k >= 0) m_merge(ml, sRed, A.macc + (int64_t)cur_k * J1 * J2, J1, J2, acc0, acc1, acc2, acc3);
            if (done) break;
            form_gc(sG, A.U3 + (int64_t)f.k * J3, sGc, J1, J2, J3);
            cur_k = f.k;
            __syncthreads();
        }
        tile_entries<CJ1, CJ2, CJ3>(A, f.e, f.valid, f.k, sGc, sRA + tid * J1P, sB + tid * J2P);
        __syncthreads();  // tile staged; the next claim is visible
        t = sTile[par ^ 1];
        par ^= 1;
        f = fetch_tile(A, t);
        m_accumulate(ml, sRA, sB, J1P, J2P, acc0, acc1, acc2, acc3);
        __syncthreads();  // sRA, sB consumed
    }
    }
}

// ---------------------------------------------------------------------------------------
// Lane-group sweep (compile-time J1, J2 <= 16, every platform's Gc in shared memory, per-wave
// row counts from the set-up table).
//
// The same per-patient-run factoring as warp_runs (w2 = Gc^T a_i once per run, per entry
// x~ = w2 . b, r = x~ - x, g(b) += r w2, s += r b; per run g(a_i) += Gc s, M_k += a_i s^T), but
// one entry is handled by a group of L = J2 / VEC lanes, each holding VEC consecutive
// components of b, w2 and s: a warp takes E = 32 / L entries per step.  A gene row is then
// gathered as L contiguous vector loads (whole 32-byte sectors) instead of one lane walking it,
// its gradient leaves as L contiguous vector reductions, x~ is an L-lane shuffle sum, and s
// stays in each lane's registers until the run closes, when one reduction over the E entry
// slots completes it.  Each warp walks one contiguous range of the wave's entries (sorted by
// platform, then patient), so no tile claim and no CTA barrier sit in the loop; a run cut by a
// range boundary is closed by both warps, each adding its part (every sum is linear).
//
// GB = 1 gathers the gene rows from a BF16 copy of U2 (VEC = 4 BF16 = 8 bytes per lane); all
// arithmetic, the gradients and the factors stay FP32.

// 4 components per lane where J2 allows (FP32: one 16-byte load; BF16: one 8-byte load),
// else 2 or 1.  (8 BF16 components per lane, 2 lanes per entry at J2 = 16, was measured slower:
// 16-entry steps cross patient runs twice as often and a run's close costs twice the shuffles.)
// In the batched sweep, entry records reach a lane-group warp by bulk copies (the TMA
// engine's cp.async.bulk) into shared memory, kRecSteps steps of records at a time, two
// chunks per warp in flight.
constexpr int kRecSteps = 16;

// lane 0 of a warp: copies `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on the mbarrier, which expects the bytes
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
                 : "memory");
}

template <int CJ2, int GB>
struct LaneGroup {
    static constexpr int VEC = (GB || CJ2 % 4 == 0) ? 4 : (CJ2 % 2 == 0 ? 2 : 1);
    static constexpr int L = CJ2 / VEC;  // lanes per entry
    static constexpr int E = 32 / L;     // entries per step
};

// sum of x over the L lanes of this lane's group (lanes g L .. g L + L - 1); every lane of the
// group gets the same value.  All 32 lanes call this.
template <int L>
__device__ __forceinline__ float group_sum(float x) {
    constexpr unsigned FULL = 0xffffffffu;
    if constexpr ((L & (L - 1)) == 0) {
#pragma unroll
        for (int o = 1; o < L; o <<= 1) x += __shfl_xor_sync(FULL, x, o);
        return x;
    } else {
        const int m = (threadIdx.x & 31) % L;
#pragma unroll
        for (int o = 1; o < L; o <<= 1) {
            const float y = __shfl_down_sync(FULL, x, o);
            if (m + o < L) x += y;
        }
        return __shfl_sync(FULL, x, ((threadIdx.x & 31) / L) * L);
    }
}

// sum of x over the E entry slots (lanes m, m + L, m + 2L, ...) of this lane's component
// group m; every lane of the component group gets the same value.  All 32 lanes call this.
template <int L, int E>
__device__ __forceinline__ float slot_sum(float x) {
    constexpr unsigned FULL = 0xffffffffu;
    if constexpr (L * E == 32 && (L & (L - 1)) == 0) {
#pragma unroll
        for (int o = L; o < 32; o <<= 1) x += __shfl_xor_sync(FULL, x, o);
        return x;
    } else {
        const int m = (threadIdx.x & 31) % L;
        float t = 0.f;
#pragma unroll
        for (int g = 0; g < E; ++g) t += __shfl_sync(FULL, x, g * L + m);
        return t;
    }
}

// CTAs per SM the lane-group kernels' registers are cut for.  The single-problem kernel fits
// 64 registers at every compiled shape, the dense pre-work's 16 x 16 eigen-solves included
// (measured at 16 x 16 x 5: 26.9 G entries/s at 4 CTAs per SM against 25.4 G at 3).  The batch
// kernel keeps its problem's arguments in shared memory and spills at 64 registers for
// 16 x 16, which halved its speed, so it is cut for 3 CTAs per SM there.
template <int CJ1, int CJ2, int GB = 0>
constexpr int lg_min_blocks() { return 4; }
template <int CJ1, int CJ2, int GB = 0>
constexpr int lg_batch_min_blocks() { return CJ1 * CJ2 <= 100 ? 4 : 3; }

// The lane-group sweep of one problem's wave by the CTA's warps: W warps share the wave,
// this CTA's warps are w0, w0 + 1, ...  (sm: the CTA's dynamic shared memory)
template <int CJ1, int CJ2, int CJ3, int GB, bool TMA>
__device__ __forceinline__ void lg_sweep_body(const FastArgs &A, float *sm, int64_t W, int64_t w0) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int J1 = CJ1, J2 = CJ2, J3 = CJ3, Q = J1 * J2, PI = Q * J3;
    using LG = LaneGroup<CJ2, GB>;
    constexpr int VEC = LG::VEC, L = LG::L, E = LG::E;
    constexpr int NM = (Q + 31) / 32;  // M_k elements per lane
    // per warp: the open run's patient row a (floats 0-31) and, when it closes, s (32-63)
    __shared__ __align__(16) float sSlot[kFastThreads / 32][64];
    const int I3 = A.d.I3;
    float *sG = sm;                       // PI
    float *sGcAll = sG + align4(PI);      // I3 x Q: Gc_k = G x3 c_k
    float *sMacc = sGcAll + I3 * Q;       // I3 x Q: this CTA's M_k
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int s = tid; s < PI; s += kFastThreads) sG[s] = A.G[s];
    __syncthreads();
    for (int s = tid; s < I3 * Q; s += kFastThreads) {
        const int kk = s / Q, pq = s % Q;
        float g = 0.f;
#pragma unroll
        for (int r = 0; r < J3; ++r) g = fmaf(sG[pq * J3 + r], A.U3[(int64_t)kk * J3 + r], g);
        sGcAll[s] = g;
        sMacc[s] = 0.f;
    }
    __syncthreads();
    float *slot = sSlot[warp];
    const int g = lane / L, m = lane % L;  // entry slot and component group of this lane
    const bool act = g < E;
    const int64_t w = w0 + warp;
    const int64_t lo = A.e_first + w * A.e_count / W, hi = A.e_first + (w + 1) * A.e_count / W;
    float mreg[NM];
#pragma unroll
    for (int t = 0; t < NM; ++t) mreg[t] = 0.f;
    int mk = -1, ci = -1, ck = -1;  // platform of mreg; the open run (patient, platform)
    float w2v[VEC], sv[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) w2v[v] = sv[v] = 0.f;
    auto flush_m = [&]() {  // this warp's M_k shares into the CTA's M
        if (mk < 0) return;
#pragma unroll
        for (int t = 0; t < NM; ++t) {
            const int idx = lane + 32 * t;
            if (idx < Q && mreg[t] != 0.f) atomicAdd(sMacc + mk * Q + idx, mreg[t]);
            mreg[t] = 0.f;
        }
    };
    auto close_run = [&]() {
        float st[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) st[v] = slot_sum<L, E>(sv[v]);
        if (lane < L)
#pragma unroll
            for (int v = 0; v < VEC; ++v) slot[32 + m * VEC + v] = st[v];
        __syncwarp();
        if (lane < J1) {  // patient gradient (Gc s)[p], p = lane
            const float *gc = sGcAll + ck * Q + lane * J2;
            float acc = 0.f;
            if constexpr (GB && (J2 & (J2 - 1)) == 0) {
                // lane p starts its walk at q = p: with rows J2 apart (a power of two) the lanes
                // would otherwise meet in two banks, an 8-way conflict at J2 = 16.  Measured at
                // 16 x 16 x 5 on the paper-scale tensor: BF16 gathers 24.0 -> 25.2 G entries/s;
                // the FP32 sweep went 25.95 -> 25.56 G with it and keeps the plain walk.
#pragma unroll
                for (int q = 0; q < J2; ++q) {
                    const int qq = (q + lane) & (J2 - 1);
                    acc = fmaf(gc[qq], slot[32 + qq], acc);
                }
            } else {
#pragma unroll
                for (int q = 0; q < J2; ++q) acc = fmaf(gc[q], slot[32 + q], acc);
            }
            atomicAdd(A.gA + (int64_t)ci * A.rs1 + lane, acc);
        }
#pragma unroll
        for (int t = 0; t < NM; ++t) {  // M_k += a s^T
            const int idx = lane + 32 * t;
            if (idx < Q) mreg[t] = fmaf(slot[idx / J2], slot[32 + idx % J2], mreg[t]);
        }
        __syncwarp();
#pragma unroll
        for (int v = 0; v < VEC; ++v) sv[v] = 0.f;
    };
    auto open_run = [&](int i, int k) {
        if (k != mk) {
            flush_m();
            mk = k;
        }
        ci = i;
        ck = k;
        if (lane < J1) slot[lane] = __ldg(A.U1 + (int64_t)i * J1 + lane);
        __syncwarp();
        const float *gc = sGcAll + k * Q;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {  // w2 = Gc^T a, components m VEC + v
            float acc = 0.f;
#pragma unroll
            for (int p = 0; p < J1; ++p) acc = fmaf(gc[p * J2 + m * VEC + v], slot[p], acc);
            w2v[v] = acc;
        }
    };
    // entry positions and row offsets fit in 32 bits here (the kernel is chosen only then)
    const int lo32 = (int)lo, hi32 = (int)hi;
    // TMA: the warp's records arrive in chunks of kRecSteps steps (CH records) by bulk copies
    // into two shared buffers: chunk c goes to buffer c & 1 and completes its barrier's phase
    // (c >> 1) & 1.  Entering chunk c the warp starts chunk c + 1's copy (into chunk c - 1's
    // buffer, which every lane has read) and waits for chunk c.  A wait that gives up sets the
    // error word and ends the warp's range before the records it never got.  Otherwise each
    // lane loads its records from global memory, evict-first (they are streamed once per
    // epoch).  Measured on the paper-scale problem, the copies made the single-problem sweep
    // slower (45.98 -> 50.97 us per wave at 10 x 10 x 5, 1.040 -> 1.104 ms per epoch at
    // 16 x 16 x 5) and the batched sweep faster (19.15 -> 18.41 ms per epoch of the 96
    // decompositions), so only the batch kernel takes them.
    constexpr int CH = kRecSteps * E;
    Rec *rbuf = nullptr;
    uint64_t *rbar = nullptr;
    if constexpr (TMA) {
        __shared__ __align__(128) Rec sRec[kFastThreads / 32][2][CH];
        __shared__ __align__(8) uint64_t sRecBar[kFastThreads / 32][2];
        rbuf = &sRec[warp][0][0];
        rbar = sRecBar[warp];
    }
    int issued = -1, waited = -1;  // the same in every lane
    int hi_eff = hi32;
    auto issue = [&](int c) {
        const int s0 = lo32 + c * CH;
        if (s0 >= hi_eff) return;
        issued = c;
        if (lane == 0)
            bulk_load(rbuf + (c & 1) * CH, A.rec + s0, (uint32_t)(min(CH, hi32 - s0) * (int)sizeof(Rec)),
                      rbar + (c & 1));
    };
    auto await = [&](int c) {
        const bool ok = __all_sync(FULL, tc::mbar_wait(rbar + (c & 1), (uint32_t)((c >> 1) & 1)));
        waited = c;
        if (!ok) {
            if (lane == 0) atomicOr(A.err, 1);
            hi_eff = min(hi_eff, lo32 + c * CH);
        }
    };
    // the record of slot g at step t (entry e = lo + t E + g)
    auto load_rec = [&](int t, int e, bool ok) {
        Rec r;
        r.i = r.j = r.k = -1;
        r.x = 0.f;
        if (ok) {
            int4 v;
            if constexpr (TMA)
                v = *reinterpret_cast<const int4 *>(rbuf + ((t / kRecSteps) & 1) * CH + (t % kRecSteps) * E + g);
            else
                v = __ldcs(reinterpret_cast<const int4 *>(A.rec + e));
            r.i = v.x;
            r.j = v.y;
            r.k = v.z;
            r.x = __int_as_float(v.w);
        }
        return r;
    };
    if constexpr (TMA) {
        if (lane == 0) {
            tc::mbar_init(rbar);
            tc::mbar_init(rbar + 1);
        }
        __syncwarp();
        issue(0);
        issue(1);
        if (issued >= 0) await(0);
    }
    // this lane's VEC components of the gene row of record r (zeros when !ok), as loaded: VEC
    // floats, or for BF16 gathers 4 BF16 values in one 8-byte word (unpacked when used, so the
    // prefetched row takes 2 registers)
    struct FRow {
        float v[VEC];
    };
    using Raw = std::conditional_t<GB != 0, uint2, FRow>;
    auto load_row = [&](const Rec &r, bool ok) {
        Raw x;
        if constexpr (GB) {
            x = ok ? __ldg(reinterpret_cast<const uint2 *>(A.U2h + r.j * J2 + m * VEC)) : make_uint2(0u, 0u);
        } else {
            const int bo = r.j * J2 + m * VEC;
            if (!ok) {
#pragma unroll
                for (int v = 0; v < VEC; ++v) x.v[v] = 0.f;
            } else if constexpr (VEC == 4) {
                const float4 t4 = __ldg(reinterpret_cast<const float4 *>(A.U2 + bo));
                x.v[0] = t4.x;
                x.v[1] = t4.y;
                x.v[2] = t4.z;
                x.v[3] = t4.w;
            } else if constexpr (VEC == 2) {
                const float2 t2 = __ldg(reinterpret_cast<const float2 *>(A.U2 + bo));
                x.v[0] = t2.x;
                x.v[1] = t2.y;
            } else {
                x.v[0] = __ldg(A.U2 + bo);
            }
        }
        return x;
    };
    auto unpack = [&](const Raw &x, float (&b)[VEC]) {
        if constexpr (GB) {  // BF16 values are the upper halves of FP32 words
            const uint32_t w[2] = {x.x, x.y};
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                b[2 * t] = __uint_as_float(w[t] << 16);
                b[2 * t + 1] = __uint_as_float(w[t] & 0xffff0000u);
            }
        } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) b[v] = x.v[v];
        }
    };
    // software pipeline: records two steps ahead, gene rows one step ahead.  With groups of 5
    // lanes (J2 = 5, 10) the loop is unrolled by three, so the records rotate through registers
    // without moves (measured at 10 x 10 x 5: 46.95 -> 45.22 us per paper-scale wave, with the
    // shuffle-tree group sum); at J2 = 16 the unrolled loop spilled, and it is left rolled.
    constexpr int UNROLL = (!GB && CJ2 % 4 != 0) ? 3 : 1;
    static_assert(kRecSteps >= 2, "the first two steps' records come from chunk 0");
    Rec cur = load_rec(0, lo32 + g, act && lo32 + g < (TMA ? hi_eff : hi32));
    Rec nxt = load_rec(1, lo32 + g + E, act && lo32 + g + E < (TMA ? hi_eff : hi32));
    Raw bnext = load_row(cur, act && lo32 + g < (TMA ? hi_eff : hi32));
    auto step = [&](int base) {
        const int e = base + g;
        const bool valid = act && e < (TMA ? hi_eff : hi32);
        float b[VEC];
        unpack(bnext, b);
        int tn = 0;  // the step whose records are fetched now
        if constexpr (TMA) {
            tn = (base - lo32) / E + 2;
            if (tn % kRecSteps == 0 && lo32 + tn * E < (TMA ? hi_eff : hi32)) {  // entering a chunk (the same in every lane)
                __syncwarp();  // every lane is done with the previous chunk's buffer
                issue(tn / kRecSteps + 1);
                await(tn / kRecSteps);
            }
        }
        const Rec nn = load_rec(tn, e + 2 * E, act && e + 2 * E < (TMA ? hi_eff : hi32));
        bnext = load_row(nxt, act && e + E < (TMA ? hi_eff : hi32));
        // an entry's residual, its gene-row gradient and its share of s (b = 0 off the wave)
        auto entry = [&](bool mine) {
            float part = 0.f;
#pragma unroll
            for (int v = 0; v < VEC; ++v) part = fmaf(w2v[v], b[v], part);
            const float xt = group_sum<L>(mine ? part : 0.f);
            if (mine) {
                const float r = xt - cur.x;
                float *gb = A.gB + cur.j * A.rs2 + m * VEC;
                if constexpr (VEC == 4)
                    atomicAdd(reinterpret_cast<float4 *>(gb), make_float4(r * w2v[0], r * w2v[1], r * w2v[2], r * w2v[3]));
                else if constexpr (VEC == 2)
                    atomicAdd(reinterpret_cast<float2 *>(gb), make_float2(r * w2v[0], r * w2v[1]));
                else
                    atomicAdd(gb, r * w2v[0]);
#pragma unroll
                for (int v = 0; v < VEC; ++v) sv[v] = fmaf(r, b[v], sv[v]);
            }
        };
        if (__all_sync(FULL, !valid || (cur.i == ci && cur.k == ck))) {
            entry(valid);  // the common case: every entry of the step lies in the open run
        } else {           // otherwise the step's entries run by run
            unsigned pend = __ballot_sync(FULL, valid && m == 0);
            while (pend) {
                const int lead = __ffs(pend) - 1;
                const int ri = __shfl_sync(FULL, cur.i, lead), rk = __shfl_sync(FULL, cur.k, lead);
                if (ri != ci || rk != ck) {
                    if (ci >= 0) close_run();
                    open_run(ri, rk);
                }
                const bool mine = valid && cur.i == ci && cur.k == ck;
                pend &= ~__ballot_sync(FULL, mine && m == 0);
                entry(mine);
            }
        }
        cur = nxt;
        nxt = nn;
    };
    if constexpr (UNROLL > 1) {
#pragma unroll(UNROLL)
        for (int base = lo32; base < (TMA ? hi_eff : hi32); base += E) step(base);
    } else {
        for (int base = lo32; base < (TMA ? hi_eff : hi32); base += E) step(base);
    }
    if constexpr (TMA)
        for (int c = waited + 1; c <= issued; ++c) await(c);  // no copy left in flight at exit
    if (ci >= 0) close_run();
    flush_m();
    __syncthreads();
    for (int s = tid; s < I3 * Q; s += kFastThreads)
        if (sMacc[s] != 0.f) atomicAdd(A.macc + s, sMacc[s]);
}

template <int CJ1, int CJ2, int CJ3, int GB>
__global__ void __launch_bounds__(kFastThreads, lg_min_blocks<CJ1, CJ2, GB>()) k_fast_sweep_lg(FastArgs A) {
    extern __shared__ __align__(16) float sm[];
    if (blockIdx.x < kPreCtas) {  // the wave's dense pre-work, as in k_fast_sweep
        dense_pre<CJ1, CJ2, CJ3>(A.pre, sm, (int)blockIdx.x);
        return;
    }
    lg_sweep_body<CJ1, CJ2, CJ3, GB, false>(A, sm, (int64_t)(gridDim.x - kPreCtas) * (kFastThreads / 32),
                                     (int64_t)(blockIdx.x - kPreCtas) * (kFastThreads / 32));
}

// The lane-group sweep of one wave over every problem of a batch.  CTAs 0 .. P-1 take each
// problem's dense pre-work; every other CTA serves one problem (cta_prob), as CTA number
// cta_rank of the prob_ctas[p] CTAs the batch's autotuned allotment gave that problem.
template <int CJ1, int CJ2, int CJ3, int GB>
__global__ void __launch_bounds__(kFastThreads, lg_batch_min_blocks<CJ1, CJ2, GB>())
    k_batch_sweep_lg(const FastArgs *__restrict__ probs, const int32_t *__restrict__ cta_prob,
                     const int32_t *__restrict__ cta_rank, const int32_t *__restrict__ prob_ctas, int32_t P) {
    extern __shared__ __align__(16) float sm[];
    __shared__ FastArgs sArgs;
    if ((int)blockIdx.x < P) {
        dense_pre<CJ1, CJ2, CJ3>(probs[blockIdx.x].pre, sm, -1);
        return;
    }
    const int b = (int)blockIdx.x - P;
    const int pid = cta_prob[b];
    if (threadIdx.x == 0) sArgs = probs[pid];
    __syncthreads();
    lg_sweep_body<CJ1, CJ2, CJ3, GB, true>(sArgs, sm, (int64_t)prob_ctas[pid] * (kFastThreads / 32),
                                     (int64_t)cta_rank[b] * (kFastThreads / 32));
}

// The sweep of one wave over every problem of a batch: the same tile work as k_fast_sweep;
// the CTAs claim tiles from the concatenated tile lists of all problems (toff: prefix
// offsets) and switch problem (arguments and core in shared memory) between tiles.
template <int CJ1, int CJ2, int CJ3>
__global__ void __launch_bounds__(kFastThreads, sweep_min_blocks<CJ1, CJ2>())
    k_batch_sweep(const FastArgs *__restrict__ probs, const int32_t *__restrict__ toff, int32_t P, int32_t *ctr) {
    __shared__ FastArgs sArgs;  // the problem of the current tile
    __shared__ int sPid[2], sTile[2];
    const FastArgs &A = sArgs;
    const Dims d0 = probs[0].d;  // every problem of a batch has the same ranks
    const int J1 = CJ1 ? CJ1 : d0.J1, J2 = CJ2 ? CJ2 : d0.J2, J3 = CJ3 ? CJ3 : d0.J3;
    const int J1P = even_up(J1), J2P = even_up(J2);
    const int PI = J1 * J2 * J3;
    extern __shared__ __align__(16) float sm[];
    if ((int)blockIdx.x < P) {  // the first P CTAs: each problem's dense pre-work
        dense_pre(probs[blockIdx.x].pre, sm);
        return;
    }
    float *sG = sm;                            // PI
    float *sGc = sG + align4(PI);              // J1*J2 (G x3 c_k)
    float *sRA = sGc + align4(J1 * J2);        // kFastThreads * J1P : r a  (8-byte aligned rows)
    float *sB = sRA + kFastThreads * J1P;      // kFastThreads * J2P : b
    float *sRed = sB + kFastThreads * J2P;     // kFastThreads * 4
    const int tid = threadIdx.x;
    const MLayout ml(J1P, J2P);
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
    // a tile of the batch: problem by binary search over the tile offsets (pid -1: none left)
    auto claim = [&](int slot) {
        const int g = atomicAdd(ctr, 1);
        int pid = -1;
        if (g < toff[P]) {
            int lo = 0, hi = P - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (toff[mid] <= g) lo = mid; else hi = mid - 1;
            }
            pid = lo;
        }
        sPid[slot] = pid;
        sTile[slot] = pid >= 0 ? g - toff[pid] : 0;
    };
    auto fetch = [&](int pid, int t) {
        if (pid >= 0) return fetch_tile(probs[pid], t);
        TileFetch f;
        f.k = -1;
        f.valid = false;
        f.e.i = f.e.j = f.e.k = 0;
        f.e.x = 0.f;
        return f;
    };

    // software pipeline as in k_fast_sweep: claim and fetch one tile ahead
    if (tid == 0) claim(0);
    __syncthreads();
    int pid = sPid[0], t = sTile[0], par = 0;
    TileFetch f = fetch(pid, t);
    int cur_k = -1, cur_pid = -1;
    if constexpr (runs_path<CJ1, CJ2>()) {  // per-patient-run factoring, as in k_fast_sweep
        float *sMw = sGc + align4(J1 * J2);
        float mreg[MRows<CJ1>::n];
#pragma unroll
        for (int i = 0; i < MRows<CJ1>::n; ++i) mreg[i] = 0.f;
        for (;;) {
            const bool done = pid < 0;
            if (tid == 0 && !done) claim(par ^ 1);
            if (f.k != cur_k || pid != cur_pid || done) {
                if (cur_k >= 0) runs_merge<CJ1, CJ2>(mreg, sMw, A.macc + (int64_t)cur_k * J1 * J2);
                if (done) break;
                if (pid != cur_pid) {
                    __syncthreads();
                    if (tid == 0) sArgs = probs[pid];
                    __syncthreads();
                    for (int s = tid; s < PI; s += kFastThreads) sG[s] = A.G[s];
                    __syncthreads();
                    cur_pid = pid;
                }
                form_gc(sG, A.U3 + (int64_t)f.k * J3, sGc, J1, J2, J3);
                cur_k = f.k;
                __syncthreads();
            }
            warp_runs<CJ1, CJ2>(A, f.e, f.valid, f.k, sGc, mreg);
            __syncthreads();
            pid = sPid[par ^ 1];
            t = sTile[par ^ 1];
            par ^= 1;
            f = fetch(pid, t);
        }
    } else {
    for (;;) {
        const bool done = pid < 0;
        if (tid == 0 && !done) claim(par ^ 1);
        if (f.k != cur_k || pid != cur_pid || done) {
            // merge into the previous tile's problem (sArgs still holds it)
            if (cur_k >= 0) m_merge(ml, sRed, A.macc + (int64_t)cur_k * J1 * J2, J1, J2, acc0, acc1, acc2, acc3);
            if (done) break;
            if (pid != cur_pid) {  // the next problem's arguments and core
                __syncthreads();
                if (tid == 0) sArgs = probs[pid];
                __syncthreads();
                for (int s = tid; s < PI; s += kFastThreads) sG[s] = A.G[s];
                __syncthreads();
                cur_pid = pid;
            }
            form_gc(sG, A.U3 + (int64_t)f.k * J3, sGc, J1, J2, J3);
            cur_k = f.k;
            __syncthreads();
        }
        tile_entries<CJ1, CJ2, CJ3>(A, f.e, f.valid, f.k, sGc, sRA + tid * J1P, sB + tid * J2P);
        __syncthreads();  // tile staged; the next claim is visible
        pid = sPid[par ^ 1];
        t = sTile[par ^ 1];
        par ^= 1;
        f = fetch(pid, t);
        m_accumulate(ml, sRA, sB, J1P, J2P, acc0, acc1, acc2, acc3);
        __syncthreads();  // sRA, sB consumed
    }
    }
}

// ---------------------------------------------------------------------------------------
// BF16 precision form of the sweep on the tensor cores (tcgen05, accumulators in TMEM).
//
// Same wave semantics and FP32 accumulators as k_fast_sweep; the three products of a tile
// of 128 entries run as BF16 x BF16 -> FP32 matrix products:
//   V  = B_tile Gc^T    (128 x J1, K = J2)      v_e  = Gc b_e
//   W2 = A_tile Gc      (128 x J2, K = J1)      w2_e = Gc^T a_e
//   M_k += (r A)^T B    (J1 x J2, K = 128)      accumulated in TMEM across the platform's tiles
// The gathered rows a, b and Gc = G x3 c_k are rounded to BF16 for the products; x~ = a . v,
// the residual, the row gradients and every update stay FP32 (FP32 master factors).  One
// thread issues the MMAs; tcgen05.commit arrives on an mbarrier that all threads wait on.
// TMEM columns of one CTA: V (J1), W2 (J2) and M_k (J2), rounded up to a power of two
template <int CJ1, int CJ2>
__host__ __device__ constexpr int tc_tmem_cols() { return CJ1 + 2 * CJ2 <= 64 ? 64 : 128; }

// Shared memory of the tensor-core sweep.  (rA)^T is the A operand of the M_k product, an
// M = 128-row operand of which only rows p < J1 are meaningful (D row p depends only on A row
// p, and rows >= J1 of D are never read): only its J1 rows are stored, at the start of the
// buffer, and the descriptor's remaining rows fall on the other buffers that follow; the
// allocation is padded so that the whole 128-row span stays inside it.
__host__ __device__ constexpr size_t tc_smem_bytes(int J1, int J2, int PI) {
    const size_t used = 2 * ((size_t)J1 * 128 + 128 * J1 + 128 * J2 + J2 * 128 + 2 * J1 * J2) + 4 * (size_t)PI;
    const size_t span = 2 * 128 * 128;  // the (rA)^T operand's 128-row span
    return used > span ? used : span;
}

template <int CJ1, int CJ2>
__global__ void __launch_bounds__(128) k_fast_sweep_tc(FastArgs A) {
    constexpr int J1 = CJ1, J2 = CJ2, M = 128;
    constexpr int JA = (J1 + 3) & ~3, JB = (J2 + 3) & ~3;
    constexpr int NC = tc_tmem_cols<CJ1, CJ2>();
    const int J3 = A.d.J3, PI = J1 * J2 * J3;
    extern __shared__ __align__(1024) uint8_t smb[];
    if (blockIdx.x == 0) {  // CTA 0: the wave's dense pre-work (no TMEM)
        dense_pre(A.pre, reinterpret_cast<float *>(smb));
        return;
    }
    __nv_bfloat16 *sRAT = reinterpret_cast<__nv_bfloat16 *>(smb);           // J1 x M (rows of (rA)^T)
    __nv_bfloat16 *sA = sRAT + J1 * M;                                        // M x J1
    __nv_bfloat16 *sB = sA + M * J1;                                          // M x J2
    __nv_bfloat16 *sBT = sB + M * J2;                                         // J2 x M
    __nv_bfloat16 *bGc = sBT + J2 * M;                                        // J1 x J2
    __nv_bfloat16 *bGcT = bGc + J1 * J2;                                      // J2 x J1
    float *sG = reinterpret_cast<float *>(bGcT + J2 * J1);                    // PI
    __shared__ __align__(8) uint64_t mbar_vw, mbar_m;
    __shared__ uint32_t tmem_base;
    __shared__ int sTile[2];
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::smem_u32(&tmem_base)),
                     "r"(NC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        tc::mbar_init(&mbar_vw);
        tc::mbar_init(&mbar_m);
        sTile[0] = atomicAdd(A.ctr, 1);
    }
    for (int t = tid; t < PI; t += M) sG[t] = A.G[t];
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t t_v = tmem, t_w = tmem + J1, t_m = tmem + J1 + J2;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    uint32_t ph_vw = 0, ph_m = 0;
    bool m_started = false, m_pending = false, failed = false;
    // the M_k product of the previous half still reads sRAT and sBT: wait for it before they
    // are rewritten (false: the wait gave up)
    auto settle_m = [&]() {
        bool ok = true;
        if (m_pending) {
            ok = tc::mbar_wait(&mbar_m, ph_m);
            ph_m ^= 1u;
            m_pending = false;
        }
        return ok;
    };
    // software pipeline: the records of the next tile (both halves) are fetched one tile ahead
    int t = sTile[0], par = 0;
    int nk = -1, n_e = 0;
    Rec rec_next[2];
    auto fetch = [&](int tt) {
        nk = -1;
        n_e = 0;
        if (tt < A.n_tiles) {
            nk = A.tile_k[tt];
            n_e = A.tile_len[tt];
            const int64_t s0 = A.tile_start[tt];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int el = h * M + tid;
                if (el < n_e) {
                    const int4 v4 = __ldcs(reinterpret_cast<const int4 *>(A.rec + s0 + el));
                    rec_next[h].i = v4.x;
                    rec_next[h].j = v4.y;
                    rec_next[h].k = v4.z;
                    rec_next[h].x = __int_as_float(v4.w);
                }
            }
        }
    };
    fetch(t);
    int cur_k = -1;
    for (;;) {
        const bool done = t >= A.n_tiles;
        const int k = nk, tile_n = n_e;
        Rec rec[2] = {rec_next[0], rec_next[1]};
        if (tid == 0 && !done) sTile[par ^ 1] = atomicAdd(A.ctr, 1);
        if (k != cur_k || done) {  // (a CTA that finds no tile at its first claim leaves too)
            if (cur_k >= 0 && m_started) {  // merge this CTA's M_k (rows p < J1 in lanes 0..J1-1)
                if (__syncthreads_or(!settle_m())) failed = true;
                tc::fence_after();
                if (!failed && warp < (J1 + 31) / 32) {
                    float mv[J2];
#pragma unroll
                    for (int c0 = 0; c0 < J2; c0 += 16) tc::ld16(t_m + lane_off + c0, mv + c0);
                    const int p = warp * 32 + (tid & 31);
                    if (p < J1)
#pragma unroll
                        for (int q = 0; q < J2; ++q) atomicAdd(A.macc + ((int64_t)cur_k * J1 + p) * J2 + q, mv[q]);
                }
                m_started = false;
            }
            if (done || failed) break;
            const float *ck = A.U3 + (int64_t)k * J3;
            for (int s = tid; s < J1 * J2; s += M) {
                const int p = s / J2, q = s % J2;
                float g = 0.f;
                for (int r = 0; r < J3; ++r) g = fmaf(sG[s * J3 + r], ck[r], g);
                const __nv_bfloat16 gb = __float2bfloat16(g);
                *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<uint8_t *>(bGc) + tc::kmajor_off(p, q, J2)) = gb;
                *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<uint8_t *>(bGcT) + tc::kmajor_off(q, p, J1)) = gb;
            }
            cur_k = k;
        }
        for (int h = 0; h < 2 && h * M < tile_n; ++h) {
            const int el = h * M + tid;
            const bool valid = el < tile_n;
            float a[J1], b[J2];
            float x = 0.f;
            int ei = 0, ej = 0;
            if (valid) {
                const Rec &e = rec[h];
                ei = e.i;
                ej = e.j;
                x = e.x;
                const float4 *ua = reinterpret_cast<const float4 *>(A.U1 + (int64_t)e.i * J1);
                const float4 *ub = reinterpret_cast<const float4 *>(A.U2 + (int64_t)e.j * J2);
#pragma unroll
                for (int p = 0; p < J1 / 4; ++p) {
                    const float4 t4 = __ldg(ua + p);
                    a[4 * p] = t4.x, a[4 * p + 1] = t4.y, a[4 * p + 2] = t4.z, a[4 * p + 3] = t4.w;
                }
#pragma unroll
                for (int q = 0; q < J2 / 4; ++q) {
                    const float4 t4 = __ldg(ub + q);
                    b[4 * q] = t4.x, b[4 * q + 1] = t4.y, b[4 * q + 2] = t4.z, b[4 * q + 3] = t4.w;
                }
            } else {
#pragma unroll
                for (int p = 0; p < J1; ++p) a[p] = 0.f;
#pragma unroll
                for (int q = 0; q < J2; ++q) b[q] = 0.f;
            }
            // the gathers above overlap the previous half's M_k product; sBT is its operand
            const bool ok0 = settle_m();
            uint8_t *pa = reinterpret_cast<uint8_t *>(sA), *pb = reinterpret_cast<uint8_t *>(sB);
            uint8_t *pbt = reinterpret_cast<uint8_t *>(sBT), *prt = reinterpret_cast<uint8_t *>(sRAT);
#pragma unroll
            for (int p = 0; p < J1; p += 2)
                *reinterpret_cast<__nv_bfloat162 *>(pa + tc::kmajor_off(tid, p, J1)) = __floats2bfloat162_rn(a[p], a[p + 1]);
#pragma unroll
            for (int q = 0; q < J2; q += 2)
                *reinterpret_cast<__nv_bfloat162 *>(pb + tc::kmajor_off(tid, q, J2)) = __floats2bfloat162_rn(b[q], b[q + 1]);
#pragma unroll
            for (int q = 0; q < J2; ++q)
                *reinterpret_cast<__nv_bfloat16 *>(pbt + tc::kmajor_off(q, tid, M)) = __float2bfloat16(b[q]);
            tc::fence_smem_to_async();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            if (tid == 0) {
                tc::mma_kmajor(t_v, tc::smem_u32(sB), tc::smem_u32(bGc), J2, J1, false);
                tc::mma_kmajor(t_w, tc::smem_u32(sA), tc::smem_u32(bGcT), J1, J2, false);
                tc::commit(&mbar_vw);
            }
            const bool ok1 = tc::mbar_wait(&mbar_vw, ph_vw);
            ph_vw ^= 1u;
            tc::fence_after();
            float v[J1], w2[J2];
#pragma unroll
            for (int c0 = 0; c0 < J1; c0 += 16) tc::ld16(t_v + lane_off + c0, v + c0);
#pragma unroll
            for (int c0 = 0; c0 < J2; c0 += 16) tc::ld16(t_w + lane_off + c0, w2 + c0);
            float r = 0.f;
            float gva[JA];
#pragma unroll
            for (int p = 0; p < JA; ++p) gva[p] = 0.f;
            if (valid) {
                float xt = 0.f;
#pragma unroll
                for (int p = 0; p < J1; ++p) xt = fmaf(a[p], v[p], xt);
                r = xt - x;
                float *gb = A.gB + (int64_t)ej * A.rs2;
#pragma unroll
                for (int p = 0; p < J1; ++p) gva[p] = r * v[p];
#pragma unroll
                for (int q = 0; q < JB; q += 4) {
                    float g4[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) g4[u] = (q + u < J2) ? r * w2[q + u] : 0.f;
                    atomicAdd(reinterpret_cast<float4 *>(gb + q), make_float4(g4[0], g4[1], g4[2], g4[3]));
                }
                if (A.count_atomics) atomicAdd(gb + JB + k, 1.f);
            }
            add_patient_runs<JA>(gva, J1, valid ? ei : -1, A.gA, A.rs1, k, A.count_atomics);
#pragma unroll
            for (int p = 0; p < J1; ++p)
                *reinterpret_cast<__nv_bfloat16 *>(prt + tc::kmajor_off(p, tid, M)) = __float2bfloat16(r * a[p]);
            tc::fence_smem_to_async();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            if (tid == 0) {
                tc::mma_kmajor(t_m, tc::smem_u32(sRAT), tc::smem_u32(sBT), M, J2, m_started);
                tc::commit(&mbar_m);
            }
            m_started = true;
            m_pending = true;  // waited for before sRAT / sBT are rewritten, or at the merge
            if (__syncthreads_or(!(ok0 && ok1))) {
                failed = true;
                break;
            }
        }
        if (failed) break;
        __syncthreads();  // the next claim is visible
        t = sTile[par ^ 1];
        par ^= 1;
        fetch(t);
    }
    if (failed && tid == 0) atomicOr(A.err, 1);
    // nothing may be in flight when TMEM is released: a pending product is waited for (bounded)
    if (!settle_m() && tid == 0) atomicOr(A.err, 1);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NC));
}

// ---------------------------------------------------------------------------------------
// End of a wave

// Every entry's residual is fitted by four parameter blocks at once (its patient row, gene row,
// platform row and the core), all from the wave-start values; their curvatures are counted
// kBlocks times so that the four proximal steps together do not overshoot the residual
// (additive Schwarz damping).  Directions of small curvature keep the step lr * g.
constexpr float kBlocks = 4.f;
constexpr int kRowWarps = 8;       // warps per CTA of the row step (one row per warp at a time)
constexpr int kRowsPerCta = 64;    // rows of one mode per CTA
constexpr int kTileStride = kMaxRank + 1;
constexpr int kCkStage = 8192;     // platform curvatures staged in shared memory up to this size
// Jacobi sweeps per wave: the eigenbases of the moments drift slowly from wave to wave and
// each decomposition starts from the previous one, so a couple of sweeps keep it tracking
constexpr int kJacobiSweeps = 2;
constexpr int kEigEvery = 4;
constexpr int kRowsPerThreadCta = 256;  // rows per CTA of the thread-per-row step
__host__ __device__ constexpr int pow2_floor(int x) { return x >= 2 ? 2 * pow2_floor(x / 2) : 1; }

// Patient / gene rows: u <- u - (H + (n lambda/|Omega^{n,i}| + 1/lr) I)^{-1} g with
// H = sum_k n_ik C_k (C_k = the platform curvature of this mode), accumulators cleared; then
// the count-weighted second moments of the updated rows (sum_i cnt_i/n u_i u_i^T) into
// gram_out.  With do_step = 0 only the moments are formed.
__device__ void wave_rows(bool first, int blk, int do_step, float *__restrict__ U1, float *__restrict__ U2,
                          float *__restrict__ gA, float *__restrict__ gB, int32_t rs1, int32_t rs2,
                          const int32_t *__restrict__ cnt1, const int32_t *__restrict__ cnt2,
                          const Dims &d, float lam, float inv_lr, float inv_n,
                          const float *__restrict__ curv_in, float *__restrict__ gram_out,
                          const float *__restrict__ wc1, const float *__restrict__ wc2, float *sm) {
    const int J = first ? d.J1 : d.J2;
    const int JP = (J + 3) & ~3;
    const int RS = first ? rs1 : rs2;
    const int I = first ? d.I1 : d.I2;
    const int I3 = d.I3;
    float *U = first ? U1 : U2;
    float *g = first ? gA : gB;
    const int32_t *cnt = first ? cnt1 : cnt2;
    const float *wc = first ? wc1 : wc2;
    const float *Ckg = curv_in + (first ? 0 : (int64_t)I3 * d.J1 * d.J1);  // I3 blocks of J x J
    const int64_t r0 = (int64_t)blk * kRowsPerCta;
    const int64_t left = (int64_t)I - r0;
    const int nr = left < kRowsPerCta ? (int)left : kRowsPerCta;
    if (nr <= 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sH = sm + warp * (kMaxRank * kTileStride + 2 * kMaxRank);  // J x J tile, stride 33
    float *sg = sH + kMaxRank * kTileStride;                           // J
    float *su = sg + kMaxRank;                                         // J
    float *sMom = sm + kRowWarps * (kMaxRank * kTileStride + 2 * kMaxRank);  // kRowWarps x J*J
    float *sCk = sMom + kRowWarps * kMaxRank * kMaxRank;  // platform curvatures, if they fit
    const bool stage = I3 * J * J <= kCkStage;
    if (stage && do_step)
        for (int e = threadIdx.x; e < I3 * J * J; e += blockDim.x) sCk[e] = Ckg[e];
    __syncthreads();
    const float *Ck = stage ? sCk : Ckg;
    float mom[kMaxRank];  // this lane's moment elements lane, lane+32, ... < J*J
    const int nmine = (J * J + 31 - lane) / 32;
    for (int t = 0; t < nmine; ++t) mom[t] = 0.f;
    for (int ri = warp; ri < nr; ri += kRowWarps) {
        const int64_t row = r0 + ri;
        float *acc = g + row * RS;
        // the row's entries per platform in this wave: the set-up table, or the sweep's counts
        const float *wn = wc ? wc + row * I3 : acc + JP;
        float n = 0.f;
        for (int k = 0; k < I3; ++k) n += wn[k];
        if (lane < J) su[lane] = U[row * J + lane];
        __syncwarp();
        if (do_step && n > 0.f) {
            const float diag = kBlocks * n * lam / (float)max(cnt[row], 1) + inv_lr;
            for (int e = lane; e < J * J; e += 32) {
                const int p = e / J, q = e % J;
                float h = p == q ? diag : 0.f;
                for (int k = 0; k < I3; ++k) {
                    const float nk = wn[k];
                    if (nk > 0.f) h = fmaf(kBlocks * nk, Ck[(int64_t)k * J * J + e], h);
                }
                sH[p * kTileStride + q] = h;
            }
            __syncwarp();
            // Cholesky H = L L^T, right-looking (lane l owns row l of the lower triangle)
            for (int j = 0; j < J; ++j) {
                const float dj = sqrtf(fmaxf(sH[j * kTileStride + j], 1e-20f));
                __syncwarp();
                if (lane == j) sH[j * kTileStride + j] = dj;
                if (lane > j && lane < J) sH[lane * kTileStride + j] /= dj;
                __syncwarp();
                if (lane > j && lane < J) {
                    const float lj = sH[lane * kTileStride + j];
                    for (int m = j + 1; m <= lane; ++m) sH[lane * kTileStride + m] -= lj * sH[m * kTileStride + j];
                }
                __syncwarp();
            }
            // L y = g, then L^T x = y; lane l holds component l, columns broadcast by shuffles
            // the data term summed by the sweep, plus the wave's L2 term n lambda/|Omega| u
            const float nreg = n * lam / (float)max(cnt[row], 1);
            float gl = lane < J ? fmaf(nreg, su[lane], acc[lane]) : 0.f;
            for (int i = 0; i < J; ++i) {
                const float xi = __shfl_sync(0xffffffffu, gl, i) / sH[i * kTileStride + i];
                if (lane == i) gl = xi;
                else if (lane > i && lane < J) gl -= sH[lane * kTileStride + i] * xi;
            }
            for (int i = J - 1; i >= 0; --i) {
                const float xi = __shfl_sync(0xffffffffu, gl, i) / sH[i * kTileStride + i];
                if (lane == i) gl = xi;
                else if (lane < i) gl -= sH[i * kTileStride + lane] * xi;
            }
            if (lane < J) {
                su[lane] -= gl;
                U[row * J + lane] = su[lane];
            }
            __syncwarp();
        }
        for (int e = lane; e < RS; e += 32) acc[e] = 0.f;
        const float wgt = (float)cnt[row] * inv_n;
        for (int t = 0; t < nmine; ++t) {
            const int e = lane + 32 * t;
            mom[t] = fmaf(wgt * su[e / J], su[e % J], mom[t]);
        }
        __syncwarp();
    }
    for (int t = 0; t < nmine; ++t) sMom[warp * J * J + lane + 32 * t] = mom[t];
    __syncthreads();
    float *out = gram_out + (first ? 0 : d.J1 * d.J1);
    for (int e = threadIdx.x; e < J * J; e += blockDim.x) {
        float x = 0.f;
        for (int w = 0; w < kRowWarps; ++w) x += sMom[w * J * J + e];
        atomicAdd(out + e, x);
    }
}

// floats of shared memory of the thread-per-row step at rank J: the stepped rows (stride J
// rounded up to even) and the staged platform curvatures
__host__ __device__ inline int64_t rows_thread_floats(int J) {
    return (int64_t)kRowsPerThreadCta * ((J + 1) & ~1) + kCkStage;
}

// The same row step with one thread per row for a compile-time rank J <= 16: H (packed lower
// triangle), its Cholesky factor and both triangular solves stay in registers, with no
// synchronisation inside a row.
template <int CJ>
__device__ void wave_rows_thread(int blk, int do_step, float *__restrict__ U, float *__restrict__ g, int32_t RS,
                                 const int32_t *__restrict__ cnt, int32_t I, int32_t I3, float lam,
                                 float inv_lr, float inv_n, const float *__restrict__ Ckg,
                                 float *__restrict__ gram_out, const float *__restrict__ wc, float *sm,
                                 __nv_bfloat16 *__restrict__ Uh = nullptr) {
    constexpr int J = CJ, JP = (J + 3) & ~3, NL = J * (J + 1) / 2, NLP = (NL + 3) & ~3, JE = (J + 1) & ~1;
    const int64_t r0 = (int64_t)blk * kRowsPerThreadCta;
    if (r0 >= I) return;
    float *rows = sm;                           // kRowsPerThreadCta x JE: updated rows times sqrt(weight)
    float *sCk = rows + kRowsPerThreadCta * JE; // I3 packed lower triangles (NLP floats each), if they fit
    const bool stage = I3 * NLP <= kCkStage;
    const int64_t row = r0 + threadIdx.x;
    const bool valid = row < I;
    // the row's inputs, all loads in flight together
    float u[J], b[J];
    int nrow = 0;
    float n = 0.f;  // the row's entries in this wave
    float *acc = g + row * RS;
    // the row's entries per platform in this wave: the set-up table, or the sweep's counts
    const float *wn = wc ? wc + row * I3 : acc + JP;
    if (valid) {
        nrow = cnt[row];
        if (do_step) {
#pragma unroll 4
            for (int k = 0; k < I3; ++k) n += wn[k];
        }
        if constexpr (J % 2 == 0) {  // the row starts on an 8-byte boundary
#pragma unroll
            for (int p = 0; p < J; p += 2) {
                const float2 v = *reinterpret_cast<const float2 *>(U + row * J + p);
                u[p] = v.x;
                u[p + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int p = 0; p < J; ++p) u[p] = U[row * J + p];
        }
#pragma unroll
        for (int p = 0; p < J; p += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(acc + p);
            b[p] = v.x;
            if (p + 1 < J) b[p + 1] = v.y;
            if (p + 2 < J) b[p + 2] = v.z;
            if (p + 3 < J) b[p + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int p = 0; p < J; ++p) u[p] = b[p] = 0.f;
    }
    if (stage && do_step)  // lower triangles, row p at p (p + 1) / 2
        for (int e = threadIdx.x; e < I3 * NLP; e += blockDim.x) {
            const int k = e / NLP, t = e % NLP;
            int p = 0;
            while ((p + 1) * (p + 2) / 2 <= t) ++p;
            const int q = t - p * (p + 1) / 2;
            sCk[e] = t < NL ? Ckg[(int64_t)k * J * J + p * J + q] : 0.f;
        }
    __syncthreads();
    if (valid) {
        if (do_step && n > 0.f) {
            float L[NL];
            const float nreg = n * lam / (float)max(nrow, 1);  // the wave's L2 weight
            const float diag = kBlocks * nreg + inv_lr;
#pragma unroll
            for (int p = 0, t = 0; p < J; ++p)
#pragma unroll
                for (int q = 0; q <= p; ++q, ++t) L[t] = p == q ? diag : 0.f;
            for (int k = 0; k < I3; ++k) {
                const float nk = kBlocks * wn[k];
                if (nk > 0.f) {
                    if (stage) {
                        const float4 *C4 = reinterpret_cast<const float4 *>(sCk + k * NLP);
#pragma unroll
                        for (int t = 0; t < NLP; t += 4) {
                            const float4 c4 = C4[t / 4];
                            L[t] = fmaf(nk, c4.x, L[t]);
                            if (t + 1 < NL) L[t + 1] = fmaf(nk, c4.y, L[t + 1]);
                            if (t + 2 < NL) L[t + 2] = fmaf(nk, c4.z, L[t + 2]);
                            if (t + 3 < NL) L[t + 3] = fmaf(nk, c4.w, L[t + 3]);
                        }
                    } else {
                        const float *C = Ckg + (int64_t)k * J * J;
#pragma unroll
                        for (int p = 0, t = 0; p < J; ++p)
#pragma unroll
                            for (int q = 0; q <= p; ++q, ++t) L[t] = fmaf(nk, C[p * J + q], L[t]);
                    }
                }
            }
            // Cholesky (packed lower triangle, row p starts at p (p + 1) / 2); the inverse
            // diagonal is kept, so the solves below multiply instead of dividing
            float dinv[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                float dd = L[j * (j + 1) / 2 + j];
#pragma unroll
                for (int k = 0; k < j; ++k) dd -= L[j * (j + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
                const float inv = rsqrtf(fmaxf(dd, 1e-20f));
                dinv[j] = inv;
#pragma unroll
                for (int i = j + 1; i < J; ++i) {
                    float x = L[i * (i + 1) / 2 + j];
#pragma unroll
                    for (int k = 0; k < j; ++k) x -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
                    L[i * (i + 1) / 2 + j] = x * inv;
                }
            }
            float y[J];
#pragma unroll
            for (int i = 0; i < J; ++i) {
                // the data term summed by the sweep, plus the wave's L2 term n lambda/|Omega| u
                float x = fmaf(nreg, u[i], b[i]);
#pragma unroll
                for (int k = 0; k < i; ++k) x -= L[i * (i + 1) / 2 + k] * y[k];
                y[i] = x * dinv[i];
            }
#pragma unroll
            for (int i = J - 1; i >= 0; --i) {
                float x = y[i];
#pragma unroll
                for (int k = i + 1; k < J; ++k) x -= L[k * (k + 1) / 2 + i] * y[k];
                y[i] = x * dinv[i];
            }
#pragma unroll
            for (int p = 0; p < J; ++p) u[p] -= y[p];
            if constexpr (J % 2 == 0) {
#pragma unroll
                for (int p = 0; p < J; p += 2)
                    *reinterpret_cast<float2 *>(U + row * J + p) = make_float2(u[p], u[p + 1]);
            } else {
#pragma unroll
                for (int p = 0; p < J; ++p) U[row * J + p] = u[p];
            }
            if (Uh) {  // the BF16 copy the BF16-gather sweep reads
                if constexpr (J % 2 == 0) {
#pragma unroll
                    for (int p = 0; p < J; p += 2)
                        *reinterpret_cast<__nv_bfloat162 *>(Uh + row * J + p) = __floats2bfloat162_rn(u[p], u[p + 1]);
                } else {
#pragma unroll
                    for (int p = 0; p < J; ++p) Uh[row * J + p] = __float2bfloat16(u[p]);
                }
            }
        }
    }
    {  // the row's share of the moments: weight cnt / n, folded into the row as its square root
        const float sw = sqrtf((float)nrow * inv_n);
#pragma unroll
        for (int p = 0; p < JE; ++p) rows[threadIdx.x * JE + p] = p < J ? sw * u[p] : 0.f;
    }
    __syncthreads();
    {  // every thread has read its accumulators: clear the CTA's rows of them, coalesced
        const int nr = (int)(I - r0 < kRowsPerThreadCta ? I - r0 : kRowsPerThreadCta);
        float4 *a4 = reinterpret_cast<float4 *>(g + r0 * RS);  // RS is a multiple of 4
        for (int t = threadIdx.x; t < nr * RS / 4; t += blockDim.x) a4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // moments sum_i w_i u_i u_i^T: one 2 x 2 block (rows p, p + 1; columns q, q + 1; p <= q) per
    // group of R consecutive lanes, lane h of the group taking rows h, h + R, ...; the group's
    // sums meet by shuffles and its first lane adds the block and its mirror image
    constexpr int NB = JE / 2, NBLK = NB * (NB + 1) / 2;
    constexpr int R = pow2_floor(NBLK >= kRowsPerThreadCta ? 1 : (kRowsPerThreadCta / NBLK < 32 ? kRowsPerThreadCta / NBLK : 32));
    static_assert(kRowsPerThreadCta % R == 0 && 32 % R == 0, "row groups");
    for (int base = 0; base < NBLK * R; base += blockDim.x) {
        const int t = base + threadIdx.x, bk = t / R, h = t % R;
        float m00 = 0.f, m01 = 0.f, m10 = 0.f, m11 = 0.f;
        int bp = 0, bq = 0;
        if (bk < NBLK) {
            // block bk -> (bp, bq), bp <= bq, in row-major order of the upper triangle
            int rem = bk;
            while (rem >= NB - bp) { rem -= NB - bp; ++bp; }
            bq = bp + rem;
#pragma unroll 4
            for (int i = h; i < kRowsPerThreadCta; i += R) {
                const float2 x = *reinterpret_cast<const float2 *>(rows + i * JE + 2 * bp);
                const float2 y = *reinterpret_cast<const float2 *>(rows + i * JE + 2 * bq);
                m00 = fmaf(x.x, y.x, m00);
                m01 = fmaf(x.x, y.y, m01);
                m10 = fmaf(x.y, y.x, m10);
                m11 = fmaf(x.y, y.y, m11);
            }
        }
#pragma unroll
        for (int o = R / 2; o; o >>= 1) {
            m00 += __shfl_xor_sync(0xffffffffu, m00, o);
            m01 += __shfl_xor_sync(0xffffffffu, m01, o);
            m10 += __shfl_xor_sync(0xffffffffu, m10, o);
            m11 += __shfl_xor_sync(0xffffffffu, m11, o);
        }
        if (bk < NBLK && h == 0) {
            const int p = 2 * bp, q = 2 * bq;
            const float m[4] = {m00, m01, m10, m11};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int pp = p + (c >> 1), qq = q + (c & 1);
                if (pp < J && qq < J) {
                    atomicAdd(gram_out + pp * J + qq, m[c]);
                    if (bp != bq) atomicAdd(gram_out + qq * J + pp, m[c]);
                }
            }
        }
    }
}

// Eigen-decomposition of a symmetric n x n matrix (n <= 32) by Jacobi rotations, one warp.
// M (row stride ld >= n) is overwritten: its diagonal ends as the eigenvalues; V (stride ld)
// holds the eigenvectors as columns.  Vwarm (n x n, global) is the previous decomposition: M
// is first rotated into that basis, so a slowly changing matrix needs few sweeps; the result
// is written back to Vwarm.  T (n x ld, and at least 64 floats) is scratch.
// A sweep runs in round-robin order: n - 1 rounds (n rounded up to even) of n/2 disjoint
// pairs, whose rotations are found from the same M and applied together (disjoint Givens
// rotations commute), so a round costs about as much as one rotation of the cyclic order.
__device__ __forceinline__ int rr_pos(int i, int r, int np) { return i == 0 ? 0 : 1 + (i - 1 + r) % (np - 1); }

__device__ void warp_jacobi(float *M, float *V, float *T, int n, int ld, float *Vwarm, int max_sweeps) {
    const int lane = threadIdx.x & 31;
    // V = Vwarm (identity if it is all zero), M <- V^T M V
    float vsum = 0.f;
    for (int e = lane; e < n * n; e += 32) vsum += fabsf(Vwarm[e]);
#pragma unroll
    for (int o = 16; o; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
    for (int e = lane; e < n * n; e += 32) {
        const int p = e / n, q = e % n;
        V[p * ld + q] = vsum > 0.f ? Vwarm[e] : (p == q ? 1.f : 0.f);
    }
    __syncwarp();
    for (int e = lane; e < n * n; e += 32) {  // T = M V
        const int p = e / n, q = e % n;
        float x = 0.f;
        for (int k = 0; k < n; ++k) x = fmaf(M[p * ld + k], V[k * ld + q], x);
        T[p * ld + q] = x;
    }
    __syncwarp();
    for (int e = lane; e < n * n; e += 32) {  // M = V^T T
        const int p = e / n, q = e % n;
        float x = 0.f;
        for (int k = 0; k < n; ++k) x = fmaf(V[k * ld + p], T[k * ld + q], x);
        M[p * ld + q] = x;
    }
    __syncwarp();
    const int np = (n + 1) & ~1, npairs = np / 2;
    // the round's pairs and rotations, in the scratch tile
    int *rP = reinterpret_cast<int *>(T), *rQ = rP + 16;
    float *rC = T + 32, *rS = T + 48;
    for (int sweep = 0; sweep < max_sweeps && n > 1; ++sweep) {
        float off = 0.f, dia = 0.f;
        for (int e = lane; e < n * n; e += 32) {
            const float x = M[(e / n) * ld + e % n];
            if (e / n != e % n) off += x * x; else dia += x * x;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if (off <= 1e-12f * dia || !(dia > 0.f)) break;
        for (int r = 0; r < np - 1; ++r) {
            if (lane < npairs) {
                const int a = rr_pos(lane, r, np), b = rr_pos(np - 1 - lane, r, np);
                const int p = min(a, b), q = max(a, b);
                float cs = 1.f, sn = 0.f;
                if (q < n) {  // (index n is the padding of an odd n)
                    const float apq = M[p * ld + q];
                    const float app = M[p * ld + p], aqq = M[q * ld + q];
                    if (fabsf(apq) > 1e-9f * sqrtf(fabsf(app * aqq)) + 1e-30f) {
                        const float theta = (aqq - app) / (2.f * apq);
                        const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
                        cs = rsqrtf(t * t + 1.f);
                        sn = t * cs;
                    }
                }
                rP[lane] = p;
                rQ[lane] = q < n ? q : p;  // a padded pair rotates nothing (cs = 1, sn = 0)
                rC[lane] = cs;
                rS[lane] = sn;
            }
            __syncwarp();
            for (int t = lane; t < n * npairs; t += 32) {  // columns p, q of M and of V
                const int i = t / npairs, k = t % npairs;
                const int p = rP[k], q = rQ[k];
                if (p == q) continue;
                const float cs = rC[k], sn = rS[k];
                const float mip = M[i * ld + p], miq = M[i * ld + q];
                M[i * ld + p] = cs * mip - sn * miq;
                M[i * ld + q] = sn * mip + cs * miq;
                const float vip = V[i * ld + p], viq = V[i * ld + q];
                V[i * ld + p] = cs * vip - sn * viq;
                V[i * ld + q] = sn * vip + cs * viq;
            }
            __syncwarp();
            for (int t = lane; t < npairs * n; t += 32) {  // rows p, q of M
                const int k = t / n, j = t % n;
                const int p = rP[k], q = rQ[k];
                if (p == q) continue;
                const float cs = rC[k], sn = rS[k];
                const float mpj = M[p * ld + j], mqj = M[q * ld + j];
                M[p * ld + j] = cs * mpj - sn * mqj;
                M[q * ld + j] = sn * mpj + cs * mqj;
            }
            __syncwarp();
        }
    }
    for (int e = lane; e < n * n; e += 32) Vwarm[e] = V[(e / n) * ld + e % n];
    __syncwarp();
}

// The wave-independent half of the dense step, taken during the wave's sweep by extra CTAs
// of the sweep launch (three in the FP32 fast sweep, one part each; one CTA elsewhere): it
// needs only values fixed before the sweep (G, the platform rows, the moments of the
// previous wave end, the wave's platform counts).  Its three parts are independent.
//   * Cn = sum_k n_k c_k c_k^T and the eigen-decompositions of Ma, Mb, Cn (Jacobi sweeps from
//     the previous eigenbasis every kEigEvery-th wave; in between the eigenbasis is kept and
//     the eigenvalues refreshed as its Rayleigh quotients) -> eigv, eigval;
//   * H = G_(3) (Ma kron Mb) G_(3)^T and the inverse of each platform row's system
//     (4 (n_k H + n_k lambda/|Omega^{3,k}| I) + I/lr) -> ainv (zero for a platform without
//     entries in the wave);
//   * the platform curvatures C1_k = Gc_k Mb Gc_k^T, C2_k = Gc_k^T Ma Gc_k (Gc_k = G x3 c_k)
//     for the wave's row steps -> curv.
template <int CJ1, int CJ2, int CJ3>
__device__ void dense_pre(const DenseArgs &A, float *sm, int part) {
    const Dims &d = A.d;
    constexpr bool kFixed = CJ1 > 0 && CJ2 > 0 && CJ3 > 0;
    const int J1 = kFixed ? CJ1 : d.J1, J2 = kFixed ? CJ2 : d.J2, J3 = kFixed ? CJ3 : d.J3;
    const int I3 = d.I3, PI = J1 * J2 * J3, Q = J1 * J2;
    const int ld = kFixed ? (CJ1 > CJ2 ? (CJ1 > CJ3 ? CJ1 : CJ3) : (CJ2 > CJ3 ? CJ2 : CJ3)) + 1 : eig_ld(d);
    const int TS = eig_tile(d);
    float *sG = sm;                  // PI
    float *sX = sG + PI;             // PI (scratch)
    float *sT = sX + PI;             // PI (scratch)
    float *sC = sT + PI;             // I3*J3
    float *sCn = sC + I3 * J3;       // J3*J3
    float *sH = sCn + J3 * J3;       // J3*J3
    float *sMa = sH + J3 * J3;       // J1*J1
    float *sMb = sMa + J1 * J1;      // J2*J2
    float *sJ = sMb + J2 * J2;       // 3 x (M, V, T) tiles
    float *sAk = sJ + 9 * TS;        // I3 x J3 x J3 platform systems
    const int tid = threadIdx.x, nt = blockDim.x;
    // part 0: eigenbases; 1: H and the platform-system inverses; 2: row curvatures; -1: all
    const bool want_eig = part < 0 || part == 0, want_h = part < 0 || part == 1, want_curv = part < 0 || part == 2;
    if (want_h || want_curv)
        for (int s = tid; s < PI; s += nt) sG[s] = A.G[s];
    if (want_eig || want_curv)
        for (int s = tid; s < I3 * J3; s += nt) sC[s] = A.U3[s];
    for (int s = tid; s < J1 * J1 + J2 * J2; s += nt) sMa[s] = A.gram_in[s];  // Ma, Mb (contiguous)
    __syncthreads();
    if (want_eig)
        for (int s = tid; s < J3 * J3; s += nt) {
            const int r = s / J3, t = s % J3;
            float a = 0.f;
            for (int k = 0; k < I3; ++k) a = fmaf(A.nk[k] * sC[k * J3 + r], sC[k * J3 + t], a);
            sCn[s] = a;
        }
    if (want_h)
        for (int s = tid; s < PI; s += nt) {  // X[r][p][q'] = sum_p' Ma[p][p'] g(p', q', r)
            const int r = s / Q, p = (s / J2) % J1, q = s % J2;
            float a = 0.f;
#pragma unroll
            for (int pp = 0; pp < J1; ++pp) a = fmaf(sMa[p * J1 + pp], sG[(pp * J2 + q) * J3 + r], a);
            sX[s] = a;
        }
    __syncthreads();
    const int warp = tid >> 5;
    if (want_eig && warp < 3) {  // eigen-decompositions of Ma, Mb, Cn, one warp each
        const bool full_eig = (*A.wave_counter % kEigEvery) == 0;
        const int n = warp == 0 ? J1 : (warp == 1 ? J2 : J3);
        const float *src = warp == 0 ? sMa : (warp == 1 ? sMb : sCn);
        float *M = sJ + warp * 3 * TS, *V = M + TS, *T = V + TS;
        for (int e = (tid & 31); e < n * n; e += 32) M[(e / n) * ld + e % n] = src[e];
        __syncwarp();
        const int off = warp == 0 ? 0 : (warp == 1 ? J1 * J1 : J1 * J1 + J2 * J2);
        warp_jacobi(M, V, T, n, ld, A.eigv + off, full_eig ? kJacobiSweeps : 0);
        const int eoff = warp == 0 ? 0 : (warp == 1 ? J1 : J1 + J2);
        for (int p = (tid & 31); p < n; p += 32) A.eigval[eoff + p] = M[p * ld + p];
    }
    if (want_h) {
        for (int s = tid; s < PI; s += nt) {  // T[r][p][q] = sum_q' X[r][p][q'] Mb[q'][q]
            const int r = s / Q, p = (s / J2) % J1, q = s % J2;
            float a = 0.f;
#pragma unroll
            for (int qq = 0; qq < J2; ++qq) a = fmaf(sX[(r * J1 + p) * J2 + qq], sMb[qq * J2 + q], a);
            sT[s] = a;
        }
        __syncthreads();
        // H[r][t] = sum_pq g(p,q,r) T[t][p][q]: TP lanes per output, partial sums met by shuffles
        const int NO = J3 * J3;
        int TP = 1;
        while (TP < 32 && 2 * TP * NO <= nt) TP *= 2;
        for (int base = 0; base < NO * TP; base += nt) {  // the same trip count in every thread
            const int t = base + tid, o = t / TP, h = t % TP;
            float a = 0.f;
            if (o < NO) {
                const int r = o / J3, tt = o % J3;
                for (int pq = h; pq < Q; pq += TP) a = fmaf(sG[pq * J3 + r], sT[tt * Q + pq], a);
            }
            for (int w = TP / 2; w; w >>= 1) a += __shfl_xor_sync(0xffffffffu, a, w);
            if (o < NO && h == 0) sH[o] = a;
        }
        __syncthreads();
        for (int k = tid; k < I3; k += nt) {  // platform row k: the inverse of (4 (n_k H + reg I) + I/lr)
            float *inv = A.ainv + (int64_t)k * J3 * J3;
            const float nk = A.nk[k];
            if (!(nk > 0.f)) {
                for (int e = 0; e < J3 * J3; ++e) inv[e] = 0.f;
                continue;
            }
            const float reg = A.cnt3[k] > 0 ? nk * A.lam / (float)A.cnt3[k] : 0.f;
            if constexpr (kFixed) {  // Cholesky and both solves in registers
                constexpr int N = CJ3;
                float L[N][N], dinv[N];
#pragma unroll
                for (int r = 0; r < N; ++r)
#pragma unroll
                    for (int t = 0; t <= r; ++t)
                        L[r][t] = kBlocks * (nk * sH[r * N + t] + (r == t ? reg : 0.f)) + (r == t ? 1.f / A.lr : 0.f);
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    float dd = L[j][j];
#pragma unroll
                    for (int q = 0; q < j; ++q) dd -= L[j][q] * L[j][q];
                    dinv[j] = rsqrtf(fmaxf(dd, 1e-20f));
#pragma unroll
                    for (int i = j + 1; i < N; ++i) {
                        float x = L[i][j];
#pragma unroll
                        for (int q = 0; q < j; ++q) x -= L[i][q] * L[j][q];
                        L[i][j] = x * dinv[j];
                    }
                }
#pragma unroll
                for (int c = 0; c < N; ++c) {  // column c of the inverse: L L^T x = e_c
                    float y[N];
#pragma unroll
                    for (int i = 0; i < N; ++i) {
                        float x = i == c ? 1.f : 0.f;
#pragma unroll
                        for (int q = 0; q < i; ++q) x -= L[i][q] * y[q];
                        y[i] = x * dinv[i];
                    }
#pragma unroll
                    for (int i = N - 1; i >= 0; --i) {
                        float x = y[i];
#pragma unroll
                        for (int q = i + 1; q < N; ++q) x -= L[q][i] * y[q];
                        y[i] = x * dinv[i];
                    }
#pragma unroll
                    for (int i = 0; i < N; ++i) inv[i * N + c] = y[i];
                }
            } else {
                float *Ak = sAk + k * J3 * J3;
                for (int r = 0; r < J3; ++r)
                    for (int t = 0; t < J3; ++t)
                        Ak[r * J3 + t] =
                            kBlocks * (nk * sH[r * J3 + t] + (r == t ? reg : 0.f)) + (r == t ? 1.f / A.lr : 0.f);
                for (int j = 0; j < J3; ++j) {
                    float dd = Ak[j * J3 + j];
                    for (int q = 0; q < j; ++q) dd -= Ak[j * J3 + q] * Ak[j * J3 + q];
                    dd = sqrtf(fmaxf(dd, 1e-20f));
                    Ak[j * J3 + j] = dd;
                    for (int i = j + 1; i < J3; ++i) {
                        float x = Ak[i * J3 + j];
                        for (int q = 0; q < j; ++q) x -= Ak[i * J3 + q] * Ak[j * J3 + q];
                        Ak[i * J3 + j] = x / dd;
                    }
                }
                for (int c = 0; c < J3; ++c) {  // column c of the inverse: L L^T x = e_c
                    float y[kMaxRank];
                    for (int i = 0; i < J3; ++i) {
                        float x = i == c ? 1.f : 0.f;
                        for (int q = 0; q < i; ++q) x -= Ak[i * J3 + q] * y[q];
                        y[i] = x / Ak[i * J3 + i];
                    }
                    for (int i = J3 - 1; i >= 0; --i) {
                        float x = y[i];
                        for (int q = i + 1; q < J3; ++q) x -= Ak[q * J3 + i] * y[q];
                        y[i] = x / Ak[i * J3 + i];
                    }
                    for (int i = 0; i < J3; ++i) inv[i * J3 + c] = y[i];
                }
            }
        }
    }
    if (!want_curv) return;
    // platform curvatures for the wave's row steps (moments of gram_in): all platforms at once
    // when their Gc and W fit in the two PI-sized scratch buffers
    __syncthreads();  // sX, sT free (part -1)
    float *sGc = sX, *sW = sT;
    const int kb = (I3 * Q <= PI) ? I3 : 1;  // platforms per batch
    for (int k0 = 0; k0 < I3; k0 += kb) {
        const int nkb = min(kb, I3 - k0);
        for (int s = tid; s < nkb * Q; s += nt) {  // Gc_k = G x3 c_k
            const int k = k0 + s / Q, pq = s % Q;
            float a = 0.f;
#pragma unroll
            for (int r = 0; r < J3; ++r) a = fmaf(sG[pq * J3 + r], sC[k * J3 + r], a);
            sGc[s] = a;
        }
        __syncthreads();
        for (int s = tid; s < nkb * Q; s += nt) {  // W1 = Gc Mb  (J1 x J2)
            const int b = s / Q, p = (s % Q) / J2, q = s % J2;
            float a = 0.f;
#pragma unroll
            for (int qq = 0; qq < J2; ++qq) a = fmaf(sGc[b * Q + p * J2 + qq], sMb[qq * J2 + q], a);
            sW[s] = a;
        }
        __syncthreads();
        for (int s = tid; s < nkb * J1 * J1; s += nt) {  // C1 = W1 Gc^T
            const int b = s / (J1 * J1), p = (s / J1) % J1, t = s % J1;
            float a = 0.f;
#pragma unroll
            for (int q = 0; q < J2; ++q) a = fmaf(sW[b * Q + p * J2 + q], sGc[b * Q + t * J2 + q], a);
            A.curv[(int64_t)(k0 + b) * J1 * J1 + p * J1 + t] = a;
        }
        __syncthreads();
        for (int s = tid; s < nkb * Q; s += nt) {  // W2 = Ma Gc  (J1 x J2)
            const int b = s / Q, p = (s % Q) / J2, q = s % J2;
            float a = 0.f;
#pragma unroll
            for (int pp = 0; pp < J1; ++pp) a = fmaf(sMa[p * J1 + pp], sGc[b * Q + pp * J2 + q], a);
            sW[s] = a;
        }
        __syncthreads();
        float *C2 = A.curv + (int64_t)I3 * J1 * J1;
        for (int s = tid; s < nkb * J2 * J2; s += nt) {  // C2 = Gc^T W2
            const int b = s / (J2 * J2), q = (s / J2) % J2, t = s % J2;
            float a = 0.f;
#pragma unroll
            for (int p = 0; p < J1; ++p) a = fmaf(sGc[b * Q + p * J2 + q], sW[b * Q + p * J2 + t], a);
            C2[(int64_t)(k0 + b) * J2 * J2 + q * J2 + t] = a;
        }
        __syncthreads();
    }
}

// The rest of the dense step at the end of the wave (one CTA), with the wave's M_k:
//   platform gradients g_k = G_(3) vec(M_k) + reg c_k and steps delta_k = ainv_k g_k;
//   core gradient D = sum_k M_k kron c_k + n lambda/|Omega| G, solved in the eigenbases:
//   G <- G - (Va, Vb, Vc) [ (D x1 Va^T x2 Vb^T x3 Vc^T) / (4 la lb lc + diag) ];
//   then the moments of the previous wave end are cleared for reuse.
// CJ1, CJ2, CJ3: the core ranks when fixed at compile time (0: read from A.d).
template <int CJ1, int CJ2, int CJ3>
__device__ void dense_post(const DenseArgs &A, float *sm) {
    const Dims &d = A.d;
    constexpr bool kFixed = CJ1 > 0 && CJ2 > 0 && CJ3 > 0;
    const int J1 = kFixed ? CJ1 : d.J1, J2 = kFixed ? CJ2 : d.J2, J3 = kFixed ? CJ3 : d.J3;
    const int I3 = d.I3, PI = J1 * J2 * J3, Q = J1 * J2, J23 = J2 * J3;
    const int ld = kFixed ? (CJ1 > CJ2 ? (CJ1 > CJ3 ? CJ1 : CJ3) : (CJ2 > CJ3 ? CJ2 : CJ3)) + 1 : eig_ld(d);
    float *sG = sm;                  // PI
    float *sX = sG + PI;             // PI (scratch)
    float *sT = sX + PI;             // PI (scratch)
    float *sC = sT + PI;             // I3*J3
    float *sGk = sC + I3 * J3;       // I3*J3 platform gradients
    float *sDel = sGk + I3 * J3;     // I3*J3 platform steps
    float *Va = sDel + I3 * J3;      // J1 x ld
    float *Vb = Va + J1 * ld;        // J2 x ld
    float *Vc = Vb + J2 * ld;        // J3 x ld
    float *la = Vc + J3 * ld;        // J1 + J2 + J3 eigenvalues
    float *sInv = la + J1 + J2 + J3; // I3 x J3 x J3 platform-system inverses
    float *sNk = sInv + I3 * J3 * J3;  // I3: the wave's entries per platform
    float *sCnt = sNk + I3;          // I3: all entries per platform
    float *sMacc = sCnt + I3;        // the wave's M_k, if they fit
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool stage_m = I3 * Q <= kMaccStage;
    const float *Mk = stage_m ? sMacc : A.macc;
    {  // every input of the step, eight loads per thread in flight at a time
        const int o1 = stage_m ? I3 * Q : 0, o2 = o1 + PI, o3 = o2 + I3 * J3, o4 = o3 + J1 * J1,
                  o5 = o4 + J2 * J2, o6 = o5 + J3 * J3, o7 = o6 + J1 + J2 + J3, o8 = o7 + I3 * J3 * J3,
                  o9 = o8 + I3, N = o9 + I3;
        for (int base = tid; base < N; base += 8 * nt) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = base + u * nt;
                v[u] = t >= N ? 0.f
                       : t < o1 ? A.macc[t]
                       : t < o2 ? A.G[t - o1]
                       : t < o3 ? A.U3[t - o2]
                       : t < o6 ? A.eigv[t - o3]  // Ma, Mb, Cn eigenvectors, contiguous
                       : t < o7 ? A.eigval[t - o6]
                       : t < o8 ? A.ainv[t - o7]
                       : t < o9 ? A.nk[t - o8]
                                : (float)A.cnt3[t - o9];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = base + u * nt;
                if (t >= N) continue;
                if (t < o1) {
                    sMacc[t] = v[u];
                } else if (t < o2) {
                    sG[t - o1] = v[u];
                } else if (t < o3) {
                    sC[t - o2] = v[u];
                } else if (t < o4) {
                    const int e = t - o3;
                    Va[(e / J1) * ld + e % J1] = v[u];
                } else if (t < o5) {
                    const int e = t - o4;
                    Vb[(e / J2) * ld + e % J2] = v[u];
                } else if (t < o6) {
                    const int e = t - o5;
                    Vc[(e / J3) * ld + e % J3] = v[u];
                } else if (t < o7) {
                    la[t - o6] = fmaxf(v[u], 0.f);
                } else {
                    sInv[t - o7] = v[u];  // then sNk, sCnt (contiguous)
                }
            }
        }
    }
    __syncthreads();
    const float *lb = la + J1, *lc = la + J1 + J2;
    {  // platform gradients: TP lanes per output, partial sums met by shuffles
        const int NO = I3 * J3;
        int TP = 1;
        while (TP < 32 && 2 * TP * NO <= nt) TP *= 2;
        for (int base = 0; base < NO * TP; base += nt) {  // the same trip count in every thread
            const int t = base + tid, o = t / TP, h = t % TP;
            float a = 0.f;
            if (o < NO) {
                const int k = o / J3, r = o % J3;
                const float *M = Mk + (int64_t)k * Q;
                for (int pq = h; pq < Q; pq += TP) a = fmaf(sG[pq * J3 + r], M[pq], a);
            }
            for (int w = TP / 2; w; w >>= 1) a += __shfl_xor_sync(0xffffffffu, a, w);
            if (o < NO && h == 0) {
                const int k = o / J3;
                const float reg = sCnt[k] > 0.f ? sNk[k] * A.lam / sCnt[k] : 0.f;
                sGk[o] = fmaf(reg, sC[o], a);
            }
        }
    }
    for (int s = tid; s < PI; s += nt) {  // core gradient D
        const int pq = s / J3, r = s % J3;
        float a = 0.f;
        for (int k = 0; k < I3; ++k) a = fmaf(Mk[(int64_t)k * Q + pq], sC[k * J3 + r], a);
        sX[s] = fmaf(A.n_wave * A.lam_core, sG[s], a);
    }
    __syncthreads();
    for (int s = tid; s < I3 * J3; s += nt) {  // platform steps
        const int k = s / J3, r = s % J3;
        const float *inv = sInv + (k * J3 + r) * J3;
        float a = 0.f;
#pragma unroll
        for (int t = 0; t < J3; ++t) a = fmaf(inv[t], sGk[k * J3 + t], a);
        sDel[s] = a;
    }
    // D <- D x1 Va^T x2 Vb^T x3 Vc^T   (index s = (p*J2 + q)*J3 + r)
    for (int s = tid; s < PI; s += nt) {
        const int p = s / J23, qr = s % J23;
        float a = 0.f;
#pragma unroll
        for (int pp = 0; pp < J1; ++pp) a = fmaf(Va[pp * ld + p], sX[pp * J23 + qr], a);
        sT[s] = a;
    }
    __syncthreads();
    for (int s = tid; s < PI; s += nt) {
        const int p = s / J23, q = (s / J3) % J2, r = s % J3;
        float a = 0.f;
#pragma unroll
        for (int qq = 0; qq < J2; ++qq) a = fmaf(Vb[qq * ld + q], sT[p * J23 + qq * J3 + r], a);
        sX[s] = a;
    }
    __syncthreads();
    const float diag = 1.f / A.lr + kBlocks * A.n_wave * A.lam_core;
    for (int s = tid; s < PI; s += nt) {
        const int p = s / J23, q = (s / J3) % J2, r = s % J3;
        float a = 0.f;
#pragma unroll
        for (int rr = 0; rr < J3; ++rr) a = fmaf(Vc[rr * ld + r], sX[(s - r) + rr], a);
        sT[s] = a / (kBlocks * la[p] * lb[q] * lc[r] + diag);
    }
    __syncthreads();
    // back: D <- D x1 Va x2 Vb x3 Vc
    for (int s = tid; s < PI; s += nt) {
        const int p = s / J23, qr = s % J23;
        float a = 0.f;
#pragma unroll
        for (int pp = 0; pp < J1; ++pp) a = fmaf(Va[p * ld + pp], sT[pp * J23 + qr], a);
        sX[s] = a;
    }
    __syncthreads();
    for (int s = tid; s < PI; s += nt) {
        const int p = s / J23, q = (s / J3) % J2, r = s % J3;
        float a = 0.f;
#pragma unroll
        for (int qq = 0; qq < J2; ++qq) a = fmaf(Vb[q * ld + qq], sX[p * J23 + qq * J3 + r], a);
        sT[s] = a;
    }
    __syncthreads();
    for (int s = tid; s < PI; s += nt) {
        const int r = s % J3;
        float a = 0.f;
#pragma unroll
        for (int rr = 0; rr < J3; ++rr) a = fmaf(Vc[r * ld + rr], sT[(s - r) + rr], a);
        A.G[s] = sG[s] - a;
    }
    for (int s = tid; s < I3 * J3; s += nt) A.U3[s] = sC[s] - sDel[s];
    for (int s = tid; s < I3 * Q; s += nt) A.macc[s] = 0.f;
    for (int s = tid; s < J1 * J1 + J2 * J2; s += nt) A.gram_in[s] = 0.f;
    if (tid == 0) *A.wave_counter += 1;
}

struct RowArgs {
    float *U1, *U2, *gA, *gB;
    int32_t rs1, rs2;
    const int32_t *cnt1, *cnt2;
    float inv_n;
    int32_t nb1;
    const float *curv_in;
    float *gram_out;
    const float *wc1, *wc2;  // this wave's entries per (row, platform) of each mode, or null
    __nv_bfloat16 *U2h;      // BF16 copy of the gene rows to keep current, or null
};

// End of a wave.  mode 0: CTA 0 = the rest of the core and platform-row step (dense_post),
// CTAs 1.. = patient and gene rows (curvatures from the wave's pre-work) + new moments.
// mode 1 (set-up): rows form moments only.
// The row step runs one thread per row when both row ranks are compile-time (CJ1, CJ2 > 0),
// one warp per row otherwise; R.nb1 CTAs cover the patient rows, the rest the gene rows.
template <int CJ1, int CJ2>
__device__ void wave_end_rows(const DenseArgs &A, const RowArgs &R, int blk, int mode, float *smw) {
    const bool first = blk < R.nb1;
    const int mb = first ? blk : blk - R.nb1;
    const Dims &d = A.d;
    if constexpr (CJ1 > 0 && CJ2 > 0) {
        const float *Ckg = R.curv_in + (first ? 0 : (int64_t)d.I3 * d.J1 * d.J1);
        float *gout = R.gram_out + (first ? 0 : d.J1 * d.J1);
        if (first)
            wave_rows_thread<CJ1>(mb, mode == 0, R.U1, R.gA, R.rs1, R.cnt1, d.I1, d.I3, A.lam, 1.f / A.lr,
                                  R.inv_n, Ckg, gout, R.wc1, smw);
        else
            wave_rows_thread<CJ2>(mb, mode == 0, R.U2, R.gB, R.rs2, R.cnt2, d.I2, d.I3, A.lam, 1.f / A.lr,
                                  R.inv_n, Ckg, gout, R.wc2, smw, R.U2h);
    } else {
        wave_rows(first, mb, mode == 0, R.U1, R.U2, R.gA, R.gB, R.rs1, R.rs2, R.cnt1, R.cnt2, d, A.lam,
                  1.f / A.lr, R.inv_n, R.curv_in, R.gram_out, R.wc1, R.wc2, smw);
    }
}

template <int CJ1, int CJ2, int CJ3>
__global__ void __launch_bounds__(256) k_fast_wave_end(DenseArgs A, RowArgs R, int mode) {
    extern __shared__ __align__(16) float smw[];
    if (blockIdx.x == 0) {
        if (mode == 0) dense_post<CJ1, CJ2, CJ3>(A, smw);
        return;
    }
    wave_end_rows<CJ1, CJ2>(A, R, blockIdx.x - 1, mode, smw);
}

// The end of one wave for every problem of a batch: per problem one CTA takes the dense step
// and the next ones its row steps (boff: prefix offsets of the problems' CTAs).
template <int CJ1, int CJ2, int CJ3>
__global__ void __launch_bounds__(256)
    k_batch_wave_end(const DenseArgs *__restrict__ dargs, const RowArgs *__restrict__ rargs,
                     const int32_t *__restrict__ boff, int32_t P) {
    extern __shared__ __align__(16) float smw[];
    __shared__ int sPid;
    if (threadIdx.x == 0) {
        int lo = 0, hi = P - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (boff[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        sPid = lo;
    }
    __syncthreads();
    const int pid = sPid;
    const int local = (int)blockIdx.x - boff[pid];
    const DenseArgs A = dargs[pid];
    const RowArgs R = rargs[pid];
    if (local == 0) {
        dense_post<CJ1, CJ2, CJ3>(A, smw);
        return;
    }
    wave_end_rows<CJ1, CJ2>(A, R, local - 1, 0, smw);
}

// compile-time row ranks of the thread-per-row step, and all three ranks of the dense step
// where they match a common configuration
#define SNECT_DISPATCH_ROWS(J1, J2, J3, FN, ...)                                  \
    (((J1) == 5 && (J2) == 5)     ? ((J3) == 2 ? FN<5, 5, 2>(__VA_ARGS__)          \
                                               : FN<5, 5, 0>(__VA_ARGS__))         \
     : ((J1) == 10 && (J2) == 10) ? ((J3) == 5 ? FN<10, 10, 5>(__VA_ARGS__)        \
                                               : FN<10, 10, 0>(__VA_ARGS__))       \
     : ((J1) == 16 && (J2) == 16) ? ((J3) == 5 ? FN<16, 16, 5>(__VA_ARGS__)        \
                                               : FN<16, 16, 0>(__VA_ARGS__))       \
                                  : FN<0, 0, 0>(__VA_ARGS__))

template <int CJ1, int CJ2>
int rows_per_cta() { return (CJ1 > 0 && CJ2 > 0) ? kRowsPerThreadCta : kRowsPerCta; }

// the sweep's shared-memory carveout too, so that the SMs keep one configuration across
// the kernels of an epoch
template <int CJ1, int CJ2, int CJ3>
cudaError_t set_wave_end_attr(Ctx *, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_fast_wave_end<CJ1, CJ2, CJ3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_fast_wave_end<CJ1, CJ2, CJ3>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t launch_wave_end_k(Ctx *c, const DenseArgs &A, RowArgs R, int mode, size_t smem) {
    const int rpc = rows_per_cta<CJ1, CJ2>();
    R.nb1 = ceil_div(c->d.I1, rpc);
    const int nb2 = ceil_div(c->d.I2, rpc);
    const unsigned grid = (unsigned)(1 + R.nb1 + nb2);
    k_fast_wave_end<CJ1, CJ2, CJ3><<<grid, 256, smem, c->stream>>>(A, R, mode);
    return cudaGetLastError();
}

// the sweep's shared memory, or the dense pre-work's if larger (one CTA of the launch runs it)
template <int CJ1, int CJ2, int CJ3>
size_t sweep_smem(const Ctx *c) {
    const int J1P = even_up(c->d.J1), J2P = even_up(c->d.J2);
    const size_t Q = (size_t)c->d.J1 * c->d.J2;
    const size_t sweep = runs_path<CJ1, CJ2>()
                             ? (size_t)align4(c->PI) +
                                   std::max(align4((int)Q) + (size_t)(kFastThreads / 32) * Q,
                                            (size_t)c->d.I3 * Q <= (size_t)kGcAll ? 2 * (size_t)c->d.I3 * Q : 0)
                             : (size_t)align4(c->PI) + align4(c->d.J1 * c->d.J2) + (size_t)kFastThreads * (J1P + J2P + 4);
    return sizeof(float) * std::max<size_t>(sweep, (size_t)dense_pre_floats(c->d));
}

// Which sweep kernel a context runs: 1 the lane-group kernel (FP32 gathers), 2 the lane-group
// kernel gathering gene rows from the BF16 copy, 0 k_fast_sweep (the warp-per-unit kernel for
// compile-time ranks up to 16, the per-entry kernel otherwise), -1 the tensor-core kernel.
// The lane-group kernel needs compile-time J1, J2 <= 16, every platform's Gc in shared memory
// and the set-up table of per-wave row counts.  SNECT_SWEEP_KERNEL=warp in the environment
// selects k_fast_sweep where the lane-group kernel would run (both are complete sweeps; the
// switch exists to compare them).
int row_stride(int J, int I3);

template <int CJ1, int CJ2, int CJ3>
int pick_sweep(const Ctx *c) {
    const int prec = c->cfg.precision;
    bool lg = false;
    if constexpr (runs_path<CJ1, CJ2>())
        lg = c->wcnt && (int64_t)c->d.I3 * CJ1 * CJ2 <= kGcAll &&
             (int64_t)c->d.I2 * row_stride(CJ2, c->d.I3) < INT32_MAX &&
             (int64_t)c->d.I1 * row_stride(CJ1, c->d.I3) < INT32_MAX;  // 32-bit offsets in the sweep
    if (prec == SNECT_BF16_TC) return -1;
    if (prec == SNECT_BF16) return (lg && CJ2 % 4 == 0) ? 2 : -1;
    const char *env = getenv("SNECT_SWEEP_KERNEL");
    if (env && strcmp(env, "warp") == 0) return 0;
    return lg ? 1 : 0;
}

// the sweep kernel of a context (sweep_kind >= 0)
template <int CJ1, int CJ2, int CJ3>
void (*sweep_kernel(const Ctx *c))(FastArgs) {
    if constexpr (runs_path<CJ1, CJ2>()) {
        if (c->sweep_kind == 1) return k_fast_sweep_lg<CJ1, CJ2, CJ3, 0>;
        if constexpr (CJ2 % 4 == 0)
            if (c->sweep_kind == 2) return k_fast_sweep_lg<CJ1, CJ2, CJ3, 1>;
    }
    return c->wcnt ? k_fast_sweep<CJ1, CJ2, CJ3, false> : k_fast_sweep<CJ1, CJ2, CJ3, true>;
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t init_sweep(Ctx *c) {
    const size_t smem = sweep_smem<CJ1, CJ2, CJ3>(c);
    c->sweep_kind = pick_sweep<CJ1, CJ2, CJ3>(c);
    auto kern = sweep_kernel<CJ1, CJ2, CJ3>(c);
    cudaError_t e = cudaFuncSetAttribute(kern,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFastThreads, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return e;
    c->fast_grid = std::max(1, per_sm) * sms;
    return cudaSuccess;
}

int row_stride(int J, int I3) { return ((J + 3) & ~3) + ((I3 + 3) & ~3); }

size_t sweep_tc_smem(const Ctx *c) {
    return std::max<size_t>(tc_smem_bytes(c->d.J1, c->d.J2, (int)c->PI), sizeof(float) * dense_pre_floats(c->d));
}

template <int CJ1, int CJ2>
cudaError_t init_sweep_tc(Ctx *c) {
    const size_t smem = sweep_tc_smem(c);
    cudaError_t e = cudaFuncSetAttribute(k_fast_sweep_tc<CJ1, CJ2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    // the largest shared-memory carveout, so that the occupancy query (and the launch) see
    // room for several CTAs of ~50 KB each
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fast_sweep_tc<CJ1, CJ2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fast_sweep_tc<CJ1, CJ2>, 128, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return e;
    // The occupancy query has answered 1 CTA per SM for this kernel where registers and shared
    // memory admit 4 (the profiler's limits); so the CTAs per SM are also counted from the
    // kernel's own registers and shared memory, and the larger count is taken.
    cudaFuncAttributes fa;
    int regs_sm = 0, smem_sm = 0, reserved = 0;
    e = cudaFuncGetAttributes(&fa, k_fast_sweep_tc<CJ1, CJ2>);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, c->device);
    if (e != cudaSuccess) return e;
    const int regs_cta = ((fa.numRegs + 7) & ~7) * 128;
    const int by_regs = regs_cta > 0 ? regs_sm / regs_cta : 1;
    const int by_smem = smem_sm / (int)(fa.sharedSizeBytes + smem + (size_t)reserved);
    per_sm = std::max(per_sm, std::min(by_regs, by_smem));
    // TMEM: 512 columns per SM shared by the resident CTAs
    c->fast_grid = std::max(1, std::min(per_sm, 512 / tc_tmem_cols<CJ1, CJ2>())) * sms;
    return cudaSuccess;
}

#define SNECT_DISPATCH_TC(J1, J2, FN, ...)                                  \
    (((J1) == 16 && (J2) == 16)   ? FN<16, 16>(__VA_ARGS__)                 \
     : ((J1) == 16 && (J2) == 32) ? FN<16, 32>(__VA_ARGS__)                 \
     : ((J1) == 32 && (J2) == 16) ? FN<32, 16>(__VA_ARGS__)                 \
                                  : FN<32, 32>(__VA_ARGS__))

template <int CJ1, int CJ2>
cudaError_t launch_sweep_tc(Ctx *c, const FastArgs &A, int grid) {
    k_fast_sweep_tc<CJ1, CJ2><<<grid, 128, sweep_tc_smem(c), c->stream>>>(A);
    return cudaGetLastError();
}

void make_wave_args(Ctx *c, int64_t w, int parity, int mode, DenseArgs *Ap, RowArgs *Rp);

FastArgs make_fast_args(Ctx *c, int64_t w) {
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
    A.macc = c->macc;
    A.gA = c->gacc[0];
    A.gB = c->gacc[1];
    A.rs1 = row_stride(c->d.J1, c->d.I3);
    A.rs2 = row_stride(c->d.J2, c->d.I3);
    A.err = c->flag + 3;
    A.count_atomics = c->wcnt ? 0 : 1;
    A.e_first = w * c->wave;
    A.e_count = c->wave_len[w];
    A.U2h = c->U2h;
    RowArgs unused;
    make_wave_args(c, w, (int)(w & 1), 0, &A.pre, &unused);
    return A;
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t run_sweep(Ctx *c, int64_t w) {
    const FastArgs A = make_fast_args(c, w);
    const int64_t nt = A.n_tiles;
    // CTAs 0-2 take the wave's dense pre-work (CTA 0 alone in the tensor-core form), the
    // others the tiles (one resident wave of CTAs)
    const bool tc = c->sweep_kind < 0;
    const int pre = tc ? 1 : kPreCtas;
    const int grid = (int)std::min<int64_t>(std::max(1, c->fast_grid - pre), nt) + pre;
    c->launches++;
    if (tc) return SNECT_DISPATCH_TC(c->d.J1, c->d.J2, launch_sweep_tc, c, A, grid);
    auto kern = sweep_kernel<CJ1, CJ2, CJ3>(c);
    kern<<<grid, kFastThreads, sweep_smem<CJ1, CJ2, CJ3>(c), c->stream>>>(A);
    return cudaGetLastError();
}

size_t wave_end_smem(const Ctx *c) {
    const Dims &d = c->d;
    const size_t dense = (size_t)dense_post_floats(d);
    const size_t rows = std::max<size_t>(kRowWarps * ((size_t)kMaxRank * kTileStride + 2 * kMaxRank) +
                                             kRowWarps * (size_t)kMaxRank * kMaxRank + kCkStage,
                                         (size_t)std::max(rows_thread_floats(d.J1), rows_thread_floats(d.J2)));
    return sizeof(float) * std::max(dense, rows);
}

int64_t curv_stride(const Ctx *c) {
    return ((int64_t)c->d.I3 * (c->d.J1 * c->d.J1 + c->d.J2 * c->d.J2) + 3) & ~(int64_t)3;
}

void make_wave_args(Ctx *c, int64_t w, int parity, int mode, DenseArgs *Ap, RowArgs *Rp) {
    const Dims &d = c->d;
    DenseArgs &A = *Ap;
    RowArgs &R = *Rp;
    A.d = d;
    A.G = c->G;
    A.U3 = c->U[2];
    A.cnt3 = c->cnt[2];
    A.macc = c->macc;
    A.gram_in = c->gram + (size_t)(parity ^ 1) * c->gram_stride;
    A.eigv = c->gram + 2 * (size_t)c->gram_stride;
    A.eigval = A.eigv + d.J1 * d.J1 + d.J2 * d.J2 + d.J3 * d.J3;
    A.ainv = A.eigval + d.J1 + d.J2 + d.J3;
    A.wave_counter = c->flag + 2;
    A.curv = c->curv;
    A.nk = c->wave_nk + (w >= 0 ? w : 0) * d.I3;
    A.n_wave = w >= 0 ? (float)c->wave_len[w] : 0.f;
    A.lam = c->cfg.lambda;
    A.lr = c->cfg.lr;
    A.lam_core = c->nnz ? c->cfg.lambda / (float)c->nnz : 0.f;
    R.U1 = c->U[0];
    R.U2 = c->U[1];
    R.gA = c->gacc[0];
    R.gB = c->gacc[1];
    R.rs1 = row_stride(d.J1, d.I3);
    R.rs2 = row_stride(d.J2, d.I3);
    R.cnt1 = c->cnt[0];
    R.cnt2 = c->cnt[1];
    R.inv_n = c->nnz ? 1.f / (float)c->nnz : 0.f;
    R.nb1 = 0;  // set by the launcher for its row step
    R.curv_in = c->curv;
    R.gram_out = c->gram + (size_t)parity * c->gram_stride;
    R.wc1 = R.wc2 = nullptr;
    R.U2h = c->U2h;
    if (c->wcnt && w >= 0) {
        R.wc1 = c->wcnt + (size_t)w * ((size_t)d.I1 + d.I2) * d.I3;
        R.wc2 = R.wc1 + (size_t)d.I1 * d.I3;
    }
    (void)mode;
}

cudaError_t launch_wave_end(Ctx *c, int64_t w, int parity, int mode) {
    DenseArgs A;
    RowArgs R;
    make_wave_args(c, w, parity, mode, &A, &R);
    c->launches++;
    return SNECT_DISPATCH_ROWS(c->d.J1, c->d.J2, c->d.J3, launch_wave_end_k, c, A, R, mode, wave_end_smem(c));
}

__global__ void k_rows_to_bf16(const float *__restrict__ U, int64_t n, __nv_bfloat16 *__restrict__ Uh) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) Uh[t] = __float2bfloat16(U[t]);
}

}  // namespace

cudaError_t refresh_bf16_rows(Ctx *c) {
    if (!c->U2h) return cudaSuccess;
    const int64_t n = (int64_t)c->d.I2 * c->d.J2;
    k_rows_to_bf16<<<ceil_div(n, 256), 256, 0, c->stream>>>(c->U[1], n, c->U2h);
    c->launches++;
    return cudaGetLastError();
}

int init_fast(Ctx *c) {
    const Dims &d = c->d;
    SNECT_CUDA(c, scratch_alloc(c, &c->tile_ctr, sizeof(int32_t) * std::max<int64_t>(1, c->n_waves)));
    SNECT_CUDA(c, scratch_alloc(c, &c->macc, sizeof(float) * d.I3 * d.J1 * d.J2));
    SNECT_CUDA(c, cudaMemsetAsync(c->macc, 0, sizeof(float) * d.I3 * d.J1 * d.J2, c->stream));
    // moments: two buffers (this wave's, the previous wave's) + warm-start eigenvectors
    c->gram_stride = ((int64_t)d.J1 * d.J1 + d.J2 * d.J2 + 3) & ~3;
    // + eigenvectors and eigenvalues of Ma, Mb, Cn + the platform systems' inverses
    const int64_t gf = 2 * c->gram_stride + d.J1 * d.J1 + d.J2 * d.J2 + d.J3 * d.J3 + d.J1 + d.J2 + d.J3 +
                       (int64_t)d.I3 * d.J3 * d.J3;
    c->gram_floats = gf;
    SNECT_CUDA(c, scratch_alloc(c, &c->gram, sizeof(float) * gf));
    SNECT_CUDA(c, cudaMemsetAsync(c->gram, 0, sizeof(float) * gf, c->stream));
    // platform curvatures for the row steps (formed by each wave's pre-work)
    SNECT_CUDA(c, scratch_alloc(c, &c->curv, sizeof(float) * curv_stride(c)));
    SNECT_CUDA(c, cudaMemsetAsync(c->curv, 0, sizeof(float) * curv_stride(c), c->stream));
    for (int n = 0; n < 2; ++n) {
        const int64_t nf = (int64_t)(n ? d.I2 : d.I1) * row_stride(n ? d.J2 : d.J1, d.I3);
        SNECT_CUDA(c, scratch_alloc(c, &c->gacc[n], sizeof(float) * nf));
        SNECT_CUDA(c, cudaMemsetAsync(c->gacc[n], 0, sizeof(float) * nf, c->stream));
    }
    SNECT_CUDA(c, SNECT_DISPATCH_RANKS(d.J1, d.J2, d.J3, init_sweep, c));
    if (c->sweep_kind < 0) SNECT_CUDA(c, SNECT_DISPATCH_TC(d.J1, d.J2, init_sweep_tc, c));
    if (c->sweep_kind == 2) {
        SNECT_CUDA(c, scratch_alloc(c, &c->U2h, sizeof(__nv_bfloat16) * (size_t)d.I2 * d.J2));
        SNECT_CUDA(c, refresh_bf16_rows(c));
    }
    SNECT_CUDA(c, cudaMemsetAsync(c->flag + 2, 0, 2 * sizeof(int32_t), c->stream));
    SNECT_CUDA(c, SNECT_DISPATCH_ROWS(d.J1, d.J2, d.J3, set_wave_end_attr, c, wave_end_smem(c)));
    // the first wave's moments: those of the initial rows, into the odd buffer (the first
    // wave's pre-work forms its curvatures and eigenbases from them)
    SNECT_CUDA(c, launch_wave_end(c, -1, 1, 1));
    return timing_events(c, c->n_waves);
}

int enqueue_fast_epoch(Ctx *c) {
    if (c->n_waves == 0) return SNECT_OK;
    const Dims &d = c->d;
    SNECT_CUDA(c, cudaMemsetAsync(c->tile_ctr, 0, sizeof(int32_t) * c->n_waves, c->stream));
    // n_waves is even, so wave w's parity (w % 2) continues across epochs
    for (int64_t w = 0; w < c->n_waves; ++w) {
        const bool tm = c->time_launch(w, c->n_waves, c->wave_len[w]);
        if (tm) SNECT_CUDA(c, cudaEventRecordWithFlags(c->ev_begin[w], c->stream, cudaEventRecordExternal));
        SNECT_CUDA(c, SNECT_DISPATCH_RANKS(d.J1, d.J2, d.J3, run_sweep, c, w));
        if (tm) SNECT_CUDA(c, cudaEventRecordWithFlags(c->ev_end[w], c->stream, cudaEventRecordExternal));
        int rc = aux_event(c, 1, false);
        if (rc) return rc;
        SNECT_CUDA(c, launch_wave_end(c, w, (int)(w & 1), 0));
        if ((rc = aux_event(c, 1, true))) return rc;
    }
    return SNECT_OK;
}

int fast_wave_grads(Ctx *c, int64_t w, float *gA, float *gB, float *M, float *nA, float *nB) {
    const Dims &d = c->d;
    if (w < 0 || w >= c->n_waves) return fail(c, SNECT_EINVAL, "wave index outside [0, n_waves)");
    const size_t rs1 = (size_t)row_stride(d.J1, d.I3), rs2 = (size_t)row_stride(d.J2, d.I3);
    const size_t na = (size_t)d.I1 * rs1, nb = (size_t)d.I2 * rs2, nm = (size_t)d.I3 * d.J1 * d.J2;
    auto clear = [&]() -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(c->gacc[0], 0, sizeof(float) * na, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->gacc[1], 0, sizeof(float) * nb, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->macc, 0, sizeof(float) * nm, c->stream);
        return e;
    };
    SNECT_CUDA(c, clear());
    SNECT_CUDA(c, cudaMemsetAsync(c->tile_ctr + w, 0, sizeof(int32_t), c->stream));
    SNECT_CUDA(c, cudaMemsetAsync(c->flag + 3, 0, sizeof(int32_t), c->stream));
    SNECT_CUDA(c, SNECT_DISPATCH_RANKS(d.J1, d.J2, d.J3, run_sweep, c, w));
    const int JA = (d.J1 + 3) & ~3, JB = (d.J2 + 3) & ~3;
    const cudaMemcpyKind kd = cudaMemcpyDefault;
    if (gA)
        SNECT_CUDA(c, cudaMemcpy2DAsync(gA, sizeof(float) * d.J1, c->gacc[0], sizeof(float) * rs1,
                                        sizeof(float) * d.J1, d.I1, kd, c->stream));
    if (gB)
        SNECT_CUDA(c, cudaMemcpy2DAsync(gB, sizeof(float) * d.J2, c->gacc[1], sizeof(float) * rs2,
                                        sizeof(float) * d.J2, d.I2, kd, c->stream));
    if (M) SNECT_CUDA(c, cudaMemcpyAsync(M, c->macc, sizeof(float) * nm, kd, c->stream));
    if (c->wcnt) {  // the set-up table of the wave's entries per (row, platform)
        const float *t = c->wcnt + (size_t)w * ((size_t)d.I1 + d.I2) * d.I3;
        if (nA) SNECT_CUDA(c, cudaMemcpyAsync(nA, t, sizeof(float) * d.I1 * d.I3, kd, c->stream));
        if (nB)
            SNECT_CUDA(c, cudaMemcpyAsync(nB, t + (size_t)d.I1 * d.I3, sizeof(float) * (size_t)d.I2 * d.I3, kd,
                                          c->stream));
    } else {  // counted by the sweep's atomics, after each row's gradient
        if (nA)
            SNECT_CUDA(c, cudaMemcpy2DAsync(nA, sizeof(float) * d.I3, c->gacc[0] + JA, sizeof(float) * rs1,
                                            sizeof(float) * d.I3, d.I1, kd, c->stream));
        if (nB)
            SNECT_CUDA(c, cudaMemcpy2DAsync(nB, sizeof(float) * d.I3, c->gacc[1] + JB, sizeof(float) * rs2,
                                            sizeof(float) * d.I3, d.I2, kd, c->stream));
    }
    int32_t tc_err = 0;
    SNECT_CUDA(c, cudaMemcpyAsync(&tc_err, c->flag + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    SNECT_CUDA(c, clear());
    SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (tc_err) return fail(c, SNECT_ETIMEDOUT, "a completion wait timed out in the sweep");
    return SNECT_OK;
}

void free_fast(Ctx *c) {
    auto f = [c](auto *&p) {
        if (p) cudaFreeAsync(p, c->stream);
        p = nullptr;
    };
    f(c->tile_start);
    f(c->tile_len);
    f(c->tile_k);
    f(c->tile_ctr);
    f(c->wave_nk);
    f(c->macc);
    f(c->gram);
    f(c->curv);
    f(c->gacc[0]);
    f(c->gacc[1]);
    f(c->wcnt);
    f(c->U2h);
}

}  // namespace snect

// ---------------------------------------------------------------------------------------
// Batched form: many independent decompositions stepped together.  Every wave runs one
// sweep launch over the tiles of all problems and one wave-end launch over all problems'
// dense and row steps; an epoch of the whole batch is one CUDA graph.

namespace snect {

struct Batch {
    std::vector<Ctx *> ctx;
    int32_t P = 0;
    int64_t n_waves = 0;
    Dims d{};
    FastArgs *d_fast = nullptr;   // [n_waves][P]
    int32_t *d_toff = nullptr;    // [n_waves][P + 1] tile offsets
    DenseArgs *d_dense = nullptr; // [n_waves][P]
    RowArgs *d_rows = nullptr;    // [n_waves][P]
    int32_t *d_boff = nullptr;    // [P + 1] CTA offsets of the wave end
    int32_t *d_ctr = nullptr;     // [n_waves]
    EdgeArgs *d_edge = nullptr;   // [P] network passes
    int64_t edge_cells = 0, edge_heavy = 0;  // largest I2 * J2 and hub count over the problems
    std::vector<int32_t> tiles_per_wave;
    int32_t wave_end_blocks = 0;
    int64_t epoch_kernels = 0;  // kernels in one epoch's graph
    int64_t launches = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string err;
    // the lane-group batch sweep (contexts of sweep kind 1 or 2): per wave, the tile CTAs'
    // problem and rank and each problem's CTA count, from the autotuned allotment
    int32_t kind = 0;
    std::vector<int32_t> lg_tiles;        // per wave: tile CTAs
    std::vector<int64_t> lg_off;          // per wave: offset of its (prob, rank) arrays in d_cta
    int32_t *d_cta = nullptr;
    int32_t *d_prob_ctas = nullptr;       // [n_waves][P]
    int32_t tune_cps = 0;                 // autotuned: tile CTAs per SM
    int32_t tune_over = 0;                // autotuned: tile CTAs per resident CTA slot
    int32_t tune_min_entries = 0;         // autotuned: fewest entries a warp is given
    double tune_ms = 0.0;                 // the chosen configuration's sweep time on wave 0
    void *d_bf = nullptr;                 // BF16 copies to refresh after the network passes
    int64_t bf_max = 0;
};

namespace {

struct BfRows {
    const float *U2;
    __nv_bfloat16 *U2h;
    int64_t n;
};

__global__ void k_batch_rows_to_bf16(const BfRows *__restrict__ a) {
    const BfRows r = a[blockIdx.y];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < r.n; t += (int64_t)gridDim.x * blockDim.x)
        r.U2h[t] = __float2bfloat16(r.U2[t]);
}

// the lane-group sweep's allotment of tile CTAs to the problems of wave w: about `tiles` CTAs
// in proportion to each problem's entries (at least one CTA for a problem with entries), and
// no more than one warp per min_e entries when min_e > 0
void lg_allot(const Batch *b, int64_t w, int tiles, int64_t min_e, std::vector<int32_t> &prob,
              std::vector<int32_t> &rank, std::vector<int32_t> &pc) {
    const int P = b->P;
    int64_t N = 0;
    for (int p = 0; p < P; ++p) N += b->ctx[p]->wave_len[w];
    prob.clear();
    rank.clear();
    pc.assign((size_t)P, 0);
    for (int p = 0; p < P; ++p) {
        const int64_t n = b->ctx[p]->wave_len[w];
        if (n <= 0) continue;
        int64_t c = std::max<int64_t>(1, (int64_t)tiles * n / std::max<int64_t>(N, 1));
        if (min_e > 0) c = std::min<int64_t>(c, std::max<int64_t>(1, (n + 8 * min_e - 1) / (8 * min_e)));
        pc[p] = (int32_t)c;
        for (int64_t r = 0; r < c; ++r) {
            prob.push_back(p);
            rank.push_back((int32_t)r);
        }
    }
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t batch_lg_launch(Batch *b, const FastArgs *d_fast_w, const int32_t *d_prob, const int32_t *d_rank,
                            const int32_t *d_pc, int tiles, cudaStream_t st) {
    if constexpr (runs_path<CJ1, CJ2>()) {
        const size_t smem = sweep_smem<CJ1, CJ2, CJ3>(b->ctx[0]);
        if (b->kind == 2) {
            if constexpr (CJ2 % 4 == 0) {
                k_batch_sweep_lg<CJ1, CJ2, CJ3, 1><<<b->P + tiles, kFastThreads, smem, st>>>(d_fast_w, d_prob, d_rank,
                                                                                          d_pc, b->P);
                return cudaGetLastError();
            }
            return cudaErrorInvalidValue;
        }
        k_batch_sweep_lg<CJ1, CJ2, CJ3, 0><<<b->P + tiles, kFastThreads, smem, st>>>(d_fast_w, d_prob, d_rank, d_pc,
                                                                                  b->P);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t batch_lg_attr(Batch *b, int *per_sm) {
    *per_sm = 1;
    if constexpr (runs_path<CJ1, CJ2>()) {
        const size_t smem = sweep_smem<CJ1, CJ2, CJ3>(b->ctx[0]);
        auto set = [&](auto kern) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, kFastThreads, smem);
            return e;
        };
        if (b->kind == 2) {
            if constexpr (CJ2 % 4 == 0) return set(k_batch_sweep_lg<CJ1, CJ2, CJ3, 1>);
            return cudaErrorInvalidValue;
        }
        return set(k_batch_sweep_lg<CJ1, CJ2, CJ3, 0>);
    }
    return cudaErrorInvalidValue;
}

// every problem's wave accumulators back to zero (after an autotuning launch)
cudaError_t batch_clear_acc(Batch *b, cudaStream_t st) {
    for (Ctx *c : b->ctx) {
        const Dims &d = c->d;
        cudaError_t e = cudaMemsetAsync(c->gacc[0], 0, sizeof(float) * d.I1 * row_stride(d.J1, d.I3), st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c->gacc[1], 0, sizeof(float) * (size_t)d.I2 * row_stride(d.J2, d.I3), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->macc, 0, sizeof(float) * d.I3 * d.J1 * d.J2, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Autotuner of the lane-group batch sweep: every candidate (resident tile CTAs per SM, tile
// CTAs per resident slot, fewest entries per warp) sweeps wave 0 at the current parameters,
// timed with CUDA events (best of two after a warm-up launch); its accumulations are cleared
// again.  Then the per-wave allotment tables of the fastest candidate are built and uploaded.
// More tile CTAs than resident slots make each CTA's share smaller; the CTAs are dispatched in
// index order, which follows the problems, so fewer problems' factors and accumulators are in
// use at once (the batch's rows and accumulators together outgrow the L2).
cudaError_t batch_lg_tune(Batch *b, cudaStream_t st) {
    const Dims &d = b->d;
    int per_sm = 1, sms = 1;
    cudaError_t e = SNECT_DISPATCH_RANKS(d.J1, d.J2, d.J3, batch_lg_attr, b, &per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->ctx[0]->device);
    if (e != cudaSuccess) return e;
    // the trial sweeps' dense pre-work rewrites each problem's curvature state (moments,
    // eigenbases, platform systems): saved here and put back afterwards
    std::vector<float *> saved(b->P, nullptr);
    for (int p = 0; p < b->P && e == cudaSuccess; ++p) {
        Ctx *c = b->ctx[p];
        const size_t nf = (size_t)c->gram_floats + curv_stride(c);
        e = cudaMalloc((void **)&saved[p], sizeof(float) * nf);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(saved[p], c->gram, sizeof(float) * c->gram_floats, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(saved[p] + c->gram_floats, c->curv, sizeof(float) * curv_stride(c),
                                cudaMemcpyDeviceToDevice, st);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    std::vector<int32_t> prob, rank, pc;
    double best = 1e30;
    for (int cps = 2; cps <= std::max(2, per_sm) && e == cudaSuccess; ++cps)
      for (int over : {1, 4})
        for (int64_t me : {(int64_t)0, (int64_t)2048}) {
            if (e != cudaSuccess) break;
            const int tiles = std::max(over * cps * sms - b->P, b->P);
            lg_allot(b, 0, tiles, me, prob, rank, pc);
            const int T = (int)prob.size();
            std::vector<int32_t> h(prob);
            h.insert(h.end(), rank.begin(), rank.end());
            h.insert(h.end(), pc.begin(), pc.end());
            int32_t *dt = nullptr;
            e = cudaMalloc((void **)&dt, sizeof(int32_t) * h.size());
            if (e == cudaSuccess) e = cudaMemcpy(dt, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice);
            float ms_best = 1e30f;
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                e = cudaEventRecord(e0, st);
                if (e == cudaSuccess)
                    e = SNECT_DISPATCH_RANKS(d.J1, d.J2, d.J3, batch_lg_launch, b, b->d_fast, dt, dt + T, dt + 2 * T,
                                             T, st);
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = batch_clear_acc(b, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_best = std::min(ms_best, ms);
            }
            if (dt) cudaFree(dt);
            if (e == cudaSuccess && ms_best < best) {
                best = ms_best;
                b->tune_cps = cps;
                b->tune_over = over;
                b->tune_min_entries = (int32_t)me;
                b->tune_ms = ms_best;
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int p = 0; p < b->P; ++p) {
        Ctx *c = b->ctx[p];
        if (saved[p] && e == cudaSuccess) {
            e = cudaMemcpyAsync(c->gram, saved[p], sizeof(float) * c->gram_floats, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->curv, saved[p] + c->gram_floats, sizeof(float) * curv_stride(c),
                                    cudaMemcpyDeviceToDevice, st);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (float *q : saved)
        if (q) cudaFree(q);
    if (e != cudaSuccess) return e;
    // the chosen allotment for every wave
    const int tiles = std::max(b->tune_over * b->tune_cps * sms - b->P, b->P);
    std::vector<int32_t> all, allpc;
    b->lg_tiles.assign((size_t)b->n_waves, 0);
    b->lg_off.assign((size_t)b->n_waves, 0);
    for (int64_t w = 0; w < b->n_waves; ++w) {
        lg_allot(b, w, tiles, b->tune_min_entries, prob, rank, pc);
        b->lg_off[w] = (int64_t)all.size();
        b->lg_tiles[w] = (int32_t)prob.size();
        all.insert(all.end(), prob.begin(), prob.end());
        all.insert(all.end(), rank.begin(), rank.end());
        allpc.insert(allpc.end(), pc.begin(), pc.end());
    }
    e = cudaMalloc((void **)&b->d_cta, sizeof(int32_t) * std::max<size_t>(1, all.size()));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_cta, all.data(), sizeof(int32_t) * all.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_prob_ctas, sizeof(int32_t) * std::max<size_t>(1, allpc.size()));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_prob_ctas, allpc.data(), sizeof(int32_t) * allpc.size(), cudaMemcpyHostToDevice);
    return e;
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t batch_sweep_k(Batch *b, int64_t w, cudaStream_t st) {
    Ctx *c0 = b->ctx[0];
    const int nt = b->tiles_per_wave[w];
    // one CTA per problem for its dense pre-work, then the tile CTAs
    const int grid = std::min(std::max(1, c0->fast_grid - b->P), nt) + b->P;
    k_batch_sweep<CJ1, CJ2, CJ3><<<grid, kFastThreads, sweep_smem<CJ1, CJ2, CJ3>(c0), st>>>(
        b->d_fast + w * b->P, b->d_toff + w * (b->P + 1), b->P, b->d_ctr + w);
    return cudaGetLastError();
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t batch_wave_end_k(Batch *b, int64_t w, cudaStream_t st) {
    const size_t smem = wave_end_smem(b->ctx[0]);
    cudaError_t e = cudaFuncSetAttribute(k_batch_wave_end<CJ1, CJ2, CJ3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_wave_end<CJ1, CJ2, CJ3>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    k_batch_wave_end<CJ1, CJ2, CJ3><<<b->wave_end_blocks, 256, smem, st>>>(b->d_dense + w * b->P, b->d_rows + w * b->P,
                                                                     b->d_boff, b->P);
    return cudaGetLastError();
}

template <int CJ1, int CJ2, int CJ3>
cudaError_t batch_sweep_attr(Batch *b) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_sweep<CJ1, CJ2, CJ3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sweep_smem<CJ1, CJ2, CJ3>(b->ctx[0]));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_batch_sweep<CJ1, CJ2, CJ3>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

template <int CJ1, int CJ2, int CJ3>
int batch_rows_per_cta(Batch *) { return rows_per_cta<CJ1, CJ2>(); }

int batch_fail(Batch *b, int code, const std::string &m) {
    b->err = m;
    return code;
}

#define BATCH_CUDA(b, call)                                                                          \
    do {                                                                                             \
        cudaError_t e__ = (call);                                                                    \
        if (e__ != cudaSuccess) return batch_fail((b), SNECT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

int batch_build_graph(Batch *b) {
    const Dims &d = b->d;
    cudaStream_t cap = nullptr;
    BATCH_CUDA(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int rc = SNECT_OK;
    if (e == cudaSuccess) {
        e = cudaMemsetAsync(b->d_ctr, 0, sizeof(int32_t) * b->n_waves, cap);
        b->epoch_kernels = 0;
        for (int64_t w = 0; w < b->n_waves && e == cudaSuccess; ++w) {
            if (b->kind > 0) {
                const int T = b->lg_tiles[w];
                const int32_t *tab = b->d_cta + b->lg_off[w];
                e = SNECT_DISPATCH_RANKS(d.J1, d.J2, d.J3, batch_lg_launch, b, b->d_fast + w * b->P, tab, tab + T,
                                         b->d_prob_ctas + w * b->P, T, cap);
            } else {
                e = SNECT_DISPATCH_RANKS(d.J1, d.J2, d.J3, batch_sweep_k, b, w, cap);
            }
            if (e == cudaSuccess) e = SNECT_DISPATCH_ROWS(d.J1, d.J2, d.J3, batch_wave_end_k, b, w, cap);
            b->epoch_kernels += 2;
        }
        if (e == cudaSuccess)  // every problem's network pass
            e = launch_batch_edge_pass(b->d_edge, b->P, b->edge_cells, b->edge_heavy, cap, &b->epoch_kernels);
        if (e == cudaSuccess && b->d_bf) {  // the BF16 gene-row copies after the passes
            k_batch_rows_to_bf16<<<dim3((unsigned)std::min<int64_t>(ceil_div(b->bf_max, 256), 1024), b->P), 256, 0,
                                   cap>>>(static_cast<const BfRows *>(b->d_bf));
            e = cudaGetLastError();
            b->epoch_kernels += 1;
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        rc = batch_fail(b, SNECT_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    return rc;
}

void batch_free(Batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaFree(b->d_fast);
    cudaFree(b->d_toff);
    cudaFree(b->d_dense);
    cudaFree(b->d_rows);
    cudaFree(b->d_boff);
    cudaFree(b->d_ctr);
    cudaFree(b->d_edge);
    cudaFree(b->d_cta);
    cudaFree(b->d_prob_ctas);
    cudaFree(b->d_bf);
}

thread_local std::string g_batch_error;

}  // namespace
}  // namespace snect

using namespace snect;

extern "C" {

int snect_batch_create(snect_batch **out, snect_ctx *const *ctxs, int32_t n, void *stream) {
    if (!out || !ctxs || n < 1) return g_batch_error = "null argument or empty batch", SNECT_EINVAL;
    *out = nullptr;
    Batch *b = new Batch();
    b->P = n;
    b->stream = (cudaStream_t)stream;
    for (int32_t p = 0; p < n; ++p) b->ctx.push_back(reinterpret_cast<Ctx *>(ctxs[p]));
    Ctx *c0 = b->ctx[0];
    auto bad = [&](const std::string &m) {
        g_batch_error = m;
        batch_free(b);
        delete b;
        return SNECT_EINVAL;
    };
    for (Ctx *c : b->ctx) {
        if (!c) return bad("null context");
        if (c->cfg.batch != 0 || c->sweep_kind < 0)
            return bad("a batch takes fast-mode contexts whose sweep runs on the FP32 cores "
                       "(SNECT_FP32, or SNECT_BF16 at 16 x 16 x 5)");
        if (c->sweep_kind != c0->sweep_kind)
            return bad("every problem of a batch must run the same sweep kernel (precision and ranks)");
        if (c->d.J1 != c0->d.J1 || c->d.J2 != c0->d.J2 || c->d.J3 != c0->d.J3)
            return bad("every problem of a batch must have the same core ranks");
        if (c->n_waves != c0->n_waves) return bad("every problem of a batch must have the same number of waves");
        if (c->device != c0->device) return bad("every problem of a batch must live on the same device");
    }
    b->d = c0->d;
    b->n_waves = c0->n_waves;
    b->kind = c0->sweep_kind;

    const int64_t W = b->n_waves, P = n;
    std::vector<FastArgs> hf((size_t)(W * P));
    std::vector<DenseArgs> hd((size_t)(W * P));
    std::vector<RowArgs> hr((size_t)(W * P));
    std::vector<int32_t> toff((size_t)(W * (P + 1))), boff((size_t)P + 1);
    const int rpc = SNECT_DISPATCH_ROWS(b->d.J1, b->d.J2, b->d.J3, batch_rows_per_cta, b);
    boff[0] = 0;
    for (int64_t p = 0; p < P; ++p) {
        Ctx *c = b->ctx[p];
        boff[p + 1] = boff[p] + 1 + ceil_div(c->d.I1, rpc) + ceil_div(c->d.I2, rpc);
    }
    b->wave_end_blocks = boff[P];
    b->tiles_per_wave.assign((size_t)W, 0);
    for (int64_t w = 0; w < W; ++w) {
        int32_t acc = 0;
        for (int64_t p = 0; p < P; ++p) {
            Ctx *c = b->ctx[p];
            hf[w * P + p] = make_fast_args(c, w);
            make_wave_args(c, w, (int)(w & 1), 0, &hd[w * P + p], &hr[w * P + p]);
            hr[w * P + p].nb1 = ceil_div(c->d.I1, rpc);
            toff[w * (P + 1) + p] = acc;
            acc += hf[w * P + p].n_tiles;
        }
        toff[w * (P + 1) + P] = acc;
        b->tiles_per_wave[w] = acc;
    }
    cudaError_t e = cudaSuccess;
    auto up = [&](void **dst, const void *src, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(dst, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up((void **)&b->d_fast, hf.data(), sizeof(FastArgs) * hf.size());
    up((void **)&b->d_dense, hd.data(), sizeof(DenseArgs) * hd.size());
    up((void **)&b->d_rows, hr.data(), sizeof(RowArgs) * hr.size());
    up((void **)&b->d_toff, toff.data(), sizeof(int32_t) * toff.size());
    up((void **)&b->d_boff, boff.data(), sizeof(int32_t) * boff.size());
    std::vector<EdgeArgs> he;
    for (Ctx *c : b->ctx) {
        he.push_back(make_edge_args(c));
        b->edge_cells = std::max<int64_t>(b->edge_cells, (int64_t)he.back().I2 * he.back().J2);
        b->edge_heavy = std::max<int64_t>(b->edge_heavy, he.back().n_heavy);
    }
    up((void **)&b->d_edge, he.data(), sizeof(EdgeArgs) * he.size());
    if (b->kind == 2) {
        std::vector<BfRows> hb;
        for (Ctx *c : b->ctx) {
            hb.push_back(BfRows{c->U[1], c->U2h, (int64_t)c->d.I2 * c->d.J2});
            b->bf_max = std::max<int64_t>(b->bf_max, hb.back().n);
        }
        up((void **)&b->d_bf, hb.data(), sizeof(BfRows) * hb.size());
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_ctr, sizeof(int32_t) * std::max<int64_t>(1, W));
    if (e == cudaSuccess) e = SNECT_DISPATCH_RANKS(b->d.J1, b->d.J2, b->d.J3, batch_sweep_attr, b);
    if (e != cudaSuccess) {
        g_batch_error = std::string("batch set-up: ") + cudaGetErrorString(e);
        batch_free(b);
        delete b;
        return SNECT_ECUDA;
    }
    *out = reinterpret_cast<snect_batch *>(b);
    return SNECT_OK;
}

int snect_batch_epoch(snect_batch *h, int32_t n_epochs) {
    Batch *b = reinterpret_cast<Batch *>(h);
    if (!b || n_epochs < 0) return SNECT_EINVAL;
    if (!b->exec) {
        // the contexts' own set-up work must be finished before the batch graph runs
        for (Ctx *c : b->ctx)
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) return batch_fail(b, SNECT_ECUDA, "context stream");
        if (b->kind > 0 && !b->d_cta) BATCH_CUDA(b, batch_lg_tune(b, b->stream));
        int rc = batch_build_graph(b);
        if (rc) return rc;
    }
    for (int32_t t = 0; t < n_epochs; ++t) {
        BATCH_CUDA(b, cudaGraphLaunch(b->exec, b->stream));
        b->launches += b->epoch_kernels;
    }
    for (Ctx *c : b->ctx) c->param_version++;
    return SNECT_OK;
}

int snect_batch_tuning(const snect_batch *h, int32_t *ctas_per_sm, int32_t *oversubscription,
                       int32_t *min_entries_per_warp, double *sweep_ms) {
    const Batch *b = reinterpret_cast<const Batch *>(h);
    if (!b) return SNECT_EINVAL;
    if (ctas_per_sm) *ctas_per_sm = b->tune_cps;
    if (oversubscription) *oversubscription = b->tune_over;
    if (min_entries_per_warp) *min_entries_per_warp = b->tune_min_entries;
    if (sweep_ms) *sweep_ms = b->tune_ms;
    return SNECT_OK;
}

int64_t snect_batch_launch_count(const snect_batch *h) {
    const Batch *b = reinterpret_cast<const Batch *>(h);
    return b ? b->launches : 0;
}

const char *snect_batch_last_error(const snect_batch *h) {
    const Batch *b = reinterpret_cast<const Batch *>(h);
    return b ? b->err.c_str() : g_batch_error.c_str();
}

void snect_batch_destroy(snect_batch *h) {
    Batch *b = reinterpret_cast<Batch *>(h);
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
}

}  // extern "C"
