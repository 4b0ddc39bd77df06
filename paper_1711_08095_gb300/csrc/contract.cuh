// Per-entry Tucker contraction shared by the sweep and objective kernels.
//
// For one observed entry (i, j, k) with factor rows a = u^(1)_i, b = u^(2)_j, c = u^(3)_k:
//   x~   = G x1 a x2 b x3 c                         (Eq. 2 entrywise; Alg. 1 lines 5-6)
//   v    = G x2 b x3 c      (length J1)             (gradient equation, mode 1)
//   w2   = G x1 a x3 c      (length J2)             (mode 2)
//   w3   = G x1 a x2 b      (length J3)             (mode 3)
// One pass over G: for every (p, q), t = sum_r g_pqr c_r feeds v_p (t * b_q) and w2_q
// (a_p * t), and a_p b_q feeds w3.  2*J1*J2*J3 + 2*J1*J2 multiply-adds.
//
// CJ* are compile-time ranks (0 = use the runtime value, arrays sized for kMaxRank).
#pragma once

#include "common.cuh"

namespace snect {

template <int CJ>
struct RankCap {
    static constexpr int value = CJ ? CJ : kMaxRank;
};

template <int CJ1, int CJ2, int CJ3>
__device__ __forceinline__ float contract_entry(const float *__restrict__ G, int J1r, int J2r, int J3r,
                                                const float *a, const float *b, const float *c,
                                                float *v, float *w2, float *w3) {
    // With compile-time ranks every loop below has a constant trip count and unrolls fully;
    // with runtime ranks (CJ* == 0) the loops stay loops.
    const int J1 = CJ1 ? CJ1 : J1r;
    const int J2 = CJ2 ? CJ2 : J2r;
    const int J3 = CJ3 ? CJ3 : J3r;
#pragma unroll
    for (int q = 0; q < J2; ++q) w2[q] = 0.f;
#pragma unroll
    for (int r = 0; r < J3; ++r) w3[r] = 0.f;
#pragma unroll
    for (int p = 0; p < J1; ++p) {
        float vp = 0.f;
#pragma unroll
        for (int q = 0; q < J2; ++q) {
            const float *g = G + (p * J2 + q) * J3;
            float t = 0.f;
            const float ab = a[p] * b[q];
#pragma unroll
            for (int r = 0; r < J3; ++r) {
                t = fmaf(g[r], c[r], t);
                w3[r] = fmaf(ab, g[r], w3[r]);
            }
            vp = fmaf(t, b[q], vp);
            w2[q] = fmaf(a[p], t, w2[q]);
        }
        v[p] = vp;
    }
    float xt = 0.f;
#pragma unroll
    for (int p = 0; p < J1; ++p) xt = fmaf(a[p], v[p], xt);
    return xt;
}

// x~ alone (Eq. 2 entrywise): sum_p a_p sum_q b_q sum_r g_pqr c_r.
template <int CJ1, int CJ2, int CJ3>
__device__ __forceinline__ float predict_entry(const float *__restrict__ G, int J1r, int J2r, int J3r,
                                               const float *a, const float *b, const float *c) {
    const int J1 = CJ1 ? CJ1 : J1r;
    const int J2 = CJ2 ? CJ2 : J2r;
    const int J3 = CJ3 ? CJ3 : J3r;
    float xt = 0.f;
#pragma unroll
    for (int p = 0; p < J1; ++p) {
        float vp = 0.f;
#pragma unroll
        for (int q = 0; q < J2; ++q) {
            const float *g = G + (p * J2 + q) * J3;
            float t = 0.f;
#pragma unroll
            for (int r = 0; r < J3; ++r) t = fmaf(g[r], c[r], t);
            vp = fmaf(t, b[q], vp);
        }
        xt = fmaf(a[p], vp, xt);
    }
    return xt;
}

// Supported compile-time shapes; anything else runs the runtime-rank instantiation.
#define SNECT_DISPATCH_RANKS(J1, J2, J3, FN, ...)                                      \
    (((J1) == 5 && (J2) == 5 && (J3) == 2)      ? FN<5, 5, 2>(__VA_ARGS__)            \
     : ((J1) == 10 && (J2) == 10 && (J3) == 5)  ? FN<10, 10, 5>(__VA_ARGS__)          \
     : ((J1) == 16 && (J2) == 16 && (J3) == 5)  ? FN<16, 16, 5>(__VA_ARGS__)          \
     : ((J1) == 32 && (J2) == 32 && (J3) == 5)  ? FN<32, 32, 5>(__VA_ARGS__)          \
                                                : FN<0, 0, 0>(__VA_ARGS__))

}  // namespace snect
