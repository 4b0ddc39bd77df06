// QR orthogonalisation post-pass (Alg. 1, the step after the sweeps): for each mode n,
// U^(n) = Q R with Q orthonormal (I_n x J_n) and R upper triangular (J_n x J_n), then
// U^(n) <- Q and G <- G x_n R.  x~ is unchanged (Tucker gauge: U R^{-1} with G x_n R).
//
// The thin QR of a tall factor is taken as Cholesky-QR applied twice: R1 = chol(U^T U),
// Q1 = U R1^{-1}, R2 = chol(Q1^T Q1), Q = Q1 R2^{-1}, R = R2 R1.  The Gram matrices, the
// factors and the inverses are FP64; the second pass restores the orthonormality the first
// loses to rounding.  Q has a positive diagonal in R (the Householder QR of the same matrix
// differs by the signs of R's rows and Q's columns).  A mode with J_n > I_n has no J_n
// orthonormal columns and keeps its factor.
#include "common.cuh"

namespace snect {

namespace {

constexpr int kQrRows = 256;  // rows of U per CTA of the Gram kernel

// gram += U^T U over this CTA's rows (upper triangle, FP64)
__global__ void __launch_bounds__(256) k_qr_gram(const float *__restrict__ U, int64_t I, int J, double *gram) {
    __shared__ float sU[kQrRows * kMaxRank];
    const int64_t r0 = (int64_t)blockIdx.x * kQrRows;
    const int nr = (int)((I - r0) < kQrRows ? (I - r0) : kQrRows);
    for (int e = threadIdx.x; e < nr * J; e += blockDim.x) sU[e] = U[r0 * J + e];
    __syncthreads();
    for (int s = threadIdx.x; s < J * J; s += blockDim.x) {
        const int p = s / J, q = s % J;
        if (p > q) continue;
        double a = 0.0;
        for (int i = 0; i < nr; ++i) a += (double)sU[i * J + p] * (double)sU[i * J + q];
        atomicAdd(gram + s, a);
    }
}

// R = chol(gram)^T (upper), Rinv = R^{-1}, and Rtot <- R Rtot (Rtot = I on the first pass);
// one thread (J <= 32).  status[0] = 1 if the Gram matrix is not positive definite.
__global__ void k_qr_chol(const double *__restrict__ gram, int J, double *R, double *Rinv, double *Rtot, int first,
                          int *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int e = 0; e < J * J; ++e) R[e] = 0.0;
    for (int j = 0; j < J; ++j) {  // upper R with R^T R = gram, row j
        double d = gram[j * J + j];
        for (int k = 0; k < j; ++k) d -= R[k * J + j] * R[k * J + j];
        if (!(d > 0.0)) {
            status[0] = 1;
            d = 1e-300;
        }
        d = sqrt(d);
        R[j * J + j] = d;
        for (int c = j + 1; c < J; ++c) {
            double x = gram[j * J + c];
            for (int k = 0; k < j; ++k) x -= R[k * J + j] * R[k * J + c];
            R[j * J + c] = x / d;
        }
    }
    for (int c = 0; c < J; ++c) {  // Rinv column c: back substitution of R x = e_c
        for (int i = J - 1; i >= 0; --i) {
            double x = i == c ? 1.0 : 0.0;
            for (int k = i + 1; k < J; ++k) x -= R[i * J + k] * Rinv[k * J + c];
            Rinv[i * J + c] = x / R[i * J + i];
        }
    }
    double T[kMaxRank * kMaxRank];
    for (int i = 0; i < J; ++i)
        for (int c = 0; c < J; ++c) {
            double x = 0.0;
            if (first) {
                x = R[i * J + c];
            } else {
                for (int k = 0; k < J; ++k) x += R[i * J + k] * Rtot[k * J + c];
            }
            T[i * J + c] = x;
        }
    for (int e = 0; e < J * J; ++e) Rtot[e] = T[e];
}

// U <- U Rinv, row by row (FP64 products, FP32 storage)
__global__ void k_qr_apply(float *__restrict__ U, int64_t I, int J, const double *__restrict__ Rinv) {
    __shared__ double sR[kMaxRank * kMaxRank];
    for (int e = threadIdx.x; e < J * J; e += blockDim.x) sR[e] = Rinv[e];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    double u[kMaxRank];
    for (int t = 0; t < J; ++t) u[t] = U[i * J + t];
    for (int c = 0; c < J; ++c) {
        double x = 0.0;
        for (int t = 0; t <= c; ++t) x += u[t] * sR[t * J + c];
        U[i * J + c] = (float)x;
    }
}

// G <- G x_md R: new g at index t along mode md = sum_z R[t][z] g(.. z ..); one CTA
__global__ void k_qr_core(float *__restrict__ G, Dims d, int md, const double *__restrict__ R) {
    extern __shared__ float sG[];
    const int PI = d.J1 * d.J2 * d.J3;
    for (int s = threadIdx.x; s < PI; s += blockDim.x) sG[s] = G[s];
    __syncthreads();
    const int nc = md == 0 ? d.J1 : (md == 1 ? d.J2 : d.J3);
    for (int s = threadIdx.x; s < PI; s += blockDim.x) {
        const int p = s / (d.J2 * d.J3), q = (s / d.J3) % d.J2, r = s % d.J3;
        const int t = md == 0 ? p : (md == 1 ? q : r);
        double a = 0.0;
        for (int z = 0; z < nc; ++z) {
            const int pp = md == 0 ? z : p, qq = md == 1 ? z : q, rr = md == 2 ? z : r;
            a += R[t * nc + z] * (double)sG[(pp * d.J2 + qq) * d.J3 + rr];
        }
        G[s] = (float)a;
    }
}

}  // namespace

int qr_post(Ctx *c, int *skipped) {
    const Dims &d = c->d;
    const int64_t I[3] = {d.I1, d.I2, d.I3};
    const int J[3] = {d.J1, d.J2, d.J3};
    *skipped = 0;
    double *buf = nullptr;
    int *status = nullptr;
    // gram, R, Rinv, Rtot (J x J each, J <= 32)
    SNECT_CUDA(c, scratch_alloc(c, (void **)&buf, sizeof(double) * 4 * kMaxRank * kMaxRank));
    SNECT_CUDA(c, scratch_alloc(c, (void **)&status, sizeof(int)));
    SNECT_CUDA(c, cudaMemsetAsync(status, 0, sizeof(int), c->stream));
    double *gram = buf, *R = buf + kMaxRank * kMaxRank, *Rinv = R + kMaxRank * kMaxRank, *Rtot = Rinv + kMaxRank * kMaxRank;
    cudaError_t e = cudaSuccess;
    for (int md = 0; md < 3 && e == cudaSuccess; ++md) {
        if (J[md] > I[md]) {  // no J orthonormal columns in I rows: the factor is kept
            *skipped |= 1 << md;
            continue;
        }
        for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
            e = cudaMemsetAsync(gram, 0, sizeof(double) * J[md] * J[md], c->stream);
            if (e != cudaSuccess) break;
            k_qr_gram<<<(unsigned)ceil_div(I[md], kQrRows), 256, 0, c->stream>>>(c->U[md], I[md], J[md], gram);
            k_qr_chol<<<1, 32, 0, c->stream>>>(gram, J[md], R, Rinv, Rtot, pass == 0, status);
            k_qr_apply<<<(unsigned)ceil_div(I[md], 256), 256, 0, c->stream>>>(c->U[md], I[md], J[md], Rinv);
            c->launches += 3;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_qr_core<<<1, 256, sizeof(float) * c->PI, c->stream>>>(c->G, d, md, Rtot);
            c->launches++;
            e = cudaGetLastError();
        }
    }
    int h_status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFreeAsync(buf, c->stream);
    cudaFreeAsync(status, c->stream);
    if (e != cudaSuccess) return fail(c, SNECT_ECUDA, std::string("QR post-pass: ") + cudaGetErrorString(e));
    if (h_status) return fail(c, SNECT_EINVAL, "QR post-pass: a factor is rank deficient (Gram not positive definite)");
    c->param_version++;
    return SNECT_OK;
}

}  // namespace snect
