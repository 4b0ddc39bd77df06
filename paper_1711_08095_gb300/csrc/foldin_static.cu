// Fold-in of one new patient that allocates no device memory (snect_foldin_static).
//
// Some callers cannot call cudaMalloc: a process that runs inside another framework's memory
// budget or allocator, a real-time serving loop that must not stall on the allocator, or
// code that keeps every device buffer it touches pre-reserved.  For them this entry point
// takes the frozen factors, the query and the output row as caller-owned device buffers and
// keeps its only working memory -- the per-CTA partial sums of the J1 x J1 Gram matrix and
// right-hand side, and two status words -- in one file-scope device array of fixed size,
// reserved on every GPU that loads the library until the process exits.
//
// Host code cannot use the array's name as a device address (in host code it names a
// host-side stand-in), so the first call on each device does a one-time set-up with that
// device current: it looks the address up with cudaGetSymbolAddress and caches it, and it
// raises the partial-sum kernel's dynamic shared-memory limit so that every core the entry
// point accepts (J1*J2*J3 <= 5,120) fits beside the kernel's static tiles.  Every call ends
// by reading two status words back and synchronising, so none can be captured into a CUDA
// graph.  Every call shares the array and leaves its
// contents behind: the status words are cleared at the start of each call and every partial
// is overwritten before it is read.  Two calls whose work overlaps on the GPU race on the
// array.
//
// The arithmetic is that of snect_foldin: w_jk = G x2 u2_j x3 u3_k (computed here per cell,
// in the same order as snect_foldin's table), a fixed-order FP32 Gram per CTA, the partials
// added in CTA order, lambda I added and an FP64 Cholesky solve.
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace snect {

namespace {

constexpr int64_t kStaticMaxCells = 1 << 20;  // largest query: 1,048,576 cells
constexpr int kSThreads = 256;
constexpr int kSTile = 256;
constexpr int64_t kSChunk = 4096;             // cells per CTA
constexpr int64_t kSMaxParts = (kStaticMaxCells + kSChunk - 1) / kSChunk;
constexpr int kSPartStride = kMaxRank * kMaxRank + kMaxRank;
constexpr int kSPerThread = (kMaxRank * kMaxRank + kSThreads - 1) / kSThreads;
constexpr int64_t kSStatusWords = 64;         // [0]: bad cell, [1]: not positive definite
constexpr int64_t kSScratchFloats = kSMaxParts * kSPartStride + kSStatusWords;  // ~1.03 MiB

static __device__ __align__(256) float g_foldin_scratch[kSScratchFloats];

std::mutex g_addr_mu;
float *g_addr[256] = {};  // per device: device address of g_foldin_scratch (null: not set up)

__global__ void k_static_check(const int32_t *__restrict__ jk, const float *__restrict__ val, int64_t n,
                               int32_t I2, int32_t I3, int32_t *status) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int32_t j = jk[2 * e], k = jk[2 * e + 1];
    if (j < 0 || j >= I2 || k < 0 || k >= I3 || !isfinite(val[e])) atomicOr(status, 1);
}

// one CTA per run of kSChunk cells: w per cell (thread per (cell, p)), then the Gram and the
// right-hand side summed over the run in cell order (thread per Gram element)
__global__ void __launch_bounds__(kSThreads)
    k_static_partial(const int32_t *__restrict__ jk, const float *__restrict__ val, int64_t n,
                     const float *__restrict__ G, const float *__restrict__ U2,
                     const float *__restrict__ U3, int32_t I2, int32_t I3, int32_t J1, int32_t J2,
                     int32_t J3, float *__restrict__ part) {
    extern __shared__ float sG[];
    __shared__ float sw[kSTile * kMaxRank];
    __shared__ float sx[kSTile];
    const int PI = J1 * J2 * J3;
    for (int t = threadIdx.x; t < PI; t += blockDim.x) sG[t] = G[t];
    const int64_t c0 = (int64_t)blockIdx.x * kSChunk;
    const int64_t c1 = n < c0 + kSChunk ? n : c0 + kSChunk;
    const int nG = J1 * J1;
    float acc[kSPerThread];
#pragma unroll
    for (int t = 0; t < kSPerThread; ++t) acc[t] = 0.f;
    float accx = 0.f;
    for (int64_t base = c0; base < c1; base += kSTile) {
        const int len = (c1 - base) < kSTile ? (int)(c1 - base) : kSTile;
        __syncthreads();
        for (int t = threadIdx.x; t < len * J1; t += blockDim.x) {
            const int e = t / J1, p = t % J1;
            const int32_t j = jk[2 * (base + e)], k = jk[2 * (base + e) + 1];
            float s = 0.f;
            if (j >= 0 && j < I2 && k >= 0 && k < I3) {  // a bad cell is flagged and contributes 0
                const float *b = U2 + (int64_t)j * J2;
                const float *c = U3 + (int64_t)k * J3;
                for (int q = 0; q < J2; ++q) {
                    float tq = 0.f;
                    const float *g = sG + (p * J2 + q) * J3;
                    for (int r = 0; r < J3; ++r) tq = fmaf(g[r], c[r], tq);
                    s = fmaf(tq, b[q], s);
                }
            }
            sw[e * J1 + p] = s;
        }
        for (int t = threadIdx.x; t < len; t += blockDim.x) {
            const float x = val[base + t];
            sx[t] = isfinite(x) ? x : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kSPerThread; ++t) {
            const int s = threadIdx.x + t * kSThreads;
            if (s < nG) {
                const int p = s / J1, q = s % J1;
                float a = acc[t];
                for (int e = 0; e < len; ++e) a = fmaf(sw[e * J1 + p], sw[e * J1 + q], a);
                acc[t] = a;
            }
        }
        if (threadIdx.x < J1) {
            const int p = threadIdx.x;
            for (int e = 0; e < len; ++e) accx = fmaf(sx[e], sw[e * J1 + p], accx);
        }
    }
    float *out = part + (int64_t)blockIdx.x * (nG + J1);
#pragma unroll
    for (int t = 0; t < kSPerThread; ++t) {
        const int s = threadIdx.x + t * kSThreads;
        if (s < nG) out[s] = acc[t];
    }
    if (threadIdx.x < J1) out[nG + threadIdx.x] = accx;
}

__global__ void __launch_bounds__(kSThreads)
    k_static_solve(const float *__restrict__ part, int32_t n_part, int32_t J1, float ridge,
                   float *__restrict__ u_out, int32_t *__restrict__ status) {
    __shared__ double M[kMaxRank * kMaxRank];
    __shared__ double rhs[kMaxRank];
    const int nG = J1 * J1;
    if (status[0]) {  // a bad cell was flagged: the output row is zero, not a partial solution
        if (threadIdx.x < J1) u_out[threadIdx.x] = 0.f;
        return;
    }
    for (int s = threadIdx.x; s < nG + J1; s += blockDim.x) {
        float a = 0.f;
        for (int t = 0; t < n_part; ++t) a += part[(int64_t)t * (nG + J1) + s];
        if (s < nG)
            M[s] = (double)a + ((s / J1 == s % J1) ? (double)ridge : 0.0);
        else
            rhs[s - nG] = (double)a;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int j = 0; j < J1; ++j) {
        double d = M[j * J1 + j];
        for (int k = 0; k < j; ++k) d -= M[j * J1 + k] * M[j * J1 + k];
        if (!(d > 0.0)) {
            status[1] = 1;
            for (int p = 0; p < J1; ++p) u_out[p] = 0.f;
            return;
        }
        d = sqrt(d);
        M[j * J1 + j] = d;
        for (int i = j + 1; i < J1; ++i) {
            double s = M[i * J1 + j];
            for (int k = 0; k < j; ++k) s -= M[i * J1 + k] * M[j * J1 + k];
            M[i * J1 + j] = s / d;
        }
    }
    for (int i = 0; i < J1; ++i) {
        double s = rhs[i];
        for (int k = 0; k < i; ++k) s -= M[i * J1 + k] * rhs[k];
        rhs[i] = s / M[i * J1 + i];
    }
    for (int i = J1 - 1; i >= 0; --i) {
        double s = rhs[i];
        for (int k = i + 1; k < J1; ++k) s -= M[k * J1 + i] * rhs[k];
        rhs[i] = s / M[i * J1 + i];
    }
    for (int p = 0; p < J1; ++p) u_out[p] = (float)rhs[p];
}

// device address of the scratch array on the current device (looked up once per device)
int scratch_address(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, SNECT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return fail(nullptr, SNECT_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_foldin_scratch);
        if (e != cudaSuccess || !p)
            return fail(nullptr, SNECT_ECUDA,
                        std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        // the core (up to kMaxCore floats) is the kernel's dynamic shared memory, beside about
        // 33 KB of static tiles: above the 48 KB default once J1*J2*J3 > 3,840
        e = cudaFuncSetAttribute(k_static_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float) * kMaxCore));
        if (e != cudaSuccess)
            return fail(nullptr, SNECT_ECUDA,
                        std::string("cudaFuncSetAttribute(k_static_partial): ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<float *>(p);
    }
    *out = g_addr[dev];
    return SNECT_OK;
}

}  // namespace

}  // namespace snect

using namespace snect;

extern "C" int snect_foldin_static(const float *G, const float *U2, const float *U3, int32_t I2, int32_t I3,
                                   int32_t J1, int32_t J2, int32_t J3, const int32_t *jk, const float *val,
                                   int64_t n, float lambda, float *u_out, void *stream) {
    if (!G || !U2 || !U3 || !jk || !val || !u_out) return fail(nullptr, SNECT_EINVAL, "null pointer");
    if (I2 < 1 || I3 < 1 || J1 < 1 || J2 < 1 || J3 < 1 || J1 > kMaxRank || J2 > kMaxRank || J3 > kMaxRank ||
        (int64_t)J1 * J2 * J3 > kMaxCore)
        return fail(nullptr, SNECT_EINVAL, "dims: I2, I3 >= 1, J_n in [1, 32], J1*J2*J3 <= 5120");
    if (n < 1) return fail(nullptr, SNECT_EINVAL, "a query needs at least one observed cell");
    if (n > kStaticMaxCells)
        return fail(nullptr, SNECT_EINVAL,
                    "query has more cells than the static scratch allows (1,048,576); use snect_foldin");
    if (!isfinite(lambda) || lambda < 0.f) return fail(nullptr, SNECT_EINVAL, "lambda must be finite and >= 0");
    float *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    float *part = scratch;
    int32_t *status = reinterpret_cast<int32_t *>(scratch + kSMaxParts * kSPartStride);
    const int64_t np = (n + kSChunk - 1) / kSChunk;
    SNECT_CUDA(nullptr, cudaMemsetAsync(status, 0, 2 * sizeof(int32_t), st));
    k_static_check<<<ceil_div(n, 256), 256, 0, st>>>(jk, val, n, I2, I3, status);
    const size_t smem = sizeof(float) * (size_t)J1 * J2 * J3;
    k_static_partial<<<(unsigned)np, kSThreads, smem, st>>>(jk, val, n, G, U2, U3, I2, I3, J1, J2, J3, part);
    k_static_solve<<<1, kSThreads, 0, st>>>(part, (int32_t)np, J1, lambda, u_out, status);
    SNECT_CUDA(nullptr, cudaGetLastError());
    int32_t hs[2] = {0, 0};
    SNECT_CUDA(nullptr, cudaMemcpyAsync(hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st));
    SNECT_CUDA(nullptr, cudaStreamSynchronize(st));
    if (hs[0]) return fail(nullptr, SNECT_EINVAL, "query cell out of range or value not finite");
    if (hs[1]) return fail(nullptr, SNECT_EINVAL, "fold-in normal matrix is not positive definite");
    return SNECT_OK;
}
