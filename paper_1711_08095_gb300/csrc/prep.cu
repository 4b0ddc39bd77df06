// Set-up work done once per problem on the GPU: validation and packing of the entries,
// the training counts |Omega^{n,i}|, the per-batch row grouping of the deterministic mode,
// and the sorted adjacency (CSR) of the gene network.
#include <cub/cub.cuh>

#include <vector>

#include "common.cuh"

namespace snect {

namespace {

enum : int32_t {
    kBadIndex = 1,
    kBadValue = 2,
    kSelfLoop = 4,
    kDupEdge = 8,
    kBadWeight = 16,
};

__global__ void k_pack(const int32_t *__restrict__ idx, const float *__restrict__ val, int64_t n,
                       int32_t n_modes, int32_t I1, int32_t I2, int32_t I3, Rec *__restrict__ out,
                       int32_t *flag) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    Rec r;
    r.i = idx[e * n_modes + 0];
    r.j = idx[e * n_modes + 1];
    r.k = n_modes == 3 ? idx[e * 3 + 2] : 0;
    r.x = val[e];
    bool bad = r.i < 0 || r.i >= I1 || r.j < 0 || r.j >= I2 || r.k < 0 || r.k >= I3;
    if (bad) {
        atomicOr(flag, kBadIndex);
        r.i = r.j = r.k = 0;  // keep later kernels in bounds; the call reports the error
    }
    if (!isfinite(r.x)) atomicOr(flag, kBadValue);
    out[e] = r;
}

// per-row counts; the platform counts (few, heavily shared rows) go through a per-CTA
// shared-memory histogram first
__global__ void k_counts(const Rec *__restrict__ rec, int64_t n, int32_t I3, int32_t *c1, int32_t *c2,
                         int32_t *c3) {
    __shared__ int32_t h3[kMaxPlatforms];
    const bool small3 = I3 <= kMaxPlatforms;
    for (int t = threadIdx.x; t < kMaxPlatforms; t += blockDim.x) h3[t] = 0;
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) {
        const Rec r = rec[e];
        atomicAdd(c1 + r.i, 1);
        atomicAdd(c2 + r.j, 1);
        if (small3)
            atomicAdd(h3 + r.k, 1);
        else
            atomicAdd(c3 + r.k, 1);
    }
    __syncthreads();
    if (small3)
        for (int t = threadIdx.x; t < I3; t += blockDim.x)
            if (h3[t]) atomicAdd(c3 + t, h3[t]);
}

// the same counts with every mode's histogram in shared memory (when I1 + I2 + I3 bins fit):
// a grid-stride loop counts many entries per CTA with shared atomics, then each nonzero bin
// goes to global memory once per CTA
constexpr int kCountBins = 24576;  // ints of shared memory (96 KB)

__global__ void __launch_bounds__(1024) k_counts_smem(const Rec *__restrict__ rec, int64_t n, int32_t I1, int32_t I2,
                                                      int32_t I3, int32_t *c1, int32_t *c2, int32_t *c3) {
    extern __shared__ int32_t hs[];  // I1 | I2 | I3
    const int nb = I1 + I2 + I3;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) hs[t] = 0;
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const Rec r = rec[e];
        atomicAdd(hs + r.i, 1);
        atomicAdd(hs + I1 + r.j, 1);
        atomicAdd(hs + I1 + I2 + r.k, 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        const int v = hs[t];
        if (v == 0) continue;
        if (t < I1) atomicAdd(c1 + t, v);
        else if (t < I1 + I2) atomicAdd(c2 + (t - I1), v);
        else atomicAdd(c3 + (t - I1 - I2), v);
    }
}

// key = (batch << 32) | row of the given mode; value = entry position
__global__ void k_group_keys(const Rec *__restrict__ rec, int64_t n, int32_t batch, int mode,
                             uint64_t *keys, int32_t *vals) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    Rec r = rec[e];
    uint32_t row = mode == 0 ? r.i : (mode == 1 ? r.j : r.k);
    keys[e] = ((uint64_t)(e / batch) << 32) | row;
    vals[e] = (int32_t)e;
}

__global__ void k_heads(const uint64_t *__restrict__ keys, int64_t n, uint8_t *head) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    head[s] = (s == 0 || keys[s] != keys[s - 1]) ? 1 : 0;
}

__global__ void k_half_edges(const int32_t *__restrict__ edges, const float *__restrict__ w,
                             int64_t m, int32_t I2, uint64_t *keys, int32_t *vals, int2 *out_edges,
                             float *out_w, int32_t *flag) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int32_t u = edges[2 * t], v = edges[2 * t + 1];
    float y = w[t];
    if (u < 0 || u >= I2 || v < 0 || v >= I2) {
        atomicOr(flag, kBadIndex);
        u = 0;
        v = 1;
    }
    if (u == v) atomicOr(flag, kSelfLoop);
    if (!(y > 0.0f) || !isfinite(y)) atomicOr(flag, kBadWeight);
    out_edges[t] = make_int2(u, v);
    out_w[t] = y;
    keys[2 * t] = ((uint64_t)(uint32_t)u << 32) | (uint32_t)v;
    vals[2 * t] = (int32_t)t;
    keys[2 * t + 1] = ((uint64_t)(uint32_t)v << 32) | (uint32_t)u;
    vals[2 * t + 1] = (int32_t)t;
}

// ptr[k] = first sorted half-edge whose source is >= k; col/w from the sorted keys
__global__ void k_csr(const uint64_t *__restrict__ keys, const int32_t *__restrict__ vals,
                      int64_t n2, int32_t I2, const float *__restrict__ w, int32_t *ptr,
                      int32_t *col, float *cw, int32_t *flag) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > n2) return;
    if (s == n2) {  // tail: rows after the last source
        int32_t last = n2 ? (int32_t)(keys[n2 - 1] >> 32) : -1;
        for (int32_t k = last + 1; k <= I2; ++k) ptr[k] = (int32_t)n2;
        return;
    }
    uint64_t key = keys[s];
    int32_t src = (int32_t)(key >> 32);
    col[s] = (int32_t)(key & 0xffffffffu);
    cw[s] = w[vals[s]];
    int32_t prev = s ? (int32_t)(keys[s - 1] >> 32) : -1;
    if (s && keys[s - 1] == key) atomicOr(flag, kDupEdge);
    for (int32_t k = prev + 1; k <= src; ++k) ptr[k] = (int32_t)s;
}

__global__ void k_max_degree(const int32_t *__restrict__ ptr, int32_t I2, int32_t *out) {
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= I2) return;
    atomicMax(out, ptr[k + 1] - ptr[k]);
}

// key = (wave << 32) | platform; value = entry position (fast mode grouping)
// entries per (wave, row, platform) of the two row modes, from the wave-grouped order (wave w
// holds positions [w W, (w + 1) W)).  A patient's entries inside a wave and platform sit next
// to each other, so each run in a warp adds its length once; gene rows add one per entry.
__global__ void k_wave_row_counts(const Rec *__restrict__ rec, int64_t n, int64_t W, int32_t I1, int32_t I2,
                                  int32_t I3, float *tab) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = e < n;
    Rec r;
    r.i = r.j = r.k = 0;
    r.x = 0.f;
    if (ok) r = rec[e];
    const int64_t w = ok ? e / W : 0;
    float *t = tab + w * ((int64_t)I1 + I2) * I3;
    const unsigned long long key =
        ok ? (((unsigned long long)w << 40) | ((unsigned long long)r.k << 32) | (unsigned)r.i) : ~0ull;
    const unsigned run = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    if (ok && __ffs(run) - 1 == lane) atomicAdd(t + (int64_t)r.i * I3 + r.k, (float)__popc(run));
    if (ok) atomicAdd(t + ((int64_t)I1 + r.j) * I3 + r.k, 1.f);
}

// the same key in 32 bits, when it fits
__global__ void k_wave_keys32(const Rec *__restrict__ rec, int64_t n, int64_t wave, int bi, int bk,
                              uint32_t *keys, int32_t *vals) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const Rec r = rec[e];
    keys[e] = ((uint32_t)(e / wave) << (bi + bk)) | ((uint32_t)r.k << bi) | (bi ? (uint32_t)r.i : 0u);
    vals[e] = (int32_t)e;
}

// key (wave, platform, patient): bits [0, bi) patient (0 when bi = 0), [bi, bi + bk) platform,
// above that the wave
__global__ void k_wave_keys(const Rec *__restrict__ rec, int64_t n, int64_t wave, int bi, int bk,
                            uint64_t *keys, int32_t *vals) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const Rec r = rec[e];
    keys[e] = ((uint64_t)(e / wave) << (bi + bk)) | ((uint64_t)r.k << bi) | (bi ? (uint64_t)r.i : 0u);
    vals[e] = (int32_t)e;
}

__global__ void k_permute(const Rec *__restrict__ src, const int32_t *__restrict__ perm, int64_t n,
                          Rec *__restrict__ dst) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    dst[e] = src[perm[e]];
}

// entries per (wave, platform); a CTA's 1,024 entries span at most two waves when
// wave >= 1,024, so each CTA first counts into a shared histogram of 2 x I3 bins
__global__ void k_wave_hist(const Rec *__restrict__ rec, int64_t n, int64_t wave, int32_t I3,
                            int32_t *hist) {
    __shared__ int32_t h[2 * kMaxPlatforms];
    const int64_t e0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t w0 = e0 / wave;
    for (int t = threadIdx.x; t < 2 * kMaxPlatforms; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const int64_t e = e0 + threadIdx.x;
    if (e < n) {
        const int64_t dw = e / wave - w0;
        if (dw < 2)
            atomicAdd(h + dw * I3 + rec[e].k, 1);
        else
            atomicAdd(hist + (e / wave) * I3 + rec[e].k, 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * I3; t += blockDim.x) {
        const int64_t w = w0 + t / I3;
        if (h[t]) atomicAdd(hist + w * I3 + t % I3, h[t]);
    }
}

// ---- fast mode: one pass over the inputs orders the entries by counting ----------------
// Every entry falls in a bucket (wave, platform, patient), wave = position / W; buckets in
// that order are the order the fast sweep wants.  The packing pass counts each bucket with an
// atomic that also hands the entry its rank inside the bucket; an exclusive scan of the counts
// gives each bucket's first position, and a scatter puts every entry at first + rank.  Inside
// a bucket (one patient's entries of one platform in one wave) the order is that of the
// atomics, which the sweep does not depend on: every gradient of a wave is taken at the
// wave-start parameters.
constexpr int kPackWarps = 32;   // warps per CTA of the packing pass
constexpr int kPackChunk = 128;  // entries per warp step, four per lane

struct PackFastArgs {
    const int32_t *idx;  // nnz x 3, where a kernel can read it (device or pinned host memory)
    const float *val;
    int64_t n, W;
    int32_t I1, I2, I3;
    int32_t vec;         // idx and val 16-byte aligned: the warp reads its chunk with vector loads
    Rec *out;            // entries in input order
    int32_t *rank;       // rank of each entry inside its bucket
    int32_t *bcnt;       // (wave, platform, patient) bucket counts, zeroed
    float *wcnt;         // per-wave (row, platform) entry table or NULL; gene rows counted here
    int32_t *c1, *c2, *c3, *flag;
};

// Packs, validates and counts the entries: rows of every mode (|Omega^{n,i}|, through shared
// histograms when SMEM), buckets, and the wave table's gene rows.  A warp takes 128 entries
// at a time; with aligned inputs its 1,536 index bytes arrive as three coalesced 512-byte
// loads (the right shape for reads of host memory over the link) and are redistributed
// through shared memory, four entries to a lane.
template <bool SMEM>
__global__ void __launch_bounds__(kPackWarps * 32) k_pack_fast(PackFastArgs A) {
    extern __shared__ int32_t psm[];  // per warp 3 x 128 ints | histograms I1 | I2 | I3 (SMEM)
    int32_t *tr = psm + (threadIdx.x >> 5) * 3 * kPackChunk;
    int32_t *hs = psm + kPackWarps * 3 * kPackChunk;
    const int32_t I1 = A.I1, I2 = A.I2, I3 = A.I3;
    if (SMEM) {
        for (int t = threadIdx.x; t < I1 + I2 + I3; t += blockDim.x) hs[t] = 0;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int64_t n_chunks = (A.n + kPackChunk - 1) / kPackChunk;
    const int64_t n_warps = (int64_t)gridDim.x * kPackWarps;
    for (int64_t ch = (int64_t)blockIdx.x * kPackWarps + (threadIdx.x >> 5); ch < n_chunks; ch += n_warps) {
        const int64_t e0 = ch * kPackChunk + 4 * lane;  // this lane's first entry
        int32_t ii[4], jj[4], kk[4];
        float xx[4];
        int m = 0;  // entries of this lane inside the input
        if (A.vec && ch * kPackChunk + kPackChunk <= A.n) {  // uniform across the warp
            const int4 *s4 = reinterpret_cast<const int4 *>(A.idx) + ch * (3 * kPackChunk / 4);
            int4 *t4 = reinterpret_cast<int4 *>(tr);
            t4[lane] = s4[lane];
            t4[lane + 32] = s4[lane + 32];
            t4[lane + 64] = s4[lane + 64];
            const float4 v = reinterpret_cast<const float4 *>(A.val)[ch * (kPackChunk / 4) + lane];
            __syncwarp();
            // entries 4 lane .. 4 lane + 3 are ints 12 lane .. 12 lane + 11
            const int4 a = t4[3 * lane], b = t4[3 * lane + 1], c = t4[3 * lane + 2];
            __syncwarp();  // read before the next chunk overwrites them
            ii[0] = a.x, jj[0] = a.y, kk[0] = a.z;
            ii[1] = a.w, jj[1] = b.x, kk[1] = b.y;
            ii[2] = b.z, jj[2] = b.w, kk[2] = c.x;
            ii[3] = c.y, jj[3] = c.z, kk[3] = c.w;
            xx[0] = v.x, xx[1] = v.y, xx[2] = v.z, xx[3] = v.w;
            m = 4;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ii[q] = jj[q] = kk[q] = 0;
                xx[q] = 0.f;
                if (e0 + q < A.n) {
                    ii[q] = A.idx[3 * (e0 + q)];
                    jj[q] = A.idx[3 * (e0 + q) + 1];
                    kk[q] = A.idx[3 * (e0 + q) + 2];
                    xx[q] = A.val[e0 + q];
                    m = q + 1;
                }
            }
        }
        int32_t rk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            rk[q] = 0;
            if (q >= m) continue;
            const int64_t e = e0 + q;
            Rec r;
            r.i = ii[q], r.j = jj[q], r.k = kk[q], r.x = xx[q];
            if (r.i < 0 || r.i >= I1 || r.j < 0 || r.j >= I2 || r.k < 0 || r.k >= I3) {
                atomicOr(A.flag, kBadIndex);
                r.i = r.j = r.k = 0;  // keep later kernels in bounds; the call reports the error
            }
            if (!isfinite(r.x)) atomicOr(A.flag, kBadValue);
            A.out[e] = r;
            const int64_t w = e / A.W;
            rk[q] = atomicAdd(A.bcnt + (w * I3 + r.k) * I1 + r.i, 1);
            if (A.wcnt) atomicAdd(A.wcnt + (w * ((int64_t)I1 + I2) + I1 + r.j) * I3 + r.k, 1.f);
            if (SMEM) {
                atomicAdd(hs + r.i, 1);
                atomicAdd(hs + I1 + r.j, 1);
                atomicAdd(hs + I1 + I2 + r.k, 1);
            } else {
                atomicAdd(A.c1 + r.i, 1);
                atomicAdd(A.c2 + r.j, 1);
                atomicAdd(A.c3 + r.k, 1);
            }
        }
        if (m == 4)  // e0 is a multiple of 4: one aligned 16-byte store
            *reinterpret_cast<int4 *>(A.rank + e0) = make_int4(rk[0], rk[1], rk[2], rk[3]);
        else
            for (int q = 0; q < m; ++q) A.rank[e0 + q] = rk[q];
    }
    if (SMEM) {
        __syncthreads();
        for (int t = threadIdx.x; t < I1 + I2 + I3; t += blockDim.x) {
            const int v = hs[t];
            if (v == 0) continue;
            if (t < I1) atomicAdd(A.c1 + t, v);
            else if (t < I1 + I2) atomicAdd(A.c2 + (t - I1), v);
            else atomicAdd(A.c3 + (t - I1 - I2), v);
        }
    }
}

// every entry to its bucket's first position + its rank
__global__ void k_bucket_scatter(const Rec *__restrict__ src, const int32_t *__restrict__ rank,
                                 const int32_t *__restrict__ first, int64_t n, int64_t W, int32_t I1, int32_t I3,
                                 Rec *__restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const Rec r = src[e];
    dst[first[(e / W * I3 + r.k) * I1 + r.i] + rank[e]] = r;
}

// the wave table's patient rows: bucket (w, k, i)'s count is row i's entries of platform k
// in wave w
__global__ void k_bucket_wave_rows(const int32_t *__restrict__ bcnt, int64_t nb, int32_t I1, int32_t I2,
                                   int32_t I3, float *__restrict__ wcnt) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int64_t i = b % I1, wk = b / I1, k = wk % I3, w = wk / I3;
    wcnt[(w * ((int64_t)I1 + I2) + i) * I3 + k] = (float)bcnt[b];
}

// tile t of the wave kernels: found by binary search over the segments' first tiles; seg
// holds S segment starts, S counts and S + 1 first tiles (segment s = wave s / I3, platform
// s % I3)
__global__ void k_build_tiles(const int32_t *__restrict__ seg, int32_t S, int32_t I3, int64_t n_tiles,
                              int32_t *__restrict__ ts, int32_t *__restrict__ tl, int32_t *__restrict__ tk) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const int32_t *pos = seg, *cnt = seg + S, *t0 = seg + 2 * S;
    int lo = 0, hi = S;  // t0[lo] <= t < t0[hi]; the answer is the last segment with t0 <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (t0[mid] <= t) lo = mid;
        else hi = mid;
    }
    const int32_t lt = (int32_t)(t - t0[lo]);
    ts[t] = pos[lo] + lt * kFastTile;
    tl[t] = min(kFastTile, cnt[lo] - lt * kFastTile);
    tk[t] = lo % I3;
}

std::string flag_message(int32_t f) {
    std::string s;
    if (f & kBadIndex) s += " index out of range;";
    if (f & kBadValue) s += " non-finite value;";
    if (f & kSelfLoop) s += " self loop in the gene network;";
    if (f & kDupEdge) s += " duplicate edge in the gene network;";
    if (f & kBadWeight) s += " edge weight not finite and positive;";
    return s;
}

int read_flag(Ctx *c, int32_t *out) {
    SNECT_CUDA(c, cudaMemcpyAsync(out, c->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
    return SNECT_OK;
}

// stable radix sort of (key, value) pairs; temporary buffers allocated here
template <typename K>
int sort_pairs(Ctx *c, K *keys, int32_t *vals, K *keys_out, int32_t *vals_out, int64_t n, int end_bit) {
    size_t tmp_bytes = 0;
    SNECT_CUDA(c, cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys, keys_out, vals, vals_out,
                                                   n, 0, end_bit, c->stream));
    void *tmp = nullptr;
    SNECT_CUDA(c, scratch_alloc(c, &tmp, tmp_bytes));
    cudaError_t e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys, keys_out, vals, vals_out, n,
                                                    0, end_bit, c->stream);
    c->launches += 4;  // radix passes (an estimate; set-up only)
    cudaFreeAsync(tmp, c->stream);
    if (e != cudaSuccess) return fail(c, SNECT_ECUDA, std::string("radix sort: ") + cudaGetErrorString(e));
    return SNECT_OK;
}

int bits_for(uint64_t v) {
    int b = 1;
    while (b < 64 && (v >> b)) ++b;
    return b;
}

}  // namespace

std::string entries_error(int32_t flag) { return "entries:" + flag_message(flag); }

int pack_records(Ctx *c, const int32_t *d_idx, const float *d_val, int64_t n, Rec *out,
                 bool check_ranges, int32_t n_modes) {
    if (n == 0) return SNECT_OK;
    SNECT_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    int32_t I3 = n_modes == 3 ? c->d.I3 : 1;
    k_pack<<<ceil_div(n, 256), 256, 0, c->stream>>>(d_idx, d_val, n, n_modes, c->d.I1, c->d.I2, I3,
                                                     out, c->flag);
    c->launches++;
    SNECT_CUDA(c, cudaGetLastError());
    if (check_ranges) {
        int32_t f = 0;
        int rc = read_flag(c, &f);
        if (rc) return rc;
        if (f) return fail(c, SNECT_EINVAL, "entries:" + flag_message(f));
    }
    return SNECT_OK;
}

int prep_problem(Ctx *c, const int32_t *d_idx, const float *d_val) {
    int rc = pack_records(c, d_idx, d_val, c->nnz, c->rec, true, 3);
    if (rc) return rc;
    for (int md = 0; md < 3; ++md) {
        int32_t In = md == 0 ? c->d.I1 : (md == 1 ? c->d.I2 : c->d.I3);
        SNECT_CUDA(c, cudaMemsetAsync(c->cnt[md], 0, sizeof(int32_t) * In, c->stream));
    }
    if (c->nnz) {
        const int64_t bins = (int64_t)c->d.I1 + c->d.I2 + c->d.I3;
        if (bins <= kCountBins) {
            const size_t smem = sizeof(int32_t) * (size_t)bins;
            SNECT_CUDA(c, cudaFuncSetAttribute(k_counts_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int sms = 0;
            SNECT_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
            const int grid = (int)std::min<int64_t>(ceil_div(c->nnz, 1024), 2 * (int64_t)sms);
            k_counts_smem<<<grid, 1024, smem, c->stream>>>(c->rec, c->nnz, c->d.I1, c->d.I2, c->d.I3, c->cnt[0],
                                                           c->cnt[1], c->cnt[2]);
        } else {
            k_counts<<<ceil_div(c->nnz, 1024), 1024, 0, c->stream>>>(c->rec, c->nnz, c->d.I3, c->cnt[0], c->cnt[1],
                                                                     c->cnt[2]);
        }
        c->launches++;
        SNECT_CUDA(c, cudaGetLastError());
    }
    return SNECT_OK;
}

int prep_det_groups(Ctx *c) {
    int64_t n = c->nnz;
    if (n == 0) return SNECT_OK;
    uint64_t *keys = nullptr, *keys2 = nullptr;
    int32_t *vals = nullptr;
    SNECT_CUDA(c, scratch_alloc(c, &keys, sizeof(uint64_t) * n));
    SNECT_CUDA(c, scratch_alloc(c, &keys2, sizeof(uint64_t) * n));
    SNECT_CUDA(c, scratch_alloc(c, &vals, sizeof(int32_t) * n));
    int rc = SNECT_OK;
    int end_bit = 32 + bits_for((uint64_t)c->n_batches);
    for (int md = 0; md < 3 && rc == SNECT_OK; ++md) {
        k_group_keys<<<ceil_div(n, 256), 256, 0, c->stream>>>(c->rec, n, c->cfg.batch, md, keys, vals);
        c->launches++;
        rc = sort_pairs(c, keys, vals, keys2, c->grp_pos[md], n, end_bit);
        if (rc) break;
        k_heads<<<ceil_div(n, 256), 256, 0, c->stream>>>(keys2, n, c->grp_head[md]);
        c->launches++;
    }
    cudaFreeAsync(keys, c->stream);
    cudaFreeAsync(keys2, c->stream);
    cudaFreeAsync(vals, c->stream);
    if (rc) return rc;
    SNECT_CUDA(c, cudaGetLastError());
    return SNECT_OK;
}

int prep_graph(Ctx *c, const int32_t *d_edges, const float *d_w) {
    int64_t m = c->m;
    int32_t I2 = c->d.I2;
    // the network's own status words (validation, maximum degree), so that it can run beside
    // the packing of the entries, which uses the first
    int32_t *gflag = c->flag + 4;
    SNECT_CUDA(c, cudaMemsetAsync(gflag, 0, sizeof(int32_t), c->stream));
    if (m == 0) {
        SNECT_CUDA(c, cudaMemsetAsync(c->csr_ptr, 0, sizeof(int32_t) * (I2 + 1), c->stream));
        c->max_degree = 0;
        return SNECT_OK;
    }
    uint64_t *keys = nullptr, *keys2 = nullptr;
    int32_t *vals = nullptr, *vals2 = nullptr;
    SNECT_CUDA(c, scratch_alloc(c, &keys, sizeof(uint64_t) * 2 * m));
    SNECT_CUDA(c, scratch_alloc(c, &keys2, sizeof(uint64_t) * 2 * m));
    SNECT_CUDA(c, scratch_alloc(c, &vals, sizeof(int32_t) * 2 * m));
    SNECT_CUDA(c, scratch_alloc(c, &vals2, sizeof(int32_t) * 2 * m));
    k_half_edges<<<ceil_div(m, 256), 256, 0, c->stream>>>(d_edges, d_w, m, I2, keys, vals, c->edges,
                                                          c->ew, gflag);
    c->launches++;
    int rc = sort_pairs(c, keys, vals, keys2, vals2, 2 * m, 32 + bits_for((uint64_t)I2));
    if (rc == SNECT_OK) {
        k_csr<<<ceil_div(2 * m + 1, 256), 256, 0, c->stream>>>(keys2, vals2, 2 * m, I2, c->ew,
                                                               c->csr_ptr, c->csr_col, c->csr_w,
                                                               gflag);
        c->launches++;
    }
    int32_t *d_maxdeg = nullptr;
    if (rc == SNECT_OK) {
        // the flag word's neighbour holds the maximum degree
        d_maxdeg = gflag + 1;
        cudaMemsetAsync(d_maxdeg, 0, sizeof(int32_t), c->stream);
        k_max_degree<<<ceil_div(I2, 256), 256, 0, c->stream>>>(c->csr_ptr, I2, d_maxdeg);
        c->launches++;
    }
    cudaFreeAsync(keys, c->stream);
    cudaFreeAsync(keys2, c->stream);
    cudaFreeAsync(vals, c->stream);
    cudaFreeAsync(vals2, c->stream);
    if (rc) return rc;
    SNECT_CUDA(c, cudaGetLastError());
    int32_t hf[2] = {0, 0};
    SNECT_CUDA(c, cudaMemcpyAsync(hf, gflag, sizeof(hf), cudaMemcpyDeviceToHost, c->stream));
    SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hf[0]) return fail(c, SNECT_EINVAL, "gene network:" + flag_message(hf[0]));
    c->max_degree = hf[1];
    if (c->max_degree > kHeavyDegree) {  // hub rows for the chunked network pass
        std::vector<int32_t> ptr((size_t)I2 + 1), heavy;
        SNECT_CUDA(c, cudaMemcpyAsync(ptr.data(), c->csr_ptr, sizeof(int32_t) * ptr.size(), cudaMemcpyDeviceToHost,
                                      c->stream));
        SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int32_t k = 0; k < I2; ++k)
            if (ptr[k + 1] - ptr[k] > kHeavyDegree) heavy.push_back(k);
        c->n_heavy = (int64_t)heavy.size();
        SNECT_CUDA(c, scratch_alloc(c, &c->heavy_rows, sizeof(int32_t) * heavy.size()));
        SNECT_CUDA(c, cudaMemcpyAsync(c->heavy_rows, heavy.data(), sizeof(int32_t) * heavy.size(),
                                      cudaMemcpyHostToDevice, c->stream));
        SNECT_CUDA(c, cudaStreamSynchronize(c->stream));  // the host vector goes out of scope
    }
    return SNECT_OK;
}

namespace {

// Fast mode: the visit order is cut into waves of c->wave entries, an even number of them
// (>= 2, so the moment buffers alternate across epochs); inside a wave the entries are grouped
// by platform (one tile of kFastTile entries holds one platform) and, inside a platform, by
// patient (the sweep sums a patient's neighbouring entries before adding them to its row).
// Gradients inside a wave all use the wave-start values, so the order inside a wave is free.
void fast_waves(Ctx *c) {
    const int64_t n = c->nnz;
    int64_t W = c->cfg.wave > 0 ? c->cfg.wave : std::min<int64_t>(kMaxWave, std::max<int64_t>(kMinWave, (n + 15) / 16));
    if (n) {
        int64_t nw = (n + W - 1) / W;
        nw = std::max<int64_t>(2, (nw + 1) & ~(int64_t)1);
        W = (n + nw - 1) / nw;
        c->n_waves = nw;
    } else {
        c->n_waves = 0;
    }
    c->wave = W;
    c->wave_tile.assign(1, 0);
    c->wave_len.clear();
}

// the per-wave (row, platform) entry table is kept when it is no larger than the entries
// themselves (else the sweep counts a wave's rows with atomics)
int64_t wave_table_cells(const Ctx *c) {
    const int64_t cells = c->n_waves * ((int64_t)c->d.I1 + c->d.I2) * c->d.I3;
    return (size_t)cells * sizeof(float) <= std::max<size_t>((size_t)64 << 20, sizeof(Rec) * (size_t)c->nnz) ? cells
                                                                                                               : 0;
}

int64_t fast_buckets(const Ctx *c) { return c->n_waves * (int64_t)c->d.I3 * c->d.I1; }

// The tile lists of the wave kernels from the entries per (wave, platform), h[w I3 + k]: wave
// w's platform-k segment starts where the previous one ends and is cut into tiles of
// kFastTile entries.  The host walks the segments; one kernel writes the tiles.
int build_fast_tiles(Ctx *c, const std::vector<int32_t> &h) {
    const int64_t n = c->nnz, W = c->wave;
    const int32_t I3 = c->d.I3;
    const int64_t S = c->n_waves * I3;
    std::vector<int32_t> seg((size_t)(3 * S + 1));  // starts | counts | first tiles (S + 1)
    std::vector<float> nk((size_t)S);
    int64_t tiles = 0;
    for (int64_t w = 0; w < c->n_waves; ++w) {
        int64_t pos = std::min<int64_t>(w * W, n);
        c->wave_len.push_back(std::min<int64_t>(W, n - pos));
        for (int32_t k = 0; k < I3; ++k) {
            const int64_t s = w * I3 + k, cnt = h[(size_t)s];
            seg[(size_t)s] = (int32_t)pos;
            seg[(size_t)(S + s)] = (int32_t)cnt;
            seg[(size_t)(2 * S + s)] = (int32_t)tiles;
            nk[(size_t)s] = (float)cnt;
            tiles += (cnt + kFastTile - 1) / kFastTile;
            pos += cnt;
        }
        c->wave_tile.push_back(tiles);
    }
    seg[(size_t)(3 * S)] = (int32_t)tiles;
    c->n_tiles = tiles;
    int32_t *d_seg = nullptr;
    const size_t tb = sizeof(int32_t) * (size_t)std::max<int64_t>(tiles, 1);
    SNECT_CUDA(c, scratch_alloc(c, &c->tile_start, tb));
    SNECT_CUDA(c, scratch_alloc(c, &c->tile_len, tb));
    SNECT_CUDA(c, scratch_alloc(c, &c->tile_k, tb));
    SNECT_CUDA(c, scratch_alloc(c, &c->wave_nk, sizeof(float) * nk.size()));
    SNECT_CUDA(c, scratch_alloc(c, &d_seg, sizeof(int32_t) * seg.size()));
    SNECT_CUDA(c, cudaMemcpyAsync(d_seg, seg.data(), sizeof(int32_t) * seg.size(), cudaMemcpyHostToDevice, c->stream));
    SNECT_CUDA(c, cudaMemcpyAsync(c->wave_nk, nk.data(), sizeof(float) * nk.size(), cudaMemcpyHostToDevice, c->stream));
    if (tiles) {
        k_build_tiles<<<ceil_div(tiles, 256), 256, 0, c->stream>>>(d_seg, (int32_t)S, I3, tiles, c->tile_start,
                                                                    c->tile_len, c->tile_k);
        c->launches++;
    }
    // (the host vectors may go out of scope: an asynchronous copy from pageable memory has
    // staged the data before it returns)
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(d_seg, c->stream);
    if (e != cudaSuccess) return fail(c, SNECT_ECUDA, std::string("tile lists: ") + cudaGetErrorString(e));
    return SNECT_OK;
}

}  // namespace

bool fast_counting_fits(Ctx *c) {
    fast_waves(c);
    const int64_t nb = fast_buckets(c);
    return c->nnz > 0 && nb <= INT32_MAX && nb <= std::max<int64_t>((int64_t)1 << 24, 2 * c->nnz);
}

// The radix-sort form of the fast mode's ordering, for problems whose bucket table would be
// too large for the counting form: the entries (packed in input order by prep_problem) are
// sorted stably by (wave, platform, patient), which keeps the visit order among one
// patient's entries.
int prep_fast_tiles(Ctx *c) {
    fast_waves(c);
    const int64_t n = c->nnz, W = c->wave;
    const int32_t I3 = c->d.I3;
    if (n == 0) return SNECT_OK;
    uint64_t *keys = nullptr, *keys2 = nullptr;
    int32_t *vals = nullptr, *vals2 = nullptr, *hist = nullptr;
    Rec *tmp = nullptr;
    SNECT_CUDA(c, scratch_alloc(c, &keys, sizeof(uint64_t) * n));
    SNECT_CUDA(c, scratch_alloc(c, &keys2, sizeof(uint64_t) * n));
    SNECT_CUDA(c, scratch_alloc(c, &vals, sizeof(int32_t) * n));
    SNECT_CUDA(c, scratch_alloc(c, &vals2, sizeof(int32_t) * n));
    SNECT_CUDA(c, scratch_alloc(c, &tmp, sizeof(Rec) * n));
    SNECT_CUDA(c, scratch_alloc(c, &hist, sizeof(int32_t) * c->n_waves * I3));
    const int bw = bits_for((uint64_t)(c->n_waves - 1)), bk = bits_for((uint64_t)(I3 - 1));
    int bi = bits_for((uint64_t)(c->d.I1 - 1));
    if (bw + bk + bi > 64) bi = 0;
    int rc;
    if (bw + bk + bi <= 32) {  // 32-bit keys: half the key traffic of the radix passes
        uint32_t *k32 = reinterpret_cast<uint32_t *>(keys), *k32b = reinterpret_cast<uint32_t *>(keys2);
        k_wave_keys32<<<ceil_div(n, 256), 256, 0, c->stream>>>(c->rec, n, W, bi, bk, k32, vals);
        c->launches++;
        rc = sort_pairs(c, k32, vals, k32b, vals2, n, bw + bk + bi);
    } else {
        k_wave_keys<<<ceil_div(n, 256), 256, 0, c->stream>>>(c->rec, n, W, bi, bk, keys, vals);
        c->launches++;
        rc = sort_pairs(c, keys, vals, keys2, vals2, n, bw + bk + bi);
    }
    if (rc == SNECT_OK) {
        k_permute<<<ceil_div(n, 256), 256, 0, c->stream>>>(c->rec, vals2, n, tmp);
        cudaMemcpyAsync(c->rec, tmp, sizeof(Rec) * n, cudaMemcpyDeviceToDevice, c->stream);
        cudaMemsetAsync(hist, 0, sizeof(int32_t) * c->n_waves * I3, c->stream);
        k_wave_hist<<<ceil_div(n, 1024), 1024, 0, c->stream>>>(c->rec, n, W, I3, hist);
        c->launches += 2;
        if (const int64_t cells = wave_table_cells(c)) {
            if (scratch_alloc(c, &c->wcnt, sizeof(float) * cells) == cudaSuccess) {
                cudaMemsetAsync(c->wcnt, 0, sizeof(float) * cells, c->stream);
                k_wave_row_counts<<<ceil_div(n, 256), 256, 0, c->stream>>>(c->rec, n, W, c->d.I1, c->d.I2, I3,
                                                                           c->wcnt);
                c->launches++;
            } else {
                cudaGetLastError();
                c->wcnt = nullptr;
            }
        }
    }
    std::vector<int32_t> h((size_t)c->n_waves * I3);
    if (rc == SNECT_OK) {
        cudaError_t e = cudaMemcpyAsync(h.data(), hist, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost,
                                        c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = fail(c, SNECT_ECUDA, std::string("wave histogram: ") + cudaGetErrorString(e));
    }
    cudaFreeAsync(keys, c->stream);
    cudaFreeAsync(keys2, c->stream);
    cudaFreeAsync(vals, c->stream);
    cudaFreeAsync(vals2, c->stream);
    cudaFreeAsync(tmp, c->stream);
    cudaFreeAsync(hist, c->stream);
    if (rc) return rc;
    return build_fast_tiles(c, h);
}

// The counting form (fast_counting_fits): packing, validation, the counts |Omega^{n,i}|, the
// wave table and the ordering in one read of the inputs, which stay where the caller has
// them when a kernel can read them there.
int prep_fast_entries(Ctx *c, const int32_t *idx, const float *val, bool vec, const std::function<int()> &between) {
    fast_waves(c);
    const int64_t n = c->nnz, W = c->wave, nb = fast_buckets(c), S = c->n_waves * c->d.I3;
    const Dims &d = c->d;
    for (int md = 0; md < 3; ++md)
        SNECT_CUDA(c, cudaMemsetAsync(c->cnt[md], 0, sizeof(int32_t) * (md == 0 ? d.I1 : (md == 1 ? d.I2 : d.I3)),
                                      c->stream));
    SNECT_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    if (n == 0) return SNECT_OK;
    Rec *tmp = nullptr;
    int32_t *rank = nullptr, *bcnt = nullptr, *first = nullptr;
    SNECT_CUDA(c, scratch_alloc(c, &tmp, sizeof(Rec) * n));
    SNECT_CUDA(c, scratch_alloc(c, &rank, sizeof(int32_t) * n));
    SNECT_CUDA(c, scratch_alloc(c, &bcnt, sizeof(int32_t) * nb));
    SNECT_CUDA(c, scratch_alloc(c, &first, sizeof(int32_t) * nb));
    SNECT_CUDA(c, cudaMemsetAsync(bcnt, 0, sizeof(int32_t) * nb, c->stream));
    if (const int64_t cells = wave_table_cells(c)) {
        if (scratch_alloc(c, &c->wcnt, sizeof(float) * cells) == cudaSuccess) {
            SNECT_CUDA(c, cudaMemsetAsync(c->wcnt, 0, sizeof(float) * cells, c->stream));
        } else {
            cudaGetLastError();
            c->wcnt = nullptr;
        }
    }
    PackFastArgs A{idx, val, n, W, d.I1, d.I2, d.I3, vec ? 1 : 0, tmp, rank, bcnt, c->wcnt,
                   c->cnt[0], c->cnt[1], c->cnt[2], c->flag};
    const int64_t bins = (int64_t)d.I1 + d.I2 + d.I3;
    const bool smem_hist = bins <= kCountBins;
    const size_t smem = sizeof(int32_t) * (size_t)(kPackWarps * 3 * kPackChunk + (smem_hist ? bins : 0));
    int sms = 0;
    SNECT_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const int64_t chunks = (n + kPackChunk - 1) / kPackChunk;
    const int grid = (int)std::min<int64_t>(ceil_div(chunks, kPackWarps), (int64_t)sms * (smem_hist ? 1 : 2));
    if (smem_hist) {
        SNECT_CUDA(c, cudaFuncSetAttribute(k_pack_fast<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_pack_fast<true><<<grid, kPackWarps * 32, smem, c->stream>>>(A);
    } else {
        SNECT_CUDA(c, cudaFuncSetAttribute(k_pack_fast<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_pack_fast<false><<<grid, kPackWarps * 32, smem, c->stream>>>(A);
    }
    c->launches++;
    SNECT_CUDA(c, cudaGetLastError());
    size_t tmp_bytes = 0;
    SNECT_CUDA(c, cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, bcnt, first, (int)nb, c->stream));
    void *scan_tmp = nullptr;
    SNECT_CUDA(c, scratch_alloc(c, &scan_tmp, tmp_bytes));
    SNECT_CUDA(c, cub::DeviceScan::ExclusiveSum(scan_tmp, tmp_bytes, bcnt, first, (int)nb, c->stream));
    c->launches++;
    cudaFreeAsync(scan_tmp, c->stream);
    // the caller's work that can run while the packing pass does (the host waits below)
    if (between) {
        const int r = between();
        if (r) {
            cudaFreeAsync(tmp, c->stream);
            cudaFreeAsync(rank, c->stream);
            cudaFreeAsync(bcnt, c->stream);
            cudaFreeAsync(first, c->stream);
            return r;
        }
    }
    // the validation flag, and each (wave, platform) segment's start: bucket (w, k, 0)'s
    std::vector<int32_t> seg((size_t)S);
    int32_t bad = 0;
    SNECT_CUDA(c, cudaMemcpyAsync(&bad, c->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    SNECT_CUDA(c, cudaMemcpy2DAsync(seg.data(), sizeof(int32_t), first, sizeof(int32_t) * (size_t)d.I1,
                                    sizeof(int32_t), (size_t)S, cudaMemcpyDeviceToHost, c->stream));
    k_bucket_scatter<<<ceil_div(n, 256), 256, 0, c->stream>>>(tmp, rank, first, n, W, d.I1, d.I3, c->rec);
    c->launches++;
    if (c->wcnt) {
        k_bucket_wave_rows<<<ceil_div(nb, 256), 256, 0, c->stream>>>(bcnt, nb, d.I1, d.I2, d.I3, c->wcnt);
        c->launches++;
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(tmp, c->stream);
    cudaFreeAsync(rank, c->stream);
    cudaFreeAsync(bcnt, c->stream);
    cudaFreeAsync(first, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SNECT_ECUDA, std::string("entry ordering: ") + cudaGetErrorString(e));
    if (bad) return fail(c, SNECT_EINVAL, "entries:" + flag_message(bad));
    std::vector<int32_t> h((size_t)S);
    for (int64_t s = 0; s < S; ++s) h[(size_t)s] = (s + 1 < S ? seg[(size_t)s + 1] : (int32_t)n) - seg[(size_t)s];
    return build_fast_tiles(c, h);
}

}  // namespace snect
