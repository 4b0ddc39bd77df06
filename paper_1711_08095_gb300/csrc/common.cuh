// Internal declarations shared by the translation units of libsnect.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <functional>
#include <atomic>
#include <string>
#include <vector>

#include "../../include/snect.h"

namespace snect {

constexpr int kMaxDevices = 64;  // devices with a library scratch pool
constexpr int kMaxRank = 32;      // largest J_n
constexpr int kMaxCore = 5120;    // largest J1*J2*J3
constexpr int kMaxBatch = 4096;   // largest deterministic mini-batch
constexpr int kMaxPlatforms = 64; // largest I3 in fast mode (platform rows are dense there)
constexpr int kHeavyDegree = 128;  // network rows above this degree take the chunked pass

// One observed entry, 16 bytes: (i, j, k) and the value's bits.  One vector load per entry.
struct __align__(16) Rec {
    int32_t i, j, k;
    float x;
};

struct Dims {
    int32_t I1, I2, I3;
    int32_t J1, J2, J3;
};

struct Ctx {
    snect_config cfg{};
    Dims d{};
    int64_t nnz = 0, m = 0;
    int32_t PI = 0, SJ = 0;  // J1*J2*J3 and J1+J2+J3
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // a second stream for set-up and objective work that overlaps work on `stream`, and the
    // events that order the two (created with the context)
    cudaStream_t side = nullptr;
    cudaEvent_t side_ev[2] = {nullptr, nullptr};
    int device = 0;
    std::atomic<int64_t> launches{0};
    std::string err;

    // problem
    Rec *rec = nullptr;       // nnz entries in visit order
    int32_t *cnt[3] = {};     // |Omega^{n,i}| per mode (training entries)
    float *G = nullptr;       // core
    float *U[3] = {};         // factors
    // gene network
    int2 *edges = nullptr;    // m undirected edges
    float *ew = nullptr;      // m weights
    int32_t *csr_ptr = nullptr;  // I2 + 1
    int32_t *csr_col = nullptr;  // 2m neighbours, ascending within a row
    float *csr_w = nullptr;      // 2m weights
    float *snap = nullptr;       // I2*J2 snapshot for the network pass
    int32_t max_degree = 0;
    int32_t *heavy_rows = nullptr;  // genes of degree > kHeavyDegree (one CTA each in the pass)
    int64_t n_heavy = 0;
    // deterministic mode
    int64_t n_batches = 0;
    int32_t *grp_pos[3] = {};    // per mode: entry positions grouped by (batch, row), stable
    uint8_t *grp_head[3] = {};   // 1 where a row segment starts
    float *gbuf = nullptr;       // scratch: batch * SJ per-entry row gradients
    float *part = nullptr;       // scratch: per-CTA core partial sums
    int32_t grad_blocks = 0;     // CTAs of the gradient kernel per full batch
    // fast mode
    int64_t n_waves = 0;
    int64_t wave = 0;               // entries per wave
    int64_t n_tiles = 0;
    int32_t *tile_start = nullptr;  // per tile: first entry (entries grouped by platform per wave)
    int32_t *tile_len = nullptr;
    int32_t *tile_k = nullptr;
    int32_t *tile_ctr = nullptr;    // per wave: tiles claimed so far
    std::vector<int64_t> wave_tile; // first tile of each wave (n_waves + 1)
    std::vector<int64_t> wave_len;  // entries of each wave
    float *wave_nk = nullptr;       // per wave and platform: entries (n_waves * I3)
    float *macc = nullptr;          // per platform: sum over the wave of r a b^T (I3 * J1 * J2)
    float *gram = nullptr;          // moments of U1, U2 (two buffers of gram_stride) + eigenvectors
    int64_t gram_stride = 0;
    int64_t gram_floats = 0;        // the whole gram buffer (moments, eigenbases, platform systems)
    int32_t fast_grid = 0;          // persistent CTAs of the wave kernel (occupancy)
    float *gacc[2] = {};            // per patient / gene row: gradient sums + entries per platform
    // entries per (wave, row, platform), fixed at set-up: n_waves x (I1 + I2) x I3, patients
    // before genes in each wave (null: the sweep counts with atomics instead)
    float *wcnt = nullptr;
    float *curv = nullptr;          // platform curvatures of the row steps (two buffers)
    // which sweep kernel runs (1 lane-group FP32, 2 lane-group with BF16 gene rows, 0 the
    // warp-per-unit or per-entry kernel, -1 the tensor-core kernel) and, for 2, the BF16
    // copy of the gene factor it gathers from (kept current by every writer of U2)
    int32_t sweep_kind = 0;
    __nv_bfloat16 *U2h = nullptr;
    // fold-in / top-k
    float *wtable = nullptr;        // I2*I3*J1: w_jk = G x2 u2_j x3 u3_k
    int64_t param_version = 0;      // bumped whenever G or a factor may have changed
    int64_t wtable_version = -1;
    float *fold_part = nullptr;     // scratch: per-CTA Gram partials of one query
    int64_t fold_part_cap = 0;      // floats
    int2 *q_jk = nullptr;           // staging for one query's cells
    float *q_val = nullptr;
    int64_t q_cap = 0;
    float *q_u = nullptr;           // kMaxRank
    int32_t *q_status = nullptr;
    float *score = nullptr;         // I1
    uint8_t *taken = nullptr;       // I1
    int32_t *top_i = nullptr;       // 64
    float *top_s = nullptr;         // 64
    // loss
    double *lacc = nullptr;         // 8 doubles
    // CUDA graph of one epoch
    cudaGraphExec_t epoch_exec = nullptr;
    int64_t epoch_kernels = 0;      // kernels in one replay of the graph
    // events around the sweep launches of one epoch (recorded inside the epoch graph); each
    // recorded event is a graph node that costs several microseconds of the epoch, so only
    // the launches chosen by `timed` carry them (0: none, 1: the middle one, -1: all)
    std::vector<cudaEvent_t> ev_begin, ev_end;
    int32_t timed = 0;
    std::vector<int64_t> timed_idx, timed_len;  // event pairs recorded by the epoch graph, entries

    // true if launch i of n_launches carries timing events; records it with its entries
    // (timed == 2 times every sweep launch, like -1, and the other kernels as well)
    bool time_launch(int64_t i, int64_t n_launches, int64_t entries) {
        if (timed == 0 || (timed == 1 && i != n_launches / 2)) return false;
        timed_idx.push_back(i);
        timed_len.push_back(entries);
        return true;
    }
    // timed == 2: event pairs around the other kernels of the epoch (wave ends or the
    // deterministic apply kernels: class 1; the network pass: class 2), in recording order
    std::vector<cudaEvent_t> aux_begin, aux_end;
    std::vector<int32_t> aux_cls;
    // error word written by kernels (validation)
    int32_t *flag = nullptr;
};

// error helpers ---------------------------------------------------------------------------
int fail(Ctx *c, int code, const std::string &msg);

// Stream-ordered scratch for set-up and queries comes from a memory pool the library owns on
// each device, which keeps the memory it has handed out mapped after it is freed (its
// high-water mark stays reserved until the process exits), so repeated set-ups do not pay
// to map and unmap hundreds of megabytes.
cudaMemPool_t scratch_pool(int device);
template <typename T>
cudaError_t scratch_alloc(Ctx *c, T **p, size_t bytes) {
    return cudaMallocFromPoolAsync((void **)p, bytes, scratch_pool(c->device), c->stream);
}
#define SNECT_CUDA(c, call)                                                                  \
    do {                                                                                     \
        cudaError_t e__ = (call);                                                            \
        if (e__ != cudaSuccess)                                                              \
            return ::snect::fail((c), SNECT_ECUDA,                                           \
                                 std::string(#call) + ": " + cudaGetErrorString(e__));       \
    } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// launchers (each returns a CUDA error code; they increment c->launches) ------------------
cudaError_t launch_det_grad(Ctx *c, int64_t first, int64_t len);
cudaError_t launch_det_apply(Ctx *c, int64_t first, int64_t len);
cudaError_t launch_edge_pass(Ctx *c);
int qr_post(Ctx *c, int *skipped);

// one problem's network pass, for the batched pass (all problems of a batch in three
// launches: snapshot, light rows, hub rows; blockIdx.y = problem)
struct EdgeArgs {
    const int32_t *ptr, *col;
    const float *w;
    float *snap, *U2;
    int32_t I2, J2;  // I2 = 0: no network pass for this problem
    float step;
    const int32_t *heavy;
    int64_t n_heavy;
};
EdgeArgs make_edge_args(const Ctx *c);
cudaError_t launch_batch_edge_pass(const EdgeArgs *d_args, int32_t P, int64_t max_cells, int64_t max_heavy,
                                   cudaStream_t st, int64_t *launches);
// the loss kernels' per-(patient, platform) rows W[i][k] = (G x3 c_k)^T a_i, when there are
// no more of them than training entries (*W from the pool, freed by the caller; NULL
// otherwise, and the kernels form the products themselves)
cudaError_t loss_rows(Ctx *c, float **W);
cudaError_t launch_loss(Ctx *c, const Rec *recs, int64_t n, int which, const float *W);
// the same over the caller's entries (idx n x 3, val n, device memory), checked on the way:
// bit 1 of *flag for an index outside the tensor (the entry is left out), bit 2 for a
// non-finite value
cudaError_t launch_loss_checked(Ctx *c, const int32_t *idx, const float *val, int64_t n, int which,
                                int32_t *flag, const float *W);
std::string entries_error(int32_t flag);  // the message for such flag bits
cudaError_t launch_loss_reg_graph(Ctx *c);

// prep (prep.cu)
int prep_problem(Ctx *c, const int32_t *d_idx, const float *d_val);
int prep_graph(Ctx *c, const int32_t *d_edges, const float *d_w);
int prep_det_groups(Ctx *c);
int prep_fast_tiles(Ctx *c);       // prep.cu: groups each wave's entries by platform, tiles
// fast mode: true when the set-up can order the entries by counting (sets the wave size);
// prep_fast_entries then packs, validates, counts and orders them in one read of the inputs
bool fast_counting_fits(Ctx *c);
// (between: called once the packing pass is queued and before the host waits for it)
int prep_fast_entries(Ctx *c, const int32_t *idx, const float *val, bool vec, const std::function<int()> &between);
int init_fast(Ctx *c);             // sweep_fast.cu: buffers and launch shape of the fast sweep
int enqueue_fast_epoch(Ctx *c);
cudaError_t refresh_bf16_rows(Ctx *c);  // U2 -> its BF16 copy, when the context keeps one
// the entry sweep of one wave alone, its accumulators copied out (snect_wave_grads)
int fast_wave_grads(Ctx *c, int64_t w, float *gA, float *gB, float *M, float *nA, float *nB);
void free_fast(Ctx *c);
// downstream analyses (analysis.cu) and the lock-free form of Alg. 1 (hogwild.cu)
int run_subtype(Ctx *c, const float *u, int64_t n, float *S, float *row_norm, float *plat_norm);
int run_kmeans(Ctx *c, int32_t k, const double *init, int32_t max_iter, int32_t *assign, double *centroids,
               int32_t *n_updates, double *inertia);
int kmeans_max_clusters();
int run_hogwild(Ctx *c, const int32_t *order, int64_t n_items, int32_t P, int32_t n_epochs);
constexpr int kFastTile = 256;     // entries per tile (one per thread of the wave kernel)
constexpr int64_t kMinWave = 4096;      // default wave: nnz/16 clamped to [kMinWave, kMaxWave]
constexpr int64_t kMaxWave = 1 << 21;
int det_scratch_floats(const Ctx *c, int64_t *gbuf_floats, int64_t *part_floats);
cudaError_t det_init_attrs(Ctx *c);
cudaError_t loss_init_attrs(Ctx *c);
int timing_events(Ctx *c, int64_t n);  // makes n begin/end event pairs
// timed == 2: records the begin (end = false) or end event of the next kernel of class cls
// around which the epoch graph carries timing events; no-op otherwise
int aux_event(Ctx *c, int32_t cls, bool end);
int pack_records(Ctx *c, const int32_t *d_idx, const float *d_val, int64_t n, Rec *out,
                 bool check_ranges, int32_t n_modes);

}  // namespace snect
