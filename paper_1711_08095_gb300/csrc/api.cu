// C ABI entry points (include/snect.h): argument checks, device buffers, the epoch graph.
#include <mutex>
#include <math.h>

#include <algorithm>
#include <new>
#include <string>

#include "common.cuh"
#include "serve.cuh"

namespace snect {

namespace {
thread_local std::string g_init_error;

// A context's device buffers come from the library's per-device memory pool, in stream order on
// the context's stream: memory a destroyed context returns stays mapped in the pool, so the
// next context's set-up reuses it instead of mapping and unmapping hundreds of megabytes.
template <typename T>
int dmalloc(Ctx *c, T **p, int64_t count) {
    *p = nullptr;
    if (count <= 0) return SNECT_OK;
    cudaError_t e = scratch_alloc(c, p, sizeof(T) * (size_t)count);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, SNECT_ENOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
    }
    return SNECT_OK;
}

template <typename T>
void dfree(Ctx *c, T *&p) {
    if (p) cudaFreeAsync(p, c->stream);
    p = nullptr;
}

// The address through which a kernel on the context's device reads p: device memory of that
// device, managed memory, or page-locked host memory mapped into the device's address space
// (read over the host link); NULL for pageable host memory, which is copied instead.
template <typename T>
const T *kernel_readable(const Ctx *c, const T *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const bool ok = (a.type == cudaMemoryTypeDevice && a.device == c->device) || a.type == cudaMemoryTypeManaged ||
                    a.type == cudaMemoryTypeHost;
    return ok ? static_cast<const T *>(a.devicePointer) : nullptr;
}

// p is memory of the context's device (or managed memory): a kernel reads it in place
bool on_device(const Ctx *c, const void *p) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == c->device) || a.type == cudaMemoryTypeManaged;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// copies count elements from any memory into a fresh device buffer, ordered on the context's
// stream (or on its side stream)
template <typename T>
int stage(Ctx *c, T **dst, const T *src, int64_t count, bool side = false) {
    *dst = nullptr;
    if (count <= 0) return SNECT_OK;
    if (!src) return fail(c, SNECT_EINVAL, "null input pointer");
    cudaStream_t st = side ? c->side : c->stream;
    SNECT_CUDA(c, cudaMallocFromPoolAsync((void **)dst, sizeof(T) * (size_t)count, scratch_pool(c->device), st));
    SNECT_CUDA(c, cudaMemcpyAsync(*dst, src, sizeof(T) * (size_t)count, cudaMemcpyDefault, st));
    return SNECT_OK;
}

int copy_in(Ctx *c, float *dst, const float *src, int64_t count) {
    if (!src) return fail(c, SNECT_EINVAL, "null factor pointer");
    SNECT_CUDA(c, cudaMemcpyAsync(dst, src, sizeof(float) * count, cudaMemcpyDefault, c->stream));
    return SNECT_OK;
}

void free_all(Ctx *c) {
    if (c->epoch_exec) cudaGraphExecDestroy(c->epoch_exec);
    c->epoch_exec = nullptr;
    for (auto e : c->ev_begin) cudaEventDestroy(e);
    for (auto e : c->ev_end) cudaEventDestroy(e);
    for (auto e : c->aux_begin) cudaEventDestroy(e);
    for (auto e : c->aux_end) cudaEventDestroy(e);
    c->ev_begin.clear();
    c->ev_end.clear();
    c->aux_begin.clear();
    c->aux_end.clear();
    free_fast(c);
    dfree(c, c->rec);
    for (int m = 0; m < 3; ++m) {
        dfree(c, c->cnt[m]);
        dfree(c, c->U[m]);
        dfree(c, c->grp_pos[m]);
        dfree(c, c->grp_head[m]);
    }
    dfree(c, c->G);
    dfree(c, c->edges);
    dfree(c, c->ew);
    dfree(c, c->csr_ptr);
    dfree(c, c->csr_col);
    dfree(c, c->csr_w);
    dfree(c, c->heavy_rows);
    dfree(c, c->snap);
    dfree(c, c->gbuf);
    dfree(c, c->part);
    dfree(c, c->wtable);
    dfree(c, c->fold_part);
    dfree(c, c->q_jk);
    dfree(c, c->q_val);
    dfree(c, c->q_u);
    dfree(c, c->q_status);
    dfree(c, c->score);
    dfree(c, c->taken);
    dfree(c, c->top_i);
    dfree(c, c->top_s);
    dfree(c, c->lacc);
    dfree(c, c->flag);
    if (c->side) cudaStreamDestroy(c->side);
    c->side = nullptr;
    for (auto &e : c->side_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
}

int check_config(const snect_config *cfg, std::string *why) {
    for (int n = 0; n < 3; ++n) {
        if (cfg->I[n] < 1) return *why = "I_n must be >= 1", SNECT_EINVAL;
        if (cfg->J[n] < 1 || cfg->J[n] > kMaxRank) return *why = "J_n must be in [1, 32]", SNECT_EINVAL;
    }
    if ((int64_t)cfg->J[0] * cfg->J[1] * cfg->J[2] > kMaxCore)
        return *why = "J1*J2*J3 must be <= 5120", SNECT_EINVAL;
    if (!isfinite(cfg->lambda) || cfg->lambda < 0.f) return *why = "lambda must be finite and >= 0", SNECT_EINVAL;
    if (!isfinite(cfg->lambda_g) || cfg->lambda_g < 0.f)
        return *why = "lambda_g must be finite and >= 0", SNECT_EINVAL;
    if (!isfinite(cfg->lr) || cfg->lr <= 0.f) return *why = "lr must be finite and > 0", SNECT_EINVAL;
    if (cfg->batch < 0 || cfg->batch > kMaxBatch) return *why = "batch must be in [0, 4096]", SNECT_EINVAL;
    if (cfg->wave < 0) return *why = "wave must be >= 0", SNECT_EINVAL;
    if (cfg->precision != SNECT_FP32 && cfg->precision != SNECT_BF16 && cfg->precision != SNECT_BF16_TC)
        return *why = "precision must be SNECT_FP32, SNECT_BF16 or SNECT_BF16_TC", SNECT_EINVAL;
    if (cfg->precision != SNECT_FP32 &&
        (cfg->batch != 0 || (cfg->J[0] != 16 && cfg->J[0] != 32) || (cfg->J[1] != 16 && cfg->J[1] != 32)))
        return *why = "SNECT_BF16 and SNECT_BF16_TC need fast mode (batch = 0) and J1, J2 in {16, 32}", SNECT_EINVAL;
    return SNECT_OK;
}

int enqueue_det_epoch(Ctx *c) {
    const int64_t B = c->cfg.batch;
    for (int64_t b = 0; b < c->n_batches; ++b) {
        const int64_t first = b * B, len = std::min<int64_t>(B, c->nnz - first);
        const bool tm = c->time_launch(b, c->n_batches, len);
        if (tm) SNECT_CUDA(c, cudaEventRecordWithFlags(c->ev_begin[b], c->stream, cudaEventRecordExternal));
        SNECT_CUDA(c, launch_det_grad(c, first, len));
        if (tm) SNECT_CUDA(c, cudaEventRecordWithFlags(c->ev_end[b], c->stream, cudaEventRecordExternal));
        int rc = aux_event(c, 1, false);
        if (rc) return rc;
        SNECT_CUDA(c, launch_det_apply(c, first, len));
        if ((rc = aux_event(c, 1, true))) return rc;
    }
    return SNECT_OK;
}

int enqueue_epoch(Ctx *c) {
    int rc = c->cfg.batch > 0 ? enqueue_det_epoch(c) : enqueue_fast_epoch(c);
    if (rc) return rc;
    if ((rc = aux_event(c, 2, false))) return rc;
    SNECT_CUDA(c, launch_edge_pass(c));
    if ((rc = aux_event(c, 2, true))) return rc;
    SNECT_CUDA(c, refresh_bf16_rows(c));  // the pass moved gene rows
    return SNECT_OK;
}

// one epoch captured once into a CUDA graph (on a private stream: capture is not allowed on
// the legacy default stream), replayed on the context's stream
int build_epoch_graph(Ctx *c) {
    cudaStream_t orig = c->stream, cap = nullptr;
    SNECT_CUDA(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    c->stream = cap;
    const int64_t before = c->launches;
    c->timed_idx.clear();
    c->timed_len.clear();
    c->aux_cls.clear();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int rc = SNECT_OK;
    if (e == cudaSuccess) {
        rc = enqueue_epoch(c);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (rc == SNECT_OK && e2 != cudaSuccess) e = e2;
    }
    c->stream = orig;
    c->epoch_kernels = c->launches - before;
    c->launches = before;
    if (rc == SNECT_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->epoch_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (rc) return rc;
    if (e != cudaSuccess) {
        c->epoch_exec = nullptr;
        return fail(c, SNECT_ECUDA, std::string("epoch graph: ") + cudaGetErrorString(e));
    }
    return SNECT_OK;
}

int ensure_query_capacity(Ctx *c, int64_t n) {
    if (n <= c->q_cap) return SNECT_OK;
    dfree(c, c->q_jk);
    dfree(c, c->q_val);
    dfree(c, c->fold_part);
    c->q_cap = 0;
    int64_t cap = std::max<int64_t>(n, 1 << 16);
    int rc = dmalloc(c, &c->q_jk, cap);
    if (!rc) rc = dmalloc(c, &c->q_val, cap);
    const int64_t pf = foldin_parts(cap) * ((int64_t)c->d.J1 * c->d.J1 + c->d.J1);
    if (!rc) rc = dmalloc(c, &c->fold_part, pf);
    if (rc) return rc;
    c->q_cap = cap;
    c->fold_part_cap = pf;
    return SNECT_OK;
}

int ensure_wtable(Ctx *c) {
    if (c->wtable_version == c->param_version && c->wtable) return SNECT_OK;
    if (!c->wtable) {
        int rc = dmalloc(c, &c->wtable, (int64_t)c->d.I2 * c->d.I3 * c->d.J1);
        if (rc) return rc;
    }
    SNECT_CUDA(c, launch_wtable(c, c->wtable));
    c->wtable_version = c->param_version;
    return SNECT_OK;
}

}  // namespace

int ensure_wtable_for_serving(Ctx *c) { return ensure_wtable(c); }

int timing_events(Ctx *c, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        cudaEvent_t a = nullptr, b = nullptr;
        SNECT_CUDA(c, cudaEventCreate(&a));
        c->ev_begin.push_back(a);
        SNECT_CUDA(c, cudaEventCreate(&b));
        c->ev_end.push_back(b);
    }
    return SNECT_OK;
}

int aux_event(Ctx *c, int32_t cls, bool end) {
    if (c->timed != 2) return SNECT_OK;
    if (!end) {
        const size_t i = c->aux_cls.size();
        if (i >= c->aux_begin.size()) {  // made on demand, before the graph that records them
            cudaEvent_t a = nullptr, b = nullptr;
            SNECT_CUDA(c, cudaEventCreate(&a));
            SNECT_CUDA(c, cudaEventCreate(&b));
            c->aux_begin.push_back(a);
            c->aux_end.push_back(b);
        }
        c->aux_cls.push_back(cls);
        SNECT_CUDA(c, cudaEventRecordWithFlags(c->aux_begin[i], c->stream, cudaEventRecordExternal));
    } else {
        SNECT_CUDA(c, cudaEventRecordWithFlags(c->aux_end[c->aux_cls.size() - 1], c->stream,
                                               cudaEventRecordExternal));
    }
    return SNECT_OK;
}

int fail(Ctx *c, int code, const std::string &msg) {
    if (c)
        c->err = msg;
    else
        g_init_error = msg;
    return code;
}

cudaMemPool_t scratch_pool(int device) {
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices] = {};
    if (device < 0 || device >= kMaxDevices) {
        cudaMemPool_t def = nullptr;
        cudaDeviceGetDefaultMemPool(&def, device);
        return def;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        } else {  // the device's default pool
            cudaGetLastError();
            cudaDeviceGetDefaultMemPool(&pool, device);
        }
        pools[device] = pool;
    }
    return pools[device];
}

}  // namespace snect

using namespace snect;

extern "C" {

int snect_init(snect_ctx **out, const snect_config *cfg, const int32_t *idx, const float *val,
               int64_t nnz, const int32_t *edges, const float *w, int64_t m, const float *G0,
               const float *U1, const float *U2, const float *U3, void *stream) {
    if (!out || !cfg) return fail(nullptr, SNECT_EINVAL, "null argument");
    *out = nullptr;
    std::string why;
    if (check_config(cfg, &why)) return fail(nullptr, SNECT_EINVAL, why);
    if (nnz < 0 || m < 0) return fail(nullptr, SNECT_EINVAL, "negative size");
    if (nnz > INT32_MAX - 1 || 2 * m > INT32_MAX - 1) return fail(nullptr, SNECT_EINVAL, "too many entries or edges");
    if (cfg->batch == 0 && cfg->I[2] > kMaxPlatforms)
        return fail(nullptr, SNECT_EINVAL, "fast mode needs I3 <= 64");
    Ctx *c = new (std::nothrow) Ctx();
    if (!c) return fail(nullptr, SNECT_ENOMEM, "host allocation");
    c->cfg = *cfg;
    c->d = Dims{cfg->I[0], cfg->I[1], cfg->I[2], cfg->J[0], cfg->J[1], cfg->J[2]};
    c->nnz = nnz;
    c->m = m;
    c->PI = cfg->J[0] * cfg->J[1] * cfg->J[2];
    c->SJ = cfg->J[0] + cfg->J[1] + cfg->J[2];
    cudaGetDevice(&c->device);
    int rc = SNECT_OK;
    auto bail = [&](int code) {
        std::string msg = c->err;
        cudaStreamSynchronize(c->stream);
        free_all(c);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return fail(nullptr, code, msg);
    };
    c->stream = (cudaStream_t)stream;  // NULL: the default stream
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->side_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->side_ev[1], cudaEventDisableTiming) != cudaSuccess) {
        c->err = std::string("side stream: ") + cudaGetErrorString(cudaGetLastError());
        return bail(SNECT_ECUDA);
    }
    const Dims &d = c->d;
    if ((rc = dmalloc(c, &c->rec, nnz)) || (rc = dmalloc(c, &c->cnt[0], d.I1)) ||
        (rc = dmalloc(c, &c->cnt[1], d.I2)) || (rc = dmalloc(c, &c->cnt[2], d.I3)) ||
        (rc = dmalloc(c, &c->G, c->PI)) || (rc = dmalloc(c, &c->U[0], (int64_t)d.I1 * d.J1)) ||
        (rc = dmalloc(c, &c->U[1], (int64_t)d.I2 * d.J2)) ||
        (rc = dmalloc(c, &c->U[2], (int64_t)d.I3 * d.J3)) || (rc = dmalloc(c, &c->edges, m)) ||
        (rc = dmalloc(c, &c->ew, m)) || (rc = dmalloc(c, &c->csr_ptr, (int64_t)d.I2 + 1)) ||
        (rc = dmalloc(c, &c->csr_col, 2 * m)) || (rc = dmalloc(c, &c->csr_w, 2 * m)) ||
        (rc = dmalloc(c, &c->snap, (int64_t)d.I2 * d.J2)) || (rc = dmalloc(c, &c->lacc, 8)) ||
        (rc = dmalloc(c, &c->flag, 8)) || (rc = dmalloc(c, &c->q_u, kMaxRank)) ||
        (rc = dmalloc(c, &c->q_status, 1)) || (rc = dmalloc(c, &c->score, d.I1)) ||
        (rc = dmalloc(c, &c->taken, d.I1)) || (rc = dmalloc(c, &c->top_i, 64)) ||
        (rc = dmalloc(c, &c->top_s, 64)))
        return bail(rc);
    // inputs (any memory) -> device.  The fast mode orders its entries by counting when its
    // bucket table is small enough, in one pass that reads them where they are if a kernel can
    // (device memory, or pinned host memory over the host link); otherwise they are copied
    // to the device first.
    const bool counting = cfg->batch == 0 && fast_counting_fits(c);
    const int32_t *src_idx = counting ? kernel_readable(c, idx) : nullptr;
    const float *src_val = counting ? kernel_readable(c, val) : nullptr;
    int32_t *d_idx = nullptr, *d_edges = nullptr;
    float *d_val = nullptr, *d_w = nullptr;
    if ((!src_idx && (rc = stage(c, &d_idx, idx, nnz * 3))) || (!src_val && (rc = stage(c, &d_val, val, nnz))) ||
        (rc = stage(c, &d_edges, edges, m * 2)) || (rc = stage(c, &d_w, w, m)))
        return bail(rc);
    if (!src_idx) src_idx = d_idx;
    if (!src_val) src_val = d_val;
    // the gene network's set-up runs on the side stream, beside the packing of the entries
    // (which waits on the host link when they are in pinned host memory): it starts once the
    // network's inputs are staged and the stream waits for it before anything that uses them
    if (cudaEventRecord(c->side_ev[0], c->stream) != cudaSuccess) {
        c->err = "event record";
        return bail(SNECT_ECUDA);
    }
    auto graph_on_side = [&]() -> int {
        SNECT_CUDA(c, cudaStreamWaitEvent(c->side, c->side_ev[0], 0));
        cudaStream_t main_stream = c->stream;
        c->stream = c->side;
        const int r = prep_graph(c, d_edges, d_w);
        c->stream = main_stream;
        SNECT_CUDA(c, cudaEventRecord(c->side_ev[1], c->side));
        SNECT_CUDA(c, cudaStreamWaitEvent(c->stream, c->side_ev[1], 0));
        return r;
    };
    if (!rc) rc = copy_in(c, c->G, G0, c->PI);
    if (!rc) rc = copy_in(c, c->U[0], U1, (int64_t)d.I1 * d.J1);
    if (!rc) rc = copy_in(c, c->U[1], U2, (int64_t)d.I2 * d.J2);
    if (!rc) rc = copy_in(c, c->U[2], U3, (int64_t)d.I3 * d.J3);
    if (!rc) {
        if (counting) {
            rc = prep_fast_entries(c, src_idx, src_val, aligned16(src_idx) && aligned16(src_val), graph_on_side);
        } else {
            rc = prep_problem(c, src_idx, src_val);
            if (!rc) rc = graph_on_side();
        }
    }
    if (d_idx) cudaFreeAsync(d_idx, c->stream);
    if (d_val) cudaFreeAsync(d_val, c->stream);
    if (d_edges) cudaFreeAsync(d_edges, c->stream);
    if (d_w) cudaFreeAsync(d_w, c->stream);
    if (rc) return bail(rc);
    if (cfg->batch > 0) {
        c->n_batches = (nnz + cfg->batch - 1) / cfg->batch;
        int64_t gf = 0, pf = 0;
        det_scratch_floats(c, &gf, &pf);
        if ((rc = dmalloc(c, &c->grp_pos[0], nnz)) || (rc = dmalloc(c, &c->grp_pos[1], nnz)) ||
            (rc = dmalloc(c, &c->grp_pos[2], nnz)) || (rc = dmalloc(c, &c->grp_head[0], nnz)) ||
            (rc = dmalloc(c, &c->grp_head[1], nnz)) || (rc = dmalloc(c, &c->grp_head[2], nnz)) ||
            (rc = dmalloc(c, &c->gbuf, gf)) || (rc = dmalloc(c, &c->part, pf)))
            return bail(rc);
        if ((rc = prep_det_groups(c)) || (rc = timing_events(c, c->n_batches))) return bail(rc);
        cudaError_t e = det_init_attrs(c);
        if (e != cudaSuccess) {
            c->err = std::string("kernel attributes: ") + cudaGetErrorString(e);
            return bail(SNECT_ECUDA);
        }
    } else {
        if ((!counting && (rc = prep_fast_tiles(c))) || (rc = init_fast(c))) return bail(rc);
    }
    cudaError_t e = loss_init_attrs(c);
    if (e != cudaSuccess) {
        c->err = std::string("set-up: ") + cudaGetErrorString(e);
        return bail(SNECT_ECUDA);
    }
    // the epoch's CUDA graph is captured (on a stream of its own) while the set-up's last
    // kernels run; if that fails, the first snect_epoch captures it again and reports why
    if (build_epoch_graph(c) != SNECT_OK) {
        c->epoch_exec = nullptr;
        c->err.clear();
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("set-up: ") + cudaGetErrorString(e);
        return bail(SNECT_ECUDA);
    }
    *out = reinterpret_cast<snect_ctx *>(c);
    return SNECT_OK;
}

int snect_epoch(snect_ctx *h, int32_t n_epochs) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    if (n_epochs < 0) return fail(c, SNECT_EINVAL, "n_epochs must be >= 0");
    if (n_epochs == 0) return SNECT_OK;
    if (!c->epoch_exec) {
        int rc = build_epoch_graph(c);
        if (rc) return rc;
    }
    for (int32_t t = 0; t < n_epochs; ++t) {
        SNECT_CUDA(c, cudaGraphLaunch(c->epoch_exec, c->stream));
        c->launches += c->epoch_kernels;
    }
    c->param_version++;
    return SNECT_OK;
}

int snect_batches(snect_ctx *h, int64_t first, int64_t count) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    if (c->cfg.batch <= 0) return fail(c, SNECT_EINVAL, "snect_batches needs deterministic mode");
    if (first < 0 || count < 0 || first + count > c->n_batches)
        return fail(c, SNECT_EINVAL, "batch range outside [0, n_batches)");
    const int64_t B = c->cfg.batch;
    for (int64_t b = first; b < first + count; ++b) {
        const int64_t f = b * B, len = std::min<int64_t>(B, c->nnz - f);
        SNECT_CUDA(c, launch_det_grad(c, f, len));
        SNECT_CUDA(c, launch_det_apply(c, f, len));
    }
    c->param_version++;
    return SNECT_OK;
}

int snect_edge_pass(snect_ctx *h) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    SNECT_CUDA(c, launch_edge_pass(c));
    SNECT_CUDA(c, refresh_bf16_rows(c));
    c->param_version++;
    return SNECT_OK;
}

int snect_loss(snect_ctx *h, const int32_t *test_idx, const float *test_val, int64_t n_test,
               snect_loss_t *out) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c || !out) return SNECT_EINVAL;
    if (n_test < 0) return fail(c, SNECT_EINVAL, "n_test must be >= 0");
    SNECT_CUDA(c, cudaMemsetAsync(c->lacc, 0, sizeof(double) * 8, c->stream));
    SNECT_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    float *W = nullptr;
    SNECT_CUDA(c, loss_rows(c, &W));
    {
        cudaError_t e = launch_loss(c, c->rec, c->nnz, 0, W);
        if (e != cudaSuccess) {
            dfree(c, W);
            return fail(c, SNECT_ECUDA, cudaGetErrorString(e));
        }
    }
    int32_t *d_idx = nullptr;
    float *d_val = nullptr;
    int rc = SNECT_OK;
    if (n_test > 0) {
        // test entries in device memory are read in place; others are copied on the side
        // stream while the training entries' pass runs; the loss kernel checks them as it
        // reads them
        const int32_t *ti = on_device(c, test_idx) ? test_idx : nullptr;
        const float *tv = on_device(c, test_val) ? test_val : nullptr;
        if (!ti || !tv) {
            if ((!ti && (rc = stage(c, &d_idx, test_idx, n_test * 3, true))) ||
                (!tv && (rc = stage(c, &d_val, test_val, n_test, true))) ||
                (cudaEventRecord(c->side_ev[1], c->side) != cudaSuccess &&
                 (rc = fail(c, SNECT_ECUDA, "event record"))) ||
                (cudaStreamWaitEvent(c->stream, c->side_ev[1], 0) != cudaSuccess &&
                 (rc = fail(c, SNECT_ECUDA, "stream wait")))) {
                cudaStreamSynchronize(c->side);
                dfree(c, d_idx);
                dfree(c, d_val);
                dfree(c, W);
                return rc;
            }
        }
        cudaError_t e = launch_loss_checked(c, ti ? ti : d_idx, tv ? tv : d_val, n_test, 1, c->flag, W);
        if (e != cudaSuccess) rc = fail(c, SNECT_ECUDA, cudaGetErrorString(e));
    }
    if (rc == SNECT_OK) {
        cudaError_t e = launch_loss_reg_graph(c);
        if (e != cudaSuccess) rc = fail(c, SNECT_ECUDA, cudaGetErrorString(e));
    }
    double acc[8] = {0};
    int32_t bad = 0;
    if (rc == SNECT_OK) {
        cudaError_t e = cudaMemcpyAsync(acc, c->lacc, sizeof(acc), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, c->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = fail(c, SNECT_ECUDA, cudaGetErrorString(e));
    }
    dfree(c, d_idx);
    dfree(c, d_val);
    dfree(c, W);
    if (rc == SNECT_OK && bad) rc = fail(c, SNECT_EINVAL, "test " + entries_error(bad));
    if (rc) return rc;
    if (c->cfg.batch == 0) {  // a sweep wait that gave up (tensor-core completion, record copies)
        int32_t sweep_err = 0;
        SNECT_CUDA(c, cudaMemcpy(&sweep_err, c->flag + 3, sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (sweep_err) return fail(c, SNECT_ETIMEDOUT, "a completion wait timed out in the sweep");
    }
    const double lam = c->cfg.lambda, lg = c->cfg.lambda_g;
    out->data = 0.5 * acc[0];
    out->reg = 0.5 * lam * acc[2];
    out->graph = 0.5 * acc[3];
    out->total = out->data + out->reg + lg * out->graph;
    out->rmse_train = c->nnz ? sqrt(acc[0] / (double)c->nnz) : 0.0;
    out->rmse_test = n_test ? sqrt(acc[1] / (double)n_test) : 0.0;
    return SNECT_OK;
}

int snect_get_factors(snect_ctx *h, float *G, float *U1, float *U2, float *U3) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    const Dims &d = c->d;
    if (G) SNECT_CUDA(c, cudaMemcpyAsync(G, c->G, sizeof(float) * c->PI, cudaMemcpyDefault, c->stream));
    if (U1)
        SNECT_CUDA(c, cudaMemcpyAsync(U1, c->U[0], sizeof(float) * d.I1 * d.J1, cudaMemcpyDefault, c->stream));
    if (U2)
        SNECT_CUDA(c, cudaMemcpyAsync(U2, c->U[1], sizeof(float) * (int64_t)d.I2 * d.J2, cudaMemcpyDefault,
                                      c->stream));
    if (U3)
        SNECT_CUDA(c, cudaMemcpyAsync(U3, c->U[2], sizeof(float) * d.I3 * d.J3, cudaMemcpyDefault, c->stream));
    SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
    return SNECT_OK;
}

int snect_qr_post(snect_ctx *h, int32_t *skipped_modes) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    int skipped = 0;
    const int rc = qr_post(c, &skipped);
    if (skipped_modes) *skipped_modes = skipped;
    if (rc == SNECT_OK) SNECT_CUDA(c, refresh_bf16_rows(c));
    return rc;
}

int snect_set_factors(snect_ctx *h, const float *G, const float *U1, const float *U2, const float *U3) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    const Dims &d = c->d;
    if (G) SNECT_CUDA(c, cudaMemcpyAsync(c->G, G, sizeof(float) * c->PI, cudaMemcpyDefault, c->stream));
    if (U1)
        SNECT_CUDA(c, cudaMemcpyAsync(c->U[0], U1, sizeof(float) * d.I1 * d.J1, cudaMemcpyDefault, c->stream));
    if (U2)
        SNECT_CUDA(c, cudaMemcpyAsync(c->U[1], U2, sizeof(float) * (int64_t)d.I2 * d.J2, cudaMemcpyDefault,
                                      c->stream));
    if (U3)
        SNECT_CUDA(c, cudaMemcpyAsync(c->U[2], U3, sizeof(float) * d.I3 * d.J3, cudaMemcpyDefault, c->stream));
    if (U2) SNECT_CUDA(c, refresh_bf16_rows(c));
    SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->param_version++;
    return SNECT_OK;
}

int snect_foldin(snect_ctx *h, const int32_t *jk, const float *val, int64_t n, float *u_out) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c || !u_out) return SNECT_EINVAL;
    if (n < 1) return fail(c, SNECT_EINVAL, "a query needs at least one observed cell");
    if (!jk || !val) return fail(c, SNECT_EINVAL, "null query pointer");
    int rc = ensure_query_capacity(c, n);
    if (!rc) rc = ensure_wtable(c);
    if (rc) return rc;
    SNECT_CUDA(c, cudaMemcpyAsync(c->q_val, val, sizeof(float) * n, cudaMemcpyDefault, c->stream));
    SNECT_CUDA(c, cudaMemcpyAsync(c->q_jk, jk, sizeof(int2) * n, cudaMemcpyDefault, c->stream));
    SNECT_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    SNECT_CUDA(c, launch_foldin(c, c->stream, c->q_jk, c->q_val, n, c->wtable, c->fold_part, c->q_u,
                                c->q_status, c->flag, nullptr));
    int32_t status = 0, bad = 0;
    SNECT_CUDA(c, cudaMemcpyAsync(&status, c->q_status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    SNECT_CUDA(c, cudaMemcpyAsync(&bad, c->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    SNECT_CUDA(c, cudaMemcpyAsync(u_out, c->q_u, sizeof(float) * c->d.J1, cudaMemcpyDefault, c->stream));
    SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (bad) return fail(c, SNECT_EINVAL, "query cell out of range or value not finite");
    if (status) return fail(c, SNECT_EINVAL, "fold-in normal matrix is not positive definite");
    return SNECT_OK;
}

int snect_topk(snect_ctx *h, const float *u, int32_t k, int32_t *idx_out, float *score_out) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c || !u || !idx_out || !score_out) return SNECT_EINVAL;
    if (k < 1 || k > 64 || k > c->d.I1) return fail(c, SNECT_EINVAL, "k must be in [1, min(I1, 64)]");
    SNECT_CUDA(c, cudaMemcpyAsync(c->q_u, u, sizeof(float) * c->d.J1, cudaMemcpyDefault, c->stream));
    SNECT_CUDA(c, launch_topk(c, c->stream, c->q_u, k, c->score, c->taken, c->top_i, c->top_s));
    SNECT_CUDA(c, cudaMemcpyAsync(idx_out, c->top_i, sizeof(int32_t) * k, cudaMemcpyDefault, c->stream));
    SNECT_CUDA(c, cudaMemcpyAsync(score_out, c->top_s, sizeof(float) * k, cudaMemcpyDefault, c->stream));
    SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
    return SNECT_OK;
}

int snect_set_sweep_timing(snect_ctx *h, int32_t mode) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    if (mode < -1 || mode > 2) return fail(c, SNECT_EINVAL, "sweep timing mode must be -1, 0, 1 or 2");
    if (mode == c->timed) return SNECT_OK;
    c->timed = mode;
    if (c->epoch_exec) {  // the next epoch captures a graph with the new event nodes
        SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
        cudaGraphExecDestroy(c->epoch_exec);
        c->epoch_exec = nullptr;
    }
    c->timed_idx.clear();
    c->timed_len.clear();
    c->aux_cls.clear();
    return SNECT_OK;
}

int snect_sweep_times(snect_ctx *h, double *ms_total, int64_t *n_launches, int64_t *n_entries) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c || !ms_total || !n_launches) return SNECT_EINVAL;
    *ms_total = 0.0;
    *n_launches = 0;
    if (n_entries) *n_entries = 0;
    if (!c->epoch_exec) return SNECT_OK;  // no epoch has run with the current setting
    SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
    for (size_t t = 0; t < c->timed_idx.size(); ++t) {
        const int64_t i = c->timed_idx[t];
        float ms = 0.f;
        SNECT_CUDA(c, cudaEventElapsedTime(&ms, c->ev_begin[i], c->ev_end[i]));
        *ms_total += ms;
        ++*n_launches;
        if (n_entries) *n_entries += c->timed_len[t];
    }
    return SNECT_OK;
}

int snect_subtype(snect_ctx *h, const float *u, int64_t n, float *S, float *row_norm, float *platform_norm) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    if (n < 0) return fail(c, SNECT_EINVAL, "n must be >= 0");
    if (n == 0) return SNECT_OK;
    if (!u) return fail(c, SNECT_EINVAL, "null profile pointer");
    return run_subtype(c, u, n, S, row_norm, platform_norm);
}

int snect_kmeans(snect_ctx *h, int32_t k, const double *init, int32_t max_iter, int32_t *assign,
                 double *centroids, int32_t *n_updates, double *inertia) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    if (k < 1 || k > kmeans_max_clusters() || k > c->d.I1)
        return fail(c, SNECT_EINVAL, "k must be in [1, min(I1, 128)]");
    if (max_iter < 1) return fail(c, SNECT_EINVAL, "max_iter must be >= 1");
    if (!init) return fail(c, SNECT_EINVAL, "null initial centroids");
    return run_kmeans(c, k, init, max_iter, assign, centroids, n_updates, inertia);
}

int snect_hogwild_epoch(snect_ctx *h, const int32_t *order, int64_t n_items, int32_t P, int32_t n_epochs) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    if (c->cfg.batch <= 0)
        return fail(c, SNECT_EINVAL, "snect_hogwild_epoch needs a deterministic-mode context (batch > 0), "
                                     "which keeps the entries in the visit order");
    if (P < 1) return fail(c, SNECT_EINVAL, "P must be >= 1");
    if (n_items < 0 || n_items > INT32_MAX || n_epochs < 0) return fail(c, SNECT_EINVAL, "bad n_items or n_epochs");
    if (n_items == 0 || n_epochs == 0) return SNECT_OK;
    if (!order) return fail(c, SNECT_EINVAL, "null order");
    return run_hogwild(c, order, n_items, P, n_epochs);
}

int snect_wave_grads(snect_ctx *h, int64_t w, float *gA, float *gB, float *M, float *nA, float *nB,
                     int64_t *first, int64_t *count) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return SNECT_EINVAL;
    if (c->cfg.batch > 0) return fail(c, SNECT_EINVAL, "snect_wave_grads needs fast mode");
    if (w < 0 || w >= c->n_waves) return fail(c, SNECT_EINVAL, "wave index outside [0, n_waves)");
    const int rc = fast_wave_grads(c, w, gA, gB, M, nA, nB);
    if (rc) return rc;
    if (first) *first = w * c->wave;
    if (count) *count = c->wave_len[w];
    return SNECT_OK;
}

int snect_kernel_times(snect_ctx *h, double *ms, int64_t *n) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c || !ms || !n) return SNECT_EINVAL;
    for (int t = 0; t < 3; ++t) {
        ms[t] = 0.0;
        n[t] = 0;
    }
    if (!c->epoch_exec || c->timed != 2) return SNECT_OK;
    SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
    for (size_t t = 0; t < c->timed_idx.size(); ++t) {
        float x = 0.f;
        SNECT_CUDA(c, cudaEventElapsedTime(&x, c->ev_begin[c->timed_idx[t]], c->ev_end[c->timed_idx[t]]));
        ms[0] += x;
        ++n[0];
    }
    for (size_t t = 0; t < c->aux_cls.size(); ++t) {
        float x = 0.f;
        SNECT_CUDA(c, cudaEventElapsedTime(&x, c->aux_begin[t], c->aux_end[t]));
        ms[c->aux_cls[t]] += x;
        ++n[c->aux_cls[t]];
    }
    return SNECT_OK;
}

int64_t snect_launch_count(const snect_ctx *h) {
    const Ctx *c = reinterpret_cast<const Ctx *>(h);
    return c ? c->launches.load() : 0;
}

const char *snect_last_error(const snect_ctx *h) {
    const Ctx *c = reinterpret_cast<const Ctx *>(h);
    return c ? c->err.c_str() : g_init_error.c_str();
}

void snect_destroy(snect_ctx *h) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
