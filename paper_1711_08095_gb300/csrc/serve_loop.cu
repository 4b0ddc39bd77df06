// Continuous-batching service for fold-in + top-k queries (Eq. 9, Sec. 3.2.1).
//
// Requests (a new patient's observed (gene, platform, value) cells) are submitted from any
// host thread and copied into a host queue.  One scheduler thread admits queued requests,
// oldest first, whenever a slot is free and the request's device memory -- its cells and its
// fold-in partial sums -- can be carved out of the server's arena, one device allocation of
// exactly the memory budget made at start; requests that arrive while others are running are
// admitted as soon as slots and arena space free up.  So the budget bounds the device memory
// the requests in flight really use.  Each slot owns a CUDA stream, pinned staging buffers
// and small fixed buffers (the fold-in row, the scores, the top-k), so admitted requests
// overlap on the device.  Per request the slot stream runs: copy in -> cell check -> fold-in
// partials (fixed CTA partition) -> FP64 Cholesky solve -> cosine scores -> top-k -> copy out,
// then a host callback on that stream marks the slot finished and wakes the scheduler, which
// publishes the result, returns the arena space and admits the next requests (no polling).
// The kernels and their partition depend only on the request, so a request's result is the
// same alone and in any mix.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "common.cuh"
#include "serve.cuh"

namespace snect {

int ensure_wtable_for_serving(Ctx *c);  // api.cu
struct Server;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket;
    int64_t n = 0;            // cells
    char *pin = nullptr;      // pinned staging from the server's pool, laid out like the arena
                              // block (cells, then values at their aligned offset), or null:
    std::vector<int32_t> jk;  // then the cells and values are held here
    std::vector<float> val;
    int32_t k;
    Clock::time_point t_submit;
};

struct Result {
    int status = 0;  // 0 ok, else SNECT_E*
    std::vector<float> u;
    std::vector<int32_t> idx;
    std::vector<float> score;
    double latency_ms = 0.0;
    double queue_ms = 0.0;
};

// byte offsets of a request's results in a slot's result block
constexpr int64_t kResU = 0;                            // J1 <= 32 floats
constexpr int64_t kResIdx = kResU + 4 * kMaxRank;       // k <= 64 rows
constexpr int64_t kResScore = kResIdx + 4 * 64;         // their scores
constexpr int64_t kResFlag = kResScore + 4 * 64;        // cell flag, solve status
constexpr int64_t kResBytes = kResFlag + 8;

struct Slot {
    Server *srv = nullptr;
    int index = 0;
    cudaStream_t stream = nullptr;
    // pinned staging of a request: its cells, then its values at the offset they take in the
    // arena block, so that one copy moves both
    char *h_in = nullptr;
    // a request's results, one block on the device and its pinned copy (one copy back):
    // the fold-in row, the top-k rows and scores, the cell flag and the solve status
    char *h_res = nullptr, *d_res = nullptr;
    float *h_u = nullptr;  // views of h_res
    int32_t *h_idx = nullptr;
    float *h_score = nullptr;
    int32_t *h_flag = nullptr;
    int2 *d_jk = nullptr;  // carved from the arena per request
    float *d_val = nullptr, *d_part = nullptr;
    float *d_u = nullptr, *d_score = nullptr, *d_top_s = nullptr;
    int32_t *d_status = nullptr, *d_top_i = nullptr, *d_flag = nullptr;
    // the fold-in's cell flag: its solve moves it to d_flag and zeroes it for the next request
    int32_t *d_cell_flag = nullptr;
    uint8_t *d_taken = nullptr;
    bool busy = false;
    Request req;
    int64_t bytes = 0, arena_off = -1;
    Clock::time_point t_admit;
};

}  // namespace

struct Server {
    Ctx *c = nullptr;
    int32_t max_cells = 0;
    int64_t budget = 0;
    int64_t in_flight_bytes = 0;
    char *arena = nullptr;                 // the budget: one device allocation
    ArenaBlocks blocks;                    // the arena's free blocks (first fit, merged)
    std::vector<int> finished;             // slots whose stream work has completed
    bool kick = false;                     // a request was submitted since the scheduler last looked
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_submit, cv_done;
    std::deque<Request> queue;
    std::unordered_map<int64_t, Result> done;
    // pinned staging for submitted requests (4 per slot): submit copies a request's cells and
    // values into one on the submitting thread, so the scheduler only issues the copy to the
    // device; a request that finds none free keeps its own copy, staged at admission
    std::vector<char *> pin_free, pin_all;
    std::condition_variable cv_pin;  // a pinned buffer was returned (or the server stops)
    std::chrono::milliseconds pin_wait{100};
    std::atomic<bool> stop{false};
    std::thread worker;
    int64_t next_ticket = 1;
    int64_t admitted = 0, completed = 0, max_concurrent = 0;
    std::string err;
};

namespace {

constexpr int64_t kArenaAlign = 256;
// How long snect_serve_submit waits for a pinned staging buffer when all are in use (100 ms,
// or SNECT_SERVE_PIN_WAIT_MS in the environment at snect_serve_start): buffers come back as
// requests complete, so under load the wait is short and keeps every request on the pinned
// path; only a server that stops completing requests sends them to the fallback.
constexpr int kPinWaitMs = 100;

int64_t align_up(int64_t x) { return (x + kArenaAlign - 1) / kArenaAlign * kArenaAlign; }

// arena bytes of a request of n cells: its (gene, platform) pairs, values and the fold-in's
// per-CTA partial sums, each 256-byte aligned
int64_t request_bytes(const Ctx *c, int64_t n) {
    return align_up(n * (int64_t)sizeof(int2)) + align_up(n * (int64_t)sizeof(float)) +
           align_up(foldin_parts(n) * ((int64_t)c->d.J1 * c->d.J1 + c->d.J1) * (int64_t)sizeof(float));
}

void free_slot(Slot &s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaFreeHost(s.h_in);
    cudaFreeHost(s.h_res);
    cudaFree(s.d_res);
    cudaFree(s.d_score);
    cudaFree(s.d_taken);
    cudaFree(s.d_cell_flag);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot();
}

// the slot's stream, pinned staging for max_cells cells and its small fixed device
// buffers; the request's cells and partials come from the arena at admission
cudaError_t alloc_slot(Ctx *c, Slot &s, int32_t max_cells) {
    cudaError_t e;
#define TRY(x)                         \
    if ((e = (x)) != cudaSuccess) return e;
    TRY(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
    TRY(cudaMallocHost((void **)&s.h_in, align_up((int64_t)max_cells * sizeof(int2)) + sizeof(float) * max_cells));
    TRY(cudaMallocHost((void **)&s.h_res, kResBytes));
    TRY(cudaMalloc((void **)&s.d_res, kResBytes));
    s.h_u = reinterpret_cast<float *>(s.h_res + kResU);
    s.h_idx = reinterpret_cast<int32_t *>(s.h_res + kResIdx);
    s.h_score = reinterpret_cast<float *>(s.h_res + kResScore);
    s.h_flag = reinterpret_cast<int32_t *>(s.h_res + kResFlag);
    s.d_u = reinterpret_cast<float *>(s.d_res + kResU);
    s.d_top_i = reinterpret_cast<int32_t *>(s.d_res + kResIdx);
    s.d_top_s = reinterpret_cast<float *>(s.d_res + kResScore);
    s.d_flag = reinterpret_cast<int32_t *>(s.d_res + kResFlag);
    s.d_status = s.d_flag + 1;
    TRY(cudaMalloc((void **)&s.d_score, sizeof(float) * c->d.I1));
    TRY(cudaMalloc((void **)&s.d_taken, c->d.I1));
    TRY(cudaMalloc((void **)&s.d_cell_flag, sizeof(int32_t)));
    TRY(cudaMemset(s.d_cell_flag, 0, sizeof(int32_t)));
#undef TRY
    return cudaSuccess;
}

// runs on the CUDA driver's callback thread once a slot's stream work is done: no CUDA
// calls here, only the hand-over to the scheduler
void CUDART_CB on_slot_done(void *p) {
    Slot *s = static_cast<Slot *>(p);
    Server *S = s->srv;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->finished.push_back(s->index);
    }
    S->cv_submit.notify_all();
}

// launches one request on its slot (scheduler thread); its device buffers start at arena_off
cudaError_t launch_request(Ctx *c, Slot &s) {
    const Request &r = s.req;
    const int64_t n = r.n;
    char *base = s.srv->arena + s.arena_off;
    s.d_jk = reinterpret_cast<int2 *>(base);
    s.d_val = reinterpret_cast<float *>(base + align_up(n * (int64_t)sizeof(int2)));
    s.d_part = reinterpret_cast<float *>(base + align_up(n * (int64_t)sizeof(int2)) +
                                         align_up(n * (int64_t)sizeof(float)));
    // cells and values staged as they lie in the arena block: one copy in
    const int64_t val_off = align_up(n * (int64_t)sizeof(int2));
    const char *staged = r.pin;
    if (!staged) {
        std::memcpy(s.h_in, r.jk.data(), sizeof(int32_t) * 2 * n);
        std::memcpy(s.h_in + val_off, r.val.data(), sizeof(float) * n);
        staged = s.h_in;
    }
    cudaError_t e;
    // six calls: the copy in, four kernels (the cells are checked inside the fold-in's
    // partials), the copy back of every result; then the hand-over to the scheduler
    if ((e = cudaMemcpyAsync(base, staged, val_off + sizeof(float) * n, cudaMemcpyHostToDevice, s.stream))) return e;
    if ((e = launch_foldin(c, s.stream, s.d_jk, s.d_val, n, c->wtable, s.d_part, s.d_u, s.d_status, s.d_cell_flag,
                           s.d_flag)))
        return e;
    if ((e = launch_topk(c, s.stream, s.d_u, r.k, s.d_score, s.d_taken, s.d_top_i, s.d_top_s))) return e;
    if ((e = cudaMemcpyAsync(s.h_res, s.d_res, kResBytes, cudaMemcpyDeviceToHost, s.stream))) return e;
    return cudaLaunchHostFunc(s.stream, on_slot_done, &s);
}

void scheduler(Server *S) {
    Ctx *c = S->c;
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // retire the slots whose stream work has completed (handed over by on_slot_done)
        std::vector<int> fin;
        fin.swap(S->finished);
        for (int i : fin) {
            Slot &s = S->slots[i];
            Result res;
            const auto now = Clock::now();
            res.latency_ms = std::chrono::duration<double, std::milli>(now - s.req.t_submit).count();
            res.queue_ms = std::chrono::duration<double, std::milli>(s.t_admit - s.req.t_submit).count();
            // the stream holds only this request's work, all done but for the hand-over call,
            // which may still be returning (not ready); any other answer is a device error
            cudaError_t q = cudaStreamQuery(s.stream);
            if (q == cudaErrorNotReady) {
                cudaGetLastError();
                q = cudaSuccess;
            }
            if (q != cudaSuccess) {
                res.status = SNECT_ECUDA;
                S->err = std::string("serving: ") + cudaGetErrorString(q);
            } else if (s.h_flag[0] || s.h_flag[1]) {
                res.status = SNECT_EINVAL;
            } else {
                res.u.assign(s.h_u, s.h_u + c->d.J1);
                res.idx.assign(s.h_idx, s.h_idx + s.req.k);
                res.score.assign(s.h_score, s.h_score + s.req.k);
            }
            S->done[s.req.ticket] = std::move(res);
            if (s.req.pin) {
                S->pin_free.push_back(s.req.pin);
                S->cv_pin.notify_one();
            }
            s.req.pin = nullptr;
            s.busy = false;
            S->blocks.release(s.arena_off, s.bytes);
            s.arena_off = -1;
            S->in_flight_bytes -= s.bytes;
            S->completed++;
        }
        if (!fin.empty()) S->cv_done.notify_all();
        // admit: oldest first, while a slot is free and the arena has room
        while (!S->queue.empty()) {
            int free_slot_i = -1;
            for (size_t i = 0; i < S->slots.size(); ++i)
                if (!S->slots[i].busy) {
                    free_slot_i = (int)i;
                    break;
                }
            if (free_slot_i < 0) break;
            const int64_t need = request_bytes(c, S->queue.front().n);
            const int64_t off = S->blocks.alloc(need);  // first fit
            if (off < 0) break;  // wait for requests in flight to return their memory
            Slot &s = S->slots[free_slot_i];
            s.req = std::move(S->queue.front());
            S->queue.pop_front();
            s.busy = true;
            s.bytes = need;
            s.arena_off = off;
            s.t_admit = Clock::now();
            S->in_flight_bytes += need;
            S->admitted++;
            int64_t conc = 0;
            for (auto &x : S->slots) conc += x.busy;
            S->max_concurrent = std::max(S->max_concurrent, conc);
            lk.unlock();
            cudaError_t e = launch_request(c, s);
            lk.lock();
            if (e != cudaSuccess) {  // nothing of it will complete: retire it here
                Result res;
                res.status = SNECT_ECUDA;
                S->done[s.req.ticket] = std::move(res);
                S->err = std::string("serving launch: ") + cudaGetErrorString(e);
                cudaStreamSynchronize(s.stream);
                // a partial launch may have left cell flags for the next request on this slot
                cudaMemset(s.d_cell_flag, 0, sizeof(int32_t));
                if (s.req.pin) {
                    S->pin_free.push_back(s.req.pin);
                    S->cv_pin.notify_one();
                }
                s.req.pin = nullptr;
                s.busy = false;
                S->blocks.release(s.arena_off, s.bytes);
                s.arena_off = -1;
                S->in_flight_bytes -= s.bytes;
                S->cv_done.notify_all();
            }
        }
        bool any_busy = false;
        for (auto &s : S->slots) any_busy |= s.busy;
        if (S->stop.load() && S->queue.empty() && !any_busy) break;
        // sleep until a completion, a new submission (it may be admissible) or stop
        S->cv_submit.wait(lk, [&] { return !S->finished.empty() || S->kick || S->stop.load(); });
        S->kick = false;
    }
}

}  // namespace

}  // namespace snect

using namespace snect;

extern "C" {

int snect_serve_start(snect_ctx *h, int32_t n_slots, int64_t mem_budget_bytes, int32_t max_cells,
                      snect_server **out) {
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c || !out) return SNECT_EINVAL;
    *out = nullptr;
    if (n_slots < 1 || n_slots > 256) return fail(c, SNECT_EINVAL, "n_slots must be in [1, 256]");
    if (max_cells < 1) return fail(c, SNECT_EINVAL, "max_cells must be >= 1");
    if (mem_budget_bytes < request_bytes(c, max_cells))
        return fail(c, SNECT_EINVAL, "memory budget smaller than one largest request");
    int rc = ensure_wtable_for_serving(c);
    if (rc) return rc;
    SNECT_CUDA(c, cudaStreamSynchronize(c->stream));
    Server *S = new Server();
    S->c = c;
    S->max_cells = max_cells;
    S->budget = mem_budget_bytes;
    cudaError_t ea = cudaMalloc((void **)&S->arena, (size_t)mem_budget_bytes);
    if (ea != cudaSuccess) {
        delete S;
        cudaGetLastError();
        return fail(c, SNECT_ENOMEM, std::string("serving arena: ") + cudaGetErrorString(ea));
    }
    S->blocks.reset(mem_budget_bytes);
    S->slots.resize(n_slots);
    for (int i = 0; i < n_slots; ++i) {
        Slot &s = S->slots[i];
        cudaError_t e = alloc_slot(c, s, max_cells);
        s.srv = S;
        s.index = i;
        if (e != cudaSuccess) {
            for (auto &x : S->slots) free_slot(x);
            cudaFree(S->arena);
            delete S;
            cudaGetLastError();
            return fail(c, SNECT_ENOMEM, std::string("serving slot: ") + cudaGetErrorString(e));
        }
    }
    {
        const char *env = getenv("SNECT_SERVE_PIN_WAIT_MS");
        S->pin_wait = std::chrono::milliseconds(env ? std::max(0, atoi(env)) : kPinWaitMs);
    }
    // pinned request staging: up to 4 per slot (fewer if pinned memory runs short)
    const size_t pin_bytes = (size_t)(align_up((int64_t)max_cells * sizeof(int2)) + (int64_t)sizeof(float) * max_cells);
    for (int i = 0; i < 4 * n_slots; ++i) {
        char *b = nullptr;
        if (cudaMallocHost((void **)&b, pin_bytes) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        S->pin_all.push_back(b);
        S->pin_free.push_back(b);
    }
    S->worker = std::thread(scheduler, S);
    *out = reinterpret_cast<snect_server *>(S);
    return SNECT_OK;
}

int snect_serve_submit(snect_server *h, const int32_t *jk, const float *val, int64_t n, int32_t k,
                       int64_t *ticket) {
    Server *S = reinterpret_cast<Server *>(h);
    if (!S || !jk || !val || !ticket) return SNECT_EINVAL;
    if (n < 1 || n > S->max_cells) return SNECT_EINVAL;
    if (k < 1 || k > 64 || k > S->c->d.I1) return SNECT_EINVAL;
    Request r;
    r.t_submit = Clock::now();
    r.n = n;
    r.k = k;
    {  // a pooled buffer, waiting up to kPinWait for one to come back when all are taken
        std::unique_lock<std::mutex> lk(S->mu);
        if (!S->pin_all.empty())
            S->cv_pin.wait_for(lk, S->pin_wait, [S] { return !S->pin_free.empty() || S->stop.load(); });
        if (!S->pin_free.empty()) {
            r.pin = S->pin_free.back();
            S->pin_free.pop_back();
        }
    }
    if (r.pin) {  // staged as it will lie in the arena block, outside the lock
        std::memcpy(r.pin, jk, sizeof(int32_t) * 2 * n);
        std::memcpy(r.pin + align_up(n * (int64_t)sizeof(int2)), val, sizeof(float) * n);
    } else {
        r.jk.assign(jk, jk + 2 * n);
        r.val.assign(val, val + n);
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop.load()) {
            if (r.pin) S->pin_free.push_back(r.pin);
            return SNECT_EBUSY;
        }
        r.ticket = S->next_ticket++;
        *ticket = r.ticket;
        S->queue.push_back(std::move(r));
        S->kick = true;
    }
    S->cv_submit.notify_all();
    return SNECT_OK;
}

int snect_serve_poll(snect_server *h, int64_t ticket, int32_t wait, float *u_out, int32_t *idx_out,
                     float *score_out, double *latency_ms) {
    Server *S = reinterpret_cast<Server *>(h);
    if (!S) return SNECT_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    while (it == S->done.end()) {
        if (!wait) return SNECT_EBUSY;
        S->cv_done.wait_for(lk, std::chrono::milliseconds(50));
        it = S->done.find(ticket);
    }
    Result res = std::move(it->second);
    S->done.erase(it);
    lk.unlock();
    if (res.status) return res.status;
    if (u_out) std::memcpy(u_out, res.u.data(), sizeof(float) * res.u.size());
    if (idx_out) std::memcpy(idx_out, res.idx.data(), sizeof(int32_t) * res.idx.size());
    if (score_out) std::memcpy(score_out, res.score.data(), sizeof(float) * res.score.size());
    if (latency_ms) *latency_ms = res.latency_ms;
    return SNECT_OK;
}

int snect_serve_stats(snect_server *h, int64_t *admitted, int64_t *completed, int64_t *max_concurrent) {
    Server *S = reinterpret_cast<Server *>(h);
    if (!S) return SNECT_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (admitted) *admitted = S->admitted;
    if (completed) *completed = S->completed;
    if (max_concurrent) *max_concurrent = S->max_concurrent;
    return SNECT_OK;
}

int snect_serve_stop(snect_server *h) {
    Server *S = reinterpret_cast<Server *>(h);
    if (!S) return SNECT_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop.store(true);
    }
    S->cv_submit.notify_all();
    S->cv_pin.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &s : S->slots) free_slot(s);
    for (char *b : S->pin_all) cudaFreeHost(b);
    cudaFree(S->arena);
    delete S;
    return SNECT_OK;
}

}  // extern "C"
