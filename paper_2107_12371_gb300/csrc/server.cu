// server.cu -- continuous-batching CG solve server.
//
// Requests (a CSR system and a right-hand side, copied at submit) wait in a queue in arrival
// order.  A free slot admits the first queued request whose estimated device footprint fits
// in what the memory budget has left, so a large request waiting for memory does not hold up
// smaller ones behind it; a request that has been passed over kMaxBypass times is admitted
// next (admission waits for it), so none starves.  Its solve then runs on the slot's own CUDA
// stream, so the kernels of all admitted solves overlap on the GPU while new requests keep
// arriving.  A slot takes the next request the moment its solve finishes (no batch
// boundaries).  Each solve keeps its matrix, vectors and CG state in HBM until it completes;
// only x returns to the host.  Every per-problem kernel uses the same fixed grid and reduction
// order whatever else runs, so a result is bit-identical alone and in a mix.  Optionally the
// largest requests run on high-priority streams (spmv_server_set_priority_bytes).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace gb {
void release_matrix(spmv_matrix_t A);

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    std::vector<int32_t> rp, ci;
    std::vector<double> val, b, x;
    cg_options_t opt{};
    cg_result_t result{};
    spmv_status_t status = SPMV_ERR_PENDING;
    std::atomic<int> cancel{0};
    size_t est_bytes = 0;
    Clock::time_point t_submit, t_start, t_done;
    double setup_s = 0, solve_s = 0, teardown_s = 0;
    int bypassed = 0;  // times a later request was admitted before this one
    bool done = false;
};

// admissions of later requests that a queued request tolerates before it must go next
constexpr int kMaxBypass = 16;

// Conservative device footprint of one solve: CSR copy + sliced ELLPACK (+ FP32 values for
// mixed precision) + conversion temporaries + CG work vectors + b and x.
size_t estimate_bytes(int32_t n, int64_t nnz, bool mixed) {
    const double N = (double)n, Z = (double)nnz;
    double b = 4.0 * (N + 1) + 12.0 * Z          // CSR copy
               + 12.0 * Z * 1.1 + 8.0 * N / 32.0   // sliced ELLPACK, padding margin
               + 4.0 * (N + 1) + 12.0 * Z          // input copies during conversion
               + 5.0 * 8.0 * N                     // x r p q dinv
               + 2.0 * 8.0 * N;                    // b, x of the request
    if (mixed) b += 4.0 * Z + 4.0 * Z * 1.1 + 5.0 * 4.0 * N;
    return (size_t)b + (4u << 20);
}

}  // namespace
}  // namespace gb

struct spmv_server_s {
    size_t budget = 0;
    std::atomic<size_t> priority_bytes{0};  // requests at least this large run at high priority
    cudaMemPool_t pool = nullptr;  // stream-ordered allocations of the slots
    int max_slots = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<gb::Request *> queue;
    std::unordered_map<uint64_t, gb::Request *> all;
    size_t bytes_in_use = 0, peak = 0;
    int active = 0;
    uint64_t next_ticket = 1, submitted = 0, completed = 0, rejected = 0, cancelled = 0;
    std::vector<double> latencies;
    double setup_s = 0, solve_s = 0, teardown_s = 0;
    std::vector<std::thread> workers;
    bool stop = false;
};

namespace gb {
namespace {

// One solve on the slot's stream.  The handle, b and x live on the device only for its
// duration; they are freed stream-ordered on the slot's stream.
double since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

// The request a free slot admits now (queue end: none): the first in arrival order whose
// footprint fits the budget's remainder, not passing a request that was passed over
// kMaxBypass times.  Call with S->mu held.
std::deque<Request *>::iterator admissible(spmv_server_t S) {
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        if (S->bytes_in_use + (*it)->est_bytes <= S->budget) return it;
        if ((*it)->bypassed >= kMaxBypass) break;
    }
    return S->queue.end();
}

void run_request(Request *r, cudaStream_t st) {
    AllocStream scope(st);
    NvtxRange nvtx("server/request");
    auto t0 = Clock::now();
    spmv_options_t o;
    spmv_default_options(&o);
    o.precision = r->opt.mixed ? SPMV_PREC_DUAL : SPMV_PREC_FP64;
    o.reorder = SPMV_REORDER_NONE;
    spmv_matrix_t A = nullptr;
    r->status = spmv_create(r->n, r->n, r->nnz, r->rp.data(), r->nnz ? r->ci.data() : nullptr,
                            r->nnz ? r->val.data() : nullptr, 0, &o, st, &A);
    if (r->status != SPMV_OK) return;
    double *d_b = nullptr, *d_x = nullptr;
    const size_t vb = sizeof(double) * (size_t)(r->n > 0 ? r->n : 1);
    spmv_status_t s = cuda_status(gb_malloc_async((void **)&d_b, vb, st));
    if (s == SPMV_OK) s = cuda_status(gb_malloc_async((void **)&d_x, vb, st));
    if (s == SPMV_OK && r->n > 0)
        s = cuda_status(cudaMemcpyAsync(d_b, r->b.data(), vb, cudaMemcpyHostToDevice, st));
    if (s == SPMV_OK && r->cancel.load(std::memory_order_relaxed)) s = SPMV_ERR_CANCELLED;
    if (s == SPMV_OK) {
        cg_options_t co = r->opt;
        co.use_x0 = 0;
        // every solve runs as batches of separately launched kernels: those of different slot
        // streams overlap on the GPU, whereas cooperative launches (the persistent kernel)
        // from several streams were measured to run one after another.  All paths give
        // bit-identical results.
        co.persistent = 0;
        r->setup_s = since(t0);
        t0 = Clock::now();
        SolveControl ctl;
        ctl.cancel = &r->cancel;
        ctl.graphs = false;  // a request's handle solves once: launch its kernels directly
        s = cg_solve_ex(A, d_b, d_x, &co, &r->result, st, ctl);
        r->solve_s = since(t0);
        t0 = Clock::now();
        if (r->n > 0 && (s == SPMV_OK || s == SPMV_ERR_NOT_CONVERGED || s == SPMV_ERR_TIMEOUT)) {
            r->x.resize((size_t)r->n);
            spmv_status_t c =
                cuda_status(cudaMemcpyAsync(r->x.data(), d_x, vb, cudaMemcpyDeviceToHost, st));
            if (c == SPMV_OK) c = cuda_status(cudaStreamSynchronize(st));
            if (c != SPMV_OK) s = c;
        }
    }
    r->status = s;
    cudaStreamSynchronize(st);
    if (d_b) cudaFreeAsync(d_b, st);
    if (d_x) cudaFreeAsync(d_x, st);
    release_matrix(A);
    cudaStreamSynchronize(st);
    r->teardown_s = since(t0);
}

void worker(spmv_server_t S) {
    cudaSetDevice(S->device);
    AllocPool pool_scope(S->pool);
    // two streams per slot: the default priority, and the device's highest for the requests
    // the priority threshold names
    cudaStream_t st = nullptr, st_hi = nullptr;
    int least = 0, greatest = 0;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        st = nullptr;
    }
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&st_hi, cudaStreamNonBlocking, greatest) != cudaSuccess) {
        cudaGetLastError();
        st_hi = nullptr;
    }
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            S->cv.wait(lock, [&] { return S->stop || admissible(S) != S->queue.end(); });
            if (S->stop) break;
            auto it = admissible(S);
            for (auto q = S->queue.begin(); q != it; ++q) (*q)->bypassed += 1;
            r = *it;
            S->queue.erase(it);
            S->bytes_in_use += r->est_bytes;
            S->peak = std::max(S->peak, S->bytes_in_use);
            S->active += 1;
        }
        r->t_start = Clock::now();
        const size_t pb = S->priority_bytes.load(std::memory_order_relaxed);
        cudaStream_t use = (pb > 0 && r->est_bytes >= pb && st_hi) ? st_hi : st;
        if (use) run_request(r, use);
        else r->status = SPMV_ERR_CUDA;
        r->t_done = Clock::now();
        {
            std::lock_guard<std::mutex> lock(S->mu);
            S->bytes_in_use -= r->est_bytes;
            S->active -= 1;
            S->setup_s += r->setup_s;
            S->solve_s += r->solve_s;
            S->teardown_s += r->teardown_s;
            if (r->status == SPMV_ERR_CANCELLED) {
                S->cancelled += 1;
            } else {
                S->completed += 1;
                S->latencies.push_back(
                    std::chrono::duration<double>(r->t_done - r->t_submit).count());
            }
            r->result.status = r->status;
            r->done = true;
        }
        S->cv.notify_all();
    }
    if (st) cudaStreamDestroy(st);
    if (st_hi) cudaStreamDestroy(st_hi);
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" {

spmv_status_t spmv_server_create(size_t hbm_budget_bytes, int max_slots, spmv_server_t *out) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    if (hbm_budget_bytes == 0 || max_slots < 1 || max_slots > 256) return SPMV_ERR_INVALID_ARG;
    spmv_server_t S = new (std::nothrow) spmv_server_s();
    if (!S) return SPMV_ERR_OOM;
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return SPMV_ERR_CUDA;
    }
    // a pool of the server's own: freed blocks stay mapped up to the budget, so the next
    // requests reuse them instead of mapping fresh memory
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return SPMV_ERR_CUDA;
    }
    uint64_t keep = (uint64_t)hbm_budget_bytes;
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    try {
        for (int i = 0; i < max_slots; ++i) S->workers.emplace_back(worker, S);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lock(S->mu);
            S->stop = true;
        }
        S->cv.notify_all();
        for (auto &t : S->workers) t.join();
        cudaMemPoolDestroy(S->pool);
        delete S;
        return SPMV_ERR_OOM;
    }
    *out = S;
    return SPMV_OK;
}

spmv_status_t spmv_server_submit(spmv_server_t S, int32_t n, int64_t nnz, const int32_t *row_ptr,
                                 const int32_t *col_idx, const double *values, const double *b,
                                 const cg_options_t *opt, uint64_t *ticket) {
    if (!S || !ticket || n < 0 || nnz < 0 || nnz > INT32_MAX || !row_ptr) return SPMV_ERR_INVALID_ARG;
    if (n > 0 && !b) return SPMV_ERR_INVALID_ARG;
    if (nnz > 0 && (!col_idx || !values)) return SPMV_ERR_INVALID_ARG;
    Request *r = new (std::nothrow) Request();
    if (!r) return SPMV_ERR_OOM;
    try {
        r->rp.assign(row_ptr, row_ptr + (size_t)n + 1);
        r->ci.assign(col_idx, col_idx + nnz);
        r->val.assign(values, values + nnz);
        r->b.assign(b, b + n);
    } catch (...) {
        delete r;
        return SPMV_ERR_OOM;
    }
    r->n = n;
    r->nnz = nnz;
    cg_default_options(&r->opt);
    if (opt) r->opt = *opt;
    r->est_bytes = estimate_bytes(n, nnz, r->opt.mixed != 0);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (r->est_bytes > S->budget) {
            S->rejected += 1;
            delete r;
            return SPMV_ERR_BUDGET;
        }
        r->ticket = S->next_ticket++;
        S->submitted += 1;
        S->all[r->ticket] = r;
        S->queue.push_back(r);
        *ticket = r->ticket;
    }
    S->cv.notify_all();
    return SPMV_OK;
}

spmv_status_t spmv_server_poll(spmv_server_t S, uint64_t ticket, double *x_host,
                               cg_result_t *result) {
    if (!S) return SPMV_ERR_INVALID_ARG;
    Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        auto it = S->all.find(ticket);
        if (it == S->all.end()) return SPMV_ERR_INVALID_ARG;
        if (!it->second->done) return SPMV_ERR_PENDING;
        r = it->second;
        S->all.erase(it);
    }
    if (x_host && !r->x.empty() && r->status != SPMV_ERR_CANCELLED) std::memcpy(x_host, r->x.data(), sizeof(double) * r->x.size());
    if (result) *result = r->result;
    const spmv_status_t s = r->status;
    delete r;
    return s;
}

spmv_status_t spmv_server_set_priority_bytes(spmv_server_t S, size_t bytes) {
    if (!S) return SPMV_ERR_INVALID_ARG;
    S->priority_bytes.store(bytes, std::memory_order_relaxed);
    return SPMV_OK;
}

spmv_status_t spmv_server_get_stats(spmv_server_t S, spmv_server_stats_t *st) {
    if (!S || !st) return SPMV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->rejected = S->rejected;
    st->active_slots = S->active;
    st->queued = (int)S->queue.size();
    st->bytes_in_use = S->bytes_in_use;
    st->peak_bytes = S->peak;
    st->p50_latency_s = percentile(S->latencies, 0.50);
    st->p99_latency_s = percentile(S->latencies, 0.99);
    st->cancelled = S->cancelled;
    st->setup_s = S->setup_s;
    st->solve_s = S->solve_s;
    st->teardown_s = S->teardown_s;
    return SPMV_OK;
}

spmv_status_t spmv_server_cancel(spmv_server_t S, uint64_t ticket) {
    if (!S) return SPMV_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        auto it = S->all.find(ticket);
        if (it == S->all.end()) return SPMV_ERR_INVALID_ARG;
        Request *r = it->second;
        if (r->done) return SPMV_OK;
        auto q = std::find(S->queue.begin(), S->queue.end(), r);
        if (q != S->queue.end()) {
            // never started: it leaves the queue and is done at once
            S->queue.erase(q);
            r->status = SPMV_ERR_CANCELLED;
            r->result.status = SPMV_ERR_CANCELLED;
            r->t_start = r->t_done = Clock::now();
            r->done = true;
            S->cancelled += 1;
        } else {
            r->cancel.store(1, std::memory_order_relaxed);  // running: its host loop stops
        }
    }
    S->cv.notify_all();  // the queue head may have changed
    return SPMV_OK;
}

spmv_status_t spmv_server_destroy(spmv_server_t S) {
    if (!S) return SPMV_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto &t : S->workers) t.join();
    for (auto &kv : S->all) delete kv.second;
    cudaMemPoolDestroy(S->pool);  // every block was freed (and synchronised) by its worker
    delete S;
    return SPMV_OK;
}

}  // extern "C"
