// common.cuh -- shared host/device definitions of the GB300 SpMV library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>

#include <nvtx3/nvToolsExt.h>

#include "../../include/spmv.h"

namespace gb {

// NVTX range for profilers (header-only NVTX v3; no cost when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Number of SMs and other device facts, queried once per device.
struct DeviceFacts {
    int device = -1;
    int sm_count = 0;
    int max_smem_optin = 0;  // bytes of shared memory a CTA may opt into
    int l2_bytes = 0;
};
const DeviceFacts &device_facts();

// Dependent load rounds of a row of w stored entries read in blocks of u with the rest one at a
// time: the kernels that keep u entries in flight choose u by this count for the widest slice.
constexpr int load_rounds(int w, int u) { return w / u + w % u; }

// Status from a CUDA error code.
inline spmv_status_t cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SPMV_OK;
    if (e == cudaErrorMemoryAllocation) return SPMV_ERR_OOM;
    return SPMV_ERR_CUDA;
}

#define GB_CUDA(expr)                                            \
    do {                                                         \
        cudaError_t gb_e_ = (expr);                              \
        if (gb_e_ != cudaSuccess) return ::gb::cuda_status(gb_e_); \
    } while (0)

#define GB_TRY(expr)                            \
    do {                                        \
        spmv_status_t gb_s_ = (expr);           \
        if (gb_s_ != SPMV_OK) return gb_s_;     \
    } while (0)

#define GB_LAUNCHED() GB_CUDA(cudaGetLastError())

// Stream on which handle buffers are allocated and freed (stream-ordered allocator), set for
// the duration of an entry point by AllocStream.  Stream-ordered frees never synchronize the
// whole device, so solves running concurrently on other streams are not stalled.
cudaStream_t &alloc_stream();
struct AllocStream {
    cudaStream_t saved;
    explicit AllocStream(cudaStream_t s) : saved(alloc_stream()) { alloc_stream() = s; }
    ~AllocStream() { alloc_stream() = saved; }
};

// Memory pool that stream-ordered allocations come from, set per host thread by AllocPool
// (nullptr: the device's default pool).  The server gives its slot threads a pool of its own
// whose release threshold keeps freed memory mapped, so that allocations of later requests
// neither map nor unmap device memory.
cudaMemPool_t &alloc_pool();
struct AllocPool {
    cudaMemPool_t saved;
    explicit AllocPool(cudaMemPool_t p) : saved(alloc_pool()) { alloc_pool() = p; }
    ~AllocPool() { alloc_pool() = saved; }
};
inline cudaError_t gb_malloc_async(void **p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = alloc_pool();
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
}

// A device allocation owned by the handle.
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    spmv_status_t alloc(size_t count, size_t *tally) {
        release(tally);
        if (count == 0) count = 1;
        cudaError_t e = gb_malloc_async((void **)&p, count * sizeof(T), alloc_stream());
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return cuda_status(e);
        }
        n = count;
        if (tally) *tally += count * sizeof(T);
        return SPMV_OK;
    }
    void release(size_t *tally) {
        if (p) {
            cudaFreeAsync(p, alloc_stream());
            if (tally) *tally -= n * sizeof(T);
        }
        p = nullptr;
        n = 0;
    }
};

// Device scalars of one CG recurrence (written by the last CTA of a reduction).
struct CgScalars {
    double alpha, beta, rho, rr, bb, tol2, s, inv_s;
    int done;   // 0 running, 1 converged, 2 iteration cap, 3 breakdown, 4 timeout
    int iters;
    int max_iter;
    int pad;
    unsigned tickets[4];
    unsigned bar_count, bar_gen;    // grid barrier of the persistent kernel
    long long budget_ns;            // persistent kernel: wall-clock budget (0 = none)
};

// Work vectors of a CG solve (allocated on first use, kept with the handle).
struct CgWork {
    DevBuf<double> x, r, p, q, dinv;
    DevBuf<float> r32, p32, q32, d32, dinv32;
    DevBuf<double> part;        // per-CTA partial sums
    DevBuf<double> scal;        // two CgScalars blocks (outer / inner)
    DevBuf<int> flags;          // status flags
    int h_flags[16] = {};       // host mirrors (read back synchronously; no pinned buffers)
    CgScalars h_scal[2] = {};
    int part_len = 0;
    int pq_len = 0;  // leading p.q partials: one per CTA of the product grid (cg_pq_grid)
    bool ready = false;
    bool mixed_ready = false;
    cudaGraphExec_t graph64 = nullptr, graph32 = nullptr, graph_pers = nullptr;
    int graph64_iters = 0, graph32_iters = 0;
    int pers_grid = 0;
};

struct McgWork;  // multi-right-hand-side CG work (mcg.cu)

}  // namespace gb

struct spmv_matrix_s {
    cudaStream_t stream = nullptr;  // creation stream: buffers are allocated / freed on it
    int32_t n = 0;       // rows
    int32_t n_cols = 0;  // columns (== n unless the matrix is rectangular)
    int64_t nnz = 0;
    spmv_options_t opt{};
    int S = 64;        // rows per slice
    int block = 256;   // threads per CTA
    int variant = SPMV_VARIANT_SELL;
    int window_words = 0;
    int index_bits = 32;  // 16: sell_col16 holds offsets from the slice's col_start
    int32_t bandwidth = 0;
    int32_t max_span = 0;
    int32_t n_slices = 0;
    int32_t max_width = 0;  // widest slice: its stored entries per row
    int64_t sell_entries = 0;
    size_t bytes = 0;  // device bytes owned

    gb::DevBuf<int32_t> perm;       // new -> old (only when reordered)
    gb::DevBuf<int32_t> row_ptr;    // CSR, internal numbering
    gb::DevBuf<int32_t> col;
    gb::DevBuf<double> val;
    gb::DevBuf<float> val32;
    gb::DevBuf<int64_t> slice_ptr;  // sliced ELLPACK
    gb::DevBuf<int32_t> sell_col;
    gb::DevBuf<uint16_t> sell_col16;  // 16-bit relative columns (Sec. 5.1), 0xFFFF = padding
    gb::DevBuf<double> sell_val;
    gb::DevBuf<float> sell_val32;
    gb::DevBuf<int32_t> col_start;  // per-slice x range (Sec. 5.1)
    gb::DevBuf<int32_t> col_end;
    int bulk_G = 0;                  // CTAs of the staged product (SPMV_VARIANT_SELL_BULK)
    gb::DevBuf<int32_t> bulk_part;   // CTA b takes slices [bulk_part[b], bulk_part[b + 1])
    gb::DevBuf<int> dev_status;      // bit 0: a staged product gave up a bounded wait
    gb::CgWork cg;
    gb::McgWork *mcg = nullptr;  // created by the first cg_solve_multi
    int mcg_bytes = 32;          // cg_solve_multi: bytes of a row each product lane gathers
    bool mcg_tuned = false;      // mcg_bytes chosen by the tuner
    int pq_ctas = 0;             // CG product grid: CTAs per SM (0: pq_min_ctas)
    int pq_unroll = 0;           // CG product entries in flight (0: by load rounds)
    bool pq_tuned = false;       // pq_ctas / pq_unroll chosen by the tuner
    // SpMM form per precision (0 FP64, 1 FP32) and lanes per row (1, 2, 4, 8) chosen by the
    // tuner on the first multi-vector product of that shape (SPMV_SPMM_AUTO: not tuned)
    int spmm_tuned[2][4] = {};
    // spmv_apply_chain with this handle as B: form picked per precision (SPMV_CHAIN_AUTO: not
    // tuned) and the temporaries t = C x of the two-product form
    int chain_pick[2] = {};
    gb::DevBuf<double> chain_t;
    gb::DevBuf<float> chain_t32;

    // spmv_apply_host(_async): three staging sets used in turn, each with device copies of x
    // and y, two streams of its own (product, device-to-host) and events; created on first use
    static constexpr int kHostChunks = 8;
    static constexpr int kHostStages = 3;
    struct HostStage {
        gb::DevBuf<double> x, y;
        cudaStream_t sk = nullptr, sy = nullptr;
        cudaEvent_t ev_x[kHostChunks] = {}, ev_k[kHostChunks] = {};
        cudaEvent_t x_free = nullptr, y_free = nullptr;  // end of the last use's reads of x, y
    } h_stage[kHostStages];
    int h_next = 0;                         // staging set of the next call
    int h_chunks = 0;                       // 0 = not prepared
    int32_t h_slice[kHostChunks + 1] = {};  // chunk c = slices [h_slice[c], h_slice[c + 1])
    int32_t h_xend[kHostChunks] = {};       // x entries [0, h_xend[c]) cover chunks 0..c

    bool has64() const { return opt.precision != SPMV_PREC_FP32; }
    bool has32() const { return opt.precision != SPMV_PREC_FP64; }
};

namespace gb {

// conversion pipeline (convert.cu)
spmv_status_t build_matrix(spmv_matrix_t A, const int32_t *d_rp, const int32_t *d_ci,
                           const double *d_val, cudaStream_t st);
spmv_status_t build_sell(spmv_matrix_t A, int S, cudaStream_t st);

// kernels (spmv.cu)
spmv_status_t launch_spmv64(spmv_matrix_t A, const double *x, double *y, cudaStream_t st);
spmv_status_t launch_axpby64(spmv_matrix_t A, double alpha, const double *x, double beta,
                             double *y, cudaStream_t st);
spmv_status_t launch_axpby32(spmv_matrix_t A, float alpha, const float *x, float beta, float *y,
                             cudaStream_t st);
spmv_status_t launch_spmv32(spmv_matrix_t A, const float *x, float *y, cudaStream_t st);
spmv_status_t launch_spmv_csr64(spmv_matrix_t A, const double *x, double *y, cudaStream_t st);
spmv_status_t launch_spmm64(spmv_matrix_t A, int k, const double *X, double *Y, cudaStream_t st);
spmv_status_t launch_spmm32(spmv_matrix_t A, int k, const float *X, float *Y, cudaStream_t st);
spmv_status_t tune_spmm64(spmv_matrix_t A, int k, const double *X, double *Y, cudaStream_t st);
spmv_status_t tune_spmm32(spmv_matrix_t A, int k, const float *X, float *Y, cudaStream_t st);
int spmm_form_of(const spmv_matrix_t A, bool f32, int gi);
int chain_form_of(const spmv_matrix_t B, bool f32);
spmv_status_t launch_permute(spmv_matrix_t A, int direction, int elem_bytes, const void *in,
                             void *out, cudaStream_t st);
int window_capacity_words(int elem_bytes);
spmv_status_t launch_window64(spmv_matrix_t A, const double *x, double *y, cudaStream_t st);
spmv_status_t launch_window32(spmv_matrix_t A, const float *x, float *y, cudaStream_t st);
spmv_status_t choose_variant(spmv_matrix_t A, cudaStream_t st);

// staged product (bulk.cu): per-CTA slice runs of a handle, and the launches (*launched =
// false when the handle's slices do not fit the shared-memory stages: nothing was enqueued)
spmv_status_t bulk_partition(spmv_matrix_t A, cudaStream_t st);
spmv_status_t launch_bulk64(spmv_matrix_t A, const double *x, double *y, cudaStream_t st,
                            bool *launched);
spmv_status_t launch_bulk32(spmv_matrix_t A, const float *x, float *y, cudaStream_t st,
                            bool *launched);
spmv_status_t bulk_diag_timeout(spmv_matrix_t A, cudaStream_t st, int *recorded);

// device scan utilities (scan.cu): exclusive prefix sum of n int64 values in place; the
// total is written to out[n] (the array holds n + 1 entries).
spmv_status_t exclusive_scan_i64(int64_t *d, int64_t n, cudaStream_t st);

// Controls of cg_solve_ex (cg.cu); the defaults give cg_solve.
struct SolveControl {
    const std::atomic<int> *cancel = nullptr;  // polled at every convergence check
    // true: each batch of iterations is a CUDA graph captured once per handle; false: the
    // same kernels launched directly (for one-off handles: capturing, instantiating and
    // destroying a graph per handle was measured to stall concurrent solves)
    bool graphs = true;
};
spmv_status_t cg_solve_ex(spmv_matrix_t A, const double *b, double *x, const cg_options_t *opt,
                          cg_result_t *result, cudaStream_t st, const SolveControl &ctl);

}  // namespace gb
