// capi.cu -- extern "C" entry points declared in include/spmv.h: argument checks, handle
// life cycle, dispatch to the kernels.  No torch types, no host-side compute on the path.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "common.cuh"

namespace gb {

cudaStream_t &alloc_stream() {
    static thread_local cudaStream_t s = nullptr;
    return s;
}

cudaMemPool_t &alloc_pool() {
    static thread_local cudaMemPool_t p = nullptr;
    return p;
}

const DeviceFacts &device_facts() {
    static DeviceFacts facts[64];
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        dev = 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    DeviceFacts &f = facts[dev];
    if (f.device != dev) {
        f.device = dev;
        cudaDeviceGetAttribute(&f.sm_count, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&f.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&f.l2_bytes, cudaDevAttrL2CacheSize, dev);
        cudaGetLastError();
    }
    return f;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static spmv_status_t normalize_options(const spmv_options_t *in, spmv_options_t *o) {
    spmv_default_options(o);
    if (!in) return SPMV_OK;
    *o = *in;
    if (o->slice_height == 0) o->slice_height = 64;
    if (o->block == 0) o->block = 256;
    const int S = o->slice_height;
    if (S != 32 && S != 64 && S != 128 && S != 256) return SPMV_ERR_INVALID_ARG;
    if (o->block < 64 || o->block > 1024 || (o->block % 32) != 0) return SPMV_ERR_INVALID_ARG;
    if (o->variant < SPMV_VARIANT_AUTO || o->variant > SPMV_VARIANT_SELL_BULK)
        return SPMV_ERR_INVALID_ARG;
    if (o->reorder < SPMV_REORDER_NONE || o->reorder > SPMV_REORDER_CM) return SPMV_ERR_INVALID_ARG;
    if (o->precision < SPMV_PREC_FP64 || o->precision > SPMV_PREC_DUAL) return SPMV_ERR_INVALID_ARG;
    if (o->window_words < 0) return SPMV_ERR_INVALID_ARG;
    if (o->index_bits != 0 && o->index_bits != 16 && o->index_bits != 32) return SPMV_ERR_INVALID_ARG;
    if (o->sigma != 0 && (o->sigma < 32 || o->sigma > 4096 || (o->sigma & (o->sigma - 1)) != 0))
        return SPMV_ERR_INVALID_ARG;
    if (o->checks != 0 && o->checks != 1) return SPMV_ERR_INVALID_ARG;
    if (o->spmm_form < SPMV_SPMM_AUTO || o->spmm_form > SPMV_SPMM_UNROLLED)
        return SPMV_ERR_INVALID_ARG;
    if (o->pq_ctas != 0 && (o->pq_ctas < 2 || o->pq_ctas > 4)) return SPMV_ERR_INVALID_ARG;
    if (o->pq_unroll != 0 && o->pq_unroll != 2 && o->pq_unroll != 5) return SPMV_ERR_INVALID_ARG;
    if (o->gather_bytes != 0 && o->gather_bytes != 16 && o->gather_bytes != 32)
        return SPMV_ERR_INVALID_ARG;
    if (o->chain_form < SPMV_CHAIN_AUTO || o->chain_form > SPMV_CHAIN_TWO)
        return SPMV_ERR_INVALID_ARG;
    return SPMV_OK;
}

void release_matrix(spmv_matrix_t A);
spmv_status_t autotune_matrix(spmv_matrix_t A, cudaStream_t st);
spmv_status_t verify_matrix(spmv_matrix_t A, cudaStream_t st, int *flags);
spmv_status_t checks_self_test(spmv_matrix_t A, cudaStream_t st, int *detected, int *planted);
spmv_status_t diag_barrier_timeout(int ctas, double limit_s, int *done_out, cudaStream_t st);

}  // namespace gb

using namespace gb;

extern "C" {

spmv_status_t spmv_default_options(spmv_options_t *opt) {
    if (!opt) return SPMV_ERR_INVALID_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->slice_height = 64;
    opt->block = 256;
    opt->variant = SPMV_VARIANT_AUTO;
    opt->reorder = SPMV_REORDER_NONE;
    opt->precision = SPMV_PREC_FP64;
    opt->autotune = 0;
    opt->peripheral = 1;
    opt->window_words = 0;
    opt->index_bits = 0;
    opt->sigma = 0;
    return SPMV_OK;
}

const char *spmv_status_string(spmv_status_t s) {
    switch (s) {
        case SPMV_OK: return "ok";
        case SPMV_ERR_INVALID_ARG: return "invalid argument";
        case SPMV_ERR_INVALID_CSR: return "invalid CSR matrix";
        case SPMV_ERR_OOM: return "out of device memory";
        case SPMV_ERR_BUDGET: return "request exceeds the memory budget";
        case SPMV_ERR_CUDA: return "CUDA error";
        case SPMV_ERR_NOT_CONVERGED: return "not converged";
        case SPMV_ERR_TIMEOUT: return "timeout";
        case SPMV_ERR_PENDING: return "pending";
        case SPMV_ERR_UNSUPPORTED: return "unsupported for this handle";
        case SPMV_ERR_CANCELLED: return "cancelled";
    }
    return "unknown status";
}

spmv_status_t spmv_create(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col_idx, const double *values, int inputs_on_device,
                          const spmv_options_t *opt, void *stream, spmv_matrix_t *out) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_rows < 0 || n_cols < 0 || nnz < 0 || nnz > INT32_MAX) return SPMV_ERR_INVALID_ARG;
    if (!row_ptr) return SPMV_ERR_INVALID_ARG;
    if (nnz > 0 && (!col_idx || !values)) return SPMV_ERR_INVALID_ARG;
    spmv_options_t o;
    GB_TRY(normalize_options(opt, &o));
    // a symmetric renumbering needs a square matrix
    if (n_cols != n_rows && (o.reorder != SPMV_REORDER_NONE || o.sigma != 0))
        return SPMV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    NvtxRange nvtx("spmv_create");

    spmv_matrix_t A = new (std::nothrow) spmv_matrix_s();
    if (!A) return SPMV_ERR_OOM;
    AllocStream alloc_scope(st);
    A->stream = st;
    A->n = n_rows;
    A->n_cols = n_cols;
    A->nnz = nnz;
    A->opt = o;
    A->S = o.slice_height;
    A->block = o.block;
    A->pq_ctas = o.pq_ctas;
    A->pq_unroll = o.pq_unroll;
    A->mcg_bytes = o.gather_bytes ? o.gather_bytes : 32;

    int32_t *d_rp = nullptr, *d_ci = nullptr;
    double *d_val = nullptr;
    spmv_status_t s = SPMV_OK;
    if (!inputs_on_device) {
        s = cuda_status(gb_malloc_async((void **)&d_rp, sizeof(int32_t) * ((size_t)n_rows + 1), st));
        if (s == SPMV_OK)
            s = cuda_status(gb_malloc_async((void **)&d_ci, sizeof(int32_t) * (nnz ? nnz : 1), st));
        if (s == SPMV_OK)
            s = cuda_status(gb_malloc_async((void **)&d_val, sizeof(double) * (nnz ? nnz : 1), st));
        if (s == SPMV_OK)
            s = cuda_status(cudaMemcpyAsync(d_rp, row_ptr, sizeof(int32_t) * ((size_t)n_rows + 1),
                                            cudaMemcpyHostToDevice, st));
        if (s == SPMV_OK && nnz)
            s = cuda_status(cudaMemcpyAsync(d_ci, col_idx, sizeof(int32_t) * nnz,
                                            cudaMemcpyHostToDevice, st));
        if (s == SPMV_OK && nnz)
            s = cuda_status(cudaMemcpyAsync(d_val, values, sizeof(double) * nnz,
                                            cudaMemcpyHostToDevice, st));
    } else {
        d_rp = const_cast<int32_t *>(row_ptr);
        d_ci = const_cast<int32_t *>(col_idx);
        d_val = const_cast<double *>(values);
    }
    if (s == SPMV_OK) s = build_matrix(A, d_rp, d_ci, d_val, st);
    if (!inputs_on_device) {
        if (d_rp) cudaFreeAsync(d_rp, st);
        if (d_ci) cudaFreeAsync(d_ci, st);
        if (d_val) cudaFreeAsync(d_val, st);
    }
    if (s == SPMV_OK) s = choose_variant(A, st);
    if (s == SPMV_OK && o.autotune) s = autotune_matrix(A, st);
    if (s == SPMV_OK && o.checks) {
        int flags = 0;
        s = verify_matrix(A, st, &flags);
        if (s == SPMV_OK && flags) s = SPMV_ERR_INVALID_CSR;
    }
    if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
    if (s != SPMV_OK) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
        release_matrix(A);
        return s;
    }
    *out = A;
    return SPMV_OK;
}

spmv_status_t spmv_destroy(spmv_matrix_t A) {
    if (!A) return SPMV_OK;
    // the creation stream may no longer exist: free on the legacy stream after a device sync
    cudaDeviceSynchronize();
    {
        AllocStream alloc_scope(nullptr);
        release_matrix(A);
    }
    cudaDeviceSynchronize();
    return SPMV_OK;
}

spmv_status_t spmv_verify(spmv_matrix_t A, int *violations, void *stream) {
    if (violations) *violations = 0;
    if (!A) return SPMV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    int flags = 0;
    GB_TRY(verify_matrix(A, st, &flags));
    if (violations) *violations = flags;
    return flags ? SPMV_ERR_INVALID_CSR : SPMV_OK;
}

spmv_status_t spmv_device_status(spmv_matrix_t A, void *stream) {
    if (!A) return SPMV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!A->dev_status.p) return SPMV_OK;
    int v = 0;
    GB_CUDA(cudaMemcpyAsync(&v, A->dev_status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemsetAsync(A->dev_status.p, 0, sizeof(int), st));
    GB_CUDA(cudaStreamSynchronize(st));
    return v ? SPMV_ERR_TIMEOUT : SPMV_OK;
}

spmv_status_t spmv_diag_bulk_timeout(spmv_matrix_t A, void *stream) {
    if (!A || A->n == 0 || A->sell_entries == 0) return SPMV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    int recorded = 0;
    GB_TRY(bulk_diag_timeout(A, st, &recorded));
    return (recorded & 1) ? SPMV_ERR_TIMEOUT : SPMV_ERR_CUDA;
}

spmv_status_t spmv_diag_checks(spmv_matrix_t A, int *planted, int *detected, void *stream) {
    if (planted) *planted = 0;
    if (detected) *detected = 0;
    if (!A || !planted || !detected) return SPMV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    return checks_self_test(A, st, detected, planted);
}

spmv_status_t spmv_get_info(spmv_matrix_t A, spmv_info_t *info) {
    if (!A || !info) return SPMV_ERR_INVALID_ARG;
    info->n_rows = A->n;
    info->n_cols = A->n_cols;
    info->nnz = A->nnz;
    info->slice_height = A->S;
    info->block = A->block;
    info->variant = A->variant;
    info->precision = A->opt.precision;
    info->reorder = A->opt.reorder;
    info->n_slices = A->n_slices;
    info->sell_entries = A->sell_entries;
    info->bandwidth = A->bandwidth;
    info->max_slice_span = A->max_span;
    info->window_words = A->window_words;
    info->device_bytes = A->bytes;
    info->index_bits = A->index_bits;
    for (int p = 0; p < 2; ++p)
        for (int g = 0; g < 4; ++g) info->spmm_form[p][g] = spmm_form_of(A, p == 1, g);
    info->pq_ctas = A->pq_ctas;
    info->pq_unroll = A->pq_unroll;
    info->gather_bytes = A->mcg_bytes;
    info->chain_form[0] = chain_form_of(A, false);
    info->chain_form[1] = chain_form_of(A, true);
    return SPMV_OK;
}

spmv_status_t spmv_get_permutation(spmv_matrix_t A, int32_t *perm_host) {
    if (!A || (!perm_host && A->n > 0)) return SPMV_ERR_INVALID_ARG;
    if (A->perm.p) {
        GB_CUDA(cudaMemcpy(perm_host, A->perm.p, sizeof(int32_t) * A->n, cudaMemcpyDeviceToHost));
    } else {
        for (int32_t i = 0; i < A->n; ++i) perm_host[i] = i;
    }
    return SPMV_OK;
}

spmv_status_t spmv_export_csr(spmv_matrix_t A, int32_t *row_ptr, int32_t *col_idx,
                              double *values) {
    if (!A || !row_ptr || (A->nnz > 0 && !col_idx)) return SPMV_ERR_INVALID_ARG;
    GB_CUDA(cudaDeviceSynchronize());
    GB_CUDA(cudaMemcpy(row_ptr, A->row_ptr.p, sizeof(int32_t) * ((size_t)A->n + 1),
                       cudaMemcpyDeviceToHost));
    if (A->nnz) {
        GB_CUDA(cudaMemcpy(col_idx, A->col.p, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost));
        if (values)
            GB_CUDA(cudaMemcpy(values, A->val.p, sizeof(double) * A->nnz, cudaMemcpyDeviceToHost));
    }
    return SPMV_OK;
}

spmv_status_t spmv_export_sell(spmv_matrix_t A, int64_t *slice_ptr, int32_t *col, double *values,
                               int32_t *col_start, int32_t *col_end) {
    if (!A || !slice_ptr || (A->sell_entries > 0 && !col)) return SPMV_ERR_INVALID_ARG;
    if (values && !A->has64()) return SPMV_ERR_UNSUPPORTED;
    GB_CUDA(cudaDeviceSynchronize());
    GB_CUDA(cudaMemcpy(slice_ptr, A->slice_ptr.p, sizeof(int64_t) * ((size_t)A->n_slices + 1),
                       cudaMemcpyDeviceToHost));
    if (A->sell_entries) {
        GB_CUDA(cudaMemcpy(col, A->sell_col.p, sizeof(int32_t) * A->sell_entries,
                           cudaMemcpyDeviceToHost));
        if (values)
            GB_CUDA(cudaMemcpy(values, A->sell_val.p, sizeof(double) * A->sell_entries,
                               cudaMemcpyDeviceToHost));
    }
    if (A->n_slices) {
        if (col_start)
            GB_CUDA(cudaMemcpy(col_start, A->col_start.p, sizeof(int32_t) * A->n_slices,
                               cudaMemcpyDeviceToHost));
        if (col_end)
            GB_CUDA(cudaMemcpy(col_end, A->col_end.p, sizeof(int32_t) * A->n_slices,
                               cudaMemcpyDeviceToHost));
    }
    return SPMV_OK;
}

spmv_status_t spmv_apply(spmv_matrix_t A, const double *x, double *y, void *stream) {
    if (!A) return SPMV_ERR_INVALID_ARG;
    if (A->n > 0 && (!x || !y || !aligned16(x) || !aligned16(y) || x == y))
        return SPMV_ERR_INVALID_ARG;
    if (!A->has64()) return SPMV_ERR_UNSUPPORTED;
    return launch_spmv64(A, x, y, (cudaStream_t)stream);
}

spmv_status_t spmv_apply_f32(spmv_matrix_t A, const float *x, float *y, void *stream) {
    if (!A) return SPMV_ERR_INVALID_ARG;
    if (A->n > 0 && (!x || !y || !aligned16(x) || !aligned16(y) || x == y))
        return SPMV_ERR_INVALID_ARG;
    if (!A->has32()) return SPMV_ERR_UNSUPPORTED;
    return launch_spmv32(A, x, y, (cudaStream_t)stream);
}

spmv_status_t spmv_apply_axpby(spmv_matrix_t A, double alpha, const double *x, double beta,
                               double *y, void *stream) {
    if (!A) return SPMV_ERR_INVALID_ARG;
    if ((A->n > 0 || A->n_cols > 0) &&
        (!x || !y || !aligned16(x) || !aligned16(y) || x == y))
        return SPMV_ERR_INVALID_ARG;
    if (!A->has64()) return SPMV_ERR_UNSUPPORTED;
    return launch_axpby64(A, alpha, x, beta, y, (cudaStream_t)stream);
}

spmv_status_t spmv_apply_axpby_f32(spmv_matrix_t A, float alpha, const float *x, float beta,
                                   float *y, void *stream) {
    if (!A) return SPMV_ERR_INVALID_ARG;
    if ((A->n > 0 || A->n_cols > 0) &&
        (!x || !y || !aligned16(x) || !aligned16(y) || x == y))
        return SPMV_ERR_INVALID_ARG;
    if (!A->has32()) return SPMV_ERR_UNSUPPORTED;
    return launch_axpby32(A, alpha, x, beta, y, (cudaStream_t)stream);
}

spmv_status_t spmv_apply_csr(spmv_matrix_t A, const double *x, double *y, void *stream) {
    if (!A) return SPMV_ERR_INVALID_ARG;
    if (A->n > 0 && (!x || !y || x == y)) return SPMV_ERR_INVALID_ARG;
    if (!A->has64()) return SPMV_ERR_UNSUPPORTED;
    return launch_spmv_csr64(A, x, y, (cudaStream_t)stream);
}

spmv_status_t spmv_apply_multi(spmv_matrix_t A, int k, const double *X, double *Y, void *stream) {
    if (!A || k < 1 || k > 64) return SPMV_ERR_INVALID_ARG;
    if (A->n > 0 && (!X || !Y || X == Y || !aligned16(X) || !aligned16(Y)))
        return SPMV_ERR_INVALID_ARG;
    if (!A->has64()) return SPMV_ERR_UNSUPPORTED;
    if (A->opt.autotune && A->opt.spmm_form == SPMV_SPMM_AUTO)
        GB_TRY(tune_spmm64(A, k, X, Y, (cudaStream_t)stream));
    return launch_spmm64(A, k, X, Y, (cudaStream_t)stream);
}

spmv_status_t spmv_apply_multi_f32(spmv_matrix_t A, int k, const float *X, float *Y,
                                   void *stream) {
    if (!A || k < 1 || k > 64) return SPMV_ERR_INVALID_ARG;
    if (A->n > 0 && (!X || !Y || X == Y || !aligned16(X) || !aligned16(Y)))
        return SPMV_ERR_INVALID_ARG;
    if (!A->has32()) return SPMV_ERR_UNSUPPORTED;
    if (A->opt.autotune && A->opt.spmm_form == SPMV_SPMM_AUTO)
        GB_TRY(tune_spmm32(A, k, X, Y, (cudaStream_t)stream));
    return launch_spmm32(A, k, X, Y, (cudaStream_t)stream);
}

spmv_status_t spmv_diag_barrier_timeout(int ctas, double limit_s, void *stream) {
    if (ctas < 1 || ctas > device_facts().sm_count || !(limit_s > 0.0) || limit_s > 10.0)
        return SPMV_ERR_INVALID_ARG;
    int done = 0;
    GB_TRY(diag_barrier_timeout(ctas, limit_s, &done, (cudaStream_t)stream));
    return done == 4 ? SPMV_ERR_TIMEOUT : SPMV_ERR_CUDA;
}

spmv_status_t spmv_permute(spmv_matrix_t A, int direction, int elem_bytes, const void *in,
                           void *out, void *stream) {
    if (!A || (direction != 0 && direction != 1) || (elem_bytes != 4 && elem_bytes != 8))
        return SPMV_ERR_INVALID_ARG;
    if (A->n > 0 && (!in || !out || in == out)) return SPMV_ERR_INVALID_ARG;
    return launch_permute(A, direction, elem_bytes, in, out, (cudaStream_t)stream);
}

}  // extern "C"

namespace gb {

void release_cg(spmv_matrix_t A);
void release_mcg(spmv_matrix_t A);

void release_matrix(spmv_matrix_t A) {
    size_t *t = &A->bytes;
    release_cg(A);
    release_mcg(A);
    for (auto &h : A->h_stage) {
        h.x.release(t);
        h.y.release(t);
        for (int c = 0; c < spmv_matrix_s::kHostChunks; ++c) {
            if (h.ev_x[c]) cudaEventDestroy(h.ev_x[c]);
            if (h.ev_k[c]) cudaEventDestroy(h.ev_k[c]);
        }
        if (h.x_free) cudaEventDestroy(h.x_free);
        if (h.y_free) cudaEventDestroy(h.y_free);
        if (h.sk) cudaStreamDestroy(h.sk);
        if (h.sy) cudaStreamDestroy(h.sy);
    }
    A->perm.release(t);
    A->row_ptr.release(t);
    A->col.release(t);
    A->val.release(t);
    A->val32.release(t);
    A->slice_ptr.release(t);
    A->sell_col.release(t);
    A->sell_col16.release(t);
    A->sell_val.release(t);
    A->sell_val32.release(t);
    A->col_start.release(t);
    A->col_end.release(t);
    A->bulk_part.release(t);
    A->dev_status.release(t);
    A->chain_t.release(t);
    A->chain_t32.release(t);
    delete A;
}

}  // namespace gb
