// host_apply.cu -- y = A x for x and y in host memory, with the copies overlapping the product.
//
// The rows are cut into up to kHostChunks runs of slices.  With a banded (Cuthill-McKee)
// numbering the slices of run c read x only below col_end of its slices (Sec. 5.1), so the
// host-to-device copy of x proceeds in increasing column order on the caller's stream, run
// c's product starts on a second stream as soon as the columns it reads have arrived, and its
// rows of y go back to the host on a third stream while later runs compute: the three
// transfers of the paper's task (x in, product, y out) are pipelined instead of serialised.
// The asynchronous form moves x, the product and y in one piece each instead (runs of slices
// cost copy efficiency when calls already overlap each other); its calls take three staging
// sets in turn, so calls on different streams overlap (the copy of one call's x with the copy
// of an earlier call's y and with products); a set is reused only after its previous call has
// finished with it.  With two sets the copy of x for call i + 2 had to wait for call i's y,
// which starts a product later than the copy of x for call i + 1 ends, leaving the
// host-to-device link idle for a product's time every step.  Each run is the ordinary
// product kernel on a view of the handle restricted to its slices, so y is bit-identical to
// spmv_apply's.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gb {
namespace {

spmv_status_t prepare_host_apply(spmv_matrix_t A, cudaStream_t st) {
    if (A->h_chunks > 0) return SPMV_OK;
    size_t *t = &A->bytes;
    const int C = A->n_slices < spmv_matrix_s::kHostChunks ? A->n_slices
                                                            : spmv_matrix_s::kHostChunks;
    for (auto &h : A->h_stage) {
        GB_TRY(h.x.alloc((size_t)(A->n_cols > 0 ? A->n_cols : 1), t));
        GB_TRY(h.y.alloc((size_t)A->n, t));
        if (!h.sk) GB_CUDA(cudaStreamCreateWithFlags(&h.sk, cudaStreamNonBlocking));
        if (!h.sy) GB_CUDA(cudaStreamCreateWithFlags(&h.sy, cudaStreamNonBlocking));
        for (int c = 0; c < C; ++c) {
            if (!h.ev_x[c]) GB_CUDA(cudaEventCreateWithFlags(&h.ev_x[c], cudaEventDisableTiming));
            if (!h.ev_k[c]) GB_CUDA(cudaEventCreateWithFlags(&h.ev_k[c], cudaEventDisableTiming));
        }
        if (!h.x_free) GB_CUDA(cudaEventCreateWithFlags(&h.x_free, cudaEventDisableTiming));
        if (!h.y_free) GB_CUDA(cudaEventCreateWithFlags(&h.y_free, cudaEventDisableTiming));
    }
    // per-slice end of the x range (exclusive; 0 for a slice without entries)
    std::vector<int32_t> ce((size_t)A->n_slices);
    GB_CUDA(cudaMemcpyAsync(ce.data(), A->col_end.p, sizeof(int32_t) * ce.size(),
                            cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    int32_t xend = 0;
    for (int c = 0; c < C; ++c) {
        A->h_slice[c] = (int32_t)((int64_t)c * A->n_slices / C);
        A->h_slice[c + 1] = (int32_t)((int64_t)(c + 1) * A->n_slices / C);
        for (int32_t s = A->h_slice[c]; s < A->h_slice[c + 1]; ++s) xend = std::max(xend, ce[(size_t)s]);
        A->h_xend[c] = xend;
    }
    A->h_chunks = C;
    return SPMV_OK;
}

// Enqueues the whole call; `st` waits at the end until y is on the host.  runs = 1 sends x,
// computes and returns y in one piece each (for calls that overlap each other); otherwise the
// call is cut into the prepared runs of slices.
spmv_status_t enqueue_host_apply(spmv_matrix_t A, const double *x_host, double *y_host,
                                 cudaStream_t st, bool one_run) {
    GB_TRY(prepare_host_apply(A, st));
    auto &h = A->h_stage[A->h_next];
    A->h_next = (A->h_next + 1) % spmv_matrix_s::kHostStages;
    const int C = one_run ? 1 : A->h_chunks;
    // this set's previous call: its products have read x (x_free) and its copies have read y
    // (y_free); events never recorded yet are no-ops
    GB_CUDA(cudaStreamWaitEvent(st, h.x_free, 0));
    GB_CUDA(cudaStreamWaitEvent(h.sk, h.y_free, 0));
    int32_t copied = 0;
    for (int c = 0; c < C; ++c) {
        // x columns this run reads that have not been sent yet
        const int32_t xend = one_run ? A->h_xend[A->h_chunks - 1] : A->h_xend[c];
        if (xend > copied) {
            GB_CUDA(cudaMemcpyAsync(h.x.p + copied, x_host + copied,
                                    sizeof(double) * (size_t)(xend - copied),
                                    cudaMemcpyHostToDevice, st));
            copied = xend;
        }
        GB_CUDA(cudaEventRecord(h.ev_x[c], st));
        GB_CUDA(cudaStreamWaitEvent(h.sk, h.ev_x[c], 0));
        // the product of run c on a view of the handle holding only its slices
        const int32_t s0 = one_run ? 0 : A->h_slice[c];
        const int32_t s1 = one_run ? A->n_slices : A->h_slice[c + 1];
        const int64_t r0 = (int64_t)s0 * A->S;
        const int64_t r1 = std::min<int64_t>((int64_t)s1 * A->S, A->n);
        if (r1 > r0) {
            spmv_matrix_s view = *A;
            view.n = (int32_t)(r1 - r0);
            view.n_slices = s1 - s0;
            view.slice_ptr.p = A->slice_ptr.p + s0;
            view.col_start.p = A->col_start.p + s0;
            view.col_end.p = A->col_end.p + s0;
            view.row_ptr.p = A->row_ptr.p + r0;
            GB_TRY(launch_spmv64(&view, h.x.p, h.y.p + r0, h.sk));
        }
        GB_CUDA(cudaEventRecord(h.ev_k[c], h.sk));
        GB_CUDA(cudaStreamWaitEvent(h.sy, h.ev_k[c], 0));
        if (r1 > r0)
            GB_CUDA(cudaMemcpyAsync(y_host + r0, h.y.p + r0, sizeof(double) * (size_t)(r1 - r0),
                                    cudaMemcpyDeviceToHost, h.sy));
    }
    GB_CUDA(cudaEventRecord(h.x_free, h.sk));
    GB_CUDA(cudaEventRecord(h.y_free, h.sy));
    GB_CUDA(cudaStreamWaitEvent(st, h.y_free, 0));  // y on the host when st gets here
    return SPMV_OK;
}

spmv_status_t check_host_args(spmv_matrix_t A, const double *x_host, const double *y_host) {
    if (!A) return SPMV_ERR_INVALID_ARG;
    if (A->n > 0 && (!y_host || (A->n_cols > 0 && !x_host))) return SPMV_ERR_INVALID_ARG;
    if (!A->has64()) return SPMV_ERR_UNSUPPORTED;
    return SPMV_OK;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" spmv_status_t spmv_apply_host_async(spmv_matrix_t A, const double *x_host,
                                               double *y_host, void *stream) {
    GB_TRY(check_host_args(A, x_host, y_host));
    if (A->n == 0) return SPMV_OK;
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    NvtxRange nvtx("spmv_apply_host_async");
    return enqueue_host_apply(A, x_host, y_host, st, true);
}

extern "C" spmv_status_t spmv_apply_host(spmv_matrix_t A, const double *x_host, double *y_host,
                                         void *stream) {
    GB_TRY(check_host_args(A, x_host, y_host));
    if (A->n == 0) return SPMV_OK;
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    NvtxRange nvtx("spmv_apply_host");
    spmv_status_t s = enqueue_host_apply(A, x_host, y_host, st, false);
    spmv_status_t w = cuda_status(cudaStreamSynchronize(st));
    return s != SPMV_OK ? s : w;
}
