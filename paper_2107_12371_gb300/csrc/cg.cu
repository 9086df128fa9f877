// cg.cu -- Jacobi-preconditioned conjugate gradients (FP64) and FP32-inner / FP64-refinement
// solves on top of the SpMV kernels.
#include "common.cuh"

namespace gb {

void release_cg(spmv_matrix_t A) {
    size_t *t = &A->bytes;
    CgWork &w = A->cg;
    w.r.release(t); w.z.release(t); w.p.release(t); w.q.release(t); w.dinv.release(t);
    w.r32.release(t); w.p32.release(t); w.q32.release(t); w.d32.release(t); w.dinv32.release(t);
    w.part.release(t); w.scal.release(t); w.flags.release(t);
    if (w.h_flags) cudaFreeHost(w.h_flags);
    if (w.h_scal) cudaFreeHost(w.h_scal);
    w.h_flags = nullptr;
    w.h_scal = nullptr;
    w.ready = false;
}

}  // namespace gb

extern "C" {

spmv_status_t cg_default_options(cg_options_t *o) {
    if (!o) return SPMV_ERR_INVALID_ARG;
    o->rtol = 1e-10;
    o->max_iter = 20000;
    o->mixed = 0;
    o->inner_rtol = 1e-4;
    o->max_outer = 20;
    o->use_x0 = 0;
    o->persistent = 0;
    o->check_every = 16;
    o->timeout_s = 0.0;
    return SPMV_OK;
}

spmv_status_t cg_solve(spmv_matrix_t A, const double *, double *, const cg_options_t *,
                       cg_result_t *, void *) {
    if (!A) return SPMV_ERR_INVALID_ARG;
    return SPMV_ERR_UNSUPPORTED;
}

}  // extern "C"
