// server.cu -- continuous-batching CG solve server.
#include "common.cuh"

extern "C" {

spmv_status_t spmv_server_create(size_t, int, spmv_server_t *out) {
    if (out) *out = nullptr;
    return SPMV_ERR_UNSUPPORTED;
}
spmv_status_t spmv_server_submit(spmv_server_t s, int32_t, int64_t, const int32_t *,
                                 const int32_t *, const double *, const double *,
                                 const cg_options_t *, uint64_t *) {
    if (!s) return SPMV_ERR_INVALID_ARG;
    return SPMV_ERR_UNSUPPORTED;
}
spmv_status_t spmv_server_poll(spmv_server_t s, uint64_t, double *, cg_result_t *) {
    if (!s) return SPMV_ERR_INVALID_ARG;
    return SPMV_ERR_UNSUPPORTED;
}
spmv_status_t spmv_server_get_stats(spmv_server_t, spmv_server_stats_t *) {
    return SPMV_ERR_UNSUPPORTED;
}
spmv_status_t spmv_server_destroy(spmv_server_t) { return SPMV_OK; }

}  // extern "C"
