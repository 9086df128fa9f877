// autotune.cu -- picks the slice height S, the CTA size and the product variant of a handle by
// timing every candidate on the matrix itself (CUDA events, median of 5 launches after 2
// warm-up launches).  Each slice height needs its own sliced-ELLPACK arrays, so the arrays are
// rebuilt per candidate and finally for the winner.  Candidates: S in {32, 64, 128, 256}
// (S = 512 of the FPGA design is a pipelining depth, Sec. 6.1, and has no GPU meaning),
// CTA sizes {128, 256, 512}, the matrix staged by bulk copies, the shared-memory window
// variant, and the naive CSR kernel (FP64 handles).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gb {

namespace {

spmv_status_t time_launch(spmv_matrix_t A, const void *x, void *y, cudaStream_t st,
                          cudaEvent_t e0, cudaEvent_t e1, float *ms_out) {
    auto launch = [&]() -> spmv_status_t {
        if (A->has64()) return launch_spmv64(A, (const double *)x, (double *)y, st);
        return launch_spmv32(A, (const float *)x, (float *)y, st);
    };
    for (int i = 0; i < 2; ++i) GB_TRY(launch());
    std::vector<float> t;
    for (int i = 0; i < 5; ++i) {
        GB_CUDA(cudaEventRecord(e0, st));
        GB_TRY(launch());
        GB_CUDA(cudaEventRecord(e1, st));
        GB_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        GB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    *ms_out = t[t.size() / 2];
    return SPMV_OK;
}

}  // namespace

spmv_status_t autotune_matrix(spmv_matrix_t A, cudaStream_t st) {
    if (A->n == 0) return SPMV_OK;
    NvtxRange nvtx("spmv_create/autotune");
    const size_t eb = A->has64() ? sizeof(double) : sizeof(float);
    void *x = nullptr, *y = nullptr;
    const size_t nx = (size_t)(A->n_cols > 0 ? A->n_cols : 1);
    GB_CUDA(gb_malloc_async(&x, eb * nx, st));
    spmv_status_t s = cuda_status(gb_malloc_async(&y, eb * (size_t)A->n, st));
    if (s == SPMV_OK) s = cuda_status(cudaMemsetAsync(x, 0, eb * nx, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s == SPMV_OK) s = cuda_status(cudaEventCreate(&e0));
    if (s == SPMV_OK) s = cuda_status(cudaEventCreate(&e1));
    const int heights[] = {32, 64, 128, 256};
    const int blocks[] = {128, 256, 512};
    float best = 1e30f;
    int best_S = A->S, best_block = A->block, best_variant = SPMV_VARIANT_SELL;
    const int user_variant = A->opt.variant;
    for (int S : heights) {
        if (s != SPMV_OK) break;
        s = build_sell(A, S, st);
        if (s != SPMV_OK) break;
        for (int b : blocks) {
            A->block = b;
            A->variant = SPMV_VARIANT_SELL;
            float ms;
            s = time_launch(A, x, y, st, e0, e1, &ms);
            if (s != SPMV_OK) break;
            if (ms < best) {
                best = ms;
                best_S = S;
                best_block = b;
                best_variant = SPMV_VARIANT_SELL;
            }
        }
        if (s != SPMV_OK) break;
        if (user_variant == SPMV_VARIANT_AUTO || user_variant == SPMV_VARIANT_SELL_BULK) {
            // matrix staged through shared memory by bulk copies (one CTA per SM)
            A->variant = SPMV_VARIANT_SELL_BULK;
            float ms;
            s = time_launch(A, x, y, st, e0, e1, &ms);
            if (s != SPMV_OK) break;
            if (ms < best) {
                best = ms;
                best_S = S;
                best_variant = SPMV_VARIANT_SELL_BULK;
            }
        }
        if (user_variant == SPMV_VARIANT_AUTO || user_variant == SPMV_VARIANT_SELL_WINDOW) {
            // shared-memory window of x (one 1024-thread CTA per SM)
            A->variant = SPMV_VARIANT_SELL_WINDOW;
            float ms;
            s = time_launch(A, x, y, st, e0, e1, &ms);
            if (s != SPMV_OK) break;
            if (ms < best) {
                best = ms;
                best_S = S;
                best_variant = SPMV_VARIANT_SELL_WINDOW;
            }
        }
    }
    if (s == SPMV_OK && A->has64() && user_variant == SPMV_VARIANT_AUTO) {
        A->variant = SPMV_VARIANT_CSR;
        float ms;
        s = time_launch(A, x, y, st, e0, e1, &ms);
        if (s == SPMV_OK && ms < best) {
            best = ms;
            best_variant = SPMV_VARIANT_CSR;
        }
    }
    if (s == SPMV_OK && best_S != A->S) s = build_sell(A, best_S, st);
    A->block = best_block;
    if (user_variant == SPMV_VARIANT_AUTO) A->variant = best_variant;
    else A->variant = user_variant;
    A->window_words = A->variant == SPMV_VARIANT_SELL_WINDOW
                          ? window_capacity_words(A->has64() ? 8 : 4)
                          : 0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (x) cudaFreeAsync(x, st);
    if (y) cudaFreeAsync(y, st);
    return s;
}

}  // namespace gb
