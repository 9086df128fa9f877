// autotune.cu -- picks the slice height S, the CTA size and the product variant of a handle by
// timing every candidate on the matrix itself with x = 1 (CUDA events, median of 5 launches
// after 2 warm-up launches, L2 overwritten before each timed launch).  Each slice height needs
// its own sliced-ELLPACK arrays, so the arrays are rebuilt per candidate and finally for the
// winner.  Candidates: S in {32, 64, 128, 256}
// (S = 512 of the FPGA design is a pipelining depth, Sec. 6.1, and has no GPU meaning),
// CTA sizes {128, 256, 512}, the matrix staged by bulk copies, the shared-memory window
// variant, and the naive CSR kernel (FP64 handles).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gb {

namespace {

__global__ void fill_ones(size_t n, double *x64, float *x32) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (x64) x64[i] = 1.0;
        else x32[i] = 1.0f;
    }
}

// median of 5 launches after 2 warm-up launches, each timed launch after writing a buffer of
// twice the L2 size, so that the matrix and x come from DRAM as in steady use
spmv_status_t time_launch(spmv_matrix_t A, const void *x, void *y, void *flush, size_t fb,
                          cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float *ms_out) {
    auto launch = [&]() -> spmv_status_t {
        if (A->has64()) return launch_spmv64(A, (const double *)x, (double *)y, st);
        return launch_spmv32(A, (const float *)x, (float *)y, st);
    };
    for (int i = 0; i < 2; ++i) GB_TRY(launch());
    std::vector<float> t;
    for (int i = 0; i < 5; ++i) {
        GB_CUDA(cudaMemsetAsync(flush, i + 1, fb, st));
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
    if (s == SPMV_OK) {  // a real x (ones), not zeros
        fill_ones<<<(unsigned)std::min<size_t>((nx + 255) / 256, 4096), 256, 0, st>>>(
            nx, A->has64() ? (double *)x : nullptr, A->has64() ? nullptr : (float *)x);
        s = cuda_status(cudaGetLastError());
    }
    const size_t fb = 2 * (size_t)(device_facts().l2_bytes > 0 ? device_facts().l2_bytes
                                                               : (128 << 20));
    void *flush = nullptr;
    if (s == SPMV_OK) s = cuda_status(gb_malloc_async(&flush, fb, st));
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
            s = time_launch(A, x, y, flush, fb, st, e0, e1, &ms);
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
            s = time_launch(A, x, y, flush, fb, st, e0, e1, &ms);
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
            s = time_launch(A, x, y, flush, fb, st, e0, e1, &ms);
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
        s = time_launch(A, x, y, flush, fb, st, e0, e1, &ms);
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
    if (flush) cudaFreeAsync(flush, st);
    return s;
}

}  // namespace gb
