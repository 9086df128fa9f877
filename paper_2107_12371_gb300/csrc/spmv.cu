// spmv.cu -- SpMV kernels (the multi-vector products are in spmm.cu).
//
// spmv_sell<T, R, L>: L lanes per slice of S = L R rows, lane l owns rows l R .. l R + R - 1
//   of the slice.  Because a slice is stored column-major (Sec. 4.2), step t of the lanes
//   reads S consecutive values and column indices: one R-wide vector load per lane, fully
//   coalesced, streamed evict-first so the matrix never displaces x from L2.  x is gathered
//   through the read-only L1 path; with a banded (Cuthill-McKee) order the gathers of
//   neighbouring rows hit the same lines (Sec. 4.3, 5.1).  Each row accumulates its entries
//   in ascending column order with fused multiply-add from +0.0; padding entries (column -1)
//   are skipped.  Column indices come as int32 or (when every slice spans fewer than 65,535
//   columns) as 16-bit offsets from the slice's col_start (Sec. 5.1), 10 instead of 12 bytes
//   per FP64 non-zero.
// spmv_sell_occ / spmv_sell_gs: the FP64 forms with one or two rows per lane, one slice-lane
//   per thread at 32 registers, or a grid of four CTAs per SM striding over the slice-lanes
//   with five entries of each row in flight; the one whose widest slice needs fewer dependent
//   load rounds is launched.
// spmv_csr: the naive baseline of Sec. 4.3, thread per CSR row.
#include "common.cuh"
#include "ptx.cuh"

namespace gb {
namespace {

// y = A x, or with AXPBY y = alpha (A x) + beta y evaluated as fma(alpha, t, beta y) (y is not
// read when beta == 0), t being the row sum in column order.
// gt: the slice-lane this thread computes (slice gt / L, lane gt % L).  The entries of a row
// go in blocks of U (all loads of a block issued before its gathers, and those before its
// FMAs), the rest one at a time.
template <typename T, int R, int L, int U, typename ColT, bool AXPBY>
__device__ __forceinline__ void spmv_sell_body(int64_t gt, int32_t n, int32_t n_slices,
                                               const int64_t *__restrict__ sp, ColT cols,
                                               const T *__restrict__ val,
                                               const T *__restrict__ x, T *__restrict__ y,
                                               T alpha, T beta) {
    // L lanes per slice, R rows per lane: S = L R rows per slice
    constexpr int S = L * R;
    const int64_t slice = gt / L;
    const int lane = (int)(gt % L);
    if (slice >= n_slices) return;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cbase = cols.base(slice);
    const T *vp = val + base + lane * R;
    const int64_t cat = base + lane * R;
    const uint64_t pol = policy_evict_first();
    T acc[R];
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = T(0);
    int t = 0;
    for (; t + U <= w; t += U) {
        T v[U][R];
        int32_t c[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ld_stream(vp + (int64_t)(t + u) * S, pol, v[u]);
            cols.template load<R>(cat + (int64_t)(t + u) * S, slice, pol, cbase, c[u]);
        }
        T xv[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int i = 0; i < R; ++i) xv[u][i] = c[u][i] >= 0 ? ld_x(x + c[u][i]) : T(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (c[u][i] >= 0) acc[i] = fma_t(v[u][i], xv[u][i], acc[i]);
    }
    for (; t < w; ++t) {
        T v[R];
        int32_t c[R];
        ld_stream(vp + (int64_t)t * S, pol, v);
        cols.template load<R>(cat + (int64_t)t * S, slice, pol, cbase, c);
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (c[i] >= 0) acc[i] = fma_t(v[i], ld_x(x + c[i]), acc[i]);
    }
    const int64_t row0 = slice * S + (int64_t)lane * R;
    if constexpr (AXPBY) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (row0 + i < n)
                acc[i] = beta != T(0) ? fma_t(alpha, acc[i], beta * y[row0 + i]) : alpha * acc[i];
        }
    }
    store_rows<T, R>(y, row0, n, acc);
}

template <typename T, int R, int L, int U, typename ColT, bool AXPBY>
__global__ void __launch_bounds__(1024)
spmv_sell(int32_t n, int32_t n_slices, const int64_t *__restrict__ sp, ColT cols,
          const T *__restrict__ val, const T *__restrict__ x, T *__restrict__ y, T alpha,
          T beta) {
    spmv_sell_body<T, R, L, U, ColT, AXPBY>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, n,
                                            n_slices, sp, cols, val, x, y, alpha, beta);
}

// FP64 with one or two rows per lane, capped at 32 registers (2 x 1024 threads per SM), four
// entries in flight: for matrices whose widest slice needs fewer load rounds in blocks of four
// than of five (see go_sell).
template <typename T, int R, int L, int U, typename ColT, bool AXPBY>
__global__ void __launch_bounds__(1024, 2)
spmv_sell_occ(int32_t n, int32_t n_slices, const int64_t *__restrict__ sp, ColT cols,
              const T *__restrict__ val, const T *__restrict__ x, T *__restrict__ y, T alpha,
              T beta) {
    spmv_sell_body<T, R, L, U, ColT, AXPBY>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, n,
                                            n_slices, sp, cols, val, x, y, alpha, beta);
}

// FP64 with one or two rows per lane: a grid of at most kGsCtasPerSm 256-thread CTAs per SM
// strides over the slice-lanes, each thread keeping U = 5 entries of its rows in flight (a
// whole row of the tetrahedral meshes) at 64 registers.  Measured on the 6M-row mesh (S = 64):
// 66.0 us, against 69.6 us for one slice-lane per thread at 32 registers and 2,048 threads per
// SM (four entries in flight), 77.1 us with four entries and 68.3 us with two at six CTAs.
constexpr int kGsBlock = 256;
constexpr int kGsCtasPerSm = 4;
template <typename T, int R, int L, int U, typename ColT, bool AXPBY>
__global__ void __launch_bounds__(kGsBlock, kGsCtasPerSm)
spmv_sell_gs(int32_t n, int32_t n_slices, const int64_t *__restrict__ sp, ColT cols,
             const T *__restrict__ val, const T *__restrict__ x, T *__restrict__ y, T alpha,
             T beta) {
    const int64_t items = (int64_t)n_slices * L;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gt < items; gt += stride)
        spmv_sell_body<T, R, L, U, ColT, AXPBY>(gt, n, n_slices, sp, cols, val, x, y, alpha, beta);
}

// naive CSR baseline (Sec. 4.3): the column index is read first, then x[col] from global
// memory, thread per row
template <typename T>
__global__ void __launch_bounds__(256)
spmv_csr(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
         const T *__restrict__ val, const T *__restrict__ x, T *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc = T(0);
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) acc = fma_t(val[k], x[ci[k]], acc);
    y[i] = acc;
}

template <typename T>
__global__ void permute_kernel(int32_t n, int direction, const int32_t *__restrict__ perm,
                               const T *__restrict__ in, T *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (direction == 0) out[i] = in[perm[i]];
    else out[perm[i]] = in[i];
}

inline unsigned grid_for(int64_t threads, int block) {
    int64_t b = (threads + block - 1) / block;
    return (unsigned)(b < 1 ? 1 : b);
}

// (R, L) per slice height: FP64 lanes read 8R bytes of values (16 B at S = 64, 32 B at
// S >= 128); FP32 lanes read 16 B (R = 4) or 32 B (R = 8).
template <typename T, int R, int L, int U, bool AXPBY>
spmv_status_t go_sell(spmv_matrix_t A, const T *val, const T *x, T *y, T alpha, T beta,
                      cudaStream_t st) {
    const int block = A->block;
    const unsigned grid = grid_for((int64_t)A->n_slices * L, block);
    auto go = [&](auto c) {
        using ColT = decltype(c);
        if constexpr (sizeof(T) == 8 && R <= 2) {
            if (load_rounds(A->max_width, 5) < load_rounds(A->max_width, 4)) {
                const int64_t cap = (int64_t)device_facts().sm_count * kGsCtasPerSm;
                const unsigned want = grid_for((int64_t)A->n_slices * L, kGsBlock);
                const unsigned g = (int64_t)want < cap ? want : (unsigned)cap;
                spmv_sell_gs<T, R, L, 5, ColT, AXPBY><<<g, kGsBlock, 0, st>>>(
                    A->n, A->n_slices, A->slice_ptr.p, c, val, x, y, alpha, beta);
            } else {
                spmv_sell_occ<T, R, L, U, ColT, AXPBY><<<grid, block, 0, st>>>(
                    A->n, A->n_slices, A->slice_ptr.p, c, val, x, y, alpha, beta);
            }
        } else {
            spmv_sell<T, R, L, U, ColT, AXPBY><<<grid, block, 0, st>>>(
                A->n, A->n_slices, A->slice_ptr.p, c, val, x, y, alpha, beta);
        }
    };
    if (A->index_bits == 16) go(Cols16{A->sell_col16.p, A->col_start.p});
    else go(Cols32{A->sell_col.p});
    GB_LAUNCHED();
    return SPMV_OK;
}

template <typename T, bool AXPBY = false>
spmv_status_t launch_sell(spmv_matrix_t A, const T *val, const T *x, T *y, T alpha = T(1),
                          T beta = T(0), cudaStream_t st = nullptr) {
    if (A->n == 0) return SPMV_OK;
    if constexpr (sizeof(T) == 8) {
        switch (A->S) {
            case 32: return go_sell<T, 1, 32, 4, AXPBY>(A, val, x, y, alpha, beta, st);
            case 64: return go_sell<T, 2, 32, 4, AXPBY>(A, val, x, y, alpha, beta, st);
            case 128: return go_sell<T, 4, 32, 2, AXPBY>(A, val, x, y, alpha, beta, st);
            case 256: return go_sell<T, 8, 32, 1, AXPBY>(A, val, x, y, alpha, beta, st);
        }
    } else {
        switch (A->S) {
            case 32: return go_sell<T, 4, 8, 4, AXPBY>(A, val, x, y, alpha, beta, st);
            // five entries in flight per row: a whole row of the tetrahedral meshes in one
            // round of loads (measured 41.0 -> 38.9 us at S = 64 on the 6M-row mesh)
            case 64: return go_sell<T, 4, 16, 5, AXPBY>(A, val, x, y, alpha, beta, st);
            case 128: return go_sell<T, 4, 32, 5, AXPBY>(A, val, x, y, alpha, beta, st);
            case 256: return go_sell<T, 8, 32, 2, AXPBY>(A, val, x, y, alpha, beta, st);
        }
    }
    return SPMV_ERR_INVALID_ARG;
}

}  // namespace

spmv_status_t launch_spmv64(spmv_matrix_t A, const double *x, double *y, cudaStream_t st) {
    if (A->variant == SPMV_VARIANT_CSR) return launch_spmv_csr64(A, x, y, st);
    if (A->variant == SPMV_VARIANT_SELL_WINDOW) return launch_window64(A, x, y, st);
    if (A->variant == SPMV_VARIANT_SELL_BULK) {
        bool launched = false;
        GB_TRY(launch_bulk64(A, x, y, st, &launched));
        if (launched) return SPMV_OK;
    }
    return launch_sell<double>(A, A->sell_val.p, x, y, 1.0, 0.0, st);
}

spmv_status_t launch_axpby64(spmv_matrix_t A, double alpha, const double *x, double beta,
                             double *y, cudaStream_t st) {
    return launch_sell<double, true>(A, A->sell_val.p, x, y, alpha, beta, st);
}

spmv_status_t launch_axpby32(spmv_matrix_t A, float alpha, const float *x, float beta, float *y,
                             cudaStream_t st) {
    return launch_sell<float, true>(A, A->sell_val32.p, x, y, alpha, beta, st);
}

spmv_status_t launch_spmv32(spmv_matrix_t A, const float *x, float *y, cudaStream_t st) {
    if (A->variant == SPMV_VARIANT_SELL_WINDOW) return launch_window32(A, x, y, st);
    if (A->variant == SPMV_VARIANT_SELL_BULK) {
        bool launched = false;
        GB_TRY(launch_bulk32(A, x, y, st, &launched));
        if (launched) return SPMV_OK;
    }
    return launch_sell<float>(A, A->sell_val32.p, x, y, 1.0f, 0.0f, st);
}

spmv_status_t launch_spmv_csr64(spmv_matrix_t A, const double *x, double *y, cudaStream_t st) {
    if (A->n == 0) return SPMV_OK;
    spmv_csr<double><<<grid_for(A->n, 256), 256, 0, st>>>(A->n, A->row_ptr.p, A->col.p, A->val.p,
                                                          x, y);
    GB_LAUNCHED();
    return SPMV_OK;
}

spmv_status_t launch_permute(spmv_matrix_t A, int direction, int elem_bytes, const void *in,
                             void *out, cudaStream_t st) {
    if (A->n == 0) return SPMV_OK;
    const unsigned grid = grid_for(A->n, 256);
    if (!A->perm.p) {
        GB_CUDA(cudaMemcpyAsync(out, in, (size_t)A->n * elem_bytes, cudaMemcpyDeviceToDevice, st));
        return SPMV_OK;
    }
    if (elem_bytes == 8)
        permute_kernel<double><<<grid, 256, 0, st>>>(A->n, direction, A->perm.p,
                                                     (const double *)in, (double *)out);
    else
        permute_kernel<float><<<grid, 256, 0, st>>>(A->n, direction, A->perm.p,
                                                    (const float *)in, (float *)out);
    GB_LAUNCHED();
    return SPMV_OK;
}

spmv_status_t choose_variant(spmv_matrix_t A, cudaStream_t) {
    A->variant = A->opt.variant == SPMV_VARIANT_AUTO ? SPMV_VARIANT_SELL : A->opt.variant;
    A->window_words = A->variant == SPMV_VARIANT_SELL_WINDOW
                          ? window_capacity_words(A->has64() ? 8 : 4)
                          : 0;
    return SPMV_OK;
}

}  // namespace gb
