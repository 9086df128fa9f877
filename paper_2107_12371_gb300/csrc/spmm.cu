// spmm.cu -- multi-right-hand-side products Y = A X (not in the paper).
//
// spmm_sell<T, G, C, U>: X and Y row-major (n x k), G lanes per row, each lane C columns;
// every gathered row of X (k contiguous values) is read once per matrix entry and used for
// all k columns.  Column c of Y equals the single-vector product of column c bit for bit
// (same entry order, fused multiply-add from +0.0).
#include <type_traits>

#include "common.cuh"
#include "ptx.cuh"

namespace gb {
namespace {

inline unsigned grid_for(int64_t threads, int block) {
    int64_t b = (threads + block - 1) / block;
    return (unsigned)(b < 1 ? 1 : b);
}

// SpMM: G lanes per row (G divides 32), lane owns columns g, g + G, ... (C of them).  The
// (value, column) pairs of U consecutive steps are loaded before their rows of X are gathered,
// so every lane keeps U * C gathers in flight instead of one.
template <typename T, int G, int C, int U, typename ColT>
__global__ void __launch_bounds__(256)
spmm_sell(int32_t n, int32_t S, int32_t n_slices, int k, const int64_t *__restrict__ sp,
          ColT cols, const T *__restrict__ val, const T *__restrict__ X, T *__restrict__ Y) {
    constexpr int RPW = 32 / G;  // rows per warp
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, g = lane % G;
    const int64_t rows_total = (int64_t)n_slices * S;
    const int64_t row = gw * RPW + sub;
    if (row >= rows_total) return;
    const int64_t slice = row / S;
    const int64_t r = row - slice * S;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cbase = cols.base(slice);
    const uint64_t pol = policy_evict_first();
    T acc[C];
#pragma unroll
    for (int j = 0; j < C; ++j) acc[j] = T(0);
    int t = 0;
    for (; t + U <= w; t += U) {
        T a[U][1];
        int32_t c[U][1];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ld_stream(val + base + (int64_t)(t + u) * S + r, pol, a[u]);
            cols.template load<1>(base + (int64_t)(t + u) * S + r, slice, pol, cbase, c[u]);
        }
        T xv[U][C];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const int cc = g + j * G;
                xv[u][j] = (c[u][0] >= 0 && cc < k) ? ld_x(X + (int64_t)c[u][0] * k + cc) : T(0);
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < C; ++j)
                if (c[u][0] >= 0) acc[j] = fma_t(a[u][0], xv[u][j], acc[j]);
    }
    for (; t < w; ++t) {
        T a[1];
        int32_t c[1];
        ld_stream(val + base + (int64_t)t * S + r, pol, a);
        cols.template load<1>(base + (int64_t)t * S + r, slice, pol, cbase, c);
        if (c[0] < 0) continue;
        const T *xr = X + (int64_t)c[0] * k;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const int cc = g + j * G;
            if (cc < k) acc[j] = fma_t(a[0], ld_x(xr + cc), acc[j]);
        }
    }
    if (row < n) {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const int cc = g + j * G;
            if (cc < k) Y[row * k + cc] = acc[j];
        }
    }
}

template <typename T>
spmv_status_t launch_spmm(spmv_matrix_t A, int k, const T *val, const T *X, T *Y,
                          cudaStream_t st) {
    if (A->n == 0) return SPMV_OK;
    const int block = 256;
    const int64_t rows_total = (int64_t)A->n_slices * A->S;
    auto go = [&](auto gtag, auto ctag) -> spmv_status_t {
        constexpr int G = decltype(gtag)::value;
        constexpr int C = decltype(ctag)::value;
        const int64_t warps = (rows_total + (32 / G) - 1) / (32 / G);
        const unsigned grid = grid_for(warps * 32, block);
        if (A->index_bits == 16)
            spmm_sell<T, G, C, 4, Cols16><<<grid, block, 0, st>>>(
                A->n, A->S, A->n_slices, k, A->slice_ptr.p, Cols16{A->sell_col16.p, A->col_start.p},
                val, X, Y);
        else
            spmm_sell<T, G, C, 4, Cols32><<<grid, block, 0, st>>>(
                A->n, A->S, A->n_slices, k, A->slice_ptr.p, Cols32{A->sell_col.p}, val, X, Y);
        GB_LAUNCHED();
        return SPMV_OK;
    };
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I4 = std::integral_constant<int, 4>;
    using I8 = std::integral_constant<int, 8>;
    using I16 = std::integral_constant<int, 16>;
    using I32 = std::integral_constant<int, 32>;
    if (k <= 1) return go(I1{}, I1{});
    if (k <= 2) return go(I2{}, I1{});
    if (k <= 4) return go(I4{}, I1{});
    if (k <= 8) return go(I8{}, I1{});
    if (k <= 16) return go(I16{}, I1{});
    if (k <= 32) return go(I32{}, I1{});
    return go(I32{}, I2{});
}

}  // namespace

spmv_status_t launch_spmm64(spmv_matrix_t A, int k, const double *X, double *Y, cudaStream_t st) {
    return launch_spmm<double>(A, k, A->sell_val.p, X, Y, st);
}

spmv_status_t launch_spmm32(spmv_matrix_t A, int k, const float *X, float *Y, cudaStream_t st) {
    return launch_spmm<float>(A, k, A->sell_val32.p, X, Y, st);
}

}  // namespace gb
