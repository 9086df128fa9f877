// chain.cu -- fused product of an operator chain y = B (C x) (not in the paper; its
// operator-based formulation, Sec. 2, evaluates a time step as chains of sparse products such
// as the divergence of a gradient).
//
// spmv_chain<R, L, ColT>: B in sliced ELLPACK (as spmv_sell), C in CSR.  For every entry b_if
// of a row of B the lane evaluates t_f = sum_j c_fj x_j over C's row f in column order with
// fused multiply-add from +0.0 -- exactly what spmv_apply(C) stores -- and accumulates
// b_if t_f in B's column order, so y equals spmv_apply(B) of spmv_apply(C) bit for bit while
// the intermediate vector C x is never written to or read back from HBM.  Each row of C is
// evaluated once per entry of B that names it (twice for the face operators of a mesh); the
// second evaluation finds C's row in L2 when B's rows follow C's numbering closely.
#include "common.cuh"
#include "ptx.cuh"

namespace gb {
namespace {

template <typename T, int R, int L, typename ColT>
__global__ void __launch_bounds__(1024)
spmv_chain(int32_t n, int32_t n_slices, const int64_t *__restrict__ sp, ColT cols,
           const T *__restrict__ bval, const int32_t *__restrict__ c_rp,
           const int32_t *__restrict__ c_ci, const T *__restrict__ c_val,
           const T *__restrict__ x, T *__restrict__ y) {
    constexpr int S = L * R;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t slice = gt / L;
    const int lane = (int)(gt % L);
    if (slice >= n_slices) return;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cbase = cols.base(slice);
    const uint64_t pol = policy_evict_first();
    T acc[R];
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = T(0);
    for (int t = 0; t < w; ++t) {
        T v[R];
        int32_t f[R];
        ld_stream(bval + base + (int64_t)t * S + lane * R, pol, v);
        cols.template load<R>(base + (int64_t)t * S + lane * R, slice, pol, cbase, f);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (f[i] < 0) continue;
            const int32_t k0 = __ldg(c_rp + f[i]), k1 = __ldg(c_rp + f[i] + 1);
            T tf = T(0);
            for (int32_t k = k0; k < k1; ++k)
                tf = fma_t(__ldg(c_val + k), __ldg(x + __ldg(c_ci + k)), tf);
            acc[i] = fma_t(v[i], tf, acc[i]);
        }
    }
    store_rows<T, R>(y, slice * S + (int64_t)lane * R, n, acc);
}

template <typename T, int R, int L>
spmv_status_t go_chain(spmv_matrix_t B, spmv_matrix_t C, const T *bval, const T *cval,
                       const T *x, T *y, cudaStream_t st) {
    const int block = 256;
    const int64_t threads = (int64_t)B->n_slices * L;
    const unsigned grid = (unsigned)((threads + block - 1) / block > 0 ? (threads + block - 1) / block : 1);
    if (B->index_bits == 16)
        spmv_chain<T, R, L, Cols16><<<grid, block, 0, st>>>(
            B->n, B->n_slices, B->slice_ptr.p, Cols16{B->sell_col16.p, B->col_start.p}, bval,
            C->row_ptr.p, C->col.p, cval, x, y);
    else
        spmv_chain<T, R, L, Cols32><<<grid, block, 0, st>>>(
            B->n, B->n_slices, B->slice_ptr.p, Cols32{B->sell_col.p}, bval, C->row_ptr.p,
            C->col.p, cval, x, y);
    GB_LAUNCHED();
    return SPMV_OK;
}

spmv_status_t check_chain(spmv_matrix_t B, spmv_matrix_t C, const void *x, const void *y) {
    if (!B || !C || B->n_cols != C->n) return SPMV_ERR_INVALID_ARG;
    if (B->perm.p || C->perm.p) return SPMV_ERR_INVALID_ARG;  // numberings must compose as given
    if (B->n > 0 && (!y || ((uintptr_t)y & 15u))) return SPMV_ERR_INVALID_ARG;
    if (C->n_cols > 0 && !x) return SPMV_ERR_INVALID_ARG;
    if (x == y) return SPMV_ERR_INVALID_ARG;
    return SPMV_OK;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" spmv_status_t spmv_apply_chain(spmv_matrix_t B, spmv_matrix_t C, const double *x,
                                          double *y, void *stream) {
    GB_TRY(check_chain(B, C, x, y));
    if (!B->has64() || !C->has64()) return SPMV_ERR_UNSUPPORTED;
    if (B->n == 0) return SPMV_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const double *bv = B->sell_val.p, *cv = C->val.p;
    switch (B->S) {
        case 32: return go_chain<double, 1, 32>(B, C, bv, cv, x, y, st);
        case 64: return go_chain<double, 2, 32>(B, C, bv, cv, x, y, st);
        case 128: return go_chain<double, 4, 32>(B, C, bv, cv, x, y, st);
        case 256: return go_chain<double, 8, 32>(B, C, bv, cv, x, y, st);
    }
    return SPMV_ERR_INVALID_ARG;
}

extern "C" spmv_status_t spmv_apply_chain_f32(spmv_matrix_t B, spmv_matrix_t C, const float *x,
                                              float *y, void *stream) {
    GB_TRY(check_chain(B, C, x, y));
    if (!B->has32() || !C->has32()) return SPMV_ERR_UNSUPPORTED;
    if (B->n == 0) return SPMV_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const float *bv = B->sell_val32.p, *cv = C->val32.p;
    switch (B->S) {  // (R, L) of the FP32 sliced kernels
        case 32: return go_chain<float, 4, 8>(B, C, bv, cv, x, y, st);
        case 64: return go_chain<float, 4, 16>(B, C, bv, cv, x, y, st);
        case 128: return go_chain<float, 4, 32>(B, C, bv, cv, x, y, st);
        case 256: return go_chain<float, 8, 32>(B, C, bv, cv, x, y, st);
    }
    return SPMV_ERR_INVALID_ARG;
}
