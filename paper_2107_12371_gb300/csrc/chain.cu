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

template <int R, int L, typename ColT>
__global__ void __launch_bounds__(1024)
spmv_chain(int32_t n, int32_t n_slices, const int64_t *__restrict__ sp, ColT cols,
           const double *__restrict__ bval, const int32_t *__restrict__ c_rp,
           const int32_t *__restrict__ c_ci, const double *__restrict__ c_val,
           const double *__restrict__ x, double *__restrict__ y) {
    constexpr int S = L * R;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t slice = gt / L;
    const int lane = (int)(gt % L);
    if (slice >= n_slices) return;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cbase = cols.base(slice);
    const uint64_t pol = policy_evict_first();
    double acc[R];
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = 0.0;
    for (int t = 0; t < w; ++t) {
        double v[R];
        int32_t f[R];
        ld_stream(bval + base + (int64_t)t * S + lane * R, pol, v);
        cols.template load<R>(base + (int64_t)t * S + lane * R, slice, pol, cbase, f);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (f[i] < 0) continue;
            const int32_t k0 = __ldg(c_rp + f[i]), k1 = __ldg(c_rp + f[i] + 1);
            double tf = 0.0;
            for (int32_t k = k0; k < k1; ++k) tf = fma(__ldg(c_val + k), __ldg(x + __ldg(c_ci + k)), tf);
            acc[i] = fma(v[i], tf, acc[i]);
        }
    }
    store_rows<double, R>(y, slice * S + (int64_t)lane * R, n, acc);
}

template <int R, int L>
spmv_status_t go_chain(spmv_matrix_t B, spmv_matrix_t C, const double *x, double *y,
                       cudaStream_t st) {
    const int block = 256;
    const int64_t threads = (int64_t)B->n_slices * L;
    const unsigned grid = (unsigned)((threads + block - 1) / block > 0 ? (threads + block - 1) / block : 1);
    if (B->index_bits == 16)
        spmv_chain<R, L, Cols16><<<grid, block, 0, st>>>(
            B->n, B->n_slices, B->slice_ptr.p, Cols16{B->sell_col16.p, B->col_start.p},
            B->sell_val.p, C->row_ptr.p, C->col.p, C->val.p, x, y);
    else
        spmv_chain<R, L, Cols32><<<grid, block, 0, st>>>(
            B->n, B->n_slices, B->slice_ptr.p, Cols32{B->sell_col.p}, B->sell_val.p,
            C->row_ptr.p, C->col.p, C->val.p, x, y);
    GB_LAUNCHED();
    return SPMV_OK;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" spmv_status_t spmv_apply_chain(spmv_matrix_t B, spmv_matrix_t C, const double *x,
                                          double *y, void *stream) {
    if (!B || !C || B->n_cols != C->n) return SPMV_ERR_INVALID_ARG;
    if (B->perm.p || C->perm.p) return SPMV_ERR_INVALID_ARG;  // numberings must compose as given
    if (!B->has64() || !C->has64()) return SPMV_ERR_UNSUPPORTED;
    if (B->n > 0 && (!y || ((uintptr_t)y & 15u))) return SPMV_ERR_INVALID_ARG;
    if (C->n_cols > 0 && !x) return SPMV_ERR_INVALID_ARG;
    if ((const void *)x == (const void *)y) return SPMV_ERR_INVALID_ARG;
    if (B->n == 0) return SPMV_OK;
    cudaStream_t st = (cudaStream_t)stream;
    switch (B->S) {
        case 32: return go_chain<1, 32>(B, C, x, y, st);
        case 64: return go_chain<2, 32>(B, C, x, y, st);
        case 128: return go_chain<4, 32>(B, C, x, y, st);
        case 256: return go_chain<8, 32>(B, C, x, y, st);
    }
    return SPMV_ERR_INVALID_ARG;
}
