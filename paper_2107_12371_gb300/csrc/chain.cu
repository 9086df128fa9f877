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
// spmv_apply_chain runs either this kernel or the two sliced products through a temporary
// t = C x kept by B's handle (chosen by option or by timing both; see run_chain).
#include <algorithm>

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

template <typename T>
DevBuf<T> &chain_tmp(spmv_matrix_t B);
template <>
DevBuf<double> &chain_tmp<double>(spmv_matrix_t B) {
    return B->chain_t;
}
template <>
DevBuf<float> &chain_tmp<float>(spmv_matrix_t B) {
    return B->chain_t32;
}

spmv_status_t check_chain(spmv_matrix_t B, spmv_matrix_t C, const void *x, const void *y) {
    if (!B || !C || B->n_cols != C->n) return SPMV_ERR_INVALID_ARG;
    if (B->perm.p || C->perm.p) return SPMV_ERR_INVALID_ARG;  // numberings must compose as given
    if (B->n > 0 && (!y || ((uintptr_t)y & 15u))) return SPMV_ERR_INVALID_ARG;
    if (C->n_cols > 0 && !x) return SPMV_ERR_INVALID_ARG;
    if (x == y) return SPMV_ERR_INVALID_ARG;
    return SPMV_OK;
}

// Kernel launches of one form of the chain (fused kernel, or the two sliced products through
// the temporary t = C x that B's handle keeps).
template <typename T>
spmv_status_t chain_form_launch(spmv_matrix_t B, spmv_matrix_t C, int form, const T *x, T *y,
                                cudaStream_t st) {
    if (form == SPMV_CHAIN_TWO) {
        DevBuf<T> &t = chain_tmp<T>(B);
        if (t.n < (size_t)(C->n > 0 ? C->n : 1)) {
            AllocStream scope(st);
            GB_TRY(t.alloc((size_t)(C->n > 0 ? C->n : 1), &B->bytes));
        }
        if constexpr (sizeof(T) == 8) {
            GB_TRY(launch_spmv64(C, x, t.p, st));
            return launch_spmv64(B, t.p, y, st);
        } else {
            GB_TRY(launch_spmv32(C, x, t.p, st));
            return launch_spmv32(B, t.p, y, st);
        }
    }
    const T *bv, *cv;
    if constexpr (sizeof(T) == 8) {
        bv = B->sell_val.p;
        cv = C->val.p;
        switch (B->S) {
            case 32: return go_chain<T, 1, 32>(B, C, bv, cv, x, y, st);
            case 64: return go_chain<T, 2, 32>(B, C, bv, cv, x, y, st);
            case 128: return go_chain<T, 4, 32>(B, C, bv, cv, x, y, st);
            case 256: return go_chain<T, 8, 32>(B, C, bv, cv, x, y, st);
        }
    } else {
        bv = B->sell_val32.p;
        cv = C->val32.p;
        switch (B->S) {  // (R, L) of the FP32 sliced kernels
            case 32: return go_chain<T, 4, 8>(B, C, bv, cv, x, y, st);
            case 64: return go_chain<T, 4, 16>(B, C, bv, cv, x, y, st);
            case 128: return go_chain<T, 4, 32>(B, C, bv, cv, x, y, st);
            case 256: return go_chain<T, 8, 32>(B, C, bv, cv, x, y, st);
        }
    }
    return SPMV_ERR_INVALID_ARG;
}

// Form for this call: B's option, else B's tuned pick for the precision, else (untuned) the
// two products, measured faster on GB300 in both precisions (t = C x stays in L2 between them,
// while the fused kernel evaluates each row of C once per entry of B that names it).  With
// autotune on, the first call times both forms (the median of three launches each after
// overwriting L2) and keeps the faster; either form leaves the same y.
template <typename T>
spmv_status_t run_chain(spmv_matrix_t B, spmv_matrix_t C, const T *x, T *y, cudaStream_t st) {
    if (B->opt.chain_form != SPMV_CHAIN_AUTO)
        return chain_form_launch<T>(B, C, B->opt.chain_form, x, y, st);
    int &pick = B->chain_pick[sizeof(T) == 4 ? 1 : 0];
    if (pick == SPMV_CHAIN_AUTO && B->opt.autotune) {
        const size_t fb = 2 * (size_t)(device_facts().l2_bytes > 0 ? device_facts().l2_bytes
                                                                   : (128 << 20));
        void *flush = nullptr;
        {
            AllocStream scope(st);
            GB_CUDA(gb_malloc_async(&flush, fb, st));
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        spmv_status_t s = cuda_status(cudaEventCreate(&e0));
        if (s == SPMV_OK) s = cuda_status(cudaEventCreate(&e1));
        float best = 1e30f;
        int best_form = SPMV_CHAIN_TWO;
        for (int form : {SPMV_CHAIN_FUSED, SPMV_CHAIN_TWO}) {
            float t[3] = {0.f, 0.f, 0.f};
            for (int i = -1; i < 3 && s == SPMV_OK; ++i) {  // i = -1: warm-up
                s = cuda_status(cudaMemsetAsync(flush, i + 2, fb, st));
                if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e0, st));
                if (s == SPMV_OK) s = chain_form_launch<T>(B, C, form, x, y, st);
                if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e1, st));
                if (s == SPMV_OK) s = cuda_status(cudaEventSynchronize(e1));
                if (s == SPMV_OK && i >= 0) s = cuda_status(cudaEventElapsedTime(&t[i], e0, e1));
            }
            if (s != SPMV_OK) break;
            const float med =
                std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
            if (med < best) {
                best = med;
                best_form = form;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFreeAsync(flush, st);
        GB_TRY(s);
        pick = best_form;
    }
    return chain_form_launch<T>(B, C, pick == SPMV_CHAIN_AUTO ? SPMV_CHAIN_TWO : pick, x, y, st);
}

}  // namespace

int chain_form_of(const spmv_matrix_t B, bool f32) {
    if (B->opt.chain_form != SPMV_CHAIN_AUTO) return B->opt.chain_form;
    const int p = B->chain_pick[f32 ? 1 : 0];
    return p == SPMV_CHAIN_AUTO ? SPMV_CHAIN_TWO : p;
}

}  // namespace gb

using namespace gb;

extern "C" spmv_status_t spmv_apply_chain(spmv_matrix_t B, spmv_matrix_t C, const double *x,
                                          double *y, void *stream) {
    GB_TRY(check_chain(B, C, x, y));
    if (!B->has64() || !C->has64()) return SPMV_ERR_UNSUPPORTED;
    if (B->n == 0) return SPMV_OK;
    return run_chain<double>(B, C, x, y, (cudaStream_t)stream);
}

extern "C" spmv_status_t spmv_apply_chain_f32(spmv_matrix_t B, spmv_matrix_t C, const float *x,
                                              float *y, void *stream) {
    GB_TRY(check_chain(B, C, x, y));
    if (!B->has32() || !C->has32()) return SPMV_ERR_UNSUPPORTED;
    if (B->n == 0) return SPMV_OK;
    return run_chain<float>(B, C, x, y, (cudaStream_t)stream);
}
