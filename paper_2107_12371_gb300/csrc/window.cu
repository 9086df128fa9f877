// window.cu -- sliced-ELLPACK SpMV with x staged in a circular shared-memory window, the GPU
// counterpart of the paper's cached SpMV (Sec. 5.1-5.2).
//
// Each CTA (one per SM, 1024 threads) owns a contiguous run of slices and walks it in rounds
// of Q slices (one or two slices per warp).  Before a round it computes the round's column
// range [lo, hi) from the per-slice col_start / col_end and loads into the window only the
// columns it does not hold yet (hi_prev .. hi, coalesced), overwriting the oldest ones: the
// window is a circular list of W entries, entry c at position c mod W.  The round's gathers
// then read shared memory.  If a round's range does not fit (lo < hi - W), the window restarts
// at lo; if even that does not fit, the round gathers x from global memory instead.  Every row
// sums its entries in column order with fused multiply-add, exactly as spmv_sell, so the
// result is bit-identical.
#include <climits>

#include "common.cuh"
#include "ptx.cuh"

namespace gb {
namespace {

constexpr int kWinThreads = 1024;
constexpr int kWinBytes = 192 * 1024;

template <typename T>
constexpr int win_entries() {
    return kWinBytes / (int)sizeof(T);
}

template <typename T, int R, int L, typename ColT>
__global__ void __launch_bounds__(kWinThreads, 1)
spmv_sell_window(int32_t n, int32_t n_slices, const int64_t *__restrict__ sp, ColT cols,
                 const int32_t *__restrict__ cs, const int32_t *__restrict__ ce,
                 const T *__restrict__ val, const T *__restrict__ x, T *__restrict__ y,
                 int32_t slices_per_cta) {
    constexpr int32_t W = win_entries<T>();  // compile-time: c % W is a multiply-shift
    extern __shared__ __align__(16) unsigned char win_raw[];
    T *win = reinterpret_cast<T *>(win_raw);
    __shared__ int32_t r_lo, r_hi;
    constexpr int S = L * R;
    constexpr int SPW = 32 / L;  // slices per warp
    const int Q = (kWinThreads / 32) * SPW;
    const int64_t s_begin = (int64_t)blockIdx.x * slices_per_cta;
    const int64_t s_end = s_begin + slices_per_cta < n_slices ? s_begin + slices_per_cta : n_slices;
    const int warp = threadIdx.x >> 5, lane32 = threadIdx.x & 31;
    const int lane = lane32 % L;
    const uint64_t pol = policy_evict_first();
    int32_t hi = INT_MIN, lo_valid = INT_MAX;  // window holds [lo_valid, hi)
    for (int64_t s0 = s_begin; s0 < s_end; s0 += Q) {
        // column range of the round
        if (threadIdx.x == 0) {
            r_lo = INT_MAX;
            r_hi = INT_MIN;
        }
        __syncthreads();
        if (threadIdx.x < Q && s0 + threadIdx.x < s_end) {
            const int64_t s = s0 + threadIdx.x;
            if (ce[s] > cs[s]) {
                atomicMin(&r_lo, cs[s]);
                atomicMax(&r_hi, ce[s]);
            }
        }
        __syncthreads();
        const int32_t lo = r_lo, rh = r_hi;
        bool use_win = false;
        if (lo < rh) {
            int32_t from, to;
            if (hi != INT_MIN && lo >= lo_valid && (rh <= hi || lo >= (rh > hi ? rh : hi) - W)) {
                // delta: add (hi, rh]; the oldest entries drop out of the window
                from = hi;
                to = rh > hi ? rh : hi;
                use_win = true;
            } else if (rh - lo <= W) {
                from = lo;  // restart the window at the round's first column
                to = rh;
                lo_valid = lo;
                use_win = true;
            } else {
                from = to = 0;
            }
            if (use_win) {
                for (int32_t c = from + (int32_t)threadIdx.x; c < to; c += kWinThreads)
                    win[c % W] = __ldg(x + c);
                hi = to;
                if (hi - W > lo_valid) lo_valid = hi - W;
            }
            __syncthreads();
        }
        // the round's slices: warp w takes slices s0 + w SPW .. s0 + w SPW + SPW - 1
        const int64_t slice = s0 + (int64_t)warp * SPW + lane32 / L;
        if (slice < s_end) {
            const int64_t base = sp[slice];
            const int w = (int)((sp[slice + 1] - base) / S);
            const int32_t cbase = cols.base(slice);
            const T *vp = val + base + lane * R;
            const int64_t cat = base + lane * R;
            T acc[R];
#pragma unroll
            for (int i = 0; i < R; ++i) acc[i] = T(0);
            for (int t = 0; t < w; ++t) {
                T v[R];
                int32_t c[R];
                ld_stream(vp + (int64_t)t * S, pol, v);
                cols.template load<R>(cat + (int64_t)t * S, slice, pol, cbase, c);
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    if (c[i] >= 0) {
                        const T xv = use_win ? win[c[i] % W] : __ldg(x + c[i]);
                        acc[i] = fma_t(v[i], xv, acc[i]);
                    }
                }
            }
            store_rows<T, R>(y, slice * S + (int64_t)lane * R, n, acc);
        }
        __syncthreads();  // the next round's loads overwrite the oldest entries
    }
}

template <typename T, int R, int L>
spmv_status_t go_window(spmv_matrix_t A, const T *val, const T *x, T *y, cudaStream_t st) {
    const int smem = kWinBytes;
    const int Q = (kWinThreads / 32) * (32 / L);
    const int G = device_facts().sm_count;
    int64_t per = ((int64_t)A->n_slices + G - 1) / G;
    per = (per + Q - 1) / Q * Q;
    const unsigned grid = (unsigned)(((int64_t)A->n_slices + per - 1) / per);
    auto run = [&](auto kern, auto cols) -> spmv_status_t {
        GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        kern<<<grid, kWinThreads, smem, st>>>(A->n, A->n_slices, A->slice_ptr.p, cols,
                                              A->col_start.p, A->col_end.p, val, x, y,
                                              (int32_t)per);
        GB_LAUNCHED();
        return SPMV_OK;
    };
    if (A->index_bits == 16)
        return run(spmv_sell_window<T, R, L, Cols16>, Cols16{A->sell_col16.p, A->col_start.p});
    return run(spmv_sell_window<T, R, L, Cols32>, Cols32{A->sell_col.p});
}

}  // namespace

int window_capacity_words(int elem_bytes) { return kWinBytes / elem_bytes; }

spmv_status_t launch_window64(spmv_matrix_t A, const double *x, double *y, cudaStream_t st) {
    if (A->n == 0) return SPMV_OK;
    switch (A->S) {
        case 32: return go_window<double, 1, 32>(A, A->sell_val.p, x, y, st);
        case 64: return go_window<double, 2, 32>(A, A->sell_val.p, x, y, st);
        case 128: return go_window<double, 4, 32>(A, A->sell_val.p, x, y, st);
        case 256: return go_window<double, 8, 32>(A, A->sell_val.p, x, y, st);
    }
    return SPMV_ERR_INVALID_ARG;
}

spmv_status_t launch_window32(spmv_matrix_t A, const float *x, float *y, cudaStream_t st) {
    if (A->n == 0) return SPMV_OK;
    switch (A->S) {
        case 32: return go_window<float, 4, 8>(A, A->sell_val32.p, x, y, st);
        case 64: return go_window<float, 4, 16>(A, A->sell_val32.p, x, y, st);
        case 128: return go_window<float, 4, 32>(A, A->sell_val32.p, x, y, st);
        case 256: return go_window<float, 8, 32>(A, A->sell_val32.p, x, y, st);
    }
    return SPMV_ERR_INVALID_ARG;
}

}  // namespace gb
