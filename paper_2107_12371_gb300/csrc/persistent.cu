// persistent.cu -- a whole Jacobi-PCG loop in one cooperative kernel (FP64 solves, and the FP32
// inner solves of iterative refinement).
//
// Every CTA of a co-resident grid (cooperative launch) runs the iterations; the three phases
// of an iteration (q = A p with p.q; x/r update with r.z and r.r; p update) are separated by a
// grid barrier.  After each barrier every CTA sums the per-CTA partials of the previous phase
// in the same fixed order, so all CTAs hold bit-identical scalars and take identical branch
// decisions.  The results equal the graph-launched path's (same per-CTA partitions, same
// reduction trees).  Every barrier wait is bounded: after 2 s without progress the waiting
// CTA records done = 4 (timeout) and the whole grid leaves the loop, so a fault can never
// leave the GPU spinning.  p, q, r and x change while the kernel runs, so they are read with
// coherent loads only (never through the read-only .nc path).
#include "cgkern.cuh"

namespace gb {
namespace {

__device__ __forceinline__ long long global_timer_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr long long kBarrierLimitNs = 2000000000LL;

// Grid barrier over `expected` CTAs (gridDim.x in the solver).  A CTA that waits longer than
// limit_ns records done = 4 and returns false instead of spinning on.
__device__ bool grid_barrier(CgScalars *sc, unsigned expected = 0,
                             long long limit_ns = kBarrierLimitNs) {
    __shared__ int ok;
    if (expected == 0) expected = gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *genp = &sc->bar_gen;
        const unsigned g = *genp;
        __threadfence();
        const unsigned arrived = atomicAdd(&sc->bar_count, 1u);
        int good = 1;
        if (arrived == expected - 1) {
            atomicExch(&sc->bar_count, 0u);
            __threadfence();
            atomicAdd(&sc->bar_gen, 1u);
        } else {
            const long long t0 = global_timer_ns();
            while (*genp == g) {
                if (global_timer_ns() - t0 > limit_ns) {
                    good = 0;
                    atomicExch(&sc->done, 4);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// sum of part[k * count + i] over i < count in the fixed order of grid_sum_last, broadcast
// to all threads
template <int NV>
__device__ void reduce_parts(const double *part, int count, double (&tot)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        tot[k] = 0.0;
        for (int i = threadIdx.x; i < count; i += kCgBlock)
            tot[k] += __ldcg(part + (int64_t)k * count + i);
    }
    block_sum_all<NV>(tot);
}

template <int NV>
__device__ void store_parts(double (&v)[NV], double *part) {
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[k * gridDim.x + blockIdx.x] = v[k];
    }
}

template <typename T, int R, int L, typename ColT>
__global__ void __launch_bounds__(kCgBlock, kCgCtasPerSm)
cg_persistent(int32_t n, int32_t n_slices, const int64_t *sp, ColT col, const T *val, T *x,
              T *r, T *p, T *q, const T *dinv, double *part, int32_t Gpq, int32_t pq_len,
              int deep, CgScalars *sc) {
    constexpr int S = L * R;
    const uint64_t pol = policy_evict_first();
    const long long t_start = global_timer_ns();
    const long long budget = sc->budget_ns;
    double rho = sc->rho;
    const double bb = sc->bb, tol2 = sc->tol2;
    int iters = sc->iters;
    const int max_iter = sc->max_iter;
    int done = sc->done;
    // the product's p.q partials (one per CTA of its grid), the sweep's r.z and r.r per CTA,
    // then CTA 0's stop vote
    double *part1 = part;
    double *part2 = part + pq_len;
    double *vote = part + pq_len + 2 * gridDim.x;
    const int64_t tasks = (int64_t)n_slices * L;
    const int64_t pq_lanes = (int64_t)Gpq * kCgBlock;
    double beta = 0.0;
    while (!done) {
        // phase 1: q = A p, p.q on the product grid of the graph path (cg_pq_grid): its CTA b
        // runs here as a virtual CTA on CTA b mod gridDim.x, with the same grid-stride order
        // and the same CTA tree
        for (int b = blockIdx.x; b < Gpq; b += gridDim.x) {
            T vt = T(0);
            for (int64_t g = (int64_t)b * kCgBlock + threadIdx.x; g < tasks; g += pq_lanes) {
                const int64_t slice = g / L;
                const int lane = (int)(g % L);
                T acc[R];
                // entries in flight as in the graph path's product (the order, hence the
                // result, is the same either way)
                if (deep)
                    slice_rows<T, R, L, true, pq_unroll((int)sizeof(T) * R)>(slice, lane, sp, col,
                                                                           val, p, pol, acc);
                else
                    slice_rows<T, R, L, true>(slice, lane, sp, col, val, p, pol, acc);
                const int64_t row0 = slice * S + (int64_t)lane * R;
                store_rows<T, R>(q, row0, n, acc);
#pragma unroll
                for (int i = 0; i < R; ++i)
                    if (row0 + i < n) vt = fma_t(p[row0 + i], acc[i], vt);
            }
            double v1[1] = {(double)vt};
            block_sum<1>(v1);
            if (threadIdx.x == 0) part1[b] = v1[0];
        }
        // CTA 0's vote to stop on the wall-clock budget
        if (blockIdx.x == 0 && threadIdx.x == 0)
            vote[0] = (budget > 0 && global_timer_ns() - t_start > budget) ? 1.0 : 0.0;
        if (!grid_barrier(sc)) {
            done = 4;
            break;
        }
        double t1[1];
        reduce_parts<1>(part1, Gpq, t1);
        if (__ldcg(vote) != 0.0) {
            done = 4;
            break;
        }
        if (t1[0] == 0.0 || !isfinite(t1[0])) {
            done = 3;
            break;
        }
        const T alpha = (T)(rho / t1[0]);
        // phase 2: x += alpha p, r -= alpha q, r.z, r.r
        T vz = T(0), vr = T(0);
        sweep_update_xr<T>(n, alpha, x, r, p, q, dinv, vz, vr);
        double v2[2] = {(double)vz, (double)vr};
        store_parts<2>(v2, part2);
        if (!grid_barrier(sc)) {
            done = 4;
            break;
        }
        double t2[2];
        reduce_parts<2>(part2, (int)gridDim.x, t2);
        beta = t2[0] / rho;
        rho = t2[0];
        ++iters;
        if (t2[1] <= tol2 * bb) done = 1;
        else if (!isfinite(t2[1])) done = 3;
        else if (iters >= max_iter) done = 2;
        if (done) {
            if (blockIdx.x == 0 && threadIdx.x == 0) sc->rr = t2[1];
            break;
        }
        // phase 3: p = D^-1 r + beta p
        sweep_update_p<T>(n, (T)beta, r, dinv, p);
        if (!grid_barrier(sc)) {
            done = 4;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (done == 4) atomicExch(&sc->done, 4);
        else atomicCAS(&sc->done, 0, done);
        sc->iters = iters;
        sc->rho = rho;
        sc->beta = beta;
    }
}

// Diagnostic: a barrier that expects one CTA more than the grid has, so no wait can ever be
// released -- every CTA must leave through the time limit and record done = 4.
__global__ void barrier_timeout_probe(CgScalars *sc, long long limit_ns) {
    grid_barrier(sc, gridDim.x + 1, limit_ns);
}

}  // namespace

spmv_status_t diag_barrier_timeout(int ctas, double limit_s, int *done_out, cudaStream_t st) {
    CgScalars *sc = nullptr;
    GB_CUDA(gb_malloc_async((void **)&sc, sizeof(CgScalars), st));
    spmv_status_t s = cuda_status(cudaMemsetAsync(sc, 0, sizeof(CgScalars), st));
    long long limit_ns = (long long)(limit_s * 1e9);
    void *args[] = {&sc, &limit_ns};
    if (s == SPMV_OK)
        s = cuda_status(cudaLaunchCooperativeKernel((const void *)barrier_timeout_probe,
                                                    dim3(ctas), dim3(32), args, 0, st));
    CgScalars h{};
    if (s == SPMV_OK)
        s = cuda_status(cudaMemcpyAsync(&h, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
    cudaFreeAsync(sc, st);
    cudaStreamSynchronize(st);
    *done_out = h.done;
    return s;
}

// One cooperative launch running the recurrence to its end; FP64 (outer scalars, FP64 work
// vectors) or FP32 (inner scalars of the refinement, FP32 work vectors and values).
static spmv_status_t run_persistent(spmv_matrix_t A, bool f32, const cg_options_t &o,
                                    CgScalars *out, cudaStream_t st) {
    CgWork &w = A->cg;
    CgScalars *sc = (CgScalars *)w.scal.p + (f32 ? 1 : 0);
    auto launch = [&](auto tag, auto cols) -> spmv_status_t {
        using T = decltype(tag);
        using ColT = decltype(cols);
        return with_shape(A->S, f32, [&](auto rt, auto lt) -> spmv_status_t {
            constexpr int R = decltype(rt)::value, L = decltype(lt)::value;
            auto kern = cg_persistent<T, R, L, ColT>;
            int per_sm = 0;
            GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCgBlock, 0));
            // the grid must be co-resident and equal to the graph path's grid
            if (per_sm < kCgCtasPerSm) return SPMV_ERR_UNSUPPORTED;
            w.pers_grid = cg_grid(A->n);
            const long long budget = o.timeout_s > 0 ? (long long)(o.timeout_s * 1e9) : 0;
            GB_CUDA(cudaMemcpyAsync(&sc->budget_ns, &budget, sizeof(budget),
                                    cudaMemcpyHostToDevice, st));
            int32_t n = A->n, ns = A->n_slices;
            const int64_t *sp = A->slice_ptr.p;
            const T *val;
            T *x, *r, *p, *q;
            const T *dinv;
            if constexpr (sizeof(T) == 8) {
                val = A->sell_val.p;
                x = w.x.p, r = w.r.p, p = w.p.p, q = w.q.p, dinv = w.dinv.p;
            } else {
                val = A->sell_val32.p;
                x = w.d32.p, r = w.r32.p, p = w.p32.p, q = w.q32.p, dinv = w.dinv32.p;
            }
            double *part = w.part.p;
            // the graph path's product grid for this shape (see cg_pq_grid)
            int32_t Gpq = cg_pq_grid(A, L, (int)sizeof(T) * R);
            int32_t pq_len = w.pq_len;
            constexpr int UU = pq_unroll((int)sizeof(T) * R);
            int deep = cg_pq_deep(A, UU) ? 1 : 0;
            void *args[] = {&n, &ns, &sp, &cols, &val, &x, &r, &p, &q, &dinv, &part, &Gpq,
                            &pq_len, &deep, &sc};
            GB_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3(w.pers_grid),
                                                dim3(kCgBlock), args, 0, st));
            GB_CUDA(cudaMemcpyAsync(w.h_scal, w.scal.p, 2 * sizeof(CgScalars),
                                    cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaStreamSynchronize(st));
            *out = w.h_scal[f32 ? 1 : 0];
            return SPMV_OK;
        });
    };
    auto by_cols = [&](auto tag) -> spmv_status_t {
        if (A->index_bits == 16) return launch(tag, Cols16{A->sell_col16.p, A->col_start.p});
        return launch(tag, Cols32{A->sell_col.p});
    };
    if (f32) return by_cols(float{});
    return by_cols(double{});
}

spmv_status_t cg_persistent64(spmv_matrix_t A, const cg_options_t &o, CgScalars *out,
                              cudaStream_t st) {
    return run_persistent(A, false, o, out, st);
}

spmv_status_t cg_persistent32(spmv_matrix_t A, const cg_options_t &o, CgScalars *out,
                              cudaStream_t st) {
    return run_persistent(A, true, o, out, st);
}

}  // namespace gb
