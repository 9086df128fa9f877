// mcg.cu -- Jacobi-preconditioned CG for k right-hand sides in lock-step (cg_solve_multi).
// Not in the paper: the paper's linear solver is SpMV-bound (Sec. 2); batching k systems that
// share one matrix turns k products into one multi-vector product (Y = A X) in which every
// gathered matrix entry and every streamed slice is used for all k columns.
//
// The k systems are the columns of row-major n x KP arrays (KP = k rounded up to 8, 16 or 32;
// the extra columns have b = 0 and are done from the start).  Each column keeps its own
// alpha, beta, rho and stop state; a column that has converged keeps its x and drops out of
// the updates.  One iteration is three kernels (graph-launched) or three phases of one
// cooperative kernel (persistent), with the same per-CTA partitions and reduction trees, so
// both forms give bit-identical results:
//   product  Q = A P (each lane gathers a 32- or 16-byte piece of a row of P), p_c.q_c
//            -> alpha_c = rho_c / (p_c.q_c)
//   r sweep  r_c -= alpha_c q_c, r_c.(D^-1 r_c), r_c.r_c -> beta_c, rho_c, convergence
//   p sweep  x_c += alpha_c p_c (the x update of the same iteration, applied here where p_c is
//            read anyway: one pass over P fewer), p_c = D^-1 r_c + beta_c p_c
// Every per-column sum is reduced deterministically: per CTA in a fixed tree, then over the
// CTAs in a fixed order (by the last CTA to arrive, or by every CTA after a grid barrier).
//
// With opt->mixed the same kernels run in FP32 as the inner solves of FP64 iterative
// refinement (per column: FP64 residual, FP32 inner Jacobi-PCG on r_c / ||r_c|| to the inner
// tolerance of the single-RHS refinement, FP64 update x_c += ||r_c|| d_c).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "cgkern.cuh"

namespace gb {

spmv_status_t ensure_cg_work(spmv_matrix_t A, bool mixed, cudaStream_t st);

constexpr int kMcgMaxCols = 32;
constexpr int kMcgWarps = kCgBlock / 32;

// State of one column's recurrence.
struct McgCol {
    double alpha, beta, rho, rr, bb, tol2, s, inv_s;
    int done;      // 0 running, 1 converged, 2 iteration cap, 3 breakdown
    int iters;     // iterations of this recurrence (inner solve: of this inner solve)
    int upd;       // updated by the last r sweep: its x update is applied by the p sweep
    int restarts;  // true-residual restarts (FP64) / refinement steps (outer block, mixed)
    int total;     // outer block, mixed: inner iterations summed over the refinement steps
    int pad[3];
};

struct McgScalars {
    McgCol col[kMcgMaxCols];
    int active;      // columns with done == 0
    int pending;     // an r sweep ran since the last product: the p sweep applies
    int max_iter;
    int timed_out;   // persistent kernel: a grid-barrier wait or the wall-clock budget ran out
    unsigned tickets[4];
    unsigned bar_count, bar_gen;
    long long budget_ns;
};

// Host-side work of a handle's multi-RHS solves (allocated on the first call, kept).
struct McgWork {
    int kp = 0;
    DevBuf<double> X, R, P, Q, B;      // n x kp, row-major
    DevBuf<float> R32, P32, Q32, D32;  // inner solves of the refinement
    DevBuf<double> part;               // per-CTA partial sums
    DevBuf<McgScalars> scal;           // [0] FP64 / outer, [1] inner
    McgScalars h[2];
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // batches of iterations (FP64, FP32)
    int graph_iters[2] = {0, 0};
    int graph_gw[2] = {0, 0};
};

namespace {

// ---- 16- and 32-byte accesses of a row piece ------------------------------------------------
template <typename T, int BYTES>
struct Piece {
    static constexpr int n = BYTES / (int)sizeof(T);
};

// read-only (.nc) gather: for arrays no thread writes while the kernel runs
template <int BYTES, typename T>
__device__ __forceinline__ void ld_piece_nc(const T *p, T (&v)[Piece<T, BYTES>::n]) {
    if constexpr (BYTES == 32 && sizeof(T) == 8) {
        asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
            : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
    } else if constexpr (BYTES == 32) {
        asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
              "=f"(v[6]), "=f"(v[7])
            : "l"(p));
    } else if constexpr (sizeof(T) == 8) {
        asm("ld.global.nc.v2.f64 {%0,%1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "l"(p));
    } else {
        asm("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
            : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p));
    }
}

// coherent gather (weak ld.global, L1 allocating): for the persistent kernel, where other CTAs
// rewrite the array between grid barriers
template <int BYTES, typename T>
__device__ __forceinline__ void ld_piece_co(const T *p, T (&v)[Piece<T, BYTES>::n]) {
    if constexpr (BYTES == 32 && sizeof(T) == 8) {
        asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                     : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p) : "memory");
    } else if constexpr (BYTES == 32) {
        asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                       "=f"(v[6]), "=f"(v[7])
                     : "l"(p) : "memory");
    } else if constexpr (sizeof(T) == 8) {
        asm volatile("ld.global.v2.f64 {%0,%1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "l"(p) : "memory");
    } else {
        asm volatile("ld.global.v4.f32 {%0,%1,%2,%3}, [%4];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p) : "memory");
    }
}

template <int BYTES, bool COH, typename T>
__device__ __forceinline__ void ld_piece(const T *p, T (&v)[Piece<T, BYTES>::n]) {
    if constexpr (COH) ld_piece_co<BYTES>(p, v);
    else ld_piece_nc<BYTES>(p, v);
}

template <int BYTES, typename T>
__device__ __forceinline__ void st_piece(T *p, const T (&v)[Piece<T, BYTES>::n]) {
    if constexpr (BYTES == 32 && sizeof(T) == 8) {
        asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]),
                     "d"(v[2]), "d"(v[3]) : "memory");
    } else if constexpr (BYTES == 32) {
        asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]),
                     "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                     : "memory");
    } else if constexpr (sizeof(T) == 8) {
        asm volatile("st.global.v2.f64 [%0], {%1,%2};" ::"l"(p), "d"(v[0]), "d"(v[1]) : "memory");
    } else {
        asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                     "f"(v[2]), "f"(v[3]) : "memory");
    }
}

// ---- deterministic per-column reductions ------------------------------------------------------
// v[q][j]: this thread's partial of quantity q for column (lane % CG) * V + j; lanes of a warp
// with the same lane % CG hold the same columns.  The CTA's sums (fixed shuffle tree, then the
// warps in order) go to part[(q * KP + c) * vgrid + vb].
template <int CG, int V, int NQ>
__device__ __forceinline__ void cta_cols(double (&v)[NQ][V], double *part, int vb, int vgrid) {
    constexpr int KP = CG * V;
    __shared__ double sh[NQ][kMcgWarps][KP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int j = 0; j < V; ++j)
#pragma unroll
            for (int o = CG; o < 32; o <<= 1) v[q][j] += __shfl_xor_sync(0xffffffffu, v[q][j], o);
    __syncthreads();  // sh may still be read by a previous call's final loop
    if (lane < CG) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int j = 0; j < V; ++j) sh[q][warp][lane * V + j] = v[q][j];
    }
    __syncthreads();
    if (threadIdx.x < KP) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kMcgWarps; ++w) s += sh[q][w][threadIdx.x];
            part[(int64_t)(q * KP + threadIdx.x) * vgrid + vb] = s;
        }
        __threadfence();
    }
}

// tot[q][c] = the sum over i < count of part[(q * KP + c) * count + i], in a fixed order
// (warp w takes (q, c) pairs w, w + 8, ...; its lanes stride over i; a fixed shuffle tree).
// Valid in every thread after return.
template <int KP, int NQ>
__device__ __forceinline__ void grid_cols(const double *part, int count, double (&tot)[NQ][KP]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int qc = warp; qc < NQ * KP; qc += kMcgWarps) {
        const double *pp = part + (int64_t)qc * count;
        double s = 0.0;
        for (int i = lane; i < count; i += 32) s += __ldcg(pp + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) tot[qc / KP][qc % KP] = s;
    }
    __syncthreads();
}

// true in the CTA that arrives last at `ticket` (which is reset for the next launch)
__device__ __forceinline__ bool last_cta(unsigned *ticket) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (last) *ticket = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// ---- per-column scalar updates (shared by the graph kernels and the persistent kernel) ------
__device__ __forceinline__ void col_after_pq(McgCol &c, double pq) {
    if (c.done) return;
    if (pq == 0.0 || !isfinite(pq)) c.done = 3;
    else c.alpha = c.rho / pq;
}

__device__ __forceinline__ void col_after_r(McgCol &c, double rz, double rr, int max_iter) {
    c.upd = c.done == 0 ? 1 : 0;
    if (c.done) return;
    c.beta = rz / c.rho;
    c.rho = rz;
    c.rr = rr;
    c.iters += 1;
    if (rr <= c.tol2 * c.bb) c.done = 1;
    else if (!isfinite(rr)) c.done = 3;
    else if (c.iters >= max_iter) c.done = 2;
}

// ---- phase bodies (virtual CTA vb of a grid of vgrid CTAs) -----------------------------------
// Q = A P and per-column p.q.  G lanes per row, each owning a BYTES-wide piece (VW columns) of
// the row; entries two at a time so two gathers are in flight, in stored order with fused
// multiply-add from +0.0 (column c of Q equals spmv_apply on column c of P bit for bit).
template <typename T, int G, int BYTES, bool COH, typename ColT>
__device__ __forceinline__ void product_phase(int vb, int vgrid, int32_t n, int32_t S,
                                              int32_t n_slices, const int64_t *__restrict__ sp,
                                              ColT cols, const T *__restrict__ val, const T *P,
                                              T *Q, double *part) {
    constexpr int VW = Piece<T, BYTES>::n;
    constexpr int KP = VW * G;
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / G, g = lane % G;
    const int64_t groups = (int64_t)n_slices * S / RPW;
    const uint64_t pol = policy_evict_first();
    double pq[1][VW];
    T pqt[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) pqt[j] = T(0);
    for (int64_t wg = (int64_t)vb * kMcgWarps + warp; wg < groups;
         wg += (int64_t)vgrid * kMcgWarps) {
        const int64_t row0 = wg * RPW;
        const int64_t row = row0 + sub;
        const int64_t slice = row0 / S;
        const int64_t r = row - slice * S;
        const int64_t base = sp[slice];
        const int w = (int)((sp[slice + 1] - base) / S);
        const int32_t cbase = cols.base(slice);
        const T *vp = val + base + r;
        const int64_t cat = base + r;
        const T *pg = P + g * VW;
        T acc[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) acc[j] = T(0);
        int t = 0;
        for (; t + 2 <= w; t += 2) {
            T a[2][1];
            int32_t c[2][1];
            ld_stream(vp + (int64_t)t * S, pol, a[0]);
            cols.template load<1>(cat + (int64_t)t * S, slice, pol, cbase, c[0]);
            ld_stream(vp + (int64_t)(t + 1) * S, pol, a[1]);
            cols.template load<1>(cat + (int64_t)(t + 1) * S, slice, pol, cbase, c[1]);
            T xv[2][VW];
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (c[u][0] >= 0) ld_piece<BYTES, COH>(pg + (int64_t)c[u][0] * KP, xv[u]);
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (c[u][0] >= 0) {
#pragma unroll
                    for (int j = 0; j < VW; ++j) acc[j] = fma_t(a[u][0], xv[u][j], acc[j]);
                }
        }
        if (t < w) {
            T a[1];
            int32_t c[1];
            ld_stream(vp + (int64_t)t * S, pol, a);
            cols.template load<1>(cat + (int64_t)t * S, slice, pol, cbase, c);
            if (c[0] >= 0) {
                T xv[VW];
                ld_piece<BYTES, COH>(pg + (int64_t)c[0] * KP, xv);
#pragma unroll
                for (int j = 0; j < VW; ++j) acc[j] = fma_t(a[0], xv[j], acc[j]);
            }
        }
        if (row < n) {
            st_piece<BYTES>(Q + row * KP + g * VW, acc);
            T pv[VW];
            ld_piece<BYTES, COH>(P + row * KP + g * VW, pv);
#pragma unroll
            for (int j = 0; j < VW; ++j) pqt[j] = fma_t(pv[j], acc[j], pqt[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < VW; ++j) pq[0][j] = (double)pqt[j];
    cta_cols<G, VW, 1>(pq, part, vb, vgrid);
}

// R = B - A X (x_zero: R = B), P = D^-1 R when P is given; per-column r.z, r.r, b.b.  FP64.
template <int G, int BYTES, typename ColT>
__device__ __forceinline__ void residual_phase(int vb, int vgrid, int32_t n, int32_t S,
                                               int32_t n_slices, const int64_t *__restrict__ sp,
                                               ColT cols, const double *__restrict__ val,
                                               const double *X, int x_zero, const double *B,
                                               double *R, double *P, const double *dinv,
                                               double *part) {
    using T = double;
    constexpr int VW = Piece<T, BYTES>::n;
    constexpr int KP = VW * G;
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / G, g = lane % G;
    const int64_t groups = (int64_t)n_slices * S / RPW;
    const uint64_t pol = policy_evict_first();
    double v[3][VW];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int j = 0; j < VW; ++j) v[q][j] = 0.0;
    for (int64_t wg = (int64_t)vb * kMcgWarps + warp; wg < groups;
         wg += (int64_t)vgrid * kMcgWarps) {
        const int64_t row0 = wg * RPW;
        const int64_t row = row0 + sub;
        const int64_t slice = row0 / S;
        const int64_t r = row - slice * S;
        T acc[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) acc[j] = T(0);
        if (!x_zero) {
            const int64_t base = sp[slice];
            const int w = (int)((sp[slice + 1] - base) / S);
            const int32_t cbase = cols.base(slice);
            for (int t = 0; t < w; ++t) {
                T a[1];
                int32_t c[1];
                ld_stream(val + base + (int64_t)t * S + r, pol, a);
                cols.template load<1>(base + (int64_t)t * S + r, slice, pol, cbase, c);
                if (c[0] >= 0) {
                    T xv[VW];
                    ld_piece<BYTES, false>(X + (int64_t)c[0] * KP + g * VW, xv);
#pragma unroll
                    for (int j = 0; j < VW; ++j) acc[j] = fma_t(a[0], xv[j], acc[j]);
                }
            }
        }
        if (row < n) {
            T bv[VW], rv[VW], zv[VW];
            ld_piece<BYTES, false>(B + row * KP + g * VW, bv);
            const T d = dinv[row];
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                rv[j] = bv[j] - acc[j];
                zv[j] = d * rv[j];
                v[0][j] += rv[j] * zv[j];
                v[1][j] += rv[j] * rv[j];
                v[2][j] += bv[j] * bv[j];
            }
            st_piece<BYTES>(R + row * KP + g * VW, rv);
            if (P) st_piece<BYTES>(P + row * KP + g * VW, zv);
        }
    }
    cta_cols<G, VW, 3>(v, part, vb, vgrid);
}

// r_c -= alpha_c q_c for running columns; per-column r.(D^-1 r) and r.r.  16-byte pieces, a
// grid stride that is a multiple of the column groups, so each thread keeps its columns.
template <typename T, int KP>
__device__ __forceinline__ void r_phase(int vb, int vgrid, int32_t n, T *R, const T *Q,
                                        const T *dinv, const T *s_alpha, const int *s_run,
                                        double *part) {
    constexpr int V = 16 / (int)sizeof(T);
    constexpr int CG = KP / V;
    const int64_t nvec = (int64_t)n * CG;
    const int64_t stride = (int64_t)vgrid * kCgBlock;
    const int c0 = (int)(threadIdx.x % CG) * V;
    T al[V];
    bool run[V], any = false;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        al[j] = s_alpha[c0 + j];
        run[j] = s_run[c0 + j] != 0;
        any = any || run[j];
    }
    T vz[V], vr[V];
#pragma unroll
    for (int j = 0; j < V; ++j) vz[j] = vr[j] = T(0);
    if (any) {
        for (int64_t v = (int64_t)vb * kCgBlock + threadIdx.x; v < nvec; v += stride) {
            const int64_t i = v * V;
            const T d = dinv[v / CG];
            T rv[V], qv[V];
            ld_piece<16, true>(R + i, rv);
            ld_piece<16, true>(Q + i, qv);
#pragma unroll
            for (int j = 0; j < V; ++j)
                if (run[j]) {
                    rv[j] = fma_t(-al[j], qv[j], rv[j]);
                    vz[j] = fma_t(rv[j], d * rv[j], vz[j]);
                    vr[j] = fma_t(rv[j], rv[j], vr[j]);
                }
            st_piece<16>(R + i, rv);
        }
    }
    double v2[2][V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        v2[0][j] = (double)vz[j];
        v2[1][j] = (double)vr[j];
    }
    cta_cols<CG, V, 2>(v2, part, vb, vgrid);
}

// x_c += alpha_c p_c for the columns the r sweep updated, then p_c = D^-1 r_c + beta_c p_c for
// the columns still running.
template <typename T, int KP>
__device__ __forceinline__ void p_phase(int vb, int vgrid, int32_t n, T *X, T *P, const T *R,
                                        const T *dinv, const T *s_alpha, const T *s_beta,
                                        const int *s_upd, const int *s_run) {
    constexpr int V = 16 / (int)sizeof(T);
    constexpr int CG = KP / V;
    const int64_t nvec = (int64_t)n * CG;
    const int64_t stride = (int64_t)vgrid * kCgBlock;
    const int c0 = (int)(threadIdx.x % CG) * V;
    T al[V], be[V];
    bool upd[V], run[V], any = false;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        al[j] = s_alpha[c0 + j];
        be[j] = s_beta[c0 + j];
        upd[j] = s_upd[c0 + j] != 0;
        run[j] = s_run[c0 + j] != 0;
        any = any || upd[j];
    }
    if (!any) return;
    for (int64_t v = (int64_t)vb * kCgBlock + threadIdx.x; v < nvec; v += stride) {
        const int64_t i = v * V;
        const T d = dinv[v / CG];
        T xv[V], pv[V], rv[V];
        ld_piece<16, true>(X + i, xv);
        ld_piece<16, true>(P + i, pv);
        ld_piece<16, true>(R + i, rv);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            if (upd[j]) xv[j] = fma_t(al[j], pv[j], xv[j]);
            if (run[j]) pv[j] = fma_t(be[j], pv[j], d * rv[j]);
        }
        st_piece<16>(X + i, xv);
        st_piece<16>(P + i, pv);
    }
}

// ---- graph-launched kernels -------------------------------------------------------------------
template <typename T, int G, int BYTES, typename ColT>
__global__ void __launch_bounds__(kCgBlock, 4)
mcg_product(int32_t n, int32_t S, int32_t n_slices, const int64_t *sp, ColT cols, const T *val,
            const T *P, T *Q, double *part, McgScalars *sc) {
    constexpr int KP = Piece<T, BYTES>::n * G;
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->pending = 0;
    if (sc->active == 0) return;
    product_phase<T, G, BYTES, false>(blockIdx.x, gridDim.x, n, S, n_slices, sp, cols, val, P, Q,
                                      part);
    if (last_cta(&sc->tickets[0])) {
        __shared__ double tot[1][KP];
        grid_cols<KP, 1>(part, gridDim.x, tot);
        if (threadIdx.x < KP) col_after_pq(sc->col[threadIdx.x], tot[0][threadIdx.x]);
        __syncthreads();
        if (threadIdx.x == 0) {
            int a = 0;
            for (int c = 0; c < KP; ++c) a += sc->col[c].done == 0;
            sc->active = a;
        }
    }
}

template <typename T, int KP>
__global__ void __launch_bounds__(kCgBlock)
mcg_rsweep(int32_t n, T *R, const T *Q, const T *dinv, double *part, McgScalars *sc) {
    __shared__ T s_alpha[KP];
    __shared__ int s_run[KP];
    if (sc->active == 0) return;
    if (threadIdx.x < KP) {
        s_alpha[threadIdx.x] = (T)sc->col[threadIdx.x].alpha;
        s_run[threadIdx.x] = sc->col[threadIdx.x].done == 0;
    }
    __syncthreads();
    r_phase<T, KP>(blockIdx.x, gridDim.x, n, R, Q, dinv, s_alpha, s_run, part);
    if (last_cta(&sc->tickets[1])) {
        __shared__ double tot[2][KP];
        grid_cols<KP, 2>(part, gridDim.x, tot);
        if (threadIdx.x < KP)
            col_after_r(sc->col[threadIdx.x], tot[0][threadIdx.x], tot[1][threadIdx.x],
                        sc->max_iter);
        __syncthreads();
        if (threadIdx.x == 0) {
            int a = 0;
            for (int c = 0; c < KP; ++c) a += sc->col[c].done == 0;
            sc->active = a;
            sc->pending = 1;
        }
    }
}

template <typename T, int KP>
__global__ void __launch_bounds__(kCgBlock)
mcg_psweep(int32_t n, T *X, T *P, const T *R, const T *dinv, const McgScalars *sc) {
    __shared__ T s_alpha[KP], s_beta[KP];
    __shared__ int s_upd[KP], s_run[KP];
    if (!sc->pending) return;
    if (threadIdx.x < KP) {
        const McgCol &c = sc->col[threadIdx.x];
        s_alpha[threadIdx.x] = (T)c.alpha;
        s_beta[threadIdx.x] = (T)c.beta;
        s_upd[threadIdx.x] = c.upd;
        s_run[threadIdx.x] = c.done == 0;
    }
    __syncthreads();
    p_phase<T, KP>(blockIdx.x, gridDim.x, n, X, P, R, dinv, s_alpha, s_beta, s_upd, s_run);
}

// R = B - A X, P = D^-1 R and the per-column sums; last CTA by mode:
//   0 start    rho, rr, bb; done = converged already; iterations and restarts cleared
//   1 check    a converged column whose true residual fails restarts (at most twice)
//   2 report   rr, bb only (final true residuals)
//   3 outer    refinement residual: rr, bb, s = ||r||, inv_s; done = converged
template <int G, int BYTES, typename ColT>
__global__ void __launch_bounds__(kCgBlock, 3)
mcg_residual(int32_t n, int32_t S, int32_t n_slices, const int64_t *sp, ColT cols,
             const double *val, const double *X, int x_zero, const double *B, double *R,
             double *P, const double *dinv, double *part, McgScalars *sc, int mode) {
    constexpr int KP = Piece<double, BYTES>::n * G;
    residual_phase<G, BYTES>(blockIdx.x, gridDim.x, n, S, n_slices, sp, cols, val, X, x_zero, B,
                             R, P, dinv, part);
    if (last_cta(&sc->tickets[2])) {
        __shared__ double tot[3][KP];
        grid_cols<KP, 3>(part, gridDim.x, tot);
        if (threadIdx.x < KP) {
            McgCol &c = sc->col[threadIdx.x];
            const double rz = tot[0][threadIdx.x], rr = tot[1][threadIdx.x],
                         bb = tot[2][threadIdx.x];
            c.rr = rr;
            c.bb = bb;
            if (mode == 0) {
                c.rho = rz;
                c.done = rr <= c.tol2 * bb ? 1 : 0;
                c.iters = 0;
                c.restarts = 0;
                c.upd = 0;
            } else if (mode == 1) {
                if (c.done == 1 && !(rr <= c.tol2 * bb)) {
                    if (c.restarts < 2) {
                        c.restarts += 1;
                        c.rho = rz;
                        c.done = 0;
                    } else {
                        c.done = 2;
                    }
                }
            } else if (mode == 3) {
                c.s = sqrt(rr);
                c.inv_s = rr > 0.0 ? 1.0 / c.s : 0.0;
                c.done = rr <= c.tol2 * bb ? 1 : 0;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int a = 0;
            for (int c = 0; c < KP; ++c) a += sc->col[c].done == 0;
            sc->active = a;
            sc->pending = 0;
        }
    }
}

// Refinement: start of the inner FP32 solves of the columns the outer residual has not
// converged: r32 = fp32(r64 / ||r64||), d = 0, p32 = D32^-1 r32; inner rho, rr; the inner
// tolerance of each column: inner_rtol, or (adaptive) max(inner_rtol, min(1/2, the reduction the
// outer residual still needs with a factor 2 of margin)), as in the single-RHS refinement.
template <int KP>
__global__ void __launch_bounds__(kCgBlock)
mcg_inner_start(int32_t n, const double *R64, const McgScalars *outer, float *R32, float *P32,
                float *D32, const float *dinv32, double *part, McgScalars *inner, double rtol,
                double inner_rtol, int adaptive) {
    constexpr int V = 4;
    constexpr int CG = KP / V;
    __shared__ double s_inv[KP];
    __shared__ int s_run[KP];
    if (threadIdx.x < KP) {
        s_inv[threadIdx.x] = outer->col[threadIdx.x].inv_s;
        s_run[threadIdx.x] = outer->col[threadIdx.x].done == 0;
    }
    __syncthreads();
    const int64_t nvec = (int64_t)n * CG;
    const int64_t stride = (int64_t)gridDim.x * kCgBlock;
    const int c0 = (int)(threadIdx.x % CG) * V;
    float vz[V] = {0.f, 0.f, 0.f, 0.f}, vr[V] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t v = (int64_t)blockIdx.x * kCgBlock + threadIdx.x; v < nvec; v += stride) {
        const int64_t i = v * V;
        const float d = dinv32[v / CG];
        float rv[V], pv[V];
        const float zero[V] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < V; ++j) {
            rv[j] = s_run[c0 + j] ? __double2float_rn(R64[i + j] * s_inv[c0 + j]) : 0.0f;
            pv[j] = d * rv[j];
            vz[j] = fmaf(rv[j], pv[j], vz[j]);
            vr[j] = fmaf(rv[j], rv[j], vr[j]);
        }
        st_piece<16>(R32 + i, rv);
        st_piece<16>(P32 + i, pv);
        st_piece<16>(D32 + i, zero);
    }
    double v2[2][V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        v2[0][j] = (double)vz[j];
        v2[1][j] = (double)vr[j];
    }
    cta_cols<CG, V, 2>(v2, part, blockIdx.x, gridDim.x);
    if (last_cta(&inner->tickets[3])) {
        __shared__ double tot[2][KP];
        grid_cols<KP, 2>(part, gridDim.x, tot);
        if (threadIdx.x < KP) {
            McgCol &c = inner->col[threadIdx.x];
            const McgCol &o = outer->col[threadIdx.x];
            double tol_in = inner_rtol;
            if (adaptive && o.rr > 0.0) {
                const double need = 0.5 * rtol * sqrt(o.bb / o.rr);
                if (need > tol_in) tol_in = need < 0.5 ? need : 0.5;
            }
            c.tol2 = tol_in * tol_in;
            c.rho = tot[0][threadIdx.x];
            c.rr = tot[1][threadIdx.x];
            c.bb = tot[1][threadIdx.x];
            c.iters = 0;
            c.upd = 0;
            c.done = (o.done == 0 && c.rr > 0.0) ? 0 : 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int a = 0;
            for (int c = 0; c < KP; ++c) a += inner->col[c].done == 0;
            inner->active = a;
            inner->pending = 0;
        }
    }
}

// Refinement update x_c += s_c d_c (FP64) for the columns whose outer residual has not
// converged; their refinement step and inner iterations are counted.
template <int KP>
__global__ void mcg_outer_update(int32_t n, double *X, const float *D32, McgScalars *outer,
                                 const McgScalars *inner) {
    __shared__ double s_s[KP];
    __shared__ int s_run[KP];
    if (threadIdx.x < KP) {
        s_s[threadIdx.x] = outer->col[threadIdx.x].s;
        s_run[threadIdx.x] = outer->col[threadIdx.x].done == 0;
    }
    __syncthreads();
    const int64_t total = (int64_t)n * KP;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int c = (int)(i % KP);
        if (s_run[c]) X[i] = fma(s_s[c], (double)D32[i], X[i]);
    }
    if (blockIdx.x == 0 && threadIdx.x < KP && s_run[threadIdx.x]) {
        outer->col[threadIdx.x].restarts += 1;
        outer->col[threadIdx.x].total += inner->col[threadIdx.x].iters;
    }
}

// per-column set-up of a scalar block
__global__ void mcg_set(McgScalars *sc, int k, int kp, double tol2, int max_iter) {
    const int c = threadIdx.x;
    if (c < kp) {
        McgCol z{};
        z.tol2 = tol2;
        z.done = c < k ? 0 : 1;
        sc->col[c] = z;
    }
    if (c == 0) {
        sc->active = 0;
        sc->pending = 0;
        sc->max_iter = max_iter;
        sc->timed_out = 0;
        for (int t = 0; t < 4; ++t) sc->tickets[t] = 0u;
        sc->bar_count = 0u;
        sc->bar_gen = 0u;
        sc->budget_ns = 0;
    }
}

// caller's n x k <-> internal n x kp (padding columns 0)
template <typename T>
__global__ void mcg_pack(int32_t n, int k, int kp, const T *src, T *dst) {
    const int64_t total = (int64_t)n * kp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t row = i / kp;
        const int c = (int)(i % kp);
        dst[i] = (src && c < k) ? src[row * k + c] : T(0);
    }
}

template <typename T>
__global__ void mcg_unpack(int32_t n, int k, int kp, const T *src, T *dst) {
    const int64_t total = (int64_t)n * k;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
        dst[i] = src[(i / k) * kp + i % k];
}

// ---- persistent kernel ------------------------------------------------------------------------
__device__ __forceinline__ long long mcg_timer_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr long long kMcgBarrierLimitNs = 2000000000LL;

// Grid barrier of the co-resident grid.  A CTA that waits longer than the limit records the
// timeout and returns false instead of spinning on.
__device__ bool mcg_barrier(McgScalars *sc) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *genp = &sc->bar_gen;
        const unsigned g = *genp;
        __threadfence();
        const unsigned arrived = atomicAdd(&sc->bar_count, 1u);
        int good = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(&sc->bar_count, 0u);
            __threadfence();
            atomicAdd(&sc->bar_gen, 1u);
        } else {
            const long long t0 = mcg_timer_ns();
            while (*genp == g) {
                if (mcg_timer_ns() - t0 > kMcgBarrierLimitNs) {
                    good = 0;
                    atomicExch(&sc->timed_out, 1);
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

// The whole lock-step recurrence in one cooperative launch: the product runs on the graph
// path's product grid as virtual CTAs (CTA b on CTA b mod gridDim.x), the sweeps on the grid
// itself (the graph path's sweep grid), and after each barrier every CTA reduces the partials
// in the graph path's fixed order, so all CTAs hold the same column states and the results are
// the graph path's bit for bit.  Vectors are read with coherent loads (they change between
// barriers).  The wall-clock budget is voted by CTA 0 once per iteration.
template <typename T, int G, int BYTES, typename ColT>
__global__ void __launch_bounds__(kCgBlock, 4)
mcg_persistent(int32_t n, int32_t S, int32_t n_slices, const int64_t *sp, ColT cols,
               const T *val, T *X, T *R, T *P, T *Q, const T *dinv, double *part, int Gpq,
               int pq_len, McgScalars *sc) {
    constexpr int KP = Piece<T, BYTES>::n * G;
    __shared__ McgCol s_col[KP];
    __shared__ T s_alpha[KP], s_beta[KP];
    __shared__ int s_run[KP], s_upd[KP];
    __shared__ double tot1[1][KP];
    __shared__ double tot2[2][KP];
    __shared__ int s_active;
    const long long t_start = mcg_timer_ns();
    const long long budget = sc->budget_ns;
    const int max_iter = sc->max_iter;
    double *part1 = part;
    double *part2 = part + (int64_t)KP * pq_len;
    double *vote = part2 + (int64_t)2 * KP * gridDim.x;
    if (threadIdx.x < KP) s_col[threadIdx.x] = sc->col[threadIdx.x];
    if (threadIdx.x == 0) s_active = sc->active;
    __syncthreads();
    bool timed_out = false;
    while (s_active > 0) {
        for (int b = blockIdx.x; b < Gpq; b += gridDim.x)
            product_phase<T, G, BYTES, true>(b, Gpq, n, S, n_slices, sp, cols, val, P, Q, part1);
        if (blockIdx.x == 0 && threadIdx.x == 0)
            vote[0] = (budget > 0 && mcg_timer_ns() - t_start > budget) ? 1.0 : 0.0;
        if (!mcg_barrier(sc)) {
            timed_out = true;
            break;
        }
        if (__ldcg(vote) != 0.0) {
            timed_out = true;
            break;
        }
        grid_cols<KP, 1>(part1, Gpq, tot1);
        if (threadIdx.x < KP) {
            col_after_pq(s_col[threadIdx.x], tot1[0][threadIdx.x]);
            s_alpha[threadIdx.x] = (T)s_col[threadIdx.x].alpha;
            s_run[threadIdx.x] = s_col[threadIdx.x].done == 0;
        }
        __syncthreads();
        r_phase<T, KP>(blockIdx.x, gridDim.x, n, R, Q, dinv, s_alpha, s_run, part2);
        if (!mcg_barrier(sc)) {
            timed_out = true;
            break;
        }
        grid_cols<KP, 2>(part2, gridDim.x, tot2);
        if (threadIdx.x < KP) {
            McgCol &c = s_col[threadIdx.x];
            col_after_r(c, tot2[0][threadIdx.x], tot2[1][threadIdx.x], max_iter);
            s_beta[threadIdx.x] = (T)c.beta;
            s_upd[threadIdx.x] = c.upd;
            s_run[threadIdx.x] = c.done == 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int a = 0;
            for (int c = 0; c < KP; ++c) a += s_col[c].done == 0;
            s_active = a;
        }
        p_phase<T, KP>(blockIdx.x, gridDim.x, n, X, P, R, dinv, s_alpha, s_beta, s_upd, s_run);
        if (!mcg_barrier(sc)) {
            timed_out = true;
            break;
        }
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x < KP) sc->col[threadIdx.x] = s_col[threadIdx.x];
        if (threadIdx.x == 0) {
            sc->active = s_active;
            sc->pending = 0;
            if (timed_out) atomicExch(&sc->timed_out, 1);
        }
    }
}

// ---- host ---------------------------------------------------------------------------------------
int sweep_grid(int32_t n, int kp, int elem_bytes) {
    const int64_t vecs = (int64_t)n * kp * elem_bytes / 16;
    const int64_t cap = (int64_t)device_facts().sm_count * kCgCtasPerSm;
    const int64_t want = (vecs + 4 * kCgBlock - 1) / (4 * kCgBlock);
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

int product_grid(const spmv_matrix_t A, int G, int elem_bytes) {
    const int64_t groups = (int64_t)A->n_slices * A->S / (32 / G);
    (void)elem_bytes;
    const int64_t cap = (int64_t)device_facts().sm_count * 4;
    const int64_t want = (groups + kMcgWarps - 1) / kMcgWarps;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

template <typename F>
spmv_status_t with_kp(int kp, F &&f) {
    using std::integral_constant;
    if (kp == 8) return f(integral_constant<int, 8>{});
    if (kp == 16) return f(integral_constant<int, 16>{});
    if (kp == 32) return f(integral_constant<int, 32>{});
    return SPMV_ERR_INVALID_ARG;
}

// (G lanes per row, piece bytes) of the product for kp columns: each lane gathers a 32-byte
// piece of a row (G = kp / pieces), or a 16-byte one when the handle's tuner chose that width
template <typename T, typename F>
spmv_status_t with_piece(int kp, int bytes, F &&f) {
    using std::integral_constant;
    auto by_kp = [&](auto bt) -> spmv_status_t {
        constexpr int BY = decltype(bt)::value;
        constexpr int V = BY / (int)sizeof(T);
        return with_kp(kp, [&](auto kt) -> spmv_status_t {
            constexpr int KP = decltype(kt)::value;
            return f(integral_constant<int, KP / V>{}, bt);
        });
    };
    if (bytes == 16) return by_kp(integral_constant<int, 16>{});
    return by_kp(integral_constant<int, 32>{});
}

template <typename F>
spmv_status_t with_mcg_cols(spmv_matrix_t A, F &&f) {
    if (A->index_bits == 16) return f(Cols16{A->sell_col16.p, A->col_start.p});
    return f(Cols32{A->sell_col.p});
}

McgScalars *block_of(spmv_matrix_t A, int which) { return A->mcg->scal.p + which; }

// enqueue `iters` iterations (three kernels each) of the FP64 (f32 = false) or FP32 recurrence
spmv_status_t enqueue_iters(spmv_matrix_t A, bool f32, int iters, int bytes, cudaStream_t st) {
    McgWork &w = *A->mcg;
    const int kp = w.kp;
    auto run = [&](auto tag) -> spmv_status_t {
        using T = decltype(tag);
        T *X = f32 ? (T *)w.D32.p : (T *)w.X.p;
        T *R = f32 ? (T *)w.R32.p : (T *)w.R.p;
        T *P = f32 ? (T *)w.P32.p : (T *)w.P.p;
        T *Q = f32 ? (T *)w.Q32.p : (T *)w.Q.p;
        const T *dinv = f32 ? (const T *)A->cg.dinv32.p : (const T *)A->cg.dinv.p;
        const T *val = f32 ? (const T *)A->sell_val32.p : (const T *)A->sell_val.p;
        McgScalars *sc = block_of(A, f32 ? 1 : 0);
        const int Gsw = sweep_grid(A->n, kp, (int)sizeof(T));
        return with_mcg_cols(A, [&](auto cols) -> spmv_status_t {
            using ColT = decltype(cols);
            return with_piece<T>(kp, bytes, [&](auto gt, auto bt) -> spmv_status_t {
                constexpr int G = decltype(gt)::value, BY = decltype(bt)::value;
                constexpr int KP = Piece<T, BY>::n * G;
                const int Gpq = product_grid(A, G, (int)sizeof(T));
                for (int it = 0; it < iters; ++it) {
                    mcg_product<T, G, BY, ColT><<<Gpq, kCgBlock, 0, st>>>(
                        A->n, A->S, A->n_slices, A->slice_ptr.p, cols, val, P, Q, w.part.p, sc);
                    mcg_rsweep<T, KP><<<Gsw, kCgBlock, 0, st>>>(A->n, R, Q, dinv, w.part.p, sc);
                    mcg_psweep<T, KP><<<Gsw, kCgBlock, 0, st>>>(A->n, X, P, R, dinv, sc);
                }
                GB_LAUNCHED();
                return SPMV_OK;
            });
        });
    };
    if (f32) return run(float{});
    return run(double{});
}

// every column running (for timing the product outside a solve)
__global__ void mcg_activate(McgScalars *sc, int kp) {
    const int c = threadIdx.x;
    if (c < kp) {
        sc->col[c].done = 0;
        sc->col[c].rho = 1.0;
    }
    if (c == 0) {
        sc->active = kp;
        sc->pending = 0;
        for (int t = 0; t < 4; ++t) sc->tickets[t] = 0u;
    }
}

// Tuner of the FP64 product's gather width (32- or 16-byte pieces of a row of P per lane):
// each width computes Q = A P for P = the packed right-hand sides, timed as the median of
// three launches each after writing a buffer of twice the L2 size; the faster is kept for
// the handle.  The width fixes the p.q reduction order of the handle's later multi-RHS solves.
spmv_status_t tune_gather(spmv_matrix_t A, cudaStream_t st) {
    A->mcg_tuned = true;
    if (A->opt.gather_bytes) return SPMV_OK;
    McgWork &w = *A->mcg;
    McgScalars *sc = block_of(A, 1);
    GB_CUDA(cudaMemcpyAsync(w.P.p, w.B.p, sizeof(double) * (size_t)A->n * w.kp,
                            cudaMemcpyDeviceToDevice, st));
    const size_t fb = 2 * (size_t)(device_facts().l2_bytes > 0 ? device_facts().l2_bytes
                                                               : (128 << 20));
    void *flush = nullptr;
    GB_CUDA(gb_malloc_async(&flush, fb, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    spmv_status_t s = cuda_status(cudaEventCreate(&e0));
    if (s == SPMV_OK) s = cuda_status(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_bytes = 32;
    for (int bytes : {32, 16}) {
        float t[3] = {0.f, 0.f, 0.f};
        for (int i = -1; i < 3 && s == SPMV_OK; ++i) {  // i = -1: warm-up
            mcg_activate<<<1, kMcgMaxCols, 0, st>>>(sc, w.kp);
            s = cuda_status(cudaGetLastError());
            if (s == SPMV_OK) s = cuda_status(cudaMemsetAsync(flush, i + 2, fb, st));
            if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e0, st));
            if (s == SPMV_OK)
                s = with_mcg_cols(A, [&](auto cols) -> spmv_status_t {
                    using ColT = decltype(cols);
                    return with_piece<double>(w.kp, bytes, [&](auto gt, auto bt) -> spmv_status_t {
                        constexpr int G = decltype(gt)::value, BY = decltype(bt)::value;
                        mcg_product<double, G, BY, ColT><<<product_grid(A, G, 8), kCgBlock, 0,
                                                           st>>>(A->n, A->S, A->n_slices,
                                                                 A->slice_ptr.p, cols,
                                                                 A->sell_val.p, w.P.p, w.Q.p,
                                                                 w.part.p, sc);
                        GB_LAUNCHED();
                        return SPMV_OK;
                    });
                });
            if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e1, st));
            if (s == SPMV_OK) s = cuda_status(cudaEventSynchronize(e1));
            if (s == SPMV_OK && i >= 0) s = cuda_status(cudaEventElapsedTime(&t[i], e0, e1));
        }
        if (s != SPMV_OK) break;
        const float med = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
        if (med < best) {
            best = med;
            best_bytes = bytes;
        }
    }
    if (s == SPMV_OK) A->mcg_bytes = best_bytes;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(flush, st);
    return s;
}

spmv_status_t enqueue_residual(spmv_matrix_t A, bool x_zero, bool want_p, int mode,
                               cudaStream_t st) {
    McgWork &w = *A->mcg;
    return with_mcg_cols(A, [&](auto cols) -> spmv_status_t {
        using ColT = decltype(cols);
        return with_piece<double>(w.kp, 32, [&](auto gt, auto) -> spmv_status_t {
            constexpr int G = decltype(gt)::value;
            const int grid = product_grid(A, G, 8);
            mcg_residual<G, 32, ColT><<<grid, kCgBlock, 0, st>>>(
                A->n, A->S, A->n_slices, A->slice_ptr.p, cols, A->sell_val.p, w.X.p,
                x_zero ? 1 : 0, w.B.p, w.R.p, want_p ? w.P.p : nullptr, A->cg.dinv.p, w.part.p,
                block_of(A, 0), mode);
            GB_LAUNCHED();
            return SPMV_OK;
        });
    });
}

// streams for capturing the graphs of a batch (process lifetime; see cg.cu)
cudaStream_t capture_stream() {
    static std::mutex mu;
    static cudaStream_t s = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        s = nullptr;
    }
    return s;
}

std::mutex &capture_mutex() {
    static std::mutex mu;
    return mu;
}

spmv_status_t get_graph(spmv_matrix_t A, bool f32, int iters, int bytes, cudaGraphExec_t *out) {
    McgWork &w = *A->mcg;
    const int i = f32 ? 1 : 0;
    if (w.graph[i] && w.graph_iters[i] == iters && w.graph_gw[i] == bytes) {
        *out = w.graph[i];
        return SPMV_OK;
    }
    if (w.graph[i]) {
        cudaGraphExecDestroy(w.graph[i]);
        w.graph[i] = nullptr;
    }
    std::lock_guard<std::mutex> lock(capture_mutex());
    cudaStream_t cs = capture_stream();
    if (!cs) return SPMV_ERR_CUDA;
    GB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    spmv_status_t s = enqueue_iters(A, f32, iters, bytes, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (s != SPMV_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    GB_CUDA(e);
    e = cudaGraphInstantiate(&w.graph[i], graph, 0);
    cudaGraphDestroy(graph);
    GB_CUDA(e);
    w.graph_iters[i] = iters;
    w.graph_gw[i] = bytes;
    *out = w.graph[i];
    return SPMV_OK;
}

spmv_status_t launch_persistent(spmv_matrix_t A, bool f32, int bytes, double timeout_s,
                                cudaStream_t st) {
    McgWork &w = *A->mcg;
    auto run = [&](auto tag) -> spmv_status_t {
        using T = decltype(tag);
        T *X = f32 ? (T *)w.D32.p : (T *)w.X.p;
        T *R = f32 ? (T *)w.R32.p : (T *)w.R.p;
        T *P = f32 ? (T *)w.P32.p : (T *)w.P.p;
        T *Q = f32 ? (T *)w.Q32.p : (T *)w.Q.p;
        const T *dinv = f32 ? (const T *)A->cg.dinv32.p : (const T *)A->cg.dinv.p;
        const T *val = f32 ? (const T *)A->sell_val32.p : (const T *)A->sell_val.p;
        McgScalars *sc = block_of(A, f32 ? 1 : 0);
        return with_mcg_cols(A, [&](auto cols) -> spmv_status_t {
            using ColT = decltype(cols);
            return with_piece<T>(w.kp, bytes, [&](auto gt, auto bt) -> spmv_status_t {
                constexpr int G = decltype(gt)::value, BY = decltype(bt)::value;
                auto kern = mcg_persistent<T, G, BY, ColT>;
                int per_sm = 0;
                GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCgBlock, 0));
                int Gsw = sweep_grid(A->n, w.kp, (int)sizeof(T));
                if ((int64_t)per_sm * device_facts().sm_count < Gsw) return SPMV_ERR_UNSUPPORTED;
                int Gpq = product_grid(A, G, (int)sizeof(T));
                int pq_len = Gpq;
                const long long budget = timeout_s > 0 ? (long long)(timeout_s * 1e9) : 0;
                GB_CUDA(cudaMemcpyAsync(&sc->budget_ns, &budget, sizeof(budget),
                                        cudaMemcpyHostToDevice, st));
                int32_t n = A->n, S = A->S, ns = A->n_slices;
                const int64_t *sp = A->slice_ptr.p;
                double *part = w.part.p;
                void *args[] = {&n, &S, &ns, &sp, &cols, &val, &X, &R, &P, &Q, &dinv, &part,
                                &Gpq, &pq_len, &sc};
                GB_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3(Gsw),
                                                    dim3(kCgBlock), args, 0, st));
                return SPMV_OK;
            });
        });
    };
    if (f32) return run(float{});
    return run(double{});
}

spmv_status_t read_block(spmv_matrix_t A, int which, cudaStream_t st, McgScalars *out) {
    McgWork &w = *A->mcg;
    GB_CUDA(cudaMemcpyAsync(&w.h[which], w.scal.p + which, sizeof(McgScalars),
                            cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    *out = w.h[which];
    return SPMV_OK;
}

using Clock = std::chrono::steady_clock;

double since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

// Runs the recurrence of block `which` (FP64 / FP32) until every column is done, the budget
// runs out (returns TIMEOUT) or an error occurs.
spmv_status_t run_recurrence(spmv_matrix_t A, bool f32, const cg_options_t &o, int bytes,
                             cudaStream_t st, Clock::time_point t0, McgScalars *h) {
    const int which = f32 ? 1 : 0;
    const int batch = o.check_every > 0 ? o.check_every : 16;
    if (o.persistent) {
        const double left = o.timeout_s > 0 ? o.timeout_s - since(t0) : 0.0;
        if (o.timeout_s > 0 && left <= 0) return SPMV_ERR_TIMEOUT;
        GB_TRY(launch_persistent(A, f32, bytes, left, st));
        GB_TRY(read_block(A, which, st, h));
        if (h->timed_out) return SPMV_ERR_TIMEOUT;
        return SPMV_OK;
    }
    cudaGraphExec_t g = nullptr;
    GB_TRY(get_graph(A, f32, batch, bytes, &g));
    for (;;) {
        GB_CUDA(cudaGraphLaunch(g, st));
        GB_TRY(read_block(A, which, st, h));
        if (h->active == 0) return SPMV_OK;
        if (o.timeout_s > 0 && since(t0) > o.timeout_s) return SPMV_ERR_TIMEOUT;
    }
}

spmv_status_t ensure_mcg_work(spmv_matrix_t A, int kp, bool mixed, cudaStream_t st) {
    if (!A->mcg) A->mcg = new McgWork();
    McgWork &w = *A->mcg;
    size_t *t = &A->bytes;
    const size_t nk = (size_t)A->n * kp;
    if (w.kp != kp) {
        for (int i = 0; i < 2; ++i)
            if (w.graph[i]) {
                cudaGraphExecDestroy(w.graph[i]);
                w.graph[i] = nullptr;
            }
        w.X.release(t); w.R.release(t); w.P.release(t); w.Q.release(t); w.B.release(t);
        w.R32.release(t); w.P32.release(t); w.Q32.release(t); w.D32.release(t);
        w.part.release(t);
        w.kp = 0;
        GB_TRY(w.X.alloc(nk, t));
        GB_TRY(w.R.alloc(nk, t));
        GB_TRY(w.P.alloc(nk, t));
        GB_TRY(w.Q.alloc(nk, t));
        GB_TRY(w.B.alloc(nk, t));
        // partials: KP per CTA of the largest grid, three quantities, plus the persistent
        // kernel's vote
        const int64_t cap = (int64_t)device_facts().sm_count * 6;
        GB_TRY(w.part.alloc((size_t)(3 * kp * cap + 2 * kp * cap + 8), t));
        if (!w.scal.p) GB_TRY(w.scal.alloc(2, t));
        w.kp = kp;
    }
    if (mixed && !w.D32.p) {
        GB_TRY(w.R32.alloc(nk, t));
        GB_TRY(w.P32.alloc(nk, t));
        GB_TRY(w.Q32.alloc(nk, t));
        GB_TRY(w.D32.alloc(nk, t));
    }
    return SPMV_OK;
}

unsigned pack_grid(int64_t total) {
    const int64_t g = (total + 255) / 256;
    const int64_t cap = (int64_t)device_facts().sm_count * 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

// FP64 lock-step Jacobi-PCG of all columns, with true-residual restarts
spmv_status_t solve64_multi(spmv_matrix_t A, int k, const cg_options_t &o, int bytes,
                            cudaStream_t st, Clock::time_point t0, spmv_status_t *col_status) {
    McgWork &w = *A->mcg;
    McgScalars *sc = block_of(A, 0);
    mcg_set<<<1, kMcgMaxCols, 0, st>>>(sc, k, w.kp, o.rtol * o.rtol, o.max_iter);
    GB_LAUNCHED();
    GB_TRY(enqueue_residual(A, !o.use_x0, true, 0, st));
    McgScalars h{};
    GB_TRY(read_block(A, 0, st, &h));
    for (;;) {
        if (h.active > 0) {
            spmv_status_t s = run_recurrence(A, false, o, bytes, st, t0, &h);
            if (s == SPMV_ERR_TIMEOUT) {
                for (int c = 0; c < k; ++c) col_status[c] = h.col[c].done == 0 ? SPMV_ERR_TIMEOUT
                                                                               : col_status[c];
                break;
            }
            GB_TRY(s);
        }
        // true residuals of the converged columns; restart those that fail (at most twice)
        GB_TRY(enqueue_residual(A, false, true, 1, st));
        GB_TRY(read_block(A, 0, st, &h));
        if (h.active == 0) break;
    }
    return SPMV_OK;
}

// FP32-inner / FP64-refinement of all columns
spmv_status_t solve_mixed_multi(spmv_matrix_t A, int k, const cg_options_t &o, int bytes,
                                cudaStream_t st, Clock::time_point t0, spmv_status_t *col_status,
                                int *outer_steps) {
    McgWork &w = *A->mcg;
    McgScalars *so = block_of(A, 0), *si = block_of(A, 1);
    mcg_set<<<1, kMcgMaxCols, 0, st>>>(so, k, w.kp, o.rtol * o.rtol, 1);
    GB_LAUNCHED();
    GB_TRY(enqueue_residual(A, !o.use_x0, false, 3, st));
    McgScalars ho{}, hi{};
    GB_TRY(read_block(A, 0, st, &ho));
    int outer = 0;
    const int Gsw = sweep_grid(A->n, w.kp, 4);
    while (ho.active > 0) {
        if (outer >= o.max_outer) {
            for (int c = 0; c < k; ++c)
                if (ho.col[c].done == 0) col_status[c] = SPMV_ERR_NOT_CONVERGED;
            break;
        }
        if (o.timeout_s > 0 && since(t0) > o.timeout_s) {
            for (int c = 0; c < k; ++c)
                if (ho.col[c].done == 0) col_status[c] = SPMV_ERR_TIMEOUT;
            break;
        }
        mcg_set<<<1, kMcgMaxCols, 0, st>>>(si, k, w.kp, 0.0, o.max_iter);
        GB_LAUNCHED();
        GB_TRY(with_kp(w.kp, [&](auto kt) -> spmv_status_t {
            constexpr int KP = decltype(kt)::value;
            mcg_inner_start<KP><<<Gsw, kCgBlock, 0, st>>>(A->n, w.R.p, so, w.R32.p, w.P32.p,
                                                          w.D32.p, A->cg.dinv32.p, w.part.p, si,
                                                          o.rtol, o.inner_rtol, o.adaptive_inner);
            GB_LAUNCHED();
            return SPMV_OK;
        }));
        GB_TRY(read_block(A, 1, st, &hi));
        if (hi.active > 0) {
            spmv_status_t s = run_recurrence(A, true, o, bytes, st, t0, &hi);
            if (s == SPMV_ERR_TIMEOUT) {
                for (int c = 0; c < k; ++c)
                    if (ho.col[c].done == 0) col_status[c] = SPMV_ERR_TIMEOUT;
                break;
            }
            GB_TRY(s);
        }
        GB_TRY(with_kp(w.kp, [&](auto kt) -> spmv_status_t {
            constexpr int KP = decltype(kt)::value;
            mcg_outer_update<KP><<<pack_grid((int64_t)A->n * KP), 256, 0, st>>>(A->n, w.X.p,
                                                                               w.D32.p, so, si);
            GB_LAUNCHED();
            return SPMV_OK;
        }));
        ++outer;
        GB_TRY(enqueue_residual(A, false, false, 3, st));
        GB_TRY(read_block(A, 0, st, &ho));
    }
    *outer_steps = outer;
    return SPMV_OK;
}

}  // namespace

void release_mcg(spmv_matrix_t A) {
    if (!A->mcg) return;
    McgWork &w = *A->mcg;
    size_t *t = &A->bytes;
    for (int i = 0; i < 2; ++i)
        if (w.graph[i]) cudaGraphExecDestroy(w.graph[i]);
    w.X.release(t); w.R.release(t); w.P.release(t); w.Q.release(t); w.B.release(t);
    w.R32.release(t); w.P32.release(t); w.Q32.release(t); w.D32.release(t);
    w.part.release(t); w.scal.release(t);
    delete A->mcg;
    A->mcg = nullptr;
}

}  // namespace gb

using namespace gb;

extern "C" spmv_status_t cg_solve_multi(spmv_matrix_t A, int k, const double *B, double *X,
                                        const cg_options_t *opt, cg_result_t *results,
                                        void *stream) {
    if (!A || k < 1 || k > kMcgMaxCols) return SPMV_ERR_INVALID_ARG;
    cg_result_t local[kMcgMaxCols];
    cg_result_t *res = results ? results : local;
    for (int c = 0; c < k; ++c) {
        res[c] = cg_result_t{};
        res[c].status = SPMV_ERR_INVALID_ARG;
    }
    if (A->n > 0 && (!B || !X || (const void *)B == (const void *)X)) return SPMV_ERR_INVALID_ARG;
    cg_options_t o;
    cg_default_options(&o);
    if (opt) o = *opt;
    if (!(o.rtol >= 0.0) || o.max_iter < 1 || o.check_every < 0 || o.max_outer < 0 ||
        !(o.inner_rtol > 0.0 && o.inner_rtol < 1.0) || o.timeout_s < 0)
        return SPMV_ERR_INVALID_ARG;
    if (A->n != A->n_cols) return SPMV_ERR_INVALID_ARG;
    spmv_status_t s = SPMV_OK;
    if (!A->has64() || (o.mixed && !A->has32())) s = SPMV_ERR_UNSUPPORTED;
    if (s != SPMV_OK) {
        for (int c = 0; c < k; ++c) res[c].status = s;
        return s;
    }
    if (A->n == 0) {
        for (int c = 0; c < k; ++c) res[c].status = SPMV_OK;
        return SPMV_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    NvtxRange nvtx(o.mixed ? "cg_solve_multi/mixed" : "cg_solve_multi/fp64");
    const auto t0 = Clock::now();
    const int kp = k <= 8 ? 8 : (k <= 16 ? 16 : 32);
    auto fail = [&](spmv_status_t e) {
        for (int c = 0; c < k; ++c) res[c].status = e;
        return e;
    };
    s = ensure_cg_work(A, o.mixed != 0, st);
    if (s != SPMV_OK) return fail(s);
    s = ensure_mcg_work(A, kp, o.mixed != 0, st);
    if (s != SPMV_OK) return fail(s);
    McgWork &w = *A->mcg;
    const unsigned pg = pack_grid((int64_t)A->n * kp);
    mcg_pack<double><<<pg, 256, 0, st>>>(A->n, k, kp, B, w.B.p);
    mcg_pack<double><<<pg, 256, 0, st>>>(A->n, k, kp, o.use_x0 ? X : nullptr, w.X.p);
    s = cuda_status(cudaGetLastError());
    if (s != SPMV_OK) return fail(s);
    if (A->opt.autotune && !A->mcg_tuned) {
        s = tune_gather(A, st);
        if (s != SPMV_OK) return fail(s);
    }
    const int bytes = A->mcg_bytes == 16 ? 16 : 32;
    spmv_status_t col_status[kMcgMaxCols];
    for (int c = 0; c < k; ++c) col_status[c] = SPMV_OK;
    int outer = 0;
    s = o.mixed ? solve_mixed_multi(A, k, o, bytes, st, t0, col_status, &outer)
                : solve64_multi(A, k, o, bytes, st, t0, col_status);
    if (s != SPMV_OK) return fail(s);
    // final true residuals, x to the caller
    McgScalars h{};
    s = enqueue_residual(A, false, false, 2, st);
    if (s == SPMV_OK) s = read_block(A, 0, st, &h);
    if (s != SPMV_OK) return fail(s);
    mcg_unpack<double><<<pack_grid((int64_t)A->n * k), 256, 0, st>>>(A->n, k, kp, w.X.p, X);
    s = cuda_status(cudaGetLastError());
    if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
    if (s != SPMV_OK) return fail(s);
    spmv_status_t worst = SPMV_OK;
    for (int c = 0; c < k; ++c) {
        const McgCol &col = h.col[c];
        cg_result_t &r = res[c];
        r.rel_residual = col.bb > 0.0 ? std::sqrt(col.rr / col.bb) : 0.0;
        if (o.mixed) {
            r.iterations = col.total;
            r.outer_iterations = col.restarts;
            r.status = col_status[c];
            if (r.status == SPMV_OK && !(col.rr <= o.rtol * o.rtol * col.bb))
                r.status = SPMV_ERR_NOT_CONVERGED;
        } else {
            r.iterations = col.iters;
            r.outer_iterations = col.restarts;
            r.status = col_status[c];
            if (r.status == SPMV_OK && col.done != 1) r.status = SPMV_ERR_NOT_CONVERGED;
        }
        if (worst == SPMV_OK && r.status != SPMV_OK) worst = r.status;
    }
    return worst;
}
