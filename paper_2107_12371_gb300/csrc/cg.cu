// cg.cu -- Jacobi-preconditioned conjugate gradients (FP64) and FP32-inner / FP64-refinement
// solves built on the sliced-ELLPACK product.  Neither solver is in the paper; the paper puts
// the SpMV at the heart of the linear solver of an incompressible-flow time step (Sec. 2).
//
// One CG iteration is three kernels, each a grid-stride sweep over a fixed grid (the product
// over a grid of its own, see cg_pq_grid):
//   cg_spmv_pq   q = A p and p.q                      -> alpha = rho / (p.q)
//   cg_update_xr x += alpha p, r -= alpha q, r.(D^-1 r), r.r -> beta, rho, convergence
//   cg_update_p  p = D^-1 r + beta p
// Every kernel ends with a deterministic reduction: each CTA writes its partial sums, the
// last CTA to arrive (atomic ticket) reduces all partials in a fixed order and computes the
// scalars the next kernel reads.  Results therefore do not depend on CTA scheduling.  A
// "done" flag set by that last CTA turns the remaining kernels of a CUDA-graph batch into
// no-ops, so the host only checks convergence once per batch of iterations.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <vector>

#include "cgkern.cuh"

namespace gb {

namespace {

constexpr int kMaxParts = 4;

// ---- Jacobi diagonal ---------------------------------------------------------------------
__global__ void cg_dinv(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                        double *dinv64, float *dinv32, int *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == (int32_t)i) d = val[k];
    if (d == 0.0) {
        atomicOr(err, 1);
        return;
    }
    if (dinv64) dinv64[i] = 1.0 / d;
    if (dinv32) {
        const float d32 = __double2float_rn(d);
        if (d32 == 0.0f) atomicOr(err, 1);
        else dinv32[i] = 1.0f / d32;
    }
}

// r = b - A x (x_zero: r = b), p = D^-1 r (if p), partials r.(D^-1 r), r.r, b.b.
// Last CTA: rho, rr, bb, s = ||r||, done = rr <= tol2 bb.  Used to start and to restart CG,
// and for the FP64 residual of iterative refinement (p == nullptr).
template <typename T, int R, int L, typename ColT>
__global__ void __launch_bounds__(kCgBlock)
cg_residual(int32_t n, int32_t n_slices, const int64_t *sp, ColT col, const T *val,
            const T *x, int x_zero, const T *b, T *r, T *p, const T *dinv, double *part,
            CgScalars *sc) {
    constexpr int S = L * R;
    const uint64_t pol = policy_evict_first();
    const int64_t lanes = (int64_t)gridDim.x * blockDim.x;
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < (int64_t)n_slices * L;
         g += lanes) {
        const int64_t slice = g / L;
        const int lane = (int)(g % L);
        T acc[R];
        if (x_zero) {
#pragma unroll
            for (int i = 0; i < R; ++i) acc[i] = T(0);
        } else {
            slice_rows<T, R, L>(slice, lane, sp, col, val, x, pol, acc);
        }
        const int64_t row0 = slice * S + (int64_t)lane * R;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int64_t row = row0 + i;
            if (row < n) {
                const T bi = b[row];
                const T ri = bi - acc[i];
                r[row] = ri;
                const T zi = dinv ? dinv[row] * ri : ri;
                if (p) p[row] = zi;
                v[0] += (double)(ri * zi);
                v[1] += (double)(ri * ri);
                v[2] += (double)(bi * bi);
            }
        }
    }
    double tot[3];
    if (grid_sum_last<3>(v, part, &sc->tickets[0], tot) && threadIdx.x == 0) {
        sc->rho = tot[0];
        sc->rr = tot[1];
        sc->bb = tot[2];
        sc->s = sqrt(tot[1]);
        sc->inv_s = tot[1] > 0.0 ? 1.0 / sc->s : 0.0;
        sc->done = (tot[1] <= sc->tol2 * tot[2]) ? 1 : 0;
    }
}

// q = A p; partial p.q; last CTA: alpha = rho / (p.q).  Grid cg_pq_grid (see cgkern.cuh).
// UU: entries in flight per lane (pq_unroll, or 2 for matrices whose widest slice needs fewer
// load rounds that way; the per-row order, hence the result, is the same).
template <typename T, int R, int L, typename ColT, int UU>
__global__ void __launch_bounds__(kCgBlock, pq_min_ctas((int)sizeof(T) * R))
cg_spmv_pq(int32_t n, int32_t n_slices, const int64_t *sp, ColT col, const T *val,
           const T *p, T *q, double *part, CgScalars *sc) {
    // start the first slice's pointer loads while the stop flag is read, so that memory
    // traffic begins at once (a CTA would otherwise wait a full round trip for the flag)
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g0 < (int64_t)n_slices * L) {
        prefetch_l1(sp + g0 / L);
        prefetch_l1(sp + g0 / L + 1);
        prefetch_col_base(col, g0 / L);
    }
    if (sc->done) return;
    constexpr int S = L * R;
    const uint64_t pol = policy_evict_first();
    const int64_t lanes = (int64_t)gridDim.x * blockDim.x;
    T vt = T(0);
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < (int64_t)n_slices * L;
         g += lanes) {
        const int64_t slice = g / L;
        const int lane = (int)(g % L);
        T acc[R];
        slice_rows<T, R, L, false, UU>(slice, lane, sp, col, val, p, pol, acc);
        const int64_t row0 = slice * S + (int64_t)lane * R;
        store_rows<T, R>(q, row0, n, acc);
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (row0 + i < n) vt = fma_t(p[row0 + i], acc[i], vt);
    }
    double v[1] = {(double)vt};
    double tot[1];
    if (grid_sum_last<1>(v, part, &sc->tickets[1], tot) && threadIdx.x == 0) {
        if (tot[0] == 0.0 || !isfinite(tot[0])) {
            sc->done = 3;
        } else {
            sc->alpha = sc->rho / tot[0];
        }
    }
}

// x += alpha p; r -= alpha q; partials r.(D^-1 r), r.r; last CTA: beta, rho, convergence
template <typename T>
__global__ void __launch_bounds__(kCgBlock)
cg_update_xr(int32_t n, T *x, T *r, const T *p, const T *q, const T *dinv, double *part,
             CgScalars *sc) {
    // the first vectors of the sweep and the scalars are requested together (one round trip)
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * Vec16<T>::n;
    if (i0 < n) {
        prefetch_l1(x + i0);
        prefetch_l1(r + i0);
        prefetch_l1(p + i0);
        prefetch_l1(q + i0);
        prefetch_l1(dinv + i0);
    }
    const int done = sc->done;
    const T alpha = (T)sc->alpha;
    if (done) return;
    T vz = T(0), vr = T(0);
    sweep_update_xr<T>(n, alpha, x, r, p, q, dinv, vz, vr);
    double v[2] = {(double)vz, (double)vr};
    double tot[2];
    if (grid_sum_last<2>(v, part, &sc->tickets[2], tot) && threadIdx.x == 0) {
        const double rho_new = tot[0];
        sc->beta = rho_new / sc->rho;
        sc->rho = rho_new;
        sc->rr = tot[1];
        sc->iters += 1;
        if (tot[1] <= sc->tol2 * sc->bb) sc->done = 1;
        else if (!isfinite(tot[1])) sc->done = 3;
        else if (sc->iters >= sc->max_iter) sc->done = 2;
    }
}

// p = D^-1 r + beta p
template <typename T>
__global__ void __launch_bounds__(kCgBlock)
cg_update_p(int32_t n, const T *r, const T *dinv, T *p, const CgScalars *sc) {
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * Vec16<T>::n;
    if (i0 < n) {
        prefetch_l1(r + i0);
        prefetch_l1(dinv + i0);
        prefetch_l1(p + i0);
    }
    const int done = sc->done;
    const T beta = (T)sc->beta;
    if (done) return;
    sweep_update_p<T>(n, beta, r, dinv, p);
}

// refinement: right-hand side of the inner solve r32 = fp32(r64 / ||r64||), start of the
// inner FP32 PCG (d = 0, r_in = r32, p = D32^-1 r32), partials rho, rr0; inner scalars set
// by the last CTA.
__global__ void __launch_bounds__(kCgBlock)
ir_start_inner(int32_t n, const double *r64, const CgScalars *outer, float *r32, float *p32,
               float *d32, const float *dinv32, double *part, CgScalars *inner) {
    const double inv_s = outer->inv_s;
    float vz = 0.0f, vr = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float ri = __double2float_rn(r64[i] * inv_s);
        const float zi = dinv32[i] * ri;
        r32[i] = ri;
        p32[i] = zi;
        d32[i] = 0.0f;
        vz = fmaf(ri, zi, vz);
        vr = fmaf(ri, ri, vr);
    }
    double v[2] = {(double)vz, (double)vr};
    double tot[2];
    if (grid_sum_last<2>(v, part, &inner->tickets[3], tot) && threadIdx.x == 0) {
        inner->rho = tot[0];
        inner->rr = tot[1];
        inner->bb = tot[1];
        inner->iters = 0;
        inner->done = tot[1] > 0.0 ? 0 : 1;
    }
}

// refinement update x += s d (FP64)
__global__ void ir_update_x(int32_t n, double *x, const float *d32, const CgScalars *outer) {
    const double s = outer->s;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        x[i] = fma(s, (double)d32[i], x[i]);
}

__global__ void set_scalars(CgScalars *sc, double tol2, int max_iter) {
    sc->tol2 = tol2;
    sc->max_iter = max_iter;
    sc->iters = 0;
    sc->done = 0;
    for (int k = 0; k < 4; ++k) sc->tickets[k] = 0u;
    sc->bar_count = 0u;
    sc->budget_ns = 0;
}

__global__ void add_iters(CgScalars *inner, int *total) { *total += inner->iters; }

}  // namespace

// Grid of the CG product q = A p: one thread per slice-lane, at most the handle's pq_ctas CTAs
// per SM (tuned, or set by option; default pq_min_ctas).  The grid fixes the order of the p.q
// reduction, so it is a property of the handle, shared by the graph path and the persistent
// kernel (which runs it as virtual CTAs): both give identical results.
int cg_pq_grid(const spmv_matrix_t A, int L, int value_bytes) {
    const int per_sm = A->pq_ctas > 0 ? A->pq_ctas : pq_min_ctas(value_bytes);
    const int64_t cap = (int64_t)device_facts().sm_count * per_sm;
    const int64_t want = ((int64_t)A->n_slices * L + kCgBlock - 1) / kCgBlock;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

// Entries the product keeps in flight per lane: the handle's pq_unroll (tuned, or set by
// option), else five when the widest slice then needs fewer dependent load rounds than with
// two (the per-row order, hence the result, is the same either way).
bool cg_pq_deep(const spmv_matrix_t A, int uu) {
    if (A->pq_unroll > 0) return A->pq_unroll > 2;
    return load_rounds(A->max_width, uu) < load_rounds(A->max_width, 2);
}

// (lanes per slice, value bytes per lane entry) of the FP64 and FP32 product kernels for a
// slice height, as with_shape picks them
static int pq_grid64(const spmv_matrix_t A) {
    return cg_pq_grid(A, 32, 8 * (A->S / 32));
}
static int pq_grid32(const spmv_matrix_t A) {
    const int L = A->S / 4 < 32 ? A->S / 4 : 32;
    return cg_pq_grid(A, L, 4 * (A->S / L));
}

// Grid of the CG sweeps of a matrix with n rows: about 1,024 rows (4 per thread) per CTA, at
// most kCgCtasPerSm CTAs per SM (the persistent kernel uses the same grid).  It depends only
// on n and the device, so the reduction order is fixed per handle and both paths give
// identical results; small systems use fewer CTAs and leave room for concurrent solves.
int cg_grid(int32_t n) {
    const int cap = device_facts().sm_count * kCgCtasPerSm;
    const int64_t want = ((int64_t)n + 1023) / 1024;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

spmv_status_t ensure_cg_work(spmv_matrix_t A, bool mixed, cudaStream_t st) {
    CgWork &w = A->cg;
    size_t *t = &A->bytes;
    const size_t n = (size_t)A->n;
    if (!w.ready) {
        const int G = cg_grid(A->n);
        w.part_len = G;
        // the product's p.q partials (room for the largest grid any pq_ctas gives), then
        // kMaxParts partials per CTA of the sweeps
        w.pq_len = device_facts().sm_count * 4;
        GB_TRY(w.part.alloc((size_t)w.pq_len + (size_t)G * kMaxParts * 2, t));
        GB_TRY(w.scal.alloc(2 * ((sizeof(CgScalars) + 7) / 8), t));
        GB_CUDA(cudaMemsetAsync(w.scal.p, 0, w.scal.n * sizeof(double), st));
        GB_TRY(w.flags.alloc(16, t));
        GB_TRY(w.x.alloc(n, t));
        GB_TRY(w.r.alloc(n, t));
        GB_TRY(w.p.alloc(n, t));
        GB_TRY(w.q.alloc(n, t));
        GB_TRY(w.dinv.alloc(n, t));
        GB_CUDA(cudaMemsetAsync(w.flags.p, 0, 16 * sizeof(int), st));
        cg_dinv<<<(unsigned)((n + 255) / 256 ? (n + 255) / 256 : 1), 256, 0, st>>>(
            A->n, A->row_ptr.p, A->col.p, A->val.p, w.dinv.p, nullptr, w.flags.p);
        GB_LAUNCHED();
        w.ready = true;
    }
    if (mixed && !w.mixed_ready) {
        if (!A->has32()) return SPMV_ERR_UNSUPPORTED;
        GB_TRY(w.r32.alloc(n, t));
        GB_TRY(w.p32.alloc(n, t));
        GB_TRY(w.q32.alloc(n, t));
        GB_TRY(w.d32.alloc(n, t));
        GB_TRY(w.dinv32.alloc(n, t));
        cg_dinv<<<(unsigned)((n + 255) / 256 ? (n + 255) / 256 : 1), 256, 0, st>>>(
            A->n, A->row_ptr.p, A->col.p, A->val.p, nullptr, w.dinv32.p, w.flags.p + 1);
        GB_LAUNCHED();
        w.mixed_ready = true;
    }
    GB_CUDA(cudaMemcpyAsync(w.h_flags, w.flags.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (w.h_flags[0] || (mixed && w.h_flags[1])) return SPMV_ERR_INVALID_CSR;
    return SPMV_OK;
}

static CgScalars *outer_scalars(spmv_matrix_t A) { return (CgScalars *)A->cg.scal.p; }
static CgScalars *inner_scalars(spmv_matrix_t A) { return (CgScalars *)A->cg.scal.p + 1; }

// column-index format of the handle's sliced ELLPACK (see spmv.cu)
template <typename F>
static spmv_status_t with_cols(spmv_matrix_t A, F &&f) {
    if (A->index_bits == 16) return f(Cols16{A->sell_col16.p, A->col_start.p});
    return f(Cols32{A->sell_col.p});
}

// enqueue `iters` FP64 iterations (3 kernels each)
static spmv_status_t enqueue_cg64(spmv_matrix_t A, int iters, cudaStream_t st) {
    CgWork &w = A->cg;
    const int G = cg_grid(A->n);
    CgScalars *sc = outer_scalars(A);
    return with_cols(A, [&](auto cols) -> spmv_status_t {
        using ColT = decltype(cols);
        return with_shape(A->S, false, [&](auto rt, auto lt) -> spmv_status_t {
            constexpr int R = decltype(rt)::value, L = decltype(lt)::value;
            const int Gpq = pq_grid64(A);
            constexpr int UU = pq_unroll(8 * R);
            const bool deep = cg_pq_deep(A, UU);
            for (int it = 0; it < iters; ++it) {
                if (deep)
                    cg_spmv_pq<double, R, L, ColT, UU><<<Gpq, kCgBlock, 0, st>>>(
                        A->n, A->n_slices, A->slice_ptr.p, cols, A->sell_val.p, w.p.p, w.q.p,
                        w.part.p, sc);
                else
                    cg_spmv_pq<double, R, L, ColT, 2><<<Gpq, kCgBlock, 0, st>>>(
                        A->n, A->n_slices, A->slice_ptr.p, cols, A->sell_val.p, w.p.p, w.q.p,
                        w.part.p, sc);
                cg_update_xr<double><<<G, kCgBlock, 0, st>>>(A->n, w.x.p, w.r.p, w.p.p, w.q.p,
                                                             w.dinv.p, w.part.p + w.pq_len, sc);
                cg_update_p<double><<<G, kCgBlock, 0, st>>>(A->n, w.r.p, w.dinv.p, w.p.p, sc);
            }
            GB_LAUNCHED();
            return SPMV_OK;
        });
    });
}

__global__ void fill_value(int32_t n, double *v, double value) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        v[i] = value;
}

// one FP64 product q = A p with p.q (the first kernel of an iteration), on scalar block sc
static spmv_status_t enqueue_pq64(spmv_matrix_t A, CgScalars *sc, cudaStream_t st) {
    CgWork &w = A->cg;
    return with_cols(A, [&](auto cols) -> spmv_status_t {
        using ColT = decltype(cols);
        return with_shape(A->S, false, [&](auto rt, auto lt) -> spmv_status_t {
            constexpr int R = decltype(rt)::value, L = decltype(lt)::value;
            constexpr int UU = pq_unroll(8 * R);
            if (cg_pq_deep(A, UU))
                cg_spmv_pq<double, R, L, ColT, UU><<<pq_grid64(A), kCgBlock, 0, st>>>(
                    A->n, A->n_slices, A->slice_ptr.p, cols, A->sell_val.p, w.p.p, w.q.p,
                    w.part.p, sc);
            else
                cg_spmv_pq<double, R, L, ColT, 2><<<pq_grid64(A), kCgBlock, 0, st>>>(
                    A->n, A->n_slices, A->slice_ptr.p, cols, A->sell_val.p, w.p.p, w.q.p,
                    w.part.p, sc);
            GB_LAUNCHED();
            return SPMV_OK;
        });
    });
}

// Tuner of the CG product: its grid (2, 3 or 4 CTAs per SM) and the entries each lane keeps in
// flight (2 or 5).  Each candidate computes q = A p with p = 1 (the gathers and multiply-adds
// of a solve; the scalars go to the inner block, which every solve resets before use), timed
// as the median of three launches each after writing a buffer of twice the L2 size, as in
// steady use; the fastest is kept.  The FP32 product of a refinement uses the same grid.  The
// choice fixes the handle's p.q reduction order for every later solve, on both paths.
static spmv_status_t tune_cg_product(spmv_matrix_t A, cudaStream_t st) {
    A->pq_tuned = true;
    if (A->opt.pq_ctas || A->opt.pq_unroll) return SPMV_OK;
    CgWork &w = A->cg;
    CgScalars *sc = inner_scalars(A);
    fill_value<<<(unsigned)std::min<int64_t>(((int64_t)A->n + 255) / 256, 4096), 256, 0, st>>>(
        A->n, w.p.p, 1.0);
    GB_LAUNCHED();
    const size_t fb = 2 * (size_t)(device_facts().l2_bytes > 0 ? device_facts().l2_bytes
                                                               : (128 << 20));
    void *flush = nullptr;
    GB_CUDA(gb_malloc_async(&flush, fb, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    spmv_status_t s = cuda_status(cudaEventCreate(&e0));
    if (s == SPMV_OK) s = cuda_status(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_ctas = 0, best_uu = 0;
    for (int ctas = 2; ctas <= 4 && s == SPMV_OK; ++ctas) {
        for (int uu : {2, 5}) {
            A->pq_ctas = ctas;
            A->pq_unroll = uu;
            float t[3] = {0.f, 0.f, 0.f};
            for (int i = -1; i < 3 && s == SPMV_OK; ++i) {  // i = -1: warm-up
                set_scalars<<<1, 1, 0, st>>>(sc, 0.0, 1);
                s = cuda_status(cudaGetLastError());
                if (s == SPMV_OK) s = cuda_status(cudaMemsetAsync(flush, i + 2, fb, st));
                if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e0, st));
                if (s == SPMV_OK) s = enqueue_pq64(A, sc, st);
                if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e1, st));
                if (s == SPMV_OK) s = cuda_status(cudaEventSynchronize(e1));
                if (s == SPMV_OK && i >= 0) s = cuda_status(cudaEventElapsedTime(&t[i], e0, e1));
            }
            if (s != SPMV_OK) break;
            const float med = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
            if (med < best) {
                best = med;
                best_ctas = ctas;
                best_uu = uu;
            }
        }
    }
    A->pq_ctas = s == SPMV_OK ? best_ctas : 0;
    A->pq_unroll = s == SPMV_OK ? best_uu : 0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(flush, st);
    return s;
}

static spmv_status_t enqueue_cg32(spmv_matrix_t A, int iters, cudaStream_t st) {
    CgWork &w = A->cg;
    const int G = cg_grid(A->n);
    CgScalars *sc = inner_scalars(A);
    return with_cols(A, [&](auto cols) -> spmv_status_t {
        using ColT = decltype(cols);
        return with_shape(A->S, true, [&](auto rt, auto lt) -> spmv_status_t {
            constexpr int R = decltype(rt)::value, L = decltype(lt)::value;
            const int Gpq = pq_grid32(A);
            constexpr int UU = pq_unroll(4 * R);
            const bool deep = cg_pq_deep(A, UU);
            for (int it = 0; it < iters; ++it) {
                if (deep)
                    cg_spmv_pq<float, R, L, ColT, UU><<<Gpq, kCgBlock, 0, st>>>(
                        A->n, A->n_slices, A->slice_ptr.p, cols, A->sell_val32.p, w.p32.p,
                        w.q32.p, w.part.p, sc);
                else
                    cg_spmv_pq<float, R, L, ColT, 2><<<Gpq, kCgBlock, 0, st>>>(
                        A->n, A->n_slices, A->slice_ptr.p, cols, A->sell_val32.p, w.p32.p,
                        w.q32.p, w.part.p, sc);
                cg_update_xr<float><<<G, kCgBlock, 0, st>>>(A->n, w.d32.p, w.r32.p, w.p32.p,
                                                            w.q32.p, w.dinv32.p,
                                                            w.part.p + w.pq_len, sc);
                cg_update_p<float><<<G, kCgBlock, 0, st>>>(A->n, w.r32.p, w.dinv32.p, w.p32.p, sc);
            }
            GB_LAUNCHED();
            return SPMV_OK;
        });
    });
}

// r = b - A x on the FP64 values, p = D^-1 r when want_p
static spmv_status_t enqueue_residual64(spmv_matrix_t A, const double *b, bool x_zero,
                                        bool want_p, cudaStream_t st) {
    CgWork &w = A->cg;
    const int G = cg_grid(A->n);
    return with_cols(A, [&](auto cols) -> spmv_status_t {
        using ColT = decltype(cols);
        return with_shape(A->S, false, [&](auto rt, auto lt) -> spmv_status_t {
            constexpr int R = decltype(rt)::value, L = decltype(lt)::value;
            cg_residual<double, R, L, ColT><<<G, kCgBlock, 0, st>>>(
                A->n, A->n_slices, A->slice_ptr.p, cols, A->sell_val.p, w.x.p, x_zero ? 1 : 0, b,
                w.r.p, want_p ? w.p.p : nullptr, w.dinv.p, w.part.p, outer_scalars(A));
            GB_LAUNCHED();
            return SPMV_OK;
        });
    });
}

// Streams that graphs are captured on (capture needs a stream of its own: the caller's may be
// the legacy default stream).  They live as long as the process and are shared by all
// handles: creating and destroying a stream per handle was measured to wait behind the work
// of other streams, stalling concurrent solves.
struct CaptureStreams {
    std::mutex mu;
    std::vector<cudaStream_t> idle;
    cudaStream_t get() {
        {
            std::lock_guard<std::mutex> lock(mu);
            if (!idle.empty()) {
                cudaStream_t s = idle.back();
                idle.pop_back();
                return s;
            }
        }
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return s;
    }
    void put(cudaStream_t s) {
        std::lock_guard<std::mutex> lock(mu);
        idle.push_back(s);
    }
};

static CaptureStreams &capture_streams() {
    static CaptureStreams *cs = new CaptureStreams();  // never destroyed (process lifetime)
    return *cs;
}

// Graph of `iters` iterations, captured once per handle and kind.
static spmv_status_t get_graph(spmv_matrix_t A, bool f32, int iters, cudaGraphExec_t *out) {
    CgWork &w = A->cg;
    cudaGraphExec_t &g = f32 ? w.graph32 : w.graph64;
    int &gi = f32 ? w.graph32_iters : w.graph64_iters;
    if (g && gi == iters) {
        *out = g;
        return SPMV_OK;
    }
    if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
    }
    cudaStream_t cs = capture_streams().get();
    if (!cs) return SPMV_ERR_CUDA;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        capture_streams().put(cs);
        return cuda_status(e);
    }
    spmv_status_t s = f32 ? enqueue_cg32(A, iters, cs) : enqueue_cg64(A, iters, cs);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    capture_streams().put(cs);
    if (s != SPMV_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    GB_CUDA(e);
    e = cudaGraphInstantiate(&g, graph, 0);
    cudaGraphDestroy(graph);
    GB_CUDA(e);
    gi = iters;
    *out = g;
    return SPMV_OK;
}

using Clock = std::chrono::steady_clock;

static double seconds_since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

static bool cancelled(const std::atomic<int> *cancel) {
    return cancel && cancel->load(std::memory_order_relaxed) != 0;
}

// read both scalar blocks to the host
static spmv_status_t read_scalars(spmv_matrix_t A, cudaStream_t st, CgScalars *outer,
                                  CgScalars *inner) {
    CgWork &w = A->cg;
    GB_CUDA(cudaMemcpyAsync(w.h_scal, w.scal.p, 2 * sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (outer) *outer = w.h_scal[0];
    if (inner) *inner = w.h_scal[1];
    return SPMV_OK;
}

spmv_status_t cg_persistent64(spmv_matrix_t A, const cg_options_t &o, CgScalars *out,
                              cudaStream_t st);
spmv_status_t cg_persistent32(spmv_matrix_t A, const cg_options_t &o, CgScalars *out,
                              cudaStream_t st);

// Plain FP64 Jacobi-PCG in the handle's x buffer; x holds x0 (or anything if !use_x0).
static spmv_status_t solve64(spmv_matrix_t A, const double *b, const cg_options_t &o,
                             cg_result_t *res, cudaStream_t st, Clock::time_point t0,
                             const SolveControl &ctl) {
    const std::atomic<int> *cancel = ctl.cancel;
    CgWork &w = A->cg;
    const int batch = o.check_every > 0 ? o.check_every : 16;
    CgScalars *sc = outer_scalars(A);
    set_scalars<<<1, 1, 0, st>>>(sc, o.rtol * o.rtol, o.max_iter);
    GB_LAUNCHED();
    GB_TRY(enqueue_residual64(A, b, !o.use_x0, true, st));
    CgScalars h{};
    int restarts = 0;
    int total_iters = 0;
    for (;;) {
        if (o.persistent) {
            GB_TRY(cg_persistent64(A, o, &h, st));
        } else {
            cudaGraphExec_t g = nullptr;
            if (ctl.graphs) GB_TRY(get_graph(A, false, batch, &g));
            for (;;) {
                if (g) GB_CUDA(cudaGraphLaunch(g, st));
                else GB_TRY(enqueue_cg64(A, batch, st));
                GB_TRY(read_scalars(A, st, &h, nullptr));
                if (h.done || cancelled(cancel)) break;
                if (o.timeout_s > 0 && seconds_since(t0) > o.timeout_s) break;
            }
        }
        total_iters = h.iters;
        if (cancelled(cancel)) {
            res->status = SPMV_ERR_CANCELLED;
            break;
        }
        if (h.done == 0 || h.done == 4) {
            res->status = SPMV_ERR_TIMEOUT;
            break;
        }
        if (h.done == 2) {
            res->status = SPMV_ERR_NOT_CONVERGED;
            break;
        }
        if (h.done == 3) {
            res->status = SPMV_ERR_NOT_CONVERGED;
            break;
        }
        // recurrence converged: recompute the true residual; restart the recurrence from it
        // if it is still above the tolerance (at most two restarts)
        GB_TRY(enqueue_residual64(A, b, false, true, st));
        GB_TRY(read_scalars(A, st, &h, nullptr));
        if (h.done == 1) {
            res->status = SPMV_OK;
            break;
        }
        if (restarts >= 2) {
            res->status = SPMV_ERR_NOT_CONVERGED;
            break;
        }
        ++restarts;
    }
    res->iterations = total_iters;
    res->outer_iterations = restarts;
    (void)w;
    return SPMV_OK;
}

static spmv_status_t solve_mixed(spmv_matrix_t A, const double *b, const cg_options_t &o,
                                 cg_result_t *res, cudaStream_t st, Clock::time_point t0,
                                 const SolveControl &ctl) {
    const std::atomic<int> *cancel = ctl.cancel;
    CgWork &w = A->cg;
    const int batch = o.check_every > 0 ? o.check_every : 16;
    const int G = cg_grid(A->n);
    CgScalars *so = outer_scalars(A);
    CgScalars *si = inner_scalars(A);
    int *d_total = w.flags.p + 4;
    GB_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int), st));
    set_scalars<<<1, 1, 0, st>>>(so, o.rtol * o.rtol, 1);
    GB_LAUNCHED();
    GB_TRY(enqueue_residual64(A, b, !o.use_x0, false, st));
    CgScalars ho{}, hi{};
    GB_TRY(read_scalars(A, st, &ho, nullptr));
    int outer = 0;
    res->status = SPMV_OK;
    while (!ho.done) {
        if (outer >= o.max_outer) {
            res->status = SPMV_ERR_NOT_CONVERGED;
            break;
        }
        if (o.timeout_s > 0 && seconds_since(t0) > o.timeout_s) {
            res->status = SPMV_ERR_TIMEOUT;
            break;
        }
        if (cancelled(cancel)) {
            res->status = SPMV_ERR_CANCELLED;
            break;
        }
        // inner tolerance: inner_rtol, or (adaptive) just the reduction the outer residual
        // still needs, with a factor 2 of margin for the FP32 inner solve
        double tol_in = o.inner_rtol;
        if (o.adaptive_inner && ho.rr > 0.0) {
            const double need = 0.5 * o.rtol * std::sqrt(ho.bb / ho.rr);
            if (need > tol_in) tol_in = need < 0.5 ? need : 0.5;
        }
        set_scalars<<<1, 1, 0, st>>>(si, tol_in * tol_in, o.max_iter);
        ir_start_inner<<<G, kCgBlock, 0, st>>>(A->n, w.r.p, so, w.r32.p, w.p32.p, w.d32.p,
                                               w.dinv32.p, w.part.p, si);
        GB_LAUNCHED();
        if (o.persistent) {
            GB_TRY(cg_persistent32(A, o, &hi, st));
            if (hi.done == 4) hi.done = 0;  // timed out
        } else {
            cudaGraphExec_t g = nullptr;
            if (ctl.graphs) GB_TRY(get_graph(A, true, batch, &g));
            for (;;) {
                if (g) GB_CUDA(cudaGraphLaunch(g, st));
                else GB_TRY(enqueue_cg32(A, batch, st));
                GB_TRY(read_scalars(A, st, nullptr, &hi));
                if (hi.done || cancelled(cancel)) break;
                if (o.timeout_s > 0 && seconds_since(t0) > o.timeout_s) break;
            }
        }
        if (cancelled(cancel)) {
            res->status = SPMV_ERR_CANCELLED;
            break;
        }
        add_iters<<<1, 1, 0, st>>>(si, d_total);
        ir_update_x<<<G, kCgBlock, 0, st>>>(A->n, w.x.p, w.d32.p, so);
        GB_LAUNCHED();
        ++outer;
        GB_TRY(enqueue_residual64(A, b, false, false, st));
        GB_TRY(read_scalars(A, st, &ho, nullptr));
        if (hi.done == 0) {
            res->status = SPMV_ERR_TIMEOUT;
            break;
        }
    }
    GB_CUDA(cudaMemcpyAsync(w.h_flags + 4, d_total, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    res->iterations = w.h_flags[4];
    res->outer_iterations = outer;
    return SPMV_OK;
}

// true relative residual ||b - A x|| / ||b|| of the handle's x, in FP64
static spmv_status_t final_residual(spmv_matrix_t A, const double *b, cudaStream_t st,
                                    double *rel) {
    CgScalars *sc = outer_scalars(A);
    set_scalars<<<1, 1, 0, st>>>(sc, 0.0, 1);
    GB_LAUNCHED();
    GB_TRY(enqueue_residual64(A, b, false, false, st));
    CgScalars h{};
    GB_TRY(read_scalars(A, st, &h, nullptr));
    *rel = h.bb > 0.0 ? std::sqrt(h.rr / h.bb) : 0.0;
    return SPMV_OK;
}

void release_cg(spmv_matrix_t A) {
    size_t *t = &A->bytes;
    CgWork &w = A->cg;
    w.x.release(t); w.r.release(t); w.p.release(t); w.q.release(t); w.dinv.release(t);
    w.r32.release(t); w.p32.release(t); w.q32.release(t); w.d32.release(t); w.dinv32.release(t);
    w.part.release(t); w.scal.release(t); w.flags.release(t);
    if (w.graph64) cudaGraphExecDestroy(w.graph64);
    if (w.graph32) cudaGraphExecDestroy(w.graph32);
    w = CgWork{};
}

// Times (CUDA events on `st`) of the FP64 iteration of this handle, for the diagnostic entry
// point below: out[0] a CUDA-graph batch of `iters` iterations, per iteration; out[1] the same
// kernels launched directly on the stream, per iteration; out[2..4] each kernel of an
// iteration between events of its own (product, x/r sweep, p sweep); out[5] a read-back of
// the scalars to the host (copy + synchronisation).  The recurrence runs on b = 1 with rtol =
// 0, so no kernel turns into a no-op; the handle's solve state is overwritten.
spmv_status_t cg_timing(spmv_matrix_t A, int iters, double *out, cudaStream_t st) {
    GB_TRY(ensure_cg_work(A, false, st));
    CgWork &w = A->cg;
    CgScalars *sc = outer_scalars(A);
    double *b = nullptr;
    GB_CUDA(gb_malloc_async((void **)&b, sizeof(double) * (size_t)A->n, st));
    fill_value<<<(unsigned)std::min<int64_t>(((int64_t)A->n + 255) / 256, 4096), 256, 0, st>>>(
        A->n, b, 1.0);
    cudaEvent_t e[2] = {nullptr, nullptr};
    spmv_status_t s = cuda_status(cudaEventCreate(&e[0]));
    if (s == SPMV_OK) s = cuda_status(cudaEventCreate(&e[1]));
    auto restart = [&]() -> spmv_status_t {
        set_scalars<<<1, 1, 0, st>>>(sc, 0.0, 1 << 30);
        GB_LAUNCHED();
        return enqueue_residual64(A, b, true, true, st);
    };
    auto elapsed = [&](float *ms) -> spmv_status_t {
        GB_CUDA(cudaEventSynchronize(e[1]));
        GB_CUDA(cudaEventElapsedTime(ms, e[0], e[1]));
        return SPMV_OK;
    };
    const int G = cg_grid(A->n);
    float ms = 0.f;
    cudaGraphExec_t g = nullptr;
    if (s == SPMV_OK) s = get_graph(A, false, iters, &g);
    if (s == SPMV_OK) s = restart();
    if (s == SPMV_OK) s = cuda_status(cudaGraphLaunch(g, st));  // warm-up
    if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e[0], st));
    if (s == SPMV_OK) s = cuda_status(cudaGraphLaunch(g, st));
    if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e[1], st));
    if (s == SPMV_OK) s = elapsed(&ms);
    out[0] = ms / iters;
    if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e[0], st));
    if (s == SPMV_OK) s = enqueue_cg64(A, iters, st);
    if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e[1], st));
    if (s == SPMV_OK) s = elapsed(&ms);
    out[1] = ms / iters;
    double sum[3] = {0.0, 0.0, 0.0};
    for (int it = 0; it < iters && s == SPMV_OK; ++it) {
        for (int k = 0; k < 3 && s == SPMV_OK; ++k) {
            s = cuda_status(cudaEventRecord(e[0], st));
            if (s != SPMV_OK) break;
            if (k == 0) s = enqueue_pq64(A, sc, st);
            else if (k == 1)
                cg_update_xr<double><<<G, kCgBlock, 0, st>>>(A->n, w.x.p, w.r.p, w.p.p, w.q.p,
                                                             w.dinv.p, w.part.p + w.pq_len, sc);
            else
                cg_update_p<double><<<G, kCgBlock, 0, st>>>(A->n, w.r.p, w.dinv.p, w.p.p, sc);
            if (s == SPMV_OK) s = cuda_status(cudaGetLastError());
            if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e[1], st));
            if (s == SPMV_OK) s = elapsed(&ms);
            sum[k] += ms;
        }
    }
    for (int k = 0; k < 3; ++k) out[2 + k] = sum[k] / iters;
    if (s == SPMV_OK) {
        const auto t0 = Clock::now();
        for (int i = 0; i < iters && s == SPMV_OK; ++i) s = read_scalars(A, st, nullptr, nullptr);
        out[5] = seconds_since(t0) * 1e3 / iters;
    }
    if (e[0]) cudaEventDestroy(e[0]);
    if (e[1]) cudaEventDestroy(e[1]);
    cudaFreeAsync(b, st);
    return s;
}

}  // namespace gb

using namespace gb;

extern "C" {

spmv_status_t spmv_diag_cg_timing(spmv_matrix_t A, int iters, double *ms_out, void *stream) {
    if (!A || !ms_out || iters < 1 || iters > 4096 || A->n == 0 || A->n != A->n_cols)
        return SPMV_ERR_INVALID_ARG;
    if (!A->has64()) return SPMV_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    return cg_timing(A, iters, ms_out, st);
}

spmv_status_t cg_default_options(cg_options_t *o) {
    if (!o) return SPMV_ERR_INVALID_ARG;
    o->rtol = 1e-10;
    o->max_iter = 20000;
    o->mixed = 0;
    o->inner_rtol = 1e-4;
    o->max_outer = 20;
    o->use_x0 = 0;
    o->persistent = 0;
    o->check_every = 16;
    o->timeout_s = 0.0;
    o->adaptive_inner = 1;
    return SPMV_OK;
}

spmv_status_t cg_solve(spmv_matrix_t A, const double *b, double *x, const cg_options_t *opt,
                       cg_result_t *result, void *stream) {
    return cg_solve_ex(A, b, x, opt, result, (cudaStream_t)stream, SolveControl{});
}

}  // extern "C"

// cg_solve with the server's controls (cancellation flag, direct launches).
spmv_status_t gb::cg_solve_ex(spmv_matrix_t A, const double *b, double *x,
                              const cg_options_t *opt, cg_result_t *result, cudaStream_t st,
                              const SolveControl &ctl) {
    if (!A) return SPMV_ERR_INVALID_ARG;
    cg_result_t local{};
    cg_result_t *res = result ? result : &local;
    *res = cg_result_t{};
    res->status = SPMV_ERR_INVALID_ARG;
    if (A->n > 0 && (!b || !x || b == x)) return SPMV_ERR_INVALID_ARG;
    cg_options_t o;
    cg_default_options(&o);
    if (opt) o = *opt;
    if (!(o.rtol >= 0.0) || o.max_iter < 1 || o.check_every < 0 || o.max_outer < 0 ||
        !(o.inner_rtol > 0.0 && o.inner_rtol < 1.0) || o.timeout_s < 0)
        return SPMV_ERR_INVALID_ARG;
    if (A->n != A->n_cols) return SPMV_ERR_INVALID_ARG;  // CG needs a square matrix
    if (!A->has64()) return (res->status = SPMV_ERR_UNSUPPORTED);
    if (o.mixed && !A->has32()) return (res->status = SPMV_ERR_UNSUPPORTED);
    if (A->n == 0) {
        res->status = SPMV_OK;
        return SPMV_OK;
    }
    AllocStream alloc_scope(st);
    NvtxRange nvtx(o.mixed ? "cg_solve/mixed" : "cg_solve/fp64");
    const auto t0 = Clock::now();
    spmv_status_t s = ensure_cg_work(A, o.mixed != 0, st);
    if (s != SPMV_OK) return (res->status = s);
    if (A->opt.autotune && !A->pq_tuned) {
        s = tune_cg_product(A, st);
        if (s != SPMV_OK) return (res->status = s);
    }
    CgWork &w = A->cg;
    if (o.use_x0)
        s = cuda_status(cudaMemcpyAsync(w.x.p, x, sizeof(double) * A->n, cudaMemcpyDeviceToDevice, st));
    else
        s = cuda_status(cudaMemsetAsync(w.x.p, 0, sizeof(double) * A->n, st));
    if (s != SPMV_OK) return (res->status = s);
    s = o.mixed ? solve_mixed(A, b, o, res, st, t0, ctl) : solve64(A, b, o, res, st, t0, ctl);
    if (s != SPMV_OK) return (res->status = s);
    if (res->status == SPMV_ERR_CANCELLED) {
        s = cuda_status(cudaStreamSynchronize(st));
        return s != SPMV_OK ? (res->status = s) : res->status;
    }
    double rel = 0.0;
    s = final_residual(A, b, st, &rel);
    if (s != SPMV_OK) return (res->status = s);
    res->rel_residual = rel;
    s = cuda_status(cudaMemcpyAsync(x, w.x.p, sizeof(double) * A->n, cudaMemcpyDeviceToDevice, st));
    if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
    if (s != SPMV_OK) return (res->status = s);
    return res->status;
}
