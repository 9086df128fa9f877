// noalloc.cu -- cg_solve_csr_noalloc: FP64 Jacobi-PCG on caller-owned device CSR arrays
// that never allocates memory.
//
// Some callers cannot allocate device memory at solve time: a plugin living inside a host
// application that owns and pools all GPU memory itself, a real-time loop whose memory is
// fixed up front, or code running where a cudaMalloc would synchronise the device or fail.
// For them the work vectors and reduction scratch of this solve live in one file-scope
// __device__ array of fixed size (about 2.1 MB).  The array belongs to this file's module:
// with the CUDA runtime's default lazy module loading it is reserved on a device by the first
// call on that device (the set-up below, which a call with n = 0 performs alone), or when the
// library is loaded if CUDA_MODULE_LOADING=EAGER; from then on the device holds it until the
// process exits.  Systems up to kNoallocMaxRows rows fit.
//
// The iteration is the one of cg_solve (Jacobi-preconditioned CG, last-CTA reductions in a
// fixed order, true-residual check with at most two restarts), with a thread-per-row CSR
// product instead of the sliced-ELLPACK one.
#include <cuda.h>

#include <chrono>
#include <climits>
#include <cmath>
#include <mutex>

#include "cgkern.cuh"

namespace gb {
namespace {

constexpr int32_t kNoallocMaxRows = SPMV_NOALLOC_MAX_ROWS;
constexpr int kNoallocMaxGrid = 1024;                // CTAs of the grid-stride sweeps
constexpr int kScalarsDoubles = (sizeof(CgScalars) + 7) / 8;
constexpr size_t kScratchDoubles =
    4 * (size_t)kNoallocMaxRows + 4 * (size_t)kNoallocMaxGrid + kScalarsDoubles + 8;

// The scratch area: dinv | r | p | q | partials | scalars | flags.  Host code must never pass
// the symbol itself to a kernel (in host code it names a host-side stand-in); it uses the
// device address obtained with cudaGetSymbolAddress instead.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

struct Scratch {
    double *dinv, *r, *p, *q, *part;
    CgScalars *sc;
    int *flags;
};

Scratch carve(double *base) {
    Scratch s;
    s.dinv = base;
    s.r = base + kNoallocMaxRows;
    s.p = base + 2 * (size_t)kNoallocMaxRows;
    s.q = base + 3 * (size_t)kNoallocMaxRows;
    s.part = base + 4 * (size_t)kNoallocMaxRows;
    s.sc = (CgScalars *)(s.part + 4 * (size_t)kNoallocMaxGrid);
    s.flags = (int *)((double *)s.sc + kScalarsDoubles);
    return s;
}

// Identity of the current CUDA context (cuCtxGetCurrent + cuCtxGetId, fetched from the driver
// through the runtime so the library does not link the driver library itself).  A context
// created after cudaDeviceReset gets a new identity, so an address resolved in an earlier
// context is never reused.  Returns false when the driver does not offer the two calls.
bool current_context_id(unsigned long long *id) {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                             &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
                cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = (GetCurrent)f1;
            get_id = (GetId)f2;
        }
        cudaGetLastError();
    });
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Set-up: the device address of the scratch array, resolved with cudaGetSymbolAddress with the
// caller's device current, once per device and context (re-resolved when the context changes,
// e.g. after cudaDeviceReset; resolved on every call if the context cannot be identified).
spmv_status_t scratch_address(double **out) {
    static std::mutex mu;
    static double *addr[64] = {};
    static unsigned long long ctx_of[64] = {};
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SPMV_ERR_UNSUPPORTED;
    // make the device's context current (cudaSetDevice initialises it), so that it can be
    // identified before the lookup
    GB_CUDA(cudaSetDevice(dev));
    unsigned long long ctx = 0;
    const bool known = current_context_id(&ctx);
    std::lock_guard<std::mutex> lock(mu);
    if (!known || !addr[dev] || ctx_of[dev] != ctx) {
        void *p = nullptr;
        GB_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        addr[dev] = (double *)p;
        ctx_of[dev] = known ? ctx : 0;
    }
    *out = addr[dev];
    return SPMV_OK;
}

__global__ void na_reset(CgScalars *sc, int *flags, double tol2, int max_iter) {
    sc->tol2 = tol2;
    sc->max_iter = max_iter;
    sc->iters = 0;
    sc->done = 0;
    for (int k = 0; k < 4; ++k) sc->tickets[k] = 0u;
    flags[0] = 0;
}

// CSR checks (as spmv_create) and the Jacobi diagonal; flags[0] bits: 1 ends, 2 monotone,
// 4 range, 8 order, 16 zero or missing diagonal
__global__ void na_check_dinv(int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                              const double *val, double *dinv, int *flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (rp[0] != 0 || (int64_t)rp[n] != nnz)) atomicOr(flags, 1);
    if (i >= n) return;
    const int32_t a = rp[i], b = rp[i + 1];
    if (a > b || a < 0 || (int64_t)b > nnz) {
        atomicOr(flags, 2);
        return;
    }
    int32_t prev = -1;
    double d = 0.0;
    for (int32_t k = a; k < b; ++k) {
        const int32_t c = ci[k];
        if (c < 0 || c >= n) {
            atomicOr(flags, 4);
            return;
        }
        if (c <= prev) {
            atomicOr(flags, 8);
            return;
        }
        prev = c;
        if (c == (int32_t)i) d = val[k];
    }
    if (d == 0.0) atomicOr(flags, 16);
    else dinv[i] = 1.0 / d;
}

__device__ __forceinline__ double csr_row(int64_t i, const int32_t *rp, const int32_t *ci,
                                          const double *val, const double *x) {
    double acc = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) acc = fma(val[k], x[ci[k]], acc);
    return acc;
}

// r = b - A x (x_zero: r = b), p = D^-1 r; last CTA: rho, rr, bb, done
__global__ void __launch_bounds__(kCgBlock)
na_residual(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, const double *x,
            int x_zero, const double *b, double *r, double *p, const double *dinv, double *part,
            CgScalars *sc) {
    double v[3] = {0.0, 0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double ax = x_zero ? 0.0 : csr_row(i, rp, ci, val, x);
        const double bi = b[i];
        const double ri = bi - ax;
        const double zi = dinv[i] * ri;
        r[i] = ri;
        p[i] = zi;
        v[0] += ri * zi;
        v[1] += ri * ri;
        v[2] += bi * bi;
    }
    double tot[3];
    if (grid_sum_last<3>(v, part, &sc->tickets[0], tot) && threadIdx.x == 0) {
        sc->rho = tot[0];
        sc->rr = tot[1];
        sc->bb = tot[2];
        sc->done = (tot[1] <= sc->tol2 * tot[2]) ? 1 : 0;
    }
}

// q = A p, p.q -> alpha
__global__ void __launch_bounds__(kCgBlock)
na_spmv_pq(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, const double *p,
           double *q, double *part, CgScalars *sc) {
    if (sc->done) return;
    double vt = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double qi = csr_row(i, rp, ci, val, p);
        q[i] = qi;
        vt = fma(p[i], qi, vt);
    }
    double v[1] = {vt};
    double tot[1];
    if (grid_sum_last<1>(v, part, &sc->tickets[1], tot) && threadIdx.x == 0) {
        if (tot[0] == 0.0 || !isfinite(tot[0])) sc->done = 3;
        else sc->alpha = sc->rho / tot[0];
    }
}

__global__ void __launch_bounds__(kCgBlock)
na_update_xr(int32_t n, double *x, double *r, const double *p, const double *q,
             const double *dinv, double *part, CgScalars *sc) {
    if (sc->done) return;
    const double alpha = sc->alpha;
    double vz = 0.0, vr = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double xi = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        x[i] = xi;
        r[i] = ri;
        vz = fma(ri, dinv[i] * ri, vz);
        vr = fma(ri, ri, vr);
    }
    double v[2] = {vz, vr};
    double tot[2];
    if (grid_sum_last<2>(v, part, &sc->tickets[2], tot) && threadIdx.x == 0) {
        sc->beta = tot[0] / sc->rho;
        sc->rho = tot[0];
        sc->rr = tot[1];
        sc->iters += 1;
        if (tot[1] <= sc->tol2 * sc->bb) sc->done = 1;
        else if (!isfinite(tot[1])) sc->done = 3;
        else if (sc->iters >= sc->max_iter) sc->done = 2;
    }
}

__global__ void __launch_bounds__(kCgBlock)
na_update_p(int32_t n, const double *r, const double *dinv, double *p, const CgScalars *sc) {
    if (sc->done) return;
    const double beta = sc->beta;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        p[i] = fma(beta, p[i], dinv[i] * r[i]);
}

// scalars to a host variable (pageable: no pinned buffer is allocated)
spmv_status_t read_back(const CgScalars *sc, const int *flags, CgScalars *h, int *hflags,
                        cudaStream_t st) {
    GB_CUDA(cudaMemcpyAsync(h, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    if (hflags) GB_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    return SPMV_OK;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" spmv_status_t cg_solve_csr_noalloc(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                              const int32_t *col_idx, const double *values,
                                              const double *b, double *x,
                                              const cg_options_t *opt, cg_result_t *result,
                                              void *stream) {
    cg_result_t local{};
    cg_result_t *res = result ? result : &local;
    *res = cg_result_t{};
    res->status = SPMV_ERR_INVALID_ARG;
    if (n < 0 || n > kNoallocMaxRows || nnz < 0 || nnz > INT32_MAX) return SPMV_ERR_INVALID_ARG;
    if (n > 0 && (!row_ptr || !b || !x || b == x || (nnz > 0 && (!col_idx || !values))))
        return SPMV_ERR_INVALID_ARG;
    cg_options_t o;
    cg_default_options(&o);
    if (opt) o = *opt;
    if (!(o.rtol >= 0.0) || o.max_iter < 1 || o.check_every < 0 || o.timeout_s < 0)
        return SPMV_ERR_INVALID_ARG;
    if (o.mixed || o.persistent) return (res->status = SPMV_ERR_UNSUPPORTED);
    cudaStream_t st = (cudaStream_t)stream;
    double *base = nullptr;
    spmv_status_t s = scratch_address(&base);  // set-up (also for n == 0)
    if (s != SPMV_OK) return (res->status = s);
    if (n == 0) return (res->status = SPMV_OK);
    const Scratch w = carve(base);
    int G = device_facts().sm_count * 2;
    if (G > kNoallocMaxGrid) G = kNoallocMaxGrid;
    if (G < 1) G = 1;
    const int batch = o.check_every > 0 ? o.check_every : 16;
    const unsigned rows_grid = (unsigned)((n + 255) / 256);
    const auto t0 = std::chrono::steady_clock::now();
    auto expired = [&]() {
        return o.timeout_s > 0 &&
               std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >
                   o.timeout_s;
    };
    auto run = [&]() -> spmv_status_t {
        na_reset<<<1, 1, 0, st>>>(w.sc, w.flags, o.rtol * o.rtol, o.max_iter);
        na_check_dinv<<<rows_grid, 256, 0, st>>>(n, nnz, row_ptr, col_idx, values, w.dinv,
                                                 w.flags);
        GB_LAUNCHED();
        CgScalars h{};
        int hflags = 0;
        GB_TRY(read_back(w.sc, w.flags, &h, &hflags, st));
        if (hflags & 31) return (res->status = SPMV_ERR_INVALID_CSR);
        na_residual<<<G, kCgBlock, 0, st>>>(n, row_ptr, col_idx, values, x, o.use_x0 ? 0 : 1, b,
                                            w.r, w.p, w.dinv, w.part, w.sc);
        GB_LAUNCHED();
        if (!o.use_x0) GB_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
        int restarts = 0;
        for (;;) {
            for (;;) {
                for (int it = 0; it < batch; ++it) {
                    na_spmv_pq<<<G, kCgBlock, 0, st>>>(n, row_ptr, col_idx, values, w.p, w.q,
                                                       w.part, w.sc);
                    na_update_xr<<<G, kCgBlock, 0, st>>>(n, x, w.r, w.p, w.q, w.dinv,
                                                         w.part + G, w.sc);
                    na_update_p<<<G, kCgBlock, 0, st>>>(n, w.r, w.dinv, w.p, w.sc);
                }
                GB_LAUNCHED();
                GB_TRY(read_back(w.sc, w.flags, &h, nullptr, st));
                if (h.done || expired()) break;
            }
            res->iterations = h.iters;
            res->outer_iterations = restarts;
            if (h.done == 0) return (res->status = SPMV_ERR_TIMEOUT);
            if (h.done != 1) return (res->status = SPMV_ERR_NOT_CONVERGED);
            na_residual<<<G, kCgBlock, 0, st>>>(n, row_ptr, col_idx, values, x, 0, b, w.r, w.p,
                                                w.dinv, w.part, w.sc);
            GB_LAUNCHED();
            GB_TRY(read_back(w.sc, w.flags, &h, nullptr, st));
            if (h.done == 1) return (res->status = SPMV_OK);
            if (restarts >= 2) return (res->status = SPMV_ERR_NOT_CONVERGED);
            ++restarts;
        }
    };
    s = run();
    if (s != SPMV_OK && s != SPMV_ERR_NOT_CONVERGED && s != SPMV_ERR_TIMEOUT &&
        s != SPMV_ERR_INVALID_CSR)
        return (res->status = s);
    if (s == SPMV_ERR_INVALID_CSR) return s;
    // final true residual ||b - A x|| / ||b||
    CgScalars h{};
    na_reset<<<1, 1, 0, st>>>(w.sc, w.flags, 0.0, 1);
    na_residual<<<G, kCgBlock, 0, st>>>(n, row_ptr, col_idx, values, x, 0, b, w.r, w.p, w.dinv,
                                        w.part, w.sc);
    spmv_status_t s2 = cuda_status(cudaGetLastError());
    if (s2 == SPMV_OK) s2 = read_back(w.sc, w.flags, &h, nullptr, st);
    if (s2 != SPMV_OK) return (res->status = s2);
    res->rel_residual = h.bb > 0.0 ? sqrt(h.rr / h.bb) : 0.0;
    return res->status;
}
