// partition.cu -- row-block partition of a square matrix with a halo exchange of x, and
// Jacobi-PCG over the partition (not in the paper, whose kernel runs on one FPGA; for a matrix
// spread over several GPUs).
//
// Part p owns the contiguous rows [row_begin[p], row_begin[p + 1]) -- contiguous blocks of an
// RCM order keep each part's halo (the columns its rows read outside its own rows) small and
// owned by its neighbouring parts.  Its extended vector x_ext = [halo below | own | halo above]
// holds the halo entries in increasing global column order around its own entries, and the
// part's matrix is stored with its columns renumbered into x_ext monotonically, so every row
// keeps its global column order and its product equals the whole matrix's rows bit for bit.
// Before each product the parts exchange halos: part p sends to part q the entries of its own
// x that q's halo reads (spmv_partition_pack gathers them, in increasing row order, q
// ascending), and receives from each q the entries of its halo that q owns (one contiguous
// run per q, q ascending).  The transport is the caller's (NCCL, peer copies, host); the
// distributed CG takes it as a callback, together with a sum all-reduce of a few scalars.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "cgkern.cuh"

struct spmv_part_s {
    int n_parts = 0, part = 0;
    int32_t n_global = 0, row0 = 0, row1 = 0, n_local = 0, n_lo = 0, n_hi = 0, n_ext = 0;
    std::vector<int32_t> halo;        // global columns of the halo, ascending
    std::vector<int32_t> send_count;  // per part: own rows that part's halo reads
    std::vector<int32_t> recv_count;  // per part: halo entries that part owns
    std::vector<int32_t> send_rows;   // local rows to send, concatenated over parts ascending
    std::vector<int32_t> rp, ci;      // local CSR (columns in x_ext numbering)
    std::vector<double> val;
    int send_total = 0;
    spmv_matrix_t A = nullptr;        // device handle of the local rows (on_device)
    gb::DevBuf<int32_t> d_send_rows;
    size_t bytes = 0;
    // work of cg_solve_partitioned (allocated on first use)
    gb::DevBuf<double> r, p_ext, q, dinv, send, recv, part_sums, sums;
    gb::DevBuf<int> flag;
};

namespace gb {
namespace {

constexpr int kPartMaxParts = 4096;

spmv_status_t build_plan(spmv_part_s *P, int32_t n, int64_t nnz, const int32_t *rp,
                         const int32_t *ci, const double *val, int n_parts,
                         const int32_t *rb, int part) {
    if (rb[0] != 0 || rb[n_parts] != n) return SPMV_ERR_INVALID_ARG;
    for (int q = 0; q < n_parts; ++q)
        if (rb[q] > rb[q + 1]) return SPMV_ERR_INVALID_ARG;
    if (rp[0] != 0 || (int64_t)rp[n] != nnz) return SPMV_ERR_INVALID_CSR;
    for (int32_t i = 0; i < n; ++i) {
        if (rp[i] > rp[i + 1]) return SPMV_ERR_INVALID_CSR;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] < 0 || ci[k] >= n || (k > rp[i] && ci[k] <= ci[k - 1]))
                return SPMV_ERR_INVALID_CSR;
    }
    P->n_parts = n_parts;
    P->part = part;
    P->n_global = n;
    P->row0 = rb[part];
    P->row1 = rb[part + 1];
    P->n_local = P->row1 - P->row0;
    // halo: the columns outside [row0, row1) that the own rows read
    std::vector<char> mark((size_t)n, 0);
    for (int32_t i = P->row0; i < P->row1; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] < P->row0 || ci[k] >= P->row1) mark[ci[k]] = 1;
    std::vector<int32_t> ext_of((size_t)n, -1);  // global column -> x_ext index
    P->halo.clear();
    for (int32_t c = 0; c < n; ++c)
        if (mark[c]) P->halo.push_back(c);
    P->n_lo = (int32_t)(std::lower_bound(P->halo.begin(), P->halo.end(), P->row0) -
                        P->halo.begin());
    P->n_hi = (int32_t)P->halo.size() - P->n_lo;
    P->n_ext = P->n_lo + P->n_local + P->n_hi;
    for (int32_t h = 0; h < P->n_lo; ++h) ext_of[P->halo[h]] = h;
    for (int32_t i = 0; i < P->n_local; ++i) ext_of[P->row0 + i] = P->n_lo + i;
    for (int32_t h = P->n_lo; h < (int32_t)P->halo.size(); ++h)
        ext_of[P->halo[h]] = P->n_local + h;
    // receive counts: the halo entries each part owns (one contiguous run per part)
    P->recv_count.assign((size_t)n_parts, 0);
    for (int32_t c : P->halo) {
        const int q = (int)(std::upper_bound(rb, rb + n_parts + 1, c) - rb) - 1;
        P->recv_count[(size_t)q] += 1;
    }
    // send lists: for every other part, the own rows its halo reads (ascending)
    P->send_count.assign((size_t)n_parts, 0);
    P->send_rows.clear();
    std::vector<char> need((size_t)(P->n_local > 0 ? P->n_local : 1), 0);
    for (int q = 0; q < n_parts; ++q) {
        if (q == part) continue;
        std::fill(need.begin(), need.end(), 0);
        for (int32_t i = rb[q]; i < rb[q + 1]; ++i)
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
                if (ci[k] >= P->row0 && ci[k] < P->row1) need[(size_t)(ci[k] - P->row0)] = 1;
        for (int32_t i = 0; i < P->n_local; ++i)
            if (need[(size_t)i]) {
                P->send_rows.push_back(i);
                P->send_count[(size_t)q] += 1;
            }
    }
    P->send_total = (int)P->send_rows.size();
    // local CSR in the x_ext numbering (monotone, so every row keeps its column order)
    P->rp.assign((size_t)P->n_local + 1, 0);
    P->ci.clear();
    P->val.clear();
    for (int32_t i = 0; i < P->n_local; ++i) {
        const int32_t g = P->row0 + i;
        for (int32_t k = rp[g]; k < rp[g + 1]; ++k) {
            P->ci.push_back(ext_of[ci[k]]);
            P->val.push_back(val ? val[k] : 0.0);
        }
        P->rp[(size_t)i + 1] = (int32_t)P->ci.size();
    }
    return SPMV_OK;
}

__global__ void part_pack(int32_t count, const int32_t *rows, const double *x_own, double *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        out[i] = x_own[rows[i]];
}

unsigned grid_of(int64_t n) {
    const int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)device_facts().sm_count * 4;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

// ---- kernels of the partitioned CG (own rows only; sums reduced in a fixed order) --------
// dinv_i = 1 / a_ii, the diagonal at x_ext column n_lo + i
__global__ void part_dinv(int32_t n, int32_t n_lo, const int32_t *rp, const int32_t *ci,
                          const double *val, double *dinv, int *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == n_lo + (int32_t)i) d = val[k];
    if (d == 0.0) atomicOr(err, 1);
    else dinv[i] = 1.0 / d;
}

// r = b - q (q = A x, or 0), p_own = D^-1 r (when given); sums r.(D^-1 r), r.r, b.b
__global__ void __launch_bounds__(kCgBlock)
part_residual(int32_t n, const double *b, const double *q, double *r, double *p_own,
              const double *dinv, double *part, unsigned *ticket, double *out) {
    double v[3] = {0.0, 0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double ri = b[i] - (q ? q[i] : 0.0);
        const double zi = dinv[i] * ri;
        r[i] = ri;
        if (p_own) p_own[i] = zi;
        v[0] = fma(ri, zi, v[0]);
        v[1] = fma(ri, ri, v[1]);
        v[2] = fma(b[i], b[i], v[2]);
    }
    double tot[3];
    if (grid_sum_last<3>(v, part, ticket, tot) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
        out[2] = tot[2];
    }
}

// sum p.q over the own rows
__global__ void __launch_bounds__(kCgBlock)
part_dot(int32_t n, const double *p_own, const double *q, double *part, unsigned *ticket,
         double *out) {
    double v[1] = {0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        v[0] = fma(p_own[i], q[i], v[0]);
    double tot[1];
    if (grid_sum_last<1>(v, part, ticket, tot) && threadIdx.x == 0) out[0] = tot[0];
}

// x += alpha p, r -= alpha q; sums r.(D^-1 r), r.r
__global__ void __launch_bounds__(kCgBlock)
part_update_xr(int32_t n, double alpha, double *x, double *r, const double *p_own,
               const double *q, const double *dinv, double *part, unsigned *ticket,
               double *out) {
    double v[2] = {0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        x[i] = fma(alpha, p_own[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        v[0] = fma(ri, dinv[i] * ri, v[0]);
        v[1] = fma(ri, ri, v[1]);
    }
    double tot[2];
    if (grid_sum_last<2>(v, part, ticket, tot) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
    }
}

// p = D^-1 r + beta p
__global__ void part_update_p(int32_t n, double beta, const double *r, const double *dinv,
                              double *p_own) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        p_own[i] = fma(beta, p_own[i], dinv[i] * r[i]);
}

spmv_status_t read_sums(const double *d, double *h, int count, cudaStream_t st) {
    GB_CUDA(cudaMemcpyAsync(h, d, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    return SPMV_OK;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" {

spmv_status_t spmv_partition_create(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                    const int32_t *col_idx, const double *values, int n_parts,
                                    const int32_t *row_begin, int part, int on_device,
                                    const spmv_options_t *opt, void *stream, spmv_part_t *out) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || nnz < 0 || nnz > INT32_MAX || !row_ptr || !row_begin || n_parts < 1 ||
        n_parts > kPartMaxParts || part < 0 || part >= n_parts || (nnz > 0 && !col_idx) ||
        (on_device && nnz > 0 && !values))
        return SPMV_ERR_INVALID_ARG;
    spmv_options_t o;
    spmv_default_options(&o);
    if (opt) o = *opt;
    if (o.reorder != SPMV_REORDER_NONE || o.sigma != 0) return SPMV_ERR_INVALID_ARG;
    spmv_part_s *P = new (std::nothrow) spmv_part_s();
    if (!P) return SPMV_ERR_OOM;
    spmv_status_t s = SPMV_OK;
    try {
        s = build_plan(P, n, nnz, row_ptr, col_idx, values, n_parts, row_begin, part);
    } catch (const std::bad_alloc &) {
        s = SPMV_ERR_OOM;
    }
    if (s == SPMV_OK && on_device) {
        cudaStream_t st = (cudaStream_t)stream;
        s = spmv_create(P->n_local, P->n_ext, (int64_t)P->ci.size(), P->rp.data(),
                        P->ci.empty() ? nullptr : P->ci.data(),
                        P->val.empty() ? nullptr : P->val.data(), 0, &o, stream, &P->A);
        AllocStream scope(st);
        if (s == SPMV_OK) s = P->d_send_rows.alloc((size_t)P->send_total, &P->bytes);
        if (s == SPMV_OK && P->send_total > 0)
            s = cuda_status(cudaMemcpyAsync(P->d_send_rows.p, P->send_rows.data(),
                                            sizeof(int32_t) * P->send_total,
                                            cudaMemcpyHostToDevice, st));
        if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
    }
    if (s != SPMV_OK) {
        spmv_partition_destroy(P);
        return s;
    }
    *out = P;
    return SPMV_OK;
}

spmv_status_t spmv_partition_destroy(spmv_part_t P) {
    if (!P) return SPMV_OK;
    if (P->A || P->d_send_rows.p || P->r.p) {
        cudaDeviceSynchronize();
        AllocStream scope(nullptr);
        size_t *t = &P->bytes;
        P->d_send_rows.release(t);
        P->r.release(t); P->p_ext.release(t); P->q.release(t); P->dinv.release(t);
        P->send.release(t); P->recv.release(t); P->part_sums.release(t); P->sums.release(t);
        P->flag.release(t);
        spmv_destroy(P->A);
        cudaDeviceSynchronize();
    }
    delete P;
    return SPMV_OK;
}

spmv_status_t spmv_partition_info(spmv_part_t P, spmv_part_info_t *info) {
    if (!P || !info) return SPMV_ERR_INVALID_ARG;
    info->n_parts = P->n_parts;
    info->part = P->part;
    info->row_begin = P->row0;
    info->row_end = P->row1;
    info->n_local = P->n_local;
    info->n_halo_lo = P->n_lo;
    info->n_halo_hi = P->n_hi;
    info->n_ext = P->n_ext;
    info->nnz_local = (int64_t)P->ci.size();
    info->send_total = P->send_total;
    info->recv_total = P->n_lo + P->n_hi;
    info->device_bytes = P->bytes + (P->A ? P->A->bytes : 0);
    return SPMV_OK;
}

spmv_status_t spmv_partition_lists(spmv_part_t P, int32_t *send_counts, int32_t *recv_counts,
                                   int32_t *send_rows, int32_t *halo_cols) {
    if (!P) return SPMV_ERR_INVALID_ARG;
    if (send_counts) std::copy(P->send_count.begin(), P->send_count.end(), send_counts);
    if (recv_counts) std::copy(P->recv_count.begin(), P->recv_count.end(), recv_counts);
    if (send_rows) std::copy(P->send_rows.begin(), P->send_rows.end(), send_rows);
    if (halo_cols) std::copy(P->halo.begin(), P->halo.end(), halo_cols);
    return SPMV_OK;
}

spmv_status_t spmv_partition_local_csr(spmv_part_t P, int32_t *row_ptr, int32_t *col_idx,
                                       double *values) {
    if (!P || !row_ptr) return SPMV_ERR_INVALID_ARG;
    std::copy(P->rp.begin(), P->rp.end(), row_ptr);
    if (col_idx) std::copy(P->ci.begin(), P->ci.end(), col_idx);
    if (values) std::copy(P->val.begin(), P->val.end(), values);
    return SPMV_OK;
}

spmv_status_t spmv_partition_pack(spmv_part_t P, const double *x_own_dev, double *send_dev,
                                  void *stream) {
    if (!P || !P->A) return SPMV_ERR_INVALID_ARG;
    if (P->send_total == 0) return SPMV_OK;
    if (!x_own_dev || !send_dev) return SPMV_ERR_INVALID_ARG;
    part_pack<<<grid_of(P->send_total), 256, 0, (cudaStream_t)stream>>>(
        P->send_total, P->d_send_rows.p, x_own_dev, send_dev);
    GB_LAUNCHED();
    return SPMV_OK;
}

spmv_status_t spmv_partition_apply(spmv_part_t P, const double *x_ext_dev, double *y_dev,
                                   void *stream) {
    if (!P || !P->A) return SPMV_ERR_INVALID_ARG;
    return spmv_apply(P->A, x_ext_dev, y_dev, stream);
}

spmv_status_t cg_solve_partitioned(spmv_part_t P, const double *b_dev, double *x_dev,
                                   const cg_options_t *opt, cg_result_t *result,
                                   spmv_exchange_fn exchange, spmv_allreduce_fn allreduce,
                                   void *ctx, void *stream) {
    cg_result_t local{};
    cg_result_t *res = result ? result : &local;
    *res = cg_result_t{};
    res->status = SPMV_ERR_INVALID_ARG;
    if (!P || !P->A || !exchange || !allreduce) return SPMV_ERR_INVALID_ARG;
    if (P->n_local > 0 && (!b_dev || !x_dev || b_dev == x_dev)) return SPMV_ERR_INVALID_ARG;
    cg_options_t o;
    cg_default_options(&o);
    if (opt) o = *opt;
    if (!(o.rtol >= 0.0) || o.max_iter < 1) return SPMV_ERR_INVALID_ARG;
    if (o.mixed || o.persistent) return (res->status = SPMV_ERR_UNSUPPORTED);
    if (!P->A->has64()) return (res->status = SPMV_ERR_UNSUPPORTED);
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream scope(st);
    const int32_t n = P->n_local;
    const size_t one = 1;
    auto fail = [&](spmv_status_t e) { return (res->status = e); };
    size_t *t = &P->bytes;
    if (!P->r.p) {
        spmv_status_t s = P->r.alloc(n > 0 ? n : one, t);
        if (s == SPMV_OK) s = P->p_ext.alloc(P->n_ext > 0 ? P->n_ext : one, t);
        if (s == SPMV_OK) s = P->q.alloc(n > 0 ? n : one, t);
        if (s == SPMV_OK) s = P->dinv.alloc(n > 0 ? n : one, t);
        if (s == SPMV_OK) s = P->send.alloc(P->send_total > 0 ? P->send_total : one, t);
        if (s == SPMV_OK) s = P->recv.alloc(P->n_lo + P->n_hi > 0 ? P->n_lo + P->n_hi : 1, t);
        if (s == SPMV_OK) s = P->part_sums.alloc((size_t)device_facts().sm_count * 4 * 3, t);
        if (s == SPMV_OK) s = P->sums.alloc(8, t);
        if (s == SPMV_OK) s = P->flag.alloc(4, t);
        if (s == SPMV_OK) s = cuda_status(cudaMemsetAsync(P->flag.p, 0, 4 * sizeof(int), st));
        if (s == SPMV_OK && n > 0) {
            part_dinv<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                n, P->n_lo, P->A->row_ptr.p, P->A->col.p, P->A->val.p, P->dinv.p, P->flag.p);
            s = cuda_status(cudaGetLastError());
        }
        if (s != SPMV_OK) return fail(s);
    }
    int h_flag = 0;
    spmv_status_t s = cuda_status(cudaMemcpyAsync(&h_flag, P->flag.p, sizeof(int),
                                                  cudaMemcpyDeviceToHost, st));
    if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
    if (s != SPMV_OK) return fail(s);
    double g[3] = {0.0, 0.0, 0.0};  // a part with a zero diagonal makes every part fail
    g[0] = h_flag ? 1.0 : 0.0;
    if (allreduce(g, 1, ctx) != 0) return fail(SPMV_ERR_CUDA);
    if (g[0] != 0.0) return fail(SPMV_ERR_INVALID_CSR);
    double *p_own = P->p_ext.p + P->n_lo;
    unsigned *ticket = (unsigned *)P->flag.p + 1;
    const unsigned G = grid_of(n);
    // halo exchange of the own part of v (x_ext layout): pack, transport, place the runs
    auto exchange_ext = [&](double *v_ext) -> spmv_status_t {
        GB_TRY(spmv_partition_pack(P, v_ext + P->n_lo, P->send.p, st));
        GB_CUDA(cudaStreamSynchronize(st));
        if (exchange(P->send.p, P->recv.p, ctx) != 0) return SPMV_ERR_CUDA;
        if (P->n_lo > 0)
            GB_CUDA(cudaMemcpyAsync(v_ext, P->recv.p, sizeof(double) * P->n_lo,
                                    cudaMemcpyDeviceToDevice, st));
        if (P->n_hi > 0)
            GB_CUDA(cudaMemcpyAsync(v_ext + P->n_lo + n, P->recv.p + P->n_lo,
                                    sizeof(double) * P->n_hi, cudaMemcpyDeviceToDevice, st));
        return SPMV_OK;
    };
    // r = b - A x0 (x0 = 0 unless use_x0), p = D^-1 r; global r.z, r.r, b.b
    if (o.use_x0) {
        if (n > 0)
            s = cuda_status(cudaMemcpyAsync(p_own, x_dev, sizeof(double) * n,
                                            cudaMemcpyDeviceToDevice, st));
        if (s == SPMV_OK) s = exchange_ext(P->p_ext.p);
        if (s == SPMV_OK) s = spmv_apply(P->A, P->p_ext.p, P->q.p, st);
    } else if (n > 0) {
        s = cuda_status(cudaMemsetAsync(x_dev, 0, sizeof(double) * n, st));
    }
    if (s != SPMV_OK) return fail(s);
    part_residual<<<G, kCgBlock, 0, st>>>(n, b_dev, o.use_x0 ? P->q.p : nullptr, P->r.p, p_own,
                                          P->dinv.p, P->part_sums.p, ticket, P->sums.p);
    s = cuda_status(cudaGetLastError());
    if (s == SPMV_OK) s = read_sums(P->sums.p, g, 3, st);
    if (s != SPMV_OK) return fail(s);
    if (allreduce(g, 3, ctx) != 0) return fail(SPMV_ERR_CUDA);
    double rho = g[0], rr = g[1];
    const double bb = g[2], tol2 = o.rtol * o.rtol;
    int it = 0;
    res->status = SPMV_OK;
    while (!(rr <= tol2 * bb)) {
        if (it >= o.max_iter) {
            res->status = SPMV_ERR_NOT_CONVERGED;
            break;
        }
        // q = A p over the extended p: the halo first
        s = exchange_ext(P->p_ext.p);
        if (s == SPMV_OK) s = spmv_apply(P->A, P->p_ext.p, P->q.p, st);
        if (s != SPMV_OK) return fail(s);
        part_dot<<<G, kCgBlock, 0, st>>>(n, p_own, P->q.p, P->part_sums.p, ticket, P->sums.p);
        s = cuda_status(cudaGetLastError());
        if (s == SPMV_OK) s = read_sums(P->sums.p, g, 1, st);
        if (s != SPMV_OK) return fail(s);
        if (allreduce(g, 1, ctx) != 0) return fail(SPMV_ERR_CUDA);
        if (g[0] == 0.0 || !std::isfinite(g[0])) {
            res->status = SPMV_ERR_NOT_CONVERGED;
            break;
        }
        const double alpha = rho / g[0];
        part_update_xr<<<G, kCgBlock, 0, st>>>(n, alpha, x_dev, P->r.p, p_own, P->q.p, P->dinv.p,
                                               P->part_sums.p, ticket, P->sums.p);
        s = cuda_status(cudaGetLastError());
        if (s == SPMV_OK) s = read_sums(P->sums.p, g, 2, st);
        if (s != SPMV_OK) return fail(s);
        if (allreduce(g, 2, ctx) != 0) return fail(SPMV_ERR_CUDA);
        ++it;
        const double beta = g[0] / rho;
        rho = g[0];
        rr = g[1];
        if (!std::isfinite(rr)) {
            res->status = SPMV_ERR_NOT_CONVERGED;
            break;
        }
        if (rr <= tol2 * bb) break;
        part_update_p<<<G, kCgBlock, 0, st>>>(n, beta, P->r.p, P->dinv.p, p_own);
        s = cuda_status(cudaGetLastError());
        if (s != SPMV_OK) return fail(s);
    }
    // true residual ||b - A x|| / ||b|| over all parts
    if (n > 0)
        s = cuda_status(cudaMemcpyAsync(p_own, x_dev, sizeof(double) * n,
                                        cudaMemcpyDeviceToDevice, st));
    if (s == SPMV_OK) s = exchange_ext(P->p_ext.p);
    if (s == SPMV_OK) s = spmv_apply(P->A, P->p_ext.p, P->q.p, st);
    if (s != SPMV_OK) return fail(s);
    part_residual<<<G, kCgBlock, 0, st>>>(n, b_dev, P->q.p, P->r.p, nullptr, P->dinv.p,
                                          P->part_sums.p, ticket, P->sums.p);
    s = cuda_status(cudaGetLastError());
    if (s == SPMV_OK) s = read_sums(P->sums.p, g, 3, st);
    if (s != SPMV_OK) return fail(s);
    if (allreduce(g, 3, ctx) != 0) return fail(SPMV_ERR_CUDA);
    res->iterations = it;
    res->rel_residual = g[2] > 0.0 ? std::sqrt(g[1] / g[2]) : 0.0;
    return res->status;
}

}  // extern "C"
