// convert.cu -- one-time pre-processing of a matrix on the device:
//   CSR validation; (reverse) Cuthill-McKee ordering by level-synchronous BFS (Sec. 4.1);
//   the symmetric permutation P A P^T; FP32 value copy; conversion to sliced ELLPACK with S
//   rows per slice, column-major inside a slice (Sec. 4.2); per-slice x range (Sec. 5.1).
// The paper applies these once per simulation, so their cost is amortised (Sec. 2, 4.1).
#include <climits>
#include <vector>

#include "common.cuh"

namespace gb {
namespace {

constexpr int kT = 256;

inline unsigned blocks_for(int64_t n, int t = kT) {
    int64_t b = (n + t - 1) / t;
    return (unsigned)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------------------------------
// validation: row_ptr[0] = 0, row_ptr[n] = nnz, monotone, columns in range and strictly
// increasing inside each row.  Bits of *err: 1 ends, 2 monotone, 4 range, 8 order.
// ---------------------------------------------------------------------------------------
__global__ void validate_csr(int32_t n, int32_t n_cols, int64_t nnz, const int32_t *rp,
                             const int32_t *ci, int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (rp[0] != 0 || (int64_t)rp[n] != nnz)) atomicOr(err, 1);
    if (i >= n) return;
    int32_t a = rp[i], b = rp[i + 1];
    if (a > b || a < 0 || (int64_t)b > nnz) {
        atomicOr(err, 2);
        return;
    }
    int32_t prev = -1;
    for (int32_t k = a; k < b; ++k) {
        int32_t c = ci[k];
        if (c < 0 || c >= n_cols) {
            atomicOr(err, 4);
            return;
        }
        if (c <= prev) {
            atomicOr(err, 8);
            return;
        }
        prev = c;
    }
}

// ---------------------------------------------------------------------------------------
// Cuthill-McKee on the device.  A node's key is (degree, index); pos[v] = -1 until placed.
// ---------------------------------------------------------------------------------------
__global__ void degree_kernel(int32_t n, const int32_t *rp, const int32_t *ci, int32_t *deg) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t d = 0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) d += (ci[k] != (int32_t)i);
    deg[i] = d;
}

__device__ __forceinline__ unsigned long long node_key(const int32_t *deg, int32_t v) {
    return ((unsigned long long)(uint32_t)deg[v] << 32) | (uint32_t)v;
}

// min key over unplaced nodes
__global__ void min_key_unplaced(int32_t n, const int32_t *deg, const int32_t *pos,
                                 unsigned long long *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || pos[i] != -1) return;
    atomicMin(out, node_key(deg, (int32_t)i));
}

// min key over queue[ls, le)
__global__ void min_key_range(const int32_t *queue, int64_t ls, int64_t le, const int32_t *deg,
                              unsigned long long *out) {
    int64_t p = ls + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= le) return;
    atomicMin(out, node_key(deg, queue[p]));
}

__global__ void bfs_seed(int32_t r, int32_t id, int32_t *stamp, int32_t *queue, int32_t *tail) {
    stamp[r] = id;
    queue[0] = r;
    *tail = 1;
}

// expand one BFS level (level sets only, order irrelevant), restricted to unplaced nodes
__global__ void bfs_expand(const int32_t *rp, const int32_t *ci, const int32_t *pos, int32_t id,
                           int32_t *stamp, int32_t *queue, int64_t ls, int64_t le,
                           int32_t *tail) {
    int64_t p = ls + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= le) return;
    int32_t u = queue[p];
    for (int32_t k = rp[u]; k < rp[u + 1]; ++k) {
        int32_t v = ci[k];
        if (v == u || pos[v] != -1) continue;
        if (stamp[v] == id) continue;
        if (atomicExch(&stamp[v], id) != id) queue[atomicAdd(tail, 1)] = v;
    }
}

__global__ void place_start(int32_t v, int64_t at, int32_t *perm, int32_t *pos) {
    perm[at] = v;
    pos[v] = (int32_t)at;
}

// every unplaced neighbour of a frontier node records the earliest frontier position
__global__ void cm_claim(const int32_t *rp, const int32_t *ci, const int32_t *perm,
                         const int32_t *pos, int32_t *claim, int64_t ls, int64_t le) {
    int64_t p = ls + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= le) return;
    int32_t u = perm[p];
    for (int32_t k = rp[u]; k < rp[u + 1]; ++k) {
        int32_t v = ci[k];
        if (v != u && pos[v] == -1) atomicMin(&claim[v], (int32_t)p);
    }
}

__global__ void cm_count(const int32_t *rp, const int32_t *ci, const int32_t *perm,
                         const int32_t *pos, const int32_t *claim, int64_t ls, int64_t le,
                         int64_t *counts) {
    int64_t p = ls + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= le) return;
    int32_t u = perm[p];
    int64_t c = 0;
    for (int32_t k = rp[u]; k < rp[u + 1]; ++k) {
        int32_t v = ci[k];
        c += (v != u && pos[v] == -1 && claim[v] == (int32_t)p);
    }
    counts[p - ls] = c;
}

// children of frontier position p, appended in increasing (degree, index) by repeated
// selection of the next larger key (no buffer, any row length)
__global__ void cm_place(const int32_t *rp, const int32_t *ci, const int32_t *deg,
                         int32_t *perm, const int32_t *pos, const int32_t *claim, int64_t ls,
                         int64_t le, const int64_t *offsets) {
    int64_t p = ls + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= le) return;
    int32_t u = perm[p];
    int64_t at = le + offsets[p - ls];
    int64_t cnt = offsets[p - ls + 1] - offsets[p - ls];
    unsigned long long last = 0;
    bool first = true;
    for (int64_t t = 0; t < cnt; ++t) {
        unsigned long long best = ~0ull;
        for (int32_t k = rp[u]; k < rp[u + 1]; ++k) {
            int32_t v = ci[k];
            if (v == u || pos[v] != -1 || claim[v] != (int32_t)p) continue;
            unsigned long long key = node_key(deg, v);
            if ((first || key > last) && key < best) best = key;
        }
        perm[at + t] = (int32_t)(best & 0xffffffffull);
        last = best;
        first = false;
    }
}

__global__ void set_pos(const int32_t *perm, int64_t a, int64_t b, int32_t *pos) {
    int64_t q = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < b) pos[perm[q]] = (int32_t)q;
}

__global__ void reverse_kernel(int32_t n, const int32_t *src, int32_t *dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[n - 1 - i];
}

__global__ void fill_i32(int32_t *p, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

struct CmScratch {
    int32_t *deg = nullptr, *pos = nullptr, *claim = nullptr, *stamp = nullptr,
            *queue = nullptr, *cm = nullptr, *tail = nullptr;
    int64_t *counts = nullptr;
    unsigned long long *key = nullptr;
    void *host = nullptr;  // pinned: [0] = int64 scratch, [1] = key
};

spmv_status_t read_i64(const int64_t *d, int64_t *h, void *pinned, cudaStream_t st) {
    GB_CUDA(cudaMemcpyAsync(pinned, d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    *h = *(int64_t *)pinned;
    return SPMV_OK;
}

spmv_status_t read_i32(const int32_t *d, int32_t *h, void *pinned, cudaStream_t st) {
    GB_CUDA(cudaMemcpyAsync(pinned, d, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    *h = *(int32_t *)pinned;
    return SPMV_OK;
}

spmv_status_t read_key(const unsigned long long *d, unsigned long long *h, void *pinned,
                       cudaStream_t st) {
    GB_CUDA(cudaMemcpyAsync(pinned, d, sizeof(*d), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    *h = *(unsigned long long *)pinned;
    return SPMV_OK;
}

// BFS level structure from r over unplaced nodes; eccentricity and the min-key node of the
// last level.
spmv_status_t bfs_ecc(int32_t n, const int32_t *rp, const int32_t *ci, CmScratch &w,
                      int32_t r, int32_t id, cudaStream_t st, int32_t *ecc, int32_t *pick) {
    bfs_seed<<<1, 1, 0, st>>>(r, id, w.stamp, w.queue, w.tail);
    GB_LAUNCHED();
    int64_t ls = 0, le = 1;
    int32_t levels = 0;
    int64_t last_ls = 0, last_le = 1;
    while (le > ls) {
        last_ls = ls;
        last_le = le;
        bfs_expand<<<blocks_for(le - ls), kT, 0, st>>>(rp, ci, w.pos, id, w.stamp, w.queue, ls,
                                                       le, w.tail);
        GB_LAUNCHED();
        int32_t t;
        GB_TRY(read_i32(w.tail, &t, w.host, st));
        ls = le;
        le = t;
        if (le > ls) ++levels;
    }
    GB_CUDA(cudaMemsetAsync(w.key, 0xff, sizeof(unsigned long long), st));
    min_key_range<<<blocks_for(last_le - last_ls), kT, 0, st>>>(w.queue, last_ls, last_le, w.deg,
                                                               w.key);
    GB_LAUNCHED();
    unsigned long long k;
    GB_TRY(read_key(w.key, &k, w.host, st));
    *ecc = levels;
    *pick = (int32_t)(k & 0xffffffffull);
    (void)n;
    return SPMV_OK;
}

spmv_status_t cm_order_device(int32_t n, const int32_t *rp, const int32_t *ci, bool reverse,
                              bool peripheral, int32_t *perm_out, cudaStream_t st) {
    if (n == 0) return SPMV_OK;
    CmScratch w;
    spmv_status_t s = SPMV_OK;
    auto alloc = [&](void **p, size_t bytes) {
        if (s != SPMV_OK) return;
        s = cuda_status(gb_malloc_async(p, bytes, st));
    };
    alloc((void **)&w.deg, sizeof(int32_t) * n);
    alloc((void **)&w.pos, sizeof(int32_t) * n);
    alloc((void **)&w.claim, sizeof(int32_t) * n);
    alloc((void **)&w.stamp, sizeof(int32_t) * n);
    alloc((void **)&w.queue, sizeof(int32_t) * n);
    alloc((void **)&w.cm, sizeof(int32_t) * n);
    alloc((void **)&w.tail, sizeof(int32_t));
    alloc((void **)&w.counts, sizeof(int64_t) * ((size_t)n + 1));
    alloc((void **)&w.key, sizeof(unsigned long long));
    if (s == SPMV_OK) s = cuda_status(cudaMallocHost(&w.host, 64));
    if (s == SPMV_OK) {
        s = [&]() -> spmv_status_t {
            const unsigned nb = blocks_for(n);
            degree_kernel<<<nb, kT, 0, st>>>(n, rp, ci, w.deg);
            fill_i32<<<nb, kT, 0, st>>>(w.pos, n, -1);
            fill_i32<<<nb, kT, 0, st>>>(w.claim, n, INT_MAX);
            fill_i32<<<nb, kT, 0, st>>>(w.stamp, n, -1);
            GB_LAUNCHED();
            int32_t bfs_id = 0;
            int64_t placed = 0;
            while (placed < n) {
                GB_CUDA(cudaMemsetAsync(w.key, 0xff, sizeof(unsigned long long), st));
                min_key_unplaced<<<nb, kT, 0, st>>>(n, w.deg, w.pos, w.key);
                GB_LAUNCHED();
                unsigned long long k;
                GB_TRY(read_key(w.key, &k, w.host, st));
                int32_t start = (int32_t)(k & 0xffffffffull);
                if (peripheral) {
                    int32_t ecc, pick;
                    GB_TRY(bfs_ecc(n, rp, ci, w, start, bfs_id++, st, &ecc, &pick));
                    for (int moves = 0; moves < 8; ++moves) {
                        int32_t ecc2, pick2;
                        GB_TRY(bfs_ecc(n, rp, ci, w, pick, bfs_id++, st, &ecc2, &pick2));
                        if (ecc2 > ecc) {
                            start = pick;
                            ecc = ecc2;
                            pick = pick2;
                        } else {
                            break;
                        }
                    }
                }
                place_start<<<1, 1, 0, st>>>(start, placed, w.cm, w.pos);
                GB_LAUNCHED();
                int64_t ls = placed, le = placed + 1;
                placed += 1;
                while (le > ls) {
                    const int64_t nf = le - ls;
                    const unsigned fb = blocks_for(nf);
                    cm_claim<<<fb, kT, 0, st>>>(rp, ci, w.cm, w.pos, w.claim, ls, le);
                    cm_count<<<fb, kT, 0, st>>>(rp, ci, w.cm, w.pos, w.claim, ls, le, w.counts);
                    GB_LAUNCHED();
                    GB_TRY(exclusive_scan_i64(w.counts, nf, st));
                    cm_place<<<fb, kT, 0, st>>>(rp, ci, w.deg, w.cm, w.pos, w.claim, ls, le,
                                                w.counts);
                    GB_LAUNCHED();
                    int64_t total;
                    GB_TRY(read_i64(w.counts + nf, &total, w.host, st));
                    if (total > 0) {
                        set_pos<<<blocks_for(total), kT, 0, st>>>(w.cm, le, le + total, w.pos);
                        GB_LAUNCHED();
                    }
                    ls = le;
                    le = le + total;
                    placed = le;
                }
            }
            if (reverse) {
                reverse_kernel<<<nb, kT, 0, st>>>(n, w.cm, perm_out);
            } else {
                GB_CUDA(cudaMemcpyAsync(perm_out, w.cm, sizeof(int32_t) * n,
                                        cudaMemcpyDeviceToDevice, st));
            }
            GB_LAUNCHED();
            return SPMV_OK;
        }();
    }
    GB_CUDA(cudaStreamSynchronize(st));
    cudaFreeAsync(w.deg, st);
    cudaFreeAsync(w.pos, st);
    cudaFreeAsync(w.claim, st);
    cudaFreeAsync(w.stamp, st);
    cudaFreeAsync(w.queue, st);
    cudaFreeAsync(w.cm, st);
    cudaFreeAsync(w.tail, st);
    cudaFreeAsync(w.counts, st);
    cudaFreeAsync(w.key, st);
    if (w.host) cudaFreeHost(w.host);
    return s;
}

// ---------------------------------------------------------------------------------------
// length sorting inside windows of sigma rows (sliced ELLPACK with a sorting scope, ref.
// MON10): rows taken in the order perm_in (nullptr = identity) are reordered inside each window
// by decreasing length, equal lengths keeping their order, so the slices of a window pad less.
// One CTA per window: bitonic sort of the unique keys (INT_MAX - length, position).
// ---------------------------------------------------------------------------------------
__global__ void sigma_sort_kernel(int32_t n, int32_t sigma, const int32_t *rp,
                                  const int32_t *perm_in, int32_t *perm_out) {
    extern __shared__ unsigned long long keys[];
    const int64_t w0 = (int64_t)blockIdx.x * sigma;
    const int cnt = (int)((n - w0) < sigma ? (n - w0) : sigma);
    for (int j = threadIdx.x; j < sigma; j += blockDim.x) {
        if (j < cnt) {
            const int32_t old = perm_in ? perm_in[w0 + j] : (int32_t)(w0 + j);
            const uint32_t len = (uint32_t)(rp[old + 1] - rp[old]);
            keys[j] = ((unsigned long long)(0x7fffffffu - len) << 32) | (uint32_t)j;
        } else {
            keys[j] = ~0ull;
        }
    }
    __syncthreads();
    for (int k = 2; k <= sigma; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < sigma; i += blockDim.x) {
                const int ixj = i ^ jj;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long a = keys[i], b = keys[ixj];
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const int32_t src = (int32_t)(keys[j] & 0xffffffffull);
        perm_out[w0 + j] = perm_in ? perm_in[w0 + src] : (int32_t)(w0 + src);
    }
}

// ---------------------------------------------------------------------------------------
// symmetric permutation B = P A P^T (perm[new] = old), rows sorted by new column
// ---------------------------------------------------------------------------------------
__global__ void inverse_perm(int32_t n, const int32_t *perm, int32_t *inv) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) inv[perm[r]] = (int32_t)r;
}

__global__ void permuted_lengths(int32_t n, const int32_t *rp, const int32_t *perm,
                                 int64_t *len) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) len[r] = rp[perm[r] + 1] - rp[perm[r]];
}

__global__ void i64_to_i32(const int64_t *a, int32_t *b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (int32_t)a[i];
}

__global__ void permute_rows(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                             const int32_t *perm, const int32_t *inv, const int32_t *rp_out,
                             int32_t *ci_out, double *val_out) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int32_t old = perm[r];
    const int32_t a = rp[old];
    const int32_t len = rp[old + 1] - a;
    const int32_t base = rp_out[r];
    for (int32_t t = 0; t < len; ++t) {
        ci_out[base + t] = inv[ci[a + t]];
        val_out[base + t] = val[a + t];
    }
    for (int32_t t = 1; t < len; ++t) {  // insertion sort by column
        int32_t c = ci_out[base + t];
        double v = val_out[base + t];
        int32_t b = t - 1;
        while (b >= 0 && ci_out[base + b] > c) {
            ci_out[base + b + 1] = ci_out[base + b];
            val_out[base + b + 1] = val_out[base + b];
            --b;
        }
        ci_out[base + b + 1] = c;
        val_out[base + b + 1] = v;
    }
}

__global__ void to_f32(const double *a, float *b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __double2float_rn(a[i]);
}

__global__ void bandwidth_kernel(int32_t n, const int32_t *rp, const int32_t *ci, int *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = rp[i], b = rp[i + 1];
    if (a == b) return;
    int32_t d0 = (int32_t)i - ci[a];
    int32_t d1 = ci[b - 1] - (int32_t)i;
    atomicMax(out, d0 > d1 ? d0 : d1);
}

// ---------------------------------------------------------------------------------------
// sliced ELLPACK (Sec. 4.2) and the per-slice x range (Sec. 5.1)
// ---------------------------------------------------------------------------------------
__global__ void slice_sizes(int32_t n, int32_t S, int32_t n_slices, const int32_t *rp,
                            int64_t *sp) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slices) return;
    int32_t w = 0;
    int64_t r0 = s * S;
    for (int64_t r = r0; r < r0 + S && r < n; ++r) {
        int32_t len = rp[r + 1] - rp[r];
        w = len > w ? len : w;
    }
    sp[s] = (int64_t)S * w;
}

template <bool F64, bool F32>
__global__ void sell_scatter(int32_t n, int32_t S, int64_t n_pad, const int32_t *rp,
                             const int32_t *ci, const double *val, const float *val32,
                             const int64_t *sp, int32_t *scol, double *sval, float *sval32) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    const int64_t s = r / S;
    const int64_t lane = r - s * S;
    const int64_t base = sp[s];
    const int64_t w = (sp[s + 1] - base) / S;
    const int32_t a = r < n ? rp[r] : 0;
    const int32_t len = r < n ? rp[r + 1] - a : 0;
    for (int64_t t = 0; t < w; ++t) {
        const int64_t at = base + t * S + lane;
        if (t < len) {
            scol[at] = ci[a + t];
            if (F64) sval[at] = val[a + t];
            if (F32) sval32[at] = val32[a + t];
        } else {
            scol[at] = -1;
            if (F64) sval[at] = 0.0;
            if (F32) sval32[at] = 0.0f;
        }
    }
}

__global__ void window_meta(int32_t n_slices, int32_t S, const int64_t *sp, const int32_t *scol,
                            int32_t *cs, int32_t *ce, int *max_span_width) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= n_slices) return;
    int32_t lo = INT_MAX, hi = -1;
    for (int64_t at = sp[s] + lane; at < sp[s + 1]; at += 32) {
        int32_t c = scol[at];
        if (c < 0) continue;
        lo = c < lo ? c : lo;
        hi = c > hi ? c : hi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int32_t l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        int32_t h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    if (lane == 0) {
        if (hi < 0) {
            cs[s] = 0;
            ce[s] = 0;
        } else {
            cs[s] = lo;
            ce[s] = hi + 1;
            atomicMax(max_span_width, hi + 1 - lo);
        }
        atomicMax(max_span_width + 1, (int)((sp[s + 1] - sp[s]) / S));
    }
}

// 16-bit columns relative to the slice's first column (Sec. 5.1); padding -> 0xFFFF
__global__ void relative_cols16(int32_t n_slices, const int64_t *sp, const int32_t *scol,
                                const int32_t *cs, uint16_t *out) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= n_slices) return;
    const int32_t base = cs[s];
    for (int64_t at = sp[s] + lane; at < sp[s + 1]; at += 32) {
        const int32_t c = scol[at];
        out[at] = c < 0 ? (uint16_t)0xFFFFu : (uint16_t)(c - base);
    }
}

}  // namespace

spmv_status_t build_sell(spmv_matrix_t A, int S, cudaStream_t st) {
    NvtxRange nvtx("spmv_create/sliced_ellpack");
    const int32_t n = A->n;
    const int32_t n_slices = (int32_t)(((int64_t)n + S - 1) / S);
    size_t *tally = &A->bytes;
    A->S = S;
    A->n_slices = n_slices;
    GB_TRY(A->slice_ptr.alloc((size_t)n_slices + 1, tally));
    slice_sizes<<<blocks_for(n_slices), kT, 0, st>>>(n, S, n_slices, A->row_ptr.p, A->slice_ptr.p);
    GB_LAUNCHED();
    GB_TRY(exclusive_scan_i64(A->slice_ptr.p, n_slices, st));
    int64_t total = 0;
    GB_CUDA(cudaMemcpyAsync(&total, A->slice_ptr.p + n_slices, sizeof(int64_t),
                            cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    A->sell_entries = total;
    GB_TRY(A->sell_col.alloc((size_t)total, tally));
    if (A->has64()) GB_TRY(A->sell_val.alloc((size_t)total, tally));
    else A->sell_val.release(tally);
    if (A->has32()) GB_TRY(A->sell_val32.alloc((size_t)total, tally));
    else A->sell_val32.release(tally);
    const int64_t n_pad = (int64_t)n_slices * S;
    const unsigned nb = blocks_for(n_pad);
    if (A->has64() && A->has32())
        sell_scatter<true, true><<<nb, kT, 0, st>>>(n, S, n_pad, A->row_ptr.p, A->col.p, A->val.p,
                                                    A->val32.p, A->slice_ptr.p, A->sell_col.p,
                                                    A->sell_val.p, A->sell_val32.p);
    else if (A->has64())
        sell_scatter<true, false><<<nb, kT, 0, st>>>(n, S, n_pad, A->row_ptr.p, A->col.p, A->val.p,
                                                     nullptr, A->slice_ptr.p, A->sell_col.p,
                                                     A->sell_val.p, nullptr);
    else
        sell_scatter<false, true><<<nb, kT, 0, st>>>(n, S, n_pad, A->row_ptr.p, A->col.p, nullptr,
                                                     A->val32.p, A->slice_ptr.p, A->sell_col.p,
                                                     nullptr, A->sell_val32.p);
    GB_LAUNCHED();
    GB_TRY(A->col_start.alloc((size_t)n_slices, tally));
    GB_TRY(A->col_end.alloc((size_t)n_slices, tally));
    int *d_span = nullptr;  // max span, max width
    GB_CUDA(gb_malloc_async((void **)&d_span, 2 * sizeof(int), st));
    cudaMemsetAsync(d_span, 0, 2 * sizeof(int), st);
    window_meta<<<blocks_for((int64_t)n_slices * 32), kT, 0, st>>>(
        n_slices, S, A->slice_ptr.p, A->sell_col.p, A->col_start.p, A->col_end.p, d_span);
    spmv_status_t s = cuda_status(cudaGetLastError());
    int span_width[2] = {0, 0};
    if (s == SPMV_OK)
        s = cuda_status(cudaMemcpyAsync(span_width, d_span, 2 * sizeof(int),
                                        cudaMemcpyDeviceToHost, st));
    cudaFreeAsync(d_span, st);
    if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
    if (s != SPMV_OK) return s;
    const int span = span_width[0];
    A->max_span = span;
    A->max_width = span_width[1];
    GB_TRY(bulk_partition(A, st));
    if (!A->dev_status.p) {
        GB_TRY(A->dev_status.alloc(1, tally));
        GB_CUDA(cudaMemsetAsync(A->dev_status.p, 0, sizeof(int), st));
    }
    // 16-bit relative columns when every slice spans fewer than 65,535 columns
    const int want = A->opt.index_bits;
    A->sell_col16.release(tally);
    A->index_bits = 32;
    if (want != 32 && span < 65535 && total > 0) {
        GB_TRY(A->sell_col16.alloc((size_t)total, tally));
        relative_cols16<<<blocks_for((int64_t)n_slices * 32), kT, 0, st>>>(
            n_slices, A->slice_ptr.p, A->sell_col.p, A->col_start.p, A->sell_col16.p);
        GB_LAUNCHED();
        A->index_bits = 16;
    }
    return SPMV_OK;
}

spmv_status_t build_matrix(spmv_matrix_t A, const int32_t *d_rp, const int32_t *d_ci,
                           const double *d_val, cudaStream_t st) {
    const int32_t n = A->n;
    const int64_t nnz = A->nnz;
    size_t *tally = &A->bytes;

    // 1. validation
    {
        int *d_err = nullptr;
        GB_CUDA(gb_malloc_async((void **)&d_err, sizeof(int), st));
        cudaMemsetAsync(d_err, 0, sizeof(int), st);
        validate_csr<<<blocks_for(n), kT, 0, st>>>(n, A->n_cols, nnz, d_rp, d_ci, d_err);
        spmv_status_t s = cuda_status(cudaGetLastError());
        int err = 0;
        if (s == SPMV_OK)
            s = cuda_status(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        cudaFreeAsync(d_err, st);
        if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
        if (s != SPMV_OK) return s;
        if (err) return SPMV_ERR_INVALID_CSR;
    }

    GB_TRY(A->row_ptr.alloc((size_t)n + 1, tally));
    GB_TRY(A->col.alloc((size_t)nnz, tally));
    GB_TRY(A->val.alloc((size_t)nnz, tally));

    // 2. ordering (Sec. 4.1), optional length sorting inside windows, symmetric permutation
    NvtxRange nvtx_order("spmv_create/reorder");
    const bool reorder = A->opt.reorder != SPMV_REORDER_NONE;
    const int sigma = A->opt.sigma;
    if ((reorder || sigma > 0) && n > 0) {
        GB_TRY(A->perm.alloc((size_t)n, tally));
        if (reorder)
            GB_TRY(cm_order_device(n, d_rp, d_ci, A->opt.reorder == SPMV_REORDER_RCM,
                                   A->opt.peripheral != 0, A->perm.p, st));
        if (sigma > 0) {
            int32_t *tmp = nullptr;
            GB_CUDA(gb_malloc_async((void **)&tmp, sizeof(int32_t) * n, st));
            const unsigned windows = (unsigned)(((int64_t)n + sigma - 1) / sigma);
            sigma_sort_kernel<<<windows, 1024, sizeof(unsigned long long) * sigma, st>>>(
                n, sigma, d_rp, reorder ? A->perm.p : nullptr, tmp);
            spmv_status_t s = cuda_status(cudaGetLastError());
            if (s == SPMV_OK)
                s = cuda_status(cudaMemcpyAsync(A->perm.p, tmp, sizeof(int32_t) * n,
                                                cudaMemcpyDeviceToDevice, st));
            cudaFreeAsync(tmp, st);
            if (s != SPMV_OK) return s;
        }
        int32_t *inv = nullptr;
        int64_t *len = nullptr;
        GB_CUDA(gb_malloc_async((void **)&inv, sizeof(int32_t) * n, st));
        GB_CUDA(gb_malloc_async((void **)&len, sizeof(int64_t) * ((size_t)n + 1), st));
        const unsigned nb = blocks_for(n);
        inverse_perm<<<nb, kT, 0, st>>>(n, A->perm.p, inv);
        permuted_lengths<<<nb, kT, 0, st>>>(n, d_rp, A->perm.p, len);
        spmv_status_t s = cuda_status(cudaGetLastError());
        if (s == SPMV_OK) s = exclusive_scan_i64(len, n, st);
        if (s == SPMV_OK) {
            i64_to_i32<<<blocks_for((int64_t)n + 1), kT, 0, st>>>(len, A->row_ptr.p, (int64_t)n + 1);
            permute_rows<<<nb, kT, 0, st>>>(n, d_rp, d_ci, d_val, A->perm.p, inv, A->row_ptr.p,
                                            A->col.p, A->val.p);
            s = cuda_status(cudaGetLastError());
        }
        cudaFreeAsync(inv, st);
        cudaFreeAsync(len, st);
        if (s != SPMV_OK) return s;
    } else {
        GB_CUDA(cudaMemcpyAsync(A->row_ptr.p, d_rp, sizeof(int32_t) * ((size_t)n + 1),
                                cudaMemcpyDeviceToDevice, st));
        if (nnz) {
            GB_CUDA(cudaMemcpyAsync(A->col.p, d_ci, sizeof(int32_t) * nnz,
                                    cudaMemcpyDeviceToDevice, st));
            GB_CUDA(cudaMemcpyAsync(A->val.p, d_val, sizeof(double) * nnz,
                                    cudaMemcpyDeviceToDevice, st));
        }
    }

    // 3. FP32 copy of the values
    if (A->has32()) {
        GB_TRY(A->val32.alloc((size_t)nnz, tally));
        to_f32<<<blocks_for(nnz), kT, 0, st>>>(A->val.p, A->val32.p, nnz);
        GB_LAUNCHED();
    }

    // 4. bandwidth (reported; Sec. 4.1 defines it as the band width the reordering shrinks)
    {
        int *d_bw = nullptr;
        GB_CUDA(gb_malloc_async((void **)&d_bw, sizeof(int), st));
        cudaMemsetAsync(d_bw, 0, sizeof(int), st);
        bandwidth_kernel<<<blocks_for(n), kT, 0, st>>>(n, A->row_ptr.p, A->col.p, d_bw);
        spmv_status_t s = cuda_status(cudaGetLastError());
        int bw = 0;
        if (s == SPMV_OK)
            s = cuda_status(cudaMemcpyAsync(&bw, d_bw, sizeof(int), cudaMemcpyDeviceToHost, st));
        cudaFreeAsync(d_bw, st);
        if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
        if (s != SPMV_OK) return s;
        A->bandwidth = bw;
    }

    // 5. sliced ELLPACK + per-slice x range
    GB_TRY(build_sell(A, A->S, st));
    return SPMV_OK;
}

}  // namespace gb
