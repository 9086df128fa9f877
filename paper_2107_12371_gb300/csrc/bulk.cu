// bulk.cu -- sliced-ELLPACK product with the matrix staged in shared memory by bulk
// asynchronous copies (Sec. 4.2 layout, Sec. 4.3 product, Sec. 5.1 column ranges).
//
// One CTA per SM walks a contiguous run of slices, the runs balanced by stored entries.  Each
// warp of the CTA owns a ring of K one-slice buffers in shared memory and K mbarriers of its
// own: lane 0 copies the warp's next slices -- values and column indices, each contiguous in
// the sliced-ELLPACK arrays -- with cp.async.bulk (completion counted in bytes on the slot's
// mbarrier) while all lanes multiply the current slice from shared memory, gather x (kept
// resident in L2) and accumulate every row in ascending column order with FMA from +0.0: the
// order of the register-streaming kernel, so both give the same bits.  The HBM latency of the
// matrix stream leaves the warps' dependency chains (they wait only for x gathers), and the
// warps never wait on each other.
//
// Every wait is bounded (1 s of %globaltimer).  A warp that gives up records it in the
// handle's device status word, waits (bounded) for the copies it has in flight and exits.
#include <atomic>
#include <cstring>

#include "common.cuh"
#include "ptx.cuh"

namespace gb {
namespace {

constexpr int kBulkMaxWarps = 32;
constexpr int kBulkMaxSlots = 4;
constexpr int kBulkHeader = kBulkMaxWarps * kBulkMaxSlots * 8;  // the mbarriers
constexpr unsigned long long kBulkWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long bulk_clock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits until the phase of the given parity has completed; false after kBulkWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = bulk_clock();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (bulk_clock() - t0 > kBulkWaitNs) return false;
    }
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16), completion
// counted on the mbarrier; the matrix is read once, so it is marked evict-first in L2
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}

// B bytes from shared memory (B-aligned) into registers
template <int B>
__device__ __forceinline__ void lds_bytes(const void *p, void *out) {
    if constexpr (B % 16 == 0) {
#pragma unroll
        for (int k = 0; k < B / 16; ++k) {
            const uint4 q = reinterpret_cast<const uint4 *>(p)[k];
            memcpy(static_cast<char *>(out) + 16 * k, &q, 16);
        }
    } else if constexpr (B == 8) {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        memcpy(out, &q, 8);
    } else if constexpr (B == 4) {
        const uint32_t q = *reinterpret_cast<const uint32_t *>(p);
        memcpy(out, &q, 4);
    } else {
        static_assert(B == 2, "2 to 64 bytes per lane");
        const uint16_t q = *reinterpret_cast<const uint16_t *>(p);
        memcpy(out, &q, 2);
    }
}

__device__ __forceinline__ int32_t decode_col(uint16_t rel, int32_t base) {
    return rel == 0xFFFFu ? -1 : base + (int32_t)rel;
}
__device__ __forceinline__ int32_t decode_col(int32_t c, int32_t) { return c; }

// Warp w of a CTA takes slices s_begin + w, s_begin + w + nw, ... of the CTA's run; its slice
// j lives in slot j % K.  R rows per lane (S = 32 R rows per slice); U entries per row are
// gathered before they are multiplied.
template <typename T, typename CT, int R, int U>
__global__ void __launch_bounds__(1024, 1)
spmv_sell_bulk(int32_t n, const int64_t *__restrict__ sp, const CT *__restrict__ scol,
               const int32_t *__restrict__ col_start, const T *__restrict__ val,
               const T *__restrict__ x, T *__restrict__ y, const int32_t *__restrict__ part,
               int K, int slot_entries, int *__restrict__ status, int plant) {
    constexpr int S = 32 * R;
    constexpr bool kRel16 = sizeof(CT) == 2;
    extern __shared__ __align__(128) unsigned char smem[];
    const int nw = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem) + warp * kBulkMaxSlots;
    const size_t slot_bytes = (size_t)slot_entries * (sizeof(T) + sizeof(CT));
    unsigned char *ring = smem + kBulkHeader + (size_t)warp * K * slot_bytes;
    const int32_t s_begin = part[blockIdx.x];
    const int32_t s_end = part[blockIdx.x + 1];
    const int m = s_end - s_begin > warp ? (s_end - s_begin - warp + nw - 1) / nw : 0;
    const uint64_t pol = policy_evict_first();

    // lane 0: copy slice j of this warp (entries [sb, se)) into slot j % K.  False (nothing
    // issued) when the slice would not fit its slot, which a consistent handle never has.
    auto issue = [&](int j, int64_t sb, int64_t se) -> bool {
        if (se < sb || se - sb > slot_entries) return false;
        const int slot = j % K;
        const uint32_t fb = smem_addr(full + slot);
        const uint32_t nv = (uint32_t)((se - sb) * (int64_t)sizeof(T));
        const uint32_t nc = (uint32_t)((se - sb) * (int64_t)sizeof(CT));
        unsigned char *dst = ring + slot * slot_bytes;
        mbar_arrive_expect_tx(fb, nv + nc);
        if (nv) {
            bulk_copy(smem_addr(dst), val + sb, nv, fb, pol);
            bulk_copy(smem_addr(dst + (size_t)slot_entries * sizeof(T)), scol + sb, nc, fb, pol);
        }
        return true;
    };
    // lane 0, on the way out: wait for the copies of slices first .. last - 1
    auto drain = [&](int first, int last) {
        for (int i = first; i < last && i < m; ++i) mbar_wait(smem_addr(full + i % K), (i / K) & 1);
    };

    int bad = 0;
    if (lane == 0) {
        for (int i = 0; i < K; ++i) mbar_init(smem_addr(full + i), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int j = 0; j < K && j < m; ++j) {
            const int32_t s = s_begin + warp + j * nw;
            // self-test of the bounded wait: warp 0 of CTA 0 never copies its first slice, so
            // its wait runs out (no copy is left in flight into that slot)
            if (plant && j == 0 && warp == 0 && blockIdx.x == 0) continue;
            if (!issue(j, sp[s], sp[s + 1])) {
                bad = 2;
                drain(0, j);
                break;
            }
        }
    }
    if (__shfl_sync(0xffffffffu, bad, 0)) {
        if (lane == 0) atomicOr(status, bad);
        return;
    }

    for (int j = 0; j < m; ++j) {
        const int slot = j % K;
        const int32_t s = s_begin + warp + j * nw;
        const int64_t sb = __ldg(sp + s);
        const int64_t se = __ldg(sp + s + 1);
        const int32_t cb = kRel16 ? __ldg(col_start + s) : 0;
        // the slice that will reuse this slot, looked up before the wait
        const bool refill = j + K < m;
        int64_t nb = 0, ne = 0;
        if (refill && lane == 0) {
            nb = __ldg(sp + s + K * nw);
            ne = __ldg(sp + s + K * nw + 1);
        }
        // every lane waits; the warp goes on only if all of them saw the copy complete
        const bool ok = mbar_wait(smem_addr(full + slot), (j / K) & 1);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                atomicOr(status, 1);
                drain(j, j + K);  // slices j .. j + K - 1 may still be arriving
            }
            return;
        }
        const int w = (int)((se - sb) / S);
        const T *sv = reinterpret_cast<const T *>(ring + slot * slot_bytes) + lane * R;
        const CT *sc = reinterpret_cast<const CT *>(ring + slot * slot_bytes +
                                                    (size_t)slot_entries * sizeof(T)) +
                       lane * R;
        T acc[R];
#pragma unroll
        for (int i = 0; i < R; ++i) acc[i] = T(0);
        for (int t0 = 0; t0 < w; t0 += U) {
            int32_t c[U][R];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (t0 + u < w) {
                    CT raw[R];
                    lds_bytes<(int)sizeof(CT) * R>(sc + (t0 + u) * S, raw);
#pragma unroll
                    for (int i = 0; i < R; ++i) c[u][i] = decode_col(raw[i], cb);
                } else {
#pragma unroll
                    for (int i = 0; i < R; ++i) c[u][i] = -1;
                }
            }
            T xv[U][R];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int i = 0; i < R; ++i) xv[u][i] = c[u][i] >= 0 ? ld_x(x + c[u][i]) : T(0);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (t0 + u < w) {
                    T v[R];
                    lds_bytes<(int)sizeof(T) * R>(sv + (t0 + u) * S, v);
#pragma unroll
                    for (int i = 0; i < R; ++i)
                        if (c[u][i] >= 0) acc[i] = fma_t(v[i], xv[u][i], acc[i]);
                }
            }
        }
        // every lane has read the slot: lane 0 refills it with the warp's slice j + K (the
        // proxy fence orders those generic reads before the asynchronous copy's writes)
        __syncwarp();
        if (refill && lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (!issue(j + K, nb, ne)) {
                bad = 2;
                drain(j + 1, j + K);
            }
        }
        if (__shfl_sync(0xffffffffu, bad, 0)) {
            if (lane == 0) atomicOr(status, bad);
            return;
        }
        store_rows<T, R>(y, (int64_t)s * S + lane * R, n, acc);
    }
}

// first slice whose entries start at or after CTA b's share of the stored entries
__global__ void bulk_partition_kernel(int32_t n_slices, const int64_t *__restrict__ sp, int G,
                                      int32_t *__restrict__ part) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > G) return;
    if (b == G) {
        part[G] = n_slices;
        return;
    }
    const int64_t total = sp[n_slices];
    const int64_t target = total / G * b + (total % G) * b / G;
    int32_t lo = 0, hi = n_slices;
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (sp[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    part[b] = lo;
}

struct BulkGeometry {
    int warps = 0;         // warps per CTA
    int slots = 0;         // K, slices resident or in flight per warp
    int slot_entries = 0;  // entries of one slot (S times the widest slice)
    size_t smem = 0;       // dynamic shared memory per CTA
};

// The most warps (up to 32) whose rings fit in a CTA's shared memory, with three slots per warp
// when 32 warps fit that way, else two.  False when fewer than four warps fit.
bool bulk_geometry(spmv_matrix_t A, int value_bytes, BulkGeometry *g) {
    const int col_bytes = A->index_bits == 16 ? 2 : 4;
    const size_t budget = (size_t)device_facts().max_smem_optin;
    if (budget <= (size_t)kBulkHeader || A->bulk_G <= 0 || !A->bulk_part.p) return false;
    const int64_t slot_entries = (int64_t)A->S * (A->max_width > 0 ? A->max_width : 1);
    const int64_t slot_bytes = slot_entries * (value_bytes + col_bytes);
    const int64_t room = (int64_t)(budget - kBulkHeader);
    int K = 3;
    int64_t warps = room / (K * slot_bytes);
    if (warps < kBulkMaxWarps) {
        K = 2;
        warps = room / (K * slot_bytes);
    }
    if (warps > kBulkMaxWarps) warps = kBulkMaxWarps;
    if (warps < 4 || slot_entries > INT32_MAX / 8) return false;
    g->warps = (int)warps;
    g->slots = K;
    g->slot_entries = (int)slot_entries;
    g->smem = (size_t)kBulkHeader + (size_t)(warps * K * slot_bytes);
    return true;
}

template <typename T, typename CT, int R, int U>
spmv_status_t go_bulk(spmv_matrix_t A, const CT *scol, const T *val, const T *x, T *y,
                      cudaStream_t st, int plant) {
    BulkGeometry g;
    if (!bulk_geometry(A, (int)sizeof(T), &g)) return SPMV_ERR_UNSUPPORTED;
    auto kernel = spmv_sell_bulk<T, CT, R, U>;
    // largest dynamic shared memory set for this instantiation so far
    static std::atomic<size_t> configured{0};
    if (g.smem > configured.load()) {
        GB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)g.smem));
        configured.store(g.smem);
    }
    kernel<<<A->bulk_G, g.warps * 32, g.smem, st>>>(A->n, A->slice_ptr.p, scol, A->col_start.p,
                                                    val, x, y, A->bulk_part.p, g.slots,
                                                    g.slot_entries, A->dev_status.p, plant);
    GB_LAUNCHED();
    return SPMV_OK;
}

// (R, U) per slice height: U entries of each row are gathered at once (a whole row of the
// tetrahedral meshes, <= 5 entries, for S <= 64); eight FP64 rows per lane leave room for one.
template <typename T, typename CT>
spmv_status_t dispatch_bulk(spmv_matrix_t A, const CT *scol, const T *val, const T *x, T *y,
                            cudaStream_t st, int plant) {
    switch (A->S) {
        case 32: return go_bulk<T, CT, 1, 6>(A, scol, val, x, y, st, plant);
        case 64: return go_bulk<T, CT, 2, 6>(A, scol, val, x, y, st, plant);
        case 128: return go_bulk<T, CT, 4, 3>(A, scol, val, x, y, st, plant);
        case 256: return go_bulk<T, CT, 8, sizeof(T) == 8 ? 1 : 2>(A, scol, val, x, y, st, plant);
    }
    return SPMV_ERR_UNSUPPORTED;
}

template <typename T>
spmv_status_t launch_bulk_t(spmv_matrix_t A, const T *val, const T *x, T *y, cudaStream_t st,
                            bool *launched, int plant = 0) {
    *launched = false;
    if (A->n == 0) {
        *launched = true;
        return SPMV_OK;
    }
    const void *cols =
        A->index_bits == 16 ? (const void *)A->sell_col16.p : (const void *)A->sell_col.p;
    if (((uintptr_t)val & 15u) || ((uintptr_t)cols & 15u) || ((uintptr_t)y & 15u)) return SPMV_OK;
    const spmv_status_t s =
        A->index_bits == 16 ? dispatch_bulk<T, uint16_t>(A, A->sell_col16.p, val, x, y, st, plant)
                            : dispatch_bulk<T, int32_t>(A, A->sell_col.p, val, x, y, st, plant);
    if (s == SPMV_ERR_UNSUPPORTED) return SPMV_OK;  // slices too wide for the rings
    *launched = true;
    return s;
}

}  // namespace

spmv_status_t bulk_partition(spmv_matrix_t A, cudaStream_t st) {
    const int G = device_facts().sm_count;
    A->bulk_G = 0;
    if (G <= 0 || A->n_slices <= 0) return SPMV_OK;
    GB_TRY(A->bulk_part.alloc((size_t)G + 1, &A->bytes));
    bulk_partition_kernel<<<(G + 1 + 255) / 256, 256, 0, st>>>(A->n_slices, A->slice_ptr.p, G,
                                                               A->bulk_part.p);
    GB_LAUNCHED();
    A->bulk_G = G;
    return SPMV_OK;
}

spmv_status_t launch_bulk64(spmv_matrix_t A, const double *x, double *y, cudaStream_t st,
                            bool *launched) {
    return launch_bulk_t<double>(A, A->sell_val.p, x, y, st, launched);
}

spmv_status_t launch_bulk32(spmv_matrix_t A, const float *x, float *y, cudaStream_t st,
                            bool *launched) {
    return launch_bulk_t<float>(A, A->sell_val32.p, x, y, st, launched);
}

// One staged product with the planted missing copy: *recorded = the status bits the kernel
// wrote (bit 0: a wait ran out).  UNSUPPORTED when the handle's slices do not fit the rings.
spmv_status_t bulk_diag_timeout(spmv_matrix_t A, cudaStream_t st, int *recorded) {
    *recorded = 0;
    if (A->n == 0 || A->sell_entries == 0) return SPMV_ERR_INVALID_ARG;
    const bool f64 = A->has64();
    const size_t eb = f64 ? sizeof(double) : sizeof(float);
    void *x = nullptr, *y = nullptr;
    GB_CUDA(gb_malloc_async(&x, eb * (size_t)A->n_cols, st));
    spmv_status_t s = cuda_status(gb_malloc_async(&y, eb * (size_t)A->n, st));
    if (s == SPMV_OK) s = cuda_status(cudaMemsetAsync(x, 0, eb * (size_t)A->n_cols, st));
    if (s == SPMV_OK) s = cuda_status(cudaMemsetAsync(A->dev_status.p, 0, sizeof(int), st));
    bool launched = false;
    if (s == SPMV_OK)
        s = f64 ? launch_bulk_t<double>(A, A->sell_val.p, (const double *)x, (double *)y, st,
                                        &launched, 1)
                : launch_bulk_t<float>(A, A->sell_val32.p, (const float *)x, (float *)y, st,
                                       &launched, 1);
    if (s == SPMV_OK && !launched) s = SPMV_ERR_UNSUPPORTED;
    int v = 0;
    if (s == SPMV_OK)
        s = cuda_status(cudaMemcpyAsync(&v, A->dev_status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (s == SPMV_OK) s = cuda_status(cudaMemsetAsync(A->dev_status.p, 0, sizeof(int), st));
    if (x) cudaFreeAsync(x, st);
    if (y) cudaFreeAsync(y, st);
    if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
    *recorded = v;
    return s;
}

}  // namespace gb
