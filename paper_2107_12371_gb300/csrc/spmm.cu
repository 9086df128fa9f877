// spmm.cu -- multi-right-hand-side products Y = A X (not in the paper).
//
// spmm_sell<T, G, C>: X and Y row-major (n x k), G lanes per row, each lane C columns;
// every gathered row of X (k contiguous values) is read once per matrix entry and used for
// all k columns.  Column c of Y equals the single-vector product of column c bit for bit
// (same entry order, fused multiply-add from +0.0).
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "ptx.cuh"

namespace gb {
namespace {

inline unsigned grid_for(int64_t threads, int block) {
    int64_t b = (threads + block - 1) / block;
    return (unsigned)(b < 1 ? 1 : b);
}

// SpMM: G lanes per row (G divides 32, so the RPW = 32 / G rows of a warp lie in one slice and
// share its width), lane g owns columns g, g + G, ... (C of them).  The lanes of a row first
// load G of its (value, column) pairs at once, one per lane; the pairs are then broadcast
// inside the row's lane group by shuffles, four at a time, so each lane issues 4 C gathers of
// X back to back instead of one dependent load-then-gather round per entry.
template <typename T, int G, int C, typename ColT>
__global__ void __launch_bounds__(256)
spmm_sell(int32_t n, int32_t S, int32_t n_slices, int k, const int64_t *__restrict__ sp,
          ColT cols, const T *__restrict__ val, const T *__restrict__ X, T *__restrict__ Y) {
    constexpr int RPW = 32 / G;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, g = lane % G;
    const int64_t rows_total = (int64_t)n_slices * S;
    const int64_t row0 = gw * RPW;
    if (row0 >= rows_total) return;  // whole warp: rows_total is a multiple of RPW
    const int64_t row = row0 + sub;
    const int64_t slice = row0 / S;
    const int64_t r = row - slice * S;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cbase = cols.base(slice);
    const uint64_t pol = policy_evict_first();
    T acc[C];
#pragma unroll
    for (int j = 0; j < C; ++j) acc[j] = T(0);
    for (int t0 = 0; t0 < w; t0 += G) {
        T a_l = T(0);
        int32_t c_l = -1;
        if (t0 + g < w) {
            T a1[1];
            int32_t c1[1];
            ld_stream(val + base + (int64_t)(t0 + g) * S + r, pol, a1);
            cols.template load<1>(base + (int64_t)(t0 + g) * S + r, slice, pol, cbase, c1);
            a_l = a1[0];
            c_l = c1[0];
        }
        const int cnt = (w - t0) < G ? (w - t0) : G;
        int tt = 0;
        for (; tt + 4 <= cnt; tt += 4) {
            T a[4], xv[4][C];
            int32_t c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = __shfl_sync(0xffffffffu, a_l, tt + u, G);
                c[u] = __shfl_sync(0xffffffffu, c_l, tt + u, G);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const int cc = g + j * G;
                    xv[u][j] = (c[u] >= 0 && cc < k) ? ld_x(X + (int64_t)c[u] * k + cc) : T(0);
                }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < C; ++j)
                    if (c[u] >= 0) acc[j] = fma_t(a[u], xv[u][j], acc[j]);
        }
        for (; tt < cnt; ++tt) {
            const T a = __shfl_sync(0xffffffffu, a_l, tt, G);
            const int32_t c = __shfl_sync(0xffffffffu, c_l, tt, G);
            if (c < 0) continue;
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const int cc = g + j * G;
                if (cc < k) acc[j] = fma_t(a, ld_x(X + (int64_t)c * k + cc), acc[j]);
            }
        }
    }
    if (row < n) {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const int cc = g + j * G;
            if (cc < k) Y[row * k + cc] = acc[j];
        }
    }
}

// Vectorised SpMM for k = VW * G: lane g of a row's G lanes owns the VW consecutive columns
// g VW .. g VW + VW - 1 and gathers them with one VW-wide load (8 or 16 bytes).  Each lane
// preloads PE / G of its row's (value, column) pairs, so PE = 16 pairs are fetched in one
// round; they are broadcast by shuffles four at a time.
template <typename T, int VW>
struct VecOf;
template <>
struct VecOf<double, 2> {
    static __device__ __forceinline__ void load(const double *p, double (&v)[2]) {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        v[0] = t.x;
        v[1] = t.y;
    }
    static __device__ __forceinline__ void store(double *p, const double (&v)[2]) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
};
template <>
struct VecOf<float, 4> {
    static __device__ __forceinline__ void load(const float *p, float (&v)[4]) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
    static __device__ __forceinline__ void store(float *p, const float (&v)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};

template <typename T, int VW, int G, typename ColT>
__global__ void __launch_bounds__(256)
spmm_sell_vec(int32_t n, int32_t S, int32_t n_slices, const int64_t *__restrict__ sp, ColT cols,
              const T *__restrict__ val, const T *__restrict__ X, T *__restrict__ Y) {
    constexpr int K = VW * G;
    constexpr int RPW = 32 / G;
    constexpr int PE = 16;                      // pairs preloaded per round
    constexpr int PL = PE / G > 0 ? PE / G : 1;  // pairs per lane per round
    constexpr int PR = PL * G;                  // pairs per round
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, g = lane % G;
    const int64_t rows_total = (int64_t)n_slices * S;
    const int64_t row0 = gw * RPW;
    if (row0 >= rows_total) return;  // whole warp: rows_total is a multiple of RPW
    const int64_t row = row0 + sub;
    const int64_t slice = row0 / S;
    const int64_t r = row - slice * S;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cbase = cols.base(slice);
    const uint64_t pol = policy_evict_first();
    T acc[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) acc[j] = T(0);
    for (int t0 = 0; t0 < w; t0 += PR) {
        T a_l[PL];
        int32_t c_l[PL];
#pragma unroll
        for (int q = 0; q < PL; ++q) {
            const int t = t0 + q * G + g;
            a_l[q] = T(0);
            c_l[q] = -1;
            if (t < w) {
                T a1[1];
                int32_t c1[1];
                ld_stream(val + base + (int64_t)t * S + r, pol, a1);
                cols.template load<1>(base + (int64_t)t * S + r, slice, pol, cbase, c1);
                a_l[q] = a1[0];
                c_l[q] = c1[0];
            }
        }
        const int cnt = (w - t0) < PR ? (w - t0) : PR;
#pragma unroll
        for (int e0 = 0; e0 < PR; e0 += 4) {
            if (e0 >= cnt) break;
            T a[4], xv[4][VW];
            int32_t c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u;  // pair e lives in lane e % G, slot e / G
                a[u] = __shfl_sync(0xffffffffu, a_l[(e / G) % PL], e % G, G);
                c[u] = __shfl_sync(0xffffffffu, c_l[(e / G) % PL], e % G, G);
                if (e >= cnt) c[u] = -1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (c[u] >= 0) VecOf<T, VW>::load(X + (int64_t)c[u] * K + g * VW, xv[u]);
                else {
#pragma unroll
                    for (int j = 0; j < VW; ++j) xv[u][j] = T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < VW; ++j)
                    if (c[u] >= 0) acc[j] = fma_t(a[u], xv[u][j], acc[j]);
        }
    }
    if (row < n) VecOf<T, VW>::store(Y + row * K + g * VW, acc);
}

// 32-byte gathers and stores of X / Y rows (256-bit accesses, sm_100 and later).
template <typename T>
struct Wide;
template <>
struct Wide<float> {
    static constexpr int n = 8;
    static __device__ __forceinline__ void load(const float *p, float (&v)[8]) {
        asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
              "=f"(v[7])
            : "l"(p));
    }
    static __device__ __forceinline__ void store(float *p, const float (&v)[8]) {
        asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]),
                     "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                     : "memory");
    }
};
template <>
struct Wide<double> {
    static constexpr int n = 4;
    static __device__ __forceinline__ void load(const double *p, double (&v)[4]) {
        asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
            : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
            : "l"(p));
    }
    static __device__ __forceinline__ void store(double *p, const double (&v)[4]) {
        asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]),
                     "d"(v[2]), "d"(v[3])
                     : "memory");
    }
};

// SpMM for k = G * (32 bytes / sizeof(T)) with 32-byte aligned X and Y: lane g of a row's G
// lanes owns 32 consecutive bytes of the row and gathers them with one 256-bit load.  Every
// lane reads its row's (value, column) pairs itself (the G lanes of a row read the same
// address, served by one transaction), two entries per step so that two gathers are in
// flight, with no shuffles.  Same entry order and fused multiply-add from +0.0 as the other
// SpMM kernels, so the results are identical.  FP32 products are bound by the latency of the
// gathers and run at six CTAs per SM (40 registers; a few bytes spill), FP64 ones by the FP64
// pipe at four.
template <typename T, int G, typename ColT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 4)
spmm_sell_wide(int32_t n, int32_t S, int32_t n_slices, const int64_t *__restrict__ sp,
               ColT cols, const T *__restrict__ val, const T *__restrict__ X, T *__restrict__ Y) {
    constexpr int VW = Wide<T>::n;
    constexpr int K = VW * G;
    constexpr int RPW = 32 / G;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, g = lane % G;
    const int64_t rows_total = (int64_t)n_slices * S;
    const int64_t row0 = gw * RPW;
    if (row0 >= rows_total) return;  // whole warp: rows_total is a multiple of RPW
    const int64_t row = row0 + sub;
    const int64_t slice = row0 / S;
    const int64_t r = row - slice * S;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cbase = cols.base(slice);
    const uint64_t pol = policy_evict_first();
    const T *vp = val + base + r;
    const int64_t cat = base + r;
    const T *xg = X + g * VW;
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
        for (int u = 0; u < 2; ++u) {
            if (c[u][0] >= 0) Wide<T>::load(xg + (int64_t)c[u][0] * K, xv[u]);
        }
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
            Wide<T>::load(xg + (int64_t)c[0] * K, xv);
#pragma unroll
            for (int j = 0; j < VW; ++j) acc[j] = fma_t(a[0], xv[j], acc[j]);
        }
    }
    if (row < n) Wide<T>::store(Y + row * K + g * VW, acc);
}

// The same product software-pipelined: the (value, column) pairs of a row's next two entries
// are loaded while the current two entries' X rows are gathered, at four CTAs per SM (48-64
// registers).  Measured on the 87^3 mixed mesh: FP32 k = 8 (one lane per row) 73.7 -> 65.4 us;
// no gain at k = 32 FP32 (213 us either way) and slower for FP64, which keep spmm_sell_wide.
template <typename T, int G, typename ColT>
__global__ void __launch_bounds__(256, 4)
spmm_sell_wide_pipe(int32_t n, int32_t S, int32_t n_slices, const int64_t *__restrict__ sp,
                    ColT cols, const T *__restrict__ val, const T *__restrict__ X,
                    T *__restrict__ Y) {
    constexpr int VW = Wide<T>::n;
    constexpr int K = VW * G;
    constexpr int RPW = 32 / G;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, g = lane % G;
    const int64_t rows_total = (int64_t)n_slices * S;
    const int64_t row0 = gw * RPW;
    if (row0 >= rows_total) return;  // whole warp: rows_total is a multiple of RPW
    const int64_t row = row0 + sub;
    const int64_t slice = row0 / S;
    const int64_t r = row - slice * S;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cbase = cols.base(slice);
    const uint64_t pol = policy_evict_first();
    const T *vp = val + base + r;
    const int64_t cat = base + r;
    const T *xg = X + g * VW;
    T acc[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) acc[j] = T(0);
    // entries t and t + 1 of the row (column -1 past the slice width: nothing gathered)
    auto load_pair = [&](int t, T (&a)[2], int32_t (&c)[2]) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (t + u < w) {
                T av[1];
                int32_t cv[1];
                ld_stream(vp + (int64_t)(t + u) * S, pol, av);
                cols.template load<1>(cat + (int64_t)(t + u) * S, slice, pol, cbase, cv);
                a[u] = av[0];
                c[u] = cv[0];
            } else {
                a[u] = T(0);
                c[u] = -1;
            }
        }
    };
    T a[2];
    int32_t c[2];
    load_pair(0, a, c);
    for (int t = 0; t < w; t += 2) {
        T an[2];
        int32_t cn[2];
        load_pair(t + 2, an, cn);
        T xv[2][VW];
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (c[u] >= 0) Wide<T>::load(xg + (int64_t)c[u] * K, xv[u]);
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (c[u] >= 0) {
#pragma unroll
                for (int j = 0; j < VW; ++j) acc[j] = fma_t(a[u], xv[u][j], acc[j]);
            }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            a[u] = an[u];
            c[u] = cn[u];
        }
    }
    if (row < n) Wide<T>::store(Y + row * K + g * VW, acc);
}

// The rows of one warp (RPW = 32 / G rows from row0, inside one slice) of the 256-bit SpMM:
// the body of spmm_sell_wide, two entries per step.
template <typename T, int G, typename ColT>
__device__ __forceinline__ void wide_warp_rows(int64_t row0, int32_t n, int32_t S,
                                               const int64_t *__restrict__ sp, ColT cols,
                                               const T *__restrict__ val,
                                               const T *__restrict__ X, T *__restrict__ Y,
                                               uint64_t pol) {
    constexpr int VW = Wide<T>::n;
    constexpr int K = VW * G;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, g = lane % G;
    const int64_t row = row0 + sub;
    const int64_t slice = row0 / S;
    const int64_t r = row - slice * S;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cbase = cols.base(slice);
    const T *vp = val + base + r;
    const int64_t cat = base + r;
    const T *xg = X + g * VW;
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
        for (int u = 0; u < 2; ++u) {
            if (c[u][0] >= 0) Wide<T>::load(xg + (int64_t)c[u][0] * K, xv[u]);
        }
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
            Wide<T>::load(xg + (int64_t)c[0] * K, xv);
#pragma unroll
            for (int j = 0; j < VW; ++j) acc[j] = fma_t(a[0], xv[j], acc[j]);
        }
    }
    if (row < n) Wide<T>::store(Y + row * K + g * VW, acc);
}

// L2 prefetch of the matrix data (values and column indices) of the slices holding rows
// [rlo, rhi): one 128-byte line per lane of the calling warp.
template <typename T, typename ColT>
__device__ __forceinline__ void prefetch_rows_l2(int64_t rlo, int64_t rhi, int32_t S,
                                                 const int64_t *sp, ColT cols, const T *val) {
    const int lane = threadIdx.x & 31;
    const int64_t e0 = sp[rlo / S], e1 = sp[(rhi + S - 1) / S];
    const uintptr_t v0 = (uintptr_t)(val + e0) & ~(uintptr_t)127;
    const uintptr_t v1 = (uintptr_t)(val + e1);
    for (uintptr_t p = v0 + 128 * (uintptr_t)lane; p < v1; p += 128 * 32)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    const uintptr_t c0 = (uintptr_t)(cols.col + e0) & ~(uintptr_t)127;
    const uintptr_t c1 = (uintptr_t)(cols.col + e1);
    for (uintptr_t p = c0 + 128 * (uintptr_t)lane; p < c1; p += 128 * 32)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The 256-bit SpMM as a grid-stride loop over blocks of 8 RPW rows (one per CTA step) on a
// grid of MINB CTAs per SM, warp 0 prefetching into L2 the matrix data of the block the CTA
// takes next, so that the (value, column) loads of the next block hit L2 instead of waiting on
// DRAM before their gathers can start.  Same per-row order, hence the same bits.
template <typename T, int G, int MINB, typename ColT>
__global__ void __launch_bounds__(256, MINB)
spmm_sell_wide_gs(int32_t n, int32_t S, int32_t n_slices, const int64_t *__restrict__ sp,
                  ColT cols, const T *__restrict__ val, const T *__restrict__ X,
                  T *__restrict__ Y) {
    constexpr int RPW = 32 / G;
    constexpr int64_t RB = 8 * RPW;
    const int warp = threadIdx.x >> 5;
    const int64_t rows_total = (int64_t)n_slices * S;
    const int64_t nblocks = (rows_total + RB - 1) / RB;
    const uint64_t pol = policy_evict_first();
    for (int64_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
        const int64_t nxt = blk + gridDim.x;
        if (warp == 0 && nxt < nblocks)
            prefetch_rows_l2(nxt * RB, nxt * RB + RB < rows_total ? nxt * RB + RB : rows_total,
                             S, sp, cols, val);
        const int64_t row0 = blk * RB + (int64_t)warp * RPW;
        if (row0 < rows_total) wide_warp_rows<T, G>(row0, n, S, sp, cols, val, X, Y, pol);
    }
}

// The rows of one warp of the 256-bit SpMM with the slice width W known at compile time: the W
// (value, column) pairs of the lane's row are requested together, then the X rows gathered two
// at a time and multiplied in entry order.  With a runtime width the compiler keeps each pair's
// matrix loads behind the previous pair's gathers; unrolled, the matrix loads of the whole row
// are in flight at once and a row costs one dependent matrix round instead of one per pair.
template <typename T, int G, int W, typename ColT>
__device__ __forceinline__ void wide_row_w(int64_t at, int32_t S, ColT cols, int32_t cb,
                                           const T *__restrict__ val, const T *__restrict__ xg,
                                           uint64_t pol, T (&acc)[Wide<T>::n]) {
    constexpr int VW = Wide<T>::n;
    constexpr int K = VW * G;
    T a[W];
    int32_t c[W];
#pragma unroll
    for (int t = 0; t < W; ++t) {
        T a1[1];
        int32_t c1[1];
        ld_stream(val + at + (int64_t)t * S, pol, a1);
        cols.template load<1>(at + (int64_t)t * S, 0, pol, cb, c1);
        a[t] = a1[0];
        c[t] = c1[0];
    }
#pragma unroll
    for (int t = 0; t < W; t += 2) {
        T xv[2][VW];
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (t + u < W && c[t + u] >= 0) Wide<T>::load(xg + (int64_t)c[t + u] * K, xv[u]);
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (t + u < W && c[t + u] >= 0) {
#pragma unroll
                for (int j = 0; j < VW; ++j) acc[j] = fma_t(a[t + u], xv[u][j], acc[j]);
            }
    }
}

// The 256-bit SpMM with each slice's width dispatched to a fully unrolled row body for widths
// up to WMAX (wider slices: the two-entries-per-step loop of spmm_sell_wide), MINB CTAs per SM.
// Measured on the 87^3 mixed mesh (us, k = 8 / 32): FP32 59 / 170 against 64 / 207 for the best
// earlier form, FP64 174 / 651 against 178 / 664, at six CTAs per SM and WMAX = 10.  Same
// entry order and fused multiply-add from +0.0 as the other SpMM kernels, so the results are
// identical.
template <typename T, int G, int MINB, int WMAX, typename ColT>
__global__ void __launch_bounds__(256, MINB)
spmm_sell_unrolled(int32_t n, int32_t S, int32_t n_slices, const int64_t *__restrict__ sp,
                   ColT cols, const T *__restrict__ val, const T *__restrict__ X,
                   T *__restrict__ Y) {
    constexpr int VW = Wide<T>::n;
    constexpr int K = VW * G;
    constexpr int RPW = 32 / G;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, g = lane % G;
    const int64_t rows_total = (int64_t)n_slices * S;
    const int64_t row0 = gw * RPW;
    if (row0 >= rows_total) return;  // whole warp: rows_total is a multiple of RPW
    const int64_t row = row0 + sub;
    const int64_t slice = row0 / S;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cb = cols.base(slice);
    const uint64_t pol = policy_evict_first();
    const int64_t at = base + (row - slice * S);
    const T *xg = X + g * VW;
    T acc[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) acc[j] = T(0);
    switch (w) {
        case 0: break;
        case 1: wide_row_w<T, G, 1>(at, S, cols, cb, val, xg, pol, acc); break;
        case 2: wide_row_w<T, G, 2>(at, S, cols, cb, val, xg, pol, acc); break;
        case 3: wide_row_w<T, G, 3>(at, S, cols, cb, val, xg, pol, acc); break;
        case 4: wide_row_w<T, G, 4>(at, S, cols, cb, val, xg, pol, acc); break;
        case 5: wide_row_w<T, G, 5>(at, S, cols, cb, val, xg, pol, acc); break;
        case 6: wide_row_w<T, G, 6>(at, S, cols, cb, val, xg, pol, acc); break;
        case 7:
            if constexpr (WMAX >= 7) {
                wide_row_w<T, G, 7>(at, S, cols, cb, val, xg, pol, acc);
                break;
            }
            [[fallthrough]];
        case 8:
            if constexpr (WMAX >= 8) {
                wide_row_w<T, G, 8>(at, S, cols, cb, val, xg, pol, acc);
                break;
            }
            [[fallthrough]];
        case 9:
            if constexpr (WMAX >= 9) {
                wide_row_w<T, G, 9>(at, S, cols, cb, val, xg, pol, acc);
                break;
            }
            [[fallthrough]];
        case 10:
            if constexpr (WMAX >= 10) {
                wide_row_w<T, G, 10>(at, S, cols, cb, val, xg, pol, acc);
                break;
            }
            [[fallthrough]];
        default: {
            int t = 0;
            for (; t + 2 <= w; t += 2) {
                T a[2][1];
                int32_t c[2][1];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    ld_stream(val + at + (int64_t)(t + u) * S, pol, a[u]);
                    cols.template load<1>(at + (int64_t)(t + u) * S, 0, pol, cb, c[u]);
                }
                T xv[2][VW];
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    if (c[u][0] >= 0) Wide<T>::load(xg + (int64_t)c[u][0] * K, xv[u]);
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
                ld_stream(val + at + (int64_t)t * S, pol, a);
                cols.template load<1>(at + (int64_t)t * S, 0, pol, cb, c);
                if (c[0] >= 0) {
                    T xv[VW];
                    Wide<T>::load(xg + (int64_t)c[0] * K, xv);
#pragma unroll
                    for (int j = 0; j < VW; ++j) acc[j] = fma_t(a[0], xv[j], acc[j]);
                }
            }
        }
    }
    if (row < n) Wide<T>::store(Y + row * K + g * VW, acc);
}

}  // namespace

// Kernel form of the 256-bit SpMM for a handle, precision and lanes-per-row class: the
// handle's choice (option or tuner), else the measured default, the width-unrolled form
// (fastest of the forms for k = 8 and 32 in both precisions on the mixed-element mesh).
int spmm_form_of(const spmv_matrix_t A, bool f32, int gi) {
    if (A->opt.spmm_form != SPMV_SPMM_AUTO) return A->opt.spmm_form;
    const int t = A->spmm_tuned[f32 ? 1 : 0][gi];
    if (t != SPMV_SPMM_AUTO) return t;
    return SPMV_SPMM_UNROLLED;
}

namespace {

template <typename T>
spmv_status_t launch_spmm(spmv_matrix_t A, int k, const T *val, const T *X, T *Y,
                          cudaStream_t st) {
    if (A->n == 0) return SPMV_OK;
    const int block = 256;
    const int64_t rows_total = (int64_t)A->n_slices * A->S;
    // 256-bit kernel when k is a power-of-two multiple of 32 bytes and X, Y allow it
    constexpr int WV = Wide<T>::n;
    const bool al32 = ((uintptr_t)X % 32 == 0) && ((uintptr_t)Y % 32 == 0);
    auto wide = [&](auto gtag) -> spmv_status_t {
        constexpr int G = decltype(gtag)::value;
        constexpr int gi = G == 1 ? 0 : (G == 2 ? 1 : (G == 4 ? 2 : 3));
        const int64_t warps = (rows_total + (32 / G) - 1) / (32 / G);
        const unsigned grid = grid_for(warps * 32, block);
        const int sms = device_facts().sm_count;
        const int form = spmm_form_of(A, sizeof(T) == 4, gi);
        auto go = [&](auto cols) -> spmv_status_t {
            using ColT = decltype(cols);
            switch (form) {
                case SPMV_SPMM_WIDE_PIPE:
                    spmm_sell_wide_pipe<T, G, ColT><<<grid, block, 0, st>>>(
                        A->n, A->S, A->n_slices, A->slice_ptr.p, cols, val, X, Y);
                    break;
                case SPMV_SPMM_WIDE_GS4:
                    spmm_sell_wide_gs<T, G, 4, ColT><<<sms * 4, block, 0, st>>>(
                        A->n, A->S, A->n_slices, A->slice_ptr.p, cols, val, X, Y);
                    break;
                case SPMV_SPMM_WIDE_GS6:
                    spmm_sell_wide_gs<T, G, 6, ColT><<<sms * 6, block, 0, st>>>(
                        A->n, A->S, A->n_slices, A->slice_ptr.p, cols, val, X, Y);
                    break;
                case SPMV_SPMM_UNROLLED:
                    spmm_sell_unrolled<T, G, 6, 10, ColT><<<grid, block, 0, st>>>(
                        A->n, A->S, A->n_slices, A->slice_ptr.p, cols, val, X, Y);
                    break;
                default:
                    spmm_sell_wide<T, G, ColT><<<grid, block, 0, st>>>(
                        A->n, A->S, A->n_slices, A->slice_ptr.p, cols, val, X, Y);
            }
            GB_LAUNCHED();
            return SPMV_OK;
        };
        if (A->index_bits == 16) return go(Cols16{A->sell_col16.p, A->col_start.p});
        return go(Cols32{A->sell_col.p});
    };
    if (al32) {
        using std::integral_constant;
        if (k == WV * 1) return wide(integral_constant<int, 1>{});
        if (k == WV * 2) return wide(integral_constant<int, 2>{});
        if (k == WV * 4) return wide(integral_constant<int, 4>{});
        if (k == WV * 8) return wide(integral_constant<int, 8>{});
    }
    // vectorised kernel when k is a power of two with k >= 16 / sizeof(T), k <= 64
    constexpr int VW = sizeof(T) == 8 ? 2 : 4;
    auto vec = [&](auto gtag) -> spmv_status_t {
        constexpr int G = decltype(gtag)::value;
        const int64_t warps = (rows_total + (32 / G) - 1) / (32 / G);
        const unsigned grid = grid_for(warps * 32, block);
        if (A->index_bits == 16)
            spmm_sell_vec<T, VW, G, Cols16><<<grid, block, 0, st>>>(
                A->n, A->S, A->n_slices, A->slice_ptr.p, Cols16{A->sell_col16.p, A->col_start.p},
                val, X, Y);
        else
            spmm_sell_vec<T, VW, G, Cols32><<<grid, block, 0, st>>>(
                A->n, A->S, A->n_slices, A->slice_ptr.p, Cols32{A->sell_col.p}, val, X, Y);
        GB_LAUNCHED();
        return SPMV_OK;
    };
    using std::integral_constant;
    if (k == VW * 1) return vec(integral_constant<int, 1>{});
    if (k == VW * 2) return vec(integral_constant<int, 2>{});
    if (k == VW * 4) return vec(integral_constant<int, 4>{});
    if (k == VW * 8) return vec(integral_constant<int, 8>{});
    if (k == VW * 16) return vec(integral_constant<int, 16>{});
    if (k == VW * 32 && VW * 32 <= 64) return vec(integral_constant<int, 32>{});
    auto go = [&](auto gtag, auto ctag) -> spmv_status_t {
        constexpr int G = decltype(gtag)::value;
        constexpr int C = decltype(ctag)::value;
        const int64_t warps = (rows_total + (32 / G) - 1) / (32 / G);
        const unsigned grid = grid_for(warps * 32, block);
        if (A->index_bits == 16)
            spmm_sell<T, G, C, Cols16><<<grid, block, 0, st>>>(
                A->n, A->S, A->n_slices, k, A->slice_ptr.p, Cols16{A->sell_col16.p, A->col_start.p},
                val, X, Y);
        else
            spmm_sell<T, G, C, Cols32><<<grid, block, 0, st>>>(
                A->n, A->S, A->n_slices, k, A->slice_ptr.p, Cols32{A->sell_col.p}, val, X, Y);
        GB_LAUNCHED();
        return SPMV_OK;
    };
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I4 = std::integral_constant<int, 4>;
    using I8 = std::integral_constant<int, 8>;
    using I16 = std::integral_constant<int, 16>;
    using I32 = std::integral_constant<int, 32>;
    if (k <= 1) return go(I1{}, I1{});
    if (k <= 2) return go(I2{}, I1{});
    if (k <= 4) return go(I4{}, I1{});
    if (k <= 8) return go(I8{}, I1{});
    if (k <= 16) return go(I16{}, I1{});
    if (k <= 32) return go(I32{}, I1{});
    return go(I32{}, I2{});
}

// Tuner of the 256-bit SpMM's form for this (precision, k): each form in turn computes the
// caller's product (warm-up launch, then the median of three launches, each after writing a
// buffer of twice the L2 size so that the matrix and X come from DRAM as in steady use); the
// fastest is kept for the handle.  The product left in Y is the last form's, and every form
// gives the same bits.
template <typename T>
spmv_status_t tune_spmm(spmv_matrix_t A, int k, const T *val, const T *X, T *Y,
                        cudaStream_t st) {
    constexpr int WV = Wide<T>::n;
    const bool al32 = ((uintptr_t)X % 32 == 0) && ((uintptr_t)Y % 32 == 0);
    int gi = -1;
    for (int g = 0, G = 1; g < 4; ++g, G *= 2)
        if (k == WV * G) gi = g;
    if (!al32 || gi < 0 || A->n == 0) return SPMV_OK;
    int &slot = A->spmm_tuned[sizeof(T) == 4 ? 1 : 0][gi];
    if (slot != SPMV_SPMM_AUTO) return SPMV_OK;
    const size_t fb = 2 * (size_t)(device_facts().l2_bytes > 0 ? device_facts().l2_bytes
                                                               : (128 << 20));
    void *flush = nullptr;
    GB_CUDA(gb_malloc_async(&flush, fb, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    spmv_status_t s = cuda_status(cudaEventCreate(&e0));
    if (s == SPMV_OK) s = cuda_status(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_form = SPMV_SPMM_WIDE;
    for (int form = SPMV_SPMM_WIDE; form <= SPMV_SPMM_UNROLLED && s == SPMV_OK; ++form) {
        slot = form;
        s = launch_spmm<T>(A, k, val, X, Y, st);
        float t[3];
        for (int i = 0; i < 3 && s == SPMV_OK; ++i) {
            s = cuda_status(cudaMemsetAsync(flush, i + 1, fb, st));
            if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e0, st));
            if (s == SPMV_OK) s = launch_spmm<T>(A, k, val, X, Y, st);
            if (s == SPMV_OK) s = cuda_status(cudaEventRecord(e1, st));
            if (s == SPMV_OK) s = cuda_status(cudaEventSynchronize(e1));
            if (s == SPMV_OK) s = cuda_status(cudaEventElapsedTime(&t[i], e0, e1));
        }
        if (s != SPMV_OK) break;
        const float med = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
        if (med < best) {
            best = med;
            best_form = form;
        }
    }
    slot = s == SPMV_OK ? best_form : SPMV_SPMM_AUTO;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(flush, st);
    return s;
}

}  // namespace

spmv_status_t tune_spmm64(spmv_matrix_t A, int k, const double *X, double *Y, cudaStream_t st) {
    return tune_spmm<double>(A, k, A->sell_val.p, X, Y, st);
}

spmv_status_t tune_spmm32(spmv_matrix_t A, int k, const float *X, float *Y, cudaStream_t st) {
    return tune_spmm<float>(A, k, A->sell_val32.p, X, Y, st);
}

spmv_status_t launch_spmm64(spmv_matrix_t A, int k, const double *X, double *Y, cudaStream_t st) {
    return launch_spmm<double>(A, k, A->sell_val.p, X, Y, st);
}

spmv_status_t launch_spmm32(spmv_matrix_t A, int k, const float *X, float *Y, cudaStream_t st) {
    return launch_spmm<float>(A, k, A->sell_val32.p, X, Y, st);
}

}  // namespace gb
