// cgkern.cuh -- device building blocks shared by the CG kernels (graph-launched and
// persistent): deterministic reductions, the product rows of one slice, shape dispatch.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "ptx.cuh"

namespace gb {

constexpr int kCgBlock = 256;
constexpr int kCgCtasPerSm = 4;  // at most this many CTAs per SM in a CG sweep

int cg_grid(int32_t n);

// The product phase q = A p, p.q runs on a grid of its own: the sweeps' grid (at most
// kCgCtasPerSm CTAs per SM) leaves the latency-bound gathers without enough warps in flight.
// A lane holding at most 16 bytes of values per entry keeps pq_unroll = 5 entries in flight
// (a whole row of the tetrahedral meshes) at four CTAs per SM and 64 registers -- measured on
// the 6M-row mesh against two entries at six CTAs per SM (40 registers): FP64 CG 185 -> 176 us
// per iteration, the FP32 refinement solve 4.7 % faster; wider lanes keep two entries at
// pq_min_ctas CTAs per SM, and so do matrices whose widest slice needs fewer load rounds
// that way (load_rounds).  The persistent kernel runs the same grid as virtual CTAs, so
// both paths stay bit-identical.
constexpr int pq_min_ctas(int value_bytes) { return value_bytes >= 64 ? 3 : 4; }
constexpr int pq_unroll(int value_bytes) { return value_bytes <= 16 ? 5 : 2; }
int cg_pq_grid(const spmv_matrix_t A, int L, int value_bytes);
bool cg_pq_deep(const spmv_matrix_t A, int uu);

// Hint: bring the line holding p into L1 without waiting for it (a later load of it hits).
__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// prefetch of a slice's column base (16-bit relative columns only)
__device__ __forceinline__ void prefetch_col_base(const Cols32 &, int64_t) {}
__device__ __forceinline__ void prefetch_col_base(const Cols16 &c, int64_t slice) {
    prefetch_l1(c.col_start + slice);
}

// Sum over the CTA in a fixed tree; the total is left in every lane of warp 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][kCgBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < kCgBlock / 32 ? sh[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            v[k] = t;
        }
    }
}

// Same sum, broadcast to every thread of the CTA.
template <int NV>
__device__ __forceinline__ void block_sum_all(double (&v)[NV]) {
    __shared__ double bc[NV];
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) bc[k] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = bc[k];
    __syncthreads();
}

// Each CTA stores its partial sums in part[k * gridDim.x + cta]; the CTA that arrives last
// (atomic ticket) sums all partials in a fixed order.  Returns true in that CTA, with the
// grid totals in tot[] (valid in thread 0); the ticket is reset for the next launch.
template <int NV>
__device__ bool grid_sum_last(double (&v)[NV], double *part, unsigned *ticket, double (&tot)[NV]) {
    __shared__ bool last;
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        s[k] = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += kCgBlock)
            s[k] += __ldcg(part + k * gridDim.x + i);
    }
    block_sum<NV>(s);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = s[k];
        *ticket = 0u;
    }
    return true;
}

// y-rows (R of them) of lane `lane` in slice `slice`: sum over the slice's columns in order,
// fused multiply-add from +0.0, padding skipped (the same order as spmv_sell).  COHERENT
// selects coherent gathers of x, for kernels in which other CTAs rewrite x between barriers.
template <typename T, int R, int L, bool COHERENT = false, int UU = 2, typename ColT>
__device__ __forceinline__ void slice_rows(int64_t slice, int lane, const int64_t *sp,
                                           const ColT &cols, const T *val, const T *x,
                                           uint64_t pol, T (&acc)[R]) {
    constexpr int S = L * R;
    const int64_t base = sp[slice];
    const int w = (int)((sp[slice + 1] - base) / S);
    const int32_t cbase = cols.base(slice);
    const T *vp = val + base + lane * R;
    const int64_t cat = base + lane * R;
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = T(0);
    int t = 0;
    for (; t + UU <= w; t += UU) {
        T v[UU][R];
        int32_t c[UU][R];
#pragma unroll
        for (int u = 0; u < UU; ++u) {
            ld_stream(vp + (int64_t)(t + u) * S, pol, v[u]);
            cols.template load<R>(cat + (int64_t)(t + u) * S, slice, pol, cbase, c[u]);
        }
        T xv[UU][R];
#pragma unroll
        for (int u = 0; u < UU; ++u)
#pragma unroll
            for (int i = 0; i < R; ++i)
                xv[u][i] = c[u][i] >= 0 ? (COHERENT ? ld_x_coherent(x + c[u][i]) : ld_x(x + c[u][i]))
                                        : T(0);
#pragma unroll
        for (int u = 0; u < UU; ++u)
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (c[u][i] >= 0) acc[i] = fma_t(v[u][i], xv[u][i], acc[i]);
    }
    for (; t < w; ++t) {
        T v[R];
        int32_t c[R];
        ld_stream(vp + (int64_t)t * S, pol, v);
        cols.template load<R>(cat + (int64_t)t * S, slice, pol, cbase, c);
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (c[i] >= 0)
                acc[i] = fma_t(v[i], COHERENT ? ld_x_coherent(x + c[i]) : ld_x(x + c[i]), acc[i]);
    }
}

// ---- vector sweeps of one CG iteration (grid-stride, 16-byte vectors, scalar tail) --------
// Shared by the graph-launched kernels and the persistent kernel, so both produce the same
// per-thread partial sums.  Vectors are plain (coherent) loads: inside the persistent kernel
// they are rewritten between grid barriers.
template <typename T>
struct Vec16;
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
};
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
};

template <typename T>
__device__ __forceinline__ void vload(const T *p, T (&v)[Vec16<T>::n]) {
    const typename Vec16<T>::type t = *reinterpret_cast<const typename Vec16<T>::type *>(p);
    if constexpr (Vec16<T>::n == 2) {
        v[0] = t.x;
        v[1] = t.y;
    } else {
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
}

template <typename T>
__device__ __forceinline__ void vstore(T *p, const T (&v)[Vec16<T>::n]) {
    typename Vec16<T>::type t;
    if constexpr (Vec16<T>::n == 2) {
        t.x = v[0];
        t.y = v[1];
    } else {
        t.x = v[0];
        t.y = v[1];
        t.z = v[2];
        t.w = v[3];
    }
    *reinterpret_cast<typename Vec16<T>::type *>(p) = t;
}

// 16-byte loads and stores marked evict-first in L2 (and not kept in L1), for the vectors an
// FP32 sweep is the last to touch in its iteration, so that the ones the next kernel reads
// stay in L2: measured on the 6M-row mesh, the FP32 refinement solve 99 -> 94 ms.  The FP64
// sweeps, co-bound by the FP64 pipe, measured slower with the hints (FP64 CG 194 -> 206 ms)
// and keep plain loads and stores.  vload_h / vstore_h pick the form by element type.
__device__ __forceinline__ void vload_ef(const float *p, float (&v)[4], uint64_t pol) {
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "l"(p), "l"(pol));
}
__device__ __forceinline__ void vstore_ef(float *p, const float (&v)[4], uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "f"(v[0]),
                 "f"(v[1]), "f"(v[2]), "f"(v[3]), "l"(pol)
                 : "memory");
}

template <typename T>
__device__ __forceinline__ void vload_h(const T *p, T (&v)[Vec16<T>::n], uint64_t pol) {
    if constexpr (sizeof(T) == 4) vload_ef(p, v, pol);
    else vload(p, v);
}
template <typename T>
__device__ __forceinline__ void vstore_h(T *p, const T (&v)[Vec16<T>::n], uint64_t pol) {
    if constexpr (sizeof(T) == 4) vstore_ef(p, v, pol);
    else vstore(p, v);
}

// x += alpha p; r -= alpha q; accumulates r.(D^-1 r) into vz and r.r into vr.  x and q are
// not needed again in this iteration (evict-first in FP32); r, p and D^-1 are read by the p
// update.
template <typename T>
__device__ __forceinline__ void sweep_update_xr(int32_t n, T alpha, T *x, T *r, const T *p,
                                                const T *q, const T *dinv, T &vz, T &vr) {
    constexpr int V = Vec16<T>::n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nv = n / V;
    const uint64_t pol = policy_evict_first();
    for (int64_t v = tid; v < nv; v += stride) {
        const int64_t i = v * V;
        T xv[V], rv[V], pv[V], qv[V], dv[V];
        vload_h(x + i, xv, pol);
        vload(r + i, rv);
        vload(p + i, pv);
        vload_h(q + i, qv, pol);
        vload(dinv + i, dv);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            xv[e] = fma_t(alpha, pv[e], xv[e]);
            rv[e] = fma_t(-alpha, qv[e], rv[e]);
            vz = fma_t(rv[e], dv[e] * rv[e], vz);
            vr = fma_t(rv[e], rv[e], vr);
        }
        vstore_h(x + i, xv, pol);
        vstore(r + i, rv);
    }
    for (int64_t i = nv * V + tid; i < n; i += stride) {
        const T xi = fma_t(alpha, p[i], x[i]);
        const T ri = fma_t(-alpha, q[i], r[i]);
        x[i] = xi;
        r[i] = ri;
        vz = fma_t(ri, dinv[i] * ri, vz);
        vr = fma_t(ri, ri, vr);
    }
}

// p = D^-1 r + beta p.  r and D^-1 are next read by the next iteration's x/r update
// (evict-first in FP32); the new p stays in L2 for the product's gathers.
template <typename T>
__device__ __forceinline__ void sweep_update_p(int32_t n, T beta, const T *r, const T *dinv,
                                               T *p) {
    constexpr int V = Vec16<T>::n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nv = n / V;
    const uint64_t pol = policy_evict_first();
    for (int64_t v = tid; v < nv; v += stride) {
        const int64_t i = v * V;
        T rv[V], dv[V], pv[V];
        vload_h(r + i, rv, pol);
        vload_h(dinv + i, dv, pol);
        vload(p + i, pv);
#pragma unroll
        for (int e = 0; e < V; ++e) pv[e] = fma_t(beta, pv[e], dv[e] * rv[e]);
        vstore(p + i, pv);
    }
    for (int64_t i = nv * V + tid; i < n; i += stride) p[i] = fma_t(beta, p[i], dinv[i] * r[i]);
}

// (R, L) of the sliced kernels for a slice height and value type.
template <typename F>
spmv_status_t with_shape(int S, bool f32, F &&f) {
    using std::integral_constant;
    if (!f32) {
        switch (S) {
            case 32: return f(integral_constant<int, 1>{}, integral_constant<int, 32>{});
            case 64: return f(integral_constant<int, 2>{}, integral_constant<int, 32>{});
            case 128: return f(integral_constant<int, 4>{}, integral_constant<int, 32>{});
            case 256: return f(integral_constant<int, 8>{}, integral_constant<int, 32>{});
        }
    } else {
        switch (S) {
            case 32: return f(integral_constant<int, 4>{}, integral_constant<int, 8>{});
            case 64: return f(integral_constant<int, 4>{}, integral_constant<int, 16>{});
            case 128: return f(integral_constant<int, 4>{}, integral_constant<int, 32>{});
            case 256: return f(integral_constant<int, 8>{}, integral_constant<int, 32>{});
        }
    }
    return SPMV_ERR_INVALID_ARG;
}

}  // namespace gb
