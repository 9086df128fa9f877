// ptx.cuh -- inline-PTX memory access helpers for sm_103a.
//
// The matrix (values + column indices) is read exactly once per product, so it is streamed
// with L1::no_allocate and an L2 evict-first policy: it must not push the multiplying
// vector x out of L2, where x stays resident between gathers (the GPU counterpart of the
// paper's on-chip cache of x, Sec. 5.1).  256-bit loads (v4.b64 / v8.b32) are used where a
// lane reads 32 contiguous bytes.
#pragma once

#include <cstdint>

namespace gb {

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// ---- streamed matrix loads -------------------------------------------------------------
__device__ __forceinline__ void ld_stream(const double *p, uint64_t pol, double (&v)[1]) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;"
        : "=d"(v[0]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const double *p, uint64_t pol, double (&v)[2]) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
        : "=d"(v[0]), "=d"(v[1]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const double *p, uint64_t, double (&v)[4]) {
    uint64_t a, b, c, d;
    asm("ld.global.nc.L1::no_allocate.L2::evict_first.v4.b64 {%0,%1,%2,%3}, [%4];"
        : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
    v[0] = __longlong_as_double((long long)a);
    v[1] = __longlong_as_double((long long)b);
    v[2] = __longlong_as_double((long long)c);
    v[3] = __longlong_as_double((long long)d);
}
__device__ __forceinline__ void ld_stream(const double *p, uint64_t pol, double (&v)[8]) {
    double a[4], b[4];
    ld_stream(p, pol, a);
    ld_stream(p + 4, pol, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[i] = a[i];
        v[4 + i] = b[i];
    }
}

__device__ __forceinline__ void ld_stream(const float *p, uint64_t pol, float (&v)[1]) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
        : "=f"(v[0]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const float *p, uint64_t pol, float (&v)[2]) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
        : "=f"(v[0]), "=f"(v[1]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const float *p, uint64_t pol, float (&v)[4]) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const float *p, uint64_t, float (&v)[8]) {
    uint32_t r[8];
    asm("ld.global.nc.L1::no_allocate.L2::evict_first.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "l"(p));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void ld_stream(const int32_t *p, uint64_t pol, int32_t (&v)[1]) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
        : "=r"(v[0]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const int32_t *p, uint64_t pol, int32_t (&v)[2]) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.s32 {%0,%1}, [%2], %3;"
        : "=r"(v[0]), "=r"(v[1]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const int32_t *p, uint64_t pol, int32_t (&v)[4]) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const int32_t *p, uint64_t, int32_t (&v)[8]) {
    asm("ld.global.nc.L1::no_allocate.L2::evict_first.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7])
        : "l"(p));
}

// ---- streamed 16-bit relative column indices (Sec. 5.1: columns rewritten relative to the
// slice's first column, 2 bytes instead of 4).  0xFFFF marks padding (-1 after decoding).
__device__ __forceinline__ int32_t decode_rel16(uint32_t rel, int32_t base) {
    return rel == 0xFFFFu ? -1 : base + (int32_t)rel;
}
__device__ __forceinline__ void ld_stream_rel16(const uint16_t *p, uint64_t pol, int32_t base,
                                                int32_t (&c)[1]) {
    uint16_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b16 %0, [%1], %2;"
        : "=h"(v) : "l"(p), "l"(pol));
    c[0] = decode_rel16(v, base);
}
__device__ __forceinline__ void ld_stream_rel16(const uint16_t *p, uint64_t pol, int32_t base,
                                                int32_t (&c)[2]) {
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;"
        : "=r"(v) : "l"(p), "l"(pol));
    c[0] = decode_rel16(v & 0xFFFFu, base);
    c[1] = decode_rel16(v >> 16, base);
}
__device__ __forceinline__ void ld_stream_rel16(const uint16_t *p, uint64_t pol, int32_t base,
                                                int32_t (&c)[4]) {
    uint32_t a, b;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.b32 {%0,%1}, [%2], %3;"
        : "=r"(a), "=r"(b) : "l"(p), "l"(pol));
    c[0] = decode_rel16(a & 0xFFFFu, base);
    c[1] = decode_rel16(a >> 16, base);
    c[2] = decode_rel16(b & 0xFFFFu, base);
    c[3] = decode_rel16(b >> 16, base);
}
__device__ __forceinline__ void ld_stream_rel16(const uint16_t *p, uint64_t pol, int32_t base,
                                                int32_t (&c)[8]) {
    uint32_t a, b, d, e;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.b32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(a), "=r"(b), "=r"(d), "=r"(e) : "l"(p), "l"(pol));
    const uint32_t w[4] = {a, b, d, e};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c[2 * k] = decode_rel16(w[k] & 0xFFFFu, base);
        c[2 * k + 1] = decode_rel16(w[k] >> 16, base);
    }
}

// Column indices of a slice: 32-bit absolute, or 16-bit relative to the slice's col_start.
struct Cols32 {
    const int32_t *col;
    template <int R>
    __device__ __forceinline__ void load(int64_t at, int64_t, uint64_t pol, int32_t base,
                                         int32_t (&c)[R]) const {
        (void)base;
        ld_stream(col + at, pol, c);
    }
    __device__ __forceinline__ int32_t base(int64_t) const { return 0; }
};
struct Cols16 {
    const uint16_t *col;
    const int32_t *col_start;
    template <int R>
    __device__ __forceinline__ void load(int64_t at, int64_t, uint64_t pol, int32_t base,
                                         int32_t (&c)[R]) const {
        ld_stream_rel16(col + at, pol, base, c);
    }
    __device__ __forceinline__ int32_t base(int64_t slice) const { return col_start[slice]; }
};

// ---- gathers of the multiplying vector (read-only path, L1 allocating) ----------------
// Only for vectors that no thread writes while the kernel runs.
__device__ __forceinline__ double ld_x(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ld_x(const float *p) { return __ldg(p); }

// Coherent gathers (weak ld.global, L1 allocating) for vectors that other CTAs rewrite during
// the same kernel, between grid barriers whose fences order the writes before these loads
// (the read-only .nc path above would be allowed to return stale data there).
__device__ __forceinline__ double ld_x_coherent(const double *p) {
    double v;
    asm volatile("ld.global.ca.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ float ld_x_coherent(const float *p) {
    float v;
    asm volatile("ld.global.ca.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}

// ---- stores of R consecutive results -----------------------------------------------------
template <typename T, int R>
__device__ __forceinline__ void store_rows(T *y, int64_t row0, int32_t n, const T (&acc)[R]) {
    if (row0 + R <= n) {
        if constexpr (sizeof(T) * R >= 16) {
#pragma unroll
            for (int i = 0; i < R; i += 16 / (int)sizeof(T)) {
                if constexpr (sizeof(T) == 8) {
                    *reinterpret_cast<double2 *>(y + row0 + i) = make_double2(acc[i], acc[i + 1]);
                } else {
                    *reinterpret_cast<float4 *>(y + row0 + i) =
                        make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
                }
            }
        } else if constexpr (sizeof(T) * R == 8 && sizeof(T) == 4) {
            *reinterpret_cast<float2 *>(y + row0) = make_float2(acc[0], acc[1]);
        } else {
#pragma unroll
            for (int i = 0; i < R; ++i) y[row0 + i] = acc[i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (row0 + i < n) y[row0 + i] = acc[i];
    }
}

__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

}  // namespace gb
