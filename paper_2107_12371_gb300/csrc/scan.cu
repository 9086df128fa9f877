// scan.cu -- exclusive prefix sums used by the format conversion (slice offsets, row
// pointers, frontier offsets).  Three phases: per-tile sums, a recursive scan of the tile
// sums, then a tile-local scan plus the tile offset.
#include "common.cuh"

namespace gb {
namespace {

constexpr int kThreads = 512;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

// Exclusive scan of one value per thread over the CTA; returns the CTA total in *total.
__device__ int64_t block_exclusive(int64_t v, int64_t *total) {
    __shared__ int64_t warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = (lane < kThreads / 32) ? warp_sums[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kThreads / 32) warp_sums[lane] = wi - w;  // exclusive warp offsets
        if (lane == kThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    int64_t r = warp_sums[warp] + incl - v;
    __syncthreads();
    return r;
}

__global__ void tile_sums(const int64_t *d, int64_t n, int64_t *sums) {
    const int64_t base = (int64_t)blockIdx.x * kTile;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kItems + k;
        if (i < n) s += d[i];
    }
    __shared__ int64_t total;
    block_exclusive(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Tile-local exclusive scan plus offset; offsets == nullptr means offset 0 and the total goes
// to d[n] (single-tile case).
__global__ void tile_scan(int64_t *d, int64_t n, const int64_t *offsets) {
    const int64_t base = (int64_t)blockIdx.x * kTile;
    int64_t v[kItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kItems + k;
        v[k] = (i < n) ? d[i] : 0;
        s += v[k];
    }
    __shared__ int64_t total;
    int64_t run = block_exclusive(s, &total) + (offsets ? offsets[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kItems + k;
        if (i < n) d[i] = run;
        run += v[k];
    }
    if (!offsets && threadIdx.x == 0) d[n] = total;
}

}  // namespace

spmv_status_t exclusive_scan_i64(int64_t *d, int64_t n, cudaStream_t st) {
    if (n <= kTile) {
        tile_scan<<<1, kThreads, 0, st>>>(d, n, nullptr);
        GB_LAUNCHED();
        return SPMV_OK;
    }
    const int64_t nb = (n + kTile - 1) / kTile;
    int64_t *sums = nullptr;
    GB_CUDA(gb_malloc_async((void **)&sums, (size_t)(nb + 1) * sizeof(int64_t), st));
    tile_sums<<<(unsigned)nb, kThreads, 0, st>>>(d, n, sums);
    spmv_status_t s = cuda_status(cudaGetLastError());
    if (s == SPMV_OK) s = exclusive_scan_i64(sums, nb, st);
    if (s == SPMV_OK) {
        tile_scan<<<(unsigned)nb, kThreads, 0, st>>>(d, n, sums);
        s = cuda_status(cudaGetLastError());
    }
    if (s == SPMV_OK)
        s = cuda_status(cudaMemcpyAsync(d + n, sums + nb, sizeof(int64_t),
                                        cudaMemcpyDeviceToDevice, st));
    cudaFreeAsync(sums, st);
    return s;
}

}  // namespace gb
