// verify.cu -- device-side verification of a handle's converted structures (the `checks`
// option), and a self-test that plants one fault at a time in copies of them.
//
// The product kernels stay in bounds and reproduce the CSR row sums only if the conversion
// kept these invariants; each violated one sets a bit of the result:
//   slice pointers start at 0, grow by multiples of S and end at the entry count;
//   every CSR row fits its slice's width, and its columns increase strictly;
//   entry (row, t) of the sliced ELLPACK arrays equals the row's t-th CSR entry (column and
//   value bits) or is padding (column -1, value 0);
//   every column lies in [0, n_cols) and in its slice's [col_start, col_end) (Sec. 5.1);
//   16-bit offsets decode to the columns, 0xFFFF only for padding;
//   the renumbering is a permutation.
#include <climits>
#include <vector>

#include "common.cuh"

namespace gb {
namespace {

constexpr int kVT = 256;

struct SellView {
    int32_t n, n_cols, S, n_slices;
    int64_t total;
    const int64_t *sp;
    const int32_t *rp, *ci;
    const double *val;
    const float *val32;
    const int32_t *scol;
    const uint16_t *scol16;
    const double *sval;
    const float *sval32;
    const int32_t *cs, *ce;
};

__global__ void verify_rows(SellView v, int *err) {
    const int64_t rows = (int64_t)v.n_slices * v.S;
    int bad = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = r / v.S;
        const int lane = (int)(r - s * v.S);
        const int64_t base = v.sp[s], end = v.sp[s + 1];
        if (r == 0 && base != 0) bad |= SPMV_CHECK_SLICE_PTR;
        if (lane == 0 && s == v.n_slices - 1 && end != v.total) bad |= SPMV_CHECK_SLICE_PTR;
        if (base < 0 || end < base || (end - base) % v.S != 0 || end > v.total) {
            bad |= SPMV_CHECK_SLICE_PTR;
            continue;
        }
        const int64_t w = (end - base) / v.S;
        const int32_t a = r < v.n ? v.rp[r] : 0;
        const int32_t len = r < v.n ? v.rp[r + 1] - a : 0;
        if (len > w) {
            bad |= SPMV_CHECK_ROW;
            continue;
        }
        int32_t prev = -1;
        for (int64_t t = 0; t < w; ++t) {
            const int64_t at = base + t * v.S + lane;
            const int32_t c = v.scol[at];
            if (t < len) {
                const int32_t cc = v.ci[a + t];
                if (cc <= prev) bad |= SPMV_CHECK_ROW;
                prev = cc;
                if (c != cc || c < 0 || c >= v.n_cols) bad |= SPMV_CHECK_COLUMN;
                if (v.sval && __double_as_longlong(v.sval[at]) != __double_as_longlong(v.val[a + t]))
                    bad |= SPMV_CHECK_VALUE;
                if (v.sval32 && __float_as_int(v.sval32[at]) != __float_as_int(v.val32[a + t]))
                    bad |= SPMV_CHECK_VALUE;
                if (c < v.cs[s] || c >= v.ce[s]) bad |= SPMV_CHECK_RANGE;
                if (v.scol16) {
                    const uint32_t o = v.scol16[at];
                    if (o == 0xFFFFu || (int64_t)v.cs[s] + (int64_t)o != (int64_t)c)
                        bad |= SPMV_CHECK_REL16;
                }
            } else {
                if (c != -1) bad |= SPMV_CHECK_COLUMN;
                if (v.sval && v.sval[at] != 0.0) bad |= SPMV_CHECK_VALUE;
                if (v.sval32 && v.sval32[at] != 0.0f) bad |= SPMV_CHECK_VALUE;
                if (v.scol16 && v.scol16[at] != 0xFFFFu) bad |= SPMV_CHECK_REL16;
            }
        }
    }
    if (bad) atomicOr(err, bad);
}

__global__ void verify_perm(int32_t n, const int32_t *perm, unsigned *seen, int *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t p = perm[i];
    if (p < 0 || p >= n) {
        atomicOr(err, SPMV_CHECK_PERM);
        return;
    }
    const unsigned bit = 1u << (p & 31);
    if (atomicOr(&seen[p >> 5], bit) & bit) atomicOr(err, SPMV_CHECK_PERM);  // a repeat
}

unsigned blocks_of(int64_t work) {
    int64_t b = (work + kVT - 1) / kVT;
    if (b < 1) b = 1;
    if (b > 65535LL * 64) b = 65535LL * 64;
    return (unsigned)b;
}

SellView view_of(spmv_matrix_t A) {
    SellView v{};
    v.n = A->n;
    v.n_cols = A->n_cols;
    v.S = A->S;
    v.n_slices = A->n_slices;
    v.total = A->sell_entries;
    v.sp = A->slice_ptr.p;
    v.rp = A->row_ptr.p;
    v.ci = A->col.p;
    v.val = A->has64() ? A->val.p : nullptr;
    v.val32 = A->has32() ? A->val32.p : nullptr;
    v.scol = A->sell_col.p;
    v.scol16 = A->index_bits == 16 ? A->sell_col16.p : nullptr;
    v.sval = A->has64() ? A->sell_val.p : nullptr;
    v.sval32 = A->has32() ? A->sell_val32.p : nullptr;
    v.cs = A->col_start.p;
    v.ce = A->col_end.p;
    return v;
}

// Runs the verification kernels on view v (and perm when not null); *flags = violated bits.
spmv_status_t run_verify(const SellView &v, const int32_t *perm, cudaStream_t st, int *flags) {
    *flags = 0;
    if (v.n == 0 && v.n_slices == 0) return SPMV_OK;
    int *d_err = nullptr;
    unsigned *seen = nullptr;
    const size_t words = ((size_t)v.n + 31) / 32;
    spmv_status_t s = cuda_status(gb_malloc_async((void **)&d_err, sizeof(int), st));
    if (s == SPMV_OK && perm) s = cuda_status(gb_malloc_async((void **)&seen, words * 4, st));
    if (s == SPMV_OK) s = cuda_status(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    if (s == SPMV_OK && perm) s = cuda_status(cudaMemsetAsync(seen, 0, words * 4, st));
    if (s == SPMV_OK && v.n_slices > 0) {
        verify_rows<<<blocks_of((int64_t)v.n_slices * v.S), kVT, 0, st>>>(v, d_err);
        s = cuda_status(cudaGetLastError());
    }
    if (s == SPMV_OK && perm && v.n > 0) {
        verify_perm<<<blocks_of(v.n), kVT, 0, st>>>(v.n, perm, seen, d_err);
        s = cuda_status(cudaGetLastError());
    }
    int h = 0;
    if (s == SPMV_OK) s = cuda_status(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (d_err) cudaFreeAsync(d_err, st);
    if (seen) cudaFreeAsync(seen, st);
    spmv_status_t s2 = cuda_status(cudaStreamSynchronize(st));
    if (s == SPMV_OK) s = s2;
    *flags = h;
    return s;
}

// a device copy of `count` elements of src with element `at` replaced by `value`
template <typename T>
spmv_status_t planted_copy(const T *src, size_t count, size_t at, T value, cudaStream_t st,
                           T **out) {
    *out = nullptr;
    GB_CUDA(gb_malloc_async((void **)out, sizeof(T) * (count ? count : 1), st));
    GB_CUDA(cudaMemcpyAsync(*out, src, sizeof(T) * count, cudaMemcpyDeviceToDevice, st));
    GB_CUDA(cudaMemcpyAsync(*out + at, &value, sizeof(T), cudaMemcpyHostToDevice, st));
    return cuda_status(cudaStreamSynchronize(st));  // `value` lives on this stack frame
}

}  // namespace

spmv_status_t verify_matrix(spmv_matrix_t A, cudaStream_t st, int *flags) {
    return run_verify(view_of(A), A->perm.p, st, flags);
}

// Plants each fault the checker must see, one at a time, in a copy of the handle's arrays,
// and reports in *detected one bit per planted fault that the checker flagged.
spmv_status_t checks_self_test(spmv_matrix_t A, cudaStream_t st, int *detected, int *planted) {
    *detected = 0;
    *planted = 0;
    if (A->n < 2 || A->sell_entries == 0) return SPMV_ERR_INVALID_ARG;
    // first stored entry that is not padding
    std::vector<int32_t> scol((size_t)A->sell_entries);
    GB_CUDA(cudaMemcpyAsync(scol.data(), A->sell_col.p, sizeof(int32_t) * scol.size(),
                            cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    size_t at = 0;
    while (at < scol.size() && scol[at] < 0) ++at;
    if (at == scol.size()) return SPMV_ERR_INVALID_ARG;
    const SellView base = view_of(A);
    struct Case {
        int bit;     // bit of *detected
        int expect;  // checker flag that must appear
    };
    auto run_case = [&](const Case &c, const SellView &v, const int32_t *perm) -> spmv_status_t {
        int f = 0;
        GB_TRY(run_verify(v, perm, st, &f));
        *planted |= c.bit;
        if (f & c.expect) *detected |= c.bit;
        return SPMV_OK;
    };
    spmv_status_t s = SPMV_OK;
    // 1. a column out of range
    {
        int32_t *p = nullptr;
        s = planted_copy(A->sell_col.p, scol.size(), at, A->n_cols, st, &p);
        SellView v = base;
        v.scol = p;
        if (s == SPMV_OK) s = run_case({1, SPMV_CHECK_COLUMN}, v, nullptr);
        if (p) cudaFreeAsync(p, st);
    }
    // 2. a value that differs from the CSR's
    if (s == SPMV_OK && A->has64()) {
        double *p = nullptr, h = 0.0;
        s = cuda_status(cudaMemcpyAsync(&h, A->sell_val.p + at, sizeof(double),
                                        cudaMemcpyDeviceToHost, st));
        if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
        if (s == SPMV_OK) s = planted_copy(A->sell_val.p, scol.size(), at, h + 1.0, st, &p);
        SellView v = base;
        v.sval = p;
        if (s == SPMV_OK) s = run_case({2, SPMV_CHECK_VALUE}, v, nullptr);
        if (p) cudaFreeAsync(p, st);
    }
    // 3. a slice pointer off by one entry
    if (s == SPMV_OK && A->n_slices >= 1) {
        int64_t *p = nullptr, h = 0;
        s = cuda_status(cudaMemcpyAsync(&h, A->slice_ptr.p + 1, sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, st));
        if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
        if (s == SPMV_OK)
            s = planted_copy(A->slice_ptr.p, (size_t)A->n_slices + 1, 1, h + 1, st, &p);
        SellView v = base;
        v.sp = p;
        if (s == SPMV_OK) s = run_case({4, SPMV_CHECK_SLICE_PTR}, v, nullptr);
        if (p) cudaFreeAsync(p, st);
    }
    // 4. a 16-bit offset that decodes to another column
    if (s == SPMV_OK && A->index_bits == 16) {
        uint16_t *p = nullptr, h = 0;
        s = cuda_status(cudaMemcpyAsync(&h, A->sell_col16.p + at, sizeof(uint16_t),
                                        cudaMemcpyDeviceToHost, st));
        if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
        if (s == SPMV_OK)
            s = planted_copy(A->sell_col16.p, scol.size(), at, (uint16_t)(h ^ 1u), st, &p);
        SellView v = base;
        v.scol16 = p;
        if (s == SPMV_OK) s = run_case({8, SPMV_CHECK_REL16}, v, nullptr);
        if (p) cudaFreeAsync(p, st);
    }
    // 5. a slice column range that excludes its columns (col_end = col_start)
    if (s == SPMV_OK) {
        std::vector<int64_t> sp((size_t)A->n_slices + 1);
        s = cuda_status(cudaMemcpyAsync(sp.data(), A->slice_ptr.p, sizeof(int64_t) * sp.size(),
                                        cudaMemcpyDeviceToHost, st));
        if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
        int64_t slice = 0;  // the slice holding entry `at`
        while (slice + 1 < (int64_t)sp.size() - 1 && sp[(size_t)slice + 1] <= (int64_t)at) ++slice;
        int32_t h = 0;
        s = cuda_status(cudaMemcpyAsync(&h, A->col_start.p + slice, sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, st));
        if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
        int32_t *p = nullptr;
        if (s == SPMV_OK) s = planted_copy(A->col_end.p, (size_t)A->n_slices, (size_t)slice, h, st, &p);
        SellView v = base;
        v.ce = p;
        if (s == SPMV_OK) s = run_case({16, SPMV_CHECK_RANGE}, v, nullptr);
        if (p) cudaFreeAsync(p, st);
    }
    // 6. a renumbering that repeats a row
    if (s == SPMV_OK && A->perm.p) {
        int32_t h = 0, *p = nullptr;
        s = cuda_status(cudaMemcpyAsync(&h, A->perm.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        if (s == SPMV_OK) s = cuda_status(cudaStreamSynchronize(st));
        if (s == SPMV_OK) s = planted_copy(A->perm.p, (size_t)A->n, 1, h, st, &p);
        if (s == SPMV_OK) s = run_case({32, SPMV_CHECK_PERM}, base, p);
        if (p) cudaFreeAsync(p, st);
    }
    GB_CUDA(cudaStreamSynchronize(st));
    return s;
}

}  // namespace gb
