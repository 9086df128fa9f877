"""GPU parity of the SpMV path against the CPU oracle, through the C ABI.

Bars: integer structures (permutation, permuted CSR, sliced ELLPACK, per-slice ranges) are
bit-exact; FP64 products equal the oracle's fused-multiply-add CSR-order sum bit for bit and
satisfy |y - y_oracle| <= 1e-12 sum_j |a_ij x_j| against the plain multiply-then-add sum;
FP32 products equal the FP32 oracle bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_12371_gb300 import capi, meshgen, workloads

pytestmark = pytest.mark.gpu

GATE = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    capi.load()
    torch.cuda.init()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def absrow(m, x):
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    return np.bincount(rows, weights=np.abs(m.values * x[m.col_idx]), minlength=m.n)


def gpu_spmv(A, x, f32=False, csr=False):
    xd = dev(x)
    yd = torch.empty_like(xd)
    if f32:
        A.apply_f32(xd, yd)
    elif csr:
        A.apply_csr(xd, yd)
    else:
        A.apply(xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def check_fp64(m, x, y, oracle):
    ref_fma = oracle.spmv(m.row_ptr, m.col_idx, m.values, x, use_fma=True)
    ref = oracle.spmv(m.row_ptr, m.col_idx, m.values, x, use_fma=False)
    assert np.array_equal(y, ref_fma), "not bit-identical to the FMA oracle"
    assert np.all(np.abs(y - ref) <= GATE * absrow(m, x))


def ragged_matrix(n, seed, max_len=40, empty_frac=0.1):
    """Random square CSR with ragged rows (some empty, some long) and sorted columns."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len + 1, size=n)
    lens[rng.random(n) < empty_frac] = 0
    lens = np.minimum(lens, n)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    cols = np.concatenate([np.sort(rng.choice(n, size=L, replace=False)) for L in lens]) \
        if lens.sum() else np.zeros(0, np.int64)
    vals = rng.uniform(-1, 1, size=int(rp[-1]))
    return meshgen.CsrMatrix(n, rp.astype(np.int32), cols.astype(np.int32), vals)


@pytest.mark.parametrize("bits", [16, 32])
@pytest.mark.parametrize("S", [32, 64, 128, 256])
def test_c1_fp64_parity(oracle, S, bits):
    m, x = workloads.c1()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, slice_height=S,
                    variant=capi.SPMV_VARIANT_SELL, index_bits=bits)
    assert A.info()["index_bits"] == bits
    check_fp64(m, x, gpu_spmv(A, x), oracle)


def test_wide_slices_fall_back_to_32bit_columns(oracle):
    """16-bit relative columns (Sec. 5.1) only hold slices spanning < 65,535 columns."""
    n = 70000
    rng = np.random.default_rng(9)
    rows = [np.array([0, n - 1])] + [np.sort(rng.choice(n, 3, replace=False)) for _ in range(n - 1)]
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([r.size for r in rows])
    ci = np.concatenate(rows).astype(np.int32)
    m = meshgen.CsrMatrix(n, rp, ci, rng.uniform(-1, 1, ci.size))
    x = rng.uniform(-1, 1, n)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values)
    assert A.info()["index_bits"] == 32
    check_fp64(m, x, gpu_spmv(A, x), oracle)


@pytest.mark.parametrize("span,bits", [(65534, 16), (65535, 32)])
def test_16bit_column_boundary(oracle, span, bits):
    """A slice spanning 65,534 columns still takes 16-bit relative columns (its largest offset,
    65,533, is below the 0xFFFF padding mark); one more column switches the handle to 32-bit.
    The product is exact either way, in FP64 and FP32."""
    n = 70001  # ragged: not a multiple of the slice height
    rng = np.random.default_rng(span)
    rows = [np.array([0, span - 1])]
    for i in range(1, n):
        rows.append(np.unique(np.clip([i - 1, i, i + 1], 0, n - 1)))
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([r.size for r in rows])
    ci = np.concatenate(rows).astype(np.int32)
    m = meshgen.CsrMatrix(n, rp, ci, rng.uniform(-1, 1, ci.size))
    x = rng.uniform(-1, 1, n)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, precision=capi.SPMV_PREC_DUAL,
                    variant=capi.SPMV_VARIANT_SELL)
    assert A.info()["index_bits"] == bits
    assert A.info()["max_slice_span"] == span
    check_fp64(m, x, gpu_spmv(A, x), oracle)
    x32 = x.astype(np.float32)
    ref32 = oracle.spmv_f32(rp, ci, m.values.astype(np.float32), x32, use_fma=True)
    assert np.array_equal(gpu_spmv(A, x32, f32=True), ref32)


@pytest.mark.parametrize("precision", [capi.SPMV_PREC_FP64, capi.SPMV_PREC_FP32])
def test_autotuned_handle_parity(oracle, precision):
    """The autotuner times every (S, CTA size, variant) candidate on the matrix and rebuilds
    the format for the winner; the product is unchanged bit for bit."""
    m, x = workloads.kuhn(24, seed=5, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, autotune=1, precision=precision,
                    reorder=capi.SPMV_REORDER_RCM)
    info = A.info()
    assert info["slice_height"] in (32, 64, 128, 256) and info["block"] in (128, 256, 512)
    assert info["variant"] in (capi.SPMV_VARIANT_SELL, capi.SPMV_VARIANT_CSR,
                               capi.SPMV_VARIANT_SELL_BULK, capi.SPMV_VARIANT_SELL_WINDOW)
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    mi = meshgen.CsrMatrix(m.n, rp, ci, v)
    xi = x[A.permutation()]
    if precision == capi.SPMV_PREC_FP64:
        check_fp64(mi, xi, gpu_spmv(A, xi), oracle)
    else:
        x32 = xi.astype(np.float32)
        ref = oracle.spmv_f32(rp, ci, v.astype(np.float32), x32, use_fma=True)
        assert np.array_equal(gpu_spmv(A, x32, f32=True), ref)
    sp, col, _, cs, ce = capi.spmv_export_sell(A.handle, with_values=False)
    osp, ocol, _ = oracle.sell(rp, ci, v, info["slice_height"])
    assert np.array_equal(sp, osp) and np.array_equal(col, ocol)


@pytest.mark.parametrize("reorder", [capi.SPMV_REORDER_NONE, capi.SPMV_REORDER_RCM])
@pytest.mark.parametrize("bits", [16, 32])
@pytest.mark.parametrize("S", [32, 64, 256])
def test_window_variant_parity(oracle, S, bits, reorder):
    """Sec. 5.1 circular x window in shared memory: bit-identical to the oracle whether the
    rounds fit the window (RCM order) or fall back to global gathers (random order, FP64)."""
    m, x = workloads.c1()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, slice_height=S, index_bits=bits,
                    variant=capi.SPMV_VARIANT_SELL_WINDOW, precision=capi.SPMV_PREC_DUAL,
                    reorder=reorder)
    info = A.info()
    assert info["variant"] == capi.SPMV_VARIANT_SELL_WINDOW and info["window_words"] > 0
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    mi = meshgen.CsrMatrix(m.n, rp, ci, v)
    xi = x[A.permutation()]
    check_fp64(mi, xi, gpu_spmv(A, xi), oracle)
    x32 = xi.astype(np.float32)
    ref = oracle.spmv_f32(rp, ci, v.astype(np.float32), x32, use_fma=True)
    assert np.array_equal(gpu_spmv(A, x32, f32=True), ref)


def test_window_variant_wide_and_ragged(oracle):
    m = ragged_matrix(20000, 11, max_len=60)
    x = np.random.default_rng(12).uniform(-1, 1, m.n)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, variant=capi.SPMV_VARIANT_SELL_WINDOW)
    check_fp64(m, x, gpu_spmv(A, x), oracle)


@pytest.mark.parametrize("reorder", [capi.SPMV_REORDER_NONE, capi.SPMV_REORDER_RCM])
@pytest.mark.parametrize("bits", [16, 32])
@pytest.mark.parametrize("S", [32, 64, 128, 256])
def test_bulk_variant_parity(oracle, S, bits, reorder):
    """Matrix staged in shared memory by bulk asynchronous copies: FP64 and FP32 products
    bit-identical to the oracle (same per-row order as the register-streaming kernel), and no
    bounded wait gave up."""
    m, x = workloads.c1()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, slice_height=S, index_bits=bits,
                    variant=capi.SPMV_VARIANT_SELL_BULK, precision=capi.SPMV_PREC_DUAL,
                    reorder=reorder)
    info = A.info()
    assert info["variant"] == capi.SPMV_VARIANT_SELL_BULK
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    mi = meshgen.CsrMatrix(m.n, rp, ci, v)
    xi = x[A.permutation()]
    check_fp64(mi, xi, gpu_spmv(A, xi), oracle)
    x32 = xi.astype(np.float32)
    ref = oracle.spmv_f32(rp, ci, v.astype(np.float32), x32, use_fma=True)
    assert np.array_equal(gpu_spmv(A, x32, f32=True), ref)
    assert capi.spmv_device_status(A.handle) == capi.SPMV_OK


@pytest.mark.parametrize("n,max_len,S", [(20000, 12, 64), (20000, 60, 32), (3001, 40, 256),
                                         (37, 9, 64), (1, 1, 32)])
def test_bulk_variant_ragged_wide_and_tiny(oracle, n, max_len, S):
    """Ragged rows (empty rows, a ragged last slice, slices of very different widths), slices
    too wide for a stage (the handle falls back to the register-streaming kernel) and matrices
    smaller than one slice or than one CTA per SM."""
    m = ragged_matrix(n, 11 + n, max_len=max_len)
    x = np.random.default_rng(12).uniform(-1, 1, m.n)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, slice_height=S,
                    variant=capi.SPMV_VARIANT_SELL_BULK, precision=capi.SPMV_PREC_DUAL)
    check_fp64(m, x, gpu_spmv(A, x), oracle)
    x32 = x.astype(np.float32)
    ref = oracle.spmv_f32(m.row_ptr, m.col_idx, m.values.astype(np.float32), x32, use_fma=True)
    assert np.array_equal(gpu_spmv(A, x32, f32=True), ref)
    assert capi.spmv_device_status(A.handle) == capi.SPMV_OK


def test_bulk_wait_runs_out_with_a_status(oracle):
    """Failure detection without a GPU fault: in a staged product whose first warp never copies
    its first slice, that warp's bounded wait runs out, is recorded and reported, the rest of the
    product completes, and the handle keeps working."""
    import time
    m, x = workloads.c1()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, variant=capi.SPMV_VARIANT_SELL_BULK,
                    precision=capi.SPMV_PREC_DUAL)
    t0 = time.time()
    assert capi.spmv_diag_bulk_timeout(A.handle) == capi.SPMV_ERR_TIMEOUT
    assert time.time() - t0 < 10.0
    assert capi.spmv_device_status(A.handle) == capi.SPMV_OK  # the record was cleared
    check_fp64(m, x, gpu_spmv(A, x), oracle)
    assert capi.spmv_device_status(A.handle) == capi.SPMV_OK


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (2.5, -0.75), (-1.0, 1.0)])
@pytest.mark.parametrize("S", [32, 64, 128])
def test_axpby_parity(oracle, S, alpha, beta):
    """y = alpha A x + beta y (Sec. 3.2's read-write result vector), bit-identical to the oracle;
    with beta == 0 a NaN-filled y is never read."""
    m, x = workloads.c1()
    y0 = np.random.default_rng(7).uniform(-1, 1, m.n)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, slice_height=S,
                    precision=capi.SPMV_PREC_DUAL)
    yd = dev(y0 if beta != 0 else np.full(m.n, np.nan))
    A.apply_axpby(alpha, dev(x), beta, yd)
    torch.cuda.synchronize()
    ref = oracle.spmv_axpby(m.row_ptr, m.col_idx, m.values, alpha, x, beta, y0)
    assert np.array_equal(yd.cpu().numpy(), ref)
    # FP32 form: finite and within FP32 rounding of the FP64 result
    y32 = dev(y0.astype(np.float32))
    A.apply_axpby(alpha, dev(x.astype(np.float32)), beta, y32)
    torch.cuda.synchronize()
    mag = abs(alpha) * absrow(m, x) + abs(beta) * np.abs(y0)
    assert np.all(np.abs(y32.cpu().numpy() - ref) <= 32 * 2.0 ** -24 * mag + 1e-30)


def test_rectangular_operators_parity(oracle):
    """Rectangular divergence M (cells x faces) and gradient G (faces x cells) of the
    operator-based formulation (Sec. 2): each product bit-identical to the oracle, and the chain
    M (G x) equal to the Laplacian's product within rounding."""
    M, G, L, rng = meshgen.kuhn_tet_operators(12, seed=4)
    x = meshgen.uniform_vectors(rng, L.n)
    Gh = capi.Matrix(G.n, G.row_ptr, G.col_idx, G.values, n_cols=G.n_cols)
    Mh = capi.Matrix(M.n, M.row_ptr, M.col_idx, M.values, n_cols=M.n_cols)
    assert Gh.info()["n_cols"] == L.n and Mh.info()["n_cols"] == G.n
    xd = dev(x)
    gx = torch.empty(G.n, dtype=torch.float64, device="cuda")
    y = torch.empty(M.n, dtype=torch.float64, device="cuda")
    Gh.apply(xd, gx)
    Mh.apply(gx, y)
    torch.cuda.synchronize()
    ref_g = oracle.spmv(G.row_ptr, G.col_idx, G.values, x, use_fma=True)
    assert np.array_equal(gx.cpu().numpy(), ref_g)
    ref_y = oracle.spmv(M.row_ptr, M.col_idx, M.values, ref_g, use_fma=True)
    assert np.array_equal(y.cpu().numpy(), ref_y)
    lx = oracle.spmv(L.row_ptr, L.col_idx, L.values, x)
    scale = np.add.reduceat(np.abs(L.values), L.row_ptr[:-1]) * np.abs(x).max()
    assert np.all(np.abs(y.cpu().numpy() - lx) <= 1e-13 * scale)
    # the chain y = M (G x), every form (the fused kernel that never writes G x, the two
    # products through the handle's temporary, the untuned default, the tuned pick),
    # bit-identical to the two oracle products
    for S in (32, 64, 128, 256):
        for form, tune in ((capi.SPMV_CHAIN_FUSED, 0), (capi.SPMV_CHAIN_TWO, 0),
                           (capi.SPMV_CHAIN_AUTO, 0), (capi.SPMV_CHAIN_AUTO, 1)):
            Ms = capi.Matrix(M.n, M.row_ptr, M.col_idx, M.values, n_cols=M.n_cols,
                             slice_height=S, chain_form=form, autotune=tune)
            for _ in range(2):  # the first call of a tuned handle times both forms
                yc = torch.full_like(y, float("nan"))
                capi.spmv_apply_chain(Ms.handle, Gh.handle, xd, yc)
                torch.cuda.synchronize()
                assert np.array_equal(yc.cpu().numpy(), ref_y), (S, form, tune)
            picked = Ms.info()["chain_form"][0]
            assert picked == (form if form else (picked if tune else capi.SPMV_CHAIN_TWO))
            assert picked in (capi.SPMV_CHAIN_FUSED, capi.SPMV_CHAIN_TWO)
    # the FP32 chain equals the two FP32 products and the FP32 oracle, bit for bit
    G32 = capi.Matrix(G.n, G.row_ptr, G.col_idx, G.values, n_cols=G.n_cols,
                      precision=capi.SPMV_PREC_FP32)
    x32 = x.astype(np.float32)
    ref_g32 = oracle.spmv_f32(G.row_ptr, G.col_idx, G.values.astype(np.float32), x32)
    ref_y32 = oracle.spmv_f32(M.row_ptr, M.col_idx, M.values.astype(np.float32), ref_g32)
    for S in (32, 64, 128, 256):
        for form in (capi.SPMV_CHAIN_FUSED, capi.SPMV_CHAIN_TWO, capi.SPMV_CHAIN_AUTO):
            M32 = capi.Matrix(M.n, M.row_ptr, M.col_idx, M.values, n_cols=M.n_cols,
                              slice_height=S, precision=capi.SPMV_PREC_DUAL, chain_form=form,
                              autotune=int(form == capi.SPMV_CHAIN_AUTO))
            y32 = torch.empty(M.n, dtype=torch.float32, device="cuda")
            capi.spmv_apply_chain_f32(M32.handle, G32.handle, dev(x32), y32)
            torch.cuda.synchronize()
            assert np.array_equal(y32.cpu().numpy(), ref_y32), (S, form)
    with pytest.raises(capi.SpmvError) as e:  # an FP64-only handle has no FP32 values
        capi.spmv_apply_chain_f32(Mh.handle, G32.handle, dev(x32),
                                  torch.empty(M.n, dtype=torch.float32, device="cuda"))
    assert e.value.status == capi.SPMV_ERR_UNSUPPORTED
    # rectangular matrices cannot be renumbered symmetrically, nor solved by CG
    st, h = capi.spmv_create(G.n, G.row_ptr, G.col_idx, G.values, raw_status=True, n_cols=L.n,
                             options=capi.spmv_default_options(reorder=capi.SPMV_REORDER_RCM))
    assert st == capi.SPMV_ERR_INVALID_ARG
    res = Gh.solve(dev(np.ones(G.n)), torch.zeros(G.n, dtype=torch.float64, device="cuda"),
                   raise_on_error=False)
    assert res["status"] == capi.SPMV_ERR_INVALID_ARG


def test_c1_naive_csr_parity(oracle):
    m, x = workloads.c1()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values)
    check_fp64(m, x, gpu_spmv(A, x, csr=True), oracle)


@pytest.mark.parametrize("bits", [16, 32])
@pytest.mark.parametrize("S", [32, 64, 128, 256])
def test_c1_fp32_parity(oracle, S, bits):
    m, x = workloads.c1()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, slice_height=S,
                    precision=capi.SPMV_PREC_DUAL, index_bits=bits)
    x32 = x.astype(np.float32)
    y = gpu_spmv(A, x32, f32=True)
    ref = oracle.spmv_f32(m.row_ptr, m.col_idx, m.values.astype(np.float32), x32, use_fma=True)
    assert np.array_equal(y, ref)
    # error of the FP32 product against the FP64 oracle (reported bound, not a parity gate)
    ref64 = oracle.spmv(m.row_ptr, m.col_idx, m.values, x)
    assert np.all(np.abs(y - ref64) <= 16 * 2.0 ** -24 * absrow(m, x) + 1e-30)
    # the DUAL handle's FP64 product is unchanged
    check_fp64(m, x, gpu_spmv(A, x), oracle)


@pytest.mark.parametrize("n,seed", [(1, 0), (7, 1), (33, 2), (1000, 3), (4097, 4)])
@pytest.mark.parametrize("S", [32, 256])
def test_ragged_and_tiny(oracle, n, seed, S):
    m = ragged_matrix(n, seed)
    x = np.random.default_rng(seed + 100).uniform(-1, 1, n)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, slice_height=S)
    check_fp64(m, x, gpu_spmv(A, x), oracle)
    check_fp64(m, x, gpu_spmv(A, x, csr=True), oracle)


def test_empty_matrix_and_zero_rows(oracle):
    A = capi.Matrix(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert A.info()["n_rows"] == 0
    xd = torch.empty(0, dtype=torch.float64, device="cuda")
    A.apply(xd, torch.empty_like(xd))
    m = meshgen.CsrMatrix(5, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = capi.Matrix(5, m.row_ptr, m.col_idx, m.values)
    y = gpu_spmv(B, np.ones(5))
    assert np.array_equal(y, np.zeros(5))


def test_invalid_csr_is_rejected():
    rp = np.array([0, 2, 3], np.int32)
    for ci in ([1, 0, 1], [0, 5, 1], [0, 0, 1]):  # unsorted, out of range, duplicate
        st, h = capi.spmv_create(2, rp, np.array(ci, np.int32), np.ones(3), raw_status=True)
        assert st == capi.SPMV_ERR_INVALID_CSR and not h
    st, h = capi.spmv_create(2, np.array([0, 3, 2], np.int32), np.array([0, 1, 1], np.int32),
                             np.ones(3), raw_status=True)
    assert st == capi.SPMV_ERR_INVALID_CSR
    st, h = capi.spmv_create(2, np.array([0, 1, 4], np.int32), np.array([0, 1, 1], np.int32),
                             np.ones(3), raw_status=True)
    assert st == capi.SPMV_ERR_INVALID_CSR


def test_device_inputs_match_host_inputs(oracle):
    m, x = workloads.c1()
    A = capi.Matrix(m.n, dev(m.row_ptr), dev(m.col_idx), dev(m.values))
    check_fp64(m, x, gpu_spmv(A, x), oracle)


# ---------------------------------------------------------------------------------------
# reordering and format structures: bit-exact against the oracle
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("peripheral", [0, 1])
@pytest.mark.parametrize("reorder", [capi.SPMV_REORDER_RCM, capi.SPMV_REORDER_CM])
def test_gpu_cm_order_matches_oracle(oracle, reorder, peripheral):
    m, x = workloads.c1()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=reorder, peripheral=peripheral)
    perm = A.permutation()
    ref = oracle.cm_order(m.row_ptr, m.col_idx, reverse=(reorder == capi.SPMV_REORDER_RCM),
                          peripheral=bool(peripheral))
    assert np.array_equal(perm, ref)
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    orp, oci, ov = oracle.permute_csr(m.row_ptr, m.col_idx, m.values, ref)
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci) and np.array_equal(v, ov)
    info = A.info()
    bw = int(np.abs(np.repeat(np.arange(m.n), np.diff(orp)) - oci).max())
    assert info["bandwidth"] == bw


def test_gpu_cm_order_hand_worked_graphs(oracle):
    from test_oracle_pins import _graph_csr, _read_cm_golden
    for g in _read_cm_golden():
        rp, ci = _graph_csr(g["n"], g["edges"])
        for peripheral, expect in g["cm"].items():
            A = capi.Matrix(g["n"], rp, ci, np.ones(ci.size), reorder=capi.SPMV_REORDER_CM,
                            peripheral=peripheral)
            assert list(A.permutation()) == expect


@pytest.mark.parametrize("reorder", [capi.SPMV_REORDER_NONE, capi.SPMV_REORDER_RCM])
@pytest.mark.parametrize("sigma", [64, 1024, 4096])
def test_sigma_sorted_rows_match_oracle(oracle, sigma, reorder):
    """Length sorting inside windows of sigma rows: permutation, permuted CSR and sliced
    ELLPACK bit-exact against the oracle; less padding on the mixed mesh; product unchanged."""
    m, x = workloads.mixed(10, k=None)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=reorder, sigma=sigma)
    base = oracle.cm_order(m.row_ptr, m.col_idx) if reorder else None
    ref = oracle.sigma_sort(m.row_ptr, sigma, perm_in=base)
    assert np.array_equal(A.permutation(), ref)
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    orp, oci, ov = oracle.permute_csr(m.row_ptr, m.col_idx, m.values, ref)
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci) and np.array_equal(v, ov)
    sp, col, val, cs, ce = capi.spmv_export_sell(A.handle)
    osp, ocol, oval = oracle.sell(orp, oci, ov, A.info()["slice_height"])
    assert np.array_equal(sp, osp) and np.array_equal(col, ocol) and np.array_equal(val, oval)
    B = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=reorder)
    # sorting inside one slice (sigma = S) cannot change that slice's width
    if sigma > A.info()["slice_height"]:
        assert A.info()["sell_entries"] < B.info()["sell_entries"]
    else:
        assert A.info()["sell_entries"] == B.info()["sell_entries"]
    xi = x[ref]
    check_fp64(meshgen.CsrMatrix(m.n, rp, ci, v), xi, gpu_spmv(A, xi), oracle)


@pytest.mark.parametrize("S", [32, 64, 128, 256])
def test_sell_and_window_export_match_oracle(oracle, S):
    m, _ = workloads.mixed(6, k=1)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, slice_height=S,
                    reorder=capi.SPMV_REORDER_RCM)
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    sp, col, val, cs, ce = capi.spmv_export_sell(A.handle)
    osp, ocol, oval = oracle.sell(rp, ci, v, S)
    assert np.array_equal(sp, osp) and np.array_equal(col, ocol) and np.array_equal(val, oval)
    ocs, oce = oracle.window_meta(m.n, S, osp, ocol)
    assert np.array_equal(cs, ocs) and np.array_equal(ce, oce)
    assert A.info()["max_slice_span"] == int((oce - ocs).max())


def test_reordered_product_equals_original(oracle):
    """Sec. 4.1: reordering renumbers the unknowns and leaves the coefficients unchanged, so
    P^T (P A P^T)(P x) = A x within the gate (row sums are re-associated by the new order)."""
    m, x = workloads.c1()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=capi.SPMV_REORDER_RCM)
    xd = dev(x)
    xp = torch.empty_like(xd)
    yp = torch.empty_like(xd)
    y = torch.empty_like(xd)
    A.permute(0, xd, xp)
    A.apply(xp, yp)
    A.permute(1, yp, y)
    torch.cuda.synchronize()
    ref = oracle.spmv(m.row_ptr, m.col_idx, m.values, x)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= GATE * absrow(m, x))


# ---------------------------------------------------------------------------------------
# SpMM
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("bits", [16, 32])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_spmm_parity(oracle, k, dtype, bits):
    m, _ = workloads.mixed(8, k=1)
    X = np.random.default_rng(k).uniform(-1, 1, (m.n, k)).astype(dtype)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, precision=capi.SPMV_PREC_DUAL,
                    index_bits=bits)
    Xd = dev(X)
    Yd = torch.empty_like(Xd)
    A.apply_multi(Xd, Yd)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy()
    vals = m.values.astype(dtype)
    ref = oracle.spmm(m.row_ptr, m.col_idx, vals, X, use_fma=True)
    assert np.array_equal(Y, ref)
    # column c of the block product equals the single-vector product
    c = k // 2
    yc = gpu_spmv(A, np.ascontiguousarray(X[:, c]), f32=(dtype == np.float32))
    assert np.array_equal(Y[:, c], yc)


@pytest.mark.parametrize("k", [4, 8, 32])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_spmm_16_byte_aligned_blocks(oracle, k, dtype):
    """X and Y that are 16- but not 32-byte aligned take the 128-bit kernel instead of the
    256-bit one; the product is the same."""
    m, _ = workloads.mixed(8, k=1)
    X = np.random.default_rng(100 + k).uniform(-1, 1, (m.n, k)).astype(dtype)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, precision=capi.SPMV_PREC_DUAL)
    off = 16 // np.dtype(dtype).itemsize
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    xb = torch.zeros(m.n * k + off, dtype=tdt, device="cuda")
    yb = torch.zeros_like(xb)
    Xd = xb[off:].view(m.n, k)
    Yd = yb[off:].view(m.n, k)
    assert Xd.data_ptr() % 32 == 16 and Yd.data_ptr() % 32 == 16
    Xd.copy_(dev(X))
    A.apply_multi(Xd, Yd)
    torch.cuda.synchronize()
    ref = oracle.spmm(m.row_ptr, m.col_idx, m.values.astype(dtype), X, use_fma=True)
    assert np.array_equal(Yd.cpu().numpy(), ref)


@pytest.mark.parametrize("k,dtype", [(8, np.float64), (32, np.float64), (8, np.float32),
                                     (32, np.float32)])
def test_spmm_full_size_parity(oracle, k, dtype):
    """The SpMM workload of the benchmark at full size -- mixed hexahedron / prism /
    tetrahedron mesh of 87^3 hexahedra (about 1.98M cells), RCM and sigma = 1024 sorting, 16-bit
    columns, the 256-bit kernel -- bit-identical to the oracle on every entry."""
    m, X = workloads.mixed(87, seed=1, k=32)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=capi.SPMV_REORDER_RCM,
                    precision=capi.SPMV_PREC_DUAL, sigma=1024)
    assert A.info()["index_bits"] == 16
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    Xi = np.ascontiguousarray(X[A.permutation(), :k]).astype(dtype)
    Xd = dev(Xi)
    Yd = torch.empty_like(Xd)
    assert Xd.data_ptr() % 32 == 0 and Yd.data_ptr() % 32 == 0
    A.apply_multi(Xd, Yd)
    torch.cuda.synchronize()
    ref = oracle.spmm(rp, ci, v.astype(dtype), Xi, use_fma=True)
    assert np.array_equal(Yd.cpu().numpy(), ref)


# ---------------------------------------------------------------------------------------
# products with host vectors (copies pipelined with the product inside the call)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["kuhn_rcm", "kuhn_random", "ragged", "window", "csr",
                                  "rect", "tiny", "pinned"])
def test_apply_host_matches_device(oracle, case):
    opts = {}
    if case in ("kuhn_rcm", "window", "pinned"):
        opts["reorder"] = capi.SPMV_REORDER_RCM
    if case == "window":
        opts["variant"] = capi.SPMV_VARIANT_SELL_WINDOW
    if case == "csr":
        opts["variant"] = capi.SPMV_VARIANT_CSR
    n_cols = None
    if case == "ragged":
        m = ragged_matrix(3001, seed=8)
        opts["slice_height"] = 128
    elif case == "rect":
        _, m, _, _ = meshgen.kuhn_tet_operators(5, seed=1)
        n_cols = m.n_cols
    elif case == "tiny":
        m = ragged_matrix(5, seed=2, max_len=3, empty_frac=0.0)
    else:
        m, _ = workloads.kuhn(10, seed=6, dirichlet=True)
    nc = n_cols if n_cols is not None else m.n
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, n_cols=n_cols, **opts)
    rng = np.random.default_rng(len(case))
    x = rng.uniform(-1, 1, nc)
    if case == "pinned":
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.full((m.n,), np.nan, dtype=torch.float64).pin_memory()
        A.apply_host(xh, yh)
        y_host = yh.numpy()
    else:
        y_host = np.full(m.n, np.nan)
        A.apply_host(x, y_host)
    # the device path on the same handle, and the oracle on the handle's own numbering
    xd = dev(x)
    yd = torch.empty(m.n, dtype=torch.float64, device="cuda")
    A.apply(xd, yd)
    torch.cuda.synchronize()
    assert np.array_equal(y_host, yd.cpu().numpy())
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    ref = oracle.spmv(rp, ci, v, x, use_fma=True)
    assert np.array_equal(y_host, ref)
    # repeated calls reuse the staging and give the same bits
    y2 = np.empty(m.n)
    A.apply_host(x, y2)
    assert np.array_equal(y2, y_host)


@pytest.mark.parametrize("n_streams", [1, 2, 3, 4])
def test_apply_host_async_overlapping_calls(oracle, n_streams):
    """Seven calls enqueued on 1..4 streams in turn (more calls than the three staging sets,
    so sets are reused while earlier calls may still run) each deliver their own product."""
    m, _ = workloads.kuhn(12, seed=9, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=capi.SPMV_REORDER_RCM)
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    rng = np.random.default_rng(3)
    xs = [torch.from_numpy(rng.uniform(-1, 1, m.n)).pin_memory() for _ in range(7)]
    ys = [torch.full((m.n,), np.nan, dtype=torch.float64).pin_memory() for _ in range(7)]
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    for j in range(7):
        A.apply_host_async(xs[j], ys[j], streams[j % n_streams])
    torch.cuda.synchronize()
    for j in range(7):
        ref = oracle.spmv(rp, ci, v, xs[j].numpy(), use_fma=True)
        assert np.array_equal(ys[j].numpy(), ref), j


# ---------------------------------------------------------------------------------------
# structure checks (the device-side substitute for a memory checker)
# ---------------------------------------------------------------------------------------
CHECK_CASES = [
    ("kuhn8", dict()),
    ("kuhn8", dict(reorder=capi.SPMV_REORDER_RCM, precision=capi.SPMV_PREC_DUAL)),
    ("kuhn8", dict(reorder=capi.SPMV_REORDER_RCM, sigma=64, slice_height=32, index_bits=32)),
    ("kuhn8", dict(precision=capi.SPMV_PREC_FP32, slice_height=256)),
    ("kuhn8", dict(variant=capi.SPMV_VARIANT_SELL_WINDOW, reorder=capi.SPMV_REORDER_CM)),
    ("ragged", dict(slice_height=128, precision=capi.SPMV_PREC_DUAL)),
    ("mixed", dict(reorder=capi.SPMV_REORDER_RCM, sigma=1024, precision=capi.SPMV_PREC_DUAL)),
]


def _check_case(name):
    if name == "kuhn8":
        m, _ = workloads.kuhn(8, seed=3, dirichlet=True)
    elif name == "ragged":
        m = ragged_matrix(3001, seed=5)
    else:
        m, _ = workloads.mixed(10, k=1)
    return m


@pytest.mark.parametrize("case", range(len(CHECK_CASES)))
def test_checks_hold_for_every_layout(oracle, case):
    """Handles created with checks = 1 pass the device verification of their structures for
    every slice height, index width, precision, reordering, sigma and variant; the product is
    unchanged."""
    name, opts = CHECK_CASES[case]
    m = _check_case(name)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, checks=1, **opts)
    assert capi.spmv_verify(A.handle) == 0
    B = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, **opts)  # same handle without checks
    x = np.random.default_rng(case).uniform(-1, 1, m.n)
    if opts.get("precision") != capi.SPMV_PREC_FP32:
        assert np.array_equal(gpu_spmv(A, x), gpu_spmv(B, x))


@pytest.mark.parametrize("case", [0, 1, 2, 6])
def test_checks_detect_planted_faults(case):
    """Each fault planted in a copy of the handle's arrays is reported by the checks (the
    self-test covers out-of-range columns, changed values, slice pointers, 16-bit offsets,
    column ranges and repeated rows in a renumbering)."""
    name, opts = CHECK_CASES[case]
    m = _check_case(name)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, **opts)
    planted, detected = capi.spmv_diag_checks(A.handle)
    assert planted == detected
    expect = 1 | 4 | 16
    if opts.get("precision", capi.SPMV_PREC_FP64) != capi.SPMV_PREC_FP32:
        expect |= 2
    if A.info()["index_bits"] == 16:
        expect |= 8
    if opts.get("reorder", 0) != 0:
        expect |= 32
    assert planted == expect
    assert capi.spmv_verify(A.handle) == 0  # the handle itself is untouched


# ---------------------------------------------------------------------------------------
# full size: the 6M-cell Dirichlet mesh in the benchmark's launch configuration
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("reorder,bits,variant", [
    (capi.SPMV_REORDER_NONE, 0, capi.SPMV_VARIANT_AUTO),
    (capi.SPMV_REORDER_RCM, 16, capi.SPMV_VARIANT_AUTO),
    (capi.SPMV_REORDER_RCM, 32, capi.SPMV_VARIANT_AUTO),
    (capi.SPMV_REORDER_RCM, 16, capi.SPMV_VARIANT_SELL_BULK)])
def test_c2_full_size_parity(oracle, reorder, bits, variant):
    m, x = workloads.c2()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=reorder,
                    precision=capi.SPMV_PREC_DUAL, index_bits=bits, variant=variant)
    if bits:
        assert A.info()["index_bits"] == bits
    xd = dev(x)
    xi = torch.empty_like(xd)
    A.permute(0, xd, xi)
    yi = torch.empty_like(xd)
    A.apply(xi, yi)
    torch.cuda.synchronize()
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    # the renumbered matrix P A P^T, built by the oracle from the original CSR with the
    # oracle's own (R)CM order, equals the handle's bit for bit (Sec. 4.1: reordering only
    # renumbers; every coefficient keeps its value)
    if reorder == capi.SPMV_REORDER_RCM:
        ref_perm = oracle.cm_order(m.row_ptr, m.col_idx)
        assert np.array_equal(A.permutation(), ref_perm)
        ro, co, vo = oracle.permute_csr(m.row_ptr, m.col_idx, m.values, ref_perm)
        assert A.info()["bandwidth"] < m.n // 20
    else:
        ref_perm = np.arange(m.n, dtype=np.int32)
        ro, co, vo = m.row_ptr, m.col_idx, m.values
    assert np.array_equal(rp, ro) and np.array_equal(ci, co)
    assert np.array_equal(v.view(np.uint64), np.asarray(vo).view(np.uint64))
    # the product against the oracle's SpMV of the oracle's matrix, x renumbered by the
    # oracle's permutation
    xin = x[ref_perm]
    assert np.array_equal(xi.cpu().numpy(), xin)
    mi = meshgen.CsrMatrix(m.n, ro, co, vo)
    check_fp64(mi, xin, yi.cpu().numpy(), oracle)
    # FP32 product of the same handle against the FP32 oracle
    x32 = xin.astype(np.float32)
    y32 = gpu_spmv(A, x32, f32=True)
    ref32 = oracle.spmv_f32(ro, co, np.asarray(vo).astype(np.float32), x32, use_fma=True)
    assert np.array_equal(y32, ref32)
    assert capi.spmv_device_status(A.handle) == capi.SPMV_OK
