"""Every candidate the tuners can pick gives a product or solve that passes the oracle's bar,
and a tuned handle reports its picks (spmv_get_info) and stays on that bar.

Tuned shapes: the multi-vector product's kernel form (bit-identical to the oracle's FMA-order
SpMM for every form), the CG product's grid and entries in flight (iteration counts within 2
of the oracle's, true residual, persistent == graph path bit for bit), and the multi-RHS CG
product's gather width (per-column iterations within 2 of the oracle's, true residual).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_12371_gb300 import capi, meshgen, workloads

pytestmark = pytest.mark.gpu

FORMS = [capi.SPMV_SPMM_WIDE, capi.SPMV_SPMM_WIDE_PIPE, capi.SPMV_SPMM_WIDE_GS4,
         capi.SPMV_SPMM_WIDE_GS6, capi.SPMV_SPMM_UNROLLED]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    capi.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _spmm(A, X):
    Xd = dev(X)
    Yd = torch.empty_like(Xd)
    assert Xd.data_ptr() % 32 == 0 and Yd.data_ptr() % 32 == 0
    A.apply_multi(Xd, Yd)
    torch.cuda.synchronize()
    return Yd.cpu().numpy()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("bits,S,reorder", [(16, 64, capi.SPMV_REORDER_RCM),
                                            (32, 32, capi.SPMV_REORDER_NONE),
                                            (16, 128, capi.SPMV_REORDER_RCM)])
def test_every_spmm_form_is_bit_exact(oracle, form, bits, S, reorder):
    """Each form on a 20^3 mixed mesh (several thousand slices, rows of 4..13 entries), k =
    4, 8, 16, 32 FP64 and 8, 16, 32, 64 FP32 (one to eight lanes per row)."""
    m, _ = workloads.mixed(20, k=1)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=reorder, index_bits=bits,
                    slice_height=S, precision=capi.SPMV_PREC_DUAL, spmm_form=form)
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    for dtype, ks in ((np.float64, (4, 8, 16, 32)), (np.float32, (8, 16, 32, 64))):
        for k in ks:
            X = np.random.default_rng(k).uniform(-1, 1, (m.n, k)).astype(dtype)
            ref = oracle.spmm(rp, ci, v.astype(dtype), X, use_fma=True)
            assert np.array_equal(_spmm(A, X), ref), (dtype, k)
    info = A.info()
    assert info["spmm_form"] == [[form] * 4, [form] * 4]


@pytest.mark.parametrize("form", FORMS)
def test_every_spmm_form_on_every_slice_width(oracle, form):
    """Slices of every width from 0 (all rows empty) to 13: slice s of 64 rows holds rows of s
    entries (distinct seeded columns), no reordering and no sorting, so the width-unrolled form
    runs each of its unrolled bodies (1..10), its empty case and its loop for 11..13; a ragged
    last slice of 20 rows.  k = 8 and 32, FP64 and FP32."""
    rng = np.random.default_rng(7)
    widths = [s for s in range(14) for _ in range(64)] + [5] * 20
    n = len(widths)
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum(widths)
    ci = np.concatenate([np.sort(rng.choice(n, w, replace=False)) for w in widths]).astype(np.int32)
    v = rng.uniform(-1, 1, ci.size)
    A = capi.Matrix(n, rp, ci, v, reorder=capi.SPMV_REORDER_NONE, precision=capi.SPMV_PREC_DUAL,
                    slice_height=64, spmm_form=form)
    for dtype in (np.float64, np.float32):
        for k in (8, 32):
            X = rng.uniform(-1, 1, (n, k)).astype(dtype)
            ref = oracle.spmm(rp, ci, v.astype(dtype), X, use_fma=True)
            assert np.array_equal(_spmm(A, X), ref), (dtype, k)


def test_tuned_spmm_reports_its_pick_and_is_bit_exact(oracle):
    m, _ = workloads.mixed(30, k=1)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=capi.SPMV_REORDER_RCM,
                    precision=capi.SPMV_PREC_DUAL, autotune=1)
    rp, ci, v = capi.spmv_export_csr(A.handle, m.n, m.nnz)
    for dtype, k, p, g in ((np.float64, 32, 0, 3), (np.float32, 32, 1, 2),
                           (np.float32, 8, 1, 0)):
        X = np.random.default_rng(k).uniform(-1, 1, (m.n, k)).astype(dtype)
        ref = oracle.spmm(rp, ci, v.astype(dtype), X, use_fma=True)
        assert np.array_equal(_spmm(A, X), ref)  # the first call tunes
        assert A.info()["spmm_form"][p][g] in FORMS
        assert np.array_equal(_spmm(A, X), ref)  # later calls use the pick


def _solve(A, b, **opts):
    bd = dev(b)
    xd = torch.zeros_like(bd)
    res = A.solve(bd, xd, raise_on_error=False, **opts)
    torch.cuda.synchronize()
    return xd.cpu().numpy(), res


@pytest.mark.parametrize("ctas", [2, 3, 4])
@pytest.mark.parametrize("unroll", [2, 5])
def test_every_cg_product_grid_matches_oracle(oracle, ctas, unroll):
    m, b = workloads.kuhn(16, seed=5, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, precision=capi.SPMV_PREC_DUAL,
                    pq_ctas=ctas, pq_unroll=unroll)
    assert A.info()["pq_ctas"] == ctas and A.info()["pq_unroll"] == unroll
    x, res = _solve(A, b, rtol=1e-10)
    assert res["status"] == capi.SPMV_OK
    _, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, b, rtol=1e-10)
    assert abs(res["iterations"] - info["iterations"]) <= 2
    r = b - oracle.spmv(m.row_ptr, m.col_idx, m.values, x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    x2, res2 = _solve(A, b, rtol=1e-10, persistent=1)
    assert res2["iterations"] == res["iterations"] and np.array_equal(x, x2)
    for pers in (0, 1):
        xm, rm = _solve(A, b, rtol=1e-10, mixed=1, persistent=pers)
        assert rm["status"] == capi.SPMV_OK
        r = b - oracle.spmv(m.row_ptr, m.col_idx, m.values, xm)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)


def test_tuned_cg_reports_its_pick(oracle):
    m, b = workloads.kuhn(24, seed=6, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=capi.SPMV_REORDER_RCM,
                    autotune=1)
    perm = A.permutation()
    xi, res = _solve(A, b[perm], rtol=1e-10)
    info = A.info()
    assert info["pq_ctas"] in (2, 3, 4) and info["pq_unroll"] in (2, 5)
    assert res["status"] == capi.SPMV_OK
    x = np.empty_like(xi)
    x[perm] = xi
    _, ref = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, b, rtol=1e-10)
    assert abs(res["iterations"] - ref["iterations"]) <= 2
    r = b - oracle.spmv(m.row_ptr, m.col_idx, m.values, x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    x2, res2 = _solve(A, b[perm], rtol=1e-10, persistent=1)
    assert np.array_equal(xi, x2)


@pytest.mark.parametrize("gather", [16, 32, 0])
@pytest.mark.parametrize("k", [8, 32])
def test_every_multi_cg_gather_width_matches_oracle(oracle, gather, k):
    """gather = 0 with autotune: the tuner's pick."""
    m, rng = meshgen.mixed_matrix(14, seed=1, dirichlet=True)
    B = meshgen.uniform_vectors(rng, m.n, k)
    opts = dict(gather_bytes=gather) if gather else dict(autotune=1)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=capi.SPMV_REORDER_RCM,
                    precision=capi.SPMV_PREC_DUAL, **opts)
    perm = A.permutation()
    Bd = dev(B[perm])
    Xd = torch.zeros_like(Bd)
    st, cols = A.solve_multi(Bd, Xd, rtol=1e-10)
    torch.cuda.synchronize()
    assert st == capi.SPMV_OK
    assert A.info()["gather_bytes"] == (gather or A.info()["gather_bytes"])
    assert A.info()["gather_bytes"] in (16, 32)
    X = np.empty_like(B)
    X[perm] = Xd.cpu().numpy()
    for c in range(k):
        _, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, B[:, c], rtol=1e-10)
        assert abs(cols[c]["iterations"] - info["iterations"]) <= 2
        r = B[:, c] - oracle.spmv(m.row_ptr, m.col_idx, m.values, X[:, c])
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(B[:, c])
    # the persistent kernel agrees bit for bit at the same width
    X2 = torch.zeros_like(Bd)
    A.solve_multi(Bd, X2, rtol=1e-10, persistent=1)
    torch.cuda.synchronize()
    assert torch.equal(X2, Xd)
