"""GPU CG solves (FP64 Jacobi-PCG, graph-launched and persistent; FP32/FP64 iterative
refinement) through the C ABI, checked against the CPU oracle.

Bars: the true FP64 residual ||b - A x|| / ||b|| recomputed by the oracle SpMV meets the
requested tolerance; FP64 iteration counts agree with the oracle's within 2; the persistent
kernel reproduces the graph-launched path bit for bit; statuses for caps, timeouts and bad
inputs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_12371_gb300 import capi, meshgen, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    capi.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def true_relres(oracle, m, x, b):
    r = b - oracle.spmv(m.row_ptr, m.col_idx, m.values, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


def solve(A, b, **opts):
    bd = dev(b)
    xd = torch.zeros_like(bd)
    res = A.solve(bd, xd, raise_on_error=False, **opts)
    torch.cuda.synchronize()
    return xd.cpu().numpy(), res


@pytest.mark.parametrize("n", [3, 8, 14, 30])
def test_fp64_pcg_matches_oracle(oracle, n):
    """n = 30: 162,000 rows, several hundred iterations, the product's grid at many CTAs."""
    m, b = workloads.kuhn(n, seed=n, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values)
    x, res = solve(A, b, rtol=1e-10)
    assert res["status"] == capi.SPMV_OK
    xo, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, b, rtol=1e-10)
    assert abs(res["iterations"] - info["iterations"]) <= 2
    assert true_relres(oracle, m, x, b) <= 1e-10
    assert abs(res["rel_residual"] - true_relres(oracle, m, x, b)) <= 1e-12
    assert np.linalg.norm(x - xo) <= 1e-7 * np.linalg.norm(xo)


@pytest.mark.parametrize("bits", [16, 32])
def test_persistent_equals_graph_path(oracle, bits):
    m, b = workloads.kuhn(12, seed=4, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, index_bits=bits)
    x1, r1 = solve(A, b, rtol=1e-10)
    x2, r2 = solve(A, b, rtol=1e-10, persistent=1)
    assert r1["status"] == r2["status"] == capi.SPMV_OK
    assert r1["iterations"] == r2["iterations"]
    assert np.array_equal(x1, x2)
    # repeated solves are deterministic
    x3, r3 = solve(A, b, rtol=1e-10)
    assert np.array_equal(x1, x3)
    # the FP32 inner solves of the refinement, persistent vs graph-launched
    D = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, index_bits=bits,
                    precision=capi.SPMV_PREC_DUAL)
    x4, r4 = solve(D, b, rtol=1e-10, mixed=1)
    x5, r5 = solve(D, b, rtol=1e-10, mixed=1, persistent=1)
    assert r4["status"] == r5["status"] == capi.SPMV_OK
    assert (r4["iterations"], r4["outer_iterations"]) == (r5["iterations"], r5["outer_iterations"])
    assert np.array_equal(x4, x5)


def tridiag(n):
    """SPD 1-D Laplacian with a mildly varying diagonal (ragged sizes, one row per slice lane)."""
    rows, cols, vals = [], [], []
    for i in range(n):
        if i > 0:
            rows.append(i); cols.append(i - 1); vals.append(-1.0)
        rows.append(i); cols.append(i); vals.append(2.0 + 0.01 * (i % 7))
        if i + 1 < n:
            rows.append(i); cols.append(i + 1); vals.append(-1.0)
    rp = np.zeros(n + 1, np.int32)
    np.add.at(rp, np.asarray(rows) + 1, 1)
    return np.cumsum(rp).astype(np.int32), np.asarray(cols, np.int32), np.asarray(vals)


@pytest.mark.parametrize("case,bits,S", [
    ("kuhn3", 32, 64), ("kuhn12", 16, 64), ("kuhn20", 16, 64), ("kuhn26", 32, 128),
    ("kuhn30", 16, 32), ("tri12345", 32, 256), ("tri777", 16, 64)])
def test_persistent_equals_graph_path_shapes(oracle, case, bits, S):
    """The cooperative persistent kernel reproduces the graph path bit for bit for grids of one
    CTA (kuhn3) to 159 CTAs (kuhn30), ragged vector tails (tri*), every slice shape, FP64 and
    the FP32 inner solves."""
    if case.startswith("kuhn"):
        m, b = workloads.kuhn(int(case[4:]), seed=7, dirichlet=True)
        n, rp, ci, v = m.n, m.row_ptr, m.col_idx, m.values
    else:
        n = int(case[3:])
        rp, ci, v = tridiag(n)
        b = np.random.default_rng(n).uniform(-1, 1, n)
    for prec, mixed in ((capi.SPMV_PREC_FP64, 0), (capi.SPMV_PREC_DUAL, 1)):
        A = capi.Matrix(n, rp, ci, v, index_bits=bits, slice_height=S, precision=prec)
        x1, r1 = solve(A, b, rtol=1e-10, mixed=mixed, max_iter=4000)
        x2, r2 = solve(A, b, rtol=1e-10, mixed=mixed, max_iter=4000, persistent=1)
        assert r1["status"] == r2["status"] == capi.SPMV_OK, (r1, r2)
        assert (r1["iterations"], r1["outer_iterations"]) == (r2["iterations"],
                                                              r2["outer_iterations"])
        assert np.array_equal(x1, x2)
        r = b - oracle.spmv(rp, ci, v, x2)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)


def mixed_solve(oracle, m, b, reorder, **opts):
    """GPU refinement through the C ABI in the handle's numbering; x returned in the original one."""
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=reorder,
                    precision=capi.SPMV_PREC_DUAL)
    bi = torch.empty_like(dev(b))
    A.permute(0, dev(b), bi)
    xi = torch.zeros_like(bi)
    res = A.solve(bi, xi, raise_on_error=False, mixed=1, **opts)
    x = torch.empty_like(xi)
    A.permute(1, xi, x)
    torch.cuda.synchronize()
    return x.cpu().numpy(), res


@pytest.mark.parametrize("n,reorder,adaptive", [
    (12, capi.SPMV_REORDER_NONE, 1), (12, capi.SPMV_REORDER_RCM, 1),
    (12, capi.SPMV_REORDER_NONE, 0), (12, capi.SPMV_REORDER_RCM, 0),
    (30, capi.SPMV_REORDER_RCM, 1)])
def test_mixed_refinement_matches_oracle(oracle, n, reorder, adaptive):
    """The refinement against the oracle's refinement (same inner tolerance rule): the same
    number of refinement steps, inner iteration totals within 2 per step, the true FP64
    residual <= 1e-10 by the oracle's SpMV, and the two solutions within the bound that two
    1e-10-residual solutions of this system can differ by (cond(A) * 2e-10, cond(A) below 5e3
    on these meshes, so 1e-6 relative)."""
    m, b = workloads.kuhn(n, seed=1, dirichlet=True)
    x, res = mixed_solve(oracle, m, b, reorder, rtol=1e-10, inner_rtol=1e-4,
                         adaptive_inner=adaptive)
    assert res["status"] == capi.SPMV_OK
    xo, info = oracle.mixed_ir(m.row_ptr, m.col_idx, m.values, b, rtol=1e-10, inner_rtol=1e-4,
                               inner_max_iter=20000, adaptive=bool(adaptive))
    assert info["converged"]
    assert res["outer_iterations"] == info["outer_iterations"] >= 2
    assert abs(res["iterations"] - info["inner_iterations"]) <= 2 * info["outer_iterations"]
    assert true_relres(oracle, m, x, b) <= 1e-10
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    # both against the FP64 oracle's solution, within the same bound
    x64, _ = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, b, rtol=1e-12)
    assert np.linalg.norm(x - x64) <= 1e-6 * np.linalg.norm(x64)
    assert np.linalg.norm(xo - x64) <= 1e-6 * np.linalg.norm(x64)


def test_start_from_solution_and_zero_rhs(oracle):
    m, b = workloads.kuhn(6, seed=2, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values)
    x, res = solve(A, b, rtol=1e-10)
    xd = dev(x)
    res2 = A.solve(dev(b), xd, raise_on_error=False, rtol=1e-8, use_x0=1)
    assert res2["status"] == capi.SPMV_OK and res2["iterations"] == 0
    z, res3 = solve(A, np.zeros(m.n))
    assert res3["status"] == capi.SPMV_OK and res3["iterations"] == 0 and not z.any()


def test_iteration_cap_and_timeouts():
    m, b = workloads.kuhn(10, seed=3, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, precision=capi.SPMV_PREC_DUAL)
    _, res = solve(A, b, rtol=1e-12, max_iter=5, check_every=2)
    assert res["status"] == capi.SPMV_ERR_NOT_CONVERGED and res["iterations"] == 5
    _, res = solve(A, b, rtol=1e-12, max_iter=5, persistent=1)
    assert res["status"] == capi.SPMV_ERR_NOT_CONVERGED and res["iterations"] == 5
    # a wall-clock budget that has already expired: the graph path stops after one batch,
    # the persistent kernel stops at its first budget vote; both report TIMEOUT
    _, res = solve(A, b, rtol=1e-14, timeout_s=1e-9, check_every=4)
    assert res["status"] == capi.SPMV_ERR_TIMEOUT
    _, res = solve(A, b, rtol=1e-14, timeout_s=1e-9, persistent=1)
    assert res["status"] == capi.SPMV_ERR_TIMEOUT
    _, res = solve(A, b, rtol=1e-14, timeout_s=1e-9, mixed=1)
    assert res["status"] == capi.SPMV_ERR_TIMEOUT


def test_bad_inputs():
    # a row without a diagonal entry cannot be Jacobi-preconditioned
    rp = np.array([0, 1, 2], np.int32)
    ci = np.array([1, 0], np.int32)
    A = capi.Matrix(2, rp, ci, np.ones(2))
    _, res = solve(A, np.ones(2))
    assert res["status"] == capi.SPMV_ERR_INVALID_CSR
    m, b = workloads.kuhn(3, seed=0, dirichlet=True)
    F = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values)
    _, res = solve(F, b, mixed=1)  # FP64-only handle has no FP32 values
    assert res["status"] == capi.SPMV_ERR_UNSUPPORTED
    _, res = solve(F, b, inner_rtol=2.0)
    assert res["status"] == capi.SPMV_ERR_INVALID_ARG


@pytest.mark.parametrize("mixed", [0, 1])
def test_c2_full_size_solve(oracle, mixed):
    """6M-cell Dirichlet mesh in RCM order: the true FP64 residual reaches 1e-10."""
    m, b = workloads.c2()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=capi.SPMV_REORDER_RCM,
                    precision=capi.SPMV_PREC_DUAL)
    bd = dev(b)
    bi = torch.empty_like(bd)
    A.permute(0, bd, bi)
    xi = torch.zeros_like(bi)
    res = A.solve(bi, xi, raise_on_error=False, rtol=1e-10, mixed=mixed)
    assert res["status"] == capi.SPMV_OK
    x = torch.empty_like(xi)
    A.permute(1, xi, x)
    assert true_relres(oracle, m, x.cpu().numpy(), b) <= 1e-10


def test_barrier_wait_runs_out_with_a_status():
    """Failure detection without a GPU fault: a grid barrier waiting for a CTA that does not
    exist gives up after its time limit and reports a timeout; the context stays usable."""
    import time
    t0 = time.time()
    st = capi.load().spmv_diag_barrier_timeout(8, 0.2, None)
    assert st == capi.SPMV_ERR_TIMEOUT
    assert time.time() - t0 < 5.0
    # the device still works afterwards
    m, b = workloads.kuhn(4, seed=1, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values)
    _, res = solve(A, b, rtol=1e-10)
    assert res["status"] == capi.SPMV_OK


def test_cg_timing_diagnostic():
    """spmv_diag_cg_timing reports positive, finite times; the handle still solves afterwards."""
    m, b = workloads.kuhn(10, seed=2, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values)
    t = capi.spmv_diag_cg_timing(A.handle, 8)
    assert all(np.isfinite(v) and v > 0 for v in t.values()), t
    _, res = solve(A, b, rtol=1e-10)
    assert res["status"] == capi.SPMV_OK
