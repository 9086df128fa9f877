"""Multi-right-hand-side CG (cg_solve_multi) through the C ABI against the CPU oracle.

The oracle of k systems solved in lock-step is k independent solves: oracle.jacobi_pcg (FP64)
or oracle.mixed_ir (refinement) per column.  Bars per column: iteration count within 2 of the
oracle's (refinement: the same number of refinement steps, inner totals within 2 per step),
the true FP64 residual ||b - A x|| / ||b|| recomputed by the oracle's SpMV <= 1e-10, the
reported residual equal to it, and x within 1e-7 (FP64) of the oracle's x; the persistent
kernel reproduces the graph-launched path bit for bit.
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


def _mesh(name):
    if name.startswith("kuhn"):
        m, rng = meshgen.kuhn_tet_matrix(int(name[4:]), seed=3, dirichlet=True)
    else:
        m, rng = meshgen.mixed_matrix(int(name[5:]), seed=1, dirichlet=True)
    return m, rng


def _solve(m, B, reorder=capi.SPMV_REORDER_NONE, precision=capi.SPMV_PREC_FP64, X0=None,
           **opts):
    """cg_solve_multi on a handle of m; B, X in the caller's numbering (n x k)."""
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=reorder, precision=precision)
    perm = A.permutation()
    Bd = torch.from_numpy(np.ascontiguousarray(B[perm])).cuda()
    if X0 is None:
        Xd = torch.full_like(Bd, float("nan"))
    else:
        Xd = torch.from_numpy(np.ascontiguousarray(X0[perm])).cuda()
    st, cols = A.solve_multi(Bd, Xd, **opts)
    torch.cuda.synchronize()
    X = np.empty_like(B)
    X[perm] = Xd.cpu().numpy()
    A.close()
    return st, cols, X


def _relres(oracle, m, x, b):
    nb = np.linalg.norm(b)
    if nb == 0:
        return 0.0
    return np.linalg.norm(b - oracle.spmv(m.row_ptr, m.col_idx, m.values, x)) / nb


@pytest.mark.parametrize("mesh,k,reorder", [
    ("kuhn6", 1, capi.SPMV_REORDER_NONE), ("kuhn6", 3, capi.SPMV_REORDER_RCM),
    ("mixed10", 8, capi.SPMV_REORDER_NONE), ("mixed10", 8, capi.SPMV_REORDER_RCM),
    ("mixed14", 13, capi.SPMV_REORDER_RCM), ("mixed14", 32, capi.SPMV_REORDER_NONE),
    ("kuhn12", 32, capi.SPMV_REORDER_RCM)])
def test_multi_pcg_matches_oracle(oracle, mesh, k, reorder):
    m, rng = _mesh(mesh)
    B = meshgen.uniform_vectors(rng, m.n, k).reshape(m.n, k)
    st, cols, X = _solve(m, B, reorder=reorder, rtol=1e-10)
    assert st == capi.SPMV_OK, cols
    for c in range(k):
        xo, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, B[:, c], rtol=1e-10)
        assert cols[c]["status"] == capi.SPMV_OK
        assert abs(cols[c]["iterations"] - info["iterations"]) <= 2, (c, cols[c], info)
        rr = _relres(oracle, m, X[:, c], B[:, c])
        assert rr <= 1e-10
        assert abs(cols[c]["rel_residual"] - rr) <= 1e-12
        assert np.linalg.norm(X[:, c] - xo) <= 1e-7 * np.linalg.norm(xo)


@pytest.mark.parametrize("mesh,k,adaptive", [("mixed10", 8, 1), ("mixed14", 16, 0),
                                              ("kuhn12", 32, 1)])
def test_multi_refinement_matches_oracle(oracle, mesh, k, adaptive):
    m, rng = _mesh(mesh)
    B = meshgen.uniform_vectors(rng, m.n, k).reshape(m.n, k)
    st, cols, X = _solve(m, B, reorder=capi.SPMV_REORDER_RCM, precision=capi.SPMV_PREC_DUAL,
                         rtol=1e-10, mixed=1, inner_rtol=1e-4, adaptive_inner=adaptive)
    assert st == capi.SPMV_OK, cols
    for c in range(k):
        xo, info = oracle.mixed_ir(m.row_ptr, m.col_idx, m.values, B[:, c], rtol=1e-10,
                                   inner_rtol=1e-4, inner_max_iter=20000,
                                   adaptive=bool(adaptive))
        assert cols[c]["outer_iterations"] == info["outer_iterations"], (c, cols[c], info)
        assert abs(cols[c]["iterations"] - info["inner_iterations"]) <= 2 * info["outer_iterations"]
        rr = _relres(oracle, m, X[:, c], B[:, c])
        assert rr <= 1e-10
        assert abs(cols[c]["rel_residual"] - rr) <= 1e-12
        assert np.linalg.norm(X[:, c] - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("mixed", [0, 1])
@pytest.mark.parametrize("mesh,k", [("kuhn4", 8), ("mixed14", 16), ("kuhn12", 32)])
def test_multi_persistent_equals_graph_path(oracle, mesh, k, mixed):
    m, rng = _mesh(mesh)
    B = meshgen.uniform_vectors(rng, m.n, k).reshape(m.n, k)
    prec = capi.SPMV_PREC_DUAL if mixed else capi.SPMV_PREC_FP64
    st1, c1, X1 = _solve(m, B, precision=prec, rtol=1e-10, mixed=mixed)
    st2, c2, X2 = _solve(m, B, precision=prec, rtol=1e-10, mixed=mixed, persistent=1)
    assert st1 == st2 == capi.SPMV_OK
    assert [(c["iterations"], c["outer_iterations"]) for c in c1] == \
        [(c["iterations"], c["outer_iterations"]) for c in c2]
    assert np.array_equal(X1, X2)
    # repeated solves are deterministic
    _, _, X3 = _solve(m, B, precision=prec, rtol=1e-10, mixed=mixed)
    assert np.array_equal(X1, X3)


def test_multi_columns_stop_independently(oracle):
    """A zero right-hand side is done at once (x = 0); a column started from its solution needs
    no iteration; the other columns run to their own counts."""
    m, rng = _mesh("kuhn8")
    k = 5
    B = meshgen.uniform_vectors(rng, m.n, k).reshape(m.n, k)
    B[:, 2] = 0.0
    X0 = np.zeros_like(B)
    xs, _ = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, B[:, 4], rtol=1e-12)
    X0[:, 4] = xs
    st, cols, X = _solve(m, B, X0=X0, rtol=1e-10, use_x0=1)
    assert st == capi.SPMV_OK
    assert cols[2]["iterations"] == 0 and not X[:, 2].any()
    assert cols[4]["iterations"] == 0 and np.array_equal(X[:, 4], xs)
    for c in (0, 1, 3):
        _, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, B[:, c], rtol=1e-10)
        assert abs(cols[c]["iterations"] - info["iterations"]) <= 2
        assert _relres(oracle, m, X[:, c], B[:, c]) <= 1e-10


def test_multi_caps_timeouts_and_bad_inputs():
    m, rng = _mesh("kuhn8")
    B = meshgen.uniform_vectors(rng, m.n, 4).reshape(m.n, 4)
    st, cols, _ = _solve(m, B, rtol=1e-12, max_iter=5, check_every=2)
    assert st == capi.SPMV_ERR_NOT_CONVERGED
    assert all(c["status"] == capi.SPMV_ERR_NOT_CONVERGED and c["iterations"] == 5 for c in cols)
    st, cols, _ = _solve(m, B, rtol=1e-12, max_iter=5, persistent=1)
    assert st == capi.SPMV_ERR_NOT_CONVERGED and all(c["iterations"] == 5 for c in cols)
    st, cols, _ = _solve(m, B, rtol=1e-14, timeout_s=1e-9, check_every=4)
    assert st == capi.SPMV_ERR_TIMEOUT
    st, cols, _ = _solve(m, B, rtol=1e-14, timeout_s=1e-9, persistent=1)
    assert st == capi.SPMV_ERR_TIMEOUT
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values)
    Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    Xd = torch.zeros_like(Bd)
    for k in (0, 33):
        st, _ = capi.cg_solve_multi(A.handle, k, Bd, Xd)
        assert st == capi.SPMV_ERR_INVALID_ARG
    st, _ = capi.cg_solve_multi(A.handle, 4, Bd, Bd)
    assert st == capi.SPMV_ERR_INVALID_ARG
    st, cols = capi.cg_solve_multi(A.handle, 4, Bd, Xd, capi.cg_default_options(mixed=1))
    assert st == capi.SPMV_ERR_UNSUPPORTED and cols[0]["status"] == capi.SPMV_ERR_UNSUPPORTED
    F = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, precision=capi.SPMV_PREC_FP32)
    st, _ = capi.cg_solve_multi(F.handle, 4, Bd, Xd)
    assert st == capi.SPMV_ERR_UNSUPPORTED


def test_multi_pcg_mixed_mesh_mid_size(oracle):
    """A 40^3 mixed-element mesh (about 190K cells) in RCM order, k = 8: the iteration counts of
    the first and last columns against the oracle's solves, every column's true residual."""
    m, Bv = workloads.mixed(40, seed=1, k=8)
    B = Bv.reshape(m.n, 8)
    st, cols, X = _solve(m, B, reorder=capi.SPMV_REORDER_RCM, rtol=1e-10)
    assert st == capi.SPMV_OK
    for c in range(8):
        assert _relres(oracle, m, X[:, c], B[:, c]) <= 1e-10
    for c in (0, 7):
        _, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, B[:, c], rtol=1e-10)
        assert abs(cols[c]["iterations"] - info["iterations"]) <= 2, (c, cols[c], info)


@pytest.mark.parametrize("k,mixed", [(8, 0), (32, 0), (32, 1)])
def test_multi_pcg_mixed_mesh_full_size(oracle, k, mixed):
    """The 87^3 mixed-element mesh (about 2M cells, rows up to 13 entries) in RCM order, as the
    benchmark solves it: every column's true FP64 residual reaches 1e-10 by the oracle's SpMV
    (an oracle solve per column at this size takes minutes, so the iteration counts are
    compared at the mid size above)."""
    m, Bv = workloads.mixed(87, seed=1, k=k)
    B = Bv.reshape(m.n, k)
    prec = capi.SPMV_PREC_DUAL if mixed else capi.SPMV_PREC_FP64
    st, cols, X = _solve(m, B, reorder=capi.SPMV_REORDER_RCM, precision=prec, rtol=1e-10,
                         mixed=mixed)
    assert st == capi.SPMV_OK
    for c in range(k):
        rr = _relres(oracle, m, X[:, c], B[:, c])
        assert rr <= 1e-10
        assert abs(cols[c]["rel_residual"] - rr) <= 1e-12
