"""cg_solve_csr_noalloc: the allocation-free solve for callers that cannot allocate device
memory at solve time (for example a plugin whose host application owns all GPU memory, or a
real-time loop with memory fixed in advance).  It must give the same solution as cg_solve on
a matrix handle, within the tolerance the CG tests use, on consecutive calls that share its
fixed scratch array; its answer is checked against the CPU oracle (true residual by the
oracle's SpMV, iteration count against the oracle's Jacobi-PCG); and after its set-up it must
take no device memory.  Collected last so a failure here does not hide the other GPU tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_12371_gb300 import capi, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    capi.load()


def _dev_csr(m):
    return (torch.from_numpy(m.row_ptr).cuda(), torch.from_numpy(m.col_idx).cuda(),
            torch.from_numpy(m.values).cuda())


def _true_relres(oracle, m, x, b):
    r = b - oracle.spmv(m.row_ptr, m.col_idx, m.values, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


def _reference(m, bd):
    """The existing entry point: cg_solve on a matrix handle."""
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values)
    x_ref = torch.zeros_like(bd)
    ref = A.solve(bd, x_ref, rtol=1e-10)
    assert ref["status"] == capi.SPMV_OK
    A.close()
    return x_ref.cpu().numpy(), ref


def test_noalloc_solve_matches_cg_solve_on_consecutive_calls(oracle):
    # set-up alone (n = 0): resolves the scratch array's address on this device
    empty = capi.cg_solve_csr_noalloc(0, None, None, None, None, None)
    assert empty["status"] == capi.SPMV_OK

    m, rng = meshgen.kuhn_tet_matrix(20, seed=7, dirichlet=True)  # 48,000 rows
    b = meshgen.uniform_vectors(rng, m.n)
    assert m.n <= capi.SPMV_NOALLOC_MAX_ROWS
    bd = torch.from_numpy(b).cuda()
    xr, ref = _reference(m, bd)
    _, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, b, rtol=1e-10)

    rp, ci, va = _dev_csr(m)
    xs = [torch.full_like(bd, float("nan")) for _ in range(2)]  # overwritten: starts from 0
    torch.cuda.synchronize()
    free = []
    outs = []
    for x in xs:
        res = capi.cg_solve_csr_noalloc(m.n, rp, ci, va, bd, x,
                                        capi.cg_default_options(rtol=1e-10))
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert res["status"] == capi.SPMV_OK, res
        xh = x.cpu().numpy()
        assert res["rel_residual"] <= 1e-10
        assert _true_relres(oracle, m, xh, b) <= 1e-10
        assert abs(res["rel_residual"] - _true_relres(oracle, m, xh, b)) <= 1e-12
        assert abs(res["iterations"] - ref["iterations"]) <= 2
        assert abs(res["iterations"] - info["iterations"]) <= 2
        assert np.linalg.norm(xh - xr) <= 1e-7 * np.linalg.norm(xr)
        outs.append(xh)
    # the shared scratch keeps no state that changes the next call's answer
    assert np.array_equal(outs[0], outs[1])
    # the second call took no device memory
    assert free[0] == free[1]

    # a warm start from the solution needs no iteration
    xw = xs[0]
    res = capi.cg_solve_csr_noalloc(m.n, rp, ci, va, bd, xw,
                                    capi.cg_default_options(rtol=1e-10, use_x0=1))
    torch.cuda.synchronize()
    assert res["status"] == capi.SPMV_OK and res["iterations"] == 0, res
    assert np.array_equal(xw.cpu().numpy(), outs[0])

    # a smaller system right after the larger one, in the same scratch
    m6, rng6 = meshgen.kuhn_tet_matrix(6, seed=3, dirichlet=True)
    b6 = meshgen.uniform_vectors(rng6, m6.n)
    b6d = torch.from_numpy(b6).cuda()
    x6r, ref6 = _reference(m6, b6d)
    rp6, ci6, va6 = _dev_csr(m6)
    x6 = torch.zeros_like(b6d)
    res = capi.cg_solve_csr_noalloc(m6.n, rp6, ci6, va6, b6d, x6,
                                    capi.cg_default_options(rtol=1e-10))
    torch.cuda.synchronize()
    assert res["status"] == capi.SPMV_OK
    assert abs(res["iterations"] - ref6["iterations"]) <= 2
    x6h = x6.cpu().numpy()
    assert np.linalg.norm(x6h - x6r) <= 1e-7 * np.linalg.norm(x6r)
    assert _true_relres(oracle, m6, x6h, b6) <= 1e-10

    # sizes beyond the fixed scratch are refused before any device work
    big = capi.cg_solve_csr_noalloc(capi.SPMV_NOALLOC_MAX_ROWS + 1, rp, ci, va, bd, xs[1])
    assert big["status"] == capi.SPMV_ERR_INVALID_ARG
    # FP32 refinement and the persistent kernel are not offered here
    for opt in (dict(mixed=1), dict(persistent=1)):
        r = capi.cg_solve_csr_noalloc(m6.n, rp6, ci6, va6, b6d, x6,
                                      capi.cg_default_options(**opt))
        assert r["status"] == capi.SPMV_ERR_UNSUPPORTED


def test_noalloc_rejects_a_missing_diagonal():
    """A row without its diagonal cannot be Jacobi-preconditioned: INVALID_CSR, x untouched."""
    m, rng = meshgen.kuhn_tet_matrix(4, seed=1, dirichlet=True)
    b = meshgen.uniform_vectors(rng, m.n)
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    keep = ~((rows == 5) & (m.col_idx == 5))
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=m.n))]).astype(np.int32)
    ci = m.col_idx[keep].astype(np.int32)
    va = m.values[keep]
    x0 = np.linspace(-1.0, 1.0, m.n)
    x = torch.from_numpy(x0.copy()).cuda()
    res = capi.cg_solve_csr_noalloc(m.n, torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
                                    torch.from_numpy(va).cuda(), torch.from_numpy(b).cuda(), x)
    torch.cuda.synchronize()
    assert res["status"] == capi.SPMV_ERR_INVALID_CSR
    assert np.array_equal(x.cpu().numpy(), x0)
