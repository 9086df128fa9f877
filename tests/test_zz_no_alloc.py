"""cg_solve_csr_noalloc: the allocation-free solve for callers that cannot allocate device
memory at solve time (for example a plugin whose host application owns all GPU memory, or a
real-time loop with memory fixed in advance).  It must give the same solution as cg_solve on
a matrix handle, within the tolerance the CG tests use, on consecutive calls that share its
fixed scratch array.  Collected last so a failure here does not hide the other GPU tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_12371_gb300 import capi, meshgen

pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_cg_solve_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    capi.load()
    m, rng = meshgen.kuhn_tet_matrix(20, seed=7, dirichlet=True)  # 48,000 rows
    b = meshgen.uniform_vectors(rng, m.n)
    assert m.n <= capi.SPMV_NOALLOC_MAX_ROWS
    bd = torch.from_numpy(b).cuda()

    # the existing entry point: cg_solve on a matrix handle
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values)
    x_ref = torch.zeros_like(bd)
    ref = A.solve(bd, x_ref, rtol=1e-10)
    assert ref["status"] == capi.SPMV_OK

    rp = torch.from_numpy(m.row_ptr).cuda()
    ci = torch.from_numpy(m.col_idx).cuda()
    va = torch.from_numpy(m.values).cuda()
    outs = []
    for _ in range(2):
        x = torch.full_like(bd, float("nan"))  # overwritten: the solve starts from 0
        res = capi.cg_solve_csr_noalloc(m.n, rp, ci, va, bd, x,
                                        capi.cg_default_options(rtol=1e-10))
        torch.cuda.synchronize()
        assert res["status"] == capi.SPMV_OK, res
        assert res["rel_residual"] <= 1e-10
        assert abs(res["iterations"] - ref["iterations"]) <= 2
        xr = x_ref.cpu().numpy()
        assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-7 * np.linalg.norm(xr)
        outs.append(x.cpu().numpy())
    # the shared scratch keeps no state that changes the next call's answer
    assert np.array_equal(outs[0], outs[1])

    # sizes beyond the fixed scratch are refused before any device work
    big = capi.cg_solve_csr_noalloc(capi.SPMV_NOALLOC_MAX_ROWS + 1, rp, ci, va, bd, x)
    assert big["status"] == capi.SPMV_ERR_INVALID_ARG
