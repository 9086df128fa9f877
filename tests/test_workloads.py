"""The synthetic workloads follow their stated recipes (CPU only): the serving stream's cell
counts are log-uniform in [1e4, 2e6] with the stated mean, and each request's box has about
the target number of cells."""
import math

import numpy as np

from paper_2107_12371_gb300 import meshgen, workloads


def test_serving_sizes_log_uniform():
    s = workloads.serving_sizes(2000, seed=0)
    assert s.min() >= 1e4 and s.max() <= 2e6
    u = (np.log(s) - math.log(1e4)) / (math.log(2e6) - math.log(1e4))
    # Kolmogorov-Smirnov distance to the uniform distribution on [0, 1] (n = 2000: the 1 %
    # critical value is 1.63 / sqrt(n) = 0.036)
    u = np.sort(u)
    i = np.arange(1, u.size + 1)
    ks = max(np.max(i / u.size - u), np.max(u - (i - 1) / u.size))
    assert ks < 0.036
    # mean of a log-uniform variable on [a, b]: (b - a) / ln(b / a) = 3.76e5
    expect = (2e6 - 1e4) / math.log(2e6 / 1e4)
    assert abs(s.mean() / expect - 1.0) < 0.08
    assert np.array_equal(s, workloads.serving_sizes(2000, seed=0))  # seeded


def test_box_for_cells_hits_the_target():
    for target in (1e4, 4.8e4, 3.76e5, 1e6, 2e6):
        nx, ny, nz = meshgen.box_for_cells(target)
        cells = 6 * nx * ny * nz
        assert abs(cells / target - 1.0) < 0.05, (target, cells)


def test_serving_request_is_a_dirichlet_kuhn_mesh():
    m, b = workloads.serving_request(7, 10000)
    nx, ny, nz = meshgen.box_for_cells(10000)
    assert m.n == 6 * nx * ny * nz and b.shape == (m.n,)
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    diag = rows == m.col_idx
    assert np.all(m.values[diag] > 0) and np.all(m.values[~diag] <= 0)
    assert np.count_nonzero(diag) == m.n
    # symmetric: the (row, col, value) triples equal the transposed ones
    fwd = sorted(zip(rows.tolist(), m.col_idx.tolist(), m.values.tolist()))
    bwd = sorted(zip(m.col_idx.tolist(), rows.tolist(), m.values.tolist()))
    assert fwd == bwd


def test_fast_kuhn_assembler_equals_generator():
    """The closed-form C assembler used for large boxes and the serving stream gives the
    generator's matrix bit for bit: same structure, same values, same permutation, same
    random stream afterwards (cubes and uneven boxes, Neumann and Dirichlet, permuted or not,
    with and without jitter)."""
    cases = [(2, 2, 2, 0, True, True, 0.2), (3, 4, 5, 1, False, True, 0.2),
             (5, 5, 5, 2, True, False, 0.2), (7, 3, 9, 3, True, True, 0.2),
             (6, 6, 6, 4, False, True, 0.0), (20, 20, 20, 0, False, True, 0.2),
             (11, 11, 40, 7, True, True, 0.2)]
    for nx, ny, nz, seed, dirichlet, permute, jitter in cases:
        ref, r1 = meshgen.kuhn_tet_matrix(nx, ny, nz, seed=seed, dirichlet=dirichlet,
                                          permute=permute, jitter=jitter)
        got, r2 = meshgen.kuhn_tet_matrix_fast(nx, ny, nz, seed=seed, dirichlet=dirichlet,
                                               permute=permute, jitter=jitter)
        assert got.n == ref.n
        assert np.array_equal(got.row_ptr, ref.row_ptr)
        assert np.array_equal(got.col_idx, ref.col_idx)
        assert np.array_equal(got.values.view(np.uint64), ref.values.view(np.uint64))
        if permute:
            assert np.array_equal(got.perm, ref.perm)
        assert r1.uniform() == r2.uniform()


def test_serving_request_uses_the_generator_matrix():
    """A serving request's matrix is the generator's for its box and seed."""
    m, b = workloads.serving_request(17, 2.0e4)
    nx, ny, nz = meshgen.box_for_cells(2.0e4)
    ref, rng = meshgen.kuhn_tet_matrix(nx, ny, nz, seed=17, dirichlet=True)
    assert np.array_equal(m.col_idx, ref.col_idx)
    assert np.array_equal(m.values.view(np.uint64), ref.values.view(np.uint64))
    assert np.array_equal(b, meshgen.uniform_vectors(rng, ref.n))
