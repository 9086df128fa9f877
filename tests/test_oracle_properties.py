"""Randomised properties of the CPU oracle (hypothesis), on random sparse matrices: each
property follows from the definition of the step, independently of the oracle's code --
dense matrix-vector products, permutation matrices, the sliced-ELLPACK layout rules, the
reverse relation of CM and RCM, and the sigma-window sorting rule."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

SETTINGS = settings(max_examples=40, deadline=None)


def _random_csr(seed, n, density, symmetric):
    rng = np.random.default_rng(seed)
    mask = rng.random((n, n)) < density
    if symmetric:
        mask = mask | mask.T
    np.fill_diagonal(mask, True)
    dense = np.where(mask, rng.uniform(-1, 1, (n, n)), 0.0)
    rows, cols = np.nonzero(mask)
    rp = np.zeros(n + 1, np.int32)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    return rp, cols.astype(np.int32), dense[rows, cols], dense


matrices = st.tuples(st.integers(0, 2**31 - 1), st.integers(1, 48), st.floats(0.0, 0.3))


@SETTINGS
@given(matrices)
def test_spmv_equals_dense_product(oracle, case):
    seed, n, density = case
    rp, ci, v, dense = _random_csr(seed, n, density, False)
    x = np.random.default_rng(seed + 1).uniform(-1, 1, n)
    mag = np.abs(dense) @ np.abs(x)
    for use_fma in (False, True):
        y = oracle.spmv(rp, ci, v, x, use_fma=use_fma)
        assert np.all(np.abs(y - dense @ x) <= 4 * n * 2.0 ** -53 * mag + 1e-300)


@SETTINGS
@given(matrices)
def test_permuted_csr_is_p_a_pt(oracle, case):
    seed, n, density = case
    rp, ci, v, dense = _random_csr(seed, n, density, False)
    perm = np.random.default_rng(seed + 2).permutation(n).astype(np.int32)  # new -> old
    rpo, cio, vo = oracle.permute_csr(rp, ci, v, perm)
    B = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rpo))
    B[rows, cio] = vo
    assert np.array_equal(B, dense[np.ix_(perm, perm)])  # values moved, never computed
    assert all(np.all(np.diff(cio[rpo[i]:rpo[i + 1]]) > 0) for i in range(n))


@SETTINGS
@given(matrices, st.sampled_from([1, 2, 4, 8, 32]))
def test_sell_layout_rules(oracle, case, S):
    seed, n, density = case
    rp, ci, v, dense = _random_csr(seed, n, density, False)
    sp, scol, sval = oracle.sell(rp, ci, v, S)
    n_slices = (n + S - 1) // S
    lens = np.diff(rp)
    assert sp[0] == 0 and sp.size == n_slices + 1
    for s in range(n_slices):
        rows = range(s * S, min(n, (s + 1) * S))
        w = max(lens[list(rows)])
        assert sp[s + 1] - sp[s] == S * w  # width = longest row of the slice
        for r in range(s * S, (s + 1) * S):
            for t in range(w):
                at = sp[s] + t * S + (r - s * S)  # column-major inside the slice
                if r < n and t < lens[r]:
                    assert scol[at] == ci[rp[r] + t] and sval[at] == v[rp[r] + t]
                else:
                    assert scol[at] == -1 and sval[at] == 0.0
    cs, ce = oracle.window_meta(n, S, sp, scol)
    for s in range(n_slices):
        c = scol[sp[s]:sp[s + 1]]
        c = c[c >= 0]
        assert (cs[s], ce[s]) == ((c.min(), c.max() + 1) if c.size else (0, 0))


@SETTINGS
@given(matrices)
def test_cm_and_rcm_are_reverse_permutations(oracle, case):
    seed, n, density = case
    rp, ci, _, _ = _random_csr(seed, n, density, True)
    for peripheral in (False, True):
        cm = oracle.cm_order(rp, ci, reverse=False, peripheral=peripheral)
        rcm = oracle.cm_order(rp, ci, reverse=True, peripheral=peripheral)
        assert np.array_equal(np.sort(cm), np.arange(n))
        assert np.array_equal(rcm, cm[::-1])


@SETTINGS
@given(matrices, st.sampled_from([1, 2, 4, 16, 64]))
def test_sigma_sort_rule(oracle, case, sigma):
    seed, n, density = case
    rp, _, _, _ = _random_csr(seed, n, density, False)
    perm_in = np.random.default_rng(seed + 3).permutation(n).astype(np.int32)
    out = oracle.sigma_sort(rp, sigma, perm_in)
    lens = np.diff(rp)
    for w0 in range(0, n, sigma):
        window = perm_in[w0:w0 + sigma]
        # stable sort of the window's rows by decreasing length
        expect = sorted(window, key=lambda r: -lens[r])
        assert list(out[w0:w0 + sigma]) == expect


@SETTINGS
@given(matrices, st.sampled_from([1, 3, 8]))
def test_spmm_columns_are_spmvs(oracle, case, k):
    seed, n, density = case
    rp, ci, v, _ = _random_csr(seed, n, density, False)
    X = np.random.default_rng(seed + 4).uniform(-1, 1, (n, k))
    Y = oracle.spmm(rp, ci, v, X, use_fma=True)
    for c in range(k):
        assert np.array_equal(Y[:, c], oracle.spmv(rp, ci, v, np.ascontiguousarray(X[:, c]),
                                                   use_fma=True))
