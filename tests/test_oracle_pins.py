"""Pins of the CPU oracle and of the synthetic input generator (CPU only).

Each test checks the oracle against something other than itself: dense brute force,
closed-form eigenpairs, invariants of the finite-volume matrices, hand-worked orderings,
the paper's Table 1 statistics, or textbook special cases of CG.
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_2107_12371_gb300 import meshgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------------------
# generator: brute-force re-assembly of tiny meshes
# ----------------------------------------------------------------------------------------
def _brute_force_tet_matrix(n, jitter, seed, dirichlet):
    """Independent O(N^2) assembly: cells listed by plain loops, faces found by searching
    every pair of cells for three shared vertices, boundary faces as unshared triples."""
    rng = np.random.default_rng(seed)
    nv = n + 1
    h = 1.0 / n
    coords = np.zeros((nv ** 3, 3))
    for k in range(nv):
        for j in range(nv):
            for i in range(nv):
                coords[i + nv * (j + nv * k)] = (i * h, j * h, k * h)
    if jitter:
        jit = rng.uniform(-jitter * h, jitter * h, size=(nv ** 3, 3))
        for v in range(nv ** 3):
            i, j, k = v % nv, (v // nv) % nv, v // (nv * nv)
            for ax, c in enumerate((i, j, k)):
                if c == 0 or c == n:
                    jit[v, ax] = 0.0
        coords = coords + jit
    cells = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for perm in itertools.permutations(range(3)):
                    p = [0, 0, 0]
                    verts = [(i, j, k)]
                    for ax in perm:
                        p[ax] += 1
                        verts.append((i + p[0], j + p[1], k + p[2]))
                    cells.append([a + nv * (b + nv * c) for a, b, c in verts])
    N = len(cells)
    cent = np.array([coords[c].mean(axis=0) for c in cells])
    A = np.zeros((N, N))

    def tri_area(ids):
        a, b, c = coords[list(ids)]
        return 0.5 * np.linalg.norm(np.cross(b - a, c - a))

    shared_faces = {i: [] for i in range(N)}
    for a in range(N):
        sa = set(cells[a])
        for b in range(a + 1, N):
            s = sa & set(cells[b])
            if len(s) == 3:
                w = tri_area(sorted(s)) / np.linalg.norm(cent[a] - cent[b])
                A[a, b] = A[b, a] = w
                shared_faces[a].append(frozenset(s))
                shared_faces[b].append(frozenset(s))
    sign = -1.0 if dirichlet else 1.0
    A *= sign
    for a in range(N):
        A[a, a] = -A[a].sum()
        if dirichlet:
            for f in itertools.combinations(cells[a], 3):
                if frozenset(f) not in shared_faces[a]:
                    fc = coords[list(f)].mean(axis=0)
                    A[a, a] += tri_area(f) / np.linalg.norm(cent[a] - fc)
    return A, rng


@pytest.mark.parametrize("jitter", [0.0, 0.2])
@pytest.mark.parametrize("dirichlet", [False, True])
def test_generator_matches_brute_force(jitter, dirichlet):
    m, _ = meshgen.kuhn_tet_matrix(2, jitter=jitter, seed=3, dirichlet=dirichlet, permute=False)
    ref, _ = _brute_force_tet_matrix(2, jitter, 3, dirichlet)
    A = m.to_dense()
    scale = np.abs(ref).max()
    assert np.array_equal(A != 0, ref != 0) or np.abs(A - ref).max() < 1e-14 * scale
    assert np.abs(A - ref).max() <= 1e-14 * scale


def test_generator_permutation_is_symmetric_relabelling():
    m0, _ = meshgen.kuhn_tet_matrix(3, seed=5, dirichlet=True, permute=False)
    m1, _ = meshgen.kuhn_tet_matrix(3, seed=5, dirichlet=True, permute=True)
    p = m1.perm
    A0 = m0.to_dense()
    A1 = m1.to_dense()
    np.testing.assert_allclose(A1, A0[np.ix_(p, p)], rtol=0, atol=1e-15 * np.abs(A0).max())


@pytest.mark.parametrize("n", [2, 3, 5, 20])
def test_tet_nnz_formula_and_row_length(n):
    m, _ = meshgen.kuhn_tet_matrix(n, seed=0)
    assert m.n == 6 * n ** 3
    assert m.nnz == 30 * n ** 3 - 12 * n ** 2
    assert np.diff(m.row_ptr).max() == 5  # at most 5 non-zeros per row on tets (Sec. 2)
    for i in range(0, m.n, max(1, m.n // 50)):
        seg = m.col_idx[m.row_ptr[i]:m.row_ptr[i + 1]]
        assert np.all(np.diff(seg) > 0)


def test_table1_nnz_per_row_statistic():
    """Table 1: the paper's tet Laplacians carry 4.936-4.970 non-zeros per row; the Kuhn
    generator gives 5 - 2/n per row, which lies within 1% of the paper's C50K..C800K values
    at the comparable sizes n = 20 (48,000 cells) .. n = 50 (750,000 cells)."""
    rows = []
    with open(os.path.join(GOLDEN, "table1_matrices.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, r, z = line.split()
                rows.append((name, int(r), int(z)))
    assert len(rows) == 5
    for (name, r, z), n in zip(rows, [20, 25, 31, 40, 50]):
        paper = z / r
        assert 4.93 < paper < 4.98
        ours = (30 * n ** 3 - 12 * n ** 2) / (6 * n ** 3)
        assert abs(ours - paper) / paper < 0.01, (name, ours, paper)
    m, _ = meshgen.kuhn_tet_matrix(20, seed=0)
    assert abs(m.nnz / m.n - 4.9) < 1e-12


def test_symmetry_bitwise_and_m_matrix():
    m, _ = meshgen.kuhn_tet_matrix(6, seed=0, dirichlet=True)
    A = m.to_dense()
    assert np.array_equal(A, A.T)
    d = np.diag(A)
    off = A - np.diag(d)
    assert np.all(d > 0) and np.all(off <= 0)
    rowsum = A.sum(axis=1)
    assert np.all(rowsum >= -1e-15 * d)
    np.linalg.cholesky(A)  # SPD


def test_mixed_generator_reduces_to_kuhn_and_keeps_invariants():
    """All-tet mixed mesh = Kuhn mesh; all-prism and random mixed meshes stay symmetric with
    A 1 = 0 (Neumann) and positive definite (Dirichlet)."""
    a, _ = meshgen.kuhn_tet_matrix(3, jitter=0.0, dirichlet=True, permute=False)
    b, _ = meshgen.mixed_matrix(3, p_hex=0.0, p_prism=0.0, jitter=0.0, dirichlet=True,
                                permute=False)
    assert np.array_equal(a.values, b.values) and np.array_equal(a.col_idx, b.col_idx)
    for ph, pp in [(0.0, 1.0), (1 / 3, 1 / 3)]:
        mn, _ = meshgen.mixed_matrix(4, p_hex=ph, p_prism=pp, seed=1, dirichlet=False)
        A = mn.to_dense()
        assert np.array_equal(A, A.T)
        assert np.abs(A.sum(axis=1)).max() <= 1e-15 * np.abs(A).max() * 16
        md, _ = meshgen.mixed_matrix(4, p_hex=ph, p_prism=pp, seed=1, dirichlet=True)
        np.linalg.cholesky(md.to_dense())
    assert np.diff(md.row_ptr).max() <= 13


def test_dirichlet_spectrum_matches_continuum_and_neumann_is_semidefinite():
    """Smallest Lanczos Ritz value of the 20^3 Dirichlet matrix (48,000 cells) is positive and
    approximates the continuum one: the FV matrix with face weights area/distance behaves like
    V_cell * (-Laplacian), whose smallest Dirichlet eigenvalue on the unit cube is 3 pi^2, with
    V_cell = h^3 / 6 for the six Kuhn tets of a hexahedron (discretisation error O(h^2)).
    The Neumann matrix is negative semidefinite with the constants as its null space."""
    sla = pytest.importorskip("scipy.sparse.linalg")
    sp = pytest.importorskip("scipy.sparse")
    n = 20
    md, _ = meshgen.kuhn_tet_matrix(n, seed=0, dirichlet=True)
    A = sp.csr_matrix((md.values, md.col_idx, md.row_ptr), shape=(md.n, md.n))
    lam = sla.eigsh(A, k=1, which="SA", return_eigenvectors=False, tol=1e-8, maxiter=20000)[0]
    assert lam > 0.0
    assert abs(lam / (3.0 * math.pi ** 2 / (6.0 * n ** 3)) - 1.0) < 0.05
    mn, _ = meshgen.kuhn_tet_matrix(8, seed=0, dirichlet=False)
    w = np.linalg.eigvalsh(mn.to_dense())
    scale = np.abs(w).max()
    assert w[-1] <= 1e-13 * scale and abs(w[-1]) <= 1e-13 * scale  # one zero eigenvalue
    assert w[-2] < -1e-6 * scale  # connected mesh: the zero is simple


def test_generator_rejects_inverted_tets():
    """The orientation check is live: jitter of half a cell width inverts some tetrahedra."""
    with pytest.raises(ValueError, match="inverted"):
        meshgen.kuhn_tet_matrix(5, jitter=0.5, seed=0)


def test_generator_deterministic():
    a, _ = meshgen.kuhn_tet_matrix(4, seed=11, dirichlet=True)
    b, _ = meshgen.kuhn_tet_matrix(4, seed=11, dirichlet=True)
    assert np.array_equal(a.values, b.values) and np.array_equal(a.col_idx, b.col_idx)


# ----------------------------------------------------------------------------------------
# oracle SpMV
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("use_fma", [False, True])
def test_spmv_matches_dense(oracle, use_fma):
    m, rng = meshgen.kuhn_tet_matrix(3, seed=0, dirichlet=False)
    x = meshgen.uniform_vectors(rng, m.n)
    y = oracle.spmv(m.row_ptr, m.col_idx, m.values, x, use_fma=use_fma)
    A = m.to_dense()
    ref = A @ x
    bound = 1e-15 * (np.abs(A) @ np.abs(x)) + 1e-300
    assert np.all(np.abs(y - ref) <= bound * 4)


def test_spmv_neumann_annihilates_constants(oracle):
    """A 1 = 0 for the pure-Neumann Laplacian, within the rounding of the diagonal sum."""
    m, _ = meshgen.kuhn_tet_matrix(20, seed=0, dirichlet=False)
    y = oracle.spmv(m.row_ptr, m.col_idx, m.values, np.ones(m.n))
    absrow = np.add.reduceat(np.abs(m.values), m.row_ptr[:-1])
    assert np.all(np.abs(y) <= 8 * 2.0 ** -53 * absrow)


def test_spmv_sine_modes_all_hex_dirichlet(oracle):
    """Closed form: on the unjittered all-hexahedron Dirichlet mesh (h = 1/n, interior face
    coefficient h, wall coefficient 2h) the grid sine modes prod_d sin(pi k_d (i_d + 1/2)/n)
    are eigenvectors with eigenvalue h * sum_d 4 sin^2(pi k_d / (2n))."""
    n = 6
    m, _ = meshgen.mixed_matrix(n, p_hex=1.0, p_prism=0.0, jitter=0.0, dirichlet=True,
                                permute=False)
    h = 1.0 / n
    idx = np.arange(n ** 3)
    ii, jj, kk = idx % n, (idx // n) % n, idx // (n * n)
    for kvec in [(1, 1, 1), (2, 1, 3), (5, 5, 5), (1, 4, 2)]:
        v = (np.sin(np.pi * kvec[0] * (ii + 0.5) / n) * np.sin(np.pi * kvec[1] * (jj + 0.5) / n)
             * np.sin(np.pi * kvec[2] * (kk + 0.5) / n))
        lam = h * sum(4 * np.sin(np.pi * kd / (2 * n)) ** 2 for kd in kvec)
        y = oracle.spmv(m.row_ptr, m.col_idx, m.values, v)
        assert np.abs(y - lam * v).max() <= 1e-13 * 8 * h


def _kuhn_symbol(kvec, h):
    """6x6 Bloch symbol of the periodic unjittered Kuhn-tet Laplacian, from analytic
    geometry: tets as lattice-point paths, faces found by shared lattice points among the
    tets of the 27 surrounding hexahedra."""
    def tet(t, off):
        perm = meshgen.KUHN_PERMS[t]
        p = np.array(off, dtype=float)
        pts = [tuple(p)]
        for ax in perm:
            p = p.copy()
            p[ax] += 1
            pts.append(tuple(p))
        return pts

    S = np.zeros((6, 6), dtype=complex)
    for t in range(6):
        a = tet(t, (0, 0, 0))
        ca = np.mean(np.array(a), axis=0) * h
        for off in itertools.product((-1, 0, 1), repeat=3):
            for u in range(6):
                if off == (0, 0, 0) and u == t:
                    continue
                b = tet(u, off)
                s = set(a) & set(b)
                if len(s) != 3:
                    continue
                p0, p1, p2 = (np.array(q) * h for q in s)
                area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0))
                cb = np.mean(np.array(b), axis=0) * h
                w = area / np.linalg.norm(cb - ca)
                S[t, u] += w * np.exp(1j * np.dot(kvec, np.array(off) * h))
                S[t, t] -= w
    return S


def test_spmv_bloch_modes_periodic_kuhn(oracle):
    """Closed form: on the periodic unjittered Kuhn-tet mesh, v = exp(i k.x_hex) (x) phi with
    (lambda, phi) an eigenpair of the 6x6 Bloch symbol satisfies A v = lambda v; at k = 0 the
    smallest eigenvalue is 0 (constants)."""
    n = 4
    m, _ = meshgen.kuhn_tet_matrix(n, jitter=0.0, dirichlet=False, permute=False, periodic=True)
    assert m.nnz == 5 * m.n  # no boundary: every tet has 4 neighbours
    h = 1.0 / n
    hexes = np.arange(n ** 3)
    pos = np.stack([hexes % n, (hexes // n) % n, hexes // (n * n)], axis=1) * h
    for mvec in [(0, 0, 0), (1, 0, 0), (1, 2, 3), (2, 2, 1)]:
        kvec = 2 * np.pi * np.array(mvec) / (n * h)
        S = _kuhn_symbol(kvec, h)
        assert np.abs(S - S.conj().T).max() < 1e-14
        lam, phi = np.linalg.eigh(S)
        if mvec == (0, 0, 0):
            assert abs(lam[-1]) < 1e-14  # constant mode (eigh sorts ascending; A <= 0)
        for e in range(6):
            v = (np.exp(1j * pos @ kvec)[:, None] * phi[None, :, e]).ravel()
            for part in (v.real, v.imag):
                y = oracle.spmv(m.row_ptr, m.col_idx, m.values, np.ascontiguousarray(part))
                assert np.abs(y - lam[e] * part).max() <= 1e-13 * 20 * h


def test_operators_divergence_of_gradient_is_laplacian(oracle):
    """Sec. 2 operator form: M (G x) equals the Neumann Laplacian L x (same faces, same draws)
    up to rounding, checked with the oracle's rectangular CSR products."""
    M, G, L, rng = meshgen.kuhn_tet_operators(6, seed=2)
    x = meshgen.uniform_vectors(rng, L.n)
    assert (M.n, M.n_cols, G.n, G.n_cols) == (L.n, G.n, M.n_cols, L.n)
    assert G.n == (L.nnz - L.n) // 2  # one face per pair of off-diagonals
    gx = oracle.spmv(G.row_ptr, G.col_idx, G.values, x)
    y = oracle.spmv(M.row_ptr, M.col_idx, M.values, gx)
    ref = oracle.spmv(L.row_ptr, L.col_idx, L.values, x)
    scale = np.add.reduceat(np.abs(L.values), L.row_ptr[:-1]) * np.abs(x).max()
    assert np.all(np.abs(y - ref) <= 1e-13 * scale)
    D = M.to_dense() @ G.to_dense()
    np.testing.assert_allclose(D, L.to_dense(), rtol=0, atol=1e-13 * np.abs(L.values).max())


def test_spmv_axpby_matches_definition(oracle):
    m, rng = meshgen.kuhn_tet_matrix(4, seed=3, dirichlet=True)
    x = meshgen.uniform_vectors(rng, m.n)
    y0 = meshgen.uniform_vectors(rng, m.n)
    A = m.to_dense()
    for alpha, beta in [(1.0, 0.0), (2.5, -0.75), (-1.0, 1.0)]:
        y = oracle.spmv_axpby(m.row_ptr, m.col_idx, m.values, alpha, x, beta, y0)
        ref = alpha * (A @ x) + beta * y0
        mag = abs(alpha) * (np.abs(A) @ np.abs(x)) + abs(beta) * np.abs(y0)
        assert np.all(np.abs(y - ref) <= 8 * 2.0 ** -53 * mag)
    y = oracle.spmv_axpby(m.row_ptr, m.col_idx, m.values, 1.0, x, 0.0, np.full(m.n, np.nan))
    assert np.all(np.isfinite(y))  # beta == 0 never reads y


def test_spmv_f32_within_rounding_bound(oracle):
    m, rng = meshgen.kuhn_tet_matrix(5, seed=2, dirichlet=True)
    x = meshgen.uniform_vectors(rng, m.n)
    v32 = m.values.astype(np.float32)
    x32 = x.astype(np.float32)
    y32 = oracle.spmv_f32(m.row_ptr, m.col_idx, v32, x32)
    # exact product of the rounded inputs, then the FP32 accumulation bound (len+1) u
    A32 = meshgen.CsrMatrix(m.n, m.row_ptr, m.col_idx, v32.astype(np.float64)).to_dense()
    exact = A32 @ x32.astype(np.float64)
    mag = np.abs(A32) @ np.abs(x32.astype(np.float64))
    assert np.all(np.abs(y32 - exact) <= 6 * 2.0 ** -24 * mag + 1e-30)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_spmm_matches_dense(oracle, dtype):
    m, rng = meshgen.mixed_matrix(4, seed=1)
    X = meshgen.uniform_vectors(rng, m.n, 8).astype(dtype)
    vals = m.values.astype(dtype)
    Y = oracle.spmm(m.row_ptr, m.col_idx, vals, X)
    A = meshgen.CsrMatrix(m.n, m.row_ptr, m.col_idx, vals.astype(np.float64)).to_dense()
    ref = A @ X.astype(np.float64)
    mag = np.abs(A) @ np.abs(X.astype(np.float64))
    u = 2.0 ** -53 if dtype == np.float64 else 2.0 ** -24
    assert np.all(np.abs(Y - ref) <= 16 * u * mag + 1e-300)


# ----------------------------------------------------------------------------------------
# reordering, permutation, sliced ELLPACK, window metadata
# ----------------------------------------------------------------------------------------
def _read_cm_golden():
    graphs = []
    with open(os.path.join(GOLDEN, "cm_orders.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "graph":
                n = int(tok[2])
                edges = [tuple(map(int, e.split("-"))) for e in tok[3:]]
                graphs.append(dict(name=tok[1], n=n, edges=edges, cm={}))
            elif tok[0] == "cm":
                graphs[-1]["cm"][int(tok[1])] = [int(t) for t in tok[2:]]
    return graphs


def _graph_csr(n, edges, shuffle_cols=False):
    adj = [{i} for i in range(n)]
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    rp = [0]
    ci = []
    for i in range(n):
        ci.extend(sorted(adj[i]))
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32)


def test_cm_orders_hand_worked(oracle):
    graphs = _read_cm_golden()
    assert len(graphs) == 3
    for g in graphs:
        rp, ci = _graph_csr(g["n"], g["edges"])
        for peripheral, expect in g["cm"].items():
            cm = oracle.cm_order(rp, ci, reverse=False, peripheral=bool(peripheral))
            assert list(cm) == expect, (g["name"], peripheral)
            rcm = oracle.cm_order(rp, ci, reverse=True, peripheral=bool(peripheral))
            assert list(rcm) == expect[::-1]


def _bandwidth(rp, ci):
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    return int(np.abs(rows - ci).max())


def test_rcm_reduces_bandwidth_and_is_permutation(oracle):
    """Sec. 4.1 / Figs. before-after: the reordering turns the scattered pattern into a band."""
    m, _ = meshgen.kuhn_tet_matrix(12, seed=0, dirichlet=True)
    perm = oracle.cm_order(m.row_ptr, m.col_idx)
    assert np.array_equal(np.sort(perm), np.arange(m.n))
    rp, ci, vals = oracle.permute_csr(m.row_ptr, m.col_idx, m.values, perm)
    bw_rand = _bandwidth(m.row_ptr, m.col_idx)
    bw_rcm = _bandwidth(rp, ci)
    assert bw_rand > 0.9 * m.n
    assert bw_rcm < 0.1 * m.n
    # a randomly permuted path graph comes back as a path: bandwidth 1
    n = 200
    order = np.random.default_rng(0).permutation(n)
    edges = [(int(order[i]), int(order[i + 1])) for i in range(n - 1)]
    prp, pci = _graph_csr(n, edges)
    pp = oracle.cm_order(prp, pci)
    qrp, qci, _ = oracle.permute_csr(prp, pci, np.ones(pci.size), pp)
    assert _bandwidth(qrp, qci) == 1


def test_sigma_sort_hand_worked_and_invariants(oracle):
    """Row lengths 2 5 2 3 | 1 4 with windows of 4: longest first, equal lengths in order,
    windows never mix -> order 1 3 0 2 | 5 4 (worked by hand).  Starting from the reversed
    order 5 4 3 2 | 1 0 (lengths 4 1 3 2 | 5 2) -> 5 3 2 4 | 1 0."""
    lens = np.array([2, 5, 2, 3, 1, 4])
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    assert list(oracle.sigma_sort(rp, 4)) == [1, 3, 0, 2, 5, 4]
    assert list(oracle.sigma_sort(rp, 4, perm_in=[5, 4, 3, 2, 1, 0])) == [5, 3, 2, 4, 1, 0]
    m, _ = meshgen.mixed_matrix(6, seed=1)
    base = oracle.cm_order(m.row_ptr, m.col_idx)
    p = oracle.sigma_sort(m.row_ptr, 64, perm_in=base)
    assert np.array_equal(np.sort(p), np.arange(m.n))
    L = np.diff(m.row_ptr)[p]
    for w0 in range(0, m.n, 64):
        seg = L[w0:w0 + 64]
        assert np.all(np.diff(seg) <= 0)
        assert set(p[w0:w0 + 64]) == set(base[w0:w0 + 64])


def test_permute_csr_is_pap_t(oracle):
    m, _ = meshgen.kuhn_tet_matrix(3, seed=1, dirichlet=True)
    perm = np.random.default_rng(4).permutation(m.n).astype(np.int32)
    rp, ci, vals = oracle.permute_csr(m.row_ptr, m.col_idx, m.values, perm)
    B = meshgen.CsrMatrix(m.n, rp, ci, vals).to_dense()
    A = m.to_dense()
    assert np.array_equal(B, A[np.ix_(perm, perm)])
    for r in range(m.n):
        assert np.all(np.diff(ci[rp[r]:rp[r + 1]]) > 0)


@pytest.mark.parametrize("S", [1, 4, 32, 64])
def test_sell_round_trip_and_layout(oracle, S):
    m, _ = meshgen.mixed_matrix(3, seed=1)
    sp, scol, sval = oracle.sell(m.row_ptr, m.col_idx, m.values, S)
    n_slices = (m.n + S - 1) // S
    lens = np.zeros(n_slices * S, np.int64)
    lens[:m.n] = np.diff(m.row_ptr)
    widths = lens.reshape(n_slices, S).max(axis=1)
    assert np.array_equal(np.diff(sp), widths * S)
    # rebuild CSR from the column-major slices
    for r in range(m.n):
        s, lane = divmod(r, S)
        w = widths[s]
        at = sp[s] + np.arange(w) * S + lane
        cols = scol[at]
        vals = sval[at]
        L = lens[r]
        assert np.array_equal(cols[:L], m.col_idx[m.row_ptr[r]:m.row_ptr[r + 1]])
        assert np.array_equal(vals[:L], m.values[m.row_ptr[r]:m.row_ptr[r + 1]])
        assert np.all(cols[L:] == -1) and np.all(vals[L:] == 0.0)
    cs, ce = oracle.window_meta(m.n, S, sp, scol)
    for s in range(n_slices):
        lo_r, hi_r = s * S, min((s + 1) * S, m.n)
        c = m.col_idx[m.row_ptr[lo_r]:m.row_ptr[hi_r]]
        if c.size:
            assert cs[s] == c.min() and ce[s] == c.max() + 1
        else:
            assert cs[s] == 0 and ce[s] == 0


# ----------------------------------------------------------------------------------------
# CG and mixed-precision refinement
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 3])
def test_pcg_matches_dense_solve(oracle, n):
    m, rng = meshgen.kuhn_tet_matrix(n, seed=0, dirichlet=True)
    b = meshgen.uniform_vectors(rng, m.n)
    x, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, b, rtol=1e-12)
    A = m.to_dense()
    ref = np.linalg.solve(A, b)
    assert info["converged"]
    assert info["iterations"] <= m.n + 10
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b) * 1.01
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - ref) <= 10 * kappa * 1e-12 * np.linalg.norm(ref)


def test_pcg_diagonal_converges_in_one_iteration(oracle):
    n = 50
    d = np.linspace(1.0, 100.0, n)
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    b = np.random.default_rng(0).uniform(-1, 1, n)
    x, info = oracle.jacobi_pcg(rp, ci, d, b, rtol=1e-14)
    assert info["iterations"] == 1
    np.testing.assert_allclose(x, b / d, rtol=1e-15)


def test_pcg_two_eigenvalues_converges_in_two(oracle):
    """With diag(A) = d and D^{-1/2} A D^{-1/2} = (1 - g) I + g s s^T (s_i = +-1, unit
    diagonal), the Jacobi-preconditioned operator has two distinct eigenvalues, so CG
    terminates after two iterations in exact arithmetic."""
    n = 30
    rng = np.random.default_rng(1)
    d = rng.uniform(1, 10, n)
    s = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    g = 0.3
    M = (1 - g) * np.eye(n) + g * np.outer(s, s)
    A = np.sqrt(d)[:, None] * M * np.sqrt(d)[None, :]
    rp = (np.arange(n + 1) * n).astype(np.int32)
    ci = np.tile(np.arange(n), n).astype(np.int32)
    b = rng.uniform(-1, 1, n)
    x, info = oracle.jacobi_pcg(rp, ci, A.ravel(), b, rtol=1e-10)
    assert info["iterations"] == 2
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)


def test_pcg_zero_rhs_and_iteration_cap(oracle):
    m, rng = meshgen.kuhn_tet_matrix(3, seed=0, dirichlet=True)
    x, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, np.zeros(m.n))
    assert info["converged"] and info["iterations"] == 0 and not x.any()
    b = meshgen.uniform_vectors(rng, m.n)
    x, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, b, rtol=1e-12, max_iter=3)
    assert not info["converged"] and info["iterations"] == 3


def test_pcg_energy_error_decreases_monotonically(oracle):
    """Preconditioned CG minimises the A-norm of the error over a growing Krylov space, so
    ||x_k - x*||_A never increases from one iteration to the next and, in exact arithmetic,
    reaches zero within n steps.  The iterates are the oracle's runs capped at k iterations.
    A wrong step length or direction update (alpha, beta, the preconditioner) breaks this."""
    m, rng = meshgen.kuhn_tet_matrix(3, seed=5, dirichlet=True)
    b = meshgen.uniform_vectors(rng, m.n)
    A = m.to_dense()
    xs = np.linalg.solve(A, b)

    def energy(x):
        e = x - xs
        return float(e @ (A @ e))

    prev = energy(np.zeros(m.n))
    for k in range(1, 40):
        x, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, b, rtol=0.0, max_iter=k,
                                    max_restarts=0)
        assert info["iterations"] == k
        e = energy(x)
        assert e <= prev * (1 + 1e-9) + 1e-28, k
        prev = e
    assert prev <= 1e-16 * energy(np.zeros(m.n))  # converged to rounding (error ~1e-9)


def test_mixed_ir_outer_steps_contract(oracle):
    """Each refinement step solves A d = r to the inner tolerance, so the outer residual falls
    by about that factor per step: with a fixed inner tolerance of 1e-3, reaching 1e-10 takes
    at most ceil(10 / 3) + 1 = 5 steps and at least 2 (an FP32 inner solve cannot give 1e-10)."""
    m, rng = meshgen.kuhn_tet_matrix(5, seed=2, dirichlet=True)
    b = meshgen.uniform_vectors(rng, m.n)
    x, info = oracle.mixed_ir(m.row_ptr, m.col_idx, m.values, b, rtol=1e-10, inner_rtol=1e-3,
                              adaptive=False)
    assert info["converged"]
    assert 2 <= info["outer_iterations"] <= 5
    assert info["rel_residual"] <= 1e-10


@pytest.mark.parametrize("adaptive", [False, True])
def test_mixed_ir_reaches_fp64_residual(oracle, adaptive):
    m, rng = meshgen.kuhn_tet_matrix(6, seed=0, dirichlet=True)
    b = meshgen.uniform_vectors(rng, m.n)
    x, info = oracle.mixed_ir(m.row_ptr, m.col_idx, m.values, b, rtol=1e-10, adaptive=adaptive)
    A = m.to_dense()
    assert info["converged"]
    assert 2 <= info["outer_iterations"] <= 8
    res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert res <= 1e-10
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= np.linalg.cond(A) * 1e-10 * np.linalg.norm(ref)


def _jacobi_pcg_dense(A, rhs, tol, cap):
    """Textbook Jacobi-preconditioned CG in FP64 on a dense matrix (numpy products), from
    x = 0: returns (iterations until ||r|| <= tol ||rhs||, capped at cap; the iterate)."""
    dinv = 1.0 / np.diag(A)
    x = np.zeros_like(rhs)
    r = rhs.copy()
    z = dinv * r
    p = z.copy()
    rho = r @ z
    nb = np.linalg.norm(rhs)
    for it in range(1, cap + 1):
        q = A @ p
        a = rho / (p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= tol * nb:
            return it, x
        z = dinv * r
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return cap, x


def _adaptive_inner_tol(rtol, inner_rtol, bnorm, rnorm):
    """Inner tolerance of a refinement step, as the reading of the refinement defines it: the
    reduction the outer residual still needs with a factor 2 of margin, at least inner_rtol and
    at most 1/2."""
    return max(inner_rtol, min(0.5, 0.5 * rtol * bnorm / rnorm))


def test_mixed_ir_adaptive_inner_tolerance_first_step(oracle):
    """With rtol = 1e-3 and inner_rtol = 1e-6 the adaptive rule sets the first inner tolerance to
    0.5 rtol = 5e-4 (r = b at the first step): one refinement step whose inner solve takes as
    many iterations as textbook FP64 Jacobi-PCG needs to reduce its residual by 5e-4 (within one,
    for the FP32 rounding); without the rule the inner solve runs to 1e-6."""
    m, rng = meshgen.kuhn_tet_matrix(5, seed=4, dirichlet=True)
    b = meshgen.uniform_vectors(rng, m.n)
    A = m.to_dense()
    tol1 = _adaptive_inner_tol(1e-3, 1e-6, 1.0, 1.0)
    m1, _ = _jacobi_pcg_dense(A, b, tol1, 1000)
    _, info = oracle.mixed_ir(m.row_ptr, m.col_idx, m.values, b, rtol=1e-3, inner_rtol=1e-6,
                              adaptive=True)
    assert info["converged"] and info["outer_iterations"] == 1
    assert abs(info["inner_iterations"] - m1) <= 1
    m_fixed, _ = _jacobi_pcg_dense(A, b, 1e-6, 1000)
    assert m_fixed > m1 + 5
    _, info = oracle.mixed_ir(m.row_ptr, m.col_idx, m.values, b, rtol=1e-3, inner_rtol=1e-6,
                              adaptive=False)
    assert info["outer_iterations"] == 1 and abs(info["inner_iterations"] - m_fixed) <= 1


def test_mixed_ir_adaptive_inner_tolerance_second_step(oracle):
    """The rule's ratio ||b|| / ||r||: the first inner solve is capped at j iterations (j chosen
    so that textbook FP64 PCG leaves a relative residual rho1 < 3e-3), so the second step starts
    from ||r1|| = rho1 ||b|| and must stop at max(1e-7, min(1/2, 0.5 rtol / rho1)) -- a loose
    tolerance that a fresh PCG on r1 / ||r1|| reaches in m2 < j iterations.  Expected: two
    refinement steps and j + m2 inner iterations (within one).  Taking ||r|| / ||b|| instead of
    ||b|| / ||r||, or max instead of min, changes the second step's count."""
    m, rng = meshgen.kuhn_tet_matrix(5, seed=4, dirichlet=True)
    b = meshgen.uniform_vectors(rng, m.n)
    A = m.to_dense()
    rtol, inner_rtol = 1e-4, 1e-7
    j = next(k for k in range(1, 200)
             if np.linalg.norm(b - A @ _jacobi_pcg_dense(A, b, 0.0, k)[1]) < 3e-3 * np.linalg.norm(b))
    _, xj = _jacobi_pcg_dense(A, b, 0.0, j)
    r1 = b - A @ xj
    rho1 = np.linalg.norm(r1) / np.linalg.norm(b)
    tol2 = _adaptive_inner_tol(rtol, inner_rtol, np.linalg.norm(b), np.linalg.norm(r1))
    assert inner_rtol < tol2 < 0.5 and rho1 > 2 * rtol  # the rule is active at step 2
    m2, _ = _jacobi_pcg_dense(A, r1 / np.linalg.norm(r1), tol2, 1000)
    assert m2 + 2 < j  # the second inner solve stops on its tolerance, not on the cap
    _, info = oracle.mixed_ir(m.row_ptr, m.col_idx, m.values, b, rtol=rtol, inner_rtol=inner_rtol,
                              inner_max_iter=j, adaptive=True)
    assert info["converged"] and info["outer_iterations"] == 2
    assert abs(info["inner_iterations"] - (j + m2)) <= 1
