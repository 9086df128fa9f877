"""Named synthetic workloads (seeded inputs only; no method arithmetic).

C1  Kuhn-tet 20^3 cube (48,000 cells), jitter +-0.2h, seed 0, Neumann, cells permuted.
C2  Kuhn-tet 100^3 cube (6,000,000 cells, 29,880,000 non-zeros), Dirichlet (SPD), permuted;
    used in random order and RCM order.
C4  mixed hexahedron / 2-prism / 6-tet mesh, seed 1, Dirichlet, permuted (87^3 ~ 2M cells).
C5  serving stream: independently seeded Kuhn-tet boxes, cell counts log-uniform in
    [1e4, 2e6].

Kuhn-tet boxes of 30^3 hexahedra and more (and every serving request) are assembled by the
closed-form C assembler meshgen.kuhn_tet_matrix_fast, which gives meshgen.kuhn_tet_matrix's
matrix bit for bit (tests/test_workloads.py compares the two).

Large matrices are cached as .npz files under ``$GB300_SPMV_CACHE`` (default: the system temp
directory) keyed by their parameters, so repeated runs skip generation.
"""
from __future__ import annotations

import os
import tempfile

import numpy as np

from . import meshgen


def _cache_dir():
    d = os.environ.get("GB300_SPMV_CACHE", os.path.join(tempfile.gettempdir(), "gb300_spmv_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def _cached(key, make):
    path = os.path.join(_cache_dir(), key + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        m = meshgen.CsrMatrix(int(z["n"]), z["row_ptr"], z["col_idx"], z["values"],
                              z["perm"] if z["perm"].size else None)
        return m, z["vec"]
    m, vec = make()
    tmp = path + ".tmp%d.npz" % os.getpid()
    np.savez(tmp, n=m.n, row_ptr=m.row_ptr, col_idx=m.col_idx, values=m.values,
             perm=m.perm if m.perm is not None else np.empty(0, np.int64), vec=vec)
    os.replace(tmp, path)
    return m, vec


def kuhn(n, seed=0, dirichlet=False, jitter=0.2, permute=True, k=None, cache=None):
    """Kuhn-tet n^3 matrix and its U[-1,1] vector (or n x k block) drawn after it."""
    def make():
        # the closed-form assembler gives meshgen.kuhn_tet_matrix's matrix bit for bit
        gen = meshgen.kuhn_tet_matrix_fast if n >= 30 else meshgen.kuhn_tet_matrix
        m, rng = gen(n, seed=seed, dirichlet=dirichlet, jitter=jitter, permute=permute)
        return m, meshgen.uniform_vectors(rng, m.n, k)
    if cache is None:
        cache = n >= 60
    if not cache:
        return make()
    key = "kuhn_n%d_s%d_d%d_j%g_p%d_k%s" % (n, seed, int(dirichlet), jitter, int(permute), k)
    return _cached(key, make)


def c1():
    return kuhn(20, seed=0, dirichlet=False)


def c2():
    return kuhn(100, seed=0, dirichlet=True)


def mixed(n, seed=1, k=8, cache=None):
    def make():
        m, rng = meshgen.mixed_matrix(n, seed=seed, dirichlet=True)
        return m, meshgen.uniform_vectors(rng, m.n, k)
    if cache is None:
        cache = n >= 40
    if not cache:
        return make()
    return _cached("mixed_n%d_s%d_k%d" % (n, seed, k), make)


def serving_sizes(count, seed=0, lo=1e4, hi=2e6):
    """Cell-count targets of the serving stream, log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))


def serving_request(index, target_cells):
    """Request ``index``: Kuhn-tet box of about ``target_cells`` cells, seed = index,
    Dirichlet, cells permuted, right-hand side U[-1,1]."""
    nx, ny, nz = meshgen.box_for_cells(target_cells)
    m, rng = meshgen.kuhn_tet_matrix_fast(nx, ny, nz, seed=index, dirichlet=True)
    return m, meshgen.uniform_vectors(rng, m.n)
