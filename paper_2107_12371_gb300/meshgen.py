"""Seeded synthetic inputs: cell-centred finite-volume Laplacians on unstructured meshes.

The paper measures its SpMV on Laplacian matrices from a second-order finite-volume
discretisation on tetrahedral meshes (Sec. 6, Table 1; at most five non-zeros per row on
tetrahedra, Sec. 2).  Its meshes are not published, so this module builds stand-ins with
the same structure:

* a box of ``nx * ny * nz`` hexahedra, vertices jittered uniformly by ``+-jitter*h`` per
  axis (boundary vertices only tangentially, so the domain keeps its shape);
* every hexahedron split into the six Kuhn (Freudenthal) tetrahedra that share the main
  diagonal v000-v111, or (mixed meshes) kept whole, split into two triangular prisms by
  the vertical plane through v000-v110, or split into six tetrahedra;
* one matrix row per cell; for every face shared by cells i and j the coefficient
  ``w = area / |c_i - c_j|`` (c = vertex average of the cell);
* Neumann variant: ``a_ij = +w``, ``a_ii = -sum_j a_ij`` (so ``A 1 = 0``);
  Dirichlet variant: ``a_ij = -w``, ``a_ii = sum_j w_ij + sum_{boundary faces} area /
  |c_i - c_f|`` (c_f = face vertex average), an irreducibly diagonally dominant M-matrix
  and therefore SPD;
* optionally the cells randomly permuted (a symmetric permutation of the matrix).

Faces are handled as triangles: a quadrilateral hexahedron or prism face is split by its
diagonal through its lowest and highest corner, which is exactly the diagonal the Kuhn
split uses on every hexahedron face, so triangles of neighbouring cells match one to one
and non-conforming hexahedron/tetrahedron interfaces connect the hexahedron to each
sub-cell through its own triangle.

This module holds only input generation: no SpMV, CG or reordering arithmetic.  Random
numbers come from ``numpy.random.default_rng(seed)`` (PCG64) in a fixed order: the
per-hexahedron element choice (mixed meshes only), the vertex jitter (vertex order, then
x, y, z), the cell permutation, then any vectors drawn with :func:`uniform_vectors`.
Every floating-point step is an element-wise IEEE operation in a fixed order, so the same
seed gives the same bits on any platform.
"""
from __future__ import annotations

import os
import threading
from dataclasses import dataclass, field

import numpy as np

# Kuhn split: tetrahedron t of a hexahedron follows the axis order KUHN_PERMS[t]:
# vertices 0, e_a, e_a + e_b, e_a + e_b + e_c.
KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))

ELEM_HEX, ELEM_PRISM, ELEM_TET = 0, 1, 2


@dataclass
class CsrMatrix:
    """A CSR matrix (n rows, n_cols columns, square unless n_cols is given) with strictly
    increasing columns in every row."""

    n: int
    row_ptr: np.ndarray  # int32[n + 1]
    col_idx: np.ndarray  # int32[nnz]
    values: np.ndarray  # float64[nnz]
    perm: np.ndarray | None = None  # new -> old cell index of the random permutation
    info: dict = field(default_factory=dict)
    n_cols: int | None = None

    def __post_init__(self):
        if self.n_cols is None:
            self.n_cols = self.n

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n_cols))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        a[rows, self.col_idx] = self.values
        return a


def _bit(v: int, a: int) -> int:
    return (v >> a) & 1


def _corner(di: int, dj: int, dk: int) -> int:
    return di | (dj << 1) | (dk << 2)


def _quad_tris(face_corners):
    """Split a hexahedron face given by its 4 corner codes (all sharing one fixed axis) along
    the diagonal from its lowest to its highest corner; return two triangles and the quad."""
    lo = min(face_corners)
    hi = max(face_corners)
    others = [c for c in face_corners if c not in (lo, hi)]
    return [(lo, others[0], hi), (lo, others[1], hi)]


def _hex_face_corners(axis: int, side: int):
    return [c for c in range(8) if _bit(c, axis) == side]


def _tet_local():
    """Local corner codes of the 6 Kuhn tetrahedra and their 4 triangular faces."""
    tets = []
    for a, b, c in KUHN_PERMS:
        v0 = 0
        v1 = 1 << a
        v2 = v1 | (1 << b)
        v3 = 7
        verts = (v0, v1, v2, v3)
        faces = [tuple(verts[m] for m in range(4) if m != omit) for omit in range(4)]
        tets.append((verts, [(f, list(f)) for f in faces]))
    return tets


def _prism_local():
    """Two prisms split by the vertical plane through v000-v110 (z is the prism axis)."""
    prisms = []
    for side in (0, 1):
        # bottom triangle: v000, v100 (side 0) or v010 (side 1), v110
        mid = _corner(1, 0, 0) if side == 0 else _corner(0, 1, 0)
        bot = (_corner(0, 0, 0), mid, _corner(1, 1, 0))
        top = tuple(c | 4 for c in bot)
        verts = bot + top
        faces = [(bot, list(bot)), (top, list(top))]
        # outer vertical faces: full hexahedron faces
        if side == 0:
            outer = [_hex_face_corners(1, 0), _hex_face_corners(0, 1)]  # y=0, x=1
        else:
            outer = [_hex_face_corners(0, 0), _hex_face_corners(1, 1)]  # x=0, y=1
        for fc in outer:
            for tri in _quad_tris(fc):
                faces.append((tri, fc))
        # internal diagonal quad v000, v110, v111, v001 split along v000-v111
        diag = [_corner(0, 0, 0), _corner(1, 1, 0), _corner(1, 1, 1), _corner(0, 0, 1)]
        faces.append(((diag[0], diag[1], diag[2]), diag))
        faces.append(((diag[0], diag[2], diag[3]), diag))
        prisms.append((verts, faces))
    return prisms


def _hex_local():
    verts = tuple(range(8))
    faces = []
    for axis in range(3):
        for side in (0, 1):
            fc = _hex_face_corners(axis, side)
            for tri in _quad_tris(fc):
                faces.append((tri, fc))
    return [(verts, faces)]


def _local_tables(kind):
    """Return (cell corner lists, per-face triangle corner triples, face id within the cell,
    face corner lists) for one element kind.  Faces of a cell are numbered by their corner
    list, so the two triangles of a quadrilateral share one face id."""
    cells = {ELEM_TET: _tet_local, ELEM_PRISM: _prism_local, ELEM_HEX: _hex_local}[kind]()
    out = []
    for verts, faces in cells:
        face_keys = []
        tris = []
        fids = []
        fcorners = []
        for tri, fc in faces:
            key = tuple(sorted(fc))
            if key not in face_keys:
                face_keys.append(key)
                fcorners.append(list(fc))
            fids.append(face_keys.index(key))
            tris.append(tri)
        out.append((verts, tris, fids, fcorners))
    return out


def _seq_sum(cols):
    """Left-to-right sum of a list of arrays (fixed order, platform independent)."""
    acc = cols[0].copy()
    for c in cols[1:]:
        acc = acc + c
    return acc


def _build(nx, ny, nz, choice, jitter, rng, dirichlet, permute, periodic):
    h = 1.0 / nx
    nvx, nvy, nvz = (nx, ny, nz) if periodic else (nx + 1, ny + 1, nz + 1)
    n_vert = nvx * nvy * nvz
    vi = np.arange(nvx)
    vj = np.arange(nvy)
    vk = np.arange(nvz)
    # jitter (vertex order x fastest, then y, then z; per vertex x, y, z)
    jit = np.zeros((n_vert, 3))
    if jitter > 0.0:
        jit = rng.uniform(-jitter * h, jitter * h, size=(n_vert, 3))
        if not periodic:
            kk, jj, ii = np.meshgrid(vk, vj, vi, indexing="ij")
            ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
            jit[(ii == 0) | (ii == nx), 0] = 0.0
            jit[(jj == 0) | (jj == ny), 1] = 0.0
            jit[(kk == 0) | (kk == nz), 2] = 0.0

    hexes = np.arange(nx * ny * nz)
    hi = hexes % nx
    hj = (hexes // nx) % ny
    hk = hexes // (nx * ny)
    n_per = np.array([1, 2, 6])[choice]
    cell_base = np.zeros(hexes.size + 1, dtype=np.int64)
    np.cumsum(n_per, out=cell_base[1:])
    n_cells = int(cell_base[-1])

    # per-corner unwrapped positions and vertex ids of every hexahedron
    corner_pos = np.empty((hexes.size, 8, 3))
    corner_vid = np.empty((hexes.size, 8), dtype=np.int64)
    for c in range(8):
        ci = hi + _bit(c, 0)
        cj = hj + _bit(c, 1)
        ck = hk + _bit(c, 2)
        if periodic:
            wi, wj, wk = ci % nx, cj % ny, ck % nz
        else:
            wi, wj, wk = ci, cj, ck
        vid = wi + nvx * (wj + nvy * wk)
        corner_vid[:, c] = vid
        corner_pos[:, c, 0] = ci * h + jit[vid, 0]
        corner_pos[:, c, 1] = cj * h + jit[vid, 1]
        corner_pos[:, c, 2] = ck * h + jit[vid, 2]

    centroid = np.empty((n_cells, 3))
    tri_cell, tri_v, tri_area, tri_face, face_cent_parts = [], [], [], [], []
    for kind in (ELEM_HEX, ELEM_PRISM, ELEM_TET):
        sel = np.nonzero(choice == kind)[0]
        if sel.size == 0:
            continue
        for local, (verts, tris, fids, fcorners) in enumerate(_local_tables(kind)):
            cells = cell_base[sel] + local
            pos = corner_pos[sel]
            centroid[cells] = _seq_sum([pos[:, v] for v in verts]) / float(len(verts))
            if kind == ELEM_TET:
                p0, p1, p2, p3 = (pos[:, v] for v in verts)
                vol = np.einsum("ij,ij->i", np.cross(p1 - p0, p2 - p0), p3 - p0)
                q = [np.array([_bit(v, a) for a in range(3)], float) for v in verts]
                ref = np.dot(np.cross(q[1] - q[0], q[2] - q[0]), q[3] - q[0])
                if np.any(vol * ref <= 0.0):
                    raise ValueError("jitter produced an inverted tetrahedron")
            fcent = [
                _seq_sum([pos[:, v] for v in fc]) / float(len(fc)) for fc in fcorners
            ]
            for tri, fid in zip(tris, fids):
                a, b, c = (pos[:, v] for v in tri)
                u = b - a
                w = c - a
                cx = u[:, 1] * w[:, 2] - u[:, 2] * w[:, 1]
                cy = u[:, 2] * w[:, 0] - u[:, 0] * w[:, 2]
                cz = u[:, 0] * w[:, 1] - u[:, 1] * w[:, 0]
                tri_area.append(0.5 * np.sqrt(cx * cx + cy * cy + cz * cz))
                tri_cell.append(cells)
                tri_v.append(np.stack([corner_vid[sel, v] for v in tri], axis=1))
                tri_face.append(cells * 8 + fid)
                face_cent_parts.append(fcent[fid])
    tri_cell = np.concatenate(tri_cell)
    tri_v = np.sort(np.concatenate(tri_v), axis=1)
    tri_area = np.concatenate(tri_area)
    tri_face = np.concatenate(tri_face)
    tri_fcent = np.concatenate(face_cent_parts)

    key = (tri_v[:, 0] * n_vert + tri_v[:, 1]) * n_vert + tri_v[:, 2]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same_next = np.zeros(ks.size, dtype=bool)
    same_next[:-1] = ks[:-1] == ks[1:]
    if np.any(same_next[:-1] & same_next[1:]):
        raise ValueError("a triangle is shared by more than two cells")
    first = np.nonzero(same_next)[0]
    paired = np.zeros(ks.size, dtype=bool)
    paired[first] = True
    paired[first + 1] = True
    ta = order[first]
    tb = order[first + 1]
    ci_ = tri_cell[ta]
    cj_ = tri_cell[tb]
    # interior: sum triangle areas per cell pair, then divide by the centroid distance
    lo = np.minimum(ci_, cj_)
    hi_ = np.maximum(ci_, cj_)
    pkey = lo * n_cells + hi_
    porder = np.argsort(pkey, kind="stable")
    pk = pkey[porder]
    starts = np.nonzero(np.r_[True, pk[1:] != pk[:-1]])[0]
    area_sorted = tri_area[ta][porder]
    pair_area = area_sorted[starts].copy()
    # at most a handful of triangles per pair: add the rest left to right
    counts = np.diff(np.r_[starts, pk.size])
    for extra in range(1, int(counts.max()) if counts.size else 1):
        m = counts > extra
        pair_area[m] = pair_area[m] + area_sorted[starts[m] + extra]
    pi = lo[porder][starts]
    pj = hi_[porder][starts]
    d = centroid[pj] - centroid[pi]
    if periodic:
        ext = np.array([nx * h, ny * h, nz * h])
        d = d - ext * np.round(d / ext)
    dist = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    w = pair_area / dist

    # boundary faces: group triangles by (cell, face), area sum over the face
    bdiag = np.zeros(n_cells)
    bidx = order[~paired]
    n_bfaces = 0
    if bidx.size and not periodic:
        bf = tri_face[bidx]
        border = np.argsort(bf, kind="stable")
        bfs = bf[border]
        bst = np.nonzero(np.r_[True, bfs[1:] != bfs[:-1]])[0]
        bcnt = np.diff(np.r_[bst, bfs.size])
        barea_s = tri_area[bidx][border]
        farea = barea_s[bst].copy()
        for extra in range(1, int(bcnt.max())):
            m = bcnt > extra
            farea[m] = farea[m] + barea_s[bst[m] + extra]
        fcell = tri_cell[bidx][border][bst]
        fc = tri_fcent[bidx][border][bst]
        dd = fc - centroid[fcell]
        fd = np.sqrt(dd[:, 0] * dd[:, 0] + dd[:, 1] * dd[:, 1] + dd[:, 2] * dd[:, 2])
        fw = farea / fd
        n_bfaces = int(fw.size)
        if dirichlet:
            # faces of one cell added in face-id order, left to right
            fo = np.argsort(fcell, kind="stable")
            fcs = fcell[fo]
            fst = np.nonzero(np.r_[True, fcs[1:] != fcs[:-1]])[0]
            fcn = np.diff(np.r_[fst, fcs.size])
            fws = fw[fo]
            acc = fws[fst].copy()
            for extra in range(1, int(fcn.max())):
                m = fcn > extra
                acc[m] = acc[m] + fws[fst[m] + extra]
            bdiag[fcs[fst]] = acc

    # relabel cells (random symmetric permutation), assemble sorted CSR
    perm = None
    if permute:
        perm = rng.permutation(n_cells)  # new -> old
        inv = np.empty(n_cells, dtype=np.int64)
        inv[perm] = np.arange(n_cells)
    else:
        inv = np.arange(n_cells)
    sign = -1.0 if dirichlet else 1.0
    r_off = np.concatenate([inv[pi], inv[pj]])
    c_off = np.concatenate([inv[pj], inv[pi]])
    v_off = np.concatenate([w, w]) * sign
    oorder = np.argsort(r_off * n_cells + c_off, kind="stable")
    r_off, c_off, v_off = r_off[oorder], c_off[oorder], v_off[oorder]
    off_cnt = np.bincount(r_off, minlength=n_cells)
    off_start = np.zeros(n_cells + 1, dtype=np.int64)
    np.cumsum(off_cnt, out=off_start[1:])
    # diagonal: minus the off-diagonals, summed left to right in column order
    diag = np.zeros(n_cells)
    for t in range(int(off_cnt.max()) if n_cells else 0):
        m = off_cnt > t
        diag[m] = diag[m] - v_off[off_start[:-1][m] + t]
    if dirichlet:
        bd = np.empty(n_cells)
        bd[inv] = bdiag
        diag = diag + bd
    rows = np.concatenate([r_off, np.arange(n_cells)])
    cols = np.concatenate([c_off, np.arange(n_cells)])
    vals = np.concatenate([v_off, diag])
    o2 = np.argsort(rows * n_cells + cols, kind="stable")
    rows, cols, vals = rows[o2], cols[o2], vals[o2]
    row_ptr = np.zeros(n_cells + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n_cells), out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("matrix too large for int32 CSR")
    info = dict(
        nx=nx, ny=ny, nz=nz, h=h, jitter=jitter, dirichlet=dirichlet,
        periodic=periodic, n_boundary_faces=n_bfaces,
        # interior faces in the final numbering: lower cell, higher cell, area, distance
        faces=(np.minimum(inv[pi], inv[pj]), np.maximum(inv[pi], inv[pj]), pair_area, dist),
    )
    return CsrMatrix(
        n=n_cells,
        row_ptr=row_ptr.astype(np.int32),
        col_idx=cols.astype(np.int32),
        values=vals.astype(np.float64),
        perm=perm,
        info=info,
    )


def kuhn_tet_matrix(n, ny=None, nz=None, *, jitter=0.2, seed=0, dirichlet=False,
                    permute=True, periodic=False, rng=None):
    """FV Laplacian on an ``n x ny x nz`` box of hexahedra, each split into 6 Kuhn tets.

    Returns ``(matrix, rng)``; draw vectors from the returned generator to follow the
    documented draw order.  ``nnz = 30 n^3 - 12 n^2`` for an ``n^3`` cube."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed) if rng is None else rng
    choice = np.full(n * ny * nz, ELEM_TET, dtype=np.int64)
    m = _build(n, ny, nz, choice, jitter, rng, dirichlet, permute, periodic)
    m.info["kind"] = "kuhn_tet"
    m.info["seed"] = seed
    return m, rng


_FAST_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kuhnbox.c")
_fast_lib = None
_fast_lock = threading.Lock()


def build_fast(force: bool = False) -> str:
    """Compile kuhnbox.c (the closed-form Kuhn-box assembler) into lib/libgb300_kuhnbox.so.
    Safe to call from several threads (the generator threads of the serving stream)."""
    import subprocess
    out_dir = os.path.join(os.path.dirname(_FAST_SRC), "lib")
    os.makedirs(out_dir, exist_ok=True)
    path = os.path.join(out_dir, "libgb300_kuhnbox.so")
    with _fast_lock:
        if (not force and os.path.exists(path)
                and os.path.getmtime(path) >= os.path.getmtime(_FAST_SRC)):
            return path
        tmp = path + ".tmp%d.%d" % (os.getpid(), threading.get_ident())
        subprocess.check_call([os.environ.get("CC", "gcc"), "-O3", "-ffp-contract=off", "-fPIC",
                               "-shared", "-std=c11", "-o", tmp, _FAST_SRC, "-lm"])
        os.replace(tmp, path)
    return path


def _fast():
    global _fast_lib
    if _fast_lib is None:
        import ctypes
        L = ctypes.CDLL(build_fast())
        L.kuhnbox_assemble.restype = ctypes.c_int
        L.kuhnbox_assemble.argtypes = [ctypes.c_int64] * 3 + [ctypes.c_void_p] * 2 + [
            ctypes.c_int] + [ctypes.c_void_p] * 3 + [ctypes.c_int64,
                                                     ctypes.POINTER(ctypes.c_int64)]
        _fast_lib = L
    return _fast_lib


def kuhn_tet_matrix_fast(n, ny=None, nz=None, *, jitter=0.2, seed=0, dirichlet=False,
                         permute=True, rng=None):
    """The matrix of :func:`kuhn_tet_matrix` (non-periodic boxes), bit for bit, assembled by
    kuhnbox.c in closed form (no triangle sorting): the same random draws in the same order
    (vertex jitter, then the cell permutation), then the same element-wise IEEE operations.
    About ten times faster; ``info`` holds only the box description."""
    import ctypes
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed) if rng is None else rng
    h = 1.0 / n
    n_vert = (n + 1) * (ny + 1) * (nz + 1)
    if jitter > 0.0:
        jit = np.ascontiguousarray(rng.uniform(-jitter * h, jitter * h, size=(n_vert, 3)))
    else:
        jit = np.zeros((n_vert, 3))
    n_cells = 6 * n * ny * nz
    perm = rng.permutation(n_cells).astype(np.int64) if permute else None
    row_ptr = np.empty(n_cells + 1, np.int32)
    col = np.empty(5 * n_cells, np.int32)
    val = np.empty(5 * n_cells, np.float64)
    nnz = ctypes.c_int64()
    rc = _fast().kuhnbox_assemble(n, ny, nz, jit.ctypes.data,
                                  perm.ctypes.data if perm is not None else None,
                                  int(bool(dirichlet)), row_ptr.ctypes.data, col.ctypes.data,
                                  val.ctypes.data, 5 * n_cells, ctypes.byref(nnz))
    if rc != 0:
        raise ValueError("kuhnbox_assemble failed with code %d" % rc)
    k = int(nnz.value)
    m = CsrMatrix(n=n_cells, row_ptr=row_ptr, col_idx=col[:k].copy(), values=val[:k].copy(),
                  perm=perm,
                  info=dict(nx=n, ny=ny, nz=nz, h=h, jitter=jitter, dirichlet=dirichlet,
                            periodic=False, kind="kuhn_tet", seed=seed))
    return m, rng


def mixed_matrix(n, ny=None, nz=None, *, p_hex=1 / 3, p_prism=1 / 3, jitter=0.2, seed=1,
                 dirichlet=True, permute=True, rng=None):
    """FV Laplacian on a mixed mesh: every hexahedron is kept (probability ``p_hex``),
    split into 2 prisms (``p_prism``) or into 6 Kuhn tets (the rest)."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed) if rng is None else rng
    nh = n * ny * nz
    if p_hex >= 1.0:
        choice = np.full(nh, ELEM_HEX, dtype=np.int64)
    else:
        u = rng.random(nh)
        choice = np.where(u < p_hex, ELEM_HEX,
                          np.where(u < p_hex + p_prism, ELEM_PRISM, ELEM_TET)).astype(np.int64)
    m = _build(n, ny, nz, choice, jitter, rng, dirichlet, permute, False)
    m.info["kind"] = "mixed"
    m.info["seed"] = seed
    return m, rng


def kuhn_tet_operators(n, ny=None, nz=None, *, jitter=0.2, seed=0, permute=True):
    """Operators of the operator-based finite-volume formulation (Sec. 2) on the Kuhn-tet mesh
    of :func:`kuhn_tet_matrix`: with interior faces f = (lo, hi) numbered by (lo, hi),

    * G (faces x cells): (G x)_f = (x_hi - x_lo) / d_f, the face-normal gradient;
    * M (cells x faces): (M u)_i = sum over faces of i of +area_f u_f (i = lo) or -area_f u_f
      (i = hi), the divergence of face fluxes;

    so that M G equals the Neumann Laplacian L (off-diagonal area/d, diagonal minus their sum)
    up to rounding.  Returns (M, G, L, rng) with L built from the same draws."""
    L, rng = kuhn_tet_matrix(n, ny, nz, jitter=jitter, seed=seed, dirichlet=False,
                             permute=permute)
    lo, hi, area, dist = L.info["faces"]
    order = np.lexsort((hi, lo))
    lo, hi, area, dist = lo[order], hi[order], area[order], dist[order]
    F = lo.size
    N = L.n
    g_rp = (np.arange(F + 1) * 2).astype(np.int32)
    g_ci = np.stack([lo, hi], axis=1).ravel().astype(np.int32)
    inv_d = 1.0 / dist
    g_v = np.stack([-inv_d, inv_d], axis=1).ravel()
    G = CsrMatrix(F, g_rp, g_ci, g_v, n_cols=N)
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([np.arange(F), np.arange(F)])
    vals = np.concatenate([area, -area])
    o = np.lexsort((cols, rows))
    rows, cols, vals = rows[o], cols[o], vals[o]
    m_rp = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=N), out=m_rp[1:])
    M = CsrMatrix(N, m_rp.astype(np.int32), cols.astype(np.int32), vals, n_cols=F)
    return M, G, L, rng


def uniform_vectors(rng, n, k=None, dtype=np.float64):
    """Vector (or row-major ``n x k`` block) of U[-1, 1] draws from ``rng``."""
    shape = (n,) if k is None else (n, k)
    return rng.uniform(-1.0, 1.0, size=shape).astype(dtype)


def box_for_cells(n_cells):
    """Box of Kuhn-tet hexahedra with about ``n_cells`` cells: nx = ny = floor((N/6)^(1/3)),
    nz = round(N / (6 nx ny))."""
    nx = max(1, int(np.floor((n_cells / 6.0) ** (1.0 / 3.0))))
    nz = max(1, int(round(n_cells / (6.0 * nx * nx))))
    return nx, nx, nz
