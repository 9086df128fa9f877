/*
 * kuhnbox.c -- fast assembly of the finite-volume Laplacian of a jittered box of Kuhn
 * tetrahedra.  INPUT GENERATION ONLY: no SpMV, CG or reordering arithmetic.
 *
 * It builds the same matrix, bit for bit, as meshgen.kuhn_tet_matrix for a non-periodic box
 * (the Python module remains the definition; a CPU test compares the two): the caller draws
 * the random numbers with numpy in meshgen's order (vertex jitter, then the cell permutation)
 * and passes them in, and every floating-point step below is the same IEEE operation in the
 * same order as meshgen's element-wise numpy expressions (compile with -ffp-contract=off).
 * What it saves is meshgen's general face matching (sorting every triangle by its vertex
 * triple): in a Kuhn box the neighbour across each tetrahedron face is known in closed form.
 *
 * Geometry.  Hexahedron (i, j, k) has corners coded c = di | dj << 1 | dk << 2.  Tetrahedron t
 * of a hexahedron follows the axis order (a, b, c) = KUHN[t] with vertices 0, e_a, e_a + e_b,
 * 7; its face f omits vertex f.  Faces 1 and 2 contain the main diagonal and are shared with
 * tetrahedra (b, a, c) and (a, c, b) of the same hexahedron (same face index); face 0 lies on
 * the hexahedron face x_a = 1 and is shared with tetrahedron (b, c, a), face 3, of the next
 * hexahedron along axis a; face 3 lies on x_c = 0 and is shared with tetrahedron (c, a, b),
 * face 0, of the previous hexahedron along axis c.  Faces without a neighbour are boundary
 * faces.  Cell id = 6 * hexahedron + t; hexahedron = i + nx (j + ny k).  When two triangles
 * meet, the area is the one computed with the vertex order of the triangle that comes first
 * in meshgen's triangle list, position (4 t + f) * n_hex + hexahedron.
 *
 * Return codes: 0 ok, -1 invalid argument, -2 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static const int KUHN[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static int kuhn_index(int a, int b, int c)
{
    for (int t = 0; t < 6; ++t)
        if (KUHN[t][0] == a && KUHN[t][1] == b && KUHN[t][2] == c) return t;
    return -1;
}

typedef struct {
    int64_t nx, ny, nz, nvx, nvy;
    double h;
    const double *jit; /* n_vert x 3, raw draws (boundary components are ignored) */
} Box;

/* position of vertex (vi, vj, vk): index * h + jitter (jitter zero across the boundary) */
static void vertex_pos(const Box *B, int64_t vi, int64_t vj, int64_t vk, double p[3])
{
    const int64_t vid = vi + B->nvx * (vj + B->nvy * vk);
    const double jx = (vi == 0 || vi == B->nx) ? 0.0 : B->jit[3 * vid + 0];
    const double jy = (vj == 0 || vj == B->ny) ? 0.0 : B->jit[3 * vid + 1];
    const double jz = (vk == 0 || vk == B->nz) ? 0.0 : B->jit[3 * vid + 2];
    p[0] = (double)vi * B->h + jx;
    p[1] = (double)vj * B->h + jy;
    p[2] = (double)vk * B->h + jz;
}

/* the 8 corner positions of hexahedron (i, j, k) */
static void hex_corners(const Box *B, int64_t i, int64_t j, int64_t k, double pos[8][3])
{
    for (int c = 0; c < 8; ++c)
        vertex_pos(B, i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1), pos[c]);
}

static void tet_verts(int t, int v[4])
{
    v[0] = 0;
    v[1] = 1 << KUHN[t][0];
    v[2] = v[1] | (1 << KUHN[t][1]);
    v[3] = 7;
}

/* the triangle of face f (vertex codes in the face's order) */
static void face_tri(int t, int f, int tri[3])
{
    int v[4], m = 0;
    tet_verts(t, v);
    for (int q = 0; q < 4; ++q)
        if (q != f) tri[m++] = v[q];
}

static double tri_area(double pos[8][3], const int tri[3])
{
    const double *a = pos[tri[0]], *b = pos[tri[1]], *c = pos[tri[2]];
    double u[3], w[3];
    for (int d = 0; d < 3; ++d) {
        u[d] = b[d] - a[d];
        w[d] = c[d] - a[d];
    }
    const double cx = u[1] * w[2] - u[2] * w[1];
    const double cy = u[2] * w[0] - u[0] * w[2];
    const double cz = u[0] * w[1] - u[1] * w[0];
    return 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

static double dist3(const double *p, const double *q)
{
    const double d0 = p[0] - q[0], d1 = p[1] - q[1], d2 = p[2] - q[2];
    return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

/* neighbour of face f of tetrahedron t in hexahedron hx: its hexahedron, tetrahedron and face;
 * returns 0 for a boundary face */
static int neighbour(const Box *B, int64_t hx, const int64_t idx[3], int t, int f, int64_t *nhx,
                     int *nt, int *nf)
{
    const int a = KUHN[t][0], b = KUHN[t][1], c = KUHN[t][2];
    const int64_t ext[3] = {B->nx, B->ny, B->nz};
    const int64_t stride[3] = {1, B->nx, B->nx * B->ny};
    if (f == 1) {
        *nhx = hx, *nt = kuhn_index(b, a, c), *nf = 1;
        return 1;
    }
    if (f == 2) {
        *nhx = hx, *nt = kuhn_index(a, c, b), *nf = 2;
        return 1;
    }
    if (f == 0) {
        if (idx[a] + 1 >= ext[a]) return 0;
        *nhx = hx + stride[a], *nt = kuhn_index(b, c, a), *nf = 3;
        return 1;
    }
    if (idx[c] == 0) return 0;
    *nhx = hx - stride[c], *nt = kuhn_index(c, a, b), *nf = 0;
    return 1;
}

/*
 * nx, ny, nz >= 1 hexahedra per axis; jit: (nx+1)(ny+1)(nz+1) x 3 jitter draws; perm: cell
 * permutation (new -> old, 6 nx ny nz entries) or NULL for the unpermuted numbering;
 * dirichlet: 1 for the SPD variant.  Outputs: row_ptr int32[n+1], col int32[cap],
 * val double[cap] with cap >= 5 n; *nnz_out receives the number of entries.
 */
int kuhnbox_assemble(int64_t nx, int64_t ny, int64_t nz, const double *jit, const int64_t *perm,
                     int dirichlet, int32_t *row_ptr, int32_t *col, double *val, int64_t cap,
                     int64_t *nnz_out)
{
    if (nx < 1 || ny < 1 || nz < 1 || !jit || !row_ptr || !col || !val || !nnz_out) return -1;
    const int64_t n_hex = nx * ny * nz, n = 6 * n_hex;
    if (n >= INT32_MAX || cap < 5 * n) return -1;
    Box B = {nx, ny, nz, nx + 1, ny + 1, 1.0 / (double)nx, jit};
    double *cent = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)n); /* -1: boundary face */
    double *nw = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    double *bdiag = (double *)calloc((size_t)n, sizeof(double));
    int32_t *inv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!cent || !nb || !nw || !bdiag || !inv) {
        free(cent); free(nb); free(nw); free(bdiag); free(inv);
        return -2;
    }
    /* centroids: vertex averages, summed left to right in vertex order, then divided by 4 */
    for (int64_t hx = 0; hx < n_hex; ++hx) {
        const int64_t i = hx % nx, j = (hx / nx) % ny, k = hx / (nx * ny);
        double pos[8][3];
        hex_corners(&B, i, j, k, pos);
        for (int t = 0; t < 6; ++t) {
            int v[4];
            tet_verts(t, v);
            double *c = cent + 3 * (6 * hx + t);
            for (int d = 0; d < 3; ++d)
                c[d] = (((pos[v[0]][d] + pos[v[1]][d]) + pos[v[2]][d]) + pos[v[3]][d]) / 4.0;
        }
    }
    /* face weights: area / centroid distance; boundary faces: area / |face centroid - cell
     * centroid|, added to the cell's boundary sum in face order */
    for (int64_t hx = 0; hx < n_hex; ++hx) {
        const int64_t idx[3] = {hx % nx, (hx / nx) % ny, hx / (nx * ny)};
        double pos[8][3];
        hex_corners(&B, idx[0], idx[1], idx[2], pos);
        for (int t = 0; t < 6; ++t) {
            const int64_t cell = 6 * hx + t;
            int have_b = 0;
            for (int f = 0; f < 4; ++f) {
                int tri[3];
                face_tri(t, f, tri);
                int64_t nhx;
                int nt, nf;
                if (!neighbour(&B, hx, idx, t, f, &nhx, &nt, &nf)) {
                    const double area = tri_area(pos, tri);
                    double fc[3];
                    for (int d = 0; d < 3; ++d)
                        fc[d] = ((pos[tri[0]][d] + pos[tri[1]][d]) + pos[tri[2]][d]) / 3.0;
                    const double fw = area / dist3(fc, cent + 3 * cell);
                    bdiag[cell] = have_b ? bdiag[cell] + fw : fw;
                    have_b = 1;
                    nb[4 * cell + f] = -1;
                    continue;
                }
                const int64_t other = 6 * nhx + nt;
                nb[4 * cell + f] = (int32_t)other;
                const int64_t g_self = (int64_t)(4 * t + f) * n_hex + hx;
                const int64_t g_other = (int64_t)(4 * nt + nf) * n_hex + nhx;
                if (g_self > g_other) continue; /* the first triangle of the pair computes */
                const double area = tri_area(pos, tri);
                const int64_t lo = cell < other ? cell : other, hi = cell < other ? other : cell;
                const double *pl = cent + 3 * lo, *ph = cent + 3 * hi;
                const double d0 = ph[0] - pl[0], d1 = ph[1] - pl[1], d2 = ph[2] - pl[2];
                const double w = area / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                nw[4 * cell + f] = w;
                nw[4 * other + nf] = w;
            }
        }
    }
    /* rows in the permuted numbering, columns ascending; diagonal = minus the off-diagonals
     * summed left to right in column order (+ the boundary sum for the Dirichlet variant).
     * Rows are written in the old cells' order (neighbours' new numbers are then read from
     * nearby entries of inv), each at its place in the new order. */
    for (int64_t r = 0; r < n; ++r) inv[perm ? perm[r] : r] = (int32_t)r;
    row_ptr[0] = 0;
    for (int64_t r = 0; r < n; ++r) {
        const int64_t old = perm ? perm[r] : r;
        int32_t len = 1;
        for (int f = 0; f < 4; ++f) len += nb[4 * old + f] >= 0;
        row_ptr[r + 1] = row_ptr[r] + len;
    }
    const double sign = dirichlet ? -1.0 : 1.0;
    for (int64_t old = 0; old < n; ++old) {
        const int64_t r = inv[old];
        int32_t cc[4];
        double vv[4];
        int m = 0;
        for (int f = 0; f < 4; ++f) {
            const int32_t o = nb[4 * old + f];
            if (o < 0) continue;
            const int32_t c = inv[o];
            const double v = nw[4 * old + f] * sign;
            int q = m++;
            while (q > 0 && cc[q - 1] > c) {
                cc[q] = cc[q - 1];
                vv[q] = vv[q - 1];
                --q;
            }
            cc[q] = c;
            vv[q] = v;
        }
        double diag = 0.0;
        for (int q = 0; q < m; ++q) diag = diag - vv[q];
        if (dirichlet) diag = diag + bdiag[old];
        int64_t at = row_ptr[r];
        int placed = 0;
        for (int q = 0; q < m; ++q) {
            if (!placed && cc[q] > r) {
                col[at] = (int32_t)r;
                val[at++] = diag;
                placed = 1;
            }
            col[at] = cc[q];
            val[at++] = vv[q];
        }
        if (!placed) {
            col[at] = (int32_t)r;
            val[at++] = diag;
        }
    }
    const int64_t at = row_ptr[n];
    *nnz_out = at;
    free(cent); free(nb); free(nw); free(bdiag); free(inv);
    return 0;
}
