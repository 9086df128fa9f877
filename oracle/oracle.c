/*
 * oracle.c -- plain, slow, obviously correct FP64 CPU reference for the SpMV / CG path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header or constant with
 * the CUDA library and never calls it.
 *
 * Every routine is the plain definition, written out sequentially:
 *   - y = A x in CSR order (Sec. 4.3, the naive SpMV; Sec. 4.2 for the formats);
 *   - Cuthill-McKee ordering by breadth-first search (Sec. 4.1, ref. CUT69);
 *   - sliced ELLPACK with S rows per slice, column-major inside a slice, rows padded to the
 *     slice's longest row (Sec. 4.2, ref. MON10);
 *   - per-slice first/last column of the multiplying vector (Sec. 5.1, col_start / col_end);
 *   - Jacobi-preconditioned CG and FP32-inner / FP64-outer iterative refinement (not in the
 *     paper; each is defined step by step above its routine below).
 * Compile with -O2 -ffp-contract=off so a*b+c is never fused unless fma() is called.
 *
 * Return codes: 0 ok, -1 invalid argument/matrix, -2 out of memory, 1 not converged.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* SpMV (Sec. 4.3): y_i = sum over k in [row_ptr[i], row_ptr[i+1]) of val[k] * x[col[k]],  */
/* accumulated left to right starting from +0.0.  use_fma selects acc = fma(a, x, acc)     */
/* instead of acc = acc + (a * x).                                                          */
/* ------------------------------------------------------------------------------------ */
void oracle_csr_spmv(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                     const double *val, const double *x, double *y, int use_fma)
{
    for (int32_t i = 0; i < n_rows; ++i) {
        double acc = 0.0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (use_fma) {
                acc = fma(val[k], x[col_idx[k]], acc);
            } else {
                double p = val[k] * x[col_idx[k]];
                acc = acc + p;
            }
        }
        y[i] = acc;
    }
}

/* Accumulating form y = alpha (A x) + beta y (the paper's task signature reads and writes the */
/* result vector, Sec. 3.2): t = the CSR-order row sum with fused multiply-add from +0.0, then */
/* y_i = fma(alpha, t, beta * y_i), or alpha * t when beta == 0 (y_i is then not read).        */
void oracle_csr_spmv_axpby(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                           const double *val, double alpha, const double *x, double beta,
                           double *y)
{
    for (int32_t i = 0; i < n_rows; ++i) {
        double t = 0.0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) t = fma(val[k], x[col_idx[k]], t);
        y[i] = (beta != 0.0) ? fma(alpha, t, beta * y[i]) : alpha * t;
    }
}

/* Same definition with FP32 values, vector and accumulator. */
void oracle_csr_spmv_f32(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                         const float *val, const float *x, float *y, int use_fma)
{
    for (int32_t i = 0; i < n_rows; ++i) {
        float acc = 0.0f;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (use_fma) {
                acc = fmaf(val[k], x[col_idx[k]], acc);
            } else {
                float p = val[k] * x[col_idx[k]];
                acc = acc + p;
            }
        }
        y[i] = acc;
    }
}

/* Multi-RHS product Y = A X as k independent SpMVs; X is n_cols x k and Y n_rows x k, both  */
/* row-major (column c of X is X[j*k + c]).                                                 */
void oracle_spmm(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                 const double *val, int32_t k, const double *X, double *Y, int use_fma)
{
    for (int32_t c = 0; c < k; ++c) {
        for (int32_t i = 0; i < n_rows; ++i) {
            double acc = 0.0;
            for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                double xv = X[(int64_t)col_idx[e] * k + c];
                if (use_fma) {
                    acc = fma(val[e], xv, acc);
                } else {
                    double p = val[e] * xv;
                    acc = acc + p;
                }
            }
            Y[(int64_t)i * k + c] = acc;
        }
    }
}

void oracle_spmm_f32(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                     const float *val, int32_t k, const float *X, float *Y, int use_fma)
{
    for (int32_t c = 0; c < k; ++c) {
        for (int32_t i = 0; i < n_rows; ++i) {
            float acc = 0.0f;
            for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                float xv = X[(int64_t)col_idx[e] * k + c];
                if (use_fma) {
                    acc = fmaf(val[e], xv, acc);
                } else {
                    float p = val[e] * xv;
                    acc = acc + p;
                }
            }
            Y[(int64_t)i * k + c] = acc;
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Cuthill-McKee (Sec. 4.1).  Breadth-first search over the row adjacency (entries with     */
/* col != row).  Rules, in this order:                                                      */
/*   start node  : among unvisited nodes the one of minimum degree, lowest index on ties;   */
/*                 with peripheral != 0 refined by George-Liu: repeatedly move to the       */
/*                 min-(degree, index) node of the last BFS level while the eccentricity    */
/*                 grows (at most 8 moves);                                                 */
/*   visiting    : a node's unvisited neighbours are appended in increasing (degree, index);*/
/*   components  : when the queue empties, restart from the next start node;               */
/*   reverse     : reverse != 0 returns the reversed order (RCM).                           */
/* perm[new] = old.                                                                         */
/* ------------------------------------------------------------------------------------ */
static int32_t degree_of(const int32_t *row_ptr, const int32_t *col_idx, int32_t i)
{
    int32_t d = 0;
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
        if (col_idx[k] != i) ++d;
    return d;
}

static int key_less(const int32_t *deg, int32_t a, int32_t b)
{
    if (deg[a] != deg[b]) return deg[a] < deg[b];
    return a < b;
}

/* BFS levels from r over nodes with blocked[] == 0; returns the eccentricity and the      */
/* min-(degree, index) node of the last level in *last_pick.                                */
static int32_t bfs_levels(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                          const int32_t *deg, const unsigned char *blocked, int32_t r,
                          int32_t *level, int32_t *queue, int32_t *last_pick)
{
    for (int32_t i = 0; i < n; ++i) level[i] = -1;
    int32_t head = 0, tail = 0;
    queue[tail++] = r;
    level[r] = 0;
    int32_t ecc = 0;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int32_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
            int32_t v = col_idx[k];
            if (v == u || blocked[v] || level[v] >= 0) continue;
            level[v] = level[u] + 1;
            if (level[v] > ecc) ecc = level[v];
            queue[tail++] = v;
        }
    }
    int32_t pick = -1;
    for (int32_t t = 0; t < tail; ++t) {
        int32_t v = queue[t];
        if (level[v] == ecc && (pick < 0 || key_less(deg, v, pick))) pick = v;
    }
    *last_pick = pick;
    return ecc;
}

int oracle_cm_order(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int reverse,
                    int peripheral, int32_t *perm)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    unsigned char *visited = (unsigned char *)calloc((size_t)n, 1);
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t maxdeg = 0;
    if (!deg || !visited || !level || !queue) {
        free(deg); free(visited); free(level); free(queue);
        return -2;
    }
    for (int32_t i = 0; i < n; ++i) {
        deg[i] = degree_of(row_ptr, col_idx, i);
        if (deg[i] > maxdeg) maxdeg = deg[i];
    }
    int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxdeg + 1));
    if (!nb) { free(deg); free(visited); free(level); free(queue); return -2; }

    int32_t pos = 0;
    while (pos < n) {
        int32_t start = -1;
        for (int32_t i = 0; i < n; ++i)
            if (!visited[i] && (start < 0 || key_less(deg, i, start))) start = i;
        if (peripheral) {
            int32_t pick;
            int32_t ecc = bfs_levels(n, row_ptr, col_idx, deg, visited, start, level, queue, &pick);
            for (int moves = 0; moves < 8; ++moves) {
                int32_t pick2;
                int32_t ecc2 = bfs_levels(n, row_ptr, col_idx, deg, visited, pick, level, queue, &pick2);
                if (ecc2 > ecc) {
                    start = pick;
                    ecc = ecc2;
                    pick = pick2;
                } else {
                    break;
                }
            }
        }
        int32_t head = pos;
        perm[pos++] = start;
        visited[start] = 1;
        while (head < pos) {
            int32_t u = perm[head++];
            int32_t cnt = 0;
            for (int32_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
                int32_t v = col_idx[k];
                if (v == u || visited[v]) continue;
                nb[cnt++] = v;
                visited[v] = 1;
            }
            /* insertion sort by (degree, index) */
            for (int32_t a = 1; a < cnt; ++a) {
                int32_t v = nb[a];
                int32_t b = a - 1;
                while (b >= 0 && key_less(deg, v, nb[b])) {
                    nb[b + 1] = nb[b];
                    --b;
                }
                nb[b + 1] = v;
            }
            for (int32_t a = 0; a < cnt; ++a) perm[pos++] = nb[a];
        }
    }
    if (reverse) {
        for (int32_t a = 0, b = n - 1; a < b; ++a, --b) {
            int32_t t = perm[a];
            perm[a] = perm[b];
            perm[b] = t;
        }
    }
    free(nb); free(deg); free(visited); free(level); free(queue);
    return 0;
}

/* Length sorting inside windows (sliced ELLPACK with sorting scope sigma, ref. MON10 and its  */
/* SELL-C-sigma refinement): rows are taken in the order perm_in (perm_in[new] = old; NULL =  */
/* identity); inside each window of sigma consecutive positions they are reordered by         */
/* decreasing row length, rows of equal length keeping their order.  perm_out[new] = old.     */
int oracle_sigma_sort(int32_t n, const int32_t *row_ptr, const int32_t *perm_in, int32_t sigma,
                      int32_t *perm_out)
{
    if (n < 0 || sigma < 1) return -1;
    for (int32_t i = 0; i < n; ++i) perm_out[i] = perm_in ? perm_in[i] : i;
    for (int32_t w0 = 0; w0 < n; w0 += sigma) {
        int32_t w1 = w0 + sigma < n ? w0 + sigma : n;
        for (int32_t a = w0 + 1; a < w1; ++a) { /* stable insertion sort, longest first */
            int32_t v = perm_out[a];
            int32_t lv = row_ptr[v + 1] - row_ptr[v];
            int32_t b = a - 1;
            while (b >= w0 && row_ptr[perm_out[b] + 1] - row_ptr[perm_out[b]] < lv) {
                perm_out[b + 1] = perm_out[b];
                --b;
            }
            perm_out[b + 1] = v;
        }
    }
    return 0;
}

/* Symmetric permutation B = P A P^T with perm[new] = old: row r of B is row perm[r] of A,  */
/* every column c renumbered to inv[c], then the row sorted by new column (Sec. 4.1: the    */
/* coefficients are unchanged, only renumbered).                                            */
int oracle_permute_csr(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                       const double *val, const int32_t *perm, int32_t *row_ptr_out,
                       int32_t *col_out, double *val_out)
{
    int32_t *inv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!inv) return -2;
    for (int32_t r = 0; r < n; ++r) inv[perm[r]] = r;
    row_ptr_out[0] = 0;
    for (int32_t r = 0; r < n; ++r) {
        int32_t old = perm[r];
        int32_t len = row_ptr[old + 1] - row_ptr[old];
        int32_t base = row_ptr_out[r];
        for (int32_t t = 0; t < len; ++t) {
            col_out[base + t] = inv[col_idx[row_ptr[old] + t]];
            val_out[base + t] = val[row_ptr[old] + t];
        }
        for (int32_t a = 1; a < len; ++a) {
            int32_t c = col_out[base + a];
            double v = val_out[base + a];
            int32_t b = a - 1;
            while (b >= 0 && col_out[base + b] > c) {
                col_out[base + b + 1] = col_out[base + b];
                val_out[base + b + 1] = val_out[base + b];
                --b;
            }
            col_out[base + b + 1] = c;
            val_out[base + b + 1] = v;
        }
        row_ptr_out[r + 1] = base + len;
    }
    free(inv);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Sliced ELLPACK (Sec. 4.2): S rows per slice (rows >= n are empty), slice width w_s = the */
/* longest row in the slice, slice_ptr[s+1] = slice_ptr[s] + S * w_s, entry t of row r at   */
/* slice_ptr[s] + t*S + (r - s*S).  Padding entries hold col = -1 and val = 0.0.            */
/* ------------------------------------------------------------------------------------ */
int64_t oracle_sell_slice_ptr(int32_t n, const int32_t *row_ptr, int32_t S, int64_t *slice_ptr)
{
    int32_t n_slices = (n + S - 1) / S;
    slice_ptr[0] = 0;
    for (int32_t s = 0; s < n_slices; ++s) {
        int32_t w = 0;
        for (int32_t r = s * S; r < (s + 1) * S && r < n; ++r) {
            int32_t len = row_ptr[r + 1] - row_ptr[r];
            if (len > w) w = len;
        }
        slice_ptr[s + 1] = slice_ptr[s] + (int64_t)S * w;
    }
    return slice_ptr[n_slices];
}

void oracle_sell_fill(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                      const double *val, int32_t S, const int64_t *slice_ptr,
                      int32_t *sell_col, double *sell_val)
{
    int32_t n_slices = (n + S - 1) / S;
    for (int32_t s = 0; s < n_slices; ++s) {
        int64_t w = (slice_ptr[s + 1] - slice_ptr[s]) / S;
        for (int32_t lane = 0; lane < S; ++lane) {
            int32_t r = s * S + lane;
            int32_t len = (r < n) ? row_ptr[r + 1] - row_ptr[r] : 0;
            for (int64_t t = 0; t < w; ++t) {
                int64_t at = slice_ptr[s] + t * S + lane;
                if (t < len) {
                    sell_col[at] = col_idx[row_ptr[r] + t];
                    sell_val[at] = val[row_ptr[r] + t];
                } else {
                    sell_col[at] = -1;
                    sell_val[at] = 0.0;
                }
            }
        }
    }
}

/* Per-slice range of the multiplying vector (Sec. 5.1): col_start = smallest column used   */
/* by the slice, col_end = one past the largest; (0, 0) for a slice without entries.  The   */
/* words slice s must add to a window that already holds columns below col_end of the       */
/* previous slice are col_end[s] - col_end[s-1], starting at offset col_end[s-1].           */
void oracle_window_meta(int32_t n, int32_t S, const int64_t *slice_ptr, const int32_t *sell_col,
                        int32_t *col_start, int32_t *col_end)
{
    int32_t n_slices = (n + S - 1) / S;
    for (int32_t s = 0; s < n_slices; ++s) {
        int32_t lo = 0, hi = 0, any = 0;
        for (int64_t at = slice_ptr[s]; at < slice_ptr[s + 1]; ++at) {
            int32_t c = sell_col[at];
            if (c < 0) continue;
            if (!any || c < lo) lo = c;
            if (!any || c + 1 > hi) hi = c + 1;
            any = 1;
        }
        col_start[s] = lo;
        col_end[s] = hi;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Jacobi-preconditioned CG in FP64.                                                        */
/*   r = b - A x0, z = D^-1 r, p = z, rho = r.z                                             */
/*   repeat: q = A p; alpha = rho / (p.q); x += alpha p; r -= alpha q;                      */
/*           stop when ||r||_2 <= rtol ||b||_2 (then recompute r = b - A x and restart the  */
/*           recurrence if the true residual is still above rtol, at most max_restarts);   */
/*           z = D^-1 r; rho' = r.z; beta = rho'/rho; p = z + beta p.                       */
/* Dot products and norms are sequential FP64 sums.  x holds x0 on entry.                   */
/* ------------------------------------------------------------------------------------ */
static double dot64(int32_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double p = a[i] * b[i];
        s = s + p;
    }
    return s;
}

static int diag_inverse(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                        const double *val, double *dinv)
{
    for (int32_t i = 0; i < n; ++i) {
        double d = 0.0;
        int found = 0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            if (col_idx[k] == i) { d = val[k]; found = 1; }
        if (!found || d == 0.0) return -1;
        dinv[i] = 1.0 / d;
    }
    return 0;
}

static void residual64(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                       const double *val, const double *b, const double *x, double *r)
{
    oracle_csr_spmv(n, row_ptr, col_idx, val, x, r, 0);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
}

int oracle_jacobi_pcg(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                      const double *val, const double *b, double *x, double rtol, int32_t max_iter,
                      int32_t max_restarts, int32_t *iters_out, double *relres_out,
                      double *true_relres_out)
{
    double *dinv = (double *)malloc(sizeof(double) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    int rc = 1;
    int32_t it = 0, restarts = 0;
    double bnorm = 0.0, rnorm = 0.0;
    if (n <= 0) {
        if (iters_out) *iters_out = 0;
        if (relres_out) *relres_out = 0.0;
        if (true_relres_out) *true_relres_out = 0.0;
        free(dinv); free(r); free(z); free(p); free(q);
        return n == 0 ? 0 : -1;
    }
    if (!dinv || !r || !z || !p || !q) { rc = -2; goto done; }
    if (diag_inverse(n, row_ptr, col_idx, val, dinv)) { rc = -1; goto done; }
    bnorm = sqrt(dot64(n, b, b));
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
        rc = 0;
        rnorm = 0.0;
        goto done;
    }
    residual64(n, row_ptr, col_idx, val, b, x, r);
    rnorm = sqrt(dot64(n, r, r));
    if (rnorm <= rtol * bnorm) { rc = 0; goto done; }
    for (int32_t i = 0; i < n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
    double rho = dot64(n, r, z);
    while (it < max_iter) {
        oracle_csr_spmv(n, row_ptr, col_idx, val, p, q, 0);
        double alpha = rho / dot64(n, p, q);
        for (int32_t i = 0; i < n; ++i) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * q[i];
        }
        ++it;
        rnorm = sqrt(dot64(n, r, r));
        if (rnorm <= rtol * bnorm) {
            residual64(n, row_ptr, col_idx, val, b, x, r);
            rnorm = sqrt(dot64(n, r, r));
            if (rnorm <= rtol * bnorm) { rc = 0; break; }
            if (restarts >= max_restarts) { rc = 1; break; }
            ++restarts;
            for (int32_t i = 0; i < n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
            rho = dot64(n, r, z);
            continue;
        }
        for (int32_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        double rho_new = dot64(n, r, z);
        double beta = rho_new / rho;
        for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rho = rho_new;
    }
done:
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = (rc >= 0 && bnorm > 0.0) ? rnorm / bnorm : 0.0;
    if (true_relres_out && rc >= 0) {
        if (bnorm > 0.0 && r) {
            residual64(n, row_ptr, col_idx, val, b, x, r);
            *true_relres_out = sqrt(dot64(n, r, r)) / bnorm;
        } else {
            *true_relres_out = 0.0;
        }
    }
    free(dinv); free(r); free(z); free(p); free(q);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Mixed-precision iterative refinement.                                                    */
/*   x = 0; r = b - A x (FP64)                                                              */
/*   repeat while ||r|| > rtol ||b|| and outer < max_outer:                                 */
/*     s = ||r||; solve A32 d = fp32(r / s) by FP32 Jacobi-PCG from d = 0 to inner_rtol     */
/*     (adaptive != 0: to max(inner_rtol, min(0.5, 0.5 rtol ||b|| / ||r||)), the reduction    */
/*     the outer residual still needs with a factor 2 of margin)                            */
/*     (FP32 values = fp32(a_ij), FP32 vectors, FP32 SpMV accumulation, dinv32 = 1/a32_ii); */
/*     x += s * d (FP64); r = b - A x (FP64 values).                                        */
/* Inner dot products are evaluated exactly enough to be the plain definition: the FP32     */
/* operands are multiplied and summed in FP64 and the sum rounded to FP32.                  */
/* ------------------------------------------------------------------------------------ */
static float dot32(int32_t n, const float *a, const float *b)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double p = (double)a[i] * (double)b[i];
        s = s + p;
    }
    return (float)s;
}

static int32_t pcg32(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const float *val,
                     const float *dinv, const float *rhs, float *d, float rtol, int32_t max_iter,
                     float *r, float *z, float *p, float *q)
{
    for (int32_t i = 0; i < n; ++i) { d[i] = 0.0f; r[i] = rhs[i]; z[i] = dinv[i] * r[i]; p[i] = z[i]; }
    float rnorm0 = sqrtf(dot32(n, r, r));
    float rho = dot32(n, r, z);
    int32_t it = 0;
    while (it < max_iter) {
        oracle_csr_spmv_f32(n, row_ptr, col_idx, val, p, q, 1);
        float alpha = rho / dot32(n, p, q);
        for (int32_t i = 0; i < n; ++i) {
            d[i] = d[i] + alpha * p[i];
            r[i] = r[i] - alpha * q[i];
        }
        ++it;
        if (sqrtf(dot32(n, r, r)) <= rtol * rnorm0) break;
        for (int32_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        float rho_new = dot32(n, r, z);
        float beta = rho_new / rho;
        for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rho = rho_new;
    }
    return it;
}

int oracle_mixed_ir(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *val,
                    const double *b, double *x, double rtol, double inner_rtol,
                    int32_t inner_max_iter, int32_t max_outer, int adaptive, int32_t *outer_out,
                    int32_t *inner_total_out, double *relres_out)
{
    int64_t nnz = row_ptr[n];
    float *val32 = (float *)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    double *dinv64 = (double *)malloc(sizeof(double) * (size_t)n);
    float *dinv = (float *)malloc(sizeof(float) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    float *bufs = (float *)malloc(sizeof(float) * (size_t)n * 6);
    int rc = 1;
    int32_t outer = 0, inner_total = 0;
    double bnorm = 0.0, rnorm = 0.0;
    if (n <= 0) {
        if (outer_out) *outer_out = 0;
        if (inner_total_out) *inner_total_out = 0;
        if (relres_out) *relres_out = 0.0;
        free(val32); free(dinv64); free(dinv); free(r); free(bufs);
        return n == 0 ? 0 : -1;
    }
    if (!val32 || !dinv64 || !dinv || !r || !bufs) { rc = -2; goto done; }
    if (diag_inverse(n, row_ptr, col_idx, val, dinv64)) { rc = -1; goto done; }
    for (int64_t k = 0; k < nnz; ++k) val32[k] = (float)val[k];
    for (int32_t i = 0; i < n; ++i) {
        float dd = 0.0f;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            if (col_idx[k] == i) dd = val32[k];
        if (dd == 0.0f) { rc = -1; goto done; }
        dinv[i] = 1.0f / dd;
    }
    float *rhs = bufs, *d = bufs + n, *rr = bufs + 2 * (size_t)n, *z = bufs + 3 * (size_t)n,
          *p = bufs + 4 * (size_t)n, *q = bufs + 5 * (size_t)n;
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    bnorm = sqrt(dot64(n, b, b));
    if (bnorm == 0.0) { rc = 0; goto done; }
    residual64(n, row_ptr, col_idx, val, b, x, r);
    rnorm = sqrt(dot64(n, r, r));
    while (rnorm > rtol * bnorm) {
        if (outer >= max_outer) { rc = 1; goto done; }
        double s = rnorm;
        for (int32_t i = 0; i < n; ++i) rhs[i] = (float)(r[i] / s);
        double tol_in = inner_rtol;
        if (adaptive) {
            double need = 0.5 * rtol * bnorm / rnorm;
            if (need > tol_in) tol_in = need < 0.5 ? need : 0.5;
        }
        inner_total += pcg32(n, row_ptr, col_idx, val32, dinv, rhs, d, (float)tol_in,
                             inner_max_iter, rr, z, p, q);
        for (int32_t i = 0; i < n; ++i) x[i] = x[i] + s * (double)d[i];
        ++outer;
        residual64(n, row_ptr, col_idx, val, b, x, r);
        rnorm = sqrt(dot64(n, r, r));
    }
    rc = 0;
done:
    if (outer_out) *outer_out = outer;
    if (inner_total_out) *inner_total_out = inner_total;
    if (relres_out) *relres_out = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    free(val32); free(dinv64); free(dinv); free(r); free(bufs);
    return rc;
}
