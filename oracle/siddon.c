/*
 * FP64 CPU oracle for the system matrix A = M R of the parallel-beam Radon
 * transform restricted to the measured angles (Sec. 1, Eq. objmin: M keeps the
 * angles along which data are taken; R is the Radon transform).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load it.  It shares no code with the CUDA
 * library.
 *
 * The paper gives no image-domain discretisation of R; the entries here are
 * the exact intersection lengths of each ray with each pixel, computed with
 * Siddon's method (R. L. Siddon, Med. Phys. 12(2), 1985): the parameters at
 * which the ray crosses the vertical and the horizontal grid lines are two
 * sorted lists; merging them splits the ray into segments, one per pixel, and
 * the pixel of a segment is the one containing its midpoint.
 *
 * Geometry (one reading, shared by every part of the project):
 *   image N x N, pixel (i,j) covers x in [j-N/2, j-N/2+1], y in [i-N/2, i-N/2+1],
 *   column index p = i*N + j;
 *   theta_k = k*pi/n_total, k = 0..n_total-1, kept when k % keep_every == 0;
 *   bin b sits at offset s_b = b - (n_bins-1)/2, width 1;
 *   ray (k,b) is the line { x : x*cos(theta_k) + y*sin(theta_k) = s_b };
 *   row index q = (k/keep_every)*n_bins + b.
 * Readings where the paper is silent:
 *   - theta exactly 0 or pi/2 use the exact direction cosines (1,0) / (0,1);
 *   - a ray lying exactly on a grid line gives half of its length to each of
 *     the two pixels sharing that edge (half to the single inside pixel on
 *     the outer boundary);
 *   - segments shorter than 1e-12 are dropped.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MIN_LEN 1e-12
#define ORACLE_PI 3.14159265358979323846

typedef struct {
    int32_t col;
    double val;
} oracle_entry;

static void oracle_direction(int k, int n_total, double *c, double *s)
{
    if (k == 0) {
        *c = 1.0;
        *s = 0.0;
    } else if (2 * k == n_total) {
        *c = 0.0;
        *s = 1.0;
    } else {
        double th = (double)k * ORACLE_PI / (double)n_total;
        *c = cos(th);
        *s = sin(th);
    }
}

static int cmp_entry(const void *a, const void *b)
{
    const oracle_entry *x = (const oracle_entry *)a, *y = (const oracle_entry *)b;
    return (x->col > y->col) - (x->col < y->col);
}

/* Sorts the entries of one ray by pixel and merges repeats; returns the count. */
static int finish_row(oracle_entry *e, int n)
{
    if (n <= 1) return n;
    qsort(e, (size_t)n, sizeof(oracle_entry), cmp_entry);
    int m = 0;
    for (int t = 0; t < n; ++t) {
        if (m > 0 && e[m - 1].col == e[t].col)
            e[m - 1].val += e[t].val;
        else
            e[m++] = e[t];
    }
    return m;
}

/* Parameters at which the line x(t) = x0 + t*dx meets the planes
 * P_m = m - N/2, m = 0..N, written in ascending order into out[]. */
static int plane_params(int n, double x0, double dx, double *out)
{
    for (int m = 0; m <= n; ++m) out[m] = ((double)m - 0.5 * n - x0) / dx;
    if (dx < 0) {
        for (int a = 0, b = n; a < b; ++a, --b) {
            double t = out[a];
            out[a] = out[b];
            out[b] = t;
        }
    }
    return n + 1;
}

/* Traces one ray; writes its (pixel, length) pairs into e[] (capacity >= 3N+4). */
static int trace_ray(int n, double c, double s, double sb, oracle_entry *e,
                     double *tx, double *ty)
{
    const double half = 0.5 * n;
    /* point on the line closest to the origin, and the unit direction */
    const double x0 = sb * c, y0 = sb * s;
    const double dx = -s, dy = c;
    int cnt = 0;

    if (dx == 0.0 || dy == 0.0) {
        /* axis-aligned ray: constant coordinate v along the fixed axis */
        const int vertical = (dx == 0.0); /* x constant */
        const double v = vertical ? x0 : y0;
        if (v < -half || v > half) return 0;
        const double e_coord = v + half; /* in [0, N] */
        if (e_coord == floor(e_coord)) {
            const int m = (int)e_coord; /* lies on grid line m: cells m-1 and m */
            for (int t = 0; t < n; ++t) {
                for (int cell = m - 1; cell <= m; ++cell) {
                    if (cell < 0 || cell >= n) continue;
                    const int i = vertical ? t : cell;
                    const int j = vertical ? cell : t;
                    e[cnt].col = i * n + j;
                    e[cnt].val = 0.5;
                    ++cnt;
                }
            }
            return finish_row(e, cnt);
        }
        /* otherwise the general merge below handles it with one plane list */
    }

    /* entry/exit parameters of the box [-N/2, N/2]^2 */
    double tlo = -INFINITY, thi = INFINITY;
    int nx = 0, ny = 0;
    if (dx != 0.0) {
        nx = plane_params(n, x0, dx, tx);
        if (tx[0] > tlo) tlo = tx[0];
        if (tx[nx - 1] < thi) thi = tx[nx - 1];
    }
    if (dy != 0.0) {
        ny = plane_params(n, y0, dy, ty);
        if (ty[0] > tlo) tlo = ty[0];
        if (ty[ny - 1] < thi) thi = ty[ny - 1];
    }
    if (!(thi > tlo)) return 0;

    /* merge both sorted lists restricted to (tlo, thi), bracketed by tlo, thi */
    int a = 0, b = 0;
    while (a < nx && tx[a] <= tlo) ++a;
    while (b < ny && ty[b] <= tlo) ++b;
    double prev = tlo;
    for (;;) {
        double next;
        if (a < nx && tx[a] < thi && (b >= ny || ty[b] >= thi || tx[a] <= ty[b]))
            next = tx[a++];
        else if (b < ny && ty[b] < thi)
            next = ty[b++];
        else
            next = thi;
        const double len = next - prev;
        if (len >= ORACLE_MIN_LEN) {
            const double tm = 0.5 * (prev + next);
            int j = (int)floor(x0 + tm * dx + half);
            int i = (int)floor(y0 + tm * dy + half);
            if (j < 0) j = 0;
            if (j > n - 1) j = n - 1;
            if (i < 0) i = 0;
            if (i > n - 1) i = n - 1;
            e[cnt].col = i * n + j;
            e[cnt].val = len;
            ++cnt;
        }
        prev = next;
        if (next >= thi) break;
    }
    return finish_row(e, cnt);
}

static int check_geometry(int n, int n_total, int keep_every, int n_bins)
{
    if (n <= 0 || n_total <= 0 || keep_every <= 0 || n_bins <= 0) return -1;
    if ((int64_t)n * n > INT32_MAX) return -1;
    return 0;
}

int oracle_num_kept(int n_total, int keep_every)
{
    return (n_total + keep_every - 1) / keep_every;
}

/* Pass 1: number of entries of every row; returns the total, or -1. */
int64_t oracle_siddon_count(int n, int n_total, int keep_every, int n_bins,
                            int64_t *row_nnz)
{
    if (check_geometry(n, n_total, keep_every, n_bins)) return -1;
    oracle_entry *e = (oracle_entry *)malloc(sizeof(oracle_entry) * (size_t)(3 * n + 8) * 2);
    double *tx = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *ty = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (!e || !tx || !ty) {
        free(e);
        free(tx);
        free(ty);
        return -1;
    }
    int64_t total = 0;
    const int n_kept = oracle_num_kept(n_total, keep_every);
    for (int kk = 0; kk < n_kept; ++kk) {
        double c, s;
        oracle_direction(kk * keep_every, n_total, &c, &s);
        for (int b = 0; b < n_bins; ++b) {
            const double sb = (double)b - 0.5 * (double)(n_bins - 1);
            const int m = trace_ray(n, c, s, sb, e, tx, ty);
            row_nnz[(int64_t)kk * n_bins + b] = m;
            total += m;
        }
    }
    free(e);
    free(tx);
    free(ty);
    return total;
}

/* Pass 2: fills cols/vals of a CSR whose row_ptr was built from pass 1. */
int oracle_siddon_fill(int n, int n_total, int keep_every, int n_bins,
                       const int64_t *row_ptr, int32_t *cols, double *vals)
{
    if (check_geometry(n, n_total, keep_every, n_bins)) return -1;
    oracle_entry *e = (oracle_entry *)malloc(sizeof(oracle_entry) * (size_t)(3 * n + 8) * 2);
    double *tx = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *ty = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (!e || !tx || !ty) {
        free(e);
        free(tx);
        free(ty);
        return -1;
    }
    const int n_kept = oracle_num_kept(n_total, keep_every);
    int rc = 0;
    for (int kk = 0; kk < n_kept && rc == 0; ++kk) {
        double c, s;
        oracle_direction(kk * keep_every, n_total, &c, &s);
        for (int b = 0; b < n_bins; ++b) {
            const double sb = (double)b - 0.5 * (double)(n_bins - 1);
            const int m = trace_ray(n, c, s, sb, e, tx, ty);
            const int64_t q = (int64_t)kk * n_bins + b;
            if (row_ptr[q + 1] - row_ptr[q] != m) {
                rc = -2;
                break;
            }
            for (int t = 0; t < m; ++t) {
                cols[row_ptr[q] + t] = e[t].col;
                vals[row_ptr[q] + t] = e[t].val;
            }
        }
    }
    free(e);
    free(tx);
    free(ty);
    return rc;
}

/* The listed rays only (row indices q = kept angle * n_bins + bin), for
 * checking matrices too large to build whole.  Pass 1 (cols == NULL): writes
 * row_nnz[r], the entries of ray rows[r], and returns their total.  Pass 2:
 * writes each ray's entries at row_ptr[r] of cols/vals.  Returns -1 on an
 * invalid geometry or row, -2 if a ray's count differs from row_ptr. */
int64_t oracle_siddon_rows(int n, int n_total, int keep_every, int n_bins, int64_t nrows,
                           const int64_t *rows, const int64_t *row_ptr, int64_t *row_nnz,
                           int32_t *cols, double *vals)
{
    if (check_geometry(n, n_total, keep_every, n_bins)) return -1;
    const int n_kept = oracle_num_kept(n_total, keep_every);
    oracle_entry *e = (oracle_entry *)malloc(sizeof(oracle_entry) * (size_t)(3 * n + 8) * 2);
    double *tx = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *ty = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (!e || !tx || !ty) {
        free(e);
        free(tx);
        free(ty);
        return -1;
    }
    int64_t total = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t q = rows[r];
        if (q < 0 || q >= (int64_t)n_kept * n_bins) {
            total = -1;
            break;
        }
        const int kk = (int)(q / n_bins), b = (int)(q % n_bins);
        double c, s;
        oracle_direction(kk * keep_every, n_total, &c, &s);
        const double sb = (double)b - 0.5 * (double)(n_bins - 1);
        const int m = trace_ray(n, c, s, sb, e, tx, ty);
        if (!cols) {
            row_nnz[r] = m;
        } else {
            if (row_ptr[r + 1] - row_ptr[r] != m) {
                total = -2;
                break;
            }
            for (int t = 0; t < m; ++t) {
                cols[row_ptr[r] + t] = e[t].col;
                vals[row_ptr[r] + t] = e[t].val;
            }
        }
        total += m;
    }
    free(e);
    free(tx);
    free(ty);
    return total;
}

/* Direction cosines of every kept angle (for tests of the angle reading). */
void oracle_directions(int n_total, int keep_every, double *cs, double *sn)
{
    const int n_kept = oracle_num_kept(n_total, keep_every);
    for (int kk = 0; kk < n_kept; ++kk)
        oracle_direction(kk * keep_every, n_total, &cs[kk], &sn[kk]);
}
