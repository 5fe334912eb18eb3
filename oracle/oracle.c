/*
 * CPU oracle for time-iterated affine star stencils and for the recursive
 * (cache-oblivious) schedule of the PCOT paper (arXiv 1802.00166).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm load this library.  It shares no
 * code with the CUDA library and the CUDA library never calls it.
 *
 * Everything is plain IEEE-754 binary64: every multiply and every add is a
 * separately rounded operation (compiled with -ffp-contract=off, no fast-math),
 * in the fixed operand order stated below.
 *
 * Storage layout: row-major, last axis contiguous.  Dirichlet grids store
 * n_a + 2r entries per axis with a fixed ring of width r; periodic grids store
 * n_a entries per axis and wrap every neighbour index modulo n_a.
 *
 * Coefficient order (1 + 2*dims*r entries): centre, then axis 0 (slowest) to
 * axis dims-1 (fastest), for each axis the offsets -r..-1 then +1..+r.
 *
 * Point update (Sec. 4.2 base function body; Jacobi/heat stencils of Sec. 5.1.2):
 *     acc = c[0]*u[x];  for k = 1..K-1: acc = acc + c[k]*u[x + off_k];
 * Storage across time steps is the two-buffer t%2 scheme of the Appendix A
 * motivating example (Fig. "fig:motiv"): step t reads buffer (t-1)%2 and
 * writes buffer t%2.
 *
 * Parity status: oracle_sweep is pinned by closed forms (Fourier-mode decay,
 * Dirichlet sine modes, FFT convolution with asymmetric coefficients, sum
 * conservation, fixed points, hand-derived steps).  oracle_pcot is pinned by
 * bitwise equality with oracle_sweep on brute-forced tiny problems, and
 * oracle_orthant_empty by brute-force enumeration of orthant points.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 3

typedef struct {
    int dims, r, periodic;
    int64_t n[OR_MAXD];      /* interior sizes */
    int64_t e[OR_MAXD];      /* stored extents */
    int64_t stride[OR_MAXD]; /* element strides of the storage */
    int64_t total;           /* stored elements */
    const double *c;
    int ncoef;
} or_geom;

static int or_setup(or_geom *g, int dims, int r, const int64_t *n, int periodic,
                    const double *coeffs)
{
    if (dims < 1 || dims > OR_MAXD || r < 1 || !n || !coeffs) return -1;
    g->dims = dims;
    g->r = r;
    g->periodic = periodic ? 1 : 0;
    g->c = coeffs;
    g->ncoef = 1 + 2 * dims * r;
    for (int a = 0; a < dims; ++a) {
        if (n[a] < 1) return -1;
        if (periodic && n[a] < r) return -1;
        g->n[a] = n[a];
        g->e[a] = periodic ? n[a] : n[a] + 2 * r;
    }
    int64_t s = 1;
    for (int a = dims - 1; a >= 0; --a) {
        g->stride[a] = s;
        s *= g->e[a];
    }
    g->total = s;
    return 0;
}

/* One point: interior coordinates i[] (0-based), reading src, returns the new value. */
static double or_point(const or_geom *g, const int64_t *i, const double *src)
{
    int64_t s = 0;
    for (int a = 0; a < g->dims; ++a)
        s += (g->periodic ? i[a] : i[a] + g->r) * g->stride[a];
    double acc = g->c[0] * src[s];
    int k = 1;
    for (int a = 0; a < g->dims; ++a) {
        for (int pass = 0; pass < 2; ++pass) {
            for (int q = 1; q <= g->r; ++q) {
                /* pass 0: offsets -r..-1 ; pass 1: offsets +1..+r */
                int64_t o = pass == 0 ? (int64_t)(q - g->r - 1) : (int64_t)q;
                int64_t nb;
                if (g->periodic) {
                    int64_t j = i[a] + o;
                    j %= g->n[a];
                    if (j < 0) j += g->n[a];
                    nb = s + (j - i[a]) * g->stride[a];
                } else {
                    nb = s + o * g->stride[a];
                }
                acc = acc + g->c[k] * src[nb];
                ++k;
            }
        }
    }
    return acc;
}

/*
 * Naive sweep: T steps of the point update over every interior point, in
 * row-major order, two buffers.  `grid` (storage layout) is read as the
 * initial state and overwritten with the state after T steps.
 * nthreads: 0 = OpenMP default; the outermost axis is split across threads,
 * which does not change any value (each point is computed independently).
 */
int oracle_sweep(int dims, int r, const int64_t *n, int periodic,
                 const double *coeffs, int64_t T, double *grid, int nthreads)
{
    or_geom g;
    if (or_setup(&g, dims, r, n, periodic, coeffs) != 0 || T < 0 || !grid) return -1;
    if (T == 0) return 0;
    double *buf = (double *)malloc(sizeof(double) * (size_t)g.total);
    if (!buf) return -2;
    memcpy(buf, grid, sizeof(double) * (size_t)g.total); /* ring values in both buffers */
    double *A = grid, *B = buf;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const int64_t n0 = g.n[0];
    const int64_t n1 = dims > 1 ? g.n[1] : 1;
    const int64_t n2 = dims > 2 ? g.n[2] : 1;
    for (int64_t t = 1; t <= T; ++t) {
#pragma omp parallel for schedule(static)
        for (int64_t i0 = 0; i0 < n0; ++i0) {
            int64_t i[OR_MAXD] = {i0, 0, 0};
            for (int64_t i1 = 0; i1 < n1; ++i1) {
                for (int64_t i2 = 0; i2 < n2; ++i2) {
                    if (dims > 1) i[1] = i1;
                    if (dims > 2) i[2] = i2;
                    int64_t s = 0;
                    for (int a = 0; a < dims; ++a)
                        s += (g.periodic ? i[a] : i[a] + g.r) * g.stride[a];
                    B[s] = or_point(&g, i, A);
                }
            }
        }
        double *tmp = A; A = B; B = tmp;
    }
    if (A != grid) memcpy(grid, A, sizeof(double) * (size_t)g.total);
    free(buf);
    return 0;
}

/* ------------------------------------------------------------------------
 * PCOT recursive executor (Sec. 4.1-4.5), Dirichlet boundaries only.
 *
 * Iteration space after time skewing (Sec. 4.3.2 mentions the skew that makes
 * Heat2D tilable; the map (t,i) -> (t, i + t) of Appendix A, with factor r):
 *     D = { (t, x'_0..x'_{d-1}) : 1 <= t <= T,  r*t <= x'_a <= r*t + n_a - 1 }
 * where x'_a = i_a + r*t and i_a is the 0-based interior coordinate.
 * Dimension 0 of the skewed space is time; dimension a+1 is spatial axis a.
 * ------------------------------------------------------------------------ */

typedef struct {
    or_geom g;
    int D;                   /* dims + 1 */
    int64_t T;
    int64_t leaf[OR_MAXD + 1];
    double *X[2];
    int64_t stats[6];        /* recursive calls, base calls, zero exits, empty exits, points, max depth */
    int64_t *record;         /* when set: base loops record (t, i_0..i_{d-1}) instead of computing */
    int64_t record_cap;
} or_pcot;

/* Bounding box of D (Sec. 4.5): eliminating t from r t <= x'_a <= r t + n_a - 1
 * over 1 <= t <= T gives x'_a in [r, r T + n_a - 1]. */
static void or_bbox(const or_geom *g, int64_t T, int64_t *lo, int64_t *size)
{
    lo[0] = 1;
    size[0] = T;
    for (int a = 0; a < g->dims; ++a) {
        lo[a + 1] = g->r;
        size[a + 1] = g->r * T + g->n[a] - 1 - g->r + 1;
    }
}

/* Padding of Sec. 4.5: the least b * 2^k >= N (k >= 0). */
static int64_t or_pad(int64_t N, int64_t b, int *levels)
{
    int64_t s = b;
    int k = 0;
    while (s < N) { s *= 2; ++k; }
    if (levels) *levels = k;
    return s;
}

static int64_t or_floordiv(int64_t a, int64_t b) { int64_t q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) --q; return q; }
static int64_t or_ceildiv(int64_t a, int64_t b) { return -or_floordiv(-a, b); }

/*
 * checkEmpty of Sec. 4.3: an orthant is skipped when any width is zero
 * (Sec. 4.3.1) or when it holds no point of D (Sec. 4.3.2).  The emptiness
 * test is exact: for spatial axis a the orthant meets the constraint band
 * r t <= x'_a <= r t + n_a - 1 at time t iff
 *     ceil((lo_a - n_a + 1)/r) <= t <= floor(hi_a / r),
 * and the axes share t, so the orthant is non-empty iff the intersection of
 * these intervals with [t_lo, t_hi] and [1, T] is non-empty.
 * Returns 1 for zero width, 2 for empty, 0 otherwise.
 */
static int or_check_empty(const or_geom *g, int64_t T, const int64_t *lo, const int64_t *size)
{
    const int D = g->dims + 1;
    for (int i = 0; i < D; ++i)
        if (size[i] <= 0) return 1;
    int64_t tl = lo[0] > 1 ? lo[0] : 1;
    int64_t th = lo[0] + size[0] - 1;
    if (th > T) th = T;
    for (int a = 0; a < g->dims; ++a) {
        int64_t l = lo[a + 1], h = lo[a + 1] + size[a + 1] - 1;
        int64_t a_lo = or_ceildiv(l - g->n[a] + 1, g->r);
        int64_t a_hi = or_floordiv(h, g->r);
        if (a_lo > tl) tl = a_lo;
        if (a_hi < th) th = a_hi;
    }
    return tl > th ? 2 : 0;
}

/* Base function (Sec. 4.2): lexicographic point loops over leaf ∩ D. */
static void or_base(or_pcot *p, const int64_t *lo, const int64_t *size)
{
    const or_geom *g = &p->g;
    int64_t t0 = lo[0] > 1 ? lo[0] : 1;
    int64_t t1 = lo[0] + size[0] - 1;
    if (t1 > p->T) t1 = p->T;
    for (int64_t t = t0; t <= t1; ++t) {
        int64_t xl[OR_MAXD], xh[OR_MAXD];
        int any = 1;
        for (int a = 0; a < g->dims; ++a) {
            xl[a] = lo[a + 1] > g->r * t ? lo[a + 1] : g->r * t;
            xh[a] = lo[a + 1] + size[a + 1] - 1;
            if (xh[a] > g->r * t + g->n[a] - 1) xh[a] = g->r * t + g->n[a] - 1;
            if (xl[a] > xh[a]) any = 0;
        }
        if (!any) continue;
        const double *src = p->X[(t - 1) % 2];
        double *dst = p->X[t % 2];
        (void)src;
        (void)dst;
        int64_t x[OR_MAXD];
        for (int a = 0; a < g->dims; ++a) x[a] = xl[a];
        for (;;) {
            int64_t i[OR_MAXD];
            int64_t s = 0;
            for (int a = 0; a < g->dims; ++a) {
                i[a] = x[a] - g->r * t;
                s += (i[a] + g->r) * g->stride[a];
            }
            if (p->record) {
                int64_t k = p->stats[4];
                if (k < p->record_cap) {
                    p->record[k * (g->dims + 1)] = t;
                    for (int a = 0; a < g->dims; ++a) p->record[k * (g->dims + 1) + 1 + a] = i[a];
                }
            } else {
                dst[s] = or_point(g, i, src);
            }
            p->stats[4]++;
            int a = g->dims - 1;
            while (a >= 0) {
                if (++x[a] <= xh[a]) break;
                x[a] = xl[a];
                --a;
            }
            if (a < 0) break;
        }
    }
}

/* Recursive function (Sec. 4.2): halve every dimension wider than its leaf
 * size, visit the 2^D orthants in lexicographic order (time bit most
 * significant).  A dimension already at or below its leaf size is given to
 * the first child whole and the second child gets width 0 (the zero orthants
 * of Sec. 4.3.1). */
static void or_recurse(or_pcot *p, const int64_t *lo, const int64_t *size, int depth)
{
    p->stats[0]++;
    if (depth > p->stats[5]) p->stats[5] = depth;
    int e = or_check_empty(&p->g, p->T, lo, size);
    if (e == 1) { p->stats[2]++; return; }
    if (e == 2) { p->stats[3]++; return; }
    int leaf = 1;
    for (int i = 0; i < p->D; ++i)
        if (size[i] > p->leaf[i]) leaf = 0;
    if (leaf) {
        p->stats[1]++;
        or_base(p, lo, size);
        return;
    }
    const int nchild = 1 << p->D;
    for (int c = 0; c < nchild; ++c) {
        int64_t clo[OR_MAXD + 1], csz[OR_MAXD + 1];
        for (int i = 0; i < p->D; ++i) {
            int bit = (c >> (p->D - 1 - i)) & 1;
            if (size[i] > p->leaf[i]) {
                int64_t h0 = size[i] / 2;
                int64_t h1 = size[i] - h0;
                clo[i] = lo[i] + (bit ? h0 : 0);
                csz[i] = bit ? h1 : h0;
            } else {
                clo[i] = lo[i];
                csz[i] = bit ? 0 : size[i];
            }
        }
        or_recurse(p, clo, csz, depth + 1);
    }
}

/*
 * Run T steps with the PCOT recursion.  leaf[0] is the time extent of a leaf
 * orthant, leaf[1+a] its extent along skewed axis a.  `stats` (6 entries, may
 * be NULL) receives: recursive calls, base calls, zero-orthant exits,
 * empty-orthant exits, points computed, maximum recursion depth.
 */
int oracle_pcot(int dims, int r, const int64_t *n, const double *coeffs, int64_t T,
                const int64_t *leaf, double *grid, int64_t *stats)
{
    or_pcot p;
    memset(&p, 0, sizeof(p));
    if (or_setup(&p.g, dims, r, n, 0, coeffs) != 0 || T < 0 || !grid || !leaf) return -1;
    p.D = dims + 1;
    p.T = T;
    for (int i = 0; i < p.D; ++i) {
        if (leaf[i] < 1) return -1;
        p.leaf[i] = leaf[i];
    }
    if (T > 0) {
        double *buf = (double *)malloc(sizeof(double) * (size_t)p.g.total);
        if (!buf) return -2;
        memcpy(buf, grid, sizeof(double) * (size_t)p.g.total);
        p.X[0] = grid;
        p.X[1] = buf;
        int64_t lo[OR_MAXD + 1], size[OR_MAXD + 1];
        or_bbox(&p.g, T, lo, size);
        for (int i = 0; i < p.D; ++i) size[i] = or_pad(size[i], p.leaf[i], NULL);
        or_recurse(&p, lo, size, 0);
        if (T % 2 == 1) memcpy(grid, buf, sizeof(double) * (size_t)p.g.total);
        free(buf);
    }
    if (stats) memcpy(stats, p.stats, sizeof(p.stats));
    return 0;
}

/* Exposed for tests: the padded bounding box (origin, size, levels k_i). */
int oracle_padded_box(int dims, int r, const int64_t *n, int64_t T, const int64_t *leaf,
                      int64_t *lo, int64_t *size, int32_t *levels)
{
    or_geom g;
    double dummy = 0.0;
    double cdummy[1 + 2 * OR_MAXD * 8];
    (void)dummy;
    memset(cdummy, 0, sizeof(cdummy));
    if (r > 8 || or_setup(&g, dims, r, n, 0, cdummy) != 0 || T < 1) return -1;
    or_bbox(&g, T, lo, size);
    for (int i = 0; i <= dims; ++i) {
        int k = 0;
        size[i] = or_pad(size[i], leaf[i], &k);
        if (levels) levels[i] = k;
    }
    return 0;
}

/* Exposed for tests: the checkEmpty result for one orthant (0, 1 = zero width, 2 = empty). */
int oracle_orthant_empty(int dims, int r, const int64_t *n, int64_t T,
                         const int64_t *lo, const int64_t *size)
{
    or_geom g;
    double cdummy[1 + 2 * OR_MAXD * 8];
    memset(cdummy, 0, sizeof(cdummy));
    if (r > 8 || or_setup(&g, dims, r, n, 0, cdummy) != 0) return -1;
    return or_check_empty(&g, T, lo, size);
}

/*
 * Visit order of the recursion: the points (t, i_0..i_{d-1}) in the order the
 * base function reaches them (same recursion as oracle_pcot, nothing computed).
 * `out` receives up to `cap` records of dims+1 int64 each; returns the number
 * of points of the domain (which may exceed cap), or -1 on bad arguments.
 */
int64_t oracle_pcot_order(int dims, int r, const int64_t *n, int64_t T, const int64_t *leaf,
                          int64_t *out, int64_t cap)
{
    or_pcot p;
    double cdummy[1 + 2 * OR_MAXD * 8];
    memset(&p, 0, sizeof(p));
    memset(cdummy, 0, sizeof(cdummy));
    if (r > 8 || or_setup(&p.g, dims, r, n, 0, cdummy) != 0 || T < 0 || !leaf) return -1;
    p.D = dims + 1;
    p.T = T;
    for (int i = 0; i < p.D; ++i) {
        if (leaf[i] < 1) return -1;
        p.leaf[i] = leaf[i];
    }
    p.record = out;
    p.record_cap = out ? cap : 0;
    if (!out) { static int64_t sink[OR_MAXD + 1]; p.record = sink; p.record_cap = 0; }
    if (T > 0) {
        int64_t lo[OR_MAXD + 1], size[OR_MAXD + 1];
        or_bbox(&p.g, T, lo, size);
        for (int i = 0; i < p.D; ++i) size[i] = or_pad(size[i], p.leaf[i], NULL);
        or_recurse(&p, lo, size, 0);
    }
    return p.stats[4];
}
