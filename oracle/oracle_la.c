/*
 * CPU oracle for the two linear-algebra kernels of the PCOT paper's benchmark
 * suite (Sec. 5.1.2: Cholesky decomposition and LU decomposition), whose
 * iteration spaces are not boxes: the recursion over their bounding box
 * meets empty orthants (Sec. 4.3, early exit for empty orthants).
 *
 * TEST INFRASTRUCTURE ONLY.  Loaded by the test-suite and the benchmark's
 * CPU-baseline arm together with oracle.c; shares no code with the CUDA
 * library, which never calls it.
 *
 * Matrix: n x n binary64 values, row-major with row stride lda >= n, factored
 * in place.  Every update is c <- c - a*b, evaluated either as a rounded
 * product followed by a rounded subtraction (fma = 0) or as one fused
 * multiply-add, fma(-a, b, c) (fma = 1); divisions and square roots are the
 * correctly rounded IEEE-754 operations.
 *
 * LU (Gaussian elimination without pivoting, unit lower L below the
 * diagonal, U on and above it).  For k = 0 .. n-1:
 *   S1(k, i):    A[i][k] = A[i][k] / A[k][k]                  (i > k)
 *   S2(k, i, j): A[i][j] = A[i][j] - A[i][k] * A[k][j]        (i > k, j > k)
 * Cholesky (lower triangle; the strict upper triangle is neither read nor
 * written).  For k = 0 .. n-1:
 *   S0(k):       A[k][k] = sqrt(A[k][k])
 *   S1(k, i):    A[i][k] = A[i][k] / A[k][k]                  (i > k)
 *   S2(k, i, j): A[i][j] = A[i][j] - A[i][k] * A[j][k]        (k < j <= i)
 * Any loop order that respects the dependences applies to each element the
 * same operations in the same order, so every correct schedule is bitwise
 * equal to these loops.
 *
 * Recursive schedule (Sec. 4 applied to these loop nests).  The statements
 * live in one three-dimensional space (k, i, j): S2(k, i, j) at (k, i, j),
 * S1(k, i) at (k, i, k) and S0(k) at (k, k, k).  The domains are
 *   LU:       0 <= k < i < n,  k <= j < n
 *   Cholesky: 0 <= k <= j <= i < n
 * and every dependence has non-negative components (an update waits for the
 * same element at k-1, for the multipliers of its row at the same (k, i)
 * with a smaller j, and for row k or row j of the same k), so the space needs
 * no skew: its bounding box [0, n)^3 is padded to leaf_d * 2^m_d, split into
 * 2^3 orthants (a width above the leaf is halved, one at or below goes whole
 * to the lower child and leaves a zero-width upper child), orthants are
 * visited in lexicographic order with k most significant, zero-width and
 * empty orthants return at once, and a leaf box runs its domain points in
 * lexicographic (k, i, j) order.
 *
 * Emptiness of an inclusive box [k0,k1] x [i0,i1] x [j0,j1]: within each
 * domain, decreasing k only widens the admissible i and j, so the box holds a
 * point iff its smallest admissible k, k* = max(k0, 0) <= k1, does:
 *   LU:       max(i0, k*+1) <= min(i1, n-1)  and  max(j0, k*) <= min(j1, n-1)
 *   Cholesky: j* = max(j0, k*) <= min(j1, n-1)  and  max(i0, j*) <= min(i1, n-1)
 *
 * Tile order (the order the GPU planner must reproduce): the same recursion
 * over the lattice of b x b x b tiles (tile (kb, ib, jb) holds the points
 * with k in [kb b, kb b + b) and likewise for i, j), a tile counting as empty
 * when it holds no domain point; children by the number of upper halves
 * they take (orthants with equal counts are independent: the wavefronts of
 * the paper's parallel recursion), ties lexicographic with k most
 * significant; leaves list their tiles lexicographically.  The single-level
 * order lists all non-empty tiles lexicographically.
 *
 * Parity status: oracle_lu and oracle_cholesky are pinned by exact
 * factorizations of integer matrices built as L*U and L*L^T, by agreement
 * with library factorizations within the backward-error bound, and by a
 * worked 3 x 3 example (tests/golden/la_steps.txt).  oracle_la_pcot is pinned
 * by bitwise equality with the plain loops on brute-forced small sizes, and
 * oracle_la_box_empty by point enumeration.
 */
#include <math.h>
#include <stdint.h>

static double la_upd(double c, double a, double b, int fused)
{
    if (fused) return fma(-a, b, c);
    const double p = a * b;
    return c - p;
}

int oracle_lu(int64_t n, int64_t lda, double *A, int fused)
{
    if (n < 0 || lda < n || (n > 0 && !A)) return -1;
    for (int64_t k = 0; k < n; ++k) {
        for (int64_t i = k + 1; i < n; ++i) A[i * lda + k] = A[i * lda + k] / A[k * lda + k];
        for (int64_t i = k + 1; i < n; ++i)
            for (int64_t j = k + 1; j < n; ++j)
                A[i * lda + j] = la_upd(A[i * lda + j], A[i * lda + k], A[k * lda + j], fused);
    }
    return 0;
}

int oracle_cholesky(int64_t n, int64_t lda, double *A, int fused)
{
    if (n < 0 || lda < n || (n > 0 && !A)) return -1;
    for (int64_t k = 0; k < n; ++k) {
        A[k * lda + k] = sqrt(A[k * lda + k]);
        for (int64_t i = k + 1; i < n; ++i) A[i * lda + k] = A[i * lda + k] / A[k * lda + k];
        for (int64_t i = k + 1; i < n; ++i)
            for (int64_t j = k + 1; j <= i; ++j)
                A[i * lda + j] = la_upd(A[i * lda + j], A[i * lda + k], A[j * lda + k], fused);
    }
    return 0;
}

static int64_t la_max(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t la_min(int64_t a, int64_t b) { return a < b ? a : b; }

/* kind 0 = LU, 1 = Cholesky.  1 if the inclusive box holds no domain point. */
int oracle_la_box_empty(int kind, int64_t n, const int64_t *lo, const int64_t *hi)
{
    const int64_t ks = la_max(lo[0], 0);
    if (ks > hi[0]) return 1;
    if (kind == 0) {
        if (la_max(lo[1], ks + 1) > la_min(hi[1], n - 1)) return 1;
        if (la_max(lo[2], ks) > la_min(hi[2], n - 1)) return 1;
        return 0;
    }
    const int64_t js = la_max(lo[2], ks);
    if (js > la_min(hi[2], n - 1)) return 1;
    if (la_max(lo[1], js) > la_min(hi[1], n - 1)) return 1;
    return 0;
}

/* 1 if (k, i, j) is a point of the domain. */
static int la_in_domain(int kind, int64_t n, int64_t k, int64_t i, int64_t j)
{
    if (k < 0 || i >= n || j >= n) return 0;
    if (kind == 0) return k < i && k <= j;
    return k <= j && j <= i;
}

/* The statement at domain point (k, i, j). */
static void la_point(int kind, int64_t lda, double *A, int fused, int64_t k, int64_t i, int64_t j)
{
    if (kind == 0) {
        if (j == k)
            A[i * lda + k] = A[i * lda + k] / A[k * lda + k];
        else
            A[i * lda + j] = la_upd(A[i * lda + j], A[i * lda + k], A[k * lda + j], fused);
        return;
    }
    if (j == k) {
        if (i == k)
            A[k * lda + k] = sqrt(A[k * lda + k]);
        else
            A[i * lda + k] = A[i * lda + k] / A[k * lda + k];
    } else {
        A[i * lda + j] = la_upd(A[i * lda + j], A[i * lda + k], A[j * lda + k], fused);
    }
}

typedef struct {
    int kind, fused;
    int64_t n, lda;
    double *A;
    int64_t leaf[3];
    int64_t leaves, zero_exits, empty_exits, points;
} la_pcot;

static void la_recurse(la_pcot *p, const int64_t *lo, const int64_t *size)
{
    for (int d = 0; d < 3; ++d)
        if (size[d] == 0) {
            ++p->zero_exits;
            return;
        }
    int64_t hi[3];
    for (int d = 0; d < 3; ++d) hi[d] = lo[d] + size[d] - 1;
    if (oracle_la_box_empty(p->kind, p->n, lo, hi)) {
        ++p->empty_exits;
        return;
    }
    int base = 1;
    for (int d = 0; d < 3; ++d)
        if (size[d] > p->leaf[d]) base = 0;
    if (base) {
        ++p->leaves;
        for (int64_t k = lo[0]; k <= hi[0]; ++k)
            for (int64_t i = lo[1]; i <= hi[1]; ++i)
                for (int64_t j = lo[2]; j <= hi[2]; ++j)
                    if (la_in_domain(p->kind, p->n, k, i, j)) {
                        la_point(p->kind, p->lda, p->A, p->fused, k, i, j);
                        ++p->points;
                    }
        return;
    }
    int64_t half[3][2];
    for (int d = 0; d < 3; ++d) {
        if (size[d] > p->leaf[d]) {
            half[d][0] = size[d] / 2;
            half[d][1] = size[d] - size[d] / 2;
        } else {
            half[d][0] = size[d];
            half[d][1] = 0;
        }
    }
    for (int m = 0; m < 8; ++m) { /* bit 2 = k (most significant), bit 0 = j */
        int64_t clo[3], csz[3];
        for (int d = 0; d < 3; ++d) {
            const int bit = (m >> (2 - d)) & 1;
            clo[d] = lo[d] + (bit ? half[d][0] : 0);
            csz[d] = half[d][bit];
        }
        la_recurse(p, clo, csz);
    }
}

static int64_t la_pad(int64_t N, int64_t b)
{
    int64_t w = b;
    while (w < N) w *= 2;
    return w;
}

/* The factorization in the recursive order; stats (may be NULL) receives
 * {leaves, zero exits, empty exits, points}. */
int oracle_la_pcot(int kind, int64_t n, int64_t lda, double *A, int fused, const int64_t *leaf, int64_t *stats)
{
    if ((kind != 0 && kind != 1) || n < 0 || lda < n || (n > 0 && !A) || !leaf) return -1;
    for (int d = 0; d < 3; ++d)
        if (leaf[d] < 1) return -1;
    la_pcot p = {kind, fused, n, lda, A, {leaf[0], leaf[1], leaf[2]}, 0, 0, 0, 0};
    if (n > 0) {
        const int64_t lo[3] = {0, 0, 0};
        int64_t size[3];
        for (int d = 0; d < 3; ++d) size[d] = la_pad(n, leaf[d]);
        la_recurse(&p, lo, size);
    }
    if (stats) {
        stats[0] = p.leaves;
        stats[1] = p.zero_exits;
        stats[2] = p.empty_exits;
        stats[3] = p.points;
    }
    return 0;
}

/* ---- tile order --------------------------------------------------------- */

typedef struct {
    int kind;
    int64_t n, b, L;
    int64_t theta[3];
    int64_t *out;
    int64_t cap, count;
} la_tiles;

/* 1 if tile (kb, ib, jb) holds a domain point (checked point by point). */
static int la_tile_nonempty(const la_tiles *q, int64_t kb, int64_t ib, int64_t jb)
{
    if (kb < 0 || ib < 0 || jb < 0 || kb >= q->L || ib >= q->L || jb >= q->L) return 0;
    for (int64_t k = kb * q->b; k < (kb + 1) * q->b; ++k)
        for (int64_t i = ib * q->b; i < (ib + 1) * q->b; ++i)
            for (int64_t j = jb * q->b; j < (jb + 1) * q->b; ++j)
                if (la_in_domain(q->kind, q->n, k, i, j)) return 1;
    return 0;
}

static int la_tile_box_empty(const la_tiles *q, const int64_t *lo, const int64_t *size)
{
    for (int64_t kb = lo[0]; kb < lo[0] + size[0]; ++kb)
        for (int64_t ib = lo[1]; ib < lo[1] + size[1]; ++ib)
            for (int64_t jb = lo[2]; jb < lo[2] + size[2]; ++jb)
                if (la_tile_nonempty(q, kb, ib, jb)) return 0;
    return 1;
}

static void la_emit(la_tiles *q, int64_t kb, int64_t ib, int64_t jb)
{
    if (q->out && q->count < q->cap) {
        q->out[3 * q->count + 0] = kb;
        q->out[3 * q->count + 1] = ib;
        q->out[3 * q->count + 2] = jb;
    }
    ++q->count;
}

static void la_tiles_lex(la_tiles *q, const int64_t *lo, const int64_t *size)
{
    for (int64_t kb = lo[0]; kb < lo[0] + size[0]; ++kb)
        for (int64_t ib = lo[1]; ib < lo[1] + size[1]; ++ib)
            for (int64_t jb = lo[2]; jb < lo[2] + size[2]; ++jb)
                if (la_tile_nonempty(q, kb, ib, jb)) la_emit(q, kb, ib, jb);
}

static void la_tiles_recurse(la_tiles *q, const int64_t *lo, const int64_t *size)
{
    for (int d = 0; d < 3; ++d)
        if (size[d] == 0) return;
    if (la_tile_box_empty(q, lo, size)) return;
    int base = 1;
    for (int d = 0; d < 3; ++d)
        if (size[d] > q->theta[d]) base = 0;
    if (base) {
        la_tiles_lex(q, lo, size);
        return;
    }
    int64_t half[3][2];
    for (int d = 0; d < 3; ++d) {
        if (size[d] > q->theta[d]) {
            half[d][0] = size[d] / 2;
            half[d][1] = size[d] - size[d] / 2;
        } else {
            half[d][0] = size[d];
            half[d][1] = 0;
        }
    }
    for (int ups = 0; ups <= 3; ++ups)
        for (int m = 0; m < 8; ++m) {
            const int pc = ((m >> 2) & 1) + ((m >> 1) & 1) + (m & 1);
            if (pc != ups) continue;
            int64_t clo[3], csz[3];
            for (int d = 0; d < 3; ++d) {
                const int bit = (m >> (2 - d)) & 1;
                clo[d] = lo[d] + (bit ? half[d][0] : 0);
                csz[d] = half[d][bit];
            }
            la_tiles_recurse(q, clo, csz);
        }
}

/* Non-empty tiles (kb, ib, jb) in execution order: recursive (recursive = 1,
 * leaf theta[3] tiles) or lexicographic.  Writes up to cap triples to out
 * (may be NULL) and returns the number of tiles, or -1 on bad arguments. */
int64_t oracle_la_tile_order(int kind, int64_t n, int64_t b, const int64_t *theta, int recursive, int64_t *out,
                             int64_t cap)
{
    if ((kind != 0 && kind != 1) || n < 1 || b < 1) return -1;
    la_tiles q = {kind, n, b, (n + b - 1) / b, {1, 1, 1}, out, cap, 0};
    if (recursive) {
        if (!theta) return -1;
        for (int d = 0; d < 3; ++d) {
            if (theta[d] < 1) return -1;
            q.theta[d] = theta[d];
        }
        const int64_t lo[3] = {0, 0, 0};
        int64_t size[3];
        for (int d = 0; d < 3; ++d) size[d] = la_pad(q.L, q.theta[d]);
        la_tiles_recurse(&q, lo, size);
    } else {
        const int64_t lo[3] = {0, 0, 0}, size[3] = {q.L, q.L, q.L};
        la_tiles_lex(&q, lo, size);
    }
    return q.count;
}
