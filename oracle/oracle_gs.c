/*
 * CPU oracle for Gauss-Seidel 2-D (GS-2D, one of the stencils of the PCOT
 * paper's benchmark suite, Sec. 5.1.2) and for its recursive schedule.
 *
 * TEST INFRASTRUCTURE ONLY.  Loaded by the test-suite and the benchmark's
 * CPU-baseline arm together with oracle.c; shares no code with the CUDA
 * library, which never calls it.
 *
 * Grid: (n0 + 2) x (n1 + 2) values stored row-major with row stride s0 >=
 * n1 + 2; the outer ring (rows 0 and n0+1, columns 0 and n1+1) is fixed.
 * One time step visits the interior in lexicographic order (row i = 1..n0
 * ascending, column j = 1..n1 ascending) and replaces, in place,
 *
 *   u[i][j] <- ( u[i-1][j-1] + u[i-1][j] + u[i-1][j+1]
 *              + u[i][j-1]   + u[i][j]   + u[i][j+1]
 *              + u[i+1][j-1] + u[i+1][j] + u[i+1][j+1] ) / 9
 *
 * adding left to right in exactly that order (each add a separately rounded
 * IEEE-754 binary64 operation) and dividing once (correctly rounded).  Because
 * the update is in place, u[i-1][*] and u[i][j-1] already hold step t values
 * and the other five neighbours still hold step t-1 values.
 *
 * Recursive schedule (Sec. 4 applied to this loop nest): the iteration space
 * is skewed by (t, i, j) -> (t, t + i, 2t + i + j); every dependence (flow,
 * anti, output) then has non-negative components, so rectangular boxes of
 * the skewed space may run in any order that respects them, in particular
 * the lexicographic one.  The recursion takes the bounding box of the skewed
 * domain, pads each axis to theta_d * 2^k_d, splits a box into 2^3 orthants
 * (a width above theta is halved, a width at or below theta goes whole to the
 * lower child and leaves a zero-width upper child), visits orthants in
 * lexicographic order with the time bit most significant, returns early from
 * zero-width and empty orthants (exact emptiness test below), and runs a
 * leaf box's points in lexicographic (t, i', j') order.
 *
 * Emptiness of a box [t_lo,t_hi] x [a_lo,a_hi] x [c_lo,c_hi] (inclusive) of
 * skewed points (t, a = t + i, c = 2t + i + j), with 0 <= t < T,
 * 1 <= i <= n0, 1 <= j <= n1: for fixed t and a the admissible c form
 * [a+t+1, a+t+n1], which meet [c_lo, c_hi] iff a lies in
 * [c_lo - n1 - t, c_hi - 1 - t]; the admissible a for fixed t form
 * [t+1, t+n0].  Eliminating a pairwise, the box holds a point iff a_lo <= a_hi,
 * c_lo <= c_hi and some integer t lies in
 *   [max(t_lo, 0, a_lo - n0, ceil((c_lo - n0 - n1)/2), c_lo - n1 - a_hi),
 *    min(t_hi, T-1, a_hi - 1, floor((c_hi - 2)/2), c_hi - 1 - a_lo)].
 *
 * Parity status: oracle_gs2d is pinned by exact fixed points (affine fields
 * with small integer coefficients), a hand-derived worked example
 * (tests/golden/gs2d_steps.txt) and the in-place order (it differs from the
 * two-buffer update on random data).  oracle_gs2d_pcot is pinned by bitwise
 * equality with oracle_gs2d on brute-forced tiny problems, and
 * oracle_gs2d_box_empty by point enumeration.
 */
#include <stdint.h>
#include <stdlib.h>

static double gs_point(double *u, int64_t s0, int64_t i, int64_t j)
{
    const double *a = u + (i - 1) * s0 + j;
    const double *b = u + i * s0 + j;
    const double *c = u + (i + 1) * s0 + j;
    double acc = a[-1];
    acc = acc + a[0];
    acc = acc + a[1];
    acc = acc + b[-1];
    acc = acc + b[0];
    acc = acc + b[1];
    acc = acc + c[-1];
    acc = acc + c[0];
    acc = acc + c[1];
    return acc / 9.0;
}

/* T steps of the plain in-place loop nest. */
int oracle_gs2d(int64_t n0, int64_t n1, int64_t s0, double *u, int64_t T)
{
    if (n0 < 1 || n1 < 1 || s0 < n1 + 2 || !u || T < 0) return -1;
    for (int64_t t = 0; t < T; ++t)
        for (int64_t i = 1; i <= n0; ++i)
            for (int64_t j = 1; j <= n1; ++j) u[i * s0 + j] = gs_point(u, s0, i, j);
    return 0;
}

static int64_t gs_max(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t gs_min(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t gs_fdiv2(int64_t a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }  /* floor(a/2) */
static int64_t gs_cdiv2(int64_t a) { return -gs_fdiv2(-a); }                     /* ceil(a/2) */

/* 1 if the inclusive skewed box holds no point of the domain. */
int oracle_gs2d_box_empty(int64_t n0, int64_t n1, int64_t T, const int64_t *lo, const int64_t *hi)
{
    if (lo[0] > hi[0] || lo[1] > hi[1] || lo[2] > hi[2]) return 1;
    const int64_t tl = gs_max(gs_max(gs_max(lo[0], 0), gs_max(lo[1] - n0, gs_cdiv2(lo[2] - n0 - n1))),
                              lo[2] - n1 - hi[1]);
    const int64_t th = gs_min(gs_min(gs_min(hi[0], T - 1), gs_min(hi[1] - 1, gs_fdiv2(hi[2] - 2))),
                              hi[2] - 1 - lo[1]);
    return tl > th;
}

typedef struct {
    int64_t n0, n1, s0, T;
    double *u;
    int64_t leaf[3];
    int64_t *order;      /* recorded leaf points (t, a, c) or NULL */
    int64_t cap, count;  /* record capacity / points visited */
    int64_t zero_exits, empty_exits, leaves;
} gs_pcot;

static void gs_leaf(gs_pcot *p, const int64_t *lo, const int64_t *size)
{
    ++p->leaves;
    for (int64_t t = lo[0]; t < lo[0] + size[0]; ++t)
        for (int64_t a = lo[1]; a < lo[1] + size[1]; ++a)
            for (int64_t c = lo[2]; c < lo[2] + size[2]; ++c) {
                const int64_t i = a - t, j = c - a - t;
                if (t < 0 || t >= p->T || i < 1 || i > p->n0 || j < 1 || j > p->n1) continue;
                if (p->u) p->u[i * p->s0 + j] = gs_point(p->u, p->s0, i, j);
                if (p->order && p->count < p->cap) {
                    p->order[3 * p->count + 0] = t;
                    p->order[3 * p->count + 1] = a;
                    p->order[3 * p->count + 2] = c;
                }
                ++p->count;
            }
}

static void gs_recurse(gs_pcot *p, const int64_t *lo, const int64_t *size)
{
    for (int d = 0; d < 3; ++d)
        if (size[d] == 0) {
            ++p->zero_exits;
            return;
        }
    int64_t hi[3];
    for (int d = 0; d < 3; ++d) hi[d] = lo[d] + size[d] - 1;
    if (oracle_gs2d_box_empty(p->n0, p->n1, p->T, lo, hi)) {
        ++p->empty_exits;
        return;
    }
    int base = 1;
    for (int d = 0; d < 3; ++d)
        if (size[d] > p->leaf[d]) base = 0;
    if (base) {
        gs_leaf(p, lo, size);
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
    for (int m = 0; m < 8; ++m) {  /* bit 2 = time (most significant), bit 0 = c */
        int64_t clo[3], csz[3];
        for (int d = 0; d < 3; ++d) {
            const int bit = (m >> (2 - d)) & 1;
            clo[d] = lo[d] + (bit ? half[d][0] : 0);
            csz[d] = half[d][bit];
        }
        gs_recurse(p, clo, csz);
    }
}

static int64_t gs_pad(int64_t N, int64_t b)
{
    int64_t w = b;
    while (w < N) w *= 2;
    return w;
}

/* Bounding box of the skewed domain: t in [0, T), a in [1, T-1+n0],
 * c in [2, 2(T-1)+n0+n1]; each axis padded to leaf_d * 2^k_d. */
static void gs_box(int64_t n0, int64_t n1, int64_t T, const int64_t *leaf, int64_t *lo, int64_t *size)
{
    lo[0] = 0;
    lo[1] = 1;
    lo[2] = 2;
    const int64_t ext[3] = {T, T - 1 + n0, 2 * T - 3 + n0 + n1};
    for (int d = 0; d < 3; ++d) size[d] = gs_pad(ext[d], leaf[d]);
}

/* The T steps in the recursive order; stats (may be NULL) receives
 * {leaves, zero exits, empty exits, points}. */
int oracle_gs2d_pcot(int64_t n0, int64_t n1, int64_t s0, double *u, int64_t T, const int64_t *leaf,
                     int64_t *stats)
{
    if (n0 < 1 || n1 < 1 || s0 < n1 + 2 || !u || T < 0 || !leaf) return -1;
    for (int d = 0; d < 3; ++d)
        if (leaf[d] < 1) return -1;
    gs_pcot p = {n0, n1, s0, T, u, {leaf[0], leaf[1], leaf[2]}, NULL, 0, 0, 0, 0, 0};
    if (T > 0) {
        int64_t lo[3], size[3];
        gs_box(n0, n1, T, leaf, lo, size);
        gs_recurse(&p, lo, size);
    }
    if (stats) {
        stats[0] = p.leaves;
        stats[1] = p.zero_exits;
        stats[2] = p.empty_exits;
        stats[3] = p.count;
    }
    return 0;
}

/* Tile-level form of the same recursion, the order a tiled executor follows:
 * tiles of kt x ha x wc skewed points, tile (b0, b1, b2) covering t in
 * [b0*kt, b0*kt + kt), a in [1 + b1*ha, ...), c in [2 + b2*wc, ...).  The
 * lattice's bounding box [0, L0) x [0, L1) x [0, L2) is padded to
 * theta_d * 2^k_d tiles, split into orthants as above (zero and empty exits,
 * a box of tiles being empty when the points it covers are), and a leaf box
 * lists its non-empty tiles lexicographically.  With `wavefront` set, the
 * children of a box are visited grouped by their number of upper halves
 * (orthants with equal counts are independent: the wavefronts of the
 * parallel recursion) and a leaf lists its tiles by b0 + b1 + b2, then
 * lexicographically -- the order a GPU executor uses to expose parallelism.  Records (b0, b1, b2) of each
 * non-empty tile in order, up to cap; returns their number. */
typedef struct {
    int64_t n0, n1, T, tile[3], theta[3];
    int64_t *out;
    int64_t cap, count;
    int wavefront;  /* children by number of upper halves, leaves by b0+b1+b2 */
} gs_tiles;

static void gs_tiles_emit(gs_tiles *q, const int64_t *b)
{
    if (q->out && q->count < q->cap)
        for (int d = 0; d < 3; ++d) q->out[3 * q->count + d] = b[d];
    ++q->count;
}

static int gs_tiles_empty(const gs_tiles *q, const int64_t *blo, const int64_t *bhi)
{
    const int64_t base[3] = {0, 1, 2};
    int64_t lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = base[d] + blo[d] * q->tile[d];
        hi[d] = base[d] + (bhi[d] + 1) * q->tile[d] - 1;
    }
    return oracle_gs2d_box_empty(q->n0, q->n1, q->T, lo, hi);
}

static void gs_tiles_recurse(gs_tiles *q, const int64_t *lo, const int64_t *size)
{
    for (int d = 0; d < 3; ++d)
        if (size[d] == 0) return;
    int64_t hi[3];
    for (int d = 0; d < 3; ++d) hi[d] = lo[d] + size[d] - 1;
    if (gs_tiles_empty(q, lo, hi)) return;
    int base = 1;
    for (int d = 0; d < 3; ++d)
        if (size[d] > q->theta[d]) base = 0;
    if (base) {
        int64_t b[3];
        if (q->wavefront) {
            for (int64_t w = lo[0] + lo[1] + lo[2]; w <= hi[0] + hi[1] + hi[2]; ++w)
                for (b[0] = lo[0]; b[0] <= hi[0]; ++b[0])
                    for (b[1] = lo[1]; b[1] <= hi[1]; ++b[1]) {
                        b[2] = w - b[0] - b[1];
                        if (b[2] < lo[2] || b[2] > hi[2] || gs_tiles_empty(q, b, b)) continue;
                        gs_tiles_emit(q, b);
                    }
        } else {
            for (b[0] = lo[0]; b[0] <= hi[0]; ++b[0])
                for (b[1] = lo[1]; b[1] <= hi[1]; ++b[1])
                    for (b[2] = lo[2]; b[2] <= hi[2]; ++b[2])
                        if (!gs_tiles_empty(q, b, b)) gs_tiles_emit(q, b);
        }
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
    /* lexicographic children, or grouped by their number of upper halves */
    for (int pass = 0; pass < (q->wavefront ? 4 : 1); ++pass)
        for (int m = 0; m < 8; ++m) {
            const int ups = ((m >> 2) & 1) + ((m >> 1) & 1) + (m & 1);
            if (q->wavefront && ups != pass) continue;
            int64_t clo[3], csz[3];
            for (int d = 0; d < 3; ++d) {
                const int bit = (m >> (2 - d)) & 1;
                clo[d] = lo[d] + (bit ? half[d][0] : 0);
                csz[d] = half[d][bit];
            }
            gs_tiles_recurse(q, clo, csz);
        }
}

int64_t oracle_gs2d_tile_order(int64_t n0, int64_t n1, int64_t T, const int64_t *tile, const int64_t *theta,
                               int wavefront, int64_t *out, int64_t cap)
{
    if (n0 < 1 || n1 < 1 || T < 0 || !tile || !theta) return -1;
    for (int d = 0; d < 3; ++d)
        if (tile[d] < 1 || theta[d] < 1) return -1;
    gs_tiles q = {n0, n1, T, {tile[0], tile[1], tile[2]}, {theta[0], theta[1], theta[2]}, out, cap, 0, wavefront};
    if (T == 0) return 0;
    const int64_t ext[3] = {T, T - 1 + n0, 2 * T - 3 + n0 + n1};
    int64_t lo[3] = {0, 0, 0}, size[3];
    for (int d = 0; d < 3; ++d) size[d] = gs_pad((ext[d] + tile[d] - 1) / tile[d], theta[d]);
    gs_tiles_recurse(&q, lo, size);
    return q.count;
}
