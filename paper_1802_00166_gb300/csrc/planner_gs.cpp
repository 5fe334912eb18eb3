// Tile planners over skewed 3-D lattices: Gauss-Seidel 2-D (GS-2D, Sec.
// 5.1.2; the in-place, lexicographic 9-point average) and the two-buffer 2-D
// Jacobi star stencil tiled by parallelograms of its skewed space (skew_plan
// at the end; the same orders and dependency rule, another skew).
//
// The iteration space (t, i, j) is skewed to (t, a, c) = (t, t + i, 2t + i + j):
// a point reads its north row and west neighbour at step t and its own, east
// and south neighbours at step t-1, and in the skewed coordinates every such
// dependence (and every anti/output dependence of the in-place update) has
// components in {0, 1, 2} (Sec. 4.1: tiling the skewed space is legal).  Tiles
// are boxes of kt x ha x wc skewed points; with wc >= 2 a tile depends only
// on its seven lower neighbours (b - d, d in {0,1}^3 \ 0).
//
// Orders (both topological):
//  * wavefront: non-empty tiles by b0 + b1 + b2, then lexicographically; the
//    tiles of one wavefront are independent, so a persistent executor that
//    pops in order runs a whole wavefront at once (the single-level schedule);
//  * recursive (Sec. 4.2-4.3): the lattice's bounding box padded to
//    theta_d * 2^k_d tiles, split into 2^3 orthants (a width above theta is
//    halved, one at or below goes whole to the lower child), zero-width and
//    empty orthants skipped; children are visited by the number of upper
//    halves they take (orthants with equal counts are independent, the
//    wavefronts of the paper's parallel recursion), ties in lexicographic
//    order with the time bit most significant; a leaf lists its tiles in
//    wavefront order.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "planner.h"

namespace pcot {

namespace {

// A 3-D lattice of tiles with a per-tile emptiness flag; the orders and
// dependency counts below depend on nothing else.
struct GsLattice {
    int64_t n0, n1, T;
    int32_t tile[3];
    int32_t L[3];
    std::vector<uint8_t> nonempty;   // per lattice id
    std::vector<int32_t> prefix;     // (L0+1)(L1+1)(L2+1) inclusive-exclusive prefix counts

    int64_t id(int64_t b0, int64_t b1, int64_t b2) const { return (b0 * L[1] + b1) * L[2] + b2; }
    int64_t pid(int64_t b0, int64_t b1, int64_t b2) const {
        return (b0 * (L[1] + 1) + b1) * (int64_t)(L[2] + 1) + b2;
    }
    // Non-empty tiles in [lo, lo+size) (lattice box), by inclusion-exclusion.
    int64_t count(const int64_t* lo, const int64_t* size) const {
        int64_t hi[3], l[3];
        for (int d = 0; d < 3; ++d) {
            l[d] = std::max<int64_t>(0, lo[d]);
            hi[d] = std::min<int64_t>(L[d], lo[d] + size[d]);
            if (hi[d] <= l[d]) return 0;
        }
        // sum over the 8 corners, sign (-1)^(number of low coordinates)
        int64_t s = 0;
        for (int m = 0; m < 8; ++m) {
            const int64_t x = (m & 4) ? hi[0] : l[0], y = (m & 2) ? hi[1] : l[1], z = (m & 1) ? hi[2] : l[2];
            const int lows = 3 - (((m >> 2) & 1) + ((m >> 1) & 1) + (m & 1));
            s += (lows % 2 == 0 ? 1 : -1) * (int64_t)prefix[pid(x, y, z)];
        }
        return s;
    }
};

// Does tile b hold a point (t, a, c) with 0 <= t < T, 1 <= a-t <= n0,
// 1 <= c-a-t <= n1?  Scans the tile's time steps.
bool tile_nonempty(const GsLattice& g, int64_t b0, int64_t b1, int64_t b2) {
    const int64_t t_lo = b0 * g.tile[0], a_lo = 1 + b1 * g.tile[1], c_lo = 2 + b2 * g.tile[2];
    const int64_t a_hi = a_lo + g.tile[1] - 1, c_hi = c_lo + g.tile[2] - 1;
    for (int64_t t = t_lo; t < t_lo + g.tile[0] && t < g.T; ++t) {
        // a admissible for this t: [t+1, t+n0]; c for a: [a+t+1, a+t+n1]
        const int64_t lo = std::max({a_lo, t + 1, c_lo - g.n1 - t});
        const int64_t hi = std::min({a_hi, t + g.n0, c_hi - 1 - t});
        if (lo <= hi) return true;
    }
    return false;
}

// Lattice extents, emptiness flags (by `nonempty(b0, b1, b2)`) and the prefix
// counts used to test orthants for emptiness.
template <class F>
void build_lattice(GsLattice& g, const int64_t* ext, F nonempty) {
    for (int d = 0; d < 3; ++d) g.L[d] = (int32_t)((ext[d] + g.tile[d] - 1) / g.tile[d]);
    const int64_t n = (int64_t)g.L[0] * g.L[1] * g.L[2];
    g.nonempty.assign((size_t)n, 0);
    for (int64_t b0 = 0; b0 < g.L[0]; ++b0)
        for (int64_t b1 = 0; b1 < g.L[1]; ++b1)
            for (int64_t b2 = 0; b2 < g.L[2]; ++b2) g.nonempty[(size_t)g.id(b0, b1, b2)] = nonempty(b0, b1, b2);
    g.prefix.assign((size_t)(g.L[0] + 1) * (g.L[1] + 1) * (g.L[2] + 1), 0);
    for (int64_t b0 = 1; b0 <= g.L[0]; ++b0)
        for (int64_t b1 = 1; b1 <= g.L[1]; ++b1)
            for (int64_t b2 = 1; b2 <= g.L[2]; ++b2) {
                int64_t v = g.nonempty[(size_t)g.id(b0 - 1, b1 - 1, b2 - 1)];
                v += g.prefix[g.pid(b0 - 1, b1, b2)] + g.prefix[g.pid(b0, b1 - 1, b2)] + g.prefix[g.pid(b0, b1, b2 - 1)];
                v -= g.prefix[g.pid(b0 - 1, b1 - 1, b2)] + g.prefix[g.pid(b0 - 1, b1, b2 - 1)] +
                     g.prefix[g.pid(b0, b1 - 1, b2 - 1)];
                v += g.prefix[g.pid(b0 - 1, b1 - 1, b2 - 1)];
                g.prefix[g.pid(b0, b1, b2)] = (int32_t)v;
            }
}

// Non-empty tiles of a lattice box in wavefront order.
void emit_wavefront(const GsLattice& g, const int64_t* lo, const int64_t* size, std::vector<int32_t>& out) {
    const int64_t l[3] = {std::max<int64_t>(0, lo[0]), std::max<int64_t>(0, lo[1]), std::max<int64_t>(0, lo[2])};
    const int64_t h[3] = {std::min<int64_t>(g.L[0], lo[0] + size[0]), std::min<int64_t>(g.L[1], lo[1] + size[1]),
                          std::min<int64_t>(g.L[2], lo[2] + size[2])};
    if (h[0] <= l[0] || h[1] <= l[1] || h[2] <= l[2]) return;
    for (int64_t w = l[0] + l[1] + l[2]; w <= (h[0] - 1) + (h[1] - 1) + (h[2] - 1); ++w)
        for (int64_t b0 = l[0]; b0 < h[0]; ++b0)
            for (int64_t b1 = l[1]; b1 < h[1]; ++b1) {
                const int64_t b2 = w - b0 - b1;
                if (b2 < l[2] || b2 >= h[2]) continue;
                const int64_t k = g.id(b0, b1, b2);
                if (g.nonempty[(size_t)k]) out.push_back((int32_t)k);
            }
}

void recurse(const GsLattice& g, const int32_t* theta, const int64_t* lo, const int64_t* size,
             std::vector<int32_t>& out) {
    for (int d = 0; d < 3; ++d)
        if (size[d] == 0) return;  // zero orthant
    if (g.count(lo, size) == 0) return;  // empty orthant
    bool leaf = true;
    for (int d = 0; d < 3; ++d)
        if (size[d] > theta[d]) leaf = false;
    if (leaf) {
        emit_wavefront(g, lo, size, out);
        return;
    }
    int64_t half[3][2];
    for (int d = 0; d < 3; ++d) {
        if (size[d] > theta[d]) {
            half[d][0] = size[d] / 2;
            half[d][1] = size[d] - size[d] / 2;
        } else {
            half[d][0] = size[d];
            half[d][1] = 0;
        }
    }
    static const int kChildOrder[8] = {0, 1, 2, 4, 3, 5, 6, 7};  // by number of upper halves, then lexicographic
    for (int k = 0; k < 8; ++k) {
        const int m = kChildOrder[k];
        int64_t clo[3], csz[3];
        for (int d = 0; d < 3; ++d) {
            const int bit = (m >> (2 - d)) & 1;
            clo[d] = lo[d] + (bit ? half[d][0] : 0);
            csz[d] = half[d][bit];
        }
        recurse(g, theta, clo, csz, out);
    }
}

// Queue (wavefront or recursive order) and per-tile dependency counts (the
// non-empty tiles among the seven lower neighbours) of a built lattice.
void order_and_deps(const GsLattice& g, int recursive, const int32_t* theta, std::vector<int32_t>& queue,
                    std::vector<int32_t>& deps) {
    queue.clear();
    if (recursive) {
        int64_t lo[3] = {0, 0, 0}, size[3];
        for (int d = 0; d < 3; ++d) {
            int64_t w = theta[d];
            while (w < g.L[d]) w *= 2;
            size[d] = w;
        }
        recurse(g, theta, lo, size, queue);
    } else {
        const int64_t lo[3] = {0, 0, 0}, size[3] = {g.L[0], g.L[1], g.L[2]};
        emit_wavefront(g, lo, size, queue);
    }
    const int64_t n = (int64_t)g.L[0] * g.L[1] * g.L[2];
    deps.assign((size_t)n, 0);
    for (int64_t b0 = 0; b0 < g.L[0]; ++b0)
        for (int64_t b1 = 0; b1 < g.L[1]; ++b1)
            for (int64_t b2 = 0; b2 < g.L[2]; ++b2) {
                if (!g.nonempty[(size_t)g.id(b0, b1, b2)]) continue;
                int c = 0;
                for (int m = 1; m < 8; ++m) {
                    const int64_t p0 = b0 - ((m >> 2) & 1), p1 = b1 - ((m >> 1) & 1), p2 = b2 - (m & 1);
                    if (p0 < 0 || p1 < 0 || p2 < 0) continue;
                    if (g.nonempty[(size_t)g.id(p0, p1, p2)]) ++c;
                }
                deps[(size_t)g.id(b0, b1, b2)] = c;
            }
}

bool lattice_too_big(const int64_t* ext, const int32_t* tile) {
    int64_t cells = 1;
    for (int d = 0; d < 3; ++d) {
        cells *= (ext[d] + tile[d] - 1) / tile[d];
        if (cells > (int64_t)1 << 28) return true;
    }
    return false;
}

}  // namespace

bool gs_plan(int64_t n0, int64_t n1, int64_t T, const int32_t* tile, int recursive, const int32_t* theta,
             GsPlanHost* out) {
    if (n0 < 1 || n1 < 1 || T < 1 || !tile || !out) return false;
    // A dependence moves at most 1 in t and a and at most 2 in c, so tiles at
    // least 1 x 1 x 2 wide cross at most one tile boundary per axis.
    if (tile[0] < 1 || tile[1] < 1 || tile[2] < 2) return false;
    for (int d = 0; d < 3; ++d)
        if (recursive && (!theta || theta[d] < 1)) return false;
    GsLattice g;
    g.n0 = n0;
    g.n1 = n1;
    g.T = T;
    for (int d = 0; d < 3; ++d) g.tile[d] = tile[d];
    const int64_t ext[3] = {T, T - 1 + n0, 2 * T - 3 + n0 + n1};
    if (lattice_too_big(ext, tile)) return false;
    build_lattice(g, ext, [&](int64_t b0, int64_t b1, int64_t b2) { return tile_nonempty(g, b0, b1, b2); });
    order_and_deps(g, recursive, theta, out->queue, out->deps);
    for (int d = 0; d < 3; ++d) out->lattice[d] = g.L[d];
    return true;
}

bool skew_plan(int64_t n0, int64_t n1, int64_t T, const int32_t* tile, int recursive, const int32_t* theta,
               GsPlanHost* out) {
    if (n0 < 1 || n1 < 1 || T < 1 || !tile || !out) return false;
    // Dependences move at most 1 in t and at most 2 in a and c, so tiles at
    // least 1 x 2 x 2 wide cross at most one tile boundary per axis.
    if (tile[0] < 1 || tile[1] < 2 || tile[2] < 2) return false;
    for (int d = 0; d < 3; ++d)
        if (recursive && (!theta || theta[d] < 1)) return false;
    GsLattice g;
    g.n0 = n0;
    g.n1 = n1;
    g.T = T;
    for (int d = 0; d < 3; ++d) g.tile[d] = tile[d];
    // (t, a, c) = (t, t + i, t + j): 0 <= t < T, 1 <= i <= n0, 1 <= j <= n1;
    // a and c start at 1
    const int64_t ext[3] = {T, T - 1 + n0, T - 1 + n1};
    if (lattice_too_big(ext, tile)) return false;
    // Exact emptiness: the steps t at which the tile's a-range meets
    // [t + 1, t + n0] form the interval [a_lo - n0, a_hi - 1]; likewise for
    // c; the tile holds a point iff these intervals, the tile's steps and
    // [0, T) share a step.
    build_lattice(g, ext, [&](int64_t b0, int64_t b1, int64_t b2) {
        const int64_t t_lo = b0 * tile[0], t_hi = std::min<int64_t>(t_lo + tile[0], T) - 1;
        const int64_t a_lo = 1 + b1 * tile[1], a_hi = a_lo + tile[1] - 1;
        const int64_t c_lo = 1 + b2 * tile[2], c_hi = c_lo + tile[2] - 1;
        const int64_t lo = std::max({t_lo, a_lo - n0, c_lo - n1, (int64_t)0});
        const int64_t hi = std::min({t_hi, a_hi - 1, c_hi - 1});
        return lo <= hi;
    });
    order_and_deps(g, recursive, theta, out->queue, out->deps);
    for (int d = 0; d < 3; ++d) out->lattice[d] = g.L[d];
    return true;
}

}  // namespace pcot
