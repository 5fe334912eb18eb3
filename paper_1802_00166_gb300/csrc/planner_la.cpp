// Tile planner for the blocked LU and Cholesky factorizations (the
// linear-algebra kernels of the benchmark suite, Sec. 5.1.2).
//
// The lattice of b x b x b tiles over the (k, i, j) space is a cube of
// L = ceil(n / b) tiles per side of which only a pyramid holds work (LU:
// ib, jb >= kb; Cholesky: kb <= jb <= ib), so the recursion of Sec. 4.2-4.3
// over its bounding box meets many empty orthants and returns from them at
// once (Sec. 4.3, early exit for empty orthants).  Orders (both
// topological, since every edge of the tile graph has non-negative
// components):
//  * single-level: all non-empty tiles lexicographically (k most significant);
//  * recursive: the lattice padded to theta_d * 2^m_d tiles, split into 2^3
//    orthants (a width above theta is halved, one at or below goes whole to
//    the lower child), zero-width and empty orthants skipped, children by the
//    number of upper halves they take (equal counts are independent: the
//    wavefronts of the paper's parallel recursion), ties lexicographic; a
//    leaf lists its tiles lexicographically.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "la_graph.h"
#include "planner.h"

namespace pcot {

namespace {

struct LaLattice {
    int kind;
    int64_t n;
    int32_t b;
    int64_t L;
    std::vector<uint8_t> nonempty;  // per lattice id
    std::vector<int32_t> prefix;    // (L+1)^3 prefix counts of non-empty tiles

    int64_t pid(int64_t x, int64_t y, int64_t z) const { return (x * (L + 1) + y) * (L + 1) + z; }

    // Non-empty tiles in the lattice box [lo, lo + size), by inclusion-exclusion.
    int64_t count(const int64_t* lo, const int64_t* size) const {
        int64_t l[3], h[3];
        for (int d = 0; d < 3; ++d) {
            l[d] = std::max<int64_t>(0, lo[d]);
            h[d] = std::min<int64_t>(L, lo[d] + size[d]);
            if (h[d] <= l[d]) return 0;
        }
        int64_t s = 0;
        for (int m = 0; m < 8; ++m) {
            const int64_t x = (m & 4) ? h[0] : l[0], y = (m & 2) ? h[1] : l[1], z = (m & 1) ? h[2] : l[2];
            const int lows = 3 - (((m >> 2) & 1) + ((m >> 1) & 1) + (m & 1));
            s += (lows % 2 == 0 ? 1 : -1) * (int64_t)prefix[(size_t)pid(x, y, z)];
        }
        return s;
    }
};

void build_lattice(LaLattice& g) {
    const int64_t L = g.L;
    g.nonempty.assign((size_t)(L * L * L), 0);
    for (int64_t kb = 0; kb < L; ++kb)
        for (int64_t ib = 0; ib < L; ++ib)
            for (int64_t jb = 0; jb < L; ++jb)
                g.nonempty[(size_t)la_tile_id(L, kb, ib, jb)] = la_tile_nonempty(g.kind, g.n, g.b, L, kb, ib, jb);
    g.prefix.assign((size_t)((L + 1) * (L + 1) * (L + 1)), 0);
    for (int64_t x = 1; x <= L; ++x)
        for (int64_t y = 1; y <= L; ++y)
            for (int64_t z = 1; z <= L; ++z) {
                int64_t v = g.nonempty[(size_t)la_tile_id(L, x - 1, y - 1, z - 1)];
                v += g.prefix[(size_t)g.pid(x - 1, y, z)] + g.prefix[(size_t)g.pid(x, y - 1, z)] +
                     g.prefix[(size_t)g.pid(x, y, z - 1)];
                v -= g.prefix[(size_t)g.pid(x - 1, y - 1, z)] + g.prefix[(size_t)g.pid(x - 1, y, z - 1)] +
                     g.prefix[(size_t)g.pid(x, y - 1, z - 1)];
                v += g.prefix[(size_t)g.pid(x - 1, y - 1, z - 1)];
                g.prefix[(size_t)g.pid(x, y, z)] = (int32_t)v;
            }
}

void emit_lex(const LaLattice& g, const int64_t* lo, const int64_t* size, std::vector<int32_t>& out) {
    for (int64_t kb = std::max<int64_t>(0, lo[0]); kb < std::min<int64_t>(g.L, lo[0] + size[0]); ++kb)
        for (int64_t ib = std::max<int64_t>(0, lo[1]); ib < std::min<int64_t>(g.L, lo[1] + size[1]); ++ib)
            for (int64_t jb = std::max<int64_t>(0, lo[2]); jb < std::min<int64_t>(g.L, lo[2] + size[2]); ++jb) {
                const int64_t id = la_tile_id(g.L, kb, ib, jb);
                if (g.nonempty[(size_t)id]) out.push_back((int32_t)id);
            }
}

void recurse(const LaLattice& g, const int32_t* theta, const int64_t* lo, const int64_t* size,
             std::vector<int32_t>& out) {
    for (int d = 0; d < 3; ++d)
        if (size[d] == 0) return;        // zero orthant
    if (g.count(lo, size) == 0) return;  // empty orthant
    bool leaf = true;
    for (int d = 0; d < 3; ++d)
        if (size[d] > theta[d]) leaf = false;
    if (leaf) {
        emit_lex(g, lo, size, out);
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
    for (int c = 0; c < 8; ++c) {
        const int m = kChildOrder[c];
        int64_t clo[3], csz[3];
        for (int d = 0; d < 3; ++d) {
            const int bit = (m >> (2 - d)) & 1;
            clo[d] = lo[d] + (bit ? half[d][0] : 0);
            csz[d] = half[d][bit];
        }
        recurse(g, theta, clo, csz, out);
    }
}

}  // namespace

bool la_plan(int kind, int64_t n, int32_t b, int recursive, const int32_t* theta, LaPlanHost* out) {
    if ((kind != kLaLU && kind != kLaCholesky) || n < 1 || b < 1 || !out) return false;
    if (recursive && !theta) return false;
    for (int d = 0; d < 3; ++d)
        if (recursive && theta[d] < 1) return false;
    LaLattice g;
    g.kind = kind;
    g.n = n;
    g.b = b;
    g.L = (n + b - 1) / b;
    if (g.L > 256) return false;  // L^3 counters and the lattice's prefix table
    build_lattice(g);
    out->L = (int32_t)g.L;
    out->queue.clear();
    const int64_t lo[3] = {0, 0, 0};
    if (recursive) {
        int64_t size[3];
        for (int d = 0; d < 3; ++d) {
            int64_t w = theta[d];
            while (w < g.L) w *= 2;
            size[d] = w;
        }
        recurse(g, theta, lo, size, out->queue);
    } else {
        const int64_t size[3] = {g.L, g.L, g.L};
        emit_lex(g, lo, size, out->queue);
    }
    out->deps.assign(g.nonempty.size(), 0);
    for (int32_t id : out->queue) {
        const int64_t jb = id % g.L, ib = (id / g.L) % g.L, kb = id / (g.L * g.L);
        la_for_each_successor(kind, n, b, g.L, kb, ib, jb, [&](int64_t s) { ++out->deps[(size_t)s]; });
    }
    return true;
}

}  // namespace pcot
