// Tile graph of the blocked LU and Cholesky factorizations (the
// linear-algebra kernels of the benchmark suite, Sec. 5.1.2), shared by the
// host planner (dependency counts) and the device executor (releases), so
// that the two agree by construction.
//
// The statements live in the (k, i, j) space (LU: 0 <= k < i < n,
// k <= j < n; Cholesky: 0 <= k <= j <= i < n); tile (kb, ib, jb) holds the
// points with k in [kb b, kb b + b) and likewise for i and j, so it is the
// work of block step kb on matrix block (ib, jb):
//   LU        kb = ib = jb   factor the diagonal block
//             ib = kb < jb   row panel: apply the unit lower factor of (kb, kb)
//             jb = kb < ib   column panel: apply the upper factor of (kb, kb)
//             ib, jb > kb    A(ib, jb) -= A(ib, kb) A(kb, jb)
//   Cholesky  kb = ib = jb   factor the diagonal block
//             jb = kb < ib   panel: solve against the factor of (kb, kb)
//             ib >= jb > kb  A(ib, jb) -= A(ib, kb) A(jb, kb)^T (lower part)
// Every point dependence has non-negative components (Sec. 4.1), so tiles
// may run in any order that respects the edges below; the edges cover every
// point dependence between distinct tiles (a block's next update waits for
// its previous one; a panel waits for its diagonal block; an update waits
// for the panels it reads).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define PCOT_LA_HD __host__ __device__ __forceinline__
#else
#define PCOT_LA_HD inline
#endif

namespace pcot {

enum { kLaLU = 0, kLaCholesky = 1 };

// Does tile (kb, ib, jb) hold a point of the domain?  Within a domain a
// smaller k only widens the admissible i and j, so the tile's smallest k
// decides.
PCOT_LA_HD bool la_tile_nonempty(int kind, int64_t n, int b, int64_t L, int64_t kb, int64_t ib, int64_t jb) {
    if (kb < 0 || ib < 0 || jb < 0 || kb >= L || ib >= L || jb >= L) return false;
    const int64_t k = kb * b;
    const int64_t imin = ib * b, jmin = jb * b;
    const int64_t imax = ((ib + 1) * b < n ? (ib + 1) * b : n) - 1;
    const int64_t jmax = ((jb + 1) * b < n ? (jb + 1) * b : n) - 1;
    if (kind == kLaLU) {
        const int64_t i = imin > k + 1 ? imin : k + 1;
        const int64_t j = jmin > k ? jmin : k;
        return i <= imax && j <= jmax;
    }
    const int64_t j = jmin > k ? jmin : k;
    const int64_t i = imin > j ? imin : j;
    return j <= jmax && i <= imax;
}

PCOT_LA_HD int64_t la_tile_id(int64_t L, int64_t kb, int64_t ib, int64_t jb) { return (kb * L + ib) * L + jb; }

// Calls f(id) for every non-empty successor of the non-empty tile
// (kb, ib, jb).
template <class F>
PCOT_LA_HD void la_for_each_successor(int kind, int64_t n, int b, int64_t L, int64_t kb, int64_t ib, int64_t jb,
                                      F&& f) {
    auto emit = [&](int64_t k2, int64_t i2, int64_t j2) {
        if (la_tile_nonempty(kind, n, b, L, k2, i2, j2)) f(la_tile_id(L, k2, i2, j2));
    };
    if (kind == kLaLU) {
        if (ib == kb && jb == kb) {
            for (int64_t j = kb + 1; j < L; ++j) emit(kb, kb, j);
            for (int64_t i = kb + 1; i < L; ++i) emit(kb, i, kb);
        } else if (ib == kb) {
            for (int64_t i = kb + 1; i < L; ++i) emit(kb, i, jb);
        } else if (jb == kb) {
            for (int64_t j = kb + 1; j < L; ++j) emit(kb, ib, j);
        } else {
            emit(kb + 1, ib, jb);
        }
        return;
    }
    if (ib == kb) {  // diagonal block (jb == kb)
        for (int64_t i = kb + 1; i < L; ++i) emit(kb, i, kb);
    } else if (jb == kb) {  // panel of row block ib: read by row ib and by column ib
        for (int64_t j = kb + 1; j <= ib; ++j) emit(kb, ib, j);
        for (int64_t i = ib + 1; i < L; ++i) emit(kb, i, ib);
    } else {
        emit(kb + 1, ib, jb);
    }
}

}  // namespace pcot
