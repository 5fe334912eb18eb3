// Host-side schedule planning: time blocks and the recursive tile order.
#pragma once

#include <stdint.h>

#include <vector>

namespace pcot {

// Time blocks of the single-level schedule: depths in execution order.  The
// number of blocks is made even (each block swaps the two buffers, so an even
// count leaves the result in the caller's grid); when every block has depth 1
// and the count is odd, final_copy asks for one buffer copy at the end.
struct BlockPlan {
    std::vector<int> depths;
    bool final_copy = false;
};

// `supported` (ascending) lists the depths a kernel family can run; an empty
// list means "any depth".
BlockPlan plan_blocks(int64_t T, int k, const std::vector<int>& supported);

// Order of the (time block, tile) lattice under the recursive schedule of
// Sec. 4: skew every spatial lattice axis by the block index (tiles of block
// b depend on tiles of block b-1 at lattice distance <= 1, so J_a = I_a + b
// makes every dependence non-negative), take the bounding box, pad each axis
// to theta_i * 2^k_i (Sec. 4.5), split into 2^D orthants visited in
// lexicographic order with zero/empty exits (Sec. 4.3) and enumerate each
// leaf orthant lexicographically (Sec. 4.2).  Returns linear tile ids
// ((b * L0 + i0) * L1 + i1) * L2 + i2 (unused axes have L = 1).
struct LatticeOrderStats {
    int64_t recursive_calls = 0, leaves = 0, zero_exits = 0, empty_exits = 0;
};
std::vector<int32_t> pcot_lattice_order(int P, int dims, const int64_t* L, const int64_t* theta,
                                        LatticeOrderStats* stats);

// Initial dependency count of every tile id: the number of tiles of the
// previous block within lattice distance 1 (0 for the first block).
std::vector<int32_t> lattice_dep_counts(int P, int dims, const int64_t* L);

// Gauss-Seidel 2-D tile plan (planner_gs.cpp): lattice extents of the
// skewed (t, t+i, 2t+i+j) space in tiles, the non-empty tiles' linear ids
// (b0 * L1 + b1) * L2 + b2 in execution order (wavefront, or the recursive
// order when `recursive`), and per lattice id the number of non-empty
// predecessors among its seven lower neighbours.
struct GsPlanHost {
    int32_t lattice[3] = {0, 0, 0};
    std::vector<int32_t> queue;
    std::vector<int32_t> deps;
};
bool gs_plan(int64_t n0, int64_t n1, int64_t T, const int32_t* tile, int recursive, const int32_t* theta,
             GsPlanHost* out);

// Skewed-tile plan of a 2-D Jacobi star stencil (planner_gs.cpp, same orders
// and dependency rule): tiles of the skewed space (t, a, c) = (t, t + i,
// t + j), 0 <= t < T, 1 <= i <= n0, 1 <= j <= n1; tile = {kt, ha, wc} with
// ha, wc >= 2.  Every flow and two-buffer anti dependence has components in
// {0, 1, 2}, so the tiles are parallelograms that recompute nothing and
// depend only on their seven lower lattice neighbours.
bool skew_plan(int64_t n0, int64_t n1, int64_t T, const int32_t* tile, int recursive, const int32_t* theta,
               GsPlanHost* out);

// LU / Cholesky tile plan (planner_la.cpp): the non-empty tiles
// (kb * L + ib) * L + jb of the b x b x b lattice over the (k, i, j) space in
// execution order (lexicographic, or the recursive order when `recursive`),
// and per lattice id its number of predecessors in the tile graph of
// la_graph.h.
struct LaPlanHost {
    int32_t L = 0;
    std::vector<int32_t> queue;
    std::vector<int32_t> deps;
};
bool la_plan(int kind, int64_t n, int32_t b, int recursive, const int32_t* theta, LaPlanHost* out);

}  // namespace pcot
