// Internal interface between the kernel families and the dispatcher.
#pragma once

#include <cuda.h>

#include "kernels.h"

namespace pcot {

template <int U>
struct IC {
    static constexpr int value = U;
};

template <class T>
struct Vec;
template <>
struct Vec<float> {
    using V = float4;
    static constexpr int E = 4;
};
template <>
struct Vec<double> {
    using V = double2;
    static constexpr int E = 2;
};

template <class T>
inline Coeffs<T> coeffs_as(const double* c) {
    Coeffs<T> k;
    for (int i = 0; i < 7; ++i) k.c[i] = (T)c[i];
    return k;
}

// Release the dependency counters of the successors of lattice tile
// (b, i0, i1, i2): every (b+1, j) with |j_a - i_a| <= 1 inside the lattice.
// Called by thread 0 after a CTA barrier: one fence.acq_rel.gpu followed by
// relaxed reductions is a release pattern (cumulative), so the tile's stores
// by all threads of the CTA (ordered before the barrier) are visible to a CTA
// that observes a decrement with ld.acquire.gpu.  One fence per tile instead
// of one per counter: a fence waits for this SM's outstanding stores.
__device__ __forceinline__ void release_successors(const CotDev& q, int dims, int b, int i0, int i1, int i2) {
    if (b + 1 >= q.lattice[0]) return;
    __threadfence();
    const int L0 = q.lattice[1], L1 = q.lattice[2], L2 = q.lattice[3];
    for (int d0 = -1; d0 <= 1; ++d0) {
        const int j0 = i0 + d0;
        if (j0 < 0 || j0 >= L0) continue;
        for (int d1 = (dims > 1 ? -1 : 0); d1 <= (dims > 1 ? 1 : 0); ++d1) {
            const int j1 = i1 + d1;
            if (j1 < 0 || j1 >= L1) continue;
            for (int d2 = (dims > 2 ? -1 : 0); d2 <= (dims > 2 ? 1 : 0); ++d2) {
                const int j2 = i2 + d2;
                if (j2 < 0 || j2 >= L2) continue;
                const int id = (((b + 1) * L0 + j0) * L1 + j1) * L2 + j2;
                red_relaxed_add_gpu(q.counts + id, -1);
            }
        }
    }
}

// Pop the next queue entry and wait for its dependencies (thread 0 only).
// Returns the tile id, or -1 when the queue is exhausted or a wait gave up.
__device__ __forceinline__ int pop_and_wait(const CotDev& q) {
    const int pos = atomicAdd(q.head, 1);
    if (pos >= q.ntiles) return -1;
    const int tile = q.queue[pos];
    if (!wait_zero(q.counts + tile, q.status, q.timeout_ns, tile, pos)) return -1;
    return tile;  // wait_zero's ld.acquire.gpu orders this CTA's later reads (after the CTA barrier)
}

// ---- batched persistent launch (many 2-D grids, one kernel) -------------
// Per-grid descriptor, device resident.  Block b of grid g reads buf[b%2] and
// writes buf[(b+1)%2]; blocks < Pmain advance `depth` steps, later blocks one.
struct alignas(128) BatchDesc {
    CUtensorMap map[2];   // TMA maps of buf[0] and buf[1] (valid when tma_ok)
    void* buf[2];         // buf[0]: the caller's grid, buf[1]: its twin
    DevGeo g;
    int64_t H, Wt;        // tile height and width
    int32_t L0, L1;       // tiles along axis 0 and axis 1
    int32_t Pmain, Ptotal;
    int32_t count_base;   // first dependency counter of this grid
    int32_t ntiles;
    int32_t vec_ok, tma_ok;
    int32_t final_copy;   // odd block count: copy buf[1] back into buf[0] at the end
    int64_t span;         // elements spanned by the grid's layout
};

struct BatchDev {
    const BatchDesc* desc;
    const int2* queue;    // (grid, local tile id) in execution order
    int32_t* counts;
    int32_t* remaining;   // tiles left per grid
    int32_t* head;
    int64_t ntiles;
    uint64_t* done_ns;    // [0] start, [1+g] completion of grid g (may be NULL)
    DevStatus* status;
    uint64_t timeout_ns;
    int nb;
    int nbox, BW, box_elems, slot_elems;  // TMA ring geometry (common)
    int all_tma;                          // every grid uses the TMA ring
};

// Family entry points (one per kernel family).
namespace stream2d {
bool choose(const LaunchCtx& L, const int32_t* req, int depth, TileGeo* t);
int depths(int dtype, int* out, int cap);
cudaError_t slt(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst, DevStatus* st);
cudaError_t cot(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas);
int ctas_per_sm(const LaunchCtx& L, const TileGeo& t);
// Batched launch: common depth and warps, per-grid height.
bool batch_tiles(const LaunchCtx& L, int depth, int nwarps, int64_t H, TileGeo* t);
bool batch_desc_tma(const LaunchCtx& L, const TileGeo& t, BatchDesc* d, BatchDev* ring);
cudaError_t batch_launch(int dtype, int depth, int nwarps, const double* coeffs, const BatchDev& q, int nctas,
                         cudaStream_t s);
int batch_ctas_per_sm(int dtype, int depth, int nwarps, const BatchDev& q);
cudaError_t batch_ring_copy(int dtype, const BatchDev& q, cudaStream_t s);
cudaError_t batch_final_copy(int dtype, const BatchDev& q, cudaStream_t s);
}  // namespace stream2d

namespace stream3d {
bool choose(const LaunchCtx& L, const int32_t* req, int depth, TileGeo* t);
int depths(int dtype, int* out, int cap);
cudaError_t slt(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst);
cudaError_t cot(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas);
int ctas_per_sm(const LaunchCtx& L, const TileGeo& t);
size_t smem(const LaunchCtx& L, const TileGeo& t);
}  // namespace stream3d

namespace generic {
bool choose(const LaunchCtx& L, const int32_t* req, int depth, TileGeo* t);
cudaError_t slt(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst);
cudaError_t cot(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas);
int ctas_per_sm(const LaunchCtx& L, const TileGeo& t);
size_t smem(const LaunchCtx& L, const TileGeo& t);
}  // namespace generic

}  // namespace pcot
