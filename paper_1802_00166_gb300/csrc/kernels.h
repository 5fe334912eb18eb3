// Host-side launchers of the stencil kernels (implemented in the k_*.cu files).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace pcot {

enum DType { kF32 = 0, kF64 = 1, kF64Exact = 2 };

inline int dtype_size(int dt) { return dt == kF32 ? 4 : 8; }

// Everything a launch needs about the problem.
struct LaunchCtx {
    DevGeo geo;
    double coeffs[7];
    int dtype;
    cudaStream_t stream;
};

// Output-tile geometry of one time block (storage coordinates).
struct TileGeo {
    int64_t ext[kMaxDims];   // output extent of a tile per axis
    int64_t count[kMaxDims]; // tiles per axis
    int nwarps;              // warps per CTA (kernel specific)
    int depth;               // time steps per tile
    int family;              // kernel family, see below
};

enum Family { kFamGeneric = 0, kFamStream2D = 1, kFamStream3D = 2 };

// Device view of a persistent-executor plan (PCOT_COT).
struct CotDev {
    const int32_t* queue;  // tile ids in execution order
    int32_t* counts;       // remaining dependencies per tile id
    int32_t* head;         // next queue position to pop
    int64_t ntiles;
    int32_t lattice[kMaxDims + 1];  // blocks, tiles per axis (unused axes 1)
    DevStatus* status;
    uint64_t timeout_ns;
};

// ---- k_gs2d.cu: Gauss-Seidel 2-D tiles over the skewed (t, t+i, 2t+i+j) space ----
struct GsDev {
    const int32_t* queue;  // non-empty tile ids in execution order
    int32_t* counts;       // remaining predecessors per lattice id
    int32_t* head;         // next queue position to pop
    int64_t ntiles;
    int32_t lattice[3];    // tiles along t, a = t+i, c = 2t+i+j
    int32_t tile[3];       // kt, ha, wc (skewed points per tile)
    int64_t n0, n1, T;     // interior rows, columns, time steps
    int64_t pitch;         // row stride of the grid (elements)
    int32_t rows, cols;    // shared-memory window of a tile (halo included; cols padded)
    DevStatus* status;
    uint64_t timeout_ns;
};
// Window geometry of a tile (rows, padded columns) and its shared-memory bytes.
void gs2d_window(GsDev* q);
size_t gs2d_smem_bytes(int dtype, const GsDev& q);
int gs2d_ctas_per_sm(int dtype, const GsDev& q);
cudaError_t launch_gs2d(int dtype, void* grid, const GsDev& q, int nctas, cudaStream_t s);

// ---- k_skew2d.cu: 2-D Jacobi star stencil on parallelogram tiles of the skewed (t, t+i, t+j) space ----
struct SkewDev {
    const int32_t* queue;  // non-empty tile ids in execution order
    int32_t* counts;       // remaining predecessors per lattice id
    int32_t* head;         // next queue position to pop
    int64_t ntiles;
    int32_t lattice[3];    // tiles along t, a = t+i, c = t+j
    int32_t tile[3];       // kt, ha, wc (skewed points per tile)
    int64_t n0, n1, T;     // interior rows, columns, time steps
    int64_t pitch;         // row stride of both buffers (elements)
    int32_t rows, cols;    // shared-memory window of a tile (halo included)
    DevStatus* status;
    uint64_t timeout_ns;
};
// Window geometry of a tile and its shared-memory bytes (a window of each buffer).
void skew2d_window(SkewDev* q);
size_t skew2d_smem_bytes(int dtype, const SkewDev& q);
int skew2d_ctas_per_sm(int dtype, const SkewDev& q, int threads);
// buf0 holds the even time levels, buf1 the odd ones.
cudaError_t launch_skew2d(const LaunchCtx& L, void* buf0, void* buf1, const SkewDev& q, int nctas, int threads);

// ---- k_fdtd2d.cu: FDTD-2D (three fields, two copies) ----
struct FdDev {
    int64_t nx, ny;        // field rows and columns
    int64_t pitch;         // row stride (elements), the same for the three fields
    int32_t tile[2];       // output tile H x W of the tiled schedules
    int32_t depth;         // steps per block K (the shared-memory window has a halo of K)
};
size_t fdtd2d_smem_bytes(int dtype, const FdDev& q);
int fdtd2d_cot_ctas_per_sm(int dtype, const FdDev& q);
cudaError_t launch_fdtd2d_step(int dtype, const FdDev& q, void* const* src, void* const* dst, const void* fict,
                               int64_t t, cudaStream_t s);
cudaError_t launch_fdtd2d_block(int dtype, const FdDev& q, void* const* src, void* const* dst, const void* fict,
                                int64_t t0, int k, cudaStream_t s);
cudaError_t launch_fdtd2d_cot(int dtype, const FdDev& q, const CotDev& c, void* const* f0, void* const* f1,
                              const void* fict, int nctas, cudaStream_t s);

// ---- k_sweep.cu ----
cudaError_t launch_sweep(const LaunchCtx& L, const void* src, void* dst);
cudaError_t launch_ring_copy(const LaunchCtx& L, const void* src, void* dst);
// Copy the stored cells of the grid (the dims-shaped extent, ring included)
// from src to dst, row by row with the grid's strides: the padding between
// rows is neither read nor written.
cudaError_t launch_grid_copy(const LaunchCtx& L, const void* src, void* dst);
cudaError_t launch_grid_sum(const LaunchCtx& L, const void* grid, double* out, double* partials,
                            int npartials);
int grid_sum_partials();

// ---- tiled schedules ----
// Kernel family and tile geometry for (dims, dtype, requested tile, depth).
// Returns false when no kernel of this build supports the request.
bool choose_tiles(const LaunchCtx& L, const int32_t* req_tile, int depth, TileGeo* out);
// Depths a family has compiled variants for (ascending); returns the count.
int supported_depths(int family, int dtype, int* out, int cap);
// Time depth used when the caller leaves it open (0).
int default_depth(const LaunchCtx& L);
// The depth a tiled run uses for a requested depth k: k itself when a kernel
// of this build supports it with the requested tile, else the deepest
// compiled depth below k of the dims' fast family (at least 1).
int resolve_depth(const LaunchCtx& L, const int32_t* req_tile, int k);

// One single-level time block: all tiles of `t` read src, write dst.  `st`
// (may be NULL) is the status block bounded waits report to; without it the
// kernels use plain loads instead of the TMA ring.
cudaError_t launch_slt_block(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst, DevStatus* st);
// The persistent executor over a tile queue; block b reads buf[b%2], writes buf[(b+1)%2].
cudaError_t launch_cot(const LaunchCtx& L, const TileGeo& t, void* buf0, void* buf1,
                       const CotDev& q, int num_ctas);
// Resident CTAs per SM of the persistent executor for this geometry.
int cot_ctas_per_sm(const LaunchCtx& L, const TileGeo& t);
// Dynamic shared memory of one CTA for this geometry.
size_t tile_smem_bytes(const LaunchCtx& L, const TileGeo& t);

// ---- k_la.cu: blocked LU / Cholesky (tile graph in la_graph.h) ----
enum { kLaSweep = 0, kLaSlt = 1, kLaCot = 2 };
struct LaDev {
    double* A;             // n x n, row stride lda, factored in place
    int64_t lda, n;
    int32_t b;             // tile side (32 or 64)
    int32_t L;             // tiles per side, ceil(n / b)
    const int32_t* queue;  // recursive schedule: non-empty tile ids in execution order
    int32_t* counts;       // remaining predecessors per tile id (L^3)
    int32_t* head;         // next queue position to pop
    int64_t ntiles;
    DevStatus* status;
    uint64_t timeout_ns;
};
bool la_block_supported(int b);
// Resident CTAs per SM of the persistent kernel.
int la_ctas_per_sm(int b, bool fused, int kind);
// Runs the schedule (kLaSweep / kLaSlt / kLaCot) on `s`; *launches counts the
// kernel launches issued.
cudaError_t launch_la(const LaDev& d, int kind, bool fused, int schedule, int nctas, cudaStream_t s,
                      int64_t* launches);

// ---- k_mlp.cu ----
namespace mlp {
int param_count();
size_t scratch_bytes(int batch);
cudaError_t forward(const float* P, const float* X, int B, float* Y, cudaStream_t s);
cudaError_t grad(const float* P, const float* X, const float* Tg, int B, float* G, float* loss, void* scratch,
                 cudaStream_t s);
cudaError_t adam(float* P, const float* G, float* M, float* V, int n, int step, float lr, float b1, float b2,
                 float eps, cudaStream_t s);
cudaError_t argmin(const float* Y, int n, int stride, int col, int* out, cudaStream_t s);
}  // namespace mlp

// ---- k_misc ----
cudaError_t launch_wait_timeout_probe(int32_t* counter, DevStatus* st, uint64_t timeout_ns,
                                      cudaStream_t s);

}  // namespace pcot
