// Gauss-Seidel 2-D (GS-2D of Sec. 5.1.2) on the GPU: tiles of the skewed
// iteration space (t, a, c) = (t, t + i, 2t + i + j) run by a persistent
// kernel that pops a tile queue in order and waits (bounded) on per-tile
// dependency counters, the executor of the recursive schedule (Sec. 4.2)
// with the wavefront or recursive order built by planner_gs.cpp.
//
// A tile (kt x ha x wc skewed points) is computed in shared memory: the CTA
// copies the rectangle of grid cells its points read (rows i, columns j of
// the tile's parallelogram plus a halo of one) from global memory, sweeps
// the tile by wavefronts t + a + c = const (every dependence raises that sum
// by at least 1, so the points of one wavefront are independent), one thread
// per (t, a) pencil and one barrier per wavefront, updating the cells in
// place, and writes back the cells it updated.  Cells of the rectangle that
// the tile does not update belong to tiles that are predecessors (finished)
// or successors (not started) of this one, or to tiles with no dependence on
// it, whose cells this tile never reads or writes.
//
// Point update, in place: (sum of the 3 x 3 neighbourhood in row-major
// order, each add separately rounded) / 9, correctly rounded -- the same
// operations in the same order as the definition, so FP64 results are
// bitwise those of the plain loop nest.
#include "kernels.h"

namespace pcot {

namespace {

template <class T>
struct GsOps;
template <>
struct GsOps<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double avg(double s) { return __ddiv_rn(s, 9.0); }
};
template <>
struct GsOps<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float avg(float s) { return __fdiv_rn(s, 9.0f); }
};

__device__ __forceinline__ int gs_pop_and_wait(const GsDev& q) {
    const int pos = atomicAdd(q.head, 1);
    if (pos >= q.ntiles) return -1;
    const int tile = q.queue[pos];
    if (!wait_zero(q.counts + tile, q.status, q.timeout_ns, tile, pos)) return -1;
    return tile;
}

template <class T>
__global__ void __launch_bounds__(1024) gs2d_kernel(T* __restrict__ u, GsDev q) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* const sm = reinterpret_cast<T*>(smraw);
    unsigned char* const touched = smraw + sizeof(T) * (size_t)q.rows * q.cols;
    __shared__ int s_tile;
    const int kt = q.tile[0], ha = q.tile[1], wc = q.tile[2];
    const int R = q.rows, C = q.cols, cells = R * C;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int dt = tid / ha, da = tid - dt * ha;  // this thread's (t, a) pencil
    const int levels = kt + ha + wc - 2;
    for (;;) {
        if (tid == 0) s_tile = gs_pop_and_wait(q);
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) return;
        const int b2 = tile % q.lattice[2];
        const int r1 = tile / q.lattice[2];
        const int b1 = r1 % q.lattice[1];
        const int b0 = r1 / q.lattice[1];
        const int64_t t0 = (int64_t)b0 * kt, a0 = 1 + (int64_t)b1 * ha, c0 = 2 + (int64_t)b2 * wc;
        // window origin: the tile reads rows a-t-1 .. a-t+1 and columns
        // c-a-t-1 .. c-a-t+1 of its points (i = a - t, j = c - a - t)
        const int64_t i_lo = a0 - (t0 + kt - 1) - 1;
        const int64_t j_lo = c0 - (a0 + ha - 1) - (t0 + kt - 1) - 1;
        for (int k = tid; k < cells; k += nthr) {
            const int lr = k / C, lc = k - lr * C;
            const int64_t i = i_lo + lr, j = j_lo + lc;
            touched[k] = 0;
            if (i >= 0 && i <= q.n0 + 1 && j >= 0 && j <= q.n1 + 1) sm[k] = __ldcg(u + i * q.pitch + j);
        }
        __syncthreads();
        const int64_t t = t0 + dt, a = a0 + da, i = a - t;
        const bool pencil = dt < kt && t < q.T && i >= 1 && i <= q.n0;
        // local address of this pencil's point at dc = 0 (column j = c0 - a - t)
        const int base = (int)((i - i_lo) * C + (c0 - a - t - j_lo));
        const int64_t j0 = c0 - a - t;
        for (int lev = 0; lev < levels; ++lev) {
            const int dc = lev - dt - da;
            if (pencil && dc >= 0 && dc < wc && j0 + dc >= 1 && j0 + dc <= q.n1) {
                const int k = base + dc;
                const T* up = sm + k - C;
                const T* mid = sm + k;
                const T* dn = sm + k + C;
                using O = GsOps<T>;
                T s = O::add(up[-1], up[0]);
                s = O::add(s, up[1]);
                s = O::add(s, mid[-1]);
                s = O::add(s, mid[0]);
                s = O::add(s, mid[1]);
                s = O::add(s, dn[-1]);
                s = O::add(s, dn[0]);
                s = O::add(s, dn[1]);
                sm[k] = O::avg(s);
                touched[k] = 1;
            }
            __syncthreads();
        }
        for (int k = tid; k < cells; k += nthr) {
            if (!touched[k]) continue;
            const int lr = k / C, lc = k - lr * C;
            u[(i_lo + lr) * q.pitch + (j_lo + lc)] = sm[k];
        }
        __syncthreads();  // every thread's stores precede thread 0's release
        if (tid == 0) {
            __threadfence();  // one fence, then relaxed decrements: a release pattern
            for (int m = 1; m < 8; ++m) {
                const int s0 = b0 + ((m >> 2) & 1), s1 = b1 + ((m >> 1) & 1), s2 = b2 + (m & 1);
                if (s0 >= q.lattice[0] || s1 >= q.lattice[1] || s2 >= q.lattice[2]) continue;
                red_relaxed_add_gpu(q.counts + (s0 * q.lattice[1] + s1) * q.lattice[2] + s2, -1);
            }
        }
    }
}

}  // namespace

void gs2d_window(GsDev* q) {
    const int kt = q->tile[0], ha = q->tile[1], wc = q->tile[2];
    q->rows = ha + kt + 1;
    int cols = wc + ha + kt;
    if (((cols - 2) & 1) == 0) ++cols;  // odd row-to-row distance between a warp's lanes: no bank conflicts
    q->cols = cols;
}

size_t gs2d_smem_bytes(int dtype, const GsDev& q) {
    const size_t cells = (size_t)q.rows * q.cols;
    return cells * (size_t)dtype_size(dtype) + cells;
}

int gs2d_ctas_per_sm(int dtype, const GsDev& q) {
    const size_t sm = gs2d_smem_bytes(dtype, q);
    const int threads = q.tile[0] * q.tile[1];
    int n = 0;
    cudaError_t e;
    if (dtype == kF32) {
        e = cudaFuncSetAttribute(gs2d_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gs2d_kernel<float>, threads, sm);
    } else {
        e = cudaFuncSetAttribute(gs2d_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gs2d_kernel<double>, threads, sm);
    }
    return (e == cudaSuccess && n > 0) ? n : 0;
}

cudaError_t launch_gs2d(int dtype, void* grid, const GsDev& q, int nctas, cudaStream_t s) {
    const size_t sm = gs2d_smem_bytes(dtype, q);
    const int threads = q.tile[0] * q.tile[1];
    if (threads < 1 || threads > 1024) return cudaErrorInvalidConfiguration;
    if (dtype == kF32) {
        cudaError_t e = cudaFuncSetAttribute(gs2d_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        gs2d_kernel<float><<<nctas, threads, sm, s>>>((float*)grid, q);
    } else {
        cudaError_t e = cudaFuncSetAttribute(gs2d_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        gs2d_kernel<double><<<nctas, threads, sm, s>>>((double*)grid, q);
    }
    return cudaGetLastError();
}

}  // namespace pcot
