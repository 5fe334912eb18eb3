// 2-D Jacobi star stencil on parallelogram tiles of the skewed iteration
// space (t, a, c) = (t, t + i, t + j) -- the tiling of Sec. 3.1 after the skew
// of Sec. 4.3.2, in which every flow and two-buffer anti dependence has
// non-negative components -- run by a persistent kernel that pops a tile
// queue in order and waits (bounded) on per-tile dependency counters: the
// executor of the recursive schedule (Sec. 4.2), with the wavefront or
// recursive order built by planner_gs.cpp (skew_plan).
//
// Unlike the overlapped trapezoids of the stream kernels, these tiles
// recompute nothing: each point (t, i, j) belongs to exactly one tile.  A
// tile (kt x ha x wc skewed points) runs in shared memory.  Its points at
// step t form the ha x wc rectangle rows a - t, columns c - t, which moves up
// and left by one cell per step; the CTA copies the window those rectangles
// and their one-cell halo cover from BOTH buffers (level t lives in buffer
// t % 2), runs its steps there -- step t reads level t and writes level t + 1,
// all points of a step are independent, one barrier per step -- and writes
// back the cells it updated in each buffer (found from the tile's bounds).  When a tile starts, its
// predecessors have finished and its successors have not started, and the
// skew makes every value it reads either its own or a predecessor's: the
// window holds exactly what the loop nest would see (the two-buffer anti
// dependences also point forward, so nothing it writes is still needed by an
// earlier tile).  Every point applies the same rounded operations in the
// same order as the definition (upd2), so FP64 exact mode is bitwise the
// loop nest.
#include "kernels.h"

namespace pcot {

namespace {

__device__ __forceinline__ int skew_pop_and_wait(const SkewDev& q) {
    const int pos = atomicAdd(q.head, 1);
    if (pos >= q.ntiles) return -1;
    const int tile = q.queue[pos];
    if (pos < 0 || tile < 0 || tile >= q.lattice[0] * q.lattice[1] * q.lattice[2]) {
        if (atomicCAS(&q.status->code, 0, kStatusBounds) == 0) {
            q.status->info[0] = pos;
            q.status->info[1] = tile;
        }
        atomicExch(&q.status->abort, 1);
        return -1;
    }
    if (!wait_zero(q.counts + tile, q.status, q.timeout_ns, tile, pos)) return -1;
    return tile;  // wait_zero's ld.acquire.gpu orders this CTA's later reads (after the CTA barrier)
}

template <class T, bool EXACT>
__global__ void __launch_bounds__(512) skew2d_kernel(T* __restrict__ buf0, T* __restrict__ buf1, SkewDev q,
                                                     Coeffs<T> c) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int C = q.cols, cells = q.rows * q.cols;
    T* const s0 = reinterpret_cast<T*>(smraw);  // window of buffer 0 (even levels)
    T* const s1 = s0 + cells;                   // window of buffer 1 (odd levels)
    __shared__ int s_tile;
    const int kt = q.tile[0], ha = q.tile[1], wc = q.tile[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (;;) {
        if (tid == 0) s_tile = skew_pop_and_wait(q);
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) return;
        const int b2 = tile % q.lattice[2];
        const int r1 = tile / q.lattice[2];
        const int b1 = r1 % q.lattice[1];
        const int b0 = r1 / q.lattice[1];
        const int64_t t_lo = (int64_t)b0 * kt, a_lo = 1 + (int64_t)b1 * ha, c_lo = 1 + (int64_t)b2 * wc;
        const int64_t t_hi = (t_lo + kt < q.T ? t_lo + kt : q.T) - 1;
        // window origin: the rectangles reach up to row a_lo - t_hi and
        // column c_lo - t_hi, plus one cell of halo
        const int64_t i_lo = a_lo - t_hi - 1, j_lo = c_lo - t_hi - 1;
        // warps walk rows, lanes walk columns (coalesced along a row)
        for (int lr = warp; lr < q.rows; lr += nwarps) {
            const int64_t i = i_lo + lr;
            if (i < 0 || i > q.n0 + 1) continue;
            for (int lc = lane; lc < C; lc += 32) {
                const int64_t j = j_lo + lc;
                if (j >= 0 && j <= q.n1 + 1) {
                    s0[lr * C + lc] = __ldcg(buf0 + i * q.pitch + j);
                    s1[lr * C + lc] = __ldcg(buf1 + i * q.pitch + j);
                }
            }
        }
        __syncthreads();
        for (int64_t t = t_lo; t <= t_hi; ++t) {
            const T* const src = (t & 1) ? s1 : s0;  // level t
            T* const dst = (t & 1) ? s0 : s1;        // level t + 1
            const int64_t ia = a_lo - t > 1 ? a_lo - t : 1;
            const int64_t ib = a_lo + ha - 1 - t < q.n0 ? a_lo + ha - 1 - t : q.n0;
            const int64_t ja = c_lo - t > 1 ? c_lo - t : 1;
            const int64_t jb = c_lo + wc - 1 - t < q.n1 ? c_lo + wc - 1 - t : q.n1;
            if (ia <= ib && ja <= jb) {
                const int nr = (int)(ib - ia + 1), nc = (int)(jb - ja + 1);
                const int base = (int)((ia - i_lo) * C + (ja - j_lo));
                for (int r = warp; r < nr; r += nwarps)
                    for (int cc = lane; cc < nc; cc += 32) {
                        const int lk = base + r * C + cc;
                        dst[lk] = upd2<T, EXACT>(c, src[lk], src[lk - C], src[lk + C], src[lk - 1], src[lk + 1]);
                    }
            }
            __syncthreads();
        }
        // Write back the cells this tile updated, each buffer's last value.
        // Cell (i, j) is updated at the steps t with i + t in [a_lo, a_lo +
        // ha) and j + t in [c_lo, c_lo + wc), inside the tile's steps; step t
        // writes buffer (t + 1) % 2.
        for (int lr = warp; lr < q.rows; lr += nwarps) {
            const int64_t i = i_lo + lr;
            if (i < 1 || i > q.n0) continue;
            const int64_t ti_lo = a_lo - i, ti_hi = a_lo + ha - 1 - i;
            for (int lc = lane; lc < C; lc += 32) {
                const int64_t j = j_lo + lc;
                if (j < 1 || j > q.n1) continue;
                int64_t lo = t_lo > ti_lo ? t_lo : ti_lo;
                int64_t hi = t_hi < ti_hi ? t_hi : ti_hi;
                lo = lo > c_lo - j ? lo : c_lo - j;
                hi = hi < c_lo + wc - 1 - j ? hi : c_lo + wc - 1 - j;
                if (lo > hi) continue;
                const int k = lr * C + lc;
                const int64_t off = i * q.pitch + j;
                if (hi > lo || (lo & 1)) buf0[off] = s0[k];   // an odd step wrote buffer 0
                if (hi > lo || !(lo & 1)) buf1[off] = s1[k];  // an even step wrote buffer 1
            }
        }
        __syncthreads();  // every thread's stores precede thread 0's release
        if (tid == 0) {
            __threadfence();  // one fence, then relaxed decrements: a release pattern
            for (int m = 1; m < 8; ++m) {
                const int s0i = b0 + ((m >> 2) & 1), s1i = b1 + ((m >> 1) & 1), s2i = b2 + (m & 1);
                if (s0i >= q.lattice[0] || s1i >= q.lattice[1] || s2i >= q.lattice[2]) continue;
                red_relaxed_add_gpu(q.counts + (s0i * q.lattice[1] + s1i) * q.lattice[2] + s2i, -1);
            }
        }
    }
}

template <class T>
Coeffs<T> coeffs_as(const double* c) {
    Coeffs<T> k;
    for (int i = 0; i < 7; ++i) k.c[i] = (T)c[i];
    return k;
}

template <class T, bool EXACT>
cudaError_t launch_t(const LaunchCtx& L, void* b0, void* b1, const SkewDev& q, int nctas, int threads) {
    const size_t sm = skew2d_smem_bytes(L.dtype, q);
    cudaError_t e = cudaFuncSetAttribute(skew2d_kernel<T, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    skew2d_kernel<T, EXACT><<<nctas, threads, sm, L.stream>>>((T*)b0, (T*)b1, q, coeffs_as<T>(L.coeffs));
    return cudaGetLastError();
}

template <class T, bool EXACT>
int occupancy_t(size_t sm, int threads) {
    int n = 0;
    if (cudaFuncSetAttribute(skew2d_kernel<T, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, skew2d_kernel<T, EXACT>, threads, sm) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace

void skew2d_window(SkewDev* q) {
    q->rows = q->tile[1] + q->tile[0] + 1;
    q->cols = q->tile[2] + q->tile[0] + 1;
}

size_t skew2d_smem_bytes(int dtype, const SkewDev& q) {
    return 2 * (size_t)q.rows * q.cols * (size_t)dtype_size(dtype);
}

int skew2d_ctas_per_sm(int dtype, const SkewDev& q, int threads) {
    const size_t sm = skew2d_smem_bytes(dtype, q);
    switch (dtype) {
        case kF32: return occupancy_t<float, false>(sm, threads);
        case kF64: return occupancy_t<double, false>(sm, threads);
        default: return occupancy_t<double, true>(sm, threads);
    }
}

cudaError_t launch_skew2d(const LaunchCtx& L, void* buf0, void* buf1, const SkewDev& q, int nctas, int threads) {
    if (threads < 32 || threads > 512 || threads % 32 != 0 || nctas < 1) return cudaErrorInvalidConfiguration;
    switch (L.dtype) {
        case kF32: return launch_t<float, false>(L, buf0, buf1, q, nctas, threads);
        case kF64: return launch_t<double, false>(L, buf0, buf1, q, nctas, threads);
        default: return launch_t<double, true>(L, buf0, buf1, q, nctas, threads);
    }
}

}  // namespace pcot
