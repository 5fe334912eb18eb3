// FDTD-2D (the two-dimensional FDTD kernel of Sec. 5.1.2) on the GPU.
//
// One time step t of the three fields (nx x ny each, row stride s):
//   ey[0][j] = fict[t];  ey[i][j] -= 0.5 (hz[i][j] - hz[i-1][j])   (i >= 1)
//   ex[i][j] -= 0.5 (hz[i][j] - hz[i][j-1])                          (j >= 1)
//   hz[i][j] -= 0.7 (((ex'[i][j+1] - ex'[i][j]) + ey'[i+1][j]) - ey'[i][j])
//                                                       (i <= nx-2, j <= ny-2)
// where ex', ey' are the step's new electric fields.  Every product and
// difference is a separately rounded operation in that order (no fused
// multiply-add), so FP64 results are bitwise those of the loop nest and FP32
// rounds the same operations to binary32.
//
// Three schedules, all on two copies of the fields (the caller's and a
// workspace twin; a step or block reads one copy and writes the other):
//  * sweep: one launch per step; a thread recomputes the two neighbouring
//    electric values its hz update needs (the same operations, hence the
//    same bits as their owners compute);
//  * single-level: tiles of H x W outputs advanced k steps in shared memory
//    (the overlapped tile of Sec. 3.3: every step's valid region shrinks by
//    one cell per side, so a tile loads a halo of k), one launch per block;
//  * recursive: the same tiles as leaves of the persistent executor over the
//    skewed (block, tile) lattice (Sec. 4), one launch for all full blocks.
#include "kernels.h"
#include "tiled.cuh"

namespace pcot {

namespace {

template <class T>
struct FdOps;
template <>
struct FdOps<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static constexpr double kHalf = 0.5, kCoef = 0.7;
};
template <>
struct FdOps<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static constexpr float kHalf = 0.5f, kCoef = 0.7f;
};

// e - 0.5 (h - hn)
template <class T>
__device__ __forceinline__ T e_upd(T e, T h, T hn) {
    using O = FdOps<T>;
    return O::sub(e, O::mul(O::kHalf, O::sub(h, hn)));
}
// h - 0.7 (((exe - ex0) + eys) - ey0)
template <class T>
__device__ __forceinline__ T h_upd(T h, T exe, T ex0, T eys, T ey0) {
    using O = FdOps<T>;
    return O::sub(h, O::mul(O::kCoef, O::sub(O::add(O::sub(exe, ex0), eys), ey0)));
}

template <class T>
__global__ void __launch_bounds__(256) fdtd_step_kernel(FdDev q, const T* __restrict__ ex, const T* __restrict__ ey,
                                                        const T* __restrict__ hz, T* __restrict__ ex2,
                                                        T* __restrict__ ey2, T* __restrict__ hz2,
                                                        const T* __restrict__ fict, int64_t t) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = blockIdx.y;
    if (j >= q.ny || i >= q.nx) return;
    const int64_t s = q.pitch, k = i * s + j;
    const T h = hz[k];
    const T eyn = i == 0 ? fict[t] : e_upd(ey[k], h, hz[k - s]);
    const T exn = j == 0 ? ex[k] : e_upd(ex[k], h, hz[k - 1]);
    T hn = h;
    if (i <= q.nx - 2 && j <= q.ny - 2) {
        const T exe = e_upd(ex[k + 1], hz[k + 1], h);       // ex'[i][j+1] (j+1 >= 1)
        const T eys = e_upd(ey[k + s], hz[k + s], h);       // ey'[i+1][j] (i+1 >= 1)
        hn = h_upd(h, exe, exn, eys, eyn);
    }
    ex2[k] = exn;
    ey2[k] = eyn;
    hz2[k] = hn;
}

// k steps of one H x W output tile in shared memory; (i0, j0) is the tile's
// first output cell, t0 its first step.  The window is (H+2k) x (W+2k).
template <class T>
__device__ __forceinline__ void fdtd_tile(const FdDev& q, const T* __restrict__ ex, const T* __restrict__ ey,
                                          const T* __restrict__ hz, T* __restrict__ ex2, T* __restrict__ ey2,
                                          T* __restrict__ hz2, const T* __restrict__ fict, int64_t t0, int k,
                                          int64_t i0, int64_t j0, T* sm, bool cg) {
    const int H = q.tile[0], W = q.tile[1], K = q.depth;  // window sized for the block depth K (a tail block runs k < K)
    const int Hs = H + 2 * K, Ws = W + 2 * K, cells = Hs * Ws;
    T* sx = sm;
    T* sy = sm + cells;
    T* sh = sm + 2 * cells;
    const int64_t wi = i0 - K, wj = j0 - K;  // window origin (global)
    // Each thread walks the window's cells tid, tid + n, ... in row-major
    // order; the (row, column) of the next cell follows by a fixed step, so the
    // loops carry no index division.
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int drow = nthr / Ws, dcol = nthr - drow * Ws;
    const int li0 = tid / Ws, lj0 = tid - li0 * Ws;
    const int64_t s = q.pitch;
    for (int c = tid, li = li0, lj = lj0; c < cells; c += nthr) {
        const int64_t i = wi + li, j = wj + lj;
        T vx = T(0), vy = T(0), vh = T(0);
        if (i >= 0 && i < q.nx && j >= 0 && j < q.ny) {
            const int64_t g = i * s + j;
            if (cg) {
                vx = __ldcg(ex + g);
                vy = __ldcg(ey + g);
                vh = __ldcg(hz + g);
            } else {
                vx = ex[g];
                vy = ey[g];
                vh = hz[g];
            }
        }
        sx[c] = vx;
        sy[c] = vy;
        sh[c] = vh;
        li += drow;
        lj += dcol;
        if (lj >= Ws) {
            lj -= Ws;
            ++li;
        }
    }
    __syncthreads();
    for (int st = 0; st < k; ++st) {
        const T src = fict[t0 + st];
        // electric fields from the magnetic field of the previous step
        for (int c = tid, li = li0, lj = lj0; c < cells; c += nthr) {
            const int64_t i = wi + li, j = wj + lj;
            if (i >= 0 && i < q.nx && j >= 0 && j < q.ny) {
                if (i == 0) sy[c] = src;
                else if (li >= 1) sy[c] = e_upd(sy[c], sh[c], sh[c - Ws]);
                if (j >= 1 && lj >= 1) sx[c] = e_upd(sx[c], sh[c], sh[c - 1]);
            }
            li += drow;
            lj += dcol;
            if (lj >= Ws) {
                lj -= Ws;
                ++li;
            }
        }
        __syncthreads();
        // magnetic field from the new electric fields
        for (int c = tid, li = li0, lj = lj0; c < cells; c += nthr) {
            const int64_t i = wi + li, j = wj + lj;
            if (i >= 0 && i <= q.nx - 2 && j >= 0 && j <= q.ny - 2 && li + 1 < Hs && lj + 1 < Ws)
                sh[c] = h_upd(sh[c], sx[c + 1], sx[c], sy[c + Ws], sy[c]);
            li += drow;
            lj += dcol;
            if (lj >= Ws) {
                lj -= Ws;
                ++li;
            }
        }
        __syncthreads();
    }
    // the tile's outputs (valid: k cells from every window edge)
    const int lane = tid & 31, wrp = tid >> 5, nw = nthr >> 5;
    for (int oi = wrp; oi < H; oi += nw) {
        const int64_t i = i0 + oi;
        if (i >= q.nx) break;
        for (int oj = lane; oj < W; oj += 32) {
            const int64_t j = j0 + oj;
            if (j >= q.ny) break;
            const int w = (oi + K) * Ws + (oj + K);
            const int64_t g = i * s + j;
            ex2[g] = sx[w];
            ey2[g] = sy[w];
            hz2[g] = sh[w];
        }
    }
}

template <class T>
__global__ void __launch_bounds__(256) fdtd_slt_kernel(FdDev q, const T* ex, const T* ey, const T* hz, T* ex2, T* ey2,
                                                       T* hz2, const T* fict, int64_t t0, int k) {
    extern __shared__ __align__(16) unsigned char smraw[];
    fdtd_tile<T>(q, ex, ey, hz, ex2, ey2, hz2, fict, t0, k, (int64_t)blockIdx.y * q.tile[0],
                 (int64_t)blockIdx.x * q.tile[1], reinterpret_cast<T*>(smraw), false);
}

// Persistent executor: block b of the lattice reads copy b%2 and writes copy
// (b+1)%2; tile (b, iy, ix) waits for the tiles of block b-1 at lattice
// distance <= 1 (they wrote its input window and read the cells it
// overwrites) and releases those of block b+1.
template <class T>
__global__ void __launch_bounds__(256) fdtd_cot_kernel(FdDev q, CotDev c, T* ex0, T* ey0, T* hz0, T* ex1, T* ey1,
                                                       T* hz1, const T* fict) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = pop_and_wait(c);
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) return;
        const int L1 = c.lattice[2], L0 = c.lattice[1];
        const int ix = tile % L1;
        const int rest = tile / L1;
        const int iy = rest % L0;
        const int b = rest / L0;
        const bool odd = (b & 1) != 0;
        fdtd_tile<T>(q, odd ? ex1 : ex0, odd ? ey1 : ey0, odd ? hz1 : hz0, odd ? ex0 : ex1, odd ? ey0 : ey1,
                     odd ? hz0 : hz1, fict, (int64_t)b * q.depth, q.depth, (int64_t)iy * q.tile[0],
                     (int64_t)ix * q.tile[1], reinterpret_cast<T*>(smraw), true);
        __syncthreads();  // the tile's stores by every thread precede thread 0's release
        if (threadIdx.x == 0) release_successors(c, 2, b, iy, ix, 0);
    }
}

}  // namespace

size_t fdtd2d_smem_bytes(int dtype, const FdDev& q) {
    return (size_t)3 * (q.tile[0] + 2 * q.depth) * (q.tile[1] + 2 * q.depth) * dtype_size(dtype);
}

cudaError_t launch_fdtd2d_step(int dtype, const FdDev& q, void* const* src, void* const* dst, const void* fict,
                               int64_t t, cudaStream_t s) {
    if (q.nx > 65535) return cudaErrorInvalidConfiguration;
    dim3 grd((unsigned)((q.ny + 255) / 256), (unsigned)q.nx);
    if (dtype == kF32)
        fdtd_step_kernel<float><<<grd, 256, 0, s>>>(q, (const float*)src[0], (const float*)src[1],
                                                    (const float*)src[2], (float*)dst[0], (float*)dst[1],
                                                    (float*)dst[2], (const float*)fict, t);
    else
        fdtd_step_kernel<double><<<grd, 256, 0, s>>>(q, (const double*)src[0], (const double*)src[1],
                                                     (const double*)src[2], (double*)dst[0], (double*)dst[1],
                                                     (double*)dst[2], (const double*)fict, t);
    return cudaGetLastError();
}

cudaError_t launch_fdtd2d_block(int dtype, const FdDev& q, void* const* src, void* const* dst, const void* fict,
                                int64_t t0, int k, cudaStream_t s) {
    const size_t sm = fdtd2d_smem_bytes(dtype, q);
    const int64_t gy = (q.nx + q.tile[0] - 1) / q.tile[0], gx = (q.ny + q.tile[1] - 1) / q.tile[1];
    if (gy > 65535 || gx > (1LL << 31) - 1 || k < 1 || k > q.depth) return cudaErrorInvalidConfiguration;
    dim3 grd((unsigned)gx, (unsigned)gy);
    cudaError_t e;
    if (dtype == kF32) {
        e = cudaFuncSetAttribute(fdtd_slt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        fdtd_slt_kernel<float><<<grd, 256, sm, s>>>(q, (const float*)src[0], (const float*)src[1],
                                                    (const float*)src[2], (float*)dst[0], (float*)dst[1],
                                                    (float*)dst[2], (const float*)fict, t0, k);
    } else {
        e = cudaFuncSetAttribute(fdtd_slt_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        fdtd_slt_kernel<double><<<grd, 256, sm, s>>>(q, (const double*)src[0], (const double*)src[1],
                                                     (const double*)src[2], (double*)dst[0], (double*)dst[1],
                                                     (double*)dst[2], (const double*)fict, t0, k);
    }
    return cudaGetLastError();
}

int fdtd2d_cot_ctas_per_sm(int dtype, const FdDev& q) {
    const size_t sm = fdtd2d_smem_bytes(dtype, q);
    int n = 0;
    cudaError_t e;
    if (dtype == kF32) {
        e = cudaFuncSetAttribute(fdtd_cot_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fdtd_cot_kernel<float>, 256, sm);
    } else {
        e = cudaFuncSetAttribute(fdtd_cot_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fdtd_cot_kernel<double>, 256, sm);
    }
    return (e == cudaSuccess && n > 0) ? n : 0;
}

cudaError_t launch_fdtd2d_cot(int dtype, const FdDev& q, const CotDev& c, void* const* f0, void* const* f1,
                              const void* fict, int nctas, cudaStream_t s) {
    const size_t sm = fdtd2d_smem_bytes(dtype, q);
    cudaError_t e;
    if (dtype == kF32) {
        e = cudaFuncSetAttribute(fdtd_cot_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        fdtd_cot_kernel<float><<<nctas, 256, sm, s>>>(q, c, (float*)f0[0], (float*)f0[1], (float*)f0[2],
                                                      (float*)f1[0], (float*)f1[1], (float*)f1[2],
                                                      (const float*)fict);
    } else {
        e = cudaFuncSetAttribute(fdtd_cot_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        fdtd_cot_kernel<double><<<nctas, 256, sm, s>>>(q, c, (double*)f0[0], (double*)f0[1], (double*)f0[2],
                                                       (double*)f1[0], (double*)f1[1], (double*)f1[2],
                                                       (const double*)fict);
    }
    return cudaGetLastError();
}

}  // namespace pcot
