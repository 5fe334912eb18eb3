// Plain single-sweep kernels (one launch = one time step over the whole
// grid), the Dirichlet ring copy, the FP64 interior sum and the wait probe.
//
// The sweep is the untiled loop nest of the paper's problem statement
// (Sec. 4.1): every interior point of step t+1 from the 2r+1 neighbours of
// step t along each axis, buffers alternating by t%2 (Appendix A example).
#include "tiled.cuh"

namespace pcot {

namespace {

template <class T, bool EXACT>
__global__ void __launch_bounds__(256) sweep1d_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                      DevGeo g, Coeffs<T> c) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = g.n[0];
    if (i >= n) return;
    int64_t x, xm, xp;
    if (g.periodic) {
        x = i;
        xm = i == 0 ? n - 1 : i - 1;
        xp = i == n - 1 ? 0 : i + 1;
    } else {
        x = i + 1;
        xm = i;
        xp = i + 2;
    }
    dst[x] = upd1<T, EXACT>(c, __ldg(src + x), __ldg(src + xm), __ldg(src + xp));
}

// Thread = one column x, ROWS consecutive rows (register reuse along axis 0).
template <class T, bool EXACT, int ROWS>
__global__ void __launch_bounds__(256) sweep2d_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                      DevGeo g, Coeffs<T> c) {
    const int64_t ix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t iy0 = ((int64_t)blockIdx.y * blockDim.y + threadIdx.y) * ROWS;
    const int64_t ny = g.n[0], nx = g.n[1];
    if (ix >= nx || iy0 >= ny) return;
    const bool per = g.periodic != 0;
    const int64_t P = g.s[0];
    int64_t x, xm, xp;
    if (per) {
        x = ix;
        xm = ix == 0 ? nx - 1 : ix - 1;
        xp = ix == nx - 1 ? 0 : ix + 1;
    } else {
        x = ix + 1;
        xm = ix;
        xp = ix + 2;
    }
    auto row = [&](int64_t iy) -> int64_t { return per ? wrap_fast(iy, ny) : iy + 1; };
    T N = __ldg(src + row(iy0 - 1) * P + x);
    T C = __ldg(src + row(iy0) * P + x);
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int64_t iy = iy0 + r;
        if (iy >= ny) break;
        const int64_t rs = row(iy) * P;
        const T S = __ldg(src + row(iy + 1) * P + x);
        const T W = __ldg(src + rs + xm);
        const T E = __ldg(src + rs + xp);
        dst[rs + x] = upd2<T, EXACT>(c, C, N, S, W, E);
        N = C;
        C = S;
    }
}

// Thread = one (y, x) column, ZR consecutive planes along axis 0.
template <class T, bool EXACT, int ZR>
__global__ void __launch_bounds__(256) sweep3d_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                      DevGeo g, Coeffs<T> c) {
    const int64_t ix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t iy = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
    const int64_t iz0 = (int64_t)blockIdx.z * ZR;
    const int64_t nz = g.n[0], ny = g.n[1], nx = g.n[2];
    if (ix >= nx || iy >= ny) return;
    const bool per = g.periodic != 0;
    const int64_t Pz = g.s[0], Py = g.s[1];
    int64_t x, xm, xp, y, ym, yp;
    if (per) {
        x = ix;
        xm = ix == 0 ? nx - 1 : ix - 1;
        xp = ix == nx - 1 ? 0 : ix + 1;
        y = iy;
        ym = iy == 0 ? ny - 1 : iy - 1;
        yp = iy == ny - 1 ? 0 : iy + 1;
    } else {
        x = ix + 1;
        xm = ix;
        xp = ix + 2;
        y = iy + 1;
        ym = iy;
        yp = iy + 2;
    }
    auto plane = [&](int64_t iz) -> int64_t { return (per ? wrap_fast(iz, nz) : iz + 1) * Pz; };
    T D = __ldg(src + plane(iz0 - 1) + y * Py + x);
    T C = __ldg(src + plane(iz0) + y * Py + x);
#pragma unroll
    for (int r = 0; r < ZR; ++r) {
        const int64_t iz = iz0 + r;
        if (iz >= nz) break;
        const int64_t ps = plane(iz);
        const T U = __ldg(src + plane(iz + 1) + y * Py + x);
        const T N = __ldg(src + ps + ym * Py + x);
        const T S = __ldg(src + ps + yp * Py + x);
        const T W = __ldg(src + ps + y * Py + xm);
        const T E = __ldg(src + ps + y * Py + xp);
        dst[ps + y * Py + x] = upd3<T, EXACT>(c, C, D, U, N, S, W, E);
        D = C;
        C = U;
    }
}


// Vectorised sweeps: a warp covers 32*E contiguous storage columns (one
// 16-byte vector per lane) of R rows (2-D) or R planes of one row (3-D); every
// row it needs is loaded up front so R+2 (2-D) or 3R+2 (3-D) vector loads per
// lane are in flight; x-neighbours come from warp shuffles plus one scalar
// load at each end of the span.  Used when rows are 16-byte aligned and, for
// periodic grids, the contiguous extent is a multiple of the warp span.
template <class T, bool EXACT, int R>
__global__ void __launch_bounds__(256, 4) sweep2d_vec_kernel(const T* __restrict__ src, T* __restrict__ dst, DevGeo g,
                                                          Coeffs<T> c) {
    constexpr int E = Vec<T>::E;
    using V = typename Vec<T>::V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool per = g.periodic != 0;
    const int64_t ny = g.n[0], nx = g.n[1], ex = g.e[1], P = g.s[0];
    const int64_t off = per ? 0 : 1;
    const int64_t x0 = (int64_t)blockIdx.x * (32 * E);
    const int64_t xl = x0 + lane * E;
    const int64_t iy0 = ((int64_t)blockIdx.y * (blockDim.x >> 5) + warp) * R;  // first interior row
    if (iy0 >= ny) return;
    auto srow = [&](int64_t iy) -> int64_t { return per ? wrap_fast(iy, ny) : iy + 1; };
    const bool full = xl + E <= ex;
    T v[R + 2][E];
#pragma unroll
    for (int i = 0; i < R + 2; ++i) {
        const int64_t iy = iy0 - 1 + i;
        const bool ok = iy <= ny;  // rows past the far ring are never needed
        const T* rp = src + srow(iy) * P;
        if (ok && full) {
            const V q = __ldg(reinterpret_cast<const V*>(rp + xl));
            const T* qq = reinterpret_cast<const T*>(&q);
#pragma unroll
            for (int j = 0; j < E; ++j) v[i][j] = qq[j];
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) v[i][j] = (ok && xl + j < ex) ? __ldg(rp + xl + j) : T(0);
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int64_t iy = iy0 + i;
        if (iy >= ny) break;
        const T* rp = src + srow(iy) * P;
        T wl = __shfl_up_sync(0xffffffffu, v[i + 1][E - 1], 1);
        T er = __shfl_down_sync(0xffffffffu, v[i + 1][0], 1);
        if (lane == 0) {
            const int64_t xm = x0 - 1;
            wl = per ? __ldg(rp + wrap_fast(xm, nx)) : (xm >= 0 ? __ldg(rp + xm) : T(0));
        }
        if (lane == 31) {
            const int64_t xp = x0 + 32 * E;
            er = per ? __ldg(rp + wrap_fast(xp, nx)) : (xp < ex ? __ldg(rp + xp) : T(0));
        }
        T out[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const T W = j > 0 ? v[i + 1][j - 1] : wl;
            const T Ea = j < E - 1 ? v[i + 1][j + 1] : er;
            out[j] = upd2<T, EXACT>(c, v[i + 1][j], v[i][j], v[i + 2][j], W, Ea);
        }
        T* wp = dst + (iy + off) * P;
        bool all = true;
#pragma unroll
        for (int j = 0; j < E; ++j) all = all && (xl + j >= off) && (xl + j < off + nx);
        if (all) {
            V q;
            T* qq = reinterpret_cast<T*>(&q);
#pragma unroll
            for (int j = 0; j < E; ++j) qq[j] = out[j];
            *reinterpret_cast<V*>(wp + xl) = q;
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j)
                if (xl + j >= off && xl + j < off + nx) wp[xl + j] = out[j];
        }
    }
}

template <class T, bool EXACT, int R>
__global__ void __launch_bounds__(256, 4) sweep3d_vec_kernel(const T* __restrict__ src, T* __restrict__ dst, DevGeo g,
                                                          Coeffs<T> c) {
    constexpr int E = Vec<T>::E;
    using V = typename Vec<T>::V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool per = g.periodic != 0;
    const int64_t nz = g.n[0], ny = g.n[1], nx = g.n[2], ex = g.e[2], Pz = g.s[0], Py = g.s[1];
    const int64_t off = per ? 0 : 1;
    const int64_t x0 = (int64_t)blockIdx.x * (32 * E);
    const int64_t xl = x0 + lane * E;
    const int64_t iy = (int64_t)blockIdx.y * (blockDim.x >> 5) + warp;
    const int64_t iz0 = (int64_t)blockIdx.z * R;
    if (iy >= ny) return;
    auto sz = [&](int64_t iz) -> int64_t { return per ? wrap_fast(iz, nz) : iz + 1; };
    auto sy = [&](int64_t jy) -> int64_t { return per ? wrap_fast(jy, ny) : jy + 1; };
    const bool full = xl + E <= ex;
    auto ld = [&](int64_t base, T (&v)[E], bool ok) {
        if (ok && full) {
            const V q = __ldg(reinterpret_cast<const V*>(src + base + xl));
            const T* qq = reinterpret_cast<const T*>(&q);
#pragma unroll
            for (int j = 0; j < E; ++j) v[j] = qq[j];
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) v[j] = (ok && xl + j < ex) ? __ldg(src + base + xl + j) : T(0);
        }
    };
    const int64_t yc = sy(iy) * Py, yn = sy(iy - 1) * Py, ys = sy(iy + 1) * Py;
    T C[R + 2][E], N[R][E], S[R][E];
#pragma unroll
    for (int i = 0; i < R + 2; ++i) ld(sz(iz0 - 1 + i) * Pz + yc, C[i], iz0 - 1 + i <= nz);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const bool ok = iz0 + i < nz;
        ld(sz(iz0 + i) * Pz + yn, N[i], ok);
        ld(sz(iz0 + i) * Pz + ys, S[i], ok);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int64_t iz = iz0 + i;
        if (iz >= nz) break;
        const T* rp = src + sz(iz) * Pz + yc;
        T wl = __shfl_up_sync(0xffffffffu, C[i + 1][E - 1], 1);
        T er = __shfl_down_sync(0xffffffffu, C[i + 1][0], 1);
        if (lane == 0) {
            const int64_t xm = x0 - 1;
            wl = per ? __ldg(rp + wrap_fast(xm, nx)) : (xm >= 0 ? __ldg(rp + xm) : T(0));
        }
        if (lane == 31) {
            const int64_t xp = x0 + 32 * E;
            er = per ? __ldg(rp + wrap_fast(xp, nx)) : (xp < ex ? __ldg(rp + xp) : T(0));
        }
        T out[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const T W = j > 0 ? C[i + 1][j - 1] : wl;
            const T Ea = j < E - 1 ? C[i + 1][j + 1] : er;
            out[j] = upd3<T, EXACT>(c, C[i + 1][j], C[i][j], C[i + 2][j], N[i][j], S[i][j], W, Ea);
        }
        T* wp = dst + sz(iz) * Pz + yc;
        bool all = true;
#pragma unroll
        for (int j = 0; j < E; ++j) all = all && (xl + j >= off) && (xl + j < off + nx);
        if (all) {
            V q;
            T* qq = reinterpret_cast<T*>(&q);
#pragma unroll
            for (int j = 0; j < E; ++j) qq[j] = out[j];
            *reinterpret_cast<V*>(wp + xl) = q;
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j)
                if (xl + j >= off && xl + j < off + nx) wp[xl + j] = out[j];
        }
    }
}

template <class T>
bool sweep_vec_ok(const DevGeo& g, const void* a, const void* b) {
    constexpr int E = Vec<T>::E;
    if (((uintptr_t)a & 15) || ((uintptr_t)b & 15)) return false;
    for (int d = 0; d < g.dims - 1; ++d)
        if ((g.s[d] * (int64_t)sizeof(T)) & 15) return false;
    if (g.periodic && (g.n[g.dims - 1] % (32 * E)) != 0) return false;
    return g.dims >= 2;
}

template <class T>
Coeffs<T> make_coeffs(const double* c) {
    Coeffs<T> k;
    for (int i = 0; i < 7; ++i) k.c[i] = (T)c[i];
    return k;
}

template <class T, bool EXACT>
cudaError_t sweep_t(const LaunchCtx& L, const void* src, void* dst) {
    const DevGeo& g = L.geo;
    const Coeffs<T> c = make_coeffs<T>(L.coeffs);
    const T* s = (const T*)src;
    T* d = (T*)dst;
    if (g.dims == 1) {
        dim3 blk(256), grd((unsigned)((g.n[0] + 255) / 256));
        sweep1d_kernel<T, EXACT><<<grd, blk, 0, L.stream>>>(s, d, g, c);
    } else if (g.dims == 2 && sweep_vec_ok<T>(g, src, dst)) {
        constexpr int R = 4;
        constexpr int E = Vec<T>::E;
        dim3 grd((unsigned)((g.e[1] + 32 * E - 1) / (32 * E)), (unsigned)((g.n[0] + 8 * R - 1) / (8 * R)));
        if (grd.y > 65535) return cudaErrorInvalidConfiguration;
        sweep2d_vec_kernel<T, EXACT, R><<<grd, 256, 0, L.stream>>>(s, d, g, c);
    } else if (g.dims == 3 && sweep_vec_ok<T>(g, src, dst)) {
        constexpr int R = 2;
        constexpr int E = Vec<T>::E;
        dim3 grd((unsigned)((g.e[2] + 32 * E - 1) / (32 * E)), (unsigned)((g.n[1] + 7) / 8),
                 (unsigned)((g.n[0] + R - 1) / R));
        if (grd.y > 65535 || grd.z > 65535) return cudaErrorInvalidConfiguration;
        sweep3d_vec_kernel<T, EXACT, R><<<grd, 256, 0, L.stream>>>(s, d, g, c);
    } else if (g.dims == 2) {
        constexpr int ROWS = 4;
        dim3 blk(32, 8);
        dim3 grd((unsigned)((g.n[1] + 31) / 32), (unsigned)((g.n[0] + 8 * ROWS - 1) / (8 * ROWS)));
        if (grd.y > 65535) return cudaErrorInvalidConfiguration;
        sweep2d_kernel<T, EXACT, ROWS><<<grd, blk, 0, L.stream>>>(s, d, g, c);
    } else {
        constexpr int ZR = 4;
        dim3 blk(32, 8);
        dim3 grd((unsigned)((g.n[2] + 31) / 32), (unsigned)((g.n[1] + 7) / 8), (unsigned)((g.n[0] + ZR - 1) / ZR));
        if (grd.y > 65535 || grd.z > 65535) return cudaErrorInvalidConfiguration;
        sweep3d_kernel<T, EXACT, ZR><<<grd, blk, 0, L.stream>>>(s, d, g, c);
    }
    return cudaGetLastError();
}

// Copy every cell on the outer faces (the Dirichlet ring of width 1).
template <class T>
__global__ void ring_copy_kernel(const T* __restrict__ src, T* __restrict__ dst, DevGeo g, int64_t total) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        // Enumerate faces: for axis a, two sides, all combinations of the other axes.
        int64_t rem = k;
        int a = 0;
        int64_t face = 0;
        for (a = 0; a < g.dims; ++a) {
            face = 1;
            for (int b = 0; b < g.dims; ++b)
                if (b != a) face *= g.e[b];
            if (rem < 2 * face) break;
            rem -= 2 * face;
        }
        if (a >= g.dims) continue;
        const int side = rem >= face ? 1 : 0;
        int64_t r = rem - side * face;
        int64_t coord[kMaxDims] = {0, 0, 0};
        for (int b = g.dims - 1; b >= 0; --b) {
            if (b == a) continue;
            coord[b] = r % g.e[b];
            r /= g.e[b];
        }
        coord[a] = side ? g.e[a] - 1 : 0;
        int64_t off = 0;
        for (int b = 0; b < g.dims; ++b) off += coord[b] * g.s[b];
        dst[off] = src[off];
    }
}

// Deterministic FP64 sum of the interior: fixed blocks, fixed per-thread
// order, fixed tree order in shared memory, then one block over the partials.
template <class T>
__global__ void __launch_bounds__(256) sum_partial_kernel(const T* __restrict__ grid, DevGeo g, double* partials) {
    __shared__ double sh[256];
    const int64_t last = g.n[g.dims - 1];
    int64_t rows = 1;
    for (int a = 0; a < g.dims - 1; ++a) rows *= g.n[a];
    const int64_t off = g.periodic ? 0 : 1;
    double acc = 0.0;
    for (int64_t rw = blockIdx.x; rw < rows; rw += gridDim.x) {
        int64_t rr = rw, base = 0;
        for (int a = g.dims - 2; a >= 0; --a) {
            base += (rr % g.n[a] + off) * g.s[a];
            rr /= g.n[a];
        }
        for (int64_t x = threadIdx.x; x < last; x += blockDim.x) acc += (double)grid[base + x + off];
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) sum_final_kernel(const double* partials, int np, double* out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void wait_probe_kernel(int32_t* counter, DevStatus* st, uint64_t timeout_ns) {
    if (threadIdx.x == 0) wait_zero(counter, st, timeout_ns, -1, -1);
}

}  // namespace

cudaError_t launch_sweep(const LaunchCtx& L, const void* src, void* dst) {
    switch (L.dtype) {
        case kF32: return sweep_t<float, false>(L, src, dst);
        case kF64: return sweep_t<double, false>(L, src, dst);
        case kF64Exact: return sweep_t<double, true>(L, src, dst);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_ring_copy(const LaunchCtx& L, const void* src, void* dst) {
    const DevGeo& g = L.geo;
    if (g.periodic) return cudaSuccess;
    int64_t total = 0;
    for (int a = 0; a < g.dims; ++a) {
        int64_t face = 1;
        for (int b = 0; b < g.dims; ++b)
            if (b != a) face *= g.e[b];
        total += 2 * face;
    }
    const int blk = 256;
    int64_t nb = (total + blk - 1) / blk;
    if (nb > 4096) nb = 4096;
    if (L.dtype == kF32)
        ring_copy_kernel<float><<<(unsigned)nb, blk, 0, L.stream>>>((const float*)src, (float*)dst, g, total);
    else
        ring_copy_kernel<double><<<(unsigned)nb, blk, 0, L.stream>>>((const double*)src, (double*)dst, g, total);
    return cudaGetLastError();
}

cudaError_t launch_grid_copy(const LaunchCtx& L, const void* src, void* dst) {
    const DevGeo& g = L.geo;
    const size_t es = (size_t)dtype_size(L.dtype);
    const int d = g.dims;
    const size_t width = (size_t)g.e[d - 1] * es;
    if (d == 1) return cudaMemcpyAsync(dst, src, width, cudaMemcpyDeviceToDevice, L.stream);
    const size_t pitch = (size_t)g.s[d - 2] * es;
    if (d == 2) return cudaMemcpy2DAsync(dst, pitch, src, pitch, width, (size_t)g.e[0], cudaMemcpyDeviceToDevice,
                                         L.stream);
    if (g.s[0] == g.s[1] * g.e[1])  // planes follow each other without a gap: one pitched copy
        return cudaMemcpy2DAsync(dst, pitch, src, pitch, width, (size_t)(g.e[0] * g.e[1]),
                                 cudaMemcpyDeviceToDevice, L.stream);
    for (int64_t z = 0; z < g.e[0]; ++z) {
        const size_t off = (size_t)(z * g.s[0]) * es;
        cudaError_t e = cudaMemcpy2DAsync((char*)dst + off, pitch, (const char*)src + off, pitch, width,
                                          (size_t)g.e[1], cudaMemcpyDeviceToDevice, L.stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int grid_sum_partials() { return 1024; }

cudaError_t launch_grid_sum(const LaunchCtx& L, const void* grid, double* out, double* partials, int np) {
    if (L.dtype == kF32)
        sum_partial_kernel<float><<<np, 256, 0, L.stream>>>((const float*)grid, L.geo, partials);
    else
        sum_partial_kernel<double><<<np, 256, 0, L.stream>>>((const double*)grid, L.geo, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_final_kernel<<<1, 256, 0, L.stream>>>(partials, np, out);
    return cudaGetLastError();
}

cudaError_t launch_wait_timeout_probe(int32_t* counter, DevStatus* st, uint64_t timeout_ns, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(counter, st, timeout_ns);
    return cudaGetLastError();
}

}  // namespace pcot
