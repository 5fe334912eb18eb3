// 3-D tile kernel: trapezoid in (y, x), streamed along axis 0 (z).
//
// One CTA = NW warps stacked along y (one row each), every warp covering a
// span of 64 contiguous x cells (two elements per lane).  Planes of the tile
// stream through from z0-K to z0+Hz+K-1; stage s keeps its last three planes
// of the lane's cells in a register ring, x-neighbours come from warp
// shuffles and y-neighbours from a per-stage shared-memory plane written once
// per z-step (double buffered, one barrier per step).  After K stages the
// valid cells are the rows [K, NW-K) and the span minus K cells per side,
// which is the tile's output (the overlapped/trapezoid tile of Sec. 3.3).
#include "tiled.cuh"

namespace pcot {
namespace stream3d {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int E = 2;  // elements per lane
constexpr int kMaxWarps = 32;

template <class T>
struct V2;
template <>
struct V2<float> {
    using V = float2;
};
template <>
struct V2<double> {
    using V = double2;
};

template <int K>
struct Shape {
    static constexpr int Kp = ((K + E - 1) / E) * E;
    static constexpr int Wo = 32 * E - 2 * Kp;
};

template <class T, bool EXACT, int K, bool CG>
__device__ __forceinline__ void cta_tile(const T* __restrict__ src, T* __restrict__ dst, const DevGeo& g,
                                         const Coeffs<T>& c, int64_t z0, int64_t Hz, int64_t y0, int64_t Hy,
                                         int64_t x0, int64_t Wx, bool vec_ok, T* sm) {
    using V = typename V2<T>::V;
    constexpr int Kp = Shape<K>::Kp;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int NW = blockDim.x >> 5;
    const bool per = g.periodic != 0;
    const int64_t ez = g.e[0], ey = g.e[1], ex = g.e[2];
    const int64_t nz = g.n[0], ny = g.n[1], nx = g.n[2];
    const int64_t Pz = g.s[0], Py = g.s[1];

    const int64_t y = y0 - K + w;  // storage row of this warp
    const int64_t xl = x0 - Kp + (int64_t)lane * E;
    const int64_t xhi = x0 + Wx;

    int64_t ysrc;
    bool yin, yint;
    if (per) {
        ysrc = wrap_fast(y, ny);
        yin = true;
        yint = true;
    } else {
        ysrc = y;
        yin = y >= 0 && y < ey;
        yint = y >= 1 && y <= ny;
    }
    const bool ystore = w >= K && w < NW - K && y < y0 + Hy && (per ? y < ny : yint);

    bool inb[E], xint[E], st[E];
    int64_t col[E];
    bool all_in = true, all_st = true, lane_xint = true;
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int64_t x = xl + j;
        if (per) {
            col[j] = wrap_fast(x, nx);
            inb[j] = true;
            xint[j] = true;
        } else {
            col[j] = x;
            inb[j] = x >= 0 && x < ex;
            xint[j] = x >= 1 && x <= nx;
        }
        st[j] = ystore && x >= x0 && x < xhi && (per ? x < nx : xint[j]);
        all_in = all_in && inb[j];
        all_st = all_st && st[j];
        lane_xint = lane_xint && xint[j];
    }
    const bool lvec = vec_ok && all_in && col[1] == col[0] + 1 && (col[0] % E) == 0;
    const bool svec = vec_ok && all_st && (xl % E) == 0;
    const bool warp_xint = __all_sync(kFull, lane_xint);
    const bool row_ok = per || (yint && warp_xint);  // no pass-through needed on this row

    auto load_plane = [&](int64_t zi, T (&v)[E]) {
        int64_t zs;
        bool zin;
        if (per) {
            zs = wrap_fast(zi, nz);
            zin = true;
        } else {
            zs = zi;
            zin = zi >= 0 && zi < ez;
        }
        if (!zin || !yin) {
            v[0] = T(0);
            v[1] = T(0);
            return;
        }
        const T* rowp = src + zs * Pz + ysrc * Py;
        if (lvec) {
            const V q = gload<CG>(reinterpret_cast<const V*>(rowp + col[0]));
            v[0] = q.x;
            v[1] = q.y;
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) v[j] = inb[j] ? gload<CG>(rowp + col[j]) : T(0);
        }
    };

    // sm[buf][s][w][32*E]
    const int rowlen = 32 * E;
    const int stage_stride = NW * rowlen;
    const int buf_stride = K * stage_stride;

    T R[K][3][E];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int j = 0; j < E; ++j) R[s][u][j] = T(0);

    const int64_t zbeg = z0 - K, zend = z0 + Hz + K;
    T pf[3][E];  // three planes in flight per lane
    load_plane(zbeg, pf[0]);
    if (zbeg + 1 < zend) load_plane(zbeg + 1, pf[1]);
    if (zbeg + 2 < zend) load_plane(zbeg + 2, pf[2]);
    int buf = 0;

    auto step = [&](auto Uc, int64_t zi) {
        constexpr int U = decltype(Uc)::value;
        constexpr int SA = U % 3, SB = (U + 1) % 3, SN = (U + 2) % 3;
        R[0][SN][0] = pf[U][0];
        R[0][SN][1] = pf[U][1];
        if (zi + 3 < zend) load_plane(zi + 3, pf[U]);
        T* smb = sm + buf * buf_stride;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            V q;
            q.x = R[s][SB][0];
            q.y = R[s][SB][1];
            *reinterpret_cast<V*>(smb + s * stage_stride + w * rowlen + lane * E) = q;
        }
        __syncthreads();
        T out[E];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            const int64_t zr = zi - s - 1;  // plane of time level s+1 produced now
            const T* sp = smb + s * stage_stride + lane * E;
            V nq, sq;
            if (w > 0) nq = *reinterpret_cast<const V*>(sp + (w - 1) * rowlen);
            else { nq.x = R[s][SB][0]; nq.y = R[s][SB][1]; }
            if (w < NW - 1) sq = *reinterpret_cast<const V*>(sp + (w + 1) * rowlen);
            else { sq.x = R[s][SB][0]; sq.y = R[s][SB][1]; }
            const T wl = __shfl_up_sync(kFull, R[s][SB][1], 1);
            const T er = __shfl_down_sync(kFull, R[s][SB][0], 1);
            out[0] = upd3<T, EXACT>(c, R[s][SB][0], R[s][SA][0], R[s][SN][0], nq.x, sq.x, wl, R[s][SB][1]);
            out[1] = upd3<T, EXACT>(c, R[s][SB][1], R[s][SA][1], R[s][SN][1], nq.y, sq.y, R[s][SB][0], er);
            if (!per) {
                const bool zint = zr >= 1 && zr <= nz;
                if (!(zint && row_ok)) {
#pragma unroll
                    for (int j = 0; j < E; ++j)
                        if (!(zint && yint && xint[j])) out[j] = R[s][SB][j];
                }
            }
            if (s + 1 < K) {
                R[s + 1][SN][0] = out[0];
                R[s + 1][SN][1] = out[1];
            }
        }
        const int64_t zo = zi - K;
        const bool zok = zo >= z0 && zo < z0 + Hz && (per ? zo < nz : (zo >= 1 && zo <= nz));
        if (zok) {
            T* rowp = dst + zo * Pz + y * Py;
            if (svec) {
                V q;
                q.x = out[0];
                q.y = out[1];
                *reinterpret_cast<V*>(rowp + xl) = q;
            } else {
#pragma unroll
                for (int j = 0; j < E; ++j)
                    if (st[j]) rowp[xl + j] = out[j];
            }
        }
        buf ^= 1;
    };

    for (int64_t zi = zbeg; zi < zend; zi += 3) {
        step(IC<0>{}, zi);
        if (zi + 1 < zend) step(IC<1>{}, zi + 1);
        if (zi + 2 < zend) step(IC<2>{}, zi + 2);
    }
}

template <class T, bool EXACT, int K>
__global__ void __launch_bounds__(32 * kMaxWarps) slt_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                             DevGeo g, Coeffs<T> c, TileGeo t, bool vec_ok) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int64_t ix = blockIdx.x, iy = blockIdx.y, iz = blockIdx.z;
    cta_tile<T, EXACT, K, false>(src, dst, g, c, iz * t.ext[0], t.ext[0], iy * t.ext[1], t.ext[1], ix * t.ext[2],
                                 t.ext[2], vec_ok, reinterpret_cast<T*>(smraw));
}

template <class T, bool EXACT, int K>
__global__ void __launch_bounds__(32 * kMaxWarps) cot_kernel(T* buf0, T* buf1, DevGeo g, Coeffs<T> c, TileGeo t,
                                                             bool vec_ok, CotDev q) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = pop_and_wait(q);
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) return;
        const int L0 = q.lattice[1], L1 = q.lattice[2], L2 = q.lattice[3];
        int r = tile;
        const int ix = r % L2;
        r /= L2;
        const int iy = r % L1;
        r /= L1;
        const int iz = r % L0;
        const int b = r / L0;
        const T* src = (b & 1) ? buf1 : buf0;
        T* dst = (b & 1) ? buf0 : buf1;
        cta_tile<T, EXACT, K, true>(src, dst, g, c, (int64_t)iz * t.ext[0], t.ext[0], (int64_t)iy * t.ext[1],
                                    t.ext[1], (int64_t)ix * t.ext[2], t.ext[2], vec_ok, reinterpret_cast<T*>(smraw));
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            release_successors(q, 3, b, iz, iy, ix);
        }
    }
}

template <class T>
bool vec_aligned(const DevGeo& g, const void* a, const void* b) {
    const uintptr_t m = sizeof(T) * E - 1;
    const int64_t bytes = (int64_t)(sizeof(T) * E);
    return ((uintptr_t)a & m) == 0 && ((uintptr_t)b & m) == 0 && ((g.s[0] * (int64_t)sizeof(T)) % bytes) == 0 &&
           ((g.s[1] * (int64_t)sizeof(T)) % bytes) == 0;
}

template <class T>
size_t smem_t(const TileGeo& t) {
    return (size_t)2 * t.depth * t.nwarps * 32 * E * sizeof(T);
}

template <class T, bool EXACT, int K>
cudaError_t slt_k(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst) {
    const size_t sm = smem_t<T>(t);
    cudaError_t e = cudaFuncSetAttribute(slt_kernel<T, EXACT, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (t.count[0] > 65535 || t.count[1] > 65535) return cudaErrorInvalidConfiguration;
    dim3 grd((unsigned)t.count[2], (unsigned)t.count[1], (unsigned)t.count[0]);
    slt_kernel<T, EXACT, K><<<grd, 32 * t.nwarps, sm, L.stream>>>((const T*)src, (T*)dst, L.geo,
                                                                  coeffs_as<T>(L.coeffs), t,
                                                                  vec_aligned<T>(L.geo, src, dst));
    return cudaGetLastError();
}

template <class T, bool EXACT, int K>
cudaError_t cot_k(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
    const size_t sm = smem_t<T>(t);
    cudaError_t e = cudaFuncSetAttribute(cot_kernel<T, EXACT, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    cot_kernel<T, EXACT, K><<<nctas, 32 * t.nwarps, sm, L.stream>>>((T*)b0, (T*)b1, L.geo, coeffs_as<T>(L.coeffs), t,
                                                                    vec_aligned<T>(L.geo, b0, b1), q);
    return cudaGetLastError();
}

template <class T, bool EXACT, int K>
int occ_k(const TileGeo& t) {
    const size_t sm = smem_t<T>(t);
    if (cudaFuncSetAttribute(cot_kernel<T, EXACT, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cot_kernel<T, EXACT, K>, 32 * t.nwarps, sm) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace

int depths(int dtype, int* out, int cap) {
    static const int f32[] = {1, 2, 3, 4};
    static const int f64[] = {1, 2};
    const int* src = dtype == kF32 ? f32 : f64;
    const int n = dtype == kF32 ? 4 : 2;
    for (int i = 0; i < n && i < cap; ++i) out[i] = src[i];
    return n;
}

size_t smem(const LaunchCtx& L, const TileGeo& t) {
    return L.dtype == kF32 ? smem_t<float>(t) : smem_t<double>(t);
}

bool choose(const LaunchCtx& L, const int32_t* req, int depth, TileGeo* t) {
    if (L.geo.dims != 3) return false;
    int ds[8];
    const int nd = depths(L.dtype, ds, 8);
    bool ok = false;
    for (int i = 0; i < nd; ++i) ok = ok || ds[i] == depth;
    if (!ok) return false;
    const int Kp = ((depth + E - 1) / E) * E;
    const int Wo = 32 * E - 2 * Kp;
    int64_t Hz = req && req[0] > 0 ? req[0] : 64;
    int64_t Hy = req && req[1] > 0 ? req[1] : 32 - 2 * depth;
    if (Hy < depth) Hy = depth;
    int nw = (int)Hy + 2 * depth;
    if (nw > kMaxWarps) {
        nw = kMaxWarps;
        Hy = nw - 2 * depth;
    }
    if (Hy < depth) return false;
    if (Hz < depth) Hz = depth;
    // Tiles along x: as few warps as the span allows, extents balanced and
    // rounded to whole lanes so every span starts on a vector boundary.
    const int64_t ex = L.geo.e[2];
    int64_t nxt = (ex + Wo - 1) / Wo;
    int64_t Wx = (ex + nxt - 1) / nxt;
    Wx = ((Wx + E - 1) / E) * E;
    if (req && req[2] > 0 && req[2] < Wx) Wx = ((req[2] + E - 1) / E) * E;
    if (Wx > Wo) Wx = Wo;
    if (Wx < Kp) Wx = Kp;
    t->family = kFamStream3D;
    t->depth = depth;
    t->nwarps = nw;
    t->ext[0] = Hz;
    t->ext[1] = Hy;
    t->ext[2] = Wx;
    t->count[0] = (L.geo.e[0] + Hz - 1) / Hz;
    t->count[1] = (L.geo.e[1] + Hy - 1) / Hy;
    t->count[2] = (ex + Wx - 1) / Wx;
    return smem(L, *t) <= 200 * 1024;
}

#define PCOT_DISPATCH3(FN, ...)                                               \
    switch (t.depth) {                                                        \
        case 1:                                                               \
            if (L.dtype == kF32) return FN<float, false, 1>(__VA_ARGS__);     \
            if (L.dtype == kF64) return FN<double, false, 1>(__VA_ARGS__);    \
            return FN<double, true, 1>(__VA_ARGS__);                          \
        case 2:                                                               \
            if (L.dtype == kF32) return FN<float, false, 2>(__VA_ARGS__);     \
            if (L.dtype == kF64) return FN<double, false, 2>(__VA_ARGS__);    \
            return FN<double, true, 2>(__VA_ARGS__);                          \
        case 3:                                                               \
            if (L.dtype == kF32) return FN<float, false, 3>(__VA_ARGS__);     \
            break;                                                            \
        case 4:                                                               \
            if (L.dtype == kF32) return FN<float, false, 4>(__VA_ARGS__);     \
            break;                                                            \
    }

cudaError_t slt(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst) {
    PCOT_DISPATCH3(slt_k, L, t, src, dst)
    return cudaErrorInvalidValue;
}

cudaError_t cot(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
    PCOT_DISPATCH3(cot_k, L, t, b0, b1, q, nctas)
    return cudaErrorInvalidValue;
}

int ctas_per_sm(const LaunchCtx& L, const TileGeo& t) {
    PCOT_DISPATCH3(occ_k, t)
    return 1;
}

#undef PCOT_DISPATCH3

}  // namespace stream3d
}  // namespace pcot
