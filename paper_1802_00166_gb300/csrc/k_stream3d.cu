// 3-D tile kernel: trapezoid in (y, x), streamed along axis 0 (z).
//
// One CTA = NW warps stacked along y; each warp owns a brick of RY rows x 64
// contiguous x cells (two elements per lane).  Planes of the tile stream
// through from z0-K to z0+Hz+K-1; stage s keeps its last three planes of the
// brick in a register ring, x-neighbours come from warp shuffles, y-neighbours
// inside the brick from registers and across bricks from the brick edge rows
// that every warp publishes in a per-stage shared-memory slot once per z-step
// (double buffered, one barrier per z-step).  After K stages the valid cells
// are the rows [K, NW*RY-K) and the span minus K cells per side, which is the
// tile's output (the overlapped/trapezoid tile of Sec. 3.3).
#include <type_traits>

#include "tiled.cuh"

namespace pcot {
namespace stream3d {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int E = 2;    // elements per lane
constexpr int RY = 4;   // rows per warp
constexpr int kMaxWarps = 16;

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

// FP32 FMA-mode tiles update a lane's two cells with packed f32x2
// instructions.
template <class T, bool EXACT, int K>
constexpr bool kPacked3 = std::is_same<T, float>::value && !EXACT;

// Register budget per thread: the stage rings hold 3*K*RY*E values.
template <class T, int K>
constexpr int kRegBudget3 = sizeof(T) == 8 ? (K <= 1 ? 168 : 232) : (K <= 1 ? 104 : (K <= 2 ? 128 : 168));

// Warps per CTA the budget allows within the 64K-register file.
inline int max_warps_for(int dtype, int depth) {
    if (dtype != kF32) return 8;
    return depth <= 2 ? kMaxWarps : 12;
}

// PER: periodic grid (compile time, so a periodic run carries no boundary
// tests and a Dirichlet run no wrap-around).
template <class T, bool EXACT, int K, bool CG, bool PER>
__device__ __forceinline__ void cta_tile(const T* __restrict__ src, T* __restrict__ dst, const DevGeo& g,
                                         const Coeffs<T>& c, int64_t z0, int64_t Hz, int64_t y0, int64_t Hy,
                                         int64_t x0, int64_t Wx, bool vec_ok, T* sm) {
    using V = typename V2<T>::V;
    constexpr int Kp = Shape<K>::Kp;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int NW = blockDim.x >> 5;
    const int NR = NW * RY;  // rows of the CTA
    constexpr bool per = PER;
    const int64_t ez = g.e[0], ey = g.e[1], ex = g.e[2];
    const int64_t nz = g.n[0], ny = g.n[1], nx = g.n[2];
    const int64_t Pz = g.s[0], Py = g.s[1];

    const int64_t ybase = y0 - K + (int64_t)w * RY;  // storage row of the brick's first row
    const int64_t xl = x0 - Kp + (int64_t)lane * E;
    const int64_t xhi = x0 + Wx;

    int64_t ysrc[RY];
    bool yin[RY], yint[RY], ystore[RY];
    bool brick_int = true;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int64_t y = ybase + r;
        if (per) {
            ysrc[r] = wrap_fast(y, ny);
            yin[r] = true;
            yint[r] = true;
        } else {
            ysrc[r] = y;
            yin[r] = y >= 0 && y < ey;
            yint[r] = y >= 1 && y <= ny;
        }
        const int ry = w * RY + r;
        ystore[r] = ry >= K && ry < NR - K && y < y0 + Hy && (per ? y < ny : yint[r]);
        brick_int = brick_int && yint[r];
    }

    bool inb[E], xint[E], stx[E];
    int64_t col[E];
    bool all_in = true, all_stx = true, lane_xint = true;
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
        stx[j] = x >= x0 && x < xhi && (per ? x < nx : xint[j]);
        all_in = all_in && inb[j];
        all_stx = all_stx && stx[j];
        lane_xint = lane_xint && xint[j];
    }
    const bool lvec = vec_ok && all_in && col[1] == col[0] + 1 && (col[0] % E) == 0;
    const bool svec = vec_ok && all_stx && (xl % E) == 0;
    const bool warp_xint = __all_sync(kFull, lane_xint);
    const bool brick_ok = per || (brick_int && warp_xint);  // no pass-through inside this brick

    // Offsets inside a plane (computed once per tile, 32-bit: choose() admits
    // planes of fewer than 2^30 cells): of the brick's rows, of this lane's
    // first loaded cell in each row, of its first stored cell.
    int32_t yoff[RY], loff[RY], soff[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        yoff[r] = (int32_t)(ysrc[r] * Py);
        loff[r] = yoff[r] + (int32_t)col[0];
        soff[r] = (int32_t)((ybase + r) * Py + xl);
    }

    // The brick's rows of one input plane (its offset and bounds tracked
    // incrementally, one plane per z-step).  Per row a lane loads its two
    // cells as one vector (lfast) or, next to a wrap-around or the grid's
    // edge and on unaligned layouts, cell by cell (lslow) -- decided once per
    // tile.
    bool lfast[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) lfast[r] = yin[r] && lvec;
    const bool lslow = !lvec;
    bool rows_fast = true;
#pragma unroll
    for (int r = 0; r < RY; ++r) rows_fast = rows_fast && lfast[r];
    const bool warp_lfast = __all_sync(kFull, rows_fast);  // every row of every lane: one vector load
    int64_t lz = per ? wrap_fast(z0 - K, nz) : z0 - K;  // storage index of the plane loaded next
    int64_t lofs = lz * Pz;
    auto load_plane = [&](T (&v)[RY][E]) {
        const bool zin = per || (lz >= 0 && lz < ez);
        const T* plane = src + lofs;
        if (zin && warp_lfast) {
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const V q = gload<CG>(reinterpret_cast<const V*>(plane + loff[r]));
                v[r][0] = q.x;
                v[r][1] = q.y;
            }
            // plane lz + 2 into L2 ahead of its load (skipped at a wrap or the grid's end)
            if (lz + 2 < (per ? nz : ez)) {
#pragma unroll
                for (int r = 0; r < RY; ++r)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(plane + 2 * Pz + loff[r]));
            }
        } else {
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                if (zin && lfast[r]) {
                    const V q = gload<CG>(reinterpret_cast<const V*>(plane + loff[r]));
                    v[r][0] = q.x;
                    v[r][1] = q.y;
                } else {
                    v[r][0] = T(0);
                    v[r][1] = T(0);
                }
            }
            if (lslow) {
#pragma unroll
                for (int r = 0; r < RY; ++r)
#pragma unroll
                    for (int j = 0; j < E; ++j)
                        if (zin && yin[r] && inb[j]) v[r][j] = gload<CG>(plane + yoff[r] + (int32_t)col[j]);
            }
        }
        if (per && lz + 1 == nz) {
            lz = 0;
            lofs = 0;
        } else {
            ++lz;
            lofs += Pz;
        }
    };

    // sm[buf][w][s][edge][32*E]: edge 0 = the brick's first row, 1 = its last.
    // A warp's slots sit at a compile-time stride, so its neighbours' slots
    // are at fixed offsets from its own.
    constexpr int rowlen = 32 * E;
    constexpr int WS = K * 2 * rowlen;  // one warp's slots of one buffer
    T* const my0 = sm + w * WS + lane * E;
    T* const my1 = my0 + NW * WS;
    // The first and last warps read their own slots in place of a missing
    // neighbour's: those rows are the tile's halo, whose values never reach
    // a stored cell within K steps, so no per-stage select is needed.
    const int up_off = w > 0 ? -WS : 0;
    const int dn_off = w < NW - 1 ? WS : 0;

    T R[K][3][RY][E];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int r = 0; r < RY; ++r)
#pragma unroll
                for (int j = 0; j < E; ++j) R[s][u][r][j] = T(0);

    // The planes z0-K .. z0+Hz+K-1 stream through, rounded up to whole
    // iterations of the 3-step loop below (the extra planes are computed and
    // not stored), so every iteration runs all three steps unconditionally.
    const int64_t zbeg = z0 - K, zend = zbeg + (Hz + 2 * K + 2) / 3 * 3;
    // Stores: plane zi - K is written for zi in [zs_lo, zs_hi) (the tile's
    // planes inside the grid's interior); per row, a lane either stores its
    // two cells as one vector (sfast) or, on a ragged or unaligned edge, cell
    // by cell (sslow) -- decided once per tile, not per plane.
    int64_t zs_lo = z0 + K, zs_hi = z0 + Hz + K;
    if (per) {
        zs_hi = zs_hi < nz + K ? zs_hi : nz + K;
    } else {
        zs_lo = zs_lo > 1 + K ? zs_lo : 1 + K;
        zs_hi = zs_hi < nz + 1 + K ? zs_hi : nz + 1 + K;
    }
    bool any_stx = false;
#pragma unroll
    for (int j = 0; j < E; ++j) any_stx = any_stx || stx[j];
    bool sfast[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) sfast[r] = ystore[r] && svec;
    const bool sslow = !svec && any_stx;
    int64_t sofs = (zbeg - K) * Pz;  // offset of plane zi - K, advanced one plane per z-step
    load_plane(R[0][2]);  // the first plane: stage 0's newest plane of step 0
    int buf = 0;

    auto step = [&](auto Uc, int64_t zi) {
        constexpr int U = decltype(Uc)::value;
        constexpr int SA = U % 3, SB = (U + 1) % 3, SN = (U + 2) % 3;
        T* const mine = buf ? my1 : my0;
        const T* const up = mine + up_off;
        const T* const dn = mine + dn_off;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            V q0, q1;
            q0.x = R[s][SB][0][0];
            q0.y = R[s][SB][0][1];
            q1.x = R[s][SB][RY - 1][0];
            q1.y = R[s][SB][RY - 1][1];
            *reinterpret_cast<V*>(mine + s * 2 * rowlen) = q0;
            *reinterpret_cast<V*>(mine + s * 2 * rowlen + rowlen) = q1;
        }
        __syncthreads();
        T out[RY][E];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            const int64_t zr = zi - s - 1;  // plane of time level s+1 produced now
            // row above the brick, row below the brick
            const V nq = *reinterpret_cast<const V*>(up + s * 2 * rowlen + rowlen);
            const V sq = *reinterpret_cast<const V*>(dn + s * 2 * rowlen);
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const T n0 = r > 0 ? R[s][SB][r - 1][0] : nq.x;
                const T n1 = r > 0 ? R[s][SB][r - 1][1] : nq.y;
                const T s0 = r < RY - 1 ? R[s][SB][r + 1][0] : sq.x;
                const T s1 = r < RY - 1 ? R[s][SB][r + 1][1] : sq.y;
                const T wl = __shfl_up_sync(kFull, R[s][SB][r][1], 1);
                const T er = __shfl_down_sync(kFull, R[s][SB][r][0], 1);
                if constexpr (kPacked3<T, EXACT, K>) {
                    // the lane's two cells (c0, c1) as one f32x2 pair, same
                    // operations and order per cell as upd3's FMA mode
                    // (bitwise equal); the x-neighbours (c-1, c0) and (c1, c2)
                    // are shifted by one cell, so they enter as scalar FMAs
                    // on the pair's halves instead of being assembled into
                    // register pairs
                    const float2 k0 = make_float2(c.c[0], c.c[0]), k1 = make_float2(c.c[1], c.c[1]);
                    const float2 k2 = make_float2(c.c[2], c.c[2]), k3 = make_float2(c.c[3], c.c[3]);
                    const float2 k4 = make_float2(c.c[4], c.c[4]);
                    float2 a = __fmul2_rn(k0, make_float2(R[s][SB][r][0], R[s][SB][r][1]));
                    a = __ffma2_rn(k1, make_float2(R[s][SA][r][0], R[s][SA][r][1]), a);
                    a = __ffma2_rn(k3, make_float2(n0, n1), a);
                    a = __ffma2_rn(k4, make_float2(s0, s1), a);
                    a.x = __fmaf_rn(c.c[5], wl, a.x);
                    a.y = __fmaf_rn(c.c[5], R[s][SB][r][0], a.y);
                    a.x = __fmaf_rn(c.c[6], R[s][SB][r][1], a.x);
                    a.y = __fmaf_rn(c.c[6], er, a.y);
                    a = __ffma2_rn(k2, make_float2(R[s][SN][r][0], R[s][SN][r][1]), a);
                    out[r][0] = a.x;
                    out[r][1] = a.y;
                } else {
                    out[r][0] = upd3<T, EXACT>(c, R[s][SB][r][0], R[s][SA][r][0], R[s][SN][r][0], n0, s0, wl,
                                               R[s][SB][r][1]);
                    out[r][1] = upd3<T, EXACT>(c, R[s][SB][r][1], R[s][SA][r][1], R[s][SN][r][1], n1, s1,
                                               R[s][SB][r][0], er);
                }
            }
            if (!per) {
                const bool zint = zr >= 1 && zr <= nz;
                if (!(zint && brick_ok)) {
#pragma unroll
                    for (int r = 0; r < RY; ++r)
#pragma unroll
                        for (int j = 0; j < E; ++j)
                            if (!(zint && yint[r] && xint[j])) out[r][j] = R[s][SB][r][j];
                }
            }
            if (s + 1 < K) {
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    R[s + 1][SN][r][0] = out[r][0];
                    R[s + 1][SN][r][1] = out[r][1];
                }
            }
            // stage 0 is done with its oldest plane: the next input plane,
            // stage 0's newest in the next step, is loaded into that slot
            if (s == 0 && zi + 1 < zend) load_plane(R[0][SA]);
        }
        if (zi >= zs_lo && zi < zs_hi) {
            T* const plane = dst + sofs;
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                if (sfast[r]) {
                    V q;
                    q.x = out[r][0];
                    q.y = out[r][1];
                    *reinterpret_cast<V*>(plane + soff[r]) = q;
                }
            }
            if (sslow) {
#pragma unroll
                for (int r = 0; r < RY; ++r)
#pragma unroll
                    for (int j = 0; j < E; ++j)
                        if (ystore[r] && stx[j]) plane[soff[r] + j] = out[r][j];
            }
        }
        sofs += Pz;
        buf ^= 1;
    };

    for (int64_t zi = zbeg; zi < zend; zi += 3) {
        step(IC<0>{}, zi);
        step(IC<1>{}, zi + 1);
        step(IC<2>{}, zi + 2);
    }
}

template <class T, bool EXACT, int K, bool PER>
__global__ void __maxnreg__((kRegBudget3<T, K>)) slt_kernel(const T* __restrict__ src, T* __restrict__ dst, DevGeo g,
                                                       Coeffs<T> c, TileGeo t, bool vec_ok) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int64_t ix = blockIdx.x, iy = blockIdx.y, iz = blockIdx.z;
    cta_tile<T, EXACT, K, false, PER>(src, dst, g, c, iz * t.ext[0], t.ext[0], iy * t.ext[1], t.ext[1],
                                      ix * t.ext[2], t.ext[2], vec_ok, reinterpret_cast<T*>(smraw));
}

template <class T, bool EXACT, int K, bool PER>
__global__ void __maxnreg__((kRegBudget3<T, K>)) cot_kernel(T* buf0, T* buf1, DevGeo g, Coeffs<T> c, TileGeo t,
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
        cta_tile<T, EXACT, K, true, PER>(src, dst, g, c, (int64_t)iz * t.ext[0], t.ext[0], (int64_t)iy * t.ext[1],
                                         t.ext[1], (int64_t)ix * t.ext[2], t.ext[2], vec_ok,
                                         reinterpret_cast<T*>(smraw));
        __syncthreads();  // the tile's stores by every thread precede thread 0's release
        if (threadIdx.x == 0) release_successors(q, 3, b, iz, iy, ix);
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
    return (size_t)2 * t.depth * t.nwarps * 2 * 32 * E * sizeof(T);
}

template <class T, bool EXACT, int K, bool PER>
cudaError_t slt_kp(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst) {
    const size_t sm = smem_t<T>(t);
    cudaError_t e =
        cudaFuncSetAttribute(slt_kernel<T, EXACT, K, PER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (t.count[0] > 65535 || t.count[1] > 65535) return cudaErrorInvalidConfiguration;
    dim3 grd((unsigned)t.count[2], (unsigned)t.count[1], (unsigned)t.count[0]);
    slt_kernel<T, EXACT, K, PER><<<grd, 32 * t.nwarps, sm, L.stream>>>((const T*)src, (T*)dst, L.geo,
                                                                       coeffs_as<T>(L.coeffs), t,
                                                                       vec_aligned<T>(L.geo, src, dst));
    return cudaGetLastError();
}

template <class T, bool EXACT, int K>
cudaError_t slt_k(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst) {
    return L.geo.periodic ? slt_kp<T, EXACT, K, true>(L, t, src, dst) : slt_kp<T, EXACT, K, false>(L, t, src, dst);
}

template <class T, bool EXACT, int K, bool PER>
cudaError_t cot_kp(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
    const size_t sm = smem_t<T>(t);
    cudaError_t e =
        cudaFuncSetAttribute(cot_kernel<T, EXACT, K, PER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    cot_kernel<T, EXACT, K, PER><<<nctas, 32 * t.nwarps, sm, L.stream>>>((T*)b0, (T*)b1, L.geo,
                                                                         coeffs_as<T>(L.coeffs), t,
                                                                         vec_aligned<T>(L.geo, b0, b1), q);
    return cudaGetLastError();
}

template <class T, bool EXACT, int K>
cudaError_t cot_k(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
    return L.geo.periodic ? cot_kp<T, EXACT, K, true>(L, t, b0, b1, q, nctas)
                          : cot_kp<T, EXACT, K, false>(L, t, b0, b1, q, nctas);
}

template <class T, bool EXACT, int K, bool PER>
int occ_kp(const TileGeo& t) {
    const size_t sm = smem_t<T>(t);
    if (cudaFuncSetAttribute(cot_kernel<T, EXACT, K, PER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cot_kernel<T, EXACT, K, PER>, 32 * t.nwarps, sm) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <class T, bool EXACT, int K>
int occ_k(const LaunchCtx& L, const TileGeo& t) {
    return L.geo.periodic ? occ_kp<T, EXACT, K, true>(t) : occ_kp<T, EXACT, K, false>(t);
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
    // Rows of a CTA = warps x RY, as many warps as the register budget allows.
    const int maxw = max_warps_for(L.dtype, depth);
    int64_t Hy = req && req[1] > 0 ? req[1] : 8 * RY - 2 * depth;
    if (Hy < depth) Hy = depth;
    int nw = (int)((Hy + 2 * depth + RY - 1) / RY);
    if (nw > maxw) nw = maxw;
    Hy = (int64_t)nw * RY - 2 * depth;
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
    // 32-bit in-plane offsets (larger planes go to the generic kernel)
    if (L.geo.s[0] >= ((int64_t)1 << 30)) return false;
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
    PCOT_DISPATCH3(occ_k, L, t)
    return 1;
}

#undef PCOT_DISPATCH3

}  // namespace stream3d
}  // namespace pcot
