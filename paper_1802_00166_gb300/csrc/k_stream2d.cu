// 2-D tile kernel: a register-resident trapezoid streamed along axis 0.
//
// A tile of the single-level tiling (Sec. 3.3) or a leaf of the recursive
// schedule (Sec. 4.2, base function) advances an output block of H rows x Wt
// columns by K time steps.  Each warp owns a span of 32*E contiguous columns
// (E = one 16-byte vector per lane) and streams the rows of its span from
// y0-K to y0+H+K-1.  Stage s (s = 1..K) of the pipeline holds the last rows of
// time level s in registers; a new input row lets every stage emit one row,
// so the row leaving stage K is K steps ahead (the overlapped/trapezoid tile:
// the valid part of the span shrinks by one column per step on each side).
// Horizontal neighbours come from warp shuffles, vertical ones from the
// stage's register ring; HBM sees one read of the span plus one write of the
// warp's output columns per pass.  The Dirichlet ring passes through
// unchanged (its cells are never updated).
#include "tiled.cuh"

namespace pcot {
namespace stream2d {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int K, int E>
struct Shape {
    static constexpr int Kp = ((K + E - 1) / E) * E;   // halo rounded to whole lanes
    static constexpr int Wo = 32 * E - 2 * Kp;          // output columns per warp
};

template <class T, bool EXACT, int K, bool CG>
__device__ __forceinline__ void warp_tile(const T* __restrict__ src, T* __restrict__ dst, const DevGeo& g,
                                          const Coeffs<T>& c, int64_t y0, int64_t H, int64_t olo, int64_t ohi,
                                          bool vec_ok) {
    constexpr int E = Vec<T>::E;
    using V = typename Vec<T>::V;
    constexpr int Kp = Shape<K, E>::Kp;
    const int lane = threadIdx.x & 31;
    const bool per = g.periodic != 0;
    const int64_t ey = g.e[0], ex = g.e[1], ny = g.n[0], nx = g.n[1], P = g.s[0];
    const int64_t xl = olo - Kp + (int64_t)lane * E;  // first column of this lane

    // Column flags of the lane's E elements.
    bool inb[E], xint[E], st[E];
    int64_t col[E];
    bool all_in = true, all_st = true, lane_xint = true;
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int64_t x = xl + j;
        if (per) {
            col[j] = wrapc(x, nx);
            inb[j] = true;
            xint[j] = true;
        } else {
            col[j] = x;
            inb[j] = x >= 0 && x < ex;
            xint[j] = x >= 1 && x <= nx;
        }
        st[j] = x >= olo && x < ohi && xint[j];
        all_in = all_in && inb[j];
        all_st = all_st && st[j];
        lane_xint = lane_xint && xint[j];
    }
    const bool lvec = vec_ok && all_in && col[E - 1] == col[0] + (E - 1) && (col[0] % E) == 0;
    const bool svec = vec_ok && all_st && (xl % E) == 0;
    const bool warp_xint = __all_sync(kFull, lane_xint);

    auto load_row = [&](int64_t yi, T (&v)[E]) {
        int64_t ys;
        bool rin;
        if (per) {
            ys = wrapc(yi, ny);
            rin = true;
        } else {
            ys = yi;
            rin = yi >= 0 && yi < ey;
        }
        if (!rin) {
#pragma unroll
            for (int j = 0; j < E; ++j) v[j] = T(0);
            return;
        }
        const T* rowp = src + ys * P;
        if (lvec) {
            const V q = gload<CG>(reinterpret_cast<const V*>(rowp + col[0]));
            const T* qq = reinterpret_cast<const T*>(&q);
#pragma unroll
            for (int j = 0; j < E; ++j) v[j] = qq[j];
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) v[j] = inb[j] ? gload<CG>(rowp + col[j]) : T(0);
        }
    };

    // R[s][slot][j]: ring of the last three rows of time level s (s = 0 is
    // the input).  At unrolled phase U the slots (U, U+1, U+2) mod 3 hold rows
    // r-2, r-1 and the incoming row r, so no register moves are needed.
    T R[K][3][E];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int j = 0; j < E; ++j) R[s][u][j] = T(0);

    const int64_t ybeg = y0 - K, yend = y0 + H + K;
    T pf[E];
    load_row(ybeg, pf);

    auto step = [&](auto Uc, int64_t yi) {
        constexpr int U = decltype(Uc)::value;
        constexpr int SA = U % 3, SB = (U + 1) % 3, SN = (U + 2) % 3;
#pragma unroll
        for (int j = 0; j < E; ++j) R[0][SN][j] = pf[j];
        if (yi + 1 < yend) load_row(yi + 1, pf);
        T out[E];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            const int64_t r = yi - s - 1;  // row of time level s+1 produced now
            const T wl = __shfl_up_sync(kFull, R[s][SB][E - 1], 1);
            const T er = __shfl_down_sync(kFull, R[s][SB][0], 1);
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const T W = j > 0 ? R[s][SB][j - 1] : wl;
                const T Ea = j < E - 1 ? R[s][SB][j + 1] : er;
                out[j] = upd2<T, EXACT>(c, R[s][SB][j], R[s][SA][j], R[s][SN][j], W, Ea);
            }
            if (!per) {
                const bool rint = r >= 1 && r <= ny;
                if (!(rint && warp_xint)) {
#pragma unroll
                    for (int j = 0; j < E; ++j)
                        if (!(rint && xint[j])) out[j] = R[s][SB][j];
                }
            }
            if (s + 1 < K) {
#pragma unroll
                for (int j = 0; j < E; ++j) R[s + 1][SN][j] = out[j];
            }
        }
        const int64_t ro = yi - K;
        const bool rok = ro >= y0 && ro < y0 + H && (per ? ro < ny : (ro >= 1 && ro <= ny));
        if (rok) {
            T* rowp = dst + ro * P;
            if (svec) {
                V q;
                T* qq = reinterpret_cast<T*>(&q);
#pragma unroll
                for (int j = 0; j < E; ++j) qq[j] = out[j];
                *reinterpret_cast<V*>(rowp + xl) = q;
            } else {
#pragma unroll
                for (int j = 0; j < E; ++j)
                    if (st[j]) rowp[xl + j] = out[j];
            }
        }
    };

    for (int64_t yi = ybeg; yi < yend; yi += 3) {
        step(IC<0>{}, yi);
        if (yi + 1 < yend) step(IC<1>{}, yi + 1);
        if (yi + 2 < yend) step(IC<2>{}, yi + 2);
    }
}

constexpr int kMaxWarps = 8;

template <class T, bool EXACT, int K>
__global__ void __launch_bounds__(32 * kMaxWarps) slt_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                             DevGeo g, Coeffs<T> c, int64_t H, int64_t Wt,
                                                             bool vec_ok) {
    constexpr int Wo = Shape<K, Vec<T>::E>::Wo;
    const int64_t x0 = (int64_t)blockIdx.x * Wt, y0 = (int64_t)blockIdx.y * H;
    const int w = threadIdx.x >> 5;
    const int64_t olo = x0 + (int64_t)w * Wo;
    int64_t ohi = olo + Wo;
    if (ohi > x0 + Wt) ohi = x0 + Wt;
    if (ohi > g.e[1]) ohi = g.e[1];
    if (olo >= ohi) return;
    warp_tile<T, EXACT, K, false>(src, dst, g, c, y0, H, olo, ohi, vec_ok);
}

template <class T, bool EXACT, int K>
__global__ void __launch_bounds__(32 * kMaxWarps) cot_kernel(T* buf0, T* buf1, DevGeo g, Coeffs<T> c, int64_t H,
                                                             int64_t Wt, bool vec_ok, CotDev q) {
    constexpr int Wo = Shape<K, Vec<T>::E>::Wo;
    __shared__ int s_tile;
    const int w = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_tile = pop_and_wait(q);
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) return;
        const int L1 = q.lattice[2], L0 = q.lattice[1];
        const int ix = tile % L1;
        const int rest = tile / L1;
        const int iy = rest % L0;
        const int b = rest / L0;
        const T* src = (b & 1) ? buf1 : buf0;
        T* dst = (b & 1) ? buf0 : buf1;
        const int64_t x0 = (int64_t)ix * Wt, y0 = (int64_t)iy * H;
        const int64_t olo = x0 + (int64_t)w * Wo;
        int64_t ohi = olo + Wo;
        if (ohi > x0 + Wt) ohi = x0 + Wt;
        if (ohi > g.e[1]) ohi = g.e[1];
        if (olo < ohi) warp_tile<T, EXACT, K, true>(src, dst, g, c, y0, H, olo, ohi, vec_ok);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            release_successors(q, 2, b, iy, ix, 0);
        }
    }
}

template <class T>
bool vec_aligned(const DevGeo& g, const void* a, const void* b) {
    const uintptr_t m = 15;
    return ((uintptr_t)a & m) == 0 && ((uintptr_t)b & m) == 0 && ((g.s[0] * (int64_t)sizeof(T)) & 15) == 0;
}

template <class T, bool EXACT, int K>
cudaError_t slt_k(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst) {
    const Coeffs<T> c = coeffs_as<T>(L.coeffs);
    dim3 grd((unsigned)t.count[1], (unsigned)t.count[0]);
    if (t.count[0] > 65535) return cudaErrorInvalidConfiguration;
    slt_kernel<T, EXACT, K><<<grd, 32 * t.nwarps, 0, L.stream>>>((const T*)src, (T*)dst, L.geo, c, t.ext[0],
                                                                 t.ext[1], vec_aligned<T>(L.geo, src, dst));
    return cudaGetLastError();
}

template <class T, bool EXACT, int K>
cudaError_t cot_k(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
    const Coeffs<T> c = coeffs_as<T>(L.coeffs);
    cot_kernel<T, EXACT, K><<<nctas, 32 * t.nwarps, 0, L.stream>>>((T*)b0, (T*)b1, L.geo, c, t.ext[0], t.ext[1],
                                                                   vec_aligned<T>(L.geo, b0, b1), q);
    return cudaGetLastError();
}

template <class T, bool EXACT, int K>
int occ_k(const TileGeo& t) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cot_kernel<T, EXACT, K>, 32 * t.nwarps, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

// Depth dispatch.  F32 depths: 1 2 3 4 6 8; F64 (both modes): 1 2 3 4.
#define PCOT_F32_DEPTHS(X) X(1) X(2) X(3) X(4) X(6) X(8)
#define PCOT_F64_DEPTHS(X) X(1) X(2) X(3) X(4)

template <class T, bool EXACT>
int wo_for(int K) {
    constexpr int E = Vec<T>::E;
    const int Kp = ((K + E - 1) / E) * E;
    return 32 * E - 2 * Kp;
}

}  // namespace

int depths(int dtype, int* out, int cap) {
    static const int f32[] = {1, 2, 3, 4, 6, 8};
    static const int f64[] = {1, 2, 3, 4};
    const int* src = dtype == kF32 ? f32 : f64;
    const int n = dtype == kF32 ? 6 : 4;
    for (int i = 0; i < n && i < cap; ++i) out[i] = src[i];
    return n;
}

bool choose(const LaunchCtx& L, const int32_t* req, int depth, TileGeo* t) {
    if (L.geo.dims != 2) return false;
    int ds[16];
    const int nd = depths(L.dtype, ds, 16);
    bool ok = false;
    for (int i = 0; i < nd; ++i) ok = ok || ds[i] == depth;
    if (!ok) return false;
    const int Wo = L.dtype == kF32 ? wo_for<float, false>(depth) : wo_for<double, false>(depth);
    int64_t H = req && req[0] > 0 ? req[0] : 64;
    int64_t Wreq = req && req[1] > 0 ? req[1] : 4 * Wo;
    int nw = (int)((Wreq + Wo / 2) / Wo);
    if (nw < 1) nw = 1;
    if (nw > kMaxWarps) nw = kMaxWarps;
    if (H < depth) H = depth;  // the halo must stay within the neighbouring tile
    t->family = kFamStream2D;
    t->depth = depth;
    t->nwarps = nw;
    t->ext[0] = H;
    t->ext[1] = (int64_t)nw * Wo;
    t->ext[2] = 1;
    t->count[0] = (L.geo.e[0] + H - 1) / H;
    t->count[1] = (L.geo.e[1] + t->ext[1] - 1) / t->ext[1];
    t->count[2] = 1;
    return true;
}

cudaError_t slt(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst) {
#define PCOT_CASE(K)                                                    \
    case K:                                                             \
        if (L.dtype == kF32) return slt_k<float, false, K>(L, t, src, dst); \
        if (L.dtype == kF64) return slt_k<double, false, K>(L, t, src, dst); \
        return slt_k<double, true, K>(L, t, src, dst);
    switch (t.depth) {
        PCOT_F64_DEPTHS(PCOT_CASE)
        case 6: if (L.dtype == kF32) return slt_k<float, false, 6>(L, t, src, dst); break;
        case 8: if (L.dtype == kF32) return slt_k<float, false, 8>(L, t, src, dst); break;
    }
#undef PCOT_CASE
    return cudaErrorInvalidValue;
}

cudaError_t cot(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
#define PCOT_CASE(K)                                                          \
    case K:                                                                   \
        if (L.dtype == kF32) return cot_k<float, false, K>(L, t, b0, b1, q, nctas); \
        if (L.dtype == kF64) return cot_k<double, false, K>(L, t, b0, b1, q, nctas); \
        return cot_k<double, true, K>(L, t, b0, b1, q, nctas);
    switch (t.depth) {
        PCOT_F64_DEPTHS(PCOT_CASE)
        case 6: if (L.dtype == kF32) return cot_k<float, false, 6>(L, t, b0, b1, q, nctas); break;
        case 8: if (L.dtype == kF32) return cot_k<float, false, 8>(L, t, b0, b1, q, nctas); break;
    }
#undef PCOT_CASE
    return cudaErrorInvalidValue;
}

int ctas_per_sm(const LaunchCtx& L, const TileGeo& t) {
#define PCOT_CASE(K)                                               \
    case K:                                                        \
        if (L.dtype == kF32) return occ_k<float, false, K>(t);     \
        if (L.dtype == kF64) return occ_k<double, false, K>(t);    \
        return occ_k<double, true, K>(t);
    switch (t.depth) {
        PCOT_F64_DEPTHS(PCOT_CASE)
        case 6: return occ_k<float, false, 6>(t);
        case 8: return occ_k<float, false, 8>(t);
    }
#undef PCOT_CASE
    return 1;
}

}  // namespace stream2d
}  // namespace pcot
