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
//
// Input rows arrive in one of two ways:
//  * TMA: the CTA's whole span (all warps plus the halo) is fetched with
//    cp.async.bulk.tensor into a ring of S shared-memory slots of G rows,
//    S-1 slots ahead of the consumers (full/empty mbarriers; warp 0's first
//    lane issues the copies).  Out-of-grid cells arrive as zeros.
//  * plain loads (periodic grids, layouts without 16-byte rows): each lane
//    keeps three rows of 16-byte loads in flight in registers.
#include <cstring>

#include "tiled.cuh"
#include "tma.cuh"

namespace pcot {
namespace stream2d {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxWarps = 8;
constexpr int kRingSlots = 4;   // S
constexpr int kRingRows = 4;    // G

template <int K, int E>
struct Shape {
    static constexpr int Kp = ((K + E - 1) / E) * E;   // halo rounded to whole lanes
    static constexpr int Wo = 32 * E - 2 * Kp;          // output columns per warp
};

template <class T>
struct Args {
    const T* src;
    T* dst;
    DevGeo g;
    Coeffs<T> c;
    int64_t H, Wt;
    bool vec_ok;
    // TMA ring
    int nbox, BW, box_elems, slot_elems;
    DevStatus* st;
    uint64_t timeout_ns;
};

// One warp's trapezoid.  x_cta: first column of the CTA's span (TMA ring
// origin); fill_base: fills of the ring consumed before this tile (COT).
template <class T, bool EXACT, int K, bool CG, bool TMA, bool CHECK>
__device__ __forceinline__ void warp_tile(const Args<T>& A, const CUtensorMap* tmap, T* ring, uint64_t* full,
                                          uint64_t* empty, int nwarps, int64_t y0, int64_t olo, int64_t ohi,
                                          int64_t x_cta, uint32_t fill_base) {
    constexpr int E = Vec<T>::E;
    using V = typename Vec<T>::V;
    constexpr int Kp = Shape<K, E>::Kp;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const DevGeo& g = A.g;
    const bool per = g.periodic != 0;
    const int64_t ey = g.e[0], ex = g.e[1], ny = g.n[0], nx = g.n[1], P = g.s[0];
    const int64_t xl = olo - Kp + (int64_t)lane * E;  // first column of this lane
    const int64_t H = A.H;

    bool inb[E], xint[E], st[E];
    int64_t col0 = 0;
    bool all_in = true, all_st = true;
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int64_t x = xl + j;
        if (per) {
            if (j == 0) col0 = wrap_fast(x, nx);
            inb[j] = true;
            xint[j] = true;
        } else {
            inb[j] = x >= 0 && x < ex;
            xint[j] = x >= 1 && x <= nx;
        }
        st[j] = x >= olo && x < ohi && xint[j];
        all_in = all_in && inb[j];
        all_st = all_st && st[j];
    }
    if (!per) col0 = xl;
    const bool contiguous = !per || (col0 + (E - 1) < nx);
    const bool lvec = A.vec_ok && all_in && contiguous && (col0 % E) == 0;
    const bool svec = A.vec_ok && all_st && (xl % E) == 0;

    const int64_t ybeg = y0 - K, yend = y0 + H + K;
    const int nrows = (int)(H + 2 * K);

    // ---- plain-load path: three rows in flight per lane --------------------
    auto load_row = [&](int64_t yi, T (&v)[E]) {
        int64_t ys;
        bool rin;
        if (per) {
            ys = wrap_fast(yi, ny);
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
        const T* rowp = A.src + ys * P;
        if (lvec) {
            const V q = gload<CG>(reinterpret_cast<const V*>(rowp + col0));
            const T* qq = reinterpret_cast<const T*>(&q);
#pragma unroll
            for (int j = 0; j < E; ++j) v[j] = qq[j];
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) {
                if (!inb[j]) {
                    v[j] = T(0);
                } else {
                    const int64_t cj = per ? wrap_fast(xl + j, nx) : xl + j;
                    v[j] = gload<CG>(rowp + cj);
                }
            }
        }
    };

    // ---- TMA path ----------------------------------------------------------
    const bool producer = TMA && warp == 0 && lane == 0;
    const int nfill = (nrows + kRingRows - 1) / kRingRows;
    const int col_off = (int)(olo - Kp - x_cta) + lane * E;  // column inside the CTA span
    const int box = TMA ? col_off / A.BW : 0;
    const int cc = TMA ? col_off - box * A.BW : 0;
    auto issue = [&](int f) {
        const uint32_t gi = fill_base + (uint32_t)f;
        const int slot = (int)(gi % kRingSlots);
        if (gi >= (uint32_t)kRingSlots)
            mbar_wait(&empty[slot], ((gi / kRingSlots) - 1) & 1, A.st, A.timeout_ns, 1);
        mbar_arrive_expect_tx(&full[slot], (unsigned)(A.nbox * kRingRows * A.BW * sizeof(T)));
        for (int b = 0; b < A.nbox; ++b)
            tma_load_2d(ring + (size_t)slot * A.slot_elems + (size_t)b * A.box_elems, tmap, (int)(x_cta + b * A.BW),
                        (int)(ybeg + f * kRingRows), &full[slot]);
    };
    if constexpr (TMA) {
        if (producer) {
            for (int f = 0; f < kRingSlots - 1 && f < nfill; ++f) issue(f);
        }
    }
    auto tma_row = [&](int i, T (&v)[E]) {
        const int f = i / kRingRows, r = i - f * kRingRows;
        const uint32_t gi = fill_base + (uint32_t)f;
        const int slot = (int)(gi % kRingSlots);
        if (r == 0) {
            if (producer && f + kRingSlots - 1 < nfill) issue(f + kRingSlots - 1);
            mbar_wait(&full[slot], (gi / kRingSlots) & 1, A.st, A.timeout_ns, 2);
        }
        const T* p = ring + (size_t)slot * A.slot_elems + (size_t)box * A.box_elems + r * A.BW + cc;
        const V q = *reinterpret_cast<const V*>(p);
        const T* qq = reinterpret_cast<const T*>(&q);
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = qq[j];
    };
    auto tma_done = [&](int i) {
        const int f = i / kRingRows, r = i - f * kRingRows;
        if (r == kRingRows - 1 || i == nrows - 1) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[(fill_base + (uint32_t)f) % kRingSlots]);
        }
    };

    const bool warp_xint = __all_sync(kFull, xint[0] && xint[E - 1]);

    T R[K][3][E];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int j = 0; j < E; ++j) R[s][u][j] = T(0);

    T pf[3][E];
    if constexpr (!TMA) {
        load_row(ybeg, pf[0]);
        if (ybeg + 1 < yend) load_row(ybeg + 1, pf[1]);
        if (ybeg + 2 < yend) load_row(ybeg + 2, pf[2]);
    }

    auto step = [&](auto Uc, int64_t yi) {
        constexpr int U = decltype(Uc)::value;
        constexpr int SA = U % 3, SB = (U + 1) % 3, SN = (U + 2) % 3;
        const int i = (int)(yi - ybeg);
        if constexpr (TMA) {
            tma_row(i, R[0][SN]);
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) R[0][SN][j] = pf[U][j];
            if (yi + 3 < yend) load_row(yi + 3, pf[U]);
        }
        T out[E];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            const T wl = __shfl_up_sync(kFull, R[s][SB][E - 1], 1);
            const T er = __shfl_down_sync(kFull, R[s][SB][0], 1);
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const T W = j > 0 ? R[s][SB][j - 1] : wl;
                const T Ea = j < E - 1 ? R[s][SB][j + 1] : er;
                out[j] = upd2<T, EXACT>(A.c, R[s][SB][j], R[s][SA][j], R[s][SN][j], W, Ea);
            }
            if constexpr (CHECK) {
                const int64_t r = yi - s - 1;  // row of time level s+1 produced now
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
        if constexpr (TMA) tma_done(i);
        const int64_t ro = yi - K;
        const bool rok = ro >= y0 && ro < y0 + H && (per ? ro < ny : (ro >= 1 && ro <= ny));
        if (rok) {
            T* rowp = A.dst + ro * P;
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

// Does any cell this warp computes need the Dirichlet pass-through?
template <int K, int E>
__device__ __forceinline__ bool needs_check(const DevGeo& g, int64_t y0, int64_t H, int64_t olo) {
    if (g.periodic) return false;
    constexpr int Kp = Shape<K, E>::Kp;
    const int64_t xa = olo - Kp, xb = olo - Kp + 32 * E - 1;
    const int64_t ya = y0 - K - 1, yb = y0 + H + K;
    return !(xa >= 1 && xb <= g.n[1] && ya >= 1 && yb <= g.n[0]);
}

template <class T, bool EXACT, int K, bool CG, bool TMA>
__device__ __forceinline__ void warp_tile_any(const Args<T>& A, const CUtensorMap* tmap, T* ring, uint64_t* full,
                                              uint64_t* empty, int nwarps, int64_t y0, int64_t olo, int64_t ohi,
                                              int64_t x_cta, uint32_t fill_base) {
    if (needs_check<K, Vec<T>::E>(A.g, y0, A.H, olo))
        warp_tile<T, EXACT, K, CG, TMA, true>(A, tmap, ring, full, empty, nwarps, y0, olo, ohi, x_cta, fill_base);
    else
        warp_tile<T, EXACT, K, CG, TMA, false>(A, tmap, ring, full, empty, nwarps, y0, olo, ohi, x_cta, fill_base);
}

template <class T>
struct SmemRing {
    T* ring;
    uint64_t* full;
    uint64_t* empty;
};

template <class T>
__device__ __forceinline__ SmemRing<T> carve(unsigned char* sm, const Args<T>& A) {
    SmemRing<T> r;
    const uint32_t a = smem_u32(sm);
    sm += ((a + 127u) & ~127u) - a;  // TMA destinations on 128-byte boundaries
    r.ring = reinterpret_cast<T*>(sm);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + (size_t)kRingSlots * A.slot_elems * sizeof(T));
    r.full = bars;
    r.empty = bars + kRingSlots;
    return r;
}

template <class T>
__device__ __forceinline__ void init_ring(const SmemRing<T>& r, int nwarps) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kRingSlots; ++s) {
            mbar_init(&r.full[s], 1);
            mbar_init(&r.empty[s], nwarps);
        }
        mbar_fence_init();
    }
    __syncthreads();
}

template <class T, bool EXACT, int K, bool TMA>
__global__ void __launch_bounds__(32 * kMaxWarps) slt_kernel(Args<T> A, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int Wo = Shape<K, Vec<T>::E>::Wo;
    constexpr int Kp = Shape<K, Vec<T>::E>::Kp;
    const int nwarps = blockDim.x >> 5;
    const int64_t x0 = (int64_t)blockIdx.x * A.Wt, y0 = (int64_t)blockIdx.y * A.H;
    const int w = threadIdx.x >> 5;
    const int64_t olo = x0 + (int64_t)w * Wo;
    int64_t ohi = olo + Wo;
    if (ohi > x0 + A.Wt) ohi = x0 + A.Wt;
    if (ohi > A.g.e[1]) ohi = A.g.e[1];
    if constexpr (TMA) {
        const SmemRing<T> r = carve<T>(smraw, A);
        init_ring(r, nwarps);
        if (ohi < olo) ohi = olo;  // idle warps still consume the ring
        warp_tile_any<T, EXACT, K, false, true>(A, &tmap, r.ring, r.full, r.empty, nwarps, y0, olo, ohi, x0 - Kp, 0);
    } else {
        if (olo >= ohi) return;
        warp_tile_any<T, EXACT, K, false, false>(A, nullptr, nullptr, nullptr, nullptr, nwarps, y0, olo, ohi, 0, 0);
    }
}

template <class T, bool EXACT, int K, bool TMA>
__global__ void __launch_bounds__(32 * kMaxWarps) cot_kernel(Args<T> A, T* buf0, T* buf1, CotDev q,
                                                             const __grid_constant__ CUtensorMap map0,
                                                             const __grid_constant__ CUtensorMap map1) {
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int Wo = Shape<K, Vec<T>::E>::Wo;
    constexpr int Kp = Shape<K, Vec<T>::E>::Kp;
    __shared__ int s_tile;
    const int nwarps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5;
    SmemRing<T> r{nullptr, nullptr, nullptr};
    if constexpr (TMA) {
        r = carve<T>(smraw, A);
        init_ring(r, nwarps);
    }
    const int nfill = (int)((A.H + 2 * K + kRingRows - 1) / kRingRows);
    uint32_t fill_base = 0;
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
        Args<T> B = A;
        B.src = (b & 1) ? buf1 : buf0;
        B.dst = (b & 1) ? buf0 : buf1;
        const int64_t x0 = (int64_t)ix * A.Wt, y0 = (int64_t)iy * A.H;
        const int64_t olo = x0 + (int64_t)w * Wo;
        int64_t ohi = olo + Wo;
        if (ohi > x0 + A.Wt) ohi = x0 + A.Wt;
        if (ohi > A.g.e[1]) ohi = A.g.e[1];
        if constexpr (TMA) {
            if (threadIdx.x == 0) fence_proxy_async_global();
            if (ohi < olo) ohi = olo;
            warp_tile_any<T, EXACT, K, true, true>(B, (b & 1) ? &map1 : &map0, r.ring, r.full, r.empty, nwarps, y0,
                                                   olo, ohi, x0 - Kp, fill_base);
            fill_base += (uint32_t)nfill;
        } else {
            if (olo < ohi)
                warp_tile_any<T, EXACT, K, true, false>(B, nullptr, nullptr, nullptr, nullptr, nwarps, y0, olo, ohi, 0,
                                                        0);
        }
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

template <int K, int E>
constexpr int wo_of() {
    return Shape<K, E>::Wo;
}

int wo_for(int K, int E) {
    const int Kp = ((K + E - 1) / E) * E;
    return 32 * E - 2 * Kp;
}

// Fill the TMA fields of Args; returns false when the ring cannot be used.
template <class T>
bool tma_setup(const LaunchCtx& L, const TileGeo& t, Args<T>* A, const void* bufs[2], CUtensorMap maps[2]) {
    constexpr int E = Vec<T>::E;
    const DevGeo& g = L.geo;
    if (g.periodic || !A->vec_ok) return false;
    if (g.e[1] >= (1LL << 31) || g.e[0] >= (1LL << 31)) return false;
    const int Kp = ((t.depth + E - 1) / E) * E;
    const int64_t SW = t.ext[1] + 2 * Kp;
    const int nbox = (int)((SW + 255) / 256);
    if (nbox > 4) return false;
    int BW = (int)((SW + nbox - 1) / nbox);
    BW = ((BW + E - 1) / E) * E;
    if (BW > 256) return false;
    A->nbox = nbox;
    A->BW = BW;
    const int align_elems = 128 / (int)sizeof(T);
    A->box_elems = ((BW * kRingRows + align_elems - 1) / align_elems) * align_elems;
    A->slot_elems = nbox * A->box_elems;
    for (int i = 0; i < 2; ++i) {
        if (!bufs[i]) {
            maps[i] = maps[0];
            continue;
        }
        if (!encode_tmap_2d(&maps[i], bufs[i], (int)sizeof(T), (uint64_t)g.e[1], (uint64_t)g.e[0],
                            (uint64_t)(g.s[0] * (int64_t)sizeof(T)), (uint32_t)BW, (uint32_t)kRingRows))
            return false;
    }
    return true;
}

template <class T>
size_t ring_bytes(const Args<T>& A) {
    return 128 + (size_t)kRingSlots * A.slot_elems * sizeof(T) + 2 * kRingSlots * sizeof(uint64_t);
}

template <class T, bool EXACT, int K>
cudaError_t slt_k(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst, DevStatus* st) {
    Args<T> A{};
    A.src = (const T*)src;
    A.dst = (T*)dst;
    A.g = L.geo;
    A.c = coeffs_as<T>(L.coeffs);
    A.H = t.ext[0];
    A.Wt = t.ext[1];
    A.vec_ok = vec_aligned<T>(L.geo, src, dst);
    A.st = st;
    A.timeout_ns = 2000000000ull;
    if (t.count[0] > 65535) return cudaErrorInvalidConfiguration;
    dim3 grd((unsigned)t.count[1], (unsigned)t.count[0]);
    CUtensorMap maps[2];
    const void* bufs[2] = {src, nullptr};
    if (st && tma_setup<T>(L, t, &A, bufs, maps)) {
        const size_t sm = ring_bytes(A);
        cudaError_t e = cudaFuncSetAttribute(slt_kernel<T, EXACT, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm);
        if (e != cudaSuccess) return e;
        slt_kernel<T, EXACT, K, true><<<grd, 32 * t.nwarps, sm, L.stream>>>(A, maps[0]);
    } else {
        CUtensorMap dummy;
        std::memset(&dummy, 0, sizeof(dummy));
        slt_kernel<T, EXACT, K, false><<<grd, 32 * t.nwarps, 0, L.stream>>>(A, dummy);
    }
    return cudaGetLastError();
}

template <class T, bool EXACT, int K>
cudaError_t cot_k(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
    Args<T> A{};
    A.g = L.geo;
    A.c = coeffs_as<T>(L.coeffs);
    A.H = t.ext[0];
    A.Wt = t.ext[1];
    A.vec_ok = vec_aligned<T>(L.geo, b0, b1);
    A.st = q.status;
    A.timeout_ns = q.timeout_ns;
    CUtensorMap maps[2];
    const void* bufs[2] = {b0, b1};
    if (tma_setup<T>(L, t, &A, bufs, maps)) {
        const size_t sm = ring_bytes(A);
        cudaError_t e = cudaFuncSetAttribute(cot_kernel<T, EXACT, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm);
        if (e != cudaSuccess) return e;
        cot_kernel<T, EXACT, K, true><<<nctas, 32 * t.nwarps, sm, L.stream>>>(A, (T*)b0, (T*)b1, q, maps[0], maps[1]);
    } else {
        CUtensorMap dummy;
        std::memset(&dummy, 0, sizeof(dummy));
        cot_kernel<T, EXACT, K, false><<<nctas, 32 * t.nwarps, 0, L.stream>>>(A, (T*)b0, (T*)b1, q, dummy, dummy);
    }
    return cudaGetLastError();
}

template <class T, bool EXACT, int K>
int occ_k(const LaunchCtx& L, const TileGeo& t) {
    // Occupancy of the TMA variant (the one used for aligned Dirichlet grids).
    Args<T> A{};
    A.g = L.geo;
    A.vec_ok = true;
    CUtensorMap maps[2];
    const void* bufs[2] = {nullptr, nullptr};
    size_t sm = 0;
    int n = 0;
    if (!L.geo.periodic) {
        constexpr int E = Vec<T>::E;
        const int Kp = ((t.depth + E - 1) / E) * E;
        const int64_t SW = t.ext[1] + 2 * Kp;
        const int nbox = (int)((SW + 255) / 256);
        int BW = (int)((SW + nbox - 1) / nbox);
        BW = ((BW + E - 1) / E) * E;
        const int align_elems = 128 / (int)sizeof(T);
        A.nbox = nbox;
        A.BW = BW;
        A.box_elems = ((BW * kRingRows + align_elems - 1) / align_elems) * align_elems;
        A.slot_elems = nbox * A.box_elems;
        sm = ring_bytes(A);
        (void)maps;
        (void)bufs;
        if (cudaFuncSetAttribute(cot_kernel<T, EXACT, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
            cudaSuccess)
            return 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cot_kernel<T, EXACT, K, true>, 32 * t.nwarps, sm) !=
            cudaSuccess)
            return 1;
    } else {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cot_kernel<T, EXACT, K, false>, 32 * t.nwarps, 0) !=
            cudaSuccess)
            return 1;
    }
    return n > 0 ? n : 1;
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
    const int E = L.dtype == kF32 ? 4 : 2;
    const int Wo = wo_for(depth, E);
    int64_t H = req && req[0] > 0 ? req[0] : 128;
    int64_t Wreq = req && req[1] > 0 ? req[1] : 2 * Wo;
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

#define PCOT_F64_DEPTHS(X) X(1) X(2) X(3) X(4)

cudaError_t slt(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst, DevStatus* st) {
#define PCOT_CASE(K)                                                                \
    case K:                                                                         \
        if (L.dtype == kF32) return slt_k<float, false, K>(L, t, src, dst, st);     \
        if (L.dtype == kF64) return slt_k<double, false, K>(L, t, src, dst, st);    \
        return slt_k<double, true, K>(L, t, src, dst, st);
    switch (t.depth) {
        PCOT_F64_DEPTHS(PCOT_CASE)
        case 6: if (L.dtype == kF32) return slt_k<float, false, 6>(L, t, src, dst, st); break;
        case 8: if (L.dtype == kF32) return slt_k<float, false, 8>(L, t, src, dst, st); break;
    }
#undef PCOT_CASE
    return cudaErrorInvalidValue;
}

cudaError_t cot(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
#define PCOT_CASE(K)                                                                \
    case K:                                                                         \
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
#define PCOT_CASE(K)                                                   \
    case K:                                                            \
        if (L.dtype == kF32) return occ_k<float, false, K>(L, t);      \
        if (L.dtype == kF64) return occ_k<double, false, K>(L, t);     \
        return occ_k<double, true, K>(L, t);
    switch (t.depth) {
        PCOT_F64_DEPTHS(PCOT_CASE)
        case 6: return occ_k<float, false, 6>(L, t);
        case 8: return occ_k<float, false, 8>(L, t);
    }
#undef PCOT_CASE
    return 1;
}

}  // namespace stream2d
}  // namespace pcot
