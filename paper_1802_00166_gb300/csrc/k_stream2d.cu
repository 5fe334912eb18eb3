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
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "tiled.cuh"
#include "tma.cuh"

namespace pcot {
namespace stream2d {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxWarps = 8;
constexpr int kRingSlots = 4;   // S
constexpr int kRingRows = 3;    // G: one fill per cycle of the 3-phase register ring

template <int K, int E>
struct Shape {
    static constexpr int Kp = ((K + E - 1) / E) * E;   // halo rounded to whole lanes
    static constexpr int Wo = 32 * E - 2 * Kp;          // output columns per warp
};

// FP32 warps fed by TMA evaluate the update two cells at a time with the packed
// f32x2 multiply and fused multiply-add.  A lane's four columns c0..c3 are
// held in their natural order as the pairs P = (c0, c1) and Q = (c2, c3),
// exactly as a 16-byte vector load delivers them and a 16-byte store takes
// them.  The centre, north and south terms are whole pairs (packed); the west
// and east neighbours of a pair are shifted by one column -- (c-1, c0),
// (c1, c2), (c3, c4) -- and are applied as scalar FMAs on the halves of the
// running pair sums.  Assembling the shifted operands into register pairs
// instead took 3.5 register moves per stage and lane, and reordering the
// columns into (c0, c2), (c1, c3) pairs around every load and store another
// 14 per row; the compiler issued most of those moves as integer
// multiply-adds on the FMA pipe that the stencil itself saturates.  Every
// cell still sees the same rounded operations in the same order as the
// scalar path, so the results are bitwise unchanged.
//
// Boundary warps (CHECK: Dirichlet pass-through, partial stores) of the
// launch-per-block kernels run the same unrolled TMA loop as interior warps:
// a boundary tile row ends every single-level launch, so its speed sets the
// launch's tail (3.3x the instructions per row in a compact body made it
// 1.3-1.6x slower).  The persistent kernels interleave boundary tiles with
// interior ones and keep the compact body: a second unrolled body cost them
// more in instruction fetch than it saved (COT at k = 8: -11%).
template <bool CG>
constexpr bool kUnrolledCheck = !CG;

template <class T, bool EXACT, bool CHECK, bool TMA, bool CG>
constexpr bool kPacked = std::is_same<T, float>::value && !EXACT && TMA && (!CHECK || kUnrolledCheck<CG>);

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
// KPS: columns of the warp span left of the output (at least the halo of K
// steps; a single-step tile inside a deeper tile geometry keeps that
// geometry's span so it reads the same ring columns).
template <class T, bool EXACT, int K, bool CG, bool TMA, bool CHECK, int KPS>
__device__ __forceinline__ void warp_tile(const Args<T>& A, const CUtensorMap* tmap, T* ring, uint64_t* full,
                                          uint64_t* empty, int nwarps, int64_t y0, int64_t olo, int64_t ohi,
                                          int64_t x_cta, uint32_t fill_base) {
    constexpr int E = Vec<T>::E;
    using V = typename Vec<T>::V;
    constexpr int Kp = KPS;
    static_assert(KPS >= K && KPS % E == 0 && 2 * KPS < 32 * E, "warp span too small for the halo");
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
    bool any_st = false;
#pragma unroll
    for (int j = 0; j < E; ++j) any_st = any_st || st[j];

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
    int col_off = (int)(olo - Kp - x_cta) + lane * E;  // column inside the CTA span
    if (TMA && (col_off < 0 || col_off + E > A.nbox * A.BW)) {
        if (atomicCAS(&A.st->code, 0, kStatusBounds) == 0) A.st->info[3] = col_off;
        col_off = 0;  // never read outside the ring
    }
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
    const bool warp_xint = __all_sync(kFull, xint[0] && xint[E - 1]);

    constexpr bool PK = kPacked<T, EXACT, CHECK, TMA, CG>;
    static_assert(!PK || E == 4, "packed path assumes four columns per lane");
    float2 k2[3];  // centre, north, south as pairs; west and east as scalars
#pragma unroll
    for (int c = 0; c < 3; ++c) k2[c] = make_float2((float)A.c.c[c], (float)A.c.c[c]);
    const float kw = (float)A.c.c[3], ke = (float)A.c.c[4];

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

    // 32-bit row bookkeeping relative to ybeg: step i reads input row ybeg+i
    // and emits output row ro = y0 + i - 2K, stored for i in [ist_lo, ist_hi).
    auto clamp32 = [](int64_t v) { return (int)(v < -(1LL << 30) ? -(1LL << 30) : v > (1LL << 30) ? (1LL << 30) : v); };
    int ist_lo = 2 * K, ist_hi = 2 * K + (int)H;
    if (per) {
        ist_hi = min(ist_hi, clamp32(2 * K + ny - y0));
    } else {
        ist_lo = max(ist_lo, clamp32(2 * K + 1 - y0));
        ist_hi = min(ist_hi, clamp32(2 * K + ny + 1 - y0));
    }
    // Rows of time level s+1 produced at step i are ybeg + i - s - 1; they are
    // interior rows when i - s - 1 lies in [rlo, rhi].
    const int rlo = clamp32(1 - ybeg), rhi = clamp32(ny - ybeg);
    T* const dst_row0 = A.dst + xl + (y0 - 2 * K) * P;  // row of step 0 (only dereferenced in the store range)
    const int lane_ring = TMA ? box * A.box_elems + cc : 0;

    // The K stages of step i (phase U of the register ring): level s+1 of row
    // ybeg+i-s-1 from the three rows of level s, into out[] (level K).
    struct Row {
        T v[E];
    };
    auto stages = [&](auto Uc, int i) -> Row {
        constexpr int U = decltype(Uc)::value;
        constexpr int SA = U % 3, SB = (U + 1) % 3, SN = (U + 2) % 3;
        Row res;
        T* out = res.v;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if constexpr (PK) {
                // P = (c0, c1), Q = (c2, c3); operand order of upd2 in the
                // FMA modes: centre, north, west, east, and the south row
                // (this step's output of the previous stage) last
                const float wl = __shfl_up_sync(kFull, R[s][SB][3], 1);    // c3 of the lane to the west
                const float er = __shfl_down_sync(kFull, R[s][SB][0], 1);  // c0 of the lane to the east
                const float* b = R[s][SB];
                float2 oP = __fmul2_rn(k2[0], make_float2(b[0], b[1]));
                oP = __ffma2_rn(k2[1], make_float2(R[s][SA][0], R[s][SA][1]), oP);
                oP.x = __fmaf_rn(kw, wl, oP.x);
                oP.y = __fmaf_rn(kw, b[0], oP.y);
                oP.x = __fmaf_rn(ke, b[1], oP.x);
                oP.y = __fmaf_rn(ke, b[2], oP.y);
                oP = __ffma2_rn(k2[2], make_float2(R[s][SN][0], R[s][SN][1]), oP);
                float2 oQ = __fmul2_rn(k2[0], make_float2(b[2], b[3]));
                oQ = __ffma2_rn(k2[1], make_float2(R[s][SA][2], R[s][SA][3]), oQ);
                oQ.x = __fmaf_rn(kw, b[1], oQ.x);
                oQ.y = __fmaf_rn(kw, b[2], oQ.y);
                oQ.x = __fmaf_rn(ke, b[3], oQ.x);
                oQ.y = __fmaf_rn(ke, er, oQ.y);
                oQ = __ffma2_rn(k2[2], make_float2(R[s][SN][2], R[s][SN][3]), oQ);
                out[0] = oP.x;
                out[1] = oP.y;
                out[2] = oQ.x;
                out[3] = oQ.y;
            } else {
                const T wl = __shfl_up_sync(kFull, R[s][SB][E - 1], 1);
                const T er = __shfl_down_sync(kFull, R[s][SB][0], 1);
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const T W = j > 0 ? R[s][SB][j - 1] : wl;
                    const T Ea = j < E - 1 ? R[s][SB][j + 1] : er;
                    out[j] = upd2<T, EXACT>(A.c, R[s][SB][j], R[s][SA][j], R[s][SN][j], W, Ea);
                }
            }
            if constexpr (CHECK) {
                // Dirichlet pass-through
                const int rr = i - s - 1;
                const bool rint = rr >= rlo && rr <= rhi;
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
        return res;
    };

    auto store = [&](int i, T* rowp, const Row& res) {
        const T* out = res.v;
        if (i >= ist_lo && i < ist_hi) {
            if (svec) {
                V q;
                T* qq = reinterpret_cast<T*>(&q);
#pragma unroll
                for (int j = 0; j < E; ++j) qq[j] = out[j];
                *reinterpret_cast<V*>(rowp) = q;
            } else if (any_st) {
#pragma unroll
                for (int j = 0; j < E; ++j)
                    if (st[j]) rowp[j] = out[j];
            }
        }
    };

    // One step of the general loop (plain-load input; boundary warps of the
    // persistent kernels).
    auto step = [&](auto Uc, int i) {
        constexpr int U = decltype(Uc)::value;
        constexpr int SN = (U + 2) % 3;
        if constexpr (TMA) {
            const int f = i / kRingRows, r = i - f * kRingRows;
            const uint32_t gi = fill_base + (uint32_t)f;
            const int slot = (int)(gi & (kRingSlots - 1));
            if (r == 0) {
                if (producer && f + kRingSlots - 1 < nfill) issue(f + kRingSlots - 1);
                mbar_wait(&full[slot], (gi / kRingSlots) & 1, A.st, A.timeout_ns, 2);
            }
            const V q = *reinterpret_cast<const V*>(ring + (lane_ring + slot * A.slot_elems + r * A.BW));
            const T* qq = reinterpret_cast<const T*>(&q);
#pragma unroll
            for (int j = 0; j < E; ++j) R[0][SN][j] = qq[j];
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) R[0][SN][j] = pf[U][j];
            if (i + 3 < nrows) load_row(ybeg + i + 3, pf[U]);
        }
        const Row out = stages(Uc, i);
        if constexpr (TMA) {
            const int f = i / kRingRows;
            if (i - f * kRingRows == kRingRows - 1 || i == nrows - 1) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[(fill_base + (uint32_t)f) & (kRingSlots - 1)]);
            }
        }
        store(i, dst_row0 + (int64_t)i * P, out);
    };

    if constexpr (CHECK && !(TMA && kUnrolledCheck<CG>)) {
        // Boundary warps on plain loads or in a persistent kernel: one compact
        // body and explicit rotation of the rings, to keep the instruction
        // footprint small.
        for (int i = 0; i < nrows; ++i) {
            step(IC<0>{}, i);
#pragma unroll
            for (int s = 0; s < K; ++s)
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    R[s][0][j] = R[s][1][j];
                    R[s][1][j] = R[s][2][j];
                }
            if constexpr (!TMA) {
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const T t0 = pf[0][j];
                    pf[0][j] = pf[1][j];
                    pf[1][j] = pf[2][j];
                    pf[2][j] = t0;
                }
            }
        }
    } else if constexpr (TMA) {
        // Warps fed by TMA: one ring fill of kRingRows = 3 rows per iteration,
        // so the fill's wait and release and the phases of the register ring
        // are fixed at compile time.  The last fill's rows past H + 2K are
        // computed from real or zero-filled rows and never stored.  Boundary
        // warps of the single-level kernel run the same loop with the
        // pass-through in stages().
        static_assert(kRingRows == 3, "one fill per cycle of the register ring");
        auto fstep = [&](auto Uc, int ii, const T* src_row, T* out_row) {
            constexpr int SN = (decltype(Uc)::value + 2) % 3;
            const V q = *reinterpret_cast<const V*>(src_row);
            const T* qq = reinterpret_cast<const T*>(&q);
#pragma unroll
            for (int j = 0; j < E; ++j) R[0][SN][j] = qq[j];
            store(ii, out_row, stages(Uc, ii));
        };
        T* orow = dst_row0;
        const T* const lane_base = ring + lane_ring;
        for (int f = 0; f < nfill; ++f) {
            const uint32_t gi = fill_base + (uint32_t)f;
            const int slot = (int)(gi & (kRingSlots - 1));
            if (producer && f + kRingSlots - 1 < nfill) issue(f + kRingSlots - 1);
            mbar_wait(&full[slot], (gi / kRingSlots) & 1, A.st, A.timeout_ns, 2);
            const T* srow = lane_base + slot * A.slot_elems;
            const int i = 3 * f;
            fstep(IC<0>{}, i, srow, orow);
            fstep(IC<1>{}, i + 1, srow + A.BW, orow + P);
            fstep(IC<2>{}, i + 2, srow + 2 * A.BW, orow + 2 * P);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            orow += 3 * P;
        }
    } else {
        for (int i = 0; i < nrows; i += 3) {
            step(IC<0>{}, i);
            if (i + 1 < nrows) step(IC<1>{}, i + 1);
            if (i + 2 < nrows) step(IC<2>{}, i + 2);
        }
    }
}

// Does any cell this warp computes need the Dirichlet pass-through?
template <int K, int E, int KPS>
__device__ __forceinline__ bool needs_check(const DevGeo& g, int64_t y0, int64_t H, int64_t olo) {
    if (g.periodic) return false;
    constexpr int Kp = KPS;
    const int64_t xa = olo - Kp, xb = olo - Kp + 32 * E - 1;
    const int64_t ya = y0 - K - 1, yb = y0 + H + K;
    return !(xa >= 1 && xb <= g.n[1] && ya >= 1 && yb <= g.n[0]);
}

template <class T, bool EXACT, int K, bool CG, bool TMA, int KPS = Shape<K, Vec<T>::E>::Kp>
__device__ __forceinline__ void warp_tile_any(const Args<T>& A, const CUtensorMap* tmap, T* ring, uint64_t* full,
                                              uint64_t* empty, int nwarps, int64_t y0, int64_t olo, int64_t ohi,
                                              int64_t x_cta, uint32_t fill_base) {
    if (needs_check<K, Vec<T>::E, KPS>(A.g, y0, A.H, olo))
        warp_tile<T, EXACT, K, CG, TMA, true, KPS>(A, tmap, ring, full, empty, nwarps, y0, olo, ohi, x_cta, fill_base);
    else
        warp_tile<T, EXACT, K, CG, TMA, false, KPS>(A, tmap, ring, full, empty, nwarps, y0, olo, ohi, x_cta,
                                                    fill_base);
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

// Register budgets (registers per thread) of the K-stage tile kernels; the
// stage rings hold 3*K*E values.  The kernels are latency-bound, so resident
// warps matter: with one-warp CTAs an SM holds floor(2048 / budget) of them.
// Measured on Heat-2D 8192^2: the single-level kernel gains 4-13% from
// budgets near its spill-free minimum (more resident warps); the persistent
// kernels lose with them (the compiler's schedule under a tight budget costs
// more than the extra warps give), so they keep the roomier budgets.
enum class Kern { Slt, Cot, Batch };
template <Kern W, class T, int K, bool TMA>
constexpr int reg_budget() {
    if (std::is_same<T, float>::value && TMA) {
        if (W == Kern::Slt) return K >= 8 ? 152 : K >= 6 ? 120 : K >= 4 ? 96 : 128;
        if (W == Kern::Cot) return K >= 8 ? 184 : K >= 6 ? 160 : 128;
        return K >= 8 ? 184 : K >= 6 ? 160 : 128;
    }
    return K >= 8 ? 184 : (K >= 6 ? 160 : 128);
}

template <class T, bool EXACT, int K, bool TMA>
__global__ void __maxnreg__((reg_budget<Kern::Slt, T, K, TMA>())) slt_kernel(Args<T> A, const __grid_constant__ CUtensorMap tmap) {
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
__global__ void __maxnreg__((reg_budget<Kern::Cot, T, K, TMA>())) cot_kernel(Args<T> A, T* buf0, T* buf1, CotDev q,
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
        __syncthreads();  // the tile's stores by every thread precede thread 0's release
        if (threadIdx.x == 0) release_successors(q, 2, b, iy, ix, 0);
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


// Persistent kernel over the merged tile queue of a batch of grids.
template <class T, bool EXACT, int K, bool TMA>
__global__ void __maxnreg__((reg_budget<Kern::Batch, T, K, TMA>())) batch_kernel(BatchDev q, Coeffs<T> c) {
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int E = Vec<T>::E;
    constexpr int Wo = Shape<K, E>::Wo;
    constexpr int Kp = Shape<K, E>::Kp;
    __shared__ int s_g, s_local, s_pos;
    const int nwarps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5;
    Args<T> A{};
    A.c = c;
    A.st = q.status;
    A.timeout_ns = q.timeout_ns;
    A.nbox = q.nbox;
    A.BW = q.BW;
    A.box_elems = q.box_elems;
    A.slot_elems = q.slot_elems;
    const SmemRing<T> r = carve<T>(smraw, A);
    init_ring(r, nwarps);
    uint32_t fill_base = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int pos = atomicAdd(q.head, 1);
            int g = -1, local = 0;
            if (pos < q.ntiles) {
                if (pos == 0 && q.done_ns) q.done_ns[0] = globaltimer_ns();
                const int2 e = q.queue[pos];
                g = e.x;
                local = e.y;
                if (g < 0 || g >= q.nb || local < 0 || local >= q.desc[g].ntiles) {
                    if (atomicCAS(&q.status->code, 0, kStatusBounds) == 0) {
                        q.status->info[0] = pos;
                        q.status->info[1] = g;
                    }
                    atomicExch(&q.status->abort, 1);
                    g = -1;
                } else if (!wait_zero(q.counts + q.desc[g].count_base + local, q.status, q.timeout_ns, local, pos)) {
                    g = -1;
                }
                fence_proxy_async_global();  // TMA reads after the acquire of the counter
            }
            s_g = g;
            s_local = local;
            s_pos = pos;
        }
        __syncthreads();
        const int g = s_g;
        if (g < 0) return;
        const int local = s_local;
        const BatchDesc& d = q.desc[g];
        const int L1 = d.L1, L0 = d.L0;
        const int ix = local % L1;
        const int rest = local / L1;
        const int iy = rest % L0;
        const int b = rest / L0;
        Args<T> B = A;
        B.src = (const T*)d.buf[b & 1];
        B.dst = (T*)d.buf[(b + 1) & 1];
        B.g = d.g;
        B.H = d.H;
        B.Wt = d.Wt;
        B.vec_ok = d.vec_ok != 0;
        const int64_t x0 = (int64_t)ix * d.Wt, y0 = (int64_t)iy * d.H;
        const int64_t olo = x0 + (int64_t)w * Wo;
        int64_t ohi = olo + Wo;
        if (ohi > x0 + d.Wt) ohi = x0 + d.Wt;
        if (ohi > d.g.e[1]) ohi = d.g.e[1];
        if (ohi < olo) ohi = olo;
        const int depth = b < d.Pmain ? K : 1;
        if constexpr (TMA) {
            const CUtensorMap* map = &d.map[b & 1];
            if (threadIdx.x == 0) fence_tensormap_acquire(map);
            if (depth == K) {
                warp_tile_any<T, EXACT, K, true, true>(B, map, r.ring, r.full, r.empty, nwarps, y0, olo, ohi, x0 - Kp,
                                                       fill_base);
                fill_base += (uint32_t)((d.H + 2 * K + kRingRows - 1) / kRingRows);
            } else {
                warp_tile_any<T, EXACT, 1, true, true, Kp>(B, map, r.ring, r.full, r.empty, nwarps, y0, olo, ohi,
                                                           x0 - Kp, fill_base);
                fill_base += (uint32_t)((d.H + 2 + kRingRows - 1) / kRingRows);
            }
        } else if (olo < ohi) {
            (void)fill_base;
            if (depth == K)
                warp_tile_any<T, EXACT, K, true, false>(B, nullptr, nullptr, nullptr, nullptr, nwarps, y0, olo, ohi, 0, 0);
            else
                warp_tile_any<T, EXACT, 1, true, false, Kp>(B, nullptr, nullptr, nullptr, nullptr, nwarps, y0, olo, ohi,
                                                            0, 0);
        }
        __syncthreads();  // the tile's stores by every thread precede thread 0's release
        if (threadIdx.x == 0) {
            __threadfence();  // one fence, then relaxed decrements: a release pattern
            if (b + 1 < d.Ptotal) {
                for (int dy = -1; dy <= 1; ++dy) {
                    const int jy = iy + dy;
                    if (jy < 0 || jy >= L0) continue;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int jx = ix + dx;
                        if (jx < 0 || jx >= L1) continue;
                        const int succ = ((b + 1) * L0 + jy) * L1 + jx;
                        if (succ >= d.ntiles) {
                            atomicCAS(&q.status->code, 0, kStatusBounds);
                            continue;
                        }
                        red_relaxed_add_gpu(q.counts + d.count_base + succ, -1);
                    }
                }
            }
            if (atomicSub(q.remaining + g, 1) == 1 && q.done_ns) q.done_ns[1 + g] = globaltimer_ns();
        }
    }
}

// Copy the Dirichlet ring of every grid of the batch into its twin.
template <class T>
__global__ void batch_ring_kernel(BatchDev q) {
    const BatchDesc& d = q.desc[blockIdx.x];
    if (d.g.periodic) return;
    const T* src = (const T*)d.buf[0];
    T* dst = (T*)d.buf[1];
    const int64_t ey = d.g.e[0], ex = d.g.e[1], P = d.g.s[0];
    for (int64_t x = threadIdx.x; x < ex; x += blockDim.x) {
        dst[x] = src[x];
        dst[(ey - 1) * P + x] = src[(ey - 1) * P + x];
    }
    for (int64_t y = threadIdx.x; y < ey; y += blockDim.x) {
        dst[y * P] = src[y * P];
        dst[y * P + ex - 1] = src[y * P + ex - 1];
    }
}

// Grids whose block count is odd end in their twin: copy it back.
template <class T>
__global__ void batch_copy_kernel(BatchDev q) {
    const BatchDesc& d = q.desc[blockIdx.y];
    if (!d.final_copy) return;
    const T* src = (const T*)d.buf[1];
    T* dst = (T*)d.buf[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.span; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

template <class T>
size_t batch_smem(const BatchDev& q) {
    return 128 + (size_t)kRingSlots * q.slot_elems * sizeof(T) + 2 * kRingSlots * sizeof(uint64_t);
}

template <class T, bool EXACT, int K>
cudaError_t batch_launch_k(const double* coeffs, const BatchDev& q, int nwarps, int nctas, cudaStream_t s) {
    const size_t sm = batch_smem<T>(q);
    if (q.all_tma) {
        cudaError_t e = cudaFuncSetAttribute(batch_kernel<T, EXACT, K, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        batch_kernel<T, EXACT, K, true><<<nctas, 32 * nwarps, sm, s>>>(q, coeffs_as<T>(coeffs));
    } else {
        cudaError_t e = cudaFuncSetAttribute(batch_kernel<T, EXACT, K, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        batch_kernel<T, EXACT, K, false><<<nctas, 32 * nwarps, sm, s>>>(q, coeffs_as<T>(coeffs));
    }
    return cudaGetLastError();
}

template <class T, bool EXACT, int K>
int batch_occ_k(const BatchDev& q, int nwarps) {
    const size_t sm = batch_smem<T>(q);
    int n = 0;
    if (q.all_tma) {
        if (cudaFuncSetAttribute(batch_kernel<T, EXACT, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm) != cudaSuccess)
            return 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<T, EXACT, K, true>, 32 * nwarps, sm) !=
            cudaSuccess)
            return 1;
    } else {
        if (cudaFuncSetAttribute(batch_kernel<T, EXACT, K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm) != cudaSuccess)
            return 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<T, EXACT, K, false>, 32 * nwarps, sm) !=
            cudaSuccess)
            return 1;
    }
    return n > 0 ? n : 1;
}

}  // namespace

int ctas_per_sm(const LaunchCtx& L, const TileGeo& t);

int depths(int dtype, int* out, int cap) {
    static const int f32[] = {1, 2, 3, 4, 6, 8};
    static const int f64[] = {1, 2, 3, 4};
    const int* src = dtype == kF32 ? f32 : f64;
    const int n = dtype == kF32 ? 6 : 4;
    for (int i = 0; i < n && i < cap; ++i) out[i] = src[i];
    return n;
}

// Resident CTAs of the single-level kernel on the whole GPU (0 if no device).
int resident_slots(const LaunchCtx& L, int depth, int nwarps, int64_t Wt) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    TileGeo t{};
    t.depth = depth;
    t.nwarps = nwarps;
    t.ext[1] = Wt;
    const int per = ctas_per_sm(L, t);
    return per > 0 ? per * sms : 0;
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
    int64_t Wreq = req && req[1] > 0 ? req[1] : Wo;
    int nw = (int)((Wreq + Wo / 2) / Wo);
    if (nw < 1) nw = 1;
    if (nw > kMaxWarps) nw = kMaxWarps;
    const int64_t Wt = (int64_t)nw * Wo;
    const int64_t ey = L.geo.e[0];
    const int64_t Lx = (L.geo.e[1] + Wt - 1) / Wt;
    int64_t H = req && req[0] > 0 ? req[0] : 0;
    if (H == 0) {
        // Default height: the tallest tiles (least halo work) whose count
        // fills whole waves of resident CTAs, so no partial last wave idles
        // most of the GPU.  Without a device the height is a fixed 128.
        H = 128;
        const int slots = resident_slots(L, depth, nw, Wt);
        const int64_t hmin = std::max<int64_t>(16, 4 * depth), hmax = 512;
        if (slots > 0) {
            for (int64_t m = 1; m <= 64; ++m) {
                const int64_t Ly = m * slots / Lx;
                if (Ly < 1) continue;
                const int64_t h = (ey + Ly - 1) / Ly;
                if (h <= hmax) {
                    H = std::max(h, std::min(hmin, ey));
                    break;
                }
            }
        }
    }
    if (H < depth) H = depth;  // the halo must stay within the neighbouring tile
    t->family = kFamStream2D;
    t->depth = depth;
    t->nwarps = nw;
    t->ext[0] = H;
    t->ext[1] = Wt;
    t->ext[2] = 1;
    t->count[0] = (ey + H - 1) / H;
    t->count[1] = Lx;
    t->count[2] = 1;
    return true;
}


bool batch_tiles(const LaunchCtx& L, int depth, int nwarps, int64_t H, TileGeo* t) {
    if (L.geo.dims != 2 || L.geo.periodic) return false;
    int ds[16];
    const int nd = depths(L.dtype, ds, 16);
    bool ok = false;
    for (int i = 0; i < nd; ++i) ok = ok || ds[i] == depth;
    if (!ok || nwarps < 1 || nwarps > kMaxWarps) return false;
    const int E = L.dtype == kF32 ? 4 : 2;
    const int64_t Wt = (int64_t)nwarps * wo_for(depth, E);
    if (H < depth) H = depth;
    t->family = kFamStream2D;
    t->depth = depth;
    t->nwarps = nwarps;
    t->ext[0] = H;
    t->ext[1] = Wt;
    t->ext[2] = 1;
    t->count[0] = (L.geo.e[0] + H - 1) / H;
    t->count[1] = (L.geo.e[1] + Wt - 1) / Wt;
    t->count[2] = 1;
    return true;
}

bool batch_desc_tma(const LaunchCtx& L, const TileGeo& t, BatchDesc* d, BatchDev* ring) {
    const void* bufs[2] = {d->buf[0], d->buf[1]};
    CUtensorMap maps[2];
    bool ok;
    if (L.dtype == kF32) {
        Args<float> A{};
        A.vec_ok = d->vec_ok != 0;
        ok = tma_setup<float>(L, t, &A, bufs, maps);
        if (ok) {
            ring->nbox = A.nbox; ring->BW = A.BW; ring->box_elems = A.box_elems; ring->slot_elems = A.slot_elems;
        }
    } else {
        Args<double> A{};
        A.vec_ok = d->vec_ok != 0;
        ok = tma_setup<double>(L, t, &A, bufs, maps);
        if (ok) {
            ring->nbox = A.nbox; ring->BW = A.BW; ring->box_elems = A.box_elems; ring->slot_elems = A.slot_elems;
        }
    }
    if (ok) {
        d->map[0] = maps[0];
        d->map[1] = maps[1];
    }
    d->tma_ok = ok ? 1 : 0;
    return ok;
}

#define PCOT_BATCH_DISPATCH(FN, ...)                                                      \
    switch (depth) {                                                                      \
        case 1: if (dtype == kF32) return FN<float, false, 1>(__VA_ARGS__);               \
                if (dtype == kF64) return FN<double, false, 1>(__VA_ARGS__);              \
                return FN<double, true, 1>(__VA_ARGS__);                                  \
        case 2: if (dtype == kF32) return FN<float, false, 2>(__VA_ARGS__);               \
                if (dtype == kF64) return FN<double, false, 2>(__VA_ARGS__);              \
                return FN<double, true, 2>(__VA_ARGS__);                                  \
        case 4: if (dtype == kF32) return FN<float, false, 4>(__VA_ARGS__);               \
                if (dtype == kF64) return FN<double, false, 4>(__VA_ARGS__);              \
                return FN<double, true, 4>(__VA_ARGS__);                                  \
        case 6: if (dtype == kF32) return FN<float, false, 6>(__VA_ARGS__);               \
                break;                                                                    \
        case 8: if (dtype == kF32) return FN<float, false, 8>(__VA_ARGS__);               \
                break;                                                                    \
    }

cudaError_t batch_launch(int dtype, int depth, int nwarps, const double* coeffs, const BatchDev& q, int nctas,
                         cudaStream_t s) {
    PCOT_BATCH_DISPATCH(batch_launch_k, coeffs, q, nwarps, nctas, s)
    return cudaErrorInvalidValue;
}

int batch_ctas_per_sm(int dtype, int depth, int nwarps, const BatchDev& q) {
    PCOT_BATCH_DISPATCH(batch_occ_k, q, nwarps)
    return 1;
}

#undef PCOT_BATCH_DISPATCH

cudaError_t batch_final_copy(int dtype, const BatchDev& q, cudaStream_t s) {
    dim3 grd(64, (unsigned)q.nb);
    if (dtype == kF32) batch_copy_kernel<float><<<grd, 256, 0, s>>>(q);
    else batch_copy_kernel<double><<<grd, 256, 0, s>>>(q);
    return cudaGetLastError();
}

cudaError_t batch_ring_copy(int dtype, const BatchDev& q, cudaStream_t s) {
    if (dtype == kF32) batch_ring_kernel<float><<<q.nb, 256, 0, s>>>(q);
    else batch_ring_kernel<double><<<q.nb, 256, 0, s>>>(q);
    return cudaGetLastError();
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
