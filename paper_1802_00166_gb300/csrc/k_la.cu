// Blocked LU (no pivoting) and Cholesky factorizations on the GPU, the
// linear-algebra kernels of the benchmark suite (Sec. 5.1.2) whose
// iteration spaces are triangular (Sec. 4.3).  Three schedules:
//  * sweep: the plain loop over k, two launches per k (the column of
//    multipliers, then the trailing update), one thread per element;
//  * single-level: b x b x b tiles of the (k, i, j) space, block step kb by
//    block step: one launch for the panels and one for the updates (tiles of
//    one launch are independent); the diagonal tile of step kb+1 is factored
//    inside step kb's update launch by the CTA that updates that block last;
//  * recursive: the same tiles in the recursive order of planner_la.cpp, run
//    by a persistent kernel that pops the queue in order, waits (bounded) on
//    per-tile dependency counters and releases the successors of la_graph.h.
//
// A tile is computed by one CTA of 256 threads in FP64.  Every element sees
// the definition's operations in the definition's order: its updates
// c <- c - a*b for k ascending (a rounded product and a rounded difference,
// or one fused multiply-add in the fused mode), then its division (and, on
// the Cholesky diagonal, its square root), all correctly rounded -- so each
// schedule is bitwise equal to the plain loops.  An update tile keeps its
// output block in registers (each thread a 4 x 4 or 2 x 2 sub-block spread
// over rows ty + 16a and columns tx + 16b) and reads the two operand blocks
// from shared memory, rows padded by one element so that column walks are
// free of bank conflicts.  The work is bound by the FP64 pipe, which on this
// part issues far below the FP32 rate, not by memory: an update tile moves
// 4 b^2 words for b^3 multiply-adds.
#include "kernels.h"
#include "la_graph.h"

namespace pcot {

namespace {

constexpr int kLaThreads = 256;

template <bool FUSED>
__device__ __forceinline__ double la_upd(double c, double a, double b) {
    if constexpr (FUSED)
        return __fma_rn(-a, b, c);
    else
        return __dsub_rn(c, __dmul_rn(a, b));
}

template <int B>
struct LaTile {
    double v[B][B + 1];
};

template <int B>
constexpr size_t la_smem_bytes() {
    return 3 * sizeof(LaTile<B>);
}

template <int B>
__device__ __forceinline__ void load_tile(LaTile<B>& t, const double* A, int64_t lda, int64_t r0, int64_t c0, int nr,
                                          int nc) {
    for (int idx = threadIdx.x; idx < B * B; idx += kLaThreads) {
        const int r = idx / B, c = idx % B;
        t.v[r][c] = (r < nr && c < nc) ? __ldcg(A + (r0 + r) * lda + c0 + c) : 0.0;
    }
}

template <int B>
__device__ __forceinline__ void store_tile(const LaTile<B>& t, double* A, int64_t lda, int64_t r0, int64_t c0,
                                           int nr, int nc, bool lower_only) {
    for (int idx = threadIdx.x; idx < B * B; idx += kLaThreads) {
        const int r = idx / B, c = idx % B;
        if (r < nr && c < nc && (!lower_only || r >= c)) A[(r0 + r) * lda + c0 + c] = t.v[r][c];
    }
}

// LU of a diagonal block in place (nd x nd).
template <int B, bool FUSED>
__device__ void lu_diag(LaTile<B>& S, int nd) {
    for (int k = 0; k < nd; ++k) {
        const double piv = S.v[k][k];
        for (int i = k + 1 + (int)threadIdx.x; i < nd; i += kLaThreads) S.v[i][k] = __ddiv_rn(S.v[i][k], piv);
        __syncthreads();
        const int w = nd - k - 1;
        for (int idx = threadIdx.x; idx < w * w; idx += kLaThreads) {
            const int i = k + 1 + idx / w, j = k + 1 + idx % w;
            S.v[i][j] = la_upd<FUSED>(S.v[i][j], S.v[i][k], S.v[k][j]);
        }
        __syncthreads();
    }
}

// LU row panel: P (nd x nc) <- L^-1 P with L the unit lower factor in D.
template <int B, bool FUSED>
__device__ void lu_row_panel(const LaTile<B>& D, LaTile<B>& P, int nd, int nc) {
    for (int k = 0; k + 1 < nd; ++k) {
        const int w = nd - k - 1;
        for (int idx = threadIdx.x; idx < w * nc; idx += kLaThreads) {
            const int i = k + 1 + idx / nc, j = idx % nc;
            P.v[i][j] = la_upd<FUSED>(P.v[i][j], D.v[i][k], P.v[k][j]);
        }
        __syncthreads();
    }
}

// LU column panel: P (nr x nd) <- P U^-1 with U the upper factor in D.
template <int B, bool FUSED>
__device__ void lu_col_panel(const LaTile<B>& D, LaTile<B>& P, int nr, int nd) {
    for (int k = 0; k < nd; ++k) {
        const double piv = D.v[k][k];
        for (int i = threadIdx.x; i < nr; i += kLaThreads) P.v[i][k] = __ddiv_rn(P.v[i][k], piv);
        __syncthreads();
        const int w = nd - k - 1;
        for (int idx = threadIdx.x; idx < nr * w; idx += kLaThreads) {
            const int i = idx / w, j = k + 1 + idx % w;
            P.v[i][j] = la_upd<FUSED>(P.v[i][j], P.v[i][k], D.v[k][j]);
        }
        __syncthreads();
    }
}

// Cholesky of a diagonal block in place (lower triangle, nd x nd).
template <int B, bool FUSED>
__device__ void chol_diag(LaTile<B>& S, int nd) {
    for (int k = 0; k < nd; ++k) {
        if (threadIdx.x == 0) S.v[k][k] = __dsqrt_rn(S.v[k][k]);
        __syncthreads();
        const double piv = S.v[k][k];
        for (int i = k + 1 + (int)threadIdx.x; i < nd; i += kLaThreads) S.v[i][k] = __ddiv_rn(S.v[i][k], piv);
        __syncthreads();
        const int w = nd - k - 1;
        for (int idx = threadIdx.x; idx < w * w; idx += kLaThreads) {
            const int i = k + 1 + idx / w, j = k + 1 + idx % w;
            if (j <= i) S.v[i][j] = la_upd<FUSED>(S.v[i][j], S.v[i][k], S.v[j][k]);
        }
        __syncthreads();
    }
}

// Cholesky panel: P (nr x nd) <- P L^-T with L the factor in D.
template <int B, bool FUSED>
__device__ void chol_panel(const LaTile<B>& D, LaTile<B>& P, int nr, int nd) {
    for (int k = 0; k < nd; ++k) {
        const double piv = D.v[k][k];
        for (int i = threadIdx.x; i < nr; i += kLaThreads) P.v[i][k] = __ddiv_rn(P.v[i][k], piv);
        __syncthreads();
        const int w = nd - k - 1;
        for (int idx = threadIdx.x; idx < nr * w; idx += kLaThreads) {
            const int i = idx / w, j = k + 1 + idx % w;
            P.v[i][j] = la_upd<FUSED>(P.v[i][j], P.v[i][k], D.v[j][k]);
        }
        __syncthreads();
    }
}

// C (nr x nc at (r0, c0)) -= Sa * op(Sb) over nk terms, k ascending; op(Sb)
// is Sb (LU: Sb[k][c]) or Sb^T (Cholesky: Sb[c][k]).  lower_only keeps the
// strict upper part of a diagonal block untouched.
template <int B, bool FUSED, bool TRANS_B>
__device__ void update_tile(double* A, int64_t lda, int64_t r0, int64_t c0, int nr, int nc, int nk,
                            const LaTile<B>& Sa, const LaTile<B>& Sb, bool lower_only) {
    constexpr int R = B / 16;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    double c[R][R];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) {
            const int r = ty + 16 * a, col = tx + 16 * b;
            c[a][b] = (r < nr && col < nc) ? __ldcg(A + (r0 + r) * lda + c0 + col) : 0.0;
        }
#pragma unroll 4
    for (int k = 0; k < nk; ++k) {
        double av[R], bv[R];
#pragma unroll
        for (int a = 0; a < R; ++a) av[a] = Sa.v[ty + 16 * a][k];
#pragma unroll
        for (int b = 0; b < R; ++b) bv[b] = TRANS_B ? Sb.v[tx + 16 * b][k] : Sb.v[k][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < R; ++b) c[a][b] = la_upd<FUSED>(c[a][b], av[a], bv[b]);
    }
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) {
            const int r = ty + 16 * a, col = tx + 16 * b;
            if (r < nr && col < nc && (!lower_only || r >= col)) A[(r0 + r) * lda + c0 + col] = c[a][b];
        }
}

// The work of tile (kb, ib, jb); ends with a CTA barrier.
template <int B, bool FUSED, int KIND>
__device__ void run_tile(const LaDev& d, LaTile<B>* sm, int64_t kb, int64_t ib, int64_t jb) {
    const int64_t n = d.n, lda = d.lda;
    double* A = d.A;
    auto ext = [&](int64_t blk) { return (int)(n - blk * B < B ? n - blk * B : B); };
    const int nk = ext(kb), nr = ext(ib), nc = ext(jb);
    const int64_t k0 = kb * B, r0 = ib * B, c0 = jb * B;
    if (ib == kb && jb == kb) {
        load_tile<B>(sm[0], A, lda, k0, k0, nk, nk);
        __syncthreads();
        if constexpr (KIND == kLaLU)
            lu_diag<B, FUSED>(sm[0], nk);
        else
            chol_diag<B, FUSED>(sm[0], nk);
        store_tile<B>(sm[0], A, lda, k0, k0, nk, nk, KIND == kLaCholesky);
    } else if (ib == kb) {  // LU row panel (empty for Cholesky)
        load_tile<B>(sm[0], A, lda, k0, k0, nk, nk);
        load_tile<B>(sm[1], A, lda, k0, c0, nk, nc);
        __syncthreads();
        lu_row_panel<B, FUSED>(sm[0], sm[1], nk, nc);
        store_tile<B>(sm[1], A, lda, k0, c0, nk, nc, false);
    } else if (jb == kb) {
        load_tile<B>(sm[0], A, lda, k0, k0, nk, nk);
        load_tile<B>(sm[1], A, lda, r0, k0, nr, nk);
        __syncthreads();
        if constexpr (KIND == kLaLU)
            lu_col_panel<B, FUSED>(sm[0], sm[1], nr, nk);
        else
            chol_panel<B, FUSED>(sm[0], sm[1], nr, nk);
        store_tile<B>(sm[1], A, lda, r0, k0, nr, nk, false);
    } else {
        load_tile<B>(sm[0], A, lda, r0, k0, nr, nk);  // A(ib, kb)
        if constexpr (KIND == kLaLU) {
            load_tile<B>(sm[1], A, lda, k0, c0, nk, nc);  // A(kb, jb)
            __syncthreads();
            update_tile<B, FUSED, false>(A, lda, r0, c0, nr, nc, nk, sm[0], sm[1], false);
        } else {
            if (ib != jb) load_tile<B>(sm[1], A, lda, c0, k0, nc, nk);  // A(jb, kb)
            __syncthreads();
            update_tile<B, FUSED, true>(A, lda, r0, c0, nr, nc, nk, sm[0], ib == jb ? sm[0] : sm[1], ib == jb);
        }
    }
    __syncthreads();
}

template <int B, bool FUSED, int KIND>
__global__ void __launch_bounds__(kLaThreads) la_cot_kernel(LaDev d) {
    extern __shared__ __align__(16) unsigned char la_smraw[];
    LaTile<B>* sm = reinterpret_cast<LaTile<B>*>(la_smraw);
    __shared__ int s_tile;
    const int64_t L = d.L;
    for (;;) {
        if (threadIdx.x == 0) {
            int tile = -1;
            const int pos = atomicAdd(d.head, 1);
            if (pos < d.ntiles) {
                tile = d.queue[pos];
                if (tile < 0 || tile >= L * L * L) {
                    if (atomicCAS(&d.status->code, 0, kStatusBounds) == 0) {
                        d.status->info[0] = pos;
                        d.status->info[1] = tile;
                    }
                    atomicExch(&d.status->abort, 1);
                    tile = -1;
                } else if (!wait_zero(d.counts + tile, d.status, d.timeout_ns, tile, pos)) {
                    tile = -1;
                }
            }
            s_tile = tile;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) return;
        const int64_t jb = tile % L, ib = (tile / L) % L, kb = tile / (L * L);
        run_tile<B, FUSED, KIND>(d, sm, kb, ib, jb);
        if (threadIdx.x == 0) {
            // the barrier at the end of run_tile orders every thread's stores
            // before this fence; fence + relaxed reductions form the release
            __threadfence();
            la_for_each_successor(KIND, d.n, B, L, kb, ib, jb,
                                  [&](int64_t s) { red_relaxed_add_gpu(d.counts + s, -1); });
        }
    }
}

// One launch of the single-level schedule: phase 0 the diagonal tile of
// block step kb, phase 1 its panels, phase 2 its updates.  In phase 2 the
// CTA of the first update tile, (kb, kb+1, kb+1), goes on to factor that
// block as the diagonal tile of step kb+1 (it depends on nothing else), so
// the next step needs no launch of its own for it and the factorization
// overlaps the rest of this step's updates.
template <int B, bool FUSED, int KIND>
__global__ void __launch_bounds__(kLaThreads) la_step_kernel(LaDev d, int kb, int phase) {
    extern __shared__ __align__(16) unsigned char la_smraw[];
    LaTile<B>* sm = reinterpret_cast<LaTile<B>*>(la_smraw);
    const int64_t L = d.L, m = L - 1 - kb, x = blockIdx.x;
    int64_t ib = kb, jb = kb;
    if (phase == 1) {
        if (KIND == kLaLU && x < m) {
            jb = kb + 1 + x;  // row panel
        } else {
            ib = kb + 1 + (KIND == kLaLU ? x - m : x);  // column panel
        }
    } else if (phase == 2) {
        if (KIND == kLaLU) {
            ib = kb + 1 + x / m;
            jb = kb + 1 + x % m;
        } else {
            // x-th pair (p, q), q <= p, of the lower triangle of m x m, row by row
            int64_t p = (int64_t)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
            while (p * (p + 1) / 2 > x) --p;
            while ((p + 1) * (p + 2) / 2 <= x) ++p;
            ib = kb + 1 + p;
            jb = kb + 1 + (x - p * (p + 1) / 2);
        }
    }
    if (!la_tile_nonempty(KIND, d.n, B, L, kb, ib, jb)) return;
    run_tile<B, FUSED, KIND>(d, sm, kb, ib, jb);
    // run_tile ends with a CTA barrier, so this CTA's stores of the block are
    // visible to its own loads of it below
    if (phase == 2 && x == 0 && la_tile_nonempty(KIND, d.n, B, L, kb + 1, kb + 1, kb + 1))
        run_tile<B, FUSED, KIND>(d, sm, kb + 1, kb + 1, kb + 1);
}

// ---- the plain loop over k ------------------------------------------------

template <int KIND>
__global__ void la_sweep_col(double* A, int64_t lda, int64_t n, int64_t k) {
    const int64_t i = k + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double piv = KIND == kLaLU ? A[k * lda + k] : __dsqrt_rn(A[k * lda + k]);
    A[i * lda + k] = __ddiv_rn(A[i * lda + k], piv);
}

// Trailing update of step k: block (32 x 8) covers columns j and rows i > k.
// Cholesky updates j <= i only and its first thread stores the diagonal's
// square root (which no thread of this launch reads).
template <bool FUSED, int KIND>
__global__ void la_sweep_trail(double* A, int64_t lda, int64_t n, int64_t k) {
    const int64_t j = k + 1 + (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
    const int64_t i = k + 1 + (int64_t)blockIdx.y * 8 + (threadIdx.x >> 5);
    if (KIND == kLaCholesky && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
        A[k * lda + k] = __dsqrt_rn(A[k * lda + k]);
    if (i >= n || j >= n) return;
    if (KIND == kLaLU) {
        A[i * lda + j] = la_upd<FUSED>(A[i * lda + j], A[i * lda + k], A[k * lda + j]);
    } else if (j <= i) {
        A[i * lda + j] = la_upd<FUSED>(A[i * lda + j], A[i * lda + k], A[j * lda + k]);
    }
}

template <int B, bool FUSED, int KIND>
cudaError_t la_launch_t(const LaDev& d, int schedule, int nctas, cudaStream_t s, int64_t* launches) {
    const size_t sm = la_smem_bytes<B>();
    if (schedule == kLaSweep) {
        for (int64_t k = 0; k < d.n; ++k) {
            const int64_t w = d.n - k - 1;
            if (w > 0) {
                la_sweep_col<KIND><<<(unsigned)((w + 255) / 256), 256, 0, s>>>(d.A, d.lda, d.n, k);
                ++*launches;
            }
            if (w > 0 || KIND == kLaCholesky) {
                const dim3 g((unsigned)(w > 0 ? (w + 31) / 32 : 1), (unsigned)(w > 0 ? (w + 7) / 8 : 1));
                la_sweep_trail<FUSED, KIND><<<g, 256, 0, s>>>(d.A, d.lda, d.n, k);
                ++*launches;
            }
        }
        return cudaGetLastError();
    }
    if (schedule == kLaSlt) {
        cudaError_t e = cudaFuncSetAttribute(la_step_kernel<B, FUSED, KIND>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        bool diag_done = false;  // factored by the previous step's update launch
        for (int64_t kb = 0; kb < d.L; ++kb) {
            const int64_t m = d.L - 1 - kb;
            const int64_t counts[3] = {diag_done ? 0 : 1, KIND == kLaLU ? 2 * m : m,
                                       KIND == kLaLU ? m * m : m * (m + 1) / 2};
            for (int ph = 0; ph < 3; ++ph) {
                if (counts[ph] == 0) continue;
                la_step_kernel<B, FUSED, KIND><<<(unsigned)counts[ph], kLaThreads, sm, s>>>(d, (int)kb, ph);
                ++*launches;
            }
            diag_done = counts[2] > 0;
        }
        return cudaGetLastError();
    }
    cudaError_t e =
        cudaFuncSetAttribute(la_cot_kernel<B, FUSED, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    la_cot_kernel<B, FUSED, KIND><<<nctas, kLaThreads, sm, s>>>(d);
    ++*launches;
    return cudaGetLastError();
}

template <int B>
int la_ctas_per_sm_t(bool fused, int kind) {
    int n = 0;
    const size_t sm = la_smem_bytes<B>();
    auto occ = [&](auto kern) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return 0;
        int r = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kern, kLaThreads, sm) != cudaSuccess) return 0;
        return r;
    };
    if (kind == kLaLU)
        n = fused ? occ(la_cot_kernel<B, true, kLaLU>) : occ(la_cot_kernel<B, false, kLaLU>);
    else
        n = fused ? occ(la_cot_kernel<B, true, kLaCholesky>) : occ(la_cot_kernel<B, false, kLaCholesky>);
    return n;
}

}  // namespace

bool la_block_supported(int b) { return b == 32 || b == 64; }

int la_ctas_per_sm(int b, bool fused, int kind) {
    return b == 32 ? la_ctas_per_sm_t<32>(fused, kind) : la_ctas_per_sm_t<64>(fused, kind);
}

cudaError_t launch_la(const LaDev& d, int kind, bool fused, int schedule, int nctas, cudaStream_t s,
                      int64_t* launches) {
    if (!la_block_supported(d.b)) return cudaErrorInvalidValue;
#define PCOT_LA_CASE(BB, FF, KK) \
    if (d.b == BB && fused == FF && kind == KK) return la_launch_t<BB, FF, KK>(d, schedule, nctas, s, launches);
    PCOT_LA_CASE(32, false, kLaLU)
    PCOT_LA_CASE(32, true, kLaLU)
    PCOT_LA_CASE(64, false, kLaLU)
    PCOT_LA_CASE(64, true, kLaLU)
    PCOT_LA_CASE(32, false, kLaCholesky)
    PCOT_LA_CASE(32, true, kLaCholesky)
    PCOT_LA_CASE(64, false, kLaCholesky)
    PCOT_LA_CASE(64, true, kLaCholesky)
#undef PCOT_LA_CASE
    return cudaErrorInvalidValue;
}

}  // namespace pcot
