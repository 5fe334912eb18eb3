// Generic tile kernel: the whole trapezoid of one tile in shared memory.
//
// The CTA loads its output box widened by K cells per side, then applies K
// steps in shared memory (ping-pong), each step updating a box one cell
// narrower per side, and stores the output box.  This is the base function of
// Sec. 4.2 run on a GPU tile (lexicographic point order is irrelevant inside
// a step because points of one step are independent).  Any dims (1..3) and
// any depth K; used for 1-D grids and for shapes the streaming families do
// not cover.
#include "tiled.cuh"

namespace pcot {
namespace generic {

namespace {

constexpr int kThreads = 256;
constexpr size_t kMaxSmem = 200 * 1024;

template <int DIMS>
struct Box {
    int64_t lo[3];  // storage coordinate of local index 0
    int64_t R[3];   // local extent
    int64_t ls[3];  // local strides
    int64_t total;
};

template <class T, bool EXACT, int DIMS, bool CG>
__device__ void tile_body(const T* __restrict__ src, T* __restrict__ dst, const DevGeo& g, const Coeffs<T>& c,
                          const int64_t* o, const int64_t* w, int K, T* sm) {
    Box<DIMS> bx;
    bx.total = 1;
    for (int a = DIMS - 1; a >= 0; --a) {
        bx.lo[a] = o[a] - K;
        bx.R[a] = w[a] + 2 * K;
        bx.ls[a] = bx.total;
        bx.total *= bx.R[a];
    }
    T* A = sm;
    T* B = sm + bx.total;
    const bool per = g.periodic != 0;

    // Load the widened box (cells outside a Dirichlet grid read as 0).
    for (int64_t idx = threadIdx.x; idx < bx.total; idx += blockDim.x) {
        int64_t r = idx, off = 0;
        bool in = true;
        for (int a = DIMS - 1; a >= 0; --a) {
            const int64_t p = r % bx.R[a];
            r /= bx.R[a];
            int64_t q = bx.lo[a] + p;
            if (per) q = wrapc(q, g.n[a]);
            else if (q < 0 || q >= g.e[a]) in = false;
            off += q * g.s[a];
        }
        A[idx] = in ? gload<CG>(src + off) : T(0);
    }
    __syncthreads();

    for (int s = 1; s <= K; ++s) {
        int64_t sub[3], subt = 1;
        for (int a = 0; a < DIMS; ++a) {
            sub[a] = bx.R[a] - 2 * s;
            subt *= sub[a];
        }
        for (int64_t idx = threadIdx.x; idx < subt; idx += blockDim.x) {
            int64_t r = idx, li = 0;
            bool inner = true;
            for (int a = DIMS - 1; a >= 0; --a) {
                const int64_t p = r % sub[a] + s;
                r /= sub[a];
                li += p * bx.ls[a];
                if (!per) {
                    const int64_t q = bx.lo[a] + p;
                    inner = inner && q >= 1 && q <= g.n[a];
                }
            }
            T v;
            if (!inner) {
                v = A[li];  // ring (or outside): never updated
            } else if (DIMS == 1) {
                v = upd1<T, EXACT>(c, A[li], A[li - 1], A[li + 1]);
            } else if (DIMS == 2) {
                v = upd2<T, EXACT>(c, A[li], A[li - bx.ls[0]], A[li + bx.ls[0]], A[li - 1], A[li + 1]);
            } else {
                v = upd3<T, EXACT>(c, A[li], A[li - bx.ls[0]], A[li + bx.ls[0]], A[li - bx.ls[1]],
                                   A[li + bx.ls[1]], A[li - 1], A[li + 1]);
            }
            B[li] = v;
        }
        __syncthreads();
        T* tmp = A;
        A = B;
        B = tmp;
    }

    // Store the output box (interior cells only).
    int64_t ot = 1;
    for (int a = 0; a < DIMS; ++a) ot *= w[a];
    for (int64_t idx = threadIdx.x; idx < ot; idx += blockDim.x) {
        int64_t r = idx, li = 0, off = 0;
        bool ok = true;
        for (int a = DIMS - 1; a >= 0; --a) {
            const int64_t p = r % w[a];
            r /= w[a];
            const int64_t q = o[a] + p;
            ok = ok && (per ? q < g.n[a] : (q >= 1 && q <= g.n[a]));
            li += (p + K) * bx.ls[a];
            off += q * g.s[a];
        }
        if (ok) dst[off] = A[li];
    }
}

template <class T, bool EXACT, int DIMS>
__global__ void __launch_bounds__(kThreads) slt_kernel(const T* __restrict__ src, T* __restrict__ dst, DevGeo g,
                                                       Coeffs<T> c, TileGeo t) {
    extern __shared__ __align__(16) unsigned char smraw[];
    int64_t r = blockIdx.x, o[3], w[3];
    for (int a = DIMS - 1; a >= 0; --a) {
        const int64_t i = r % t.count[a];
        r /= t.count[a];
        o[a] = i * t.ext[a];
        w[a] = t.ext[a];
    }
    tile_body<T, EXACT, DIMS, false>(src, dst, g, c, o, w, t.depth, reinterpret_cast<T*>(smraw));
}

template <class T, bool EXACT, int DIMS>
__global__ void __launch_bounds__(kThreads) cot_kernel(T* buf0, T* buf1, DevGeo g, Coeffs<T> c, TileGeo t,
                                                       CotDev q) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = pop_and_wait(q);
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) return;
        int64_t r = tile, o[3], w[3];
        int ii[3] = {0, 0, 0};
        for (int a = DIMS - 1; a >= 0; --a) {
            const int64_t i = r % q.lattice[1 + a];
            r /= q.lattice[1 + a];
            ii[a] = (int)i;
            o[a] = i * t.ext[a];
            w[a] = t.ext[a];
        }
        // Unused lattice axes have extent 1, so the remaining quotient is b.
        for (int a = DIMS; a < 3; ++a) r /= q.lattice[1 + a];
        const int b = (int)r;
        const T* src = (b & 1) ? buf1 : buf0;
        T* dst = (b & 1) ? buf0 : buf1;
        tile_body<T, EXACT, DIMS, true>(src, dst, g, c, o, w, t.depth, reinterpret_cast<T*>(smraw));
        __syncthreads();  // the tile's stores by every thread precede thread 0's release
        if (threadIdx.x == 0) release_successors(q, DIMS, b, ii[0], ii[1], ii[2]);
    }
}

template <class T>
size_t smem_t(const TileGeo& t, int dims) {
    size_t tot = 1;
    for (int a = 0; a < dims; ++a) tot *= (size_t)(t.ext[a] + 2 * t.depth);
    return 2 * tot * sizeof(T);
}

template <class T, bool EXACT, int DIMS>
cudaError_t slt_t(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst) {
    const size_t sm = smem_t<T>(t, DIMS);
    cudaError_t e = cudaFuncSetAttribute(slt_kernel<T, EXACT, DIMS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int64_t n = 1;
    for (int a = 0; a < DIMS; ++a) n *= t.count[a];
    if (n > 0x7fffffff) return cudaErrorInvalidConfiguration;
    slt_kernel<T, EXACT, DIMS><<<(unsigned)n, kThreads, sm, L.stream>>>((const T*)src, (T*)dst, L.geo,
                                                                        coeffs_as<T>(L.coeffs), t);
    return cudaGetLastError();
}

template <class T, bool EXACT, int DIMS>
cudaError_t cot_t(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
    const size_t sm = smem_t<T>(t, DIMS);
    cudaError_t e = cudaFuncSetAttribute(cot_kernel<T, EXACT, DIMS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    cot_kernel<T, EXACT, DIMS><<<nctas, kThreads, sm, L.stream>>>((T*)b0, (T*)b1, L.geo, coeffs_as<T>(L.coeffs), t, q);
    return cudaGetLastError();
}

template <class T, bool EXACT, int DIMS>
int occ_t(const TileGeo& t) {
    const size_t sm = smem_t<T>(t, DIMS);
    if (cudaFuncSetAttribute(cot_kernel<T, EXACT, DIMS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cot_kernel<T, EXACT, DIMS>, kThreads, sm) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace

bool choose(const LaunchCtx& L, const int32_t* req, int depth, TileGeo* t) {
    const int d = L.geo.dims;
    if (depth < 1 || depth > 64) return false;
    static const int64_t def[3][3] = {{1024, 1, 1}, {32, 64, 1}, {8, 8, 32}};
    t->family = kFamGeneric;
    t->depth = depth;
    t->nwarps = kThreads / 32;
    for (int a = 0; a < 3; ++a) {
        if (a < d) {
            int64_t w = req && req[a] > 0 ? req[a] : def[d - 1][a];
            if (w < depth) w = depth;  // halo within the neighbouring tile
            t->ext[a] = w;
            t->count[a] = (L.geo.e[a] + w - 1) / w;
        } else {
            t->ext[a] = 1;
            t->count[a] = 1;
        }
    }
    return smem(L, *t) <= kMaxSmem;
}

size_t smem(const LaunchCtx& L, const TileGeo& t) {
    return L.dtype == kF32 ? smem_t<float>(t, L.geo.dims) : smem_t<double>(t, L.geo.dims);
}

#define PCOT_DISPATCH(FN, ...)                                                             \
    switch (L.geo.dims) {                                                                  \
        case 1:                                                                            \
            if (L.dtype == kF32) return FN<float, false, 1>(__VA_ARGS__);                  \
            if (L.dtype == kF64) return FN<double, false, 1>(__VA_ARGS__);                 \
            return FN<double, true, 1>(__VA_ARGS__);                                       \
        case 2:                                                                            \
            if (L.dtype == kF32) return FN<float, false, 2>(__VA_ARGS__);                  \
            if (L.dtype == kF64) return FN<double, false, 2>(__VA_ARGS__);                 \
            return FN<double, true, 2>(__VA_ARGS__);                                       \
        default:                                                                           \
            if (L.dtype == kF32) return FN<float, false, 3>(__VA_ARGS__);                  \
            if (L.dtype == kF64) return FN<double, false, 3>(__VA_ARGS__);                 \
            return FN<double, true, 3>(__VA_ARGS__);                                       \
    }

cudaError_t slt(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst) {
    PCOT_DISPATCH(slt_t, L, t, src, dst)
}

cudaError_t cot(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
    PCOT_DISPATCH(cot_t, L, t, b0, b1, q, nctas)
}

int ctas_per_sm(const LaunchCtx& L, const TileGeo& t) { PCOT_DISPATCH(occ_t, t) }

#undef PCOT_DISPATCH

}  // namespace generic
}  // namespace pcot
