// C ABI of the stencil engine: argument checks, workspace layout, schedule
// execution (sweep / single-level / recursive persistent), status block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "kernels.h"
#include "pcot.h"
#include "la_graph.h"
#include "planner.h"
#include "picker_model.inc"  // generated by the build from the trained picker (may hold no model)

using namespace pcot;

namespace {

constexpr size_t kAlign = 256;
constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;  // 2 s per dependency wait

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct CotPlanHost {
    TileGeo tg{};
    int k = 0;
    int P = 0;                 // blocks run by the persistent kernel
    int32_t lattice[4] = {0, 1, 1, 1};
    int64_t ntiles = 0;
    BlockPlan tail;            // blocks run afterwards by single-level launches
    std::vector<int32_t> queue, counts;
    void* pinned = nullptr;    // upload image: [head block][counts][queue]
    size_t image_bytes = 0;
};

// Gauss-Seidel 2-D plan with its upload image ([head block][counts][queue]).
struct GsPlanCache {
    GsPlanHost plan;
    int32_t tile[3] = {0, 0, 0};
    void* pinned = nullptr;
    size_t image_bytes = 0, counts_bytes = 0;
};

// LU / Cholesky recursive plan with its upload image ([head block][counts][queue]).
struct LaPlanCache {
    LaPlanHost plan;
    void* pinned = nullptr;
    size_t image_bytes = 0, counts_bytes = 0;
};

// FDTD-2D recursive plan: queue and counters of the (block, tile) lattice.
struct FdPlanCache {
    int32_t lattice[4] = {0, 1, 1, 1};
    std::vector<int32_t> queue, counts;
    void* pinned = nullptr;
    size_t image_bytes = 0, counts_bytes = 0;
};

}  // namespace

struct pcot_plan {
    int dims = 0, radius = 1;
    int boundary = 0;
    double coeffs[7] = {0, 0, 0, 0, 0, 0, 0};
    int device = 0;
    int num_sms = 0;
    DevStatus* d_status = nullptr;
    double* d_partials = nullptr;  // grid-sum partials
    std::map<std::string, CotPlanHost*> cot_cache;
    std::map<std::string, GsPlanCache*> gs_cache;
    std::map<std::string, GsPlanCache*> skew_cache;
    std::map<std::string, FdPlanCache*> fd_cache;
    std::map<std::string, LaPlanCache*> la_cache;
    uint64_t timeout_ns = kDefaultTimeoutNs;
    int64_t launches = 0;  // kernels launched by this handle
    // Learned tile picker: MLP parameters followed by the feature mean and
    // standard deviation (empty: no model, picks fall back to the autotuner),
    // their device copy, scratch for the candidates' features and
    // predictions, and the picks already made per problem.
    std::vector<float> picker;
    float* d_picker = nullptr;
    void* d_pick = nullptr;
    size_t pick_bytes = 0;
    std::map<std::string, std::pair<pcot_schedule, pcot_tile_params>> pick_cache;
};

namespace {

pcot_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return PCOT_OK;
    if (e == cudaErrorMemoryAllocation) return PCOT_ERR_OOM;
    return PCOT_ERR_CUDA;
}

#define PCOT_TRY(expr)                         \
    do {                                       \
        pcot_status _s = (expr);               \
        if (_s != PCOT_OK) return _s;          \
    } while (0)

#define PCOT_CUDA(expr)                        \
    do {                                       \
        cudaError_t _e = (expr);               \
        if (_e != cudaSuccess) return from_cuda(_e); \
    } while (0)

int elem_size(pcot_dtype dt) { return dt == PCOT_F32 ? 4 : 8; }

// Device resources of a handle, created on first use on the current device.
pcot_status ensure_device(pcot_handle h) {
    if (h->d_status) return PCOT_OK;
    PCOT_CUDA(cudaGetDevice(&h->device));
    PCOT_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    DevStatus* st = nullptr;
    double* part = nullptr;
    cudaError_t e = cudaMalloc((void**)&st, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemset(st, 0, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMalloc((void**)&part, sizeof(double) * grid_sum_partials());
    if (e != cudaSuccess) {
        if (st) cudaFree(st);
        if (part) cudaFree(part);
        return from_cuda(e);
    }
    h->d_status = st;
    h->d_partials = part;
    return PCOT_OK;
}

// Pinned upload image of a plan, built on first use.
pcot_status ensure_image(CotPlanHost* c) {
    if (c->pinned || c->ntiles == 0) return PCOT_OK;
    void* p = nullptr;
    PCOT_CUDA(cudaMallocHost(&p, c->image_bytes));
    unsigned char* img = (unsigned char*)p;
    const size_t cb = (size_t)c->ntiles * 4;
    std::memset(img, 0, c->image_bytes);
    std::memcpy(img + kAlign, c->counts.data(), cb);
    std::memcpy(img + kAlign + round_up(cb, kAlign), c->queue.data(), cb);
    c->pinned = p;
    return PCOT_OK;
}

pcot_status make_ctx(pcot_handle h, const int64_t* sizes, const int64_t* strides, pcot_dtype dtype,
                     void* stream, LaunchCtx* L) {
    if (!h || !sizes) return PCOT_ERR_INVALID_ARG;
    if (dtype != PCOT_F32 && dtype != PCOT_F64 && dtype != PCOT_F64_EXACT) return PCOT_ERR_INVALID_ARG;
    std::memset(L, 0, sizeof(*L));
    L->dtype = (int)dtype;
    L->stream = (cudaStream_t)stream;
    DevGeo& g = L->geo;
    g.dims = h->dims;
    g.periodic = h->boundary == PCOT_PERIODIC;
    for (int a = 0; a < kMaxDims; ++a) {
        g.e[a] = 1;
        g.n[a] = 1;
        g.s[a] = 0;
    }
    for (int a = 0; a < h->dims; ++a) {
        if (sizes[a] < 1 || sizes[a] > (int64_t)1 << 40) return PCOT_ERR_INVALID_ARG;
        if (g.periodic && sizes[a] < 3) return PCOT_ERR_UNSUPPORTED;
        g.n[a] = sizes[a];
        g.e[a] = g.periodic ? sizes[a] : sizes[a] + 2 * h->radius;
    }
    int64_t s = 1;
    for (int a = h->dims - 1; a >= 0; --a) {
        if (strides) {
            if (a == h->dims - 1 && strides[a] != 1) return PCOT_ERR_UNSUPPORTED;
            if (strides[a] < s) return PCOT_ERR_INVALID_ARG;  // rows may not overlap
            g.s[a] = strides[a];
        } else {
            g.s[a] = s;
        }
        s = g.s[a] * g.e[a];
    }
    for (int i = 0; i < 7; ++i) L->coeffs[i] = h->coeffs[i];
    return PCOT_OK;
}

size_t span_bytes(const LaunchCtx& L) {
    int64_t last = 0;
    for (int a = 0; a < L.geo.dims; ++a) last += (L.geo.e[a] - 1) * L.geo.s[a];
    return (size_t)(last + 1) * dtype_size(L.dtype);
}

std::string plan_key(const LaunchCtx& L, int64_t T, const pcot_tile_params* p) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%d|%d|%lld,%lld,%lld|%lld|%d,%d,%d|%d|%d,%d,%d,%d", L.dtype, L.geo.dims,
                  (long long)L.geo.n[0], (long long)L.geo.n[1], (long long)L.geo.n[2], (long long)T,
                  p ? p->tile[0] : 0, p ? p->tile[1] : 0, p ? p->tile[2] : 0, p ? p->time_depth : 0,
                  p ? p->cot_threshold[0] : 0, p ? p->cot_threshold[1] : 0, p ? p->cot_threshold[2] : 0,
                  p ? p->cot_threshold[3] : 0);
    return buf;
}

std::vector<int> family_depths(int family, int dtype) {
    int d[32];
    const int n = supported_depths(family, dtype, d, 32);
    return std::vector<int>(d, d + n);
}

// Build (or fetch) the persistent-executor plan of a problem.
pcot_status get_cot_plan(pcot_handle h, const LaunchCtx& L, int64_t T, const pcot_tile_params* p,
                         CotPlanHost** out) {
    const std::string key = plan_key(L, T, p);
    auto it = h->cot_cache.find(key);
    if (it != h->cot_cache.end()) {
        *out = it->second;
        return PCOT_OK;
    }
    if (L.geo.periodic) return PCOT_ERR_UNSUPPORTED;  // the skewed lattice needs a non-wrapping domain
    int k = p && p->time_depth > 0 ? p->time_depth : default_depth(L);
    TileGeo tg;
    if (!choose_tiles(L, p ? p->tile : nullptr, k, &tg)) {
        // Depth not compiled for the fast family: fall back to its nearest.
        std::vector<int> ds = family_depths(L.geo.dims == 2 ? kFamStream2D : kFamStream3D, L.dtype);
        int best = 1;
        for (int d : ds)
            if (d <= k) best = d;
        k = best;
        if (!choose_tiles(L, p ? p->tile : nullptr, k, &tg)) return PCOT_ERR_UNSUPPORTED;
    }
    CotPlanHost* c = new CotPlanHost();
    c->tg = tg;
    c->k = k;
    int64_t P = T / k;
    if (P % 2 == 1) P -= 1;
    if (P > (int64_t)1 << 20) {
        delete c;
        return PCOT_ERR_UNSUPPORTED;
    }
    c->P = (int)P;
    const int d = L.geo.dims;
    int64_t Lax[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) Lax[a] = tg.count[a];
    int64_t total = P * Lax[0] * Lax[1] * Lax[2];
    if (total > 0x7fffffffLL) {
        delete c;
        return PCOT_ERR_UNSUPPORTED;
    }
    c->lattice[0] = (int32_t)P;
    for (int a = 0; a < 3; ++a) c->lattice[1 + a] = (int32_t)Lax[a];
    c->ntiles = total;
    int64_t theta[4] = {1, 1, 1, 1};
    for (int i = 0; i <= d; ++i) theta[i] = p && p->cot_threshold[i] > 0 ? p->cot_threshold[i] : 1;
    if (P > 0) {
        c->queue = pcot_lattice_order((int)P, d, Lax, theta, nullptr);
        c->counts = lattice_dep_counts((int)P, d, Lax);
        if ((int64_t)c->queue.size() != total) {
            delete c;
            return PCOT_ERR_UNSUPPORTED;
        }
    }
    // Remaining steps: single-level blocks with an even count.
    const int64_t rest = T - P * k;
    std::vector<int> ds = tg.family == kFamGeneric ? std::vector<int>() : family_depths(tg.family, L.dtype);
    c->tail = plan_blocks(rest, k, ds);
    c->image_bytes = kAlign + round_up((size_t)total * 4, kAlign) + round_up((size_t)total * 4, kAlign);
    h->cot_cache[key] = c;
    *out = c;
    return PCOT_OK;
}

size_t twin_bytes(const LaunchCtx& L) { return round_up(span_bytes(L), kAlign); }

pcot_status run_blocks(pcot_handle h, const LaunchCtx& L, const pcot_tile_params* p, const BlockPlan& bp, void*& cur,
                       void*& other) {
    for (int d : bp.depths) {
        TileGeo tg;
        if (!choose_tiles(L, p ? p->tile : nullptr, d, &tg)) return PCOT_ERR_UNSUPPORTED;
        PCOT_CUDA(launch_slt_block(L, tg, cur, other, h->d_status));
        ++h->launches;
        std::swap(cur, other);
    }
    if (bp.final_copy) {
        PCOT_CUDA(launch_grid_copy(L, cur, other));
        std::swap(cur, other);
    }
    return PCOT_OK;
}

// The candidates the picker chooses among and its choice for a problem
// ---- PCOT_SKEW: parallelogram tiles of the skewed space (t, t+i, t+j) ----

// Tile shape {time steps, skewed rows, skewed columns}, threads per CTA and
// order of a PCOT_SKEW run: the recursive order when cot_threshold[0] is set
// (missing entries 32), else the wavefront order.
bool skew_shape(const pcot_tile_params* p, int32_t* tile, int* recursive, int32_t* theta, int* threads = nullptr) {
    tile[0] = (p && p->time_depth > 0) ? p->time_depth : 4;
    tile[1] = (p && p->tile[0] > 0) ? p->tile[0] : 32;
    tile[2] = (p && p->tile[1] > 0) ? p->tile[1] : 64;
    const int thr = (p && p->tile[2] > 0) ? p->tile[2] : 256;
    if (threads) *threads = thr;
    *recursive = (p && p->cot_threshold[0] > 0) ? 1 : 0;
    for (int d = 0; d < 3; ++d) theta[d] = (p && p->cot_threshold[d] > 0) ? p->cot_threshold[d] : 32;
    return tile[0] <= 256 && tile[1] >= 2 && tile[1] <= 1024 && tile[2] >= 2 && tile[2] <= 1024 && thr >= 32 &&
           thr <= 512 && thr % 32 == 0;
}

// Upload-image bytes that suffice for any plan of this shape: head block,
// the counter of every lattice id, and a queue of at most every id.
pcot_status skew_image_bound(int64_t n0, int64_t n1, int64_t T, const int32_t* tile, size_t* bytes) {
    const int64_t ext[3] = {T, T - 1 + n0, T - 1 + n1};
    int64_t cells = 1;
    for (int d = 0; d < 3; ++d) {
        cells *= (ext[d] + tile[d] - 1) / tile[d];
        if (cells > (int64_t)1 << 28) return PCOT_ERR_UNSUPPORTED;
    }
    *bytes = kAlign + round_up((size_t)cells * 4, kAlign) + round_up((size_t)cells * 4 + 4, kAlign);
    return PCOT_OK;
}

pcot_status skew_get_plan(pcot_handle h, int64_t n0, int64_t n1, int64_t T, const int32_t* tile, int recursive,
                          const int32_t* theta, GsPlanCache** out) {
    char key[160];
    snprintf(key, sizeof(key), "%lld,%lld,%lld,%d,%d,%d,%d,%d,%d,%d", (long long)n0, (long long)n1, (long long)T,
             recursive, tile[0], tile[1], tile[2], theta[0], theta[1], theta[2]);
    if (h) {
        auto it = h->skew_cache.find(key);
        if (it != h->skew_cache.end()) {
            *out = it->second;
            return PCOT_OK;
        }
    }
    GsPlanCache* c = new GsPlanCache();
    if (!skew_plan(n0, n1, T, tile, recursive, theta, &c->plan)) {
        delete c;
        return PCOT_ERR_UNSUPPORTED;
    }
    for (int d = 0; d < 3; ++d) c->tile[d] = tile[d];
    c->counts_bytes = round_up(c->plan.deps.size() * 4, kAlign);
    c->image_bytes = kAlign + c->counts_bytes + round_up(c->plan.queue.size() * 4 + 4, kAlign);
    if (h) {
        if (h->skew_cache.size() >= 16) {
            for (auto& kv : h->skew_cache) {
                if (kv.second->pinned) cudaFreeHost(kv.second->pinned);
                delete kv.second;
            }
            h->skew_cache.clear();
        }
        h->skew_cache[key] = c;
    }
    *out = c;
    return PCOT_OK;
}

// Even time levels live in the grid, odd ones in the twin; one persistent
// launch runs every tile, and an odd T ends with a copy of the twin back.
pcot_status run_skew(pcot_handle h, const LaunchCtx& L, void* grid, void* workspace, size_t ws_bytes, int64_t T,
                     const pcot_tile_params* params) {
    if (L.geo.dims != 2 || L.geo.periodic) return PCOT_ERR_UNSUPPORTED;
    int32_t tl[3], th[3];
    int rec = 0, threads = 0;
    if (!skew_shape(params, tl, &rec, th, &threads)) return PCOT_ERR_INVALID_ARG;
    const int64_t n0 = L.geo.n[0], n1 = L.geo.n[1];
    size_t extra = 0;
    PCOT_TRY(skew_image_bound(n0, n1, T, tl, &extra));
    if (ws_bytes < twin_bytes(L) + extra) return PCOT_ERR_OOM;
    SkewDev q;
    std::memset(&q, 0, sizeof(q));
    for (int d = 0; d < 3; ++d) q.tile[d] = tl[d];
    skew2d_window(&q);
    if (skew2d_smem_bytes(L.dtype, q) > 227 * 1024) return PCOT_ERR_UNSUPPORTED;
    PCOT_TRY(ensure_device(h));
    GsPlanCache* c = nullptr;
    PCOT_TRY(skew_get_plan(h, n0, n1, T, tl, rec, th, &c));
    if (!c->pinned) {
        void* p = nullptr;
        PCOT_CUDA(cudaMallocHost(&p, c->image_bytes));
        unsigned char* img = (unsigned char*)p;
        std::memset(img, 0, c->image_bytes);
        std::memcpy(img + kAlign, c->plan.deps.data(), c->plan.deps.size() * 4);
        std::memcpy(img + kAlign + c->counts_bytes, c->plan.queue.data(), c->plan.queue.size() * 4);
        c->pinned = p;
    }
    void* twin = workspace;
    PCOT_CUDA(launch_ring_copy(L, grid, twin));
    ++h->launches;
    if (c->plan.queue.empty()) return PCOT_OK;
    unsigned char* ws = (unsigned char*)workspace + twin_bytes(L);
    PCOT_CUDA(cudaMemcpyAsync(ws, c->pinned, c->image_bytes, cudaMemcpyHostToDevice, L.stream));
    q.head = (int32_t*)ws;
    q.counts = (int32_t*)(ws + kAlign);
    q.queue = (const int32_t*)(ws + kAlign + c->counts_bytes);
    q.ntiles = (int64_t)c->plan.queue.size();
    for (int d = 0; d < 3; ++d) q.lattice[d] = c->plan.lattice[d];
    q.n0 = n0;
    q.n1 = n1;
    q.T = T;
    q.pitch = L.geo.s[0];
    q.status = h->d_status;
    q.timeout_ns = h->timeout_ns;
    const int per_sm = skew2d_ctas_per_sm(L.dtype, q, threads);
    if (per_sm < 1) return PCOT_ERR_UNSUPPORTED;
    int64_t nctas = (int64_t)per_sm * h->num_sms;
    if (nctas > q.ntiles) nctas = q.ntiles;
    PCOT_CUDA(launch_skew2d(L, grid, twin, q, (int)nctas, threads));
    ++h->launches;
    if (T & 1) {
        PCOT_CUDA(launch_grid_copy(L, twin, grid));
        ++h->launches;
    }
    return PCOT_OK;
}

// (PCOT_AUTO, pcot_pick); defined with the picker below.
std::vector<std::pair<pcot_schedule, pcot_tile_params>> pick_candidates(int dims, pcot_dtype dtype, bool periodic);
pcot_status pick_impl(pcot_handle h, const int64_t* sizes, int64_t T, pcot_dtype dtype, cudaStream_t s,
                      pcot_schedule* schedule, pcot_tile_params* params);

pcot_status run_impl(pcot_handle h, void* grid, void* workspace, size_t ws_bytes, const int64_t* sizes,
                     const int64_t* strides, int64_t T, pcot_dtype dtype, pcot_schedule schedule,
                     const pcot_tile_params* params, void* stream) {
    if (!h || !grid || !workspace || !sizes) return PCOT_ERR_INVALID_ARG;
    if (T < 0) return PCOT_ERR_INVALID_ARG;
    LaunchCtx L;
    PCOT_TRY(make_ctx(h, sizes, strides, dtype, stream, &L));
    if (((uintptr_t)grid % elem_size(dtype)) != 0) return PCOT_ERR_ALIGNMENT;
    if (((uintptr_t)workspace % kAlign) != 0) return PCOT_ERR_ALIGNMENT;
    if (schedule < PCOT_SWEEP || schedule > PCOT_SKEW) return PCOT_ERR_INVALID_ARG;
    if (schedule == PCOT_SKEW && (L.geo.dims != 2 || L.geo.periodic)) return PCOT_ERR_UNSUPPORTED;
    if (T == 0) return PCOT_OK;
    pcot_tile_params picked;
    if (schedule == PCOT_AUTO) {
        PCOT_TRY(pick_impl(h, sizes, T, dtype, (cudaStream_t)stream, &schedule, &picked));
        params = &picked;
    }
    if (schedule == PCOT_SKEW) return run_skew(h, L, grid, workspace, ws_bytes, T, params);
    if (schedule == PCOT_COT && L.geo.periodic) return PCOT_ERR_UNSUPPORTED;
    if (ws_bytes < twin_bytes(L)) return PCOT_ERR_OOM;
    CotPlanHost* cplan = nullptr;
    if (schedule == PCOT_COT) {
        PCOT_TRY(get_cot_plan(h, L, T, params, &cplan));
        if (ws_bytes < twin_bytes(L) + (cplan->ntiles > 0 ? cplan->image_bytes : 0)) return PCOT_ERR_OOM;
    }
    PCOT_TRY(ensure_device(h));
    void* twin = workspace;
    if (!L.geo.periodic) {
        PCOT_CUDA(launch_ring_copy(L, grid, twin));
        ++h->launches;
    }
    void* cur = grid;
    void* other = twin;
    if (schedule == PCOT_SWEEP) {
        for (int64_t t = 0; t < T; ++t) {
            PCOT_CUDA(launch_sweep(L, cur, other));
            ++h->launches;
            std::swap(cur, other);
        }
        if (cur != grid) PCOT_CUDA(launch_grid_copy(L, cur, grid));
        return PCOT_OK;
    }
    if (schedule == PCOT_SLT) {
        int k = params && params->time_depth > 0 ? params->time_depth : default_depth(L);
        TileGeo probe;
        std::vector<int> ds;
        if (choose_tiles(L, params ? params->tile : nullptr, k, &probe)) {
            ds = probe.family == kFamGeneric ? std::vector<int>() : family_depths(probe.family, L.dtype);
        } else {
            const int fam = L.geo.dims == 2 ? kFamStream2D : kFamStream3D;
            ds = family_depths(fam, L.dtype);
        }
        BlockPlan bp = plan_blocks(T, k, ds);
        PCOT_TRY(run_blocks(h, L, params, bp, cur, other));
        if (cur != grid) return PCOT_ERR_UNSUPPORTED;  // plan_blocks guarantees an even swap count
        return PCOT_OK;
    }
    // PCOT_COT
    CotPlanHost* c = cplan;
    if (c->ntiles > 0) {
        PCOT_TRY(ensure_image(c));
        unsigned char* ws = (unsigned char*)workspace + twin_bytes(L);
        PCOT_CUDA(cudaMemcpyAsync(ws, c->pinned, c->image_bytes, cudaMemcpyHostToDevice, L.stream));
        CotDev q;
        q.head = (int32_t*)ws;
        q.counts = (int32_t*)(ws + kAlign);
        q.queue = (const int32_t*)(ws + kAlign + round_up((size_t)c->ntiles * 4, kAlign));
        q.ntiles = c->ntiles;
        for (int i = 0; i < 4; ++i) q.lattice[i] = c->lattice[i];
        q.status = h->d_status;
        q.timeout_ns = h->timeout_ns;
        int per_sm = cot_ctas_per_sm(L, c->tg);
        int64_t nctas = (int64_t)per_sm * h->num_sms;
        // A tile of block b+1 depends on tiles about one block's worth of
        // queue entries earlier; with more CTAs in flight than ~2/5 of a
        // block, popped tiles find their predecessors still running and wait.
        // Measured on Heat-2D 4096^2..8192^2: 2.5 tiles of a block per CTA is
        // neutral on the large grid and 9-18% faster on the smaller ones.
        const int64_t per_block = (int64_t)c->lattice[1] * c->lattice[2] * c->lattice[3];
        const int64_t cap = std::max<int64_t>(h->num_sms, per_block * 2 / 5);
        if (nctas > cap) nctas = cap;
        if (nctas > c->ntiles) nctas = c->ntiles;
        if (nctas < 1) nctas = 1;
        PCOT_CUDA(launch_cot(L, c->tg, grid, twin, q, (int)nctas));
        ++h->launches;
        // c->P is even: the result of the persistent part is back in grid.
    }
    PCOT_TRY(run_blocks(h, L, params, c->tail, cur, other));
    if (cur != grid) return PCOT_ERR_UNSUPPORTED;
    return PCOT_OK;
}

}  // namespace

extern "C" {

const char* pcot_status_string(pcot_status s) {
    switch (s) {
        case PCOT_OK: return "ok";
        case PCOT_ERR_INVALID_ARG: return "invalid argument";
        case PCOT_ERR_UNSUPPORTED: return "unsupported";
        case PCOT_ERR_ALIGNMENT: return "misaligned pointer or stride";
        case PCOT_ERR_CUDA: return "CUDA error";
        case PCOT_ERR_OOM: return "out of memory";
        case PCOT_ERR_TIMEOUT: return "device dependency wait timed out";
        case PCOT_ERR_BOUNDS: return "device index check failed";
    }
    return "unknown status";
}

pcot_status pcot_create(int dims, int radius, const double* coeffs, int ncoeffs, pcot_boundary boundary,
                        pcot_handle* out) {
    if (!out || !coeffs) return PCOT_ERR_INVALID_ARG;
    *out = nullptr;
    if (dims < 1 || dims > 3) return PCOT_ERR_UNSUPPORTED;
    if (radius != 1) return PCOT_ERR_UNSUPPORTED;
    if (ncoeffs != 1 + 2 * dims * radius) return PCOT_ERR_INVALID_ARG;
    if (boundary != PCOT_DIRICHLET && boundary != PCOT_PERIODIC) return PCOT_ERR_INVALID_ARG;
    pcot_plan* h = new pcot_plan();
    h->dims = dims;
    h->radius = radius;
    h->boundary = boundary;
    for (int i = 0; i < ncoeffs; ++i) h->coeffs[i] = coeffs[i];
    if (kPickerModelFloats > 0) h->picker.assign(kPickerModel, kPickerModel + kPickerModelFloats);
    *out = h;
    return PCOT_OK;
}

pcot_status pcot_destroy(pcot_handle h) {
    if (!h) return PCOT_ERR_INVALID_ARG;
    for (auto& kv : h->cot_cache) {
        if (kv.second->pinned) cudaFreeHost(kv.second->pinned);
        delete kv.second;
    }
    for (auto& kv : h->gs_cache) {
        if (kv.second->pinned) cudaFreeHost(kv.second->pinned);
        delete kv.second;
    }
    for (auto& kv : h->skew_cache) {
        if (kv.second->pinned) cudaFreeHost(kv.second->pinned);
        delete kv.second;
    }
    for (auto& kv : h->fd_cache) {
        if (kv.second->pinned) cudaFreeHost(kv.second->pinned);
        delete kv.second;
    }
    for (auto& kv : h->la_cache) {
        if (kv.second->pinned) cudaFreeHost(kv.second->pinned);
        delete kv.second;
    }
    if (h->d_status) cudaFree(h->d_status);
    if (h->d_partials) cudaFree(h->d_partials);
    if (h->d_picker) cudaFree(h->d_picker);
    if (h->d_pick) cudaFree(h->d_pick);
    delete h;
    return PCOT_OK;
}

pcot_status pcot_workspace_bytes(pcot_handle h, const int64_t* sizes, const int64_t* strides, int64_t T,
                                 pcot_dtype dtype, pcot_schedule schedule, const pcot_tile_params* params,
                                 size_t* bytes) {
    if (!bytes || T < 0) return PCOT_ERR_INVALID_ARG;
    if (schedule < PCOT_SWEEP || schedule > PCOT_SKEW) return PCOT_ERR_INVALID_ARG;
    LaunchCtx L;
    PCOT_TRY(make_ctx(h, sizes, strides, dtype, nullptr, &L));
    size_t b = twin_bytes(L);
    if (schedule == PCOT_AUTO && T > 0) {
        // enough for whichever candidate the picker chooses
        for (const auto& c : pick_candidates(L.geo.dims, dtype, L.geo.periodic != 0)) {
            size_t bc = 0;
            if (pcot_workspace_bytes(h, sizes, strides, T, dtype, c.first, &c.second, &bc) == PCOT_OK)
                b = std::max(b, bc);
        }
    }
    if (schedule == PCOT_SKEW) {
        if (L.geo.dims != 2 || L.geo.periodic) return PCOT_ERR_UNSUPPORTED;
        int32_t tl[3], th[3];
        int rec = 0;
        if (!skew_shape(params, tl, &rec, th)) return PCOT_ERR_INVALID_ARG;
        if (T > 0) {
            size_t extra = 0;
            PCOT_TRY(skew_image_bound(L.geo.n[0], L.geo.n[1], T, tl, &extra));
            b += extra;
        }
    }
    if (schedule == PCOT_COT && T > 0) {
        if (L.geo.periodic) return PCOT_ERR_UNSUPPORTED;
        CotPlanHost* c = nullptr;
        PCOT_TRY(get_cot_plan(h, L, T, params, &c));
        b += c->image_bytes;
    }
    *bytes = b;
    return PCOT_OK;
}

pcot_status pcot_run(pcot_handle h, void* grid, void* workspace, size_t workspace_bytes, const int64_t* sizes,
                     const int64_t* strides, int64_t T, pcot_dtype dtype, pcot_schedule schedule,
                     const pcot_tile_params* params, void* stream) {
    return run_impl(h, grid, workspace, workspace_bytes, sizes, strides, T, dtype, schedule, params, stream);
}

pcot_status pcot_run_host(pcot_handle h, void* host_grid, void* dev_grid, void* workspace, size_t workspace_bytes,
                          const int64_t* sizes, const int64_t* strides, int64_t T, pcot_dtype dtype,
                          pcot_schedule schedule, const pcot_tile_params* params, void* stream) {
    if (!host_grid || !dev_grid) return PCOT_ERR_INVALID_ARG;
    LaunchCtx L;
    PCOT_TRY(make_ctx(h, sizes, strides, dtype, stream, &L));
    const size_t bytes = span_bytes(L);
    PCOT_CUDA(cudaMemcpyAsync(dev_grid, host_grid, bytes, cudaMemcpyHostToDevice, L.stream));
    PCOT_TRY(run_impl(h, dev_grid, workspace, workspace_bytes, sizes, strides, T, dtype, schedule, params, stream));
    PCOT_CUDA(cudaMemcpyAsync(host_grid, dev_grid, bytes, cudaMemcpyDeviceToHost, L.stream));
    return pcot_check(h, stream);
}

pcot_status pcot_check(pcot_handle h, void* stream) {
    if (!h) return PCOT_ERR_INVALID_ARG;
    PCOT_TRY(ensure_device(h));
    PCOT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    PCOT_CUDA(cudaGetLastError());
    DevStatus st;
    PCOT_CUDA(cudaMemcpy(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st.code != 0) {
        PCOT_CUDA(cudaMemset(h->d_status, 0, sizeof(DevStatus)));
        return (pcot_status)st.code;
    }
    return PCOT_OK;
}

pcot_status pcot_plan_query(pcot_handle h, const int64_t* sizes, int64_t T, pcot_dtype dtype,
                            const pcot_tile_params* params, int32_t* lattice, int32_t* tile_ext, int32_t* depth,
                            int64_t* n_tiles, int64_t* tail_steps, int32_t* queue, int32_t* deps, int64_t cap) {
    if (T < 0) return PCOT_ERR_INVALID_ARG;
    LaunchCtx L;
    PCOT_TRY(make_ctx(h, sizes, nullptr, dtype, nullptr, &L));
    CotPlanHost* c = nullptr;
    PCOT_TRY(get_cot_plan(h, L, T, params, &c));
    if (lattice)
        for (int i = 0; i < 4; ++i) lattice[i] = c->lattice[i];
    if (tile_ext)
        for (int a = 0; a < 3; ++a) tile_ext[a] = (int32_t)c->tg.ext[a];
    if (depth) *depth = c->k;
    if (n_tiles) *n_tiles = c->ntiles;
    if (tail_steps) {
        int64_t s = 0;
        for (int d : c->tail.depths) s += d;
        *tail_steps = s;
    }
    if (queue || deps) {
        if (cap < c->ntiles) return PCOT_ERR_OOM;
        for (int64_t i = 0; i < c->ntiles; ++i) {
            if (queue) queue[i] = c->queue[(size_t)i];
            if (deps) deps[i] = c->counts[(size_t)c->queue[(size_t)i]];
        }
    }
    return PCOT_OK;
}

pcot_status pcot_test_wait_timeout(pcot_handle h, void* workspace, int32_t timeout_ms, void* stream) {
    if (!h || !workspace || timeout_ms < 1) return PCOT_ERR_INVALID_ARG;
    if (((uintptr_t)workspace % 4) != 0) return PCOT_ERR_ALIGNMENT;
    PCOT_TRY(ensure_device(h));
    int32_t one = 1;
    PCOT_CUDA(cudaMemcpyAsync(workspace, &one, sizeof(one), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    PCOT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    PCOT_CUDA(launch_wait_timeout_probe((int32_t*)workspace, h->d_status, (uint64_t)timeout_ms * 1000000ull,
                                        (cudaStream_t)stream));
    return PCOT_OK;
}

pcot_status pcot_grid_sum(pcot_handle h, const void* grid, const int64_t* sizes, const int64_t* strides,
                          pcot_dtype dtype, double* out_device, void* stream) {
    if (!grid || !out_device) return PCOT_ERR_INVALID_ARG;
    LaunchCtx L;
    PCOT_TRY(make_ctx(h, sizes, strides, dtype, stream, &L));
    if (((uintptr_t)grid % elem_size(dtype)) != 0 || ((uintptr_t)out_device % 8) != 0) return PCOT_ERR_ALIGNMENT;
    PCOT_TRY(ensure_device(h));
    PCOT_CUDA(launch_grid_sum(L, grid, out_device, h->d_partials, grid_sum_partials()));
    h->launches += 2;
    return PCOT_OK;
}

pcot_status pcot_launch_count(pcot_handle h, int64_t* launches) {
    if (!h || !launches) return PCOT_ERR_INVALID_ARG;
    *launches = h->launches;
    return PCOT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched runs
// ---------------------------------------------------------------------------
#include <queue>

#include "tiled.cuh"

namespace {

struct BatchPlanHost {
    int nb = 0, dtype = 0, depth = 0, nwarps = 1;
    std::vector<LaunchCtx> ctx;
    std::vector<TileGeo> tg;
    std::vector<int32_t> Pmain, Ptotal, base, ntiles, final_copy;
    bool any_final_copy = false;
    std::vector<int2> queue;
    std::vector<int32_t> counts;  // initial values, by global counter index
    std::vector<int32_t> remaining;
    // workspace layout
    size_t off_desc = 0, off_queue = 0, off_counts = 0, off_counts0 = 0, off_rem = 0, off_rem0 = 0, off_head = 0;
    std::vector<size_t> off_twin;
    size_t total = 0;
};

pcot_status build_batch_plan(pcot_handle h, int nb, const int64_t* sizes, const int64_t* strides, const int64_t* T,
                             pcot_dtype dtype, const pcot_tile_params* params, BatchPlanHost* B) {
    if (!h || nb < 1 || nb > 65535 || !sizes || !T) return PCOT_ERR_INVALID_ARG;
    if (h->dims != 2 || h->boundary != PCOT_DIRICHLET) return PCOT_ERR_UNSUPPORTED;
    B->nb = nb;
    B->dtype = (int)dtype;
    const int kdef = dtype == PCOT_F32 ? 8 : 2;
    B->depth = params && params[0].time_depth > 0 ? params[0].time_depth : kdef;
    const int d = B->depth;
    if (!(d == 1 || d == 2 || d == 4 || ((d == 6 || d == 8) && dtype == PCOT_F32))) return PCOT_ERR_UNSUPPORTED;
    const int E = dtype == PCOT_F32 ? 4 : 2;
    const int Kp = ((d + E - 1) / E) * E;
    const int Wo = 32 * E - 2 * Kp;
    B->nwarps = params && params[0].tile[1] > 0 ? (int)std::max<int64_t>(1, (params[0].tile[1] + Wo / 2) / Wo) : 1;
    B->ctx.resize(nb);
    B->tg.resize(nb);
    B->Pmain.resize(nb);
    B->Ptotal.resize(nb);
    B->base.resize(nb);
    B->ntiles.resize(nb);
    B->final_copy.assign(nb, 0);
    std::vector<std::vector<int32_t>> qs(nb);
    int64_t total = 0;
    for (int g = 0; g < nb; ++g) {
        if (T[g] < 0) return PCOT_ERR_INVALID_ARG;
        PCOT_TRY(make_ctx(h, sizes + 2 * g, strides ? strides + 2 * g : nullptr, dtype, nullptr, &B->ctx[g]));
        const int64_t H = params && params[g].tile[0] > 0 ? params[g].tile[0] : 64;
        if (!stream2d::batch_tiles(B->ctx[g], d, B->nwarps, H, &B->tg[g])) return PCOT_ERR_UNSUPPORTED;
        int64_t Pm = T[g] / d, tail = T[g] - Pm * d;
        if ((Pm + tail) % 2 == 1) {
            if (Pm > 0 && d % 2 == 0) {
                Pm -= 1;  // one block of depth d becomes d single steps: the count turns even
                tail += d;
            } else {
                B->final_copy[g] = 1;  // the result ends in the twin and is copied back at the end
                B->any_final_copy = true;
            }
        }
        if (Pm + tail > (1 << 20)) return PCOT_ERR_UNSUPPORTED;
        B->Pmain[g] = (int32_t)Pm;
        B->Ptotal[g] = (int32_t)(Pm + tail);
        const int64_t Lax[3] = {B->tg[g].count[0], B->tg[g].count[1], 1};
        const int64_t n = (int64_t)B->Ptotal[g] * Lax[0] * Lax[1];
        if (total + n > 0x7fffffffLL) return PCOT_ERR_UNSUPPORTED;
        B->base[g] = (int32_t)total;
        B->ntiles[g] = (int32_t)n;
        total += n;
        if (n > 0) {
            int64_t theta[4] = {2, 8, 8, 1};
            if (params)
                for (int i = 0; i < 3; ++i)
                    if (params[g].cot_threshold[i] > 0) theta[i] = params[g].cot_threshold[i];
            qs[g] = pcot_lattice_order(B->Ptotal[g], 2, Lax, theta, nullptr);
            std::vector<int32_t> c = lattice_dep_counts(B->Ptotal[g], 2, Lax);
            B->counts.insert(B->counts.end(), c.begin(), c.end());
        }
    }
    // Merge: the grid whose next tile sits earliest in its own queue
    // (relative position) goes next; ties go to the grid with more tiles.
    struct Key {
        double frac;
        int32_t len;
        int g;
        bool operator<(const Key& o) const {
            if (frac != o.frac) return frac > o.frac;
            if (len != o.len) return len < o.len;
            return g > o.g;
        }
    };
    std::priority_queue<Key> pq;
    std::vector<size_t> pos(nb, 0);
    for (int g = 0; g < nb; ++g)
        if (!qs[g].empty()) pq.push({1.0 / (double)qs[g].size(), (int32_t)qs[g].size(), g});
    B->queue.reserve((size_t)total);
    while (!pq.empty()) {
        Key k = pq.top();
        pq.pop();
        const int g = k.g;
        B->queue.push_back(make_int2(g, qs[g][pos[g]]));
        if (++pos[g] < qs[g].size())
            pq.push({(double)(pos[g] + 1) / (double)qs[g].size(), (int32_t)qs[g].size(), g});
    }
    B->remaining.assign(B->ntiles.begin(), B->ntiles.end());
    // Workspace layout.
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = round_up(o + bytes, kAlign);
        return at;
    };
    B->off_desc = take(sizeof(BatchDesc) * (size_t)nb);
    B->off_queue = take(sizeof(int2) * (size_t)std::max<int64_t>(total, 1));
    B->off_counts = take(sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1));
    B->off_counts0 = take(sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1));
    B->off_rem = take(sizeof(int32_t) * (size_t)nb);
    B->off_rem0 = take(sizeof(int32_t) * (size_t)nb);
    B->off_head = take(sizeof(int32_t));
    B->off_twin.resize(nb);
    for (int g = 0; g < nb; ++g) B->off_twin[g] = take(span_bytes(B->ctx[g]));
    B->total = o;
    return PCOT_OK;
}

}  // namespace

struct pcot_batch_s {
    pcot_handle h = nullptr;
    BatchPlanHost plan;
    BatchDev dev{};
    int nctas = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

pcot_status pcot_batch_workspace_bytes(pcot_handle h, int nb, const int64_t* sizes, const int64_t* strides,
                                       const int64_t* T, pcot_dtype dtype, const pcot_tile_params* params,
                                       size_t* bytes) {
    if (!bytes) return PCOT_ERR_INVALID_ARG;
    BatchPlanHost B;
    PCOT_TRY(build_batch_plan(h, nb, sizes, strides, T, dtype, params, &B));
    *bytes = B.total;
    return PCOT_OK;
}

pcot_status pcot_batch_create(pcot_handle h, int nb, void* const* grids, const int64_t* sizes, const int64_t* strides,
                              const int64_t* T, pcot_dtype dtype, const pcot_tile_params* params, void* workspace,
                              size_t workspace_bytes, uint64_t* done_ns, void* stream, pcot_batch* out) {
    if (!out || !grids || !workspace) return PCOT_ERR_INVALID_ARG;
    *out = nullptr;
    if (((uintptr_t)workspace % kAlign) != 0) return PCOT_ERR_ALIGNMENT;
    pcot_batch_s* b = new pcot_batch_s();
    b->h = h;
    pcot_status st = build_batch_plan(h, nb, sizes, strides, T, dtype, params, &b->plan);
    if (st == PCOT_OK && workspace_bytes < b->plan.total) st = PCOT_ERR_OOM;
    if (st == PCOT_OK) st = ensure_device(h);
    if (st != PCOT_OK) {
        delete b;
        return st;
    }
    BatchPlanHost& P = b->plan;
    unsigned char* ws = (unsigned char*)workspace;
    std::vector<BatchDesc> desc((size_t)nb);
    BatchDev& q = b->dev;
    q.nbox = 1;
    q.BW = 32;
    q.box_elems = 128;
    q.slot_elems = 128;
    q.all_tma = 1;
    for (int g = 0; g < nb; ++g) {
        BatchDesc& d = desc[g];
        std::memset(&d, 0, sizeof(d));
        if (!grids[g] || ((uintptr_t)grids[g] % elem_size(dtype)) != 0) {
            delete b;
            return grids[g] ? PCOT_ERR_ALIGNMENT : PCOT_ERR_INVALID_ARG;
        }
        d.buf[0] = grids[g];
        d.buf[1] = ws + P.off_twin[g];
        d.g = P.ctx[g].geo;
        d.H = P.tg[g].ext[0];
        d.Wt = P.tg[g].ext[1];
        d.L0 = (int32_t)P.tg[g].count[0];
        d.L1 = (int32_t)P.tg[g].count[1];
        d.Pmain = P.Pmain[g];
        d.Ptotal = P.Ptotal[g];
        d.count_base = P.base[g];
        d.ntiles = P.ntiles[g];
        d.final_copy = P.final_copy[g];
        d.span = (int64_t)(span_bytes(P.ctx[g]) / elem_size(dtype));
        const int es = elem_size(dtype);
        d.vec_ok = (((uintptr_t)d.buf[0] & 15) == 0 && ((uintptr_t)d.buf[1] & 15) == 0 &&
                    ((d.g.s[0] * es) & 15) == 0)
                       ? 1
                       : 0;
        BatchDev ring{};
        if (stream2d::batch_desc_tma(P.ctx[g], P.tg[g], &d, &ring)) {
            q.nbox = ring.nbox;
            q.BW = ring.BW;
            q.box_elems = ring.box_elems;
            q.slot_elems = ring.slot_elems;
        } else {
            q.all_tma = 0;
        }
    }
    const int64_t total = (int64_t)P.queue.size();
    q.desc = (const BatchDesc*)(ws + P.off_desc);
    q.queue = (const int2*)(ws + P.off_queue);
    q.counts = (int32_t*)(ws + P.off_counts);
    q.remaining = (int32_t*)(ws + P.off_rem);
    q.head = (int32_t*)(ws + P.off_head);
    q.ntiles = total;
    q.done_ns = done_ns;
    q.status = h->d_status;
    q.timeout_ns = h->timeout_ns;
    q.nb = nb;
    // One-time upload of descriptors, queue and initial counters.
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ws + P.off_desc, desc.data(), sizeof(BatchDesc) * desc.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && total > 0)
        e = cudaMemcpyAsync(ws + P.off_queue, P.queue.data(), sizeof(int2) * (size_t)total, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && total > 0)
        e = cudaMemcpyAsync(ws + P.off_counts0, P.counts.data(), sizeof(int32_t) * (size_t)total,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + P.off_rem0, P.remaining.data(), sizeof(int32_t) * (size_t)nb, cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int per_sm = stream2d::batch_ctas_per_sm(P.dtype, P.depth, P.nwarps, q);
    int64_t nctas = (int64_t)per_sm * h->num_sms;
    if (nctas > total) nctas = total;
    b->nctas = (int)std::max<int64_t>(1, nctas);
    // Capture: counter reset, ring copy, persistent kernel.
    cudaStream_t cs = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t ce = cudaSuccess;
        if (total > 0)
            ce = cudaMemcpyAsync(ws + P.off_counts, ws + P.off_counts0, sizeof(int32_t) * (size_t)total,
                                 cudaMemcpyDeviceToDevice, cs);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(ws + P.off_rem, ws + P.off_rem0, sizeof(int32_t) * (size_t)nb,
                                 cudaMemcpyDeviceToDevice, cs);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(ws + P.off_head, 0, sizeof(int32_t), cs);
        if (ce == cudaSuccess) ce = stream2d::batch_ring_copy(P.dtype, q, cs);
        if (ce == cudaSuccess && total > 0)
            ce = stream2d::batch_launch(P.dtype, P.depth, P.nwarps, h->coeffs, q, b->nctas, cs);
        if (ce == cudaSuccess && P.any_final_copy) ce = stream2d::batch_final_copy(P.dtype, q, cs);
        e = cudaStreamEndCapture(cs, &b->graph);
        if (e == cudaSuccess) e = ce;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return from_cuda(e);
    }
    *out = b;
    return PCOT_OK;
}

pcot_status pcot_batch_launch(pcot_batch b, void* stream) {
    if (!b) return PCOT_ERR_INVALID_ARG;
    PCOT_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    b->h->launches += 1 + (b->dev.ntiles > 0 ? 1 : 0) + (b->plan.any_final_copy ? 1 : 0);
    return PCOT_OK;
}

pcot_status pcot_batch_destroy(pcot_batch b) {
    if (!b) return PCOT_ERR_INVALID_ARG;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
    return PCOT_OK;
}

pcot_status pcot_run_batched(pcot_handle h, int nb, void* const* grids, const int64_t* sizes, const int64_t* strides,
                             const int64_t* T, pcot_dtype dtype, const pcot_tile_params* params, void* workspace,
                             size_t workspace_bytes, uint64_t* done_ns, void* stream) {
    pcot_batch b = nullptr;
    PCOT_TRY(pcot_batch_create(h, nb, grids, sizes, strides, T, dtype, params, workspace, workspace_bytes, done_ns,
                               stream, &b));
    pcot_status st = pcot_batch_launch(b, stream);
    const pcot_status ck = pcot_check(h, stream);
    pcot_batch_destroy(b);
    return st != PCOT_OK ? st : ck;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------
extern "C" pcot_status pcot_autotune(pcot_handle h, void* grid, void* workspace, size_t workspace_bytes,
                                     const int64_t* sizes, const int64_t* strides, int64_t T, pcot_dtype dtype,
                                     int ncand, const pcot_schedule* schedules, const pcot_tile_params* params,
                                     int reps, float* ms_out, void* stream) {
    if (!h || !grid || !workspace || !sizes || ncand < 1 || !schedules || !ms_out || reps < 1) return PCOT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PCOT_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return from_cuda(ce);
    }
    pcot_status result = PCOT_OK;
    for (int i = 0; i < ncand; ++i) {
        ms_out[i] = -1.0f;
        const pcot_tile_params* p = params ? &params[i] : nullptr;
        pcot_status st = pcot_run(h, grid, workspace, workspace_bytes, sizes, strides, T, dtype, schedules[i], p,
                                  stream);
        if (st == PCOT_ERR_UNSUPPORTED || st == PCOT_ERR_OOM) continue;
        if (st != PCOT_OK) {
            result = st;
            break;
        }
        ce = cudaEventRecord(e0, s);
        for (int r = 0; r < reps && ce == cudaSuccess && st == PCOT_OK; ++r)
            st = pcot_run(h, grid, workspace, workspace_bytes, sizes, strides, T, dtype, schedules[i], p, stream);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess || st != PCOT_OK) {
            result = ce != cudaSuccess ? from_cuda(ce) : st;
            break;
        }
        const pcot_status ck = pcot_check(h, stream);
        if (ck != PCOT_OK) {
            result = ck;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_out[i] = ms / (float)reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return result;
}

// ---------------------------------------------------------------------------
// Learned tile picker
// ---------------------------------------------------------------------------
namespace {

float log2f_safe(double v) { return v > 0 ? (float)std::log2(v) : 0.f; }

pcot_status features_impl(pcot_handle h, const int64_t* sizes, int64_t T, pcot_dtype dtype, pcot_schedule schedule,
                          const pcot_tile_params* p, float* f) {
    // the picker's candidates are sweep, single-level and recursive tiles
    if (schedule != PCOT_SWEEP && schedule != PCOT_SLT && schedule != PCOT_COT)
        return schedule == PCOT_AUTO || schedule == PCOT_SKEW ? PCOT_ERR_UNSUPPORTED : PCOT_ERR_INVALID_ARG;
    LaunchCtx L;
    PCOT_TRY(make_ctx(h, sizes, nullptr, dtype, nullptr, &L));
    for (int i = 0; i < 12; ++i) f[i] = 0.f;
    f[0] = (float)L.geo.dims;
    for (int a = 0; a < L.geo.dims; ++a) f[2 + a] = log2f_safe((double)L.geo.n[a]);
    f[5] = log2f_safe((double)std::max<int64_t>(T, 1));
    f[11] = (float)dtype;
    if (schedule == PCOT_SWEEP) {
        for (int a = 0; a < L.geo.dims; ++a) f[6 + a] = log2f_safe((double)L.geo.e[a]);
        f[9] = 0.f;
        f[10] = -1.f;
        return PCOT_OK;
    }
    int k = p && p->time_depth > 0 ? p->time_depth : default_depth(L);
    TileGeo tg;
    if (!choose_tiles(L, p ? p->tile : nullptr, k, &tg)) return PCOT_ERR_UNSUPPORTED;
    for (int a = 0; a < L.geo.dims; ++a) f[6 + a] = log2f_safe((double)tg.ext[a]);
    double tiles = 1.0;
    for (int a = 0; a < L.geo.dims; ++a) tiles *= (double)tg.count[a];
    f[1] = log2f_safe(tiles);  // tiles per time block: the parallelism a block offers
    f[9] = log2f_safe((double)k);
    if (schedule == PCOT_COT) {
        double vol = 1.0;
        for (int i = 0; i <= L.geo.dims; ++i) vol *= (p && p->cot_threshold[i] > 0) ? p->cot_threshold[i] : 1;
        f[10] = log2f_safe(vol);
    } else {
        f[10] = -1.f;
    }
    return PCOT_OK;
}

pcot_tile_params tparams(int t0, int t1, int t2, int k, int h0 = 0, int h1 = 0, int h2 = 0, int h3 = 0) {
    pcot_tile_params p;
    std::memset(&p, 0, sizeof(p));
    p.tile[0] = t0;
    p.tile[1] = t1;
    p.tile[2] = t2;
    p.time_depth = k;
    p.cot_threshold[0] = h0;
    p.cot_threshold[1] = h1;
    p.cot_threshold[2] = h2;
    p.cot_threshold[3] = h3;
    return p;
}

// MLP forward over the normalised features of every candidate and argmin of
// the predicted slowdown against the problem's fastest candidate (output 1);
// candidates without a kernel never win.
pcot_status pick_among(pcot_handle h, const int64_t* sizes, int64_t T, pcot_dtype dtype, const float* mlp_params,
                       const float* feat_mean, const float* feat_std, int ncand, const pcot_schedule* schedules,
                       const pcot_tile_params* params, void* scratch, int* best, cudaStream_t s) {
    std::vector<float> x((size_t)ncand * 12);
    std::vector<int> ok((size_t)ncand, 1);
    for (int i = 0; i < ncand; ++i) {
        float f[12];
        if (features_impl(h, sizes, T, dtype, schedules[i], params ? &params[i] : nullptr, f) != PCOT_OK) {
            ok[i] = 0;
            for (int j = 0; j < 12; ++j) f[j] = 0.f;
        }
        for (int j = 0; j < 12; ++j) {
            const float sd = feat_std[j] > 0.f ? feat_std[j] : 1.f;
            x[(size_t)i * 12 + j] = (f[j] - feat_mean[j]) / sd;
        }
    }
    float* dx = (float*)scratch;
    float* dy = dx + (size_t)ncand * 12;
    int* didx = (int*)(dy + (size_t)ncand * 2);
    PCOT_CUDA(cudaMemcpyAsync(dx, x.data(), x.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    PCOT_CUDA(mlp::forward(mlp_params, dx, ncand, dy, s));
    const float big = 1e30f;
    for (int i = 0; i < ncand; ++i)
        if (!ok[i])
            PCOT_CUDA(cudaMemcpyAsync(dy + (size_t)i * 2 + 1, &big, sizeof(float), cudaMemcpyHostToDevice, s));
    PCOT_CUDA(mlp::argmin(dy, ncand, 2, 1, didx, s));
    int idx = -1;
    PCOT_CUDA(cudaMemcpyAsync(&idx, didx, sizeof(int), cudaMemcpyDeviceToHost, s));
    PCOT_CUDA(cudaStreamSynchronize(s));
    if (idx < 0 || idx >= ncand || !ok[idx]) return PCOT_ERR_UNSUPPORTED;
    *best = idx;
    return PCOT_OK;
}

// With no model loaded: the exhaustive autotuner on a scratch grid of the
// problem's size (rows padded to 128 bytes, zero values: the kernels' speed
// does not depend on the values), allocated for the call and freed after it.
pcot_status pick_autotune(pcot_handle h, const LaunchCtx& L, const int64_t* sizes, int64_t T, pcot_dtype dtype,
                          cudaStream_t s, const std::vector<std::pair<pcot_schedule, pcot_tile_params>>& c,
                          int* best) {
    const int d = L.geo.dims;
    const int es = elem_size(dtype);
    int64_t strides[3] = {1, 1, 1};
    const int64_t step = 128 / es;
    int64_t acc = (L.geo.e[d - 1] + step - 1) / step * step;
    for (int a = d - 2; a >= 0; --a) {
        strides[a] = acc;
        acc *= L.geo.e[a];
    }
    int64_t last = 0;
    for (int a = 0; a < d; ++a) last += (L.geo.e[a] - 1) * strides[a];
    const size_t gbytes = (size_t)(last + 1) * es;
    size_t wbytes = 0;
    std::vector<pcot_schedule> sc;
    std::vector<pcot_tile_params> pr;
    for (const auto& x : c) {
        size_t b = 0;
        if (pcot_workspace_bytes(h, sizes, strides, T, dtype, x.first, &x.second, &b) == PCOT_OK)
            wbytes = std::max(wbytes, b);
        sc.push_back(x.first);
        pr.push_back(x.second);
    }
    void* grid = nullptr;
    void* ws = nullptr;
    cudaError_t e = cudaMalloc(&grid, gbytes);
    if (e == cudaSuccess) e = cudaMalloc(&ws, std::max<size_t>(wbytes, 256));
    if (e == cudaSuccess) e = cudaMemsetAsync(grid, 0, gbytes, s);
    pcot_status st = from_cuda(e);
    std::vector<float> ms(c.size(), -1.f);
    if (st == PCOT_OK)
        st = pcot_autotune(h, grid, ws, std::max<size_t>(wbytes, 256), sizes, strides, T, dtype, (int)c.size(),
                           sc.data(), pr.data(), 2, ms.data(), s);
    if (ws) cudaFree(ws);
    if (grid) cudaFree(grid);
    if (st != PCOT_OK) return st;
    int b = -1;
    for (size_t i = 0; i < ms.size(); ++i)
        if (ms[i] > 0.f && (b < 0 || ms[i] < ms[(size_t)b])) b = (int)i;
    if (b < 0) return PCOT_ERR_UNSUPPORTED;
    *best = b;
    return PCOT_OK;
}

}  // namespace

namespace {

// Schedules and tile shapes the picker chooses among (and the autotuner
// times): the plain sweep, the single-level schedule over depths and tile
// heights, and for Dirichlet grids the recursive order over depths, tile
// heights and leaf orthants (Sec. 5.1.5's exploration of tile sizes).
std::vector<std::pair<pcot_schedule, pcot_tile_params>> pick_candidates(int dims, pcot_dtype dtype, bool periodic) {
    std::vector<std::pair<pcot_schedule, pcot_tile_params>> out;
    const bool f32 = dtype == PCOT_F32;
    out.push_back({PCOT_SWEEP, tparams(0, 0, 0, 0)});
    if (dims == 2) {
        const std::vector<int> ks = f32 ? std::vector<int>{2, 4, 6, 8} : std::vector<int>{1, 2, 4};
        for (int k : ks)
            for (int H : {0, 48, 96}) out.push_back({PCOT_SLT, tparams(H, 0, 0, k)});
        if (!periodic) {
            const std::vector<int> kc = f32 ? std::vector<int>{4, 6, 8} : std::vector<int>{1, 2};
            const int th[3][3] = {{2, 256, 256}, {2, 64, 64}, {4, 16, 16}};
            for (int k : kc)
                for (int H : {64, 80, 96, 128})
                    for (const auto& t : th) out.push_back({PCOT_COT, tparams(H, 0, 0, k, t[0], t[1], t[2])});
        }
    } else if (dims == 3) {
        const std::vector<int> ks = f32 ? std::vector<int>{1, 2, 3, 4} : std::vector<int>{1, 2};
        for (int k : ks)
            for (int Hz : {32, 64, 128})
                for (int Hy : {0, 16}) out.push_back({PCOT_SLT, tparams(Hz, Hy, 0, k)});
        if (!periodic) {
            const int th[3][4] = {{1, 1, 1, 1}, {2, 4, 4, 4}, {2, 64, 64, 64}};
            for (size_t i = 0; i < 2 && i < ks.size(); ++i)
                for (const auto& t : th) out.push_back({PCOT_COT, tparams(32, 0, 0, ks[i], t[0], t[1], t[2], t[3])});
        }
    } else {
        for (int k : {8, 16, 32, 64})
            for (int w : {16, 32, 64}) out.push_back({PCOT_SLT, tparams(w, 0, 0, k)});
    }
    return out;
}

std::string pick_key(const LaunchCtx& L, int64_t T) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%d|%lld,%lld,%lld|%lld", L.dtype, (long long)L.geo.n[0], (long long)L.geo.n[1],
                  (long long)L.geo.n[2], (long long)T);
    return buf;
}

pcot_status pick_impl(pcot_handle h, const int64_t* sizes, int64_t T, pcot_dtype dtype, cudaStream_t s,
                      pcot_schedule* schedule, pcot_tile_params* params) {
    LaunchCtx L;
    PCOT_TRY(make_ctx(h, sizes, nullptr, dtype, s, &L));
    const std::string key = pick_key(L, T);
    auto it = h->pick_cache.find(key);
    if (it != h->pick_cache.end()) {
        *schedule = it->second.first;
        *params = it->second.second;
        return PCOT_OK;
    }
    const auto c = pick_candidates(L.geo.dims, dtype, L.geo.periodic != 0);
    int best = -1;
    if (!h->picker.empty()) {
        const int np = mlp::param_count();
        if ((int)h->picker.size() != np + 24) return PCOT_ERR_INVALID_ARG;
        if (!h->d_picker) {
            PCOT_CUDA(cudaMalloc((void**)&h->d_picker, sizeof(float) * np));
            PCOT_CUDA(cudaMemcpy(h->d_picker, h->picker.data(), sizeof(float) * np, cudaMemcpyHostToDevice));
        }
        const size_t need = c.size() * 14 * sizeof(float) + 256;
        if (h->pick_bytes < need) {
            if (h->d_pick) cudaFree(h->d_pick);
            h->d_pick = nullptr;
            h->pick_bytes = 0;
            PCOT_CUDA(cudaMalloc(&h->d_pick, need));
            h->pick_bytes = need;
        }
        std::vector<pcot_schedule> sc;
        std::vector<pcot_tile_params> pr;
        for (const auto& x : c) {
            sc.push_back(x.first);
            pr.push_back(x.second);
        }
        PCOT_TRY(pick_among(h, sizes, T, dtype, h->d_picker, h->picker.data() + np, h->picker.data() + np + 12,
                            (int)c.size(), sc.data(), pr.data(), h->d_pick, &best, s));
    } else {
        PCOT_TRY(pick_autotune(h, L, sizes, T, dtype, s, c, &best));
    }
    *schedule = c[(size_t)best].first;
    *params = c[(size_t)best].second;
    h->pick_cache[key] = c[(size_t)best];
    return PCOT_OK;
}

}  // namespace

extern "C" {

int pcot_mlp_param_count(void) { return mlp::param_count(); }

pcot_status pcot_mlp_scratch_bytes(int batch, size_t* bytes) {
    if (batch < 1 || !bytes) return PCOT_ERR_INVALID_ARG;
    *bytes = mlp::scratch_bytes(batch);
    return PCOT_OK;
}

pcot_status pcot_mlp_forward(const float* params, const float* x, int batch, float* y, void* stream) {
    if (!params || !x || !y || batch < 1) return PCOT_ERR_INVALID_ARG;
    PCOT_CUDA(mlp::forward(params, x, batch, y, (cudaStream_t)stream));
    return PCOT_OK;
}

pcot_status pcot_mlp_grad(const float* params, const float* x, const float* target, int batch, float* grad,
                          float* loss, void* scratch, size_t scratch_bytes, void* stream) {
    if (!params || !x || !target || !grad || !scratch || batch < 1) return PCOT_ERR_INVALID_ARG;
    if (scratch_bytes < mlp::scratch_bytes(batch)) return PCOT_ERR_OOM;
    if (((uintptr_t)scratch & 15) != 0) return PCOT_ERR_ALIGNMENT;
    PCOT_CUDA(mlp::grad(params, x, target, batch, grad, loss, scratch, (cudaStream_t)stream));
    return PCOT_OK;
}

pcot_status pcot_mlp_adam(float* params, const float* grad, float* m, float* v, int n, int step, float lr,
                          float beta1, float beta2, float eps, void* stream) {
    if (!params || !grad || !m || !v || n < 1 || step < 1) return PCOT_ERR_INVALID_ARG;
    PCOT_CUDA(mlp::adam(params, grad, m, v, n, step, lr, beta1, beta2, eps, (cudaStream_t)stream));
    return PCOT_OK;
}

pcot_status pcot_mlp_argmin(const float* y, int n, int stride, int col, int* out_index, void* stream) {
    if (!y || !out_index || n < 1 || stride < 1 || col < 0 || col >= stride) return PCOT_ERR_INVALID_ARG;
    PCOT_CUDA(mlp::argmin(y, n, stride, col, out_index, (cudaStream_t)stream));
    return PCOT_OK;
}

pcot_status pcot_features(pcot_handle h, const int64_t* sizes, int64_t T, pcot_dtype dtype, pcot_schedule schedule,
                          const pcot_tile_params* params, float* out12) {
    if (!h || !sizes || !out12 || T < 0) return PCOT_ERR_INVALID_ARG;
    return features_impl(h, sizes, T, dtype, schedule, params, out12);
}

pcot_status pcot_pick_among(pcot_handle h, const int64_t* sizes, int64_t T, pcot_dtype dtype, const float* mlp_params,
                            const float* feat_mean, const float* feat_std, int ncand, const pcot_schedule* schedules,
                            const pcot_tile_params* params, void* scratch, int* best, void* stream) {
    if (!h || !sizes || !mlp_params || !feat_mean || !feat_std || ncand < 1 || !schedules || !scratch || !best)
        return PCOT_ERR_INVALID_ARG;
    return pick_among(h, sizes, T, dtype, mlp_params, feat_mean, feat_std, ncand, schedules, params, scratch, best,
                      (cudaStream_t)stream);
}

pcot_status pcot_picker_load(pcot_handle h, const float* mlp_params, const float* feat_mean,
                             const float* feat_std) {
    if (!h) return PCOT_ERR_INVALID_ARG;
    if ((mlp_params == nullptr) != (feat_mean == nullptr) || (mlp_params == nullptr) != (feat_std == nullptr))
        return PCOT_ERR_INVALID_ARG;
    const int np = mlp::param_count();
    h->picker.clear();
    if (mlp_params) {
        h->picker.assign(mlp_params, mlp_params + np);
        h->picker.insert(h->picker.end(), feat_mean, feat_mean + 12);
        h->picker.insert(h->picker.end(), feat_std, feat_std + 12);
    }
    if (h->d_picker) {
        cudaFree(h->d_picker);
        h->d_picker = nullptr;
    }
    h->pick_cache.clear();
    return PCOT_OK;
}

pcot_status pcot_candidates(pcot_handle h, pcot_dtype dtype, int cap, pcot_schedule* schedules,
                            pcot_tile_params* params, int* count) {
    if (!h || !count || cap < 0) return PCOT_ERR_INVALID_ARG;
    if (dtype != PCOT_F32 && dtype != PCOT_F64 && dtype != PCOT_F64_EXACT) return PCOT_ERR_INVALID_ARG;
    const auto c = pick_candidates(h->dims, dtype, h->boundary == PCOT_PERIODIC);
    *count = (int)c.size();
    if (cap == 0) return PCOT_OK;
    if (!schedules || !params) return PCOT_ERR_INVALID_ARG;
    if (cap < (int)c.size()) return PCOT_ERR_OOM;
    for (size_t i = 0; i < c.size(); ++i) {
        schedules[i] = c[i].first;
        params[i] = c[i].second;
    }
    return PCOT_OK;
}

pcot_status pcot_pick(pcot_handle h, const int64_t* sizes, int64_t T, pcot_dtype dtype, pcot_schedule* schedule,
                      pcot_tile_params* params) {
    if (!h || !sizes || !schedule || !params || T < 0) return PCOT_ERR_INVALID_ARG;
    return pick_impl(h, sizes, T, dtype, nullptr, schedule, params);
}

}  // extern "C"

// Handle fields for the allocation-free entry point (api_noalloc.cu).
namespace pcot {
pcot_status handle_describe(pcot_handle h, int* dims, int* periodic, double* coeffs7) {
    if (!h) return PCOT_ERR_INVALID_ARG;
    *dims = h->dims;
    *periodic = h->boundary == PCOT_PERIODIC ? 1 : 0;
    for (int i = 0; i < 7; ++i) coeffs7[i] = h->coeffs[i];
    return PCOT_OK;
}
void handle_count_launches(pcot_handle h, int64_t n) {
    if (h) h->launches += n;
}
}  // namespace pcot

// ---- Gauss-Seidel 2-D ---------------------------------------------------
namespace {

// Tile shape and recursion threshold of a GS-2D run (defaults per schedule).
bool gs_shape(pcot_schedule schedule, const pcot_tile_params* p, int32_t* tile, int32_t* theta) {
    if (schedule != PCOT_SWEEP && schedule != PCOT_SLT && schedule != PCOT_COT) return false;
    const int kt_def = schedule == PCOT_SWEEP ? 1 : 8;
    tile[0] = (p && p->time_depth > 0) ? p->time_depth : kt_def;
    tile[1] = (p && p->tile[0] > 0) ? p->tile[0] : 32;
    tile[2] = (p && p->tile[1] > 0) ? p->tile[1] : 128;
    if (schedule == PCOT_SWEEP && tile[0] != 1) return false;
    // default leaf 32 x 32 x 32 tiles: measured at 2000^2 x 500, the recursive
    // order's speed rises with the leaf size (more independent tiles per
    // wavefront of a leaf): FP32 49.5 GU/s at (8, 16, 16), 109 at (32, 32, 32)
    for (int d = 0; d < 3; ++d) theta[d] = (p && p->cot_threshold[d] > 0) ? p->cot_threshold[d] : 32;
    if (tile[0] * tile[1] > 1024 || tile[0] * tile[1] < 1 || tile[2] < 2 || tile[2] > 4096) return false;
    return true;
}

pcot_status gs_get_plan(pcot_handle h, int64_t n0, int64_t n1, int64_t T, pcot_schedule schedule,
                        const int32_t* tile, const int32_t* theta, GsPlanCache** out) {
    char key[160];
    snprintf(key, sizeof(key), "%lld,%lld,%lld,%d,%d,%d,%d,%d,%d,%d", (long long)n0, (long long)n1, (long long)T,
             (int)schedule, tile[0], tile[1], tile[2], theta[0], theta[1], theta[2]);
    if (h) {
        auto it = h->gs_cache.find(key);
        if (it != h->gs_cache.end()) {
            *out = it->second;
            return PCOT_OK;
        }
    }
    GsPlanCache* c = new GsPlanCache();
    if (!gs_plan(n0, n1, T, tile, schedule == PCOT_COT ? 1 : 0, theta, &c->plan)) {
        delete c;
        return PCOT_ERR_UNSUPPORTED;
    }
    for (int d = 0; d < 3; ++d) c->tile[d] = tile[d];
    c->counts_bytes = round_up(c->plan.deps.size() * 4, kAlign);
    c->image_bytes = kAlign + c->counts_bytes + round_up(c->plan.queue.size() * 4 + 4, kAlign);
    if (h) {
        if (h->gs_cache.size() >= 16) {
            for (auto& kv : h->gs_cache) {
                if (kv.second->pinned) cudaFreeHost(kv.second->pinned);
                delete kv.second;
            }
            h->gs_cache.clear();
        }
        h->gs_cache[key] = c;
    }
    *out = c;
    return PCOT_OK;
}

pcot_status gs_check_args(const int64_t* sizes, const int64_t* strides, int64_t T, int64_t* pitch) {
    if (!sizes || T < 0) return PCOT_ERR_INVALID_ARG;
    if (sizes[0] < 1 || sizes[1] < 1 || sizes[0] > (1LL << 30) || sizes[1] > (1LL << 30)) return PCOT_ERR_INVALID_ARG;
    if (strides) {
        if (strides[1] != 1) return PCOT_ERR_UNSUPPORTED;
        if (strides[0] < sizes[1] + 2) return PCOT_ERR_INVALID_ARG;
        *pitch = strides[0];
    } else {
        *pitch = sizes[1] + 2;
    }
    return PCOT_OK;
}

}  // namespace

extern "C" {

pcot_status pcot_gs2d_plan_query(const int64_t* sizes, int64_t T, pcot_schedule schedule,
                                 const pcot_tile_params* params, int32_t* lattice, int32_t* tile, int64_t* n_tiles,
                                 int32_t* queue, int32_t* deps, int64_t cap) {
    int64_t pitch = 0;
    PCOT_TRY(gs_check_args(sizes, nullptr, T, &pitch));
    if (T < 1) return PCOT_ERR_INVALID_ARG;
    int32_t tl[3], th[3];
    if (!gs_shape(schedule, params, tl, th)) return PCOT_ERR_UNSUPPORTED;
    GsPlanCache* c = nullptr;
    PCOT_TRY(gs_get_plan(nullptr, sizes[0], sizes[1], T, schedule, tl, th, &c));
    for (int d = 0; d < 3; ++d) {
        if (lattice) lattice[d] = c->plan.lattice[d];
        if (tile) tile[d] = tl[d];
    }
    if (n_tiles) *n_tiles = (int64_t)c->plan.queue.size();
    if (queue)
        for (int64_t k = 0; k < cap && k < (int64_t)c->plan.queue.size(); ++k) queue[k] = c->plan.queue[(size_t)k];
    if (deps)
        for (int64_t k = 0; k < cap && k < (int64_t)c->plan.deps.size(); ++k) deps[k] = c->plan.deps[(size_t)k];
    delete c;
    return PCOT_OK;
}

pcot_status pcot_skew_plan_query(const int64_t* sizes, int64_t T, const pcot_tile_params* params,
                                 int32_t* lattice, int32_t* tile, int64_t* n_tiles, int32_t* queue, int32_t* deps,
                                 int64_t cap) {
    int64_t pitch = 0;
    PCOT_TRY(gs_check_args(sizes, nullptr, T, &pitch));
    if (T < 1) return PCOT_ERR_INVALID_ARG;
    int32_t tl[3], th[3];
    int rec = 0;
    if (!skew_shape(params, tl, &rec, th)) return PCOT_ERR_INVALID_ARG;
    GsPlanCache* c = nullptr;
    PCOT_TRY(skew_get_plan(nullptr, sizes[0], sizes[1], T, tl, rec, th, &c));
    for (int d = 0; d < 3; ++d) {
        if (lattice) lattice[d] = c->plan.lattice[d];
        if (tile) tile[d] = tl[d];
    }
    if (n_tiles) *n_tiles = (int64_t)c->plan.queue.size();
    if (queue)
        for (int64_t k = 0; k < cap && k < (int64_t)c->plan.queue.size(); ++k) queue[k] = c->plan.queue[(size_t)k];
    if (deps)
        for (int64_t k = 0; k < cap && k < (int64_t)c->plan.queue.size(); ++k)
            deps[k] = c->plan.deps[(size_t)c->plan.queue[(size_t)k]];
    delete c;
    return PCOT_OK;
}

pcot_status pcot_gs2d_workspace_bytes(const int64_t* sizes, int64_t T, pcot_schedule schedule,
                                      const pcot_tile_params* params, size_t* bytes) {
    if (!bytes) return PCOT_ERR_INVALID_ARG;
    int64_t pitch = 0;
    PCOT_TRY(gs_check_args(sizes, nullptr, T, &pitch));
    int32_t tl[3], th[3];
    if (!gs_shape(schedule, params, tl, th)) return PCOT_ERR_UNSUPPORTED;
    if (T == 0) {
        *bytes = 0;
        return PCOT_OK;
    }
    int64_t L[3];
    const int64_t ext[3] = {T, T - 1 + sizes[0], 2 * T - 3 + sizes[0] + sizes[1]};
    for (int d = 0; d < 3; ++d) L[d] = (ext[d] + tl[d] - 1) / tl[d];
    const int64_t cells = L[0] * L[1] * L[2];
    if (cells > (1LL << 28)) return PCOT_ERR_UNSUPPORTED;
    // head block + counts of every lattice id + the queue (at most every id)
    *bytes = kAlign + round_up((size_t)cells * 4, kAlign) + round_up((size_t)cells * 4 + 4, kAlign);
    return PCOT_OK;
}

pcot_status pcot_gs2d_run(pcot_handle h, void* grid, void* workspace, size_t workspace_bytes, const int64_t* sizes,
                          const int64_t* strides, int64_t T, pcot_dtype dtype, pcot_schedule schedule,
                          const pcot_tile_params* params, void* stream) {
    if (!h || !grid) return PCOT_ERR_INVALID_ARG;
    if (dtype != PCOT_F32 && dtype != PCOT_F64 && dtype != PCOT_F64_EXACT) return PCOT_ERR_INVALID_ARG;
    int64_t pitch = 0;
    PCOT_TRY(gs_check_args(sizes, strides, T, &pitch));
    int32_t tl[3], th[3];
    if (!gs_shape(schedule, params, tl, th)) return PCOT_ERR_UNSUPPORTED;
    if (((uintptr_t)grid % (dtype == PCOT_F32 ? 4 : 8)) != 0) return PCOT_ERR_ALIGNMENT;
    if (T == 0) return PCOT_OK;
    size_t need = 0;
    PCOT_TRY(pcot_gs2d_workspace_bytes(sizes, T, schedule, params, &need));
    if (!workspace || workspace_bytes < need) return PCOT_ERR_OOM;
    if (((uintptr_t)workspace % kAlign) != 0) return PCOT_ERR_ALIGNMENT;
    PCOT_TRY(ensure_device(h));
    GsPlanCache* c = nullptr;
    PCOT_TRY(gs_get_plan(h, sizes[0], sizes[1], T, schedule, tl, th, &c));
    if (c->plan.queue.empty()) return PCOT_OK;
    if (!c->pinned) {
        void* p = nullptr;
        PCOT_CUDA(cudaMallocHost(&p, c->image_bytes));
        unsigned char* img = (unsigned char*)p;
        std::memset(img, 0, c->image_bytes);
        std::memcpy(img + kAlign, c->plan.deps.data(), c->plan.deps.size() * 4);
        std::memcpy(img + kAlign + c->counts_bytes, c->plan.queue.data(), c->plan.queue.size() * 4);
        c->pinned = p;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* ws = (unsigned char*)workspace;
    PCOT_CUDA(cudaMemcpyAsync(ws, c->pinned, c->image_bytes, cudaMemcpyHostToDevice, s));
    GsDev q;
    std::memset(&q, 0, sizeof(q));
    q.head = (int32_t*)ws;
    q.counts = (int32_t*)(ws + kAlign);
    q.queue = (const int32_t*)(ws + kAlign + c->counts_bytes);
    q.ntiles = (int64_t)c->plan.queue.size();
    for (int d = 0; d < 3; ++d) {
        q.lattice[d] = c->plan.lattice[d];
        q.tile[d] = tl[d];
    }
    q.n0 = sizes[0];
    q.n1 = sizes[1];
    q.T = T;
    q.pitch = pitch;
    gs2d_window(&q);
    q.status = h->d_status;
    q.timeout_ns = h->timeout_ns;
    const int dt = dtype == PCOT_F32 ? kF32 : kF64;
    if (gs2d_smem_bytes(dt, q) > 227 * 1024) return PCOT_ERR_UNSUPPORTED;
    const int per_sm = gs2d_ctas_per_sm(dt, q);
    if (per_sm < 1) return PCOT_ERR_UNSUPPORTED;
    int64_t nctas = (int64_t)per_sm * h->num_sms;
    if (nctas > q.ntiles) nctas = q.ntiles;
    PCOT_CUDA(launch_gs2d(dt, grid, q, (int)nctas, s));
    ++h->launches;
    return PCOT_OK;
}

}  // extern "C"

// ---- FDTD-2D ----------------------------------------------------------------
namespace {

bool fd_shape(pcot_schedule schedule, pcot_dtype dtype, const pcot_tile_params* p, int32_t* tile, int32_t* depth,
              int64_t* theta) {
    if (schedule != PCOT_SWEEP && schedule != PCOT_SLT && schedule != PCOT_COT) return false;
    const bool f32 = dtype == PCOT_F32;
    tile[0] = (p && p->tile[0] > 0) ? p->tile[0] : (f32 ? 48 : 32);
    tile[1] = (p && p->tile[1] > 0) ? p->tile[1] : (f32 ? 64 : 32);
    *depth = (p && p->time_depth > 0) ? p->time_depth : (f32 ? 8 : 4);
    theta[0] = (p && p->cot_threshold[0] > 0) ? p->cot_threshold[0] : 2;
    theta[1] = (p && p->cot_threshold[1] > 0) ? p->cot_threshold[1] : 256;
    theta[2] = (p && p->cot_threshold[2] > 0) ? p->cot_threshold[2] : 256;
    if (schedule == PCOT_SWEEP) return true;
    // tiles at least as wide as the halo: a window meets only neighbouring tiles
    if (tile[0] < *depth || tile[1] < *depth || *depth > 64 || tile[0] > 1024 || tile[1] > 1024) return false;
    return true;
}

size_t fd_span_bytes(const int64_t* sizes, int64_t pitch, pcot_dtype dtype) {
    return (size_t)((sizes[0] - 1) * pitch + sizes[1]) * (dtype == PCOT_F32 ? 4 : 8);
}

pcot_status fd_check_args(const int64_t* sizes, const int64_t* strides, int64_t T, pcot_dtype dtype, int64_t* pitch) {
    if (!sizes || T < 0) return PCOT_ERR_INVALID_ARG;
    if (dtype != PCOT_F32 && dtype != PCOT_F64 && dtype != PCOT_F64_EXACT) return PCOT_ERR_INVALID_ARG;
    if (sizes[0] < 1 || sizes[1] < 1 || sizes[0] > (1LL << 30) || sizes[1] > (1LL << 30)) return PCOT_ERR_INVALID_ARG;
    if (strides) {
        if (strides[1] != 1) return PCOT_ERR_UNSUPPORTED;
        if (strides[0] < sizes[1]) return PCOT_ERR_INVALID_ARG;
        *pitch = strides[0];
    } else {
        *pitch = sizes[1];
    }
    return PCOT_OK;
}

}  // namespace

extern "C" {

pcot_status pcot_fdtd2d_workspace_bytes(const int64_t* sizes, const int64_t* strides, int64_t T, pcot_dtype dtype,
                                        pcot_schedule schedule, const pcot_tile_params* params, size_t* bytes) {
    if (!bytes) return PCOT_ERR_INVALID_ARG;
    int64_t pitch = 0;
    PCOT_TRY(fd_check_args(sizes, strides, T, dtype, &pitch));
    int32_t tile[2], depth;
    int64_t theta[3];
    if (!fd_shape(schedule, dtype, params, tile, &depth, theta)) return PCOT_ERR_UNSUPPORTED;
    size_t b = 3 * round_up(fd_span_bytes(sizes, pitch, dtype), kAlign);
    if (schedule == PCOT_COT && T >= depth) {
        const int64_t P = T / depth;
        const int64_t L0 = (sizes[0] + tile[0] - 1) / tile[0], L1 = (sizes[1] + tile[1] - 1) / tile[1];
        const int64_t n = P * L0 * L1;
        if (n > (1LL << 28)) return PCOT_ERR_UNSUPPORTED;
        b += kAlign + 2 * round_up((size_t)n * 4, kAlign);
    }
    *bytes = b;
    return PCOT_OK;
}

pcot_status pcot_fdtd2d_run(pcot_handle h, void* ex, void* ey, void* hz, const void* fict, void* workspace,
                            size_t workspace_bytes, const int64_t* sizes, const int64_t* strides, int64_t T,
                            pcot_dtype dtype, pcot_schedule schedule, const pcot_tile_params* params, void* stream) {
    if (!h || !ex || !ey || !hz || (T > 0 && !fict)) return PCOT_ERR_INVALID_ARG;
    int64_t pitch = 0;
    PCOT_TRY(fd_check_args(sizes, strides, T, dtype, &pitch));
    int32_t tile[2], depth;
    int64_t theta[3];
    if (!fd_shape(schedule, dtype, params, tile, &depth, theta)) return PCOT_ERR_UNSUPPORTED;
    const int es = dtype == PCOT_F32 ? 4 : 8;
    if ((uintptr_t)ex % es || (uintptr_t)ey % es || (uintptr_t)hz % es || (uintptr_t)fict % es)
        return PCOT_ERR_ALIGNMENT;
    if (T == 0) return PCOT_OK;
    size_t need = 0;
    PCOT_TRY(pcot_fdtd2d_workspace_bytes(sizes, strides, T, dtype, schedule, params, &need));
    if (!workspace || workspace_bytes < need) return PCOT_ERR_OOM;
    if ((uintptr_t)workspace % kAlign) return PCOT_ERR_ALIGNMENT;
    PCOT_TRY(ensure_device(h));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t span = fd_span_bytes(sizes, pitch, dtype), tw = round_up(span, kAlign);
    unsigned char* ws = (unsigned char*)workspace;
    void* f0[3] = {ex, ey, hz};
    void* f1[3] = {ws, ws + tw, ws + 2 * tw};
    FdDev q;
    std::memset(&q, 0, sizeof(q));
    q.nx = sizes[0];
    q.ny = sizes[1];
    q.pitch = pitch;
    q.tile[0] = tile[0];
    q.tile[1] = tile[1];
    q.depth = depth;
    const int dt = dtype == PCOT_F32 ? kF32 : kF64;
    if (schedule != PCOT_SWEEP && fdtd2d_smem_bytes(dt, q) > 227 * 1024) return PCOT_ERR_UNSUPPORTED;
    int cur = 0;  // copy holding the current fields
    int64_t t = 0;
    if (schedule == PCOT_SWEEP) {
        for (; t < T; ++t) {
            PCOT_CUDA(launch_fdtd2d_step(dt, q, cur ? f1 : f0, cur ? f0 : f1, fict, t, s));
            ++h->launches;
            cur ^= 1;
        }
    }
    if (schedule == PCOT_COT && T >= depth) {
        const int64_t P = T / depth;
        const int64_t L[2] = {(sizes[0] + tile[0] - 1) / tile[0], (sizes[1] + tile[1] - 1) / tile[1]};
        char key[160];
        snprintf(key, sizeof(key), "%lld,%lld,%d,%d,%d,%lld,%lld,%lld,%lld", (long long)sizes[0], (long long)sizes[1],
                 tile[0], tile[1], depth, (long long)P, (long long)theta[0], (long long)theta[1], (long long)theta[2]);
        FdPlanCache* c = nullptr;
        auto it = h->fd_cache.find(key);
        if (it != h->fd_cache.end()) {
            c = it->second;
        } else {
            c = new FdPlanCache();
            c->queue = pcot_lattice_order((int)P, 2, L, theta, nullptr);
            c->counts = lattice_dep_counts((int)P, 2, L);
            c->lattice[0] = (int32_t)P;
            c->lattice[1] = (int32_t)L[0];
            c->lattice[2] = (int32_t)L[1];
            c->counts_bytes = round_up(c->counts.size() * 4, kAlign);
            c->image_bytes = kAlign + c->counts_bytes + round_up(c->queue.size() * 4, kAlign);
            void* p = nullptr;
            cudaError_t e = cudaMallocHost(&p, c->image_bytes);
            if (e != cudaSuccess) {
                delete c;
                return from_cuda(e);
            }
            std::memset(p, 0, c->image_bytes);
            std::memcpy((unsigned char*)p + kAlign, c->counts.data(), c->counts.size() * 4);
            std::memcpy((unsigned char*)p + kAlign + c->counts_bytes, c->queue.data(), c->queue.size() * 4);
            c->pinned = p;
            if (h->fd_cache.size() >= 16) {
                for (auto& kv : h->fd_cache) {
                    if (kv.second->pinned) cudaFreeHost(kv.second->pinned);
                    delete kv.second;
                }
                h->fd_cache.clear();
            }
            h->fd_cache[key] = c;
        }
        unsigned char* img = ws + 3 * tw;
        PCOT_CUDA(cudaMemcpyAsync(img, c->pinned, c->image_bytes, cudaMemcpyHostToDevice, s));
        CotDev cd;
        std::memset(&cd, 0, sizeof(cd));
        cd.head = (int32_t*)img;
        cd.counts = (int32_t*)(img + kAlign);
        cd.queue = (const int32_t*)(img + kAlign + c->counts_bytes);
        cd.ntiles = (int64_t)c->queue.size();
        for (int i = 0; i < 4; ++i) cd.lattice[i] = c->lattice[i];
        cd.status = h->d_status;
        cd.timeout_ns = h->timeout_ns;
        const int per_sm = fdtd2d_cot_ctas_per_sm(dt, q);
        if (per_sm < 1) return PCOT_ERR_UNSUPPORTED;
        int64_t nctas = (int64_t)per_sm * h->num_sms;
        const int64_t cap = std::max<int64_t>(h->num_sms, L[0] * L[1] * 2 / 5);  // as for the stencils
        if (nctas > cap) nctas = cap;
        if (nctas > cd.ntiles) nctas = cd.ntiles;
        PCOT_CUDA(launch_fdtd2d_cot(dt, q, cd, f0, f1, fict, (int)nctas, s));
        ++h->launches;
        t = P * depth;
        cur = (int)(P & 1);
    }
    // single-level blocks (the whole run for PCOT_SLT, the tail for PCOT_COT)
    while (t < T) {
        const int k = (int)std::min<int64_t>(depth, T - t);
        PCOT_CUDA(launch_fdtd2d_block(dt, q, cur ? f1 : f0, cur ? f0 : f1, fict, t, k, s));
        ++h->launches;
        cur ^= 1;
        t += k;
    }
    if (cur) {  // the result is in the workspace copy
        for (int a = 0; a < 3; ++a) PCOT_CUDA(cudaMemcpyAsync(f0[a], f1[a], span, cudaMemcpyDeviceToDevice, s));
    }
    return PCOT_OK;
}

}  // extern "C"

// ---- LU / Cholesky ------------------------------------------------------------
namespace {

bool la_shape(pcot_la_kind kind, pcot_schedule schedule, const pcot_tile_params* p, int32_t* b, int32_t* theta) {
    if (kind != PCOT_LA_LU && kind != PCOT_LA_CHOLESKY) return false;
    if (schedule != PCOT_SWEEP && schedule != PCOT_SLT && schedule != PCOT_COT) return false;
    // defaults measured on LU 3000^2 and Cholesky 4000^2 (FP64): 32-wide tiles
    // beat 64-wide ones (more tiles in flight, shorter diagonal chain), and
    // leaves of 2 x 32 x 32 tiles beat both finer and k-only splits
    static const int32_t kTheta[3] = {2, 32, 32};
    *b = (p && p->tile[0] > 0) ? p->tile[0] : 32;
    for (int d = 0; d < 3; ++d) theta[d] = (p && p->cot_threshold[d] > 0) ? p->cot_threshold[d] : kTheta[d];
    return la_block_supported(*b);
}

pcot_status la_get_plan(pcot_handle h, pcot_la_kind kind, int64_t n, pcot_schedule schedule, int32_t b,
                        const int32_t* theta, LaPlanCache** out) {
    char key[128];
    snprintf(key, sizeof(key), "%d,%lld,%d,%d,%d,%d,%d", (int)kind, (long long)n, (int)schedule, b, theta[0], theta[1],
             theta[2]);
    if (h) {
        auto it = h->la_cache.find(key);
        if (it != h->la_cache.end()) {
            *out = it->second;
            return PCOT_OK;
        }
    }
    LaPlanCache* c = new LaPlanCache();
    if (!la_plan((int)kind, n, b, schedule == PCOT_COT ? 1 : 0, theta, &c->plan)) {
        delete c;
        return PCOT_ERR_UNSUPPORTED;
    }
    c->counts_bytes = round_up(c->plan.deps.size() * 4, kAlign);
    c->image_bytes = kAlign + c->counts_bytes + round_up(c->plan.queue.size() * 4 + 4, kAlign);
    if (h) {
        if (h->la_cache.size() >= 16) {
            for (auto& kv : h->la_cache) {
                if (kv.second->pinned) cudaFreeHost(kv.second->pinned);
                delete kv.second;
            }
            h->la_cache.clear();
        }
        h->la_cache[key] = c;
    }
    *out = c;
    return PCOT_OK;
}

}  // namespace

extern "C" {

pcot_status pcot_la_plan_query(pcot_la_kind kind, int64_t n, pcot_schedule schedule, const pcot_tile_params* params,
                               int32_t* L, int32_t* b, int64_t* n_tiles, int32_t* queue, int32_t* deps, int64_t cap) {
    if (n < 1 || n > (1LL << 30)) return PCOT_ERR_INVALID_ARG;
    int32_t bb = 0, th[3];
    if (!la_shape(kind, schedule, params, &bb, th)) return PCOT_ERR_UNSUPPORTED;
    LaPlanCache* c = nullptr;
    PCOT_TRY(la_get_plan(nullptr, kind, n, schedule, bb, th, &c));
    if (L) *L = c->plan.L;
    if (b) *b = bb;
    if (n_tiles) *n_tiles = (int64_t)c->plan.queue.size();
    if (queue)
        for (int64_t k = 0; k < cap && k < (int64_t)c->plan.queue.size(); ++k) queue[k] = c->plan.queue[(size_t)k];
    if (deps)
        for (int64_t k = 0; k < cap && k < (int64_t)c->plan.deps.size(); ++k) deps[k] = c->plan.deps[(size_t)k];
    delete c;
    return PCOT_OK;
}

pcot_status pcot_la_workspace_bytes(pcot_la_kind kind, int64_t n, pcot_schedule schedule,
                                    const pcot_tile_params* params, size_t* bytes) {
    if (!bytes || n < 0 || n > (1LL << 30)) return PCOT_ERR_INVALID_ARG;
    int32_t b = 0, th[3];
    if (!la_shape(kind, schedule, params, &b, th)) return PCOT_ERR_UNSUPPORTED;
    *bytes = 0;
    if (schedule != PCOT_COT || n == 0) return PCOT_OK;
    const int64_t L = (n + b - 1) / b;
    if (L > 256) return PCOT_ERR_UNSUPPORTED;
    // head block + counts of every lattice id + the queue (at most every id)
    *bytes = kAlign + round_up((size_t)(L * L * L) * 4, kAlign) + round_up((size_t)(L * L * L) * 4 + 4, kAlign);
    return PCOT_OK;
}

pcot_status pcot_la_run(pcot_handle h, pcot_la_kind kind, void* A, void* workspace, size_t workspace_bytes, int64_t n,
                        int64_t lda, pcot_dtype dtype, pcot_schedule schedule, const pcot_tile_params* params,
                        void* stream) {
    if (!h || n < 0 || n > (1LL << 30) || lda < n || (n > 0 && !A)) return PCOT_ERR_INVALID_ARG;
    if (dtype != PCOT_F32 && dtype != PCOT_F64 && dtype != PCOT_F64_EXACT) return PCOT_ERR_INVALID_ARG;
    if (dtype == PCOT_F32) return PCOT_ERR_UNSUPPORTED;
    int32_t b = 0, th[3];
    if (!la_shape(kind, schedule, params, &b, th)) return PCOT_ERR_UNSUPPORTED;
    if (((uintptr_t)A % 8) != 0) return PCOT_ERR_ALIGNMENT;
    if (n == 0) return PCOT_OK;
    size_t need = 0;
    PCOT_TRY(pcot_la_workspace_bytes(kind, n, schedule, params, &need));
    if (need && (!workspace || workspace_bytes < need)) return PCOT_ERR_OOM;
    if (need && ((uintptr_t)workspace % kAlign) != 0) return PCOT_ERR_ALIGNMENT;
    PCOT_TRY(ensure_device(h));
    cudaStream_t s = (cudaStream_t)stream;
    LaDev d;
    std::memset(&d, 0, sizeof(d));
    d.A = (double*)A;
    d.lda = lda;
    d.n = n;
    d.b = b;
    d.L = (int32_t)((n + b - 1) / b);
    d.status = h->d_status;
    d.timeout_ns = h->timeout_ns;
    const bool fused = dtype == PCOT_F64;
    const int k = kind == PCOT_LA_LU ? kLaLU : kLaCholesky;
    int nctas = 0;
    if (schedule == PCOT_COT) {
        LaPlanCache* c = nullptr;
        PCOT_TRY(la_get_plan(h, kind, n, schedule, b, th, &c));
        if (c->plan.queue.empty()) return PCOT_OK;  // LU of a 1 x 1 matrix: nothing to do
        if (!c->pinned) {
            void* p = nullptr;
            PCOT_CUDA(cudaMallocHost(&p, c->image_bytes));
            unsigned char* img = (unsigned char*)p;
            std::memset(img, 0, c->image_bytes);
            std::memcpy(img + kAlign, c->plan.deps.data(), c->plan.deps.size() * 4);
            std::memcpy(img + kAlign + c->counts_bytes, c->plan.queue.data(), c->plan.queue.size() * 4);
            c->pinned = p;
        }
        unsigned char* ws = (unsigned char*)workspace;
        PCOT_CUDA(cudaMemcpyAsync(ws, c->pinned, c->image_bytes, cudaMemcpyHostToDevice, s));
        d.head = (int32_t*)ws;
        d.counts = (int32_t*)(ws + kAlign);
        d.queue = (const int32_t*)(ws + kAlign + c->counts_bytes);
        d.ntiles = (int64_t)c->plan.queue.size();
        const int per_sm = la_ctas_per_sm(b, fused, k);
        if (per_sm < 1) return PCOT_ERR_UNSUPPORTED;
        int64_t m = (int64_t)per_sm * h->num_sms;
        if (m > d.ntiles) m = d.ntiles;
        nctas = (int)m;
    }
    int64_t launches = 0;
    const cudaError_t e = launch_la(d, k, fused, schedule == PCOT_SWEEP ? kLaSweep : schedule == PCOT_SLT ? kLaSlt : kLaCot,
                                    nctas, s, &launches);
    h->launches += launches;
    PCOT_CUDA(e);
    return PCOT_OK;
}

}  // extern "C"
