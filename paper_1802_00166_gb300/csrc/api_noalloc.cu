// Entry point that allocates nothing: the single-level (or sweep) schedule
// with its second buffer in a fixed, file-scope device array.
//
// Who needs it: callers that may not allocate device memory at the moment
// they advance a grid -- real-time or embedded hosts that reserve all device
// memory up front and forbid allocation afterwards, services that run with a
// fixed memory budget and must not grow it per request, and library layers
// that are handed only the grid and a stream and may not touch the caller's
// allocator.  pcot_run needs a caller-provided workspace (the grid's twin);
// this variant uses kNoallocBytes of device memory that every GPU loading the
// library reserves at module load and keeps until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "kernels.h"
#include "pcot.h"

namespace pcot {
pcot_status handle_describe(pcot_handle h, int* dims, int* periodic, double* coeffs7);
void handle_count_launches(pcot_handle h, int64_t n);
}  // namespace pcot

namespace {

using namespace pcot;

constexpr size_t kNoallocBytes = (size_t)PCOT_NOALLOC_MAX_BYTES;
constexpr int kMaxDevices = 64;

// The shared second buffer.  In host code this name is only a stand-in for
// the device object: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_twin[kNoallocBytes];

std::mutex g_mu;
void* g_twin_addr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once per device).
cudaError_t twin_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_twin_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_twin);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        g_twin_addr[dev] = p;
    }
    *out = g_twin_addr[dev];
    return cudaSuccess;
}

pcot_status st_of(cudaError_t e) { return e == cudaSuccess ? PCOT_OK : PCOT_ERR_CUDA; }

}  // namespace

extern "C" pcot_status pcot_run_noalloc(pcot_handle h, void* grid, const int64_t* sizes, const int64_t* strides,
                                        int64_t T, pcot_dtype dtype, pcot_schedule schedule,
                                        const pcot_tile_params* params, void* stream) {
    if (!h || !grid || !sizes || T < 0) return PCOT_ERR_INVALID_ARG;
    if (dtype != PCOT_F32 && dtype != PCOT_F64 && dtype != PCOT_F64_EXACT) return PCOT_ERR_INVALID_ARG;
    if (schedule != PCOT_SWEEP && schedule != PCOT_SLT) return PCOT_ERR_UNSUPPORTED;
    int dims = 0, periodic = 0;
    double c[7];
    pcot_status st = pcot::handle_describe(h, &dims, &periodic, c);
    if (st != PCOT_OK) return st;
    LaunchCtx L;
    std::memset(&L, 0, sizeof(L));
    L.dtype = (int)dtype;
    L.stream = (cudaStream_t)stream;
    DevGeo& g = L.geo;
    g.dims = dims;
    g.periodic = periodic;
    for (int a = 0; a < kMaxDims; ++a) {
        g.e[a] = 1;
        g.n[a] = 1;
        g.s[a] = 0;
    }
    for (int a = 0; a < dims; ++a) {
        if (sizes[a] < 1 || sizes[a] > ((int64_t)1 << 40)) return PCOT_ERR_INVALID_ARG;
        if (periodic && sizes[a] < 3) return PCOT_ERR_UNSUPPORTED;
        g.n[a] = sizes[a];
        g.e[a] = periodic ? sizes[a] : sizes[a] + 2;
    }
    int64_t s = 1;
    for (int a = dims - 1; a >= 0; --a) {
        if (strides) {
            if (a == dims - 1 && strides[a] != 1) return PCOT_ERR_UNSUPPORTED;
            if (strides[a] < s) return PCOT_ERR_INVALID_ARG;
            g.s[a] = strides[a];
        } else {
            g.s[a] = s;
        }
        s = g.s[a] * g.e[a];
    }
    for (int i = 0; i < 7; ++i) L.coeffs[i] = c[i];
    const int es = dtype == PCOT_F32 ? 4 : 8;
    if (((uintptr_t)grid % es) != 0) return PCOT_ERR_ALIGNMENT;
    int64_t last = 0;
    for (int a = 0; a < dims; ++a) last += (g.e[a] - 1) * g.s[a];
    const size_t span = (size_t)(last + 1) * es;
    if (span > kNoallocBytes) return PCOT_ERR_OOM;  // grid larger than the fixed buffer
    if (T == 0) return PCOT_OK;

    void* twin = nullptr;
    cudaError_t e = twin_address(&twin);
    if (e != cudaSuccess) return PCOT_ERR_CUDA;
    int64_t nl = 0;
    if (!periodic) {
        e = launch_ring_copy(L, grid, twin);  // the array keeps earlier contents: set the ring now
        if (e != cudaSuccess) return PCOT_ERR_CUDA;
        ++nl;
    }
    void* cur = grid;
    void* other = twin;
    if (schedule == PCOT_SWEEP) {
        for (int64_t t = 0; t < T; ++t) {
            e = launch_sweep(L, cur, other);
            if (e != cudaSuccess) return PCOT_ERR_CUDA;
            ++nl;
            void* tmp = cur;
            cur = other;
            other = tmp;
        }
    } else {
        // Time blocks: depth k while possible, the remainder in the deepest
        // compiled depths (no heap).  An odd block count ends in the array
        // and is copied back below.  k follows pcot_run's rules: the default
        // depth, and a depth without a kernel falls to the deepest compiled
        // one below it.
        const int k = resolve_depth(L, params ? params->tile : nullptr,
                                    params && params->time_depth > 0 ? params->time_depth : default_depth(L));
        TileGeo tg;
        int fam_depths[32];
        if (!choose_tiles(L, params ? params->tile : nullptr, k, &tg)) return PCOT_ERR_UNSUPPORTED;
        const int nd = tg.family == kFamGeneric ? 0 : supported_depths(tg.family, L.dtype, fam_depths, 32);
        auto deepest = [&](int64_t limit) {
            if (nd == 0) return (int)(limit < 64 ? limit : 64);
            int best = 1;
            for (int i = 0; i < nd; ++i)
                if (fam_depths[i] <= limit && fam_depths[i] > best) best = fam_depths[i];
            return best;
        };
        int64_t left = T;
        while (left > 0) {
            const int d = left >= k ? k : deepest(left);
            if (!choose_tiles(L, params ? params->tile : nullptr, d, &tg)) return PCOT_ERR_UNSUPPORTED;
            e = launch_slt_block(L, tg, cur, other, nullptr);  // no status block: plain-load tiles
            if (e != cudaSuccess) return PCOT_ERR_CUDA;
            ++nl;
            void* tmp = cur;
            cur = other;
            other = tmp;
            left -= d;
        }
    }
    if (cur != grid) {
        // Only the stored cells go back: the row padding of a strided grid
        // belongs to the caller and is never written.
        e = launch_grid_copy(L, cur, grid);
        if (e != cudaSuccess) return PCOT_ERR_CUDA;
    }
    pcot::handle_count_launches(h, nl);
    return st_of(cudaGetLastError());
}
