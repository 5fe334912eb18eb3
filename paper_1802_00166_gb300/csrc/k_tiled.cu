// Dispatch from (dims, dtype, depth) to a kernel family.
#include <cudaTypedefs.h>

#include "tiled.cuh"
#include "tma.cuh"

namespace pcot {

bool choose_tiles(const LaunchCtx& L, const int32_t* req, int depth, TileGeo* out) {
    if (L.geo.dims == 2 && stream2d::choose(L, req, depth, out)) return true;
    if (L.geo.dims == 3 && stream3d::choose(L, req, depth, out)) return true;
    return generic::choose(L, req, depth, out);
}

int supported_depths(int family, int dtype, int* out, int cap) {
    if (family == kFamStream2D) return stream2d::depths(dtype, out, cap);
    if (family == kFamStream3D) return stream3d::depths(dtype, out, cap);
    return 0;  // any depth
}

int default_depth(const LaunchCtx& L) {
    if (L.geo.dims == 1) return 16;
    if (L.dtype != kF32) return 1;
    return L.geo.dims == 2 ? 4 : 2;
}

int resolve_depth(const LaunchCtx& L, const int32_t* req_tile, int k) {
    if (k < 1) k = 1;
    TileGeo tg;
    if (choose_tiles(L, req_tile, k, &tg)) return k;
    const int fam = L.geo.dims == 2 ? kFamStream2D : kFamStream3D;
    int ds[32];
    const int n = supported_depths(fam, L.dtype, ds, 32);
    int best = 1;
    for (int i = 0; i < n; ++i)
        if (ds[i] <= k && ds[i] > best) best = ds[i];
    return best;
}

cudaError_t launch_slt_block(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst, DevStatus* st) {
    switch (t.family) {
        case kFamStream2D: return stream2d::slt(L, t, src, dst, st);
        case kFamStream3D: return stream3d::slt(L, t, src, dst);
        default: return generic::slt(L, t, src, dst);
    }
}

cudaError_t launch_cot(const LaunchCtx& L, const TileGeo& t, void* b0, void* b1, const CotDev& q, int nctas) {
    switch (t.family) {
        case kFamStream2D: return stream2d::cot(L, t, b0, b1, q, nctas);
        case kFamStream3D: return stream3d::cot(L, t, b0, b1, q, nctas);
        default: return generic::cot(L, t, b0, b1, q, nctas);
    }
}

int cot_ctas_per_sm(const LaunchCtx& L, const TileGeo& t) {
    switch (t.family) {
        case kFamStream2D: return stream2d::ctas_per_sm(L, t);
        case kFamStream3D: return stream3d::ctas_per_sm(L, t);
        default: return generic::ctas_per_sm(L, t);
    }
}

size_t tile_smem_bytes(const LaunchCtx& L, const TileGeo& t) {
    switch (t.family) {
        case kFamStream2D: return 0;
        case kFamStream3D: return stream3d::smem(L, t);
        default: return generic::smem(L, t);
    }
}

bool encode_tmap_2d(CUtensorMap* map, const void* base, int elem_bytes, uint64_t width, uint64_t height,
                    uint64_t pitch_bytes, uint32_t box_w, uint32_t box_h) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    if (!fn || !base || ((uintptr_t)base & 15) || (pitch_bytes & 15) || box_w > 256 || box_h > 256) return false;
    const cuuint64_t dims[2] = {width, height};
    const cuuint64_t strides[1] = {pitch_bytes};
    const cuuint32_t box[2] = {box_w, box_h};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r =
        fn(map, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
           const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace pcot
