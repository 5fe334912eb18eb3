// Dispatch from (dims, dtype, depth) to a kernel family.
#include "tiled.cuh"

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

cudaError_t launch_slt_block(const LaunchCtx& L, const TileGeo& t, const void* src, void* dst) {
    switch (t.family) {
        case kFamStream2D: return stream2d::slt(L, t, src, dst);
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

}  // namespace pcot
