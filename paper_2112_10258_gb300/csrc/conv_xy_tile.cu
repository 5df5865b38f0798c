// Single-volume y/x passes over 64x32 tiles, for rows wider than 256 (the
// tile body is conv_xy_tile in conv_tile.cuh; conv.cu has the overview).
#include "conv_body.cuh"

namespace sift3d {

namespace {

using namespace conv_detail;

template <int R, typename Tin, bool SUB, typename Tbase>
__global__ void __launch_bounds__(XY_THREADS) conv_xy_kernel(const ConvXYArgs a) {
    extern __shared__ float sm[];
    conv_xy_tile<R, Tin, SUB, Tbase>(a, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

template <typename Tin, bool SUB, typename Tbase, int... Rs>
const void* xy_func_table(int r, int* smem, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_xy_kernel<Rs + 1, Tin, SUB, Tbase>)...};
    const int sm[] = {XYGeom<Rs + 1>::SMEM...};
    *smem = sm[r - 1];
    return fns[r - 1];
}

template <typename Tin, bool SUB, typename Tbase>
const void* xy_func(int r, int* smem) {
    return xy_func_table<Tin, SUB, Tbase>(r, smem, RadiusSeq{});
}

}  // namespace

LaunchSpec conv_xy_tile_spec(int radius, int src_kind, int storage, bool sub, const ConvXYArgs& a) {
    LaunchSpec s;
    int smem = 0;
    if (radius < 1 || radius > kMaxRadius) return s;
    if (!sub) {
        if (src_kind == 0) s.func = xy_func<float, false, float>(radius, &smem);
        else if (src_kind == 1) s.func = xy_func<uint8_t, false, float>(radius, &smem);
        else if (storage == SIFT3D_STORAGE_F32) s.func = xy_func<float, false, float>(radius, &smem);
        else if (storage == SIFT3D_STORAGE_F16) s.func = xy_func<__half, false, float>(radius, &smem);
        else s.func = xy_func<__nv_bfloat16, false, float>(radius, &smem);
    } else {
        if (storage == SIFT3D_STORAGE_F32) s.func = xy_func<float, true, float>(radius, &smem);
        else if (storage == SIFT3D_STORAGE_F16) s.func = xy_func<__half, true, __half>(radius, &smem);
        else s.func = xy_func<__nv_bfloat16, true, __nv_bfloat16>(radius, &smem);
    }
    s.grid = dim3((a.nx + XY_TX - 1) / XY_TX, (a.ny + XY_TY - 1) / XY_TY, a.nz);
    s.block = dim3(XY_THREADS);
    s.smem = smem;
    s.name = sub ? "conv_xy_sub" : "conv_xy";
    return s;
}

}  // namespace sift3d
