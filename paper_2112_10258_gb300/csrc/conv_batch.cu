// Batched y/x and z passes over the tiles of many volumes in one launch
// (sift3d_detect_batch); every volume's pointers and dims travel in the kernel
// parameters.  The bodies are in conv_body.cuh; conv.cu has the overview.
#include "conv_body.cuh"

namespace sift3d {

namespace {

using namespace conv_detail;

// Batched: one flat list of (volume, column block, z tile) items.
template <int R, typename S, int RB>
__global__ void __launch_bounds__(Z_THREADS) conv_z_batch(const __grid_constant__ BatchZ b) {
    {
        const int item = blockIdx.x;
        const int v = batch_param_volume(b.prefix, b.n, item);
        const ZVol& a = b.vol[v];   // read in place from the kernel parameters
        const int local = item - b.prefix[v];
        const int cols = (int)((a.pz / 2 + Z_THREADS - 1) / Z_THREADS);
        z_body<R, S, RB, ZVol>(a, b.taps, b.taps2, local % cols, local / cols);
    }
}

// Batched: the CTAs walk the tiles of every volume of the batch (grid-stride
// over one flat tile list; a tile's volume is found in the prefix sums).
template <int R, int MODE, typename Tin, typename Tbase, int RB>
__global__ void __launch_bounds__(ROW_MAX_NX) conv_xy_row_batch(const __grid_constant__ BatchXY b) {
    extern __shared__ __align__(16) float2 rows_sm[];
    {
        const int item = blockIdx.x;
        const int v = batch_param_volume(b.prefix, b.n, item);
        const XYVol& a = b.vol[v];   // read in place from the kernel parameters
        const int local = item - b.prefix[v];
        const int nyb = (a.ny + a.row_tile - 1) / a.row_tile;
        row_body<R, MODE, Tin, Tbase, RB, XYVol>(a, b.taps, b.taps2, local % nyb, local / nyb, rows_sm);
    }
}

// Batched instances: float32 storage (float32 or uint8 input).
template <int MODE, typename Tin, int... Rs>
const void* row_batch_table(int r, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_xy_row_batch<Rs + 1, MODE, Tin, float, 0>)...};
    return fns[r - 1];
}

template <int... Rs>
const void* row_blur_batch_table(int r, std::integer_sequence<int, Rs...>) {
    constexpr int RB = kFusedBlurRadius;
    const void* fns[] = {reinterpret_cast<const void*>(&conv_xy_row_batch<Rs + RB, 0, float, float, RB>)...};
    return r < RB ? nullptr : fns[r - RB];
}

template <int... Rs>
const void* z_batch_table(int r, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_batch<Rs + 1, float, 0>)...};
    return fns[r - 1];
}

template <int... Rs>
const void* z_blur_batch_table(int r, std::integer_sequence<int, Rs...>) {
    constexpr int RB = kFusedBlurRadius;
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_batch<Rs + RB, float, RB>)...};
    return r < RB ? nullptr : fns[r - RB];
}

}  // namespace

LaunchSpec conv_xy_batch_spec(int radius, int src_kind, bool sub, bool blur, int nx_max, int row_tile, int total) {
    LaunchSpec s;
    if (radius < 1 || radius > kMaxRadius || nx_max > ROW_MAX_NX) return s;
    const int ty = row_tile;
    if (blur) {
        if (sub || src_kind != 2) return s;
        s.func = row_blur_batch_table(radius, BlurRadiusSeq{});
    } else if (sub) {
        s.func = row_batch_table<2, float>(radius, RadiusSeq{});
    } else if (src_kind == 0) {
        s.func = row_batch_table<1, float>(radius, RadiusSeq{});
    } else if (src_kind == 1) {
        s.func = row_batch_table<1, uint8_t>(radius, RadiusSeq{});
    } else {
        s.func = row_batch_table<0, float>(radius, RadiusSeq{});
    }
    if (s.func == nullptr) return s;
    const int smem = row_smem(nx_max, radius, blur ? kFusedBlurRadius : 0, ty);
    if (smem > 48 * 1024) cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    s.block = dim3(row_threads(nx_max, ty));
    s.smem = smem;
    s.grid = dim3((unsigned)std::max(1, total));   // one tile per CTA
    s.name = blur ? "conv_xy_blur_batch" : (sub ? "conv_xy_sub_batch" : "conv_xy_batch");
    return s;
}

LaunchSpec conv_z_batch_spec(int radius, bool blur, int total) {
    LaunchSpec s;
    if (radius < 1 || radius > kMaxRadius) return s;
    s.func = blur ? z_blur_batch_table(radius, BlurRadiusSeq{}) : z_batch_table(radius, RadiusSeq{});
    if (s.func == nullptr) return s;
    s.block = dim3(Z_THREADS);
    s.grid = dim3((unsigned)std::max(1, total));   // one tile per CTA
    s.name = blur ? "conv_z_dog_blur_batch" : "conv_z_dog_batch";
    return s;
}

// Work items of one volume in a batched pass.
int conv_xy_items(const ConvXYArgs& a) { return ((a.ny + a.row_tile - 1) / a.row_tile) * a.nz; }
int conv_z_items(const ConvZArgs& a) {
    return (int)((a.pz / 2 + Z_THREADS - 1) / Z_THREADS) * ((a.nz + Z_TZ - 1) / Z_TZ);
}

}  // namespace sift3d
