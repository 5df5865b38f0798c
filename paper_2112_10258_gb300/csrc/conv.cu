// Separable 3D Gaussian convolution for sm_103a (Sec. 2.2.2 "Gaussian
// Convolution": three 1D passes in x, y and z), split in two kernels:
//
//   conv_xy  one CTA per 64x32 output tile of one z plane.  The tile plus a
//            radius-R halo is staged in shared memory with clamp-to-edge
//            indices, filtered along y, then along x, and written as float32
//            to an intermediate volume that stays resident in L2 for conv_z.
//            In sub-sample mode the staged values are the 2x2x2 means of the
//            previous octave's level S (Sec. 2.2.2 "Sub-sampling"), and the
//            tile's own means are written out as the octave's G_0.
//   conv_xy_row  (rows up to 256 wide) one CTA per 8 or 16 full rows of a
//            plane, column pairs in the y pass and row pairs in the x pass, each
//            tap one paired FP32 FMA (see below).
//   conv_z   one thread per two adjacent columns and TZ outputs along z: the
//            TZ + 2R inputs are loaded into registers (clamped z) and the TZ
//            outputs accumulate from registers.  The epilogue stores G_s and the
//            difference of Gaussians D_{s-1} = G_{s-1} - G_s (Sec. 2.2.2
//            "Difference-of-Gaussian") so the DoG costs no extra pass; at level S
//            (float32 storage) a variant also writes the next octave's G_0.
//   *_batch  the same bodies over the tiles of many volumes in one launch.
//
// Every 1D pass is out[i] = sum_{k=-R..R} w_|k| in[clamp(i+k)], summed in
// ascending k, in float32.
//
// This unit instantiates the single-volume y/x passes of full rows;
// conv_xy_tile.cu the 64x32-tile ones, conv_z.cu the z passes, conv_batch.cu
// the batched ones; the device bodies are in conv_body.cuh.
#include "conv_body.cuh"

namespace sift3d {

namespace {

using namespace conv_detail;

template <int R, int MODE, typename Tin, typename Tbase, int RB>
__global__ void __launch_bounds__(ROW_MAX_NX) conv_xy_row_kernel(const ConvXYArgs a) {
    extern __shared__ __align__(16) float2 rows_sm[];
    row_body<R, MODE, Tin, Tbase, RB, ConvXYArgs>(a, a.taps, a.taps2, blockIdx.x, blockIdx.y, rows_sm);
}

template <int MODE, typename Tin, typename Tbase, int... Rs>
const void* row_func_table(int r, int nx, int ty, int* smem, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_xy_row_kernel<Rs + 1, MODE, Tin, Tbase, 0>)...};
    *smem = row_smem(nx, r, 0, ty);
    return fns[r - 1];
}

template <int MODE, typename Tin, typename Tbase>
const void* row_func(int r, int nx, int ty, int* smem) {
    return row_func_table<MODE, Tin, Tbase>(r, nx, ty, smem, RadiusSeq{});
}

}  // namespace

LaunchSpec conv_xy_spec(int radius, int src_kind, int storage, bool sub, ConvXYArgs& a) {
    LaunchSpec s;
    int smem = 0;
    if (radius < 1 || radius > kMaxRadius) return s;
    if (a.row_tile != 8 && a.row_tile != 16) a.row_tile = ROW_TY;
    const int ty = a.row_tile;
    if (a.dst2 != nullptr) return s;   // the fused descriptor pre-blur exists in the batched kernels only
    if (a.nx <= ROW_MAX_NX) {
        if (!sub) {
            if (src_kind == 0) s.func = row_func<1, float, float>(radius, a.nx, ty, &smem);
            else if (src_kind == 1) s.func = row_func<1, uint8_t, float>(radius, a.nx, ty, &smem);
            else if (storage == SIFT3D_STORAGE_F32) s.func = row_func<0, float, float>(radius, a.nx, ty, &smem);
            else if (storage == SIFT3D_STORAGE_F16) s.func = row_func<0, __half, float>(radius, a.nx, ty, &smem);
            else s.func = row_func<0, __nv_bfloat16, float>(radius, a.nx, ty, &smem);
        } else {
            if (storage == SIFT3D_STORAGE_F32) s.func = row_func<2, float, float>(radius, a.nx, ty, &smem);
            else if (storage == SIFT3D_STORAGE_F16) s.func = row_func<2, __half, __half>(radius, a.nx, ty, &smem);
            else s.func = row_func<2, __nv_bfloat16, __nv_bfloat16>(radius, a.nx, ty, &smem);
        }
        if (smem > 48 * 1024) cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        s.grid = dim3((a.ny + ty - 1) / ty, a.nz, 1);
        s.block = dim3(row_threads(a.nx, ty));
        s.smem = smem;
        s.name = sub ? "conv_xy_sub" : "conv_xy";
        return s;
    }
    return conv_xy_tile_spec(radius, src_kind, storage, sub, a);   // rows wider than 256: conv_xy_tile.cu
}

}  // namespace sift3d
