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
//   conv_z   one thread per two adjacent columns and TZ outputs along z: the
//            TZ + 2R inputs are loaded into registers (clamped z) and the TZ
//            outputs accumulate from registers.  The epilogue stores G_s and the
//            difference of Gaussians D_{s-1} = G_{s-1} - G_s (Sec. 2.2.2
//            "Difference-of-Gaussian") so the DoG costs no extra pass.
//
// Every 1D pass is out[i] = sum_{k=-R..R} w_|k| in[clamp(i+k)], summed in
// ascending k, in float32.
#include "conv_tile.cuh"

namespace sift3d {

namespace {

using namespace conv_detail;

template <int R, typename Tin, bool SUB, typename Tbase>
__global__ void __launch_bounds__(XY_THREADS) conv_xy_kernel(const ConvXYArgs a) {
    extern __shared__ float sm[];
    pdl_launch_dependents();
    pdl_wait();
    conv_xy_tile<R, Tin, SUB, Tbase>(a, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

// RB > 0: also filter the staged plane with the descriptor pre-blur (radius
// RB <= R, taps2) into dst2, reusing the staged rows.
template <int R, int TY, typename Tin, bool SUB, typename Tbase, int RB>
__global__ void __launch_bounds__(ROW_MAX_NX) conv_xy_row_kernel(const ConvXYArgs a) {
    static_assert(RB <= R, "the fused pre-blur reads inside the staged halo");
    extern __shared__ float sm[];
    pdl_launch_dependents();
    pdl_wait();
    const int nx = a.nx;
    const int WP = row_pitch(nx);
    float* in = sm;                          // (TY + 2R) x WP
    float* mid = sm + (TY + 2 * R) * WP;     // TY x WP
    float* mid2 = mid + TY * WP;             // TY x WP (RB > 0)
    const int y0 = blockIdx.x * TY;
    const int z = blockIdx.y;
    const int c = threadIdx.x;
    const Tin* src = static_cast<const Tin*>(a.src);
    if (a.zero_count != nullptr && y0 == 0 && z == 0 && c < kDetectCounters) a.zero_count[c] = 0;

    if (c < nx) {
        float v[TY + 2 * R];
#pragma unroll
        for (int r = 0; r < TY + 2 * R; ++r) {
            const int gy = min(max(y0 - R + r, 0), a.ny - 1);
            v[r] = stage_value<Tin, SUB>(a, src, z, gy, c);
        }
        if constexpr (SUB) {   // this CTA's own rows of the sub-sampled level are G_0
#pragma unroll
            for (int r = 0; r < TY; ++r)
                if (y0 + r < a.ny)
                    static_cast<Tbase*>(a.base_out)[(int64_t)z * a.pz + (int64_t)(y0 + r) * a.py + c] =
                        from_f32<Tbase>(v[R + r]);
        }
        // y pass straight from the register window
#pragma unroll
        for (int j = 0; j < TY; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int k = -R; k <= R; ++k) acc = fmaf(a.taps.w[k < 0 ? -k : k], v[j + R + k], acc);
            mid[j * WP + c] = acc;
        }
        if constexpr (RB > 0) {
#pragma unroll
            for (int j = 0; j < TY; ++j) {
                float acc = 0.f;
#pragma unroll
                for (int k = -RB; k <= RB; ++k) acc = fmaf(a.taps2.w[k < 0 ? -k : k], v[j + R + k], acc);
                mid2[j * WP + c] = acc;
            }
        }
    }
    __syncthreads();

    // x pass: item = (row r, group g of 8 columns), r fastest so a warp's lanes
    // read different rows (odd pitch: no bank conflicts)
    const int groups = (nx + ROW_J - 1) / ROW_J;
    for (int item = threadIdx.x; item < TY * groups; item += blockDim.x) {
        const int r = item % TY;
        const int g = item / TY;
        const int y = y0 + r;
        if (y >= a.ny) continue;
        const int x0 = g * ROW_J;
        float v[ROW_J + 2 * R];
#pragma unroll
        for (int t = 0; t < ROW_J + 2 * R; ++t) v[t] = mid[r * WP + min(max(x0 - R + t, 0), nx - 1)];
        float o[ROW_J];
#pragma unroll
        for (int j = 0; j < ROW_J; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int k = -R; k <= R; ++k) acc = fmaf(a.taps.w[k < 0 ? -k : k], v[j + R + k], acc);
            o[j] = acc;
        }
        float* dst = a.dst + (int64_t)z * a.pz + (int64_t)y * a.py + x0;
        reinterpret_cast<float4*>(dst)[0] = make_float4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(o[4], o[5], o[6], o[7]);
        if constexpr (RB > 0) {
            float u[ROW_J + 2 * RB];
#pragma unroll
            for (int t = 0; t < ROW_J + 2 * RB; ++t) u[t] = mid2[r * WP + min(max(x0 - RB + t, 0), nx - 1)];
#pragma unroll
            for (int j = 0; j < ROW_J; ++j) {
                float acc = 0.f;
#pragma unroll
                for (int k = -RB; k <= RB; ++k) acc = fmaf(a.taps2.w[k < 0 ? -k : k], u[j + RB + k], acc);
                o[j] = acc;
            }
            float* dst2 = a.dst2 + (int64_t)z * a.pz + (int64_t)y * a.py + x0;
            reinterpret_cast<float4*>(dst2)[0] = make_float4(o[0], o[1], o[2], o[3]);
            reinterpret_cast<float4*>(dst2)[1] = make_float4(o[4], o[5], o[6], o[7]);
        }
    }
}

template <int R, typename S, int RB>
__global__ void __launch_bounds__(Z_THREADS) conv_z_kernel(const ConvZArgs a) {
    pdl_launch_dependents();
    pdl_wait();
    conv_z_column<R, S, false, RB>(a, (int64_t)blockIdx.x * Z_THREADS + threadIdx.x, blockIdx.y * Z_TZ);
}

// ---- dispatch tables over the radius -------------------------------------
template <typename Tin, bool SUB, typename Tbase, int... Rs>
const void* xy_func_table(int r, int* smem, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_xy_kernel<Rs + 1, Tin, SUB, Tbase>)...};
    const int sm[] = {XYGeom<Rs + 1>::SMEM...};
    *smem = sm[r - 1];
    return fns[r - 1];
}

template <int TY, typename Tin, bool SUB, typename Tbase, int... Rs>
const void* row_func_table(int r, int nx, int* smem, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_xy_row_kernel<Rs + 1, TY, Tin, SUB, Tbase, 0>)...};
    const int sm[] = {row_smem_bytes<Rs + 1, TY>(nx)...};
    *smem = sm[r - 1];
    return fns[r - 1];
}

// Fused pre-blur variants exist for radii >= kFusedBlurRadius (index r-RB).
template <int TY, typename Tin, int... Rs>
const void* row_blur_func_table(int r, int nx, int* smem, std::integer_sequence<int, Rs...>) {
    constexpr int RB = kFusedBlurRadius;
    const void* fns[] = {
        reinterpret_cast<const void*>(&conv_xy_row_kernel<Rs + RB, TY, Tin, false, float, RB>)...};
    const int sm[] = {(row_smem_bytes<Rs + RB, TY>(nx) + TY * row_pitch(nx) * 4)...};
    if (r < RB) return nullptr;
    *smem = sm[r - RB];
    return fns[r - RB];
}

template <typename S, int... Rs>
const void* z_func_table(int r, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_kernel<Rs + 1, S, 0>)...};
    return fns[r - 1];
}

template <typename S, int... Rs>
const void* z_blur_func_table(int r, std::integer_sequence<int, Rs...>) {
    constexpr int RB = kFusedBlurRadius;
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_kernel<Rs + RB, S, RB>)...};
    if (r < RB) return nullptr;
    return fns[r - RB];
}

using BlurRadiusSeq = std::make_integer_sequence<int, kMaxRadius - kFusedBlurRadius + 1>;

using RadiusSeq = std::make_integer_sequence<int, kMaxRadius>;

template <typename Tin, bool SUB, typename Tbase>
const void* xy_func(int r, int* smem) {
    return xy_func_table<Tin, SUB, Tbase>(r, smem, RadiusSeq{});
}

constexpr int ROW_TY = 16;

template <typename Tin, bool SUB, typename Tbase>
const void* row_func(int r, int nx, int* smem) {
    return row_func_table<ROW_TY, Tin, SUB, Tbase>(r, nx, smem, RadiusSeq{});
}

}  // namespace

LaunchSpec conv_xy_spec(int radius, int src_kind, int storage, bool sub, const ConvXYArgs& a) {
    LaunchSpec s;
    int smem = 0;
    if (radius < 1 || radius > kMaxRadius) return s;
    if (a.dst2 != nullptr) {   // level pass with the descriptor pre-blur fused in
        if (sub || src_kind != 2 || a.nx > ROW_MAX_NX) return s;
        if (storage == SIFT3D_STORAGE_F32) s.func = row_blur_func_table<ROW_TY, float>(radius, a.nx, &smem, BlurRadiusSeq{});
        else if (storage == SIFT3D_STORAGE_F16) s.func = row_blur_func_table<ROW_TY, __half>(radius, a.nx, &smem, BlurRadiusSeq{});
        else s.func = row_blur_func_table<ROW_TY, __nv_bfloat16>(radius, a.nx, &smem, BlurRadiusSeq{});
        if (s.func == nullptr) return s;
        if (smem > 48 * 1024) cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        s.grid = dim3((a.ny + ROW_TY - 1) / ROW_TY, a.nz, 1);
        s.block = dim3((a.nx + 31) / 32 * 32);
        s.smem = smem;
        s.name = "conv_xy_blur";
        return s;
    }
    if (a.nx <= ROW_MAX_NX) {
        if (!sub) {
            if (src_kind == 0) s.func = row_func<float, false, float>(radius, a.nx, &smem);
            else if (src_kind == 1) s.func = row_func<uint8_t, false, float>(radius, a.nx, &smem);
            else if (storage == SIFT3D_STORAGE_F32) s.func = row_func<float, false, float>(radius, a.nx, &smem);
            else if (storage == SIFT3D_STORAGE_F16) s.func = row_func<__half, false, float>(radius, a.nx, &smem);
            else s.func = row_func<__nv_bfloat16, false, float>(radius, a.nx, &smem);
        } else {
            if (storage == SIFT3D_STORAGE_F32) s.func = row_func<float, true, float>(radius, a.nx, &smem);
            else if (storage == SIFT3D_STORAGE_F16) s.func = row_func<__half, true, __half>(radius, a.nx, &smem);
            else s.func = row_func<__nv_bfloat16, true, __nv_bfloat16>(radius, a.nx, &smem);
        }
        if (smem > 48 * 1024) cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        s.grid = dim3((a.ny + ROW_TY - 1) / ROW_TY, a.nz, 1);
        s.block = dim3((a.nx + 31) / 32 * 32);
        s.smem = smem;
        s.name = sub ? "conv_xy_sub" : "conv_xy";
        return s;
    }
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

LaunchSpec conv_z_spec(int radius, int storage, const ConvZArgs& a) {
    LaunchSpec s;
    if (radius < 1 || radius > kMaxRadius) return s;
    if (a.dst2 != nullptr) {
        if (storage == SIFT3D_STORAGE_F32) s.func = z_blur_func_table<float>(radius, BlurRadiusSeq{});
        else if (storage == SIFT3D_STORAGE_F16) s.func = z_blur_func_table<__half>(radius, BlurRadiusSeq{});
        else s.func = z_blur_func_table<__nv_bfloat16>(radius, BlurRadiusSeq{});
    } else if (storage == SIFT3D_STORAGE_F32) s.func = z_func_table<float>(radius, RadiusSeq{});
    else if (storage == SIFT3D_STORAGE_F16) s.func = z_func_table<__half>(radius, RadiusSeq{});
    else s.func = z_func_table<__nv_bfloat16>(radius, RadiusSeq{});
    s.grid = dim3((unsigned)((a.pz + Z_THREADS - 1) / Z_THREADS), (a.nz + Z_TZ - 1) / Z_TZ, 1);
    s.block = dim3(Z_THREADS);
    s.smem = 0;
    s.name = a.dst2 ? "conv_z_dog_blur" : (a.dog ? "conv_z_dog" : "conv_z");
    return s;
}

}  // namespace sift3d
