// Single-volume z passes of the separable Gaussian (Sec. 2.2.2 "Gaussian
// Convolution"): the register-window column pass with the DoG epilogue, and
// the level-S variant that also writes the next octave's G_0.  The bodies are
// in conv_body.cuh; conv.cu has the overview.
#include "conv_body.cuh"

namespace sift3d {

namespace {

using namespace conv_detail;

// TZ outputs per thread: 16, or 8 (float32 storage) where the autotuner finds
// the shorter column faster; every output is the same chain either way.
template <int R, typename S, int RB, int TZ>
__global__ void __launch_bounds__(Z_THREADS) conv_z_kernel(const ConvZArgs a) {
    z_body<R, S, RB, ConvZArgs, TZ>(a, a.taps, a.taps2, blockIdx.x, blockIdx.y);
}

// z pass of level S (float32 storage, rows up to 256 wide) that also writes
// the next octave's G_0 (Sec. 2.2.2 "Sub-sampling": the mean of each 2x2x2
// block of G_S; a trailing odd voxel on an axis is dropped).  A CTA owns rows
// 2rp and 2rp+1 of a z tile (its py threads are the two rows' column pairs),
// parks its G_S values in shared memory and averages the blocks in the order
// (z, y, x), (z, y, x+1), (z, y+1, x), (z, y+1, x+1), then the same in z+1 -- the
// order of the sub-sampling y/x pass -- so the next octave gets the same bits
// without reading G_S back.
template <int R>
__global__ void __launch_bounds__(ROW_MAX_NX) conv_z_sub_kernel(const ConvZArgs a) {
    extern __shared__ __align__(16) float2 gsz[];   // [Z_TZ][py] G_S of the CTA's two rows
    const int rp = blockIdx.x, zt = blockIdx.y, t = threadIdx.x;
    const int py = (int)a.py;                       // = blockDim.x
    const int64_t pz2 = a.pz / 2;
    const int64_t pair = (int64_t)rp * py + t;      // rows 2rp, 2rp+1 hold py pairs
    const int z0 = zt * Z_TZ;
    if (pair < pz2) {   // the second row of an odd last row pair does not exist
        const bool interior = z0 - R >= 0 && z0 + Z_TZ + R <= a.nz;
        float2 v[Z_TZ + 2 * R];
        load_z_window<Z_TZ + 2 * R, R>(reinterpret_cast<const float2*>(a.src) + pair, pz2, z0, a.nz, interior, v);
        float2 pv[Z_TZ];
        const float2* prev = static_cast<const float2*>(a.prev) + pair;
#pragma unroll
        for (int j = 0; j < Z_TZ; ++j) pv[j] = prev[(int64_t)min(z0 + j, a.nz - 1) * pz2];
        float2* dst = static_cast<float2*>(a.dst) + pair + (int64_t)z0 * pz2;
        float2* dog = reinterpret_cast<float2*>(a.dog) + pair + (int64_t)z0 * pz2;
#pragma unroll
        for (int j = 0; j < Z_TZ; ++j) {
            if (z0 + j >= a.nz) break;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = -R; k <= R; ++k) acc = __ffma2_rn(f2(a.taps.w[k < 0 ? -k : k]), v[j + R + k], acc);
            *dst = acc;
            *dog = make_float2(pv[j].x - acc.x, pv[j].y - acc.y);
            gsz[j * py + t] = acc;
            dst += pz2;
            dog += pz2;
        }
    }
    __syncthreads();
    const int nxs = a.nx / 2, nys = a.ny / 2, nzs = a.nz / 2;
    if (rp >= nys) return;
    const int zo0 = z0 / 2;
    const int nzo = min(Z_TZ / 2, nzs - zo0);
    const int half = py / 2;   // pairs per row
    for (int item = t; item < nzo * nxs; item += blockDim.x) {
        const int k = item / nxs, xo = item - k * nxs;
        const float2 a0 = gsz[2 * k * py + xo], a1 = gsz[2 * k * py + half + xo];
        const float2 b0 = gsz[(2 * k + 1) * py + xo], b1 = gsz[(2 * k + 1) * py + half + xo];
        float m = 0.f;
        m += a0.x;
        m += a0.y;
        m += a1.x;
        m += a1.y;
        m += b0.x;
        m += b0.y;
        m += b1.x;
        m += b1.y;
        a.sub_dst[(int64_t)(zo0 + k) * a.sub_pz + (int64_t)rp * a.sub_py + xo] = m * 0.125f;
    }
}

template <int... Rs>
const void* z_sub_func_table(int r, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_sub_kernel<Rs + 1>)...};
    return fns[r - 1];
}

template <typename S, int... Rs>
const void* z_func_table(int r, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_kernel<Rs + 1, S, 0, Z_TZ>)...};
    return fns[r - 1];
}

template <int... Rs>
const void* z_func_table_short(int r, std::integer_sequence<int, Rs...>) {   // float32, 8 outputs per thread
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_kernel<Rs + 1, float, 0, 8>)...};
    return fns[r - 1];
}

}  // namespace

LaunchSpec conv_z_spec(int radius, int storage, const ConvZArgs& a) {
    LaunchSpec s;
    if (radius < 1 || radius > kMaxRadius) return s;
    if (a.dst2 != nullptr) return s;   // the fused descriptor pre-blur exists in the batched kernels only
    if (a.sub_dst != nullptr) {        // level S writing the next octave's G_0
        if (storage != SIFT3D_STORAGE_F32 || a.dog == nullptr || a.py > ROW_MAX_NX || a.py % 2 != 0) return s;
        s.func = z_sub_func_table(radius, RadiusSeq{});
        s.grid = dim3((unsigned)((a.ny + 1) / 2), (a.nz + Z_TZ - 1) / Z_TZ, 1);
        s.block = dim3((unsigned)a.py);
        s.smem = (size_t)Z_TZ * a.py * sizeof(float2);
        s.name = "conv_z_dog_sub";
        return s;
    }
    const int tz = storage == SIFT3D_STORAGE_F32 && a.z_tile == 8 ? 8 : Z_TZ;
    if (storage == SIFT3D_STORAGE_F32) {
        s.func = tz == 8 ? z_func_table_short(radius, RadiusSeq{}) : z_func_table<float>(radius, RadiusSeq{});
    } else if (storage == SIFT3D_STORAGE_F16) {
        s.func = z_func_table<__half>(radius, RadiusSeq{});
    } else {
        s.func = z_func_table<__nv_bfloat16>(radius, RadiusSeq{});
    }
    s.grid = dim3((unsigned)((a.pz / 2 + Z_THREADS - 1) / Z_THREADS), (a.nz + tz - 1) / tz, 1);
    s.block = dim3(Z_THREADS);
    s.smem = 0;
    s.name = a.dog ? "conv_z_dog" : "conv_z";
    return s;
}

}  // namespace sift3d
