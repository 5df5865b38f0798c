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
#include "common.cuh"

namespace sift3d {

namespace {

constexpr int XY_TX = 64;
constexpr int XY_TY = 32;
constexpr int XY_J = 8;          // outputs per thread in each pass
constexpr int XY_THREADS = 256;
constexpr int Z_TZ = 16;
constexpr int Z_THREADS = 256;

template <int R>
struct XYGeom {
    static constexpr int W = XY_TX + 2 * R;         // staged columns
    static constexpr int H = XY_TY + 2 * R;         // staged rows
    static constexpr int WP = W | 1;                // odd pitch: no bank conflicts
    static constexpr int SMEM = (H + XY_TY) * WP * 4;
};

template <typename T>
__device__ __forceinline__ float load_f(const T* p) { return to_f32(*p); }

template <int R, typename Tin, bool SUB, typename Tbase>
__global__ void __launch_bounds__(XY_THREADS) conv_xy_kernel(const ConvXYArgs a) {
    using G = XYGeom<R>;
    extern __shared__ float sm[];
    float* in = sm;                       // H x WP staged source
    float* mid = sm + G::H * G::WP;       // TY x WP after the y pass
    const int x0 = blockIdx.x * XY_TX;
    const int y0 = blockIdx.y * XY_TY;
    const int z = blockIdx.z;
    const Tin* src = static_cast<const Tin*>(a.src);
    if (a.zero_count != nullptr && x0 == 0 && y0 == 0 && z == 0 && threadIdx.x == 0) *a.zero_count = 0;

    for (int i = threadIdx.x; i < G::H * G::W; i += XY_THREADS) {
        const int r = i / G::W;
        const int c = i - r * G::W;
        const int gy = min(max(y0 - R + r, 0), a.ny - 1);
        const int gx = min(max(x0 - R + c, 0), a.nx - 1);
        float v;
        if constexpr (!SUB) {
            v = load_f(src + (int64_t)z * a.src_pz + (int64_t)gy * a.src_py + gx) * a.src_scale;
        } else {
            const Tin* p = src + (int64_t)(2 * z) * a.src_pz + (int64_t)(2 * gy) * a.src_py + 2 * gx;
            float acc = 0.f;
            acc += load_f(p);
            acc += load_f(p + 1);
            acc += load_f(p + a.src_py);
            acc += load_f(p + a.src_py + 1);
            acc += load_f(p + a.src_pz);
            acc += load_f(p + a.src_pz + 1);
            acc += load_f(p + a.src_pz + a.src_py);
            acc += load_f(p + a.src_pz + a.src_py + 1);
            v = acc * 0.125f;
            const int ty = r - R, tx = c - R;
            if (ty >= 0 && ty < XY_TY && tx >= 0 && tx < XY_TX && y0 + ty < a.ny && x0 + tx < a.nx) {
                static_cast<Tbase*>(a.base_out)[(int64_t)z * a.pz + (int64_t)(y0 + ty) * a.py + x0 + tx] =
                    from_f32<Tbase>(v);
            }
        }
        in[r * G::WP + c] = v;
    }
    __syncthreads();

    // y pass: item = (column c, group of J rows)
    for (int item = threadIdx.x; item < G::W * (XY_TY / XY_J); item += XY_THREADS) {
        const int c = item % G::W;
        const int r0 = (item / G::W) * XY_J;
        float v[XY_J + 2 * R];
#pragma unroll
        for (int t = 0; t < XY_J + 2 * R; ++t) v[t] = in[(r0 + t) * G::WP + c];
#pragma unroll
        for (int j = 0; j < XY_J; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int k = -R; k <= R; ++k) acc = fmaf(a.taps.w[k < 0 ? -k : k], v[j + R + k], acc);
            mid[(r0 + j) * G::WP + c] = acc;
        }
    }
    __syncthreads();

    // x pass: item = (row r, group of J columns); J contiguous outputs per thread
    for (int item = threadIdx.x; item < XY_TY * (XY_TX / XY_J); item += XY_THREADS) {
        const int r = item % XY_TY;
        const int c0 = (item / XY_TY) * XY_J;
        const int y = y0 + r;
        if (y >= a.ny) continue;
        float v[XY_J + 2 * R];
#pragma unroll
        for (int t = 0; t < XY_J + 2 * R; ++t) v[t] = mid[r * G::WP + c0 + t];
        float o[XY_J];
#pragma unroll
        for (int j = 0; j < XY_J; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int k = -R; k <= R; ++k) acc = fmaf(a.taps.w[k < 0 ? -k : k], v[j + R + k], acc);
            o[j] = acc;
        }
        float* dst = a.dst + (int64_t)z * a.pz + (int64_t)y * a.py + x0 + c0;
        // The row pitch is a multiple of 8 elements, so writing the padding
        // columns beyond nx stays inside the row; rows are 32-byte aligned.
        if (x0 + c0 < a.nx) {
            reinterpret_cast<float4*>(dst)[0] = make_float4(o[0], o[1], o[2], o[3]);
            reinterpret_cast<float4*>(dst)[1] = make_float4(o[4], o[5], o[6], o[7]);
        }
    }
}

template <typename S> struct Pair;
template <> struct Pair<float> {
    static __device__ __forceinline__ float2 load(const void* p) { return *static_cast<const float2*>(p); }
    static __device__ __forceinline__ void store(void* p, float a, float b) {
        *static_cast<float2*>(p) = make_float2(a, b);
    }
};
template <> struct Pair<__half> {
    static __device__ __forceinline__ float2 load(const void* p) {
        return __half22float2(*static_cast<const __half2*>(p));
    }
    static __device__ __forceinline__ void store(void* p, float a, float b) {
        *static_cast<__half2*>(p) = __floats2half2_rn(a, b);
    }
};
template <> struct Pair<__nv_bfloat16> {
    static __device__ __forceinline__ float2 load(const void* p) {
        return __bfloat1622float2(*static_cast<const __nv_bfloat162*>(p));
    }
    static __device__ __forceinline__ void store(void* p, float a, float b) {
        *static_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
    }
};

template <int R, typename S>
__global__ void __launch_bounds__(Z_THREADS) conv_z_kernel(const ConvZArgs a) {
    // Columns are addressed linearly inside a plane (pitch layout, padding
    // columns included): the z pass does not care about x/y structure.
    const int64_t col = ((int64_t)blockIdx.x * Z_THREADS + threadIdx.x) * 2;
    if (col >= a.pz) return;
    const int z0 = blockIdx.y * Z_TZ;
    float2 v[Z_TZ + 2 * R];
#pragma unroll
    for (int t = 0; t < Z_TZ + 2 * R; ++t) {
        const int zz = min(max(z0 - R + t, 0), a.nz - 1);
        v[t] = *reinterpret_cast<const float2*>(a.src + (int64_t)zz * a.pz + col);
    }
#pragma unroll
    for (int j = 0; j < Z_TZ; ++j) {
        const int z = z0 + j;
        if (z >= a.nz) break;
        float ax = 0.f, ay = 0.f;
#pragma unroll
        for (int k = -R; k <= R; ++k) {
            const float w = a.taps.w[k < 0 ? -k : k];
            ax = fmaf(w, v[j + R + k].x, ax);
            ay = fmaf(w, v[j + R + k].y, ay);
        }
        const int64_t off = (int64_t)z * a.pz + col;
        Pair<S>::store(static_cast<S*>(a.dst) + off, ax, ay);
        if (a.dog != nullptr) {
            const float2 p = Pair<S>::load(static_cast<const S*>(a.prev) + off);
            Pair<S>::store(static_cast<S*>(a.dog) + off, p.x - ax, p.y - ay);
        }
    }
}

// ---- dispatch tables over the radius -------------------------------------
template <typename Tin, bool SUB, typename Tbase, int... Rs>
const void* xy_func_table(int r, int* smem, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_xy_kernel<Rs + 1, Tin, SUB, Tbase>)...};
    const int sm[] = {XYGeom<Rs + 1>::SMEM...};
    *smem = sm[r - 1];
    return fns[r - 1];
}

template <typename S, int... Rs>
const void* z_func_table(int r, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_kernel<Rs + 1, S>)...};
    return fns[r - 1];
}

using RadiusSeq = std::make_integer_sequence<int, kMaxRadius>;

template <typename Tin, bool SUB, typename Tbase>
const void* xy_func(int r, int* smem) {
    return xy_func_table<Tin, SUB, Tbase>(r, smem, RadiusSeq{});
}

}  // namespace

LaunchSpec conv_xy_spec(int radius, int src_kind, int storage, bool sub, const ConvXYArgs& a) {
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

LaunchSpec conv_z_spec(int radius, int storage, const ConvZArgs& a) {
    LaunchSpec s;
    if (radius < 1 || radius > kMaxRadius) return s;
    if (storage == SIFT3D_STORAGE_F32) s.func = z_func_table<float>(radius, RadiusSeq{});
    else if (storage == SIFT3D_STORAGE_F16) s.func = z_func_table<__half>(radius, RadiusSeq{});
    else s.func = z_func_table<__nv_bfloat16>(radius, RadiusSeq{});
    const int64_t threads = (a.pz + 1) / 2;
    s.grid = dim3((unsigned)((threads + Z_THREADS - 1) / Z_THREADS), (a.nz + Z_TZ - 1) / Z_TZ, 1);
    s.block = dim3(Z_THREADS);
    s.smem = 0;
    s.name = a.dog ? "conv_z_dog" : "conv_z";
    return s;
}

}  // namespace sift3d
