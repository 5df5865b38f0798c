// BRIEF and RRIEF descriptors for sm_103a (Sec. 2.2.3 "FAST 3D Descriptors").
//
// One warp per keypoint.  Lane l owns point pairs k = l and k = l + 32: it reads
// the four trilinear samples I(c + sigma_s p1_k), I(c + sigma_s p2_k) from the
// keypoint's pre-blurred level (clamped coordinates) and forms d_k.  BRIEF is two
// warp ballots of [d_k > 0]; RRIEF gives each d_k its rank among the 64 values
// (ties by lower index) by streaming the other 63 values through warp shuffles.
// The 64-pair pattern sits in shared memory (lanes read different pairs, which
// the constant cache would serialise).
#include "common.cuh"

namespace sift3d {

namespace {

constexpr int DS_THREADS = 256;
constexpr int DS_WARPS = DS_THREADS / 32;

// Split a sample offset t (octave voxels, relative to integer centre c) into a
// clamped base index and fraction; equals floor/frac of clamp(c + t, 0, n-1).
__device__ __forceinline__ void axis_coord(int c, float t, int n, int& i0, int& i1, float& f) {
    const float ft = floorf(t);
    i0 = c + (int)ft;
    f = t - ft;
    if (i0 < 0) {
        i0 = 0;
        f = 0.f;
    } else if (i0 >= n - 1) {
        i0 = n - 1;
        f = 0.f;
    }
    i1 = min(i0 + 1, n - 1);
}

template <typename S>
__device__ __forceinline__ float sample(const DescLevel& L, int cx, int cy, int cz, float tx, float ty,
                                        float tz) {
    int x0, x1, y0, y1, z0, z1;
    float fx, fy, fz;
    axis_coord(cx, tx, L.nx, x0, x1, fx);
    axis_coord(cy, ty, L.ny, y0, y1, fy);
    axis_coord(cz, tz, L.nz, z0, z1, fz);
    const S* p = static_cast<const S*>(L.ptr);
    const int64_t r00 = (int64_t)z0 * L.pz + (int64_t)y0 * L.py, r01 = (int64_t)z0 * L.pz + (int64_t)y1 * L.py;
    const int64_t r10 = (int64_t)z1 * L.pz + (int64_t)y0 * L.py, r11 = (int64_t)z1 * L.pz + (int64_t)y1 * L.py;
    const float gx = 1.f - fx, gy = 1.f - fy, gz = 1.f - fz;
    float v = 0.f;
    v += gz * gy * gx * to_f32(p[r00 + x0]);
    v += gz * gy * fx * to_f32(p[r00 + x1]);
    v += gz * fy * gx * to_f32(p[r01 + x0]);
    v += gz * fy * fx * to_f32(p[r01 + x1]);
    v += fz * gy * gx * to_f32(p[r10 + x0]);
    v += fz * gy * fx * to_f32(p[r10 + x1]);
    v += fz * fy * gx * to_f32(p[r11 + x0]);
    v += fz * fy * fx * to_f32(p[r11 + x1]);
    return v;
}

template <typename S>
__global__ void __launch_bounds__(DS_THREADS) describe_kernel(const DescribeArgs a) {
    __shared__ float pat[SIFT3D_N_PAIRS * 6];
    for (int i = threadIdx.x; i < SIFT3D_N_PAIRS * 6; i += DS_THREADS) pat[i] = a.pattern[i];
    __syncthreads();
    const int n = a.n >= 0 ? a.n : min(*a.n_dev, a.n_cap);
    const int lane = threadIdx.x & 31;
    for (int kp = blockIdx.x * DS_WARPS + (threadIdx.x >> 5); kp < n; kp += gridDim.x * DS_WARPS) {
        const sift3d_keypoint K = a.kps[kp];
        // records that do not name a level of the last detect get no descriptor
        if (K.octave < 0 || K.octave >= a.n_octaves || K.scale < 1 || K.scale > a.n_scales) continue;
        const DescLevel& L = a.lv[K.octave][K.scale - 1];
        const float sg = L.sigma;
        float d[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float* q = pat + (lane + 32 * h) * 6;
            const float v1 = sample<S>(L, K.ix, K.iy, K.iz, sg * q[0], sg * q[1], sg * q[2]);
            const float v2 = sample<S>(L, K.ix, K.iy, K.iz, sg * q[3], sg * q[4], sg * q[5]);
            d[h] = v1 - v2;
        }
        if (a.brief != nullptr) {
            const unsigned lo = __ballot_sync(0xffffffffu, d[0] > 0.f);
            const unsigned hi = __ballot_sync(0xffffffffu, d[1] > 0.f);
            if (lane == 0) a.brief[kp] = (uint64_t)lo | ((uint64_t)hi << 32);
        }
        if (a.rrief != nullptr) {
            int r0 = 0, r1 = 0;
            const int k0 = lane, k1 = lane + 32;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                for (int src = 0; src < 32; ++src) {
                    const float dj = __shfl_sync(0xffffffffu, d[h], src);
                    const int j = src + 32 * h;
                    r0 += (dj < d[0]) || (dj == d[0] && j < k0);
                    r1 += (dj < d[1]) || (dj == d[1] && j < k1);
                }
            }
            a.rrief[(int64_t)kp * 64 + k0] = (uint8_t)r0;
            a.rrief[(int64_t)kp * 64 + k1] = (uint8_t)r1;
        }
    }
}

template <typename S>
__global__ void read_level_kernel(const ReadLevelArgs a) {
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % a.nx);
        const int64_t r = i / a.nx;
        const int y = (int)(r % a.ny);
        const int z = (int)(r / a.ny);
        a.dst[i] = to_f32(static_cast<const S*>(a.src)[(int64_t)z * a.pz + (int64_t)y * a.py + x]);
    }
}

}  // namespace

LaunchSpec describe_spec(int storage, const DescribeArgs&, int n_max) {
    LaunchSpec s;
    if (storage == SIFT3D_STORAGE_F32) s.func = reinterpret_cast<const void*>(&describe_kernel<float>);
    else if (storage == SIFT3D_STORAGE_F16) s.func = reinterpret_cast<const void*>(&describe_kernel<__half>);
    else s.func = reinterpret_cast<const void*>(&describe_kernel<__nv_bfloat16>);
    int blocks = (n_max + DS_WARPS - 1) / DS_WARPS;
    blocks = blocks < 1 ? 1 : (blocks > 4 * 152 ? 4 * 152 : blocks);
    s.grid = dim3(blocks);
    s.block = dim3(DS_THREADS);
    s.smem = 0;
    s.name = "describe";
    return s;
}

LaunchSpec read_level_spec(int storage, const ReadLevelArgs& a) {
    LaunchSpec s;
    if (storage == SIFT3D_STORAGE_F32) s.func = reinterpret_cast<const void*>(&read_level_kernel<float>);
    else if (storage == SIFT3D_STORAGE_F16) s.func = reinterpret_cast<const void*>(&read_level_kernel<__half>);
    else s.func = reinterpret_cast<const void*>(&read_level_kernel<__nv_bfloat16>);
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    int64_t blocks = (n + 255) / 256;
    s.grid = dim3((unsigned)(blocks > 4096 ? 4096 : (blocks < 1 ? 1 : blocks)));
    s.block = dim3(256);
    s.name = "read_level";
    return s;
}

}  // namespace sift3d
