// BRIEF and RRIEF descriptors for sm_103a (Sec. 2.2.3 "FAST 3D Descriptors").
//
// One warp per keypoint.  Lane l owns point pairs k = l and k = l + 32: it reads
// the four trilinear samples I(c + sigma_s p1_k), I(c + sigma_s p2_k) from the
// keypoint's pre-blurred level (clamped coordinates) and forms d_k.  BRIEF is two
// warp ballots of [d_k > 0]; RRIEF gives each d_k its rank among the 64 values
// (ties by lower index) by streaming the other 63 values through warp shuffles.
// The 64-pair pattern sits in shared memory (lanes read different pairs, which
// the constant cache would serialise).
#include <algorithm>
#include <cmath>

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

// ---- 3D SIFT-Rank (the paper's comparison baseline; Sec. 1 and Sec. 3.5) -----
// One CTA per keypoint, on the keypoint's Gaussian level G_s (not pre-blurred).
//   samples    the 8^3 cell centres of [-r, r]^3 (r = 3 sigma_s) inside the
//              ball |u| <= r (280 of them), weight exp(-|u|^2 / (2 (r/2)^2));
//   gradient   central differences of trilinear samples, unit steps;
//   frame      e1 = mean gradient of the peak bin of the 12-direction
//              (icosahedron) histogram of w |g|; e2 the same for the parts of
//              the gradients perpendicular to e1; e3 = e1 x e2;
//   histogram  samples at c + R u, g' = R^T g; element 8 * octant(u) +
//              octant(g') gets w |g'|;
//   output     the ranks of the 64 values (ties by lower index), as RRIEF.
// Sample i belongs to thread i % SR_THREADS.  The 12-direction histograms and
// the bin means are per-thread partials reduced by a fixed xor butterfly in
// each warp and then warp by warp in index order; the 64-bin histogram sums
// each bin over its spatial octant's samples (the table is ordered by octant)
// in table order.  Every sum has a fixed order, so the descriptor does not
// depend on scheduling.
constexpr int SR_THREADS = 128;
constexpr int SR_WARPS = SR_THREADS / 32;
constexpr int SR_SAMPLES = 280;        // cell centres of the 8^3 grid on [-1, 1]^3 inside the unit ball
constexpr int SR_SLOTS = (SR_SAMPLES + SR_THREADS - 1) / SR_THREADS;

struct SiftRankArgs {
    const sift3d_keypoint* kps;
    int n;                     // >= 0: count; < 0: read *n_dev, clamp to n_cap
    const int* n_dev;
    int n_cap;
    int n_scales, n_octaves;
    DescLevel lv[SIFT3D_MAX_OCTAVES][SIFT3D_MAX_SCALES];   // G_s (not pre-blurred)
    uint8_t* desc;             // n x 64 ranks
    float* rot;                // n x 9 (row-major R, columns e1 e2 e3) or null
    float ico[12][3];          // the icosahedron's unit vertices
    int oct_start[9];          // samples of spatial octant o: [oct_start[o], oct_start[o + 1])
    float smp[SR_SAMPLES][4];  // the samples by octant: offset in units of r (x, y, z) and weight
};

template <typename S>
__device__ __forceinline__ void gradient_at(const DescLevel& L, int cx, int cy, int cz, float tx, float ty, float tz,
                                            float* g) {
    g[0] = 0.5f * (sample<S>(L, cx, cy, cz, tx + 1.f, ty, tz) - sample<S>(L, cx, cy, cz, tx - 1.f, ty, tz));
    g[1] = 0.5f * (sample<S>(L, cx, cy, cz, tx, ty + 1.f, tz) - sample<S>(L, cx, cy, cz, tx, ty - 1.f, tz));
    g[2] = 0.5f * (sample<S>(L, cx, cy, cz, tx, ty, tz + 1.f) - sample<S>(L, cx, cy, cz, tx, ty, tz - 1.f));
}

__device__ __forceinline__ int nearest_direction(const float (*ico)[3], const float* v) {
    int best = 0;
    float bd = -INFINITY;
#pragma unroll
    for (int m = 0; m < 12; ++m) {
        const float d = v[0] * ico[m][0] + v[1] * ico[m][1] + v[2] * ico[m][2];
        if (d > bd) {
            bd = d;
            best = m;
        }
    }
    return best;
}

// Sum of v over the CTA, written to out[0..NV) for every thread to read.
template <int NV>
__device__ __forceinline__ void cta_sum(float (&v)[NV], float (*red)[16], float* out) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (t < NV) {
        float acc = red[0][t];
#pragma unroll
        for (int w = 1; w < SR_WARPS; ++w) acc += red[w][t];
        out[t] = acc;
    }
    __syncthreads();
}

// Peak bin of the 12-direction histogram of w |v| over the samples and the
// weighted mean of that bin's vectors (mean[0..3) in shared memory).
__device__ __forceinline__ void direction_peak(const float (*ico)[3], const float (&v)[SR_SLOTS][3],
                                               const float (&w)[SR_SLOTS], float (*red)[16], float* hist,
                                               float* mean) {
    int b[SR_SLOTS];
    float h[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) h[m] = 0.f;
#pragma unroll
    for (int j = 0; j < SR_SLOTS; ++j) {
        b[j] = nearest_direction(ico, v[j]);
        const float mag = w[j] * sqrtf(v[j][0] * v[j][0] + v[j][1] * v[j][1] + v[j][2] * v[j][2]);
#pragma unroll
        for (int m = 0; m < 12; ++m) h[m] += b[j] == m ? mag : 0.f;
    }
    cta_sum<12>(h, red, hist);
    int m = 0;
    for (int k = 1; k < 12; ++k)
        if (hist[k] > hist[m]) m = k;
    float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < SR_SLOTS; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] += b[j] == m ? w[j] * v[j][c] : 0.f;
    cta_sum<3>(acc, red, mean);
}

template <typename S>
__global__ void __launch_bounds__(SR_THREADS, 8) siftrank_kernel(const SiftRankArgs a) {
    __shared__ float sval[SR_SAMPLES];      // w |g'| of each sample
    __shared__ int sbin[SR_SAMPLES];        // its orientation octant
    __shared__ float red[SR_WARPS][16];
    __shared__ float hist[64];
    __shared__ float mean[3];
    __shared__ float R[3][3];               // columns e1 e2 e3: R[row][col]
    __shared__ float ico[12][3];
    __shared__ int oct[9];
    __shared__ float4 smp[SR_SAMPLES];
    const int t = threadIdx.x;
    if (t < 36) ico[t / 3][t % 3] = a.ico[t / 3][t % 3];
    if (t < 9) oct[t] = a.oct_start[t];
    for (int i = t; i < SR_SAMPLES; i += SR_THREADS)   // unit-radius offsets and weights
        smp[i] = make_float4(a.smp[i][0], a.smp[i][1], a.smp[i][2], a.smp[i][3]);
    __syncthreads();
    const int n = a.n >= 0 ? a.n : min(*a.n_dev, a.n_cap);
    for (int kp = blockIdx.x; kp < n; kp += gridDim.x) {
        const sift3d_keypoint K = a.kps[kp];
        if (K.octave < 0 || K.octave >= a.n_octaves || K.scale < 1 || K.scale > a.n_scales) continue;
        const DescLevel& L = a.lv[K.octave][K.scale - 1];
        const float r = 3.0f * L.sigma;
        // primary direction (w = 0 pads a thread's unused slots)
        float g[SR_SLOTS][3], sw[SR_SLOTS];
#pragma unroll
        for (int j = 0; j < SR_SLOTS; ++j) {
            const int i = t + j * SR_THREADS;
            if (i < SR_SAMPLES) {
                const float4 u = smp[i];
                gradient_at<S>(L, K.ix, K.iy, K.iz, r * u.x, r * u.y, r * u.z, g[j]);
                sw[j] = u.w;
            } else {
                g[j][0] = g[j][1] = g[j][2] = 0.f;
                sw[j] = 0.f;
            }
        }
        direction_peak(ico, g, sw, red, hist, mean);
        float e1x, e1y, e1z;
        {
            const float nm = sqrtf(mean[0] * mean[0] + mean[1] * mean[1] + mean[2] * mean[2]);
            if (nm > 0.f) e1x = mean[0] / nm, e1y = mean[1] / nm, e1z = mean[2] / nm;
            else e1x = 1.f, e1y = 0.f, e1z = 0.f;
        }
        // secondary direction from the parts perpendicular to e1
#pragma unroll
        for (int j = 0; j < SR_SLOTS; ++j) {
            const float d = g[j][0] * e1x + g[j][1] * e1y + g[j][2] * e1z;
            g[j][0] -= d * e1x;
            g[j][1] -= d * e1y;
            g[j][2] -= d * e1z;
        }
        direction_peak(ico, g, sw, red, hist, mean);
        if (t == 0) {
            float m0 = mean[0], m1 = mean[1], m2 = mean[2];
            const float d = m0 * e1x + m1 * e1y + m2 * e1z;
            m0 -= d * e1x, m1 -= d * e1y, m2 -= d * e1z;
            float nm = sqrtf(m0 * m0 + m1 * m1 + m2 * m2);
            if (!(nm > 0.f)) {   // any axis perpendicular to e1
                const bool px = fabsf(e1x) < 0.9f;
                m0 = px ? 0.f : -e1z, m1 = px ? e1z : 0.f, m2 = px ? -e1y : e1x;
                nm = sqrtf(m0 * m0 + m1 * m1 + m2 * m2);
            }
            R[0][0] = e1x, R[1][0] = e1y, R[2][0] = e1z;
            R[0][1] = m0 / nm, R[1][1] = m1 / nm, R[2][1] = m2 / nm;
            R[0][2] = e1y * R[2][1] - e1z * R[1][1];
            R[1][2] = e1z * R[0][1] - e1x * R[2][1];
            R[2][2] = e1x * R[1][1] - e1y * R[0][1];
        }
        __syncthreads();
        // descriptor: samples at c + R u, gradients in the keypoint frame
#pragma unroll
        for (int j = 0; j < SR_SLOTS; ++j) {
            const int i = t + j * SR_THREADS;
            if (i >= SR_SAMPLES) continue;
            const float4 u = smp[i];
            const float ux = r * u.x, uy = r * u.y, uz = r * u.z;
            const float tx = R[0][0] * ux + R[0][1] * uy + R[0][2] * uz;
            const float ty = R[1][0] * ux + R[1][1] * uy + R[1][2] * uz;
            const float tz = R[2][0] * ux + R[2][1] * uy + R[2][2] * uz;
            float q[3];
            gradient_at<S>(L, K.ix, K.iy, K.iz, tx, ty, tz, q);
            const float gx = R[0][0] * q[0] + R[1][0] * q[1] + R[2][0] * q[2];
            const float gy = R[0][1] * q[0] + R[1][1] * q[1] + R[2][1] * q[2];
            const float gz = R[0][2] * q[0] + R[1][2] * q[1] + R[2][2] * q[2];
            sbin[i] = (gx >= 0.f) + 2 * (gy >= 0.f) + 4 * (gz >= 0.f);
            sval[i] = u.w * sqrtf(gx * gx + gy * gy + gz * gz);
        }
        __syncthreads();
        if (t < 64) {   // element 8 * spatial octant + orientation octant
            const int o = t >> 3, ob = t & 7;
            float h = 0.f;
            for (int i = oct[o]; i < oct[o + 1]; ++i) h += sbin[i] == ob ? sval[i] : 0.f;
            hist[t] = h;
        }
        __syncthreads();
        if (t < 64) {
            const float v = hist[t];
            int rank = 0;
#pragma unroll 8
            for (int j = 0; j < 64; ++j) rank += (hist[j] < v) || (hist[j] == v && j < t);
            a.desc[(int64_t)kp * 64 + t] = (uint8_t)rank;
        }
        if (a.rot != nullptr && t < 9) a.rot[(int64_t)kp * 9 + t] = R[t / 3][t % 3];
        __syncthreads();
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

// One CTA of 256 threads per 64 records: 16-byte words of the records (3 per
// keypoint), the BRIEF words and the RRIEF rows (4 per keypoint), grid-strided.
__global__ void pack_results_kernel(const PackArgs a) {
    const int total = *a.count;
    const int n = total < 0 ? 0 : min(total, a.capacity);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.out_count = total;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint4* ks = reinterpret_cast<const uint4*>(a.kps);
    uint4* kd = reinterpret_cast<uint4*>(a.out_kps);
    for (int64_t i = t0; i < (int64_t)n * 3; i += stride) kd[i] = ks[i];
    if (a.out_brief != nullptr)
        for (int64_t i = t0; i < n; i += stride) a.out_brief[i] = a.brief[i];
    if (a.out_rrief != nullptr) {
        const uint4* rs = reinterpret_cast<const uint4*>(a.rrief);
        uint4* rd = reinterpret_cast<uint4*>(a.out_rrief);
        for (int64_t i = t0; i < (int64_t)n * 4; i += stride) rd[i] = rs[i];
    }
}

}  // namespace

LaunchSpec pack_spec(const PackArgs& a) {
    LaunchSpec s;
    s.func = reinterpret_cast<const void*>(&pack_results_kernel);
    s.grid = dim3((unsigned)std::max(1, std::min(148, (a.capacity + 63) / 64)));
    s.block = dim3(256);
    s.name = "pack_results";
    return s;
}

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

int enqueue_siftrank(int storage, const DescribeArgs& d, const sift3d_keypoint* kps, int n, const int* n_dev,
                     int n_cap, uint8_t* desc, float* rot, cudaStream_t st) {
    SiftRankArgs a{};
    {   // the 8^3 cell centres of [-1, 1]^3 inside the unit ball, weight
        // exp(-|u|^2 / (2 (1/2)^2)) (offsets and weight in units of r = 3 sigma),
        // grouped by spatial octant and in z, y, x order within each
        int k = 0;
        for (int o = 0; o < 8; ++o) {
            a.oct_start[o] = k;
            for (int z = 0; z < 8; ++z)
                for (int y = 0; y < 8; ++y)
                    for (int x = 0; x < 8; ++x) {
                        const float ux = ((x + 0.5f) / 8.f) * 2.f - 1.f, uy = ((y + 0.5f) / 8.f) * 2.f - 1.f;
                        const float uz = ((z + 0.5f) / 8.f) * 2.f - 1.f;
                        const float q = ux * ux + uy * uy + uz * uz;
                        const int oct = (ux >= 0.f) + 2 * (uy >= 0.f) + 4 * (uz >= 0.f);
                        if (q <= 1.f && oct == o && k < SR_SAMPLES) {
                            a.smp[k][0] = ux, a.smp[k][1] = uy, a.smp[k][2] = uz;
                            a.smp[k][3] = (float)std::exp(-(double)q / (2.0 * 0.25));
                            ++k;
                        }
                    }
        }
        a.oct_start[8] = k;
        if (k != SR_SAMPLES) return SIFT3D_EINVAL;
    }
    {   // cyclic permutations of (0, +-1, +-phi), normalised
        const double phi = (1.0 + std::sqrt(5.0)) / 2.0, inv = 1.0 / std::sqrt(1.0 + phi * phi);
        int k = 0;
        for (double u : {1.0, -1.0})
            for (double v : {phi, -phi}) a.ico[k][0] = 0.f, a.ico[k][1] = (float)(u * inv), a.ico[k][2] = (float)(v * inv), ++k;
        for (double u : {1.0, -1.0})
            for (double v : {phi, -phi}) a.ico[k][0] = (float)(u * inv), a.ico[k][1] = (float)(v * inv), a.ico[k][2] = 0.f, ++k;
        for (double u : {1.0, -1.0})
            for (double v : {phi, -phi}) a.ico[k][0] = (float)(v * inv), a.ico[k][1] = 0.f, a.ico[k][2] = (float)(u * inv), ++k;
    }
    a.kps = kps;
    a.n = n;
    a.n_dev = n_dev;
    a.n_cap = n_cap;
    a.n_scales = d.n_scales;
    a.n_octaves = d.n_octaves;
    memcpy(a.lv, d.lv, sizeof(a.lv));
    a.desc = desc;
    a.rot = rot;
    const void* f = storage == SIFT3D_STORAGE_F32   ? reinterpret_cast<const void*>(&siftrank_kernel<float>)
                    : storage == SIFT3D_STORAGE_F16 ? reinterpret_cast<const void*>(&siftrank_kernel<__half>)
                                                    : reinterpret_cast<const void*>(&siftrank_kernel<__nv_bfloat16>);
    const int n_max = n >= 0 ? n : n_cap;
    if (n_max <= 0) return SIFT3D_OK;
    const int blocks = std::min(n_max, 8 * 152);
    void* args[1] = {&a};
    return cudaLaunchKernel(f, dim3(blocks), dim3(SR_THREADS), args, 0, st) == cudaSuccess ? SIFT3D_OK
                                                                                           : SIFT3D_ECUDA;
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
