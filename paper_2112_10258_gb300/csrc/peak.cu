// 4D extremum detection for sm_103a (Sec. 2.2.2 "4D Peak Detection").
//
// For every interior voxel v of an octave and every detection scale s = 1..S:
//   1. contrast  |D_s(v)| >= t_c (cheap, and it rejects almost every voxel);
//   2. sum of signs  S = sum over the 80 neighbours n (3x3x3 in D_{s-1} and
//      D_{s+1}, 3x3x3 minus v in D_s) of sign(D_s(v) - D(n)); keep |S| >= cut
//      (+-80 = strict peak / valley, the paper's default interval);
//   3. curvature  H' = -sign(S) * Hessian(D_s at v) positive definite (leading
//      minors) and tr(H')^3 r^2 < (2r+1)^3 det(H').
// Survivors are compacted without an extrema map: a warp ballot plus an
// intra-warp prefix (popc of the lower lanes) and a block prefix over the warp
// totals give each keypoint its slot, and one atomicAdd per block reserves the
// block's range in the staging array.  A single-CTA bitonic sort then writes the
// records to the caller in the canonical order (octave, scale, iz, iy, ix).
#include "common.cuh"

namespace sift3d {

namespace {

constexpr int PK_BX = 32;
constexpr int PK_BY = 8;
constexpr int PK_THREADS = PK_BX * PK_BY;

// The 80 neighbours as (dx, dy, dz, level offset): the 26 of D_s first (faces,
// then edges, then corners: the likeliest to break an extremum early), then the
// 27 of D_{s-1} and the 27 of D_{s+1}.
struct NbrTable {
    int4 v[80];
};

constexpr NbrTable make_nbr_table() {
    NbrTable t{};
    int n = 0;
    for (int order = 1; order <= 3; ++order)          // |dx|+|dy|+|dz|
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int m = (dx != 0) + (dy != 0) + (dz != 0);
                    if (m == order) t.v[n++] = int4{dx, dy, dz, 0};
                }
    for (int dl = -1; dl <= 1; dl += 2)
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) t.v[n++] = int4{dx, dy, dz, dl};
    return t;
}

__constant__ int4 c_nbr[80];

template <typename S>
__device__ __forceinline__ float ldv(const void* base, int64_t off) {
    return to_f32(static_cast<const S*>(base)[off]);
}

template <typename S>
__global__ void __launch_bounds__(PK_THREADS) peak_kernel(const PeakArgs a) {
    const int b = a.border;
    const int x = blockIdx.x * PK_BX + threadIdx.x + b;
    const int y = blockIdx.y * PK_BY + threadIdx.y + b;
    const int z = blockIdx.z + b;
    const bool inside = x < a.nx - b && y < a.ny - b && z < a.nz - b;
    const int64_t py = a.py, pz = a.pz;
    const int64_t off = (int64_t)z * pz + (int64_t)y * py + x;

    unsigned found = 0;          // bit s: keypoint at scale s
    int ssum[SIFT3D_MAX_SCALES + 1];
    float cval[SIFT3D_MAX_SCALES + 1];
    if (inside) {
        for (int s = 1; s <= a.n_scales; ++s) {
            const float c = ldv<S>(a.dog[s], off);
            cval[s] = c;
            if (!(fabsf(c) >= a.contrast)) continue;
            // Sum of signs with early exit: after k of the 80 comparisons, |S| can
            // change by at most 80 - k, so stop once the cut is out of reach.
            int sum = 0;
            int k = 0;
            for (; k < 80; ++k) {
                const int4 nb = c_nbr[k];
                const float n = ldv<S>(a.dog[s + nb.w], off + nb.z * pz + nb.y * py + nb.x);
                sum += (c > n) - (c < n);
                const int reach = (sum < 0 ? -sum : sum) + (79 - k);
                if (reach < a.sign_sum_min) break;
            }
            if (k < 80) continue;
            ssum[s] = sum;
            if (sum < a.sign_sum_min && sum > -a.sign_sum_min) continue;
            const void* D = a.dog[s];
            auto d = [&](int dz, int dy, int dx) { return ldv<S>(D, off + dz * pz + dy * py + dx); };
            const float hxx = d(0, 0, 1) + d(0, 0, -1) - 2.0f * c;
            const float hyy = d(0, 1, 0) + d(0, -1, 0) - 2.0f * c;
            const float hzz = d(1, 0, 0) + d(-1, 0, 0) - 2.0f * c;
            const float hxy = (d(0, 1, 1) - d(0, -1, 1) - d(0, 1, -1) + d(0, -1, -1)) * 0.25f;
            const float hxz = (d(1, 0, 1) - d(-1, 0, 1) - d(1, 0, -1) + d(-1, 0, -1)) * 0.25f;
            const float hyz = (d(1, 1, 0) - d(-1, 1, 0) - d(1, -1, 0) + d(-1, -1, 0)) * 0.25f;
            const float sg = sum > 0 ? -1.0f : 1.0f;
            const float A = sg * hxx, B = sg * hyy, C = sg * hzz;
            const float XY = sg * hxy, XZ = sg * hxz, YZ = sg * hyz;
            const float m2 = A * B - XY * XY;
            const float det = A * (B * C - YZ * YZ) - XY * (XY * C - YZ * XZ) + XZ * (XY * YZ - B * XZ);
            const float tr = A + B + C;
            const float g = a.curv_k1 * det - a.curv_k2 * (tr * tr * tr);
            if (A > 0.f && m2 > 0.f && det > 0.f && g > 0.f) found |= 1u << s;
        }
    }

    // ---- compaction: ballot / popc within the warp, prefix over warps, one atomic
    const int lane = threadIdx.x + PK_BX * threadIdx.y;     // linear thread id
    const int wid = lane >> 5, lid = lane & 31;
    const int mine = __popc(found);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lid >= o) incl += t;
    }
    __shared__ int warp_tot[PK_THREADS / 32];
    __shared__ int block_base;
    if (lid == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (lane == 0) {
        int acc = 0;
        for (int w = 0; w < PK_THREADS / 32; ++w) {
            const int t = warp_tot[w];
            warp_tot[w] = acc;
            acc += t;
        }
        block_base = acc > 0 ? atomicAdd(a.count, acc) : 0;
    }
    __syncthreads();
    if (mine == 0) return;
    int slot = block_base + warp_tot[wid] + incl - mine;
    const float scale = (float)(1 << a.octave);
    for (int s = 1; s <= a.n_scales; ++s) {
        if (!(found & (1u << s))) continue;
        if (slot < a.capacity) {
            sift3d_keypoint k;
            k.x = ((float)x + 0.5f) * scale - 0.5f;
            k.y = ((float)y + 0.5f) * scale - 0.5f;
            k.z = ((float)z + 0.5f) * scale - 0.5f;
            k.sigma = a.sigma_level[s] * scale;
            k.ix = x;
            k.iy = y;
            k.iz = z;
            k.octave = (int16_t)a.octave;
            k.scale = (int16_t)s;
            k.polarity = ssum[s] > 0 ? 1 : -1;
            k.reserved0[0] = k.reserved0[1] = k.reserved0[2] = 0;
            k.dog = cval[s];
            k.sign_sum = ssum[s];
            k.reserved1 = 0;
            a.out[slot] = k;
        }
        ++slot;
    }
}

// ---- canonical order ------------------------------------------------------
constexpr int SORT_THREADS = 1024;
constexpr int SORT_SMEM_KEYS = 16384;   // 128 KiB of keys in shared memory
constexpr unsigned long long kIdxMask = (1ull << 20) - 1;

__device__ __forceinline__ unsigned long long sort_key(const sift3d_keypoint& k, int idx) {
    return ((unsigned long long)(k.octave & 0xF) << 60) | ((unsigned long long)(k.scale & 0xF) << 56) |
           ((unsigned long long)(k.iz & 0xFFF) << 44) | ((unsigned long long)(k.iy & 0xFFF) << 32) |
           ((unsigned long long)(k.ix & 0xFFF) << 20) | (unsigned long long)idx;
}

__device__ void bitonic(unsigned long long* keys, int n_pow2) {
    for (int k = 2; k <= n_pow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n_pow2; i += SORT_THREADS) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long u = keys[i], v = keys[ixj];
                    const bool up = (i & k) == 0;
                    if ((u > v) == up) {
                        keys[i] = v;
                        keys[ixj] = u;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(SORT_THREADS) sort_kernel(const SortArgs a) {
    extern __shared__ unsigned long long skeys[];
    const int total = *a.count;
    const int n = min(total, a.capacity);
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    unsigned long long* keys = n2 <= SORT_SMEM_KEYS ? skeys : a.scratch_keys;
    if (keys == nullptr || n2 > (keys == skeys ? SORT_SMEM_KEYS : a.scratch_len)) {
        if (threadIdx.x == 0) *a.count_out = -1;  // no room to sort: reported as an error
        return;
    }
    for (int i = threadIdx.x; i < n2; i += SORT_THREADS)
        keys[i] = i < n ? sort_key(a.staging[i], i) : ~0ull;
    __syncthreads();
    bitonic(keys, n2);
    for (int i = threadIdx.x; i < n; i += SORT_THREADS) a.out[i] = a.staging[keys[i] & kIdxMask];
    if (threadIdx.x == 0) *a.count_out = total;
}

}  // namespace

LaunchSpec peak_spec(int storage, const PeakArgs& a) {
    static const bool table_ready = [] {
        constexpr NbrTable t = make_nbr_table();
        static_assert(t.v[25].w == 0 && t.v[26].w == -1 && t.v[79].w == 1, "neighbour table layout");
        return cudaMemcpyToSymbol(c_nbr, t.v, sizeof(t.v)) == cudaSuccess;
    }();
    LaunchSpec s;
    if (!table_ready) return s;
    if (storage == SIFT3D_STORAGE_F32) s.func = reinterpret_cast<const void*>(&peak_kernel<float>);
    else if (storage == SIFT3D_STORAGE_F16) s.func = reinterpret_cast<const void*>(&peak_kernel<__half>);
    else s.func = reinterpret_cast<const void*>(&peak_kernel<__nv_bfloat16>);
    const int ix = a.nx - 2 * a.border, iy = a.ny - 2 * a.border, iz = a.nz - 2 * a.border;
    s.grid = dim3((ix + PK_BX - 1) / PK_BX, (iy + PK_BY - 1) / PK_BY, iz);
    s.block = dim3(PK_BX, PK_BY);
    s.smem = 0;
    s.name = "peak";
    return s;
}

LaunchSpec sort_spec(const SortArgs&) {
    LaunchSpec s;
    s.func = reinterpret_cast<const void*>(&sort_kernel);
    s.grid = dim3(1);
    s.block = dim3(SORT_THREADS);
    s.smem = SORT_SMEM_KEYS * sizeof(unsigned long long);
    cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
    s.name = "sort";
    return s;
}

}  // namespace sift3d
