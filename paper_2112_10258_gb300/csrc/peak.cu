// 4D extremum detection for sm_103a (Sec. 2.2.2 "4D Peak Detection").
//
// For every interior voxel v of an octave and every detection scale s = 1..S:
//   1. contrast  |D_s(v)| >= t_c (cheap, and it rejects almost every voxel);
//   2. sum of signs  S = sum over the 80 neighbours n (3x3x3 in D_{s-1} and
//      D_{s+1}, 3x3x3 minus v in D_s) of sign(D_s(v) - D(n)); keep |S| >= cut
//      (+-80 = strict peak / valley, the paper's default interval);
//   3. curvature  H' = -sign(S) * Hessian(D_s at v) positive definite (leading
//      minors) and tr(H')^3 r^2 < (2r+1)^3 det(H').
// A CTA stages its 32x8x8 tile of D_1..D_S (plus a one-voxel halo) in shared
// memory, so the neighbour reads are shared-memory reads; D_0 and D_{S+1} are
// read from global memory only for voxels that survive the in-scale
// comparisons.  A branch-free first pass applies exact necessary conditions to
// every voxel-scale (contrast, the same voxel in D_{s-1} and D_{s+1}, the six
// face neighbours); the ~1% that survive are listed in shared memory and get
// the full test in a second pass spread over all lanes.  Keypoints are
// compacted without an extrema map: a warp ballot, an intra-warp prefix (popc
// of the lower lanes) and one atomicAdd per warp that has any.  A rank sort then writes
// the records in canonical order (octave, scale, iz, iy, ix).  A single-CTA bitonic sort then writes the
// records to the caller in the canonical order (octave, scale, iz, iy, ix).
#include <algorithm>

#include "peak_tile.cuh"

namespace sift3d {

namespace {

using namespace peak_detail;

template <typename S>
__global__ void __launch_bounds__(PK_THREADS, 3) peak_kernel(const PeakArgs a) {
    extern __shared__ float pk_sm[];
    __shared__ unsigned surv[PK_SURV];
    __shared__ int n_surv;
    pdl_launch_dependents();
    pdl_wait();
    peak_tile<S>(a, blockIdx.x, blockIdx.y, blockIdx.z, pk_sm, surv, n_surv);
}

// ---- canonical order ------------------------------------------------------
// Rank sort: the key of record i packs (octave, scale, iz, iy, ix, i), so keys
// are unique and record i's place is the number of smaller keys.  Each CTA
// ranks 1024 records against all keys, read through shared memory in tiles.
constexpr int SORT_THREADS = 128;
constexpr int SORT_TILE = kSortSmemKeys;

__device__ __forceinline__ unsigned long long sort_key(const sift3d_keypoint& k, int idx) {
    return ((unsigned long long)(k.octave & 0xF) << 60) | ((unsigned long long)(k.scale & 0xF) << 56) |
           ((unsigned long long)(k.iz & 0xFFF) << 44) | ((unsigned long long)(k.iy & 0xFFF) << 32) |
           ((unsigned long long)(k.ix & 0xFFF) << 20) | (unsigned long long)idx;
}

__global__ void __launch_bounds__(SORT_THREADS) sort_kernel(const SortArgs a) {
    __shared__ unsigned long long skeys[SORT_TILE];
    pdl_wait();
    const int total = *a.count;
    const int n = min(total, a.capacity);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.count_out = (a.tail_err != nullptr && *a.tail_err != 0) ? -2 : total;
    if ((int)blockIdx.x * SORT_THREADS >= n) return;
    const int i = blockIdx.x * SORT_THREADS + threadIdx.x;
    const unsigned long long mine = i < n ? sort_key(a.staging[i], i) : ~0ull;
    int rank = 0;
    for (int base = 0; base < n; base += SORT_TILE) {
        const int len = min(SORT_TILE, n - base);
        __syncthreads();
        for (int j = threadIdx.x; j < len; j += SORT_THREADS) skeys[j] = sort_key(a.staging[base + j], base + j);
        __syncthreads();
        for (int j = 0; j < len; ++j) rank += skeys[j] < mine;
    }
    if (i < n) a.out[rank] = a.staging[i];
}

}  // namespace

LaunchSpec peak_spec(int storage, const PeakArgs& a) {
    LaunchSpec s;
    if (storage == SIFT3D_STORAGE_F32) s.func = reinterpret_cast<const void*>(&peak_kernel<float>);
    else if (storage == SIFT3D_STORAGE_F16) s.func = reinterpret_cast<const void*>(&peak_kernel<__half>);
    else s.func = reinterpret_cast<const void*>(&peak_kernel<__nv_bfloat16>);
    const int ix = a.nx - 2 * a.border, iy = a.ny - 2 * a.border, iz = a.nz - 2 * a.border;
    s.grid = dim3((ix + PK_BX - 1) / PK_BX, (iy + PK_BY - 1) / PK_BY, (iz + PK_TZ - 1) / PK_TZ);
    s.block = dim3(PK_BX, PK_BY);
    s.smem = peak_smem_bytes(a.n_scales);
    if (s.smem > 48 * 1024) cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
    s.name = "peak";
    return s;
}

LaunchSpec sort_spec(const SortArgs& a) {
    LaunchSpec s;
    s.func = reinterpret_cast<const void*>(&sort_kernel);
    s.grid = dim3((unsigned)std::max(1, (a.capacity + SORT_THREADS - 1) / SORT_THREADS));
    s.block = dim3(SORT_THREADS);
    s.smem = 0;
    s.name = "sort";
    return s;
}

}  // namespace sift3d
