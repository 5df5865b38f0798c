// Internal declarations shared by the sm_103a kernels and the host runtime.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include <utility>

#include "sift3d.h"

namespace sift3d {

constexpr int kMaxRadius = 16;     // largest 1D filter radius with a kernel instance
constexpr int kMaxLevels = SIFT3D_MAX_SCALES + 3;
constexpr int kMaxDogs = SIFT3D_MAX_SCALES + 2;
constexpr int kSortSmemKeys = 4096;  // sort keys staged in shared memory per tile

// ---- storage types: levels may be stored narrower than the float32 arithmetic
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(uint8_t v) { return (float)v; }

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// Taps of a symmetric 1D Gaussian: w[0] is the centre, w[k] the weight at +-k.
struct Taps {
    float w[kMaxRadius + 1];
};

// ---- conv_xy: y pass then x pass of one plane tile, result (float) to dst -------
// The source plane is read with clamp-to-edge in x and y.  With `sub` set, the
// source is the previous octave's level S and each source voxel is the 2x2x2
// mean at (2x.., 2y.., 2z..) (the octave sub-sampling, Sec. 2.2.2); the tile's
// own voxels of that mean are also written to `base_out` (G_0 of the octave).
struct ConvXYArgs {
    const void* src;          // element type per kernel instance
    int64_t src_py, src_pz;   // source pitches (elements)
    float src_scale;          // multiplies each source value (1/255 for uint8)
    float* dst;               // intermediate (float32), level pitches
    int64_t py, pz;           // pitches of dst / base_out
    int nx, ny, nz;           // dims of this octave
    void* base_out;           // sub mode: G_0 of this octave (storage type), else null
    __half* res_out;          // sub mode, 16-bit storage: G_0's rounding residual (G_0 - stored G_0)
    int* zero_count;          // if set, block (0,0,0) zeroes kDetectCounters ints first
    Taps taps;
    float* dst2;              // if set: the same plane filtered with taps2 too (the
    Taps taps2;               //   descriptor pre-blur, radius kFusedBlurRadius)
    int row_tile;             // rows per CTA of the full-row kernel (multiple of 8; 0: 16)
};

// Radius of the descriptor pre-blur that the level kernels can fuse (sigma 0.95).
constexpr int kFusedBlurRadius = 4;

// Per-detect device counters: [0] keypoints found, [1] total reported by the
// sort (-2 = a bounded device wait ran out), [2] unused, [3] error flag.
constexpr int kDetectCounters = 4;

// ---- conv_z: z pass over columns, epilogue writes G_s and the DoG -------------
struct ConvZArgs {
    const float* src;         // intermediate from conv_xy
    void* dst;                // G_s (storage type)
    const void* prev;         // G_{s-1} for the DoG, or null
    float* dog;               // D_{s-1} = G_{s-1} - G_s (float32 for every storage type), or null
    __half* res;              // 16-bit storage: rounding residuals, in place: read G_{s-1}'s (when
                              //   prev is set) and write G_s's; null for float32 storage
    int64_t py, pz;           // shared pitches
    int nx, ny, nz;
    Taps taps;
    const float* src2;        // if set: z pass of this second intermediate with taps2
    void* dst2;               //   into dst2 (the pre-blurred level for the descriptors)
    Taps taps2;
    float* sub_dst;           // if set (float32 storage, level S): also write the next
    int64_t sub_py, sub_pz;   //   octave's G_0, the 2x2x2 means of G_s, with these pitches
    int z_tile;               // outputs per thread: 8 or 16 (float32 storage), else 16
};

// ---- peak detection + compaction --------------------------------------------
struct PeakArgs {
    const void* dog[kMaxDogs];   // D_0..D_{S+1} of the octave (storage type)
    int64_t py, pz;
    int nx, ny, nz;
    int octave, n_scales, border, sign_sum_min;   // n_scales: S, the octave's scales
    int ns, scale_base;                 // this launch tests scales scale_base+1 .. scale_base+ns,
                                        // staged as DoG levels scale_base .. scale_base+ns+1
    float contrast, curv_k1, curv_k2;   // (2r+1)^3 and r^2
    float sigma_level[kMaxLevels];      // sigma_s in octave voxels
    int refine;                         // report the 4D quadratic's extremum
    sift3d_keypoint* out;               // staging records
    int* count;                         // running total (all octaves)
    int capacity;
};

// Arguments of the TMA-fed peak kernel: the octave's DoG levels D_0..D_{S+1}
// lie at a constant stride in the workspace and are described by one 4D tensor
// map (x, y, z, level), passed as a __grid_constant__ kernel parameter.
struct PeakTmaArgs {   // 128-byte aligned through CUtensorMap
    CUtensorMap dogs;                   // box: a CTA's tile plus halo of one DoG level
    PeakArgs a;
    int x_start;                        // x of the first tile's halo origin (multiple of 8)
    const int* test_flag;               // null, or *test_flag != 0: a CTA's first wait is one non-blocking test
    int* err;                           // set to 1 when a TMA wait runs out
    int gx, gy, gz;                     // tiles per axis (batched launches)
};

// Tile geometry of the peak kernel for a storage type: the halo origin of the
// first x tile and the TMA box (x, y, z, levels) of one copy.
void peak_layout(int storage, const PeakArgs& a, int* x_start, int* box_x, int* box_y, int* box_z, int* box_l);

// ---- canonical sort of the staging records into the caller's array --------
struct SortArgs {
    const sift3d_keypoint* staging;
    sift3d_keypoint* out;
    const int* count;
    const int* err;             // non-zero: a bounded wait ran out, report -2
    int* count_out;             // total detected (may exceed capacity)
    int* count_copy;            // null, or a second place for that total (batched detects)
    int capacity;
};

// ---- descriptors --------------------------------------------------------------
struct DescLevel {
    const void* ptr;           // pre-blurred G_s (storage type)
    int64_t py, pz;
    int nx, ny, nz;
    float sigma;               // sigma_s in octave voxels
};

struct DescribeArgs {
    const sift3d_keypoint* kps;
    int n;                     // >= 0: count; < 0: read *n_dev, clamp to n_cap
    const int* n_dev;
    int n_cap;
    int n_scales;
    int n_octaves;
    DescLevel lv[SIFT3D_MAX_OCTAVES][SIFT3D_MAX_SCALES];
    float pattern[SIFT3D_N_PAIRS * 6];
    uint64_t* brief;
    uint8_t* rrief;
};

// ---- nearest-neighbour matching ------------------------------------------------
struct MatchArgs {
    const void* a;             // na descriptors (uint64 BRIEF words or 64-byte RRIEF rows)
    const void* b;             // nb descriptors of the same kind
    int na, nb;
    int32_t* nn;               // per query: index of the nearest in b (-1 if nb == 0)
    int32_t* dist;             //            its distance (INT_MAX if nb == 0)
    int32_t* dist2;            //            second-nearest distance (INT_MAX if none), or null
};

// Results of a served request into mapped pinned host memory: the total
// count and exactly min(count, capacity) records and descriptors.
struct PackArgs {
    const int* count;                  // device: keypoints detected (< 0: the detect failed)
    int capacity;
    const sift3d_keypoint* kps;        // device arrays of capacity entries
    const uint64_t* brief;
    const uint8_t* rrief;
    int* out_count;                    // mapped host memory (device addresses)
    sift3d_keypoint* out_kps;
    uint64_t* out_brief;
    uint8_t* out_rrief;
};

struct ReadLevelArgs {
    const void* src;
    int64_t py, pz;
    int nx, ny, nz;
    float* dst;
};

// A batched launch: the per-volume argument structs of one pass and the
// prefix sums of their work items; item i belongs to the volume v with
// prefix[v] <= i < prefix[v + 1].
struct BatchTable {
    const void* args;          // device array of n per-volume argument structs
    const int* prefix;         // device array of n + 1 item offsets
    int n, total;              // volumes, items (= prefix[n])
};

// A batched convolution pass over at most kBatchVols volumes: every volume
// filters the same level, so the taps are shared, and the volumes' pointers
// and dims travel in the kernel parameters as well (uniform across a CTA, so
// they stay in the constant bank and uniform registers).
constexpr int kBatchVols = 64;

struct XYVol {                 // the per-volume fields of ConvXYArgs
    const void* src;
    int64_t src_py, src_pz;
    float* dst;
    int64_t py, pz;
    void* base_out;
    __half* res_out;
    int* zero_count;
    float* dst2;
    float src_scale;
    int nx, ny, nz, row_tile;
};

struct ZVol {                  // the per-volume fields of ConvZArgs
    const float* src;
    void* dst;
    const void* prev;
    float* dog;
    __half* res;
    const float* src2;
    void* dst2;
    int64_t py, pz;
    int nx, ny, nz;
};

struct BatchXY {
    int n, total;
    int prefix[kBatchVols + 1];
    Taps taps, taps2;
    XYVol vol[kBatchVols];
};

struct BatchZ {
    int n, total;
    int prefix[kBatchVols + 1];
    Taps taps, taps2;
    ZVol vol[kBatchVols];
};
// Kernel parameters are limited to 32764 bytes.
static_assert(sizeof(BatchXY) <= 32764 && sizeof(BatchZ) <= 32764, "batch parameters too large");

// The volume of item i of a parameter-embedded batch (a uniform search).
__host__ __device__ inline int batch_param_volume(const int* prefix, int n, int item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

#if defined(__CUDACC__)
__device__ __forceinline__ int batch_volume(const BatchTable& b, int item) {
    int lo = 0, hi = b.n - 1;  // the last v with prefix[v] <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(b.prefix + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
#endif

// A kernel launch with its single by-value argument struct, usable both for a
// direct launch and as a CUDA graph kernel node.
struct LaunchSpec {
    const void* func = nullptr;
    dim3 grid, block;
    size_t smem = 0;
    const char* name = "";
};

int device_sm_count();   // SMs of the current device (cached)

// Launch of a spec on a stream.
cudaError_t launch_spec(const LaunchSpec& s, void** args, cudaStream_t st);

// Launch builders (one per kernel family).  `storage` is SIFT3D_STORAGE_*,
// `src_kind` for conv_xy is 0 = float32, 1 = uint8, 2 = storage type.
LaunchSpec conv_xy_spec(int radius, int src_kind, int storage, bool sub, ConvXYArgs& a);   // sets a.row_tile
LaunchSpec conv_z_spec(int radius, int storage, const ConvZArgs& a);
LaunchSpec peak_spec(int storage, const PeakTmaArgs& a);
LaunchSpec sort_spec(const SortArgs& a);
void peak_fill_tiles(PeakTmaArgs* A);             // sets gx, gy, gz
LaunchSpec peak_batch_spec(int ns, int total);    // batched peaks over a BatchTable of PeakTmaArgs
LaunchSpec describe_spec(int storage, const DescribeArgs& a, int n_max);
LaunchSpec read_level_spec(int storage, const ReadLevelArgs& a);
// Batched passes over many volumes (float32 storage): persistent grids over
// per-volume arguments (BatchXY / BatchZ); *_items gives one volume's work items.
LaunchSpec conv_xy_batch_spec(int radius, int src_kind, bool sub, bool blur, int nx_max, int row_tile, int total);
LaunchSpec conv_z_batch_spec(int radius, bool blur, int total);
int conv_xy_items(const ConvXYArgs& a);
int conv_z_items(const ConvZArgs& a);
LaunchSpec pack_spec(const PackArgs& a);
LaunchSpec match_spec(int kind, const MatchArgs& a);
// SIFT-Rank descriptors of keypoints on the levels of d.lv (G_s, not pre-blurred).
int enqueue_siftrank(int storage, const DescribeArgs& d, const sift3d_keypoint* kps, int n, const int* n_dev,
                     int n_cap, uint8_t* desc, float* rot, cudaStream_t st);

}  // namespace sift3d
