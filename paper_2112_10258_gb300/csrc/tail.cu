// Octave-tail kernel for sm_103a: every octave after the first few runs inside
// one cooperative launch.
//
// Small octaves do little work per pass (octave 2 of a 145x174x145 volume has
// 56K voxels), so as separate launches each pass costs mostly launch latency
// and ramp-up.  Here the passes of the remaining octaves - y/x filtering, z
// filtering with the DoG epilogue (Sec. 2.2.2), the descriptor pre-blur
// (Sec. 2.2.3) and 4D peak detection - are tasks grouped into phases; the tiles
// of all tasks of a phase are spread over the CTAs, and phases are separated by
// a grid-wide barrier.  The next octave starts (from the sub-sampled level S)
// in the same phase as level S+1 of the current one, so octaves overlap.
//
// The barrier waits are bounded: a CTA that waits longer than the spin limit
// raises the error flag and returns, every other CTA sees the flag and returns,
// and the detect reports the failure instead of hanging the device.
//
// Buffers are rewritten from phase to phase, so every load here is a plain
// (coherent) load; the acquire side of the barrier orders them after the
// previous phase's stores.
#include <algorithm>

#include "conv_tile.cuh"
#include "peak_tile.cuh"

namespace sift3d {

namespace {

constexpr int TL_THREADS = 256;
constexpr int TL_TX = conv_detail::XY_TX, TL_TY = conv_detail::XY_TY;   // y/x tile (64 x 32)
constexpr int TL_ZC = TL_THREADS, TL_TZ = conv_detail::Z_TZ;           // z tile: 256 columns x 16 planes
static_assert(conv_detail::XY_THREADS == TL_THREADS, "y/x tile body is written for 256 threads");
constexpr unsigned kSpinLimit = 1u << 22; // about 0.3 s of polling

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier over a monotone counter.  Returns false when the wait ran out
// (or another CTA already failed); the caller must then return.
__device__ bool grid_barrier(int* counter, int* err, int target) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter, 1);
        int good = 1;
        for (unsigned spin = 0;; ++spin) {
            if (ld_acquire(counter) >= target) break;
            if (ld_acquire(err) != 0 || spin > kSpinLimit) {
                atomicExch(err, 1);
                good = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

template <typename T>
__device__ __forceinline__ float ldf(const T* p) { return to_f32(*p); }

// y pass then x pass of one 64x32 tile of one plane, any radius R <= 16 (for
// radii without a compiled register-window body).
template <typename S>
__device__ void xy_tile_generic(const ConvXYArgs& a, int R, bool sub, int tile, float* sm) {
    const int tiles_x = (a.nx + TL_TX - 1) / TL_TX, tiles_y = (a.ny + TL_TY - 1) / TL_TY;
    const int x0 = (tile % tiles_x) * TL_TX;
    const int y0 = ((tile / tiles_x) % tiles_y) * TL_TY;
    const int z = tile / (tiles_x * tiles_y);
    const int W = TL_TX + 2 * R, H = TL_TY + 2 * R, WP = W | 1;
    float* in = sm;
    float* mid = sm + H * WP;
    const S* src = static_cast<const S*>(a.src);
    const int tid = threadIdx.x;
#pragma unroll 4
    for (int i = tid; i < H * W; i += TL_THREADS) {
        const int r = i / W, c = i - (i / W) * W;
        const int gy = min(max(y0 - R + r, 0), a.ny - 1);
        const int gx = min(max(x0 - R + c, 0), a.nx - 1);
        float v;
        if (!sub) {
            v = ldf(src + (int64_t)z * a.src_pz + (int64_t)gy * a.src_py + gx) * a.src_scale;
        } else {
            const S* p = src + (int64_t)(2 * z) * a.src_pz + (int64_t)(2 * gy) * a.src_py + 2 * gx;
            float acc = 0.f;
            acc += ldf(p);
            acc += ldf(p + 1);
            acc += ldf(p + a.src_py);
            acc += ldf(p + a.src_py + 1);
            acc += ldf(p + a.src_pz);
            acc += ldf(p + a.src_pz + 1);
            acc += ldf(p + a.src_pz + a.src_py);
            acc += ldf(p + a.src_pz + a.src_py + 1);
            v = acc * 0.125f;
            const int ty = r - R, tx = c - R;
            if (ty >= 0 && ty < TL_TY && tx >= 0 && tx < TL_TX && y0 + ty < a.ny && x0 + tx < a.nx)
                static_cast<S*>(a.base_out)[(int64_t)z * a.pz + (int64_t)(y0 + ty) * a.py + x0 + tx] = from_f32<S>(v);
        }
        in[r * WP + c] = v;
    }
    __syncthreads();
    for (int i = tid; i < TL_TY * W; i += TL_THREADS) {
        const int r = i / W, c = i - (i / W) * W;
        float acc = 0.f;
        for (int k = -R; k <= R; ++k) acc = fmaf(a.taps.w[k < 0 ? -k : k], in[(r + R + k) * WP + c], acc);
        mid[r * WP + c] = acc;
    }
    __syncthreads();
    for (int i = tid; i < TL_TY * TL_TX; i += TL_THREADS) {
        const int r = i / TL_TX, c = i - (i / TL_TX) * TL_TX;
        const int y = y0 + r, x = x0 + c;
        if (y >= a.ny || x >= a.nx) continue;
        float acc = 0.f;
        for (int k = -R; k <= R; ++k) acc = fmaf(a.taps.w[k < 0 ? -k : k], mid[r * WP + c + R + k], acc);
        a.dst[(int64_t)z * a.pz + (int64_t)y * a.py + x] = acc;
    }
}

// z pass of 256 columns x 16 planes, any radius, with the optional DoG epilogue.
template <typename S>
__device__ void z_tile_generic(const ConvZArgs& a, int R, int tile) {
    const int col_blocks = (int)((a.pz + TL_ZC - 1) / TL_ZC);
    const int64_t col = (int64_t)(tile % col_blocks) * TL_ZC + threadIdx.x;
    const int z0 = (tile / col_blocks) * TL_TZ;
    if (col >= a.pz) return;
    float acc[TL_TZ];
#pragma unroll
    for (int j = 0; j < TL_TZ; ++j) acc[j] = 0.f;
    for (int k = -R; k <= R; ++k) {
        const float w = a.taps.w[k < 0 ? -k : k];
        float v[TL_TZ];
#pragma unroll
        for (int j = 0; j < TL_TZ; ++j) v[j] = a.src[(int64_t)min(max(z0 + j + k, 0), a.nz - 1) * a.pz + col];
#pragma unroll
        for (int j = 0; j < TL_TZ; ++j) acc[j] = fmaf(w, v[j], acc[j]);
    }
    float pv[TL_TZ];
    if (a.dog != nullptr) {
#pragma unroll
        for (int j = 0; j < TL_TZ; ++j)
            pv[j] = ldf(static_cast<const S*>(a.prev) + (int64_t)min(z0 + j, a.nz - 1) * a.pz + col);
    }
#pragma unroll
    for (int j = 0; j < TL_TZ; ++j) {
        const int z = z0 + j;
        if (z >= a.nz) break;
        const int64_t off = (int64_t)z * a.pz + col;
        static_cast<S*>(a.dst)[off] = from_f32<S>(acc[j]);
        if (a.dog != nullptr) static_cast<S*>(a.dog)[off] = from_f32<S>(pv[j] - acc[j]);
    }
}

// Radius dispatch: the radii of the default scale schedule (initial 7, then
// 5 7 8 10 13, descriptor pre-blur 4) run the register-window bodies of the
// conv kernels; any other radius runs the generic loops above.
#define SIFT3D_TAIL_RADII(X) X(4) X(5) X(7) X(8) X(10) X(13)

// Each tile body is a separate (not inlined) function so that it gets its own
// register allocation; inlined into one kernel the bodies of all radii would
// be allocated together and spill.
template <int R, typename S, bool SUB, typename TB>
__device__ __noinline__ void xy_call(const ConvXYArgs& a, int bx, int by, int z, float* sm) {
    conv_detail::conv_xy_tile<R, S, SUB, TB>(a, bx, by, z, sm);
}
template <int R, typename S>
__device__ __noinline__ void z_call(const ConvZArgs& a, int64_t col, int z0) {
    conv_detail::conv_z_column<R, S, true, 0>(a, col, z0);
}
template <typename S>
__device__ __noinline__ void peak_call(const PeakArgs& a, int bx, int by, int bz, float* fl, unsigned* surv, int* n) {
    peak_detail::peak_tile<S>(a, bx, by, bz, fl, surv, *n);
}

template <typename S>
__device__ __forceinline__ void run_xy(const TailTask& t, int local, float* sm) {
    const ConvXYArgs& a = t.xy;
    const int tiles_x = (a.nx + TL_TX - 1) / TL_TX, tiles_y = (a.ny + TL_TY - 1) / TL_TY;
    const int bx = local % tiles_x, by = (local / tiles_x) % tiles_y, z = local / (tiles_x * tiles_y);
    const bool sub = t.type == TailTask::XY_SUB;
    if (sub) {   // only the first level of an octave sub-samples: radius 5 by default
        if (t.radius == 5) xy_call<5, S, true, S>(a, bx, by, z, sm);
        else xy_tile_generic<S>(a, t.radius, true, local, sm);
        return;
    }
    switch (t.radius) {
#define SIFT3D_XY_CASE(R)                                                    \
    case R:                                                                   \
        xy_call<R, S, false, float>(a, bx, by, z, sm);                        \
        return;
        SIFT3D_TAIL_RADII(SIFT3D_XY_CASE)
#undef SIFT3D_XY_CASE
        default:
            xy_tile_generic<S>(a, t.radius, false, local, sm);
    }
}

template <typename S>
__device__ __forceinline__ void run_z(const TailTask& t, int local) {
    const ConvZArgs& a = t.z;
    const int col_blocks = (int)((a.pz + TL_ZC - 1) / TL_ZC);
    const int64_t col = (int64_t)(local % col_blocks) * TL_ZC + threadIdx.x;
    const int z0 = (local / col_blocks) * TL_TZ;
    switch (t.radius) {
#define SIFT3D_Z_CASE(R)                                       \
    case R:                                                     \
        z_call<R, S>(a, col, z0);                               \
        return;
        SIFT3D_TAIL_RADII(SIFT3D_Z_CASE)
#undef SIFT3D_Z_CASE
        default:
            z_tile_generic<S>(a, t.radius, local);
    }
}

template <typename S>
__global__ void __launch_bounds__(TL_THREADS, 2) tail_kernel(const TailArgs t) {
    extern __shared__ float tl_sm[];
    for (int p = 0; p < t.n_phases; ++p) {
        const int b = t.phase_begin[p], e = t.phase_begin[p + 1];
        int total = 0;
        for (int i = b; i < e; ++i) total += t.tasks[i].n_tiles;
        for (int w = blockIdx.x; w < total; w += gridDim.x) {
            int i = b, local = w;
            while (local >= t.tasks[i].n_tiles) local -= t.tasks[i].n_tiles, ++i;
            const TailTask& task = t.tasks[i];
            switch (task.type) {
                case TailTask::XY:
                case TailTask::XY_SUB:
                    run_xy<S>(task, local, tl_sm);
                    break;
                case TailTask::Z:
                    run_z<S>(task, local);
                    break;
                case TailTask::PEAK: {
                    const int ix = (task.pk.nx - 2 * task.pk.border + peak_detail::PK_BX - 1) / peak_detail::PK_BX;
                    const int iy = (task.pk.ny - 2 * task.pk.border + peak_detail::PK_BY - 1) / peak_detail::PK_BY;
                    float* fl = tl_sm;
                    unsigned* surv = reinterpret_cast<unsigned*>(tl_sm + task.pk.n_scales * peak_detail::PK_LEVEL);
                    int& n_surv = *reinterpret_cast<int*>(surv + peak_detail::PK_SURV);
                    peak_call<S>(task.pk, local % ix, (local / ix) % iy, local / (ix * iy), fl, surv, &n_surv);
                    break;
                }
                default:
                    break;
            }
            __syncthreads();   // shared memory is reused by the next tile
        }
        if (p + 1 < t.n_phases && !grid_barrier(t.bar, t.err, (p + 1) * (int)gridDim.x)) return;
    }
}

}  // namespace

int tail_smem_bytes(int n_scales) {
    const int xy = conv_detail::XYGeom<kMaxRadius>::SMEM;
    const int pk = peak_detail::peak_smem_bytes(n_scales) + peak_detail::PK_SURV * 4 + 16;
    return std::max(xy, pk);
}

int tail_tiles(const TailTask& t) {
    switch (t.type) {
        case TailTask::XY:
        case TailTask::XY_SUB:
            return ((t.xy.nx + TL_TX - 1) / TL_TX) * ((t.xy.ny + TL_TY - 1) / TL_TY) * t.xy.nz;
        case TailTask::Z:
            return (int)((t.z.pz + TL_ZC - 1) / TL_ZC) * ((t.z.nz + TL_TZ - 1) / TL_TZ);
        case TailTask::PEAK: {
            const int b = t.pk.border;
            return ((t.pk.nx - 2 * b + peak_detail::PK_BX - 1) / peak_detail::PK_BX) *
                   ((t.pk.ny - 2 * b + peak_detail::PK_BY - 1) / peak_detail::PK_BY) *
                   ((t.pk.nz - 2 * b + peak_detail::PK_TZ - 1) / peak_detail::PK_TZ);
        }
    }
    return 0;
}

LaunchSpec tail_spec(int storage, int n_scales, int max_ctas) {
    LaunchSpec s;
    if (storage == SIFT3D_STORAGE_F32) s.func = reinterpret_cast<const void*>(&tail_kernel<float>);
    else if (storage == SIFT3D_STORAGE_F16) s.func = reinterpret_cast<const void*>(&tail_kernel<__half>);
    else s.func = reinterpret_cast<const void*>(&tail_kernel<__nv_bfloat16>);
    s.smem = tail_smem_bytes(n_scales);
    if (s.smem > 48 * 1024) cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s.func, TL_THREADS, s.smem);
    const int fit = std::max(1, sms * std::max(per_sm, 1));
    s.grid = dim3((unsigned)std::min(max_ctas * 2, fit));
    s.block = dim3(TL_THREADS);
    s.name = "tail";
    return s;
}

}  // namespace sift3d
