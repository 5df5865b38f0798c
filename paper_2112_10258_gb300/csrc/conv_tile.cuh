// Device bodies of the separable-convolution tiles (see conv.cu), shared by
// the conv kernels and the octave-tail kernel.
#pragma once

#include "common.cuh"

namespace sift3d {
namespace conv_detail {

constexpr int XY_TX = 64;
constexpr int XY_TY = 32;
constexpr int XY_J = 8;          // outputs per thread in each pass
constexpr int XY_THREADS = 256;
constexpr int Z_TZ = 16;
constexpr int Z_THREADS = 128;

template <int R>
struct XYGeom {
    static constexpr int W = XY_TX + 2 * R;         // staged columns
    static constexpr int H = XY_TY + 2 * R;         // staged rows
    static constexpr int WP = W | 1;                // odd pitch: no bank conflicts
    static constexpr int SMEM = (H + XY_TY) * WP * 4;
};

template <typename T>
__device__ __forceinline__ float load_f(const T* p) { return to_f32(*p); }

// One 64x32 tile (tile coordinates bx, by, plane z) by 256 threads.
template <int R, typename Tin, bool SUB, typename Tbase>
__device__ __forceinline__ void conv_xy_tile(const ConvXYArgs& a, int bx, int by, int z, float* sm) {
    using G = XYGeom<R>;
    float* in = sm;                       // H x WP staged source
    float* mid = sm + G::H * G::WP;       // TY x WP after the y pass
    const int x0 = bx * XY_TX;
    const int y0 = by * XY_TY;
    const Tin* src = static_cast<const Tin*>(a.src);
    if (a.zero_count != nullptr && x0 == 0 && y0 == 0 && z == 0 && threadIdx.x < kDetectCounters)
        a.zero_count[threadIdx.x] = 0;

    // Each thread issues its staging loads in groups that are all in flight
    // before the first shared-memory store.
    constexpr int N = G::H * G::W;
    constexpr int PER = (N + XY_THREADS - 1) / XY_THREADS;
    constexpr int GROUP = 8;
#pragma unroll
    for (int k0 = 0; k0 < PER; k0 += GROUP) {
        float vv[GROUP];
#pragma unroll
        for (int k = 0; k < GROUP; ++k) {
            const int i = threadIdx.x + (k0 + k) * XY_THREADS;
            if (k0 + k < PER && i < N) {
                const int r = i / G::W;
                const int c = i - r * G::W;
                const int gy = min(max(y0 - R + r, 0), a.ny - 1);
                const int gx = min(max(x0 - R + c, 0), a.nx - 1);
                if constexpr (!SUB) {
                    vv[k] = load_f(src + (int64_t)z * a.src_pz + (int64_t)gy * a.src_py + gx) * a.src_scale;
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
                    vv[k] = acc * 0.125f;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < GROUP; ++k) {
            const int i = threadIdx.x + (k0 + k) * XY_THREADS;
            if (k0 + k < PER && i < N) {
                const int r = i / G::W;
                const int c = i - r * G::W;
                in[r * G::WP + c] = vv[k];
                if constexpr (SUB) {
                    const int ty = r - R, tx = c - R;
                    if (ty >= 0 && ty < XY_TY && tx >= 0 && tx < XY_TX && y0 + ty < a.ny && x0 + tx < a.nx)
                        static_cast<Tbase*>(a.base_out)[(int64_t)z * a.pz + (int64_t)(y0 + ty) * a.py + x0 + tx] =
                            from_f32<Tbase>(vv[k]);
                }
            }
        }
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


// ---- full-row variant (nx <= 256): one thread per column, no x halo ----------
// The CTA stages rows y0-R .. y0+TY+R-1 (clamped) of one plane at full width;
// thread c filters column c along y from a register window (TY outputs), then
// each thread filters groups of 8 outputs along x reading shared memory with the
// column index clamped to [0, nx-1], which is the clamp-to-edge border.  No
// halo column is filtered and no thread covers a column beyond the row.
constexpr int ROW_MAX_NX = 256;
constexpr int ROW_J = 8;

__host__ __device__ constexpr int row_pitch(int nx) { return ((nx + 7) & ~7) | 1; }

template <int R, int TY>
__host__ __device__ constexpr int row_smem_bytes(int nx) {
    return (TY + 2 * R + TY) * row_pitch(nx) * 4;
}

template <typename Tin, bool SUB>
__device__ __forceinline__ float stage_value(const ConvXYArgs& a, const Tin* src, int z, int gy, int gx) {
    if constexpr (!SUB) {
        return load_f(src + (int64_t)z * a.src_pz + (int64_t)gy * a.src_py + gx) * a.src_scale;
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
        return acc * 0.125f;
    }
}


// Column col, planes z0 .. z0+TZ-1.
template <int R, typename S, bool COHERENT, int RB>
__device__ __forceinline__ void conv_z_column(const ConvZArgs& a, int64_t col, int z0) {
    // Columns are addressed linearly inside a plane (pitch layout, padding
    // columns included): the z pass does not care about x/y structure.  Each
    // thread holds TZ + 2R inputs of one column and, for the DoG, the TZ values
    // of G_{s-1}; every load is issued before the first store, so a thread waits
    // for memory once (the stores could alias the loads as far as the compiler
    // knows, which would otherwise serialise each output behind its own load).
    // COHERENT: plain loads (the octave-tail kernel rewrites its inputs between
    // phases, so the read-only path may not be used there).
    if (col >= a.pz) return;
    const bool with_dog = a.dog != nullptr;
    float v[Z_TZ + 2 * R];
#pragma unroll
    for (int t = 0; t < Z_TZ + 2 * R; ++t) {
        const int zz = min(max(z0 - R + t, 0), a.nz - 1);
        const float* p = a.src + (int64_t)zz * a.pz + col;
        v[t] = COHERENT ? *p : __ldg(p);
    }
    float u[RB > 0 ? Z_TZ + 2 * RB : 1];   // second intermediate (fused pre-blur)
    if constexpr (RB > 0) {
#pragma unroll
        for (int t = 0; t < Z_TZ + 2 * RB; ++t) {
            const int zz = min(max(z0 - RB + t, 0), a.nz - 1);
            const float* p = a.src2 + (int64_t)zz * a.pz + col;
            u[t] = COHERENT ? *p : __ldg(p);
        }
    }
    float pv[Z_TZ];
    if (with_dog) {
        const S* prev = static_cast<const S*>(a.prev);
#pragma unroll
        for (int j = 0; j < Z_TZ; ++j) {
            const int zz = min(z0 + j, a.nz - 1);
            pv[j] = to_f32(prev[(int64_t)zz * a.pz + col]);
        }
    }
    S* dst = static_cast<S*>(a.dst);
    S* dog = static_cast<S*>(a.dog);
#pragma unroll
    for (int j = 0; j < Z_TZ; ++j) {
        const int z = z0 + j;
        if (z >= a.nz) break;
        float acc = 0.f;
#pragma unroll
        for (int k = -R; k <= R; ++k) acc = fmaf(a.taps.w[k < 0 ? -k : k], v[j + R + k], acc);
        const int64_t off = (int64_t)z * a.pz + col;
        dst[off] = from_f32<S>(acc);
        if (with_dog) dog[off] = from_f32<S>(pv[j] - acc);
        if constexpr (RB > 0) {
            float acc2 = 0.f;
#pragma unroll
            for (int k = -RB; k <= RB; ++k) acc2 = fmaf(a.taps2.w[k < 0 ? -k : k], u[j + RB + k], acc2);
            static_cast<S*>(a.dst2)[off] = from_f32<S>(acc2);
        }
    }
}


}  // namespace conv_detail
}  // namespace sift3d
