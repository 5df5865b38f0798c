// Tile body of the y/x pass for rows wider than 256 (instantiated in
// conv_xy_tile.cu) and the constants the conv kernels share.
#pragma once

#include "common.cuh"

namespace sift3d {
namespace conv_detail {

constexpr int XY_TX = 64;
constexpr int XY_TY = 32;
constexpr int XY_J = 8;          // outputs per thread in each pass
constexpr int XY_THREADS = 256;
constexpr int Z_TZ = 16;          // conv_z outputs per thread
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
                    if (ty >= 0 && ty < XY_TY && tx >= 0 && tx < XY_TX && y0 + ty < a.ny && x0 + tx < a.nx) {
                        const int64_t o = (int64_t)z * a.pz + (int64_t)(y0 + ty) * a.py + x0 + tx;
                        const Tbase g = from_f32<Tbase>(vv[k]);
                        static_cast<Tbase*>(a.base_out)[o] = g;
                        if constexpr (sizeof(Tbase) == 2)   // rounding residual of the stored G_0
                            a.res_out[o] = __float2half_rn(vv[k] - to_f32(g));
                    }
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


// Rows up to this width take the full-row kernel (conv.cu); wider ones the tiles above.
constexpr int ROW_MAX_NX = 256;
constexpr int ROW_J = 8;          // outputs per thread of the full-row x pass

}  // namespace conv_detail
}  // namespace sift3d
