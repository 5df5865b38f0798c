// Device bodies of the separable Gaussian passes (see conv.cu for the
// overview), shared by the translation units that instantiate them: conv.cu
// (y/x passes), conv_z.cu (z passes) and conv_batch.cu (batched passes), which
// compile in parallel.
#pragma once

#include <utility>

#include "conv_tile.cuh"

namespace sift3d {
namespace conv_detail {

// ---- z pass on column pairs with paired FP32 FMAs ---------------------------
// A thread owns two adjacent columns (pitched rows hold a multiple of 8
// elements, so a pair never straddles a row) and TZ outputs along z.  Loads and
// stores move both columns at once, and each tap is one __ffma2_rn for the
// pair: per column this is exactly the scalar chain acc = fmaf(w_|k|, in, acc)
// in ascending k, so results are bitwise those of a one-column-per-thread pass.
template <typename S> struct Pair;
template <> struct Pair<float> {
    using T = float2;
    static __device__ __forceinline__ float2 get(T v) { return v; }
    static __device__ __forceinline__ T put(float2 v) { return v; }
};
template <> struct Pair<__half> {
    using T = __half2;
    static __device__ __forceinline__ float2 get(T v) { return __half22float2(v); }
    static __device__ __forceinline__ T put(float2 v) { return __floats2half2_rn(v.x, v.y); }
};
template <> struct Pair<__nv_bfloat16> {
    using T = __nv_bfloat162;
    static __device__ __forceinline__ float2 get(T v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ T put(float2 v) { return __floats2bfloat162_rn(v.x, v.y); }
};

__device__ __forceinline__ float2 f2(float w) { return make_float2(w, w); }

// Loads the TZ + 2R inputs of a column pair, z clamped to [0, nz-1]; the
// branch on `interior` is uniform over the CTA.
template <int N, int R>
__device__ __forceinline__ void load_z_window(const float2* src, int64_t pz2, int z0, int nz, bool interior,
                                              float2 (&v)[N]) {
    if (interior) {   // walk the planes
        const float2* p = src + (int64_t)(z0 - R) * pz2;
#pragma unroll
        for (int t = 0; t < N; ++t) {
            v[t] = __ldg(p);
            p += pz2;
        }
    } else {
#pragma unroll
        for (int t = 0; t < N; ++t) v[t] = __ldg(src + (int64_t)min(max(z0 - R + t, 0), nz - 1) * pz2);
    }
}

// A: ConvZArgs, or the batched ZVol (the same field names, no taps).
template <int R, typename S, int RB, class A, int TZ = Z_TZ>
__device__ __forceinline__ void z_body(const A& a, const Taps& taps, const Taps& taps2, int pb, int zt) {
    using P = Pair<S>;
    using PT = typename P::T;
    constexpr bool narrow = sizeof(S) == 2;   // 16-bit storage: residuals travel with the levels
    const int64_t pair = (int64_t)pb * Z_THREADS + threadIdx.x;
    const int64_t pz2 = a.pz / 2;
    if (pair >= pz2) return;
    const int z0 = zt * TZ;
    const bool interior = z0 - R >= 0 && z0 + TZ + R <= a.nz;
    const bool with_dog = a.dog != nullptr;
    const bool with_res = a.res != nullptr;   // 16-bit storage of a level (null: descriptor pre-blur)
    float2 v[TZ + 2 * R];
    load_z_window<TZ + 2 * R, R>(reinterpret_cast<const float2*>(a.src) + pair, pz2, z0, a.nz, interior, v);
    // G_{s-1} as computed, before its rounding to storage: the stored value plus
    // its rounding residual (16-bit storage), so that the DoG carries no
    // storage rounding of G_{s-1}
    float2 pv[TZ];
    const PT* prev = static_cast<const PT*>(a.prev) + pair;
    __half2* res = reinterpret_cast<__half2*>(a.res) + pair;
    if (with_dog) {
        if (z0 + TZ <= a.nz) {   // walk the planes
            const PT* q = prev + (int64_t)z0 * pz2;
            const __half2* rq = res + (int64_t)z0 * pz2;
#pragma unroll
            for (int j = 0; j < TZ; ++j) {
                pv[j] = P::get(*q);
                q += pz2;
                if constexpr (narrow) {
                    const float2 r = __half22float2(*rq);
                    pv[j] = make_float2(pv[j].x + r.x, pv[j].y + r.y);
                    rq += pz2;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < TZ; ++j) {
                const int64_t zo = (int64_t)min(z0 + j, a.nz - 1) * pz2;
                pv[j] = P::get(prev[zo]);
                if constexpr (narrow) {
                    const float2 r = __half22float2(res[zo]);
                    pv[j] = make_float2(pv[j].x + r.x, pv[j].y + r.y);
                }
            }
        }
    }
    PT* dst = static_cast<PT*>(a.dst) + pair + (int64_t)z0 * pz2;
    float2* dog = reinterpret_cast<float2*>(a.dog) + pair + (int64_t)z0 * pz2;
    __half2* rout = res + (int64_t)z0 * pz2;
#pragma unroll
    for (int j = 0; j < TZ; ++j) {
        if (z0 + j >= a.nz) break;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = -R; k <= R; ++k) acc = __ffma2_rn(f2(taps.w[k < 0 ? -k : k]), v[j + R + k], acc);
        const PT g = P::put(acc);
        *dst = g;
        if constexpr (narrow) {   // acc - stored value, exact in float32 (levels only: the
            if (with_res) {       // descriptor pre-blur keeps no residual)
                const float2 gs = P::get(g);
                *rout = __floats2half2_rn(acc.x - gs.x, acc.y - gs.y);
            }
        }
        if (with_dog) *dog = make_float2(pv[j].x - acc.x, pv[j].y - acc.y);
        dst += pz2;
        dog += pz2;
        rout += pz2;
    }
    if constexpr (RB > 0) {   // the fused descriptor pre-blur, after the level so registers are reused
        float2 u[TZ + 2 * RB];
        load_z_window<TZ + 2 * RB, RB>(reinterpret_cast<const float2*>(a.src2) + pair, pz2, z0, a.nz,
                                         z0 - RB >= 0 && z0 + TZ + RB <= a.nz, u);
        PT* dst2 = static_cast<PT*>(a.dst2) + pair + (int64_t)z0 * pz2;
#pragma unroll
        for (int j = 0; j < TZ; ++j) {
            if (z0 + j >= a.nz) break;
            float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = -RB; k <= RB; ++k) acc2 = __ffma2_rn(f2(taps2.w[k < 0 ? -k : k]), u[j + RB + k], acc2);
            *dst2 = P::put(acc2);
            dst2 += pz2;
        }
    }
}

// ---- y/x pass of full rows (nx <= 256) with paired FP32 FMAs -----------------
// One CTA filters rows y0 .. y0+15 of one plane, full width.
//   y pass: a task owns a column pair and 8 output rows; it loads the 8 + 2R
//           source rows (clamped y; a task whose rows all lie inside the plane
//           walks a row pointer instead) into registers and filters both
//           columns at once with __ffma2_rn.  Results go to shared memory as row pairs:
//           element [rp][c] holds (row 2rp, row 2rp+1) of column c, so the x
//           pass reads two rows with one 8-byte access.
//   aprons: each row-pair line carries RA = R + (R & 1) copies of column 0 on
//           the left and copies of column nx-1 on the right, which is the
//           clamp-to-edge border: the x pass reads without index clamps.  A
//           warp fills one line at a time, lanes along it.
//   x pass: a task owns a row pair and 8 output columns; it reads its window
//           with 16-byte shared loads and filters both rows at once.
// Per column and row every output is the scalar chain fmaf(w_|k|, in, acc) in
// ascending k, so the pairing changes no result bit.
// MODE 0: source is a pitched pyramid level (storage type Tin), read in pairs;
// MODE 1: source is the caller's dense volume (float32 or uint8, row pitch nx);
// MODE 2: source is the previous octave's level S, each value the 2x2x2 mean
//         (Sec. 2.2.2 "Sub-sampling"), and the CTA's own rows of the means are
//         written to base_out as the octave's G_0.
constexpr int RY = 8;                 // rows per y task
constexpr int ROW_TY = 2 * RY;        // default rows per CTA (ConvXYArgs.row_tile: 8 or 16)

__host__ __device__ constexpr int row_apron(int R) { return R + (R & 1); }

// Row-pair line length in float2: window reads stay inside, and it is 2 mod 4
// so that 8 lanes reading 8 different lines at one column hit 8 distinct
// 16-byte bank groups.
__host__ __device__ constexpr int row_line(int nx, int R) {
    const int w = 8 * ((nx + 7) / 8) + 2 * R + 4;
    return w + ((2 - (w & 3)) & 3);
}

__host__ __device__ constexpr int row_smem(int nx, int R, int RB, int ty) {
    return (RB > 0 ? 2 : 1) * (ty / 2) * row_line(nx, R) * 8;
}

// Threads of a row CTA of ty rows (8 or 16): enough for every y task (column
// pair x RY rows, at most 256 for nx <= 256) in one round; the x pass loops
// over its tasks (row pair x 8 columns).
__host__ __device__ constexpr int row_threads(int nx, int ty) {
    const int pairs = (nx + 1) / 2, groups = (nx + 7) / 8;
    const int ytasks = pairs * (ty / RY), xtasks = (ty / 2) * groups;
    const int t = ((ytasks > xtasks ? ytasks : xtasks) + 31) / 32 * 32;
    return t < ROW_MAX_NX ? t : ROW_MAX_NX;
}

template <typename Tin>
__device__ __forceinline__ float sub_mean(const Tin* p, int64_t py, int64_t pz) {
    float acc = 0.f;
    acc += load_f(p);
    acc += load_f(p + 1);
    acc += load_f(p + py);
    acc += load_f(p + py + 1);
    acc += load_f(p + pz);
    acc += load_f(p + pz + 1);
    acc += load_f(p + pz + py);
    acc += load_f(p + pz + py + 1);
    return acc * 0.125f;
}

// Source values of columns (c, c+1) at row gy of plane z (MODE as above); the
// second column repeats the first when c+1 is beyond the row (odd nx).
template <int MODE, typename Tin, class A>
__device__ __forceinline__ float2 load_src_pair(const A& a, const Tin* src, int z, int gy, int c, bool full) {
    if constexpr (MODE == 0) {
        using PT = typename Pair<Tin>::T;
        return Pair<Tin>::get(*reinterpret_cast<const PT*>(src + (int64_t)z * a.src_pz + (int64_t)gy * a.src_py + c));
    } else if constexpr (MODE == 1) {
        const Tin* r = src + (int64_t)z * a.src_pz + (int64_t)gy * a.src_py;
        const float v0 = load_f(r + c) * a.src_scale;
        return make_float2(v0, full ? load_f(r + c + 1) * a.src_scale : v0);
    } else {
        const Tin* p = src + (int64_t)(2 * z) * a.src_pz + (int64_t)(2 * gy) * a.src_py + 2 * c;
        const float v0 = sub_mean(p, a.src_py, a.src_pz);
        return make_float2(v0, full ? sub_mean(p + 2, a.src_py, a.src_pz) : v0);
    }
}

// x pass of one row pair over columns x0 .. x0+7 with radius RK from a line
// whose apron is row_apron(RW); stores row 2rp to dst0 and row 2rp+1 to dst1
// (null: beyond the volume).
template <int RW, int RK>
__device__ __forceinline__ void x_pass_rows(const float2* line, const Taps& taps, int x0, float* dst0, float* dst1) {
    constexpr int AK = row_apron(RK);
    constexpr int NE = (ROW_J + 2 * RK + (RK & 1) + 1) & ~1;   // window length (float2), even
    float2 win[NE];                                          // win[i] is column x0 - AK + i
    const float4* l4 = reinterpret_cast<const float4*>(line + x0 + row_apron(RW) - AK);
#pragma unroll
    for (int q = 0; q < NE / 2; ++q) {
        const float4 t = l4[q];
        win[2 * q] = make_float2(t.x, t.y);
        win[2 * q + 1] = make_float2(t.z, t.w);
    }
    float2 o[ROW_J];
#pragma unroll
    for (int j = 0; j < ROW_J; ++j) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = -RK; k <= RK; ++k) acc = __ffma2_rn(f2(taps.w[k < 0 ? -k : k]), win[j + AK + k], acc);
        o[j] = acc;
    }
    reinterpret_cast<float4*>(dst0)[0] = make_float4(o[0].x, o[1].x, o[2].x, o[3].x);
    reinterpret_cast<float4*>(dst0)[1] = make_float4(o[4].x, o[5].x, o[6].x, o[7].x);
    if (dst1 != nullptr) {
        reinterpret_cast<float4*>(dst1)[0] = make_float4(o[0].y, o[1].y, o[2].y, o[3].y);
        reinterpret_cast<float4*>(dst1)[1] = make_float4(o[4].y, o[5].y, o[6].y, o[7].y);
    }
}

// RB > 0: also filter the same source rows with the descriptor pre-blur
// (radius RB <= R, taps2) into dst2.
// A: ConvXYArgs, or the batched XYVol (the same field names, no taps).
template <int R, int MODE, typename Tin, typename Tbase, int RB, class A>
__device__ __forceinline__ void row_body(const A& a, const Taps& taps, const Taps& taps2, int yb, int z,
                                         float2* rows_sm) {
    static_assert(RB <= R, "the fused pre-blur reads inside the staged halo");
    const int nx = a.nx;
    const int W = row_line(nx, R);
    constexpr int RA = row_apron(R);
    const int ty = a.row_tile;                          // rows of this CTA: 8 or 16
    const int lg_lines = ty == 16 ? 3 : 2;              // log2 of the row-pair lines (no divisions below)
    const int nlines = 1 << lg_lines;
    float2* mid = rows_sm;                              // [nlines][W]
    float2* mid2 = rows_sm + nlines * W;                // same, pre-blur (RB > 0)
    const int y0 = yb * ty;
    const int tid = threadIdx.x;
    const Tin* src = static_cast<const Tin*>(a.src);
    if (a.zero_count != nullptr && y0 == 0 && z == 0 && tid < kDetectCounters) a.zero_count[tid] = 0;

    // y pass
    const int pairs = (nx + 1) / 2;
    if (tid < pairs * (ty / RY)) {   // one y task per thread (row_threads guarantees enough threads)
        const int task = tid;
        const int h = task / pairs, p = task - h * pairs;
        const int c = 2 * p, r0 = h * RY;
        const bool full = c + 1 < nx;
        const int gy0 = y0 + r0 - R;   // first source row
        float2 v[RY + 2 * R];
        bool walked = false;
        if constexpr (MODE == 0) {
            if (gy0 >= 0 && gy0 + RY + 2 * R <= a.ny) {
                // rows inside the plane: walk them without clamps (pitch in pairs)
                using PT = typename Pair<Tin>::T;
                const PT* q = reinterpret_cast<const PT*>(src + (int64_t)z * a.src_pz + (int64_t)gy0 * a.src_py + c);
                const int64_t step = a.src_py / 2;
#pragma unroll
                for (int t = 0; t < RY + 2 * R; ++t) {
                    v[t] = Pair<Tin>::get(*q);
                    q += step;
                }
                walked = true;
            }
        } else if constexpr (MODE == 1) {
            if (gy0 >= 0 && gy0 + RY + 2 * R <= a.ny) {   // rows inside: walk them without clamps
                const Tin* q = src + (int64_t)z * a.src_pz + (int64_t)gy0 * a.src_py + c;
#pragma unroll
                for (int t = 0; t < RY + 2 * R; ++t) {
                    const float v0 = load_f(q) * a.src_scale;
                    v[t] = make_float2(v0, full ? load_f(q + 1) * a.src_scale : v0);
                    q += a.src_py;
                }
                walked = true;
            }
        }
        if (!walked) {
#pragma unroll
            for (int t = 0; t < RY + 2 * R; ++t)
                v[t] = load_src_pair<MODE, Tin, A>(a, src, z, min(max(gy0 + t, 0), a.ny - 1), c, full);
        }
        if constexpr (MODE == 2) {   // this CTA's own rows of the sub-sampled level are G_0
            using PB = Pair<Tbase>;
#pragma unroll
            for (int j = 0; j < RY; ++j)
                if (y0 + r0 + j < a.ny) {
                    const int64_t o = (int64_t)z * a.pz + (int64_t)(y0 + r0 + j) * a.py + c;
                    const typename PB::T g = PB::put(v[R + j]);
                    reinterpret_cast<typename PB::T*>(static_cast<Tbase*>(a.base_out) + o)[0] = g;
                    if constexpr (sizeof(Tbase) == 2) {   // rounding residual of the stored G_0
                        const float2 gs = PB::get(g);
                        reinterpret_cast<__half2*>(a.res_out + o)[0] =
                            __floats2half2_rn(v[R + j].x - gs.x, v[R + j].y - gs.y);
                    }
                }
        }
#pragma unroll
        for (int j = 0; j < RY; j += 2) {
            float2 e = make_float2(0.f, 0.f), f = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = -R; k <= R; ++k) {
                const float2 w = f2(taps.w[k < 0 ? -k : k]);
                e = __ffma2_rn(w, v[j + R + k], e);
                f = __ffma2_rn(w, v[j + 1 + R + k], f);
            }
            reinterpret_cast<float4*>(mid + ((r0 + j) / 2) * W + RA + c)[0] = make_float4(e.x, f.x, e.y, f.y);
            if constexpr (RB > 0) {
                e = make_float2(0.f, 0.f);
                f = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = -RB; k <= RB; ++k) {
                    const float2 w = f2(taps2.w[k < 0 ? -k : k]);
                    e = __ffma2_rn(w, v[j + R + k], e);
                    f = __ffma2_rn(w, v[j + 1 + R + k], f);
                }
                reinterpret_cast<float4*>(mid2 + ((r0 + j) / 2) * W + RA + c)[0] = make_float4(e.x, f.x, e.y, f.y);
            }
        }
    }
    __syncthreads();
    // aprons: left copies of column 0, right copies of column nx-1 (this also
    // overwrites the duplicate a pair wrote at column nx for odd nx)
    {
        const int right = W - (RA + nx);
        const int per_line = RA + right;
        const int nb = RB > 0 ? 2 : 1;
        const int lane = tid & 31, nwarps = blockDim.x >> 5;   // blockDim.x is a multiple of 32
        for (int l = tid >> 5; l < nb * nlines; l += nwarps) {   // a warp per line
            float2* line = (l < nlines ? mid : mid2) + (l & (nlines - 1)) * W;
            for (int e = lane; e < per_line; e += 32) {
                if (e < RA) line[e] = line[RA];
                else line[RA + nx + (e - RA)] = line[RA + nx - 1];
            }
        }
    }
    __syncthreads();

    // x pass
    const int groups = (nx + ROW_J - 1) / ROW_J;
    for (int item = tid; item < nlines * groups; item += blockDim.x) {
        const int rp = item & (nlines - 1);
        const int g = item >> lg_lines;
        const int x0 = g * ROW_J;
        const int y = y0 + 2 * rp;
        if (y >= a.ny) continue;
        const int64_t off = (int64_t)z * a.pz + (int64_t)y * a.py + x0;
        const bool second = y + 1 < a.ny;
        x_pass_rows<R, R>(mid + rp * W, taps, x0, a.dst + off, second ? a.dst + off + a.py : nullptr);
        if constexpr (RB > 0)
            x_pass_rows<R, RB>(mid2 + rp * W, taps2, x0, a.dst2 + off, second ? a.dst2 + off + a.py : nullptr);
    }
}

using BlurRadiusSeq = std::make_integer_sequence<int, kMaxRadius - kFusedBlurRadius + 1>;

using RadiusSeq = std::make_integer_sequence<int, kMaxRadius>;

}  // namespace conv_detail

// The y/x pass over 64x32 tiles for rows wider than 256 (conv_xy_tile.cu).
LaunchSpec conv_xy_tile_spec(int radius, int src_kind, int storage, bool sub, const ConvXYArgs& a);

}  // namespace sift3d
