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
//   conv_xy_row  (rows up to 256 wide) one CTA per 8 or 16 full rows of a
//            plane, column pairs in the y pass and row pairs in the x pass, each
//            tap one paired FP32 FMA (see below).
//   conv_z   one thread per two adjacent columns and TZ outputs along z: the
//            TZ + 2R inputs are loaded into registers (clamped z) and the TZ
//            outputs accumulate from registers.  The epilogue stores G_s and the
//            difference of Gaussians D_{s-1} = G_{s-1} - G_s (Sec. 2.2.2
//            "Difference-of-Gaussian") so the DoG costs no extra pass; at level S
//            (float32 storage) a variant also writes the next octave's G_0.
//   *_batch  the same bodies over the tiles of many volumes in one launch.
//
// Every 1D pass is out[i] = sum_{k=-R..R} w_|k| in[clamp(i+k)], summed in
// ascending k, in float32.
#include "conv_tile.cuh"

namespace sift3d {

namespace {

using namespace conv_detail;

template <int R, typename Tin, bool SUB, typename Tbase>
__global__ void __launch_bounds__(XY_THREADS) conv_xy_kernel(const ConvXYArgs a) {
    extern __shared__ float sm[];
    conv_xy_tile<R, Tin, SUB, Tbase>(a, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

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
template <int R, typename S, int RB, class A>
__device__ __forceinline__ void z_body(const A& a, const Taps& taps, const Taps& taps2, int pb, int zt) {
    using P = Pair<S>;
    using PT = typename P::T;
    constexpr bool narrow = sizeof(S) == 2;   // 16-bit storage: residuals travel with the levels
    const int64_t pair = (int64_t)pb * Z_THREADS + threadIdx.x;
    const int64_t pz2 = a.pz / 2;
    if (pair >= pz2) return;
    const int z0 = zt * Z_TZ;
    const bool interior = z0 - R >= 0 && z0 + Z_TZ + R <= a.nz;
    const bool with_dog = a.dog != nullptr;
    const bool with_res = a.res != nullptr;   // 16-bit storage of a level (null: descriptor pre-blur)
    float2 v[Z_TZ + 2 * R];
    load_z_window<Z_TZ + 2 * R, R>(reinterpret_cast<const float2*>(a.src) + pair, pz2, z0, a.nz, interior, v);
    // G_{s-1} as computed, before its rounding to storage: the stored value plus
    // its rounding residual (16-bit storage), so that the DoG carries no
    // storage rounding of G_{s-1}
    float2 pv[Z_TZ];
    const PT* prev = static_cast<const PT*>(a.prev) + pair;
    __half2* res = reinterpret_cast<__half2*>(a.res) + pair;
    if (with_dog) {
        if (z0 + Z_TZ <= a.nz) {   // walk the planes
            const PT* q = prev + (int64_t)z0 * pz2;
            const __half2* rq = res + (int64_t)z0 * pz2;
#pragma unroll
            for (int j = 0; j < Z_TZ; ++j) {
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
            for (int j = 0; j < Z_TZ; ++j) {
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
    for (int j = 0; j < Z_TZ; ++j) {
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
        float2 u[Z_TZ + 2 * RB];
        load_z_window<Z_TZ + 2 * RB, RB>(reinterpret_cast<const float2*>(a.src2) + pair, pz2, z0, a.nz,
                                         z0 - RB >= 0 && z0 + Z_TZ + RB <= a.nz, u);
        PT* dst2 = static_cast<PT*>(a.dst2) + pair + (int64_t)z0 * pz2;
#pragma unroll
        for (int j = 0; j < Z_TZ; ++j) {
            if (z0 + j >= a.nz) break;
            float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = -RB; k <= RB; ++k) acc2 = __ffma2_rn(f2(taps2.w[k < 0 ? -k : k]), u[j + RB + k], acc2);
            *dst2 = P::put(acc2);
            dst2 += pz2;
        }
    }
}

template <int R, typename S, int RB>
__global__ void __launch_bounds__(Z_THREADS) conv_z_kernel(const ConvZArgs a) {
    z_body<R, S, RB, ConvZArgs>(a, a.taps, a.taps2, blockIdx.x, blockIdx.y);
}

// z pass of level S (float32 storage, rows up to 256 wide) that also writes
// the next octave's G_0 (Sec. 2.2.2 "Sub-sampling": the mean of each 2x2x2
// block of G_S; a trailing odd voxel on an axis is dropped).  A CTA owns rows
// 2rp and 2rp+1 of a z tile (its py threads are the two rows' column pairs),
// parks its G_S values in shared memory and averages the blocks in the order
// (z, y, x), (z, y, x+1), (z, y+1, x), (z, y+1, x+1), then the same in z+1 -- the
// order of the sub-sampling y/x pass -- so the next octave gets the same bits
// without reading G_S back.
template <int R>
__global__ void __launch_bounds__(ROW_MAX_NX) conv_z_sub_kernel(const ConvZArgs a) {
    extern __shared__ __align__(16) float2 gsz[];   // [Z_TZ][py] G_S of the CTA's two rows
    const int rp = blockIdx.x, zt = blockIdx.y, t = threadIdx.x;
    const int py = (int)a.py;                       // = blockDim.x
    const int64_t pz2 = a.pz / 2;
    const int64_t pair = (int64_t)rp * py + t;      // rows 2rp, 2rp+1 hold py pairs
    const int z0 = zt * Z_TZ;
    if (pair < pz2) {   // the second row of an odd last row pair does not exist
        const bool interior = z0 - R >= 0 && z0 + Z_TZ + R <= a.nz;
        float2 v[Z_TZ + 2 * R];
        load_z_window<Z_TZ + 2 * R, R>(reinterpret_cast<const float2*>(a.src) + pair, pz2, z0, a.nz, interior, v);
        float2 pv[Z_TZ];
        const float2* prev = static_cast<const float2*>(a.prev) + pair;
#pragma unroll
        for (int j = 0; j < Z_TZ; ++j) pv[j] = prev[(int64_t)min(z0 + j, a.nz - 1) * pz2];
        float2* dst = static_cast<float2*>(a.dst) + pair + (int64_t)z0 * pz2;
        float2* dog = reinterpret_cast<float2*>(a.dog) + pair + (int64_t)z0 * pz2;
#pragma unroll
        for (int j = 0; j < Z_TZ; ++j) {
            if (z0 + j >= a.nz) break;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = -R; k <= R; ++k) acc = __ffma2_rn(f2(a.taps.w[k < 0 ? -k : k]), v[j + R + k], acc);
            *dst = acc;
            *dog = make_float2(pv[j].x - acc.x, pv[j].y - acc.y);
            gsz[j * py + t] = acc;
            dst += pz2;
            dog += pz2;
        }
    }
    __syncthreads();
    const int nxs = a.nx / 2, nys = a.ny / 2, nzs = a.nz / 2;
    if (rp >= nys) return;
    const int zo0 = z0 / 2;
    const int nzo = min(Z_TZ / 2, nzs - zo0);
    const int half = py / 2;   // pairs per row
    for (int item = t; item < nzo * nxs; item += blockDim.x) {
        const int k = item / nxs, xo = item - k * nxs;
        const float2 a0 = gsz[2 * k * py + xo], a1 = gsz[2 * k * py + half + xo];
        const float2 b0 = gsz[(2 * k + 1) * py + xo], b1 = gsz[(2 * k + 1) * py + half + xo];
        float m = 0.f;
        m += a0.x;
        m += a0.y;
        m += a1.x;
        m += a1.y;
        m += b0.x;
        m += b0.y;
        m += b1.x;
        m += b1.y;
        a.sub_dst[(int64_t)(zo0 + k) * a.sub_pz + (int64_t)rp * a.sub_py + xo] = m * 0.125f;
    }
}

// Batched: one flat list of (volume, column block, z tile) items.
template <int R, typename S, int RB>
__global__ void __launch_bounds__(Z_THREADS) conv_z_batch(const __grid_constant__ BatchZ b) {
    {
        const int item = blockIdx.x;
        const int v = batch_param_volume(b.prefix, b.n, item);
        const ZVol& a = b.vol[v];   // read in place from the kernel parameters
        const int local = item - b.prefix[v];
        const int cols = (int)((a.pz / 2 + Z_THREADS - 1) / Z_THREADS);
        z_body<R, S, RB, ZVol>(a, b.taps, b.taps2, local % cols, local / cols);
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

template <int R, int MODE, typename Tin, typename Tbase, int RB>
__global__ void __launch_bounds__(ROW_MAX_NX) conv_xy_row_kernel(const ConvXYArgs a) {
    extern __shared__ __align__(16) float2 rows_sm[];
    row_body<R, MODE, Tin, Tbase, RB, ConvXYArgs>(a, a.taps, a.taps2, blockIdx.x, blockIdx.y, rows_sm);
}

// Batched: the CTAs walk the tiles of every volume of the batch (grid-stride
// over one flat tile list; a tile's volume is found in the prefix sums).
template <int R, int MODE, typename Tin, typename Tbase, int RB>
__global__ void __launch_bounds__(ROW_MAX_NX) conv_xy_row_batch(const __grid_constant__ BatchXY b) {
    extern __shared__ __align__(16) float2 rows_sm[];
    {
        const int item = blockIdx.x;
        const int v = batch_param_volume(b.prefix, b.n, item);
        const XYVol& a = b.vol[v];   // read in place from the kernel parameters
        const int local = item - b.prefix[v];
        const int nyb = (a.ny + a.row_tile - 1) / a.row_tile;
        row_body<R, MODE, Tin, Tbase, RB, XYVol>(a, b.taps, b.taps2, local % nyb, local / nyb, rows_sm);
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

template <int MODE, typename Tin, typename Tbase, int... Rs>
const void* row_func_table(int r, int nx, int ty, int* smem, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_xy_row_kernel<Rs + 1, MODE, Tin, Tbase, 0>)...};
    *smem = row_smem(nx, r, 0, ty);
    return fns[r - 1];
}

template <int... Rs>
const void* z_sub_func_table(int r, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_sub_kernel<Rs + 1>)...};
    return fns[r - 1];
}

template <typename S, int... Rs>
const void* z_func_table(int r, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_kernel<Rs + 1, S, 0>)...};
    return fns[r - 1];
}

using BlurRadiusSeq = std::make_integer_sequence<int, kMaxRadius - kFusedBlurRadius + 1>;

using RadiusSeq = std::make_integer_sequence<int, kMaxRadius>;

template <typename Tin, bool SUB, typename Tbase>
const void* xy_func(int r, int* smem) {
    return xy_func_table<Tin, SUB, Tbase>(r, smem, RadiusSeq{});
}

template <int MODE, typename Tin, typename Tbase>
const void* row_func(int r, int nx, int ty, int* smem) {
    return row_func_table<MODE, Tin, Tbase>(r, nx, ty, smem, RadiusSeq{});
}

// Batched instances: float32 storage (float32 or uint8 input).
template <int MODE, typename Tin, int... Rs>
const void* row_batch_table(int r, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_xy_row_batch<Rs + 1, MODE, Tin, float, 0>)...};
    return fns[r - 1];
}

template <int... Rs>
const void* row_blur_batch_table(int r, std::integer_sequence<int, Rs...>) {
    constexpr int RB = kFusedBlurRadius;
    const void* fns[] = {reinterpret_cast<const void*>(&conv_xy_row_batch<Rs + RB, 0, float, float, RB>)...};
    return r < RB ? nullptr : fns[r - RB];
}

template <int... Rs>
const void* z_batch_table(int r, std::integer_sequence<int, Rs...>) {
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_batch<Rs + 1, float, 0>)...};
    return fns[r - 1];
}

template <int... Rs>
const void* z_blur_batch_table(int r, std::integer_sequence<int, Rs...>) {
    constexpr int RB = kFusedBlurRadius;
    const void* fns[] = {reinterpret_cast<const void*>(&conv_z_batch<Rs + RB, float, RB>)...};
    return r < RB ? nullptr : fns[r - RB];
}


}  // namespace

LaunchSpec conv_xy_spec(int radius, int src_kind, int storage, bool sub, ConvXYArgs& a) {
    LaunchSpec s;
    int smem = 0;
    if (radius < 1 || radius > kMaxRadius) return s;
    if (a.row_tile != 8 && a.row_tile != 16) a.row_tile = ROW_TY;
    const int ty = a.row_tile;
    if (a.dst2 != nullptr) return s;   // the fused descriptor pre-blur exists in the batched kernels only
    if (a.nx <= ROW_MAX_NX) {
        if (!sub) {
            if (src_kind == 0) s.func = row_func<1, float, float>(radius, a.nx, ty, &smem);
            else if (src_kind == 1) s.func = row_func<1, uint8_t, float>(radius, a.nx, ty, &smem);
            else if (storage == SIFT3D_STORAGE_F32) s.func = row_func<0, float, float>(radius, a.nx, ty, &smem);
            else if (storage == SIFT3D_STORAGE_F16) s.func = row_func<0, __half, float>(radius, a.nx, ty, &smem);
            else s.func = row_func<0, __nv_bfloat16, float>(radius, a.nx, ty, &smem);
        } else {
            if (storage == SIFT3D_STORAGE_F32) s.func = row_func<2, float, float>(radius, a.nx, ty, &smem);
            else if (storage == SIFT3D_STORAGE_F16) s.func = row_func<2, __half, __half>(radius, a.nx, ty, &smem);
            else s.func = row_func<2, __nv_bfloat16, __nv_bfloat16>(radius, a.nx, ty, &smem);
        }
        if (smem > 48 * 1024) cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        s.grid = dim3((a.ny + ty - 1) / ty, a.nz, 1);
        s.block = dim3(row_threads(a.nx, ty));
        s.smem = smem;
        s.name = sub ? "conv_xy_sub" : "conv_xy";
        return s;
    }
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
    if (a.dst2 != nullptr) return s;   // the fused descriptor pre-blur exists in the batched kernels only
    if (a.sub_dst != nullptr) {        // level S writing the next octave's G_0
        if (storage != SIFT3D_STORAGE_F32 || a.dog == nullptr || a.py > ROW_MAX_NX || a.py % 2 != 0) return s;
        s.func = z_sub_func_table(radius, RadiusSeq{});
        s.grid = dim3((unsigned)((a.ny + 1) / 2), (a.nz + Z_TZ - 1) / Z_TZ, 1);
        s.block = dim3((unsigned)a.py);
        s.smem = (size_t)Z_TZ * a.py * sizeof(float2);
        s.name = "conv_z_dog_sub";
        return s;
    }
    if (storage == SIFT3D_STORAGE_F32) s.func = z_func_table<float>(radius, RadiusSeq{});
    else if (storage == SIFT3D_STORAGE_F16) s.func = z_func_table<__half>(radius, RadiusSeq{});
    else s.func = z_func_table<__nv_bfloat16>(radius, RadiusSeq{});
    s.grid = dim3((unsigned)((a.pz / 2 + Z_THREADS - 1) / Z_THREADS), (a.nz + Z_TZ - 1) / Z_TZ, 1);
    s.block = dim3(Z_THREADS);
    s.smem = 0;
    s.name = a.dog ? "conv_z_dog" : "conv_z";
    return s;
}

}  // namespace sift3d

namespace sift3d {

LaunchSpec conv_xy_batch_spec(int radius, int src_kind, bool sub, bool blur, int nx_max, int row_tile, int total) {
    LaunchSpec s;
    if (radius < 1 || radius > kMaxRadius || nx_max > ROW_MAX_NX) return s;
    const int ty = row_tile;
    if (blur) {
        if (sub || src_kind != 2) return s;
        s.func = row_blur_batch_table(radius, BlurRadiusSeq{});
    } else if (sub) {
        s.func = row_batch_table<2, float>(radius, RadiusSeq{});
    } else if (src_kind == 0) {
        s.func = row_batch_table<1, float>(radius, RadiusSeq{});
    } else if (src_kind == 1) {
        s.func = row_batch_table<1, uint8_t>(radius, RadiusSeq{});
    } else {
        s.func = row_batch_table<0, float>(radius, RadiusSeq{});
    }
    if (s.func == nullptr) return s;
    const int smem = row_smem(nx_max, radius, blur ? kFusedBlurRadius : 0, ty);
    if (smem > 48 * 1024) cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    s.block = dim3(row_threads(nx_max, ty));
    s.smem = smem;
    s.grid = dim3((unsigned)std::max(1, total));   // one tile per CTA
    s.name = blur ? "conv_xy_blur_batch" : (sub ? "conv_xy_sub_batch" : "conv_xy_batch");
    return s;
}

LaunchSpec conv_z_batch_spec(int radius, bool blur, int total) {
    LaunchSpec s;
    if (radius < 1 || radius > kMaxRadius) return s;
    s.func = blur ? z_blur_batch_table(radius, BlurRadiusSeq{}) : z_batch_table(radius, RadiusSeq{});
    if (s.func == nullptr) return s;
    s.block = dim3(Z_THREADS);
    s.grid = dim3((unsigned)std::max(1, total));   // one tile per CTA
    s.name = blur ? "conv_z_dog_blur_batch" : "conv_z_dog_batch";
    return s;
}

// Work items of one volume in a batched pass.
int conv_xy_items(const ConvXYArgs& a) { return ((a.ny + a.row_tile - 1) / a.row_tile) * a.nz; }
int conv_z_items(const ConvZArgs& a) {
    return (int)((a.pz / 2 + Z_THREADS - 1) / Z_THREADS) * ((a.nz + Z_TZ - 1) / Z_TZ);
}

}  // namespace sift3d
