// Device code of one peak-detection tile (see peak.cu), shared by the peak
// kernel and the octave-tail kernel.
#pragma once

#include "common.cuh"

namespace sift3d {
namespace peak_detail {

constexpr int PK_BX = 32;
constexpr int PK_BY = 8;
constexpr int PK_THREADS = PK_BX * PK_BY;

// The 80 neighbours as (dx, dy, dz, level offset): the 26 of D_s first (faces,
// then edges, then corners: the likeliest to break an extremum early), then the
// 27 of D_{s-1} and the 27 of D_{s+1}.
struct NbrTable {
    int v[80][4];
};

__host__ __device__ constexpr NbrTable make_nbr_table() {
    NbrTable t{};
    int n = 0;
    for (int order = 1; order <= 3; ++order)          // number of non-zero offsets
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int m = (dx != 0) + (dy != 0) + (dz != 0);
                    if (m == order) {
                        t.v[n][0] = dx, t.v[n][1] = dy, t.v[n][2] = dz, t.v[n][3] = 0;
                        ++n;
                    }
                }
    for (int dl = -1; dl <= 1; dl += 2)
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    t.v[n][0] = dx, t.v[n][1] = dy, t.v[n][2] = dz, t.v[n][3] = dl;
                    ++n;
                }
    return t;
}

constexpr NbrTable kNbrHost = make_nbr_table();
static_assert(kNbrHost.v[5][3] == 0 && kNbrHost.v[6][0] * kNbrHost.v[6][0] + kNbrHost.v[6][1] * kNbrHost.v[6][1] +
                                              kNbrHost.v[6][2] * kNbrHost.v[6][2] == 2,
              "faces first, then edges");
static_assert(kNbrHost.v[25][3] == 0 && kNbrHost.v[26][3] == -1 && kNbrHost.v[79][3] == 1, "neighbour table layout");

// Tile of the detection-scale DoGs staged in shared memory with a one-voxel
// halo: [z: TZ+2][y: BY+2][x: BX+2] floats per level.  Lanes of a warp hold
// consecutive x, so every shared read of a warp is conflict-free.
constexpr int PK_TZ = 8;
constexpr int PK_SX = PK_BX + 2, PK_SY = PK_BY + 2, PK_SZ = PK_TZ + 2;
constexpr int PK_LEVEL = PK_SX * PK_SY * PK_SZ;

__host__ __device__ constexpr int peak_smem_bytes(int n_scales) { return n_scales * PK_LEVEL * 4; }
constexpr int PK_SURV = 1024;    // pass-2 list of one CTA (overflow is tested in pass 1)

struct PeakCtx {
    const float* sm;        // staged D_1..D_S
    int si;                 // this voxel's index inside one staged level
    int64_t off, py, pz;    // global offset and pitches (outer levels D_0, D_{S+1})
    int n_scales;
};

// D_l at offset (dx,dy,dz) from the voxel: shared memory for 1 <= l <= S,
// global memory (outer levels D_0, D_{S+1}) otherwise.
template <typename S>
__device__ __forceinline__ float nbr_value(const PeakArgs& a, const PeakCtx& q, int l, int dx, int dy, int dz) {
    if (l >= 1 && l <= q.n_scales) return q.sm[(l - 1) * PK_LEVEL + q.si + (dz * PK_SY + dy) * PK_SX + dx];
    return to_f32(static_cast<const S*>(a.dog[l])[q.off + dz * q.pz + dy * q.py + dx]);
}

// Neighbours K0..K1-1 of scale s: all reads before any comparison.
template <typename S, int K0, int K1>
__device__ __forceinline__ void sign_batch(const PeakArgs& a, const PeakCtx& q, int s, float c, int& sum) {
    constexpr NbrTable T = make_nbr_table();
    float n[K1 - K0];
#pragma unroll
    for (int i = 0; i < K1 - K0; ++i) {
        const int* nb = T.v[K0 + i];
        n[i] = nbr_value<S>(a, q, s + nb[3], nb[0], nb[1], nb[2]);
    }
#pragma unroll
    for (int i = 0; i < K1 - K0; ++i) sum += (c > n[i]) - (c < n[i]);
}

template <int K1>
__device__ __forceinline__ bool out_of_reach(int sum, int cut) {
    return (sum < 0 ? -sum : sum) + (80 - K1) < cut;
}

// Sum-of-signs and curvature tests of the voxel at scale s (contrast already
// passed); stores the sum of signs in *ssum.
template <typename S>
__device__ __forceinline__ bool full_test(const PeakArgs& a, const PeakCtx& q, int s, float c, int* ssum) {
    // Five batches (faces, edges, corners of D_s, then D_{s-1}, D_{s+1}); after
    // k comparisons |S| can still change by at most 80 - k, so stop once the
    // cut is out of reach.
    int sum = 0;
    const int cut = a.sign_sum_min;
    sign_batch<S, 0, 6>(a, q, s, c, sum);
    if (out_of_reach<6>(sum, cut)) return false;
    sign_batch<S, 6, 18>(a, q, s, c, sum);
    if (out_of_reach<18>(sum, cut)) return false;
    sign_batch<S, 18, 26>(a, q, s, c, sum);
    if (out_of_reach<26>(sum, cut)) return false;
    sign_batch<S, 26, 53>(a, q, s, c, sum);
    if (out_of_reach<53>(sum, cut)) return false;
    sign_batch<S, 53, 80>(a, q, s, c, sum);
    if (out_of_reach<80>(sum, cut)) return false;
    // curvature: H' = -sign(S) * Hessian of D_s by central differences
    const float* d = q.sm + (s - 1) * PK_LEVEL + q.si;
    auto v = [&](int dz, int dy, int dx) { return d[(dz * PK_SY + dy) * PK_SX + dx]; };
    const float hxx = v(0, 0, 1) + v(0, 0, -1) - 2.0f * c;
    const float hyy = v(0, 1, 0) + v(0, -1, 0) - 2.0f * c;
    const float hzz = v(1, 0, 0) + v(-1, 0, 0) - 2.0f * c;
    const float hxy = (v(0, 1, 1) - v(0, -1, 1) - v(0, 1, -1) + v(0, -1, -1)) * 0.25f;
    const float hxz = (v(1, 0, 1) - v(-1, 0, 1) - v(1, 0, -1) + v(-1, 0, -1)) * 0.25f;
    const float hyz = (v(1, 1, 0) - v(-1, 1, 0) - v(1, -1, 0) + v(-1, -1, 0)) * 0.25f;
    const float sg = sum > 0 ? -1.0f : 1.0f;
    const float A = sg * hxx, B = sg * hyy, C = sg * hzz;
    const float XY = sg * hxy, XZ = sg * hxz, YZ = sg * hyz;
    const float m2 = A * B - XY * XY;
    const float det = A * (B * C - YZ * YZ) - XY * (XY * C - YZ * XZ) + XZ * (XY * YZ - B * XZ);
    const float tr = A + B + C;
    const float g = a.curv_k1 * det - a.curv_k2 * (tr * tr * tr);
    *ssum = sum;
    return A > 0.f && m2 > 0.f && det > 0.f && g > 0.f;
}

__device__ __forceinline__ void write_keypoint(const PeakArgs& a, int slot, int x, int y, int z, int s, int ssum,
                                               float c, float scale) {
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
    k.polarity = ssum > 0 ? 1 : -1;
    k.reserved0[0] = k.reserved0[1] = k.reserved0[2] = 0;
    k.dog = c;
    k.sign_sum = ssum;
    k.reserved1 = 0;
    a.out[slot] = k;
}

// One 32x8x8 tile (tile coordinates bx, by, bz) by a CTA of 32x8 threads.
// pk_sm holds peak_smem_bytes(S); surv / n_surv are the pass-2 list.
template <typename S>
__device__ __forceinline__ void peak_tile(const PeakArgs& a, int bx, int by, int bz, float* pk_sm, unsigned* surv,
                                          int& n_surv) {
    const int b = a.border;
    const int x0 = bx * PK_BX + b, y0 = by * PK_BY + b, z0 = bz * PK_TZ + b;
    const int lane = threadIdx.x & 31, warp = (threadIdx.x + PK_BX * threadIdx.y) >> 5;
    const int tid = lane + 32 * warp;
    const int nS = a.n_scales;
    if (tid == 0) n_surv = 0;
    // Stage D_1..D_S around the tile (indices clamped; values outside the
    // volume are never compared).  float32 levels are copied with cp.async, so
    // every element of every level is in flight at once without registers;
    // 16-bit levels go through registers (converted), four rows per round.
    if constexpr (sizeof(S) == 4) {
        for (int l = 1; l <= nS; ++l) {
            const float* src = static_cast<const float*>(a.dog[l]);
            const unsigned dst0 = (unsigned)__cvta_generic_to_shared(pk_sm + (l - 1) * PK_LEVEL);
            for (int i = tid; i < PK_LEVEL; i += PK_THREADS) {
                const int xx = i % PK_SX, r = i / PK_SX, yy = r % PK_SY, zz = r / PK_SY;
                const int gx = min(max(x0 - 1 + xx, 0), a.nx - 1);
                const int gy = min(max(y0 - 1 + yy, 0), a.ny - 1);
                const int gz = min(max(z0 - 1 + zz, 0), a.nz - 1);
                const float* g = src + (int64_t)gz * a.pz + (int64_t)gy * a.py + gx;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst0 + 4u * (unsigned)i), "l"(g)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    } else {
        for (int l = 1; l <= nS; ++l) {
            const S* src = static_cast<const S*>(a.dog[l]);
            float* dstl = pk_sm + (l - 1) * PK_LEVEL;
            const int gx0 = min(max(x0 - 1 + lane, 0), a.nx - 1);
            const int gx1 = min(max(x0 + 31 + lane, 0), a.nx - 1);   // columns 32, 33 (lanes 0, 1)
            for (int row0 = warp; row0 < PK_SY * PK_SZ; row0 += 4 * (PK_THREADS / 32)) {
                float v0[4], v1[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int row = row0 + k * (PK_THREADS / 32);
                    if (row < PK_SY * PK_SZ) {
                        const int gy = min(max(y0 - 1 + row % PK_SY, 0), a.ny - 1);
                        const int gz = min(max(z0 - 1 + row / PK_SY, 0), a.nz - 1);
                        const S* r = src + (int64_t)gz * a.pz + (int64_t)gy * a.py;
                        v0[k] = to_f32(r[gx0]);
                        v1[k] = lane < PK_SX - 32 ? to_f32(r[gx1]) : 0.f;
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int row = row0 + k * (PK_THREADS / 32);
                    if (row < PK_SY * PK_SZ) {
                        dstl[row * PK_SX + lane] = v0[k];
                        if (lane < PK_SX - 32) dstl[row * PK_SX + 32 + lane] = v1[k];
                    }
                }
            }
        }
    }
    // the outer levels D_0 and D_{S+1} at this thread's column, all planes at once
    float outer_lo[PK_TZ], outer_hi[PK_TZ];
    {
        const int cx = min(x0 + lane, a.nx - 1), cy = min(y0 + warp, a.ny - 1);
        const S* lo = static_cast<const S*>(a.dog[0]);
        const S* hi = static_cast<const S*>(a.dog[nS + 1]);
#pragma unroll
        for (int tz = 0; tz < PK_TZ; ++tz) {
            const int64_t o = (int64_t)min(z0 + tz, a.nz - 1) * a.pz + (int64_t)cy * a.py + cx;
            outer_lo[tz] = to_f32(lo[o]);
            outer_hi[tz] = to_f32(hi[o]);
        }
    }
    if constexpr (sizeof(S) == 4) asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();

    const int x = x0 + lane, y = y0 + warp;
    const bool strict = a.sign_sum_min >= 80;
    const float scale = (float)(1 << a.octave);
    PeakCtx q;
    q.sm = pk_sm;
    q.py = a.py;
    q.pz = a.pz;
    q.n_scales = nS;
    // Pass 1, branch free: the contrast test and the eight nearest comparisons
    // (the same voxel in D_{s-1} and D_{s+1}, the six face neighbours in D_s).
    // With the strict cut all eight must go the same way; otherwise
    // |S_8| + 72 >= cut is necessary.  Survivors are listed for pass 2.
#pragma unroll
    for (int tz = 0; tz < PK_TZ; ++tz) {
        const bool inside = x < a.nx - b && y < a.ny - b && z0 + tz < a.nz - b;
        const int si = ((tz + 1) * PK_SY + warp + 1) * PK_SX + lane + 1;
        for (int s = 1; s <= nS; ++s) {
            const float* d = pk_sm + (s - 1) * PK_LEVEL + si;
            const float c = d[0];
            // in-tile index for every s, so no load can leave the staged levels
            const float lo_in = d[s > 1 ? -PK_LEVEL : 0], hi_in = d[s < nS ? PK_LEVEL : 0];
            const float lo = s == 1 ? outer_lo[tz] : lo_in;
            const float hi = s == nS ? outer_hi[tz] : hi_in;
            const float f0 = d[-1], f1 = d[1], f2 = d[-PK_SX], f3 = d[PK_SX];
            const float f4 = d[-PK_SX * PK_SY], f5 = d[PK_SX * PK_SY];
            bool cand;
            if (strict) {
                const float mx = fmaxf(fmaxf(fmaxf(lo, hi), fmaxf(f0, f1)), fmaxf(fmaxf(f2, f3), fmaxf(f4, f5)));
                const float mn = fminf(fminf(fminf(lo, hi), fminf(f0, f1)), fminf(fminf(f2, f3), fminf(f4, f5)));
                cand = c > mx || c < mn;
            } else {
                const int s8 = (c > lo) - (c < lo) + (c > hi) - (c < hi) + (c > f0) - (c < f0) + (c > f1) - (c < f1) +
                               (c > f2) - (c < f2) + (c > f3) - (c < f3) + (c > f4) - (c < f4) + (c > f5) - (c < f5);
                cand = (s8 < 0 ? -s8 : s8) + 72 >= a.sign_sum_min;
            }
            if (inside && cand && fabsf(c) >= a.contrast) {
                const int pos = atomicAdd(&n_surv, 1);
                if (pos < PK_SURV) {
                    surv[pos] = (unsigned)lane | ((unsigned)warp << 5) | ((unsigned)tz << 8) | ((unsigned)s << 12);
                } else {
                    // list full: test here (rare; same result, slower path)
                    q.si = si;
                    q.off = (int64_t)(z0 + tz) * a.pz + (int64_t)y * a.py + x;
                    int ssum = 0;
                    if (full_test<S>(a, q, s, c, &ssum)) {
                        const int slot = atomicAdd(a.count, 1);
                        if (slot < a.capacity) write_keypoint(a, slot, x, y, z0 + tz, s, ssum, c, scale);
                    }
                }
            }
        }
    }
    __syncthreads();
    // Pass 2: the full 80-neighbour and curvature tests on the listed voxel-
    // scales, spread over all lanes; keypoints are compacted with a warp ballot,
    // an intra-warp prefix (popc of the lower lanes) and one atomicAdd per warp.
    const int n = min(n_surv, PK_SURV);
    for (int base = warp * 32; base < n; base += PK_THREADS) {
        const int i = base + lane;
        bool kp = false;
        int ssum = 0, kx = 0, ky = 0, kz = 0, s = 1;
        float c = 0.f;
        if (i < n) {
            const unsigned e = surv[i];
            const int l = e & 31, w = (e >> 5) & 7, tz = (e >> 8) & 15;
            s = (e >> 12) & 7;
            kx = x0 + l, ky = y0 + w, kz = z0 + tz;
            q.si = ((tz + 1) * PK_SY + w + 1) * PK_SX + l + 1;
            q.off = (int64_t)kz * a.pz + (int64_t)ky * a.py + kx;
            c = pk_sm[(s - 1) * PK_LEVEL + q.si];
            kp = full_test<S>(a, q, s, c, &ssum);
        }
        const unsigned m = __ballot_sync(0xffffffffu, kp);
        if (m == 0u) continue;
        const int leader = __ffs(m) - 1;
        int slot0 = 0;
        if (lane == leader) slot0 = atomicAdd(a.count, __popc(m));
        slot0 = __shfl_sync(0xffffffffu, slot0, leader);
        if (!kp) continue;
        const int slot = slot0 + __popc(m & ((1u << lane) - 1u));
        if (slot < a.capacity) write_keypoint(a, slot, kx, ky, kz, s, ssum, c, scale);
    }
}

}  // namespace peak_detail
}  // namespace sift3d
