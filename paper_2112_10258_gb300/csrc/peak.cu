// 4D extremum detection for sm_103a (Sec. 2.2.2 "4D Peak Detection").
//
// For every interior voxel v of an octave and every detection scale s = 1..S:
//   1. contrast  |D_s(v)| >= t_c;
//   2. sum of signs  S = sum over the 80 neighbours n (3x3x3 in D_{s-1} and
//      D_{s+1}, 3x3x3 minus v in D_s) of sign(D_s(v) - D(n)); keep |S| >= cut
//      (+-80 = strict peak / valley, the paper's default interval);
//   3. curvature  H' = -sign(S) * Hessian(D_s at v) positive definite (leading
//      minors) and tr(H')^3 r^2 < (2r+1)^3 det(H').
//
// One CTA of 32x8 threads owns a 32x8x8 voxel tile.  A single 4D TMA load
// (x, y, z, level) brings the tile plus a one-voxel halo of all S+2 DoG levels
// into shared memory; the DoG levels of an octave lie at a constant stride in
// the workspace, so the level is simply the fourth tensor dimension.  Halo
// voxels outside the volume are zero-filled by the TMA unit; they are never
// compared, because every detected voxel is at least `border` >= 1 voxels from
// each face.
//
// Pass 1 (branch free): each thread walks its (x, y) column through the 8
// planes with a register window over z and applies the exact necessary
// conditions of a strict extremum: the contrast test and the eight nearest
// comparisons (six faces in D_s, the same voxel in D_{s-1} and D_{s+1}).
// Survivors are listed in shared memory.  Pass 2 runs the full 80-neighbour sum
// (faces, edges and corners of D_s, then D_{s-1}, then D_{s+1}; it stops once
// the cut is out of reach) and the curvature test, spread over all lanes.
// Keypoints are compacted without an extrema map: a warp ballot, an intra-warp
// prefix (popc of the lower lanes) and one atomicAdd per warp.  A rank sort
// then writes the records to the caller in canonical order (octave, scale, iz,
// iy, ix), independent of scheduling.
#include <algorithm>

#include "common.cuh"
#include "tma.cuh"

namespace sift3d {

namespace {

constexpr int TX = 32, TY = 8, TZ = 8;
constexpr int THREADS = TX * TY;
constexpr int SY = TY + 2, SZ = TZ + 2;
constexpr int SURV = 512;                     // pass-2 list of one CTA
constexpr int kDrainPolls = 1 << 26;          // wait for a copy still landing after a failed wait

// Staged row width: the 34 voxels of a halo row rounded up so that the TMA box
// row is a multiple of 16 bytes.
template <typename S>
__host__ __device__ constexpr int box_w() { return sizeof(S) == 4 ? 36 : 40; }

template <typename S>
__host__ __device__ constexpr int level_elems() { return box_w<S>() * SY * SZ; }

template <typename S>
constexpr size_t peak_smem(int n_levels) { return (size_t)n_levels * level_elems<S>() * sizeof(S); }

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

constexpr NbrTable kNbr = make_nbr_table();
static_assert(kNbr.v[5][3] == 0 && kNbr.v[6][0] * kNbr.v[6][0] + kNbr.v[6][1] * kNbr.v[6][1] +
                                           kNbr.v[6][2] * kNbr.v[6][2] == 2,
              "faces first, then edges");
static_assert(kNbr.v[25][3] == 0 && kNbr.v[26][3] == -1 && kNbr.v[79][3] == 1, "neighbour table layout");

// Offsets of the 80 neighbours inside the staged levels (elements).
struct OffTable {
    int o[80];
};

template <typename S>
__host__ __device__ constexpr OffTable make_off_table() {
    const NbrTable t = make_nbr_table();
    OffTable r{};
    for (int k = 0; k < 80; ++k)
        r.o[k] = ((t.v[k][3] * SZ + t.v[k][2]) * SY + t.v[k][1]) * box_w<S>() + t.v[k][0];
    return r;
}

template <typename S>
__device__ __forceinline__ float ld(const S* p) { return to_f32(*p); }

// Neighbours K0..K1-1 around the staged centre p: all reads before any comparison.
template <typename S, int K0, int K1>
__device__ __forceinline__ void sign_batch(const S* p, float c, int& sum) {
    constexpr OffTable T = make_off_table<S>();
    float n[K1 - K0];
#pragma unroll
    for (int i = 0; i < K1 - K0; ++i) n[i] = ld(p + T.o[K0 + i]);
#pragma unroll
    for (int i = 0; i < K1 - K0; ++i) sum += (c > n[i]) - (c < n[i]);
}

template <int K1>
__device__ __forceinline__ bool out_of_reach(int sum, int cut) {
    return (sum < 0 ? -sum : sum) + (80 - K1) < cut;
}

// Sum-of-signs and curvature tests of the staged centre p (contrast already
// passed); stores the sum of signs in *ssum.
template <typename S>
__device__ __forceinline__ bool full_test(const S* p, float c, int cut, float k1, float k2, int* ssum) {
    // After k comparisons |S| can still change by at most 80 - k: stop once the
    // cut is out of reach.
    int sum = 0;
    sign_batch<S, 0, 6>(p, c, sum);
    if (out_of_reach<6>(sum, cut)) return false;
    sign_batch<S, 6, 18>(p, c, sum);
    if (out_of_reach<18>(sum, cut)) return false;
    sign_batch<S, 18, 26>(p, c, sum);
    if (out_of_reach<26>(sum, cut)) return false;
    sign_batch<S, 26, 53>(p, c, sum);
    if (out_of_reach<53>(sum, cut)) return false;
    sign_batch<S, 53, 80>(p, c, sum);
    if (out_of_reach<80>(sum, cut)) return false;
    // curvature: H' = -sign(S) * Hessian of D_s by central differences
    constexpr int BX = box_w<S>();
    auto v = [&](int dz, int dy, int dx) { return ld(p + (dz * SY + dy) * BX + dx); };
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
    const float g = k1 * det - k2 * (tr * tr * tr);
    *ssum = sum;
    return A > 0.f && m2 > 0.f && det > 0.f && g > 0.f;
}

// Sub-voxel refinement (no counterpart in the paper): one Newton step on the 4D
// quadratic through the staged 3^4 neighbourhood of centre p.  Gradient and
// Hessian by central differences with unit steps in x, y, z and the level
// index; the 4x4 system H off = -g is solved by Gaussian elimination with
// partial pivoting in float32.  Returns 1 (off[4], *val = c + g.off / 2) or 2
// when a pivot vanishes against the Hessian's largest entry (off = 0, *val = c).
template <typename S>
__device__ __noinline__ int refine_point(const S* p, float c, float* off, float* val) {
    constexpr int BX = box_w<S>();
    const int step[4] = {1, BX, SY * BX, SZ * SY * BX};   // x, y, z, level
    float M[4][5];
    float hmax = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const float vp = ld(p + step[a]), vm = ld(p - step[a]);
        M[a][4] = -0.5f * (vp - vm);                       // -g
        M[a][a] = vp + vm - 2.0f * c;
        hmax = fmaxf(hmax, fabsf(M[a][a]));
#pragma unroll
        for (int b = a + 1; b < 4; ++b) {
            const float h = 0.25f * (ld(p + step[a] + step[b]) - ld(p + step[a] - step[b]) -
                                     ld(p - step[a] + step[b]) + ld(p - step[a] - step[b]));
            M[a][b] = M[b][a] = h;
            hmax = fmaxf(hmax, fabsf(h));
        }
    }
    float g[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) g[a] = -M[a][4];
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabsf(M[r][col]) > fabsf(M[piv][col])) piv = r;
        if (!(fabsf(M[piv][col]) > 1e-6f * hmax)) {
            off[0] = off[1] = off[2] = off[3] = 0.f;
            *val = c;
            return 2;
        }
        if (piv != col)
            for (int k = 0; k < 5; ++k) {
                const float t = M[col][k];
                M[col][k] = M[piv][k];
                M[piv][k] = t;
            }
        for (int r = col + 1; r < 4; ++r) {
            const float f = M[r][col] / M[col][col];
            for (int k = col; k < 5; ++k) M[r][k] -= f * M[col][k];
        }
    }
    for (int r = 3; r >= 0; --r) {
        float acc = M[r][4];
        for (int k = r + 1; k < 4; ++k) acc -= M[r][k] * off[k];
        off[r] = acc / M[r][r];
    }
    *val = c + 0.5f * (g[0] * off[0] + g[1] * off[1] + g[2] * off[2] + g[3] * off[3]);
    return 1;
}

// Writes keypoint record `slot`; p is the staged centre (for the refinement).
template <typename S>
__device__ __forceinline__ void write_keypoint(const PeakArgs& a, int slot, int x, int y, int z, int s, int ssum,
                                               float c, float scale, const S* p) {
    sift3d_keypoint k;
    float off[4] = {0.f, 0.f, 0.f, 0.f};
    float val = c;
    int refined = 0;
    if (a.refine) refined = refine_point<S>(p, c, off, &val);
    k.x = ((float)x + off[0] + 0.5f) * scale - 0.5f;
    k.y = ((float)y + off[1] + 0.5f) * scale - 0.5f;
    k.z = ((float)z + off[2] + 0.5f) * scale - 0.5f;
    const int so = s + a.scale_base;   // the octave's scale index
    k.sigma = a.sigma_level[so] * (refined == 1 ? exp2f(off[3] / (float)a.n_scales) : 1.0f) * scale;
    k.ix = x;
    k.iy = y;
    k.iz = z;
    k.octave = (int16_t)a.octave;
    k.scale = (int16_t)so;
    k.polarity = ssum > 0 ? 1 : -1;
    k.refined = (int8_t)refined;
    k.reserved0[0] = k.reserved0[1] = 0;
    k.dog = val;
    k.sign_sum = ssum;
    k.reserved1 = 0;
    a.out[slot] = k;
}

// Full test of a voxel-scale that found the pass-2 list full (rare): kept out
// of line so that the unrolled pass-1 loop holds one call, not 24 copies.
template <typename S>
__device__ __noinline__ void test_overflow(const PeakArgs& a, const S* p, float c, int x, int y, int z, int s,
                                           float scale) {
    int ssum = 0;
    if (full_test<S>(p, c, a.sign_sum_min, a.curv_k1, a.curv_k2, &ssum)) {
        const int slot = atomicAdd(a.count, 1);
        if (slot < a.capacity) write_keypoint<S>(a, slot, x, y, z, s, ssum, c, scale, p);
    }
}

// One 32x8x8 tile (tile coordinates bx, by, bz) of the octave A describes,
// staged through the CTA's barrier `bar` in the given phase parity.  Returns
// false when the copy's wait ran out (the CTA must leave).
template <typename S, int NS>
__device__ __forceinline__ bool peak_tile(const PeakTmaArgs& A, int bx, int by, int bz, unsigned parity, S* sm,
                                          uint64_t* bar_p, unsigned* surv, int* n_surv_p) {
    constexpr int NL = NS + 2;
    constexpr int BX = box_w<S>();
    constexpr int PL = SY * BX;            // one staged z plane
    constexpr int LV = level_elems<S>();   // one staged level
    uint64_t& bar = *bar_p;
    int& n_surv = *n_surv_p;
    const PeakArgs& a = A.a;
    const int lane = threadIdx.x, w = threadIdx.y;
    const int tid = lane + TX * w;
    const int xs = A.x_start + bx * TX;                   // halo origin of this tile
    const int ys = a.border - 1 + by * TY;
    const int zs = a.border - 1 + bz * TZ;

    if (tid == 0) {
        n_surv = 0;
        tma::mbar_expect_tx(&bar, (unsigned)(NL * LV * sizeof(S)));
        tma::load_4d(sm, &A.dogs, xs, ys, zs, 0, &bar);
    }
    // Bounded wait, CTA-uniform.  With the test flag it is a single non-blocking
    // test, which finds the copy still in flight.  On a timeout the detect's
    // error flag is set and thread 0 waits for the copy to land (a far longer
    // bound) before the whole CTA leaves, so no copy reaches shared memory after
    // the CTA's exit.
    const bool first_test = A.test_flag != nullptr && *A.test_flag != 0;
    const bool landed =
        first_test ? tma::mbar_test(&bar, parity) : tma::mbar_wait_bounded(&bar, parity, tma::kWaitPolls);
    if (!__syncthreads_and(landed)) {
        if (tid == 0) {
            atomicExch(A.err, 1);
            tma::mbar_wait_bounded(&bar, parity, kDrainPolls);
        }
        return false;
    }

    const int b = a.border;
    const int x = xs + 1 + lane, y = ys + 1 + w;
    const bool col_inside = x >= b && x < a.nx - b && y < a.ny - b;
    const bool strict = a.sign_sum_min >= 80;
    const float scale = (float)(1 << a.octave);
    const S* col = sm + (w + 1) * BX + lane + 1;           // level 0, staged plane 0

    // Pass 1 with a register window over z: D_l at planes z-1, z, z+1.
    float prv[NL], cur[NL], nxt[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        prv[l] = ld(col + l * LV);
        cur[l] = ld(col + l * LV + PL);
    }
#pragma unroll
    for (int tz = 0; tz < TZ; ++tz) {
        const int zz = tz + 1;
        const bool inside = col_inside && zs + zz < a.nz - b;
#pragma unroll
        for (int l = 0; l < NL; ++l) nxt[l] = ld(col + l * LV + (zz + 1) * PL);
#pragma unroll
        for (int s = 1; s <= NS; ++s) {
            const S* p = col + s * LV + zz * PL;
            const float c = cur[s];
            const float f0 = ld(p - 1), f1 = ld(p + 1), f2 = ld(p - BX), f3 = ld(p + BX);
            const float lo = cur[s - 1], hi = cur[s + 1], f4 = prv[s], f5 = nxt[s];
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
                if (pos < SURV) {
                    surv[pos] = (unsigned)lane | ((unsigned)w << 5) | ((unsigned)tz << 8) | ((unsigned)s << 12);
                } else {
                    test_overflow<S>(a, p, c, x, y, zs + zz, s, scale);   // list full: same result, slower
                }
            }
        }
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            prv[l] = cur[l];
            cur[l] = nxt[l];
        }
    }
    __syncthreads();

    // Pass 2: the full 80-neighbour and curvature tests of the listed
    // voxel-scales, 32 per warp at a time.
    const int n = min(n_surv, SURV);
    for (int base = w * 32; base < n; base += THREADS) {
        const int i = base + lane;
        bool kp = false;
        int ssum = 0, kx = 0, ky = 0, kz = 0, s = 1;
        float c = 0.f;
        const S* pc = sm;
        if (i < n) {
            const unsigned e = surv[i];
            const int l = e & 31, ww = (e >> 5) & 7, tz = (e >> 8) & 7;
            s = (e >> 12) & 7;
            kx = xs + 1 + l, ky = ys + 1 + ww, kz = zs + 1 + tz;
            pc = sm + s * LV + (tz + 1) * PL + (ww + 1) * BX + l + 1;
            c = ld(pc);
            kp = full_test<S>(pc, c, a.sign_sum_min, a.curv_k1, a.curv_k2, &ssum);
        }
        const unsigned m = __ballot_sync(0xffffffffu, kp);
        if (m == 0u) continue;
        const int leader = __ffs(m) - 1;
        int slot0 = 0;
        if (lane == leader) slot0 = atomicAdd(a.count, __popc(m));
        slot0 = __shfl_sync(0xffffffffu, slot0, leader);
        if (!kp) continue;
        const int slot = slot0 + __popc(m & ((1u << lane) - 1u));
        if (slot < a.capacity) write_keypoint<S>(a, slot, kx, ky, kz, s, ssum, c, scale, pc);
    }
    return true;
}

template <typename S, int NS>
__global__ void __launch_bounds__(THREADS, 3) peak_kernel(const __grid_constant__ PeakTmaArgs A) {
    extern __shared__ __align__(128) unsigned char pk_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned surv[SURV];
    __shared__ int n_surv;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        tma::mbar_init(&bar, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    peak_tile<S, NS>(A, blockIdx.x, blockIdx.y, blockIdx.z, 0u, reinterpret_cast<S*>(pk_raw), &bar, surv, &n_surv);
}

// Batched: the CTAs walk the tiles of every volume's octave in one flat list;
// each volume's arguments (and tensor map) come from the table in global
// memory, and the CTA's barrier changes phase with every tile it stages.
template <typename S, int NS>
__global__ void __launch_bounds__(THREADS, 3) peak_batch(const BatchTable t) {
    extern __shared__ __align__(128) unsigned char pk_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned surv[SURV];
    __shared__ int n_surv;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        tma::mbar_init(&bar, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const PeakTmaArgs* vols = static_cast<const PeakTmaArgs*>(t.args);
    unsigned k = 0;
    for (int item = blockIdx.x; item < t.total; item += gridDim.x, ++k) {
        const int v = batch_volume(t, item);
        const PeakTmaArgs& A = vols[v];
        const int local = item - t.prefix[v];
        if (!peak_tile<S, NS>(A, local % A.gx, (local / A.gx) % A.gy, local / (A.gx * A.gy), k & 1u,
                              reinterpret_cast<S*>(pk_raw), &bar, surv, &n_surv))
            return;
        __syncthreads();   // the next tile reuses the staged levels and the list
    }
}

// ---- canonical order ------------------------------------------------------
// Rank sort: the key of record i packs (octave, scale, iz, iy, ix, i), so keys
// are unique and record i's place is the number of smaller keys.  Each CTA
// ranks 32 records against all keys, read through shared memory in tiles that
// all 512 threads stage at once; the 16 consecutive lanes of a record each
// count every 16th key and add their counts.  Small CTAs spread a few thousand
// records over many SMs: the sort closes the detect's critical path.
constexpr int SORT_RECORDS = 32;
constexpr int SORT_LANES = 16;
constexpr int SORT_THREADS = SORT_RECORDS * SORT_LANES;
constexpr int SORT_TILE = kSortSmemKeys;

__device__ __forceinline__ unsigned long long sort_key(const sift3d_keypoint& k, int idx) {
    return ((unsigned long long)(k.octave & 0xF) << 60) | ((unsigned long long)(k.scale & 0xF) << 56) |
           ((unsigned long long)(k.iz & 0xFFF) << 44) | ((unsigned long long)(k.iy & 0xFFF) << 32) |
           ((unsigned long long)(k.ix & 0xFFF) << 20) | (unsigned long long)idx;
}

__global__ void __launch_bounds__(SORT_THREADS) sort_kernel(const SortArgs a) {
    __shared__ unsigned long long skeys[SORT_TILE];
    const int total = *a.count;
    const int n = min(total, a.capacity);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int reported = (a.err != nullptr && *a.err != 0) ? -2 : total;
        *a.count_out = reported;
        if (a.count_copy != nullptr) *a.count_copy = reported;
    }
    if ((int)blockIdx.x * SORT_RECORDS >= n) return;
    const int sub = threadIdx.x % SORT_LANES;
    const int i = blockIdx.x * SORT_RECORDS + threadIdx.x / SORT_LANES;
    const unsigned long long mine = i < n ? sort_key(a.staging[i], i) : ~0ull;
    int rank = 0;
    for (int base = 0; base < n; base += SORT_TILE) {
        const int len = min(SORT_TILE, n - base);
        __syncthreads();
        for (int j = threadIdx.x; j < len; j += SORT_THREADS) skeys[j] = sort_key(a.staging[base + j], base + j);
        __syncthreads();
#pragma unroll 4
        for (int j = sub; j < len; j += SORT_LANES) rank += skeys[j] < mine;
    }
#pragma unroll
    for (int off = 1; off < SORT_LANES; off <<= 1) rank += __shfl_xor_sync(0xffffffffu, rank, off);
    if (i < n && sub == 0) a.out[rank] = a.staging[i];
}

template <typename S>
const void* peak_func(int ns) {
    switch (ns) {
        case 1: return reinterpret_cast<const void*>(&peak_kernel<S, 1>);
        case 2: return reinterpret_cast<const void*>(&peak_kernel<S, 2>);
        case 3: return reinterpret_cast<const void*>(&peak_kernel<S, 3>);
        case 4: return reinterpret_cast<const void*>(&peak_kernel<S, 4>);
        case 5: return reinterpret_cast<const void*>(&peak_kernel<S, 5>);
        default: return nullptr;
    }
}

template <typename S>
void peak_geometry(const PeakArgs& a, int* x_start, int* box_x, int* gx, size_t* smem) {
    // The first halo origin is border-1 rounded down to 8 voxels, so that every
    // tile's TMA x coordinate is 16-byte aligned for 4- and 2-byte elements.
    *x_start = ((a.border - 1) / 8) * 8;
    *box_x = box_w<S>();
    const int covered = a.nx - a.border - (*x_start + 1);    // x = x_start+1 .. nx-border-1
    *gx = std::max(1, (covered + TX - 1) / TX);
    *smem = peak_smem<S>(a.ns + 2);
}

}  // namespace

void peak_layout(int /*storage*/, const PeakArgs& a, int* x_start, int* box_x, int* box_y, int* box_z, int* box_l) {
    int gx;
    size_t smem;
    peak_geometry<float>(a, x_start, box_x, &gx, &smem);   // DoG levels are float32
    *box_y = SY;
    *box_z = SZ;
    *box_l = a.ns + 2;   // the launch's DoG levels in one copy
}

LaunchSpec peak_spec(int /*storage: DoG levels are float32 for every storage type*/, const PeakTmaArgs& A) {
    LaunchSpec s;
    const PeakArgs& a = A.a;
    int x_start = 0, box_x = 0, gx = 1;
    size_t smem = 0;
    s.func = peak_func<float>(a.ns);
    peak_geometry<float>(a, &x_start, &box_x, &gx, &smem);
    if (s.func == nullptr || x_start != A.x_start) {
        s.func = nullptr;
        return s;
    }
    const int iy = a.ny - 2 * a.border, iz = a.nz - 2 * a.border;
    s.grid = dim3(gx, (iy + TY - 1) / TY, (iz + TZ - 1) / TZ);
    s.block = dim3(TX, TY);
    s.smem = smem;
    if (s.smem > 48 * 1024) cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
    s.name = "peak";
    return s;
}

void peak_fill_tiles(PeakTmaArgs* A) {
    int x_start = 0, box_x = 0, gx = 1;
    size_t smem = 0;
    peak_geometry<float>(A->a, &x_start, &box_x, &gx, &smem);
    A->gx = gx;
    A->gy = (A->a.ny - 2 * A->a.border + TY - 1) / TY;
    A->gz = (A->a.nz - 2 * A->a.border + TZ - 1) / TZ;
}

LaunchSpec peak_batch_spec(int ns, int total) {
    LaunchSpec s;
    switch (ns) {
        case 1: s.func = reinterpret_cast<const void*>(&peak_batch<float, 1>); break;
        case 2: s.func = reinterpret_cast<const void*>(&peak_batch<float, 2>); break;
        case 3: s.func = reinterpret_cast<const void*>(&peak_batch<float, 3>); break;
        case 4: s.func = reinterpret_cast<const void*>(&peak_batch<float, 4>); break;
        case 5: s.func = reinterpret_cast<const void*>(&peak_batch<float, 5>); break;
        default: return s;
    }
    s.block = dim3(TX, TY);
    s.smem = peak_smem<float>(ns + 2);
    if (s.smem > 48 * 1024) cudaFuncSetAttribute(s.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s.func, THREADS, s.smem) != cudaSuccess || per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    s.grid = dim3((unsigned)std::max(1, std::min(total, per_sm * device_sm_count())));
    s.name = "peak_batch";
    return s;
}

LaunchSpec sort_spec(const SortArgs& a) {
    LaunchSpec s;
    s.func = reinterpret_cast<const void*>(&sort_kernel);
    s.grid = dim3((unsigned)std::max(1, (a.capacity + SORT_RECORDS - 1) / SORT_RECORDS));
    s.block = dim3(SORT_THREADS);
    s.smem = 0;
    s.name = "sort";
    return s;
}

}  // namespace sift3d
