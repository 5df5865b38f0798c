// Small-octave kernel for sm_103a: the whole pyramid of every small octave in
// one launch of one thread-block cluster.
//
// Octave o+1 starts from the sub-sampled level S of octave o (Sec. 2.2.2), so
// the octaves form a chain of dependent passes.  Run as separate launches, each
// pass of a small octave (octave 2 of a 145x174x145 volume has 56K voxels)
// costs mostly launch latency, and the chain through octaves 1..3 outlasts the
// bandwidth-bound work of octave 0.  Here the CLUSTER CTAs of one cluster own
// contiguous z-slabs of the octave; every level of the slab stays in shared
// memory:
//   y pass   own planes of G_{s-1} (shared)       -> U  (shared)
//   x pass   U                                    -> T  (shared, two buffers)
//   cluster barrier
//   z pass   T of this and the neighbouring CTAs  -> G_s (shared + global),
//            read through distributed shared memory     D_{s-1} (global)
// and the descriptor pre-blur B_s of G_s (Sec. 2.2.3) the same way.  T
// alternates between two buffers, so one cluster barrier per pass suffices: a
// CTA can only overwrite a T buffer after every CTA has passed the barrier that
// follows the last read of it.  Every level, DoG and pre-blurred level is also
// written to its place in the workspace, where the peak kernels, describe and
// sift3d_read_level find it.
//
// Every output is the same float32 chain as in the separate kernels (taps in
// ascending k from 0, the 2x2x2 mean summed in the same order, levels rounded
// to the storage type before they are filtered again), so the results are
// bitwise those of the separate launches.  Cluster barriers are hardware
// barriers: no spin loop here can run out.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace sift3d {

namespace {

namespace cg = cooperative_groups;

constexpr int CT = 512;               // threads per CTA
constexpr int STRIP = 8;              // outputs per thread along the y and x passes
constexpr int MAXP = kTailMaxSlab;    // planes per CTA slab

// Taps of the pass being run, copied to shared memory so that strip functions
// can hold them in registers by compile-time index.
struct PassTaps {
    float w[kMaxRadius + 1];
};

template <int R>
__device__ __forceinline__ void load_taps(const PassTaps& t, float (&w)[R + 1]) {
#pragma unroll
    for (int k = 0; k <= R; ++k) w[k] = t.w[k];
}

// y pass of one column strip: rows r0 .. r0+7 of column x of one plane.
template <int R>
__device__ __forceinline__ void y_strip(const float* src, float* dst, int py, int ny, int x, int r0,
                                        const PassTaps& t) {
    float w[R + 1];
    load_taps<R>(t, w);
    float v[STRIP + 2 * R];
#pragma unroll
    for (int i = 0; i < STRIP + 2 * R; ++i) v[i] = src[min(max(r0 - R + i, 0), ny - 1) * py + x];
#pragma unroll
    for (int j = 0; j < STRIP; ++j) {
        if (r0 + j >= ny) break;
        float acc = 0.f;
#pragma unroll
        for (int k = -R; k <= R; ++k) acc = fmaf(w[k < 0 ? -k : k], v[j + R + k], acc);
        dst[(r0 + j) * py + x] = acc;
    }
}

// x pass of one row strip: columns c0 .. c0+7 of one row.
template <int R>
__device__ __forceinline__ void x_strip(const float* src, float* dst, int nx, int c0, const PassTaps& t) {
    float w[R + 1];
    load_taps<R>(t, w);
    float v[STRIP + 2 * R];
#pragma unroll
    for (int i = 0; i < STRIP + 2 * R; ++i) v[i] = src[min(max(c0 - R + i, 0), nx - 1)];
#pragma unroll
    for (int j = 0; j < STRIP; ++j) {
        if (c0 + j >= nx) break;
        float acc = 0.f;
#pragma unroll
        for (int k = -R; k <= R; ++k) acc = fmaf(w[k < 0 ? -k : k], v[j + R + k], acc);
        dst[c0 + j] = acc;
    }
}

// Geometry of the current octave as seen by one CTA.  The shared slabs use an
// odd row pitch (nx | 1), so the lanes of a warp reading one column each (the x
// pass walks rows) fall in distinct banks.
struct Slab {
    int nx, ny, nz;
    int py, P;            // row pitch and plane size of the shared slabs
    int z0, n;            // first plane and number of planes owned by this CTA
    int rank, ncta;       // this CTA's rank and the cluster size
};

__device__ __forceinline__ int slab_begin(int k, int nz, int ncta) { return (k * nz) / ncta; }

// y then x pass of the CTA's own planes: src (shared, float) -> dst (shared).
// U is the scratch plane set between the passes.
template <int R>
__device__ void xy_pass(const Slab& g, const float* src, float* U, float* dst, const PassTaps& t) {
    const int ystrips = (g.ny + STRIP - 1) / STRIP;
    for (int i = threadIdx.x; i < g.n * g.nx * ystrips; i += CT) {
        const int x = i % g.nx;
        const int rest = i / g.nx;
        const int rs = rest % ystrips, lz = rest / ystrips;
        y_strip<R>(src + lz * g.P, U + lz * g.P, g.py, g.ny, x, rs * STRIP, t);
    }
    __syncthreads();
    const int xstrips = (g.nx + STRIP - 1) / STRIP;
    for (int i = threadIdx.x; i < g.n * g.ny * xstrips; i += CT) {
        const int y = i % g.ny;            // lanes on consecutive rows: odd pitch, no bank conflict
        const int rest = i / g.ny;
        const int xs = rest % xstrips, lz = rest / xstrips;
        x_strip<R>(U + lz * g.P + y * g.py, dst + lz * g.P + y * g.py, g.nx, xs * STRIP, t);
    }
}

// z pass of the CTA's own planes from the T buffers of the cluster (this CTA
// and its neighbours, through distributed shared memory).  For every output
// voxel calls out(lz, shared offset in the plane, global offset in the plane,
// value); gpy is the global row pitch.
template <int R, class Out>
__device__ void z_pass(const Slab& g, int64_t gpy, float* T, const PassTaps& t, const float** zplane, Out out) {
    cg::cluster_group cluster = cg::this_cluster();
    // Input plane q of this CTA's window is plane z = clamp(z0 - R + q) of the
    // octave, held by the CTA k that owns z (the largest k with
    // slab_begin(k) <= z, k = ceil((z+1) * ncta / nz) - 1).  The window's plane
    // addresses are resolved once per pass.
    if (threadIdx.x < g.n + 2 * R) {
        const int z = min(max(g.z0 - R + (int)threadIdx.x, 0), g.nz - 1);
        const int k = ((z + 1) * g.ncta + g.nz - 1) / g.nz - 1;
        zplane[threadIdx.x] = cluster.map_shared_rank(T, k) + (z - slab_begin(k, g.nz, g.ncta)) * g.P;
    }
    __syncthreads();
    float w[R + 1];
    load_taps<R>(t, w);
    const int cols = g.nx * g.ny;
    for (int i = threadIdx.x; i < cols; i += CT) {
        const int x = i % g.nx, y = i / g.nx;
        const int off = y * g.py + x;
        float v[MAXP + 2 * R];
#pragma unroll
        for (int q = 0; q < MAXP + 2 * R; ++q) v[q] = q < g.n + 2 * R ? zplane[q][off] : 0.f;
        const int64_t goff = (int64_t)y * gpy + x;
#pragma unroll
        for (int j = 0; j < MAXP; ++j) {
            if (j >= g.n) break;
            float acc = 0.f;
#pragma unroll
            for (int k = -R; k <= R; ++k) acc = fmaf(w[k < 0 ? -k : k], v[j + R + k], acc);
            out(j, off, goff, acc);
        }
    }
}

// Dispatch on the radius (only radii of the schedule are ever hot).
#define SIFT3D_RADIUS_SWITCH(R_RUNTIME, CALL)                          \
    switch (R_RUNTIME) {                                              \
        case 1: { constexpr int RR = 1; CALL; } break;                \
        case 2: { constexpr int RR = 2; CALL; } break;                \
        case 3: { constexpr int RR = 3; CALL; } break;                \
        case 4: { constexpr int RR = 4; CALL; } break;                \
        case 5: { constexpr int RR = 5; CALL; } break;                \
        case 6: { constexpr int RR = 6; CALL; } break;                \
        case 7: { constexpr int RR = 7; CALL; } break;                \
        case 8: { constexpr int RR = 8; CALL; } break;                \
        case 9: { constexpr int RR = 9; CALL; } break;                \
        case 10: { constexpr int RR = 10; CALL; } break;              \
        case 11: { constexpr int RR = 11; CALL; } break;              \
        case 12: { constexpr int RR = 12; CALL; } break;              \
        case 13: { constexpr int RR = 13; CALL; } break;              \
        case 14: { constexpr int RR = 14; CALL; } break;              \
        case 15: { constexpr int RR = 15; CALL; } break;              \
        default: { constexpr int RR = 16; CALL; } break;              \
    }

template <typename S>
__device__ __forceinline__ float ld_s(const S* p) { return to_f32(*p); }

// 2x2x2 mean of the previous octave's level S at (2x, 2y, 2z), summed in the
// same order as the separate sub-sampling pass.  The source may have been
// written by this cluster: read at L2 (ld.cg), never through a stale L1 line.
template <typename S>
__device__ __forceinline__ float sub_mean_cg(const S* p, int64_t py, int64_t pz) {
    auto g = [](const S* q) { return to_f32(__ldcg(q)); };
    float acc = 0.f;
    acc += g(p);
    acc += g(p + 1);
    acc += g(p + py);
    acc += g(p + py + 1);
    acc += g(p + pz);
    acc += g(p + pz + 1);
    acc += g(p + pz + py);
    acc += g(p + pz + py + 1);
    return acc * 0.125f;
}

template <typename S>
__global__ void __launch_bounds__(CT, 1) tail_kernel(const __grid_constant__ TailArgs a) {
    extern __shared__ __align__(16) float tl_sm[];
    __shared__ PassTaps taps;
    __shared__ const float* zplane[MAXP + 2 * kMaxRadius];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int ncta = (int)cluster.num_blocks();
    pdl_wait();   // level S of the octave before (no-op without a programmatic edge)

    for (int oi = 0; oi < a.n_oct; ++oi) {
        const TailOctave& o = a.oct[oi];
        Slab g;
        g.nx = o.nx;
        g.ny = o.ny;
        g.nz = o.nz;
        g.py = tail_row_pitch(o.nx);
        g.P = g.py * o.ny;
        g.rank = rank;
        g.ncta = ncta;
        g.z0 = slab_begin(rank, o.nz, ncta);
        g.n = slab_begin(rank + 1, o.nz, ncta) - g.z0;
        const int SL = a.slab_planes * g.P;         // floats per slab buffer
        float* Gprev = tl_sm;
        float* Gcur = tl_sm + SL;
        float* U = tl_sm + 2 * SL;
        float* Tb[2] = {tl_sm + 3 * SL, tl_sm + 4 * SL};
        int tb = 0;

        // ---- level 1 from the sub-sampled level S of the previous octave
        {
            const S* src = static_cast<const S*>(oi == 0 ? a.src : a.oct[oi - 1].G[a.S]);
            const int64_t spy = oi == 0 ? a.src_py : a.oct[oi - 1].py;
            const int64_t spz = oi == 0 ? a.src_pz : a.oct[oi - 1].pz;
            S* G0 = static_cast<S*>(o.G[0]);
            // Gprev <- G_0 rounded to the storage type (it is what D_0 uses and
            // what the separate path stores); Gcur <- the unrounded mean, which
            // the separate path filters.
            // Batches of NB voxels per thread: all 8 * NB loads are issued
            // before the first store, so a thread waits for L2 once per batch.
            constexpr int NB = 8;
            const int nvox = g.n * g.nx * g.ny;
            for (int base = 0; base < nvox; base += NB * CT) {
                float m[NB];
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int i = base + b * CT + threadIdx.x;
                    m[b] = 0.f;
                    if (i < nvox) {
                        const int x = i % g.nx;
                        const int rest = i / g.nx;
                        const int y = rest % g.ny, z = g.z0 + rest / g.ny;
                        m[b] = sub_mean_cg<S>(src + (int64_t)(2 * z) * spz + (int64_t)(2 * y) * spy + 2 * x, spy, spz);
                    }
                }
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int i = base + b * CT + threadIdx.x;
                    if (i < nvox) {
                        const int x = i % g.nx;
                        const int rest = i / g.nx;
                        const int y = rest % g.ny, lz = rest / g.ny;
                        const S ms = from_f32<S>(m[b]);
                        G0[(int64_t)(g.z0 + lz) * o.pz + (int64_t)y * o.py + x] = ms;
                        Gprev[lz * g.P + y * g.py + x] = to_f32(ms);
                        Gcur[lz * g.P + y * g.py + x] = m[b];
                    }
                }
            }
        }
        for (int s = 1; s < a.L; ++s) {
            if (threadIdx.x <= kMaxRadius) taps.w[threadIdx.x] = a.t_inc[s - 1].w[threadIdx.x];
            __syncthreads();
            float* T = Tb[tb];
            const int R = a.r_inc[s - 1];
            // level 1 filters the unrounded mean held in Gcur, later levels G_{s-1}
            const float* xsrc = s == 1 ? Gcur : Gprev;
            SIFT3D_RADIUS_SWITCH(R, (xy_pass<RR>(g, xsrc, U, T, taps)));
            cluster.sync();
            S* Gs = static_cast<S*>(o.G[s]);
            S* Ds = static_cast<S*>(o.D[s - 1]);
            const int64_t zoff = (int64_t)g.z0 * o.pz;
            SIFT3D_RADIUS_SWITCH(R, (z_pass<RR>(g, o.py, T, taps, zplane,
                                                [&](int j, int off, int64_t goff, float acc) {
                                                    const S gs = from_f32<S>(acc);
                                                    const int li = j * g.P + off;
                                                    Gs[zoff + (int64_t)j * o.pz + goff] = gs;
                                                    Ds[zoff + (int64_t)j * o.pz + goff] = from_f32<S>(Gprev[li] - acc);
                                                    Gcur[li] = to_f32(gs);
                                                })));
            __syncthreads();
            float* t = Gprev;   // G_s becomes the next level's source
            Gprev = Gcur;
            Gcur = t;
            tb ^= 1;
            // descriptor pre-blur of G_s, s = 1..S
            if (a.r_desc > 0 && s <= a.S) {
                if (threadIdx.x <= kMaxRadius) taps.w[threadIdx.x] = a.t_desc.w[threadIdx.x];
                __syncthreads();
                float* T2 = Tb[tb];
                SIFT3D_RADIUS_SWITCH(a.r_desc, (xy_pass<RR>(g, Gprev, U, T2, taps)));
                cluster.sync();
                S* Bs = static_cast<S*>(o.B[s - 1]);
                SIFT3D_RADIUS_SWITCH(a.r_desc, (z_pass<RR>(g, o.py, T2, taps, zplane,
                                                           [&](int j, int, int64_t goff, float acc) {
                                                               Bs[zoff + (int64_t)j * o.pz + goff] = from_f32<S>(acc);
                                                           })));
                __syncthreads();
                tb ^= 1;
            }
        }
        // the next octave sub-samples this octave's level S, written by every
        // CTA: all stores before this barrier are visible after it
        cluster.sync();
    }
}

}  // namespace

// Cluster size for the small-octave kernel: 16 CTAs where the device can
// schedule such a cluster with this shared memory, else the portable 8.
static int pick_cluster(const void* func, const TailArgs& a, size_t* smem_out) {
    int max_plane = 0, max_nz = 0;
    for (int i = 0; i < a.n_oct; ++i) {
        max_plane = std::max(max_plane, tail_row_pitch(a.oct[i].nx) * a.oct[i].ny);
        max_nz = std::max(max_nz, a.oct[i].nz);
    }
    for (int ncta : {kTailCluster, kTailClusterPortable}) {
        const int slab = (max_nz + ncta - 1) / ncta;
        if (slab > kTailMaxSlab) continue;
        const size_t smem = tail_smem_bytes(max_plane, slab);
        if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (ncta > 8 && cudaFuncSetAttribute(func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(ncta, 1, 1);
        cfg.blockDim = dim3(CT, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr{};
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = ncta;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, func, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (n >= 1) {
            *smem_out = smem;
            return ncta;
        }
    }
    return 0;
}

LaunchSpec tail_spec(int storage, const TailArgs& a) {
    LaunchSpec s;
    if (storage == SIFT3D_STORAGE_F32) s.func = reinterpret_cast<const void*>(&tail_kernel<float>);
    else if (storage == SIFT3D_STORAGE_F16) s.func = reinterpret_cast<const void*>(&tail_kernel<__half>);
    else s.func = reinterpret_cast<const void*>(&tail_kernel<__nv_bfloat16>);
    size_t smem = 0;
    const int ncta = pick_cluster(s.func, a, &smem);
    if (ncta == 0 || a.slab_planes != (a.max_nz + ncta - 1) / ncta) {
        s.func = nullptr;
        s.name = "tail (cluster)";
        return s;
    }
    s.grid = dim3(ncta, 1, 1);
    s.block = dim3(CT);
    s.smem = smem;
    s.cluster = ncta;
    s.name = "tail";
    return s;
}

int tail_cluster_size(int storage, const TailArgs& a) {
    const void* f = storage == SIFT3D_STORAGE_F32   ? reinterpret_cast<const void*>(&tail_kernel<float>)
                    : storage == SIFT3D_STORAGE_F16 ? reinterpret_cast<const void*>(&tail_kernel<__half>)
                                                    : reinterpret_cast<const void*>(&tail_kernel<__nv_bfloat16>);
    size_t smem = 0;
    return pick_cluster(f, a, &smem);
}

size_t tail_smem_bytes(int plane_elems, int slab_planes) {
    return (size_t)5 * slab_planes * plane_elems * sizeof(float);
}

}  // namespace sift3d
