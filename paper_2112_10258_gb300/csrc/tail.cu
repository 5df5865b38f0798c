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
// and, in the same phases, the descriptor pre-blur B_{s-1} of G_{s-1}
// (Sec. 2.2.3) when s-1 is a detection scale.  T alternates between two
// buffers, so one cluster barrier per level suffices: a CTA can only overwrite
// a T buffer after every CTA has passed the barrier that follows the last read
// of it.  Every level, DoG and pre-blurred level is also
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
constexpr int MAXP = kTailMaxSlab;    // planes per CTA slab

// Taps of the pass being run, in shared memory (w[k] = w_|k|).
struct PassTaps {
    float w[kMaxRadius + 1];
};

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

// The passes below loop over the taps at run time and read every tap from
// (distributed) shared memory: the octaves this kernel takes are small, so the
// loads cost little, and one compact body serves every radius (fully unrolled
// per-radius bodies measured slower here: each pass jumped into cold code).
// Every output is acc = fmaf(w_|k|, in[clamp(i + k)], acc) for k = -R..R from
// 0, the chain the separate kernels compute.

// y then x pass of the CTA's own planes: src (shared) -> U (shared) -> dst (shared).
__device__ void xy_pass(const Slab& g, const float* src, float* U, float* dst, const PassTaps& t, int R) {
    for (int i = threadIdx.x; i < g.n * g.nx * g.ny; i += CT) {
        const int x = i % g.nx;
        const int rest = i / g.nx;
        const int y = rest % g.ny, lz = rest / g.ny;
        const float* col = src + lz * g.P + x;
        float acc = 0.f;
        for (int k = -R; k <= R; ++k) acc = fmaf(t.w[k < 0 ? -k : k], col[min(max(y + k, 0), g.ny - 1) * g.py], acc);
        U[lz * g.P + y * g.py + x] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < g.n * g.nx * g.ny; i += CT) {
        const int x = i % g.nx;
        const int rest = i / g.nx;
        const int y = rest % g.ny, lz = rest / g.ny;
        const float* row = U + lz * g.P + y * g.py;
        float acc = 0.f;
        for (int k = -R; k <= R; ++k) acc = fmaf(t.w[k < 0 ? -k : k], row[min(max(x + k, 0), g.nx - 1)], acc);
        dst[lz * g.P + y * g.py + x] = acc;
    }
}

// z pass of the CTA's own planes from the T buffers of the cluster (this CTA
// and its neighbours, through distributed shared memory).  For every output
// voxel calls out(lz, shared offset in the plane, global offset in the plane,
// value); gpy is the global row pitch.
template <class Out>
__device__ void z_pass(const Slab& g, int64_t gpy, float* T, const PassTaps& t, const float** zplane, int R,
                       Out out) {
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
    for (int i = threadIdx.x; i < g.n * g.nx * g.ny; i += CT) {
        const int x = i % g.nx;
        const int rest = i / g.nx;
        const int y = rest % g.ny, j = rest / g.ny;
        const int off = y * g.py + x;
        float acc = 0.f;
        for (int k = -R; k <= R; ++k) acc = fmaf(t.w[k < 0 ? -k : k], zplane[j + R + k][off], acc);
        out(j, off, (int64_t)y * gpy + x, acc);
    }
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
    __shared__ PassTaps taps, taps2;
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
        float* U2 = tl_sm + 3 * SL;
        float* Tb[2] = {tl_sm + 4 * SL, tl_sm + 5 * SL};
        float* T2b[2] = {tl_sm + 6 * SL, tl_sm + 7 * SL};
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
            // Level s also pre-blurs G_{s-1} for the descriptors when s-1 is a
            // detection scale (as the separate level kernels do), so each
            // level is one y/x phase, one cluster barrier and one z phase.
            const bool blur = a.r_desc > 0 && s >= 2 && s - 1 <= a.S;
            if (threadIdx.x <= kMaxRadius) {
                taps.w[threadIdx.x] = a.t_inc[s - 1].w[threadIdx.x];
                taps2.w[threadIdx.x] = a.t_desc.w[threadIdx.x];
            }
            __syncthreads();
            float* T = Tb[tb];
            float* T2 = T2b[tb];
            const int R = a.r_inc[s - 1];
            // level 1 filters the unrounded mean held in Gcur, later levels G_{s-1}
            const float* xsrc = s == 1 ? Gcur : Gprev;
            xy_pass(g, xsrc, U, T, taps, R);
            if (blur) xy_pass(g, Gprev, U2, T2, taps2, a.r_desc);
            cluster.sync();
            S* Gs = static_cast<S*>(o.G[s]);
            S* Ds = static_cast<S*>(o.D[s - 1]);
            const int64_t zoff = (int64_t)g.z0 * o.pz;
            z_pass(g, o.py, T, taps, zplane, R, [&](int j, int off, int64_t goff, float acc) {
                const S gs = from_f32<S>(acc);
                const int li = j * g.P + off;
                Gs[zoff + (int64_t)j * o.pz + goff] = gs;
                Ds[zoff + (int64_t)j * o.pz + goff] = from_f32<S>(Gprev[li] - acc);
                Gcur[li] = to_f32(gs);
            });
            if (blur) {
                __syncthreads();   // the plane table is rebuilt for T2
                S* Bs = static_cast<S*>(o.B[s - 2]);
                z_pass(g, o.py, T2, taps2, zplane, a.r_desc, [&](int j, int, int64_t goff, float acc) {
                    Bs[zoff + (int64_t)j * o.pz + goff] = from_f32<S>(acc);
                });
            }
            __syncthreads();
            float* t = Gprev;   // G_s becomes the next level's source
            Gprev = Gcur;
            Gcur = t;
            tb ^= 1;
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
    return (size_t)8 * slab_planes * plane_elems * sizeof(float);   // G_{s-1}, G_s, 2 y scratch, 2 x 2 T
}

}  // namespace sift3d
