// Host runtime: parameter validation, the octave plan (Sec. 2.2.2 scale
// schedule), the method-3 point-pair pattern (Sec. 2.2.3), device workspaces,
// the detect DAG and its execution.
#include "runtime.hpp"

#include <cudaTypedefs.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace sift3d {

namespace {

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ceil(trunc * sigma), or kMaxRadius + 1 for any sigma or trunc that is not a
// positive finite number with trunc * sigma <= kMaxRadius (checked before the
// conversion to int, which is undefined for NaN or out-of-range values).
int radius_of(double sigma, double trunc) {
    const double r = trunc * sigma;
    if (!(sigma > 0.0) || !(trunc > 0.0) || !(r <= (double)kMaxRadius)) return kMaxRadius + 1;
    return (int)std::ceil(r);
}

}  // namespace

int gaussian_radius(double sigma, double trunc) { return radius_of(sigma, trunc); }

// Sampled Gaussian on |k| <= R, normalised to unit sum in double, then float.
Taps gaussian_taps(double sigma, int R) {
    Taps t{};
    double w[kMaxRadius + 1];
    double sum = 0.0;
    for (int k = 0; k <= R; ++k) {
        w[k] = std::exp(-(double)(k * k) / (2.0 * sigma * sigma));
        sum += k == 0 ? w[k] : 2.0 * w[k];
    }
    for (int k = 0; k <= R; ++k) t.w[k] = (float)(w[k] / sum);
    return t;
}

namespace {

Taps make_taps(double sigma, int R) { return gaussian_taps(sigma, R); }

int fail(std::string* err, const char* msg) {
    if (err) *err = msg;
    return SIFT3D_EINVAL;
}

}  // namespace

int validate_params(const sift3d_params& p, std::string* err) {
    if (!(p.sigma0 > 0.0) || !(p.sigma_in >= 0.0) || !(p.sigma0 > p.sigma_in) || !std::isfinite(p.sigma0))
        return fail(err, "need finite sigma0 > sigma_in >= 0");
    if (p.scales_per_octave < 1 || p.scales_per_octave > SIFT3D_MAX_SCALES)
        return fail(err, "scales_per_octave must be in 1..5");
    if (p.border < 1) return fail(err, "border must be >= 1");
    if (p.min_octave_dim < 3 || p.min_octave_dim < 2 * p.border + 1)
        return fail(err, "min_octave_dim must be >= max(3, 2*border+1)");
    if (p.max_octaves < 0 || p.max_octaves > SIFT3D_MAX_OCTAVES) return fail(err, "max_octaves must be in 0..16");
    if (p.sign_sum_min < 1 || p.sign_sum_min > 80) return fail(err, "sign_sum_min must be in 1..80");
    if (!(p.contrast_thresh >= 0.0) || !std::isfinite(p.contrast_thresh))
        return fail(err, "contrast_thresh must be finite and >= 0");
    if (!(p.curvature_r >= 1.0) || !std::isfinite(p.curvature_r)) return fail(err, "curvature_r must be >= 1");
    if (!(p.trunc > 0.0) || !(p.trunc <= 10.0)) return fail(err, "trunc must be in (0, 10]");
    if (!(p.desc_blur_sigma >= 0.0) || !std::isfinite(p.desc_blur_sigma))
        return fail(err, "desc_blur_sigma must be finite and >= 0");
    if (p.desc_method < 1 || p.desc_method > 5) return fail(err, "desc_method must be 1..5");
    if (p.storage < SIFT3D_STORAGE_F32 || p.storage > SIFT3D_STORAGE_BF16) return fail(err, "bad storage");
    if (p.max_keypoints < 0 || p.max_keypoints > (1 << 20)) return fail(err, "max_keypoints must be in 0..2^20");
    if (p.max_inflight < 1 || p.max_inflight > 64) return fail(err, "max_inflight must be in 1..64");
    if (p.refine < 0 || p.refine > 1) return fail(err, "refine must be 0 or 1");
    if (p.test_wait_timeout < 0 || p.test_wait_timeout > 1000) return fail(err, "test_wait_timeout must be in 0..1000");
    if (p.autotune < 0 || p.autotune > 1) return fail(err, "autotune must be 0 or 1");
    if (p.conv_row_tile != 0 && p.conv_row_tile != 8 && p.conv_row_tile != 16)
        return fail(err, "conv_row_tile must be 0, 8 or 16");
    if (p.conv_z_tile != 0 && p.conv_z_tile != 8 && p.conv_z_tile != 16)
        return fail(err, "conv_z_tile must be 0, 8 or 16");

    // filter radii of the schedule
    const int S = p.scales_per_octave;
    double sig[kMaxLevels];
    for (int s = 0; s < S + 3; ++s) sig[s] = p.sigma0 * std::pow(2.0, (double)s / S);
    const double s_init = std::sqrt(p.sigma0 * p.sigma0 - p.sigma_in * p.sigma_in);
    int rmax = radius_of(s_init, p.trunc);
    for (int s = 1; s < S + 3; ++s) {
        const double inc = std::sqrt(sig[s] * sig[s] - sig[s - 1] * sig[s - 1]);
        rmax = std::max(rmax, radius_of(inc, p.trunc));
    }
    if (p.desc_blur_sigma > 0.0) rmax = std::max(rmax, radius_of(p.desc_blur_sigma, p.trunc));
    if (rmax > kMaxRadius) return fail(err, "a filter radius ceil(trunc*sigma) exceeds 16");
    return SIFT3D_OK;
}

int make_plan(const sift3d_params& p, int nx, int ny, int nz, int in_dtype, Plan* out, std::string* err) {
    int rc = validate_params(p, err);
    if (rc != SIFT3D_OK) return rc;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4095 || ny > 4095 || nz > 4095)
        return fail(err, "each dimension must be in 1..4095");
    Plan& pl = *out;
    pl = Plan{};
    pl.p = p;
    pl.nx = nx;
    pl.ny = ny;
    pl.nz = nz;
    pl.S = p.scales_per_octave;
    pl.L = pl.S + 3;
    pl.nD = pl.S + 2;
    pl.elem = p.storage == SIFT3D_STORAGE_F32 ? 4 : 2;
    for (int s = 0; s < pl.L; ++s) pl.sig_level[s] = p.sigma0 * std::pow(2.0, (double)s / pl.S);
    pl.sig_init = std::sqrt(p.sigma0 * p.sigma0 - p.sigma_in * p.sigma_in);
    pl.r_init = radius_of(pl.sig_init, p.trunc);
    pl.t_init = make_taps(pl.sig_init, pl.r_init);
    for (int s = 1; s < pl.L; ++s) {
        pl.sig_inc[s - 1] = std::sqrt(pl.sig_level[s] * pl.sig_level[s] - pl.sig_level[s - 1] * pl.sig_level[s - 1]);
        pl.r_inc[s - 1] = radius_of(pl.sig_inc[s - 1], p.trunc);
        pl.t_inc[s - 1] = make_taps(pl.sig_inc[s - 1], pl.r_inc[s - 1]);
    }
    pl.sig_desc = p.desc_blur_sigma;
    pl.r_desc = p.desc_blur_sigma > 0.0 ? radius_of(p.desc_blur_sigma, p.trunc) : 0;
    if (pl.r_desc > 0) pl.t_desc = make_taps(pl.sig_desc, pl.r_desc);

    int cx = nx, cy = ny, cz = nz;
    while (std::min(cx, std::min(cy, cz)) >= p.min_octave_dim &&
           (p.max_octaves <= 0 || pl.nO < p.max_octaves) && pl.nO < SIFT3D_MAX_OCTAVES) {
        OctaveGeom& g = pl.oct[pl.nO++];
        g.nx = cx;
        g.ny = cy;
        g.nz = cz;
        g.py = (int64_t)round_up((size_t)cx, 8);
        g.pz = g.py * cy;
        cx /= 2;
        cy /= 2;
        cz /= 2;
    }
    if ((int64_t)pl.oct[0].pz * nz >= (1ll << 31) && pl.nO > 0) return fail(err, "volume too large");
    size_t off = 0;
    for (int o = 0; o < pl.nO; ++o) {
        const size_t vox = (size_t)(pl.oct[o].pz * pl.oct[o].nz);
        const size_t lvl = round_up(vox * pl.elem, 256);
        const size_t lvl_d = round_up(vox * Plan::elem_d, 256);
        const size_t tmp = round_up(vox * 4, 256);
        for (int s = 0; s < pl.L; ++s) { pl.off_G[o][s] = off; off += lvl; }
        for (int s = 0; s < pl.nD; ++s) { pl.off_D[o][s] = off; off += lvl_d; }
        if (pl.elem == 2) { pl.off_R[o] = off; off += round_up(vox * 2, 256); }
        if (pl.r_desc > 0)
            for (int s = 0; s < pl.S; ++s) { pl.off_B[o][s] = off; off += lvl; }
        pl.off_T[o] = off;
        off += tmp;
        if (pl.r_desc > 0)
            for (int s = 0; s < pl.S; ++s) { pl.off_TB[o][s] = off; off += tmp; }
    }
    pl.bytes = off;

    // Byte model of the pyramid + DoG + peak path per volume: per octave
    // 1 read of the base, L-1 writes of G_1.., L-2 re-reads of G_1.. as filter
    // input, 1 read of G_S, 1/8 write of the next base (Gaussian levels, elem
    // bytes each), and L-1 writes and L-1 reads of D (elem_d bytes); octave 0
    // also writes G_0 and reads the input at its own width.
    const double per_octave_g = 2.0 * pl.L - 0.875, per_octave_d = 2.0 * (pl.L - 1);
    double model = 0.0;
    for (int o = 0; o < pl.nO; ++o)
        model += (per_octave_g * (double)pl.elem + per_octave_d * (double)Plan::elem_d) * (double)pl.oct[o].voxels();
    if (pl.nO > 0) {
        const double in_elem = in_dtype == SIFT3D_DTYPE_U8 ? 1.0 : 4.0;
        const double n0 = (double)pl.oct[0].voxels();
        model += n0 * (double)pl.elem;                  // octave 0 writes G_0
        model += n0 * (in_elem - (double)pl.elem);      // its base read is the input
    }
    pl.algo_bytes = (uint64_t)std::llround(model);
    return SIFT3D_OK;
}

void fill_plan_info(const Plan& pl, sift3d_plan_info* info) {
    memset(info, 0, sizeof(*info));
    info->n_octaves = pl.nO;
    info->n_levels = pl.L;
    for (int o = 0; o < pl.nO; ++o) {
        info->dims[o][0] = pl.oct[o].nx;
        info->dims[o][1] = pl.oct[o].ny;
        info->dims[o][2] = pl.oct[o].nz;
        info->pitch_y[o] = pl.oct[o].py;
        info->pitch_z[o] = pl.oct[o].pz;
    }
    for (int s = 0; s < pl.L; ++s) info->sigma_level[s] = pl.sig_level[s];
    info->sigma_initial = pl.sig_init;
    info->radius_initial = pl.r_init;
    for (int s = 0; s + 1 < pl.L; ++s) {
        info->sigma_increment[s] = pl.sig_inc[s];
        info->radius_increment[s] = pl.r_inc[s];
    }
    info->radius_desc = pl.r_desc;
    info->workspace_bytes = pl.bytes;
    info->algorithmic_bytes = pl.algo_bytes;
}

// ---- point-pair pattern ------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): the state advances by the golden-ratio
// increment and each output is the state passed through the two-multiply mixer.
namespace {
struct SplitMix64 {
    uint64_t state;
    uint64_t next() {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    // 53 random bits mapped to the open interval (0, 1)
    double uniform() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    // Box-Muller, cosine branch only
    double normal() {
        const double u = uniform();
        const double v = uniform();
        return std::sqrt(-2.0 * std::log(u)) * std::cos(2.0 * 3.14159265358979323846 * v);
    }
};
}  // namespace

namespace {
// mean + N(0, I), redrawn until every |coordinate| <= clip
void normal_point(SplitMix64& g, const double* mean, double clip, double* q) {
    for (;;) {
        for (int c = 0; c < 3; ++c) q[c] = mean[c] + g.normal();
        if (std::fabs(q[0]) <= clip && std::fabs(q[1]) <= clip && std::fabs(q[2]) <= clip) return;
    }
}

// uniform in the ball of radius r: three uniforms on (-r, r), redrawn until inside
void ball_point(SplitMix64& g, double r, double* q) {
    for (;;) {
        for (int c = 0; c < 3; ++c) q[c] = r * (2.0 * g.uniform() - 1.0);
        if (q[0] * q[0] + q[1] * q[1] + q[2] * q[2] <= r * r) return;
    }
}
}  // namespace

// Point pairs in units of the keypoint scale (Sec. 2.2.3):
//   1: p1, p2 uniform in the ball of radius 2;   2: p1, p2 ~ N(0, I);
//   3: p1 ~ N(0, I), p2 ~ N(p1, I);                4: p1 = 0, p2 ~ N(0, I);
//   5: p1 = 0, p2 on the spherical grid radius {0.5, 1, 1.5, 2} x cos(theta)
//      {0.75, 0.25, -0.25, -0.75} x azimuth pi/2 * a (+ pi/4 on odd rings),
//      pair 16 m + 4 j + a.
// Normal draws are redrawn while any |coordinate| > 4.
void make_pattern(const sift3d_params& p, float* out) {
    SplitMix64 g{p.pattern_seed};
    const double clip = 4.0;
    const double zero[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < SIFT3D_N_PAIRS; ++k) {
        double p1[3] = {0.0, 0.0, 0.0}, p2[3] = {0.0, 0.0, 0.0};
        switch (p.desc_method) {
            case 1:
                ball_point(g, 2.0, p1);
                ball_point(g, 2.0, p2);
                break;
            case 2:
                normal_point(g, zero, clip, p1);
                normal_point(g, zero, clip, p2);
                break;
            case 4:
                normal_point(g, zero, clip, p2);
                break;
            case 5: {
                static const double radii[4] = {0.5, 1.0, 1.5, 2.0};
                static const double cos_theta[4] = {0.75, 0.25, -0.25, -0.75};
                const int m = (k / 16) % 4, j = (k / 4) % 4, a = k % 4;
                const double pi = 3.14159265358979323846;
                const double ct = cos_theta[j], st = std::sqrt(1.0 - ct * ct);
                const double phi = 0.5 * pi * a + (j % 2 == 1 ? 0.25 * pi : 0.0);
                p2[0] = radii[m] * st * std::cos(phi);
                p2[1] = radii[m] * st * std::sin(phi);
                p2[2] = radii[m] * ct;
                break;
            }
            default:   // 3
                normal_point(g, zero, clip, p1);
                normal_point(g, p1, clip, p2);
                break;
        }
        for (int c = 0; c < 3; ++c) {
            out[k * 6 + c] = (float)p1[c];
            out[k * 6 + 3 + c] = (float)p2[c];
        }
    }
}

// ---- workspaces -------------------------------------------------------------
size_t workspace_bytes(const Plan& plan, int capacity) {
    const size_t rec = round_up((size_t)std::max(capacity, 1) * sizeof(sift3d_keypoint), 256);
    return plan.bytes + rec + 256;
}

int bind_workspace(const Plan& plan, int capacity, char* base, Workspace* ws, std::string* err) {
    ws->plan = plan;
    ws->capacity = capacity;
    ws->base = base;
    ws->bytes = workspace_bytes(plan, capacity);
    const size_t rec = round_up((size_t)std::max(capacity, 1) * sizeof(sift3d_keypoint), 256);
    ws->staging = reinterpret_cast<sift3d_keypoint*>(ws->base + plan.bytes);
    ws->count = reinterpret_cast<int*>(ws->base + plan.bytes + rec);
    ws->count_out = ws->count + 1;
    return SIFT3D_OK;
}

namespace {
std::atomic<int> g_fail_countdown{0};   // > 0: allocations left until the one that fails

bool injected_failure() {
    int n = g_fail_countdown.load();
    while (n > 0)
        if (g_fail_countdown.compare_exchange_weak(n, n - 1)) return n == 1;
    return false;
}
}  // namespace

void set_allocation_failure(int n) { g_fail_countdown.store(n > 0 ? n : 0); }

cudaError_t dev_alloc(void** p, size_t bytes) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t pinned_alloc(void** p, size_t bytes, unsigned flags) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaHostAlloc(p, bytes, flags);
}

int alloc_device_zeroed(size_t bytes, char** out, std::string* err) {
    void* p = nullptr;
    cudaError_t e = dev_alloc(&p, bytes);
    if (e == cudaSuccess) e = cudaMemset(p, 0, bytes);   // padding columns start finite
    if (e != cudaSuccess) {
        if (p) cudaFree(p);
        (void)cudaGetLastError();
        if (err) *err = std::string("device allocation of the workspace failed: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SIFT3D_ENOMEM : SIFT3D_ECUDA;
    }
    *out = static_cast<char*>(p);
    return SIFT3D_OK;
}

int alloc_workspace(const Plan& plan, int capacity, Workspace* ws, std::string* err) {
    char* base = nullptr;
    int rc = alloc_device_zeroed(workspace_bytes(plan, capacity), &base, err);
    if (rc != SIFT3D_OK) return rc;
    rc = bind_workspace(plan, capacity, base, ws, err);
    ws->owns_base = true;
    return rc;
}

void free_workspace(Workspace* ws) {
    if (ws->base && ws->owns_base) cudaFree(ws->base);
    ws->base = nullptr;
}

int device_sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            (void)cudaGetLastError();
            v = 148;   // a grid for plans built without a device (host tests)
        }
        return v;
    }();
    return n;
}

cudaError_t launch_spec(const LaunchSpec& s, void** args, cudaStream_t st) {
    return cudaLaunchKernel(s.func, s.grid, s.block, args, s.smem, st);
}

PeakArgs make_peak_args(const Workspace& ws, int o) {
    const Plan& pl = ws.plan;
    const OctaveGeom& g = pl.oct[o];
    PeakArgs pa{};
    for (int s = 0; s < pl.nD; ++s) pa.dog[s] = ws.D(o, s);
    pa.py = g.py;
    pa.pz = g.pz;
    pa.nx = g.nx;
    pa.ny = g.ny;
    pa.nz = g.nz;
    pa.octave = o;
    pa.n_scales = pl.S;
    pa.ns = pl.S;
    pa.scale_base = 0;
    pa.border = pl.p.border;
    pa.sign_sum_min = pl.p.sign_sum_min;
    pa.contrast = (float)pl.p.contrast_thresh;
    const double r = pl.p.curvature_r;
    pa.curv_k1 = (float)((2.0 * r + 1.0) * (2.0 * r + 1.0) * (2.0 * r + 1.0));
    pa.curv_k2 = (float)(r * r);
    for (int s = 0; s < pl.L; ++s) pa.sigma_level[s] = (float)pl.sig_level[s];
    pa.refine = pl.p.refine;
    pa.out = ws.staging;
    pa.count = ws.count;
    pa.capacity = ws.capacity;
    return pa;
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    // The driver entry point, looked up once (no link-time dependency on libcuda).
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        (void)cudaGetLastError();
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}
}  // namespace


bool make_peak_tma_args(const Workspace& ws, int o, int first_scale, int ns, PeakTmaArgs* out) {
    const Plan& pl = ws.plan;
    const OctaveGeom& g = pl.oct[o];
    PeakTmaArgs& A = *out;
    memset(&A, 0, sizeof(A));
    A.a = make_peak_args(ws, o);
    A.a.ns = ns;
    A.a.scale_base = first_scale - 1;
    A.err = ws.count + 3;
    int box_x, box_y, box_z, box_l;
    peak_layout(pl.p.storage, A.a, &A.x_start, &box_x, &box_y, &box_z, &box_l);
    A.test_flag = ws.test_flag;
    const int l0 = first_scale - 1, nl = ns + 2;   // staged DoG levels l0 .. l0+nl-1
    const size_t stride = pl.off_D[o][1] - pl.off_D[o][0];
    for (int s = l0; s + 1 < l0 + nl; ++s)
        if (pl.off_D[o][s + 1] - pl.off_D[o][s] != stride) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (enc == nullptr) return false;
    const CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;   // DoG levels are float32
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)nl};
    const cuuint64_t strides[3] = {(cuuint64_t)g.py * Plan::elem_d, (cuuint64_t)g.pz * Plan::elem_d,
                                   (cuuint64_t)stride};
    const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)box_z, (cuuint32_t)box_l};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(&A.dogs, dt, 4, ws.D(o, l0), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Whether the level-S z pass of octave o writes octave o+1's G_0 (float32
// storage, rows that fit one CTA pair); the next octave's first y/x pass then
// reads that G_0 instead of sub-sampling G_S itself.
static bool z_writes_next_base(const Plan& pl, int o) {
    return pl.p.storage == SIFT3D_STORAGE_F32 && o + 1 < pl.nO && pl.oct[o].py <= 256;
}

LevelArgs level_args(const Workspace& ws, int o, int s, const void* input, int dtype, bool fuse_blur,
                     bool z_sub) {
    const Plan& pl = ws.plan;
    const OctaveGeom& g = pl.oct[o];
    LevelArgs la;
    ConvXYArgs& xa = la.xy;
    xa = ConvXYArgs{};
    xa.dst = ws.T(o);
    xa.py = g.py;
    xa.pz = g.pz;
    xa.nx = g.nx;
    xa.ny = g.ny;
    xa.nz = g.nz;
    xa.src_scale = 1.0f;
    la.src_kind = 2;
    la.sub = false;
    if (o == 0 && s == 0) {   // the caller's volume, blurred from sigma_in to sigma_0
        xa.src = input;
        xa.src_py = pl.nx;
        xa.src_pz = (int64_t)pl.nx * pl.ny;
        la.src_kind = dtype == SIFT3D_DTYPE_U8 ? 1 : 0;
        xa.src_scale = dtype == SIFT3D_DTYPE_U8 ? 1.0f / 255.0f : 1.0f;
        xa.zero_count = ws.count;
        xa.taps = pl.t_init;
        la.radius = pl.r_init;
    } else if (s == 1 && o > 0 && z_sub && z_writes_next_base(pl, o - 1)) {
        // G_0 written by the previous octave's level-S z pass
        xa.src = ws.G(o, 0);
        xa.src_py = g.py;
        xa.src_pz = g.pz;
        xa.taps = pl.t_inc[0];
        la.radius = pl.r_inc[0];
    } else if (s == 1 && o > 0) {   // sub-sample of the previous octave's level S
        la.sub = true;
        xa.src = ws.G(o - 1, pl.S);
        xa.src_py = pl.oct[o - 1].py;
        xa.src_pz = pl.oct[o - 1].pz;
        xa.base_out = ws.G(o, 0);
        xa.res_out = ws.Res(o);
        xa.taps = pl.t_inc[0];
        la.radius = pl.r_inc[0];
    } else {
        xa.src = ws.G(o, s - 1);
        xa.src_py = g.py;
        xa.src_pz = g.pz;
        xa.taps = pl.t_inc[s - 1];
        la.radius = pl.r_inc[s - 1];
    }
    // With fuse_blur the level's own y/x pass also applies the descriptor
    // pre-blur to its source G_{s-1} (s-1 = 1..S) when the fused variant exists.
    la.fused_blur = fuse_blur && pl.r_desc == kFusedBlurRadius && g.nx <= 256 && !la.sub && la.src_kind == 2 && s - 1 >= 1 &&
                    s - 1 <= pl.S && la.radius >= kFusedBlurRadius;
    if (la.fused_blur) {
        xa.dst2 = ws.TB(o, s - 1);
        xa.taps2 = pl.t_desc;
    }
    xa.row_tile = pl.p.conv_row_tile;
    ConvZArgs& za = la.z;
    za = ConvZArgs{};
    za.src = ws.T(o);
    za.dst = ws.G(o, s);
    za.py = g.py;
    za.pz = g.pz;
    za.nx = g.nx;
    za.ny = g.ny;
    za.nz = g.nz;
    za.taps = xa.taps;
    za.z_tile = pl.p.conv_z_tile;
    if (s > 0) {
        za.prev = ws.G(o, s - 1);
        za.dog = static_cast<float*>(ws.D(o, s - 1));
    }
    za.res = ws.Res(o);
    if (z_sub && s == pl.S && z_writes_next_base(pl, o)) {
        za.sub_dst = static_cast<float*>(ws.G(o + 1, 0));
        za.sub_py = pl.oct[o + 1].py;
        za.sub_pz = pl.oct[o + 1].pz;
    }
    if (la.fused_blur) {
        za.src2 = ws.TB(o, s - 1);
        za.dst2 = ws.B(o, s - 1);
        za.taps2 = pl.t_desc;
    }
    return la;
}

// ---- detect DAG ---------------------------------------------------------------
std::vector<Node> build_detect(const Workspace& ws, const DetectCall& c, int* first_node, int* sort_node) {
    const Plan& pl = ws.plan;
    const int st = pl.p.storage;
    std::vector<Node> nodes;
    auto add = [&](const LaunchSpec& s, auto args, std::vector<int> deps) {
        Node n;
        n.spec = s;
        n.set_args(args);
        n.deps = std::move(deps);
        nodes.push_back(std::move(n));
        return (int)nodes.size() - 1;
    };
    auto tag = [&](int idx, const char* fmt, int a, int b, uint64_t bytes) {
        char buf[64];
        snprintf(buf, sizeof(buf), fmt, a, b, nodes[idx].spec.name);
        nodes[idx].label = buf;
        nodes[idx].algo_bytes = bytes;
        nodes[idx].octave = a;
    };
    const uint64_t e = pl.elem;
    const uint64_t ed = Plan::elem_d;
    const uint64_t in_e = c.dtype == SIFT3D_DTYPE_U8 ? 1 : 4;
    std::vector<int> peak_nodes;
    int g_node[SIFT3D_MAX_OCTAVES][kMaxLevels];
    *first_node = -1;
    for (int o = 0; o < pl.nO; ++o) {
        const OctaveGeom& g = pl.oct[o];
        int prev = -1;  // node that produced G_{s-1}
        for (int s = (o == 0 ? 0 : 1); s < pl.L; ++s) {
            LevelArgs la = level_args(ws, o, s, c.input, c.dtype, false, true);
            ConvXYArgs& xa = la.xy;
            const int src_kind = la.src_kind, radius = la.radius;
            const bool sub = la.sub;
            std::vector<int> deps;
            if (s == 1 && o > 0) deps.push_back(g_node[o - 1][pl.S]);
            else if (!(o == 0 && s == 0)) deps.push_back(prev);
            xa.row_tile = pl.p.conv_row_tile;
            const LaunchSpec xspec = conv_xy_spec(radius, src_kind, st, sub, xa);   // sets xa.row_tile
            const int nxy = add(xspec, xa, deps);
            nodes[nxy].xy = {radius, src_kind, sub, true};
            if (*first_node < 0) *first_node = nxy;
            {
                const uint64_t N = (uint64_t)g.voxels();
                // reads its source once, writes the float32 intermediate
                // (sub-sample mode: reads 8 source voxels per voxel, also writes G_0)
                const uint64_t rd = (o == 0 && s == 0) ? in_e * N : (sub ? 8 * e * N : e * N);
                tag(nxy, "o%d.s%d.%s", o, s, rd + 4 * N + (sub ? e * N : 0) + (xa.dst2 ? 4 * N : 0));
            }
            ConvZArgs& za = la.z;
            prev = add(conv_z_spec(radius, st, za), za, {nxy});
            if (za.sub_dst == nullptr) nodes[prev].zk = {radius, true};
            {
                const uint64_t N = (uint64_t)g.voxels();
                // reads the intermediate, writes G_s; with the DoG also reads
                // G_{s-1} and writes D_{s-1}; with the fused pre-blur also reads
                // its intermediate and writes the pre-blurred level
                tag(prev, "o%d.s%d.%s", o, s,
                    4 * N + e * N + (s > 0 ? (e + ed) * N : 0) + (za.dst2 ? (4 + e) * N : 0) +
                        (za.sub_dst ? (uint64_t)pl.oct[o + 1].voxels() * e : 0));   // + the next G_0
            }
            g_node[o][s] = prev;
        }
        if (o > 0) g_node[o][0] = g_node[o][1];
        // peak detection on D_1..D_S: one launch per octave after its last level
        // (one launch per scale, each as soon as its DoG levels exist, reads
        // every DoG level up to three times and measured slower: 0.309 against
        // 0.286 ms per detect + describe of 145x174x145)
        if (g.nx - 2 * pl.p.border >= 1 && g.ny - 2 * pl.p.border >= 1 && g.nz - 2 * pl.p.border >= 1) {
            PeakTmaArgs pa;
            LaunchSpec ps;
            if (make_peak_tma_args(ws, o, 1, pl.S, &pa)) ps = peak_spec(st, pa);
            else ps.name = "peak (DoG tensor map)";
            peak_nodes.push_back(add(ps, pa, {g_node[o][pl.S + 2]}));
            // the 80-neighbour test reads the S + 2 DoG levels in full
            tag(peak_nodes.back(), "o%d.d1-%d.%s", o, pl.S, (uint64_t)(pl.S + 2) * ed * (uint64_t)g.voxels());
        }
        // pre-blur of G_1..G_S for the descriptors (Sec. 2.2.3): a y/x and a z
        // pass per level, each branch depending only on its G_s, so the work
        // runs beside the octave chain instead of on it (fused into the level
        // passes it measured 0.286 against 0.277 ms per detect + describe of
        // 145x174x145)
        if (pl.r_desc > 0) {
            for (int s = 1; s <= pl.S; ++s) {
                ConvXYArgs xa{};
                xa.src = ws.G(o, s);
                xa.src_py = g.py;
                xa.src_pz = g.pz;
                xa.src_scale = 1.0f;
                xa.dst = ws.TB(o, s);
                xa.py = g.py;
                xa.pz = g.pz;
                xa.nx = g.nx;
                xa.ny = g.ny;
                xa.nz = g.nz;
                xa.taps = pl.t_desc;
                xa.row_tile = pl.p.conv_row_tile;
                const LaunchSpec xspec = conv_xy_spec(pl.r_desc, 2, st, false, xa);   // sets xa.row_tile
                const int nxy = add(xspec, xa, {g_node[o][s]});
                nodes[nxy].xy = {pl.r_desc, 2, false, true};
                tag(nxy, "o%d.b%d.%s", o, s, (e + 4) * (uint64_t)g.voxels());
                ConvZArgs za{};
                za.src = ws.TB(o, s);
                za.dst = ws.B(o, s);
                za.py = g.py;
                za.pz = g.pz;
                za.nx = g.nx;
                za.ny = g.ny;
                za.nz = g.nz;
                za.taps = pl.t_desc;
                za.z_tile = pl.p.conv_z_tile;
                const int nz_ = add(conv_z_spec(pl.r_desc, st, za), za, {nxy});
                nodes[nz_].zk = {pl.r_desc, true};
                tag(nz_, "o%d.b%d.%s", o, s, (4 + e) * (uint64_t)g.voxels());
            }
        }
    }
    SortArgs sa{};
    sa.staging = ws.staging;
    sa.err = ws.count + 3;
    sa.out = c.out;
    sa.count = ws.count;
    sa.count_out = ws.count_out;
    sa.capacity = ws.capacity;
    std::vector<int> deps = peak_nodes;
    if (deps.empty() && *first_node >= 0) deps.push_back((int)nodes.size() - 1);
    *sort_node = add(sort_spec(sa), sa, deps);
    tag(*sort_node, "o%d.x%d.%s", 0, 0, 0);
    nodes[*sort_node].label = "sort";
    nodes[*sort_node].octave = -1;
    return nodes;
}

int64_t blur_pitch_elems(int nx, int ny, int nz) {
    return (int64_t)round_up((size_t)nx, 8) * ny * nz;
}

int enqueue_blur(const float* in, int nx, int ny, int nz, double sigma, double trunc, float* t, float* u,
                 float* out, cudaStream_t st, std::string* err) {
    const int R = radius_of(sigma, trunc);
    if (!(sigma > 0.0) || R < 1 || R > kMaxRadius) {
        if (err) *err = "sigma must be > 0 with ceil(trunc*sigma) in 1..16";
        return SIFT3D_EINVAL;
    }
    const int64_t py = (int64_t)round_up((size_t)nx, 8), pz = py * ny;
    ConvXYArgs xa{};
    xa.src = in;
    xa.src_py = nx;
    xa.src_pz = (int64_t)nx * ny;
    xa.src_scale = 1.0f;
    xa.dst = t;
    xa.py = py;
    xa.pz = pz;
    xa.nx = nx;
    xa.ny = ny;
    xa.nz = nz;
    xa.taps = gaussian_taps(sigma, R);
    ConvZArgs za{};
    za.src = t;
    za.dst = u;
    za.py = py;
    za.pz = pz;
    za.nx = nx;
    za.ny = ny;
    za.nz = nz;
    za.taps = xa.taps;
    ReadLevelArgs ra{};
    ra.src = u;
    ra.py = py;
    ra.pz = pz;
    ra.nx = nx;
    ra.ny = ny;
    ra.nz = nz;
    ra.dst = out;
    const LaunchSpec s1 = conv_xy_spec(R, 0, SIFT3D_STORAGE_F32, false, xa);
    const LaunchSpec s2 = conv_z_spec(R, SIFT3D_STORAGE_F32, za);
    const LaunchSpec s3 = read_level_spec(SIFT3D_STORAGE_F32, ra);
    void* a1 = &xa;
    void* a2 = &za;
    void* a3 = &ra;
    cudaError_t e = cudaLaunchKernel(s1.func, s1.grid, s1.block, &a1, s1.smem, st);
    if (e == cudaSuccess) e = cudaLaunchKernel(s2.func, s2.grid, s2.block, &a2, s2.smem, st);
    if (e == cudaSuccess) e = cudaLaunchKernel(s3.func, s3.grid, s3.block, &a3, s3.smem, st);
    if (e != cudaSuccess) {
        if (err) *err = std::string("blur launch: ") + cudaGetErrorString(e);
        return SIFT3D_ECUDA;
    }
    return SIFT3D_OK;
}

DescribeArgs make_describe_args(const Workspace& ws, const float* pattern) {
    DescribeArgs a{};
    const Plan& pl = ws.plan;
    a.n_scales = pl.S;
    a.n_octaves = pl.nO;
    for (int o = 0; o < pl.nO; ++o)
        for (int s = 1; s <= pl.S; ++s) {
            DescLevel& L = a.lv[o][s - 1];
            L.ptr = ws.B(o, s);
            L.py = pl.oct[o].py;
            L.pz = pl.oct[o].pz;
            L.nx = pl.oct[o].nx;
            L.ny = pl.oct[o].ny;
            L.nz = pl.oct[o].nz;
            L.sigma = (float)pl.sig_level[s];
        }
    memcpy(a.pattern, pattern, sizeof(a.pattern));
    return a;
}

DetectExec::~DetectExec() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : ev_begin) cudaEventDestroy(e);
    for (cudaEvent_t e : ev_end) cudaEventDestroy(e);
}

namespace {
int cuda_fail(std::string* err, const char* what, cudaError_t e) {
    if (err) *err = std::string(what) + ": " + cudaGetErrorString(e);
    return SIFT3D_ECUDA;
}

cudaKernelNodeParams node_params(Node& n) {
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(n.spec.func);
    kp.gridDim = n.spec.grid;
    kp.blockDim = n.spec.block;
    kp.sharedMemBytes = (unsigned)n.spec.smem;
    kp.kernelParams = &n.argp;
    kp.extra = nullptr;
    return kp;
}
}  // namespace

namespace {
// Tile heights of the y/x pass chosen by timing, per (dims, radius, source
// kind, storage, sub-sampling, fused pre-blur), for the whole process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int, int, int>, int> g_tuned;

// Time one y/x node at each candidate tile height on stream st (CUDA events,
// one warm-up and three timed launches each) and keep the fastest in the node.
// Its outputs are workspace intermediates the detect overwrites afterwards.
int tune_xy_node(Node& n, int storage, cudaStream_t st, std::string* err) {
    ConvXYArgs xa;
    memcpy(&xa, n.arg.data(), sizeof(xa));
    if (xa.nx > 256) return SIFT3D_OK;   // the tiled kernel for wide rows has no tile height
    const auto key = std::make_tuple(xa.nx, xa.ny, xa.nz, n.xy.radius, n.xy.src_kind, storage, (int)n.xy.sub,
                                     xa.dst2 != nullptr ? 1 : 0);
    int best = 0;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) best = it->second;
    }
    if (best == 0) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        float best_ms = 0.f;
        for (int ty : {8, 16}) {
            if (e != cudaSuccess) break;
            xa.row_tile = ty;
            const LaunchSpec s = conv_xy_spec(n.xy.radius, n.xy.src_kind, storage, n.xy.sub, xa);
            if (s.func == nullptr) continue;
            void* args[1] = {&xa};
            e = launch_spec(s, args, st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_spec(s, args, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (best == 0 || ms < best_ms)) best = ty, best_ms = ms;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e != cudaSuccess) {
            if (err) *err = std::string("autotune: ") + cudaGetErrorString(e);
            return SIFT3D_ECUDA;
        }
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tuned[key] = best;
    }
    memcpy(&xa, n.arg.data(), sizeof(xa));
    xa.row_tile = best;
    n.spec = conv_xy_spec(n.xy.radius, n.xy.src_kind, storage, n.xy.sub, xa);
    n.set_args(xa);
    return SIFT3D_OK;
}

// Outputs per thread of a float32 z pass (8 or 16) chosen by timing, per
// (dims, radius, with DoG), for the whole process; as tune_xy_node.
std::map<std::tuple<int, int, int, int, int>, int> g_tuned_z;

int tune_z_node(Node& n, int storage, cudaStream_t st, std::string* err) {
    if (storage != SIFT3D_STORAGE_F32) return SIFT3D_OK;   // 16-bit storage has one depth
    ConvZArgs za;
    memcpy(&za, n.arg.data(), sizeof(za));
    const auto key = std::make_tuple(za.nx, za.ny, za.nz, n.zk.radius, za.dog != nullptr ? 1 : 0);
    int best = 0;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tuned_z.find(key);
        if (it != g_tuned_z.end()) best = it->second;
    }
    if (best == 0) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        float best_ms = 0.f;
        for (int tz : {16, 8}) {
            if (e != cudaSuccess) break;
            za.z_tile = tz;
            const LaunchSpec s = conv_z_spec(n.zk.radius, storage, za);
            if (s.func == nullptr) continue;
            void* args[1] = {&za};
            e = launch_spec(s, args, st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_spec(s, args, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (best == 0 || ms < best_ms)) best = tz, best_ms = ms;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e != cudaSuccess) {
            if (err) *err = std::string("autotune: ") + cudaGetErrorString(e);
            return SIFT3D_ECUDA;
        }
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tuned_z[key] = best;
    }
    memcpy(&za, n.arg.data(), sizeof(za));
    za.z_tile = best;
    n.spec = conv_z_spec(n.zk.radius, storage, za);
    n.set_args(za);
    return SIFT3D_OK;
}
}  // namespace

int run_detect(Workspace& ws, DetectExec& ex, const DetectCall& c, bool use_graph, bool profile,
               cudaStream_t st, std::string* err) {
    if (ex.nodes.empty()) {
        ex.profile = profile;
        ex.nodes = build_detect(ws, c, &ex.first, &ex.sort);
        for (auto& n : ex.nodes)
            if (n.spec.func == nullptr) {
                if (err) *err = std::string("no kernel instance for this configuration: ") + n.spec.name;
                ex.nodes.clear();
                return SIFT3D_EINVAL;
            }
        // tile heights of the y/x passes and depths of the z passes: timed on
        // this device unless fixed, or unless the stream is being captured (no
        // synchronisation allowed there)
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) (void)cudaGetLastError();
        if (ws.plan.p.autotune && cap == cudaStreamCaptureStatusNone)
            for (auto& n : ex.nodes) {
                int rc = SIFT3D_OK;
                if (n.xy.valid && ws.plan.p.conv_row_tile == 0) rc = tune_xy_node(n, ws.plan.p.storage, st, err);
                if (n.zk.valid && ws.plan.p.conv_z_tile == 0 && rc == SIFT3D_OK)
                    rc = tune_z_node(n, ws.plan.p.storage, st, err);
                if (rc != SIFT3D_OK) {
                    ex.nodes.clear();
                    return rc;
                }
            }
        ex.cur_input = c.input;
        ex.cur_out = c.out;
        if (ex.profile) {
            ex.ev_begin.resize(ex.nodes.size());
            ex.ev_end.resize(ex.nodes.size());
            for (size_t i = 0; i < ex.nodes.size(); ++i) {
                cudaError_t e = cudaEventCreate(&ex.ev_begin[i]);
                if (e == cudaSuccess) e = cudaEventCreate(&ex.ev_end[i]);
                if (e != cudaSuccess) return cuda_fail(err, "cudaEventCreate", e);
            }
        }
    } else if (ex.cur_input != c.input || ex.cur_out != c.out) {
        // only the first conv (input) and the sort (output) see caller pointers
        ConvXYArgs xa;
        memcpy(&xa, ex.nodes[ex.first].arg.data(), sizeof(xa));
        xa.src = c.input;
        ex.nodes[ex.first].set_args(xa);
        SortArgs sa;
        memcpy(&sa, ex.nodes[ex.sort].arg.data(), sizeof(sa));
        sa.out = c.out;
        ex.nodes[ex.sort].set_args(sa);
        if (ex.exec) {
            for (int idx : {ex.first, ex.sort}) {
                cudaKernelNodeParams kp = node_params(ex.nodes[idx]);
                cudaError_t e = cudaGraphExecKernelNodeSetParams(ex.exec, ex.gnodes[idx], &kp);
                if (e != cudaSuccess) return cuda_fail(err, "cudaGraphExecKernelNodeSetParams", e);
            }
        }
        ex.cur_input = c.input;
        ex.cur_out = c.out;
    }
    if (!use_graph) {
        for (size_t i = 0; i < ex.nodes.size(); ++i) {
            Node& n = ex.nodes[i];
            if (ex.profile) cudaEventRecord(ex.ev_begin[i], st);
            cudaError_t e = launch_spec(n.spec, &n.argp, st);
            if (e != cudaSuccess) return cuda_fail(err, n.spec.name, e);
            if (ex.profile) cudaEventRecord(ex.ev_end[i], st);
        }
        return SIFT3D_OK;
    }
    if (!ex.exec) {
        cudaError_t e = cudaGraphCreate(&ex.graph, 0);
        if (e != cudaSuccess) return cuda_fail(err, "cudaGraphCreate", e);
        ex.gnodes.resize(ex.nodes.size());
        for (size_t i = 0; i < ex.nodes.size(); ++i) {
            std::vector<cudaGraphNode_t> deps;
            for (int d : ex.nodes[i].deps) deps.push_back(ex.gnodes[d]);
            if (ex.profile) {   // begin event -> kernel -> end event
                cudaGraphNode_t b;
                e = cudaGraphAddEventRecordNode(&b, ex.graph, deps.data(), deps.size(), ex.ev_begin[i]);
                if (e != cudaSuccess) return cuda_fail(err, "cudaGraphAddEventRecordNode", e);
                deps.assign(1, b);
            }
            cudaKernelNodeParams kp = node_params(ex.nodes[i]);
            e = cudaGraphAddKernelNode(&ex.gnodes[i], ex.graph, deps.data(), deps.size(), &kp);
            if (e != cudaSuccess) return cuda_fail(err, "cudaGraphAddKernelNode", e);
            if (ex.profile) {
                cudaGraphNode_t en;
                e = cudaGraphAddEventRecordNode(&en, ex.graph, &ex.gnodes[i], 1, ex.ev_end[i]);
                if (e != cudaSuccess) return cuda_fail(err, "cudaGraphAddEventRecordNode", e);
            }
        }
        e = cudaGraphInstantiate(&ex.exec, ex.graph, 0);
        if (e != cudaSuccess) return cuda_fail(err, "cudaGraphInstantiate", e);
    }
    cudaError_t e = cudaGraphLaunch(ex.exec, st);
    if (e != cudaSuccess) return cuda_fail(err, "cudaGraphLaunch", e);
    return SIFT3D_OK;
}

}  // namespace sift3d
