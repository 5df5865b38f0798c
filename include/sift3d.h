/*
 * sift3d.h - C ABI of the GB300 (sm_103a) 3D SIFT detector and BRIEF/RRIEF
 * descriptor library.
 *
 * The operations follow Carluer et al., "GPU optimization of the 3D
 * Scale-invariant Feature Transform Algorithm and a Novel BRIEF-inspired 3D Fast
 * Descriptor" (arXiv 2112.10258):
 *   - Gaussian scale space by separable x/y/z filtering ........ Sec. 2.2.2
 *     "Gaussian Convolution"; Fig. 8 (6 convolutions per octave)
 *   - octave sub-sampling by 2 (8 voxels -> 1) ................. Sec. 2.2.2
 *     "Sub-sampling"
 *   - difference of Gaussians DoG = I(sigma) - I(kappa sigma) .. Sec. 2.2.2
 *     "Difference-of-Gaussian"
 *   - 4D peak detection by the sum of signs over 80 neighbours . Sec. 2.2.2
 *     "4D Peak Detection" (sum-of-signs equation, +-80 cut)
 *   - BRIEF and RRIEF descriptors, point-pair method 3 ......... Sec. 2.2.3;
 *     pre-blur sigma 0.95 (Sec. 4.5)
 * The contrast and Hessian curvature tests and the serving calls have no
 * counterpart in the paper; their definitions are given below.
 *
 * Conventions (every function):
 *   - Return value: SIFT3D_OK (0), SIFT3D_PENDING (1, poll only) or a negative
 *     SIFT3D_E* code.  No C++ exception crosses this boundary.  The message of
 *     the last failure on a context is available from sift3d_last_error().
 *   - Volumes are dense, x fastest: voxel (x, y, z) is at x + nx*(y + ny*z).
 *     Each dimension must be in [1, 4095].
 *   - "dev_" pointers are CUDA device pointers owned by the caller; "host"
 *     pointers are ordinary host memory owned by the caller unless stated.
 *   - A context is not thread safe: calls on one context must not overlap,
 *     except sift3d_poll, which may be called from any thread.
 *   - Work is ordered on the caller's CUDA stream (cudaStream_t passed as
 *     void*; NULL = legacy default stream).  Only the calls that return host
 *     results (n_out != NULL in detect, poll) wait for the device.
 */
#ifndef SIFT3D_H
#define SIFT3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define SIFT3D_OK          0
#define SIFT3D_PENDING     1   /* sift3d_poll: request not finished yet          */
#define SIFT3D_EINVAL     -1   /* bad argument or parameter                      */
#define SIFT3D_ENOMEM     -2   /* device or host allocation failed               */
#define SIFT3D_ECAPACITY  -3   /* more keypoints than the output capacity        */
#define SIFT3D_ETIMEDOUT  -4   /* a bounded wait ran out                         */
#define SIFT3D_ECUDA      -5   /* a CUDA runtime call failed                     */
#define SIFT3D_ENOTFOUND  -6   /* unknown ticket                                 */
#define SIFT3D_EBUDGET    -7   /* request can never fit the HBM budget           */

/* ---- enumerations ------------------------------------------------------------ */
#define SIFT3D_DTYPE_F32   0   /* input voxels: float32, used as they are        */
#define SIFT3D_DTYPE_U8    1   /* input voxels: uint8 codes, converted to c/255  */

/* Storage of the pyramid.  Arithmetic is float32 in every mode, and the DoG
 * levels are always stored in float32: with the Gaussian levels in 16 bits,
 * each DoG D_{s-1} = G_{s-1} - G_s is formed from G_{s-1} as computed (the
 * stored 16-bit value plus its rounding residual, kept in a 16-bit side
 * buffer) and G_s before its rounding, so no storage rounding enters the
 * DoG; rounding the DoG itself to 16 bits would break near ties among the 80
 * neighbours.  The Gaussian and descriptor levels, the convolution sources
 * and the octave sub-sampling use the stored 16-bit values. */
#define SIFT3D_STORAGE_F32  0  /* Gaussian levels stored in float32              */
#define SIFT3D_STORAGE_F16  1  /* Gaussian levels stored in IEEE half            */
#define SIFT3D_STORAGE_BF16 2  /* Gaussian levels stored in bfloat16             */

#define SIFT3D_DESC_BRIEF  1
#define SIFT3D_DESC_RRIEF  2
#define SIFT3D_DESC_BOTH   3

#define SIFT3D_LEVEL_GAUSS 0   /* G_s,   s = 0..S+2                              */
#define SIFT3D_LEVEL_DOG   1   /* D_s = G_s - G_{s+1}, s = 0..S+1                */
#define SIFT3D_LEVEL_DESC  2   /* G_s pre-blurred for descriptors, s = 1..S      */

#define SIFT3D_SUBMIT_NOCOPY 1 /* submit flag: the caller keeps host_vol valid and
                                  unchanged until the request finishes; the
                                  library copies from it asynchronously (pinned
                                  host memory is read by DMA, no staging copy)  */
#define SIFT3D_SUBMIT_DEVICE 2 /* submit flag: the volume is device memory of the
                                  context's GPU, complete when sift3d_submit is
                                  called (its producer stream synchronised); the
                                  detect reads it in place, so the caller keeps
                                  it valid and unchanged until the request
                                  finishes.  No host-to-device copy.             */

#define SIFT3D_MAX_OCTAVES 16
#define SIFT3D_MAX_SCALES   5  /* scales_per_octave <= 5                         */
#define SIFT3D_N_PAIRS     64  /* point pairs per descriptor                     */

/* ---- parameters ---------------------------------------------------------------
 * The Gaussian levels of an octave are G_s, s = 0..S+2, at
 * sigma_s = sigma0 * 2^(s/S) octave voxels (S = scales_per_octave).  Octave 0
 * starts with a blur of sqrt(sigma0^2 - sigma_in^2) of the input; G_s is G_{s-1}
 * blurred by sqrt(sigma_s^2 - sigma_{s-1}^2); octave o+1 starts from the 2x2x2
 * mean of G_S of octave o.  A 1D pass uses w_k ~ exp(-k^2/2 sigma^2) for
 * |k| <= ceil(trunc*sigma), normalised to unit sum, with clamp-to-edge borders.
 * Octaves continue while min(nx,ny,nz) of the octave >= min_octave_dim (and,
 * if max_octaves > 0, for at most max_octaves octaves).
 * A voxel v of D_s (s = 1..S, at least `border` voxels from every face) is a
 * keypoint when
 *   |sum over the 80 neighbours n of sign(D_s(v) - D(n))| >= sign_sum_min
 *        (neighbours: 3x3x3 in D_{s-1} and D_{s+1}, 3x3x3 minus v in D_s),
 *   |D_s(v)| >= contrast_thresh, and
 *   H' = -polarity * (central-difference Hessian of D_s at v) is positive
 *   definite with tr(H')^3 * r^2 < (2r+1)^3 * det(H'), r = curvature_r.
 */
typedef struct sift3d_params {
    double   sigma0;             /* 1.6                                        */
    double   sigma_in;           /* 0.5  nominal blur of the input             */
    int32_t  scales_per_octave;  /* 3    (S), 1..SIFT3D_MAX_SCALES             */
    int32_t  min_octave_dim;     /* 16, >= 3                                   */
    int32_t  max_octaves;        /* 0 = no limit                               */
    int32_t  sign_sum_min;       /* 80 = strict extremum; 1..80                */
    int32_t  border;             /* 1, >= 1                                    */
    int32_t  profile;            /* 0; 1 = time every detect kernel with CUDA
                                    events (sift3d_stage_times).  The
                                    environment variable SIFT3D_PROFILE=1 sets
                                    it for every context sift3d_create makes. */
    double   contrast_thresh;    /* 0.005 (compared in float32 on the device)  */
    double   curvature_r;        /* 10, > 1                                    */
    double   trunc;              /* 4.0  filter radius = ceil(trunc * sigma)   */
    double   desc_blur_sigma;    /* 0.95; 0 = sample G_s without pre-blur     */
    int32_t  desc_method;        /* point pairs (Sec. 2.2.3), keypoint-scale
                                    units: 1 = both uniform in the ball of
                                    radius 2; 2 = both N(0,1); 3 (default) =
                                    p1 ~ N(0,1), p2 ~ N(p1,1); 4 = p1 = 0,
                                    p2 ~ N(0,1); 5 = p1 = 0, p2 on a spherical
                                    grid (4 radii x 16 directions)            */
    uint64_t pattern_seed;       /* seeds the SplitMix64 pattern generator     */
    int32_t  storage;            /* SIFT3D_STORAGE_*                           */
    int32_t  use_graphs;         /* 1 = replay detect as a captured CUDA graph */
    uint64_t hbm_budget_bytes;   /* serving admission budget (0 = 40 GiB)      */
    int32_t  max_keypoints;      /* serving: keypoints kept per request (8192) */
    int32_t  max_inflight;       /* serving: requests on the device at once (4) */
    int32_t  refine;             /* 0 (default); 1 = one Newton step on the
                                    4D (x, y, z, scale) quadratic of the DoG
                                    through the keypoint's 3^4 neighbourhood
                                    (central differences): x, y, z, sigma and
                                    dog report the interpolated extremum.  No
                                    counterpart in the paper; the keypoint set
                                    does not change.                          */
    int32_t  test_wait_timeout;  /* 0 (default).  k > 0 = for testing the error
                                    path: the first k detects of this context
                                    make the first wait of every peak-kernel
                                    CTA for its staged planes one non-blocking
                                    test, which finds the copy still in
                                    flight; the CTA sets the error flag, waits
                                    for all of its copies to land and leaves,
                                    and sift3d_detect returns
                                    SIFT3D_ETIMEDOUT.  Later detects on the
                                    same context run normally.  0..1000.     */
    int32_t  autotune;           /* 1 (default): at the first detect of a
                                    volume shape (outside stream capture),
                                    time each full-row y/x pass at tile
                                    heights of 8 and 16 rows, and each float32
                                    z pass at 8 and 16 outputs per thread,
                                    with CUDA events and keep the faster
                                    (cached per process); results are bitwise
                                    the same for either choice.  0 = 16 rows
                                    and 16 outputs.                           */
    int32_t  conv_row_tile;      /* 0 (default): as autotune says; 8 or 16 =
                                    rows per CTA of the y/x pass              */
    int32_t  conv_z_tile;        /* 0 (default): as autotune says; 8 or 16 =
                                    outputs per thread of the z pass (float32
                                    storage; 16-bit storage uses 16): the z
                                    halo of 2R planes is re-read per that many
                                    outputs                                   */
} sift3d_params;

/* A detected keypoint (48 bytes).  x,y,z are input-voxel coordinates of the
 * octave voxel centre, (i + 0.5) * 2^octave - 0.5; sigma = sigma_scale * 2^octave
 * input voxels. */
typedef struct sift3d_keypoint {
    float   x, y, z;
    float   sigma;
    int32_t ix, iy, iz;          /* position in the octave grid                */
    int16_t octave, scale;       /* scale s in 1..S                            */
    int8_t  polarity;            /* +1 DoG peak, -1 valley                     */
    int8_t  refined;             /* 0 = refinement off; 1 = x, y, z, sigma, dog
                                    refined (params.refine); 2 = its 4D
                                    Hessian was singular: left at the voxel  */
    int8_t  reserved0[2];
    float   dog;                 /* D_s(ix,iy,iz), or the refined value        */
    int32_t sign_sum;            /* sum of signs over the 80 neighbours        */
    int32_t reserved1;
} sift3d_keypoint;

/* Host-side description of the work for one volume size. */
typedef struct sift3d_plan_info {
    int32_t  n_octaves;
    int32_t  n_levels;                          /* S + 3                        */
    int32_t  dims[SIFT3D_MAX_OCTAVES][3];       /* nx, ny, nz per octave        */
    int64_t  pitch_y[SIFT3D_MAX_OCTAVES];       /* elements between rows        */
    int64_t  pitch_z[SIFT3D_MAX_OCTAVES];       /* elements between planes      */
    double   sigma_level[SIFT3D_MAX_SCALES + 3];/* sigma_s in octave voxels     */
    double   sigma_initial;                     /* octave-0 initial blur        */
    double   sigma_increment[SIFT3D_MAX_SCALES + 3]; /* [s-1]: G_{s-1} -> G_s   */
    int32_t  radius_initial;
    int32_t  radius_increment[SIFT3D_MAX_SCALES + 3];
    int32_t  radius_desc;                       /* 0 when desc_blur_sigma == 0  */
    uint64_t workspace_bytes;                   /* device bytes one detect holds */
    uint64_t algorithmic_bytes;                 /* byte model of the detect path */
} sift3d_plan_info;

/* Result of a served request (sift3d_poll).  Arrays are host memory owned by
 * the library, valid until sift3d_release(ticket). */
typedef struct sift3d_result {
    int32_t status;              /* SIFT3D_OK or SIFT3D_ECAPACITY               */
    int32_t n_keypoints;         /* records in keypoints / brief / rrief        */
    int32_t n_needed;            /* keypoints detected (> n_keypoints on ECAPACITY) */
    int32_t nx, ny, nz;
    const sift3d_keypoint* keypoints;
    const uint64_t* brief;       /* n_keypoints words, bit k = pair k          */
    const uint8_t*  rrief;       /* n_keypoints x 64 ranks                      */
    double  latency_ms;          /* submit -> results ready (host clock)        */
    double  queue_ms;            /* submit -> admitted to the device            */
} sift3d_result;

typedef struct sift3d_ctx sift3d_ctx;

/* Fill *out with the defaults listed beside each field above. */
int sift3d_default_params(sift3d_params* out);

/* Validate params and compute the octave schedule for an nx*ny*nz volume.
 * Host only; touches no device.  SIFT3D_EINVAL on bad params or dims. */
int sift3d_plan(const sift3d_params* params, int nx, int ny, int nz,
                sift3d_plan_info* out);

/* Write the 64 point pairs the descriptors use, as float
 * out[k*6 + p*3 + c] (pair k, point p in {0,1}, coordinate c = x,y,z), in units
 * of the keypoint's scale, for params->desc_method (Sec. 2.2.3, point selection
 * methods 1-5):
 *   1  p1, p2 uniform in the ball of radius 2 (three uniforms on (-2, 2) per
 *      point, redrawn until inside);
 *   2  p1, p2 ~ N(0,1) per coordinate;
 *   3  p1 ~ N(0,1), p2 ~ N(p1,1) per coordinate;
 *   4  p1 = 0, p2 ~ N(0,1);
 *   5  p1 = 0, p2 = r (sin t cos f, sin t sin f, cos t) with pair 16m + 4j + a:
 *      r = 0.5 (m+1), cos t = 0.75 - 0.5 j, f = pi/2 a + (j odd ? pi/4 : 0).
 * A normal point with any |coordinate| > 4 is redrawn.  Uniforms and normals
 * come from SplitMix64 seeded with pattern_seed (normals by Box-Muller, one cos
 * branch per pair of uniforms); method 5 uses no random numbers.  Host only.
 * SIFT3D_EINVAL on bad params. */
int sift3d_pattern(const sift3d_params* params, float* out);

/* Create a context.  Validates params (SIFT3D_EINVAL) and stores them; device
 * memory is allocated lazily by the first call that needs it.  *out receives
 * the context, or NULL on failure. */
int sift3d_create(const sift3d_params* params, sift3d_ctx** out);

/* Release a context and all device memory it owns.  NULL is ignored.  Waits
 * for the context's outstanding work. */
void sift3d_destroy(sift3d_ctx* ctx);

/* Message of the last failure on ctx ("" if none).  Owned by ctx. */
const char* sift3d_last_error(const sift3d_ctx* ctx);

/* Detect keypoints in one volume (Sec. 2.2.2: Gaussian pyramid, sub-sampling,
 * DoG, 4D sum-of-signs peaks; plus the contrast and curvature tests).
 *   dev_vol   device volume of nx*ny*nz voxels of `dtype`, x fastest.
 *   stream    cudaStream_t the work is ordered on.
 *   dev_out   device array of `capacity` keypoints, written in the canonical
 *             order (octave, scale, iz, iy, ix).
 *   n_out     host int; if non-NULL the call waits for the device and stores
 *             the number of keypoints detected (which may exceed capacity).  If
 *             NULL the call returns without waiting; the count is then
 *             available on the device through sift3d_device_count().
 * The pyramid stays on the device, owned by ctx, until the next detect on ctx;
 * sift3d_describe and sift3d_read_level read it.
 * Errors: SIFT3D_EINVAL (dims, dtype, capacity < 0), SIFT3D_ENOMEM,
 * SIFT3D_ECUDA, SIFT3D_ECAPACITY (only with n_out: more keypoints than
 * capacity; the first `capacity` in canonical order were written). */
int sift3d_detect(sift3d_ctx* ctx, const void* dev_vol, int dtype,
                  int nx, int ny, int nz, void* stream,
                  sift3d_keypoint* dev_out, int capacity, int* n_out);

/* Device pointer to the int that the last detect on ctx writes its keypoint
 * count to (stream ordered).  NULL before the first detect. */
const int* sift3d_device_count(const sift3d_ctx* ctx);

/* BRIEF / RRIEF descriptors of keypoints from the last detect on ctx
 * (Sec. 2.2.3).  For keypoint (octave o, scale s, ix, iy, iz) the level G_s of
 * octave o is blurred by desc_blur_sigma (clamp), and for each pair k the
 * values I(c + sigma_s*p1_k) and I(c + sigma_s*p2_k) are read by trilinear
 * interpolation with coordinates clamped to the octave grid (c = (ix,iy,iz),
 * sigma_s in octave voxels);  d_k = I(p1_k) - I(p2_k).
 *   BRIEF: bit k of dev_brief[i] is [d_k > 0].
 *   RRIEF: dev_rrief[i*64 + k] = #{j : d_j < d_k} + #{j < k : d_j == d_k}.
 *   n      number of keypoints in dev_kps; -1 = use the device-side count of
 *          the last detect (min(count, that detect's capacity)), no host wait.
 *   kind   SIFT3D_DESC_BRIEF / _RRIEF / _BOTH; the unused output may be NULL.
 * Errors: SIFT3D_EINVAL (no prior detect, bad kind, NULL output), SIFT3D_ECUDA. */
int sift3d_describe(sift3d_ctx* ctx, const sift3d_keypoint* dev_kps, int n, int kind,
                    uint64_t* dev_brief, uint8_t* dev_rrief, void* stream);

/* Separable 3D Gaussian blur of a dense float32 volume (Sec. 2.2.2 "Gaussian
 * Convolution": a y pass and an x pass per plane, then a z pass), with the
 * library's discrete kernel w_k ~ exp(-k^2/2 sigma^2), |k| <= ceil(trunc*sigma)
 * (trunc from the context's params), unit sum, clamp-to-edge borders.
 *   dev_in, dev_out  dense nx*ny*nz float32 device arrays (x fastest); they
 *                    must not overlap.
 *   sigma            > 0, with ceil(trunc*sigma) <= 16.
 * Scratch for the intermediate passes is device memory owned by ctx, allocated
 * on first use and grown when a larger volume arrives.
 * Errors: SIFT3D_EINVAL (arguments, sigma), SIFT3D_ENOMEM, SIFT3D_ECUDA. */
int sift3d_gaussian_blur(sift3d_ctx* ctx, const float* dev_in, int nx, int ny, int nz,
                         double sigma, float* dev_out, void* stream);

/* The same blur for callers that cannot allocate device memory: code that runs
 * where cudaMalloc is unavailable or not allowed (in an allocator's own reclaim
 * path, in a loop that must never enter the allocator) or that is handed only
 * its input and output buffers.  This call allocates nothing, needs no context,
 * and takes trunc explicitly (4.0 matches the default params).  It launches
 * kernels and, on its first call on a device, looks up a symbol address, so it
 * must not be called from a host function or callback running on a CUDA stream
 * (CUDA forbids CUDA calls there).  No counterpart in the paper.
 *   Scratch: one library-owned device array of 2 * SIFT3D_BLUR_NOALLOC_MAX_ELEMS
 *   floats (32 MiB) that every GPU loading the library holds until the process
 *   exits.  A volume fits when roundup(nx, 8) * ny * nz <= the maximum (a
 *   145x174x145 volume does); larger volumes return SIFT3D_ECAPACITY.
 *   The first call on a device looks up that device's address of the array
 *   (cudaGetSymbolAddress, with the device current); make that first call
 *   before any stream capture.
 *   All calls share the array: calls whose work overlaps on the GPU (different
 *   streams, or host threads without ordering) race and corrupt each other's
 *   results.  Serialise them, e.g. on one stream.
 * Errors: SIFT3D_EINVAL (arguments, sigma, trunc), SIFT3D_ECAPACITY (volume
 * larger than the scratch), SIFT3D_ECUDA. */
#define SIFT3D_BLUR_NOALLOC_MAX_ELEMS (1 << 22)
int sift3d_gaussian_blur_noalloc(const float* dev_in, int nx, int ny, int nz, double sigma,
                                 double trunc, float* dev_out, void* stream);

/* Detect (and, with dev_brief and dev_rrief, describe) n volumes of possibly
 * different sizes in one CUDA graph launch (no counterpart in the paper; the
 * batched form of sift3d_detect + sift3d_describe).  Every pyramid pass (the
 * y/x and z passes of a level, the peak test of an octave) is one persistent
 * launch over the tiles of all volumes of a wave, so small octaves of some
 * volumes run beside the large octaves of others; the canonical sort and the
 * descriptors run per volume.  Results equal sift3d_detect / sift3d_describe
 * on each volume alone, bit for bit.  Volumes are taken in waves whose
 * workspaces fit params.hbm_budget_bytes (0: 40 GiB); the batch's device
 * memory is held by ctx until a batch of another signature (dims, dtype,
 * capacity, describe or not) arrives or ctx is destroyed.
 *   dev_vols   host array of n device volume pointers (x fastest), dtype each.
 *   dims       host array of 3n ints: nx, ny, nz of each volume.
 *   dev_out    host array of n device arrays of capacity keypoints.
 *   dev_brief, dev_rrief  host arrays of n device arrays (capacity words /
 *              capacity x 64 bytes), or both NULL for detect only.
 *   n_out      host array of n: keypoints detected per volume (may exceed
 *              capacity; then that volume's array holds the first capacity in
 *              canonical order), or NULL to return without waiting.
 * Requirements: float32 storage, nx <= 256 and at least one octave for every
 * volume.  The descriptor pre-blur rides on the level passes where its radius
 * is 4 and every level's radius is at least 4 (the defaults), else it runs as
 * separate batched passes.  Errors: SIFT3D_EINVAL (arguments, requirements),
 * SIFT3D_ENOMEM, SIFT3D_ECAPACITY (some volume exceeded capacity; n_out
 * complete), SIFT3D_ETIMEDOUT, SIFT3D_ECUDA. */
int sift3d_detect_batch(sift3d_ctx* ctx, int n, const void* const* dev_vols, const int* dims, int dtype,
                        void* stream, sift3d_keypoint* const* dev_out, int capacity,
                        uint64_t* const* dev_brief, uint8_t* const* dev_rrief, int* n_out);

/* 3D SIFT-Rank descriptors of keypoints from the last detect on ctx: the
 * paper's comparison baseline (Sec. 1 and Sec. 3.5), of which the paper fixes
 * a dominant 3x3 orientation from peaks of a discrete spherical histogram of
 * gradient, 2x2x2 spatial x 8 orientation bins after reorientation, and rank
 * normalisation.  This library's reading of the rest: on the keypoint's
 * level G_s (not pre-blurred), gradients by central differences of trilinear
 * samples at the 8^3 cell centres of [-r, r]^3 inside the ball of radius
 * r = 3 sigma_s (280 samples, weight exp(-|u|^2 / (2 (r/2)^2))); e1 = the
 * weighted mean gradient of the peak bin of a histogram of w |g| over the 12
 * icosahedron directions, e2 the same for the gradients' parts perpendicular
 * to e1, e3 = e1 x e2; the samples are then taken at c + R u, and element
 * 8 * octant(u) + octant(R^T g) (octant = (x >= 0) + 2 (y >= 0) + 4 (z >= 0))
 * accumulates w |g|; the output is the rank of each of the 64 values,
 * ascending, ties by lower index.
 *   n         number of keypoints in dev_kps; -1 = the device-side count of
 *             the last detect (no host wait).
 *   dev_desc  n x 64 uint8 ranks (device, caller owned).
 *   dev_rot   n x 9 floats, R row-major with columns e1, e2, e3, or NULL.
 * Errors: SIFT3D_EINVAL (no prior detect, NULL outputs), SIFT3D_ECUDA. */
int sift3d_describe_siftrank(sift3d_ctx* ctx, const sift3d_keypoint* dev_kps, int n, uint8_t* dev_desc,
                             float* dev_rot, void* stream);

/* Nearest-neighbour matching of descriptors (Sec. 2.1 (e): descriptors are
 * matched by nearest neighbour).  For each descriptor i of set A the call
 * finds, by brute force over set B:
 *   dev_nn[i]     index of the nearest descriptor in B (the lowest index among
 *                 equal distances), -1 if nb == 0;
 *   dev_dist[i]   its distance, INT32_MAX if nb == 0;
 *   dev_dist2[i]  the smallest distance to any other descriptor of B (the
 *                 second nearest, for a ratio test), INT32_MAX if nb < 2; may be
 *                 NULL.
 * kind SIFT3D_DESC_BRIEF: A and B are uint64 words as sift3d_describe writes
 *   them (8-byte aligned); the distance is the Hamming distance, 0..64.
 * kind SIFT3D_DESC_RRIEF: A and B are rows of 64 uint8 ranks (16-byte aligned,
 *   row i at byte 64 i); the distance is sum_k (a_k - b_k)^2, exact.
 * All pointers are device memory owned by the caller; the call allocates
 * nothing and is ordered on `stream`.  na == 0 launches nothing.
 * Errors: SIFT3D_EINVAL (kind, negative counts, NULL or misaligned pointers),
 * SIFT3D_ECUDA. */
int sift3d_match(const void* dev_a, int na, const void* dev_b, int nb, int kind, int32_t* dev_nn,
                 int32_t* dev_dist, int32_t* dev_dist2, void* stream);

/* Copy one pyramid level of the last detect into a dense float32 device array
 * dev_dst of dims[octave] voxels (x fastest).  kind = SIFT3D_LEVEL_*.
 * Errors: SIFT3D_EINVAL (no prior detect, index out of range), SIFT3D_ECUDA. */
int sift3d_read_level(sift3d_ctx* ctx, int octave, int kind, int index,
                      float* dev_dst, void* stream);

/* Per-kernel device times of the last detect on ctx, when the context was
 * created with params.profile = 1 (CUDA events recorded around every kernel of
 * the detect, inside the graph when graphs are used).  Waits for that detect.
 *   max      capacity of ms_out / names_out.
 *   ms_out   host array, kernel i's elapsed milliseconds.
 *   names_out host array of pointers to library-owned labels such as
 *            "o0.s5.conv_z_dog" (octave 0, level 5); may be NULL.
 *   algo_bytes_out host array, each kernel's algorithmic bytes (minimum reads
 *            and writes of its inputs and outputs); may be NULL.
 *   n_out    receives the number of kernels (may exceed max).
 * Errors: SIFT3D_EINVAL (no prior detect or profiling off), SIFT3D_ECUDA. */
int sift3d_stage_times(sift3d_ctx* ctx, int max, float* ms_out, const char** names_out,
                       uint64_t* algo_bytes_out, int* n_out);

/* Timeline of the last profiled detect (no counterpart in the paper): for each
 * kernel, in the order of sift3d_stage_times, the times in ms of its begin and
 * end events relative to the begin event of the first kernel (the root of the
 * detect graph).  Kernels on concurrent octave branches overlap in time.
 *   begin_ms_out, end_ms_out  host arrays of max floats (caller owned).
 *   n_out    receives the number of kernels (may exceed max).
 * Errors: SIFT3D_EINVAL (no prior detect or profiling off), SIFT3D_ECUDA. */
int sift3d_stage_timeline(sift3d_ctx* ctx, int max, float* begin_ms_out, float* end_ms_out, int* n_out);

/* Serving (no counterpart in the paper).  sift3d_submit queues a volume: by
 * default a HOST volume, which the library copies before returning (with
 * SIFT3D_SUBMIT_NOCOPY it reads the caller's buffer later, by DMA); with
 * SIFT3D_SUBMIT_DEVICE a device volume that the detect reads in place.  The
 * library admits requests to the device while their device memory fits in
 * hbm_budget_bytes and fewer than max_inflight are on the device, runs detect
 * then BRIEF+RRIEF describe for each on its own stream, and a device kernel
 * writes the count and exactly that many keypoint records and descriptors into
 * mapped pinned host memory (no round trip to size the copy).  Requests that
 * overlap in time overlap on the device.
 *   host_or_dev_vol  x-fastest nx*ny*nz volume of dtype (see flags).
 *   ticket  receives an id for sift3d_poll / sift3d_release.
 * Errors: SIFT3D_EINVAL (also: SIFT3D_SUBMIT_DEVICE with a pointer that is not
 * device memory of the context's GPU), SIFT3D_EBUDGET (the volume alone exceeds
 * the budget), SIFT3D_ENOMEM.  Failures while a request runs (allocation,
 * CUDA) are reported by sift3d_poll for that ticket; later requests are
 * served normally. */
int sift3d_submit(sift3d_ctx* ctx, const void* host_or_dev_vol, int dtype,
                  int nx, int ny, int nz, int flags, uint64_t* ticket);

/* Wait up to timeout_us microseconds (0 = do not wait) for a request.  Returns
 * SIFT3D_OK with *out filled, SIFT3D_PENDING if still running, or an error
 * (SIFT3D_ENOTFOUND for an unknown or released ticket, SIFT3D_ECUDA if its
 * device work failed).  A result's ECAPACITY is reported in out->status. */
int sift3d_poll(sift3d_ctx* ctx, uint64_t ticket, int timeout_us, sift3d_result* out);

/* Free the host result of a finished request.  SIFT3D_ENOTFOUND if unknown,
 * SIFT3D_PENDING if it has not finished (nothing is freed). */
int sift3d_release(sift3d_ctx* ctx, uint64_t ticket);

/* Testing the allocation-failure paths without exhausting memory (no
 * counterpart in the paper): after this call, the n-th device or pinned host
 * allocation the library makes (counted from 1, process wide) fails as if out
 * of memory, once; n = 0 cancels a pending failure.  The call that needed the
 * allocation returns SIFT3D_ENOMEM (a served request reports it through
 * sift3d_poll) and releases whatever it had allocated; the context stays
 * usable.  Returns SIFT3D_OK, or SIFT3D_EINVAL for n < 0. */
int sift3d_test_fail_allocation(int n);

#ifdef __cplusplus
}
#endif

#endif /* SIFT3D_H */
