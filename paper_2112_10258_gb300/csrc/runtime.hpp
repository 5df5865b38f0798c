// Host runtime of the sift3d library: plans, device workspaces, the launch DAG
// of one detect, and its execution as direct launches or as a CUDA graph.
#pragma once

#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace sift3d {

struct OctaveGeom {
    int nx = 0, ny = 0, nz = 0;
    int64_t py = 0, pz = 0;          // pitches in elements (py multiple of 8)
    int64_t voxels() const { return (int64_t)nx * ny * nz; }
};

struct Plan {
    sift3d_params p{};
    int nx = 0, ny = 0, nz = 0;
    int S = 0, L = 0, nD = 0;        // scales, Gaussian levels (S+3), DoGs (S+2)
    int nO = 0;
    OctaveGeom oct[SIFT3D_MAX_OCTAVES];
    double sig_level[kMaxLevels] = {};
    double sig_init = 0, sig_inc[kMaxLevels] = {}, sig_desc = 0;
    int r_init = 0, r_inc[kMaxLevels] = {}, r_desc = 0;
    Taps t_init{}, t_inc[kMaxLevels]{}, t_desc{};
    size_t elem = 4;                 // bytes per stored Gaussian / pre-blurred value
    static constexpr size_t elem_d = 4;   // bytes per stored DoG value (float32 for every storage type)
    // byte offsets into one workspace allocation
    size_t off_G[SIFT3D_MAX_OCTAVES][kMaxLevels] = {};
    size_t off_D[SIFT3D_MAX_OCTAVES][kMaxDogs] = {};
    size_t off_B[SIFT3D_MAX_OCTAVES][SIFT3D_MAX_SCALES] = {};
    size_t off_T[SIFT3D_MAX_OCTAVES] = {};
    size_t off_R[SIFT3D_MAX_OCTAVES] = {};   // 16-bit storage: rounding residuals (__half), one level
    size_t off_TB[SIFT3D_MAX_OCTAVES][SIFT3D_MAX_SCALES] = {};
    size_t bytes = 0;
    uint64_t algo_bytes = 0;
};

// Validate params (without dims when nx <= 0) and build the plan.
int validate_params(const sift3d_params& p, std::string* err);
int make_plan(const sift3d_params& p, int nx, int ny, int nz, int in_dtype, Plan* out, std::string* err);
void fill_plan_info(const Plan& pl, sift3d_plan_info* info);
void make_pattern(const sift3d_params& p, float* out);   // 64*6 floats

// Device memory for one volume size: the whole pyramid plus detect scratch.
struct Workspace {
    Plan plan;
    char* base = nullptr;
    size_t bytes = 0;
    bool owns_base = false;               // false: base lives in a context arena
    sift3d_keypoint* staging = nullptr;   // unsorted records
    int* count = nullptr;                 // kDetectCounters ints (see common.cuh)
    int* count_out = nullptr;             // total written by the sort
    int capacity = 0;
    int* test_flag = nullptr;             // device flag of the timeout test (null: off)
    void* G(int o, int s) const { return base + plan.off_G[o][s]; }
    void* D(int o, int s) const { return base + plan.off_D[o][s]; }
    void* B(int o, int s) const {  // s = 1..S
        return plan.r_desc > 0 ? (void*)(base + plan.off_B[o][s - 1]) : G(o, s);
    }
    float* T(int o) const { return reinterpret_cast<float*>(base + plan.off_T[o]); }
    __half* Res(int o) const {   // null for float32 storage
        return plan.elem == 2 ? reinterpret_cast<__half*>(base + plan.off_R[o]) : nullptr;
    }
    float* TB(int o, int s) const { return reinterpret_cast<float*>(base + plan.off_TB[o][s - 1]); }
};

// Every device and pinned host allocation of the library goes through these,
// so that a test can make the n-th one fail (sift3d_test_fail_allocation).
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t pinned_alloc(void** p, size_t bytes, unsigned flags);
void set_allocation_failure(int n);

size_t workspace_bytes(const Plan& plan, int capacity);
int bind_workspace(const Plan& plan, int capacity, char* base, Workspace* ws, std::string* err);
int alloc_device_zeroed(size_t bytes, char** out, std::string* err);
int alloc_workspace(const Plan& plan, int capacity, Workspace* ws, std::string* err);
PeakArgs make_peak_args(const Workspace& ws, int o);
// Peak kernel arguments with the DoG tensor map of octave o for a launch that
// tests scales first_scale .. first_scale+ns-1; false if it cannot be encoded.
bool make_peak_tma_args(const Workspace& ws, int o, int first_scale, int ns, PeakTmaArgs* out);
void free_workspace(Workspace* ws);

// One kernel launch of the detect DAG with its argument bytes and dependencies.
struct Node {
    LaunchSpec spec;
    std::vector<unsigned long long> arg;   // 8-byte aligned copy of the arg struct
    void* argp = nullptr;
    std::vector<int> deps;
    std::string label;                     // e.g. "o0.s5.conv_z_dog"
    uint64_t algo_bytes = 0;               // minimum bytes the kernel must move
    int octave = -1;                       // octave of a pyramid / peak node (-1: sort)
    struct XYKey {                         // a y/x pass node: what conv_xy_spec needs again
        int radius = 0, src_kind = 0;
        bool sub = false, valid = false;
    } xy;
    struct ZKey {                          // a z pass node whose depth may be tuned
        int radius = 0;
        bool valid = false;
    } zk;
    template <class A>
    void set_args(const A& a) {
        arg.assign((sizeof(A) + 7) / 8, 0ull);
        memcpy(arg.data(), &a, sizeof(A));
        argp = arg.data();
    }
};

struct DetectCall {
    const void* input;
    int dtype;
    sift3d_keypoint* out;
    int capacity;
};

// Arguments of level s of octave o (y/x pass then z pass with the DoG
// epilogue): the sources, destinations and taps.  fuse_blur: the level passes
// also produce the descriptor pre-blur of G_{s-1} where a fused variant exists
// (the batched path); the single-volume detect runs the pre-blur as separate
// passes on their own graph branches, off the octave chain.
struct LevelArgs {
    ConvXYArgs xy;
    ConvZArgs z;
    int radius = 0, src_kind = 2;   // src_kind: 0 float32 input, 1 uint8 input, 2 a pyramid level
    bool sub = false, fused_blur = false;
};
// z_sub: the level-S z pass also writes the next octave's G_0 where it can
// (the single-volume detect), and the next octave's first y/x pass reads it.
LevelArgs level_args(const Workspace& ws, int o, int s, const void* input, int dtype, bool fuse_blur,
                     bool z_sub);

// Build the detect DAG (topologically ordered).  first_node / sort_node index
// the two nodes that carry caller pointers.
std::vector<Node> build_detect(const Workspace& ws, const DetectCall& c, int* first_node, int* sort_node);

// A detect for one (shape, dtype, capacity), replayable as a CUDA graph.
struct DetectExec {
    std::vector<Node> nodes;
    int first = -1, sort = -1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> gnodes;
    const void* cur_input = nullptr;
    sift3d_keypoint* cur_out = nullptr;
    bool profile = false;
    std::vector<cudaEvent_t> ev_begin, ev_end;   // per node, when profiling
    ~DetectExec();
};

int run_detect(Workspace& ws, DetectExec& ex, const DetectCall& c, bool use_graph, bool profile,
               cudaStream_t st, std::string* err);

DescribeArgs make_describe_args(const Workspace& ws, const float* pattern);

// Sampled Gaussian taps (unit sum) and their radius ceil(trunc * sigma).
int gaussian_radius(double sigma, double trunc);
Taps gaussian_taps(double sigma, int radius);

// Pitch of the intermediate volumes of a standalone blur of an nx*ny*nz volume.
int64_t blur_pitch_elems(int nx, int ny, int nz);
// Enqueue a standalone separable blur: dense float32 in -> dense float32 out,
// through two pitched float32 scratch volumes t and u of blur_pitch_elems each.
int enqueue_blur(const float* in, int nx, int ny, int nz, double sigma, double trunc, float* t, float* u,
                 float* out, cudaStream_t st, std::string* err);

}  // namespace sift3d
