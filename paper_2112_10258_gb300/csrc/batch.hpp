// Batched detect of many volumes under one CUDA graph (see batch.cpp).
#pragma once

#include <array>
#include <string>
#include <vector>

#include "runtime.hpp"

namespace sift3d {

struct BatchVolume {
    Workspace ws;                       // bound into the batch arena (its wave's slot)
    const void* input = nullptr;        // the caller's pointers of the last run
    sift3d_keypoint* out = nullptr;
    sift3d_keypoint* kps = nullptr;
    uint64_t* brief = nullptr;
    uint8_t* rrief = nullptr;
    int sort_node = -1, describe_node = -1;
};

struct BatchExec {
    std::vector<std::array<int, 3>> dims;
    int dtype = 0, capacity = 0;
    bool describe = false;
    bool fuse_blur = true;             // descriptor pre-blur carried by the level passes
    int slots = 0;                      // volumes per wave
    char* arena = nullptr;              // slots x the largest workspace
    void* tables = nullptr;             // device copy of host_tables
    int* counts = nullptr;              // per-volume totals (inside tables)
    size_t table_bytes = 0;
    std::vector<unsigned char> host_tables;
    struct InputNode {                  // the input pass of one wave: its node and volumes
        int node;
        int first, count;
    };
    std::vector<InputNode> input_nodes;
    std::vector<BatchVolume> vols;
    std::vector<Node> nodes;
    std::vector<cudaGraphNode_t> gnodes;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool matches(const std::vector<std::array<int, 3>>& d, int dt, int cap, bool desc) const;
    ~BatchExec();
};

// Plans, workspaces, tables and nodes of a batch (float32 storage, rows of at
// most 256 voxels, the descriptor pre-blur fused into the level passes).
int build_batch(const sift3d_params& p, const std::vector<std::array<int, 3>>& dims, int dtype, int capacity,
                bool describe, const float* pattern, BatchExec* bx, std::string* err);
// Point the batch at this call's buffers and launch its graph on st.
int run_batch(BatchExec& bx, const void* const* inputs, sift3d_keypoint* const* outs, uint64_t* const* briefs,
              uint8_t* const* rriefs, cudaStream_t st, std::string* err);

}  // namespace sift3d
