// Batched detect (+ describe) of many volumes of uneven sizes under one CUDA
// graph.  Every pass of the pyramid (the y/x and z passes of level s of octave
// o, and the peak detection of an octave) is one launch for all volumes of a
// wave: a persistent grid whose CTAs walk one flat list of the volumes' tiles
// (per-volume arguments in a device table, a tile's volume found by prefix
// sums), with the same per-output arithmetic as the single-volume kernels, so
// every level, keypoint and descriptor equals the single-volume path bit for
// bit.  The canonical-order sort and the descriptors run per volume.  Volumes
// are processed in waves whose workspaces fit the context's HBM budget; waves
// reuse the same device slots one after the other.
#include <algorithm>
#include <array>
#include <cstring>

#include "batch.hpp"

namespace sift3d {

namespace {

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

XYVol xy_vol(const ConvXYArgs& a) {
    XYVol q{};
    q.src = a.src;
    q.src_py = a.src_py;
    q.src_pz = a.src_pz;
    q.dst = a.dst;
    q.py = a.py;
    q.pz = a.pz;
    q.base_out = a.base_out;
    q.res_out = a.res_out;
    q.zero_count = a.zero_count;
    q.dst2 = a.dst2;
    q.src_scale = a.src_scale;
    q.nx = a.nx;
    q.ny = a.ny;
    q.nz = a.nz;
    q.row_tile = a.row_tile;
    return q;
}

ZVol z_vol(const ConvZArgs& a) {
    ZVol q{};
    q.src = a.src;
    q.dst = a.dst;
    q.prev = a.prev;
    q.dog = a.dog;
    q.res = a.res;
    q.src2 = a.src2;
    q.dst2 = a.dst2;
    q.py = a.py;
    q.pz = a.pz;
    q.nx = a.nx;
    q.ny = a.ny;
    q.nz = a.nz;
    return q;
}

int fail(std::string* err, int code, const std::string& msg) {
    if (err) *err = msg;
    return code;
}

}  // namespace

BatchExec::~BatchExec() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (arena) cudaFree(arena);
    if (tables) cudaFree(tables);
}

bool BatchExec::matches(const std::vector<std::array<int, 3>>& d, int dt, int cap, bool desc) const {
    return d == dims && dt == dtype && cap == capacity && desc == describe;
}

int build_batch(const sift3d_params& p, const std::vector<std::array<int, 3>>& dims, int dtype, int capacity,
                bool describe, const float* pattern, BatchExec* bx, std::string* err) {
    const int n = (int)dims.size();
    bx->dims = dims;
    bx->dtype = dtype;
    bx->capacity = capacity;
    bx->describe = describe;
    bx->fuse_blur = true;
    if (p.storage != SIFT3D_STORAGE_F32) return fail(err, SIFT3D_EINVAL, "batched detect needs float32 storage");
    // plans, and the largest workspace (every slot gets that size)
    std::vector<Plan> plans(n);
    size_t slot_bytes = 0;
    for (int v = 0; v < n; ++v) {
        int rc = make_plan(p, dims[v][0], dims[v][1], dims[v][2], dtype, &plans[v], err);
        if (rc != SIFT3D_OK) return rc;
        const Plan& pl = plans[v];
        if (pl.nO == 0) return fail(err, SIFT3D_EINVAL, "every batched volume needs at least one octave");
        if (pl.oct[0].nx > 256) return fail(err, SIFT3D_EINVAL, "batched detect needs nx <= 256");
        // the descriptor pre-blur rides on the level passes when every level can
        // carry it (0.333 ms per volume against 0.347 with separate passes, 256
        // volumes 96..256 per axis), else it runs as separate batched passes
        for (int o = 0; o < pl.nO; ++o)
            for (int s = 2; s <= pl.S + 1; ++s)
                if (pl.r_desc > 0 && !(pl.r_desc == kFusedBlurRadius && pl.r_inc[s - 1] >= kFusedBlurRadius))
                    bx->fuse_blur = false;
        slot_bytes = std::max(slot_bytes, round_up(workspace_bytes(pl, capacity), 256));
    }
    const uint64_t budget = p.hbm_budget_bytes ? p.hbm_budget_bytes : (40ull << 30);
    bx->slots = (int)std::max<uint64_t>(1, std::min<uint64_t>(std::min(n, kBatchVols),
                                                                budget / std::max<size_t>(slot_bytes, 1)));
    int rc = alloc_device_zeroed(slot_bytes * (size_t)bx->slots, &bx->arena, err);
    if (rc != SIFT3D_OK) return rc;

    // ---- nodes, wave by wave; every batched node records its table's bytes
    std::vector<unsigned char> host_tables;
    struct PendingTable {
        int node;
        size_t offset;     // byte offset of the args in the table buffer
        size_t prefix;     // byte offset of the prefix array
        int nvol, total;
    };
    std::vector<PendingTable> pend;
    auto put = [&](const void* src, size_t bytes, size_t align) {
        const size_t off = round_up(host_tables.size(), align);
        host_tables.resize(off + bytes);
        memcpy(host_tables.data() + off, src, bytes);
        return off;
    };
    std::vector<Node>& nodes = bx->nodes;
    nodes.clear();
    auto add = [&](const LaunchSpec& s, std::vector<int> deps, const char* label) {
        Node nd;
        nd.spec = s;
        nd.deps = std::move(deps);
        nd.label = label;
        nodes.push_back(std::move(nd));
        return (int)nodes.size() - 1;
    };
    bx->vols.assign(n, BatchVolume{});
    std::vector<int> wave_end;   // nodes every node of the next wave waits for
    for (int w0 = 0; w0 < n; w0 += bx->slots) {
        const int w1 = std::min(n, w0 + bx->slots);
        for (int v = w0; v < w1; ++v) {
            BatchVolume& bv = bx->vols[v];
            rc = bind_workspace(plans[v], capacity, bx->arena + (size_t)(v - w0) * slot_bytes, &bv.ws, err);
            if (rc != SIFT3D_OK) return rc;
        }
        int maxO = 0, S = plans[w0].S, L = plans[w0].L;
        for (int v = w0; v < w1; ++v) maxO = std::max(maxO, plans[v].nO);
        int g_node[SIFT3D_MAX_OCTAVES][kMaxLevels];
        std::vector<int> peak_nodes, blur_nodes;
        for (int o = 0; o < maxO; ++o) {
            std::vector<int> in_o;
            for (int v = w0; v < w1; ++v)
                if (plans[v].nO > o) in_o.push_back(v);
            for (int s = (o == 0 ? 0 : 1); s < L; ++s) {
                std::vector<ConvXYArgs> xys;
                std::vector<ConvZArgs> zs;
                std::vector<int> pxy{0}, pz{0};
                LevelArgs first{};
                int nx_max = 0;
                for (size_t i = 0; i < in_o.size(); ++i) {
                    const int v = in_o[i];
                    LevelArgs la = level_args(bx->vols[v].ws, o, s, nullptr, dtype, bx->fuse_blur, false);
                    la.xy.row_tile = 16;
                    if (i == 0) first = la;
                    if (la.radius != first.radius || la.src_kind != first.src_kind || la.sub != first.sub ||
                        la.fused_blur != first.fused_blur)
                        return fail(err, SIFT3D_EINVAL, "batched volumes need the same level passes");
                    nx_max = std::max(nx_max, la.xy.nx);
                    xys.push_back(la.xy);
                    zs.push_back(la.z);
                    pxy.push_back(pxy.back() + conv_xy_items(la.xy));
                    pz.push_back(pz.back() + conv_z_items(la.z));
                }
                std::vector<int> deps = (o == 0 && s == 0) ? wave_end
                                                           : std::vector<int>{(s == 1 && o > 0) ? g_node[o - 1][S]
                                                                                                : g_node[o][s - 1]};
                const LaunchSpec xs = conv_xy_batch_spec(first.radius, first.src_kind, first.sub, first.fused_blur,
                                                         nx_max, 16, pxy.back());
                if (xs.func == nullptr) return fail(err, SIFT3D_EINVAL, "no batched y/x kernel for this level");
                const int nxy = add(xs, deps, "batch.conv_xy");
                BatchXY bcx{};
                bcx.n = (int)xys.size();
                bcx.total = pxy.back();
                for (size_t i = 0; i < pxy.size(); ++i) bcx.prefix[i] = pxy[i];
                bcx.taps = first.xy.taps;
                bcx.taps2 = first.xy.taps2;
                for (size_t i = 0; i < xys.size(); ++i) bcx.vol[i] = xy_vol(xys[i]);
                nodes[nxy].set_args(bcx);
                if (o == 0 && s == 0) bx->input_nodes.push_back({nxy, w0, (int)xys.size()});
                const LaunchSpec zsp = conv_z_batch_spec(first.radius, first.fused_blur, pz.back());
                if (zsp.func == nullptr) return fail(err, SIFT3D_EINVAL, "no batched z kernel for this level");
                const int nz = add(zsp, {nxy}, "batch.conv_z");
                BatchZ bcz{};
                bcz.n = (int)zs.size();
                bcz.total = pz.back();
                for (size_t i = 0; i < pz.size(); ++i) bcz.prefix[i] = pz[i];
                bcz.taps = first.z.taps;
                bcz.taps2 = first.z.taps2;
                for (size_t i = 0; i < zs.size(); ++i) bcz.vol[i] = z_vol(zs[i]);
                nodes[nz].set_args(bcz);
                g_node[o][s] = nz;
            }
            if (o > 0) g_node[o][0] = g_node[o][1];
            // peaks: one launch per octave over all scales
            {
                std::vector<PeakTmaArgs> pks;
                std::vector<int> pp{0};
                for (int v : in_o) {
                    const Plan& pl = plans[v];
                    const OctaveGeom& g = pl.oct[o];
                    if (g.nx - 2 * pl.p.border < 1 || g.ny - 2 * pl.p.border < 1 || g.nz - 2 * pl.p.border < 1)
                        continue;
                    PeakTmaArgs pa;
                    if (!make_peak_tma_args(bx->vols[v].ws, o, 1, S, &pa))
                        return fail(err, SIFT3D_ECUDA, "DoG tensor map");
                    peak_fill_tiles(&pa);
                    pks.push_back(pa);
                    pp.push_back(pp.back() + pa.gx * pa.gy * pa.gz);
                }
                if (!pks.empty()) {
                    const LaunchSpec ps = peak_batch_spec(S, pp.back());
                    if (ps.func == nullptr) return fail(err, SIFT3D_EINVAL, "no batched peak kernel");
                    const int np = add(ps, {g_node[o][S + 2]}, "batch.peak");
                    pend.push_back({np, put(pks.data(), pks.size() * sizeof(PeakTmaArgs), 128),
                                    put(pp.data(), pp.size() * sizeof(int), 16), (int)pks.size(), pp.back()});
                    peak_nodes.push_back(np);
                }
            }
            // descriptor pre-blur of G_1..G_S (Sec. 2.2.3): a y/x and a z pass per
            // level over the wave, beside the octave chain
            if (describe && plans[w0].r_desc > 0 && !bx->fuse_blur) {
                for (int s = 1; s <= S; ++s) {
                    BatchXY bcx{};
                    BatchZ bcz{};
                    int nx_max = 0;
                    bcx.prefix[0] = bcz.prefix[0] = 0;
                    for (size_t i = 0; i < in_o.size(); ++i) {
                        const Workspace& ws = bx->vols[in_o[i]].ws;
                        const OctaveGeom& g = ws.plan.oct[o];
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
                        xa.row_tile = 16;
                        ConvZArgs za{};
                        za.src = ws.TB(o, s);
                        za.dst = ws.B(o, s);
                        za.py = g.py;
                        za.pz = g.pz;
                        za.nx = g.nx;
                        za.ny = g.ny;
                        za.nz = g.nz;
                        nx_max = std::max(nx_max, g.nx);
                        bcx.vol[i] = xy_vol(xa);
                        bcz.vol[i] = z_vol(za);
                        bcx.prefix[i + 1] = bcx.prefix[i] + conv_xy_items(xa);
                        bcz.prefix[i + 1] = bcz.prefix[i] + conv_z_items(za);
                    }
                    const int nv = (int)in_o.size();
                    bcx.n = bcz.n = nv;
                    bcx.total = bcx.prefix[nv];
                    bcz.total = bcz.prefix[nv];
                    bcx.taps = bcz.taps = plans[w0].t_desc;
                    const LaunchSpec xs = conv_xy_batch_spec(plans[w0].r_desc, 2, false, false, nx_max, 16, bcx.total);
                    const LaunchSpec zsp = conv_z_batch_spec(plans[w0].r_desc, false, bcz.total);
                    if (xs.func == nullptr || zsp.func == nullptr)
                        return fail(err, SIFT3D_EINVAL, "no batched kernel for the descriptor pre-blur");
                    const int nxy = add(xs, {g_node[o][s]}, "batch.blur_xy");
                    nodes[nxy].set_args(bcx);
                    const int nz = add(zsp, {nxy}, "batch.blur_z");
                    nodes[nz].set_args(bcz);
                    blur_nodes.push_back(nz);
                }
            }
        }
        // per volume: canonical order, then the descriptors
        std::vector<int> ends;
        for (int v = w0; v < w1; ++v) {
            BatchVolume& bv = bx->vols[v];
            if (plans[v].nO == 0) continue;
            SortArgs sa{};
            sa.staging = bv.ws.staging;
            sa.err = bv.ws.count + 3;
            sa.out = nullptr;   // the caller's array, set per call
            sa.count = bv.ws.count;
            sa.count_out = bv.ws.count_out;
            sa.count_copy = nullptr;   // the batch's count array, set below
            sa.capacity = capacity;
            std::vector<int> sdeps = peak_nodes;
            sdeps.push_back(g_node[0][L - 1]);
            bv.sort_node = add(sort_spec(sa), sdeps, "batch.sort");
            nodes[bv.sort_node].set_args(sa);
            ends.push_back(bv.sort_node);
            if (describe) {
                DescribeArgs da = make_describe_args(bv.ws, pattern);
                da.n = -1;
                da.n_dev = bv.ws.count_out;
                da.n_cap = capacity;
                std::vector<int> ddeps = blur_nodes;
                ddeps.push_back(bv.sort_node);
                bv.describe_node = add(describe_spec(p.storage, da, capacity), ddeps, "batch.describe");
                nodes[bv.describe_node].set_args(da);
                ends.back() = bv.describe_node;
            }
        }
        wave_end = ends;
    }
    // the per-volume totals at the end of the table buffer (the workspaces'
    // counters are overwritten by the next wave)
    const size_t counts_off = round_up(host_tables.size(), 256);
    host_tables.resize(counts_off + (size_t)n * sizeof(int), 0);
    // one device buffer for every table; patch the table pointers into the nodes
    bx->table_bytes = round_up(std::max<size_t>(host_tables.size(), 256), 256);
    if (dev_alloc(&bx->tables, bx->table_bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        bx->tables = nullptr;
        return fail(err, SIFT3D_ENOMEM, "batch tables");
    }
    if (cudaMemcpy(bx->tables, host_tables.data(), host_tables.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(err, SIFT3D_ECUDA, "batch tables copy");
    bx->host_tables = std::move(host_tables);
    bx->counts = reinterpret_cast<int*>(static_cast<char*>(bx->tables) + counts_off);
    for (int v = 0; v < n; ++v) {
        const int sn = bx->vols[v].sort_node;
        if (sn < 0) continue;
        SortArgs sa;
        memcpy(&sa, nodes[sn].arg.data(), sizeof(sa));
        sa.count_copy = bx->counts + v;
        nodes[sn].set_args(sa);
    }
    for (const PendingTable& t : pend) {
        Node& nd = nodes[t.node];
        BatchTable bt{static_cast<char*>(bx->tables) + t.offset,
                      reinterpret_cast<const int*>(static_cast<char*>(bx->tables) + t.prefix), t.nvol, t.total};
        nd.set_args(bt);   // only the peak nodes use device tables
    }
    return SIFT3D_OK;
}

int run_batch(BatchExec& bx, const void* const* inputs, sift3d_keypoint* const* outs, uint64_t* const* briefs,
              uint8_t* const* rriefs, cudaStream_t st, std::string* err) {
    const int n = (int)bx.dims.size();
    // inputs: the first pass's table entries of the first wave's volumes, and a
    // table per later wave; rewrite every entry whose pointer changed
    bool tables_dirty = false;
    for (int v = 0; v < n; ++v) {
        BatchVolume& bv = bx.vols[v];
        if (bv.input != inputs[v]) {
            bv.input = inputs[v];
            tables_dirty = true;
        }
    }
    // inputs: the first y/x node of each wave carries its volumes' pointers
    std::vector<int> changed;
    if (tables_dirty)
        for (const BatchExec::InputNode& r : bx.input_nodes) {
            Node& nd = bx.nodes[r.node];
            BatchXY bxy;
            memcpy(&bxy, nd.arg.data(), sizeof(bxy));
            for (int i = 0; i < r.count; ++i) bxy.vol[i].src = bx.vols[r.first + i].input;
            nd.set_args(bxy);
            changed.push_back(r.node);
        }
    // outputs: sort and describe node parameters
    for (int v = 0; v < n; ++v) {
        BatchVolume& bv = bx.vols[v];
        if (bv.sort_node < 0) continue;
        if (bv.out != outs[v]) {
            bv.out = outs[v];
            SortArgs sa;
            memcpy(&sa, bx.nodes[bv.sort_node].arg.data(), sizeof(sa));
            sa.out = outs[v];
            bx.nodes[bv.sort_node].set_args(sa);
            changed.push_back(bv.sort_node);
        }
        if (bv.describe_node >= 0 && (bv.brief != briefs[v] || bv.rrief != rriefs[v] || bv.kps != outs[v])) {
            bv.brief = briefs[v];
            bv.rrief = rriefs[v];
            bv.kps = outs[v];
            DescribeArgs da;
            memcpy(&da, bx.nodes[bv.describe_node].arg.data(), sizeof(da));
            da.kps = outs[v];
            da.brief = briefs[v];
            da.rrief = rriefs[v];
            bx.nodes[bv.describe_node].set_args(da);
            changed.push_back(bv.describe_node);
        }
    }
    cudaError_t e = cudaSuccess;
    if (!bx.exec) {
        e = cudaGraphCreate(&bx.graph, 0);
        if (e != cudaSuccess) return fail(err, SIFT3D_ECUDA, std::string("cudaGraphCreate: ") + cudaGetErrorString(e));
        bx.gnodes.resize(bx.nodes.size());
        for (size_t i = 0; i < bx.nodes.size(); ++i) {
            Node& nd = bx.nodes[i];
            std::vector<cudaGraphNode_t> deps;
            for (int d : nd.deps) deps.push_back(bx.gnodes[d]);
            cudaKernelNodeParams kp{};
            kp.func = const_cast<void*>(nd.spec.func);
            kp.gridDim = nd.spec.grid;
            kp.blockDim = nd.spec.block;
            kp.sharedMemBytes = (unsigned)nd.spec.smem;
            kp.kernelParams = &nd.argp;
            e = cudaGraphAddKernelNode(&bx.gnodes[i], bx.graph, deps.data(), deps.size(), &kp);
            if (e != cudaSuccess)
                return fail(err, SIFT3D_ECUDA, std::string("cudaGraphAddKernelNode: ") + cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&bx.exec, bx.graph, 0);
        if (e != cudaSuccess)
            return fail(err, SIFT3D_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    } else {
        for (int i : changed) {
            Node& nd = bx.nodes[i];
            cudaKernelNodeParams kp{};
            kp.func = const_cast<void*>(nd.spec.func);
            kp.gridDim = nd.spec.grid;
            kp.blockDim = nd.spec.block;
            kp.sharedMemBytes = (unsigned)nd.spec.smem;
            kp.kernelParams = &nd.argp;
            e = cudaGraphExecKernelNodeSetParams(bx.exec, bx.gnodes[i], &kp);
            if (e != cudaSuccess)
                return fail(err, SIFT3D_ECUDA, std::string("cudaGraphExecKernelNodeSetParams: ") + cudaGetErrorString(e));
        }
    }
    e = cudaGraphLaunch(bx.exec, st);
    if (e != cudaSuccess) return fail(err, SIFT3D_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    return SIFT3D_OK;
}

}  // namespace sift3d
