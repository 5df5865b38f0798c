// extern "C" entry points of include/sift3d.h and the serving scheduler.
#include <chrono>
#include <atomic>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "batch.hpp"

using namespace sift3d;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// A workspace for one (shape, dtype, capacity) with its replayable detect.
struct DetectEntry {
    Workspace ws;
    std::unique_ptr<DetectExec> ex[2];   // per input dtype
    ~DetectEntry() {
        ex[0].reset();
        ex[1].reset();
        free_workspace(&ws);
    }
};

using ShapeKey = std::tuple<int, int, int, int>;  // nx, ny, nz, capacity

struct Server;

}  // namespace

struct sift3d_ctx {
    sift3d_params p{};
    std::string err;
    float pattern[SIFT3D_N_PAIRS * 6];
    int device = -1;
    std::map<ShapeKey, std::unique_ptr<DetectEntry>> cache;
    DetectEntry* last = nullptr;
    int last_dtype = 0;
    std::unique_ptr<Server> server;
    std::mutex err_mu;
    float* blur_scratch = nullptr;     // two pitched float32 volumes
    int64_t blur_scratch_elems = 0;    // per volume
    char* arena = nullptr;             // device memory every cached shape's pyramid uses
    size_t arena_bytes = 0;
    int test_timeouts_left = 0;        // detects still to run with the peak wait test
    int* test_flag = nullptr;          // device int read by the peak kernel (test_wait_timeout > 0)
    std::unique_ptr<BatchExec> batch;  // the last batched detect's graph and memory
};

namespace {

int set_err(sift3d_ctx* c, int code, const std::string& msg) {
    if (c) {
        std::lock_guard<std::mutex> g(c->err_mu);
        c->err = msg;
    }
    return code;
}

int ensure_device(sift3d_ctx* c) {
    if (c->device >= 0) return cudaSetDevice(c->device) == cudaSuccess ? SIFT3D_OK : SIFT3D_ECUDA;
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return set_err(c, SIFT3D_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    c->device = d;
    return SIFT3D_OK;
}

int get_entry(sift3d_ctx* c, int nx, int ny, int nz, int dtype, int capacity, DetectEntry** out) {
    // Every shape's pyramid lives in one context arena (a context runs one
    // detect at a time, and a pyramid only has to last until the next detect);
    // each shape keeps its own plan and graph.  The arena grows to the largest
    // shape seen; growing it drops the cached graphs, which point into it.
    const ShapeKey key{nx, ny, nz, capacity};
    auto it = c->cache.find(key);
    if (it == c->cache.end()) {
        Plan pl;
        std::string err;
        int rc = make_plan(c->p, nx, ny, nz, dtype, &pl, &err);
        if (rc != SIFT3D_OK) return set_err(c, rc, err);
        const size_t need = workspace_bytes(pl, capacity);
        if (need > c->arena_bytes) {
            cudaDeviceSynchronize();
            c->cache.clear();
            c->last = nullptr;
            if (c->arena) cudaFree(c->arena);
            c->arena = nullptr;
            c->arena_bytes = 0;
            rc = alloc_device_zeroed(need, &c->arena, &err);
            if (rc != SIFT3D_OK) return set_err(c, rc, err);
            c->arena_bytes = need;
        }
        auto ent = std::make_unique<DetectEntry>();
        rc = bind_workspace(pl, capacity, c->arena, &ent->ws, &err);
        if (rc != SIFT3D_OK) return set_err(c, rc, err);
        ent->ws.test_flag = c->test_flag;
        it = c->cache.emplace(key, std::move(ent)).first;
    }
    DetectEntry* e = it->second.get();
    if (!e->ex[dtype]) e->ex[dtype] = std::make_unique<DetectExec>();
    *out = e;
    return SIFT3D_OK;
}

int launch(const LaunchSpec& s, void* argp, cudaStream_t st, std::string* err) {
    void* args[1] = {argp};
    cudaError_t e = launch_spec(s, args, st);
    if (e != cudaSuccess) {
        if (err) *err = std::string(s.name) + ": " + cudaGetErrorString(e);
        return SIFT3D_ECUDA;
    }
    return SIFT3D_OK;
}

// Enqueue detect (no host wait) on an entry's workspace.
int enqueue_detect(DetectEntry* ent, const void* vol, int dtype, sift3d_keypoint* out, bool graphs,
                   cudaStream_t st, std::string* err) {
    if (ent->ws.plan.nO == 0) {
        cudaError_t e = cudaMemsetAsync(ent->ws.count_out, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ent->ws.count, 0, sizeof(int), st);
        if (e != cudaSuccess) {
            if (err) *err = cudaGetErrorString(e);
            return SIFT3D_ECUDA;
        }
        return SIFT3D_OK;
    }
    DetectCall call{vol, dtype, out, ent->ws.capacity};
    return run_detect(ent->ws, *ent->ex[dtype], call, graphs, ent->ws.plan.p.profile != 0, st, err);
}

int enqueue_describe(const DetectEntry* ent, const float* pattern, const sift3d_keypoint* kps, int n, int kind,
                     uint64_t* brief, uint8_t* rrief, cudaStream_t st, std::string* err) {
    DescribeArgs a = make_describe_args(ent->ws, pattern);
    a.kps = kps;
    a.n = n;
    a.n_dev = ent->ws.count_out;
    a.n_cap = ent->ws.capacity;
    a.brief = (kind & SIFT3D_DESC_BRIEF) ? brief : nullptr;
    a.rrief = (kind & SIFT3D_DESC_RRIEF) ? rrief : nullptr;
    const int n_max = n >= 0 ? n : ent->ws.capacity;
    if (n_max == 0 || ent->ws.plan.nO == 0) return SIFT3D_OK;
    LaunchSpec s = describe_spec(ent->ws.plan.p.storage, a, n_max);
    return launch(s, &a, st, err);
}

// ----------------------------------------------------------------------------
// Serving: a worker thread admits queued requests while their device bytes fit
// the HBM budget and a slot is free, runs each on its own stream (so requests
// overlap on the device), and retires them when their completion event fires.
// ----------------------------------------------------------------------------
struct ServeBuffers {            // device + pinned buffers for one (shape, dtype)
    std::unique_ptr<DetectEntry> ent;
    int dtype = 0;
    void* d_in = nullptr;
    size_t in_bytes = 0;
    sift3d_keypoint* d_kps = nullptr;
    uint64_t* d_brief = nullptr;
    uint8_t* d_rrief = nullptr;
    void* h_in = nullptr;        // pinned staging of the input
    // results: mapped pinned host memory, written by the pack kernel through
    // their device addresses (d_out_*)
    sift3d_keypoint* h_kps = nullptr;
    uint64_t* h_brief = nullptr;
    uint8_t* h_rrief = nullptr;
    int* h_count = nullptr;
    PackArgs pack{};
    size_t bytes = 0;            // device bytes held
    ~ServeBuffers() {
        cudaFree(d_in);
        cudaFree(d_kps);
        cudaFree(d_brief);
        cudaFree(d_rrief);
        cudaFreeHost(h_in);
        cudaFreeHost(h_kps);
        cudaFreeHost(h_brief);
        cudaFreeHost(h_rrief);
        cudaFreeHost(h_count);
    }
};

struct Request {
    uint64_t ticket = 0;
    int dtype = 0, nx = 0, ny = 0, nz = 0, flags = 0;
    const void* user_in = nullptr;       // NOCOPY
    std::vector<uint8_t> host_copy;      // default: copied at submit
    enum State { QUEUED, RUNNING, DONE, FAILED } state = QUEUED;
    int status = SIFT3D_OK;
    std::string err;
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::unique_ptr<ServeBuffers> buf;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int n_kps = 0, n_needed = 0;
    std::vector<sift3d_keypoint> kps;
    std::vector<uint64_t> brief;
    std::vector<uint8_t> rrief;
};

struct Server {
    sift3d_ctx* ctx;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::vector<Request*> running;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::multimap<std::tuple<int, int, int, int>, std::unique_ptr<ServeBuffers>> pool;  // idle buffers
    std::vector<cudaStream_t> streams;   // free streams
    uint64_t next_ticket = 1;
    uint64_t budget = 0, used = 0, pooled = 0;
    bool stop = false;
    std::thread th;
    // Completions reported by a host function at the end of each request's
    // stream work; the worker wakes on them instead of polling.
    std::atomic<uint64_t> signals{0};
    uint64_t seen = 0;
    std::map<std::tuple<int, int, int, int>, uint64_t> est_cache;   // request_bytes per shape (worker only)

    static void CUDART_CB on_done(void* self) {   // no CUDA calls and no lock in here
        Server* sv = static_cast<Server*>(self);
        sv->signals.fetch_add(1, std::memory_order_release);
        sv->cv_work.notify_one();
    }

    explicit Server(sift3d_ctx* c) : ctx(c) {
        budget = c->p.hbm_budget_bytes ? c->p.hbm_budget_bytes : (40ull << 30);
        th = std::thread([this] { loop(); });
    }
    ~Server() {
        {
            std::lock_guard<std::mutex> g(mu);
            stop = true;
        }
        cv_work.notify_all();
        th.join();
        for (Request* r : running) {
            cudaEventSynchronize(r->done);
            cudaEventDestroy(r->done);
        }
        for (cudaStream_t s : streams) {
            cudaStreamSynchronize(s);   // each request's completion host function has run
            cudaStreamDestroy(s);
        }
        pool.clear();
    }

    uint64_t request_bytes(int nx, int ny, int nz, int dtype, std::string* err, int* rc) {
        Plan pl;
        *rc = make_plan(ctx->p, nx, ny, nz, dtype, &pl, err);
        if (*rc != SIFT3D_OK) return 0;
        const size_t cap = (size_t)std::max(ctx->p.max_keypoints, 1);
        return pl.bytes + cap * (sizeof(sift3d_keypoint) * 2 + 8 + 64) + (size_t)nx * ny * nz * 4 + (1 << 20);
    }

    // request_bytes of a shape that planned once (the worker thread only).
    uint64_t estimate(const Request& r, std::string* err, int* rc) {
        const auto key = std::make_tuple(r.nx, r.ny, r.nz, r.dtype);
        auto it = est_cache.find(key);
        if (it != est_cache.end()) {
            *rc = SIFT3D_OK;
            return it->second;
        }
        const uint64_t b = request_bytes(r.nx, r.ny, r.nz, r.dtype, err, rc);
        if (*rc == SIFT3D_OK) est_cache.emplace(key, b);
        return b;
    }

    std::unique_ptr<ServeBuffers> take_buffers(const Request& r, std::string* err, int* rc) {
        const auto key = std::make_tuple(r.nx, r.ny, r.nz, r.dtype);
        auto it = pool.find(key);
        if (it != pool.end()) {
            auto b = std::move(it->second);
            pool.erase(it);
            pooled -= b->bytes;
            return b;
        }
        auto b = std::make_unique<ServeBuffers>();
        b->dtype = r.dtype;
        const int cap = std::max(ctx->p.max_keypoints, 1);
        Plan pl;
        *rc = make_plan(ctx->p, r.nx, r.ny, r.nz, r.dtype, &pl, err);
        if (*rc != SIFT3D_OK) return nullptr;
        b->ent = std::make_unique<DetectEntry>();
        *rc = alloc_workspace(pl, cap, &b->ent->ws, err);
        if (*rc != SIFT3D_OK) return nullptr;
        b->ent->ex[r.dtype] = std::make_unique<DetectExec>();
        b->in_bytes = (size_t)r.nx * r.ny * r.nz * (r.dtype == SIFT3D_DTYPE_U8 ? 1 : 4);
        const unsigned mapped = cudaHostAllocMapped;
        cudaError_t e = dev_alloc(&b->d_in, b->in_bytes);
        if (e == cudaSuccess) e = dev_alloc((void**)&b->d_kps, (size_t)cap * sizeof(sift3d_keypoint));
        if (e == cudaSuccess) e = dev_alloc((void**)&b->d_brief, (size_t)cap * 8);
        if (e == cudaSuccess) e = dev_alloc((void**)&b->d_rrief, (size_t)cap * 64);
        if (e == cudaSuccess) e = pinned_alloc(&b->h_in, b->in_bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = pinned_alloc((void**)&b->h_kps, (size_t)cap * sizeof(sift3d_keypoint), mapped);
        if (e == cudaSuccess) e = pinned_alloc((void**)&b->h_brief, (size_t)cap * 8, mapped);
        if (e == cudaSuccess) e = pinned_alloc((void**)&b->h_rrief, (size_t)cap * 64, mapped);
        if (e == cudaSuccess) e = pinned_alloc((void**)&b->h_count, 2 * sizeof(int), mapped);
        PackArgs& pk = b->pack;
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&pk.out_kps, b->h_kps, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&pk.out_brief, b->h_brief, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&pk.out_rrief, b->h_rrief, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&pk.out_count, b->h_count, 0);
        pk.count = b->ent->ws.count_out;
        pk.capacity = cap;
        pk.kps = b->d_kps;
        pk.brief = b->d_brief;
        pk.rrief = b->d_rrief;
        if (e != cudaSuccess) {
            *err = std::string("serving buffers: ") + cudaGetErrorString(e);
            *rc = e == cudaErrorMemoryAllocation ? SIFT3D_ENOMEM : SIFT3D_ECUDA;
            (void)cudaGetLastError();
            return nullptr;
        }
        b->bytes = b->ent->ws.bytes + b->in_bytes + (size_t)cap * (sizeof(sift3d_keypoint) + 8 + 64);
        return b;
    }

    // Free idle pooled buffers until `need` more bytes fit in the budget.
    void evict_for(uint64_t need) {
        while (used + pooled + need > budget && !pool.empty()) {
            auto it = pool.begin();
            pooled -= it->second->bytes;
            pool.erase(it);   // synchronising cudaFree: only on shape churn
        }
    }

    // Runs on the worker thread without the lock: it touches only worker-owned
    // members (pool, streams, used, pooled) and fields of r that API threads
    // read after the worker publishes r's state under the lock.  Returns true
    // when r holds buffers and is running on the device.
    bool admit(Request* r) {
        std::string err;
        int rc = SIFT3D_OK;
        const uint64_t est = estimate(*r, &err, &rc);
        evict_for(est);
        r->buf = take_buffers(*r, &err, &rc);
        if (!r->buf) {
            r->status = rc == SIFT3D_OK ? SIFT3D_ECUDA : rc;
            r->err = err;
            r->t_admit = r->t_done = now_ms();
            return false;
        }
        used += r->buf->bytes;
        if (streams.empty()) {
            cudaStream_t s;
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            streams.push_back(s);
        }
        r->stream = streams.back();
        streams.pop_back();
        cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming);
        ServeBuffers& b = *r->buf;
        const void* src = r->user_in;
        const void* vol = b.d_in;
        cudaError_t e = cudaSuccess;
        if (r->flags & SIFT3D_SUBMIT_DEVICE) {   // read in place on the device
            vol = r->user_in;
        } else {
            if (!(r->flags & SIFT3D_SUBMIT_NOCOPY)) {
                memcpy(b.h_in, r->host_copy.data(), b.in_bytes);
                src = b.h_in;
            }
            e = cudaMemcpyAsync(b.d_in, src, b.in_bytes, cudaMemcpyHostToDevice, r->stream);
            if (e != cudaSuccess) rc = SIFT3D_ECUDA, err = cudaGetErrorString(e);
        }
        if (rc == SIFT3D_OK)
            rc = enqueue_detect(b.ent.get(), vol, r->dtype, b.d_kps, ctx->p.use_graphs != 0, r->stream, &err);
        if (rc == SIFT3D_OK)
            rc = enqueue_describe(b.ent.get(), ctx->pattern, b.d_kps, -1, SIFT3D_DESC_BOTH, b.d_brief, b.d_rrief,
                                  r->stream, &err);
        if (rc == SIFT3D_OK) {   // exactly the detected records, written to mapped host memory
            rc = launch(pack_spec(b.pack), &b.pack, r->stream, &err);
            if (rc == SIFT3D_OK) {
                e = cudaEventRecord(r->done, r->stream);
                if (e != cudaSuccess) rc = SIFT3D_ECUDA, err = cudaGetErrorString(e);
            }
            // wake the worker when the stream gets here (without it the worker
            // still finds the event complete at its next timed wake-up)
            if (rc == SIFT3D_OK) (void)cudaLaunchHostFunc(r->stream, &Server::on_done, this);
        }
        r->t_admit = now_ms();
        if (rc != SIFT3D_OK) {
            r->status = rc;
            r->err = err;
        }
        return true;
    }

    void retire(Request* r) {
        ServeBuffers& b = *r->buf;
        if (r->status == SIFT3D_OK) {
            const int total = *(volatile int*)b.h_count;
            const int cap = b.ent->ws.capacity;
            r->n_needed = total;
            r->n_kps = std::min(total, cap);
            r->kps.assign(b.h_kps, b.h_kps + r->n_kps);
            r->brief.assign(b.h_brief, b.h_brief + r->n_kps);
            r->rrief.assign(b.h_rrief, b.h_rrief + (size_t)r->n_kps * 64);
            if (total > cap) r->status = SIFT3D_ECAPACITY;
        }
        cudaEventDestroy(r->done);
        r->done = nullptr;
        streams.push_back(r->stream);
        r->stream = nullptr;
        used -= b.bytes;
        pooled += b.bytes;
        pool.emplace(std::make_tuple(r->nx, r->ny, r->nz, r->dtype), std::move(r->buf));
        r->host_copy.clear();
        r->host_copy.shrink_to_fit();
        r->t_done = now_ms();
        r->state = (r->status == SIFT3D_OK || r->status == SIFT3D_ECAPACITY) ? Request::DONE : Request::FAILED;
    }

    void loop() {
        cudaSetDevice(ctx->device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            bool progressed = false, budget_blocked = false;
            seen = signals.load(std::memory_order_acquire);   // a later signal re-runs this loop
            for (size_t i = 0; i < running.size();) {
                Request* r = running[i];
                const cudaError_t q = r->status == SIFT3D_OK ? cudaEventQuery(r->done) : cudaSuccess;
                if (q == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                if (q != cudaSuccess && r->status == SIFT3D_OK) {
                    r->status = SIFT3D_ECUDA;
                    r->err = cudaGetErrorString(q);
                }
                if (r->status != SIFT3D_OK && r->done) cudaEventSynchronize(r->done);
                retire(r);
                running.erase(running.begin() + i);
                progressed = true;
            }
            while (!queue.empty() && (int)running.size() < ctx->p.max_inflight) {
                Request* r = queue.front();
                std::string err;
                int rc = SIFT3D_OK;
                const uint64_t est = estimate(*r, &err, &rc);
                if (used + est > budget && !running.empty()) {   // wait for memory to free up
                    budget_blocked = true;
                    break;
                }
                queue.pop_front();
                lk.unlock();   // the CUDA calls of admission run without the lock
                const bool on_device = admit(r);
                lk.lock();
                if (on_device) {
                    r->state = Request::RUNNING;
                    running.push_back(r);
                } else {
                    r->state = Request::FAILED;
                }
                progressed = true;
            }
            if (progressed) cv_done.notify_all();
            if (stop && queue.empty() && running.empty()) break;
            if (running.empty() && queue.empty()) {
                cv_work.wait(lk, [&] { return stop || !queue.empty(); });
            } else if (!progressed) {
                // a completion signal, new work, or (a signal lost between the
                // check and the wait) the next timed wake-up
                cv_work.wait_for(lk, std::chrono::microseconds(200), [&] {
                    return stop || signals.load(std::memory_order_acquire) != seen ||
                           (!budget_blocked && !queue.empty() && (int)running.size() < ctx->p.max_inflight);
                });
            }
        }
    }
};

}  // namespace

// ============================================================================
extern "C" {

int sift3d_default_params(sift3d_params* out) {
    if (!out) return SIFT3D_EINVAL;
    memset(out, 0, sizeof(*out));
    out->sigma0 = 1.6;
    out->sigma_in = 0.5;
    out->scales_per_octave = 3;
    out->min_octave_dim = 16;
    out->max_octaves = 0;
    out->sign_sum_min = 80;
    out->border = 1;
    out->contrast_thresh = 0.005;
    out->curvature_r = 10.0;
    out->trunc = 4.0;
    out->desc_blur_sigma = 0.95;
    out->desc_method = 3;
    out->pattern_seed = 0x5EED5EEDull;
    out->storage = SIFT3D_STORAGE_F32;
    out->use_graphs = 1;
    out->hbm_budget_bytes = 40ull << 30;
    out->max_keypoints = 8192;
    out->max_inflight = 4;
    out->test_wait_timeout = 0;
    out->autotune = 1;
    out->conv_row_tile = 0;
    out->conv_z_tile = 0;
    out->refine = 0;
    return SIFT3D_OK;
}

int sift3d_plan(const sift3d_params* params, int nx, int ny, int nz, sift3d_plan_info* out) {
    if (!params || !out) return SIFT3D_EINVAL;
    Plan pl;
    int rc = make_plan(*params, nx, ny, nz, SIFT3D_DTYPE_F32, &pl, nullptr);
    if (rc != SIFT3D_OK) return rc;
    fill_plan_info(pl, out);
    return SIFT3D_OK;
}

int sift3d_pattern(const sift3d_params* params, float* out) {
    if (!params || !out) return SIFT3D_EINVAL;
    make_pattern(*params, out);
    return SIFT3D_OK;
}

int sift3d_create(const sift3d_params* params, sift3d_ctx** out) {
    if (!out) return SIFT3D_EINVAL;
    *out = nullptr;
    if (!params) return SIFT3D_EINVAL;
    std::string err;
    const int rc = validate_params(*params, &err);
    if (rc != SIFT3D_OK) return rc;
    auto* c = new (std::nothrow) sift3d_ctx();
    if (!c) return SIFT3D_ENOMEM;
    c->p = *params;
    if (const char* env = std::getenv("SIFT3D_PROFILE")) {   // per-stage timing without code changes
        if (env[0] == '1') c->p.profile = 1;
    }
    c->test_timeouts_left = params->test_wait_timeout;
    make_pattern(c->p, c->pattern);
    *out = c;
    return SIFT3D_OK;
}

void sift3d_destroy(sift3d_ctx* ctx) {
    if (!ctx) return;
    if (ctx->device >= 0) cudaSetDevice(ctx->device);
    ctx->server.reset();
    if (ctx->device >= 0) cudaDeviceSynchronize();
    ctx->cache.clear();
    ctx->batch.reset();
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->blur_scratch) cudaFree(ctx->blur_scratch);
    if (ctx->test_flag) cudaFree(ctx->test_flag);
    delete ctx;
}

const char* sift3d_last_error(const sift3d_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

int sift3d_detect(sift3d_ctx* ctx, const void* dev_vol, int dtype, int nx, int ny, int nz, void* stream,
                  sift3d_keypoint* dev_out, int capacity, int* n_out) {
    if (!ctx) return SIFT3D_EINVAL;
    if (!dev_vol) return set_err(ctx, SIFT3D_EINVAL, "dev_vol is NULL");
    if (dtype != SIFT3D_DTYPE_F32 && dtype != SIFT3D_DTYPE_U8) return set_err(ctx, SIFT3D_EINVAL, "bad dtype");
    if (capacity < 0 || capacity > (1 << 20)) return set_err(ctx, SIFT3D_EINVAL, "capacity must be in 0..2^20");
    if (capacity > 0 && !dev_out) return set_err(ctx, SIFT3D_EINVAL, "dev_out is NULL");
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4095 || ny > 4095 || nz > 4095)
        return set_err(ctx, SIFT3D_EINVAL, "each dimension must be in 1..4095");
    int rc = ensure_device(ctx);
    if (rc != SIFT3D_OK) return rc;
    if (ctx->p.test_wait_timeout > 0 && ctx->test_flag == nullptr) {
        if (dev_alloc((void**)&ctx->test_flag, sizeof(int)) != cudaSuccess) {
            (void)cudaGetLastError();
            ctx->test_flag = nullptr;
            return set_err(ctx, SIFT3D_ENOMEM, "test flag allocation");
        }
        ctx->cache.clear();   // cached graphs were built without the flag
        ctx->last = nullptr;
    }
    DetectEntry* ent = nullptr;
    rc = get_entry(ctx, nx, ny, nz, dtype, capacity, &ent);
    if (rc != SIFT3D_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::string err;
    if (ctx->test_flag != nullptr) {   // testing the timeout path: set or clear the device flag
        const int flag = ctx->test_timeouts_left > 0 ? 1 : 0;
        if (ctx->test_timeouts_left > 0) --ctx->test_timeouts_left;
        if (cudaMemsetAsync(ctx->test_flag, flag, sizeof(int), st) != cudaSuccess)
            return set_err(ctx, SIFT3D_ECUDA, "test flag");
    }
    rc = enqueue_detect(ent, dev_vol, dtype, dev_out, ctx->p.use_graphs != 0, st, &err);
    if (rc != SIFT3D_OK) return set_err(ctx, rc, err);
    ctx->last = ent;
    ctx->last_dtype = dtype;
    if (n_out) {
        int h = 0;
        cudaError_t e = cudaMemcpyAsync(&h, ent->ws.count_out, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_err(ctx, SIFT3D_ECUDA, std::string("detect: ") + cudaGetErrorString(e));
        if (h == -2) return set_err(ctx, SIFT3D_ETIMEDOUT, "a bounded device wait ran out (peak kernel plane copy)");
        *n_out = h;
        if (h > capacity) return set_err(ctx, SIFT3D_ECAPACITY, "more keypoints than capacity");
    }
    return SIFT3D_OK;
}

const int* sift3d_device_count(const sift3d_ctx* ctx) {
    return (ctx && ctx->last) ? ctx->last->ws.count_out : nullptr;
}

int sift3d_describe(sift3d_ctx* ctx, const sift3d_keypoint* dev_kps, int n, int kind, uint64_t* dev_brief,
                    uint8_t* dev_rrief, void* stream) {
    if (!ctx) return SIFT3D_EINVAL;
    if (!ctx->last) return set_err(ctx, SIFT3D_EINVAL, "describe needs a prior detect");
    if (kind < SIFT3D_DESC_BRIEF || kind > SIFT3D_DESC_BOTH) return set_err(ctx, SIFT3D_EINVAL, "bad kind");
    if (((kind & SIFT3D_DESC_BRIEF) && !dev_brief) || ((kind & SIFT3D_DESC_RRIEF) && !dev_rrief))
        return set_err(ctx, SIFT3D_EINVAL, "descriptor output is NULL");
    if (n < -1) return set_err(ctx, SIFT3D_EINVAL, "n must be >= -1");
    if (n != 0 && !dev_kps) return set_err(ctx, SIFT3D_EINVAL, "dev_kps is NULL");
    int rc = ensure_device(ctx);
    if (rc != SIFT3D_OK) return rc;
    std::string err;
    rc = enqueue_describe(ctx->last, ctx->pattern, dev_kps, n, kind, dev_brief, dev_rrief,
                          static_cast<cudaStream_t>(stream), &err);
    return rc == SIFT3D_OK ? rc : set_err(ctx, rc, err);
}

int sift3d_detect_batch(sift3d_ctx* ctx, int n, const void* const* dev_vols, const int* dims, int dtype,
                        void* stream, sift3d_keypoint* const* dev_out, int capacity, uint64_t* const* dev_brief,
                        uint8_t* const* dev_rrief, int* n_out) {
    if (!ctx) return SIFT3D_EINVAL;
    if (n < 1 || !dev_vols || !dims || !dev_out) return set_err(ctx, SIFT3D_EINVAL, "bad batch arrays");
    if (dtype != SIFT3D_DTYPE_F32 && dtype != SIFT3D_DTYPE_U8) return set_err(ctx, SIFT3D_EINVAL, "bad dtype");
    if (capacity < 1 || capacity > (1 << 20)) return set_err(ctx, SIFT3D_EINVAL, "capacity must be in 1..2^20");
    if ((dev_brief == nullptr) != (dev_rrief == nullptr))
        return set_err(ctx, SIFT3D_EINVAL, "dev_brief and dev_rrief must both be set or both be NULL");
    const bool describe = dev_brief != nullptr;
    std::vector<std::array<int, 3>> d(n);
    for (int v = 0; v < n; ++v) {
        d[v] = {dims[3 * v], dims[3 * v + 1], dims[3 * v + 2]};
        if (!dev_vols[v] || !dev_out[v] || (describe && (!dev_brief[v] || !dev_rrief[v])))
            return set_err(ctx, SIFT3D_EINVAL, "a batch pointer is NULL");
        for (int a = 0; a < 3; ++a)
            if (d[v][a] < 1 || d[v][a] > 4095) return set_err(ctx, SIFT3D_EINVAL, "each dimension must be in 1..4095");
    }
    int rc = ensure_device(ctx);
    if (rc != SIFT3D_OK) return rc;
    std::string err;
    if (!ctx->batch || !ctx->batch->matches(d, dtype, capacity, describe)) {
        ctx->batch.reset();   // frees the previous batch's memory (cudaFree waits for its work)
        auto b = std::make_unique<BatchExec>();
        rc = build_batch(ctx->p, d, dtype, capacity, describe, ctx->pattern, b.get(), &err);
        if (rc != SIFT3D_OK) return set_err(ctx, rc, err);
        ctx->batch = std::move(b);
    }
    std::vector<uint64_t*> nb(n, nullptr);
    std::vector<uint8_t*> nr(n, nullptr);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = run_batch(*ctx->batch, dev_vols, dev_out, describe ? dev_brief : nb.data(), describe ? dev_rrief : nr.data(),
                   st, &err);
    if (rc != SIFT3D_OK) return set_err(ctx, rc, err);
    if (n_out) {
        cudaError_t e = cudaMemcpyAsync(n_out, ctx->batch->counts, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_err(ctx, SIFT3D_ECUDA, std::string("detect_batch: ") + cudaGetErrorString(e));
        bool over = false;
        for (int v = 0; v < n; ++v) {
            if (n_out[v] == -2) return set_err(ctx, SIFT3D_ETIMEDOUT, "a bounded device wait ran out (peak copy)");
            over = over || n_out[v] > capacity;
        }
        if (over) return set_err(ctx, SIFT3D_ECAPACITY, "more keypoints than capacity in some volume");
    }
    return SIFT3D_OK;
}

int sift3d_describe_siftrank(sift3d_ctx* ctx, const sift3d_keypoint* dev_kps, int n, uint8_t* dev_desc,
                             float* dev_rot, void* stream) {
    if (!ctx) return SIFT3D_EINVAL;
    if (!ctx->last) return set_err(ctx, SIFT3D_EINVAL, "describe needs a prior detect");
    if (!dev_desc) return set_err(ctx, SIFT3D_EINVAL, "dev_desc is NULL");
    if (n < -1) return set_err(ctx, SIFT3D_EINVAL, "n must be >= -1");
    if (n != 0 && !dev_kps) return set_err(ctx, SIFT3D_EINVAL, "dev_kps is NULL");
    int rc = ensure_device(ctx);
    if (rc != SIFT3D_OK) return rc;
    const Workspace& ws = ctx->last->ws;
    if (ws.plan.nO == 0) return SIFT3D_OK;
    DescribeArgs d = make_describe_args(ws, ctx->pattern);
    for (int o = 0; o < ws.plan.nO; ++o)            // the Gaussian levels themselves
        for (int s = 1; s <= ws.plan.S; ++s) d.lv[o][s - 1].ptr = ws.G(o, s);
    rc = enqueue_siftrank(ws.plan.p.storage, d, dev_kps, n, ws.count_out, ws.capacity, dev_desc, dev_rot,
                          static_cast<cudaStream_t>(stream));
    return rc == SIFT3D_OK ? rc : set_err(ctx, rc, "siftrank launch failed");
}

int sift3d_gaussian_blur(sift3d_ctx* ctx, const float* dev_in, int nx, int ny, int nz, double sigma,
                         float* dev_out, void* stream) {
    if (!ctx) return SIFT3D_EINVAL;
    if (!dev_in || !dev_out) return set_err(ctx, SIFT3D_EINVAL, "dev_in / dev_out is NULL");
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4095 || ny > 4095 || nz > 4095)
        return set_err(ctx, SIFT3D_EINVAL, "each dimension must be in 1..4095");
    const int R = gaussian_radius(sigma, ctx->p.trunc);
    if (!(sigma > 0.0) || R < 1 || R > kMaxRadius)
        return set_err(ctx, SIFT3D_EINVAL, "sigma must be > 0 with ceil(trunc*sigma) <= 16");
    int rc = ensure_device(ctx);
    if (rc != SIFT3D_OK) return rc;
    const int64_t need = blur_pitch_elems(nx, ny, nz);
    if (need > ctx->blur_scratch_elems) {
        if (ctx->blur_scratch) cudaFree(ctx->blur_scratch);
        ctx->blur_scratch = nullptr;
        ctx->blur_scratch_elems = 0;
        cudaError_t e = dev_alloc((void**)&ctx->blur_scratch, (size_t)need * 2 * sizeof(float));
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            ctx->blur_scratch = nullptr;
            return set_err(ctx, SIFT3D_ENOMEM, std::string("blur scratch: ") + cudaGetErrorString(e));
        }
        ctx->blur_scratch_elems = need;
    }
    std::string err;
    rc = enqueue_blur(dev_in, nx, ny, nz, sigma, ctx->p.trunc, ctx->blur_scratch,
                      ctx->blur_scratch + ctx->blur_scratch_elems, dev_out, static_cast<cudaStream_t>(stream), &err);
    return rc == SIFT3D_OK ? rc : set_err(ctx, rc, err);
}

int sift3d_match(const void* dev_a, int na, const void* dev_b, int nb, int kind, int32_t* dev_nn,
                 int32_t* dev_dist, int32_t* dev_dist2, void* stream) {
    if (kind != SIFT3D_DESC_BRIEF && kind != SIFT3D_DESC_RRIEF) return SIFT3D_EINVAL;
    if (na < 0 || nb < 0) return SIFT3D_EINVAL;
    if (na == 0) return SIFT3D_OK;
    const uintptr_t align = kind == SIFT3D_DESC_BRIEF ? 8 : 16;
    if (!dev_a || !dev_nn || !dev_dist || (nb > 0 && !dev_b)) return SIFT3D_EINVAL;
    if (((uintptr_t)dev_a % align) != 0 || (nb > 0 && ((uintptr_t)dev_b % align) != 0)) return SIFT3D_EINVAL;
    MatchArgs a{};
    a.a = dev_a;
    a.b = dev_b;
    a.na = na;
    a.nb = nb;
    a.nn = dev_nn;
    a.dist = dev_dist;
    a.dist2 = dev_dist2;
    const LaunchSpec s = match_spec(kind, a);
    std::string err;
    return launch(s, &a, static_cast<cudaStream_t>(stream), &err);
}

int sift3d_read_level(sift3d_ctx* ctx, int octave, int kind, int index, float* dev_dst, void* stream) {
    if (!ctx) return SIFT3D_EINVAL;
    if (!ctx->last) return set_err(ctx, SIFT3D_EINVAL, "read_level needs a prior detect");
    if (!dev_dst) return set_err(ctx, SIFT3D_EINVAL, "dev_dst is NULL");
    const Workspace& ws = ctx->last->ws;
    const Plan& pl = ws.plan;
    if (octave < 0 || octave >= pl.nO) return set_err(ctx, SIFT3D_EINVAL, "octave out of range");
    const void* src = nullptr;
    if (kind == SIFT3D_LEVEL_GAUSS && index >= 0 && index < pl.L) src = ws.G(octave, index);
    else if (kind == SIFT3D_LEVEL_DOG && index >= 0 && index < pl.nD) src = ws.D(octave, index);
    else if (kind == SIFT3D_LEVEL_DESC && index >= 1 && index <= pl.S) src = ws.B(octave, index);
    if (!src) return set_err(ctx, SIFT3D_EINVAL, "level kind/index out of range");
    int rc = ensure_device(ctx);
    if (rc != SIFT3D_OK) return rc;
    ReadLevelArgs a{};
    a.src = src;
    a.py = pl.oct[octave].py;
    a.pz = pl.oct[octave].pz;
    a.nx = pl.oct[octave].nx;
    a.ny = pl.oct[octave].ny;
    a.nz = pl.oct[octave].nz;
    a.dst = dev_dst;
    std::string err;
    const int level_storage = kind == SIFT3D_LEVEL_DOG ? SIFT3D_STORAGE_F32 : pl.p.storage;   // DoG: float32
    rc = launch(read_level_spec(level_storage, a), &a, static_cast<cudaStream_t>(stream), &err);
    return rc == SIFT3D_OK ? rc : set_err(ctx, rc, err);
}

int sift3d_stage_times(sift3d_ctx* ctx, int max, float* ms_out, const char** names_out, uint64_t* algo_bytes_out,
                       int* n_out) {
    if (!ctx) return SIFT3D_EINVAL;
    if (!ctx->last || !ctx->last->ex[ctx->last_dtype]) return set_err(ctx, SIFT3D_EINVAL, "no prior detect");
    const DetectExec& ex = *ctx->last->ex[ctx->last_dtype];
    if (!ex.profile || ex.ev_end.empty()) return set_err(ctx, SIFT3D_EINVAL, "context created with profile = 0");
    if (max < 0 || (max > 0 && !ms_out)) return set_err(ctx, SIFT3D_EINVAL, "bad output array");
    const int n = (int)ex.nodes.size();
    if (n_out) *n_out = n;
    for (int i = 0; i < n && i < max; ++i) {
        cudaError_t e = cudaEventSynchronize(ex.ev_end[i]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ex.ev_begin[i], ex.ev_end[i]);
        if (e != cudaSuccess) return set_err(ctx, SIFT3D_ECUDA, std::string("stage_times: ") + cudaGetErrorString(e));
        ms_out[i] = ms;
        if (names_out) names_out[i] = ex.nodes[i].label.c_str();
        if (algo_bytes_out) algo_bytes_out[i] = ex.nodes[i].algo_bytes;
    }
    return SIFT3D_OK;
}

int sift3d_stage_timeline(sift3d_ctx* ctx, int max, float* begin_ms_out, float* end_ms_out, int* n_out) {
    if (!ctx) return SIFT3D_EINVAL;
    if (!ctx->last || !ctx->last->ex[ctx->last_dtype]) return set_err(ctx, SIFT3D_EINVAL, "no prior detect");
    const DetectExec& ex = *ctx->last->ex[ctx->last_dtype];
    if (!ex.profile || ex.ev_end.empty()) return set_err(ctx, SIFT3D_EINVAL, "context created with profile = 0");
    if (max < 0 || (max > 0 && (!begin_ms_out || !end_ms_out))) return set_err(ctx, SIFT3D_EINVAL, "bad output array");
    const int n = (int)ex.nodes.size();
    if (n_out) *n_out = n;
    for (int i = 0; i < n && i < max; ++i) {
        cudaError_t e = cudaEventSynchronize(ex.ev_end[i]);
        float b = 0.f, t = 0.f;
        // node 0 is the first pass of octave 0, the root of the DAG
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ex.ev_begin[0], ex.ev_begin[i]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ex.ev_begin[0], ex.ev_end[i]);
        if (e != cudaSuccess) return set_err(ctx, SIFT3D_ECUDA, std::string("stage_timeline: ") + cudaGetErrorString(e));
        begin_ms_out[i] = b;
        end_ms_out[i] = t;
    }
    return SIFT3D_OK;
}

int sift3d_submit(sift3d_ctx* ctx, const void* host_vol, int dtype, int nx, int ny, int nz, int flags,
                  uint64_t* ticket) {
    if (!ctx) return SIFT3D_EINVAL;
    if (!host_vol || !ticket) return set_err(ctx, SIFT3D_EINVAL, "host_vol and ticket must be non-NULL");
    if (dtype != SIFT3D_DTYPE_F32 && dtype != SIFT3D_DTYPE_U8) return set_err(ctx, SIFT3D_EINVAL, "bad dtype");
    if (flags & ~(SIFT3D_SUBMIT_NOCOPY | SIFT3D_SUBMIT_DEVICE)) return set_err(ctx, SIFT3D_EINVAL, "unknown flags");
    Plan pl;
    std::string err;
    int rc = make_plan(ctx->p, nx, ny, nz, dtype, &pl, &err);
    if (rc != SIFT3D_OK) return set_err(ctx, rc, err);
    rc = ensure_device(ctx);
    if (rc != SIFT3D_OK) return rc;
    if (flags & SIFT3D_SUBMIT_DEVICE) {   // must be device memory of this context's GPU
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, host_vol) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != ctx->device) {
            (void)cudaGetLastError();
            return set_err(ctx, SIFT3D_EINVAL, "SIFT3D_SUBMIT_DEVICE: not device memory of the context's GPU");
        }
    }
    if (!ctx->server) ctx->server = std::make_unique<Server>(ctx);
    Server& sv = *ctx->server;
    const uint64_t need = sv.request_bytes(nx, ny, nz, dtype, &err, &rc);
    if (rc != SIFT3D_OK) return set_err(ctx, rc, err);
    if (need > sv.budget) return set_err(ctx, SIFT3D_EBUDGET, "volume alone exceeds hbm_budget_bytes");
    auto r = std::make_unique<Request>();
    r->dtype = dtype;
    r->nx = nx;
    r->ny = ny;
    r->nz = nz;
    r->flags = flags;
    r->t_submit = now_ms();
    const size_t bytes = (size_t)nx * ny * nz * (dtype == SIFT3D_DTYPE_U8 ? 1 : 4);
    if (flags & (SIFT3D_SUBMIT_NOCOPY | SIFT3D_SUBMIT_DEVICE)) {
        r->user_in = host_vol;
    } else {
        try {
            r->host_copy.assign(static_cast<const uint8_t*>(host_vol), static_cast<const uint8_t*>(host_vol) + bytes);
        } catch (...) {
            return set_err(ctx, SIFT3D_ENOMEM, "host copy of the volume failed");
        }
    }
    {
        std::lock_guard<std::mutex> g(sv.mu);
        r->ticket = sv.next_ticket++;
        *ticket = r->ticket;
        sv.queue.push_back(r.get());
        sv.reqs.emplace(r->ticket, std::move(r));
    }
    sv.cv_work.notify_all();
    return SIFT3D_OK;
}

int sift3d_poll(sift3d_ctx* ctx, uint64_t ticket, int timeout_us, sift3d_result* out) {
    if (!ctx || !out) return SIFT3D_EINVAL;
    if (!ctx->server) return SIFT3D_ENOTFOUND;
    Server& sv = *ctx->server;
    std::unique_lock<std::mutex> lk(sv.mu);
    auto it = sv.reqs.find(ticket);
    if (it == sv.reqs.end()) return SIFT3D_ENOTFOUND;
    Request* r = it->second.get();
    auto finished = [&] { return r->state == Request::DONE || r->state == Request::FAILED; };
    if (!finished() && timeout_us > 0)
        sv.cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), finished);
    if (!finished()) return SIFT3D_PENDING;
    memset(out, 0, sizeof(*out));
    out->status = r->status;
    out->nx = r->nx;
    out->ny = r->ny;
    out->nz = r->nz;
    out->latency_ms = r->t_done - r->t_submit;
    out->queue_ms = r->t_admit - r->t_submit;
    if (r->state == Request::FAILED) {
        lk.unlock();
        return set_err(ctx, r->status == SIFT3D_OK ? SIFT3D_ECUDA : r->status, r->err);
    }
    out->n_keypoints = r->n_kps;
    out->n_needed = r->n_needed;
    out->keypoints = r->kps.data();
    out->brief = r->brief.data();
    out->rrief = r->rrief.data();
    return SIFT3D_OK;
}

int sift3d_test_fail_allocation(int n) {
    if (n < 0) return SIFT3D_EINVAL;
    set_allocation_failure(n);
    return SIFT3D_OK;
}

int sift3d_release(sift3d_ctx* ctx, uint64_t ticket) {
    if (!ctx) return SIFT3D_EINVAL;
    if (!ctx->server) return SIFT3D_ENOTFOUND;
    Server& sv = *ctx->server;
    std::lock_guard<std::mutex> g(sv.mu);
    auto it = sv.reqs.find(ticket);
    if (it == sv.reqs.end()) return SIFT3D_ENOTFOUND;
    const auto st = it->second->state;
    if (st != Request::DONE && st != Request::FAILED) return SIFT3D_PENDING;
    sv.reqs.erase(it);
    return SIFT3D_OK;
}

}  // extern "C"
