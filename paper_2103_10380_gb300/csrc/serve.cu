// serve.cu -- continuous-batching request loop: fnr_submit / fnr_poll / fnr_wait.
//
// A scheduler thread admits queued requests into batch slots as slots and
// HBM budget free up. Each slot runs one launch per batch on its own stream,
// replaying a captured CUDA graph of one kernel node whose grid size and
// parameters -- the batch table itself, passed by value as a __grid_constant__
// kernel parameter, so no upload precedes the kernel -- are set per batch.
// Every block marches 4 consecutive 8 x 4 pixel tiles of the batch's requests
// (one warp each), then adds its finished tiles to each touched request's
// counter; the block that completes a request resets that counter for the
// slot's next batch and writes the batch epoch into the request's host-mapped
// completion word, so a request completes as soon as its own tiles are done
// while the rest of its batch -- and batches on the other slots -- keep the
// GPU busy. (A persistent grid that pops tiles from a counter measured 20-30%
// slower per frame than letting the hardware schedule a grid sized to the
// batch.) No device code waits on anything: completion is observed by the host.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

#include "march_device.cuh"
#include "nvtx_range.h"

namespace fnr {

fnr_status fail(fnr_status st, const char *fmt, ...);
fnr_status cuda_fail(cudaError_t e, const char *what);
void clear_error();
fnr_status make_render_const(const fnr_render_params *p, RenderConst *rc);
fnr_status check_camera(const fnr_camera *c);
void fill_frame(FrameDesc *f, const fnr_camera *cam, float *rgba, fnr_ray_stats *stats, int32_t *cells,
                int tile_begin);
int frame_tiles(const fnr_camera *cam);
bool cache_belongs(fnr_context *ctx, const fnr_cache *c);
bool budget_charge(fnr_context *ctx, uint64_t bytes);
void budget_uncharge(fnr_context *ctx, uint64_t bytes);

constexpr int kMaxBatch = 64;
constexpr int kMaxSlots = 8;
constexpr uint64_t kSpinAfterActivityNs = 5000000;  // default: keep polling 5 ms after the last event

struct ServeFrame {
    CacheView c;
    RenderConst r;
    FrameDesc f;  // f.tile_begin: first batch tile of this request
    int32_t n_tiles;
    int32_t pad;
};

struct ServeTable {
    int32_t n_frames;
    int32_t total_tiles;
    uint32_t epoch;
    int32_t pad;
    int32_t tile_begin[kMaxBatch + 1];
    ServeFrame frames[kMaxBatch];
};

// Kernel parameters are limited to 32764 bytes; the table travels as one.
static_assert(sizeof(ServeTable) <= 32764, "the batch table is a kernel parameter");

struct ServeScratch {  // zeroed once; every request's counter returns to 0 when the request completes
    unsigned int done_tiles[kMaxBatch];
};

namespace {

// Request of batch tile t: the last request whose first tile is <= t.
__device__ __forceinline__ int serve_frame_of(const ServeTable &tab, int nf, int t) {
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab.tile_begin[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int PREC, int D, bool SKIP, bool BRICKS>
__global__ void __launch_bounds__(FNR_BLOCK, dev::min_blocks(PREC))
    serve_kernel(const __grid_constant__ ServeTable tab, ServeScratch *scr, volatile uint32_t *done_flags) {
    constexpr int kWarps = FNR_BLOCK / 32;
    __shared__ dev::QueueFor<PREC, D> queues[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int total = tab.total_tiles;
    const int nf = tab.n_frames;
    const int base = blockIdx.x * kWarps;
    if (base >= total) return;  // whole block
    const int t = base + warp;
    if (t < total) {
        const int f = serve_frame_of(tab, nf, t);
        const ServeFrame &sf = tab.frames[f];
        const int lt = t - tab.tile_begin[f];
        int x0, y0;
        tile_origin(sf.f, lt, x0, y0);
        const int px = x0 + (lane & (kTileW - 1)), py = y0 + lane / kTileW;
        dev::march_tile_queued<PREC, D, SKIP, BRICKS>(sf.c, sf.r, sf.f, px, py, px < sf.f.W && py < sf.f.H,
                                                      queues[warp]);
    }
    __syncthreads();  // the block's outputs are written
    if (threadIdx.x == 0) {
        __threadfence();
        const int last = min(base + kWarps, total);
        for (int t0 = base; t0 < last;) {  // the block's tiles, grouped by request
            const int f = serve_frame_of(tab, nf, t0);
            const int f_end = f + 1 < nf ? tab.tile_begin[f + 1] : total;
            const int t1 = min(last, f_end);
            const unsigned prev = atomicAdd(&scr->done_tiles[f], unsigned(t1 - t0));
            if (prev + unsigned(t1 - t0) == static_cast<unsigned>(tab.frames[f].n_tiles)) {
                scr->done_tiles[f] = 0u;  // every other block of this request has counted
                __threadfence_system();
                done_flags[f] = tab.epoch;
            }
            t0 = t1;
        }
    }
}

using ServeFn = void (*)(const ServeTable, ServeScratch *, volatile uint32_t *);

template <int PREC, bool SKIP, bool BRICKS>
ServeFn serve_fn_p(int D) {
    switch (D) {
        case 1: return serve_kernel<PREC, 1, SKIP, BRICKS>;
        case 2: return serve_kernel<PREC, 2, SKIP, BRICKS>;
        case 3: return serve_kernel<PREC, 3, SKIP, BRICKS>;
        case 4: return serve_kernel<PREC, 4, SKIP, BRICKS>;
        case 6: return serve_kernel<PREC, 6, SKIP, BRICKS>;
        case 8: return serve_kernel<PREC, 8, SKIP, BRICKS>;
        case 12: return serve_kernel<PREC, 12, SKIP, BRICKS>;
        case 16: return serve_kernel<PREC, 16, SKIP, BRICKS>;
        default: return nullptr;
    }
}

template <bool SKIP, bool BRICKS>
ServeFn serve_fn_s(int prec, int D) {
    switch (prec) {
        case FNR_PREC_FP32: return serve_fn_p<FNR_PREC_FP32, SKIP, BRICKS>(D);
        case FNR_PREC_FP16: return serve_fn_p<FNR_PREC_FP16, SKIP, BRICKS>(D);
        case FNR_PREC_FP8_E4M3: return serve_fn_p<FNR_PREC_FP8_E4M3, SKIP, BRICKS>(D);
        default: return nullptr;
    }
}

// Kernel key of a batch: requests share a launch when precision, D, the skip
// flag and the cache layout agree (brick caches always skip).
int serve_key(int prec, int D, bool skip, bool bricks) {
    return (bricks ? 256 : 0) + ((skip || bricks) ? 128 : 0) + prec * 32 + D;
}

ServeFn serve_fn(int key) {
    const int prec = (key & 127) / 32, D = key % 32;
    if (key & 256) return serve_fn_s<true, true>(prec, D);
    return key & 128 ? serve_fn_s<true, false>(prec, D) : serve_fn_s<false, false>(prec, D);
}

uint64_t now_ns() {
    return static_cast<uint64_t>(
        std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
            .count());
}

struct Request {
    fnr_request req;
    RenderConst rc;
    uint64_t bytes = 0;  // charged against the budget while admitted
    int key = 0;         // serve_key(prec, D, skip): one kernel instance per batch
    int64_t rays = 0;
    int32_t tiles = 0;
    uint64_t t_submit = 0, t_admit = 0, t_done = 0;
    fnr_status status = FNR_ERR_NOT_READY;
    bool queued = true;
    int64_t batch = -1;
    cudaEvent_t ready = nullptr;  // recorded on the request's stream at submit
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    ServeTable *h_table = nullptr;  // pinned; passed to the kernel by value
    ServeScratch *d_scratch = nullptr;
    uint32_t *h_flags = nullptr;  // pinned, mapped
    uint32_t *d_flags = nullptr;
    uint32_t epoch = 0;
    bool busy = false;
    int n = 0;
    uint64_t tickets[kMaxBatch];
    bool done[kMaxBatch];
    int remaining = 0;
    struct Graph {
        cudaGraph_t graph = nullptr;  // kept: its kernel node is updated per batch
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t kernel = nullptr;
        cudaKernelNodeParams params{};
    };
    std::map<int, Graph> graphs;
};

}  // namespace

struct Server {
    fnr_context *ctx = nullptr;
    fnr_serve_config cfg;
    uint64_t spin_after_ns = kSpinAfterActivityNs;
    bool spin_forever = false;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::vector<Slot> slots;
    std::thread th;
    bool stop = false;
    bool abandon = false;  // at process exit: drop the queued requests, finish only the launched batches
    uint64_t next_ticket = 1;
    int64_t next_batch = 0;
    fnr_status fatal = FNR_OK;
    std::vector<cudaEvent_t> free_events;  // recycled request-ordering events
    uint64_t last_activity_ns = 0;

    cudaEvent_t take_event() {
        if (!free_events.empty()) {
            cudaEvent_t e = free_events.back();
            free_events.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        return e;
    }

    void complete(Request &r, fnr_status st) {
        r.status = st;
        r.t_done = now_ns();
        budget_uncharge(ctx, r.bytes);
        r.bytes = 0;
        const_cast<fnr_cache *>(r.req.cache)->inflight.fetch_sub(1);
    }

    // Completion words of busy slots -> finished requests; frees slots.
    bool poll_locked() {
        bool progress = false;
        for (Slot &s : slots) {
            if (!s.busy) continue;
            for (int f = 0; f < s.n; ++f) {
                if (s.done[f]) continue;
                if (reinterpret_cast<volatile uint32_t *>(s.h_flags)[f] == s.epoch) {
                    std::atomic_thread_fence(std::memory_order_acquire);
                    auto it = reqs.find(s.tickets[f]);
                    if (it != reqs.end()) complete(it->second, FNR_OK);
                    s.done[f] = true;
                    --s.remaining;
                    progress = true;
                }
            }
            const cudaError_t q = cudaEventQuery(s.done_ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess || s.remaining > 0) {
                // the launch failed, or ended without flagging some request
                const fnr_status st = q != cudaSuccess ? FNR_ERR_CUDA : FNR_ERR_DEVICE;
                for (int f = 0; f < s.n; ++f)
                    if (!s.done[f]) {
                        if (reinterpret_cast<volatile uint32_t *>(s.h_flags)[f] == s.epoch && q == cudaSuccess) {
                            auto it = reqs.find(s.tickets[f]);
                            if (it != reqs.end()) complete(it->second, FNR_OK);
                        } else {
                            auto it = reqs.find(s.tickets[f]);
                            if (it != reqs.end()) complete(it->second, st);
                        }
                        s.done[f] = true;
                    }
                s.remaining = 0;
                if (q != cudaSuccess) fatal = FNR_ERR_CUDA;
            }
            s.busy = false;
            progress = true;
        }
        if (progress) cv_done.notify_all();
        return progress;
    }

    fnr_status launch(Slot &s, int key, int total_tiles) {
        NvtxRange range("fnr_serve_batch");
        ServeFn fn = serve_fn(key);
        const unsigned grid = unsigned((total_tiles + FNR_BLOCK / 32 - 1) / (FNR_BLOCK / 32));
        cudaError_t e;
        if (cfg.use_graphs) {
            auto it = s.graphs.find(key);
            if (it == s.graphs.end()) {
                Slot::Graph G;
                if ((e = cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                    return cuda_fail(e, "graph capture");
                fn<<<1, FNR_BLOCK, 0, s.stream>>>(*s.h_table, s.d_scratch, s.d_flags);
                if ((e = cudaStreamEndCapture(s.stream, &G.graph)) != cudaSuccess) return cuda_fail(e, "graph capture");
                size_t n = 0;
                cudaGraphGetNodes(G.graph, nullptr, &n);
                std::vector<cudaGraphNode_t> nodes(n);
                cudaGraphGetNodes(G.graph, nodes.data(), &n);
                for (cudaGraphNode_t nd : nodes) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) G.kernel = nd;
                }
                if (!G.kernel || (e = cudaGraphKernelNodeGetParams(G.kernel, &G.params)) != cudaSuccess ||
                    (e = cudaGraphInstantiate(&G.exec, G.graph, 0)) != cudaSuccess) {
                    cudaGraphDestroy(G.graph);
                    return cuda_fail(e, "graph instantiate");
                }
                it = s.graphs.emplace(key, G).first;
            }
            Slot::Graph &G = it->second;
            void *args[3] = {s.h_table, &s.d_scratch, &s.d_flags};  // the table by value
            cudaKernelNodeParams kp = G.params;
            kp.gridDim = dim3(grid);
            kp.kernelParams = args;
            kp.extra = nullptr;
            if ((e = cudaGraphExecKernelNodeSetParams(G.exec, G.kernel, &kp)) != cudaSuccess)
                return cuda_fail(e, "graph update");
            if ((e = cudaGraphLaunch(G.exec, s.stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
        } else {
            fn<<<grid, FNR_BLOCK, 0, s.stream>>>(*s.h_table, s.d_scratch, s.d_flags);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "serve launch");
        }
        if ((e = cudaEventRecord(s.done_ev, s.stream)) != cudaSuccess) return cuda_fail(e, "event record");
        return FNR_OK;
    }

    // Queued requests -> free slots, in arrival order, one kernel key per batch.
    bool admit_locked() {
        if (abandon) return false;
        bool progress = false;
        for (Slot &s : slots) {
            if (s.busy || pending.empty()) continue;
            ServeTable &tb = *s.h_table;
            int n = 0, tiles = 0, key = -1;
            int64_t rays = 0;
            bool blocked = false;
            for (auto it = pending.begin(); it != pending.end() && n < cfg.max_batch_requests;) {
                Request &r = reqs[*it];
                if (key < 0) key = r.key;
                if (r.key != key) {
                    ++it;
                    continue;
                }
                if (n > 0 && rays + r.rays > cfg.max_batch_rays) break;
                if (!budget_charge(ctx, r.bytes)) {  // wait for memory to free up
                    blocked = true;
                    break;
                }
                ServeFrame &sf = tb.frames[n];
                sf.c = r.req.cache->view;
                sf.r = r.rc;
                fill_frame(&sf.f, &r.req.camera, r.req.rgba_dev, r.req.stats_dev, nullptr, tiles);
                sf.n_tiles = r.tiles;
                tb.tile_begin[n] = tiles;
                tiles += r.tiles;
                rays += r.rays;
                r.queued = false;
                r.t_admit = now_ns();
                r.batch = next_batch;
                s.tickets[n] = *it;
                s.done[n] = false;
                ++n;
                it = pending.erase(it);
            }
            if (n == 0) {
                if (blocked) break;
                continue;
            }
            tb.n_frames = n;
            tb.total_tiles = tiles;
            tb.tile_begin[n] = tiles;
            tb.epoch = ++s.epoch;
            for (int f = 0; f < n; ++f) {  // outputs prepared on the callers' streams come first
                Request &r = reqs[s.tickets[f]];
                if (r.ready) {
                    cudaStreamWaitEvent(s.stream, r.ready, 0);
                    free_events.push_back(r.ready);  // reusable once the wait is enqueued
                    r.ready = nullptr;
                }
            }
            s.n = n;
            s.remaining = n;
            s.busy = true;
            ++next_batch;
            const fnr_status st = launch(s, key, tiles);
            if (st != FNR_OK) {
                for (int f = 0; f < n; ++f) {
                    auto it = reqs.find(s.tickets[f]);
                    if (it != reqs.end()) complete(it->second, st);
                }
                s.busy = false;
                fatal = st;
                cv_done.notify_all();
            }
            progress = true;
            if (blocked) break;
        }
        return progress;
    }

    void loop() {
        cudaSetDevice(ctx->device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            bool busy = false;
            for (Slot &s : slots) busy |= s.busy;
            if (stop && (pending.empty() || abandon) && !busy) break;
            const bool p1 = poll_locked();
            const bool p2 = admit_locked();
            busy = false;
            for (Slot &s : slots) busy |= s.busy;
            const uint64_t now = now_ns();
            if (p1 || p2) {
                last_activity_ns = now;
                continue;
            }
            // Completion words are polled, not waited on. While work is in flight,
            // and for idle_spin_us after the last activity (requests tend to come
            // in bursts; -1: always), the thread spins; otherwise it sleeps until a
            // submit, and a request arriving then pays the thread's wake-up.
            if (busy || !pending.empty() || spin_forever || now - last_activity_ns < spin_after_ns) {
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            } else {
                cv_sched.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
};

// Request loops still running when the process exits. Their threads poll
// pinned host memory and CUDA events, which the CUDA runtime releases when it
// shuts down at exit; a thread still polling then crashes the process. The
// guard below is constructed at the first loop start, after the runtime has
// initialised, so its destructor runs before the runtime's shutdown (exit
// handlers run in reverse order of registration): it drops the queued
// requests of every live loop, lets the launched batches finish and joins the
// threads. Resources are left to the process's end.
constexpr int kMaxLiveLoops = 256;

struct LiveLoops {
    std::mutex mu;
    Server *sv[kMaxLiveLoops] = {};

    ~LiveLoops() {
        std::lock_guard<std::mutex> g(mu);
        for (Server *&s : sv) {
            if (!s) continue;
            {
                std::lock_guard<std::mutex> l(s->mu);
                s->stop = true;
                s->abandon = true;
            }
            s->cv_sched.notify_all();
            if (s->th.joinable()) s->th.join();
            s = nullptr;
        }
    }
};

static LiveLoops &live_loops() {
    static LiveLoops loops;
    return loops;
}

static void live_add(Server *s) {
    LiveLoops &L = live_loops();
    std::lock_guard<std::mutex> g(L.mu);
    for (Server *&e : L.sv)
        if (!e) {
            e = s;
            return;
        }
}

static void live_remove(Server *s) {
    LiveLoops &L = live_loops();
    std::lock_guard<std::mutex> g(L.mu);
    for (Server *&e : L.sv)
        if (e == s) e = nullptr;
}

static fnr_status server_start(fnr_context *ctx, const fnr_serve_config *cfg_in) {
    fnr_serve_config cfg;
    memset(&cfg, 0, sizeof(cfg));
    if (cfg_in) cfg = *cfg_in;
    if (cfg.queue_capacity <= 0) cfg.queue_capacity = 4096;
    if (cfg.max_batch_requests <= 0) cfg.max_batch_requests = kMaxBatch;
    if (cfg.max_batch_requests > kMaxBatch)
        return fail(FNR_ERR_INVALID_ARG, "max_batch_requests > %d", kMaxBatch);
    if (cfg.max_batch_rays <= 0) cfg.max_batch_rays = int64_t(16) << 20;
    if (cfg.n_slots <= 0) cfg.n_slots = 3;
    if (cfg.n_slots > kMaxSlots) return fail(FNR_ERR_INVALID_ARG, "n_slots > %d", kMaxSlots);
    if (cfg.idle_spin_us < -1) return fail(FNR_ERR_INVALID_ARG, "idle_spin_us %d < -1", cfg.idle_spin_us);
    if (cfg.reserved != 0) return fail(FNR_ERR_INVALID_ARG, "reserved field of fnr_serve_config is not 0");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    Server *sv = new Server();
    sv->ctx = ctx;
    sv->cfg = cfg;
    sv->spin_forever = cfg.idle_spin_us == -1;
    if (cfg.idle_spin_us > 0) sv->spin_after_ns = uint64_t(cfg.idle_spin_us) * 1000u;
    sv->slots.resize(cfg.n_slots);
    fnr_status st = FNR_OK;
    for (Slot &s : sv->slots) {
        if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s.done_ev, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaHostAlloc(reinterpret_cast<void **>(&s.h_table), sizeof(ServeTable), cudaHostAllocDefault)) !=
                cudaSuccess ||
            (e = dev_malloc(&s.d_scratch, sizeof(ServeScratch))) != cudaSuccess ||
            (e = cudaMemsetAsync(s.d_scratch, 0, sizeof(ServeScratch), s.stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s.stream)) != cudaSuccess ||
            (e = cudaHostAlloc(reinterpret_cast<void **>(&s.h_flags), sizeof(uint32_t) * kMaxBatch,
                               cudaHostAllocMapped)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&s.d_flags), s.h_flags, 0)) != cudaSuccess) {
            st = cuda_fail(e, "serving slot setup");
            break;
        }
        memset(s.h_table, 0, sizeof(ServeTable));
        memset(s.h_flags, 0, sizeof(uint32_t) * kMaxBatch);
    }
    if (st != FNR_OK) {
        for (Slot &s : sv->slots) {
            if (s.stream) cudaStreamDestroy(s.stream);
            if (s.done_ev) cudaEventDestroy(s.done_ev);
            if (s.h_table) cudaFreeHost(s.h_table);
            if (s.d_scratch) cudaFree(s.d_scratch);
            if (s.h_flags) cudaFreeHost(s.h_flags);
        }
        delete sv;
        return st;
    }
    live_loops();  // the exit guard exists before the thread does
    sv->th = std::thread([sv] { sv->loop(); });
    live_add(sv);
    ctx->server = sv;
    return FNR_OK;
}

void server_stop(fnr_context *ctx) {
    Server *sv = ctx->server;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
    }
    sv->cv_sched.notify_all();
    live_remove(sv);
    if (sv->th.joinable()) sv->th.join();
    cudaSetDevice(ctx->device);
    for (Slot &s : sv->slots) {
        cudaStreamSynchronize(s.stream);
        for (auto &kv : s.graphs) {
            cudaGraphExecDestroy(kv.second.exec);
            cudaGraphDestroy(kv.second.graph);
        }
        cudaStreamDestroy(s.stream);
        cudaEventDestroy(s.done_ev);
        cudaFreeHost(s.h_table);
        cudaFree(s.d_scratch);
        cudaFreeHost(s.h_flags);
    }
    for (auto &kv : sv->reqs) {
        if (kv.second.status == FNR_ERR_NOT_READY) const_cast<fnr_cache *>(kv.second.req.cache)->inflight.fetch_sub(1);
        if (kv.second.ready) cudaEventDestroy(kv.second.ready);
    }
    for (cudaEvent_t e : sv->free_events) cudaEventDestroy(e);
    delete sv;
    ctx->server = nullptr;
}

static void fill_result(const Request &r, uint64_t ticket, fnr_result *out) {
    if (!out) return;
    out->status = r.status;
    out->reserved = 0;
    out->t_submit_ns = r.t_submit;
    out->t_admit_ns = r.t_admit;
    out->t_done_ns = r.t_done;
    out->n_rays = static_cast<uint64_t>(r.rays);
    out->batch = r.batch;
    out->ticket = ticket;
}

}  // namespace fnr

using namespace fnr;

extern "C" {

fnr_status fnr_serve_start(fnr_context *ctx, const fnr_serve_config *cfg) {
    clear_error();
    if (!ctx) return fail(FNR_ERR_INVALID_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    if (ctx->server) return fail(FNR_ERR_INVALID_ARG, "the request loop is already running");
    return server_start(ctx, cfg);
}

fnr_status fnr_serve_stop(fnr_context *ctx) {
    clear_error();
    if (!ctx) return fail(FNR_ERR_INVALID_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    server_stop(ctx);
    return FNR_OK;
}

fnr_status fnr_submit(fnr_context *ctx, const fnr_request *req, uint64_t *ticket) {
    clear_error();
    if (!ctx || !req || !ticket) return fail(FNR_ERR_INVALID_ARG, "NULL argument");
    *ticket = 0;
    if (!req->cache || !req->rgba_dev) return fail(FNR_ERR_INVALID_ARG, "request needs a cache and an output");
    if (!cache_belongs(ctx, req->cache)) return fail(FNR_ERR_INVALID_ARG, "cache does not belong to this context");
    Request r;
    r.req = *req;
    fnr_status st = make_render_const(&req->params, &r.rc);
    if (st != FNR_OK) return st;
    if (r.rc.flags & FNR_RENDER_VOXELS) return fail(FNR_ERR_UNSUPPORTED, "served requests take uniform samples");
    if ((st = check_camera(&req->camera)) != FNR_OK) return st;
    const int D = req->cache->desc.D;
    r.key = serve_key(req->cache->desc.pos_precision, D, (r.rc.flags & FNR_RENDER_SKIP_EMPTY) != 0u,
                      req->cache->view.layout == FNR_LAYOUT_BRICKS);
    if (!serve_fn(r.key))
        return fail(FNR_ERR_UNSUPPORTED, "served rendering supports D in {1,2,3,4,6,8,12,16}, got %d", D);
    r.rays = int64_t(req->camera.width) * req->camera.height;
    r.tiles = frame_tiles(&req->camera);
    r.bytes = uint64_t(r.rays) * (16u + (req->stats_dev ? 16u : 0u));
    {
        std::lock_guard<std::mutex> g(ctx->serve_mu);
        if (!ctx->server && (st = server_start(ctx, nullptr)) != FNR_OK) return st;
    }
    Server *sv = ctx->server;
    if (ctx->budget && r.bytes > ctx->budget)
        return fail(FNR_ERR_BUDGET, "request output (%llu bytes) exceeds the HBM budget",
                    (unsigned long long)r.bytes);
    {
        std::lock_guard<std::mutex> g(sv->mu);
        if (sv->fatal != FNR_OK) return fail(sv->fatal, "the request loop stopped after a device error");
        if (static_cast<int>(sv->pending.size()) >= sv->cfg.queue_capacity)
            return fail(FNR_ERR_QUEUE_FULL, "request queue is full (%d)", sv->cfg.queue_capacity);
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
        if (!(r.ready = sv->take_event())) return fail(FNR_ERR_CUDA, "request event");
        if ((e = cudaEventRecord(r.ready, reinterpret_cast<cudaStream_t>(req->stream))) != cudaSuccess) {
            sv->free_events.push_back(r.ready);
            return cuda_fail(e, "request event record");
        }
        r.t_submit = now_ns();
        const uint64_t t = sv->next_ticket++;
        const_cast<fnr_cache *>(req->cache)->inflight.fetch_add(1);
        sv->reqs.emplace(t, r);
        sv->pending.push_back(t);
        *ticket = t;
    }
    sv->cv_sched.notify_one();
    return FNR_OK;
}

fnr_status fnr_poll(fnr_context *ctx, uint64_t ticket, fnr_result *out) {
    clear_error();
    if (!ctx || !ctx->server) return fail(FNR_ERR_INVALID_ARG, "no request loop");
    Server *sv = ctx->server;
    std::lock_guard<std::mutex> g(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(FNR_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second.status == FNR_ERR_NOT_READY) sv->poll_locked();
    if (it->second.status == FNR_ERR_NOT_READY) {
        fill_result(it->second, ticket, out);
        return FNR_ERR_NOT_READY;
    }
    fill_result(it->second, ticket, out);
    sv->reqs.erase(it);
    return FNR_OK;
}

fnr_status fnr_wait(fnr_context *ctx, uint64_t ticket, uint32_t timeout_ms, fnr_result *out) {
    clear_error();
    if (!ctx || !ctx->server) return fail(FNR_ERR_INVALID_ARG, "no request loop");
    Server *sv = ctx->server;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(FNR_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    // Poll the completion words directly for a short while (low latency), then sleep.
    const auto spin_until = std::chrono::steady_clock::now() + std::chrono::microseconds(2000);
    while (it->second.status == FNR_ERR_NOT_READY && std::chrono::steady_clock::now() < spin_until &&
           std::chrono::steady_clock::now() < deadline) {
        sv->poll_locked();
        if (it->second.status != FNR_ERR_NOT_READY) break;
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
        it = sv->reqs.find(ticket);
    }
    while (it->second.status == FNR_ERR_NOT_READY) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            it = sv->reqs.find(ticket);
            if (it->second.status != FNR_ERR_NOT_READY) break;
            fill_result(it->second, ticket, out);
            return fail(FNR_ERR_TIMEOUT, "request %llu not done after %u ms", (unsigned long long)ticket,
                        timeout_ms);
        }
        it = sv->reqs.find(ticket);
    }
    fill_result(it->second, ticket, out);
    sv->reqs.erase(it);
    return FNR_OK;
}

}  // extern "C"
