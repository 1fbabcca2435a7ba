// Serving loop: a request queue drained by one host thread that admits
// requests by count and HBM budget, groups every admitted render of one kind
// into a single heterogeneous persistent launch, spreads batches over several
// CUDA streams (new arrivals overlap batches already on the GPU) and completes
// requests from CUDA events.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "vrc_internal.h"

vrc_status stats_launch_with(vrc_ctx *ctx, Cube *c, int32_t nbins, vrc_stats *dev_out, uint64_t *dev_hist,
                             void *partials, cudaStream_t st);
size_t stats_scratch_bytes(vrc_ctx *ctx);
vrc_status validate_raycfg(vrc_ctx *ctx, const vrc_raycfg *rc);
bool camera_is_valid(const vrc_camera &c);

namespace {

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct SReq {
    uint64_t ticket = 0;
    vrc_request r{};
    Cube *cube = nullptr;
    double t_submit = 0, t_launch = 0, t_done = 0;
    double t_wait0 = 0, t_wait1 = 0;   // waiting for the cube to become resident (registered cubes)
    bool loaded_for = false;           // this request triggered the cube's upload
    int32_t path = 0;
    vrc_status status = VRC_OK;
    vrc_stats stats{};
    uint64_t samples = 0;
    bool done = false;
};

struct SBatch {
    std::vector<SReq *> reqs;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    void *dmem = nullptr;      // device scratch (stream-ordered allocation, charged to the budget)
    size_t dbytes = 0;
    void *hmem = nullptr;      // pinned: [vrc_stats x n][samples x n][job-table stage]
    size_t hbytes = 0;
};

}  // namespace

struct Server {
    vrc_ctx *ctx = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<SReq *> queue;
    std::map<uint64_t, SReq *> tickets;
    uint64_t next_ticket = 1;
    std::vector<cudaStream_t> streams;   // render batches (normal priority)
    cudaStream_t urgent = nullptr;        // statistics and small renders (highest priority)
    size_t rr = 0;
    std::vector<SBatch *> running;
    int inflight = 0;
    std::vector<std::pair<void *, size_t>> pinned_free;   // reusable pinned buffers
    std::vector<std::pair<void *, size_t>> pinned_all;
    // batch scratch comes from a pool of its own that keeps freed memory
    // (the default pool returns it at every synchronisation, and mapping it
    // again stalls later allocations)
    cudaMemPool_t pool = nullptr;
    // loader of registered cubes: uploads run on a thread of their own so that
    // admission and completion go on meanwhile
    std::thread loader;
    std::deque<std::pair<Cube *, int64_t>> load_q;   // cube, bytes reserved for it
    std::condition_variable cv_load;
    bool loader_stop = false;                         // set once the serving loop has drained
    cudaStream_t load_stream = nullptr;
    std::map<Cube *, vrc_status> load_err;            // failed uploads, reported to the waiting requests
};

namespace {

void finish_req(Server *S, SReq *q, vrc_status st)
{
    q->status = st;
    q->t_done = now_ms();
    q->done = true;
    if (q->cube) q->cube->refs.fetch_sub(1);
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

void *pinned_take(Server *S, size_t bytes, size_t *got)
{
    for (size_t i = 0; i < S->pinned_free.size(); ++i)
        if (S->pinned_free[i].second >= bytes) {
            auto b = S->pinned_free[i];
            S->pinned_free.erase(S->pinned_free.begin() + i);
            *got = b.second;
            return b.first;
        }
    const size_t sz = std::max<size_t>(bytes, 1 << 16);
    void *p = nullptr;
    if (cudaMallocHost(&p, sz) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    S->pinned_all.push_back({p, sz});
    *got = sz;
    return p;
}

size_t batch_bytes(vrc_ctx *ctx, const std::vector<SReq *> &reqs, bool render)
{
    if (render) {
        std::vector<HetJob> dummy(reqs.size());
        return round256(render_hetero_scratch_bytes(dummy)) + round256(16 * reqs.size());
    }
    size_t per = ((stats_scratch_bytes(ctx) + 255) & ~(size_t)255) + 256;
    size_t b = 0;
    for (SReq *q : reqs) b += per + (q->r.out ? 0 : ((size_t)q->r.nbins * 8 + 255) / 256 * 256);
    return b;
}

// Launch one batch (all renders of one mode/sampling/dtype, or a group of
// statistics requests) on its stream; returns false if scratch does not fit.
bool launch_batch(Server *S, SBatch *B, bool render)
{
    vrc_ctx *ctx = S->ctx;
    B->dbytes = batch_bytes(ctx, B->reqs, render);
    if (inject_fire(ctx, VRC_INJECT_ALLOC)) return false;
    if (ctx->used.load() + (int64_t)B->dbytes > ctx->budget) return false;
    if ((S->pool ? cudaMallocFromPoolAsync(&B->dmem, B->dbytes, S->pool, B->st)
                 : cudaMallocAsync(&B->dmem, B->dbytes, B->st)) != cudaSuccess) {
        cudaGetLastError();
        B->dmem = nullptr;
        return false;
    }
    ctx->used.fetch_add((int64_t)B->dbytes);
    const size_t n = B->reqs.size();
    B->hmem = pinned_take(S, n * (sizeof(vrc_stats) + 16) + render_hetero_stage_bytes(n) + 256, &B->hbytes);
    if (!B->hmem) {
        cudaFreeAsync(B->dmem, B->st);
        ctx->used.fetch_sub((int64_t)B->dbytes);
        B->dmem = nullptr;
        return false;
    }
    const double t = now_ms();
    for (SReq *q : B->reqs) q->t_launch = t;
    vrc_status s = VRC_OK;
    if (render) {
        std::vector<HetJob> jobs;
        for (SReq *q : B->reqs) {
            q->path = q->cube->dtex && q->r.rc.sampling == VRC_TRILINEAR ? VRC_PATH_FUSED : VRC_PATH_FUSED_LDG;
            HetJob j;
            j.cube = q->cube;
            j.cam = q->r.cam;
            j.rc = q->r.rc;
            j.mode = q->r.kind == VRC_REQ_DVR ? 1 : 0;
            j.term = q->r.term_alpha;
            j.tf_host = q->r.tf_rgba;
            j.out = (float *)q->r.out;
            jobs.push_back(j);
        }
        const size_t sbytes = round256(render_hetero_scratch_bytes(jobs));
        unsigned long long *cnt = (unsigned long long *)((char *)B->dmem + sbytes);
        char *hcnt = (char *)B->hmem + n * sizeof(vrc_stats);
        void *stage = (void *)round256((size_t)(hcnt + 16 * n));
        // batches on the normal streams run in slices, so that later arrivals on
        // the urgent stream get SMs between them
        s = render_hetero(ctx, jobs, B->st, B->dmem, sbytes, cnt, stage,
                          B->st == S->urgent ? 0 : render_hetero_slice_items(ctx, jobs));
        if (s == VRC_OK) cudaMemcpyAsync(hcnt, cnt, 16 * n, cudaMemcpyDeviceToHost, B->st);
    } else {
        const size_t per = ((stats_scratch_bytes(ctx) + 255) & ~(size_t)255) + 256;
        char *p = (char *)B->dmem;
        for (size_t i = 0; i < B->reqs.size() && s == VRC_OK; ++i) {
            SReq *q = B->reqs[i];
            vrc_stats *dout = (vrc_stats *)(p + per - 256);
            uint64_t *dhist = (uint64_t *)q->r.out;
            char *next = p + per;
            if (!dhist && q->r.nbins > 0) {
                dhist = (uint64_t *)next;
                next += ((size_t)q->r.nbins * 8 + 255) / 256 * 256;
            }
            s = stats_launch_with(ctx, q->cube, q->r.nbins, dout, dhist, p, B->st);
            if (s == VRC_OK)
                cudaMemcpyAsync((vrc_stats *)B->hmem + i, dout, sizeof(vrc_stats), cudaMemcpyDeviceToHost, B->st);
            p = next;
        }
    }
    cudaEventRecord(B->ev, B->st);
    if (s != VRC_OK) {
        // the launch failed before reaching the GPU: complete the requests with the error
        for (SReq *q : B->reqs) q->status = s;
    }
    return true;
}

void retire(Server *S, SBatch *B, bool render)
{
    vrc_ctx *ctx = S->ctx;
    const double t = now_ms();
    const unsigned long long *cnt =
        (const unsigned long long *)((const char *)B->hmem + B->reqs.size() * sizeof(vrc_stats));
    for (size_t i = 0; i < B->reqs.size(); ++i) {
        SReq *q = B->reqs[i];
        if (q->status == VRC_OK) {
            if (render) {
                q->samples = cnt[2 * i];
            } else {
                q->stats = ((const vrc_stats *)B->hmem)[i];
                if (q->stats.n == 0) q->status = VRC_E_NONFINITE;
            }
        }
        const vrc_status st = q->status;
        finish_req(S, q, st);
        q->t_done = t;
    }
    cudaFreeAsync(B->dmem, B->st);
    ctx->used.fetch_sub((int64_t)B->dbytes);
    S->pinned_free.push_back({B->hmem, B->hbytes});
    cudaEventDestroy(B->ev);
}

void serve_loop(Server *S)
{
    vrc_ctx *ctx = S->ctx;
    cudaSetDevice(ctx->device);
    std::vector<std::pair<SBatch *, bool>> live;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        if (S->queue.empty() && live.empty()) {
            if (S->stop) break;
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            continue;
        }
        // retire finished batches
        bool any_done = false;
        for (size_t i = 0; i < live.size();) {
            if (cudaEventQuery(live[i].first->ev) == cudaSuccess) {
                retire(S, live[i].first, live[i].second);
                S->inflight -= (int)live[i].first->reqs.size();
                delete live[i].first;
                live.erase(live.begin() + i);
                any_done = true;
            } else {
                ++i;
            }
        }
        if (any_done) S->cv_done.notify_all();
        // admit: FIFO, up to max_inflight requests on the GPU
        const int room = ctx->cfg.max_inflight - S->inflight;
        if (room > 0 && !S->queue.empty()) {
            std::vector<SReq *> take, waiting;
            while (!S->queue.empty() && (int)take.size() < room) {
                SReq *q = S->queue.front();
                S->queue.pop_front();
                if (inject_fire(ctx, VRC_INJECT_DROP_REQ)) {
                    finish_req(S, q, VRC_E_INJECTED);
                    any_done = true;
                    continue;
                }
                if (q->cube->managed) {
                    // registered cube: admitted once resident; its upload starts as
                    // soon as the memory it needs fits the budget (idle cubes evicted)
                    std::lock_guard<std::mutex> rl(ctx->res_mu);
                    const int state = q->cube->state.load();
                    if (state != CUBE_RESIDENT) {
                        auto fe = S->load_err.find(q->cube);
                        if (state == CUBE_ABSENT && fe != S->load_err.end()) {
                            finish_req(S, q, fe->second);   // its upload failed
                            any_done = true;
                            continue;
                        }
                        if (q->t_wait0 == 0) q->t_wait0 = now_ms();
                        if (state == CUBE_ABSENT) {
                            const int64_t need = upload_peak_bytes(q->cube);
                            if (need > ctx->budget) {
                                finish_req(S, q, VRC_E_NOMEM);
                                set_err(ctx, VRC_E_NOMEM, "registered cube needs %lld bytes, budget %lld",
                                        (long long)need, (long long)ctx->budget);
                                any_done = true;
                                continue;
                            }
                            if (evict_for(ctx, need, q->cube)) {
                                ctx->reserved += need;
                                q->cube->state.store(CUBE_LOADING);
                                q->loaded_for = true;
                                S->load_q.push_back({q->cube, need});
                                S->cv_load.notify_one();
                            }
                        }
                        waiting.push_back(q);
                        continue;
                    }
                    q->cube->last_use = now_ms();
                    if (q->t_wait0 > 0 && q->t_wait1 == 0) q->t_wait1 = now_ms();
                }
                take.push_back(q);
            }
            // requests whose cube is not resident yet keep their place in the queue
            for (auto it = waiting.rbegin(); it != waiting.rend(); ++it) S->queue.push_front(*it);
            // group: one batch per (mode, sampling, dtype) of renders, one for statistics
            std::map<int, std::vector<SReq *>> groups;
            for (SReq *q : take) {
                const int key = q->r.kind == VRC_REQ_STATS
                                    ? -1
                                    : (q->r.kind * 16 + q->r.rc.sampling * 4 + q->cube->g.dtype);
                groups[key].push_back(q);
            }
            std::vector<SReq *> deferred;
            for (auto &kv : groups) {
                SBatch *B = new SBatch();
                B->reqs = kv.second;
                // statistics and small renders (at most 512 x 512 pixels in the
                // batch) take the urgent stream; larger render batches the others
                int64_t pixels = 0;
                for (SReq *q : B->reqs)
                    if (q->r.kind != VRC_REQ_STATS) pixels += (int64_t)q->r.rc.width * q->r.rc.height;
                const bool urgent = S->urgent && (kv.first < 0 || pixels <= 512 * 512);
                B->st = urgent ? S->urgent : S->streams[S->rr++ % S->streams.size()];
                cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
                lk.unlock();
                const bool ok = launch_batch(S, B, kv.first >= 0);
                lk.lock();
                if (!ok) {
                    cudaEventDestroy(B->ev);
                    if (live.empty()) {
                        // nothing will free memory: fail instead of waiting forever
                        for (SReq *q : B->reqs) finish_req(S, q, VRC_E_NOMEM);
                        any_done = true;
                    } else {
                        deferred.insert(deferred.end(), B->reqs.begin(), B->reqs.end());
                    }
                    delete B;
                    continue;
                }
                S->inflight += (int)B->reqs.size();
                live.push_back({B, kv.first >= 0});
            }
            for (auto it = deferred.rbegin(); it != deferred.rend(); ++it) S->queue.push_front(*it);
            if (any_done) S->cv_done.notify_all();
        }
        // poll the GPU without spinning hard
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
    }
}

// Uploads registered cubes handed over by the admission step.
void load_loop(Server *S)
{
    vrc_ctx *ctx = S->ctx;
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_load.wait(lk, [&] { return S->loader_stop || !S->load_q.empty(); });
        if (S->load_q.empty()) {
            if (S->loader_stop) break;
            continue;
        }
        auto job = S->load_q.front();
        S->load_q.pop_front();
        lk.unlock();
        Cube *c = job.first;
        const vrc_status st = load_registered(ctx, c, S->load_stream);
        {
            std::lock_guard<std::mutex> rl(ctx->res_mu);
            ctx->reserved -= job.second;
            if (st == VRC_OK) {
                ++c->loads;
                c->last_use = now_ms();
            }
            c->state.store(st == VRC_OK ? CUBE_RESIDENT : CUBE_ABSENT);
        }
        lk.lock();
        if (st == VRC_OK) S->load_err.erase(c);
        else S->load_err[c] = st;
        S->cv_work.notify_all();
    }
}

Server *server_get(vrc_ctx *ctx)
{
    std::lock_guard<std::mutex> g(ctx->srv_mu);
    if (!ctx->server) {
        Server *S = new Server();
        S->ctx = ctx;
        cudaSetDevice(ctx->device);
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
            cudaGetLastError();
            least = greatest = 0;
        }
        for (int i = 0; i < ctx->cfg.n_streams; ++i) {
            cudaStream_t st;
            if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, least) != cudaSuccess) {
                cudaGetLastError();
                break;
            }
            S->streams.push_back(st);
        }
        if (cudaStreamCreateWithPriority(&S->urgent, cudaStreamNonBlocking, greatest) != cudaSuccess) {
            cudaGetLastError();
            S->urgent = nullptr;
        }
        if (S->streams.empty()) {
            delete S;
            return nullptr;
        }
        // a device memory pool that keeps up to 1 GiB of freed batch scratch
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        if (cudaMemPoolCreate(&S->pool, &props) == cudaSuccess) {
            uint64_t keep = (uint64_t)1 << 30;
            cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        } else {
            cudaGetLastError();
            S->pool = nullptr;
        }
        // pinned host blocks for the largest batch, one per request that can be
        // in flight: pinned allocations while serving may wait for the device
        {
            const size_t n = (size_t)std::max(ctx->cfg.max_inflight, 1);
            const size_t full = n * (sizeof(vrc_stats) + 16) + render_hetero_stage_bytes(n) + 256;
            for (size_t i = 0; i < n; ++i) {
                void *p = nullptr;
                if (cudaMallocHost(&p, full) != cudaSuccess) {
                    cudaGetLastError();
                    break;
                }
                S->pinned_all.push_back({p, full});
                S->pinned_free.push_back({p, full});
            }
        }
        if (cudaStreamCreateWithFlags(&S->load_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            S->load_stream = nullptr;
        }
        S->th = std::thread(serve_loop, S);
        S->loader = std::thread(load_loop, S);
        ctx->server = S;
    }
    return ctx->server;
}

}  // namespace

void server_stop(vrc_ctx *ctx)
{
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->srv_mu);
        S = ctx->server;
        ctx->server = nullptr;
    }
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->th.join();   // every queued request finishes first (uploads included)
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->loader_stop = true;
    }
    S->cv_load.notify_all();
    S->loader.join();
    if (S->load_stream) cudaStreamDestroy(S->load_stream);
    for (auto &kv : S->tickets) delete kv.second;
    if (S->urgent) S->streams.push_back(S->urgent);
    for (cudaStream_t st : S->streams) cudaStreamSynchronize(st);
    for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
    for (auto &b : S->pinned_all) cudaFreeHost(b.first);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    delete S;
}

extern "C" {

vrc_status vrc_submit(vrc_ctx *ctx, const vrc_request *req, uint64_t *ticket)
{
    if (!ctx || !req || !ticket) return VRC_E_INVAL;
    if (req->kind != VRC_REQ_MIP && req->kind != VRC_REQ_DVR && req->kind != VRC_REQ_STATS)
        return set_err(ctx, VRC_E_INVAL, "bad request kind");
    Cube *c = find_cube(ctx, req->cube_id);
    if (!c) return set_err(ctx, VRC_E_BADID, "unknown cube %lld", (long long)req->cube_id);
    if (c->streamed) return set_err(ctx, VRC_E_UNSUPPORTED, "serving needs resident cubes");
    if (req->kind == VRC_REQ_STATS) {
        if (req->nbins < 0 || req->nbins > 65536) return set_err(ctx, VRC_E_INVAL, "bad nbins");
    } else {
        vrc_status s = validate_raycfg(ctx, &req->rc);
        if (s == VRC_OK) s = validate_step(ctx, c, req->rc.step);
        if (s != VRC_OK) return s;
        if (req->rc.path != VRC_PATH_FUSED) return set_err(ctx, VRC_E_UNSUPPORTED, "serving renders use the fused path");
        if (!camera_is_valid(req->cam)) return set_err(ctx, VRC_E_INVAL, "bad camera");
        if (!req->out) return set_err(ctx, VRC_E_INVAL, "null output image");
        if (req->kind == VRC_REQ_DVR) {
            if (!(req->term_alpha > 0.f)) return set_err(ctx, VRC_E_INVAL, "bad term_alpha");
            for (int i = 0; i < 1024; ++i)
                if (!std::isfinite(req->tf_rgba[i])) return set_err(ctx, VRC_E_INVAL, "tf has non-finite entries");
        }
    }
    Server *S = server_get(ctx);
    if (!S) return set_err(ctx, VRC_E_CUDA, "could not start the serving thread");
    SReq *q = new SReq();
    q->r = *req;
    q->cube = c;
    q->t_submit = now_ms();
    c->refs.fetch_add(1);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q->ticket = S->next_ticket++;
        S->tickets[q->ticket] = q;
        S->queue.push_back(q);
    }
    S->cv_work.notify_one();
    *ticket = q->ticket;
    return VRC_OK;
}

vrc_status vrc_poll(vrc_ctx *ctx, uint64_t ticket, vrc_result *res, int32_t timeout_ms)
{
    if (!ctx || !res) return VRC_E_INVAL;
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->srv_mu);
        S = ctx->server;
    }
    if (!S) return VRC_E_BADID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return VRC_E_BADID;
    SReq *q = it->second;
    if (!q->done) {
        if (timeout_ms == 0) return VRC_PENDING;
        if (timeout_ms < 0) {
            S->cv_done.wait(lk, [&] { return q->done; });
        } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return q->done; })) {
            return VRC_E_TIMEOUT;
        }
    }
    std::memset(res, 0, sizeof(*res));
    res->status = q->status;
    res->stats = q->stats;
    res->queue_ms = q->t_launch > 0 ? q->t_launch - q->t_submit : 0;
    res->latency_ms = q->t_done - q->t_submit;
    res->samples = q->samples;
    res->path = q->path;
    res->memory_wait_ms = q->t_wait0 > 0 ? (q->t_wait1 > 0 ? q->t_wait1 : q->t_done) - q->t_wait0 : 0.0;
    res->cube_loaded = q->loaded_for ? 1 : 0;
    S->tickets.erase(it);
    delete q;
    return VRC_OK;
}

}  // extern "C"
