// Context, memory budget, errors, brick geometry, cube bookkeeping.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <iterator>

#include <cstring>

#include "vrc_internal.h"

vrc_status set_err(vrc_ctx *ctx, vrc_status s, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        ctx->last_error = buf;
    }
    return s;
}

vrc_status cuda_err(vrc_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_err(ctx, VRC_E_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_err(ctx, VRC_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool inject_fire(vrc_ctx *ctx, int32_t what)
{
    std::lock_guard<std::mutex> lk(ctx->inj_mu);
    if (ctx->inj_what != what || ctx->inj_left <= 0) return false;
    if (--ctx->inj_left == 0) {
        ctx->inj_what = VRC_INJECT_NONE;
        return true;
    }
    return false;
}

// Block sizes are rounded (512 B below 1 MiB, 2 MiB above) so that repeated
// allocations of one shape (cube pools, staging, metadata) hit the cache.
static size_t round_block(size_t bytes)
{
    const size_t q = bytes < ((size_t)1 << 20) ? 512 : ((size_t)2 << 20);
    return (bytes + q - 1) / q * q;
}

void destroy_tex_array(const TexArray &a)
{
    if (a.tex) cudaDestroyTextureObject(a.tex);
    if (a.surf) cudaDestroySurfaceObject(a.surf);
    if (a.arr) cudaFreeArray(a.arr);
}

void cache_trim(vrc_ctx *ctx, int64_t keep_bytes)
{
    std::lock_guard<std::mutex> lk(ctx->cache_mu);
    while (ctx->cached.load() > keep_bytes && !ctx->cached_arrays.empty()) {
        auto it = ctx->cached_arrays.begin();
        destroy_tex_array(it->second);
        ctx->cached.fetch_sub(it->second.bytes);
        ctx->cached_arrays.erase(it);
    }
    while (ctx->cached.load() > keep_bytes && !ctx->cached_blocks.empty()) {
        auto it = std::prev(ctx->cached_blocks.end());   // largest first
        cudaFree(it->second);
        ctx->cached.fetch_sub((int64_t)it->first);
        ctx->cached_blocks.erase(it);
    }
}

// Cubes released by vrc_cube_free_async whose event has completed (all of
// them, waiting, if `wait`) give their memory to the cache.
bool reap_pending(vrc_ctx *ctx, bool wait)
{
    std::vector<std::pair<cudaEvent_t, Cube *>> done;
    {
        std::lock_guard<std::mutex> lk(ctx->pend_mu);
        for (auto it = ctx->pending.begin(); it != ctx->pending.end();) {
            const cudaError_t q = wait ? cudaEventSynchronize(it->first) : cudaEventQuery(it->first);
            if (q == cudaErrorNotReady) {
                ++it;
                continue;
            }
            if (q != cudaSuccess) cudaGetLastError();   // a failed stream: its work is over all the same
            done.push_back(*it);
            it = ctx->pending.erase(it);
        }
    }
    for (auto &d : done) {
        cudaEventDestroy(d.first);
        release_cube(ctx, d.second, false);
    }
    return !done.empty();
}

namespace {
constexpr int kStageMax = 8;
struct StageArgs {
    int n;
    uint32_t *dst[kStageMax];
    const uint32_t *src[kStageMax];   // mapped pinned host memory, or null: zero fill
    uint32_t words[kStageMax];
};
__global__ void k_stage(StageArgs a)
{
    for (int i = 0; i < a.n; ++i)
        for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < a.words[i]; w += gridDim.x * blockDim.x)
            a.dst[i][w] = a.src[i] ? a.src[i][w] : 0u;
}

vrc_status slot_alloc(vrc_ctx *ctx, vrc_ctx::PinnedSlot &s, size_t cap)
{
    if (s.p) cudaFreeHost(s.p);
    s.p = s.dp = nullptr;
    s.cap = 0;
    VRC_CK(ctx, cudaHostAlloc((void **)&s.p, cap, cudaHostAllocMapped));
    VRC_CK(ctx, cudaHostGetDevicePointer((void **)&s.dp, s.p, 0));
    s.cap = cap;
    return VRC_OK;
}
}  // namespace

vrc_status stage_h2d(vrc_ctx *ctx, cudaStream_t st, const std::vector<H2DCopy> &copies)
{
    size_t total = 0;
    for (const H2DCopy &c : copies) {
        if (c.bytes % 4) return set_err(ctx, VRC_E_INVAL, "staged copy of %zu bytes", c.bytes);
        if (c.src) total += (c.bytes + 255) & ~(size_t)255;
    }
    std::lock_guard<std::mutex> lk(ctx->stage_mu);
    // a slot whose previous contents have been read (never wait for one: its
    // stream may be held back by work the caller has yet to issue)
    vrc_ctx::PinnedSlot *slot = nullptr;
    for (int k = 0; k < 4 && !slot; ++k) {
        vrc_ctx::PinnedSlot &c = ctx->stage[(ctx->stage_next + k) % 4];
        const cudaError_t q = c.ev ? cudaEventQuery(c.ev) : cudaSuccess;
        if (q == cudaSuccess) {
            slot = &c;
            ctx->stage_next = (ctx->stage_next + k + 1) % 4;
        } else if (q != cudaErrorNotReady) {
            return cuda_err(ctx, q, "staging slot");
        }
    }
    if (!slot) {
        // every slot still in flight: plain copies and fills on `st`
        for (const H2DCopy &c : copies) {
            if (!c.bytes) continue;
            if (c.src) VRC_CK(ctx, cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, st));
            else VRC_CK(ctx, cudaMemsetAsync(c.dst, 0, c.bytes, st));
        }
        return VRC_OK;
    }
    vrc_ctx::PinnedSlot &s = *slot;
    if (!s.ev) VRC_CK(ctx, cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
    if (s.cap < total) {
        const vrc_status r = slot_alloc(ctx, s, std::max<size_t>(total, (size_t)256 << 10));
        if (r != VRC_OK) return r;
    }
    StageArgs a = {};
    size_t off = 0, most = 0;
    for (const H2DCopy &c : copies) {
        if (!c.bytes) continue;
        if (a.n == kStageMax) {
            k_stage<<<(unsigned)std::min<size_t>((most + 1023) / 1024, 256), 256, 0, st>>>(a);
            count_launch(ctx);
            a = StageArgs{};
            most = 0;
        }
        a.dst[a.n] = static_cast<uint32_t *>(c.dst);
        a.src[a.n] = nullptr;
        if (c.src) {
            std::memcpy(s.p + off, c.src, c.bytes);
            a.src[a.n] = reinterpret_cast<const uint32_t *>(s.dp + off);
            off += (c.bytes + 255) & ~(size_t)255;
        }
        a.words[a.n] = (uint32_t)(c.bytes / 4);
        most = std::max(most, c.bytes / 4);
        ++a.n;
    }
    if (a.n) {
        k_stage<<<(unsigned)std::min<size_t>((most + 1023) / 1024, 256), 256, 0, st>>>(a);
        count_launch(ctx);
    }
    VRC_CK(ctx, cudaGetLastError());
    VRC_CK(ctx, cudaEventRecord(s.ev, st));
    return VRC_OK;
}

vrc_status dev_alloc(vrc_ctx *ctx, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return VRC_OK;
    if (inject_fire(ctx, VRC_INJECT_ALLOC)) return set_err(ctx, VRC_E_NOMEM, "injected allocation failure");
    reap_pending(ctx, false);
    const size_t rb = round_block(bytes);
    int64_t prev = ctx->used.fetch_add((int64_t)rb);
    if (prev + (int64_t)rb > ctx->budget) {
        ctx->used.fetch_sub((int64_t)rb);
        // cubes still waiting for their stream hold memory: wait for them once
        if (reap_pending(ctx, true)) return dev_alloc(ctx, p, bytes);
        return set_err(ctx, VRC_E_NOMEM, "HBM budget exceeded: %lld used + %zu requested > %lld",
                       (long long)prev, rb, (long long)ctx->budget);
    }
    {
        std::lock_guard<std::mutex> lk(ctx->cache_mu);
        auto it = ctx->cached_blocks.find(rb);
        if (it != ctx->cached_blocks.end()) {
            *p = it->second;
            ctx->cached_blocks.erase(it);
            ctx->cached.fetch_sub((int64_t)rb);
            return VRC_OK;
        }
    }
    cache_trim(ctx, std::max<int64_t>(0, ctx->budget - ctx->used.load()));
    cudaError_t e = cudaMalloc(p, rb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cache_trim(ctx, 0);   // cached blocks may be what fills the device
        e = cudaMalloc(p, rb);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->used.fetch_sub((int64_t)rb);
        *p = nullptr;
        return cuda_err(ctx, e, "cudaMalloc");
    }
    return VRC_OK;
}

void dev_free(vrc_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    const size_t rb = round_block(bytes);
    {
        std::lock_guard<std::mutex> lk(ctx->cache_mu);
        ctx->cached_blocks.emplace(rb, p);
        ctx->cached.fetch_add((int64_t)rb);
    }
    ctx->used.fetch_sub((int64_t)rb);
}

bool tex_array_take(vrc_ctx *ctx, uint64_t key, TexArray *a)
{
    std::lock_guard<std::mutex> lk(ctx->cache_mu);
    auto it = ctx->cached_arrays.find(key);
    if (it == ctx->cached_arrays.end()) return false;
    *a = it->second;
    ctx->cached.fetch_sub(a->bytes);
    ctx->cached_arrays.erase(it);
    return true;
}

void tex_array_give(vrc_ctx *ctx, uint64_t key, const TexArray &a)
{
    std::lock_guard<std::mutex> lk(ctx->cache_mu);
    ctx->cached_arrays.emplace(key, a);
    ctx->cached.fetch_add(a.bytes);
}

vrc_status scratch_get(vrc_ctx *ctx, size_t bytes, void **p)
{
    if (bytes > ctx->scratch_bytes) {
        if (ctx->scratch) {
            cudaDeviceSynchronize();  // scratch may be in use by earlier launches
            dev_free(ctx, ctx->scratch, ctx->scratch_bytes);
            ctx->scratch = nullptr;
            ctx->scratch_bytes = 0;
        }
        size_t want = bytes + bytes / 4 + (1 << 20);
        vrc_status s = dev_alloc(ctx, &ctx->scratch, want);
        if (s != VRC_OK) return s;
        ctx->scratch_bytes = want;
    }
    *p = ctx->scratch;
    return VRC_OK;
}

Cube *find_cube(vrc_ctx *ctx, int64_t id)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->cubes.find(id);
    return it == ctx->cubes.end() ? nullptr : it->second;
}

bool make_geom(int64_t nx, int64_t ny, int64_t nz, int32_t B, int32_t dtype, BrickGeom *g, int32_t align)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20)) return false;
    if (dtype < 0 || dtype > 2) return false;
    if (B == 0) {
        int64_t m = nx > ny ? nx : ny;
        m = m > nz ? m : nz;
        B = 16;
        while (B < m && B < 256) B <<= 1;
    }
    if (B < 16 || B > 512 || (B & (B - 1))) return false;
    g->dims[0] = nx;
    g->dims[1] = ny;
    g->dims[2] = nz;
    g->B = B;
    g->logB = 0;
    while ((1 << g->logB) < B) ++g->logB;
    g->dtype = dtype;
    g->esize = dtype == VRC_F32 ? 4 : (dtype == VRC_BF16 ? 2 : 1);
    for (int a = 0; a < 3; ++a) g->nb[a] = (int32_t)((g->dims[a] + B - 1) / B);
    g->nbricks = (int64_t)g->nb[0] * g->nb[1] * g->nb[2];
    g->O = align / g->esize;   // the interior of every row starts `align` bytes in
    g->P = B + 2 * g->O;
    g->R = B + 2;
    g->brick_elems = (int64_t)g->P * g->R * g->R;
    g->brick_bytes = g->brick_elems * g->esize;
    return true;
}

// Ray basis in binary64, rounded to binary32 (formula stated in vrc.h).
void camera_basis(const vrc_camera &cam, int W, int H, float basis[12])
{
    double e[3], w[3], r[3], u[3], up[3];
    for (int a = 0; a < 3; ++a) {
        e[a] = cam.eye[a];
        w[a] = (double)cam.center[a] - (double)cam.eye[a];
        up[a] = cam.up[a];
    }
    double lw = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int a = 0; a < 3; ++a) w[a] = w[a] / lw;
    r[0] = w[1] * up[2] - w[2] * up[1];
    r[1] = w[2] * up[0] - w[0] * up[2];
    r[2] = w[0] * up[1] - w[1] * up[0];
    double lr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) r[a] = r[a] / lr;
    u[0] = r[1] * w[2] - r[2] * w[1];
    u[1] = r[2] * w[0] - r[0] * w[2];
    u[2] = r[0] * w[1] - r[1] * w[0];
    double asp = (double)W / (double)H;
    double h = cam.kind == VRC_CAM_PERSP ? std::tan((double)cam.fovy_deg * 3.14159265358979323846 / 360.0)
                                         : 0.5 * (double)cam.ortho_height;
    for (int a = 0; a < 3; ++a) {
        double o0, d0;
        if (cam.kind == VRC_CAM_PERSP) {
            o0 = e[a];
            d0 = w[a] - (h * asp) * r[a] + h * u[a];
        } else {
            o0 = e[a] - (h * asp) * r[a] + h * u[a];
            d0 = w[a];
        }
        basis[a] = (float)o0;
        basis[3 + a] = (float)d0;
        basis[6 + a] = (float)((2.0 * h * asp / (double)W) * r[a]);
        basis[9 + a] = (float)((-2.0 * h / (double)H) * u[a]);
    }
}

extern "C" {

const char *vrc_status_str(vrc_status s)
{
    switch (s) {
    case VRC_OK: return "ok";
    case VRC_PENDING: return "pending";
    case VRC_E_INVAL: return "invalid argument";
    case VRC_E_NOMEM: return "out of memory / over HBM budget";
    case VRC_E_CUDA: return "CUDA error";
    case VRC_E_TIMEOUT: return "timeout";
    case VRC_E_BADID: return "unknown id";
    case VRC_E_BUSY: return "busy";
    case VRC_E_NONFINITE: return "no finite values";
    case VRC_E_INJECTED: return "injected failure";
    case VRC_E_UNSUPPORTED: return "unsupported";
    case VRC_E_SOURCE: return "brick provider failed";
    default: return "unknown status";
    }
}

const char *vrc_last_error(vrc_ctx *ctx)
{
    static thread_local std::string copy;
    if (!ctx) return "";
    std::lock_guard<std::mutex> lk(ctx->err_mu);
    copy = ctx->last_error;
    return copy.c_str();
}

vrc_status vrc_create(vrc_ctx **out, const vrc_config *cfg)
{
    if (!out) return VRC_E_INVAL;
    *out = nullptr;
    vrc_config c{};
    if (cfg) c = *cfg;
    if (c.n_streams < 0 || c.max_inflight < 0 || c.hbm_budget_bytes < 0) return VRC_E_INVAL;
    if (c.n_streams == 0) c.n_streams = 4;
    if (c.max_inflight == 0) c.max_inflight = 32;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        return VRC_E_CUDA;
    }
    if (c.device < 0 || c.device >= ndev) return VRC_E_INVAL;
    if (cudaSetDevice(c.device) != cudaSuccess) return VRC_E_CUDA;
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) return VRC_E_CUDA;
    vrc_ctx *ctx = new (std::nothrow) vrc_ctx();
    if (!ctx) return VRC_E_NOMEM;
    ctx->device = c.device;
    ctx->cfg = c;
    ctx->budget = c.hbm_budget_bytes ? c.hbm_budget_bytes : (int64_t)(0.9 * (double)freeb);
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, c.device);
    if (cudaHostAlloc(&ctx->h_samples, 4 * sizeof(unsigned long long), cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_samples, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->h_samples) cudaFreeHost(ctx->h_samples);
        delete ctx;
        return VRC_E_CUDA;
    }
    ctx->h_samples[0] = ctx->h_samples[1] = ctx->h_samples[2] = 0;
    // pinned staging slots now: allocating pinned memory later may wait for the device
    for (vrc_ctx::PinnedSlot &sl : ctx->stage) {
        if (slot_alloc(ctx, sl, (size_t)256 << 10) != VRC_OK ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            vrc_destroy(ctx);
            return VRC_E_CUDA;
        }
    }
    *out = ctx;
    return VRC_OK;
}

vrc_status vrc_destroy(vrc_ctx *ctx)
{
    if (!ctx) return VRC_E_INVAL;
    cudaSetDevice(ctx->device);
    server_stop(ctx);
    cudaDeviceSynchronize();
    reap_pending(ctx, true);
    std::vector<int64_t> ids;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (auto &kv : ctx->cubes) ids.push_back(kv.first);
    }
    for (int64_t id : ids) vrc_cube_free(ctx, id);
    if (ctx->scratch) dev_free(ctx, ctx->scratch, ctx->scratch_bytes);
    cudaDeviceSynchronize();
    cache_trim(ctx, 0);
    for (vrc_ctx::PinnedSlot &sl : ctx->stage) {
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.p) cudaFreeHost(sl.p);
    }
    if (ctx->ev_samples) cudaEventDestroy(ctx->ev_samples);
    if (ctx->h_samples) cudaFreeHost(ctx->h_samples);
    delete ctx;
    return VRC_OK;
}

vrc_status vrc_memory(vrc_ctx *ctx, int64_t *used_bytes, int64_t *budget_bytes)
{
    if (!ctx) return VRC_E_INVAL;
    if (used_bytes) *used_bytes = ctx->used.load();
    if (budget_bytes) *budget_bytes = ctx->budget;
    return VRC_OK;
}

vrc_status vrc_debug_inject(vrc_ctx *ctx, int32_t what, int64_t nth)
{
    if (!ctx || what < 0 || what > VRC_INJECT_SLAB_WAIT || (what != VRC_INJECT_NONE && nth < 1)) return VRC_E_INVAL;
    std::lock_guard<std::mutex> lk(ctx->inj_mu);
    ctx->inj_what = what;
    ctx->inj_left = what == VRC_INJECT_NONE ? 0 : nth;
    return VRC_OK;
}

uint64_t vrc_launch_count(vrc_ctx *ctx) { return ctx ? ctx->launches.load() : 0; }

vrc_status vrc_last_render_samples(vrc_ctx *ctx, uint64_t *samples, uint64_t *evaluated)
{
    if (!ctx || !samples) return VRC_E_INVAL;
    VRC_CK(ctx, cudaEventSynchronize(ctx->ev_samples));
    *samples = ctx->h_samples[0];
    if (evaluated) *evaluated = ctx->h_samples[1];
    if (ctx->h_samples[2]) return set_err(ctx, VRC_E_TIMEOUT, "a device-side wait of the last render gave up");
    return VRC_OK;
}

vrc_status vrc_last_render_bricks(vrc_ctx *ctx, int64_t *traversed, int64_t *culled)
{
    if (!ctx || !traversed || !culled) return VRC_E_INVAL;
    *traversed = ctx->last_bricks[0].load();
    *culled = ctx->last_bricks[1].load();
    return VRC_OK;
}

}  // extern "C"
