// Statistics without any device allocation.
//
// Who needs this: callers that must not allocate device memory when they ask
// for a statistic.  Typical cases are an interactive or serving loop with a
// latency budget (cudaMalloc and cudaFree can synchronise the whole device and
// stall every stream), a plug-in living inside a host application that has
// reserved the device memory for its own pool, and programs whose policy is to
// allocate only at start-up.  vrc_cube_stats_async may grow the context's
// scratch buffer with cudaMalloc; this entry point never does.
//
// How: the block partials of the statistics pass live in one file-scope
// device array of fixed size, shared by every call in the process.  Its device
// address is looked up once per device (host code may not use the array's
// name as an address).  The caller owns the inputs (the resident cube) and
// the outputs (device vrc_stats record and histogram), as with
// vrc_cube_stats_async.
#include <mutex>

#include "vrc_internal.h"

vrc_status stats_launch_with(vrc_ctx *ctx, Cube *c, int32_t nbins, vrc_stats *dev_out, uint64_t *dev_hist,
                             void *partials, cudaStream_t st);
size_t stats_scratch_bytes(vrc_ctx *ctx);

namespace {

constexpr size_t kNoAllocScratchBytes = 64 << 10;   // 64 KiB, held by every device that loads the library
constexpr int kMaxDevices = 64;

// Block partials of the statistics pass.  Nothing here has to start at zero:
// each launch writes every partial slot before its final merge reads it.
static __device__ __align__(256) unsigned char g_stats_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_stats_scratch on `device` (which must be current).
vrc_status scratch_address(vrc_ctx *ctx, void **out)
{
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return set_err(ctx, VRC_E_INVAL, "device ordinal too large");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[ctx->device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_stats_scratch);
        if (e != cudaSuccess || !p) return cuda_err(ctx, e, "cudaGetSymbolAddress(static statistics scratch)");
        g_addr[ctx->device] = p;
    }
    *out = g_addr[ctx->device];
    return VRC_OK;
}

}  // namespace

extern "C" vrc_status vrc_cube_stats_noalloc(vrc_ctx *ctx, int64_t cube_id, int32_t nbins, vrc_stats *dev_out,
                                             uint64_t *dev_hist, void *stream)
{
    if (!ctx) return VRC_E_INVAL;
    if (nbins < 0 || nbins > 65536) return set_err(ctx, VRC_E_INVAL, "nbins must be in [0, 65536]");
    if (!dev_out || (nbins > 0 && !dev_hist)) return set_err(ctx, VRC_E_INVAL, "null output");
    Cube *c = nullptr;
    CubeUse use;   // held for the call: a registered cube is not evicted meanwhile
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->cubes.find(cube_id);
        if (it == ctx->cubes.end()) return set_err(ctx, VRC_E_BADID, "unknown cube %lld", (long long)cube_id);
        c = it->second;
        c->refs.fetch_add(1);
    }
    use.c = c;
    if (c->streamed) return set_err(ctx, VRC_E_UNSUPPORTED, "statistics need a resident cube");
    // making a registered cube resident would allocate
    if (c->managed && c->state.load() != CUBE_RESIDENT)
        return set_err(ctx, VRC_E_UNSUPPORTED, "registered cube %lld is not resident", (long long)cube_id);
    const size_t need = stats_scratch_bytes(ctx);
    if (need > kNoAllocScratchBytes)
        return set_err(ctx, VRC_E_NOMEM, "the statistics pass needs %zu bytes of scratch on this device; the static "
                       "array holds %zu", need, kNoAllocScratchBytes);
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    void *scratch = nullptr;
    vrc_status s = scratch_address(ctx, &scratch);
    if (s != VRC_OK) return s;
    return stats_launch_with(ctx, c, nbins, dev_out, dev_hist, scratch, (cudaStream_t)stream);
}
