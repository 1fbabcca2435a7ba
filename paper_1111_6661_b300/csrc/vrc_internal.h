// Internal declarations of the cube ray-casting / statistics library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/vrc.h"

// ------------------------------------------------------------------ brick store
//
// A cube of dims (nx, ny, nz) is stored as nb[0] x nb[1] x nb[2] bricks of edge
// B (power of two).  Brick (bx, by, bz) has index (bz*nb[1] + by)*nb[0] + bx and
// stores local voxels l in [-1, B] on each axis (a one-voxel halo; positions
// outside the cube hold the clamp-to-edge value).  Memory layout of one brick,
// in elements of the stored type (esize bytes):
//   slice z (R = B+2 slices), row y (R rows per slice), row pitch P elements;
//   local voxel (lx, ly, lz) sits at ((lz+1)*R + (ly+1))*P + (lx + O),
//   O = 16/esize, P = B + 2*O, so every interior row starts 16-byte aligned and
//   the halo voxels lx = -1 and lx = B sit at O-1 and O+B.
struct BrickGeom {
    int64_t dims[3];
    int32_t B, logB, dtype, esize;
    int32_t nb[3];
    int64_t nbricks;
    int32_t O, P, R;
    int64_t brick_elems, brick_bytes;
};

// Brick geometry.  Rows hold P = B + 2*O elements: O - 1 padding elements,
// the halo voxel, B interior voxels, the halo voxel, O - 1 padding elements,
// with O * esize = align bytes (32 for resident bricks, so that interior rows
// start on 32-byte sectors; 16 for streamed bricks, which cross the host link).
bool make_geom(int64_t nx, int64_t ny, int64_t nz, int32_t B, int32_t dtype, BrickGeom *g, int32_t align);

struct vrc_ctx;

// One brick's render copy: a layered CUDA array with the surface used to fill
// it and the point-sampled texture object that reads it.
struct TexArray {
    cudaArray_t arr = nullptr;
    cudaSurfaceObject_t surf = 0;
    cudaTextureObject_t tex = 0;
    int64_t bytes = 0;
};

struct Cube {
    int64_t id = 0;
    BrickGeom g{};
    bool streamed = false;
    void *pool = nullptr;         // device bricks (resident cubes)
    float *scales = nullptr;      // device [nbricks] (1 unless FP8)
    float *bmin = nullptr;        // device [nbricks] stored interior min (finite values)
    float *bmax = nullptr;        // device [nbricks] stored interior max
    int32_t *bnonfinite = nullptr;// device [nbricks] non-finite interior voxels
    std::vector<float> h_bmin, h_bmax;
    std::vector<int32_t> h_bnonfinite;
    // largest stored value a sample of brick b can read (interior plus halo;
    // NaN ignored, +inf kept): bricks at or below the transparent threshold of a
    // transfer function are culled from sort-last renders
    std::vector<float> h_bhalo_max;
    float *bhalo = nullptr;       // device [nbricks]: the same maxima (filled at upload)
    float vmin = 0.f, vmax = 0.f; // stored extrema over finite voxels
    float shift = 0.f;            // approximate mean (upload pass): centres the statistics sums
    bool has_finite = false;
    int64_t charged = 0;          // bytes charged to the budget
    // out-of-core
    void *host_pool = nullptr;    // pinned and mapped, n_host slots of brick_bytes
    void *host_pool_dev = nullptr;// device address of host_pool (zero-copy reads)
    int64_t n_host = 0;
    int32_t ring = 0;
    void *ring_pool = nullptr;    // device, ring slots
    std::vector<uint8_t> host_filled;
    int64_t n_filled = 0;         // host slots written at least once
    // out-of-core cubes with a brick provider: host slot s caches brick
    // slot_brick[s] (-1: none); slot_ev[s] follows the last copy out of slot s
    vrc_brick_source_fn source = nullptr;
    void *source_user = nullptr;
    std::vector<int64_t> slot_brick;
    std::vector<cudaEvent_t> slot_ev;
    std::vector<uint8_t> slot_ev_live;
    std::vector<float> source_buf;      // (B+2)^3 floats handed to the provider
    // bf16 / fp8 provider cubes: a provided brick is packed on the device
    // (pack_src: its (B+2)^3 floats, pack_out: the stored brick) on pack_stream
    // and copied back into its host slot; brick scales in h_scales
    void *pack_src = nullptr, *pack_out = nullptr;
    cudaStream_t pack_stream = nullptr;
    bool source_pinned = false;         // source_buf page-locked (unlocked at release)
    uint64_t source_calls = 0;          // provider calls since creation
    std::vector<double> h_bsum;         // per brick: sum and count of its finite interior values
    std::vector<int64_t> h_bcnt;
    // render copies of the bricks as 2D layered CUDA arrays (layers along z),
    // read by texture gathers (2x2 texel footprints) in the fused renderer
    std::vector<TexArray> tex_arrays;
    std::vector<unsigned long long> h_tex;   // texture handles staged for the device table
    unsigned long long *dtex = nullptr;   // device [4][nbricks]: texture handles by layer axis (0 where absent), then surfaces
    int32_t tex_axes = 0;                 // bit a set: copy layered along axis a exists (only z is built)
    int64_t tex_bytes = 0;
    // maximum stored value of every 8^3 macro-cell plus a one-voxel margin,
    // read from the brick that owns the cell (empty-space skipping)
    float *cellmax = nullptr;
    int32_t ncell[3] = {0, 0, 0};
    // slab renderer (float32 resident cubes): clamp-to-edge halo copy, dims + 2 on
    // every axis, rows of halo_pitch elements, and its three TMA tensor maps
    float *halo = nullptr;
    int64_t halo_bytes = 0, halo_pitch = 0;
    alignas(64) unsigned char slab_maps[3 * 128];
    // tuning (0 = default)
    int32_t tile_w = 0, tile_h = 0, ctas_per_sm = 0;
    std::atomic<int> refs{0};     // queued or running requests and direct calls using the cube
    // render copy: VRC_COPY_AUTO, VRC_COPY_REQUIRED or VRC_COPY_NONE
    int32_t copy_mode = 0;
    // registered cubes (vrc_cube_register): voxels stay in the caller's host
    // memory; the library makes the cube resident when it is needed and evicts
    // it (least recently used, when no request or call holds it) to make room
    bool managed = false;
    const float *host_src = nullptr;
    bool host_pinned = false;     // host_src was page-locked by the registration (unlocked at release)
    // bf16 / fp8 registered cubes: the packed bricks (nbricks x brick_bytes)
    // and brick scales, kept in page-locked host memory from the registration
    // on; loads copy these instead of packing the source again
    void *host_packed = nullptr;
    std::vector<float> h_scales;
    std::atomic<int> state{2};    // CUBE_ABSENT, CUBE_LOADING, CUBE_RESIDENT
    double last_use = 0;          // host ms of the last admission or direct use
    bool direct_used = false;     // work of direct calls may be in flight: evictions wait for the device
    uint64_t loads = 0;           // uploads of this cube so far
};
constexpr int CUBE_ABSENT = 0, CUBE_LOADING = 1, CUBE_RESIDENT = 2;

struct Server;  // serving loop (serve.cu)

struct vrc_ctx {
    int device = 0;
    vrc_config cfg{};
    int sm_count = 148;
    int64_t budget = 0;
    std::atomic<int64_t> used{0};
    std::mutex mu;
    std::map<int64_t, Cube *> cubes;
    int64_t next_id = 1;
    std::string last_error;
    std::mutex err_mu;            // last_error is written by the serving thread too
    std::atomic<uint64_t> launches{0};
    // scratch reused by statistics / rendering (grown on demand)
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    // host fault injection
    std::mutex inj_mu;
    int32_t inj_what = VRC_INJECT_NONE;
    int64_t inj_left = 0;
    Server *server = nullptr;
    std::mutex srv_mu;
    // sample counts of the last render: [lattice, evaluated, device-wait failure]
    // (pinned host words + completion event)
    unsigned long long *h_samples = nullptr;
    cudaEvent_t ev_samples = nullptr;
    // sort-last brick counts of the last render: [traversed, culled] (host)
    std::atomic<int64_t> last_bricks[2] = {{0}, {0}};
    // caching allocator: device blocks and texture arrays released by freed
    // cubes and scratch, reused by later allocations of the same size.  `used`
    // counts live bytes; live + cached bytes never exceed the budget.
    std::mutex cache_mu;
    std::multimap<size_t, void *> cached_blocks;       // rounded size -> block
    std::multimap<uint64_t, TexArray> cached_arrays;   // tex_array_key -> array
    std::atomic<int64_t> cached{0};
    // cubes released by vrc_cube_free_async: their memory goes to the cache once
    // the event recorded on the caller's stream has completed
    std::mutex pend_mu;
    std::vector<std::pair<cudaEvent_t, Cube *>> pending;
    // residency of registered cubes: state changes and evictions
    std::mutex res_mu;
    int64_t reserved = 0;         // bytes promised to uploads in progress (serving loader)
    std::atomic<uint64_t> evictions{0};
    // path of the most recent render (VRC_PATH_*)
    std::atomic<int32_t> last_path{0};
    // pinned staging slots for small host-to-device inputs (stage_h2d)
    std::mutex stage_mu;
    struct PinnedSlot {
        char *p = nullptr;        // pinned, mapped host memory
        char *dp = nullptr;       // its device address
        size_t cap = 0;
        cudaEvent_t ev = nullptr;
    } stage[4];
    int stage_next = 0;
};

// One host-to-device copy of a small input (transfer function, job table, work
// items), or a zero fill when src is null; bytes a multiple of 4.  stage_h2d
// copies the sources into a pinned, mapped slot whose previous contents have
// been read and one small kernel on `st` moves them to the device.  The copy
// engines are not used: a copy from pageable memory waited 36 ms behind a 1 GB
// image download, and a copy from pinned memory at times waited 78 ms behind a
// cube's 4.3 GB upload.  With all four slots still in flight it falls back to
// plain copies and fills on `st` instead of waiting for a slot.
struct H2DCopy {
    void *dst;
    const void *src;
    size_t bytes;
};
vrc_status stage_h2d(vrc_ctx *ctx, cudaStream_t st, const std::vector<H2DCopy> &copies);

// ------------------------------------------------------------------ helpers
vrc_status set_err(vrc_ctx *ctx, vrc_status s, const char *fmt, ...);
vrc_status cuda_err(vrc_ctx *ctx, cudaError_t e, const char *what);
bool inject_fire(vrc_ctx *ctx, int32_t what);
vrc_status dev_alloc(vrc_ctx *ctx, void **p, size_t bytes);
void dev_free(vrc_ctx *ctx, void *p, size_t bytes);   // the block must be idle (no work in flight uses it)
bool tex_array_take(vrc_ctx *ctx, uint64_t key, TexArray *a);
void tex_array_give(vrc_ctx *ctx, uint64_t key, const TexArray &a);   // idle arrays only
void cache_trim(vrc_ctx *ctx, int64_t keep_bytes);                     // release cached memory down to keep_bytes
bool reap_pending(vrc_ctx *ctx, bool wait);   // release completed (wait: all) async-freed cubes; true if any
void destroy_tex_array(const TexArray &a);
vrc_status scratch_get(vrc_ctx *ctx, size_t bytes, void **p);
Cube *find_cube(vrc_ctx *ctx, int64_t id);
vrc_status validate_step(vrc_ctx *ctx, const Cube *c, float step);   // at most 2^22 samples per ray
inline void count_launch(vrc_ctx *ctx, uint64_t n = 1) { ctx->launches.fetch_add(n); }

#define VRC_CK(ctx, call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call); \
    } while (0)

// ------------------------------------------------------------------ rendering
// Per-view ray basis (binary32) as defined in vrc.h.
struct ViewParams {
    float O0[3], D0[3], DX[3], DY[3];
    int32_t kind, W, H;
    int32_t ec[3];          // eye brick cell for the visibility order
    int32_t tex_axis;       // layer axis of the texture copy this view reads
    int64_t out_offset;     // element offset of the view's image (pixels)
};
void camera_basis(const vrc_camera &cam, int W, int H, float basis[12]);

// Statistics launch (stats.cu), used by the serving loop too.
vrc_status stats_launch(vrc_ctx *ctx, Cube *c, int32_t nbins, vrc_stats *dev_out, uint64_t *dev_hist,
                        cudaStream_t st);

// Heterogeneous persistent render launch (render.cu), used by the serving loop.
struct HetJob {             // one request inside a heterogeneous launch
    Cube *cube;
    vrc_camera cam;
    vrc_raycfg rc;
    int32_t mode;           // 0 MIP, 1 DVR
    float term;
    const float *tf_host;   // 1024 floats (DVR)
    float *out;             // device image
};
vrc_status render_hetero(vrc_ctx *ctx, const std::vector<HetJob> &jobs, cudaStream_t st, void *scratch,
                         size_t scratch_bytes, unsigned long long *dev_samples, void *host_stage, int64_t slice_items);
int64_t render_hetero_slice_items(vrc_ctx *ctx, const std::vector<HetJob> &jobs);
size_t render_hetero_scratch_bytes(const std::vector<HetJob> &jobs);
size_t render_hetero_stage_bytes(size_t n_jobs);

void server_stop(vrc_ctx *ctx);

// Resident cubes (pack.cu).  upload_cube runs the upload passes into a cube
// record whose geometry and render-copy mode are set; release_device gives
// back its device memory (the record stays).
vrc_status upload_cube(vrc_ctx *ctx, Cube *c, const float *src, int32_t src_on_device, cudaStream_t st);
// Make a registered cube resident: from its packed host copy when it has one,
// else by the upload passes on the caller's array.
vrc_status load_registered(vrc_ctx *ctx, Cube *c, cudaStream_t st);
void release_device(vrc_ctx *ctx, Cube *c, bool sync);
void release_cube(vrc_ctx *ctx, Cube *c, bool sync);
int64_t register_cube(vrc_ctx *ctx, Cube *c);
// Stored values of a resident cube into dst (device, nx*ny*nz floats, x fastest).
vrc_status unpack_cube(vrc_ctx *ctx, const Cube *c, float *dst, cudaStream_t st);
// Device bytes a registered cube needs while its upload runs (bricks,
// metadata, render copy, staging of the source, scratch reserve).
int64_t upload_peak_bytes(const Cube *c);
// Evict idle registered cubes (no references, least recently used first)
// until `need` more bytes fit the budget beside the reservations; true if
// they fit.  Caller holds ctx->res_mu.
bool evict_for(vrc_ctx *ctx, int64_t need, const Cube *keep);
double host_ms();

// A cube held by a direct call: it is not evicted while the call runs.
struct CubeUse {
    Cube *c = nullptr;
    CubeUse() = default;
    CubeUse(const CubeUse &) = delete;
    ~CubeUse()
    {
        if (c) c->refs.fetch_sub(1);
    }
};
// Look up a cube for a direct call, hold it, and make a registered cube
// resident (uploading it on `st`, evicting idle registered cubes first).
vrc_status acquire_cube(vrc_ctx *ctx, int64_t id, cudaStream_t st, Cube **out, CubeUse &use);

// Out-of-core cubes (pack.cu).  host_brick makes host slot brick % n_host hold
// brick `brick` (calling the provider when another brick is there, after the
// slot's previous copy has completed) and returns the slot; host_copied
// records, on `st`, the end of a copy out of that slot.
vrc_status host_brick(vrc_ctx *ctx, Cube *c, int64_t brick, int64_t *slot);
vrc_status host_copied(vrc_ctx *ctx, Cube *c, int64_t slot, cudaStream_t st);
// Copy bricks [b0, b0 + n) of an out-of-core cube into consecutive device ring
// slots starting at ring slot `first` (copy stream cs, after `after`); records
// `done` on cs when the copies are complete.
vrc_status ring_load(vrc_ctx *ctx, Cube *c, int64_t b0, int64_t n, int first, cudaStream_t cs, cudaEvent_t done);

// Slab renderer (slab.cu).
struct JobDesc;
bool slab_supported(const Cube *c);
vrc_status slab_prepare(vrc_ctx *ctx, Cube *c, cudaStream_t st);
void slab_release(vrc_ctx *ctx, Cube *c);
int slab_occupancy(int mode);
void slab_launch(const Cube *c, int mode, int grid, cudaStream_t st, const JobDesc *jobs, int n_jobs, int64_t total,
                 int *counter, int *err, bool withhold);
