/*
 * vrc.h -- C ABI of the B300 cube ray-casting and statistics library.
 *
 * The paper (Hassan, Fluke, Barnes) offers, as a service, analysis and
 * visualisation of spectral data cubes larger than one machine's memory:
 * minimum/maximum and histograms (Abstract), standard deviation and median as
 * global multi-pass tasks (Sec. 3), and interactive volume rendering of cubes
 * split into sub-cubes whose partial images are gathered (Sec. 2, Table 1),
 * with CUDA streams overlapping computation and I/O (Sec. 2) and multi-user
 * on-demand sharing (Abstract, Sec. 3).  This library is the single-GPU hot
 * path of that service.  All work runs in hand-written CUDA kernels for
 * sm_103a; the host side only validates, plans and launches.
 *
 * Conventions used by every entry point
 *   - A cube has dims (nx, ny, nz), x fastest: voxel (i, j, k) is element
 *     (k*ny + j)*nx + i of a linear source array and has its centre at
 *     (i+0.5, j+0.5, k+0.5) in the continuous domain [0,nx]x[0,ny]x[0,nz].
 *   - Images are row-major, row 0 at the top: pixel (px, py) of view v is
 *     element (v*H + py)*W + px (MIP: one float; DVR: four floats, RGBA,
 *     premultiplied).
 *   - Device pointers are plain CUDA device addresses in the context's device;
 *     streams are cudaStream_t values passed as void* (NULL = legacy stream).
 *   - No call aborts, throws or exits: every failure is a negative status.
 *     Arguments are validated before anything is launched; on an error return
 *     caller-owned outputs are left unspecified.
 *   - Ownership: the library owns cube storage, brick pools and scratch; the
 *     caller owns every output buffer it passes in.
 *   - Thread safety: one context may be used from one thread at a time, except
 *     vrc_submit / vrc_poll, which may be called from any thread.
 */
#ifndef VRC_H
#define VRC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t vrc_status;
#define VRC_OK            0
#define VRC_PENDING       1   /* vrc_poll: request not finished yet */
#define VRC_E_INVAL      -1   /* bad argument (null pointer, size, enum, unknown flag) */
#define VRC_E_NOMEM      -2   /* HBM budget exceeded or allocation failed */
#define VRC_E_CUDA       -3   /* a CUDA runtime call failed; vrc_last_error() has text */
#define VRC_E_TIMEOUT    -4   /* vrc_poll timed out (request is still pending), or a
                                 bounded device-side wait gave up */
#define VRC_E_BADID      -5   /* unknown cube id, ticket or graph handle */
#define VRC_E_BUSY       -6   /* cube still referenced by queued or running requests */
#define VRC_E_NONFINITE  -7   /* statistic undefined: the cube has no finite voxel */
#define VRC_E_INJECTED   -8   /* failure produced by vrc_debug_inject (tests) */
#define VRC_E_UNSUPPORTED -9  /* operation not available for this cube kind / dtype */
#define VRC_E_SOURCE     -10  /* the brick provider of an out-of-core cube reported a failure */

typedef enum { VRC_F32 = 0, VRC_BF16 = 1, VRC_FP8E4M3 = 2 } vrc_dtype;

typedef struct vrc_ctx vrc_ctx;

typedef struct {
    int32_t device;            /* CUDA device ordinal */
    int32_t n_streams;         /* serving: streams requests are spread over (0 = 4) */
    int32_t max_inflight;      /* serving: requests on the GPU at once (0 = 32) */
    int32_t reserved0;
    int64_t hbm_budget_bytes;  /* cube storage + scratch cap; 0 = 90% of free memory */
} vrc_config;

/* Statistics of the finite voxel values (stored values for BF16/FP8 cubes). */
typedef struct {
    double min, max, mean, std;  /* std is the population deviation (divide by n) */
    uint64_t n, n_nonfinite;
} vrc_stats;

#define VRC_CAM_ORTHO 0
#define VRC_CAM_PERSP 1
typedef struct {
    int32_t kind;              /* VRC_CAM_ORTHO or VRC_CAM_PERSP */
    float eye[3], center[3], up[3];
    float fovy_deg;            /* perspective: full vertical field of view (degrees) */
    float ortho_height;        /* orthographic: image-plane height (voxel units) */
} vrc_camera;

#define VRC_NEAREST   0
#define VRC_TRILINEAR 1
#define VRC_PATH_FUSED    0    /* one thread per ray walks every brick in ray order;
                                  trilinear samples through texture gathers */
#define VRC_PATH_SORTLAST 1    /* per-brick partial images, composited in visibility order */
#define VRC_PATH_FUSED_LDG 2   /* fused, trilinear samples by 8 global loads (no textures) */
#define VRC_PATH_ZEROCOPY  3   /* streamed cubes: the sort-last kernels read the bricks in place
                                  from mapped pinned host memory (no copies, no device ring) */
#define VRC_PATH_SLAB      4   /* resident float32 cubes, trilinear: each 16x16 ray tile marches
                                  through the cube in slabs; the region its samples touch is
                                  staged in shared memory by TMA from a clamp-to-edge copy of
                                  the cube (built on first use, counted against the budget).
                                  Same image as VRC_PATH_FUSED, bit for bit */
typedef struct {
    int32_t width, height;     /* image size in pixels (1..16384) */
    float step;                /* sample spacing along the unit ray, voxel units (> 0, and
                                  at least the cube's diagonal / 2^22: VRC_E_INVAL below) */
    int32_t sampling;          /* VRC_NEAREST or VRC_TRILINEAR */
    int32_t opacity_correction;/* DVR: 0 = alpha as in the transfer function,
                                  1 = 1-(1-alpha)^step */
    int32_t path;              /* VRC_PATH_FUSED, VRC_PATH_SORTLAST, VRC_PATH_FUSED_LDG,
                                  VRC_PATH_ZEROCOPY (streamed cubes only) or VRC_PATH_SLAB */
    int32_t tile_w, tile_h;    /* ray tile; 0,0 = tuned default.  tile_w*tile_h = 256,
                                  tile_w in {8,16,32} */
    int32_t skip_empty;        /* 1 = skip work that cannot change the image; the
                                  image is identical.  Fused trilinear path: skip
                                  samples whose 8^3 macro-cell maximum is transparent
                                  under the transfer function (DVR) or cannot raise
                                  the ray's max (MIP).  Sort-last paths (DVR): cull
                                  whole bricks whose maximum, halo included, is
                                  transparent; a streamed cube then copies fewer
                                  bricks.  0 = sample everything */
    int32_t reserved;          /* must be 0 */
} vrc_raycfg;

/*
 * Ray geometry (both renderers; the fixed formula makes sample positions,
 * sample counts and voxel choices reproducible).  From the camera, in binary64
 * and then rounded to binary32:
 *   w = normalise(center - eye); r = normalise(w x up); u = r x w; asp = W/H
 *   perspective:  h = tan(fovy/2);      O0 = eye,  D0 = w - (h asp) r + h u
 *   orthographic: h = ortho_height/2;  O0 = eye - (h asp) r + h u,  D0 = w
 *   DX = (2 h asp / W) r,  DY = (-2 h / H) u
 * Per pixel, in binary32 with every operation rounded (no FMA):
 *   fx = px + 0.5, fy = py + 0.5
 *   perspective:  o = O0, q = (D0 + fx DX) + fy DY, d = q / sqrt((qx qx + qy qy) + qz qz)
 *   orthographic: o = (O0 + fx DX) + fy DY, d = D0
 *   slab test against [0,nx]x[0,ny]x[0,nz] from lo = 0, hi = +inf, using
 *   t0 = (0 - o_a)/d_a and t1 = (n_a - o_a)/d_a per axis with d_a != 0;
 *   sample k at t_k = t_entry + (k + 0.5) step while t_k < t_exit,
 *   position p = o + t_k d.
 * Sampling: nearest reads voxel floor(p) (clamped); trilinear uses q = p - 0.5,
 * i0 = floor(q), f = q - i0, clamp-to-edge neighbours.  A sample belongs to the
 * brick that contains voxel floor(p).
 * MIP: maximum sample (rays without samples give -FLT_MAX; NaN samples ignored).
 * DVR: transfer function tf_rgba[256][4] (colour not premultiplied) indexed by
 * u = clamp((s - min)/(max - min), 0, 1) * 255 with linear interpolation between
 * entries; front-to-back C += (1-A) a c, A += (1-A) a, stopping after the first
 * sample with A >= term_alpha; background (0,0,0,0); NaN samples transparent.
 */

/* ---------------------------------------------------------------- context */

/* Create a context on cfg->device (cfg may be NULL for defaults).  *out is set
 * on success.  Errors: VRC_E_INVAL, VRC_E_CUDA, VRC_E_NOMEM. */
vrc_status vrc_create(vrc_ctx **out, const vrc_config *cfg);

/* Finish every queued serving request, stop the serving thread, free every
 * cube, graph-independent scratch buffer and stream, and destroy the context.
 * Graphs created on the context must be destroyed first. */
vrc_status vrc_destroy(vrc_ctx *ctx);

/* Text of a status code (static storage). */
const char *vrc_status_str(vrc_status s);

/* Last error message recorded on this context (valid until the next call). */
const char *vrc_last_error(vrc_ctx *ctx);

/* Bytes currently charged against the HBM budget, and the budget itself. */
vrc_status vrc_memory(vrc_ctx *ctx, int64_t *used_bytes, int64_t *budget_bytes);

/* ------------------------------------------------------------------ cubes */

/*
 * Upload a float32 cube and keep it resident in bricks (Sec. 2: the cube is
 * split into sub-cubes).  src holds nx*ny*nz floats, x fastest, on the host
 * (src_on_device = 0; any host memory) or on the device (1).  storage selects
 * the stored type: VRC_F32, VRC_BF16 (round to nearest even) or VRC_FP8E4M3
 * (per-brick scale = absmax/448 over the brick and its halo, codes =
 * e4m3(x/scale) rounded to nearest even, saturating).  brick is the brick edge
 * B (a power of two in 16..512; 0 = 256, or the smallest power of two >= the
 * largest dimension when that is smaller); each
 * brick keeps a one-voxel clamp-to-edge halo.  The call records per-brick
 * min/max and returns when the cube is resident; src may then be reused.
 * Resident cubes also get a render copy (one z-layered texture array per
 * brick, read by the fused renderer's gathers) when it fits the budget with
 * 2 GiB to spare.  Without it the cube still renders, through global loads:
 * when the budget has no room a note goes to stderr, and the environment
 * variable VRC_NO_TEXTURES skips the copy on purpose.  The host-to-device copy runs on `stream` and overlaps
 * work on other streams; the packing kernels follow it on `stream`.
 * Errors: VRC_E_INVAL (dims <= 0, bad storage/brick), VRC_E_NOMEM (over budget).
 */
vrc_status vrc_cube_upload(vrc_ctx *ctx, const float *src, int32_t src_on_device, int64_t nx, int64_t ny,
                           int64_t nz, int32_t storage, int32_t brick, void *stream, int64_t *cube_id);

/* Render-copy flags, OR-ed into the storage argument of vrc_cube_upload and
 * vrc_cube_register.  AUTO: make the copy when it fits the budget with 2 GiB
 * to spare, else render through global loads (vrc_last_render_path tells);
 * REQUIRED: fail with VRC_E_NOMEM instead; NONE: no copy (the global-load
 * path, half the resident memory of the default). */
#define VRC_COPY_AUTO     0x000
#define VRC_COPY_REQUIRED 0x100
#define VRC_COPY_NONE     0x200
#define VRC_COPY_MASK     0x300

/*
 * Register a cube without keeping it resident (Abstract, Sec. 3: a shared,
 * multi-user service holds many users' cubes; on one GPU it keeps as many
 * resident as its HBM budget allows).  src: caller-owned HOST array of
 * nx*ny*nz floats, x fastest.  storage and brick as for vrc_cube_upload (the
 * render copy is made unless VRC_COPY_NONE is given).
 *   VRC_F32: src must stay valid and unchanged until vrc_cube_free; it is
 *   page-locked (cudaHostRegister) until then when it is not page-locked
 *   already, so that uploads run at the host link's speed, and no device
 *   memory is used until the cube is needed.
 *   VRC_BF16 / VRC_FP8E4M3: the call packs the cube once (the upload passes,
 *   on the device, evicting idle registered cubes if the budget needs it) and
 *   keeps its packed bricks and brick scales in page-locked host memory (half
 *   / a quarter of the source's bytes) until vrc_cube_free; every later load
 *   copies those, and src is not read after the call returns.  The cube is
 *   resident when the call returns.  If no page-locked host memory can be had
 *   the cube falls back to the VRC_F32 rules for src.
 * The serving loop admits a request for a registered cube once the
 * cube is resident: it uploads it (the vrc_cube_upload passes, on a loader
 * thread) as soon as the memory the upload needs fits the budget, evicting
 * registered cubes that no queued or running request references, least
 * recently used first; until then the request waits in the queue
 * (vrc_result.memory_wait_ms).  A direct call (render, statistics, median,
 * brick read) on a registered cube makes it resident first, on the calling
 * thread.  Errors: VRC_E_INVAL; VRC_E_NOMEM (bf16 / fp8: no room to pack).
 */
vrc_status vrc_cube_register(vrc_ctx *ctx, const float *src, int64_t nx, int64_t ny, int64_t nz, int32_t storage,
                             int32_t brick, int64_t *cube_id);

/* Registered cubes currently resident, uploads and evictions so far. */
vrc_status vrc_residency(vrc_ctx *ctx, int64_t *resident, uint64_t *loads, uint64_t *evictions);

/*
 * Out-of-core cube (Sec. 2: larger-than-memory cubes; streams overlap I/O):
 * bricks live in pinned host memory and are streamed to the device on side
 * streams while rendering.  n_host_bricks pinned brick slots are allocated;
 * logical brick b uses slot b % n_host_bricks (n_host_bricks < number of
 * bricks aliases bricks, for benchmarking links when host memory is short).
 * ring_bricks device slots are charged to the budget (0 = 8).  float32 only.
 * Errors: VRC_E_INVAL, VRC_E_NOMEM (pinned or device allocation failed).
 */
vrc_status vrc_cube_create_streamed(vrc_ctx *ctx, int64_t nx, int64_t ny, int64_t nz, int32_t brick,
                                    int64_t n_host_bricks, int32_t ring_bricks, int64_t *cube_id);

/*
 * Brick provider of an out-of-core cube (Sec. 2: cubes larger than memory,
 * read sub-cube by sub-cube).  Writes brick `brick` = (bx, by, bz) (index
 * (bz*nby + by)*nbx + bx) with its one-voxel halo into dst: (B+2)^3 floats,
 * x fastest, covering voxels [b*B-1, b*B+B] of each axis, the clamp-to-edge
 * value outside the cube.  dst is host memory owned by the library, valid
 * for the duration of the call.  Returns 0 on success; any other value makes
 * the calling library operation fail with VRC_E_SOURCE.  Called on the thread
 * of the library call that needs the brick, never concurrently for one cube.
 */
typedef int32_t (*vrc_brick_source_fn)(void *user, int64_t brick, int32_t bx, int32_t by, int32_t bz, float *dst);

/*
 * Out-of-core cube whose bricks come from a provider (Sec. 2: cubes larger
 * than the memory of one node, streamed to the GPU on side streams).  The
 * provider hands float32 bricks; storage (VRC_F32, VRC_BF16, VRC_FP8E4M3) is
 * the type the host cache and the device ring keep them in, packed as
 * vrc_cube_upload packs (bf16 / fp8: on the device, a provided brick at a
 * time, then copied into its host slot; the FP8 scale of a brick comes from
 * the absmax of its provided values, halo included), so a bf16 / fp8 cube
 * needs half / a quarter of the host memory and of the bytes each frame moves
 * over the host link.  Stored extrema, statistics, median and images equal
 * those of the same cube uploaded with that storage.
 * The call asks `source` for every brick once, in index order, to record each
 * brick's minimum and maximum (the transfer-function range, brick culling),
 * the sums that centre the statistics and its non-finite voxels; it returns
 * when all bricks have been seen.  n_host_bricks pinned host slots (1 ..
 * number of bricks) cache provided bricks: with a slot for every brick, brick
 * b lives in slot b; otherwise the first n_host_bricks - T bricks keep their
 * slots and the others share the last T = min(n_host_bricks, 16) slots.
 * Renders, statistics and the median stream the bricks
 * they need through ring_bricks device slots (0 = 8; at least 2; charged to
 * the budget) and call `source` again, on the calling thread, for every brick
 * whose slot holds another brick (after the slot's previous copy to the
 * device has completed); with n_host_bricks = number of bricks the provider
 * is called once per brick only.  The zero-copy path needs every brick cached
 * (n_host_bricks = number of bricks).  `user` is passed through and must stay
 * valid until the cube is freed.
 * Errors: VRC_E_INVAL, VRC_E_NOMEM (pinned or device allocation failed),
 * VRC_E_SOURCE (the provider failed; no cube is created).
 */
vrc_status vrc_cube_upload_streamed(vrc_ctx *ctx, vrc_brick_source_fn source, void *user, int64_t nx, int64_t ny,
                                    int64_t nz, int32_t storage, int32_t brick, int64_t n_host_bricks,
                                    int32_t ring_bricks, int64_t *cube_id);

/*
 * Fill host slot `slot` of a streamed cube with one brick given as
 * (B+2)^3 floats, x fastest, covering voxels [b*B-1, b*B+B] of each axis with
 * clamp-to-edge values outside the cube.  Host memory, copied; records the
 * slot's min/max.  Errors: VRC_E_BADID, VRC_E_INVAL.
 */
vrc_status vrc_cube_put_brick(vrc_ctx *ctx, int64_t cube_id, int64_t slot, const float *brick_with_halo);

/* Release a cube.  Waits for the device (the memory may be reused at once).
 * VRC_E_BUSY while serving requests still reference it.  Like every call
 * except vrc_submit / vrc_poll, it must not overlap another call on the same
 * context from another host thread: a statistics or render call in flight on
 * another thread may still be reading the cube's host-side record. */
vrc_status vrc_cube_free(vrc_ctx *ctx, int64_t cube_id);

/*
 * Release a cube without waiting for the device.  The caller guarantees that
 * every piece of work that reads the cube was issued on `stream`, or before
 * work already issued on `stream` (stream order, e.g. through events).  The id
 * is invalid on return; the cube's memory goes back to the context's cache
 * when the work issued on `stream` so far has completed, and a later upload
 * of the same shape reuses it without new device allocations.  Errors:
 * VRC_E_BADID, VRC_E_BUSY (serving requests reference the cube; nothing is
 * released), VRC_E_CUDA (the cube was released after a device-wide wait).
 */
vrc_status vrc_cube_free_async(vrc_ctx *ctx, int64_t cube_id, void *stream);

/* dims, brick edge, storage dtype, brick count, stored bytes, the stored
 * min/max recorded at upload, and the bytes of the texture render copies
 * (0 when the cube has none, e.g. no room in the budget; any output pointer
 * may be NULL). */
vrc_status vrc_cube_info(vrc_ctx *ctx, int64_t cube_id, int64_t dims[3], int32_t *brick, int32_t *storage,
                         int64_t *n_bricks, int64_t *bytes, float *vmin, float *vmax, int64_t *render_copy_bytes);

/*
 * Copy the stored form of brick `brick` (x fastest over the brick grid) of a
 * cube into host memory `dst` of at least `dst_bytes` bytes (Sec. 2:
 * sub-cubes; the quantised storage of the precision form).  Layout: R = B + 2
 * planes (local z = -1..B) of R rows (local y = -1..B) of P = B + 2*O elements
 * of esize bytes (4 fp32, 2 bf16 bits, 1 e4m3 code; O = 32 / esize for
 * resident cubes, 16 / esize for out-of-core cubes: rows start interior voxels
 * on 32- / 16-byte boundaries), the
 * voxel at local x at element O + x of its row: x = -1 and x = B are the
 * halo, elements before and after them are padding (0).  Halo voxels outside
 * the cube repeat the nearest edge voxel; FP8 codes use this brick's scale.
 * Brick bytes = P * R * R * esize.  Synchronous (waits for the device).
 * Out-of-core cubes: the brick's host slot (a provider cube provides and
 * packs the brick again when its slot holds another one; a caller-filled cube
 * reads slot brick % n_host_bricks).
 * Errors: VRC_E_BADID, VRC_E_INVAL (brick out of range, dst NULL, dst_bytes
 * too small, caller-filled slots not all written), VRC_E_SOURCE.
 */
vrc_status vrc_cube_read_brick(vrc_ctx *ctx, int64_t cube_id, int64_t brick, void *dst, int64_t dst_bytes);

/* ------------------------------------------------------------- statistics */

/*
 * Global statistics in one fused pass over the bricks (Abstract: min/max and
 * histogram; Sec. 3: standard deviation): min and max (recorded at upload),
 * n, mean and population std (binary64 block partials, fixed-order final
 * merge), n_nonfinite, and, when nbins > 0, hist[nbins] counts over [min,
 * max] with the binary32 bin formula
 *   range = fl(max - min), scale = fl(nbins / range),
 *   bin = trunc(fl(fl(x - min) * scale)) clamped to [0, nbins-1]
 *   (range == 0: every value in bin 0).
 * out and hist are HOST memory; the call waits for `stream`.  nbins <= 65536.
 * Out-of-core cubes (Sec. 3: min/max accumulate sub-cube by sub-cube; std
 * needs all data) take the same pass chunk by chunk: runs of consecutive
 * bricks are copied through the cube's device ring (bricks that are not in
 * the host cache are provided first) and each chunk's pass writes its own
 * block partials, merged in a fixed order at the end; min, max and every
 * histogram count equal those of the same cube uploaded resident, mean and
 * std agree to rounding.
 * Errors: VRC_E_BADID, VRC_E_INVAL, VRC_E_NONFINITE (no finite voxel),
 * VRC_E_SOURCE (out-of-core cube: the provider failed).
 */
vrc_status vrc_cube_stats(vrc_ctx *ctx, int64_t cube_id, int32_t nbins, vrc_stats *out, uint64_t *hist,
                          void *stream);

/*
 * Asynchronous form: writes a vrc_stats record to DEVICE memory dev_out and
 * counts to DEVICE memory dev_hist[nbins] (may be NULL when nbins == 0),
 * stream-ordered; nothing waits (out-of-core cubes: the call returns when
 * every chunk's copy and pass has been issued).  dev_out->n == 0 flags a cube
 * without finite voxels.
 */
vrc_status vrc_cube_stats_async(vrc_ctx *ctx, int64_t cube_id, int32_t nbins, vrc_stats *dev_out,
                                uint64_t *dev_hist, void *stream);

/*
 * Allocation-free form of vrc_cube_stats_async (the paper has no counterpart;
 * this serves callers that must not allocate device memory at this point: a
 * latency-bound interactive or serving loop, where cudaMalloc/cudaFree may
 * stall the whole device, or a plug-in inside an application that keeps the
 * device memory in its own pool).  Same inputs, outputs and errors as
 * vrc_cube_stats_async, for resident cubes (VRC_E_UNSUPPORTED for out-of-core
 * cubes, which stream through their device ring, and for registered cubes that
 * are not resident at the time); the pass's block partials go to one static device
 * array of 64 KiB that the library holds on every device that loads it, so
 * the call performs no cudaMalloc, cudaFree or other allocation.  Devices whose
 * statistics pass needs more scratch than that are refused with VRC_E_NOMEM.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture.  A cudaDeviceReset by the host
 * application invalidates the kept address: do not call this entry point on
 * that device again afterwards.
 * All calls share the array: calls whose work overlaps on the GPU (different
 * streams, or other host threads) race and give wrong results, so serialise
 * them (e.g. one stream).  Nothing in the array needs clearing between calls.
 */
vrc_status vrc_cube_stats_noalloc(vrc_ctx *ctx, int64_t cube_id, int32_t nbins, vrc_stats *dev_out,
                                  uint64_t *dev_hist, void *stream);

/*
 * Median of the finite stored values (Sec. 3: a global task needing all data):
 * the lower median, value of rank floor((n-1)/2) in ascending order.  Exact:
 * radix selection on the order-preserving 32-bit keys of the values (-0 and +0
 * are one value), three passes counting 12, 10 and 10 key bits in
 * shared-memory histograms; each pass counts the keys whose leading bits match
 * the digits chosen so far.  Float32 cubes: the second pass also keeps the keys
 * of the first pass's selected bin in a device buffer (allocated for the call
 * when they number at most 2^26 and the budget allows; otherwise the third
 * pass reads the cube again), and the third pass reads those.  FP8 cubes take one pass over the cube that
 * counts each brick's 8-bit codes; the three radix passes then run over the
 * (brick, code) entries weighted by their counts (a stored fp8 value depends
 * only on its brick's scale and its code).  bf16 keys have 16 significant
 * bits, so two passes fix them.  Out-of-core cubes stream their bricks
 * through the device ring once per pass.
 * Resident float32 / bf16 cubes of at least 2^22 voxels first bracket the
 * median.  A first-digit pass over every 61st chunk of rows (1.6% of the cube)
 * bounds the first-digit bins the median falls in.  One pass over the cube then
 * counts the finite values and those below the bounded bins, and keeps the
 * keys of those bins in a device buffer (allocated for the call when they
 * number at most 2^26 and the budget allows).  The digits are selected among
 * the kept keys.  When the median's rank falls outside them (a sample unlike
 * the cube), or a buffer cannot be had, the radix passes above run; the result
 * is the same exact value either way.  *out is HOST memory; waits for
 * `stream`.  Errors: VRC_E_BADID, VRC_E_NONFINITE, VRC_E_SOURCE.
 */
vrc_status vrc_cube_median(vrc_ctx *ctx, int64_t cube_id, double *out, void *stream);

/* -------------------------------------------------------------- rendering */

/*
 * Every render call copies its small inputs (cameras turned into per-view job
 * records, the transfer function) into pinned host memory and a small kernel
 * on `stream` reads them into device memory, so no copy engine is involved
 * (when four earlier calls' inputs are all still waiting on their streams,
 * plain host-to-device copies are used instead).
 * Reads of host memory by the device wait behind a large device-to-host copy
 * already in flight (a render issued after a 1 GB image download had started
 * began only when the download ended): in a pipeline, issue the next render
 * before starting to copy the previous images back.
 */

/*
 * Maximum-intensity projection of n_views views in one persistent launch
 * (batched (view, ray tile) work items).  cams: HOST array of n_views cameras.
 * out: DEVICE float[n_views*H*W].  Stream-ordered; returns after launching.
 * Streamed cubes always take the sort-last path with brick streaming.
 * Errors: VRC_E_BADID, VRC_E_INVAL.
 */
vrc_status vrc_render_mip(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views,
                          const vrc_raycfg *rc, float *out, void *stream);

/*
 * Front-to-back transfer-function compositing with early termination
 * (term_alpha in (0, 1]; > 1 disables termination).  tf_rgba: HOST float[1024].
 * The transfer-function range is the cube's stored [min, max].
 * out: DEVICE float[n_views*H*W*4].  Stream-ordered.
 * Errors: VRC_E_BADID, VRC_E_INVAL.
 */
vrc_status vrc_render_dvr(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views,
                          const vrc_raycfg *rc, const float *tf_rgba, float term_alpha, float *out,
                          void *stream);

/*
 * Ray samples of the most recent vrc_render_mip / vrc_render_dvr call on this
 * context: *samples = lattice samples inside the cube up to early termination
 * (the work the method defines); *evaluated = samples actually fetched and
 * composited (smaller only with skip_empty; may be NULL).  Waits for that
 * render to finish.  Outputs are HOST memory.  VRC_E_TIMEOUT (counts still
 * written) if a bounded device-side wait of that render gave up (VRC_PATH_SLAB:
 * a shared-memory staging copy that did not complete within 0.5 s); its image
 * is then unspecified.
 */
vrc_status vrc_last_render_samples(vrc_ctx *ctx, uint64_t *samples, uint64_t *evaluated);

/*
 * Path the most recent vrc_render_mip / vrc_render_dvr call on this context
 * took: VRC_PATH_FUSED (texture gathers from the render copy), VRC_PATH_FUSED_LDG
 * (global loads: requested, nearest sampling, or the cube has no render copy),
 * VRC_PATH_SORTLAST, VRC_PATH_STREAMED (out-of-core: bricks copied through the
 * device ring), VRC_PATH_ZEROCOPY, VRC_PATH_SLAB or VRC_PATH_ROWS (nearest MIP
 * of orthographic views along y or z; groups of rays whose voxel columns are
 * not consecutive x of one brick row take the per-ray loop inside the same
 * launch).  *path is HOST memory.
 */
#define VRC_PATH_STREAMED  5   /* reported only: sort-last with brick streaming */
#define VRC_PATH_ROWS      6   /* reported only: fused nearest MIP of an orthographic view along
                                  y or z, 8 pixels of an image row per thread (one 8-, 16- or
                                  32-byte load per sample of the group's rays); same image as
                                  the per-ray loop, bit for bit */
vrc_status vrc_last_render_path(vrc_ctx *ctx, int32_t *path);

/*
 * Bricks of the most recent sort-last render on this context (Sec. 2: each
 * brick is rendered on its own into a partial image): *traversed = distinct
 * bricks that some view's rays cross and that were rendered (for a streamed
 * cube: copied to the device, or read in place on the zero-copy path);
 * *culled = distinct bricks those rays cross that were skipped because no
 * sample inside them can be visible (skip_empty with DVR: the brick's largest
 * value, halo included, is at or below the transfer function's transparent
 * threshold).  Both 0 after a fused render.  Outputs are HOST memory;
 * VRC_E_INVAL on NULL arguments.  Culled bricks' samples are not traversed and
 * are not counted by vrc_last_render_samples.
 */
vrc_status vrc_last_render_bricks(vrc_ctx *ctx, int64_t *traversed, int64_t *culled);

/*
 * Sort-last combination of two image buffers (Sec. 2: gathered partial
 * images): mode 0 (MIP) out = max(front, back); mode 1 (DVR) out = front +
 * (1 - front.A) * back per channel.  All DEVICE float arrays of n_pixels
 * (x4 for DVR); out may alias front or back.  Stream-ordered.
 */
vrc_status vrc_composite(vrc_ctx *ctx, const float *front, const float *back, float *out, int64_t n_pixels,
                         int32_t mode, void *stream);

/* -------------------------------------------------- batching: graphs, tuning */

typedef struct vrc_graph vrc_graph;

/*
 * Capture one multi-view render (MIP when tf_rgba is NULL, else DVR) of a
 * resident cube into a CUDA graph: camera data are uploaded once, the graph
 * resets the work counter and runs the persistent kernel.  out (DEVICE) is
 * baked into the graph.  Errors: VRC_E_BADID, VRC_E_INVAL, VRC_E_CUDA.
 */
vrc_status vrc_graph_create(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views,
                            const vrc_raycfg *rc, const float *tf_rgba, float term_alpha, float *out,
                            vrc_graph **graph);
vrc_status vrc_graph_launch(vrc_graph *graph, void *stream);
vrc_status vrc_graph_destroy(vrc_graph *graph);

typedef struct {
    int32_t tile_w, tile_h;      /* chosen ray tile */
    int32_t ctas_per_sm;         /* chosen persistent-grid occupancy */
    int32_t brick;               /* brick edge of the cube after tuning */
    float step;                  /* chosen step: the requested one unless a step tolerance was given */
    int32_t reserved;
    double best_ms, default_ms;  /* time of the chosen and of the default configuration (requested step) */
    double step_max_abs_diff;    /* largest image difference of the chosen step against the requested one */
} vrc_tuning;

/*
 * Autotuner: times the candidate ray tiles (8x32, 16x16, 32x8) and persistent
 * grid sizes for this cube and workload with CUDA events and stores the best
 * as the cube's default (used when rc->tile_w == 0).  The step is never
 * changed.  Runs the render several times into `out` (DEVICE, as for the
 * render call); waits for `stream`.
 */
vrc_status vrc_autotune(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views,
                        const vrc_raycfg *rc, const float *tf_rgba, float term_alpha, float *out, void *stream,
                        vrc_tuning *result);

#define VRC_TUNE_BRICK 1
/*
 * Autotuner of the batching form: vrc_autotune's ray tile and grid search on
 * the cube as it is, and
 *   - with VRC_TUNE_BRICK (fp32 and bf16 cubes): the same search on the cube
 *     re-packed at each other brick edge in {64, 128, 256} (at most the
 *     smallest power of two >= the largest dimension), built on the device
 *     from the cube's stored values (exact: the storage rounding is
 *     idempotent); the fastest brick edge replaces the cube's storage under the
 *     same id (images are the same bit for bit at every brick edge).  Edges
 *     whose trial copy does not fit the budget are skipped.  FP8 cubes keep
 *     their edge (their per-brick scales depend on it).
 *   - with step_tolerance > 0: the requested step times 1.25, 1.5 and 2 is
 *     timed with the chosen configuration, and the fastest step whose image
 *     (all views, every channel) differs from the requested step's image by at
 *     most step_tolerance is returned in result->step (renders keep using the
 *     step the caller passes; step_tolerance = 0 never changes it).
 * `out` (DEVICE, as for the render call) holds the last render.  Waits for
 * `stream`.  Errors: as vrc_autotune; VRC_E_INVAL for unknown flags or a
 * negative tolerance; VRC_E_BUSY when serving requests use the cube and its
 * storage would be replaced.
 */
vrc_status vrc_autotune_cube(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views,
                             const vrc_raycfg *rc, const float *tf_rgba, float term_alpha, float *out, void *stream,
                             int32_t flags, float step_tolerance, vrc_tuning *result);

/* ---------------------------------------------------------------- serving */

#define VRC_REQ_MIP   0
#define VRC_REQ_DVR   1
#define VRC_REQ_STATS 2
typedef struct {
    int32_t kind;          /* VRC_REQ_MIP, VRC_REQ_DVR or VRC_REQ_STATS */
    int32_t nbins;         /* stats: histogram bins (0..65536) */
    int64_t cube_id;
    vrc_camera cam;        /* render: one view */
    vrc_raycfg rc;
    float tf_rgba[1024];   /* DVR */
    float term_alpha;      /* DVR */
    int32_t reserved;
    void *out;             /* render: DEVICE image (float[H*W] or float[H*W*4]);
                              stats: DEVICE uint64[nbins] or NULL */
} vrc_request;

typedef struct {
    vrc_status status;     /* VRC_OK or the request's error */
    int32_t path;          /* render: VRC_PATH_FUSED (texture gathers) or VRC_PATH_FUSED_LDG (global loads) */
    vrc_stats stats;       /* stats requests */
    double queue_ms;       /* submit -> launch */
    double latency_ms;     /* submit -> completion observed */
    uint64_t samples;      /* render: ray samples taken */
    double memory_wait_ms; /* part of queue_ms spent waiting for the cube to become resident */
    int32_t cube_loaded;   /* 1 if the cube was uploaded for this request (registered cubes) */
    int32_t reserved;
} vrc_result;

/*
 * Serving loop (Abstract, Sec. 3: analysis and visualisation as a shared,
 * on-demand service).  vrc_submit copies the request, queues it and returns a
 * ticket at once.  A background thread admits queued requests while the
 * number on the GPU is below max_inflight and their scratch fits the budget,
 * groups every admitted render into one heterogeneous persistent launch (each
 * request keeps its own cube, camera, image size and transfer function) on one
 * of n_streams streams, and runs statistics requests and render batches of at
 * most 512 x 512 pixels on a stream of the highest priority.  Larger render
 * batches run as a series of launches of two waves of tiles each, so a
 * request that arrives while they are on the GPU is admitted at once and gets
 * SMs at the next launch boundary instead of after the whole batch.  The cube must stay allocated
 * until the request completes (vrc_cube_free returns VRC_E_BUSY before).
 * Errors at submit: VRC_E_BADID, VRC_E_INVAL; later errors arrive in
 * vrc_result.status.
 */
vrc_status vrc_submit(vrc_ctx *ctx, const vrc_request *req, uint64_t *ticket);

/*
 * Wait up to timeout_ms (0 = just check, < 0 = forever) for a ticket.
 * Returns VRC_OK and fills *res (the ticket is then retired), VRC_PENDING when
 * timeout_ms == 0 and it is not done, VRC_E_TIMEOUT when the wait expired,
 * VRC_E_BADID for an unknown or retired ticket.
 */
vrc_status vrc_poll(vrc_ctx *ctx, uint64_t ticket, vrc_result *res, int32_t timeout_ms);

/* ------------------------------------------------------ failure injection */

#define VRC_INJECT_NONE        0
#define VRC_INJECT_ALLOC       1  /* the nth device/pinned allocation fails (VRC_E_NOMEM) */
#define VRC_INJECT_H2D         2  /* the nth host->device brick copy fails (VRC_E_INJECTED) */
#define VRC_INJECT_DROP_REQ    3  /* the nth admitted serving request fails (VRC_E_INJECTED) */
#define VRC_INJECT_SLAB_WAIT   4  /* the nth VRC_PATH_SLAB render issues none of its staging copies:
                                     its bounded waits run out (about 1 s), the image is unspecified
                                     and vrc_last_render_samples returns VRC_E_TIMEOUT */
/*
 * Host-side fault injection for tests: arm failure `what` to fire on its nth
 * occurrence from now (n >= 1); VRC_INJECT_NONE disarms.  Nothing faults on
 * the GPU: VRC_INJECT_SLAB_WAIT only withholds copies that kernels then wait
 * for with a time limit.
 */
vrc_status vrc_debug_inject(vrc_ctx *ctx, int32_t what, int64_t nth);

/* Kernel launches issued by this context so far (all entry points). */
uint64_t vrc_launch_count(vrc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* VRC_H */
