// Brick pack + quantise (upload), out-of-core cube registration, cube lifetime.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <float.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <type_traits>

#include "vrc_internal.h"

int64_t host_slot(const Cube *c, int64_t b);   // out-of-core host cache (below)

namespace {

// Blocks per brick for a pass over the bricks whose blocks (256 threads) each
// take an equal share of a brick's rows: the split that fills the resident
// block slots best over whole waves (the smallest such split), at most one
// block per 64 rows.
int blocks_per_brick(const vrc_ctx *ctx, const void *kern, int64_t nbricks, int64_t rows_per_brick)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0) != cudaSuccess || occ <= 0) {
        cudaGetLastError();
        occ = 4;
    }
    const int64_t slots = (int64_t)ctx->sm_count * occ;
    const int max_split = (int)std::max<int64_t>(1, std::min<int64_t>(256, rows_per_brick / 64));
    int best = 1;
    double best_fill = 0.0;
    for (int s = 1; s <= max_split; ++s) {
        const int64_t blocks = nbricks * s, waves = (blocks + slots - 1) / slots;
        const double fill = (double)blocks / (double)(waves * slots);
        if (fill > best_fill + 1e-9) {
            best_fill = fill;
            best = s;
        }
    }
    return best;
}

struct ScanPartial {
    float mn, mx, absmax;
    int32_t nonfinite;
    double sum;   // sum of finite interior source values (for the statistics shift)
    int64_t cnt;
};

__device__ __forceinline__ int64_t clamp64(int64_t i, int64_t n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

struct ScanAcc {
    float mn = INFINITY, mx = -INFINITY, am = 0.f, sum = 0.f;
    int nnf = 0, cnt = 0;

    // every value finite (checked afterwards through the sum)
    __device__ __forceinline__ void fast(float x, bool fp8)
    {
        mn = fminf(mn, x);
        mx = fmaxf(mx, x);
        sum += x;
        if (fp8) am = fmaxf(am, fabsf(x));
    }
    // an interior value of any kind
    __device__ __forceinline__ void exact(float x)
    {
        if (fabsf(x) <= FLT_MAX) {
            mn = fminf(mn, x);
            mx = fmaxf(mx, x);
            sum += x;
            am = fmaxf(am, fabsf(x));
            ++cnt;
        } else {
            ++nnf;
        }
    }
    // a halo value: it only bounds the FP8 scale
    __device__ __forceinline__ void halo(float x)
    {
        if (fabsf(x) <= FLT_MAX) am = fmaxf(am, fabsf(x));
    }
};

// Interior rows [w0, nrows) step nw of one brick: extents (nxb, nyb) of its
// interior inside the cube, x0 = its first column.  16-byte loads where the
// rows allow them.  FP8 storage also folds in the row's two halo columns.
template <bool FP8, bool EXACT>
__device__ __forceinline__ void scan_rows(const float *__restrict__ src, const BrickGeom &g, int64_t x0, int64_t y0,
                                          int64_t z0, int nxb, int nyb, int nrows, int w0, int nw, bool vec,
                                          int lane, ScanAcc &a)
{
    const int64_t NX = g.dims[0];
    for (int r = w0; r < nrows; r += nw) {
        const int ly = r % nyb, lz = r / nyb;
        const float *rowp = src + ((z0 + lz) * g.dims[1] + y0 + ly) * NX;
        if (vec) {
            const float4 *r4 = reinterpret_cast<const float4 *>(rowp + x0);
            const int nch = nxb >> 2;
            for (int c0 = 0; c0 < nch; c0 += 64) {
                float4 q[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int c = c0 + lane + 32 * k;
                    q[k] = c < nch ? __ldg(r4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (c0 + lane + 32 * k < nch) {
                        if (EXACT) {
                            a.exact(q[k].x); a.exact(q[k].y); a.exact(q[k].z); a.exact(q[k].w);
                        } else {
                            a.fast(q[k].x, FP8); a.fast(q[k].y, FP8); a.fast(q[k].z, FP8); a.fast(q[k].w, FP8);
                            a.cnt += 4;
                        }
                    }
                }
            }
        } else {
            for (int x = lane; x < nxb; x += 32) {
                const float v = __ldg(rowp + x0 + x);
                if (EXACT) a.exact(v);
                else { a.fast(v, FP8); ++a.cnt; }
            }
        }
        if (FP8 && lane == 0) {
            a.halo(__ldg(rowp + clamp64(x0 - 1, NX)));
            a.halo(__ldg(rowp + clamp64(x0 + g.B, NX)));
        }
    }
}

// Pass 1: per brick, over its interior voxels inside the cube: min/max, sum
// and count of the finite values and the count of non-finite ones; for FP8
// storage also the largest finite magnitude over the whole stored region
// (interior plus the clamp-to-edge halo), which sets the brick's scale.  The
// first sweep assumes finite values (three operations per value); a block
// whose sum comes out non-finite, which any NaN or infinity causes, sweeps
// its rows again testing every value.  Stored rows and columns past the cube
// edge repeat interior values and are not read.
template <bool FP8>
__global__ void __launch_bounds__(256) k_brick_scan(const float *__restrict__ src, BrickGeom g, int split,
                                                    ScanPartial *__restrict__ part)
{
    const int64_t b = blockIdx.x;
    const int bx = (int)(b % g.nb[0]), by = (int)((b / g.nb[0]) % g.nb[1]), bz = (int)(b / ((int64_t)g.nb[0] * g.nb[1]));
    const int lane = threadIdx.x & 31;
    const int64_t x0 = (int64_t)bx * g.B, y0 = (int64_t)by * g.B, z0 = (int64_t)bz * g.B;
    const int nxb = (int)(g.dims[0] - x0 < g.B ? g.dims[0] - x0 : g.B);
    const int nyb = (int)(g.dims[1] - y0 < g.B ? g.dims[1] - y0 : g.B);
    const int nzb = (int)(g.dims[2] - z0 < g.B ? g.dims[2] - z0 : g.B);
    const int nrows = nyb * nzb;
    const int w0 = blockIdx.y * (blockDim.x / 32) + threadIdx.x / 32, nw = split * (blockDim.x / 32);
    const bool vec = (g.dims[0] & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    ScanAcc a;
    scan_rows<FP8, false>(src, g, x0, y0, z0, nxb, nyb, nrows, w0, nw, vec, lane, a);
    if (__syncthreads_or(!(fabsf(a.sum) <= FLT_MAX))) {
        a = ScanAcc();
        scan_rows<FP8, true>(src, g, x0, y0, z0, nxb, nyb, nrows, w0, nw, vec, lane, a);
    }
    if (FP8) {
        // the halo rows: ly or lz at -1 or B (columns -1..B), 4B + 4 rows
        const int R = g.R;
        for (int h = w0; h < 4 * g.B + 4; h += nw) {
            int ly, lz;
            if (h < 2 * R) {
                lz = h < R ? -1 : g.B;
                ly = h % R - 1;
            } else {
                const int j = h - 2 * R;
                ly = j < g.B ? -1 : g.B;
                lz = j % g.B;
            }
            const float *rowp = src + (clamp64(z0 + lz, g.dims[2]) * g.dims[1] + clamp64(y0 + ly, g.dims[1])) * g.dims[0];
            for (int x = lane - 1; x <= g.B; x += 32) a.halo(__ldg(rowp + clamp64(x0 + x, g.dims[0])));
        }
    }
    double dsum = a.sum;
    float mn = a.mn, mx = a.mx, am = a.am;
    int nnf = a.nnf, cnt = a.cnt;
    for (int o = 16; o; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
        nnf += __shfl_xor_sync(0xffffffffu, nnf, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    }
    __shared__ ScanPartial sp[8];
    if (lane == 0) sp[threadIdx.x / 32] = ScanPartial{mn, mx, am, nnf, dsum, cnt};
    __syncthreads();
    if (threadIdx.x == 0) {
        ScanPartial r = sp[0];
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) {
            r.mn = fminf(r.mn, sp[w].mn);
            r.mx = fmaxf(r.mx, sp[w].mx);
            r.absmax = fmaxf(r.absmax, sp[w].absmax);
            r.nonfinite += sp[w].nonfinite;
            r.sum += sp[w].sum;
            r.cnt += sp[w].cnt;
        }
        part[b * split + blockIdx.y] = r;
    }
}

// e4m3 code of x / scale, nearest even, finite values saturated to +-448.
// E4M3 has no infinity: every non-finite x (NaN or +-inf) is stored as NaN
// (0x7f), so non-finite voxels stay non-finite in every storage type.
__device__ __forceinline__ uint8_t fp8_code(float x, float scale)
{
    if (!(fabsf(x) <= FLT_MAX)) return 0x7f;
    return (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(x, scale), __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ float fp8_round_trip(float x, float scale)
{
    const __half h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)fp8_code(x, scale), __NV_E4M3);
    return __fmul_rn(__half2float(h), scale);
}

__device__ __forceinline__ float stored_value(float x, int dtype, float scale)
{
    if (dtype == VRC_BF16) return __bfloat162float(__float2bfloat16_rn(x));
    if (dtype == VRC_FP8E4M3) return fp8_round_trip(x, scale);
    return x;
}

// Per brick: reduce the scan partials, derive the FP8 scale and the stored
// min/max (rounding is monotone, so stored(min) is the stored minimum).
__global__ void k_brick_finish(const ScanPartial *__restrict__ part, BrickGeom g, int split, float *scales,
                               float *bmin, float *bmax, int32_t *bnonfinite, double *bsum)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= g.nbricks) return;
    ScanPartial r = part[b * split];
    for (int s = 1; s < split; ++s) {
        const ScanPartial p = part[b * split + s];
        r.mn = fminf(r.mn, p.mn);
        r.mx = fmaxf(r.mx, p.mx);
        r.absmax = fmaxf(r.absmax, p.absmax);
        r.nonfinite += p.nonfinite;
        r.sum += p.sum;
        r.cnt += p.cnt;
    }
    bsum[2 * b] = r.sum;
    bsum[2 * b + 1] = (double)r.cnt;
    float scale = 1.f;
    if (g.dtype == VRC_FP8E4M3 && r.absmax > 0.f) scale = __fdiv_rn(r.absmax, 448.f);
    scales[b] = scale;
    const bool any = r.mn <= r.mx;
    bmin[b] = any ? stored_value(r.mn, g.dtype, scale) : FLT_MAX;
    bmax[b] = any ? stored_value(r.mx, g.dtype, scale) : -FLT_MAX;
    bnonfinite[b] = r.nonfinite;
}

// One provided brick ((B+2)^3 floats, x fastest, halo included) in brick
// storage: row (zr, yr) of P elements with the halo voxel lx = -1 at element
// O - 1, padding 0; values stored as the upload's pack pass stores them.
template <int DT>
__global__ void k_pack_provided(const float *__restrict__ bw, BrickGeom g, float scale, uint8_t *__restrict__ out)
{
    const int64_t nrow = (int64_t)g.R * g.R;
    for (int64_t row = blockIdx.x; row < nrow; row += gridDim.x) {
        const float *in = bw + row * g.R;
        for (int e = threadIdx.x; e < g.P; e += blockDim.x) {
            const int i = e - (g.O - 1);
            const bool v = i >= 0 && i < g.R;
            if (DT == VRC_BF16)
                reinterpret_cast<uint16_t *>(out)[row * g.P + e] =
                    v ? __bfloat16_as_ushort(__float2bfloat16_rn(in[i])) : (uint16_t)0;
            else
                out[row * g.P + e] = v ? fp8_code(in[i], scale) : (uint8_t)0;
        }
    }
}

// Stored values of per-brick extrema measured on provided float32 bricks
// (rounding is monotone, so the stored extremum is the extremum stored); a
// brick without finite values keeps its markers, non-finite halo maxima stay.
template <int DT>
__global__ void k_stored_extrema(float *mn, float *mx, float *hmx, const float *scales, int64_t n)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const float s = scales[b];
    if (mn[b] <= mx[b]) {
        mn[b] = stored_value(mn[b], DT, s);
        mx[b] = stored_value(mx[b], DT, s);
    }
    if (fabsf(hmx[b]) <= FLT_MAX) hmx[b] = stored_value(hmx[b], DT, s);
}

// 16 bytes of stored elements from 16 / esize source values.
template <int DT> struct Chunk {
    static constexpr int n = DT == VRC_F32 ? 4 : (DT == VRC_BF16 ? 8 : 16);
};

template <int DT>
__device__ __forceinline__ uint4 pack_chunk(const float (&x)[Chunk<DT>::n], float scale)
{
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (DT == VRC_F32) {
            w[i] = __float_as_uint(x[i]);
        } else if (DT == VRC_BF16) {
            w[i] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[2 * i])) |
                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[2 * i + 1])) << 16);
        } else {
            w[i] = (uint32_t)fp8_code(x[4 * i], scale) | ((uint32_t)fp8_code(x[4 * i + 1], scale) << 8) |
                   ((uint32_t)fp8_code(x[4 * i + 2], scale) << 16) | ((uint32_t)fp8_code(x[4 * i + 3], scale) << 24);
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Pass 2: write every stored row of every brick as 16-byte chunks: L = O *
// esize / 16 left chunks (padding, then the halo column lx = -1 as the last
// element), B * esize / 16 interior chunks, L right chunks (the halo column
// lx = B as the first element, then padding).  Halo rows and columns clamp to
// the cube edge; padding is 0.  A warp writes one row at a time; interior
// source values are read as 16-byte vectors where the rows allow them.
template <int DT>
__global__ void __launch_bounds__(256) k_brick_pack(const float *__restrict__ src, BrickGeom g, int split,
                                                    const float *__restrict__ scales, void *pool)
{
    constexpr int N = Chunk<DT>::n;
    const int64_t b = blockIdx.x;
    const int bx = (int)(b % g.nb[0]), by = (int)((b / g.nb[0]) % g.nb[1]), bz = (int)(b / ((int64_t)g.nb[0] * g.nb[1]));
    const float scale = scales[b];
    char *bp = reinterpret_cast<char *>(pool) + b * g.brick_bytes;
    const int R = g.R, lane = threadIdx.x & 31;
    const int64_t NX = g.dims[0], x0 = (int64_t)bx * g.B;
    const int nin = g.B / N, L = g.O / N;
    const bool vec = (NX & 3) == 0 && x0 + g.B <= NX && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    const int64_t row_bytes = (int64_t)g.P * g.esize;
    for (int row = blockIdx.y * (blockDim.x / 32) + threadIdx.x / 32; row < R * R; row += split * (blockDim.x / 32)) {
        const int ly = row % R - 1, lz = row / R - 1;
        const int64_t gy = clamp64((int64_t)by * g.B + ly, g.dims[1]), gz = clamp64((int64_t)bz * g.B + lz, g.dims[2]);
        const float *rowp = src + (gz * g.dims[1] + gy) * NX;
        uint4 *out = reinterpret_cast<uint4 *>(bp + row * row_bytes);
        // two chunks per lane in flight (a B = 256 fp32 row is 64 chunks)
        for (int j0 = lane; j0 < nin; j0 += 64) {
            float x[2][N];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + 32 * h;
                if (j >= nin) break;
                if (vec) {
                    const float4 *p4 = reinterpret_cast<const float4 *>(rowp + x0 + (int64_t)j * N);
#pragma unroll
                    for (int m = 0; m < N / 4; ++m) {
                        const float4 q = __ldg(p4 + m);
                        x[h][4 * m] = q.x; x[h][4 * m + 1] = q.y; x[h][4 * m + 2] = q.z; x[h][4 * m + 3] = q.w;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < N; ++e) x[h][e] = __ldg(rowp + clamp64(x0 + (int64_t)j * N + e, NX));
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (j0 + 32 * h < nin) out[L + j0 + 32 * h] = pack_chunk<DT>(x[h], scale);
        }
        if (lane < 2 * L) {
            // lanes 0 .. L-1: left chunks (halo at the end of chunk L-1); lanes L .. 2L-1: right chunks
            float x[N];
#pragma unroll
            for (int e = 0; e < N; ++e) x[e] = 0.f;
            if (lane == L - 1) x[N - 1] = __ldg(rowp + clamp64(x0 - 1, NX));
            if (lane == L) x[0] = __ldg(rowp + clamp64(x0 + g.B, NX));
            out[lane < L ? lane : nin + lane] = pack_chunk<DT>(x, scale);
        }
    }
}

// Per-brick metadata to the host: brick extrema, non-finite counts, sums,
// halo-inclusive maxima.  Issued last on the upload stream; the device-to-
// pageable copies return when they are done.
vrc_status fetch_metadata(vrc_ctx *ctx, Cube *c, cudaStream_t st, const double *dbsum, std::vector<double> &bsum)
{
    const BrickGeom &g = c->g;
    bsum.resize(2 * g.nbricks);
    c->h_bmin.resize(g.nbricks);
    c->h_bmax.resize(g.nbricks);
    c->h_bnonfinite.resize(g.nbricks);
    c->h_bhalo_max.resize(g.nbricks);
    VRC_CK(ctx, cudaMemcpyAsync(bsum.data(), dbsum, g.nbricks * 16, cudaMemcpyDeviceToHost, st));
    VRC_CK(ctx, cudaMemcpyAsync(c->h_bmin.data(), c->bmin, g.nbricks * 4, cudaMemcpyDeviceToHost, st));
    VRC_CK(ctx, cudaMemcpyAsync(c->h_bmax.data(), c->bmax, g.nbricks * 4, cudaMemcpyDeviceToHost, st));
    VRC_CK(ctx, cudaMemcpyAsync(c->h_bnonfinite.data(), c->bnonfinite, g.nbricks * 4, cudaMemcpyDeviceToHost, st));
    VRC_CK(ctx, cudaMemcpyAsync(c->h_bhalo_max.data(), c->bhalo, g.nbricks * 4, cudaMemcpyDeviceToHost, st));
    return VRC_OK;
}

// Cube extrema (TF range) and the statistics shift from the per-brick values.
void finish_metadata(Cube *c, const std::vector<double> &bsum)
{
    const BrickGeom &g = c->g;
    float mn = FLT_MAX, mx = -FLT_MAX;
    bool any = false;
    for (int64_t b = 0; b < g.nbricks; ++b) {
        if (c->h_bmin[b] <= c->h_bmax[b]) {
            any = true;
            mn = std::fmin(mn, c->h_bmin[b]);
            mx = std::fmax(mx, c->h_bmax[b]);
        }
    }
    c->has_finite = any;
    c->vmin = any ? mn : 0.f;
    c->vmax = any ? mx : 0.f;
    double tot = 0, cnt = 0;
    for (int64_t b = 0; b < g.nbricks; ++b) {
        tot += bsum[2 * b];
        cnt += bsum[2 * b + 1];
    }
    c->shift = cnt > 0 ? (float)(tot / cnt) : 0.f;
    if (!std::isfinite(c->shift)) c->shift = c->vmin;
}

// Copy the packed bricks (interior + halo) into their layered CUDA arrays
// through surfaces: stored element (sx, sy, sz) of brick b goes to texel
// (sx, sy, layer sz) of array b, i.e. layers along z.  One launch for all
// bricks.  A warp copies a pair of rows (sy, sy + 1) of one layer at a time:
// half-warps take the two rows, 16 texels each per store, so that one store
// covers whole 2-row blocks of the array's tiled layout instead of leaving
// partly written sectors behind (a warp per row measured 4.2 ms on a 1024^3
// fp32 cube, with 2x the DRAM reads).  R = B + 2 is even.  The surface
// handles come from `surfs`.
// BF16 and FP8 copies pack two stored layers per texel (layer j holds layers
// j and j + 1, the lower layer in the low bits; B + 1 layers), so that the
// renderer's single 2x2 gather returns a whole trilinear footprint: BF16 as
// 32-bit texels of two bf16 bit patterns, FP8 as 16-bit texels of two e4m3
// codes (the per-brick scale is applied after the lerps).
struct Bf16Pair {};
struct Fp8Pair {};
template <typename T> struct TexElem {
    using type = T;
    static constexpr bool pair = false;
};
template <> struct TexElem<Bf16Pair> {
    using type = unsigned int;
    static constexpr bool pair = true;
};
template <> struct TexElem<Fp8Pair> {
    using type = unsigned short;
    static constexpr bool pair = true;
};

// Texel of stored element e (S = elements per stored layer).
template <typename T>
__device__ __forceinline__ typename TexElem<T>::type tex_value(const uint8_t *brick, int64_t e, int64_t S)
{
    if constexpr (std::is_same<T, Bf16Pair>::value) {
        const unsigned short *h = reinterpret_cast<const unsigned short *>(brick);
        return (unsigned int)h[e] | ((unsigned int)h[e + S] << 16);
    } else if constexpr (std::is_same<T, Fp8Pair>::value) {
        return (unsigned short)(brick[e] | (brick[e + S] << 8));
    } else {
        return reinterpret_cast<const T *>(brick)[e];
    }
}

constexpr int kFillK = 17;   // 16-texel steps per lane in flight (a B = 256 row is 258 texels: 17 steps)
template <typename T>
__global__ void __launch_bounds__(256) k_fill_copy(const uint8_t *__restrict__ pool, BrickGeom g,
                                                   const unsigned long long *__restrict__ surfs)
{
    using E = typename TexElem<T>::type;
    const int R = g.R, lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const int NL = TexElem<T>::pair ? R - 1 : R;   // layers of the copy
    const int64_t S = (int64_t)R * g.P;
    const int64_t pairs = (int64_t)NL * (R >> 1), total = pairs * g.nbricks;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < total; w += nw) {
        const int64_t b = w / pairs;
        const int p = (int)(w - b * pairs);
        const int layer = p / (R >> 1), v = 2 * (p - layer * (R >> 1)) + half;
        const uint8_t *brick = pool + b * g.brick_bytes;
        const cudaSurfaceObject_t surf = surfs[b];
        const int64_t e0 = ((int64_t)layer * R + v) * g.P + (g.O - 1);
        for (int u0 = 0; u0 < R; u0 += 16 * kFillK) {
            E val[kFillK];
#pragma unroll
            for (int k = 0; k < kFillK; ++k) {
                const int u = u0 + hl + 16 * k;
                val[k] = u < R ? tex_value<T>(brick, e0 + u, S) : E();
            }
#pragma unroll
            for (int k = 0; k < kFillK; ++k) {
                const int u = u0 + hl + 16 * k;
                if (u < R) surf2DLayeredwrite(val[k], surf, u * (int)sizeof(E), v, layer);
            }
        }
    }
}

template <int DT>
__device__ __forceinline__ float stored_at(const uint8_t *bp, int64_t e, float scale)
{
    if (DT == VRC_F32) return reinterpret_cast<const float *>(bp)[e];
    if (DT == VRC_BF16) return __uint_as_float((uint32_t)reinterpret_cast<const unsigned short *>(bp)[e] << 16);
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)bp[e], __NV_E4M3);
    return __fmul_rn(__half2float(__half(h)), scale);
}

// Stored values of a resident cube back into a linear float array (x
// fastest, interior voxels only): the source of a re-pack at another brick
// size (autotuner).  One thread per voxel, grid-stride.
template <int DT>
__global__ void k_unpack(const uint8_t *__restrict__ pool, BrickGeom g, const float *__restrict__ scales,
                         float *__restrict__ out)
{
    const int64_t n = g.dims[0] * g.dims[1] * g.dims[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % g.dims[0], yz = i / g.dims[0], y = yz % g.dims[1], z = yz / g.dims[1];
        const int64_t bx = x >> g.logB, by = y >> g.logB, bz = z >> g.logB;
        const int64_t b = (bz * g.nb[1] + by) * g.nb[0] + bx;
        const int64_t lx = x - (bx << g.logB), ly = y - (by << g.logB), lz = z - (bz << g.logB);
        const int64_t e = ((lz + 1) * g.R + (ly + 1)) * g.P + lx + g.O;
        out[i] = stored_at<DT>(pool + b * g.brick_bytes, e, DT == VRC_FP8E4M3 ? scales[b] : 1.f);
    }
}

// Maximum stored value over local voxels [8l-1, 8l+8]^3 of each 8^3 macro-cell
// l of each brick (the brick's own copy, so FP8 halos use the brick's scale).
// NaN voxels never raise the maximum.  One block per (brick, layer of cells),
// one thread per stored column sx (local x = sx - 1): the thread takes the
// maximum over the layer's ten stored planes row by row and folds each row
// into the cell rows whose windows hold it (stored rows 8c .. 8c+9 form cell
// row c); the column maxima then reduce over each cell's ten columns in
// shared memory.
template <int DT>
__global__ void k_cell_max(const uint8_t *__restrict__ pool, BrickGeom g, const float *__restrict__ scales,
                           int ncx, int ncy, float *__restrict__ cellmax)
{
    extern __shared__ float colmax[];   // [cpb][R]
    const int cpb = g.B >> 3, R = g.R;
    const int64_t b = blockIdx.x;
    const int lzc = blockIdx.y, sx = threadIdx.x;
    const uint8_t *bp = pool + b * g.brick_bytes;
    const float scale = scales[b];
    if (sx < R) {
        float cur = -INFINITY, prev = -INFINITY;
        for (int sy = 0; sy < R; ++sy) {
            float m = -INFINITY;
#pragma unroll
            for (int k = 0; k < 10; ++k)
                m = fmaxf(m, stored_at<DT>(bp, ((int64_t)(8 * lzc + k) * R + sy) * g.P + (g.O - 1) + sx, scale));
            const int c = sy >> 3, q = sy & 7;
            if (q == 0) {
                prev = cur;
                cur = -INFINITY;
            }
            if (q <= 1 && c >= 1) {
                prev = fmaxf(prev, m);
                if (q == 1) colmax[(c - 1) * R + sx] = prev;
            }
            cur = fmaxf(cur, m);
        }
    }
    __syncthreads();
    const int bx = (int)(b % g.nb[0]), by = (int)((b / g.nb[0]) % g.nb[1]), bz = (int)(b / ((int64_t)g.nb[0] * g.nb[1]));
    for (int i = threadIdx.x; i < cpb * cpb; i += blockDim.x) {
        const int cy = i / cpb, cx = i - cy * cpb;
        float m = -INFINITY;
#pragma unroll
        for (int x = 0; x < 10; ++x) m = fmaxf(m, colmax[cy * R + 8 * cx + x]);
        cellmax[((int64_t)(bz * cpb + lzc) * ncy + (by * cpb + cy)) * ncx + (bx * cpb + cx)] = m;
    }
}

// Largest cell maximum of each brick (the cells with their margins cover the
// brick's interior and halo).  One block per brick.
__global__ void k_brick_halo_max(const float *__restrict__ cellmax, BrickGeom g, int ncx, int ncy, int cpb,
                                 float *__restrict__ bhalo)
{
    const int b = blockIdx.x;
    const int bx = b % g.nb[0], by = (b / g.nb[0]) % g.nb[1], bz = b / (g.nb[0] * g.nb[1]);
    const int n = cpb * cpb * cpb;
    float m = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int lx = i % cpb, ly = (i / cpb) % cpb, lz = i / (cpb * cpb);
        const int64_t cell = ((int64_t)(bz * cpb + lz) * ncy + (by * cpb + ly)) * ncx + (bx * cpb + lx);
        m = fmaxf(m, cellmax[cell]);
    }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wm[w]);
        bhalo[b] = m;
    }
}

vrc_status alloc_cellmax(vrc_ctx *ctx, Cube *c)
{
    const BrickGeom &g = c->g;
    const int cpb = g.B / 8;
    for (int a = 0; a < 3; ++a) c->ncell[a] = g.nb[a] * cpb;
    const int64_t n = (int64_t)c->ncell[0] * c->ncell[1] * c->ncell[2];
    return dev_alloc(ctx, (void **)&c->cellmax, n * 4);
}

vrc_status launch_cellmax(vrc_ctx *ctx, Cube *c, cudaStream_t st)
{
    const BrickGeom &g = c->g;
    const int cpb = g.B / 8;
    const dim3 grid((unsigned)g.nbricks, (unsigned)cpb);
    const int threads = (g.R + 31) / 32 * 32;
    const size_t smem = (size_t)cpb * g.R * sizeof(float);
    auto launch = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<grid, threads, smem, st>>>((const uint8_t *)c->pool, g, c->scales, c->ncell[0], c->ncell[1],
                                          c->cellmax);
        return cudaGetLastError();
    };
    cudaError_t e = g.dtype == VRC_F32    ? launch(k_cell_max<VRC_F32>)
                    : g.dtype == VRC_BF16 ? launch(k_cell_max<VRC_BF16>)
                                          : launch(k_cell_max<VRC_FP8E4M3>);
    if (e != cudaSuccess) return cuda_err(ctx, e, "macro-cell maxima");
    k_brick_halo_max<<<(unsigned)g.nbricks, 256, 0, st>>>(c->cellmax, g, c->ncell[0], c->ncell[1], cpb, c->bhalo);
    count_launch(ctx, 2);
    VRC_CK(ctx, cudaGetLastError());
    return VRC_OK;
}

static uint64_t tex_array_key(const BrickGeom &g) { return ((uint64_t)g.R << 8) | (uint64_t)g.dtype; }

// Return the cube's render copies to the context's cache (the arrays keep
// their surface and texture objects).  The caller guarantees no work in
// flight reads them.
void release_textures(vrc_ctx *ctx, Cube *c)
{
    for (const TexArray &a : c->tex_arrays) tex_array_give(ctx, tex_array_key(c->g), a);
    c->tex_arrays.clear();
    if (c->dtex) dev_free(ctx, c->dtex, 4 * c->g.nbricks * 8);
    c->dtex = nullptr;
    c->tex_axes = 0;
    ctx->used.fetch_sub(c->tex_bytes);
    c->tex_bytes = 0;
}

// Allocate the render copy (one 2D-layered array per brick, layers along z)
// as long as it fits the budget; charged to the budget.  Arrays come from the
// context's cache when a freed cube left some of this shape.  Only host work:
// it may run while earlier work still occupies the device.
vrc_status alloc_textures(vrc_ctx *ctx, Cube *c)
{
    const BrickGeom &g = c->g;
    // fp32: one texel per stored voxel, R layers; bf16 / fp8: two stored
    // layers per texel (32 / 16 bits), R - 1 layers
    const int64_t tex_esize = g.dtype == VRC_F32 ? 4 : 2 * g.esize;
    const int64_t tex_layers = g.dtype == VRC_F32 ? g.R : g.R - 1;
    const int64_t arr_bytes = tex_esize * (int64_t)g.R * g.R * tex_layers;
    const int64_t per_copy = arr_bytes * g.nbricks + (1 << 20);
    // optional copies leave room in the budget for the render scratch of a
    // large multi-view call; a required copy is charged as it is
    const int64_t reserve = c->copy_mode == VRC_COPY_REQUIRED ? 0 : (int64_t)2 << 30;
    if (ctx->used.load() + per_copy + reserve > ctx->budget &&
        !(reap_pending(ctx, true) && ctx->used.load() + per_copy + reserve <= ctx->budget))
        return set_err(ctx, VRC_E_NOMEM, "budget: no room for texture copies");
    vrc_status s = dev_alloc(ctx, (void **)&c->dtex, 4 * g.nbricks * 8);
    if (s != VRC_OK) return s;
    ctx->used.fetch_add(per_copy);
    c->tex_bytes += per_copy;
    cudaChannelFormatDesc desc = g.dtype == VRC_F32 ? cudaCreateChannelDesc<float>()
                               : (g.dtype == VRC_BF16 ? cudaCreateChannelDesc<unsigned int>()
                                                      : cudaCreateChannelDesc<unsigned short>());
    const uint64_t key = tex_array_key(g);
    c->h_tex.assign(4 * g.nbricks, 0ull);
    for (int64_t b = 0; b < g.nbricks; ++b) {
        if (inject_fire(ctx, VRC_INJECT_ALLOC)) return set_err(ctx, VRC_E_NOMEM, "injected allocation failure");
        TexArray a;
        if (!tex_array_take(ctx, key, &a)) {
            cache_trim(ctx, std::max<int64_t>(0, ctx->budget - ctx->used.load()));
            a.bytes = arr_bytes;
            cudaError_t e = cudaMalloc3DArray(&a.arr, &desc, make_cudaExtent(g.R, g.R, tex_layers),
                                              cudaArrayLayered | cudaArraySurfaceLoadStore);
            cudaResourceDesc rd = {};
            rd.resType = cudaResourceTypeArray;
            rd.res.array.array = a.arr;
            if (e == cudaSuccess) e = cudaCreateSurfaceObject(&a.surf, &rd);
            cudaTextureDesc td = {};
            td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
            td.filterMode = cudaFilterModePoint;
            td.readMode = cudaReadModeElementType;
            td.normalizedCoords = 0;
            if (e == cudaSuccess) e = cudaCreateTextureObject(&a.tex, &rd, &td, nullptr);
            if (e != cudaSuccess) {
                cudaGetLastError();
                destroy_tex_array(a);
                return cuda_err(ctx, e, "render copy array");
            }
        }
        c->tex_arrays.push_back(a);
        c->h_tex[2 * g.nbricks + b] = a.tex;    // the z-layered copy
        c->h_tex[3 * g.nbricks + b] = a.surf;   // its surface, for the fill
    }
    return VRC_OK;
}

// Upload the table of texture handles (the z copy; x and y entries are 0)
// followed by the surface handles, then fill the render copy from the packed
// bricks in one launch.  (Writing the copy from k_brick_pack instead measured
// 6.6 ms against 4.9 ms for the two passes on a 1024^3 cube.)
vrc_status launch_textures(vrc_ctx *ctx, Cube *c, cudaStream_t st)
{
    const BrickGeom &g = c->g;
    vrc_status s = stage_h2d(ctx, st, {{c->dtex, c->h_tex.data(), (size_t)8 * 4 * g.nbricks}});
    if (s != VRC_OK) return s;
    const unsigned long long *surfs = reinterpret_cast<const unsigned long long *>(c->dtex) + 3 * g.nbricks;
    const uint8_t *pool = (const uint8_t *)c->pool;
    const unsigned grid = (unsigned)ctx->sm_count * 8;
    if (g.dtype == VRC_F32) k_fill_copy<float><<<grid, 256, 0, st>>>(pool, g, surfs);
    else if (g.dtype == VRC_BF16) k_fill_copy<Bf16Pair><<<grid, 256, 0, st>>>(pool, g, surfs);
    else k_fill_copy<Fp8Pair><<<grid, 256, 0, st>>>(pool, g, surfs);
    count_launch(ctx);
    VRC_CK(ctx, cudaGetLastError());
    c->tex_axes |= 1 << 2;
    return VRC_OK;
}

}  // namespace

// Give back every device allocation of a cube (bricks, metadata, render copy,
// halo copy, ring) and clear the pointers; the record itself stays.
void release_device(vrc_ctx *ctx, Cube *c, bool sync)
{
    const BrickGeom &g = c->g;
    // the memory goes back to the context's cache and may be handed out at
    // once: no launch still in flight may read it (the caller's event
    // guarantees that when sync is false)
    if (sync) cudaDeviceSynchronize();
    release_textures(ctx, c);
    slab_release(ctx, c);
    if (c->pool) dev_free(ctx, c->pool, g.nbricks * g.brick_bytes);
    if (c->ring_pool) dev_free(ctx, c->ring_pool, (size_t)c->ring * g.brick_bytes);
    if (c->scales) dev_free(ctx, c->scales, g.nbricks * 4);
    if (c->cellmax) dev_free(ctx, c->cellmax, (int64_t)c->ncell[0] * c->ncell[1] * c->ncell[2] * 4);
    if (c->bmin) dev_free(ctx, c->bmin, g.nbricks * 4);
    if (c->bmax) dev_free(ctx, c->bmax, g.nbricks * 4);
    if (c->bnonfinite) dev_free(ctx, c->bnonfinite, g.nbricks * 4);
    if (c->bhalo) dev_free(ctx, c->bhalo, g.nbricks * 4);
    if (c->pack_src) dev_free(ctx, c->pack_src, (size_t)g.R * g.R * g.R * sizeof(float));
    if (c->pack_out) dev_free(ctx, c->pack_out, (size_t)g.brick_bytes);
    c->pack_src = c->pack_out = nullptr;
    c->pool = c->ring_pool = nullptr;
    c->scales = c->cellmax = c->bmin = c->bmax = c->bhalo = nullptr;
    c->bnonfinite = nullptr;
    c->h_tex.clear();
}

void release_cube(vrc_ctx *ctx, Cube *c, bool sync)
{
    release_device(ctx, c, sync);
    if (c->host_pool) cudaFreeHost(c->host_pool);
    if (c->host_pinned) cudaHostUnregister((void *)c->host_src);
    if (c->host_packed) cudaFreeHost(c->host_packed);
    if (c->pack_stream) cudaStreamDestroy(c->pack_stream);
    if (c->source_pinned) cudaHostUnregister(c->source_buf.data());
    for (cudaEvent_t e : c->slot_ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

int64_t register_cube(vrc_ctx *ctx, Cube *c)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    c->id = ctx->next_id++;
    ctx->cubes[c->id] = c;
    return c->id;
}

namespace {

vrc_status alloc_meta(vrc_ctx *ctx, Cube *c)
{
    const int64_t n = c->g.nbricks;
    vrc_status s;
    if ((s = dev_alloc(ctx, (void **)&c->scales, n * 4)) != VRC_OK) return s;
    if ((s = dev_alloc(ctx, (void **)&c->bmin, n * 4)) != VRC_OK) return s;
    if ((s = dev_alloc(ctx, (void **)&c->bmax, n * 4)) != VRC_OK) return s;
    if ((s = dev_alloc(ctx, (void **)&c->bnonfinite, n * 4)) != VRC_OK) return s;
    if ((s = dev_alloc(ctx, (void **)&c->bhalo, n * 4)) != VRC_OK) return s;
    return VRC_OK;
}


// Extrema and sums of one host brick (Sec. 2: sub-cubes of a cube larger
// than memory): interior voxels inside the cube, plus the largest value a
// sample can read (halo included) for brick culling.
struct BrickMeta {
    float mn = FLT_MAX, mx = -FLT_MAX, hmx = -INFINITY;
    int32_t nnf = 0;
    double sum = 0.0;
    int64_t cnt = 0;
};

// Measure z-planes [z0, z1) of provided brick `bw` ((B+2)^3 floats, x
// fastest): interior extrema, sum (per row in binary32, rows in binary64: it
// only centres the statistics) and non-finite count, the halo-inclusive
// maximum (NaN ignored, +inf kept) and the largest finite magnitude (halo
// included: the FP8 scale's absmax).  rows: float32 host-slot storage to fill
// in the same pass (rows of P elements, the halo voxel at element O-1,
// padding 0), or null.
void measure_planes(const BrickGeom &g, const float *bw, int z0, int z1, BrickMeta *m, float *absmax, float *rows)
{
    const int R = g.R, B = g.B;
    float hmx = -INFINITY, am = 0.f, mn = FLT_MAX, mx = -FLT_MAX;
    int32_t nnf = 0;
    int64_t cnt = 0;
    double sum = 0.0;
    for (int zr = z0; zr < z1; ++zr)
        for (int yr = 0; yr < R; ++yr) {
            const float *in = bw + ((int64_t)zr * R + yr) * R;
            if (rows) {
                float *row = rows + ((int64_t)zr * R + yr) * g.P;
                std::memset(row, 0, sizeof(float) * g.P);
                std::memcpy(row + g.O - 1, in, sizeof(float) * R);
            }
            if (!m) continue;
            for (int x = 0; x < R; ++x) {
                const float v = in[x], a = std::fabs(v);
                hmx = v > hmx ? v : hmx;
                am = a <= FLT_MAX && a > am ? a : am;
            }
            if (zr >= 1 && zr <= B && yr >= 1 && yr <= B) {
                float rs = 0.f;
                int rc = 0;
                for (int x = 1; x <= B; ++x) {
                    const float v = in[x];
                    const bool fin = std::fabs(v) <= FLT_MAX;
                    mn = fin && v < mn ? v : mn;
                    mx = fin && v > mx ? v : mx;
                    rs += fin ? v : 0.f;
                    rc += fin;
                }
                sum += rs;
                cnt += rc;
                nnf += B - rc;
            }
        }
    if (!m) return;
    m->hmx = hmx;
    m->mn = mn;
    m->mx = mx;
    m->nnf = nnf;
    m->cnt = cnt;
    m->sum = sum;
    *absmax = am;
}

// measure_planes over the whole brick, split by z-planes over host threads
// for large bricks (merged in plane order: the result does not depend on
// timing).
void measure_brick(const BrickGeom &g, const float *bw, BrickMeta *m, float *absmax, float *rows)
{
    const int R = g.R;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = (int64_t)R * R * R < (1 << 20) ? 1 : (int)std::min<unsigned>(hw, 16u);
    if (nt == 1) {
        measure_planes(g, bw, 0, R, m, absmax, rows);
        return;
    }
    std::vector<BrickMeta> part(nt);
    std::vector<float> am(nt, 0.f);
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back(measure_planes, std::cref(g), bw, R * t / nt, R * (t + 1) / nt, m ? &part[t] : nullptr,
                        &am[t], rows);
    for (std::thread &x : th) x.join();
    if (!m) return;
    BrickMeta r;
    float a = 0.f;
    for (int t = 0; t < nt; ++t) {
        r.hmx = part[t].hmx > r.hmx ? part[t].hmx : r.hmx;
        r.mn = std::min(r.mn, part[t].mn);
        r.mx = std::max(r.mx, part[t].mx);
        r.nnf += part[t].nnf;
        r.cnt += part[t].cnt;
        r.sum += part[t].sum;
        a = std::max(a, am[t]);
    }
    *m = r;
    *absmax = a;
}

// Store provided brick b (`bw`, (B+2)^3 floats) in host slot `slot` (rows of
// P elements, the halo voxel at element O-1), measuring it when m is given.
// float32: copied on the host.  bf16 / fp8: packed on the device as the
// upload packs (the brick's FP8 scale from the measured absmax when measuring,
// else the recorded one) and copied back into the slot.
vrc_status pack_host_slot(vrc_ctx *ctx, Cube *c, int64_t slot, int64_t b, const float *bw, BrickMeta *m)
{
    const BrickGeom &g = c->g;
    const int R = g.R;
    float absmax = 0.f;
    char *dst = (char *)c->host_pool + slot * g.brick_bytes;
    if (g.dtype == VRC_F32) {
        measure_brick(g, bw, m, &absmax, reinterpret_cast<float *>(dst));
        return VRC_OK;
    }
    if (m) measure_brick(g, bw, m, &absmax, nullptr);
    if (m) c->h_scales[b] = g.dtype == VRC_FP8E4M3 && absmax > 0.f ? absmax / 448.f : 1.f;
    const float scale = c->h_scales[b];
    const size_t nsrc = (size_t)R * R * R * sizeof(float);
    cudaStream_t ps = c->pack_stream;
    VRC_CK(ctx, cudaMemcpyAsync(c->pack_src, bw, nsrc, cudaMemcpyHostToDevice, ps));
    const unsigned grid = (unsigned)std::min<int64_t>((int64_t)R * R, 4096);
    if (g.dtype == VRC_BF16)
        k_pack_provided<VRC_BF16><<<grid, 128, 0, ps>>>((const float *)c->pack_src, g, scale, (uint8_t *)c->pack_out);
    else
        k_pack_provided<VRC_FP8E4M3><<<grid, 128, 0, ps>>>((const float *)c->pack_src, g, scale,
                                                           (uint8_t *)c->pack_out);
    count_launch(ctx);
    VRC_CK(ctx, cudaGetLastError());
    VRC_CK(ctx, cudaMemcpyAsync(dst, c->pack_out, (size_t)g.brick_bytes, cudaMemcpyDeviceToHost, ps));
    VRC_CK(ctx, cudaStreamSynchronize(ps));
    return VRC_OK;
}

// Record brick b's measurements.  For a brick on the cube's far border the
// measured B^3 interior includes positions past the cube, which repeat edge
// voxels: the extrema are unchanged, the sum only centres the statistics, and
// the non-finite count only steers the statistics pass to its checked path
// (the pass counts non-finite voxels itself, inside the cube).
void set_brick_meta(Cube *c, int64_t b, const BrickMeta &m)
{
    c->h_bmin[b] = m.mn;
    c->h_bmax[b] = m.mx;
    c->h_bnonfinite[b] = m.nnf;
    c->h_bhalo_max[b] = m.hmx;
    c->h_bsum[b] = m.sum;
    c->h_bcnt[b] = m.cnt;
}

// Cube extrema and the statistics centre from the per-brick records.
void finish_streamed_meta(Cube *c)
{
    float vmn = FLT_MAX, vmx = -FLT_MAX;
    double sum = 0.0;
    int64_t cnt = 0;
    for (int64_t b = 0; b < c->g.nbricks; ++b) {
        if (c->h_bmin[b] <= c->h_bmax[b]) {
            vmn = std::fmin(vmn, c->h_bmin[b]);
            vmx = std::fmax(vmx, c->h_bmax[b]);
        }
        sum += c->h_bsum[b];
        cnt += c->h_bcnt[b];
    }
    c->has_finite = vmn <= vmx;
    c->vmin = c->has_finite ? vmn : 0.f;
    c->vmax = c->has_finite ? vmx : 0.f;
    c->shift = cnt ? (float)(sum / (double)cnt) : 0.f;
    if (!std::isfinite(c->shift)) c->shift = c->vmin;
}

// Ask the provider for brick b into c->source_buf.
vrc_status call_source(vrc_ctx *ctx, Cube *c, int64_t b)
{
    const BrickGeom &g = c->g;
    const int32_t bx = (int32_t)(b % g.nb[0]), by = (int32_t)((b / g.nb[0]) % g.nb[1]),
                  bz = (int32_t)(b / ((int64_t)g.nb[0] * g.nb[1]));
    ++c->source_calls;
    const int32_t rc = c->source(c->source_user, b, bx, by, bz, c->source_buf.data());
    if (rc != 0) return set_err(ctx, VRC_E_SOURCE, "brick provider failed on brick %lld (returned %d)", (long long)b, rc);
    return VRC_OK;
}

}  // namespace

// Make cube c (geometry and render-copy mode set) resident from `src`: the
// upload passes of vrc_cube_upload on `st`.  On failure every device
// allocation of c is given back.
vrc_status upload_cube(vrc_ctx *ctx, Cube *c, const float *src, int32_t src_on_device, cudaStream_t st)
{
    const BrickGeom &g = c->g;
    const int32_t storage = g.dtype;
    const int64_t nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    // 1. every allocation first (host work that overlaps earlier device work)
    vrc_status s = dev_alloc(ctx, &c->pool, g.nbricks * g.brick_bytes);
    if (s == VRC_OK) s = alloc_meta(ctx, c);
    if (s == VRC_OK) s = alloc_cellmax(ctx, c);
    void *staging = nullptr;
    const size_t src_bytes = (size_t)(nx * ny * nz) * 4;
    if (s == VRC_OK && !src_on_device) s = dev_alloc(ctx, &staging, src_bytes);
    ScanPartial *part = nullptr;
    const int split = blocks_per_brick(ctx, storage == VRC_FP8E4M3 ? (const void *)k_brick_scan<true>
                                                                   : (const void *)k_brick_scan<false>,
                                       g.nbricks, (int64_t)g.B * g.B);
    const size_t part_bytes = g.nbricks * (split * sizeof(ScanPartial) + 16);
    if (s == VRC_OK) s = dev_alloc(ctx, (void **)&part, part_bytes);
    double *dbsum = part ? reinterpret_cast<double *>(part + g.nbricks * split) : nullptr;
    bool tex = false;
    if (s == VRC_OK && c->copy_mode == VRC_COPY_REQUIRED) {
        tex = (s = alloc_textures(ctx, c)) == VRC_OK;
    } else if (s == VRC_OK && c->copy_mode == VRC_COPY_AUTO && getenv("VRC_NO_TEXTURES") == nullptr) {
        // texture copies are an accelerator: without room for them the cube still
        // renders (vrc_last_render_path then reports the global-load path)
        tex = alloc_textures(ctx, c) == VRC_OK;
        if (!tex) {
            release_textures(ctx, c);
            fprintf(stderr, "vrc: no texture render copies for this cube (%s)\n", vrc_last_error(ctx));
        }
    }
    // 2. the device work, in stream order
    const float *dsrc = src;
    if (s == VRC_OK && staging) {
        cudaError_t e = cudaMemcpyAsync(staging, src, src_bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = cuda_err(ctx, e, "cube upload H2D");
        dsrc = (const float *)staging;
    }
    if (s == VRC_OK) {
        const dim3 grid((unsigned)g.nbricks, (unsigned)split);
        if (storage == VRC_FP8E4M3) k_brick_scan<true><<<grid, 256, 0, st>>>(dsrc, g, split, part);
        else k_brick_scan<false><<<grid, 256, 0, st>>>(dsrc, g, split, part);
        k_brick_finish<<<(unsigned)((g.nbricks + 127) / 128), 128, 0, st>>>(part, g, split, c->scales, c->bmin,
                                                                            c->bmax, c->bnonfinite, dbsum);
        const void *pk = storage == VRC_F32    ? (const void *)k_brick_pack<VRC_F32>
                         : storage == VRC_BF16 ? (const void *)k_brick_pack<VRC_BF16>
                                               : (const void *)k_brick_pack<VRC_FP8E4M3>;
        const int psplit = blocks_per_brick(ctx, pk, g.nbricks, (int64_t)g.R * g.R);
        const dim3 pgrid((unsigned)g.nbricks, (unsigned)psplit);
        if (storage == VRC_F32) k_brick_pack<VRC_F32><<<pgrid, 256, 0, st>>>(dsrc, g, psplit, c->scales, c->pool);
        else if (storage == VRC_BF16) k_brick_pack<VRC_BF16><<<pgrid, 256, 0, st>>>(dsrc, g, psplit, c->scales, c->pool);
        else k_brick_pack<VRC_FP8E4M3><<<pgrid, 256, 0, st>>>(dsrc, g, psplit, c->scales, c->pool);
        count_launch(ctx, 3);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_err(ctx, e, "brick pack launch");
    }
    if (s == VRC_OK) s = launch_cellmax(ctx, c, st);
    if (s == VRC_OK && tex) s = launch_textures(ctx, c, st);
    std::vector<double> bsum;
    if (s == VRC_OK) s = fetch_metadata(ctx, c, st, dbsum, bsum);
    // 3. one wait, then the host-side metadata
    cudaError_t e = cudaStreamSynchronize(st);
    if (s == VRC_OK && e != cudaSuccess) s = cuda_err(ctx, e, "cube upload");
    if (s == VRC_OK) finish_metadata(c, bsum);
    if (part) dev_free(ctx, part, part_bytes);
    if (staging) dev_free(ctx, staging, src_bytes);
    if (s != VRC_OK) {
        release_device(ctx, c, true);
        return s;
    }
    c->charged = g.nbricks * g.brick_bytes + 16 * g.nbricks;
    return VRC_OK;
}

namespace {

// Resident bricks of a registered cube from its packed host copy: the bricks,
// brick scales and extrema are copied (the host kept them since the
// registration), the macro-cell maxima and the render copy are rebuilt on the
// device.  On failure every device allocation of c is given back.
vrc_status upload_packed(vrc_ctx *ctx, Cube *c, cudaStream_t st)
{
    const BrickGeom &g = c->g;
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    vrc_status s = dev_alloc(ctx, &c->pool, g.nbricks * g.brick_bytes);
    if (s == VRC_OK) s = alloc_meta(ctx, c);
    if (s == VRC_OK) s = alloc_cellmax(ctx, c);
    bool tex = false;
    if (s == VRC_OK && c->copy_mode == VRC_COPY_REQUIRED) tex = (s = alloc_textures(ctx, c)) == VRC_OK;
    const int64_t nb4 = g.nbricks * 4;
    auto h2d = [&](void *dst, const void *src, size_t n) {
        if (s != VRC_OK) return;
        const cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = cuda_err(ctx, e, "packed cube H2D");
    };
    h2d(c->pool, c->host_packed, (size_t)(g.nbricks * g.brick_bytes));
    h2d(c->scales, c->h_scales.data(), nb4);
    h2d(c->bmin, c->h_bmin.data(), nb4);
    h2d(c->bmax, c->h_bmax.data(), nb4);
    h2d(c->bnonfinite, c->h_bnonfinite.data(), nb4);
    if (s == VRC_OK) s = launch_cellmax(ctx, c, st);
    if (s == VRC_OK && tex) s = launch_textures(ctx, c, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (s == VRC_OK && e != cudaSuccess) s = cuda_err(ctx, e, "packed cube upload");
    if (s != VRC_OK) {
        release_device(ctx, c, true);
        return s;
    }
    c->charged = g.nbricks * g.brick_bytes + 16 * g.nbricks;
    return VRC_OK;
}

// Keep the packed bricks and scales of a resident bf16 / fp8 cube in
// page-locked host memory.  False (nothing kept) when the host memory cannot
// be had or a copy fails.
bool save_packed(vrc_ctx *ctx, Cube *c, cudaStream_t st)
{
    const BrickGeom &g = c->g;
    const size_t n = (size_t)(g.nbricks * g.brick_bytes);
    void *h = nullptr;
    if (cudaHostAlloc(&h, n, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    c->h_scales.resize(g.nbricks);
    if (cudaMemcpyAsync(h, c->pool, n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(c->h_scales.data(), c->scales, g.nbricks * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(h);
        return false;
    }
    c->host_packed = h;
    return true;
}

}  // namespace

vrc_status load_registered(vrc_ctx *ctx, Cube *c, cudaStream_t st)
{
    if (c->host_packed) return upload_packed(ctx, c, st);
    return upload_cube(ctx, c, c->host_src, 0, st);
}

extern "C" {

vrc_status vrc_cube_upload(vrc_ctx *ctx, const float *src, int32_t src_on_device, int64_t nx, int64_t ny,
                           int64_t nz, int32_t storage, int32_t brick, void *stream, int64_t *cube_id)
{
    if (!ctx || !src || !cube_id) return VRC_E_INVAL;
    if (src_on_device != 0 && src_on_device != 1) return set_err(ctx, VRC_E_INVAL, "src_on_device must be 0 or 1");
    const int32_t copy_mode = storage & VRC_COPY_MASK;
    if (copy_mode != VRC_COPY_AUTO && copy_mode != VRC_COPY_REQUIRED && copy_mode != VRC_COPY_NONE)
        return set_err(ctx, VRC_E_INVAL, "bad render-copy flags %d", copy_mode);
    BrickGeom g;
    if (!make_geom(nx, ny, nz, brick, storage & ~VRC_COPY_MASK, &g, 32))
        return set_err(ctx, VRC_E_INVAL, "bad dims/storage/brick (%lld %lld %lld, %d, %d)", (long long)nx,
                       (long long)ny, (long long)nz, storage, brick);
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    Cube *c = new (std::nothrow) Cube();
    if (!c) return VRC_E_NOMEM;
    c->g = g;
    c->copy_mode = copy_mode;
    const vrc_status s = upload_cube(ctx, c, src, src_on_device, (cudaStream_t)stream);
    if (s != VRC_OK) {
        delete c;
        return s;
    }
    *cube_id = register_cube(ctx, c);
    return VRC_OK;
}

vrc_status vrc_cube_register(vrc_ctx *ctx, const float *src, int64_t nx, int64_t ny, int64_t nz, int32_t storage,
                             int32_t brick, int64_t *cube_id)
{
    if (!ctx || !src || !cube_id) return VRC_E_INVAL;
    const int32_t copy_mode = storage & VRC_COPY_MASK;
    if (copy_mode != VRC_COPY_AUTO && copy_mode != VRC_COPY_REQUIRED && copy_mode != VRC_COPY_NONE)
        return set_err(ctx, VRC_E_INVAL, "bad render-copy flags %d", copy_mode);
    BrickGeom g;
    if (!make_geom(nx, ny, nz, brick, storage & ~VRC_COPY_MASK, &g, 32))
        return set_err(ctx, VRC_E_INVAL, "bad dims/storage/brick (%lld %lld %lld, %d, %d)", (long long)nx,
                       (long long)ny, (long long)nz, storage, brick);
    Cube *c = new (std::nothrow) Cube();
    if (!c) return VRC_E_NOMEM;
    c->g = g;
    // a registered cube keeps its render copy whenever it is resident: the
    // memory it needs is counted when the cube is admitted
    c->copy_mode = copy_mode == VRC_COPY_NONE ? VRC_COPY_NONE : VRC_COPY_REQUIRED;
    c->managed = true;
    c->host_src = src;
    c->state.store(CUBE_ABSENT);
    // page-lock the caller's array so that uploads copy at the link's speed;
    // an array already page-locked (by the caller or another registration) is
    // used as it is, and a failure only makes uploads slower
    auto pin = [&] {
        if (cudaSetDevice(ctx->device) == cudaSuccess &&
            cudaHostRegister((void *)src, (size_t)(nx * ny * nz) * sizeof(float), cudaHostRegisterPortable) ==
                cudaSuccess)
            c->host_pinned = true;
        else
            cudaGetLastError();
    };
    if (g.dtype == VRC_F32) {
        pin();
    } else {
        // bf16 / fp8: packed once now; the packed bricks (half / a quarter of
        // the source's bytes) stay in page-locked host memory and every later
        // load copies them, so the caller's array is not read again
        vrc_status s = VRC_OK;
        {
            std::unique_lock<std::mutex> lk(ctx->res_mu);
            if (!evict_for(ctx, upload_peak_bytes(c), c))
                s = set_err(ctx, VRC_E_NOMEM, "budget: no room to pack the registered cube");
            if (s == VRC_OK) s = upload_cube(ctx, c, src, 0, nullptr);
            if (s == VRC_OK) {
                c->state.store(CUBE_RESIDENT);
                c->loads = 1;
                c->last_use = host_ms();
            }
        }
        if (s != VRC_OK) {
            release_cube(ctx, c, true);
            return s;
        }
        // (the one copy of the source ran from pageable memory: page-locking a
        // large array costs more than that copy saves)
        if (!save_packed(ctx, c, nullptr)) pin();   // no packed copy: loads read src as for float32
    }
    *cube_id = register_cube(ctx, c);
    return VRC_OK;
}

namespace {

vrc_status create_streamed(vrc_ctx *ctx, int64_t nx, int64_t ny, int64_t nz, int32_t storage, int32_t brick,
                           int64_t n_host_bricks, int32_t ring_bricks, int64_t *cube_id)
{
    if (!ctx || !cube_id) return VRC_E_INVAL;
    BrickGeom g;
    if (!make_geom(nx, ny, nz, brick, storage, &g, 16)) return set_err(ctx, VRC_E_INVAL, "bad dims/storage/brick");
    if (n_host_bricks <= 0 || n_host_bricks > g.nbricks) return set_err(ctx, VRC_E_INVAL, "bad n_host_bricks");
    if (ring_bricks < 0 || ring_bricks > 4096) return set_err(ctx, VRC_E_INVAL, "bad ring_bricks");
    if (ring_bricks == 0) ring_bricks = 8;
    if (ring_bricks < 2) return set_err(ctx, VRC_E_INVAL, "ring needs at least 2 bricks");
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    Cube *c = new (std::nothrow) Cube();
    if (!c) return VRC_E_NOMEM;
    c->g = g;
    c->streamed = true;
    c->n_host = n_host_bricks;
    c->ring = ring_bricks;
    vrc_status s = VRC_OK;
    if (inject_fire(ctx, VRC_INJECT_ALLOC)) s = set_err(ctx, VRC_E_NOMEM, "injected allocation failure");
    if (s == VRC_OK) {
        cudaError_t e = cudaHostAlloc(&c->host_pool, (size_t)n_host_bricks * g.brick_bytes,
                                      cudaHostAllocPortable | cudaHostAllocMapped);
        if (e != cudaSuccess) {
            c->host_pool = nullptr;
            s = cuda_err(ctx, e, "cudaHostAlloc (pinned brick store)");
            if (s == VRC_E_CUDA) s = VRC_E_NOMEM;
        } else if ((e = cudaHostGetDevicePointer(&c->host_pool_dev, c->host_pool, 0)) != cudaSuccess) {
            s = cuda_err(ctx, e, "cudaHostGetDevicePointer (pinned brick store)");
        }
    }
    if (s == VRC_OK) s = dev_alloc(ctx, &c->ring_pool, (size_t)ring_bricks * g.brick_bytes);
    if (s == VRC_OK) s = alloc_meta(ctx, c);
    if (s != VRC_OK) {
        release_cube(ctx, c, true);
        return s;
    }
    c->host_filled.assign(n_host_bricks, 0);
    c->h_bmin.assign(g.nbricks, FLT_MAX);
    c->h_bmax.assign(g.nbricks, -FLT_MAX);
    c->h_bnonfinite.assign(g.nbricks, 0);
    c->h_bhalo_max.assign(g.nbricks, -INFINITY);
    c->h_bsum.assign(g.nbricks, 0.0);
    c->h_bcnt.assign(g.nbricks, 0);
    c->h_scales.assign(g.nbricks, 1.f);
    cudaMemcpy(c->scales, c->h_scales.data(), g.nbricks * 4, cudaMemcpyHostToDevice);
    c->charged = (int64_t)ring_bricks * g.brick_bytes;
    *cube_id = register_cube(ctx, c);
    return VRC_OK;
}

}  // namespace

vrc_status vrc_cube_create_streamed(vrc_ctx *ctx, int64_t nx, int64_t ny, int64_t nz, int32_t brick,
                                    int64_t n_host_bricks, int32_t ring_bricks, int64_t *cube_id)
{
    return create_streamed(ctx, nx, ny, nz, VRC_F32, brick, n_host_bricks, ring_bricks, cube_id);
}

vrc_status vrc_cube_put_brick(vrc_ctx *ctx, int64_t cube_id, int64_t slot, const float *bw)
{
    if (!ctx || !bw) return VRC_E_INVAL;
    Cube *c = find_cube(ctx, cube_id);
    if (!c) return VRC_E_BADID;
    if (!c->streamed) return set_err(ctx, VRC_E_UNSUPPORTED, "cube is resident, not streamed");
    if (c->source) return set_err(ctx, VRC_E_UNSUPPORTED, "cube takes its bricks from its provider");
    if (slot < 0 || slot >= c->n_host) return set_err(ctx, VRC_E_INVAL, "slot out of range");
    BrickMeta m;
    vrc_status s = pack_host_slot(ctx, c, slot, slot, bw, &m);
    if (s != VRC_OK) return s;
    if (!c->host_filled[slot]) {
        c->host_filled[slot] = 1;
        ++c->n_filled;
    }
    // every logical brick aliased to this slot gets its extrema
    for (int64_t b = slot; b < c->g.nbricks; b += c->n_host) set_brick_meta(c, b, m);
    finish_streamed_meta(c);
    return VRC_OK;
}

vrc_status vrc_cube_upload_streamed(vrc_ctx *ctx, vrc_brick_source_fn source, void *user, int64_t nx, int64_t ny,
                                    int64_t nz, int32_t storage, int32_t brick, int64_t n_host_bricks,
                                    int32_t ring_bricks, int64_t *cube_id)
{
    if (!ctx || !cube_id) return VRC_E_INVAL;
    if (!source) return set_err(ctx, VRC_E_INVAL, "null brick provider");
    int64_t id = 0;
    vrc_status s = create_streamed(ctx, nx, ny, nz, storage, brick, n_host_bricks, ring_bricks, &id);
    if (s != VRC_OK) return s;
    Cube *c = find_cube(ctx, id);
    c->source = source;
    c->source_user = user;
    const BrickGeom &g = c->g;
    if (g.dtype != VRC_F32) {
        // device staging of the packing of provided bricks
        s = dev_alloc(ctx, &c->pack_src, (size_t)g.R * g.R * g.R * sizeof(float));
        if (s == VRC_OK) s = dev_alloc(ctx, &c->pack_out, (size_t)g.brick_bytes);
        if (s == VRC_OK) {
            const cudaError_t e = cudaStreamCreateWithFlags(&c->pack_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                c->pack_stream = nullptr;
                s = cuda_err(ctx, e, "packing stream");
            }
        }
        if (s != VRC_OK) {
            vrc_cube_free(ctx, id);
            return s;
        }
    }
    c->slot_brick.assign(c->n_host, -1);
    c->slot_ev.assign(c->n_host, nullptr);
    c->slot_ev_live.assign(c->n_host, 0);
    c->source_buf.resize((size_t)g.R * g.R * g.R);
    // bf16 / fp8: provided bricks are copied to the device for packing, from page-locked memory
    if (g.dtype != VRC_F32) {
        if (cudaHostRegister(c->source_buf.data(), c->source_buf.size() * sizeof(float), cudaHostRegisterPortable) ==
            cudaSuccess)
            c->source_pinned = true;
        else
            cudaGetLastError();
    }
    for (int64_t sl = 0; sl < c->n_host && s == VRC_OK; ++sl) {
        const cudaError_t e = cudaEventCreateWithFlags(&c->slot_ev[sl], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            c->slot_ev[sl] = nullptr;
            s = cuda_err(ctx, e, "slot event");
        }
    }
    // every brick once, in index order: extrema, sums and non-finite counts;
    // the host cache keeps the last brick of each slot
    for (int64_t b = 0; b < g.nbricks && s == VRC_OK; ++b) {
        const int64_t slot = host_slot(c, b);
        BrickMeta m;
        s = call_source(ctx, c, b);
        if (s != VRC_OK) break;
        s = pack_host_slot(ctx, c, slot, b, c->source_buf.data(), &m);
        if (s != VRC_OK) break;
        c->slot_brick[slot] = b;
        set_brick_meta(c, b, m);
    }
    if (s != VRC_OK) {
        vrc_cube_free(ctx, id);
        return s;
    }
    if (s == VRC_OK && g.dtype != VRC_F32) {
        // brick scales to the device; the extrema measured on the provided
        // float32 bricks become those of the stored values
        const size_t nb4 = (size_t)g.nbricks * 4;
        cudaStream_t ps = c->pack_stream;
        auto ck = [&](cudaError_t e, const char *what) {
            if (s == VRC_OK && e != cudaSuccess) s = cuda_err(ctx, e, what);
        };
        ck(cudaMemcpyAsync(c->scales, c->h_scales.data(), nb4, cudaMemcpyHostToDevice, ps), "brick scales");
        ck(cudaMemcpyAsync(c->bmin, c->h_bmin.data(), nb4, cudaMemcpyHostToDevice, ps), "brick extrema");
        ck(cudaMemcpyAsync(c->bmax, c->h_bmax.data(), nb4, cudaMemcpyHostToDevice, ps), "brick extrema");
        ck(cudaMemcpyAsync(c->bhalo, c->h_bhalo_max.data(), nb4, cudaMemcpyHostToDevice, ps), "brick extrema");
        if (s == VRC_OK) {
            const unsigned grid = (unsigned)((g.nbricks + 127) / 128);
            if (g.dtype == VRC_BF16)
                k_stored_extrema<VRC_BF16><<<grid, 128, 0, ps>>>(c->bmin, c->bmax, c->bhalo, c->scales, g.nbricks);
            else
                k_stored_extrema<VRC_FP8E4M3><<<grid, 128, 0, ps>>>(c->bmin, c->bmax, c->bhalo, c->scales,
                                                                    g.nbricks);
            count_launch(ctx);
            ck(cudaGetLastError(), "stored extrema");
        }
        ck(cudaMemcpyAsync(c->h_bmin.data(), c->bmin, nb4, cudaMemcpyDeviceToHost, ps), "brick extrema");
        ck(cudaMemcpyAsync(c->h_bmax.data(), c->bmax, nb4, cudaMemcpyDeviceToHost, ps), "brick extrema");
        ck(cudaMemcpyAsync(c->h_bhalo_max.data(), c->bhalo, nb4, cudaMemcpyDeviceToHost, ps), "brick extrema");
        ck(cudaStreamSynchronize(ps), "brick extrema");
        if (s != VRC_OK) {
            vrc_cube_free(ctx, id);
            return s;
        }
    }
    c->host_filled.assign(c->n_host, 1);
    c->n_filled = c->n_host;
    finish_streamed_meta(c);
    *cube_id = id;
    return VRC_OK;
}

vrc_status vrc_cube_read_brick(vrc_ctx *ctx, int64_t cube_id, int64_t brick, void *dst, int64_t dst_bytes)
{
    if (!ctx) return VRC_E_INVAL;
    if (!dst) return set_err(ctx, VRC_E_INVAL, "dst is NULL");
    Cube *c = nullptr;
    CubeUse use;
    vrc_status s = acquire_cube(ctx, cube_id, nullptr, &c, use);
    if (s != VRC_OK) return s;
    const BrickGeom &g = c->g;
    if (brick < 0 || brick >= g.nbricks) return set_err(ctx, VRC_E_INVAL, "brick %lld out of range", (long long)brick);
    if (dst_bytes < g.brick_bytes)
        return set_err(ctx, VRC_E_INVAL, "dst_bytes %lld < brick bytes %lld", (long long)dst_bytes,
                       (long long)g.brick_bytes);
    if (c->streamed) {
        // the brick's host slot (a provider cube provides and packs it again when
        // the slot holds another brick)
        if (c->n_filled < c->n_host) return set_err(ctx, VRC_E_INVAL, "streamed cube: host slots not all written");
        int64_t slot = 0;
        if ((s = host_brick(ctx, c, brick, &slot)) != VRC_OK) return s;
        std::memcpy(dst, (const char *)c->host_pool + slot * g.brick_bytes, (size_t)g.brick_bytes);
        return VRC_OK;
    }
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    VRC_CK(ctx, cudaDeviceSynchronize());
    VRC_CK(ctx, cudaMemcpy(dst, (const char *)c->pool + brick * g.brick_bytes, (size_t)g.brick_bytes,
                           cudaMemcpyDeviceToHost));
    return VRC_OK;
}

vrc_status vrc_cube_free(vrc_ctx *ctx, int64_t cube_id)
{
    if (!ctx) return VRC_E_INVAL;
    Cube *c = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->cubes.find(cube_id);
        if (it == ctx->cubes.end()) return VRC_E_BADID;
        if (it->second->refs.load() > 0 || it->second->state.load() == CUBE_LOADING)
            return set_err(ctx, VRC_E_BUSY, "cube referenced by serving requests or being uploaded");
        c = it->second;
        ctx->cubes.erase(it);
    }
    cudaDeviceSynchronize();
    release_cube(ctx, c, true);
    return VRC_OK;
}

vrc_status vrc_cube_free_async(vrc_ctx *ctx, int64_t cube_id, void *stream)
{
    if (!ctx) return VRC_E_INVAL;
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    cudaEvent_t ev;
    VRC_CK(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    Cube *c = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->cubes.find(cube_id);
        if (it == ctx->cubes.end() || it->second->refs.load() > 0 || it->second->state.load() == CUBE_LOADING) {
            const bool busy = it != ctx->cubes.end();
            cudaEventDestroy(ev);
            return busy ? set_err(ctx, VRC_E_BUSY, "cube referenced by serving requests") : VRC_E_BADID;
        }
        c = it->second;
        ctx->cubes.erase(it);
    }
    const cudaError_t e = cudaEventRecord(ev, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev);
        release_cube(ctx, c, true);   // the cube is gone either way; fall back to a device-wide wait
        return cuda_err(ctx, e, "vrc_cube_free_async event");
    }
    std::lock_guard<std::mutex> lk(ctx->pend_mu);
    ctx->pending.emplace_back(ev, c);
    return VRC_OK;
}

vrc_status vrc_cube_info(vrc_ctx *ctx, int64_t cube_id, int64_t dims[3], int32_t *brick, int32_t *storage,
                         int64_t *n_bricks, int64_t *bytes, float *vmin, float *vmax, int64_t *render_copy_bytes)
{
    if (!ctx) return VRC_E_INVAL;
    Cube *c = find_cube(ctx, cube_id);
    if (!c) return VRC_E_BADID;
    if (dims)
        for (int a = 0; a < 3; ++a) dims[a] = c->g.dims[a];
    if (brick) *brick = c->g.B;
    if (storage) *storage = c->g.dtype;
    if (n_bricks) *n_bricks = c->g.nbricks;
    if (bytes) *bytes = c->streamed ? (int64_t)c->ring * c->g.brick_bytes : c->g.nbricks * c->g.brick_bytes;
    if (vmin) *vmin = c->vmin;
    if (vmax) *vmax = c->vmax;
    if (render_copy_bytes) *render_copy_bytes = c->tex_bytes;
    return VRC_OK;
}

}  // extern "C"

// ------------------------------------------------------------ out-of-core

// Host slot of brick b.  Caller-filled cubes: b % n_host.  Provider cubes:
// when the cache holds every brick, slot b; otherwise the first n_host - T
// bricks keep their slots for good and the others share the last T slots
// (T = min(n_host, 16)), so a frame that touches every brick provides
// nbricks - (n_host - T) of them again instead of evicting cached ones.
int64_t host_slot(const Cube *c, int64_t b)
{
    if (!c->source || c->n_host >= c->g.nbricks) return b % c->n_host;
    const int64_t T = std::min<int64_t>(c->n_host, 16), keep = c->n_host - T;
    return b < keep ? b : keep + (b - keep) % T;
}

vrc_status host_brick(vrc_ctx *ctx, Cube *c, int64_t brick, int64_t *slot)
{
    const int64_t sl = host_slot(c, brick);
    *slot = sl;
    if (!c->source || c->slot_brick[sl] == brick) return VRC_OK;
    // another brick lives in the slot: its last copy to the device must be done
    if (c->slot_ev_live[sl]) {
        const cudaError_t e = cudaEventSynchronize(c->slot_ev[sl]);
        if (e != cudaSuccess) return cuda_err(ctx, e, "host slot reuse");
        c->slot_ev_live[sl] = 0;
    }
    c->slot_brick[sl] = -1;
    vrc_status s = call_source(ctx, c, brick);
    if (s != VRC_OK) return s;
    if ((s = pack_host_slot(ctx, c, sl, brick, c->source_buf.data(), nullptr)) != VRC_OK) return s;
    c->slot_brick[sl] = brick;
    return VRC_OK;
}

vrc_status host_copied(vrc_ctx *ctx, Cube *c, int64_t slot, cudaStream_t st)
{
    if (!c->source) return VRC_OK;
    const cudaError_t e = cudaEventRecord(c->slot_ev[slot], st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "host slot event");
    c->slot_ev_live[slot] = 1;
    return VRC_OK;
}

vrc_status ring_load(vrc_ctx *ctx, Cube *c, int64_t b0, int64_t n, int first, cudaStream_t cs, cudaEvent_t done)
{
    const BrickGeom &g = c->g;
    for (int64_t q = 0; q < n; ++q) {
        if (inject_fire(ctx, VRC_INJECT_H2D)) return set_err(ctx, VRC_E_INJECTED, "injected host-to-device brick copy failure");
        int64_t sl = 0;
        vrc_status s = host_brick(ctx, c, b0 + q, &sl);
        if (s != VRC_OK) return s;
        const cudaError_t e = cudaMemcpyAsync((char *)c->ring_pool + (int64_t)(first + q) * g.brick_bytes,
                                              (const char *)c->host_pool + sl * g.brick_bytes, g.brick_bytes,
                                              cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return cuda_err(ctx, e, "brick H2D");
        if ((s = host_copied(ctx, c, sl, cs)) != VRC_OK) return s;
    }
    const cudaError_t e = cudaEventRecord(done, cs);
    if (e != cudaSuccess) return cuda_err(ctx, e, "ring event");
    return VRC_OK;
}

// ------------------------------------------------------------ residency

double host_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int64_t upload_peak_bytes(const Cube *c)
{
    const BrickGeom &g = c->g;
    const int64_t slack = (int64_t)2 << 20;   // block rounding, per allocation
    const int64_t cells = (int64_t)g.nb[0] * g.nb[1] * g.nb[2] * (g.B / 8) * (g.B / 8) * (g.B / 8);
    int64_t n = g.nbricks * g.brick_bytes + slack;                 // bricks
    n += 5 * (g.nbricks * 4 + slack);                              // per-brick metadata
    n += cells * 4 + slack;                                        // macro-cell maxima
    if (!c->host_packed) {
        n += g.dims[0] * g.dims[1] * g.dims[2] * 4 + slack;        // staging of the source
        n += g.nbricks * 4096 + slack;                             // scan partials
    }
    if (c->copy_mode != VRC_COPY_NONE) {
        const int64_t tex_esize = g.dtype == VRC_F32 ? 4 : 2 * g.esize;
        const int64_t layers = g.dtype == VRC_F32 ? g.R : g.R - 1;
        n += tex_esize * (int64_t)g.R * g.R * layers * g.nbricks + (1 << 20);   // render copy
        n += 4 * g.nbricks * 8 + slack;                                          // handle table
    }
    return n;
}

bool evict_for(vrc_ctx *ctx, int64_t need, const Cube *keep)
{
    auto fits = [&] { return ctx->used.load() + ctx->reserved + need <= ctx->budget; };
    if (fits()) return true;
    std::vector<Cube *> idle;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (auto &kv : ctx->cubes) {
            Cube *c = kv.second;
            if (c != keep && c->managed && c->state.load() == CUBE_RESIDENT && c->refs.load() == 0) idle.push_back(c);
        }
    }
    std::sort(idle.begin(), idle.end(), [](const Cube *a, const Cube *b) { return a->last_use < b->last_use; });
    for (Cube *c : idle) {
        if (fits()) break;
        if (c->refs.load() != 0) continue;
        c->state.store(CUBE_ABSENT);
        // requests that used it have completed; work of direct calls may still run
        release_device(ctx, c, c->direct_used);
        c->direct_used = false;
        ctx->evictions.fetch_add(1);
    }
    if (!fits()) reap_pending(ctx, true);
    return fits();
}

vrc_status acquire_cube(vrc_ctx *ctx, int64_t id, cudaStream_t st, Cube **out, CubeUse &use)
{
    Cube *c = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->cubes.find(id);
        if (it == ctx->cubes.end()) return set_err(ctx, VRC_E_BADID, "unknown cube %lld", (long long)id);
        c = it->second;
        c->refs.fetch_add(1);   // held until the call returns: never evicted or freed meanwhile
    }
    use.c = c;
    if (c->managed) {
        for (;;) {
            std::unique_lock<std::mutex> lk(ctx->res_mu);
            const int state = c->state.load();
            if (state == CUBE_RESIDENT) break;
            if (state == CUBE_LOADING) {   // the serving loader is uploading it
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(200));
                continue;
            }
            if (!evict_for(ctx, upload_peak_bytes(c), c))
                return set_err(ctx, VRC_E_NOMEM, "budget: no room to make registered cube %lld resident",
                               (long long)id);
            c->state.store(CUBE_LOADING);
            lk.unlock();
            const vrc_status s = load_registered(ctx, c, st);
            lk.lock();
            c->state.store(s == VRC_OK ? CUBE_RESIDENT : CUBE_ABSENT);
            if (s != VRC_OK) return s;
            ++c->loads;
            break;
        }
        c->last_use = host_ms();
        c->direct_used = true;
    }
    *out = c;
    return VRC_OK;
}

extern "C" vrc_status vrc_residency(vrc_ctx *ctx, int64_t *resident, uint64_t *loads, uint64_t *evictions)
{
    if (!ctx) return VRC_E_INVAL;
    int64_t r = 0;
    uint64_t l = 0;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (auto &kv : ctx->cubes)
            if (kv.second->managed) {
                r += kv.second->state.load() == CUBE_RESIDENT;
                l += kv.second->loads;
            }
    }
    if (resident) *resident = r;
    if (loads) *loads = l;
    if (evictions) *evictions = ctx->evictions.load();
    return VRC_OK;
}

vrc_status unpack_cube(vrc_ctx *ctx, const Cube *c, float *dst, cudaStream_t st)
{
    const BrickGeom &g = c->g;
    const unsigned grid = (unsigned)ctx->sm_count * 8;
    const uint8_t *pool = (const uint8_t *)c->pool;
    if (g.dtype == VRC_F32) k_unpack<VRC_F32><<<grid, 256, 0, st>>>(pool, g, c->scales, dst);
    else if (g.dtype == VRC_BF16) k_unpack<VRC_BF16><<<grid, 256, 0, st>>>(pool, g, c->scales, dst);
    else k_unpack<VRC_FP8E4M3><<<grid, 256, 0, st>>>(pool, g, c->scales, dst);
    count_launch(ctx);
    VRC_CK(ctx, cudaGetLastError());
    return VRC_OK;
}

