// Device-side ray set-up, sampling and compositing shared by the render kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <float.h>

#include "vrc_internal.h"

// Cube storage as seen by the kernels.
struct CubeView {
    const uint8_t *pool;      // brick b at pool + b * brick_bytes (resident)
    const unsigned long long *tex;  // brick b's layered-array texture (null: none)
    const float *scales;      // FP8 per-brick scale
    int64_t brick_bytes;
    int32_t B, logB, P, O, R;
    int32_t nb[3];
    int32_t dims[3];
    float fdims[3];
    int32_t dtype;
};

// One render inside a (possibly heterogeneous) launch.
struct JobDesc {
    CubeView cv;
    ViewParams vp;
    float step, term, vmin, inv_range;   // TF index u = (s - vmin) * inv_range
    int32_t opacity_correction;
    int32_t tile_w, tile_h, tiles_x, tiles_y;
    int32_t warp_w;                      // a warp covers warp_w x (32 / warp_w) pixels
    int64_t item_begin;                  // first work item of this job
    const float4 *tf;                    // device [256] (DVR)
    float *out;                          // image of this job (view)
    unsigned long long *samples;         // [lattice, evaluated] sample counters of this job (may be shared or null)
    const float *cellmax;                // empty-space skipping: macro-cell maxima (null: no skipping)
    int32_t ncx, ncy;                    // macro-cells per row / per slice
    float skip_below;                    // DVR: samples whose cell max <= this are transparent
};

// Binary32 ray of pixel (px, py), exactly as stated in vrc.h (every operation
// rounded, no contraction).  Returns false when the ray misses the cube.
__device__ __forceinline__ bool ray_setup(const ViewParams &v, const float fd[3], int px, int py, float o[3],
                                          float d[3], float &tin, float &tout)
{
    const float fx = __fadd_rn((float)px, 0.5f), fy = __fadd_rn((float)py, 0.5f);
    if (v.kind == VRC_CAM_PERSP) {
        float q[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = v.O0[a];
            q[a] = __fadd_rn(__fadd_rn(v.D0[a], __fmul_rn(fx, v.DX[a])), __fmul_rn(fy, v.DY[a]));
        }
        const float n = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(q[0], q[0]), __fmul_rn(q[1], q[1])),
                                             __fmul_rn(q[2], q[2])));
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = __fdiv_rn(q[a], n);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = __fadd_rn(__fadd_rn(v.O0[a], __fmul_rn(fx, v.DX[a])), __fmul_rn(fy, v.DY[a]));
            d[a] = v.D0[a];
        }
    }
    float lo = 0.f, hi = __int_as_float(0x7f800000);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.f) {
            if (o[a] < 0.f || o[a] > fd[a]) return false;
            continue;
        }
        float t0 = __fdiv_rn(__fsub_rn(0.f, o[a]), d[a]);
        float t1 = __fdiv_rn(__fsub_rn(fd[a], o[a]), d[a]);
        if (t0 > t1) {
            const float tmp = t0;
            t0 = t1;
            t1 = tmp;
        }
        if (t0 > lo) lo = t0;
        if (t1 < hi) hi = t1;
    }
    tin = lo;
    tout = hi;
    return lo < hi;
}

__device__ __forceinline__ float sample_t(float tin, int k, float step)
{
    return __fadd_rn(tin, __fmul_rn(__fadd_rn((float)k, 0.5f), step));
}

template <int DT>
__device__ __forceinline__ float raw_voxel(const uint8_t *brick, int64_t e)
{
    if (DT == VRC_F32) return __ldg(reinterpret_cast<const float *>(brick) + e);
    if (DT == VRC_BF16)
        return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short *>(brick) + e) << 16);
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)__ldg(brick + e), __NV_E4M3);
    return __half2float(__half(h));
}

// Per-axis trilinear set-up of one coordinate: q = p - 0.5, i0 = floor(q),
// f = q - i0; the voxel floor(p) is i0 + (f >= 0.5) (exact because p - 0.5 is
// exact for p >= 0.5; for p < 0.5 both choices clamp to voxel 0).
struct AxisT {
    int i0, ip;
    float f;
};
__device__ __forceinline__ AxisT axis_tri(float p, int n)
{
    const float q = __fsub_rn(p, 0.5f);
    const float fl = floorf(q);
    AxisT r;
    r.f = __fsub_rn(q, fl);
    r.i0 = (int)fl;
    r.ip = min(max(r.i0 + (r.f >= 0.5f ? 1 : 0), 0), n - 1);
    return r;
}

__device__ __forceinline__ int brick_index(const CubeView &cv, int bx, int by, int bz)
{
    return (bz * cv.nb[1] + by) * cv.nb[0] + bx;
}

// Trilinear sample from brick storage `bp` whose local origin is (ox, oy, oz)
// voxels; needs i0 - o in [-1, B-1] on each axis (guaranteed when the brick
// contains voxel floor(p)).
template <int DT>
__device__ __forceinline__ float tri_in_brick(const CubeView &cv, const uint8_t *bp, const AxisT &ax, const AxisT &ay,
                                              const AxisT &az, int ox, int oy, int oz, float scale)
{
    const int lx = ax.i0 - ox, ly = ay.i0 - oy, lz = az.i0 - oz;
    const int64_t e = ((int64_t)(lz + 1) * cv.R + (ly + 1)) * cv.P + (lx + cv.O);
    const int64_t S = (int64_t)cv.P * cv.R;
    const float v000 = raw_voxel<DT>(bp, e), v100 = raw_voxel<DT>(bp, e + 1);
    const float v010 = raw_voxel<DT>(bp, e + cv.P), v110 = raw_voxel<DT>(bp, e + cv.P + 1);
    const float v001 = raw_voxel<DT>(bp, e + S), v101 = raw_voxel<DT>(bp, e + S + 1);
    const float v011 = raw_voxel<DT>(bp, e + S + cv.P), v111 = raw_voxel<DT>(bp, e + S + cv.P + 1);
    const float c00 = fmaf(ax.f, v100 - v000, v000), c10 = fmaf(ax.f, v110 - v010, v010);
    const float c01 = fmaf(ax.f, v101 - v001, v001), c11 = fmaf(ax.f, v111 - v011, v011);
    const float c0 = fmaf(ay.f, c10 - c00, c00), c1 = fmaf(ay.f, c11 - c01, c01);
    const float v = fmaf(az.f, c1 - c0, c0);
    return DT == VRC_FP8E4M3 ? v * scale : v;
}

template <int DT>
__device__ __forceinline__ float nearest_in_brick(const CubeView &cv, const uint8_t *bp, int ix, int iy, int iz, int ox,
                                                  int oy, int oz, float scale)
{
    const int64_t e = ((int64_t)(iz - oz + 1) * cv.R + (iy - oy + 1)) * cv.P + (ix - ox + cv.O);
    const float v = raw_voxel<DT>(bp, e);
    return DT == VRC_FP8E4M3 ? __fmul_rn(v, scale) : v;
}

// Voxel (ix, iy, iz) (inside the cube) read from the resident brick holding it.
template <int DT>
__device__ __forceinline__ float voxel_resident(const CubeView &cv, int ix, int iy, int iz)
{
    const int bx = ix >> cv.logB, by = iy >> cv.logB, bz = iz >> cv.logB;
    const int b = brick_index(cv, bx, by, bz);
    const float scale = DT == VRC_FP8E4M3 ? __ldg(cv.scales + b) : 1.f;
    return nearest_in_brick<DT>(cv, cv.pool + (int64_t)b * cv.brick_bytes, ix, iy, iz, bx << cv.logB, by << cv.logB,
                                bz << cv.logB, scale);
}

// Nearest voxel index of coordinate p on an axis of n voxels.
// (floor and conversion in one round-down conversion: the same integer as
// (int)floorf(p) for every p, NaN giving 0 in both.)
__device__ __forceinline__ int nearest_index(float p, int n) { return min(max(__float2int_rd(p), 0), n - 1); }

// Sample at p from the resident brick that contains voxel floor(p).
template <int SAMPLING, int DT>
__device__ __forceinline__ float sample_resident(const CubeView &cv, float px, float py, float pz)
{
    if (SAMPLING == VRC_NEAREST) {
        return voxel_resident<DT>(cv, nearest_index(px, cv.dims[0]), nearest_index(py, cv.dims[1]),
                                  nearest_index(pz, cv.dims[2]));
    } else {
        const AxisT ax = axis_tri(px, cv.dims[0]), ay = axis_tri(py, cv.dims[1]), az = axis_tri(pz, cv.dims[2]);
        const int bx = ax.ip >> cv.logB, by = ay.ip >> cv.logB, bz = az.ip >> cv.logB;
        const int b = brick_index(cv, bx, by, bz);
        const float scale = DT == VRC_FP8E4M3 ? __ldg(cv.scales + b) : 1.f;
        return tri_in_brick<DT>(cv, cv.pool + (int64_t)b * cv.brick_bytes, ax, ay, az, bx << cv.logB, by << cv.logB,
                                bz << cv.logB, scale);
    }
}

// Render copies (one 2D-layered texture per brick, layers along z; local
// voxel (lx, ly, lz) at texel (lx+1, ly+1) of layer lz+1).  With point sampling
// and unnormalised coordinates a 2x2 gather at the integer coordinate (u, v)
// returns texels (u-1, v-1) .. (u, v) exactly, as x = (u-1, v), y = (u, v),
// z = (u, v-1), w = (u-1, v-1).
//   fp32: one texel per stored voxel; the 2x2x2 trilinear footprint takes two
//         gathers, one per layer.
//   bf16: texel (u, v) of layer j packs the stored voxels of layers j (low 16
//         bits) and j + 1 (high 16 bits) as one 32-bit texel;
//   fp8:  it packs their e4m3 codes as one 16-bit texel (layer j in the low
//         byte).
// For bf16 and fp8 one gather therefore returns the whole footprint (the
// copies hold B + 1 layers), and the texture unit moves half the gathers.
__device__ __forceinline__ float2 e4m3x2_to_float2(uint32_t t)
{
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)t, __NV_E4M3);
    return __half22float2(__half2(h));
}

// The 2x2 footprints of layers `layer` (g0) and `layer + 1` (g1) at (u, v),
// as fp32 values (fp8: code values, the brick scale not yet applied).
template <int DT>
__device__ __forceinline__ void gather_pair(unsigned long long tex, int layer, float u, float v, float4 &g0, float4 &g1)
{
    if (DT == VRC_F32) {
        asm volatile("tld4.r.a2d.v4.f32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
                     : "=f"(g0.x), "=f"(g0.y), "=f"(g0.z), "=f"(g0.w)
                     : "l"(tex), "r"(layer), "f"(u), "f"(v));
        asm volatile("tld4.r.a2d.v4.f32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
                     : "=f"(g1.x), "=f"(g1.y), "=f"(g1.z), "=f"(g1.w)
                     : "l"(tex), "r"(layer + 1), "f"(u), "f"(v));
    } else {
        uint32_t a, b, c, d;
        asm volatile("tld4.r.a2d.v4.u32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
                     : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
                     : "l"(tex), "r"(layer), "f"(u), "f"(v));
        if (DT == VRC_BF16) {
            g0 = make_float4(__uint_as_float(a << 16), __uint_as_float(b << 16), __uint_as_float(c << 16),
                             __uint_as_float(d << 16));
            g1 = make_float4(__uint_as_float(a & 0xffff0000u), __uint_as_float(b & 0xffff0000u),
                             __uint_as_float(c & 0xffff0000u), __uint_as_float(d & 0xffff0000u));
        } else {
            const float2 fa = e4m3x2_to_float2(a), fb = e4m3x2_to_float2(b), fc = e4m3x2_to_float2(c),
                         fd = e4m3x2_to_float2(d);
            g0 = make_float4(fa.x, fb.x, fc.x, fd.x);
            g1 = make_float4(fa.y, fb.y, fc.y, fd.y);
        }
    }
}

// Trilinear sample of a brick with origin (ox, oy, oz) from its render copy:
// footprint (l, l+1) on an axis is gathered at coordinate l + 2 (layer l + 1).
// The lerps run in x, then y, then z order, as in the global-load sampler, so
// both give the same value bit for bit.
template <int DT>
__device__ __forceinline__ float tri_tex(unsigned long long t, const AxisT &ax, const AxisT &ay, const AxisT &az,
                                         int ox, int oy, int oz, float scale)
{
    float4 g0, g1;
    gather_pair<DT>(t, az.i0 - oz + 1, (float)(ax.i0 - ox + 2), (float)(ay.i0 - oy + 2), g0, g1);
    // footprint corners: w = (x0, y0), z = (x1, y0), x = (x0, y1), y = (x1, y1)
    const float c00 = fmaf(ax.f, g0.z - g0.w, g0.w), c10 = fmaf(ax.f, g0.y - g0.x, g0.x);
    const float c01 = fmaf(ax.f, g1.z - g1.w, g1.w), c11 = fmaf(ax.f, g1.y - g1.x, g1.x);
    const float c0 = fmaf(ay.f, c10 - c00, c00), c1 = fmaf(ay.f, c11 - c01, c01);
    const float val = fmaf(az.f, c1 - c0, c0);
    return DT == VRC_FP8E4M3 ? val * scale : val;
}

// Transfer function: 256 RGBA entries, linear between entries.  Every
// operation is rounded on its own (explicit intrinsics, so the compiler cannot
// contract a product into a later sum differently in different kernels): all
// renderers give the same colour for the same sample, bit for bit.  The four
// channel lerps run as packed f32x2 fused multiply-adds (each lane rounds as
// fmaf does).
__device__ __forceinline__ float4 classify(const float4 *tf, float s, float vmin, float inv_range)
{
    float u = __fmul_rn(__fsub_rn(s, vmin), inv_range);
    u = fminf(fmaxf(u, 0.f), 1.f);
    const float x = __fmul_rn(u, 255.f);
    const int j = min((int)x, 254);
    const float f = __fsub_rn(x, (float)j);
    const float4 a = tf[j], b = tf[j + 1];
    const float2 m1 = make_float2(-1.f, -1.f), ff = make_float2(f, f);
    const float2 a01 = make_float2(a.x, a.y), a23 = make_float2(a.z, a.w);
    const float2 rg = __ffma2_rn(ff, __ffma2_rn(a01, m1, make_float2(b.x, b.y)), a01);   // a + f (b - a)
    const float2 ba = __ffma2_rn(ff, __ffma2_rn(a23, m1, make_float2(b.z, b.w)), a23);
    return make_float4(rg.x, rg.y, ba.x, ba.y);
}

__device__ __forceinline__ float opacity(float a, float step, int correct)
{
    return correct ? 1.f - __powf(fmaxf(1.f - a, 0.f), step) : a;
}

// Front-to-back premultiplied compositing: C += (1 - A) a c, A += (1 - A) a,
// with w = (1 - A) a rounded once and used for every channel.
struct OverAcc {
    float2 rg = make_float2(0.f, 0.f);
    float b = 0.f, A = 0.f;
};
__device__ __forceinline__ void over(OverAcc &acc, const float4 &c, float step, int correct)
{
    const float w = __fmul_rn(__fsub_rn(1.f, acc.A), opacity(c.w, step, correct));
    acc.rg = __ffma2_rn(make_float2(w, w), make_float2(c.x, c.y), acc.rg);
    acc.b = fmaf(w, c.z, acc.b);
    acc.A = __fadd_rn(acc.A, w);
}

// ------------------------------------------------------------------ work items

// Thread -> pixel inside a tile_w x tile_h tile: warps cover ww x (32/ww)
// pixel blocks (ww a power of two dividing tile_w).
__device__ __forceinline__ void tile_pixel(int tile_w, int ww, int &lx, int &ly)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wx = tile_w / ww, wh = 32 / ww;
    lx = (warp % wx) * ww + (lane % ww);
    ly = (warp / wx) * wh + (lane / ww);
}

// Tile t of a view, in strips of kSuper tile rows walked kSuper tile columns
// at a time: the tiles in flight at any moment cover a compact patch of the
// image, so their rays cross a narrow part of the cube (cache and TLB reach).
// Measured against row-major order: +0.4% on a 1024^3 cube, +2.5% on a
// 2048x2048x4096 cube (kSuper 4 and 8 in between).
constexpr int kSuper = 16;
__device__ __forceinline__ void tile_of(const JobDesc &J, int64_t t, int &tx, int &ty)
{
    if (kSuper <= 1) {
        tx = (int)(t % J.tiles_x);
        ty = (int)(t / J.tiles_x);
        return;
    }
    const int64_t strip_tiles = (int64_t)kSuper * J.tiles_x;
    const int strip = (int)(t / strip_tiles);
    const int r = (int)(t - strip * strip_tiles);
    const int h = min(kSuper, J.tiles_y - strip * kSuper);    // tile rows in this strip
    const int nblk = (J.tiles_x + kSuper - 1) / kSuper;
    const int cb = min(r / (kSuper * h), nblk - 1);
    const int rr = r - cb * kSuper * h;
    const int w = cb == nblk - 1 ? J.tiles_x - cb * kSuper : kSuper;   // tile columns in this block
    ty = strip * kSuper + rr / w;
    tx = cb * kSuper + rr % w;
}

__device__ __forceinline__ int find_job(const JobDesc *jobs, int n_jobs, int64_t item)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].item_begin <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void warp_count2(unsigned long long *counters, uint32_t lattice, uint32_t evaluated)
{
    for (int o = 16; o; o >>= 1) {
        lattice += __shfl_xor_sync(0xffffffffu, lattice, o);
        evaluated += __shfl_xor_sync(0xffffffffu, evaluated, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (lattice) atomicAdd(counters, (unsigned long long)lattice);
        if (evaluated) atomicAdd(counters + 1, (unsigned long long)evaluated);
    }
}
