// Slab-marching renderer for resident float32 cubes.
//
// A CTA owns one screen tile of 16x16 rays and marches it through the cube in
// slabs of kD voxels along the tile's principal axis (the axis along which
// its centre ray moves fastest).  For every slab, the region of the cube that
// the tile's samples can touch there -- their trilinear footprints plus a
// margin -- is staged in shared memory by one TMA tensor load from a
// clamp-to-edge halo copy of the cube, and every sample of the slab reads its
// 2x2x2 footprint from shared memory.  The sample lattice, the trilinear
// arithmetic and the compositing are those of the fused renderer (Sec. 2 ray
// casting of sub-cubes; samples t_k = t_entry + (k + 1/2) step, binary32), so
// the image is bit-identical to it; only where the voxel values come from
// differs.  A sample whose footprint falls outside the staged box (a ray far
// from the rest of its tile) reads the halo copy directly.
//
// Measured on B300 (1024^3 cube, 32 views at 1920x1080, step 0.5): 227 ms
// against 171 ms for the texture-gather renderer.  Eight shared-memory loads
// plus their address arithmetic per sample cost more issue slots than two
// texture gathers, and boxes whose layers run along x (8-12 elements per row)
// put the lanes of a warp into few shared-memory banks.  The fused texture
// path therefore stays the default; this path is the staging alternative.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <float.h>
#include <limits.h>

#include <algorithm>
#include <cstring>

#include "ray.cuh"

namespace {

constexpr int kSlabThreads = 256;
constexpr int kD = 8;   // slab depth along the principal axis, voxels (a multiple of 4)

// Staged box per principal axis A, in halo-copy elements, x fastest.  The x
// extent is a multiple of 4 (TMA rows are whole 16-byte units) and x origins
// are multiples of 4; the layer axis holds kD + 2 layers (kD + 4 when x is
// principal, for the same 16-byte rule).  Lateral extents cover a 16x16 ray
// tile's footprint plus the drift of oblique rays across one slab.
template <int A>
struct Box;
template <>
struct Box<2> {   // z principal: lateral x, y
    static constexpr int ex = 40, ey = 36, ez = kD + 2;
};
template <>
struct Box<1> {   // y principal: lateral x, z
    static constexpr int ex = 40, ey = kD + 2, ez = 36;
};
template <>
struct Box<0> {   // x principal: lateral y, z
    static constexpr int ex = kD + 4, ey = 37, ez = 36;
};
template <int A>
struct BoxS {
    static constexpr int ex = Box<A>::ex, ey = Box<A>::ey, ez = Box<A>::ez;
    static constexpr int sy = ex, sz = ex * ey, elems = ex * ey * ez;
    __host__ __device__ static constexpr int e(int a) { return a == 0 ? ex : (a == 1 ? ey : ez); }
};
constexpr int kBufElems = std::max(BoxS<0>::elems, std::max(BoxS<1>::elems, BoxS<2>::elems));
constexpr size_t kSlabSmem = (size_t)kBufElems * sizeof(float) + 128;   // + alignment slack

struct HaloView {
    const float *base;      // element (hx, hy, hz) at hz * plane + hy * pitch + hx; voxel v has h = v + 1
    int64_t pitch, plane;
    int32_t nh[3];          // dims + 2
    int32_t withhold;       // test injection: issue no staging copy (the bounded waits run out)
};

struct SlabMaps {
    CUtensorMap m[3];       // TMA maps of the halo copy, box shapes Box<0..2>
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for a phase of the staging barrier: gives up after ~0.5 s.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity)
{
    if (bar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int i = 0; i < (1 << 24); ++i) {
        if (bar_try(bar, parity)) return true;
        if (global_ns() - t0 > 500000000ull) break;
    }
    return false;
}

__device__ __forceinline__ void tma_load3(float *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2),
          "r"(smem_addr(bar))
        : "memory");
}

// Lateral origin of a staged box: cover [lo, hi] if it fits (else centre on
// it), stay inside [0, nh - e] where possible, x origins multiples of 4.
__device__ __forceinline__ int fit_origin(int lo, int hi, int e, int nh, bool xaxis)
{
    if (hi - lo + 1 > e) lo = (lo + hi + 1 - e) / 2;
    lo = min(lo, nh - e);
    lo = max(lo, 0);
    return xaxis ? (lo & ~3) : lo;
}

// Trilinear from 8 corner values v[dz][dy][dx], lerps in x, then y, then z
// (the order and formulas of the fused renderer).
__device__ __forceinline__ float tri8(const float v[8], float wx, float wy, float wz)
{
    const float c00 = fmaf(wx, v[1] - v[0], v[0]);
    const float c10 = fmaf(wx, v[3] - v[2], v[2]);
    const float c01 = fmaf(wx, v[5] - v[4], v[4]);
    const float c11 = fmaf(wx, v[7] - v[6], v[6]);
    const float e0 = fmaf(wy, c10 - c00, c00), e1 = fmaf(wy, c11 - c01, c01);
    return fmaf(wz, e1 - e0, e0);
}

__device__ __forceinline__ void halo_corners(const HaloView &hv, int hx, int hy, int hz, float v[8])
{
    const float *p = hv.base + (int64_t)hz * hv.plane + (int64_t)hy * hv.pitch + hx;
    v[0] = __ldg(p);
    v[1] = __ldg(p + 1);
    v[2] = __ldg(p + hv.pitch);
    v[3] = __ldg(p + hv.pitch + 1);
    v[4] = __ldg(p + hv.plane);
    v[5] = __ldg(p + hv.plane + 1);
    v[6] = __ldg(p + hv.plane + hv.pitch);
    v[7] = __ldg(p + hv.plane + hv.pitch + 1);
}

// Per-ray state of the tile march.
struct RayState {
    float o[3], d[3], tin, tout;
    float kh;          // k + 1/2 of the next sample (exact in binary32: fewer than 2^22 samples)
    bool act;          // the ray still has samples to take
    float m, cr, cg, cb, A;
    uint32_t nsamp;
};

// Job constants of the tile, kept in shared memory (reloads are cheap there).
struct Par {
    float step, term, skip_below, vmin, inv_range;
    int32_t opc;
};

// Composite one sample value (MIP max, or DVR over + termination); returns
// false when the ray terminates.
template <int MODE>
__device__ __forceinline__ bool composite(const Par &P, const float4 *s_tf, RayState &r, float sv)
{
    if (MODE == 0) {
        r.m = fmaxf(r.m, sv);
        return true;
    }
    if (sv > P.skip_below) {   // false for NaN: alpha exactly 0 below the TF's transparent threshold
        // the arithmetic of over() in ray.cuh: w rounded once, fused channel updates
        const float4 c = classify(s_tf, sv, P.vmin, P.inv_range);
        const float w = __fmul_rn(__fsub_rn(1.f, r.A), opacity(c.w, P.step, P.opc));
        r.cr = fmaf(w, c.x, r.cr);
        r.cg = fmaf(w, c.y, r.cg);
        r.cb = fmaf(w, c.z, r.cb);
        r.A = __fadd_rn(r.A, w);
    }
    return !(r.A >= P.term);
}

// Every remaining sample of one ray from the halo copy (rays that do not fit
// the tile's march: principal axis of the wrong sign or too oblique).
template <int MODE>
__device__ __forceinline__ void trace_halo(const Par &P, const HaloView &hv, const float4 *s_tf, RayState &r)
{
    const float step = P.step;
    while (r.act) {
        const float t = __fadd_rn(r.tin, __fmul_rn(r.kh, step));
        if (!(t < r.tout)) break;
        float f[3], w[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float q = __fsub_rn(__fadd_rn(r.o[a], __fmul_rn(t, r.d[a])), 0.5f);
            f[a] = floorf(q);
            w[a] = __fsub_rn(q, f[a]);
        }
        float v[8];
        halo_corners(hv, (int)f[0] + 1, (int)f[1] + 1, (int)f[2] + 1, v);
        ++r.nsamp;
        r.kh = __fadd_rn(r.kh, 1.f);
        if (!composite<MODE>(P, s_tf, r, tri8(v, w[0], w[1], w[2]))) break;
    }
    r.act = false;
}

// Halo-copy index range [lo, hi] of the footprints this ray's samples in
// slab j can touch on lateral axis b (empty: lo > hi).  The slab holds the
// samples with p_A in [j kD, (j+1) kD); the t range comes from the slab planes
// widened by 1/100 voxel, positions from the exact line, the footprint of a
// coordinate p is halo indices floor(p - 1/2) + 1 .. + 2, widened by a
// 1/100-voxel margin.  A sample outside the box only costs a direct read.
template <int A>
__device__ __forceinline__ void slab_extent(const RayState &r, float inv_da, int j, bool pos, int lo[2], int hi[2])
{
    constexpr int B = A == 0 ? 1 : 0, C = A == 2 ? 1 : 2;
    lo[0] = lo[1] = INT_MAX;
    hi[0] = hi[1] = INT_MIN;
    if (!r.act) return;
    const float s0 = (float)(j * kD) - 0.01f, s1 = (float)((j + 1) * kD) + 0.01f;
    float ta = (__fsub_rn(pos ? s0 : s1, r.o[A])) * inv_da;
    float tb = (__fsub_rn(pos ? s1 : s0, r.o[A])) * inv_da;
    ta = fmaxf(ta, r.tin);
    tb = fminf(tb, r.tout);
    if (!(ta <= tb)) return;
    const int ax[2] = {B, C};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float pa = fmaf(ta, r.d[ax[i]], r.o[ax[i]]), pb = fmaf(tb, r.d[ax[i]], r.o[ax[i]]);
        lo[i] = (int)floorf(fminf(pa, pb) - 0.51f) + 1;
        hi[i] = (int)floorf(fmaxf(pa, pb) - 0.49f) + 2;
    }
}

struct SlabShared {
    int box[4];          // next box to stage: lo/hi on lateral axis B, lo/hi on lateral axis C
    int rng[2];          // first / last slab index of the tile (min / max)
    int org[3];          // halo origin of the staged box (x, y, z)
    int full;            // a box was staged for this slab
    Par par;
};

__device__ __forceinline__ void warp_minmax(int &lo, int &hi, int *slo, int *shi)
{
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        if (lo != INT_MAX) atomicMin(slo, lo);
        if (hi != INT_MIN) atomicMax(shi, hi);
    }
}

template <int A>
__device__ __forceinline__ void add_extent(const RayState &r, float inv_da, int j, bool pos, SlabShared &sh)
{
    int lo[2], hi[2];
    slab_extent<A>(r, inv_da, j, pos, lo, hi);
    warp_minmax(lo[0], hi[0], &sh.box[0], &sh.box[1]);
    warp_minmax(lo[1], hi[1], &sh.box[2], &sh.box[3]);
}

// Thread 0: stage the box accumulated in sh.box for slab j (if any ray
// reaches it) and reset the accumulator.
template <int A>
__device__ __forceinline__ void stage(const HaloView &hv, const CUtensorMap *map, float *buf, uint64_t *bar,
                                      SlabShared &sh, int j)
{
    using S = BoxS<A>;
    constexpr int B = A == 0 ? 1 : 0, C = A == 2 ? 1 : 2;
    const int lb = sh.box[0], hb = sh.box[1], lc = sh.box[2], hc = sh.box[3];
    sh.box[0] = sh.box[2] = INT_MAX;
    sh.box[1] = sh.box[3] = INT_MIN;
    const bool any = lb <= hb && lc <= hc;
    sh.full = any;
    if (!any) return;
    int org[3];
    org[A] = j * kD;   // halo index of the slab's first footprint layer
    org[B] = fit_origin(lb, hb, S::e(B), hv.nh[B], B == 0);
    org[C] = fit_origin(lc, hc, S::e(C), hv.nh[C], C == 0);
    sh.org[0] = org[0];
    sh.org[1] = org[1];
    sh.org[2] = org[2];
    if (hv.withhold) return;   // nothing arrives on the barrier: every wait for it runs out
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bar_expect_tx(bar, (uint32_t)(S::elems * sizeof(float)));
    tma_load3(buf, map, org[0], org[1], org[2], bar);
}

// March the tile's rays through the slabs along axis A (pos: increasing
// coordinate).  Every thread of the CTA calls this (the loop is CTA-uniform).
// Returns false if a staging wait gave up (the CTA must stop).
template <int MODE, int A>
__device__ __forceinline__ bool march(const JobDesc &J, const HaloView &hv, const CUtensorMap *map,
                                      const float4 *s_tf, float *s_buf, uint64_t *bar, uint32_t &phase,
                                      SlabShared &sh, RayState &r, bool slab_ray, bool pos)
{
    using S = BoxS<A>;
    const Par &P = sh.par;
    const int nslab = (J.cv.dims[A] + kD - 1) / kD;
    const float inv_da = slab_ray ? __frcp_rn(r.d[A]) : 0.f;
    // slab range of the tile: the slabs of each ray's first and last sample
    {
        int jf = INT_MAX, jl = INT_MIN;
        if (slab_ray) {
            const float t0 = __fadd_rn(r.tin, __fmul_rn(0.5f, P.step));
            const float pf = __fadd_rn(r.o[A], __fmul_rn(t0, r.d[A]));
            const float pl = __fadd_rn(r.o[A], __fmul_rn(r.tout, r.d[A]));
            const int a = min(max((int)floorf(pf * (1.f / kD)), 0), nslab - 1);
            const int b = min(max((int)floorf(pl * (1.f / kD)), 0), nslab - 1);
            jf = min(a, b);
            jl = max(a, b);
        }
        warp_minmax(jf, jl, &sh.rng[0], &sh.rng[1]);
    }
    __syncthreads();
    if (sh.rng[0] > sh.rng[1]) return true;   // no ray of this tile marches
    const int jbeg = pos ? sh.rng[0] : sh.rng[1], jend = pos ? sh.rng[1] : sh.rng[0], dj = pos ? 1 : -1;
    add_extent<A>(r, inv_da, jbeg, pos, sh);
    __syncthreads();
    for (int j = jbeg;; j += dj) {
        if (threadIdx.x == 0) stage<A>(hv, map, s_buf, bar, sh, j);
        __syncthreads();
        const bool full = sh.full != 0;
        if (full) {
            const bool got = __syncthreads_and(bar_wait(bar, phase));
            phase ^= 1u;
            if (!got) {
                bar_wait(bar, phase ^ 1u);   // the staged copy never completed: wait (bounded) for it, stop
                return false;
            }
        }
        if (j != jend) add_extent<A>(r, inv_da, j + dj, pos, sh);
        if (slab_ray && r.act) {
            // a sample belongs to the slab of p_A; the first and last slab are open
            // outwards (a position rounded onto or past a face of the cube)
            const float fs0 = j == 0 ? -INFINITY : (float)(j * kD);
            const float fs1 = j == nslab - 1 ? INFINITY : (float)((j + 1) * kD);
            // local box coordinates l = floor(p - 1/2) + 1 - origin, in binary32 (exact small integers)
            const float ox = (float)(1 - sh.org[0]), oy = (float)(1 - sh.org[1]), oz = (float)(1 - sh.org[2]);
            constexpr float cx = 0.5f * (S::ex - 2), cy = 0.5f * (S::ey - 2), cz = 0.5f * (S::ez - 2);
            const float step = P.step;
            for (;;) {
                const float t = __fadd_rn(r.tin, __fmul_rn(r.kh, step));
                if (!(t < r.tout)) {
                    r.act = false;
                    break;
                }
                float p[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) p[a] = __fadd_rn(r.o[a], __fmul_rn(t, r.d[a]));
                if (pos ? !(p[A] < fs1) : (p[A] < fs0)) break;   // next slab
                float f[3], w[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float q = __fsub_rn(p[a], 0.5f);
                    f[a] = floorf(q);
                    w[a] = __fsub_rn(q, f[a]);
                }
                const float lx = f[0] + ox, ly = f[1] + oy, lz = f[2] + oz;
                float v[8];
                // 0 <= l <= e - 2 on every axis: the 2x2x2 footprint lies in the box
                if (full && fabsf(lx - cx) <= cx && fabsf(ly - cy) <= cy && fabsf(lz - cz) <= cz) {
                    const float *sp = s_buf + (int)fmaf(lz, (float)S::sz, fmaf(ly, (float)S::sy, lx));
                    v[0] = sp[0];
                    v[1] = sp[1];
                    v[2] = sp[S::sy];
                    v[3] = sp[S::sy + 1];
                    v[4] = sp[S::sz];
                    v[5] = sp[S::sz + 1];
                    v[6] = sp[S::sz + S::sy];
                    v[7] = sp[S::sz + S::sy + 1];
                } else {
                    halo_corners(hv, (int)f[0] + 1, (int)f[1] + 1, (int)f[2] + 1, v);
                }
                ++r.nsamp;
                r.kh = __fadd_rn(r.kh, 1.f);
                if (!composite<MODE>(P, s_tf, r, tri8(v, w[0], w[1], w[2]))) {
                    r.act = false;
                    break;
                }
            }
        }
        // every read of the staged box is done; the next box's extent is complete
        const bool any_active = __syncthreads_or(slab_ray && r.act);
        if (!any_active || j == jend) break;
    }
    return true;
}

template <int MODE>
__global__ void __launch_bounds__(kSlabThreads, 3)
    k_render_slab(const JobDesc *__restrict__ jobs, int n_jobs, int64_t total_items, int *counter, HaloView hv,
                  const __grid_constant__ SlabMaps maps, int *err)
{
    extern __shared__ unsigned char s_dyn[];
    float *s_buf = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(s_dyn) + 127) & ~(uintptr_t)127);
    __shared__ float4 s_tf[256];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ SlabShared sh;
    __shared__ int64_t s_item;
    __shared__ int s_job;
    if (threadIdx.x == 0) {
        bar_init(&s_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    uint32_t phase = 0;
    int loaded = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(counter, 1);
            s_job = s_item < total_items ? find_job(jobs, n_jobs, s_item) : -1;
            sh.box[0] = sh.box[2] = sh.rng[0] = INT_MAX;
            sh.box[1] = sh.box[3] = sh.rng[1] = INT_MIN;
            sh.full = 0;
            if (s_job >= 0) {
                const JobDesc &Jt = jobs[s_job];
                sh.par = Par{Jt.step, Jt.term, Jt.skip_below, Jt.vmin, Jt.inv_range, Jt.opacity_correction};
            }
        }
        __syncthreads();
        const int64_t item = s_item;
        const int jid = s_job;
        if (item >= total_items) break;
        const JobDesc &J = jobs[jid];
        if (MODE == 1 && jid != loaded) {
            s_tf[threadIdx.x] = J.tf[threadIdx.x];
            __syncthreads();
            loaded = jid;
        }
        int tx, ty, lx, ly;
        tile_of(J, item - J.item_begin, tx, ty);
        tile_pixel(J.tile_w, J.warp_w, lx, ly);
        const int px = tx * J.tile_w + lx, py = ty * J.tile_h + ly;
        // principal axis of the tile: largest component of its centre ray
        int A = 2;
        bool pos = true;
        {
            const ViewParams &v = J.vp;
            const float fx = (float)(tx * J.tile_w) + 0.5f * (float)J.tile_w;
            const float fy = (float)(ty * J.tile_h) + 0.5f * (float)J.tile_h;
            float q[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) q[a] = v.kind == VRC_CAM_PERSP ? v.D0[a] + fx * v.DX[a] + fy * v.DY[a] : v.D0[a];
            const float ax = fabsf(q[0]), ay = fabsf(q[1]), az = fabsf(q[2]);
            A = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
            pos = (A == 0 ? q[0] : (A == 1 ? q[1] : q[2])) > 0.f;   // selects: no local-memory indexing
        }
        RayState r;
        r.m = -FLT_MAX;
        r.cr = r.cg = r.cb = r.A = 0.f;
        r.nsamp = 0;
        r.kh = 0.5f;
        const bool inside = px < J.vp.W && py < J.vp.H;
        const bool hit = inside && ray_setup(J.vp, J.cv.fdims, px, py, r.o, r.d, r.tin, r.tout);
        r.act = hit;
        const float da = A == 0 ? r.d[0] : (A == 1 ? r.d[1] : r.d[2]);
        const bool slab_ray = hit && (pos ? da > 0.25f : da < -0.25f);
        bool ok;
        if (A == 0) ok = march<MODE, 0>(J, hv, &maps.m[0], s_tf, s_buf, &s_bar, phase, sh, r, slab_ray, pos);
        else if (A == 1) ok = march<MODE, 1>(J, hv, &maps.m[1], s_tf, s_buf, &s_bar, phase, sh, r, slab_ray, pos);
        else ok = march<MODE, 2>(J, hv, &maps.m[2], s_tf, s_buf, &s_bar, phase, sh, r, slab_ray, pos);
        if (!ok) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            return;   // CTA-uniform: every thread saw the same failed wait
        }
        if (hit && !slab_ray) trace_halo<MODE>(sh.par, hv, s_tf, r);
        if (inside) {
            const int64_t pix = (int64_t)py * J.vp.W + px;
            if (MODE == 0) J.out[pix] = r.m;
            else reinterpret_cast<float4 *>(J.out)[pix] = make_float4(r.cr, r.cg, r.cb, r.A);
        }
        if (J.samples) warp_count2(J.samples, r.nsamp, r.nsamp);
        __syncthreads();
    }
}

// Halo copy: element (hx, hy, hz) holds voxel clamp(h - 1) read from the
// cube's float32 bricks.
__global__ void k_fill_halo(const uint8_t *__restrict__ pool, BrickGeom g, float *__restrict__ out, int64_t pitch,
                            int64_t plane, int32_t nhx, int32_t nhy, int32_t nhz)
{
    const int64_t rows = (int64_t)nhy * nhz;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int hy = (int)(row % nhy), hz = (int)(row / nhy);
        const int y = min(max(hy - 1, 0), (int)g.dims[1] - 1), z = min(max(hz - 1, 0), (int)g.dims[2] - 1);
        const int by = y >> g.logB, bz = z >> g.logB;
        const int ly = y - (by << g.logB), lz = z - (bz << g.logB);
        float *dst = out + (int64_t)hz * plane + (int64_t)hy * pitch;
        for (int hx = threadIdx.x; hx < nhx; hx += blockDim.x) {
            const int x = min(max(hx - 1, 0), (int)g.dims[0] - 1);
            const int bx = x >> g.logB, lx = x - (bx << g.logB);
            const int64_t b = ((int64_t)bz * g.nb[1] + by) * g.nb[0] + bx;
            const float *bp = reinterpret_cast<const float *>(pool + b * g.brick_bytes);
            dst[hx] = __ldg(bp + ((int64_t)(lz + 1) * g.R + (ly + 1)) * g.P + (lx + g.O));
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

template <int A>
bool encode_map(PFN_cuTensorMapEncodeTiled_v12000 fn, CUtensorMap *m, float *base, const int64_t nh[3], int64_t pitch,
                int64_t plane)
{
    const cuuint64_t dims[3] = {(cuuint64_t)nh[0], (cuuint64_t)nh[1], (cuuint64_t)nh[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)plane * 4};
    const cuuint32_t box[3] = {(cuuint32_t)Box<A>::ex, (cuuint32_t)Box<A>::ey, (cuuint32_t)Box<A>::ez};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool slab_supported(const Cube *c)
{
    return c && !c->streamed && c->pool && c->g.dtype == VRC_F32;
}

// Build the halo copy of a resident float32 cube and its tensor maps (once).
vrc_status slab_prepare(vrc_ctx *ctx, Cube *c, cudaStream_t st)
{
    if (c->halo) return VRC_OK;
    if (!slab_supported(c)) return set_err(ctx, VRC_E_UNSUPPORTED, "slab path: resident float32 cubes only");
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return set_err(ctx, VRC_E_UNSUPPORTED, "slab path: cuTensorMapEncodeTiled unavailable");
    const BrickGeom &g = c->g;
    const int64_t nh[3] = {g.dims[0] + 2, g.dims[1] + 2, g.dims[2] + 2};
    const int64_t pitch = (nh[0] + 3) & ~(int64_t)3;   // 16-byte rows
    const int64_t plane = pitch * nh[1];
    const int64_t bytes = plane * nh[2] * 4;
    float *h = nullptr;
    vrc_status s = dev_alloc(ctx, (void **)&h, bytes);
    if (s != VRC_OK) return s;
    alignas(64) SlabMaps maps;
    if (!encode_map<0>(fn, &maps.m[0], h, nh, pitch, plane) || !encode_map<1>(fn, &maps.m[1], h, nh, pitch, plane) ||
        !encode_map<2>(fn, &maps.m[2], h, nh, pitch, plane)) {
        dev_free(ctx, h, bytes);
        return set_err(ctx, VRC_E_UNSUPPORTED, "slab path: tensor map encoding failed");
    }
    const int grid = (int)std::min<int64_t>(nh[1] * nh[2], (int64_t)ctx->sm_count * 16);
    k_fill_halo<<<grid, 256, 0, st>>>((const uint8_t *)c->pool, g, h, pitch, plane, (int32_t)nh[0], (int32_t)nh[1],
                                      (int32_t)nh[2]);
    count_launch(ctx);
    VRC_CK(ctx, cudaGetLastError());
    static_assert(sizeof(SlabMaps) <= sizeof(c->slab_maps), "tensor map storage");
    std::memcpy(c->slab_maps, &maps, sizeof(SlabMaps));
    c->halo = h;
    c->halo_bytes = bytes;
    c->halo_pitch = pitch;
    return VRC_OK;
}

void slab_release(vrc_ctx *ctx, Cube *c)
{
    if (c->halo) dev_free(ctx, c->halo, c->halo_bytes);
    c->halo = nullptr;
    c->halo_bytes = 0;
}

namespace {
void slab_attrs()
{
    static bool done = false;
    if (done) return;
    done = true;
    cudaFuncSetAttribute(k_render_slab<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmem);
    cudaFuncSetAttribute(k_render_slab<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmem);
}
}  // namespace

int slab_occupancy(int mode)
{
    slab_attrs();
    int n = 0;
    if (mode == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_render_slab<0>, kSlabThreads, kSlabSmem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_render_slab<1>, kSlabThreads, kSlabSmem);
    return std::max(n, 1);
}

// Persistent slab launch over (view, 16x16 tile) work items of `jobs` (all of
// cube c); err: device int set to 1 if a staging wait gave up.
void slab_launch(const Cube *c, int mode, int grid, cudaStream_t st, const JobDesc *jobs, int n_jobs, int64_t total,
                 int *counter, int *err, bool withhold)
{
    HaloView hv;
    hv.withhold = withhold ? 1 : 0;
    hv.base = c->halo;
    hv.pitch = c->halo_pitch;
    hv.plane = c->halo_pitch * (c->g.dims[1] + 2);
    for (int a = 0; a < 3; ++a) hv.nh[a] = (int32_t)(c->g.dims[a] + 2);
    alignas(64) SlabMaps maps;
    std::memcpy(&maps, c->slab_maps, sizeof(SlabMaps));
    slab_attrs();
    if (mode == 0) k_render_slab<0><<<grid, kSlabThreads, kSlabSmem, st>>>(jobs, n_jobs, total, counter, hv, maps, err);
    else k_render_slab<1><<<grid, kSlabThreads, kSlabSmem, st>>>(jobs, n_jobs, total, counter, hv, maps, err);
}
