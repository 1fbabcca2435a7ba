// Ray casting: fused persistent multi-view kernel, sort-last brick kernel with
// partial images, composite kernel, out-of-core streaming, graphs, autotuner.
#include <float.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "ray.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kNearU = 8;   // nearest MIP: sample loads in flight per ray

// ------------------------------------------------------------------ kernels

// One ray of the fused path: all samples in ray order, each read from the
// brick that contains it (per-brick segments are composited in registers).
// TEXAXIS < 0: trilinear/nearest from the packed bricks with global loads;
// TEXAXIS = 2: trilinear from the texture copy layered along z.
template <int MODE, int SAMPLING, int DT, int TEXAXIS, bool SKIP>
__device__ __forceinline__ void trace_fused(const JobDesc &J, const float4 *s_tf, int px, int py, uint32_t &nsamp,
                                            uint32_t &neval)
{
    float o[3], d[3], tin, tout;
    const bool hit = ray_setup(J.vp, J.cv.fdims, px, py, o, d, tin, tout);
    const int64_t pix = (int64_t)py * J.vp.W + px;
    const unsigned long long *tex =
        TEXAXIS >= 0 ? J.cv.tex + (int64_t)TEXAXIS * J.cv.nb[0] * J.cv.nb[1] * J.cv.nb[2] : nullptr;
    float m = -FLT_MAX;
    OverAcc acc;
    if (hit) {
        const float step = J.step;
        // reciprocals for the macro-cell exit estimate (a guess, verified with
        // the exact sample positions, so rounding here cannot change the image)
        float invd[3] = {0.f, 0.f, 0.f}, inv_step = 0.f;
        if (SKIP) {
#pragma unroll
            for (int a = 0; a < 3; ++a) invd[a] = d[a] != 0.f ? __frcp_rn(d[a]) : 0.f;
            inv_step = __frcp_rn(step);
        }
        // nearest MIP along an axis-aligned ray (two direction components 0):
        // p = o + t*d keeps those two coordinates exactly (t*0 = 0), so their
        // voxel indices are fixed for the ray and each sample reads one voxel
        // of the moving axis; kNearU samples' loads are issued before they are
        // folded into the maximum.  An axis-aligned view at native resolution
        // reads each voxel once, so HBM bounds it.  Same samples, same maximum.
        const int moving = d[0] != 0.f ? 0 : (d[1] != 0.f ? 1 : 2);
        const bool aligned = TEXAXIS < 0 && MODE == 0 && SAMPLING == VRC_NEAREST &&
                             (d[0] != 0.f) + (d[1] != 0.f) + (d[2] != 0.f) == 1;
        if (aligned) {
            const CubeView &cv = J.cv;
            // the two fixed axes contribute constant brick-index and in-brick
            // element terms; per sample only the moving axis's voxel im is new:
            // brick term (im >> logB) * bstr_m, element term (im & (B-1)) * estr_m
            // (element of local (lx, ly, lz) = (lz+1) R P + (ly+1) P + lx + O)
            const int fixed[3] = {nearest_index(o[0], cv.dims[0]), nearest_index(o[1], cv.dims[1]),
                                  nearest_index(o[2], cv.dims[2])};
            const int64_t estr[3] = {1, cv.P, (int64_t)cv.R * cv.P};
            const int64_t eadd[3] = {cv.O, cv.P, (int64_t)cv.R * cv.P};   // the +O / +1 of each axis
            const int bstr[3] = {1, cv.nb[0], cv.nb[0] * cv.nb[1]};
            int64_t e_c = 0;
            int b_c = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                e_c += eadd[a];
                if (a != moving) {
                    e_c += (int64_t)(fixed[a] & (cv.B - 1)) * estr[a];
                    b_c += (fixed[a] >> cv.logB) * bstr[a];
                }
            }
            const uint32_t estr_m = (uint32_t)(moving == 0 ? estr[0] : (moving == 1 ? estr[1] : estr[2]));
            const int bstr_m = moving == 0 ? bstr[0] : (moving == 1 ? bstr[1] : bstr[2]);
            const float om = moving == 0 ? o[0] : (moving == 1 ? o[1] : o[2]);
            const float dm = moving == 0 ? d[0] : (moving == 1 ? d[1] : d[2]);
            const int nm = moving == 0 ? cv.dims[0] : (moving == 1 ? cv.dims[1] : cv.dims[2]);
            // in-brick element offsets fit 32 bits (a brick is below 2^32 bytes).
            // No branch per sample: a sample past the ray's end still reads an
            // in-bounds voxel (its index is clamped) and is then replaced by
            // -FLT_MAX; its position k + u + 0.5 is formed by exact float adds.
            const uint32_t e_c32 = (uint32_t)e_c;
            const int64_t bstride = (int64_t)bstr_m * cv.brick_bytes;
            const uint8_t *const base = cv.pool + (int64_t)b_c * cv.brick_bytes;
            for (int k = 0;; k += kNearU) {
                const float kf = (float)k;
                float sv[kNearU];
                int nv = 0;
#pragma unroll
                for (int u = 0; u < kNearU; ++u) {
                    const float tk = __fadd_rn(tin, __fmul_rn(__fadd_rn(kf, (float)u + 0.5f), step));
                    const bool valid = tk < tout;
                    const int im = nearest_index(__fadd_rn(om, __fmul_rn(tk, dm)), nm);
                    const int bm = im >> cv.logB;
                    const float v = raw_voxel<DT>(base + bm * bstride, e_c32 + (uint32_t)(im & (cv.B - 1)) * estr_m);
                    const float vs = DT == VRC_FP8E4M3 ? __fmul_rn(v, __ldg(cv.scales + b_c + bm * bstr_m)) : v;
                    sv[u] = valid ? vs : -FLT_MAX;
                    nv += valid;
                }
#pragma unroll
                for (int u = 0; u < kNearU; ++u) m = fmaxf(m, sv[u]);
                nsamp += nv;
                neval += nv;
                if (nv < kNearU) break;
            }
        } else if (TEXAXIS < 0 && MODE == 0 && SAMPLING == VRC_NEAREST) {
            // nearest MIP along any other ray: the same branch-free groups of
            // kNearU samples (indices clamped, so every load is in bounds);
            // 8 perspective 1080p views of a 1024^3 cube 21.5 ms against
            // 26.4 ms one sample at a time
            for (int k = 0;; k += kNearU) {
                const float kf = (float)k;
                float sv[kNearU];
                int nv = 0;
#pragma unroll
                for (int u = 0; u < kNearU; ++u) {
                    const float tk = __fadd_rn(tin, __fmul_rn(__fadd_rn(kf, (float)u + 0.5f), step));
                    const bool valid = tk < tout;
                    const float v = sample_resident<SAMPLING, DT>(J.cv, __fadd_rn(o[0], __fmul_rn(tk, d[0])),
                                                                  __fadd_rn(o[1], __fmul_rn(tk, d[1])),
                                                                  __fadd_rn(o[2], __fmul_rn(tk, d[2])));
                    sv[u] = valid ? v : -FLT_MAX;
                    nv += valid;
                }
#pragma unroll
                for (int u = 0; u < kNearU; ++u) m = fmaxf(m, sv[u]);
                nsamp += nv;
                neval += nv;
                if (nv < kNearU) break;
            }
        } else if (TEXAXIS < 0 && MODE == 1 && SAMPLING == VRC_NEAREST) {
            // nearest DVR: U samples' loads in flight (indices clamped, so
            // every load is in bounds), then composited in ray order with the
            // same termination test; samples past the end or after termination
            // are loaded but not composited
            constexpr int U = 4;   // 8 spills at 48 registers
            bool done = false;
            for (int k = 0; !done; k += U) {
                const float kf = (float)k;
                float sv[U];
                bool vv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float tk = __fadd_rn(tin, __fmul_rn(__fadd_rn(kf, (float)u + 0.5f), step));
                    vv[u] = tk < tout;
                    sv[u] = sample_resident<SAMPLING, DT>(J.cv, __fadd_rn(o[0], __fmul_rn(tk, d[0])),
                                                          __fadd_rn(o[1], __fmul_rn(tk, d[1])),
                                                          __fadd_rn(o[2], __fmul_rn(tk, d[2])));
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (!vv[u]) {
                        done = true;
                        break;
                    }
                    ++nsamp;
                    ++neval;
                    const float sn = sv[u];
                    if (sn == sn && !(sn <= J.skip_below))
                        over(acc, classify(s_tf, sn, J.vmin, J.inv_range), step, J.opacity_correction);
                    if (acc.A >= J.term) {
                        done = true;
                        break;
                    }
                }
            }
        } else {
#pragma unroll 1
            for (int k = 0;; ++k) {
                const float tk = sample_t(tin, k, step);
                if (!(tk < tout)) break;
                const float p0 = __fadd_rn(o[0], __fmul_rn(tk, d[0]));
                const float p1 = __fadd_rn(o[1], __fmul_rn(tk, d[1]));
                const float p2 = __fadd_rn(o[2], __fmul_rn(tk, d[2]));
                float s;
                if (TEXAXIS >= 0) {
                    const CubeView &cv = J.cv;
                    const AxisT ax = axis_tri(p0, cv.dims[0]), ay = axis_tri(p1, cv.dims[1]), az = axis_tri(p2, cv.dims[2]);
                    if (SKIP) {
                        // empty-space skipping: every sample whose voxel floor(p) lies in an
                        // 8^3 macro-cell that cannot change the result is counted, not fetched
                        const int cx = ax.ip >> 3, cy = ay.ip >> 3, cz = az.ip >> 3;
                        const float cm = __ldg(J.cellmax + ((int64_t)cz * J.ncy + cy) * J.ncx + cx);
                        if (MODE == 0 ? cm <= m : cm <= J.skip_below) {
                            // last sample still inside the cell: slab estimate, then corrected
                            // with the exact binary32 positions (positions are monotone along
                            // the ray and the cell is convex, so every sample in between is in)
                            const float lo[3] = {(float)(cx << 3), (float)(cy << 3), (float)(cz << 3)};
                            float te = tout;
#pragma unroll
                            for (int a = 0; a < 3; ++a) {
                                if (d[a] != 0.f) {
                                    const float bnd = d[a] > 0.f ? lo[a] + 8.f : lo[a];
                                    te = fminf(te, (bnd - o[a]) * invd[a]);
                                }
                            }
                            int kl = max(k, (int)((te - tin) * inv_step - 0.5f));
                            bool verified = false;
                            for (int it = 0; it < 6 && kl > k; ++it) {
                                const float t2 = sample_t(tin, kl, step);
                                bool in = t2 < tout;
#pragma unroll
                                for (int a = 0; a < 3; ++a) {
                                    const float pa = __fadd_rn(o[a], __fmul_rn(t2, d[a]));
                                    const int ia = min(max((int)floorf(pa), 0), cv.dims[a] - 1) >> 3;
                                    in = in && ia == (a == 0 ? cx : (a == 1 ? cy : cz));
                                }
                                if (in) {
                                    verified = true;
                                    break;
                                }
                                // overshoot: the estimate is usually one sample too far, else back off
                                kl = it == 0 ? kl - 1 : k + (kl - k) / 2;
                            }
                            if (!verified) kl = k;       // sample k itself is known to be in the cell
                            nsamp += kl - k + 1;
                            k = kl;
                            continue;
                        }
                    }
                    const int bx = ax.ip >> cv.logB, by = ay.ip >> cv.logB, bz = az.ip >> cv.logB;
                    const int b = (bz * cv.nb[1] + by) * cv.nb[0] + bx;
                    const unsigned long long th = __ldg(tex + b);
                    const float scale = DT == VRC_FP8E4M3 ? __ldg(cv.scales + b) : 1.f;
                    s = tri_tex<DT>(th, ax, ay, az, bx << cv.logB, by << cv.logB, bz << cv.logB, scale);
                } else {
                    s = sample_resident<SAMPLING, DT>(J.cv, p0, p1, p2);
                }
                ++nsamp;
                ++neval;
                if (MODE == 0) {
                    m = fmaxf(m, s);
                } else {
                    // s <= skip_below gives alpha exactly 0 under the TF: the over step
                    // would add zero, so the lookup is not made (exact)
                    if (s == s && !(s <= J.skip_below))
                        over(acc, classify(s_tf, s, J.vmin, J.inv_range), step, J.opacity_correction);
                    if (acc.A >= J.term) break;
                }
            }
        }
    }
    if (MODE == 0) J.out[pix] = m;
    else reinterpret_cast<float4 *>(J.out)[pix] = make_float4(acc.rg.x, acc.rg.y, acc.b, acc.A);
}

// One ray of the fused path on the texture copies.  A sample belongs to the
// brick of voxel clamp(floor(p)); along one ray the binary32 positions are
// monotone on every axis, so the samples of one brick are consecutive.  When
// the ray enters a brick, the first sample past the brick (past one of the
// faces the ray moves towards, faces on the cube's border being infinite, or
// past the ray's end) is found once, from a slab estimate corrected with the
// exact binary32 sample positions; each sample then compares one counter
// (one loop, so the lanes of a warp stay in step).  Texel coordinates are
// formed in binary32 from floor(p - 0.5) (exact small integers): every sample
// reads the same texels with the same weights as the per-sample lookup of
// trace_fused.  Positions, weights and lerps use packed f32x2 instructions
// where the operands pair up; each lane rounds as the scalar instruction does,
// so every value is unchanged.
template <int MODE, int DT>
__device__ __forceinline__ void trace_tex(const JobDesc &J, const float4 *s_tf, int px, int py, uint32_t &nsamp)
{
    float o[3], d[3], tin, tout;
    const bool hit = ray_setup(J.vp, J.cv.fdims, px, py, o, d, tin, tout);
    const int64_t pix = (int64_t)py * J.vp.W + px;
    float m = -FLT_MAX;
    OverAcc acc;
    if (hit) {
        const float step = J.step;
        const CubeView &cv = J.cv;
        const float2 m1 = make_float2(-1.f, -1.f);
        // t of the sample whose k + 0.5 is kh, as stated (binary32, every operation rounded)
        auto t_at = [&](float kh) { return __fadd_rn(tin, __fmul_rn(kh, step)); };
        const float inv_step = __frcp_rn(step);
        // samples k = 0 .. n-1 have t_k < tout; kh_end = n + 0.5 (estimate, then exact;
        // t_k grows with k, and rays hold fewer than 2^22 samples, so kh is exact)
        float kh_end = fmaxf(ceilf(__fmul_rn(tout - tin, inv_step) - 0.5f), 0.f) + 0.5f;
        while (kh_end > 0.5f && !(t_at(kh_end - 1.f) < tout)) kh_end -= 1.f;
        while (t_at(kh_end) < tout) kh_end += 1.f;
        const bool neg0 = d[0] < 0.f, neg1 = d[1] < 0.f, neg2 = d[2] < 0.f;
        const float id0 = d[0] != 0.f ? __frcp_rn(d[0]) : 0.f, id1 = d[1] != 0.f ? __frcp_rn(d[1]) : 0.f,
                    id2 = d[2] != 0.f ? __frcp_rn(d[2]) : 0.f;
        float E0 = 0.f, E1 = 0.f, E2 = 0.f;   // exit faces of the current brick
        float scale = 1.f, kh_stop = 0.5f;    // kh_stop: first sample past the current brick
        float2 mc = make_float2(0.f, 0.f);    // -(texel origin) of the brick on x and y
        int zo = 0;
        unsigned long long th = 0;
        // fp32: texels of the previous sample's 2x2x2 cell, reused when the
        // next sample falls in the same cell (step < 1).  Measured: +7% for
        // MIP, +2.2% for DVR on a 1024^3 cube and +4..5% on a 2048^3 cube
        // (32 / 16 views 1080p); images unchanged.  Packed texels need one
        // gather per sample and gain nothing from it.  Reusing one layer when
        // the next sample moves by one layer in the same 2x2 column measured
        // slower (branches: 169 against 227 G samples/s; predicated gathers
        // with selects: 217 against 232), as did the reuse in an earlier,
        // heavier loop.
        constexpr bool kReuse = DT == VRC_F32;
        float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
        float pu = -1.f, pv = -1.f;
        int pl = -1;
        // one compare per sample: kh_stop <= kh_end, so the ray's end is tested
        // only where a brick ends; the samples taken are counted once at the end
        float kh = 0.5f;
#pragma unroll 1
        for (;; kh = __fadd_rn(kh, 1.f)) {
            // positions as stated: each product and sum rounded on its own (the
            // scalar intrinsics are never contracted into a fused multiply-add)
            const float t = t_at(kh);
            const float2 pxy = make_float2(__fadd_rn(o[0], __fmul_rn(t, d[0])), __fadd_rn(o[1], __fmul_rn(t, d[1])));
            const float p2 = __fadd_rn(o[2], __fmul_rn(t, d[2]));
            if (kh >= kh_stop) {
                if (!(kh < kh_end)) break;
                // entering the brick of this sample
                const int bx = min(max((int)floorf(pxy.x), 0), cv.dims[0] - 1) >> cv.logB;
                const int by = min(max((int)floorf(pxy.y), 0), cv.dims[1] - 1) >> cv.logB;
                const int bz = min(max((int)floorf(p2), 0), cv.dims[2] - 1) >> cv.logB;
                const int b = (bz * cv.nb[1] + by) * cv.nb[0] + bx;
                th = __ldg(cv.tex + (int64_t)2 * cv.nb[0] * cv.nb[1] * cv.nb[2] + b);
                if (DT == VRC_FP8E4M3) scale = __ldg(cv.scales + b);
                auto face = [&](int bi, int nbi, float da) {
                    if (da > 0.f) return bi == nbi - 1 ? INFINITY : (float)((bi + 1) << cv.logB);
                    if (da < 0.f) return bi == 0 ? -INFINITY : (float)(bi << cv.logB);
                    return INFINITY;
                };
                E0 = face(bx, cv.nb[0], d[0]);
                E1 = face(by, cv.nb[1], d[1]);
                E2 = face(bz, cv.nb[2], d[2]);
                // texel (u, v) = floor(p - 0.5) - origin + 2; layer = floor(p_z - 0.5) - origin_z + 1
                mc = make_float2((float)(2 - (bx << cv.logB)), (float)(2 - (by << cv.logB)));
                zo = (bz << cv.logB) - 1;
                pl = -1;   // texel coordinates are local to the brick
                // first sample past the brick: the nearest finite exit face gives
                // an estimate, the exact positions correct it (samples past the
                // brick form a suffix of the ray)
                auto past = [&](float khq) {
                    const float tq = t_at(khq);
                    const float q0 = __fadd_rn(o[0], __fmul_rn(tq, d[0]));
                    const float q1 = __fadd_rn(o[1], __fmul_rn(tq, d[1]));
                    const float q2 = __fadd_rn(o[2], __fmul_rn(tq, d[2]));
                    return ((q0 >= E0) != neg0) || ((q1 >= E1) != neg1) || ((q2 >= E2) != neg2);
                };
                float tf = INFINITY;
                if (fabsf(E0) < INFINITY) tf = fminf(tf, (E0 - o[0]) * id0);
                if (fabsf(E1) < INFINITY) tf = fminf(tf, (E1 - o[1]) * id1);
                if (fabsf(E2) < INFINITY) tf = fminf(tf, (E2 - o[2]) * id2);
                float ks = fminf(ceilf(__fmul_rn(tf - tin, inv_step) - 0.5f) + 0.5f, kh_end);
                ks = fmaxf(ks, __fadd_rn(kh, 1.f));
                while (ks > __fadd_rn(kh, 1.f) && past(ks - 1.f)) ks -= 1.f;
                while (ks < kh_end && !past(ks)) ks += 1.f;
                kh_stop = ks;
            }
            const float2 qxy = __fadd2_rn(pxy, make_float2(-0.5f, -0.5f));
            const float q2 = __fsub_rn(p2, 0.5f);
            const float f0 = floorf(qxy.x), f1 = floorf(qxy.y), f2 = floorf(q2);
            const float2 fxy = make_float2(f0, f1);
            const float2 wxy = __ffma2_rn(fxy, m1, qxy);     // q - floor(q), exact
            const float wz = __fsub_rn(q2, f2);
            const float2 uv = __fadd2_rn(fxy, mc);
            const int layer = (int)f2 - zo;
            if (!kReuse || layer != pl || uv.x != pu || uv.y != pv) {
                gather_pair<DT>(th, layer, uv.x, uv.y, g0, g1);
                pl = layer;
                pu = uv.x;
                pv = uv.y;
            }
            // gather order: x = (u-1, v), y = (u, v), z = (u, v-1), w = (u-1, v-1);
            // lerps in x, then y, then z
            float sv;
            if (DT == VRC_F32) {
                const float c00 = fmaf(wxy.x, g0.z - g0.w, g0.w), c10 = fmaf(wxy.x, g0.y - g0.x, g0.x);
                const float c01 = fmaf(wxy.x, g1.z - g1.w, g1.w), c11 = fmaf(wxy.x, g1.y - g1.x, g1.x);
                const float2 C0 = make_float2(c00, c01), C1 = make_float2(c10, c11);
                const float2 e = __ffma2_rn(make_float2(wxy.y, wxy.y), __ffma2_rn(C0, m1, C1), C0);
                sv = fmaf(wz, e.y - e.x, e.x);
            } else {
                // both layers of a texel pair come from one texel: lerp the two layers at once
                const float2 wx2 = make_float2(wxy.x, wxy.x);
                const float2 L0 = make_float2(g0.w, g1.w), H0 = make_float2(g0.z, g1.z);
                const float2 L1 = make_float2(g0.x, g1.x), H1 = make_float2(g0.y, g1.y);
                const float2 C0 = __ffma2_rn(wx2, __ffma2_rn(L0, m1, H0), L0);   // (c00, c01)
                const float2 C1 = __ffma2_rn(wx2, __ffma2_rn(L1, m1, H1), L1);   // (c10, c11)
                const float2 e = __ffma2_rn(make_float2(wxy.y, wxy.y), __ffma2_rn(C0, m1, C1), C0);
                sv = fmaf(wz, e.y - e.x, e.x);
                if (DT == VRC_FP8E4M3) sv = sv * scale;
            }
            if (MODE == 0) {
                m = fmaxf(m, sv);
            } else if (sv > J.skip_below) {   // false for NaN; transparent samples leave A as it is
                over(acc, classify(s_tf, sv, J.vmin, J.inv_range), step, J.opacity_correction);
                if (acc.A >= J.term) {
                    kh = __fadd_rn(kh, 1.f);   // this sample counts
                    break;
                }
            }
        }
        nsamp += (uint32_t)(kh - 0.5f);   // samples k = 0 .. kh - 1.5 were taken
    }
    if (MODE == 0) J.out[pix] = m;
    else reinterpret_cast<float4 *>(J.out)[pix] = make_float4(acc.rg.x, acc.rg.y, acc.b, acc.A);
}

// Fused path, persistent: CTAs pull (job, tile) items from an atomic counter.
// TEX: trilinear samples come from the cubes' texture copies.  Register caps
// (CTAs per SM) are the measured best.  6 for the texture ray walk of MIP and
// of bf16/fp8 DVR (32-view 1080p DVR of a 1024^3 cube: bf16 302 -> 338, fp8
// 318 -> 355 G samples/s against 5; a 2048^3 cube +9..13%; 7: 307 / 302).
// fp32 DVR keeps 5 (48 registers, no spills): at 6 (40 registers, spills) it
// gained 1% on the 1024^3 cube and lost 7..11% on a 2048^3 cube, where the
// autotuner also found no better grid for the 6-CTA build.  5 otherwise.
template <int MODE, int SAMPLING, int DT, bool TEX, bool SKIP>
__global__ void __launch_bounds__(kThreads, (TEX && !SKIP && !(MODE == 1 && DT == VRC_F32)) ? 6 : 5)
    k_render_fused(const JobDesc *__restrict__ jobs, int n_jobs, int64_t total_items, int *counter)
{
    __shared__ float4 s_tf[256];
    __shared__ int64_t s_item;
    __shared__ int s_job;
    int loaded = -1;
    uint32_t nsamp = 0, neval = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(counter, 1);
            s_job = s_item < total_items ? find_job(jobs, n_jobs, s_item) : -1;
        }
        __syncthreads();
        const int64_t item = s_item;
        const int jid = s_job;
        if (item >= total_items) break;
        const JobDesc &J = jobs[jid];
        if (MODE == 1 && jid != loaded) {
            s_tf[threadIdx.x] = J.tf[threadIdx.x];   // tiles are 256 pixels: one entry per thread
            __syncthreads();
            loaded = jid;
        }
        int tx, ty;
        tile_of(J, item - J.item_begin, tx, ty);
        int lx, ly;
        tile_pixel(J.tile_w, J.warp_w, lx, ly);
        const int px = tx * J.tile_w + lx, py = ty * J.tile_h + ly;
        // TEX kernels are launched only when every job's cube has texture copies
        if (px < J.vp.W && py < J.vp.H) {
            if (TEX && SAMPLING == VRC_TRILINEAR && !SKIP) {
                trace_tex<MODE, DT>(J, s_tf, px, py, nsamp);
                neval = nsamp;
            } else {
                trace_fused<MODE, SAMPLING, DT, ((TEX && SAMPLING == VRC_TRILINEAR) ? 2 : -1),
                            (SKIP && TEX && SAMPLING == VRC_TRILINEAR)>(J, s_tf, px, py, nsamp, neval);
            }
        }
        if (J.samples) warp_count2(J.samples, nsamp, neval);   // one atomic pair per warp and item
        nsamp = neval = 0;
        __syncthreads();
    }
}

// Orthographic nearest MIP along the cube's y or z axis, G = 8 pixels of an
// image row per thread.  When the G rays share their direction, their t range
// and their coordinate on the moving axis, and their voxel columns are G
// consecutive x (in either order, the lowest a multiple of G) at one index of
// the other fixed axis, each sample of the G rays reads G consecutive stored
// voxels of one brick row: one vector load per sample (fp32 two 16-byte loads,
// bf16 one 16-byte load, fp8 one 8-byte load) instead of G scalar loads with
// their index arithmetic.  The samples, their positions and values and the
// order in which each ray takes them are those of the per-ray loop, so every
// pixel gets the same maximum bit for bit; a group that fails the test takes
// the per-ray loop.  At native resolution each voxel is read once, and the
// vector loads leave HBM as the bound for fp32.
// pixels per thread and samples whose loads are in flight together.
// Measured on the 1024^3 cube (native z view): fp32 0.678 / bf16 0.409 / fp8
// 0.435 ms; 16 pixels per thread (fewer threads, 16-byte fp8 loads) 0.472 /
// 0.656 ms for bf16 / fp8, 8 samples in flight 0.862 / 0.405 / 0.453 ms,
// 2 samples 0.681 ms for fp32, 4 pixels (16-byte fp32 loads) 0.950 ms.
constexpr int kRowG = 8;
constexpr int kRowU = 4;

// G stored voxels of a brick row as 32-bit words (G x esize bytes, 8-byte
// aligned at least): loaded by 16-byte (or, below 16 bytes, 8-byte) loads
template <int DT, int G>
struct RowVec {
    static constexpr int kBytes = G * (DT == VRC_F32 ? 4 : (DT == VRC_BF16 ? 2 : 1));
    static constexpr int kWords = kBytes / 4;
    uint32_t w[kWords];
};

// The loads are volatile asm: each is issued where it stands, ahead of the
// samples that consume them, so the group's loads are all in flight at once
// (a compiler free to sink a load next to its use would serialise them).
template <int DT, int G>
__device__ __forceinline__ void row_load(const uint8_t *p, RowVec<DT, G> &r)
{
    if constexpr (RowVec<DT, G>::kBytes >= 16) {
#pragma unroll
        for (int i = 0; i < RowVec<DT, G>::kWords / 4; ++i)
            asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(r.w[4 * i]), "=r"(r.w[4 * i + 1]), "=r"(r.w[4 * i + 2]), "=r"(r.w[4 * i + 3])
                         : "l"(p + 16 * i));
    } else {
        asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(r.w[0]), "=r"(r.w[1]) : "l"(p));
    }
}

// Voxel values x = lowest .. lowest + G - 1 (fp8: code values, the brick scale
// not yet applied), each as raw_voxel reads it.
template <int DT, int G>
__device__ __forceinline__ void row_values(const RowVec<DT, G> &r, float v[G])
{
#pragma unroll
    for (int i = 0; i < RowVec<DT, G>::kWords; ++i) {
        const uint32_t w = r.w[i];
        if constexpr (DT == VRC_F32) {
            v[i] = __uint_as_float(w);
        } else if constexpr (DT == VRC_BF16) {
            v[2 * i] = __uint_as_float(w << 16);
            v[2 * i + 1] = __uint_as_float(w & 0xffff0000u);
        } else {
            const float2 lo = e4m3x2_to_float2(w & 0xffffu), hi = e4m3x2_to_float2(w >> 16);
            v[4 * i] = lo.x, v[4 * i + 1] = lo.y, v[4 * i + 2] = hi.x, v[4 * i + 3] = hi.y;
        }
    }
}

// The G rays of pixels (px0 .. px0 + G - 1, py).  Returns false (nothing
// written) when they do not form a row group as described above.
template <int DT>
__device__ __forceinline__ bool mip_row_group(const JobDesc &J, int px0, int py, uint32_t &nsamp)
{
    const CubeView &cv = J.cv;
    if (px0 + kRowG > J.vp.W) return false;
    float o[3], d[3], tin = 0.f, tout = 0.f;
    const bool hit = ray_setup(J.vp, cv.fdims, px0, py, o, d, tin, tout);
    if (d[0] != 0.f || (d[1] != 0.f) == (d[2] != 0.f)) return false;   // rays along y or z only
    const int m = d[1] != 0.f ? 1 : 2, f = 3 - m;   // moving axis; the fixed axis besides x
    // (components picked by selects: a runtime index would put the arrays in local memory)
    const float om = m == 1 ? o[1] : o[2], dm = m == 1 ? d[1] : d[2];
    const int nm = m == 1 ? cv.dims[1] : cv.dims[2], nf = f == 1 ? cv.dims[1] : cv.dims[2];
    const int X0 = nearest_index(o[0], cv.dims[0]), F = nearest_index(f == 1 ? o[1] : o[2], nf);
    int sx = 0;
#pragma unroll 1
    for (int i = 1; i < kRowG; ++i) {
        float oi[3], di[3], ti = 0.f, to = 0.f;
        const bool hi = ray_setup(J.vp, cv.fdims, px0 + i, py, oi, di, ti, to);
        const int Xi = nearest_index(oi[0], cv.dims[0]);
        if (i == 1) sx = Xi - X0;
        if (hi != hit || (sx != 1 && sx != -1) || Xi != X0 + sx * i || di[0] != d[0] || di[1] != d[1] ||
            di[2] != d[2])
            return false;
        if (hit && (ti != tin || to != tout || (m == 1 ? oi[1] : oi[2]) != om ||
                    nearest_index(f == 1 ? oi[1] : oi[2], nf) != F))
            return false;
    }
    const int Xlo = sx > 0 ? X0 : X0 - (kRowG - 1);
    if (hit && (Xlo & (kRowG - 1))) return false;
    float mx[kRowG];
#pragma unroll
    for (int j = 0; j < kRowG; ++j) mx[j] = -FLT_MAX;
    if (hit) {
        // brick and in-brick element terms of x and of the other fixed axis;
        // element of local (lx, ly, lz) = (lz+1) R P + (ly+1) P + lx + O
        const uint32_t estr_f = f == 1 ? (uint32_t)cv.P : (uint32_t)(cv.R * cv.P);
        const uint32_t estr_m = m == 1 ? (uint32_t)cv.P : (uint32_t)(cv.R * cv.P);
        const int bstr_f = f == 1 ? cv.nb[0] : cv.nb[0] * cv.nb[1];
        const int bstr_m = m == 1 ? cv.nb[0] : cv.nb[0] * cv.nb[1];
        const uint32_t e_c = (uint32_t)(cv.O + cv.P + cv.R * cv.P) + (uint32_t)(Xlo & (cv.B - 1)) +
                             (uint32_t)(F & (cv.B - 1)) * estr_f;
        const int b_c = (Xlo >> cv.logB) + (F >> cv.logB) * bstr_f;
        const uint8_t *const base = cv.pool + (int64_t)b_c * cv.brick_bytes;
        const int64_t bstride = (int64_t)bstr_m * cv.brick_bytes;
        constexpr int es = DT == VRC_F32 ? 4 : (DT == VRC_BF16 ? 2 : 1);
        const float step = J.step;
        // sample k + u of every ray of the group, as the per-ray loop forms it
        auto index_of = [&](float kf, int u) {
            const float tk = __fadd_rn(tin, __fmul_rn(__fadd_rn(kf, (float)u + 0.5f), step));
            return make_int2(nearest_index(__fadd_rn(om, __fmul_rn(tk, dm)), nm), tk < tout);
        };
        for (int k = 0;; k += kRowU) {
            const float kf = (float)k;
            RowVec<DT, kRowG> rv[kRowU];
            int nv = 0;   // t grows with k, so the samples inside the ray form a prefix
#pragma unroll
            for (int u = 0; u < kRowU; ++u) {
                const int2 iv = index_of(kf, u);
                row_load<DT, kRowG>(base + (iv.x >> cv.logB) * bstride +
                                 (size_t)(e_c + (uint32_t)(iv.x & (cv.B - 1)) * estr_m) * es,
                             rv[u]);
                nv += iv.y;
            }
#pragma unroll
            for (int u = 0; u < kRowU; ++u) {
                // a sample past the rays' end read an in-bounds voxel (its index is
                // clamped) and counts as -FLT_MAX, which leaves every maximum as it is
                const bool in = u < nv;
                float v[kRowG];
                row_values<DT, kRowG>(rv[u], v);
                if (DT == VRC_FP8E4M3) {
                    // the brick's scale (its index formed again: fewer registers held across the loads)
                    const float sc = __ldg(cv.scales + b_c + (index_of(kf, u).x >> cv.logB) * bstr_m);
#pragma unroll
                    for (int j = 0; j < kRowG; ++j) mx[j] = fmaxf(mx[j], in ? __fmul_rn(v[j], sc) : -FLT_MAX);
                } else {
#pragma unroll
                    for (int j = 0; j < kRowG; ++j) mx[j] = fmaxf(mx[j], in ? v[j] : -FLT_MAX);
                }
            }
            nsamp += (uint32_t)(kRowG * nv);
            if (nv < kRowU) break;
        }
    }
    float *out = J.out + (int64_t)py * J.vp.W + px0;
#pragma unroll
    for (int i = 0; i < kRowG; ++i) out[i] = mx[sx > 0 ? i : kRowG - 1 - i];
    return true;
}

// One thread per group of kRowG pixels of a row (64 registers, 4 CTAs per SM:
// a 1024^2 view's 131,072 groups are all resident at once), every view of the launch the
// same size (groups_x groups per row, groups_per_job per view).
template <int DT>
__global__ void __launch_bounds__(kThreads, 4) k_mip_rows(const JobDesc *__restrict__ jobs, int n_jobs,
                                                      int64_t groups_per_job, int groups_x)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t nsamp = 0, neval = 0;
    if (g < groups_per_job * n_jobs) {
        const int jid = (int)(g / groups_per_job);
        const int64_t r = g - (int64_t)jid * groups_per_job;
        const JobDesc &J = jobs[jid];
        const int py = (int)(r / groups_x), px0 = (int)(r - (int64_t)py * groups_x) * kRowG;
        if (mip_row_group<DT>(J, px0, py, nsamp)) {
            neval = nsamp;
        } else {
#pragma unroll 1
            for (int i = 0; i < kRowG && px0 + i < J.vp.W; ++i)
                trace_fused<0, VRC_NEAREST, DT, -1, false>(J, nullptr, px0 + i, py, nsamp, neval);
        }
    }
    if (jobs[0].samples) warp_count2(jobs[0].samples, nsamp, neval);   // every job of the launch shares them
}

// Sort-last work item: one screen tile of one brick of one view.
struct BrickItem {
    int32_t job;
    int32_t brick;     // brick index in the cube's grid
    int32_t slot;      // storage slot: resident pool index or streaming ring slot
    int16_t tx, ty;    // tile origin / tile size
};

__device__ __forceinline__ bool member(const CubeView &cv, const float o[3], const float d[3], float tk, int bx,
                                       int by, int bz, float p[3])
{
    int ib[3];
    const int bc[3] = {bx, by, bz};
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p[a] = __fadd_rn(o[a], __fmul_rn(tk, d[a]));
        ib[a] = min(max((int)floorf(p[a]), 0), cv.dims[a] - 1) >> cv.logB;
        in = in && ib[a] == bc[a];
    }
    return in;
}

__device__ __forceinline__ int brick_key_of(const CubeView &cv, const ViewParams &vp, const float p[3])
{
    int key = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int b = min(max((int)floorf(p[a]), 0), cv.dims[a] - 1) >> cv.logB;
        key += abs(b - vp.ec[a]);
    }
    return key;
}

// Sort-last path: per item, the rays of one tile sample only their segment in
// one brick, starting from zero (DVR: premultiplied partial RGBA, stopping when
// the total alpha A_front + (1 - A_front) A_partial reaches term, A_front read
// from the running image), and write the brick's partial image.  Bricks of one
// wavefront (equal visibility key) never share a ray, so their partials are
// disjoint.  `slots` maps item.slot to brick storage.  TEX: trilinear
// samples from the brick's texture copy (two gathers, the same texels and
// weights as the global-load sampler; resident cubes with render copies).
template <int MODE, int SAMPLING, int DT, bool TEX>
__global__ void __launch_bounds__(kThreads) k_render_bricks(const JobDesc *__restrict__ jobs,
                                                            const BrickItem *__restrict__ items, int64_t n_items,
                                                            const uint8_t *slot_base, int64_t slot_bytes,
                                                            const float *__restrict__ running,
                                                            float *__restrict__ partial,
                                                            unsigned long long *samples)
{
    __shared__ float4 s_tf[256];
    const int64_t item_id = blockIdx.x;
    if (item_id >= n_items) return;
    const BrickItem it = items[item_id];
    const JobDesc &J = jobs[it.job];
    if (MODE == 1) {
        s_tf[threadIdx.x] = J.tf[threadIdx.x];
        __syncthreads();
    }
    const CubeView &cv = J.cv;
    int lx, ly;
    tile_pixel(J.tile_w, J.warp_w, lx, ly);
    const int px = it.tx + lx, py = it.ty + ly;
    uint32_t nsamp = 0;
    if (px < J.vp.W && py < J.vp.H) {
        const int bx = it.brick % cv.nb[0], by = (it.brick / cv.nb[0]) % cv.nb[1], bz = it.brick / (cv.nb[0] * cv.nb[1]);
        const int ox = bx << cv.logB, oy = by << cv.logB, oz = bz << cv.logB;
        const uint8_t *bp = slot_base + (int64_t)it.slot * slot_bytes;
        const float scale = DT == VRC_FP8E4M3 ? __ldg(cv.scales + it.brick) : 1.f;
        const unsigned long long th =
            TEX ? __ldg(cv.tex + 2 * (int64_t)cv.nb[0] * cv.nb[1] * cv.nb[2] + it.brick) : 0ull;
        const int bkey = abs(bx - J.vp.ec[0]) + abs(by - J.vp.ec[1]) + abs(bz - J.vp.ec[2]);
        float o[3], d[3], tin, tout;
        const int64_t pix = (int64_t)py * J.vp.W + px;
        const int64_t gpix = J.vp.out_offset + pix;
        float afront = 0.f;
        if (MODE == 1) afront = running[4 * gpix + 3];
        if (ray_setup(J.vp, cv.fdims, px, py, o, d, tin, tout) && !(MODE == 1 && afront >= J.term)) {
            // estimate the first sample inside the brick box from a slab test
            float lo = tin, hi = tout;
            const int oc[3] = {ox, oy, oz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (d[a] == 0.f) continue;
                const float b0 = (float)oc[a], b1 = fminf((float)(oc[a] + cv.B), cv.fdims[a]);
                float t0 = (b0 - o[a]) / d[a], t1 = (b1 - o[a]) / d[a];
                if (t0 > t1) {
                    const float tmp = t0;
                    t0 = t1;
                    t1 = tmp;
                }
                lo = fmaxf(lo, t0);
                hi = fminf(hi, t1);
            }
            int k = max(0, (int)ceilf((lo - tin) / J.step - 0.5f) - 1);
            float p[3];
            bool found = false;
            // walk to the first sample whose voxel lies in this brick: keys grow along the ray
            for (int it2 = 0; it2 < 8 && lo <= hi + 1.f; ++it2) {
                const float tk = sample_t(tin, k, J.step);
                if (!(tk < tout)) {
                    if (k == 0) break;
                    --k;
                    continue;
                }
                if (member(cv, o, d, tk, bx, by, bz, p)) {
                    found = true;
                    break;
                }
                const int key = brick_key_of(cv, J.vp, p);
                if (key < bkey) ++k;
                else if (key > bkey && k > 0) --k;
                else break;
            }
            if (found) {
                while (k > 0 && member(cv, o, d, sample_t(tin, k - 1, J.step), bx, by, bz, p)) --k;
                float m = -FLT_MAX;
                OverAcc acc;
                for (;; ++k) {
                    const float tk = sample_t(tin, k, J.step);
                    if (!(tk < tout)) break;
                    if (!member(cv, o, d, tk, bx, by, bz, p)) break;
                    float s;
                    if (SAMPLING == VRC_NEAREST) {
                        s = nearest_in_brick<DT>(cv, bp, min(max((int)floorf(p[0]), 0), cv.dims[0] - 1),
                                                 min(max((int)floorf(p[1]), 0), cv.dims[1] - 1),
                                                 min(max((int)floorf(p[2]), 0), cv.dims[2] - 1), ox, oy, oz, scale);
                    } else if (TEX) {
                        s = tri_tex<DT>(th, axis_tri(p[0], cv.dims[0]), axis_tri(p[1], cv.dims[1]),
                                           axis_tri(p[2], cv.dims[2]), ox, oy, oz, scale);
                    } else {
                        s = tri_in_brick<DT>(cv, bp, axis_tri(p[0], cv.dims[0]), axis_tri(p[1], cv.dims[1]),
                                             axis_tri(p[2], cv.dims[2]), ox, oy, oz, scale);
                    }
                    ++nsamp;
                    if (MODE == 0) {
                        m = fmaxf(m, s);
                    } else {
                        if (s == s) over(acc, classify(s_tf, s, J.vmin, J.inv_range), J.step, J.opacity_correction);
                        if (fmaf(1.f - afront, acc.A, afront) >= J.term) break;
                    }
                }
                if (MODE == 0) partial[gpix] = m;
                else reinterpret_cast<float4 *>(partial)[gpix] = make_float4(acc.rg.x, acc.rg.y, acc.b, acc.A);
            }
        }
    }
    if (samples) warp_count2(samples, nsamp, nsamp);
}

// Sort-last composite of a partial image into the running image (DVR: over,
// running = running + (1 - running.A) * partial; MIP: max), then reset the
// partial (DVR 0, MIP -FLT_MAX) when `reset` is set.
template <int MODE>
__global__ void k_composite(float *running, float *partial, const float *front, const float *back, float *out,
                            int64_t n, int reset)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (MODE == 0) {
            if (running) {
                running[i] = fmaxf(running[i], partial[i]);
                if (reset) partial[i] = -FLT_MAX;
            } else {
                out[i] = fmaxf(front[i], back[i]);
            }
        } else {
            float4 f, b;
            if (running) {
                f = reinterpret_cast<float4 *>(running)[i];
                b = reinterpret_cast<float4 *>(partial)[i];
            } else {
                f = reinterpret_cast<const float4 *>(front)[i];
                b = reinterpret_cast<const float4 *>(back)[i];
            }
            const float t = 1.f - f.w;
            const float4 r = make_float4(fmaf(t, b.x, f.x), fmaf(t, b.y, f.y), fmaf(t, b.z, f.z), fmaf(t, b.w, f.w));
            if (running) {
                reinterpret_cast<float4 *>(running)[i] = r;
                if (reset) reinterpret_cast<float4 *>(partial)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                reinterpret_cast<float4 *>(out)[i] = r;
            }
        }
    }
}

template <int MODE>
__global__ void k_fill(float *img, int64_t n, float v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        img[i] = v;
}

// ------------------------------------------------------------------ host side

CubeView cube_view(const Cube *c)
{
    CubeView v;
    const BrickGeom &g = c->g;
    v.pool = (const uint8_t *)c->pool;
    v.tex = c->dtex;
    v.scales = c->scales;
    v.brick_bytes = g.brick_bytes;
    v.B = g.B;
    v.logB = g.logB;
    v.P = g.P;
    v.O = g.O;
    v.R = g.R;
    for (int a = 0; a < 3; ++a) {
        v.nb[a] = g.nb[a];
        v.dims[a] = (int32_t)g.dims[a];
        v.fdims[a] = (float)g.dims[a];
    }
    v.dtype = g.dtype;
    return v;
}

ViewParams view_params(const vrc_camera &cam, const BrickGeom &g, int W, int H, int64_t out_offset)
{
    ViewParams vp;
    float basis[12];
    camera_basis(cam, W, H, basis);
    for (int a = 0; a < 3; ++a) {
        vp.O0[a] = basis[a];
        vp.D0[a] = basis[3 + a];
        vp.DX[a] = basis[6 + a];
        vp.DY[a] = basis[9 + a];
    }
    vp.kind = cam.kind;
    vp.W = W;
    vp.H = H;
    for (int a = 0; a < 3; ++a) {
        if (cam.kind == VRC_CAM_PERSP) {
            double f = std::floor((double)cam.eye[a] / (double)g.B);
            f = std::min(std::max(f, -1.0), (double)g.nb[a]);
            vp.ec[a] = (int32_t)f;
        } else {
            vp.ec[a] = vp.D0[a] > 0 ? -1 : (vp.D0[a] < 0 ? g.nb[a] : 0);
        }
    }
    vp.out_offset = out_offset;
    vp.tex_axis = 2;
    return vp;
}

bool valid_cam(const vrc_camera &c)
{
    if (c.kind != VRC_CAM_ORTHO && c.kind != VRC_CAM_PERSP) return false;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(c.eye[a]) || !std::isfinite(c.center[a]) || !std::isfinite(c.up[a])) return false;
    double w[3], cr[3];
    for (int a = 0; a < 3; ++a) w[a] = (double)c.center[a] - c.eye[a];
    cr[0] = w[1] * c.up[2] - w[2] * c.up[1];
    cr[1] = w[2] * c.up[0] - w[0] * c.up[2];
    cr[2] = w[0] * c.up[1] - w[1] * c.up[0];
    if (cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2] == 0.0) return false;  // up parallel to view / eye == center
    if (c.kind == VRC_CAM_PERSP && !(c.fovy_deg > 0.f && c.fovy_deg < 179.f)) return false;
    if (c.kind == VRC_CAM_ORTHO && !(c.ortho_height > 0.f && std::isfinite(c.ortho_height))) return false;
    return true;
}

vrc_status check_rc(vrc_ctx *ctx, const vrc_raycfg *rc)
{
    if (!rc) return set_err(ctx, VRC_E_INVAL, "null raycfg");
    if (rc->width < 1 || rc->height < 1 || rc->width > 16384 || rc->height > 16384)
        return set_err(ctx, VRC_E_INVAL, "image size out of range");
    if (!(rc->step > 0.f) || !std::isfinite(rc->step) || rc->step < 1e-3f)
        return set_err(ctx, VRC_E_INVAL, "step must be >= 1e-3");
    if (rc->sampling != VRC_NEAREST && rc->sampling != VRC_TRILINEAR) return set_err(ctx, VRC_E_INVAL, "bad sampling");
    if (rc->opacity_correction != 0 && rc->opacity_correction != 1) return set_err(ctx, VRC_E_INVAL, "bad opacity flag");
    if (rc->path != VRC_PATH_FUSED && rc->path != VRC_PATH_SORTLAST && rc->path != VRC_PATH_FUSED_LDG &&
        rc->path != VRC_PATH_ZEROCOPY && rc->path != VRC_PATH_SLAB)
        return set_err(ctx, VRC_E_INVAL, "bad path");
    if ((rc->skip_empty != 0 && rc->skip_empty != 1) || rc->reserved != 0)
        return set_err(ctx, VRC_E_INVAL, "bad skip_empty/reserved");
    const bool tile0 = rc->tile_w == 0 && rc->tile_h == 0;
    const bool tile_ok = (rc->tile_w == 8 || rc->tile_w == 16 || rc->tile_w == 32) && rc->tile_w * rc->tile_h == 256;
    if (!tile0 && !tile_ok) return set_err(ctx, VRC_E_INVAL, "tile must be 8x32, 16x16 or 32x8");
    return VRC_OK;
}

void pick_tile(const Cube *c, const vrc_raycfg &rc, int &tw, int &th)
{
    if (rc.tile_w) {
        tw = rc.tile_w;
        th = rc.tile_h;
    } else if (c->tile_w) {
        tw = c->tile_w;
        th = c->tile_h;
    } else if (rc.sampling == VRC_NEAREST) {
        // warps of 32 pixels along a row (nearest reads stored rows with
        // global loads): axis-aligned native MIP 1.06 ms against 1.11 ms with
        // 16x16 tiles on a 1024^3 fp32 cube
        tw = 32;
        th = 8;
    } else {
        tw = 16;
        th = 16;
    }
}

// Warp shape for a view.  Texture copies are layered along z, so a warp should
// spread its 32 pixels along the image axis that moves least in z: tall and
// narrow when the image's x axis runs along z (rays mostly along x), wide and
// flat when its y axis does, square-ish otherwise.
int warp_shape(const ViewParams &vp, int tw, int th)
{
    const float rz = std::fabs(vp.DX[2]), uz = std::fabs(vp.DY[2]);
    const float rn = std::sqrt(vp.DX[0] * vp.DX[0] + vp.DX[1] * vp.DX[1] + vp.DX[2] * vp.DX[2]);
    const float un = std::sqrt(vp.DY[0] * vp.DY[0] + vp.DY[1] * vp.DY[1] + vp.DY[2] * vp.DY[2]);
    const float fr = rn > 0 ? rz / rn : 0.f, fu = un > 0 ? uz / un : 0.f;
    int ww = 8;
    if (fr > 0.7f && fu < 0.5f) ww = 2;
    else if (fu > 0.7f && fr < 0.5f) ww = 16;
    while (ww > 1 && (tw % ww || th % (32 / ww))) ww >>= 1;   // fit the tile
    while (ww < 32 && (tw % ww || th % (32 / ww))) ww <<= 1;
    return ww;
}

// Warp shape for nearest sampling, which reads the packed bricks with global
// loads: a warp should spread its 32 pixels along the image axis that runs
// along the cube's x axis (the stored rows), so that each load instruction
// covers long runs of consecutive voxels.
int warp_shape_rows(const ViewParams &vp, int tw, int th)
{
    const float rn = std::sqrt(vp.DX[0] * vp.DX[0] + vp.DX[1] * vp.DX[1] + vp.DX[2] * vp.DX[2]);
    const float un = std::sqrt(vp.DY[0] * vp.DY[0] + vp.DY[1] * vp.DY[1] + vp.DY[2] * vp.DY[2]);
    const float fr = rn > 0 ? std::fabs(vp.DX[0]) / rn : 0.f, fu = un > 0 ? std::fabs(vp.DY[0]) / un : 0.f;
    int ww = 8;
    if (fr > 0.7f) ww = 32;
    else if (fu > 0.7f) ww = 1;
    while (ww > 1 && (tw % ww || th % (32 / ww))) ww >>= 1;   // fit the tile
    while (ww < 32 && (tw % ww || th % (32 / ww))) ww <<= 1;
    return ww;
}

// DVR empty-space threshold: with j0 the first TF entry of nonzero alpha, a
// sample value s gives alpha exactly 0 when 255 (s - min)/(max - min) <= j0 - 1
// (interpolation between zero entries).  The threshold keeps a 1e-5 relative
// margin so that binary32 evaluation of the TF index cannot cross j0 - 1.
float transparent_below(const Cube *c, const float *tf)
{
    int j0 = 0;
    while (j0 < 256 && tf[4 * j0 + 3] == 0.f) ++j0;
    if (j0 == 0) return -INFINITY;
    const double range = (double)c->vmax - (double)c->vmin;
    if (!(range > 0)) return j0 >= 1 ? INFINITY : -INFINITY;   // every sample has u = 0
    if (j0 >= 256) return INFINITY;                            // the TF is transparent everywhere
    const double thr = (double)c->vmin + (double)(j0 - 1) / 255.0 * range * (1.0 - 1e-5) - 1e-6 * std::fabs(c->vmin);
    return (float)thr;
}

JobDesc make_job(const Cube *c, const vrc_camera &cam, const vrc_raycfg &rc, int mode, float term, const float4 *dtf,
                 float *out, int64_t out_offset, int tw, int th)
{
    JobDesc j;
    j.cv = cube_view(c);
    j.vp = view_params(cam, c->g, rc.width, rc.height, out_offset);
    j.step = rc.step;
    j.term = term;
    j.vmin = c->vmin;
    const float range = c->vmax - c->vmin;
    j.inv_range = range > 0.f ? 1.f / range : 0.f;
    j.opacity_correction = rc.opacity_correction;
    j.tile_w = tw;
    j.tile_h = th;
    j.warp_w = rc.sampling == VRC_NEAREST ? warp_shape_rows(j.vp, tw, th) : warp_shape(j.vp, tw, th);
    j.tiles_x = (rc.width + tw - 1) / tw;
    j.tiles_y = (rc.height + th - 1) / th;
    j.item_begin = 0;
    j.tf = dtf;
    j.out = out + (mode == 0 ? 1 : 4) * out_offset;
    j.samples = nullptr;
    j.cellmax = (rc.skip_empty && c->cellmax && c->dtex && rc.sampling == VRC_TRILINEAR) ? c->cellmax : nullptr;
    j.ncx = c->ncell[0];
    j.ncy = c->ncell[1];
    j.skip_below = -INFINITY;
    (void)mode;
    return j;
}

template <int MODE, int SAMPLING, int DT, bool TEX, bool SKIP>
int fused_occupancy(int nthreads)
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_render_fused<MODE, SAMPLING, DT, TEX, SKIP>, nthreads, 0);
    return n > 0 ? n : 1;
}

// nthreads = the jobs' tile_w x tile_h (one thread per pixel of a tile; 256)
template <int MODE, int SAMPLING, int DT, bool TEX, bool SKIP>
void launch_fused_t(int grid, int nthreads, cudaStream_t st, const JobDesc *jobs, int n_jobs, int64_t total,
                    int *counter)
{
    k_render_fused<MODE, SAMPLING, DT, TEX, SKIP><<<grid, nthreads, 0, st>>>(jobs, n_jobs, total, counter);
}

// Views that the row-group MIP kernel can take: nearest MIP, orthographic,
// rays along y or z whose coordinate on that axis does not vary over the
// image, and image x moving along the cube's x axis one voxel per pixel (at
// other pixel spacings no group of 8 rays would fit, and the kernel would
// trace 8 rays per thread one after another).  The kernel checks each group
// of eight rays itself and takes the per-ray loop where they do not fit.
bool rows_views(const std::vector<JobDesc> &jobs, int mode, const vrc_raycfg &rc)
{
    if (mode != 0 || rc.sampling != VRC_NEAREST || rc.width < kRowG) return false;
    for (const JobDesc &j : jobs) {
        const ViewParams &vp = j.vp;
        if (vp.kind != VRC_CAM_ORTHO || vp.D0[0] != 0.f || (vp.D0[1] != 0.f) == (vp.D0[2] != 0.f)) return false;
        const int m = vp.D0[1] != 0.f ? 1 : 2;
        if (vp.DX[m] != 0.f || vp.DY[m] != 0.f || std::fabs(vp.DX[0]) != 1.f) return false;
    }
    return true;
}

void launch_rows(int dt, cudaStream_t st, const JobDesc *jobs, int n_jobs, int W, int H)
{
    const int gx = (W + kRowG - 1) / kRowG;
    const int64_t gpj = (int64_t)gx * H;
    const unsigned grid = (unsigned)((gpj * n_jobs + kThreads - 1) / kThreads);
    if (dt == VRC_F32) k_mip_rows<VRC_F32><<<grid, kThreads, 0, st>>>(jobs, n_jobs, gpj, gx);
    else if (dt == VRC_BF16) k_mip_rows<VRC_BF16><<<grid, kThreads, 0, st>>>(jobs, n_jobs, gpj, gx);
    else k_mip_rows<VRC_FP8E4M3><<<grid, kThreads, 0, st>>>(jobs, n_jobs, gpj, gx);
}

typedef void (*fused_fn)(int, int, cudaStream_t, const JobDesc *, int, int64_t, int *);
typedef int (*occ_fn)(int);

// Variant: nearest reads one voxel; trilinear reads texture gathers when the
// cubes have texture copies (TEX), optionally with empty-space skipping (SKIP).
template <int MODE, int DT>
fused_fn pick_fused3(int sampling, bool tex, bool skip)
{
    if (sampling == VRC_NEAREST) return launch_fused_t<MODE, VRC_NEAREST, DT, false, false>;
    if (!tex) return launch_fused_t<MODE, VRC_TRILINEAR, DT, false, false>;
    return skip ? launch_fused_t<MODE, VRC_TRILINEAR, DT, true, true> : launch_fused_t<MODE, VRC_TRILINEAR, DT, true, false>;
}
template <int MODE>
fused_fn pick_fused2(int sampling, int dt, bool tex, bool skip)
{
    if (dt == VRC_F32) return pick_fused3<MODE, VRC_F32>(sampling, tex, skip);
    if (dt == VRC_BF16) return pick_fused3<MODE, VRC_BF16>(sampling, tex, skip);
    return pick_fused3<MODE, VRC_FP8E4M3>(sampling, tex, skip);
}
fused_fn pick_fused(int mode, int sampling, int dt, bool tex, bool skip = false)
{
    return mode == 0 ? pick_fused2<0>(sampling, dt, tex, skip) : pick_fused2<1>(sampling, dt, tex, skip);
}
template <int MODE, int DT>
occ_fn pick_occ3(int sampling, bool tex, bool skip)
{
    if (sampling == VRC_NEAREST) return fused_occupancy<MODE, VRC_NEAREST, DT, false, false>;
    if (!tex) return fused_occupancy<MODE, VRC_TRILINEAR, DT, false, false>;
    return skip ? fused_occupancy<MODE, VRC_TRILINEAR, DT, true, true> : fused_occupancy<MODE, VRC_TRILINEAR, DT, true, false>;
}
template <int MODE>
occ_fn pick_occ2(int sampling, int dt, bool tex, bool skip)
{
    if (dt == VRC_F32) return pick_occ3<MODE, VRC_F32>(sampling, tex, skip);
    if (dt == VRC_BF16) return pick_occ3<MODE, VRC_BF16>(sampling, tex, skip);
    return pick_occ3<MODE, VRC_FP8E4M3>(sampling, tex, skip);
}
int occupancy(int mode, int sampling, int dt, bool tex, bool skip = false, int nthreads = kThreads)
{
    return mode == 0 ? pick_occ2<0>(sampling, dt, tex, skip)(nthreads)
                     : pick_occ2<1>(sampling, dt, tex, skip)(nthreads);
}

template <int MODE, int SAMPLING, int DT, bool TEX>
void launch_bricks_t(int64_t n, cudaStream_t st, const JobDesc *jobs, const BrickItem *items, const uint8_t *slot_base,
                     int64_t slot_bytes, const float *running, float *partial, unsigned long long *samples)
{
    k_render_bricks<MODE, SAMPLING, DT, TEX><<<(unsigned)n, kThreads, 0, st>>>(jobs, items, n, slot_base, slot_bytes,
                                                                              running, partial, samples);
}
typedef void (*bricks_fn)(int64_t, cudaStream_t, const JobDesc *, const BrickItem *, const uint8_t *, int64_t,
                          const float *, float *, unsigned long long *);
template <int MODE>
bricks_fn pick_bricks2(int sampling, int dt, bool tex)
{
    if (sampling == VRC_NEAREST) {
        if (dt == VRC_F32) return launch_bricks_t<MODE, VRC_NEAREST, VRC_F32, false>;
        if (dt == VRC_BF16) return launch_bricks_t<MODE, VRC_NEAREST, VRC_BF16, false>;
        return launch_bricks_t<MODE, VRC_NEAREST, VRC_FP8E4M3, false>;
    }
    if (tex) {
        if (dt == VRC_F32) return launch_bricks_t<MODE, VRC_TRILINEAR, VRC_F32, true>;
        if (dt == VRC_BF16) return launch_bricks_t<MODE, VRC_TRILINEAR, VRC_BF16, true>;
        return launch_bricks_t<MODE, VRC_TRILINEAR, VRC_FP8E4M3, true>;
    }
    if (dt == VRC_F32) return launch_bricks_t<MODE, VRC_TRILINEAR, VRC_F32, false>;
    if (dt == VRC_BF16) return launch_bricks_t<MODE, VRC_TRILINEAR, VRC_BF16, false>;
    return launch_bricks_t<MODE, VRC_TRILINEAR, VRC_FP8E4M3, false>;
}
bricks_fn pick_bricks(int mode, int sampling, int dt, bool tex)
{
    return mode == 0 ? pick_bricks2<0>(sampling, dt, tex) : pick_bricks2<1>(sampling, dt, tex);
}

// Scratch layout helpers: [counter | samples | tf | jobs | items ...]
struct Arena {
    char *base;
    size_t off, cap;
    template <class T>
    T *take(size_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += sizeof(T) * n;
        return p;
    }
};

// ----------------------------------------------------- brick screen footprints

// Pixel bounding box of brick b (conservative; full image if the brick reaches
// behind the eye).  Returns false if it is entirely off screen.
bool brick_bbox(const vrc_camera &cam, const BrickGeom &g, int W, int H, int b, int box[4])
{
    const int bx = b % g.nb[0], by = (b / g.nb[0]) % g.nb[1], bz = b / (g.nb[0] * g.nb[1]);
    double lo[3] = {(double)bx * g.B, (double)by * g.B, (double)bz * g.B};
    double hi[3] = {std::min((double)(bx + 1) * g.B, (double)g.dims[0]), std::min((double)(by + 1) * g.B, (double)g.dims[1]),
                    std::min((double)(bz + 1) * g.B, (double)g.dims[2])};
    for (int a = 0; a < 3; ++a) {
        lo[a] -= 1.0;
        hi[a] += 1.0;
    }
    double e[3], w[3], r[3], u[3];
    for (int a = 0; a < 3; ++a) {
        e[a] = cam.eye[a];
        w[a] = (double)cam.center[a] - cam.eye[a];
    }
    double lw = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int a = 0; a < 3; ++a) w[a] /= lw;
    r[0] = w[1] * cam.up[2] - w[2] * cam.up[1];
    r[1] = w[2] * cam.up[0] - w[0] * cam.up[2];
    r[2] = w[0] * cam.up[1] - w[1] * cam.up[0];
    double lr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) r[a] /= lr;
    u[0] = r[1] * w[2] - r[2] * w[1];
    u[1] = r[2] * w[0] - r[0] * w[2];
    u[2] = r[0] * w[1] - r[1] * w[0];
    const double asp = (double)W / H;
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int c = 0; c < 8; ++c) {
        double p[3] = {(c & 1) ? hi[0] : lo[0], (c & 2) ? hi[1] : lo[1], (c & 4) ? hi[2] : lo[2]};
        double dv[3] = {p[0] - e[0], p[1] - e[1], p[2] - e[2]};
        double zc = dv[0] * w[0] + dv[1] * w[1] + dv[2] * w[2];
        double xc = dv[0] * r[0] + dv[1] * r[1] + dv[2] * r[2];
        double yc = dv[0] * u[0] + dv[1] * u[1] + dv[2] * u[2];
        double xn, yn;
        if (cam.kind == VRC_CAM_PERSP) {
            if (zc <= 1e-6) {
                box[0] = 0;
                box[1] = 0;
                box[2] = W;
                box[3] = H;
                return true;
            }
            const double h = std::tan((double)cam.fovy_deg * 3.14159265358979323846 / 360.0);
            xn = xc / (zc * h * asp);
            yn = yc / (zc * h);
        } else {
            const double h = 0.5 * cam.ortho_height;
            xn = xc / (h * asp);
            yn = yc / h;
        }
        const double pxf = (xn + 1.0) * 0.5 * W - 0.5, pyf = (1.0 - yn) * 0.5 * H - 0.5;
        xmin = std::min(xmin, pxf);
        xmax = std::max(xmax, pxf);
        ymin = std::min(ymin, pyf);
        ymax = std::max(ymax, pyf);
    }
    const double x0 = std::floor(xmin) - 2, x1 = std::ceil(xmax) + 3, y0 = std::floor(ymin) - 2, y1 = std::ceil(ymax) + 3;
    if (x1 <= 0 || y1 <= 0 || x0 >= W || y0 >= H) return false;
    box[0] = (int)std::max(0.0, x0);
    box[1] = (int)std::max(0.0, y0);
    box[2] = (int)std::min((double)W, x1);
    box[3] = (int)std::min((double)H, y1);
    return box[0] < box[2] && box[1] < box[3];
}

struct Wave {
    int key;
    std::vector<int> bricks;  // bricks of this wavefront that some view sees
};

// Sort-last plan: wavefronts (equal Manhattan distance of the brick from the
// eye's brick cell) in front-to-back order, with per-(view, brick) tiles.
struct SortLastPlan {
    std::vector<int> wave_key;                 // per wavefront
    std::vector<std::vector<int>> wave_bricks; // distinct bricks per wavefront
    std::vector<BrickItem> items;              // grouped by wavefront, then brick
    std::vector<int64_t> brick_item_begin;     // per (wavefront, brick) entry
    std::vector<int64_t> wave_item_begin;      // per wavefront (+ end)
    int64_t culled = 0;                        // crossed bricks left out (transparent)
    int64_t traversed() const
    {
        int64_t n = 0;
        for (const auto &w : wave_bricks) n += (int64_t)w.size();
        return n;
    }
};

// Bricks whose largest sample value (halo included) is at or below cull_le
// hold no visible sample (DVR, transparent transfer function) and are left out;
// cull_le = -inf keeps every brick.
void plan_sortlast(const Cube *c, const std::vector<JobDesc> &jobs, const std::vector<vrc_camera> &cams,
                   float cull_le, SortLastPlan &plan)
{
    const BrickGeom &g = c->g;
    const int nb = (int)g.nbricks;
    // keys per view; wavefront index = key (0 .. max) is a valid order for every view
    int maxkey = 0;
    std::vector<std::vector<int>> key(jobs.size(), std::vector<int>(nb));
    for (size_t v = 0; v < jobs.size(); ++v)
        for (int b = 0; b < nb; ++b) {
            const int bx = b % g.nb[0], by = (b / g.nb[0]) % g.nb[1], bz = b / (g.nb[0] * g.nb[1]);
            const int k = std::abs(bx - jobs[v].vp.ec[0]) + std::abs(by - jobs[v].vp.ec[1]) + std::abs(bz - jobs[v].vp.ec[2]);
            key[v][b] = k;
            maxkey = std::max(maxkey, k);
        }
    plan.items.clear();
    plan.wave_key.clear();
    plan.wave_bricks.clear();
    plan.wave_item_begin.clear();
    plan.brick_item_begin.clear();
    plan.culled = 0;
    const bool cull = cull_le > -INFINITY && (int64_t)c->h_bhalo_max.size() == g.nbricks;
    for (int k = 0; k <= maxkey; ++k) {
        std::vector<int> bricks;
        const int64_t wbeg = (int64_t)plan.items.size();
        for (int b = 0; b < nb; ++b) {
            const int64_t bbeg = (int64_t)plan.items.size();
            const bool culled = cull && c->h_bhalo_max[b] <= cull_le;
            bool crossed = false;
            for (size_t v = 0; v < jobs.size(); ++v) {
                if (key[v][b] != k) continue;
                int box[4];
                if (!brick_bbox(cams[v], g, jobs[v].vp.W, jobs[v].vp.H, b, box)) continue;
                crossed = true;
                if (culled) continue;
                const int tw = jobs[v].tile_w, th = jobs[v].tile_h;
                for (int y = (box[1] / th) * th; y < box[3]; y += th)
                    for (int x = (box[0] / tw) * tw; x < box[2]; x += tw)
                        plan.items.push_back(BrickItem{(int32_t)v, b, b, (int16_t)x, (int16_t)y});
            }
            if ((int64_t)plan.items.size() > bbeg) {
                bricks.push_back(b);
                plan.brick_item_begin.push_back(bbeg);
            }
            plan.culled += culled && crossed;
        }
        if ((int64_t)plan.items.size() > wbeg) {
            plan.wave_key.push_back(k);
            plan.wave_bricks.push_back(bricks);
            plan.wave_item_begin.push_back(wbeg);
        }
    }
    plan.wave_item_begin.push_back((int64_t)plan.items.size());
    plan.brick_item_begin.push_back((int64_t)plan.items.size());
}

int grid_for(int64_t n, int cap) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, cap)); }

vrc_status render_common(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views,
                         const vrc_raycfg *rc, const float *tf_rgba, float term, float *out, cudaStream_t st, int mode,
                         int ctas_override, unsigned long long *samples_out, bool host_sync_samples);

}  // namespace

// ------------------------------------------------------------------ render entry

namespace {

vrc_status validate_render(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views, const vrc_raycfg *rc,
                           const float *tf, float term, float *out, int mode, Cube **cube, CubeUse &use,
                           cudaStream_t st)
{
    if (!ctx) return VRC_E_INVAL;
    if (!cams || !out || n_views < 1 || n_views > 4096) return set_err(ctx, VRC_E_INVAL, "bad cams/out/n_views");
    vrc_status s = check_rc(ctx, rc);
    if (s != VRC_OK) return s;
    if (mode == 1 && (!tf || !(term > 0.f) || std::isnan(term))) return set_err(ctx, VRC_E_INVAL, "bad tf/term");
    if (mode == 1)
        for (int i = 0; i < 1024; ++i)
            if (!std::isfinite(tf[i])) return set_err(ctx, VRC_E_INVAL, "tf has non-finite entries");
    for (int v = 0; v < n_views; ++v)
        if (!valid_cam(cams[v])) return set_err(ctx, VRC_E_INVAL, "bad camera %d", v);
    Cube *c = nullptr;
    if ((s = acquire_cube(ctx, cube_id, st, &c, use)) != VRC_OK) return s;
    if ((s = validate_step(ctx, c, rc->step)) != VRC_OK) return s;
    *cube = c;
    return VRC_OK;
}

vrc_status render_streamed(vrc_ctx *ctx, Cube *c, SortLastPlan &plan, const vrc_raycfg &rc, float *out,
                           int64_t npix_total, int mode, cudaStream_t st, unsigned long long *dsamples, Arena &ar,
                           const JobDesc *djobs);

vrc_status render_common(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views, const vrc_raycfg *rc,
                         const float *tf_rgba, float term, float *out, cudaStream_t st, int mode, int ctas_override,
                         unsigned long long *samples_out, bool host_sync_samples)
{
    Cube *c = nullptr;
    CubeUse use;
    vrc_status s = validate_render(ctx, cube_id, cams, n_views, rc, tf_rgba, term, out, mode, &c, use, st);
    if (s != VRC_OK) return s;
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    int tw, th;
    pick_tile(c, *rc, tw, th);
    const int64_t npix = (int64_t)rc->width * rc->height;
    std::vector<JobDesc> jobs(n_views);
    std::vector<vrc_camera> camv(cams, cams + n_views);
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) {
        jobs[v] = make_job(c, cams[v], *rc, mode, term, nullptr, out, v * npix, tw, th);
        jobs[v].item_begin = total;
        total += (int64_t)jobs[v].tiles_x * jobs[v].tiles_y;
    }
    if (rc->path == VRC_PATH_ZEROCOPY && !c->streamed)
        return set_err(ctx, VRC_E_UNSUPPORTED, "zero-copy rendering is for streamed cubes");
    const bool slab = rc->path == VRC_PATH_SLAB;
    if (slab) {
        if (!slab_supported(c) || rc->sampling != VRC_TRILINEAR || rc->skip_empty)
            return set_err(ctx, VRC_E_UNSUPPORTED, "slab path: resident float32 cubes, trilinear, no skip_empty");
        if ((s = slab_prepare(ctx, c, st)) != VRC_OK) return s;
        for (auto &j : jobs) j.warp_w = 8;   // 8x4-pixel warps: compact footprints in the staged box
    }
    const bool zerocopy = rc->path == VRC_PATH_ZEROCOPY;
    const bool sortlast = c->streamed || rc->path == VRC_PATH_SORTLAST;
    const bool rows = !slab && !sortlast && !zerocopy && rows_views(jobs, mode, *rc);
    ctx->last_path = rows ? VRC_PATH_ROWS : slab ? VRC_PATH_SLAB
                          : (zerocopy ? VRC_PATH_ZEROCOPY
                                      : (c->streamed ? VRC_PATH_STREAMED
                                                     : (sortlast ? VRC_PATH_SORTLAST
                                                                 : (rc->path == VRC_PATH_FUSED && c->dtex &&
                                                                            rc->sampling == VRC_TRILINEAR
                                                                        ? VRC_PATH_FUSED
                                                                        : VRC_PATH_FUSED_LDG))));
    if (!sortlast && !c->pool) return set_err(ctx, VRC_E_UNSUPPORTED, "cube has no resident bricks");
    if (c->streamed && c->n_filled < c->n_host)
        return set_err(ctx, VRC_E_INVAL, "streamed cube: %lld of %lld host slots never written",
                       (long long)(c->n_host - c->n_filled), (long long)c->n_host);
    if (zerocopy && c->source && c->n_host < c->g.nbricks)
        return set_err(ctx, VRC_E_UNSUPPORTED, "zero-copy rendering reads every brick in place: the host cache "
                       "must hold all %lld bricks", (long long)c->g.nbricks);
    const float thr = mode == 1 ? transparent_below(c, tf_rgba) : -INFINITY;
    SortLastPlan plan;
    if (sortlast) plan_sortlast(c, jobs, camv, rc->skip_empty && mode == 1 ? thr : -INFINITY, plan);
    ctx->last_bricks[0] = sortlast ? plan.traversed() : 0;
    ctx->last_bricks[1] = sortlast ? plan.culled : 0;
    const size_t img_floats = (size_t)n_views * npix * (mode == 0 ? 1 : 4);
    size_t need = 4096 + 1024 * 4 + sizeof(JobDesc) * n_views + 256 * 4;
    if (sortlast) need += sizeof(BrickItem) * plan.items.size() + sizeof(float) * img_floats + 1024;
    void *scr = nullptr;
    if ((s = scratch_get(ctx, need, &scr)) != VRC_OK) return s;
    Arena ar{(char *)scr, 0, need};
    int *counter = ar.take<int>(1);
    unsigned long long *dsamples = ar.take<unsigned long long>(3);   // lattice, evaluated, wait failure
    float4 *dtf = ar.take<float4>(256);
    JobDesc *djobs = ar.take<JobDesc>(n_views);
    for (auto &j : jobs) {
        if (mode == 1) j.tf = dtf;
        j.samples = dsamples;
        j.skip_below = thr;
    }
    // tables in, counters zeroed: one small kernel, no copy-engine work
    if ((s = stage_h2d(ctx, st, {{dtf, tf_rgba, mode == 1 ? (size_t)1024 * 4 : 0},
                                 {djobs, jobs.data(), sizeof(JobDesc) * n_views},
                                 {dsamples, nullptr, 3 * sizeof(unsigned long long)},
                                 {counter, nullptr, sizeof(int)}})) != VRC_OK)
        return s;
    if (slab) {
        const int per_sm = ctas_override > 0 ? ctas_override : slab_occupancy(mode);
        const int grid = (int)std::min<int64_t>((int64_t)ctx->sm_count * per_sm, total);
        slab_launch(c, mode, grid, st, djobs, n_views, total, counter, reinterpret_cast<int *>(dsamples + 2),
                    inject_fire(ctx, VRC_INJECT_SLAB_WAIT));
        count_launch(ctx);
        VRC_CK(ctx, cudaGetLastError());
    } else if (rows) {
        launch_rows(c->g.dtype, st, djobs, n_views, rc->width, rc->height);
        count_launch(ctx);
        VRC_CK(ctx, cudaGetLastError());
    } else if (!sortlast) {
        const bool tex = rc->path == VRC_PATH_FUSED && c->dtex != nullptr;
        const bool skip = tex && jobs[0].cellmax != nullptr;
        int per_sm = ctas_override > 0 ? ctas_override
                                       : (c->ctas_per_sm > 0 ? c->ctas_per_sm
                                                             : occupancy(mode, rc->sampling, c->g.dtype, tex, skip,
                                                                         tw * th));
        const int grid = (int)std::min<int64_t>((int64_t)ctx->sm_count * per_sm, total);
        pick_fused(mode, rc->sampling, c->g.dtype, tex, skip)(grid, tw * th, st, djobs, n_views, total, counter);
        count_launch(ctx);
        VRC_CK(ctx, cudaGetLastError());
    } else if (!c->streamed || zerocopy) {
        // resident bricks, or (zero-copy) bricks read in place from mapped pinned host memory
        if (zerocopy)
            for (BrickItem &it : plan.items) it.slot = (int32_t)(it.brick % c->n_host);
        const uint8_t *slot_base = (const uint8_t *)(zerocopy ? c->host_pool_dev : c->pool);
        BrickItem *ditems = ar.take<BrickItem>(std::max<size_t>(1, plan.items.size()));
        float *partial = ar.take<float>(img_floats);
        if (!plan.items.empty() &&
            (s = stage_h2d(ctx, st, {{ditems, plan.items.data(), sizeof(BrickItem) * plan.items.size()}})) != VRC_OK)
            return s;
        const int64_t n = (int64_t)img_floats;
        const int g = grid_for(n, ctx->sm_count * 8);
        if (mode == 0) {
            k_fill<0><<<g, 256, 0, st>>>(out, n, -FLT_MAX);
            k_fill<0><<<g, 256, 0, st>>>(partial, n, -FLT_MAX);
        } else {
            VRC_CK(ctx, cudaMemsetAsync(out, 0, sizeof(float) * n, st));
            VRC_CK(ctx, cudaMemsetAsync(partial, 0, sizeof(float) * n, st));
        }
        count_launch(ctx, mode == 0 ? 2 : 0);
        // resident bricks with render copies sample them through texture gathers
        bricks_fn bf = pick_bricks(mode, rc->sampling, c->g.dtype, !zerocopy && !c->streamed && c->dtex != nullptr);
        const int64_t npx = (int64_t)n_views * npix;
        for (size_t w = 0; w + 1 < plan.wave_item_begin.size(); ++w) {
            const int64_t b0 = plan.wave_item_begin[w], b1 = plan.wave_item_begin[w + 1];
            if (b1 <= b0) continue;
            bf(b1 - b0, st, djobs, ditems + b0, slot_base, c->g.brick_bytes, out, partial, dsamples);
            const int gc = grid_for(npx, ctx->sm_count * 8);
            if (mode == 0) k_composite<0><<<gc, 256, 0, st>>>(out, partial, nullptr, nullptr, nullptr, npx, 1);
            else k_composite<1><<<gc, 256, 0, st>>>(out, partial, nullptr, nullptr, nullptr, npx, 1);
            count_launch(ctx, 2);
        }
        VRC_CK(ctx, cudaGetLastError());
    } else {
        s = render_streamed(ctx, c, plan, *rc, out, (int64_t)n_views * npix, mode, st, dsamples, ar, djobs);
        if (s != VRC_OK) return s;
    }
    if (samples_out) {
        VRC_CK(ctx, cudaMemcpyAsync(samples_out, dsamples, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        if (host_sync_samples) VRC_CK(ctx, cudaStreamSynchronize(st));
    } else {
        VRC_CK(ctx, cudaMemcpyAsync(ctx->h_samples, dsamples, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        VRC_CK(ctx, cudaEventRecord(ctx->ev_samples, st));
    }
    return VRC_OK;
}

// Out-of-core: bricks of a streamed cube are copied from pinned host slots to a
// device ring on a side stream, in wavefront order, in chunks of half the ring;
// chunk i renders while chunk i+1 copies.  Each wavefront's partial image is
// composited after its last chunk.
vrc_status render_streamed(vrc_ctx *ctx, Cube *c, SortLastPlan &plan, const vrc_raycfg &rc, float *out,
                           int64_t npx, int mode, cudaStream_t st, unsigned long long *dsamples, Arena &ar,
                           const JobDesc *djobs)
{
    const BrickGeom &g = c->g;
    // chunks: runs of consecutive bricks inside one wavefront, at most half the ring
    const int half = c->ring / 2;
    struct Chunk {
        int64_t item_b, item_e;
        std::vector<int> bricks;
        bool wave_end;
        int parity;
    };
    std::vector<Chunk> chunks;
    size_t bi = 0;  // index into plan.brick_item_begin
    for (size_t w = 0; w < plan.wave_bricks.size(); ++w) {
        const auto &wb = plan.wave_bricks[w];
        for (size_t k = 0; k < wb.size(); k += half) {
            Chunk ch;
            ch.item_b = plan.brick_item_begin[bi];
            const size_t n = std::min<size_t>(half, wb.size() - k);
            for (size_t q = 0; q < n; ++q) ch.bricks.push_back(wb[k + q]);
            bi += n;
            ch.item_e = plan.brick_item_begin[bi];
            ch.wave_end = k + n == wb.size();
            ch.parity = (int)(chunks.size() & 1);
            chunks.push_back(ch);
        }
    }
    // ring slot of each item: parity half + position of its brick in the chunk
    for (const Chunk &ch : chunks)
        for (int64_t it = ch.item_b; it < ch.item_e; ++it) {
            const int pos = (int)(std::find(ch.bricks.begin(), ch.bricks.end(), plan.items[it].brick) - ch.bricks.begin());
            plan.items[it].slot = ch.parity * half + pos;
        }
    const int64_t img_floats = npx * (mode == 0 ? 1 : 4);
    BrickItem *ditems = ar.take<BrickItem>(std::max<size_t>(1, plan.items.size()));
    float *partial = ar.take<float>(img_floats);
    if (!plan.items.empty()) {
        const vrc_status ss = stage_h2d(ctx, st, {{ditems, plan.items.data(), sizeof(BrickItem) * plan.items.size()}});
        if (ss != VRC_OK) return ss;
    }
    const int gfill = grid_for(img_floats, ctx->sm_count * 8);
    if (mode == 0) {
        k_fill<0><<<gfill, 256, 0, st>>>(out, img_floats, -FLT_MAX);
        k_fill<0><<<gfill, 256, 0, st>>>(partial, img_floats, -FLT_MAX);
        count_launch(ctx, 2);
    } else {
        VRC_CK(ctx, cudaMemsetAsync(out, 0, sizeof(float) * img_floats, st));
        VRC_CK(ctx, cudaMemsetAsync(partial, 0, sizeof(float) * img_floats, st));
    }
    cudaStream_t cs;
    VRC_CK(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    std::vector<cudaEvent_t> ready(chunks.size()), consumed(chunks.size());
    cudaEvent_t entry;
    cudaEventCreateWithFlags(&entry, cudaEventDisableTiming);
    cudaEventRecord(entry, st);             // earlier work on `st` may still use the ring
    cudaStreamWaitEvent(cs, entry, 0);
    vrc_status status = VRC_OK;
    bricks_fn bf = pick_bricks(mode, rc.sampling, c->g.dtype, false);
    size_t made = 0;
    for (size_t i = 0; i < chunks.size() && status == VRC_OK; ++i) {
        const Chunk &ch = chunks[i];
        cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&consumed[i], cudaEventDisableTiming);
        made = i + 1;
        if (i >= 2) cudaStreamWaitEvent(cs, consumed[i - 2], 0);   // slots of this parity are free again
        for (size_t q = 0; q < ch.bricks.size(); ++q) {
            if (inject_fire(ctx, VRC_INJECT_H2D)) {
                status = set_err(ctx, VRC_E_INJECTED, "injected host-to-device brick copy failure");
                break;
            }
            // the host slot of the brick (a provider cube refills it when it holds another brick)
            int64_t hslot = 0;
            if ((status = host_brick(ctx, c, ch.bricks[q], &hslot)) != VRC_OK) break;
            const char *src = (const char *)c->host_pool + hslot * g.brick_bytes;
            char *dst = (char *)c->ring_pool + (int64_t)(ch.parity * half + q) * g.brick_bytes;
            cudaError_t e = cudaMemcpyAsync(dst, src, g.brick_bytes, cudaMemcpyHostToDevice, cs);
            if (e != cudaSuccess) {
                status = cuda_err(ctx, e, "brick H2D");
                break;
            }
            if ((status = host_copied(ctx, c, hslot, cs)) != VRC_OK) break;
        }
        if (status != VRC_OK) break;
        cudaEventRecord(ready[i], cs);
        cudaStreamWaitEvent(st, ready[i], 0);
        if (ch.item_e > ch.item_b)
            bf(ch.item_e - ch.item_b, st, djobs, ditems + ch.item_b, (const uint8_t *)c->ring_pool, g.brick_bytes,
               out, partial, dsamples);
        count_launch(ctx);
        cudaEventRecord(consumed[i], st);
        if (ch.wave_end) {
            const int gc = grid_for(npx, ctx->sm_count * 8);
            if (mode == 0) k_composite<0><<<gc, 256, 0, st>>>(out, partial, nullptr, nullptr, nullptr, npx, 1);
            else k_composite<1><<<gc, 256, 0, st>>>(out, partial, nullptr, nullptr, nullptr, npx, 1);
            count_launch(ctx);
        }
    }
    // the copy stream must not outlive pending copies unnoticed: join it into `st`
    cudaEvent_t tail;
    cudaEventCreateWithFlags(&tail, cudaEventDisableTiming);
    cudaEventRecord(tail, cs);
    cudaStreamWaitEvent(st, tail, 0);
    cudaEventDestroy(tail);
    cudaEventDestroy(entry);
    for (size_t i = 0; i < made; ++i) {
        cudaEventDestroy(ready[i]);
        cudaEventDestroy(consumed[i]);
    }
    cudaStreamDestroy(cs);
    if (status != VRC_OK) return status;
    VRC_CK(ctx, cudaGetLastError());
    return VRC_OK;
}

}  // namespace

extern "C" {

vrc_status vrc_render_mip(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views, const vrc_raycfg *rc,
                          float *out, void *stream)
{
    return render_common(ctx, cube_id, cams, n_views, rc, nullptr, 0.f, out, (cudaStream_t)stream, 0, 0, nullptr, false);
}

vrc_status vrc_render_dvr(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views, const vrc_raycfg *rc,
                          const float *tf_rgba, float term_alpha, float *out, void *stream)
{
    return render_common(ctx, cube_id, cams, n_views, rc, tf_rgba, term_alpha, out, (cudaStream_t)stream, 1, 0, nullptr,
                         false);
}

vrc_status vrc_last_render_path(vrc_ctx *ctx, int32_t *path)
{
    if (!ctx || !path) return VRC_E_INVAL;
    *path = ctx->last_path.load();
    return VRC_OK;
}

vrc_status vrc_composite(vrc_ctx *ctx, const float *front, const float *back, float *out, int64_t n_pixels, int32_t mode,
                         void *stream)
{
    if (!ctx || !front || !back || !out || n_pixels < 0 || (mode != 0 && mode != 1)) return VRC_E_INVAL;
    if (n_pixels == 0) return VRC_OK;
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int g = grid_for(n_pixels, ctx->sm_count * 8);
    if (mode == 0) k_composite<0><<<g, 256, 0, st>>>(nullptr, nullptr, front, back, out, n_pixels, 0);
    else k_composite<1><<<g, 256, 0, st>>>(nullptr, nullptr, front, back, out, n_pixels, 0);
    count_launch(ctx);
    VRC_CK(ctx, cudaGetLastError());
    return VRC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ graphs

struct vrc_graph {
    vrc_ctx *ctx;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    void *mem;
    size_t mem_bytes;
};

extern "C" {

vrc_status vrc_graph_create(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views,
                            const vrc_raycfg *rc, const float *tf_rgba, float term_alpha, float *out,
                            vrc_graph **graph)
{
    if (!graph) return VRC_E_INVAL;
    *graph = nullptr;
    const int mode = tf_rgba ? 1 : 0;
    Cube *c = nullptr;
    CubeUse use;
    vrc_status s = validate_render(ctx, cube_id, cams, n_views, rc, tf_rgba, term_alpha, out, mode, &c, use, nullptr);
    if (s != VRC_OK) return s;
    if (c->managed) return set_err(ctx, VRC_E_UNSUPPORTED, "graphs need a cube uploaded with vrc_cube_upload");
    if (c->streamed || rc->path == VRC_PATH_SORTLAST || rc->path == VRC_PATH_SLAB)
        return set_err(ctx, VRC_E_UNSUPPORTED, "graphs capture the fused path of resident cubes");
    const bool tex = rc->path == VRC_PATH_FUSED && c->dtex != nullptr;
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    int tw, th;
    pick_tile(c, *rc, tw, th);
    const int64_t npix = (int64_t)rc->width * rc->height;
    std::vector<JobDesc> jobs(n_views);
    int64_t total = 0;
    const size_t bytes = 4096 + 4096 + sizeof(JobDesc) * n_views + 1024;
    void *mem = nullptr;
    if ((s = dev_alloc(ctx, &mem, bytes)) != VRC_OK) return s;
    Arena ar{(char *)mem, 0, bytes};
    int *counter = ar.take<int>(1);
    unsigned long long *dsamples = ar.take<unsigned long long>(3);   // lattice, evaluated, wait failure
    float4 *dtf = ar.take<float4>(256);
    JobDesc *djobs = ar.take<JobDesc>(n_views);
    const float thr = mode ? transparent_below(c, tf_rgba) : -INFINITY;
    for (int v = 0; v < n_views; ++v) {
        jobs[v] = make_job(c, cams[v], *rc, mode, term_alpha, mode ? dtf : nullptr, out, v * npix, tw, th);
        jobs[v].samples = dsamples;
        jobs[v].skip_below = thr;
        jobs[v].item_begin = total;
        total += (int64_t)jobs[v].tiles_x * jobs[v].tiles_y;
    }
    cudaError_t e = cudaSuccess;
    if (mode) e = cudaMemcpy(dtf, tf_rgba, 4096, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(djobs, jobs.data(), sizeof(JobDesc) * n_views, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dev_free(ctx, mem, bytes);
        return cuda_err(ctx, e, "graph upload");
    }
    const bool skip = tex && jobs[0].cellmax != nullptr;
    const int per_sm =
        c->ctas_per_sm > 0 ? c->ctas_per_sm : occupancy(mode, rc->sampling, c->g.dtype, tex, skip, tw * th);
    const int grid = (int)std::min<int64_t>((int64_t)ctx->sm_count * per_sm, total);
    cudaStream_t cs;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
        dev_free(ctx, mem, bytes);
        return cuda_err(ctx, e, "graph stream");
    }
    vrc_graph *gph = new vrc_graph{ctx, nullptr, nullptr, mem, bytes};
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(counter, 0, sizeof(int), cs);
        cudaMemsetAsync(dsamples, 0, 2 * sizeof(unsigned long long), cs);
        pick_fused(mode, rc->sampling, c->g.dtype, tex, skip)(grid, tw * th, cs, djobs, n_views, total, counter);
        e = cudaStreamEndCapture(cs, &gph->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gph->exec, gph->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (gph->graph) cudaGraphDestroy(gph->graph);
        dev_free(ctx, mem, bytes);
        delete gph;
        return cuda_err(ctx, e, "graph capture");
    }
    *graph = gph;
    return VRC_OK;
}

vrc_status vrc_graph_launch(vrc_graph *g, void *stream)
{
    if (!g) return VRC_E_INVAL;
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_err(g->ctx, e, "cudaGraphLaunch");
    count_launch(g->ctx);
    return VRC_OK;
}

vrc_status vrc_graph_destroy(vrc_graph *g)
{
    if (!g) return VRC_E_INVAL;
    cudaDeviceSynchronize();
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    dev_free(g->ctx, g->mem, g->mem_bytes);
    delete g;
    return VRC_OK;
}

// ------------------------------------------------------------------ autotuner

vrc_status vrc_autotune(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views, const vrc_raycfg *rc,
                        const float *tf_rgba, float term_alpha, float *out, void *stream, vrc_tuning *result)
{
    const int mode = tf_rgba ? 1 : 0;
    Cube *c = nullptr;
    CubeUse use;
    vrc_status s = validate_render(ctx, cube_id, cams, n_views, rc, tf_rgba, term_alpha, out, mode, &c, use,
                                   (cudaStream_t)stream);
    if (s != VRC_OK) return s;
    if (c->streamed) return set_err(ctx, VRC_E_UNSUPPORTED, "autotuning needs a resident cube");
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int tiles[3][2] = {{8, 32}, {16, 16}, {32, 8}};
    const int occ = occupancy(mode, rc->sampling, c->g.dtype, rc->path == VRC_PATH_FUSED && c->dtex != nullptr);
    cudaEvent_t e0, e1;
    VRC_CK(ctx, cudaEventCreate(&e0));
    VRC_CK(ctx, cudaEventCreate(&e1));
    const int old_w = c->tile_w, old_h = c->tile_h, old_c = c->ctas_per_sm;
    c->tile_w = c->tile_h = c->ctas_per_sm = 0;
    double best = 1e300, dflt = 0;
    int bw = 16, bh = 16, bc = occ;
    for (int t = 0; t < 3; ++t)
        for (int per_sm = 1; per_sm <= occ; ++per_sm) {
            vrc_raycfg r = *rc;
            if (r.path == VRC_PATH_SORTLAST) r.path = VRC_PATH_FUSED;
            r.tile_w = tiles[t][0];
            r.tile_h = tiles[t][1];
            double ms_best = 1e300;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(e0, st);
                s = render_common(ctx, cube_id, cams, n_views, &r, tf_rgba, term_alpha, out, st, mode, per_sm, nullptr,
                                  false);
                cudaEventRecord(e1, st);
                if (s != VRC_OK) break;
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                ms_best = std::min(ms_best, (double)ms);
            }
            if (s != VRC_OK) break;
            if (tiles[t][0] == 16 && per_sm == occ) dflt = ms_best;
            if (ms_best < best) {
                best = ms_best;
                bw = tiles[t][0];
                bh = tiles[t][1];
                bc = per_sm;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != VRC_OK) {
        c->tile_w = old_w;
        c->tile_h = old_h;
        c->ctas_per_sm = old_c;
        return s;
    }
    c->tile_w = bw;
    c->tile_h = bh;
    c->ctas_per_sm = bc;
    if (result) {
        result->tile_w = bw;
        result->tile_h = bh;
        result->ctas_per_sm = bc;
        result->brick = c->g.B;
        result->step = rc->step;
        result->reserved = 0;
        result->best_ms = best;
        result->default_ms = dflt;
        result->step_max_abs_diff = 0.0;
    }
    return VRC_OK;
}

}  // extern "C"

namespace {

// Largest |a - b| over n floats, as the bits of a non-negative float (which
// order like unsigned integers) in *out (zeroed by the caller).
__global__ void k_max_abs_diff(const float *__restrict__ a, const float *__restrict__ b, int64_t n, unsigned int *out)
{
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(a[i] - b[i]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Time one render (best of two) with the cube's tuned configuration.
vrc_status time_render(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views, const vrc_raycfg &r,
                       const float *tf, float term, float *out, cudaStream_t st, double *ms_out)
{
    cudaEvent_t e0, e1;
    VRC_CK(ctx, cudaEventCreate(&e0));
    VRC_CK(ctx, cudaEventCreate(&e1));
    double best = 1e300;
    vrc_status s = VRC_OK;
    for (int rep = 0; rep < 2 && s == VRC_OK; ++rep) {
        cudaEventRecord(e0, st);
        s = render_common(ctx, cube_id, cams, n_views, &r, tf, term, out, st, tf ? 1 : 0, 0, nullptr, false);
        cudaEventRecord(e1, st);
        if (s != VRC_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, (double)ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = best;
    return s;
}

}  // namespace

extern "C" {

vrc_status vrc_autotune_cube(vrc_ctx *ctx, int64_t cube_id, const vrc_camera *cams, int32_t n_views,
                             const vrc_raycfg *rc, const float *tf_rgba, float term_alpha, float *out, void *stream,
                             int32_t flags, float step_tolerance, vrc_tuning *result)
{
    if (!ctx || !result) return VRC_E_INVAL;
    if ((flags & ~VRC_TUNE_BRICK) != 0) return set_err(ctx, VRC_E_INVAL, "unknown tuning flags %d", flags);
    if (!(step_tolerance >= 0.f)) return set_err(ctx, VRC_E_INVAL, "step tolerance must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    vrc_tuning best{};
    vrc_status s = vrc_autotune(ctx, cube_id, cams, n_views, rc, tf_rgba, term_alpha, out, stream, &best);
    if (s != VRC_OK) return s;
    const double default_ms = best.default_ms;
    int64_t best_id = cube_id;
    // held for the whole call: a registered cube is not evicted while it is re-packed
    Cube *c = nullptr;
    CubeUse use;
    if ((s = acquire_cube(ctx, cube_id, st, &c, use)) != VRC_OK) return s;
    // 1. brick edges: trial cubes re-packed on the device from the stored values
    if ((flags & VRC_TUNE_BRICK) && c->g.dtype != VRC_FP8E4M3 && c->pool) {
        const BrickGeom g = c->g;
        const int64_t n = g.dims[0] * g.dims[1] * g.dims[2];
        int64_t maxd = std::max(g.dims[0], std::max(g.dims[1], g.dims[2])), cap = 16;
        while (cap < maxd) cap *= 2;
        float *lin = nullptr;
        if ((s = dev_alloc(ctx, (void **)&lin, (size_t)n * 4)) != VRC_OK) return s;
        s = unpack_cube(ctx, c, lin, st);
        for (int B = 64; B <= 256 && s == VRC_OK; B *= 2) {
            if (B == g.B || B > cap) continue;
            Cube *t = new (std::nothrow) Cube();
            if (!t) break;
            if (!make_geom(g.dims[0], g.dims[1], g.dims[2], B, g.dtype, &t->g, 32)) {
                delete t;
                continue;
            }
            t->copy_mode = c->copy_mode == VRC_COPY_NONE ? VRC_COPY_NONE : VRC_COPY_REQUIRED;
            if (upload_cube(ctx, t, lin, 1, st) != VRC_OK) {   // no room in the budget: skip this edge
                delete t;
                continue;
            }
            const int64_t tid = register_cube(ctx, t);
            vrc_tuning r{};
            const vrc_status ts = vrc_autotune(ctx, tid, cams, n_views, rc, tf_rgba, term_alpha, out, stream, &r);
            if (ts == VRC_OK && r.best_ms < best.best_ms) {
                if (best_id != cube_id) vrc_cube_free(ctx, best_id);
                best = r;
                best_id = tid;
            } else {
                vrc_cube_free(ctx, tid);
            }
        }
        cudaStreamSynchronize(st);
        dev_free(ctx, lin, (size_t)n * 4);
        if (s != VRC_OK) {
            if (best_id != cube_id) vrc_cube_free(ctx, best_id);
            return s;
        }
        if (best_id != cube_id) {
            // the winner's storage takes the cube's id; the old storage is released
            Cube *old = nullptr, *w = nullptr;
            {
                std::lock_guard<std::mutex> lk(ctx->mu);
                old = ctx->cubes[cube_id];
                w = ctx->cubes[best_id];
                // this call's own reference is the only one allowed
                if (old->refs.load() > 1 || old->state.load() == CUBE_LOADING) {
                    s = set_err(ctx, VRC_E_BUSY, "cube in use by serving requests: storage not replaced");
                } else {
                    ctx->cubes.erase(best_id);
                    w->id = cube_id;
                    w->managed = old->managed;
                    w->host_src = old->host_src;
                    w->host_pinned = old->host_pinned;
                    old->host_pinned = false;
                    w->loads = old->loads;
                    w->last_use = old->last_use;
                    ctx->cubes[cube_id] = w;
                }
            }
            if (s != VRC_OK) {
                vrc_cube_free(ctx, best_id);
                return s;
            }
            // hand the reference over to the new storage before the old one goes
            w->refs.fetch_add(1);
            use.c = w;
            old->refs.fetch_sub(1);
            release_cube(ctx, old, true);
            c = w;
        }
    }
    best.brick = c->g.B;
    best.default_ms = default_ms;
    best.step = rc->step;
    best.step_max_abs_diff = 0.0;
    // 2. step: faster steps whose image stays within the tolerance
    if (step_tolerance > 0.f) {
        const int64_t nfl = (int64_t)n_views * rc->width * rc->height * (tf_rgba ? 4 : 1);
        float *ref = nullptr;
        unsigned int *dmax = nullptr;
        if ((s = dev_alloc(ctx, (void **)&ref, (size_t)nfl * 4 + 256)) != VRC_OK) return s;
        dmax = reinterpret_cast<unsigned int *>(ref + nfl);
        vrc_raycfg r = *rc;
        double step_ms = 0;
        s = time_render(ctx, cube_id, cams, n_views, r, tf_rgba, term_alpha, out, st, &step_ms);
        if (s == VRC_OK && cudaMemcpyAsync(ref, out, (size_t)nfl * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            s = cuda_err(ctx, cudaGetLastError(), "reference image");
        const float factors[3] = {1.25f, 1.5f, 2.f};
        for (int i = 0; i < 3 && s == VRC_OK; ++i) {
            r.step = rc->step * factors[i];
            if (validate_step(ctx, c, r.step) != VRC_OK) break;
            double ms = 0;
            if ((s = time_render(ctx, cube_id, cams, n_views, r, tf_rgba, term_alpha, out, st, &ms)) != VRC_OK) break;
            cudaMemsetAsync(dmax, 0, 4, st);
            k_max_abs_diff<<<grid_for(nfl, ctx->sm_count * 8), 256, 0, st>>>(out, ref, nfl, dmax);
            count_launch(ctx);
            unsigned int bits = 0;
            if (cudaMemcpyAsync(&bits, dmax, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                s = cuda_err(ctx, cudaGetLastError(), "image difference");
                break;
            }
            float diff;
            std::memcpy(&diff, &bits, 4);
            if (diff <= step_tolerance && ms < step_ms) {
                step_ms = ms;
                best.step = r.step;
                best.step_max_abs_diff = diff;
            }
        }
        cudaStreamSynchronize(st);
        dev_free(ctx, ref, (size_t)nfl * 4 + 256);
        if (s != VRC_OK) return s;
    }
    *result = best;
    return VRC_OK;
}

}  // extern "C"

// ------------------------------------------------------------- serving helper

constexpr int kMaxSlices = 1024;   // launches per heterogeneous render batch (each with its own counter)

size_t render_hetero_scratch_bytes(const std::vector<HetJob> &jobs)
{
    return 4 * kMaxSlices + 1024 + 4096 * jobs.size() + sizeof(JobDesc) * jobs.size() + 1024;
}

size_t render_hetero_counter_bytes(size_t n_jobs) { return 16 * n_jobs; }

size_t render_hetero_stage_bytes(size_t n_jobs) { return 4096 * n_jobs + sizeof(JobDesc) * n_jobs + 4 * kMaxSlices + 512; }

// Persistent launches over renders of different cubes, image sizes, cameras
// and transfer functions (all with the same mode/sampling/dtype).  The batch's
// (job, tile) items are cut into slices of at most `slice_items` (0: one
// launch), each one launch with its own work counter: requests that arrive
// while a large batch runs get SMs at the next slice boundary (from a stream
// of higher priority) instead of after the whole batch; every pixel is
// computed the same way whichever launch takes its tile.  Job i counts its
// samples into dev_samples[2i] (lattice) and [2i+1] (evaluated), zeroed here.
// host_stage: pinned host memory of render_hetero_stage_bytes() used to upload
// the job table without waiting.
vrc_status render_hetero(vrc_ctx *ctx, const std::vector<HetJob> &hj, cudaStream_t st, void *scratch,
                         size_t scratch_bytes, unsigned long long *dev_samples, void *host_stage, int64_t slice_items)
{
    if (hj.empty()) return VRC_OK;
    const int mode = hj[0].mode, sampling = hj[0].rc.sampling, dt = hj[0].cube->g.dtype;
    Arena ar{(char *)scratch, 0, scratch_bytes};
    int *counters = ar.take<int>(kMaxSlices);
    float4 *dtf = ar.take<float4>(256 * hj.size());
    JobDesc *djobs = ar.take<JobDesc>(hj.size());
    float *htf = (float *)host_stage;
    JobDesc *hjobs = (JobDesc *)((char *)host_stage + 4096 * hj.size());
    int *hcount = (int *)((char *)hjobs + sizeof(JobDesc) * hj.size());
    int64_t total = 0;
    for (size_t i = 0; i < hj.size(); ++i) {
        const HetJob &h = hj[i];
        int tw, th;
        pick_tile(h.cube, h.rc, tw, th);
        hjobs[i] = make_job(h.cube, h.cam, h.rc, mode, h.term, mode ? dtf + 256 * i : nullptr, h.out, 0, tw, th);
        hjobs[i].samples = dev_samples + 2 * i;
        hjobs[i].skip_below = mode ? transparent_below(h.cube, h.tf_host) : -INFINITY;
        hjobs[i].item_begin = total;
        total += (int64_t)hjobs[i].tiles_x * hjobs[i].tiles_y;
        if (mode) std::memcpy(htf + 1024 * i, h.tf_host, 4096);
    }
    bool tex = true, skip = true;
    for (size_t i = 0; i < hj.size(); ++i) {
        tex = tex && hj[i].cube->dtex != nullptr;
        skip = skip && hjobs[i].cellmax != nullptr;
    }
    skip = skip && tex;
    // slices: slice s takes items [begin_s, begin_{s+1}); its counter starts at begin_s
    int64_t per = slice_items > 0 ? slice_items : total;
    per = std::max<int64_t>(per, (total + kMaxSlices - 1) / kMaxSlices);
    const int nslices = (int)((total + per - 1) / per);
    for (int k = 0; k < nslices; ++k) hcount[k] = (int)(k * per);
    VRC_CK(ctx, cudaMemcpyAsync(counters, hcount, sizeof(int) * nslices, cudaMemcpyHostToDevice, st));
    VRC_CK(ctx, cudaMemsetAsync(dev_samples, 0, 2 * sizeof(unsigned long long) * hj.size(), st));
    if (mode) VRC_CK(ctx, cudaMemcpyAsync(dtf, htf, 4096 * hj.size(), cudaMemcpyHostToDevice, st));
    VRC_CK(ctx, cudaMemcpyAsync(djobs, hjobs, sizeof(JobDesc) * hj.size(), cudaMemcpyHostToDevice, st));
    const int per_sm = occupancy(mode, sampling, dt, tex, skip);
    const fused_fn fn = pick_fused(mode, sampling, dt, tex, skip);
    for (int k = 0; k < nslices; ++k) {
        const int64_t end = std::min<int64_t>(total, (int64_t)(k + 1) * per);
        const int grid = (int)std::min<int64_t>((int64_t)ctx->sm_count * per_sm, end - (int64_t)k * per);
        fn(grid, kThreads, st, djobs, (int)hj.size(), end, counters + k);
        count_launch(ctx);
    }
    VRC_CK(ctx, cudaGetLastError());
    return VRC_OK;
}

// Tiles per slice of a heterogeneous launch: two waves of persistent CTAs.
int64_t render_hetero_slice_items(vrc_ctx *ctx, const std::vector<HetJob> &hj)
{
    if (hj.empty()) return 0;
    bool tex = true;
    for (const HetJob &h : hj) tex = tex && h.cube->dtex != nullptr;
    return 2 * (int64_t)ctx->sm_count * occupancy(hj[0].mode, hj[0].rc.sampling, hj[0].cube->g.dtype, tex, false);
}

vrc_status validate_raycfg(vrc_ctx *ctx, const vrc_raycfg *rc) { return check_rc(ctx, rc); }

// A ray crosses at most the cube's diagonal; the samplers count samples in
// binary32 (k + 0.5 must stay exact), so a ray may hold at most 2^22 samples.
vrc_status validate_step(vrc_ctx *ctx, const Cube *c, float step)
{
    const double diag = std::sqrt((double)c->g.dims[0] * c->g.dims[0] + (double)c->g.dims[1] * c->g.dims[1] +
                                  (double)c->g.dims[2] * c->g.dims[2]);
    if (!(diag / (double)step < 4194304.0))
        return set_err(ctx, VRC_E_INVAL, "step %g too small: more than 2^22 samples per ray", (double)step);
    return VRC_OK;
}
bool camera_is_valid(const vrc_camera &c) { return valid_cam(c); }
