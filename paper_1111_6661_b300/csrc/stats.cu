// Fused global statistics over resident bricks (min/max, mean, std, histogram)
// and exact median by radix selection (bracketed by a sampled first digit on resident cubes).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <float.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "vrc_internal.h"

namespace {

constexpr int kStatsThreads = 256;
constexpr int kSmemBinsMax = 16384;   // 64 KB of shared-memory counters

struct StatPartial {
    double s1, s2;                 // sum of d and d^2, d = x - shift
    unsigned long long n, nnf;
};

struct StatsArgs {
    const uint8_t *pool;
    BrickGeom g;
    const float *scales;
    const int32_t *bnonfinite;     // per brick: non-finite interior voxels
    float vmin, hscale;            // histogram: bin = trunc(fl(fl(x - vmin) * hscale))
    float shift;                   // c: moments use d = (x - c) * dscale (c has 8 significant bits)
    float dscale;                  // power of two keeping d^2 finite in binary32
    float kq;                      // power of two >= max d^2: seed of the Fast2Sum accumulator
    int nbins;
    int all_full;                  // every brick lies inside the cube (dims are multiples of B)
    unsigned long long *hist;      // device [nbins], zeroed by the caller
    StatPartial *partials;         // device [gridDim.x]
    int accumulate;                // add to the partials instead of writing them (runs of an out-of-core cube)
    int64_t brick0, nrun;          // the pool holds bricks brick0 .. brick0 + nrun - 1 of the cube
};

template <int DT>
__device__ __forceinline__ void decode16(const uint4 &raw, float scale, float *x)
{
    if (DT == VRC_F32) {
        x[0] = __uint_as_float(raw.x);
        x[1] = __uint_as_float(raw.y);
        x[2] = __uint_as_float(raw.z);
        x[3] = __uint_as_float(raw.w);
    } else if (DT == VRC_BF16) {
        const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[2 * i] = __uint_as_float(w[i] << 16);
            x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    } else {
        const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] & 0xffffu), __NV_E4M3);
            const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] >> 16), __NV_E4M3);
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
            x[4 * i + 0] = __fmul_rn(a.x, scale);
            x[4 * i + 1] = __fmul_rn(a.y, scale);
            x[4 * i + 2] = __fmul_rn(b.x, scale);
            x[4 * i + 3] = __fmul_rn(b.y, scale);
        }
    }
}

// Measured on the 1024^3 fp32 cube with 4096 bins: 8 vectors in flight per
// lane at 3 CTAs of 256 per SM (80 registers, no spills) 0.83 ms; 8 at 4 CTAs
// (64 registers, spills) 0.84 ms; 4 at 4 or 3 CTAs 0.89-0.90 ms; the next
// chunk's 8 vectors loaded before the current chunk is accumulated (2 CTAs
// per SM) 0.845 ms, with 4 + 4 vectors at 3 CTAs 0.94 ms.
constexpr int kVecPerLane = 8;                 // 16-byte vectors in flight per lane
constexpr int kLogChunk = 8;                   // 256 vectors per warp iteration (32 lanes x 8)
constexpr int kStatsCtasPerSm = 3;
static_assert((1 << kLogChunk) == 32 * kVecPerLane, "chunk");

struct Acc {
    float2 s_hi, s_lo;                         // TwoSum accumulation of d (two lanes of f32x2)
    float2 q_hi, q_lo;                         // Fast2Sum accumulation of d^2
    uint32_t n = 0, nnf = 0;
};

// One 16-byte vector of VE values.  CHECK: mask element e by `nvalid` and
// finiteness; otherwise every element is a finite voxel inside the cube.
// Every accumulation is error-free per element: d by TwoSum, d^2 = P - En by
// TwoProd and a Fast2Sum into q_hi (seeded with kq >= every P), so repeated
// values (quantised cubes) cannot bias the sums.
template <int VE, int HIST, bool CHECK>
__device__ __forceinline__ void accumulate(const float *x, int nvalid, const StatsArgs &a, uint32_t *sh, Acc &acc)
{
    const float2 s2 = make_float2(a.dscale, a.dscale), ns2 = make_float2(-a.dscale, -a.dscale);
    const float cs = __fmul_rn(a.shift, a.dscale);
    const float2 cs2 = make_float2(cs, cs), ncs2 = make_float2(-cs, -cs);
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 nvmin2 = make_float2(-a.vmin, -a.vmin), hs2 = make_float2(a.hscale, a.hscale);
#pragma unroll
    for (int e = 0; e < VE; e += 2) {
        float2 X = make_float2(x[e], x[e + 1]);
        bool v0 = true, v1 = true;
        if (CHECK) {
            v0 = e < nvalid && fabsf(X.x) <= FLT_MAX;
            v1 = e + 1 < nvalid && fabsf(X.y) <= FLT_MAX;
            acc.nnf += (e < nvalid && !v0 ? 1u : 0u) + (e + 1 < nvalid && !v1 ? 1u : 0u);
            acc.n += (v0 ? 1u : 0u) + (v1 ? 1u : 0u);
            if (!v0) X.x = a.shift;           // contributes d = 0
            if (!v1) X.y = a.shift;
        }
        // d = fl(x - c) * s, computed as fl((x - c) s): scaling by 2^k commutes with rounding
        const float2 D = __ffma2_rn(X, s2, ncs2);
        const float2 Dn = __ffma2_rn(X, ns2, cs2);
        // TwoSum of d into s_hi + s_lo
        const float2 T1 = __fadd2_rn(acc.s_hi, D);
        const float2 BP = __ffma2_rn(acc.s_hi, m1, T1);
        const float2 AP = __ffma2_rn(BP, m1, T1);
        const float2 E1 = __ffma2_rn(AP, m1, acc.s_hi);
        const float2 E2 = __ffma2_rn(BP, m1, D);
        acc.s_hi = T1;
        acc.s_lo = __fadd2_rn(acc.s_lo, __fadd2_rn(E1, E2));
        // exact square d^2 = P - En; Fast2Sum of P into q_hi (q_hi >= kq >= P)
        const float2 P = __fmul2_rn(D, D);
        const float2 En = __ffma2_rn(Dn, D, P);
        const float2 T = __fadd2_rn(acc.q_hi, P);
        const float2 Z = __ffma2_rn(acc.q_hi, m1, T);
        const float2 Er = __ffma2_rn(Z, m1, P);
        acc.q_hi = T;
        acc.q_lo = __fadd2_rn(acc.q_lo, __ffma2_rn(En, m1, Er));
        if (HIST) {
            // bin = trunc(t), t = fl(fl(x - min) * scale) in [0, nbins * (1 + 2^-23)]: t == nbins
            // (x == max) lands in a guard counter that the flush folds into the last bin
            const float2 Tb = __fmul2_rn(__fadd2_rn(X, nvmin2), hs2);
            const int nbm1 = a.nbins - 1;
            const int b0 = HIST == 1 ? (int)Tb.x : min((int)Tb.x, nbm1);
            const int b1 = HIST == 1 ? (int)Tb.y : min((int)Tb.y, nbm1);
            if (!CHECK || v0) {
                if (HIST == 1) atomicAdd(&sh[b0], 1u);
                else atomicAdd(&a.hist[b0], 1ull);
            }
            if (!CHECK || v1) {
                if (HIST == 1) atomicAdd(&sh[b1], 1u);
                else atomicAdd(&a.hist[b1], 1ull);
            }
        }
    }
    if (!CHECK) acc.n += VE;
}

// One pass over the interior of every brick.  A warp takes 256 16-byte vectors
// (whole interior rows of one brick) per iteration, 8 per lane in flight;
// addresses inside a brick are 32-bit byte offsets and a brick's coordinates
// are only computed (32-bit division) for bricks on the cube's border.
// Moments: d = (x - c) s with c ~ the mean (8 significant bits, so x - c is exact
// for every voxel not far below |c|; c = 0 for FP8 cubes, whose values repeat);
// d summed by TwoSum, d^2 exactly (TwoProd) into a Fast2Sum accumulator seeded
// with a power of two kq >= every square; binary32 pairs (f32x2) throughout;
// binary64 per block.  Histogram: the stated binary32 bin formula into shared-memory
// counters (HIST 1) or global counters (HIST 2), flushed once per block.
template <int DT, int HIST>
__global__ void __launch_bounds__(kStatsThreads, kStatsCtasPerSm) k_stats(StatsArgs a)
{
    extern __shared__ uint32_t sh_hist[];
    constexpr int VE = DT == VRC_F32 ? 4 : (DT == VRC_BF16 ? 8 : 16);
    constexpr int LOG_VE = DT == VRC_F32 ? 2 : (DT == VRC_BF16 ? 3 : 4);
    const BrickGeom &g = a.g;
    if (HIST == 1) {
        for (int i = threadIdx.x; i <= a.nbins; i += blockDim.x) sh_hist[i] = 0;   // nbins + guard
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int logVPR = g.logB - LOG_VE;
    const int logRPC = kLogChunk - logVPR;     // rows per chunk (divides B*B)
    const int logCPB = 2 * g.logB - logRPC;    // chunks per brick
    const int64_t total_chunks = a.nrun << logCPB;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // byte offsets inside a brick (a brick is below 2^32 bytes): rows of P elements,
    // slices of R rows; vector i of this lane sits loff[i] bytes after its chunk's
    // first row when the chunk's rows lie in one slice (B >= 64)
    const uint32_t Pb = (uint32_t)(g.P * g.esize), RPb = (uint32_t)g.R * Pb, Ob = (uint32_t)(g.O * g.esize);
    const bool one_slice = logRPC <= g.logB;
    uint32_t loff[kVecPerLane];
#pragma unroll
    for (int i = 0; i < kVecPerLane; ++i) {
        const uint32_t j = lane + 32 * i;
        loff[i] = (j >> logVPR) * Pb + Ob + ((j & ((1u << logVPR) - 1)) << 4);
    }
    Acc acc;
    acc.s_hi = make_float2(0.f, 0.f);
    acc.s_lo = make_float2(0.f, 0.f);
    acc.q_hi = make_float2(a.kq, a.kq);
    acc.q_lo = make_float2(0.f, 0.f);
    for (int64_t ch = warp0; ch < total_chunks; ch += nwarps) {
        const uint32_t pb = (uint32_t)(ch >> logCPB);          // brick slot in the pool
        const uint32_t b = pb + (uint32_t)a.brick0;            // brick of the cube
        const uint32_t lr0 = ((uint32_t)ch & ((1u << logCPB) - 1)) << logRPC;
        // bricks that lie inside the cube and hold only finite voxels take the
        // unchecked path; their coordinates are needed only otherwise
        bool clean;
        if (a.all_full) {
            clean = __ldg(a.bnonfinite + b) == 0;
        } else {
            const uint32_t bx = b % (uint32_t)g.nb[0], byz = b / (uint32_t)g.nb[0];
            const uint32_t by = byz % (uint32_t)g.nb[1], bz = byz / (uint32_t)g.nb[1];
            clean = ((int64_t)(bx + 1) << g.logB) <= g.dims[0] && ((int64_t)(by + 1) << g.logB) <= g.dims[1] &&
                    ((int64_t)(bz + 1) << g.logB) <= g.dims[2] && __ldg(a.bnonfinite + b) == 0;
        }
        const uint8_t *bp = a.pool + (uint64_t)pb * (uint64_t)g.brick_bytes;
        const float scale = DT == VRC_FP8E4M3 ? __ldg(a.scales + b) : 1.f;
        uint4 raw[kVecPerLane];
        if (one_slice) {
            const uint32_t rb = ((lr0 >> g.logB) + 1) * RPb + ((lr0 & (g.B - 1)) + 1) * Pb;
#pragma unroll
            for (int i = 0; i < kVecPerLane; ++i) raw[i] = __ldcs(reinterpret_cast<const uint4 *>(bp + rb + loff[i]));
        } else {
#pragma unroll
            for (int i = 0; i < kVecPerLane; ++i) {
                const uint32_t j = lane + 32 * i;
                const uint32_t lr = lr0 + (j >> logVPR);
                const uint32_t off = ((lr >> g.logB) + 1) * RPb + ((lr & (g.B - 1)) + 1) * Pb + Ob +
                                     ((j & ((1u << logVPR) - 1)) << 4);
                raw[i] = __ldcs(reinterpret_cast<const uint4 *>(bp + off));
            }
        }
#pragma unroll
        for (int i = 0; i < kVecPerLane; ++i) {
            float x[VE];
            decode16<DT>(raw[i], scale, x);
            if (clean) {
                accumulate<VE, HIST, false>(x, VE, a, sh_hist, acc);
            } else {
                // brick at the cube's border or holding non-finite voxels: mask by position
                const uint32_t j = lane + 32 * i;
                const uint32_t lr = lr0 + (j >> logVPR);
                const uint32_t bx = b % (uint32_t)g.nb[0], byz = b / (uint32_t)g.nb[0];
                const uint32_t by = byz % (uint32_t)g.nb[1], bz = byz / (uint32_t)g.nb[1];
                const int64_t gx0 = ((int64_t)bx << g.logB) + ((int64_t)(j & ((1u << logVPR) - 1)) << LOG_VE);
                const int64_t gy = ((int64_t)by << g.logB) + (lr & (g.B - 1)), gz = ((int64_t)bz << g.logB) + (lr >> g.logB);
                int nvalid = (int)min((int64_t)VE, g.dims[0] - gx0);
                if (gy >= g.dims[1] || gz >= g.dims[2] || nvalid < 0) nvalid = 0;
                accumulate<VE, HIST, true>(x, nvalid, a, sh_hist, acc);
            }
        }
    }
    double s1 = ((double)acc.s_hi.x + (double)acc.s_lo.x) + ((double)acc.s_hi.y + (double)acc.s_lo.y);
    double s2 = ((double)acc.q_hi.x - (double)a.kq) + (double)acc.q_lo.x + ((double)acc.q_hi.y - (double)a.kq) +
                (double)acc.q_lo.y;
    unsigned long long n64 = acc.n, nnf64 = acc.nnf;
    for (int o = 16; o; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        n64 += __shfl_xor_sync(0xffffffffu, n64, o);
        nnf64 += __shfl_xor_sync(0xffffffffu, nnf64, o);
    }
    __shared__ StatPartial wp[kStatsThreads / 32];
    if ((threadIdx.x & 31) == 0) wp[threadIdx.x / 32] = StatPartial{s1, s2, n64, nnf64};
    __syncthreads();
    if (threadIdx.x == 0) {
        StatPartial r = wp[0];
        for (int w = 1; w < kStatsThreads / 32; ++w) {
            r.s1 += wp[w].s1;
            r.s2 += wp[w].s2;
            r.n += wp[w].n;
            r.nnf += wp[w].nnf;
        }
        if (a.accumulate) {
            StatPartial &p = a.partials[blockIdx.x];
            p.s1 += r.s1;
            p.s2 += r.s2;
            p.n += r.n;
            p.nnf += r.nnf;
        } else {
            a.partials[blockIdx.x] = r;
        }
    }
    if (HIST == 1) {
        __syncthreads();
        for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) {
            const uint32_t cnt = sh_hist[i] + (i == a.nbins - 1 ? sh_hist[a.nbins] : 0u);
            if (cnt) atomicAdd(&a.hist[i], (unsigned long long)cnt);
        }
    }
}

// FP8 storage: a voxel's stored value depends only on its brick's scale and
// its 8-bit code, so the statistics follow exactly from per-brick code counts.
// Work items are runs of 2^6 chunks (chunks as in k_stats) of one brick,
// assigned to blocks in a fixed order; a block counts an item's codes in
// shared memory (one shared-memory increment per voxel and no arithmetic),
// then thread q turns code q's count k into its share of n or n_nonfinite,
// the moments in binary64 (k * d and k * d^2 with d = value * dscale; the
// shift c is 0 for FP8) and the value histogram (the same binary32 bin
// formula as k_stats, one global add per code present).  One partial per
// block, merged by k_stats_final like those of k_stats.
constexpr int kLogCodeChunks = 6;

// Work items of the code-count passes over an FP8 cube: runs of 2^lcpi chunks
// of one brick (chunks as in k_stats: 256 16-byte vectors of interior rows).
struct CodeItems {
    int logVPR, logRPC, lcpi, ipb;
    int64_t items;
    uint32_t Pb, RPb, Ob;
};

// nrun: bricks in the pool (the whole cube, or one run of an out-of-core cube)
__device__ __forceinline__ CodeItems code_items(const BrickGeom &g, int64_t nrun)
{
    CodeItems ci;
    ci.logVPR = g.logB - 4;                          // 16 codes per vector
    ci.logRPC = kLogChunk - ci.logVPR;
    const int logCPB = 2 * g.logB - ci.logRPC;
    ci.lcpi = min(kLogCodeChunks, logCPB);
    ci.ipb = logCPB - ci.lcpi;
    ci.items = nrun << ci.ipb;
    ci.Pb = (uint32_t)g.P;
    ci.RPb = (uint32_t)g.R * ci.Pb;
    ci.Ob = (uint32_t)g.O;
    return ci;
}

// Add the codes of item `it` to cnt[256] (interior voxels inside the cube
// only); returns the item's brick of the cube (the pool holds bricks brick0 ..).
// Every thread of the block takes part.
__device__ __forceinline__ uint32_t count_codes(const uint8_t *__restrict__ pool, const BrickGeom &g,
                                                const CodeItems &ci, int64_t it, uint32_t *cnt, int64_t brick0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t pb = (uint32_t)(it >> ci.ipb);              // brick slot in the pool
    const uint32_t b = pb + (uint32_t)brick0;                  // brick of the cube
    const uint32_t c0 = ((uint32_t)it & ((1u << ci.ipb) - 1)) << ci.lcpi;
    const uint32_t bx = b % (uint32_t)g.nb[0], byz = b / (uint32_t)g.nb[0];
    const uint32_t by = byz % (uint32_t)g.nb[1], bz = byz / (uint32_t)g.nb[1];
    const bool clean = ((int64_t)(bx + 1) << g.logB) <= g.dims[0] && ((int64_t)(by + 1) << g.logB) <= g.dims[1] &&
                       ((int64_t)(bz + 1) << g.logB) <= g.dims[2];
    const uint8_t *bp = pool + (uint64_t)pb * (uint64_t)g.brick_bytes;
    for (uint32_t ch = c0 + warp; ch < c0 + (1u << ci.lcpi); ch += kStatsThreads / 32) {
        const uint32_t lr0 = ch << ci.logRPC;
        uint4 raw[kVecPerLane];
#pragma unroll
        for (int i = 0; i < kVecPerLane; ++i) {
            const uint32_t j = lane + 32 * i;
            const uint32_t lr = lr0 + (j >> ci.logVPR);
            const uint32_t off = ((lr >> g.logB) + 1) * ci.RPb + ((lr & (g.B - 1)) + 1) * ci.Pb + ci.Ob +
                                 ((j & ((1u << ci.logVPR) - 1)) << 4);
            raw[i] = __ldcs(reinterpret_cast<const uint4 *>(bp + off));
        }
#pragma unroll
        for (int i = 0; i < kVecPerLane; ++i) {
            int nvalid = 16;
            if (!clean) {
                const uint32_t j = lane + 32 * i;
                const uint32_t lr = lr0 + (j >> ci.logVPR);
                const int64_t gx0 = ((int64_t)bx << g.logB) + ((int64_t)(j & ((1u << ci.logVPR) - 1)) << 4);
                const int64_t gy = ((int64_t)by << g.logB) + (lr & (g.B - 1));
                const int64_t gz = ((int64_t)bz << g.logB) + (lr >> g.logB);
                nvalid = (int)min((int64_t)16, g.dims[0] - gx0);
                if (gy >= g.dims[1] || gz >= g.dims[2] || nvalid < 0) nvalid = 0;
            }
            const uint32_t w[4] = {raw[i].x, raw[i].y, raw[i].z, raw[i].w};
#pragma unroll
            for (int e = 0; e < 16; ++e)
                if (clean || e < nvalid) atomicAdd(&cnt[(w[e >> 2] >> (8 * (e & 3))) & 0xffu], 1u);
        }
    }
    return b;
}

// Stored value of code q of brick b (FP8): fl32(e4m3(q) * scale_b).
__device__ __forceinline__ float fp8_value(uint32_t q, float scale)
{
    const __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3);
    return __fmul_rn(__half2float(__half(hr)), scale);
}

__global__ void __launch_bounds__(kStatsThreads) k_stats_codes(StatsArgs a)
{
    static_assert(kStatsThreads == 256, "one thread per code");
    __shared__ uint32_t cnt[256];
    const BrickGeom &g = a.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const CodeItems ci = code_items(g, a.nrun);
    double s1 = 0.0, s2 = 0.0;
    unsigned long long n = 0, nnf = 0;
    for (int64_t it = blockIdx.x; it < ci.items; it += gridDim.x) {
        cnt[threadIdx.x] = 0;
        __syncthreads();
        const uint32_t b = count_codes(a.pool, g, ci, it, cnt, a.brick0);
        __syncthreads();
        const uint32_t k = cnt[threadIdx.x];
        if (k) {
            const float v = fp8_value(threadIdx.x, __ldg(a.scales + b));
            if (fabsf(v) <= FLT_MAX) {
                const double d = (double)v * (double)a.dscale;
                s1 += (double)k * d;
                s2 += (double)k * (d * d);
                n += k;
                if (a.nbins > 0) {
                    const float t = __fmul_rn(__fadd_rn(v, -a.vmin), a.hscale);
                    atomicAdd(&a.hist[max(0, min((int)t, a.nbins - 1))], (unsigned long long)k);
                }
            } else {
                nnf += k;
            }
        }
        __syncthreads();   // the next item zeroes the counters
    }
    for (int o = 16; o; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
        nnf += __shfl_xor_sync(0xffffffffu, nnf, o);
    }
    __shared__ StatPartial wp[kStatsThreads / 32];
    if (lane == 0) wp[warp] = StatPartial{s1, s2, n, nnf};
    __syncthreads();
    if (threadIdx.x == 0) {
        StatPartial r = wp[0];
        for (int w = 1; w < kStatsThreads / 32; ++w) {
            r.s1 += wp[w].s1;
            r.s2 += wp[w].s2;
            r.n += wp[w].n;
            r.nnf += wp[w].nnf;
        }
        if (a.accumulate) {
            StatPartial &p = a.partials[blockIdx.x];
            p.s1 += r.s1;
            p.s2 += r.s2;
            p.n += r.n;
            p.nnf += r.nnf;
        } else {
            a.partials[blockIdx.x] = r;
        }
    }
}

// Fixed-order merge of the block partials (deterministic for a given grid).
__global__ void k_stats_final(const StatPartial *__restrict__ p, int nparts, float vmin, float vmax, float shift,
                              float dscale, vrc_stats *out)
{
    __shared__ double s1[256], s2[256];
    __shared__ unsigned long long nn[256], nf[256];
    double a = 0, b = 0;
    unsigned long long c = 0, d = 0;
    for (int i = threadIdx.x; i < nparts; i += 256) {
        a += p[i].s1;
        b += p[i].s2;
        c += p[i].n;
        d += p[i].nnf;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    nn[threadIdx.x] = c;
    nf[threadIdx.x] = d;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
            nn[threadIdx.x] += nn[threadIdx.x + w];
            nf[threadIdx.x] += nf[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        vrc_stats r;
        r.n = nn[0];
        r.n_nonfinite = nf[0];
        r.min = vmin;
        r.max = vmax;
        if (r.n) {
            const double inv = 1.0 / (double)dscale;     // exact: power of two
            const double m1 = s1[0] / (double)r.n;
            const double var = s2[0] / (double)r.n - m1 * m1;
            r.mean = (double)shift + m1 * inv;
            r.std = sqrt(var > 0 ? var : 0.0) * inv;
        } else {
            r.mean = r.std = nan("");
        }
        *out = r;
    }
}

// ----------------------------------------------------------------- median

// Order-preserving map from float bits to uint32 (negative values reversed);
// the FP8 passes apply it to 0 for both zeros.
__device__ __forceinline__ uint32_t ord_key(float x)
{
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// One radix-selection pass over the finite stored values: keys k = sel_key(x)
// whose bits above `shift + nbits` equal `prefix` are counted by their digit
// (k >> shift) & (2^nbits - 1).  Counters live in shared memory per block and
// are added to the global histogram once per block (a global atomic per voxel
// collides heavily: noise values share their leading key bits).
struct SelArgs {
    const uint8_t *pool;
    BrickGeom g;
    const float *scales;
    const int32_t *bnonfinite;
    int all_full;
    int shift, nbits;              // digit of this pass
    int prefix_all;                // 1: no prefix condition (first pass)
    uint32_t prefix;               // required value of k >> (shift + nbits)
    unsigned long long *hist;      // device [2^nbits], zeroed by the caller
    int64_t brick0, nrun;          // the pool holds bricks brick0 .. brick0 + nrun - 1 of the cube
    uint32_t *keys;                // not null: the keys counted by this pass are also appended here
    unsigned int *nkeys;           // keys appended so far (zeroed by the caller)
    uint32_t key_cap;              // room in `keys`
    uint32_t keep_lo, keep_hi;     // bracket pass: keys whose digit lies in [keep_lo, keep_hi] are appended
    unsigned long long *counts;    // bracket pass: [0] finite values, [1] values whose digit is below keep_lo
    int64_t cstride;               // every cstride-th chunk is read (1: the whole cube; more: a sample)
};

constexpr int kSelMaxBins = 4096;
// Candidates of the float32 median kept for its last pass (4 bytes each), and
// the key slots a warp reserves at a time
constexpr uint32_t kMaxMedianCandidates = 1u << 26;
constexpr unsigned kKeyChunk = 256;
// Bracket of the float32 / bf16 median: cubes of at least kBracketMinVoxels
// voxels; a sample of every kBracketStride-th chunk (a prime, so that the
// sampled rows spread over every row position of a brick slice), used when it
// holds at least kBracketMinSample finite values
constexpr int64_t kBracketMinVoxels = int64_t(1) << 22;
constexpr int64_t kBracketStride = 61;
constexpr uint64_t kBracketMinSample = 1u << 16;

// Order-preserving key of a stored value for the radix passes: u ^ (sign ?
// 0xffffffff : 0x80000000).  -0 gets the key just below +0's and no value lies
// between them, so an order statistic that falls among the zeros is 0 either
// way (-0 and +0 are one value).
__device__ __forceinline__ uint32_t sel_key(float x)
{
    const uint32_t u = __float_as_uint(x);
    return u ^ (uint32_t)(((int32_t)u >> 31) | (int32_t)0x80000000);
}

// FIRST: the first pass (no prefix condition; digit = the key's top a.nbits bits).
template <int DT, bool FIRST>
__global__ void __launch_bounds__(kStatsThreads, kStatsCtasPerSm) k_select_hist(SelArgs a)
{
    __shared__ uint32_t sh[kSelMaxBins];
    constexpr int VE = DT == VRC_F32 ? 4 : (DT == VRC_BF16 ? 8 : 16);
    constexpr int LOG_VE = DT == VRC_F32 ? 2 : (DT == VRC_BF16 ? 3 : 4);
    const int nb = 1 << a.nbits;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const BrickGeom &g = a.g;
    const int lane = threadIdx.x & 31;
    const int logVPR = g.logB - LOG_VE;
    const int logRPC = kLogChunk - logVPR;
    const int logCPB = 2 * g.logB - logRPC;
    const int64_t total_chunks = a.nrun << logCPB;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t Pb = (uint32_t)(g.P * g.esize), RPb = (uint32_t)g.R * Pb, Ob = (uint32_t)(g.O * g.esize);
    const uint32_t dmask = (uint32_t)nb - 1u;
    const int hshift = a.shift + a.nbits;
    // byte offsets of this lane's vectors after its chunk's first row, when the
    // chunk's rows lie in one slice (as in the statistics pass)
    const bool one_slice = logRPC <= g.logB;
    uint32_t loff[kVecPerLane];
#pragma unroll
    for (int i = 0; i < kVecPerLane; ++i) {
        const uint32_t j = lane + 32 * i;
        loff[i] = (j >> logVPR) * Pb + Ob + ((j & ((1u << logVPR) - 1)) << 4);
    }
    unsigned wpos = 0, wend = 0;   // this warp's reserved key slots [wpos, wend)
    const int64_t nread = (total_chunks + a.cstride - 1) / a.cstride;
    for (int64_t ci = warp0; ci < nread; ci += nwarps) {
        const int64_t ch = ci * a.cstride;
        const uint32_t pb = (uint32_t)(ch >> logCPB);          // brick slot in the pool
        const uint32_t b = pb + (uint32_t)a.brick0;            // brick of the cube
        const uint32_t lr0 = ((uint32_t)ch & ((1u << logCPB) - 1)) << logRPC;
        bool clean;
        uint32_t bx = 0, by = 0, bz = 0;
        if (a.all_full) {
            clean = __ldg(a.bnonfinite + b) == 0;
        } else {
            bx = b % (uint32_t)g.nb[0];
            const uint32_t byz = b / (uint32_t)g.nb[0];
            by = byz % (uint32_t)g.nb[1];
            bz = byz / (uint32_t)g.nb[1];
            clean = ((int64_t)(bx + 1) << g.logB) <= g.dims[0] && ((int64_t)(by + 1) << g.logB) <= g.dims[1] &&
                    ((int64_t)(bz + 1) << g.logB) <= g.dims[2] && __ldg(a.bnonfinite + b) == 0;
        }
        const uint8_t *bp = a.pool + (uint64_t)pb * (uint64_t)g.brick_bytes;
        const float scale = DT == VRC_FP8E4M3 ? __ldg(a.scales + b) : 1.f;
        uint4 raw[kVecPerLane];
        if (one_slice) {
            const uint32_t rb = ((lr0 >> g.logB) + 1) * RPb + ((lr0 & (g.B - 1)) + 1) * Pb;
#pragma unroll
            for (int i = 0; i < kVecPerLane; ++i) raw[i] = __ldcs(reinterpret_cast<const uint4 *>(bp + rb + loff[i]));
        } else {
#pragma unroll
            for (int i = 0; i < kVecPerLane; ++i) {
                const uint32_t j = lane + 32 * i;
                const uint32_t lr = lr0 + (j >> logVPR);
                const uint32_t off = ((lr >> g.logB) + 1) * RPb + ((lr & (g.B - 1)) + 1) * Pb + Ob +
                                     ((j & ((1u << logVPR) - 1)) << 4);
                raw[i] = __ldcs(reinterpret_cast<const uint4 *>(bp + off));
            }
        }
#pragma unroll
        for (int i = 0; i < kVecPerLane; ++i) {
            float x[VE];
            decode16<DT>(raw[i], scale, x);
            int nvalid = VE;
            if (!clean) {
                if (a.all_full) {
                    bx = b % (uint32_t)g.nb[0];
                    const uint32_t byz = b / (uint32_t)g.nb[0];
                    by = byz % (uint32_t)g.nb[1];
                    bz = byz / (uint32_t)g.nb[1];
                }
                const uint32_t j = lane + 32 * i;
                const uint32_t lr = lr0 + (j >> logVPR);
                const int64_t gx0 = ((int64_t)bx << g.logB) + ((int64_t)(j & ((1u << logVPR) - 1)) << LOG_VE);
                const int64_t gy = ((int64_t)by << g.logB) + (lr & (g.B - 1)), gz = ((int64_t)bz << g.logB) + (lr >> g.logB);
                nvalid = (int)min((int64_t)VE, g.dims[0] - gx0);
                if (gy >= g.dims[1] || gz >= g.dims[2] || nvalid < 0) nvalid = 0;
            }
            uint32_t kk[VE];
            bool mm[VE], any = false;
#pragma unroll
            for (int e = 0; e < VE; ++e) {
                const bool ok = clean || (e < nvalid && fabsf(x[e]) <= FLT_MAX);
                kk[e] = sel_key(x[e]);
                mm[e] = ok && (FIRST || (kk[e] >> hshift) == a.prefix);
                if (mm[e]) atomicAdd(&sh[FIRST ? (kk[e] >> a.shift) : ((kk[e] >> a.shift) & dmask)], 1u);
                any = any || mm[e];
            }
            // the warp's matching keys appended into slots it reserved kKeyChunk at
            // a time (one global atomic per chunk: a single counter bumped per
            // match serialises in L2); matches are rare, so one vote per vector
            // skips the vectors where no lane matched (the warp is converged
            // here).  Slots a warp leaves unused keep the caller's key 0, which
            // no finite value's key has.
            if (a.keys && __any_sync(0xffffffffu, any)) {
#pragma unroll
                for (int e = 0; e < VE; ++e) {
                    const unsigned bal = __ballot_sync(0xffffffffu, mm[e]);
                    const unsigned n = (unsigned)__popc(bal);
                    if (n == 0) continue;
                    if (wpos + n > wend) {
                        unsigned base = 0;
                        if (lane == 0) base = atomicAdd(a.nkeys, kKeyChunk);
                        wpos = __shfl_sync(0xffffffffu, base, 0);
                        wend = wpos + kKeyChunk;
                    }
                    const unsigned i = wpos + (unsigned)__popc(bal & ((1u << lane) - 1u));
                    if (mm[e] && i < a.key_cap) a.keys[i] = kk[e];
                    wpos += n;
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (sh[i]) atomicAdd(&a.hist[i], (unsigned long long)sh[i]);
}

// Key of element e of a 16-byte vector of stored values (float32: 4 elements, bf16: 8).
template <int DT>
__device__ __forceinline__ uint32_t word_key(const uint4 &w, int e)
{
    const int wi = DT == VRC_F32 ? e : (e >> 1);
    const uint32_t t = wi == 0 ? w.x : (wi == 1 ? w.y : (wi == 2 ? w.z : w.w));
    const uint32_t bits = DT == VRC_F32 ? t : ((e & 1) ? (t & 0xffff0000u) : (t << 16));
    return sel_key(__uint_as_float(bits));
}

// Bracket pass of the float32 / bf16 median: one pass over the cube that
// counts the finite stored values and those whose key's leading digit
// (key >> a.shift) lies below a.keep_lo, and appends the keys whose digit lies
// in [a.keep_lo, a.keep_hi].  No histogram: the digits of the median are then
// selected among the appended keys.  A warp appends a chunk's kept keys
// together: one vote per chunk and, where a lane keeps any, one prefix scan of
// the lanes' counts and one reservation when its open slots run out; each
// lane then writes its keys (taken again from the loaded words) in element
// order.
template <int DT>
__global__ void __launch_bounds__(kStatsThreads, kStatsCtasPerSm) k_select_bracket(SelArgs a)
{
    constexpr int VE = DT == VRC_F32 ? 4 : 8;
    constexpr int LOG_VE = DT == VRC_F32 ? 2 : 3;
    static_assert(DT != VRC_FP8E4M3, "FP8 medians come from code counts");
    static_assert(kVecPerLane * VE <= 64, "one 64-bit mask per chunk and lane");
    const BrickGeom &g = a.g;
    const int lane = threadIdx.x & 31;
    const int logVPR = g.logB - LOG_VE;
    const int logRPC = kLogChunk - logVPR;
    const int logCPB = 2 * g.logB - logRPC;
    const int64_t total_chunks = a.nrun << logCPB;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t Pb = (uint32_t)(g.P * g.esize), RPb = (uint32_t)g.R * Pb, Ob = (uint32_t)(g.O * g.esize);
    const bool one_slice = logRPC <= g.logB;
    uint32_t loff[kVecPerLane];
#pragma unroll
    for (int i = 0; i < kVecPerLane; ++i) {
        const uint32_t j = lane + 32 * i;
        loff[i] = (j >> logVPR) * Pb + Ob + ((j & ((1u << logVPR) - 1)) << 4);
    }
    const uint32_t lo = a.keep_lo, span = a.keep_hi - a.keep_lo;
    uint32_t nfin = 0, nbelow = 0;
    unsigned wpos = 0, wend = 0;   // this warp's reserved key slots [wpos, wend)
    for (int64_t ch = warp0; ch < total_chunks; ch += nwarps) {
        const uint32_t pb = (uint32_t)(ch >> logCPB);
        const uint32_t b = pb + (uint32_t)a.brick0;
        const uint32_t lr0 = ((uint32_t)ch & ((1u << logCPB) - 1)) << logRPC;
        bool clean;
        uint32_t bx = 0, by = 0, bz = 0;
        if (a.all_full) {
            clean = __ldg(a.bnonfinite + b) == 0;
        } else {
            bx = b % (uint32_t)g.nb[0];
            const uint32_t byz = b / (uint32_t)g.nb[0];
            by = byz % (uint32_t)g.nb[1];
            bz = byz / (uint32_t)g.nb[1];
            clean = ((int64_t)(bx + 1) << g.logB) <= g.dims[0] && ((int64_t)(by + 1) << g.logB) <= g.dims[1] &&
                    ((int64_t)(bz + 1) << g.logB) <= g.dims[2] && __ldg(a.bnonfinite + b) == 0;
        }
        const uint8_t *bp = a.pool + (uint64_t)pb * (uint64_t)g.brick_bytes;
        uint4 raw[kVecPerLane];
        if (one_slice) {
            const uint32_t rb = ((lr0 >> g.logB) + 1) * RPb + ((lr0 & (g.B - 1)) + 1) * Pb;
#pragma unroll
            for (int i = 0; i < kVecPerLane; ++i) raw[i] = __ldcs(reinterpret_cast<const uint4 *>(bp + rb + loff[i]));
        } else {
#pragma unroll
            for (int i = 0; i < kVecPerLane; ++i) {
                const uint32_t j = lane + 32 * i;
                const uint32_t lr = lr0 + (j >> logVPR);
                const uint32_t off = ((lr >> g.logB) + 1) * RPb + ((lr & (g.B - 1)) + 1) * Pb + Ob +
                                     ((j & ((1u << logVPR) - 1)) << 4);
                raw[i] = __ldcs(reinterpret_cast<const uint4 *>(bp + off));
            }
        }
        uint64_t km = 0;   // kept elements of this lane's chunk share, bit i VE + e
        if (clean) {
            nfin += kVecPerLane * VE;
#pragma unroll
            for (int i = 0; i < kVecPerLane; ++i) {
#pragma unroll
                for (int e = 0; e < VE; ++e) {
                    const uint32_t dg = word_key<DT>(raw[i], e) >> a.shift;
                    nbelow += dg < lo ? 1u : 0u;
                    km |= (uint64_t)(dg - lo <= span ? 1u : 0u) << (i * VE + e);
                }
            }
        } else {
            if (a.all_full) {
                bx = b % (uint32_t)g.nb[0];
                const uint32_t byz = b / (uint32_t)g.nb[0];
                by = byz % (uint32_t)g.nb[1];
                bz = byz / (uint32_t)g.nb[1];
            }
#pragma unroll
            for (int i = 0; i < kVecPerLane; ++i) {
                float x[VE];
                decode16<DT>(raw[i], 1.f, x);
                const uint32_t j = lane + 32 * i;
                const uint32_t lr = lr0 + (j >> logVPR);
                const int64_t gx0 = ((int64_t)bx << g.logB) + ((int64_t)(j & ((1u << logVPR) - 1)) << LOG_VE);
                const int64_t gy = ((int64_t)by << g.logB) + (lr & (g.B - 1)), gz = ((int64_t)bz << g.logB) + (lr >> g.logB);
                int nvalid = (int)min((int64_t)VE, g.dims[0] - gx0);
                if (gy >= g.dims[1] || gz >= g.dims[2] || nvalid < 0) nvalid = 0;
#pragma unroll
                for (int e = 0; e < VE; ++e) {
                    const bool ok = e < nvalid && fabsf(x[e]) <= FLT_MAX;
                    const uint32_t dg = sel_key(x[e]) >> a.shift;
                    nfin += ok ? 1u : 0u;
                    nbelow += (ok && dg < lo) ? 1u : 0u;
                    km |= (uint64_t)(ok && dg - lo <= span ? 1u : 0u) << (i * VE + e);
                }
            }
        }
        if (__any_sync(0xffffffffu, km != 0)) {   // converged: the chunk loop is warp-uniform
            const unsigned cnt = (unsigned)__popcll(km);
            unsigned incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned tot = __shfl_sync(0xffffffffu, incl, 31);
            if (wpos + tot > wend) {
                const unsigned need = (tot + kKeyChunk - 1) / kKeyChunk * kKeyChunk;
                unsigned base = 0;
                if (lane == 0) base = atomicAdd(a.nkeys, need);
                wpos = __shfl_sync(0xffffffffu, base, 0);
                wend = wpos + need;
            }
            unsigned pos = wpos + incl - cnt;
#pragma unroll
            for (int i = 0; i < kVecPerLane; ++i) {
                uint32_t m = (uint32_t)(km >> (i * VE)) & ((1u << VE) - 1u);
                while (m) {
                    const int e = __ffs(m) - 1;
                    m &= m - 1;
                    if (pos < a.key_cap) a.keys[pos] = word_key<DT>(raw[i], e);
                    ++pos;
                }
            }
            wpos += tot;
        }
    }
    for (int o = 16; o; o >>= 1) {
        nfin += __shfl_xor_sync(0xffffffffu, nfin, o);
        nbelow += __shfl_xor_sync(0xffffffffu, nbelow, o);
    }
    if (lane == 0) {
        if (nfin) atomicAdd(a.counts, (unsigned long long)nfin);
        if (nbelow) atomicAdd(a.counts + 1, (unsigned long long)nbelow);
    }
}

// Radix-selection pass over keys appended by an earlier pass (the candidates
// that share the selected leading digit, or the bracket's keys): the digit
// histogram of those whose bits above `shift + nbits` equal `prefix` (every
// key when prefix_all).  Slots left unused hold key 0, which no finite value
// has; they are skipped.
__global__ void __launch_bounds__(kStatsThreads) k_select_keys(const uint32_t *__restrict__ keys, uint32_t n, SelArgs a)
{
    __shared__ uint32_t sh[kSelMaxBins];
    const int nb = 1 << a.nbits;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint32_t dmask = (uint32_t)nb - 1u;
    const int hshift = a.shift + a.nbits;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        const bool in = a.prefix_all || (hshift < 32 && (k >> (hshift & 31)) == a.prefix);
        if (k != 0 && in) atomicAdd(&sh[(k >> a.shift) & dmask], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (sh[i]) atomicAdd(&a.hist[i], (unsigned long long)sh[i]);
}

// FP8 median, step 1: table[b * 256 + q] = number of interior voxels of brick
// b stored with code q (zeroed by the caller).
__global__ void __launch_bounds__(kStatsThreads) k_code_table(const uint8_t *__restrict__ pool, BrickGeom g,
                                                             uint32_t *__restrict__ table, int64_t brick0,
                                                             int64_t nrun)
{
    __shared__ uint32_t cnt[256];
    const CodeItems ci = code_items(g, nrun);
    for (int64_t it = blockIdx.x; it < ci.items; it += gridDim.x) {
        cnt[threadIdx.x] = 0;
        __syncthreads();
        const uint32_t b = count_codes(pool, g, ci, it, cnt, brick0);
        __syncthreads();
        if (cnt[threadIdx.x]) atomicAdd(&table[(int64_t)b * 256 + threadIdx.x], cnt[threadIdx.x]);
        __syncthreads();
    }
}

// FP8 median, step 2 (one per radix digit): the radix-selection pass of
// k_select_hist over the (brick, code) entries of the table, each counted
// with its number of voxels instead of voxel by voxel.
__global__ void k_select_codes(const uint32_t *__restrict__ table, const float *__restrict__ scales,
                               int64_t nentries, SelArgs a)
{
    const uint32_t dmask = (1u << a.nbits) - 1u;
    const int hshift = a.shift + a.nbits;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nentries; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = table[e];
        if (!w) continue;
        const float v = fp8_value((uint32_t)(e & 255), __ldg(scales + (e >> 8)));
        if (!(fabsf(v) <= FLT_MAX)) continue;
        const uint32_t k = ord_key(v == 0.f ? 0.f : v);   // -0 and +0 are one value
        if (a.prefix_all || (k >> hshift) == a.prefix) atomicAdd(&a.hist[(k >> a.shift) & dmask], (unsigned long long)w);
    }
}

int stats_grid(vrc_ctx *ctx) { return ctx->sm_count * 4; }

// Persistent grid: as many blocks as fit on the SMs (at most grid_cap).
template <int DT>
int launch_stats(const StatsArgs &a, int sm_count, int grid_cap, size_t smem, int hist, cudaStream_t st)
{
    int occ = 1;
    if (hist == 1) {
        cudaFuncSetAttribute(k_stats<DT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_stats<DT, 1>, kStatsThreads, smem);
    } else if (hist == 2) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_stats<DT, 2>, kStatsThreads, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_stats<DT, 0>, kStatsThreads, 0);
    }
    const int grid = std::max(1, std::min(grid_cap, sm_count * std::max(occ, 1)));
    if (hist == 1) {
        cudaFuncSetAttribute(k_stats<DT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_stats<DT, 1><<<grid, kStatsThreads, smem, st>>>(a);
    } else if (hist == 2) {
        k_stats<DT, 2><<<grid, kStatsThreads, 0, st>>>(a);
    } else {
        k_stats<DT, 0><<<grid, kStatsThreads, 0, st>>>(a);
    }
    return grid;
}

}  // namespace

size_t stats_scratch_bytes(vrc_ctx *ctx) { return sizeof(StatPartial) * (size_t)stats_grid(ctx); }

namespace {

// Pass arguments shared by resident and out-of-core cubes.
StatsArgs make_stats_args(const Cube *c, int32_t nbins, uint64_t *dev_hist, void *partials, const uint8_t *pool)
{
    const BrickGeom &g = c->g;
    StatsArgs a;
    a.pool = pool;
    a.g = g;
    a.scales = c->scales;
    a.vmin = c->vmin;
    a.bnonfinite = c->bnonfinite;
    // c: the upload-time mean rounded to 8 significant bits (x - c is then exact
    // for every voxel not far below |c|); s: power of two keeping d^2 finite;
    // kq: power of two bounding every d^2, seed of the Fast2Sum accumulator
    {
        int e = 0;
        const double m = std::frexp((double)c->shift, &e);
        a.shift = (float)std::ldexp(std::nearbyint(std::ldexp(m, 8)), e - 8);
        if (!(a.shift >= c->vmin && a.shift <= c->vmax)) a.shift = c->vmin;
        // FP8 values repeat (256 codes per brick): take c = 0 so that d = x is exact
        if (g.dtype == VRC_FP8E4M3) a.shift = 0.f;
        const double maxd = std::fmax(std::fabs((double)c->vmax - a.shift), std::fabs((double)a.shift - c->vmin));
        int k = 0;
        while (std::ldexp(maxd, -k) > 0x1p60) ++k;
        a.dscale = (float)std::ldexp(1.0, -k);
        const double md = std::ldexp(maxd, -k) * (1.0 + 0x1p-20);
        double kq = 1.0;
        while (kq < md * md) kq *= 2.0;
        a.kq = (float)kq;
    }
    // histogram scale in binary32: range = fl(max - min), scale = fl(nbins / range)
    volatile float range = c->vmax - c->vmin;
    a.hscale = (nbins > 0 && range > 0.f) ? (float)nbins / (float)range : 0.f;
    a.nbins = nbins;
    a.all_full = g.dims[0] % g.B == 0 && g.dims[1] % g.B == 0 && g.dims[2] % g.B == 0;
    a.hist = (unsigned long long *)dev_hist;
    a.partials = (StatPartial *)partials;
    a.accumulate = 0;
    a.brick0 = 0;
    a.nrun = g.nbricks;
    return a;
}

int launch_stats_dt(vrc_ctx *ctx, const StatsArgs &a, int grid, int nbins, cudaStream_t st)
{
    const int hist = nbins == 0 ? 0 : (nbins <= kSmemBinsMax ? 1 : 2);
    const size_t smem = hist == 1 ? sizeof(uint32_t) * (nbins + 1) : 0;
    if (a.g.dtype == VRC_F32) return launch_stats<VRC_F32>(a, ctx->sm_count, grid, smem, hist, st);
    if (a.g.dtype == VRC_BF16) return launch_stats<VRC_BF16>(a, ctx->sm_count, grid, smem, hist, st);
    k_stats_codes<<<grid, kStatsThreads, 0, st>>>(a);
    return grid;
}

// Out-of-core cubes: run `pass(pool, brick0, nrun)` over the cube in runs of
// consecutive bricks copied through the two halves of the device ring; run r
// loads while run r - 1 is processed (copies on a side stream, Sec. 2: streams
// overlap I/O).  Bricks not in the host cache are provided on this thread.
template <class Pass>
vrc_status for_ring_runs(vrc_ctx *ctx, Cube *c, cudaStream_t st, Pass pass)
{
    const int half = c->ring / 2;
    const int64_t nb = c->g.nbricks;
    cudaStream_t cs;
    VRC_CK(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t ev[5] = {};
    vrc_status s = VRC_OK;
    for (int i = 0; i < 5 && s == VRC_OK; ++i) {
        const cudaError_t e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) s = cuda_err(ctx, e, "ring events");
    }
    cudaEvent_t *ready = ev, *consumed = ev + 2, entry = ev[4];
    if (s == VRC_OK) {
        cudaEventRecord(entry, st);   // earlier work on `st` may still read the ring
        cudaStreamWaitEvent(cs, entry, 0);
    }
    for (int64_t r = 0, b0 = 0; s == VRC_OK && b0 < nb; ++r, b0 += half) {
        const int h = (int)(r & 1);
        const int64_t n = std::min<int64_t>(half, nb - b0);
        if (r >= 2) cudaStreamWaitEvent(cs, consumed[h], 0);   // run r - 2 has left this half
        if ((s = ring_load(ctx, c, b0, n, h * half, cs, ready[h])) != VRC_OK) break;
        cudaStreamWaitEvent(st, ready[h], 0);
        if ((s = pass((const uint8_t *)c->ring_pool + (int64_t)h * half * c->g.brick_bytes, b0, n)) != VRC_OK) break;
        cudaEventRecord(consumed[h], st);
    }
    // the side stream's copies are joined into `st` before anything is released
    cudaEventRecord(entry, cs);
    cudaStreamWaitEvent(st, entry, 0);
    for (int i = 0; i < 5; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    cudaStreamDestroy(cs);
    return s;
}

}  // namespace

// Launch the fused statistics pass + final merge on `st`.  dev_hist (nbins
// counters) is zeroed here; partials is scratch of stats_scratch_bytes().
vrc_status stats_launch_with(vrc_ctx *ctx, Cube *c, int32_t nbins, vrc_stats *dev_out, uint64_t *dev_hist,
                             void *partials, cudaStream_t st)
{
    const int grid = stats_grid(ctx);
    StatsArgs a = make_stats_args(c, nbins, dev_hist, partials, (const uint8_t *)c->pool);
    if (nbins > 0) VRC_CK(ctx, cudaMemsetAsync(dev_hist, 0, sizeof(uint64_t) * nbins, st));
    int used = grid;
    if (!c->streamed) {
        used = launch_stats_dt(ctx, a, grid, nbins, st);
        count_launch(ctx);
    } else {
        // per-brick non-finite counts steer the pass; every run adds into one
        // partial per block (fixed order: block, then run)
        vrc_status s = stage_h2d(ctx, st, {{c->bnonfinite, c->h_bnonfinite.data(), sizeof(int32_t) * (size_t)c->g.nbricks}});
        if (s != VRC_OK) return s;
        VRC_CK(ctx, cudaMemsetAsync(partials, 0, stats_scratch_bytes(ctx), st));
        a.accumulate = 1;
        s = for_ring_runs(ctx, c, st, [&](const uint8_t *pool, int64_t b0, int64_t n) {
            StatsArgs r = a;
            r.pool = pool;
            r.brick0 = b0;
            r.nrun = n;
            // the same grid for every run: partial i always belongs to block i
            launch_stats_dt(ctx, r, grid, nbins, st);
            count_launch(ctx);
            const cudaError_t e = cudaGetLastError();
            return e == cudaSuccess ? VRC_OK : cuda_err(ctx, e, "statistics run");
        });
        if (s != VRC_OK) return s;
        used = grid;
    }
    k_stats_final<<<1, 256, 0, st>>>(a.partials, used, c->vmin, c->vmax, a.shift, a.dscale, dev_out);
    count_launch(ctx);
    VRC_CK(ctx, cudaGetLastError());
    return VRC_OK;
}

static vrc_status check_stats_args(vrc_ctx *ctx, int64_t cube_id, int32_t nbins, Cube **out, CubeUse &use,
                                   void *stream)
{
    if (!ctx) return VRC_E_INVAL;
    if (nbins < 0 || nbins > 65536) return set_err(ctx, VRC_E_INVAL, "nbins must be in [0, 65536]");
    Cube *c = nullptr;
    vrc_status s = acquire_cube(ctx, cube_id, (cudaStream_t)stream, &c, use);
    if (s != VRC_OK) return s;
    if (c->streamed && c->n_filled < c->n_host)
        return set_err(ctx, VRC_E_INVAL, "streamed cube: %lld of %lld host slots never written",
                       (long long)(c->n_host - c->n_filled), (long long)c->n_host);
    *out = c;
    return VRC_OK;
}

extern "C" {

vrc_status vrc_cube_stats_async(vrc_ctx *ctx, int64_t cube_id, int32_t nbins, vrc_stats *dev_out,
                                uint64_t *dev_hist, void *stream)
{
    Cube *c = nullptr;
    CubeUse use;
    vrc_status s = check_stats_args(ctx, cube_id, nbins, &c, use, stream);
    if (s != VRC_OK) return s;
    if (!dev_out || (nbins > 0 && !dev_hist)) return set_err(ctx, VRC_E_INVAL, "null output");
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    void *scr = nullptr;
    if ((s = scratch_get(ctx, stats_scratch_bytes(ctx), &scr)) != VRC_OK) return s;
    return stats_launch_with(ctx, c, nbins, dev_out, dev_hist, scr, (cudaStream_t)stream);
}

vrc_status vrc_cube_stats(vrc_ctx *ctx, int64_t cube_id, int32_t nbins, vrc_stats *out, uint64_t *hist,
                          void *stream)
{
    Cube *c = nullptr;
    CubeUse use;
    vrc_status s = check_stats_args(ctx, cube_id, nbins, &c, use, stream);
    if (s != VRC_OK) return s;
    if (!out || (nbins > 0 && !hist)) return set_err(ctx, VRC_E_INVAL, "null output");
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t pbytes = (stats_scratch_bytes(ctx) + 255) & ~(size_t)255;
    const size_t need = pbytes + 256 + sizeof(uint64_t) * (size_t)nbins;
    void *scr = nullptr;
    if ((s = scratch_get(ctx, need, &scr)) != VRC_OK) return s;
    vrc_stats *dout = (vrc_stats *)((char *)scr + pbytes);
    uint64_t *dhist = (uint64_t *)((char *)scr + pbytes + 256);
    if ((s = stats_launch_with(ctx, c, nbins, dout, dhist, scr, st)) != VRC_OK) return s;
    VRC_CK(ctx, cudaMemcpyAsync(out, dout, sizeof(vrc_stats), cudaMemcpyDeviceToHost, st));
    if (nbins > 0) VRC_CK(ctx, cudaMemcpyAsync(hist, dhist, sizeof(uint64_t) * nbins, cudaMemcpyDeviceToHost, st));
    VRC_CK(ctx, cudaStreamSynchronize(st));
    if (out->n == 0) return set_err(ctx, VRC_E_NONFINITE, "cube has no finite voxel");
    return VRC_OK;
}

vrc_status vrc_cube_median(vrc_ctx *ctx, int64_t cube_id, double *out, void *stream)
{
    Cube *c = nullptr;
    CubeUse use;
    vrc_status s = check_stats_args(ctx, cube_id, 0, &c, use, stream);
    if (s != VRC_OK) return s;
    if (!out) return VRC_E_INVAL;
    VRC_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    // FP8: one pass counts each brick's codes; the radix passes then run over
    // the (brick, code) entries with their counts
    const bool codes = c->g.dtype == VRC_FP8E4M3;
    const int64_t nentries = codes ? c->g.nbricks * 256 : 0;
    void *scr = nullptr;
    if ((s = scratch_get(ctx, kSelMaxBins * sizeof(unsigned long long) + nentries * sizeof(uint32_t), &scr)) != VRC_OK)
        return s;
    unsigned long long *dh = (unsigned long long *)scr;
    uint32_t *table = reinterpret_cast<uint32_t *>(dh + kSelMaxBins);
    if (codes) {
        VRC_CK(ctx, cudaMemsetAsync(table, 0, nentries * sizeof(uint32_t), st));
        if (c->streamed) {
            // out-of-core: the counts are taken run by run through the ring
            const vrc_status sr = for_ring_runs(ctx, c, st, [&](const uint8_t *pool, int64_t b0, int64_t n) {
                k_code_table<<<stats_grid(ctx), kStatsThreads, 0, st>>>(pool, c->g, table, b0, n);
                count_launch(ctx);
                const cudaError_t e = cudaGetLastError();
                return e == cudaSuccess ? VRC_OK : cuda_err(ctx, e, "code table run");
            });
            if (sr != VRC_OK) return sr;
        } else {
            k_code_table<<<stats_grid(ctx), kStatsThreads, 0, st>>>((const uint8_t *)c->pool, c->g, table, 0,
                                                                    c->g.nbricks);
            count_launch(ctx);
        }
        VRC_CK(ctx, cudaGetLastError());
    }
    std::vector<unsigned long long> h(kSelMaxBins);
    SelArgs a;
    a.pool = (const uint8_t *)c->pool;
    a.g = c->g;
    a.scales = c->scales;
    a.bnonfinite = c->bnonfinite;
    a.all_full = c->g.dims[0] % c->g.B == 0 && c->g.dims[1] % c->g.B == 0 && c->g.dims[2] % c->g.B == 0;
    a.hist = dh;
    a.brick0 = 0;
    a.nrun = c->g.nbricks;
    a.keys = nullptr;
    a.nkeys = nullptr;
    a.key_cap = 0;
    a.keep_lo = a.keep_hi = 0;
    a.counts = nullptr;
    a.cstride = 1;
    if (c->streamed &&
        (s = stage_h2d(ctx, st, {{c->bnonfinite, c->h_bnonfinite.data(), sizeof(int32_t) * (size_t)c->g.nbricks}})) !=
            VRC_OK)
        return s;
    int occ = 1;
    if (c->g.dtype == VRC_F32) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_select_hist<VRC_F32, true>, kStatsThreads, 0);
    else if (c->g.dtype == VRC_BF16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_select_hist<VRC_BF16, true>, kStatsThreads, 0);
    const int grid = ctx->sm_count * std::max(occ, 1);
    // three digits of the 32-bit ordered key: 12, 10 and 10 bits
    const int shifts[3] = {20, 10, 0}, widths[3] = {12, 10, 10};
    uint64_t rank = 0;
    uint32_t key = 0;
    // bf16 keys carry 16 significant bits (the value's low 16 bits are 0, so the
    // key's are 0 for positive values and 1 for negative ones): two passes fix
    // bits 31..10 and with them the value
    const int npass = c->g.dtype == VRC_BF16 ? 2 : 3;
    // float32: the second pass also appends the keys of its candidates (those
    // in the first digit's selected bin, whose number the first pass gave), so
    // the third pass reads them instead of the cube (when at most
    // kMaxMedianCandidates and their buffer fits the budget; else it reads the
    // cube again)
    uint32_t ncand = 0;
    unsigned int hk = 0;
    uint64_t prev_count = 0;   // keys in the digit bin the previous pass selected
    struct CandBuf {   // device buffer of the candidates' keys; released once `st` has finished with it
        vrc_ctx *ctx;
        cudaStream_t st;
        void *p = nullptr;
        size_t n = 0;
        ~CandBuf()
        {
            if (!p) return;
            cudaStreamSynchronize(st);
            dev_free(ctx, p, n);
        }
    } cand{ctx, st};
    // Bracket (resident float32 / bf16 cubes of at least kBracketMinVoxels
    // voxels): one pass over the cube instead of two.
    //  1. A first-digit pass over every kBracketStride-th chunk (1/61 of the
    //     rows, spread over every brick and row position) gives the sample's
    //     histogram of the leading 12-bit digit; the bins holding the sample's
    //     ranks (0.5 -+ delta)(ns - 1), delta ten times the rank error of ns
    //     independent draws, bound the bins of the median.
    //  2. The bracket pass counts the finite values and those below the first
    //     bounded bin, and appends the keys of the bounded bins.
    //  3. When the median's rank falls among the appended keys (and all of them
    //     were kept), its three digits (bf16: two) are selected among those keys.
    // Otherwise the passes below read the cube, as without the bracket.
    // Measured on the 1024^3 bench cube: the sample's rank error is 0.3 of that
    // unit at stride 61 (28 units at stride 64, whose chunks fall on the same
    // four rows of every brick slice).
    if (!codes && !c->streamed && c->g.dims[0] * c->g.dims[1] * c->g.dims[2] >= kBracketMinVoxels) {
        SelArgs r = a;
        r.shift = shifts[0];
        r.nbits = widths[0];
        r.prefix_all = 1;
        r.prefix = 0;
        r.cstride = kBracketStride;
        const int nb0 = 1 << r.nbits;
        VRC_CK(ctx, cudaMemsetAsync(dh, 0, nb0 * sizeof(unsigned long long), st));
        if (c->g.dtype == VRC_F32) k_select_hist<VRC_F32, true><<<grid, kStatsThreads, 0, st>>>(r);
        else k_select_hist<VRC_BF16, true><<<grid, kStatsThreads, 0, st>>>(r);
        count_launch(ctx);
        VRC_CK(ctx, cudaGetLastError());
        VRC_CK(ctx, cudaMemcpyAsync(h.data(), dh, nb0 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        VRC_CK(ctx, cudaStreamSynchronize(st));
        uint64_t ns = 0;
        for (int i = 0; i < nb0; ++i) ns += h[i];
        int blo = -1, bhi = -1;
        uint64_t in = 0;
        if (ns >= kBracketMinSample) {
            const double delta = 10.0 * 0.5 / std::sqrt((double)ns) + 64.0 / (double)ns;
            const uint64_t rlo = (uint64_t)std::floor(std::max(0.0, 0.5 - delta) * (double)(ns - 1));
            const uint64_t rhi =
                std::min<uint64_t>(ns - 1, (uint64_t)std::ceil(std::min(1.0, 0.5 + delta) * (double)(ns - 1)));
            uint64_t acc = 0;
            for (int i = 0; i < nb0; ++i) {
                if (blo < 0 && acc + h[i] > rlo) blo = i;
                if (blo >= 0) in += h[i];
                if (acc + h[i] > rhi) {
                    bhi = i;
                    break;
                }
                acc += h[i];
            }
        }
        // keys expected in the bounded bins, with room for a sampling error of
        // 1/4, the chunk tails the warps leave and one open chunk per warp
        const double est = ns ? (double)in / (double)ns * (double)(c->g.dims[0] * c->g.dims[1] * c->g.dims[2]) : 0.0;
        const uint64_t warps = (uint64_t)grid * (kStatsThreads / 32);
        const double capd = est * 1.25 * 1.125 + (double)kKeyChunk * (double)(warps + 1);
        if (blo >= 0 && bhi >= blo && capd <= (double)kMaxMedianCandidates) {
            const uint64_t cap = (uint64_t)capd;
            cand.n = 32 + (size_t)cap * sizeof(uint32_t);
            if (dev_alloc(ctx, &cand.p, cand.n) != VRC_OK) {
                cand.p = nullptr;   // no room: the passes below read the cube
            } else {
                SelArgs q = a;
                q.shift = shifts[0];
                q.nbits = widths[0];
                q.nkeys = reinterpret_cast<unsigned int *>(cand.p);
                q.counts = reinterpret_cast<unsigned long long *>((char *)cand.p + 16);
                q.keys = reinterpret_cast<uint32_t *>((char *)cand.p + 32);
                q.key_cap = (uint32_t)cap;
                q.keep_lo = (uint32_t)blo;
                q.keep_hi = (uint32_t)bhi;
                VRC_CK(ctx, cudaMemsetAsync(cand.p, 0, cand.n, st));   // counters 0, every slot key 0
                if (c->g.dtype == VRC_F32) k_select_bracket<VRC_F32><<<grid, kStatsThreads, 0, st>>>(q);
                else k_select_bracket<VRC_BF16><<<grid, kStatsThreads, 0, st>>>(q);
                count_launch(ctx);
                VRC_CK(ctx, cudaGetLastError());
                unsigned long long cnt[2] = {0, 0};
                VRC_CK(ctx, cudaMemcpyAsync(cnt, q.counts, sizeof cnt, cudaMemcpyDeviceToHost, st));
                VRC_CK(ctx, cudaMemcpyAsync(&hk, q.nkeys, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
                VRC_CK(ctx, cudaStreamSynchronize(st));
                if (cnt[0] == 0) return set_err(ctx, VRC_E_NONFINITE, "cube has no finite voxel");
                const uint64_t rk = (cnt[0] - 1) / 2;   // lower median
                bool held = hk <= q.key_cap && cnt[1] <= rk;
                uint64_t r1 = rk - (held ? cnt[1] : 0);
                uint32_t bkey = 0;
                for (int d = 0; held && d < npass; ++d) {
                    SelArgs r2 = a;
                    r2.shift = shifts[d];
                    r2.nbits = widths[d];
                    r2.prefix_all = d == 0;
                    r2.prefix = d == 0 ? 0u : bkey >> (r2.shift + r2.nbits);
                    const int nbd = 1 << r2.nbits;
                    VRC_CK(ctx, cudaMemsetAsync(dh, 0, nbd * sizeof(unsigned long long), st));
                    k_select_keys<<<(unsigned)std::min<int64_t>((hk + 255) / 256, grid), kStatsThreads, 0, st>>>(
                        q.keys, hk, r2);
                    count_launch(ctx);
                    VRC_CK(ctx, cudaGetLastError());
                    VRC_CK(ctx, cudaMemcpyAsync(h.data(), dh, nbd * sizeof(unsigned long long),
                                                cudaMemcpyDeviceToHost, st));
                    VRC_CK(ctx, cudaStreamSynchronize(st));
                    uint64_t acc = 0;
                    int sel = -1;
                    for (int i = 0; i < nbd; ++i) {
                        if (acc + h[i] > r1) {
                            sel = i;
                            break;
                        }
                        acc += h[i];
                    }
                    // the first digit's bin must be a bounded one: every key of it was kept
                    if (sel < 0 || (d == 0 && ((uint32_t)sel < q.keep_lo || (uint32_t)sel > q.keep_hi))) {
                        held = false;
                        break;
                    }
                    r1 -= acc;
                    bkey |= (uint32_t)sel << r2.shift;
                }
                if (held) {
                    if (npass == 2) bkey |= (bkey & 0x80000000u) ? 0u : 0x3ffu;
                    const uint32_t u = (bkey & 0x80000000u) ? (bkey & 0x7fffffffu) : ~bkey;
                    float f;
                    memcpy(&f, &u, 4);
                    *out = f;
                    return VRC_OK;
                }
                // the median lies outside the bounded bins: the passes below read the cube
                cudaStreamSynchronize(st);
                dev_free(ctx, cand.p, cand.n);
                cand.p = nullptr;
                hk = 0;
            }
        }
    }
    for (int pass = 0; pass < npass; ++pass) {
        a.shift = shifts[pass];
        a.nbits = widths[pass];
        a.prefix_all = pass == 0;
        a.prefix = pass == 0 ? 0u : key >> (a.shift + a.nbits);
        const int nb = 1 << a.nbits;
        const bool from_keys = pass == 2 && a.keys != nullptr;
        if (pass == 1 && npass == 3 && !codes && ncand > 0 && ncand <= kMaxMedianCandidates) {
            // room for the candidates, the chunk tails the warps leave (under 1/8)
            // and one open chunk per warp and launch
            const uint64_t warps = (uint64_t)grid * (kStatsThreads / 32);
            const uint64_t cap = (uint64_t)ncand + ncand / 8 + (uint64_t)kKeyChunk * (warps + 1);
            cand.n = 16 + (size_t)cap * sizeof(uint32_t);
            if (dev_alloc(ctx, &cand.p, cand.n) == VRC_OK) {
                a.nkeys = reinterpret_cast<unsigned int *>(cand.p);
                a.keys = reinterpret_cast<uint32_t *>((char *)cand.p + 16);
                a.key_cap = (uint32_t)cap;
                VRC_CK(ctx, cudaMemsetAsync(cand.p, 0, cand.n, st));   // count 0, every slot key 0
            } else {
                cand.p = nullptr;   // no room: the third pass reads the cube again
            }
        }
        VRC_CK(ctx, cudaMemsetAsync(dh, 0, nb * sizeof(unsigned long long), st));
        if (from_keys) {
            SelArgs r = a;
            r.keys = nullptr;
            k_select_keys<<<(unsigned)std::min<int64_t>((hk + 255) / 256, grid), kStatsThreads, 0, st>>>(a.keys, hk,
                                                                                                       r);
            count_launch(ctx);
        } else if (codes) {
            k_select_codes<<<(unsigned)std::min<int64_t>((nentries + 255) / 256, grid), 256, 0, st>>>(
                table, c->scales, nentries, a);
            count_launch(ctx);
        } else if (c->streamed) {
            // out-of-core: the pass runs over the cube run by run through the ring
            s = for_ring_runs(ctx, c, st, [&](const uint8_t *pool, int64_t b0, int64_t n) {
                SelArgs r = a;
                r.pool = pool;
                r.brick0 = b0;
                r.nrun = n;
                if (c->g.dtype == VRC_F32) {
                    if (pass == 0) k_select_hist<VRC_F32, true><<<grid, kStatsThreads, 0, st>>>(r);
                    else k_select_hist<VRC_F32, false><<<grid, kStatsThreads, 0, st>>>(r);
                } else {
                    if (pass == 0) k_select_hist<VRC_BF16, true><<<grid, kStatsThreads, 0, st>>>(r);
                    else k_select_hist<VRC_BF16, false><<<grid, kStatsThreads, 0, st>>>(r);
                }
                count_launch(ctx);
                const cudaError_t e = cudaGetLastError();
                return e == cudaSuccess ? VRC_OK : cuda_err(ctx, e, "median run");
            });
            if (s != VRC_OK) return s;
        } else {
            if (c->g.dtype == VRC_F32) {
                if (pass == 0) k_select_hist<VRC_F32, true><<<grid, kStatsThreads, 0, st>>>(a);
                else k_select_hist<VRC_F32, false><<<grid, kStatsThreads, 0, st>>>(a);
            } else {
                if (pass == 0) k_select_hist<VRC_BF16, true><<<grid, kStatsThreads, 0, st>>>(a);
                else k_select_hist<VRC_BF16, false><<<grid, kStatsThreads, 0, st>>>(a);
            }
            count_launch(ctx);
        }
        VRC_CK(ctx, cudaGetLastError());
        VRC_CK(ctx, cudaMemcpyAsync(h.data(), dh, nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        if (pass == 1 && a.keys)
            VRC_CK(ctx, cudaMemcpyAsync(&hk, a.nkeys, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        VRC_CK(ctx, cudaStreamSynchronize(st));
        if (pass == 1 && a.keys && hk > a.key_cap) {
            // more slots reserved than the buffer holds: the third pass reads the cube
            a.keys = nullptr;
            a.nkeys = nullptr;
            a.key_cap = 0;
        }
        if (from_keys) {
            uint64_t got = 0;
            for (int i = 0; i < nb; ++i) got += h[i];
            if (got != prev_count) {
                // the kept keys do not hold every key of the selected bin: this pass
                // again, over the cube
                a.keys = nullptr;
                --pass;
                continue;
            }
        }
        if (pass == 0) {
            uint64_t total = 0;
            for (int i = 0; i < nb; ++i) total += h[i];
            if (total == 0) return set_err(ctx, VRC_E_NONFINITE, "cube has no finite voxel");
            rank = (total - 1) / 2;   // lower median
        }
        uint64_t acc = 0;
        int sel = -1;
        for (int i = 0; i < nb; ++i) {
            if (acc + h[i] > rank) {
                sel = i;
                break;
            }
            acc += h[i];
        }
        if (sel < 0) return set_err(ctx, VRC_E_CUDA, "median selection inconsistent");
        if (pass == 0) ncand = h[sel] <= 0xffffffffull ? (uint32_t)h[sel] : 0u;
        prev_count = h[sel];
        rank -= acc;
        key |= (uint32_t)sel << a.shift;
    }
    if (npass == 2) key |= (key & 0x80000000u) ? 0u : 0x3ffu;
    const uint32_t u = (key & 0x80000000u) ? (key & 0x7fffffffu) : ~key;
    float f;
    memcpy(&f, &u, 4);
    *out = f;
    return VRC_OK;
}

}  // extern "C"
