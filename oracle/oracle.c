/*
 * oracle.c -- plain, slow CPU reference of the cube analysis and rendering path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header or constant table with
 * the CUDA library.
 *
 * Scope (the paper's analysis tasks and its volume-rendering case study):
 *   - statistics: minimum/maximum and histogram (Abstract), standard deviation
 *     and median as global multi-pass tasks (Sec. 3);
 *   - ray casting of a data cube split into sub-cubes (bricks) whose partial
 *     images are gathered and composited (Sec. 2, the case study of Table 1).
 * The paper defers the rendering algorithm to its companion work, so the
 * rendering rules below are the stated readings of this project: trilinear /
 * nearest sampling on a global sample lattice, maximum-intensity projection,
 * front-to-back emission-absorption compositing with early termination, and
 * sort-last "over" compositing of per-brick partial images.
 *
 * Precision: all accumulation is in binary64.  The ray set-up (origin,
 * direction, entry/exit parameters, sample positions) and the histogram bin
 * formula are defined in binary32 with round-to-nearest-even and no FMA
 * contraction, because floating point there decides integers (sample counts,
 * voxel indices, bin numbers); this file is compiled with -ffp-contract=off.
 *
 * Parity pins live in tests/ (closed forms, brute force, invariants).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* --------------------------------------------------------------- statistics */

/* Neumaier-compensated running sum. */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

/*
 * min, max, mean and population standard deviation of the finite values
 * (Abstract: minimum/maximum; Sec. 3: standard deviation as a global task).
 * out = {min, max, mean, std}; counts = {n_finite, n_nonfinite}.
 * mean = compensated sum / n; std = sqrt(compensated sum of (x-mean)^2 / n),
 * i.e. the two-pass textbook definition.  Returns 0, or -1 if n_finite == 0.
 */
int orc_stats(const float *v, int64_t n, double *out, int64_t *counts)
{
    double mn = INFINITY, mx = -INFINITY;
    nsum s = {0, 0};
    int64_t nf = 0, nn = 0;
    for (int64_t i = 0; i < n; ++i) {
        double x = v[i];
        if (!isfinite(x)) { ++nn; continue; }
        if (x < mn) mn = x;
        if (x > mx) mx = x;
        nsum_add(&s, x);
        ++nf;
    }
    counts[0] = nf;
    counts[1] = nn;
    if (nf == 0) { out[0] = out[1] = out[2] = out[3] = NAN; return -1; }
    double mean = nsum_get(&s) / (double)nf;
    nsum q = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double x = v[i];
        if (!isfinite(x)) continue;
        double d = x - mean;
        nsum_add(&q, d * d);
    }
    out[0] = mn;
    out[1] = mx;
    out[2] = mean;
    out[3] = sqrt(nsum_get(&q) / (double)nf);
    return 0;
}

/*
 * Bin index of x for a histogram of nbins equal bins over [vmin, vmax]
 * (Abstract: "calculating a histogram").  Stated binary32 formula:
 *   range = fl32(vmax - vmin), scale = fl32(nbins / range),
 *   t = fl32(fl32(x - vmin) * scale), bin = trunc(t) clamped to [0, nbins-1];
 *   range == 0 puts every value in bin 0; t NaN -> bin 0; x == vmax -> last bin.
 */
static int32_t orc_bin(float x, float vmin, float range, float scale, int32_t nbins)
{
    if (!(range > 0.0f)) return 0;
    float d = x - vmin;
    float t = d * scale;
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)nbins) return nbins - 1;
    int32_t b = (int32_t)t;
    return b > nbins - 1 ? nbins - 1 : b;
}

int orc_histogram(const float *v, int64_t n, float vmin, float vmax, int32_t nbins, uint64_t *hist)
{
    if (nbins <= 0) return -1;
    float range = vmax - vmin;
    float scale = range > 0.0f ? (float)nbins / range : 0.0f;
    for (int32_t b = 0; b < nbins; ++b) hist[b] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(v[i])) continue;
        hist[orc_bin(v[i], vmin, range, scale, nbins)] += 1;
    }
    return 0;
}

static int cmp_float(const void *a, const void *b)
{
    float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/*
 * Median of the finite values (Sec. 3 names it as a global multi-pass task):
 * the lower median, i.e. the value of rank floor((n-1)/2) in ascending order.
 * Plain definition: copy, sort, pick.  Returns -1 when there is no finite value.
 */
int orc_median(const float *v, int64_t n, double *out)
{
    float *c = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    if (!c) return -2;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (isfinite(v[i])) c[m++] = v[i];
    if (m == 0) { free(c); *out = NAN; return -1; }
    qsort(c, (size_t)m, sizeof(float), cmp_float);
    *out = c[(m - 1) / 2];
    free(c);
    return 0;
}

/* ----------------------------------------------------------- storage formats */

/* bf16 value of x, round to nearest even (8 significant bits). */
float orc_bf16_round(float x)
{
    if (!isfinite(x) || x == 0.0f) return x;
    int e;
    frexp((double)x, &e);            /* |x| in [2^(e-1), 2^e) */
    int lo = e - 1;
    if (lo < -126) lo = -126;        /* subnormal spacing */
    double q = ldexp(1.0, lo - 7);   /* spacing of bf16 values near x */
    double r = rint((double)x / q) * q;
    if (fabs(r) > (double)FLT_MAX) return x > 0 ? INFINITY : -INFINITY;
    return (float)r;
}

/* Value of the OCP FP8 E4M3 (finite-only) number nearest to y, ties to even,
 * saturated to +-448.  Spacing: 2^(e-3) for |y| in [2^e, 2^(e+1)), e >= -6;
 * 2^-9 below 2^-6 (subnormals).  The format has no infinity: a non-finite y
 * (NaN or +-inf) becomes NaN, its only non-finite value, so that a stored
 * cube keeps its non-finite voxels non-finite (statistics skip them). */
double orc_e4m3_round(float y)
{
    if (isnan(y) || isinf(y)) return NAN;
    double a = fabs((double)y);
    if (a == 0.0) return 0.0 * (y < 0 ? -1.0 : 1.0);
    double q;
    if (a < ldexp(1.0, -6)) {
        q = ldexp(1.0, -9);
    } else {
        int e;
        frexp(a, &e);                /* a in [2^(e-1), 2^e) */
        q = ldexp(1.0, (e - 1) - 3);
    }
    double r = rint(a / q) * q;
    if (r > 448.0) r = 448.0;
    return y < 0 ? -r : r;
}

/* Per-brick FP8 scale: absmax of the finite values over the brick's stored
 * region (interior plus the one-voxel halo, clamp-to-edge),
 * scale = fl32(absmax / 448), and 1 if absmax == 0. */
static float orc_scale_of_brick(const float *v, const int64_t *dims, int32_t B,
                                int64_t bx, int64_t by, int64_t bz)
{
    float am = 0.0f;
    for (int64_t k = bz * B - 1; k <= bz * B + B; ++k)
        for (int64_t j = by * B - 1; j <= by * B + B; ++j)
            for (int64_t i = bx * B - 1; i <= bx * B + B; ++i) {
                int64_t ci = i < 0 ? 0 : (i >= dims[0] ? dims[0] - 1 : i);
                int64_t cj = j < 0 ? 0 : (j >= dims[1] ? dims[1] - 1 : j);
                int64_t ck = k < 0 ? 0 : (k >= dims[2] ? dims[2] - 1 : k);
                float a = fabsf(v[(ck * dims[1] + cj) * dims[0] + ci]);
                if (!isfinite(a)) continue;   /* non-finite voxels do not set the scale */
                if (a > am) am = a;
            }
    if (am == 0.0f) return 1.0f;
    return am / 448.0f;
}

int orc_brick_scales(const float *v, const int64_t *dims, int32_t B, float *scales)
{
    if (B <= 0) return -1;
    int64_t nb[3];
    for (int a = 0; a < 3; ++a) nb[a] = (dims[a] + B - 1) / B;
#pragma omp parallel for collapse(3) schedule(static)
    for (int64_t bz = 0; bz < nb[2]; ++bz)
        for (int64_t by = 0; by < nb[1]; ++by)
            for (int64_t bx = 0; bx < nb[0]; ++bx)
                scales[(bz * nb[1] + by) * nb[0] + bx] = orc_scale_of_brick(v, dims, B, bx, by, bz);
    return 0;
}

/* Stored (dequantised) value of voxel value x under storage dtype
 * 0 = fp32, 1 = bf16 (RNE), 2 = fp8 e4m3 with scale: fl32(e4m3(fl32(x/scale)) * scale). */
static double orc_stored(float x, int32_t dtype, float scale)
{
    if (dtype == 0) return x;
    if (dtype == 1) return orc_bf16_round(x);
    float y = x / scale;
    float q = (float)orc_e4m3_round(y);
    return (double)(q * scale);
}

/* Dequantised cube: every voxel stored by the brick that owns it. */
int orc_dequantize(const float *v, const int64_t *dims, int32_t dtype, int32_t B, const float *scales,
                   float *out)
{
    int64_t nbx = B > 0 ? (dims[0] + B - 1) / B : 1, nby = B > 0 ? (dims[1] + B - 1) / B : 1;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < dims[2]; ++k)
        for (int64_t j = 0; j < dims[1]; ++j)
            for (int64_t i = 0; i < dims[0]; ++i) {
                int64_t idx = (k * dims[1] + j) * dims[0] + i;
                float s = 1.0f;
                if (dtype == 2) s = scales[((k / B) * nby + (j / B)) * nbx + (i / B)];
                out[idx] = (float)orc_stored(v[idx], dtype, s);
            }
    return 0;
}

/* -------------------------------------------------------------- camera, rays */

typedef struct {
    int32_t kind;  /* 0 orthographic, 1 perspective */
    float eye[3], center[3], up[3];
    float fovy_deg, ortho_height;
} orc_camera;

/*
 * Per-view ray basis, evaluated in binary64 and rounded to binary32:
 *   w = normalise(center - eye); r = normalise(w x up); u = r x w; asp = W/H
 *   perspective: h = tan(fovy/2);   O0 = eye, D0 = w - (h*asp) r + h u
 *   orthographic: h = height/2;     O0 = eye - (h*asp) r + h u, D0 = w
 *   DX = (2 h asp / W) r, DY = (-2 h / H) u
 * basis = {O0[3], D0[3], DX[3], DY[3]}.  Pixel (px, py), row 0 at the top,
 * goes through the image point at (px+0.5, py+0.5) pixel units from O0/D0.
 */
void orc_camera_basis(const orc_camera *cam, int32_t W, int32_t H, float *basis)
{
    double e[3], w[3], r[3], u[3], up[3];
    for (int a = 0; a < 3; ++a) {
        e[a] = cam->eye[a];
        w[a] = (double)cam->center[a] - (double)cam->eye[a];
        up[a] = cam->up[a];
    }
    double lw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int a = 0; a < 3; ++a) w[a] = w[a] / lw;
    r[0] = w[1] * up[2] - w[2] * up[1];
    r[1] = w[2] * up[0] - w[0] * up[2];
    r[2] = w[0] * up[1] - w[1] * up[0];
    double lr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) r[a] = r[a] / lr;
    u[0] = r[1] * w[2] - r[2] * w[1];
    u[1] = r[2] * w[0] - r[0] * w[2];
    u[2] = r[0] * w[1] - r[1] * w[0];
    double asp = (double)W / (double)H;
    double h = cam->kind == 1 ? tan((double)cam->fovy_deg * 3.14159265358979323846 / 360.0)
                              : 0.5 * (double)cam->ortho_height;
    for (int a = 0; a < 3; ++a) {
        double o0, d0;
        if (cam->kind == 1) {
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

/*
 * Ray of pixel (px, py) in binary32 (every operation rounded, no FMA):
 *   fx = px + 0.5, fy = py + 0.5
 *   perspective:  o = O0;  q_a = (D0_a + fx DX_a) + fy DY_a;
 *                 n = sqrt((q_x q_x + q_y q_y) + q_z q_z);  d_a = q_a / n
 *   orthographic: o_a = (O0_a + fx DX_a) + fy DY_a;  d = D0
 * Slab test against [0,N_x] x [0,N_y] x [0,N_z]:
 *   start with lo = 0, hi = +inf; for each axis with d_a != 0:
 *   t0 = (0 - o_a)/d_a, t1 = (N_a - o_a)/d_a, swap so t0 <= t1,
 *   lo = max(lo, t0), hi = min(hi, t1); an axis with d_a == 0 misses when
 *   o_a < 0 or o_a > N_a.  The ray hits when lo < hi; t_entry = lo, t_exit = hi.
 * Returns 1 on a hit, 0 on a miss.
 */
int orc_ray(const float *basis, int32_t kind, int32_t px, int32_t py, const int64_t *dims,
            float *o, float *d, float *t)
{
    float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    if (kind == 1) {
        float q[3];
        for (int a = 0; a < 3; ++a) {
            o[a] = basis[a];
            float s = fx * basis[6 + a];
            float s2 = fy * basis[9 + a];
            q[a] = (basis[3 + a] + s) + s2;
        }
        float xx = q[0] * q[0], yy = q[1] * q[1], zz = q[2] * q[2];
        float n = sqrtf((xx + yy) + zz);
        for (int a = 0; a < 3; ++a) d[a] = q[a] / n;
    } else {
        for (int a = 0; a < 3; ++a) {
            float s = fx * basis[6 + a];
            float s2 = fy * basis[9 + a];
            o[a] = (basis[a] + s) + s2;
            d[a] = basis[3 + a];
        }
    }
    float lo = 0.0f, hi = INFINITY;
    for (int a = 0; a < 3; ++a) {
        float n = (float)dims[a];
        if (d[a] == 0.0f) {
            if (o[a] < 0.0f || o[a] > n) return 0;
            continue;
        }
        float t0 = (0.0f - o[a]) / d[a];
        float t1 = (n - o[a]) / d[a];
        if (t0 > t1) { float tmp = t0; t0 = t1; t1 = tmp; }
        if (t0 > lo) lo = t0;
        if (t1 < hi) hi = t1;
    }
    t[0] = lo;
    t[1] = hi;
    return lo < hi;
}

/* Sample k: t_k = t_entry + (k + 0.5) * step, p = o + t_k d (binary32). Sampling
 * continues while t_k < t_exit. */
static float orc_tk(float tentry, int64_t k, float step)
{
    float kk = (float)k + 0.5f;
    float m = kk * step;
    return tentry + m;
}
static void orc_pos(const float *o, const float *d, float tk, float *p)
{
    for (int a = 0; a < 3; ++a) {
        float m = tk * d[a];
        p[a] = o[a] + m;
    }
}

static int64_t clampi(int64_t i, int64_t n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

/* ------------------------------------------------------------------ sampling */

/* Volume accessor: either the plain cube (brick < 0) or brick b's stored copy
 * (voxel values quantised with that brick's scale; halo = clamp-to-edge). */
typedef struct {
    const float *v;
    int64_t dims[3];
    int32_t dtype, B;
    const float *scales;
    int64_t nb[3];
} orc_vol;

static double orc_voxel(const orc_vol *vol, int64_t brick, int64_t i, int64_t j, int64_t k)
{
    i = clampi(i, vol->dims[0]);
    j = clampi(j, vol->dims[1]);
    k = clampi(k, vol->dims[2]);
    float x = vol->v[(k * vol->dims[1] + j) * vol->dims[0] + i];
    float s = 1.0f;
    if (vol->dtype == 2) s = vol->scales[brick];
    return orc_stored(x, vol->dtype, s);
}

/* Nearest: voxel floor(p), clamped.  Trilinear: q = p - 0.5 (binary32),
 * i0 = floor(q), f = q - i0, weights (1-f, f) per axis, indices clamped to the
 * cube, product weights, evaluated in binary64. */
static double orc_sample(const orc_vol *vol, int64_t brick, const float *p, int32_t sampling)
{
    if (sampling == 0) {
        int64_t i = (int64_t)floorf(p[0]), j = (int64_t)floorf(p[1]), k = (int64_t)floorf(p[2]);
        return orc_voxel(vol, brick, i, j, k);
    }
    int64_t i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        float q = p[a] - 0.5f;
        float fl = floorf(q);
        i0[a] = (int64_t)fl;
        f[a] = (double)q - (double)fl;
    }
    double acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                acc += w * orc_voxel(vol, brick, i0[0] + dx, i0[1] + dy, i0[2] + dz);
            }
    return acc;
}

/* Brick containing sample position p: floor(p) clamped to the cube, / B. */
static int64_t orc_brick_of(const orc_vol *vol, const float *p, int64_t *bc)
{
    for (int a = 0; a < 3; ++a) bc[a] = clampi((int64_t)floorf(p[a]), vol->dims[a]) / vol->B;
    return (bc[2] * vol->nb[1] + bc[1]) * vol->nb[0] + bc[0];
}

/* --------------------------------------------------------------- compositing */

typedef struct {
    const float *tf;   /* 256 x RGBA, colour not premultiplied */
    double vmin, vmax;
    double term;
    int32_t opacity_correction;
    double step;
} orc_dvr;

/* Transfer function: u = clamp((s - vmin)/(vmax - vmin), 0, 1), x = 255 u,
 * linear between entries floor(x) and floor(x)+1.  NaN samples are transparent. */
static void orc_classify(const orc_dvr *c, double s, double *rgba)
{
    if (isnan(s)) { rgba[0] = rgba[1] = rgba[2] = rgba[3] = 0.0; return; }
    double u = c->vmax > c->vmin ? (s - c->vmin) / (c->vmax - c->vmin) : 0.0;
    if (u < 0.0) u = 0.0;
    if (u > 1.0) u = 1.0;
    double x = u * 255.0;
    double jf = floor(x);
    int j = (int)jf;
    if (j >= 255) {
        for (int ch = 0; ch < 4; ++ch) rgba[ch] = c->tf[255 * 4 + ch];
    } else {
        double fr = x - jf;
        for (int ch = 0; ch < 4; ++ch)
            rgba[ch] = (double)c->tf[j * 4 + ch] * (1.0 - fr) + (double)c->tf[(j + 1) * 4 + ch] * fr;
    }
    if (c->opacity_correction) rgba[3] = 1.0 - pow(1.0 - rgba[3], c->step);
}

/* front-to-back, premultiplied: C += (1-A) a c, A += (1-A) a */
static void orc_over_sample(double *acc, const double *rgba)
{
    double wgt = (1.0 - acc[3]) * rgba[3];
    acc[0] += wgt * rgba[0];
    acc[1] += wgt * rgba[1];
    acc[2] += wgt * rgba[2];
    acc[3] += wgt;
}

/* ------------------------------------------------------------------ renderers */

typedef struct {
    int32_t W, H;
    float step;
    int32_t sampling;  /* 0 nearest, 1 trilinear */
    int32_t mode;      /* 0 MIP, 1 DVR */
} orc_raycfg;

/*
 * Render selected pixels of one view.
 *   MIP:  out[i] = max over samples (or -FLT_MAX when the ray has none).
 *   DVR:  out[4i..4i+3] = premultiplied RGBA after compositing samples in ray
 *         order until A >= term (tested after each sample); background 0.
 * For DVR, lo/hi receive the RGBA at the earliest / latest sample index at which
 * a binary32 evaluation could stop, given an accumulated-alpha uncertainty of
 * tau(n) = 2e-7 n + 1e-6 (see DVR tests); flags[i] = 1 when lo != hi.
 * nsamp[i] = number of samples of the ray (DVR: composited before stopping).
 *
 * brick_size B > 0 selects the bricked, sort-last form: samples are grouped by
 * the brick containing them, bricks are visited in visibility order (Manhattan
 * distance of brick coordinates from the eye's brick cell), each brick yields a
 * partial result (MIP: max; DVR: premultiplied RGBA from zero, stopping when
 * the total alpha A + (1-A) A_partial reaches term), and partials are combined
 * with max / over: C = C + (1-A) C_p, A = A + (1-A) A_p.
 * Returns 0, or -3 if the visibility order disagrees with the ray order.
 */
int orc_render(const float *v, const int64_t *dims, int32_t dtype, int32_t brick_size,
               const float *scales, const orc_camera *cam, const orc_raycfg *rc, const float *tf,
               float vmin, float vmax, float term, int32_t opacity_correction,
               const int64_t *pix, int64_t npix, double *out, double *lo, double *hi,
               int32_t *flags, int64_t *nsamp)
{
    float basis[12];
    orc_camera_basis(cam, rc->W, rc->H, basis);
    orc_vol vol;
    vol.v = v;
    for (int a = 0; a < 3; ++a) vol.dims[a] = dims[a];
    vol.dtype = dtype;
    vol.B = brick_size;
    vol.scales = scales;
    for (int a = 0; a < 3; ++a) vol.nb[a] = brick_size > 0 ? (dims[a] + brick_size - 1) / brick_size : 1;
    orc_dvr dc = {tf, (double)vmin, (double)vmax, (double)term, opacity_correction, (double)rc->step};
    int bad = 0;

#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t ip = 0; ip < npix; ++ip) {
        int32_t px = (int32_t)(pix[ip] % rc->W), py = (int32_t)(pix[ip] / rc->W);
        float o[3], d[3], t[2];
        int hit = orc_ray(basis, cam->kind, px, py, dims, o, d, t);
        int64_t n = 0;
        if (hit)
            while (orc_tk(t[0], n, rc->step) < t[1]) ++n;
        double res[4] = {0, 0, 0, 0}, rlo[4] = {0, 0, 0, 0}, rhi[4] = {0, 0, 0, 0};
        int fragile = 0;
        int64_t used = n;

        if (rc->mode == 0) {
            double m = -FLT_MAX;
            if (brick_size <= 0) {
                for (int64_t k = 0; k < n; ++k) {
                    float p[3];
                    orc_pos(o, d, orc_tk(t[0], k, rc->step), p);
                    double s = orc_sample(&vol, -1, p, rc->sampling);
                    if (s > m) m = s;   /* NaN samples never win */
                }
            } else {
                /* per-brick partial maxima, combined with max */
                int64_t *bid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
                for (int64_t k = 0; k < n; ++k) {
                    float p[3];
                    int64_t bc[3];
                    orc_pos(o, d, orc_tk(t[0], k, rc->step), p);
                    bid[k] = orc_brick_of(&vol, p, bc);
                }
                for (int64_t k0 = 0; k0 < n;) {
                    int64_t b = bid[k0], k1 = k0;
                    double part = -FLT_MAX;
                    for (; k1 < n && bid[k1] == b; ++k1) {
                        float p[3];
                        orc_pos(o, d, orc_tk(t[0], k1, rc->step), p);
                        double s = orc_sample(&vol, b, p, rc->sampling);
                        if (s > part) part = s;
                    }
                    if (part > m) m = part;
                    k0 = k1;
                }
                free(bid);
            }
            res[0] = m;
        } else {
            /* DVR: alpha history to locate the stopping window */
            double *ahist = (double *)malloc(sizeof(double) * (size_t)(n + 1));
            double (*chist)[4] = (double (*)[4])malloc(sizeof(double) * 4 * (size_t)(n + 1));
            double acc[4] = {0, 0, 0, 0};
            ahist[0] = 0.0;
            for (int c = 0; c < 4; ++c) chist[0][c] = 0.0;
            int64_t stop = n;   /* index (number of samples) at which the exact rule stops */
            if (brick_size <= 0) {
                for (int64_t k = 0; k < n; ++k) {
                    float p[3];
                    double rgba[4];
                    orc_pos(o, d, orc_tk(t[0], k, rc->step), p);
                    orc_classify(&dc, orc_sample(&vol, -1, p, rc->sampling), rgba);
                    orc_over_sample(acc, rgba);
                    ahist[k + 1] = acc[3];
                    for (int c = 0; c < 4; ++c) chist[k + 1][c] = acc[c];
                    if (acc[3] >= dc.term && stop == n) { stop = k + 1; }
                    if (acc[3] >= dc.term + 1e-2) break;   /* nothing later can be selected */
                }
            } else {
                /* bricked: visibility order of bricks, partials from zero, over */
                int64_t *bid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
                int64_t *bkey = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
                int64_t ec[3];
                for (int a = 0; a < 3; ++a) {
                    if (cam->kind == 1) {
                        double f = floor((double)cam->eye[a] / (double)brick_size);
                        if (f < -1) f = -1;
                        if (f > (double)vol.nb[a]) f = (double)vol.nb[a];
                        ec[a] = (int64_t)f;
                    } else {
                        ec[a] = d[a] > 0 ? -1 : (d[a] < 0 ? vol.nb[a] : 0);
                    }
                }
                for (int64_t k = 0; k < n; ++k) {
                    float p[3];
                    int64_t bc[3];
                    orc_pos(o, d, orc_tk(t[0], k, rc->step), p);
                    bid[k] = orc_brick_of(&vol, p, bc);
                    bkey[k] = llabs(bc[0] - ec[0]) + llabs(bc[1] - ec[1]) + llabs(bc[2] - ec[2]);
                }
                /* visibility order must agree with ray order: keys strictly increase
                 * whenever the brick changes (checked, not assumed) */
                for (int64_t k = 1; k < n; ++k)
                    if (bid[k] != bid[k - 1] && !(bkey[k] > bkey[k - 1])) {
#pragma omp atomic write
                        bad = 1;
                    }
                int64_t k0 = 0;
                int done = 0;
                while (k0 < n && !done) {
                    int64_t b = bid[k0], k1 = k0;
                    double part[4] = {0, 0, 0, 0};
                    double a_front = acc[3];
                    for (; k1 < n && bid[k1] == b; ++k1) {
                        float p[3];
                        double rgba[4];
                        orc_pos(o, d, orc_tk(t[0], k1, rc->step), p);
                        orc_classify(&dc, orc_sample(&vol, b, p, rc->sampling), rgba);
                        orc_over_sample(part, rgba);
                        double a_tot = a_front + (1.0 - a_front) * part[3];
                        ahist[k1 + 1] = a_tot;
                        for (int c = 0; c < 3; ++c) chist[k1 + 1][c] = acc[c] + (1.0 - a_front) * part[c];
                        chist[k1 + 1][3] = a_tot;
                        if (a_tot >= dc.term && stop == n) stop = k1 + 1;
                        if (a_tot >= dc.term + 1e-2) { done = 1; ++k1; break; }
                    }
                    for (int c = 0; c < 3; ++c) acc[c] = acc[c] + (1.0 - a_front) * part[c];
                    acc[3] = a_front + (1.0 - a_front) * part[3];
                    k0 = k1;
                }
                /* fill the history past an early break so indices stay defined */
                for (int64_t k = k0; k < n; ++k) {
                    ahist[k + 1] = ahist[k];
                    for (int c = 0; c < 4; ++c) chist[k + 1][c] = chist[k][c];
                }
                free(bid);
                free(bkey);
            }
            /* stopping window for a binary32 evaluation with alpha error tau */
            double tau = 2e-7 * (double)n + 1e-6;
            int64_t klo = n, khi = n;
            for (int64_t k = 1; k <= n; ++k)
                if (ahist[k] >= dc.term - tau) { klo = k; break; }
            for (int64_t k = 1; k <= n; ++k)
                if (ahist[k] >= dc.term + tau) { khi = k; break; }
            if (klo > n) klo = n;
            /* history entries past a break are only valid up to the break */
            for (int c = 0; c < 4; ++c) {
                res[c] = chist[stop][c];
                rlo[c] = chist[klo][c];
                rhi[c] = chist[khi][c];
            }
            fragile = (klo != khi);
            used = stop;
            free(ahist);
            free(chist);
        }
        if (rc->mode == 0) {
            out[ip] = res[0];
        } else {
            for (int c = 0; c < 4; ++c) {
                out[4 * ip + c] = res[c];
                if (lo) lo[4 * ip + c] = rlo[c];
                if (hi) hi[4 * ip + c] = rhi[c];
            }
            if (flags) flags[ip] = fragile;
        }
        if (nsamp) nsamp[ip] = used;
    }
    return bad ? -3 : 0;
}

/* Sort-last combination of two partial images (Sec. 2 gathering of per-GPU
 * images, here per brick): DVR over, front + (1 - front.A) back, per channel;
 * MIP max. */
void orc_composite(const double *front, const double *back, int64_t npix, int32_t mode, double *out)
{
    for (int64_t i = 0; i < npix; ++i) {
        if (mode == 0) {
            out[i] = front[i] > back[i] ? front[i] : back[i];
        } else {
            double a = front[4 * i + 3];
            for (int c = 0; c < 4; ++c) out[4 * i + c] = front[4 * i + c] + (1.0 - a) * back[4 * i + c];
        }
    }
}

/* Array forms of the storage roundings (used by the tests). */
void orc_bf16_round_n(const float *x, int64_t n, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_bf16_round(x[i]);
}
void orc_e4m3_round_n(const float *x, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_e4m3_round(x[i]);
}
