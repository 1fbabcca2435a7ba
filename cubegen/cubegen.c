/*
 * cubegen.c -- seeded synthetic spectral-cube generator.
 *
 * This module only produces INPUTS: voxel values of a synthetic data cube
 * (Gaussian noise plus anisotropic Gaussian "sources").  It holds none of the
 * arithmetic of the method being tested (statistics, sampling, compositing);
 * both the CPU oracle and the CUDA library receive the bytes it writes.
 *
 * The paper's case study renders real spectral cubes (ASKAP-like, Sec. 3;
 * Table 1 sizes).  Those are not available, so a cube is defined here as
 *
 *   v(x,y,z) = fp32( noise(x,y,z) + sum_{s=0}^{S-1} src_s(x,y,z) )
 *
 * evaluated in double precision and rounded once to binary32, where
 *
 *   noise  = Box-Muller N(0,1) from two counter-based splitmix64 draws keyed by
 *            (seed, global linear voxel index), so any sub-box (brick) of the
 *            cube is generated bit-identically to the same voxels of the whole;
 *   src_s  = ((A_s * g_z) * g_y) * g_x with g_a = exp(-0.5*((X_a-c_a)/sigma_a)^2)
 *            for |X_a - c_a| <= 5 sigma_a and 0 outside (X_a = voxel centre,
 *            x_a + 0.5), A_s ~ U[5,50], sigma_a ~ U[2,10], c_a ~ U[0,N_a).
 *
 * Sources are added to the noise value in source-index order, voxel by voxel,
 * so the result does not depend on the number of threads.
 *
 * splitmix64 is the published mixer of Steele, Lea and Flood ("Fast splittable
 * pseudorandom number generators", OOPSLA 2014).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* uniform in [0,1) with 53 random bits */
static double u01(uint64_t key, uint64_t i)
{
    return (double)(splitmix64(key + i) >> 11) * 0x1.0p-53;
}

static uint64_t noise_key(uint64_t seed) { return splitmix64(seed); }
static uint64_t source_key(uint64_t seed) { return splitmix64(seed + 0x632BE59BD9B4E019ull); }

double cg_noise(uint64_t seed, uint64_t idx)
{
    const double two_pi = 6.283185307179586476925286766559;
    uint64_t key = noise_key(seed);
    double u1 = ((double)(splitmix64(key + 2 * idx) >> 11) + 0.5) * 0x1.0p-53; /* (0,1) */
    double u2 = (double)(splitmix64(key + 2 * idx + 1) >> 11) * 0x1.0p-53;     /* [0,1) */
    return sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

/* Source parameters, 7 doubles each: cx, cy, cz, A, sigma_x, sigma_y, sigma_z. */
void cg_sources(int64_t nx, int64_t ny, int64_t nz, uint64_t seed, int32_t n, double *out)
{
    uint64_t key = source_key(seed);
    for (int32_t s = 0; s < n; ++s) {
        uint64_t b = 8ull * (uint64_t)s;
        out[7 * s + 0] = u01(key, b + 0) * (double)nx;
        out[7 * s + 1] = u01(key, b + 1) * (double)ny;
        out[7 * s + 2] = u01(key, b + 2) * (double)nz;
        out[7 * s + 3] = 5.0 + 45.0 * u01(key, b + 3);
        out[7 * s + 4] = 2.0 + 8.0 * u01(key, b + 4);
        out[7 * s + 5] = 2.0 + 8.0 * u01(key, b + 5);
        out[7 * s + 6] = 2.0 + 8.0 * u01(key, b + 6);
    }
}

/* 1-D truncated Gaussian factor at voxel index i (centre i+0.5). */
static double gfac(int64_t i, double c, double sigma)
{
    double d = ((double)i + 0.5) - c;
    if (fabs(d) > 5.0 * sigma) return 0.0;
    double r = d / sigma;
    return exp(-0.5 * r * r);
}

/*
 * Generate the sub-box [x0,x0+sx) x [y0,y0+sy) x [z0,z0+sz) of the cube
 * (nx,ny,nz; seed; n_sources) into out (sx*sy*sz floats, x fastest).
 * Box coordinates outside the cube are allowed only as long as the box lies
 * inside it; returns 0 on success, -1 on bad arguments or allocation failure.
 */
int cg_generate_box(int64_t nx, int64_t ny, int64_t nz, uint64_t seed, int32_t n_sources,
                    int64_t x0, int64_t y0, int64_t z0, int64_t sx, int64_t sy, int64_t sz,
                    float *out)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || sx <= 0 || sy <= 0 || sz <= 0 || n_sources < 0) return -1;
    if (x0 < 0 || y0 < 0 || z0 < 0 || x0 + sx > nx || y0 + sy > ny || z0 + sz > nz) return -1;
    double *src = NULL;
    if (n_sources > 0) {
        src = (double *)malloc(sizeof(double) * 7 * (size_t)n_sources);
        if (!src) return -1;
        cg_sources(nx, ny, nz, seed, n_sources, src);
    }
    int failed = 0;
#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * (size_t)(sx * sy));
        double *gx = (double *)malloc(sizeof(double) * (size_t)sx);
        if (!buf || !gx) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(static)
        for (int64_t z = z0; z < z0 + sz; ++z) {
            if (!buf || !gx) continue;
            for (int64_t y = y0; y < y0 + sy; ++y) {
                uint64_t row = ((uint64_t)z * (uint64_t)ny + (uint64_t)y) * (uint64_t)nx;
                double *b = buf + (y - y0) * sx;
                for (int64_t x = x0; x < x0 + sx; ++x) b[x - x0] = cg_noise(seed, row + (uint64_t)x);
            }
            for (int32_t s = 0; s < n_sources; ++s) {
                const double *p = src + 7 * s;
                double gz = gfac(z, p[2], p[6]);
                if (gz == 0.0) continue;
                /* index range of voxels whose centre is within 5 sigma, clipped to the box */
                int64_t xa = (int64_t)floor(p[0] - 5.0 * p[4] - 0.5) - 1, xb = (int64_t)ceil(p[0] + 5.0 * p[4]) + 1;
                int64_t ya = (int64_t)floor(p[1] - 5.0 * p[5] - 0.5) - 1, yb = (int64_t)ceil(p[1] + 5.0 * p[5]) + 1;
                if (xa < x0) xa = x0;
                if (xb > x0 + sx) xb = x0 + sx;
                if (ya < y0) ya = y0;
                if (yb > y0 + sy) yb = y0 + sy;
                if (xa >= xb || ya >= yb) continue;
                for (int64_t x = xa; x < xb; ++x) gx[x - xa] = gfac(x, p[0], p[4]);
                double az = p[3] * gz;
                for (int64_t y = ya; y < yb; ++y) {
                    double gy = gfac(y, p[1], p[5]);
                    if (gy == 0.0) continue;
                    double amp = az * gy;
                    double *b = buf + (y - y0) * sx - x0;
                    for (int64_t x = xa; x < xb; ++x) {
                        double g = gx[x - xa];
                        if (g != 0.0) b[x] += amp * g;
                    }
                }
            }
            float *o = out + (z - z0) * sx * sy;
            for (int64_t i = 0; i < sx * sy; ++i) o[i] = (float)buf[i];
        }
        free(buf);
        free(gx);
    }
    free(src);
    return failed ? -1 : 0;
}

/*
 * Brick provider for out-of-core cubes: brick (bx, by, bz) of edge B with its
 * one-voxel halo, (B+2)^3 floats x fastest, covering voxels [b*B-1, b*B+B] of
 * each axis, positions outside the cube taking the value of the nearest voxel
 * inside it (clamp to edge).  `user` points to a cg_cube record; its `calls`
 * field counts the bricks generated.  Returns 0, or -1 when generation fails.
 */
typedef struct {
    int64_t nx, ny, nz;
    uint64_t seed;
    int32_t n_sources, B;
    int64_t calls;
} cg_cube;

int32_t cg_brick_source(void *user, int64_t brick, int32_t bx, int32_t by, int32_t bz, float *dst)
{
    (void)brick;
    cg_cube *c = (cg_cube *)user;
    const int64_t B = c->B, R = B + 2;
    const int64_t lo[3] = {(int64_t)bx * B - 1, (int64_t)by * B - 1, (int64_t)bz * B - 1};
    const int64_t n[3] = {c->nx, c->ny, c->nz};
    int64_t a[3], e[3];
    int inside = 1;
    for (int k = 0; k < 3; ++k) {
        a[k] = lo[k] < 0 ? 0 : lo[k];
        e[k] = lo[k] + R > n[k] ? n[k] : lo[k] + R;
        if (a[k] != lo[k] || e[k] != lo[k] + R) inside = 0;
        if (a[k] >= e[k]) return -1;
    }
    c->calls++;
    if (inside)
        return cg_generate_box(c->nx, c->ny, c->nz, c->seed, c->n_sources, a[0], a[1], a[2], R, R, R, dst) ? -1 : 0;
    /* border brick: generate the part inside the cube, then spread it with
       clamped indices */
    const int64_t sx = e[0] - a[0], sy = e[1] - a[1], sz = e[2] - a[2];
    float *tmp = (float *)malloc(sizeof(float) * (size_t)(sx * sy * sz));
    if (!tmp) return -1;
    if (cg_generate_box(c->nx, c->ny, c->nz, c->seed, c->n_sources, a[0], a[1], a[2], sx, sy, sz, tmp)) {
        free(tmp);
        return -1;
    }
    for (int64_t z = 0; z < R; ++z) {
        int64_t gz = lo[2] + z;
        gz = gz < a[2] ? a[2] : (gz >= e[2] ? e[2] - 1 : gz);
        for (int64_t y = 0; y < R; ++y) {
            int64_t gy = lo[1] + y;
            gy = gy < a[1] ? a[1] : (gy >= e[1] ? e[1] - 1 : gy);
            const float *row = tmp + ((gz - a[2]) * sy + (gy - a[1])) * sx;
            float *out = dst + (z * R + y) * R;
            for (int64_t x = 0; x < R; ++x) {
                int64_t gx = lo[0] + x;
                gx = gx < a[0] ? a[0] : (gx >= e[0] ? e[0] - 1 : gx);
                out[x] = row[gx - a[0]];
            }
        }
    }
    free(tmp);
    return 0;
}

