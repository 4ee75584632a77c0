/*
 * cgdir_oracle.c -- plain FP64 CPU oracle of contour-guided demons
 * registration (CG-DIR, Gu et al., "A Contour-Guided Deformable Image
 * Registration Algorithm for Adaptive Radiotherapy").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * restatement that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, header or table with the
 * CUDA library.
 *
 * Every step is one loop nest over the volume, in the order of Algorithm A
 * (Sec. 2.2), with no fusion and no reordering; OpenMP only splits the
 * outermost (z) loop, and every reduction is summed per z-plane and then in
 * plane order, so results do not depend on the thread count.
 *
 * Layout: scalar volumes are [nz][ny][nx] (x fastest), displacement fields
 * are [3][nz][ny][nx] with components (x, y, z), in voxel units.  Masks are
 * k consecutive uint8 volumes, nonzero = inside.
 *
 * Readings where the paper is silent or garbled (each is stated again at the
 * function that implements it):
 *  - warp convention: pull-back, I0~u(x) = I0(x + u(x)) (Sec. 2.1, the Taylor
 *    step before Eq. 5 makes T0 - I0~ the residual of Eq. 7);
 *  - out-of-domain samples are clamped to the volume (replicate border);
 *  - modified images use CT number = HU + offset: I_i = (1 + s_i m_i/2) J,
 *    J = I0 + offset, T_i = (1 + s_i n_i/2)(T0 + offset) (Sec. 2.1);
 *  - du = 0 where |grad I0~|^2 == 0 exactly (the direction n of Eq. 5 is
 *    undefined there);
 *  - Gaussian: sigma in voxels, radius ceil(3 sigma), normalised taps,
 *    clamp-to-edge, passes x then y then z (Sec. 2.2);
 *  - stopping: see oracle_stop_test.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(x, y, z) ((((size_t)(z)) * (size_t)ny + (size_t)(y)) * (size_t)nx + (size_t)(x))

static long clampl(long v, long lo, long hi) { return v < lo ? lo : (v > hi ? hi : v); }
static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Trilinear sample of f at the continuous voxel position (px, py, pz).        */
/* Each coordinate is clamped to [0, n-1] before the floor; the upper corner   */
/* is clamped too; the weight of the upper corner is p - floor(p).             */
/* This is the interpolation of kernel 4 (Sec. 2.2).                          */
/* ------------------------------------------------------------------------- */
static double sample(const double *f, int nx, int ny, int nz, double px, double py, double pz)
{
    px = clampd(px, 0.0, (double)(nx - 1));
    py = clampd(py, 0.0, (double)(ny - 1));
    pz = clampd(pz, 0.0, (double)(nz - 1));
    long x0 = (long)floor(px), y0 = (long)floor(py), z0 = (long)floor(pz);
    long x1 = clampl(x0 + 1, 0, nx - 1), y1 = clampl(y0 + 1, 0, ny - 1), z1 = clampl(z0 + 1, 0, nz - 1);
    double wx = px - (double)x0, wy = py - (double)y0, wz = pz - (double)z0;
    double c000 = f[IDX(x0, y0, z0)], c100 = f[IDX(x1, y0, z0)];
    double c010 = f[IDX(x0, y1, z0)], c110 = f[IDX(x1, y1, z0)];
    double c001 = f[IDX(x0, y0, z1)], c101 = f[IDX(x1, y0, z1)];
    double c011 = f[IDX(x0, y1, z1)], c111 = f[IDX(x1, y1, z1)];
    return (1 - wz) * ((1 - wy) * ((1 - wx) * c000 + wx * c100) + wy * ((1 - wx) * c010 + wx * c110))
         + wz * ((1 - wy) * ((1 - wx) * c001 + wx * c101) + wy * ((1 - wx) * c011 + wx * c111));
}

/* Warp (kernel 4, Algorithm A step 5): out(x) = f(x + u(x)), pull-back. */
void oracle_warp(const double *f, const double *u, int nx, int ny, int nz, double *out)
{
    const size_t N = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = IDX(x, y, z);
                out[i] = sample(f, nx, ny, nz, x + u[i], y + u[N + i], z + u[2 * N + i]);
            }
}

/* Gradient (kernel 2): central difference (f[x+1] - f[x-1]) / 2 per axis with */
/* clamped indices, so a border value is the half one-sided difference.       */
void oracle_gradient(const double *f, int nx, int ny, int nz, double *g)
{
    const size_t N = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = IDX(x, y, z);
                g[i] = 0.5 * (f[IDX(clampl(x + 1, 0, nx - 1), y, z)] - f[IDX(clampl(x - 1, 0, nx - 1), y, z)]);
                g[N + i] = 0.5 * (f[IDX(x, clampl(y + 1, 0, ny - 1), z)] - f[IDX(x, clampl(y - 1, 0, ny - 1), z)]);
                g[2 * N + i] = 0.5 * (f[IDX(x, y, clampl(z + 1, 0, nz - 1))] - f[IDX(x, y, clampl(z - 1, 0, nz - 1))]);
            }
}

/* ------------------------------------------------------------------------- */
/* Gaussian low-pass filter (kernel 1, Sec. 2.2): unit standard deviation in  */
/* the paper; sigma here is in voxels of the current level.  Separable, x    */
/* then y then z, radius R = ceil(3 sigma), taps exp(-j^2 / (2 sigma^2))      */
/* normalised to sum 1, clamp-to-edge.  sigma == 0 is the identity.           */
/* ------------------------------------------------------------------------- */
int oracle_gauss_radius(double sigma)
{
    if (!(sigma > 0.0)) return 0;
    return (int)ceil(3.0 * sigma - 1e-9);
}

void oracle_gauss_taps(double sigma, double *taps /* 2R+1 */)
{
    int R = oracle_gauss_radius(sigma);
    if (R == 0) { taps[0] = 1.0; return; }
    double s = 0.0;
    for (int j = -R; j <= R; ++j) { taps[j + R] = exp(-(double)(j * j) / (2.0 * sigma * sigma)); s += taps[j + R]; }
    for (int j = -R; j <= R; ++j) taps[j + R] /= s;
}

static void gauss_axis(const double *in, double *out, int nx, int ny, int nz, const double *w, int R, int axis)
{
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double acc = 0.0;
                for (int j = -R; j <= R; ++j) {
                    size_t s;
                    if (axis == 0) s = IDX(clampl(x + j, 0, nx - 1), y, z);
                    else if (axis == 1) s = IDX(x, clampl(y + j, 0, ny - 1), z);
                    else s = IDX(x, y, clampl(z + j, 0, nz - 1));
                    acc += w[j + R] * in[s];
                }
                out[IDX(x, y, z)] = acc;
            }
}

void oracle_gauss(const double *in, int nx, int ny, int nz, double sigma, double *out)
{
    const size_t N = (size_t)nx * ny * nz;
    int R = oracle_gauss_radius(sigma);
    if (R == 0) { memmove(out, in, N * sizeof(double)); return; }
    double *w = (double *)malloc((2 * R + 1) * sizeof(double));
    double *a = (double *)malloc(N * sizeof(double));
    double *b = (double *)malloc(N * sizeof(double));
    oracle_gauss_taps(sigma, w);
    gauss_axis(in, a, nx, ny, nz, w, R, 0);
    gauss_axis(a, b, nx, ny, nz, w, R, 1);
    gauss_axis(b, out, nx, ny, nz, w, R, 2);
    free(w); free(a); free(b);
}

/* Smooth each of the three components of a displacement field. */
void oracle_gauss_field(const double *in, int nx, int ny, int nz, double sigma, double *out)
{
    const size_t N = (size_t)nx * ny * nz;
    for (int c = 0; c < 3; ++c) oracle_gauss(in + c * N, nx, ny, nz, sigma, out + c * N);
}

/* ------------------------------------------------------------------------- */
/* Composite update (Algorithm A step 3, kernel 4): u <- u o (Id + du), i.e.  */
/* u_new(x) = du(x) + u(x + du(x)), trilinear with clamped coordinates.       */
/* mode 1 is the additive variant u_new = u + du.                             */
/* ------------------------------------------------------------------------- */
void oracle_compose(const double *u, const double *du, int nx, int ny, int nz, int mode, double *out)
{
    const size_t N = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = IDX(x, y, z);
                if (mode == 1) {
                    for (int c = 0; c < 3; ++c) out[c * N + i] = u[c * N + i] + du[c * N + i];
                    continue;
                }
                double px = x + du[i], py = y + du[N + i], pz = z + du[2 * N + i];
                for (int c = 0; c < 3; ++c)
                    out[c * N + i] = du[c * N + i] + sample(u + c * N, nx, ny, nz, px, py, pz);
            }
}

/* ------------------------------------------------------------------------- */
/* Moving-vector kernel (kernels 2 + 3, Algorithm A step 1): du = v n with v  */
/* from Eq. 7, n = grad I0~ / |grad I0~| (Sec. 2.1) and beta = (T0 - I0~)^2    */
/* (the choice stated after Eq. 7).  The modified images of Sec. 2.1 are built */
/* explicitly, one structure at a time, then warped and differentiated like    */
/* I0:                                                                         */
/*   I_i = (1 + s_i m_i / 2) (I0 + offset),  T_i = (1 + s_i n_i / 2)(T0 + off),*/
/* m_i, n_i = moving / static mask of structure i (0/1), s_i = +-1.            */
/* Eq. 7's sums are accumulated in structure order:                            */
/*   num = a0 r0 + sum_i lambda_i a_i r_i,                                     */
/*   den = a0^2 + sum_i lambda_i a_i^2 + beta,                                 */
/* with a0 = grad I0~ . n, a_i = grad I_i~ . n, r0 = T0 - I0~, r_i = T_i - I_i~.*/
/* contour == 0 drops the structure terms (plain demons, used at coarse       */
/* levels, Sec. 2.2).  Where |grad I0~|^2 == 0, du = 0.                        */
/* Optional outputs (may be NULL): warped = I0~.                               */
/* ------------------------------------------------------------------------- */
void oracle_force(const double *I0, const double *T0, const uint8_t *mmask, const uint8_t *smask, int k,
                  const double *lambda, const int *sign, double offset, int contour,
                  const double *u, int nx, int ny, int nz, double *du, double *warped_out)
{
    const size_t N = (size_t)nx * ny * nz;
    double *w0 = (double *)malloc(N * sizeof(double));
    double *g0 = (double *)malloc(3 * N * sizeof(double));
    double *num = (double *)malloc(N * sizeof(double));
    double *den = (double *)malloc(N * sizeof(double));
    oracle_warp(I0, u, nx, ny, nz, w0);
    oracle_gradient(w0, nx, ny, nz, g0);

    /* demons term */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)N; ++i) {
        double gx = g0[i], gy = g0[N + i], gz = g0[2 * N + i];
        double g2 = gx * gx + gy * gy + gz * gz;
        if (g2 == 0.0) { num[i] = 0.0; den[i] = 1.0; continue; }
        double gn = sqrt(g2);
        double a0 = (gx * gx + gy * gy + gz * gz) / gn;     /* grad I0~ . n */
        double r0 = T0[i] - w0[i];
        num[i] = a0 * r0;
        den[i] = a0 * a0;
    }

    if (contour && k > 0) {
        double *Ii = (double *)malloc(N * sizeof(double));
        double *wi = (double *)malloc(N * sizeof(double));
        double *gi = (double *)malloc(3 * N * sizeof(double));
        for (int s = 0; s < k; ++s) {
            const uint8_t *m = mmask + (size_t)s * N;
            const uint8_t *n = smask + (size_t)s * N;
            double sg = (double)sign[s];
#pragma omp parallel for schedule(static)
            for (long i = 0; i < (long)N; ++i)
                Ii[i] = (1.0 + sg * (m[i] ? 1.0 : 0.0) / 2.0) * (I0[i] + offset);
            oracle_warp(Ii, u, nx, ny, nz, wi);
            oracle_gradient(wi, nx, ny, nz, gi);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < (long)N; ++i) {
                double gx = g0[i], gy = g0[N + i], gz = g0[2 * N + i];
                double g2 = gx * gx + gy * gy + gz * gz;
                if (g2 == 0.0) continue;
                double gn = sqrt(g2);
                double ai = (gi[i] * gx + gi[N + i] * gy + gi[2 * N + i] * gz) / gn;   /* grad I_i~ . n */
                double Ti = (1.0 + sg * (n[i] ? 1.0 : 0.0) / 2.0) * (T0[i] + offset);
                double ri = Ti - wi[i];
                num[i] += lambda[s] * ai * ri;
                den[i] += lambda[s] * ai * ai;
            }
        }
        free(Ii); free(wi); free(gi);
    }

#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)N; ++i) {
        double gx = g0[i], gy = g0[N + i], gz = g0[2 * N + i];
        double g2 = gx * gx + gy * gy + gz * gz;
        if (g2 == 0.0) { du[i] = du[N + i] = du[2 * N + i] = 0.0; continue; }
        double gn = sqrt(g2);
        double r0 = T0[i] - w0[i];
        double v = num[i] / (den[i] + r0 * r0);          /* + beta */
        du[i] = v * gx / gn;
        du[N + i] = v * gy / gn;
        du[2 * N + i] = v * gz / gn;
    }
    if (warped_out) memcpy(warped_out, w0, N * sizeof(double));
    free(w0); free(g0); free(num); free(den);
}

/* ------------------------------------------------------------------------- */
/* Pyramid (Sec. 2.2: factor-2 down-sampling per dimension, up-sampling of    */
/* the moving vectors).  Restriction: 2x2x2 box mean, size ceil(n/2), source  */
/* indices clamped for odd sizes.  Masks: the box mean of the 0/1 values,     */
/* >= 0.5 counts as inside.  Prolongation: cell-centred trilinear, the fine   */
/* voxel x reads the coarse field at (x + 0.5)/2 - 0.5 (clamped) and the      */
/* displacement doubles because it is in voxel units.                         */
/* ------------------------------------------------------------------------- */
void oracle_restrict_image(const double *in, int nx, int ny, int nz, double *out)
{
    int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int Z = 0; Z < cz; ++Z)
        for (int Y = 0; Y < cy; ++Y)
            for (int X = 0; X < cx; ++X) {
                double s = 0.0;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx)
                            s += in[IDX(clampl(2 * X + dx, 0, nx - 1), clampl(2 * Y + dy, 0, ny - 1),
                                        clampl(2 * Z + dz, 0, nz - 1))];
                out[((size_t)Z * cy + Y) * cx + X] = s / 8.0;
            }
}

void oracle_restrict_mask(const uint8_t *in, int nx, int ny, int nz, uint8_t *out)
{
    int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int Z = 0; Z < cz; ++Z)
        for (int Y = 0; Y < cy; ++Y)
            for (int X = 0; X < cx; ++X) {
                double s = 0.0;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx)
                            s += in[IDX(clampl(2 * X + dx, 0, nx - 1), clampl(2 * Y + dy, 0, ny - 1),
                                        clampl(2 * Z + dz, 0, nz - 1))] ? 1.0 : 0.0;
                out[((size_t)Z * cy + Y) * cx + X] = (s / 8.0 >= 0.5) ? 1 : 0;
            }
}

void oracle_prolong(const double *uc, int cx, int cy, int cz, int nx, int ny, int nz, double *uf)
{
    const size_t N = (size_t)nx * ny * nz, Nc = (size_t)cx * cy * cz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double px = (x + 0.5) / 2.0 - 0.5, py = (y + 0.5) / 2.0 - 0.5, pz = (z + 0.5) / 2.0 - 0.5;
                for (int c = 0; c < 3; ++c)
                    uf[c * N + IDX(x, y, z)] = 2.0 * sample(uc + c * Nc, cx, cy, cz, px, py, pz);
            }
}

/* ------------------------------------------------------------------------- */
/* UROI (Sec. 2.2, stopping criterion): the union of the static-space ROIs,   */
/* each expanded by a margin (1 cm in the paper).  A voxel x is in the UROI   */
/* if some ROI voxel y has sum_a ((x_a - y_a) spacing_a)^2 <= margin^2.       */
/* k == 0 (no structures) makes the whole volume the UROI.                    */
/* ------------------------------------------------------------------------- */
void oracle_uroi(const uint8_t *smask, int k, int nx, int ny, int nz, const double *spacing, double margin,
                 uint8_t *out)
{
    const size_t N = (size_t)nx * ny * nz;
    if (k <= 0) { memset(out, 1, N); return; }
    uint8_t *uni = (uint8_t *)calloc(N, 1);
    for (int s = 0; s < k; ++s)
        for (size_t i = 0; i < N; ++i) uni[i] |= smask[(size_t)s * N + i] ? 1 : 0;
    int rx = (int)floor(margin / spacing[0]), ry = (int)floor(margin / spacing[1]), rz = (int)floor(margin / spacing[2]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                uint8_t hit = 0;
                for (int dz = -rz; dz <= rz && !hit; ++dz) {
                    int zz = z + dz;
                    if (zz < 0 || zz >= nz) continue;
                    for (int dy = -ry; dy <= ry && !hit; ++dy) {
                        int yy = y + dy;
                        if (yy < 0 || yy >= ny) continue;
                        for (int dx = -rx; dx <= rx; ++dx) {
                            int xx = x + dx;
                            if (xx < 0 || xx >= nx) continue;
                            double d2 = (dx * spacing[0]) * (dx * spacing[0]) + (dy * spacing[1]) * (dy * spacing[1])
                                      + (dz * spacing[2]) * (dz * spacing[2]);
                            if (d2 <= margin * margin && uni[IDX(xx, yy, zz)]) { hit = 1; break; }
                        }
                    }
                }
                out[IDX(x, y, z)] = hit;
            }
    free(uni);
}

/* ------------------------------------------------------------------------- */
/* Automatic sign of M_i, N_i (Sec. 2.1: positive when the ROI is brighter   */
/* than its surroundings).  "Surroundings" is read as the shell of voxels    */
/* within Chebyshev distance 2 of the static ROI and outside it; the sign is */
/* +1 when mean(T0 in ROI) >= mean(T0 in shell), else -1 (+1 for an empty    */
/* ROI or shell).                                                             */
/* ------------------------------------------------------------------------- */
void oracle_auto_sign(const double *T0, const uint8_t *smask, int k, int nx, int ny, int nz, int *sign_out)
{
    for (int s = 0; s < k; ++s) {
        const uint8_t *m = smask + (size_t)s * nx * ny * nz;
        double sin_ = 0, ssh = 0; long cin = 0, csh = 0;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t i = IDX(x, y, z);
                    if (m[i]) { sin_ += T0[i]; cin++; continue; }
                    int near = 0;
                    for (int dz = -2; dz <= 2 && !near; ++dz)
                        for (int dy = -2; dy <= 2 && !near; ++dy)
                            for (int dx = -2; dx <= 2; ++dx) {
                                int xx = x + dx, yy = y + dy, zz = z + dz;
                                if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
                                if (m[IDX(xx, yy, zz)]) { near = 1; break; }
                            }
                    if (near) { ssh += T0[i]; csh++; }
                }
        if (cin == 0 || csh == 0) sign_out[s] = 1;
        else sign_out[s] = (sin_ / cin >= ssh / csh) ? 1 : -1;
    }
}

/* ------------------------------------------------------------------------- */
/* RMS-ID over the UROI (Sec. 2.2): delta = sqrt(sum (I0~ - T0)^2 / |UROI|); */
/* 0 when the UROI is empty.  Summed per z-plane, then in plane order.       */
/* ------------------------------------------------------------------------- */
double oracle_rms_id(const double *warped, const double *T0, const uint8_t *uroi, int nx, int ny, int nz,
                     long *count_out)
{
    double *ps = (double *)calloc(nz, sizeof(double));
    long *pc = (long *)calloc(nz, sizeof(long));
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
        double s = 0.0; long c = 0;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = IDX(x, y, z);
                if (!uroi[i]) continue;
                double d = warped[i] - T0[i];
                s += d * d; c++;
            }
        ps[z] = s; pc[z] = c;
    }
    double s = 0.0; long c = 0;
    for (int z = 0; z < nz; ++z) { s += ps[z]; c += pc[z]; }
    free(ps); free(pc);
    if (count_out) *count_out = c;
    return c > 0 ? sqrt(s / (double)c) : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Stopping test (Sec. 2.2), given delta^0 .. delta^n.                        */
/*  mode 0 FIXED: never (the level runs its iteration cap);                   */
/*  mode 1 WINDOW10 (default reading): stop once n >= 10 and                  */
/*         delta^(n-10) - delta^n <= eps;                                     */
/*  mode 2 PAPER_LITERAL: with l^(n) = delta^n - delta^(n-1), stop once       */
/*         n >= 11 and l^(n-10) - l^(n) <= eps.  Read literally this fires at */
/*         the first chance whenever delta decreases and decelerates, which   */
/*         is why WINDOW10 is the default reading.                            */
/* ------------------------------------------------------------------------- */
int oracle_stop_test(const double *d, int n, int mode, double eps)
{
    if (mode == 1) return (n >= 10) && (d[n - 10] - d[n] <= eps);
    if (mode == 2) {
        if (n < 11) return 0;
        double l_n = d[n] - d[n - 1], l_m = d[n - 10] - d[n - 11];
        return (l_m - l_n) <= eps;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* One iteration of the Algorithm A loop at one level, steps 1-4:            */
/* force (Eq. 7) -> smooth du -> compose -> smooth u.                         */
/* u_out may alias nothing; du_out (optional) receives the smoothed du.       */
/* ------------------------------------------------------------------------- */
void oracle_step(const double *I0, const double *T0, const uint8_t *mmask, const uint8_t *smask, int k,
                 const double *lambda, const int *sign, double offset, int contour,
                 double sigma_fluid, double sigma_diff, int compose_mode,
                 const double *u_in, int nx, int ny, int nz, double *u_out, double *du_out)
{
    const size_t N = (size_t)nx * ny * nz;
    double *du = (double *)malloc(3 * N * sizeof(double));
    double *dus = (double *)malloc(3 * N * sizeof(double));
    double *un = (double *)malloc(3 * N * sizeof(double));
    oracle_force(I0, T0, mmask, smask, k, lambda, sign, offset, contour, u_in, nx, ny, nz, du, NULL);
    oracle_gauss_field(du, nx, ny, nz, sigma_fluid, dus);            /* step 2 */
    oracle_compose(u_in, dus, nx, ny, nz, compose_mode, un);          /* step 3 */
    oracle_gauss_field(un, nx, ny, nz, sigma_diff, u_out);            /* step 4 */
    if (du_out) memcpy(du_out, dus, 3 * N * sizeof(double));
    free(du); free(dus); free(un);
}

/* ------------------------------------------------------------------------- */
/* Algorithm A, whole registration over a coarse-to-fine pyramid.             */
/*  levels, iters[levels] (coarse -> fine), sigma_fluid / sigma_diff,         */
/*  lambda[k], sign[k] (0 = automatic, decided once on the full-resolution    */
/*  static image), contour_mask (bit l: structure terms at level l, 0 =       */
/*  coarsest), stop_mode / eps, spacing[3] (mm at full resolution, doubled    */
/*  per coarser level), margin (mm), offset, compose_mode, init_dvf (NULL or  */
/*  a full-resolution field; it replaces the coarse levels, Sec. 4).          */
/* Outputs: dvf [3][N], and per level iters_run, stop_reason (0 = iteration   */
/*  cap, 1 = converged, 2 = skipped), hist_len and the delta history, level l */
/*  at hist + l * hist_stride.                                                */
/* Level loop (iteration n = 0, 1, ...): warp, delta^n, stop test, cap test,  */
/*  then steps 1-4.  The first warp stands in for step 5 of the previous      */
/*  iteration.  Between levels u is prolongated.                              */
/* ------------------------------------------------------------------------- */
int oracle_register(const double *static_img, const double *moving_img, const uint8_t *smask, const uint8_t *mmask,
                    int k, int nx, int ny, int nz,
                    int levels, const int *iters, double sigma_fluid, double sigma_diff,
                    const double *lambda, const int *sign_in, unsigned contour_mask,
                    int stop_mode, double eps, const double *spacing, double margin, double offset,
                    int compose_mode, const double *init_dvf,
                    double *dvf, int *iters_run, int *stop_reason, int *hist_len, double *hist, int hist_stride)
{
    if (levels < 1 || levels > 8 || k < 0 || nx < 1 || ny < 1 || nz < 1) return 1;
    int *sign = (int *)malloc((k > 0 ? k : 1) * sizeof(int));
    int *auto_s = (int *)malloc((k > 0 ? k : 1) * sizeof(int));
    if (k > 0) oracle_auto_sign(static_img, smask, k, nx, ny, nz, auto_s);
    for (int s = 0; s < k; ++s) sign[s] = sign_in && sign_in[s] ? (sign_in[s] > 0 ? 1 : -1) : auto_s[s];

    /* pyramid, finest = level levels-1 */
    int dims[8][3];
    double *T[8], *I[8];
    uint8_t *SM[8], *MM[8];
    dims[levels - 1][0] = nx; dims[levels - 1][1] = ny; dims[levels - 1][2] = nz;
    for (int l = levels - 2; l >= 0; --l)
        for (int a = 0; a < 3; ++a) dims[l][a] = (dims[l + 1][a] + 1) / 2;
    size_t Nf = (size_t)nx * ny * nz;
    T[levels - 1] = (double *)malloc(Nf * sizeof(double));
    I[levels - 1] = (double *)malloc(Nf * sizeof(double));
    SM[levels - 1] = (uint8_t *)malloc(k * Nf + 1);
    MM[levels - 1] = (uint8_t *)malloc(k * Nf + 1);
    memcpy(T[levels - 1], static_img, Nf * sizeof(double));
    memcpy(I[levels - 1], moving_img, Nf * sizeof(double));
    if (k) { memcpy(SM[levels - 1], smask, k * Nf); memcpy(MM[levels - 1], mmask, k * Nf); }
    for (int l = levels - 2; l >= 0; --l) {
        size_t Nl = (size_t)dims[l][0] * dims[l][1] * dims[l][2];
        size_t Nu = (size_t)dims[l + 1][0] * dims[l + 1][1] * dims[l + 1][2];
        T[l] = (double *)malloc(Nl * sizeof(double));
        I[l] = (double *)malloc(Nl * sizeof(double));
        SM[l] = (uint8_t *)malloc(k * Nl + 1);
        MM[l] = (uint8_t *)malloc(k * Nl + 1);
        oracle_restrict_image(T[l + 1], dims[l + 1][0], dims[l + 1][1], dims[l + 1][2], T[l]);
        oracle_restrict_image(I[l + 1], dims[l + 1][0], dims[l + 1][1], dims[l + 1][2], I[l]);
        for (int s = 0; s < k; ++s) {
            oracle_restrict_mask(SM[l + 1] + s * Nu, dims[l + 1][0], dims[l + 1][1], dims[l + 1][2], SM[l] + s * Nl);
            oracle_restrict_mask(MM[l + 1] + s * Nu, dims[l + 1][0], dims[l + 1][1], dims[l + 1][2], MM[l] + s * Nl);
        }
    }

    double *u = NULL;
    int first = 0;
    if (init_dvf) {
        first = levels - 1;
        for (int l = 0; l < first; ++l) { iters_run[l] = 0; stop_reason[l] = 2; hist_len[l] = 0; }
        u = (double *)malloc(3 * Nf * sizeof(double));
        memcpy(u, init_dvf, 3 * Nf * sizeof(double));
    }
    for (int l = first; l < levels; ++l) {
        int lx = dims[l][0], ly = dims[l][1], lz = dims[l][2];
        size_t Nl = (size_t)lx * ly * lz;
        if (!u) {
            u = (double *)calloc(3 * Nl, sizeof(double));          /* u0 := 0 */
        } else if (l > first) {
            double *uf = (double *)malloc(3 * Nl * sizeof(double));
            oracle_prolong(u, dims[l - 1][0], dims[l - 1][1], dims[l - 1][2], lx, ly, lz, uf);
            free(u); u = uf;
        }
        double sp[3];
        for (int a = 0; a < 3; ++a) sp[a] = spacing[a] * (double)(1 << (levels - 1 - l));
        uint8_t *uroi = (uint8_t *)malloc(Nl);
        oracle_uroi(SM[l], k, lx, ly, lz, sp, margin, uroi);
        int contour = (int)((contour_mask >> l) & 1u);
        double *warped = (double *)malloc(Nl * sizeof(double));
        double *un = (double *)malloc(3 * Nl * sizeof(double));
        double *d = hist + (size_t)l * hist_stride;
        int n = 0;
        for (;; ++n) {
            oracle_warp(I[l], u, lx, ly, lz, warped);                          /* step 5 */
            d[n] = oracle_rms_id(warped, T[l], uroi, lx, ly, lz, NULL);          /* step 6 */
            if (oracle_stop_test(d, n, stop_mode, eps)) { stop_reason[l] = 1; break; }
            if (n >= iters[l] || n + 1 >= hist_stride) { stop_reason[l] = 0; break; }
            oracle_step(I[l], T[l], MM[l], SM[l], k, lambda, sign, offset, contour, sigma_fluid, sigma_diff,
                        compose_mode, u, lx, ly, lz, un, NULL);                  /* steps 1-4 */
            double *t = u; u = un; un = t;
        }
        iters_run[l] = n;
        hist_len[l] = n + 1;
        free(uroi); free(warped); free(un);
    }
    memcpy(dvf, u, 3 * Nf * sizeof(double));
    free(u);
    for (int l = 0; l < levels; ++l) { free(T[l]); free(I[l]); free(SM[l]); free(MM[l]); }
    free(sign); free(auto_s);
    return 0;
}
