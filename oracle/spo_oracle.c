/*
 * FP64 CPU oracle for periodic tricubic B-spline orbital evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the test suite, the smoke check and the CPU baseline
 * leg of the benchmark do.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * What it computes (arXiv 1708.02645, Sec. 3 "QMC algorithms": the Slater
 * matrix entries A(i,j) = phi_i(r_j) and their derivatives needed by Alg. 1
 * "ratio" and "derivatives"; Sec. 6.1 names the routines Bspline-v,
 * Bspline-vgh and SPO-vgl; the table is Sec. 6.2's read-only table with
 * four indices).  The paper cites but does not print the B-spline formula;
 * this file follows the textbook uniform cubic B-spline:
 *
 *   B3(s) = (2-|s|)^3/6              1 <= |s| < 2
 *         = 2/3 - s^2 + |s|^3/2      |s| < 1
 *         = 0                        otherwise
 *
 *   phi_n(r) = sum_{m in Z^3} c[m mod n][n] prod_d B3(r_d n_d - m_d)
 *
 * on the periodic unit cube, grid n_x x n_y x n_z, basis function m centred
 * on grid node m/n.  For u = r n with cell i = floor(u) and t = u - i, only
 * m = i-1, i, i+1, i+2 contribute, with weights
 *
 *   w0 = (1-t)^3/6, w1 = (3t^3 - 6t^2 + 4)/6, w2 = (-3t^3 + 3t^2 + 3t + 1)/6,
 *   w3 = t^3/6,
 *
 * their first derivatives in u times n (Cartesian gradient) and second
 * derivatives times n^2.  Every output is the plain 64-term sum over the
 * 4x4x4 window, in the order (a, b, g) = x, y, z corner offsets.  Nothing is
 * factored: each of the 10 outputs is its own sum of weight product times
 * coefficient.
 *
 * Coefficient table: C order [nx][ny][nz][N] (orbital fastest), FP64.
 * Positions: [P][3], FP64 (the tests pass FP32 values promoted to FP64, so
 *            u = r n is exact and t is the exact fractional part).
 * Outputs (orbital fastest, one row per component):
 *   kind 0 (V):   [P][N]
 *   kind 1 (VGL): [P][5][N]   v, gx, gy, gz, lap
 *   kind 2 (VGH): [P][10][N]  v, gx, gy, gz, hxx, hxy, hxz, hyy, hyz, hzz
 *
 * Parity status: pinned (see tests/test_oracle_pins.py: partition of unity,
 * impulse response, polynomial reproduction, plane-wave closed form at
 * nodes, C2 continuity, finite differences, periodic wrap, brute-force
 * global sum, linearity); the condition sums by their closed forms for
 * tables with constant |c|, a brute-force sum over all images, and
 * beta_V = V for non-negative tables.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* cell index and fractional coordinate of one Cartesian coordinate r on a
 * periodic axis with n intervals: u = r n, i = floor(u) mod n, t = u - floor(u) */
static void reduce_coordinate(double r, int n, long *i_out, double *t_out)
{
    double u = r * (double)n;
    double fl = floor(u);
    double t = u - fl;
    long i;
    if (!(fl == fl) || fabs(fl) > 9.0e15) { /* NaN or absurd: clamp to cell 0 */
        i = 0;
        t = 0.0;
    } else {
        i = (long)fmod(fl, (double)n);
        if (i < 0) i += n;
    }
    *i_out = i;
    *t_out = t;
}

/* the four cubic B-spline weights of a cell with fractional coordinate t,
 * and their first and second derivatives with respect to r = u / n */
static void basis_weights(double t, int n, double w[4], double dw[4], double d2w[4])
{
    double s = 1.0 - t;
    double nn = (double)n;
    w[0] = s * s * s / 6.0;
    w[1] = (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;
    w[2] = (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;
    w[3] = t * t * t / 6.0;

    dw[0] = -0.5 * s * s * nn;
    dw[1] = 0.5 * (3.0 * t * t - 4.0 * t) * nn;
    dw[2] = 0.5 * (-3.0 * t * t + 2.0 * t + 1.0) * nn;
    dw[3] = 0.5 * t * t * nn;

    d2w[0] = s * nn * nn;
    d2w[1] = (3.0 * t - 2.0) * nn * nn;
    d2w[2] = (1.0 - 3.0 * t) * nn * nn;
    d2w[3] = t * nn * nn;
}

static int n_components(int kind)
{
    return kind == 0 ? 1 : (kind == 1 ? 5 : 10);
}

/* The ten 64-term sums (v, gx, gy, gz, hxx, hxy, hxz, hyy, hyz, hzz) of one
 * position for all N orbitals, written to h[10][N]. */
static void window_sums_vgh(int nx, int ny, int nz, long N, const double *coefs,
                            const double pos[3], double *h)
{
    long ix, iy, iz;
    double tx, ty, tz;
    reduce_coordinate(pos[0], nx, &ix, &tx);
    reduce_coordinate(pos[1], ny, &iy, &ty);
    reduce_coordinate(pos[2], nz, &iz, &tz);
    double wx[4], dwx[4], d2wx[4];
    double wy[4], dwy[4], d2wy[4];
    double wz[4], dwz[4], d2wz[4];
    basis_weights(tx, nx, wx, dwx, d2wx);
    basis_weights(ty, ny, wy, dwy, d2wy);
    basis_weights(tz, nz, wz, dwz, d2wz);

    for (long k = 0; k < 10 * N; ++k) h[k] = 0.0;
    for (int a = 0; a < 4; ++a) {
        long xa = (ix + a - 1 + nx) % nx;
        for (int b = 0; b < 4; ++b) {
            long yb = (iy + b - 1 + ny) % ny;
            for (int g = 0; g < 4; ++g) {
                long zg = (iz + g - 1 + nz) % nz;
                const double *c = coefs + (((size_t)xa * ny + yb) * nz + zg) * (size_t)N;
                double W[10];
                W[0] = wx[a] * wy[b] * wz[g];    /* v   */
                W[1] = dwx[a] * wy[b] * wz[g];   /* gx  */
                W[2] = wx[a] * dwy[b] * wz[g];   /* gy  */
                W[3] = wx[a] * wy[b] * dwz[g];   /* gz  */
                W[4] = d2wx[a] * wy[b] * wz[g];  /* hxx */
                W[5] = dwx[a] * dwy[b] * wz[g];  /* hxy */
                W[6] = dwx[a] * wy[b] * dwz[g];  /* hxz */
                W[7] = wx[a] * d2wy[b] * wz[g];  /* hyy */
                W[8] = wx[a] * dwy[b] * dwz[g];  /* hyz */
                W[9] = wx[a] * wy[b] * d2wz[g];  /* hzz */
                for (int q = 0; q < 10; ++q) {
                    double *hq = h + (size_t)q * N;
                    for (long j = 0; j < N; ++j) hq[j] += W[q] * c[j];
                }
            }
        }
    }
}

/* The value sum alone (the Bspline-v form), written to v[N]. */
static void window_sum_v(int nx, int ny, int nz, long N, const double *coefs,
                         const double pos[3], double *v)
{
    long ix, iy, iz;
    double tx, ty, tz;
    reduce_coordinate(pos[0], nx, &ix, &tx);
    reduce_coordinate(pos[1], ny, &iy, &ty);
    reduce_coordinate(pos[2], nz, &iz, &tz);
    double wx[4], dwx[4], d2wx[4];
    double wy[4], dwy[4], d2wy[4];
    double wz[4], dwz[4], d2wz[4];
    basis_weights(tx, nx, wx, dwx, d2wx);
    basis_weights(ty, ny, wy, dwy, d2wy);
    basis_weights(tz, nz, wz, dwz, d2wz);

    for (long j = 0; j < N; ++j) v[j] = 0.0;
    for (int a = 0; a < 4; ++a) {
        long xa = (ix + a - 1 + nx) % nx;
        for (int b = 0; b < 4; ++b) {
            long yb = (iy + b - 1 + ny) % ny;
            for (int g = 0; g < 4; ++g) {
                long zg = (iz + g - 1 + nz) % nz;
                const double *c = coefs + (((size_t)xa * ny + yb) * nz + zg) * (size_t)N;
                double W = wx[a] * wy[b] * wz[g];
                for (long j = 0; j < N; ++j) v[j] += W * c[j];
            }
        }
    }
}

/* Evaluate all N orbitals at P positions.  Returns 0 on success, -1 on bad
 * arguments, -2 if scratch memory for the VGL form cannot be had.
 * nthreads <= 0 uses the OpenMP default. */
int oracle_spo_eval(int nx, int ny, int nz, long N, const double *coefs,
                    long P, const double *pos, int kind, double *out,
                    int nthreads)
{
    if (nx < 4 || ny < 4 || nz < 4 || N < 0 || P < 0 || kind < 0 || kind > 2)
        return -1;
    if (P == 0 || N == 0) return 0;
    if (!coefs || !pos || !out) return -1;
    const int nc = n_components(kind);
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *h = NULL;
        if (kind == 1) {
            h = (double *)malloc(sizeof(double) * 10 * (size_t)N);
            if (!h) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                failed = 1;
            }
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (long p = 0; p < P; ++p) {
            double *o = out + (size_t)p * nc * N;
            if (kind == 0) {
                window_sum_v(nx, ny, nz, N, coefs, pos + 3 * p, o);
            } else if (kind == 2) {
                window_sums_vgh(nx, ny, nz, N, coefs, pos + 3 * p, o);
            } else if (h) {
                /* SPO-vgl form: v, gradient, and the Laplacian as the trace
                 * of the Hessian, lap = hxx + hyy + hzz */
                window_sums_vgh(nx, ny, nz, N, coefs, pos + 3 * p, h);
                for (long j = 0; j < N; ++j) {
                    o[0 * N + j] = h[0 * N + j];
                    o[1 * N + j] = h[1 * N + j];
                    o[2 * N + j] = h[2 * N + j];
                    o[3 * N + j] = h[3 * N + j];
                    o[4 * N + j] = h[4 * N + j] + h[7 * N + j] + h[9 * N + j];
                }
            }
        }
        free(h);
    }
    return failed ? -2 : 0;
}

/* Condition sums beta_q = sum over the window of |W_q| |c| for the ten VGH
 * components, [P][10][N].  They scale the rounding-error bound of any
 * evaluation of the same sums (a sum of 64 products computed in precision u
 * errs by at most about 64 u beta_q).  Same window and weights as above. */
int oracle_spo_condition(int nx, int ny, int nz, long N, const double *coefs,
                         long P, const double *pos, double *out, int nthreads)
{
    if (nx < 4 || ny < 4 || nz < 4 || N < 0 || P < 0) return -1;
    if (P == 0 || N == 0) return 0;
    if (!coefs || !pos || !out) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (long p = 0; p < P; ++p) {
        long ix, iy, iz;
        double tx, ty, tz;
        reduce_coordinate(pos[3 * p + 0], nx, &ix, &tx);
        reduce_coordinate(pos[3 * p + 1], ny, &iy, &ty);
        reduce_coordinate(pos[3 * p + 2], nz, &iz, &tz);
        double wx[4], dwx[4], d2wx[4];
        double wy[4], dwy[4], d2wy[4];
        double wz[4], dwz[4], d2wz[4];
        basis_weights(tx, nx, wx, dwx, d2wx);
        basis_weights(ty, ny, wy, dwy, d2wy);
        basis_weights(tz, nz, wz, dwz, d2wz);
        double *h = out + (size_t)p * 10 * N;
        for (long k = 0; k < 10 * N; ++k) h[k] = 0.0;
        for (int a = 0; a < 4; ++a) {
            long xa = (ix + a - 1 + nx) % nx;
            for (int b = 0; b < 4; ++b) {
                long yb = (iy + b - 1 + ny) % ny;
                for (int g = 0; g < 4; ++g) {
                    long zg = (iz + g - 1 + nz) % nz;
                    const double *c = coefs + (((size_t)xa * ny + yb) * nz + zg) * (size_t)N;
                    double W[10];
                    W[0] = wx[a] * wy[b] * wz[g];
                    W[1] = dwx[a] * wy[b] * wz[g];
                    W[2] = wx[a] * dwy[b] * wz[g];
                    W[3] = wx[a] * wy[b] * dwz[g];
                    W[4] = d2wx[a] * wy[b] * wz[g];
                    W[5] = dwx[a] * dwy[b] * wz[g];
                    W[6] = dwx[a] * wy[b] * dwz[g];
                    W[7] = wx[a] * d2wy[b] * wz[g];
                    W[8] = wx[a] * dwy[b] * dwz[g];
                    W[9] = wx[a] * wy[b] * d2wz[g];
                    for (int q = 0; q < 10; ++q) {
                        double *hq = h + (size_t)q * N;
                        double aw = fabs(W[q]);
                        for (long j = 0; j < N; ++j) hq[j] += aw * fabs(c[j]);
                    }
                }
            }
        }
    }
    return 0;
}

/* number of OpenMP threads a parallel region of this library would use */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
