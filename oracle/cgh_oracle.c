/*
 * cgh_oracle.c -- plain, slow, obviously correct CPU oracle for the
 * point-source Fresnel computer-generated hologram.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (Shimobaba et al., Section 1, Eq. 1):
 *
 *     I(x_h, y_h) = sum_j A_j cos( P_j ((x_h - x_j)^2 + (y_h - y_j)^2) ),
 *     P_j = pi p^2 / (lambda z_j),
 *
 * with (x_h, y_h) and (x_j, y_j) in units of the pixel pitch p.  Readings of
 * what the paper leaves open: pixel (x_h, y_h) is the integer array index
 * (x_h in 0..Nx-1, y_h in 0..Ny-1, no centring); the output is row-major
 * out[y_h * Nx + x_h]; no post-processing (I may be negative).
 *
 * Precision: FP64 throughout.  oracle_forward reduces the phase in turns,
 * t = Q_j r^2 with Q_j = P_j / (2 pi) = p^2 / (2 lambda z_j), f = t - rint(t),
 * before cos(2 pi f): this keeps the argument in [-pi, pi] so that libm's cos
 * works on a small argument.  oracle_forward_ld evaluates the paper's form
 * P_j r^2 unreduced in long double (brute force).  oracle_forward_recurrence
 * is the paper's Eq. 2 recurrence (Section 2.1) along each row, in radians.
 *
 * Adjoint (derivatives of Eq. 1; phi = P_j r^2, dx = x_h - x_j,
 * dy = y_h - y_j, dP_j/dz_j = -P_j / z_j):
 *     dI/dA_j =  cos phi
 *     dI/dx_j =  2 P_j A_j sin(phi) dx
 *     dI/dy_j =  2 P_j A_j sin(phi) dy
 *     dI/dz_j =  (P_j A_j / z_j) sin(phi) r^2
 * oracle_grad returns sum over pixels of G(x_h, y_h) times each of these,
 * with G = dL/dI supplied by the caller.
 *
 * Build: plain C99 + OpenMP, no fast-math, no FP contraction.
 */
#include <math.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_BAD_ARG 1

static const double TWO_PI = 6.283185307179586476925286766559;
static const long double PI_L = 3.14159265358979323846264338327950288L;

static int set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(int nthreads) { return set_threads(nthreads); }

/* Q_j = P_j / (2 pi) = p^2 / (2 lambda z_j): phase in turns per pixel^2. */
static double turns_per_px2(double p, double lambda, float zj)
{
    return (p * p) / (2.0 * lambda * (double)zj);
}

/*
 * Eq. 1 in FP64.  rows == NULL: all Ny rows, out is Ny*Nx.  Otherwise
 * out is nrows*Nx and row r of out holds hologram row rows[r].
 */
int oracle_forward(const float *xy, const float *A, const float *z, int N,
                   double lambda, double p, int Nx, int Ny,
                   const int *rows, int nrows, double *out, int nthreads)
{
    if (N < 0 || Nx <= 0 || Ny <= 0 || !out) return ORACLE_BAD_ARG;
    if (N > 0 && (!xy || !A || !z)) return ORACLE_BAD_ARG;
    int R = rows ? nrows : Ny;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < R; ++r) {
        int yh = rows ? rows[r] : r;
        double *orow = out + (size_t)r * (size_t)Nx;
        for (int xh = 0; xh < Nx; ++xh) {
            double acc = 0.0;
            for (int j = 0; j < N; ++j) {
                double dx = (double)xh - (double)xy[2 * j];
                double dy = (double)yh - (double)xy[2 * j + 1];
                double t = turns_per_px2(p, lambda, z[j]) * (dx * dx + dy * dy);
                double f = t - nearbyint(t);
                acc += (double)A[j] * cos(TWO_PI * f);
            }
            orow[xh] = acc;
        }
    }
    return ORACLE_OK;
}

/* Eq. 1 by brute force in long double, unreduced: A_j cosl(P_j r^2). */
int oracle_forward_ld(const float *xy, const float *A, const float *z, int N,
                      double lambda, double p, int Nx, int Ny, double *out)
{
    if (N < 0 || Nx <= 0 || Ny <= 0 || !out) return ORACLE_BAD_ARG;
    long double lam = (long double)lambda, pp = (long double)p;
    for (int yh = 0; yh < Ny; ++yh)
        for (int xh = 0; xh < Nx; ++xh) {
            long double acc = 0.0L;
            for (int j = 0; j < N; ++j) {
                long double Pj = PI_L * pp * pp / (lam * (long double)z[j]);
                long double dx = (long double)xh - (long double)xy[2 * j];
                long double dy = (long double)yh - (long double)xy[2 * j + 1];
                acc += (long double)A[j] * cosl(Pj * (dx * dx + dy * dy));
            }
            out[(size_t)yh * Nx + xh] = (double)acc;
        }
    return ORACLE_OK;
}

/*
 * Eq. 2 (Section 2.1): along a row, Gamma_n = Gamma_{n-1} + delta_{n-1},
 * delta_n = delta_{n-1} + Delta, with Gamma_0 = P_j r^2 at x_h = 0,
 * delta_0 = P_j (2 (0 - x_j) + 1), Delta = 2 P_j.  FP64 radians.
 * Same row selection as oracle_forward.
 */
int oracle_forward_recurrence(const float *xy, const float *A, const float *z,
                              int N, double lambda, double p, int Nx, int Ny,
                              const int *rows, int nrows, double *out,
                              int nthreads)
{
    if (N < 0 || Nx <= 0 || Ny <= 0 || !out) return ORACLE_BAD_ARG;
    int R = rows ? nrows : Ny;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < R; ++r) {
        int yh = rows ? rows[r] : r;
        double *orow = out + (size_t)r * (size_t)Nx;
        for (int xh = 0; xh < Nx; ++xh) orow[xh] = 0.0;
        for (int j = 0; j < N; ++j) {
            double Pj = M_PI * p * p / (lambda * (double)z[j]);
            double x0 = 0.0 - (double)xy[2 * j];
            double dy = (double)yh - (double)xy[2 * j + 1];
            double gamma = Pj * (x0 * x0 + dy * dy);
            double delta = Pj * (2.0 * x0 + 1.0);
            double Delta = 2.0 * Pj;
            for (int xh = 0; xh < Nx; ++xh) {
                orow[xh] += (double)A[j] * cos(gamma);
                gamma += delta;
                delta += Delta;
            }
        }
    }
    return ORACLE_OK;
}

/*
 * Adjoint of Eq. 1 in FP64.  G is Ny*Nx row-major (dL/dI).  pts == NULL:
 * all N points, outputs have N entries (gxy: 2N interleaved).  Otherwise
 * the outputs have npts entries for points pts[0..npts-1].
 */
int oracle_grad(const float *xy, const float *A, const float *z, int N,
                double lambda, double p, int Nx, int Ny, const double *G,
                const int *pts, int npts, double *gxy, double *gA, double *gz,
                int nthreads)
{
    if (N < 0 || Nx <= 0 || Ny <= 0 || !G || !gxy || !gA || !gz)
        return ORACLE_BAD_ARG;
    int M = pts ? npts : N;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int m = 0; m < M; ++m) {
        int j = pts ? pts[m] : m;
        double Q = turns_per_px2(p, lambda, z[j]);
        double Pj = TWO_PI * Q;
        double sc = 0.0, ssx = 0.0, ssy = 0.0, ssr = 0.0;
        for (int yh = 0; yh < Ny; ++yh) {
            double dy = (double)yh - (double)xy[2 * j + 1];
            const double *grow = G + (size_t)yh * (size_t)Nx;
            for (int xh = 0; xh < Nx; ++xh) {
                double dx = (double)xh - (double)xy[2 * j];
                double r2 = dx * dx + dy * dy;
                double t = Q * r2;
                double f = t - nearbyint(t);
                double g = grow[xh];
                double s = sin(TWO_PI * f);
                sc += g * cos(TWO_PI * f);
                ssx += g * s * dx;
                ssy += g * s * dy;
                ssr += g * s * r2;
            }
        }
        double Aj = (double)A[j];
        gA[m] = sc;
        gxy[2 * m] = 2.0 * Pj * Aj * ssx;
        gxy[2 * m + 1] = 2.0 * Pj * Aj * ssy;
        gz[m] = Pj * Aj / (double)z[j] * ssr;
    }
    return ORACLE_OK;
}
