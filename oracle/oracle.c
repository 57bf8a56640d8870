/*
 * CPU oracle for repeated star-stencil sweeps -- TEST INFRASTRUCTURE.
 *
 * Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs
 * of bench.py load this file's library.  It shares no code with the CUDA
 * path and is never called by the product.
 *
 * What it computes (Zohouri, Podobas, Matsuoka, "High-Performance High-Order
 * Stencil Computation on FPGAs Using OpenCL", Section IV.A, Eq. 1): one
 * Jacobi step of a star stencil of radius r,
 *
 *   g(p) = c_c f(p) + sum_{i=1..r} ( c_{W,i} f(p - i ex) + c_{E,i} f(p + i ex)
 *                                  + c_{S,i} f(p - i ey) + c_{N,i} f(p + i ey)
 *                                  [+ c_{B,i} f(p - i ez) + c_{A,i} f(p + i ez)] )
 *
 * with one coefficient per (direction, distance) -- the paper's worst case
 * in which no coefficient is shared (Section IV.A) -- repeated `iters`
 * times.  Out-of-bound neighbours fall back on the border cell (clamp to
 * edge, Section III.B and Section IV.B), at every time step.
 *
 * Readings taken where the paper is silent or garbled:
 *  - Eq. 1 prints the sum from i = 0; the sum runs i = 1..rad, which is what
 *    the FLOP count 12*rad + 1 (3D) / 8*rad + 1 (2D) of Table I requires.
 *  - The paper forbids reordering the floating-point operations (Section
 *    IV.A) but fixes no order; the order here is the left-to-right order of
 *    Eq. 1: centre, then for i = 1..r the directions W, E, S, N, B, A.
 *  - W = -x, E = +x, S = -y, N = +y, B = -z, A = +z.
 *  - Coefficient layout: c[0] = centre, c[1 + (i-1)*2*dim + d], d = W..A.
 *
 * Two arithmetic variants:
 *  - oracle_sweep_f64: promoted to double, one multiply then plain adds
 *    (built with -ffp-contract=off so no add is fused).
 *  - oracle_sweep_f32: single precision, one rounded multiply for the
 *    centre and then one fused multiply-add (fmaf) per neighbour in the same
 *    order -- the multiply-then-FMA chain of Section V.A (each
 *    multiplication fused with the addition that follows it).
 *
 * Shared-coefficient form (one coefficient per distance, the stencils the
 * paper compares against in Section IV.C; Sections IV.A and V.A note that
 * sharing removes multiplications but not additions):
 *
 *   g(p) = c_0 f(p) + sum_{i=1..r} c_i * (f(W,i) + f(E,i) + f(S,i) + f(N,i) [+ f(B,i) + f(A,i)])
 *
 * Reordering is allowed for this form and the paper gives no order; the
 * order here: the 2*dim neighbours at distance i summed left to right (W, E,
 * S, N, B, A), then acc + c_i * sum.  oracle_sweep_shared_f64 uses plain
 * double multiplies and adds; oracle_sweep_shared_f32 uses single-precision
 * adds for the sum and one fmaf per distance.  Coefficients c[0..r].
 *
 * Grid layout: x fastest, element (x, y, z) at x + nx*(y + ny*z); 2D uses
 * nz = 1 and dim = 2.  The sweep is a plain triple loop per time step over
 * a ping-pong buffer; OpenMP only splits the (z, y) rows across threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline int64_t clamp_index(int64_t i, int64_t n)
{
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

#define IDX(x, y, z) ((x) + nx * ((y) + ny * (z)))

static void step_f64(const double *f, double *g, int64_t nx, int64_t ny, int64_t nz,
                     int dim, int r, const double *c)
{
    int64_t rows = ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t y = row % ny, z = row / ny;
        for (int64_t x = 0; x < nx; ++x) {
            double acc = c[0] * f[IDX(x, y, z)];
            for (int i = 1; i <= r; ++i) {
                const double *ci = c + 1 + (i - 1) * 2 * dim;
                acc = acc + ci[0] * f[IDX(clamp_index(x - i, nx), y, z)];
                acc = acc + ci[1] * f[IDX(clamp_index(x + i, nx), y, z)];
                acc = acc + ci[2] * f[IDX(x, clamp_index(y - i, ny), z)];
                acc = acc + ci[3] * f[IDX(x, clamp_index(y + i, ny), z)];
                if (dim == 3) {
                    acc = acc + ci[4] * f[IDX(x, y, clamp_index(z - i, nz))];
                    acc = acc + ci[5] * f[IDX(x, y, clamp_index(z + i, nz))];
                }
            }
            g[IDX(x, y, z)] = acc;
        }
    }
}

static void step_f32(const float *f, float *g, int64_t nx, int64_t ny, int64_t nz,
                     int dim, int r, const float *c)
{
    int64_t rows = ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t y = row % ny, z = row / ny;
        for (int64_t x = 0; x < nx; ++x) {
            float acc = c[0] * f[IDX(x, y, z)];
            for (int i = 1; i <= r; ++i) {
                const float *ci = c + 1 + (i - 1) * 2 * dim;
                acc = fmaf(ci[0], f[IDX(clamp_index(x - i, nx), y, z)], acc);
                acc = fmaf(ci[1], f[IDX(clamp_index(x + i, nx), y, z)], acc);
                acc = fmaf(ci[2], f[IDX(x, clamp_index(y - i, ny), z)], acc);
                acc = fmaf(ci[3], f[IDX(x, clamp_index(y + i, ny), z)], acc);
                if (dim == 3) {
                    acc = fmaf(ci[4], f[IDX(x, y, clamp_index(z - i, nz))], acc);
                    acc = fmaf(ci[5], f[IDX(x, y, clamp_index(z + i, nz))], acc);
                }
            }
            g[IDX(x, y, z)] = acc;
        }
    }
}

static void step_shared_f64(const double *f, double *g, int64_t nx, int64_t ny, int64_t nz,
                            int dim, int r, const double *c)
{
    int64_t rows = ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t y = row % ny, z = row / ny;
        for (int64_t x = 0; x < nx; ++x) {
            double acc = c[0] * f[IDX(x, y, z)];
            for (int i = 1; i <= r; ++i) {
                double sum = f[IDX(clamp_index(x - i, nx), y, z)] + f[IDX(clamp_index(x + i, nx), y, z)];
                sum = sum + f[IDX(x, clamp_index(y - i, ny), z)];
                sum = sum + f[IDX(x, clamp_index(y + i, ny), z)];
                if (dim == 3) {
                    sum = sum + f[IDX(x, y, clamp_index(z - i, nz))];
                    sum = sum + f[IDX(x, y, clamp_index(z + i, nz))];
                }
                acc = acc + c[i] * sum;
            }
            g[IDX(x, y, z)] = acc;
        }
    }
}

static void step_shared_f32(const float *f, float *g, int64_t nx, int64_t ny, int64_t nz,
                            int dim, int r, const float *c)
{
    int64_t rows = ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t y = row % ny, z = row / ny;
        for (int64_t x = 0; x < nx; ++x) {
            float acc = c[0] * f[IDX(x, y, z)];
            for (int i = 1; i <= r; ++i) {
                float sum = f[IDX(clamp_index(x - i, nx), y, z)] + f[IDX(clamp_index(x + i, nx), y, z)];
                sum = sum + f[IDX(x, clamp_index(y - i, ny), z)];
                sum = sum + f[IDX(x, clamp_index(y + i, ny), z)];
                if (dim == 3) {
                    sum = sum + f[IDX(x, y, clamp_index(z - i, nz))];
                    sum = sum + f[IDX(x, y, clamp_index(z + i, nz))];
                }
                acc = fmaf(c[i], sum, acc);
            }
            g[IDX(x, y, z)] = acc;
        }
    }
}

static int check_args(int64_t nx, int64_t ny, int64_t nz, int dim, int r, int iters)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || iters < 0) return -1;
    if (dim != 2 && dim != 3) return -1;
    if (dim == 2 && nz != 1) return -1;
    if (r < 1) return -1;
    return 0;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Returns 0 on success, -1 on bad arguments, -2 on allocation failure. */
int oracle_sweep_f64(const double *in, double *out, int64_t nx, int64_t ny, int64_t nz,
                     int dim, int r, const double *c, int iters, int nthreads)
{
    if (check_args(nx, ny, nz, dim, r, iters)) return -1;
    int64_t n = nx * ny * nz;
    set_threads(nthreads);
    if (iters == 0) { memcpy(out, in, (size_t)n * sizeof(double)); return 0; }
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!tmp) return -2;
    /* ping-pong so that the last step writes `out` */
    const double *src = in;
    for (int s = 0; s < iters; ++s) {
        double *dst = ((iters - 1 - s) % 2 == 0) ? out : tmp;
        step_f64(src, dst, nx, ny, nz, dim, r, c);
        src = dst;
    }
    free(tmp);
    return 0;
}

int oracle_sweep_f32(const float *in, float *out, int64_t nx, int64_t ny, int64_t nz,
                     int dim, int r, const float *c, int iters, int nthreads)
{
    if (check_args(nx, ny, nz, dim, r, iters)) return -1;
    int64_t n = nx * ny * nz;
    set_threads(nthreads);
    if (iters == 0) { memcpy(out, in, (size_t)n * sizeof(float)); return 0; }
    float *tmp = (float *)malloc((size_t)n * sizeof(float));
    if (!tmp) return -2;
    const float *src = in;
    for (int s = 0; s < iters; ++s) {
        float *dst = ((iters - 1 - s) % 2 == 0) ? out : tmp;
        step_f32(src, dst, nx, ny, nz, dim, r, c);
        src = dst;
    }
    free(tmp);
    return 0;
}

int oracle_sweep_shared_f64(const double *in, double *out, int64_t nx, int64_t ny, int64_t nz,
                            int dim, int r, const double *c, int iters, int nthreads)
{
    if (check_args(nx, ny, nz, dim, r, iters)) return -1;
    int64_t n = nx * ny * nz;
    set_threads(nthreads);
    if (iters == 0) { memcpy(out, in, (size_t)n * sizeof(double)); return 0; }
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!tmp) return -2;
    const double *src = in;
    for (int s = 0; s < iters; ++s) {
        double *dst = ((iters - 1 - s) % 2 == 0) ? out : tmp;
        step_shared_f64(src, dst, nx, ny, nz, dim, r, c);
        src = dst;
    }
    free(tmp);
    return 0;
}

int oracle_sweep_shared_f32(const float *in, float *out, int64_t nx, int64_t ny, int64_t nz,
                            int dim, int r, const float *c, int iters, int nthreads)
{
    if (check_args(nx, ny, nz, dim, r, iters)) return -1;
    int64_t n = nx * ny * nz;
    set_threads(nthreads);
    if (iters == 0) { memcpy(out, in, (size_t)n * sizeof(float)); return 0; }
    float *tmp = (float *)malloc((size_t)n * sizeof(float));
    if (!tmp) return -2;
    const float *src = in;
    for (int s = 0; s < iters; ++s) {
        float *dst = ((iters - 1 - s) % 2 == 0) ? out : tmp;
        step_shared_f32(src, dst, nx, ny, nz, dim, r, c);
        src = dst;
    }
    free(tmp);
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
