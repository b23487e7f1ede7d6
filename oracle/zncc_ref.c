/*
 * CPU FP64 oracle for zero-mean normalised cross-correlation template search.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it exists so that tests, the smoke check and the bench's
 * CPU-baseline leg can compare the GPU library against a plain, slow and
 * obviously correct statement of what it computes.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Every routine is the literal definition, written out in double precision
 * with no blocking, no running sums and no reordering beyond the order of
 * the sums in the definition:
 *
 *   rho(a, b) = sum (a - mu_a)(b - mu_b) / (sigma_a sigma_b),
 *   sigma_a   = sqrt(sum (a - mu_a)^2)            (Section 1, Eq. rho1)
 *
 * Convention where the paper is silent: rho := 0 when either block is
 * flat (sigma == 0).
 *
 * Images are row-major double arrays with a row stride `ld` (elements).
 * Locations are window top-left corners (y, x), y in [0, p-m], x in [0, q-n].
 * OpenMP parallelises over independent locations only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* rho between the m x n window of A at (ya, xa) and of B at (yb, xb). */
double oracle_window_rho(const double *A, int64_t lda, const double *B, int64_t ldb,
                         int m, int n, int ya, int xa, int yb, int xb)
{
    const double mn = (double)m * (double)n;
    double sa = 0.0, sb = 0.0;
    for (int u = 0; u < m; ++u)
        for (int v = 0; v < n; ++v) {
            sa += A[(int64_t)(ya + u) * lda + xa + v];
            sb += B[(int64_t)(yb + u) * ldb + xb + v];
        }
    const double mua = sa / mn, mub = sb / mn;
    double num = 0.0, va = 0.0, vb = 0.0;
    for (int u = 0; u < m; ++u)
        for (int v = 0; v < n; ++v) {
            const double da = A[(int64_t)(ya + u) * lda + xa + v] - mua;
            const double db = B[(int64_t)(yb + u) * ldb + xb + v] - mub;
            num += da * db;
            va += da * da;
            vb += db * db;
        }
    if (va == 0.0 || vb == 0.0) return 0.0;
    return num / (sqrt(va) * sqrt(vb));
}

/* rho(t, I window at (y, x)) for every location; rho_out is (p-m+1) x (q-n+1). */
void oracle_zncc_map(const double *I, int64_t ld, int p, int q,
                     const double *t, int m, int n, double *rho_out, int nthreads)
{
    const int Ly = p - m + 1, Lx = q - n + 1;
    if (Ly <= 0 || Lx <= 0) return;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x)
            rho_out[(int64_t)y * Lx + x] = oracle_window_rho(t, n, I, ld, m, n, 0, 0, y, x);
}

/* rho(t, I window) at k listed locations ys[i], xs[i]. */
void oracle_rho_at(const double *I, int64_t ld, const double *t, int m, int n,
                   const int *ys, const int *xs, int k, double *out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < k; ++i)
        out[i] = oracle_window_rho(t, n, I, ld, m, n, 0, 0, ys[i], xs[i]);
}

/* Blur-correlation R_oo(x) = rho(P window at x, I window at x) (Algorithm 3). */
void oracle_blur_corr_map(const double *P, const double *I, int64_t ld, int p, int q,
                          int m, int n, double *out, int nthreads)
{
    const int Ly = p - m + 1, Lx = q - n + 1;
    if (Ly <= 0 || Lx <= 0) return;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x)
            out[(int64_t)y * Lx + x] = oracle_window_rho(P, ld, I, ld, m, n, y, x, y, x);
}

/* Centre of the group that covers location coordinate `c` along an axis of
 * `len` locations with group size h: groups tile the location grid from 0,
 * the last one may be truncated, and the centre is start + (size-1)/2. */
static int group_centre(int c, int len, int h)
{
    const int start = (c / h) * h;
    int size = len - start;
    if (size > h) size = h;
    return start + (size - 1) / 2;
}

/* rho_co(x) = rho(P window at centre(x), I window at x) for every location
 * (Algorithm 1, with the pivot block read from P). */
void oracle_rho_co_map(const double *P, const double *I, int64_t ld, int p, int q,
                       int m, int n, int h, double *out, int nthreads)
{
    const int Ly = p - m + 1, Lx = q - n + 1;
    if (Ly <= 0 || Lx <= 0) return;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < Ly; ++y) {
        const int cy = group_centre(y, Ly, h);
        for (int x = 0; x < Lx; ++x) {
            const int cx = group_centre(x, Lx, h);
            out[(int64_t)y * Lx + x] = oracle_window_rho(P, ld, I, ld, m, n, cy, cx, y, x);
        }
    }
}

/* Spatially varying Gaussian blur, Eq. defblur with Gaussian weights
 * (Eq. Gauss, read with the minus sign in the exponent):
 *   out(y,x) = sum_{i,j=-d..d} w(i,j) I(clamp(y+i), clamp(x+j)),
 *   w(i,j) = exp(-(i^2+j^2)/(2 s^2)) / alpha,   d = ceil(3 s),
 * where s = sigma of the block that contains the output pixel
 * (sigma_map is (ceil(p/block) x ceil(q/block)), row-major) and alpha makes
 * the weights sum to one.  s == 0 copies the pixel.  Borders clamp to edge. */
void oracle_blur(const double *I, int64_t ld, int p, int q, const double *sigma_map,
                 int block, double *out, int nthreads)
{
    const int bq = (q + block - 1) / block;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < p; ++y) {
        for (int x = 0; x < q; ++x) {
            const double s = sigma_map[(int64_t)(y / block) * bq + (x / block)];
            if (s <= 0.0) { out[(int64_t)y * q + x] = I[(int64_t)y * ld + x]; continue; }
            const int d = (int)ceil(3.0 * s);
            double acc = 0.0, alpha = 0.0;
            for (int i = -d; i <= d; ++i) {
                int yy = y + i; if (yy < 0) yy = 0; if (yy > p - 1) yy = p - 1;
                for (int j = -d; j <= d; ++j) {
                    int xx = x + j; if (xx < 0) xx = 0; if (xx > q - 1) xx = q - 1;
                    const double w = exp(-((double)(i * i + j * j)) / (2.0 * s * s));
                    alpha += w;
                    acc += w * I[(int64_t)yy * ld + xx];
                }
            }
            out[(int64_t)y * q + x] = acc / alpha;
        }
    }
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
