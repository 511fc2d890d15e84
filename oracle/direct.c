/*
 * Oracle O1: the plain O(N M) direct sum of Eq. (2) ("FEM-direct").
 *
 * Test infrastructure only: the CUDA library never links or calls this file.
 *
 *   phi(x_i)  = sum_{j : y_j != x_i} q_j G(x_i - y_j),   G(d) = -(1/2 pi) log |d|
 *   H(x_i)    = -grad phi(x_i) = (1/2 pi) sum_j q_j d / |d|^2,   d = x_i - y_j
 *   Hess(x_i) = grad grad phi(x_i) = -(1/2 pi) sum_j q_j (I |d|^2 - 2 d d^T) / |d|^4
 *
 * Coincident pairs (d = 0) are skipped: G(0) := 0, grad G(0) := 0.
 * Positions are interleaved (x, y) pairs in FP64; plain FP64 accumulation,
 * one OpenMP thread per block of targets.
 */
#include <math.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

int o1_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* phi (n_tgt), field (n_tgt x 2) and hess (n_tgt x 3: xx, xy, yy) may each be NULL. */
void o1_direct(const double *tgt, long n_tgt, const double *src, long n_src,
               const double *q, double *phi, double *field, double *hess)
{
    const double inv2pi = 1.0 / (2.0 * ORACLE_PI);
    long i;
#pragma omp parallel for schedule(dynamic, 8)
    for (i = 0; i < n_tgt; ++i) {
        const double xi = tgt[2 * i], yi = tgt[2 * i + 1];
        double p = 0.0, hx = 0.0, hy = 0.0, hxx = 0.0, hxy = 0.0, hyy = 0.0;
        long j;
        for (j = 0; j < n_src; ++j) {
            const double dx = xi - src[2 * j];
            const double dy = yi - src[2 * j + 1];
            const double r2 = dx * dx + dy * dy;
            if (r2 == 0.0)
                continue;
            const double qj = q[j];
            p += qj * (-0.5 * log(r2) * inv2pi);
            const double c = qj * inv2pi / r2;
            hx += c * dx;
            hy += c * dy;
            if (hess) {
                const double c2 = c / r2;
                hxx += -c2 * (r2 - 2.0 * dx * dx);
                hxy += -c2 * (-2.0 * dx * dy);
                hyy += -c2 * (r2 - 2.0 * dy * dy);
            }
        }
        if (phi)
            phi[i] = p;
        if (field) {
            field[2 * i] = hx;
            field[2 * i + 1] = hy;
        }
        if (hess) {
            hess[3 * i] = hxx;
            hess[3 * i + 1] = hxy;
            hess[3 * i + 2] = hyy;
        }
    }
}
