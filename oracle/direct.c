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

/*
 * Adjoint of the direct sum for a loss L(phi, H) with gphi = dL/dphi (n_tgt) and
 * gH = dL/dH (n_tgt x 2), all FP64:
 *   A(y)      = sum_i gphi_i G(x_i - y) - sum_i gH_i . grad G(x_i - y)
 *   dL/dq_j   = A(y_j)
 *   dL/dy_j   = q_j grad A(y_j) = q_j sum_i [ -gphi_i grad G(x_i - y_j) + Hess G(x_i - y_j) gH_i ]
 *   dL/dx_i   = -gphi_i H(x_i) - Hess phi(x_i) gH_i
 * with grad G(d) = -(1/2pi) d / |d|^2, Hess G(d) = -(1/2pi) (I |d|^2 - 2 d d^T) / |d|^4,
 * coincident pairs skipped.  dq (n_src), dy (n_src x 2), dx (n_tgt x 2) may each be NULL.
 */
void o1_adjoint(const double *tgt, long n_tgt, const double *src, long n_src, const double *q,
                const double *gphi, const double *gH, double *dq, double *dy, double *dx)
{
    const double inv2pi = 1.0 / (2.0 * ORACLE_PI);
    long j, i;
    if (dq || dy) {
#pragma omp parallel for schedule(dynamic, 8)
        for (j = 0; j < n_src; ++j) {
            const double yx = src[2 * j], yy = src[2 * j + 1];
            double a = 0.0, ax = 0.0, ay = 0.0;
            for (i = 0; i < n_tgt; ++i) {
                const double dx0 = tgt[2 * i] - yx, dy0 = tgt[2 * i + 1] - yy;
                const double r2 = dx0 * dx0 + dy0 * dy0;
                if (r2 == 0.0)
                    continue;
                const double g = -0.5 * log(r2) * inv2pi;
                const double gx = -inv2pi * dx0 / r2, gy = -inv2pi * dy0 / r2;   /* grad G(d) */
                const double c2 = -inv2pi / (r2 * r2);
                const double hxx = c2 * (r2 - 2.0 * dx0 * dx0), hxy = c2 * (-2.0 * dx0 * dy0);
                const double hyy = c2 * (r2 - 2.0 * dy0 * dy0);
                const double gp = gphi[i], hx = gH[2 * i], hy = gH[2 * i + 1];
                a += gp * g - (hx * gx + hy * gy);
                ax += -gp * gx + (hxx * hx + hxy * hy);
                ay += -gp * gy + (hxy * hx + hyy * hy);
            }
            if (dq)
                dq[j] = a;
            if (dy) {
                dy[2 * j] = q[j] * ax;
                dy[2 * j + 1] = q[j] * ay;
            }
        }
    }
    if (dx) {
#pragma omp parallel for schedule(dynamic, 8)
        for (i = 0; i < n_tgt; ++i) {
            const double xx = tgt[2 * i], xy = tgt[2 * i + 1];
            double Hx = 0.0, Hy = 0.0, pxx = 0.0, pxy = 0.0, pyy = 0.0;
            for (j = 0; j < n_src; ++j) {
                const double d0 = xx - src[2 * j], d1 = xy - src[2 * j + 1];
                const double r2 = d0 * d0 + d1 * d1;
                if (r2 == 0.0)
                    continue;
                const double c = q[j] * inv2pi / r2;
                Hx += c * d0;
                Hy += c * d1;
                const double c2 = -c / r2;
                pxx += c2 * (r2 - 2.0 * d0 * d0);
                pxy += c2 * (-2.0 * d0 * d1);
                pyy += c2 * (r2 - 2.0 * d1 * d1);
            }
            const double gp = gphi[i], hx = gH[2 * i], hy = gH[2 * i + 1];
            dx[2 * i] = -gp * Hx - (pxx * hx + pxy * hy);
            dx[2 * i + 1] = -gp * Hy - (pxy * hx + pyy * hy);
        }
    }
}
