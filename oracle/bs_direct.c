/*
 * Plain FP64 direct-sum oracle for the regularised 2-D Biot-Savart kernel.
 *
 * TEST INFRASTRUCTURE ONLY: the product path never calls this file.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg load it.
 *
 * Every routine is the textbook double loop over targets i and sources j,
 * written straight from the paper's definitions, with no blocking, fusion or
 * reordering.  OpenMP splits the outer target loop only (each target's sum
 * runs in source order, so results do not depend on the thread count).
 *
 * State layout (Sec. 2, Eq. 3): x = [chi_1..chi_n, psi_1..psi_n].
 * Kernel (Sec. 2, Eq. 2):
 *     f_i = sum_{j != i} Gamma_j/(2 pi) * e3 x (x_i - x_j) / (|x_i - x_j|^2 + delta)
 * with e3 x (a, b) = (-b, a).  A pair with |x_i - x_j| == 0 is the j == i
 * term of Eq. 1 (or a coincident body) and is skipped.
 *
 * Jacobian block of one pair (derivative of K(r) = (-b, a)/s, s = a^2+b^2+delta,
 * with respect to r = (a, b)):
 *     A(r) = [[ 2ab/s^2,       -1/s + 2b^2/s^2 ],
 *             [ 1/s - 2a^2/s^2, -2ab/s^2       ]]
 * so d f_i / d x_i = D_i = sum_{j!=i} gamma_j A(r_ij) and, for k != i,
 * d f_i / d x_k = -gamma_k A(r_ik), with gamma = Gamma / (2 pi) (Eq. 4).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_TWO_PI 6.283185307179586476925286766559

/* A(r) for r = (a, b); out[0..3] = A00, A01, A10, A11 */
static void pair_block(double a, double b, double delta, double out[4]) {
    double s = a * a + b * b + delta;
    double s2 = s * s;
    out[0] = 2.0 * a * b / s2;
    out[1] = -1.0 / s + 2.0 * b * b / s2;
    out[2] = 1.0 / s - 2.0 * a * a / s2;
    out[3] = -2.0 * a * b / s2;
}

/* Velocity of nt targets induced by ns sources (Eq. 2).  D (3*nt, optional):
 * the per-target self block d f_i/d x_i stored as [D00 (nt), D01 (nt), D10 (nt)]
 * (D11 = -D00: the block is trace-free). */
void or_velocity(int nt, const double *xt, int ns, const double *xs,
                 const double *Gamma, double delta, double *f, double *D) {
    int i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < nt; ++i) {
        double u = 0.0, v = 0.0, d00 = 0.0, d01 = 0.0, d10 = 0.0;
        for (int j = 0; j < ns; ++j) {
            double a = xt[i] - xs[j];
            double b = xt[nt + i] - xs[ns + j];
            if (a == 0.0 && b == 0.0) continue;
            double g = Gamma[j] / OR_TWO_PI;
            double s = a * a + b * b + delta;
            u += g * (-b) / s;
            v += g * a / s;
            if (D) {
                double A[4];
                pair_block(a, b, delta, A);
                d00 += g * A[0];
                d01 += g * A[1];
                d10 += g * A[2];
            }
        }
        f[i] = u;
        f[nt + i] = v;
        if (D) {
            D[i] = d00;
            D[nt + i] = d01;
            D[2 * nt + i] = d10;
        }
    }
}

/* J v with J = d f / d x (all blocks, Sec. 3.2 Jacobian of the kernel):
 * (J v)_i = D_i v_i + sum_{j != i} (-gamma_j A(x_i - x_j)) v_j.
 * or_jvp_rows evaluates only the rows (bodies) listed in rows[0..nrows). */
void or_jvp_rows(int n, const double *x, const double *Gamma, double delta,
                 const double *v, const int *rows, int nrows, double *jv) {
    int r;
#pragma omp parallel for schedule(static)
    for (r = 0; r < nrows; ++r) {
        int i = rows[r];
        double D[4] = {0.0, 0.0, 0.0, 0.0};
        double off0 = 0.0, off1 = 0.0;
        for (int j = 0; j < n; ++j) {
            double a = x[i] - x[j];
            double b = x[n + i] - x[n + j];
            if (a == 0.0 && b == 0.0) continue;
            double g = Gamma[j] / OR_TWO_PI;
            double A[4];
            pair_block(a, b, delta, A);
            for (int e = 0; e < 4; ++e) D[e] += g * A[e];
            off0 += -g * (A[0] * v[j] + A[1] * v[n + j]);
            off1 += -g * (A[2] * v[j] + A[3] * v[n + j]);
        }
        jv[r] = D[0] * v[i] + D[1] * v[n + i] + off0;
        jv[nrows + r] = D[2] * v[i] + D[3] * v[n + i] + off1;
    }
}

void or_jvp(int n, const double *x, const double *Gamma, double delta,
            const double *v, double *jv) {
    int *rows = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) rows[i] = i;
    or_jvp_rows(n, x, Gamma, delta, v, rows, n, jv);
    free(rows);
}

/* Transposed products.
 * gx (2n, optional):  (J^T w)_k = sum_i (d f_i / d x_k)^T w_i
 *                              = D_k^T w_k + sum_{i != k} (-gamma_k A(x_i - x_k))^T w_i
 * gG (n, optional):   (d f / d Gamma)^T w, i.e.
 *                     gG_k = sum_{i != k} w_i . (1/(2 pi)) e3 x (x_i - x_k) / s_ik */
void or_vjp_rows(int n, const double *x, const double *Gamma, double delta,
                 const double *w, const int *rows, int nrows, double *gx, double *gG) {
    int r;
#pragma omp parallel for schedule(static)
    for (r = 0; r < nrows; ++r) {
        int k = rows[r];
        double D[4] = {0.0, 0.0, 0.0, 0.0};
        double t0 = 0.0, t1 = 0.0, gg = 0.0;
        double gk = Gamma[k] / OR_TWO_PI;
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            /* self block of k: pairs (k, i) */
            double a = x[k] - x[i];
            double b = x[n + k] - x[n + i];
            if (a == 0.0 && b == 0.0) continue;
            double A[4];
            pair_block(a, b, delta, A);
            double gi = Gamma[i] / OR_TWO_PI;
            for (int e = 0; e < 4; ++e) D[e] += gi * A[e];
            /* block d f_i / d x_k = -gamma_k A(x_i - x_k) */
            double Ai[4];
            pair_block(-a, -b, delta, Ai);
            t0 += -gk * (Ai[0] * w[i] + Ai[2] * w[n + i]);
            t1 += -gk * (Ai[1] * w[i] + Ai[3] * w[n + i]);
            /* d f_i / d Gamma_k = (1/2pi) e3 x (x_i - x_k) / s */
            double s = a * a + b * b + delta;
            gg += (w[i] * (b) + w[n + i] * (-a)) / (OR_TWO_PI * s);
        }
        if (gx) {
            gx[r] = D[0] * w[k] + D[2] * w[n + k] + t0;
            gx[nrows + r] = D[1] * w[k] + D[3] * w[n + k] + t1;
        }
        if (gG) gG[r] = gg;
    }
}

void or_vjp(int n, const double *x, const double *Gamma, double delta,
            const double *w, double *gx, double *gG) {
    int *rows = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) rows[i] = i;
    or_vjp_rows(n, x, Gamma, delta, w, rows, n, gx, gG);
    free(rows);
}

/* J Phi for an (2n x M) column-major basis: each column is one J v product. */
void or_jphi(int n, const double *x, const double *Gamma, double delta,
             const double *phi, int M, double *out) {
    for (int m = 0; m < M; ++m)
        or_jvp(n, x, Gamma, delta, phi + (size_t)m * 2 * n, out + (size_t)m * 2 * n);
}

/* Number of OpenMP threads a parallel region gets (1 when built without). */
int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
