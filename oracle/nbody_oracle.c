/*
 * Plain FP64 CPU oracle for direct-summation gravity.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only the test suite, the smoke check and the timed CPU
 * baseline in the benchmark use it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Everything is the plain definition, evaluated in double precision in the
 * obvious order (j ascending for every i), with no blocking, fusion or
 * reordering:
 *
 *   acceleration (Eq. 1 divided by m_i, Sec. 2.1), with Plummer softening
 *   (App. A adds a softening length to the pair distance without giving the
 *   form; read as r^2 + eps^2):
 *       a_i   =  G sum_{j != i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^{3/2}
 *   potential (not printed in the paper; the companion quantity of Eq. 1):
 *       phi_i = -G sum_{j != i} m_j / (|x_j - x_i|^2 + eps^2)^{1/2}
 *   kick-drift-kick leapfrog with fixed step h:
 *       v_{n+1/2} = v_n + (h/2) a(x_n)
 *       x_{n+1}   = x_n + h v_{n+1/2}
 *       v_{n+1}   = v_{n+1/2} + (h/2) a(x_{n+1})
 *   energy:  K = 1/2 sum m_i |v_i|^2,  W = 1/2 sum m_i phi_i,  E = K + W
 *   jerk (App. A, Algorithm 3): the time derivative of a_i along the motion,
 *       j_i = G sum_{j != i} m_j [ (v_j - v_i) / s^3 - 3 (d . (v_j - v_i)) d / s^5 ]
 *   fourth-order Hermite predictor-corrector (Sec. 2.1's predict, evaluate,
 *   correct cycle, at fourth rather than sixth order)
 *   force vector-Jacobian product, from the chain rule written out block by
 *   block (J_ik = d a_i / d x_k, a 3x3 matrix):
 *       xbar_k = sum_i J_ik^T abar_i + sum_i (d phi_i / d x_k) phibar_i
 *       mbar_k = sum_i (d a_i / d m_k) . abar_i + sum_i (d phi_i / d m_k) phibar_i
 *
 * With eps = 0 a pair at zero separation is singular; the oracle then skips
 * it (the same convention as excluding j = i).
 *
 * Arrays: pos/vel/acc/xbar are [N][3] row-major, mass/pot/phibar/mbar are [N].
 * OpenMP parallelises only the outer loop over the output index; each output
 * is still summed serially in the order above, so results do not depend on the
 * thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* One row i of the definition: a_i and phi_i against every j != i. */
static void row_force(int64_t N, const double *pos, const double *mass, double eps,
                      double G, int64_t i, double *ai, double *phii) {
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const double eps2 = eps * eps;
    double ax = 0.0, ay = 0.0, az = 0.0, phi = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        if (j == i) continue;
        const double dx = pos[3 * j] - xi;
        const double dy = pos[3 * j + 1] - yi;
        const double dz = pos[3 * j + 2] - zi;
        const double s2 = dx * dx + dy * dy + dz * dz + eps2;
        if (s2 == 0.0) continue;
        const double s = sqrt(s2);
        const double inv_s3 = 1.0 / (s2 * s);
        ax += mass[j] * dx * inv_s3;
        ay += mass[j] * dy * inv_s3;
        az += mass[j] * dz * inv_s3;
        phi -= mass[j] / s;
    }
    ai[0] = G * ax;
    ai[1] = G * ay;
    ai[2] = G * az;
    *phii = G * phi;
}

/* acc [N][3] and pot [N] (pot may be NULL) for every particle. */
void orc_forces(int64_t N, const double *pos, const double *mass, double eps, double G,
                double *acc, double *pot) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
        double phi;
        row_force(N, pos, mass, eps, G, i, acc + 3 * i, &phi);
        if (pot) pot[i] = phi;
    }
}

/* Exact rows for a subset: acc [nrows][3], pot [nrows] for rows[r]. */
void orc_forces_rows(int64_t N, const double *pos, const double *mass, double eps, double G,
                     int64_t nrows, const int64_t *rows, double *acc, double *pot) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        double phi;
        row_force(N, pos, mass, eps, G, rows[r], acc + 3 * r, &phi);
        if (pot) pot[r] = phi;
    }
}

/*
 * nsteps KDK steps in place.  acc holds a(x_0) on entry when acc_valid != 0
 * (otherwise it is computed first) and a(x_n) on exit; pot (nullable) holds
 * phi(x_n) on exit.
 */
void orc_kdk(int64_t N, double *pos, double *vel, const double *mass, double eps, double G,
             double h, int64_t nsteps, int acc_valid, double *acc, double *pot) {
    if (!acc_valid || (nsteps == 0 && pot)) orc_forces(N, pos, mass, eps, G, acc, pot);
    for (int64_t n = 0; n < nsteps; ++n) {
        for (int64_t k = 0; k < 3 * N; ++k) vel[k] += 0.5 * h * acc[k];
        for (int64_t k = 0; k < 3 * N; ++k) pos[k] += h * vel[k];
        orc_forces(N, pos, mass, eps, G, acc, pot);
        for (int64_t k = 0; k < 3 * N; ++k) vel[k] += 0.5 * h * acc[k];
    }
}

/* out3 = {K, W, E} with K = 1/2 sum m v^2 and W = 1/2 sum m phi, summed in index order. */
void orc_energy(int64_t N, const double *vel, const double *mass, const double *pot,
                double *out3) {
    double K = 0.0, W = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        const double v2 = vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] +
                          vel[3 * i + 2] * vel[3 * i + 2];
        K += 0.5 * mass[i] * v2;
        W += 0.5 * mass[i] * pot[i];
    }
    out3[0] = K;
    out3[1] = W;
    out3[2] = K + W;
}

/*
 * K(d) = s^-3 I - 3 s^-5 d d^T with s^2 = |d|^2 + eps^2: the derivative of
 * d / s^3 with respect to d.  Written into M (3x3 row-major); returns 0 for a
 * skipped singular pair.
 */
static int pair_kernel(const double d[3], double eps2, double M[9], double *inv_s,
                       double *inv_s3) {
    const double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
    if (s2 == 0.0) return 0;
    const double s = sqrt(s2);
    const double is3 = 1.0 / (s2 * s);
    const double is5 = is3 / s2;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            M[3 * a + b] = (a == b ? is3 : 0.0) - 3.0 * is5 * d[a] * d[b];
    *inv_s = 1.0 / s;
    *inv_s3 = is3;
    return 1;
}

/*
 * Vector-Jacobian product of (a, phi) with respect to (x, m), overwriting
 * xbar [N][3] and mbar [N].  phibar may be NULL (treated as zero).
 *
 * Blocks used (d_ik = x_k - x_i, s_ik^2 = |d_ik|^2 + eps^2):
 *   i != k:  d a_i / d x_k   =  G m_k K(d_ik)
 *            d phi_i / d x_k =  G m_k d_ik / s_ik^3
 *            d a_i / d m_k   =  G d_ik / s_ik^3
 *            d phi_i / d m_k = -G / s_ik
 *   i == k:  d a_k / d x_k   = -G sum_{j != k} m_j K(x_j - x_k)
 *            d phi_k / d x_k = -G sum_{j != k} m_j (x_j - x_k) / s_kj^3
 *            d a_k / d m_k = 0,  d phi_k / d m_k = 0
 */
void orc_forces_vjp(int64_t N, const double *pos, const double *mass, double eps, double G,
                    const double *abar, const double *phibar, double *xbar, double *mbar) {
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < N; ++k) {
        double xb[3] = {0.0, 0.0, 0.0};
        double mb = 0.0;
        /* diagonal blocks d a_k / d x_k and d phi_k / d x_k */
        double Jkk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        double gphi_kk[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < N; ++j) {
            if (j == k) continue;
            double d[3] = {pos[3 * j] - pos[3 * k], pos[3 * j + 1] - pos[3 * k + 1],
                           pos[3 * j + 2] - pos[3 * k + 2]};
            double M[9], is, is3;
            if (!pair_kernel(d, eps2, M, &is, &is3)) continue;
            for (int e = 0; e < 9; ++e) Jkk[e] -= G * mass[j] * M[e];
            for (int a = 0; a < 3; ++a) gphi_kk[a] -= G * mass[j] * d[a] * is3;
        }
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) xb[a] += Jkk[3 * b + a] * abar[3 * k + b];
            if (phibar) xb[a] += gphi_kk[a] * phibar[k];
        }
        /* off-diagonal blocks: every i != k sees x_k and m_k */
        for (int64_t i = 0; i < N; ++i) {
            if (i == k) continue;
            double d[3] = {pos[3 * k] - pos[3 * i], pos[3 * k + 1] - pos[3 * i + 1],
                           pos[3 * k + 2] - pos[3 * i + 2]};
            double M[9], is, is3;
            if (!pair_kernel(d, eps2, M, &is, &is3)) continue;
            for (int a = 0; a < 3; ++a) {
                for (int b = 0; b < 3; ++b)
                    xb[a] += G * mass[k] * M[3 * b + a] * abar[3 * i + b];
                if (phibar) xb[a] += G * mass[k] * d[a] * is3 * phibar[i];
                mb += G * d[a] * is3 * abar[3 * i + a];
            }
            if (phibar) mb -= G * is * phibar[i];
        }
        xbar[3 * k] = xb[0];
        xbar[3 * k + 1] = xb[1];
        xbar[3 * k + 2] = xb[2];
        mbar[k] = mb;
    }
}

/*
 * Acceleration, jerk (its time derivative along the motion) and potential:
 * the quantities of the pair kernel in App. A, Algorithm 3, with the same
 * softening.  For d = x_j - x_i, w = v_j - v_i, s^2 = |d|^2 + eps^2:
 *   jerk_i = G sum_{j != i} m_j [ w / s^3 - 3 (d . w) d / s^5 ]
 */
void orc_forces_jerk(int64_t N, const double *pos, const double *vel, const double *mass,
                     double eps, double G, double *acc, double *jerk, double *pot) {
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
        double a[3] = {0, 0, 0}, jk[3] = {0, 0, 0}, phi = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d[3], w[3];
            for (int c = 0; c < 3; ++c) {
                d[c] = pos[3 * j + c] - pos[3 * i + c];
                w[c] = vel[3 * j + c] - vel[3 * i + c];
            }
            const double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
            if (s2 == 0.0) continue;
            const double s = sqrt(s2);
            const double inv3 = 1.0 / (s2 * s);
            const double dw = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
            for (int c = 0; c < 3; ++c) {
                a[c] += mass[j] * d[c] * inv3;
                jk[c] += mass[j] * (w[c] * inv3 - 3.0 * dw * d[c] * inv3 / s2);
            }
            phi -= mass[j] / s;
        }
        for (int c = 0; c < 3; ++c) {
            acc[3 * i + c] = G * a[c];
            jerk[3 * i + c] = G * jk[c];
        }
        if (pot) pot[i] = G * phi;
    }
}

/*
 * nsteps of the fourth-order Hermite predictor-corrector (the
 * predict-evaluate-correct cycle of Sec. 2.1 at fourth order):
 *   predict  xp = x + v h + a h^2/2 + j h^3/6,   vp = v + a h + j h^2/2
 *   evaluate a1, j1 at (xp, vp)
 *   correct  v1 = v + (a + a1) h/2 + (j - j1) h^2/12
 *            x1 = x + (v + v1) h/2 + (a - a1) h^2/12
 * acc/jerk hold a(x0), j(x0) on entry when valid != 0 and a1, j1 on exit.
 */
void orc_hermite4(int64_t N, double *pos, double *vel, const double *mass, double eps, double G,
                  double h, int64_t nsteps, int valid, double *acc, double *jerk) {
    if (!valid) orc_forces_jerk(N, pos, vel, mass, eps, G, acc, jerk, 0);
    double *xp = (double *)malloc(sizeof(double) * 3 * N);
    double *vp = (double *)malloc(sizeof(double) * 3 * N);
    double *a1 = (double *)malloc(sizeof(double) * 3 * N);
    double *j1 = (double *)malloc(sizeof(double) * 3 * N);
    for (int64_t n = 0; n < nsteps; ++n) {
        for (int64_t k = 0; k < 3 * N; ++k) {
            xp[k] = pos[k] + vel[k] * h + acc[k] * h * h / 2.0 + jerk[k] * h * h * h / 6.0;
            vp[k] = vel[k] + acc[k] * h + jerk[k] * h * h / 2.0;
        }
        orc_forces_jerk(N, xp, vp, mass, eps, G, a1, j1, 0);
        for (int64_t k = 0; k < 3 * N; ++k) {
            const double v1 = vel[k] + (acc[k] + a1[k]) * h / 2.0 + (jerk[k] - j1[k]) * h * h / 12.0;
            pos[k] = pos[k] + (vel[k] + v1) * h / 2.0 + (acc[k] - a1[k]) * h * h / 12.0;
            vel[k] = v1;
            acc[k] = a1[k];
            jerk[k] = j1[k];
        }
    }
    free(xp);
    free(vp);
    free(a1);
    free(j1);
}

/* orc_forces_jerk restricted to the rows listed in `rows` (each against all N). */
void orc_forces_jerk_rows(int64_t N, const double *pos, const double *vel, const double *mass,
                          double eps, double G, int64_t nrows, const int64_t *rows, double *acc,
                          double *jerk) {
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        double a[3] = {0, 0, 0}, jk[3] = {0, 0, 0};
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d[3], w[3];
            for (int c = 0; c < 3; ++c) {
                d[c] = pos[3 * j + c] - pos[3 * i + c];
                w[c] = vel[3 * j + c] - vel[3 * i + c];
            }
            const double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
            if (s2 == 0.0) continue;
            const double s = sqrt(s2);
            const double inv3 = 1.0 / (s2 * s);
            const double dw = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
            for (int c = 0; c < 3; ++c) {
                a[c] += mass[j] * d[c] * inv3;
                jk[c] += mass[j] * (w[c] * inv3 - 3.0 * dw * d[c] * inv3 / s2);
            }
        }
        for (int c = 0; c < 3; ++c) {
            acc[3 * r + c] = G * a[c];
            jerk[3 * r + c] = G * jk[c];
        }
    }
}
