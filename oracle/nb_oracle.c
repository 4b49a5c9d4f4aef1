/*
 * nb_oracle.c -- plain FP64 CPU oracle for the exact softened gravitational
 * force and potential of Fujiwara & Nakasato, "Fast Simulations of
 * Gravitational Many-body Problem on RV770 GPU" (arXiv:0904.3659).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark call this file. The CUDA library never links,
 * includes or calls it, and it includes nothing from the CUDA library: the two
 * share no code. It is deliberately slow and obvious: double precision, the
 * summation order of the definition (j ascending), no blocking, no
 * vectorisation tricks. OpenMP only splits the independent i rows across
 * cores (Section "Introduction": the force on each particle is independent).
 *
 * Conventions (readings of the paper, see the project's design notes):
 *  - Eq. (gravity) is returned literally:
 *        a_i = sum_{j != i} m_j (x_i - x_j) / (|x_i - x_j|^2 + eps^2)^{3/2}
 *        p_i = sum_{j != i} m_j / (|x_i - x_j|^2 + eps^2)^{1/2}
 *    i.e. a_i points away from the other masses and p_i > 0. The physical
 *    gravitational acceleration (G = 1) is g_i = -a_i and the potential
 *    energy is W = -1/2 sum_i m_i p_i.
 *  - j == i is skipped by index (Eq. (gravity) says j != i). Distinct
 *    particles at the same position are summed (they add 0 to a_i and
 *    m_j/eps to p_i).
 *  - eps^2 is formed in double from the (FP32) eps the caller passes.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no FMA contraction,
 * so x86 and Arm hosts round identically).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of OpenMP threads a parallel region of this library will use. */
int nbo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void nbo_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * One row i of Eq. (gravity): the sum over j != i in ascending j, the loop
 * shape of the paper's Fig. 1 with the j == i term left out.
 * x is [n][3], m is [n]. Writes a[3], *p and *amag, where
 * amag = sum_{j != i} m_j |x_i - x_j| / s_ij^{3/2} is the sum of the
 * magnitudes of the terms of a_i (the scale the relative error of a_i is
 * measured against where the vector sum cancels).
 */
static void force_row(int64_t n, const double *x, const double *m, double eps2,
                      int64_t i, double a[3], double *p, double *amag)
{
    double ax = 0.0, ay = 0.0, az = 0.0, pp = 0.0, am = 0.0;
    const double xi = x[3 * i + 0], yi = x[3 * i + 1], zi = x[3 * i + 2];
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const double dx = xi - x[3 * j + 0];
        const double dy = yi - x[3 * j + 1];
        const double dz = zi - x[3 * j + 2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double s = r2 + eps2;            /* |x_i - x_j|^2 + eps^2 */
        const double inv_sqrt_s = 1.0 / sqrt(s); /* s^{-1/2} */
        const double inv_s32 = inv_sqrt_s * inv_sqrt_s * inv_sqrt_s; /* s^{-3/2} */
        ax += m[j] * dx * inv_s32;
        ay += m[j] * dy * inv_s32;
        az += m[j] * dz * inv_s32;
        pp += m[j] * inv_sqrt_s;
        am += m[j] * sqrt(r2) * inv_s32;
    }
    a[0] = ax;
    a[1] = ay;
    a[2] = az;
    *p = pp;
    if (amag) *amag = am;
}

/*
 * Eq. (gravity) for every particle. a is [n][3], p and amag are [n]
 * (amag may be NULL).
 */
void nbo_force(int64_t n, const double *x, const double *m, double eps,
               double *a, double *p, double *amag)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        force_row(n, x, m, eps2, i, &a[3 * i], &p[i], amag ? &amag[i] : NULL);
}

/*
 * Eq. (gravity) for the listed rows only (sampled check of a large run).
 * rows[k] in [0, n); a is [nrows][3], p and amag are [nrows].
 */
void nbo_force_rows(int64_t n, const double *x, const double *m, double eps,
                    int64_t nrows, const int64_t *rows,
                    double *a, double *p, double *amag)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nrows; ++k)
        force_row(n, x, m, eps2, rows[k], &a[3 * k], &p[k], amag ? &amag[k] : NULL);
}

/*
 * Vector-Jacobian product of Eq. (gravity): given upstream gradients
 * ga [n][3] on a and gp [n] on p, the gradient of
 *     L = sum_i ( ga_i . a_i + gp_i p_i )
 * with respect to the positions (gx [n][3]) and masses (gm [n]).
 *
 * Derivation (chain rule of the definition). The ordered pair (i, j), j != i,
 * contributes m_j [ ga_i . r s^{-3/2} + gp_i s^{-1/2} ] to L, with
 * r = x_i - x_j and s = |r|^2 + eps^2. Its derivative with respect to r is
 *     m_j G(r, ga_i, gp_i),
 *     G(r, g, q) = s^{-3/2} g - 3 s^{-5/2} (r . g) r - q s^{-3/2} r,
 * which enters dL/dx_i with sign + and dL/dx_j with sign -. Its derivative
 * with respect to m_j is ga_i . r s^{-3/2} + gp_i s^{-1/2}.
 *
 * Collecting, for particle k every pair that contains it, with r = x_k - x_l:
 *   gx_k = sum_{l != k}  m_l G(r, ga_k, gp_k)              (k as the i of the pair)
 *                      - m_k G(-r, ga_l, gp_l)             (k as the j of the pair)
 *   gm_k = sum_{l != k}  ga_l . (-r) s^{-3/2} + gp_l s^{-1/2}
 * Each row k is written out plainly below, l ascending.
 */
static void vjp_row(int64_t n, const double *x, const double *m, double eps2,
                    const double *ga, const double *gp, int64_t k,
                    double gxk[3], double *gmk)
{
    double gx0 = 0.0, gx1 = 0.0, gx2 = 0.0, gmm = 0.0;
    for (int64_t l = 0; l < n; ++l) {
        if (l == k) continue;
        /* r = x_k - x_l */
        const double r0 = x[3 * k + 0] - x[3 * l + 0];
        const double r1 = x[3 * k + 1] - x[3 * l + 1];
        const double r2 = x[3 * k + 2] - x[3 * l + 2];
        const double s = r0 * r0 + r1 * r1 + r2 * r2 + eps2;
        const double sm12 = 1.0 / sqrt(s);          /* s^{-1/2} */
        const double sm32 = sm12 * sm12 * sm12;     /* s^{-3/2} */
        const double sm52 = sm32 / s;               /* s^{-5/2} */

        /* k as the i of the pair (k, l): + m_l G(r, ga_k, gp_k) */
        const double rgk = r0 * ga[3 * k + 0] + r1 * ga[3 * k + 1] + r2 * ga[3 * k + 2];
        gx0 += m[l] * (sm32 * ga[3 * k + 0] - 3.0 * sm52 * rgk * r0 - gp[k] * sm32 * r0);
        gx1 += m[l] * (sm32 * ga[3 * k + 1] - 3.0 * sm52 * rgk * r1 - gp[k] * sm32 * r1);
        gx2 += m[l] * (sm32 * ga[3 * k + 2] - 3.0 * sm52 * rgk * r2 - gp[k] * sm32 * r2);

        /* k as the j of the pair (l, k): the pair's r is x_l - x_k = -r, and
         * it enters with sign -: - m_k G(-r, ga_l, gp_l)
         *   G(-r, g, q) = s^{-3/2} g - 3 s^{-5/2} (r . g) r + q s^{-3/2} r */
        const double rgl = r0 * ga[3 * l + 0] + r1 * ga[3 * l + 1] + r2 * ga[3 * l + 2];
        gx0 -= m[k] * (sm32 * ga[3 * l + 0] - 3.0 * sm52 * rgl * r0 + gp[l] * sm32 * r0);
        gx1 -= m[k] * (sm32 * ga[3 * l + 1] - 3.0 * sm52 * rgl * r1 + gp[l] * sm32 * r1);
        gx2 -= m[k] * (sm32 * ga[3 * l + 2] - 3.0 * sm52 * rgl * r2 + gp[l] * sm32 * r2);

        /* m_k is the m_j of the pair (l, k): ga_l . (x_l - x_k) s^{-3/2} + gp_l s^{-1/2} */
        gmm += -rgl * sm32 + gp[l] * sm12;
    }
    gxk[0] = gx0;
    gxk[1] = gx1;
    gxk[2] = gx2;
    *gmk = gmm;
}

void nbo_force_vjp(int64_t n, const double *x, const double *m, double eps,
                   const double *ga, const double *gp, double *gx, double *gm)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k)
        vjp_row(n, x, m, eps2, ga, gp, k, &gx[3 * k], &gm[k]);
}

void nbo_force_vjp_rows(int64_t n, const double *x, const double *m, double eps,
                        const double *ga, const double *gp,
                        int64_t nrows, const int64_t *rows, double *gx, double *gm)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nrows; ++k)
        vjp_row(n, x, m, eps2, ga, gp, rows[k], &gx[3 * k], &gm[k]);
}

/*
 * Leap-frog integration, Section "Method", Eqs. (1)-(3), following the
 * seven-step algorithm given there:
 *   step 2:  a_0 = Eq. (gravity) at x_0
 *   step 3:  v_{1/2} = v_0 + 1/2 g_0 dt                       Eq. (1)
 *   step 4:  x_1     = x_0 + v_0 dt + 1/2 g_0 dt^2            Eq. (2)
 *   step 5:  a_1 = Eq. (gravity) at x_1
 *   step 6:  v_1     = v_{1/2} + 1/2 g_1 dt                    Eq. (3)
 *   step 7:  repeat from step 3.
 * g = -a is the physical (attractive, G = 1) acceleration: Eq. (gravity)
 * as printed has the sign of a repulsion, so it is negated before it enters
 * Eqs. (1)-(3).
 *
 * x, v: [n][3] in/out. g_out: [n][3], the physical acceleration at the
 * final positions (may be NULL). work: caller scratch of 4n doubles.
 */
void nbo_leapfrog(int64_t n, double *x, double *v, const double *m, double eps,
                  double dt, int64_t nsteps, double *g_out, double *work)
{
    double *a = work;          /* [n][3] */
    double *p = work + 3 * n;  /* [n] */
    nbo_force(n, x, m, eps, a, p, NULL);                    /* step 2 */
    for (int64_t step = 0; step < nsteps; ++step) {
        for (int64_t k = 0; k < 3 * n; ++k) {
            const double g0 = -a[k];
            const double v0 = v[k];
            v[k] = v0 + 0.5 * g0 * dt;                      /* step 3, Eq. (1) */
            x[k] = x[k] + v0 * dt + 0.5 * g0 * dt * dt;     /* step 4, Eq. (2) */
        }
        nbo_force(n, x, m, eps, a, p, NULL);                /* step 5 */
        for (int64_t k = 0; k < 3 * n; ++k)
            v[k] = v[k] + 0.5 * (-a[k]) * dt;               /* step 6, Eq. (3) */
    }
    if (g_out)
        for (int64_t k = 0; k < 3 * n; ++k) g_out[k] = -a[k];
}

/*
 * Total energy of the system: kinetic K = 1/2 sum_i m_i |v_i|^2 and
 * potential W = -1/2 sum_i m_i p_i with p_i from Eq. (gravity) (each pair
 * counted once). out[0] = K, out[1] = W. work: caller scratch of 4n doubles.
 */
void nbo_energy(int64_t n, const double *x, const double *v, const double *m,
                double eps, double out[2], double *work)
{
    double *a = work;
    double *p = work + 3 * n;
    nbo_force(n, x, m, eps, a, p, NULL);
    double kin = 0.0, pot = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double v2 = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
        kin += 0.5 * m[i] * v2;
        pot += -0.5 * m[i] * p[i];
    }
    out[0] = kin;
    out[1] = pot;
}
