/*
 * bd_oracle.c -- plain, slow, obviously-correct CPU oracle for one periodic
 * Brownian-dynamics Euler step with Ewald-summed RPY hydrodynamics
 * (Jain, Sunthar, Duenweg & Prakash, "Optimisation of a Brownian dynamics
 * algorithm for semidilute polymer solutions").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * Precision: IEEE binary64 throughout, compiled without fast-math and without
 * FMA contraction (so x86-64 and aarch64 give identical results).  The one
 * exception is the overlap correction (Eqs. cor3-cor5, DFmodified): for an
 * image closer than 2a the sum M1 + M* cancels like (a/r)^3, so that single
 * image is evaluated in long double and then rounded to double.
 *
 * The PLANT_* preprocessor switches exist only for the mutation test in the
 * test-suite, which compiles variants with one deliberate mistake each and
 * checks that some pin fails; the default build defines none of them.
 *
 * Every function states the passage it follows.  Readings of the paper that
 * the code takes where the text is ambiguous or misprinted:
 *   R1 (Eq. DF, reciprocal sum): the bracket is read as
 *      cos(k.r_nu) sum cos(k.r_mu) F + sin(k.r_nu) sum sin(k.r_mu) F, i.e.
 *      cos(k.(r_nu - r_mu)).  The printed minus sign gives cos(k.(r_nu+r_mu)),
 *      which is not translation invariant.
 *   R2 (Eq. cor5, overlap tensor M*): M* = Omega_B - Omega_A.  The identity
 *      coefficient is as printed; the rr coefficient is 3(x^2-4)^2/(32 x^3),
 *      not the printed (3x^2/4-1)^2/(2x^3) (which does not vanish at x=2 and
 *      makes D indefinite).
 *   R3 (Sec. II C): M* is applied to the (at most one) image of a pair ν≠μ
 *      whose separation is below 2a, whatever the lattice vector.
 *   R4 (Sec. II D, Eqs. rparameter/kparameter): the real-space sum includes
 *      images with |r_νμ,n| <= r_c; the reciprocal sum includes k = 2πn/L for
 *      integer n != 0 with n.n <= n2max (the caller converts k_c to n2max).
 *   R5 (Sec. IV, Eq. cheb1): Chebyshev coefficients are those of the
 *      Chebyshev interpolant of sqrt on [d_min, d_max] at the N_Ch
 *      Chebyshev-Gauss nodes, c_p = (2/N_Ch) sum_j f(cos t_j) cos(p t_j),
 *      t_j = π(j+1/2)/N_Ch (the paper does not print them).
 *   R6 (narrow-Gaussian excluded volume, not defined in the paper):
 *      U/kT = (z/d^3) exp(-r^2/(2 d^2)), force (z/d^5) r exp(-r^2/(2 d^2)) with
 *      z = z_star, d = d_star,
 *      summed over all periodic images with |r| <= r_ev.
 *   R7 (Sec. VII, FENE rejection): a step is rejected when any spring of the
 *      new configuration has |Q|^2 >= b; the configuration is then unchanged.
 *   R8 (Eq. sde): kappa = 0 (no flow); the step advances with Wiener column 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t n;            /* number of beads N                                  */
    int32_t nb;           /* beads per chain N_b (chains are contiguous)        */
    double  L;            /* box edge                                           */
    double  a;            /* bead radius a = sqrt(pi) h*                        */
    double  alpha;        /* Ewald splitting parameter                          */
    double  rc;           /* real-space cutoff                                  */
    int32_t n2max;        /* reciprocal cutoff: integer n.n <= n2max            */
    int32_t overlap_corr; /* 1: add M* for images closer than 2a                */
    int32_t spring;       /* 0 Hookean, 1 FENE                                  */
    double  fene_b;       /* FENE extensibility b                               */
    int32_t ev_on;        /* narrow-Gaussian excluded volume on/off             */
    double  z_star, d_star, r_ev;
    double  dt;           /* time step                                          */
} oracle_params;

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Eq. (M1): real-space Ewald tensor M1(r) = c1 I + c2 rhat rhat.            */
static void m1_coeffs(double r, double a, double al, double *c1, double *c2)
{
    double a3 = a * a * a;
    double r2 = r * r, r3 = r2 * r, r4 = r2 * r2;
    double al2 = al * al, al3 = al2 * al, al5 = al3 * al2, al7 = al5 * al2;
    double ec = erfc(al * r);
    double ex = exp(-al2 * r2) / sqrt(PI);
    *c1 = ec * (3.0 * a / (4.0 * r) + a3 / (2.0 * r3))
        + ex * (3.0 * a * al3 * r2 - 9.0 * a * al / 2.0 + 4.0 * a3 * al7 * r4
#ifdef PLANT_M1_COEF
                - 16.0 * a3 * al5 * r2 + 14.0 * a3 * al3 + a3 * al / r2);
#else
                - 20.0 * a3 * al5 * r2 + 14.0 * a3 * al3 + a3 * al / r2);
#endif
    *c2 = ec * (3.0 * a / (4.0 * r) - 3.0 * a3 / (2.0 * r3))
        + ex * (3.0 * a * al / 2.0 - 3.0 * a * al3 * r2 - 4.0 * a3 * al7 * r4
                + 16.0 * a3 * al5 * r2 - 2.0 * a3 * al3 - 3.0 * a3 * al / r2);
}

/* Eq. (M1) + Eq. (cor5) (reading R2) in long double, for one image closer
 * than 2a.  Returns the 3x3 block contribution M1(v) + M*(v).              */
static void m1_plus_mstar_ld(const double v[3], double a_d, double al_d, double B[9])
{
    long double a = a_d, al = al_d;
    long double vx = v[0], vy = v[1], vz = v[2];
    long double r2 = vx * vx + vy * vy + vz * vz;
    long double r = sqrtl(r2), r3 = r2 * r, r4 = r2 * r2;
    long double a3 = a * a * a;
    long double al2 = al * al, al3 = al2 * al, al5 = al3 * al2, al7 = al5 * al2;
    long double ec = erfcl(al * r);
    long double ex = expl(-al2 * r2) / sqrtl(3.14159265358979323846264338327950288L);
    long double c1 = ec * (3.0L * a / (4.0L * r) + a3 / (2.0L * r3))
        + ex * (3.0L * a * al3 * r2 - 9.0L * a * al / 2.0L + 4.0L * a3 * al7 * r4
                - 20.0L * a3 * al5 * r2 + 14.0L * a3 * al3 + a3 * al / r2);
    long double c2 = ec * (3.0L * a / (4.0L * r) - 3.0L * a3 / (2.0L * r3))
        + ex * (3.0L * a * al / 2.0L - 3.0L * a * al3 * r2 - 4.0L * a3 * al7 * r4
                + 16.0L * a3 * al5 * r2 - 2.0L * a3 * al3 - 3.0L * a3 * al / r2);
    long double x = r / a, x2 = x * x, x3 = x2 * x;
    long double q = 0.75L * x2 + 1.0L;
    long double s1 = 1.0L - q * q / (2.0L * x3);                       /* delta coef   */
#ifdef PLANT_PRINTED_MSTAR
    long double s2 = (0.75L * x2 - 1.0L) * (0.75L * x2 - 1.0L) / (2.0L * x3);
#else
    long double s2 = 3.0L * (x2 - 4.0L) * (x2 - 4.0L) / (32.0L * x3); /* rr coef (R2) */
#endif
    long double d1 = c1 + s1;
    long double d2 = (c2 + s2) / r2;
    long double w[3] = {vx, vy, vz};
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            B[3 * i + j] += (double)((i == j ? d1 : 0.0L) + d2 * w[i] * w[j]);
}

/* Self term of Eq. (DF): (1 - 6 a alpha/sqrt(pi) + 40 a^3 alpha^3/(3 sqrt(pi))). */
static double self_coeff(double a, double al)
{
#ifdef PLANT_SELF_SIGN
    return 1.0 - 6.0 * a * al / sqrt(PI) - 40.0 * a * a * a * al * al * al / (3.0 * sqrt(PI));
#else
    return 1.0 - 6.0 * a * al / sqrt(PI) + 40.0 * a * a * a * al * al * al / (3.0 * sqrt(PI));
#endif
}

/* Eq. (M2) scalar prefactor; M2(k) = f(k) (I - khat khat), V = L^3.        */
#ifdef PLANT_M2_VOLUME
static double p_L_for_plant = 1.0;
#endif
static double m2_prefactor(double k2, double a, double al, double V)
{
    double al2 = al * al;
    return (a - a * a * a * k2 / 3.0) * (1.0 + k2 / (4.0 * al2) + k2 * k2 / (8.0 * al2 * al2))
#ifdef PLANT_M2_VOLUME
         * (6.0 * PI / (k2 * V / p_L_for_plant)) * exp(-k2 / (4.0 * al2));
#else
         * (6.0 * PI / (k2 * V)) * exp(-k2 / (4.0 * al2));
#endif
}

typedef struct { double k[3]; double f; } kterm;

static int build_klist(const oracle_params *p, kterm **out)
{
    int K = 0;
    while ((K + 1) * (K + 1) <= p->n2max) K++;
    int cap = (2 * K + 1) * (2 * K + 1) * (2 * K + 1);
    kterm *t = (kterm *)malloc(sizeof(kterm) * (size_t)(cap > 0 ? cap : 1));
    int cnt = 0;
    double V = p->L * p->L * p->L;
#ifdef PLANT_M2_VOLUME
    p_L_for_plant = p->L;
#endif
    for (int nx = -K; nx <= K; nx++)
        for (int ny = -K; ny <= K; ny++)
            for (int nz = -K; nz <= K; nz++) {
                int nn = nx * nx + ny * ny + nz * nz;
                if (nn == 0 || nn > p->n2max) continue;
                kterm *e = &t[cnt++];
                e->k[0] = 2.0 * PI * nx / p->L;
                e->k[1] = 2.0 * PI * ny / p->L;
                e->k[2] = 2.0 * PI * nz / p->L;
                double k2 = e->k[0] * e->k[0] + e->k[1] * e->k[1] + e->k[2] * e->k[2];
                e->f = m2_prefactor(k2, p->a, p->alpha, V);
            }
    *out = t;
    return cnt;
}

/* One 3x3 block D_{nu mu} of the periodic diffusion tensor: Eq. (DFmodified)
 * = self term (nu = mu) + real-space image sum of M1 (Eq. M1, prime: n = 0
 * omitted for nu = mu) + reciprocal sum of M2 cos(k.(r_nu - r_mu)) (Eq. M2,
 * reading R1) + M* for the image closer than 2a (Eq. cor5, readings R2/R3). */
static void d_block(const oracle_params *p, const kterm *kl, int nk,
                    const double *rn, const double *rm, int same, double B[9])
{
    double L = p->L, a = p->a, al = p->alpha, rc2 = p->rc * p->rc;
    for (int i = 0; i < 9; i++) B[i] = 0.0;
    double d[3];
    for (int i = 0; i < 3; i++) {
        d[i] = rn[i] - rm[i];
        d[i] -= L * nearbyint(d[i] / L);          /* minimum image (Fig. pbc) */
    }
    int nmax = (int)floor(p->rc / L + 0.5) + 1;
    for (int nx = -nmax; nx <= nmax; nx++) {
        double vx = d[0] + nx * L;
        if (vx * vx > rc2) continue;
        for (int ny = -nmax; ny <= nmax; ny++) {
            double vy = d[1] + ny * L;
            if (vx * vx + vy * vy > rc2) continue;
            for (int nz = -nmax; nz <= nmax; nz++) {
                if (same && nx == 0 && ny == 0 && nz == 0) continue;
                double vz = d[2] + nz * L;
                double u = vx * vx + vy * vy + vz * vz;
                if (u > rc2) continue;
                double v[3] = {vx, vy, vz};
                if (!same && u == 0.0) {
                    /* coincident beads: the r -> 0 limit of M1 + M* is the
                     * self coefficient times I (smooth limit of Eq. DFmodified) */
                    double s = p->overlap_corr ? self_coeff(a, al) : NAN;
                    B[0] += s; B[4] += s; B[8] += s;
                    continue;
                }
                if (!same && p->overlap_corr && u < 4.0 * a * a) {
                    m1_plus_mstar_ld(v, a, al, B);
                    continue;
                }
                double r = sqrt(u), c1, c2;
                m1_coeffs(r, a, al, &c1, &c2);
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++)
                        B[3 * i + j] += (i == j ? c1 : 0.0) + c2 * v[i] * v[j] / u;
            }
        }
    }
    for (int t = 0; t < nk; t++) {
        const double *k = kl[t].k;
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
#ifdef PLANT_RECIP_SIGN
        double cs = cos(k[0] * (rn[0] + rm[0]) + k[1] * (rn[1] + rm[1]) + k[2] * (rn[2] + rm[2]));
#else
        double cs = cos(k[0] * d[0] + k[1] * d[1] + k[2] * d[2]);
#endif
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                B[3 * i + j] += kl[t].f * ((i == j ? 1.0 : 0.0) - k[i] * k[j] / k2) * cs;
    }
    if (same) {
        double s = self_coeff(a, al);
        B[0] += s; B[4] += s; B[8] += s;
    }
}

/* Rows [row_begin, row_end) of beads of D (row-major, each bead row holds
 * 3 matrix rows of length 3n).  Eq. (Domega) via Eq. (DFmodified).         */
void oracle_build_D_rows(const oracle_params *p, const double *R,
                         int32_t row_begin, int32_t row_end, double *Dout)
{
    kterm *kl;
    int nk = build_klist(p, &kl);
    int n = p->n;
    long n3 = 3L * n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int nu = row_begin; nu < row_end; nu++) {
        for (int mu = 0; mu < n; mu++) {
            double B[9];
            d_block(p, kl, nk, &R[3 * nu], &R[3 * mu], nu == mu, B);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++)
                    Dout[(3L * (nu - row_begin) + i) * n3 + 3L * mu + j] = B[3 * i + j];
        }
    }
    free(kl);
}

void oracle_build_D(const oracle_params *p, const double *R, double *D)
{
    oracle_build_D_rows(p, R, 0, p->n, D);
}

/* One block, for sampled checks at sizes where the full D is too large.    */
void oracle_D_block(const oracle_params *p, const double *R, int32_t nu, int32_t mu, double *B9)
{
    kterm *kl;
    int nk = build_klist(p, &kl);
    d_block(p, kl, nk, &R[3 * nu], &R[3 * mu], nu == mu, B9);
    free(kl);
}

/* ------------------------------------------------------------------------ */
/* Sec. II A: spring forces F_mu = F^c(Q_mu) - F^c(Q_{mu-1}), Q_mu =
 * r_{mu+1} - r_mu within a chain; Hookean F^c(Q) = Q, FENE F^c(Q) =
 * Q / (1 - |Q|^2/b).  Plus narrow-Gaussian excluded volume (reading R6).
 * Returns the number of FENE springs with |Q|^2 >= b (force undefined).   */
int32_t oracle_forces(const oracle_params *p, const double *R, double *F)
{
    int n = p->n, nb = p->nb;
    int32_t bad = 0;
    for (long i = 0; i < 3L * n; i++) F[i] = 0.0;
    for (int c = 0; c < n / nb; c++) {
        for (int j = 0; j + 1 < nb; j++) {
            int mu = c * nb + j;
            double Q[3], q2 = 0.0;
            for (int s = 0; s < 3; s++) {
                Q[s] = R[3 * (mu + 1) + s] - R[3 * mu + s];
                q2 += Q[s] * Q[s];
            }
            double g = 1.0;
            if (p->spring == 1) {
                if (q2 >= p->fene_b) { bad++; g = NAN; }
                else g = 1.0 / (1.0 - q2 / p->fene_b);
            }
            for (int s = 0; s < 3; s++) {
                F[3 * mu + s] += g * Q[s];          /* F^c(Q_mu) on bead mu        */
#ifdef PLANT_SPRING_SIGN
                F[3 * (mu + 1) + s] += g * Q[s];
#else
                F[3 * (mu + 1) + s] -= g * Q[s];    /* -F^c(Q_mu) on bead mu+1     */
#endif
            }
        }
    }
    if (p->ev_on) {
        double L = p->L, d2 = p->d_star * p->d_star;
        double pref = p->z_star / (d2 * d2 * p->d_star);
        double rev2 = p->r_ev * p->r_ev;
        int nmax = (int)floor(p->r_ev / L + 0.5) + 1;
#pragma omp parallel for schedule(dynamic, 4)
        for (int nu = 0; nu < n; nu++) {
            double acc[3] = {0.0, 0.0, 0.0};
            for (int mu = 0; mu < n; mu++) {
                if (mu == nu) continue;
                double d[3];
                for (int s = 0; s < 3; s++) {
                    d[s] = R[3 * nu + s] - R[3 * mu + s];
                    d[s] -= L * nearbyint(d[s] / L);
                }
                for (int nx = -nmax; nx <= nmax; nx++)
                    for (int ny = -nmax; ny <= nmax; ny++)
                        for (int nz = -nmax; nz <= nmax; nz++) {
                            double v[3] = {d[0] + nx * L, d[1] + ny * L, d[2] + nz * L};
                            double u = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                            if (u > rev2) continue;
                            double w = pref * exp(-u / (2.0 * d2));
                            for (int s = 0; s < 3; s++) acc[s] += w * v[s];
                        }
            }
            for (int s = 0; s < 3; s++) F[3 * nu + s] += acc[s];
        }
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Y = D X with plain loops; D is n3 x n3 row-major, X and Y are n3 x m
 * column-major (column j starts at j*n3).                                  */
void oracle_apply_D(int32_t n3, const double *D, const double *X, int32_t m, double *Y)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n3; i++) {
        for (int j = 0; j < m; j++) {
            double s = 0.0;
            for (int k = 0; k < n3; k++) s += D[(long)i * n3 + k] * X[(long)j * n3 + k];
            Y[(long)j * n3 + i] = s;
        }
    }
}

/* Same product restricted to rows [r0, r1) of D given as a row block.      */
void oracle_apply_rows(int32_t n3, int32_t r0, int32_t r1, const double *Drows,
                       const double *X, int32_t m, double *Y)
{
#pragma omp parallel for schedule(static)
    for (int i = r0; i < r1; i++) {
        for (int j = 0; j < m; j++) {
            double s = 0.0;
            for (int k = 0; k < n3; k++) s += Drows[(long)(i - r0) * n3 + k] * X[(long)j * n3 + k];
            Y[(long)j * n3 + i] = s;
        }
    }
}

/* Reading R5: coefficients of the Chebyshev interpolant of sqrt on
 * [dmin, dmax] at N_Ch Chebyshev-Gauss nodes.                               */
void oracle_cheb_coeffs(int32_t nch, double dmin, double dmax, double *c)
{
    double h = 0.5 * (dmax - dmin), m = 0.5 * (dmax + dmin);
    for (int p = 0; p < nch; p++) {
        double s = 0.0;
        for (int j = 0; j < nch; j++) {
            double t = PI * (j + 0.5) / nch;
            s += sqrt(h * cos(t) + m) * cos(p * t);
        }
        c[p] = 2.0 * s / nch;
    }
}

/* Sec. IV, Eqs. (cheb1)-(cheb3): dS = sum_{p<N_Ch} c_p V_p - (c_0/2) dW,
 * V_0 = dW, V_1 = Y V_0, V_p = 2 Y V_{p-1} - V_{p-2},
 * Y = 2/(dmax-dmin) D - (dmax+dmin)/(dmax-dmin) I.
 * E_f per column as defined in Sec. IV:
 * sqrt(|dS.dS - dW.D.dW| / dW.D.dW).  All vectors n3 x m column-major.     */
void oracle_cheb_sqrt(int32_t n3, const double *D, double dmin, double dmax, int32_t nch,
                      const double *dW, int32_t m, double *dS, double *Ef)
{
    long len = (long)n3 * m;
    double *c = (double *)malloc(sizeof(double) * (size_t)nch);
    double *Vm2 = (double *)malloc(sizeof(double) * (size_t)len);
    double *Vm1 = (double *)malloc(sizeof(double) * (size_t)len);
    double *Vp = (double *)malloc(sizeof(double) * (size_t)len);
    double *DV = (double *)malloc(sizeof(double) * (size_t)len);
    oracle_cheb_coeffs(nch, dmin, dmax, c);
    double ys = 2.0 / (dmax - dmin), yt = (dmax + dmin) / (dmax - dmin);
#ifdef PLANT_CHEB_NO_HALF
    for (long i = 0; i < len; i++) { Vm1[i] = dW[i]; dS[i] = c[0] * dW[i]; }
#else
    for (long i = 0; i < len; i++) { Vm1[i] = dW[i]; dS[i] = c[0] * dW[i] - 0.5 * c[0] * dW[i]; }
#endif
    oracle_apply_D(n3, D, dW, m, DV);
    /* quadratic forms dW.D.dW, used by E_f */
    double *wdw = (double *)malloc(sizeof(double) * (size_t)m);
    for (int j = 0; j < m; j++) {
        double s = 0.0;
        for (long i = 0; i < n3; i++) s += dW[(long)j * n3 + i] * DV[(long)j * n3 + i];
        wdw[j] = s;
    }
    if (nch > 1) {
        for (long i = 0; i < len; i++) {
            Vp[i] = ys * DV[i] - yt * Vm1[i];          /* V_1 = Y V_0 */
            dS[i] += c[1] * Vp[i];
        }
        for (long i = 0; i < len; i++) { Vm2[i] = Vm1[i]; Vm1[i] = Vp[i]; }
    }
    for (int p = 2; p < nch; p++) {
        oracle_apply_D(n3, D, Vm1, m, DV);
        for (long i = 0; i < len; i++) {
#ifdef PLANT_CHEB_RECURRENCE
            Vp[i] = 2.0 * (ys * DV[i] - yt * Vm1[i]) + Vm2[i];
#else
            Vp[i] = 2.0 * (ys * DV[i] - yt * Vm1[i]) - Vm2[i];
#endif
            dS[i] += c[p] * Vp[i];
        }
        for (long i = 0; i < len; i++) { Vm2[i] = Vm1[i]; Vm1[i] = Vp[i]; }
    }
    if (Ef) {
        for (int j = 0; j < m; j++) {
            double ss = 0.0;
            for (long i = 0; i < n3; i++) ss += dS[(long)j * n3 + i] * dS[(long)j * n3 + i];
            Ef[j] = sqrt(fabs(ss - wdw[j]) / wdw[j]);
        }
    }
    free(c); free(Vm2); free(Vm1); free(Vp); free(DV); free(wdw);
}

/* ------------------------------------------------------------------------ */
/* Eq. (sde) with kappa = 0 (reading R8):
 * r(t+dt) = r + (dt/4) D.F + (1/sqrt 2) dS[:,0], dS from the Chebyshev
 * expansion with the given bounds and N_Ch.  FENE rejection per R7.
 * Outputs: DF (3n), dS (3n x m), Ef (m) when non-NULL.  Returns the number
 * of over-stretched springs of the proposed configuration (0 = accepted);
 * a negative value -k means the input configuration already had k of them. */
int32_t oracle_step(const oracle_params *p, double *R, const double *dW, int32_t m,
                    double dmin, double dmax, int32_t nch, double *DF_out, double *dS_out,
                    double *Ef_out)
{
    int n = p->n;
    long n3 = 3L * n;
    double *D = (double *)malloc(sizeof(double) * (size_t)(n3 * n3));
    double *F = (double *)malloc(sizeof(double) * (size_t)n3);
    double *DF = (double *)malloc(sizeof(double) * (size_t)n3);
    double *dS = (double *)malloc(sizeof(double) * (size_t)(n3 * m));
    double *Rn = (double *)malloc(sizeof(double) * (size_t)n3);
    int32_t bad = oracle_forces(p, R, F);
    int32_t ret = 0;
    if (bad) { ret = -bad; goto done; }
    oracle_build_D(p, R, D);
    oracle_apply_D((int32_t)n3, D, F, 1, DF);
    oracle_cheb_sqrt((int32_t)n3, D, dmin, dmax, nch, dW, m, dS, Ef_out);
    for (long i = 0; i < n3; i++)
#ifdef PLANT_STEP_DRIFT
        Rn[i] = R[i] + 0.5 * p->dt * DF[i] + dS[i] / sqrt(2.0);
#else
        Rn[i] = R[i] + 0.25 * p->dt * DF[i] + dS[i] / sqrt(2.0);
#endif
    if (p->spring == 1) {
        int32_t over = 0;
        for (int c = 0; c < n / p->nb; c++)
            for (int j = 0; j + 1 < p->nb; j++) {
                int mu = c * p->nb + j;
                double q2 = 0.0;
                for (int s = 0; s < 3; s++) {
                    double q = Rn[3 * (mu + 1) + s] - Rn[3 * mu + s];
                    q2 += q * q;
                }
                if (q2 >= p->fene_b) over++;
            }
        ret = over;
    }
    if (ret == 0) memcpy(R, Rn, sizeof(double) * (size_t)n3);
    if (DF_out) memcpy(DF_out, DF, sizeof(double) * (size_t)n3);
    if (dS_out) memcpy(dS_out, dS, sizeof(double) * (size_t)(n3 * m));
done:
    free(D); free(F); free(DF); free(dS); free(Rn);
    return ret;
}


/* ------------------------------------------------------------------------ */
/* Gradient of L = g . D(R) F with respect to R (the adjoint of the drift
 * product of Eq. sde; dL/dF = D g is a plain product).  D_{nu mu} = B(d),
 * d = r_nu - r_mu, with B the pair tensor of Eq. (DFmodified); the diagonal
 * blocks do not depend on R.  For each ordered pair,
 *   dL/dr_nu^c += sum_ab dB_ab/dd_c (d) W_ab,  W_ab = g_nu^a F_mu^b + g_mu^a F_nu^b,
 * and dB/dd is the analytic derivative of the image sum of M1 (Eq. M1), of
 * M* (Eq. cor5, reading R2) and of the reciprocal sum (Eq. M2).            */

/* dc1/dr and dc2/dr of Eq. (M1) written out by hand, with s = alpha r. */
static void m1_coeffs_dr(double r, double a, double al, double *d1, double *d2)
{
    double a3 = a * a * a, r2 = r * r, r3 = r2 * r, r4 = r2 * r2, r5 = r4 * r;
    double al2 = al * al, al3 = al2 * al, al5 = al3 * al2, al7 = al5 * al2;
    double ec = erfc(al * r);
    double ex = exp(-al2 * r2) / sqrt(PI);
    double dec = -2.0 * al * ex;                   /* d erfc(alpha r)/dr      */
    double dex = -2.0 * al2 * r * ex;              /* d [exp(-a^2r^2)/sqrt(pi)]/dr */
    double p1 = 3.0 * a * al3 * r2 - 9.0 * a * al / 2.0 + 4.0 * a3 * al7 * r4
              - 20.0 * a3 * al5 * r2 + 14.0 * a3 * al3 + a3 * al / r2;
    double dp1 = 6.0 * a * al3 * r + 16.0 * a3 * al7 * r3 - 40.0 * a3 * al5 * r
               - 2.0 * a3 * al / r3;
    double p2 = 3.0 * a * al / 2.0 - 3.0 * a * al3 * r2 - 4.0 * a3 * al7 * r4
              + 16.0 * a3 * al5 * r2 - 2.0 * a3 * al3 - 3.0 * a3 * al / r2;
    double dp2 = -6.0 * a * al3 * r - 16.0 * a3 * al7 * r3 + 32.0 * a3 * al5 * r
               + 6.0 * a3 * al / r3;
    double q1 = 3.0 * a / (4.0 * r) + a3 / (2.0 * r3);
    double dq1 = -3.0 * a / (4.0 * r2) - 3.0 * a3 / (2.0 * r4);
    double q2 = 3.0 * a / (4.0 * r) - 3.0 * a3 / (2.0 * r3);
    double dq2 = -3.0 * a / (4.0 * r2) + 9.0 * a3 / (2.0 * r4);
    (void)r5;
    *d1 = dec * q1 + ec * dq1 + dex * p1 + ex * dp1;
    *d2 = dec * q2 + ec * dq2 + dex * p2 + ex * dp2;
}

/* d/dd_c of f1(r) I + f2(r) rhat rhat contracted with W, added to out[c]. */
static void add_radial_grad(const double v[3], double r, double f1, double f2, double df1,
                            double df2, const double W[9], double out[3])
{
    double trW = W[0] + W[4] + W[8];
    double vWv = 0.0, Wv[3], WTv[3];
    for (int i = 0; i < 3; i++) {
        Wv[i] = W[3 * i] * v[0] + W[3 * i + 1] * v[1] + W[3 * i + 2] * v[2];
        WTv[i] = W[i] * v[0] + W[3 + i] * v[1] + W[6 + i] * v[2];
        vWv += v[i] * Wv[i];
    }
    double r2 = r * r;
    for (int c = 0; c < 3; c++) {
        double e = v[c] / r;                        /* dr/dd_c */
        out[c] += df1 * e * trW                     /* f1' e_c delta_ab            */
                + df2 * e * vWv / r2                /* f2' e_c v_a v_b / r^2       */
                + f2 * (Wv[c] + WTv[c]) / r2        /* f2 (delta_ac v_b + v_a delta_bc)/r^2 */
                - 2.0 * f2 * vWv * v[c] / (r2 * r2);/* f2 v_a v_b d(1/r^2)/dd_c    */
    }
}

/* General form: dL/dR for dL/dD = G = sum_q x_q y_q^T (Q pairs of 3N-vectors,
 * X and Y stored [q][3N]); the drift adjoint is Q = 1 with x = g, y = F. */
void oracle_grad_pairs_R(const oracle_params *p, const double *R, const double *X, const double *Y,
                         int32_t Q, double *gR);

void oracle_grad_DF_R(const oracle_params *p, const double *R, const double *F, const double *g,
                      double *gR)
{
    oracle_grad_pairs_R(p, R, g, F, 1, gR);
}

void oracle_grad_pairs_R(const oracle_params *p, const double *R, const double *X, const double *Y,
                         int32_t Q, double *gR)
{
    kterm *kl;
    int nk = build_klist(p, &kl);
    int n = p->n;
    double L = p->L, a = p->a, al = p->alpha, rc2 = p->rc * p->rc;
    int nmax = (int)floor(p->rc / L + 0.5) + 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int nu = 0; nu < n; nu++) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int mu = 0; mu < n; mu++) {
            if (mu == nu) continue;
            double W[9];
            long n3 = 3L * n;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    double w = 0.0;
                    for (int q = 0; q < Q; q++)
                        w += X[q * n3 + 3 * nu + i] * Y[q * n3 + 3 * mu + j]
                           + X[q * n3 + 3 * mu + i] * Y[q * n3 + 3 * nu + j];
                    W[3 * i + j] = w;
                }
            double d[3];
            for (int i = 0; i < 3; i++) {
                d[i] = R[3 * nu + i] - R[3 * mu + i];
                d[i] -= L * nearbyint(d[i] / L);
            }
            for (int nx = -nmax; nx <= nmax; nx++)
                for (int ny = -nmax; ny <= nmax; ny++)
                    for (int nz = -nmax; nz <= nmax; nz++) {
                        double v[3] = {d[0] + nx * L, d[1] + ny * L, d[2] + nz * L};
                        double u = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                        if (u > rc2 || u == 0.0) continue;
                        double r = sqrt(u), c1, c2, d1, d2;
                        m1_coeffs(r, a, al, &c1, &c2);
                        m1_coeffs_dr(r, a, al, &d1, &d2);
                        add_radial_grad(v, r, c1, c2, d1, d2, W, acc);
                        if (p->overlap_corr && u < 4.0 * a * a) {
                            /* M* of Eq. (cor5), reading R2, with x = r/a */
                            double x = r / a, x2 = x * x, x3 = x2 * x, x4 = x2 * x2;
                            double q = 0.75 * x2 + 1.0;
                            double s1 = 1.0 - q * q / (2.0 * x3);
                            double ds1 = (-(2.0 * q * 1.5 * x) * 2.0 * x3 + q * q * 6.0 * x2)
                                       / (4.0 * x3 * x3) / a;
                            double s2 = 3.0 * (x2 - 4.0) * (x2 - 4.0) / (32.0 * x3);
                            double ds2 = (3.0 * 2.0 * (x2 - 4.0) * 2.0 * x * 32.0 * x3
                                          - 3.0 * (x2 - 4.0) * (x2 - 4.0) * 96.0 * x2)
                                       / (1024.0 * x3 * x3) / a;
                            (void)x4;
                            add_radial_grad(v, r, s1, s2, ds1, ds2, W, acc);
                        }
                    }
            for (int t = 0; t < nk; t++) {
                const double *k = kl[t].k;
                double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                double sn = sin(k[0] * d[0] + k[1] * d[1] + k[2] * d[2]);
                double mw = 0.0;
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++)
                        mw += kl[t].f * ((i == j ? 1.0 : 0.0) - k[i] * k[j] / k2) * W[3 * i + j];
                for (int c = 0; c < 3; c++) acc[c] -= mw * k[c] * sn;
            }
        }
        for (int c = 0; c < 3; c++) gR[3 * nu + c] = acc[c];
    }
    free(kl);
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
 * SC'11), written from its published definition: ten rounds of
 * (hi,lo) = mulhilo(M, x) on words 0 and 2, key bumped by the Weyl
 * constants between rounds.                                               */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Wiener increments from Philox: element pair q uses counter
 * (q_lo, q_hi, step_lo, step_hi) and key (seed_lo, seed_hi); the four words
 * give two 53-bit uniforms u1, u2 in (0,1) and the Box-Muller pair
 * sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2), scaled by sqrt(dt).          */
void oracle_wiener_philox(uint64_t seed, uint64_t step, int64_t count, double dt, double *out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double sdt = sqrt(dt);
    for (int64_t q = 0; 2 * q < count; q++) {
        uint32_t ctr[4] = {(uint32_t)q, (uint32_t)((uint64_t)q >> 32), (uint32_t)step,
                           (uint32_t)(step >> 32)};
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        uint64_t b1 = ((uint64_t)w[0] << 32) | w[1];
        uint64_t b2 = ((uint64_t)w[2] << 32) | w[3];
        double u1 = ((double)(b1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        double u2 = ((double)(b2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        double rr = sqrt(-2.0 * log(u1));
        out[2 * q] = sdt * rr * cos(2.0 * PI * u2);
        if (2 * q + 1 < count) out[2 * q + 1] = sdt * rr * sin(2.0 * PI * u2);
    }
}

int32_t oracle_num_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
