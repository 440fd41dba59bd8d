/*
 * Oracle (test infrastructure only): plain FP64 periodic sums of the Laplace
 * and Stokes-velocity kernels, Eq. (pfmmDef) of Sec. 2.2 with the kernels of
 * Eq. (kexamples), Sec. 2.4, and of the Laplace field (gradient) at the end.  Only tests/, the smoke check and the CPU
 * baseline leg of the benchmark may call this code.  It shares nothing with
 * the CUDA library: it is written from the textbook definitions, with no
 * blocking, fusion or reordering beyond what those definitions state.
 *
 * Conventions (all functions):
 *   y[S][3] sources, x[T][3] targets, box B0 = [0,L)^3 (cubic).
 *   Laplace: phi[S], q[T];   K = 1/r.
 *   Stokes:  phi[S][3], q[T][3];  K = (1/8pi)(I/r + r r^T / r^3)  (mu = 1).
 *   A source image that coincides with the target (the p = 0, s = t term) is
 *   excluded, as in the statement of the problem.
 *   Sums are accumulated with Neumaier compensation.
 *
 * Periodic sums (K^P of Sec. 2.1) are made absolutely convergent by Ewald
 * splitting:
 *   - Laplace TP: erfc real-space sum + Fourier sum with the k = 0 mode
 *     removed, plus the -pi/(xi^2 V) sum(phi) background term (zero for the
 *     neutral charges the compatibility condition Eq. (compatcondition)
 *     requires).
 *   - Stokes TP: Hasimoto split (Sec. 3.4): Fourier weight
 *     (1 + k^2/4xi^2) exp(-k^2/4xi^2) (I - k k^T/k^2)/k^2, k = 0 removed
 *     (zero mean flow, Eq. (flowvolume)); the real-space kernel follows in
 *     closed form: with S = (I lap - grad grad) r the smooth part is
 *     (I lap - grad grad) B, B' = erf(xi r), B'' = (2 xi/sqrt(pi)) e^{-xi^2 r^2},
 *     leaving I (erfc(xi r)/r - 2xi/sqrt(pi) e^{-xi^2 r^2})
 *     + (r r^T/r^2)(erfc(xi r)/r + 2xi/sqrt(pi) e^{-xi^2 r^2}) (over 8 pi) in real
 *     space and the self term -(4 xi/sqrt(pi))/(8 pi).
 *   - Laplace SP: direct symmetric image sum |n| <= M with a per-pair
 *     regularisation -2 H_M and an Euler-Maclaurin tail (Sec. 3.2 notes the
 *     neutral direct sum converges like 1/n^2); the pair-independent constant
 *     cancels by neutrality.
 *   - Laplace / Stokes DP (periodic in x and y, z free; Sec. 3.3 leaves the
 *     doubly periodic Ewald sum to the literature): the same real-space
 *     kernels summed over in-plane images only; the smooth part as the 2D
 *     lattice sum of its 3D Fourier transform, whose k_z integral is taken by
 *     the trapezoid rule for every in-plane mode k_par != 0 and in closed
 *     form for k_par = 0 (a function of z_t - z_s alone); constants dropped
 *     from the k_par = 0 term cancel for neutral charges / zero net
 *     in-plane force.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------- Neumaier compensated accumulator ---------- */
typedef struct { double s, c; } acc_t;
static inline void acc_add(acc_t *a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static inline double acc_get(const acc_t *a) { return a->s + a->c; }

/* ---------- free-space kernels ---------- */
static inline void stokeslet(const double d[3], double r, double G[9]) {
    double ir = 1.0 / r, ir3 = ir * ir * ir, c = 1.0 / (8.0 * M_PI);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            G[3 * i + j] = c * ((i == j ? ir : 0.0) + d[i] * d[j] * ir3);
}

/* Free-space direct sum q_t = sum_s K(x_t, y_s) phi_s, coincident pairs excluded. */
void orc_free(int kernel, long S, const double *y, const double *phi, long T,
              const double *x, double *q) {
    int k = kernel == 0 ? 1 : 3;
#pragma omp parallel for schedule(dynamic, 8)
    for (long t = 0; t < T; t++) {
        acc_t a[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (long s = 0; s < S; s++) {
            double d[3] = {x[3 * t] - y[3 * s], x[3 * t + 1] - y[3 * s + 1], x[3 * t + 2] - y[3 * s + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            if (k == 1) {
                acc_add(&a[0], phi[s] / r);
            } else {
                double G[9];
                stokeslet(d, r, G);
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) acc_add(&a[i], G[3 * i + j] * phi[3 * s + j]);
            }
        }
        for (int i = 0; i < k; i++) q[k * t + i] = acc_get(&a[i]);
    }
}

/* ---------- triply periodic Ewald ---------- */

/* Wave vectors m (integer, unit cell) of a half space with 0 < |2 pi m| < kc. */
static long half_space_modes(int mmax, double kc, int **out) {
    long cap = (long)(2 * mmax + 1) * (2 * mmax + 1) * (2 * mmax + 1), n = 0;
    int *m = (int *)malloc(sizeof(int) * 3 * cap);
    for (int mz = 0; mz <= mmax; mz++)
        for (int my = -mmax; my <= mmax; my++)
            for (int mx = -mmax; mx <= mmax; mx++) {
                if (mz == 0 && (my < 0 || (my == 0 && mx <= 0))) continue;
                double k = 2.0 * M_PI * sqrt((double)(mx * mx + my * my + mz * mz));
                if (k >= kc) continue;
                m[3 * n] = mx; m[3 * n + 1] = my; m[3 * n + 2] = mz; n++;
            }
    *out = m;
    return n;
}

/* Structure factors F_c(m) = sum_s phi_s,c exp(-i 2 pi m.y_s) (unit cell),
 * for nc density components; re/im laid out [nm][nc]. */
static void structure_factors(long S, const double *y, const double *phi, int nc, double L,
                              int mmax, long nm, const int *m, double *re, double *im) {
    int w = 2 * mmax + 1;
    memset(re, 0, sizeof(double) * nm * nc);
    memset(im, 0, sizeof(double) * nm * nc);
#pragma omp parallel
    {
        double *lre = (double *)calloc(nm * nc, sizeof(double));
        double *lim = (double *)calloc(nm * nc, sizeof(double));
        double *ec = (double *)malloc(sizeof(double) * 3 * w), *es = (double *)malloc(sizeof(double) * 3 * w);
#pragma omp for schedule(static)
        for (long s = 0; s < S; s++) {
            for (int a = 0; a < 3; a++)
                for (int j = -mmax; j <= mmax; j++) {
                    double th = -2.0 * M_PI * j * (y[3 * s + a] / L);
                    ec[a * w + j + mmax] = cos(th);
                    es[a * w + j + mmax] = sin(th);
                }
            for (long i = 0; i < nm; i++) {
                int ix = m[3 * i] + mmax, iy = m[3 * i + 1] + mmax, iz = m[3 * i + 2] + mmax;
                double xr = ec[ix], xi_ = es[ix], yr = ec[w + iy], yi = es[w + iy], zr = ec[2 * w + iz], zi = es[2 * w + iz];
                double pr = xr * yr - xi_ * yi, pi_ = xr * yi + xi_ * yr;
                double er = pr * zr - pi_ * zi, ei = pr * zi + pi_ * zr;
                for (int c = 0; c < nc; c++) {
                    double v = phi[(long)nc * s + c];
                    lre[i * nc + c] += v * er;
                    lim[i * nc + c] += v * ei;
                }
            }
        }
#pragma omp critical
        for (long i = 0; i < nm * nc; i++) { re[i] += lre[i]; im[i] += lim[i]; }
        free(lre); free(lim); free(ec); free(es);
    }
}

/* Laplace TP Ewald.  Unit-cell quantities (r/L), result scaled by 1/L.
 * xi: splitting parameter (unit cell), rc: real-space cutoff (unit cell),
 * mmax / kc: Fourier cutoff |2 pi m| < kc with |m_a| <= mmax. */
void orc_laplace_tp(long S, const double *y, const double *phi, long T, const double *x,
                    double L, double xi, double rc, int mmax, double kc, double *q) {
    int *m; long nm = half_space_modes(mmax, kc, &m);
    double *re = (double *)malloc(sizeof(double) * nm), *im = (double *)malloc(sizeof(double) * nm);
    structure_factors(S, y, phi, 1, L, mmax, nm, m, re, im);
    double *wk = (double *)malloc(sizeof(double) * nm);
    for (long i = 0; i < nm; i++) {
        double k2 = 4.0 * M_PI * M_PI * (double)(m[3 * i] * m[3 * i] + m[3 * i + 1] * m[3 * i + 1] + m[3 * i + 2] * m[3 * i + 2]);
        wk[i] = 2.0 * (4.0 * M_PI) * exp(-k2 / (4.0 * xi * xi)) / k2; /* x2: +m and -m */
    }
    acc_t tot = {0, 0};
    for (long s = 0; s < S; s++) acc_add(&tot, phi[s]);
    double background = -M_PI * acc_get(&tot) / (xi * xi);
    int nr = rc > 0.5 ? (int)ceil(rc - 0.5) : 0;
    double rc2 = rc * rc, self = -2.0 * xi / sqrt(M_PI);
#pragma omp parallel for schedule(dynamic, 4)
    for (long t = 0; t < T; t++) {
        acc_t a = {0, 0};
        for (long s = 0; s < S; s++) {
            double r[3];
            for (int c = 0; c < 3; c++) { r[c] = (x[3 * t + c] - y[3 * s + c]) / L; r[c] -= floor(r[c] + 0.5); }
            for (int n0 = -nr; n0 <= nr; n0++)
                for (int n1 = -nr; n1 <= nr; n1++)
                    for (int n2 = -nr; n2 <= nr; n2++) {
                        double d0 = r[0] + n0, d1 = r[1] + n1, d2 = r[2] + n2;
                        double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                        if (r2 == 0.0) { acc_add(&a, self * phi[s]); continue; }
                        if (r2 >= rc2) continue;
                        double rr = sqrt(r2);
                        acc_add(&a, erfc(xi * rr) / rr * phi[s]);
                    }
        }
        for (long i = 0; i < nm; i++) {
            double th = 2.0 * M_PI * (m[3 * i] * x[3 * t] + m[3 * i + 1] * x[3 * t + 1] + m[3 * i + 2] * x[3 * t + 2]) / L;
            acc_add(&a, wk[i] * (re[i] * cos(th) - im[i] * sin(th)));
        }
        acc_add(&a, background);
        q[t] = acc_get(&a) / L;
    }
    free(m); free(re); free(im); free(wk);
}

/* Stokes TP Ewald, zero mean flow.  split = 0: Hasimoto (Fourier weight
 * (1 + a) e^{-a}, a = k^2/4xi^2); split = 1: Beenakker (weight
 * (1 + a + 2a^2) e^{-a}, i.e. (1 + k^2/4xi^2 + k^4/8xi^4) e^{-k^2/4xi^2}).  The
 * Beenakker smooth part adds B_x = -e^{-xi^2 r^2}/(8 xi pi^{3/2}) to the
 * biharmonic potential B (S = (I lap - grad grad) B), which moves
 * 2 g0 e^{-xi^2 r^2} [I (1 - xi^2 r^2) + r r^T xi^2] / (8 pi) from the real-space
 * kernel to the smooth part and adds -2 g0/(8 pi) to the self term
 * (g0 = 2 xi/sqrt(pi)).  Same other parameters. */
static void stokes_tp_split(long S, const double *y, const double *f, long T, const double *x,
                            double L, double xi, double rc, int mmax, double kc, int split, double *u);

void orc_stokes_tp(long S, const double *y, const double *f, long T, const double *x,
                   double L, double xi, double rc, int mmax, double kc, double *u) {
    stokes_tp_split(S, y, f, T, x, L, xi, rc, mmax, kc, 0, u);
}

void orc_stokes_tp_beenakker(long S, const double *y, const double *f, long T, const double *x,
                             double L, double xi, double rc, int mmax, double kc, double *u) {
    stokes_tp_split(S, y, f, T, x, L, xi, rc, mmax, kc, 1, u);
}

static void stokes_tp_split(long S, const double *y, const double *f, long T, const double *x,
                            double L, double xi, double rc, int mmax, double kc, int split, double *u) {
    int *m; long nm = half_space_modes(mmax, kc, &m);
    double *re = (double *)malloc(sizeof(double) * nm * 3), *im = (double *)malloc(sizeof(double) * nm * 3);
    structure_factors(S, y, f, 3, L, mmax, nm, m, re, im);
    double *wk = (double *)malloc(sizeof(double) * nm);
    for (long i = 0; i < nm; i++) {
        double k2 = 4.0 * M_PI * M_PI * (double)(m[3 * i] * m[3 * i] + m[3 * i + 1] * m[3 * i + 1] + m[3 * i + 2] * m[3 * i + 2]);
        double a = k2 / (4.0 * xi * xi);
        wk[i] = 2.0 * (1.0 + a + (split ? 2.0 * a * a : 0.0)) * exp(-a) / k2; /* x2: +m and -m; 8 pi / 8 pi = 1 */
    }
    int nr = rc > 0.5 ? (int)ceil(rc - 0.5) : 0;
    double rc2 = rc * rc, c8 = 1.0 / (8.0 * M_PI), g0 = 2.0 * xi / sqrt(M_PI);
    double self = -c8 * 4.0 * xi / sqrt(M_PI) - (split ? 2.0 * c8 * g0 : 0.0);
#pragma omp parallel for schedule(dynamic, 4)
    for (long t = 0; t < T; t++) {
        acc_t a[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (long s = 0; s < S; s++) {
            const double *fs = f + 3 * s;
            double r[3];
            for (int c = 0; c < 3; c++) { r[c] = (x[3 * t + c] - y[3 * s + c]) / L; r[c] -= floor(r[c] + 0.5); }
            for (int n0 = -nr; n0 <= nr; n0++)
                for (int n1 = -nr; n1 <= nr; n1++)
                    for (int n2 = -nr; n2 <= nr; n2++) {
                        double d[3] = {r[0] + n0, r[1] + n1, r[2] + n2};
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 == 0.0) {
                            for (int i = 0; i < 3; i++) acc_add(&a[i], self * fs[i]);
                            continue;
                        }
                        if (r2 >= rc2) continue;
                        double rr = sqrt(r2), ec = erfc(xi * rr) / rr, ga = g0 * exp(-xi * xi * r2);
                        double cI = ec - ga, cR = (ec + ga) / r2; /* I and r r^T coefficients */
                        if (split) { /* minus the part that moved to the smooth side */
                            cI -= 2.0 * ga * (1.0 - xi * xi * r2);
                            cR -= 2.0 * ga * xi * xi;
                        }
                        double df = d[0] * fs[0] + d[1] * fs[1] + d[2] * fs[2];
                        for (int i = 0; i < 3; i++) acc_add(&a[i], c8 * (cI * fs[i] + cR * d[i] * df));
                    }
        }
        for (long i = 0; i < nm; i++) {
            double k[3] = {2.0 * M_PI * m[3 * i], 2.0 * M_PI * m[3 * i + 1], 2.0 * M_PI * m[3 * i + 2]};
            double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
            double th = (k[0] * x[3 * t] + k[1] * x[3 * t + 1] + k[2] * x[3 * t + 2]) / L;
            double ct = cos(th), st = sin(th), v[3];
            for (int c = 0; c < 3; c++) v[c] = re[i * 3 + c] * ct - im[i * 3 + c] * st;
            double kv = (k[0] * v[0] + k[1] * v[1] + k[2] * v[2]) / k2;
            for (int c = 0; c < 3; c++) acc_add(&a[c], wk[i] * (v[c] - k[c] * kv));
        }
        for (int c = 0; c < 3; c++) u[3 * t + c] = acc_get(&a[c]) / L;
    }
    free(m); free(re); free(im); free(wk);
}

/* ---------- singly periodic Laplace ---------- */

/* Regularised 1D lattice sum for one pair: axial offset a (unit period),
 * perpendicular distance^2 rho2:
 *   sum_{|n|<=M} 1/|r + n e|  - 2 H_M  + sum_{n>M} [1/|r+ne| + 1/|r-ne| - 2/n]
 * The last sum is the Euler-Maclaurin tail from n0 = M+1:
 *   int_{n0}^inf g + g(n0)/2 - g'(n0)/12.
 * The term with r + n e = 0 (coincident image) is excluded. */
static double sp_pair(double a, double rho2, long M) {
    acc_t s = {0, 0};
    for (long n = -M; n <= M; n++) {
        double z = a + (double)n, r2 = z * z + rho2;
        if (r2 == 0.0) continue;
        acc_add(&s, 1.0 / sqrt(r2));
    }
    for (long n = M; n >= 1; n--) acc_add(&s, -2.0 / (double)n);
    double n0 = (double)(M + 1);
    double zp = n0 + a, zm = n0 - a;
    double Rp = sqrt(zp * zp + rho2), Rm = sqrt(zm * zm + rho2);
    /* int_{n0}^inf g dn = -log((zp+Rp)/(2 n0)) - log((zm+Rm)/(2 n0)), via log1p */
    double up = (a + (2.0 * n0 * a + a * a + rho2) / (Rp + n0)) / (2.0 * n0);
    double um = (-a + (-2.0 * n0 * a + a * a + rho2) / (Rm + n0)) / (2.0 * n0);
    double integral = -log1p(up) - log1p(um);
    double g = 1.0 / Rp + 1.0 / Rm - 2.0 / n0;
    double dg = -zp / (Rp * Rp * Rp) - zm / (Rm * Rm * Rm) + 2.0 / (n0 * n0);
    acc_add(&s, integral);
    acc_add(&s, 0.5 * g);
    acc_add(&s, -dg / 12.0);
    return acc_get(&s);
}

void orc_laplace_sp(long S, const double *y, const double *phi, long T, const double *x,
                    int axis, double L, long M, double *q) {
#pragma omp parallel for schedule(dynamic, 4)
    for (long t = 0; t < T; t++) {
        acc_t a = {0, 0};
        for (long s = 0; s < S; s++) {
            double r[3];
            for (int c = 0; c < 3; c++) r[c] = (x[3 * t + c] - y[3 * s + c]) / L;
            double ax = r[axis] - floor(r[axis] + 0.5);
            double rho2 = 0.0;
            for (int c = 0; c < 3; c++) if (c != axis) rho2 += r[c] * r[c];
            acc_add(&a, phi[s] * sp_pair(ax, rho2, M));
        }
        q[t] = acc_get(&a) / L;
    }
}

/* ---------- doubly periodic (x, y periodic, z free) ---------- */

/* Structure factors F_c(m) = sum_s phi_s,c exp(-i 2 pi sum_a m_a y_s,a / P_a)
 * for per-axis periods P (unit cell: 1, 1, H) and per-axis |m_a| <= mm[a]. */
static void structure_factors_box(long S, const double *y, const double *phi, int nc, double L,
                                  const int mm[3], const double P[3], long nm, const int *m,
                                  double *re, double *im) {
    int w[3] = {2 * mm[0] + 1, 2 * mm[1] + 1, 2 * mm[2] + 1}, off[3] = {0, w[0], w[0] + w[1]};
    int wt = w[0] + w[1] + w[2];
    memset(re, 0, sizeof(double) * nm * nc);
    memset(im, 0, sizeof(double) * nm * nc);
#pragma omp parallel
    {
        double *lre = (double *)calloc(nm * nc, sizeof(double));
        double *lim = (double *)calloc(nm * nc, sizeof(double));
        double *ec = (double *)malloc(sizeof(double) * wt), *es = (double *)malloc(sizeof(double) * wt);
#pragma omp for schedule(static)
        for (long s = 0; s < S; s++) {
            for (int a = 0; a < 3; a++)
                for (int j = -mm[a]; j <= mm[a]; j++) {
                    double th = -2.0 * M_PI * j * (y[3 * s + a] / L) / P[a];
                    ec[off[a] + j + mm[a]] = cos(th);
                    es[off[a] + j + mm[a]] = sin(th);
                }
            for (long i = 0; i < nm; i++) {
                int ix = off[0] + m[3 * i] + mm[0], iy = off[1] + m[3 * i + 1] + mm[1], iz = off[2] + m[3 * i + 2] + mm[2];
                double xr = ec[ix], xi_ = es[ix], yr = ec[iy], yi = es[iy], zr = ec[iz], zi = es[iz];
                double pr = xr * yr - xi_ * yi, pi_ = xr * yi + xi_ * yr;
                double er = pr * zr - pi_ * zi, ei = pr * zi + pi_ * zr;
                for (int c = 0; c < nc; c++) {
                    double v = phi[(long)nc * s + c];
                    lre[i * nc + c] += v * er;
                    lim[i * nc + c] += v * ei;
                }
            }
        }
#pragma omp critical
        for (long i = 0; i < nm * nc; i++) { re[i] += lre[i]; im[i] += lim[i]; }
        free(lre); free(lim); free(ec); free(es);
    }
}

/* Doubly periodic Ewald sum, periods L along x and y, z free.
 * kernel 0: Laplace (phi[S], q[T]);  kernel 1: Stokes (phi[S][3], q[T][3]).
 * xi, rc: splitting parameter and real-space cutoff (unit cell);
 * kc: Fourier cutoff; H: z period (unit cells) of the trapezoid rule in k_z,
 * which must exceed the z extent of sources and targets by enough that
 * exp(-2 pi (H - extent)) is negligible.
 * Unit-cell area A = 1.  Per pair (r = x_t - y_s, unit cell):
 *   real space  sum_{n in Z^2} K_R(r + n), the same kernels as in TP;
 *   k_par != 0  (1/H) sum_{k = (2pi mx, 2pi my, 2pi mz/H)} K_F^(k) e^{i k.r};
 *   k_par = 0   Laplace 4 pi [-(z/2) erf(xi z) - e^{-xi^2 z^2}/(2 xi sqrt(pi))],
 *               Stokes (I - e_z e_z) [-(z/2) erf(xi z) - e^{-xi^2 z^2}/(4 xi sqrt(pi))],
 *               z = z_t - z_s: the k_z integral of K_F^(0, 0, k_z) (e^{i k_z z} - 1)
 *               with z-independent constants dropped;
 *   self        as in TP. */
void orc_dp(int kernel, long S, const double *y, const double *phi, long T, const double *x,
            double L, double xi, double rc, double kc, double H, double *q) {
    const int nc = kernel == 0 ? 1 : 3;
    int mm[3] = {(int)ceil(kc / (2.0 * M_PI)), (int)ceil(kc / (2.0 * M_PI)), (int)ceil(kc * H / (2.0 * M_PI))};
    double P[3] = {1.0, 1.0, H};
    long cap = (long)(2 * mm[0] + 1) * (2 * mm[1] + 1) * (mm[2] + 1), nm = 0;
    int *m = (int *)malloc(sizeof(int) * 3 * cap);
    for (int mz = 0; mz <= mm[2]; mz++)
        for (int my = -mm[1]; my <= mm[1]; my++)
            for (int mx = -mm[0]; mx <= mm[0]; mx++) {
                if (mx == 0 && my == 0) continue; /* k_par = 0 handled in closed form */
                if (mz == 0 && (my < 0 || (my == 0 && mx <= 0))) continue;
                double kx = 2.0 * M_PI * mx, ky = 2.0 * M_PI * my, kz = 2.0 * M_PI * mz / H;
                if (kx * kx + ky * ky + kz * kz >= kc * kc) continue;
                m[3 * nm] = mx; m[3 * nm + 1] = my; m[3 * nm + 2] = mz; nm++;
            }
    double *re = (double *)malloc(sizeof(double) * (nm ? nm : 1) * nc);
    double *im = (double *)malloc(sizeof(double) * (nm ? nm : 1) * nc);
    structure_factors_box(S, y, phi, nc, L, mm, P, nm, m, re, im);
    int nr = rc > 0.5 ? (int)ceil(rc - 0.5) : 0;
    double rc2 = rc * rc, g0 = 2.0 * xi / sqrt(M_PI), c8 = 1.0 / (8.0 * M_PI), sqpi = sqrt(M_PI);
#pragma omp parallel for schedule(dynamic, 4)
    for (long t = 0; t < T; t++) {
        acc_t a[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (long s = 0; s < S; s++) {
            const double *fs = phi + (long)nc * s;
            double r[3];
            for (int c = 0; c < 3; c++) r[c] = (x[3 * t + c] - y[3 * s + c]) / L;
            for (int c = 0; c < 2; c++) r[c] -= floor(r[c] + 0.5);
            for (int n0 = -nr; n0 <= nr; n0++)
                for (int n1 = -nr; n1 <= nr; n1++) {
                    double d[3] = {r[0] + n0, r[1] + n1, r[2]};
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 == 0.0) {
                        if (kernel == 0) acc_add(&a[0], -g0 * fs[0]);
                        else
                            for (int i = 0; i < 3; i++) acc_add(&a[i], -c8 * 2.0 * g0 * fs[i]);
                        continue;
                    }
                    if (r2 >= rc2) continue;
                    double rr = sqrt(r2);
                    if (kernel == 0) {
                        acc_add(&a[0], erfc(xi * rr) / rr * fs[0]);
                    } else {
                        double ec = erfc(xi * rr) / rr, ga = g0 * exp(-xi * xi * r2);
                        double cI = ec - ga, cR = (ec + ga) / r2;
                        double df = d[0] * fs[0] + d[1] * fs[1] + d[2] * fs[2];
                        for (int i = 0; i < 3; i++) acc_add(&a[i], c8 * (cI * fs[i] + cR * d[i] * df));
                    }
                }
            /* k_par = 0 term */
            double z = r[2], ez = exp(-xi * xi * z * z), lin = -0.5 * z * erf(xi * z);
            if (kernel == 0) {
                acc_add(&a[0], 4.0 * M_PI * (lin - ez / (2.0 * xi * sqpi)) * fs[0]);
            } else {
                double g = lin - ez / (4.0 * xi * sqpi);
                acc_add(&a[0], g * fs[0]);
                acc_add(&a[1], g * fs[1]);
            }
        }
        for (long i = 0; i < nm; i++) {
            double k[3] = {2.0 * M_PI * m[3 * i], 2.0 * M_PI * m[3 * i + 1], 2.0 * M_PI * m[3 * i + 2] / H};
            double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2], e = k2 / (4.0 * xi * xi);
            double th = (k[0] * x[3 * t] + k[1] * x[3 * t + 1] + k[2] * x[3 * t + 2]) / L;
            double ct = cos(th), st = sin(th);
            if (kernel == 0) {
                double wk = 2.0 * 4.0 * M_PI / H * exp(-e) / k2;
                acc_add(&a[0], wk * (re[i] * ct - im[i] * st));
            } else {
                double wk = 2.0 / H * (1.0 + e) * exp(-e) / k2, v[3];
                for (int c = 0; c < 3; c++) v[c] = re[i * 3 + c] * ct - im[i * 3 + c] * st;
                double kv = (k[0] * v[0] + k[1] * v[1] + k[2] * v[2]) / k2;
                for (int c = 0; c < 3; c++) acc_add(&a[c], wk * (v[c] - k[c] * kv));
            }
        }
        for (int c = 0; c < nc; c++) q[(long)nc * t + c] = acc_get(&a[c]) / L;
    }
    free(m); free(re); free(im);
}

/* ---------- singly periodic Stokes ---------- */

/* Regularised 1D lattice sum of the Stokeslet for one pair, axis `ax`
 * (unit period), r the minimum-image offset:
 *   G = sum_{|n|<=M} S(r + n e) - (1/8pi)(I + e e^T) 2 H_M
 *       + sum_{n>M} [S(r + n e) + S(r - n e) - (1/8pi)(I + e e^T) 2/n],
 * the pair-independent 2 H_M term cancelling for zero net force.  The tail
 * is summed by Euler-Maclaurin from n0 = M + 1 (integral + g/2 - g'/12);
 * the integral is closed form: with w1 = a + n0, w2 = n0 - a (a the axial
 * offset), rho the perpendicular offset, R_i = sqrt(w_i^2 + rho^2),
 * Lg = -ln((w1 + R1)/2n0) - ln((w2 + R2)/2n0), c = 1/8pi:
 *   (e,e)    c [2 Lg + w1/R1 + w2/R2 - 2]
 *   (p,p)    c Lg + c rho_p^2 B,   (p,q) c rho_p rho_q B,
 *            B = 1/(R1 (R1 + w1)) + 1/(R2 (R2 + w2))
 *   (e,p)    c rho_p (1/R1 - 1/R2).
 * The coincident image is excluded. */
static void stokes_grad(const double d[3], int k, double out[9]) {
    /* d/dd_k of S(d), times 8 pi */
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2), ir3 = 1.0 / (r2 * r), ir5 = ir3 / r2;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            out[3 * i + j] = -(i == j ? d[k] * ir3 : 0.0) + ((i == k ? d[j] : 0.0) + (j == k ? d[i] : 0.0)) * ir3 -
                             3.0 * d[i] * d[j] * d[k] * ir5;
}

static void sp_stokes_pair(const double r[3], int ax, long M, double G[9]) {
    const double c = 1.0 / (8.0 * M_PI);
    acc_t s[9];
    memset(s, 0, sizeof s);
    double blk[9];
    for (long n = -M; n <= M; n++) {
        double d[3] = {r[0], r[1], r[2]};
        d[ax] += (double)n;
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 == 0.0) continue;
        stokeslet(d, sqrt(r2), blk);
        for (int i = 0; i < 9; i++) acc_add(&s[i], blk[i]);
    }
    double H = 0.0;
    {
        acc_t h = {0, 0};
        for (long n = M; n >= 1; n--) acc_add(&h, 1.0 / (double)n);
        H = acc_get(&h);
    }
    for (int i = 0; i < 3; i++) {
        acc_add(&s[4 * i], -c * 2.0 * H);
        if (i == ax) acc_add(&s[4 * i], -c * 2.0 * H);
    }
    /* Euler-Maclaurin tail */
    double n0 = (double)(M + 1), a = r[ax], rho2 = 0.0, rho[3] = {0, 0, 0};
    for (int i = 0; i < 3; i++)
        if (i != ax) {
            rho[i] = r[i];
            rho2 += r[i] * r[i];
        }
    double w1 = a + n0, w2 = n0 - a, R1 = sqrt(w1 * w1 + rho2), R2 = sqrt(w2 * w2 + rho2);
    double up = (a + (2.0 * n0 * a + a * a + rho2) / (R1 + n0)) / (2.0 * n0);
    double um = (-a + (-2.0 * n0 * a + a * a + rho2) / (R2 + n0)) / (2.0 * n0);
    double Lg = -log1p(up) - log1p(um);
    double B = 1.0 / (R1 * (R1 + w1)) + 1.0 / (R2 * (R2 + w2));
    double J[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double v;
            if (i == ax && j == ax) v = 2.0 * Lg - rho2 / (R1 * (R1 + w1)) - rho2 / (R2 * (R2 + w2));
            else if (i == ax) v = rho[j] * (1.0 / R1 - 1.0 / R2);
            else if (j == ax) v = rho[i] * (1.0 / R1 - 1.0 / R2);
            else v = (i == j ? Lg : 0.0) + rho[i] * rho[j] * B;
            J[3 * i + j] = c * v;
        }
    /* g(n0) and g'(n0) */
    double dp[3] = {r[0], r[1], r[2]}, dm[3] = {r[0], r[1], r[2]};
    dp[ax] += n0;
    dm[ax] -= n0;
    double Sp[9], Sm[9], Gp[9], Gm[9];
    stokeslet(dp, sqrt(dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2]), Sp);
    stokeslet(dm, sqrt(dm[0] * dm[0] + dm[1] * dm[1] + dm[2] * dm[2]), Sm);
    stokes_grad(dp, ax, Gp);
    stokes_grad(dm, ax, Gm);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            int q = 3 * i + j;
            double reg = (i == j ? 1.0 : 0.0) + (i == ax && j == ax ? 1.0 : 0.0);
            double g = Sp[q] + Sm[q] - c * reg * 2.0 / n0;
            double dg = c * (Gp[q] - Gm[q]) + c * reg * 2.0 / (n0 * n0);
            acc_add(&s[q], J[q]);
            acc_add(&s[q], 0.5 * g);
            acc_add(&s[q], -dg / 12.0);
        }
    for (int i = 0; i < 9; i++) G[i] = acc_get(&s[i]);
}

void orc_stokes_sp(long S, const double *y, const double *f, long T, const double *x,
                   int axis, double L, long M, double *u) {
#pragma omp parallel for schedule(dynamic, 4)
    for (long t = 0; t < T; t++) {
        acc_t a[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (long s = 0; s < S; s++) {
            double r[3], G[9];
            for (int c = 0; c < 3; c++) r[c] = (x[3 * t + c] - y[3 * s + c]) / L;
            r[axis] -= floor(r[axis] + 0.5);
            sp_stokes_pair(r, axis, M, G);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) acc_add(&a[i], G[3 * i + j] * f[3 * s + j]);
        }
        for (int c = 0; c < 3; c++) u[3 * t + c] = acc_get(&a[c]) / L;
    }
}

/* ---------- Laplace field: the gradient of the potential at the target ----------
 * Each periodic sum above is differentiated term by term with respect to the
 * target position (the sums converge uniformly away from the sources):
 *   free space       grad (1/r) = -r / r^3;
 *   real-space term  erfc(xi r)/r -> -(erfc(xi r) + g0 r e^{-xi^2 r^2}) r / r^3,
 *                    g0 = 2 xi/sqrt(pi); the self term is a constant;
 *   Fourier term     w (Re F cos th - Im F sin th), th = k.x
 *                    -> -w k (Re F sin th + Im F cos th);
 *   DP k_par = 0     d/dz of 4 pi [-(z/2) erf(xi z) - e^{-xi^2 z^2}/(2 xi sqrt(pi))]
 *                    = -2 pi erf(xi z);
 *   SP               the image sum term by term, and the Euler-Maclaurin tail
 *                    (integral + g/2 - g'/12) differentiated in closed form in the
 *                    axial offset a and the perpendicular offset rho.
 * Output g[T][3]: unit-cell gradients divided by L^2 (physical units). */

void orc_laplace_grad_free(long S, const double *y, const double *phi, long T, const double *x, double *g) {
#pragma omp parallel for schedule(dynamic, 16)
    for (long t = 0; t < T; t++) {
        acc_t a[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (long s = 0; s < S; s++) {
            double d[3] = {x[3 * t] - y[3 * s], x[3 * t + 1] - y[3 * s + 1], x[3 * t + 2] - y[3 * s + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double ir3 = 1.0 / (r2 * sqrt(r2));
            for (int c = 0; c < 3; c++) acc_add(&a[c], -phi[s] * d[c] * ir3);
        }
        for (int c = 0; c < 3; c++) g[3 * t + c] = acc_get(&a[c]);
    }
}

void orc_laplace_tp_grad(long S, const double *y, const double *phi, long T, const double *x,
                         double L, double xi, double rc, int mmax, double kc, double *g) {
    int *m; long nm = half_space_modes(mmax, kc, &m);
    double *re = (double *)malloc(sizeof(double) * nm), *im = (double *)malloc(sizeof(double) * nm);
    structure_factors(S, y, phi, 1, L, mmax, nm, m, re, im);
    double *wk = (double *)malloc(sizeof(double) * nm);
    for (long i = 0; i < nm; i++) {
        double k2 = 4.0 * M_PI * M_PI * (double)(m[3 * i] * m[3 * i] + m[3 * i + 1] * m[3 * i + 1] + m[3 * i + 2] * m[3 * i + 2]);
        wk[i] = 2.0 * (4.0 * M_PI) * exp(-k2 / (4.0 * xi * xi)) / k2;
    }
    int nr = rc > 0.5 ? (int)ceil(rc - 0.5) : 0;
    double rc2 = rc * rc, g0 = 2.0 * xi / sqrt(M_PI);
#pragma omp parallel for schedule(dynamic, 4)
    for (long t = 0; t < T; t++) {
        acc_t a[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (long s = 0; s < S; s++) {
            double r[3];
            for (int c = 0; c < 3; c++) { r[c] = (x[3 * t + c] - y[3 * s + c]) / L; r[c] -= floor(r[c] + 0.5); }
            for (int n0 = -nr; n0 <= nr; n0++)
                for (int n1 = -nr; n1 <= nr; n1++)
                    for (int n2 = -nr; n2 <= nr; n2++) {
                        double d[3] = {r[0] + n0, r[1] + n1, r[2] + n2};
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 == 0.0 || r2 >= rc2) continue;
                        double rr = sqrt(r2);
                        double cf = -(erfc(xi * rr) + g0 * rr * exp(-xi * xi * r2)) / (r2 * rr);
                        for (int c = 0; c < 3; c++) acc_add(&a[c], cf * d[c] * phi[s]);
                    }
        }
        for (long i = 0; i < nm; i++) {
            double th = 2.0 * M_PI * (m[3 * i] * x[3 * t] + m[3 * i + 1] * x[3 * t + 1] + m[3 * i + 2] * x[3 * t + 2]) / L;
            double v = -wk[i] * (re[i] * sin(th) + im[i] * cos(th));
            for (int c = 0; c < 3; c++) acc_add(&a[c], v * 2.0 * M_PI * m[3 * i + c]);
        }
        for (int c = 0; c < 3; c++) g[3 * t + c] = acc_get(&a[c]) / (L * L);
    }
    free(m); free(re); free(im); free(wk);
}

void orc_laplace_dp_grad(long S, const double *y, const double *phi, long T, const double *x,
                         double L, double xi, double rc, double kc, double H, double *g) {
    int mm[3] = {(int)ceil(kc / (2.0 * M_PI)), (int)ceil(kc / (2.0 * M_PI)), (int)ceil(kc * H / (2.0 * M_PI))};
    double P[3] = {1.0, 1.0, H};
    long cap = (long)(2 * mm[0] + 1) * (2 * mm[1] + 1) * (mm[2] + 1), nm = 0;
    int *m = (int *)malloc(sizeof(int) * 3 * cap);
    for (int mz = 0; mz <= mm[2]; mz++)
        for (int my = -mm[1]; my <= mm[1]; my++)
            for (int mx = -mm[0]; mx <= mm[0]; mx++) {
                if (mx == 0 && my == 0) continue;
                if (mz == 0 && (my < 0 || (my == 0 && mx <= 0))) continue;
                double kx = 2.0 * M_PI * mx, ky = 2.0 * M_PI * my, kz = 2.0 * M_PI * mz / H;
                if (kx * kx + ky * ky + kz * kz >= kc * kc) continue;
                m[3 * nm] = mx; m[3 * nm + 1] = my; m[3 * nm + 2] = mz; nm++;
            }
    double *re = (double *)malloc(sizeof(double) * (nm ? nm : 1));
    double *im = (double *)malloc(sizeof(double) * (nm ? nm : 1));
    structure_factors_box(S, y, phi, 1, L, mm, P, nm, m, re, im);
    int nr = rc > 0.5 ? (int)ceil(rc - 0.5) : 0;
    double rc2 = rc * rc, g0 = 2.0 * xi / sqrt(M_PI);
#pragma omp parallel for schedule(dynamic, 4)
    for (long t = 0; t < T; t++) {
        acc_t a[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (long s = 0; s < S; s++) {
            double r[3];
            for (int c = 0; c < 3; c++) r[c] = (x[3 * t + c] - y[3 * s + c]) / L;
            for (int c = 0; c < 2; c++) r[c] -= floor(r[c] + 0.5);
            for (int n0 = -nr; n0 <= nr; n0++)
                for (int n1 = -nr; n1 <= nr; n1++) {
                    double d[3] = {r[0] + n0, r[1] + n1, r[2]};
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 == 0.0 || r2 >= rc2) continue;
                    double rr = sqrt(r2);
                    double cf = -(erfc(xi * rr) + g0 * rr * exp(-xi * xi * r2)) / (r2 * rr);
                    for (int c = 0; c < 3; c++) acc_add(&a[c], cf * d[c] * phi[s]);
                }
            acc_add(&a[2], -2.0 * M_PI * erf(xi * r[2]) * phi[s]); /* k_par = 0 term */
        }
        for (long i = 0; i < nm; i++) {
            double k[3] = {2.0 * M_PI * m[3 * i], 2.0 * M_PI * m[3 * i + 1], 2.0 * M_PI * m[3 * i + 2] / H};
            double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
            double th = (k[0] * x[3 * t] + k[1] * x[3 * t + 1] + k[2] * x[3 * t + 2]) / L;
            double wk = 2.0 * 4.0 * M_PI / H * exp(-k2 / (4.0 * xi * xi)) / k2;
            double v = -wk * (re[i] * sin(th) + im[i] * cos(th));
            for (int c = 0; c < 3; c++) acc_add(&a[c], v * k[c]);
        }
        for (int c = 0; c < 3; c++) g[3 * t + c] = acc_get(&a[c]) / (L * L);
    }
    free(m); free(re); free(im);
}

/* gradient of the regularised 1D image sum of one pair (see sp_pair):
 * out[0] = d/da, out[1 + c] = d/d rho_c for the perpendicular offsets */
static void sp_pair_grad(double a, const double rho[2], long M, double out[3]) {
    acc_t s[3] = {{0, 0}, {0, 0}, {0, 0}};
    double rho2 = rho[0] * rho[0] + rho[1] * rho[1];
    for (long n = -M; n <= M; n++) {
        double z = a + (double)n, r2 = z * z + rho2;
        if (r2 == 0.0) continue;
        double ir3 = 1.0 / (r2 * sqrt(r2));
        acc_add(&s[0], -z * ir3);
        acc_add(&s[1], -rho[0] * ir3);
        acc_add(&s[2], -rho[1] * ir3);
    }
    double n0 = (double)(M + 1);
    double zp = n0 + a, zm = n0 - a;
    double Rp = sqrt(zp * zp + rho2), Rm = sqrt(zm * zm + rho2);
    double Rp3 = Rp * Rp * Rp, Rm3 = Rm * Rm * Rm, Rp5 = Rp3 * Rp * Rp, Rm5 = Rm3 * Rm * Rm;
    /* integral I = -ln((zp+Rp)/2n0) - ln((zm+Rm)/2n0) */
    double dI_a = -1.0 / Rp + 1.0 / Rm;
    double bI = 1.0 / (Rp * (zp + Rp)) + 1.0 / (Rm * (zm + Rm));
    /* g = 1/Rp + 1/Rm - 2/n0 */
    double dg_a = -zp / Rp3 + zm / Rm3;
    double bg = 1.0 / Rp3 + 1.0 / Rm3;
    /* g' = -zp/Rp^3 - zm/Rm^3 + 2/n0^2 */
    double dgp_a = -1.0 / Rp3 + 3.0 * zp * zp / Rp5 + 1.0 / Rm3 - 3.0 * zm * zm / Rm5;
    double bgp = 3.0 * zp / Rp5 + 3.0 * zm / Rm5;
    acc_add(&s[0], dI_a + 0.5 * dg_a - dgp_a / 12.0);
    for (int c = 0; c < 2; c++) acc_add(&s[1 + c], rho[c] * (-bI - 0.5 * bg - bgp / 12.0));
    for (int c = 0; c < 3; c++) out[c] = acc_get(&s[c]);
}

void orc_laplace_sp_grad(long S, const double *y, const double *phi, long T, const double *x,
                         int axis, double L, long M, double *g) {
    int p0 = axis == 0 ? 1 : 0, p1 = axis == 2 ? 1 : 2;
#pragma omp parallel for schedule(dynamic, 4)
    for (long t = 0; t < T; t++) {
        acc_t a[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (long s = 0; s < S; s++) {
            double r[3];
            for (int c = 0; c < 3; c++) r[c] = (x[3 * t + c] - y[3 * s + c]) / L;
            double ax = r[axis] - floor(r[axis] + 0.5), rho[2] = {r[p0], r[p1]}, d[3];
            sp_pair_grad(ax, rho, M, d);
            acc_add(&a[axis], phi[s] * d[0]);
            acc_add(&a[p0], phi[s] * d[1]);
            acc_add(&a[p1], phi[s] * d[2]);
        }
        for (int c = 0; c < 3; c++) g[3 * t + c] = acc_get(&a[c]) / (L * L);
    }
}
