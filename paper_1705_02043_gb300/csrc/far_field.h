// Free-space kernel blocks and the far-field periodic kernels K^{P,F}_ell
// (Algorithm 2, Stage 1; Sec. 2.3, 3.2-3.4), written once for the host
// precompute (g++) and the device precompute (nvcc): every function is
// __host__ __device__ under nvcc and plain C++ otherwise.
//
// * Triply periodic (Sec. 3.4): Ewald sums, Laplace with k = 0 removed and the
//   background term, Stokes with the Hasimoto split; the near images
//   |n|_inf <= ell enter as minus their smooth parts (their real-space terms
//   minus K), far real-space images are below rounding for xi = 7.5.
// * Doubly periodic in x and y (Sec. 3.3): 2D Ewald split; per in-plane mode
//   the k_z transform of the smooth part is taken in closed form, the k = 0
//   mode is the sheet term with its z-independent constant dropped.
// * Singly periodic (Sec. 3.2, Eq. (KPFdirect)): direct neutral image sums up
//   to n = 512 with an Euler-Maclaurin tail from the closed-form integral.
// Each returns the k x k block (row-major) for a unit cell and a difference
// vector r with |r_a| <= ~1.1.
#pragma once
#include <cmath>

#ifdef __CUDACC__
#define PK_HD __host__ __device__
#else
#define PK_HD
#endif

namespace pk {
namespace ff {

constexpr double kPiF = 3.14159265358979323846;

struct Neumaier {
    double s = 0, c = 0;
    PK_HD void add(double v) {
        double t = s + v;
        if (::fabs(s) >= ::fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    PK_HD double get() const { return s + c; }
};

// k x k block of the free-space kernel: Laplace 1/r, Stokes
// (I/r + r r^T/r^3)/8pi; zero at r = 0 (coincident points are excluded).
PK_HD inline void kernel_block(int kernel, const double *x, const double *y, double *out) {
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (kernel == 0) {
        out[0] = r2 > 0 ? 1.0 / ::sqrt(r2) : 0.0;
        return;
    }
    if (r2 == 0) {
        for (int i = 0; i < 9; i++) out[i] = 0.0;
        return;
    }
    double ir = 1.0 / ::sqrt(r2), ir3 = ir * ir * ir, c = 1.0 / (8.0 * kPiF);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) out[3 * a + b] = c * ((a == b ? ir : 0.0) + d[a] * d[b] * ir3);
}

// minus the smooth (erf) part of one real-space image d, added to acc
PK_HD inline void add_minus_smooth(int kernel, const double d[3], double xi, double g0, Neumaier *acc) {
    double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double dd = ::sqrt(d2);
    if (kernel == 0) {
        acc[0].add(d2 > 0 ? -::erf(xi * dd) / dd : -g0);
        return;
    }
    // Hasimoto smooth part S_F (times 1/8pi)
    double cI, cR;
    if (d2 > 0) {
        double e = g0 * ::exp(-xi * xi * d2), f = ::erf(xi * dd) / dd;
        cI = e + f;
        cR = -(e - f) / d2;
    } else {
        cI = 2.0 * g0;
        cR = 0.0;
    }
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) acc[3 * a + b].add(-((a == b ? cI : 0.0) + cR * d[a] * d[b]) / (8.0 * kPiF));
}

// Triply periodic, unit cell: K^{P,F}_ell(r) = K^P(r) - sum_{|n|_inf<=ell} K(r+n).
PK_HD inline void far_tp(int kernel, int ell, const double *r, double *out) {
    const double xi = 7.5, kc = 2.0 * 6.6 * xi;
    const int mmax = (int)::ceil(kc / (2 * kPiF));
    const double g0 = 2.0 * xi / ::sqrt(kPiF);
    const int k = kernel == 0 ? 1 : 3;
    Neumaier acc[9];
    for (int n0 = -ell; n0 <= ell; n0++)
        for (int n1 = -ell; n1 <= ell; n1++)
            for (int n2 = -ell; n2 <= ell; n2++) {
                double d[3] = {r[0] + n0, r[1] + n1, r[2] + n2};
                add_minus_smooth(kernel, d, xi, g0, acc);
            }
    // Fourier part, half space of modes, k = 0 removed
    for (int mz = 0; mz <= mmax; mz++)
        for (int my = -mmax; my <= mmax; my++)
            for (int mx = -mmax; mx <= mmax; mx++) {
                if (mz == 0 && (my < 0 || (my == 0 && mx <= 0))) continue;
                double kv[3] = {2 * kPiF * mx, 2 * kPiF * my, 2 * kPiF * mz};
                double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
                if (k2 >= kc * kc) continue;
                double cs = ::cos(kv[0] * r[0] + kv[1] * r[1] + kv[2] * r[2]);
                double a = k2 / (4 * xi * xi);
                if (kernel == 0) {
                    acc[0].add(2.0 * 4.0 * kPiF * ::exp(-a) / k2 * cs);
                } else {
                    double w = 2.0 * (1.0 + a) * ::exp(-a) / k2 * cs;
                    for (int i = 0; i < 3; i++)
                        for (int j = 0; j < 3; j++) acc[3 * i + j].add(w * ((i == j ? 1.0 : 0.0) - kv[i] * kv[j] / k2));
                }
            }
    if (kernel == 0) acc[0].add(-kPiF / (xi * xi));  // zero-mean K^P
    for (int i = 0; i < k * k; i++) out[i] = acc[i].get();
}

// Singly periodic Laplace along `axis`, unit period:
// sum_{n > ell} [1/|r + n e| + 1/|r - n e| - 2/n] - sum_{2<=n<=ell} 2/n  (the constant
// cancels for neutral densities), n <= M explicitly, Euler-Maclaurin beyond.
PK_HD inline void far_sp_laplace(int axis, int ell, const double *r, double *out) {
    const long M = 512;
    double x = r[axis], rho2 = 0;
    for (int a = 0; a < 3; a++)
        if (a != axis) rho2 += r[a] * r[a];
    Neumaier s;
    // the regularising constant -2/n is subtracted for every n >= 2 so that
    // the operator does not depend on ell (layers 2..ell are added back as
    // free-space images by the caller)
    for (long n = ell; n >= 2; n--) s.add(-2.0 / n);
    for (long n = M; n > ell; n--) {
        double zp = x + n, zm = x - n;
        s.add(1.0 / ::sqrt(zp * zp + rho2) + 1.0 / ::sqrt(zm * zm + rho2) - 2.0 / n);
    }
    double n0 = M + 1.0, zp = n0 + x, zm = n0 - x;
    double Rp = ::sqrt(zp * zp + rho2), Rm = ::sqrt(zm * zm + rho2);
    // integral_{n0}^{inf} of the summand, written with log1p to avoid cancellation
    double up = (x + (2 * n0 * x + x * x + rho2) / (Rp + n0)) / (2 * n0);
    double um = (-x + (-2 * n0 * x + x * x + rho2) / (Rm + n0)) / (2 * n0);
    s.add(-::log1p(up) - ::log1p(um));
    s.add(0.5 * (1.0 / Rp + 1.0 / Rm - 2.0 / n0));
    s.add(-(-zp / (Rp * Rp * Rp) - zm / (Rm * Rm * Rm) + 2.0 / (n0 * n0)) / 12.0);
    out[0] = s.get();
}

// Doubly periodic (x, y periodic, z free), unit cell, 2D Ewald split with
// the Hasimoto smooth part K_F (Laplace: erf(xi r)/r).  Per in-plane Fourier
// mode k = (k_x, k_y) != 0 the z transform of K_F^ is taken in closed form:
//   J(z) = int dk_z/2pi e^{-K^2/4xi^2}/K^2 e^{i k_z z}
//        = [e^{kz} erfc(k/2xi + xi z) + e^{-kz} erfc(k/2xi - xi z)] / 4k,
//   H(z) = int dk_z/2pi (1 + K^2/4xi^2) e^{-K^2/4xi^2}/K^4 e^{i k_z z}
//        = -dJ/d(k^2),   H'(z) = -z P / 8k,
// with K^2 = k^2 + k_z^2, P the bracket of J and D the same with a minus sign.
// The Stokes block is (K^2 I - kk^T) H with k_z -> -i d/dz:
//   in-plane (J + E/(4 xi sqrt(pi))) delta_ij - k_i k_j H,  (i,z): i k_i H',
//   (z,z) k^2 H,  E = e^{-k^2/4xi^2 - xi^2 z^2}.
// The k = 0 mode is the sheet field with z-independent constants dropped
// (they cancel for neutral densities):
//   Laplace 4 pi [-(z/2) erf(xi z) - e^{-xi^2 z^2}/(2 xi sqrt(pi))],
//   Stokes  (I - e_z e_z) [-(z/2) erf(xi z) - e^{-xi^2 z^2}/(4 xi sqrt(pi))].
// Near images |n|_inf <= ell (in-plane) contribute K_R - K = -K_F; farther
// real-space images are negligible for |r_a| <= 1.1 and xi = 7.5.
PK_HD inline void far_dp(int kernel, int ell, const double *r, double *out) {
    const double xi = 7.5, kc = 2.0 * 6.6 * xi, sqpi = ::sqrt(kPiF);
    const int mmax = (int)::ceil(kc / (2 * kPiF));
    const double g0 = 2.0 * xi / sqpi;
    const int k = kernel == 0 ? 1 : 3;
    Neumaier acc[9];
    for (int n0 = -ell; n0 <= ell; n0++)
        for (int n1 = -ell; n1 <= ell; n1++) {
            double d[3] = {r[0] + n0, r[1] + n1, r[2]};
            add_minus_smooth(kernel, d, xi, g0, acc);
        }
    const double z = r[2];
    for (int my = 0; my <= mmax; my++)
        for (int mx = -mmax; mx <= mmax; mx++) {
            if (my == 0 && mx <= 0) continue;  // half plane of in-plane modes, k = 0 below
            double kx = 2 * kPiF * mx, ky = 2 * kPiF * my, kk = ::sqrt(kx * kx + ky * ky);
            if (kk >= kc) continue;
            double th = kx * r[0] + ky * r[1], cs = ::cos(th), sn = ::sin(th);
            double ap = kk / (2 * xi) + xi * z, am = kk / (2 * xi) - xi * z;
            double tp = ::exp(kk * z) * ::erfc(ap), tm = ::exp(-kk * z) * ::erfc(am);
            double P = tp + tm, D = tp - tm;
            double E = ::exp(-kk * kk / (4 * xi * xi) - xi * xi * z * z);
            double J = P / (4 * kk);
            if (kernel == 0) {
                acc[0].add(2.0 * 4.0 * kPiF * J * cs);
                continue;
            }
            double H = P / (8 * kk * kk * kk) - z * D / (8 * kk * kk) + E / (4 * kk * kk * xi * sqpi);
            double Hp = -z * P / (8 * kk);
            double kv[2] = {kx, ky};
            for (int i = 0; i < 2; i++)
                for (int j = 0; j < 2; j++)
                    acc[3 * i + j].add(2.0 * cs * ((i == j ? J + E / (4 * xi * sqpi) : 0.0) - kv[i] * kv[j] * H));
            for (int i = 0; i < 2; i++) {
                double v = -2.0 * kv[i] * Hp * sn;  // (k, -k) pair of i k_i H' e^{i k.r}
                acc[3 * i + 2].add(v);
                acc[3 * 2 + i].add(v);
            }
            acc[8].add(2.0 * cs * kk * kk * H);
        }
    double lin = -0.5 * z * ::erf(xi * z), ez = ::exp(-xi * xi * z * z);
    if (kernel == 0) {
        acc[0].add(4.0 * kPiF * (lin - ez / (2 * xi * sqpi)));
    } else {
        double g = lin - ez / (4 * xi * sqpi);
        acc[0].add(g);
        acc[4].add(g);
    }
    for (int i = 0; i < k * k; i++) out[i] = acc[i].get();
}

// Stokeslet block (I/|d| + d d^T/|d|^3)/8pi and its derivative along `axis`
PK_HD inline void stokeslet(const double d[3], double o[9]) {
    const double c8 = 1.0 / (8.0 * kPiF);
    double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], id = 1.0 / ::sqrt(d2), id3 = id * id * id;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) o[3 * i + j] = c8 * ((i == j ? id : 0.0) + d[i] * d[j] * id3);
}

PK_HD inline double stokeslet_d(const double d[3], int axis, int i, int j) {
    const double c8 = 1.0 / (8.0 * kPiF);
    double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], dd = ::sqrt(d2), i3 = 1.0 / (d2 * dd), i5 = i3 / d2;
    double v = -(i == j ? d[axis] * i3 : 0.0) + ((i == axis ? d[j] : 0.0) + (j == axis ? d[i] : 0.0)) * i3 -
               3.0 * d[i] * d[j] * d[axis] * i5;
    return c8 * v;
}

// Singly periodic Stokes along `axis`, unit period, zero net force:
// K^{P,F}_ell(r) = sum_{n > ell} [S(r + n e) + S(r - n e) - (2/n) C] - sum_{2<=n<=ell} (2/n) C,
// C = (I + e e^T)/8pi (the monopole far field of one image), which cancels
// for zero net force; n <= M explicitly, then Euler-Maclaurin from n0 = M+1
// with the closed-form integral of the summand.  In the frame (e, p, q):
// w1 = x + n0, w2 = n0 - x, R_i = |(w_i, rho)|, lg = -ln((w1+R1)/2n0) - ln((w2+R2)/2n0),
// beta = 1/(R1(R1+w1)) + 1/(R2(R2+w2)):
//   int (e,e) = (2 lg - rho^2 beta)/8pi,  int (e,p) = rho_p (1/R1 - 1/R2)/8pi,
//   int (p,q) = (lg delta_pq + rho_p rho_q beta)/8pi.
PK_HD inline void far_sp_stokes(int axis, int ell, const double *r, double *out) {
    const long M = 512;
    const double c8 = 1.0 / (8.0 * kPiF);
    double C[9];
    for (int i = 0; i < 9; i++) C[i] = 0.0;
    for (int i = 0; i < 3; i++) C[4 * i] = c8;
    C[4 * axis] += c8;
    Neumaier acc[9];
    for (long n = ell; n >= 2; n--)
        for (int i = 0; i < 9; i++) acc[i].add(-2.0 / n * C[i]);
    double sp[9], sm[9];
    for (long n = M; n > ell; n--) {
        double dp[3] = {r[0], r[1], r[2]}, dm[3] = {r[0], r[1], r[2]};
        dp[axis] += n;
        dm[axis] -= n;
        stokeslet(dp, sp);
        stokeslet(dm, sm);
        for (int i = 0; i < 9; i++) acc[i].add(sp[i] + sm[i] - 2.0 / n * C[i]);
    }
    const double n0 = M + 1.0, x = r[axis];
    double rho[3] = {r[0], r[1], r[2]};
    rho[axis] = 0.0;
    const double rho2 = rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2];
    const double w1 = x + n0, w2 = n0 - x, R1 = ::sqrt(w1 * w1 + rho2), R2 = ::sqrt(w2 * w2 + rho2);
    const double u1 = (x + (2 * n0 * x + x * x + rho2) / (R1 + n0)) / (2 * n0);
    const double u2 = (-x + (-2 * n0 * x + x * x + rho2) / (R2 + n0)) / (2 * n0);
    const double lg = -::log1p(u1) - ::log1p(u2);
    const double beta = 1.0 / (R1 * (R1 + w1)) + 1.0 / (R2 * (R2 + w2));
    // g(n0) and its derivative in n: d/dn S(r +- n e) = +-(e.grad) S
    double dp[3] = {r[0], r[1], r[2]}, dm[3] = {r[0], r[1], r[2]};
    dp[axis] += n0;
    dm[axis] -= n0;
    stokeslet(dp, sp);
    stokeslet(dm, sm);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double in;
            if (i == axis && j == axis) in = 2 * lg - rho2 * beta;
            else if (i == axis) in = rho[j] * (1.0 / R1 - 1.0 / R2);
            else if (j == axis) in = rho[i] * (1.0 / R1 - 1.0 / R2);
            else in = (i == j ? lg : 0.0) + rho[i] * rho[j] * beta;
            const int q = 3 * i + j;
            double g = sp[q] + sm[q] - 2.0 / n0 * C[q];
            double dg = stokeslet_d(dp, axis, i, j) - stokeslet_d(dm, axis, i, j) + 2.0 / (n0 * n0) * C[q];
            acc[q].add(c8 * in);
            acc[q].add(0.5 * g);
            acc[q].add(-dg / 12.0);
        }
    for (int i = 0; i < 9; i++) out[i] = acc[i].get();
}

// K^{P,F}_ell block for the periodicity mask; false for masks not built
// (0, the doubly periodic pairs other than x-y).
PK_HD inline bool far_kernel_block(int kernel, unsigned periodic, int ell, const double *r, double *out) {
    if (periodic == 7) {
        far_tp(kernel, ell, r, out);
    } else if (periodic == 3) {
        far_dp(kernel, ell, r, out);
    } else if (periodic == 1 || periodic == 2 || periodic == 4) {
        const int axis = periodic == 1 ? 0 : periodic == 2 ? 1 : 2;
        if (kernel == 0) far_sp_laplace(axis, ell, r, out);
        else far_sp_stokes(axis, ell, r, out);
    } else {
        return false;
    }
    return true;
}

// Entry t of the difference-lattice table of the root operator: K^{P,F}_ell
// plus the free-space images of layers 2..ell (those within the near field
// beyond the colleagues), at r = (di, dj, dk) * step, t = ((di + p - 1) w +
// dj + p - 1) w + dk + p - 1 with w = 2p - 1 and step = 2 * 0.525 / (p - 1).
PK_HD inline bool root_table_entry(int kernel, unsigned periodic, int ell, int p, double inner_half, int t,
                                   double *acc) {
    const int w = 2 * p - 1, k = kernel == 0 ? 1 : 3;
    const int di = t / (w * w) - (p - 1), dj = (t / w) % w - (p - 1), dk = t % w - (p - 1);
    const double step = 2.0 * inner_half / (p - 1);
    double r[3] = {di * step, dj * step, dk * step};
    if (!far_kernel_block(kernel, periodic, ell, r, acc)) return false;
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        bool per = periodic >> a & 1;
        lo[a] = per ? -ell : 0;
        hi[a] = per ? ell : 0;
    }
    double blk[9];
    for (int n0 = lo[0]; n0 <= hi[0]; n0++)
        for (int n1 = lo[1]; n1 <= hi[1]; n1++)
            for (int n2 = lo[2]; n2 <= hi[2]; n2++) {
                int a0 = n0 < 0 ? -n0 : n0, a1 = n1 < 0 ? -n1 : n1, a2 = n2 < 0 ? -n2 : n2;
                int m = a0 > a1 ? a0 : a1;
                m = m > a2 ? m : a2;
                if (m <= 1) continue;
                double zero[3] = {0, 0, 0}, d[3] = {r[0] + n0, r[1] + n1, r[2] + n2};
                kernel_block(kernel, d, zero, blk);
                for (int i = 0; i < k * k; i++) acc[i] += blk[i];
            }
    return true;
}

// Entry t of the root operator's table for a finite array of cells along
// `axis` (the cell and its copies shifted by n e, |n| <= nimg; the
// finite-length channel of Sec. 4): the plain free-space sum over the copies
// that are not the root's colleagues, 2 <= |n| <= nimg.  Same lattice as above.
PK_HD inline void finite_table_entry(int kernel, int axis, int nimg, int p, double inner_half, int t, double *acc) {
    const int w = 2 * p - 1, k = kernel == 0 ? 1 : 3;
    const int di = t / (w * w) - (p - 1), dj = (t / w) % w - (p - 1), dk = t % w - (p - 1);
    const double step = 2.0 * inner_half / (p - 1);
    const double r[3] = {di * step, dj * step, dk * step};
    Neumaier s[9];
    double blk[9], zero[3] = {0, 0, 0};
    for (int n = nimg; n >= 2; n--)
        for (int sg = -1; sg <= 1; sg += 2) {
            double d[3] = {r[0], r[1], r[2]};
            d[axis] += sg * n;
            kernel_block(kernel, d, zero, blk);
            for (int i = 0; i < k * k; i++) s[i].add(blk[i]);
        }
    for (int i = 0; i < k * k; i++) acc[i] = s[i].get();
}

}  // namespace ff
}  // namespace pk
