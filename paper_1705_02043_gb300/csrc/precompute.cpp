// Host-side operator precompute (Algorithm 2, Stage 1).
//
// * Surfaces (Sec. 2.2): a regular grid with p points per edge (vertices
//   included) on the cube [-1,1]^3, n = 6(p-1)^2 + 2 points, listed in
//   lexicographic (i, j, k) order with k fastest; scaled by the half-width of
//   each surface (edge 1.05 -> 0.525, edge 2.95 -> 1.475, times the box edge).
// * Check-to-equivalent solves (Sec. 3.1): SVD A = U S V^T by one-sided
//   Jacobi, singular values <= eps * s_max dropped, applied as two products
//   (V S+) (U^T q), never as an explicit pseudo-inverse.
// * Translation operators are scale invariant because both kernels are
//   homogeneous of degree -1; they are computed once on a unit child box.
//   With q~ = h q (check potential times box edge) every operator is level
//   independent.
// * Root operator (Eq. (M2Lsolve), Sec. 2.3): the far-field periodic kernel
//   K^{P,F} on the downward check and upward equivalent surfaces of B0.
//   Triply periodic K^P is an Ewald sum (Hasimoto for Stokes, Sec. 3.4); the
//   near images are removed analytically (their real-space terms become the
//   smooth erf parts), so far real-space images are below rounding for the
//   splitting used.  Singly periodic Laplace uses the direct neutral image
//   sum of Eq. (KPFdirect) with an Euler-Maclaurin tail instead of a finite
//   n (Sec. 3.2).  Values depend only on r = x - y, so they are tabulated on
//   the difference lattice of the surface grid.
#include "precompute.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <filesystem>
#include <fstream>
#include <numeric>
#include <stdexcept>
#include <unistd.h>

namespace pk {

static const double kPi = 3.14159265358979323846;

int surface_count(int p) { return 6 * (p - 1) * (p - 1) + 2; }

std::vector<double> surface_grid(int p) {
    std::vector<double> g;
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++)
            for (int k = 0; k < p; k++) {
                if (i != 0 && i != p - 1 && j != 0 && j != p - 1 && k != 0 && k != p - 1) continue;
                g.push_back(-1.0 + 2.0 * i / (p - 1));
                g.push_back(-1.0 + 2.0 * j / (p - 1));
                g.push_back(-1.0 + 2.0 * k / (p - 1));
            }
    return g;
}

void kernel_block(int kernel, const double *x, const double *y, double *out) {
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (kernel == 0) {
        out[0] = r2 > 0 ? 1.0 / std::sqrt(r2) : 0.0;
        return;
    }
    if (r2 == 0) {
        std::fill(out, out + 9, 0.0);
        return;
    }
    double ir = 1.0 / std::sqrt(r2), ir3 = ir * ir * ir, c = 1.0 / (8.0 * kPi);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) out[3 * a + b] = c * ((a == b ? ir : 0.0) + d[a] * d[b] * ir3);
}

std::vector<double> kernel_matrix(int kernel, const std::vector<double> &x, const std::vector<double> &y) {
    int k = kernel == 0 ? 1 : 3;
    size_t nx = x.size() / 3, ny = y.size() / 3, cols = ny * k;
    std::vector<double> M(nx * k * cols);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)nx; i++) {
        double blk[9];
        for (size_t j = 0; j < ny; j++) {
            kernel_block(kernel, &x[3 * i], &y[3 * j], blk);
            for (int a = 0; a < k; a++)
                for (int b = 0; b < k; b++) M[(i * k + a) * cols + j * k + b] = blk[a * k + b];
        }
    }
    return M;
}

void matmul(int m, int n, int kk, const double *A, const double *B, double *C) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; i++) {
        double *c = C + (size_t)i * n;
        std::fill(c, c + n, 0.0);
        for (int l = 0; l < kk; l++) {
            double a = A[(size_t)i * kk + l];
            const double *b = B + (size_t)l * n;
            for (int j = 0; j < n; j++) c[j] += a * b[j];
        }
    }
}

// One-sided (Hestenes) Jacobi: orthogonalise the columns of A by plane
// rotations, accumulating them in V.  Pairs are scheduled round-robin so the
// m/2 rotations of one round are independent.  Columns are stored as rows
// (At = A^T) for contiguous access.
void jacobi_svd(int m, const std::vector<double> &A, std::vector<double> &U,
                std::vector<double> &S, std::vector<double> &V) {
    int mm = m + (m & 1);  // even player count; index m (if odd) is a bye
    std::vector<double> At((size_t)m * m), Vt((size_t)m * m, 0.0);
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) At[(size_t)j * m + i] = A[(size_t)i * m + j];
    for (int i = 0; i < m; i++) Vt[(size_t)i * m + i] = 1.0;
    std::vector<int> ring(mm);
    std::iota(ring.begin(), ring.end(), 0);
    const double tol = 1e-15;
    for (int sweep = 0; sweep < 80; sweep++) {
        long rotations = 0;
        for (int round = 0; round < mm - 1; round++) {
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : rotations)
            for (int t = 0; t < mm / 2; t++) {
                int p = ring[t], q = ring[mm - 1 - t];
                if (p >= m || q >= m) continue;
                if (p > q) std::swap(p, q);
                double *ap = &At[(size_t)p * m], *aq = &At[(size_t)q * m];
                double alpha = 0, beta = 0, gamma = 0;
                for (int i = 0; i < m; i++) {
                    alpha += ap[i] * ap[i];
                    beta += aq[i] * aq[i];
                    gamma += ap[i] * aq[i];
                }
                if (gamma == 0.0 || std::fabs(gamma) <= tol * std::sqrt(alpha * beta)) continue;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double tt = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + tt * tt), s = c * tt;
                for (int i = 0; i < m; i++) {
                    double x = ap[i], y = aq[i];
                    ap[i] = c * x - s * y;
                    aq[i] = s * x + c * y;
                }
                double *vp = &Vt[(size_t)p * m], *vq = &Vt[(size_t)q * m];
                for (int i = 0; i < m; i++) {
                    double x = vp[i], y = vq[i];
                    vp[i] = c * x - s * y;
                    vq[i] = s * x + c * y;
                }
                rotations++;
            }
            // rotate the ring, keeping position 0 fixed (circle method)
            int last = ring[mm - 1];
            for (int i = mm - 1; i > 1; i--) ring[i] = ring[i - 1];
            ring[1] = last;
        }
        if (rotations == 0) break;
    }
    std::vector<double> sig(m);
    for (int j = 0; j < m; j++) {
        double s = 0;
        for (int i = 0; i < m; i++) s += At[(size_t)j * m + i] * At[(size_t)j * m + i];
        sig[j] = std::sqrt(s);
    }
    std::vector<int> order(m);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sig[a] > sig[b]; });
    U.assign((size_t)m * m, 0.0);
    V.assign((size_t)m * m, 0.0);
    S.assign(m, 0.0);
    for (int jj = 0; jj < m; jj++) {
        int j = order[jj];
        S[jj] = sig[j];
        double inv = sig[j] > 0 ? 1.0 / sig[j] : 0.0;
        for (int i = 0; i < m; i++) {
            U[(size_t)i * m + jj] = At[(size_t)j * m + i] * inv;
            V[(size_t)i * m + jj] = Vt[(size_t)j * m + i];
        }
    }
}

// ---------------- far-field periodic kernel K^{P,F} ----------------

namespace {

struct Neumaier {
    double s = 0, c = 0;
    void add(double v) {
        double t = s + v;
        if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    double get() const { return s + c; }
};

// Triply periodic, unit cell.  K^{P,F}_ell(r) = K^P(r) - sum_{|n|_inf<=ell} K(r+n).
// Real-space Ewald terms of the near images combine with -K into minus the
// smooth part; far images are negligible for |r_a| <= 1.1 and xi = 7.5.
void far_tp(int kernel, int ell, const double *r, double *out) {
    const double xi = 7.5, kc = 2.0 * 6.6 * xi;
    const int mmax = (int)std::ceil(kc / (2 * kPi));
    const double g0 = 2.0 * xi / std::sqrt(kPi);
    int k = kernel == 0 ? 1 : 3;
    Neumaier acc[9];
    for (int n0 = -ell; n0 <= ell; n0++)
        for (int n1 = -ell; n1 <= ell; n1++)
            for (int n2 = -ell; n2 <= ell; n2++) {
                double d[3] = {r[0] + n0, r[1] + n1, r[2] + n2};
                double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double dd = std::sqrt(d2);
                if (kernel == 0) {
                    acc[0].add(d2 > 0 ? -std::erf(xi * dd) / dd : -g0);
                } else {
                    // smooth part S_F of the Hasimoto split (times 1/8pi)
                    double cI, cR;
                    if (d2 > 0) {
                        double e = g0 * std::exp(-xi * xi * d2), f = std::erf(xi * dd) / dd;
                        cI = e + f;
                        cR = -(e - f) / d2;
                    } else {
                        cI = 2.0 * g0;
                        cR = 0.0;
                    }
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            acc[3 * a + b].add(-((a == b ? cI : 0.0) + cR * d[a] * d[b]) / (8.0 * kPi));
                }
            }
    // Fourier part, half space of modes, k = 0 removed
    for (int mz = 0; mz <= mmax; mz++)
        for (int my = -mmax; my <= mmax; my++)
            for (int mx = -mmax; mx <= mmax; mx++) {
                if (mz == 0 && (my < 0 || (my == 0 && mx <= 0))) continue;
                double kv[3] = {2 * kPi * mx, 2 * kPi * my, 2 * kPi * mz};
                double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
                if (k2 >= kc * kc) continue;
                double cs = std::cos(kv[0] * r[0] + kv[1] * r[1] + kv[2] * r[2]);
                double a = k2 / (4 * xi * xi);
                if (kernel == 0) {
                    acc[0].add(2.0 * 4.0 * kPi * std::exp(-a) / k2 * cs);
                } else {
                    double w = 2.0 * (1.0 + a) * std::exp(-a) / k2 * cs;
                    for (int i = 0; i < 3; i++)
                        for (int j = 0; j < 3; j++) acc[3 * i + j].add(w * ((i == j ? 1.0 : 0.0) - kv[i] * kv[j] / k2));
                }
            }
    if (kernel == 0) acc[0].add(-kPi / (xi * xi));  // zero-mean K^P
    for (int i = 0; i < k * k; i++) out[i] = acc[i].get();
}

// Singly periodic Laplace along `axis`, unit period:
// sum_{n > ell} [1/|r + n e| + 1/|r - n e| - 2/n] - sum_{2<=n<=ell} 2/n  (the constant
// cancels for neutral densities), n <= M explicitly, Euler-Maclaurin beyond.
void far_sp_laplace(int axis, int ell, const double *r, double *out) {
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
        s.add(1.0 / std::sqrt(zp * zp + rho2) + 1.0 / std::sqrt(zm * zm + rho2) - 2.0 / n);
    }
    double n0 = M + 1.0, zp = n0 + x, zm = n0 - x;
    double Rp = std::sqrt(zp * zp + rho2), Rm = std::sqrt(zm * zm + rho2);
    // integral_{n0}^{inf} of the summand, written with log1p to avoid cancellation
    double up = (x + (2 * n0 * x + x * x + rho2) / (Rp + n0)) / (2 * n0);
    double um = (-x + (-2 * n0 * x + x * x + rho2) / (Rm + n0)) / (2 * n0);
    s.add(-std::log1p(up) - std::log1p(um));
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
void far_dp(int kernel, int ell, const double *r, double *out) {
    const double xi = 7.5, kc = 2.0 * 6.6 * xi, sqpi = std::sqrt(kPi);
    const int mmax = (int)std::ceil(kc / (2 * kPi));
    const double g0 = 2.0 * xi / sqpi;
    int k = kernel == 0 ? 1 : 3;
    Neumaier acc[9];
    for (int n0 = -ell; n0 <= ell; n0++)
        for (int n1 = -ell; n1 <= ell; n1++) {
            double d[3] = {r[0] + n0, r[1] + n1, r[2]};
            double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double dd = std::sqrt(d2);
            if (kernel == 0) {
                acc[0].add(d2 > 0 ? -std::erf(xi * dd) / dd : -g0);
            } else {
                double cI, cR;
                if (d2 > 0) {
                    double e = g0 * std::exp(-xi * xi * d2), f = std::erf(xi * dd) / dd;
                    cI = e + f;
                    cR = -(e - f) / d2;
                } else {
                    cI = 2.0 * g0;
                    cR = 0.0;
                }
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++)
                        acc[3 * a + b].add(-((a == b ? cI : 0.0) + cR * d[a] * d[b]) / (8.0 * kPi));
            }
        }
    const double z = r[2];
    for (int my = 0; my <= mmax; my++)
        for (int mx = -mmax; mx <= mmax; mx++) {
            if (my == 0 && mx <= 0) continue;  // half plane of in-plane modes, k = 0 below
            double kx = 2 * kPi * mx, ky = 2 * kPi * my, kk = std::sqrt(kx * kx + ky * ky);
            if (kk >= kc) continue;
            double th = kx * r[0] + ky * r[1], cs = std::cos(th), sn = std::sin(th);
            double ap = kk / (2 * xi) + xi * z, am = kk / (2 * xi) - xi * z;
            double tp = std::exp(kk * z) * std::erfc(ap), tm = std::exp(-kk * z) * std::erfc(am);
            double P = tp + tm, D = tp - tm;
            double E = std::exp(-kk * kk / (4 * xi * xi) - xi * xi * z * z);
            double J = P / (4 * kk);
            if (kernel == 0) {
                acc[0].add(2.0 * 4.0 * kPi * J * cs);
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
    double lin = -0.5 * z * std::erf(xi * z), ez = std::exp(-xi * xi * z * z);
    if (kernel == 0) {
        acc[0].add(4.0 * kPi * (lin - ez / (2 * xi * sqpi)));
    } else {
        double g = lin - ez / (4 * xi * sqpi);
        acc[0].add(g);
        acc[4].add(g);
    }
    for (int i = 0; i < k * k; i++) out[i] = acc[i].get();
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
void far_sp_stokes(int axis, int ell, const double *r, double *out) {
    const long M = 512;
    const double c8 = 1.0 / (8.0 * kPi);
    double C[9];
    for (int i = 0; i < 9; i++) C[i] = 0.0;
    for (int i = 0; i < 3; i++) C[4 * i] = c8;
    C[4 * axis] += c8;
    auto stokeslet = [&](const double d[3], double o[9]) {
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], id = 1.0 / std::sqrt(d2), id3 = id * id * id;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) o[3 * i + j] = c8 * ((i == j ? id : 0.0) + d[i] * d[j] * id3);
    };
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
    const double w1 = x + n0, w2 = n0 - x, R1 = std::sqrt(w1 * w1 + rho2), R2 = std::sqrt(w2 * w2 + rho2);
    const double u1 = (x + (2 * n0 * x + x * x + rho2) / (R1 + n0)) / (2 * n0);
    const double u2 = (-x + (-2 * n0 * x + x * x + rho2) / (R2 + n0)) / (2 * n0);
    const double lg = -std::log1p(u1) - std::log1p(u2);
    const double beta = 1.0 / (R1 * (R1 + w1)) + 1.0 / (R2 * (R2 + w2));
    // g(n0) and its derivative in n: d/dn S(r +- n e) = +-(e.grad) S
    double dp[3] = {r[0], r[1], r[2]}, dm[3] = {r[0], r[1], r[2]};
    dp[axis] += n0;
    dm[axis] -= n0;
    stokeslet(dp, sp);
    stokeslet(dm, sm);
    auto dS = [&](const double d[3], int i, int j) {  // d S_ij / d d_axis
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], dd = std::sqrt(d2), i3 = 1.0 / (d2 * dd), i5 = i3 / d2;
        double v = -(i == j ? d[axis] * i3 : 0.0) + ((i == axis ? d[j] : 0.0) + (j == axis ? d[i] : 0.0)) * i3 -
                   3.0 * d[i] * d[j] * d[axis] * i5;
        return c8 * v;
    };
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double in;
            if (i == axis && j == axis) in = 2 * lg - rho2 * beta;
            else if (i == axis) in = rho[j] * (1.0 / R1 - 1.0 / R2);
            else if (j == axis) in = rho[i] * (1.0 / R1 - 1.0 / R2);
            else in = (i == j ? lg : 0.0) + rho[i] * rho[j] * beta;
            const int q = 3 * i + j;
            double g = sp[q] + sm[q] - 2.0 / n0 * C[q];
            double dg = dS(dp, i, j) - dS(dm, i, j) + 2.0 / (n0 * n0) * C[q];
            acc[q].add(c8 * in);
            acc[q].add(0.5 * g);
            acc[q].add(-dg / 12.0);
        }
    for (int i = 0; i < 9; i++) out[i] = acc[i].get();
}

}  // namespace

void far_kernel_block(int kernel, unsigned periodic, int ell, const double *r, double *out) {
    if (periodic == 7) {
        far_tp(kernel, ell, r, out);
    } else if (periodic == 3) {
        far_dp(kernel, ell, r, out);
    } else if (periodic == 1 || periodic == 2 || periodic == 4) {
        const int axis = periodic == 1 ? 0 : periodic == 2 ? 1 : 2;
        if (kernel == 0) far_sp_laplace(axis, ell, r, out);
        else far_sp_stokes(axis, ell, r, out);
    } else {
        throw std::runtime_error("far kernel: periodicity not supported");
    }
}

std::vector<double> root_operator(int kernel, int p, unsigned periodic, int ell,
                                  const std::vector<double> &g) {
    int k = kernel == 0 ? 1 : 3, n = (int)g.size() / 3, kn = n * k, w = 2 * p - 1;
    // table of K^{P,F} + near-layer images 2..ell on the difference lattice
    std::vector<double> tab((size_t)w * w * w * k * k);
    double step = 2.0 * kInnerHalf / (p - 1);
#pragma omp parallel for schedule(dynamic, 8)
    for (int t = 0; t < w * w * w; t++) {
        int di = t / (w * w) - (p - 1), dj = (t / w) % w - (p - 1), dk = t % w - (p - 1);
        double r[3] = {di * step, dj * step, dk * step};
        double blk[9], acc[9];
        far_kernel_block(kernel, periodic, ell, r, acc);
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            bool per = periodic >> a & 1;
            lo[a] = per ? -ell : 0;
            hi[a] = per ? ell : 0;
        }
        for (int n0 = lo[0]; n0 <= hi[0]; n0++)
            for (int n1 = lo[1]; n1 <= hi[1]; n1++)
                for (int n2 = lo[2]; n2 <= hi[2]; n2++) {
                    int m = std::max(std::abs(n0), std::max(std::abs(n1), std::abs(n2)));
                    if (m <= 1) continue;
                    double zero[3] = {0, 0, 0}, d[3] = {r[0] + n0, r[1] + n1, r[2] + n2};
                    kernel_block(kernel, d, zero, blk);
                    for (int i = 0; i < k * k; i++) acc[i] += blk[i];
                }
        std::memcpy(&tab[(size_t)t * k * k], acc, sizeof(double) * k * k);
    }
    std::vector<double> Mr((size_t)kn * kn);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            int d[3];
            for (int a = 0; a < 3; a++) d[a] = (int)std::lround((g[3 * i + a] - g[3 * j + a]) * (p - 1) / 2.0) + (p - 1);
            const double *b = &tab[(size_t)((d[0] * w + d[1]) * w + d[2]) * k * k];
            for (int a = 0; a < k; a++)
                for (int c = 0; c < k; c++) Mr[(size_t)(i * k + a) * kn + j * k + c] = b[a * k + c];
        }
    return Mr;
}

// ---------------- cache ----------------

namespace {

const uint64_t kMagic = 0x504b49464d4d3031ULL;  // "PKIFMM01"
const int kVersion = 3;

uint64_t fnv(const void *data, size_t n, uint64_t h = 1469598103934665603ULL) {
    const unsigned char *c = (const unsigned char *)data;
    for (size_t i = 0; i < n; i++) h = (h ^ c[i]) * 1099511628211ULL;
    return h;
}

std::string cache_path(const std::string &dir, const HostOps &o) {
    char buf[256];
    std::snprintf(buf, sizeof buf, "/pkifmm_k%d_p%d_per%u_l%d_e%.3e_v%d.bin", o.kernel, o.p, o.periodic,
                  o.ell, o.eps_rel, kVersion);
    return dir + buf;
}

std::vector<std::vector<double> *> payload(HostOps &o) {
    return {&o.U, &o.S, &o.V, &o.m2m, &o.l2l, &o.root};
}

bool load_cache(const std::string &path, HostOps &o) {
    std::ifstream f(path, std::ios::binary);
    if (!f) return false;
    uint64_t magic = 0, sum = 0;
    int hdr[6];
    f.read((char *)&magic, 8);
    f.read((char *)hdr, sizeof hdr);
    if (!f || magic != kMagic || hdr[0] != kVersion || hdr[1] != o.kernel || hdr[2] != o.p ||
        hdr[3] != (int)o.periodic || hdr[4] != o.ell || hdr[5] != o.kn)
        throw std::runtime_error("cache: header mismatch in " + path);
    uint64_t h = 1469598103934665603ULL;
    for (auto *v : payload(o)) {
        uint64_t len = 0;
        f.read((char *)&len, 8);
        if (!f || len > (1ull << 32)) throw std::runtime_error("cache: truncated " + path);
        v->resize(len);
        f.read((char *)v->data(), len * 8);
        if (!f) throw std::runtime_error("cache: truncated " + path);
        h = fnv(v->data(), len * 8, h);
    }
    f.read((char *)&sum, 8);
    if (!f || sum != h) throw std::runtime_error("cache: checksum mismatch in " + path);
    return true;
}

void save_cache(const std::string &path, HostOps &o) {
    std::error_code ec;
    std::filesystem::create_directories(std::filesystem::path(path).parent_path(), ec);
    std::string tmp = path + ".tmp" + std::to_string((long long)std::hash<std::string>{}(path) ^ (long long)getpid());
    std::ofstream f(tmp, std::ios::binary);
    if (!f) throw std::runtime_error("cache: cannot write " + tmp);
    int hdr[6] = {kVersion, o.kernel, o.p, (int)o.periodic, o.ell, o.kn};
    f.write((const char *)&kMagic, 8);
    f.write((const char *)hdr, sizeof hdr);
    uint64_t h = 1469598103934665603ULL;
    for (auto *v : payload(o)) {
        uint64_t len = v->size();
        f.write((const char *)&len, 8);
        f.write((const char *)v->data(), len * 8);
        h = fnv(v->data(), len * 8, h);
    }
    f.write((const char *)&h, 8);
    f.close();
    if (!f || std::rename(tmp.c_str(), path.c_str()) != 0) throw std::runtime_error("cache: write failed " + path);
}

}  // namespace

void build_host_ops(HostOps &o, int kernel, int p, unsigned periodic, int ell, double eps_rel,
                    const std::string &cache_dir) {
    o.kernel = kernel;
    o.k = kernel == 0 ? 1 : 3;
    o.p = p;
    o.n = surface_count(p);
    o.kn = o.n * o.k;
    o.periodic = periodic;
    o.ell = ell;
    o.eps_rel = eps_rel;
    o.g = surface_grid(p);
    const int kn = o.kn, n = o.n;
    bool cached = false;
    if (!cache_dir.empty()) cached = load_cache(cache_path(cache_dir, o), o);
    if (!cached) {
        std::vector<double> xu(3 * n), yu(3 * n);
        for (int i = 0; i < 3 * n; i++) {
            xu[i] = kOuterHalf * o.g[i];
            yu[i] = kInnerHalf * o.g[i];
        }
        std::vector<double> A = kernel_matrix(kernel, xu, yu);  // A_up1
        jacobi_svd(kn, A, o.U, o.S, o.V);
    }
    double cut = eps_rel * o.S[0];
    std::vector<double> sinv(kn);
    for (int j = 0; j < kn; j++) sinv[j] = o.S[j] > cut ? 1.0 / o.S[j] : 0.0;
    o.uc2e_a.resize((size_t)kn * kn);
    o.uc2e_b.resize((size_t)kn * kn);
    o.dc2e_a.resize((size_t)kn * kn);
    o.dc2e_b.resize((size_t)kn * kn);
    for (int i = 0; i < kn; i++)
        for (int j = 0; j < kn; j++) {
            o.uc2e_a[(size_t)i * kn + j] = o.V[(size_t)i * kn + j] * sinv[j];
            o.uc2e_b[(size_t)i * kn + j] = o.U[(size_t)j * kn + i];
            o.dc2e_a[(size_t)i * kn + j] = o.U[(size_t)i * kn + j] * sinv[j];
            o.dc2e_b[(size_t)i * kn + j] = o.V[(size_t)j * kn + i];
        }
    if (!cached) {
        o.m2m.assign((size_t)8 * kn * kn, 0.0);
        o.l2l.assign((size_t)8 * kn * kn, 0.0);
        std::vector<double> tmp((size_t)kn * kn);
        for (int c = 0; c < 8; c++) {
            double sg[3] = {(c & 1) ? 0.5 : -0.5, (c & 2) ? 0.5 : -0.5, (c & 4) ? 0.5 : -0.5};
            // M2M: parent (edge 2) up-check at 2.95 g, child (edge 1) up-equiv at sg + 0.525 g
            std::vector<double> xc(3 * n), ye(3 * n);
            for (int i = 0; i < n; i++)
                for (int a = 0; a < 3; a++) {
                    xc[3 * i + a] = 2.0 * kOuterHalf * o.g[3 * i + a];
                    ye[3 * i + a] = sg[a] + kInnerHalf * o.g[3 * i + a];
                }
            std::vector<double> K = kernel_matrix(kernel, xc, ye);
            for (auto &v : K) v *= 2.0;  // q~ = (parent edge) q with child edge 1
            matmul(kn, kn, kn, o.uc2e_b.data(), K.data(), tmp.data());
            matmul(kn, kn, kn, o.uc2e_a.data(), tmp.data(), &o.m2m[(size_t)c * kn * kn]);
            // L2L: child (edge 1) down-check at 0.525 g, parent (edge 2) down-equiv at -sg + 2.95 g
            for (int i = 0; i < n; i++)
                for (int a = 0; a < 3; a++) {
                    xc[3 * i + a] = kInnerHalf * o.g[3 * i + a];
                    ye[3 * i + a] = -sg[a] + 2.0 * kOuterHalf * o.g[3 * i + a];
                }
            K = kernel_matrix(kernel, xc, ye);
            matmul(kn, kn, kn, o.dc2e_b.data(), K.data(), tmp.data());
            matmul(kn, kn, kn, o.dc2e_a.data(), tmp.data(), &o.l2l[(size_t)c * kn * kn]);
        }
        if (periodic) o.root = root_operator(kernel, p, periodic, ell, o.g);
        else o.root.clear();
        if (!cache_dir.empty()) save_cache(cache_path(cache_dir, o), o);
    }
}

}  // namespace pk
