// Plain binary64 kernel-independent FMM on the host (C++17, OpenMP): the CPU
// baseline that the GPU library's throughput is reported against.  It is a
// separate program written for plainness, not speed, and shares no code with
// the library or with the oracle.
//
//  * uniform octree of the unit cell [0,1)^3, depth chosen so that no leaf
//    holds more than leaf_max points (sources = targets);
//  * equivalent / check surfaces: the boundary points of a p x p x p grid on
//    cubes of half-width 0.525 h and 1.475 h around a box of width h (Sec. 2.2);
//  * S2M, M2M, M2L, L2L, L2T: check-surface kernel sums, then the
//    check-to-equivalent pseudo-inverse of Sec. 3.1 (one-sided Jacobi SVD,
//    singular values below a relative cut-off dropped), the operators formed
//    once at unit width and scaled by the kernels' homogeneity (degree -1);
//  * V list: children of the parent's neighbours that do not touch the box,
//    U list: the 27 boxes touching a leaf, both with periodic images;
//  * triply periodic: the root's downward check values from all images beyond
//    the adjacent layer, one dense operator (Algorithm 2 step c) assembled from
//    an Ewald sum of the periodic kernel minus the 27 nearest images.
// Kernels: Laplace 1/r (kernel 0) and the Stokeslet (1/8 pi)(I/r + r r^T/r^3)
// (kernel 1); periodic axes 0 (free space) or 7 (x, y, z).  Stokes TP needs a
// zero net force and Laplace TP a zero net charge (the k = 0 modes are left out).
#include <omp.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------- kernels ----------------

// K(r) into a k x k block (row-major), r = x - y != 0
inline void kernel_block(int kernel, double rx, double ry, double rz, double *K) {
    const double r2 = rx * rx + ry * ry + rz * rz, ir = 1.0 / std::sqrt(r2);
    if (kernel == 0) {
        K[0] = ir;
        return;
    }
    const double c = 1.0 / (8.0 * kPi), ir3 = ir * ir * ir, r[3] = {rx, ry, rz};
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) K[3 * a + b] = c * ((a == b ? ir : 0.0) + r[a] * r[b] * ir3);
}

// ---------------- surfaces ----------------

// boundary points of the p^3 grid on [-1, 1]^3 (6 (p-1)^2 + 2 of them)
std::vector<double> unit_surface(int p) {
    std::vector<double> s;
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++)
            for (int k = 0; k < p; k++) {
                if (i != 0 && i != p - 1 && j != 0 && j != p - 1 && k != 0 && k != p - 1) continue;
                s.push_back(-1.0 + 2.0 * i / (p - 1));
                s.push_back(-1.0 + 2.0 * j / (p - 1));
                s.push_back(-1.0 + 2.0 * k / (p - 1));
            }
    return s;
}

// ---------------- dense linear algebra ----------------

using Mat = std::vector<double>;  // row-major unless stated

// kernel matrix K(X, Y): rows = points of X x k, columns = points of Y x k
Mat kernel_matrix(int kernel, const std::vector<double> &X, const std::vector<double> &Y) {
    const int k = kernel == 0 ? 1 : 3, nx = (int)X.size() / 3, ny = (int)Y.size() / 3;
    Mat M((size_t)nx * k * ny * k);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nx; i++) {
        double B[9];
        for (int j = 0; j < ny; j++) {
            kernel_block(kernel, X[3 * i] - Y[3 * j], X[3 * i + 1] - Y[3 * j + 1], X[3 * i + 2] - Y[3 * j + 2], B);
            for (int a = 0; a < k; a++)
                for (int b = 0; b < k; b++) M[((size_t)i * k + a) * ny * k + (size_t)j * k + b] = B[a * k + b];
        }
    }
    return M;
}

// C (m x n) = A (m x q) B (q x n), all row-major
Mat matmul(const Mat &A, const Mat &B, int m, int q, int n) {
    Mat C((size_t)m * n, 0.0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; i++)
        for (int l = 0; l < q; l++) {
            const double a = A[(size_t)i * q + l];
            const double *b = &B[(size_t)l * n];
            double *c = &C[(size_t)i * n];
            for (int j = 0; j < n; j++) c[j] += a * b[j];
        }
    return C;
}

// Pseudo-inverse of a square m x m matrix by a one-sided (Hestenes) Jacobi SVD:
// columns of W = A V are rotated pairwise until mutually orthogonal; then
// A = U S V^T with S the column norms.  Singular values below cut * s_max are
// dropped.  Pairs are visited in round-robin order, each round's disjoint
// pairs in parallel.
Mat pinv(const Mat &A, int m, double cut) {
    std::vector<double> W((size_t)m * m), V((size_t)m * m, 0.0);  // column-major
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) W[(size_t)j * m + i] = A[(size_t)i * m + j];
    for (int i = 0; i < m; i++) V[(size_t)i * m + i] = 1.0;
    const int n2 = m + (m & 1);  // even count for the round robin (a dummy column when odd)
    std::vector<int> order(n2);
    for (int i = 0; i < n2; i++) order[i] = i;
    for (int sweep = 0; sweep < 60; sweep++) {
        int rotated = 0;
        for (int round = 0; round < n2 - 1; round++) {
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : rotated)
            for (int t = 0; t < n2 / 2; t++) {
                int i = order[t], j = order[n2 - 1 - t];
                if (i >= m || j >= m) continue;
                if (i > j) std::swap(i, j);
                double *wi = &W[(size_t)i * m], *wj = &W[(size_t)j * m];
                double a = 0, b = 0, g = 0;
                for (int r = 0; r < m; r++) {
                    a += wi[r] * wi[r];
                    b += wj[r] * wj[r];
                    g += wi[r] * wj[r];
                }
                if (std::fabs(g) <= 1e-15 * std::sqrt(a * b) || g == 0.0) continue;
                const double zeta = (b - a) / (2.0 * g);
                const double tn = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + tn * tn), s = c * tn;
                for (int r = 0; r < m; r++) {
                    const double x = wi[r], y = wj[r];
                    wi[r] = c * x - s * y;
                    wj[r] = s * x + c * y;
                }
                double *vi = &V[(size_t)i * m], *vj = &V[(size_t)j * m];
                for (int r = 0; r < m; r++) {
                    const double x = vi[r], y = vj[r];
                    vi[r] = c * x - s * y;
                    vj[r] = s * x + c * y;
                }
                rotated++;
            }
            // round-robin: keep order[0], rotate the rest by one
            const int last = order[n2 - 1];
            for (int t = n2 - 1; t > 1; t--) order[t] = order[t - 1];
            order[1] = last;
        }
        if (!rotated) break;
    }
    std::vector<double> sig(m);
    double smax = 0;
    for (int j = 0; j < m; j++) {
        double s = 0;
        for (int r = 0; r < m; r++) s += W[(size_t)j * m + r] * W[(size_t)j * m + r];
        sig[j] = std::sqrt(s);
        smax = std::max(smax, sig[j]);
    }
    // pinv = V S^-1 U^T, U column j = W column j / sig_j: pinv[i][l] = sum_j V[i][j] W[l][j] / sig_j^2
    Mat P((size_t)m * m, 0.0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; i++) {
        double *row = &P[(size_t)i * m];
        for (int j = 0; j < m; j++) {
            if (sig[j] <= cut * smax) continue;
            const double v = V[(size_t)j * m + i] / (sig[j] * sig[j]);
            const double *w = &W[(size_t)j * m];
            for (int l = 0; l < m; l++) row[l] += v * w[l];
        }
    }
    return P;
}

// ---------------- periodic far field (triply periodic, unit cell) ----------------

// Ewald sum of the periodic kernel minus its 27 nearest images, at r = x - y
// with |r_a| <= ~1.1.  Splitting parameter xi = 3: real-space images |n| <= 4,
// Fourier modes k = 2 pi m, |m| <= 6 (both tails below 1e-15).  The k = 0 mode
// is left out (zero cell average).
//  Laplace: psi = sum_n erfc(xi rho)/rho + 4 pi sum_k exp(-k^2/4xi^2)/k^2 cos(k.r) - pi/xi^2;
//  Stokes, the Stokeslet written as (1/8 pi)(I lap - grad grad) rho and its
//  biharmonic factor split so that the Fourier weight is
//  (I - k k^T/k^2)(1/k^2 + 1/4xi^2) exp(-k^2/4xi^2) and the real-space image
//  (1/8 pi)[(erfc(xi rho)/rho - (2 xi/sqrt pi) e^{-xi^2 rho^2}) I
//          + (erfc(xi rho)/rho + (2 xi/sqrt pi) e^{-xi^2 rho^2}) rho^ rho^^T].
// Near images (|n|_inf <= 1) enter as real-space image minus free-space kernel,
// finite at rho = 0 (Laplace -2 xi/sqrt pi, Stokes -(1/8 pi)(4 xi/sqrt pi) I).
struct Ewald {
    int kernel;
    double xi = 3.0;
    std::vector<double> km;  // Fourier modes: kx, ky, kz, weight (half space, doubled)
    explicit Ewald(int kern) : kernel(kern) {
        const int M = 6;
        for (int a = -M; a <= M; a++)
            for (int b = -M; b <= M; b++)
                for (int c = -M; c <= M; c++) {
                    // one of each +-m pair (cos is even): first nonzero index positive
                    if (a < 0 || (a == 0 && (b < 0 || (b == 0 && c <= 0)))) continue;
                    const double kx = 2 * kPi * a, ky = 2 * kPi * b, kz = 2 * kPi * c, k2 = kx * kx + ky * ky + kz * kz;
                    const double e = std::exp(-k2 / (4 * xi * xi));
                    const double w = kernel == 0 ? 2.0 * 4 * kPi * e / k2 : 2.0 * (1.0 / k2 + 1.0 / (4 * xi * xi)) * e;
                    km.insert(km.end(), {kx, ky, kz, w});
                }
    }
    void far(double rx, double ry, double rz, double *out) const {
        const int k = kernel == 0 ? 1 : 3;
        double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        const double c2 = 2 * xi / std::sqrt(kPi);
        const int NR = 4;
        for (int a = -NR; a <= NR; a++)
            for (int b = -NR; b <= NR; b++)
                for (int c = -NR; c <= NR; c++) {
                    const double d[3] = {rx + a, ry + b, rz + c};
                    const double rho2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    const bool near = std::abs(a) <= 1 && std::abs(b) <= 1 && std::abs(c) <= 1;
                    if (rho2 == 0.0) {  // coincident with a near image: the finite limit
                        if (kernel == 0) acc[0] += -c2;
                        else
                            for (int i = 0; i < 3; i++) acc[4 * i] += -2.0 * c2 / (8 * kPi);
                        continue;
                    }
                    const double rho = std::sqrt(rho2), ef = std::erfc(xi * rho), g = c2 * std::exp(-xi * xi * rho2);
                    const double s = near ? ef - 1.0 : ef;  // minus the free-space image when near
                    if (kernel == 0) {
                        acc[0] += s / rho;
                    } else {
                        const double A = (s / rho - g) / (8 * kPi), B = (s / rho + g) / (8 * kPi) / rho2;
                        for (int i = 0; i < 3; i++)
                            for (int j = 0; j < 3; j++) acc[3 * i + j] += (i == j ? A : 0.0) + B * d[i] * d[j];
                    }
                }
        for (size_t m = 0; m < km.size(); m += 4) {
            const double kx = km[m], ky = km[m + 1], kz = km[m + 2], w = km[m + 3];
            const double cs = w * std::cos(kx * rx + ky * ry + kz * rz);
            if (kernel == 0) {
                acc[0] += cs;
            } else {
                const double kv[3] = {kx, ky, kz}, k2 = kx * kx + ky * ky + kz * kz;
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) acc[3 * i + j] += cs * ((i == j ? 1.0 : 0.0) - kv[i] * kv[j] / k2);
            }
        }
        if (kernel == 0) acc[0] -= kPi / (xi * xi);
        for (int i = 0; i < k * k; i++) out[i] = acc[i];
    }
};

// ---------------- operators at unit box width ----------------

struct Ops {
    int kernel, p, periodic, k, n, kn;
    std::vector<double> surf;           // unit surface, n points
    Mat uc2e;                           // kn x kn: equivalent density from upward check values, width 1
    Mat dc2e;                           // kn x kn: the same for the downward pair (transpose of uc2e)
    Mat m2m[8];                         // parent check from child equivalent, through uc2e (level-free)
    Mat l2l[8];                         // child downward check from parent downward equivalent, parent width 1
    std::map<int, Mat> m2l;             // offset code -> K(dc_B, ue_A), width 1
    Mat far;                            // root: downward check values from the upward equivalent density
    double precompute_s = 0;
};

std::vector<double> place(const std::vector<double> &u, double half, double cx, double cy, double cz) {
    std::vector<double> s(u.size());
    for (size_t i = 0; i < u.size(); i += 3) {
        s[i] = cx + half * u[i];
        s[i + 1] = cy + half * u[i + 1];
        s[i + 2] = cz + half * u[i + 2];
    }
    return s;
}

inline int offset_code(int a, int b, int c) { return ((a + 3) * 7 + (b + 3)) * 7 + (c + 3); }

double svd_cut(int kernel, int p, int kn) {
    const double c = kernel == 0 ? std::pow(10.0, -(p + 2)) : std::pow(10.0, -p);
    return std::max(c, std::ldexp(1.0, -52) * kn);
}

std::shared_ptr<Ops> build_ops(int kernel, int p, int periodic) {
    auto t0 = std::chrono::steady_clock::now();
    auto O = std::make_shared<Ops>();
    O->kernel = kernel;
    O->p = p;
    O->periodic = periodic;
    O->k = kernel == 0 ? 1 : 3;
    O->surf = unit_surface(p);
    O->n = (int)O->surf.size() / 3;
    O->kn = O->n * O->k;
    const int kn = O->kn;
    const double ein = 0.525, eout = 1.475;  // half-widths (h = 1) of the inner and outer surfaces
    const auto inner = place(O->surf, ein, 0, 0, 0), outer = place(O->surf, eout, 0, 0, 0);
    // upward: check on the outer surface, equivalent on the inner one
    const Mat Kce = kernel_matrix(kernel, outer, inner);
    O->uc2e = pinv(Kce, kn, svd_cut(kernel, p, kn));
    // downward: check on the inner surface, equivalent on the outer one; the
    // kernels are symmetric, so that matrix is Kce^T and its pseudo-inverse uc2e^T
    O->dc2e.assign((size_t)kn * kn, 0.0);
    for (int i = 0; i < kn; i++)
        for (int j = 0; j < kn; j++) O->dc2e[(size_t)i * kn + j] = O->uc2e[(size_t)j * kn + i];
    for (int c = 0; c < 8; c++) {
        const double cx = (c & 1) ? 0.25 : -0.25, cy = (c & 2) ? 0.25 : -0.25, cz = (c & 4) ? 0.25 : -0.25;
        // M2M: child (width 1/2) equivalent -> parent (width 1) check -> parent equivalent
        const Mat Kpc = kernel_matrix(kernel, outer, place(O->surf, 0.5 * ein, cx, cy, cz));
        O->m2m[c] = matmul(O->uc2e, Kpc, kn, kn, kn);
        // L2L: parent (width 1) downward equivalent -> child (width 1/2) downward check
        O->l2l[c] = kernel_matrix(kernel, place(O->surf, 0.5 * ein, cx, cy, cz), outer);
    }
    for (int a = -3; a <= 3; a++)
        for (int b = -3; b <= 3; b++)
            for (int c = -3; c <= 3; c++) {
                if (std::max({std::abs(a), std::abs(b), std::abs(c)}) < 2) continue;
                O->m2l[offset_code(a, b, c)] = kernel_matrix(kernel, inner, place(O->surf, ein, a, b, c));
            }
    if (periodic == 7) {
        // root (width 1): downward check on the inner surface from the upward equivalent density (inner surface)
        const Ewald E(kernel);
        const int n = O->n, k = O->k;
        O->far.assign((size_t)kn * kn, 0.0);
#pragma omp parallel for schedule(dynamic, 4)
        for (int i = 0; i < n; i++) {
            double B[9];
            for (int j = 0; j < n; j++) {
                E.far(inner[3 * i] - inner[3 * j], inner[3 * i + 1] - inner[3 * j + 1], inner[3 * i + 2] - inner[3 * j + 2], B);
                for (int a = 0; a < k; a++)
                    for (int b = 0; b < k; b++) O->far[((size_t)i * k + a) * kn + (size_t)j * k + b] = B[a * k + b];
            }
        }
    }
    O->precompute_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return O;
}

std::mutex g_ops_mutex;
std::map<std::tuple<int, int, int>, std::shared_ptr<Ops>> g_ops;

std::shared_ptr<Ops> ops_for(int kernel, int p, int periodic, bool *built) {
    std::lock_guard<std::mutex> lk(g_ops_mutex);
    auto key = std::make_tuple(kernel, p, periodic);
    auto it = g_ops.find(key);
    *built = it == g_ops.end();
    if (*built) it = g_ops.emplace(key, build_ops(kernel, p, periodic)).first;
    return it->second;
}

// Rows r0 <= i < r1 of Y_j += scale * M X_j for j < nc, M given column-major
// (MT[l * kn + i] = M[i][l]).  Blocks of 16 rows x 4 vectors are accumulated in registers over
// the full inner dimension (an outer product per column of M: the 8 row
// entries are contiguous, so the row loop vectorises without reassociating
// any sum); rows past the last full block are summed one by one.
void apply_block(const double *MT, int kn, const double *const *X, double *const *Y, int nc, double scale, int r0,
                 int r1) {
    constexpr int RB = 16, CB = 4;
    const int kr = r0 + (r1 - r0) / RB * RB;
    for (int i0 = r0; i0 < kr; i0 += RB)
        for (int j0 = 0; j0 < nc; j0 += CB) {
            const int nb = std::min(CB, nc - j0);
            const double *x[CB];
            for (int j = 0; j < CB; j++) x[j] = X[j0 + std::min(j, nb - 1)];
            double acc[CB][RB] = {};
            for (int l = 0; l < kn; l++) {
                const double *m = MT + (size_t)l * kn + i0;
#pragma GCC unroll 4
                for (int j = 0; j < CB; j++) {
                    const double xv = x[j][l];
#pragma GCC unroll 16
                    for (int i = 0; i < RB; i++) acc[j][i] += m[i] * xv;
                }
            }
            for (int j = 0; j < nb; j++)
                for (int i = 0; i < RB; i++) Y[j0 + j][i0 + i] += scale * acc[j][i];
        }
    for (int i = kr; i < r1; i++)
        for (int j = 0; j < nc; j++) {
            double a = 0.0;
            for (int l = 0; l < kn; l++) a += MT[(size_t)l * kn + i] * X[j][l];
            Y[j][i] += scale * a;
        }
}

Mat transpose(const Mat &M, int n) {
    Mat T((size_t)n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) T[(size_t)j * n + i] = M[(size_t)i * n + j];
    return T;
}

struct Transposed {  // column-major copies of the operators for apply_block
    Mat uc2e, dc2e, m2m[8], l2l[8], far;
    std::map<int, Mat> m2l;
};

std::mutex g_tr_mutex;
std::map<const Ops *, std::shared_ptr<Transposed>> g_tr;

std::shared_ptr<Transposed> transposed(const Ops &O) {
    std::lock_guard<std::mutex> lk(g_tr_mutex);
    auto &t = g_tr[&O];
    if (!t) {
        t = std::make_shared<Transposed>();
        t->uc2e = transpose(O.uc2e, O.kn);
        t->dc2e = transpose(O.dc2e, O.kn);
        for (int c = 0; c < 8; c++) {
            t->m2m[c] = transpose(O.m2m[c], O.kn);
            t->l2l[c] = transpose(O.l2l[c], O.kn);
        }
        for (auto &kv : O.m2l) t->m2l[kv.first] = transpose(kv.second, O.kn);
        if (!O.far.empty()) t->far = transpose(O.far, O.kn);
    }
    return t;
}

}  // namespace

extern "C" {

// Evaluate u(x_i) = sum_j K(x_i - y_j) f_j (with all periodic images when
// periodic = 7) for N points x (sources = targets) in [0, 1)^3, row-major
// [N][3]; f and u are [N][k] (k = 1 Laplace, 3 Stokes).  The coincident pair
// is left out.  times[0..2] (may be NULL): operator setup (0 when cached),
// tree, evaluation, in seconds.  *depth_out (may be NULL): the tree depth.
// Returns 0, or -1 for bad arguments (kernel not 0/1, periodic not 0/7,
// p < 2, leaf_max < 1, a point outside the cell).
int kifmm_cpu_eval(int kernel, int periodic, int p, int leaf_max, int64_t N, const double *x, const double *f,
                   double *u, double *times, int *depth_out) {
    if ((kernel != 0 && kernel != 1) || (periodic != 0 && periodic != 7) || p < 2 || leaf_max < 1 || N < 0)
        return -1;
    for (int64_t i = 0; i < 3 * N; i++)
        if (!(x[i] >= 0.0 && x[i] < 1.0)) return -1;
    using clk = std::chrono::steady_clock;
    bool built = false;
    auto O = ops_for(kernel, p, periodic, &built);
    auto TR = transposed(*O);
    const auto t1 = clk::now();
    const int k = O->k, kn = O->kn, n = O->n;
    // ---- uniform tree: the shallowest depth (<= 10) with at most leaf_max points per box ----
    int D = 0;
    std::vector<int> cnt;
    for (;; D++) {
        const int64_t side = 1LL << D;
        cnt.assign((size_t)(side * side * side), 0);
        int mx = 0;
        for (int64_t i = 0; i < N; i++) {
            const int64_t a = (int64_t)(x[3 * i] * side), b = (int64_t)(x[3 * i + 1] * side),
                          c = (int64_t)(x[3 * i + 2] * side);
            mx = std::max(mx, ++cnt[(size_t)((a * side + b) * side + c)]);
        }
        if (mx <= leaf_max || D == 10) break;
    }
    const int S = 1 << D;
    const size_t nleaf = (size_t)S * S * S;
    std::vector<int64_t> start(nleaf + 1, 0), perm(N);
    for (size_t b = 0; b < nleaf; b++) start[b + 1] = start[b] + cnt[b];
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < N; i++) {
            const int64_t a = (int64_t)(x[3 * i] * S), b = (int64_t)(x[3 * i + 1] * S), c = (int64_t)(x[3 * i + 2] * S);
            perm[fill[(size_t)((a * S + b) * S + c)]++] = i;
        }
    }
    std::vector<double> xs(3 * N), fs((size_t)N * k), us((size_t)N * k, 0.0);
    for (int64_t i = 0; i < N; i++) {
        for (int a = 0; a < 3; a++) xs[3 * i + a] = x[3 * perm[i] + a];
        for (int a = 0; a < k; a++) fs[(size_t)i * k + a] = f[(size_t)perm[i] * k + a];
    }
    const auto t2 = clk::now();
    // ---- per-level densities ----
    std::vector<std::vector<double>> up(D + 1), dn(D + 1), chk(D + 1);
    for (int l = 0; l <= D; l++) {
        const size_t nb = (size_t)1 << (3 * l);
        up[l].assign(nb * kn, 0.0);
        dn[l].assign(nb * kn, 0.0);
        chk[l].assign(nb * kn, 0.0);
    }
    auto box_of = [](int a, int b, int c, int l) { return ((size_t)a << (2 * l)) + ((size_t)b << l) + (size_t)c; };
    auto centre = [](int a, double h) { return (a + 0.5) * h; };
    const double hD = 1.0 / S;
    // ---- S2M: check values on the outer surface of each leaf, then its equivalent density ----
#pragma omp parallel for schedule(dynamic, 16)
    for (size_t B = 0; B < nleaf; B++) {
        const int a = (int)(B >> (2 * D)), b = (int)((B >> D) & (S - 1)), c = (int)(B & (S - 1));
        const double cx = centre(a, hD), cy = centre(b, hD), cz = centre(c, hD), e = 1.475 * hD;
        double *q = &chk[D][B * kn], K[9];
        for (int i = 0; i < n; i++) {
            const double px = cx + e * O->surf[3 * i], py = cy + e * O->surf[3 * i + 1], pz = cz + e * O->surf[3 * i + 2];
            for (int64_t s = start[B]; s < start[B + 1]; s++) {
                kernel_block(kernel, px - xs[3 * s], py - xs[3 * s + 1], pz - xs[3 * s + 2], K);
                for (int r = 0; r < k; r++)
                    for (int t = 0; t < k; t++) q[i * k + r] += K[r * k + t] * fs[(size_t)s * k + t];
            }
        }
    }
    // every vector of X through one operator; tasks of up to 128 vectors x 128
    // rows (distinct tasks write distinct entries: each Y_j occurs once)
    auto apply_all = [&](const Mat &MT, std::vector<const double *> &X, std::vector<double *> &Y, double scale) {
        const int nc = (int)X.size(), per = 128, rows = 128;
        const int ncb = (nc + per - 1) / per, nrb = (kn + rows - 1) / rows;
#pragma omp parallel for schedule(dynamic, 1)
        for (int t = 0; t < ncb * nrb; t++) {
            const int j0 = t / nrb * per, r0 = t % nrb * rows;
            apply_block(MT.data(), kn, X.data() + j0, Y.data() + j0, std::min(per, nc - j0), scale, r0,
                        std::min(kn, r0 + rows));
        }
    };
    {
        std::vector<const double *> X;
        std::vector<double *> Y;
        for (size_t B = 0; B < nleaf; B++) {
            X.push_back(&chk[D][B * kn]);
            Y.push_back(&up[D][B * kn]);
        }
        apply_all(TR->uc2e, X, Y, hD);
    }
    // ---- M2M ----
    for (int l = D - 1; l >= 0; l--) {
        const int s = 1 << l;
        for (int oc = 0; oc < 8; oc++) {
            std::vector<const double *> X;
            std::vector<double *> Y;
            for (int a = 0; a < s; a++)
                for (int b = 0; b < s; b++)
                    for (int c = 0; c < s; c++) {
                        const size_t ch = box_of(2 * a + (oc & 1), 2 * b + (oc >> 1 & 1), 2 * c + (oc >> 2 & 1), l + 1);
                        X.push_back(&up[l + 1][ch * kn]);
                        Y.push_back(&up[l][box_of(a, b, c, l) * kn]);
                    }
            apply_all(TR->m2m[oc], X, Y, 1.0);
        }
    }
    // ---- root: far field of the images beyond the adjacent layer ----
    if (periodic == 7) {
        std::vector<const double *> X{up[0].data()};
        std::vector<double *> Y{chk[0].data()};
        apply_all(TR->far, X, Y, 1.0);
        std::vector<const double *> X2{chk[0].data()};
        std::vector<double *> Y2{dn[0].data()};
        apply_all(TR->dc2e, X2, Y2, 1.0);
    }
    // ---- downward: L2L from the parent, V-list M2L, then the equivalent density ----
    for (int l = 1; l <= D; l++) {
        const int s = 1 << l;
        const double h = 1.0 / s;
        std::fill(chk[l].begin(), chk[l].end(), 0.0);
        for (int oc = 0; oc < 8; oc++) {
            std::vector<const double *> X;
            std::vector<double *> Y;
            for (int a = 0; a < s / 2; a++)
                for (int b = 0; b < s / 2; b++)
                    for (int c = 0; c < s / 2; c++) {
                        X.push_back(&dn[l - 1][box_of(a, b, c, l - 1) * kn]);
                        Y.push_back(&chk[l][box_of(2 * a + (oc & 1), 2 * b + (oc >> 1 & 1), 2 * c + (oc >> 2 & 1), l) * kn]);
                    }
            apply_all(TR->l2l[oc], X, Y, 1.0 / (2.0 * h));  // operator formed at parent width 1
        }
        for (auto &kv : TR->m2l) {
            const int code = kv.first, oa = code / 49 - 3, ob = code / 7 % 7 - 3, ocz = code % 7 - 3;
            std::vector<const double *> X;
            std::vector<double *> Y;
            for (int a = 0; a < s; a++)
                for (int b = 0; b < s; b++)
                    for (int c = 0; c < s; c++) {
                        const int A[3] = {a + oa, b + ob, c + ocz}, Bc[3] = {a, b, c};
                        bool ok = true;
                        for (int d = 0; d < 3 && ok; d++) {
                            // the source's parent must touch (or be) the target's parent
                            const int dp = (int)std::floor(A[d] / 2.0) - Bc[d] / 2;
                            if (dp < -1 || dp > 1) ok = false;
                            if (periodic == 0 && (A[d] < 0 || A[d] >= s)) ok = false;
                        }
                        if (!ok) continue;
                        const int wa = ((A[0] % s) + s) % s, wb = ((A[1] % s) + s) % s, wc = ((A[2] % s) + s) % s;
                        X.push_back(&up[l][box_of(wa, wb, wc, l) * kn]);
                        Y.push_back(&chk[l][box_of(a, b, c, l) * kn]);
                    }
            if (!X.empty()) apply_all(kv.second, X, Y, 1.0 / h);
        }
        std::vector<const double *> X;
        std::vector<double *> Y;
        for (size_t B = 0; B < ((size_t)1 << (3 * l)); B++) {
            X.push_back(&chk[l][B * kn]);
            Y.push_back(&dn[l][B * kn]);
        }
        apply_all(TR->dc2e, X, Y, h);
    }
    // ---- leaves: L2T from the downward equivalent surface, P2P over the 27 neighbours ----
#pragma omp parallel for schedule(dynamic, 16)
    for (size_t B = 0; B < nleaf; B++) {
        const int a = (int)(B >> (2 * D)), b = (int)((B >> D) & (S - 1)), c = (int)(B & (S - 1));
        const double cx = centre(a, hD), cy = centre(b, hD), cz = centre(c, hD), e = 1.475 * hD;
        const double *phi = &dn[D][B * kn];
        double K[9];
        for (int64_t t = start[B]; t < start[B + 1]; t++) {
            double acc[3] = {0, 0, 0};
            const double tx = xs[3 * t], ty = xs[3 * t + 1], tz = xs[3 * t + 2];
            for (int i = 0; i < n; i++) {
                kernel_block(kernel, tx - (cx + e * O->surf[3 * i]), ty - (cy + e * O->surf[3 * i + 1]),
                             tz - (cz + e * O->surf[3 * i + 2]), K);
                for (int r = 0; r < k; r++)
                    for (int q = 0; q < k; q++) acc[r] += K[r * k + q] * phi[i * k + q];
            }
            for (int da = -1; da <= 1; da++)
                for (int db = -1; db <= 1; db++)
                    for (int dc = -1; dc <= 1; dc++) {
                        const int A[3] = {a + da, b + db, c + dc};
                        double shift[3] = {0, 0, 0};
                        bool ok = true;
                        for (int d = 0; d < 3; d++) {
                            if (A[d] < 0 || A[d] >= S) {
                                if (periodic == 0) ok = false;
                                shift[d] = A[d] < 0 ? -1.0 : 1.0;  // the image of the wrapped box
                            }
                        }
                        if (!ok) continue;
                        const size_t Ab = box_of((A[0] + S) % S, (A[1] + S) % S, (A[2] + S) % S, D);
                        for (int64_t s2 = start[Ab]; s2 < start[Ab + 1]; s2++) {
                            const double rx = tx - (xs[3 * s2] + shift[0]), ry = ty - (xs[3 * s2 + 1] + shift[1]),
                                         rz = tz - (xs[3 * s2 + 2] + shift[2]);
                            if (rx == 0.0 && ry == 0.0 && rz == 0.0) continue;
                            kernel_block(kernel, rx, ry, rz, K);
                            for (int r = 0; r < k; r++)
                                for (int q = 0; q < k; q++) acc[r] += K[r * k + q] * fs[(size_t)s2 * k + q];
                        }
                    }
            for (int r = 0; r < k; r++) us[(size_t)t * k + r] = acc[r];
        }
    }
    // Laplace, triply periodic: the Ewald convention (k = 0 left out) makes the
    // potential of a neutral cell depend on its trace second moment
    // sum q |y - c|^2, which the exterior field -- and so the root's equivalent
    // density -- does not carry.  The root operator applied to the equivalent
    // density misses (2 pi / 3)(sum q |y - c|^2 - sum phi^u |y^u - c|^2), c the
    // cell centre; it is added back here.
    double cst = 0.0;
    if (kernel == 0 && periodic == 7) {
        double m_src = 0.0, m_eq = 0.0;
        for (int64_t i = 0; i < N; i++) {
            const double dx = xs[3 * i] - 0.5, dy = xs[3 * i + 1] - 0.5, dz = xs[3 * i + 2] - 0.5;
            m_src += fs[i] * (dx * dx + dy * dy + dz * dz);
        }
        for (int i = 0; i < n; i++) {
            const double e = 0.525, dx = e * O->surf[3 * i], dy = e * O->surf[3 * i + 1], dz = e * O->surf[3 * i + 2];
            m_eq += up[0][i] * (dx * dx + dy * dy + dz * dz);
        }
        cst = 2.0 * kPi / 3.0 * (m_src - m_eq);
    }
    for (int64_t i = 0; i < N; i++)
        for (int r = 0; r < k; r++) u[(size_t)perm[i] * k + r] = us[(size_t)i * k + r] + cst;
    const auto t3 = clk::now();
    if (times) {
        times[0] = built ? O->precompute_s : 0.0;
        times[1] = std::chrono::duration<double>(t2 - t1).count();
        times[2] = std::chrono::duration<double>(t3 - t2).count();
    }
    if (depth_out) *depth_out = D;
    return 0;
}

int kifmm_cpu_threads() { return omp_get_max_threads(); }

}  // extern "C"
