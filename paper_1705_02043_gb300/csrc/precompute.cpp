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
#include "far_field.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <filesystem>
#include <fstream>
#include <numeric>
#include <stdexcept>
#include <unistd.h>

namespace pk {


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

void kernel_block(int kernel, const double *x, const double *y, double *out) { ff::kernel_block(kernel, x, y, out); }

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

// One-sided (Hestenes) Jacobi preconditioned by QR with column pivoting
// (Drmac and Veselic): A P = Q R by Householder reflectors, then the columns of
// R^T are orthogonalised by plane rotations accumulated in Vt, so that
// R^T = U_x S V_x^T and A = (Q V_x) S (P U_x)^T; on these matrices the
// rotations settle in about a third of the sweeps plain Jacobi on A needs.
// Pairs are scheduled round-robin so the m/2 rotations of one round are
// independent.  Columns are stored as rows for contiguous access.
void jacobi_svd(int m, const std::vector<double> &A, std::vector<double> &U,
                std::vector<double> &S, std::vector<double> &V) {
    int mm = m + (m & 1);  // even player count; index m (if odd) is a bye
    // ---- A P = Q R: W holds the columns of A as rows; reflector k in hv[k] ----
    std::vector<double> W((size_t)m * m), hv((size_t)m * m, 0.0), tau(m, 0.0), c2(m);
    std::vector<int> perm(m);
    std::iota(perm.begin(), perm.end(), 0);
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) W[(size_t)j * m + i] = A[(size_t)i * m + j];
    for (int j = 0; j < m; j++) {
        double v = 0;
        for (int i = 0; i < m; i++) v += W[(size_t)j * m + i] * W[(size_t)j * m + i];
        c2[j] = v;
    }
    for (int k = 0; k < m; k++) {
        int js = k;  // largest trailing norm, lowest index on ties
        for (int j = k + 1; j < m; j++)
            if (c2[j] > c2[js]) js = j;
        if (js != k) {
            std::swap_ranges(W.begin() + (size_t)k * m, W.begin() + (size_t)(k + 1) * m, W.begin() + (size_t)js * m);
            std::swap(c2[k], c2[js]);
            std::swap(perm[k], perm[js]);
        }
        double *x = &W[(size_t)k * m], ss = 0;
        for (int i = k; i < m; i++) ss += x[i] * x[i];
        const double x0 = x[k], nrm = std::sqrt(ss), alpha = x0 >= 0 ? -nrm : nrm, v0 = x0 - alpha;
        const double vn2 = ss - x0 * x0 + v0 * v0, t = vn2 > 0 ? 2.0 / vn2 : 0.0;
        double *v = &hv[(size_t)k * m];
        v[k] = v0;
        for (int i = k + 1; i < m; i++) v[i] = x[i];
        tau[k] = t;
        x[k] = alpha;
        for (int i = k + 1; i < m; i++) x[i] = 0.0;
#pragma omp parallel for schedule(static)
        for (int j = k + 1; j < m; j++) {
            double *w = &W[(size_t)j * m], d = 0, n2 = 0;
            for (int i = k; i < m; i++) d += v[i] * w[i];
            d *= t;
            for (int i = k; i < m; i++) {
                w[i] -= d * v[i];
                if (i > k) n2 += w[i] * w[i];
            }
            c2[j] = n2;
        }
    }
    // ---- Jacobi on the columns of R^T (the rows of R) ----
    std::vector<double> At((size_t)m * m, 0.0), Vt((size_t)m * m, 0.0);
    for (int i = 0; i < m; i++)
        for (int j = i; j < m; j++) At[(size_t)i * m + j] = W[(size_t)j * m + i];
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
    // Q V_x: the reflectors applied in reverse order to the rows of Vt
    for (int k = m - 1; k >= 0; k--) {
        const double t = tau[k];
        if (t == 0.0) continue;
        const double *v = &hv[(size_t)k * m];
#pragma omp parallel for schedule(static)
        for (int j = 0; j < m; j++) {
            double *y = &Vt[(size_t)j * m], d = 0;
            for (int i = k; i < m; i++) d += v[i] * y[i];
            d *= t;
            for (int i = k; i < m; i++) y[i] -= d * v[i];
        }
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
            U[(size_t)i * m + jj] = Vt[(size_t)j * m + i];              // Q V_x
            V[(size_t)perm[i] * m + jj] = At[(size_t)j * m + i] * inv;  // P U_x
        }
    }
}

// ---------------- far-field periodic kernel K^{P,F} (far_field.h) ----------------

void far_kernel_block(int kernel, unsigned periodic, int ell, const double *r, double *out) {
    if (!ff::far_kernel_block(kernel, periodic, ell, r, out))
        throw std::runtime_error("far kernel: periodicity not supported");
}

std::vector<double> root_operator(int kernel, int p, unsigned periodic, int ell,
                                  const std::vector<double> &g, int nimg) {
    int k = kernel == 0 ? 1 : 3, n = (int)g.size() / 3, kn = n * k, w = 2 * p - 1;
    // table of K^{P,F} + near-layer images 2..ell on the difference lattice
    std::vector<double> tab((size_t)w * w * w * k * k);
    const int axis = periodic == 1 ? 0 : periodic == 2 ? 1 : 2;
    if (nimg >= 0) {
        if (!(periodic == 1 || periodic == 2 || periodic == 4))
            throw std::runtime_error("root operator: a finite array runs along one axis");
    } else {
        double probe[9], r0[3] = {0, 0, 0};
        if (!ff::far_kernel_block(kernel, periodic, ell, r0, probe))
            throw std::runtime_error("root operator: periodicity not supported");
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int t = 0; t < w * w * w; t++) {
        if (nimg >= 0) ff::finite_table_entry(kernel, axis, nimg, p, kInnerHalf, t, &tab[(size_t)t * k * k]);
        else ff::root_table_entry(kernel, periodic, ell, p, kInnerHalf, t, &tab[(size_t)t * k * k]);
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
    std::string name = buf;
    if (o.nimg >= 0) name.insert(name.size() - 4, "_n" + std::to_string(o.nimg));  // finite arrays
    return dir + name;
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

double svd_cut(int kernel, int p, int precision, int kn) {
    // Sec. 3.1 leaves eps_SVD open.  The near-null right singular vectors of
    // the surface matrix (the Stokes double-layer-like modes, and the
    // smallest Laplace modes) fit the check values but not the fields at the
    // other surfaces an equivalent density is later evaluated on (the
    // parent's check surface, a V-list box's check surface, the targets), so
    // inverting them amplifies the error the check values already carry from
    // the previous translation.  The cut that minimises the error of a
    // translation chain (S2M, M2M up 1-5 levels, M2L, L2L down, L2T, against
    // direct sums) is about 1e-2 of the error the surfaces reach at that p:
    // Stokes 10^-p, Laplace 10^-(p+2), never below the numerical-rank
    // threshold of Table 1, 2^-52 dim(A).  Binary32 operators (MIXED) carry
    // rounding of ~1e-7 relative into every solve, which the same argument
    // turns into a floor of 1e-7.
    const double table1 = std::ldexp(1.0, -52) * kn;
    double eps = std::pow(10.0, -(kernel == 0 ? p + 2 : p));
    if (precision != 0) eps = std::max(eps, 1e-7);
    if (const char *e = std::getenv("PKIFMM_EPS"); e && std::atof(e) > 0) eps = std::atof(e);  // measurement sweeps
    return std::max(eps, table1);
}

void init_ops(HostOps &o, int kernel, int p, unsigned periodic, int ell, double eps_rel, int nimg) {
    o.nimg = nimg;
    o.kernel = kernel;
    o.k = kernel == 0 ? 1 : 3;
    o.p = p;
    o.n = surface_count(p);
    o.kn = o.n * o.k;
    o.periodic = periodic;
    o.ell = ell;
    o.eps_rel = eps_rel;
    o.g = surface_grid(p);
}

bool load_cached_ops(HostOps &o, const std::string &cache_dir) {
    return !cache_dir.empty() && load_cache(cache_path(cache_dir, o), o);
}

void save_cached_ops(HostOps &o, const std::string &cache_dir) {
    if (!cache_dir.empty()) save_cache(cache_path(cache_dir, o), o);
}

void c2e_factors(HostOps &o) {
    const int kn = o.kn;
    double cut = o.eps_rel * o.S[0];
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
}

void build_host_ops(HostOps &o, int kernel, int p, unsigned periodic, int ell, double eps_rel,
                    const std::string &cache_dir, int nimg) {
    init_ops(o, kernel, p, periodic, ell, eps_rel, nimg);
    const int kn = o.kn, n = o.n;
    bool cached = load_cached_ops(o, cache_dir);
    if (!cached) {
        std::vector<double> xu(3 * n), yu(3 * n);
        for (int i = 0; i < 3 * n; i++) {
            xu[i] = kOuterHalf * o.g[i];
            yu[i] = kInnerHalf * o.g[i];
        }
        std::vector<double> A = kernel_matrix(kernel, xu, yu);  // A_up1
        jacobi_svd(kn, A, o.U, o.S, o.V);
    }
    c2e_factors(o);
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
        if (periodic) o.root = root_operator(kernel, p, periodic, ell, o.g, nimg);
        else o.root.clear();
        save_cached_ops(o, cache_dir);
    }
}

}  // namespace pk
