// Host-side operator precompute (Algorithm 2, Stage 1; Sec. 2.2-2.3, 3.1).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace pk {

// Surface radii as multiples of the box edge (Sec. 2.2): the upward
// equivalent and downward check surfaces are cubes of edge 1.05, the upward
// check and downward equivalent surfaces cubes of edge 2.95, all centred on
// the box.  Half-widths:
constexpr double kInnerHalf = 0.525;
constexpr double kOuterHalf = 1.475;

int surface_count(int p);                       // 6(p-1)^2 + 2
std::vector<double> surface_grid(int p);        // [n][3] on the cube [-1,1]^3

// k x k block K(x, y) of the free-space kernel (row-major).
void kernel_block(int kernel, const double *x, const double *y, double *out);

// Dense kernel matrix [n_x*k][n_y*k] (row-major).
std::vector<double> kernel_matrix(int kernel, const std::vector<double> &x,
                                  const std::vector<double> &y);

// One-sided Jacobi SVD of a square m x m row-major matrix A = U S V^T.
// U, V row-major m x m, S descending.
void jacobi_svd(int m, const std::vector<double> &A, std::vector<double> &U,
                std::vector<double> &S, std::vector<double> &V);

struct HostOps {
    int kernel = 0, k = 1, p = 0, n = 0, kn = 0;
    unsigned periodic = 0;
    int ell = 0;
    int nimg = -1;                  // >= 0: finite array of cells along the periodic axis (copies |n| <= nimg)
    double eps_rel = 0;             // singular values <= eps_rel * s_max are dropped
    std::vector<double> g;          // [n][3] unit surface grid
    std::vector<double> U, S, V;    // SVD of A_up1 = K(1.475 g, 0.525 g)
    // check-to-equivalent factors, applied as two products (Sec. 3.1):
    //   upward:   phi = (V S+) (U^T q)      downward: phi = (U S+) (V^T q)
    std::vector<double> uc2e_a, uc2e_b, dc2e_a, dc2e_b;
    std::vector<double> m2m;        // [8][kn][kn] child octant -> parent up density
    std::vector<double> l2l;        // [8][kn][kn] parent down density -> child octant
    std::vector<double> root;       // [kn][kn] far-field check operator (periodic)
};

// Singular values <= svd_cut(...) * s_max are dropped in the check-to-equivalent
// solves (Sec. 3.1's eps_SVD, relative): precision 0 = binary64 operators,
// 1 = binary32 (MIXED); kn = the matrix dimension.  PKIFMM_EPS in the
// environment replaces the rule (measurement sweeps).
double svd_cut(int kernel, int p, int precision, int kn);

// Pieces shared by the host and device builds: field set-up and surface grid;
// the operator cache (false / no-op for an empty directory); the
// check-to-equivalent factors (V S+, U^T, U S+, V^T) from U, S, V and eps_rel.
void init_ops(HostOps &o, int kernel, int p, unsigned periodic, int ell, double eps_rel, int nimg = -1);
bool load_cached_ops(HostOps &o, const std::string &cache_dir);
void save_cached_ops(HostOps &o, const std::string &cache_dir);
void c2e_factors(HostOps &o);

// Build all host operators; throws std::runtime_error on failure.
// cache_dir may be empty.
void build_host_ops(HostOps &ops, int kernel, int p, unsigned periodic, int ell,
                    double eps_rel, const std::string &cache_dir, int nimg = -1);

// K^{P,F}_ell(r) block for a unit periodic box, r a difference vector with
// |r_a| <= ~1.1; periodic in the axes of `periodic`.
void far_kernel_block(int kernel, unsigned periodic, int ell, const double *r, double *out);

// Root operator M[kn][kn] = K^{P,F}_ell(x^d, y^u) + sum_{1<|p|<=ell} K(x^d, y^u + p).
// nimg >= 0: the finite array of cells along the periodic axis instead.
std::vector<double> root_operator(int kernel, int p, unsigned periodic, int ell,
                                  const std::vector<double> &g, int nimg = -1);

void matmul(int m, int n, int kk, const double *A, const double *B, double *C);  // C = A B

// The same operators built on the current CUDA device (precompute_dev.cu):
// surface kernel matrices, the one-sided Jacobi SVD, the M2M / L2L products
// and the root operator's far-field table in binary64 kernels; U, S, V and
// the operators are copied back into `ops`.  Throws pk::Error on failure.
// phases (may be null, 4 entries): seconds of the SVD, the M2M / L2L products
// and the root table, then the number of Jacobi sweeps (the last one rotating
// nothing); left untouched when the operators come from the cache.
void build_device_ops(HostOps &ops, int kernel, int p, unsigned periodic, int ell,
                      double eps_rel, const std::string &cache_dir, double *phases = nullptr, int nimg = -1);

// The V-list M2L operators of the 316 offsets o in one shared basis (the
// MIXED path): G = sum_o K_o K_o^T = U S U^T (K_o = K(0.525 g_i, o + 0.525 g_j),
// kn x kn), Ub = the first r columns of U, C_o = Ub^T K_o Ub.  r: the smallest
// multiple of 64 whose next relative singular value sqrt(S_r / S_0) is <= tau,
// or rank_override if > 0 (r = kn keeps every column).  Built on the device in
// binary64.  Throws pk::Error on failure.
struct M2LBasis {
    int r = 0;                  // 0: no basis (dense operators)
    std::vector<double> Ub;     // [kn][r] orthonormal columns
    std::vector<float> C;       // [316][r][r]
    std::vector<double> sig;    // [kn] singular values of the stacked operators / the largest
};
void build_m2l_basis(int kernel, int p, double tau, int rank_override, M2LBasis &B);

// C[b] = A[b] B[b] for b < batch, row-major binary64 host arrays with element
// strides between the batch's matrices (0: one matrix for all), computed on the
// current device.
void matmul_device(int m, int n, int kk, const double *A, long long sA, const double *B, long long sB, double *C,
                   long long sC, int batch);

}  // namespace pk
