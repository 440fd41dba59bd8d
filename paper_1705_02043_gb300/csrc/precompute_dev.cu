// Device operator precompute (Algorithm 2, Stage 1; Sec. 2.2-2.3, 3.1), in
// binary64 on the current CUDA device.  Same operators as the host build
// (precompute.cpp), built by kernels:
//
// * surface kernel matrices: one thread per (check point, equivalent point);
// * A_up1 = U S V^T by QR with column pivoting (Householder, one launch for
//   the pivot and reflector and one for the trailing update per column), then
//   one-sided (Hestenes) Jacobi on R^T: the columns of R^T are kept as rows of
//   At and orthogonalised by plane rotations, accumulated in Vt; Q and the
//   permutation are applied at the end.
//   Pairs follow the circle method (player 0 fixed, the others rotating one
//   place per round), so the m/2 rotations of a round touch disjoint rows and
//   run as one launch, one block per pair; a sweep is m - 1 rounds and the
//   sweeps stop when a sweep rotates nothing (|a_p . a_q| <= 1e-15 |a_p||a_q|
//   for every pair), at most 80 sweeps.  Singular values are the row norms of
//   At, ranked in descending order (ties by index, as a stable sort);
// * M2M and L2L: (V S+) (U^T K) for the 8 octants, two batched binary64
//   GEMMs per family;
// * root operator: the K^{P,F}_ell table on the difference lattice of the
//   surface grid (far_field.h, one thread per entry; for a finite array of
//   cells the plain sum over the non-adjacent copies), then scattered to the
//   kn x kn matrix.
// The check-to-equivalent factors themselves (O(kn^2) scalings of U, S, V)
// are formed on the host from the copied-back SVD, as in the host build.
#include <chrono>

#include "far_field.h"
#include "internal.h"

namespace pk {
namespace {

template <typename T>
struct DevArr {
    T *p = nullptr;
    explicit DevArr(size_t n) { PK_CUDA(cudaMalloc(&p, (n ? n : 1) * sizeof(T))); }
    ~DevArr() { cudaFree(p); }
    DevArr(const DevArr &) = delete;
    DevArr &operator=(const DevArr &) = delete;
};

inline unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Matrix c = blockIdx.y (stride kn x kn): block (i, j) = scale K(sx g_i, o_c + sy g_j),
// o_c = (+-cy, +-cy, +-cy) by the bits of c (bit set: +cy); one thread per (i, j).
__global__ void k_kmat(int kernel, const double *__restrict__ g, int n, double sx, double sy, double cy,
                       double scale, double *__restrict__ M) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n), c = blockIdx.y, k = kernel == 0 ? 1 : 3;
    const double o[3] = {(c & 1) ? cy : -cy, (c & 2) ? cy : -cy, (c & 4) ? cy : -cy};
    double x[3], y[3], blk[9];
    for (int a = 0; a < 3; a++) {
        x[a] = sx * g[3 * i + a];
        y[a] = o[a] + sy * g[3 * j + a];
    }
    ff::kernel_block(kernel, x, y, blk);
    const size_t kn = (size_t)n * k;
    double *Mc = M + (size_t)c * kn * kn;
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++) Mc[(i * k + a) * kn + j * k + b] = scale * blk[a * k + b];
}

__global__ void k_transpose_eye(const double *__restrict__ A, int m, double *__restrict__ At,
                                double *__restrict__ Vt) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)m * m) return;
    const int i = (int)(t / m), j = (int)(t % m);
    At[(size_t)j * m + i] = A[t];
    Vt[t] = i == j ? 1.0 : 0.0;
}

constexpr int kJT = 256;

// sum over a block of NT threads; every thread gets the total (red: NT/32 doubles)
template <int NT = kJT>
__device__ inline double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0;
    for (int i = 0; i < NT / 32; i++) s += red[i];
    return s;
}

// ---- QR with column pivoting, A P = Q R (Householder), preconditioning the
// Jacobi SVD: one-sided Jacobi on R^T needs about a third of the sweeps that
// A itself needs (Drmac and Veselic's preconditioned Jacobi SVD).  W holds the
// columns of A as rows (W[j] = column j); reflector k is I - tau_k v_k v_k^T
// with v_k stored in hv[k] (zero above k).

// squared norms of the rows of W (columns of A)
__global__ void __launch_bounds__(kJT) k_row_norm2(const double *__restrict__ W, int m, double *__restrict__ c2) {
    __shared__ double red[kJT / 32];
    const double *a = W + (size_t)blockIdx.x * m;
    double v = 0;
    for (int i = threadIdx.x; i < m; i += kJT) v += a[i] * a[i];
    v = block_sum(v, red);
    if (threadIdx.x == 0) c2[blockIdx.x] = v;
}

constexpr int kQT = 1024;

// step k, one block: pivot = the column of largest trailing norm (ties: lowest
// index), swapped into place; its Householder reflector into hv[k], tau[k];
// column k of W becomes column k of R
__global__ void __launch_bounds__(kQT) k_qr_pivot(double *__restrict__ W, int m, int k, double *__restrict__ c2,
                                                  int *__restrict__ perm, double *__restrict__ hv,
                                                  double *__restrict__ tau) {
    __shared__ double bv[kQT / 32];
    __shared__ int bi[kQT / 32];
    __shared__ int jstar;
    __shared__ double red[kQT / 32];
    const int tid = threadIdx.x;
    double best = -1.0;
    int bj = m;
    for (int j = k + tid; j < m; j += kQT) {
        const double c = c2[j];
        if (c > best || (c == best && j < bj)) {
            best = c;
            bj = j;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oj = __shfl_down_sync(0xffffffffu, bj, o);
        if (ob > best || (ob == best && oj < bj)) {
            best = ob;
            bj = oj;
        }
    }
    if ((tid & 31) == 0) {
        bv[tid >> 5] = best;
        bi[tid >> 5] = bj;
    }
    __syncthreads();
    if (tid == 0) {
        double b = bv[0];
        int j = bi[0];
        for (int w = 1; w < kQT / 32; w++)
            if (bv[w] > b || (bv[w] == b && bi[w] < j)) {
                b = bv[w];
                j = bi[w];
            }
        jstar = j < m ? j : k;
    }
    __syncthreads();
    const int js = jstar;
    if (js != k) {
        double *a = W + (size_t)k * m, *b = W + (size_t)js * m;
        for (int i = tid; i < m; i += kQT) {
            const double t = a[i];
            a[i] = b[i];
            b[i] = t;
        }
        if (tid == 0) {
            const double t = c2[k];
            c2[k] = c2[js];
            c2[js] = t;
            const int q = perm[k];
            perm[k] = perm[js];
            perm[js] = q;
        }
    }
    __syncthreads();
    double *x = W + (size_t)k * m;
    double ss = 0;
    for (int i = k + tid; i < m; i += kQT) ss += x[i] * x[i];
    ss = block_sum<kQT>(ss, red);
    const double x0 = x[k], nrm = sqrt(ss);
    const double alpha = x0 >= 0 ? -nrm : nrm, v0 = x0 - alpha;
    const double vn2 = ss - x0 * x0 + v0 * v0;
    const double t = vn2 > 0 ? 2.0 / vn2 : 0.0;
    double *v = hv + (size_t)k * m;
    __syncthreads();  // every thread has read x[k]
    for (int i = tid; i < m; i += kQT) {
        if (i < k) {
            v[i] = 0.0;
        } else if (i == k) {
            v[i] = v0;
            x[i] = alpha;
        } else {
            v[i] = x[i];
            x[i] = 0.0;
        }
    }
    if (tid == 0) tau[k] = t;
}

// step k: reflector k applied to the trailing columns j > k (one block each),
// and their squared norms over rows > k for the next pivot
__global__ void __launch_bounds__(kJT) k_qr_apply(double *__restrict__ W, int m, int k, const double *__restrict__ hv,
                                                  const double *__restrict__ tau, double *__restrict__ c2) {
    __shared__ double red[kJT / 32];
    const int j = k + 1 + blockIdx.x;
    double *w = W + (size_t)j * m;
    const double *v = hv + (size_t)k * m;
    const double t = tau[k];
    double d = 0;
    for (int i = k + threadIdx.x; i < m; i += kJT) d += v[i] * w[i];
    d = block_sum(d, red) * t;
    double n2 = 0;
    for (int i = k + threadIdx.x; i < m; i += kJT) {
        const double y = w[i] - d * v[i];
        w[i] = y;
        if (i > k) n2 += y * y;
    }
    n2 = block_sum(n2, red);
    if (threadIdx.x == 0) c2[j] = n2;
}

// At = R (row i of R: W[j][i] for j >= i), Vt = I
__global__ void k_r_rows(const double *__restrict__ W, int m, double *__restrict__ At, double *__restrict__ Vt) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)m * m) return;
    const int i = (int)(t / m), j = (int)(t % m);
    At[t] = j >= i ? W[(size_t)j * m + i] : 0.0;
    Vt[t] = i == j ? 1.0 : 0.0;
}

// rows of Y (one block each) <- reflector k applied to them: y -= tau_k (v_k . y) v_k
__global__ void __launch_bounds__(kJT) k_apply_reflector(double *__restrict__ Y, int m, int k,
                                                         const double *__restrict__ hv,
                                                         const double *__restrict__ tau) {
    __shared__ double red[kJT / 32];
    const double t = tau[k];
    if (t == 0.0) return;
    double *y = Y + (size_t)blockIdx.x * m;
    const double *v = hv + (size_t)k * m;
    double d = 0;
    for (int i = k + threadIdx.x; i < m; i += kJT) d += v[i] * y[i];
    d = block_sum(d, red) * t;
    for (int i = k + threadIdx.x; i < m; i += kJT) y[i] -= d * v[i];
}

// One round of the circle method: block t rotates the pair of positions
// (t, mm - 1 - t).  Position 0 holds player 0; position i >= 1 holds player
// 1 + ((i - 1 - round) mod (mm - 1)).  Players >= m are byes.
__global__ void __launch_bounds__(kJT) k_jacobi_round(double *__restrict__ At, double *__restrict__ Vt, int m,
                                                      int mm, int round, double tol,
                                                      unsigned long long *__restrict__ rotations) {
    __shared__ double red[kJT / 32];
    const int t = blockIdx.x, r = mm - 1;
    auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (((pos - 1 - round) % r) + r) % r; };
    int p = player(t), q = player(mm - 1 - t);
    if (p >= m || q >= m) return;
    if (p > q) {
        const int x = p;
        p = q;
        q = x;
    }
    double *ap = At + (size_t)p * m, *aq = At + (size_t)q * m;
    double al = 0, be = 0, ga = 0;
    for (int i = threadIdx.x; i < m; i += kJT) {
        const double x = ap[i], y = aq[i];
        al += x * x;
        be += y * y;
        ga += x * y;
    }
    al = block_sum(al, red);
    be = block_sum(be, red);
    ga = block_sum(ga, red);
    if (ga == 0.0 || fabs(ga) <= tol * sqrt(al * be)) return;
    const double zeta = (be - al) / (2.0 * ga);
    const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    const double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
    for (int i = threadIdx.x; i < m; i += kJT) {
        const double x = ap[i], y = aq[i];
        ap[i] = c * x - s * y;
        aq[i] = s * x + c * y;
    }
    double *vp = Vt + (size_t)p * m, *vq = Vt + (size_t)q * m;
    for (int i = threadIdx.x; i < m; i += kJT) {
        const double x = vp[i], y = vq[i];
        vp[i] = c * x - s * y;
        vq[i] = s * x + c * y;
    }
    if (threadIdx.x == 0) atomicAdd(rotations, 1ull);
}

__global__ void __launch_bounds__(kJT) k_row_norms(const double *__restrict__ At, int m, double *__restrict__ sig) {
    __shared__ double red[kJT / 32];
    const double *a = At + (size_t)blockIdx.x * m;
    double v = 0;
    for (int i = threadIdx.x; i < m; i += kJT) v += a[i] * a[i];
    v = block_sum(v, red);
    if (threadIdx.x == 0) sig[blockIdx.x] = sqrt(v);
}

// rank of sig[j] in descending order, ties by index (a stable sort)
__global__ void k_rank(const double *__restrict__ sig, int m, int *__restrict__ rank) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double v = sig[j];
    int r = 0;
    for (int i = 0; i < m; i++) r += sig[i] > v || (sig[i] == v && i < j);
    rank[j] = r;
}

// A P = Q R, R^T = U_x S V_x^T (Jacobi on the rows of At = R, Vt = V_x^T, then
// Q applied to the rows of Vt):  A = (Q V_x) S (P U_x)^T, so
// U[:, rank_j] = (Q Vt[j])^T and V[perm[i]][rank_j] = At[j][i] / sig_j.
__global__ void k_extract_qr(const double *__restrict__ At, const double *__restrict__ QVt,
                             const double *__restrict__ sig, const int *__restrict__ rank,
                             const int *__restrict__ perm, int m, double *__restrict__ U, double *__restrict__ V,
                             double *__restrict__ S) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)m * m) return;
    const int j = (int)(t / m), i = (int)(t % m), jj = rank[j];
    const double inv = sig[j] > 0 ? 1.0 / sig[j] : 0.0;
    U[(size_t)i * m + jj] = QVt[t];
    V[(size_t)perm[i] * m + jj] = At[t] * inv;
    if (i == 0) S[jj] = sig[j];
}

// C = A B, row-major binary64, batched over blockIdx.z with element strides.
// 64 x 64 tiles, 16-deep K steps, 4 x 4 outputs per thread.
constexpr int kGT = 64, kGK = 16;
__global__ void __launch_bounds__(256) k_dgemm(int m, int n, int kk, const double *__restrict__ A, long long sA,
                                               const double *__restrict__ B, long long sB, double *__restrict__ C,
                                               long long sC) {
    __shared__ double As[kGK][kGT + 1];
    __shared__ double Bs[kGK][kGT];
    A += blockIdx.z * sA;
    B += blockIdx.z * sB;
    C += blockIdx.z * sC;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.y * kGT, col0 = blockIdx.x * kGT;
    double acc[4][4];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < kk; k0 += kGK) {
        for (int l = threadIdx.x; l < kGT * kGK; l += 256) {
            const int r = l / kGK, c = l % kGK, gr = row0 + r, gc = k0 + c;
            As[c][r] = (gr < m && gc < kk) ? A[(size_t)gr * kk + gc] : 0.0;
        }
        for (int l = threadIdx.x; l < kGT * kGK; l += 256) {
            const int r = l / kGT, c = l % kGT, gr = k0 + r, gc = col0 + c;
            Bs[r][c] = (gr < kk && gc < n) ? B[(size_t)gr * n + gc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kGK; k++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
            if (r < m && c < n) C[(size_t)r * n + c] = acc[i][j];
        }
}

void dgemm(int m, int n, int kk, const double *A, long long sA, const double *B, long long sB, double *C,
           long long sC, int batch, cudaStream_t s) {
    dim3 grid(nblocks(n, kGT), nblocks(m, kGT), batch);
    count_launch(), k_dgemm<<<grid, 256, 0, s>>>(m, n, kk, A, sA, B, sB, C, sC);
    PK_CUDA(cudaGetLastError());
}

// One thread per table entry, launched in 32-thread blocks so that the few
// hundred warps spread over all SMs (each runs a long binary64 Ewald sum).
__global__ void k_root_table(int kernel, unsigned periodic, int ell, int nimg, int p, int entries,
                             double *__restrict__ tab) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= entries) return;
    const int k = kernel == 0 ? 1 : 3;
    double acc[9];
    if (nimg >= 0) ff::finite_table_entry(kernel, periodic == 1 ? 0 : periodic == 2 ? 1 : 2, nimg, p, kInnerHalf, t, acc);
    else ff::root_table_entry(kernel, periodic, ell, p, kInnerHalf, t, acc);
    for (int i = 0; i < k * k; i++) tab[(size_t)t * k * k + i] = acc[i];
}

// Mr[(i k + a)][j k + b] = tab[lattice index of g_i - g_j][a][b]
__global__ void k_root_scatter(const double *__restrict__ tab, const double *__restrict__ g, int n, int p, int k,
                               double *__restrict__ Mr) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n), w = 2 * p - 1;
    int d[3];
    for (int a = 0; a < 3; a++) d[a] = (int)lround((g[3 * i + a] - g[3 * j + a]) * (p - 1) / 2.0) + (p - 1);
    const double *b = tab + (size_t)((d[0] * w + d[1]) * w + d[2]) * k * k;
    const size_t kn = (size_t)n * k;
    for (int a = 0; a < k; a++)
        for (int c = 0; c < k; c++) Mr[(i * k + a) * kn + j * k + c] = b[a * k + c];
}

template <typename T>
void to_host(std::vector<T> &h, const T *d, size_t n, cudaStream_t s) {
    h.resize(n);
    PK_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
}

// K_o for a batch of V-list offsets: out[b][i k + a][j k + c] = K_ac(0.525 g_i - (o_b + 0.525 g_j))
__global__ void k_m2l_batch(int kernel, const double *__restrict__ g, int n, const int *__restrict__ offs,
                            double *__restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    const int b = blockIdx.y, i = (int)(t / n), j = (int)(t % n), k = kernel == 0 ? 1 : 3;
    const int *o = offs + 3 * b;
    double r[3];
    for (int a = 0; a < 3; a++) r[a] = kInnerHalf * g[3 * i + a] - (o[a] + kInnerHalf * g[3 * j + a]);
    double blk[9];
    const double zero[3] = {0.0, 0.0, 0.0};
    ff::kernel_block(kernel, r, zero, blk);
    const size_t kn = (size_t)n * k;
    double *M = out + (size_t)b * kn * kn;
    for (int a = 0; a < k; a++)
        for (int c = 0; c < k; c++) M[(i * k + a) * kn + j * k + c] = blk[a * k + c];
}

// G += sum_b P[b] (len elements each)
__global__ void k_sum_batch(const double *__restrict__ P, int nb, long long len, double *__restrict__ G) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= len) return;
    double acc = G[t];
    for (int b = 0; b < nb; b++) acc += P[(size_t)b * len + t];
    G[t] = acc;
}

// A = U S V^T of a square m x m row-major device matrix (unchanged): QR with
// column pivoting, then one-sided Jacobi on R^T (see the header of this file);
// U, S, V copied back to the host (row-major, S descending).  Returns the
// number of Jacobi sweeps, counting the last one that rotated nothing.
int device_svd(const double *A, int m, cudaStream_t s, std::vector<double> &Uh, std::vector<double> &Sh,
               std::vector<double> &Vh) {
    const int kn = m, mm = kn + (kn & 1);
    const size_t kn2 = (size_t)kn * kn;
    DevArr<double> W(kn2), hv(kn2), tau(kn), c2(kn), At(kn2), Vt(kn2), U(kn2), V(kn2), S(kn), sig(kn);
    DevArr<int> rank(kn), perm(kn);
    DevArr<unsigned long long> rot(1);
    // W = A^T (columns of A as rows); Vt of the transpose kernel is scratch here
    count_launch(), k_transpose_eye<<<nblocks((long long)kn2, 256), 256, 0, s>>>(A, kn, W.p, Vt.p);
    std::vector<int> iota(kn);
    for (int i = 0; i < kn; i++) iota[i] = i;
    PK_CUDA(cudaMemcpyAsync(perm.p, iota.data(), sizeof(int) * kn, cudaMemcpyHostToDevice, s));
    count_launch(), k_row_norm2<<<kn, kJT, 0, s>>>(W.p, kn, c2.p);
    for (int k = 0; k < kn; k++) {
        count_launch(), k_qr_pivot<<<1, kQT, 0, s>>>(W.p, kn, k, c2.p, perm.p, hv.p, tau.p);
        if (kn - k - 1 > 0) count_launch(), k_qr_apply<<<kn - k - 1, kJT, 0, s>>>(W.p, kn, k, hv.p, tau.p, c2.p);
    }
    count_launch(), k_r_rows<<<nblocks((long long)kn2, 256), 256, 0, s>>>(W.p, kn, At.p, Vt.p);
    PK_CUDA(cudaGetLastError());
    unsigned long long hrot = 0;
    int sweeps = 0;
    for (int sweep = 0; sweep < 80; sweep++, sweeps++) {
        PK_CUDA(cudaMemsetAsync(rot.p, 0, sizeof(unsigned long long), s));
        for (int round = 0; round < mm - 1; round++)
            count_launch(), k_jacobi_round<<<mm / 2, kJT, 0, s>>>(At.p, Vt.p, kn, mm, round, 1e-15, rot.p);
        PK_CUDA(cudaGetLastError());
        PK_CUDA(cudaMemcpyAsync(&hrot, rot.p, sizeof hrot, cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        if (hrot == 0) break;
    }
    // Q V_x: reflectors applied in reverse order to the rows of Vt
    for (int k = kn - 1; k >= 0; k--) count_launch(), k_apply_reflector<<<kn, kJT, 0, s>>>(Vt.p, kn, k, hv.p, tau.p);
    count_launch(), k_row_norms<<<kn, kJT, 0, s>>>(At.p, kn, sig.p);
    count_launch(), k_rank<<<nblocks(kn, 256), 256, 0, s>>>(sig.p, kn, rank.p);
    count_launch(), k_extract_qr<<<nblocks((long long)kn2, 256), 256, 0, s>>>(At.p, Vt.p, sig.p, rank.p, perm.p, kn,
                                                                            U.p, V.p, S.p);
    PK_CUDA(cudaGetLastError());
    to_host(Uh, U.p, kn2, s);
    to_host(Vh, V.p, kn2, s);
    to_host(Sh, S.p, (size_t)kn, s);
    PK_CUDA(cudaStreamSynchronize(s));
    return sweeps + (hrot == 0 ? 1 : 0);
}

}  // namespace

void build_device_ops(HostOps &o, int kernel, int p, unsigned periodic, int ell, double eps_rel,
                      const std::string &cache_dir, double *phases, int nimg) {
    init_ops(o, kernel, p, periodic, ell, eps_rel, nimg);
    using clk = std::chrono::steady_clock;
    auto t_mark = clk::now();
    auto lap = [&](int i) {
        const auto t = clk::now();
        if (phases) phases[i] = std::chrono::duration<double>(t - t_mark).count();
        t_mark = t;
    };
    if (load_cached_ops(o, cache_dir)) {
        c2e_factors(o);
        return;
    }
    if (nimg >= 0) {  // validate the mask before any device work
        if (!(periodic == 1 || periodic == 2 || periodic == 4))
            throw Error(PKIFMM_ERR_UNSUPPORTED, "root operator: a finite array runs along one axis");
    } else if (periodic) {
        double probe[9], r0[3] = {0, 0, 0};
        if (!ff::far_kernel_block(kernel, periodic, ell, r0, probe))
            throw Error(PKIFMM_ERR_UNSUPPORTED, "root operator: periodicity not supported");
    }
    const int n = o.n, k = o.k, kn = o.kn;
    const size_t kn2 = (size_t)kn * kn;
    cudaStream_t s;
    PK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{s};
    DevArr<double> g(3 * (size_t)n);
    PK_CUDA(cudaMemcpyAsync(g.p, o.g.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    const long long nn = (long long)n * n;

    // ---- SVD of A_up1 = K(1.475 g, 0.525 g): QR with column pivoting, then
    // one-sided Jacobi on R^T ----
    {
        DevArr<double> A(kn2);
        count_launch(), k_kmat<<<dim3(nblocks(nn, 256), 1), 256, 0, s>>>(kernel, g.p, n, kOuterHalf, kInnerHalf, 0.0,
                                                                       1.0, A.p);
        PK_CUDA(cudaGetLastError());
        const int sweeps = device_svd(A.p, kn, s, o.U, o.S, o.V);
        if (phases) phases[3] = sweeps;
    }
    c2e_factors(o);
    lap(0);

    // ---- M2M and L2L for the 8 octants ----
    {
        DevArr<double> fa(kn2), fb(kn2), K(8 * kn2), tmp(8 * kn2), out(8 * kn2);
        // M2M: parent (edge 2) up-check at 2.95 g, child (edge 1) up-equiv at
        // +-0.5 + 0.525 g, times 2 (q~ = parent edge x q with child edge 1);
        // then (V S+) (U^T K)
        PK_CUDA(cudaMemcpyAsync(fa.p, o.uc2e_a.data(), sizeof(double) * kn2, cudaMemcpyHostToDevice, s));
        PK_CUDA(cudaMemcpyAsync(fb.p, o.uc2e_b.data(), sizeof(double) * kn2, cudaMemcpyHostToDevice, s));
        count_launch(), k_kmat<<<dim3(nblocks(nn, 256), 8), 256, 0, s>>>(kernel, g.p, n, 2.0 * kOuterHalf, kInnerHalf,
                                                                       0.5, 2.0, K.p);
        dgemm(kn, kn, kn, fb.p, 0, K.p, (long long)kn2, tmp.p, (long long)kn2, 8, s);
        dgemm(kn, kn, kn, fa.p, 0, tmp.p, (long long)kn2, out.p, (long long)kn2, 8, s);
        to_host(o.m2m, out.p, 8 * kn2, s);
        PK_CUDA(cudaStreamSynchronize(s));
        // L2L: child (edge 1) down-check at 0.525 g, parent (edge 2) down-equiv
        // at -(+-0.5) + 2.95 g; then (U S+) (V^T K)
        PK_CUDA(cudaMemcpyAsync(fa.p, o.dc2e_a.data(), sizeof(double) * kn2, cudaMemcpyHostToDevice, s));
        PK_CUDA(cudaMemcpyAsync(fb.p, o.dc2e_b.data(), sizeof(double) * kn2, cudaMemcpyHostToDevice, s));
        count_launch(), k_kmat<<<dim3(nblocks(nn, 256), 8), 256, 0, s>>>(kernel, g.p, n, kInnerHalf, 2.0 * kOuterHalf,
                                                                       -0.5, 1.0, K.p);
        dgemm(kn, kn, kn, fb.p, 0, K.p, (long long)kn2, tmp.p, (long long)kn2, 8, s);
        dgemm(kn, kn, kn, fa.p, 0, tmp.p, (long long)kn2, out.p, (long long)kn2, 8, s);
        to_host(o.l2l, out.p, 8 * kn2, s);
        PK_CUDA(cudaStreamSynchronize(s));
    }
    lap(1);

    // ---- root operator ----
    if (periodic) {
        const int w = 2 * p - 1, entries = w * w * w;
        DevArr<double> tab((size_t)entries * k * k), Mr(kn2);
        count_launch(), k_root_table<<<nblocks(entries, 32), 32, 0, s>>>(kernel, periodic, ell, nimg, p, entries,
                                                                         tab.p);
        count_launch(), k_root_scatter<<<nblocks(nn, 256), 256, 0, s>>>(tab.p, g.p, n, p, k, Mr.p);
        PK_CUDA(cudaGetLastError());
        to_host(o.root, Mr.p, kn2, s);
        PK_CUDA(cudaStreamSynchronize(s));
    } else {
        o.root.clear();
    }
    lap(2);
    save_cached_ops(o, cache_dir);
}


void matmul_device(int m, int n, int kk, const double *A, long long sA, const double *B, long long sB, double *C,
                   long long sC, int batch) {
    cudaStream_t s;
    PK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{s};
    const size_t na = (size_t)(batch - 1) * sA + (size_t)m * kk, nb = (size_t)(batch - 1) * sB + (size_t)kk * n,
                 nc = (size_t)(batch - 1) * sC + (size_t)m * n;
    DevArr<double> dA(na), dB(nb), dC(nc);
    PK_CUDA(cudaMemcpyAsync(dA.p, A, sizeof(double) * na, cudaMemcpyHostToDevice, s));
    PK_CUDA(cudaMemcpyAsync(dB.p, B, sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    dgemm(m, n, kk, dA.p, sA, dB.p, sB, dC.p, sC, batch, s);
    PK_CUDA(cudaMemcpyAsync(C, dC.p, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
}

void build_m2l_basis(int kernel, int p, double tau, int rank_override, M2LBasis &B) {
    const int n = surface_count(p), k = kernel == 0 ? 1 : 3, kn = n * k;
    const size_t kn2 = (size_t)kn * kn;
    // the V-list offsets in the enumeration of the M2L operator tables
    std::vector<int> offs, neg;
    for (int x = -3; x <= 3; x++)
        for (int y = -3; y <= 3; y++)
            for (int z = -3; z <= 3; z++) {
                if (std::max(std::abs(x), std::max(std::abs(y), std::abs(z))) <= 1) continue;
                offs.push_back(x);
                offs.push_back(y);
                offs.push_back(z);
            }
    const int nops = (int)offs.size() / 3;
    for (int a = 0; a < nops; a++)
        neg.insert(neg.end(), {-offs[3 * a], -offs[3 * a + 1], -offs[3 * a + 2]});
    cudaStream_t s;
    PK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{s};
    const std::vector<double> gh = surface_grid(p);
    DevArr<double> g(3 * (size_t)n);
    PK_CUDA(cudaMemcpyAsync(g.p, gh.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    DevArr<int> doffs(offs.size()), dneg(neg.size());
    PK_CUDA(cudaMemcpyAsync(doffs.p, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice, s));
    PK_CUDA(cudaMemcpyAsync(dneg.p, neg.data(), sizeof(int) * neg.size(), cudaMemcpyHostToDevice, s));
    const long long nn = (long long)n * n;
    constexpr int kBatch = 16;
    // G = sum_o K_o K_o^T = sum_o K_o K_{-o} (the kernel is even in r, so K_{-o} = K_o^T)
    DevArr<double> G(kn2), A(kBatch * kn2), Bm(kBatch * kn2), P(kBatch * kn2);
    PK_CUDA(cudaMemsetAsync(G.p, 0, sizeof(double) * kn2, s));
    for (int b0 = 0; b0 < nops; b0 += kBatch) {
        const int nb = std::min(kBatch, nops - b0);
        count_launch(), k_m2l_batch<<<dim3(nblocks(nn, 256), nb), 256, 0, s>>>(kernel, g.p, n, doffs.p + 3 * b0, A.p);
        count_launch(), k_m2l_batch<<<dim3(nblocks(nn, 256), nb), 256, 0, s>>>(kernel, g.p, n, dneg.p + 3 * b0, Bm.p);
        dgemm(kn, kn, kn, A.p, (long long)kn2, Bm.p, (long long)kn2, P.p, (long long)kn2, nb, s);
        count_launch(), k_sum_batch<<<nblocks((long long)kn2, 256), 256, 0, s>>>(P.p, nb, (long long)kn2, G.p);
    }
    PK_CUDA(cudaGetLastError());
    // G = U S U^T: the columns of U ordered by the singular values of the stacked operators
    std::vector<double> U, S, V;
    device_svd(G.p, kn, s, U, S, V);
    B.sig.assign(kn, 0.0);
    for (int j = 0; j < kn; j++) B.sig[j] = S[0] > 0 ? std::sqrt(std::max(S[j], 0.0) / S[0]) : 0.0;
    int r = 0;
    if (rank_override > 0) {
        r = std::min(rank_override, kn);
    } else {
        r = 64;
        while (r < kn && B.sig[r] > tau) r += 64;
        r = std::min(r, kn);
    }
    B.r = r;
    B.Ub.assign((size_t)kn * r, 0.0);
    for (int i = 0; i < kn; i++)
        for (int j = 0; j < r; j++) B.Ub[(size_t)i * r + j] = U[(size_t)i * kn + j];
    std::vector<double> Ubt((size_t)r * kn);
    for (int i = 0; i < kn; i++)
        for (int j = 0; j < r; j++) Ubt[(size_t)j * kn + i] = B.Ub[(size_t)i * r + j];
    // C_o = Ub^T K_o Ub
    DevArr<double> dUb((size_t)kn * r), dUbt((size_t)r * kn), T((size_t)kBatch * kn * r), C((size_t)kBatch * r * r);
    PK_CUDA(cudaMemcpyAsync(dUb.p, B.Ub.data(), sizeof(double) * kn * r, cudaMemcpyHostToDevice, s));
    PK_CUDA(cudaMemcpyAsync(dUbt.p, Ubt.data(), sizeof(double) * kn * r, cudaMemcpyHostToDevice, s));
    B.C.assign((size_t)nops * r * r, 0.f);
    std::vector<double> ch((size_t)kBatch * r * r);
    for (int b0 = 0; b0 < nops; b0 += kBatch) {
        const int nb = std::min(kBatch, nops - b0);
        count_launch(), k_m2l_batch<<<dim3(nblocks(nn, 256), nb), 256, 0, s>>>(kernel, g.p, n, doffs.p + 3 * b0, A.p);
        dgemm(kn, r, kn, A.p, (long long)kn2, dUb.p, 0, T.p, (long long)kn * r, nb, s);
        dgemm(r, r, kn, dUbt.p, 0, T.p, (long long)kn * r, C.p, (long long)r * r, nb, s);
        PK_CUDA(cudaMemcpyAsync(ch.data(), C.p, sizeof(double) * nb * r * r, cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        for (size_t i = 0; i < (size_t)nb * r * r; i++) B.C[(size_t)b0 * r * r + i] = (float)ch[i];
    }
}

}  // namespace pk
