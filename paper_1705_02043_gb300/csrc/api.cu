// C ABI of the periodic KIFMM library (declarations and contracts in
// include/pkifmm.h).  Orchestrates Algorithm 2: Stage 1 in
// pkifmm_plan_create, Stage 2 in pkifmm_evaluate.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include "internal.h"

using namespace pk;

struct pkifmm_plan_s {
    Plan P;
    int kernel_id = 0;                   // the public kernel (PKIFMM_*)
    pkifmm_plan_s *pressure = nullptr;   // PKIFMM_STOKES_PRESSURE: the Laplace plan with dipole sources
    pk::DBuf<double> cbuf;               // its scratch: velocities, pressures
    // doubly periodic in (x, z) or (y, z): the plans run the (x, y) case on
    // permuted coordinates, x'_a = x_{perm[a]} (the free axis last)
    int perm[3] = {0, 1, 2};
    bool permuted = false;
    pk::DBuf<double> pbuf;               // permuted points, densities and results
    int ks() const { return P.ks; }      // source density components
    int kt() const { return pressure ? 4 : P.kt; }
};

namespace pk {
void sort_points(Plan &P, const double *src, const double *dens, const double *trg, cudaStream_t s);
bool m2l_tc_device_supported();
}

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

template <typename F>
int guarded(F &&f) {
    try {
        return f();
    } catch (const Error &e) {
        return fail(e.code, e.what());
    } catch (const std::bad_alloc &) {
        return fail(PKIFMM_ERR_OOM, "host allocation failed");
    } catch (const std::exception &e) {
        std::string m = e.what();
        return fail(m.rfind("cache", 0) == 0 ? PKIFMM_ERR_CACHE : PKIFMM_ERR_INVALID_ARG, m);
    }
}

// corr [nprob][nrhs] (nullable); the problem of sorted target t is the prefix of its key
// Sorted-target results back to the caller's order, [nrhs][T][k], in box
// units: potentials scale as 1/L (K homogeneous of degree -1); mode 1 (the
// Laplace field): components 1..3, the gradient, as 1/L^2; mode 2 (Laplace
// dipole sources, the Stokes pressure): f.r/(4 pi r^3), degree -2, as
// 1/(4 pi L^2).  corr: the Laplace TP constant per (problem, vector), added to
// component 0 in the units of the sums.
__global__ void k_unpermute(const double *__restrict__ pot_s, const int *__restrict__ idx, long long T, int nrhs,
                            int k, int mode, double invL, const double *__restrict__ corr,
                            const unsigned long long *__restrict__ keyT, int key_shift, double *__restrict__ pot) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= T * nrhs * k) return;
    long long t = i / (nrhs * k);
    int rem = (int)(i % (nrhs * k)), r = rem / k, a = rem % k;
    double v = pot_s[i];
    if (corr && a == 0) v += corr[(long long)(keyT[t] >> key_shift) * nrhs + r];
    const double sc = mode == 2 ? invL * invL * 0.079577471545947668  // 1/(4 pi)
                      : (mode == 1 && a > 0) ? invL * invL : invL;
    pot[((long long)r * T + idx[t]) * k + a] = v * sc;
}

// velocity [nrhs][T][3] and pressure [nrhs][T] -> [nrhs][T][4] = (u, p)
__global__ void k_velocity_pressure(const double *__restrict__ vel, const double *__restrict__ pres, long long T,
                                    int nrhs, double *__restrict__ pot) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= T * nrhs) return;
    for (int a = 0; a < 3; a++) pot[i * 4 + a] = vel[i * 3 + a];
    pot[i * 4 + 3] = pres[i];
}

// Items of `stride` doubles: components off..off+2 are a vector, permuted
// out[off + a] = in[off + perm[a]] (forward) or out[off + perm[a]] = in[off + a]
// (inverse); the others are copied.  Rotating the frame by an axis permutation
// leaves the Laplace and Stokes kernels' form unchanged (both are isotropic).
__global__ void k_permute(const double *__restrict__ in, long long n, int stride, int off, int p0, int p1, int p2,
                          int inverse, double *__restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *a = in + i * stride;
    double *b = out + i * stride;
    for (int c = 0; c < stride; c++) b[c] = a[c];
    if (off < 0) return;
    const int pm[3] = {p0, p1, p2};
    for (int c = 0; c < 3; c++) {
        if (inverse) b[off + pm[c]] = a[off + c];
        else b[off + c] = a[off + pm[c]];
    }
}

// sums[2*(j*nk+c)] += phi, sums[2*(j*nk+c)+1] += |phi| per problem j (blockIdx.z,
// sorted sources soff[j]..soff[j+1]) and (rhs, component) c
__global__ void k_dens_sums(const double *__restrict__ dens, const long long *__restrict__ soff, int nk,
                            double *sums) {
    extern __shared__ double sh[];
    int c = blockIdx.y, j = blockIdx.z;
    double a = 0, b = 0;
    const long long s0 = soff[j], s1 = soff[j + 1];
    for (long long s = s0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; s < s1;
         s += (long long)gridDim.x * blockDim.x) {
        double v = dens[s * nk + c];
        a += v;
        b += fabs(v);
    }
    sh[threadIdx.x] = a;
    sh[blockDim.x + threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[threadIdx.x] += sh[threadIdx.x + o];
            sh[blockDim.x + threadIdx.x] += sh[blockDim.x + threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&sums[2 * ((long long)j * nk + c)], sh[0]);
        atomicAdd(&sums[2 * ((long long)j * nk + c) + 1], sh[blockDim.x]);
    }
}

// Laplace, triply periodic: the far-field kernel K^{P,F} of the Ewald
// (k = 0 removed) periodic sum is not harmonic in the source position: the
// neutralising background gives lap_y K^{P,F} = 4 pi / V inside the cell.
// Two charge sets with the same exterior field (the sources and the root's
// upward equivalent density) therefore receive far fields that differ by the
// constant (2 pi / 3V) (sum q |y - c|^2 - sum phi^u |y^u - c|^2).  That
// constant is restored here so the result is the zero-mean Ewald potential.
// m2[j*nrhs + r]: problem j (blockIdx.z), sorted sources soff[j]..soff[j+1]
// Dipole sources (ks = 3): the second moment of a dipole f at y is the limit
// of a charge pair, f.grad_y |y - c|^2 = 2 f.(y - c).
__global__ void k_second_moment_src(const double *__restrict__ xs, const double *__restrict__ dens,
                                    const long long *__restrict__ soff, int nrhs, int ks, double *__restrict__ m2) {
    int r = blockIdx.y, j = blockIdx.z;
    double acc = 0;
    for (long long i = soff[j] + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < soff[j + 1];
         i += (long long)gridDim.x * blockDim.x) {
        double dx = xs[3 * i] - 0.5, dy = xs[3 * i + 1] - 0.5, dz = xs[3 * i + 2] - 0.5;
        if (ks == 3) {
            const double *f = dens + (i * nrhs + r) * 3;
            acc += 2.0 * (f[0] * dx + f[1] * dy + f[2] * dz);
        } else {
            acc += dens[i * nrhs + r] * (dx * dx + dy * dy + dz * dz);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&m2[(long long)j * nrhs + r], acc);
}

// roots are boxes 0..nprob-1: block r = j * nrhs + rhs reads row r; writes m2[rows + r]
template <typename T>
__global__ void k_second_moment_root(const T *__restrict__ up, const double *__restrict__ g, int n, int rows,
                                     double *__restrict__ m2) {
    int r = blockIdx.x;
    double acc = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double g2 = g[3 * j] * g[3 * j] + g[3 * j + 1] * g[3 * j + 1] + g[3 * j + 2] * g[3 * j + 2];
        acc += (double)up[(long long)r * n + j] * 0.525 * 0.525 * g2;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&m2[rows + r], acc);
}

__global__ void k_moment_finish(const double *m2, int rows, double *corr) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) corr[r] = 2.0 * 3.14159265358979323846 / 3.0 * (m2[r] - m2[rows + r]);
}

const double *laplace_tp_constant(Plan &P, cudaStream_t s) {
    if (P.kernel != PKIFMM_LAPLACE || P.periodic != 7) return nullptr;
    const int nr = P.nrhs, rows = P.nprob * nr;
    P.sums.reserve(3 * (size_t)rows + 4);
    double *m2 = P.sums.p, *corr = P.sums.p + 2 * rows;
    PK_CUDA(cudaMemsetAsync(m2, 0, sizeof(double) * 2 * rows, s));
    dim3 grid((unsigned)std::min<long long>(64, (P.S / P.nprob + 255) / 256 + 1), nr, P.nprob);
    count_launch(), k_second_moment_src<<<grid, 256, 0, s>>>(P.xs.p, P.dens_s.p, P.soff.p, nr, P.ks, m2);
    if (P.precision == PKIFMM_FP64)
        count_launch(), k_second_moment_root<double><<<rows, 256, 0, s>>>(P.up64.p, P.g64.p, P.n, rows, m2);
    else
        count_launch(), k_second_moment_root<float><<<rows, 256, 0, s>>>(P.up32.p, P.g64.p, P.n, rows, m2);
    count_launch(), k_moment_finish<<<(rows + 255) / 256, 256, 0, s>>>(m2, rows, corr);
    return corr;
}

bool needs_neutral(const Plan &P) {
    if (!P.periodic || P.nimg >= 0) return false;  // free space and finite arrays: finite sums
    if (P.kernel == PKIFMM_LAPLACE) return true;
    return P.periodic != 7;  // Stokes SP/DP: zero net force; TP allows a net force
}

void record(Plan &P, int i, cudaStream_t s) {
    if (P.events) PK_CUDA(cudaEventRecord(P.ev[i], s));
}

// nprob independent problems: problem j owns sources soff[j]..soff[j+1] and
// targets toff[j]..toff[j+1] (host CSR arrays of nprob+1 entries).
int evaluate_impl(Plan &P, int nprob, const int64_t *soff, const int64_t *toff, const double *src,
                  const double *dens, const double *trg, double *pot, cudaStream_t s) {
    if (nprob < 1 || !soff || !toff) return fail(PKIFMM_ERR_INVALID_ARG, "nprob < 1 or NULL offsets");
    int pbits = 0;
    while ((1LL << pbits) < nprob) pbits++;
    if (3 * P.depth_max + pbits > 63) return fail(PKIFMM_ERR_INVALID_ARG, "too many problems for depth_max");
    if (soff[0] != 0 || toff[0] != 0) return fail(PKIFMM_ERR_INVALID_ARG, "offsets must start at 0");
    for (int j = 0; j < nprob; j++)
        if (soff[j + 1] < soff[j] || toff[j + 1] < toff[j])
            return fail(PKIFMM_ERR_INVALID_ARG, "offsets must be non-decreasing");
    const int64_t S = soff[nprob], T = toff[nprob];
    if (S > (1LL << 30) || T > (1LL << 30)) return fail(PKIFMM_ERR_INVALID_ARG, "S, T out of range");
    if ((S && (!src || !dens)) || (T && (!trg || !pot))) return fail(PKIFMM_ERR_INVALID_ARG, "NULL array");
    PK_CUDA(cudaSetDevice(P.device));
    P.S = S;
    P.T = T;
    P.nprob = nprob;
    std::fill(P.stage_ms, P.stage_ms + 9, 0.0);
    if (T == 0) return PKIFMM_OK;
    if (S == 0) {
        PK_CUDA(cudaMemsetAsync(pot, 0, sizeof(double) * T * P.nrhs * P.kt, s));
        return PKIFMM_OK;
    }
    record(P, 0, s);
    {
        std::vector<long long> h(2 * (size_t)(nprob + 1));
        P.same_offsets = true;
        for (int j = 0; j <= nprob; j++) {
            h[j] = soff[j];
            h[nprob + 1 + j] = toff[j];
            P.same_offsets &= soff[j] == toff[j];
        }
        P.soff.reserve(nprob + 1);
        P.toff.reserve(nprob + 1);
        PK_CUDA(cudaMemcpyAsync(P.soff.p, h.data(), sizeof(long long) * (nprob + 1), cudaMemcpyHostToDevice, s));
        PK_CUDA(cudaMemcpyAsync(P.toff.p, h.data() + nprob + 1, sizeof(long long) * (nprob + 1),
                                cudaMemcpyHostToDevice, s));
        PK_CUDA(cudaStreamSynchronize(s));  // h goes out of scope
    }
    sort_points(P, src, dens, trg, s);
    int err[4] = {0, 0, 0, 0};
    PK_CUDA(cudaMemcpyAsync(err, P.err.p, sizeof err, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    if (err[0]) return fail(PKIFMM_ERR_INVALID_ARG, "non-finite coordinate");
    if (err[1]) return fail(PKIFMM_ERR_OUT_OF_BOX, "point outside the box along a free axis");
    if (needs_neutral(P)) {
        const int nk = P.nrhs * P.ks;
        const size_t nsum = 2 * (size_t)nk * nprob;
        P.sums.reserve(nsum);
        PK_CUDA(cudaMemsetAsync(P.sums.p, 0, sizeof(double) * nsum, s));
        dim3 grid((unsigned)std::min<long long>(nprob > 1 ? 64 : 1024, (S / nprob + 255) / 256 + 1), nk, nprob);
        count_launch(), k_dens_sums<<<grid, 256, 2 * 256 * sizeof(double), s>>>(P.dens_s.p, P.soff.p, nk, P.sums.p);
        std::vector<double> h(nsum);
        PK_CUDA(cudaMemcpyAsync(h.data(), P.sums.p, sizeof(double) * nsum, cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        for (size_t c = 0; c < nsum / 2; c++)
            if (std::fabs(h[2 * c]) > 1e-12 * h[2 * c + 1])
                return fail(PKIFMM_ERR_NOT_NEUTRAL, "densities violate the compatibility condition (net charge / force)");
    }
    record(P, 1, s);
    build_tree(P, s);
    build_lists(P, s);
    build_tasks(P, s);
    record(P, 2, s);
    run_upward(P, s);
    record(P, 3, s);
    run_root(P, s);
    record(P, 4, s);
    run_m2l(P, s);
    record(P, 5, s);
    run_downward(P, s);
    record(P, 6, s);
    run_leaves(P, s);
    long long n = T * P.nrhs * P.kt;
    const double *corr = laplace_tp_constant(P, s);
    const int mode = P.kt == 4 ? 1 : P.ks == 3 && P.k == 1 ? 2 : 0;
    count_launch(), k_unpermute<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        P.pot_s.p, P.idxT.p, T, P.nrhs, P.kt, mode, 1.0 / P.L, corr, P.keyT.p, 3 * P.depth_max, pot);
    record(P, 7, s);
    PK_CUDA(cudaGetLastError());
    return PKIFMM_OK;
}

// Any plan: the Stokes velocity-pressure plan runs the velocity evaluation,
// then the pressure as the Laplace potential of dipoles f at the sources
// (p = sum f.r/(4 pi r^3)), and interleaves them; the others evaluate directly.
int evaluate_plain(pkifmm_plan_s *h, int nprob, const int64_t *soff, const int64_t *toff, const double *src,
                   const double *dens, const double *trg, double *pot, cudaStream_t s);

// Doubly periodic in (x, z) or (y, z): points, vector densities and vector
// results are carried into the frame where the free axis is z, evaluated
// there, and the results carried back.
int evaluate_any(pkifmm_plan_s *h, int nprob, const int64_t *soff, const int64_t *toff, const double *src,
                 const double *dens, const double *trg, double *pot, cudaStream_t s) {
    if (!h->permuted) return evaluate_plain(h, nprob, soff, toff, src, dens, trg, pot, s);
    if (nprob < 1 || !soff || !toff) return fail(PKIFMM_ERR_INVALID_ARG, "nprob < 1 or NULL offsets");
    const int64_t S = soff[nprob], T = toff[nprob];
    if (S < 0 || T < 0 || S > (1LL << 30) || T > (1LL << 30)) return fail(PKIFMM_ERR_INVALID_ARG, "S, T out of range");
    if ((S && (!src || !dens)) || (T && (!trg || !pot))) return fail(PKIFMM_ERR_INVALID_ARG, "NULL array");
    Plan &P = h->P;
    PK_CUDA(cudaSetDevice(P.device));
    const int nr = P.nrhs, ks = h->ks(), kt = h->kt();
    const size_t ns = 3 * (size_t)S, nd = (size_t)nr * S * ks, nt = 3 * (size_t)T, np = (size_t)nr * T * kt;
    h->pbuf.reserve(ns + nd + nt + np + 8);
    double *ps = h->pbuf.p, *pd = ps + ns, *pt = pd + nd, *pp = pt + nt;
    const int *m = h->perm;
    auto launch = [&](const double *in, long long n, int stride, int off, int inv, double *out) {
        if (n > 0)
            count_launch(), k_permute<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, n, stride, off, m[0], m[1], m[2],
                                                                                 inv, out);
    };
    launch(src, S, 3, 0, 0, ps);
    launch(dens, (long long)nr * S, ks, ks == 3 ? 0 : -1, 0, pd);
    launch(trg, T, 3, 0, 0, pt);
    PK_CUDA(cudaGetLastError());
    // targets that are the sources stay the sources (one sort)
    int rc = evaluate_plain(h, nprob, soff, toff, ps, pd, trg == src ? ps : pt, pp, s);
    if (rc != PKIFMM_OK) return rc;
    // vector part of the results: velocity (k_t 3, or 0..2 of the pressure kernel),
    // the gradient of the Laplace field (1..3)
    const int off = kt == 3 ? 0 : (kt == 4 && h->kernel_id == PKIFMM_LAPLACE_FIELD) ? 1 : kt == 4 ? 0 : -1;
    launch(pp, (long long)nr * T, kt, off, 1, pot);
    PK_CUDA(cudaGetLastError());
    return PKIFMM_OK;
}

int evaluate_plain(pkifmm_plan_s *h, int nprob, const int64_t *soff, const int64_t *toff, const double *src,
                   const double *dens, const double *trg, double *pot, cudaStream_t s) {
    if (!h->pressure) return evaluate_impl(h->P, nprob, soff, toff, src, dens, trg, pot, s);
    if (nprob < 1 || !soff || !toff) return fail(PKIFMM_ERR_INVALID_ARG, "nprob < 1 or NULL offsets");
    Plan &P = h->P;
    const int nr = P.nrhs;
    const int64_t S = soff[nprob], T = toff[nprob];
    if (S < 0 || T < 0 || S > (1LL << 30) || T > (1LL << 30)) return fail(PKIFMM_ERR_INVALID_ARG, "S, T out of range");
    PK_CUDA(cudaSetDevice(P.device));
    const size_t nv = (size_t)nr * T * 3, np = (size_t)nr * T;
    h->cbuf.reserve(nv + np + 8);
    double *vel = h->cbuf.p, *pres = vel + nv;
    int rc = evaluate_impl(P, nprob, soff, toff, src, dens, trg, vel, s);
    if (rc != PKIFMM_OK) return rc;
    rc = evaluate_impl(h->pressure->P, nprob, soff, toff, src, dens, trg, pres, s);
    if (rc != PKIFMM_OK) return rc;
    if (T > 0)
        count_launch(), k_velocity_pressure<<<(unsigned)((nr * T + 255) / 256), 256, 0, s>>>(vel, pres, T, nr, pot);
    PK_CUDA(cudaGetLastError());
    return PKIFMM_OK;
}

}  // namespace

namespace pk {
int set_last_error(int code, const std::string &msg) { return fail(code, msg); }
}  // namespace pk

extern "C" {

static void destroy_plan(pkifmm_plan_s *plan) {
    if (!plan) return;
    destroy_plan(plan->pressure);
    plan->pressure = nullptr;
    plan->cbuf.release();
    plan->pbuf.release();
    Plan &P = plan->P;
    cudaSetDevice(P.device);
    cudaDeviceSynchronize();
    m2l_tc_release(P);
    trans_tc_release(P);
    for (auto &e : P.ev)
        if (P.events && e) cudaEventDestroy(e);
    DBuf<double> *d64[] = {&P.g64, &P.uc2e_a, &P.uc2e_b, &P.dc2e_a, &P.dc2e_b, &P.m2m, &P.l2l, &P.m2l, &P.root,
                           &P.xs, &P.xt, &P.dens_s, &P.pot_s, &P.ysrel64, &P.xtrel64, &P.sums, &P.up64, &P.chk64,
                           &P.dn64, &P.tmp64};
    for (auto *b : d64) b->release();
    DBuf<float> *d32[] = {&P.g32, &P.uc2e_a32, &P.uc2e_b32, &P.dc2e_a32, &P.dc2e_b32, &P.m2m32, &P.l2l32, &P.m2l32,
                          &P.ysrel32, &P.xtrel32, &P.dens32, &P.pot32, &P.up32, &P.chk32, &P.dn32, &P.tmp32,
                          &P.uphat32, &P.chkhat32};
    for (auto *b : d32) b->release();
    DBuf<int> *di[] = {&P.class_slot_op, &P.idxS, &P.idxT, &P.idxS2, &P.idxT2, &P.hist, &P.err, &P.cnt, &P.off,
                       &P.gather_idx, &P.leaves_src, &P.leaves_trg, &P.xboxes, &P.tree.parent, &P.tree.child,
                       &P.tree.lvl_begin_d, &P.tree.u_ptr, &P.tree.u_box, &P.tree.w_ptr, &P.tree.w_box,
                       &P.tree.x_ptr, &P.tree.x_box, &P.tree.v_slot};
    for (auto *b : di) b->release();
    P.keyS.release();
    P.keyT.release();
    P.keyS2.release();
    P.keyT2.release();
    P.tree.key.release();
    P.tree.bpos.release();
    P.tree.srange.release();
    P.tree.trange.release();
    P.tree.u_sh.release();
    P.tree.w_sh.release();
    P.tree.x_sh.release();
    P.slot_of.release();
    P.csr.release();
    P.xn.release();
    P.lcnt.release();
    P.scan_tmp.release();
    P.lpairs.release();
    P.ctr.release();
    P.soff.release();
    P.toff.release();
    P.far64.release();
    if (P.stage_h) cudaFreeHost(P.stage_h);
    if (P.down_h) cudaFreeHost(P.down_h);
    if (P.stage_ev) cudaEventDestroy(P.stage_ev);
    Task *ts[] = {&P.t_uc2e, &P.t_m2l, &P.t_dc2e, &P.t_root, &P.t_dcx};
    for (auto *t : ts) {
        t->boxes.release();
        t->tiles.release();
        t->class_ops.release();
    }
    for (auto *v : {&P.t_m2m, &P.t_l2l})
        for (auto &t : *v) {
            t.boxes.release();
            t.tiles.release();
            t.class_ops.release();
        }
    delete plan;
}

// One plan of an internal kernel (0 Laplace, 1 Stokes) with kt target components.
static pkifmm_plan_s *make_plan(int kernel, int kt, unsigned periodic_axes, const double box_lo[3], double box_len,
                                int p, int ell, int leaf_max, int depth_max, int precision, int nrhs,
                                const char *cache_dir, bool host_stage1, int ks = 0, int nimg = -1) {
    auto *h = new pkifmm_plan_s;
    Plan &P = h->P;
    P.kernel = kernel;
    P.k = kernel == 0 ? 1 : 3;
    P.kt = kt;
    P.ks = ks ? ks : P.k;
    P.nimg = nimg;
    P.p = p;
    P.n = surface_count(p);
    P.kn = P.n * P.k;
    P.ell = ell;
    P.leaf_max = leaf_max;
    P.depth_max = depth_max;
    P.precision = precision;
    P.nrhs = nrhs;
    P.periodic = periodic_axes;
    for (int a = 0; a < 3; a++) P.lo[a] = box_lo[a];
    P.L = box_len;
    try {
        PK_CUDA(cudaGetDevice(&P.device));
        // singular values <= eps * s_max are dropped (svd_cut: by kernel, p and precision)
        const double eps = svd_cut(kernel, p, precision == PKIFMM_FP64 ? 0 : 1, P.kn);
        if (host_stage1) build_host_ops(P.host, kernel, p, periodic_axes, ell, eps, cache_dir ? cache_dir : "", nimg);
        else build_device_ops(P.host, kernel, p, periodic_axes, ell, eps, cache_dir ? cache_dir : "", nullptr, nimg);
        upload_operators(P);
        for (auto &e : P.ev) PK_CUDA(cudaEventCreate(&e));
        P.events = true;
    } catch (...) {
        destroy_plan(h);
        throw;
    }
    return h;
}

// nimg >= 0: a finite array of cells along the single periodic axis
static int create_impl(pkifmm_plan *out, int kernel, unsigned periodic_axes, int nimg, const double box_lo[3],
                       double box_len, int p, int ell, int leaf_max, int depth_max, int precision, int nrhs,
                       const char *cache_dir) {
    if (!out) return fail(PKIFMM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    const bool host_stage1 = (precision & PKIFMM_PRECOMPUTE_HOST) != 0;
    precision &= ~PKIFMM_PRECOMPUTE_HOST;
    if (kernel < PKIFMM_LAPLACE || kernel > PKIFMM_STOKES_PRESSURE) return fail(PKIFMM_ERR_INVALID_ARG, "kernel");
    if (periodic_axes > 7) return fail(PKIFMM_ERR_INVALID_ARG, "periodic_axes");
    if (!box_lo || !(box_len > 0) || !std::isfinite(box_len)) return fail(PKIFMM_ERR_INVALID_ARG, "box");
    if (p < 4 || p > 16 || ell < 1 || ell > 8 || leaf_max < 1 || depth_max < 1 || depth_max > kMaxLevel - 1 ||
        nrhs < 1 || nrhs > 64 || (precision != PKIFMM_FP64 && precision != PKIFMM_MIXED))
        return fail(PKIFMM_ERR_INVALID_ARG, "p / ell / leaf_max / depth_max / nrhs / precision out of range");
    // doubly periodic in (x, z) or (y, z): the (x, y) plans in a permuted frame
    int perm[3] = {0, 1, 2};
    const bool permuted = periodic_axes == 5 || periodic_axes == 6;
    if (periodic_axes == 5) {  // x' = x, y' = z, z' = y
        perm[1] = 2;
        perm[2] = 1;
    } else if (periodic_axes == 6) {  // x' = y, y' = z, z' = x
        perm[0] = 1;
        perm[1] = 2;
        perm[2] = 0;
    }
    double lo_p[3] = {0, 0, 0};
    if (box_lo)
        for (int a = 0; a < 3; a++) lo_p[a] = box_lo[perm[a]];
    if (permuted) {
        periodic_axes = 3;
        if (nimg >= 0) return fail(PKIFMM_ERR_INVALID_ARG, "finite arrays run along one axis");
    }
    if (box_lo) box_lo = lo_p;
    return guarded([&]() {
        const int internal = (kernel == PKIFMM_LAPLACE || kernel == PKIFMM_LAPLACE_FIELD) ? 0 : 1;
        const int kt = kernel == PKIFMM_LAPLACE ? 1 : kernel == PKIFMM_LAPLACE_FIELD ? 4 : 3;
        pkifmm_plan_s *h = make_plan(internal, kt, periodic_axes, box_lo, box_len, p, ell, leaf_max, depth_max,
                                     precision, nrhs, cache_dir, host_stage1, 0, nimg);
        h->kernel_id = kernel;
        h->permuted = permuted;
        for (int a = 0; a < 3; a++) h->perm[a] = perm[a];
        if (kernel == PKIFMM_STOKES_PRESSURE) {
            try {
                // the pressure: Laplace translations, dipole sources (the forces), one value per target
                h->pressure = make_plan(0, 1, periodic_axes, box_lo, box_len, p, ell, leaf_max, depth_max, precision,
                                        nrhs, cache_dir, host_stage1, 3, nimg);
                h->pressure->kernel_id = -1;
            } catch (...) {
                destroy_plan(h);
                throw;
            }
        }
        *out = h;
        return PKIFMM_OK;
    });
}

int pkifmm_plan_create(pkifmm_plan *out, int kernel, unsigned periodic_axes, const double box_lo[3],
                       double box_len, int p, int ell, int leaf_max, int depth_max, int precision, int nrhs,
                       const char *cache_dir) {
    return create_impl(out, kernel, periodic_axes, -1, box_lo, box_len, p, ell, leaf_max, depth_max, precision, nrhs,
                       cache_dir);
}

int pkifmm_plan_create_finite(pkifmm_plan *out, int kernel, int axis, int nimg, const double box_lo[3],
                              double box_len, int p, int ell, int leaf_max, int depth_max, int precision, int nrhs,
                              const char *cache_dir) {
    if (axis < 0 || axis > 2 || nimg < 1 || nimg > (1 << 20)) {
        if (out) *out = nullptr;
        return fail(PKIFMM_ERR_INVALID_ARG, "axis must be 0..2 and the image count 1..2^20");
    }
    return create_impl(out, kernel, 1u << axis, nimg, box_lo, box_len, p, ell, leaf_max, depth_max, precision, nrhs,
                       cache_dir);
}

int pkifmm_evaluate(pkifmm_plan plan, int64_t S, const double *src_xyz, const double *dens, int64_t T,
                    const double *trg_xyz, double *pot, void *cuda_stream) {
    if (!plan) return fail(PKIFMM_ERR_INVALID_ARG, "plan is NULL");
    return guarded([&]() {
        if (S < 0 || T < 0) return fail(PKIFMM_ERR_INVALID_ARG, "S, T out of range");
        int64_t so[2] = {0, S}, to[2] = {0, T};
        return evaluate_any(plan, 1, so, to, src_xyz, dens, trg_xyz, pot, (cudaStream_t)cuda_stream);
    });
}

int pkifmm_evaluate_batched(pkifmm_plan plan, int nprob, const int64_t *src_off, const int64_t *trg_off,
                            const double *src_xyz, const double *dens, const double *trg_xyz, double *pot,
                            void *cuda_stream) {
    if (!plan) return fail(PKIFMM_ERR_INVALID_ARG, "plan is NULL");
    return guarded([&]() {
        return evaluate_any(plan, nprob, src_off, trg_off, src_xyz, dens, trg_xyz, pot, (cudaStream_t)cuda_stream);
    });
}

int pkifmm_evaluate_host(pkifmm_plan plan, int64_t S, const double *src_xyz, const double *dens, int64_t T,
                         const double *trg_xyz, double *pot, void *cuda_stream) {
    if (!plan) return fail(PKIFMM_ERR_INVALID_ARG, "plan is NULL");
    return guarded([&]() {
        Plan &P = plan->P;
        cudaStream_t s = (cudaStream_t)cuda_stream;
        if (S < 0 || T < 0 || S > (1LL << 30) || T > (1LL << 30)) return fail(PKIFMM_ERR_INVALID_ARG, "S, T out of range");
        PK_CUDA(cudaSetDevice(P.device));
        size_t bs = sizeof(double) * 3 * S, bd = sizeof(double) * S * P.nrhs * plan->ks();
        size_t bt = sizeof(double) * 3 * T, bp = sizeof(double) * T * P.nrhs * plan->kt();
        DBuf<char> buf;
        buf.reserve(bs + bd + bt + bp + 64);
        double *ds = (double *)buf.p, *dd = (double *)(buf.p + bs), *dt = (double *)(buf.p + bs + bd),
               *dp = (double *)(buf.p + bs + bd + bt);
        if (S) {
            PK_CUDA(cudaMemcpyAsync(ds, src_xyz, bs, cudaMemcpyHostToDevice, s));
            PK_CUDA(cudaMemcpyAsync(dd, dens, bd, cudaMemcpyHostToDevice, s));
        }
        if (T) PK_CUDA(cudaMemcpyAsync(dt, trg_xyz, bt, cudaMemcpyHostToDevice, s));
        if (S < 0 || T < 0) return fail(PKIFMM_ERR_INVALID_ARG, "S, T out of range");
        int64_t so[2] = {0, S}, to[2] = {0, T};
        int rc = evaluate_any(plan, 1, so, to, ds, dd, dt, dp, s);
        if (rc == PKIFMM_OK && T) PK_CUDA(cudaMemcpyAsync(pot, dp, bp, cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        buf.release();
        return rc;
    });
}

int pkifmm_last_stage_times(pkifmm_plan plan, double *ms, int max) {
    if (!plan || !ms || max < 0) return fail(PKIFMM_ERR_INVALID_ARG, "bad argument");
    return guarded([&]() {
        double tot[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        // the velocity-pressure kernel: both evaluations, stage by stage
        for (pkifmm_plan_s *h = plan; h; h = h->pressure) {
            Plan &P = h->P;
            if (P.events && P.T > 0 && P.S > 0) {
                PK_CUDA(cudaEventSynchronize(P.ev[7]));
                for (int i = 0; i < 7; i++) {
                    float t = 0;
                    PK_CUDA(cudaEventElapsedTime(&t, P.ev[i], P.ev[i + 1]));
                    P.stage_ms[i] = t;
                }
                float t = 0;
                PK_CUDA(cudaEventElapsedTime(&t, P.ev[0], P.ev[7]));
                P.stage_ms[7] = t;
            }
            P.stage_ms[8] = m2l_tc_last_ms(P);
            for (int i = 0; i < 9; i++) tot[i] += P.stage_ms[i];
        }
        int m = std::min(max, 9);
        for (int i = 0; i < m; i++) ms[i] = tot[i];
        return m;
    });
}

int pkifmm_autotune_leaf(pkifmm_plan plan, int nprob, const int64_t *src_off, const int64_t *trg_off,
                         const double *src_xyz, const double *dens, const double *trg_xyz, double *pot,
                         const int *candidates, int ncand, int reps, int *best_out, double *ms_out,
                         void *cuda_stream) {
    if (!plan || !candidates || ncand < 1 || reps < 1 || !best_out)
        return fail(PKIFMM_ERR_INVALID_ARG, "bad argument");
    for (int c = 0; c < ncand; c++)
        if (candidates[c] < 1) return fail(PKIFMM_ERR_INVALID_ARG, "leaf size < 1");
    return guarded([&]() {
        Plan &P = plan->P;
        cudaStream_t s = (cudaStream_t)cuda_stream;
        const int keep = P.leaf_max;
        auto set_leaf = [&](int v) {
            for (pkifmm_plan_s *h = plan; h; h = h->pressure) h->P.leaf_max = v;
        };
        int best = keep;
        double best_ms = 1e300;
        for (int c = 0; c < ncand; c++) {
            set_leaf(candidates[c]);
            int rc = evaluate_any(plan, nprob, src_off, trg_off, src_xyz, dens, trg_xyz, pot, s);  // warm-up
            if (rc != PKIFMM_OK) {
                set_leaf(keep);
                return rc;
            }
            PK_CUDA(cudaStreamSynchronize(s));
            double t_min = 1e300;
            for (int r = 0; r < reps; r++) {
                auto t0 = std::chrono::steady_clock::now();
                rc = evaluate_any(plan, nprob, src_off, trg_off, src_xyz, dens, trg_xyz, pot, s);
                PK_CUDA(cudaStreamSynchronize(s));
                auto t1 = std::chrono::steady_clock::now();
                if (rc != PKIFMM_OK) {
                    set_leaf(keep);
                    return rc;
                }
                t_min = std::min(t_min, std::chrono::duration<double, std::milli>(t1 - t0).count());
            }
            if (ms_out) ms_out[c] = t_min;
            if (t_min < best_ms) {
                best_ms = t_min;
                best = candidates[c];
            }
        }
        set_leaf(best);
        *best_out = best;
        return (int)PKIFMM_OK;
    });
}

int pkifmm_plan_set_far_field(pkifmm_plan plan, int mode) {
    if (!plan || (mode != PKIFMM_FAR_L2L && mode != PKIFMM_FAR_DIRECT)) return fail(PKIFMM_ERR_INVALID_ARG, "bad argument");
    for (pkifmm_plan_s *h = plan; h; h = h->pressure) h->P.far_direct = mode == PKIFMM_FAR_DIRECT;
    return PKIFMM_OK;
}

int pkifmm_tree_stats(pkifmm_plan plan, int64_t *out, int max) {
    if (!plan || !out || max < 0) return fail(PKIFMM_ERR_INVALID_ARG, "bad argument");
    Tree &t = plan->P.tree;
    int64_t v[8] = {t.nbox, t.nleaf, t.depth, t.nU, t.nV, t.nW, t.nX, t.p2p_pairs};
    int m = std::min(max, 8);
    for (int i = 0; i < m; i++) out[i] = v[i];
    return m;
}

int pkifmm_tree_export(pkifmm_plan plan, int32_t *level, int32_t *pos, int32_t *parent, int64_t *src_range,
                       int64_t *trg_range, int64_t *src_perm, int64_t *trg_perm) {
    if (!plan) return fail(PKIFMM_ERR_INVALID_ARG, "plan is NULL");
    return guarded([&]() {
        Plan &P = plan->P;
        Tree &t = P.tree;
        int nb = t.nbox;
        std::vector<int4> bp(nb);
        std::vector<int> par(nb);
        std::vector<int2> sr(nb), tr(nb);
        if (nb) {
            PK_CUDA(cudaMemcpy(bp.data(), t.bpos.p, sizeof(int4) * nb, cudaMemcpyDeviceToHost));
            PK_CUDA(cudaMemcpy(par.data(), t.parent.p, sizeof(int) * nb, cudaMemcpyDeviceToHost));
            PK_CUDA(cudaMemcpy(sr.data(), t.srange.p, sizeof(int2) * nb, cudaMemcpyDeviceToHost));
            PK_CUDA(cudaMemcpy(tr.data(), t.trange.p, sizeof(int2) * nb, cudaMemcpyDeviceToHost));
        }
        for (int b = 0; b < nb; b++) {
            if (level) level[b] = bp[b].w;
            if (pos) {
                pos[3 * b] = bp[b].x;
                pos[3 * b + 1] = bp[b].y;
                pos[3 * b + 2] = bp[b].z;
            }
            if (parent) parent[b] = par[b];
            if (src_range) {
                src_range[2 * b] = sr[b].x;
                src_range[2 * b + 1] = sr[b].y;
            }
            if (trg_range) {
                trg_range[2 * b] = tr[b].x;
                trg_range[2 * b + 1] = tr[b].y;
            }
        }
        auto perm = [&](int64_t *dst, const DBuf<int> &src, int64_t n) {
            if (!dst || !n) return;
            std::vector<int> h(n);
            PK_CUDA(cudaMemcpy(h.data(), src.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < n; i++) dst[i] = h[i];
        };
        perm(src_perm, P.idxS, P.S);
        perm(trg_perm, P.idxT, P.T);
        return PKIFMM_OK;
    });
}

int pkifmm_list_export(pkifmm_plan plan, char name, int64_t *list_ptr, int32_t *list_box, int8_t *list_shift) {
    if (!plan) return fail(PKIFMM_ERR_INVALID_ARG, "plan is NULL");
    return guarded([&]() {
        Plan &P = plan->P;
        Tree &t = P.tree;
        int nb = t.nbox;
        std::vector<int64_t> ptr(nb + 1, 0);
        std::vector<int> box;
        std::vector<int8_t> sh;
        auto csr = [&](const DBuf<int> &dp, const DBuf<int> &db, const DBuf<unsigned char> &ds, long long n) {
            std::vector<int> p32(nb + 1);
            PK_CUDA(cudaMemcpy(p32.data(), dp.p, sizeof(int) * (nb + 1), cudaMemcpyDeviceToHost));
            box.resize(n);
            std::vector<unsigned char> c(n);
            if (n) {
                PK_CUDA(cudaMemcpy(box.data(), db.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
                PK_CUDA(cudaMemcpy(c.data(), ds.p, n, cudaMemcpyDeviceToHost));
            }
            for (int b = 0; b <= nb; b++) ptr[b] = p32[b];
            sh.resize(3 * n);
            for (long long i = 0; i < n; i++) {
                sh[3 * i] = (int8_t)(c[i] / 9 - 1);
                sh[3 * i + 1] = (int8_t)((c[i] / 3) % 3 - 1);
                sh[3 * i + 2] = (int8_t)(c[i] % 3 - 1);
            }
        };
        if (name == 'U') csr(t.u_ptr, t.u_box, t.u_sh, t.nU);
        else if (name == 'W') csr(t.w_ptr, t.w_box, t.w_sh, t.nW);
        else if (name == 'X') csr(t.x_ptr, t.x_box, t.x_sh, t.nX);
        else if (name == 'V') {
            std::vector<int> vs((size_t)nb * kVSlots);
            std::vector<int4> bp(nb);
            if (nb) {
                PK_CUDA(cudaMemcpy(vs.data(), t.v_slot.p, sizeof(int) * vs.size(), cudaMemcpyDeviceToHost));
                PK_CUDA(cudaMemcpy(bp.data(), t.bpos.p, sizeof(int4) * nb, cudaMemcpyDeviceToHost));
            }
            // slot -> offset per octant class (same enumeration as the device tables)
            std::vector<int> soff(8 * kVSlots * 3);
            for (int c = 0; c < 8; c++) {
                int cb[3] = {c & 1, c >> 1 & 1, c >> 2 & 1}, s = 0;
                for (int x = -2 - cb[0]; x <= 3 - cb[0]; x++)
                    for (int y = -2 - cb[1]; y <= 3 - cb[1]; y++)
                        for (int z = -2 - cb[2]; z <= 3 - cb[2]; z++) {
                            if (std::max(std::abs(x), std::max(std::abs(y), std::abs(z))) <= 1) continue;
                            soff[(c * kVSlots + s) * 3] = x;
                            soff[(c * kVSlots + s) * 3 + 1] = y;
                            soff[(c * kVSlots + s) * 3 + 2] = z;
                            s++;
                        }
            }
            for (int b = 0; b < nb; b++) {
                ptr[b] = (int64_t)box.size();
                int pp[3] = {bp[b].x, bp[b].y, bp[b].z}, l = bp[b].w, n = 1 << l;
                int c = (pp[0] & 1) | (pp[1] & 1) << 1 | (pp[2] & 1) << 2;
                for (int s = 0; s < kVSlots; s++) {
                    int a = vs[(size_t)b * kVSlots + s];
                    if (a < 0) continue;
                    box.push_back(a);
                    for (int q = 0; q < 3; q++) {
                        int e = pp[q] + soff[(c * kVSlots + s) * 3 + q];
                        sh.push_back((int8_t)(e >= 0 ? e / n : -((-e + n - 1) / n)));
                    }
                }
            }
            ptr[nb] = (int64_t)box.size();
        } else {
            return fail(PKIFMM_ERR_INVALID_ARG, "list name must be U, V, W or X");
        }
        if (list_ptr) std::copy(ptr.begin(), ptr.end(), list_ptr);
        if (list_box) std::copy(box.begin(), box.end(), list_box);
        if (list_shift) std::copy(sh.begin(), sh.end(), list_shift);
        return (int)std::min<size_t>(box.size(), 0x7fffffff);
    });
}

int pkifmm_surface_singular_values(int kernel, int p, double *s_out) {
    if ((kernel != 0 && kernel != 1) || p < 2 || p > 16 || !s_out) return fail(PKIFMM_ERR_INVALID_ARG, "bad argument");
    return guarded([&]() {
        int n = surface_count(p);
        auto g = surface_grid(p);
        std::vector<double> x(3 * n), y(3 * n);
        for (int i = 0; i < 3 * n; i++) {
            x[i] = kInnerHalf * g[i];
            y[i] = kOuterHalf * g[i];
        }
        auto A = kernel_matrix(kernel, x, y);
        std::vector<double> U, S, V;
        jacobi_svd(n * (kernel ? 3 : 1), A, U, S, V);
        std::copy(S.begin(), S.end(), s_out);
        return PKIFMM_OK;
    });
}

int pkifmm_backward_error(int kernel, int p, double *err_out) {
    if ((kernel != 0 && kernel != 1) || p < 2 || p > 16 || !err_out) return fail(PKIFMM_ERR_INVALID_ARG, "bad argument");
    return guarded([&]() {
        int n = surface_count(p), m = n * (kernel ? 3 : 1);
        auto g = surface_grid(p);
        std::vector<double> x(3 * n), y(3 * n);
        for (int i = 0; i < 3 * n; i++) {
            x[i] = kInnerHalf * g[i];
            y[i] = kOuterHalf * g[i];
        }
        auto A = kernel_matrix(kernel, x, y);
        std::vector<double> U, S, V;
        jacobi_svd(m, A, U, S, V);
        double cut = std::ldexp(1.0, -52) * S[0];
        std::vector<double> t(m, 0.0), sol(m, 0.0);
        for (int j = 0; j < m; j++) {  // t = S+ (U^T b), b = 1
            double acc = 0;
            for (int i = 0; i < m; i++) acc += U[(size_t)i * m + j];
            t[j] = S[j] > cut ? acc / S[j] : 0.0;
        }
        for (int i = 0; i < m; i++) {  // x = V t
            double acc = 0;
            for (int j = 0; j < m; j++) acc += V[(size_t)i * m + j] * t[j];
            sol[i] = acc;
        }
        double e = 0;
        for (int i = 0; i < m; i++) {
            double acc = 0;
            for (int j = 0; j < m; j++) acc += A[(size_t)i * m + j] * sol[j];
            e = std::max(e, std::fabs(acc - 1.0));
        }
        *err_out = e;
        return PKIFMM_OK;
    });
}

int pkifmm_root_operator(int kernel, unsigned periodic_axes, int p, int ell, double *m_out) {
    bool sp = periodic_axes == 1 || periodic_axes == 2 || periodic_axes == 4;
    if ((kernel != 0 && kernel != 1) || p < 2 || p > 16 || ell < 1 || ell > 8 || !m_out)
        return fail(PKIFMM_ERR_INVALID_ARG, "bad argument");
    if (!(periodic_axes == 7 || periodic_axes == 3 || sp)) return fail(PKIFMM_ERR_UNSUPPORTED, "periodicity not built");
    return guarded([&]() {
        auto M = root_operator(kernel, p, periodic_axes, ell, surface_grid(p));
        std::copy(M.begin(), M.end(), m_out);
        return PKIFMM_OK;
    });
}

int pkifmm_root_operator_finite(int kernel, int axis, int nimg, int p, double *m_out) {
    if ((kernel != 0 && kernel != 1) || p < 2 || p > 16 || axis < 0 || axis > 2 || nimg < 0 || nimg > (1 << 20) ||
        !m_out)
        return fail(PKIFMM_ERR_INVALID_ARG, "bad argument");
    return guarded([&]() {
        auto M = root_operator(kernel, p, 1u << axis, 2, surface_grid(p), nimg);
        std::copy(M.begin(), M.end(), m_out);
        return PKIFMM_OK;
    });
}

int pkifmm_precompute_operators(int kernel, unsigned periodic_axes, int p, int ell, int precision, int where,
                                double *s_out, double *m2m_out, double *l2l_out, double *root_out,
                                double *seconds_out, double *phases_out) {
    bool sp = periodic_axes == 1 || periodic_axes == 2 || periodic_axes == 4;
    if ((kernel != 0 && kernel != 1) || p < 4 || p > 16 || ell < 1 || ell > 8 || (where != 0 && where != 1) ||
        (precision != PKIFMM_FP64 && precision != PKIFMM_MIXED))
        return fail(PKIFMM_ERR_INVALID_ARG, "bad argument");
    if (!(periodic_axes == 0 || periodic_axes == 7 || periodic_axes == 3 || sp))
        return fail(PKIFMM_ERR_UNSUPPORTED, "periodicity not built");
    return guarded([&]() {
        HostOps o;
        const int kn = surface_count(p) * (kernel ? 3 : 1);
        const double eps = svd_cut(kernel, p, precision == PKIFMM_FP64 ? 0 : 1, kn);
        if (where == 1) PK_CUDA(cudaFree(nullptr));  // context creation outside the timed build
        const auto t0 = std::chrono::steady_clock::now();
        if (where == 0) build_host_ops(o, kernel, p, periodic_axes, ell, eps, "");
        else build_device_ops(o, kernel, p, periodic_axes, ell, eps, "", phases_out);
        const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        const size_t kn2 = (size_t)kn * kn;
        if (s_out) std::copy(o.S.begin(), o.S.end(), s_out);
        if (m2m_out) std::copy(o.m2m.begin(), o.m2m.begin() + 8 * kn2, m2m_out);
        if (l2l_out) std::copy(o.l2l.begin(), o.l2l.begin() + 8 * kn2, l2l_out);
        if (root_out && periodic_axes) std::copy(o.root.begin(), o.root.end(), root_out);
        if (seconds_out) *seconds_out = sec;
        return PKIFMM_OK;
    });
}

void pkifmm_plan_destroy(pkifmm_plan plan) { destroy_plan(plan); }

const char *pkifmm_strerror(int code) {
    switch (code) {
        case PKIFMM_OK: return "ok";
        case PKIFMM_ERR_INVALID_ARG: return "invalid argument";
        case PKIFMM_ERR_OUT_OF_BOX: return "point outside the box along a free axis";
        case PKIFMM_ERR_NOT_NEUTRAL: return "compatibility condition violated (net charge or net force)";
        case PKIFMM_ERR_CUDA: return "CUDA error";
        case PKIFMM_ERR_OOM: return "out of memory";
        case PKIFMM_ERR_TIMEOUT: return "bounded device wait gave up";
        case PKIFMM_ERR_CACHE: return "operator cache unreadable or unwritable";
        case PKIFMM_ERR_UNSUPPORTED: return "combination not built";
        default: return "unknown error";
    }
}

const char *pkifmm_last_error_message(void) { return g_last_error.c_str(); }

int64_t pkifmm_launch_count(void) { return g_launches.load(); }

int pkifmm_m2l_rank(pkifmm_plan plan) {
    if (!plan) return fail(PKIFMM_ERR_INVALID_ARG, "plan is NULL");
    const Plan &P = plan->P;
    return P.basis ? P.basis->r : P.kn;
}

int pkifmm_m2l_tensor_core_enabled(void) { return m2l_tc_device_supported() ? 1 : 0; }

}  // extern "C"
