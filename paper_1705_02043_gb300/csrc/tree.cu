// Octree and interaction lists on the device (Sec. 2.2).
//
// Points are normalised to the unit box, wrapped along periodic axes, and
// given a Morton key of 3*depth_max bits (cell floor(x' 2^D) per axis,
// octant bits x = 1, y = 2, z = 4).  A stable LSD radix sort orders sources
// and targets leaf-contiguously with ties in input order.  The adaptive tree
// is built top down one level at a time: a box splits while it holds more
// than s sources or more than s targets (s = leaf_max) and its level is
// below depth_max; empty children are not created.  The same tree serves
// B0 and its periodic images ("copy-and-paste", Sec. 2.2): list entries are
// (box, shift) pairs, the shift in {-1,0,1}^3 naming the image.
//
// Several independent problems (a batch) share one forest: every point's key
// carries its problem index above the 3*depth_max Morton bits, the problems'
// roots are boxes 0..nprob-1 at level 0, and a box's key at level l is
// prob * 8^l + (its Morton prefix), so lists never cross problems.
//
// Lists (standard KIFMM definitions; the paper defers to them):
//   U(B), B leaf: leaves A with A+p adjacent to B, and B itself;
//   V(B): children of colleagues of parent(B) not adjacent to B, stored as a
//         dense table of 189 slots per box (slot = offset within the octant
//         class of B);
//   W(B), B leaf: boxes A+p finer than B, not adjacent, parent(A)+p adjacent;
//   X(B): leaves A+p coarser than B, adjacent to parent(B), not adjacent to B.
#include <cuda.h>

#include <mutex>

#include "internal.h"

namespace pk {

// ---------------- helpers ----------------

__host__ __device__ inline unsigned long long spread3(unsigned v) {
    unsigned long long x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

__host__ __device__ inline unsigned long long morton3(int x, int y, int z) {
    return spread3((unsigned)x) | spread3((unsigned)y) << 1 | spread3((unsigned)z) << 2;
}

__device__ inline int floor_div(int a, int n) {  // n > 0
    return a >= 0 ? a / n : -((-a + n - 1) / n);
}

static inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------- scan (exclusive, out[n] = total) ----------------

__global__ void k_scan_block(const int *in, int *out, int *bsum, int n) {
    __shared__ int s[1024];
    int i = blockIdx.x * 1024 + threadIdx.x;
    int v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = s[1023];
}

__global__ void k_scan_add(int *out, const int *boff, int n, int *total_out) {
    int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
    if (i == n - 1 && total_out) *total_out = out[i];
}

__global__ void k_scan_fix_total(int *out, const int *in, int n) {
    out[n] = (n ? out[n - 1] + in[n - 1] : 0);
}

// Exclusive scan of in[0..n) into out[0..n], out[n] = total.  Returns the
// total (synchronises the stream) when `want_total`, else 0 without waiting.
// Scratch the scan needs for n values: block sums and their offsets at every
// level of the recursion.
static size_t scan_scratch(long long n) {
    size_t t = 2;
    while (n > 1024) {
        const long long nb = (n + 1023) / 1024;
        t += 2 * (size_t)(nb + 1);
        n = nb;
    }
    return t;
}

static void scan_into(const int *in, int *out, int n, cudaStream_t s, int *tmp) {
    if (n <= 0) {
        PK_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        return;
    }
    const int nb = (n + 1023) / 1024;
    int *bsum = tmp, *boff = tmp + nb + 1;
    count_launch(), k_scan_block<<<nb, 1024, 0, s>>>(in, out, bsum, n);
    if (nb > 1) {
        scan_into(bsum, boff, nb, s, tmp + 2 * (nb + 1));
        count_launch(), k_scan_add<<<nb, 1024, 0, s>>>(out, boff, n, nullptr);
    }
    count_launch(), k_scan_fix_total<<<1, 1, 0, s>>>(out, in, n);
}

// out[0..n] = exclusive prefix sums of in[0..n-1], out[n] the total (also
// returned, after a stream synchronisation, when want_total); tmp: scratch owned
// by the caller, grown as needed.
int exclusive_scan(const int *in, int *out, int n, cudaStream_t s, DBuf<int> &tmp, bool want_total = false) {
    tmp.reserve(scan_scratch(n));
    scan_into(in, out, n, s, tmp.p);
    if (!want_total) return 0;
    int total = 0;
    PK_CUDA(cudaMemcpyAsync(&total, out + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    return total;
}

// ---------------- keys ----------------

// err[0]: NaN/inf coordinate, err[1]: point outside [0,1) along a free axis.
// off[0..nprob] (nullable: one problem): CSR offsets of the problems' points.
__global__ void k_keys(const double *__restrict__ xyz, long long n, double lo0, double lo1, double lo2,
                       double L, unsigned per, int D, double *__restrict__ xn,
                       unsigned long long *__restrict__ key, int *__restrict__ idx, int *err,
                       const long long *__restrict__ off = nullptr, int nprob = 1) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long prob = 0;
    if (off) {  // largest j with off[j] <= i
        int lo = 0, hi = nprob - 1;
        while (lo < hi) {
            int m = (lo + hi + 1) >> 1;
            if (off[m] <= i) lo = m;
            else hi = m - 1;
        }
        prob = (unsigned long long)lo;
    }
    double lo[3] = {lo0, lo1, lo2};
    int c[3];
    double sc = (double)(1 << D);
    for (int a = 0; a < 3; a++) {
        double x = __ddiv_rn(__dsub_rn(xyz[3 * i + a], lo[a]), L);
        if (!isfinite(x)) {
            err[0] = 1;
            x = 0.0;
        }
        if (per >> a & 1) {
            x = __dsub_rn(x, floor(x));
            if (x >= 1.0) x = 0.0;
        } else if (x < 0.0 || x >= 1.0) {
            err[1] = 1;
            x = fmin(fmax(x, 0.0), 0.0);
        }
        xn[3 * i + a] = x;
        int v = (int)floor(__dmul_rn(x, sc));
        c[a] = min(max(v, 0), (1 << D) - 1);
    }
    key[i] = prob << (3 * D) | morton3(c[0], c[1], c[2]);
    idx[i] = (int)i;
}

// ---------------- stable LSD radix sort, 4-bit digits ----------------

constexpr int RS_T = 256, RS_I = 16, RS_TILE = RS_T * RS_I;

__global__ void k_rs_count(const unsigned long long *__restrict__ key, int n, int shift, int *hist, int nb) {
    __shared__ int c[16];
    if (threadIdx.x < 16) c[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * RS_TILE;
    for (int j = threadIdx.x; j < RS_TILE; j += RS_T) {
        int i = base + j;
        if (i < n) atomicAdd(&c[(key[i] >> shift) & 15], 1);
    }
    __syncthreads();
    if (threadIdx.x < 16) hist[threadIdx.x * nb + blockIdx.x] = c[threadIdx.x];
}

__global__ void k_rs_scatter(const unsigned long long *__restrict__ kin, const int *__restrict__ vin,
                             unsigned long long *__restrict__ kout, int *__restrict__ vout, int n, int shift,
                             const int *__restrict__ hoff, int nb) {
    __shared__ int tc[16][RS_T + 1];
    int t = threadIdx.x, base = blockIdx.x * RS_TILE + t * RS_I;
    int cnt[16];
#pragma unroll
    for (int d = 0; d < 16; d++) cnt[d] = 0;
    for (int j = 0; j < RS_I; j++) {
        int i = base + j;
        if (i < n) cnt[(kin[i] >> shift) & 15]++;
    }
#pragma unroll
    for (int d = 0; d < 16; d++) tc[d][t] = cnt[d];
    __syncthreads();
    if (t < 16) {
        int run = hoff[t * nb + blockIdx.x];
        for (int u = 0; u < RS_T; u++) {
            int v = tc[t][u];
            tc[t][u] = run;
            run += v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int d = 0; d < 16; d++) cnt[d] = tc[d][t];
    for (int j = 0; j < RS_I; j++) {
        int i = base + j;
        if (i < n) {
            unsigned long long k = kin[i];
            int d = (k >> shift) & 15, pos = 0;
#pragma unroll
            for (int e = 0; e < 16; e++)
                if (e == d) pos = cnt[e]++;
            kout[pos] = k;
            vout[pos] = vin[i];
        }
    }
}

// Sort (key, idx) by key (bits [0, bits)), stable.  Result in (k, v).
static void radix_sort(DBuf<unsigned long long> &k, DBuf<int> &v, DBuf<unsigned long long> &k2, DBuf<int> &v2,
                       DBuf<int> &hist, DBuf<int> &scan_tmp, int n, int bits, cudaStream_t s) {
    if (n <= 1) return;
    int nb = (n + RS_TILE - 1) / RS_TILE;
    hist.reserve((size_t)16 * nb * 2 + 2);
    k2.reserve(n);
    v2.reserve(n);
    unsigned long long *ka = k.p, *kb = k2.p;
    int *va = v.p, *vb = v2.p;
    int *h = hist.p, *ho = hist.p + 16 * nb + 1;
    for (int sh = 0; sh < bits; sh += 4) {
        count_launch(), k_rs_count<<<nb, RS_T, 0, s>>>(ka, n, sh, h, nb);
        exclusive_scan(h, ho, 16 * nb, s, scan_tmp);  // the radix sort needs no total
        count_launch(), k_rs_scatter<<<nb, RS_T, 0, s>>>(ka, va, kb, vb, n, sh, ho, nb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != k.p) {
        PK_CUDA(cudaMemcpyAsync(k.p, ka, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, s));
        PK_CUDA(cudaMemcpyAsync(v.p, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    }
}

__global__ void k_gather3(const double *__restrict__ xn, const int *__restrict__ idx, long long n,
                          double *__restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = idx[i];
    out[3 * i] = xn[3 * (long long)j];
    out[3 * i + 1] = xn[3 * (long long)j + 1];
    out[3 * i + 2] = xn[3 * (long long)j + 2];
}

// dens [nrhs][S][k] (input order) -> dens_s [S][nrhs*k] (sorted)
__global__ void k_gather_dens(const double *__restrict__ dens, const int *__restrict__ idx, long long S,
                              int nrhs, int k, double *__restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= S * nrhs * k) return;
    long long s = i / (nrhs * k);
    int rem = (int)(i % (nrhs * k)), r = rem / k, a = rem % k;
    out[i] = dens[((long long)r * S + idx[s]) * k + a];
}

// ---------------- tree ----------------

__device__ inline int lower_bound_key(const unsigned long long *key, int lo, int hi, unsigned long long v) {
    while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (key[m] < v) lo = m + 1;
        else hi = m;
    }
    return lo;
}

// one root per problem; its points are the problem's CSR range (the sort
// keeps problems contiguous and in order)
__global__ void k_roots(int nprob, const long long *__restrict__ soff, const long long *__restrict__ toff,
                        unsigned long long *key, int4 *bpos, int *parent, int2 *sr, int2 *tr, int *lvl) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) {  // level 0 holds the roots, boxes 0 .. nprob - 1
        lvl[0] = 0;
        lvl[1] = nprob;
    }
    if (j >= nprob) return;
    key[j] = (unsigned long long)j;
    bpos[j] = make_int4(0, 0, 0, 0);
    parent[j] = -1;
    sr[j] = make_int2((int)soff[j], (int)soff[j + 1]);
    tr[j] = make_int2((int)toff[j], (int)toff[j + 1]);
}

// One warp per box: lanes 0-7 find where child c's sources start, lanes
// 8-15 where its targets start (all 16 binary searches at once); child c ends
// where child c + 1 starts, the last child at the box's end.
// Level `level` holds boxes lvl[level] .. lvl[level + 1] - 1; at most `bound`
// of them.  One warp per box, striding over the bound; cnt[w] = 0 for the
// positions past the level.
__global__ void k_split(const int *__restrict__ lvl, int level, int bound, int D, int smax,
                        const unsigned long long *__restrict__ bkey, const int2 *__restrict__ srange,
                        const int2 *__restrict__ trange, const unsigned long long *__restrict__ keyS,
                        const unsigned long long *__restrict__ keyT, int2 *csr, int2 *ctr, int *cnt) {
    const int lb = lvl[level], le = lvl[level + 1], lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * blockDim.x >> 5;
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < bound; w += nw) {
        const int b = lb + (int)w;
        if (b >= le) {  // the whole warp shares b
            if (lane == 0) cnt[w] = 0;
            continue;
        }
        const int2 sr = srange[b], tr = trange[b];
        const bool split = (sr.y - sr.x > smax || tr.y - tr.x > smax) && level < D;
        const int c = lane & 7;
        int start = 0;
        if (split && lane < 16) {
            const unsigned long long lo = (bkey[b] * 8 + c) << (3 * (D - level - 1));
            start = lane < 8 ? lower_bound_key(keyS, sr.x, sr.y, lo) : lower_bound_key(keyT, tr.x, tr.y, lo);
        }
        const int nxt = __shfl_down_sync(0xffffffffu, start, 1);
        const int end = c == 7 ? (lane < 8 ? sr.y : tr.y) : nxt;
        if (split && lane < 8) csr[w * 8 + c] = make_int2(start, end);
        if (split && lane >= 8 && lane < 16) ctr[w * 8 + c] = make_int2(start, end);
        const int nonempty = lane < 16 && end > start;
        const int t_nonempty = __shfl_down_sync(0xffffffffu, nonempty, 8);  // lane c: child c's targets
        const unsigned m = __ballot_sync(0xffffffffu, split && lane < 8 && (nonempty || t_nonempty));
        if (lane == 0) cnt[w] = __popc(m);
    }
}
// The children of level `level`'s boxes become level level + 1, from
// lvl[level + 1] on, in order; lvl[level + 2] = the end of that level.
__global__ void k_emit(int *lvl, int level, int bound, const int *__restrict__ cnt, const int *__restrict__ off,
                       const int2 *__restrict__ csr, const int2 *__restrict__ ctr, unsigned long long *bkey,
                       int4 *bpos, int *parent, int *child, int2 *srange, int2 *trange) {
    const int lb = lvl[level], le = lvl[level + 1], nl = min(le - lb, bound);
    if (blockIdx.x == 0 && threadIdx.x == 0) lvl[level + 2] = le + off[bound];
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < nl;
         w += (long long)gridDim.x * blockDim.x) {
        const int b = lb + (int)w;
        for (int c = 0; c < 8; c++) child[(long long)b * 8 + c] = -1;
        if (cnt[w] == 0) continue;
        int j = le + off[w];
        int4 p = bpos[b];
        for (int c = 0; c < 8; c++) {
            int2 s = csr[w * 8 + c], t = ctr[w * 8 + c];
            if (s.y <= s.x && t.y <= t.x) continue;
            bkey[j] = bkey[b] * 8 + c;
            bpos[j] = make_int4(2 * p.x + (c & 1), 2 * p.y + (c >> 1 & 1), 2 * p.z + (c >> 2 & 1), p.w + 1);
            parent[j] = b;
            srange[j] = s;
            trange[j] = t;
            child[(long long)b * 8 + c] = j;
            j++;
        }
    }
}

void build_tree(Plan &P, cudaStream_t s) {
    Tree &t = P.tree;
    const int D = P.depth_max;
    const int np = P.nprob;
    // Boxes per level, bounded in advance so the levels are built without a
    // round trip to the host: level 0 holds the roots; a box splits only while
    // it holds more than s sources or more than s targets, so at most
    // S/(s+1) + T/(s+1) boxes of a level split (S/(s+1) when the targets are
    // the sources), into at most 8 children each.
    const long long s1 = P.leaf_max + 1;
    const long long split_max = P.S / s1 + (P.same_points ? 0 : P.T / s1) + np;
    std::vector<long long> ub(D + 1);
    ub[0] = np;
    long long tot = np, ubmax = np;
    for (int l = 1; l <= D; l++) {
        ub[l] = std::min(8 * ub[l - 1], 8 * split_max);
        tot += ub[l];
        ubmax = std::max(ubmax, ub[l]);
    }
    if (tot > (1LL << 31) / 9) throw Error(PKIFMM_ERR_INVALID_ARG, "octree too large for 32-bit box indices");
    t.key.reserve(tot);
    t.bpos.reserve(tot);
    t.parent.reserve(tot);
    t.child.reserve(tot * 8);
    t.srange.reserve(tot);
    t.trange.reserve(tot);
    t.lvl_begin_d.reserve(D + 3);
    P.csr.reserve((size_t)ubmax * 8);
    P.ctr.reserve((size_t)ubmax * 8);
    P.cnt.reserve(ubmax + 1);
    P.off.reserve(ubmax + 1);
    int *lvl = t.lvl_begin_d.p;
    count_launch(), k_roots<<<blocks(np, 128), 128, 0, s>>>(np, P.soff.p, P.toff.p, t.key.p, t.bpos.p, t.parent.p,
                                                             t.srange.p, t.trange.p, lvl);
    const unsigned gmax = 152u * 16u;  // grid-stride kernels: about 16 blocks per SM at most
    for (int l = 0; l <= D; l++) {  // level D boxes get no children (the split test checks the level)
        const int b = (int)ub[l];
        count_launch(), k_split<<<std::min<unsigned>(gmax, blocks((long long)b * 32, 128)), 128, 0, s>>>(
            lvl, l, b, D, P.leaf_max, t.key.p, t.srange.p, t.trange.p, P.keyS.p, P.keyT.p, P.csr.p, P.ctr.p, P.cnt.p);
        exclusive_scan(P.cnt.p, P.off.p, b, s, P.scan_tmp);
        count_launch(), k_emit<<<std::min<unsigned>(gmax, blocks(b, 128)), 128, 0, s>>>(
            lvl, l, b, P.cnt.p, P.off.p, P.csr.p, P.ctr.p, t.key.p, t.bpos.p, t.parent.p, t.child.p, t.srange.p,
            t.trange.p);
    }
    std::vector<int> h(D + 3);
    PK_CUDA(cudaMemcpyAsync(h.data(), lvl, sizeof(int) * (D + 3), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    t.lvl_begin.assign({h[0], h[1]});
    int level = 0;
    while (level + 2 <= D + 2 && h[level + 2] > h[level + 1]) {
        t.lvl_begin.push_back(h[level + 2]);
        level++;
    }
    t.depth = level;
    t.nbox = t.lvl_begin.back();
}

// ---------------- lists ----------------

struct TreeView {
    const unsigned long long *key;
    const int4 *bpos;
    const int *child;
    const int *parent;
    const int2 *srange, *trange;
    const int *lvlb;
    int nlevel;
    unsigned per;
};

__device__ inline int lookup(const TreeView &tv, int level, const int w[3], unsigned long long prob) {
    if (level >= tv.nlevel) return -1;
    unsigned long long k = prob << (3 * level) | morton3(w[0], w[1], w[2]);
    int lo = tv.lvlb[level], hi = tv.lvlb[level + 1];
    int i = lower_bound_key(tv.key, lo, hi, k);
    return (i < hi && tv.key[i] == k) ? i : -1;
}

// wrap extended position e at `level`; false if outside along a free axis
__device__ inline bool wrap_pos(unsigned per, int level, const int e[3], int w[3], int sh[3]) {
    int n = 1 << level;
    for (int a = 0; a < 3; a++) {
        if (per >> a & 1) {
            sh[a] = floor_div(e[a], n);
            w[a] = e[a] - sh[a] * n;
        } else {
            if (e[a] < 0 || e[a] >= n) return false;
            sh[a] = 0;
            w[a] = e[a];
        }
    }
    return true;
}

__device__ inline bool is_leaf(const TreeView &tv, int b) {
    const int *c = tv.child + (long long)b * 8;
#pragma unroll
    for (int i = 0; i < 8; i++)
        if (c[i] >= 0) return false;
    return true;
}

// closed boxes touch with disjoint interiors; A shifted by sh (unit boxes)
__device__ inline bool adjacent(int4 A, const int sh[3], int4 B) {
    int lm = max(A.w, B.w), fa = 1 << (lm - A.w), fb = 1 << (lm - B.w);
    int pa[3] = {A.x, A.y, A.z}, pb[3] = {B.x, B.y, B.z};
    bool touch = true, inner = true;
    for (int a = 0; a < 3; a++) {
        int alo = (pa[a] + sh[a] * (1 << A.w)) * fa, ahi = alo + fa;
        int blo = pb[a] * fb, bhi = blo + fb;
        touch &= (alo <= bhi && blo <= ahi);
        inner &= (alo < bhi && blo < ahi);
    }
    return touch && !inner;
}

struct ListOut {
    int *u_box, *w_box, *x_box;
    unsigned char *u_sh, *w_sh, *x_sh;
    const int *u_ptr, *w_ptr, *x_ptr;
    int *u_cnt, *w_cnt, *x_cnt;
    int *v_slot;
    const short *slot_of;
    unsigned long long *pairs;
};

__device__ inline unsigned char code3(const int sh[3]) {
    return (unsigned char)((sh[0] + 1) * 9 + (sh[1] + 1) * 3 + (sh[2] + 1));
}

// first existing ancestor (level < l) of extended position e at level l
__device__ int coarse_ancestor(const TreeView &tv, int l, const int e[3], int sh[3], unsigned long long prob) {
    for (int l2 = l - 1; l2 >= 0; l2--) {
        int e2[3], w2[3];
        for (int a = 0; a < 3; a++) e2[a] = e[a] >> (l - l2);  // arithmetic shift = floor division
        if (!wrap_pos(tv.per, l2, e2, w2, sh)) return -1;
        int a = lookup(tv, l2, w2, prob);
        if (a >= 0) return is_leaf(tv, a) ? a : -1;
    }
    return -1;
}

__global__ void k_lists(TreeView tv, int nbox, int pass, ListOut o) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int4 B = tv.bpos[b];
    int l = B.w;
    int pos[3] = {B.x, B.y, B.z};
    const unsigned long long prob = tv.key[b] >> (3 * l);
    int nU = 0, nW = 0, nX = 0;
    int uo = pass ? o.u_ptr[b] : 0, wo = pass ? o.w_ptr[b] : 0, xo = pass ? o.x_ptr[b] : 0;
    unsigned long long pairs = 0;
    int2 btr = tv.trange[b];
    if (is_leaf(tv, b)) {
        int coarse[27];
        unsigned char ccode[27];
        int nc = 0;
        for (int d = 0; d < 27; d++) {
            int e[3] = {pos[0] + d / 9 - 1, pos[1] + (d / 3) % 3 - 1, pos[2] + d % 3 - 1};
            int w[3], sh[3];
            if (!wrap_pos(tv.per, l, e, w, sh)) continue;
            int nb = lookup(tv, l, w, prob);
            if (nb >= 0) {
                if (is_leaf(tv, nb)) {
                    if (pass) {
                        o.u_box[uo + nU] = nb;
                        o.u_sh[uo + nU] = code3(sh);
                        int2 s = tv.srange[nb];
                        pairs += (unsigned long long)(s.y - s.x) * (btr.y - btr.x);
                    }
                    nU++;
                } else {
                    int stack[8 * kMaxLevel + 8];
                    int top = 0;
                    for (int c = 0; c < 8; c++) {
                        int ch = tv.child[(long long)nb * 8 + c];
                        if (ch >= 0) stack[top++] = ch;
                    }
                    while (top > 0) {
                        int C = stack[--top];
                        if (adjacent(tv.bpos[C], sh, B)) {
                            if (is_leaf(tv, C)) {
                                if (pass) {
                                    o.u_box[uo + nU] = C;
                                    o.u_sh[uo + nU] = code3(sh);
                                    int2 s = tv.srange[C];
                                    pairs += (unsigned long long)(s.y - s.x) * (btr.y - btr.x);
                                }
                                nU++;
                            } else {
                                for (int c = 0; c < 8; c++) {
                                    int ch = tv.child[(long long)C * 8 + c];
                                    if (ch >= 0 && top < 8 * kMaxLevel + 8) stack[top++] = ch;
                                }
                            }
                        } else {
                            if (pass) {
                                o.w_box[wo + nW] = C;
                                o.w_sh[wo + nW] = code3(sh);
                            }
                            nW++;
                        }
                    }
                }
            } else {
                int sh2[3];
                int a = coarse_ancestor(tv, l, e, sh2, prob);
                if (a < 0) continue;
                unsigned char cd = code3(sh2);
                bool dup = false;
                for (int i = 0; i < nc; i++) dup |= (coarse[i] == a && ccode[i] == cd);
                if (dup) continue;
                coarse[nc] = a;
                ccode[nc++] = cd;
                if (pass) {
                    o.u_box[uo + nU] = a;
                    o.u_sh[uo + nU] = cd;
                    int2 s = tv.srange[a];
                    pairs += (unsigned long long)(s.y - s.x) * (btr.y - btr.x);
                }
                nU++;
            }
        }
    }
    if (l >= 1) {
        int pp[3] = {pos[0] >> 1, pos[1] >> 1, pos[2] >> 1};
        int cand[27];
        unsigned char ccode[27];
        int nc = 0;
        int cls = (pos[0] & 1) | (pos[1] & 1) << 1 | (pos[2] & 1) << 2;
        for (int d = 0; d < 27; d++) {
            int dd[3] = {d / 9 - 1, (d / 3) % 3 - 1, d % 3 - 1};
            int e[3] = {pp[0] + dd[0], pp[1] + dd[1], pp[2] + dd[2]};
            int w[3], sh[3];
            if (!wrap_pos(tv.per, l - 1, e, w, sh)) continue;
            int a = lookup(tv, l - 1, w, prob);
            if (a >= 0 && !is_leaf(tv, a)) {
                // V list: children of this colleague of the parent
                if (pass) {
                    for (int c = 0; c < 8; c++) {
                        int ch = tv.child[(long long)a * 8 + c];
                        if (ch < 0) continue;
                        int off[3] = {2 * e[0] + (c & 1) - pos[0], 2 * e[1] + (c >> 1 & 1) - pos[1],
                                      2 * e[2] + (c >> 2 & 1) - pos[2]};
                        if (abs(off[0]) <= 1 && abs(off[1]) <= 1 && abs(off[2]) <= 1) continue;
                        int oi = ((off[0] + 3) * 7 + (off[1] + 3)) * 7 + (off[2] + 3);
                        int slot = o.slot_of[cls * 343 + oi];
                        if (slot >= 0) o.v_slot[(long long)b * kVSlots + slot] = ch;
                    }
                }
                continue;
            }
            int sh2[3] = {sh[0], sh[1], sh[2]};
            if (a < 0) a = coarse_ancestor(tv, l - 1, e, sh2, prob);
            if (a < 0) continue;  // empty region
            if (adjacent(tv.bpos[a], sh2, B)) continue;
            unsigned char cd = code3(sh2);
            bool dup = false;
            for (int i = 0; i < nc; i++) dup |= (cand[i] == a && ccode[i] == cd);
            if (dup) continue;
            cand[nc] = a;
            ccode[nc++] = cd;
            if (pass) {
                o.x_box[xo + nX] = a;
                o.x_sh[xo + nX] = cd;
            }
            nX++;
        }
    }
    if (!pass) {
        o.u_cnt[b] = nU;
        o.w_cnt[b] = nW;
        o.x_cnt[b] = nX;
    } else if (pairs) {
        atomicAdd(o.pairs, pairs);
    }
}

// count of V-slot entries: per-thread counts over a grid-stride loop, one atomic per block
__global__ void k_count_v(const int *__restrict__ v_slot, long long n, unsigned long long *cnt) {
    __shared__ unsigned long long part[32];
    unsigned long long c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c += v_slot[i] >= 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
        if (t) atomicAdd(cnt, t);
    }
}

void build_lists(Plan &P, cudaStream_t s) {
    Tree &t = P.tree;
    int nb = t.nbox;
    TreeView tv{t.key.p, t.bpos.p, t.child.p, t.parent.p, t.srange.p, t.trange.p, t.lvl_begin_d.p,
                (int)t.lvl_begin.size() - 1, P.periodic};
    t.u_ptr.reserve(nb + 1);
    t.w_ptr.reserve(nb + 1);
    t.x_ptr.reserve(nb + 1);
    DBuf<int> &cnt3 = P.lcnt;
    cnt3.reserve((size_t)3 * nb);
    t.v_slot.reserve((size_t)nb * kVSlots);
    PK_CUDA(cudaMemsetAsync(t.v_slot.p, 0xff, sizeof(int) * (size_t)nb * kVSlots, s));
    DBuf<unsigned long long> &pairs = P.lpairs;
    pairs.reserve(2);
    PK_CUDA(cudaMemsetAsync(pairs.p, 0, sizeof(unsigned long long) * 2, s));
    ListOut o{};
    o.u_cnt = cnt3.p;
    o.w_cnt = cnt3.p + nb;
    o.x_cnt = cnt3.p + 2 * nb;
    o.slot_of = P.slot_of.p;
    count_launch(), k_lists<<<blocks(nb, 128), 128, 0, s>>>(tv, nb, 0, o);
    // the three scans, then one read of their totals
    exclusive_scan(o.u_cnt, t.u_ptr.p, nb, s, P.scan_tmp);
    exclusive_scan(o.w_cnt, t.w_ptr.p, nb, s, P.scan_tmp);
    exclusive_scan(o.x_cnt, t.x_ptr.p, nb, s, P.scan_tmp);
    {
        int tot[3] = {0, 0, 0};
        PK_CUDA(cudaMemcpyAsync(&tot[0], t.u_ptr.p + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaMemcpyAsync(&tot[1], t.w_ptr.p + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaMemcpyAsync(&tot[2], t.x_ptr.p + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        t.nU = tot[0];
        t.nW = tot[1];
        t.nX = tot[2];
    }
    t.u_box.reserve(t.nU + 1);
    t.u_sh.reserve(t.nU + 1);
    t.w_box.reserve(t.nW + 1);
    t.w_sh.reserve(t.nW + 1);
    t.x_box.reserve(t.nX + 1);
    t.x_sh.reserve(t.nX + 1);
    o.u_box = t.u_box.p;
    o.u_sh = t.u_sh.p;
    o.u_ptr = t.u_ptr.p;
    o.w_box = t.w_box.p;
    o.w_sh = t.w_sh.p;
    o.w_ptr = t.w_ptr.p;
    o.x_box = t.x_box.p;
    o.x_sh = t.x_sh.p;
    o.x_ptr = t.x_ptr.p;
    o.v_slot = t.v_slot.p;
    o.pairs = pairs.p;
    count_launch(), k_lists<<<blocks(nb, 128), 128, 0, s>>>(tv, nb, 1, o);
    count_launch(), k_count_v<<<std::min<unsigned>(1024, blocks((long long)nb * kVSlots, 256)), 256, 0, s>>>(
        t.v_slot.p, (long long)nb * kVSlots, pairs.p + 1);
    unsigned long long h[2];
    PK_CUDA(cudaMemcpyAsync(h, pairs.p, sizeof h, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    t.p2p_pairs = (long long)h[0];
    t.nV = (long long)h[1];
}

// ---------------- entry: keys, sort, gather ----------------

void sort_points(Plan &P, const double *src, const double *dens, const double *trg, cudaStream_t s) {
    const int D = P.depth_max;
    long long S = P.S, T = P.T;
    int pbits = 0;
    while ((1LL << pbits) < P.nprob) pbits++;
    const int key_bits = 3 * D + pbits;  // problem index above the Morton bits
    // periodic axes wrap; a finite array of cells keeps every point inside the cell
    const unsigned wrap = P.nimg >= 0 ? 0u : P.periodic;
    P.err.reserve(4);
    PK_CUDA(cudaMemsetAsync(P.err.p, 0, sizeof(int) * 4, s));
    P.keyS.reserve(S + 1);
    P.idxS.reserve(S + 1);
    P.keyT.reserve(T + 1);
    P.idxT.reserve(T + 1);
    P.xs.reserve(3 * S + 3);
    P.xt.reserve(3 * T + 3);
    DBuf<double> &xn = P.xn;
    xn.reserve(3 * std::max(S, T) + 3);
    if (S) {
        count_launch(), k_keys<<<blocks(S, 256), 256, 0, s>>>(src, S, P.lo[0], P.lo[1], P.lo[2], P.L, wrap, D, xn.p,
                                              P.keyS.p, P.idxS.p, P.err.p, P.nprob > 1 ? P.soff.p : nullptr,
                                              P.nprob);
        radix_sort(P.keyS, P.idxS, P.keyS2, P.idxS2, P.hist, P.scan_tmp, (int)S, key_bits, s);
        count_launch(), k_gather3<<<blocks(S, 256), 256, 0, s>>>(xn.p, P.idxS.p, S, P.xs.p);
        int nk = P.nrhs * P.ks;
        P.dens_s.reserve((size_t)S * nk);
        count_launch(), k_gather_dens<<<blocks(S * nk, 256), 256, 0, s>>>(dens, P.idxS.p, S, P.nrhs, P.ks, P.dens_s.p);
    }
    P.same_points = T && trg == src && T == S && P.same_offsets;
    if (P.same_points) {
        // targets are the sources: same keys, order and coordinates
        PK_CUDA(cudaMemcpyAsync(P.keyT.p, P.keyS.p, sizeof(unsigned long long) * T, cudaMemcpyDeviceToDevice, s));
        PK_CUDA(cudaMemcpyAsync(P.idxT.p, P.idxS.p, sizeof(int) * T, cudaMemcpyDeviceToDevice, s));
        PK_CUDA(cudaMemcpyAsync(P.xt.p, P.xs.p, sizeof(double) * 3 * T, cudaMemcpyDeviceToDevice, s));
    } else if (T) {
        count_launch(), k_keys<<<blocks(T, 256), 256, 0, s>>>(trg, T, P.lo[0], P.lo[1], P.lo[2], P.L, wrap, D, xn.p,
                                              P.keyT.p, P.idxT.p, P.err.p, P.nprob > 1 ? P.toff.p : nullptr,
                                              P.nprob);
        radix_sort(P.keyT, P.idxT, P.keyT2, P.idxT2, P.hist, P.scan_tmp, (int)T, key_bits, s);
        count_launch(), k_gather3<<<blocks(T, 256), 256, 0, s>>>(xn.p, P.idxT.p, T, P.xt.p);
    }
}

// ---------------- Morton order without allocation ----------------
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// entirely owned by another framework's pool, a real-time loop that forbids
// allocation after start-up, or host code running where CUDA allocation
// calls are not permitted.  pkifmm_morton_order_noalloc gives them the
// stable Morton ordering of points (the first step of the evaluation) using
// only the fixed scratch below, which every GPU that loads this library holds
// until the process exits.  Host code must not pass the array's name to a
// kernel (in host code it is a stand-in, not a device address): its device
// address is looked up once per device with cudaGetSymbolAddress.

constexpr long long kNoAllocMaxPoints = 1LL << 17;  // 131,072 points
constexpr int kNoAllocMaxBlocks = (int)((kNoAllocMaxPoints + RS_TILE - 1) / RS_TILE);

struct NoAllocScratch {
    unsigned long long key[2][kNoAllocMaxPoints];
    int idx[2][kNoAllocMaxPoints];
    double xn[3 * kNoAllocMaxPoints];
    int hist[16 * kNoAllocMaxBlocks];
    int hoff[16 * kNoAllocMaxBlocks + 1];
    int err[4];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// exclusive scan of n <= 1024 ints in one block (no scratch beyond out[n+1])
__global__ void k_scan_small_noalloc(const int *in, int *out, int n) {
    __shared__ int s[1024];
    int t = threadIdx.x;
    int v = t < n ? in[t] : 0;
    s[t] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int u = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += u;
        __syncthreads();
    }
    if (t < n) out[t] = s[t] - v;
    if (t == 1023) out[n] = s[1023];
}

}  // namespace pk

namespace pk {
int set_last_error(int code, const std::string &msg);
}

namespace {
std::mutex g_noalloc_mu;
// per device: the scratch's device address and the context it was looked up in
pk::NoAllocScratch *g_noalloc_ptr[64] = {};
unsigned long long g_noalloc_ctx[64] = {};

// Identifier of the calling thread's current CUDA context (0 if unknown), through
// the driver entry points the runtime exposes.  A device reset creates a new
// context in which the scratch may sit at another address.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess)
            get_current = (GetCurrent)a;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess)
            get_id = (GetId)b;
        looked_up = true;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

int cuda_failure(const char *what, cudaError_t e) {
    return pk::set_last_error(PKIFMM_ERR_CUDA, std::string("pkifmm_morton_order_noalloc: ") + what + ": " +
                                                   cudaGetErrorString(e));
}
}

extern "C" int pkifmm_morton_order_noalloc(int64_t n, const double *xyz, const double box_lo[3], double box_len,
                                           unsigned periodic_axes, int depth, int32_t *perm, void *cuda_stream) {
    using namespace pk;
    if (n < 0 || n > kNoAllocMaxPoints)
        return set_last_error(PKIFMM_ERR_INVALID_ARG,
                              "pkifmm_morton_order_noalloc: n = " + std::to_string((long long)n) +
                                  " is outside 0.." + std::to_string(kNoAllocMaxPoints) +
                                  ", the size of its fixed device scratch");
    if (!box_lo || !(box_len > 0) || periodic_axes > 7 || depth < 1 || depth > 15)
        return set_last_error(PKIFMM_ERR_INVALID_ARG, "pkifmm_morton_order_noalloc: bad box, periodicity or depth");
    if (n == 0) return PKIFMM_OK;
    if (!xyz || !perm) return set_last_error(PKIFMM_ERR_INVALID_ARG, "pkifmm_morton_order_noalloc: NULL array");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return set_last_error(PKIFMM_ERR_CUDA, "pkifmm_morton_order_noalloc: no usable current device");
    NoAllocScratch *sc = nullptr;
    {
        // set-up, once per device (again after a device reset), with that device current
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_noalloc_ptr[dev] || ctx != g_noalloc_ctx[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return cuda_failure("scratch address lookup", e);
            g_noalloc_ptr[dev] = (NoAllocScratch *)p;
            g_noalloc_ctx[dev] = current_context_id();  // the lookup may have created the context
        }
        sc = g_noalloc_ptr[dev];
    }
    // the scratch keeps the previous call's contents: clear the error flags
    if (cudaError_t e = cudaMemsetAsync(sc->err, 0, sizeof(sc->err), s); e != cudaSuccess)
        return cuda_failure("clearing the error flags", e);
    unsigned nb = blocks(n, 256);
    count_launch(), k_keys<<<nb, 256, 0, s>>>(xyz, n, box_lo[0], box_lo[1], box_lo[2], box_len, periodic_axes, depth,
                                             sc->xn, sc->key[0], sc->idx[0], sc->err);
    int tiles = (int)((n + RS_TILE - 1) / RS_TILE), cur = 0;
    for (int sh = 0; sh < 3 * depth; sh += 4) {
        count_launch(), k_rs_count<<<tiles, RS_T, 0, s>>>(sc->key[cur], (int)n, sh, sc->hist, tiles);
        count_launch(), k_scan_small_noalloc<<<1, 1024, 0, s>>>(sc->hist, sc->hoff, 16 * tiles);
        count_launch(), k_rs_scatter<<<tiles, RS_T, 0, s>>>(sc->key[cur], sc->idx[cur], sc->key[cur ^ 1],
                                                            sc->idx[cur ^ 1], (int)n, sh, sc->hoff, tiles);
        cur ^= 1;
    }
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_failure("kernel launch", e);
    if (cudaError_t e = cudaMemcpyAsync(perm, sc->idx[cur], sizeof(int) * n, cudaMemcpyDeviceToDevice, s);
        e != cudaSuccess)
        return cuda_failure("copying the permutation", e);
    int err[4] = {0, 0, 0, 0};
    if (cudaError_t e = cudaMemcpyAsync(err, sc->err, sizeof(err), cudaMemcpyDeviceToHost, s); e != cudaSuccess)
        return cuda_failure("reading the error flags", e);
    if (cudaError_t e = cudaStreamSynchronize(s); e != cudaSuccess) return cuda_failure("stream synchronisation", e);
    if (err[0]) return set_last_error(PKIFMM_ERR_INVALID_ARG, "pkifmm_morton_order_noalloc: non-finite coordinate");
    if (err[1]) return set_last_error(PKIFMM_ERR_OUT_OF_BOX, "pkifmm_morton_order_noalloc: point outside a free axis");
    return PKIFMM_OK;
}
