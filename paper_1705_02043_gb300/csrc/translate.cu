// Translations of the KIFMM passes (Sec. 2.2) on the device.
//
// Densities live per box as rows [box][nrhs][kn] (kn = k * n equivalent
// values).  With q~ = h q (check potential times box edge) every operator is
// level independent (both kernels are homogeneous of degree -1):
//   S2M   q~u  = h sum_s K(c + 1.475 h g_i, y_s) phi_s            (leaf kernel sum)
//   UC2E  phi_u = (V S+)(U^T q~u)                                  (two products, Sec. 3.1)
//   M2M   phi_u(P) = sum_children T_M2M[oct] phi_u(C)
//   root  q~d(B0) = M_root phi_u(B0)                               (Algorithm 2 step c)
//   M2L   q~d(B) = sum_{V} K(0.525 g_i, o + 0.525 g_j) phi_u(A)    (o = offset in boxes)
//   S2L   q~d(B) += h sum_{X} K(c + 0.525 h g_i, y_s + p) phi_s
//   DC2E  phi_d = (U S+)(V^T q~d)
//   L2L   phi_d(C) += T_L2L[oct] phi_d(P)                          (carries the far field down)
//   leaf  q_t = L2T + W-list M2T + U-list P2P (incl. periodic images)
// Dense translations share one "slot GEMM": each destination row gathers
// its source rows through a slot table and multiplies by the operator its
// (class, slot) selects; boxes are grouped by class so a tile of rows shares
// every operator load.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "internal.h"
#include "kernels.cuh"

namespace pk {

void sort_points(Plan &P, const double *src, const double *dens, const double *trg, cudaStream_t s);
void m2l_tc_prepare(Plan &P);
bool m2l_tc_run(Plan &P, cudaStream_t s);

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------- operator upload ----------------

// K_o[i*k+a][j*k+b] = K(0.525 g_i, o + 0.525 g_j) for the 316 M2L offsets.
template <typename T>
__global__ void k_m2l_ops(int kernel, int n, const double *__restrict__ g, const int *__restrict__ offs,
                          T *__restrict__ out) {
    int kk = kernel == 0 ? 1 : 3, kn = n * kk;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)kM2LOps * n * n;
    if (i >= total) return;
    int m = (int)(i / ((long long)n * n)), rem = (int)(i % ((long long)n * n)), a = rem / n, b = rem % n;
    double d[3];
    for (int c = 0; c < 3; c++) d[c] = 0.525 * g[3 * a + c] - (offs[3 * m + c] + 0.525 * g[3 * b + c]);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double ir = 1.0 / sqrt(r2);
    T *o = out + (long long)m * kn * kn;
    if (kernel == 0) {
        o[(long long)a * kn + b] = (T)ir;
    } else {
        double c8 = 1.0 / (8.0 * 3.14159265358979323846), ir3 = ir * ir * ir;
        for (int p = 0; p < 3; p++)
            for (int q = 0; q < 3; q++)
                o[(long long)(a * 3 + p) * kn + b * 3 + q] = (T)(c8 * ((p == q ? ir : 0.0) + d[p] * d[q] * ir3));
    }
}

template <typename T>
static void upload(DBuf<T> &d, const std::vector<double> &h) {
    d.reserve(h.size() + 1);
    std::vector<T> t(h.begin(), h.end());
    PK_CUDA(cudaMemcpy(d.p, t.data(), sizeof(T) * t.size(), cudaMemcpyHostToDevice));
}

// The V-list M2L of the MIXED path runs in the shared basis of the 316
// operators (build_m2l_basis) when that cuts the padded tensor-core work by at
// least 30%: rank r at a relative singular value tau = max(30 eps_SVD(FP64),
// 5e-7), below the error the surfaces reach at this p.  PKIFMM_M2L_RANK=0
// keeps the dense operators, a positive value fixes r.  Built once per process
// for each (kernel, p, tau, r).
static std::shared_ptr<const M2LBasis> m2l_basis_for(int kernel, int p, int kn) {
    int over = -1;
    if (const char *e = std::getenv("PKIFMM_M2L_RANK")) over = std::atoi(e);
    if (over == 0) return nullptr;
    const double tau = std::max(30.0 * svd_cut(kernel, p, 0, kn), 5e-7);
    static std::mutex mu;
    static std::map<std::tuple<int, int, double, int>, std::shared_ptr<const M2LBasis>> cache;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(kernel, p, tau, over);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    auto b = std::make_shared<M2LBasis>();
    build_m2l_basis(kernel, p, tau, over > 0 ? over : 0, *b);
    const auto pad = [](int v, int q) { return (long long)((v + q - 1) / q * q); };
    const bool worth = b->r < kn && 10 * pad(b->r, 128) * pad(b->r, 64) <= 7 * pad(kn, 128) * pad(kn, 64);
    std::shared_ptr<const M2LBasis> out = (worth || over > 0) && b->r < kn ? b : nullptr;
    cache[key] = out;
    return out;
}

void upload_operators(Plan &P) {
    HostOps &H = P.host;
    upload(P.g64, H.g);
    upload(P.g32, H.g);
    // M2L offset enumeration and per-class slot tables
    std::vector<int> offs;
    std::vector<int> op_of(343, -1);
    for (int x = -3; x <= 3; x++)
        for (int y = -3; y <= 3; y++)
            for (int z = -3; z <= 3; z++) {
                if (std::max(std::abs(x), std::max(std::abs(y), std::abs(z))) <= 1) continue;
                op_of[((x + 3) * 7 + (y + 3)) * 7 + (z + 3)] = (int)offs.size() / 3;
                offs.push_back(x);
                offs.push_back(y);
                offs.push_back(z);
            }
    std::vector<short> slot_of(8 * 343, -1);
    std::vector<int> cls_op(8 * kVSlots, -1);
    for (int c = 0; c < 8; c++) {
        int cb[3] = {c & 1, c >> 1 & 1, c >> 2 & 1}, s = 0;
        for (int x = -2 - cb[0]; x <= 3 - cb[0]; x++)
            for (int y = -2 - cb[1]; y <= 3 - cb[1]; y++)
                for (int z = -2 - cb[2]; z <= 3 - cb[2]; z++) {
                    if (std::max(std::abs(x), std::max(std::abs(y), std::abs(z))) <= 1) continue;
                    int oi = ((x + 3) * 7 + (y + 3)) * 7 + (z + 3);
                    slot_of[c * 343 + oi] = (short)s;
                    cls_op[c * kVSlots + s] = op_of[oi];
                    s++;
                }
    }
    P.slot_of.reserve(slot_of.size());
    PK_CUDA(cudaMemcpy(P.slot_of.p, slot_of.data(), sizeof(short) * slot_of.size(), cudaMemcpyHostToDevice));
    P.class_slot_op.reserve(cls_op.size());
    PK_CUDA(cudaMemcpy(P.class_slot_op.p, cls_op.data(), sizeof(int) * cls_op.size(), cudaMemcpyHostToDevice));
    P.h_class_slot_op = cls_op;
    DBuf<int> doffs;
    doffs.reserve(offs.size());
    PK_CUDA(cudaMemcpy(doffs.p, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice));

    const size_t kn2 = (size_t)P.kn * P.kn;
    long long tot = (long long)kM2LOps * P.n * P.n;
    if (P.precision == PKIFMM_FP64) {
        upload(P.uc2e_a, H.uc2e_a);
        upload(P.uc2e_b, H.uc2e_b);
        upload(P.dc2e_a, H.dc2e_a);
        upload(P.dc2e_b, H.dc2e_b);
        upload(P.m2m, H.m2m);
        upload(P.l2l, H.l2l);
        P.m2l.reserve(kM2LOps * kn2);
        count_launch(), k_m2l_ops<double><<<nblk(tot, 256), 256>>>(P.kernel, P.n, P.g64.p, doffs.p, P.m2l.p);
    } else {
        // the check-to-equivalent maps stay two factors, (V S+) and U^T: their
        // product has entries of order 1/s_min and would cancel
        // catastrophically in binary32 (the M2M / L2L products include the
        // smoothing kernel matrix and do not)
        upload(P.uc2e_a32, H.uc2e_a);
        upload(P.uc2e_b32, H.uc2e_b);
        upload(P.dc2e_a32, H.dc2e_a);
        upload(P.dc2e_b32, H.dc2e_b);
        upload(P.m2m32, H.m2m);
        upload(P.l2l32, H.l2l);
        (void)tot;
        // the root far field and its solve stay in binary64
        upload(P.dc2e_a, H.dc2e_a);
        upload(P.dc2e_b, H.dc2e_b);
    }
    if (P.periodic) upload(P.root, H.root);
    PK_CUDA(cudaGetLastError());
    PK_CUDA(cudaDeviceSynchronize());
    doffs.release();
    if (P.precision == PKIFMM_MIXED) {
        // the dense translations on the tensor cores; PKIFMM_TRANS_TC=0 keeps the
        // binary32 SIMT GEMM (timing comparisons)
        const char *e = std::getenv("PKIFMM_TRANS_TC");
        const bool tc = !e || std::atoi(e) != 0;
        if (tc) P.basis = m2l_basis_for(P.kernel, P.p, P.kn);
        m2l_tc_prepare(P);
        if (tc) trans_tc_prepare(P);
    }
}

// ---------------- slot GEMM ----------------

// Tiles: FP64 64 x 64 (4 x 4 per thread), FP32 128 x 128 (8 x 8 per thread);
// 256 threads.  Rows of a tile belong to one class, so every row of the tile
// uses the same operator for a given slot.
// Tile configurations of the slot GEMM.  Every configuration accumulates
// each output element in the same order (slot by slot, inputs in order), so
// they give bitwise identical results; the small one only raises parallelism
// for tasks with few rows (the top octree levels).
template <typename T, int BM_, int BN_, int BK_, int TM_, int TN_> struct GemmTile {
    using type = T;
    static constexpr int BM = BM_, BN = BN_, BK = BK_, TM = TM_, TN = TN_;
};
template <typename T> struct GemmCfg;
template <> struct GemmCfg<double> : GemmTile<double, 64, 64, 16, 4, 4> {};
template <> struct GemmCfg<float> : GemmTile<float, 128, 128, 16, 8, 8> {};
template <typename T> using GemmSmall = GemmTile<T, 32, 32, 16, 2, 2>;
constexpr int GB_M = 64;  // tile rows of FP64 tasks

// dst[box][rhs][:] (+)= sum_slots Op[class_ops[cls][s]] src[slot box][rhs][:]
// for one tile of task rows (blockIdx.x) split into sub-tiles of C::BM rows
// (blockIdx.z) and C::BN output components (blockIdx.y).  Global loads of the
// next K step are issued before the current one is multiplied.
template <typename C>
__global__ void __launch_bounds__(256) k_slot_gemm(const int *__restrict__ tboxes, const int4 *__restrict__ tiles,
                                                   const int *__restrict__ slot_table, int slot_stride, int nslots,
                                                   const int *__restrict__ class_ops,
                                                   const typename C::type *__restrict__ ops, long long op_stride,
                                                   const typename C::type *__restrict__ src,
                                                   typename C::type *__restrict__ dst, int kn, int nrhs, int beta) {
    using T = typename C::type;
    constexpr int BM = C::BM, BN = C::BN, BK = C::BK, TM = C::TM, TN = C::TN;
    static_assert(BM == BN && (BM / TM) * (BN / TN) == 256, "256 threads cover the tile");
    constexpr int TX = BN / TN;           // threads along N
    constexpr int LPT = BM * BK / 256;    // A (and B) elements each thread loads per K step
    constexpr int RPT = BK / LPT;         // threads per row for loads
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    __shared__ long long srow[BM], drow[BM];
    __shared__ int sbox[BM];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int4 tile = tiles[blockIdx.x];
    const int cls = tile.x, row0 = tile.y + blockIdx.z * BM, nr = tile.z - blockIdx.z * BM, n0 = blockIdx.y * BN;
    if (nr <= 0) return;
    for (int i = tid; i < BM; i += 256) {
        if (i < nr) {
            int row = row0 + i, tb = row / nrhs, rhs = row % nrhs, box = tboxes[tb];
            drow[i] = (long long)box * nrhs + rhs;
            sbox[i] = box;
        } else {
            drow[i] = -1;
            sbox[i] = -1;
        }
    }
    __syncthreads();
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) acc[i][j] = (T)0;
    const int lm = tid / RPT, lk = (tid % RPT) * LPT;
    const int nn = n0 + lm;
    for (int s = 0; s < nslots; s++) {
        int op = class_ops[cls * nslots + s];
        if (op < 0) continue;
        __syncthreads();
        int any = 0;
        for (int i = tid; i < BM; i += 256) {
            long long sr = -1;
            if (drow[i] >= 0) {
                int b = sbox[i];
                int sb = slot_table ? slot_table[(long long)b * slot_stride + s] : b;
                if (sb >= 0) sr = (long long)sb * nrhs + (drow[i] - (long long)b * nrhs);
            }
            srow[i] = sr;
            any |= sr >= 0;
        }
        if (!__syncthreads_or(any)) continue;
        const T *Op = ops + (long long)op * op_stride;
        const long long sr = srow[lm];
        const T *arow = sr >= 0 ? src + sr * kn : nullptr;
        const T *brow = nn < kn ? Op + (long long)nn * kn : nullptr;
        T ra[LPT], rb[LPT];
#pragma unroll
        for (int q = 0; q < LPT; q++) {
            int kk = lk + q;
            ra[q] = (arow && kk < kn) ? arow[kk] : (T)0;
            rb[q] = (brow && kk < kn) ? brow[kk] : (T)0;
        }
        for (int k0 = 0; k0 < kn; k0 += BK) {
#pragma unroll
            for (int q = 0; q < LPT; q++) {
                As[lk + q][lm] = ra[q];
                Bs[lk + q][lm] = rb[q];
            }
            __syncthreads();
            if (k0 + BK < kn) {
#pragma unroll
                for (int q = 0; q < LPT; q++) {
                    int kk = k0 + BK + lk + q;
                    ra[q] = (arow && kk < kn) ? arow[kk] : (T)0;
                    rb[q] = (brow && kk < kn) ? brow[kk] : (T)0;
                }
            }
#pragma unroll
            for (int kk = 0; kk < BK; kk++) {
                T a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; i++) a[i] = As[kk][ty * TM + i];
#pragma unroll
                for (int j = 0; j < TN; j++) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
                for (int i = 0; i < TM; i++)
#pragma unroll
                    for (int j = 0; j < TN; j++) acc[i][j] += a[i] * b[j];
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < TM; i++) {
        long long dr = drow[ty * TM + i];
        if (dr < 0) continue;
#pragma unroll
        for (int j = 0; j < TN; j++) {
            int nn2 = n0 + tx * TN + j;
            if (nn2 >= kn) continue;
            T *d = dst + dr * kn + nn2;
            *d = beta ? *d + acc[i][j] : acc[i][j];
        }
    }
}

// y[r][i] = sum_j M[i][j] x[r][j] for nrhs vectors (binary64), one warp per row
// (blockIdx.y covers vectors 16 y .. 16 y + 15, e.g. the roots of a batch)
__global__ void k_matvec64(const double *__restrict__ M, const double *__restrict__ x, double *__restrict__ y,
                           int n, int nrhs) {
    int row = blockIdx.x * 8 + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= n) return;
    for (int r = blockIdx.y * 16; r < min(nrhs, (int)blockIdx.y * 16 + 16); r++) {
        double acc = 0;
        for (int j = lane; j < n; j += 32) acc += M[(long long)row * n + j] * x[(long long)r * n + j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[(long long)r * n + row] = acc;
    }
}

static void matvec64(const double *M, const double *x, double *y, int n, int nrhs, cudaStream_t s) {
    if (nrhs <= 0) return;
    count_launch(), k_matvec64<<<dim3((n + 7) / 8, (nrhs + 15) / 16), 256, 0, s>>>(M, x, y, n, nrhs);
}

// ---------------- tasks ----------------

struct HostTree {  // views of the tree read back into pinned host memory
    const int4 *bpos = nullptr;
    const int *child = nullptr, *parent = nullptr;
    const int2 *sr = nullptr, *tr = nullptr;
    bool leaf(int b) const {
        for (int c = 0; c < 8; c++)
            if (child[8 * (size_t)b + c] >= 0) return false;
        return true;
    }
    bool has_src(int b) const { return sr[b].y > sr[b].x; }
    bool has_trg(int b) const { return tr[b].y > tr[b].x; }
    int octant(int b) const { return (bpos[b].x & 1) | (bpos[b].y & 1) << 1 | (bpos[b].z & 1) << 2; }
};

// boxes: per class list of dst boxes
// Host-built task arrays are packed into one pinned buffer and copied with
// one asynchronous copy per array (no stream synchronisation per task).
struct Uploads {
    std::vector<char> pack;
    struct Item {
        void *dst;
        size_t off, bytes;
    };
    std::vector<Item> items;
    template <typename T>
    void add(void *dst, const T *src, size_t n) {
        if (!n) return;
        size_t off = (pack.size() + 15) & ~(size_t)15;
        pack.resize(off + sizeof(T) * n);
        std::memcpy(pack.data() + off, src, sizeof(T) * n);
        items.push_back({dst, off, sizeof(T) * n});
    }
    void flush(Plan &P, cudaStream_t s) {
        if (pack.empty()) return;
        if (P.stage_ev_live) PK_CUDA(cudaEventSynchronize(P.stage_ev));  // the previous copies read the buffer
        if (pack.size() > P.stage_cap) {
            if (P.stage_h) PK_CUDA(cudaFreeHost(P.stage_h));
            P.stage_h = nullptr;
            P.stage_cap = pack.size() + pack.size() / 2;
            PK_CUDA(cudaHostAlloc(&P.stage_h, P.stage_cap, cudaHostAllocDefault));
        }
        std::memcpy(P.stage_h, pack.data(), pack.size());
        for (auto &it : items)
            PK_CUDA(cudaMemcpyAsync(it.dst, P.stage_h + it.off, it.bytes, cudaMemcpyHostToDevice, s));
        if (!P.stage_ev) PK_CUDA(cudaEventCreateWithFlags(&P.stage_ev, cudaEventDisableTiming));
        PK_CUDA(cudaEventRecord(P.stage_ev, s));
        P.stage_ev_live = true;
    }
};

// src (nullable): source box of (box, slot).  With one density vector a tile
// whose source boxes are src0 + i (or src0 + 8 i, the children of consecutive
// parents of a full level) for every slot of its class is marked in .w (1 or 8):
// the tensor-core translations then load its source rows by TMA.
template <typename Src = std::nullptr_t>
static void make_task(Task &t, const std::vector<std::vector<int>> &by_class, int nslots,
                      const std::vector<int> &class_ops, int nrhs, Uploads &up, int bm = GB_M, Src src = nullptr) {
    t.nclass = (int)by_class.size();
    t.nslots = nslots;
    t.h_boxes.clear();
    t.class_count.clear();
    for (auto &v : by_class) t.class_count.push_back((int)v.size());
    std::vector<int4> tiles;
    auto regular = [&](const std::vector<int> &bx, int c, int i0, int n) -> int {
        if constexpr (std::is_same_v<Src, std::nullptr_t>) {
            return 0;
        } else {
            if (nrhs != 1) return 0;
            int stride = 0;
            for (int s = 0; s < nslots; s++) {
                if (class_ops[c * nslots + s] < 0) continue;
                const int a0 = src(bx[i0], s);
                if (a0 < 0) return 0;
                int st = 0;
                if (n > 1) {
                    st = src(bx[i0 + 1], s) - a0;
                    if (st != 1 && st != 8) return 0;
                }
                for (int i = 2; i < n; i++)
                    if (src(bx[i0 + i], s) != a0 + st * i) return 0;
                if (n > 1) {
                    if (stride && st != stride) return 0;
                    stride = st;
                }
            }
            return stride ? stride : 1;
        }
    };
    for (int c = 0; c < t.nclass; c++) {
        int row0 = (int)t.h_boxes.size() * nrhs;
        int nrows = (int)by_class[c].size() * nrhs;
        for (int r = 0; r < nrows; r += bm)
            tiles.push_back(make_int4(c, row0 + r, std::min(bm, nrows - r),
                                      regular(by_class[c], c, r / nrhs, std::min(bm, nrows - r) / nrhs)));
        t.h_boxes.insert(t.h_boxes.end(), by_class[c].begin(), by_class[c].end());
    }
    t.nrows = (int)t.h_boxes.size() * nrhs;
    t.ntiles = (int)tiles.size();
    t.boxes.reserve(t.h_boxes.size() + 1);
    t.tiles.reserve(tiles.size() + 1);
    t.class_ops.reserve(class_ops.size() + 1);
    up.add(t.boxes.p, t.h_boxes.data(), t.h_boxes.size());
    up.add(t.tiles.p, tiles.data(), tiles.size());
    up.add(t.class_ops.p, class_ops.data(), class_ops.size());
}

static void upload_list(DBuf<int> &d, const std::vector<int> &v, Uploads &up) {
    d.reserve(v.size() + 1);
    up.add(d.p, v.data(), v.size());
}

void upward_leaves(Plan &P, cudaStream_t s);

void build_tasks(Plan &P, cudaStream_t s) {
    P.leaves_up = false;
    Tree &t = P.tree;
    int nb = t.nbox;
    // the tree comes back through one pinned buffer (pageable copies are staged
    // by the driver and several times slower)
    const size_t nbz = (size_t)nb;
    const size_t b_bpos = 0, b_child = b_bpos + sizeof(int4) * nbz, b_par = b_child + sizeof(int) * 8 * nbz,
                 b_sr = b_par + sizeof(int) * nbz, b_tr = b_sr + sizeof(int2) * nbz, b_x = b_tr + sizeof(int2) * nbz,
                 b_end = b_x + sizeof(int) * (nbz + 1);
    if (P.stage_ev_live) PK_CUDA(cudaEventSynchronize(P.stage_ev));  // uploads of the last evaluation done
    if (b_end > P.down_cap) {
        if (P.down_h) PK_CUDA(cudaFreeHost(P.down_h));
        P.down_h = nullptr;
        P.down_cap = b_end + b_end / 2;
        PK_CUDA(cudaHostAlloc(&P.down_h, P.down_cap, cudaHostAllocDefault));
    }
    char *dh = P.down_h;
    PK_CUDA(cudaMemcpyAsync(dh + b_bpos, t.bpos.p, sizeof(int4) * nbz, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaMemcpyAsync(dh + b_child, t.child.p, sizeof(int) * 8 * nbz, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaMemcpyAsync(dh + b_par, t.parent.p, sizeof(int) * nbz, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaMemcpyAsync(dh + b_sr, t.srange.p, sizeof(int2) * nbz, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaMemcpyAsync(dh + b_tr, t.trange.p, sizeof(int2) * nbz, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaMemcpyAsync(dh + b_x, t.x_ptr.p, sizeof(int) * (nbz + 1), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    HostTree H;
    H.bpos = (const int4 *)(dh + b_bpos);
    H.child = (const int *)(dh + b_child);
    H.parent = (const int *)(dh + b_par);
    H.sr = (const int2 *)(dh + b_sr);
    H.tr = (const int2 *)(dh + b_tr);
    const int *xptr = (const int *)(dh + b_x);
    P.h_bpos = H.bpos;
    P.h_trange = H.tr;
    Uploads up;
    up.pack.reserve((size_t)nb * 48 + 4096);  // the box lists and tiles below, without regrowth
    const int nr = P.nrhs;
    // per box, in one parallel pass over the read-back tree: bit 0 leaf, bit 1
    // sources, bit 2 targets, bits 3-5 the octant class
    std::vector<unsigned char> fl(nb);
#pragma omp parallel for schedule(static) if (nb > 8192)
    for (int b = 0; b < nb; b++)
        fl[b] = (unsigned char)((H.leaf(b) ? 1 : 0) | (H.has_src(b) ? 2 : 0) | (H.has_trg(b) ? 4 : 0) | H.octant(b) << 3);
    constexpr unsigned char kLeaf = 1, kSrc = 2, kTrg = 4;
    std::vector<int> leaves_src, leaves_trg;
    leaves_src.reserve(nb);
    leaves_trg.reserve(nb);
    t.nleaf = 0;
    for (int b = 0; b < nb; b++) {
        const unsigned char f = fl[b];
        if (!(f & kLeaf)) continue;
        t.nleaf++;
        if (f & kSrc) leaves_src.push_back(b);
        if (f & kTrg) leaves_trg.push_back(b);
    }
    P.n_leaves_src = (int)leaves_src.size();
    P.n_leaves_trg = (int)leaves_trg.size();
    upload_list(P.leaves_src, leaves_src, up);
    upload_list(P.leaves_trg, leaves_trg, up);
    // X-list boxes (with targets and a non-empty X list)
    std::vector<int> xb;
    for (int b = 0; b < nb; b++)
        if (xptr[b + 1] > xptr[b] && (fl[b] & kTrg)) xb.push_back(b);
    P.n_xboxes = (int)xb.size();
    upload_list(P.xboxes, xb, up);
    // the leaf level of the upward pass runs on the device while the host
    // groups the other tasks (the second flush waits for these copies only)
    up.flush(P, s);
    upward_leaves(P, s);
    Uploads up2;
    up2.pack.reserve((size_t)nb * 40 + 4096);

    bool mixed = P.precision == PKIFMM_MIXED;
    const int bm = mixed ? GemmCfg<float>::BM : GemmCfg<double>::BM;
    // UC2E over leaves with sources
    const auto self = [](int b, int) { return b; };
    make_task(P.t_uc2e, {leaves_src}, 1, {0}, nr, up2, bm, self);
    // M2M per level: non-leaf boxes with sources
    int depth = (int)t.lvl_begin.size() - 1;
    P.t_m2m.resize(depth);
    std::vector<int> ops8(8);
    for (int c = 0; c < 8; c++) ops8[c] = c;
    for (int l = 0; l < depth; l++) {
        std::vector<int> v;
        for (int b = t.lvl_begin[l]; b < t.lvl_begin[l + 1]; b++)
            if ((fl[b] & (kLeaf | kSrc)) == kSrc) v.push_back(b);
        make_task(P.t_m2m[l], {v}, 8, ops8, nr, up2, bm, [&](int b, int sl) { return H.child[8 * (size_t)b + sl]; });
    }
    // M2L: boxes of level >= 1 with targets, by octant class
    std::vector<std::vector<int>> byc(8);
    for (int b = P.nprob; b < nb; b++)  // boxes 0..nprob-1 are the problems' roots
        if (fl[b] & kTrg) byc[fl[b] >> 3].push_back(b);
    make_task(P.t_m2l, byc, kVSlots, P.h_class_slot_op, nr, up2, bm);
    // DC2E over boxes with targets (roots separately in binary64 for MIXED)
    std::vector<int> dc;
    dc.reserve(nb);
    for (int b = (mixed ? P.nprob : 0); b < nb; b++)
        if (fl[b] & kTrg) dc.push_back(b);
    make_task(P.t_dc2e, {dc}, 1, {0}, nr, up2, bm, self);
    // MIXED with a shared M2L basis: the X-list part of the check potential is solved separately
    if (P.basis) make_task(P.t_dcx, {xb}, 1, {0}, nr, up2, bm, self);
    // L2L per level >= 1, by octant class
    P.t_l2l.resize(depth);
    for (int l = 1; l < depth; l++) {
        std::vector<std::vector<int>> bc(8);
        for (int b = t.lvl_begin[l]; b < t.lvl_begin[l + 1]; b++)
            if (fl[b] & kTrg) bc[fl[b] >> 3].push_back(b);
        make_task(P.t_l2l[l], bc, 1, ops8, nr, up2, bm, [&](int b, int) { return H.parent[b]; });
    }
    up2.flush(P, s);
}

// Large binary32 slot GEMM: a 128 x 128 output tile per CTA, 16 K per step,
// shared memory double-buffered, next step's global loads in registers while
// the current one is multiplied, 16-byte loads where rows allow.  Each thread
// owns rows {4 ty + i, 64 + 4 ty + i} and columns {4 tx + j, 64 + 4 tx + j}
// (i, j < 4), read as float4 from shared memory without bank conflicts.  The
// slots with a source in the tile are listed first and walked as one K
// sequence; every output element is accumulated slot by slot, inputs in
// order, exactly as in k_slot_gemm.
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 16;
constexpr int SG_MAX_SLOTS = 256;

__global__ void __launch_bounds__(256) k_slot_gemm_f32(const int *__restrict__ tboxes, const int4 *__restrict__ tiles,
                                                       const int *__restrict__ slot_table, int slot_stride, int nslots,
                                                       const int *__restrict__ class_ops, const float *__restrict__ ops,
                                                       long long op_stride, const float *__restrict__ src,
                                                       float *__restrict__ dst, int kn, int nrhs, int beta) {
    __shared__ __align__(16) float As[2][SG_BK][SG_BM];
    __shared__ __align__(16) float Bs[2][SG_BK][SG_BN];
    __shared__ long long drow[SG_BM];
    __shared__ int sbox[SG_BM];
    __shared__ short act[SG_MAX_SLOTS];
    __shared__ int nact_s;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int4 tile = tiles[blockIdx.x];
    const int cls = tile.x, row0 = tile.y, nr = tile.z, n0 = blockIdx.y * SG_BN;
    for (int i = tid; i < SG_BM; i += 256) {
        if (i < nr) {
            int row = row0 + i, tb = row / nrhs, rhs = row % nrhs, box = tboxes[tb];
            drow[i] = (long long)box * nrhs + rhs;
            sbox[i] = box;
        } else {
            drow[i] = -1;
            sbox[i] = -1;
        }
    }
    __syncthreads();
    for (int sl = tid; sl < nslots; sl += 256) {
        int any = 0;
        if (class_ops[cls * nslots + sl] >= 0)
            for (int i = 0; i < nr && !any; i++)
                any = !slot_table || slot_table[(long long)sbox[i] * slot_stride + sl] >= 0;
        act[sl] = (short)any;
    }
    __syncthreads();
    if (tid == 0) {
        int c = 0;
        for (int sl = 0; sl < nslots; sl++)
            if (act[sl]) act[c++] = (short)sl;
        nact_s = c;
    }
    __syncthreads();
    const int nk = (kn + SG_BK - 1) / SG_BK, total = nact_s * nk;
    const bool vec = (kn & 3) == 0;
    // loader: row lm of A (and of B), 8 consecutive k from lk
    const int lm = tid >> 1, lk = (tid & 1) * 8;
    const int my_box = sbox[lm];
    const long long my_rhs = drow[lm] >= 0 ? drow[lm] - (long long)my_box * nrhs : 0;
    const int nn = n0 + lm;
    float ra[8], rb[8];
    auto load = [&](int it) {
        const int sl = act[it / nk], k0 = (it % nk) * SG_BK + lk;
        const int op = class_ops[cls * nslots + sl];
        const float *arow = nullptr;
        if (my_box >= 0) {
            const int sb = slot_table ? slot_table[(long long)my_box * slot_stride + sl] : my_box;
            if (sb >= 0) arow = src + ((long long)sb * nrhs + my_rhs) * kn;
        }
        const float *brow = nn < kn ? ops + (long long)op * op_stride + (long long)nn * kn : nullptr;
        if (vec && k0 + 8 <= kn) {
            if (arow) {
                float4 u = *reinterpret_cast<const float4 *>(arow + k0), v = *reinterpret_cast<const float4 *>(arow + k0 + 4);
                ra[0] = u.x; ra[1] = u.y; ra[2] = u.z; ra[3] = u.w; ra[4] = v.x; ra[5] = v.y; ra[6] = v.z; ra[7] = v.w;
            } else {
#pragma unroll
                for (int q = 0; q < 8; q++) ra[q] = 0.f;
            }
            if (brow) {
                float4 u = *reinterpret_cast<const float4 *>(brow + k0), v = *reinterpret_cast<const float4 *>(brow + k0 + 4);
                rb[0] = u.x; rb[1] = u.y; rb[2] = u.z; rb[3] = u.w; rb[4] = v.x; rb[5] = v.y; rb[6] = v.z; rb[7] = v.w;
            } else {
#pragma unroll
                for (int q = 0; q < 8; q++) rb[q] = 0.f;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; q++) {
                ra[q] = (arow && k0 + q < kn) ? arow[k0 + q] : 0.f;
                rb[q] = (brow && k0 + q < kn) ? brow[k0 + q] : 0.f;
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 8; q++) {
            As[buf][lk + q][lm] = ra[q];
            Bs[buf][lk + q][lm] = rb[q];
        }
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0.f;
    if (total > 0) {
        load(0);
        store(0);
        __syncthreads();
        for (int it = 0; it < total; it++) {
            const int buf = it & 1;
            if (it + 1 < total) load(it + 1);
#pragma unroll
            for (int kk = 0; kk < SG_BK; kk++) {
                float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][4 * ty]);
                float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + 4 * ty]);
                float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][4 * tx]);
                float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + 4 * tx]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; i++)
#pragma unroll
                    for (int j = 0; j < 8; j++) acc[i][j] += a[i] * b[j];
            }
            if (it + 1 < total) store(buf ^ 1);
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int m = (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
        const long long dr = drow[m];
        if (dr < 0) continue;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int c = n0 + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
            if (c >= kn) continue;
            float *d = dst + dr * kn + c;
            *d = beta ? *d + acc[i][j] : acc[i][j];
        }
    }
}

template <typename T>
static void gemm(const Task &t, const int *slot_table, int slot_stride, const T *ops, long long op_stride,
                 const T *src, T *dst, int kn, int nrhs, int beta, cudaStream_t s) {
    if (t.ntiles == 0) return;
    using Big = GemmCfg<T>;
    using Small = GemmSmall<T>;
    const int bm = std::is_same<T, float>::value ? Big::BM : GB_M;  // rows per task tile (make_task)
    const long long big_blocks = (long long)t.ntiles * ((kn + Big::BN - 1) / Big::BN) * ((bm + Big::BM - 1) / Big::BM);
    if (big_blocks < 152 / 2) {  // fewer large tiles than half the SMs
        dim3 g(t.ntiles, (kn + Small::BN - 1) / Small::BN, (bm + Small::BM - 1) / Small::BM);
        count_launch(), k_slot_gemm<Small><<<g, 256, 0, s>>>(t.boxes.p, t.tiles.p, slot_table, slot_stride, t.nslots,
                                                              t.class_ops.p, ops, op_stride, src, dst, kn, nrhs, beta);
        return;
    }
    dim3 grid(t.ntiles, (kn + Big::BN - 1) / Big::BN, (bm + Big::BM - 1) / Big::BM);
    if constexpr (std::is_same<T, float>::value) {
        static_assert(Big::BM == SG_BM && Big::BN == SG_BN, "binary32 tiles");
        if (t.nslots <= SG_MAX_SLOTS) {
            count_launch(), k_slot_gemm_f32<<<grid, 256, 0, s>>>(t.boxes.p, t.tiles.p, slot_table, slot_stride, t.nslots,
                                                                  t.class_ops.p, ops, op_stride, src, dst, kn, nrhs, beta);
            return;
        }
    }
    count_launch(), k_slot_gemm<Big><<<grid, 256, 0, s>>>(t.boxes.p, t.tiles.p, slot_table, slot_stride, t.nslots,
                                                          t.class_ops.p, ops, op_stride, src, dst, kn, nrhs, beta);
}

// ---------------- kernel sums ----------------

template <typename T>
struct alignas(4 * sizeof(T)) V4 { T x, y, z, w; };  // one 16-byte (binary32) access

// 1/sqrt(r2) for a normal r2 > 0: binary32 by the PTX approximate reciprocal
// square root (relative error below 2^-22.9, subnormal inputs flushed),
// binary64 by a correctly rounded square root and division
__device__ __forceinline__ float rsqrt_nz(float r2) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
    return y;
}
__device__ __forceinline__ double rsqrt_nz(double r2) { return 1.0 / sqrt(r2); }
// smallest normal number of each type
__device__ __forceinline__ float tiny_normal(float) { return 1.17549435e-38f; }
__device__ __forceinline__ double tiny_normal(double) { return 2.2250738585072014e-308; }

// How a kernel sum treats the distance r of a pair:
//   kFar   r > 0 known (equivalent and check surfaces, distinct boxes' surfaces);
//   kSelf  a source may coincide with the target: r below the smallest
//          normal number drops the pair (the self-interaction is excluded);
//   kNear  distinct points of different boxes: r^2 is clamped to the
//          smallest normal number, so a pair that rounding made coincide
//          stays finite.
enum PairMode { kFar = 0, kSelf = 1, kNear = 2 };
template <int MODE, typename T>
__device__ __forceinline__ T inv_r(T r2) {
    if constexpr (MODE == kSelf) return r2 >= tiny_normal(r2) ? rsqrt_nz(r2) : (T)0;
    else if constexpr (MODE == kNear) return rsqrt_nz(fmax(r2, tiny_normal(r2)));
    else return rsqrt_nz(r2);
}

__device__ __forceinline__ double exp2i(int l) { return ldexp(1.0, -l); }

// leaf-relative coordinates: rel[i] = x[i] - centre(leaf)
template <typename T>
__global__ void k_relcoords(const int *__restrict__ leaves, const int4 *__restrict__ bpos,
                            const int2 *__restrict__ range, const double *__restrict__ x, V4<T> *__restrict__ rel) {
    int b = leaves[blockIdx.x];
    int4 p = bpos[b];
    double h = exp2i(p.w), c[3] = {(p.x + 0.5) * h, (p.y + 0.5) * h, (p.z + 0.5) * h};
    int2 r = range[b];
    for (int i = r.x + threadIdx.x; i < r.y; i += blockDim.x) {
        V4<T> v;
        v.x = (T)(x[3 * (long long)i] - c[0]);
        v.y = (T)(x[3 * (long long)i + 1] - c[1]);
        v.z = (T)(x[3 * (long long)i + 2] - c[2]);
        v.w = (T)0;
        rel[i] = v;
    }
}

template <typename T>
__global__ void k_cast(const double *__restrict__ a, T *__restrict__ b, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (T)a[i];
}

constexpr int KS_T = 128;  // threads of the kernel-sum blocks

template <typename T, int K, int R, int KT = K, int KS = K>
struct LeafAcc {
    // Sums without the kernel's constant factor (1 for Laplace, 1/8pi for
    // Stokes), applied once to each result (scale()).  KT target components:
    // K for the kernel itself; 4 for the Laplace field (K = 1): the potential
    // and its gradient at the target, grad(1/r) = -d/r^3.  KS components of
    // a source (add_src): K, or 3 for Laplace dipoles (K = 1): f.d/r^3, the
    // potential f.grad_y(1/|x - y|) of a dipole f at y.
    static_assert(KT == K || (K == 1 && KT == 4), "target components");
    static_assert(KS == K || (K == 1 && KS == 3 && KT == 1), "source components");
    T acc[R][KT], tot[R][KT], cmp[R][KT];
    static constexpr double kScale = K == 1 ? 1.0 : 0.039788735772973836;  // 1/(8 pi)
    __device__ void init() {
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int a = 0; a < KT; a++) acc[r][a] = tot[r][a] = cmp[r][a] = 0;
    }
    __device__ void flush() {
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int a = 0; a < KT; a++) {
                T y = acc[r][a] - cmp[r][a], s = tot[r][a] + y;
                cmp[r][a] = (s - tot[r][a]) - y;
                tot[r][a] = s;
                acc[r][a] = 0;
            }
    }
    // one source at offset d = x - y with densities f[r][a]; MODE: PairMode
    template <int MODE>
    __device__ __forceinline__ void add(T dx, T dy, T dz, const T (*f)[K]) {
        const T r2 = dx * dx + dy * dy + dz * dz;
        const T ir = inv_r<MODE>(r2);
        if constexpr (KT == 4) {
            const T ir3 = ir * ir * ir;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const T q = f[r][0], qi3 = q * ir3;
                acc[r][0] += ir * q;
                acc[r][1] -= dx * qi3;
                acc[r][2] -= dy * qi3;
                acc[r][3] -= dz * qi3;
            }
        } else if constexpr (K == 1) {
#pragma unroll
            for (int r = 0; r < R; r++) acc[r][0] += ir * f[r][0];
        } else {
            // (I/r + d d^T/r^3) f = (f + d (f.d)/r^2) / r
            const T ir2 = ir * ir;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const T t = (f[r][0] * dx + f[r][1] * dy + f[r][2] * dz) * ir2;
                acc[r][0] += ir * (f[r][0] + dx * t);
                acc[r][1] += ir * (f[r][1] + dy * t);
                acc[r][2] += ir * (f[r][2] + dz * t);
            }
        }
    }
    // one source of the source kernel (KS components) at offset d = x - y
    template <int MODE>
    __device__ __forceinline__ void add_src(T dx, T dy, T dz, const T (*f)[KS]) {
        if constexpr (KS == K) {
            add<MODE>(dx, dy, dz, f);
        } else {
            const T r2 = dx * dx + dy * dy + dz * dz;
            const T ir = inv_r<MODE>(r2);
            const T ir3 = ir * ir * ir;
#pragma unroll
            for (int r = 0; r < R; r++) acc[r][0] += (f[r][0] * dx + f[r][1] * dy + f[r][2] * dz) * ir3;
        }
    }
};

template <typename T, int K, int R, int KS = K>
__global__ void __launch_bounds__(KS_T) k_s2m(const int *__restrict__ leaves, const int4 *__restrict__ bpos,
                                              const int2 *__restrict__ srange, const V4<T> *__restrict__ yrel,
                                              const T *__restrict__ dens, int nrhs, int rhs0,
                                              const T *__restrict__ g, int n, T *__restrict__ chk) {
    __shared__ V4<T> sy[KS_T];
    __shared__ T sphi[KS_T][R][KS];
    const int b = leaves[blockIdx.x];
    const int4 p = bpos[b];
    const T h = (T)exp2i(p.w), sc = (T)1.475 * h;
    const int2 r = srange[b];
    const int kn = n * K, nv = min(R, nrhs - rhs0);
    for (int i0 = 0; i0 < n; i0 += KS_T) {
        int i = i0 + threadIdx.x;
        T x0 = 0, x1 = 0, x2 = 0;
        if (i < n) {
            x0 = sc * g[3 * i];
            x1 = sc * g[3 * i + 1];
            x2 = sc * g[3 * i + 2];
        }
        LeafAcc<T, K, R, K, KS> L;
        L.init();
        for (int s0 = r.x; s0 < r.y; s0 += KS_T) {
            __syncthreads();
            int sidx = s0 + threadIdx.x;
            if (sidx < r.y) {
                sy[threadIdx.x] = yrel[sidx];
#pragma unroll
                for (int q = 0; q < R; q++)
#pragma unroll
                    for (int a = 0; a < KS; a++)
                        sphi[threadIdx.x][q][a] = q < nv ? dens[(long long)sidx * nrhs * KS + (rhs0 + q) * KS + a] : (T)0;
            }
            __syncthreads();
            int m = min(KS_T, r.y - s0);
            for (int j = 0; j < m; j++) {
                const V4<T> y = sy[j];
                L.template add_src<kFar>(x0 - y.x, x1 - y.y, x2 - y.z, sphi[j]);
            }
        }
        if (i < n) {
#pragma unroll
            for (int q = 0; q < R; q++)
                if (q < nv)
#pragma unroll
                    for (int a = 0; a < K; a++)
                        chk[((long long)b * nrhs + rhs0 + q) * kn + i * K + a] = h * (T)LeafAcc<T, K, R>::kScale * L.acc[q][a];
        }
    }
}

__device__ __forceinline__ void decode_shift(unsigned char c, int sh[3]) {
    sh[0] = c / 9 - 1;
    sh[1] = (c / 3) % 3 - 1;
    sh[2] = c % 3 - 1;
}

// offset (c_B - c_A - p) between box centres, exact dyadic
__device__ __forceinline__ void centre_offset(int4 B, int4 A, const int sh[3], double off[3]) {
    double hb = exp2i(B.w), ha = exp2i(A.w);
    off[0] = (B.x + 0.5) * hb - (A.x + 0.5) * ha - sh[0];
    off[1] = (B.y + 0.5) * hb - (A.y + 0.5) * ha - sh[1];
    off[2] = (B.z + 0.5) * hb - (A.z + 0.5) * ha - sh[2];
}

// X list: q~d[B][rhs][i] += h_B sum_{(A,p) in X(B)} sum_{s in A} K(0.525 h_B g_i - yrel_s + off) phi_s,
// for the boxes B holding more targets than a surface has points; the targets of
// the others take X(B)'s sources directly in the leaf kernel (exact, and cheaper)
template <typename T, int K, int R, int KS = K>
__global__ void __launch_bounds__(KS_T) k_s2l(const int *__restrict__ boxes, const int4 *__restrict__ bpos,
                                              const int2 *__restrict__ srange, const int2 *__restrict__ trange,
                                              const int *__restrict__ xptr,
                                              const int *__restrict__ xbox, const unsigned char *__restrict__ xsh,
                                              const V4<T> *__restrict__ yrel, const T *__restrict__ dens, int nrhs,
                                              int rhs0, const T *__restrict__ g, int n, T *__restrict__ chk) {
    __shared__ V4<T> sy[KS_T];
    __shared__ T sphi[KS_T][R][KS];
    const int b = boxes[blockIdx.x];
    if (trange[b].y - trange[b].x <= n) return;  // block-uniform
    const int4 B = bpos[b];
    const T h = (T)exp2i(B.w), sc = (T)0.525 * h;
    const int kn = n * K, nv = min(R, nrhs - rhs0);
    for (int i0 = 0; i0 < n; i0 += KS_T) {
        int i = i0 + threadIdx.x;
        T x0 = 0, x1 = 0, x2 = 0;
        if (i < n) {
            x0 = sc * g[3 * i];
            x1 = sc * g[3 * i + 1];
            x2 = sc * g[3 * i + 2];
        }
        LeafAcc<T, K, R, K, KS> L;
        L.init();
        for (int e = xptr[b]; e < xptr[b + 1]; e++) {
            int A = xbox[e], sh[3];
            decode_shift(xsh[e], sh);
            double off[3];
            centre_offset(B, bpos[A], sh, off);
            const T xo0 = x0 + (T)off[0], xo1 = x1 + (T)off[1], xo2 = x2 + (T)off[2];
            int2 r = srange[A];
            for (int s0 = r.x; s0 < r.y; s0 += KS_T) {
                __syncthreads();
                int sidx = s0 + threadIdx.x;
                if (sidx < r.y) {
                    sy[threadIdx.x] = yrel[sidx];
#pragma unroll
                    for (int q = 0; q < R; q++)
#pragma unroll
                        for (int a = 0; a < KS; a++)
                            sphi[threadIdx.x][q][a] =
                                q < nv ? dens[(long long)sidx * nrhs * KS + (rhs0 + q) * KS + a] : (T)0;
                }
                __syncthreads();
                int m = min(KS_T, r.y - s0);
                for (int j = 0; j < m; j++) {
                    const V4<T> y = sy[j];
                    L.template add_src<kFar>(xo0 - y.x, xo1 - y.y, xo2 - y.z, sphi[j]);
                }
            }
        }
        if (i < n) {
#pragma unroll
            for (int q = 0; q < R; q++)
                if (q < nv)
#pragma unroll
                    for (int a = 0; a < K; a++)
                        chk[((long long)b * nrhs + rhs0 + q) * kn + i * K + a] += h * (T)LeafAcc<T, K, R>::kScale * L.acc[q][a];
        }
    }
}

// Kernel sums at a target leaf B for up to R density vectors at once (the
// geometry and 1/r are shared): L2T from B's downward equivalent surface,
// M2T from the upward equivalent surfaces of W(B), the U-list direct sums with
// the periodic images (the near field of Sec. 2.2), and the direct sums that
// replace a surface where that is cheaper: W boxes with at most n sources, and
// the X lists of B and its ancestors holding at most n targets (k_s2l skips
// those boxes).
// One warp per block; blockIdx.y takes chunks of at most (32 / G) QMAX
// targets.  The warp's G groups of lanes split each staged tile of LT sources
// (slot j to group j mod G) over the same targets, Q targets per lane in
// registers, so one shared load of a source serves Q pairs; the groups' sums
// are added at the end.  The sources of every box of a list are staged already
// moved into B's frame (y + p - c_B), so a tile runs across box boundaries, and
// the global loads of the next tile are in flight while the current one is
// summed.  Each tile's sum joins the running total with Kahan compensation.

// blocks per SM the register budget is sized for: 24 (85 registers a thread)
// for one binary32 sum a target from one-component sources, 16 (128 registers)
// for up to 3, else 8 (measured: Laplace at 24 blocks 18% faster than at 16,
// Stokes slower at 20)
template <typename T, int R, int KT, int KS>
constexpr int leaf_min_blocks() {
    return sizeof(T) == 4 && R * KT <= 1 && KS == 1 ? 24 : (sizeof(T) == 4 && R * KT <= 3 ? 16 : 8);
}

template <typename T, int K, int R, int QMAX, int G, int KT, int KS = K>
__global__ void __launch_bounds__(32, (leaf_min_blocks<T, R, KT, KS>())) k_leaf(
    const int *__restrict__ leaves, const int4 *__restrict__ bpos, const int2 *__restrict__ srange,
    const int2 *__restrict__ trange, const int *__restrict__ uptr, const int *__restrict__ ubox,
    const unsigned char *__restrict__ ush, const int *__restrict__ wptr, const int *__restrict__ wbox,
    const unsigned char *__restrict__ wsh, const int *__restrict__ parent, const int *__restrict__ xptr,
    const int *__restrict__ xbox, const unsigned char *__restrict__ xsh, const V4<T> *__restrict__ yrel,
    const V4<T> *__restrict__ xrel, const T *__restrict__ dens, const double *__restrict__ xsrc, const T *__restrict__ up,
    const T *__restrict__ dn, int nrhs, int rhs0, const T *__restrict__ g, int n, double *__restrict__ pot) {
    using Acc = LeafAcc<T, K, R, KT, KS>;
    // sources per staged tile (LT / 32 per lane): 32 for Laplace (measured 11%
    // faster than 64: fewer prefetch registers, more warps), 64 for Stokes
    constexpr int LT = K == 1 ? 32 : 64;
    constexpr int ND = R * (K > KS ? K : KS);  // densities of a staged source
    constexpr int EP = ND & ~1 ? ND & ~1 : 1;   // beyond the first (in the fourth lane), padded to even
    __shared__ V4<T> sy[LT];
    __shared__ __align__(16) T sd[LT][EP];
    __shared__ int s_start[33], s_idx[32];
    __shared__ V4<T> s_off[32];
    __shared__ int s_xbeg[24], s_xpre[25], s_nx;  // X lists summed here: their first entries, prefix
    constexpr int LW = 32 / G;  // lanes of a source group
    const int lane = threadIdx.x, grp = lane / LW, lg = lane % LW;
    const int b = leaves[blockIdx.x];
    const int4 B = bpos[b];
    const double hB = exp2i(B.w);
    const int2 tr = trange[b];
    const int kn = n * K, nv = min(R, nrhs - rhs0);
    const int u0 = uptr[b], nu = uptr[b + 1] - u0, w0 = wptr[b], nw = wptr[b + 1] - w0;
    const T pad = (T)(4.0 * hB);  // a staged slot past the end: zero density, far from every target of B
    if (tr.x + (int)blockIdx.y * (32 / G) * QMAX >= tr.y) return;  // no targets in this block's chunks
    // the X lists of B and its ancestors whose box holds no more targets than a
    // surface has points (k_s2l leaves those out): at most 22 levels of boxes
    if (lane == 0) {
        int k = 0, tot = 0;
        for (int Bx = b; Bx >= 0 && k < 24; Bx = parent[Bx]) {
            const int x0 = xptr[Bx], x1 = xptr[Bx + 1];
            if (x1 == x0) continue;
            const int2 tb = trange[Bx];
            if (tb.y - tb.x <= n) {
                s_xbeg[k] = x0;
                s_xpre[k] = tot;
                tot += x1 - x0;
                k++;
            }
        }
        s_xpre[k] = tot;
        s_nx = k;
    }
    __syncwarp();
    const int nxa = s_nx, nx = s_xpre[nxa];

    // one chunk of at most LW QMAX targets, nq = ceil(targets / LW) of the Q
    // slots of a lane in use (the tile sums are compiled for each nq)
    auto chunk = [&](int t0, int nq) {
        constexpr int Q = QMAX;
        T xs[Q][3];
#pragma unroll
        for (int q = 0; q < Q; q++) {
            const int t = t0 + lg + LW * q;
            xs[q][0] = xs[q][1] = xs[q][2] = 0;
            if (t < tr.y) {
                const V4<T> v = xrel[t];
                xs[q][0] = v.x;
                xs[q][1] = v.y;
                xs[q][2] = v.z;
            }
        }
        Acc L[Q];
#pragma unroll
        for (int q = 0; q < Q; q++) L[q].init();

        // F staged sources of one list; fetch(f, y, d) reads source f of the
        // list in B's frame with its densities d[r * CP + a]
        auto run = [&](auto mode_tag, auto u_tag, int F, auto fetch) {
            constexpr int MODE = decltype(mode_tag)::value;
            constexpr bool U = decltype(u_tag)::value;
            constexpr int CP = U ? KS : K, NP = R * CP;
            V4<T> ry[LT / 32];
            T rd[LT / 32][NP];
            auto load = [&](int base) {
#pragma unroll
                for (int s = 0; s < LT / 32; s++) {
                    const int f = base + lane + 32 * s;
                    if (f < F) fetch(f, ry[s], rd[s]);
                }
            };
            load(0);
            for (int base = 0; base < F; base += LT) {
                const int m = min(LT, F - base);
                __syncwarp();
#pragma unroll
                for (int s = 0; s < LT / 32; s++) {
                    const int j = lane + 32 * s;
                    if (j < m) {
                        V4<T> y = ry[s];
                        y.w = rd[s][0];
                        sy[j] = y;
#pragma unroll
                        for (int i = 1; i < NP; i++) sd[j][i - 1] = rd[s][i];
                    } else if (j < (m + G - 1) / G * G) {
                        sy[j] = V4<T>{pad, pad, pad, (T)0};
#pragma unroll
                        for (int i = 1; i < NP; i++) sd[j][i - 1] = (T)0;
                    }
                }
                __syncwarp();
                if (base + LT < F) load(base + LT);
                const int n2 = (m + G - 1) / G;
                auto sum_tile = [&](auto nq_tag) {
                    constexpr int NQ = decltype(nq_tag)::value;
#pragma unroll 2
                    for (int i = 0; i < n2; i++) {
                        const int j = G * i + grp;
                        const V4<T> y = sy[j];
                        T f[R][CP];
                        f[0][0] = y.w;
#pragma unroll
                        for (int k = 1; k < NP; k++) f[k / CP][k % CP] = sd[j][k - 1];
#pragma unroll
                        for (int q = 0; q < NQ; q++) {
                            if constexpr (U)
                                L[q].template add_src<MODE>(xs[q][0] - y.x, xs[q][1] - y.y, xs[q][2] - y.z, f);
                            else
                                L[q].template add<MODE>(xs[q][0] - y.x, xs[q][1] - y.y, xs[q][2] - y.z, f);
                        }
                    }
                };
                if (nq <= 1) sum_tile(std::integral_constant<int, 1>{});
                else if (nq == 2) sum_tile(std::integral_constant<int, (Q < 2 ? Q : 2)>{});
                else if (nq == 3) sum_tile(std::integral_constant<int, (Q < 3 ? Q : 3)>{});
                else sum_tile(std::integral_constant<int, Q>{});
#pragma unroll
                for (int q = 0; q < Q; q++) L[q].flush();
            }
        };

        // entry table of a chunk of up to 32 list entries, one per lane: the
        // exclusive prefix of the entries' source counts, their first index and
        // offset; returns the chunk's source count
        auto publish = [&](int cnt, int idx, V4<T> o) {
            int inc = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += v;
            }
            const int F = __shfl_sync(0xffffffffu, inc, 31);
            __syncwarp();  // the last chunk's sources are all staged
            s_start[lane] = inc - cnt;
            s_idx[lane] = idx;
            s_off[lane] = o;
            if (lane == 31) s_start[32] = inc;
            __syncwarp();
            return F;
        };
        auto entry_of = [&](int f) {  // the last entry starting at or before f
            int ei = 0;
#pragma unroll
            for (int st = 16; st; st >>= 1)
                if (s_start[ei + st] <= f) ei += st;
            return ei;
        };
        // a W box holding no more sources than a surface has points is summed
        // from its sources (exactly, and at no more cost) instead of its
        // upward equivalent surface
        auto w_direct = [&](int A) {
            const int2 rg = srange[A];
            return rg.y - rg.x <= n;
        };

        // L2T and W: n points of an equivalent surface per entry; entry 0 is
        // B's downward surface (half-width 1.475 h_B), entry e > 0 the upward
        // surface (half-width 0.525 h_A) of the W box e - 1, moved into B's frame
        for (int c0 = 0; c0 < 1 + nw; c0 += 32) {
            const int e = c0 + lane;
            int cnt = 0, idx = 0;
            V4<T> o{(T)0, (T)0, (T)0, (T)0};
            if (e == 0) {
                cnt = n;
                idx = -1 - b;
                o.w = (T)(1.475 * hB);
            } else if (e < 1 + nw) {
                const int A = wbox[w0 + e - 1];
                if (!w_direct(A)) {
                    int sh[3];
                    decode_shift(wsh[w0 + e - 1], sh);
                    const int4 Ap = bpos[A];
                    double off[3];
                    centre_offset(B, Ap, sh, off);
                    cnt = n;
                    idx = A;
                    o = V4<T>{(T)off[0], (T)off[1], (T)off[2], (T)(0.525 * exp2i(Ap.w))};
                }
            }
            const int F = publish(cnt, idx, o);
            run(std::integral_constant<int, kFar>{}, std::false_type{}, F, [&](int f, V4<T> &y, T(&d)[R * K]) {
                const int ei = nw ? entry_of(f) : 0, j = f - s_start[ei], id = s_idx[ei];  // one entry: no search
                const V4<T> oe = s_off[ei];
                const T *phi = id < 0 ? dn + ((long long)(-1 - id) * nrhs + rhs0) * kn
                                      : up + ((long long)id * nrhs + rhs0) * kn;
                y.x = oe.w * g[3 * j] - oe.x;
                y.y = oe.w * g[3 * j + 1] - oe.y;
                y.z = oe.w * g[3 * j + 2] - oe.z;
#pragma unroll
                for (int r = 0; r < R; r++)
#pragma unroll
                    for (int a = 0; a < K; a++) d[r * K + a] = r < nv ? phi[(long long)r * kn + j * K + a] : (T)0;
            });
        }

        // U list: B itself (coincident points drop out), then the adjacent
        // leaves and images, read relative to their leaf's centre (offset
        // c_B - c_A - p); the entries of a chunk are laid end to end
        auto u_list = [&](auto mode_tag, bool self) {
            for (int c0 = 0; c0 < nu; c0 += 32) {
                const int e = c0 + lane;
                int cnt = 0, i0 = 0;
                V4<T> o{(T)0, (T)0, (T)0, (T)0};
                if (e < nu) {
                    const int A = ubox[u0 + e];
                    const unsigned char code = ush[u0 + e];
                    if ((A == b && code == 13) == self) {  // code 13: shift (0, 0, 0)
                        const int2 rg = srange[A];
                        cnt = rg.y - rg.x;
                        i0 = rg.x;
                        int sh[3];
                        decode_shift(code, sh);
                        double off[3];
                        centre_offset(B, bpos[A], sh, off);
                        o = V4<T>{(T)off[0], (T)off[1], (T)off[2], (T)0};
                    }
                }
                const int F = publish(cnt, i0, o);
                run(mode_tag, std::true_type{}, F, [&](int f, V4<T> &y, T(&d)[R * KS]) {
                    const int ei = entry_of(f), i = s_idx[ei] + f - s_start[ei];
                    const V4<T> oe = s_off[ei], v = yrel[i];
                    y.x = v.x - oe.x;
                    y.y = v.y - oe.y;
                    y.z = v.z - oe.z;
#pragma unroll
                    for (int r = 0; r < R; r++)
#pragma unroll
                        for (int a = 0; a < KS; a++)
                            d[r * KS + a] = r < nv ? dens[(long long)i * nrhs * KS + (rhs0 + r) * KS + a] : (T)0;
                });
            }
        };
        u_list(std::integral_constant<int, kSelf>{}, true);
        u_list(std::integral_constant<int, kNear>{}, false);

        // the W boxes and X lists summed from their sources, read from their
        // binary64 coordinates (a W box may span several leaves) moved by the
        // image shift p into B's frame (a pass of its own, so that the U
        // pass's code stays lean)
        for (int c0 = 0; c0 < nw + nx; c0 += 32) {
            const int e = c0 + lane;
            int cnt = 0, i0 = 0;
            V4<T> o{(T)0, (T)0, (T)0, (T)0};
            int xi = -1;
            if (e < nw) {
                if (w_direct(wbox[w0 + e])) xi = -2 - (w0 + e);  // a W entry
            } else if (e < nw + nx) {  // an X-list entry of B or of an ancestor
                const int k = e - nw;
                int a = 0;
                while (a + 1 < nxa && s_xpre[a + 1] <= k) a++;
                xi = s_xbeg[a] + k - s_xpre[a];
            }
            if (xi != -1) {
                const bool isw = xi < -1;
                const int idx = isw ? -2 - xi : xi, A = isw ? wbox[idx] : xbox[idx];
                const int2 rg = srange[A];
                cnt = rg.y - rg.x;
                i0 = rg.x;
                int sh[3];
                decode_shift(isw ? wsh[idx] : xsh[idx], sh);
                o = V4<T>{(T)sh[0], (T)sh[1], (T)sh[2], (T)0};
            }
            const int F = publish(cnt, i0, o);
            run(std::integral_constant<int, kNear>{}, std::true_type{}, F, [&](int f, V4<T> &y, T(&d)[R * KS]) {
                const int ei = entry_of(f), i = s_idx[ei] + f - s_start[ei];
                const V4<T> oe = s_off[ei];
                const double h = exp2i(B.w);
                y.x = (T)((xsrc[3 * (long long)i] - (B.x + 0.5) * h) + (double)oe.x);
                y.y = (T)((xsrc[3 * (long long)i + 1] - (B.y + 0.5) * h) + (double)oe.y);
                y.z = (T)((xsrc[3 * (long long)i + 2] - (B.z + 0.5) * h) + (double)oe.z);
#pragma unroll
                for (int r = 0; r < R; r++)
#pragma unroll
                    for (int a = 0; a < KS; a++)
                        d[r * KS + a] = r < nv ? dens[(long long)i * nrhs * KS + (rhs0 + r) * KS + a] : (T)0;
            });
        }

        // the G groups' sums of each target, added in binary64
#pragma unroll
        for (int q = 0; q < Q; q++) {
            const int t = t0 + lg + LW * q;
#pragma unroll
            for (int r = 0; r < R; r++)
#pragma unroll
                for (int a = 0; a < KT; a++) {
                    double v = (double)L[q].tot[r][a] - (double)L[q].cmp[r][a];
#pragma unroll
                    for (int o = LW; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (grp == 0 && t < tr.y && r < nv)
                        pot[(long long)t * nrhs * KT + (rhs0 + r) * KT + a] = v * Acc::kScale;
                }
        }
    };
    for (int t0 = tr.x + (int)blockIdx.y * LW * QMAX; t0 < tr.y; t0 += (int)gridDim.y * LW * QMAX) {
        chunk(t0, (min(tr.y - t0, LW * QMAX) + LW - 1) / LW);  // block-uniform
    }
}

// ---------------- passes ----------------

template <typename T>
struct Bufs;
template <>
struct Bufs<double> {
    static DBuf<double> &up(Plan &P) { return P.up64; }
    static DBuf<double> &chk(Plan &P) { return P.chk64; }
    static DBuf<double> &dn(Plan &P) { return P.dn64; }
    static DBuf<double> &tmp(Plan &P) { return P.tmp64; }
    static DBuf<double> &yrel(Plan &P) { return P.ysrel64; }
    static DBuf<double> &xrel(Plan &P) { return P.xtrel64; }
    static DBuf<double> &g(Plan &P) { return P.g64; }
    static const double *dens(Plan &P) { return P.dens_s.p; }
    static const double *uc2e_a(Plan &P) { return P.uc2e_a.p; }
    static const double *uc2e_b(Plan &P) { return P.uc2e_b.p; }
    static const double *dc2e_a(Plan &P) { return P.dc2e_a.p; }
    static const double *dc2e_b(Plan &P) { return P.dc2e_b.p; }
    static const double *m2m(Plan &P) { return P.m2m.p; }
    static const double *l2l(Plan &P) { return P.l2l.p; }
    static const double *m2l(Plan &P) { return P.m2l.p; }
};
template <>
struct Bufs<float> {
    static DBuf<float> &up(Plan &P) { return P.up32; }
    static DBuf<float> &chk(Plan &P) { return P.chk32; }
    static DBuf<float> &dn(Plan &P) { return P.dn32; }
    static DBuf<float> &tmp(Plan &P) { return P.tmp32; }
    static DBuf<float> &yrel(Plan &P) { return P.ysrel32; }
    static DBuf<float> &xrel(Plan &P) { return P.xtrel32; }
    static DBuf<float> &g(Plan &P) { return P.g32; }
    static const float *dens(Plan &P) { return P.dens32.p; }
    static const float *uc2e_a(Plan &P) { return P.uc2e_a32.p; }
    static const float *uc2e_b(Plan &P) { return P.uc2e_b32.p; }
    static const float *dc2e_a(Plan &P) { return P.dc2e_a32.p; }
    static const float *dc2e_b(Plan &P) { return P.dc2e_b32.p; }
    static const float *m2m(Plan &P) { return P.m2m32.p; }
    static const float *l2l(Plan &P) { return P.l2l32.p; }
    static const float *m2l(Plan &P) { return P.m2l32.p; }
};

template <typename T>
static void prepare_points(Plan &P, cudaStream_t s) {
    using B = Bufs<T>;
    B::yrel(P).reserve(4 * (P.S + 1));  // V4<T>: 4 values per point
    B::xrel(P).reserve(4 * (P.T + 1));
    auto *yr = reinterpret_cast<V4<T> *>(B::yrel(P).p);
    auto *xr = reinterpret_cast<V4<T> *>(B::xrel(P).p);
    if (P.n_leaves_src)
        count_launch(), k_relcoords<T><<<P.n_leaves_src, 128, 0, s>>>(P.leaves_src.p, P.tree.bpos.p, P.tree.srange.p, P.xs.p, yr);
    if (P.n_leaves_trg)
        count_launch(), k_relcoords<T><<<P.n_leaves_trg, 128, 0, s>>>(P.leaves_trg.p, P.tree.bpos.p, P.tree.trange.p, P.xt.p, xr);
    if (sizeof(T) == 4) {
        long long nd = P.S * P.nrhs * P.ks;
        P.dens32.reserve(nd + 1);
        if (nd) count_launch(), k_cast<float><<<nblk(nd, 256), 256, 0, s>>>(P.dens_s.p, P.dens32.p, nd);
    }
    size_t rows = (size_t)P.tree.nbox * P.nrhs * P.kn;
    B::up(P).reserve(rows);
    B::chk(P).reserve(rows);
    B::dn(P).reserve(rows);
    B::tmp(P).reserve(rows);
    PK_CUDA(cudaMemsetAsync(B::up(P).p, 0, sizeof(T) * rows, s));
    if (P.basis) {  // Ub^T phi_u is written for boxes with sources only; the others are V sources of zero density
        const size_t rr = (size_t)P.tree.nbox * P.nrhs * P.basis->r;
        P.uphat32.reserve(rr);
        P.chkhat32.reserve(rr);
        PK_CUDA(cudaMemsetAsync(P.uphat32.p, 0, sizeof(float) * rr, s));
    }
}

// The leaf level of the upward pass: leaf-relative coordinates, densities in
// the arithmetic of the path, S2M check values.  It needs only the leaf lists,
// so the task grouping enqueues it before it builds the other tasks on the host.
template <typename T, int K, int KS = K>
static void upward_leaves_t(Plan &P, cudaStream_t s) {
    using B = Bufs<T>;
    prepare_points<T>(P, s);
    const int nr = P.nrhs;
    auto *yr = reinterpret_cast<const V4<T> *>(B::yrel(P).p);
    if (P.n_leaves_src)
        for (int r = 0; r < nr; r += 4) {  // up to 4 density vectors per pass
            auto go = [&](auto rt) {
                constexpr int R = decltype(rt)::value;
                count_launch(), k_s2m<T, K, R, KS><<<P.n_leaves_src, KS_T, 0, s>>>(
                    P.leaves_src.p, P.tree.bpos.p, P.tree.srange.p, yr, B::dens(P), nr, r, B::g(P).p, P.n,
                    B::chk(P).p);
            };
            if (nr - r == 1) go(std::integral_constant<int, 1>{});
            else if (nr - r == 2) go(std::integral_constant<int, 2>{});
            else go(std::integral_constant<int, 4>{});
        }
    P.leaves_up = true;
}

void upward_leaves(Plan &P, cudaStream_t s) {
    if (P.precision == PKIFMM_FP64) {
        if (P.ks == 3 && P.k == 1) upward_leaves_t<double, 1, 3>(P, s);
        else if (P.k == 1) upward_leaves_t<double, 1>(P, s);
        else upward_leaves_t<double, 3>(P, s);
    } else {
        if (P.ks == 3 && P.k == 1) upward_leaves_t<float, 1, 3>(P, s);
        else if (P.k == 1) upward_leaves_t<float, 1>(P, s);
        else upward_leaves_t<float, 3>(P, s);
    }
}

template <typename T, int K, int KS = K>
static void upward_t(Plan &P, cudaStream_t s) {
    using B = Bufs<T>;
    if (!P.leaves_up) upward_leaves_t<T, K, KS>(P, s);
    P.leaves_up = false;
    const int kn = P.kn, nr = P.nrhs;
    const long long kn2 = (long long)kn * kn;
    if constexpr (std::is_same<T, float>::value) {
        if (P.tr) {  // tensor cores: tmp = S+ (U^T q~u), up = V tmp, then M2M level by level
            trans_tc_gemm(P, 0, P.t_uc2e, nullptr, 1, P.chk32.p, P.tmp32.p, 0, s);
            if (P.basis) {  // with Ub^T phi_u for the M2L in the shared basis
                trans_tc_gemm(P, 6, P.t_uc2e, nullptr, 1, P.tmp32.p, P.up32.p, 0, s, P.uphat32.p);
                for (int l = (int)P.t_m2m.size() - 1; l >= 0; l--)
                    trans_tc_gemm(P, 7, P.t_m2m[l], P.tree.child.p, 8, P.up32.p, P.up32.p, 0, s, P.uphat32.p);
                return;
            }
            trans_tc_gemm(P, 1, P.t_uc2e, nullptr, 1, P.tmp32.p, P.up32.p, 0, s);
            for (int l = (int)P.t_m2m.size() - 1; l >= 0; l--)
                trans_tc_gemm(P, 4, P.t_m2m[l], P.tree.child.p, 8, P.up32.p, P.up32.p, 0, s);
            return;
        }
    }
    // UC2E: tmp = U^T q~u ; up = (V S+) tmp
    gemm<T>(P.t_uc2e, nullptr, 1, B::uc2e_b(P), 0, B::chk(P).p, B::tmp(P).p, kn, nr, 0, s);
    gemm<T>(P.t_uc2e, nullptr, 1, B::uc2e_a(P), 0, B::tmp(P).p, B::up(P).p, kn, nr, 0, s);
    for (int l = (int)P.t_m2m.size() - 1; l >= 0; l--)
        gemm<T>(P.t_m2m[l], P.tree.child.p, 8, B::m2m(P), kn2, B::up(P).p, B::up(P).p, kn, nr, 0, s);
}

void run_upward(Plan &P, cudaStream_t s) {
    if (P.precision == PKIFMM_FP64) {
        if (P.ks == 3 && P.k == 1) upward_t<double, 1, 3>(P, s);
        else if (P.k == 1) upward_t<double, 1>(P, s);
        else upward_t<double, 3>(P, s);
    } else {
        if (P.ks == 3 && P.k == 1) upward_t<float, 1, 3>(P, s);
        else if (P.k == 1) upward_t<float, 1>(P, s);
        else upward_t<float, 3>(P, s);
    }
}

template <typename T>
__global__ void k_f2d(const T *__restrict__ a, double *__restrict__ b, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

// MIXED: the root far field (Algorithm 2 step c) and its check-to-equivalent
// solve run in binary64 on a binary64 copy of the root's upward density.
void root_mixed(Plan &P, cudaStream_t s) {
    const int kn = P.kn, nr = P.nrhs * P.nprob;  // the roots are boxes 0..nprob-1
    long long rows = (long long)nr * kn;
    P.chk64.reserve(rows);
    P.tmp64.reserve(rows);
    P.dn64.reserve(rows);
    P.up64.reserve(rows);
    if (!P.periodic) {
        PK_CUDA(cudaMemsetAsync(P.dn32.p, 0, sizeof(float) * rows, s));
        return;
    }
    count_launch(), k_f2d<float><<<nblk(rows, 256), 256, 0, s>>>(P.up32.p, P.up64.p, rows);
    matvec64(P.root.p, P.up64.p, P.chk64.p, kn, nr, s);
    matvec64(P.dc2e_b.p, P.chk64.p, P.tmp64.p, kn, nr, s);
    matvec64(P.dc2e_a.p, P.tmp64.p, P.dn64.p, kn, nr, s);
    count_launch(), k_cast<float><<<nblk(rows, 256), 256, 0, s>>>(P.dn64.p, P.dn32.p, rows);
}

void run_root(Plan &P, cudaStream_t s) {
    if (P.precision == PKIFMM_FP64) {
        const int nr = P.nrhs * P.nprob;  // the roots are boxes 0..nprob-1
        if (P.periodic) matvec64(P.root.p, P.up64.p, P.chk64.p, P.kn, nr, s);
        else  // no far field; the rows may hold root leaves' upward check values
            PK_CUDA(cudaMemsetAsync(P.chk64.p, 0, sizeof(double) * nr * P.kn, s));
        return;
    }
    root_mixed(P, s);
}

void run_m2l(Plan &P, cudaStream_t s) {
    const int kn = P.kn, nr = P.nrhs;
    const long long kn2 = (long long)kn * kn;
    if (P.precision == PKIFMM_FP64) {
        gemm<double>(P.t_m2l, P.tree.v_slot.p, kVSlots, P.m2l.p, kn2, P.up64.p, P.chk64.p, kn, nr, 0, s);
    } else {
        if (!m2l_tc_run(P, s)) throw Error(PKIFMM_ERR_UNSUPPORTED, "tensor-core M2L not prepared");
    }
}

template <typename T, int K, int KS = K>
static void downward_t(Plan &P, cudaStream_t s) {
    using B = Bufs<T>;
    const int kn = P.kn, nr = P.nrhs;
    const long long kn2 = (long long)kn * kn;
    auto *yr = reinterpret_cast<const V4<T> *>(B::yrel(P).p);
    // with a shared M2L basis the M2L output is not in the check rows: the X-list sums start from zero
    if (P.basis && P.n_xboxes) PK_CUDA(cudaMemsetAsync(P.chk32.p, 0, sizeof(float) * P.tree.nbox * nr * kn, s));
    if (P.n_xboxes)
        for (int r = 0; r < nr; r += 4) {
            auto go = [&](auto rt) {
                constexpr int R = decltype(rt)::value;
                count_launch(), k_s2l<T, K, R, KS><<<P.n_xboxes, KS_T, 0, s>>>(
                    P.xboxes.p, P.tree.bpos.p, P.tree.srange.p, P.tree.trange.p, P.tree.x_ptr.p, P.tree.x_box.p,
                    P.tree.x_sh.p, yr,
                    B::dens(P), nr, r, B::g(P).p, P.n, B::chk(P).p);
            };
            if (nr - r == 1) go(std::integral_constant<int, 1>{});
            else if (nr - r == 2) go(std::integral_constant<int, 2>{});
            else go(std::integral_constant<int, 4>{});
        }
    bool tc = false;
    if constexpr (std::is_same<T, float>::value) tc = P.tr != nullptr;
    if (tc && P.basis) {  // tmp = S+ (V^T Ub q^) + S+ (V^T q~x), dn = U tmp
        trans_tc_gemm(P, 8, P.t_dc2e, nullptr, 1, P.chkhat32.p, P.tmp32.p, 0, s);
        if (P.n_xboxes) trans_tc_gemm(P, 2, P.t_dcx, nullptr, 1, P.chk32.p, P.tmp32.p, 1, s);
        trans_tc_gemm(P, 3, P.t_dc2e, nullptr, 1, P.tmp32.p, P.dn32.p, 0, s);
    } else if (tc) {  // tensor cores: tmp = S+ (V^T q~d), dn = U tmp
        trans_tc_gemm(P, 2, P.t_dc2e, nullptr, 1, P.chk32.p, P.tmp32.p, 0, s);
        trans_tc_gemm(P, 3, P.t_dc2e, nullptr, 1, P.tmp32.p, P.dn32.p, 0, s);
    } else {
        gemm<T>(P.t_dc2e, nullptr, 1, B::dc2e_b(P), 0, B::chk(P).p, B::tmp(P).p, kn, nr, 0, s);
        gemm<T>(P.t_dc2e, nullptr, 1, B::dc2e_a(P), 0, B::tmp(P).p, B::dn(P).p, kn, nr, 0, s);
    }
    if (P.far_direct && P.periodic) {
        // step d: keep the roots' downward equivalent densities (binary64) for the
        // direct evaluation at the targets and do not pass them down
        const long long rows = (long long)P.nprob * nr * kn;
        P.far64.reserve(rows);
        PK_CUDA(cudaMemcpyAsync(P.far64.p, P.dn64.p, sizeof(double) * rows, cudaMemcpyDeviceToDevice, s));
        PK_CUDA(cudaMemsetAsync(B::dn(P).p, 0, sizeof(T) * rows, s));
    }
    for (size_t l = 1; l < P.t_l2l.size(); l++) {
        if constexpr (std::is_same<T, float>::value)
            if (tc) {
                trans_tc_gemm(P, 5, P.t_l2l[l], P.tree.parent.p, 1, P.dn32.p, P.dn32.p, 1, s);
                continue;
            }
        gemm<T>(P.t_l2l[l], P.tree.parent.p, 1, B::l2l(P), kn2, B::dn(P).p, B::dn(P).p, kn, nr, 1, s);
    }
    if (tc) trans_tc_check(P, s);  // every bounded wait of the upward and downward translations
}

void run_downward(Plan &P, cudaStream_t s) {
    if (P.precision == PKIFMM_FP64) {
        if (P.ks == 3 && P.k == 1) downward_t<double, 1, 3>(P, s);
        else if (P.k == 1) downward_t<double, 1>(P, s);
        else downward_t<double, 3>(P, s);
    } else {
        if (P.ks == 3 && P.k == 1) downward_t<float, 1, 3>(P, s);
        else if (P.k == 1) downward_t<float, 1>(P, s);
        else downward_t<float, 3>(P, s);
    }
}

template <typename T, int K, int KT, int KS = K>
static void leaves_t(Plan &P, cudaStream_t s) {
    using B = Bufs<T>;
    const int nr = P.nrhs;
    P.pot_s.reserve((size_t)P.T * nr * KT + 1);
    auto *yr = reinterpret_cast<const V4<T> *>(B::yrel(P).p);
    auto *xr = reinterpret_cast<const V4<T> *>(B::xrel(P).p);
    // one warp per target leaf and chunk of (32 / G) QMAX targets (QMAX from
    // the outputs a target carries); up to 4 density vectors per launch
    auto launch = [&](auto r_tag, int r0) {
        constexpr int R = decltype(r_tag)::value, W = R * KT * (int)(sizeof(T) / 4);
        constexpr int QMAX = W <= 1 ? 4 : (W <= 3 ? 3 : (W <= 6 ? 2 : 1));  // registers: three sums per output
        // source groups: four for Laplace (a cheap pair: one staged source serving
        // more targets pays), two for Stokes (measured faster than four: a leaf
        // of up to 64 targets stays in one block); targets per chunk
        constexpr int G = K == 1 && QMAX == 4 ? 4 : (QMAX >= 2 ? 2 : 1), CH = 32 / G * QMAX;
        const dim3 grid(P.n_leaves_trg, std::max(1, (P.leaf_max + CH - 1) / CH));
        count_launch(), k_leaf<T, K, R, QMAX, G, KT, KS><<<grid, 32, 0, s>>>(
                P.leaves_trg.p, P.tree.bpos.p, P.tree.srange.p, P.tree.trange.p, P.tree.u_ptr.p, P.tree.u_box.p,
                P.tree.u_sh.p, P.tree.w_ptr.p, P.tree.w_box.p, P.tree.w_sh.p, P.tree.parent.p, P.tree.x_ptr.p,
                P.tree.x_box.p, P.tree.x_sh.p, yr, xr, B::dens(P), P.xs.p,
                B::up(P).p, B::dn(P).p, nr, r0, B::g(P).p, P.n, P.pot_s.p);
    };
    if (P.n_leaves_trg)
        for (int r0 = 0; r0 < nr; r0 += 4) {
            if (nr - r0 == 1) launch(std::integral_constant<int, 1>{}, r0);
            else if (nr - r0 == 2) launch(std::integral_constant<int, 2>{}, r0);
            else launch(std::integral_constant<int, 4>{}, r0);
        }
}

// Algorithm 2 step d: q_t += K(x_t, y^{B0,d}) phi^{B0,d}, the far field of
// all images beyond the near layers evaluated directly from the root's
// downward equivalent density (surface of half-width 1.475 around the
// centre of the unit box), in binary64.  Problem of target t: its key prefix.
// KT = 4 (Laplace field): the potential and its gradient.
template <int K, int KT>
__global__ void k_far_direct(const double *__restrict__ xt, long long T, const unsigned long long *__restrict__ keyT,
                             int key_shift, const double *__restrict__ far, const double *__restrict__ g, int n,
                             int nrhs, double *__restrict__ pot_s) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= T) return;
    const long long j = (long long)(keyT[t] >> key_shift);
    const double x0 = xt[3 * t] - 0.5, x1 = xt[3 * t + 1] - 0.5, x2 = xt[3 * t + 2] - 0.5;
    const int kn = n * K;
    for (int r = 0; r < nrhs; r++) {
        const double *phi = far + (j * nrhs + r) * kn;
        double acc[KT];
        for (int a = 0; a < KT; a++) acc[a] = 0.0;
        for (int i = 0; i < n; i++) {
            const double d0 = x0 - 1.475 * g[3 * i], d1 = x1 - 1.475 * g[3 * i + 1], d2 = x2 - 1.475 * g[3 * i + 2];
            if constexpr (KT == 4) {
                const double ir = 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2), qi3 = phi[i] * ir * ir * ir;
                acc[0] += phi[i] * ir;
                acc[1] -= d0 * qi3;
                acc[2] -= d1 * qi3;
                acc[3] -= d2 * qi3;
            } else {
                Kern<double, K>::add(acc, d0, d1, d2, phi + i * K);
            }
        }
        for (int a = 0; a < KT; a++) pot_s[(t * nrhs + r) * KT + a] += acc[a];
    }
}

void run_leaves(Plan &P, cudaStream_t s) {
    const bool field = P.kt == 4;
    if (P.precision == PKIFMM_FP64) {
        if (field) leaves_t<double, 1, 4>(P, s);
        else if (P.ks == 3 && P.k == 1) leaves_t<double, 1, 1, 3>(P, s);
        else if (P.k == 1) leaves_t<double, 1, 1>(P, s);
        else leaves_t<double, 3, 3>(P, s);
    } else {
        if (field) leaves_t<float, 1, 4>(P, s);
        else if (P.ks == 3 && P.k == 1) leaves_t<float, 1, 1, 3>(P, s);
        else if (P.k == 1) leaves_t<float, 1, 1>(P, s);
        else leaves_t<float, 3, 3>(P, s);
    }
    if (P.far_direct && P.periodic && P.T > 0) {
        const int shift = P.nprob > 1 ? 3 * P.depth_max : 63;  // one problem: index 0
        const unsigned nb = (unsigned)((P.T + 127) / 128);
        if (field)
            count_launch(), k_far_direct<1, 4><<<nb, 128, 0, s>>>(P.xt.p, P.T, P.keyT.p, shift, P.far64.p, P.g64.p,
                                                                   P.n, P.nrhs, P.pot_s.p);
        else if (P.k == 1)
            count_launch(), k_far_direct<1, 1><<<nb, 128, 0, s>>>(P.xt.p, P.T, P.keyT.p, shift, P.far64.p, P.g64.p,
                                                                   P.n, P.nrhs, P.pot_s.p);
        else
            count_launch(), k_far_direct<3, 3><<<nb, 128, 0, s>>>(P.xt.p, P.T, P.keyT.p, shift, P.far64.p, P.g64.p,
                                                                   P.n, P.nrhs, P.pot_s.p);
    }
}

}  // namespace pk
