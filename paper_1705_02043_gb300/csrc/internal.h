// Internal declarations shared by the CUDA translation units.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/pkifmm.h"
#include "precompute.h"

namespace pk {

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define PK_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            throw ::pk::Error(e_ == cudaErrorMemoryAllocation ? PKIFMM_ERR_OOM : PKIFMM_ERR_CUDA, \
                              std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

// Kernel launches issued by this library (all threads), for launch accounting.
inline std::atomic<long long> g_launches{0};
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

constexpr int kMaxLevel = 16;
constexpr int kVSlots = 189;     // V-list slots per target octant class
constexpr int kM2LOps = 316;     // offsets o in [-3,3]^3 with |o|_inf >= 2

// Device buffer that only grows.
template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t cap = 0;
    void reserve(size_t n) {
        if (n <= cap) return;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t m = n + n / 4 + 64;
        PK_CUDA(cudaMalloc(&p, m * sizeof(T)));
        cap = m;
    }
    // grow keeping contents (first `keep` elements)
    void grow_keep(size_t n, size_t keep, cudaStream_t s) {
        if (n <= cap) return;
        T *q = nullptr;
        size_t m = n + n / 2 + 64;
        PK_CUDA(cudaMalloc(&q, m * sizeof(T)));
        if (p && keep) PK_CUDA(cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s));
        if (p) {
            PK_CUDA(cudaStreamSynchronize(s));
            cudaFree(p);
        }
        p = q;
        cap = m;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

// Octree on the device.  Boxes are numbered level by level; within a level
// they are in Morton order (octant bits x = 1, y = 2, z = 4).
struct Tree {
    int nbox = 0, depth = 0;
    std::vector<int> lvl_begin;        // host: boxes of level l in [lvl_begin[l], lvl_begin[l+1])
    DBuf<unsigned long long> key;      // Morton key at the box's level
    DBuf<int4> bpos;                   // (x, y, z, level)
    DBuf<int> parent;                  // -1 for the root
    DBuf<int> child;                   // [nbox][8], -1 if absent
    DBuf<int2> srange, trange;         // point ranges in sorted order
    DBuf<int> lvl_begin_d;             // device copy of lvl_begin
    // lists: CSR over target boxes; entries (box, shift code 0..26)
    DBuf<int> u_ptr, u_box, w_ptr, w_box, x_ptr, x_box;
    DBuf<unsigned char> u_sh, w_sh, x_sh;
    DBuf<int> v_slot;                  // [nbox][189] source box or -1
    long long nU = 0, nW = 0, nX = 0, nV = 0, p2p_pairs = 0;
    int nleaf = 0;
};

// A batch of dense translations dst[row] (+)= sum_s OP[class, s] src[slot(row, s)].
struct Task {
    int nrows = 0;            // rows = boxes * nrhs
    int nclass = 1, nslots = 1;
    DBuf<int> boxes;          // dst box per task box (class-major order)
    DBuf<int4> tiles;         // (class, row0, nrows, 0)
    int ntiles = 0;
    DBuf<int> class_ops;      // [nclass][nslots]
    std::vector<int> h_boxes; // host copies used to build tiles
    std::vector<int> class_count;  // boxes per class
};

struct TcState;  // tensor-core M2L state (m2l_tc.cu)
struct TrState;  // tensor-core translations state (trans_tc.cu)

struct Plan {
    int kernel = 0, k = 1, p = 0, n = 0, kn = 0, ell = 2, leaf_max = 64, depth_max = 10;
    int kt = 1;  // target components: k, or 4 for the Laplace field (potential and gradient)
    int ks = 1;  // source density components: k, or 3 for Laplace dipole sources
    int nimg = -1;  // >= 0: finite array of cells along the periodic axis (no wrap, no compatibility condition)
    int precision = 0, nrhs = 1, device = 0;
    unsigned periodic = 0;
    double lo[3] = {0, 0, 0}, L = 1;
    HostOps host;

    // operators on the device (FP64 master copies; FP32 copies for MIXED)
    DBuf<double> g64;                           // [n][3]
    DBuf<float> g32;
    DBuf<double> uc2e_a, uc2e_b, dc2e_a, dc2e_b, m2m, l2l, m2l, root;
    DBuf<float> uc2e_a32, uc2e_b32, dc2e_a32, dc2e_b32, m2m32, l2l32, m2l32;
    DBuf<int> class_slot_op;                    // [8][189] M2L op index per class slot
    std::vector<int> h_class_slot_op;           // host copy
    DBuf<short> slot_of;                        // [8][343] slot of offset o, -1 if none

    // evaluation workspace
    int64_t S = 0, T = 0;
    int nprob = 1;                              // independent problems in this evaluation
    int far_direct = 0;                         // 1: far field by Algorithm 2 step d instead of L2L
    char *stage_h = nullptr;                    // pinned staging for per-evaluation task uploads
    size_t stage_cap = 0;
    cudaEvent_t stage_ev = nullptr;
    bool stage_ev_live = false;
    char *down_h = nullptr;                     // pinned buffer for the tree read back each evaluation
    size_t down_cap = 0;
    const int4 *h_bpos = nullptr;               // views into down_h of this evaluation's boxes (null
    const int2 *h_trange = nullptr;             // until the tasks are built)
    DBuf<double> far64;                         // roots' downward equivalent densities (step d)
    DBuf<long long> soff, toff;                 // [nprob+1] CSR offsets of their points
    bool same_offsets = true;                   // soff == toff element by element
    DBuf<unsigned long long> keyS, keyT, keyS2, keyT2;
    DBuf<int> idxS, idxT, idxS2, idxT2;
    DBuf<int> hist;
    DBuf<int> err;                              // [4] device error flags
    DBuf<double> xs, xt;                        // sorted unit coordinates [N][3]
    DBuf<double> dens_s;                        // sorted densities [S][nrhs*k]
    DBuf<double> pot_s;                         // sorted potentials [T][nrhs*k]
    DBuf<double> ysrel64, xtrel64;              // leaf-relative coordinates [N][4]
    DBuf<float> ysrel32, xtrel32;
    DBuf<float> dens32, pot32;
    DBuf<double> sums;                          // neutrality sums
    // equivalent densities [nbox][nrhs][kn]
    DBuf<double> up64, chk64, dn64, tmp64;
    DBuf<float> up32, chk32, dn32, tmp32;
    // MIXED with a shared M2L basis Ub (r columns): Ub^T phi_u and the M2L output in that basis, [nbox][nrhs][r]
    std::shared_ptr<const M2LBasis> basis;
    DBuf<float> uphat32, chkhat32;
    // tree build scratch
    DBuf<int> cnt, off;
    DBuf<double> xn;                            // normalised coordinates before the gather
    DBuf<int> lcnt;                             // [3][nbox] U / W / X list lengths
    DBuf<int> scan_tmp;                         // prefix-sum scratch
    bool leaves_up = false;                     // the upward pass's leaf level is enqueued already
    bool same_points = false;                   // the targets are the sources (one sort)
    DBuf<unsigned long long> lpairs;            // [2] P2P pairs, V entries
    DBuf<int2> csr, ctr;                        // [nlevel boxes][8] child ranges
    DBuf<int> gather_idx;
    Tree tree;
    Task t_uc2e, t_m2l, t_dc2e, t_root;
    Task t_dcx;                                 // boxes with targets and an X list (MIXED with a shared M2L basis)
    std::vector<Task> t_m2m, t_l2l;             // per level
    DBuf<int> leaves_src, leaves_trg, xboxes;   // task lists for kernel sums
    int n_leaves_src = 0, n_leaves_trg = 0, n_xboxes = 0;
    double stage_ms[9] = {0};
    cudaEvent_t ev[9] = {};
    bool events = false;
    TcState *tc = nullptr;
    TrState *tr = nullptr;                      // null: binary32 SIMT translations
};

void m2l_tc_release(Plan &P);
float m2l_tc_last_ms(Plan &P);
// ---- trans_tc.cu: MIXED dense translations on the tensor cores ----
// set: 0 U^T (output rows scaled by S+), 1 V, 2 V^T (scaled by S+), 3 U, 4 M2M, 5 L2L
void trans_tc_prepare(Plan &P);
void trans_tc_release(Plan &P);
// sets 6, 7 (with a shared M2L basis): [V; Ub^T V], [M2M; Ub^T M2M] write phi to dst
// and Ub^T phi to dst2; set 8: V^T Ub (rows scaled by S+) from the M2L output in that basis
void trans_tc_gemm(Plan &P, int set, const Task &task, const int *slot_table, int slot_stride, const float *src,
                   float *dst, int beta, cudaStream_t s, float *dst2 = nullptr);
void trans_tc_check(Plan &P, cudaStream_t s);  // throws TIMEOUT if a bounded wait gave up

// ---- tree.cu ----
void build_tree(Plan &P, cudaStream_t s);
void build_lists(Plan &P, cudaStream_t s);
// ---- translate.cu ----
void upload_operators(Plan &P);
void build_tasks(Plan &P, cudaStream_t s);
void run_upward(Plan &P, cudaStream_t s);
void run_root(Plan &P, cudaStream_t s);
void run_m2l(Plan &P, cudaStream_t s);
void run_downward(Plan &P, cudaStream_t s);
void run_leaves(Plan &P, cudaStream_t s);

inline int shift_code(int sx, int sy, int sz) { return (sx + 1) * 9 + (sy + 1) * 3 + (sz + 1); }

}  // namespace pk
