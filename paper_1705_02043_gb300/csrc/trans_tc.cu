// Tensor-core dense translations of the MIXED path (tcgen05, split-fp16
// products): the check-to-equivalent solves of the upward and downward passes
// and the precomposed M2M and L2L operators (Sec. 2.2; the solves applied as
// two factors, Sec. 3.1).
//
// Each translation is the slot GEMM
//     dst[box][rhs][:] (+)= sum_slots Op[class, slot] src[slot box][rhs][:]
// of the binary32 path (slot table: the box itself for the solves, the eight
// children for M2M, the parent for L2L), computed as
//     D[128 operator rows x 128 (box, rhs) columns] = sum_s sum_k Op[:, k] Src_s[:, k]^T
// like the V-list M2L: operands scaled by powers of two into the fp16 range
// and split x = x_hi + x_lo (22 significant bits), three products per term.
//
// The solve phi = V S+ U^T q is applied as U^T, then the row scale S+ in the
// epilogue, then V (and U S+ V^T likewise): V S+ has columns that differ by the
// inverse singular values (up to 1/eps_SVD), which one power-of-two scale per
// operator cannot keep to 22 bits, while U, V have entries of one size.
//
// Precision: the tensor core truncates at every fp32 accumulation step, so the
// work accumulator is drained into fp32 registers (round to nearest) after
// every K chunk of 64 (PKIFMM_TRANS_DRAIN chunks; measured on a Laplace p = 8
// clustered case: 1.1e-6 draining every chunk, 1.9e-6 every two, 8.2e-7 for the
// binary32 SIMT product).
//
// Pipeline as in the M2L kernel: warps 0-3 load the source rows (fp16, split
// beforehand) into the 128B-swizzled K-major layout, by one TMA per split when
// the tile's source boxes are regular and by cp.async gathers otherwise, and
// one thread issues the TMA loads of the operator tiles; warp 4 issues the
// MMAs; warps 5-8 drain.  Every mbarrier wait is bounded in time; on timeout
// the kernel raises the error flag and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "tc_ptx.cuh"

namespace pk {

namespace {

struct TrOps {
    __half *op = nullptr;  // [2][nops][KM][KK] (hi, lo), scaled by 2^kexp
    int nops = 0, kexp = 0;
    int M = 0, K = 0;      // output rows, input length
    int msplit = 0;        // output rows [0, msplit) to dst, [msplit, M) to dst2
    int KM = 0, KK = 0;    // M padded to 128 (M tiles), K to 64 (K chunks)
    CUtensorMap tmap[2];
};

constexpr int kTrMaxSlots = 8;

}  // namespace

struct TrState {
    int drain = 1;
    // U^T, V, V^T, U, M2M[8], L2L[8]; with a shared M2L basis Ub (r columns):
    // [V; Ub^T V], [M2M; Ub^T M2M][8], V^T Ub
    TrOps ops[9];
    float *sinv = nullptr;     // [kn padded to 128] 1/s_j above the cut, else 0
    __half *phi = nullptr;     // [2][phi_rows][phi_kk] split source rows
    size_t phi_rows = 0;
    int phi_kk = 0;
    float *amax = nullptr;
    int *err = nullptr;
    int *err_host = nullptr;
    float *part = nullptr;     // slot-group partial sums of small launches (k_trans_reduce)
    size_t part_cap = 0;
    int sms = 0;
};

namespace {

struct TrArgs {
    const __half *phi_hi, *phi_lo;  // split source rows [rows][KK]
    const int *tboxes;              // task boxes, class-major
    const int4 *tiles;              // (class, row0, nrows, source-row mode: 0 gather, 1 or 8 regular)
    const int *slot_table;          // [box][slot_stride] source box per slot; null: the box itself
    int slot_stride, nslots;
    const int *class_ops;           // [nclass][nslots] operator of (class, slot), -1 none
    float *dst;                     // rows of msplit values: output components [0, msplit)
    float *dst2;                    // rows of mrows - msplit values: components [msplit, mrows)
    int beta;                       // 1: add to dst
    const float *rscale;            // [KM] scale of each output component, nullable
    const float *amax;              // max |source| over the rows the task reads
    int mrows, msplit, KM, KK, nrhs, kexp, drain;
    int *err;
    float *part;                    // non-null: slot group blockIdx.y of nsplit writes its partial sum (as dst)
    int nsplit;
};

// Tiles marked regular (tile.w = 1: source rows src0 + i; 8: src0 + 8 i, with
// one density vector) load their 128 source rows per split by one TMA, through
// a 2D view of the split rows (tB1) or a 3D view with rows grouped by eight
// (tB8, coordinates (k, src0 % 8, src0 / 8 + i)); the other tiles gather rows
// with cp.async.
template <int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_trans_tc(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
               const __grid_constant__ CUtensorMap tB1_hi, const __grid_constant__ CUtensorMap tB1_lo,
               const __grid_constant__ CUtensorMap tB8_hi, const __grid_constant__ CUtensorMap tB8_lo, TrArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)smem;          // [STAGES]
    uint64_t *empty = full + STAGES;            // [STAGES]
    uint64_t *wfull = empty + STAGES;           // [2] work accumulator ready
    uint64_t *wfree = wfull + 2;                // [2] work accumulator drained
    uint32_t *tmem_slot = (uint32_t *)(wfree + 2);
    int *nact_s = (int *)(tmem_slot + 1);
    int *act = nact_s + 1;                      // [kTrMaxSlots]
    long long *drow = (long long *)(smem + 1024);  // [128]
    int *sbox = (int *)(smem + 1024 + 8 * TC_N);   // [128]
    uint8_t *stages = smem + TC_CTRL_BYTES;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mtiles = a.KM / TC_M;
    const int4 tile = a.tiles[blockIdx.x / mtiles];
    const int cls = tile.x, row0 = tile.y, nr = tile.z;
    const int m0 = (blockIdx.x % mtiles) * TC_M;
    const int kchunks = a.KK / TC_K;
    const int ngroups = (kchunks + a.drain - 1) / a.drain;  // drains per slot

    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 128);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&wfull[b], 1);
            mbar_init(&wfree[b], 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int n = tid; n < TC_N; n += TC_THREADS) {
        if (n < nr) {
            const int row = row0 + n, tb = row / a.nrhs, rhs = row % a.nrhs, box = a.tboxes[tb];
            // a split launch writes its slot group's partial sums (the host then
            // passes the partial buffer as dst, msplit = mrows, beta = 0)
            drow[n] = a.part ? ((long long)blockIdx.y * (gridDim.x / mtiles) + blockIdx.x / mtiles) * TC_N + n
                             : (long long)box * a.nrhs + rhs;
            sbox[n] = box;
        } else {
            drow[n] = -1;
            sbox[n] = -1;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // slots of this class with an operator and at least one source in the tile
    if (tid == 0) {
        int c = 0;
        for (int s = 0; s < a.nslots; s++) {
            if (a.class_ops[cls * a.nslots + s] < 0) continue;
            int any = 0;
            for (int n = 0; n < nr && !any; n++)
                any = a.slot_table ? a.slot_table[(long long)sbox[n] * a.slot_stride + s] >= 0 : 1;
            if (any && (!a.part || s % a.nsplit == (int)blockIdx.y)) act[c++] = s;
        }
        *nact_s = c;
    }
    __syncthreads();
    const int nact = *nact_s;
    const uint32_t tmem = *tmem_slot;
    const int total = nact * kchunks;

    if (warp < 4 && tile.w) {
        // ---- producer (regular tile): one thread, TMA for both operands ----
        const int mode = tile.w;
        int cur_si = -1, src0 = 0;
        for (int it = 0; it < total; it++) {
            const int st = it % STAGES;
            const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
            if (!mbar_wait(&empty[st], ph ^ 1u, a.err)) break;
            const int si = it / kchunks, k0 = (it % kchunks) * TC_K;
            uint8_t *sb = stages + (size_t)st * TC_STAGE_BYTES;
            if (tid == 0) {
                if (si != cur_si) {
                    cur_si = si;
                    const int box0 = sbox[0];
                    src0 = a.slot_table ? a.slot_table[(long long)box0 * a.slot_stride + act[si]] : box0;
                }
                const int op = a.class_ops[cls * a.nslots + act[si]];
                mbar_expect_tx(&full[st], (uint32_t)(2 * TC_A_BYTES + 2 * TC_B_BYTES));
                tma_load_2d(sb, &tA_hi, k0, op * a.KM + m0, &full[st]);
                tma_load_2d(sb + TC_A_BYTES, &tA_lo, k0, op * a.KM + m0, &full[st]);
                if (mode == 8) {
                    tma_load_3d(sb + 2 * TC_A_BYTES, &tB8_hi, k0, src0 & 7, src0 >> 3, &full[st]);
                    tma_load_3d(sb + 2 * TC_A_BYTES + TC_B_BYTES, &tB8_lo, k0, src0 & 7, src0 >> 3, &full[st]);
                } else {
                    tma_load_2d(sb + 2 * TC_A_BYTES, &tB1_hi, k0, src0, &full[st]);
                    tma_load_2d(sb + 2 * TC_A_BYTES + TC_B_BYTES, &tB1_lo, k0, src0, &full[st]);
                }
            }
            mbar_arrive(&full[st]);  // 128 arrivals, as in the gather path
        }
    } else if (warp < 4) {
        // ---- producers: gather the source rows (cp.async) and TMA the operator tiles ----
        const int r = tid;
        const int rhs = (row0 + r) % a.nrhs, box = sbox[r];
        const int ri = r & 7;
        int cur_si = -1, op = 0;
        long long srow = -1;  // -1: no source in this slot (zeros)
        for (int it = 0; it < total; it++) {
            const int st = it % STAGES;
            const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
            if (!mbar_wait(&empty[st], ph ^ 1u, a.err)) break;
            const int si = it / kchunks, k0 = (it % kchunks) * TC_K;
            if (si != cur_si) {
                cur_si = si;
                const int s = act[si];
                op = a.class_ops[cls * a.nslots + s];
                int src = box < 0 ? -1 : a.slot_table ? a.slot_table[(long long)box * a.slot_stride + s] : box;
                srow = src >= 0 ? (long long)src * a.nrhs + rhs : -1;
            }
            uint8_t *sb = stages + (size_t)st * TC_STAGE_BYTES;
            if (tid == 0) {
                mbar_expect_tx(&full[st], (uint32_t)(2 * TC_A_BYTES));
                tma_load_2d(sb, &tA_hi, k0, op * a.KM + m0, &full[st]);
                tma_load_2d(sb + TC_A_BYTES, &tA_lo, k0, op * a.KM + m0, &full[st]);
            }
            // 128-byte swizzle: row r at (r / 8) * 1024 + (r % 8) * 128, 16-byte chunk c at c ^ (r % 8)
            uint8_t *rowdst = sb + 2 * TC_A_BYTES + (r >> 3) * 1024 + ri * 128;
            if (srow >= 0) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const __half *g = (h ? a.phi_lo : a.phi_hi) + srow * a.KK + k0;
                    uint8_t *d = rowdst + h * TC_B_BYTES;
#pragma unroll
                    for (int c = 0; c < 8; c++) cp_async16(d + ((c ^ ri) << 4), g + c * 8);
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[st]))
                             : "memory");
            } else {
                // a row of the tile without a source in this slot reads zeros; rows past
                // the tile feed output columns that are never stored and stay as they are
                if (r < nr) {
#pragma unroll
                    for (int h = 0; h < 2; h++)
#pragma unroll
                        for (int c = 0; c < 8; c++)
                            *reinterpret_cast<uint4 *>(rowdst + h * TC_B_BYTES + (c << 4)) = make_uint4(0, 0, 0, 0);
                }
                mbar_arrive(&full[st]);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == 4) {
        // ---- MMA issuer: work accumulator u & 1 for drain unit u ----
        if (lane == 0) {
            int it = 0, u = 0;
            bool okm = true;
            for (int si = 0; si < nact && okm; si++) {
                for (int g = 0; g < ngroups && okm; g++, u++) {
                    const int wb = u & 1;
                    if (!mbar_wait(&wfree[wb], ((uint32_t)(u >> 1) & 1u) ^ 1u, a.err)) {
                        okm = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dbig = tmem + wb * 2 * TC_N, dsmall = dbig + TC_N;
                    const int kc1 = min(kchunks, (g + 1) * a.drain);
                    for (int kc = g * a.drain; kc < kc1; kc++, it++) {
                        const int st = it % STAGES;
                        if (!mbar_wait(&full[st], (uint32_t)(it / STAGES) & 1u, a.err)) {
                            okm = false;
                            break;
                        }
                        // rows written by cp.async and plain stores (generic proxy) are read by the MMA
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        tc_fence_after();
                        const uint32_t sb = smem_u32(stages + (size_t)st * TC_STAGE_BYTES);
#pragma unroll
                        for (int k16 = 0; k16 < TC_K / 16; k16++) {
                            const uint64_t a_hi = smem_desc_sw128(sb + k16 * 32);
                            const uint64_t a_lo = smem_desc_sw128(sb + TC_A_BYTES + k16 * 32);
                            const uint64_t b_hl = smem_desc_sw128(sb + 2 * TC_A_BYTES + k16 * 32);
                            tc_mma(dbig, a_hi, b_hl, (kc != g * a.drain || k16) ? 1u : 0u, kIdesc2);
                            tc_mma(dsmall, a_lo, b_hl, 1u);
                        }
                        tc_commit(&empty[st]);
                    }
                    if (okm) tc_commit(&wfull[wb]);
                }
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: drain every work accumulator into fp32 registers ----
        const int sp = warp & 3;  // tensor-memory sub-partition of this warp
        float acc[TC_N];
#pragma unroll
        for (int c = 0; c < TC_N; c++) acc[c] = 0.f;
        bool oke = true;
        const int nunits = nact * ngroups;
        for (int u = 0; u < nunits && oke; u++) {
            const int wb = u & 1;
            bool w = mbar_wait(&wfull[wb], (uint32_t)(u >> 1) & 1u, a.err);
            oke = __all_sync(0xffffffffu, w);  // tcgen05.ld is warp-collective
            if (!oke) break;
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < TC_N; c0 += 16) {
                uint32_t v[16], w2[16];
                const uint32_t ta = tmem + ((uint32_t)(sp * 32) << 16) + wb * 2 * TC_N + c0;
                tc_ld16_nowait(ta, v);
                tc_ld16_nowait(ta + TC_N, w2);
                tc_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; j++) acc[c0 + j] += __uint_as_float(v[j]) + __uint_as_float(w2[j]);
            }
            tc_fence_before();
            mbar_arrive(&wfree[wb]);
        }
        const int krow = m0 + sp * 32 + lane;
        if (oke && krow >= a.msplit && krow < a.mrows) {
            const float unscale = ldexpf(a.rscale ? a.rscale[krow] : 1.0f, -(phi_exp(a.amax) + a.kexp));
            const int w2 = a.mrows - a.msplit, k2 = krow - a.msplit;
#pragma unroll
            for (int c = 0; c < TC_N; c++) {
                const long long d = drow[c];
                if (d >= 0) a.dst2[d * w2 + k2] = acc[c] * unscale;
            }
        } else if (oke && krow < a.msplit) {
            const float unscale = ldexpf(a.rscale ? a.rscale[krow] : 1.0f, -(phi_exp(a.amax) + a.kexp));
            if (a.beta) {
                // the previous values of 16 columns are loaded together (their rows differ,
                // which the compiler cannot see), then updated
#pragma unroll
                for (int c0 = 0; c0 < TC_N; c0 += 16) {
                    float old[16];
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const long long d = drow[c0 + j];
                        old[j] = d >= 0 ? a.dst[d * a.msplit + krow] : 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const long long d = drow[c0 + j];
                        if (d >= 0) a.dst[d * a.msplit + krow] = old[j] + acc[c0 + j] * unscale;
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < TC_N; c++) {
                    const long long d = drow[c];
                    if (d >= 0) a.dst[d * a.msplit + krow] = acc[c] * unscale;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

// The slot groups' partial sums of a split launch, added in group order (the
// result does not depend on scheduling): one thread per (tile, column, output
// component), components fastest; dst (components < msplit, beta: added) and
// dst2 (the rest) as in the epilogue of k_trans_tc.
__global__ void k_trans_reduce(const float *__restrict__ part, int nsplit, int ntl, const int4 *__restrict__ tiles,
                               const int *__restrict__ tboxes, int nrhs, int mrows, int msplit, float *dst,
                               float *dst2, int beta) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)ntl * TC_N * mrows) return;
    const int k = (int)(i % mrows);
    const long long tcol = i / mrows;
    const int c = (int)(tcol % TC_N), ti = (int)(tcol / TC_N);
    const int4 tile = tiles[ti];
    if (c >= tile.z) return;
    const int row = tile.y + c, box = tboxes[row / nrhs];
    const long long d = (long long)box * nrhs + row % nrhs;
    float v = 0.f;
    for (int g = 0; g < nsplit; g++) v += part[(((size_t)g * ntl + ti) * TC_N + c) * mrows + k];
    if (k < msplit) {
        float *o = dst + d * msplit + k;
        *o = beta ? *o + v : v;
    } else {
        dst2[d * (mrows - msplit) + (k - msplit)] = v;
    }
}

// op[o][i][j] (M x K each) * 2^kexp split into fp16 hi/lo, padded to KM x KK: out[h][o][i][j]
__global__ void k_op_split(const double *__restrict__ op, int nops, int M, int K, int KM, int KK, int kexp,
                           __half *__restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long total = (long long)nops * KM * KK;
    if (i >= total) return;
    const int o = (int)(i / ((long long)KM * KK));
    const int rem = (int)(i % ((long long)KM * KK)), r = rem / KK, c = rem % KK;
    double v = (r < M && c < K) ? ldexp(op[((long long)o * M + r) * K + c], kexp) : 0.0;
    const __half hi = __float2half_rn((float)v);
    out[i] = hi;
    out[total + i] = __float2half_rn((float)(v - (double)__half2float(hi)));
}

// The rows a task reads: for task box b (blockIdx.x) and slot s (blockIdx.y),
// source box slot_table[b][s] (or b itself), all its nrhs rows.
__device__ __forceinline__ long long task_src_row(const int *tboxes, const int *slot_table, int stride, int b, int s,
                                                  int nrhs, int rhs) {
    const int box = tboxes[b];
    const int src = slot_table ? slot_table[(long long)box * stride + s] : box;
    return src >= 0 ? (long long)src * nrhs + rhs : -1;
}

// max |x| over the rows a task reads: block-strided over (task box, slot)
// items, one atomic per block
__global__ void k_task_amax(const float *__restrict__ src, const int *__restrict__ tboxes, int nbt,
                            const int *__restrict__ slot_table, int stride, int nslots, int nrhs, int kn,
                            float *amax) {
    __shared__ float red[32];
    float m = 0.f;
    const int kn4 = kn / 4;  // rows start on 16-byte boundaries when kn % 4 == 0
    for (long long it = blockIdx.x; it < (long long)nbt * nslots; it += gridDim.x) {
        const int b = (int)(it / nslots), s = (int)(it % nslots);
        for (int rhs = 0; rhs < nrhs; rhs++) {
            const long long row = task_src_row(tboxes, slot_table, stride, b, s, nrhs, rhs);
            if (row < 0) break;
            const float *x = src + row * kn;
            if ((kn & 3) == 0) {
                const float4 *x4 = reinterpret_cast<const float4 *>(x);
                for (int k = threadIdx.x; k < kn4; k += blockDim.x) {
                    const float4 v = x4[k];
                    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
                }
            } else {
                for (int k = threadIdx.x; k < kn; k += blockDim.x) m = fmaxf(m, fabsf(x[k]));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0 && m > 0.f) atomicMax((int *)amax, __float_as_int(m));  // non-negative floats order as ints
    }
}

// the same rows scaled by 2^e and split into fp16 hi/lo rows of KK (zero padded)
__global__ void k_task_split(const float *__restrict__ src, const int *__restrict__ tboxes,
                             const int *__restrict__ slot_table, int stride, int nrhs, int kn, int KK,
                             const float *amax, __half *__restrict__ hi, __half *__restrict__ lo) {
    const int e = phi_exp(amax);
    for (int rhs = 0; rhs < nrhs; rhs++) {
        const long long row = task_src_row(tboxes, slot_table, stride, blockIdx.x, blockIdx.y, nrhs, rhs);
        if (row < 0) break;
        const float *x = src + row * kn;
        __half2 *h2 = reinterpret_cast<__half2 *>(hi + row * KK), *l2 = reinterpret_cast<__half2 *>(lo + row * KK);
        for (int k2 = threadIdx.x; k2 < KK / 2; k2 += blockDim.x) {
            const int k = 2 * k2;
            const float x0 = k < kn ? ldexpf(x[k], e) : 0.f, x1 = k + 1 < kn ? ldexpf(x[k + 1], e) : 0.f;
            const __half a0 = __float2half_rn(x0), a1 = __float2half_rn(x1);
            h2[k2] = __halves2half2(a0, a1);
            l2[k2] = __halves2half2(__float2half_rn(x0 - __half2float(a0)), __float2half_rn(x1 - __half2float(a1)));
        }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        PK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) throw Error(PKIFMM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = (EncodeTiledFn)p;
    }
    return fn;
}

// one operator set: nops row-major M x K binary64 matrices; output rows
// [0, msplit) and [msplit, M) go to two destinations
void make_ops(TrOps &o, const double *h, int nops, int M, int K, int msplit) {
    o.M = M;
    o.K = K;
    o.msplit = msplit;
    o.KM = (M + TC_M - 1) / TC_M * TC_M;
    o.KK = (K + TC_K - 1) / TC_K * TC_K;
    const int KM = o.KM, KK = o.KK;
    double mx = 0;
    for (size_t i = 0; i < (size_t)nops * M * K; i++) mx = std::max(mx, std::fabs(h[i]));
    int e = 0;
    if (mx > 0) std::frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
    o.kexp = 14 - e;                 // largest entry just below 2^14
    o.nops = nops;
    double *d = nullptr;
    const size_t n = (size_t)nops * M * K, nk = (size_t)nops * KM * KK;
    PK_CUDA(cudaMalloc(&d, n * sizeof(double)));
    PK_CUDA(cudaMemcpy(d, h, n * sizeof(double), cudaMemcpyHostToDevice));
    PK_CUDA(cudaMalloc(&o.op, 2 * nk * sizeof(__half)));
    count_launch(), k_op_split<<<(unsigned)((nk + 255) / 256), 256>>>(d, nops, M, K, KM, KK, o.kexp, o.op);
    PK_CUDA(cudaGetLastError());
    PK_CUDA(cudaDeviceSynchronize());
    cudaFree(d);
    EncodeTiledFn enc = encode_fn();
    for (int hh = 0; hh < 2; hh++) {
        cuuint64_t dims[2] = {(cuuint64_t)KK, (cuuint64_t)nops * KM};
        cuuint64_t strides[1] = {(cuuint64_t)KK * 2};
        cuuint32_t box[2] = {TC_K, TC_M};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = enc(&o.tmap[hh], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, o.op + hh * nk, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) throw Error(PKIFMM_ERR_CUDA, "cuTensorMapEncodeTiled (translation operators) failed");
    }
}

}  // namespace

void trans_tc_release(Plan &P) {
    TrState *t = P.tr;
    if (!t) return;
    for (auto &o : t->ops) cudaFree(o.op);
    cudaFree(t->sinv);
    cudaFree(t->phi);
    cudaFree(t->amax);
    cudaFree(t->err);
    cudaFree(t->part);
    cudaFreeHost(t->err_host);
    delete t;
    P.tr = nullptr;
}

void trans_tc_prepare(Plan &P) {
    const HostOps &H = P.host;
    const int kn = P.kn;
    TrState *t = new TrState;
    P.tr = t;
    if (const char *e = std::getenv("PKIFMM_TRANS_DRAIN"); e && std::atoi(e) >= 1) t->drain = std::atoi(e);
    const size_t kn2 = (size_t)kn * kn;
    std::vector<double> Ut(kn2), Vt(kn2);
    for (int i = 0; i < kn; i++)
        for (int j = 0; j < kn; j++) {
            Ut[(size_t)i * kn + j] = H.U[(size_t)j * kn + i];
            Vt[(size_t)i * kn + j] = H.V[(size_t)j * kn + i];
        }
    make_ops(t->ops[0], Ut.data(), 1, kn, kn, kn);
    make_ops(t->ops[1], H.V.data(), 1, kn, kn, kn);
    make_ops(t->ops[2], Vt.data(), 1, kn, kn, kn);
    make_ops(t->ops[3], H.U.data(), 1, kn, kn, kn);
    make_ops(t->ops[4], H.m2m.data(), 8, kn, kn, kn);
    make_ops(t->ops[5], H.l2l.data(), 8, kn, kn, kn);
    if (P.basis && P.basis->r > 0) {
        // the V-list M2L runs in the basis Ub: the upward passes also write
        // Ub^T phi (stacked below V and below each M2M operator), the downward
        // solve starts from the M2L output in that basis (V^T Ub)
        const int r = P.basis->r;
        const std::vector<double> &Ub = P.basis->Ub;
        std::vector<double> Ubt((size_t)r * kn);
        for (int i = 0; i < kn; i++)
            for (int j = 0; j < r; j++) Ubt[(size_t)j * kn + i] = Ub[(size_t)i * r + j];
        std::vector<double> UbtV((size_t)r * kn), UbtT((size_t)8 * r * kn), VtUb((size_t)kn * r);
        matmul_device(r, kn, kn, Ubt.data(), 0, H.V.data(), 0, UbtV.data(), 0, 1);
        matmul_device(r, kn, kn, Ubt.data(), 0, H.m2m.data(), (long long)kn2, UbtT.data(), (long long)r * kn, 8);
        matmul_device(kn, r, kn, Vt.data(), 0, Ub.data(), 0, VtUb.data(), 0, 1);
        const size_t ms = (size_t)(kn + r) * kn;
        std::vector<double> st((size_t)8 * ms);
        for (int c = 0; c < 8; c++) {
            const double *top = H.m2m.data() + (size_t)c * kn2;
            std::copy(top, top + kn2, st.begin() + (size_t)c * ms);
            std::copy(UbtT.begin() + (size_t)c * r * kn, UbtT.begin() + (size_t)(c + 1) * r * kn,
                      st.begin() + (size_t)c * ms + kn2);
        }
        make_ops(t->ops[7], st.data(), 8, kn + r, kn, kn);
        st.resize(ms);
        std::copy(H.V.begin(), H.V.end(), st.begin());
        std::copy(UbtV.begin(), UbtV.end(), st.begin() + kn2);
        make_ops(t->ops[6], st.data(), 1, kn + r, kn, kn);
        make_ops(t->ops[8], VtUb.data(), 1, kn, r, kn);
    }
    const int km = t->ops[0].KM;
    std::vector<float> sinv(km, 0.f);
    const double cut = H.eps_rel * H.S[0];
    for (int j = 0; j < kn; j++) sinv[j] = H.S[j] > cut ? (float)(1.0 / H.S[j]) : 0.f;
    PK_CUDA(cudaMalloc(&t->sinv, sizeof(float) * km));
    PK_CUDA(cudaMemcpy(t->sinv, sinv.data(), sizeof(float) * km, cudaMemcpyHostToDevice));
    PK_CUDA(cudaMalloc(&t->amax, sizeof(float)));
    PK_CUDA(cudaMalloc(&t->err, sizeof(int)));
    PK_CUDA(cudaMemset(t->err, 0, sizeof(int)));
    PK_CUDA(cudaMallocHost(&t->err_host, sizeof(int)));
    PK_CUDA(cudaFuncSetAttribute(k_trans_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(3)));
}

// 2D (rows) and 3D (rows by eight) tensor maps of one split, 64 x 128 boxes, 128-byte swizzle
static void phi_maps(const __half *base, size_t rows, int KK, CUtensorMap &m1, CUtensorMap &m8) {
    EncodeTiledFn enc = encode_fn();
    const cuuint64_t row = (cuuint64_t)KK * 2;
    {
        cuuint64_t dims[2] = {(cuuint64_t)KK, (cuuint64_t)rows};
        cuuint64_t strides[1] = {row};
        cuuint32_t box[2] = {TC_K, TC_N};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = enc(&m1, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void *)base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) throw Error(PKIFMM_ERR_CUDA, "cuTensorMapEncodeTiled (translation rows) failed");
    }
    {
        cuuint64_t dims[3] = {(cuuint64_t)KK, 8, (cuuint64_t)(rows / 8)};
        cuuint64_t strides[2] = {row, row * 8};
        cuuint32_t box[3] = {TC_K, 1, TC_N};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = enc(&m8, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, (void *)base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) throw Error(PKIFMM_ERR_CUDA, "cuTensorMapEncodeTiled (translation rows by 8) failed");
    }
}

void trans_tc_gemm(Plan &P, int set, const Task &task, const int *slot_table, int slot_stride, const float *src,
                   float *dst, int beta, cudaStream_t s, float *dst2) {
    if (task.ntiles == 0) return;
    TrState *t = P.tr;
    if (!t) throw Error(PKIFMM_ERR_UNSUPPORTED, "tensor-core translations not prepared");
    const TrOps &o = t->ops[set];
    if (!o.op) throw Error(PKIFMM_ERR_UNSUPPORTED, "translation operator set not prepared");
    if (task.nslots > kTrMaxSlots) throw Error(PKIFMM_ERR_INVALID_ARG, "translation task with too many slots");
    if (o.msplit < o.M && (!dst2 || beta)) throw Error(PKIFMM_ERR_INVALID_ARG, "stacked translation needs dst2");
    const int nr = P.nrhs, KK = o.KK;
    const size_t rows = (size_t)P.tree.nbox * nr + 1;
    if (rows > t->phi_rows || KK > t->phi_kk) {
        cudaFree(t->phi);
        t->phi = nullptr;
        t->phi_rows = std::max(t->phi_rows, rows + rows / 4);
        t->phi_kk = std::max(t->phi_kk, KK);
        PK_CUDA(cudaMalloc(&t->phi, 2 * t->phi_rows * t->phi_kk * sizeof(__half)));
    }
    __half *hi = t->phi, *lo = t->phi + t->phi_rows * t->phi_kk;
    const int nbt = (int)task.h_boxes.size();
    const dim3 g(nbt, task.nslots);
    PK_CUDA(cudaMemsetAsync(t->amax, 0, sizeof(float), s));
    const int nitems = nbt * task.nslots;
    count_launch(), k_task_amax<<<std::min(nitems, 2048), 256, 0, s>>>(src, task.boxes.p, nbt, slot_table, slot_stride,
                                                                     task.nslots, nr, o.K, t->amax);
    count_launch(), k_task_split<<<g, 256, 0, s>>>(src, task.boxes.p, slot_table, slot_stride, nr, o.K, KK, t->amax,
                                                   hi, lo);
    TrArgs a;
    std::memset(&a, 0, sizeof a);
    a.phi_hi = hi;
    a.phi_lo = lo;
    a.tboxes = task.boxes.p;
    a.tiles = task.tiles.p;
    a.slot_table = slot_table;
    a.slot_stride = slot_stride;
    a.nslots = task.nslots;
    a.class_ops = task.class_ops.p;
    a.dst = dst;
    a.dst2 = dst2;
    a.beta = beta;
    a.rscale = (set == 0 || set == 2 || set == 8) ? t->sinv : nullptr;
    a.amax = t->amax;
    a.mrows = o.M;
    a.msplit = o.msplit;
    a.KM = o.KM;
    a.KK = KK;
    a.nrhs = nr;
    a.kexp = o.kexp;
    a.drain = t->drain;
    a.err = t->err;
    const int mtiles = o.KM / TC_M;
    CUtensorMap b1[2], b8[2];
    phi_maps(hi, t->phi_rows, KK, b1[0], b8[0]);  // rows as k_task_split writes them: stride KK
    phi_maps(lo, t->phi_rows, KK, b1[1], b8[1]);
    // A launch of few CTAs (the coarse levels of M2M) streams its long K range
    // on a handful of SMs and waits on TMA latency: its slots are split over
    // up to sms / CTAs groups, each CTA writing a partial sum, added after.
    // The group count follows from the task's boxes, not its rows, so that a
    // density vector is summed the same way whatever number of vectors rides along.
    const int ctas = task.ntiles * mtiles;
    if (!t->sms) PK_CUDA(cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, P.device));
    const int ctas1 = (nbt + TC_N - 1) / TC_N * mtiles;  // the CTAs of the task with one vector
    const int nsplit = task.nslots > 1 ? std::min(task.nslots, std::max(1, t->sms / ctas1)) : 1;
    if (nsplit > 1) {
        const size_t need = (size_t)nsplit * task.ntiles * TC_N * o.M;
        if (need > t->part_cap) {
            cudaFree(t->part);
            t->part = nullptr;
            t->part_cap = need;
            PK_CUDA(cudaMalloc(&t->part, need * sizeof(float)));
        }
        a.part = t->part;
        a.nsplit = nsplit;
        a.dst = t->part;
        a.dst2 = nullptr;
        a.msplit = o.M;
        a.beta = 0;
    }
    count_launch(), k_trans_tc<3><<<dim3(ctas, nsplit), TC_THREADS, tc_smem(3), s>>>(o.tmap[0], o.tmap[1], b1[0],
                                                                                     b1[1], b8[0], b8[1], a);
    if (nsplit > 1) {
        const long long n = (long long)task.ntiles * TC_N * o.M;
        count_launch(), k_trans_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
            t->part, nsplit, task.ntiles, task.tiles.p, task.boxes.p, nr, o.M, o.msplit, dst, dst2, beta);
    }
    PK_CUDA(cudaGetLastError());
}

void trans_tc_check(Plan &P, cudaStream_t s) {
    TrState *t = P.tr;
    if (!t) return;
    PK_CUDA(cudaMemcpyAsync(t->err_host, t->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    if (*t->err_host) {
        PK_CUDA(cudaMemset(t->err, 0, sizeof(int)));
        throw Error(PKIFMM_ERR_TIMEOUT, "tensor-core translations: a bounded pipeline wait gave up");
    }
}

}  // namespace pk
