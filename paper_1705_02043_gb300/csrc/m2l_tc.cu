// Tensor-core V-list M2L for the MIXED path (tcgen05, split-fp16 products).
//
// The V-list M2L of Sec. 2.2 in the check formulation,
//     q~d[B] = sum_{slots s} K_{o(class(B), s)} phi_u[V(B, s)],
// is a dense contraction: for the boxes of one octant class every slot s
// uses the same operator K_o (kn x kn), so a CTA computes
//     D[128 kn rows x 128 (box, rhs) columns] = sum_s sum_k K_o[:, k] Phi_s[:, k]^T
// with Phi_s the gathered upward densities.  Operands are scaled by powers of
// two into the fp16 range and split into fp16 pairs x = x_hi + x_lo (22
// significant bits); each product is K_hi Phi_hi + K_hi Phi_lo + K_lo Phi_hi.
//
// Precision: the tensor core accumulates in fp32 but drops low bits at every
// accumulation step, a bias that grows with the number of MMAs summed into
// one accumulator (tens of thousands over all slots).  So each slot's
// contribution is accumulated in tensor memory and then added, rounding to
// nearest, into fp32 registers of the epilogue warps, while the next slot
// accumulates in the other buffer.  Within a slot the large hi*hi products
// and the 2^-11 smaller cross products go to separate accumulators, so the
// large one takes only KK/16 steps per slot.
//
// Pipeline (3 stages of 64 KB): warps 0-3 gather the Phi rows with 16-byte
// cp.async into the 128B-swizzled K-major layout and one thread issues the TMA
// loads of the K_o tiles; warp 4 issues tcgen05.mma from one thread and frees
// each stage with tcgen05.commit; warps 5-8 drain the work accumulators and
// finally write the check potentials.  Every mbarrier wait is bounded in time;
// on timeout the kernel raises an error flag and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "tc_ptx.cuh"

namespace pk {

struct TcState {
    int KM = 0, KK = 0;                  // operator rows padded to 128 (M tiles), columns to 32 (K chunks)
    __half *kop = nullptr;               // [2][316][KM][KK]  (hi, lo), scaled by 2^kexp
    int kexp = 0;
    float *amax = nullptr;               // max |phi| of the current evaluation
    __half *phi = nullptr;        // [2][rows+1][KK]
    size_t phi_rows = 0;
    CUtensorMap tmap[2];
    int4 *tiles = nullptr;
    int ntiles = 0, tiles_cap = 0;
    int *err = nullptr;
    int *err_host = nullptr;
    cudaEvent_t ev[2] = {};
    float last_ms = 0;
    int *slot_off = nullptr;             // [8][189][3]
    __half *grid = nullptr;              // parity sub-grids of the full levels (hi, then lo, per level)
    size_t grid_cap = 0;
    int4 *gtiles = nullptr;
    size_t gtiles_cap = 0;
    int *gboxes = nullptr;
    size_t gboxes_cap = 0;
    int *lmap = nullptr;                 // position -> box maps of the partial grid levels (-1: no box)
    size_t lmap_cap = 0;
    int stages = 3;                      // pipeline depth of the launched instantiation
    int wide = 1;                        // grid levels with two column tiles per CTA (k_m2l_tcw)
    cudaStream_t side[3] = {};           // the per-level launches run concurrently (disjoint outputs)
    cudaEvent_t fork = nullptr, join[3] = {};
};

// ---------------- kernel ----------------

struct TcArgs {
    const __half *phi_hi, *phi_lo;  // gather mode: [rows+1][KK], last row zero
    const int *tboxes;                     // gather mode: task boxes, class-major
    const int4 *tiles;                     // gather: (class, row0, nrows, 0); grid: (class | rblock << 3, i0, j0, k0)
    const int *v_slot;                     // [nbox][189]
    const int *class_ops;                  // [8][189]
    const int *slot_off;                   // [8][189][3] box offsets of the V slots
    float *chk;                            // [nbox*nrhs][kn]
    const float *amax;                     // max |phi|
    int kn, KM, KK, nrhs, zero_row, kexp;
    // grid mode (a level dense enough for 8 parity sub-grids of Phi with a 2-box halo)
    int grid, lvl_begin, zd, bx, by, bz, rb;
    const int *lmap;                       // Morton position -> box, -1 if absent; null: every box exists
    int boxg;                              // gather mode by boxes: a box's nrhs source rows by one 2D TMA
    int *err;
};

template <int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_m2l_tc(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
             const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo, TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)smem;               // [STAGES]
    uint64_t *empty = full + STAGES;              // [STAGES]
    uint64_t *wfull = empty + STAGES;             // [2] work accumulator ready
    uint64_t *wfree = wfull + 2;                     // [2] work accumulator drained
    uint32_t *tmem_slot = (uint32_t *)(wfree + 2);
    int *nact_s = (int *)(tmem_slot + 1);
    short *act = (short *)(nact_s + 1);              // [189]
    long long *drow = (long long *)(smem + 1024);    // [128]
    int *sbox = (int *)(smem + 1024 + 8 * TC_N);     // [128]
    uint8_t *stages = smem + TC_CTRL_BYTES;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // consecutive CTAs: the M tiles of one column tile (they share the
    // gathered rows), then the next column tile of the same octant class
    // (same operator stream), so one class fills a wave
    const int mtiles = a.KM / TC_M;
    const int4 tile = a.tiles[blockIdx.x / mtiles];
    const int cls = a.grid ? (tile.x & 7) : tile.x;
    const int row0 = a.grid ? 0 : tile.y, nr = a.grid ? TC_N : tile.z;
    const int m0 = (blockIdx.x % mtiles) * TC_M;
    const int kchunks = a.KK / TC_K;

    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], a.grid ? 1 : (a.boxg ? 32 : 128));
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
        if (a.grid) {
            // column n = rhs + rb (x + bx (y + by z)) of a block of class-cls boxes
            const int rl = n % a.rb, b = n / a.rb;
            const int x = b % a.bx, y = (b / a.bx) % a.by, z = b / (a.bx * a.by);
            const int px = (cls & 1) + 2 * (tile.y + x), py = (cls >> 1 & 1) + 2 * (tile.z + y),
                      pz = (cls >> 2 & 1) + 2 * (tile.w + z);
            const int m = (int)morton3_dev(px, py, pz);
            const int box = a.lmap ? a.lmap[m] : a.lvl_begin + m;
            drow[n] = box >= 0 ? (long long)box * a.nrhs + (tile.x >> 3) * a.rb + rl : -1;
            sbox[n] = box;
        } else if (n < nr) {
            int row = row0 + n, tb = row / a.nrhs, rhs = row % a.nrhs, box = a.tboxes[tb];
            drow[n] = (long long)box * a.nrhs + rhs;
            sbox[n] = box;
        } else {
            drow[n] = -1;
            sbox[n] = -1;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // slots with at least one source box in this tile
    for (int s = tid; s < kVSlots; s += TC_THREADS) {
        int any = 0;
        if (a.class_ops[cls * kVSlots + s] >= 0) {
            if (a.grid) any = 1;  // missing sources are zero rows of the grids
            else
                for (int n = 0; n < nr && !any; n++) any = a.v_slot[(long long)sbox[n] * kVSlots + s] >= 0;
        }
        act[s] = (short)any;
    }
    __syncthreads();
    if (tid == 0) {
        int c = 0;
        for (int s = 0; s < kVSlots; s++)
            if (act[s]) act[c++] = (short)s;
        *nact_s = c;
    }
    __syncthreads();
    const int nact = *nact_s;
    const uint32_t tmem = *tmem_slot;
    const int total = nact * kchunks;
    // slots summed into one work accumulator before it is drained: about 14 K
    // chunks (the truncation of the tensor core's fp32 accumulation grows with
    // the steps summed in tensor memory)
    const int spd = max(1, 14 / kchunks), nunits = (nact + spd - 1) / spd;

    if (warp < 4 && a.grid) {
        // ---- producer (grid mode): one thread, TMA for both operands ----
        if (tid == 0) {
            int cur_si = -1, op = 0, cx = 0, cy = 0, cz = 0;
            for (int it = 0; it < total; it++) {
                const int st = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (!mbar_wait(&empty[st], ph ^ 1u, a.err)) break;
                const int si = it / kchunks, k0 = (it % kchunks) * TC_K;
                if (si != cur_si) {
                    cur_si = si;
                    const int s = act[si];
                    op = a.class_ops[cls * kVSlots + s];
                    // sources of the block at offset o: parity sub-grid (c + o) mod 2, origin floor((c + o) / 2)
                    const int *o = a.slot_off + (cls * kVSlots + s) * 3;
                    const int qx = (cls & 1) + o[0], qy = (cls >> 1 & 1) + o[1], qz = (cls >> 2 & 1) + o[2];
                    const int par = (qx & 1) | (qy & 1) << 1 | (qz & 1) << 2;
                    cx = ((qx - (qx & 1)) >> 1) + tile.y + 2;
                    cy = ((qy - (qy & 1)) >> 1) + tile.z + 2;
                    cz = par * a.zd + ((qz - (qz & 1)) >> 1) + tile.w + 2;
                }
                uint8_t *sb = stages + (size_t)st * TC_STAGE_BYTES;
                mbar_expect_tx(&full[st], (uint32_t)(2 * TC_A_BYTES + 2 * TC_B_BYTES));
                tma_load_2d(sb, &tA_hi, k0, op * a.KM + m0, &full[st]);
                tma_load_2d(sb + TC_A_BYTES, &tA_lo, k0, op * a.KM + m0, &full[st]);
                const int r0 = (tile.x >> 3) * a.rb;
                tma_load_5d(sb + 2 * TC_A_BYTES, &tB_hi, k0, r0, cx, cy, cz, &full[st]);
                tma_load_5d(sb + 2 * TC_A_BYTES + TC_B_BYTES, &tB_lo, k0, r0, cx, cy, cz, &full[st]);
                mbar_arrive(&full[st]);
            }
        }
    } else if (warp == 0 && a.boxg) {
        // ---- producer (gather by boxes, nrhs >= 8): warp 0.  Lane j < 128/nrhs owns
        // target box j (rows j nrhs .. j nrhs + nrhs - 1 of the tile); its source
        // box's nrhs rows are contiguous in Phi, one 2D TMA per split; absent
        // sources are zero-filled by the warp.  Lane 0 adds the operator tiles.
        const int nbx = TC_N / a.nrhs;
        const int tbox = lane < nbx ? sbox[lane * a.nrhs] : -1;
        int cur_si = -1, op = 0, src = -1;
        for (int it = 0; it < total; it++) {
            const int st = it % STAGES;
            const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
            const bool ok = mbar_wait(&empty[st], ph ^ 1u, a.err);  // every lane acquires the free stage
            if (!__all_sync(0xffffffffu, ok)) break;
            const int si = it / kchunks, k0 = (it % kchunks) * TC_K;
            if (si != cur_si) {
                cur_si = si;
                const int s = act[si];
                op = a.class_ops[cls * kVSlots + s];
                src = tbox >= 0 ? a.v_slot[(long long)tbox * kVSlots + s] : -1;
            }
            const unsigned present = __ballot_sync(0xffffffffu, lane < nbx && src >= 0);
            uint8_t *sb = stages + (size_t)st * TC_STAGE_BYTES;
            const uint32_t rows_b = (uint32_t)a.nrhs * TC_K * 2;  // bytes of one box's rows, one split
            if (lane == 0) {
                mbar_expect_tx(&full[st], (uint32_t)(2 * TC_A_BYTES) + 2u * rows_b * (uint32_t)__popc(present));
                tma_load_2d(sb, &tA_hi, k0, op * a.KM + m0, &full[st]);
                tma_load_2d(sb + TC_A_BYTES, &tA_lo, k0, op * a.KM + m0, &full[st]);
            }
            __syncwarp();
            if (lane < nbx && src >= 0) {
                uint8_t *d = sb + 2 * TC_A_BYTES + (size_t)lane * rows_b;
                tma_load_2d(d, &tB_hi, k0, src * a.nrhs, &full[st]);
                tma_load_2d(d + TC_B_BYTES, &tB_lo, k0, src * a.nrhs, &full[st]);
            }
            // zero rows of absent sources (16-byte stores spread over the warp)
            const unsigned absent = ~present & ((nbx >= 32) ? 0xffffffffu : ((1u << nbx) - 1u));
            for (unsigned m = absent; m; m &= m - 1) {
                const int j = __ffs(m) - 1;
                uint8_t *d = sb + 2 * TC_A_BYTES + (size_t)j * rows_b;
                for (uint32_t o = (uint32_t)lane * 16; o < rows_b; o += 32 * 16) {
                    *reinterpret_cast<uint4 *>(d + o) = make_uint4(0, 0, 0, 0);
                    *reinterpret_cast<uint4 *>(d + TC_B_BYTES + o) = make_uint4(0, 0, 0, 0);
                }
            }
            mbar_arrive(&full[st]);  // 32 arrivals (+ the expected bytes)
        }
    } else if (warp < 4 && a.boxg) {
        // idle producer warps in box-gather mode
    } else if (warp < 4) {
        // ---- producers: gather Phi rows (cp.async) and TMA the operator tiles ----
        // Each thread's row copies arrive on the stage's full barrier when
        // they land (cp.async.mbarrier.arrive.noinc), so all stages stay in
        // flight; the MMA thread fences the async proxy before reading them.
        const int r = tid;
        const int rhs = (row0 + r) % a.nrhs, box = sbox[r];
        const int ri = r & 7;
        int cur_si = -1, op = 0;
        long long srow = -1;  // -1: no source box in this slot (zeros)
        for (int it = 0; it < total; it++) {
            const int st = it % STAGES;
            const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
            if (!mbar_wait(&empty[st], ph ^ 1u, a.err)) break;
            const int si = it / kchunks, k0 = (it % kchunks) * TC_K;
            if (si != cur_si) {  // new slot: its operator and this row's source
                cur_si = si;
                const int s = act[si];
                op = a.class_ops[cls * kVSlots + s];
                int src = box >= 0 ? a.v_slot[(long long)box * kVSlots + s] : -1;
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
                // absent source: zeros written here, no global read (a shared
                // zero row read by every CTA would serialise on one L2 line);
                // rows past the tile feed output columns that are never stored
                if (r < nr) {
#pragma unroll
                    for (int h = 0; h < 2; h++)
#pragma unroll
                        for (int c = 0; c < 8; c++)
                            *reinterpret_cast<uint4 *>(rowdst + h * TC_B_BYTES + (c << 4)) = make_uint4(0, 0, 0, 0);
                }
                mbar_arrive(&full[st]);  // release: orders the zero stores before the MMA's acquire
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == 4) {
        // ---- MMA issuer: spd slots per work accumulator (one drain unit) ----
        if (lane == 0) {
            int it = 0;
            bool okm = true;
            for (int u = 0; u < nunits && okm; u++) {
                const int wb = u & 1;
                if (!mbar_wait(&wfree[wb], ((uint32_t)(u >> 1) & 1u) ^ 1u, a.err)) break;
                tc_fence_after();
                // buffer wb: columns [256 wb, 256 wb + 128) hold hi*hi, the next 128 the cross terms
                const uint32_t dbig = tmem + wb * 2 * TC_N, dsmall = dbig + TC_N;
                const int si0 = u * spd, si1 = min(nact, si0 + spd);
                for (int si = si0; si < si1 && okm; si++)
                for (int kc = 0; kc < kchunks; kc++, it++) {
                    const int st = it % STAGES;
                    if (!mbar_wait(&full[st], (uint32_t)(it / STAGES) & 1u, a.err)) {
                        okm = false;
                        break;
                    }
                    // rows written by cp.async (generic proxy) are read by the MMA (async proxy)
                    if (!a.grid) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tc_fence_after();
                    const uint32_t sb = smem_u32(stages + (size_t)st * TC_STAGE_BYTES);
#pragma unroll
                    for (int k16 = 0; k16 < TC_K / 16; k16++) {
                        const uint64_t a_hi = smem_desc_sw128(sb + k16 * 32);
                        const uint64_t a_lo = smem_desc_sw128(sb + TC_A_BYTES + k16 * 32);
                        const uint64_t b_hl = smem_desc_sw128(sb + 2 * TC_A_BYTES + k16 * 32);  // B_hi then B_lo
                        // A_hi [B_hi | B_lo] -> [hi*hi | hi*lo] in one N = 256 MMA, then lo*hi onto the cross terms
                        tc_mma(dbig, a_hi, b_hl, (si != si0 || kc | k16) ? 1u : 0u, kIdesc2);
                        tc_mma(dsmall, a_lo, b_hl, 1u);
                    }
                    tc_commit(&empty[st]);
                }
                if (okm) tc_commit(&wfull[wb]);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: drain each slot's work accumulator into fp32 registers ----
        const int sp = warp & 3;  // tensor-memory sub-partition of this warp
        float acc[TC_N];
#pragma unroll
        for (int c = 0; c < TC_N; c++) acc[c] = 0.f;
        bool oke = true;
        for (int u = 0; u < nunits && oke; u++) {
            const int wb = u & 1;
            bool w = mbar_wait(&wfull[wb], (uint32_t)(u >> 1) & 1u, a.err);
            oke = __all_sync(0xffffffffu, w);  // tcgen05.ld is warp-collective
            if (!oke) break;
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < TC_N; c0 += 16) {
                uint32_t v[16], u[16];
                const uint32_t ta = tmem + ((uint32_t)(sp * 32) << 16) + wb * 2 * TC_N + c0;
                tc_ld16_nowait(ta, v);
                tc_ld16_nowait(ta + TC_N, u);
                tc_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; j++) acc[c0 + j] += __uint_as_float(v[j]) + __uint_as_float(u[j]);
            }
            tc_fence_before();
            mbar_arrive(&wfree[wb]);
        }
        const float unscale = ldexpf(1.0f, -(phi_exp(a.amax) + a.kexp));
        const int krow = m0 + sp * 32 + lane;
        if (krow < a.kn) {
#pragma unroll
            for (int c = 0; c < TC_N; c++) {
                long long d = drow[c];
                if (d >= 0) a.chk[d * a.kn + krow] = acc[c] * unscale;
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

// ---------------- grid mode, two column tiles per CTA ----------------
//
// The same contraction for two column tiles of one octant class and row block
// (256 (box, rhs) columns): each K_o tile staged once serves both, so the
// operator stream a CTA reads is halved per output column.  Per 16-wide K
// step three N = 256 MMAs: A_hi [B_hi0 | B_hi1] into the hi*hi accumulator,
// A_hi [B_lo0 | B_lo1] and A_lo [B_hi0 | B_hi1] into the cross accumulator;
// together they fill tensor memory (512 columns), so there is one work
// accumulator and the next slot's MMAs wait for the drain of the last.
// Warp 0 issues the TMA loads (one thread), warp 1 the MMAs (one thread) and
// owns the tensor memory, warps 4-11 drain (warp w: lanes 32 (w % 4) .. + 31 of
// tile (w - 4) / 4); warps 2-3 idle.  Two stages of 96 KB.  A pair whose
// second tile carries bit 30 in .x repeats the first tile and writes nothing
// for it (odd tile counts).
constexpr int TCW_THREADS = 384;
constexpr int TCW_STAGE_BYTES = 2 * TC_A_BYTES + 4 * TC_B_BYTES;  // 96 KB
constexpr int tcw_smem(int stages) { return TC_CTRL_BYTES + stages * TCW_STAGE_BYTES + TC_SLACK + 1024; }
constexpr int TCW_SKIP = 1 << 30;

template <int STAGES>
__global__ void __launch_bounds__(TCW_THREADS, 1)
    k_m2l_tcw(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
              const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo, TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)smem;                 // [STAGES]
    uint64_t *empty = full + STAGES;                   // [STAGES]
    uint64_t *wfull = empty + STAGES;                  // work accumulator ready
    uint64_t *wfree = wfull + 1;                       // work accumulator drained
    uint32_t *tmem_slot = (uint32_t *)(wfree + 1);
    int *nact_s = (int *)(tmem_slot + 1);
    short *act = (short *)(nact_s + 1);                // [189]
    long long *drow = (long long *)(smem + 1024);      // [256]
    uint8_t *stages = smem + TC_CTRL_BYTES;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mtiles = a.KM / TC_M;
    const int pair = blockIdx.x / mtiles;
    const int m0 = (blockIdx.x % mtiles) * TC_M;
    int4 tl[2] = {a.tiles[2 * pair], a.tiles[2 * pair + 1]};
    const bool skip1 = (tl[1].x & TCW_SKIP) != 0;
    tl[1].x &= ~TCW_SKIP;
    const int cls = tl[0].x & 7, rblk = tl[0].x >> 3;
    const int kchunks = a.KK / TC_K;

    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(wfull, 1);
        mbar_init(wfree, 256);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int n = tid; n < 2 * TC_N; n += TCW_THREADS) {
        // column n: tile n / 128; within it rhs + rb (x + bx (y + by z)) as in the one-tile kernel
        const int h = n / TC_N, nn = n % TC_N;
        const int4 tile = tl[h];
        const int rl = nn % a.rb, b = nn / a.rb;
        const int x = b % a.bx, y = (b / a.bx) % a.by, z = b / (a.bx * a.by);
        const int px = (cls & 1) + 2 * (tile.y + x), py = (cls >> 1 & 1) + 2 * (tile.z + y),
                  pz = (cls >> 2 & 1) + 2 * (tile.w + z);
        const int m = (int)morton3_dev(px, py, pz);
        const int box = a.lmap ? a.lmap[m] : a.lvl_begin + m;
        drow[n] = (box >= 0 && !(h == 1 && skip1)) ? (long long)box * a.nrhs + rblk * a.rb + rl : -1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    for (int s = tid; s < kVSlots; s += TCW_THREADS) act[s] = (short)(a.class_ops[cls * kVSlots + s] >= 0);
    __syncthreads();
    if (tid == 0) {
        int c = 0;
        for (int s = 0; s < kVSlots; s++)
            if (act[s]) act[c++] = (short)s;
        *nact_s = c;
    }
    __syncthreads();
    const int nact = *nact_s;
    const uint32_t tmem = *tmem_slot;
    const int total = nact * kchunks;
    const int spd = max(1, 14 / kchunks), nunits = (nact + spd - 1) / spd;  // slots per drain, as above

    if (warp == 0) {
        // ---- producer: TMA of the K_o tiles and of both column tiles' sources ----
        if (lane == 0) {
            int cur_si = -1, op = 0, cx[2] = {0, 0}, cy[2] = {0, 0}, cz[2] = {0, 0};
            for (int it = 0; it < total; it++) {
                const int st = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (!mbar_wait(&empty[st], ph ^ 1u, a.err)) break;
                const int si = it / kchunks, k0 = (it % kchunks) * TC_K;
                if (si != cur_si) {
                    cur_si = si;
                    const int s = act[si];
                    op = a.class_ops[cls * kVSlots + s];
                    const int *o = a.slot_off + (cls * kVSlots + s) * 3;
                    const int qx = (cls & 1) + o[0], qy = (cls >> 1 & 1) + o[1], qz = (cls >> 2 & 1) + o[2];
                    const int par = (qx & 1) | (qy & 1) << 1 | (qz & 1) << 2;
                    for (int h = 0; h < 2; h++) {
                        cx[h] = ((qx - (qx & 1)) >> 1) + tl[h].y + 2;
                        cy[h] = ((qy - (qy & 1)) >> 1) + tl[h].z + 2;
                        cz[h] = par * a.zd + ((qz - (qz & 1)) >> 1) + tl[h].w + 2;
                    }
                }
                uint8_t *sb = stages + (size_t)st * TCW_STAGE_BYTES;
                mbar_expect_tx(&full[st], (uint32_t)TCW_STAGE_BYTES);
                tma_load_2d(sb, &tA_hi, k0, op * a.KM + m0, &full[st]);
                tma_load_2d(sb + TC_A_BYTES, &tA_lo, k0, op * a.KM + m0, &full[st]);
                const int r0 = rblk * a.rb;
                uint8_t *b = sb + 2 * TC_A_BYTES;  // B_hi0, B_hi1, B_lo0, B_lo1
                for (int h = 0; h < 2; h++) {
                    tma_load_5d(b + h * TC_B_BYTES, &tB_hi, k0, r0, cx[h], cy[h], cz[h], &full[st]);
                    tma_load_5d(b + (2 + h) * TC_B_BYTES, &tB_lo, k0, r0, cx[h], cy[h], cz[h], &full[st]);
                }
                mbar_arrive(&full[st]);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer: the single work accumulator, one slot at a time ----
        if (lane == 0) {
            int it = 0;
            bool okm = true;
            const uint32_t dhh = tmem, dx = tmem + 2 * TC_N;  // columns [0, 256) hi*hi, [256, 512) cross
            for (int u = 0; u < nunits && okm; u++) {
                if (!mbar_wait(wfree, ((uint32_t)u & 1u) ^ 1u, a.err)) break;
                tc_fence_after();
                const int si0 = u * spd, si1 = min(nact, si0 + spd);
                for (int si = si0; si < si1 && okm; si++)
                for (int kc = 0; kc < kchunks; kc++, it++) {
                    const int st = it % STAGES;
                    if (!mbar_wait(&full[st], (uint32_t)(it / STAGES) & 1u, a.err)) {
                        okm = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sb = smem_u32(stages + (size_t)st * TCW_STAGE_BYTES);
#pragma unroll
                    for (int k16 = 0; k16 < TC_K / 16; k16++) {
                        const uint64_t a_hi = smem_desc_sw128(sb + k16 * 32);
                        const uint64_t a_lo = smem_desc_sw128(sb + TC_A_BYTES + k16 * 32);
                        const uint64_t b_hi = smem_desc_sw128(sb + 2 * TC_A_BYTES + k16 * 32);  // B_hi0 | B_hi1
                        const uint64_t b_lo = smem_desc_sw128(sb + 2 * TC_A_BYTES + 2 * TC_B_BYTES + k16 * 32);
                        const uint32_t first = (si != si0 || kc | k16) ? 1u : 0u;
                        tc_mma(dhh, a_hi, b_hi, first, kIdesc2);
                        tc_mma(dx, a_hi, b_lo, first, kIdesc2);
                        tc_mma(dx, a_lo, b_hi, 1u, kIdesc2);
                    }
                    tc_commit(&empty[st]);
                }
                if (okm) tc_commit(wfull);
            }
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ---- epilogue: tile h of the pair, lanes of this warp's sub-partition ----
        const int sp = warp & 3, h = (warp - 4) >> 2;
        float acc[TC_N];
#pragma unroll
        for (int c = 0; c < TC_N; c++) acc[c] = 0.f;
        bool oke = true;
        for (int u = 0; u < nunits && oke; u++) {
            bool w = mbar_wait(wfull, (uint32_t)u & 1u, a.err);
            oke = __all_sync(0xffffffffu, w);
            if (!oke) break;
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < TC_N; c0 += 16) {
                uint32_t v[16], u[16];
                const uint32_t ta = tmem + ((uint32_t)(sp * 32) << 16) + h * TC_N + c0;
                tc_ld16_nowait(ta, v);
                tc_ld16_nowait(ta + 2 * TC_N, u);
                tc_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; j++) acc[c0 + j] += __uint_as_float(v[j]) + __uint_as_float(u[j]);
            }
            tc_fence_before();
            mbar_arrive(wfree);
        }
        const float unscale = ldexpf(1.0f, -(phi_exp(a.amax) + a.kexp));
        const int krow = m0 + sp * 32 + lane;
        if (krow < a.kn) {
#pragma unroll
            for (int c = 0; c < TC_N; c++) {
                long long d = drow[h * TC_N + c];
                if (d >= 0) a.chk[d * a.kn + krow] = acc[c] * unscale;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

// ---------------- set-up and launch ----------------

// K_o * 2^kexp split into fp16 hi/lo, padded to KM x KK: out[h][op][i][j]
__global__ void k_kop_split(int kernel, int n, int KM, int KK, int kexp, const double *__restrict__ g,
                            const int *__restrict__ offs, __half *__restrict__ out) {
    const int kk = kernel == 0 ? 1 : 3, kn = n * kk;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)kM2LOps * KM * KK;
    if (i >= total) return;
    int m = (int)(i / ((long long)KM * KK));
    int rem = (int)(i % ((long long)KM * KK)), r = rem / KK, c = rem % KK;
    double v = 0.0;
    if (r < kn && c < kn) {
        int pa = r / kk, ca = r % kk, pb = c / kk, cb = c % kk;
        double d[3];
        for (int q = 0; q < 3; q++) d[q] = 0.525 * g[3 * pa + q] - (offs[3 * m + q] + 0.525 * g[3 * pb + q]);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], ir = 1.0 / sqrt(r2);
        if (kernel == 0) v = ir;
        else v = (1.0 / (8.0 * 3.14159265358979323846)) * ((ca == cb ? ir : 0.0) + d[ca] * d[cb] * ir * ir * ir);
    }
    v = ldexp(v, kexp);
    __half hi = __float2half_rn((float)v);
    __half lo = __float2half_rn((float)(v - (double)__half2float(hi)));
    out[i] = hi;
    out[total + i] = lo;
}

// C_o (r x r, binary32) * 2^kexp split into fp16 hi/lo, padded to KM x KK: out[h][op][i][j]
__global__ void k_cop_split(const float *__restrict__ C, int r, int KM, int KK, int kexp, __half *__restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)kM2LOps * KM * KK;
    if (i >= total) return;
    int m = (int)(i / ((long long)KM * KK));
    int rem = (int)(i % ((long long)KM * KK)), a = rem / KK, c = rem % KK;
    const float v = (a < r && c < r) ? ldexpf(C[((long long)m * r + a) * r + c], kexp) : 0.f;
    __half hi = __float2half_rn(v);
    out[i] = hi;
    out[total + i] = __float2half_rn(v - __half2float(hi));
}

__global__ void k_amax(const float *__restrict__ x, long long n, float *amax) {
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax((int *)amax, __float_as_int(m));  // non-negative floats order as ints
}

// upward densities (fp32 rows of kn) * 2^e -> fp16 hi/lo rows of KP (= KK), plus one zero row
__global__ void k_phi_split(const float *__restrict__ up, long long rows, int kn, int KP, const float *amax,
                            __half *__restrict__ hi, __half *__restrict__ lo) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (rows + 1) * KP;
    if (i >= total) return;
    long long r = i / KP;
    int c = (int)(i % KP);
    float x = (r < rows && c < kn) ? ldexpf(up[r * kn + c], phi_exp(amax)) : 0.f;
    __half h = __float2half_rn(x);
    hi[i] = h;
    lo[i] = __float2half_rn(x - __half2float(h));
}

// map[Morton position] = box for the cnt boxes of one level (map preset to -1)
__global__ void k_level_map(const int4 *__restrict__ bpos, int lb, int cnt, int *__restrict__ map) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    int4 p = bpos[lb + i];
    map[morton3_dev(p.x, p.y, p.z)] = lb + i;
}

// Phi of one level as 8 parity sub-grids with a 2-box halo:
// row (((par * Zd + z') * Yd + y') * Xd + x') * nrhs + rhs holds the box at
// position 2 (x' - 2) + (par & 1), ... (wrapped on periodic axes, zero outside
// on free axes and where the level has no box), scaled and split like k_phi_split.
// lmap (nullable): Morton position -> box at this level, -1 where no box exists.
// One block per grid row; the row's position is decoded once.
__global__ void k_phi_grid(const float *__restrict__ up, int lvl_begin, const int *__restrict__ lmap, int n, int nrhs,
                           int kn, int KP, unsigned per, const float *amax, long long rows, __half *__restrict__ hi,
                           __half *__restrict__ lo) {
    const long long row = blockIdx.x;
    if (row >= rows) return;
    const int d = n / 2 + 4;
    long long rest = row / nrhs;
    const int rhs = (int)(row % nrhs);
    const int xq = (int)(rest % d);
    rest /= d;
    const int yq = (int)(rest % d);
    rest /= d;
    const int zq = (int)(rest % d);
    const int par = (int)(rest / d);
    int pos[3] = {2 * (xq - 2) + (par & 1), 2 * (yq - 2) + (par >> 1 & 1), 2 * (zq - 2) + (par >> 2 & 1)};
    bool inside = true;
    for (int a = 0; a < 3; a++) {
        if (per >> a & 1) pos[a] = ((pos[a] % n) + n) % n;
        else if (pos[a] < 0 || pos[a] >= n) inside = false;
    }
    int box = -1;
    if (inside) {
        const int m = (int)morton3_dev(pos[0], pos[1], pos[2]);
        box = lmap ? lmap[m] : lvl_begin + m;
    }
    const float *src = box >= 0 ? up + ((long long)box * nrhs + rhs) * kn : nullptr;
    const int e = phi_exp(amax);
    for (int k = threadIdx.x; k < KP; k += blockDim.x) {
        const float x = (src && k < kn) ? ldexpf(src[k], e) : 0.f;
        const __half h = __float2half_rn(x);
        hi[row * KP + k] = h;
        lo[row * KP + k] = __float2half_rn(x - __half2float(h));
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
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

static bool tc_supported() {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return major == 10 && minor == 3;
}

void m2l_tc_release(Plan &P) {
    TcState *t = P.tc;
    if (!t) return;
    cudaFree(t->kop);
    cudaFree(t->phi);
    cudaFree(t->tiles);
    cudaFree(t->amax);
    cudaFree(t->slot_off);
    cudaFree(t->grid);
    cudaFree(t->gtiles);
    cudaFree(t->gboxes);
    cudaFree(t->lmap);
    for (int i = 0; i < 3; i++) {
        if (t->side[i]) cudaStreamDestroy(t->side[i]);
        if (t->join[i]) cudaEventDestroy(t->join[i]);
    }
    if (t->fork) cudaEventDestroy(t->fork);
    cudaFree(t->err);
    cudaFreeHost(t->err_host);
    if (t->ev[0]) cudaEventDestroy(t->ev[0]);
    if (t->ev[1]) cudaEventDestroy(t->ev[1]);
    delete t;
    P.tc = nullptr;
}

void m2l_tc_prepare(Plan &P) {
    if (!tc_supported()) throw Error(PKIFMM_ERR_UNSUPPORTED, "MIXED path needs an sm_103 GPU (tcgen05)");
    TcState *t = new TcState;
    P.tc = t;
    // dense operators (kn x kn) or their images C_o = Ub^T K_o Ub in the shared basis (r x r)
    const int rk = P.basis ? P.basis->r : P.kn;
    t->KM = (rk + TC_M - 1) / TC_M * TC_M;
    t->KK = (rk + TC_K - 1) / TC_K * TC_K;
    const int KM = t->KM, KK = t->KK;
    size_t nk = (size_t)kM2LOps * KM * KK;
    PK_CUDA(cudaMalloc(&t->kop, 2 * nk * sizeof(__half)));
    if (P.basis) {
        const std::vector<float> &C = P.basis->C;
        float mx = 0.f;
        for (float v : C) mx = std::max(mx, std::fabs(v));
        int e = 0;
        if (mx > 0.f) std::frexp(mx, &e);
        t->kexp = 14 - e;  // largest entry just below 2^14
        float *dc = nullptr;
        PK_CUDA(cudaMalloc(&dc, sizeof(float) * C.size()));
        PK_CUDA(cudaMemcpy(dc, C.data(), sizeof(float) * C.size(), cudaMemcpyHostToDevice));
        count_launch(), k_cop_split<<<(unsigned)((nk + 255) / 256), 256>>>(dc, rk, KM, KK, t->kexp, t->kop);
        PK_CUDA(cudaGetLastError());
        PK_CUDA(cudaDeviceSynchronize());
        cudaFree(dc);
    } else {
        // |K_o| <= 1/0.95 (Laplace) or 2/(8 pi 0.95) (Stokes) over the 316 offsets
        // (closest points 0.95 box edges apart): scale the largest entry to about 2^12
        t->kexp = P.kernel == 0 ? 12 : 15;
        std::vector<int> offs;
        for (int x = -3; x <= 3; x++)
            for (int y = -3; y <= 3; y++)
                for (int z = -3; z <= 3; z++) {
                    if (std::max(std::abs(x), std::max(std::abs(y), std::abs(z))) <= 1) continue;
                    offs.push_back(x);
                    offs.push_back(y);
                    offs.push_back(z);
                }
        int *doffs = nullptr;
        PK_CUDA(cudaMalloc(&doffs, sizeof(int) * offs.size()));
        PK_CUDA(cudaMemcpy(doffs, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice));
        count_launch(), k_kop_split<<<(unsigned)((nk + 255) / 256), 256>>>(P.kernel, P.n, KM, KK, t->kexp, P.g64.p,
                                                                            doffs, t->kop);
        PK_CUDA(cudaGetLastError());
        PK_CUDA(cudaDeviceSynchronize());
        cudaFree(doffs);
    }
    EncodeTiledFn enc = encode_fn();
    for (int h = 0; h < 2; h++) {
        cuuint64_t dims[2] = {(cuuint64_t)KK, (cuuint64_t)kM2LOps * KM};
        cuuint64_t strides[1] = {(cuuint64_t)KK * 2};
        cuuint32_t box[2] = {TC_K, TC_M};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = enc(&t->tmap[h], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, t->kop + h * nk, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) throw Error(PKIFMM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    }
    {  // box offset of each V slot, per octant class (the enumeration of the slot tables)
        std::vector<int> so(8 * kVSlots * 3, 0);
        for (int c = 0; c < 8; c++) {
            int cb[3] = {c & 1, c >> 1 & 1, c >> 2 & 1}, sl = 0;
            for (int x = -2 - cb[0]; x <= 3 - cb[0]; x++)
                for (int y = -2 - cb[1]; y <= 3 - cb[1]; y++)
                    for (int z = -2 - cb[2]; z <= 3 - cb[2]; z++) {
                        if (std::max(std::abs(x), std::max(std::abs(y), std::abs(z))) <= 1) continue;
                        so[(c * kVSlots + sl) * 3] = x;
                        so[(c * kVSlots + sl) * 3 + 1] = y;
                        so[(c * kVSlots + sl) * 3 + 2] = z;
                        sl++;
                    }
        }
        PK_CUDA(cudaMalloc(&t->slot_off, sizeof(int) * so.size()));
        PK_CUDA(cudaMemcpy(t->slot_off, so.data(), sizeof(int) * so.size(), cudaMemcpyHostToDevice));
    }
    PK_CUDA(cudaMalloc(&t->amax, sizeof(float)));
    PK_CUDA(cudaMalloc(&t->err, sizeof(int)));
    PK_CUDA(cudaMemset(t->err, 0, sizeof(int)));
    PK_CUDA(cudaMallocHost(&t->err_host, sizeof(int)));
    PK_CUDA(cudaEventCreate(&t->ev[0]));
    PK_CUDA(cudaEventCreate(&t->ev[1]));
    PK_CUDA(cudaFuncSetAttribute(k_m2l_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(2)));
    PK_CUDA(cudaFuncSetAttribute(k_m2l_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(3)));
    // pipeline depth: 3 stages of 64 KB (192 KB of operands in flight); 2 for timing comparisons
    t->stages = 3;
    if (const char *e = std::getenv("PKIFMM_M2L_STAGES"))
        if (std::atoi(e) == 2) t->stages = 2;
    // two column tiles per CTA on the grid levels; PKIFMM_M2L_WIDE=0 launches one
    // tile per CTA there (timing comparisons; the results are the same)
    PK_CUDA(cudaFuncSetAttribute(k_m2l_tcw<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcw_smem(2)));
    if (const char *e = std::getenv("PKIFMM_M2L_WIDE"))
        if (std::atoi(e) == 0) t->wide = 0;
}

namespace {

struct GridPlan {
    int level, n, bx, by, bz, rb;
    long long rows;
    size_t off;            // element offset of the hi grid in TcState::grid
    long long map_off;     // offset of the level's position map in TcState::lmap, -1 if the level is full
};

constexpr size_t kGridBytesMax = 24ull << 30;  // device memory the parity grids may take

template <typename T>
void grow(T *&p, size_t &cap, size_t n) {
    if (n <= cap) return;
    cudaFree(p);
    p = nullptr;
    cap = n + n / 4 + 16;
    PK_CUDA(cudaMalloc(&p, cap * sizeof(T)));
}

}  // namespace

bool m2l_tc_run(Plan &P, cudaStream_t s) {
    TcState *t = P.tc;
    if (!t) return false;
    const Task &task = P.t_m2l;
    if (task.nrows == 0) return true;
    const int KK = t->KK, nr = P.nrhs, mtiles = t->KM / TC_M;
    // sources and results: phi_u and the check rows, or both in the shared basis
    const int rk = P.basis ? P.basis->r : P.kn;
    const float *up = P.basis ? P.uphat32.p : P.up32.p;
    float *chk = P.basis ? P.chkhat32.p : P.chk32.p;
    const std::vector<int> &lb = P.tree.lvl_begin;
    const int nlev = (int)lb.size() - 1;
    long long rows = (long long)P.tree.nbox * nr;

    // levels holding at least 70% of their 8^l boxes run with TMA-loaded
    // operands (grid mode): the V-list source of a box at position p and slot
    // offset o is the box at p + o if it exists, so parity grids with zero
    // rows where no box exists reproduce the lists exactly.  Below that the
    // gather path, about 1.5x slower per tile, wins (measured: a level 48% full
    // took 32.7 ms in grid mode, 22.8 ms gathered).
    std::vector<GridPlan> gp;
    std::vector<char> is_grid(nlev, 0);
    int rb = 0;
    if (P.nprob == 1 && nr <= 128 && (nr & (nr - 1)) == 0) rb = nr;  // one tree: positions index one level
    size_t grid_elems = 0, map_elems = 0;
    if (rb) {
        int e = 0;
        while ((1 << e) < 128 / rb) e++;
        const int ez = e / 3, ey = (e - ez) / 2, ex = e - ey - ez;
        for (int l = 1; l < nlev && l <= 9; l++) {
            long long cnt = lb[l + 1] - lb[l];
            const int n = 1 << l;
            const long long full = 1LL << (3 * l);
            if (cnt * 10 < full * 7 || (n / 2) < (1 << ex)) continue;
            GridPlan g{l, n, 1 << ex, 1 << ey, 1 << ez, rb, 0, 0, -1};
            const long long d = n / 2 + 4;
            g.rows = 8 * d * d * d * nr;
            if ((grid_elems + 2 * (size_t)g.rows * KK) * sizeof(__half) > kGridBytesMax) continue;
            g.off = grid_elems;
            grid_elems += 2 * (size_t)g.rows * KK;
            if (cnt != full) {
                g.map_off = (long long)map_elems;
                map_elems += (size_t)full;
            }
            gp.push_back(g);
            is_grid[l] = 1;
        }
    }
    if (map_elems) {
        grow(t->lmap, t->lmap_cap, map_elems);
        PK_CUDA(cudaMemsetAsync(t->lmap, 0xff, sizeof(int) * map_elems, s));
        for (auto &g : gp)
            if (g.map_off >= 0) {
                const int cnt = lb[g.level + 1] - lb[g.level];
                count_launch(), k_level_map<<<(cnt + 255) / 256, 256, 0, s>>>(P.tree.bpos.p, lb[g.level], cnt,
                                                                              t->lmap + g.map_off);
            }
    }
    PK_CUDA(cudaMemsetAsync(t->amax, 0, sizeof(float), s));
    count_launch(), k_amax<<<1024, 256, 0, s>>>(up, rows * rk, t->amax);

    // remaining boxes: gather mode, class-major
    std::vector<int> gbox;
    std::vector<int4> gtiles;
    for (int c = 0, b0 = 0; c < task.nclass; c++) {
        const int start = (int)gbox.size();
        for (int i = 0; i < task.class_count[c]; i++) {
            const int b = task.h_boxes[b0 + i];
            const int l = P.h_bpos ? P.h_bpos[b].w : (int)(std::upper_bound(lb.begin(), lb.end(), b) - lb.begin()) - 1;
            if (!is_grid[l]) gbox.push_back(b);
        }
        b0 += task.class_count[c];
        const int rows_c = ((int)gbox.size() - start) * nr;
        for (int r = 0; r < rows_c; r += TC_N)
            gtiles.push_back(make_int4(c, start * nr + r, std::min(TC_N, rows_c - r), 0));
    }
    // grid tiles: (class | rblock << 3, i0, j0, k0) per level; on partial
    // levels only blocks holding a box with targets
    std::vector<int> gt_begin;
    for (auto &g : gp) {
        gt_begin.push_back((int)gtiles.size());
        const int h = g.n / 2;
        std::vector<char> occ;  // [class][block] has a target box (partial levels)
        const int bxn = h / g.bx, byn = h / g.by, bzn = h / g.bz;
        if (g.map_off >= 0) {
            const int cnt = lb[g.level + 1] - lb[g.level];
            // the level's boxes: from the tree read back for the tasks, else read here
            std::vector<int4> bpv;
            std::vector<int2> trv;
            const int4 *bp = P.h_bpos ? P.h_bpos + lb[g.level] : nullptr;
            const int2 *tr = P.h_trange ? P.h_trange + lb[g.level] : nullptr;
            if (!bp || !tr) {
                bpv.resize(cnt);
                trv.resize(cnt);
                PK_CUDA(cudaMemcpyAsync(bpv.data(), P.tree.bpos.p + lb[g.level], sizeof(int4) * cnt,
                                        cudaMemcpyDeviceToHost, s));
                PK_CUDA(cudaMemcpyAsync(trv.data(), P.tree.trange.p + lb[g.level], sizeof(int2) * cnt,
                                        cudaMemcpyDeviceToHost, s));
                PK_CUDA(cudaStreamSynchronize(s));
                bp = bpv.data();
                tr = trv.data();
            }
            occ.assign((size_t)8 * bxn * byn * bzn, 0);
            for (int i = 0; i < cnt; i++) {
                if (tr[i].y <= tr[i].x) continue;
                const int c = (bp[i].x & 1) | (bp[i].y & 1) << 1 | (bp[i].z & 1) << 2;
                const int bi = (bp[i].x >> 1) / g.bx, bj = (bp[i].y >> 1) / g.by, bk = (bp[i].z >> 1) / g.bz;
                occ[(((size_t)c * bzn + bk) * byn + bj) * bxn + bi] = 1;
            }
        }
        for (int c = 0; c < 8; c++)
            for (int r = 0; r < nr / g.rb; r++)
                for (int k0 = 0; k0 < h; k0 += g.bz)
                    for (int j0 = 0; j0 < h; j0 += g.by)
                        for (int i0 = 0; i0 < h; i0 += g.bx) {
                            if (!occ.empty() &&
                                !occ[(((size_t)c * bzn + k0 / g.bz) * byn + j0 / g.by) * bxn + i0 / g.bx])
                                continue;
                            gtiles.push_back(make_int4(c | r << 3, i0, j0, k0));
                        }
    }
    gt_begin.push_back((int)gtiles.size());
    // the same grid tiles in pairs of one (class, row block) for k_m2l_tcw,
    // appended after them; an odd tile is paired with itself (flagged)
    const size_t wbase = gtiles.size();
    std::vector<int> wt_begin;
    for (size_t gi = 0; gi < gp.size(); gi++) {
        wt_begin.push_back((int)(gtiles.size() - wbase));
        for (int i = gt_begin[gi]; i < gt_begin[gi + 1];) {
            const int4 t0 = gtiles[i];
            if (i + 1 < gt_begin[gi + 1] && gtiles[i + 1].x == t0.x) {
                const int4 t1 = gtiles[i + 1];
                gtiles.push_back(t0);
                gtiles.push_back(t1);
                i += 2;
            } else {
                gtiles.push_back(t0);
                gtiles.push_back(make_int4(t0.x | TCW_SKIP, t0.y, t0.z, t0.w));
                i += 1;
            }
        }
    }
    wt_begin.push_back((int)(gtiles.size() - wbase));
    grow(t->gtiles, t->gtiles_cap, gtiles.size() + 1);
    grow(t->gboxes, t->gboxes_cap, gbox.size() + 1);
    if (!gtiles.empty())
        PK_CUDA(cudaMemcpyAsync(t->gtiles, gtiles.data(), sizeof(int4) * gtiles.size(), cudaMemcpyHostToDevice, s));
    if (!gbox.empty())
        PK_CUDA(cudaMemcpyAsync(t->gboxes, gbox.data(), sizeof(int) * gbox.size(), cudaMemcpyHostToDevice, s));

    TcArgs a;
    std::memset(&a, 0, sizeof a);
    a.v_slot = P.tree.v_slot.p;
    a.class_ops = P.class_slot_op.p;
    a.slot_off = t->slot_off;
    a.chk = chk;
    a.amax = t->amax;
    a.kn = rk;
    a.KM = t->KM;
    a.KK = KK;
    a.nrhs = nr;
    a.zero_row = (int)rows;
    a.kexp = t->kexp;
    a.err = t->err;

    // densities for gather mode
    const int ngather_tiles = gt_begin.empty() ? (int)gtiles.size() : gt_begin[0];
    if (ngather_tiles > 0) {
        if ((size_t)(rows + 1) > t->phi_rows) {
            cudaFree(t->phi);
            t->phi = nullptr;
            t->phi_rows = (size_t)(rows + 1) + (size_t)(rows + 1) / 4;
            PK_CUDA(cudaMalloc(&t->phi, 2 * t->phi_rows * KK * sizeof(__half)));
        }
        long long tot = (rows + 1) * KK;
        count_launch(), k_phi_split<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
            up, rows, rk, KK, t->amax, t->phi, t->phi + t->phi_rows * KK);
    }
    // parity grids for grid mode
    if (!gp.empty()) {
        grow(t->grid, t->grid_cap, grid_elems);
        for (auto &g : gp) {
            __half *hi = t->grid + g.off, *lo = hi + (size_t)g.rows * KK;
            count_launch(), k_phi_grid<<<(unsigned)g.rows, 128, 0, s>>>(
                up, lb[g.level], g.map_off >= 0 ? t->lmap + g.map_off : nullptr, g.n, nr, rk, KK,
                P.periodic, t->amax, g.rows, hi, lo);
        }
    }
    PK_CUDA(cudaEventRecord(t->ev[0], s));
    // the gather launch and the grid launches (one per level) write disjoint check
    // rows: run them on side streams so small launches and wave tails overlap
    if (!t->fork) {
        PK_CUDA(cudaEventCreateWithFlags(&t->fork, cudaEventDisableTiming));
        for (int i = 0; i < 3; i++) {
            PK_CUDA(cudaStreamCreateWithFlags(&t->side[i], cudaStreamNonBlocking));
            PK_CUDA(cudaEventCreateWithFlags(&t->join[i], cudaEventDisableTiming));
        }
    }
    PK_CUDA(cudaEventRecord(t->fork, s));
    for (int i = 0; i < 3; i++) PK_CUDA(cudaStreamWaitEvent(t->side[i], t->fork, 0));
    int nlaunch = 0;
    EncodeTiledFn enc = encode_fn();
    if (ngather_tiles > 0) {
        a.phi_hi = t->phi;
        a.phi_lo = t->phi + t->phi_rows * KK;
        a.tboxes = t->gboxes;
        a.tiles = t->gtiles;
        a.grid = 0;
        // several vectors per box: a box's source rows are contiguous, one 2D TMA each
        a.boxg = (nr >= 8 && TC_N % nr == 0) ? 1 : 0;
        CUtensorMap pm[2] = {t->tmap[0], t->tmap[1]};
        if (a.boxg) {
            for (int h = 0; h < 2; h++) {
                cuuint64_t dims[2] = {(cuuint64_t)KK, (cuuint64_t)(rows + 1)};
                cuuint64_t strides[1] = {(cuuint64_t)KK * 2};
                cuuint32_t box[2] = {TC_K, (cuuint32_t)nr};
                cuuint32_t estr[2] = {1, 1};
                CUresult r = enc(&pm[h], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void *)(t->phi + (size_t)h * t->phi_rows * KK), dims, strides, box,
                                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) throw Error(PKIFMM_ERR_CUDA, "cuTensorMapEncodeTiled (Phi rows) failed");
            }
        }
        cudaStream_t ls = t->side[nlaunch++ % 3];
        if (t->stages == 2)
            count_launch(), k_m2l_tc<2><<<ngather_tiles * mtiles, TC_THREADS, tc_smem(2), ls>>>(t->tmap[0], t->tmap[1],
                                                                                               pm[0], pm[1], a);
        else
            count_launch(), k_m2l_tc<3><<<ngather_tiles * mtiles, TC_THREADS, tc_smem(3), ls>>>(t->tmap[0], t->tmap[1],
                                                                                               pm[0], pm[1], a);
        PK_CUDA(cudaGetLastError());
        a.boxg = 0;
    }
    for (size_t gi = 0; gi < gp.size(); gi++) {
        const GridPlan &g = gp[gi];
        const cuuint64_t d = (cuuint64_t)(g.n / 2 + 4);
        CUtensorMap mb[2];
        for (int h = 0; h < 2; h++) {
            __half *base = t->grid + g.off + (size_t)h * g.rows * KK;
            cuuint64_t dims[5] = {(cuuint64_t)KK, (cuuint64_t)nr, d, d, 8 * d};
            cuuint64_t row = (cuuint64_t)KK * 2;
            cuuint64_t strides[4] = {row, row * nr, row * nr * d, row * nr * d * d};
            cuuint32_t box[5] = {TC_K, (cuuint32_t)g.rb, (cuuint32_t)g.bx, (cuuint32_t)g.by, (cuuint32_t)g.bz};
            cuuint32_t estr[5] = {1, 1, 1, 1, 1};
            CUresult r = enc(&mb[h], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) throw Error(PKIFMM_ERR_CUDA, "cuTensorMapEncodeTiled (level grid) failed");
        }
        a.grid = 1;
        a.tiles = t->gtiles + gt_begin[gi];
        a.lvl_begin = lb[g.level];
        a.lmap = g.map_off >= 0 ? t->lmap + g.map_off : nullptr;
        a.zd = (int)d;
        a.bx = g.bx;
        a.by = g.by;
        a.bz = g.bz;
        a.rb = g.rb;
        const int ntl = gt_begin[gi + 1] - gt_begin[gi];
        if (ntl == 0) continue;
        cudaStream_t ls = t->side[nlaunch++ % 3];
        if (t->wide) {
            a.tiles = t->gtiles + wbase + wt_begin[gi];
            const int npair = (wt_begin[gi + 1] - wt_begin[gi]) / 2;
            count_launch(), k_m2l_tcw<2><<<npair * mtiles, TCW_THREADS, tcw_smem(2), ls>>>(t->tmap[0], t->tmap[1],
                                                                                         mb[0], mb[1], a);
        } else if (t->stages == 2)
            count_launch(), k_m2l_tc<2><<<ntl * mtiles, TC_THREADS, tc_smem(2), ls>>>(t->tmap[0], t->tmap[1], mb[0], mb[1], a);
        else
            count_launch(), k_m2l_tc<3><<<ntl * mtiles, TC_THREADS, tc_smem(3), ls>>>(t->tmap[0], t->tmap[1], mb[0], mb[1], a);
        PK_CUDA(cudaGetLastError());
    }
    for (int i = 0; i < 3; i++) {
        PK_CUDA(cudaEventRecord(t->join[i], t->side[i]));
        PK_CUDA(cudaStreamWaitEvent(s, t->join[i], 0));
    }
    PK_CUDA(cudaEventRecord(t->ev[1], s));
    PK_CUDA(cudaMemcpyAsync(t->err_host, t->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));  // host tile vectors and the error flag
    PK_CUDA(cudaEventElapsedTime(&t->last_ms, t->ev[0], t->ev[1]));
    if (*t->err_host) {
        PK_CUDA(cudaMemset(t->err, 0, sizeof(int)));
        throw Error(PKIFMM_ERR_TIMEOUT, "tensor-core M2L: a bounded pipeline wait gave up");
    }
    return true;
}

float m2l_tc_last_ms(Plan &P) { return P.tc ? P.tc->last_ms : 0.f; }

bool m2l_tc_device_supported() { return tc_supported(); }

}  // namespace pk
