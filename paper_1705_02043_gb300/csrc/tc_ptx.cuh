// Shared pieces of the tcgen05 kernels (the V-list M2L and the dense
// translations of the MIXED path): tile constants, mbarrier waits bounded in
// time, TMA and cp.async copies, shared-memory descriptors of the 128-byte
// swizzled K-major layout, and the tcgen05 MMA / commit / tensor-memory loads,
// all as inline PTX for sm_103a.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace pk {

constexpr int TC_N = 128;                          // (box, rhs) columns per CTA
constexpr int TC_M = 128;                          // kn rows per CTA
constexpr int TC_K = 64;                           // K chunk: 128 bytes of fp16 per row (128-byte swizzle)
constexpr int TC_STAGES = 3;                        // pipeline depth (the default instantiation)
constexpr int TC_A_BYTES = TC_M * TC_K * 2;        // 16 KB per split
constexpr int TC_B_BYTES = TC_N * TC_K * 2;        // 16 KB per split
constexpr int TC_STAGE_BYTES = 2 * TC_A_BYTES + 2 * TC_B_BYTES;  // 32 KB
constexpr int TC_CTRL_BYTES = 4096;
constexpr int TC_SLACK = 16384;
constexpr int tc_smem(int stages) { return TC_CTRL_BYTES + stages * TC_STAGE_BYTES + TC_SLACK + 1024; }
constexpr int TC_THREADS = 288;                    // 4 producer warps, 1 MMA warp, 4 epilogue warps
constexpr int TC_TMEM_COLS = 512;                  // 2 buffers x (hi*hi, cross terms) x 128 columns
constexpr long long TC_WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

// ---------------- PTX helpers ----------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false (and the error flag raised) after ~2 s
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > TC_WAIT_CYCLES) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ unsigned long long morton3_dev(int x, int y, int z) {
    unsigned long long r = 0;
    for (int b = 0; b < 21; b++)
        r |= ((unsigned long long)((x >> b) & 1) << (3 * b)) | ((unsigned long long)((y >> b) & 1) << (3 * b + 1)) |
             ((unsigned long long)((z >> b) & 1) << (3 * b + 2));
    return r;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// K-major operand with 128-byte rows, 128B swizzle: 8-row atoms of 1024 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF)    // start address
           | ((uint64_t)1 << 16)               // leading byte offset (unused for swizzled K-major)
           | ((uint64_t)(1024 >> 4) << 32)     // stride byte offset: 8 rows x 128 B
           | ((uint64_t)1 << 46)               // descriptor version
           | ((uint64_t)2 << 61);              // layout: 128-byte swizzle
}

// kind::f16 instruction descriptors: f16 x f16 -> f32, both K-major, M = 128,
// N = 128 or N = 256 (B_hi and B_lo, adjacent in shared memory, as one operand).
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
constexpr uint32_t kIdesc2 = (1u << 4) | ((uint32_t)((2 * TC_N) >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

// power-of-two exponent that brings max |phi| just below 2^14
__device__ __forceinline__ int phi_exp(const float *amax) {
    int e = 0;
    float m = *amax;
    if (!(m > 0.f) || !isfinite(m)) return 0;
    frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
    return 14 - e;
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc,
                                       uint32_t idesc = kIdesc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_ld16_nowait(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace pk
