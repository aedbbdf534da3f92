// tcgen05.cuh -- inline-PTX wrappers for the 5th-generation tensor cores of sm_103a:
// tensor-memory (TMEM) allocation, single-thread MMA issue with shared-memory operand
// descriptors, completion tracking through mbarriers, and TMEM -> register loads.
//
// Layout conventions used by the callers (all operands K-major, no swizzle):
//  * A core matrix is 8 rows x 16 bytes stored contiguously (row r at byte 16 r).
//  * The shared-memory descriptor gives the start address, the byte distance between
//    core matrices that are adjacent along K (the leading byte offset, LBO) and between
//    groups of 8 rows that are adjacent along M or N (the stride byte offset, SBO).
//  * The accumulator D of an M = 128 MMA occupies TMEM lanes 0..127 (row m of D in lane
//    m) and N consecutive 32-bit columns.  A warp may read only the 32 lanes of its own
//    quarter: warp w reaches lanes 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once

#include <stdint.h>

namespace imcl {

// ------------------------------------------------------------------ descriptors
// Shared-memory matrix descriptor: start address, LBO and SBO in 16-byte units (14 bits
// each), the descriptor version 1 at bit 46, base offset 0, no swizzle (layout type 0).
__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;
}

// Instruction descriptor of a dense MMA with an f32 accumulator, both operands K-major:
// bits 4-5 accumulator format (1 = f32), 7-9 A format and 10-12 B format (f16 kinds:
// 0 = f16, 1 = bf16; the tf32 kind: 2), 17-22 N / 8, 24-28 M / 16.
enum UmmaOperand : uint32_t { UMMA_F16 = 0, UMMA_BF16 = 1, UMMA_TF32 = 2 };

__host__ __device__ constexpr uint32_t umma_idesc(uint32_t ab_format, int M, int N) {
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// ------------------------------------------------------------------ TMEM allocation
// One whole warp allocates `ncols` columns (a power of two >= 32); the TMEM address is
// written to the shared-memory word `dst`.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ------------------------------------------------------------------ ordering
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ------------------------------------------------------------------ MMA
// D[tmem] (+)= A[smem] x B[smem]^T, issued by one thread.  accumulate = 0 overwrites D.
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The same with the A operand in tensor memory (M lanes x K columns at a_tmem; tf32: one
// element per 32-bit column, f16/bf16: two): only B is read from shared memory.
__device__ __forceinline__ void umma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                             uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_f16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on `bar` when every MMA this thread issued so far has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// ------------------------------------------------------------------ TMEM -> registers
// Two loads of 16 consecutive 32-bit columns of the warp's 32 lanes (thread t gets lane
// base + t) and the wait for both, in one asm statement so that no use of the results
// can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld16x2(uint32_t taddr0, uint32_t taddr1, float* v0, float* v1) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr0), "r"(taddr1)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v0[i] = __uint_as_float(r[i]);
        v1[i] = __uint_as_float(r[16 + i]);
    }
}

// 4 J consecutive 32-bit columns (J in 5..8) of the warp's 32 lanes from taddr, loaded as
// x16 / x8 / x4 / x32 pieces behind one wait: v[c] is column c.
template <int J>
__device__ __forceinline__ void tmem_ld4xJ(uint32_t taddr, float* v) {
    static_assert(J >= 5 && J <= 8, "5..8 column groups of 4");
    uint32_t r[32];
#define IMCL_O4(b) "=r"(r[b]), "=r"(r[b + 1]), "=r"(r[b + 2]), "=r"(r[b + 3])
    if constexpr (J == 5) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%20];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%16, %17, %18, %19}, [%21];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O4(0), IMCL_O4(4), IMCL_O4(8), IMCL_O4(12), IMCL_O4(16)
            : "r"(taddr), "r"(taddr + 16)
            : "memory");
    } else if constexpr (J == 6) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%24];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%25];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O4(0), IMCL_O4(4), IMCL_O4(8), IMCL_O4(12), IMCL_O4(16), IMCL_O4(20)
            : "r"(taddr), "r"(taddr + 16)
            : "memory");
    } else if constexpr (J == 7) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%28];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%29];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%24, %25, %26, %27}, [%30];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O4(0), IMCL_O4(4), IMCL_O4(8), IMCL_O4(12), IMCL_O4(16), IMCL_O4(20), IMCL_O4(24)
            : "r"(taddr), "r"(taddr + 16), "r"(taddr + 24)
            : "memory");
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O4(0), IMCL_O4(4), IMCL_O4(8), IMCL_O4(12), IMCL_O4(16), IMCL_O4(20), IMCL_O4(24), IMCL_O4(28)
            : "r"(taddr)
            : "memory");
    }
#undef IMCL_O4
#pragma unroll
    for (int i = 0; i < 4 * J; ++i) v[i] = __uint_as_float(r[i]);
}

// N (1..3) loads of 8 consecutive 32-bit columns (at taddr + 8 j, j < N) and their wait.
template <int N>
__device__ __forceinline__ void tmem_ld8xN(uint32_t taddr, float* v) {
    static_assert(N >= 1 && N <= 3, "1..3 column groups");
    uint32_t r[24];
#define IMCL_O8N(b) "=r"(r[b]), "=r"(r[b + 1]), "=r"(r[b + 2]), "=r"(r[b + 3]), "=r"(r[b + 4]), "=r"(r[b + 5]), \
                    "=r"(r[b + 6]), "=r"(r[b + 7])
    if constexpr (N == 1) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O8N(0)
            : "r"(taddr)
            : "memory");
    } else if constexpr (N == 2) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O8N(0), IMCL_O8N(8)
            : "r"(taddr), "r"(taddr + 8)
            : "memory");
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%24];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%25];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%26];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O8N(0), IMCL_O8N(8), IMCL_O8N(16)
            : "r"(taddr), "r"(taddr + 8), "r"(taddr + 16)
            : "memory");
    }
#undef IMCL_O8N
#pragma unroll
    for (int i = 0; i < 8 * N; ++i) v[i] = __uint_as_float(r[i]);
}

// Four loads of 8 consecutive 32-bit columns (at taddr + 8 j, j < 4) and their wait.
__device__ __forceinline__ void tmem_ld8x4(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%33];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%34];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%35];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr), "r"(taddr + 8), "r"(taddr + 16), "r"(taddr + 24)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// J loads of 8 consecutive 32-bit columns (at taddr + 8 j, j < J, J in 5..8) of the
// warp's 32 lanes and the wait for all of them, in one asm statement: v[8 j + c] is
// column 8 j + c of lane base + t for thread t.
template <int J>
__device__ __forceinline__ void tmem_ld8xJ(uint32_t taddr, float* v) {
    static_assert(J >= 5 && J <= 8, "5..8 column groups");
    uint32_t r[64];
#define IMCL_O8(b) "=r"(r[b]), "=r"(r[b + 1]), "=r"(r[b + 2]), "=r"(r[b + 3]), "=r"(r[b + 4]), "=r"(r[b + 5]), \
                   "=r"(r[b + 6]), "=r"(r[b + 7])
    if constexpr (J == 5) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%40];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%41];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%42];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%43];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32, %33, %34, %35, %36, %37, %38, %39}, [%44];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O8(0), IMCL_O8(8), IMCL_O8(16), IMCL_O8(24), IMCL_O8(32)
            : "r"(taddr), "r"(taddr + 8), "r"(taddr + 16), "r"(taddr + 24), "r"(taddr + 32)
            : "memory");
    } else if constexpr (J == 6) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%48];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%49];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%50];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%51];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32, %33, %34, %35, %36, %37, %38, %39}, [%52];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%40, %41, %42, %43, %44, %45, %46, %47}, [%53];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O8(0), IMCL_O8(8), IMCL_O8(16), IMCL_O8(24), IMCL_O8(32), IMCL_O8(40)
            : "r"(taddr), "r"(taddr + 8), "r"(taddr + 16), "r"(taddr + 24), "r"(taddr + 32), "r"(taddr + 40)
            : "memory");
    } else if constexpr (J == 7) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%56];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%57];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%58];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%59];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32, %33, %34, %35, %36, %37, %38, %39}, [%60];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%40, %41, %42, %43, %44, %45, %46, %47}, [%61];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%48, %49, %50, %51, %52, %53, %54, %55}, [%62];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O8(0), IMCL_O8(8), IMCL_O8(16), IMCL_O8(24), IMCL_O8(32), IMCL_O8(40), IMCL_O8(48)
            : "r"(taddr), "r"(taddr + 8), "r"(taddr + 16), "r"(taddr + 24), "r"(taddr + 32), "r"(taddr + 40),
              "r"(taddr + 48)
            : "memory");
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%64];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%65];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%66];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%67];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32, %33, %34, %35, %36, %37, %38, %39}, [%68];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%40, %41, %42, %43, %44, %45, %46, %47}, [%69];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%48, %49, %50, %51, %52, %53, %54, %55}, [%70];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%56, %57, %58, %59, %60, %61, %62, %63}, [%71];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : IMCL_O8(0), IMCL_O8(8), IMCL_O8(16), IMCL_O8(24), IMCL_O8(32), IMCL_O8(40), IMCL_O8(48), IMCL_O8(56)
            : "r"(taddr), "r"(taddr + 8), "r"(taddr + 16), "r"(taddr + 24), "r"(taddr + 32), "r"(taddr + 40),
              "r"(taddr + 48), "r"(taddr + 56)
            : "memory");
    }
#undef IMCL_O8
#pragma unroll
    for (int i = 0; i < 8 * J; ++i) v[i] = __uint_as_float(r[i]);
}

// Registers -> tensor memory: 16 (or 8) consecutive 32-bit columns of the warp's 32
// lanes (thread t writes lane base + t), then the wait for the stores to complete.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

}  // namespace imcl
