// common.cuh -- device helpers shared by the stencil kernels (sm_103a).
//
// Pixel types are converted to the accumulation type on load (f16/bf16 -> f32, u8 -> i32)
// and rounded to the output type on store with round-to-nearest-even.  The TMA and
// mbarrier wrappers are inline PTX; every wait has an iteration limit after which the
// kernel records IMCL_DEVERR_TIMEOUT in the device status word and gives up.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "imagecl.h"

namespace imcl {

// ------------------------------------------------------------------ device status
// Codes a kernel can leave in the status word (first error wins).
enum DevErr : int {
    DEVERR_NONE = 0,
    DEVERR_TIMEOUT = 1,   // an mbarrier wait exceeded its iteration limit
    DEVERR_BOUNDS = 2,    // a computed index fell outside its buffer (debug checks)
};

__device__ __forceinline__ void dev_fail(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ type helpers
template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<uint8_t> { using type = int32_t; };
template <> struct AccOf<int32_t> { using type = int32_t; };

__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ int32_t to_acc(uint8_t v) { return (int32_t)v; }
__device__ __forceinline__ int32_t to_acc(int32_t v) { return v; }

template <typename T> __device__ __forceinline__ T from_acc(float v);
template <> __device__ __forceinline__ float from_acc<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_acc<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
// integer images accumulated in f32 (exact integers below 2^24): the value is integral
template <> __device__ __forceinline__ int32_t from_acc<int32_t>(float v) { return __float2int_rn(v); }
template <typename T> __device__ __forceinline__ T from_acc_i(int32_t v);
template <> __device__ __forceinline__ int32_t from_acc_i<int32_t>(int32_t v) { return v; }

template <typename Tout, typename Acc> struct Store;
template <typename Tout> struct Store<Tout, float> {
    static __device__ __forceinline__ Tout cvt(float v) { return from_acc<Tout>(v); }
};
template <> struct Store<int32_t, int32_t> {
    static __device__ __forceinline__ int32_t cvt(int32_t v) { return v; }
};

// multiply-add in the accumulation type (FMA for float, wrapping IMAD for int32)
__device__ __forceinline__ float mad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ int32_t mad(int32_t a, int32_t b, int32_t c) {
    return (int32_t)((uint32_t)a * (uint32_t)b + (uint32_t)c);
}

// Two f32 multiply-adds in one packed f32x2 instruction; each lane is rounded exactly
// like __fmaf_rn, so a packed kernel gives the same bits as its scalar form.
__device__ __forceinline__ float2 mad2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// ------------------------------------------------------------------ vector loads
// Widen the two 16-bit pixels of a 32-bit word (element 0 in the low half) to f32.
// bf16 is the upper half of an f32, so widening is a shift or a mask (exact).
__device__ __forceinline__ void unpack2(__nv_bfloat16, uint32_t w, float* d) {
    d[0] = __uint_as_float(w << 16);
    d[1] = __uint_as_float(w & 0xffff0000u);
}
__device__ __forceinline__ void unpack2(__half, uint32_t w, float* d) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w));
    d[0] = f.x;
    d[1] = f.y;
}

// N pixels held in N/2 words (16-bit types widened to f32).
template <typename T, int N, typename A>
__device__ __forceinline__ void unpack_words(const uint32_t* w, A* dst) {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) unpack2(T(), w[k], dst + 2 * k);
}

template <typename T, typename A>
constexpr bool kWordUnpack = sizeof(T) == 2 && std::is_same<A, float>::value;

// Load N consecutive pixels (N * sizeof(T) in {2, 4, 8, 16} bytes, naturally aligned)
// and convert them to the accumulation type.
template <typename T, int N, typename A>
__device__ __forceinline__ void load_vec(const T* p, A* dst) {
    constexpr int B = N * (int)sizeof(T);
    static_assert(B == 2 || B == 4 || B == 8 || B == 16 || B == 1, "vector width");
    if constexpr (kWordUnpack<T, A> && B == 16) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        unpack_words<T, N>(w, dst);
    } else if constexpr (kWordUnpack<T, A> && B == 8) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        const uint32_t w[2] = {v.x, v.y};
        unpack_words<T, N>(w, dst);
    } else if constexpr (kWordUnpack<T, A> && B == 4) {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
        unpack_words<T, N>(&w, dst);
    } else if constexpr (B == 16) {
        uint4 v = *reinterpret_cast<const uint4*>(p);
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int k = 0; k < N; ++k) dst[k] = to_acc(e[k]);
    } else if constexpr (B == 8) {
        uint2 v = *reinterpret_cast<const uint2*>(p);
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int k = 0; k < N; ++k) dst[k] = to_acc(e[k]);
    } else if constexpr (B == 4) {
        uint32_t v = *reinterpret_cast<const uint32_t*>(p);
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int k = 0; k < N; ++k) dst[k] = to_acc(e[k]);
    } else if constexpr (B == 2) {
        uint16_t v = *reinterpret_cast<const uint16_t*>(p);
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int k = 0; k < N; ++k) dst[k] = to_acc(e[k]);
    } else {
        dst[0] = to_acc(p[0]);
    }
}

// Read-only global load through the non-coherent (texture/L1) path.
template <typename T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
template <> __device__ __forceinline__ __half ldg<__half>(const __half* p) {
    unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_half(u);
}
template <> __device__ __forceinline__ __nv_bfloat16 ldg<__nv_bfloat16>(const __nv_bfloat16* p) {
    unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_bfloat16(u);
}

template <typename T, int N, typename A>
__device__ __forceinline__ void ldg_vec(const T* p, A* dst) {
    constexpr int B = N * (int)sizeof(T);
    if constexpr (kWordUnpack<T, A> && B == 16) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        unpack_words<T, N>(w, dst);
    } else if constexpr (kWordUnpack<T, A> && B == 8) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        const uint32_t w[2] = {v.x, v.y};
        unpack_words<T, N>(w, dst);
    } else if constexpr (kWordUnpack<T, A> && B == 4) {
        const uint32_t w = __ldg(reinterpret_cast<const unsigned int*>(p));
        unpack_words<T, N>(&w, dst);
    } else if constexpr (B == 16) {
        uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int k = 0; k < N; ++k) dst[k] = to_acc(e[k]);
    } else if constexpr (B == 8) {
        uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int k = 0; k < N; ++k) dst[k] = to_acc(e[k]);
    } else if constexpr (B == 4) {
        uint32_t v = __ldg(reinterpret_cast<const unsigned int*>(p));
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int k = 0; k < N; ++k) dst[k] = to_acc(e[k]);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) dst[k] = to_acc(ldg(p + k));
    }
}

// Round pairs of f32 to packed 16-bit values (one conversion per pair).
__device__ __forceinline__ uint32_t pack2(__half, float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16, float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Store N accumulators as N consecutive output pixels with one vector store.
template <typename T, int N, typename A>
__device__ __forceinline__ void store_vec(T* p, const A* src) {
    constexpr int B = N * (int)sizeof(T);
    if constexpr (sizeof(T) == 2 && N % 2 == 0 && (B == 8 || B == 16)) {
        uint32_t w[N / 2];
#pragma unroll
        for (int k = 0; k < N / 2; ++k) w[k] = pack2(T(), src[2 * k], src[2 * k + 1]);
        if constexpr (B == 16) *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
        else *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
        return;
    }
    T e[N];
#pragma unroll
    for (int k = 0; k < N; ++k) e[k] = Store<T, A>::cvt(src[k]);
    if constexpr (B == 16) {
        *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(e);
    } else if constexpr (B == 8) {
        *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(e);
    } else if constexpr (B == 4) {
        *reinterpret_cast<uint32_t*>(p) = *reinterpret_cast<const uint32_t*>(e);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) p[k] = e[k];
    }
}

// ------------------------------------------------------------------ mbarrier / TMA
constexpr uint32_t kWaitLimit = 1u << 22;   // try_wait rounds before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier; false (and the status word set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status) {
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    dev_fail(status, DEVERR_TIMEOUT);
    return false;
}

// 2D tiled TMA load of the tensor map's box at (x, y) into shared memory, completing on
// `bar`.  x * sizeof(element) must be a multiple of 16 bytes (checked by the callers'
// tile geometry); y may be negative or beyond the image (zero fill).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__host__ __device__ constexpr int round_up(int v, int m) { return (v + m - 1) / m * m; }

// A grid is at most 65535 blocks high.  One-pixel-per-thread kernels over W x H images
// launch grid_2d(...) and walk their rows with a stride of gridDim.y * blockDim.y, so
// every height runs.
constexpr int kMaxGridY = 65535;
inline dim3 grid_2d(int W, int H, int bx, int by) {
    const int gy = (H + by - 1) / by;
    return dim3((unsigned)((W + bx - 1) / bx), (unsigned)(gy < kMaxGridY ? gy : kMaxGridY));
}

}  // namespace imcl
