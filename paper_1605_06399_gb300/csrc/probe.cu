// probe.cu -- measurement helpers.
//  * FP32 pipe throughput, the measured denominator beside the ALU roofline derived
//    from unit counts and clocks: each thread runs 16 independent FMA chains, either as
//    scalar FMAs or as 8 packed f32x2 FMAs.
//  * Integer multiply-add throughput (the u8 -> i32 correlation's arithmetic): 16
//    independent wrapping int32 multiply-add chains per thread.
//  * A bounded-wait self-test: one thread waits on an mbarrier phase that cannot
//    complete, gives up after a given number of rounds and records the timeout code in
//    the device status word, exactly as the stencil kernels do.
#include "common.cuh"
#include "internal.h"

namespace imcl {

// (d0, d1) = (a0 b0 + c0, a1 b1 + c1) as one packed f32x2 FMA
__device__ __forceinline__ void ffma2(float& d0, float& d1, float a0, float a1, float b0, float b1, float c0,
                                      float c1) {
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rc, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rc;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}

template <bool PACKED>
__global__ void __launch_bounds__(256) k_fp32_probe(float* out, float a, float b, int iters) {
    float x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = threadIdx.x * 1e-3f + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; k += 2) {
            if constexpr (PACKED) {
                ffma2(x[k], x[k + 1], x[k], x[k + 1], a, a, b, b);
            } else {
                x[k] = __fmaf_rn(x[k], a, b);
                x[k + 1] = __fmaf_rn(x[k + 1], a, b);
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += x[k];
    if (s == 1234.5f) out[blockIdx.x] = s;   // practically never; keeps the work live
}

__global__ void __launch_bounds__(256) k_imad_probe(int* out, int a, int b, int iters) {
    uint32_t x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = threadIdx.x * 7u + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = x[k] * (uint32_t)a + (uint32_t)b;
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) s ^= x[k];
    if (s == 0x9e3779b9u) out[blockIdx.x] = (int)s;   // practically never; keeps the work live
}

// One thread arms an mbarrier for a 16-byte transfer that no copy will bring, waits at
// most `rounds` try_wait rounds and records DEVERR_TIMEOUT.  Nothing is in flight when
// it returns.
__global__ void k_wait_timeout(uint32_t rounds, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, 16);
    for (uint32_t it = 0; it < rounds; ++it)
        if (mbar_try_wait(&bar, 0)) return;
    dev_fail(status, DEVERR_TIMEOUT);
}

}  // namespace imcl

using namespace imcl;

extern "C" imcl_status imagecl_probe_fp32(int32_t packed, double* tflops, void* stream) {
    if (!tflops) return fail(IMCL_ERR_INVALID, "tflops is NULL");
    DeviceInfo* dev = nullptr;
    imcl_status st = device_info(&dev);
    if (st != IMCL_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = dev->sm_count * 8, threads = 256, iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {
        cudaEventRecord(e0, s);
        if (packed) k_fp32_probe<true><<<blocks, threads, 0, s>>>(nullptr, 0.999f, 1e-3f, iters);
        else k_fp32_probe<false><<<blocks, threads, 0, s>>>(nullptr, 0.999f, 1e-3f, iters);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "fp32 probe");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = (double)blocks * threads * iters * 16 * 2;
    *tflops = flops / (best * 1e-3) / 1e12;
    return IMCL_OK;
}

extern "C" imcl_status imagecl_probe_imad(double* tops, void* stream) {
    if (!tops) return fail(IMCL_ERR_INVALID, "tops is NULL");
    DeviceInfo* dev = nullptr;
    imcl_status st = device_info(&dev);
    if (st != IMCL_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = dev->sm_count * 8, threads = 256, iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {
        cudaEventRecord(e0, s);
        k_imad_probe<<<blocks, threads, 0, s>>>(nullptr, 0x01000193, 7, iters);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "imad probe");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double ops = (double)blocks * threads * iters * 16 * 2;
    *tops = ops / (best * 1e-3) / 1e12;
    return IMCL_OK;
}

extern "C" imcl_status imagecl_selftest_wait_timeout(int32_t rounds, void* stream) {
    if (rounds < 1 || rounds > (1 << 20)) return fail(IMCL_ERR_INVALID, "rounds must be in [1, 2^20]");
    DeviceInfo* dev = nullptr;
    imcl_status st = device_info(&dev);
    if (st != IMCL_OK) return st;
    k_wait_timeout<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((uint32_t)rounds, dev->status);
    return cuda_fail(cudaGetLastError(), "wait self-test launch");
}
