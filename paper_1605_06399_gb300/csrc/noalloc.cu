// noalloc.cu -- imagecl_sepconv_noalloc: the two-pass separable correlation with its
// intermediate in a fixed, library-owned device array instead of caller memory.
//
// Who this is for: callers that must not call cudaMalloc or any other allocating routine
// while they run.  A plugin inside a host framework that owns every byte of device
// memory through its own allocator is not allowed raw allocations, and a real-time
// processing loop cannot take the device-wide synchronisation that cudaMalloc and
// cudaFree may bring.  Those callers still own their input and output images; only the
// row-pass intermediate moves into the array below.
//
// The kernels walk the image's rows with a grid-stride loop, so any height whose
// width * height fits the array runs (a grid is at most 65535 blocks high).
//
// The array is a file-scope __device__ variable, so every GPU that loads this library
// holds kNoallocScratchBytes for it until the process exits.  Host code cannot take its
// address with `&`: the symbol seen from the host is a host-side stand-in, and a kernel
// handed that would fault or, where the GPU can reach host memory, quietly use the wrong
// memory.  The real device address is fetched once per device with
// cudaGetSymbolAddress, with that device current, and cached.
#include <map>
#include <mutex>

#include "abi_internal.h"
#include "sepconv_kernels.cuh"

namespace imcl {

constexpr size_t kNoallocScratchBytes = IMAGECL_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mu;
static std::map<int, void*> g_noalloc_addr;   // device ordinal -> device address of the array

// Device address of the array on the current device (looked up on the first call per device).
static imcl_status noalloc_scratch(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) {
        *out = it->second;
        return IMCL_OK;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-alloc scratch array");
    if (!p) return fail(IMCL_ERR_CUDA, "cudaGetSymbolAddress returned a null scratch address");
    g_noalloc_addr[dev] = p;
    *out = p;
    return IMCL_OK;
}

template <typename Tin, typename Tout>
static void noalloc_launch(const ConvArgs& a, const TapsParam<float, 66>& tp, dim3 grid, dim3 block, cudaStream_t s) {
    k_sep_row_plain<Tin><<<grid, block, 0, s>>>(a, tp);
    k_sep_col_plain<Tout><<<grid, block, 0, s>>>(a, tp);
}

}  // namespace imcl

using namespace imcl;

extern "C" imcl_status imagecl_sepconv_noalloc(const imcl_image* in, const imcl_image* out, const float* row_taps,
                                               int32_t nrow, const float* col_taps, int32_t ncol, int32_t taps_mem,
                                               int32_t border, double border_value, void* stream) {
    imcl_status st;
    if ((st = check_image(in, "in")) != IMCL_OK) return st;
    if ((st = check_image(out, "out")) != IMCL_OK) return st;
    if (in->width != out->width || in->height != out->height)
        return fail(IMCL_ERR_INVALID, "in and out must have the same width and height");
    if (images_overlap(in, out)) return fail(IMCL_ERR_INVALID, "in and out overlap (operations are out of place)");
    if (nrow <= 0 || ncol <= 0) return fail(IMCL_ERR_INVALID, "tap counts must be positive");
    if (nrow % 2 == 0 || ncol % 2 == 0) return fail(IMCL_ERR_UNSUPPORTED, "tap counts must be odd (centred taps)");
    if (nrow > kMaxSepTaps || ncol > kMaxSepTaps) return fail(IMCL_ERR_UNSUPPORTED, "more than 33 taps is not provided");
    if (!row_taps || !col_taps) return fail(IMCL_ERR_INVALID, "row_taps and col_taps must not be NULL");
    if (taps_mem != IMCL_MEM_HOST && taps_mem != IMCL_MEM_DEVICE)
        return fail(IMCL_ERR_INVALID, "taps_mem must be IMCL_MEM_HOST or IMCL_MEM_DEVICE");
    if (is_int_dtype(in->dtype)) return fail(IMCL_ERR_UNSUPPORTED, "sepconv takes f32, f16 or bf16 images");
    if (out->dtype != IMCL_F32 && out->dtype != in->dtype)
        return fail(IMCL_ERR_UNSUPPORTED, "floating images write f32 or their own 16-bit type");
    if ((st = check_border(border, border_value, in->dtype)) != IMCL_OK) return st;
    const size_t need = (size_t)in->width * (size_t)in->height * sizeof(float);
    if (need > kNoallocScratchBytes)
        return fail(IMCL_ERR_UNSUPPORTED,
                    "imagecl_sepconv_noalloc: width*height*4 bytes exceeds its fixed scratch of "
                    "IMAGECL_NOALLOC_SCRATCH_BYTES (16 MiB, 4194304 pixels); use imagecl_sepconv");
    void* scratch = nullptr;
    if ((st = noalloc_scratch(&scratch)) != IMCL_OK) return st;

    ConvCall c;
    c.in = in->data;
    c.out = out->data;
    c.in_dtype = in->dtype;
    c.out_dtype = out->dtype;
    c.W = in->width;
    c.H = in->height;
    c.in_pitch_b = in->pitch_bytes;
    c.out_pitch_b = out->pitch_bytes;
    c.kw = nrow;
    c.kh = ncol;
    c.taps = row_taps;
    c.taps2 = col_taps;
    c.taps_mem = taps_mem;
    c.border = border;
    c.border_value = border_value;
    c.workspace = scratch;
    c.ws_bytes = kNoallocScratchBytes;
    imcl_variant v{};
    v.kind = IMCL_KIND_PLAIN;
    v.bx = 16;
    v.by = 16;
    ConvArgs a = make_conv_args(c, v, 1, 1);
    TapsParam<float, 66> tp;
    for (int i = 0; i < 66; ++i) tp.w[i] = 0.f;
    if (taps_mem == IMCL_MEM_HOST) {
        for (int i = 0; i < nrow; ++i) tp.w[i] = row_taps[i];
        for (int j = 0; j < ncol; ++j) tp.w[33 + j] = col_taps[j];
    }
    // The row pass writes every pixel of the intermediate before the column pass reads
    // it, so nothing left in the array by an earlier call can leak into this result.
    dim3 block(16, 16), grid = grid_2d(c.W, c.H, 16, 16);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (in->dtype * 8 + out->dtype) {
        case IMCL_F32 * 8 + IMCL_F32: noalloc_launch<float, float>(a, tp, grid, block, s); break;
        case IMCL_F16 * 8 + IMCL_F32: noalloc_launch<__half, float>(a, tp, grid, block, s); break;
        case IMCL_F16 * 8 + IMCL_F16: noalloc_launch<__half, __half>(a, tp, grid, block, s); break;
        case IMCL_BF16 * 8 + IMCL_F32: noalloc_launch<__nv_bfloat16, float>(a, tp, grid, block, s); break;
        case IMCL_BF16 * 8 + IMCL_BF16: noalloc_launch<__nv_bfloat16, __nv_bfloat16>(a, tp, grid, block, s); break;
        default: return fail(IMCL_ERR_UNSUPPORTED, "unsupported pixel-type pair");
    }
    return cuda_fail(cudaGetLastError(), "sepconv no-alloc launch");
}
