// internal.h -- declarations shared by the library's translation units (not public).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "imagecl.h"

namespace imcl {

constexpr int kMaxK = 15;   // largest odd filter side the library provides

inline int dtype_size(int dt) {
    switch (dt) {
        case IMCL_U8: return 1;
        case IMCL_I32: return 4;
        case IMCL_F32: return 4;
        case IMCL_F16: return 2;
        case IMCL_BF16: return 2;
        default: return 0;
    }
}
inline bool is_int_dtype(int dt) { return dt == IMCL_U8 || dt == IMCL_I32; }

// Per-thread error text behind imagecl_last_error().
imcl_status fail(imcl_status st, const std::string& msg);
imcl_status cuda_fail(cudaError_t e, const char* what);

// Device facts cached per device ordinal.
struct DeviceInfo {
    int ordinal = -1;
    int sm_count = 0;
    int max_smem_optin = 0;
    std::string name;
    int* status = nullptr;      // device status word (kernels' give-up codes)
};
imcl_status device_info(DeviceInfo** out);

// cuTensorMapEncodeTiled fetched from the driver at run time.
imcl_status encode_tmap_2d(CUtensorMap* map, int dtype, const void* base, int width, int height,
                           int64_t pitch_bytes, int box_w, int box_h);

// ------------------------------------------------------------------ conv2d launches
struct ConvCall {
    const void* in = nullptr;
    void* out = nullptr;
    int in_dtype = 0, out_dtype = 0;
    int W = 0, H = 0;
    int64_t in_pitch_b = 0, out_pitch_b = 0;   // bytes
    int kw = 0, kh = 0;
    const void* taps = nullptr;                // host or device, per taps_mem
    const void* taps2 = nullptr;               // sepconv: column taps; harris: Sobel y
    const void* taps3 = nullptr;               // harris: window taps
    float hk = 0.f;                            // harris: k of the response
    int taps_mem = IMCL_MEM_HOST;
    void* workspace = nullptr;                 // caller scratch (unfused variants)
    size_t ws_bytes = 0;
    int border = IMCL_BORDER_CLAMP;
    double border_value = 0.0;
    int* status = nullptr;
    const DeviceInfo* dev = nullptr;
};

using ConvLaunchFn = imcl_status (*)(const ConvCall&, const imcl_variant&, cudaStream_t);

// One compiled kernel variant.  `k` is the square filter side it is specialised for
// (0: any side, runtime loops).  `v` holds the compile-time axes; v.bx / v.by are the
// default block shape.
struct ConvEntry {
    int in_dtype, out_dtype, k;
    imcl_variant v;
    ConvLaunchFn fn;
};

void register_conv_plain(std::vector<ConvEntry>& t);
// conv2d_tiled.cu is compiled once per odd side K (3..15) and pixel-type group G
// (0 f32, 1 u8, 2 f16, 3 bf16); each object registers its tiled variants.
#define IMCL_DECL_TILED(K)                                     \
    void register_conv_tiled_k##K##_g0(std::vector<ConvEntry>& t); \
    void register_conv_tiled_k##K##_g1(std::vector<ConvEntry>& t); \
    void register_conv_tiled_k##K##_g2(std::vector<ConvEntry>& t); \
    void register_conv_tiled_k##K##_g3(std::vector<ConvEntry>& t);
IMCL_DECL_TILED(3)
IMCL_DECL_TILED(5)
IMCL_DECL_TILED(7)
IMCL_DECL_TILED(9)
IMCL_DECL_TILED(11)
IMCL_DECL_TILED(13)
IMCL_DECL_TILED(15)
#undef IMCL_DECL_TILED

// conv2d_tc.cu is compiled once per side K in {9, 11, 13, 15}: the tensor-core variants.
void register_conv_tc_k9(std::vector<ConvEntry>& t);
void register_conv_tc_k11(std::vector<ConvEntry>& t);
void register_conv_tc_k13(std::vector<ConvEntry>& t);
void register_conv_tc_k15(std::vector<ConvEntry>& t);

const std::vector<ConvEntry>& conv_table();

// Separable correlation: the same entry type; `k` is the radius R a fused kernel is
// specialised for (0 for the plain two-kernel path).  kw / kh of the call are the row
// and column tap counts.
constexpr int kMaxSepTaps = 33;
#define IMCL_DECL_SEP(G)                                          \
    void register_sep_fused_g##G##_s0(std::vector<ConvEntry>& t); \
    void register_sep_fused_g##G##_s1(std::vector<ConvEntry>& t);
IMCL_DECL_SEP(0)
IMCL_DECL_SEP(1)
IMCL_DECL_SEP(2)
#undef IMCL_DECL_SEP
const std::vector<ConvEntry>& sep_table();

// Harris: `k` is the window side a fused kernel is specialised for (0 for the plain path).
const std::vector<ConvEntry>& harris_table();

// Shared argument block of the conv2d kernels (device-visible by value).
struct ConvArgs {
    const void* in;
    void* out;
    int W, H;
    long long in_pitch, out_pitch;   // elements
    int bx, by;                      // block shape (threads)
    int tiles_x, tiles_y;
    int border;
    float bv_f;
    int bv_i;
    int vec_in, vec_out;             // 1 if vector loads / stores are aligned
    int kw, kh;                      // runtime sides (plain kernel)
    const void* taps_dev;            // device taps or nullptr
    const void* taps2_dev;           // sepconv: device column taps or nullptr
    const void* taps3_dev;           // harris: device window taps or nullptr
    float hk;                        // harris: k
    void* work;                      // caller workspace (unfused variants)
    int* status;
};

}  // namespace imcl
