// runtime.cu -- per-thread errors, per-device facts, TMA descriptors, occupancy cache,
// and the table of compiled conv2d variants.
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "internal.h"

namespace imcl {

static thread_local std::string t_last_error;

imcl_status fail(imcl_status st, const std::string& msg) {
    t_last_error = msg;
    return st;
}

imcl_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return IMCL_OK;
    t_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? IMCL_ERR_OOM : IMCL_ERR_CUDA;
}

const char* last_error_text() { return t_last_error.c_str(); }
void clear_last_error() { t_last_error.clear(); }

// ------------------------------------------------------------------ device facts
static std::mutex g_dev_mu;
static std::map<int, DeviceInfo*> g_devs;

imcl_status device_info(DeviceInfo** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = g_devs.find(dev);
    if (it != g_devs.end()) {
        *out = it->second;
        return IMCL_OK;
    }
    DeviceInfo* d = new DeviceInfo();
    d->ordinal = dev;
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) { delete d; return cuda_fail(e, "cudaGetDeviceProperties"); }
    d->sm_count = prop.multiProcessorCount;
    d->name = prop.name;
    e = cudaDeviceGetAttribute(&d->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) { delete d; return cuda_fail(e, "max shared memory attribute"); }
    e = cudaMalloc(&d->status, sizeof(int));
    if (e != cudaSuccess) { delete d; return cuda_fail(e, "status word allocation"); }
    e = cudaMemset(d->status, 0, sizeof(int));
    if (e != cudaSuccess) { cudaFree(d->status); delete d; return cuda_fail(e, "status word reset"); }
    g_devs[dev] = d;
    *out = d;
    return IMCL_OK;
}

// ------------------------------------------------------------------ TMA descriptors
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

imcl_status encode_tmap_2d(CUtensorMap* map, int dtype, const void* base, int width, int height,
                           int64_t pitch_bytes, int box_w, int box_h) {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) return fail(IMCL_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    CUtensorMapDataType t;
    switch (dtype) {
        case IMCL_U8: t = CU_TENSOR_MAP_DATA_TYPE_UINT8; break;
        case IMCL_I32: t = CU_TENSOR_MAP_DATA_TYPE_INT32; break;
        case IMCL_F32: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
        case IMCL_F16: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
        case IMCL_BF16: t = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
        default: return fail(IMCL_ERR_INVALID, "TMA: unknown dtype");
    }
    cuuint64_t gdim[2] = {(cuuint64_t)width, (cuuint64_t)height};
    cuuint64_t gstride[1] = {(cuuint64_t)pitch_bytes};
    cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, t, 2, const_cast<void*>(base), gdim, gstride, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[160];
        snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d) for %dx%d pitch %lld box %dx%d", (int)r,
                 width, height, (long long)pitch_bytes, box_w, box_h);
        return fail(IMCL_ERR_ALIGN, buf);
    }
    return IMCL_OK;
}

// ------------------------------------------------------------------ kernel attributes
static std::mutex g_attr_mu;
static std::map<std::pair<const void*, int>, int> g_smem_set;             // (fn, device) -> bytes
static std::map<std::tuple<const void*, int, int, int>, int> g_occ;        // (fn, dev, thr, smem)

imcl_status set_smem_limit(const void* fn, int smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto key = std::make_pair(fn, dev);
    auto it = g_smem_set.find(key);
    if (it != g_smem_set.end() && it->second >= smem) return IMCL_OK;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(max dynamic smem)");
    g_smem_set[key] = smem;
    return IMCL_OK;
}

int cached_occupancy(const void* fn, int threads, int smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto key = std::make_tuple(fn, dev, threads, smem);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess) n = 0;
    g_occ[key] = n;
    return n;
}

// ------------------------------------------------------------------ conv2d helpers
ConvArgs make_conv_args(const ConvCall& c, const imcl_variant& v, int in_align, int out_align) {
    ConvArgs a;
    memset(&a, 0, sizeof a);
    const int isz = dtype_size(c.in_dtype), osz = dtype_size(c.out_dtype);
    a.in = c.in;
    a.out = c.out;
    a.W = c.W;
    a.H = c.H;
    a.in_pitch = c.in_pitch_b / isz;
    a.out_pitch = c.out_pitch_b / osz;
    a.bx = v.bx;
    a.by = v.by;
    a.border = c.border;
    a.bv_f = (float)c.border_value;
    a.bv_i = (int)c.border_value;
    a.vec_in = ((reinterpret_cast<uintptr_t>(c.in) % in_align) == 0 && (c.in_pitch_b % in_align) == 0) ? 1 : 0;
    a.vec_out = ((reinterpret_cast<uintptr_t>(c.out) % out_align) == 0 && (c.out_pitch_b % out_align) == 0) ? 1 : 0;
    a.kw = c.kw;
    a.kh = c.kh;
    a.taps_dev = c.taps_mem == IMCL_MEM_DEVICE ? c.taps : nullptr;
    a.taps2_dev = c.taps_mem == IMCL_MEM_DEVICE ? c.taps2 : nullptr;
    a.taps3_dev = c.taps_mem == IMCL_MEM_DEVICE ? c.taps3 : nullptr;
    a.hk = c.hk;
    a.work = c.workspace;
    a.status = c.status;
    return a;
}

const std::vector<ConvEntry>& conv_table() {
    static std::vector<ConvEntry>* table = [] {
        auto* t = new std::vector<ConvEntry>();
        register_conv_plain(*t);
#define IMCL_REG_TILED(K)               \
    register_conv_tiled_k##K##_g0(*t); \
    register_conv_tiled_k##K##_g1(*t); \
    register_conv_tiled_k##K##_g2(*t); \
    register_conv_tiled_k##K##_g3(*t);
        IMCL_REG_TILED(3)
        IMCL_REG_TILED(5)
        IMCL_REG_TILED(7)
        IMCL_REG_TILED(9)
        IMCL_REG_TILED(11)
        IMCL_REG_TILED(13)
        IMCL_REG_TILED(15)
#undef IMCL_REG_TILED
        register_conv_tc_k9(*t);
        register_conv_tc_k11(*t);
        register_conv_tc_k13(*t);
        register_conv_tc_k15(*t);
        return t;
    }();
    return *table;
}

}  // namespace imcl
