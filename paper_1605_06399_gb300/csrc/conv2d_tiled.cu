// conv2d_tiled.cu -- instantiates the tiled conv2d variants for one filter side and one
// pixel-type group.  Built once per (K, group) with -DIMCL_TILED_K=K
// -DIMCL_TILED_GROUP=G (G: 0 f32, 1 u8, 2 f16, 3 bf16) so the heavy unrolled kernels
// compile in parallel.  The set is the tuning space the tuner sweeps (Table 1:
// coarsening PX x PY, shared-memory staging by TMA or cooperative loads versus the
// L1/texture path, taps in the constant bank or shared memory, blocked or interleaved
// row mapping); block shapes are swept at run time.  The full f32 space is compiled
// for K in {3, 5, 7, 11}; the other sides get the variants that win there.
#include "conv2d_kernels.cuh"

#if !defined(IMCL_TILED_K) || !defined(IMCL_TILED_GROUP)
#error "compile with -DIMCL_TILED_K=<odd side> -DIMCL_TILED_GROUP=<0..3>"
#endif

#define IMCL_CAT2(a, b) a##b
#define IMCL_CAT(a, b) IMCL_CAT2(a, b)
#define IMCL_REG_NAME IMCL_CAT(IMCL_CAT(IMCL_CAT(register_conv_tiled_k, IMCL_TILED_K), _g), IMCL_TILED_GROUP)

namespace imcl {

constexpr int K = IMCL_TILED_K;
constexpr int TMA = IMCL_LOAD_TMA, SMEM = IMCL_LOAD_SMEM, GLB = IMCL_LOAD_GLOBAL;
constexpr int PARAM = IMCL_FILT_PARAM, SFILT = IMCL_FILT_SMEM;
constexpr int BLK = IMCL_MAP_BLOCKED, ILV = IMCL_MAP_INTERLEAVED;
constexpr bool kFullSpace = (K == 3 || K == 5 || K == 7 || K == 11);

template <typename Tin, typename Tout>
static void add_16bit(std::vector<ConvEntry>& t) {
    t.push_back(conv_entry<Tin, Tout, K, 4, 4, TMA, PARAM, BLK>(32, 8, 1));
    t.push_back(conv_entry<Tin, Tout, K, 4, 4, TMA, SFILT, BLK>(32, 8, 1));
    t.push_back(conv_entry<Tin, Tout, K, 4, 4, GLB, SFILT, BLK>(32, 8, 0));
    if constexpr (K <= 7) {
        t.push_back(conv_entry<Tin, Tout, K, 4, 8, TMA, PARAM, BLK>(32, 4, 1));
        t.push_back(conv_entry<Tin, Tout, K, 4, 4, GLB, PARAM, BLK>(32, 8, 0));
    }
}

void IMCL_REG_NAME(std::vector<ConvEntry>& t) {
#if IMCL_TILED_GROUP == 0
    t.push_back(conv_entry<float, float, K, 4, 4, TMA, PARAM, BLK>(32, 8, 1));
    t.push_back(conv_entry<float, float, K, 4, 8, TMA, PARAM, BLK>(32, 4, 1));
    t.push_back(conv_entry<float, float, K, 4, 4, TMA, SFILT, BLK>(32, 8, 1));
    t.push_back(conv_entry<float, float, K, 4, 4, GLB, PARAM, BLK>(32, 8, 0));
    t.push_back(conv_entry<float, float, K, 4, 4, GLB, SFILT, BLK>(32, 8, 0));
    if constexpr (kFullSpace) {
        t.push_back(conv_entry<float, float, K, 4, 2, TMA, PARAM, BLK>(32, 8, 1));
        t.push_back(conv_entry<float, float, K, 8, 2, TMA, PARAM, BLK>(16, 8, 1));
        t.push_back(conv_entry<float, float, K, 8, 4, TMA, PARAM, BLK>(16, 8, 1));
        t.push_back(conv_entry<float, float, K, 4, 4, SMEM, PARAM, BLK>(32, 8, 0));
        t.push_back(conv_entry<float, float, K, 4, 8, SMEM, PARAM, BLK>(32, 4, 0));
        t.push_back(conv_entry<float, float, K, 4, 8, GLB, PARAM, BLK>(32, 4, 0));
        t.push_back(conv_entry<float, float, K, 4, 8, TMA, SFILT, BLK>(32, 4, 1));
        t.push_back(conv_entry<float, float, K, 4, 4, TMA, PARAM, ILV>(32, 8, 1));
    }
#elif IMCL_TILED_GROUP == 1
    // f32 accumulation of the integer taps (exact below 2^24, else the integer twin runs)
    t.push_back(conv_entry<uint8_t, int32_t, K, 4, 4, TMA, PARAM, BLK, true>(32, 8, 1));
    t.push_back(conv_entry<uint8_t, int32_t, K, 4, 8, TMA, PARAM, BLK, true>(32, 4, 1));
    t.push_back(conv_entry<uint8_t, int32_t, K, 4, 4, TMA, PARAM, BLK>(32, 8, 1));
    t.push_back(conv_entry<uint8_t, int32_t, K, 4, 4, TMA, SFILT, BLK>(32, 8, 1));
    if constexpr (K <= 5) {
        t.push_back(conv_entry<uint8_t, int32_t, K, 4, 2, TMA, PARAM, BLK>(32, 8, 1));
        t.push_back(conv_entry<uint8_t, int32_t, K, 4, 4, SMEM, PARAM, BLK>(32, 8, 0));
        t.push_back(conv_entry<uint8_t, int32_t, K, 4, 4, GLB, PARAM, BLK>(32, 8, 0));
    }
#elif IMCL_TILED_GROUP == 2
    add_16bit<__half, float>(t);
    add_16bit<__half, __half>(t);
#elif IMCL_TILED_GROUP == 3
    add_16bit<__nv_bfloat16, float>(t);
    add_16bit<__nv_bfloat16, __nv_bfloat16>(t);
#endif
}

}  // namespace imcl
