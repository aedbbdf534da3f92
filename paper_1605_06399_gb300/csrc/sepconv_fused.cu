// sepconv_fused.cu -- instantiates the fused separable variants for one pixel-type
// group and one range of radii.  Built once per (group, range) with
// -DIMCL_SEP_GROUP=G (0 f32, 1 f16, 2 bf16) -DIMCL_SEP_RSET=S (0: R 1..8, 1: R 9..16).
#include "sepconv_kernels.cuh"

#if !defined(IMCL_SEP_GROUP) || !defined(IMCL_SEP_RSET)
#error "compile with -DIMCL_SEP_GROUP=<0..2> -DIMCL_SEP_RSET=<0..1>"
#endif

#define IMCL_CAT2(a, b) a##b
#define IMCL_CAT(a, b) IMCL_CAT2(a, b)
#define IMCL_REG_NAME IMCL_CAT(IMCL_CAT(IMCL_CAT(register_sep_fused_g, IMCL_SEP_GROUP), _s), IMCL_SEP_RSET)

namespace imcl {

constexpr int TMA = IMCL_LOAD_TMA, SMEM = IMCL_LOAD_SMEM, GLB = IMCL_LOAD_GLOBAL;
constexpr int PARAM = IMCL_FILT_PARAM, SFILT = IMCL_FILT_SMEM;
constexpr int PK = IMCL_UNROLL_PACKED;

// register-intermediate forms (MODE 1) for the small radii
template <typename Tin, typename Tout, int R>
static void add_register_forms(std::vector<ConvEntry>& t) {
    if constexpr (R <= 8) {
        t.push_back(sep_entry<Tin, Tout, R, 4, 8, TMA, PARAM, 1>(32, 8, 1));
        t.push_back(sep_entry<Tin, Tout, R, 4, 8, TMA, SFILT, 1>(32, 8, 1));
        t.push_back(sep_entry<Tin, Tout, R, 4, 8, TMA, PARAM, 1, PK>(32, 8, 1));
    }
    if constexpr (R <= 4) {
        t.push_back(sep_entry<Tin, Tout, R, 4, 4, TMA, PARAM, 1>(16, 16, 1));
        t.push_back(sep_entry<Tin, Tout, R, 4, 16, TMA, PARAM, 1>(32, 4, 1));
        t.push_back(sep_entry<Tin, Tout, R, 4, 16, TMA, PARAM, 1, PK>(32, 4, 1));
    }
}

// packed f32x2 forms of the shared-buffer kernel
template <typename Tin, typename Tout, int R>
static void add_packed_forms(std::vector<ConvEntry>& t) {
    t.push_back(sep_entry<Tin, Tout, R, 4, 8, TMA, PARAM, 0, PK>(32, 8, 1));
    t.push_back(sep_entry<Tin, Tout, R, 4, 8, TMA, SFILT, 0, PK>(32, 8, 1));
}

template <int R>
static void add_radius(std::vector<ConvEntry>& t) {
#if IMCL_SEP_GROUP == 0
    add_register_forms<float, float, R>(t);
    t.push_back(sep_entry<float, float, R, 4, 8, TMA, PARAM>(32, 8, 1));
    t.push_back(sep_entry<float, float, R, 4, 4, TMA, PARAM>(32, 8, 1));
    t.push_back(sep_entry<float, float, R, 4, 8, SMEM, PARAM>(32, 8, 0));
    t.push_back(sep_entry<float, float, R, 4, 8, GLB, PARAM>(32, 8, 0));
    t.push_back(sep_entry<float, float, R, 4, 8, TMA, SFILT>(32, 8, 1));
    t.push_back(sep_entry<float, float, R, 4, 8, GLB, SFILT>(32, 8, 0));
    add_packed_forms<float, float, R>(t);
#elif IMCL_SEP_GROUP == 1
    add_register_forms<__half, float, R>(t);
    add_register_forms<__half, __half, R>(t);
    t.push_back(sep_entry<__half, float, R, 4, 8, TMA, PARAM>(32, 8, 1));
    t.push_back(sep_entry<__half, float, R, 4, 8, TMA, SFILT>(32, 8, 1));
    t.push_back(sep_entry<__half, float, R, 4, 8, GLB, PARAM>(32, 8, 0));
    t.push_back(sep_entry<__half, float, R, 4, 8, GLB, SFILT>(32, 8, 0));
    t.push_back(sep_entry<__half, __half, R, 4, 8, TMA, PARAM>(32, 8, 1));
    t.push_back(sep_entry<__half, __half, R, 4, 8, TMA, SFILT>(32, 8, 1));
    t.push_back(sep_entry<__half, __half, R, 4, 8, GLB, PARAM>(32, 8, 0));
    t.push_back(sep_entry<__half, __half, R, 4, 8, GLB, SFILT>(32, 8, 0));
    add_packed_forms<__half, float, R>(t);
    add_packed_forms<__half, __half, R>(t);
#else
    add_register_forms<__nv_bfloat16, float, R>(t);
    add_register_forms<__nv_bfloat16, __nv_bfloat16, R>(t);
    t.push_back(sep_entry<__nv_bfloat16, float, R, 4, 8, TMA, PARAM>(32, 8, 1));
    t.push_back(sep_entry<__nv_bfloat16, float, R, 4, 8, TMA, SFILT>(32, 8, 1));
    t.push_back(sep_entry<__nv_bfloat16, float, R, 4, 8, GLB, PARAM>(32, 8, 0));
    t.push_back(sep_entry<__nv_bfloat16, float, R, 4, 8, GLB, SFILT>(32, 8, 0));
    t.push_back(sep_entry<__nv_bfloat16, __nv_bfloat16, R, 4, 8, TMA, PARAM>(32, 8, 1));
    t.push_back(sep_entry<__nv_bfloat16, __nv_bfloat16, R, 4, 8, TMA, SFILT>(32, 8, 1));
    t.push_back(sep_entry<__nv_bfloat16, __nv_bfloat16, R, 4, 8, GLB, PARAM>(32, 8, 0));
    t.push_back(sep_entry<__nv_bfloat16, __nv_bfloat16, R, 4, 8, GLB, SFILT>(32, 8, 0));
    add_packed_forms<__nv_bfloat16, float, R>(t);
    add_packed_forms<__nv_bfloat16, __nv_bfloat16, R>(t);
#endif
}

void IMCL_REG_NAME(std::vector<ConvEntry>& t) {
#if IMCL_SEP_RSET == 0
    add_radius<1>(t); add_radius<2>(t); add_radius<3>(t); add_radius<4>(t);
    add_radius<5>(t); add_radius<6>(t); add_radius<7>(t); add_radius<8>(t);
#else
    add_radius<9>(t); add_radius<10>(t); add_radius<11>(t); add_radius<12>(t);
    add_radius<13>(t); add_radius<14>(t); add_radius<15>(t); add_radius<16>(t);
#endif
}

}  // namespace imcl
