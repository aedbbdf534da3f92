// sepconv_plain.cu -- the untuned two-kernel separable path (row pass into an f32
// workspace, then column pass) for every pixel-type pair, and the fused-table builder.
#include "sepconv_kernels.cuh"

namespace imcl {

template <typename Tin, typename Tout>
static ConvEntry sep_plain_entry() {
    imcl_variant v{};
    v.kind = IMCL_KIND_PLAIN;
    v.bx = 16;
    v.by = 16;
    v.px = 1;
    v.py = 1;
    v.load = IMCL_LOAD_GLOBAL;
    v.filt = IMCL_FILT_PARAM;
    v.map = IMCL_MAP_BLOCKED;
    return ConvEntry{DtypeOf<Tin>::v, DtypeOf<Tout>::v, 0, v, &launch_sep_plain<Tin, Tout>};
}

const std::vector<ConvEntry>& sep_table() {
    static std::vector<ConvEntry>* table = [] {
        auto* t = new std::vector<ConvEntry>();
        t->push_back(sep_plain_entry<float, float>());
        t->push_back(sep_plain_entry<__half, float>());
        t->push_back(sep_plain_entry<__half, __half>());
        t->push_back(sep_plain_entry<__nv_bfloat16, float>());
        t->push_back(sep_plain_entry<__nv_bfloat16, __nv_bfloat16>());
        register_sep_fused_g0_s0(*t);
        register_sep_fused_g0_s1(*t);
        register_sep_fused_g1_s0(*t);
        register_sep_fused_g1_s1(*t);
        register_sep_fused_g2_s0(*t);
        register_sep_fused_g2_s1(*t);
        return t;
    }();
    return *table;
}

}  // namespace imcl
