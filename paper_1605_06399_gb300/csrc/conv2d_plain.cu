// conv2d_plain.cu -- the untuned conv2d kernels (one per pixel-type pair) and their
// registration.  Any odd kw x kh up to 15 x 15, runtime loops.
#include "conv2d_kernels.cuh"

namespace imcl {

template <typename Tin, typename Tout>
static ConvEntry plain_entry() {
    imcl_variant v{};
    v.kind = IMCL_KIND_PLAIN;
    v.bx = 16;
    v.by = 16;
    v.px = 1;
    v.py = 1;
    v.load = IMCL_LOAD_GLOBAL;
    v.filt = IMCL_FILT_PARAM;
    v.map = IMCL_MAP_BLOCKED;
    v.unroll = 0;
    v.persistent = 0;
    return ConvEntry{DtypeOf<Tin>::v, DtypeOf<Tout>::v, 0, v, &launch_conv_plain<Tin, Tout>};
}

void register_conv_plain(std::vector<ConvEntry>& t) {
    t.push_back(plain_entry<uint8_t, int32_t>());
    t.push_back(plain_entry<int32_t, int32_t>());
    t.push_back(plain_entry<float, float>());
    t.push_back(plain_entry<__half, float>());
    t.push_back(plain_entry<__half, __half>());
    t.push_back(plain_entry<__nv_bfloat16, float>());
    t.push_back(plain_entry<__nv_bfloat16, __nv_bfloat16>());
}

}  // namespace imcl
