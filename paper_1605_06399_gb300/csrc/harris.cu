// harris.cu -- the Harris variant table and the untuned two-kernel launcher.
#include "harris_kernels.cuh"

namespace imcl {

imcl_status launch_harris_plain(const ConvCall& c, const imcl_variant& v, cudaStream_t s) {
    const size_t need = (size_t)2 * c.W * c.H * sizeof(float);
    if (!c.workspace || c.ws_bytes < need)
        return fail(IMCL_ERR_INVALID, "the unfused Harris kernels need a workspace of 2*width*height*4 bytes");
    if (c.kw > 7) return fail(IMCL_ERR_UNSUPPORTED, "plain harris: window side above 7");
    const int bx = v.bx > 0 ? v.bx : 16, by = v.by > 0 ? v.by : 16;
    if (bx * by > 256) return fail(IMCL_ERR_UNSUPPORTED, "plain kernel: bx*by must be <= 256");
    ConvArgs a = make_conv_args(c, v, 1, 1);
    HarrisTaps<7> tp;
    fill_harris_taps(tp, c);
    dim3 grid = grid_2d(c.W, c.H, bx, by), block(bx, by);
    k_harris_sobel_plain<<<grid, block, 0, s>>>(a, tp);
    k_harris_resp_plain<<<grid, block, 0, s>>>(a, tp);
    return cuda_fail(cudaGetLastError(), "harris plain launch");
}

const std::vector<ConvEntry>& harris_table() {
    static std::vector<ConvEntry>* table = [] {
        auto* t = new std::vector<ConvEntry>();
        imcl_variant pv{};
        pv.kind = IMCL_KIND_PLAIN;
        pv.bx = 16;
        pv.by = 16;
        pv.px = 1;
        pv.py = 1;
        t->push_back(ConvEntry{IMCL_F32, IMCL_F32, 0, pv, &launch_harris_plain});
        constexpr int TMA = IMCL_LOAD_TMA, SMEM = IMCL_LOAD_SMEM;
        constexpr int PARAM = IMCL_FILT_PARAM, SFILT = IMCL_FILT_SMEM;
        t->push_back(harris_entry<5, 2, TMA, PARAM>(16, 16, 1));
        t->push_back(harris_entry<5, 4, TMA, PARAM>(16, 8, 1));
        t->push_back(harris_entry<5, 2, SMEM, PARAM>(16, 16, 0));
        t->push_back(harris_entry<5, 2, TMA, SFILT>(16, 16, 1));
        t->push_back(harris_entry<5, 4, TMA, SFILT>(16, 8, 1));
        t->push_back(harris_entry<5, 2, SMEM, SFILT>(16, 16, 0));
        t->push_back(harris_entry<3, 2, TMA, PARAM>(16, 16, 1));
        t->push_back(harris_entry<3, 2, TMA, SFILT>(16, 16, 1));
        t->push_back(harris_entry<3, 2, SMEM, PARAM>(16, 16, 0));
        t->push_back(harris_entry<3, 2, SMEM, SFILT>(16, 16, 0));
        // the paper's 2x2 block (offsets -1, 0): products over TW + 1 columns, 4 window taps
        t->push_back(harris_entry<2, 2, TMA, PARAM>(16, 16, 1));
        t->push_back(harris_entry<2, 4, TMA, PARAM>(16, 8, 1));
        t->push_back(harris_entry<2, 2, TMA, SFILT>(16, 16, 1));
        t->push_back(harris_entry<2, 2, SMEM, PARAM>(16, 16, 0));
        t->push_back(harris_entry<2, 2, SMEM, SFILT>(16, 16, 0));
        return t;
    }();
    return *table;
}

}  // namespace imcl
