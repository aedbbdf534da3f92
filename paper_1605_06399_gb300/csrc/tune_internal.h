// tune_internal.h -- the op-independent tuner and what each operator provides to it.
#pragma once

#include <functional>
#include <vector>

#include "abi_internal.h"

namespace imcl {

// Device buffers owned by one tuning run (freed when it ends).
struct TuneScratch {
    std::vector<void*> allocs;
    ~TuneScratch();
    imcl_status alloc(void** p, size_t bytes);
    // allocate a W x H image (pitch rounded to 128 bytes) filled with a hash pattern
    imcl_status image(int dtype, int W, int H, uint32_t seed, void** p, int64_t* pitch_b, cudaStream_t s);
};

// One tuning problem: candidate variants, a way to run one on the scratch images, the
// output to check, and how far a correct variant may differ from the PLAIN kernel.
struct TuneJob {
    TuneScratch scratch;
    std::vector<imcl_variant> candidates;
    std::function<imcl_status(const imcl_variant&, cudaStream_t)> run;
    void* out = nullptr;
    int out_dtype = IMCL_F32;
    int W = 0, H = 0;
    int64_t out_pitch_b = 0;
    double working_set_bytes = 0;
    float tol_abs = 0.f;
    std::vector<float> taps_f;      // host taps kept alive for the run
    std::vector<int32_t> taps_i;
    ConvCall conv;
};

std::vector<imcl_variant> expand_shapes(const std::vector<imcl_variant>& base);
imcl_status tune_search(TuneJob& job, double budget_s, int reps, cudaStream_t s, imcl_variant* best,
                        double* best_ms, double* plain_ms);

// provided per operator (tune_ops.cu)
imcl_status list_variants(const imcl_problem& p, std::vector<imcl_variant>* out);
imcl_status default_variant(const imcl_problem& p, imcl_variant* out);
imcl_status make_tune_job(const imcl_problem& p, cudaStream_t s, TuneJob* job);

}  // namespace imcl
