// abi_internal.h -- helpers shared by the entry-point translation units (not public).
#pragma once

#include <string>
#include <vector>

#include "internal.h"

namespace imcl {

imcl_status check_image(const imcl_image* im, const char* name);
bool images_overlap(const imcl_image* a, const imcl_image* b);
imcl_status check_border(int border, double bv, int in_dtype);
imcl_status check_side(int k, const char* what);

std::string problem_key(const imcl_problem& p);
bool cache_lookup(const imcl_problem& p, imcl_variant* v);
void cache_store(const imcl_problem& p, const imcl_variant& v);

imcl_problem conv_problem(const ConvCall& c);
// The variant a call uses when none is given and none is cached: taps memory decides
// where the taps live, TMA staging only on 16-byte aligned buffers, PLAIN last.
imcl_variant pick_default(const std::vector<const ConvEntry*>& entries, int taps_mem, bool tma_ok, int want_px,
                          int want_py);
bool tma_aligned(const ConvCall& c);
// A ConvCall describing `p` on hypothetical, fully aligned buffers (no device).
ConvCall problem_call(const imcl_problem& p);
std::vector<const ConvEntry*> conv_entries_for(int in_dt, int out_dt, int kw, int kh, int taps_mem);
const ConvEntry* conv_find(const ConvCall& c, const imcl_variant& v);
imcl_variant conv_default_variant(const ConvCall& c);
imcl_status conv_prepare(const imcl_image* in, const imcl_image* out, const void* taps, int taps_dtype, int kw,
                         int kh, int taps_mem, int border, double bv, ConvCall* c);
imcl_status conv_run(const ConvCall& c, const imcl_variant* variant, cudaStream_t s);

imcl_problem sep_problem(const ConvCall& c);
std::vector<const ConvEntry*> sep_entries_for(int in_dt, int out_dt, int nr, int nc, int taps_mem);
imcl_variant sep_default_variant(const ConvCall& c);
imcl_status sep_prepare(const imcl_image* in, const imcl_image* out, const float* row, int nr, const float* col,
                        int nc, int taps_mem, int border, double bv, void* ws, size_t ws_bytes, ConvCall* c);
imcl_status sep_run(const ConvCall& c, const imcl_variant* variant, cudaStream_t s);

int harris_kernel_side(int wk);
int harris_forward_side(int wk);
ConvCall harris_problem_call(const imcl_problem& p);
imcl_problem harris_problem(const ConvCall& c);
std::vector<const ConvEntry*> harris_entries_for(int wk, int taps_mem);
imcl_variant harris_default_variant(const ConvCall& c);
imcl_status harris_prepare(const imcl_image* in, const imcl_image* out, const float* sx, const float* sy,
                           const float* win, int wk, float k, int taps_mem, void* ws, size_t ws_bytes,
                           ConvCall* c);
imcl_status harris_run(const ConvCall& c, const imcl_variant* variant, cudaStream_t s);

}  // namespace imcl
