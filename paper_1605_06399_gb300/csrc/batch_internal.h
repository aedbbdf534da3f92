// batch_internal.h -- the ragged-batch plan behind the opaque imcl_batch handle.
#pragma once

#include <vector>

#include "internal.h"

namespace imcl {

struct BImg;
struct BTile;
struct BFwdTile;

constexpr int kQueueSlots = 8;

struct Batch {
    const DeviceInfo* dev = nullptr;
    std::vector<imcl_batch_item> items;
    std::vector<BImg> himgs;               // host copy of the image descriptors
    BImg* dimgs = nullptr;                 // device copy
    BFwdTile* tiles = nullptr;             // forward work list (device)
    int ntiles = 0;
    int* queue = nullptr;                  // work-list counters (device): [0] forward, [1] conv2d
                                           // tap tiles, [2] separable tap tiles, [3] per-image
                                           // reductions, [4] input-gradient tiles
    int py = 4, bx = 32, by = 8;           // chosen tile shape (PX = 4)
    double pixels = 0;
    double fwd_ms_at_create = 0;
    double shape_ms[4] = {0, 0, 0, 0};
    cudaStream_t cap_stream = nullptr;     // private stream the graphs are recorded on
    cudaStream_t br_stream[2] = {nullptr, nullptr};   // the backward graph's other branches
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
    cudaGraph_t fwd_graph = nullptr;
    cudaGraphExec_t fwd_exec = nullptr;
    cudaGraph_t bwd_graph = nullptr;
    cudaGraphExec_t bwd_exec = nullptr;
    int bwd_items[2] = {0, 0};             // tap-gradient tiles, per-image reductions
    int bwd_dx_tiles = 0;                  // conv2d input-gradient tiles (pipelined kernel)
    std::vector<void*> owned;              // device allocations freed with the handle
    ~Batch();
};

imcl_status batch_create(const imcl_batch_item* items, int n, double budget_s, Batch** out);
imcl_status batch_validate_item(const imcl_batch_item& it, int idx);
int batch_side(int op, int kw, int kh);
size_t batch_smem_bytes(int py, int bx, int by);

}  // namespace imcl
