/*
 * imagecl.h -- C ABI of the GB300 (sm_103a) per-pixel stencil library.
 *
 * The operators follow the problem statement of ImageCL (Falch & Elster, arXiv
 * 1605.06399): a kernel runs once per pixel of an output grid (idx, idy) = (x, y)
 * (§5), reads `Image` inputs at fixed offsets (Listing 1 reads in[idx+i][idy+j]: a
 * correlation, no filter flip) and out-of-image reads follow a boundary condition,
 * clamped or constant (§5, Fig. 3).  The library is the "standalone function callable
 * from any C/C++ application" of §5.1, with the kernel variants of §5.2 / Table 1
 * (work-group size, thread coarsening, thread mapping, image/L1 versus local memory
 * staging, constant memory for the taps, loop unrolling) compiled ahead of time, and an
 * auto-tuner (§4) that times them on the device and caches the winner.
 *
 * Conventions for every entry point
 *  - Images are row-major, x fastest, with a row pitch in bytes; `data` is a DEVICE
 *    pointer owned by the caller.  The pitch must be a multiple of the element size and
 *    at least width * element size.
 *  - Operations are out of place: input and output buffers may not overlap (the paper
 *    disallows aliasing, §5.2 "Image memory"); overlap -> IMCL_ERR_INVALID.
 *  - Filter sides are odd (the taps are centred: offset = tap - (K-1)/2), 1..15.
 *    Taps are row-major, taps[j*kw + i], j the row (dy), i the column (dx).
 *  - Integer images (u8, i32) take i32 taps, accumulate in i32 with wraparound
 *    (mod 2^32) and write i32.  Floating images (f32, f16, bf16) take f32 taps,
 *    accumulate in f32 and write f32, f16 or bf16 (round to nearest even).
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream) and never synchronise, except imagecl_tune and imagecl_device_status.
 *  - No call throws.  Each returns an imcl_status; on failure imagecl_last_error()
 *    (per thread) describes it and nothing has been launched.
 *  - Kernels never trap.  A kernel that gives up on a bounded wait records a code in a
 *    per-device status word that imagecl_device_status() reads and clears.
 */
#ifndef IMAGECL_H
#define IMAGECL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IMCL_OK = 0,
    IMCL_ERR_INVALID = 1,     /* bad argument: null, size, pitch, dtype mix, aliasing  */
    IMCL_ERR_UNSUPPORTED = 2, /* well formed but not provided (even K, K > 15, variant) */
    IMCL_ERR_ALIGN = 3,       /* a requested variant needs alignment the buffers lack   */
    IMCL_ERR_OOM = 4,         /* device allocation failed (tuner, batch plans)          */
    IMCL_ERR_CUDA = 5,        /* a CUDA runtime call failed                             */
    IMCL_ERR_TIMEOUT = 6      /* a kernel gave up on a bounded wait                     */
} imcl_status;

typedef enum { IMCL_U8 = 0, IMCL_I32 = 1, IMCL_F32 = 2, IMCL_F16 = 3, IMCL_BF16 = 4 } imcl_dtype;

/* Boundary conditions of §5 / Fig. 3. */
typedef enum { IMCL_BORDER_CLAMP = 0, IMCL_BORDER_CONSTANT = 1 } imcl_border;

/* Where the filter taps live.  HOST taps are copied into the launch's parameter space
 * (the constant bank: the "constant memory" option of §5.2).  DEVICE taps are read by
 * the kernel (staged into shared memory) so the call stays asynchronous. */
typedef enum { IMCL_MEM_HOST = 0, IMCL_MEM_DEVICE = 1 } imcl_mem;

typedef struct {
    void *data;          /* device pointer, caller-owned                      */
    int32_t dtype;       /* imcl_dtype                                        */
    int32_t width;       /* pixels per row (x extent)                         */
    int32_t height;      /* rows (y extent)                                   */
    int32_t reserved;    /* must be 0                                         */
    int64_t pitch_bytes; /* bytes between the starts of consecutive rows      */
} imcl_image;

/* Kernel variant: one point of the tuning space of §5.2 / Table 1.  TENSOR (conv2d, sides
 * 9..15, f32 / f16 / bf16 images): the correlation as banded-Toeplitz matrix products on
 * the tensor cores (split-precision operands, f32 accumulation), bx = 16-column blocks
 * per work unit; the tuner offers it beside the FP32-pipe variants and keeps it only
 * when it is faster. */
typedef enum { IMCL_KIND_PLAIN = 0, IMCL_KIND_TILED = 1, IMCL_KIND_TENSOR = 2 } imcl_kind;
typedef enum { IMCL_LOAD_GLOBAL = 0, IMCL_LOAD_SMEM = 1, IMCL_LOAD_TMA = 2 } imcl_load;
typedef enum { IMCL_FILT_PARAM = 0, IMCL_FILT_SMEM = 1 } imcl_filt;
/* IMCL_MAP_REGISTER (sepconv only): the row pass result stays in each thread's registers
 * (the vertical halo rows are computed by every thread that needs them) instead of going
 * through a shared buffer -- where the intermediate of the fused pair lives. */
typedef enum { IMCL_MAP_BLOCKED = 0, IMCL_MAP_INTERLEAVED = 1, IMCL_MAP_REGISTER = 2 } imcl_map;
/* Loop form of the tap loops.  PACKED (sepconv only) is unrolled like FULL, with each
 * multiply-add instruction doing two adjacent output pixels (f32x2 FMA): the
 * vectorisation that the paper leaves to the OpenCL runtime, as a tuning knob.  It gives
 * the same bits as FULL.  F32_EXACT (conv2d, u8 images, host taps) is unrolled like FULL
 * and accumulates the integer taps and pixels with f32 FMAs: every partial sum is an
 * integer of magnitude at most sum |w| * 255, exact in f32 while that is below 2^24, so
 * the int32 result is bit-identical to integer accumulation; for larger taps the call
 * runs the integer-accumulating form of the same tile. */
typedef enum { IMCL_UNROLL_NONE = 0, IMCL_UNROLL_FULL = 1, IMCL_UNROLL_PACKED = 2,
               IMCL_UNROLL_F32_EXACT = 3 } imcl_unroll;

typedef struct {
    int32_t kind;       /* imcl_kind.  PLAIN: the untuned kernel (one pixel per thread,
                           direct clamped loads, taps read per use, rolled loops)      */
    int32_t bx, by;     /* threads per block along x and y (work-group size)          */
    int32_t px, py;     /* pixels per thread along x and y (thread coarsening)        */
    int32_t load;       /* imcl_load: L1/texture-path loads, a cooperative shared-memory
                           halo tile, or a TMA-staged shared-memory halo tile          */
    int32_t filt;       /* imcl_filt: taps in the constant bank or in shared memory   */
    int32_t map;        /* imcl_map: a thread's rows contiguous or interleaved by `by`;
                           sepconv: shared-buffer or register intermediate             */
    int32_t unroll;     /* imcl_unroll: rolled loops, taps fully unrolled (compile-time
                           K), or fully unrolled with packed f32x2 multiply-adds       */
    int32_t persistent; /* 1: one CTA per SM slot looping over tiles; 0: one tile each */
} imcl_variant;

/* What the tuner and the variant table are keyed on. */
typedef enum { IMCL_OP_CONV2D = 0, IMCL_OP_SEPCONV = 1, IMCL_OP_HARRIS = 2 } imcl_op;

typedef struct {
    int32_t op;          /* imcl_op                                                  */
    int32_t in_dtype;    /* imcl_dtype of the input image                            */
    int32_t out_dtype;   /* imcl_dtype of the output image                           */
    int32_t kw, kh;      /* conv2d: filter sides; sepconv: row taps, column taps;
                            harris: window side (both)                              */
    int32_t width, height;
    int32_t border;      /* imcl_border                                              */
    int32_t taps_mem;    /* imcl_mem                                                 */
} imcl_problem;

/* ------------------------------------------------------------------ operators */

/*
 * Non-separable correlation (§6 "non-separable convolution"; Listing 1 with weights):
 *   out(x, y) = sum_{j<kh, i<kw} taps[j*kw+i] * in(x + i - (kw-1)/2, y + j - (kh-1)/2)
 * with `border` applied to out-of-image reads of `in` (border_value for CONSTANT).
 * in:  u8/i32 (taps_dtype IMCL_I32, out IMCL_I32) or f32/f16/bf16 (taps IMCL_F32,
 *      out f32/f16/bf16).  Same width and height as out.
 * taps: kw*kh values in host or device memory as `taps_mem` says.  Host taps may be
 *      freed when the call returns; device taps must stay valid until the kernel ran.
 * variant: NULL selects the tuned variant for this problem (imagecl_tune's cache) or a
 *      default; otherwise that variant is used or IMCL_ERR_UNSUPPORTED/ALIGN returned.
 */
imcl_status imagecl_conv2d(const imcl_image *in, const imcl_image *out, const void *taps,
                           int32_t taps_dtype, int32_t kw, int32_t kh, int32_t taps_mem,
                           int32_t border, double border_value, const imcl_variant *variant,
                           void *stream);

/*
 * Separable correlation (§6 "separable convolution": a row pass then a column pass; §7
 * names fusing the two with the intermediate on chip):
 *   t(x, y)   = sum_{i<nrow} row_taps[i] * in(x + i - (nrow-1)/2, y)
 *   out(x, y) = sum_{j<ncol} col_taps[j] * t(x, y + j - (ncol-1)/2)
 * Each pass applies `border` to its own input (for CONSTANT, out-of-image reads of `in`
 * give border_value as an input pixel, those of t give it as an f32).  Under the clamped
 * rule the result equals imagecl_conv2d with the outer product col x row; under the
 * constant rule it does not unless border_value is 0.
 * in: f32, f16 or bf16; out: f32 or the input's own 16-bit type; t is kept in f32.
 * nrow, ncol: odd, 1..33 (radius up to 16).  Taps are f32, host or device per taps_mem.
 * The fused variants (the default) need no workspace.  The PLAIN variant runs the two
 * passes as two kernels with t in `workspace` (width*height*4 bytes, device memory the
 * caller owns; see imagecl_sepconv_workspace_size); a NULL or short workspace for it
 * -> IMCL_ERR_INVALID.  The default selection picks the two-kernel form only when no
 * fused variant fits or the tuner found it fastest: ask imagecl_sepconv_workspace_size.
 */
imcl_status imagecl_sepconv(const imcl_image *in, const imcl_image *out, const float *row_taps,
                            int32_t nrow, const float *col_taps, int32_t ncol, int32_t taps_mem,
                            int32_t border, double border_value, const imcl_variant *variant,
                            void *workspace, size_t workspace_bytes, void *stream);

/* Workspace bytes imagecl_sepconv needs for `problem` (op IMCL_OP_SEPCONV, sizes, tap
 * counts, types, border, taps memory) run with `variant`: 0 for the fused variants.
 * NULL: the variant a call with variant NULL would use now (the tuned one if cached). */
size_t imagecl_sepconv_workspace_size(const imcl_problem *problem, const imcl_variant *variant);

/*
 * Harris corner response (§6 corner-detection benchmark: a Sobel kernel then a Harris
 * kernel, Tables 4 and 5), clamped boundary on each stage's input:
 *   Ix = Sx (*) in,  Iy = Sy (*) in                  (3x3 correlations, sobel_x / sobel_y)
 *   Pxx = Ix^2,  Pyy = Iy^2,  Pxy = Ix Iy
 *   Sc = window (*) Pc                                (wk x wk, c in {xx, yy, xy})
 *   out = Sxx Syy - Sxy^2 - k (Sxx + Syy)^2
 * in and out: f32.  sobel_x, sobel_y: 9 taps each; window: wk*wk taps (wk 1..7);
 * all three host or device per taps_mem.  Window tap (j, i) reads the product at offset
 * (i - wk/2, j - wk/2) (integer division): centred for odd wk; for even wk (the 2x2
 * "block" of the paper's Harris benchmark) offsets -wk/2 .. wk/2-1, and the call runs
 * the (wk+1) x (wk+1) kernels with a zero last row and column (the same sums).  The
 * fused variants (the default; wk 2..5) need no workspace.  The PLAIN variant (any wk up
 * to 7) runs the paper's two kernels with Ix, Iy in `workspace` (2*width*height*4 bytes,
 * caller-owned device memory; see imagecl_harris_workspace_size); NULL or short ->
 * IMCL_ERR_INVALID.
 */
imcl_status imagecl_harris(const imcl_image *in, const imcl_image *out, const float *sobel_x,
                           const float *sobel_y, const float *window, int32_t wk, float k,
                           int32_t taps_mem, const imcl_variant *variant, void *workspace,
                           size_t workspace_bytes, void *stream);

/* Workspace bytes imagecl_harris needs for `problem` (op IMCL_OP_HARRIS, kw = window
 * side) run with `variant`: 0 for fused variants; NULL as for imagecl_sepconv. */
size_t imagecl_harris_workspace_size(const imcl_problem *problem, const imcl_variant *variant);

/* ------------------------------------------------------------------ gradients */

/*
 * Adjoint (backward) passes.  The forward operators are linear in their input and in
 * their taps (Harris: polynomial), so the gradients are the transposed maps:
 *  - input gradient: correlation of grad_out with the flipped taps under a zero border,
 *    plus, for the clamped rule, the contributions of taps that were clamped, summed
 *    onto the first/last rows and columns (the transpose of the clamp);
 *  - tap gradient: dtaps[o] = sum_p grad_out(p) * in_b(p + o), with in_b the boundary
 *    rule's read, reduced per CTA and then over CTAs in a fixed order (deterministic);
 *  - Harris: the chain rule R -> (Sxx, Syy, Sxy) -> products -> (Ix, Iy) -> image, and
 *    the window and Sobel tap gradients on the way (any window side 1..7, anchored as in
 *    imagecl_harris).
 * grad_out is f32 with the size of `in`; in is f32, f16 or bf16 (Harris: f32).
 * grad_in (f32, nullable: not computed) must not overlap grad_out or in.  The tap
 * gradients (nullable) are device f32 arrays the caller owns, written (not accumulated).
 * workspace: device memory the caller owns, at least the *_workspace_size bytes for the
 * same sizes (always required).  Asynchronous on `stream`.
 */
imcl_status imagecl_conv2d_backward(const imcl_image *grad_out, const imcl_image *in,
                                    const float *taps, int32_t kw, int32_t kh, int32_t taps_mem,
                                    int32_t border, double border_value,
                                    const imcl_image *grad_in, float *grad_taps,
                                    void *workspace, size_t workspace_bytes, void *stream);
size_t imagecl_conv2d_backward_workspace_size(int32_t width, int32_t height, int32_t kw,
                                              int32_t kh);

imcl_status imagecl_sepconv_backward(const imcl_image *grad_out, const imcl_image *in,
                                     const float *row_taps, int32_t nrow, const float *col_taps,
                                     int32_t ncol, int32_t taps_mem, int32_t border,
                                     double border_value, const imcl_image *grad_in,
                                     float *grad_row, float *grad_col, void *workspace,
                                     size_t workspace_bytes, void *stream);
size_t imagecl_sepconv_backward_workspace_size(int32_t width, int32_t height, int32_t nrow,
                                               int32_t ncol);

imcl_status imagecl_harris_backward(const imcl_image *grad_out, const imcl_image *in,
                                    const float *sobel_x, const float *sobel_y,
                                    const float *window, int32_t wk, float k, int32_t taps_mem,
                                    const imcl_image *grad_in, float *grad_sobel_x,
                                    float *grad_sobel_y, float *grad_window, void *workspace,
                                    size_t workspace_bytes, void *stream);
size_t imagecl_harris_backward_workspace_size(int32_t width, int32_t height, int32_t wk);

/* ------------------------------------------------------------------ ragged batch */

/*
 * A batch of independent image operations of uneven sizes (each image with its own
 * conv2d filter or separable pair) run by one persistent kernel: every tile of every
 * image goes into one work list, costliest first, that a grid of resident CTAs drains
 * with an atomic counter.  imagecl_batch_create validates the items, times a few tile
 * shapes on the whole batch (up to tune_budget_s) and keeps the fastest, and records the
 * launch in a CUDA graph; imagecl_batch_run replays it.  The plan stores the pointers it
 * was given: keep every buffer alive and in place while the handle lives, and change
 * pixel or tap values in place between runs as you like.
 * Per item: in f32/f16/bf16, out f32 or the input's type, same size, no overlap; conv2d
 * sides / separable tap counts odd, at most 15; taps are DEVICE f32 arrays.  The
 * gradient fields are used by imagecl_batch_backward (NULL data / pointers: skipped).
 */
typedef struct {
    int32_t op;            /* IMCL_OP_CONV2D or IMCL_OP_SEPCONV                              */
    int32_t border;        /* imcl_border                                                    */
    int32_t kw, kh;        /* conv2d: filter sides; sepconv: row / column tap counts         */
    double border_value;
    imcl_image in, out;
    const float *taps;     /* conv2d: kw*kh taps; sepconv: row taps (device)                 */
    const float *taps2;    /* sepconv: column taps (device); NULL for conv2d                 */
    imcl_image grad_out;   /* f32 upstream gradient (for imagecl_batch_backward)              */
    imcl_image grad_in;    /* f32 input gradient, written by imagecl_batch_backward           */
    float *grad_taps;      /* conv2d taps / sepconv row taps gradient (device), written       */
    float *grad_taps2;     /* sepconv column taps gradient (device), written                  */
} imcl_batch_item;

typedef struct imcl_batch imcl_batch;   /* opaque plan */

typedef struct {
    int32_t images, tiles, tile_w, tile_h;
    double pixels;             /* output pixels of one forward run                        */
    double fwd_ms_at_create;   /* forward time of the chosen shape when it was tuned      */
    double shape_ms[4];        /* forward time of each tile shape tried (0: not tried)    */
    int32_t has_backward;
} imcl_batch_info_t;

imcl_status imagecl_batch_create(const imcl_batch_item *items, int32_t n, double tune_budget_s,
                                 imcl_batch **out);
/* Forward over the whole batch: one graph launch on `stream`. */
imcl_status imagecl_batch_run(imcl_batch *batch, void *stream);
/*
 * Backward over the whole batch (the adjoints of imagecl_conv2d_backward and
 * imagecl_sepconv_backward for every item with a grad_out): one graph launch.  On one
 * branch the forward's pipelined tile kernel computes every grad_in as the correlation of
 * grad_out with the flipped taps under a zero border and adds the clamp folds at the edge
 * pixels of clamped items; beside it a persistent phase computes each tile's tap-gradient
 * partial sums (conv2d: the K x K taps; separable: column and row taps from one staging),
 * followed by fixed-order reductions of the partial sums into grad_taps / grad_taps2.
 * IMCL_ERR_INVALID if no item carries gradient buffers.
 */
imcl_status imagecl_batch_backward(imcl_batch *batch, void *stream);
imcl_status imagecl_batch_info(const imcl_batch *batch, imcl_batch_info_t *info);
void imagecl_batch_destroy(imcl_batch *batch);

/*
 * imagecl_sepconv_noalloc -- the separable correlation for callers that may not
 * allocate device memory.  The paper has no counterpart; this entry point exists for
 * deployment.  Some callers cannot call cudaMalloc (or anything that allocates) while
 * they run: plugins whose host framework owns all device memory through its own
 * allocator, and real-time loops that cannot take the device-wide synchronisation an
 * allocation or a free may cause.  They still pass their own input and output
 * images; the one intermediate this operation needs (the f32 row pass) lives in a
 * fixed array of IMAGECL_NOALLOC_SCRATCH_BYTES that the library declares in device
 * memory.  Every GPU that loads the library holds that array until the process exits.
 *
 * Arguments and result are those of imagecl_sepconv run with the PLAIN variant (same
 * kernels, same result bit for bit), without the variant and workspace arguments.
 * Limits and behaviour:
 *  - width * height * 4 must not exceed IMAGECL_NOALLOC_SCRATCH_BYTES (16 MiB, i.e.
 *    4,194,304 pixels); larger images -> IMCL_ERR_UNSUPPORTED.
 *  - No cudaMalloc, cudaFree or other allocating call is made.  The first call on each
 *    device looks up the array's device address (cudaGetSymbolAddress) with that device
 *    current and caches it; make that first call before any stream capture begins.
 *  - All calls share the one array per device, which keeps the last call's contents.
 *    Nothing in it needs clearing (the row pass writes every value the column pass
 *    reads), but calls whose kernels overlap on the same GPU race on it: order them on
 *    one stream or synchronise between them.
 */
#define IMAGECL_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
imcl_status imagecl_sepconv_noalloc(const imcl_image *in, const imcl_image *out,
                                    const float *row_taps, int32_t nrow, const float *col_taps,
                                    int32_t ncol, int32_t taps_mem, int32_t border,
                                    double border_value, void *stream);

/* ------------------------------------------------------------------ tuning */

/* Number of compiled variants applicable to `problem` (0 if none), and the idx-th one.
 * Block shapes (bx, by) of TILED entries are a default; the tuner also sweeps them. */
int32_t imagecl_variant_count(const imcl_problem *problem);
imcl_status imagecl_variant_get(const imcl_problem *problem, int32_t idx, imcl_variant *out);

/* The variant imagecl_conv2d / _sepconv / _harris would use for `problem` right now
 * (the cached tuning result if there is one, else the built-in default). */
imcl_status imagecl_variant_default(const imcl_problem *problem, imcl_variant *out);

/*
 * Auto-tune (§4, Fig. 2: pick a configuration, run and time it on the device, repeat,
 * keep the best): allocates scratch images of the problem's size, runs every
 * applicable variant and block shape (up to `budget_s` seconds), checks each against
 * the PLAIN kernel on the same input, times the survivors with CUDA events on `stream`
 * (median of `reps` runs after warm-up, L2 flushed between runs), and stores the
 * fastest in the per-process cache, which imagecl_conv2d and friends then use.
 * Synchronises `stream`.  `best` and `best_ms` / `plain_ms` (nullable) receive the
 * winner, its time and the PLAIN kernel's time.  Returns IMCL_ERR_OOM if the scratch
 * images do not fit.
 */
imcl_status imagecl_tune(const imcl_problem *problem, double budget_s, int32_t reps,
                         imcl_variant *best, double *best_ms, double *plain_ms, void *stream);

/*
 * Model-guided tuning (§4: the paper's auto-tuner times a random sample of
 * configurations, fits an artificial neural network to their run times, predicts the
 * time of every configuration and runs the best predicted ones).  The space is that of
 * imagecl_tune (variants x block shapes).  `n_sample` configurations drawn with `seed`
 * are checked against the PLAIN kernel and timed; a one-hidden-layer network (16 tanh
 * units) is fitted to their log times from the configuration's axes (one-hot per axis
 * value); the `n_confirm` untimed configurations it predicts fastest are then checked
 * and timed; then up to 8 further configurations drawn at random from the untimed ones
 * are timed as a held-out check of the model (its prediction error on data it did not
 * train on).  The fastest of all timed ones is cached as imagecl_tune would.
 * `report` (nullable) receives the counts, the model's fit, its held-out error and the
 * search's wall time.
 * Synchronises `stream`.
 */
typedef struct {
    int32_t candidates;    /* configurations in the space                              */
    int32_t sampled;       /* drawn at random and timed to train the model             */
    int32_t confirmed;     /* best-predicted configurations timed afterwards           */
    int32_t valid;         /* timed configurations that launched and passed the check  */
    double model_rmse;     /* rms error of the fitted log time on the sampled points   */
    double seconds;        /* wall time of the search                                  */
    int32_t holdout;       /* random untimed configurations timed after training       */
    int32_t holdout_valid; /* of those, the ones that launched and passed the check    */
    double holdout_rmse;   /* rms error of the predicted log time on the valid held-out */
} imcl_tune_report;

imcl_status imagecl_tune_model(const imcl_problem *problem, int32_t n_sample, int32_t n_confirm,
                               int32_t reps, uint64_t seed, imcl_variant *best, double *best_ms,
                               double *plain_ms, imcl_tune_report *report, void *stream);

/* Store / drop a tuning result by hand (the "force an optimisation" directive of §5). */
imcl_status imagecl_tune_set(const imcl_problem *problem, const imcl_variant *variant);
void imagecl_tune_clear(void);

/* Write / read the tuning cache as text (one problem and variant per line).  The file
 * records the device name and SM count; entries for another device are skipped. */
imcl_status imagecl_tune_save(const char *path);
imcl_status imagecl_tune_load(const char *path);

/* ------------------------------------------------------------------ measurement */

/* FP32 pipe throughput of the current device in TFLOP/s (2 flops per FMA), measured with
 * independent FMA chains (packed = 0: scalar FMAs; 1: packed f32x2 FMAs).  A measurement
 * helper for the ALU roofline of the stencils, not an operator; synchronises `stream`. */
imcl_status imagecl_probe_fp32(int32_t packed, double *tflops, void *stream);

/* Integer multiply-add throughput of the current device in tera-operations per second
 * (2 per wrapping int32 multiply-add), measured with independent chains: the ALU
 * roofline of the integer (u8 -> i32) correlation.  Synchronises `stream`. */
imcl_status imagecl_probe_imad(double *tops, void *stream);

/* Failure-path self-test.  Launches one thread that arms an mbarrier for a transfer that
 * never comes, waits at most `rounds` (1 .. 2^20) try_wait rounds, gives up and records
 * code 1 (a bounded wait timed out) in the device status word, as every stencil kernel
 * does when its own wait runs out.  No fault and no hang: the context stays usable, and
 * imagecl_device_status() then reports 1 (and clears it).  Asynchronous on `stream`. */
imcl_status imagecl_selftest_wait_timeout(int32_t rounds, void *stream);

/* ------------------------------------------------------------------ status */

/* Human-readable description of this thread's last failed call ("" if none). */
const char *imagecl_last_error(void);

/* Synchronises `stream`, then reads and clears the current device's kernel status word
 * (0 = no kernel gave up; 1 = a bounded wait timed out; 2 = a bounds check tripped). */
imcl_status imagecl_device_status(int32_t *code, void *stream);

/* Library version, e.g. "imagecl-gb300 0.1 sm_103a". */
const char *imagecl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IMAGECL_H */
