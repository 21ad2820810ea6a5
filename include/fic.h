/*
 * fic.h -- C ABI of the GB300 (sm_103a) fractal image encoder.
 *
 * Method: "A Fast Fractal Image Compression Algorithm Using Predefined Values
 * for Contrast Scaling" (Miar Naimi, Salarian).  Sec. 2 defines the problem:
 * partition a grey-level image into B x B range blocks; take every 2B x 2B
 * square at integer step L as a domain, decimate it to B x B and extend the
 * pool with its 4 clockwise rotations and their mirrors; for each range pick
 * the domain, isometry and contrast scale s minimising
 *     E(R, D) = sum_i (s d_i + o - r_i)^2                         (Eq. 1)
 * with o = Rbar - s Dbar (Eq. 3); save the map when the error is acceptable,
 * otherwise split the range into four (16 -> 8 -> 4 -> 2).  Sec. 3 keeps only
 * domains whose entropy (Eq. 4-5) is greater than a threshold, and Sec. 3.1
 * replaces the search of s over [0, 1] by predefined values per step.
 *
 * Conventions shared by every call:
 *   - Status: every int-returning call returns FIC_OK (0) or a negative
 *     FIC_E* code; fic_status_string() names it.  On error no output handle
 *     is written and nothing is leaked.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Calls that return a handle enqueue their GPU work on
 *     that stream and return without waiting unless stated; results are valid
 *     once the stream has synchronised.  Calls that copy to host memory
 *     synchronise the stream they use.
 *   - Memory: images and output pixel buffers belong to the caller (device
 *     memory unless the `host` flag says host memory).  Pools, matches and
 *     codes are library-owned opaque handles released with the matching
 *     *_free call (NULL is accepted and ignored).
 *   - Sizes: W and H must be multiples of the first range size B0 and at
 *     least 2 B0; B0 is 16, 8, 4 or 2 and each level halves it (Sec. 2).
 *   - Every step of the search runs in this library's CUDA kernels; there is
 *     no CPU fallback.  Without a usable sm_103a device fic_create fails with
 *     FIC_ECUDA or FIC_EUNSUPPORTED.
 */
#ifndef FIC_H
#define FIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FIC_VERSION 1

/* status codes */
#define FIC_OK 0
#define FIC_EINVAL (-1)       /* bad argument (size, level, params)          */
#define FIC_ENOMEM (-2)       /* device or host allocation failed            */
#define FIC_ECUDA (-3)        /* a CUDA call failed                          */
#define FIC_ETIMEOUT (-4)     /* a bounded device wait expired               */
#define FIC_EUNSUPPORTED (-5) /* device is not sm_103 or lacks a feature     */
#define FIC_ERANGE (-6)       /* output capacity too small                   */

/* contrast-scaling set (Sec. 2 grid search; Sec. 3.1 predefined values) */
#define FIC_S_PREDEFINED 0 /* 16:{0.1} 8:{0.2,0.4} 4:{0.3,0.8} 2:{0.5,0.9} */
#define FIC_S_GRID 1       /* s_k = k/(M-1), k = 0..M-1, 2 <= M <= 32      */
#define FIC_S_EXACT 2      /* Eq. 2's least-squares s of every (range,
                              domain, isometry), clamped to [0, 1] (a flat
                              domain takes s = 0): the exhaustive search the
                              paper derives its predefined values from
                              (Sec. 3.1).  The best map minimises Eq. 1 at its
                              own s, compared exactly; ties go to the lowest
                              dom_index * 8 + iso.  Tensor precision only
                              (FIC_EUNSUPPORTED with FIC_PREC_FP32).        */

/* arithmetic of the correlation <R, D> */
#define FIC_PREC_TENSOR 0 /* tcgen05 f16 MMA on exact small integers, exact
                             int64 scoring of every candidate that can win */
#define FIC_PREC_FP32 1   /* plain FP32 CUDA-core dot products and scoring */

typedef struct fic_ctx fic_ctx;
typedef struct fic_pool fic_pool;
typedef struct fic_matches fic_matches;
typedef struct fic_code fic_code;

typedef struct {
  int n_levels;              /* quadtree levels, 1..4 (Sec. 2)                 */
  int range_size0;           /* B at the first level: 16, 8, 4 or 2            */
  int domain_step;           /* L >= 1 (Sec. 2)                                */
  double rms_threshold;      /* accept a range when E <= n T^2, compared as
                                e <= n (T T) with e the map's double E below  */
  int single_level;          /* 1: one level, every range accepted             */
  int s_mode;                /* FIC_S_PREDEFINED, FIC_S_GRID or FIC_S_EXACT    */
  int grid_samples;          /* M for FIC_S_GRID                               */
  double entropy_percentile; /* threshold = pool entropy at this percentile    */
  int precision;             /* FIC_PREC_TENSOR or FIC_PREC_FP32               */
  int autotune;              /* 0: the default schedule (3 work items per
                                persistent CTA; on the tensor path two
                                epilogue warp groups per tile at B <= 8);
                                1: on a level's first eager run, time
                                the matcher with 2, 3, 4, 6 and 8 items per
                                CTA and, on the tensor path at B <= 8, one or
                                two epilogue groups per tile (8 or 16 ranges
                                per warp visit), each schedule the median of
                                5 launches, and keep the fastest for the
                                code's later encodes (results are unchanged;
                                fic_code_schedule reports the choice)        */
  int pool_size;             /* K > 0: the entropy filter keeps the K domains
                                of highest entropy (Tables 1-2's "pool size":
                                threshold = the (K+1)-th highest entropy, kept
                                when strictly above, ties dropped; K >= P keeps
                                the whole pool); 0: entropy_percentile         */
} fic_params;

typedef struct {
  const uint8_t* pixels; /* row-major 8-bit grey levels                        */
  int width, height;     /* W, H                                               */
  int pitch;             /* bytes between rows, >= width                       */
  int host;              /* 0: device pointer; 1: host pointer (the library
                            copies it to the device on the call's stream)     */
} fic_image;

/* One saved affine map (Sec. 2): range block, domain block, isometry, s, o. */
typedef struct {
  int32_t level, x, y, size; /* range: quadtree level, top-left, side B        */
  int32_t dom_index;         /* raster index of the domain in the unfiltered
                                pool ((y/L) * Px + x/L)                       */
  int32_t dom_x, dom_y;      /* domain top-left (a 2B x 2B square)            */
  int32_t iso;               /* 0..3: rotate 90k deg clockwise; 4..7: then
                                mirror left-right                             */
  int32_t s_idx, p, q;       /* s = p / q, s_idx its index in the level's set
                                (FIC_S_EXACT: s_idx = p = q = 0)              */
  int32_t reserved;
  int64_t e_num;             /* 16 q^2 n^2 E, exact integer (FIC_S_EXACT: 0)  */
  int64_t o_num;             /* 4 q n o, exact integer (FIC_S_EXACT: 0)       */
  double e;                  /* E of Eq. 1: e_num / (16 q^2 n^2); FIC_S_EXACT:
                                with the pair's integer moments
                                A = n sum r^2 - (sum r)^2, C = n <r, Ds> -
                                sum r sum Ds, V = n sum Ds^2 - (sum Ds)^2 (Ds
                                the 2x2 sums of the domain), in double in this
                                order: s = 0: A / n; s = 1: (16A - 8C + V) /
                                (16 n); otherwise (A - (C C) / V) / n          */
  double s;                  /* p / q; FIC_S_EXACT: 4C / V (or 0, 1)          */
  double o;                  /* o of Eq. 3: o_num / (4 q n); FIC_S_EXACT:
                                (4 d sum r - m sum Ds) / ((4 d) n) for
                                s = m / d, m = 4C, d = V (0/1, 1/1 clamped)    */
} fic_transform;

/* Per-range result of fic_match_level (same fields as fic_transform). */
typedef fic_transform fic_match;

typedef struct {
  int32_t size;        /* B                                                   */
  int32_t pool_size;   /* P = Px * Py                                         */
  int32_t n_kept;      /* domains left by the entropy filter                  */
  int32_t fallback;    /* 1 when "entropy > threshold" kept nothing and the
                          pool fell back to "entropy >= threshold"            */
  int64_t thr_key;     /* threshold as the fixed-point entropy key            */
  int32_t n_active;    /* ranges matched at this level                        */
  int32_t n_accepted;  /* ranges saved at this level                          */
  double matches;      /* n_active * n_kept * 8 range-domain-isometry triples */
} fic_level_stats;

typedef struct {
  int32_t size, step;  /* B, L                                                */
  int32_t px, py;      /* pool positions per row / column                     */
  int32_t pool_size;   /* P                                                   */
  int32_t n_kept;
  int32_t fallback;
  int32_t reserved;
  int64_t thr_key;
} fic_pool_info_t;

/* fields for fic_pool_copy */
#define FIC_POOL_KEYS 0   /* int64[P]: entropy key of every pool position,
                             sum over grey levels of round(q ln q 2^32)      */
#define FIC_POOL_KEPT 1   /* int32[n_kept]: kept raster indices, ascending   */
#define FIC_POOL_SUMS 2   /* int64[n_kept]: sum of the 2x2 sums Ds           */
#define FIC_POOL_SQSUMS 3 /* int64[n_kept]: sum of Ds^2                      */

/* Name of a status code (static string). */
const char* fic_status_string(int status);

/* FIC_VERSION of the loaded library. */
int fic_version(void);

/* Defaults: 4 levels from 16, L = 2, T = 8, predefined S, median, tensor. */
int fic_default_params(fic_params* out);

/* Create a context on CUDA device `device` (must be compute capability
 * 10.3).  Allocates per-context device state (the entropy-key table, status
 * words).  *ctx receives the handle. */
int fic_create(fic_ctx** ctx, int device);

/* Release the context and every cached plan; waits for the device. */
int fic_destroy(fic_ctx* ctx);

/* Sec. 2 + Sec. 3: entropy-filtered domain pool for ranges of size
 * `range_size` (2B x 2B squares at step params->domain_step, decimated to
 * B x B).  Computes each position's entropy key, the percentile threshold
 * (exact radix selection), the kept list (key < threshold; key <= threshold
 * when that keeps nothing) and the packed operand of the kept domains. */
int fic_build_domain_pool(fic_ctx* ctx, const fic_image* img, int range_size,
                          const fic_params* params, void* stream, fic_pool** out);

/* Counts and threshold of a pool (synchronises its stream). */
int fic_pool_info(const fic_pool* pool, fic_pool_info_t* out);

/* Copy one field (FIC_POOL_*) to host memory; `bytes` is the capacity of
 * host_dst and must hold the whole field.  Synchronises. */
int fic_pool_copy(const fic_pool* pool, int field, void* host_dst, size_t bytes);

void fic_pool_free(fic_pool* pool);

/* Sec. 2: best (domain, isometry, s) of Eq. 1 for each listed range of size
 * pool->size against the kept pool of the same image.  range_xy: 2 * n_ranges
 * int32 (x, y) top-left corners in host memory; every block must lie inside
 * the image (FIC_EINVAL otherwise).  Ties are broken by the lowest
 * (dom_index * 8 + iso) * |S| + s_idx.  params->precision selects the path. */
int fic_match_level(fic_ctx* ctx, const fic_image* img, const fic_pool* pool,
                    const int32_t* range_xy, int n_ranges, const fic_params* params,
                    void* stream, fic_matches** out);

/* Copy the per-range results to host (synchronises).  *count = n_ranges. */
int fic_matches_copy(const fic_matches* m, fic_match* host_out, size_t cap, size_t* count);

void fic_matches_free(fic_matches* m);

/* Full quadtree encoder over n_images images (Sec. 2): per level, the
 * entropy-filtered pool, the matching of every active range and the split of
 * the ranges whose error is above the threshold.  Runs entirely on the GPU
 * with device-side counts; the returned handle holds the codes on the
 * device. */
int fic_encode(fic_ctx* ctx, const fic_image* imgs, int n_images, const fic_params* params,
               void* stream, fic_code** out);

/* fic_encode into an existing handle: the images must have the sizes (and
 * the host flag) and params must equal those `code` was created with; the
 * previous codes are overwritten and no device memory is allocated (the
 * handle's buffers are reused).  Returns FIC_EINVAL otherwise.  With a
 * non-NULL stream the first such call captures the device part of the
 * encode into a CUDA graph held by `code`, and every call (that one
 * included) launches the graph on `stream` after staging host images; the
 * call returns without waiting for the encode (a copy from pageable host
 * memory may block until the driver has staged it).  With a NULL stream the
 * encode is enqueued kernel by kernel. */
int fic_encode_again(fic_ctx* ctx, const fic_image* imgs, int n_images, const fic_params* params,
                     void* stream, fic_code* code);

/* Number of codes of image `image_idx`.  The first query after an encode
 * waits for the encode's stream and reads back, in one copy, the code
 * offsets of every image and level together with the encode's status
 * (FIC_ETIMEOUT / FIC_ERANGE are reported here); later queries use them. */
int fic_code_count(const fic_code* code, int image_idx, size_t* count);

/* Copy the codes of one image to host, level-major then in range order:
 * one asynchronous copy per level on the encode's stream and one wait
 * (page-locked host_out is written by DMA directly).  Fails with FIC_ERANGE
 * when cap is too small. */
int fic_code_get(const fic_code* code, int image_idx, fic_transform* host_out, size_t cap,
                 size_t* count);

/* Per-level statistics of one image (n_levels entries; synchronises). */
int fic_code_stats(const fic_code* code, int image_idx, fic_level_stats* host_out, int cap);

/* Stored form of the maps.  The paper reports compression ratios (Tables
 * 1-2, "Com. rat") but states no bit layout; the layout here is a reading:
 *   - o is stored with o_bits bits (1..16), uniform over [-255, 255]:
 *     step = 510 / (2^o_bits - 1), o' = rint((o + 255) / step) * step - 255
 *     (round half to even, clamped to the end points);
 *   - every range of a level above the last costs one quadtree bit, and
 *     every saved map ceil(log2 P) bits of domain position (P = the level's
 *     pool positions), 3 bits of isometry, ceil(log2 |S|) bits of s and
 *     o_bits bits of o.
 * fic_code_quantize_o replaces o by o' in every saved map of every image
 * (asynchronous on the code's last stream; later decodes use o').  e, e_num
 * and o_num keep the unquantised map's values.  fic_code_bits writes the
 * total bits of one image's stored form to *bits (synchronises); the
 * compression ratio is 8 W H / bits.  FIC_EINVAL for o_bits outside 1..16,
 * and from fic_code_bits for FIC_S_EXACT codes (s is not from a finite set). */
int fic_code_quantize_o(fic_code* code, int o_bits);
int fic_code_bits(const fic_code* code, int image_idx, int o_bits, int64_t* bits);

void fic_code_free(fic_code* code);

/* Timing hooks (CUDA events recorded on the encode's stream, also inside a
 * replayed graph).  After fic_code_set_profiling(code, 1), each later
 * encode into `code` records, per level, the matcher kernel and the whole
 * level; fic_code_profile synchronises the stream and writes 2 floats per
 * level, {matcher ms, level ms}, to `ms` (cap >= 2 * n_levels).  Switching
 * profiling on or off discards a captured graph. */
int fic_code_set_profiling(fic_code* code, int on);
int fic_code_profile(const fic_code* code, float* ms, int cap);
/* With profiling on: per level, the ms of the level's pool build (Sec. 3:
 * entropy keys, threshold, kept list, packed operand), timed on the side
 * stream it runs on (cap >= n_levels floats; synchronises). */
int fic_code_pool_profile(const fic_code* code, float* ms, int cap);

/* The matcher schedule of every level of `code` (the default, or the
 * autotuner's choice once a level has been tuned): 2 ints per level, {work
 * items per persistent CTA, epilogue warp groups per tile}; cap >= 2 *
 * n_levels. */
int fic_code_schedule(const fic_code* code, int32_t* out, int cap);

/* Kernels in the graph that fic_encode_again replays (captured on its first
 * call with a non-NULL stream); -1 before that. */
int fic_code_graph_kernels(const fic_code* code, int64_t* n_kernels);

/* Decoder: fixed-point iteration of the saved maps from a flat 128 image, all
 * ranges updated from the previous iterate (Jacobi) in FP64, clamped to
 * [0, 255], until max |delta| < tol or max_iters; then rounded half to even.
 * out: W x H bytes at out_pitch, device memory (out_host = 0) or host memory
 * (out_host = 1).  *iters_done receives the iteration count (may be NULL).
 * Synchronises. */
int fic_decode(fic_ctx* ctx, const fic_code* code, int image_idx, int max_iters, double tol,
               uint8_t* out, int out_pitch, int out_host, void* stream, int* iters_done);

/* Test hook for the bounded device waits (the paper has no counterpart).
 * Arms one fault for the next tensor-path matcher launch made through this
 * context (fic_encode, fic_encode_again without graph replay, or
 * fic_match_level); the launch disarms it.  0 disarms it without a launch.
 *
 *   FIC_FAULT_DROP_TILE_COPY  the copy engine is never asked for the first
 *       domain tile of the first work item of CTA 0, so that tile's stage
 *       never fills.  The waits on it give up after their limit (2 s), the
 *       CTA abandons its remaining work, waits (also bounded) for the copies
 *       it did issue, releases its tensor memory and returns; the call's
 *       status becomes FIC_ETIMEOUT (reported by the handle's next
 *       synchronising call), and the handle's results are not valid.  The
 *       GPU is not faulted: the context and the handle stay usable, and the
 *       next encode into the same handle starts from a clear status.
 *
 * Returns FIC_EINVAL for an unknown fault. */
#define FIC_FAULT_NONE 0
#define FIC_FAULT_DROP_TILE_COPY 1
int fic_debug_inject(fic_ctx* ctx, int fault);

/* Decoder that allocates no device memory.  The paper has no counterpart:
 * this is a deployment variant of fic_decode for callers that must not let a
 * library call cudaMalloc -- processes whose device memory belongs to another
 * allocator (a framework's caching allocator, a pool sized at start-up) and
 * loops where an allocation's device synchronisation is not acceptable.
 *
 * It runs fic_decode's kernels (same iteration, same result) on a workspace
 * that is a static __device__ array inside this library, sized for at most
 * FIC_DECODE_STATIC_MAX_PIXELS pixels (width * height) and
 * FIC_DECODE_STATIC_MAX_ITERS iterations: about 20 MiB that every GPU which
 * loads the library holds until the process exits.
 *
 *   codes      n_codes maps in DEVICE memory, caller-owned (for example the
 *              output of fic_code_get copied to the device); every block must
 *              lie inside the image, sizes 2/4/8/16, iso 0..7, 0 <= s <= 1
 *              (FIC_EINVAL otherwise, checked on the device before decoding)
 *   out        width x height bytes at out_pitch, DEVICE memory, caller-owned
 *   iters_done iterations run (may be NULL)
 *
 * Returns FIC_EINVAL for sizes or iteration counts above the maximum.  The
 * first call on a device looks up the array's device address (and loads the
 * library's device code if that has not happened yet), so make it before any
 * stream capture.  Every call uses the same array and leaves its contents
 * behind; the call resets what must start from zero.  Calls whose GPU work
 * overlaps (on different streams or threads) race on the array: serialise
 * them.  Enqueues on `stream` and synchronises it before returning. */
#define FIC_DECODE_STATIC_MAX_PIXELS (1024 * 1024)
#define FIC_DECODE_STATIC_MAX_ITERS 1024
int fic_decode_static(const fic_transform* codes, int64_t n_codes, int width, int height,
                      int max_iters, double tol, uint8_t* out, int out_pitch, void* stream,
                      int* iters_done);

#ifdef __cplusplus
}
#endif
#endif
