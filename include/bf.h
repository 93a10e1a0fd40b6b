/*
 * bf.h -- C ABI of the GB300 joint-acceleration bilateral filter.
 *
 * Method: Dai, Yuan, Zhang, "Speeding up the Bilateral Filter: A Joint
 * Acceleration Way".  The bilateral filter of Eq. (1),
 *
 *   I^(x) = sum_y K_s(x - y) K_r(I(x) - I(y)) I(y) / sum_y K_s(x - y) K_r(I(x) - I(y)),
 *
 * is evaluated with both kernels truncated (Sec. IV-A), the spatial kernel
 * replaced by its best N-term 2-D Haar expansion, which is a signed sum of
 * boxes (Eqs. (30)-(32), App. A), and the range kernel by its best N-term
 * cosine series (Eq. (33)).  The cosine difference identity (Eq. (34)) turns
 * the range term into per-term basis images cos(w_k I), sin(w_k I) and their
 * products with I; every basis image is box-filtered and the results are
 * weighted by cos/sin(w_k I(x)) and summed into numerator and denominator
 * (Eq. (36)) before the final divide.  The paper's own 3-D form (period
 * P = T_r, the range box applied over intensity slices by dimension
 * promotion, Eqs. (2), (28)-(29), (35)-(36)) is the BF_RANGE_PAPER_3D policy.
 *
 * Conventions for every entry point:
 *   - Status codes only; nothing throws or aborts across this boundary.  A
 *     human-readable detail for the last failing call on the calling thread
 *     is available from bf_last_error().
 *   - Images are single-channel float32, row-major, with a row pitch in
 *     bytes (a multiple of 4, >= width * 4).  Input values are expected in
 *     [i_lo, i_hi] of the plan (default [0, 1]); values outside are filtered
 *     but the accuracy statements of the plan no longer hold
 *     (bf_debug_range_checks makes bf_filter reject them instead).
 *   - Device pointers are CUDA device memory on the plan's device; the
 *     caller owns them.  "stream" is a cudaStream_t (NULL = legacy default
 *     stream).  Filtering calls are asynchronous with respect to the host.
 *   - In-place filtering (input and output overlapping) is rejected with
 *     BF_ERR_INVALID_ARG: neighbours would be read after being overwritten.
 *   - Plans are immutable after creation and may be shared across threads
 *     and streams.
 */
#ifndef BF_H
#define BF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BF_OK = 0,
    BF_ERR_INVALID_ARG = 1,     /* bad pointer, size, pitch or parameter */
    BF_ERR_UNSUPPORTED = 2,     /* valid request the library does not implement */
    BF_ERR_OOM = 3,             /* host or device allocation failed */
    BF_ERR_CUDA = 4,            /* a CUDA runtime call failed (detail in bf_last_error) */
    BF_ERR_ADMISSION = 5,       /* server: request can never fit the memory budget */
    BF_ERR_TIMEOUT = 6,         /* server: poll timed out; the request is still in flight */
    BF_ERR_DEVICE_TIMEOUT = 7,  /* a bounded device-side wait gave up */
    BF_ERR_RANGE = 8,           /* value outside the supported range */
    BF_ERR_NO_DEVICE = 9,       /* no usable CUDA device */
    BF_ERR_NOT_FOUND = 10,      /* server: unknown or already collected ticket */
    BF_ERR_CANCELLED = 11,      /* server: request cancelled before it ran */
    BF_ERR_SCRATCH = 12         /* bf_filter_noalloc: no launch geometry's scratch fits its fixed array */
} bf_status;

typedef enum {
    BF_KERNEL_GAUSSIAN = 0,     /* exp(-t^2 / (2 sigma^2)); spatial: exp(-|d|_2^2 / (2 sigma^2)) */
    BF_KERNEL_EXPONENTIAL = 1,  /* exp(-|t| / sigma); spatial: exp(-|d|_2 / sigma), radial and
                                   not separable (R <= 255) */
    BF_KERNEL_BOX = 2           /* 1 on [-sigma, sigma] (range) or on the whole window (spatial) */
} bf_kernel;

typedef enum {
    /* Cosine series on [-P, P] with P = max(T_r, (dI + T_r) / 2), dI = i_hi - i_lo:
     * the kernel truncated at T_r is fitted and no periodic copy reaches an
     * intensity difference inside the data range, so the range box of
     * Eq. (33) is identically one (the "extended truncation region" of
     * Sec. V-C, Case 1).  Default. */
    BF_RANGE_TRUNCATED_MIN_PERIOD = 0,
    /* P = dI and the kernel is fitted untruncated on [-dI, dI]. */
    BF_RANGE_UNTRUNCATED_FULL = 1,
    /* The 3-D form of Sec. IV-D: P = T_r (the kernel truncated at T_r is
     * fitted on one period) and the range box [I(x) - T_r, I(x) + T_r] is
     * applied by dimension promotion (Eq. (2)) over Z intensity slices
     * (z_bins): the data range is sampled at Z levels i_lo + n dI / (Z - 1),
     * a pixel lies in the slice of its nearest level (n = rint((I - i_lo) s)
     * in fp32, s = fl32((Z - 1) / dI), clamped to [0, Z - 1]), and neighbour
     * y counts for centre x iff |n(y) - n(x)| <= R_z = floor(T_r (Z - 1) /
     * dI).  Eqs. (35)-(36): the window sums are 3-D boxes, box over space
     * times the slice window along z.  The basis images use I(y) itself
     * (for data on the Z levels, e.g. 8-bit images with Z = 256, the window
     * is exactly the range box).  Cost: every tile is filtered once per
     * distinct slice among its output pixels. */
    BF_RANGE_PAPER_3D = 2
} bf_range_policy;

/* The series that approximates the range kernel. */
typedef enum {
    /* The truncated cosine series of Eqs. (13)-(15), best N_r terms (Eq. (33)).  Default. */
    BF_SERIES_COSINE = 0,
    /* BF_RANGE_PAPER_3D only: the best N_r-term Haar expansion (Eqs. (17)-(20), selection by Eq. (11))
     * of the truncated range kernel on the slice axis, in slice units: domain [-T_z, T_z], T_z = R_z + 1/2,
     * J_z = ceil(log2(2 T_z)) levels, profile K_r(t dI / (Z - 1)).  Each Haar term is a pair of boxes
     * along z, so the filter is a sum of 3-D boxes with no cosine basis: a neighbour's weight is
     * K~_s(x - y) K~_r(n(x) - n(y)), K~_r read from a table of the 2 R_z + 1 slice offsets.  R_z <= 1023.
     * The paper uses Haar functions for the spatial kernel only; this applies them to the range kernel. */
    BF_SERIES_HAAR = 1
} bf_range_series;

/* Storage precision of the basis inputs.  The fused filter computes every
 * running sum, the weighting and the divide in fp32 (Kahan-compensated
 * horizontal sums), whatever the precision.  BF_PREC_FP32: the basis is
 * computed in the kernel from each pixel at every window edge (or read from an
 * fp32 pre-pass of the same values, a geometry the autotuners may time).
 * BF_PREC_FP16 / BF_PREC_BF16: a pre-pass stores each pixel's base rotation
 * (cos, sin)(pi t) as one fp16 / bf16 pair beside the fp32 pixel, and the
 * kernel reads it at every edge, rescaled to unit length; term k of a group is
 * reached from an fp32 anchor by m_k <= min(k, NK) rotations, so with unit
 * roundoff u (2^-11 fp16, 2^-8 bf16) |delta I^| <= 2 u sum_k m_k |a_k| mass
 * (1 + |I^|) / |den| beyond the fp32 path's error (mass = sum |K~_s| over the
 * window).  16-bit plans take the collapsed range policies (not
 * BF_RANGE_PAPER_3D); bf_filter_batch and the server run them as direct
 * launches beside the persistent ones.
 * The pre-computation cache of bf_precompute has its own storage precision
 * (same enum): its window sums may be stored as fp16 or bf16, rounded once
 * from the fp32 sums, with |delta I^| <= 2 u sum|a_k| mass (1 + |I^|) / |den|. */
typedef enum {
    BF_PREC_FP32 = 0,  /* fp32 */
    BF_PREC_BF16 = 1,  /* bf16 storage of the base rotation (plans) or of the cached sums (bf_precompute) */
    BF_PREC_FP16 = 2   /* fp16 storage of the base rotation (plans) or of the cached sums (bf_precompute) */
} bf_precision;

/* Plan parameters (Sec. IV-A..C).  Fill with bf_plan_desc_default() first. */
typedef struct {
    int spatial;        /* bf_kernel: GAUSSIAN, BOX (separable on the square window) or
                           EXPONENTIAL (radial, not separable) */
    double sigma_s;     /* spatial bandwidth, pixels, > 0 */
    int radius;         /* window half-width R (square |y - x|_inf <= R); 0 -> round(3 sigma_s) */
    int ns_terms;       /* N_s: Haar terms kept (best N-term), >= 1 */
    int range;          /* bf_kernel */
    double sigma_r;     /* range bandwidth in intensity units, > 0 */
    double t_r;         /* range truncation T_r; 0 -> 3 sigma_r (Gaussian), sigma_r ln 100
                           (exponential, eps = 0.01 of Sec. IV-A), sigma_r (box) */
    int nr_terms;       /* N_r: cosine terms kept (best N-term over the first 20 N_r), >= 1 */
    int policy;         /* bf_range_policy */
    float i_lo, i_hi;   /* data range of the images; default 0, 1 */
    int precision;      /* bf_precision */
    int kahan;          /* 1 (default): horizontal sliding window sums are Kahan-compensated
                           (per 8-column block); 0: plain fp32 sliding sums.  Vertical
                           running sums restart at every tile (at most a tile height of rows). */
    int device;         /* CUDA device ordinal; -1: host-only plan (bf_coeffs works,
                           filtering returns BF_ERR_NO_DEVICE) */
    int z_bins;         /* BF_RANGE_PAPER_3D: intensity slices Z in [2, 4096]; 0 -> 256 (the
                           8-bit case of Sec. II-B).  Ignored by the other policies. */
    int range_series;   /* bf_range_series; BF_SERIES_HAAR needs BF_RANGE_PAPER_3D.  nr_terms counts
                           the kept terms of whichever series */
} bf_plan_desc;

typedef struct bf_plan bf_plan;

/* Fills *desc with defaults: Gaussian/Gaussian, sigma_s = 4, R = 0 (auto),
 * N_s = 5 (the paper's three-box setting, Sec. V-C), sigma_r = 0.1, N_r = 8,
 * truncated-min-period policy, data range [0, 1], fp32, Kahan on, device 0,
 * z_bins = 0 (256). */
void bf_plan_desc_default(bf_plan_desc *desc);

/* Builds a plan (Sec. IV-A..C; App. B): truncation points, range cosine
 * coefficients a_k on [-P, P] (Eqs. (14)-(15)), 2-D Haar coefficients of the
 * truncated spatial kernel (Eqs. (21)-(22): products of 1-D coefficients for
 * the separable kernels; for the radial exponential kernel each 2-D integral
 * over the Haar cells is computed whole, by tensor Gauss-Legendre quadrature
 * with the cells at its cone point graded toward the origin), best N-term
 * selection by |coefficient|,
 * and the signed-box representation of the selected Haar terms (App. A),
 * compiled into nested horizontal and vertical box windows for the kernel.
 * Host memory only; the coefficient tables travel to the device as kernel
 * parameters.  *out receives a plan the caller releases with bf_plan_destroy.
 * Errors: BF_ERR_INVALID_ARG (NULL, sigma <= 0, N < 1, i_hi <= i_lo, bad enum,
 * z_bins outside [2, 4096] for BF_RANGE_PAPER_3D, BF_SERIES_HAAR without it),
 * BF_ERR_UNSUPPORTED (exponential spatial kernel with R > 255; a selection
 * needing more than 6 box windows per axis; 16-bit precision with
 * BF_RANGE_PAPER_3D; BF_SERIES_HAAR with R_z > 1023),
 * BF_ERR_OOM, BF_ERR_NO_DEVICE (device >= 0 that does not exist). */
bf_status bf_plan_create(const bf_plan_desc *desc, bf_plan **out);

/* Releases a plan (NULL is a no-op).  No filtering call using the plan may be
 * in flight on any stream. */
void bf_plan_destroy(bf_plan *plan);

/* Host view of a plan's coefficients (App. A/B); all pointers point into the
 * plan and stay valid until bf_plan_destroy. */
typedef struct {
    int radius;                 /* R */
    double t_s;                 /* Haar interval half-width T_s = R + 1/2 */
    int haar_levels;            /* J = ceil(log2(2 T_s)) */
    double t_r;                 /* range truncation point used */
    double period;              /* cosine half-period P */
    int nr;                     /* selected range terms */
    const int *k;               /* [nr] cosine indices, ascending */
    const double *a;            /* [nr] a_k */
    int ns;                     /* selected Haar terms, in ranking order */
    const int *haar_terms;      /* [4 ns] level_x, k_x, level_y, k_y (level -1 = phi) */
    const double *haar_coef;    /* [ns] c */
    int tie_split;              /* 1 if N_s cut a group of equal |c| (asymmetric kernel) */
    const double *kernel;       /* [(2R+1)^2] K~_s(dx, dy) at [(dy+R)(2R+1) + dx+R] */
    int n_vwin, n_hwin;         /* box windows of the kernel compilation */
    const int *vwin;            /* [2 n_vwin] first/last neighbour row offset */
    const int *hwin;            /* [2 n_hwin] first/last neighbour column offset */
    const double *wcoef;        /* [n_vwin * n_hwin] weight of window pair (v, h) */
    double range_max_err;       /* max |K_r - K~_r| over [-dI, dI] (sampled); BF_RANGE_PAPER_3D:
                                   over [-T_r, T_r], where the range box keeps the series */
    double spatial_max_err;     /* max |K_s - K~_s| over the integer window */
    double den_eps;             /* denominator guard: den <= den_eps -> output I(x) */
    int passes;                 /* term groups at the largest group size (ceil(nr / 16)) */
    int z_bins;                 /* BF_RANGE_PAPER_3D: slices Z; 0 for the other policies */
    int z_radius;               /* BF_RANGE_PAPER_3D: slice window half-width R_z; 0 otherwise */
    int range_series;           /* bf_range_series.  For BF_SERIES_HAAR, k / a above hold the one
                                   constant cosine term the kernel runs (k = 0, a = 1) and: */
    int n_range_haar;           /* kept range Haar terms (0 for the cosine series) */
    const int *range_haar;      /* [2 n_range_haar] level, k (level -1 = phi), in ranking order */
    const double *range_haar_coef;  /* [n_range_haar] c */
    const double *z_weights;    /* [2 z_radius + 1]: K~_r at slice offset d = n(x) - n(y), at [d + z_radius]
                                   (BF_SERIES_HAAR); NULL otherwise */
} bf_coeff_view;

/* Fills *out with the plan's coefficients.  Errors: BF_ERR_INVALID_ARG. */
bf_status bf_coeffs(const bf_plan *plan, bf_coeff_view *out);

/* Filters one image on the device (hot path, Eq. (36) then divide).
 * d_in / d_out: device buffers of height rows with the given pitches (bytes, multiples of 4, at least
 * width * 4 and below 4 GiB).  height, width >= 0 (0 is a no-op).  Asynchronous on `stream`.
 * Errors: BF_ERR_INVALID_ARG (NULL, pitch, overlap), BF_ERR_NO_DEVICE
 * (host-only plan), BF_ERR_CUDA (launch failure), BF_ERR_OOM (scratch for
 * multi-pass plans could not be allocated). */
bf_status bf_filter(const bf_plan *plan, const float *d_in, size_t in_pitch_bytes,
                    float *d_out, size_t out_pitch_bytes, int height, int width, void *stream);

/* bf_filter without any device allocation, for callers that cannot allocate
 * device memory while filtering: hosts that reserve all their device memory up
 * front (a framework's caching allocator owning the GPU, a real-time loop where
 * an allocation may synchronise or fail mid-frame).  The paper has no
 * counterpart; this is a deployment variant of the same computation.
 * Plans whose cosine terms are split into groups need partial numerator and
 * denominator planes (2 x groups x height x width floats), and the 3-D form a
 * slice work list; here they live in a fixed 64 MiB array inside the library
 * (16,777,216 floats), which every GPU that loads the library holds until the
 * process exits.  The launch geometry is bf_filter's, else the best-ranked one
 * whose scratch fits the array.  The array's address is looked up once per
 * CUDA context by the first call that needs it; make that first call before
 * any stream capture.  All calls share the array and it keeps the last call's
 * contents: calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it, so order them on one stream or with events, and
 * consume each result before a later call runs.  Arguments, layout, ownership
 * and results as bf_filter; with the debug range check on, it checks the input
 * as bf_filter does.  Errors: as bf_filter (never BF_ERR_OOM), plus
 * BF_ERR_SCRATCH when no launch geometry's scratch fits the array. */
bf_status bf_filter_noalloc(const bf_plan *plan, const float *d_in, size_t in_pitch_bytes,
                            float *d_out, size_t out_pitch_bytes, int height, int width, void *stream);

/* Filters one image in host memory with each of n plans (1..256, all on one
 * device): the paper's use of one image under several parameter settings
 * (Sec. V-C).  Uploads h_in (height rows of width floats, row pitch in_pitch
 * bytes; pinned memory makes the copies asynchronous), filters it with plan i
 * on internal stream i mod n_streams (1..16), forked from and joined back to
 * `stream`, and downloads result i into h_outs[i] (row pitch out_pitch bytes)
 * on an internal copy stream as soon as its filter ends.  Asynchronous on
 * `stream`: synchronize it before reading h_outs.  The device buffers (input,
 * n outputs, each plan's scratch) are two blocks per device owned by the
 * library, used by alternate calls, allocated by the first calls and grown
 * when a call needs more.  A call's upload waits for the last download of the
 * call two before it on the device (the previous user of its block), so calls
 * from several streams or threads are safe, and a call issued on another
 * stream than the one before it uploads its image while that call still
 * filters (double buffering); calls on one stream run one after another.  A
 * call that allocates or grows a block synchronizes with that block's previous
 * call: make the first two calls (at the largest size and plan count) outside
 * stream capture.  Plans' geometries as bf_filter's; the debug input-range
 * check does not apply.  Errors:
 * BF_ERR_INVALID_ARG (NULL, n or n_streams out of range, bad pitch, overlap,
 * plans on several devices), BF_ERR_NO_DEVICE, BF_ERR_OOM, BF_ERR_CUDA. */
bf_status bf_filter_host(const bf_plan *const *plans, int n, const float *h_in, size_t in_pitch,
                         float *const *h_outs, size_t out_pitch, int height, int width, int n_streams,
                         void *stream);

/* Launch geometry bf_filter would use for this plan on a height x width image:
 * info[0] tile width, [1] tile height, [2] threads per CTA, [3] cosine terms per
 * CTA, [4] term groups, [5] kernel launches (pre-pass, filter, finalize), [6] shared memory
 * bytes per CTA, [7] scratch KiB, [8] 1 when the basis inputs are kept in a
 * shared-memory ring per column, [9] exchange buffer depth, [10] columns per
 * CTA (tile width plus the halo of 2 x horizontal reach, in whole warps), [11]
 * kernel family: 1 packed (cosine terms in consecutive pairs on the two-wide
 * fp32 instructions; a gapped selection is covered by groups of consecutive
 * frequencies with zero weights), 0 scalar (any set of terms; offered only for
 * gapped selections), 2 hybrid (gapped selections: windows of consecutive
 * frequencies in the packed family, the one from the lowest selected
 * frequency and every later window whose frequencies are all selected, the
 * other terms in the scalar family, in one launch into the partial planes),
 * [12] basis inputs: 0 computed in the kernel, 1 / 2 / 3
 * read from a pre-pass buffer in fp32 / fp16 / bf16 (its 16 or 8 bytes per
 * pixel are part of the scratch).  info must hold 13 ints.  Host only; needs no
 * device for host-only plans (uses 152 SMs as the device size then).
 * Errors: BF_ERR_INVALID_ARG. */
bf_status bf_launch_info(const bf_plan *plan, int height, int width, int *info);

/* Autotuner: times candidate launch geometries (the cost model's best four of
 * each family -- ring of basis inputs or not, exchange depth, kernel family,
 * cosine terms per CTA, basis pre-pass -- within each residency class of 1, 2, or 3 and more
 * CTAs per SM by shared memory) for this plan on a synthetic height x width
 * image and remembers the fastest for later bf_filter / bf_filter_batch calls
 * with the same kernel class, reach and image size on this device.  Allocates
 * and frees its own device buffers and synchronizes `stream`; do not call it
 * during stream capture.  info (13 ints, may be NULL) receives the chosen
 * geometry as in bf_launch_info.  BF_TUNE_CACHE=<file> persists results.
 * Errors: BF_ERR_INVALID_ARG, BF_ERR_NO_DEVICE, BF_ERR_OOM, BF_ERR_CUDA. */
bf_status bf_autotune(const bf_plan *plan, int height, int width, void *stream, int *info);

/* As bf_autotune, but the candidates are timed on the caller's image: d_in
 * (device, height x width fp32, row pitch in_pitch bytes, a multiple of 4 and
 * at least width x 4; read only, caller-owned).  For the 3-D form the work is
 * one tile pass per intensity slice present in a tile, so the fastest
 * geometry depends on the content; a representative image finds it where the
 * synthetic one may not.  Errors: as bf_autotune, and BF_ERR_INVALID_ARG for
 * a NULL image or a bad pitch. */
bf_status bf_autotune_image(const bf_plan *plan, const float *d_in, size_t in_pitch, int height, int width,
                            void *stream, int *info);

/* Autotuner for plans that filter at the same time: n plans (1..256, all on
 * one device) run as a caller runs them concurrently, plan i on stream
 * i mod n_streams (1..16) in the given order, forked from and joined to one
 * stream.  The fastest launch geometries for that whole group are found by
 * coordinate descent (one kernel class at a time over the candidates
 * bf_autotune times, two sweeps, then every tile height of each class's chosen
 * width and family), timed with CUDA events from the fork to the
 * join on synthetic height x width images in the first plan's data range, and
 * pinned as bf_set_launch does.  Plans with the same kernel class, reach and
 * image size share one geometry.  A geometry that is slower alone can win in
 * the group: a grid of fewer CTAs than SMs leaves SMs to the other streams.
 * Allocates its own buffers (one input, n outputs, scratch) and streams, and
 * synchronizes them before returning; do not call it during stream capture.
 * infos (13 x n ints, may be NULL) receives each plan's geometry as in
 * bf_launch_info.  The geometry changes rounding order only.
 * Errors: BF_ERR_INVALID_ARG (no plans, a null plan, plans on several
 * devices, n_streams out of range), BF_ERR_NO_DEVICE (a host-only plan),
 * BF_ERR_UNSUPPORTED, BF_ERR_OOM, BF_ERR_CUDA. */
bf_status bf_autotune_group(const bf_plan *const *plans, int n, int height, int width, int n_streams, int *infos);

/* Launch geometries of this plan for a height x width image, best first by the
 * cost model: up to max_n records of 13 ints each (as in bf_launch_info) into
 * infos (caller-owned, 13 x max_n ints); *n_out receives how many were written.
 * Host only.
 * Errors: BF_ERR_INVALID_ARG. */
bf_status bf_launch_candidates(const bf_plan *plan, int height, int width, int max_n, int *infos, int *n_out);

/* Pins the launch geometry bf_filter / bf_filter_noalloc use for this plan's
 * kernel class on height x width images of the plan's device (as bf_autotune
 * does with the fastest one).  info (13 ints, caller-owned) must match one
 * record of bf_launch_candidates in fields 0, 1, 3, 8, 9, 10, 11 and 12; the other
 * fields are ignored.  The geometry changes rounding order only: every one gives
 * the result within the same error bound.  BF_TUNE_CACHE=<file> persists it.
 * Errors: BF_ERR_INVALID_ARG (no such geometry), BF_ERR_NO_DEVICE. */
bf_status bf_set_launch(const bf_plan *plan, int height, int width, const int *info);

/* ---------------------------------------------------------------------- */
/* Pre-computation for later range parameters (Sec. V-C, Case 1)            */
/* ---------------------------------------------------------------------- */

/* When the image is known before the range parameters, the box sums of the
 * basis images can be computed once.  They depend only on the cosine
 * half-period P, the intensity origin and the spatial kernel, not on the
 * range weights a_k: a fixed truncation t_r (bf_plan_desc.t_r > 0) or the
 * BF_RANGE_UNTRUNCATED_FULL policy gives plans for different sigma_r the same
 * P (the paper's predefined T_ri).  The cache holds, per pixel and for every
 * frequency k < kmax, the four window sums of cos(pi k t) I, sin(pi k t) I,
 * cos(pi k t), sin(pi k t): 16 x kmax bytes per pixel, allocated by the
 * library on the plan's device (kmax rounded up to whole term groups). */
typedef struct bf_cache bf_cache;

/* Runs the fused kernel over the frequencies 0 .. kmax-1 of `plan` on the
 * height x width image d_in (row pitch in bytes) and returns the cache in
 * *out (release with bf_cache_destroy).  2 <= kmax <= 128.  `precision`
 * (bf_precision) is the storage of the sums: fp32 (16 x kmax bytes per pixel),
 * or fp16 / bf16 (8 x kmax bytes per pixel, error bound above).  Asynchronous on
 * `stream` after the allocation; *out is NULL on any error.  Errors: BF_ERR_INVALID_ARG, BF_ERR_NO_DEVICE,
 * BF_ERR_OOM, BF_ERR_UNSUPPORTED, BF_ERR_CUDA. */
bf_status bf_precompute(const bf_plan *plan, const float *d_in, size_t in_pitch_bytes, int height, int width,
                        int kmax, int precision, void *stream, bf_cache **out);

/* Filters with `plan` from the cache: Eq. (36)'s weighting of the cached sums
 * by a_k cos/sin(pi k I(x) / P) and the divide; no box filtering.  d_in must
 * be the image the cache was computed from (I(x) is read from it); d_out is a
 * separate height x width buffer.  The plan must share the cache's P,
 * intensity origin and spatial kernel (BF_ERR_INVALID_ARG otherwise), and
 * select only frequencies below the cache's (BF_ERR_RANGE otherwise).
 * Asynchronous on `stream`; order it after bf_precompute. */
bf_status bf_filter_cached(const bf_cache *cache, const bf_plan *plan, const float *d_in, size_t in_pitch_bytes,
                           float *d_out, size_t out_pitch_bytes, void *stream);

/* Device bytes held by a cache. */
size_t bf_cache_bytes(const bf_cache *cache);

/* Releases a cache (NULL is a no-op); no work using it may be in flight. */
void bf_cache_destroy(bf_cache *cache);

/* One image of a batch. */
typedef struct {
    const float *d_in;
    size_t in_pitch_bytes;
    float *d_out;
    size_t out_pitch_bytes;
    int height, width;
} bf_image;

/* Filters n images, image i with plans[i] (plans may differ per image), in
 * one persistent launch per kernel class that walks a work list of
 * (image, tile) items across uneven images; images whose plans that kernel
 * does not run (the 3-D form, 16-bit basis storage) follow as one launch
 * sequence each, in their bf_filter geometry, side by side on up to eight
 * library streams forked from and joined back to `stream`.  The whole sequence is captured
 * once into a CUDA graph per batch shape and replayed.  Each image's result
 * equals bf_filter's for the same plan within fp32 rounding.  All plans must
 * be on the same device.  Errors: as bf_filter. */
bf_status bf_filter_batch(const bf_plan *const *plans, const bf_image *images, int n, void *stream);

/* Autotuner of the batched launch: runs this batch (the same arguments as
 * bf_filter_batch) under candidate geometries of each kernel class -- column
 * threads beyond the widest halo (64..384), minimum tile height (24..192) and
 * terms per CTA (as many as fit, at most 4, at most 2) -- by coordinate descent
 * (one class and one parameter at a time, two sweeps), timing the whole batch
 * with CUDA events on `stream`.  The fastest geometry of each class is kept
 * per (device, windows per axis, kernel family, widest reach) for later
 * bf_filter_batch calls and the server, and the captured graphs of the device
 * are dropped so the next call captures it.  The outputs receive valid results
 * (every geometry gives them within the same error bound).  Synchronizes
 * `stream`; do not call it during stream capture.  Errors: as
 * bf_filter_batch. */
bf_status bf_autotune_batch(const bf_plan *const *plans, const bf_image *images, int n, void *stream);

/* Exact bilateral filter of Eq. (1) by brute force on the device (fp32,
 * |y - x|_inf <= radius, untruncated range kernel): the accuracy reference
 * for images too large for the CPU.  O(radius^2) per pixel. */
bf_status bf_exact(const float *d_in, size_t in_pitch_bytes, float *d_out, size_t out_pitch_bytes,
                   int height, int width, int spatial, double sigma_s, int radius,
                   int range, double sigma_r, void *stream);

/* The brute-force baseline with a look-up table (Sec. V, Case 2): Eq. (1) as
 * in bf_exact, but the range weight of a neighbour is read from a table of
 * `levels` entries K_r(n * step), step = data_range / (levels - 1), at the
 * entry nearest to |I(x) - I(y)| (index rounded to nearest-even in fp32).
 * With images whose values lie on that grid (e.g. 8-bit data and levels =
 * 256 over data_range 1) the table is exact.  Its cost grows with the window,
 * (2R + 1)^2 taps per pixel, which is why it wins only at small radii.
 * radius <= 32 (0: round(3 sigma_s)), 2 <= levels <= 4096.  Device buffers as
 * bf_exact; asynchronous on `stream`.  Errors: BF_ERR_INVALID_ARG,
 * BF_ERR_UNSUPPORTED (radius > 32), BF_ERR_CUDA. */
bf_status bf_exact_lut(const float *d_in, size_t in_pitch_bytes, float *d_out, size_t out_pitch_bytes,
                       int height, int width, int spatial, double sigma_s, int radius,
                       int range, double sigma_r, double data_range, int levels, void *stream);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of filter requests                         */
/* ---------------------------------------------------------------------- */

typedef struct bf_server bf_server;

typedef struct {
    size_t hbm_budget_bytes;    /* device bytes of the server's arena, reserved once at creation (one
                                   cudaMalloc) and shared out to admitted requests; 0 -> 1/4 of the free
                                   device memory, at most 16 GiB */
    int max_slots;              /* requests resident on the device at once; 0 -> 64 */
    int n_streams;              /* CUDA streams the server launches on; 0 -> 4 */
    int device;                 /* CUDA device ordinal */
    int max_batch;              /* requests merged into one batched launch; 0 -> 16 */
    int plan_threads;           /* host threads building plans for new parameters; 0 -> 4 */
} bf_serve_config;

/* Where a request's images live. */
typedef enum {
    BF_MEM_DEVICE = 0,  /* device memory of the server's device, caller-owned: the server filters in to out */
    BF_MEM_HOST = 1     /* host memory (pinned recommended): the server copies through its arena */
} bf_memory;

typedef struct {
    bf_plan_desc desc;          /* filter parameters (the device field is ignored); plans are built by the
                                   server's plan thread and cached by value */
    const float *in;            /* input, height rows of width floats, row pitch in_pitch_bytes */
    size_t in_pitch_bytes;      /* a multiple of 4, >= width * 4 */
    float *out;                 /* output, same shape, row pitch out_pitch_bytes; must not overlap in */
    size_t out_pitch_bytes;
    int height, width;
    int memory;                 /* bf_memory of in and out */
} bf_request;

typedef struct {
    int status;                 /* bf_status of the request (plan errors included) */
    uint64_t latency_ns;        /* submit -> the result in out (device) or copied to the host buffer */
    uint64_t queue_ns;          /* submit -> admitted: the plan build or cache look-up plus the wait for
                                   arena memory and a slot */
    uint64_t plan_ns;           /* the plan build or cache look-up (part of queue_ns) */
    uint64_t device_ns;         /* device time of the launch group that ran the request (copies included) */
} bf_result;

/* Starts a server thread for one device.  Errors: BF_ERR_INVALID_ARG,
 * BF_ERR_NO_DEVICE, BF_ERR_CUDA, BF_ERR_OOM. */
bf_status bf_serve_create(const bf_serve_config *cfg, bf_server **out);

/* Queues a request and returns its ticket; never waits for GPU work or for
 * the plan: the request's plan is built (or found in the server's cache) by
 * one of the server's plan threads after submission, inside the request's
 * latency.
 * The request is admitted, in order of readiness, once its plan exists and
 * the arena has room for its buffers (host requests: staging for in and out;
 * every request: its share of the batched launch's parameters, work list
 * and partial planes) and a slot is free; admitted requests are merged into
 * batched launches on the server's streams.  The buffers must stay valid
 * until the result has been polled.  Errors at submission:
 * BF_ERR_INVALID_ARG (NULL, bad image or pitch, overlap, unknown memory),
 * BF_ERR_UNSUPPORTED (BF_RANGE_PAPER_3D), BF_ERR_ADMISSION (the staging alone
 * exceeds the arena).  Plan errors, and a request whose buffers exceed the
 * arena once its plan is known (BF_ERR_ADMISSION), are reported by poll in
 * the result's status. */
bf_status bf_serve_submit(bf_server *server, const bf_request *req, uint64_t *ticket);

/* Waits up to timeout_ms (0: just check; < 0: wait without limit) for a
 * request.  BF_OK: *out holds the result and the ticket is released.
 * BF_ERR_TIMEOUT: still in flight.  BF_ERR_NOT_FOUND: unknown ticket. */
bf_status bf_serve_poll(bf_server *server, uint64_t ticket, int timeout_ms, bf_result *out);

/* Cancels a request that has not been admitted yet (BF_OK), else
 * BF_ERR_NOT_FOUND.  A cancelled request polls as BF_ERR_CANCELLED. */
bf_status bf_serve_cancel(bf_server *server, uint64_t ticket);

/* Drains all admitted requests and stops the server (NULL is a no-op). */
void bf_serve_destroy(bf_server *server);

/* ---------------------------------------------------------------------- */
/* Measurement                                                             */
/* ---------------------------------------------------------------------- */

/* Measured fp32 throughput of `device`, the denominator of the fused
 * filter's roofline (the paper has no counterpart; it times its method on a
 * CPU).  Runs two kernels that fill every SM (2048 threads each) with eight
 * independent fused multiply-add chains per thread: one issuing the scalar
 * FFMA, one the two-wide FFMA2 that the filter's hot loops use.  Each is
 * timed with CUDA events over `iters` x 128 FMAs per thread, best of three
 * after a warm-up launch.  *ffma_ops and *ffma2_ops receive fp32 lane
 * operations per second (an FMA on one lane is one operation; an FFMA2
 * instruction is two).  Allocates and frees a 1 KB device buffer and a
 * stream, and synchronizes; about 2 x 4 x iters x 40 ns of GPU time on a
 * 152-SM device (iters = 20000: ~6 ms per launch).  Not for use during
 * stream capture.  Errors: BF_ERR_INVALID_ARG (NULL, iters outside
 * [1, 2^24]), BF_ERR_NO_DEVICE, BF_ERR_CUDA. */
bf_status bf_fp32_peak(int device, int iters, double *ffma_ops, double *ffma2_ops);

/* ---------------------------------------------------------------------- */

const char *bf_status_string(bf_status status);

/* Detail of the last failing call on the calling thread ("" if none). */
const char *bf_last_error(void);

/* Library version, (major << 16) | minor. */
int bf_version(void);

/* Test hook for failure handling: while set to n > 0, the next n kernel
 * launches report BF_ERR_CUDA without launching.  Process-wide. */
void bf_debug_fail_launches(int n);

/* Debug aid for the input range (off by default; the environment variable
 * BF_DEBUG_RANGE=1 switches it on at the first filtering call).  While on,
 * bf_filter first counts the input pixels outside the plan's [i_lo, i_hi]
 * (NaN included) on `stream`, waits for the count, and returns BF_ERR_RANGE
 * without filtering if there are any: the collapsed range policies assume the
 * data range (a difference beyond it can meet a periodic copy of the kernel).
 * The check synchronises the stream and uses one per-device counter, so
 * concurrent checked calls race; it is not for production.  Process-wide;
 * on != 0 switches it on, 0 off. */
void bf_debug_range_checks(int on);

#ifdef __cplusplus
}
#endif

#endif /* BF_H */
