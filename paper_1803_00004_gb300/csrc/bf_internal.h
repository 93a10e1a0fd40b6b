// Internal declarations shared by the host plan builder, the C ABI layer and
// the CUDA kernels.  Not installed; the public interface is include/bf.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bf.h"

namespace bfi {

// Largest number of box windows per axis a kernel class handles, the largest
// number of cosine terms one plan carries, and the per-thread budget of
// running sums (terms per group x windows <= kSlotBudget; 4 basis images each).
constexpr int kMaxWin = 6;
constexpr int kMaxTerms = 64;   // selected cosine terms per plan
constexpr int kMaxSlots = 128;  // term slots of a launch (groups x terms per group)
constexpr int kSlotBudget = 16;

// Everything a launch of the fused filter needs, passed by value (it lands in
// the kernel's constant parameter bank; no device allocation per plan).
//
// Vertical windows [v0[r], v1[r]] and horizontal windows [u0[q], u1[q]] are
// neighbour offsets d = y - x (rows / columns); the spatial weight of the
// neighbour at offset (dx, dy) is sum_{r,q} C[r][q] [v0_r <= dy <= v1_r][u0_q <= dx <= u1_q].
struct FilterParams {
    float inv_p;              // 1 / P: basis angle of term k is pi * k * (I - i_lo) / P
    float inv_p_lo;           // 1 / P - inv_p (two-float representation of 1 / P)
    float i_lo;               // intensity origin
    float den_eps;            // denominator guard
    // The plan stores the selected terms (k ascending, nr of them).  A launch with NK terms per group
    // passes a copy laid out by term_layout: nr = groups x NK slots, group g's slots are the consecutive
    // frequencies k[g NK] .. k[g NK] + NK - 1 with a = 0 where the selection has no term.
    int nr;
    int k[kMaxSlots];
    float a[kMaxSlots];
    int m;                    // windows per axis of this kernel class
    int v0[kMaxWin], v1[kMaxWin];
    int u0[kMaxWin], u1[kMaxWin];
    float C[kMaxWin][kMaxWin];
    int rx;                   // max |u| (horizontal reach)
    int vlo, vhi;             // min v0, max v1
    int kahan;                // 1: compensated horizontal sliding sums
    // The 3-D form (z-binned range box): zbins > 0 slices; a pixel's slice is rint((I - i_lo) zscale) in
    // fp32, clamped to [0, zbins - 1]; neighbours within rz slices of the centre's count.  zbins = 0: off.
    int zbins;
    int rz;
    float zscale;
    // zmode 1: the window is a box (weight 1 within rz slices).  zmode 2 (Haar range series): the weight of
    // a neighbour is zw[n(x) - n(y) + rz], a host table of 2 rz + 1 floats that the launcher copies into the
    // slice kernel's parameters (kernels never read this pointer).
    int zmode;
    const float *zw;
};

// Largest slice count of the 3-D form (the per-tile slice bitmap lives in shared memory), and the largest
// weight table of the Haar range series (slice offsets |d| <= 1023).
constexpr int kMaxZBins = 4096;
constexpr int kMaxZWeights = 2047;

// The Haar range series' weight table as a kernel parameter (copied into shared memory by the kernel).
struct ZWeights {
    float w[kMaxZWeights];
};

// Launch geometry chosen by the host.
struct TileConfig {
    int tw;        // output columns per CTA
    int th;        // output rows per CTA
    int ncols;     // column threads (>= tw + 2 rx, multiple of 32)
    int threads;   // ncols + scan warps
    int nk;        // cosine terms per group (template slot count)
    int groups;    // term groups (grid.z); > 1 writes partial planes + finalize
    int ring;      // 1: per-column ring of basis inputs in shared memory
    int depth;     // exchange buffers: 2 (two barriers per row) or 3 (one barrier per row)
    int packed;    // 1: packed-pair family (consecutive term groups); 0: scalar family (any term set); 2: hybrid, the
                   // first group packed (nk consecutive frequencies from the lowest), the terms above it scalar
    size_t smem;   // dynamic shared memory bytes
    int pre = 0;   // basis inputs: 0 computed in the kernel; 1, 2, 3 read from a pre-pass buffer in fp32, fp16, bf16
};

// One image of a persistent batched launch (device copy).
struct BatchImage {
    const float *in;
    float *out;
    float *part;          // partial planes (2 x groups x H x W floats) when groups > 1
    size_t in_pitch, out_pitch;  // elements
    int H, W;
    int params;           // index into the launch's FilterParams array
    int groups;
};

// One unit of work of a persistent launch: one tile of one image for one term group.
struct WorkItem {
    int img;
    int x0, y0, tw, th;
    int g;
};

void set_error(const std::string &msg);
bf_status fail(bf_status st, const std::string &msg);

// ---- device side (bf_filter.cu) ----
bool kernel_class_supported(int m);
// Ranked launch geometries from the cost model, the model's pick, and the
// geometry bf_filter uses (an autotuned one when bf_autotune measured this
// kernel class, reach and image size on this device, else the model's pick).
// Term groups of NK consecutive frequencies covering a plan's selected terms (greedy: each group starts
// at the smallest selected frequency not yet covered), and the launch copy of the parameters laid out in
// those groups (false if the slots exceed kMaxSlots).
int term_groups(const FilterParams &p, int nk);
// Term groups of a launch layout: packed (1), scalar (0) or hybrid (2: the first window of nk consecutive
// frequencies packed, the selected terms above it scalar).
int family_groups(const FilterParams &p, int nk, int packed);
bool term_layout(const FilterParams &p, int nk, FilterParams &out);

// Basis storage (TileConfig::pre) a plan's precision allows: fp32 plans compute the basis in the kernel or read
// an fp32 pre-pass (the same values); 16-bit plans read the pre-pass in their format.
inline bool pre_allowed(int precision, int pre) {
    if (precision == BF_PREC_FP16) return pre == 2;
    if (precision == BF_PREC_BF16) return pre == 3;
    return pre == 0 || pre == 1;
}

// Writes the geometry record (kInfoInts ints) of bf_launch_info / bf_autotune.
constexpr int kInfoInts = 13;
void fill_info(const TileConfig &tc, int height, int width, int *info, int zbins = 0);

std::vector<TileConfig> tile_candidates(const FilterParams &p, int height, int width, int precision, int max_n);
TileConfig model_tile(const FilterParams &p, int height, int width, int precision);
TileConfig choose_tile(const FilterParams &p, int height, int width, int precision);
void remember_tile(const FilterParams &p, int height, int width, int precision, const TileConfig &tc);
// Device scratch of a launch: the partial planes of a grouped launch, plus for the 3-D form (zbins > 0)
// the per-tile slice work list and its two counters.
size_t scratch_bytes(const TileConfig &tc, int height, int width, int zbins = 0);
bf_status launch_filter(const FilterParams &p, int precision, int kahan, const TileConfig &tc, const float *d_in,
                        size_t in_pitch_elems, float *d_out, size_t out_pitch_elems, float *d_scratch, int height,
                        int width, void *stream, int cache_mode = 0);  // 0, or kModeCache*
bf_status launch_exact(const float *d_in, size_t in_pitch_elems, float *d_out, size_t out_pitch_elems,
                       int height, int width, int spatial, float sigma_s, int radius, int range, float sigma_r,
                       void *stream);
bf_status launch_exact_lut(const float *d_in, size_t in_pitch, float *d_out, size_t out_pitch, int height, int width,
                           int spatial, float sigma_s, int radius, int range, float sigma_r, float data_range,
                           int levels, void *stream);
bool debug_consume_launch_failure();

// ---- persistent batched launch (bf_filter.cu) ----
// Terms per CTA used for kernel class m in batched launches (the largest that fits, at most cap when
// cap > 0; 0 if none), the shared-memory bytes a launch with `ncols` column threads needs, and the
// resident CTAs per SM.
int batch_class_nk(int m, int ncols, bool packed, int cap = 0);
size_t batch_smem_bytes(int m, int nk, int ncols);
int batch_ctas_per_sm(int m, int nk, int ncols);
int device_sm_count();
// Enqueues the persistent kernel of class (m, nk) over n_items items (cursor: one
// device int set to 0 before the launch) on `stream`.
bf_status launch_batch_class(int m, int nk, bool packed, int ncols, const BatchImage *d_imgs, const FilterParams *d_params,
                             const WorkItem *d_items, int n_items, int *d_cursor, int grid, void *stream);
// Batch of images in persistent launches without graph capture (device
// buffers allocated and freed stream-ordered on `stream`), and the device bytes
// such a batch needs.
bf_status enqueue_batch_direct(const bf_plan *const *plans, const bf_image *images, int n, void *stream);
// The same into a device buffer the caller reserved (cap bytes, 256-byte aligned, at least
// batch_device_bytes of the batch); allocates no device memory.
bf_status enqueue_batch_into(const bf_plan *const *plans, const bf_image *images, int n, void *stream, void *d_buf,
                             size_t cap);
size_t batch_device_bytes(const bf_plan *const *plans, const bf_image *images, int n);
bf_status check_image(const float *d_in, size_t in_pitch, const float *d_out, size_t out_pitch, int h, int w);
// Sums and divides the partial planes of the listed images (d_list: n_list indices).
bf_status launch_batch_finalize(const BatchImage *d_imgs, const int *d_list, int n_list, int max_h, int max_w,
                                const FilterParams *d_params, void *stream);

}  // namespace bfi

struct bf_plan {
    bf_plan_desc desc;
    int R = 0;
    double Ts = 0, Tr = 0, P = 0;
    int J = 0;
    std::vector<int> k;             // selected cosine indices, ascending
    std::vector<double> a;
    std::vector<int> terms;         // 4 per selected Haar term (ranking order)
    std::vector<double> tcoef;
    int tie_split = 0;
    std::vector<double> kernel;     // K~_s(dx, dy), [(dy+R)(2R+1) + dx+R]
    int nv = 0, nh = 0;
    std::vector<int> vwin, hwin;    // 2 per window
    std::vector<double> wcoef;      // nv x nh
    double range_max_err = 0, spatial_max_err = 0, den_eps = 0;
    int m = 0;                      // kernel class (windows per axis)
    bfi::FilterParams kp;           // kernel parameters (all terms)
    // Haar range series (BF_SERIES_HAAR): kept terms (level, k), coefficients, and the weight table in
    // double (reported) and float (launched; kp.zw points at it)
    std::vector<int> rh_terms;
    std::vector<double> rh_coef, zw;
    std::vector<float> zw_f;
};
