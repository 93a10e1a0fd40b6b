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
constexpr int kMaxTerms = 64;
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
    int nr;                   // cosine terms
    int k[kMaxTerms];         // ascending
    float a[kMaxTerms];
    int m;                    // windows per axis of this kernel class
    int v0[kMaxWin], v1[kMaxWin];
    int u0[kMaxWin], u1[kMaxWin];
    float C[kMaxWin][kMaxWin];
    int rx;                   // max |u| (horizontal reach)
    int vlo, vhi;             // min v0, max v1
};

// Launch geometry chosen by the host.
struct TileConfig {
    int tw;        // output columns per CTA
    int th;        // output rows per CTA
    int ncols;     // column threads (>= tw + 2 rx, multiple of 32)
    int threads;   // ncols + scan warps
    int nk;        // cosine terms per group (template slot count)
    int groups;    // term groups (grid.z); > 1 writes partial planes + finalize
    size_t smem;   // dynamic shared memory bytes
};

void set_error(const std::string &msg);
bf_status fail(bf_status st, const std::string &msg);

// ---- device side (bf_filter.cu) ----
bool kernel_class_supported(int m);
// Ranked launch geometries from the cost model, the model's pick, and the
// geometry bf_filter uses (an autotuned one when bf_autotune measured this
// kernel class, reach and image size on this device, else the model's pick).
std::vector<TileConfig> tile_candidates(const FilterParams &p, int height, int width, int precision, int max_n);
TileConfig model_tile(const FilterParams &p, int height, int width, int precision);
TileConfig choose_tile(const FilterParams &p, int height, int width, int precision);
void remember_tile(const FilterParams &p, int height, int width, int precision, const TileConfig &tc);
size_t scratch_bytes(const TileConfig &tc, int height, int width);
bf_status launch_filter(const FilterParams &p, int precision, int kahan, const TileConfig &tc, const float *d_in,
                        size_t in_pitch_elems, float *d_out, size_t out_pitch_elems, float *d_scratch, int height,
                        int width, void *stream);
bf_status launch_exact(const float *d_in, size_t in_pitch_elems, float *d_out, size_t out_pitch_elems,
                       int height, int width, int spatial, float sigma_s, int radius, int range, float sigma_r,
                       void *stream);
bool debug_consume_launch_failure();

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
};
