// C ABI entry points of include/bf.h: argument checking, plan lifecycle and
// the per-image launch sequence.  The arithmetic lives in plan.cpp (host,
// coefficient fit) and bf_filter.cu (device, the filter itself).
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>

#include "bf_internal.h"

namespace bfi {

bf_status plan_build(const bf_plan_desc &d, bf_plan &p);

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }

bf_status fail(bf_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

void debug_set_fail_launches(int n);
void debug_set_range_checks(bool on);
bool debug_range_checks();
bf_status count_out_of_range(const float *d_in, size_t in_pitch_elems, int h, int w, float lo, float hi, void *stream,
                             unsigned long long *count);

// Runs `fn` with `device` current, restoring the caller's device afterwards.
template <class F>
bf_status with_device(int device, F fn) {
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        return fail(BF_ERR_NO_DEVICE, "no CUDA device");
    }
    if (prev != device && cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return fail(BF_ERR_NO_DEVICE, "cannot select device " + std::to_string(device));
    }
    bf_status st = fn();
    if (prev != device) cudaSetDevice(prev);
    return st;
}

bool ranges_overlap(const void *a, size_t alen, const void *b, size_t blen) {
    auto pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
    return pa < pb + blen && pb < pa + alen;
}

bf_status check_image(const float *d_in, size_t in_pitch, const float *d_out, size_t out_pitch, int h, int w) {
    if (h < 0 || w < 0) return fail(BF_ERR_INVALID_ARG, "negative image size");
    if (h == 0 || w == 0) return BF_OK;
    if (!d_in || !d_out) return fail(BF_ERR_INVALID_ARG, "NULL image pointer");
    if (in_pitch % sizeof(float) || out_pitch % sizeof(float))
        return fail(BF_ERR_INVALID_ARG, "pitch must be a multiple of 4 bytes");
    if (in_pitch < (size_t)w * sizeof(float) || out_pitch < (size_t)w * sizeof(float))
        return fail(BF_ERR_INVALID_ARG, "pitch smaller than width * 4");
    // the kernels form row addresses with a 32-bit byte pitch
    if (in_pitch > 0xffffffffu || out_pitch > 0xffffffffu) return fail(BF_ERR_INVALID_ARG, "pitch of 4 GiB or more");
    size_t in_len = (size_t)(h - 1) * in_pitch + (size_t)w * sizeof(float);
    size_t out_len = (size_t)(h - 1) * out_pitch + (size_t)w * sizeof(float);
    if (ranges_overlap(d_in, in_len, d_out, out_len))
        return fail(BF_ERR_INVALID_ARG, "input and output overlap (in-place filtering is not supported)");
    return BF_OK;
}

// Launch sequence of one image (no argument checks).  d_scratch: at least
// scratch_bytes(tc, h, w, zbins) bytes when the configuration has several term groups or the plan is
// the 3-D form.
bf_status filter_image(const bf_plan *plan, const TileConfig &tc, const float *d_in, size_t in_pitch, float *d_out,
                       size_t out_pitch, int h, int w, float *d_scratch, void *stream) {
    return launch_filter(plan->kp, plan->desc.precision, plan->desc.kahan, tc, d_in, in_pitch / sizeof(float), d_out,
                         out_pitch / sizeof(float), d_scratch, h, w, stream);
}

}  // namespace bfi

using namespace bfi;

extern "C" {

void bf_plan_desc_default(bf_plan_desc *d) {
    if (!d) return;
    std::memset(d, 0, sizeof(*d));
    d->spatial = BF_KERNEL_GAUSSIAN;
    d->sigma_s = 4.0;
    d->radius = 0;
    d->ns_terms = 5;
    d->range = BF_KERNEL_GAUSSIAN;
    d->sigma_r = 0.1;
    d->t_r = 0.0;
    d->nr_terms = 8;
    d->policy = BF_RANGE_TRUNCATED_MIN_PERIOD;
    d->i_lo = 0.0f;
    d->i_hi = 1.0f;
    d->precision = BF_PREC_FP32;
    d->kahan = 1;
    d->device = 0;
    d->z_bins = 0;
    d->range_series = BF_SERIES_COSINE;
}

bf_status bf_plan_create(const bf_plan_desc *desc, bf_plan **out) {
    if (!desc || !out) return fail(BF_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (desc->device >= 0) {
        int n = 0;
        if (cudaGetDeviceCount(&n) != cudaSuccess || desc->device >= n) {
            cudaGetLastError();
            return fail(BF_ERR_NO_DEVICE, "CUDA device " + std::to_string(desc->device) + " not available");
        }
    }
    bf_plan *p = new (std::nothrow) bf_plan();
    if (!p) return fail(BF_ERR_OOM, "host allocation failed");
    bf_status st;
    try {
        st = plan_build(*desc, *p);
    } catch (const std::bad_alloc &) {
        st = fail(BF_ERR_OOM, "host allocation failed while building the plan");
    }
    if (st != BF_OK) {
        delete p;
        return st;
    }
    *out = p;
    return BF_OK;
}

void bf_plan_destroy(bf_plan *plan) { delete plan; }

bf_status bf_coeffs(const bf_plan *p, bf_coeff_view *o) {
    if (!p || !o) return fail(BF_ERR_INVALID_ARG, "NULL argument");
    o->radius = p->R;
    o->t_s = p->Ts;
    o->haar_levels = p->J;
    o->t_r = p->Tr;
    o->period = p->P;
    o->nr = (int)p->k.size();
    o->k = p->k.data();
    o->a = p->a.data();
    o->ns = (int)p->tcoef.size();
    o->haar_terms = p->terms.data();
    o->haar_coef = p->tcoef.data();
    o->tie_split = p->tie_split;
    o->kernel = p->kernel.data();
    o->n_vwin = p->nv;
    o->n_hwin = p->nh;
    o->vwin = p->vwin.data();
    o->hwin = p->hwin.data();
    o->wcoef = p->wcoef.data();
    o->range_max_err = p->range_max_err;
    o->spatial_max_err = p->spatial_max_err;
    o->den_eps = p->den_eps;
    o->passes = (int)((p->k.size() + 15) / 16);
    o->z_bins = p->kp.zbins;
    o->z_radius = p->kp.rz;
    o->range_series = p->desc.range_series;
    o->n_range_haar = (int)p->rh_coef.size();
    o->range_haar = p->rh_terms.empty() ? nullptr : p->rh_terms.data();
    o->range_haar_coef = p->rh_coef.empty() ? nullptr : p->rh_coef.data();
    o->z_weights = p->zw.empty() ? nullptr : p->zw.data();
    return BF_OK;
}

bf_status bf_filter(const bf_plan *plan, const float *d_in, size_t in_pitch, float *d_out, size_t out_pitch,
                    int height, int width, void *stream) {
    if (!plan) return fail(BF_ERR_INVALID_ARG, "NULL plan");
    bf_status st = check_image(d_in, in_pitch, d_out, out_pitch, height, width);
    if (st != BF_OK || height == 0 || width == 0) return st;
    if (plan->desc.device < 0) return fail(BF_ERR_NO_DEVICE, "host-only plan (device = -1)");
    return with_device(plan->desc.device, [&]() -> bf_status {
        if (debug_range_checks()) {
            unsigned long long n = 0;
            bf_status rs = count_out_of_range(d_in, in_pitch / sizeof(float), height, width, plan->desc.i_lo,
                                              plan->desc.i_hi, stream, &n);
            if (rs != BF_OK) return rs;
            if (n > 0)
                return fail(BF_ERR_RANGE, std::to_string(n) + " input pixels outside [i_lo, i_hi] (range check on)");
        }
        TileConfig tc = choose_tile(plan->kp, height, width, plan->desc.precision);
        float *scratch = nullptr;
        cudaStream_t s = (cudaStream_t)stream;
        size_t need = scratch_bytes(tc, height, width, plan->kp.zbins);
        if (need) {
            cudaError_t e = cudaMallocAsync((void **)&scratch, need, s);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(BF_ERR_OOM, std::string("scratch allocation: ") + cudaGetErrorString(e));
            }
        }
        bf_status r = filter_image(plan, tc, d_in, in_pitch, d_out, out_pitch, height, width, scratch, stream);
        if (scratch) cudaFreeAsync(scratch, s);
        return r;
    });
}

bf_status bf_launch_info(const bf_plan *plan, int height, int width, int *info) {
    if (!plan || !info || height < 1 || width < 1) return fail(BF_ERR_INVALID_ARG, "bad launch-info arguments");
    TileConfig tc = choose_tile(plan->kp, height, width, plan->desc.precision);
    fill_info(tc, height, width, info, plan->kp.zbins);
    return BF_OK;
}

bf_status bf_exact(const float *d_in, size_t in_pitch, float *d_out, size_t out_pitch, int height, int width,
                   int spatial, double sigma_s, int radius, int range, double sigma_r, void *stream) {
    bf_status st = check_image(d_in, in_pitch, d_out, out_pitch, height, width);
    if (st != BF_OK || height == 0 || width == 0) return st;
    if (!(sigma_s > 0) || !(sigma_r > 0) || radius < 0) return fail(BF_ERR_INVALID_ARG, "bad exact-filter parameters");
    if (spatial < BF_KERNEL_GAUSSIAN || spatial > BF_KERNEL_BOX) return fail(BF_ERR_INVALID_ARG, "spatial kernel");
    if (range < BF_KERNEL_GAUSSIAN || range > BF_KERNEL_BOX) return fail(BF_ERR_INVALID_ARG, "range kernel");
    int R = radius > 0 ? radius : (int)(3.0 * sigma_s + 0.5);
    return launch_exact(d_in, in_pitch / sizeof(float), d_out, out_pitch / sizeof(float), height, width, spatial,
                        (float)sigma_s, R, range, (float)sigma_r, stream);
}

bf_status bf_exact_lut(const float *d_in, size_t in_pitch, float *d_out, size_t out_pitch, int height, int width,
                       int spatial, double sigma_s, int radius, int range, double sigma_r, double data_range,
                       int levels, void *stream) {
    bf_status st = check_image(d_in, in_pitch, d_out, out_pitch, height, width);
    if (st != BF_OK || height == 0 || width == 0) return st;
    if (!(sigma_s > 0) || !(sigma_r > 0) || radius < 0 || !(data_range > 0) || levels < 2 || levels > 4096)
        return fail(BF_ERR_INVALID_ARG, "bad look-up-table exact-filter parameters");
    if (spatial < BF_KERNEL_GAUSSIAN || spatial > BF_KERNEL_BOX) return fail(BF_ERR_INVALID_ARG, "spatial kernel");
    if (range < BF_KERNEL_GAUSSIAN || range > BF_KERNEL_BOX) return fail(BF_ERR_INVALID_ARG, "range kernel");
    int R = radius > 0 ? radius : (int)(3.0 * sigma_s + 0.5);
    if (R > 32) return fail(BF_ERR_UNSUPPORTED, "look-up-table exact filter: radius above 32");
    return launch_exact_lut(d_in, in_pitch / sizeof(float), d_out, out_pitch / sizeof(float), height, width, spatial,
                            (float)sigma_s, R, range, (float)sigma_r, (float)data_range, levels, stream);
}

const char *bf_status_string(bf_status s) {
    switch (s) {
        case BF_OK: return "ok";
        case BF_ERR_INVALID_ARG: return "invalid argument";
        case BF_ERR_UNSUPPORTED: return "unsupported";
        case BF_ERR_OOM: return "out of memory";
        case BF_ERR_CUDA: return "CUDA error";
        case BF_ERR_ADMISSION: return "request does not fit the memory budget";
        case BF_ERR_TIMEOUT: return "timed out";
        case BF_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        case BF_ERR_RANGE: return "value out of range";
        case BF_ERR_NO_DEVICE: return "no CUDA device";
        case BF_ERR_NOT_FOUND: return "not found";
        case BF_ERR_CANCELLED: return "cancelled";
        case BF_ERR_SCRATCH: return "scratch does not fit the fixed array";
    }
    return "unknown status";
}

const char *bf_last_error(void) { return g_last_error.c_str(); }

int bf_version(void) { return (0 << 16) | 1; }

void bf_debug_fail_launches(int n) { bfi::debug_set_fail_launches(n); }

void bf_debug_range_checks(int on) { bfi::debug_set_range_checks(on != 0); }

}  // extern "C"
