// Plan construction: truncation, coefficient fit, best N-term selection and
// the compilation of the selected Haar terms into box windows for the kernel.
//
// Paper passages: kernel truncation Sec. IV-A; truncated cosine series
// Eqs. (13)-(15) and its best N-term form Eq. (33); Haar system
// Eqs. (17)-(22), best N-term spatial form Eq. (30); Haar terms as signed
// boxes App. A / Eq. (37); best N-term by largest coefficients Sec. III-A
// (Eq. (11)) with the first-20N candidate rule of App. B.
//
// The integrals are done here by composite Gauss-Legendre quadrature, so the
// same code serves any separable spatial profile and any range profile.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <new>

#include "bf_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- quadrature

struct GaussLegendre {
    std::vector<double> x, w;  // nodes / weights on [-1, 1]
    explicit GaussLegendre(int n) : x(n), w(n) {
        // Newton iteration on P_n from the Chebyshev-like initial guess.
        for (int i = 0; i < n; ++i) {
            double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int j = 2; j <= n; ++j) {
                    double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

const GaussLegendre &gl20() {
    static const GaussLegendre g(20);
    return g;
}

// int_a^b f over `pieces` equal sub-intervals, 20-point rule on each.
double integrate(const std::function<double(double)> &f, double a, double b, int pieces) {
    if (!(b > a)) return 0.0;
    const GaussLegendre &g = gl20();
    double h = (b - a) / pieces, s = 0.0;
    for (int p = 0; p < pieces; ++p) {
        double lo = a + p * h, hi = (p == pieces - 1) ? b : lo + h;
        double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo), t = 0.0;
        for (size_t i = 0; i < g.x.size(); ++i) t += g.w[i] * f(c + r * g.x[i]);
        s += r * t;
    }
    return s;
}

// ---------------------------------------------------------------- kernels

double range_value(int kind, double sigma, double t) {
    double a = std::fabs(t);
    switch (kind) {
        case BF_KERNEL_GAUSSIAN: return std::exp(-t * t / (2.0 * sigma * sigma));
        case BF_KERNEL_EXPONENTIAL: return std::exp(-a / sigma);
        case BF_KERNEL_BOX: return a <= sigma ? 1.0 : 0.0;
    }
    return 0.0;
}

double spatial_profile(int kind, double sigma, double x) {
    if (kind == BF_KERNEL_BOX) return 1.0;
    return std::exp(-x * x / (2.0 * sigma * sigma));
}

// int_a^b exp(-x^2 / (2 sigma^2)) dx (a <= b) in closed form, sigma sqrt(pi / 2) (erf(b') - erf(a')) with
// x' = x / (sigma sqrt 2), written with erfc on a one-signed interval so that a tail interval keeps its
// relative accuracy (no difference of two numbers near 1).
double gauss_int(double a, double b, double sigma) {
    const double s = 1.0 / (sigma * std::sqrt(2.0)), k = sigma * std::sqrt(0.5 * kPi);
    if (a >= 0) return k * (std::erfc(a * s) - std::erfc(b * s));
    if (b <= 0) return k * (std::erfc(-b * s) - std::erfc(-a * s));
    return k * (std::erf(b * s) + std::erf(-a * s));
}

// ---------------------------------------------------------------- Haar system

// One 1-D Haar function on [-T, T]: +1 on [lo, mid], -1 on [mid, hi]; phi has lev = -1.
struct Haar1 {
    int lev, k;
    double lo, mid, hi;
};

Haar1 haar_fn(int lev, int k, double T) {
    Haar1 h{lev, k, -T, T, T};
    if (lev < 0) return h;
    double Z = lev == 0 ? 0.0 : (k > 0 ? 1.0 : -1.0) * (2.0 * std::abs(k) - 1.0) * T;  // App. A
    double s = std::ldexp(1.0, -lev);
    h.lo = s * (Z - T);
    h.mid = s * Z;
    h.hi = s * (Z + T);
    return h;
}

// Dictionary: phi, psi_00, then levels 1..J with k = -2^{j-1}..-1, 1..2^{j-1}.
std::vector<Haar1> haar_dictionary(int J, double T) {
    std::vector<Haar1> d;
    d.push_back(haar_fn(-1, 0, T));
    d.push_back(haar_fn(0, 0, T));
    for (int j = 1; j <= J; ++j) {
        int half = 1 << (j - 1);
        for (int k = -half; k <= half; ++k)
            if (k != 0) d.push_back(haar_fn(j, k, T));
    }
    return d;
}

// Value at x with the mean of one-sided limits at a jump.
double haar_value(const Haar1 &h, double x) {
    if (h.lev < 0) return (x > h.lo && x < h.hi) ? 1.0 : ((x == h.lo || x == h.hi) ? 0.5 : 0.0);
    if (x < h.lo || x > h.hi) return 0.0;
    if (x == h.lo) return 0.5;
    if (x == h.hi) return -0.5;
    if (x == h.mid) return 0.0;
    return x < h.mid ? 1.0 : -1.0;
}

// ---------------------------------------------------------------- non-separable spatial kernel

// Tensor 20-point rule over the box [x0, x1] x [y0, y1] of exp(-|x|_2 / sigma).
double box_rule_radial_exp(double sigma, double x0, double x1, double y0, double y1, const GaussLegendre &g) {
    const double cx = 0.5 * (x0 + x1), rx = 0.5 * (x1 - x0), cy = 0.5 * (y0 + y1), ry = 0.5 * (y1 - y0);
    double s = 0.0;
    for (size_t i = 0; i < g.x.size(); ++i) {
        const double x = cx + rx * g.x[i];
        double t = 0.0;
        for (size_t j = 0; j < g.x.size(); ++j) {
            const double y = cy + ry * g.x[j];
            t += g.w[j] * std::exp(-std::sqrt(x * x + y * y) / sigma);
        }
        s += g.w[i] * t;
    }
    return s * rx * ry;
}

// Integral over the cell [0, h] x [0, h] (the kernel's cone point at its corner): the cell is split
// into its corner quarter and three quarters; the quarters away from the corner are smooth enough for
// the tensor rule, and the corner quarter is split again (geometric grading, 48 levels: the last
// corner piece is below 2^-96 of the cell).
double corner_cell_radial_exp(double sigma, double h) {
    const GaussLegendre &g = gl20();
    double s = 0.0, a = h;
    for (int lev = 0; lev < 48; ++lev) {
        const double m = 0.5 * a;
        s += box_rule_radial_exp(sigma, m, a, 0.0, m, g) + box_rule_radial_exp(sigma, 0.0, m, m, a, g) +
             box_rule_radial_exp(sigma, m, a, m, a, g);
        a = m;
    }
    return s;
}

// 2-D Haar coefficients of the radial exponential kernel for every pair of 1-D dictionary entries
// (Eqs. (21)-(22), the 2-D integral kept whole): c[i2 * n + i1] with entry i1 along x and i2 along y.
// The integrals of the kernel over the finest dyadic cells (width h = 2T / 2^(J+1)) are tabulated
// once, by the tensor rule (the four cells at the origin by corner grading), then summed into an
// extended-precision summed-area table, from which each half-support rectangle is read in O(1).
std::vector<double> haar2d_radial_exp(const std::vector<Haar1> &dict, double sigma, double T, int J) {
    const int N = 1 << (J + 1);  // finest cells per axis; the origin is grid point N / 2
    const double h = 2.0 * T / N;
    const int half = N / 2;
    // first quadrant cells q[iy][ix] = integral over [ix h, (ix+1) h] x [iy h, (iy+1) h]; the rest by symmetry
    std::vector<double> q((size_t)half * half);
    for (int iy = 0; iy < half; ++iy)
        for (int ix = 0; ix <= iy; ++ix) {
            double v;
            if (ix == 0 && iy == 0) {
                v = corner_cell_radial_exp(sigma, h);
            } else {
                const GaussLegendre &g = gl20();
                v = box_rule_radial_exp(sigma, ix * h, (ix + 1) * h, iy * h, (iy + 1) * h, g);
            }
            q[(size_t)iy * half + ix] = v;
            q[(size_t)ix * half + iy] = v;
        }
    auto cell = [&](int gx, int gy) {  // cell (gx, gy) of the full grid, 0..N-1
        const int ax = gx >= half ? gx - half : half - 1 - gx, ay = gy >= half ? gy - half : half - 1 - gy;
        return q[(size_t)ay * half + ax];
    };
    std::vector<long double> sat((size_t)(N + 1) * (N + 1), 0.0L);
    for (int gy = 0; gy < N; ++gy) {
        long double row = 0.0L;
        for (int gx = 0; gx < N; ++gx) {
            row += cell(gx, gy);
            sat[(size_t)(gy + 1) * (N + 1) + gx + 1] = sat[(size_t)gy * (N + 1) + gx + 1] + row;
        }
    }
    auto grid = [&](double x) { return (int)std::lround((x + T) / h); };
    auto rect = [&](double x0, double x1, double y0, double y1) {
        const int a = grid(x0), b = grid(x1), c = grid(y0), d = grid(y1);
        const long double v = sat[(size_t)d * (N + 1) + b] - sat[(size_t)c * (N + 1) + b] -
                              sat[(size_t)d * (N + 1) + a] + sat[(size_t)c * (N + 1) + a];
        return (double)v;
    };
    const int n = (int)dict.size();
    std::vector<double> c((size_t)n * n);
    for (int i2 = 0; i2 < n; ++i2)
        for (int i1 = 0; i1 < n; ++i1) {
            const Haar1 &hx = dict[i1], &hy = dict[i2];
            const double xs[2][2] = {{hx.lo, hx.lev < 0 ? hx.hi : hx.mid}, {hx.mid, hx.hi}};
            const double ys[2][2] = {{hy.lo, hy.lev < 0 ? hy.hi : hy.mid}, {hy.mid, hy.hi}};
            const int nx = hx.lev < 0 ? 1 : 2, ny = hy.lev < 0 ? 1 : 2;
            double sum = 0.0;
            for (int a = 0; a < nx; ++a)
                for (int b = 0; b < ny; ++b)
                    sum += (a == b ? 1.0 : -1.0) * rect(xs[a][0], xs[a][1], ys[b][0], ys[b][1]);
            const double sx = hx.lev < 0 ? 1.0 : std::ldexp(1.0, hx.lev), sy = hy.lev < 0 ? 1.0 : std::ldexp(1.0, hy.lev);
            c[(size_t)i2 * n + i1] = sx * sy * sum / (4.0 * T * T);
        }
    return c;
}

struct Cand {
    double mag, c;
    int key[5];
    int a, b;  // indices (1-D dictionary, or k for range terms)
};

bool key_less(const Cand &x, const Cand &y) {
    for (int i = 0; i < 5; ++i)
        if (x.key[i] != y.key[i]) return x.key[i] < y.key[i];
    return false;
}

// Best N-term ranking: |c| descending; values within relative 1e-12 of the
// first member of a run form a tie group, ordered by key; |c| < 1e-14 max dropped.
void rank(std::vector<Cand> &v) {
    double mx = 0;
    for (auto &e : v) mx = std::max(mx, e.mag);
    v.erase(std::remove_if(v.begin(), v.end(), [&](const Cand &e) { return !(e.mag > 0) || e.mag < 1e-14 * mx; }),
            v.end());
    std::sort(v.begin(), v.end(), [](const Cand &x, const Cand &y) {
        if (x.mag != y.mag) return x.mag > y.mag;
        return key_less(x, y);
    });
    size_t i = 0;
    while (i < v.size()) {
        size_t j = i + 1;
        while (j < v.size() && v[j].mag >= v[i].mag * (1.0 - 1e-12)) ++j;
        std::sort(v.begin() + i, v.begin() + j, key_less);
        i = j;
    }
}

// rank() restricted to what a best-`need` selection reads: afterwards v[0 .. need] (as far as v reaches) hold
// the entries rank() would put there, in its order; the rest of v is unspecified.  The top entries are
// selected by partial sorting, widened until the tie group that holds position `need` lies inside.
void rank_top(std::vector<Cand> &v, size_t need) {
    double mx = 0;
    for (auto &e : v) mx = std::max(mx, e.mag);
    v.erase(std::remove_if(v.begin(), v.end(), [&](const Cand &e) { return !(e.mag > 0) || e.mag < 1e-14 * mx; }),
            v.end());
    auto better = [](const Cand &x, const Cand &y) {
        if (x.mag != y.mag) return x.mag > y.mag;
        return key_less(x, y);
    };
    size_t k = std::min(v.size(), need + 64);
    for (;;) {
        std::partial_sort(v.begin(), v.begin() + k, v.end(), better);
        if (k == v.size()) break;
        // greedy tie groups over the sorted prefix (rank()'s rule); the group holding `need` must end before k
        size_t i = 0, end = 0;
        while (i < k) {
            size_t j = i + 1;
            while (j < k && v[j].mag >= v[i].mag * (1.0 - 1e-12)) ++j;
            if (i <= need && need < j) {
                end = j;
                break;
            }
            i = j;
        }
        if (end != 0 && end < k) break;
        k = std::min(v.size(), 2 * k);
    }
    size_t i = 0;
    while (i < k) {
        size_t j = i + 1;
        while (j < k && v[j].mag >= v[i].mag * (1.0 - 1e-12)) ++j;
        std::sort(v.begin() + i, v.begin() + j, key_less);
        if (i > need) break;
        i = j;
    }
}

// ---------------------------------------------------------------- windows

// Splits a set of 1-D profiles p_i(d), d in [-R, R], into shared windows:
// nested centred windows [-b, b] when every profile is even, otherwise the
// maximal runs on which no profile changes.  coef[i][j] is the weight of
// window j in profile i, so that p_i(d) = sum_j coef[i][j] [d in window j].
void split_profiles(const std::vector<std::vector<double>> &prof, int R, double tol,
                    std::vector<std::pair<int, int>> &win, std::vector<std::vector<double>> &coef) {
    const int w = 2 * R + 1;
    auto at = [&](const std::vector<double> &p, int d) { return (d < -R || d > R) ? 0.0 : p[d + R]; };
    bool even = true;
    for (auto &p : prof)
        for (int d = 1; d <= R; ++d)
            if (std::fabs(at(p, d) - at(p, -d)) > tol) even = false;
    win.clear();
    coef.assign(prof.size(), {});
    if (even) {
        std::vector<int> b;
        for (int c = 0; c < R; ++c) {
            bool change = false;
            for (auto &p : prof)
                if (std::fabs(at(p, c) - at(p, c + 1)) > tol) change = true;
            if (change) b.push_back(c);
        }
        b.push_back(R);
        for (size_t j = 0; j < b.size(); ++j) {
            win.push_back({-b[j], b[j]});
            for (size_t i = 0; i < prof.size(); ++i) {
                double nxt = (j + 1 < b.size()) ? at(prof[i], b[j + 1]) : 0.0;
                coef[i].push_back(at(prof[i], b[j]) - nxt);
            }
        }
    } else {
        int start = -R;
        for (int d = -R; d <= R; ++d) {
            bool change = (d == R);
            if (!change)
                for (auto &p : prof)
                    if (std::fabs(at(p, d) - at(p, d + 1)) > tol) change = true;
            if (change) {
                win.push_back({start, d});
                for (size_t i = 0; i < prof.size(); ++i) coef[i].push_back(at(prof[i], start));
                start = d + 1;
            }
        }
    }
    // drop windows no profile uses
    std::vector<std::pair<int, int>> w2;
    std::vector<std::vector<double>> c2(prof.size());
    for (size_t j = 0; j < win.size(); ++j) {
        bool used = false;
        for (size_t i = 0; i < prof.size(); ++i)
            if (std::fabs(coef[i][j]) > tol) used = true;
        if (!used) continue;
        w2.push_back(win[j]);
        for (size_t i = 0; i < prof.size(); ++i) c2[i].push_back(coef[i][j]);
    }
    win.swap(w2);
    coef.swap(c2);
    (void)w;
}

// The Haar range series of the 3-D form: the best N_r-term Haar expansion (Eqs. (17)-(20), selection
// Eq. (11)) of the range kernel truncated to the slice window, in slice units.  Domain [-T_z, T_z],
// T_z = R_z + 1/2, J_z = ceil(log2(2 T_z)); profile K_r(t step), step = dI / (Z - 1).  Ties are ordered by
// (level, k) with phi first.  Fills the kept terms and the table K~_r(d), d = -R_z .. R_z.
bf_status range_haar(const bf_plan_desc &d, double Tr, bf_plan &p) {
    using bfi::fail;
    const int Z = d.z_bins ? d.z_bins : 256;
    const double dI = (double)d.i_hi - (double)d.i_lo, step = dI / (Z - 1);
    const double rzd = std::floor(Tr * (Z - 1) / dI + 1e-9);
    if (rzd > 1023) return fail(BF_ERR_UNSUPPORTED, "the Haar range series needs R_z <= 1023 slices");
    const int rz = (int)rzd;
    const double T = rz + 0.5;
    const int J = (int)std::ceil(std::log2(2.0 * T));
    const double sz = d.sigma_r / step;  // the bandwidth in slices
    // int_a^b K_r(t step) dt: exact for the box; otherwise Gauss-Legendre on each side of the kink at 0,
    // over the span where the profile is not below double precision's range
    auto prof_int = [&](double a, double b) -> double {
        if (!(b > a)) return 0.0;
        if (d.range == BF_KERNEL_BOX) {
            const double lo = std::max(a, -sz), hi = std::min(b, sz);
            return hi > lo ? hi - lo : 0.0;
        }
        const bool gauss = d.range == BF_KERNEL_GAUSSIAN;
        const double L = (gauss ? 40.0 : 800.0) * sz, width = (gauss ? 0.5 : 2.0) * sz;
        auto part = [&](double lo, double hi) -> double {
            lo = std::max(lo, -L);
            hi = std::min(hi, L);
            if (!(hi > lo)) return 0.0;
            const int pieces = std::max(1, (int)std::ceil((hi - lo) / width));
            return integrate([&](double t) { return range_value(d.range, d.sigma_r, t * step); }, lo, hi, pieces);
        };
        return (a < 0 && b > 0) ? part(a, 0.0) + part(0.0, b) : part(a, b);
    };
    std::vector<Haar1> dict = haar_dictionary(J, T);
    std::vector<Cand> rc;
    rc.reserve(dict.size());
    for (size_t i = 0; i < dict.size(); ++i) {
        const Haar1 &h = dict[i];
        const double c = h.lev < 0 ? prof_int(h.lo, h.hi) / (2.0 * T)
                                   : std::ldexp(1.0, h.lev) * (prof_int(h.lo, h.mid) - prof_int(h.mid, h.hi)) / (2.0 * T);
        rc.push_back(Cand{std::fabs(c), c, {h.lev, h.k, 0, 0, 0}, (int)i, 0});
    }
    rank(rc);
    const int n = std::min<int>(d.nr_terms, (int)rc.size());
    if (n < 1) return fail(BF_ERR_INVALID_ARG, "range kernel has no non-zero Haar coefficient");
    p.rh_terms.clear();
    p.rh_coef.clear();
    p.zw.assign(2 * rz + 1, 0.0);
    for (int t = 0; t < n; ++t) {
        const Haar1 &h = dict[rc[t].a];
        p.rh_terms.insert(p.rh_terms.end(), {h.lev, h.k});
        p.rh_coef.push_back(rc[t].c);
        for (int dd = -rz; dd <= rz; ++dd) p.zw[dd + rz] += rc[t].c * haar_value(h, dd);
    }
    p.zw_f.assign(p.zw.begin(), p.zw.end());
    return BF_OK;
}

bf_status build(const bf_plan_desc &d, bf_plan &p) {
    using bfi::fail;
    if (!(d.sigma_s > 0) || !(d.sigma_r > 0) || !std::isfinite(d.sigma_s) || !std::isfinite(d.sigma_r))
        return fail(BF_ERR_INVALID_ARG, "sigma_s and sigma_r must be finite and > 0");
    if (d.ns_terms < 1 || d.nr_terms < 1) return fail(BF_ERR_INVALID_ARG, "ns_terms and nr_terms must be >= 1");
    if (d.nr_terms > 4096) return fail(BF_ERR_INVALID_ARG, "nr_terms too large");
    if (d.radius < 0 || d.radius > 1024) return fail(BF_ERR_INVALID_ARG, "radius must be in [0, 1024]");
    if (!(d.i_hi > d.i_lo)) return fail(BF_ERR_INVALID_ARG, "i_hi must exceed i_lo");
    if (d.t_r < 0 || !std::isfinite(d.t_r)) return fail(BF_ERR_INVALID_ARG, "t_r must be >= 0");
    if (d.spatial != BF_KERNEL_GAUSSIAN && d.spatial != BF_KERNEL_BOX && d.spatial != BF_KERNEL_EXPONENTIAL)
        return fail(BF_ERR_INVALID_ARG, "unknown spatial kernel");
    if (d.range < BF_KERNEL_GAUSSIAN || d.range > BF_KERNEL_BOX) return fail(BF_ERR_INVALID_ARG, "unknown range kernel");
    if (d.policy != BF_RANGE_TRUNCATED_MIN_PERIOD && d.policy != BF_RANGE_UNTRUNCATED_FULL &&
        d.policy != BF_RANGE_PAPER_3D)
        return fail(BF_ERR_INVALID_ARG, "unknown range policy");
    if (d.policy == BF_RANGE_PAPER_3D && d.z_bins != 0 && (d.z_bins < 2 || d.z_bins > bfi::kMaxZBins))
        return fail(BF_ERR_INVALID_ARG, "z_bins must be 0 (256) or in [2, 4096]");
    if (d.range_series != BF_SERIES_COSINE && d.range_series != BF_SERIES_HAAR)
        return fail(BF_ERR_INVALID_ARG, "unknown range series");
    if (d.range_series == BF_SERIES_HAAR && d.policy != BF_RANGE_PAPER_3D)
        return fail(BF_ERR_INVALID_ARG, "the Haar range series runs on the slice axis of BF_RANGE_PAPER_3D");
    if (d.precision < BF_PREC_FP32 || d.precision > BF_PREC_FP16)
        return fail(BF_ERR_INVALID_ARG, "unknown precision");
    if (d.precision != BF_PREC_FP32 && d.policy == BF_RANGE_PAPER_3D)
        return fail(BF_ERR_UNSUPPORTED, "16-bit basis storage applies to the collapsed range policies; the 3-D form "
                                        "is fp32");

    p.desc = d;
    const double dI = (double)d.i_hi - (double)d.i_lo;
    // ---- truncation (Sec. IV-A)
    p.R = d.radius > 0 ? d.radius : (int)std::floor(3.0 * d.sigma_s + 0.5);
    p.Ts = p.R + 0.5;
    p.J = (int)std::ceil(std::log2(2.0 * p.Ts));
    double tr = d.t_r > 0 ? d.t_r
                          : (d.range == BF_KERNEL_GAUSSIAN ? 3.0 * d.sigma_r
                             : d.range == BF_KERNEL_EXPONENTIAL ? d.sigma_r * std::log(100.0) : d.sigma_r);
    if (d.policy == BF_RANGE_UNTRUNCATED_FULL) {
        p.P = dI;
        p.Tr = dI;
    } else if (d.policy == BF_RANGE_PAPER_3D) {
        // one period of the series fits the kernel truncated at T_r; the slice window applies the box
        p.P = tr;
        p.Tr = tr;
    } else {
        p.P = std::max(tr, 0.5 * (dI + tr));
        p.Tr = tr;
    }

    const bool haar_range = d.range_series == BF_SERIES_HAAR;
    if (haar_range) {
        // the Haar range series: the kernel runs one constant cosine term (k = 0, a = 1) and weights the
        // neighbours through the slice table
        bf_status hs = range_haar(d, p.Tr, p);
        if (hs != BF_OK) return hs;
        p.k.push_back(0);
        p.a.push_back(1.0);
    } else {
        // ---- range coefficients a_k on [-P, P] (Eqs. (14), (15)), first 20 N_r candidates (App. B)
        const int ncand = 20 * d.nr_terms;
        double L = std::min(p.Tr, p.P);
        if (d.range == BF_KERNEL_BOX) L = std::min(L, d.sigma_r);
        // One composite 20-point Gauss-Legendre node set on [0, L] with at most two periods of the highest
        // candidate frequency per piece (the rule's error on (2 pi m)^40 / 40! for m periods: ~1e-16 relative at
        // m = 2), 4 + k_max L / (4 P) pieces,
        // serves every candidate: a_k = (2 - [k = 0]) / P sum_i w_i K_r(t_i)
        // cos(pi k t_i / P).  cos(k theta_i) comes from the angle-addition recurrence over k, all nodes at once,
        // re-anchored by a direct cos / sin every 64 frequencies so its rounding stays within ~64 ulp (~1e-14).
        const GaussLegendre &gq = gl20();
        const int pieces = L > 0 ? 4 + (int)std::ceil(0.25 * (ncand - 1) * L / p.P) : 0;
        const int ng = (int)gq.x.size(), nn = pieces * ng;
        std::vector<double> f(nn), th(nn), c1(nn), s1(nn), ck(nn), sk(nn);
        const double hq = pieces > 0 ? L / pieces : 0.0;
        for (int q = 0; q < pieces; ++q) {
            const double lo = q * hq, hi = (q == pieces - 1) ? L : lo + hq;
            const double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
            for (int i = 0; i < ng; ++i) {
                const double t = c + r * gq.x[i];
                f[q * ng + i] = r * gq.w[i] * (d.range == BF_KERNEL_BOX ? 1.0 : range_value(d.range, d.sigma_r, t));
                th[q * ng + i] = kPi * t / p.P;
            }
        }
        for (int n = 0; n < nn; ++n) {
            c1[n] = std::cos(th[n]);
            s1[n] = std::sin(th[n]);
        }
        // (nodes in blocks of 256, so that a block's arrays stay in the L1 cache over the frequency loop)
        std::vector<double> acc(ncand, 0.0);
        for (int n0 = 0; n0 < nn; n0 += 256) {
            const int n1 = std::min(nn, n0 + 256);
            for (int k = 0; k < ncand; ++k) {
                if (k % 64 == 0)
                    for (int n = n0; n < n1; ++n) {
                        ck[n] = k == 0 ? 1.0 : std::cos(k * th[n]);
                        sk[n] = k == 0 ? 0.0 : std::sin(k * th[n]);
                    }
                // eight partial sums: independent chains the compiler can keep in vector registers
                double part[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                int n = n0;
                for (; n + 8 <= n1; n += 8)
                    for (int u = 0; u < 8; ++u) part[u] += f[n + u] * ck[n + u];
                for (; n < n1; ++n) part[0] += f[n] * ck[n];
                acc[k] += ((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7]));
                for (int n = n0; n < n1; ++n) {
                    const double cn = ck[n] * c1[n] - sk[n] * s1[n];
                    sk[n] = sk[n] * c1[n] + ck[n] * s1[n];
                    ck[n] = cn;
                }
            }
        }
        std::vector<Cand> rc(ncand);
        for (int k = 0; k < ncand; ++k) {
            double ak = (k == 0 ? 1.0 : 2.0) * acc[k] / p.P;
            rc[k] = Cand{std::fabs(ak), ak, {k, 0, 0, 0, 0}, k, 0};
        }
        rank(rc);
        int nr = std::min<int>(d.nr_terms, (int)rc.size());
        if (nr < 1) return fail(BF_ERR_INVALID_ARG, "range kernel has no non-zero coefficient");
        std::vector<std::pair<int, double>> sel;
        for (int i = 0; i < nr; ++i) sel.push_back({rc[i].a, rc[i].c});
        std::sort(sel.begin(), sel.end());
        for (auto &e : sel) {
            p.k.push_back(e.first);
            p.a.push_back(e.second);
        }
    }

    // ---- 1-D Haar coefficients of the spatial profile (Eq. (20)); 2-D by separability (Eq. (22)), or
    // computed whole for the non-separable radial exponential
    if (p.J > 12) return fail(BF_ERR_UNSUPPORTED, "radius too large for the Haar dictionary");
    std::vector<Haar1> dict = haar_dictionary(p.J, p.Ts);
    const int n1 = (int)dict.size();
    auto prof_int = [&](double a, double b) {
        if (d.spatial == BF_KERNEL_BOX) return b - a;
        if (d.spatial == BF_KERNEL_GAUSSIAN) return gauss_int(a, b, d.sigma_s);
        int pieces = std::max(1, (int)std::ceil((b - a) / (0.5 * d.sigma_s)));
        return integrate([&](double x) { return spatial_profile(d.spatial, d.sigma_s, x); }, a, b, pieces);
    };
    std::vector<double> c1(n1);
    for (int i = 0; i < n1 && d.spatial != BF_KERNEL_EXPONENTIAL; ++i) {
        const Haar1 &h = dict[i];
        if (h.lev < 0) c1[i] = prof_int(h.lo, h.hi) / (2.0 * p.Ts);
        else c1[i] = std::ldexp(1.0, h.lev) * (prof_int(h.lo, h.mid) - prof_int(h.mid, h.hi)) / (2.0 * p.Ts);
    }
    std::vector<double> c2;  // non-separable kernel: the 2-D coefficients computed whole
    if (d.spatial == BF_KERNEL_EXPONENTIAL) {
        if (p.J > 9) return fail(BF_ERR_UNSUPPORTED, "radius too large for the non-separable spatial kernel (R <= 255)");
        c2 = haar2d_radial_exp(dict, d.sigma_s, p.Ts, p.J);
    }
    // 2-D candidates.  Separable kernels: the coefficient of (i1, i2) is c1[i1] c1[i2], so with the 1-D
    // magnitudes sorted descending, a_1 >= a_2 >= ..., every product outside the top-K1 block is at most
    // a_1 a_{K1+1}, while the block holds K1 products >= a_1 a_{K1}.  With K1 > N_s and a_{K1+1} below the
    // tie threshold of a_{K1}, the best N_s terms and the whole tie group at the cut lie in the block, so
    // only its K1^2 pairs are ranked.  Non-separable kernels rank every pair.
    std::vector<int> top(n1);
    for (int i = 0; i < n1; ++i) top[i] = i;
    int k1 = n1;
    if (c2.empty()) {
        std::sort(top.begin(), top.end(), [&](int x, int y) {
            const double ax = std::fabs(c1[x]), ay = std::fabs(c1[y]);
            return ax != ay ? ax > ay : x < y;
        });
        k1 = std::min(n1, d.ns_terms + 2);
        while (k1 < n1 && std::fabs(c1[top[k1]]) >= std::fabs(c1[top[k1 - 1]]) * (1.0 - 1e-12)) ++k1;
    }
    std::vector<Cand> sc;
    sc.reserve((size_t)k1 * k1);
    for (int a = 0; a < k1; ++a)
        for (int b = 0; b < k1; ++b) {
            const int i1 = top[a], i2 = top[b];
            double c = c2.empty() ? c1[i1] * c1[i2] : c2[(size_t)i2 * n1 + i1];
            int j1 = dict[i1].lev, j2 = dict[i2].lev;
            sc.push_back(Cand{std::fabs(c), c, {std::max(j1, j2), j1, j2, dict[i1].k, dict[i2].k}, i1, i2});
        }
    rank_top(sc, (size_t)d.ns_terms);
    int ns = std::min<int>(d.ns_terms, (int)sc.size());
    p.tie_split = (ns < (int)sc.size() && sc[ns].mag >= sc[ns - 1].mag * (1.0 - 1e-12)) ? 1 : 0;
    const int R = p.R, w = 2 * R + 1;
    p.kernel.assign((size_t)w * w, 0.0);
    for (int t = 0; t < ns; ++t) {
        const Haar1 &hx = dict[sc[t].a], &hy = dict[sc[t].b];
        p.terms.insert(p.terms.end(), {hx.lev, hx.k, hy.lev, hy.k});
        p.tcoef.push_back(sc[t].c);
        std::vector<double> ux(w), uy(w);
        for (int dd = -R; dd <= R; ++dd) {
            ux[dd + R] = haar_value(hx, dd);
            uy[dd + R] = haar_value(hy, dd);
        }
        for (int dy = 0; dy < w; ++dy)
            for (int dx = 0; dx < w; ++dx) p.kernel[(size_t)dy * w + dx] += sc[t].c * ux[dx] * uy[dy];
    }

    // ---- compile into windows.  Weight of the neighbour at offset d = y - x is K~_s(x - y) (Eq. (32)).
    double kmax = 0;
    for (double v : p.kernel) kmax = std::max(kmax, std::fabs(v));
    const double tol = 1e-13 * std::max(kmax, 1e-300);
    auto Kd = [&](int dx, int dy) { return p.kernel[(size_t)(-dy + R) * w + (-dx + R)]; };
    std::vector<std::vector<double>> rows(w, std::vector<double>(w));
    for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) rows[dy + R][dx + R] = Kd(dx, dy);
    // vertical: treat each column offset dx as a profile over dy
    std::vector<std::vector<double>> colprof(w, std::vector<double>(w));
    for (int dx = 0; dx < w; ++dx)
        for (int dy = 0; dy < w; ++dy) colprof[dx][dy] = rows[dy][dx];
    std::vector<std::pair<int, int>> vw;
    std::vector<std::vector<double>> vcoef;  // [dx][v]
    split_profiles(colprof, R, tol, vw, vcoef);
    // horizontal profile of each vertical window: hp[v](dx) = vcoef[dx][v]
    std::vector<std::vector<double>> hp(vw.size(), std::vector<double>(w));
    for (size_t v = 0; v < vw.size(); ++v)
        for (int dx = 0; dx < w; ++dx) hp[v][dx] = vcoef[dx][v];
    std::vector<std::pair<int, int>> hw;
    std::vector<std::vector<double>> hcoef;  // [v][h]
    split_profiles(hp, R, tol, hw, hcoef);
    p.nv = (int)vw.size();
    p.nh = (int)hw.size();
    for (auto &e : vw) p.vwin.insert(p.vwin.end(), {e.first, e.second});
    for (auto &e : hw) p.hwin.insert(p.hwin.end(), {e.first, e.second});
    for (int v = 0; v < p.nv; ++v)
        for (int h = 0; h < p.nh; ++h) p.wcoef.push_back(hcoef[v][h]);
    // verify the compilation reproduces the kernel (hsum[v][dx]: the horizontal windows' weights at dx)
    double maxdiff = 0;
    std::vector<std::vector<double>> hsum(p.nv, std::vector<double>(w, 0.0));
    for (int v = 0; v < p.nv; ++v)
        for (int dx = -R; dx <= R; ++dx)
            for (int h = 0; h < p.nh; ++h)
                if (dx >= hw[h].first && dx <= hw[h].second) hsum[v][dx + R] += hcoef[v][h];
    for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
            double s = 0;
            for (int v = 0; v < p.nv; ++v)
                if (dy >= vw[v].first && dy <= vw[v].second) s += hsum[v][dx + R];
            maxdiff = std::max(maxdiff, std::fabs(s - Kd(dx, dy)));
        }
    if (maxdiff > 1e-12 * std::max(kmax, 1e-300))
        return fail(BF_ERR_UNSUPPORTED, "internal: box-window compilation does not reproduce the kernel");

    // ---- reports
    double sk = 0, sa = 0;
    for (double v : p.kernel) sk += std::fabs(v);
    for (double v : p.a) sa += std::fabs(v);
    if (haar_range) {  // the range weights are the table's: scale the guard by its largest magnitude
        sa = 0;
        for (double v : p.zw) sa = std::max(sa, std::fabs(v));
    }
    p.den_eps = 1e-6 * sk * sa;
    p.range_max_err = 0;
    if (haar_range) {  // the table against the kernel at the slice offsets
        const double step = dI / ((d.z_bins ? d.z_bins : 256) - 1);
        const int rz = ((int)p.zw.size() - 1) / 2;
        for (int dd = -rz; dd <= rz; ++dd)
            p.range_max_err = std::max(p.range_max_err, std::fabs(p.zw[dd + rz] - range_value(d.range, d.sigma_r, dd * step)));
    }
    // the 3-D form keeps the series only inside the range box [-T_r, T_r]
    const double tspan = d.policy == BF_RANGE_PAPER_3D ? std::min(dI, p.Tr) : dI;
    if (!haar_range) {
        // the series at 2001 samples, tens per period of the highest selected frequency: cos(pi k t / P) for
        // k = 0 .. k_max by the angle-addition recurrence (a report: ~k_max ulp is ample), all samples at once
        constexpr int ns = 2001;
        std::vector<double> ts(ns), cth(ns), sth(ns), ck(ns, 1.0), sk(ns, 0.0), sum(ns, 0.0);
        for (int i = 0; i < ns; ++i) {
            ts[i] = -tspan + 2.0 * tspan * i / (ns - 1.0);
            const double th = kPi * ts[i] / p.P;
            cth[i] = std::cos(th);
            sth[i] = std::sin(th);
        }
        for (int k = 0, j = 0; j < (int)p.k.size(); ++k) {
            if (p.k[j] == k) {
                const double a = p.a[j++];
                for (int i = 0; i < ns; ++i) sum[i] += a * ck[i];
            }
            for (int i = 0; i < ns; ++i) {
                const double cn = ck[i] * cth[i] - sk[i] * sth[i];
                sk[i] = sk[i] * cth[i] + ck[i] * sth[i];
                ck[i] = cn;
            }
        }
        for (int i = 0; i < ns; ++i)
            p.range_max_err = std::max(p.range_max_err, std::fabs(sum[i] - range_value(d.range, d.sigma_r, ts[i])));
    }
    p.spatial_max_err = 0;
    std::vector<double> g1(w);  // the Gaussian is separable: exp(-dx^2 / 2 s^2) exp(-dy^2 / 2 s^2)
    for (int dd = -R; dd <= R; ++dd) g1[dd + R] = std::exp(-(double)(dd * dd) / (2.0 * d.sigma_s * d.sigma_s));
    for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
            const double r2 = (double)(dx * dx + dy * dy);
            double ks = d.spatial == BF_KERNEL_BOX           ? 1.0
                        : d.spatial == BF_KERNEL_EXPONENTIAL ? std::exp(-std::sqrt(r2) / d.sigma_s)
                                                             : g1[dx + R] * g1[dy + R];
            p.spatial_max_err = std::max(p.spatial_max_err, std::fabs(ks - p.kernel[(size_t)(dy + R) * w + dx + R]));
        }

    // ---- kernel passes
    p.m = std::max(p.nv, p.nh);
    if (!bfi::kernel_class_supported(p.m))
        return fail(BF_ERR_UNSUPPORTED, "spatial approximation needs " + std::to_string(p.m) +
                                            " box windows per axis; the library supports up to " +
                                            std::to_string(bfi::kMaxWin) + " (reduce ns_terms)");
    if ((int)p.k.size() > bfi::kMaxTerms)
        return fail(BF_ERR_UNSUPPORTED, "more than " + std::to_string(bfi::kMaxTerms) + " cosine terms per plan");
    bfi::FilterParams &kp = p.kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.inv_p = (float)(1.0 / p.P);
    kp.inv_p_lo = (float)(1.0 / p.P - (double)kp.inv_p);
    kp.i_lo = d.i_lo;
    kp.den_eps = (float)p.den_eps;
    const int nr = (int)p.k.size();
    kp.nr = nr;
    for (int i = 0; i < nr; ++i) {
        kp.k[i] = p.k[i];
        kp.a[i] = (float)p.a[i];
    }
    kp.m = p.m;
    int rx = 0, vlo = 0, vhi = 0;
    for (int r = 0; r < p.m; ++r) {
        // windows beyond an axis' count are zero-weight padding
        kp.v0[r] = r < p.nv ? vw[r].first : 0;
        kp.v1[r] = r < p.nv ? vw[r].second : 0;
        kp.u0[r] = r < p.nh ? hw[r].first : 0;
        kp.u1[r] = r < p.nh ? hw[r].second : 0;
        for (int q = 0; q < p.m; ++q) kp.C[r][q] = (r < p.nv && q < p.nh) ? (float)hcoef[r][q] : 0.0f;
        rx = std::max({rx, std::abs(kp.u0[r]), std::abs(kp.u1[r])});
        vlo = std::min(vlo, kp.v0[r]);
        vhi = std::max(vhi, kp.v1[r]);
    }
    kp.rx = rx;
    kp.vlo = vlo;
    kp.vhi = vhi;
    kp.kahan = d.kahan ? 1 : 0;
    if (d.policy == BF_RANGE_PAPER_3D) {
        // z axis: Z levels i_lo + n dI / (Z - 1); window R_z = floor(T_r (Z - 1) / dI) slices (the 1e-9
        // keeps a whole number of levels whole)
        const int Z = d.z_bins ? d.z_bins : 256;
        kp.zbins = Z;
        kp.zscale = (float)((Z - 1) / dI);
        const double rz = std::floor(p.Tr * (Z - 1) / dI + 1e-9);
        kp.rz = (int)std::min(rz, (double)Z);
        kp.zmode = haar_range ? 2 : 1;
        kp.zw = haar_range ? p.zw_f.data() : nullptr;
    }
    return BF_OK;
}

}  // namespace

namespace bfi {
bf_status plan_build(const bf_plan_desc &d, bf_plan &p) { return build(d, p); }
}  // namespace bfi
