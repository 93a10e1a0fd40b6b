/*
 * bf_oracle.c -- FP64 CPU oracle for the joint-acceleration bilateral filter
 * (Dai, Yuan, Zhang, "Speeding up the Bilateral Filter: A Joint Acceleration Way").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it (through oracle/oracle.py).  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * Everything is plain double precision, written to be checked against the paper
 * by eye:
 *   - range coefficients: Eqs. (13)-(15) on [-P, P], integrals by composite
 *     Romberg quadrature;
 *   - 1-D Haar dictionary and coefficients: Eqs. (17)-(20), Gaussian integrals by
 *     erf differences;
 *   - 2-D separable Haar coefficients: Eq. (22) (product of 1-D factors);
 *   - 2-D coefficients of the non-separable radial exponential kernel
 *     exp(-|x|_2 / sigma) (Eqs. (21)-(22) without the product form): integrals
 *     over rectangles, each split into signed triangles with a vertex at the
 *     origin, integrated in polar form (closed form in r, Romberg in the
 *     edge parameter);
 *   - best N-term selection by largest |coefficient|: Sec. III-A, Eq. (11);
 *     candidates limited to the first 20N range coefficients, App. B;
 *   - O1 exact bilateral filter, Eq. (1); its look-up-table form, the brute-force
 *     baseline of Sec. V (Case 2);
 *   - O2 direct evaluation of Eq. (1) with the approximated kernels of
 *     Eqs. (30) and (33) (the definition of the approximation);
 *   - O3 the paper's fast algorithm, Eqs. (34)-(36): basis images, signed
 *     2-D boxes from App. A / Eq. (37), box sums by 2-D summed-area tables
 *     (Eqs. (24)-(26)), weighting by cos/sin at I(x), divide;
 *   - O2-3D / O3-3D the 3-D form of Sec. IV-D: cosine half-period P = T_r and
 *     the range box applied by dimension promotion (Eq. (2)) over Z intensity
 *     slices; O3-3D takes per-slice 2-D box sums (Eq. (28)) and sums them over
 *     the slice window along z (Eq. (29));
 *   - the same with a Haar series in range: the truncated range kernel's best
 *     N-term Haar expansion (Eqs. (17)-(20), (11)) on the slice axis, each term
 *     a pair of boxes along z evaluated through a running sum over slices.
 *
 * Readings of points the paper leaves open:
 *   - square spatial window |y-x|_inf <= R, R = round(3 sigma_s) by default,
 *     Haar interval T_s = R + 1/2;
 *   - Haar functions take the mean of their one-sided limits at a jump
 *     (only the offset 0 can fall on a jump because T_s is a half-integer);
 *   - the Haar dictionary is {phi, psi_00} plus levels j = 1..J with
 *     J = ceil(log2(2 T_s));
 *   - ranking by raw |c|; values within relative 1e-12 form a tie group ordered
 *     by (max(j1,j2), j1, j2, k1, k2) with phi as level -1; range ties by k;
 *     coefficients below 1e-14 of the largest are never selected;
 *   - the kernel weight of neighbour y for centre x is K~_s(x - y) (Eq. (32));
 *   - collapsed range policy: cosine half-period P >= (dI + T_r)/2 so the
 *     range box of Eq. (33) is identically 1 on the data (Case 1 of Sec. V-C,
 *     "extend the truncated region"); k = 0 is a candidate;
 *   - pixels outside the image are excluded (zero padding, num and den);
 *   - den <= 1e-6 * (sum |K~_s|)(sum |a_k|) -> output I(x) and count it;
 *   - 3-D form: Z levels n dI / (Z - 1) on [0, dI]; a pixel's slice is its
 *     nearest level, decided in fp32; the window along z is R_z =
 *     floor(T_r (Z - 1) / dI) slices each side; the basis uses I(y) itself;
 *   - Haar series in range: domain [-T_z, T_z], T_z = R_z + 1/2 in slice units,
 *     J_z = ceil(log2(2 T_z)), profile K_r(t dI / (Z - 1)); weight of a
 *     neighbour = K~_r at n(x) - n(y); guard 1e-6 (sum |K~_s|) max |K~_r|.
 *
 * Parity pinned by tests/test_oracle_*.py (worked values, closed forms,
 * brute force on tiny inputs and invariants).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ECAP 2

/* kernel kinds */
#define ORC_GAUSSIAN 0
#define ORC_EXPONENTIAL 1
#define ORC_BOX 2

/* range policies */
#define ORC_TRUNCATED_MIN_PERIOD 0
#define ORC_UNTRUNCATED_FULL 1
#define ORC_PAPER_3D 2        /* P = T_r; the range box is applied over intensity bins (the 3-D form) */
#define ORC_PAPER_TRUNCATED 3 /* P = T_r exactly (the paper's own series, used for Table VII) */

static const double ORC_PI = 3.14159265358979323846;

int orc_max_threads(void);

/* ------------------------------------------------------------------ */
/* Kernel profiles                                                      */
/* ------------------------------------------------------------------ */

/* Range kernel K_r(t) (Sec. I: symmetric, decreasing on R+). */
static double range_kernel(int kind, double sigma, double t)
{
    double a = fabs(t);
    switch (kind) {
    case ORC_GAUSSIAN: return exp(-(t * t) / (2.0 * sigma * sigma));
    case ORC_EXPONENTIAL: return exp(-a / sigma);
    case ORC_BOX: return a <= sigma ? 1.0 : 0.0;
    }
    return 0.0;
}

/* Default truncation point T_r = K_r^{-1}(eps) (Sec. IV-A), with 3 sigma for the
 * Gaussian as used in Sec. V-C, eps = 0.01 for the exponential, sigma for the box. */
double orc_default_tr(int kind, double sigma_r)
{
    switch (kind) {
    case ORC_GAUSSIAN: return 3.0 * sigma_r;
    case ORC_EXPONENTIAL: return sigma_r * log(100.0);
    case ORC_BOX: return sigma_r;
    }
    return 3.0 * sigma_r;
}

/* Cosine half-period for a policy; t_r already resolved. */
double orc_period(int policy, double t_r, double data_range)
{
    if (policy == ORC_UNTRUNCATED_FULL) return data_range;
    if (policy == ORC_PAPER_TRUNCATED || policy == ORC_PAPER_3D) return t_r;
    double p = 0.5 * (data_range + t_r);
    return p > t_r ? p : t_r;
}

/* ------------------------------------------------------------------ */
/* Range coefficients, Eqs. (13)-(15) on [-P, P]                        */
/* ------------------------------------------------------------------ */

typedef struct { int kind; double sigma; double omega; } rng_integrand;

/* Integrand on [0, L], where L never exceeds the kernel's support: the box kernel is
 * therefore 1 on the whole interval (its cut-off is applied through L). */
static double rng_f(const rng_integrand *q, double t)
{
    double kv = q->kind == ORC_BOX ? 1.0 : range_kernel(q->kind, q->sigma, t);
    return kv * cos(q->omega * t);
}

/* Romberg integration of q over [a, b] to an absolute tolerance. */
static double romberg(const rng_integrand *q, double a, double b, double tol)
{
    double R[22][22];
    double h = b - a;
    R[0][0] = 0.5 * h * (rng_f(q, a) + rng_f(q, b));
    for (int n = 1; n < 22; n++) {
        h *= 0.5;
        double s = 0.0;
        long m = 1L << (n - 1);
        for (long i = 1; i <= m; i++) s += rng_f(q, a + (2 * i - 1) * h);
        R[n][0] = 0.5 * R[n - 1][0] + h * s;
        double f4 = 1.0;
        for (int j = 1; j <= n; j++) {
            f4 *= 4.0;
            R[n][j] = R[n][j - 1] + (R[n][j - 1] - R[n - 1][j - 1]) / (f4 - 1.0);
        }
        if (n >= 4 && fabs(R[n][n] - R[n - 1][n - 1]) <= tol + 1e-15 * fabs(R[n][n])) return R[n][n];
    }
    return R[21][21];
}

/* a[k], k = 0..ncand-1, of the kernel truncated at t_r, expanded on [-P, P]:
 *   a_0 = (1/2P) int_{-P}^{P} K^T_r,  a_k = (1/P) int_{-P}^{P} K^T_r cos(pi k t / P).
 * The integrand is even, so both reduce to int_0^{min(t_r,P)}. */
int orc_range_coeffs(int kind, double sigma_r, double t_r, double P, int ncand, double *a)
{
    if (!(sigma_r > 0) || !(t_r > 0) || !(P > 0) || ncand < 1 || !a) return ORC_EINVAL;
    double L = t_r < P ? t_r : P;
    if (kind == ORC_BOX && sigma_r < L) L = sigma_r;
    for (int k = 0; k < ncand; k++) {
        rng_integrand q = { kind, sigma_r, ORC_PI * k / P };
        /* composite rule: at least 8 pieces and 4 pieces per half-oscillation */
        int pieces = 8 + (int)ceil(4.0 * k * L / P);
        double h = L / pieces, s = 0.0;
        for (int i = 0; i < pieces; i++) s += romberg(&q, i * h, i == pieces - 1 ? L : (i + 1) * h, 1e-16 * h);
        a[k] = (k == 0 ? 1.0 : 2.0) * s / P;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* 1-D Haar dictionary on [-T, T], Eqs. (17)-(20)                      */
/* ------------------------------------------------------------------ */

/* Dictionary order: index 0 = phi (level -1), 1 = psi_{0,0} (level 0),
 * then level j = 1..J with k = -2^{j-1}..-1, 1..2^{j-1}.  Size 2^{J+1}. */
static void haar_index(int idx, int *lev, int *k)
{
    if (idx == 0) { *lev = -1; *k = 0; return; }
    if (idx == 1) { *lev = 0; *k = 0; return; }
    int j = 1;
    while (idx >= (1 << (j + 1))) j++;
    int off = idx - (1 << j); /* 0 .. 2^j - 1 */
    int half = 1 << (j - 1);
    *lev = j;
    *k = off < half ? off - half : off - half + 1;
}

/* Support pieces of a 1-D Haar function: +1 on [lo, mid], -1 on [mid, hi]
 * (phi: +1 on [-T, T], encoded with mid = hi). */
static void haar_support(int lev, int k, double T, double *lo, double *mid, double *hi)
{
    if (lev < 0) { *lo = -T; *mid = T; *hi = T; return; }
    double Z = (lev == 0) ? 0.0 : (k > 0 ? 1.0 : -1.0) * (2.0 * abs(k) - 1.0) * T; /* Z_k of App. A */
    double s = ldexp(1.0, -lev);
    *lo = s * (Z - T);
    *mid = s * Z;
    *hi = s * (Z + T);
}

/* Value of the Haar function at x; at a jump, the mean of the one-sided limits. */
double orc_haar_eval(int lev, int k, double T, double x)
{
    double lo, mid, hi;
    haar_support(lev, k, T, &lo, &mid, &hi);
    if (lev < 0) {
        if (x > lo && x < hi) return 1.0;
        if (x == lo || x == hi) return 0.5;
        return 0.0;
    }
    if (x > lo && x < mid) return 1.0;
    if (x > mid && x < hi) return -1.0;
    if (x == lo) return 0.5;
    if (x == hi) return -0.5;
    if (x == mid) return 0.0; /* (+1 + -1) / 2 */
    return 0.0;
}

/* int_a^b K_s(x) dx for the 1-D spatial profile. */
static double spatial_profile_int(int kind, double sigma, double a, double b)
{
    if (kind == ORC_GAUSSIAN) {
        double s2 = sigma * sqrt(2.0);
        return sigma * sqrt(ORC_PI / 2.0) * (erf(b / s2) - erf(a / s2));
    }
    /* box spatial kernel: constant 1 on the window */
    return b - a;
}

int orc_haar_levels(double T) { return (int)ceil(log2(2.0 * T)); }

/* 1-D coefficients (Eq. (20)): c_0 = int f phi / 2T, c_jk = 2^j int f psi_jk / 2T.
 * Fills c[0 .. 2^{J+1}-1], and lev/kk with the (j, k) of each entry. */
int orc_haar1d(int kind, double sigma_s, double T, int J, double *c, int *lev, int *kk)
{
    if (!(T > 0) || J < 0 || J > 20 || (kind != ORC_GAUSSIAN && kind != ORC_BOX)) return ORC_EINVAL;
    int n = 1 << (J + 1);
    for (int idx = 0; idx < n; idx++) {
        int j, k;
        double lo, mid, hi;
        haar_index(idx, &j, &k);
        haar_support(j, k, T, &lo, &mid, &hi);
        double v;
        if (j < 0) v = spatial_profile_int(kind, sigma_s, lo, hi) / (2.0 * T);
        else v = ldexp(1.0, j) * (spatial_profile_int(kind, sigma_s, lo, mid) - spatial_profile_int(kind, sigma_s, mid, hi)) / (2.0 * T);
        c[idx] = v;
        if (lev) lev[idx] = j;
        if (kk) kk[idx] = k;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Non-separable spatial kernel: K(x, y) = exp(-sqrt(x^2 + y^2) / sigma)  */
/* ------------------------------------------------------------------ */

/* F(rho) / rho^2 with F(rho) = int_0^rho exp(-r / sigma) r dr = sigma^2 (1 - (1 + u) e^{-u}), u = rho / sigma.
 * F(rho) / rho^2 = (1 - (1 + u) e^{-u}) / u^2 -> 1/2 as u -> 0; the series
 * sum_{n >= 2} (-1)^n (n - 1) u^{n-2} / n! avoids the cancellation for small u. */
static double exp_radial_F_over_rho2(double sigma, double rho)
{
    double u = rho / sigma;
    if (u < 0.5) {
        double s = 0.0, t = 0.5; /* t = u^{n-2} / n!, n = 2 */
        for (int n = 2; n < 30; n++) {
            s += ((n & 1) ? -1.0 : 1.0) * (n - 1) * t;
            t *= u / (n + 1);
        }
        return s;
    }
    return (1.0 - (1.0 + u) * exp(-u)) / (u * u);
}

typedef struct { double sigma, ax, ay, dx, dy, cr; } tri_integrand;

/* Integrand in the edge parameter s of the triangle (origin, A, B): with P(s) = A + s (B - A),
 * polar coordinates give  int_tri f = int_0^1 F(|P(s)|) / |P(s)|^2 * (A x B) ds. */
static double tri_f(const tri_integrand *q, double s)
{
    double px = q->ax + s * q->dx, py = q->ay + s * q->dy;
    double rho = sqrt(px * px + py * py);
    return exp_radial_F_over_rho2(q->sigma, rho) * q->cr;
}

static double romberg_tri(const tri_integrand *q, double a, double b)
{
    double R[22][22];
    double h = b - a;
    R[0][0] = 0.5 * h * (tri_f(q, a) + tri_f(q, b));
    for (int n = 1; n < 22; n++) {
        h *= 0.5;
        double s = 0.0;
        long m = 1L << (n - 1);
        for (long i = 1; i <= m; i++) s += tri_f(q, a + (2 * i - 1) * h);
        R[n][0] = 0.5 * R[n - 1][0] + h * s;
        double f4 = 1.0;
        for (int j = 1; j <= n; j++) {
            f4 *= 4.0;
            R[n][j] = R[n][j - 1] + (R[n][j - 1] - R[n - 1][j - 1]) / (f4 - 1.0);
        }
        if (n >= 4 && fabs(R[n][n] - R[n - 1][n - 1]) <= 1e-16 * fabs(b - a) * fabs(q->cr) + 1e-15 * fabs(R[n][n]))
            return R[n][n];
    }
    return R[21][21];
}

/* Signed integral of the kernel over the triangle (origin, A, B): positive when A -> B turns
 * counter-clockwise about the origin.  The edge is split at its point closest to the origin and
 * into pieces, so Romberg sees a smooth integrand on each piece. */
static double tri_exp(double sigma, double ax, double ay, double bx, double by)
{
    tri_integrand q = { sigma, ax, ay, bx - ax, by - ay, ax * by - ay * bx };
    if (q.cr == 0.0) return 0.0; /* degenerate: the edge's line passes through the origin */
    double len2 = q.dx * q.dx + q.dy * q.dy;
    double sc = -(ax * q.dx + ay * q.dy) / len2;
    double cuts[3] = { 0.0, 1.0, 1.0 };
    int nc = 2;
    if (sc > 0.0 && sc < 1.0) { cuts[1] = sc; cuts[2] = 1.0; nc = 3; }
    const int pieces = 4;
    double total = 0.0;
    for (int c = 0; c + 1 < nc; c++) {
        double a = cuts[c], b = cuts[c + 1];
        for (int i = 0; i < pieces; i++)
            total += romberg_tri(&q, a + (b - a) * i / pieces, i == pieces - 1 ? b : a + (b - a) * (i + 1) / pieces);
    }
    return total;
}

/* int_{x0}^{x1} int_{y0}^{y1} exp(-sqrt(x^2 + y^2) / sigma) dy dx: the rectangle is the signed sum of
 * the triangles (origin, edge) over its boundary taken counter-clockwise. */
double orc_rect_int_exp(double sigma, double x0, double x1, double y0, double y1)
{
    return tri_exp(sigma, x0, y0, x1, y0) + tri_exp(sigma, x1, y0, x1, y1) + tri_exp(sigma, x1, y1, x0, y1) +
           tri_exp(sigma, x0, y1, x0, y0);
}

/* 2-D Haar coefficient (Eqs. (21)-(22) with the 2-D integral kept whole) of the pair of 1-D dictionary
 * entries (i1 along x, i2 along y) for the radial exponential kernel:
 *   c = (s1 / 2T)(s2 / 2T) sum over the +/- halves of sign x sign' x int_{half x half'} K,
 * s = 1 for phi, 2^j for psi_{j,k}. */
static double haar2d_exp(double sigma, double T, int i1, int i2)
{
    int j1, k1, j2, k2;
    double lo1, mid1, hi1, lo2, mid2, hi2;
    haar_index(i1, &j1, &k1);
    haar_index(i2, &j2, &k2);
    haar_support(j1, k1, T, &lo1, &mid1, &hi1);
    haar_support(j2, k2, T, &lo2, &mid2, &hi2);
    double xs[2][2] = { { lo1, mid1 }, { mid1, hi1 } }, ys[2][2] = { { lo2, mid2 }, { mid2, hi2 } };
    int nx = j1 < 0 ? 1 : 2, ny = j2 < 0 ? 1 : 2;
    if (j1 < 0) xs[0][1] = hi1;
    if (j2 < 0) ys[0][1] = hi2;
    double sum = 0.0;
    for (int a = 0; a < nx; a++)
        for (int b = 0; b < ny; b++) {
            double sgn = (a == 0 ? 1.0 : -1.0) * (b == 0 ? 1.0 : -1.0);
            sum += sgn * orc_rect_int_exp(sigma, xs[a][0], xs[a][1], ys[b][0], ys[b][1]);
        }
    double s1 = j1 < 0 ? 1.0 : ldexp(1.0, j1), s2 = j2 < 0 ? 1.0 : ldexp(1.0, j2);
    return s1 * s2 * sum / (4.0 * T * T);
}

/* All 2-D coefficients c[i2 * n + i1], n = 2^{J+1}, of the radial exponential kernel. */
int orc_haar2d_exp(double sigma_s, double T, int J, double *c, int nthreads)
{
    if (!(sigma_s > 0) || !(T > 0) || J < 0 || J > 12 || !c) return ORC_EINVAL;
    int n = 1 << (J + 1);
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
    for (int i2 = 0; i2 < n; i2++)
        for (int i1 = 0; i1 < n; i1++) c[(size_t)i2 * n + i1] = haar2d_exp(sigma_s, T, i1, i2);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Best N-term selection, Sec. III-A                                    */
/* ------------------------------------------------------------------ */

typedef struct { double mag; double c; int t1, t2; int key[5]; } cand2d;

static int key_cmp(const int *a, const int *b)
{
    for (int i = 0; i < 5; i++) if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

static int cmp_mag_desc(const void *pa, const void *pb)
{
    const cand2d *a = pa, *b = pb;
    if (a->mag > b->mag) return -1;
    if (a->mag < b->mag) return 1;
    return key_cmp(a->key, b->key);
}

static int cmp_key(const void *pa, const void *pb)
{
    const cand2d *a = pa, *b = pb;
    return key_cmp(a->key, b->key);
}

/* Orders the candidates: |c| descending; a run of values within relative 1e-12 of
 * the run's first value is one tie group, ordered by key. Returns count kept. */
static int rank_candidates(cand2d *v, int n)
{
    double mx = 0;
    for (int i = 0; i < n; i++) if (v[i].mag > mx) mx = v[i].mag;
    int m = 0;
    for (int i = 0; i < n; i++) if (v[i].mag >= 1e-14 * mx && v[i].mag > 0) v[m++] = v[i];
    qsort(v, m, sizeof(cand2d), cmp_mag_desc);
    int i = 0;
    while (i < m) {
        int j = i + 1;
        while (j < m && v[j].mag >= v[i].mag * (1.0 - 1e-12)) j++;
        qsort(v + i, j - i, sizeof(cand2d), cmp_key);
        i = j;
    }
    return m;
}

/* Range selection: top nr of |a_k|, ties (relative 1e-12) by smaller k. */
int orc_select_range(const double *a, int ncand, int nr, int *ks, double *aks)
{
    cand2d *v = malloc(sizeof(cand2d) * ncand);
    if (!v) return -1;
    for (int k = 0; k < ncand; k++) {
        v[k].mag = fabs(a[k]);
        v[k].c = a[k];
        v[k].t1 = k; v[k].t2 = 0;
        v[k].key[0] = k; v[k].key[1] = v[k].key[2] = v[k].key[3] = v[k].key[4] = 0;
    }
    int m = rank_candidates(v, ncand);
    int n = nr < m ? nr : m;
    for (int i = 0; i < n; i++) { ks[i] = v[i].t1; aks[i] = v[i].c; }
    free(v);
    return n;
}

/* ------------------------------------------------------------------ */
/* Plan: everything the evaluators need                                */
/* ------------------------------------------------------------------ */

#define ORC_MAX_NR 256
#define ORC_MAX_NS 4096

typedef struct {
    int R; double Ts; int J; int n1d;
    double Tr, P;
    int nr; int ks[ORC_MAX_NR]; double ak[ORC_MAX_NR];
    int ns; int sl1[ORC_MAX_NS], sk1[ORC_MAX_NS], sl2[ORC_MAX_NS], sk2[ORC_MAX_NS]; double sc[ORC_MAX_NS];
    int tie_split;
    double *Ks; /* (2R+1)^2, Ks[(dy+R)(2R+1) + dx+R] = K~_s(dx, dy) by direct Haar evaluation */
    double den_eps;
} orc_plan;

static void plan_free(orc_plan *p) { free(p->Ks); p->Ks = NULL; }

static int plan_build(orc_plan *p, int skind, double sigma_s, int radius, int ns_terms,
                      int rkind, double sigma_r, double t_r, int nr_terms, int policy, double data_range)
{
    memset(p, 0, sizeof(*p));
    if (!(sigma_s > 0) || !(sigma_r > 0) || ns_terms < 1 || nr_terms < 1 || nr_terms > ORC_MAX_NR) return ORC_EINVAL;
    if (ns_terms > ORC_MAX_NS) return ORC_ECAP;
    if (skind != ORC_GAUSSIAN && skind != ORC_BOX && skind != ORC_EXPONENTIAL) return ORC_EINVAL;
    p->R = radius > 0 ? radius : (int)lround(3.0 * sigma_s);
    if (radius < 0) return ORC_EINVAL;
    p->Ts = p->R + 0.5;
    p->J = orc_haar_levels(p->Ts);
    p->n1d = 1 << (p->J + 1);
    p->Tr = t_r > 0 ? t_r : orc_default_tr(rkind, sigma_r);
    p->P = orc_period(policy, p->Tr, data_range);
    double trq = (policy == ORC_UNTRUNCATED_FULL) ? p->P : p->Tr;
    p->Tr = trq;

    /* range: first 20 N coefficients (App. B), top N by |a_k| */
    int ncand = 20 * nr_terms;
    double *a = malloc(sizeof(double) * ncand);
    if (!a) return ORC_ECAP;
    orc_range_coeffs(rkind, sigma_r, trq, p->P, ncand, a);
    p->nr = orc_select_range(a, ncand, nr_terms, p->ks, p->ak);
    free(a);

    /* spatial: 2-D Haar coefficients; separable kernels: c(t1,t2) = c1(t1) c1(t2) (Eq. (22));
     * the radial exponential: each 2-D integral computed whole */
    int n = p->n1d;
    double *c1 = malloc(sizeof(double) * n);
    int *lv = malloc(sizeof(int) * n), *kv = malloc(sizeof(int) * n);
    cand2d *v = malloc(sizeof(cand2d) * (size_t)n * n);
    double *c2 = skind == ORC_EXPONENTIAL ? malloc(sizeof(double) * (size_t)n * n) : NULL;
    if (!c1 || !lv || !kv || !v || (skind == ORC_EXPONENTIAL && !c2)) {
        free(c1); free(lv); free(kv); free(v); free(c2);
        return ORC_ECAP;
    }
    for (int i = 0; i < n; i++) haar_index(i, &lv[i], &kv[i]);
    if (skind == ORC_EXPONENTIAL) orc_haar2d_exp(sigma_s, p->Ts, p->J, c2, orc_max_threads());
    else orc_haar1d(skind, sigma_s, p->Ts, p->J, c1, lv, kv);
    size_t m = 0;
    for (int i1 = 0; i1 < n; i1++)
        for (int i2 = 0; i2 < n; i2++) {
            cand2d *e = &v[m++];
            e->c = c2 ? c2[(size_t)i2 * n + i1] : c1[i1] * c1[i2];
            e->mag = fabs(e->c);
            e->t1 = i1; e->t2 = i2;
            int j1 = lv[i1], j2 = lv[i2];
            e->key[0] = j1 > j2 ? j1 : j2;
            e->key[1] = j1; e->key[2] = j2; e->key[3] = kv[i1]; e->key[4] = kv[i2];
        }
    int kept = rank_candidates(v, (int)m);
    p->ns = ns_terms < kept ? ns_terms : kept;
    for (int i = 0; i < p->ns; i++) {
        p->sl1[i] = lv[v[i].t1]; p->sk1[i] = kv[v[i].t1];
        p->sl2[i] = lv[v[i].t2]; p->sk2[i] = kv[v[i].t2];
        p->sc[i] = v[i].c;
    }
    p->tie_split = (p->ns < kept && v[p->ns].mag >= v[p->ns - 1].mag * (1.0 - 1e-12)) ? 1 : 0;
    free(c1); free(lv); free(kv); free(v); free(c2);

    /* K~_s(dx, dy) at integer offsets, Eq. (30) evaluated directly */
    int w = 2 * p->R + 1;
    p->Ks = calloc((size_t)w * w, sizeof(double));
    if (!p->Ks) return ORC_ECAP;
    for (int dy = -p->R; dy <= p->R; dy++)
        for (int dx = -p->R; dx <= p->R; dx++) {
            double s = 0.0;
            for (int i = 0; i < p->ns; i++)
                s += p->sc[i] * orc_haar_eval(p->sl1[i], p->sk1[i], p->Ts, dx) * orc_haar_eval(p->sl2[i], p->sk2[i], p->Ts, dy);
            p->Ks[(dy + p->R) * w + (dx + p->R)] = s;
        }
    double sk = 0, sa = 0;
    for (int i = 0; i < w * w; i++) sk += fabs(p->Ks[i]);
    for (int i = 0; i < p->nr; i++) sa += fabs(p->ak[i]);
    p->den_eps = 1e-6 * sk * sa;
    return ORC_OK;
}

/* Plan summary for the tests.  Arrays sized by the caller: ks/ak >= nr_terms,
 * terms (5 ints + 1 double each) >= ns_terms, Ks >= (2R+1)^2 (pass NULL to skip).
 * ints_out: R, J, nr, ns, tie_split.  dbl_out: Ts, Tr, P, den_eps. */
int orc_plan_info(int skind, double sigma_s, int radius, int ns_terms,
                  int rkind, double sigma_r, double t_r, int nr_terms, int policy, double data_range,
                  int *ints_out, double *dbl_out, int *ks, double *ak,
                  int *term_idx, double *term_c, double *Ks, int Ks_cap)
{
    orc_plan p;
    int st = plan_build(&p, skind, sigma_s, radius, ns_terms, rkind, sigma_r, t_r, nr_terms, policy, data_range);
    if (st) { plan_free(&p); return st; }
    ints_out[0] = p.R; ints_out[1] = p.J; ints_out[2] = p.nr; ints_out[3] = p.ns; ints_out[4] = p.tie_split;
    dbl_out[0] = p.Ts; dbl_out[1] = p.Tr; dbl_out[2] = p.P; dbl_out[3] = p.den_eps;
    for (int i = 0; i < p.nr; i++) { ks[i] = p.ks[i]; ak[i] = p.ak[i]; }
    for (int i = 0; i < p.ns; i++) {
        term_idx[4 * i + 0] = p.sl1[i]; term_idx[4 * i + 1] = p.sk1[i];
        term_idx[4 * i + 2] = p.sl2[i]; term_idx[4 * i + 3] = p.sk2[i];
        term_c[i] = p.sc[i];
    }
    int w = 2 * p.R + 1;
    if (Ks) {
        if (Ks_cap < w * w) { plan_free(&p); return ORC_ECAP; }
        memcpy(Ks, p.Ks, sizeof(double) * w * w);
    }
    plan_free(&p);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* O1: exact bilateral filter, Eq. (1)                                  */
/* ------------------------------------------------------------------ */

static double spatial_kernel2d(int kind, double sigma, int dx, int dy)
{
    if (kind == ORC_BOX) return 1.0;
    if (kind == ORC_EXPONENTIAL) return exp(-sqrt((double)(dx * dx + dy * dy)) / sigma);
    return exp(-(double)(dx * dx + dy * dy) / (2.0 * sigma * sigma));
}

/* Range weight of the difference t: the kernel itself (levels == 0), or the look-up-table form of the
 * brute-force baseline (Sec. V, Case 2): a table of `levels` entries K_r(n * step), n = 0 .. levels-1,
 * step = data_range / (levels - 1), read at the entry nearest to |t|.  The entry is chosen in fp32 (the
 * image data are fp32: |I(x) - I(y)| times 1/step, rounded to nearest-even), the same decision the device
 * makes; the table value is evaluated in fp64. */
static double range_weight(int rkind, double sigma_r, double ix, double iy, int levels, double data_range)
{
    if (levels <= 0) return range_kernel(rkind, sigma_r, ix - iy);
    const float d = fabsf((float)ix - (float)iy);
    const float inv_step = (float)((levels - 1) / data_range);
    int n = (int)nearbyintf(d * inv_step);
    if (n > levels - 1) n = levels - 1;
    return range_kernel(rkind, sigma_r, n * (data_range / (levels - 1)));
}

static int exact_bf_impl(const double *I, int H, int W, int skind, double sigma_s, int radius, int rkind,
                         double sigma_r, int levels, double data_range, double *out, const int *rows, int nrows,
                         int nthreads)
{
    if (!I || !out || H < 0 || W < 0 || !(sigma_s > 0) || !(sigma_r > 0) || radius < 0) return ORC_EINVAL;
    if (levels < 0 || levels == 1 || (levels > 0 && !(data_range > 0))) return ORC_EINVAL;
    int R = radius > 0 ? radius : (int)lround(3.0 * sigma_s);
    int w = 2 * R + 1;
    double *Ks = malloc(sizeof(double) * w * w);
    if (!Ks) return ORC_ECAP;
    for (int dy = -R; dy <= R; dy++)
        for (int dx = -R; dx <= R; dx++) Ks[(dy + R) * w + dx + R] = spatial_kernel2d(skind, sigma_s, dx, dy);
    int nr = rows ? nrows : H;
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int ri = 0; ri < nr; ri++) {
        int y = rows ? rows[ri] : ri;
        for (int x = 0; x < W; x++) {
            double ix = I[(size_t)y * W + x], num = 0.0, den = 0.0;
            for (int dy = -R; dy <= R; dy++) {
                int yy = y + dy;
                if (yy < 0 || yy >= H) continue;
                for (int dx = -R; dx <= R; dx++) {
                    int xx = x + dx;
                    if (xx < 0 || xx >= W) continue;
                    double iy = I[(size_t)yy * W + xx];
                    double wgt = Ks[(dy + R) * w + dx + R] * range_weight(rkind, sigma_r, ix, iy, levels, data_range);
                    num += wgt * iy;
                    den += wgt;
                }
            }
            out[(size_t)ri * W + x] = num / den;
        }
    }
    free(Ks);
    return ORC_OK;
}

/* out[y*W+x] for every pixel; window |y-x|_inf <= R (R = round(3 sigma_s) if radius == 0),
 * range kernel not truncated.  rows/nrows restrict the output to a subset of rows
 * (rows == NULL: all rows). */
int orc_exact_bf(const double *I, int H, int W, int skind, double sigma_s, int radius,
                 int rkind, double sigma_r, double *out, const int *rows, int nrows, int nthreads)
{
    return exact_bf_impl(I, H, W, skind, sigma_s, radius, rkind, sigma_r, 0, 0.0, out, rows, nrows, nthreads);
}

/* The brute-force baseline with the range kernel read from a table (see range_weight). */
int orc_exact_bf_lut(const double *I, int H, int W, int skind, double sigma_s, int radius, int rkind,
                     double sigma_r, int levels, double data_range, double *out, int nthreads)
{
    if (levels < 2) return ORC_EINVAL;
    return exact_bf_impl(I, H, W, skind, sigma_s, radius, rkind, sigma_r, levels, data_range, out, NULL, 0,
                         nthreads);
}

/* ------------------------------------------------------------------ */
/* O2: Eq. (1) with the approximated kernels (definition)               */
/* ------------------------------------------------------------------ */

int orc_approx_direct(const double *I, int H, int W,
                      int skind, double sigma_s, int radius, int ns_terms,
                      int rkind, double sigma_r, double t_r, int nr_terms, int policy, double data_range,
                      double *out, int *ndegen, int nthreads)
{
    if (!I || !out || H < 0 || W < 0) return ORC_EINVAL;
    orc_plan p;
    int st = plan_build(&p, skind, sigma_s, radius, ns_terms, rkind, sigma_r, t_r, nr_terms, policy, data_range);
    if (st) { plan_free(&p); return st; }
    int R = p.R, w = 2 * R + 1;
    int degen = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+:degen) num_threads(nthreads > 0 ? nthreads : 1)
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            double ix = I[(size_t)y * W + x], num = 0.0, den = 0.0;
            for (int dy = -R; dy <= R; dy++) {
                int yy = y + dy;
                if (yy < 0 || yy >= H) continue;
                for (int dx = -R; dx <= R; dx++) {
                    int xx = x + dx;
                    if (xx < 0 || xx >= W) continue;
                    double iy = I[(size_t)yy * W + xx];
                    /* spatial weight K~_s(x - y) = K~_s(-dx, -dy) */
                    double ks = p.Ks[(-dy + R) * w + (-dx + R)];
                    if (ks == 0.0) continue;
                    double kr = 0.0, t = ix - iy;
                    for (int i = 0; i < p.nr; i++) kr += p.ak[i] * cos(ORC_PI * p.ks[i] * t / p.P);
                    num += ks * kr * iy;
                    den += ks * kr;
                }
            }
            if (den <= p.den_eps) { out[(size_t)y * W + x] = ix; degen++; }
            else out[(size_t)y * W + x] = num / den;
        }
    }
    if (ndegen) *ndegen = degen;
    plan_free(&p);
    return ORC_OK;
}

/* O2 at the listed pixels only (pts: npts (row, col) pairs; out[i] for pixel i):
 * the same definition as orc_approx_direct, for sampled checks of large images. */
int orc_approx_direct_at(const double *I, int H, int W,
                         int skind, double sigma_s, int radius, int ns_terms,
                         int rkind, double sigma_r, double t_r, int nr_terms, int policy, double data_range,
                         const int *pts, int npts, double *out, int nthreads)
{
    if (!I || !out || !pts || H < 1 || W < 1 || npts < 0) return ORC_EINVAL;
    orc_plan p;
    int st = plan_build(&p, skind, sigma_s, radius, ns_terms, rkind, sigma_r, t_r, nr_terms, policy, data_range);
    if (st) { plan_free(&p); return st; }
    int R = p.R, w = 2 * R + 1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+:bad) num_threads(nthreads > 0 ? nthreads : 1)
    for (int n = 0; n < npts; n++) {
        int y = pts[2 * n], x = pts[2 * n + 1];
        if (y < 0 || y >= H || x < 0 || x >= W) { out[n] = 0.0; bad++; continue; }
        double ix = I[(size_t)y * W + x], num = 0.0, den = 0.0;
        for (int dy = -R; dy <= R; dy++) {
            int yy = y + dy;
            if (yy < 0 || yy >= H) continue;
            for (int dx = -R; dx <= R; dx++) {
                int xx = x + dx;
                if (xx < 0 || xx >= W) continue;
                double iy = I[(size_t)yy * W + xx];
                double ks = p.Ks[(-dy + R) * w + (-dx + R)];
                if (ks == 0.0) continue;
                double kr = 0.0, t = ix - iy;
                for (int i = 0; i < p.nr; i++) kr += p.ak[i] * cos(ORC_PI * p.ks[i] * t / p.P);
                num += ks * kr * iy;
                den += ks * kr;
            }
        }
        out[n] = (den <= p.den_eps) ? ix : num / den;
    }
    plan_free(&p);
    return bad ? ORC_EINVAL : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* O3: the paper's algorithm, Eqs. (34)-(36) with App. A boxes          */
/* (den_out, if not NULL, receives the denominator of Eq. (1))          */
/* ------------------------------------------------------------------ */

/* A discrete 1-D range [lo, hi] of neighbour offsets with a weight. */
typedef struct { int lo, hi; double w; } drange;

/* The neighbour offsets d with x - (x + d) = -d in the closed continuous
 * interval [a, b] (value v inside, v/2 at an integer endpoint):
 * d in [-b, -a].  Written as one or two integer ranges with weights. */
static int piece_to_ranges(double a, double b, double v, drange *out)
{
    double na = -b, nb = -a;
    int lo_in = (int)ceil(na), hi_in = (int)floor(nb);          /* endpoints included */
    int lo_ex = (int)floor(na) + 1, hi_ex = (int)ceil(nb) - 1;  /* endpoints excluded */
    if (lo_in == lo_ex && hi_in == hi_ex) { out[0].lo = lo_in; out[0].hi = hi_in; out[0].w = v; return 1; }
    out[0].lo = lo_in; out[0].hi = hi_in; out[0].w = 0.5 * v;
    out[1].lo = lo_ex; out[1].hi = hi_ex; out[1].w = 0.5 * v;
    return 2;
}

/* Pieces of one 1-D Haar function as neighbour-offset ranges (App. A:
 * phi -> A, psi -> +A_1, -A_2). */
static int haar_ranges(int lev, int k, double T, drange *out)
{
    double lo, mid, hi;
    haar_support(lev, k, T, &lo, &mid, &hi);
    if (lev < 0) return piece_to_ranges(lo, hi, 1.0, out);
    int n = piece_to_ranges(lo, mid, 1.0, out);
    n += piece_to_ranges(mid, hi, -1.0, out + n);
    return n;
}

/* 2-D summed-area table with a zero row/column in front: S[(y+1)(W+1) + x+1]. */
static void sat_build(const double *g, int H, int W, double *S)
{
    for (int x = 0; x <= W; x++) S[x] = 0.0;
    for (int y = 0; y < H; y++) {
        double c = 0.0;
        S[(size_t)(y + 1) * (W + 1)] = 0.0;
        for (int x = 0; x < W; x++) {
            c += g[(size_t)y * W + x];
            S[(size_t)(y + 1) * (W + 1) + x + 1] = S[(size_t)y * (W + 1) + x + 1] + c;
        }
    }
}

/* Sum of g over rows [y0, y1] x cols [x0, x1], clipped to the image (Eq. (26)). */
static double sat_rect(const double *S, int H, int W, int x0, int x1, int y0, int y1)
{
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > W - 1) x1 = W - 1;
    if (y1 > H - 1) y1 = H - 1;
    if (x0 > x1 || y0 > y1) return 0.0;
    size_t P1 = (size_t)W + 1;
    return S[(size_t)(y1 + 1) * P1 + x1 + 1] - S[(size_t)y0 * P1 + x1 + 1] - S[(size_t)(y1 + 1) * P1 + x0] + S[(size_t)y0 * P1 + x0];
}

typedef struct { int x0, x1, y0, y1; double c; } dbox;

/* The signed discrete boxes of Eq. (37) for the plan's selected Haar terms: products of the 1-D piece
 * ranges (at most 16 per term).  Returns the count. */
static int plan_boxes(const orc_plan *p, dbox *boxes)
{
    int nb = 0;
    for (int i = 0; i < p->ns; i++) {
        drange rx[4], ry[4];
        int nx = haar_ranges(p->sl1[i], p->sk1[i], p->Ts, rx);
        int ny = haar_ranges(p->sl2[i], p->sk2[i], p->Ts, ry);
        for (int a = 0; a < nx; a++)
            for (int b = 0; b < ny; b++) {
                if (rx[a].lo > rx[a].hi || ry[b].lo > ry[b].hi) continue;
                dbox *e = &boxes[nb++];
                e->x0 = rx[a].lo; e->x1 = rx[a].hi; e->y0 = ry[b].lo; e->y1 = ry[b].hi;
                e->c = p->sc[i] * rx[a].w * ry[b].w;
            }
    }
    return nb;
}

int orc_approx_fast(const double *I, int H, int W,
                    int skind, double sigma_s, int radius, int ns_terms,
                    int rkind, double sigma_r, double t_r, int nr_terms, int policy, double data_range,
                    double *out, int *ndegen, int nthreads, double *den_out)
{
    if (!I || !out || H < 0 || W < 0) return ORC_EINVAL;
    orc_plan p;
    int st = plan_build(&p, skind, sigma_s, radius, ns_terms, rkind, sigma_r, t_r, nr_terms, policy, data_range);
    if (st) { plan_free(&p); return st; }
    size_t np = (size_t)H * W;
    if (np == 0) { if (ndegen) *ndegen = 0; plan_free(&p); return ORC_OK; }

    /* signed discrete boxes of Eq. (37): products of the 1-D piece ranges */
    dbox *boxes = malloc(sizeof(dbox) * 16 * p.ns);
    int nb = boxes ? plan_boxes(&p, boxes) : 0;

    double *num = calloc(np, sizeof(double)), *den = calloc(np, sizeof(double));
    double *g = malloc(sizeof(double) * np * 4);
    double *S = malloc(sizeof(double) * (size_t)(H + 1) * (W + 1) * 4);
    double *cb = malloc(sizeof(double) * np), *sb = malloc(sizeof(double) * np);
    if (!num || !den || !g || !S || !cb || !sb || !boxes) {
        free(num); free(den); free(g); free(S); free(cb); free(sb); free(boxes); plan_free(&p); return ORC_ECAP;
    }
    int nt = nthreads > 0 ? nthreads : 1;
    for (int r = 0; r < p.nr; r++) {
        double wk = ORC_PI * p.ks[r] / p.P, ak = p.ak[r];
        /* basis images (Eq. (34)): cos(w I) I, sin(w I) I, cos(w I), sin(w I) */
        for (size_t i = 0; i < np; i++) {
            cb[i] = cos(wk * I[i]); sb[i] = sin(wk * I[i]);
            g[i] = cb[i] * I[i]; g[np + i] = sb[i] * I[i]; g[2 * np + i] = cb[i]; g[3 * np + i] = sb[i];
        }
#pragma omp parallel for num_threads(nt)
        for (int q = 0; q < 4; q++) sat_build(g + q * np, H, W, S + (size_t)q * (H + 1) * (W + 1));
#pragma omp parallel for schedule(static) num_threads(nt)
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                double F[4] = { 0, 0, 0, 0 };
                for (int b = 0; b < nb; b++) {
                    const dbox *e = &boxes[b];
                    for (int q = 0; q < 4; q++)
                        F[q] += e->c * sat_rect(S + (size_t)q * (H + 1) * (W + 1), H, W, x + e->x0, x + e->x1, y + e->y0, y + e->y1);
                }
                size_t i = (size_t)y * W + x;
                num[i] += ak * (cb[i] * F[0] + sb[i] * F[1]);
                den[i] += ak * (cb[i] * F[2] + sb[i] * F[3]);
            }
    }
    int degen = 0;
    for (size_t i = 0; i < np; i++) {
        if (den[i] <= p.den_eps) { out[i] = I[i]; degen++; }
        else out[i] = num[i] / den[i];
        if (den_out) den_out[i] = den[i];
    }
    if (ndegen) *ndegen = degen;
    free(num); free(den); free(g); free(S); free(cb); free(sb); free(boxes);
    plan_free(&p);
    return ORC_OK;
}

/* Number of signed discrete boxes O3 uses (for the cost report). */
int orc_box_count(int skind, double sigma_s, int radius, int ns_terms,
                  int rkind, double sigma_r, double t_r, int nr_terms, int policy, double data_range)
{
    orc_plan p;
    int st = plan_build(&p, skind, sigma_s, radius, ns_terms, rkind, sigma_r, t_r, nr_terms, policy, data_range);
    if (st) { plan_free(&p); return -st; }
    int nb = 0;
    for (int i = 0; i < p.ns; i++) {
        drange rx[4], ry[4];
        int nx = haar_ranges(p.sl1[i], p.sk1[i], p.Ts, rx);
        int ny = haar_ranges(p.sl2[i], p.sk2[i], p.Ts, ry);
        for (int a = 0; a < nx; a++)
            for (int b = 0; b < ny; b++)
                if (rx[a].lo <= rx[a].hi && ry[b].lo <= ry[b].hi) nb++;
    }
    plan_free(&p);
    return nb;
}

/* ------------------------------------------------------------------ */
/* The 3-D form (Sec. IV-D): P = T_r, the range box applied by          */
/* dimension promotion (Eq. (2)) over intensity bins z                  */
/* ------------------------------------------------------------------ */

/* The z axis: the data range [0, dI] sampled at Z levels n dI / (Z - 1), n = 0 .. Z - 1 (for 8-bit data,
 * Z = 256 and the levels are the 256 intensities of Sec. II-B).  A pixel sits in the slice of its nearest
 * level.  The decision is taken in fp32, as the images are fp32: n = rint(I * s), s = fl32((Z - 1) / dI),
 * ties to even, clamped to [0, Z - 1]. */
static float z_scale(int Z, double data_range) { return (float)((Z - 1) / data_range); }

static int z_bin(double I, float s, int Z)
{
    float t = nearbyintf((float)I * s);
    if (!(t > 0.0f)) return 0;
    if (t > (float)(Z - 1)) return Z - 1;
    return (int)t;
}

/* The window along z: slices within R_z = floor(T_r (Z - 1) / dI) of the centre pixel's slice, i.e. the
 * levels inside [I(x) - T_r, I(x) + T_r] (Eq. (35)) for on-grid data.  The 1e-9 absorbs the rounding of
 * T_r (Z - 1) / dI when T_r is a whole number of levels. */
static int z_radius(double Tr, int Z, double data_range) { return (int)floor(Tr * (Z - 1) / data_range + 1e-9); }

/* O2-3D at one pixel: Eq. (1) with K~_s (Eq. (30)), the cosine series of period 2 T_r (Eq. (33) with
 * P = T_r) and the range box over slices: neighbour y counts for centre x iff |n(y) - n(x)| <= R_z.
 * Returns the numerator and denominator. */
static void direct3d_at(const orc_plan *p, const double *I, int H, int W, int y, int x, float zs, int Z, int Rz,
                        double *num_out, double *den_out)
{
    const int R = p->R, w = 2 * R + 1;
    double ix = I[(size_t)y * W + x], num = 0.0, den = 0.0;
    int nx = z_bin(ix, zs, Z);
    for (int dy = -R; dy <= R; dy++) {
        int yy = y + dy;
        if (yy < 0 || yy >= H) continue;
        for (int dx = -R; dx <= R; dx++) {
            int xx = x + dx;
            if (xx < 0 || xx >= W) continue;
            double iy = I[(size_t)yy * W + xx];
            if (abs(z_bin(iy, zs, Z) - nx) > Rz) continue;
            double ks = p->Ks[(-dy + R) * w + (-dx + R)];
            if (ks == 0.0) continue;
            double kr = 0.0, t = ix - iy;
            for (int i = 0; i < p->nr; i++) kr += p->ak[i] * cos(ORC_PI * p->ks[i] * t / p->P);
            num += ks * kr * iy;
            den += ks * kr;
        }
    }
    *num_out = num;
    *den_out = den;
}

/* O2-3D: the definition at every pixel (den_out, if not NULL, receives the denominators). */
int orc_approx3d_direct(const double *I, int H, int W,
                        int skind, double sigma_s, int radius, int ns_terms,
                        int rkind, double sigma_r, double t_r, int nr_terms, int policy, double data_range,
                        int zbins, double *out, int *ndegen, int nthreads, double *den_out)
{
    if (!I || !out || H < 0 || W < 0 || policy != ORC_PAPER_3D || zbins < 2 || !(data_range > 0)) return ORC_EINVAL;
    orc_plan p;
    int st = plan_build(&p, skind, sigma_s, radius, ns_terms, rkind, sigma_r, t_r, nr_terms, policy, data_range);
    if (st) { plan_free(&p); return st; }
    const int Z = zbins, Rz = z_radius(p.Tr, Z, data_range);
    const float zs = z_scale(Z, data_range);
    int degen = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+:degen) num_threads(nthreads > 0 ? nthreads : 1)
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            size_t i = (size_t)y * W + x;
            double num, den;
            direct3d_at(&p, I, H, W, y, x, zs, Z, Rz, &num, &den);
            if (den <= p.den_eps) { out[i] = I[i]; degen++; }
            else out[i] = num / den;
            if (den_out) den_out[i] = den;
        }
    }
    if (ndegen) *ndegen = degen;
    plan_free(&p);
    return ORC_OK;
}

/* O2-3D at the listed pixels only (pts: npts (row, col) pairs), for sampled checks of large images. */
int orc_approx3d_direct_at(const double *I, int H, int W,
                           int skind, double sigma_s, int radius, int ns_terms,
                           int rkind, double sigma_r, double t_r, int nr_terms, int policy, double data_range,
                           int zbins, const int *pts, int npts, double *out, double *den_out, int nthreads)
{
    if (!I || !out || !pts || H < 1 || W < 1 || npts < 0 || policy != ORC_PAPER_3D || zbins < 2 || !(data_range > 0))
        return ORC_EINVAL;
    for (int n = 0; n < npts; n++)
        if (pts[2 * n] < 0 || pts[2 * n] >= H || pts[2 * n + 1] < 0 || pts[2 * n + 1] >= W) return ORC_EINVAL;
    orc_plan p;
    int st = plan_build(&p, skind, sigma_s, radius, ns_terms, rkind, sigma_r, t_r, nr_terms, policy, data_range);
    if (st) { plan_free(&p); return st; }
    const int Z = zbins, Rz = z_radius(p.Tr, Z, data_range);
    const float zs = z_scale(Z, data_range);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
    for (int n = 0; n < npts; n++) {
        int y = pts[2 * n], x = pts[2 * n + 1];
        double num, den;
        direct3d_at(&p, I, H, W, y, x, zs, Z, Rz, &num, &den);
        out[n] = den <= p.den_eps ? I[(size_t)y * W + x] : num / den;
        if (den_out) den_out[n] = den;
    }
    plan_free(&p);
    return ORC_OK;
}

/* O3-3D: the paper's steps.  For each term k the auxiliary images of Eq. (35) are one-hot in z:
 * F(y, z) = g(y) [n(y) = z] for the four basis images g of Eq. (34).  For every slice z the 2-D box sums
 * of the signed boxes (Eq. (37)) come from 2-D summed-area tables of the slice (Eq. (28)); the sum over
 * the window [n(x) - R_z, n(x) + R_z] along z (Eq. (29)) is accumulated slice by slice at the pixels
 * whose window holds z (the sliding-window form of the 1-D table along z, Sec. V).  The window sums are
 * then weighted by a_k cos / sin at I(x) (Eq. (36)) and divided.  Slices no pixel falls in contribute
 * zero and are skipped. */
int orc_approx3d_fast(const double *I, int H, int W,
                      int skind, double sigma_s, int radius, int ns_terms,
                      int rkind, double sigma_r, double t_r, int nr_terms, int policy, double data_range,
                      int zbins, double *out, int *ndegen, int nthreads, double *den_out)
{
    if (!I || !out || H < 0 || W < 0 || policy != ORC_PAPER_3D || zbins < 2 || !(data_range > 0)) return ORC_EINVAL;
    orc_plan p;
    int st = plan_build(&p, skind, sigma_s, radius, ns_terms, rkind, sigma_r, t_r, nr_terms, policy, data_range);
    if (st) { plan_free(&p); return st; }
    size_t np = (size_t)H * W;
    if (np == 0) { if (ndegen) *ndegen = 0; plan_free(&p); return ORC_OK; }
    const int Z = zbins, Rz = z_radius(p.Tr, Z, data_range);
    const float zs = z_scale(Z, data_range);

    dbox *boxes = malloc(sizeof(dbox) * 16 * p.ns);
    int nb = boxes ? plan_boxes(&p, boxes) : 0;
    double *num = calloc(np, sizeof(double)), *den = calloc(np, sizeof(double));
    double *g = malloc(sizeof(double) * np * 4);
    double *S = malloc(sizeof(double) * (size_t)(H + 1) * (W + 1) * 4);
    double *F = malloc(sizeof(double) * np * 4);
    double *cb = malloc(sizeof(double) * np), *sb = malloc(sizeof(double) * np);
    int *nz = malloc(sizeof(int) * np), *occupied = calloc((size_t)Z, sizeof(int));
    if (!num || !den || !g || !S || !F || !cb || !sb || !boxes || !nz || !occupied) {
        free(num); free(den); free(g); free(S); free(F); free(cb); free(sb); free(boxes); free(nz); free(occupied);
        plan_free(&p);
        return ORC_ECAP;
    }
    for (size_t i = 0; i < np; i++) { nz[i] = z_bin(I[i], zs, Z); occupied[nz[i]] = 1; }
    int nt = nthreads > 0 ? nthreads : 1;
    for (int r = 0; r < p.nr; r++) {
        double wk = ORC_PI * p.ks[r] / p.P, ak = p.ak[r];
        for (size_t i = 0; i < np; i++) { cb[i] = cos(wk * I[i]); sb[i] = sin(wk * I[i]); }
        memset(F, 0, sizeof(double) * np * 4);
        for (int z = 0; z < Z; z++) {
            if (!occupied[z]) continue;
            /* slice z of the auxiliary images: the basis images where n(y) = z, zero elsewhere */
            for (size_t i = 0; i < np; i++) {
                int on = nz[i] == z;
                g[i] = on ? cb[i] * I[i] : 0.0; g[np + i] = on ? sb[i] * I[i] : 0.0;
                g[2 * np + i] = on ? cb[i] : 0.0; g[3 * np + i] = on ? sb[i] : 0.0;
            }
#pragma omp parallel for num_threads(nt)
            for (int q = 0; q < 4; q++) sat_build(g + q * np, H, W, S + (size_t)q * (H + 1) * (W + 1));
#pragma omp parallel for schedule(static) num_threads(nt)
            for (int y = 0; y < H; y++)
                for (int x = 0; x < W; x++) {
                    size_t i = (size_t)y * W + x;
                    if (abs(nz[i] - z) > Rz) continue;
                    for (int b = 0; b < nb; b++) {
                        const dbox *e = &boxes[b];
                        for (int q = 0; q < 4; q++)
                            F[q * np + i] += e->c * sat_rect(S + (size_t)q * (H + 1) * (W + 1), H, W, x + e->x0,
                                                             x + e->x1, y + e->y0, y + e->y1);
                    }
                }
        }
        for (size_t i = 0; i < np; i++) {
            num[i] += ak * (cb[i] * F[i] + sb[i] * F[np + i]);
            den[i] += ak * (cb[i] * F[2 * np + i] + sb[i] * F[3 * np + i]);
        }
    }
    int degen = 0;
    for (size_t i = 0; i < np; i++) {
        if (den[i] <= p.den_eps) { out[i] = I[i]; degen++; }
        else out[i] = num[i] / den[i];
        if (den_out) den_out[i] = den[i];
    }
    if (ndegen) *ndegen = degen;
    free(num); free(den); free(g); free(S); free(F); free(cb); free(sb); free(boxes); free(nz); free(occupied);
    plan_free(&p);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* The 3-D form with a Haar series in range: the range kernel's best   */
/* N-term Haar expansion (Eqs. (17)-(20), selection Eq. (11)) on the   */
/* slice axis; each term is a pair of boxes along z (Eqs. (28)-(29))    */
/* ------------------------------------------------------------------ */

/* int_a^b K_r(t step) dt for t in slice units (closed forms; the box kernel is 1 on |t step| <= sigma_r). */
static double range_profile_int(int kind, double sigma_r, double step, double a, double b)
{
    if (!(b > a)) return 0.0;
    double sz = sigma_r / step; /* the bandwidth in slices */
    if (kind == ORC_GAUSSIAN) return spatial_profile_int(ORC_GAUSSIAN, sz, a, b);
    if (kind == ORC_BOX) {
        double lo = a > -sz ? a : -sz, hi = b < sz ? b : sz;
        return hi > lo ? hi - lo : 0.0;
    }
    double s = 0.0; /* exponential exp(-|t| / sz), split at 0 */
    if (a < 0) { double hi = b < 0 ? b : 0.0; s += sz * (exp(hi / sz) - exp(a / sz)); }
    if (b > 0) { double lo = a > 0 ? a : 0.0; s += sz * (exp(-lo / sz) - exp(-b / sz)); }
    return s;
}

/* The range series on the slice axis.  Domain [-T_z, T_z], T_z = R_z + 1/2 (R_z as in the 3-D form, so the
 * truncated kernel covers the slice offsets |d| <= R_z); J_z = ceil(log2(2 T_z)) levels; the profile is
 * K_r(t step), step = dI / (Z - 1).  Coefficients by Eq. (20); the N_r largest |c| kept (ties as for the
 * spatial terms, ordered by (level, k) with phi first).  The weight table holds K~_r at the integer
 * offsets d = n(x) - n(y) (the range argument I(x) - I(y) in slices), w[d + R_z]. */
typedef struct {
    int Rz, Jz, n;
    double Tz, wmax;
    int lev[ORC_MAX_NR], k[ORC_MAX_NR];
    double c[ORC_MAX_NR];
    double *w;
} orc_zhaar;

static void zhaar_free(orc_zhaar *h) { free(h->w); h->w = NULL; }

static int zhaar_build(orc_zhaar *h, int rkind, double sigma_r, double Tr, int nr_terms, int Z, double data_range)
{
    memset(h, 0, sizeof(*h));
    if (nr_terms < 1 || nr_terms > ORC_MAX_NR || Z < 2 || !(data_range > 0)) return ORC_EINVAL;
    const double step = data_range / (Z - 1);
    h->Rz = z_radius(Tr, Z, data_range);
    if (h->Rz > 1023) return ORC_ECAP;
    h->Tz = h->Rz + 0.5;
    h->Jz = orc_haar_levels(h->Tz);
    const int n = 1 << (h->Jz + 1);
    cand2d *v = malloc(sizeof(cand2d) * n);
    h->w = calloc((size_t)(2 * h->Rz + 1), sizeof(double));
    if (!v || !h->w) { free(v); zhaar_free(h); return ORC_ECAP; }
    for (int idx = 0; idx < n; idx++) {
        int j, k;
        double lo, mid, hi, c;
        haar_index(idx, &j, &k);
        haar_support(j, k, h->Tz, &lo, &mid, &hi);
        if (j < 0) c = range_profile_int(rkind, sigma_r, step, lo, hi) / (2.0 * h->Tz);
        else c = ldexp(1.0, j) * (range_profile_int(rkind, sigma_r, step, lo, mid) -
                                  range_profile_int(rkind, sigma_r, step, mid, hi)) / (2.0 * h->Tz);
        cand2d *e = &v[idx];
        e->c = c; e->mag = fabs(c); e->t1 = j; e->t2 = k;
        e->key[0] = j; e->key[1] = k; e->key[2] = e->key[3] = e->key[4] = 0;
    }
    int kept = rank_candidates(v, n);
    h->n = nr_terms < kept ? nr_terms : kept;
    for (int i = 0; i < h->n; i++) { h->lev[i] = v[i].t1; h->k[i] = v[i].t2; h->c[i] = v[i].c; }
    free(v);
    h->wmax = 0.0;
    for (int d = -h->Rz; d <= h->Rz; d++) {
        double s = 0.0;
        for (int i = 0; i < h->n; i++) s += h->c[i] * orc_haar_eval(h->lev[i], h->k[i], h->Tz, d);
        h->w[d + h->Rz] = s;
        if (fabs(s) > h->wmax) h->wmax = fabs(s);
    }
    return ORC_OK;
}

/* The range series of a plan (for the tests): R_z, J_z and the kept terms (lev, k, c), and the table. */
int orc_zhaar_info(int rkind, double sigma_r, double t_r, int nr_terms, int zbins, double data_range,
                   int *ints_out, int *lev, int *kk, double *c, double *w, int w_cap)
{
    orc_zhaar h;
    double Tr = t_r > 0 ? t_r : orc_default_tr(rkind, sigma_r);
    int st = zhaar_build(&h, rkind, sigma_r, Tr, nr_terms, zbins, data_range);
    if (st) { zhaar_free(&h); return st; }
    ints_out[0] = h.Rz; ints_out[1] = h.Jz; ints_out[2] = h.n;
    for (int i = 0; i < h.n; i++) { lev[i] = h.lev[i]; kk[i] = h.k[i]; c[i] = h.c[i]; }
    if (w) {
        if (w_cap < 2 * h.Rz + 1) { zhaar_free(&h); return ORC_ECAP; }
        memcpy(w, h.w, sizeof(double) * (2 * h.Rz + 1));
    }
    zhaar_free(&h);
    return ORC_OK;
}

/* O2-3D with the Haar range series: Eq. (1) with K~_s and the range weight w[n(x) - n(y) + R_z]
 * (0 beyond R_z).  Guard: den <= 1e-6 (sum |K~_s|) max |w| -> I(x).  pts == NULL: every pixel into
 * out[H W]; else the npts listed (row, col) pixels into out[npts].  den_out as out, or NULL. */
int orc_approx3dh_direct(const double *I, int H, int W, int skind, double sigma_s, int radius, int ns_terms,
                         int rkind, double sigma_r, double t_r, int nr_terms, int zbins, double data_range,
                         const int *pts, int npts, double *out, double *den_out, int nthreads)
{
    if (!I || !out || H < 0 || W < 0 || zbins < 2 || !(data_range > 0) || (pts && npts < 0)) return ORC_EINVAL;
    orc_plan p;
    int st = plan_build(&p, skind, sigma_s, radius, ns_terms, rkind, sigma_r, t_r, 1, ORC_PAPER_3D, data_range);
    if (st) { plan_free(&p); return st; }
    orc_zhaar h;
    st = zhaar_build(&h, rkind, sigma_r, p.Tr, nr_terms, zbins, data_range);
    if (st) { zhaar_free(&h); plan_free(&p); return st; }
    const int R = p.R, w = 2 * R + 1, Z = zbins, Rz = h.Rz;
    const float zs = z_scale(Z, data_range);
    double sk = 0.0;
    for (int i = 0; i < w * w; i++) sk += fabs(p.Ks[i]);
    const double eps = 1e-6 * sk * h.wmax;
    const int n_out = pts ? npts : H * W;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+:bad) num_threads(nthreads > 0 ? nthreads : 1)
    for (int o = 0; o < n_out; o++) {
        int y = pts ? pts[2 * o] : o / W, x = pts ? pts[2 * o + 1] : o % W;
        if (y < 0 || y >= H || x < 0 || x >= W) { out[o] = 0.0; bad++; continue; }
        double ix = I[(size_t)y * W + x], num = 0.0, den = 0.0;
        int nx = z_bin(ix, zs, Z);
        for (int dy = -R; dy <= R; dy++) {
            int yy = y + dy;
            if (yy < 0 || yy >= H) continue;
            for (int dx = -R; dx <= R; dx++) {
                int xx = x + dx;
                if (xx < 0 || xx >= W) continue;
                double iy = I[(size_t)yy * W + xx];
                int d = nx - z_bin(iy, zs, Z);
                if (abs(d) > Rz) continue;
                double ks = p.Ks[(-dy + R) * w + (-dx + R)];
                num += ks * h.w[d + Rz] * iy;
                den += ks * h.w[d + Rz];
            }
        }
        out[o] = den <= eps ? ix : num / den;
        if (den_out) den_out[o] = den;
    }
    zhaar_free(&h);
    plan_free(&p);
    return bad ? ORC_EINVAL : ORC_OK;
}

/* O3-3D with the Haar range series, the paper's steps: per slice z the 2-D box sums of the one-hot
 * auxiliary images F(y, z) = (I(y), 1) [n(y) = z] (Eq. (28), summed-area tables); their running sum
 * along z (the 1-D table of Eq. (29)); then for each kept range term, its pieces as slice windows
 * relative to n(x) (App. A's boxes, in z), each a difference of two entries of the z table. */
int orc_approx3dh_fast(const double *I, int H, int W, int skind, double sigma_s, int radius, int ns_terms,
                       int rkind, double sigma_r, double t_r, int nr_terms, int zbins, double data_range,
                       double *out, int *ndegen, int nthreads)
{
    if (!I || !out || H < 0 || W < 0 || zbins < 2 || !(data_range > 0)) return ORC_EINVAL;
    orc_plan p;
    int st = plan_build(&p, skind, sigma_s, radius, ns_terms, rkind, sigma_r, t_r, 1, ORC_PAPER_3D, data_range);
    if (st) { plan_free(&p); return st; }
    orc_zhaar h;
    st = zhaar_build(&h, rkind, sigma_r, p.Tr, nr_terms, zbins, data_range);
    if (st) { zhaar_free(&h); plan_free(&p); return st; }
    size_t np = (size_t)H * W;
    if (np == 0) { if (ndegen) *ndegen = 0; zhaar_free(&h); plan_free(&p); return ORC_OK; }
    const int Z = zbins;
    const float zs = z_scale(Z, data_range);
    dbox *boxes = malloc(sizeof(dbox) * 16 * p.ns);
    int nb = boxes ? plan_boxes(&p, boxes) : 0;
    double *g = malloc(sizeof(double) * np * 2);
    double *S = malloc(sizeof(double) * (size_t)(H + 1) * (W + 1) * 2);
    double *Pz = malloc(sizeof(double) * np * 2 * (size_t)Z); /* [z][q][pixel]: sum over slices <= z */
    int *nz = malloc(sizeof(int) * np);
    if (!boxes || !g || !S || !Pz || !nz) {
        free(boxes); free(g); free(S); free(Pz); free(nz); zhaar_free(&h); plan_free(&p);
        return ORC_ECAP;
    }
    for (size_t i = 0; i < np; i++) nz[i] = z_bin(I[i], zs, Z);
    int nt = nthreads > 0 ? nthreads : 1;
    for (int z = 0; z < Z; z++) {
        for (size_t i = 0; i < np; i++) {
            int on = nz[i] == z;
            g[i] = on ? I[i] : 0.0;
            g[np + i] = on ? 1.0 : 0.0;
        }
        for (int q = 0; q < 2; q++) sat_build(g + q * np, H, W, S + (size_t)q * (H + 1) * (W + 1));
        double *cur = Pz + (size_t)z * 2 * np, *prev = z > 0 ? Pz + (size_t)(z - 1) * 2 * np : NULL;
#pragma omp parallel for schedule(static) num_threads(nt)
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                size_t i = (size_t)y * W + x;
                for (int q = 0; q < 2; q++) {
                    double b = 0.0;
                    for (int e = 0; e < nb; e++) {
                        const dbox *bx = &boxes[e];
                        b += bx->c * sat_rect(S + (size_t)q * (H + 1) * (W + 1), H, W, x + bx->x0, x + bx->x1,
                                              y + bx->y0, y + bx->y1);
                    }
                    cur[q * np + i] = (prev ? prev[q * np + i] : 0.0) + b;
                }
            }
    }
    double sk = 0.0;
    for (int i = 0; i < (2 * p.R + 1) * (2 * p.R + 1); i++) sk += fabs(p.Ks[i]);
    const double eps = 1e-6 * sk * h.wmax;
    int degen = 0;
#pragma omp parallel for schedule(static) reduction(+:degen) num_threads(nt)
    for (size_t i = 0; i < np; i++) {
        double F[2] = {0.0, 0.0};
        for (int t = 0; t < h.n; t++) {
            drange rr[4];
            int m = haar_ranges(h.lev[t], h.k[t], h.Tz, rr); /* neighbour slice offsets n(y) - n(x) */
            for (int a = 0; a < m; a++) {
                if (rr[a].lo > rr[a].hi) continue;
                int zhi = nz[i] + rr[a].hi, zlo = nz[i] + rr[a].lo - 1;
                if (zhi > Z - 1) zhi = Z - 1;
                for (int q = 0; q < 2; q++) {
                    double top = zhi >= 0 ? Pz[(size_t)zhi * 2 * np + q * np + i] : 0.0;
                    double bot = zlo >= 0 ? Pz[(size_t)(zlo < Z - 1 ? zlo : Z - 1) * 2 * np + q * np + i] : 0.0;
                    F[q] += h.c[t] * rr[a].w * (top - bot);
                }
            }
        }
        if (F[1] <= eps) { out[i] = I[i]; degen++; }
        else out[i] = F[0] / F[1];
    }
    if (ndegen) *ndegen = degen;
    free(boxes); free(g); free(S); free(Pz); free(nz);
    zhaar_free(&h);
    plan_free(&p);
    return ORC_OK;
}

/* The z axis of a plan (for the tests): R_z and the fp32 bin of each listed intensity. */
int orc_z_bins(double t_r_resolved, int zbins, double data_range, const double *I, int n, int *bins_out, int *rz_out)
{
    if (zbins < 2 || !(data_range > 0) || n < 0) return ORC_EINVAL;
    const float zs = z_scale(zbins, data_range);
    for (int i = 0; i < n; i++) bins_out[i] = z_bin(I[i], zs, zbins);
    if (rz_out) *rz_out = z_radius(t_r_resolved, zbins, data_range);
    return ORC_OK;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
