"""Pins for the oracle's three evaluators (CPU only).

O1 exact_bf, O2 approx_direct (Eq. (1) with the approximated kernels) and O3
approx_fast (the paper's box-filter algorithm).  The checks: O3 reproduces O2
(the decomposition of Eqs. (34)-(36) is exact algebra), closed-form limits,
invariants of Eq. (1), and small brute-force cases written out here.
"""
import math

import numpy as np
import pytest
from scipy import integrate, ndimage

from oracle import oracle as O
from paper_1803_00004_gb300 import synth

D = O.Desc


CASES = [
    # (H, W, desc)
    (24, 31, D()),
    (17, 9, D(sigma_s=2.0, ns_terms=13, sigma_r=0.05, nr_terms=8)),
    (1, 1, D()),
    (1, 13, D(sigma_s=3.0)),
    (11, 1, D(sigma_s=1.5, ns_terms=9)),
    (5, 7, D(sigma_s=4.0, ns_terms=2)),                         # tie group split: asymmetric kernel
    (20, 20, D(sigma_s=3.0, ns_terms=3, nr_terms=5)),           # split tie again
    (16, 18, D(range=O.EXPONENTIAL, sigma_r=0.1, nr_terms=12)),
    (16, 18, D(range=O.BOX, sigma_r=0.2, nr_terms=10)),
    (16, 18, D(policy=O.UNTRUNCATED_FULL, sigma_r=0.2, nr_terms=6)),
    (12, 14, D(spatial=O.BOX, sigma_s=2.0, ns_terms=4)),
    (13, 27, D(sigma_s=2.0, radius=4, ns_terms=25, nr_terms=16, sigma_r=0.07)),
]


@pytest.mark.parametrize("H,W,desc", CASES)
def test_fast_equals_direct(H, W, desc):
    I = synth.uniform(H, W, seed=H * 100 + W)
    a, na = O.approx_direct(I, desc)
    b, nb = O.approx_fast(I, desc)
    assert na == nb
    assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("desc", [D(), D(sigma_s=2.0, ns_terms=13), D(sigma_s=4.0, ns_terms=2),
                                  D(range=O.EXPONENTIAL, nr_terms=6)])
def test_constant_image_is_unchanged(desc):
    I = np.full((19, 23), 0.37)
    for out in (O.exact_bf(I, desc), O.approx_direct(I, desc)[0], O.approx_fast(I, desc)[0]):
        assert np.max(np.abs(out - 0.37)) < 1e-12


def _normalised_correlation(I, K):
    """sum_d K(d) I(x + d) / sum_d K(d) over in-image neighbours (zero padding)."""
    num = ndimage.correlate(I, K, mode="constant", cval=0.0)
    den = ndimage.correlate(np.ones_like(I), K, mode="constant", cval=0.0)
    return num / den


def test_exact_bf_infinite_sigma_r_is_spatial_filter():
    I = synth.uniform(21, 26, seed=3).astype(np.float64)
    desc = D(sigma_s=2.0, sigma_r=1e6)
    R = 6
    d = np.arange(-R, R + 1)
    K = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2 * 2.0 ** 2))
    assert np.max(np.abs(O.exact_bf(I, desc) - _normalised_correlation(I, K))) < 1e-9


def test_approx_infinite_sigma_r_is_approximated_spatial_filter():
    """sigma_r -> infinity: K~_r is constant on [-1, 1] (to ~1e-12), so the approximation is the
    normalised correlation with K~_s(x - y), i.e. with the mirrored kernel table."""
    I = synth.uniform(21, 26, seed=4).astype(np.float64)
    desc = D(sigma_s=2.0, ns_terms=13, sigma_r=1e6, nr_terms=3)
    p = O.plan_info(desc)
    ref = _normalised_correlation(I, p.Ks[::-1, ::-1])
    assert np.max(np.abs(O.approx_fast(I, desc)[0] - ref)) < 1e-9
    # asymmetric (tie-split) kernel: the orientation matters and must still match
    desc = D(sigma_s=2.0, ns_terms=2, sigma_r=1e6, nr_terms=3)
    p = O.plan_info(desc)
    assert p.tie_split
    ref = _normalised_correlation(I, p.Ks[::-1, ::-1])
    assert np.max(np.abs(O.approx_direct(I, desc)[0] - ref)) < 1e-9
    assert np.max(np.abs(O.approx_fast(I, desc)[0] - ref)) < 1e-9


def test_exact_bf_local_min_max():
    I = synth.blocks(32, 32, seed=5).astype(np.float64)
    out = O.exact_bf(I, D(sigma_s=2.0, sigma_r=0.1))
    mx = ndimage.maximum_filter(I, size=13, mode="nearest")
    mn = ndimage.minimum_filter(I, size=13, mode="nearest")
    assert np.all(out <= mx + 1e-12) and np.all(out >= mn - 1e-12)


def _bf_loops(I, sigma_s, R, sigma_r):
    H, W = I.shape
    out = np.zeros_like(I)
    for y in range(H):
        for x in range(W):
            n = d = 0.0
            for yy in range(max(0, y - R), min(H, y + R + 1)):
                for xx in range(max(0, x - R), min(W, x + R + 1)):
                    w = math.exp(-((yy - y) ** 2 + (xx - x) ** 2) / (2 * sigma_s ** 2)) * \
                        math.exp(-(I[y, x] - I[yy, xx]) ** 2 / (2 * sigma_r ** 2))
                    n += w * I[yy, xx]
                    d += w
            out[y, x] = n / d
    return out


@pytest.mark.parametrize("H,W", [(1, 1), (2, 2), (8, 8), (3, 11)])
def test_exact_bf_tiny_brute_force(H, W):
    I = synth.uniform(H, W, seed=H + W).astype(np.float64)
    assert np.max(np.abs(O.exact_bf(I, D(sigma_s=2.0, sigma_r=0.15)) - _bf_loops(I, 2.0, 6, 0.15))) < 1e-13


def test_exact_bf_row_subset():
    I = synth.uniform(15, 12, seed=9).astype(np.float64)
    full = O.exact_bf(I, D(sigma_s=1.0))
    rows = [0, 7, 14]
    assert np.array_equal(O.exact_bf(I, D(sigma_s=1.0), rows=rows), full[rows])


def test_box_spatial_untruncated_range_converges_to_exact():
    """Box spatial kernel: the Haar expansion is exact with one term (phi phi).  Range kernel
    untruncated on [-1, 1] with sigma_r = 0.12 (the Gaussian is 1e-15 at |t| = 1): 40 cosine
    terms reproduce it to ~1e-13.  So O2/O3 must equal O1 with the same kernels."""
    I = synth.blocks(20, 24, seed=2).astype(np.float64)
    desc = D(spatial=O.BOX, sigma_s=1.0, radius=3, ns_terms=1, sigma_r=0.12, nr_terms=40, policy=O.UNTRUNCATED_FULL)
    ex = O.exact_bf(I, desc)
    assert np.max(np.abs(O.approx_fast(I, desc)[0] - ex)) < 1e-10
    assert np.max(np.abs(O.approx_direct(I, desc)[0] - ex)) < 1e-10


def test_full_haar_dictionary_gives_cell_averages():
    """All Haar terms to level J: K~_s(d) = a(dx) a(dy), a(d) = average of the 1-D Gaussian over
    the level-J cell containing d (mean of the two neighbouring cells at d = 0)."""
    sigma, R = 1.5, 4
    T = R + 0.5
    J = O.haar_levels(T)
    n1 = 2 ** (J + 1)
    p = O.plan_info(D(sigma_s=sigma, radius=R, ns_terms=n1 * n1))
    h = 2 * T / n1
    f = lambda x: math.exp(-x * x / (2 * sigma * sigma))
    cell = lambda i: integrate.quad(f, -T + i * h, -T + (i + 1) * h, epsabs=1e-15)[0] / h

    def avg(d):
        i = (d + T) / h
        if abs(i - round(i)) < 1e-12:
            return 0.5 * (cell(int(round(i)) - 1) + cell(int(round(i))))
        return cell(int(math.floor(i)))

    a = np.array([avg(d) for d in range(-R, R + 1)])
    # dropped coefficients (< 1e-14 of the largest) bound the residual
    assert np.max(np.abs(p.Ks - np.outer(a, a))) < 1e-13


def test_transpose_invariance():
    I = synth.blocks(18, 25, seed=7).astype(np.float64)
    desc = D(sigma_s=2.0, ns_terms=13, nr_terms=8)
    a = O.approx_fast(I, desc)[0]
    b = O.approx_fast(np.ascontiguousarray(I.T), desc)[0]
    assert np.max(np.abs(a - b.T)) < 1e-12


def test_accuracy_improves_with_spatial_terms():
    """Convergence in N_s along the ranked order, at complete tie groups (1, 5, 9, 13, 25 terms)."""
    I = synth.blocks(48, 48, seed=0).astype(np.float64)
    ex = O.exact_bf(I, D(sigma_s=2.0, sigma_r=0.1))
    errs = []
    for ns in (1, 5, 13, 25):
        out = O.approx_fast(I, D(sigma_s=2.0, ns_terms=ns, sigma_r=0.1, nr_terms=16, policy=O.UNTRUNCATED_FULL))[0]
        errs.append(np.mean((out - ex) ** 2))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))


def test_direct_at_points_matches_full():
    I = synth.shapes(30, 41, seed=3, scale=0.05).astype(np.float64)
    desc = D(sigma_s=2.0, ns_terms=13)
    full, _ = O.approx_direct(I, desc)
    pts = np.array([[0, 0], [29, 40], [15, 7], [3, 39], [29, 0]])
    assert np.array_equal(O.approx_direct_at(I, desc, pts), full[pts[:, 0], pts[:, 1]])


def test_fast_denominator_is_eq1_denominator():
    """The denominator O3 reports equals the direct sum of K~_s K~_r over the window."""
    I = synth.uniform(9, 11, seed=5).astype(np.float64)
    desc = D(sigma_s=1.0)
    _, _, den = O.approx_fast(I, desc, return_den=True)
    p = O.plan_info(desc)
    R = p.R
    y, x = 4, 6
    s = 0.0
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            if 0 <= y + dy < 9 and 0 <= x + dx < 11:
                t = I[y, x] - I[y + dy, x + dx]
                s += p.Ks[-dy + R, -dx + R] * np.sum(p.ak * np.cos(np.pi * p.ks * t / p.P))
    assert abs(den[y, x] - s) < 1e-12


# --- the look-up-table brute force (Sec. V, Case 2) -------------------------------------------------------------

@pytest.mark.parametrize("desc", [D(sigma_s=1.5, sigma_r=0.1), D(sigma_s=2.0, sigma_r=0.05, range=O.EXPONENTIAL),
                                  D(spatial=O.EXPONENTIAL, sigma_s=1.0, sigma_r=0.2), D(sigma_s=1.0, range=O.BOX,
                                                                                          sigma_r=0.3)])
def test_lut_exact_on_grid_valued_images(desc):
    """Values on the table's grid (k / 256 with 257 levels over [0, 1]): every difference is a grid point,
    so the table holds the kernel's exact values there and the result is O1's."""
    I = np.round(synth.uniform(19, 26, seed=4).astype(np.float64) * 256) / 256
    assert np.max(np.abs(O.exact_bf_lut(I, desc, 257) - O.exact_bf(I, desc))) < 1e-15


def test_lut_converges_to_exact():
    """Off-grid data: the nearest entry is within step / 2 of |t|, so each range weight is within
    max|K_r'| step / 2 of the exact one; the error shrinks with the step."""
    I = synth.uniform(17, 23, seed=5).astype(np.float64)
    desc = D(sigma_s=1.5, sigma_r=0.1)
    errs = [np.max(np.abs(O.exact_bf_lut(I, desc, n) - O.exact_bf(I, desc))) for n in (64, 256, 1024, 1 << 16)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    slope = math.exp(-0.5) / 0.1                  # max |d/dt exp(-t^2 / (2 sigma^2))| = 1 / (sigma sqrt(e))
    assert errs[-1] < 2 * slope * (1.0 / ((1 << 16) - 1))
