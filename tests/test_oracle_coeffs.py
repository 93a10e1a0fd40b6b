"""Pins for the oracle's coefficient and selection steps (CPU only).

Each test checks the oracle against something other than itself: closed forms
from the mathematics, independent numerical quadrature (scipy), structural
identities of the Haar system, or values printed in the paper (tests/golden).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import wofz

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Range coefficients, Eqs. (13)-(15)
# --------------------------------------------------------------------------

def gauss_cos_integral(sigma, T, omega):
    """int_{-T}^{T} exp(-t^2/(2 s^2)) cos(w t) dt in closed form.

    = s sqrt(2 pi) Re[exp(-w^2 s^2 / 2) erf((T + i w s^2) / (s sqrt 2))], written with the
    Faddeeva function w(z) (erf(z) = 1 - exp(-z^2) w(i z)) so that it stays finite.
    """
    z = (T + 1j * omega * sigma * sigma) / (sigma * math.sqrt(2.0))
    val = np.exp(-(omega * sigma) ** 2 / 2.0) - np.exp(-T * T / (2 * sigma * sigma) - 1j * T * omega) * wofz(1j * z)
    return sigma * math.sqrt(2 * math.pi) * np.real(val)


@pytest.mark.parametrize("sigma,T,P", [(0.1, 0.3, 0.65), (0.05, 0.15, 0.575), (0.3, 0.9, 0.95), (40.0, 120.0, 120.0)])
def test_gaussian_range_coeffs_closed_form(sigma, T, P):
    n = 64
    a = O.range_coeffs(O.GAUSSIAN, sigma, T, P, n)
    k = np.arange(n)
    ref = gauss_cos_integral(sigma, T, math.pi * k / P) / P
    ref[0] /= 2.0
    assert np.max(np.abs(a - ref)) < 1e-14


@pytest.mark.parametrize("sigma,P", [(0.05, 0.615), (0.1, 0.73), (0.2, 1.0)])
def test_exponential_range_coeffs_closed_form(sigma, P):
    T = sigma * math.log(100.0)
    n = 48
    a = O.range_coeffs(O.EXPONENTIAL, sigma, T, P, n)
    k = np.arange(n)
    w = math.pi * k / P
    al = 1.0 / sigma
    # int_0^T e^{-t/s} cos(w t) dt = (al - e^{-al T}(al cos wT - w sin wT)) / (al^2 + w^2)
    half = (al - np.exp(-al * T) * (al * np.cos(w * T) - w * np.sin(w * T))) / (al * al + w * w)
    ref = 2.0 * half / P
    ref[0] /= 2.0
    assert np.max(np.abs(a - ref)) < 1e-14


def test_box_range_coeffs_closed_form():
    s, P = 0.2, 0.6
    a = O.range_coeffs(O.BOX, s, s, P, 40)
    k = np.arange(1, 40)
    assert abs(a[0] - s / P) < 1e-15
    assert np.max(np.abs(a[1:] - 2 * np.sin(math.pi * k * s / P) / (math.pi * k))) < 1e-14


def test_gaussian_untruncated_is_fourier_transform_sample():
    """A Gaussian that has vanished long before P: a_k = (s sqrt(2 pi)/P) exp(-(pi k s/P)^2/2)."""
    s, P = 0.05, 1.0
    a = O.range_coeffs(O.GAUSSIAN, s, P, P, 40)
    k = np.arange(40)
    ref = s * math.sqrt(2 * math.pi) / P * np.exp(-((math.pi * k * s / P) ** 2) / 2)
    ref[0] /= 2
    assert np.max(np.abs(a - ref)) < 1e-15


def test_range_series_parseval_and_reproduction():
    """Untruncated Gaussian that has vanished (to 1e-15) at the period boundary:
    Parseval and pointwise reproduction on [-1, 1]."""
    s, P = 0.12, 1.0
    a = O.range_coeffs(O.GAUSSIAN, s, P, P, 60)
    energy, _ = integrate.quad(lambda t: math.exp(-t * t / (s * s)), -P, P, epsabs=1e-15)
    assert abs(2 * P * a[0] ** 2 + P * np.sum(a[1:] ** 2) - energy) < 1e-13
    t = np.linspace(-1, 1, 401)
    ser = sum(a[k] * np.cos(math.pi * k * t / P) for k in range(60))
    assert np.max(np.abs(ser - np.exp(-t * t / (2 * s * s)))) < 1e-13


def test_truncated_series_converges_inside_support():
    """Truncated at T_r, period P = (1 + T_r)/2: far from the jumps the series tends to K_r,
    and it is ~0 between T_r and 2P - T_r (no alias copy inside the data range)."""
    s = 0.1
    T = 3 * s
    P = O.period(O.TRUNCATED_MIN_PERIOD, T, 1.0)
    assert abs(P - 0.65) < 1e-15
    a = O.range_coeffs(O.GAUSSIAN, s, T, P, 400)
    t_in = np.linspace(-0.2, 0.2, 81)
    t_out = np.linspace(0.4, 0.9, 51)  # the next copy starts at 2P - T_r = 1.0
    k = np.arange(400)
    f = lambda t: np.cos(math.pi * np.outer(t, k) / P) @ a
    assert np.max(np.abs(f(t_in) - np.exp(-t_in ** 2 / (2 * s * s)))) < 2e-4
    assert np.max(np.abs(f(t_out))) < 2e-4


def test_period_policies():
    assert O.period(O.UNTRUNCATED_FULL, 0.3, 1.0) == 1.0
    assert O.period(O.PAPER_TRUNCATED, 0.3, 1.0) == 0.3
    assert abs(O.period(O.TRUNCATED_MIN_PERIOD, 0.3, 1.0) - 0.65) < 1e-15
    assert O.period(O.TRUNCATED_MIN_PERIOD, 1.5, 1.0) == 1.5  # P >= T_r
    assert abs(O.default_tr(O.GAUSSIAN, 0.1) - 0.3) < 1e-15
    assert abs(O.default_tr(O.EXPONENTIAL, 0.1) - 0.1 * math.log(100)) < 1e-15


def test_table_vii_range_row():
    """Table VII: the N largest cosine coefficients of G_40 lie in the first M = 2,2,3,...,8
    (ranking by raw |a_k|, k = 0 a candidate, series on [-T_r, T_r])."""
    g = json.load(open(os.path.join(GOLD, "table_vii_nm.json")))["range_kernel"]
    sigma = g["sigma"]
    for T in (3 * sigma, sigma * math.sqrt(2 * math.log(100.0))):
        a = O.range_coeffs(O.GAUSSIAN, sigma, T, T, 20 * 8)
        got = []
        for N in g["N"]:
            ks, _ = O.select_range(a[:20 * N], N)
            got.append(int(ks.max()) + 1)
        assert got == g["M"]


def test_range_selection_order_and_ties():
    a = np.array([0.2, -0.5, 0.5 * (1 + 1e-14), 0.1, 1e-20])
    ks, aks = O.select_range(a, 5)
    assert list(ks[:2]) == [1, 2]          # tie within 1e-12 -> smaller k first
    assert list(ks) == [1, 2, 0, 3]        # 1e-20 < 1e-14 * max is never selected
    assert aks[0] == -0.5


# --------------------------------------------------------------------------
# Haar system, Eqs. (17)-(22)
# --------------------------------------------------------------------------

def test_haar_dictionary_layout():
    T = 12.5
    J = O.haar_levels(T)
    assert J == 5  # ceil(log2(25))
    c, lev, kk = O.haar1d(O.GAUSSIAN, 4.0, T)
    assert len(c) == 2 ** (J + 1)
    assert lev[0] == -1 and lev[1] == 0 and kk[1] == 0
    for j in range(1, J + 1):
        ks = sorted(kk[lev == j])
        assert ks == list(range(-2 ** (j - 1), 0)) + list(range(1, 2 ** (j - 1) + 1))


def test_haar_function_values():
    T = 2.0
    ev = O.haar_eval
    assert ev(-1, 0, T, 0.0) == 1 and ev(-1, 0, T, 1.99) == 1 and ev(-1, 0, T, 2.5) == 0
    assert ev(0, 0, T, -1.0) == 1 and ev(0, 0, T, 1.0) == -1 and ev(0, 0, T, 0.0) == 0
    # psi_{1,-1}(x) = psi_00(2x + T): +1 on [-T, -T/2), -1 on (-T/2, 0]
    assert ev(1, -1, T, -1.5) == 1 and ev(1, -1, T, -0.5) == -1 and ev(1, -1, T, 0.5) == 0
    # psi_{2,2}(x) = psi_00(4x - 3T): support [T/2, T]
    assert ev(2, 2, T, 1.2) == 1 and ev(2, 2, T, 1.7) == -1 and ev(2, 2, T, 0.9) == 0
    # mean of one-sided limits at the ends touching 0
    assert ev(1, 1, T, 0.0) == 0.5 and ev(1, -1, T, 0.0) == -0.5


def _haar_support(lev, k, T):
    if lev < 0:
        return -T, T, T
    Z = 0.0 if lev == 0 else math.copysign(1, k) * (2 * abs(k) - 1) * T
    s = 2.0 ** -lev
    return s * (Z - T), s * Z, s * (Z + T)


@pytest.mark.parametrize("sigma,T", [(4.0, 12.5), (2.0, 6.5), (8.0, 24.5)])
def test_haar_coeffs_match_quadrature(sigma, T):
    c, lev, kk = O.haar1d(O.GAUSSIAN, sigma, T)
    f = lambda x: math.exp(-x * x / (2 * sigma * sigma))
    for idx in list(range(12)) + [len(c) - 1, len(c) // 2 + 3]:
        lo, mid, hi = _haar_support(lev[idx], kk[idx], T)
        if lev[idx] < 0:
            ref = integrate.quad(f, lo, hi, epsabs=1e-15)[0] / (2 * T)
        else:
            ip = integrate.quad(f, lo, mid, epsabs=1e-15)[0] - integrate.quad(f, mid, hi, epsabs=1e-15)[0]
            ref = 2.0 ** lev[idx] * ip / (2 * T)
        assert abs(c[idx] - ref) < 1e-13, idx


@pytest.mark.parametrize("sigma,T", [(4.0, 12.5), (3.0, 9.5)])
def test_haar_full_expansion_is_cell_average(sigma, T):
    """Eq. (20) truncated at level J is the orthogonal projection onto piecewise constants on
    2^{J+1} equal cells: evaluated at each cell centre it equals the cell average of f."""
    c, lev, kk = O.haar1d(O.GAUSSIAN, sigma, T)
    J = O.haar_levels(T)
    ncell = 2 ** (J + 1)
    h = 2 * T / ncell
    f = lambda x: math.exp(-x * x / (2 * sigma * sigma))
    for i in range(ncell):
        x = -T + (i + 0.5) * h
        rec = sum(c[t] * O.haar_eval(int(lev[t]), int(kk[t]), T, x) for t in range(len(c)))
        avg = integrate.quad(f, -T + i * h, -T + (i + 1) * h, epsabs=1e-15)[0] / h
        assert abs(rec - avg) < 1e-13


def test_haar_parseval():
    sigma, T = 4.0, 12.5
    c, lev, kk = O.haar1d(O.GAUSSIAN, sigma, T)
    J = O.haar_levels(T)
    norms = np.where(lev <= 0, 2 * T, 2 * T / 2.0 ** np.maximum(lev, 0))
    ncell = 2 ** (J + 1)
    h = 2 * T / ncell
    f = lambda x: math.exp(-x * x / (2 * sigma * sigma))
    avgs = np.array([integrate.quad(f, -T + i * h, -T + (i + 1) * h)[0] / h for i in range(ncell)])
    assert abs(np.sum(c * c * norms) - h * np.sum(avgs ** 2)) < 1e-12


def test_sec5a_top5_terms_and_three_box_shapes():
    g = json.load(open(os.path.join(GOLD, "sec5a_top5_haar.json")))
    for sigma in (2.0, 4.0, 8.0, 32.0):
        p = O.plan_info(O.Desc(sigma_s=sigma, ns_terms=5))
        assert [list(t) for t in p.terms] == g["terms"]
        assert not p.tie_split
        # box shapes (App. A): phi piece length 2T, level-j piece length T/2^j
        size = lambda lv: 2 * p.Ts if lv < 0 else p.Ts / 2 ** lv
        shapes = {(size(t[0]), size(t[2])) for t in p.terms}
        assert len(shapes) == g["box_shapes"]


def test_table_vii_spatial_n1_is_phi_phi():
    g = json.load(open(os.path.join(GOLD, "table_vii_nm.json")))["spatial_kernel"]
    p = O.plan_info(O.Desc(sigma_s=g["sigma"], ns_terms=1))
    assert list(p.terms[0]) == [-1, 0, -1, 0]


def test_tie_split_reported():
    p = O.plan_info(O.Desc(sigma_s=4.0, ns_terms=3))
    assert p.tie_split
    p = O.plan_info(O.Desc(sigma_s=4.0, ns_terms=9))
    assert not p.tie_split


def test_kernel_table_is_sum_of_selected_terms():
    """K~_s from the plan equals the separable sum written out here from the selected terms."""
    p = O.plan_info(O.Desc(sigma_s=4.0, ns_terms=13))
    R = p.R
    K = np.zeros((2 * R + 1, 2 * R + 1))
    for (l1, k1, l2, k2), c in zip(p.terms, p.term_c):
        ux = np.array([O.haar_eval(int(l1), int(k1), p.Ts, d) for d in range(-R, R + 1)])
        uy = np.array([O.haar_eval(int(l2), int(k2), p.Ts, d) for d in range(-R, R + 1)])
        K += c * np.outer(uy, ux)
    assert np.max(np.abs(K - p.Ks)) < 1e-15
    # the symmetric selection gives a kernel symmetric in both axes and under transpose
    assert np.allclose(K, K[::-1, :], atol=1e-15) and np.allclose(K, K[:, ::-1], atol=1e-15)
    assert np.allclose(K, K.T, atol=1e-15)
