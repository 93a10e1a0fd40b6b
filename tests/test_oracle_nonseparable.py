"""Oracle pins for the non-separable radial spatial kernel K_s(x) = exp(-|x|_2 / sigma_s).

Its 2-D Haar coefficients (Eqs. (21)-(22)) are integrals of K_s over rectangles, computed whole
instead of as products of 1-D factors.  The pins come from outside the oracle: scipy's adaptive
cubature for the rectangle integrals, scipy's 1-D quadrature of the polar form for the phi-phi term,
the projection identity (the full dictionary to level J reproduces the finest-cell averages), the
symmetries of a radial kernel, the sigma -> infinity limit, O3 = O2, and hand-written loops for O1.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_1803_00004_gb300 import synth

D = O.Desc


def _k(sigma):
    return lambda y, x: math.exp(-math.hypot(x, y) / sigma)


@pytest.mark.parametrize("rect", [(1.0, 2.0, 3.0, 5.0), (2.0, 9.0, -7.0, -1.0), (0.0, 5.0, 0.0, 5.0),
                                  (-3.0, 0.0, 0.0, 2.5), (0.0, 1e-3, 0.0, 1e-3), (-6.0, -0.25, -1.0, 4.0)])
def test_rectangle_integrals_against_cubature(rect):
    sigma = 3.0
    ref, err = integrate.dblquad(_k(sigma), rect[0], rect[1], rect[2], rect[3], epsabs=1e-15, epsrel=1e-13)
    got = O.rect_int_exp(sigma, *rect)
    assert abs(got - ref) <= 1e-12 * abs(ref) + 1e-15


def test_rectangle_containing_origin_is_sum_of_quadrants():
    # the kink at the origin inside the rectangle: split into four quadrants, each pinned by cubature
    sigma, (x0, x1, y0, y1) = 2.0, (-2.5, 3.0, -1.5, 4.0)
    quads = [(x0, 0.0, y0, 0.0), (0.0, x1, y0, 0.0), (x0, 0.0, 0.0, y1), (0.0, x1, 0.0, y1)]
    ref = sum(integrate.dblquad(_k(sigma), a, b, c, d, epsabs=1e-15, epsrel=1e-13)[0] for a, b, c, d in quads)
    assert abs(O.rect_int_exp(sigma, x0, x1, y0, y1) - ref) <= 1e-12 * ref


@pytest.mark.parametrize("sigma,R", [(1.0, 3), (2.0, 6), (4.0, 12)])
def test_phi_phi_coefficient_by_polar_quadrature(sigma, R):
    """c(phi, phi) = (1/(2T)^2) int over [-T,T]^2 of K_s; by symmetry 8 int_0^{pi/4} F(T / cos t) dt with
    F(rho) = int_0^rho exp(-r / sigma) r dr = sigma^2 - sigma (rho + sigma) exp(-rho / sigma)."""
    T = R + 0.5
    F = lambda rho: sigma * sigma - sigma * (rho + sigma) * math.exp(-rho / sigma)
    ref = 8.0 * integrate.quad(lambda t: F(T / math.cos(t)), 0.0, math.pi / 4, epsabs=0.0, epsrel=1e-13, limit=200)[0]
    c = O.haar2d_exp(sigma, T)
    assert abs(c[0, 0] - ref / (4 * T * T)) <= 1e-13 * abs(c[0, 0])


def test_full_dictionary_reproduces_cell_averages():
    """Summing every 2-D term to level J gives the average of K_s over the finest cell containing the
    point (the level-J Haar projection).  Checked at cell centres against cubature of the cell."""
    sigma, R = 1.5, 3
    T = R + 0.5
    J = O.haar_levels(T)
    n1 = 2 ** (J + 1)
    c = O.haar2d_exp(sigma, T, J)
    _, lev, kk = O.haar1d(O.GAUSSIAN, 1.0, T, J)  # only the dictionary order (levels, shifts) is used
    h = 2 * T / n1
    rng = np.random.default_rng(3)
    for ix, iy in rng.integers(0, n1, size=(12, 2)):
        x, y = -T + (ix + 0.5) * h, -T + (iy + 0.5) * h
        ux = np.array([O.haar_eval(int(lev[i]), int(kk[i]), T, x) for i in range(n1)])
        uy = np.array([O.haar_eval(int(lev[i]), int(kk[i]), T, y) for i in range(n1)])
        val = uy @ c @ ux
        ref = integrate.dblquad(_k(sigma), -T + ix * h, -T + (ix + 1) * h, -T + iy * h, -T + (iy + 1) * h,
                                epsabs=1e-15, epsrel=1e-13)[0] / (h * h)
        assert abs(val - ref) < 1e-12, (ix, iy)


def test_radial_symmetries():
    sigma, T = 2.0, 6.5
    J = O.haar_levels(T)
    c = O.haar2d_exp(sigma, T, J)
    _, lev, kk = O.haar1d(O.GAUSSIAN, 1.0, T, J)
    scale = np.max(np.abs(c))
    assert np.max(np.abs(c - c.T)) <= 1e-14 * scale                     # x <-> y
    # x -> -x maps psi_{j,k} to -psi_{j,-k} (j >= 1), psi_00 to -psi_00, phi to phi
    mirror = np.arange(len(lev))
    sign = np.ones(len(lev))
    for i in range(len(lev)):
        if lev[i] == 0:
            sign[i] = -1.0
        elif lev[i] > 0:
            mirror[i] = next(m for m in range(len(lev)) if lev[m] == lev[i] and kk[m] == -kk[i])
            sign[i] = -1.0
    assert np.max(np.abs(c[:, mirror] * sign[None, :] - c)) <= 1e-14 * scale
    assert np.max(np.abs(c[:, 1])) <= 1e-14 * scale                      # psi_00 terms vanish


def test_infinite_sigma_is_constant_kernel():
    T = 4.5
    c = O.haar2d_exp(1e9, T)
    assert abs(c[0, 0] - 1.0) < 1e-8
    c[0, 0] = 0.0
    assert np.max(np.abs(c)) < 1e-8


@pytest.mark.parametrize("H,W,desc", [
    (17, 21, D(spatial=O.EXPONENTIAL, sigma_s=1.5)),
    (12, 30, D(spatial=O.EXPONENTIAL, sigma_s=2.0, ns_terms=13, nr_terms=6)),
    (9, 9, D(spatial=O.EXPONENTIAL, sigma_s=1.0, radius=5, ns_terms=9, range=O.EXPONENTIAL, sigma_r=0.1)),
])
def test_fast_equals_direct_exponential_spatial(H, W, desc):
    I = synth.uniform(H, W, seed=H * 7 + W)
    a, na = O.approx_direct(I, desc)
    b, nb = O.approx_fast(I, desc)
    assert na == nb
    assert np.max(np.abs(a - b)) < 1e-12


def test_exact_bf_exponential_spatial_brute_force():
    I = synth.uniform(7, 9, seed=5).astype(np.float64)
    sigma_s, R, sigma_r = 1.7, 5, 0.2
    H, W = I.shape
    ref = np.zeros_like(I)
    for y in range(H):
        for x in range(W):
            n = d = 0.0
            for yy in range(max(0, y - R), min(H, y + R + 1)):
                for xx in range(max(0, x - R), min(W, x + R + 1)):
                    w = math.exp(-math.sqrt((yy - y) ** 2 + (xx - x) ** 2) / sigma_s) * \
                        math.exp(-(I[y, x] - I[yy, xx]) ** 2 / (2 * sigma_r ** 2))
                    n += w * I[yy, xx]
                    d += w
            ref[y, x] = n / d
    got = O.exact_bf(I, D(spatial=O.EXPONENTIAL, sigma_s=sigma_s, radius=R, sigma_r=sigma_r))
    assert np.max(np.abs(got - ref)) < 1e-13


def test_selected_terms_are_symmetric_for_five_terms():
    # the five largest terms of a radial kernel: phi phi, then the four level-1 terms (an exact tie group)
    p = O.plan_info(D(spatial=O.EXPONENTIAL, sigma_s=3.0, ns_terms=5))
    Ks = p.Ks
    assert np.max(np.abs(Ks - Ks.T)) < 1e-15 and np.max(np.abs(Ks - Ks[::-1, :])) < 1e-15
