"""Oracle pins for the 3-D form with a Haar series in range: the truncated range kernel's best N-term Haar
expansion on the slice axis (Eqs. (17)-(20) applied to K_r, the selection of Eq. (11)); each kept term is a
pair of boxes along z, so the filter is a sum of 3-D boxes (Eqs. (28)-(29)).

Pins from outside the evaluators: the coefficients against scipy's quadrature of the profile; the full
dictionary reproducing the finest-cell averages of the profile (scipy); box kernels on 8-bit data, where the
expansion is the constant alone and the result is the exact filter O1; the limit N -> all terms against
Eq. (1) with the finest-cell averages of the kernel (scipy), written out here; and the definition O2
against the paper's per-slice steps O3.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_1803_00004_gb300 import synth

D = O.Desc


def on_grid(H, W, seed):
    rng = np.random.default_rng(seed)
    j = np.clip(np.rint(synth.blocks(H, W, seed=seed, noise=0.04) * 255) + rng.integers(-3, 4, (H, W)), 0, 255)
    return (j / 255.0).astype(np.float32)


def profile(kind, sigma_r, step):
    if kind == O.GAUSSIAN:
        return lambda t: math.exp(-(t * step) ** 2 / (2 * sigma_r ** 2))
    if kind == O.EXPONENTIAL:
        return lambda t: math.exp(-abs(t * step) / sigma_r)
    return lambda t: 1.0 if abs(t * step) <= sigma_r else 0.0


def support(lev, k, T):
    """(lo, mid, hi) of a Haar function on [-T, T] (App. A), phi as level -1."""
    if lev < 0:
        return -T, T, T
    Zk = 0.0 if lev == 0 else math.copysign((2 * abs(k) - 1) * T, k)
    s = 2.0 ** -lev
    return s * (Zk - T), s * Zk, s * (Zk + T)


def quad(f, a, b, points):
    pts = [p for p in points if a < p < b]
    return integrate.quad(f, a, b, points=pts or None, epsabs=1e-14, epsrel=1e-13, limit=400)[0] if b > a else 0.0


@pytest.mark.parametrize("kind,sigma_r", [(O.GAUSSIAN, 0.1), (O.EXPONENTIAL, 0.05), (O.BOX, 0.13)])
def test_coefficients_against_quadrature(kind, sigma_r):
    Z = 256
    step = 1.0 / (Z - 1)
    info = O.zhaar_info(D(range=kind, sigma_r=sigma_r, nr_terms=40), Z)
    T = info.Rz + 0.5
    f = profile(kind, sigma_r, step)
    brk = [0.0, sigma_r / step, -sigma_r / step]
    assert len(info.c) >= 15          # the box profile has only 15 non-zero terms
    for lev, k, c in zip(info.lev, info.k, info.c):
        lo, mid, hi = support(lev, k, T)
        if lev < 0:
            ref = quad(f, lo, hi, brk) / (2 * T)
        else:
            ref = 2.0 ** lev * (quad(f, lo, mid, brk) - quad(f, mid, hi, brk)) / (2 * T)
        assert abs(c - ref) < 1e-12, (lev, k, c, ref)
    mags = np.abs(info.c)
    assert np.all(mags[:-1] >= mags[1:] * (1 - 1e-12))   # largest first


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.EXPONENTIAL])
def test_full_dictionary_gives_cell_averages(kind):
    """All 2^(J+1) terms: K~_r at an integer offset is the average of the profile over the finest cell
    holding it (the mean of the two cells' averages where it sits on a cell edge)."""
    Z, sigma_r, t_r = 64, 0.05, 0.1
    step = 1.0 / (Z - 1)
    info = O.zhaar_info(D(range=kind, sigma_r=sigma_r, t_r=t_r, nr_terms=256), Z)
    T = info.Rz + 0.5
    n = 2 ** (info.Jz + 1)
    assert len(info.c) == n - 1       # psi_00 of an even profile vanishes and is never selected
    h = 2 * T / n
    f = profile(kind, sigma_r, step)
    for d in range(-info.Rz, info.Rz + 1):
        u = (d + T) / h
        cells = [int(math.floor(u))] if abs(u - round(u)) > 1e-9 else [int(round(u)) - 1, int(round(u))]
        ref = np.mean([quad(f, -T + m * h, -T + (m + 1) * h, [0.0]) / h for m in cells])
        assert abs(info.w[d + info.Rz] - ref) < 1e-12, d


@pytest.mark.parametrize("H,W,desc,Z", [
    (19, 23, D(sigma_s=1.5, sigma_r=0.1, nr_terms=8), 256),
    (16, 31, D(sigma_s=2.0, sigma_r=0.05, nr_terms=3, range=O.EXPONENTIAL), 64),
    (21, 17, D(sigma_s=1.0, radius=3, ns_terms=9, sigma_r=0.2, nr_terms=16, range=O.BOX), 128),
    (12, 40, D(spatial=O.EXPONENTIAL, sigma_s=1.2, sigma_r=0.08, nr_terms=5), 256),
])
def test_fast_equals_direct(H, W, desc, Z):
    I = synth.blocks(H, W, seed=H + 3 * W, noise=0.08)
    a, _ = O.approx3dh_direct(I, desc, Z)
    b, _ = O.approx3dh_fast(I, desc, Z)
    assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("m", [0, 4, 30])
def test_box_kernels_on_8bit_data_equal_exact_bf(m):
    """Box range kernel of half-width (m + 1/2) / 255: on the slice axis its profile fills [-T_z, T_z], so the
    expansion is the constant alone; with the box spatial kernel and 8-bit data the result is O1."""
    I = on_grid(17, 24, seed=m + 1)
    desc = D(spatial=O.BOX, sigma_s=1.0, radius=2, ns_terms=1, range=O.BOX, sigma_r=(m + 0.5) / 255.0, nr_terms=6)
    info = O.zhaar_info(desc, 256)
    assert list(info.lev) == [-1] and abs(info.c[0] - 1.0) < 1e-14
    got, _ = O.approx3dh_direct(I, desc, 256)
    assert np.max(np.abs(got - O.exact_bf(I, desc))) < 1e-13


def test_gaussian_converges_to_projected_kernel_bf():
    """N -> every term: the weights become the finest-cell averages of the profile (the level-J projection,
    cells of width 2 T_z / 2^(J+1), not centred on the integer offsets), and the result becomes Eq. (1) with
    those weights, written out here with scipy's cell averages; the error falls as N grows."""
    Z, sigma_r, R = 64, 0.08, 2
    step = 1.0 / (Z - 1)
    rng = np.random.default_rng(9)
    I = (np.clip(np.rint(synth.blocks(14, 20, seed=9, noise=0.05) * (Z - 1)) + rng.integers(-2, 3, (14, 20)), 0,
                 Z - 1) / (Z - 1)).astype(np.float32).astype(np.float64)
    info = O.zhaar_info(D(sigma_r=sigma_r, nr_terms=1), Z)
    Rz, T = info.Rz, info.Rz + 0.5
    h = 2 * T / 2 ** (O.haar_levels(T) + 1)
    f = profile(O.GAUSSIAN, sigma_r, step)

    def cell_avg(d):
        u = (d + T) / h
        cells = [int(math.floor(u))] if abs(u - round(u)) > 1e-9 else [int(round(u)) - 1, int(round(u))]
        return np.mean([quad(f, -T + m * h, -T + (m + 1) * h, [0.0]) / h for m in cells])

    wt = {d: cell_avg(d) for d in range(-Rz, Rz + 1)}
    n = np.rint(I * (Z - 1)).astype(int)
    H, W = I.shape
    ref = np.zeros_like(I)
    for y in range(H):
        for x in range(W):
            num = den = 0.0
            for yy in range(max(0, y - R), min(H, y + R + 1)):
                for xx in range(max(0, x - R), min(W, x + R + 1)):
                    d = n[y, x] - n[yy, xx]
                    if abs(d) <= Rz:
                        num += wt[d] * I[yy, xx]
                        den += wt[d]
            ref[y, x] = num / den
    errs = []
    for nr in (2, 8, 24, 64):
        desc = D(spatial=O.BOX, sigma_s=1.0, radius=R, ns_terms=1, sigma_r=sigma_r, nr_terms=nr)
        got, _ = O.approx3dh_direct(I, desc, Z)
        errs.append(np.max(np.abs(got - ref)))
    assert errs[-1] < 1e-12, errs
    assert errs[0] > errs[1] > errs[2] > errs[3], errs
