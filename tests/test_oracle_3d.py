"""Oracle pins for the 3-D form of Sec. IV-D (cosine half-period P = T_r, range box by dimension promotion).

The pins come from outside the 3-D evaluators: the exact bilateral filter O1 with box kernels on 8-bit
(on-grid) data, where the slice window is exactly the range box; the limit N_r -> infinity, where the
cosine series of period 2 T_r times the box is the truncated range kernel (checked against Eq. (1) with
K_r(t) [|t| <= T_r] written out here); the collapsed form O3 when T_r >= dI (every neighbour is inside
the window and both policies give P = T_r); and the two 3-D evaluators against each other (the
definition O2-3D and the paper's per-slice steps O3-3D).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1803_00004_gb300 import synth

D = O.Desc


def on_grid(H, W, seed, levels=256):
    """8-bit data: integer levels j / (levels - 1) stored as fp32 (the stand-in for 8-bit photographs)."""
    rng = np.random.default_rng(seed)
    base = synth.blocks(H, W, seed=seed, noise=0.04)
    j = np.clip(np.rint(base * (levels - 1)) + rng.integers(-3, 4, (H, W)), 0, levels - 1)
    return (j / (levels - 1)).astype(np.float32)


@pytest.mark.parametrize("H,W,desc,Z", [
    (19, 23, D(sigma_s=1.5, sigma_r=0.1, nr_terms=6, policy=O.PAPER_3D), 64),
    (16, 31, D(sigma_s=2.0, sigma_r=0.05, nr_terms=4, policy=O.PAPER_3D), 256),
    (21, 17, D(sigma_s=1.0, radius=4, ns_terms=9, range=O.EXPONENTIAL, sigma_r=0.08, nr_terms=7,
               policy=O.PAPER_3D), 32),
    (12, 40, D(spatial=O.BOX, sigma_s=1.0, radius=3, ns_terms=1, sigma_r=0.2, nr_terms=5, policy=O.PAPER_3D), 16),
])
def test_fast_equals_direct_3d(H, W, desc, Z):
    I = synth.blocks(H, W, seed=H + W, noise=0.08)
    a, na = O.approx3d_direct(I, desc, Z)
    b, nb = O.approx3d_fast(I, desc, Z)
    assert na == nb
    assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("m", [0, 3, 20])
def test_box_kernels_on_8bit_data_equal_exact_bf(m):
    """Box spatial kernel (one Haar term: the constant) and box range kernel of half-width (m + 1/2) / 255:
    the cosine series of a constant on [-T_r, T_r] is a_0 = 1 alone, and on 8-bit data the slice window
    |n(y) - n(x)| <= m is exactly |I(y) - I(x)| <= T_r.  So the 3-D form is O1 with box kernels."""
    I = on_grid(18, 26, seed=m)
    sr = (m + 0.5) / 255.0
    desc = D(spatial=O.BOX, sigma_s=1.0, radius=3, ns_terms=1, range=O.BOX, sigma_r=sr, nr_terms=4,
             policy=O.PAPER_3D)
    info = O.plan_info(desc)
    assert len(info.ks) == 1 and info.ks[0] == 0 and abs(info.ak[0] - 1.0) < 1e-14
    got, nd = O.approx3d_fast(I, desc, 256)
    ref = O.exact_bf(I, desc)
    assert nd == 0
    assert np.max(np.abs(got - ref)) < 1e-13


def _truncated_bf(I, R, sigma_r, T_r):
    """Eq. (1) with the box spatial kernel on the (2R+1)^2 square and K_r(t) = exp(-t^2 / (2 sigma_r^2)) for
    |t| <= T_r, 0 beyond."""
    I = I.astype(np.float64)
    H, W = I.shape
    out = np.zeros_like(I)
    for y in range(H):
        for x in range(W):
            win = I[max(0, y - R):y + R + 1, max(0, x - R):x + R + 1]
            t = I[y, x] - win
            k = np.where(np.abs(t) <= T_r, np.exp(-t * t / (2 * sigma_r ** 2)), 0.0)
            out[y, x] = np.sum(k * win) / np.sum(k)
    return out


def test_gaussian_range_converges_to_truncated_bf():
    """As N_r grows the cosine series of period 2 T_r converges to the Gaussian on [-T_r, T_r] (its periodic
    extension is continuous), and on 8-bit data the slice window is the box |t| <= T_r: the 3-D form tends
    to Eq. (1) with the truncated range kernel."""
    I = on_grid(14, 20, seed=7)
    sigma_r, T_r, R = 0.08, 24.5 / 255.0, 2
    ref = _truncated_bf(I, R, sigma_r, T_r)
    errs = []
    for nr in (2, 4, 8, 16):
        desc = D(spatial=O.BOX, sigma_s=1.0, radius=R, ns_terms=1, sigma_r=sigma_r, t_r=T_r, nr_terms=nr,
                 policy=O.PAPER_3D)
        got, _ = O.approx3d_fast(I, desc, 256)
        errs.append(np.max(np.abs(got - ref)))
    assert errs[-1] < 1e-4, errs
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < errs[0] / 20, errs


def test_wide_truncation_reduces_to_collapsed_form():
    """T_r >= dI: both policies take P = T_r and every neighbour lies inside the slice window."""
    I = synth.blocks(17, 22, seed=3, noise=0.1)
    common = dict(sigma_s=1.5, sigma_r=0.4, t_r=1.25, nr_terms=8)
    a, _ = O.approx3d_fast(I, D(policy=O.PAPER_3D, **common), 256)
    b, _ = O.approx_fast(I, D(policy=O.TRUNCATED_MIN_PERIOD, **common))
    assert O.plan_info(D(policy=O.PAPER_3D, **common)).P == O.plan_info(D(**common)).P == 1.25
    assert np.max(np.abs(a - b)) < 1e-13


def test_narrow_window_keeps_only_the_same_slice():
    """R_z = 0: only neighbours of the centre's own slice count.  With one slice per intensity present the
    output is then the centre pixel itself wherever no neighbour shares its slice."""
    I = np.array([[0.0, 0.5, 1.0], [0.25, 0.75, 0.5], [1.0, 0.0, 0.25]], dtype=np.float32)
    desc = D(spatial=O.BOX, sigma_s=1.0, radius=1, ns_terms=1, range=O.BOX, sigma_r=0.001, nr_terms=1,
             policy=O.PAPER_3D)
    bins, rz = O.z_bins(I, 0.001, 256)
    assert rz == 0
    got, _ = O.approx3d_fast(I, desc, 256)
    # pixel (1, 1) = 0.75: no neighbour shares its slice -> itself; (0, 1) = 0.5 shares with (1, 2)
    assert got[1, 1] == pytest.approx(0.75, abs=1e-15)
    assert got[0, 1] == pytest.approx(0.5, abs=1e-15)


def test_slice_rule():
    """Nearest of the Z levels, decided in fp32, clamped; R_z = floor(T_r (Z - 1) / dI)."""
    j = np.arange(256)
    bins, rz = O.z_bins((j / 255.0).astype(np.float32), 0.3, 256)
    assert np.array_equal(bins, j) and rz == 76
    _, rz = O.z_bins([0.5], 10 / 255.0, 256)
    assert rz == 10                                   # a whole number of levels is not lost to rounding
    bins, _ = O.z_bins(np.array([-0.2, 1.3, 0.0, 1.0]), 0.1, 256)
    assert list(bins) == [0, 255, 0, 255]             # clamped to the axis
    bins, rz = O.z_bins(np.array([0.2, 0.49, 0.51]), 0.25, 3)
    assert list(bins) == [0, 1, 1] and rz == 0        # three levels 0, 1/2, 1


@pytest.mark.parametrize("series", [0, 1])
def test_pointwise_evaluators_equal_the_whole_image(series):
    """The pointwise forms the full-size GPU tests sample with (O2-3D at chosen pixels, and the Haar series'
    definition with `pts`) give exactly the whole-image definition's values there, image corners included."""
    I = synth.blocks(23, 31, seed=5, noise=0.08)
    rng = np.random.default_rng(3)
    pts = np.concatenate([np.stack([rng.integers(0, 23, 40), rng.integers(0, 31, 40)], 1),
                          [[0, 0], [22, 30], [0, 30], [22, 0]]])
    if series == 0:
        desc = D(sigma_s=2.0, sigma_r=0.1, nr_terms=6, policy=O.PAPER_3D)
        whole, _, den = O.approx3d_direct(I, desc, 64, return_den=True)
        at, den_at = O.approx3d_direct_at(I, desc, pts, 64)
        assert np.max(np.abs(den_at - den[pts[:, 0], pts[:, 1]])) < 1e-12
    else:
        desc = D(sigma_s=2.0, sigma_r=0.1, nr_terms=12)
        whole, _ = O.approx3dh_direct(I, desc, 64)
        at, _ = O.approx3dh_direct(I, desc, 64, pts=pts)
    assert np.max(np.abs(np.asarray(at).ravel() - whole[pts[:, 0], pts[:, 1]])) < 1e-13
