"""Tolerance check shared by the GPU parity tests: the fp32 result against the
fp64 oracle (O(1) evaluation with box sums), conditioned on the denominator."""
import os

import numpy as np

from oracle import oracle as O

THREADS = max(1, os.cpu_count() or 1)


def window_mass(shape, ks):
    """sum |K~_s(x - y)| over the neighbours y inside the image, per pixel x (zero padding outside).
    Direct correlation for small cases, FFT convolution for large ones (relative error ~1e-13, far
    below the 1 % threshold it is compared with)."""
    from scipy import ndimage, signal
    a = np.abs(ks)
    if a.size * shape[0] * shape[1] <= 4e8:
        return ndimage.correlate(np.ones(shape), a[::-1, ::-1], mode="constant", cval=0.0)
    return signal.fftconvolve(np.ones(shape), a, mode="same")


def conditioned_check(got, img, kw, threads=THREADS, ref_den=None):
    """1e-5 max-abs on every pixel whose denominator is >= 1% of the in-window kernel mass
    sum |K~_s|; below that the fp32 rounding of the basis and window sums (~2e-7 relative)
    is amplified by sum|a_k| * mass / |den|, and the bound scales with it.
    ref_den: the oracle's (output, denominator) when the caller already has them."""
    if ref_den is None:
        ref, _, den = O.approx_fast(img.astype(np.float64), O.Desc(**kw), threads=threads, return_den=True)
    else:
        ref, den = ref_den
    p = O.plan_info(O.Desc(**kw))
    mass = window_mass(img.shape, p.Ks)
    ratio = np.abs(den) / mass
    err = np.abs(got - ref)
    good = ratio >= 0.01
    assert good.mean() > 0.99, "too many ill-conditioned pixels: %g" % (1 - good.mean())
    e_good = err[good].max() if good.any() else 0.0
    bound = 1e-5 + 2e-7 * np.sum(np.abs(p.ak)) * (1 + np.abs(ref)) / np.maximum(ratio, 1e-12)
    worst = np.max(err[~good] / bound[~good]) if (~good).any() else 0.0
    return e_good, worst, int((~good).sum())
