"""Tolerance check shared by the GPU parity tests: the fp32 result against the
fp64 oracle (O(1) evaluation with box sums), conditioned on the denominator."""
import numpy as np

from oracle import oracle as O

THREADS = 16


def conditioned_check(got, img, kw, threads=THREADS):
    """1e-5 max-abs on every pixel whose denominator is >= 1% of the in-window kernel mass
    sum |K~_s|; below that the fp32 rounding of the basis and window sums (~2e-7 relative)
    is amplified by sum|a_k| * mass / |den|, and the bound scales with it."""
    from scipy import ndimage
    ref, _, den = O.approx_fast(img.astype(np.float64), O.Desc(**kw), threads=threads, return_den=True)
    p = O.plan_info(O.Desc(**kw))
    mass = ndimage.correlate(np.ones(img.shape), np.abs(p.Ks[::-1, ::-1]), mode="constant", cval=0.0)
    ratio = np.abs(den) / mass
    err = np.abs(got - ref)
    good = ratio >= 0.01
    assert good.mean() > 0.99, "too many ill-conditioned pixels: %g" % (1 - good.mean())
    e_good = err[good].max() if good.any() else 0.0
    bound = 1e-5 + 2e-7 * np.sum(np.abs(p.ak)) * (1 + np.abs(ref)) / np.maximum(ratio, 1e-12)
    worst = np.max(err[~good] / bound[~good]) if (~good).any() else 0.0
    return e_good, worst, int((~good).sum())
