"""Pre-computation for later range parameters (Sec. V-C, Case 1): bf_precompute stores the box sums of
the basis images once; bf_filter_cached weights them for any plan with the same cosine period, intensity
origin and spatial kernel.  Each cached result must meet the fp32 bar against the oracle and agree with
bf_filter of the same plan.  Needs a GPU."""
import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
from oracle import oracle as O
from paper_1803_00004_gb300 import synth
from parity import conditioned_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00004_gb300 import _build
    _build.build()


@pytest.mark.parametrize("base,sweep", [
    # a fixed truncation T_r = 0.6 fixes P for every sigma_r (the paper's predefined T_ri)
    (dict(sigma_s=4.0, t_r=0.6), [dict(sigma_r=0.05, nr_terms=12), dict(sigma_r=0.1), dict(sigma_r=0.2, nr_terms=6)]),
    # P = dI for every plan of the untruncated policy
    (dict(sigma_s=8.0, ns_terms=9, policy=bf.RANGE_UNTRUNCATED_FULL),
     [dict(sigma_r=0.15, nr_terms=10), dict(sigma_r=0.3, nr_terms=6), dict(sigma_r=0.2, range=bf.KERNEL_EXPONENTIAL)]),
])
def test_cached_filter_matches_oracle_and_filter(base, sweep):
    img = synth.shapes(230, 310, 51, scale=0.2)
    src = torch.from_numpy(img).cuda()
    cache = bf.Cache(bf.Plan(device=0, sigma_r=0.1, **base), src, kmax=32)
    assert cache.nbytes() >= 16 * 32 * img.size
    for kw in sweep:
        kw = dict(base, **kw)
        plan = bf.Plan(device=0, **kw)
        got = torch.full_like(src, float("nan"))
        cache.filter(plan, src, got)
        ref = torch.empty_like(src)
        bf.bf_filter(plan, src, ref)
        torch.cuda.synchronize()
        g = got.cpu().numpy().astype(np.float64)
        e_good, worst, nbad = conditioned_check(g, img, kw)
        assert e_good < TOL and worst < 1.0, (kw, e_good, worst, nbad)
        assert np.max(np.abs(g - ref.cpu().numpy())) < 2 * TOL, kw
    cache.close()


def test_cached_filter_rejects_other_basis_and_missing_frequencies():
    img = synth.blocks(64, 96, 52)
    src = torch.from_numpy(img).cuda()
    dst = torch.empty_like(src)
    cache = bf.Cache(bf.Plan(device=0, sigma_s=4.0, t_r=0.6), src, kmax=8)
    with pytest.raises(bf.BFError) as ei:                      # another T_r: another period P
        cache.filter(bf.Plan(device=0, sigma_s=4.0, t_r=0.5), src, dst)
    assert ei.value.status == 1
    with pytest.raises(bf.BFError) as ei:                      # another spatial kernel
        cache.filter(bf.Plan(device=0, sigma_s=2.0, t_r=0.6), src, dst)
    assert ei.value.status == 1
    with pytest.raises(bf.BFError) as ei:                      # frequencies beyond the cache (kmax 8)
        cache.filter(bf.Plan(device=0, sigma_s=4.0, t_r=0.6, sigma_r=0.05, nr_terms=16), src, dst)
    assert ei.value.status == 8
    cache.close()


@pytest.mark.parametrize("precision,u", [(bf.PREC_FP16, 2.0 ** -11), (bf.PREC_BF16, 2.0 ** -8)])
def test_16bit_cache_within_its_rounding_bound(precision, u):
    """Sums stored in 16 bits carry a relative error of at most u each (one round-to-nearest of the fp32
    sum), so num and den are each off by at most u sum|a_k| (|F_cI| + |F_sI|) <= 2 u sum|a_k| mass, and
    |delta I^| <= 2 u sum|a_k| mass (1 + |I^|) / |den|.  Checked per pixel against the fp64 oracle (plus the
    fp32 bar); the cache is half the size of the fp32 one."""
    from scipy import ndimage
    img = synth.shapes(200, 280, 53, scale=0.2)
    src = torch.from_numpy(img).cuda()
    base = dict(sigma_s=4.0, t_r=0.6)
    c32 = bf.Cache(bf.Plan(device=0, sigma_r=0.2, **base), src, kmax=16)
    c16 = bf.Cache(bf.Plan(device=0, sigma_r=0.2, **base), src, kmax=16, precision=precision)
    assert c16.nbytes() * 2 == c32.nbytes()
    for sr in (0.1, 0.2):
        kw = dict(base, sigma_r=sr)
        plan = bf.Plan(device=0, **kw)
        got = torch.full_like(src, float("nan"))
        c16.filter(plan, src, got)
        torch.cuda.synchronize()
        ref, _, den = O.approx_fast(img.astype(np.float64), O.Desc(**kw), threads=16, return_den=True)
        p = O.plan_info(O.Desc(**kw))
        mass = ndimage.correlate(np.ones(img.shape), np.abs(p.Ks[::-1, ::-1]), mode="constant", cval=0.0)
        bound = TOL + 2 * u * np.sum(np.abs(p.ak)) * mass * (1 + np.abs(ref)) / np.abs(den)
        err = np.abs(got.cpu().numpy() - ref)
        assert np.all(err <= bound), (precision, sr, float(np.max(err / bound)))
    c16.close()
    c32.close()
