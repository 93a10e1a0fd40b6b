"""Seeded random plans on random ragged images against the oracle: kernels, bandwidths, N_s, N_r, policies,
radii and image sizes drawn at random, each filtered in the default launch geometry and in a randomly chosen
candidate geometry (any family: packed or scalar, ring or not, exchange depth, terms per CTA).  Needs a GPU."""
import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
from paper_1803_00004_gb300 import synth
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00004_gb300 import _build
    _build.build()


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        spatial = int(rng.choice([bf.KERNEL_GAUSSIAN, bf.KERNEL_BOX, bf.KERNEL_EXPONENTIAL]))
        kw = dict(spatial=spatial, sigma_s=float(rng.uniform(0.6, 6.0 if spatial == bf.KERNEL_EXPONENTIAL else 14.0)),
                  ns_terms=int(rng.choice([1, 2, 3, 5, 9, 13])), range=int(rng.integers(0, 3)),
                  sigma_r=float(rng.uniform(0.04, 0.5)), nr_terms=int(rng.integers(1, 17)),
                  policy=int(rng.choice([bf.RANGE_TRUNCATED_MIN_PERIOD, bf.RANGE_UNTRUNCATED_FULL])))
        try:
            bf.Plan(device=-1, **kw)
        except bf.BFError:
            continue
        H, W = int(rng.integers(1, 260)), int(rng.integers(1, 420))
        gen = int(rng.integers(0, 3))
        seed_img = int(rng.integers(0, 1 << 30))
        out.append((H, W, gen, seed_img, int(rng.integers(0, 1 << 30)), kw))
    return out


def _image(H, W, gen, seed):
    if gen == 0:
        return synth.shapes(H, W, seed, scale=max(H, W) / 1080.0)
    if gen == 1:
        return synth.blocks(H, W, seed)
    return synth.uniform(H, W, seed)


@pytest.mark.parametrize("H,W,gen,seed_img,seed_geo,kw", _cases(30, 2026))
def test_random_plan_and_geometry_match_oracle(H, W, gen, seed_img, seed_geo, kw):
    from scipy import ndimage
    img = _image(H, W, gen, seed_img)
    plan = bf.Plan(device=0, **kw)
    # Random plans are often crude (one or two range terms, Gibbs-heavy box kernels) with denominators near
    # cancellation at some pixels, so every pixel is held to the fp32 bar plus the fp32 rounding of the sums
    # (~2e-7 relative) amplified by sum|a_k| mass / |den|: 1e-5 + 2e-7 sum|a_k| (1 + |I^|) mass / |den|.
    # Pixels within 10x of the denominator guard are excluded (fp32 and fp64 may decide the guard
    # differently there).
    ref, _, den = O.approx_fast(img.astype(np.float64), O.Desc(**kw), threads=16, return_den=True)
    p = O.plan_info(O.Desc(**kw))
    mass = ndimage.correlate(np.ones(img.shape), np.abs(p.Ks[::-1, ::-1]), mode="constant", cval=0.0)
    ratio = np.abs(den) / mass
    bound = TOL + 2e-7 * np.sum(np.abs(p.ak)) * (1 + np.abs(ref)) / np.maximum(ratio, 1e-12)
    check = np.abs(den) > 10 * p.den_eps
    src = torch.from_numpy(img).cuda()
    default = bf.bf_launch_info(plan, H, W)
    cands = bf.bf_launch_candidates(plan, H, W)
    pick = cands[np.random.default_rng(seed_geo).integers(0, len(cands))]
    for geo in (None, pick):
        if geo is not None:
            bf.bf_set_launch(plan, H, W, geo)
        dst = torch.full_like(src, float("nan"))
        try:
            bf.bf_filter(plan, src, dst)
            torch.cuda.synchronize()
        finally:
            if geo is not None:
                bf.bf_set_launch(plan, H, W, default)
        got = dst.cpu().numpy().astype(np.float64)
        err = np.abs(got - ref)
        assert np.all(err[check] <= bound[check]), (kw, geo, float(np.max(err[check] / bound[check])))


def _cases3d(n, seed):
    """Random plans of the 3-D form: either range series, slice counts 2..2048, any spatial kernel."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        spatial = int(rng.choice([bf.KERNEL_GAUSSIAN, bf.KERNEL_BOX, bf.KERNEL_EXPONENTIAL]))
        series = int(rng.integers(0, 2))
        kw = dict(spatial=spatial, sigma_s=float(rng.uniform(0.6, 5.0)), ns_terms=int(rng.choice([1, 2, 3, 5, 9])),
                  range=int(rng.integers(0, 3)), sigma_r=float(rng.uniform(0.02, 0.4)),
                  nr_terms=int(rng.integers(1, 13)) if series == 0 else int(rng.integers(1, 65)))
        Z = int(rng.choice([2, 16, 64, 256, 1024, 2048]))
        try:
            bf.Plan(device=-1, policy=bf.RANGE_PAPER_3D, z_bins=Z, range_series=series, **kw)
        except bf.BFError:
            continue
        H, W = int(rng.integers(1, 150)), int(rng.integers(1, 240))
        out.append((H, W, int(rng.integers(0, 3)), int(rng.integers(0, 1 << 30)), int(rng.integers(0, 1 << 30)),
                    series, Z, kw))
    return out


@pytest.mark.parametrize("H,W,gen,seed_img,seed_geo,series,Z,kw", _cases3d(16, 2027))
def test_random_3d_plan_and_geometry_match_oracle(H, W, gen, seed_img, seed_geo, series, Z, kw):
    """As above for the 3-D form: the reference is the definition (O2-3D, or O2-3D with the Haar range table),
    and the bound's mass is the kernel mass inside the pixel's slice window (weighted by |K~_r| for Haar)."""
    img = _image(H, W, gen, seed_img)
    plan = bf.Plan(device=0, policy=bf.RANGE_PAPER_3D, z_bins=Z, range_series=series, **kw)
    d = O.Desc(policy=O.PAPER_3D, **kw)
    # the spatial part and T_r (for the Haar series the cosine terms are not used: plan one of them)
    p = O.plan_info(d if series == 0 else O.Desc(policy=O.PAPER_3D, **dict(kw, nr_terms=1)))
    if series == 0:
        ref, _, den = O.approx3d_direct(img.astype(np.float64), d, Z, threads=16, return_den=True)
        sa = np.sum(np.abs(p.ak))
        rz = O.z_bins([0.0], p.Tr, Z)[1]
        wt = np.ones(2 * rz + 1)
    else:
        ref, den = O.approx3dh_direct(img.astype(np.float64), O.Desc(**kw), Z, threads=16)
        zi = O.zhaar_info(O.Desc(**kw), Z)
        rz, wt, sa = zi.Rz, np.abs(zi.w), 1.0
    bins = O.z_bins(img.astype(np.float64), p.Tr, Z)[0]
    R = p.R
    pb = np.full((H + 2 * R, W + 2 * R), -10 ** 6, dtype=np.int64)
    pb[R:R + H, R:R + W] = bins
    mass = np.zeros((H, W))
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            k = abs(p.Ks[-dy + R, -dx + R])
            if k:
                dd = bins - pb[R + dy:R + dy + H, R + dx:R + dx + W]
                mass += k * np.where(np.abs(dd) <= rz, wt[np.clip(dd + rz, 0, 2 * rz)], 0.0)
    ratio = np.abs(den) / np.maximum(mass, 1e-300)
    bound = TOL + 2e-7 * sa * (1 + np.abs(ref)) / np.maximum(ratio, 1e-12)
    guard = p.den_eps if series == 0 else 1e-6 * np.sum(np.abs(p.Ks)) * np.max(wt)
    check = np.abs(den) > 10 * guard
    src = torch.from_numpy(img).cuda()
    default = bf.bf_launch_info(plan, H, W)
    cands = bf.bf_launch_candidates(plan, H, W)
    pick = cands[np.random.default_rng(seed_geo).integers(0, len(cands))]
    for geo in (None, pick):
        if geo is not None:
            bf.bf_set_launch(plan, H, W, geo)
        dst = torch.full_like(src, float("nan"))
        try:
            bf.bf_filter(plan, src, dst)
            torch.cuda.synchronize()
        finally:
            if geo is not None:
                bf.bf_set_launch(plan, H, W, default)
        got = dst.cpu().numpy().astype(np.float64)
        err = np.abs(got - ref)
        assert np.all(err[check] <= bound[check]), (kw, series, Z, geo, float(np.max(err[check] / bound[check])))


@pytest.mark.parametrize("H,W,gen,seed_img,seed_geo,kw", _cases(12, 2028))
def test_random_plan_with_16bit_basis_within_its_bound(H, W, gen, seed_img, seed_geo, kw):
    """Random plans with the base rotation stored in fp16 or bf16 (alternating by seed), in the default and a
    random geometry: every pixel within the fp32 bound plus the 16-bit storage term 2 u sum m_k |a_k|
    (1 + |I^|) mass / |den|, m_k <= min(k, NK) rotations from an fp32 anchor, u the unit roundoff."""
    from scipy import ndimage
    prec = bf.PREC_FP16 if seed_geo % 2 == 0 else bf.PREC_BF16
    u = 2.0 ** -11 if prec == bf.PREC_FP16 else 2.0 ** -8
    img = _image(H, W, gen, seed_img)
    plan = bf.Plan(device=0, precision=prec, **kw)
    ref, _, den = O.approx_fast(img.astype(np.float64), O.Desc(**kw), threads=16, return_den=True)
    p = O.plan_info(O.Desc(**kw))
    mass = ndimage.correlate(np.ones(img.shape), np.abs(p.Ks[::-1, ::-1]), mode="constant", cval=0.0)
    ratio = np.abs(den) / mass
    ak = np.abs(np.asarray(p.ak))
    ks = np.asarray(p.ks)
    src = torch.from_numpy(img).cuda()
    default = bf.bf_launch_info(plan, H, W)
    cands = bf.bf_launch_candidates(plan, H, W)
    assert cands and all(c["pre"] == (2 if prec == bf.PREC_FP16 else 3) for c in cands)
    pick = cands[np.random.default_rng(seed_geo).integers(0, len(cands))]
    check = np.abs(den) > 10 * plan.coeffs()["den_eps"]
    for geo in (None, pick):
        nk = (geo or default)["nk"]
        coef = 2e-7 * ak.sum() + 2.0 * u * float(np.sum(np.minimum(ks, nk) * ak))
        bound = TOL + coef * (1 + np.abs(ref)) / np.maximum(ratio, 1e-12)
        if geo is not None:
            bf.bf_set_launch(plan, H, W, geo)
        dst = torch.full_like(src, float("nan"))
        try:
            bf.bf_filter(plan, src, dst)
            torch.cuda.synchronize()
        finally:
            if geo is not None:
                bf.bf_set_launch(plan, H, W, default)
        err = np.abs(dst.cpu().numpy().astype(np.float64) - ref)
        assert np.all(err[check] <= bound[check]), (kw, prec, geo, float(np.max(err[check] / bound[check])))
