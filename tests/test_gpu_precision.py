"""The basis pre-pass and the 16-bit basis storage modes against the FP64 oracle (needs a GPU).

fp32 plans may read the pixel and its base rotation (cos, sin)(pi t) from an fp32 pre-pass buffer instead of
computing a sincospi at every window edge: the same values, so the same 1e-5 bar.  fp16 / bf16 plans store the
base rotation in 16 bits.  A stored pair rounded to unit roundoff u (2^-11 fp16, 2^-8 bf16) and rescaled to unit
length is off by an angle of at most u, and term k of a group is reached from an fp32 anchor by m_k <= min(k, NK)
rotations, so its basis phase at a pixel is off by at most m_k u.  In Eq. (34) the centre's and the neighbour's
phases enter as a difference: each term of numerator and denominator moves by at most 2 m_k u |a_k| times the
window's |K~_s| mass, which gives
    |I^ - I^_oracle| <= 1e-5 + (2e-7 sum|a_k| + 2 u sum m_k |a_k|) (1 + |I^|) mass / |den|.
"""
import os

import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
from oracle import oracle as O
from paper_1803_00004_gb300 import synth
from parity import window_mass

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)
U = {bf.PREC_FP16: 2.0 ** -11, bf.PREC_BF16: 2.0 ** -8}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00004_gb300 import _build
    _build.build()
    torch.cuda.init()


def filt(plan, img):
    src = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()
    dst = torch.full_like(src, float("nan"))
    bf.bf_filter(plan, src, dst)
    torch.cuda.synchronize()
    return dst.cpu().numpy().astype(np.float64)


def oracle_outputs(img, kw):
    """The FP64 oracle's output, denominator and plan for one image and parameter set."""
    ref, _, den = O.approx_fast(img.astype(np.float64), O.Desc(**kw), threads=THREADS, return_den=True)
    return ref, den, O.plan_info(O.Desc(**kw))


def check_bound(got, img, kw, u, nk, den_eps, orc=None):
    """Every pixel within the bound above (pixels within 10x of the denominator guard excluded, where the fp32
    and fp64 guard decisions may differ); returns (max-abs error, PSNR) against the oracle."""
    ref, den, p = orc if orc is not None else oracle_outputs(img, kw)
    mass = window_mass(img.shape, p.Ks)
    ks = np.asarray(p.ks)
    ak = np.abs(np.asarray(p.ak))
    m = np.minimum(ks, nk)
    coef = 2e-7 * ak.sum() + 2.0 * u * float(np.sum(m * ak))
    bound = 1e-5 + coef * (1 + np.abs(ref)) * mass / np.maximum(np.abs(den), 1e-300)
    err = np.abs(got - ref)
    keep = np.abs(den) > 10 * den_eps
    assert keep.mean() > 0.999
    worst = np.max(err[keep] / bound[keep])
    assert worst <= 1.0, "error / bound %.3g (max err %.3g)" % (worst, err[keep].max())
    mse = float(np.mean((got - ref) ** 2))
    return float(err.max()), (10 * np.log10(1.0 / mse) if mse > 0 else float("inf"))


CASES = [
    ("sweep_s8", synth.shapes(400, 640, 41, scale=0.35), dict(sigma_s=8.0, sigma_r=0.1)),
    ("s2_r005", synth.shapes(300, 517, 42, scale=0.3), dict(sigma_s=2.0, sigma_r=0.05)),
    ("s16_nr16", synth.shapes(360, 480, 43, scale=0.4), dict(sigma_s=16.0, sigma_r=0.1, nr_terms=16)),
    ("m3_exp_range", synth.blocks(257, 301, 44), dict(sigma_s=3.0, ns_terms=7, range=bf.KERNEL_EXPONENTIAL, sigma_r=0.1)),
    ("tiny", synth.uniform(6, 3, 45), dict()),
]


@pytest.mark.parametrize("name,img,kw", CASES, ids=[c[0] for c in CASES])
def test_fp32_prepass_geometries_match_oracle(name, img, kw):
    # every fp32 pre-pass geometry family (terms per CTA, exchange depth) against the oracle at the fp32 bar
    from parity import conditioned_check
    H, W = img.shape
    plan = bf.Plan(device=0, **kw)
    cands = [c for c in bf.bf_launch_candidates(plan, H, W) if c["pre"] == 1]
    assert cands
    done = set()
    for c in cands:
        fam = (c["nk"], c["depth"])
        if fam in done:
            continue
        done.add(fam)
        bf.bf_set_launch(plan, H, W, c)
        got = filt(plan, img)
        e_good, worst, nbad = conditioned_check(got, img, kw)
        assert e_good < 1e-5 and worst < 1.0, (name, c, e_good, worst)


@pytest.mark.parametrize("prec", [bf.PREC_FP16, bf.PREC_BF16], ids=["fp16", "bf16"])
@pytest.mark.parametrize("name,img,kw", CASES, ids=[c[0] for c in CASES])
def test_16bit_basis_within_its_bound(name, img, kw, prec):
    H, W = img.shape
    plan = bf.Plan(device=0, precision=prec, **kw)
    info = bf.bf_launch_info(plan, H, W)
    assert info["pre"] == (2 if prec == bf.PREC_FP16 else 3)
    got = filt(plan, img)
    check_bound(got, img, kw, U[prec], info["nk"], plan.coeffs()["den_eps"])


@pytest.mark.parametrize("prec", [bf.PREC_FP16, bf.PREC_BF16], ids=["fp16", "bf16"])
def test_16bit_basis_full_size_and_accuracy_against_exact(prec):
    """1920x1080, sigma_s = 8 and 32, sigma_r = 0.1: every pixel within the bound, and >= 40 dB against the
    exact bilateral filter (GPU brute force)."""
    img = synth.shapes(1080, 1920, seed=0)
    src = torch.from_numpy(img).cuda()
    for ss in (8.0, 32.0):
        kw = dict(sigma_s=ss, sigma_r=0.1, nr_terms=8, ns_terms=5)
        plan = bf.Plan(device=0, precision=prec, **kw)
        info = bf.bf_autotune(plan, 1080, 1920)
        got = filt(plan, img)
        check_bound(got, img, kw, U[prec], info["nk"], plan.coeffs()["den_eps"])
        ex = torch.empty_like(src)
        bf.bf_exact(src, ex, sigma_s=ss, sigma_r=0.1)
        torch.cuda.synchronize()
        mse = float(np.mean((got - ex.cpu().numpy().astype(np.float64)) ** 2))
        assert 10 * np.log10(1.0 / mse) >= 40.0


def test_16bit_basis_4k_two_groups_within_its_bound():
    """The large-image workload at 3840x2160 (objects x2), sigma_s = 16, sigma_r = 0.1, N_r = 16: fp16 and bf16
    basis storage (the pre-pass variants, three term groups and the finalize pass) in their autotuned geometries,
    every pixel within the bound against the FP64 oracle, and >= 40 dB against it."""
    img = synth.shapes(2160, 3840, seed=0, scale=2.0)
    kw = dict(sigma_s=16.0, sigma_r=0.1, nr_terms=16, ns_terms=5)
    orc = oracle_outputs(img, kw)
    for prec in (bf.PREC_FP16, bf.PREC_BF16):
        plan = bf.Plan(device=0, precision=prec, **kw)
        info = bf.bf_autotune(plan, 2160, 3840)
        assert info["pre"] == (2 if prec == bf.PREC_FP16 else 3) and info["groups"] >= 2
        got = filt(plan, img)
        _, psnr = check_bound(got, img, kw, U[prec], info["nk"], plan.coeffs()["den_eps"], orc=orc)
        assert psnr >= 40.0, (prec, psnr)


def test_16bit_plans_in_batches_and_rejected_for_the_3d_form():
    with pytest.raises(bf.BFError) as ei:
        bf.Plan(device=0, precision=bf.PREC_FP16, policy=bf.RANGE_PAPER_3D)
    assert ei.value.status == bf.ERR_UNSUPPORTED
    # 16-bit plans in a batch run one by one after the persistent launches: bf_filter's result
    imgs = [synth.shapes(140, 230, 46, scale=0.2), synth.blocks(100, 90, 47)]
    plans = [bf.Plan(device=0, precision=bf.PREC_BF16), bf.Plan(device=0, sigma_s=2.0)]
    srcs = [torch.from_numpy(im).cuda() for im in imgs]
    dsts = [torch.full_like(x, float("nan")) for x in srcs]
    bf.bf_filter_batch(plans, srcs, dsts)
    torch.cuda.synchronize()
    for p, x, d in zip(plans, srcs, dsts):
        ref = torch.empty_like(x)
        bf.bf_filter(p, x, ref)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(d - ref)).item() < 1e-5
