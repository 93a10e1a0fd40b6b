"""GPU parity of bf_filter / bf_exact against the FP64 oracle (needs a CUDA GPU).

Element-wise comparisons on seeded images that span several tiles with ragged
tails, edge cases (tiny images, kernels wider than the image, pitched buffers,
asymmetric kernels, multi-pass plans), every pixel of the nine 1920x1080
benchmark outputs in the benchmark's launch arrangement and of a 3840x2160
two-group plan, and sampled pixels at 8192x8192.  Tolerance: 1e-5 max-abs for the fp32 path (the bar
the method's FP32 evaluation is held to on [0, 1] images).
"""
import os

import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
from oracle import oracle as O
from paper_1803_00004_gb300 import synth
from parity import conditioned_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
THREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00004_gb300 import _build
    _build.build()
    torch.cuda.init()


def run(img, **kw):
    plan = bf.Plan(device=0, **kw)
    src = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()
    dst = torch.full_like(src, float("nan"))
    bf.bf_filter(plan, src, dst)
    torch.cuda.synchronize()
    return dst.cpu().numpy().astype(np.float64)


def odesc(**kw):
    return O.Desc(**kw)


CASES = [
    ("cfg1_blocks_256", synth.blocks(256, 256, 0), dict()),
    ("shapes_m3", synth.shapes(300, 517, 1, scale=0.2), dict(sigma_s=2.0, ns_terms=13, sigma_r=0.05)),
    ("m4_multipass", synth.shapes(333, 270, 2, scale=0.2), dict(sigma_s=8.0, ns_terms=25, nr_terms=16)),
    ("tie_split_asym", synth.blocks(257, 129, 3), dict(sigma_s=4.0, ns_terms=2)),
    ("tie_split_m3", synth.uniform(77, 301, 4), dict(sigma_s=3.0, ns_terms=7, nr_terms=5)),
    ("exp_range_2pass", synth.shapes(190, 260, 5, scale=0.2), dict(range=bf.KERNEL_EXPONENTIAL, sigma_r=0.1, nr_terms=12)),
    ("box_range", synth.shapes(150, 170, 6, scale=0.2), dict(range=bf.KERNEL_BOX, sigma_r=0.2, nr_terms=10)),
    ("untruncated", synth.blocks(128, 300, 7), dict(policy=bf.RANGE_UNTRUNCATED_FULL, sigma_r=0.2, nr_terms=6)),
    ("box_spatial_m1", synth.blocks(140, 150, 8), dict(spatial=bf.KERNEL_BOX, sigma_s=2.0, ns_terms=4, nr_terms=20)),
    ("sigma32_R96", synth.shapes(400, 300, 9, scale=0.3), dict(sigma_s=32.0, sigma_r=0.3)),
    ("sigma8_nr32", synth.shapes(200, 220, 10, scale=0.2), dict(sigma_s=8.0, sigma_r=0.05, nr_terms=32)),
    ("m5", synth.shapes(160, 140, 11, scale=0.2), dict(sigma_s=4.0, ns_terms=41, nr_terms=6)),
    # the non-separable radial exponential spatial kernel (2-D Haar coefficients computed whole)
    ("exp_spatial", synth.shapes(210, 330, 15, scale=0.2), dict(spatial=bf.KERNEL_EXPONENTIAL, sigma_s=3.0)),
    ("exp_spatial_m3", synth.shapes(150, 260, 16, scale=0.2),
     dict(spatial=bf.KERNEL_EXPONENTIAL, sigma_s=2.0, ns_terms=13, nr_terms=6)),
    ("exp_spatial_r48", synth.shapes(260, 300, 17, scale=0.3),
     dict(spatial=bf.KERNEL_EXPONENTIAL, sigma_s=16.0, ns_terms=9, sigma_r=0.2)),
]


@pytest.mark.parametrize("name,img,kw", CASES, ids=[c[0] for c in CASES])
def test_parity_with_oracle(name, img, kw):
    got = run(img, **kw)
    e_good, worst, nbad = conditioned_check(got, img, kw)
    assert e_good < TOL, "%s: max err %.3g on well-conditioned pixels" % (name, e_good)
    assert worst < 1.0, "%s: %d ill-conditioned pixels, error / bound %.3g" % (name, nbad, worst)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 200), (200, 1), (5, 3), (24, 7), (3, 129), (31, 17)])
def test_tiny_and_narrow_images(H, W):
    img = synth.uniform(H, W, seed=H * 1000 + W)
    for kw in (dict(), dict(sigma_s=2.0, ns_terms=13), dict(sigma_s=4.0, ns_terms=2)):
        got = run(img, **kw)
        ref, _ = O.approx_fast(img.astype(np.float64), odesc(**kw))
        assert np.max(np.abs(got - ref)) < TOL


def test_constant_image_unchanged():
    img = np.full((150, 333), 0.625, dtype=np.float32)
    for kw in (dict(), dict(sigma_s=8.0, ns_terms=13, nr_terms=16), dict(sigma_s=2.0, ns_terms=2)):
        assert np.max(np.abs(run(img, **kw) - 0.625)) < 1e-6


def test_pitched_buffers_and_offset_range():
    """Row pitch larger than the width, and data range [2, 3]: the filter commutes with
    an intensity shift, so the result is the oracle's on I - 2, plus 2."""
    img = synth.shapes(120, 200, 12, scale=0.2)
    plan = bf.Plan(device=0, i_lo=2.0, i_hi=3.0)
    big = torch.zeros((120, 256), dtype=torch.float32, device="cuda")
    big[:, :200] = torch.from_numpy(img + 2.0).cuda()
    out = torch.full((120, 264), float("nan"), dtype=torch.float32, device="cuda")
    bf.bf_filter(plan, big[:, :200], out[:, :200])
    torch.cuda.synchronize()
    got = out[:, :200].cpu().numpy().astype(np.float64) - 2.0
    ref, _ = O.approx_fast(img.astype(np.float64), odesc())
    assert np.max(np.abs(got - ref)) < 2e-5
    assert torch.isnan(out[:, 200:]).all()  # nothing written past the width


def sample_points(H, W, n, seed):
    rng = np.random.default_rng(seed)
    edge = np.array([[0, 0], [H - 1, W - 1], [0, W - 1], [H - 1, 0], [H // 2, 0], [0, W // 2], [H - 1, W // 2 + 40],
                     [H // 2 + 60, W - 1]])
    return np.concatenate([np.stack([rng.integers(0, H, n), rng.integers(0, W, n)], 1), edge])


def test_full_size_parity_every_pixel():
    """1920x1080 (the benchmark workload) at each (sigma_s, sigma_r) of the sweep, run as the benchmark runs
    its step: each plan autotuned, then the nine tuned as a group, filtering concurrently on nine streams
    forked from one (one per filter), longest first.  Every pixel of every output against the oracle (Eq. (36) and the
    divide of Eq. (1)), under the conditioned 1e-5 bar."""
    img = synth.shapes(1080, 1920, seed=0)
    kws = [dict(sigma_s=ss, sigma_r=sr, nr_terms=8, ns_terms=5) for ss in (32.0, 8.0, 2.0) for sr in (0.05, 0.1, 0.3)]
    plans = [bf.Plan(device=0, **kw) for kw in kws]
    for p in plans:
        bf.bf_autotune(p, 1080, 1920)
    chosen = bf.bf_autotune_group(plans, 1080, 1920, n_streams=9)
    src = torch.from_numpy(img).cuda()
    outs = [torch.full_like(src, float("nan")) for _ in plans]
    main = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in range(9)]
    fork = torch.cuda.Event()
    fork.record(main)
    for s in streams:
        s.wait_event(fork)
    for n, (p, o) in enumerate(zip(plans, outs)):
        bf.bf_filter(p, src, o, stream=streams[n % 9])
    for s in streams:
        main.wait_stream(s)
    torch.cuda.synchronize()
    for p, kw, c, o in zip(plans, kws, chosen, outs):
        assert bf.bf_launch_info(p, 1080, 1920) == c
        got = o.cpu().numpy().astype(np.float64)
        e_good, worst, nbad = conditioned_check(got, img, kw)
        assert e_good < TOL, "sigma_s=%g sigma_r=%g (%s): max err %.3g" % (kw["sigma_s"], kw["sigma_r"], c, e_good)
        assert worst < 1.0, "sigma_s=%g sigma_r=%g: %d ill-conditioned pixels, error / bound %.3g" % (
            kw["sigma_s"], kw["sigma_r"], nbad, worst)


def test_4k_two_group_parity_every_pixel():
    """3840x2160, sigma_s = 16 (R = 48), sigma_r = 0.1, N_r = 16: two or more term groups (partial planes and
    the finalize pass), autotuned; every pixel against the oracle under the conditioned 1e-5 bar."""
    img = synth.shapes(2160, 3840, seed=0, scale=2.0)
    kw = dict(sigma_s=16.0, sigma_r=0.1, nr_terms=16, ns_terms=5)
    plan = bf.Plan(device=0, **kw)
    info = bf.bf_autotune(plan, 2160, 3840)
    assert info["groups"] >= 2
    got = run(img, **kw)
    e_good, worst, nbad = conditioned_check(got, img, kw)
    assert e_good < TOL, "max err %.3g (%s)" % (e_good, info)
    assert worst < 1.0, "%d ill-conditioned pixels, error / bound %.3g" % (nbad, worst)


def test_8k_sampled_parity():
    """8192x8192, sigma_s = 16 (R = 48), sigma_r = 0.1, N_r = 16 (two term groups, partial planes),
    autotuned: sampled pixels against the oracle's direct evaluation."""
    H = W = 8192
    img = synth.shapes(H, W, seed=0, scale=4.0)
    kw = dict(sigma_s=16.0, sigma_r=0.1, nr_terms=16, ns_terms=5)
    bf.bf_autotune(bf.Plan(device=0, **kw), H, W)
    pts = sample_points(H, W, 120, 1)
    got = run(img, **kw)[pts[:, 0], pts[:, 1]]
    ref = O.approx_direct_at(img.astype(np.float64), odesc(**kw), pts, threads=THREADS)
    err = np.max(np.abs(got - ref))
    assert err < TOL, "%dx%d: %.3g" % (W, H, err)


def test_deterministic_and_stream():
    img = synth.shapes(300, 400, 13, scale=0.2)
    plan = bf.Plan(device=0, sigma_s=8.0, ns_terms=13, nr_terms=16)
    src = torch.from_numpy(img).cuda()
    a = torch.empty_like(src)
    b = torch.empty_like(src)
    bf.bf_filter(plan, src, a)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bf.bf_filter(plan, src, b, stream=s)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_concurrent_streams_share_one_input():
    """Several plans (one with two term groups and a grouped scratch plane) filtering one input at once on
    three streams, as the benchmark's step runs them: each result equals the same plan's result alone."""
    img = synth.shapes(270, 490, 14, scale=0.2)
    kws = [dict(sigma_s=ss, sigma_r=sr, nr_terms=8, ns_terms=5) for ss in (2.0, 8.0, 32.0) for sr in (0.05, 0.3)]
    kws.append(dict(sigma_s=8.0, sigma_r=0.1, nr_terms=16, ns_terms=5))
    plans = [bf.Plan(device=0, **kw) for kw in kws]
    src = torch.from_numpy(img).cuda()
    alone = [torch.full_like(src, float("nan")) for _ in plans]
    for p, o in zip(plans, alone):
        bf.bf_filter(p, src, o)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(3)]
    for rep in range(3):
        outs = [torch.full_like(src, float("nan")) for _ in plans]
        fork = torch.cuda.Event()
        fork.record()
        for s in streams:
            s.wait_event(fork)
        for j, (p, o) in enumerate(zip(plans, outs)):
            bf.bf_filter(p, src, o, stream=streams[j % 3])
        for s in streams:
            torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        for kw, a, o in zip(kws, alone, outs):
            assert torch.equal(a, o), (rep, kw)


def test_group_autotune_pins_valid_geometries():
    """bf_autotune_group over a mixed group (two term groups with partial planes, two plans of one kernel
    class, a 3-D plan): it pins one geometry per class, bf_filter then launches it, and every result
    matches the oracle."""
    H, W = 70, 150
    img = synth.shapes(H, W, 51, scale=0.15)
    kws = [dict(sigma_s=8.0, sigma_r=0.1, nr_terms=16, ns_terms=5), dict(sigma_s=2.0, sigma_r=0.1),
           dict(sigma_s=2.0, sigma_r=0.3)]
    k3 = dict(sigma_s=2.0, sigma_r=0.1, nr_terms=6)
    plans = [bf.Plan(device=0, **kw) for kw in kws] + [bf.Plan(device=0, policy=bf.RANGE_PAPER_3D, z_bins=256, **k3)]
    chosen = bf.bf_autotune_group(plans, H, W, n_streams=2)
    assert chosen[1] == chosen[2]                      # one kernel class, reach and size: one geometry
    assert chosen[3]["packed"] == 1 and chosen[3]["ring"] == 0
    for p, c in zip(plans, chosen):
        assert bf.bf_launch_info(p, H, W) == c
    for kw in kws:
        ref, _ = O.approx_fast(img.astype(np.float64), odesc(**kw))
        assert np.max(np.abs(run(img, **kw) - ref)) < TOL, kw
    src = torch.from_numpy(img).cuda()
    dst = torch.full_like(src, float("nan"))
    bf.bf_filter(plans[3], src, dst)
    torch.cuda.synchronize()
    ref, _ = O.approx3d_direct(img.astype(np.float64), O.Desc(policy=O.PAPER_3D, **k3), 256)
    assert np.max(np.abs(dst.cpu().numpy() - ref)) < TOL


def test_in_place_rejected_and_injected_failure():
    img = synth.blocks(64, 64, 0)
    plan = bf.Plan(device=0)
    src = torch.from_numpy(img).cuda()
    with pytest.raises(bf.BFError) as ei:
        bf.bf_filter(plan, src, src)
    assert ei.value.status == 1
    dst = torch.empty_like(src)
    bf.bf_debug_fail_launches(1)
    with pytest.raises(bf.BFError) as ei:
        bf.bf_filter(plan, src, dst)
    assert ei.value.status == 4
    bf.bf_filter(plan, src, dst)  # recovers
    torch.cuda.synchronize()
    ref, _ = O.approx_fast(img.astype(np.float64), odesc())
    assert np.max(np.abs(dst.cpu().numpy() - ref)) < TOL


def test_debug_range_check():
    """bf_debug_range_checks: pixels outside [i_lo, i_hi] (NaN included) make bf_filter return BF_ERR_RANGE
    with their count and filter nothing; in-range images filter as usual; off, nothing is checked."""
    img = synth.blocks(70, 90, 3)
    plan = bf.Plan(device=0)
    src = torch.from_numpy(img).cuda()
    bad = src.clone()
    bad[5, 7] = 1.5
    bad[60, 80] = -0.25
    bad[33, 0] = float("nan")
    dst = torch.full_like(src, 7.0)
    bf.bf_debug_range_checks(True)
    try:
        with pytest.raises(bf.BFError) as ei:
            bf.bf_filter(plan, bad, dst)
        assert ei.value.status == 8 and "3 input pixels" in bf.lib().bf_last_error().decode()
        torch.cuda.synchronize()
        assert torch.all(dst == 7.0)  # nothing filtered
        bf.bf_filter(plan, src, dst)
        torch.cuda.synchronize()
        ref, _ = O.approx_fast(img.astype(np.float64), odesc())
        assert np.max(np.abs(dst.cpu().numpy() - ref)) < TOL
        wide = bf.Plan(device=0, i_lo=-1.0, i_hi=2.0)
        bf.bf_filter(wide, torch.nan_to_num(bad, nan=0.5), dst)  # inside the wider data range
    finally:
        bf.bf_debug_range_checks(False)
    bf.bf_filter(plan, bad, dst)  # unchecked
    torch.cuda.synchronize()


@pytest.mark.parametrize("kw", [dict(sigma_s=2.0, sigma_r=0.1), dict(sigma_s=3.0, sigma_r=0.2, range=bf.KERNEL_EXPONENTIAL),
                                dict(sigma_s=1.0, sigma_r=0.15, spatial=bf.KERNEL_BOX, radius=4),
                                dict(sigma_s=2.5, sigma_r=0.1, spatial=bf.KERNEL_EXPONENTIAL)])
def test_exact_helper_matches_oracle(kw):
    img = synth.shapes(90, 130, 14, scale=0.1)
    src = torch.from_numpy(img).cuda()
    dst = torch.empty_like(src)
    bf.bf_exact(src, dst, **kw)
    torch.cuda.synchronize()
    od = dict(kw)
    ref = O.exact_bf(img.astype(np.float64), O.Desc(**od), threads=THREADS)
    assert np.max(np.abs(dst.cpu().numpy() - ref)) < 2e-5


def test_config1_accuracy_against_exact_bf():
    """Config 1: the approximation is >= 40 dB PSNR against the exact bilateral filter."""
    img = synth.blocks(256, 256, 0)
    got = run(img)
    ex = O.exact_bf(img.astype(np.float64), O.Desc(), threads=THREADS)
    psnr = 10 * np.log10(1.0 / np.mean((got - ex) ** 2))
    assert psnr >= 40.0, psnr


def test_kahan_switch_on_long_rows():
    # 4096-wide rows with sigma_s = 2: the sliding sums run over the whole tile width;
    # compensated sums meet the fp32 bar, plain ones stay within 10x of it
    img = synth.shapes(40, 4096, 41, scale=0.5)
    kw = dict(sigma_s=2.0, sigma_r=0.1)
    ref, _ = O.approx_fast(img.astype(np.float64), odesc(**kw), threads=THREADS)
    err = {}
    for k in (1, 0):
        got = run(img, kahan=k, **kw)
        err[k] = float(np.max(np.abs(got - ref)))
    assert err[1] < TOL, err
    assert err[0] < 10 * TOL, err


@pytest.mark.parametrize("H,W,kw,levels", [
    (90, 131, dict(sigma_s=1.0, sigma_r=0.1), 256),
    (67, 45, dict(sigma_s=2.0, sigma_r=0.05, range=bf.KERNEL_EXPONENTIAL), 1024),
    (40, 300, dict(sigma_s=1.0, radius=6, sigma_r=0.2, spatial=bf.KERNEL_EXPONENTIAL), 64),
    (9, 5, dict(sigma_s=3.0, sigma_r=0.1), 256),                       # window larger than the image
    (33, 70, dict(sigma_s=10.0, radius=32, sigma_r=0.3, range=bf.KERNEL_BOX), 4096),
])
def test_exact_lut_matches_oracle(H, W, kw, levels):
    """The look-up-table brute force against the oracle's same table rule (the entry index is decided in
    fp32 on both sides)."""
    img = synth.shapes(H, W, 18, scale=0.1)
    src = torch.from_numpy(img).cuda()
    dst = torch.full_like(src, float("nan"))
    bf.bf_exact_lut(src, dst, levels=levels, **kw)
    torch.cuda.synchronize()
    ref = O.exact_bf_lut(img.astype(np.float64), O.Desc(**kw), levels, threads=THREADS)
    assert np.max(np.abs(dst.cpu().numpy() - ref)) < 1e-5


def test_exact_lut_full_size_8bit():
    """1920x1080 with 8-bit-valued data (k / 255) and a 256-entry table, R = 3: the whole image against the
    oracle's table rule."""
    img = (np.round(synth.shapes(1080, 1920, seed=0) * 255) / 255).astype(np.float32)
    kw = dict(sigma_s=1.0, sigma_r=0.1)
    src = torch.from_numpy(img).cuda()
    dst = torch.empty_like(src)
    bf.bf_exact_lut(src, dst, levels=256, **kw)
    torch.cuda.synchronize()
    ref = O.exact_bf_lut(img.astype(np.float64), O.Desc(**kw), 256, threads=THREADS)
    assert np.max(np.abs(dst.cpu().numpy() - ref)) < 1e-5
