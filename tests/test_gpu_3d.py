"""GPU parity of the 3-D form (BF_RANGE_PAPER_3D: P = T_r, the range box applied over intensity slices)
against the FP64 oracle (needs a CUDA GPU).

The reference is O2-3D (the definition; pinned equal to the paper's per-slice steps O3-3D).  Slice
decisions are taken in fp32 on both sides, so every neighbour is in or out of a window identically.
Tolerance: 1e-5 max-abs where the denominator is at least 1% of the in-window kernel mass (the mass of
the neighbours inside the slice window); below that the fp32 rounding of the sums (~2e-7 relative) is
amplified by sum |a_k| mass / |den| and the bound scales with it.  Images span several tiles with ragged
tails; edge cases cover tiny images, two and 4096 slices, several term groups, windows wider than the
data range, every launch geometry family and the full 1920x1080 size (sampled).
"""
import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
from oracle import oracle as O
from paper_1803_00004_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
THREADS = 16


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00004_gb300 import _build
    _build.build()
    torch.cuda.init()


def on_grid(H, W, seed):
    """8-bit data: levels j / 255 stored as fp32."""
    rng = np.random.default_rng(seed)
    j = np.clip(np.rint(synth.shapes(H, W, seed, scale=0.2) * 255) + rng.integers(-2, 3, (H, W)), 0, 255)
    return (j / 255.0).astype(np.float32)


def plan3d(Z, **kw):
    return bf.Plan(device=0, policy=bf.RANGE_PAPER_3D, z_bins=Z, **kw)


def gpu(plan, img):
    src = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()
    dst = torch.full_like(src, float("nan"))
    bf.bf_filter(plan, src, dst)
    torch.cuda.synchronize()
    return dst.cpu().numpy().astype(np.float64)


def odesc(kw):
    return O.Desc(policy=O.PAPER_3D, **kw)


def window_mass(img, kw, Z):
    """sum over the window of |K~_s(x - y)| for the neighbours y inside x's slice window."""
    p = O.plan_info(odesc(kw))
    bins, rz = O.z_bins(img.astype(np.float64), p.Tr, Z)
    H, W = img.shape
    R = p.R
    pb = np.full((H + 2 * R, W + 2 * R), -10 ** 6, dtype=np.int64)
    pb[R:R + H, R:R + W] = bins
    mass = np.zeros((H, W))
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            k = abs(p.Ks[-dy + R, -dx + R])
            if k == 0.0:
                continue
            nb = pb[R + dy:R + dy + H, R + dx:R + dx + W]
            mass += k * (np.abs(nb - bins) <= rz)
    return mass, p


def check(got, img, kw, Z):
    ref, _, den = O.approx3d_direct(img.astype(np.float64), odesc(kw), Z, threads=THREADS, return_den=True)
    mass, p = window_mass(img, kw, Z)
    ratio = np.abs(den) / mass
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    good = ratio >= 0.01
    assert good.mean() > 0.98, "too many ill-conditioned pixels: %g" % (1 - good.mean())
    e_good = err[good].max()
    bound = TOL + 2e-7 * np.sum(np.abs(p.ak)) * (1 + np.abs(ref)) / np.maximum(ratio, 1e-12)
    worst = np.max(err[~good] / bound[~good]) if (~good).any() else 0.0
    return e_good, worst


CASES = [
    ("shapes_s2_z256", synth.shapes(150, 203, 1, scale=0.2), dict(sigma_s=2.0, sigma_r=0.1), 256),
    ("8bit_s4_z256", on_grid(170, 150, 2), dict(sigma_s=4.0, sigma_r=0.05), 256),
    ("blocks_groups", synth.blocks(131, 260, 3), dict(sigma_s=3.0, sigma_r=0.1, nr_terms=12), 64),
    ("exp_range", synth.shapes(140, 190, 4, scale=0.2),
     dict(range=bf.KERNEL_EXPONENTIAL, sigma_r=0.1, nr_terms=6, sigma_s=2.0), 128),
    ("box_spatial_m1", synth.blocks(100, 333, 5), dict(spatial=bf.KERNEL_BOX, sigma_s=2.0, ns_terms=1, nr_terms=4), 256),
    ("m3_ns13", synth.shapes(160, 170, 6, scale=0.2), dict(sigma_s=2.0, ns_terms=13, sigma_r=0.08), 256),
    ("z2", synth.uniform(64, 90, 7), dict(sigma_s=2.0, sigma_r=0.3), 2),
    ("z4096", synth.shapes(90, 120, 8, scale=0.1), dict(sigma_s=2.0, sigma_r=0.02, nr_terms=4), 4096),
    ("exp_spatial", synth.shapes(120, 150, 9, scale=0.2), dict(spatial=bf.KERNEL_EXPONENTIAL, sigma_s=2.0), 256),
    ("sigma8", synth.shapes(200, 230, 10, scale=0.2), dict(sigma_s=8.0, sigma_r=0.1), 256),
]


@pytest.mark.parametrize("name,img,kw,Z", CASES, ids=[c[0] for c in CASES])
def test_3d_matches_oracle(name, img, kw, Z):
    got = gpu(plan3d(Z, **kw), img)
    e_good, worst = check(got, img, kw, Z)
    assert e_good < TOL, "%s: max err %.3g" % (name, e_good)
    assert worst < 1.0, "%s: error / bound %.3g on ill-conditioned pixels" % (name, worst)


@pytest.mark.parametrize("H,W", [(1, 1), (2, 3), (5, 1), (1, 77), (9, 300)])
def test_3d_tiny_images(H, W):
    img = synth.uniform(H, W, seed=H * 31 + W)
    kw = dict(sigma_s=2.0, sigma_r=0.1)
    got = gpu(plan3d(256, **kw), img)
    ref, _ = O.approx3d_direct(img.astype(np.float64), odesc(kw), 256)
    assert np.max(np.abs(got - ref)) < TOL


@pytest.mark.parametrize("m", [0, 5])
def test_3d_box_kernels_on_8bit_data_are_exact_bf(m):
    """Box spatial and range kernels on 8-bit data: the 3-D form is the exact bilateral filter."""
    img = on_grid(97, 140, 11 + m)
    kw = dict(spatial=bf.KERNEL_BOX, sigma_s=1.0, radius=3, ns_terms=1, range=bf.KERNEL_BOX,
              sigma_r=(m + 0.5) / 255.0, nr_terms=2)
    got = gpu(plan3d(256, **kw), img)
    ref = O.exact_bf(img.astype(np.float64), O.Desc(**kw))
    assert np.max(np.abs(got - ref)) < 2e-6


def test_3d_wide_window_equals_collapsed_filter():
    """T_r >= dI: every neighbour is inside the slice window and both policies take P = T_r, so the 3-D
    launch and the collapsed launch compute the same sums."""
    img = synth.shapes(180, 210, 12, scale=0.2)
    kw = dict(sigma_s=3.0, sigma_r=0.4, t_r=1.25, nr_terms=8)
    a = gpu(plan3d(256, **kw), img)
    b = gpu(bf.Plan(device=0, **kw), img)
    assert np.max(np.abs(a - b)) < 2e-6


def family(c):
    return (c["nk"], c["depth"], c["tw"], c["th"])


def test_3d_every_candidate_family():
    """Launch geometries of a 3-D plan (packed family, no ring): each distinct terms-per-CTA and depth."""
    img = synth.shapes(140, 250, 13, scale=0.2)
    kw = dict(sigma_s=2.0, sigma_r=0.1, nr_terms=8)
    plan = plan3d(256, **kw)
    H, W = img.shape
    default = bf.bf_launch_info(plan, H, W)
    cands = bf.bf_launch_candidates(plan, H, W)
    assert cands and all(c["ring"] == 0 and c["packed"] == 1 for c in cands)
    firsts = {}
    for c in cands:  # terms per CTA x depth x CTAs of at most 256 threads (register-bounded kernels) or more
        firsts.setdefault((c["nk"], c["depth"], c["threads"] > 256), c)
    assert len(firsts) >= 8
    try:
        for fam, c in firsts.items():
            bf.bf_set_launch(plan, H, W, c)
            got = gpu(plan, img)
            e_good, worst = check(got, img, kw, 256)
            assert e_good < TOL and worst < 1.0, (fam, e_good, worst)
    finally:
        bf.bf_set_launch(plan, H, W, default)


def test_3d_autotune_keeps_parity():
    img = synth.shapes(96, 200, 14, scale=0.2)
    kw = dict(sigma_s=2.0, sigma_r=0.05, nr_terms=6)
    plan = plan3d(256, **kw)
    info = bf.bf_autotune(plan, *img.shape)
    assert info["ring"] == 0 and info["packed"] == 1
    got = gpu(plan, img)
    e_good, worst = check(got, img, kw, 256)
    assert e_good < TOL and worst < 1.0


def test_3d_full_size_sampled():
    """The 1920 x 1080 sweep image with sigma_s = 8, sigma_r = 0.1, N_r = 8, 256 slices: 3000 sampled pixels."""
    img = synth.shapes(1080, 1920, seed=0)
    kw = dict(sigma_s=8.0, sigma_r=0.1, nr_terms=8)
    got = gpu(plan3d(256, **kw), img)
    assert np.all(np.isfinite(got))
    rng = np.random.default_rng(5)
    pts = np.stack([rng.integers(0, 1080, 3000), rng.integers(0, 1920, 3000)], axis=1)
    pts[:4] = [[0, 0], [1079, 1919], [0, 1919], [1079, 0]]
    ref, den = O.approx3d_direct_at(img.astype(np.float64), odesc(kw), pts, 256, threads=THREADS)
    err = np.abs(got[pts[:, 0], pts[:, 1]] - ref)
    assert np.max(err) < TOL


def test_3d_in_batches_and_the_server():
    """3-D plans in a batch with collapsed ones (launched one by one after the persistent launches, captured in
    the same graph) and through the server: each result equals bf_filter's within the bar and the oracle's."""
    imgs = [synth.shapes(120, 200, 61, scale=0.2), synth.blocks(96, 130, 62), synth.shapes(150, 90, 63, scale=0.2)]
    plans = [plan3d(256, sigma_s=2.0, sigma_r=0.1, nr_terms=4), bf.Plan(device=0, sigma_s=3.0),
             bf.Plan(device=0, policy=bf.RANGE_PAPER_3D, range_series=bf.SERIES_HAAR, z_bins=256, sigma_s=2.0,
                     sigma_r=0.1, nr_terms=8)]
    srcs = [torch.from_numpy(im).cuda() for im in imgs]
    for _ in range(2):  # the second call replays the captured graph
        dsts = [torch.full_like(x, float("nan")) for x in srcs]
        bf.bf_filter_batch(plans, srcs, dsts)
        torch.cuda.synchronize()
        for p, x, d in zip(plans, srcs, dsts):
            ref = torch.empty_like(x)
            bf.bf_filter(p, x, ref)
            torch.cuda.synchronize()
            assert torch.max(torch.abs(d - ref)).item() < TOL
    want = O.approx3d_direct(imgs[0].astype(np.float64), odesc(dict(sigma_s=2.0, sigma_r=0.1, nr_terms=4)), 256,
                             threads=THREADS)[0]
    assert np.max(np.abs(dsts[0].cpu().numpy() - want)) < TOL
    srv = bf.Server(max_slots=4, n_streams=2)
    hin = torch.from_numpy(imgs[0]).pin_memory()
    hout = torch.full_like(hin, float("nan")).pin_memory()
    t = srv.submit(bf.desc(policy=bf.RANGE_PAPER_3D, z_bins=256, sigma_s=2.0, sigma_r=0.1, nr_terms=4),
                   hin.data_ptr(), hout.data_ptr(), 120, 200)
    st, r = srv.poll(t, -1)
    assert st == 0 and r.status == 0
    assert np.max(np.abs(hout.numpy() - want)) < TOL
    srv.close()


def test_3d_rejected_where_unsupported():
    plan = plan3d(256, sigma_s=2.0)
    src = torch.rand(64, 64, device="cuda")
    with pytest.raises(bf.BFError) as ei:
        bf.Cache(plan, src, kmax=8)
    assert ei.value.status == 2  # BF_ERR_UNSUPPORTED


# ---- the Haar range series (BF_SERIES_HAAR): a neighbour's weight is K~_s(x - y) K~_r(n(x) - n(y)), K~_r the
# best N-term Haar expansion of the truncated range kernel on the slice axis

def plan3dh(Z, **kw):
    return bf.Plan(device=0, policy=bf.RANGE_PAPER_3D, range_series=bf.SERIES_HAAR, z_bins=Z, **kw)


def check_haar(got, img, kw, Z):
    """As check(), with the range weights of the Haar table: mass = sum |K~_s| |K~_r| over the neighbours."""
    d = O.Desc(**kw)
    ref, den = O.approx3dh_direct(img.astype(np.float64), d, Z, threads=THREADS)
    p = O.plan_info(O.Desc(policy=O.PAPER_3D, **kw))
    zi = O.zhaar_info(d, Z)
    bins, _ = O.z_bins(img.astype(np.float64), zi.Rz / (Z - 1) + 1e-12, Z)
    H, W = img.shape
    R, Rz = p.R, zi.Rz
    pb = np.full((H + 2 * R, W + 2 * R), -10 ** 6, dtype=np.int64)
    pb[R:R + H, R:R + W] = bins
    mass = np.zeros((H, W))
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            k = abs(p.Ks[-dy + R, -dx + R])
            if k == 0.0:
                continue
            dd = bins - pb[R + dy:R + dy + H, R + dx:R + dx + W]
            inw = np.abs(dd) <= Rz
            mass += k * np.where(inw, np.abs(zi.w[np.clip(dd + Rz, 0, 2 * Rz)]), 0.0)
    ratio = np.abs(den) / np.maximum(mass, 1e-300)
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    good = ratio >= 0.01
    assert good.mean() > 0.98, "too many ill-conditioned pixels: %g" % (1 - good.mean())
    bound = TOL + 2e-7 * (1 + np.abs(ref)) / np.maximum(ratio, 1e-12)
    worst = np.max(err[~good] / bound[~good]) if (~good).any() else 0.0
    return err[good].max(), worst


HCASES = [
    ("haar_gauss_s2", synth.shapes(150, 203, 21, scale=0.2), dict(sigma_s=2.0, sigma_r=0.1, nr_terms=8), 256),
    ("haar_exp_range", synth.shapes(140, 190, 22, scale=0.2),
     dict(range=bf.KERNEL_EXPONENTIAL, sigma_r=0.05, nr_terms=6, sigma_s=2.0), 128),
    ("haar_box_range", synth.blocks(120, 260, 23), dict(range=bf.KERNEL_BOX, sigma_r=0.2, nr_terms=16, sigma_s=3.0), 256),
    ("haar_m3", synth.shapes(160, 170, 24, scale=0.2), dict(sigma_s=2.0, ns_terms=13, sigma_r=0.08, nr_terms=8), 256),
    ("haar_sigma8", synth.shapes(200, 230, 25, scale=0.2), dict(sigma_s=8.0, sigma_r=0.1, nr_terms=16), 256),
    ("haar_z2048", synth.shapes(90, 140, 26, scale=0.1), dict(sigma_s=2.0, sigma_r=0.1, nr_terms=24), 2048),
    ("haar_nr7_uniform", synth.uniform(70, 110, 27), dict(sigma_s=1.5, sigma_r=0.1, nr_terms=7), 256),
]


@pytest.mark.parametrize("name,img,kw,Z", HCASES, ids=[c[0] for c in HCASES])
def test_3d_haar_matches_oracle(name, img, kw, Z):
    got = gpu(plan3dh(Z, **kw), img)
    e_good, worst = check_haar(got, img, kw, Z)
    assert e_good < TOL, "%s: max err %.3g" % (name, e_good)
    assert worst < 1.0, "%s: error / bound %.3g on ill-conditioned pixels" % (name, worst)


@pytest.mark.parametrize("H,W", [(1, 1), (3, 2), (1, 50), (7, 300)])
def test_3d_haar_tiny_images(H, W):
    img = synth.uniform(H, W, seed=H * 17 + W)
    kw = dict(sigma_s=2.0, sigma_r=0.1, nr_terms=8)
    got = gpu(plan3dh(256, **kw), img)
    ref, _ = O.approx3dh_direct(img.astype(np.float64), O.Desc(**kw), 256)
    assert np.max(np.abs(got - ref)) < TOL


def test_3d_haar_box_kernels_on_8bit_data_are_exact_bf():
    img = on_grid(97, 140, 31)
    kw = dict(spatial=bf.KERNEL_BOX, sigma_s=1.0, radius=3, ns_terms=1, range=bf.KERNEL_BOX, sigma_r=4.5 / 255.0,
              nr_terms=3)
    got = gpu(plan3dh(256, **kw), img)
    ref = O.exact_bf(img.astype(np.float64), O.Desc(**kw))
    assert np.max(np.abs(got - ref)) < 2e-6


def test_3d_haar_every_candidate_family():
    img = synth.shapes(130, 240, 32, scale=0.2)
    kw = dict(sigma_s=2.0, sigma_r=0.1, nr_terms=8)
    plan = plan3dh(256, **kw)
    H, W = img.shape
    default = bf.bf_launch_info(plan, H, W)
    cands = bf.bf_launch_candidates(plan, H, W)
    assert cands and all(c["ring"] == 0 and c["packed"] == 1 and c["nk"] == 2 for c in cands)
    firsts = {}
    for c in cands:  # both depths, with CTAs of at most 256 threads (the register-bounded kernel) and more
        firsts.setdefault((c["depth"], c["threads"] > 256), c)
    assert len(firsts) == 4
    try:
        for fam, c in firsts.items():
            bf.bf_set_launch(plan, H, W, c)
            got = gpu(plan, img)
            e_good, worst = check_haar(got, img, kw, 256)
            assert e_good < TOL and worst < 1.0, (fam, e_good, worst)
    finally:
        bf.bf_set_launch(plan, H, W, default)


@pytest.mark.parametrize("sigma_s,nr", [(8.0, 8), (32.0, 64)])
def test_3d_haar_full_size_sampled(sigma_s, nr):
    """The 1920 x 1080 sweep image, 256 slices, in the geometry the benchmark's 3-D lines use (tuned on the
    image itself; sigma_s = 32 runs the 512-thread, 64-register slice kernel): 3000 sampled pixels."""
    img = synth.shapes(1080, 1920, seed=0)
    kw = dict(sigma_s=sigma_s, sigma_r=0.1, nr_terms=nr)
    plan = plan3dh(256, **kw)
    bf.bf_autotune_image(plan, torch.from_numpy(img).cuda())
    got = gpu(plan, img)
    assert np.all(np.isfinite(got))
    rng = np.random.default_rng(6)
    pts = np.stack([rng.integers(0, 1080, 3000), rng.integers(0, 1920, 3000)], axis=1)
    pts[:4] = [[0, 0], [1079, 1919], [0, 1919], [1079, 0]]
    ref, _ = O.approx3dh_direct(img.astype(np.float64), O.Desc(**kw), 256, pts=pts, threads=THREADS)
    assert np.max(np.abs(got[pts[:, 0], pts[:, 1]] - ref)) < TOL


@pytest.mark.parametrize("series", [0, 1])
def test_3d_pitched_buffers_leave_padding(series):
    """Pitched input and output: the slice list and slice kernels read and write inside the width only
    (the output padding keeps its NaN canary), and the result matches the oracle."""
    img = synth.shapes(70, 150, 51, scale=0.15)
    kw = dict(sigma_s=2.0, sigma_r=0.1, nr_terms=6 if series == 0 else 16)
    plan = bf.Plan(device=0, policy=bf.RANGE_PAPER_3D, z_bins=256, range_series=series, **kw)
    big = torch.full((70, 192), 0.5, dtype=torch.float32, device="cuda")
    big[:, :150] = torch.from_numpy(img).cuda()
    out = torch.full((70, 200), float("nan"), dtype=torch.float32, device="cuda")
    bf.bf_filter(plan, big[:, :150], out[:, :150])
    torch.cuda.synchronize()
    assert torch.isnan(out[:, 150:]).all()
    got = out[:, :150].cpu().numpy().astype(np.float64)
    if series == 0:
        ref, _ = O.approx3d_direct(img.astype(np.float64), odesc(kw), 256)
    else:
        ref, _ = O.approx3dh_direct(img.astype(np.float64), O.Desc(**kw), 256)
    assert np.max(np.abs(got - ref)) < TOL


def test_autotune_on_the_callers_image():
    """bf_autotune_image times the geometries on the caller's image (here a pitched view), pins one that
    bf_filter then launches, and the result matches the oracle."""
    H, W = 150, 260
    img = synth.shapes(H, W, 52, scale=0.2)
    kw = dict(sigma_s=2.0, sigma_r=0.1, nr_terms=6)
    plan = plan3d(256, **kw)
    big = torch.zeros((H, 288), dtype=torch.float32, device="cuda")
    big[:, :W] = torch.from_numpy(img).cuda()
    info = bf.bf_autotune_image(plan, big[:, :W])
    assert info["packed"] == 1 and info["ring"] == 0
    assert bf.bf_launch_info(plan, H, W) == info
    e_good, worst = check(gpu(plan, img), img, kw, 256)
    assert e_good < TOL and worst < 1.0, (e_good, worst)
