"""C-ABI library checks that need no GPU: it loads, exports every symbol the
header declares, validates arguments, and its host-side plan (coefficients,
best N-term selection, kernel table, window compilation) agrees with the
independent FP64 oracle."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1803_00004_gb300 import _build
    _build.build()


def test_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "bf.h")).read()
    names = set(re.findall(r"\b(bf_[a-z_0-9]+)\s*\(", hdr))
    assert names, "no declarations found"
    L = bf.lib()
    for n in sorted(names):
        assert hasattr(L, n), "missing export %s" % n
    assert set(bf.EXPORTS) <= names


def test_status_strings_and_version():
    L = bf.lib()
    for s in range(13):
        assert L.bf_status_string(s) and L.bf_status_string(s) != b"unknown status"
    # the fixed-scratch status of bf_filter_noalloc is its own code, not the input-range one
    assert bf.ERR_SCRATCH == 12 and bf.ERR_SCRATCH != bf.ERR_RANGE
    assert b"scratch" in L.bf_status_string(bf.ERR_SCRATCH)
    assert bf.bf_version() >= 1


DESCS = [
    dict(),
    dict(sigma_s=2.0, ns_terms=13, sigma_r=0.05),
    dict(sigma_s=8.0, ns_terms=25, nr_terms=16),
    dict(sigma_s=32.0, sigma_r=0.3),
    dict(sigma_s=4.0, ns_terms=2),
    dict(sigma_s=3.0, ns_terms=3, nr_terms=5),
    dict(range=bf.KERNEL_EXPONENTIAL, sigma_r=0.1, nr_terms=12),
    dict(range=bf.KERNEL_BOX, sigma_r=0.2, nr_terms=10),
    dict(policy=bf.RANGE_UNTRUNCATED_FULL, sigma_r=0.2, nr_terms=6),
    dict(spatial=bf.KERNEL_BOX, sigma_s=2.0, ns_terms=4),
    dict(sigma_s=2.0, radius=4, ns_terms=25, nr_terms=16, sigma_r=0.07),
    dict(spatial=bf.KERNEL_EXPONENTIAL, sigma_s=1.5),
    dict(spatial=bf.KERNEL_EXPONENTIAL, sigma_s=3.0, ns_terms=13, nr_terms=6),
    dict(spatial=bf.KERNEL_EXPONENTIAL, sigma_s=8.0, ns_terms=9),
]


def _odesc(kw):
    m = dict(kw)
    od = {}
    for k, v in m.items():
        od[{"spatial": "spatial", "range": "range", "policy": "policy"}.get(k, k)] = v
    return O.Desc(**od)


@pytest.mark.parametrize("kw", DESCS)
def test_plan_matches_oracle(kw):
    p = bf.Plan(device=-1, **kw)
    c = p.coeffs()
    o = O.plan_info(_odesc(kw))
    assert c["radius"] == o.R
    assert abs(c["t_r"] - o.Tr) < 1e-15 and abs(c["period"] - o.P) < 1e-15
    # same selected cosine terms (the product lists them by k, the oracle by rank)
    order = np.argsort(o.ks)
    assert list(c["k"]) == list(o.ks[order])
    assert np.max(np.abs(np.array(c["a"]) - o.ak[order])) < 1e-13
    # same Haar terms in the same ranking order
    assert [list(t) for t in c["haar_terms"]] == [list(t) for t in o.terms]
    assert np.max(np.abs(np.array(c["haar_coef"]) - o.term_c)) < 1e-14
    assert c["tie_split"] == o.tie_split
    assert np.max(np.abs(np.array(c["kernel"]) - o.Ks)) < 1e-14
    assert abs(c["den_eps"] - o.den_eps) < 1e-12 * max(1.0, o.den_eps)


@pytest.mark.parametrize("kw", DESCS)
def test_window_compilation_reproduces_kernel(kw):
    c = bf.Plan(device=-1, **kw).coeffs()
    R = c["radius"]
    K = np.array(c["kernel"])
    rec = np.zeros_like(K)   # indexed [dy + R, dx + R] over neighbour offsets d = y - x
    for v, (v0, v1) in enumerate(c["vwin"]):
        for h, (u0, u1) in enumerate(c["hwin"]):
            rec[v0 + R:v1 + R + 1, u0 + R:u1 + R + 1] += c["wcoef"][v][h]
    # weight of neighbour offset d is K~_s(-d)
    assert np.max(np.abs(rec - K[::-1, ::-1])) < 1e-12 * np.max(np.abs(K))


def test_paper_five_terms_compile_to_two_nested_windows():
    c = bf.Plan(device=-1).coeffs()
    assert c["vwin"] == [(-6, 6), (-12, 12)] and c["hwin"] == [(-6, 6), (-12, 12)]
    assert abs(c["wcoef"][0][0]) < 1e-15   # no inner x inner box: three box shapes, Sec. V-A
    assert c["passes"] == 1


@pytest.mark.parametrize("sigma_r,z_bins,t_r", [(0.1, 0, 0.0), (0.05, 64, 0.0), (0.2, 4096, 0.0), (0.3, 256, 10 / 255)])
def test_paper_3d_plan_matches_oracle(sigma_r, z_bins, t_r):
    """The 3-D form's plan: P = T_r, the oracle's coefficients, and the slice window R_z."""
    c = bf.Plan(device=-1, policy=bf.RANGE_PAPER_3D, sigma_r=sigma_r, z_bins=z_bins, t_r=t_r).coeffs()
    d = O.Desc(sigma_r=sigma_r, t_r=t_r, policy=O.PAPER_3D)
    info = O.plan_info(d)
    assert c["period"] == pytest.approx(info.P, rel=1e-15) and c["t_r"] == pytest.approx(info.Tr, rel=1e-15)
    order = np.argsort(info.ks)                       # the plan lists its terms by frequency
    assert list(c["k"]) == list(info.ks[order])
    assert np.max(np.abs(np.array(c["a"]) - info.ak[order])) < 1e-13
    Z = z_bins or 256
    _, rz = O.z_bins([0.0], info.Tr, Z)
    assert c["z_bins"] == Z and c["z_radius"] == rz
    assert bf.Plan(device=-1).coeffs()["z_bins"] == 0


@pytest.mark.parametrize("kw,Z", [(dict(sigma_r=0.1, nr_terms=8), 256), (dict(sigma_r=0.05, nr_terms=3, range=O.EXPONENTIAL), 256),
                                  (dict(sigma_r=0.2, nr_terms=16, range=O.BOX), 128), (dict(sigma_r=0.1, nr_terms=40), 2048)])
def test_haar_range_plan_matches_oracle(kw, Z):
    """The Haar range series of the 3-D form: the kept terms, their coefficients and the weight table."""
    c = bf.Plan(device=-1, policy=bf.RANGE_PAPER_3D, range_series=bf.SERIES_HAAR, z_bins=Z, **kw).coeffs()
    info = O.zhaar_info(O.Desc(**kw), Z)
    assert c["range_series"] == bf.SERIES_HAAR and c["z_radius"] == info.Rz
    assert c["range_haar"] == [(int(a), int(b)) for a, b in zip(info.lev, info.k)]
    assert np.max(np.abs(np.array(c["range_haar_coef"]) - info.c)) < 1e-13
    assert np.max(np.abs(np.array(c["z_weights"]) - info.w)) < 1e-13
    assert c["k"] == [0] and c["a"] == [1.0]


@pytest.mark.parametrize("kw,status", [
    (dict(range_series=bf.SERIES_HAAR), 1), (dict(range_series=7), 1),
    (dict(policy=bf.RANGE_PAPER_3D, range_series=bf.SERIES_HAAR, z_bins=4096, sigma_r=0.1), 2),
    (dict(sigma_s=0.0), 1), (dict(sigma_r=-1.0), 1), (dict(ns_terms=0), 1), (dict(nr_terms=0), 1),
    (dict(i_lo=1.0, i_hi=1.0), 1), (dict(policy=bf.RANGE_PAPER_3D, z_bins=1), 1),
    (dict(policy=bf.RANGE_PAPER_3D, z_bins=4097), 1), (dict(policy=5), 1),
    (dict(spatial=bf.KERNEL_EXPONENTIAL, sigma_s=100.0), 2),
    (dict(spatial=7), 1), (dict(precision=9), 1), (dict(radius=-2), 1), (dict(precision=bf.PREC_BF16, policy=bf.RANGE_PAPER_3D), 2), (dict(precision=bf.PREC_FP16, policy=bf.RANGE_PAPER_3D), 2),
])
def test_plan_create_rejects(kw, status):
    with pytest.raises(bf.BFError) as ei:
        bf.Plan(device=-1, **kw)
    assert ei.value.status == status


def test_filter_argument_checks_without_gpu():
    p = bf.Plan(device=-1)
    L = bf.lib()
    # look-up-table brute force: parameters are checked before any device work
    assert L.bf_exact_lut(4096, 256, 1 << 20, 256, 4, 64, 0, 2.0, 0, 0, 0.1, 1.0, 1, None) == 1    # levels < 2
    assert L.bf_exact_lut(4096, 256, 1 << 20, 256, 4, 64, 0, 2.0, 0, 0, 0.1, 1.0, 8192, None) == 1  # levels > 4096
    assert L.bf_exact_lut(4096, 256, 1 << 20, 256, 4, 64, 0, 2.0, 40, 0, 0.1, 1.0, 256, None) == 2  # radius > 32
    assert L.bf_exact_lut(4096, 256, 1 << 20, 256, 4, 64, 0, 2.0, 0, 0, 0.1, 0.0, 256, None) == 1   # data range
    # overlapping input/output -> invalid argument before any device work
    assert L.bf_filter(p.handle, 4096, 256, 4096 + 128, 256, 4, 64, None) == 1
    # bad pitch
    assert L.bf_filter(p.handle, 4096, 6, 1 << 20, 256, 4, 64, None) == 1
    assert L.bf_filter(p.handle, 4096, 64, 1 << 20, 256, 4, 64, None) == 1
    # pitches of 4 GiB or more (the kernels form row addresses with a 32-bit byte pitch)
    assert L.bf_filter(p.handle, 1 << 20, 1 << 32, 1 << 44, 256, 2, 64, None) == 1
    assert L.bf_filter(p.handle, 1 << 20, 256, 1 << 44, (1 << 32) + 256, 2, 64, None) == 1
    # empty image is a no-op
    assert L.bf_filter(p.handle, 0, 0, 0, 0, 0, 5, None) == 0
    # host-only plan cannot filter
    assert L.bf_filter(p.handle, 4096, 256, 1 << 20, 256, 4, 64, None) == 9
    assert L.bf_filter(None, 4096, 256, 1 << 20, 256, 4, 64, None) == 1
    assert L.bf_coeffs(None, None) == 1


def test_range_and_spatial_errors_reported():
    c = bf.Plan(device=-1, sigma_r=0.1, nr_terms=8).coeffs()
    assert 0 < c["range_max_err"] < 0.05
    c2 = bf.Plan(device=-1, sigma_r=0.3, nr_terms=8, policy=bf.RANGE_UNTRUNCATED_FULL).coeffs()
    assert c2["range_max_err"] < 1e-2


def test_batch_and_server_argument_checks_without_gpu():
    import ctypes as C
    L = bf.lib()
    assert L.bf_filter_batch(None, None, 0, None) == 0          # empty batch is a no-op
    assert L.bf_filter_batch(None, None, -1, None) == 1
    assert L.bf_filter_batch(None, None, 2, None) == 1
    p = bf.Plan(device=-1)
    plans = (C.c_void_p * 1)(p.handle.value)
    imgs = (bf._binding.bf_image * 1)(bf._binding.bf_image(4096, 256, 1 << 20, 256, 4, 64))
    assert L.bf_filter_batch(plans, imgs, 1, None) == 9          # host-only plan
    # the batch autotuner takes the same arguments and checks them the same way
    assert L.bf_autotune_batch(None, None, 0, None) == 0
    assert L.bf_autotune_batch(None, None, -1, None) == 1
    assert L.bf_autotune_batch(None, None, 2, None) == 1
    assert L.bf_autotune_batch(plans, imgs, 1, None) == 9
    p3 = bf.Plan(device=-1, policy=bf.RANGE_PAPER_3D)
    plans3 = (C.c_void_p * 1)(p3.handle.value)
    assert L.bf_autotune_batch(plans3, imgs, 1, None) == 9        # device checked before the form
    cfg = bf._binding.bf_serve_config(0, 0, 0, 0, 0)
    h = C.c_void_p()
    assert L.bf_serve_create(C.byref(cfg), C.byref(h)) == 9      # no device here
    assert L.bf_serve_create(None, C.byref(h)) == 1
    assert L.bf_serve_submit(None, None, None) == 1
    assert L.bf_serve_poll(None, 1, 0, None) == 1
    L.bf_serve_destroy(None)


def test_launch_info_and_autotune_without_gpu():
    p = bf.Plan(device=-1)
    info = bf.bf_launch_info(p, 1080, 1920)
    assert info["threads"] <= 512 and info["tw"] % 8 == 0 and info["groups"] >= 1
    assert info["threads"] >= info["tw"] + 2 * 12
    with pytest.raises(bf.BFError) as ei:
        bf.bf_autotune(p, 64, 64)
    assert ei.value.status == 9


def test_group_autotune_argument_checks_without_gpu():
    import ctypes as C
    p, q = bf.Plan(device=-1), bf.Plan(device=-1, sigma_s=8.0)
    for plans, h, w, ns, status in [([p, q], 64, 64, 3, 9),      # host-only plans: no device to time on
                                    ([], 64, 64, 3, 1),          # no plans
                                    ([p], 64, 64, 0, 1),         # stream count out of range
                                    ([p], 64, 64, 17, 1),
                                    ([p], 0, 64, 1, 1)]:
        with pytest.raises(bf.BFError) as ei:
            bf.bf_autotune_group(plans, h, w, n_streams=ns)
        assert ei.value.status == status, (len(plans), h, ns)
    hs = (C.c_void_p * 2)(p.handle, None)
    assert bf.lib().bf_autotune_group(hs, 2, 64, 64, 2, None) == 1   # a null plan
    assert bf.lib().bf_autotune_group(None, 1, 64, 64, 2, None) == 1


def test_image_autotune_argument_checks_without_gpu():
    # no pointer is dereferenced: every call returns at its argument or device check
    L, p = bf.lib(), bf.Plan(device=-1)
    fake = 1 << 40
    assert L.bf_autotune_image(p.handle, None, 256, 64, 64, None, None) == 1       # no image
    assert L.bf_autotune_image(p.handle, fake, 255, 64, 64, None, None) == 1       # pitch not a multiple of 4
    assert L.bf_autotune_image(p.handle, fake, 252, 64, 64, None, None) == 1       # pitch below width * 4
    assert L.bf_autotune_image(p.handle, fake, 256, 0, 64, None, None) == 1        # empty
    assert L.bf_autotune_image(p.handle, fake, 256, 64, 64, None, None) == 9       # host-only plan
    assert L.bf_autotune_image(None, fake, 256, 64, 64, None, None) == 1           # no plan


def test_launch_candidates_and_pinning_host_only():
    # host-only plan: the geometry table is keyed without a device
    plan = bf.Plan(device=-1, sigma_s=32.0, sigma_r=0.3)
    H, W = 1080, 1913
    cands = bf.bf_launch_candidates(plan, H, W)
    assert len(cands) > 10
    assert set(cands[0]) == set(bf._binding.INFO_KEYS)
    default = bf.bf_launch_info(plan, H, W)
    assert default == cands[0]                                   # the cost model's first choice
    assert all(c["ncols"] >= c["tw"] + 2 * 96 and c["ncols"] % 32 == 0 for c in cands)  # R = 96 each side
    assert all(c["threads"] == c["ncols"] + 64 and c["threads"] <= 512 for c in cands)
    assert {c["depth"] for c in cands} == {2, 3}
    assert {c["ring"] for c in cands} == {0}      # a ring of 2R + 2 rows does not fit shared memory at R = 96
    small = bf.bf_launch_candidates(bf.Plan(device=-1, sigma_s=8.0), H, W)
    assert {c["ring"] for c in small} == {0, 1}
    assert all(c["smem"] <= 227 * 1024 for c in cands + small)
    other = next(c for c in cands if (c["tw"], c["th"], c["ring"]) != (default["tw"], default["th"], default["ring"]))
    keys = ("tw", "th", "nk", "ring", "depth", "ncols")
    try:
        bf.bf_set_launch(plan, H, W, other)
        got = bf.bf_launch_info(plan, H, W)
        assert {k: got[k] for k in keys} == {k: other[k] for k in keys}
        bad = dict(other, tw=other["tw"] + 3)
        with pytest.raises(bf.BFError) as ei:
            bf.bf_set_launch(plan, H, W, bad)
        assert ei.value.status == 1
    finally:
        bf.bf_set_launch(plan, H, W, default)
    assert bf.bf_launch_info(plan, H, W) == default
    assert len(bf.bf_launch_candidates(plan, H, W, max_n=3)) == 3


def test_tune_cache_file_round_trip(tmp_path):
    # a pinned geometry is appended to BF_TUNE_CACHE and read back by a fresh process
    cache = tmp_path / "tune.txt"
    code = r'''
import json, sys
import paper_1803_00004_gb300 as bf
mode = sys.argv[1]
out = {}
for ss in (2.0, 8.0, 32.0):
    plan = bf.Plan(device=-1, sigma_s=ss)
    if mode == "write":
        cands = bf.bf_launch_candidates(plan, 720, 1280)
        bf.bf_set_launch(plan, 720, 1280, cands[3])
    out[str(ss)] = bf.bf_launch_info(plan, 720, 1280)
print(json.dumps(out))
'''
    import json
    import subprocess
    import sys
    env = dict(os.environ, BF_TUNE_CACHE=str(cache), PYTHONPATH=ROOT)
    w = subprocess.run([sys.executable, "-c", code, "write"], env=env, capture_output=True, text=True, check=True)
    r = subprocess.run([sys.executable, "-c", code, "read"], env=env, capture_output=True, text=True, check=True)
    written, read = json.loads(w.stdout), json.loads(r.stdout)
    assert written == read
    lines = cache.read_text().splitlines()
    assert len(lines) == 3 and all(len(x.split()) == 21 for x in lines)
    fresh = json.loads(subprocess.run([sys.executable, "-c", code, "read"], env=dict(os.environ, PYTHONPATH=ROOT),
                                      capture_output=True, text=True, check=True).stdout)
    assert fresh != read                               # without the file: the cost model's choice


@pytest.mark.parametrize("kw", [dict(sigma_s=8.0, sigma_r=0.1, nr_terms=16), dict(sigma_s=8.0, sigma_r=0.3, nr_terms=16),
                                dict(sigma_s=4.0, sigma_r=0.05, nr_terms=32), dict(range=bf.KERNEL_BOX, sigma_r=0.2, nr_terms=10),
                                dict(sigma_s=4.0, nr_terms=8)])
def test_term_groups_cover_the_selection(kw):
    """A launch evaluates groups of NK consecutive frequencies (zero weight where nothing was selected); the
    groups cover the selected terms greedily from the smallest uncovered frequency."""
    plan = bf.Plan(device=-1, **kw)
    k = list(plan.coeffs()["k"])

    def greedy(nk):
        groups, i = 0, 0
        while i < len(k):
            k0 = k[i]
            groups += 1
            while i < len(k) and k[i] < k0 + nk:
                i += 1
        return groups

    def hybrid(nk):
        # packed windows: the first from the lowest frequency, then every window of nk consecutive selected
        # frequencies, greedily; the other terms in slices of nk
        gp, rest, i = 0, 0, 0
        while i < len(k):
            if i == 0 or (i + nk <= len(k) and k[i + nk - 1] - k[i] == nk - 1):
                k0, gp = k[i], gp + 1
                while i < len(k) and k[i] < k0 + nk:
                    i += 1
            else:
                rest, i = rest + 1, i + 1
        assert rest > 0
        return gp + -(-rest // nk)

    # packed family: greedy windows; scalar family (offered only for gapped selections): slices of NK terms;
    # hybrid (gapped selections): the first window packed, then slices of NK of the terms above it
    consecutive = k == list(range(k[0], k[0] + len(k)))
    seen = set()
    for c in bf.bf_launch_candidates(plan, 300, 500):
        if c["packed"] == 1:
            assert c["groups"] == greedy(c["nk"]) and c["groups"] * c["nk"] <= 128 and c["nk"] % 2 == 0
        elif c["packed"] == 2:
            assert not consecutive and c["nk"] % 2 == 0
            assert c["groups"] == hybrid(c["nk"]) and c["launches"] == 2
        else:
            assert not consecutive and c["packed"] == 0 and c["groups"] == -(-len(k) // c["nk"])
        seen.add((c["packed"], c["nk"]))
    assert {f for f, _ in seen} == ({1} if consecutive else {0, 1, 2})
    if consecutive:                                    # ceil(N_r / NK) groups
        assert all(greedy(nk) == -(-len(k) // nk) for _, nk in seen)


def test_precompute_argument_checks_without_gpu():
    L = bf.lib()
    out = C.c_void_p(123)
    host = bf.Plan(device=-1, t_r=0.6)
    assert L.bf_precompute(host.handle, 4096, 256, 4, 64, 1, 0, None, C.byref(out)) == 1      # kmax < 2
    assert out.value is None
    assert L.bf_precompute(host.handle, 4096, 256, 4, 64, 200, 0, None, C.byref(out)) == 1    # kmax > 128
    assert L.bf_precompute(host.handle, 4096, 100, 4, 64, 16, 0, None, C.byref(out)) == 1     # pitch < width * 4
    assert L.bf_precompute(host.handle, 4096, 256, 4, 64, 16, 3, None, C.byref(out)) == 1     # unknown precision
    assert L.bf_precompute(host.handle, 4096, 256, 4, 64, 16, 0, None, C.byref(out)) == 9     # host-only plan
    assert L.bf_filter_cached(None, host.handle, 4096, 256, 1 << 20, 256, None) == 1
    L.bf_cache_destroy(None)                                                                # no-op
    assert L.bf_cache_bytes(None) == 0


def _random_descs(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        spatial = int(rng.choice([bf.KERNEL_GAUSSIAN, bf.KERNEL_BOX, bf.KERNEL_EXPONENTIAL]))
        kw = dict(spatial=spatial, sigma_s=float(rng.uniform(0.6, 12.0)), ns_terms=int(rng.choice([1, 2, 3, 5, 9, 13, 25])),
                  range=int(rng.integers(0, 3)), sigma_r=float(rng.uniform(0.03, 0.5)),
                  nr_terms=int(rng.integers(1, 17)), policy=int(rng.choice([bf.RANGE_TRUNCATED_MIN_PERIOD,
                                                                             bf.RANGE_UNTRUNCATED_FULL])))
        if rng.random() < 0.3:
            kw["radius"] = int(rng.integers(1, 20))
        if spatial == bf.KERNEL_EXPONENTIAL:  # the oracle's 2-D quadrature grows with 4^J: keep R <= 12
            kw["sigma_s"] = min(kw["sigma_s"], 4.0)
            kw["radius"] = min(kw.get("radius", 12), 12)
        out.append(kw)
    return out


@pytest.mark.parametrize("kw", _random_descs(40, 7))
def test_random_plans_match_oracle(kw):
    """Seeded random descriptors: the product's plan (selections, coefficients, kernel table, windows) equals
    the oracle's, or both reject it; the compiled windows reproduce the kernel."""
    try:
        o = O.plan_info(_odesc(kw))
    except ValueError:
        o = None
    try:
        p = bf.Plan(device=-1, **kw)
    except bf.BFError as e:
        # the product may reject what the oracle evaluates (more than 6 box windows per axis, more than 64
        # terms), never the other way round
        assert e.status == 2, (kw, e)
        return
    assert o is not None, kw
    c = p.coeffs()
    order = np.argsort(o.ks)
    assert list(c["k"]) == list(o.ks[order]), kw
    assert np.max(np.abs(np.array(c["a"]) - o.ak[order])) < 1e-13
    assert [list(t) for t in c["haar_terms"]] == [list(t) for t in o.terms]
    assert np.max(np.abs(np.array(c["kernel"]) - o.Ks)) < 1e-13 * max(1.0, np.max(np.abs(o.Ks)))
    R, K = c["radius"], np.array(c["kernel"])
    rec = np.zeros_like(K)
    for v, (v0, v1) in enumerate(c["vwin"]):
        for h, (u0, u1) in enumerate(c["hwin"]):
            rec[v0 + R:v1 + R + 1, u0 + R:u1 + R + 1] += c["wcoef"][v][h]
    assert np.max(np.abs(rec - K[::-1, ::-1])) < 1e-12 * max(1.0, np.max(np.abs(K)))


def test_basis_storage_of_the_geometries_follows_the_precision():
    """fp32 plans compute the basis in the kernel or read an fp32 pre-pass; fp16 / bf16 plans (16-bit basis
    storage) read the pre-pass in their format, in the packed family without the ring."""
    for prec, allowed in ((bf.PREC_FP32, {0, 1}), (bf.PREC_FP16, {2}), (bf.PREC_BF16, {3})):
        plan = bf.Plan(device=-1, sigma_s=8.0, precision=prec)
        cands = bf.bf_launch_candidates(plan, 1080, 1920)
        seen = {c["pre"] for c in cands}
        assert seen == allowed, (prec, seen)
        assert all(c["packed"] == 1 and c["ring"] == 0 for c in cands if c["pre"])
        info = bf.bf_launch_info(plan, 1080, 1920)
        assert info["pre"] in allowed
        # the pre-pass buffer is scratch: 16 bytes per pixel in fp32, 8 in 16 bits
        if info["pre"]:
            assert info["scratch_kib"] * 1024 >= (16 if info["pre"] == 1 else 8) * 1080 * 1920 - 1024
