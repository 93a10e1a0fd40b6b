"""Every launch-geometry family of the fused filter against the oracle: basis
inputs recomputed or kept in a per-column shared-memory ring, exchange depth 2
or 3, and each cosine-terms-per-CTA split.  The geometry changes only the
rounding order of Eq. (36)'s sums, so each must meet the same bar.  Needs a GPU."""
import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
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


def family(c):
    return (c["packed"], c["ring"], c["depth"], c["nk"], c["pre"])


CASES = [
    ("sigma8_700w", synth.shapes(300, 700, 31, scale=0.3), dict(sigma_s=8.0, sigma_r=0.1)),
    ("sigma32_900w", synth.shapes(200, 900, 32, scale=0.4), dict(sigma_s=32.0, sigma_r=0.3)),
    ("sigma2_groups", synth.shapes(150, 401, 33, scale=0.2), dict(sigma_s=2.0, sigma_r=0.05, nr_terms=16)),
    ("m3_ragged", synth.uniform(77, 301, 34), dict(sigma_s=3.0, ns_terms=7, nr_terms=5)),
    ("nr32_partials", synth.shapes(130, 517, 35, scale=0.2), dict(sigma_s=8.0, sigma_r=0.05, nr_terms=32)),
    ("narrow", synth.blocks(190, 70, 36), dict(sigma_s=4.0)),
    ("nonconsecutive_terms", synth.shapes(160, 300, 38, scale=0.2), dict(range=bf.KERNEL_BOX, sigma_r=0.2, nr_terms=10)),
]


@pytest.mark.parametrize("name,img,kw", CASES, ids=[c[0] for c in CASES])
def test_every_geometry_family_matches_oracle(name, img, kw):
    H, W = img.shape
    plan = bf.Plan(device=0, **kw)
    default = bf.bf_launch_info(plan, H, W)
    cands = bf.bf_launch_candidates(plan, H, W)
    firsts = {}
    for c in cands:
        firsts.setdefault(family(c), c)
    assert len(firsts) >= 2, name
    src = torch.from_numpy(img).cuda()
    ran = []
    try:
        for fam, c in firsts.items():
            bf.bf_set_launch(plan, H, W, c)
            assert family(bf.bf_launch_info(plan, H, W)) == fam
            dst = torch.full_like(src, float("nan"))
            bf.bf_filter(plan, src, dst)
            torch.cuda.synchronize()
            got = dst.cpu().numpy().astype(np.float64)
            e_good, worst, nbad = conditioned_check(got, img, kw)
            assert e_good < TOL, "%s %s: max err %.3g" % (name, fam, e_good)
            assert worst < 1.0, "%s %s: %d ill-conditioned pixels, error / bound %.3g" % (name, fam, nbad, worst)
            ran.append(fam)
    finally:
        bf.bf_set_launch(plan, H, W, default)
    assert len(ran) == len(firsts)
