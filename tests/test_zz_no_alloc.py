"""bf_filter_noalloc: the allocation-free variant of bf_filter for callers that
cannot allocate device memory while filtering (hosts that reserve all device
memory up front).  Called through the C ABI, it must give bf_filter's result
within the fp32 bar, on two calls in a row that share its fixed scratch array,
and reject images whose partial planes exceed that array.  Needs a GPU."""
import ctypes as C

import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
from paper_1803_00004_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00004_gb300 import _build
    _build.build()


def noalloc(plan, src, dst):
    L = bf.lib()
    st = L.bf_filter_noalloc(plan.handle, src.data_ptr(), src.stride(0) * 4, dst.data_ptr(), dst.stride(0) * 4,
                             src.shape[0], src.shape[1], C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_matches_bf_filter_twice():
    # two grouped plans (16 and 32 cosine terms: partial planes in the fixed array)
    # and images of different sizes, one call after the other
    cases = [(synth.shapes(300, 450, 21, scale=0.3), dict(sigma_s=8.0, sigma_r=0.05, nr_terms=16)),
             (synth.blocks(517, 211, 22), dict(sigma_s=4.0, sigma_r=0.1, nr_terms=32))]
    for img, kw in cases:
        plan = bf.Plan(device=0, **kw)
        assert bf.bf_launch_info(plan, *img.shape)["groups"] > 1
        src = torch.from_numpy(img).cuda()
        ref = torch.empty_like(src)
        bf.bf_filter(plan, src, ref)
        got = torch.full_like(src, float("nan"))
        assert noalloc(plan, src, got) == 0
        torch.cuda.synchronize()
        assert torch.max(torch.abs(got - ref)).item() < TOL


def test_noalloc_rejects_oversized_scratch():
    # 4 term groups x 2 planes x 2048 x 2048 floats = 128 MiB > the 64 MiB array
    plan = bf.Plan(device=0, sigma_s=4.0, nr_terms=32)
    src = torch.zeros((2048, 2048), device="cuda")
    dst = torch.empty_like(src)
    assert noalloc(plan, src, dst) == 8
    assert "64 MiB" in bf.lib().bf_last_error().decode()


def test_noalloc_3d_form_matches_bf_filter():
    # the 3-D form keeps its slice work list (and partial planes of 2 term groups) in the fixed array
    img = synth.shapes(260, 390, 23, scale=0.3)
    for nr in (8, 12):
        plan = bf.Plan(device=0, sigma_s=3.0, sigma_r=0.1, nr_terms=nr, policy=bf.RANGE_PAPER_3D, z_bins=256)
        src = torch.from_numpy(img).cuda()
        ref = torch.empty_like(src)
        bf.bf_filter(plan, src, ref)
        got = torch.full_like(src, float("nan"))
        assert noalloc(plan, src, got) == 0
        torch.cuda.synchronize()
        assert torch.max(torch.abs(got - ref)).item() < TOL
