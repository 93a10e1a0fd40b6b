"""bf_filter_noalloc: the variant of bf_filter for callers that cannot allocate
device memory while filtering (hosts that reserve all device memory up front,
such as a framework's caching allocator or a real-time loop).  Called through
the C ABI, it must match the FP64 oracle within the fp32 bar and bf_filter's
result, on two calls in a row that share its fixed scratch array; fall back to
a geometry whose scratch fits when the preferred one's does not; reject images
whose scratch fits no geometry with BF_ERR_SCRATCH; and take nothing from the
device's stream-ordered memory pool (which bf_filter's scratch comes from).
Needs a GPU.  This file runs last: it pins one launch geometry for an image
size no other test uses."""
import ctypes as C

import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
from oracle import oracle as O
from paper_1803_00004_gb300 import synth
from parity import conditioned_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00004_gb300 import _build
    _build.build()
    torch.cuda.init()


def noalloc(plan, src, dst):
    L = bf.lib()
    return L.bf_filter_noalloc(plan.handle, src.data_ptr(), src.stride(0) * 4, dst.data_ptr(), dst.stride(0) * 4,
                               src.shape[0], src.shape[1], C.c_void_p(torch.cuda.current_stream().cuda_stream))


def check_oracle(got, img, kw):
    e_good, worst, nbad = conditioned_check(got.cpu().numpy().astype(np.float64), img, kw)
    assert e_good < TOL, "max err %.3g on well-conditioned pixels" % e_good
    assert worst < 1.0, "%d ill-conditioned pixels, error / bound %.3g" % (nbad, worst)


def test_noalloc_matches_oracle_twice():
    # two grouped plans (16 and 32 cosine terms: partial planes in the fixed array) and images of different
    # sizes, one call after the other; each result against the oracle and against bf_filter
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
        check_oracle(got, img, kw)
        assert torch.max(torch.abs(got - ref)).item() < TOL


def test_noalloc_falls_back_to_a_geometry_that_fits():
    # pin a geometry of four term groups (4 x 2 planes of 2040 x 2056 floats = 134 MB, over the 64 MiB array);
    # bf_filter runs it with allocated scratch, bf_filter_noalloc must fall back to one that fits
    H, W = 2040, 2056
    kw = dict(sigma_s=2.0, sigma_r=0.1, nr_terms=8)
    plan = bf.Plan(device=0, **kw)
    four = [c for c in bf.bf_launch_candidates(plan, H, W) if c["groups"] == 4]
    assert four, "no four-group geometry"
    bf.bf_set_launch(plan, H, W, four[0])
    assert bf.bf_launch_info(plan, H, W)["scratch_kib"] * 1024 > 64 << 20
    img = synth.shapes(H, W, 24, scale=1.0)
    src = torch.from_numpy(img).cuda()
    ref = torch.empty_like(src)
    bf.bf_filter(plan, src, ref)
    for _ in range(2):
        got = torch.full_like(src, float("nan"))
        assert noalloc(plan, src, got) == 0, bf.lib().bf_last_error().decode()
        torch.cuda.synchronize()
        assert torch.max(torch.abs(got - ref)).item() < TOL
    check_oracle(got, img, kw)


def test_noalloc_rejects_oversized_scratch():
    # every geometry of 32 terms at 4096 x 4096 needs at least 4 groups x 2 planes x 64 MiB
    plan = bf.Plan(device=0, sigma_s=4.0, nr_terms=32)
    src = torch.zeros((4096, 4096), device="cuda")
    dst = torch.empty_like(src)
    assert noalloc(plan, src, dst) == bf.ERR_SCRATCH
    assert "64 MiB" in bf.lib().bf_last_error().decode()


def test_noalloc_3d_form_matches_oracle():
    # the 3-D form keeps its slice work list (and partial planes of 2 term groups) in the fixed array
    img = synth.shapes(260, 390, 23, scale=0.3)
    for nr in (8, 12):
        kw = dict(sigma_s=3.0, sigma_r=0.1, nr_terms=nr)
        plan = bf.Plan(device=0, policy=bf.RANGE_PAPER_3D, z_bins=256, **kw)
        src = torch.from_numpy(img).cuda()
        ref = torch.empty_like(src)
        bf.bf_filter(plan, src, ref)
        got = torch.full_like(src, float("nan"))
        assert noalloc(plan, src, got) == 0
        torch.cuda.synchronize()
        want = O.approx3d_direct(img.astype(np.float64), O.Desc(policy=O.PAPER_3D, **kw), 256, threads=8)[0]
        assert np.max(np.abs(got.cpu().numpy() - want)) < TOL
        assert torch.max(torch.abs(got - ref)).item() < TOL


def test_noalloc_takes_nothing_from_the_memory_pool():
    # bf_filter's scratch comes from the device's default stream-ordered pool; bf_filter_noalloc must leave the
    # pool's high-water mark of used bytes at zero
    cu = C.CDLL("libcuda.so.1")
    dev = C.c_int()
    assert cu.cuCtxGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(C.byref(pool), dev) == 0

    def attr(a):
        v = C.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, a, C.byref(v)) == 0
        return v.value

    def used_high():
        return attr(USED_MEM_HIGH)

    def reset():
        z = C.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, USED_MEM_HIGH, C.byref(z)) == 0

    img = synth.shapes(300, 450, 25, scale=0.3)
    plan = bf.Plan(device=0, sigma_s=8.0, sigma_r=0.05, nr_terms=16)
    src = torch.from_numpy(img).cuda()
    out = torch.empty_like(src)
    torch.cuda.synchronize()
    base = attr(USED_MEM_CURRENT)  # bytes other work holds from the pool (normally 0)
    reset()
    assert noalloc(plan, src, out) == 0
    torch.cuda.synchronize()
    assert used_high() == base
    bf.bf_filter(plan, src, out)  # the probe sees bf_filter's stream-ordered scratch
    torch.cuda.synchronize()
    assert used_high() > base
