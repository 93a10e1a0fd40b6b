"""bf_filter_host (one host image, several plans, copies inside the call) against bf_filter on device buffers
and against the oracle; repeated calls from two streams, pitched host buffers, and a call that grows the
library's device block.  Needs a GPU."""
import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
from paper_1803_00004_gb300 import synth
from parity import conditioned_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00004_gb300 import _build
    _build.build()
    torch.cuda.init()


def device_ref(plan, img):
    src = torch.from_numpy(img).cuda()
    dst = torch.empty_like(src)
    bf.bf_filter(plan, src, dst)
    torch.cuda.synchronize()
    return dst.cpu()


def test_host_call_matches_device_filter_and_oracle():
    img = synth.shapes(300, 517, 51, scale=0.3)
    kws = [dict(sigma_s=ss, sigma_r=sr) for ss in (2.0, 8.0) for sr in (0.05, 0.3)] + [dict(sigma_s=4.0, nr_terms=16)]
    plans = [bf.Plan(device=0, **kw) for kw in kws]
    h_in = torch.from_numpy(img).pin_memory()
    outs = [torch.full(img.shape, float("nan")).pin_memory() for _ in plans]
    s = torch.cuda.Stream()
    for _ in range(2):  # the second call reuses the library's block
        bf.bf_filter_host(plans, h_in, outs, n_streams=3, stream=s)
        s.synchronize()
        for p, o, kw in zip(plans, outs, kws):
            assert torch.equal(o, device_ref(p, img))  # same geometry, same arithmetic
    e_good, worst, _ = conditioned_check(outs[-1].numpy().astype(np.float64), img, kws[-1])
    assert e_good < 1e-5 and worst < 1.0


def test_host_calls_from_two_streams_and_a_larger_image():
    plans = [bf.Plan(device=0, sigma_s=3.0), bf.Plan(device=0, sigma_s=12.0, nr_terms=12)]
    small = synth.blocks(200, 240, 52)
    big = synth.shapes(700, 900, 53, scale=0.6)  # grows the device block
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    res = []
    for img, st in ((small, a), (big, b), (small, b)):
        h_in = torch.from_numpy(img).pin_memory()
        outs = [torch.empty(img.shape).pin_memory() for _ in plans]
        bf.bf_filter_host(plans, h_in, outs, n_streams=2, stream=st)
        res.append((img, outs))
    torch.cuda.synchronize()
    for img, outs in res:
        for p, o in zip(plans, outs):
            assert torch.equal(o, device_ref(p, img))


def test_host_call_pitched_buffers_and_errors():
    img = synth.shapes(120, 200, 54, scale=0.2)
    plan = bf.Plan(device=0)
    big_in = torch.zeros((120, 232)).pin_memory()
    big_in[:, :200] = torch.from_numpy(img)
    big_out = torch.full((120, 248), float("nan")).pin_memory()
    bf.bf_filter_host([plan], big_in[:, :200], [big_out[:, :200]])
    torch.cuda.synchronize()
    assert torch.equal(big_out[:, :200], device_ref(plan, img))
    assert torch.isnan(big_out[:, 200:]).all()
    with pytest.raises(bf.BFError) as ei:
        bf.bf_filter_host([plan], big_in[:, :200], [big_out[:, :200]], n_streams=17)
    assert ei.value.status == bf.ERR_INVALID_ARG


def test_host_calls_alternating_streams_overlap_without_mixing_images():
    # consecutive calls on two streams use the library's two device blocks in turn and overlap on the GPU; every
    # call's outputs must still be its own image's, also when a block grows in the middle of the run
    plans = [bf.Plan(device=0, sigma_s=ss, sigma_r=0.1) for ss in (2.0, 6.0, 16.0)]
    imgs = [synth.shapes(360, 480, 60 + i, scale=0.4) for i in range(3)] + [synth.blocks(420, 560, 63)]
    order = [0, 1, 2, 0, 3, 1, 3, 2]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    res = []
    for k, ii in enumerate(order):
        h_in = torch.from_numpy(imgs[ii]).pin_memory()
        outs = [torch.full(imgs[ii].shape, float("nan")).pin_memory() for _ in plans]
        bf.bf_filter_host(plans, h_in, outs, n_streams=3, stream=streams[k % 2])
        res.append((ii, h_in, outs))
    torch.cuda.synchronize()
    refs = {}
    for ii, _, outs in res:
        if ii not in refs:
            refs[ii] = [device_ref(p, imgs[ii]) for p in plans]
        for o, r in zip(outs, refs[ii]):
            assert torch.equal(o, r)
