"""bf_filter_batch (persistent work-list launch, CUDA-graph replay) and the
serving loop (continuous batching): every image's result equals the lone
bf_filter result within the fp32 bar, alone and in the mix (needs a GPU)."""
import time

import numpy as np
import pytest

import paper_1803_00004_gb300 as bf
from oracle import oracle as O
from paper_1803_00004_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
# alone vs in the mix: different tile geometries round differently; each result is
# within TOL of the oracle, so the two are within 2 TOL of each other
MIX_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00004_gb300 import _build
    _build.build()


def mixed_workload(n, lo, hi, seed):
    """Images with log-uniform sides and per-image kernel parameters (Gaussian or
    exponential range kernel, N_r in {8, 16})."""
    rng = np.random.default_rng(seed)
    sides = synth.batch_sizes(n, lo, hi, seed=seed)
    out = []
    for i, s in enumerate(sides):
        h = max(1, int(s * rng.uniform(0.6, 1.0)))
        img = synth.shapes(h, s, seed=seed * 1000 + i, scale=s / 1080.0)
        kw = dict(sigma_s=float(rng.uniform(2, 32)), sigma_r=float(rng.uniform(0.05, 0.3)),
                  range=int(rng.integers(0, 2)), nr_terms=int(rng.choice([8, 16])))
        out.append((img, kw))
    return out


def alone(img, kw):
    plan = bf.Plan(device=0, **kw)
    src = torch.from_numpy(img).cuda()
    dst = torch.empty_like(src)
    bf.bf_filter(plan, src, dst)
    torch.cuda.synchronize()
    return dst.cpu().numpy()


def test_batch_matches_single_image_results():
    work = mixed_workload(24, 64, 512, seed=3)
    plans = [bf.Plan(device=0, **kw) for _, kw in work]
    srcs = [torch.from_numpy(img).cuda() for img, _ in work]
    dsts = [torch.full_like(s, float("nan")) for s in srcs]
    bf.bf_filter_batch(plans, srcs, dsts)
    torch.cuda.synchronize()
    for (img, kw), d in zip(work, dsts):
        ref = alone(img, kw)
        assert np.max(np.abs(d.cpu().numpy() - ref)) < MIX_TOL, kw


def test_batch_against_oracle_small():
    work = mixed_workload(6, 40, 160, seed=5)
    plans = [bf.Plan(device=0, **kw) for _, kw in work]
    srcs = [torch.from_numpy(img).cuda() for img, _ in work]
    dsts = [torch.empty_like(s) for s in srcs]
    bf.bf_filter_batch(plans, srcs, dsts)
    torch.cuda.synchronize()
    for (img, kw), d in zip(work, dsts):
        ref, _ = O.approx_fast(img.astype(np.float64), O.Desc(**kw), threads=16)
        assert np.max(np.abs(d.cpu().numpy() - ref)) < TOL


def test_graph_replay_tracks_new_input():
    work = mixed_workload(5, 100, 300, seed=7)
    plans = [bf.Plan(device=0, **kw) for _, kw in work]
    srcs = [torch.from_numpy(img).cuda() for img, _ in work]
    dsts = [torch.empty_like(s) for s in srcs]
    bf.bf_filter_batch(plans, srcs, dsts)
    first = [d.clone() for d in dsts]
    bf.bf_filter_batch(plans, srcs, dsts)           # replay: same result
    torch.cuda.synchronize()
    for a, b in zip(first, dsts):
        assert torch.equal(a, b)
    for s in srcs:                                   # new pixels in the same buffers
        s.copy_(torch.flip(s, dims=[1]))
    bf.bf_filter_batch(plans, srcs, dsts)
    torch.cuda.synchronize()
    for (img, kw), d in zip(work, dsts):
        ref = alone(np.ascontiguousarray(img[:, ::-1]), kw)
        assert np.max(np.abs(d.cpu().numpy() - ref)) < MIX_TOL


def test_batch_edge_cases():
    p = bf.Plan(device=0)
    a = torch.rand(33, 17, device="cuda")
    e = torch.empty(0, 5, device="cuda")
    out = torch.empty_like(a)
    bf.bf_filter_batch([p, p], [e, a], [torch.empty_like(e), out])  # empty image is skipped
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - alone(a.cpu().numpy(), {}))) < MIX_TOL
    bf.bf_filter_batch([], [], [])
    with pytest.raises(bf.BFError):
        bf.bf_filter_batch([p], [a], [a])              # in place
    with pytest.raises(bf.BFError):
        bf.bf_filter_batch([bf.Plan(device=-1)], [a], [out])


# ---------------------------------------------------------------- serving

def pinned(img):
    t = torch.from_numpy(img).pin_memory()
    return t, torch.empty_like(t).pin_memory()


def test_server_results_equal_alone_under_concurrency():
    work = mixed_workload(40, 64, 768, seed=11)
    srv = bf.Server(max_slots=8, n_streams=3, max_batch=6)
    bufs = [pinned(img) for img, _ in work]
    tickets = []
    rng = np.random.default_rng(0)
    for (img, kw), (hin, hout) in zip(work, bufs):
        d = bf.desc(**kw)
        tickets.append(srv.submit(d, hin.data_ptr(), hout.data_ptr(), img.shape[0], img.shape[1]))
        time.sleep(float(rng.exponential(0.0005)))  # Poisson arrivals while earlier requests run
    lat = []
    for t in tickets:
        st, r = srv.poll(t, -1)
        assert st == 0 and r.status == 0
        lat.append(r.latency_ms)
    for (img, kw), (hin, hout) in zip(work, bufs):
        assert np.max(np.abs(hout.numpy() - alone(img, kw))) < MIX_TOL
    srv.close()
    assert all(x > 0 for x in lat)


def test_server_admission_cancel_timeout_and_errors():
    img = synth.shapes(512, 512, 1, scale=0.5)
    need = 2 * img.nbytes
    srv = bf.Server(hbm_budget_bytes=int(need * 1.6), max_slots=4, n_streams=2)
    big = synth.shapes(1024, 1024, 2)
    hb_in, hb_out = pinned(big)
    with pytest.raises(bf.BFError) as ei:                 # can never fit the budget
        srv.submit(bf.desc(), hb_in.data_ptr(), hb_out.data_ptr(), 1024, 1024)
    assert ei.value.status == 5
    bufs = [pinned(img) for _ in range(6)]
    ts = [srv.submit(bf.desc(sigma_s=8.0), i.data_ptr(), o.data_ptr(), 512, 512) for i, o in bufs]
    st, _ = srv.poll(ts[-1], 0)                             # just submitted: still in flight
    assert st == 6
    st_cancel = srv.cancel(ts[-1])                          # budget admits one at a time: last is pending
    st, r = srv.poll(ts[-1], -1)
    if st_cancel == 0:
        assert st == 11
    for t in ts[:-1]:
        st, r = srv.poll(t, -1)
        assert st == 0 and r.status == 0
    ref = alone(img, dict(sigma_s=8.0))
    for i, o in bufs[:-1]:
        assert np.max(np.abs(o.numpy() - ref)) < MIX_TOL
    assert srv.poll(123456789, 0)[0] == 10                  # unknown ticket
    # an injected launch failure fails that request only; the server keeps serving
    bf.bf_debug_fail_launches(1)
    t = srv.submit(bf.desc(), bufs[0][0].data_ptr(), bufs[0][1].data_ptr(), 512, 512)
    st, r = srv.poll(t, -1)
    assert st == 0 and r.status == 4
    t = srv.submit(bf.desc(), bufs[0][0].data_ptr(), bufs[0][1].data_ptr(), 512, 512)
    st, r = srv.poll(t, -1)
    assert st == 0 and r.status == 0
    srv.close()


def test_server_destroy_with_pending_requests():
    srv = bf.Server(max_slots=1, n_streams=1)
    img = synth.blocks(256, 256, 0)
    bufs = [pinned(img) for _ in range(5)]
    for i, o in bufs:
        srv.submit(bf.desc(), i.data_ptr(), o.data_ptr(), 256, 256)
    srv.close()  # drains admitted work, cancels the rest; must return


def test_batch_autotune_keeps_results_within_the_bar():
    """bf_autotune_batch times this batch under the candidate geometries of each class: its own outputs, and
    those of bf_filter_batch afterwards (re-captured with the tuned geometry), match the oracle."""
    work = mixed_workload(8, 40, 220, seed=11)
    plans = [bf.Plan(device=0, **kw) for _, kw in work]
    srcs = [torch.from_numpy(img).cuda() for img, _ in work]
    refs = [O.approx_fast(img.astype(np.float64), O.Desc(**kw), threads=16)[0] for img, kw in work]
    dsts = [torch.full_like(s, float("nan")) for s in srcs]
    bf.bf_filter_batch(plans, srcs, dsts)        # a graph captured before tuning must not be replayed after it
    bf.bf_autotune_batch(plans, srcs, dsts)
    torch.cuda.synchronize()
    for d, ref in zip(dsts, refs):
        assert np.max(np.abs(d.cpu().numpy() - ref)) < TOL
    dsts = [torch.full_like(s, float("nan")) for s in srcs]
    bf.bf_filter_batch(plans, srcs, dsts)
    torch.cuda.synchronize()
    for d, ref in zip(dsts, refs):
        assert np.max(np.abs(d.cpu().numpy() - ref)) < TOL


def test_server_device_pointer_requests_with_pitches():
    """Requests on caller-owned device buffers with row pitches wider than the image: the server filters in to
    out without staging; each result equals bf_filter's within the bar, and the padding stays untouched."""
    srv = bf.Server(max_slots=8, n_streams=2, max_batch=4)
    work = mixed_workload(6, 64, 400, seed=21)
    bufs, tickets = [], []
    for img, kw in work:
        H, W = img.shape
        big_in = torch.zeros((H, W + 24), device="cuda")
        big_in[:, :W] = torch.from_numpy(img).cuda()
        big_out = torch.full((H, W + 40), float("nan"), device="cuda")
        torch.cuda.synchronize()
        tickets.append(srv.submit(bf.desc(**kw), big_in.data_ptr(), big_out.data_ptr(), H, W,
                                  in_pitch=big_in.stride(0) * 4, out_pitch=big_out.stride(0) * 4,
                                  memory=bf.MEM_DEVICE))
        bufs.append((big_in, big_out))
    for t, (img, kw), (_, big_out) in zip(tickets, work, bufs):
        st, r = srv.poll(t, -1)
        assert st == 0 and r.status == 0
        W = img.shape[1]
        got = big_out[:, :W].cpu().numpy()
        assert np.max(np.abs(got - alone(img, kw))) < MIX_TOL
        assert torch.isnan(big_out[:, W:]).all()
    srv.close()


def test_server_plan_build_is_inside_the_latency():
    """A request with parameters the server has not seen: its plan is built after submission, and the
    reported latency covers the plan build and the queueing."""
    srv = bf.Server(max_slots=4, n_streams=1)
    img = synth.shapes(256, 256, 3, scale=0.3)
    hin, hout = pinned(img)
    t = srv.submit(bf.desc(sigma_s=27.3, sigma_r=0.137), hin.data_ptr(), hout.data_ptr(), 256, 256)
    st, r = srv.poll(t, -1)
    assert st == 0 and r.status == 0
    assert r.plan_ns > 0 and r.queue_ns >= r.plan_ns and r.latency_ns >= r.queue_ns
    assert np.max(np.abs(hout.numpy() - alone(img, dict(sigma_s=27.3, sigma_r=0.137)))) < MIX_TOL
    # a plan error is reported by poll
    t = srv.submit(bf.desc(sigma_s=-1.0), hin.data_ptr(), hout.data_ptr(), 256, 256)
    st, r = srv.poll(t, -1)
    assert st == 0 and r.status == bf.ERR_INVALID_ARG
    srv.close()


def test_server_mixed_memory_precision_and_3d_requests():
    """Host and device-pointer requests, fp32, 16-bit basis and 3-D plans arriving together: each result equals
    the same plan filtered alone by bf_filter (within the bar; bit-equal is not required, the batched launch may
    pick another geometry)."""
    rng = np.random.default_rng(31)
    srv = bf.Server(max_slots=16, n_streams=3, max_batch=5)
    jobs = []
    for i in range(18):
        s = int(rng.integers(48, 400))
        img = synth.shapes(s, s + int(rng.integers(0, 60)), 900 + i, scale=s / 1080.0)
        kind = i % 3
        kw = dict(sigma_s=float(rng.uniform(1.5, 12.0)), sigma_r=float(rng.uniform(0.05, 0.3)))
        if kind == 1:
            kw["precision"] = bf.PREC_FP16 if i % 2 else bf.PREC_BF16
        if kind == 2:
            kw.update(policy=bf.RANGE_PAPER_3D, z_bins=256, nr_terms=4)
        dev = bool(rng.integers(0, 2))
        H, W = img.shape
        if dev:
            src = torch.from_numpy(img).cuda()
            dst = torch.full_like(src, float("nan"))
            torch.cuda.synchronize()
            t = srv.submit(bf.desc(**kw), src.data_ptr(), dst.data_ptr(), H, W, memory=bf.MEM_DEVICE)
        else:
            src, dst = pinned(img)
            t = srv.submit(bf.desc(**kw), src.data_ptr(), dst.data_ptr(), H, W)
        jobs.append((t, img, kw, src, dst))
    for t, img, kw, src, dst in jobs:
        st, r = srv.poll(t, -1)
        assert st == 0 and r.status == 0, (kw, st, r.status)
        plan = bf.Plan(device=0, **kw)
        x = torch.from_numpy(img).cuda()
        y = torch.empty_like(x)
        bf.bf_filter(plan, x, y)
        torch.cuda.synchronize()
        got = dst.cpu().numpy() if dst.is_cuda else dst.numpy()
        assert np.max(np.abs(got - y.cpu().numpy())) < MIX_TOL, kw
    srv.close()
