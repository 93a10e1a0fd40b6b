"""The multi-GPU path of bench.py is replicas (no data exchange): each rank
times its own copy of the workload, the job time is the max over ranks and the
value counts every rank's pixels.  Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.reduce_max_ms(10.0 + 5.0 * rank)
    q.put((rank, m, bench.whole_job_value(1000.0, 4, m, world), bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v, env in got:
        assert m == 15.0
        assert abs(v - 2 * 1000.0 * 4 / 15e-3 / 1e6) < 1e-9
        assert env[0] == rank and env[1] == 2


def test_single_process_helpers():
    import bench
    assert bench.reduce_max_ms(3.5) == 3.5
    assert abs(bench.whole_job_value(2e6, 10, 100.0, 1) - 200.0) < 1e-9


def _run_bench(args, env_extra=None):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, capture_output=True, text=True,
                       timeout=600, env=env, cwd=root)
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return r.returncode, [json.loads(ln) for ln in lines]


def test_reference_arm_line():
    """`bench.py --impl reference` (the oracle on the host cores, each step the nine filters on a band) prints
    one JSON line with the contract's keys, the metric and workload of the GPU arm."""
    import bench
    rc, out = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert rc == 0 and len(out) == 1
    d = out[0]
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "Mpixel/s"
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    rc, out = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                         {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert rc == 0 and out == []


def test_roofline_op_count_of_the_benchmark_plans():
    """F = N_img (2 n_x + 2 n_xy + n_pm) + 4 (N_r - 1) + 6 k_max + 2 per pixel.  The five-term Gaussian of the
    benchmark (phi phi, phi psi_{1,+-1}, psi_{1,+-1} phi) has two box widths (2 T_s and T_s), three shapes and nine
    signed boxes; with N_r = 8 (k = 0..7) N_img = 30, so F = 30 * 19 + 28 + 42 + 2 = 642 at every sigma."""
    import bench
    import paper_1803_00004_gb300 as bf
    for ss in (2.0, 8.0, 32.0):
        c = bf.Plan(device=-1, sigma_s=ss, sigma_r=0.1, nr_terms=8, ns_terms=5).coeffs()
        assert bench.box_counts(c) == (2, 3, 9)
        assert bench.algorithmic_ops_per_pixel(c) == 642
    # a single box (N_s = 1): one width, one shape, one box
    c = bf.Plan(device=-1, sigma_s=4.0, sigma_r=0.1, nr_terms=8, ns_terms=1).coeffs()
    assert bench.box_counts(c) == (1, 1, 1)
    assert bench.algorithmic_ops_per_pixel(c) == 30 * 5 + 28 + 42 + 2
