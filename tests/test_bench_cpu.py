"""bench.py's host-side pieces without a GPU: the JSON configuration of the
workload and the bookkeeping that ties measured DRAM traffic to the kernel
sources it was measured on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_measured_traffic_matches_the_current_kernel_sources():
    """The default roofline line reports ncu traffic only for the kernel
    sources it was taken on; this fails when those sources change until the
    launch list is taken again and recorded."""
    key = (bench.kernel_source_hash(), "fp32", 8192, "pair")
    assert key in bench.MEASURED_TRAFFIC, key
    t = bench.MEASURED_TRAFFIC[key]
    algorithmic = 72 * 8192 * 8192
    assert 0.95 * algorithmic < t < 1.05 * algorithmic


def test_workload_config_names_the_workload():
    class A:
        n, precision = 8192, "fp32"
    cfg = bench.workload_config(A)
    assert cfg["workload"].startswith("8192x8192 periodic D2Q9 spinodal decomposition")
    assert cfg["nx"] == cfg["ny"] == 8192 and "L2" in cfg["l2"]


def _reference_lines(cmd):
    import json
    import subprocess
    env = dict(os.environ, MASTER_ADDR="127.0.0.1")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(s) for s in r.stdout.splitlines() if s.startswith("{")]


REF_ARGS = ["bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3",
            "--ref-side", "32"]


def _check_reference_line(d, n_gpus):
    assert d["impl"] == "reference" and d["n_gpus"] == n_gpus
    assert d["unit"] == "MLUPS" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 3 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("8192x8192 periodic D2Q9")


def test_reference_arm_prints_one_line():
    lines = _reference_lines([sys.executable, *REF_ARGS])
    assert len(lines) == 1
    _check_reference_line(lines[0], 1)


def test_reference_arm_under_torchrun_two_ranks():
    """Launched as for N = 2 (gloo on the host): rank 0 alone runs the oracle
    and prints; the other rank exits 0 without work."""
    lines = _reference_lines([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                              "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                              "--master-port", "29531", *REF_ARGS, "--gpus", "2"])
    assert len(lines) == 1
    _check_reference_line(lines[0], 2)


def _timing_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    w, r, _ = bench.dist_setup()
    bench.dist_barrier(w)
    slowest = bench.dist_max(10.0 + r, w)  # each rank's own time
    q.put((r, w, slowest))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    """The multi-rank timing of the bench: each rank's time is reduced to the
    slowest on the host (gloo), so rank 0 reports whole-job time."""
    import multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_timing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2, 11.0), (1, 2, 11.0)]


def test_cpu_baseline_reports_one_and_all_cores_and_the_host():
    d = bench.cpu_baseline(n_side=32, steps_1=2, steps_all=2, config1_steps=5)
    assert d["kind"] == "oracle" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["single_core"]["cores"] == 1 and d["single_core"]["value"] > 0
    assert d["host"]["nproc"] >= 1 and d["host"]["cpu_model"]
    assert d["cores"] >= 1
    c1 = d["config1_64x64_1e4_steps"]
    assert c1["single_core"]["steps"] == 5
    if "all_cores" in c1:
        assert c1["all_cores"]["cores"] == d["cores"]
