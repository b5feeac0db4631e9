"""Host logic of bench.py at world size 2, on CPU with gloo: the replicas solve
different instances, the reported time is the slowest rank's, and only rank 0
runs the reference arm.  (The iteration itself does not shard: several GPUs run
independent replicas, so no data-path collective exists to test.)"""
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    bench.init_ranks(world)
    got = bench.max_over_ranks(1.5 + rank, world)   # per-rank times 1.5 and 2.5
    bench.barrier(world)
    bench.finish_ranks(world)
    q.put((rank, got))


def test_time_is_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        results = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert results == [(0, 2.5), (1, 2.5)]
    assert all(p.exitcode == 0 for p in procs)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    bench.init_ranks(1)
    assert bench.max_over_ranks(3.25, 1) == 3.25
    bench.barrier(1)
    bench.finish_ranks(1)


def test_replicas_solve_distinct_instances():
    sys.path.insert(0, ROOT)
    from paper_2207_11669_gb300 import synth
    wl = synth.workload_small()
    a = wl.instance(seed=wl.seed + 0)
    b = wl.instance(seed=wl.seed + 1)
    assert a.M.shape == b.M.shape
    assert not np.array_equal(a.M, b.M)


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small",
                        "--steps", "1", "--warmup", "1"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host) prints one JSON
    line with the keys the benchmark contract asks for."""
    import json
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT,
                       env=dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0"),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_strip_groups_follow_the_wave_cost_rule():
    """The algorithmic bytes of the two-pass passes count one P partial per
    (slab, strip group); bench.py's strip-group count is the library's rule:
    the smallest G whose wave cost ceil(nslabs G / SMs) / G is within 6 % of
    the best, never more groups than strips."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.tc2_strip_groups(64, 4096, 152) == 7      # large workload: 3 waves
    assert bench.tc2_strip_groups(16, 1024, 152) == 9      # one wave of 144 CTAs
    for nslabs, nstrips, sms in [(64, 4096, 152), (16, 1024, 152), (2, 1024, 152),
                                 (17, 1024, 152), (64, 3, 152), (1, 1, 152), (40, 64, 132)]:
        g = bench.tc2_strip_groups(nslabs, nstrips, sms)
        assert 1 <= g <= max(1, nstrips)

        def cost(x):
            return -(-nslabs * x // sms) / x
        gmax = max(1, min(nstrips, max(32, sms // nslabs)))
        best = min(cost(x) for x in range(1, gmax + 1))
        assert cost(g) <= 1.06 * best
        assert all(cost(x) > 1.06 * best for x in range(1, g))


def test_kernel_bytes_and_scaled_traffic():
    """The roofline's algorithmic bytes per launch (M once, V read and written,
    the per-row factors; the two-pass kernels also move their column sums and
    P partials) and the ncu traffic scaled from the captured n to the run's n."""
    sys.path.insert(0, ROOT)
    import bench
    m, n, r = 4096, 65536, 32
    kb = bench.kernel_bytes(m, n, r, 2, 152)
    assert kb["fused_step"] == 4.0 * m * n + 8.0 * n * r + 8.0 * m * r
    m, n, r = 16384, 262144, 64
    kb = bench.kernel_bytes(m, n, r, 3, 152)
    G = bench.tc2_strip_groups(m // 256, n // 64, 152)
    assert kb["pass_a"] == 4.0 * m * n + 4.0 * n * r + 4.0 * (m // 512) * n * r + 8.0 * m * r
    assert kb["pass_b"] == 4.0 * m * n + 8.0 * n * r + 4.0 * G * m * r + 4.0 * m * r
    t = bench.ncu_traffic("pass_a", m, n, r)
    assert t == bench.NCU_TRAFFIC["pass_a"]["bytes"] * n / bench.NCU_TRAFFIC["pass_a"]["n"]
    assert bench.ncu_traffic("pass_a", m, n, 32) is None      # another rank: no capture
    # traffic within a few percent of the algorithmic bytes: M is read once per pass
    assert 0.98 < t / kb["pass_a"] < 1.05
