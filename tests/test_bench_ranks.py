"""Multi-rank host logic of bench.py on CPU: two gloo ranks (one process each, as
torchrun launches them on a GPU node) agree on the slowest rank's time, and the
whole-job value counts every rank's samples; the reference arm does its work on
rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import torch
    ranks = bench.Ranks(dist, torch.device("cpu"))
    ranks.barrier()
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    ms = ranks.allmax(local_ms)
    q.put((rank, ms, bench.job_value(1000, world, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_samples():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in out:
        assert ms == 15.0
        assert value == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(None, None)
    r.barrier()
    assert r.allmax(3.5) == 3.5
    assert bench.job_value(393216 * 50, 1, 1000.0) == pytest.approx(393216 * 50)


def test_reference_arm_prints_only_on_rank_zero():
    """Under torchrun the reference arm's other ranks exit 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "tiny_fp32"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "tiny_fp32"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["cores"] >= 1


def test_adam_roofline_counts_the_parameters_the_optimizer_visits():
    # bench.py's Adam bytes count the reachable parameters only: every entry of a
    # hashed level, the first (N_l + 1)^3 entries of a dense level (whole groups of
    # four floats) and the LN / MLP block, computed here from the oracle's level
    # resolutions
    sys.path.insert(0, ROOT)
    import bench
    import synthetic as S
    from oracle.encoding import is_dense, level_resolutions
    for name in ("tiny_fp32", "paper_fp32", "large_bf16"):
        f = S.WORKLOADS[name].field
        T, F = 2 ** f.log2_T, f.n_feat
        n = S.param_layout(f)["_total"][1] - f.n_levels * T * F
        for res in level_resolutions(f.n_levels, f.base_res, f.max_res):
            live = (res + 1) ** 3 if is_dense(res, T) else T
            n += min(T * F, -(-live * F // 4) * 4)
        assert bench.optimizer_params(f) == n
        assert n < S.param_layout(f)["_total"][1]
