"""The multi-GPU bench path is replicas only: every rank runs its own copy of the workload and the
whole-job figures are the slowest rank's time and the sum of every rank's pair interactions. The
host logic runs here as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (rank, world, rank)
    bench.rank_barrier(world)
    ms, pairs = bench.job_totals(10.0 + rank, 1000 * (rank + 1), world)
    out[rank] = (ms, pairs)
    bench.rank_barrier(world)
    dist.destroy_process_group()


def _skin_rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def choose():
        if rank != 0:
            raise AssertionError("only rank 0 runs the skin autotuner")
        return {"skin": 0.6, "table": [{"skin": 0.6, "steps_per_s": 1.0}]}

    out[rank] = bench.bench_skin("auto", rank, world, choose)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_rank_zeros_skin():
    """With an autotuned skin, rank 0 chooses and every rank runs its replicas with that skin."""
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_skin_rank_main, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    assert got[0][0] == got[1][0] == 0.6
    assert got[0][1] == got[1][1] and got[1][1]["table"][0]["skin"] == 0.6


def test_given_skin_and_no_usable_candidate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.bench_skin("0.45", 0, 1, None) == (0.45, None)
    skin, rec = bench.bench_skin("auto", 0, 1, lambda: {"skin": None, "table": []})
    assert skin == 0.3 and rec == {"skin": None, "table": []}


def test_two_gloo_ranks_take_the_slowest_time_and_the_sum_of_pairs():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    assert got[0] == got[1] == (11.0, 3000.0)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(3.5, 123, 1) == (3.5, 123.0)


def test_reference_arm_prints_one_contract_line_on_the_host():
    """`bench.py --impl reference` times the FP64 oracle on the host cores (no GPU needed) and prints
    one JSON line with the contract's keys: the metric, a positive value, the workload, and the
    cpu_baseline and e2e objects describing the same run."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "cylinder_pore_1k", "--steps", "3", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 1
    assert d["config"]["workload"] == "cylinder_pore_1k"
    for k in ("metric", "unit", "n_gpus", "ms_per_step", "higher_is_better", "scaling", "dtype",
              "data", "vs_baseline"):
        assert k in d
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
