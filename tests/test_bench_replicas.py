"""The N > 1 path of bench.py on CPU: two gloo ranks run the replica logic
(distinct seeds, a barrier, the job time as the slowest rank's, the
whole-job rate), and the reference arm leaves ranks other than 0 idle."""
import os
import socket
import sys
import types

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.barrier(ws)
        t_max = bench.max_over_ranks(1.0 + rank, ws, "cpu")      # rank r "took" 1 + r seconds
        out.put((rank, bench.replica_seed(1610067690, rank), t_max, bench.whole_job_rate(100.0, ws, t_max)))
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas_timed_by_the_slowest():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = [r[1] for r in res]
    assert len(set(seeds)) == ws and seeds[0] == 1610067690        # rank 0 keeps the workload's seed
    assert all(r[2] == 2.0 for r in res)                            # every rank sees the slowest time
    assert all(r[3] == pytest.approx(100.0 * ws / 2.0) for r in res)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_seed(7, 0) == 7
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_leaves_other_ranks_idle(capsys):
    args = types.SimpleNamespace(voltage=200.0, steps=1, warmup=3)
    assert bench.run_reference(args, 2, 1) is None
    assert capsys.readouterr().out == ""
