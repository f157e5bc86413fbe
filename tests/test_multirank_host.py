"""Multi-rank host logic of the benchmark, on CPU with the gloo backend at world size 2: each rank
advances its own replica (the path does not shard within a mesh), ranks meet at barriers, the
timed region's duration is the maximum over ranks, and the whole-job value counts every rank's
cells. The reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_env()
    d = bench.Dist(w, "gloo")
    d.barrier()
    # a rank-dependent "timed region": the job's time is the slowest rank's
    t_max = d.max(5.0 + 2.0 * r)
    d.barrier()
    d.close()
    q.put((r, w, local, t_max, bench.whole_job_value(w, 131072, 10, t_max)))


def test_two_gloo_ranks_take_the_max_time_and_count_all_cells():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    for _, _, _, t_max, value in out:
        assert t_max == 7.0   # max over ranks (5 + 2 * rank)
        assert value == pytest.approx(2 * 131072 * 3 * 10 / 7e-3 / 1e6)


def test_whole_job_value_is_weak_scaling_sum():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.whole_job_value(1, 1000, 4, 2.0)
    assert bench.whole_job_value(4, 1000, 4, 2.0) == pytest.approx(4 * one)
    assert one == pytest.approx(1000 * 3 * 4 / 2e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    # rank 1 of 2 returns at once (before reading its arguments), prints nothing and never
    # loads the oracle
    assert bench.run_reference(None, 1, 2) is None
    assert capsys.readouterr().out == ""
