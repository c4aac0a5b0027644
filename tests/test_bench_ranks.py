"""The N > 1 path of bench.py on CPU: two ranks over gloo (one process each, 127.0.0.1).

One mesh does not shard in this path, so N GPUs run N independent replicas; the only
collective steps are the barrier around the timed region and the maximum of the per-rank
times, from which the whole-job value (units of all ranks over the slowest rank's time) is
formed.  The reference arm runs on rank 0 alone; the other ranks exit 0 without work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    try:
        r, w, local = bench.dist_env()
        dist = bench.Dist(w, local, backend="gloo")
        dist.barrier()
        ms = 10.0 + 5.0 * r                       # rank r's time for its own replica
        slowest = dist.max(ms)
        units = 1000                              # unknowns x evaluations per rank
        value = bench.whole_job_value(w, units, slowest)
        # the reference arm: rank != 0 returns at once, without touching the oracle
        ref_rc = bench.run_reference(bench.parse(["--impl", "reference", "--gpus", str(w)])) if r != 0 else 0
        dist.barrier()
        dist.close()
        q.put((r, w, slowest, value, ref_rc))
    except Exception as e:   # report to the parent instead of hanging it
        q.put((rank, "error", repr(e)))


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_max_time_and_sum_the_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=100) for _ in procs]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    out.sort()
    assert all(o[1] != "error" for o in out), out
    for r, w, slowest, value, ref_rc in out:
        assert w == 2
        assert slowest == 15.0                     # the max over both ranks, on every rank
        assert value == pytest.approx(2 * 1000 / 15e-3)
        assert ref_rc == 0


def test_a_failing_side_leg_is_recorded_on_one_rank_and_raised_on_several():
    import bench

    def leg(x):
        if x < 0:
            raise ValueError("negative")
        return {"x": x}

    assert bench.side_leg(1, leg, 2) == {"x": 2}
    assert bench.side_leg(1, leg, -1) == {"error": "ValueError: negative"}
    with pytest.raises(ValueError):
        bench.side_leg(2, leg, -1)
