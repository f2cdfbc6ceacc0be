"""Host logic of the multi-GPU benchmark (one process per GPU, independent
streams dealt to the ranks, max-over-ranks timing) exercised with
world_size-2 gloo process groups on the CPU: the functions bench.run_ours and
bench.run_mixed call to split their streams and time the job."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench

MIXED_SIZES = [(w, h) for w, h, _, _ in bench.MIXED for _ in range(16)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        mine = bench.partition_streams(ws * bench.STREAMS, ws, r)     # the headline job: 16 videos per rank
        mixed = bench.partition_by_area(MIXED_SIZES, ws, r)           # the mixed batch spread by area
        t = 10.0 + 5.0 * r                         # per-rank elapsed ms
        bench.barrier()
        worst = bench.max_over_ranks(t)
        q.put((r, ws, local, mine, mixed, worst))
    finally:
        dist.destroy_process_group()


def test_two_rank_partition_and_max_over_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, l0, m0, x0, w0), (r1, ws1, l1, m1, x1, w1) = res
    assert ws0 == ws1 == 2 and (r0, r1) == (0, 1) and (l0, l1) == (0, 1)
    # every video on exactly one rank, 16 per rank, no exchange between ranks
    assert sorted(m0 + m1) == list(range(32)) and not set(m0) & set(m1)
    assert len(m0) == len(m1) == bench.STREAMS
    # the mixed streams: each once, and each rank gets 8 of every resolution
    assert sorted(x0 + x1) == list(range(64)) and not set(x0) & set(x1)
    for xs in (x0, x1):
        per_size = {}
        for i in xs:
            per_size[MIXED_SIZES[i]] = per_size.get(MIXED_SIZES[i], 0) + 1
        assert sorted(per_size.values()) == [8, 8, 8, 8]
    assert w0 == w1 == 15.0


def test_single_process_helpers():
    assert bench.partition_streams(5, 1, 0) == [0, 1, 2, 3, 4]
    assert bench.partition_by_area(MIXED_SIZES, 1, 0) == list(range(64))
    # three ranks: pixel areas within one largest stream of each other
    areas = []
    for r in range(3):
        xs = bench.partition_by_area(MIXED_SIZES, 3, r)
        areas.append(sum(MIXED_SIZES[i][0] * MIXED_SIZES[i][1] for i in xs))
    assert max(areas) - min(areas) <= 1920 * 1080
    assert bench.max_over_ranks(3.5) == 3.5


def test_detection_phases_of_the_two_schedules():
    """Staggered videos enter the detection cycle at g mod 5, so every step detects on a fifth
    of a rank's streams (16 videos: 3 or 4 per phase, each phase present); lockstep videos
    all sit at phase 0.  The bench line names the schedule it ran."""
    g = list(range(bench.STREAMS))
    stag = [bench.phase_of(v, True) for v in g]
    assert all(0 <= p < bench.PERIOD for p in stag)
    counts = [stag.count(p) for p in range(bench.PERIOD)]
    assert min(counts) >= bench.STREAMS // bench.PERIOD and max(counts) <= bench.STREAMS // bench.PERIOD + 1
    assert [bench.phase_of(v, False) for v in g] == [0] * bench.STREAMS
    assert "staggered" in bench.config_dict(bench.STREAMS, True)["detection"]
    assert "same steps" in bench.config_dict(bench.STREAMS, False)["detection"]
