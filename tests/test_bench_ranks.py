"""The multi-rank logic of bench.py on CPU ranks (gloo, world size 2):
the reported time is the slowest rank's, the throughput counts every
rank's units (weak scaling), and the estimate path has no collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench._dist()
        slow = bench.max_over_ranks(10.0 + 5.0 * rank)
        rate = bench.job_rate(12000, w, slow)
        q.put((r, w, loc, slow, rate))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 15.0 for o in out)
    assert all(abs(o[4] - 2 * 12000 / 15.0) < 1e-9 for o in out)


def test_single_process_has_no_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(100, 1, 2.0) == 50.0


def test_launch_decision_spawns_or_refuses():
    """--gpus N without a launcher starts N ranks itself; inside a launch of
    another size it refuses (exit status 2) instead of running one rank."""
    import subprocess
    import sys

    import bench
    assert bench.launch_decision(1, {}) == ("run", None)
    assert bench.launch_decision(4, {}) == ("spawn", None)
    assert bench.launch_decision(4, {"WORLD_SIZE": "4"}) == ("run", None)
    what, why = bench.launch_decision(8, {"WORLD_SIZE": "1"})
    assert what == "error" and "WORLD_SIZE=1" in why
    cmd = bench.rank_command(4, ["--gpus", "4", "--steps", "2"], 29555)
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "--master-addr=127.0.0.1" in cmd and "--master-port=29555" in cmd
    assert cmd[-4:] == ["--gpus", "4", "--steps", "2"] and cmd[-5].endswith("bench.py")
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, bench.__file__, "--gpus", "2"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 2 and "WORLD_SIZE=1" in r.stdout


def test_step2_traffic_digest_covers_the_kernel_and_its_tiling():
    """The DRAM figure of the bench line is reported only while the Step-II
    source it was captured on is unchanged: every region of that source (the
    kernel, the tile limits, the grid set and the tiling) must be found, and
    a capture whose digest differs is refused."""
    import json
    import bench
    for prec in bench.STEP2_SOURCE:
        d = bench._kernel_digest(prec)
        assert len(d) == 16 and int(d, 16) >= 0
    with open(os.path.join(bench.ROOT, "profiles", "step2_dram_mixed_tc.json")) as fh:
        rec = json.load(fh)
    assert {int(c["n_g"]) for c in rec["captures"]} >= {512}
    if rec["kernel_digest"] == bench._kernel_digest("mixed_tc"):
        assert bench._traffic(512, "mixed_tc")[0] == float(rec["captures"][0]["bytes_per_estimate"])
    else:
        assert bench._traffic(512, "mixed_tc")[0] is None
    assert bench._traffic(100, "mixed_tc")[0] is None
