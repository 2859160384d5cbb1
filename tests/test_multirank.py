"""Multi-rank logic of bench.py on the CPU: two gloo ranks.

The path shards over independent images, so the only cross-rank steps are
the barrier around the timed region, the max of the step time over ranks and
rank-0-only output; each rank draws its own seeded problems.  These run as
two spawned processes with the gloo backend (no GPU)."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import contextlib
    import io

    import bench
    from paper_1511_03296_gb300 import synth

    d = bench.Dist()
    res = {"rank": d.rank, "world": d.world, "backend": d.pg.get_backend()}
    d.barrier()
    # max over ranks of a per-rank step time
    res["max"] = d.max(10.0 + 5.0 * rank)
    # per-rank problems differ (independent images, weak scaling)
    inst = synth.plain_64x48(seed=bench.rank_seed(1, rank)).instances[0]
    res["t_sum"] = float(inst.t.sum())
    # the reference arm runs on rank 0 only: other ranks return at once, silent
    if rank != 0:
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            r = bench.run_reference(None, d)
        res["ref_other"] = (r, buf.getvalue())
    d.barrier()
    d.close()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    assert [x["rank"] for x in r] == [0, 1]
    assert all(x["world"] == 2 and x["backend"] == "gloo" for x in r)
    assert r[0]["max"] == r[1]["max"] == 15.0
    assert r[0]["t_sum"] != r[1]["t_sum"]
    assert r[1]["ref_other"] == [None, ""]


def test_whole_job_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 2,073,600 pixels in 1 ms (the slowest rank) = 4147.2 Mpix/s
    assert bench.whole_job_mpix(2, 2_073_600, 1.0) == pytest.approx(4147.2)
    assert bench.whole_job_mpix(1, 1_000_000, 2.0) == pytest.approx(500.0)
    assert bench.rank_seed(4, 0) != bench.rank_seed(4, 1)
