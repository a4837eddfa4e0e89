"""The multi-replica path of bench.py on CPU (two gloo ranks, no GPU):
max-over-ranks timing, whole-job throughput, the per-replica device records
gathered for the JSON line, and the reference arm that only rank 0 runs and
prints."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)  # the slowest rank's time
    bench.barrier(world)
    value = bench.replica_tflops(2.0e12, 4, ms, world)
    reps = bench.gather_replicas(world, {"rank": rank, "uuid": "GPU-fake-%d" % rank})
    sys.argv = ["bench.py", "--impl", "reference", "--size", "128", "--steps", "1",
                "--warmup", "0"]
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(bench.parse())
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"ms": ms, "value": value, "replicas": reps, "stdout": buf.getvalue()}, f)
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["ms"] == r1["ms"] == 15.0  # both ranks see the maximum
    assert r0["value"] == pytest.approx(2 * 2.0e12 * 4 / 0.015 / 1e12)
    assert r1["stdout"] == ""  # only rank 0 runs the reference arm and prints
    # every rank holds every replica's record, in rank order
    want = [{"rank": 0, "uuid": "GPU-fake-0"}, {"rank": 1, "uuid": "GPU-fake-1"}]
    assert r0["replicas"] == r1["replicas"] == want
    line = json.loads(r0["stdout"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
