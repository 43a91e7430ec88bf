"""Multi-rank logic of bench.py on CPU: two gloo ranks read their rank from
the launcher's environment, meet at the barrier, agree on the slowest
rank's time, and compute the whole-job rate from it; only rank 0 of the
reference arm does work."""
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
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_init(world, backend="gloo")
    bench.barrier(w)
    ms = 10.0 * (r + 1)                       # rank 1 is the slower replica
    ms_max = bench.allmax(ms, w)
    rate = bench.whole_job_rate(1000, 5, ms_max, w)
    buf = io.StringIO()

    class Args:
        n, steps, warmup, gpus = 64, 1, 0, world
    with redirect_stdout(buf):
        ref = bench.run_reference(Args) if r != 0 else None
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as fh:
        json.dump({"rank": r, "world": w, "local": local, "ms_max": ms_max, "rate": rate,
                   "ref": ref, "printed": buf.getvalue()}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, g in enumerate(got):
        assert (g["rank"], g["world"], g["local"]) == (r, 2, r)
        assert g["ms_max"] == 20.0
        assert g["rate"] == pytest.approx(2 * 1000 * 5 / 0.020)
    assert got[1]["ref"] is None and got[1]["printed"] == ""


def test_single_rank_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1) == (0, 1, 0)
    assert bench.allmax(3.5, 1) == 3.5
    assert bench.whole_job_rate(100, 10, 2.0, 1) == pytest.approx(100 * 10 / 0.002)
