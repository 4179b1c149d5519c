"""The multi-GPU path of bench.py (one realisation per rank, no collective on the
data path, barrier + max over ranks around the timed region) with the gloo
backend on CPU, world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    g = bench.Group("gloo")
    assert (g.ws, g.rank) == (ws, rank)
    g.barrier()
    t = g.max(1.5 + rank)                      # per-rank "timed region"
    seeds = g.max(float(bench.replica_seed(rank))) - bench.replica_seed(0)
    out[rank] = (t, seeds, bench.aggregate_rate(ws, 64 ** 3, 10, t))
    g.barrier()
    g.close()


def test_two_rank_max_and_aggregate():
    ws, port = 2, _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 2.5        # max over ranks
    assert out[0][1] == ws - 1                   # seeds differ per rank
    assert out[0][2] == pytest.approx(2 * 64 ** 3 * 10 / 2.5)


def test_single_process_group_is_a_no_op(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    g = bench.Group("gloo")
    assert g.ws == 1 and g.max(3.25) == 3.25
    g.barrier()
    g.close()


def test_kernel_hash_ignores_comments_only():
    import bench
    src = "// head\nint f(int a) { /* two\nlines */ return a + 1; // tail\n}\n\n"
    assert bench.code_only(src) == "int f(int a) {  return a + 1;\n}"
    assert bench.code_only(src) == bench.code_only(src.replace("// tail", "// other words"))
    assert bench.code_only(src) != bench.code_only(src.replace("a + 1", "a + 2"))


def test_failing_extra_leg_is_reported_not_raised():
    import bench

    def no_room(_):
        raise MemoryError("217 GB do not fit")
    assert bench.extra_leg(no_room, None) == {"unavailable": "MemoryError: 217 GB do not fit"}
    assert bench.extra_leg(lambda x: {"value": x}, 3) == {"value": 3}
