"""The multi-process path of bench.py (replicas only: one process per GPU,
no collective on the data path) run as two gloo ranks on the CPU: the
launcher environment, the per-rank seeds, the max-over-ranks time and the
whole-job throughput."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    b = _bench()
    r, w, local, d = b._setup_dist(world, backend="gloo")
    try:
        ms = 10.0 + 5.0 * r                # the slower rank sets the time
        t_max = b.max_over_ranks(d, ms, torch.device("cpu"))
        d.barrier()
        out[r] = (r, w, local, b.replica_seed(7, r), t_max, b.replica_value(w, 1000, 4, t_max))
    finally:
        d.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    with mp.Manager() as manager:
        out = manager.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r, (rr, w, local, seed, t_max, value) in res.items():
        assert rr == r and w == world and local == r
        assert seed == 7 + r
        assert t_max == 15.0
        assert value == pytest.approx(world * 1000 * 4 / 15e-3)


def test_single_process_needs_no_collective():
    b = _bench()
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    r, w, local, d = b._setup_dist(1)
    assert (r, w, local, d) == (0, 1, 0, None)
    assert b.max_over_ranks(None, 3.5, None) == 3.5
