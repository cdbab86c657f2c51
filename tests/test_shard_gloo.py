"""Host logic of the multi-GPU batched form on CPU: two gloo ranks partition
a batch identically and without communication, cover every problem once with
balanced cost, and reassemble the results in problem order.  The per-rank
registration is a stand-in object (no GPU in these ranks)."""
import os
import socket

import numpy as np
import pytest

from paper_2507_01439_gb300 import shard


def test_partition_covers_balances_and_is_deterministic():
    rng = np.random.default_rng(0)
    ns = rng.integers(500, 5001, size=256)
    costs = [shard.problem_cost(int(n), 1000) for n in ns]
    for world in (1, 2, 3, 8):
        parts = shard.partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(256))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs) + 1e-9      # LPT bound
        assert shard.partition(costs, world) == parts
        assert all(p == sorted(p) for p in parts)
    assert shard.partition([], 2) == [[], []]
    assert shard.partition([5.0], 3) == [[0], [], []]


def test_cost_grows_with_size_and_k():
    assert shard.problem_cost(5000, 1000) > shard.problem_cost(1000, 1000)
    assert shard.problem_cost(2000, 2000) > shard.problem_cost(2000, 100)


class _FakeResult:
    def __init__(self, n, k1):
        self.n, self.k1 = n, k1


class _FakeCtx:
    """Stands in for a TurboReg context: one 'result' per problem = (n, k1, first x)."""
    def register_batched(self, xs, ys, offs, params):
        assert xs.shape == ys.shape and offs[-1] == xs.shape[0]
        return [(int(offs[b + 1] - offs[b]), int(params[b].k1), float(xs[offs[b], 0]))
                for b in range(len(offs) - 1)]


class _P:
    def __init__(self, k1, k2=2):
        self.k1, self.k2 = k1, k2


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(1)
        ns = rng.integers(3, 400, size=37)
        ks = rng.integers(10, 2000, size=37)
        offs = np.cumsum([0] + list(ns)).astype(np.int64)
        xs = np.zeros((offs[-1], 3), np.float32)
        for b in range(37):
            xs[offs[b]:offs[b + 1], 0] = b            # first coordinate tags the problem
        ys = xs.copy()
        params = [_P(int(k)) for k in ks]
        res = shard.register_sharded(_FakeCtx(), xs, ys, offs, params, rank, world)
        want = [(int(ns[b]), int(ks[b]), float(b)) for b in range(37)]
        ok = res == want
        # the partition is the same on every rank without communication
        costs = [shard.problem_cost(int(n), int(k)) for n, k in zip(ns, ks)]
        parts = [None] * world
        dist.all_gather_object(parts, shard.partition(costs, world))
        ok = ok and all(p == parts[0] for p in parts)
        # max-over-ranks timing as the benchmark takes it
        import torch
        t = torch.tensor([float(rank + 1)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ok = ok and float(t[0]) == float(world)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write("ok" if ok else "bad")
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_shard_and_gather(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        assert (tmp_path / f"rank{r}.txt").read_text() == "ok"
