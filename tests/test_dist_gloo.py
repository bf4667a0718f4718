"""Multi-rank host logic with world_size-2 gloo process groups on the CPU:
the max/sum over ranks used for timing and throughput, the cost-balanced
partition of independent instances, and the gather of per-rank results."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import workloads as W  # noqa: E402
from paper_1909_08354_b300 import dist as D  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, q):
    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                             world_size=world)
    try:
        out = {
            "world": D.world(), "rank": D.rank(),
            "max": D.max_over_ranks(1.5 + rank),
            "sum": D.sum_over_ranks(10.0 * (rank + 1)),
            "replica": D.replica_throughput(cells=1000, steps=4, seconds=1.0 + rank),
            "sharded": D.sharded_throughput(local_cell_steps=100.0 * (rank + 1), seconds=2.0 - rank),
        }
        parts = D.partition_by_cost([D.scan_cost(n) for n in sizes], world)
        g = torch.arange(4, dtype=torch.float32) * (rank + 1)
        D.average_gradients(g)
        out["grad"] = g.tolist()
        out["mine"] = parts[rank]
        out["gathered"] = D.gather_objects(parts[rank])
        D.barrier()
        q.put((rank, out))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    sizes = [w.n[0] for w in (W.scan_instance_2d(i, sizes=(128, 256, 512, 1024)) for i in range(96))]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        o = res[r]
        assert o["world"] == world and o["rank"] == r
        assert o["max"] == 2.5
        assert o["sum"] == 30.0
        assert o["grad"] == [0.0, 1.5, 3.0, 4.5]  # the mean of ranks' 1x and 2x
        assert o["replica"] == world * 1000 * 4 / 2.0          # slowest rank's time
        assert o["sharded"] == (100.0 + 200.0) / 2.0
        assert o["gathered"] == [res[0]["mine"], res[1]["mine"]]
    # every instance on exactly one rank, both ranks compute the same partition
    allidx = sorted(res[0]["mine"] + res[1]["mine"])
    assert allidx == list(range(len(sizes)))


def test_partition_by_cost_is_balanced_and_complete():
    sizes = [w.n[0] for w in (W.scan_instance_2d(i) for i in range(96))]
    costs = [D.scan_cost(n) for n in sizes]
    for nparts in (1, 2, 3, 4, 8):
        parts = D.partition_by_cost(costs, nparts)
        assert sorted(i for p in parts for i in p) == list(range(96))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy largest-first: the spread is at most the largest single cost
        assert max(loads) - min(loads) <= max(costs) + 1e-9
        assert D.partition_by_cost(costs, nparts) == parts   # deterministic
    with pytest.raises(ValueError):
        D.partition_by_cost(costs, 0)


def test_single_process_defaults():
    assert not tdist.is_initialized()
    assert D.world() == 1 and D.rank() == 0
    assert D.max_over_ranks(3.0) == 3.0
    assert D.replica_throughput(10, 2, 4.0) == 5.0
    assert D.gather_objects("x") == ["x"]


def test_average_gradients_without_a_process_group_is_a_no_op():
    g = torch.tensor([1.0, -2.0, 3.0])
    D.average_gradients(g)
    assert g.tolist() == [1.0, -2.0, 3.0]


class _StandInNet:
    """The interface surrogate.train drives (forward, loss, backward, get_grads,
    set_grads, adam, sync) on a quadratic loss |p - target|^2, so that the
    data-parallel loop runs on CPU ranks; adam is a plain gradient step here."""

    def __init__(self, n, target, slow=0.0):
        self.nparams, self.target, self.slow = n, float(target), slow
        self.p = torch.zeros(n)
        self.g = torch.zeros(n)

    def forward(self, x, out):
        import time
        time.sleep(self.slow)
        return out

    def loss(self, y, B):
        return float(((self.p - self.target) ** 2).sum())

    def backward(self):
        self.g = 2.0 * (self.p - self.target)

    def get_grads(self, out):
        out.copy_(self.g)
        return out

    def set_grads(self, g):
        self.g = g.clone()

    def adam(self, lr, t):
        self.p -= lr * self.g

    def sync(self):
        pass


def _dp_worker(rank, world, port, q):
    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                             world_size=world)
    try:
        from paper_1909_08354_b300 import surrogate as S
        X, Y = torch.zeros(4, 5, 2, 2), torch.zeros(4, 2, 2, 2)
        # ranks pull towards different targets; the averaged gradient is that of 2.0
        net = _StandInNet(3, target=1.0 + 2.0 * rank)
        S.train(net, X, Y, iters=60, batch=2, lr=0.2, data_parallel=True, device="cpu")
        # a slow rank runs out of its time budget first: both must stop together
        slow = _StandInNet(3, target=0.0, slow=0.03 if rank == 1 else 0.0)
        losses = S.train(slow, X, Y, iters=1000, batch=2, lr=0.1, time_budget=0.3,
                         data_parallel=True, device="cpu")
        q.put((rank, {"p": net.p.tolist(), "iters": len(losses)}))
    finally:
        tdist.destroy_process_group()


def test_data_parallel_training_loop_on_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_dp_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0]["p"] == res[1]["p"]  # the replicas stay identical
    assert all(abs(v - 2.0) < 0.05 for v in res[0]["p"])
    assert res[0]["iters"] == res[1]["iters"] < 1000


def _short_shard_worker(rank, world, port, q):
    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                             world_size=world)
    try:
        from paper_1909_08354_b300 import surrogate as S
        # rank 1's shard holds one pair, less than a batch of 2: every rank must
        # raise before the first gradient all-reduce instead of waiting in it
        n = 4 if rank == 0 else 1
        X, Y = torch.zeros(n, 5, 2, 2), torch.zeros(n, 2, 2, 2)
        try:
            S.train(_StandInNet(3, target=1.0), X, Y, iters=10, batch=2, lr=0.1,
                    data_parallel=True, device="cpu")
            q.put((rank, "trained"))
        except ValueError as e:
            q.put((rank, "ValueError" if "fewer pairs than one batch" in str(e) else str(e)))
    finally:
        tdist.destroy_process_group()


def test_a_shard_smaller_than_a_batch_stops_every_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_short_shard_worker, args=(r, world, port, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: "ValueError", 1: "ValueError"}
