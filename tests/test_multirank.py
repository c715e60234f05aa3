"""The multi-rank path on CPU: two gloo ranks split a batch of circuits by
cost, simulate their share with the oracle, gather the results and take the
maximum time -- the same host logic the benchmark runs with one GPU per rank."""
import os
import socket

import numpy as np
import pytest

from paper_2203_08826_gb300 import inputs, shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        circs = inputs.batch_circuits(12, seed=3, nmin=3, nmax=6, lmin=1, lmax=3)
        costs = [(1 << c.n) * len(c.gates) for c in circs]
        mine = shard.shard_by_cost(costs, rank, world)
        local = [oracle.expectation(oracle.simulate(circs[i]), inputs.zz_chain(circs[i].n)) for i in mine]
        allres = shard.gather_results(local, mine, len(circs))
        tmax = shard.max_over_ranks(float(rank + 1))
        q.put((rank, mine, allres.tolist(), tmax))
    finally:
        dist.destroy_process_group()


def test_split_helpers():
    for n, w in ((10, 3), (2, 4), (4096, 8)):
        ranges = [shard.shard_range(n, r, w) for r in range(w)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        assert max(b - a for a, b in ranges) - min(b - a for a, b in ranges) <= 1
    costs = np.random.default_rng(1).integers(1, 100, 50).tolist()
    parts = [shard.shard_by_cost(costs, r, 4) for r in range(4)]
    assert sorted(sum(parts, [])) == list(range(50))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    with pytest.raises(ValueError):
        shard.shard_range(5, 3, 2)


def test_two_gloo_ranks_split_and_gather():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    import oracle
    circs = inputs.batch_circuits(12, seed=3, nmin=3, nmax=6, lmin=1, lmax=3)
    want = [oracle.expectation(oracle.simulate(c), inputs.zz_chain(c.n)) for c in circs]
    mine0, mine1 = res[0][1], res[1][1]
    assert sorted(mine0 + mine1) == list(range(12)) and not set(mine0) & set(mine1)
    for r in res:
        np.testing.assert_allclose(r[2], want, atol=1e-12)
        assert r[3] == 2.0


def _slice_worker(rank, world, port, q, n, g):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2203_08826_gb300 import binding, sliced
        from slice_cpu import OracleSliceEngine, global_heavy_circuit
        circ = global_heavy_circuit(n, seed=n + g)
        plan = binding.SlicePlan(circ, g, kmax=2, mode=binding.FUSE_GREEDY2)
        a = inputs.gaussian_state(n, seed=4).reshape(1 << g, -1)
        own = sliced.owned_slices(g, rank, world)
        slices = {i: torch.from_numpy(a[i].copy()) for i in own}
        sliced.run_distributed(plan, slices, OracleSliceEngine(plan, oracle))
        q.put((rank, {i: slices[i].numpy() for i in own}))
    finally:
        dist.destroy_process_group()


def _pipeline_worker(rank, world, port, q, n, g):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2203_08826_gb300 import binding, sliced
        from slice_cpu import OracleSliceEngine, global_heavy_circuit

        class Recording(OracleSliceEngine):  # the order of the engine's packs and unpacks
            def __init__(self, plan, orc):
                super().__init__(plan, orc)
                self.log = []

            def pack(self, buf, l, bit):
                self.log.append(("pack", id(buf)))
                return super().pack(buf, l, bit)

            def unpack(self, buf, l, bit, src):
                self.log.append(("unpack", id(buf)))
                return super().unpack(buf, l, bit, src)

        circ = global_heavy_circuit(n, seed=n + g)
        plan = binding.SlicePlan(circ, g, kmax=2, mode=binding.FUSE_GREEDY2)
        a = inputs.gaussian_state(n, seed=4).reshape(1 << g, -1)
        own = sliced.owned_slices(g, rank, world)
        slices = {i: torch.from_numpy(a[i].copy()) for i in own}
        eng = Recording(plan, oracle)
        sliced.run_distributed(plan, slices, eng)
        ids = {id(slices[i]): i for i in own}
        q.put((rank, [(kind, ids[b]) for kind, b in eng.log],
               np.concatenate([slices[i].numpy() for i in own])))
    finally:
        dist.destroy_process_group()


def test_rank_exchange_is_pipelined():
    """Two gloo ranks with four slices each: in every exchange on the
    rank-selecting bit, slice i + 1 is packed (and its transfer posted)
    before slice i is unpacked, every slice is unpacked exactly once, in
    order, and the result still matches the oracle."""
    import torch.multiprocessing as mp
    from paper_2203_08826_gb300 import build
    build.build()
    world, n, g = 2, 11, 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_pipeline_worker, args=(r, world, port, q, n, g)) for r in range(world)]
    for p in procs:
        p.start()
    res = {r: (log, amps) for r, log, amps in (q.get(timeout=240) for _ in procs)}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        log = res[r][0]
        assert log, "no rank-selecting exchange ran"
        # split the log into exchanges: each is 4 packs and 4 unpacks
        for e in range(0, len(log), 8):
            ex = log[e:e + 8]
            packs = [i for kind, i in ex if kind == "pack"]
            unpacks = [i for kind, i in ex if kind == "unpack"]
            assert packs == unpacks == sorted(packs) and len(packs) == 4
            order = [(kind, i) for kind, i in ex]
            for k in range(3):
                assert order.index(("pack", packs[k + 1])) < order.index(("unpack", packs[k]))
    import oracle
    from slice_cpu import global_heavy_circuit
    circ = global_heavy_circuit(n, seed=n + g)
    want = oracle.simulate(circ, inputs.gaussian_state(n, seed=4))
    got = np.concatenate([res[0][1], res[1][1]])
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("world,n,g", [(2, 11, 3), (4, 10, 2)])
def test_sliced_state_over_gloo_ranks(world, n, g):
    """Slices spread over ranks; exchanges on rank-selecting global bits go
    through point-to-point send/recv, the others stay inside a rank."""
    import torch.multiprocessing as mp
    from paper_2203_08826_gb300 import build
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slice_worker, args=(r, world, port, q, n, g)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slices = {}
    for r in range(world):
        slices.update(res[r])
    got = np.concatenate([slices[i] for i in range(1 << g)])
    import oracle
    from slice_cpu import global_heavy_circuit
    from paper_2203_08826_gb300 import binding
    circ = global_heavy_circuit(n, seed=n + g)
    plan = binding.SlicePlan(circ, g, kmax=2, mode=binding.FUSE_GREEDY2)
    assert any(s["type"] == "swap" and s["global_bit"] >= g - (world.bit_length() - 1) for s in plan.steps())
    want = oracle.simulate(circ, inputs.gaussian_state(n, seed=4))
    assert np.max(np.abs(got - want)) < 1e-12
