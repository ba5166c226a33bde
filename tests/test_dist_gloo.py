"""The multi-process path of bench.py on CPU: two gloo ranks, each with its
own seed; throughput uses the slowest rank's time (max over ranks)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2304_01772_gb300 import dist as sdist


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = sdist.rank_info()
    elapsed = 1.0 + rank                               # rank 1 is the slowest
    slowest = sdist.max_over_ranks(elapsed, dist)
    seeds = [None] * world
    dist.all_gather_object(seeds, sdist.rank_seed(123, r))
    out[rank] = (r, w, local, slowest, sdist.job_throughput(100.0, w, slowest), seeds)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_distinct_seeds():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        rank, world, local, slowest, rate, seeds = res[r]
        assert (rank, world, local) == (r, 2, r)
        assert slowest == 2.0
        assert rate == pytest.approx(100.0)              # 2 ranks x 100 units / 2 s
        assert seeds == [123, 124]


def test_single_process_defaults():
    assert sdist.max_over_ranks(3.5, None) == 3.5
    assert sdist.job_throughput(10.0, 1, 2.0) == 5.0


def to_limbs(v):
    """The limb layout of spin_pooled_limbs for one int128 value (test-local)."""
    u = v & ((1 << 128) - 1)
    l3 = v >> 96                                  # arithmetic shift: signed top limb
    return [u & 0xFFFFFFFF, (u >> 32) & 0xFFFFFFFF, (u >> 64) & 0xFFFFFFFF, l3]


def from_limbs(l):
    return l[0] + (l[1] << 32) + (l[2] << 64) + (l[3] << 96)


VALUES = [[7, -5, 2 ** 64 + 3, -(2 ** 100) + 17], [2 ** 63 - 1, -(2 ** 63), 2 ** 70, 2 ** 100 - 1]]


def _limb_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    limbs = torch.tensor([to_limbs(v) for v in VALUES[rank]], dtype=torch.int64)
    sdist.allreduce_limbs(limbs, dist)
    out[rank] = [from_limbs([int(x) for x in row]) for row in limbs.tolist()]
    dist.barrier()
    dist.destroy_process_group()


def test_moment_limbs_sum_exactly_over_two_gloo_ranks():
    """The gradient's exchange step: int128 moments split into 32-bit limbs
    (int64 words) are summed element-wise by the all-reduce; recombining the
    sum gives the exact total, carries and negative values included."""
    for v in sum(VALUES, []):
        assert from_limbs(to_limbs(v)) == v
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_limb_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        want = [a + b for a, b in zip(*VALUES)]
        assert out[0] == want and out[1] == want


def _partition_worker(rank, world, port, out):
    import numpy as np

    import oracle
    from paper_2304_01772_gb300 import workloads as wl
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lats = wl.uneven512(n=24, seed=5, emin=2, emax=5)      # sides 4 .. 32: the oracle runs them at once
    mine, idx = sdist.rank_lattices(lats, rank, world)
    # this rank's chains: the lattice word of lattice_id - 1, as the library draws it
    res = {}
    for d, gi in zip(mine, idx):
        assert d["lattice_id"] == gi + 1
        s = oracle.init_ising(d["L"], 77, d["lattice_id"] - 1).copy()
        st = oracle.ising_run(s, d["beta"], d["J"], d["h"], 77, d["lattice_id"] - 1, 0, 3)
        res[gi] = (s.tobytes(), st.tobytes())
    parts = [None] * world
    dist.all_gather_object(parts, sdist.partition_by_sites([d["L"] for d in lats], world))
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    out[rank] = (parts, gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_batch_on_two_gloo_ranks_is_the_whole_batch():
    """Each rank computes the same site-count split independently; the shares
    cover every lattice once, their loads differ from the mean by less than
    the largest lattice, and the ranks' chains (lattice word = global index)
    are the whole batch's chains."""
    import oracle
    from paper_2304_01772_gb300 import workloads as wl
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_partition_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    lats = wl.uneven512(n=24, seed=5, emin=2, emax=5)
    splits, gathered = res[0]                          # the split each rank computed
    assert splits[0] == splits[1] == res[1][0][0]
    parts = splits[0]
    assert sorted(parts[0] + parts[1]) == list(range(len(lats)))
    loads = [sum(lats[i]["L"] ** 2 for i in p) for p in parts]
    assert max(loads) - sum(loads) / 2 <= max(d["L"] ** 2 for d in lats)
    whole = {}
    for i, d in enumerate(lats):                      # one process, batch index as lattice word
        s = oracle.init_ising(d["L"], 77, i).copy()
        st = oracle.ising_run(s, d["beta"], d["J"], d["h"], 77, i, 0, 3)
        whole[i] = (s.tobytes(), st.tobytes())
    merged = {**gathered[0], **gathered[1]}
    assert merged == whole


def test_partition_by_sites_balance_and_determinism():
    from paper_2304_01772_gb300 import workloads as wl
    lats = wl.uneven512()
    sizes = [d["L"] for d in lats]
    total = sum(L * L for L in sizes)
    for world in (1, 2, 3, 4, 7, 8):
        parts = sdist.partition_by_sites(sizes, world)
        assert parts == sdist.partition_by_sites(list(sizes), world)
        assert sorted(sum(parts, [])) == list(range(len(sizes)))
        loads = [sum(sizes[i] ** 2 for i in p) for p in parts]
        assert max(loads) <= total / world + max(L * L for L in sizes)
    assert sdist.partition_by_sites([4, 6], 3)[2] == []
    with pytest.raises(ValueError):
        sdist.partition_by_sites([4], 0)
