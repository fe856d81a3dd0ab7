"""The multi-rank work split (paper_2103_03517_gb300.shard) on CPU with two
gloo ranks, driving the serial oracle: a batch of independent lattices split
by cost gives every lattice's own chain, and one lattice split into two slabs
of z planes, with the boundary planes exchanged after each colour pass and
the accepted counts summed, gives the unsplit chain of Table A1 bit for bit
(the draws are keyed by global site indices), both with the exchange written
out here and through shard.slab_sweep_ranks, the driver of the library's GPU
slabs, given oracle slabs."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

import oracle
import workloads
from paper_2103_03517_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_by_cost_covers_every_item_once_and_balances():
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        costs = [float(L) ** 3 for L in rng.choice([16, 32, 64, 128], size=32)]
        shares = shard.partition_by_cost(costs, world)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in shares]
        assert max(loads) <= sum(costs) / world + max(costs)
    # the batched temperature sweep over 8 ranks: one 128^3 lattice each
    specs = workloads.batched_mt_32()
    shares = shard.partition_by_cost([s.N for s in specs], 8)
    assert all(sum(1 for i in s if specs[i].dims[0] == 128) == 1 for s in shares)


def test_slab_planes_are_even_and_cover_the_lattice():
    for Lz, world in ((8, 2), (12, 2), (16, 3), (128, 8), (10, 4)):
        sl = shard.slab_planes(Lz, world)
        assert sl[0][0] == 0 and sl[-1][1] == Lz
        assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
        assert all((z1 - z0) % 2 == 0 and z1 > z0 for z0, z1 in sl)
    with pytest.raises(ValueError):
        shard.slab_planes(7, 2)


SPECS = [((8, 6, 4), 0.6, 1), ((4, 4, 4), 1.3, 2), ((6, 6, 6), 0.9, 3), ((8, 8, 2), 1.1, 4), ((4, 6, 8), 0.2, 5)]


def _lattice_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [d[0] * d[1] * d[2] for d, _, _ in SPECS]
        mine = shard.partition_by_cost(costs, world)[rank]
        res = {}
        for i in mine:
            dims, T, seed = SPECS[i]
            o = oracle.Lattice(dims, Ku=0.05, T=T, seed=seed)
            o.sweep(7, measure=True)
            res[i] = (o.spins().tolist(), o.theta)
        gathered = [None] * world
        dist.all_gather_object(gathered, res)
        if rank == 0:
            merged = {}
            for g in gathered:
                merged.update(g)
            out["lattices"] = merged
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_independent_lattices_without_changing_any_chain():
    port = _free_port()
    with tmp.Manager() as man:
        out = man.dict()
        tmp.spawn(_lattice_rank, args=(2, port, out), nprocs=2, join=True)
        merged = dict(out)["lattices"]
    assert sorted(merged) == list(range(len(SPECS)))
    for i, (dims, T, seed) in enumerate(SPECS):
        o = oracle.Lattice(dims, Ku=0.05, T=T, seed=seed)
        o.sweep(7, measure=True)
        assert np.array_equal(np.array(merged[i][0]), o.spins()) and merged[i][1] == o.theta


SLAB_DIMS = (8, 6, 8)


def _slab_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Lx, Ly, Lz = SLAB_DIMS
        z0, z1 = shard.slab_planes(Lz, world)[rank]
        # every rank holds a lattice of the full size but owns only planes
        # z0 .. z1 - 1; planes z0 - 1 and z1 (mod Lz) are its halo
        o = oracle.Lattice(SLAB_DIMS, Ku=0.05, Kc=0.02, H=(0.0, 0.02, 0.01), T=0.8, seed=9)
        o.set_spins(workloads.random_spins(Lx * Ly * Lz, 6))
        for _ in range(6):
            acc = 0
            for colour in (0, 1):
                acc += o.colour_pass_planes(colour, z0, z1)
                S = torch.from_numpy(o.spins().reshape(Lz, Ly * Lx * 3).copy())
                below, above = shard.exchange_halo(S[z0], S[z1 - 1], rank, world)
                S[(z0 - 1) % Lz] = below
                S[z1 % Lz] = above
                o.set_spins(S.numpy().reshape(-1, 3))
            o.end_sweep(shard.sum_over_ranks(acc, world))
        S = o.spins().reshape(Lz, Ly * Lx, 3)
        gathered = [None] * world
        dist.all_gather_object(gathered, (z0, z1, S[z0:z1].tolist(), o.theta))
        if rank == 0:
            out["slabs"] = gathered
    finally:
        dist.destroy_process_group()


def test_two_slabs_with_halo_exchange_equal_the_unsplit_chain():
    port = _free_port()
    with tmp.Manager() as man:
        out = man.dict()
        tmp.spawn(_slab_rank, args=(2, port, out), nprocs=2, join=True)
        slabs = dict(out)["slabs"]
    Lx, Ly, Lz = SLAB_DIMS
    ref = oracle.Lattice(SLAB_DIMS, Ku=0.05, Kc=0.02, H=(0.0, 0.02, 0.01), T=0.8, seed=9)
    ref.set_spins(workloads.random_spins(Lx * Ly * Lz, 6))
    ref.sweep(6)
    R = ref.spins().reshape(Lz, Ly * Lx, 3)
    for z0, z1, S, theta in slabs:
        assert np.array_equal(np.array(S), R[z0:z1])
        assert theta == ref.theta


class _OracleSlab:
    """The slab calls of shard.slab_sweep_ranks on the serial oracle: the
    rank's lattice holds every plane but moves only its own (z0 .. z1 - 1);
    the planes are views of a host copy of the spins, so the driver's halo
    writes reach the oracle before the next pass (whole planes: the other
    colour of a boundary plane is unchanged since its own exchange)."""

    def __init__(self, o, z0, z1, dims):
        self.o, self.z0, self.z1 = o, z0, z1
        Lx, Ly, Lz = dims
        self.Lz = Lz
        self.S = torch.from_numpy(o.spins().reshape(Lz, Ly * Lx, 3).copy())
        self.acc = 0

    def pass_(self, h, colour, measure):
        self.o.set_spins(self.S.numpy().reshape(-1, 3))
        self.acc += self.o.colour_pass_planes(colour, self.z0, self.z1)
        self.S.copy_(torch.from_numpy(self.o.spins().reshape(self.S.shape)))

    def planes(self, h, colour):
        zs = [self.z0, self.z1 - 1, (self.z0 - 1) % self.Lz, self.z1 % self.Lz]
        return [[self.S[z, :, a] for a in range(3)] for z in zs]

    def words(self, h):
        # the driver sums these words over the ranks in place before close
        self.w = torch.zeros(16, dtype=torch.int64)
        self.w[0] = self.acc
        self.acc = 0
        return self.w

    def close(self, h, measure):
        self.o.set_spins(self.S.numpy().reshape(-1, 3))
        self.o.end_sweep(int(self.w[0]))


def _driver_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Lx, Ly, Lz = SLAB_DIMS
        z0, z1 = shard.slab_planes(Lz, world)[rank]
        o = oracle.Lattice(SLAB_DIMS, Ku=0.05, Kc=0.02, H=(0.0, 0.02, 0.01), T=0.8, seed=9)
        o.set_spins(workloads.random_spins(Lx * Ly * Lz, 6))
        api = _OracleSlab(o, z0, z1, SLAB_DIMS)
        shard.slab_sweep_ranks(None, 6, rank=rank, world=world, api=api)
        S = o.spins().reshape(Lz, Ly * Lx, 3)
        gathered = [None] * world
        dist.all_gather_object(gathered, (z0, z1, S[z0:z1].tolist(), o.theta))
        if rank == 0:
            out["slabs"] = gathered
    finally:
        dist.destroy_process_group()


def test_slab_rank_driver_on_two_ranks_equals_the_unsplit_chain():
    """shard.slab_sweep_ranks (the driver of the library's GPU slabs) run on
    two gloo ranks with slabs of the serial oracle: its routing of boundary
    planes into halo planes and its all-reduce of the count words give the
    unsplit chain bit for bit."""
    port = _free_port()
    with tmp.Manager() as man:
        out = man.dict()
        tmp.spawn(_driver_rank, args=(2, port, out), nprocs=2, join=True)
        slabs = dict(out)["slabs"]
    Lx, Ly, Lz = SLAB_DIMS
    ref = oracle.Lattice(SLAB_DIMS, Ku=0.05, Kc=0.02, H=(0.0, 0.02, 0.01), T=0.8, seed=9)
    ref.set_spins(workloads.random_spins(Lx * Ly * Lz, 6))
    ref.sweep(6)
    R = ref.spins().reshape(Lz, Ly * Lx, 3)
    for z0, z1, S, theta in slabs:
        assert np.array_equal(np.array(S), R[z0:z1])
        assert theta == ref.theta
