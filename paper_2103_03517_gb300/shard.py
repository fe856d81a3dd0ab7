"""Work split over ranks (one process per GPU) for the two ways the path
shards (the paper's multi-GPU projection, Sec. 2: without dipole-dipole
coupling the ranks exchange little).

* Independent lattices (a temperature sweep, a theta sweep of constrained
  runs, served jobs): each rank takes a disjoint share, balanced by cost
  (spins x sweeps), and runs it alone; nothing is exchanged on the data path.
* One large lattice (a wall, a film): slabs of planes along the slowest axis
  z.  After each colour pass of Table A1 a rank sends its first and last
  planes to the ranks below and above it (periodic in z) and receives their
  boundary planes into its own halo planes; the accepted counts of the
  iteration are summed over the ranks, so the cone angle stays one value.
  The draws are keyed by global site indices, so the split chain equals the
  unsplit one bit for bit.

The partitions and the exchanges use torch.distributed (gloo on the CPU,
NCCL between GPUs).  slab_sweep_ranks drives one rank's GPU slab of the
library (mc_slab_create): the library's kernels move the spins, this module
only moves boundary planes and count words between ranks.
"""
from __future__ import annotations

__all__ = ["partition_by_cost", "slab_planes", "exchange_halo", "sum_over_ranks", "device_array",
           "LibrarySlab", "slab_sweep_ranks"]


def partition_by_cost(costs, world: int) -> list:
    """Indices of items 0 .. len(costs) - 1 for each of `world` ranks:
    largest first onto the least loaded rank (ties: the lower rank), each
    share in increasing index order.  Every item goes to exactly one rank;
    the largest load is at most the mean load plus the largest item."""
    if world < 1:
        raise ValueError("world must be >= 1")
    shares = [[] for _ in range(world)]
    load = [0.0] * world
    for i in sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i)):
        r = min(range(world), key=lambda k: (load[k], k))
        shares[r].append(i)
        load[r] += float(costs[i])
    return [sorted(s) for s in shares]


def slab_planes(Lz: int, world: int) -> list:
    """(z0, z1) plane ranges of `world` slabs of a lattice Lz planes deep, as
    equal as possible with every slab an even number of planes, so that each
    slab starts on an even plane and the colour (x + y + z) mod 2 of a site is
    the same counted locally from the slab's halo plane below it."""
    if Lz % 2 or Lz < 2 * world:
        raise ValueError("slabs need an even Lz of at least two planes per rank")
    pairs = Lz // 2
    out, z = [], 0
    for r in range(world):
        n = 2 * (pairs // world + (1 if r < pairs % world else 0))
        out.append((z, z + n))
        z += n
    return out


def exchange_halo(first_plane, last_plane, rank: int, world: int):
    """Send this slab's first plane to the rank below and its last plane to
    the rank above (periodic); return (halo_below, halo_above): the last plane
    of the rank below and the first plane of the rank above.  Tensors of one
    shape and dtype on every rank (CPU tensors with gloo, device tensors with
    NCCL).  With one rank the slab is its own neighbour."""
    import torch
    import torch.distributed as dist

    if world == 1:
        return last_plane.clone(), first_plane.clone()
    below, above = (rank - 1) % world, (rank + 1) % world
    halo_below, halo_above = torch.empty_like(last_plane), torch.empty_like(first_plane)
    # with two ranks both messages go to the same peer and are matched in
    # posting order: every rank sends (up: last plane, down: first plane) and
    # receives (from below: its last plane, from above: its first plane)
    ops = [dist.P2POp(dist.isend, last_plane.contiguous(), above),
           dist.P2POp(dist.isend, first_plane.contiguous(), below),
           dist.P2POp(dist.irecv, halo_below, below),
           dist.P2POp(dist.irecv, halo_above, above)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return halo_below, halo_above


def sum_over_ranks(value: int, world: int) -> int:
    """An integer count summed over the ranks (exact: int64)."""
    if world == 1:
        return int(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([int(value)], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


class _DeviceBuffer:
    """A device address as a CUDA array (no copy, not owned)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def device_array(ptr: int, n: int, dtype):
    """A torch tensor viewing n elements at device address ptr (float32 or
    int64); the memory stays the library's."""
    import torch

    typestr = {torch.float32: "<f4", torch.int64: "<i8"}[dtype]
    return torch.as_tensor(_DeviceBuffer(ptr, n, typestr), device="cuda")


class LibrarySlab:
    """The calls slab_sweep_ranks makes on a slab of the library
    (mc_slab_create): its colour pass, its boundary and halo planes as
    tensors viewing device memory, its exported count words, its close."""

    def pass_(self, h, colour: int, measure: bool) -> None:
        from . import _mc as mc

        mc.mc_slab_pass(h, colour, measure)

    def planes(self, h, colour: int):
        """[first own, last own, lower halo, upper halo], each three
        component tensors of one plane of the colour."""
        import torch

        from . import _mc as mc

        out = []
        for which in range(4):
            ptrs, n = mc.mc_slab_plane(h, colour, which)
            out.append([device_array(p, n, torch.float32) for p in ptrs])
        return out

    def words(self, h):
        import torch

        from . import _mc as mc

        return device_array(mc.mc_slab_export(h), mc.MC_SLAB_WORDS, torch.int64)

    def close(self, h, measure: bool) -> None:
        from . import _mc as mc

        mc.mc_slab_close(h, measure)


def slab_sweep_ranks(h, n_sweeps: int, measure: bool = False, rank: int = 0, world: int = 1, api=None) -> None:
    """n_sweeps sweeps of Table A1 of this rank's slab h (mc_slab_create, the
    rank's planes of slab_planes), the slabs of the other ranks advancing in
    step: per colour the slab's pass, then this colour's boundary planes to
    the neighbouring ranks and their planes into h's halo planes
    (exchange_halo); per sweep the slab's count words summed over the ranks
    (all-reduce) and the slab's close.  api makes the slab calls (default
    LibrarySlab); with the library, h must run on torch's current stream
    (desc.stream), so that its kernels and the exchanges are ordered.  With
    world = 1 the slab is its own neighbour."""
    import torch
    import torch.distributed as dist

    api = api or LibrarySlab()
    for _ in range(int(n_sweeps)):
        for colour in (0, 1):
            api.pass_(h, colour, measure and colour == 1)
            planes = api.planes(h, colour)
            below, above = exchange_halo(torch.cat(planes[0]), torch.cat(planes[1]), rank, world)
            n = planes[0][0].numel()
            for a in range(3):
                planes[2][a].copy_(below[a * n:(a + 1) * n])
                planes[3][a].copy_(above[a * n:(a + 1) * n])
        words = api.words(h)
        if world > 1:
            dist.all_reduce(words, op=dist.ReduceOp.SUM)
        api.close(h, measure)
