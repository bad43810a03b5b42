"""One plasma sharded by particles over several ranks (GPUs).

The paper splits its line over the UPC threads and reduces the density and
the solver's dot products globally every cycle (Sec. 3.1-3.3).  Here every
rank keeps the whole grid and 1/W of the particles in its own run
(pic_set_shard), and a step is, on every rank:

    [the rank's own sort, when due] -> pic_push -> all-reduce (sum) of the NG
    int64 density sums -> pic_solve_field

The density is an exact integer sum, so the reduction gives every rank the
whole plasma's density bit for bit, every rank solves the same field, and
each particle moves exactly as in the run that holds all of them.  The
all-reduce is the only data-path collective: NG int64 values (<= 64 KB) per
step.

`Shard` is one rank's part, driven with any `reduce(tensor)` that sums an
int64 tensor in place over the ranks (`torch_allreduce` for
torch.distributed; NCCL on GPUs).  `ShardGroup` drives several shards of one
process in lockstep, summing their densities on the device (for one GPU
holding all the shards, as in the tests).
"""
from __future__ import annotations

from . import Run, Params


def torch_allreduce(group=None):
    """reduce(t): in-place sum of t over the ranks of a torch.distributed
    group (int64 sums are exact)."""
    import torch.distributed as dist

    def reduce(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return reduce


def split(npart: int, world: int, rank: int):
    """The contiguous particle range [lo, hi) of `rank` among `world`."""
    return npart * rank // world, npart * (rank + 1) // world


class Shard:
    """One rank's shard of a plasma of `npart_total` particles: a run of
    `params.npart` particles normalised by the whole plasma."""

    def __init__(self, params: Params, npart_total: int, reduce, device=None, stream=None,
                 run=None):
        # `run`: an object with Run's methods to drive instead of a new Run
        self.run = run if run is not None else Run(params, device=device, stream=stream)
        self.run.set_shard(npart_total)
        self.reduce = reduce
        self.rho_q = self.run.density()
        self.S = params.sort_interval

    def close(self):
        self.run.close()

    # the three phases of a step; ShardGroup interleaves them over its shards
    def pre(self):
        r = self.run
        if self.S > 0 and r.step > 0 and r.step % self.S == 0:
            r.sort()
        r.push()

    def post(self):
        self.run.solve_field()

    def init(self, x, v):
        """Load this rank's particles; E^0 from the whole plasma's density."""
        self.run.init(x, v)
        self.run.deposit()
        self.reduce(self.rho_q)
        self.run.solve_field()

    def step_n(self, n: int):
        for _ in range(int(n)):
            self.pre()
            self.reduce(self.rho_q)
            self.post()


class ShardGroup:
    """Several shards of one plasma in one process, stepped in lockstep; the
    all-reduce sums their density accumulators on the device."""

    def __init__(self, shards):
        self.shards = list(shards)

    def _reduce_all(self):
        total = self.shards[0].rho_q.clone()
        for s in self.shards[1:]:
            total += s.rho_q
        for s in self.shards:
            s.rho_q.copy_(total)

    def init(self, parts):
        for s, (x, v) in zip(self.shards, parts):
            s.run.init(x, v)
            s.run.deposit()
        self._reduce_all()
        for s in self.shards:
            s.run.solve_field()

    def step_n(self, n: int):
        for _ in range(int(n)):
            for s in self.shards:
                s.pre()
            self._reduce_all()
            for s in self.shards:
                s.post()

    def close(self):
        for s in self.shards:
            s.close()
