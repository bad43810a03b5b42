"""One plasma sharded by particles (paper_1108_1954_gb300.shard), with all
shards on one GPU and stepped in lockstep, against the run that holds every
particle: the summed fixed-point density and the field bit for bit, and the
shards' particles together the whole run's particles bit for bit (as a set:
each shard sorts its own particles).  On several GPUs the same protocol sums
the densities with one int64 all-reduce per step."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402,F401
from paper_1108_1954_gb300 import shard

pytestmark = pytest.mark.gpu
L4PI = 4.0 * math.pi


def _as_set(u, v):
    i = np.lexsort((v, u))
    return u[i], v[i]


@pytest.mark.parametrize("n,ng,world,S", [(200003, 512, 2, 5), (100001, 64, 3, 0),
                                          (65536, 4096, 4, 3)])
def test_shards_equal_the_whole_run(n, ng, world, S):
    modes = W.two_stream_modes_1_to_8(1e-3, 9)
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 9, modes=modes)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    whole = pic.Run(pic.Params(npart=n, ncell=ng, length=L4PI, sort_interval=S, history=64),
                    device="cuda:0")
    whole.init(x32, v32)
    parts, shards = [], []
    for r in range(world):
        lo, hi = shard.split(n, world, r)
        parts.append((x32[lo:hi], v32[lo:hi]))
        shards.append(shard.Shard(pic.Params(npart=hi - lo, ncell=ng, length=L4PI,
                                             sort_interval=S, history=64), n, None,
                                  device="cuda:0"))
    group = shard.ShardGroup(shards)
    group.init(parts)
    fw = whole.get_field()
    for s in shards:
        f = s.run.get_field()
        assert np.array_equal(f["rho_q"], fw["rho_q"])
        assert np.array_equal(f["E"], fw["E"]) and np.array_equal(f["phi"], fw["phi"])
    steps = 17
    whole.step_n(steps)
    group.step_n(steps)
    fw = whole.get_field()
    uw, vw = _as_set(*whole.get_cells())
    us = np.concatenate([s.run.get_cells()[0] for s in shards])
    vs = np.concatenate([s.run.get_cells()[1] for s in shards])
    us, vs = _as_set(us, vs)
    assert np.array_equal(us, uw) and np.array_equal(vs, vw)
    dw = whole.diagnostics(0, steps + 1)
    kin = np.zeros(steps)
    for s in shards:
        f = s.run.get_field()
        assert np.array_equal(f["rho_q"], fw["rho_q"])
        assert np.array_equal(f["E"], fw["E"])
        d = s.run.diagnostics(0, steps + 1)
        assert np.array_equal(d["field"], dw["field"])
        assert (d["charge_q"] == n << O.FIX_BITS).all()
        kin += d["kinetic"][:-1]
    # each shard's kinetic energy is its share (mass of the whole plasma's
    # particles); the shares add up to the whole run's to float32 rounding
    assert np.allclose(kin, dw["kinetic"][:-1], rtol=1e-5)
    group.close()
    whole.close()


def test_shard_rejects_bad_totals():
    run = pic.Run(pic.Params(npart=1000, ncell=64, length=L4PI), device="cuda:0")
    with pytest.raises(pic.PicError):
        run.set_shard(999)                      # fewer than it holds
    with pytest.raises(pic.PicError):
        run.set_shard((1 << 39) + 1)            # the int64 sums would overflow
    run.set_shard(1000)
    f64 = pic.Run(pic.Params(npart=1000, ncell=64, length=L4PI, precision=pic.PIC_FP64),
                  device="cuda:0")
    with pytest.raises(pic.PicError):
        f64.set_shard(2000)                     # float densities do not sum exactly
