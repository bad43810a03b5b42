#!/usr/bin/env python3
"""Benchmark of the 1D electrostatic PIC step on GB300.

Workload (default): the single large run -- 2^26 electrons, 4096 cells,
L = 4 pi, two beams at +-0.2 with thermal spread 0.01, modes 1..8 perturbed at
1e-4 with seeded random phases, dt = 0.1, counting sort every 20 steps; float32
push, int64 fixed-point deposit, float64 field solve.  A "step" is one whole
PIC step: [sort if due] + fused gather/push/deposit + field solve.

Prints one JSON line (rank 0).  `value` is particle-steps/s with the state
resident in HBM, timed around pic_step_n (CUDA graphs of whole sort periods);
`e2e` is the same metric through the public API from pinned
host buffers (upload the initial state, run the steps, read back the
diagnostics and the final state); `roofline` is the fused push kernel's
algorithmic bytes (16 B per particle: x, v read and written, float32) over its
CUDA-event duration against the measured copy bandwidth; `cpu_baseline` is the
FP64 oracle on this host.

`--impl reference` times the FP64 oracle (the reference arm) on the same
workload: each step is the oracle's step over a bounded sample, the same
recipe (cells, box, beams, modes, seed) at 2^20 electrons.
Under torchrun each rank runs its own independent run (weak scaling, no
collective on the data path: `value`); the line adds `sharded`, the same
2^26-particle run split over the ranks with one int64 all-reduce of the
density per step (strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_PARTICLE_STEP = 16          # x, v float32 read + write
C2 = dict(npart=1 << 26, ncell=4096, length=4.0 * math.pi, dt=0.1, v0=0.2,
          vth=0.01, eps=1e-4, sort_interval=20, seed=2026)
SMALL = dict(npart=1 << 20, ncell=4096, length=4.0 * math.pi, dt=0.1, v0=0.2,
             vth=0.01, eps=1e-4, sort_interval=20, seed=2026)
# the config-2 recipe at 2^25 particles: the profiling case (256 MiB of
# particles, above L2, a few GB on the device at most)
PROFILE = dict(npart=1 << 25, ncell=4096, length=4.0 * math.pi, dt=0.1, v0=0.2,
               vth=0.01, eps=1e-4, sort_interval=20, seed=2026)
REF_SAMPLE = 1 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "small", "profile"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--bps", type=int, default=0)
    ap.add_argument("--unroll", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-runs", type=int, default=512)
    ap.add_argument("--batched-steps", type=int, default=500)
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-c1", action="store_true")
    ap.add_argument("--no-weak", action="store_true")
    ap.add_argument("--weak-steps", type=int, default=1000)
    ap.add_argument("--only-weak", action="store_true",
                    help="run only the paper's weak-scaling workload")
    ap.add_argument("--only-c1", action="store_true",
                    help="run only the config-1 latency section")
    ap.add_argument("--only-batched", action="store_true",
                    help="run only the batched-ensemble section (profiling)")
    ap.add_argument("--no-tune-batched", action="store_true")
    ap.add_argument("--pool-variant", type=int, default=1 + 16,
                    help="the pool's deposit variant (+16: 64-register build) when not tuned")
    ap.add_argument("--pool-sort", type=int, default=0,
                    help="the pool's sort interval when not tuned")
    ap.add_argument("--pool-cluster", type=int, default=8)
    ap.add_argument("--pool-block", type=int, default=256)
    ap.add_argument("--only-precision", action="store_true",
                    help="run only the precision study (config 4)")
    ap.add_argument("--only-variant-scan", action="store_true",
                    help="mean push time of each deposit variant over two sort periods, "
                         "at several points of the config-2 run")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-advance", type=int, default=50)
    ap.add_argument("--no-precision", action="store_true",
                    help="leave out the precision study (config 4)")
    ap.add_argument("--precision-steps", type=int, default=2000)
    ap.add_argument("--precision-oracle-steps", type=int, default=150)
    return ap.parse_args()


def rank_aggregate(local_seconds, npart, steps, world_size, device="cpu"):
    """Whole-job throughput over ranks that each advanced their own run of
    `npart` particles by `steps`: the slowest rank's time (max over ranks)
    and world_size * npart * steps / that time.  No collective on the data
    path; this is the only cross-rank step."""
    total_s = float(local_seconds)
    if world_size > 1:
        import torch
        t = torch.tensor([total_s], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    return world_size * npart * steps / total_s, total_s


def workload(name):
    return dict({"c2": C2, "small": SMALL, "profile": PROFILE}[name])


def make_state(w):
    import workloads as W
    x, v = W.two_stream(w["npart"], w["length"], w["v0"], w["vth"], w["seed"],
                        modes=W.two_stream_modes_1_to_8(w["eps"], w["seed"]))
    return W.to_f32_state(x, v, w["length"])


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = max(smax, float(f[1]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def push_kernel_name(variant):
    """The fused push kernel a deposit variant runs in."""
    return "pic_push_oct_kernel" if variant in (8, 9) else "pic_push_fixed_kernel"


def recorded_traffic(variant=None, unroll=None):
    """DRAM bytes per launch of the fused push from the committed ncu summary:
    the entry captured for this deposit variant and unroll (the first entry
    when none is given), if the kernel source is unchanged since the
    capture."""
    path = os.path.join(ROOT, "profiles", "push_fixed_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    entries = rec.get("launches", [])
    if variant is not None:
        entries = [e for e in entries if e.get("variant") == variant and
                   (unroll is None or e.get("unroll") == unroll)]
    if not entries:
        return None
    m = hashlib.sha256()
    for f in rec.get("source_files", []):
        try:
            m.update(open(os.path.join(ROOT, f), "rb").read())
        except OSError:
            return None
    if rec.get("source_sha256") != m.hexdigest():
        return None
    return entries[0].get("bytes_per_launch_c2")


def time_ours(args, w, x32, v32):
    import numpy as np
    import torch
    import paper_1108_1954_gb300 as pic

    n, S = w["npart"], w["sort_interval"]
    params = pic.Params(npart=n, ncell=w["ncell"], length=w["length"], dt=w["dt"],
                        sort_interval=S, history=8192, deposit_variant=args.variant,
                        block_size=args.block, blocks_per_sm=args.bps, unroll=args.unroll)
    run = pic.Run(params, device="cuda")
    stream = run.stream
    # SM clocks and throttle reasons, sampled from here to the end of the
    # push timing below: the timed region itself may be shorter than one
    # sampling period (20 steps take ~4 ms)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    run.init(x32, v32)
    launches = {"n": 0}

    def one_step(ev=None):
        if S > 0 and run.step > 0 and run.step % S == 0:
            run.sort()
            launches["n"] += 5
        if ev is not None:
            ev[0].record(stream)
        run.push()
        if ev is not None:
            ev[1].record(stream)
        run.solve_field()
        launches["n"] += 2

    for _ in range(args.warmup):
        one_step()
    sort_tune = None
    if not args.no_tune and not args.variant:
        # Tune on the order the run keeps: after a few sorts the particles of
        # a cell sit in the order of the cells they came from, so in order of
        # velocity, and neighbours stay together longer after each sort than
        # in the lattice order of the first period.  Untimed set-up steps
        # past the second sort, then the tuner, then a re-warm.
        while S > 0 and run.step <= 2 * S:
            one_step()
        run.autotune(reps=8)
        for _ in range(3):
            one_step()
        if S > 0:
            # the sort-interval tuner's model for this state, reported beside
            # the workload's own interval (which the run keeps)
            best, table = run.tune_sort_interval((0, 5, 10, 20, 40, 80), adopt=False)
            sort_tune = {"best": best, "ms_per_step": {str(k): round(t, 4) for k, t in table.items()},
                         "kept": S}
    torch.cuda.synchronize()
    K = args.steps
    # the step loop through the public API: pic_step_n replays CUDA graphs of
    # whole sort periods, one per buffer parity, each captured the first time
    # a sort point is reached with a whole period to go; three periods from
    # here pass two such sort points, so both graphs exist before the timed
    # region
    run.step_n(3 * S if S > 0 else 32)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ws, rank, _ = dist_env()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    s0 = run.step
    t0.record(stream)
    run.step_n(K)
    t1.record(stream)
    torch.cuda.synchronize()
    total_ms = t0.elapsed_time(t1)
    if ws > 1:
        torch.distributed.barrier()
    # kernels the timed region launched: push + solve per step, 5 per sort
    timed_launches = 2 * K + 5 * sum(1 for m in range(s0, s0 + K) if S > 0 and m > 0 and m % S == 0)
    # the push's own duration: the next K steps once more, one call per
    # kernel, CUDA events around each push on the run's stream
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    torch.cuda.synchronize()
    for i in range(K):
        one_step(evs[i])
    torch.cuda.synchronize()
    ck = clocks.stop()
    if ck is not None:
        ck["window"] = ("samples every 50 ms from the upload of the state to the end of the "
                        "push timing (warm-up, tuning, the timed steps and the push timing)")
    push_ms = [a.elapsed_time(b) for a, b in evs]
    # the floor of the push's memory traffic: the same bytes (x and v of N
    # particles, float32, read and written in place) streamed by torch's
    # elementwise kernel
    xa = torch.empty(n, dtype=torch.float32, device=run.device).uniform_()
    va = torch.empty(n, dtype=torch.float32, device=run.device).uniform_()
    fl = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(20)]
    cs = torch.cuda.current_stream()
    for i in range(23):
        if i >= 3:
            fl[i - 3][0].record(cs)
        xa.mul_(1.0)
        va.mul_(1.0)
        if i >= 3:
            fl[i - 3][1].record(cs)
    torch.cuda.synchronize()
    floor_ms = statistics.mean(a.elapsed_time(b) for a, b in fl)
    del xa, va
    run.sync()
    grid, block, variant, unroll = run.launch_shape()
    diag = run.diagnostics(run.step - 1, 1)[0]
    res = dict(total_ms=total_ms, push_ms=push_ms, floor_ms=floor_ms, clocks=ck,
               launches=timed_launches,
               grid=grid, block=block, variant=variant, unroll=unroll,
               blocks_per_sm=grid // max(1, torch.cuda.get_device_properties(0).multi_processor_count),
               steps=K, sort_tune=sort_tune,
               energy=float(diag["kinetic"] + diag["field"]))
    run.close()
    return res


def time_e2e(args, w, x32, v32):
    """The public API end to end: pinned host state -> pic_init -> pic_step_n
    -> diagnostics + final state back to pinned host memory."""
    import torch
    import paper_1108_1954_gb300 as pic
    n, K = w["npart"], args.steps
    xh = torch.from_numpy(x32).pin_memory()
    vh = torch.from_numpy(v32).pin_memory()
    xo = torch.empty_like(xh).pin_memory()
    vo = torch.empty_like(vh).pin_memory()
    params = pic.Params(npart=n, ncell=w["ncell"], length=w["length"], dt=w["dt"],
                        sort_interval=w["sort_interval"], history=max(8192, K + 1),
                        deposit_variant=args.variant, block_size=args.block,
                        blocks_per_sm=args.bps, unroll=args.unroll)
    run = pic.Run(params, device="cuda")
    run.init(xh, vh)                      # warm: autotune, graph capture, first touch
    run.step_n(2 * w["sort_interval"] + 1)  # tuned past the second sort, as the device-timed run
    if not args.no_tune and not args.variant:
        run.autotune(reps=8)              # (drops the captured graphs)
    # three sort periods pass two sort points with a whole period to go:
    # both buffer parities' graphs are captured before the timed region
    run.step_n(3 * w["sort_interval"] if w["sort_interval"] > 0 else 32)
    # one untimed whole pass: the first touch of the output buffers, and the
    # path warm (passes right after set-up ran up to 28% slower)
    run.init(xh, vh)
    run.step_n(K)
    run.diagnostics(0, K)
    run.get_state(xo, vo)
    run.sync()
    torch.cuda.synchronize()
    # three whole passes (upload, K steps, diagnostics and state back), timed
    # on the host clock; the mean pass
    reps = 3
    marks = [time.perf_counter()]
    for _ in range(reps):
        run.init(xh, vh)
        run.step_n(K)
        d = run.diagnostics(0, K)
        run.get_state(xo, vo)
        marks.append(time.perf_counter())
    el = (marks[-1] - marks[0]) / reps
    _, block, variant, unroll = run.launch_shape()
    run.close()
    h2d = 2 * 4 * n
    d2h = 2 * 4 * n + d.nbytes
    return dict(value=n * K / el, seconds=el, h2d_per_step=h2d / K, d2h_per_step=d2h / K,
                passes=reps, pass_s=[round(b - a, 5) for a, b in zip(marks, marks[1:])],
                launch={"block": block, "deposit_variant": variant, "unroll": unroll})


def time_sharded(args, w, x32, v32):
    """Config 2 as one plasma sharded by particles over the ranks (strong
    scaling: the whole job is the same 2^26 particles at any N): each rank
    holds 1/N of them and the whole grid, and every step all-reduces the
    int64 density sums (NCCL) between its push and its solve.  Timed over K
    steps with CUDA events, between barriers; the slowest rank's time."""
    import torch
    import paper_1108_1954_gb300 as pic
    from paper_1108_1954_gb300 import shard
    ws, rank, _ = dist_env()
    n, S, K = w["npart"], w["sort_interval"], args.steps
    lo, hi = shard.split(n, ws, rank)
    sh = shard.Shard(pic.Params(npart=hi - lo, ncell=w["ncell"], length=w["length"], dt=w["dt"],
                                sort_interval=S, history=max(64, K + 1)),
                     n, shard.torch_allreduce(), device="cuda")
    sh.init(x32[lo:hi], v32[lo:hi])
    sh.step_n(max(3, args.warmup))
    stream = sh.run.stream
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    sh.step_n(K)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.distributed.barrier()
    t = torch.tensor([e0.elapsed_time(e1) / 1e3], device="cuda", dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_s = float(t.item())                   # the slowest rank
    sh.close()
    return {"value": n * K / total_s, "unit": "particle-steps/s", "scaling": "strong",
            "npart_total": n, "npart_per_rank": hi - lo, "steps": K,
            "ms_per_step": 1e3 * total_s / K,
            "collective": "one all-reduce (sum) of %d int64 density sums per step" % w["ncell"]}


def ensemble_states(nrun, seed):
    """The batched ensemble: per run (params, x32, v32)."""
    import workloads as W
    import paper_1108_1954_gb300 as pic
    out = []
    for r in W.ensemble_runs(nrun, seed):
        x, v = W.two_stream(r["npart"], r["length"], r["v0"], r["vth"], r["seed"],
                            modes=((1, 1e-3, 0.0),))
        x32, v32 = W.to_f32_state(x, v, r["length"])
        out.append((pic.Params(npart=r["npart"], ncell=r["ncell"], length=r["length"],
                               dt=r["dt"]), x32, v32))
    return out


def tune_pool(states, steps, history):
    """Autotuner of the batched launch, over the deposit variant and build,
    the cluster size, the block size (the tile shape) and the sort interval.
    The whole ensemble is admitted once; each (variant, cluster, block) is
    timed over `steps` steps (after one untimed step) in each of three
    rounds, on the same resident runs, the shape changed with
    pic_pool_configure and the order shuffled per round; the leading six
    are timed again over steps 100-500 of a fresh ensemble.  Then,
    with the fastest shape, the ensemble is admitted again for each sort interval S
    and timed over 40 steps (after 10), long enough to include the sorts of
    every S tried.  Returns the fastest (variant, cluster, block, S) and the
    two tables."""
    import torch
    import paper_1108_1954_gb300 as pic
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)

    def admit_all(S):
        nbytes = sum(pic.pool_run_bytes(pic.Params(npart=p.npart, ncell=p.ncell, length=p.length,
                                                   sort_interval=S), history)
                     for p, _, _ in states) + (64 << 20)
        pool = pic.Pool(max_slots=len(states), ncell_max=2048, arena_bytes=nbytes,
                        history=history, variant=5, cluster=8, block=512)
        for p, x, v in states:
            q = pic.Params(npart=p.npart, ncell=p.ncell, length=p.length, dt=p.dt,
                           sort_interval=S)
            pool.admit(q, x, v, 1 << 40)
        pool.advance(0)
        pool.sync()
        return pool

    # The resident runs evolve while the shapes are timed (cold beams early,
    # mixed later), and the shapes differ most early on, so each shape is
    # timed in several short windows spread over the first few hundred
    # steps, the order shuffled every round.
    import numpy as np
    pool = admit_all(0)
    shapes = []
    for variant in (1, 5, 6, 1 + 16, 5 + 16, 6 + 16):
        for cluster in (4, 8):
            for block in (256, 512):
                try:
                    pool.configure(variant, cluster, block)
                except pic.PicError:
                    continue
                shapes.append((variant, cluster, block))
    total = {sh: 0.0 for sh in shapes}
    rng = np.random.default_rng(7)
    rounds = 3
    for _ in range(rounds):
        for i in rng.permutation(len(shapes)):
            sh = shapes[i]
            pool.configure(*sh)
            pool.advance(1)
            e0.record(pool.stream)
            pool.advance(steps)
            e1.record(pool.stream)
            pool.sync()
            total[sh] += e0.elapsed_time(e1)
    pool.close()
    table = sorted(((sh, t / rounds) for sh, t in total.items()), key=lambda t: t[1])
    # The short windows rank the shapes within a few percent; the leading
    # six are timed again in windows spread over steps 100-500 of a fresh
    # ensemble, where most of the run's time goes.
    top = [sh for sh, _ in table[:6]]
    pool = admit_all(0)
    pool.configure(*top[0])
    pool.advance(100)
    long_total = {sh: 0.0 for sh in top}
    for _ in range(4):
        for i in rng.permutation(len(top)):
            sh = top[i]
            pool.configure(*sh)
            pool.advance(1)
            e0.record(pool.stream)
            pool.advance(16)
            e1.record(pool.stream)
            pool.sync()
            long_total[sh] += e0.elapsed_time(e1)
    pool.close()
    shape = min(top, key=lambda sh: long_total[sh])
    sort_table = []
    for S in (0, 10, 20, 40):
        pool = admit_all(S)
        pool.configure(*shape)
        pool.advance(10)
        e0.record(pool.stream)
        pool.advance(40)
        e1.record(pool.stream)
        pool.sync()
        pool.close()
        sort_table.append((S, e0.elapsed_time(e1) / 40.0))
    sort_table.sort(key=lambda t: t[1])
    return shape + (sort_table[0][0],), table, sort_table


def time_batched(args):
    """Config 3: the ensemble in one persistent cluster launch vs the same
    runs one per launch (each through pic_step_n, CUDA graphs)."""
    import torch
    import paper_1108_1954_gb300 as pic
    K, H = args.batched_steps, 16
    states = ensemble_states(args.batched_runs, 3)
    total_particles = sum(p.npart for p, _, _ in states)
    if args.no_tune_batched:
        best, table, sort_table = (args.pool_variant, args.pool_cluster, args.pool_block,
                                   args.pool_sort), [], []
    else:
        best, table, sort_table = tune_pool(states, 4, H)
    S = best[3]
    sorted_states = [(pic.Params(npart=p.npart, ncell=p.ncell, length=p.length, dt=p.dt,
                                 sort_interval=S), x, v) for p, x, v in states]
    nbytes = sum(pic.pool_run_bytes(p, H) for p, _, _ in sorted_states) + (64 << 20)
    pool = pic.Pool(max_slots=len(states), ncell_max=2048, arena_bytes=nbytes, history=H,
                    variant=best[0], cluster=best[1], block=best[2])
    for p, x, v in sorted_states:
        pool.admit(p, x, v, K)
    pool.advance(0)
    pool.sync()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record(pool.stream)
    pool.advance(K)
    e1.record(pool.stream)
    pool.sync()
    t_batched = e0.elapsed_time(e1) / 1e3
    pool.close()
    del pool
    # one run per launch sequence: every run through its own pic_step_n,
    # with the same sort interval
    runs = []
    for p, x, v in sorted_states:
        r = pic.Run(pic.Params(npart=p.npart, ncell=p.ncell, length=p.length, dt=p.dt,
                               sort_interval=S, history=max(64, K + 1)))
        r.init(x, v)
        r.step_n(3 * S if S else 16)    # capture its graphs outside the timed region
        runs.append(r)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0.record(s)
    for r in runs:
        r.step_n(K)
    e1.record(s)
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    for r in runs:
        r.close()
    args.pool_variant = best[0]          # reused by the served section
    return {"runs": len(states), "steps": K, "particles": total_particles,
            "value": total_particles * K / t_batched, "unit": "particle-steps/s",
            "seconds": t_batched, "plain_value": total_particles * K / t_plain,
            "plain_seconds": t_plain, "speedup_vs_plain": t_plain / t_batched,
            "launch": {"variant": best[0], "cluster": best[1], "block": best[2],
                       "sort_interval": S},
            "tune": [[list(c), round(ms, 3)] for c, ms in table[:6]],
            "tune_sort_interval": [[S_, round(ms, 4)] for S_, ms in sort_table]}


def precision_study(args):
    """Config 4: 2^24 electrons, 1024 cells, beams +-0.2 with vth 0.02 seeded
    with the growing mode-1 eigenmode, run in the three precision modes; the
    FP64 oracle runs the same state for a bounded window."""
    import numpy as np
    import oracle as O
    import workloads as W
    import paper_1108_1954_gb300 as pic
    n, ng, L, K = 1 << 24, 1024, 4.0 * math.pi, args.precision_steps
    x, v = W.two_stream_eigenmode(n, L, 0.2, 0.02, 1e-3, 1, 4)
    x32, v32 = W.to_f32_state(x, v, L)
    dt = 0.1
    t = np.arange(K) * dt
    fit = (t >= 2.0) & (t <= 12.0)
    m = L / n
    out = {"npart": n, "ncell": ng, "steps": K, "gamma_theory": W.cold_two_stream_gamma(2 * math.pi / L, 0.2)}
    ref = O.State(O.params(ng, n, L, dt), x32.astype(np.float64), v32.astype(np.float64))
    t0 = time.perf_counter()
    nt = host_threads()
    ko_ = args.precision_oracle_steps
    h = np.zeros((ko_, 11))
    for k in range(ko_):
        # the history row of orc_run, with the threaded step (same state)
        h[k, 2] = O.field_energy(ref.p, ref.E)
        h[k, 3:] = O.mode_amplitudes(ref.p, ref.E, 8)
        h[k, 0], h[k, 1] = ref.step_threads(nt) if nt > 1 else ref.step()
    o_fe = h[:, 2]
    o_ke = 0.5 * ref.mass * h[:, 0]
    ko = args.precision_oracle_steps
    fo = fit[:ko]
    o_gamma = float(np.polyfit(t[:ko][fo], np.log(h[fo, 3]), 1)[0]) if fo.sum() > 4 else None
    out["oracle"] = {"steps": ko, "seconds": time.perf_counter() - t0, "gamma1": o_gamma,
                     "threads": nt}
    for name, mode, xs, vs in (("fp64", pic.PIC_FP64, x, v),
                               ("fp32_atomic", pic.PIC_FP32_ATOMIC, x32, v32),
                               ("fp32_fixed", pic.PIC_FP32_FIXED, x32, v32)):
        run = pic.Run(pic.Params(npart=n, ncell=ng, length=L, dt=dt, precision=mode,
                                 history=K + 1, sort_interval=20))
        run.init(xs, vs)
        t0 = time.perf_counter()
        run.step_n(K)
        run.sync()
        el = time.perf_counter() - t0
        d = run.diagnostics(0, K)
        run.close()
        tot = d["kinetic"] + d["field"]
        vabs = m * np.abs(np.asarray(vs, np.float64)).sum()
        g1 = float(np.polyfit(t[fit], np.log(d["mode"][fit, 0]), 1)[0])
        kk = min(ko, K)
        out[name] = {
            "seconds": el, "particle_steps_per_s": n * K / el,
            "energy_drift": float((tot.max() - tot.min()) / tot[0]),
            "momentum_error": float(np.abs(d["momentum"] - d["momentum"][0]).max() / vabs),
            "gamma1": g1,
            "gamma1_vs_oracle": (g1 - o_gamma) / o_gamma if o_gamma else None,
            "field_energy_vs_oracle": float(np.abs(d["field"][:kk] - o_fe[:kk]).max() / o_fe[:kk].max()),
            "kinetic_vs_oracle": float(np.abs(d["kinetic"][:kk] - o_ke[:kk]).max() / o_ke[:kk].max()),
        }
    return out


def variant_scan(args):
    """Mean fused-push time per (variant, block, unroll) over two whole sort
    periods, restarting from the same state, at steps 0, 200 and 600 of the
    config-2 run."""
    import numpy as np
    import torch
    import paper_1108_1954_gb300 as pic
    w = workload(args.workload)
    x32, v32 = make_state(w)
    S = w["sort_interval"]
    run = pic.Run(pic.Params(npart=w["npart"], ncell=w["ncell"], length=w["length"],
                             dt=w["dt"], sort_interval=S))
    run.init(x32, v32)
    stream = run.stream
    out = []
    for checkpoint in (0, 200, 600):
        while run.step < checkpoint:
            run.step_n(min(100, checkpoint - run.step))
        xs, vs = run.get_cells()
        st = run.step
        row = {"step": st}
        for var in (1, 2, 5, 6, 8, 9):
            for blk, un in ((512, 1), (512, 2), (256, 1), (256, 2)):
                run.set_cells(xs, vs, st)
                run.set_launch(var, blk, un)
                ev = [(torch.cuda.Event(True), torch.cuda.Event(True)) for _ in range(2 * S)]
                for a, b in ev:
                    if run.step > 0 and run.step % S == 0:
                        run.sort()
                    a.record(stream)
                    run.push()
                    b.record(stream)
                    run.solve_field()
                torch.cuda.synchronize()
                row["%d/%d/%d" % (var, blk, un)] = round(float(np.mean(
                    [a.elapsed_time(b) for a, b in ev])), 4)
        run.set_cells(xs, vs, st)
        out.append(row)
    run.close()
    return out


def time_c1(args):
    """Config 1 (20,000 electrons, 64 cells, 200 steps): launch-bound, so
    reported as microseconds per step -- through pic_step_n (CUDA graphs of
    16 steps) and as a one-run pool (all 200 steps in one cluster launch; the
    fastest of clusters of 1, 2, 4 and 8 blocks); and in the configuration's
    own float64 precision through pic_step_n."""
    import numpy as np
    import torch
    import workloads as W
    import paper_1108_1954_gb300 as pic
    n, ng, L, K = 20000, 64, 4.0 * math.pi, 200
    x, v = W.two_stream(n, L, 0.2, 0.01, 1)
    x32, v32 = W.to_f32_state(x, v, L)
    run = pic.Run(pic.Params(npart=n, ncell=ng, length=L, dt=0.1, history=K + 1))
    run.init(x32, v32)
    run.step_n(32)                    # capture the graph
    run.init(x32, v32)
    s = run.stream
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record(s)
    run.step_n(K)
    e1.record(s)
    torch.cuda.synchronize()
    t_graph = e0.elapsed_time(e1) / 1e3
    run.close()
    # the configuration's own precision: float64 push, deposit and solve
    run = pic.Run(pic.Params(npart=n, ncell=ng, length=L, dt=0.1, history=K + 1,
                             precision=pic.PIC_FP64))
    x64, v64 = x.astype(np.float64), v.astype(np.float64)
    run.init(x64, v64)
    run.step_n(32)
    run.init(x64, v64)
    s = run.stream
    e0.record(s)
    run.step_n(K)
    e1.record(s)
    torch.cuda.synchronize()
    t_fp64 = e0.elapsed_time(e1) / 1e3
    run.close()
    best = None
    for cluster in (1, 2, 4, 8):
        pool = pic.Pool(max_slots=1, ncell_max=64, arena_bytes=1 << 24, history=K + 1,
                        variant=5, cluster=cluster, block=256)
        for rep in range(2):                 # the first pass warms up
            slot = pool.admit(pic.Params(npart=n, ncell=ng, length=L, dt=0.1), x32, v32, K)
            pool.advance(0)
            pool.sync()
            e0.record(pool.stream)
            pool.advance(K)
            e1.record(pool.stream)
            pool.sync()
            t = e0.elapsed_time(e1) / 1e3
            pool.release(slot)
        if best is None or t < best[0]:
            best = (t, cluster)
        pool.close()
    t_pool, cluster = best
    return {"npart": n, "ncell": ng, "steps": K,
            "us_per_step_graphs": 1e6 * t_graph / K, "us_per_step_one_launch": 1e6 * t_pool / K,
            "us_per_step_graphs_fp64": 1e6 * t_fp64 / K,
            "one_launch_shape": {"variant": 5, "cluster": cluster, "block": 256},
            "value_graphs": n * K / t_graph, "value_one_launch": n * K / t_pool,
            "unit": "particle-steps/s"}


# The paper's weak-scaling table (Sec. 5.2, Table 1): relative speed-up on
# P cores of NERSC Franklin (Cray XT4, one quad-core 2.3 GHz AMD Opteron
# "Budapest" per node, Berkeley UPC 2.10.2), ideal taken at P = 4.
PAPER_SPEEDUP = {4: 4.0, 8: 6.43, 12: 8.53, 16: 10.62, 20: 12.21, 24: 13.96, 28: 14.98,
                 32: 16.84, 64: 24.73, 128: 33.91}


def time_weak(args):
    """The paper's weak-scaling workload (Sec. 5.2): per core 64 cells, 64,000
    particles and a 3.1415-long box, a Maxwellian plasma (vth 0.2, no drift),
    1000 cycles, the CG solver forced to 150 iterations.  Here the P-core
    problem is one run on one GPU (NG = 64 P, N = 64,000 P, L = 3.1415 P),
    timed with the paper's CG (150 iterations) and with the exact solve;
    'speedup' is P T(4) / T(P), the paper's measure with ideal scaling
    assumed at P = 4.  'stacked' fills the GPU with 16 independent copies of
    the P = 64 problem in one pool launch (exact solve)."""
    import torch
    import paper_1108_1954_gb300 as pic
    steps = args.weak_steps
    cores = [4, 8, 16, 32, 64, 128]
    out = {"steps": steps, "cores": cores, "paper_speedup": PAPER_SPEEDUP,
           "paper_hardware": "NERSC Franklin, Cray XT4, quad-core 2.3 GHz AMD Opteron, "
                             "Berkeley UPC 2.10.2"}
    for name, solver in (("cg150", pic.PIC_SOLVER_CG), ("exact", pic.PIC_SOLVER_EXACT)):
        rows = []
        for P in cores:
            ng, n, L = 64 * P, 64000 * P, 3.1415 * P
            run = pic.Run(pic.Params(npart=n, ncell=ng, length=L, dt=0.1, sort_interval=20,
                                     field_solver=solver))
            ld = pic.Loading(v0=0.0, vth=0.2, seed=1000 + P)
            run.init_loaded(ld)
            run.step_n(40)                       # graphs captured, warm
            s = run.stream
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record(s)
            run.step_n(steps)
            e1.record(s)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            d = run.diagnostics(run.step - 1, 1)[0]
            run.close()
            rows.append({"P": P, "ncell": ng, "npart": n, "seconds": sec,
                         "us_per_step": 1e6 * sec / steps,
                         "particle_steps_per_s": n * steps / sec,
                         "kinetic_final": float(d["kinetic"])})
        t4 = rows[0]["seconds"]
        for r in rows:
            r["speedup"] = r["P"] * t4 / r["seconds"]
        out[name] = rows
    # 16 copies of the P = 64 problem, one launch per 50 steps
    P, R = 64, 16
    ng, n, L = 64 * P, 64000 * P, 3.1415 * P
    per = pic.pool_run_bytes(pic.Params(npart=n, ncell=ng, length=L), 8)
    pool = pic.Pool(max_slots=R, ncell_max=ng, arena_bytes=R * per + (64 << 20), history=8,
                    variant=getattr(args, "pool_variant", 5), cluster=8, block=512)
    for r in range(R):
        slot = pool.admit_loaded(pic.Params(npart=n, ncell=ng, length=L, dt=0.1),
                                 pic.Loading(v0=0.0, vth=0.2, seed=5000 + r), steps + 40)
        assert slot is not None
    pool.advance(40)
    pool.sync()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record(pool.stream)
    left = steps
    while left > 0:
        k = min(50, left)
        pool.advance(k)
        left -= k
    e1.record(pool.stream)
    pool.sync()
    sec = e0.elapsed_time(e1) / 1e3
    pool.close()
    out["stacked"] = {"runs": R, "P_each": P, "npart_total": R * n, "seconds": sec,
                      "particle_steps_per_s": R * n * steps / sec}
    return out


def time_served(args):
    """Config 5: Poisson arrivals (mean 200/s) of run requests served by the
    continuous-batching loop within a 150 GB device-memory budget."""
    import workloads as W
    import paper_1108_1954_gb300 as pic
    from paper_1108_1954_gb300 import serve
    stream = W.request_stream(args.serve_requests, 200.0, 11)
    reqs = serve.requests_from_stream(stream,
                                      modes_fn=lambda r: W.two_stream_modes_1_to_8(1e-4, r["seed"]))
    budget = 150 * (1 << 30)
    variant = getattr(args, "pool_variant", 5)
    srv = serve.Server(arena_bytes=budget, max_slots=2048, ncell_max=4096, history=8,
                       advance_steps=args.serve_advance, variant=variant, cluster=8, block=512)
    _, stats = srv.serve(reqs)
    srv.close()
    stats.update({"unit": "particle-steps/s", "budget_bytes": budget,
                  "arrival_rate_per_s": 200.0})
    return stats


def host_threads():
    """The host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def time_oracle(w, x32, v32, budget_s=12.0, sample=None, steps=None, threads=1):
    """The FP64 oracle on the same state (or its first `sample` particles):
    particle-steps/s, on one thread (orc_step) or on `threads` host threads
    (orc_step_threads, the same state bit for bit)."""
    import numpy as np
    import oracle as O
    n = w["npart"] if sample is None else min(sample, w["npart"])
    x = x32[:n].astype(np.float64)
    v = v32[:n].astype(np.float64)
    st = O.State(O.params(w["ncell"], n, w["length"], w["dt"]), x, v)
    done, t0 = 0, time.perf_counter()
    while True:
        if threads > 1:
            st.step_threads(threads)
        else:
            st.step()
        done += 1
        el = time.perf_counter() - t0
        if steps is not None and done >= steps:
            break
        if steps is None and el >= budget_s:
            break
    return dict(value=n * done / el, steps=done, npart=n, seconds=el, threads=threads)


def sig(x, digits=4):
    """x rounded to `digits` significant digits (floats only)."""
    if isinstance(x, float) and math.isfinite(x) and x != 0.0:
        return float("%.*g" % (digits, x))
    return x


def compact_weak(w):
    """The weak-scaling section as parallel lists (time per cycle in us and
    the paper's speed-up measure), short enough for a log tail."""
    out = {"P": w["cores"], "steps": w["steps"]}
    for name in ("cg150", "exact"):
        out[name + "_us_per_step"] = [sig(r["us_per_step"], 4) for r in w[name]]
        out[name + "_speedup"] = [sig(r["speedup"], 4) for r in w[name]]
    out["paper_speedup"] = [w["paper_speedup"][P] for P in w["cores"]]
    out["stacked_particle_steps_per_s"] = sig(w["stacked"]["particle_steps_per_s"])
    return out


def compact_precision(pr):
    """Config 4, one row per precision mode against the FP64 oracle."""
    out = {"npart": pr["npart"], "ncell": pr["ncell"], "steps": pr["steps"],
           "oracle_steps": pr["oracle"]["steps"], "oracle_gamma1": sig(pr["oracle"]["gamma1"]),
           "gamma_theory": sig(pr["gamma_theory"])}
    for name in ("fp64", "fp32_atomic", "fp32_fixed"):
        r = pr[name]
        out[name] = {"particle_steps_per_s": sig(r["particle_steps_per_s"], 3),
                     "energy_drift": sig(r["energy_drift"], 3),
                     "momentum_error": sig(r["momentum_error"], 2),
                     "gamma1_vs_oracle": sig(r["gamma1_vs_oracle"], 2),
                     "field_energy_vs_oracle": sig(r["field_energy_vs_oracle"], 2)}
    return out


def compact_batched(b):
    return {"runs": b["runs"], "steps": b["steps"], "particles": b["particles"],
            "value": sig(b["value"]), "plain_value": sig(b["plain_value"]),
            "speedup_vs_plain": sig(b["speedup_vs_plain"], 3), "unit": b["unit"],
            "launch": b["launch"], "tune_top": b["tune"][:3],
            "tune_sort_interval_ms_per_step": b["tune_sort_interval"]}


def compact_served(sv):
    keys = ("requests", "rejected", "p50_s", "p99_s", "mean_s", "value", "unit", "wall_s",
            "arrival_rate_per_s", "advance_steps", "mean_active")
    return {k: sig(sv[k]) for k in keys if k in sv}


def main():
    args = parse()
    ws, rank, local = dist_env()
    w = workload(args.workload)

    if args.impl == "reference":
        if rank != 0:
            return
        # a bounded sample of the workload: the same recipe (cells, box,
        # beams, modes, seed) at REF_SAMPLE electrons, so that its density
        # and field are those of the full run
        ws_ = dict(w, npart=min(REF_SAMPLE, w["npart"]))
        x32, v32 = make_state(ws_)
        K, Wm = args.steps, args.warmup
        nt = host_threads()
        time_oracle(ws_, x32, v32, steps=max(1, Wm), threads=nt)
        r = time_oracle(ws_, x32, v32, steps=max(1, K), threads=nt)
        line = {
            "impl": "reference", "metric": "particle-steps/s",
            "value": r["value"], "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": K, "warmup": Wm, "ms_per_step": 1e3 * r["seconds"] / r["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "single large run, %d electrons, %d cells (oracle sample %d)"
                       % (w["npart"], w["ncell"], r["npart"])},
            "cpu_baseline": {"value": r["value"], "unit": "particle-steps/s", "cores": nt,
                             "kind": "oracle", "cpu": cpu_model(),
                             "sample": "FP64 oracle on %d host threads, the same recipe at %d "
                                       "electrons (cells, box, beams, modes unchanged), %d steps"
                             % (nt, r["npart"], r["steps"])},
            "e2e": {"value": r["value"], "unit": "particle-steps/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line))
        return

    import torch
    if ws > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    if args.only_batched:
        print(json.dumps({"batched": time_batched(args)}))
        return
    if args.only_precision:
        print(json.dumps({"precision": precision_study(args)}))
        return
    if args.only_variant_scan:
        print(json.dumps({"variant_scan_push_ms": variant_scan(args)}))
        return
    if args.only_weak:
        print(json.dumps({"weak": time_weak(args)}))
        return
    if args.only_c1:
        print(json.dumps({"c1": time_c1(args)}))
        return
    x32, v32 = make_state(w)
    res = time_ours(args, w, x32, v32)
    sharded = time_sharded(args, w, x32, v32) if ws > 1 else None
    e2e = None if args.no_e2e else time_e2e(args, w, x32, v32)
    c1 = None if args.no_c1 else time_c1(args)
    batched = None if args.no_batched else time_batched(args)
    served = None if args.no_served else time_served(args)
    weak = None if args.no_weak else time_weak(args)
    precision = precision_study(args) if (not args.no_precision and rank == 0) else None

    n, K = w["npart"], res["steps"]
    value, total_s = rank_aggregate(res["total_ms"] / 1e3, n, K, ws, device="cuda")
    push_avg_s = statistics.mean(res["push_ms"]) / 1e3
    achieved = BYTES_PER_PARTICLE_STEP * n / push_avg_s / 1e9
    peak, src = measured_peak()
    cpu = None
    if rank == 0 and not args.no_cpu:
        nt = host_threads()
        one = time_oracle(w, x32, v32, budget_s=10.0)
        c = time_oracle(w, x32, v32, budget_s=10.0, threads=nt) if nt > 1 else one
        cpu = {"value": c["value"], "unit": "particle-steps/s", "cores": nt, "kind": "oracle",
               "cpu": cpu_model(),
               "sample": "FP64 oracle on the full %d-particle state, first %d steps (%.1f s) on "
                         "%d host threads" % (c["npart"], c["steps"], c["seconds"], nt),
               "value_1core": one["value"],
               "sample_1core": "the same on one thread: first %d steps (%.1f s)"
                               % (one["steps"], one["seconds"])}
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    line = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
        "n_gpus": ws, "steps": K, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "single large run: %d electrons, %d cells, L=4pi, two-stream "
                               "+-0.2 vth 0.01, modes 1-8 at 1e-4, dt 0.1, sort every %d steps"
                               % (n, w["ncell"], w["sort_interval"]),
                   "npart": n, "ncell": w["ncell"], "sort_interval": w["sort_interval"],
                   "precision": "f32 push, int64 fixed-point deposit, f64 field solve",
                   "l2": "inputs larger than L2 (%.0f MiB particle state)" % (16 * n / 2**20 / 2),
                   "launch": {"grid": res["grid"], "block": res["block"],
                              "deposit_variant": res["variant"], "unroll": res["unroll"],
                              "blocks_per_sm": res["blocks_per_sm"]},
                   "sort_interval_tuner": res["sort_tune"]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(res["variant"], res["unroll"]),
                     "kernel": push_kernel_name(res["variant"]), "peak_source": src,
                     "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP,
                     "push_ms_avg": push_avg_s * 1e3,
                     "push_ms_by_window": [round(statistics.mean(res["push_ms"][i:i + 100]), 4)
                                           for i in range(0, len(res["push_ms"]), 100)],
                     "push_timing": "CUDA events around each push on the run's stream, over "
                                    "the K steps that follow the timed region, one call per "
                                    "kernel",
                     "copy_floor_ms": res["floor_ms"],
                     "copy_floor": "the same 16 B per particle (x, v float32 read and written "
                                   "in place) streamed by torch's elementwise kernel "
                                   "(x.mul_(1); v.mul_(1))"},
        "timing": "value: CUDA events around pic_step_n(K) (CUDA graphs of whole sort "
                  "periods) on the run's stream, after warm-up and graph capture",
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
        "paper_context": {"weak_scaling_speedup": PAPER_SPEEDUP,
                          "hardware": "NERSC Franklin, Cray XT4, quad-core 2.3 GHz AMD Opteron, "
                                      "Berkeley UPC 2.10.2",
                          "note": "relative speed-up on P cores, ideal assumed at P = 4; "
                                  "context, not a target"},
    }
    if e2e is not None:
        line["e2e"] = {"value": e2e["value"], "unit": "particle-steps/s",
                       "h2d_bytes_per_step": e2e["h2d_per_step"],
                       "d2h_bytes_per_step": e2e["d2h_per_step"],
                       "timing": "host clock, mean of %d whole passes (upload, steps, "
                                 "diagnostics and state back)" % e2e["passes"],
                       "pass_s": e2e["pass_s"], "launch": e2e["launch"]}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if sharded is not None:
        line["sharded"] = {k: sig(v) for k, v in sharded.items()}
    # the sections of the metric beyond the single run come last, compact,
    # so that the end of the line carries them: weak scaling, config 1, the
    # precision study, batched vs plain, served latency
    if weak is not None:
        line["weak"] = compact_weak(weak)
    if c1 is not None:
        line["c1"] = {k: sig(v) for k, v in c1.items()}
    if precision is not None:
        line["precision"] = compact_precision(precision)
    if batched is not None:
        line["batched"] = compact_batched(batched)
    if served is not None:
        line["served"] = compact_served(served)
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
