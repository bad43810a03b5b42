"""CUDA path against the FP64 oracle, through the C ABI.

* the fixed-point density: bit for bit against the oracle's fixed-point
  deposit of the GPU's own float32 cell coordinates (read back with
  get_cells; at init they are the documented conversion of the uploaded x);
* the field: against the oracle's direct solve of the same integer density
  (1e-9 of max |E|) and of its FP64 deposit;
* one step from identical states: positions within 1e-5 L (periodic
  distance), velocities within 1e-5 max(|v|, v0 + vth);
* the deposit variants and launch shapes give identical integers;
* edge cases: ragged N, N = 1, 3, 5, NG = 1, NG = PIC_NCELL_MAX, bad input.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from units import to_cells

import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402,F401

pytestmark = pytest.mark.gpu
L4PI = 4.0 * math.pi


def periodic_dist(a, b, L):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    return np.minimum(d, L - d)


def make_run(n, ng, L, **kw):
    return pic.Run(pic.Params(npart=n, ncell=ng, length=L, **kw), device="cuda:0")


def check_field_against_oracle(f, n, ng, L, dt=0.1):
    """E from the GPU's integer density vs the oracle's direct solve of it."""
    p = O.params(ng, n, L, dt)
    rho_ref = O.rho_from_fixed(p, f["rho_q"])
    phi_ref, E_ref = O.field(p, rho_ref)
    np.testing.assert_allclose(f["rho"], rho_ref, rtol=0, atol=1e-13 * max(1.0, np.abs(rho_ref).max()))
    escale = max(np.abs(E_ref).max(), 1e-300)
    assert np.abs(f["E"] - E_ref).max() <= 1e-9 * escale
    pscale = max(np.abs(phi_ref).max(), 1e-300)
    assert np.abs(f["phi"] - phi_ref).max() <= 1e-9 * pscale


def fp32_field_bound(n, ng, L):
    """Bound on |E_fixed - E_fp64| at the nodes when the FP64 deposit takes the
    caller's float32 positions x and the device its cell coordinates
    u = (float)(x NG/L).

    u carries a relative rounding of 2^-24, so a particle's cell fraction f is
    off by up to u 2^-24 <= NG 2^-24 (the 2^-24 truncation of the fixed-point
    weight is smaller still).  The error moves charge (NG/N) df between the
    particle's two nodes, so the prefix sum S_g of Eq. 6 only sees the ~N/NG
    particles between nodes g and g+1: |dS_g| ~ (NG/N) sqrt(N/NG) NG 2^-24.
    E_g = (L/(2 NG)) (S_g + S_{g-1} - 2 mean S) then gives
    |dE| ~ L sqrt(NG/N) 2^-24; 16 times that covers the largest of 8192 nodes
    with room.  The box is exactly [0, NG) in cell units, so no term grows
    with the box length's float32 rounding."""
    return 16.0 * L * math.sqrt(ng / n) * 2.0 ** -24 + 1e-15


def one_step_parity(n, ng, L, seed, v0=0.2, vth=0.01, **kw):
    x, v = W.two_stream(n, L, v0, vth, seed, modes=W.two_stream_modes_1_to_8(1e-4, seed))
    x32, v32 = W.to_f32_state(x, v, L)
    run = make_run(n, ng, L, **kw)
    run.init(x32, v32)
    f0 = run.get_field()
    u0, _ = run.get_cells()
    assert np.array_equal(u0, to_cells(x32, ng, L))
    assert np.array_equal(f0["rho_q"], O.deposit_fixed(ng, u0))
    assert int(f0["rho_q"].sum()) == n << O.FIX_BITS
    check_field_against_oracle(f0, n, ng, L)

    ref = O.State(O.params(ng, n, L, 0.1), x32.astype(np.float64), v32.astype(np.float64))
    assert np.abs(f0["E"] - ref.E).max() <= fp32_field_bound(n, ng, L)
    run.push()
    run.solve_field()
    x1, v1 = run.get_state()
    svv, sv = ref.step()
    assert periodic_dist(x1, ref.x, L).max() <= 1e-5 * L
    vscale = np.maximum(np.abs(ref.v), v0 + vth)
    assert (np.abs(v1 - ref.v) <= 1e-5 * vscale).all()
    f1 = run.get_field()
    assert np.array_equal(f1["rho_q"], O.deposit_fixed(ng, run.get_cells()[0]))
    check_field_against_oracle(f1, n, ng, L)
    d = run.diagnostics(0, 2)
    assert d["step"].tolist() == [0, 1]
    assert d["charge_q"].tolist() == [n << O.FIX_BITS] * 2
    m = ref.mass
    assert abs(d["kinetic"][0] - 0.5 * m * svv) <= 1e-5 * abs(0.5 * m * svv)
    assert abs(d["momentum"][0] - m * sv) <= 1e-5 * m * np.abs(ref.v).sum()
    assert math.isnan(d["kinetic"][1])
    assert abs(d["field"][1] - O.field_energy(O.params(ng, n, L), f1["E"])) <= 1e-12 * d["field"][1]
    run.close()
    return x1, v1, f1


@pytest.mark.parametrize("n,ng", [(20000, 64), (20001, 64), (20003, 256),
                                  (100000, 1024), (262147, 4096), (50000, 8192)])
def test_one_step_parity(n, ng):
    one_step_parity(n, ng, L4PI, seed=n + ng)


@pytest.mark.parametrize("variant", [1, 2, 5, 6])
@pytest.mark.parametrize("block", [64, 256, 512])
@pytest.mark.parametrize("unroll", [1, 2, 4])
def test_deposit_variants_and_shapes_identical(variant, block, unroll):
    n, ng = 70001, 512
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 3)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    ref = make_run(n, ng, L4PI, deposit_variant=1, block_size=256)
    ref.init(x32, v32)
    ref.step_n(3)
    run = make_run(n, ng, L4PI, deposit_variant=variant, block_size=block, unroll=unroll)
    run.init(x32, v32)
    run.step_n(3)
    assert np.array_equal(run.get_field()["rho_q"], ref.get_field()["rho_q"])
    xa, va = run.get_state()
    xb, vb = ref.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


@pytest.mark.parametrize("variant", [8, 9])
@pytest.mark.parametrize("block", [64, 256, 512])
@pytest.mark.parametrize("unroll", [1, 2])
def test_eight_particle_groups_identical(variant, block, unroll):
    # the 32-byte group variants give the ATOMIC kernel's particles and
    # integers bit for bit, with the N mod 8 tail
    n, ng = 70005, 512
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 3)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    ref = make_run(n, ng, L4PI, deposit_variant=1, block_size=256)
    ref.init(x32, v32)
    ref.step_n(3)
    run = make_run(n, ng, L4PI, deposit_variant=variant, block_size=block, unroll=unroll)
    run.init(x32, v32)
    run.step_n(3)
    assert np.array_equal(run.get_field()["rho_q"], ref.get_field()["rho_q"])
    assert np.array_equal(run.get_cells()[0], ref.get_cells()[0])
    assert np.array_equal(run.get_cells()[1], ref.get_cells()[1])
    with pytest.raises(pic.PicError):
        run.set_launch(variant, block, 4)           # no 4-group build of these


def test_autotune_cache_adopts_the_stored_shape(tmp_path):
    # a second run of the same kind takes the first run's shape from the file
    n, ng = 200003, 1024
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 4)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    path = str(tmp_path / "shapes.json")
    a = make_run(n, ng, L4PI, sort_interval=5)
    a.init(x32, v32)
    table = a.autotune(reps=2, cache=path)
    assert len(table) > 1
    shape = a.launch_shape()
    b = make_run(n, ng, L4PI, sort_interval=5)
    b.init(x32, v32)
    b.set_launch(1, 256, 1)
    assert len(b.autotune(reps=2, cache=path)) == 0         # no timing: from the file
    assert b.launch_shape()[1:] == shape[1:]
    a.step_n(6)
    b.step_n(6)
    assert np.array_equal(a.get_cells()[0], b.get_cells()[0])
    a.close()
    b.close()


def test_all_particles_in_one_cell():
    # every particle in one cell: a block's low words wrap many times and the
    # carries into the high words must all be counted
    n, ng, L = 300001, 64, 64.0
    x32 = np.full(n, 10.3, dtype=np.float32)
    v32 = np.zeros(n, dtype=np.float32)
    for variant in (1, 2, 5, 6, 8, 9):
        run = make_run(n, ng, L, deposit_variant=variant, block_size=256, blocks_per_sm=1)
        run.init(x32, v32)
        assert np.array_equal(run.get_field()["rho_q"], O.deposit_fixed(ng, run.get_cells()[0]))


@pytest.mark.parametrize("variant,block,unroll", [(1, 512, 1), (5, 64, 4), (2, 256, 2),
                                                  (8, 512, 1), (9, 256, 2)])
def test_one_node_of_a_tile_wraps_many_times(variant, block, unroll):
    # 2^24 particles at one position, one block per SM: a block adds ~110,000
    # weights of about 2^24 to each of two nodes of its tile, so each node's
    # low word wraps thousands of times and every carry must reach the high
    # word.  The exact sums are N (2^24 - W) and N W.
    n, ng = 1 << 24, 64
    u = np.float32(10.3)
    x32 = np.full(n, u * np.float32(2.0 / ng), dtype=np.float32)   # L = 2: x = u dx
    v32 = np.zeros(n, dtype=np.float32)
    run = make_run(n, ng, 2.0, deposit_variant=variant, block_size=block, unroll=unroll,
                   blocks_per_sm=1)
    run.init(x32, v32)
    uc, _ = run.get_cells()
    want = O.deposit_fixed(ng, uc)
    assert np.count_nonzero(want) == 2 and np.unique(uc).size == 1
    assert np.array_equal(run.get_field()["rho_q"], want)
    run.deposit()
    run.solve_field()
    assert np.array_equal(run.get_field()["rho_q"], want)
    run.close()


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7])
def test_tiny_and_ragged(n):
    ng, L = 16, 3.0
    rng = np.random.default_rng(n)
    x32 = rng.uniform(0, L, n).astype(np.float32)
    v32 = rng.uniform(-0.3, 0.3, n).astype(np.float32)
    run = make_run(n, ng, L)
    run.init(x32, v32)
    assert np.array_equal(run.get_field()["rho_q"], O.deposit_fixed(ng, to_cells(x32, ng, L)))
    ref = O.State(O.params(ng, n, L, 0.1), x32.astype(np.float64), v32.astype(np.float64))
    for _ in range(5):
        run.step_n(1)
        ref.step()
        x1, v1 = run.get_state()
        assert periodic_dist(x1, ref.x, L).max() <= 1e-5 * L
        assert np.abs(v1 - ref.v).max() <= 1e-5 * 0.3
        assert np.array_equal(run.get_field()["rho_q"], O.deposit_fixed(ng, run.get_cells()[0]))


def test_single_particle_moves_freely():
    L, dt = L4PI, 0.1
    run = make_run(1, 64, L)
    x0, v0 = np.float32(1.234), np.float32(0.37)
    run.init(np.array([x0]), np.array([v0]))
    run.step_n(300)
    x, v = run.get_state()
    # the self-force vanishes up to the float32 gather weight against the
    # 2^-24 deposit weight: |dv| stays at the 1e-5 level over 300 steps
    assert abs(float(v[0]) - float(v0)) < 1e-4
    want = math.fmod(float(x0) + 300 * float(v0) * dt, L)
    assert periodic_dist(x, want, L).max() < 1e-3


def test_one_cell_grid_has_no_field():
    n, L = 1000, 5.0
    rng = np.random.default_rng(9)
    x32 = rng.uniform(0, L, n).astype(np.float32)
    v32 = rng.uniform(-0.1, 0.1, n).astype(np.float32)
    run = make_run(n, 1, L)
    run.init(x32, v32)
    f = run.get_field()
    assert f["rho_q"].tolist() == [n << O.FIX_BITS]
    assert f["E"].tolist() == [0.0] and f["phi"].tolist() == [0.0]
    run.step_n(10)
    x, v = run.get_state()
    assert np.array_equal(v, v32)


def test_bad_input_and_call_order():
    n, ng, L = 100, 16, 2.0
    run = make_run(n, ng, L)
    with pytest.raises(pic.PicError) as e:
        run.push()
    assert e.value.code == pic.PIC_ESTATE
    x = np.linspace(0, L, n, endpoint=False).astype(np.float32)
    bad = x.copy()
    bad[7] = np.float32(L)
    with pytest.raises(pic.PicError) as e:
        run.init(bad, np.zeros(n, np.float32))
    assert e.value.code == pic.PIC_EINVAL
    with pytest.raises(pic.PicError) as e:       # a rejected upload leaves no state
        run.push()
    assert e.value.code == pic.PIC_ESTATE
    bad[7] = np.nan
    with pytest.raises(pic.PicError):
        run.init(bad, np.zeros(n, np.float32))
    run.init(x, np.zeros(n, np.float32))
    run.push()
    with pytest.raises(pic.PicError) as e:
        run.push()
    assert e.value.code == pic.PIC_ESTATE
    with pytest.raises(pic.PicError) as e:
        run.step_n(1)
    assert e.value.code == pic.PIC_ESTATE
    run.solve_field()
    run.step_n(2)
    assert run.step == 3
    with pytest.raises(pic.PicError):
        run.diagnostics(0, 10)       # beyond the current step
    run.sync()


def test_deposit_then_solve_reproduces_the_field():
    n, ng, L = 30000, 128, L4PI
    x, v = W.two_stream(n, L, 0.2, 0.01, 4)
    run = make_run(n, ng, L)
    run.init(*W.to_f32_state(x, v, L))
    run.step_n(5)
    f = run.get_field()
    run.deposit()
    run.solve_field()
    g = run.get_field()
    assert run.step == 5
    assert np.array_equal(f["rho_q"], g["rho_q"]) and np.array_equal(f["E"], g["E"])


def test_autotune_leaves_state_and_results_unchanged():
    n, ng = 300001, 1024
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 12)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    a = make_run(n, ng, L4PI, sort_interval=5)
    b = make_run(n, ng, L4PI, sort_interval=5)
    a.init(x32, v32)
    b.init(x32, v32)
    a.step_n(7)
    b.step_n(7)
    table = a.autotune(reps=2)
    assert len(table) >= 20 and (table["ms"] > 0).all()
    g, blk, var, _ = a.launch_shape()
    best = table[np.argmin(table["ms"])]
    assert (var, blk) == (int(best["variant"]), int(best["block"]))
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    a.step_n(9)
    b.step_n(9)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.get_field()["rho_q"], b.get_field()["rho_q"])


@pytest.mark.parametrize("n,ng", [(1, 16), (2047, 64), (2048, 64), (2049, 64),
                                  (70001, 512), (300000, 4096), (100003, 8192)])
def test_ragged_sizes_identical_across_variants(n, ng):
    # around the float4 groups and whole blocks of groups, and at the largest
    # grid: every variant gives the particles and the integer density of the
    # ATOMIC kernel bit for bit, through sorts
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 5 + n)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    ref = make_run(n, ng, L4PI, deposit_variant=1, block_size=256, sort_interval=4)
    ref.init(x32, v32)
    ref.step_n(9)
    xb, vb = ref.get_state()
    for variant, block, unroll in ((5, 512, 1), (6, 512, 2), (2, 128, 4), (8, 512, 1),
                                   (9, 256, 2), (8, 128, 2)):
        run = make_run(n, ng, L4PI, deposit_variant=variant, block_size=block,
                       unroll=unroll, sort_interval=4)
        run.init(x32, v32)
        run.step_n(9)
        assert np.array_equal(run.get_field()["rho_q"], ref.get_field()["rho_q"])
        xa, va = run.get_state()
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        assert run.launch_shape()[2] == variant
        da, db = run.diagnostics(0, 9), ref.diagnostics(0, 9)
        assert np.allclose(da["kinetic"], db["kinetic"], rtol=1e-5)
        run.close()


def test_partial_read_back_and_reload():
    # pic_get_state with only x or only v (the velocities go down on the
    # run's private stream), and pic_init from the read-back state: the same
    # arrays and the same next steps as the full read-back
    from paper_1108_1954_gb300 import _lib, _VP
    n, ng = 100003, 512
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 8)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    run = make_run(n, ng, L4PI, sort_interval=3)
    run.init(x32, v32)
    run.step_n(5)
    xa, va = run.get_state()
    xo = np.full(n, np.nan, np.float32)
    vo = np.full(n, np.nan, np.float32)
    assert _lib.pic_get_state(run._h, _VP(xo.ctypes.data), None) == 0
    assert np.array_equal(xo, xa)
    assert _lib.pic_get_state(run._h, None, _VP(vo.ctypes.data)) == 0
    assert np.array_equal(vo, va)
    # the run goes on unchanged after the read-backs
    other = make_run(n, ng, L4PI, sort_interval=3)
    other.init(x32, v32)
    other.step_n(9)
    run.step_n(4)
    assert np.array_equal(run.get_cells()[0], other.get_cells()[0])
    assert np.array_equal(run.get_field()["rho_q"], other.get_field()["rho_q"])
    run.close()
    other.close()
