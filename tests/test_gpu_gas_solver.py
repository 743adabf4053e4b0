"""The gas phase solved on the GPU (DEM_GAS_SOLVER: eqs (3-24), (4-2), (4-6), (4-9) with the
pseudo-turbulence closures (3-28)..(3-37)), through the C ABI, against the FP64 oracle:
the cell-centre velocities and pressures, the gas state and the parcel state after several
coupling steps of reacting beds with immersed-boundary cells; two beds of different grids in
one context (one global pressure system); the FP32 forms within their precision; a captured
graph equal to the stream path; the calls a solving context refuses."""
import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

from paper_2311_03908_gb300 import binding  # noqa: E402


def _ctx(bed, prec="fp64"):
    return binding.Context(bed, precision=prec, stream=torch.cuda.current_stream().cuda_stream)


def _rel(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def _solved(seed, wall, n=2500, nx=8, nz=40, ncouple=10, flags=0):
    bed = synth.small_packed(seed=seed, n=n, v_scale=0.3, wall_kind=wall, nx=nx, nz=nz, H=0.0018 * nz,
                             flags=flags | synth.GAS_SOLVER)
    for c in bed.beds:
        c.coupling_interval = ncouple
    return bed


def _two_beds(seed):
    """Two beds of different grids and walls in one context (beds hold their faces in order)."""
    a = _solved(seed, synth.WALL_CONE, n=1500, nx=8, nz=40)
    b = _solved(seed + 1, synth.WALL_FLAT, n=1000, nx=6, nz=30)
    cat = lambda f: np.concatenate([getattr(a, f), getattr(b, f)])
    return synth.Bed([a.beds[0], b.beds[0]], cat("x"), cat("y"), cat("z"), cat("vx"), cat("vy"), cat("vz"),
                     cat("d_real"), cat("T"), np.concatenate([a.m0, b.m0], axis=1), cat("ore"),
                     np.concatenate([np.zeros(a.n, np.int32), np.ones(b.n, np.int32)]), "two-beds")


def _compare(ctx, ref, tol_flow, tol_gas, tol_state):
    fg, it = ctx.dem_get_flow()
    fo = ref.flow()
    assert it > 0
    for q in range(3):
        assert _rel(fg[:, q], fo[:, q]) < tol_flow, ("u", q, _rel(fg[:, q], fo[:, q]))
    assert _rel(fg[:, 3], fo[:, 3]) < tol_flow, ("p", _rel(fg[:, 3], fo[:, 3]))
    gg, go = ctx.dem_get_gas(), ref.gas()
    for col in range(5):
        assert _rel(gg[:, col], go[:, col]) < tol_gas, ("gas", col, _rel(gg[:, col], go[:, col]))
    sg, so = ctx.dem_get_state(), ref.state()
    for row in range(binding.DEM_NSTATE):
        assert _rel(sg[row], so[row]) < tol_state, (binding.STATE_ROWS[row], _rel(sg[row], so[row]))


@pytest.mark.parametrize("wall", [synth.WALL_FLAT, synth.WALL_CONE])
def test_gas_solver_fp64_against_oracle(wall):
    bed = _solved(31, wall)
    ctx = _ctx(bed)
    ref = oracle.Oracle(bed)
    f0, _ = ctx.dem_get_flow()
    assert _rel(f0, ref.flow()) < 1e-14              # the initial plug flow
    for _ in range(3):
        ctx.dem_step(10)
        ref.step(10)
        _compare(ctx, ref, 1e-8, 1e-10, 1e-7)
    # the solved flow is not the plug flow: cross flow around the parcels and walls
    fg, _ = ctx.dem_get_flow()
    assert np.abs(fg[:, :2]).max() > 1e-4 * bed.beds[0].U_in
    ctx.close()


@pytest.mark.parametrize("sweeps", [0, 1])
def test_gas_solver_preconditioners(sweeps):
    # the Jacobi preconditioner and the one-sweep V-cycle reach the same solution (the default,
    # two sweeps, runs in the other tests)
    bed = _solved(33, synth.WALL_CONE)
    ctx = _ctx(bed)
    ctx.dem_set_tuning(gas_mg_sweeps=sweeps, gas_mg_weight_pct=100)
    ref = oracle.Oracle(bed)
    for _ in range(2):
        ctx.dem_step(10)
        ref.step(10)
        _compare(ctx, ref, 1e-8, 1e-10, 1e-7)
    ctx.close()


def test_gas_solver_two_beds_fp64():
    bed = _two_beds(41)
    ctx = _ctx(bed)
    ref = oracle.Oracle(bed)
    for _ in range(2):
        ctx.dem_step(10)
        ref.step(10)
        _compare(ctx, ref, 1e-8, 1e-10, 1e-7)
    ctx.close()


@pytest.mark.parametrize("prec", ["split", "split_kahan"])
def test_gas_solver_fp32_forms(prec):
    bed = _solved(51, synth.WALL_CONE)
    ctx = _ctx(bed, prec)
    ref = oracle.Oracle(bed)
    ctx.dem_step(20)
    ref.step(20)
    fg, fo = ctx.dem_get_flow()[0], ref.flow()
    # the parcels' FP32 velocities and sources enter the drag sums and the mass source
    for q in range(4):
        assert _rel(fg[:, q], fo[:, q]) < 2e-3, q
    gg, go = ctx.dem_get_gas(), ref.gas()
    assert _rel(gg[:, 4], go[:, 4]) < 1e-5                      # T
    for col in (1, 2):
        assert np.abs(gg[:, col] - go[:, col]).max() < 1e-5      # Y_H2, Y_H2O
    ctx.close()


def test_gas_solver_graph_equals_stream():
    bed = _solved(61, synth.WALL_CONE)
    a, b = _ctx(bed), _ctx(bed)
    a.dem_step(20)
    for _ in range(2):
        b.dem_step_graph(10)
    fa, fb = a.dem_get_flow()[0], b.dem_get_flow()[0]
    assert np.array_equal(fa, fb)
    assert np.array_equal(a.dem_get_gas(), b.dem_get_gas())
    assert np.array_equal(a.dem_get_state(), b.dem_get_state())
    a.close()
    b.close()


def test_gas_solver_refusals():
    bed = _solved(71, synth.WALL_FLAT, n=500)
    ctx = _ctx(bed)
    nc = ctx.ncells
    with pytest.raises(binding.DemError):
        ctx.dem_set_gas(np.tile([1.0, 0.0, 0.0], (nc, 1)), np.full(nc, 1000.0))
    with pytest.raises(binding.DemError):
        ctx.dem_adjoint(10, 5)
    ctx.close()
    # every bed or none; one coupling interval; not with the frozen gas
    two = _two_beds(81)
    two.beds[1].flags &= ~synth.GAS_SOLVER
    with pytest.raises(binding.DemError):
        _ctx(two)
    two = _two_beds(82)
    two.beds[1].coupling_interval = 5
    with pytest.raises(binding.DemError):
        _ctx(two)
    bed.beds[0].flags |= synth.NO_GAS_UPDATE
    with pytest.raises(binding.DemError):
        _ctx(bed)


def test_prescribed_flow_reported():
    bed = synth.small_packed(seed=3, n=500)
    ctx = _ctx(bed)
    ctx.dem_step(2)
    fg, it = ctx.dem_get_flow()
    eps = ctx.dem_get_gas()[:, 0]
    assert it == 0
    assert np.array_equal(fg[:, :2], np.zeros((ctx.ncells, 2))) and np.all(fg[:, 3] == 0)
    assert np.allclose(fg[:, 2], bed.beds[0].U_in / eps, rtol=1e-15)
    ctx.close()


def test_gas_solver_reacting_column_long_run():
    # a reacting column over 6000 steps (600 gas steps), static parcels: the H2O front passes
    # the outlet; flow, gas and parcel state against the oracle every 1000 steps
    from tests.helpers import bed_from_arrays
    cfg = synth.BedConfig(D=0.004, H=0.024, nx=1, ny=1, nz=8, dt=1e-5, cg_ratio=4.0, U_in=0.2, T_in=1000.0,
                          coupling_interval=10, Y_in=(0.9, 0.05, 0.05), kn=1e-3,
                          flags=synth.GAS_SOLVER | synth.NO_GRAVITY | synth.NO_CONTACTS | synth.NO_DRAG)
    rng = np.random.default_rng(3)
    n = 40
    bed = bed_from_arrays(cfg, rng.uniform(-0.001, 0.001, n), rng.uniform(-0.001, 0.001, n),
                          rng.uniform(0.004, 0.012, n), d_real=100e-6, T=1000.0, comp=(1.0, 0.0, 0.0, 0.0))
    ctx = _ctx(bed)
    ref = oracle.Oracle(bed)
    for _ in range(6):
        ctx.dem_step(1000)
        ref.step(1000)
        _compare(ctx, ref, 1e-7, 1e-9, 1e-9)
    assert ctx.dem_get_gas()[-1, 2] > 0.4
    ctx.close()
