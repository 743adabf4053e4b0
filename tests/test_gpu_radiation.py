"""Parity of the particle radiation (eqs 3-16, 3-17, 3-51) between the CUDA path and the
FP64 oracle, on the GPU.

The beds have every parcel at its own temperature, so the neighbourhood means T_se differ
from parcel to parcel. With cg_ratio 6 the sphere of radius 1.5 d_CGP of the largest
parcels reaches past the neighbouring cell (the kernel's 5 x 5 x 5 cell stencil); with 4 it
stays inside the 27 cells around. Tolerances: FP64 form 1e-9 relative over 10 steps (the
neighbourhoods are exact, only the order of the temperature sums differs); FP32 forms:
T_se to 1e-6 and Q_rad to 1e-4 of the bed's largest |Q_rad| after one step (FP32 sums and
cell-local coordinates), the temperature to 1e-5 after 10 steps.
"""
import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

from paper_2311_03908_gb300 import binding  # noqa: E402

TSE, QRAD = binding.DIAG_ROWS.index("Tse"), binding.DIAG_ROWS.index("Qrad")


def _ctx(bed, prec="fp64"):
    c = binding.Context(bed, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    c.dem_set_diagnostics(True)
    return c


def _rel(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def _bed(seed, n=2500, cg=4.0, flags=synth.RADIATION, wall=synth.WALL_CONE):
    b = synth.small_packed(seed=seed, n=n, v_scale=0.2, T0=1073.0, wall_kind=wall, cg_ratio=cg, flags=flags)
    b.T = 850.0 + 300.0 * np.random.default_rng(seed).random(b.x.size)
    return b


@pytest.mark.parametrize("cg", [4.0, 6.0])
def test_fp64_radiation_matches_oracle(cg):
    bed = _bed(40, cg=cg)
    ctx, ref = _ctx(bed), oracle.Oracle(bed)
    ctx.dem_step(1)
    ref.step(1)
    dg, do = ctx.dem_get_diag(), ref.diag()
    assert np.abs(do[oracle.D_QRAD]).max() > 0
    assert _rel(dg[TSE], do[oracle.D_TSE]) < 1e-12
    assert _rel(dg[QRAD], do[oracle.D_QRAD]) < 1e-9
    ctx.dem_step(9)
    ref.step(9)
    sg, so = ctx.dem_get_state(), ref.state()
    for row in range(binding.DEM_NSTATE):
        assert _rel(sg[row], so[row]) < 1e-9, binding.STATE_ROWS[row]
    dg, do = ctx.dem_get_diag(), ref.diag()
    assert _rel(dg[TSE], do[oracle.D_TSE]) < 1e-9 and _rel(dg[QRAD], do[oracle.D_QRAD]) < 1e-9
    ctx.close()


@pytest.mark.parametrize("prec", ["split", "split_kahan"])
def test_fp32_forms_radiation(prec):
    bed = _bed(41, cg=6.0)
    ctx, ref = _ctx(bed, prec), oracle.Oracle(bed)
    ctx.dem_step(1)
    ref.step(1)
    dg, do = ctx.dem_get_diag(), ref.diag()
    assert _rel(dg[TSE], do[oracle.D_TSE]) < 1e-6
    assert _rel(dg[QRAD], do[oracle.D_QRAD]) < 1e-4
    ctx.dem_step(9)
    ref.step(9)
    assert _rel(ctx.dem_get_state()[9], ref.state()[9]) < 1e-5
    ctx.close()


def test_radiating_and_plain_beds_in_one_context():
    parts = [_bed(42, n=900), _bed(43, n=700, flags=0)]
    beds = [p.beds[0] for p in parts]
    cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
    bedid = np.concatenate([np.full(p.n, i, np.int32) for i, p in enumerate(parts)])
    bed = synth.Bed(beds, cat("x"), cat("y"), cat("z"), cat("vx"), cat("vy"), cat("vz"), cat("d_real"),
                    cat("T"), np.concatenate([p.m0 for p in parts], axis=1), cat("ore"), bedid, "mixed")
    ctx, ref = _ctx(bed), oracle.Oracle(bed)
    ctx.dem_step(5)
    ref.step(5)
    sg, so = ctx.dem_get_state(), ref.state()
    for row in range(binding.DEM_NSTATE):
        assert _rel(sg[row], so[row]) < 1e-9, binding.STATE_ROWS[row]
    dg = ctx.dem_get_diag()
    plain = bedid == 1
    assert not dg[TSE][plain].any() and not dg[QRAD][plain].any()
    assert (dg[TSE][~plain] > 0).all()
    ctx.close()


def test_radiation_off_is_the_plain_step():
    # the switch off: no radiation kernel, and the step is the one without radiation
    bed = _bed(44, n=800, flags=0)
    ctx = _ctx(bed)
    ctx.dem_profile(True)
    ctx.dem_step(3)
    assert "k_radiation" not in ctx.dem_kernel_times()
    dg = ctx.dem_get_diag()
    assert not dg[TSE].any() and not dg[QRAD].any()
    ctx.close()


def test_adjoint_and_bad_emissivity_are_refused():
    bed = _bed(45, n=300)
    ctx = _ctx(bed)
    with pytest.raises(binding.DemError) as e:
        ctx.dem_adjoint(2, 1)
    assert e.value.status == binding.DEM_EINVAL
    ctx.close()
    bad = _bed(46, n=300)
    bad.beds[0].emissivity = 1.5
    with pytest.raises(binding.DemError) as e:
        binding.Context(bad, precision="fp64", stream=torch.cuda.current_stream().cuda_stream)
    assert e.value.status == binding.DEM_EINVAL


@pytest.mark.parametrize("tuning", [dict(neighbour_lists=1, skin_permille=5, restore_every=1),
                                    dict(neighbour_lists=1, skin_permille=5, restore_every=64),
                                    dict(neighbour_lists=0)])
def test_radiation_with_restores_graphs_and_search_modes(tuning):
    # frequent list builds re-storing the state at every build (the kernel's sorted-order
    # path right after a re-store) or almost never, and the cell search without lists;
    # stepped through a captured CUDA graph
    bed = _bed(47, n=1200, cg=6.0)
    ctx, ref = _ctx(bed), oracle.Oracle(bed)
    ctx.dem_set_tuning(**tuning)
    ctx.dem_step_graph(4)
    ctx.dem_step_graph(4)
    ref.step(8)
    steps, builds, _ = ctx.dem_get_counters()
    assert steps == 8 and (builds >= 2 or tuning["neighbour_lists"] == 0)
    sg, so = ctx.dem_get_state(), ref.state()
    for row in range(binding.DEM_NSTATE):
        assert _rel(sg[row], so[row]) < 1e-9, binding.STATE_ROWS[row]
    dg, do = ctx.dem_get_diag(), ref.diag()
    assert _rel(dg[TSE], do[oracle.D_TSE]) < 1e-9 and _rel(dg[QRAD], do[oracle.D_QRAD]) < 1e-9
    ctx.close()
