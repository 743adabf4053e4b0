"""Edge cases of the CUDA path against the FP64 oracle, on the GPU: ragged parcel counts
(one parcel, counts that are not multiples of the kernels' 4-, 32- and 64-parcel strides),
a bed without parcels in a multi-bed context, and the FP32 forms with the neighbour-list
configurations that exercise the re-store interval and frequent list builds."""
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


def _pairs(cnt, partner):
    return {(i, int(partner[i, k])) for i in range(len(cnt)) for k in range(cnt[i])}


@pytest.mark.parametrize("n", [1, 33, 65, 1001])
def test_ragged_counts_match_oracle(n):
    bed = synth.small_packed(seed=31, n=n, v_scale=0.3, wall_kind=synth.WALL_CONE)
    ctx = _ctx(bed)
    ctx.dem_set_tuning(skin_permille=5, restore_every=3)   # many list builds, few re-stores
    ref = oracle.Oracle(bed)
    for _ in range(3):
        ctx.dem_step(7)
        ref.step(7)
        sg, so = ctx.dem_get_state(), ref.state()
        for row in range(binding.DEM_NSTATE):
            assert _rel(sg[row], so[row]) < 1e-7, (n, binding.STATE_ROWS[row])
        cg, pg, _ = ctx.dem_get_contacts()
        co, po, _ = ref.contacts()
        assert _pairs(cg, pg) == _pairs(co, po)
    mg, _ = ctx.dem_reduction_degree()
    mo, _, _ = ref.reduction_degree()
    assert abs(mg[0] - mo[0]) < 1e-12
    ctx.close()


def test_bed_without_parcels_in_a_batch():
    parts = [synth.small_packed(seed=41, n=700, v_scale=0.2), synth.small_packed(seed=42, n=500, v_scale=0.2)]
    empty = synth.small_packed(seed=43, n=1)   # its bed configuration only
    beds = [parts[0].beds[0], empty.beds[0], parts[1].beds[0]]
    cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
    bedid = np.concatenate([np.full(parts[0].n, 0, np.int32), np.full(parts[1].n, 2, np.int32)])
    bed = synth.Bed(beds, cat("x"), cat("y"), cat("z"), cat("vx"), cat("vy"), cat("vz"), cat("d_real"),
                    cat("T"), np.concatenate([p.m0 for p in parts], axis=1), cat("ore"), bedid, "gap")
    ctx = _ctx(bed)
    ref = oracle.Oracle(bed)
    ctx.dem_step(12)
    ref.step(12)
    sg, so = ctx.dem_get_state(), ref.state()
    for row in range(binding.DEM_NSTATE):
        assert _rel(sg[row], so[row]) < 1e-7, binding.STATE_ROWS[row]
    mg, og = ctx.dem_reduction_degree()
    mo, oo, _ = ref.reduction_degree()
    for b in (0, 2):
        assert abs(mg[b] - mo[b]) < 1e-12 and abs(og[b] - oo[b]) < 1e-12
    ctx.close()


@pytest.mark.parametrize("prec", ["split", "split_kahan"])
def test_fp32_forms_with_frequent_builds_and_rare_restores(prec):
    bed = synth.small_packed(seed=12, n=3000, v_scale=0.3, T0=1073.0, wall_kind=synth.WALL_CONE)
    ctx = _ctx(bed, prec)
    ctx.dem_set_tuning(skin_permille=5, restore_every=8, bs_contacts=64, bs_key=64)
    ref = oracle.Oracle(bed)
    ctx.dem_step(20)
    ref.step(20)
    steps, builds, _ = ctx.dem_get_counters()
    assert builds > 5                                  # lists rebuilt, mostly without a re-store
    sg, so = ctx.dem_get_state(), ref.state()
    for row in range(3):
        assert _rel(sg[row], so[row]) < 1e-6
    assert _rel(sg[9], so[9]) < 1e-5
    cg, pg, _ = ctx.dem_get_contacts()
    co, po, _ = ref.contacts()
    # FP32 forces move positions by up to dx; a pair may then be in contact on one side and
    # not the other only if its gap on the oracle's positions is within 2 dx of zero
    a, b = _pairs(cg, pg), _pairs(co, po)
    dx = max(np.abs(sg[row] - so[row]).max() for row in range(3))
    r = 0.5 * bed.beds[0].cg_ratio * bed.d_real
    for i, j in a ^ b:
        gap = np.sqrt(sum((so[row][i] - so[row][j]) ** 2 for row in range(3))) - (r[i] + r[j])
        assert abs(gap) <= 2.0 * dx + 1e-12, (i, j, gap, dx)
    assert len(a & b) > 0.9 * len(b)
    mg, _ = ctx.dem_reduction_degree()
    mo, _, _ = ref.reduction_degree()
    assert abs(mg[0] - mo[0]) < 1e-3
    ctx.close()
