"""Launch configurations of the step -- neighbour lists or the cell-list search every step,
block sizes, neighbour-list skin, re-store interval -- and the autotuner. Each configuration
computes the same step, so each is held to the FP64 oracle: pair sets bit-exact, states to
relative 1e-7 over several list rebuilds."""
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


@pytest.mark.parametrize("lists,skin,bs,every", [(1, 100, 128, 1), (1, 5, 64, 3), (1, 600, 256, 1), (0, 100, 256, 1),
                                               (1, 50, 128, 64)])
def test_contact_configurations_match_oracle(lists, skin, bs, every):
    bed = synth.small_packed(seed=21, n=3000, v_scale=0.3, wall_kind=synth.WALL_CONE)
    ctx = _ctx(bed)
    ctx.dem_set_tuning(neighbour_lists=lists, skin_permille=skin, bs_key=bs, bs_restore=bs, bs_search=bs,
                       bs_contacts=bs, bs_gas_particle=bs, bs_cells=bs, restore_every=every)
    ref = oracle.Oracle(bed)
    for _ in range(4):
        ctx.dem_step(15)
        ref.step(15)
        sg, so = ctx.dem_get_state(), ref.state()
        for row in range(binding.DEM_NSTATE):
            assert _rel(sg[row], so[row]) < 1e-7, binding.STATE_ROWS[row]
        cg, pg, _ = ctx.dem_get_contacts()
        co, po, _ = ref.contacts()
        assert _pairs(cg, pg) == _pairs(co, po)
    assert sum(cg) > 100
    steps, builds, entries = ctx.dem_get_counters()
    assert steps == 60
    if lists:
        assert builds >= 1 and entries >= sum(cg)
        if skin == 5:
            assert builds > 5          # a thin skin forces frequent rebuilds
    else:
        assert builds == 0             # no lists: the cell list is searched every step
    ctx.close()


def test_neighbour_lists_are_reused_between_builds():
    bed = synth.small_packed(seed=22, n=2000, v_scale=0.01)
    ctx = _ctx(bed, prec="split")
    ctx.dem_set_tuning(skin_permille=500)
    ctx.dem_step(40)
    steps, builds, _ = ctx.dem_get_counters()
    assert steps == 40 and 1 <= builds <= 2
    ctx.close()


def test_set_tuning_rejects_invalid_values():
    bed = synth.small_packed(seed=1, n=300)
    ctx = _ctx(bed)
    t0 = ctx.dem_get_tuning()
    assert set(t0) == set(binding.TUNING_KEYS)
    # the gas-particle kernel launches at most 256 threads per block (launch bounds)
    for bad in (dict(neighbour_lists=2), dict(bs_key=48), dict(bs_cells=2048), dict(bs_search=0),
                dict(skin_permille=0), dict(skin_permille=1001), dict(bs_gas_particle=1024),
                dict(restore_every=0), dict(restore_every=65)):
        with pytest.raises(binding.DemError) as e:
            ctx.dem_set_tuning(**bad)
        assert e.value.status == binding.DEM_EINVAL
        assert ctx.dem_get_tuning() == t0
    ctx.close()


def test_autotune_restores_the_state_and_keeps_parity():
    bed = synth.small_packed(seed=23, n=2500, v_scale=0.3)
    ctx = _ctx(bed)
    ref = oracle.Oracle(bed)
    ctx.dem_step(5)
    ref.step(5)
    s0 = ctx.dem_get_state()
    c0 = ctx.dem_get_counters()
    t = ctx.dem_autotune(8)
    assert set(t) == set(binding.TUNING_KEYS) and t["neighbour_lists"] in (0, 1)
    assert np.array_equal(ctx.dem_get_state(), s0)
    assert ctx.dem_get_counters() == c0
    ctx.dem_step(10)
    ref.step(10)
    sg, so = ctx.dem_get_state(), ref.state()
    for row in range(binding.DEM_NSTATE):
        assert _rel(sg[row], so[row]) < 1e-7, binding.STATE_ROWS[row]
    cg, pg, _ = ctx.dem_get_contacts()
    co, po, _ = ref.contacts()
    assert _pairs(cg, pg) == _pairs(co, po)
    ctx.close()
