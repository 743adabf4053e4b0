"""Contact heat conduction (eqs (3-14), (3-15), (3-15-1), (3-15-2) with the scaling of
eqs (3-46), (3-48), (3-48-1), (3-48-2)) on the GPU, through the C ABI, against the FP64
oracle: the per-parcel conduction heat and the temperatures in dense beds with walls, in
all three precision forms; heat conservation of pair conduction in a bed without walls."""
import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth
from tests.helpers import ISOLATED, bed_from_arrays

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

from paper_2311_03908_gb300 import binding  # noqa: E402


def _ctx(bed, prec="fp64"):
    c = binding.Context(bed, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    c.dem_set_diagnostics(True)
    return c


def _rel(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def _hot_bed(seed, wall, n=3000):
    bed = synth.small_packed(seed=seed, n=n, v_scale=1.0, T0=1073.0, wall_kind=wall, flags=synth.CONDUCTION)
    bed.T = bed.T + 80.0 * (synth.uniform(seed, bed.n, 77) - 0.5)     # spread of 80 K between parcels
    return bed


@pytest.mark.parametrize("wall", [synth.WALL_FLAT, synth.WALL_CONE])
def test_conduction_fp64_against_oracle(wall):
    bed = _hot_bed(21, wall)
    ctx = _ctx(bed)
    ref = oracle.Oracle(bed)
    for _ in range(3):
        ctx.dem_step(10)
        ref.step(10)
        dg, do = ctx.dem_get_diag(), ref.diag()
        q_g, q_o = dg[binding.DIAG_ROWS.index("Qcond")], do[oracle.D_QCOND]
        assert np.count_nonzero(q_o) > 100
        assert _rel(q_g, q_o) < 1e-9
        sg, so = ctx.dem_get_state(), ref.state()
        assert _rel(sg[9], so[9]) < 1e-12      # temperatures
        for row in range(binding.DEM_NSTATE):
            assert _rel(sg[row], so[row]) < 1e-7, binding.STATE_ROWS[row]
    # wall contacts carry conduction too
    cnt, partner, _ = ctx.dem_get_contacts()
    walls = (partner < 0) & (np.arange(partner.shape[1])[None, :] < cnt[:, None])
    assert walls.any()
    ctx.close()


@pytest.mark.parametrize("prec", ["split", "split_kahan"])
def test_conduction_fp32_forms_against_oracle(prec):
    bed = _hot_bed(22, synth.WALL_CONE)
    ctx = _ctx(bed, prec)
    ref = oracle.Oracle(bed)
    ctx.dem_step(10)
    ref.step(10)
    dg, do = ctx.dem_get_diag(), ref.diag()
    q_g, q_o = dg[binding.DIAG_ROWS.index("Qcond")], do[oracle.D_QCOND]
    # the contacts' geometry in FP32 cell-local coordinates: conduction of the same contacts
    # to FP32 accuracy, a few marginal contacts (overlap ~ the coordinates' resolution) aside
    both = (q_g != 0) & (q_o != 0)
    assert both.sum() > 0.95 * np.count_nonzero(q_o)
    assert np.median(np.abs(q_g[both] - q_o[both]) / np.abs(q_o[both])) < 1e-4
    sg, so = ctx.dem_get_state(), ref.state()
    assert _rel(sg[9] - bed.T, so[9] - bed.T) < 1e-3     # the temperature change of the 10 steps
    ctx.close()


def test_pair_conduction_conserves_heat_on_the_gpu():
    cfg = synth.BedConfig(D=0.04, H=0.04, nx=8, ny=8, nz=8, dt=2e-6, cg_ratio=4.0, T_in=1000.0,
                          flags=ISOLATED | synth.CONDUCTION)
    d = 100e-6
    p = cfg.cg_ratio * d * 0.999
    g = (np.arange(8) - 3.5) * p
    X, Y, Z = np.meshgrid(g, g, g + 0.02, indexing="ij")
    n = X.size
    u = synth.uniform(6, 4 * n).reshape(4, n)
    bed = bed_from_arrays(cfg, X.ravel(), Y.ravel(), Z.ravel(), v=0.02 * (2 * u[:3] - 1), d_real=d,
                          T=950.0 + 100.0 * u[3], comp=synth.COMP_MIXED)
    for prec, tol in (("fp64", 1e-12), ("split", 1e-5)):
        ctx = _ctx(bed, prec)
        ctx.dem_step(7)
        q = ctx.dem_get_diag()[binding.DIAG_ROWS.index("Qcond")]
        assert np.count_nonzero(q) > 0.9 * n
        assert abs(q.sum()) < tol * np.abs(q).sum(), prec
        ctx.close()


def test_adjoint_refuses_a_conducting_bed():
    bed = _hot_bed(23, synth.WALL_FLAT, n=300)
    ctx = _ctx(bed)
    with pytest.raises(binding.DemError) as e:
        ctx.dem_adjoint(10, 5)
    assert e.value.status == binding.DEM_EINVAL
    ctx.close()
