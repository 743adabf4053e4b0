"""Failure detection on the GPU, made on the host: the sticky device error word reports a
non-finite state (a gas field with NaN temperatures passed through dem_set_gas) and a parcel
that left its bed's gas grid (one fast parcel crossing the side wall within a step). No
kernel faults: NaN arithmetic and a clamped cell index are ordinary operations, and the
kernels only set bits that the host reads after the step."""
import numpy as np
import pytest

from paper_2311_03908_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

from paper_2311_03908_gb300 import binding  # noqa: E402
from tests.helpers import ISOLATED, bed_from_arrays  # noqa: E402


def _ctx(bed, prec="fp64"):
    return binding.Context(bed, precision=prec, stream=torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_nan_gas_temperature_is_reported_and_sticky(prec):
    bed = synth.small_packed(seed=50, n=300)
    ctx = _ctx(bed, prec)
    ctx.dem_step(2)
    ctx.dem_sync()                                     # healthy so far
    nc = ctx.ncells
    Y = np.tile(np.array([[0.9, 0.05, 0.05]]), (nc, 1))
    T = np.full(nc, np.nan)
    ctx.dem_set_gas(Y, T)
    ctx.dem_step(1)
    with pytest.raises(binding.DemError) as e:
        ctx.dem_sync()
    assert e.value.status == binding.DEM_ENONFINITE
    with pytest.raises(binding.DemError) as e:         # sticky: the next call reports it too
        ctx.dem_step(1)
    assert e.value.status == binding.DEM_ENONFINITE
    ctx.close()


def test_parcel_leaving_the_grid_is_reported():
    cfg = synth.BedConfig(D=0.02, H=0.04, nx=4, ny=4, nz=8, dt=1e-5, flags=ISOLATED)
    # 1 mm from the side wall, moving outwards at 200 m/s: 2 mm per step, out of the grid
    # (which ends at the cylinder's radius) within the first step
    b = bed_from_arrays(cfg, [0.009, -0.005], [0.0, 0.0], [0.02, 0.02], v=[[200.0, 0.0], [0.0, 0.0], [0.0, 0.0]])
    ctx = _ctx(b)
    ctx.dem_step(1)
    with pytest.raises(binding.DemError) as e:
        ctx.dem_sync()
    assert e.value.status == binding.DEM_EDOMAIN
    ctx.close()
