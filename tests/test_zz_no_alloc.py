"""The allocation-free reduction-degree entry point, through the C ABI, on the GPU.

It is meant for callers that cannot call cudaMalloc (their device memory belongs to another
allocator, or cudaMalloc's implicit synchronisation is not acceptable in their loop) and
own their parcel arrays. Its result must equal the context entry point dem_reduction_degree
on the same masses, on two calls in a row (its scratch array keeps the previous call's
partial sums, which must not leak into the next result), and the FP64 CPU oracle's bed
reduction degree and removed-oxygen fraction on the same masses; at sizes that fill many
rows of its scratch array (and at its stated maximum) it must equal an FP64 sum of the
per-parcel reduction degrees. Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2311_03908_gb300 import binding, synth  # noqa: E402

MOLAR = np.array([159.69e-3, 231.533e-3, 71.844e-3, 55.845e-3])


def _call(masses, ore, out, n=None):
    L = binding.lib()
    st = torch.cuda.current_stream().cuda_stream
    return L.dem_reduction_degree_noalloc(*(C.c_void_p(m.data_ptr()) for m in masses),
                                          C.c_void_p(ore.data_ptr()),
                                          int(ore.numel() if n is None else n),
                                          C.c_void_p(out.data_ptr()), C.c_void_p(st) if st else None)


def _device_masses(state):
    return [torch.tensor(np.ascontiguousarray(state[10 + q]), dtype=torch.float64, device="cuda")
            for q in range(4)]


def test_noalloc_matches_context_entry_point_on_two_calls():
    torch.cuda.set_device(0)
    bed = synth.small_packed(seed=31, n=5000, v_scale=0.2, T0=1073.0)
    ctx = binding.Context(bed, precision="fp64", stream=torch.cuda.current_stream().cuda_stream)
    ore = torch.tensor(bed.ore, dtype=torch.int32, device="cuda")
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    results = []
    for k in range(2):
        ctx.dem_step(25)
        mean, oxy = ctx.dem_reduction_degree()
        masses = _device_masses(ctx.dem_get_state())
        assert _call(masses, ore, out) == binding.DEM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - mean[0]) <= 1e-12 * abs(mean[0])
        assert abs(got[1] - oxy[0]) <= 1e-12 * abs(oxy[0])
        results.append(got.copy())
    assert results[1][0] > results[0][0]   # the bed reduced further between the calls
    # a smaller input after a larger one: rows left over from the last call must not count
    half = bed.n // 2
    sub = [m[:half].contiguous() for m in masses]
    assert _call(sub, ore[:half].contiguous(), out) == binding.DEM_OK
    torch.cuda.synchronize()
    st = ctx.dem_get_state()
    M = np.array([159.69e-3, 231.533e-3, 71.844e-3, 55.845e-3])
    nn = st[10:14, :half] / M[:, None]
    nfe = 2 * nn[0] + 3 * nn[1] + nn[2] + nn[3]
    fh, fm, fw = (3 * nn[1] + nn[2] + nn[3]) / nfe, (nn[2] + nn[3]) / nfe, nn[3] / nfe
    o = bed.ore[:half]
    f = np.where(o == 0, fh / 9 + 2 * fm / 9 + 6 * fw / 9, fm / 4 + 3 * fw / 4)
    assert abs(out.cpu().numpy()[0] - f.mean()) <= 1e-12 * f.mean()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    ore = torch.zeros(4, dtype=torch.int32, device="cuda")
    masses = [torch.ones(4, dtype=torch.float64, device="cuda") for _ in range(4)]
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert _call(masses, ore, out, n=binding.DEM_NOALLOC_MAX_PARCELS + 1) == binding.DEM_EINVAL
    assert _call(masses, ore, out, n=0) == binding.DEM_EINVAL
    assert torch.all(out == 0)   # nothing was enqueued


def _random_masses(seed, n):
    """Seeded parcel masses of every composition between the pure oxides and iron."""
    u = synth.uniform(seed, 5 * n).reshape(5, n)
    w = -np.log1p(-u[:4])                     # exponential weights: compositions spread over the simplex
    w[:, u[4] < 0.1] *= np.array([[0.0], [1.0], [1.0], [1.0]])   # some parcels without Fe2O3
    m = 1e-7 * w / w.sum(0)
    ore = (synth.uniform(seed, n, 7) < 0.5).astype(np.int32)
    return m, ore


def _fov_numpy(m, ore):
    nn = m / MOLAR[:, None]
    nfe = 2 * nn[0] + 3 * nn[1] + nn[2] + nn[3]
    fh, fm, fw = (3 * nn[1] + nn[2] + nn[3]) / nfe, (nn[2] + nn[3]) / nfe, nn[3] / nfe
    return np.where(ore == 0, fh / 9 + 2 * fm / 9 + 6 * fw / 9, fm / 4 + 3 * fw / 4)


def test_noalloc_matches_the_oracle():
    bed = synth.small_packed(seed=33, n=4000)
    m, ore = _random_masses(5, bed.n)
    bed.m0 = m
    bed.ore = ore
    mo, oo, _ = oracle.Oracle(bed).reduction_degree()
    masses = [torch.tensor(np.ascontiguousarray(m[q]), dtype=torch.float64, device="cuda") for q in range(4)]
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        assert _call(masses, torch.tensor(ore, device="cuda"), out) == binding.DEM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - mo[0]) <= 1e-12 * abs(mo[0])
        assert abs(got[1] - oo[0]) <= 1e-12 * abs(oo[0])


@pytest.mark.parametrize("n", [256 * 2048 + 1, binding.DEM_NOALLOC_MAX_PARCELS])
def test_noalloc_many_rows_of_scratch(n):
    # more than 256 pass-1 blocks: the final pass loops over its rows more than once; at the
    # stated maximum every row of the scratch array is used
    m, ore = _random_masses(11, n)
    masses = [torch.tensor(np.ascontiguousarray(m[q]), dtype=torch.float64, device="cuda") for q in range(4)]
    ore_d = torch.tensor(ore, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    f = _fov_numpy(m, ore)
    expect = float(np.sum(f, dtype=np.float64)) / n
    for _ in range(2):
        assert _call(masses, ore_d, out) == binding.DEM_OK
        torch.cuda.synchronize()
        assert abs(out.cpu().numpy()[0] - expect) <= 1e-12 * expect
    del masses, ore_d
    torch.cuda.empty_cache()
