"""Parity of the CUDA path with the FP64 oracle at the benchmarked size, on the GPU.

The bed is the 2,000,000-parcel two-ore bed with the conical bottom and the perforated
distributor plate on the 64 x 64 x 384 gas grid (1,572,864 cells, 21 key bits): the radix
sort's third pass at the first binning, the incremental re-sort with thousands of moving
parcels, the grid-stride neighbour-list search over many waves of blocks, the reactor wall
at full resolution, and the launch configuration the autotuner picks on this bed (64-thread
blocks, 200 per mille skin, a re-store at every 8th list build). The FP64 form is held to
the oracle after 1 and after 20 steps (pair sets bit-exact; states and tangential
displacements 1e-7 of their vectors' lengths; cell sources and gas 1e-9; bed reduction
degree 1e-12), the split form
after 20 steps with its own tolerances. The same bed packed at touching pitch with random
velocities (the contact-dominated regime) is held to the oracle after 10 steps.
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

# the configuration the autotuner picks on this bed (bench.py prints it with every run)
BENCH_TUNING = dict(neighbour_lists=1, bs_key=64, bs_restore=64, bs_search=64, bs_contacts=64,
                    bs_gas_particle=64, bs_cells=64, skin_permille=200, restore_every=8)


def _rel(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


# rows of the state that are components of one vector: each is compared relative to the
# largest component of its vector (a component that is zero in exact arithmetic, such as the
# spin about the vertical of parcels resting on horizontal walls, carries only round-off)
_VECTOR_OF_ROW = {r: (r // 3) * 3 for r in range(9)}
_VECTOR_OF_ROW.update({r: 14 + ((r - 14) // 3) * 3 for r in range(14, 20)})


def _rel_state(g, r, row):
    if row not in _VECTOR_OF_ROW:
        return _rel(g[row], r[row])
    v0 = _VECTOR_OF_ROW[row]
    scale = max(np.abs(r[q]).max() for q in range(v0, v0 + 3))
    return np.abs(g[row] - r[row]).max() / (scale if scale > 0 else 1.0)


def _pair_keys(cnt, partner):
    """Every (parcel, partner) of the contact table as one sorted int64 key per slot."""
    mask = np.arange(partner.shape[1])[None, :] < cnt[:, None]
    i = np.nonzero(mask)[0].astype(np.int64)
    p = partner[mask].astype(np.int64)
    return np.sort(i * (1 << 32) + (p + (1 << 31))), mask


def _snap(obj, is_ref):
    st = obj.state() if is_ref else obj.dem_get_state()
    cnt, partner, xi = obj.contacts() if is_ref else obj.dem_get_contacts()
    keys, mask = _pair_keys(cnt, partner)
    src = obj.deposits() if is_ref else obj.dem_get_sources()
    gas = obj.gas() if is_ref else obj.dem_get_gas()
    fov = obj.reduction_degree()[0] if is_ref else obj.dem_reduction_degree()[0]
    return dict(state=st, keys=keys, xi=xi[mask], cnt=cnt, partner=partner, src=src, gas=gas,
                fov=np.array(fov))


@pytest.fixture(scope="module")
def bench_bed():
    bed = synth.config_ibm_2m()
    ref = oracle.Oracle(bed)
    ref.step(1)
    r1 = _snap(ref, True)
    ref.step(19)
    r20 = _snap(ref, True)
    del ref
    return bed, r1, r20


def _check_fp64(g, r, what):
    assert np.array_equal(g["keys"], r["keys"]), what
    if r["xi"].size:
        # tangential displacements: each slot's vector to 1e-7 of its length (a component that
        # is zero in exact arithmetic carries only round-off, as for the state's vectors)
        norm = np.linalg.norm(r["xi"], axis=1)[:, None]
        err = np.abs(g["xi"] - r["xi"]) / np.maximum(norm, 1e-30)
        assert float(err.max()) < 1e-7, (what, float(err.max()))
    for row in range(binding.DEM_NSTATE):
        assert _rel_state(g["state"], r["state"], row) < 1e-7, (what, binding.STATE_ROWS[row])
    for col in range(binding.DEM_NDEP):
        assert _rel(g["src"][:, col], r["src"][:, col]) < 1e-9, (what, binding.SOURCE_ROWS[col])
    for col in range(binding.DEM_NGAS):
        assert _rel(g["gas"][:, col], r["gas"][:, col]) < 1e-9, (what, col)
    assert np.all(np.abs(g["fov"] - r["fov"]) < 1e-12), what


def test_ibm_2m_fp64_form_after_1_and_20_steps(bench_bed):
    bed, r1, r20 = bench_bed
    ctx = binding.Context(bed, precision="fp64", stream=torch.cuda.current_stream().cuda_stream)
    ctx.dem_set_tuning(**BENCH_TUNING)
    ctx.dem_step(1)
    _check_fp64(_snap(ctx, False), r1, "step 1")
    ctx.dem_step_graph(19)            # the bench's way of stepping: replayed CUDA graphs
    _check_fp64(_snap(ctx, False), r20, "step 20")
    ctx.close()


def _differing_pairs_are_marginal(bed, g, r, dx):
    """FP32 contact geometry moves positions by up to dx; a pair may then be in contact on
    one side only if its gap on the oracle's positions lies within 2 dx of zero."""
    a, b = set(g["keys"].tolist()), set(r["keys"].tolist())
    so = r["state"]
    rad = 0.5 * bed.beds[0].cg_ratio * bed.d_real
    for k in a ^ b:
        i, j = k >> 32, (k & 0xFFFFFFFF) - (1 << 31)
        if j >= 0:
            gap = np.sqrt(sum((so[q][i] - so[q][j]) ** 2 for q in range(3))) - (rad[i] + rad[j])
        else:
            dist, _ = oracle.wall_distance(bed.beds[0], so[0][i], so[1][i], so[2][i])
            gap = dist[-1 - j] - rad[i]
        assert abs(gap) <= 2.0 * dx + 1e-12, (i, j, gap, dx)
    return len(a & b), len(b)


def test_ibm_2m_split_form_after_20_steps(bench_bed):
    bed, _, r20 = bench_bed
    ctx = binding.Context(bed, precision="split", stream=torch.cuda.current_stream().cuda_stream)
    ctx.dem_set_tuning(**BENCH_TUNING)
    ctx.dem_step_graph(10)
    ctx.dem_step_graph(10)
    g = _snap(ctx, False)
    sg, so = g["state"], r20["state"]
    for row in range(3):
        assert _rel(sg[row], so[row]) < 1e-6
    assert _rel(sg[9], so[9]) < 1e-5
    for q in range(4):
        dg_, do_ = sg[10 + q] - bed.m0[q], so[10 + q] - bed.m0[q]
        if np.abs(do_).max() > 0:
            assert _rel(dg_, do_) < 1e-4, binding.STATE_ROWS[10 + q]
    dx = max(np.abs(sg[row] - so[row]).max() for row in range(3))
    common, total = _differing_pairs_are_marginal(bed, g, r20, dx)
    assert common >= 0.99 * total
    # cell sources: compensated FP32 sums of FP32 per-parcel terms
    for col in (0, 1, 2, 7, 8, 9):
        assert _rel(g["src"][:, col], r20["src"][:, col]) < 1e-4, binding.SOURCE_ROWS[col]
    assert np.all(np.abs(g["fov"] - r20["fov"]) < 1e-3)
    assert np.all(np.abs(g["fov"] - r20["fov"]) < 1e-6)
    ctx.close()


def test_ibm_2m_dense_bed_fp64_and_split_after_10_steps():
    # the lattice jammed: neighbours overlap by up to 0.5 % of the larger diameter from the first step
    bed = synth.config_ibm_2m_dense(v_scale=0.05, U_in=0.3, compress=0.005, sigma=0.25)
    ref = oracle.Oracle(bed)
    ref.step(10)
    r = _snap(ref, True)
    del ref
    zbar = r["cnt"].mean()
    assert (r["cnt"] > 0).mean() > 0.2 and zbar > 0.3       # contacts everywhere in the bed
    ctx = binding.Context(bed, precision="fp64", stream=torch.cuda.current_stream().cuda_stream)
    ctx.dem_set_tuning(**BENCH_TUNING)
    ctx.dem_step_graph(10)
    _check_fp64(_snap(ctx, False), r, "dense, step 10")
    ctx.close()
    ctx = binding.Context(bed, precision="split", stream=torch.cuda.current_stream().cuda_stream)
    ctx.dem_set_tuning(**BENCH_TUNING)
    ctx.dem_step_graph(10)
    g = _snap(ctx, False)
    dx = max(np.abs(g["state"][q] - r["state"][q]).max() for q in range(3))
    assert dx < 1e-6 * 0.6
    common, total = _differing_pairs_are_marginal(bed, g, r, dx)
    assert common >= 0.99 * total
    assert np.all(np.abs(g["fov"] - r["fov"]) < 1e-6)
    ctx.close()


def _cells(bed, st):
    c = bed.beds[0]
    ix = np.clip(np.floor((st[0] + 0.5 * c.D) / (c.D / c.nx)), 0, c.nx - 1)
    iy = np.clip(np.floor((st[1] + 0.5 * c.D) / (c.D / c.ny)), 0, c.ny - 1)
    iz = np.clip(np.floor(st[2] / (c.H / c.nz)), 0, c.nz - 1)
    return (iz * c.ny + iy) * c.nx + ix


def test_many_movers_on_the_full_grid():
    # 250,000 parcels on the 64 x 64 x 384 grid (21 key bits: three radix passes at the first
    # binning) moving at up to 3 m/s: several thousand change cell every step, more than the
    # re-sort ranks in shared memory (4096), so its global-memory sort runs
    bed = synth.config_ibm_2m(n=250_000, v_scale=3.0)
    ref = oracle.Oracle(bed)
    ctx = binding.Context(bed, precision="fp64", stream=torch.cuda.current_stream().cuda_stream)
    ctx.dem_set_tuning(**BENCH_TUNING)
    most = 0
    prev = _cells(bed, ref.state())
    for k in range(4):
        ctx.dem_step(1)
        ref.step(1)
        so = ref.state()
        cur = _cells(bed, so)
        most = max(most, int((cur != prev).sum()))
        prev = cur
        sg = ctx.dem_get_state()
        for row in range(binding.DEM_NSTATE):
            assert _rel_state(sg, so, row) < 1e-7, (k, binding.STATE_ROWS[row])
        cg, pg, _ = ctx.dem_get_contacts()
        co, po, _ = ref.contacts()
        assert np.array_equal(_pair_keys(cg, pg)[0], _pair_keys(co, po)[0]), k
    assert most > 4096
    ctx.close()
