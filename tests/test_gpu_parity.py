"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, on the GPU.

Tolerances: neighbour and pair sets bit-exact (one step from the same inputs); single-step
state and forces to relative 1e-5 (FP64 form, in practice ~1e-12); multi-step states in
the FP64 form to relative 1e-7 while trajectories are still close; bed-averaged reduction
degree to 1e-3 absolute for both forms.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

from paper_2311_03908_gb300 import binding  # noqa: E402


def _ctx(bed, prec="fp64", diag=False):
    c = binding.Context(bed, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    if diag:
        c.dem_set_diagnostics(True)
    return c


def _rel(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def _lattice_bed(n_side=10, v_scale=0.1, seed=3):
    cfg = synth.BedConfig(D=0.012, H=0.012, nx=6, ny=6, nz=6, dt=1e-5, cg_ratio=4.0, T_in=1023.0,
                          Y_in=(0.9, 0.05, 0.05))
    d = 100e-6
    p = cfg.cg_ratio * d
    g = (np.arange(n_side) - (n_side - 1) / 2) * p
    X, Y, Z = np.meshgrid(g, g, g + 0.006, indexing="ij")
    x, y, z = X.ravel(), Y.ravel(), Z.ravel()
    n = x.size
    u = synth.uniform(seed, 3 * n).reshape(3, n)
    v = v_scale * (2 * u - 1)
    dc = cfg.cg_ratio * d
    m = 5000.0 * math.pi / 6 * dc ** 3
    m0 = np.outer(np.array(synth.COMP_MIXED), np.full(n, m))
    return synth.Bed([cfg], x, y, z, v[0], v[1], v[2], np.full(n, d), np.full(n, 1000.0), m0,
                     np.zeros(n, np.int32), np.zeros(n, np.int32), "lattice")


def _pairs(cnt, partner):
    out = set()
    for i in range(len(cnt)):
        for k in range(cnt[i]):
            out.add((i, int(partner[i, k])))
    return out


def test_touching_lattice_pair_sets_bit_exact_after_one_step():
    bed = _lattice_bed()
    ctx = _ctx(bed, diag=True)
    ref = oracle.Oracle(bed)
    ctx.dem_step(1)
    ref.step(1)
    cg, pg, xg = ctx.dem_get_contacts()
    co, po, xo = ref.contacts()
    pairs_g, pairs_o = _pairs(cg, pg), _pairs(co, po)
    assert len(pairs_o) > 500            # about half the lattice bonds closed
    assert pairs_g == pairs_o
    # brute force on the oracle's new positions agrees too
    st = ref.state()
    r = 0.5 * 4.0 * bed.d_real
    bf = oracle.pairs_bruteforce(st[0], st[1], st[2], r)
    assert {(int(a), int(b)) for a, b in bf} == {(a, b) for a, b in pairs_o if b >= 0 and a < b}
    # tangential displacements of every slot
    for i in range(bed.n):
        assert np.allclose(xg[i, :cg[i]], xo[i, :co[i]], rtol=1e-9, atol=1e-18)
    # state and forces to 1e-5 relative (FP64 form)
    sg, so = ctx.dem_get_state(), ref.state()
    for row in range(binding.DEM_NSTATE):
        assert _rel(sg[row], so[row]) < 1e-5, binding.STATE_ROWS[row]
    dg, do = ctx.dem_get_diag(), ref.diag()
    for row in [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15]:
        assert _rel(dg[row], do[row]) < 1e-5, binding.DIAG_ROWS[row]
    ctx.close()


@pytest.mark.parametrize("wall", [synth.WALL_FLAT, synth.WALL_CONE])
def test_packed_bed_fp64_multistep(wall):
    bed = synth.small_packed(seed=9, n=3000, v_scale=0.3, wall_kind=wall)
    ctx = _ctx(bed, diag=True)
    ref = oracle.Oracle(bed)
    for _ in range(3):
        ctx.dem_step(10)
        ref.step(10)
        sg, so = ctx.dem_get_state(), ref.state()
        for row in range(binding.DEM_NSTATE):
            assert _rel(sg[row], so[row]) < 1e-7, binding.STATE_ROWS[row]
    cg, pg, _ = ctx.dem_get_contacts()
    co, po, _ = ref.contacts()
    assert _pairs(cg, pg) == _pairs(co, po)
    assert sum(cg) > 100
    gg, go = ctx.dem_get_gas(), ref.gas()
    for col in range(binding.DEM_NGAS):
        assert _rel(gg[:, col], go[:, col]) < 1e-9
    dg, do = ctx.dem_get_diag(), ref.diag()
    for row in range(binding.DEM_NDIAG):
        assert _rel(dg[row], do[row]) < 1e-6, binding.DIAG_ROWS[row]
    sgs, sos = ctx.dem_get_sources(), ref.deposits()
    for col in range(binding.DEM_NDEP):
        assert _rel(sgs[:, col], sos[:, col]) < 1e-9, binding.SOURCE_ROWS[col]
    # the occupied cells' rows: exactly the dense rows of the cells with parcels, in cell order
    cells, rows = ctx.dem_get_sources_occupied()
    occ = np.flatnonzero(sgs[:, binding.SOURCE_ROWS.index("count")] > 0)
    assert np.array_equal(cells, occ) and np.array_equal(rows, sgs[occ])
    mg, _ = ctx.dem_reduction_degree()
    mo, _, _ = ref.reduction_degree()
    assert abs(mg[0] - mo[0]) < 1e-12
    ctx.close()


@pytest.mark.parametrize("prec", ["split", "split_kahan"])
def test_split_form_against_oracle(prec):
    bed = synth.small_packed(seed=10, n=3000, v_scale=0.3, T0=1073.0)
    ctx = _ctx(bed, prec=prec, diag=True)
    ref = oracle.Oracle(bed)
    ctx.dem_step(20)
    ref.step(20)
    sg, so = ctx.dem_get_state(), ref.state()
    # positions stay FP64; FP32 forces perturb them only slightly over 20 steps
    for row in range(3):
        assert _rel(sg[row], so[row]) < 1e-6
    assert _rel(sg[9], so[9]) < 1e-5          # temperature
    # layer masses: FP32 rates carry ~1e-6 relative error, so compare what changed
    m0 = np.vstack([bed.m0[q] for q in range(4)])
    for q in range(4):
        dg_, do_ = sg[10 + q] - m0[q], so[10 + q] - m0[q]
        if np.abs(do_).max() > 0:
            assert _rel(dg_, do_) < 1e-4, binding.STATE_ROWS[10 + q]
    mg, _ = ctx.dem_reduction_degree()
    mo, _, _ = ref.reduction_degree()
    assert abs(mg[0] - mo[0]) < 1e-3
    dg, do = ctx.dem_get_diag(), ref.diag()
    for row in (13, 14, 15, 20, 21, 22, 23, 27, 28):   # rates, film, interface, Sh, Nu
        assert _rel(dg[row], do[row]) < 1e-4, binding.DIAG_ROWS[row]
    ctx.close()


def test_plain_2k_config_200_steps():
    bed = synth.config_plain_2k()
    ctx = _ctx(bed)
    ref = oracle.Oracle(bed)
    ctx.dem_step(200)
    ref.step(200)
    sg, so = ctx.dem_get_state(), ref.state()
    for row in range(14):
        assert _rel(sg[row], so[row]) < 1e-9, binding.STATE_ROWS[row]
    mg, _ = ctx.dem_reduction_degree()
    mo, _, _ = ref.reduction_degree()
    assert abs(mg[0] - mo[0]) < 1e-3
    assert abs(mg[0] - mo[0]) < 1e-12
    ctx.close()


def test_multibed_uneven():
    beds = []
    parts = []
    for b, T in enumerate([800.0, 950.0, 1073.0]):
        p = synth.small_packed(seed=20 + b, n=500 + 400 * b, v_scale=0.2, T0=T)
        parts.append(p)
        beds.append(p.beds[0])
    cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
    bedid = np.concatenate([np.full(p.n, i, np.int32) for i, p in enumerate(parts)])
    bed = synth.Bed(beds, cat("x"), cat("y"), cat("z"), cat("vx"), cat("vy"), cat("vz"), cat("d_real"),
                    cat("T"), np.concatenate([p.m0 for p in parts], axis=1), cat("ore"), bedid, "multi")
    ctx = _ctx(bed)
    ref = oracle.Oracle(bed)
    ctx.dem_step(15)
    ref.step(15)
    sg, so = ctx.dem_get_state(), ref.state()
    for row in range(binding.DEM_NSTATE):
        assert _rel(sg[row], so[row]) < 1e-7, binding.STATE_ROWS[row]
    mg, og = ctx.dem_reduction_degree()
    mo, oo, _ = ref.reduction_degree()
    assert np.allclose(mg, mo, rtol=0, atol=1e-12) and np.allclose(og, oo, rtol=0, atol=1e-12)
    ctx.close()


def test_graph_replay_matches_plain_steps():
    bed = synth.small_packed(seed=12, n=2000, v_scale=0.3)
    a = _ctx(bed)
    b = _ctx(bed)
    a.dem_step(8)
    b.dem_step_graph(4)
    b.dem_step_graph(4)
    assert np.array_equal(a.dem_get_state(), b.dem_get_state())
    a.dem_step(3)
    b.dem_step_graph(3)   # odd count: a second graph for the other buffer parity
    assert np.array_equal(a.dem_get_state(), b.dem_get_state())
    a.close()
    b.close()


def test_capacity_overflow_is_a_sticky_error():
    # one big parcel with 40 small parcels pressed onto its surface: more contacts than slots
    cfg = synth.BedConfig(D=0.02, H=0.02, nx=4, ny=4, nz=4, dt=1e-6, cg_ratio=1.0,
                          flags=synth.NO_GRAVITY | synth.NO_DRAG | synth.NO_KINETICS | synth.NO_HEAT)
    R, r = 1.5e-3, 0.2e-3
    k = np.arange(40)
    phi = np.arccos(1 - 2 * (k + 0.5) / 40)
    th = math.pi * (1 + 5 ** 0.5) * k
    dd = R + r - 1e-6
    x = np.concatenate([[0.0], dd * np.sin(phi) * np.cos(th)])
    y = np.concatenate([[0.0], dd * np.sin(phi) * np.sin(th)])
    z = np.concatenate([[0.01], 0.01 + dd * np.cos(phi)])
    d = np.concatenate([[2 * R], np.full(40, 2 * r)])
    n = x.size
    m = 5000 * math.pi / 6 * d ** 3
    bed = synth.Bed([cfg], x, y, z, np.zeros(n), np.zeros(n), np.zeros(n), d, np.full(n, 900.0),
                    np.vstack([m, 0 * m, 0 * m, 0 * m]), np.zeros(n, np.int32), np.zeros(n, np.int32))
    ctx = _ctx(bed)
    ctx.dem_step(1)
    with pytest.raises(binding.DemError) as e:
        ctx.dem_sync()
    assert e.value.status == binding.DEM_ECAPACITY
    with pytest.raises(binding.DemError):
        ctx.dem_step(1)
    ctx.close()


def test_invalid_inputs_rejected():
    bed = synth.small_packed(seed=1, n=200)
    bad = bed.subset(np.arange(bed.n))
    bad.x[3] = np.nan
    with pytest.raises(binding.DemError) as e:
        _ctx(bad)
    assert e.value.status == binding.DEM_EINVAL
    bad = bed.subset(np.arange(bed.n))
    bad.x[0] = 1.0                  # outside the cylinder
    with pytest.raises(binding.DemError):
        _ctx(bad)
    bad = bed.subset(np.arange(bed.n))
    bad.beds = [synth.BedConfig(**{**bed.beds[0].as_dict(), "coupling_interval": 0})]
    with pytest.raises(binding.DemError):
        _ctx(bad)
    bad = bed.subset(np.arange(bed.n))
    bad.beds = [synth.BedConfig(**{**bed.beds[0].as_dict(), "dt": 1e-3})]  # omega_0 dt >= 2
    with pytest.raises(binding.DemError):
        _ctx(bad)


@pytest.mark.parametrize("prec", ["fp64", "split_kahan"])
def test_coupling_interval_parity(prec):
    # the gas is advanced every 4th step (Sec. 4); calls that end on, just after and between
    # coupling steps, the state and the gas after each; the sources after a coupling step
    bed = synth.small_packed(seed=13, n=1500, v_scale=0.2, T0=1073.0)
    bed.beds[0].coupling_interval = 4
    ctx = _ctx(bed, prec)
    ref = oracle.Oracle(bed)
    for n in (4, 1, 2, 5, 1, 3):
        ctx.dem_step(n)
        ref.step(n)
        sg, so = ctx.dem_get_state(), ref.state()
        gg, go = ctx.dem_get_gas(), ref.gas()
        if prec == "fp64":
            for row in range(binding.DEM_NSTATE):
                assert _rel(sg[row], so[row]) < 1e-7, binding.STATE_ROWS[row]
            for col in range(binding.DEM_NGAS):
                assert _rel(gg[:, col], go[:, col]) < 1e-9
        else:
            for row in range(3):
                assert _rel(sg[row], so[row]) < 1e-6
            assert _rel(sg[9], so[9]) < 1e-5
            assert _rel(gg[:, 0], go[:, 0]) < 1e-6 and _rel(gg[:, 4], go[:, 4]) < 1e-6
            assert np.abs(gg[:, 1:4] - go[:, 1:4]).max() < 1e-6
    # 16 steps: the last one is a coupling step, whose sources the oracle keeps
    sgs, sos = ctx.dem_get_sources(), ref.deposits()
    for col in range(binding.DEM_NDEP):
        assert _rel(sgs[:, col], sos[:, col]) < (1e-9 if prec == "fp64" else 1e-4), binding.SOURCE_ROWS[col]
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_set_gas_between_coupling_steps(prec):
    """A coupling input that arrives between coupling steps is the gas state until the next
    coupling step advances it, for eager steps and replayed graphs alike (the other gas
    buffer is brought up to date once, then left alone)."""
    bed = synth.small_packed(seed=17, n=1500, v_scale=0.2)
    bed.beds[0].coupling_interval = 4
    a, b = _ctx(bed, prec), _ctx(bed, prec)
    a.dem_step(5)
    b.dem_step_graph(5)
    g = a.dem_get_gas()
    Y = np.ascontiguousarray(g[:, 1:4])
    Y[:, 0] *= 0.8
    Y[:, 1] = 1.0 - Y[:, 0] - Y[:, 2]
    T = np.ascontiguousarray(g[:, 4]) + 20.0
    for c in (a, b):
        c.dem_set_gas(Y, T)
    g0 = a.dem_get_gas()
    assert np.allclose(g0[:, 4], T, rtol=1e-7) and np.array_equal(g0[:, 0], g[:, 0])
    for k in range(2):                     # the 6th and 7th steps advance no gas
        a.dem_step(1)
        b.dem_step_graph(1)
        assert np.array_equal(a.dem_get_gas(), g0) and np.array_equal(b.dem_get_gas(), g0), k
    a.dem_step(1)                          # the 8th step is a coupling step
    b.dem_step_graph(1)
    g1 = a.dem_get_gas()
    assert not np.array_equal(g1[:, 4], g0[:, 4])
    assert np.array_equal(g1, b.dem_get_gas()) and np.array_equal(a.dem_get_state(), b.dem_get_state())
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_set_gas_input_paths_agree(prec):
    """The coupling input through its three paths -- pageable host arrays (staged by a copy),
    page-locked host memory (read by the kernel itself) and device tensors -- gives the same
    state bit for bit; handing back the current field changes nothing."""
    bed = synth.small_packed(seed=5, n=2000, v_scale=0.2)
    ctxs = [_ctx(bed, prec) for _ in range(7)]
    for c in ctxs:
        c.dem_step(5)
    g = ctxs[0].dem_get_gas()
    Y0, T0 = np.ascontiguousarray(g[:, 1:4]), np.ascontiguousarray(g[:, 4])
    Y = Y0.copy()
    Y[:, 0] *= 0.9
    Y[:, 1] = 1.0 - Y[:, 0] - Y[:, 2]
    T = T0 + 15.0
    ctxs[1].dem_set_gas(Y, T)
    ctxs[2].dem_set_gas(torch.from_numpy(Y).pin_memory(), torch.from_numpy(T).pin_memory())
    ctxs[3].dem_set_gas(torch.from_numpy(Y).cuda(), torch.from_numpy(T).cuda())
    ctxs[4].dem_set_gas(Y0, T0)
    # the input read back before any step, and taken by a replayed step graph (whose first
    # gas-reading kernel waits for the input's own stream)
    ctxs[5].dem_set_gas(torch.from_numpy(Y).pin_memory(), torch.from_numpy(T).pin_memory())
    g5 = ctxs[5].dem_get_gas()
    assert np.allclose(g5[:, 1:4], Y, rtol=0, atol=1e-7) and np.allclose(g5[:, 4], T, rtol=1e-7)
    ctxs[6].dem_step_graph(2)
    ctxs[6].dem_set_gas(torch.from_numpy(Y).pin_memory(), torch.from_numpy(T).pin_memory())
    for c in ctxs[:6]:
        c.dem_step(5)
    ctxs[6].dem_step_graph(5)
    s = [c.dem_get_state() for c in ctxs]
    gs = [c.dem_get_gas() for c in ctxs]
    assert np.array_equal(s[1], s[2]) and np.array_equal(s[1], s[3]) and np.array_equal(s[1], s[5])
    assert np.array_equal(gs[1], gs[2]) and np.array_equal(gs[1], gs[3]) and np.array_equal(gs[1], gs[5])
    ref = _ctx(bed, prec)        # the graph-stepped context against eager steps of its own history
    ref.dem_step(5)
    ref.dem_step(2)
    ref.dem_set_gas(Y, T)
    ref.dem_step(5)
    assert np.array_equal(ref.dem_get_state(), s[6]) and np.array_equal(ref.dem_get_gas(), gs[6])
    ref.close()
    assert np.array_equal(s[4], s[0]) and np.array_equal(gs[4], gs[0])
    assert not np.array_equal(s[1], s[0])
    for c in ctxs:
        c.close()


def test_batched_32_beds_of_uneven_size():
    # the batched workload's shape scaled down: 32 beds of 500..5,000 parcels, 773..1073 K,
    # inlet velocities 0.2..0.5 m/s, 20 x 20 x 120 cells each, stepped as replayed graphs
    bed = synth.config_batched_32(n_min=500, n_max=5000, v_scale=0.2)
    counts = np.bincount(bed.bed, minlength=32)
    assert counts.min() >= 500 and counts.max() <= 5000 and counts.max() > 3 * counts.min()
    ref = oracle.Oracle(bed)
    ref.step(10)
    so = ref.state()
    mo, oo, _ = ref.reduction_degree()
    co, po, _ = ref.contacts()
    ctx = _ctx(bed)
    ctx.dem_step_graph(10)
    sg = ctx.dem_get_state()
    for row in range(binding.DEM_NSTATE):
        assert _rel(sg[row], so[row]) < 1e-7, binding.STATE_ROWS[row]
    cg, pg, _ = ctx.dem_get_contacts()
    assert _pairs(cg, pg) == _pairs(co, po)
    assert sum(co) > 200
    mg, og = ctx.dem_reduction_degree()
    assert np.allclose(mg, mo, rtol=0, atol=1e-12) and np.allclose(og, oo, rtol=0, atol=1e-12)
    ctx.close()
    ctx = _ctx(bed, "split")
    ctx.dem_step_graph(10)
    mg, _ = ctx.dem_reduction_degree()
    assert np.all(np.abs(mg - mo) < 1e-6)      # every bed's reduction degree (target 1e-3)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "split", "split_kahan"])
def test_kinetics_at_a_chemistry_time_step(prec):
    # the reduction-degree curve where it moves: the bed's chemistry stepped at dt = 1e-3 s
    # for 3,000 steps (3 s of reduction at 1073 K), contacts, drag and gravity off so the
    # parcels stay in their cells; heat, kinetics and the gas update on. The FP32 forms'
    # bed-mean f_ov against the FP64 oracle to 1e-3 absolute (the target) -- in practice
    # much closer -- and the FP64 form to 1e-9.
    bed = synth.small_packed(seed=14, n=1500, T0=1073.0, v_scale=0.0)
    c = bed.beds[0]
    c.dt = 1e-3
    c.kn = 0.01                         # no contact is evaluated; passes the stability check
    c.flags = synth.NO_CONTACTS | synth.NO_GRAVITY | synth.NO_DRAG
    ref = oracle.Oracle(bed)
    ctx = _ctx(bed, prec)
    worst = 0.0
    f_first = None
    for k in range(6):
        ctx.dem_step(500)
        ref.step(500)
        mg, _ = ctx.dem_reduction_degree()
        mo, _, _ = ref.reduction_degree()
        f_first = f_first if f_first is not None else mo[0]
        worst = max(worst, abs(mg[0] - mo[0]))
    assert mo[0] > 0.02 and mo[0] > 2 * f_first        # the curve really moves
    assert worst < (1e-9 if prec == "fp64" else 1e-3), worst
    if prec != "fp64":
        assert worst < 1e-4, worst
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "split_kahan"])
def test_occupied_sources_match_the_dense_rows(prec):
    # several beds with immersed-boundary cells (parcels never sit in solid cells), a bed with
    # no parcels at all, many chunks of sorted positions; and the capacity check
    beds = [synth.small_packed(seed=s, n=n, v_scale=0.3, wall_kind=w) for s, n, w in
            ((61, 2500, synth.WALL_CONE), (62, 10, synth.WALL_FLAT), (63, 1800, synth.WALL_FLAT))]
    beds[1] = beds[1].subset(np.arange(0))   # the middle bed without parcels
    cat = lambda f: np.concatenate([getattr(b, f) for b in beds])
    bed = synth.Bed([b.beds[0] for b in beds], cat("x"), cat("y"), cat("z"), cat("vx"), cat("vy"), cat("vz"),
                    cat("d_real"), cat("T"), np.concatenate([b.m0 for b in beds], axis=1), cat("ore"),
                    np.concatenate([np.full(b.n, k, np.int32) for k, b in enumerate(beds)]), "three-beds")
    ctx = _ctx(bed, prec=prec)
    for _ in range(2):
        ctx.dem_step(7)
        dense = ctx.dem_get_sources()
        cells, rows = ctx.dem_get_sources_occupied()
        occ = np.flatnonzero(dense[:, binding.SOURCE_ROWS.index("count")] > 0)
        assert len(occ) > 100
        assert np.array_equal(cells, occ)
        assert np.array_equal(rows, dense[occ])
        assert np.all(dense[np.setdiff1d(np.arange(ctx.ncells), occ)] == 0)
        # page-locked buffers take the rows from the kernel itself: the same rows
        cap = min(ctx.n, ctx.ncells)
        pc = torch.full((cap,), -7, dtype=torch.int64).pin_memory()
        po = torch.full((cap, binding.DEM_NDEP), -7.0, dtype=torch.float64).pin_memory()
        c2, r2 = ctx.dem_get_sources_occupied(pc, po)
        assert np.array_equal(c2.numpy(), occ) and np.array_equal(r2.numpy(), dense[occ])
        assert np.all(pc[len(occ):].numpy() == -7) and np.all(po[len(occ):].numpy() == -7.0)
    small = np.zeros(10, dtype=np.int64), np.zeros((10, binding.DEM_NDEP))
    with pytest.raises(binding.DemError):
        ctx.dem_get_sources_occupied(*small)
    # too small page-locked buffers: the count is refused and nothing is written
    ps = torch.full((10,), -7, dtype=torch.int64).pin_memory(), torch.full((10, binding.DEM_NDEP), -7.0).pin_memory()
    with pytest.raises(binding.DemError):
        ctx.dem_get_sources_occupied(*ps)
    assert np.all(ps[0].numpy() == -7) and np.all(ps[1].numpy() == -7.0)
    ctx.close()
