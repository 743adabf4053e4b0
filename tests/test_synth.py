"""The seeded synthetic inputs against the workloads they stand for (CPU only): parcel counts,
grids, bed geometry, size distributions, ores, temperatures and inlet velocities of the five
benchmark configurations, and that a seed reproduces its bed bit for bit."""
import math

import numpy as np
import pytest

from paper_2311_03908_gb300 import synth


def _inside_cylinder(bed, cfg):
    """Every parcel inside the cylinder, touching the wall at most by 2 % of its radius (the
    packed lattices' outermost boxes reach the wall; contacts push those parcels in)."""
    r = np.hypot(bed.x, bed.y)
    rp = 0.5 * cfg.cg_ratio * bed.d_real
    return np.all(r + rp <= 0.5 * cfg.D + 0.02 * rp) and np.all(bed.z - rp >= -0.02 * rp) and \
        np.all(bed.z + rp <= cfg.H)


def _log_stats(d):
    ld = np.log(d)
    return math.exp(np.median(ld)), ld.std()


def test_plain_2k():
    bed = synth.config_plain_2k()
    cfg = bed.beds[0]
    assert bed.n == 2000 and (cfg.D, cfg.H, cfg.nx, cfg.ny, cfg.nz) == (0.05, 0.3, 10, 10, 60)
    assert np.all(bed.d_real == 100e-6) and cfg.cg_ratio == 4.0
    assert (cfg.kn, cfg.restitution, cfg.mu_s) == (1000.0, 0.9, 0.3)
    assert cfg.U_in == 0.3 and cfg.T_in == 873.0 and tuple(cfg.Y_in) == (1.0, 0.0, 0.0) and cfg.dt == 1e-5
    assert np.all(bed.T == 873.0) and bed.meta["steps"] == 200
    assert np.all(bed.m0[1:] == 0.0)                    # pure hematite
    # hematite density 5000 kg/m3 at the coarse-grained diameter
    dc = cfg.cg_ratio * bed.d_real
    assert np.allclose(bed.m0[0], 5000.0 * math.pi / 6.0 * dc ** 3, rtol=1e-12)
    assert _inside_cylinder(bed, cfg)
    # uniform in the cylinder: the radial CDF of points is r^2 / R^2 (KS distance, loosely)
    R = 0.5 * cfg.D - 0.5 * dc[0]
    r = np.sort(np.hypot(bed.x, bed.y) / R)
    assert np.abs(r ** 2 - (np.arange(1, bed.n + 1) - 0.5) / bed.n).max() < 0.05


def test_split_200k():
    bed = synth.config_split_200k(n=20_000)             # the recipe at a tenth of the count
    cfg = bed.beds[0]
    assert (cfg.D, cfg.H, cfg.nx, cfg.ny, cfg.nz, cfg.cg_ratio, cfg.T_in) == (0.1, 0.6, 40, 40, 240, 6.0, 1023.0)
    med, sig = _log_stats(bed.d_real)
    assert abs(med / 100e-6 - 1) < 0.02 and abs(sig - 0.25) < 0.01
    assert bed.d_real.max() <= 100e-6 * math.exp(3 * 0.25) * (1 + 1e-12)
    assert bed.meta["steps"] == 1000 and _inside_cylinder(bed, cfg)


def test_ibm_2m_recipe():
    bed = synth.config_ibm_2m(n=100_000)                # the 2M bed's recipe on fewer parcels
    cfg = bed.beds[0]
    assert (cfg.nx, cfg.ny, cfg.nz, cfg.D, cfg.H) == (64, 64, 384, 0.1, 0.6)
    assert cfg.wall_kind == synth.WALL_CONE and cfg.plate_z > 0 and cfg.hole_d > 0
    med, sig = _log_stats(bed.d_real)
    assert abs(med / 120e-6 - 1) < 0.02 and abs(sig - 0.25) < 0.01
    # two ores in (nearly) equal mass: hematite Fe2O3 and magnetite-rich Fe3O4 parcels
    mass = bed.m0.sum(0)
    hem = bed.ore == synth.ORE_HEMATITE
    assert 0.45 < mass[hem].sum() / mass.sum() < 0.55
    assert np.all(bed.m0[0, hem] > 0) and np.all(bed.m0[1, ~hem] > bed.m0[0, ~hem])
    assert np.all(bed.z - 0.5 * cfg.cg_ratio * bed.d_real >= cfg.plate_z - 1e-12)   # above the plate
    assert bed.meta["steps"] == 500


def test_ibm_2m_is_two_million_parcels_and_reproducible():
    a = synth.config_ibm_2m()
    assert a.n == 2_000_000
    b = synth.config_ibm_2m()
    for f in ("x", "y", "z", "d_real", "ore"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_adjoint_64k():
    bed = synth.config_adjoint_64k()
    assert bed.n == 64_000 and bed.meta["steps"] == 2000 and bed.meta["ckpt"] == 100
    assert np.all(bed.m0[:3] > 0)                       # all three oxides present: every reaction runs


def test_batched_32():
    bed = synth.config_batched_32(n_min=1_000, n_max=20_000)   # counts scaled by 1/10
    assert len(bed.beds) == 32
    counts = np.bincount(bed.bed, minlength=32)
    assert counts.min() >= 1_000 and counts.max() <= 20_000 and counts.max() > 3 * counts.min()
    T = np.array([c.T_in for c in bed.beds])
    assert np.allclose(T, np.linspace(773.0, 1073.0, 32))          # 32 even steps
    U = np.array([c.U_in for c in bed.beds])
    assert U.min() >= 0.2 and U.max() <= 0.5 and U.std() > 0.05
    assert all((c.nx, c.ny, c.nz) == (20, 20, 120) for c in bed.beds)
    assert bed.meta["steps"] == 500
    full = synth.config_batched_32.__defaults__
    assert full[2:4] == (10_000, 200_000)               # the workload's own count range


@pytest.mark.parametrize("seed", [1, 2])
def test_seeds_reproduce_and_differ(seed):
    a, b = synth.small_packed(seed=seed), synth.small_packed(seed=seed)
    c = synth.small_packed(seed=seed + 10)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.d_real, b.d_real)
    assert not np.array_equal(a.x, c.x)
