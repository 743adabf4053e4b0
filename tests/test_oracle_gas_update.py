"""Pins of the oracle's prescribed gas update (the builder's explicit field of reading 19: the
species and energy balances of Sec. 4, eqs (4-6), (4-8)..(4-11), advected upwind by the
prescribed flow) against what the mathematics fixes, not against its own formulas (CPU only):

* advection (empty column, no sources): the first-order upwind scheme conserves each species
  between the inflow and the outflow, creates no new extrema, and moves a band of excess
  H2O (or of excess temperature) up the column at the flow speed U_in / eps_g: the band's
  first moment advances by exactly U_in dt / dz cells per step;
* heat exchange (static parcels, no flow): what the gas gains equals what the parcels lose
  (their convective heat, eq (3-10)) up to the first-order splitting of the semi-implicit
  update, and a gas already at the parcels' temperature stays there;
* species sources (reacting parcels, no flow): the updated mass fractions are the exact
  mixing of the deposited mass into the cell's gas, (m_g Y_j + S_j dt) / (m_g + S_net dt),
  to second order in the added mass.
"""
import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth
from tests.helpers import bed_from_arrays

INERT = synth.NO_GRAVITY | synth.NO_DRAG | synth.NO_HEAT | synth.NO_KINETICS | synth.NO_CONTACTS


def _column(nz, U_in, dt, flags, **kw):
    return synth.BedConfig(D=0.012, H=0.003 * nz, nx=4, ny=4, nz=nz, dt=dt, cg_ratio=4.0, U_in=U_in,
                           T_in=1000.0, Y_in=(0.9, 0.05, 0.05), coupling_interval=1, flags=flags, **kw)


def _cell(cfg):
    """Cell edges and volume of the bed's grid: the D x D x H box in nx x ny x nz cells."""
    dx, dy, dz = cfg.D / cfg.nx, cfg.D / cfg.ny, cfg.H / cfg.nz
    return dx, dy, dz, dx * dy * dz


def _fluid_columns(g, cfg):
    """Which (x, y) columns of a single bed are fluid from bottom to top."""
    mark = g[:, 5].reshape(cfg.nz, cfg.ny * cfg.nx)
    keep = np.all(mark == 0, axis=0)
    return keep


def test_upwind_advection_conserves_and_moves_a_band_at_the_flow_speed():
    nz, U, dt = 60, 0.2, 1e-3
    cfg = _column(nz, U, dt, INERT)
    bed = bed_from_arrays(cfg, np.zeros(0), 0.0, 0.0)            # no parcels: eps_g = 1
    nc = cfg.nx * cfg.ny * nz
    layer = np.repeat(np.arange(nz), cfg.nx * cfg.ny)
    band = (layer >= 8) & (layer < 12)
    Y = np.tile([0.9, 0.05, 0.05], (nc, 1))
    Y[band] = [0.7, 0.25, 0.05]                                    # 0.2 of H2 exchanged for H2O
    T = np.full(nc, 1000.0)
    T[band] = 1060.0
    ref = oracle.Oracle(bed, Y, T)
    g0 = ref.gas()
    keep = _fluid_columns(g0, cfg)
    assert keep.sum() >= 4
    k = U * dt / _cell(cfg)[2]                                     # cells per step
    assert np.allclose(g0[:, 0], 1.0)
    z = np.arange(nz)[:, None]

    def moments(g):
        ex = (g[:, 2] - 0.05).reshape(nz, -1)[:, keep]             # excess H2O per column
        et = (g[:, 4] - 1000.0).reshape(nz, -1)[:, keep]           # excess temperature
        return ex.sum(0), (z * ex).sum(0), et.sum(0), (z * et).sum(0)

    m0, f0, t0, ft0 = moments(g0)
    steps = 120
    for _ in range(steps):
        ref.step(1)
    g = ref.gas()
    m1, f1, t1, ft1 = moments(g)
    # the band (its numerical-diffusion tail included) has not reached the outlet: the excess
    # is conserved and its centroid has moved up by steps * k cells
    assert np.abs(g[:, 2].reshape(nz, -1)[-3:, keep] - 0.05).max() < 1e-12
    assert np.allclose(m1, m0, rtol=1e-12)
    assert np.allclose(f1 / m1 - f0 / m0, steps * k, rtol=1e-10)
    assert np.allclose(t1, t0, rtol=1e-12)
    assert np.allclose(ft1 / t1 - ft0 / t0, steps * k, rtol=1e-10)
    # no new extrema; the mass fractions still add up to one
    assert g[:, 2].min() >= 0.05 - 1e-15 and g[:, 2].max() <= 0.25 + 1e-15
    assert g[:, 4].min() >= 1000.0 - 1e-10 and g[:, 4].max() <= 1060.0 + 1e-10
    assert np.allclose(g[:, 1:4].sum(1), 1.0, rtol=0, atol=1e-14)


def test_upwind_outflow_balances_the_column_total():
    # a front of H2O-rich gas at the top: per step the column total changes by the inflow of
    # inlet gas minus the outflow of the top cell's gas, k (Y_in - Y_top)
    nz, U, dt = 12, 0.2, 1e-3
    cfg = _column(nz, U, dt, INERT)
    bed = bed_from_arrays(cfg, np.zeros(0), 0.0, 0.0)
    nc = cfg.nx * cfg.ny * nz
    layer = np.repeat(np.arange(nz), cfg.nx * cfg.ny)
    Y = np.tile([0.9, 0.05, 0.05], (nc, 1))
    Y[layer >= 6] = [0.6, 0.35, 0.05]
    ref = oracle.Oracle(bed, Y, np.full(nc, 1000.0))
    keep = _fluid_columns(ref.gas(), cfg)
    k = U * dt / _cell(cfg)[2]
    for _ in range(30):
        g0 = ref.gas()[:, 2].reshape(nz, -1)[:, keep]
        ref.step(1)
        g1 = ref.gas()[:, 2].reshape(nz, -1)[:, keep]
        assert np.allclose(g1.sum(0) - g0.sum(0), k * (0.05 - g0[-1]), rtol=1e-9, atol=1e-15)


def _static_parcels(cfg, T_p, seed=3, n=40):
    rng = np.random.default_rng(seed)
    return bed_from_arrays(cfg, rng.uniform(-0.003, 0.003, n), rng.uniform(-0.003, 0.003, n),
                           rng.uniform(0.004, 0.020, n), d_real=100e-6, T=T_p, comp=(1.0, 0.0, 0.0, 0.0))


def test_heat_exchange_conserves_energy_between_gas_and_parcels():
    dt = 2e-6
    cfg = _column(8, 0.0, dt, synth.NO_GRAVITY | synth.NO_DRAG | synth.NO_KINETICS | synth.NO_CONTACTS)
    bed = _static_parcels(cfg, 900.0)
    ref = oracle.Oracle(bed)
    ref.step(1)                                    # the gas state and properties of a step
    g0 = ref.gas()
    ref.step(1)
    g1, dep, dg = ref.gas(), ref.deposits(), ref.diag()
    V = _cell(cfg)[3]
    cap = np.array([g0[c, 0] * oracle.gas_props(cfg, g0[c, 4], g0[c, 1:4])["rho"] *
                    oracle.gas_props(cfg, g0[c, 4], g0[c, 1:4])["cp"] for c in range(len(g0))])
    gas_gain = (cap * V * (g1[:, 4] - g0[:, 4])).sum()
    parcel_gain = dt * dg[oracle.D_QCONV].sum()   # the parcels' convective heat this step
    assert gas_gain < 0 < parcel_gain             # parcels at 900 K in a gas at 1000 K
    # the semi-implicit factor 1 / (1 + dt H0 / cap) is the only difference, to first order
    split = (dt * dep[:, 7] / V / cap).max()
    assert abs(gas_gain + parcel_gain) <= 2.0 * split * parcel_gain + 1e-12 * parcel_gain, \
        (gas_gain, parcel_gain, split)


def test_gas_at_the_parcel_temperature_stays_there():
    cfg = _column(8, 0.0, 2e-6, synth.NO_GRAVITY | synth.NO_DRAG | synth.NO_KINETICS | synth.NO_CONTACTS)
    bed = _static_parcels(cfg, 1000.0)
    ref = oracle.Oracle(bed)
    ref.step(5)
    g = ref.gas()
    assert np.abs(g[:, 4] - 1000.0).max() < 1e-9


def test_species_sources_mix_the_deposited_mass_into_the_cell_gas():
    dt = 2e-6
    cfg = _column(8, 0.0, dt, synth.NO_GRAVITY | synth.NO_DRAG | synth.NO_CONTACTS)
    bed = _static_parcels(cfg, 1073.0, seed=5, n=60)
    ref = oracle.Oracle(bed)
    ref.step(1)
    g0 = ref.gas()
    ref.step(1)
    g1, dep = ref.gas(), ref.deposits()
    V = _cell(cfg)[3]
    S = dep[:, 1:3]                                   # S_H2 (< 0), S_H2O (> 0), kg/s
    cells = np.flatnonzero(dep[:, 13] > 0)
    assert len(cells) > 5 and S[cells, 0].max() < 0 and S[cells, 1].min() > 0
    worst = 0.0
    # (the renormalisation of the fractions alone already dilutes by S_net: the mixing rule
    # holds whether the dilution term is written out or not)
    for c in cells:
        mg = g0[c, 0] * oracle.gas_props(cfg, g0[c, 4], g0[c, 1:4])["rho"] * V
        add = np.array([S[c, 0], S[c, 1], 0.0]) * dt
        mix = (mg * g0[c, 1:4] + add) / (mg + add.sum())
        second = (add.sum() / mg) ** 2 + (np.abs(add).max() / mg) ** 2
        err = np.abs(g1[c, 1:4] - mix).max()
        assert err <= 2.0 * second + 1e-15, (c, err, second)
        worst = max(worst, np.abs(g1[c, 1:4] - g0[c, 1:4]).max())
    assert worst > 1e-12                              # the sources did change the gas
