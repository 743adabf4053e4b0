"""Pins of the oracle's gas-phase solver (CPU only): Sec. 3.2 and Sec. 4 (eqs (3-24),
(4-2), (4-6), (4-9), the pseudo-turbulence closures (3-28)..(3-37)).

Checks: a still gas column under gravity is hydrostatic (no flow, dp = rho g h per cell);
the inflow through the bottom leaves through the top (mass conservation); inside a fixed bed
of parcels the gas pressure gradient balances the drag the parcels feel (momentum exchange
between the phases) and follows Ergun's law at low flow; the pseudo-turbulent stress has the
trace 2 k_g of eq (3-28) (b traceless), its heat-flux anisotropy is that of eq (3-37), and
both vanish without slip.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth
from tests.helpers import bed_from_arrays

NO_PARTICLE_PHYSICS = synth.NO_DRAG | synth.NO_HEAT | synth.NO_KINETICS


def _column(U_in=0.0, nz=8, flags=0, **kw):
    cfg = synth.BedConfig(D=0.012, H=0.003 * nz, nx=4, ny=4, nz=nz, dt=1e-5, cg_ratio=4.0, U_in=U_in,
                          T_in=1000.0, coupling_interval=10, flags=flags | synth.GAS_SOLVER, **kw)
    return cfg


def test_still_gas_is_hydrostatic():
    cfg = _column(flags=NO_PARTICLE_PHYSICS)
    o = oracle.Oracle(bed_from_arrays(cfg, [0.0], 0.0, 0.02))
    o.step(20)
    fl = o.flow()
    rho = oracle.gas_props(cfg, 1000.0, [1, 0, 0])["rho"]
    p = fl[:, 3].reshape(cfg.nz, cfg.ny, cfg.nx)
    assert np.abs(fl[:, :3]).max() < 1e-12
    assert np.allclose(p[:-1] - p[1:], rho * 9.81 * cfg.H / cfg.nz, rtol=1e-10, atol=0)


def test_inflow_leaves_through_the_outlet():
    cfg = _column(U_in=0.2, flags=NO_PARTICLE_PHYSICS | synth.NO_GRAVITY)
    o = oracle.Oracle(bed_from_arrays(cfg, [0.0], 0.0, 0.02, d_real=1e-7))   # a parcel of negligible volume
    o.step(30)
    fl = o.flow()
    w = fl[:, 2].reshape(cfg.nz, cfg.ny, cfg.nx)
    mark = o.gas()[:, oracle.G_MARK].reshape(cfg.nz, cfg.ny, cfg.nx)
    # every horizontal plane carries the inlet's mass flow (uniform density: volume flow)
    A = (cfg.D / cfg.nx) * (cfg.D / cfg.ny)
    inflow = cfg.U_in * A * (mark[0] == 0).sum()
    for k in range(cfg.nz):
        assert abs(w[k][mark[k] == 0].sum() * A - inflow) < 1e-9 * inflow, k
    # the no-slip walls shift the inlet's plug flow toward the axis near the inlet: a small,
    # symmetric cross flow (no net lateral flow in any plane)
    assert np.abs(fl[:, :2]).max() < 0.02 * cfg.U_in
    uxy = fl[:, :2].reshape(cfg.nz, cfg.ny * cfg.nx, 2)
    assert np.abs(uxy.sum(axis=1)).max() < 1e-12


def _fixed_bed(U_in):
    # one column of gas cells (a 1-D bed: the gas cannot pass the parcels by), its lower three
    # cells filled by a cubic lattice of touching parcels; no contacts, so they rest where they
    # are over the few steps taken; gas and drag on
    cfg = synth.BedConfig(D=0.004, H=0.032, nx=1, ny=1, nz=8, dt=1e-5, cg_ratio=4.0, U_in=U_in, T_in=1000.0,
                          coupling_interval=10, kn=1e-3, flags=synth.NO_HEAT | synth.NO_KINETICS |
                          synth.GAS_SOLVER | synth.NO_CONTACTS)
    d = 100e-6
    pitch = cfg.cg_ratio * d
    g = (np.arange(10) + 0.5) * pitch - 0.002
    X, Y, Z = np.meshgrid(g, g, (np.arange(30) + 0.5) * pitch, indexing="ij")
    return cfg, bed_from_arrays(cfg, X.ravel(), Y.ravel(), Z.ravel(), d_real=d, T=1000.0)


def test_fixed_bed_pressure_gradient_balances_the_drag():
    cfg, b = _fixed_bed(0.02)
    o = oracle.Oracle(b)
    o.step(10)
    fl, gas, dg = o.flow(), o.gas(), o.diag()
    nx, ny, nz = cfg.nx, cfg.ny, cfg.nz
    p = fl[:, 3].reshape(nz, ny, nx)
    eps = gas[:, oracle.G_EPS].reshape(nz, ny, nx)
    cell = dg[oracle.D_CELL].astype(int)
    hz = cfg.H / nz
    V = (cfg.D / nx) * (cfg.D / ny) * hz
    rho = oracle.gas_props(cfg, 1000.0, [1, 0, 0])["rho"]
    # the central cells of the layers k = 1, 2 (inside the lattice): the gas column between the
    # two cell centres carries the drag of the parcels of the lower cell and its weight
    for k in (1,):
        Fz = dg[oracle.D_FD + 2][cell == k].sum()              # drag on the parcels of cell k
        dpdz = (p[k + 1, 0, 0] - p[k, 0, 0]) / hz
        e = eps[k, 0, 0]
        assert abs((-e * dpdz - e * rho * 9.81) * V - Fz) < 1e-3 * Fz
    # Ergun's law for the lattice's porosity and the real particle diameter
    mu = oracle.gas_props(cfg, 1000.0, [1, 0, 0])["mu"]
    e = eps[1, 0, 0]
    d = 100e-6
    U = cfg.U_in
    ergun = 150 * mu * (1 - e) ** 2 * U / (e ** 3 * d * d) + 1.75 * rho * (1 - e) * U * U / (e ** 3 * d)
    dpdz = (p[2, 0, 0] - p[1, 0, 0]) / hz + rho * 9.81
    assert abs(-dpdz / ergun - 1) < 0.02


def test_pseudo_turbulence_closures():
    ug, up = np.array([0.1, 0.0, 0.5]), np.zeros(3)
    t = oracle.pseudo_turbulence(0.6, 0.03, 2e-5, 0.4, 14000.0, ug, up, 2e-4)
    s = ug / np.linalg.norm(ug)
    assert np.allclose(t["s"], s, atol=1e-15)
    # eq (3-28) with b traceless: trace R = R_pa + 2 R_pe = 2 k_g, k_g of eqs (3-29), (3-30)
    ep, e = 0.4, 0.6
    slip = np.linalg.norm(ug)
    Re = e * 0.03 * slip * 2e-4 / 2e-5
    kg = 0.5 * slip ** 2 * (2 * ep + 2.5 * ep * e ** 3 * math.exp(-ep * math.sqrt(Re)))
    assert abs(t["Rpa"] + 2 * t["Rpe"] - 2 * kg) < 1e-12 * kg
    assert t["Rpa"] > t["Rpe"] > 0            # stress stronger along the slip
    # eq (3-37): alpha_pe / alpha_pa = (3 b_pe + 1) / (3 b_pa + 1) = R_pe / R_pa
    assert abs(t["ape"] / t["apa"] - t["Rpe"] / t["Rpa"]) < 1e-12
    z = oracle.pseudo_turbulence(0.6, 0.03, 2e-5, 0.4, 14000.0, up, up, 2e-4)
    assert z["Rpa"] == 0 and z["apa"] == 0
    # the heat-flux closure grows with the slip Reynolds number
    a = [oracle.pseudo_turbulence(0.6, 0.03, 2e-5, 0.4, 14000.0, np.array([0, 0, v]), up, 2e-4)["apa"]
         for v in (0.05, 0.2, 0.8)]
    assert a[0] < a[1] < a[2]


def test_equimolar_reduction_keeps_the_molar_flow():
    # H2 + O(ore) -> H2O replaces one mole of gas by one (eqs (2-25), (3-25)): with the gas
    # density of eq (3-53), continuity (eq (3-24)) then keeps the molar flow through a reacting
    # column while the H2O fraction at the outlet climbs from 5 % to above 40 %; only the slight
    # heating by the exothermic first reaction expands the gas (parcels static, gas and parcels
    # at the inlet temperature to start with)
    cfg = synth.BedConfig(D=0.004, H=0.024, nx=1, ny=1, nz=8, dt=1e-5, cg_ratio=4.0, U_in=0.2, T_in=1000.0,
                          coupling_interval=10, Y_in=(0.9, 0.05, 0.05), kn=1e-3,
                          flags=synth.GAS_SOLVER | synth.NO_GRAVITY | synth.NO_CONTACTS | synth.NO_DRAG)
    rng = np.random.default_rng(3)
    n = 40
    x = rng.uniform(-0.001, 0.001, n)
    y = rng.uniform(-0.001, 0.001, n)
    z = rng.uniform(0.004, 0.012, n)
    o = oracle.Oracle(bed_from_arrays(cfg, x, y, z, d_real=100e-6, T=1000.0, comp=(1.0, 0.0, 0.0, 0.0)))
    A = cfg.D ** 2
    molar_in = cfg.U_in * A * cfg.p0 / (8.314 * cfg.T_in)
    for _ in range(6):
        o.step(1000)
        g = o.gas()
        _, _, fw = o.faces()
        molar_out = g[-1, oracle.G_EPS] * fw[-1, 0, 0] * A * cfg.p0 / (8.314 * g[-1, 4])
        assert abs(molar_out / molar_in - 1) < 2e-3
    assert g[-1, 2] > 0.4
    assert g[:, 4].max() - cfg.T_in < 5.0


def test_solved_flow_carries_a_band_at_the_inlet_velocity():
    # one column of cells without parcels and a band of gas exchanged at the same mean molar
    # mass (more H2O, less N2 and H2), so the density stays uniform: continuity (eq (3-24))
    # makes the solved flow the plug flow U_in, and the species balance (eq (4-9)) carries the
    # band up the column at that speed -- its excess is conserved and its centroid advances
    # by U_in dt_CFD / dz cells per coupling step. The balance's molecular diffusion spreads
    # the band symmetrically; with its composition-dependent coefficient it moves the centroid
    # by ~1e-4 of that shift, so the speed is checked to 1e-3 (a wrong velocity, sign or
    # upwind direction is off by far more)
    nz, U, dt, n = 60, 0.2, 1e-4, 10
    cfg = synth.BedConfig(D=0.004, H=0.003 * nz, nx=1, ny=1, nz=nz, dt=dt, cg_ratio=4.0, U_in=U, T_in=1000.0,
                          Y_in=(0.9, 0.05, 0.05), coupling_interval=n,
                          flags=NO_PARTICLE_PHYSICS | synth.NO_GRAVITY | synth.GAS_SOLVER)
    M = np.array([2.016e-3, 18.015e-3, 28.014e-3])
    # (dH2, dH2O, dN2) with sum 0 and sum d/M 0: the mean molar mass is unchanged
    d_h2o = 0.04
    A = np.array([[1.0, 1.0], [1.0 / M[0], 1.0 / M[2]]])
    d_h2, d_n2 = np.linalg.solve(A, [-d_h2o, -d_h2o / M[1]])
    band = (np.arange(nz) >= 8) & (np.arange(nz) < 12)
    Y = np.tile([0.9, 0.05, 0.05], (nz, 1))
    Y[band] += [d_h2, d_h2o, d_n2]
    assert Y.min() > 0
    o = oracle.Oracle(bed_from_arrays(cfg, np.zeros(0), 0.0, 0.0), Y, np.full(nz, 1000.0))
    z = np.arange(nz)

    def moments():
        ex = o.gas()[:, 2] - 0.05
        return ex.sum(), (z * ex).sum()

    m0, f0 = moments()
    solves = 100
    o.step(solves * n)
    m1, f1 = moments()
    fl = o.flow()
    assert np.allclose(fl[:, 2], U, rtol=1e-10) and np.abs(fl[:, :2]).max() == 0.0
    assert abs(o.gas()[-3:, 2] - 0.05).max() < 1e-12           # the band has not reached the outlet
    k = U * n * dt / (cfg.H / nz)
    assert abs(m1 / m0 - 1.0) < 1e-10
    assert abs((f1 / m1 - f0 / m0) / (solves * k) - 1.0) < 1e-3
    assert o.gas()[:, 2].max() < 0.09 and o.gas()[:, 2].min() >= 0.05 - 1e-15   # spread, no new extrema
