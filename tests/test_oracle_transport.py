"""Pins of the oracle's drag, convection, gas properties and thermochemistry (CPU only).

Checks against textbook limits and invariants: Stokes drag, Nu = Sh = 2 in still gas,
Fuller's temperature and pressure scaling, the binary limit of Wilke's rule, the ideal
gas density of H2 at STP, NASA-type consistency dH/dT = C_p, and standard formation
enthalpies at 298.15 K.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth
from tests.helpers import ISOLATED, bed_from_arrays


def test_stokes_drag_limit():
    # dilute limit (eps_g -> 1, Wen-Yu branch) at Re -> 0: beta/eps_p * V_real = 3 pi mu d / K1
    cfg = synth.BedConfig(D=10.0)
    d = 100e-6
    Y = [1.0, 0.0, 0.0]
    slip = 1e-9
    bo, Re = oracle.drag(cfg, d, 0, 1.0, slip, 873.0, Y)
    mu = oracle.gas_props(cfg, 873.0, Y)["mu"]
    K1 = 1.0 - 2.25 * d / cfg.D
    V = math.pi / 6 * d ** 3
    assert Re < 1e-8
    assert abs(bo * V - 3 * math.pi * mu * d / K1) < 1e-6 * 3 * math.pi * mu * d


def test_nusselt_sherwood_still_gas_limit():
    cfg = synth.BedConfig()
    Nu, h = oracle.heat(cfg, 100e-6, 1.0, 0.0, 873.0, [1, 0, 0])
    assert abs(Nu - 2.0) < 1e-15
    k = oracle.kinetics(cfg, np.array([1, 0, 0, 0]) * 1e-7, 873.0, 100e-6, 0, 1.0, 0.0, 873.0,
                        [1, 0, 0], 1e-5)
    assert abs(k["Sh"] - 2.0) < 1e-15


def test_conduction_limit_in_a_full_step():
    # a parcel at rest in still gas of a huge cell: Q_conv = k^3 * 2 pi lambda d (T_g - T_p)
    cfg = synth.BedConfig(D=0.2, H=0.2, nx=1, ny=1, nz=1, U_in=0.0, T_in=900.0,
                          flags=ISOLATED & ~synth.NO_HEAT)
    d = 100e-6
    b = bed_from_arrays(cfg, [0.0], 0.0, 0.1, d_real=d, T=880.0)
    o = oracle.Oracle(b)
    o.step(1)
    q = o.diag()[oracle.D_QCONV, 0]
    lam = oracle.gas_props(cfg, 900.0, [1, 0, 0])["lam"]
    expect = 4.0 ** 3 * 2 * math.pi * lam * d * (900.0 - 880.0)
    assert abs(q - expect) < 1e-5 * expect


def test_fuller_scaling_and_wilke_binary_limit():
    cfg = synth.BedConfig()
    g1 = oracle.gas_props(cfg, 600.0, [0.5, 0.5, 0.0], p=101325.0)
    g2 = oracle.gas_props(cfg, 1200.0, [0.5, 0.5, 0.0], p=101325.0)
    g3 = oracle.gas_props(cfg, 600.0, [0.5, 0.5, 0.0], p=2 * 101325.0)
    assert abs(g2["D12"] / g1["D12"] - 2 ** 1.75) < 1e-12
    assert abs(g3["D12"] / g1["D12"] - 0.5) < 1e-12
    # two components (no N2): Wilke's mixture rule is the binary coefficient
    assert abs(g1["Dm"] - g1["D12"]) < 1e-15 * g1["D12"]
    # lighter partner diffuses faster: D(H2,H2O) > D(H2,N2)
    assert g1["D12"] > g1["D13"]


def test_ideal_gas_density_h2_at_stp():
    g = oracle.gas_props(synth.BedConfig(), 273.15, [1, 0, 0], p=101325.0)
    assert abs(g["rho"] - 0.08988) < 0.002 * 0.08988


def test_mole_fractions_from_mass_fractions():
    # equal moles of H2 and N2 -> x' = 0.5 each and x_H2 (H2 basis) = 1
    M1, M3 = oracle.molar_mass("H2"), oracle.molar_mass("N2")
    Y = [M1 / (M1 + M3), 0.0, M3 / (M1 + M3)]
    g = oracle.gas_props(synth.BedConfig(), 900.0, Y)
    assert np.allclose(g["xp"], [0.5, 0.0, 0.5], atol=1e-15)
    assert g["x"] == 1.0


@pytest.mark.parametrize("species", oracle.SPECIES)
def test_enthalpy_derivative_is_heat_capacity(species):
    ranges = {"Fe2O3": [500, 1300], "Fe3O4": [500, 1300], "Fe": [500, 1400]}.get(species, [500, 1400])
    for T in ranges:
        h = 1e-3
        dH = (oracle.enthalpy(species, T + h) - oracle.enthalpy(species, T - h)) / (2 * h)
        assert abs(dH - oracle.cp(species, T)) < 1e-6 * abs(oracle.cp(species, T))


@pytest.mark.parametrize("species,h298", [("H2", 0.0), ("N2", 0.0), ("H2O", -241.83),
                                          ("Fe2O3", -824.2), ("Fe3O4", -1118.4), ("FeO", -272.0),
                                          ("Fe", 0.0)])
def test_standard_formation_enthalpy(species, h298):
    # standard enthalpies of formation at 298.15 K (kJ/mol); the printed coefficients carry
    # about three digits, so agreement to 1.5 kJ/mol is what the table allows
    H = oracle.enthalpy(species, 298.15) * oracle.molar_mass(species) / 1e3
    assert abs(H - h298) < 1.5


def test_reaction_heat_signs_at_1073K():
    # Table 1 lists R2, R3 as endothermic; with Table C1 (as read) at 1073 K they are
    def dH(react, prod):
        f = lambda side: sum(c * oracle.enthalpy(s, 1073.0) * oracle.molar_mass(s) for c, s in side)
        return f(prod) - f(react)
    r2 = dH([(1, "Fe3O4"), (1, "H2")], [(3, "FeO"), (1, "H2O")])
    r3 = dH([(1, "FeO"), (1, "H2")], [(1, "Fe"), (1, "H2O")])
    assert r2 > 0 and r3 > 0
