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
from tests.helpers import ISOLATED, bed_from_arrays, handbook_values


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


def test_fuller_absolute_value_against_measured_diffusivities():
    # eq (2-26) as a number, not only its scaling: the binary coefficients at 1 atm against
    # measured ones (Fuller's correlation reproduces such data to a few per cent)
    hb = handbook_values()
    cfg = synth.BedConfig()
    d13 = oracle.gas_props(cfg, 298.15, [0.5, 0.0, 0.5], p=101325.0)["D13"]
    d12 = oracle.gas_props(cfg, 307.1, [0.5, 0.5, 0.0], p=101325.0)["D12"]
    assert abs(d13 / hb["D_H2_N2_298K"] - 1.0) < 0.10, d13
    assert abs(d12 / hb["D_H2_H2O_307K"] - 1.0) < 0.10, d12


@pytest.mark.parametrize("T", [600, 1000])
def test_gas_heat_capacities_against_janaf(T):
    # the gas ranges of Table C1 as numbers: molar C_p of the pure gases against JANAF
    hb = handbook_values()
    M = {"H2": 2.016e-3, "H2O": 18.015e-3, "N2": 28.014e-3}
    for name, Y in (("H2", [1, 0, 0]), ("H2O", [0, 1, 0]), ("N2", [0, 0, 1])):
        cp = oracle.gas_props(synth.BedConfig(), float(T), Y, p=101325.0)["cp"] * M[name]
        assert abs(cp / hb[f"cp_{name}_{T}K"] - 1.0) < 0.01, (name, T, cp)


@pytest.mark.parametrize("species", ["Fe2O3", "Fe3O4", "FeO", "Fe"])
def test_solid_heat_capacities_at_298K_against_janaf(species):
    # the solids' low ranges of Table C1 as numbers (J/kg/K times the molar mass)
    cp = oracle.cp(species, 298.15) * oracle.molar_mass(species)
    assert abs(cp / handbook_values()[f"cp_{species}_298K"] - 1.0) < 0.03, (species, cp)


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


# ---------------------------------------------------------------------------------------
# Pins of the finite-Re and dense-bed branches against references independent of the paper.
# ---------------------------------------------------------------------------------------
def _gas(T=873.0, Y=(1.0, 0.0, 0.0)):
    return oracle.gas_props(synth.BedConfig(), T, list(Y))


@pytest.mark.parametrize("eps,psi,U", [(0.4, 1.0, 0.05), (0.4, 0.86, 2.0), (0.55, 0.7, 5.0), (0.7, 1.0, 20.0)])
def test_ergun_branch_is_the_fixed_bed_pressure_drop(eps, psi, U):
    # eq (3-5-2), eps_g < 0.8: in a fixed bed the drag the gas exerts per unit bed volume,
    # beta (u - v), balances eps_g times Ergun's pressure gradient at the superficial
    # velocity U = eps_g (u - v):  dp/dL = 150 mu (1-eps)^2 U / (eps^3 (psi d)^2)
    #                                      + 1.75 rho (1-eps) U^2 / (eps^3 psi d).
    # The high-U cases make the inertial term dominate (a wrong power of eps or psi there fails).
    cfg = synth.BedConfig(D=10.0, sphericity=(psi, psi))
    d = 300e-6
    g = _gas()
    w = U / eps
    bo, _ = oracle.drag(cfg, d, 0, eps, w, 873.0, [1.0, 0.0, 0.0])
    beta = bo * (1.0 - eps)
    dpdl = (150.0 * g["mu"] * (1 - eps) ** 2 * U / (eps ** 3 * (psi * d) ** 2) +
            1.75 * g["rho"] * (1 - eps) * U ** 2 / (eps ** 3 * psi * d))
    assert abs(beta * w - eps * dpdl) < 1e-12 * eps * dpdl


def _ganser_cd(Re, psi=1.0):
    """C_D from the oracle's Wen-Yu/Ganser branch at eps_g = 1 (beta/eps_p = 0.75 C_D rho |u-v| / d)."""
    cfg = synth.BedConfig(D=1e6, sphericity=(psi, psi))
    d = 100e-6
    g = _gas()
    slip = Re * g["mu"] / (g["rho"] * d)
    bo, re = oracle.drag(cfg, d, 0, 1.0, slip, 873.0, [1.0, 0.0, 0.0])
    assert abs(re - Re) < 1e-9 * Re
    return bo / (0.75 * g["rho"] * slip / d)


def test_ganser_sphere_against_standard_drag_curve():
    # eq (3-5-3) with psi = 1 (K1 = K2 = 1 away from the bed wall): near the standard sphere
    # curve at Re = 1 (Stokes-Oseen region, 5 %), within the 30 % Ganser's fit keeps at
    # Re = 10..1000, and Newton's law 0.44 at Re = 1e4, 1e5 (10 %). Swapping the two
    # exponents, dropping the 0.1118 term or the 0.4305 term each fails one of these.
    h = handbook_values()
    assert abs(_ganser_cd(1.0) / h["cd_sphere_re1"] - 1) < 0.05
    for Re, key in ((10.0, "cd_sphere_re10"), (100.0, "cd_sphere_re100"), (1000.0, "cd_sphere_re1000")):
        assert abs(_ganser_cd(Re) / h[key] - 1) < 0.30, Re
    for Re in (1e4, 1e5):
        assert abs(_ganser_cd(Re) / h["cd_newton_sphere"] - 1) < 0.10, Re
    # C_D falls monotonically with Re below the drag crisis's precursor minimum (Re ~ 1e3)
    cds = [_ganser_cd(r) for r in np.logspace(-2, 2.7, 40)]
    assert all(b < a for a, b in zip(cds, cds[1:]))


@pytest.mark.parametrize("psi", [0.86, 0.7])
def test_ganser_shape_factors_against_pettyjohn_christiansen(psi):
    # Stokes regime: the drag of an isometric particle over that of the sphere of equal
    # volume is 1/K1, with Pettyjohn & Christiansen's (1948) measured K1 = 0.843 log10(psi/0.065)
    # (3 %). Newton regime: C_D = 5.31 - 4.88 psi (Pettyjohn & Christiansen), so the ratio to
    # the sphere's is (5.31 - 4.88 psi) / 0.43; Ganser's K2 of eq (3-5-5) matches it to 12 %.
    # A dropped K2, or K1 without its square root of psi, fails.
    r_stokes = _ganser_cd(1e-6, psi) / _ganser_cd(1e-6, 1.0)
    k1_pc = 0.843 * math.log10(psi / 0.065)
    assert abs(r_stokes * k1_pc - 1) < 0.03
    r_newton = _ganser_cd(1e7, psi) / _ganser_cd(1e7, 1.0)
    assert abs(r_newton / ((5.31 - 4.88 * psi) / 0.43) - 1) < 0.12


@pytest.mark.parametrize("Re", [30.0, 100.0, 300.0, 1000.0])
def test_gunn_single_sphere_limit_against_ranz_marshall(Re):
    # eqs (3-12), (2-22) at eps_g = 1 are single-sphere correlations; Ranz & Marshall's
    # Nu = 2 + 0.6 Re^(1/2) Pr^(1/3) (and Sh with Sc) agrees with Gunn's to 20 % over
    # 30 <= Re <= 1000. Swapping Gunn's 0.2 and 0.7 exponents misses by a factor of four.
    cfg = synth.BedConfig()
    d = 100e-6
    g = _gas()
    slip = Re * g["mu"] / (g["rho"] * d)
    Nu, h = oracle.heat(cfg, d, 1.0, slip, 873.0, [1.0, 0.0, 0.0])
    Pr = g["cp"] * g["mu"] / g["lam"]
    assert abs(Nu / (2 + 0.6 * Re ** 0.5 * Pr ** (1 / 3)) - 1) < 0.20
    assert abs(h - Nu * g["lam"] / d) < 1e-12 * h
    k = oracle.kinetics(cfg, np.array([1.0, 0, 0, 0]) * 1e-7, 873.0, d, 0, 1.0, slip, 873.0,
                        [1.0, 0.0, 0.0], 1e-5)
    Sc = g["mu"] / (g["rho"] * g["Dm"])
    assert abs(k["Sh"] / (2 + 0.6 * Re ** 0.5 * Sc ** (1 / 3)) - 1) < 0.20
    # gas film of eq (2-20): F = d / (Sh D)
    assert abs(k["F"] - d / (k["Sh"] * g["Dm"])) < 1e-12 * k["F"]


def test_gunn_dense_bed_dependence():
    # eq (3-12) at Re -> 0: Nu = 7 - 10 eps + 5 eps^2, which is 2 at eps = 1 (one sphere in
    # still gas) and rises as the bed closes (Gunn's conduction limit of a packed bed)
    cfg = synth.BedConfig()
    for eps in (0.4, 0.6, 0.8):
        Nu, _ = oracle.heat(cfg, 100e-6, eps, 0.0, 873.0, [1.0, 0.0, 0.0])
        assert abs(Nu - (7 - 10 * eps + 5 * eps * eps)) < 1e-14


def _pore_diffusivity(pore_cm, T=1023.0, Y=(1.0, 0.0, 0.0), p=101325.0):
    """D of eq (2-30) recovered from the oracle's D_eff = D xi / tau."""
    cfg = synth.BedConfig(pore_d_cm=(pore_cm, pore_cm), p0=p)
    k = oracle.kinetics(cfg, np.array([1.0, 0.0, 0.0, 0.0]) * 1e-7, T, 100e-6, 0, 1.0, 0.0, T, list(Y), 1e-5)
    return k["Deff"][0] * cfg.tortuosity / k["xi"][0]


def test_knudsen_coefficient_is_kinetic_theory():
    # eq (2-28), 0.97 r[cm] sqrt(T/M[g/mol]) in m^2/s, is the kinetic-theory Knudsen
    # coefficient (2r/3) sqrt(8 R T / (pi M)) (r in m, M in kg/mol) to 0.1 %. A pore far
    # below the mean free path (lambda/d = 1.013/(p x)/d >= 10) is in the Knudsen regime;
    # a cm-to-m slip (a factor 1e4) fails.
    for T in (773.0, 1023.0, 1273.0):
        pore_cm = 1e-7
        D = _pore_diffusivity(pore_cm, T)
        r = 0.5 * pore_cm * 1e-2
        M = oracle.molar_mass("H2")
        DK = (2 * r / 3) * math.sqrt(8 * 8.314 * T / (math.pi * M))
        assert abs(D / DK - 1) < 1e-3, T


def test_pore_diffusion_regimes():
    # mean free path lambda = 1.013 / (p x) cm (Sec. 2.3): wide pores (lambda/d <= 0.01)
    # diffuse at the molecular coefficient, narrow ones (>= 10) at the Knudsen coefficient,
    # and in between by Bosanquet's series resistance 1/D = 1/D_m + 1/D_K (eq (2-29))
    T = 1023.0
    Dm = _gas(T)["Dm"]
    assert abs(_pore_diffusivity(1e-2, T) / Dm - 1) < 1e-12          # lambda/d = 1e-3
    pore = 3.3e-6                                                      # Table 3: lambda/d ~ 3
    D = _pore_diffusivity(pore, T)
    r = 0.5 * pore * 1e-2
    DK = (2 * r / 3) * math.sqrt(8 * 8.314 * T / (math.pi * oracle.molar_mass("H2")))
    assert abs(D * (1 / Dm + 1 / DK) - 1) < 2e-3
    assert D < min(Dm, DK)


@pytest.mark.parametrize("T", [600.0, 1000.0])
@pytest.mark.parametrize("species,Y", [("H2", (1.0, 0.0, 0.0)), ("N2", (0.0, 0.0, 1.0))])
def test_table_c2_c3_against_tabulated_properties(T, species, Y):
    # Table C2 viscosity and Table C3 conductivity of the pure gases against handbook
    # values (Incropera & DeWitt, Table A.4) to 5 %
    h = handbook_values()
    g = _gas(T, Y)
    key = f"{species}_{int(T)}K"
    assert abs(g["mu"] / h["mu_" + key] - 1) < 0.05
    assert abs(g["lam"] / h["lam_" + key] - 1) < 0.05
