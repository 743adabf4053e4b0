"""Pins of the oracle's USCM kinetics (Sec. 2 of the paper), CPU only.

The oracle solves the resistance network by Kirchhoff's voltage law (a 3x3 loop system);
these tests check it against the paper's printed closed forms (with the corrected W),
against an independent nodal (current-law) solve, against the analytic chemical-control
law 1-(1-f)^(1/3) = kappa t, against oxygen and iron mass balance, and against the
printed q values, densities, resistance ordering and film resistance.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth
from tests.helpers import bed_from_arrays, paper_values

PV = paper_values()

RG = 8.314


def test_printed_q_values():
    # Sec. 2.3: q_{m,h} = 0.9666, q_{w,m} = 0.9309, q_{Fe,w} = 0.7773 (eq (2-36))
    M = {s: oracle.molar_mass(s) for s in oracle.SPECIES}
    assert round(2 * M["Fe3O4"] / (3 * M["Fe2O3"]), 4) == PV["q_m_h"]
    assert round(3 * M["FeO"] / M["Fe3O4"], 4) == PV["q_w_m"]
    assert round(M["Fe"] / M["FeO"], 4) == PV["q_Fe_w"]


def test_layer_porosity_chain_against_table3():
    # Bed II: initial porosity 0.34 and true density 5300 give an effective density of
    # about 3500 kg/m3 (Table 3); recover it from the magnetite-layer porosity and the
    # printed q values.
    cfg = synth.BedConfig()
    xi = oracle.layer_porosity(cfg, synth.ORE_HEMATITE)
    q1, q2, q3 = PV["q_m_h"], PV["q_w_m"], PV["q_Fe_w"]
    rho_eff_h = (1 - xi[0]) * 5180.0 / q1
    assert abs(rho_eff_h - PV["rho_eff_bed2"]) < 0.002 * PV["rho_eff_bed2"]
    assert abs((1 - xi[1]) * 5390.0 - rho_eff_h * q1 * q2) < 1.0
    assert abs((1 - xi[2]) * 7900.0 - rho_eff_h * q1 * q2 * q3) < 1.0
    # final (iron) porosity of hematite about 0.65 in the paper's run (Sec. 5.2.2): loose
    assert abs(xi[2] - PV["porosity_Fe_final_hematite"]) < 0.1 * PV["porosity_Fe_final_hematite"]


def _pure_bed(comp, ore):
    cfg = synth.BedConfig(D=0.05, H=0.05, nx=1, ny=1, nz=1)
    return bed_from_arrays(cfg, [0.0], 0.0, 0.01, comp=comp, ore=ore)


@pytest.mark.parametrize("comp,ore,expected", [
    ((1, 0, 0, 0), 0, 0.0),
    ((0, 1, 0, 0), 0, (1.5 - 4 / 3) / 1.5),
    ((0, 0, 1, 0), 0, (1.5 - 1.0) / 1.5),
    ((0, 0, 0, 1), 0, 1.0),
    ((0, 1, 0, 0), 1, 0.0),
    ((0, 0, 1, 0), 1, (4 / 3 - 1.0) / (4 / 3)),
    ((0, 0, 0, 1), 1, 1.0),
])
def test_reduction_degree_is_oxygen_removed(comp, ore, expected):
    # eqs (2-18), (2-19): the overall degree equals the fraction of lattice oxygen removed
    # (O/Fe = 1.5, 4/3, 1, 0 for Fe2O3, Fe3O4, FeO, Fe)
    o = oracle.Oracle(_pure_bed(comp, ore))
    mean, oxy, per = o.reduction_degree()
    assert abs(per[0] - expected) < 1e-14
    assert abs(oxy[0] - expected) < 1e-14


def _printed_v(A, B, F):
    """The paper's eqs (2-2)..(2-10) with W replaced by the three-reaction determinant."""
    Ahm, Amw, AwFe = A
    Bm, Bw, BFe = B
    S = BFe + F
    W = (Ahm + Bm) * (AwFe * (Amw + Bw + S) + (Amw + Bw) * S) + Amw * (AwFe * (Bw + S) + Bw * S)
    v = np.zeros((3, 3))
    v[0, 0] = (AwFe * (Amw + Bw + BFe + F) + (BFe + F) * (Amw + Bw)) / W       # (2-2)
    v[0, 1] = -(AwFe * (Bw + BFe + F) + Bw * (BFe + F)) / W                     # (2-3)
    v[0, 2] = -Amw * (BFe + F) / W                                              # (2-4)
    v[1, 0] = -(Bw * (AwFe + BFe + F) + AwFe * (BFe + F)) / W                   # (2-5)
    v[1, 1] = ((Ahm + Bm + Bw) * (AwFe + BFe + F) + AwFe * (BFe + F)) / W       # (2-6)
    v[1, 2] = -(Ahm + Bm) * (BFe + F) / W                                       # (2-7)
    v[2, 0] = -Amw * (BFe + F) / W                                              # (2-8)
    v[2, 1] = -(Ahm + Bm) * (BFe + F) / W                                       # (2-9)
    v[2, 2] = ((Ahm + Bm) * (Amw + Bw + BFe + F) + Amw * (Bw + BFe + F)) / W    # (2-10)
    return v


def _nodal(A, B, F, active, x, xeq):
    """Independent solve by Kirchhoff's current law on the node potentials of Fig. 2(a):
    bulk -> F -> surface -> B_Fe -> node w|Fe -> B_w -> node m|w -> B_m -> node h|m; each
    interface node drains through A_kl to its equilibrium potential."""
    Ahm, Amw, AwFe = A
    Bm, Bw, BFe = B
    # unknown potentials: c3 (w|Fe), c2 (m|w), c1 (h|m); series F + B_Fe from the bulk
    Ra = F + BFe
    G = np.zeros((3, 3))
    rhs = np.zeros(3)
    g3 = 1 / AwFe if active[2] else 0.0
    g2 = 1 / Amw if active[1] else 0.0
    g1 = 1 / Ahm if active[0] else 0.0
    # node c3
    G[0, 0] = 1 / Ra + g3 + 1 / Bw
    G[0, 1] = -1 / Bw
    rhs[0] = x / Ra + g3 * xeq[2]
    # node c2
    G[1, 0] = -1 / Bw
    G[1, 1] = 1 / Bw + g2 + 1 / Bm
    G[1, 2] = -1 / Bm
    rhs[1] = g2 * xeq[1]
    # node c1
    G[2, 1] = -1 / Bm
    G[2, 2] = 1 / Bm + g1
    rhs[2] = g1 * xeq[0]
    c3, c2, c1 = np.linalg.solve(G, rhs)
    return np.array([g1 * (c1 - xeq[0]), g2 * (c2 - xeq[1]), g3 * (c3 - xeq[2])])


@pytest.mark.parametrize("seed", range(6))
def test_network_matches_printed_closed_form_and_nodal_solve(seed):
    u = synth.uniform(100 + seed, 9)
    A = 10 ** (1 + 3 * u[0:3])
    B = 10 ** (-2 + 2 * u[3:6])
    F = 10 ** (-2 + u[6])
    xeq = np.sort(u[7:9] * 0.3).tolist()
    xeq = [1e-5, xeq[0], xeq[1]]
    x = 0.95
    J, v, act = oracle.network(A, B, F, [1, 1, 1], x, xeq)
    assert list(act) == [1, 1, 1]
    vp = _printed_v(A, B, F)
    assert np.allclose(v, vp, rtol=1e-12, atol=0)
    assert np.allclose(J, _nodal(A, B, F, [1, 1, 1], x, xeq), rtol=1e-10, atol=0)


def test_corrected_W_is_the_loop_determinant():
    sympy = pytest.importorskip("sympy")
    Ahm, Amw, AwFe, Bm, Bw, BFe, F = sympy.symbols("A_hm A_mw A_wFe B_m B_w B_Fe F", positive=True)
    S = F + BFe
    R = sympy.Matrix([[S + Bw + Bm + Ahm, S + Bw, S], [S + Bw, S + Bw + Amw, S], [S, S, S + AwFe]])
    W = (Ahm + Bm) * (AwFe * (Amw + Bw + S) + (Amw + Bw) * S) + Amw * (AwFe * (Bw + S) + Bw * S)
    assert sympy.expand(R.det() - W) == 0
    assert len(sympy.expand(W).args) == 21
    # the printed eq (2-11) is the two-reaction W of eq (ea2), not the determinant
    W_printed = AwFe * (Amw + Bw + BFe + F) + (Amw + Bw) * (BFe + F)
    assert sympy.expand(W_printed - W) != 0


def test_magnetite_network_eq_ea2():
    # Fig. 4(a): only m->w and w->Fe; total rate v2 (x - x_mw) + v3 (x - x_wFe) with
    # v2 = A_wFe / W, v3 = (A_mw + B_w) / W, W of eq (ea2)
    A = [0.0, 300.0, 80.0]
    B = [0.0, 0.7, 0.2]
    F = 0.05
    xeq = [0.0, 0.4, 0.6]
    x = 0.9
    J, v, act = oracle.network(A, B, F, [0, 1, 1], x, xeq)
    W = A[2] * (A[1] + B[1] + B[2] + F) + (A[1] + B[1]) * (B[2] + F)
    v2 = A[2] / W
    v3 = (A[1] + B[1]) / W
    assert list(act) == [0, 1, 1]
    assert abs(J.sum() - (v2 * (x - xeq[1]) + v3 * (x - xeq[2]))) < 1e-14
    assert J[0] == 0.0


@pytest.mark.parametrize("BFe", [0.0, 0.3])
def test_two_reaction_networks_eq_eb2_eb3(BFe):
    # Fig. 2(f),(g): h->m and m->w only; v1 = A_mw / W, v2 = (A_hm + B_m) / W
    A = [50.0, 400.0, 0.0]
    B = [0.2, 0.6, BFe]
    F = 0.04
    xeq = [1e-5, 0.5, 0.0]
    x = 0.7
    J, v, act = oracle.network(A, B, F, [1, 1, 0], x, xeq)
    W = A[1] * (A[0] + B[0] + B[1] + B[2] + F) + (A[0] + B[0]) * (B[1] + B[2] + F)
    v1 = A[1] / W
    v2 = (A[0] + B[0]) / W
    assert abs(J.sum() - (v1 * (x - xeq[0]) + v2 * (x - xeq[1]))) < 1e-14


@pytest.mark.parametrize("r,Bsum", [(0, 0.3), (1, 0.9), (2, 0.2)])
def test_single_reaction_networks(r, Bsum):
    # Fig. 2(b)-(e), Fig. 4(b)-(d): v = 1 / (A + sum of B + F)
    A = [60.0, 70.0, 80.0]
    B = [0.1, 0.5, 0.3] if r == 0 else ([0.0, 0.6, 0.3] if r == 1 else [0.0, 0.0, 0.2])
    F = 0.05
    xeq = [0.0, 0.3, 0.5]
    act = [0, 0, 0]
    act[r] = 1
    J, v, ao = oracle.network(A, B, F, act, 0.9, xeq)
    Bpath = [B[0] + B[1] + B[2], B[1] + B[2], B[2]][r]
    assert abs(J[r] - (0.9 - xeq[r]) / (A[r] + Bpath + F)) < 1e-15


def test_negative_flux_branch_is_removed():
    # a strong h->m sink pulls the outer node below the w->Fe equilibrium: that flux would
    # be negative, so w->Fe (irreversible) is removed and the rest solved again
    A = [1.0, 200.0, 5.0]
    B = [1e-3, 1e-3, 1e-3]
    F = 20.0
    xeq = [0.0, 0.2, 0.8]
    x = 1.0
    Jfull = _nodal(A, B, F, [1, 1, 1], x, xeq)
    assert Jfull[2] < 0
    J, v, act = oracle.network(A, B, F, [1, 1, 1], x, xeq)
    assert act[2] == 0 and J[2] == 0.0
    # what remains is exactly the nodal solution of the reduced network
    assert np.allclose(J, _nodal(A, B, F, act, x, xeq), rtol=1e-10, atol=1e-15)
    J2, _, _ = oracle.network(A, B, F, list(act), x, xeq)
    assert np.array_equal(J, J2)
    assert (J >= 0).all()


def test_chemical_control_law():
    # R1 only, no film and no product-layer resistance, constant x_H2 = 1 and T:
    # 1 - (1 - f_h)^(1/3) = kappa t with kappa = A_p p k_r (1+K)(x - x_eq)/(R T K n_h0)
    T = 1073.0
    dt = 1e-5
    flags = (synth.NO_FILM | synth.NO_LAYER | synth.NO_GRAVITY | synth.NO_DRAG | synth.NO_HEAT |
             synth.NO_RXN_HEAT | synth.NO_GAS_UPDATE | synth.NO_CONTACTS)
    cfg = synth.BedConfig(D=0.05, H=0.05, nx=1, ny=1, nz=1, dt=dt, T_in=T, Y_in=(1.0, 0.0, 0.0),
                          k0=(10.0, 0.0, 0.0), Ea=(42400.0, 19300.0, 33880.0), flags=flags)
    d = 100e-6
    b = bed_from_arrays(cfg, [0.0], 0.0, 0.02, d_real=d, T=T)
    o = oracle.Oracle(b)
    Mh = oracle.molar_mass("Fe2O3")
    n_h0 = 5000.0 * math.pi / 6.0 * d ** 3 / Mh
    K = math.exp(1433.4 / T + 9.08)
    xeq = 1.0 / (K + 1.0)
    kr = 10.0 * math.exp(-42400.0 / (RG * T))
    kappa = math.pi * d * d * 101325.0 * kr * (1 + K) * (1.0 - xeq) / (RG * T * K * n_h0)
    for k in range(1, 6):
        o.step(6000)
        t = 6000 * k * dt
        fh = 9.0 * o.reduction_degree()[2][0]   # pure Fe2O3 -> Fe3O4: f_ov = f_h / 9
        lhs = 1.0 - (1.0 - fh) ** (1.0 / 3.0)
        assert abs(lhs - kappa * t) < 1e-4 * kappa * t
    assert fh > 0.3


def test_oxygen_and_iron_balance():
    b = synth.small_packed(seed=11, n=1500, T0=1073.0, v_scale=0.1)
    b.beds[0].k0 = synth.HEMATITE_FIT[0]
    b.beds[0].Ea = synth.HEMATITE_FIT[1]
    comp = np.array(synth.COMP_MIXED)
    mass = b.m0.sum(axis=0)
    b.m0 = mass[None, :] * comp[:, None]
    o = oracle.Oracle(b)
    M = np.array([oracle.molar_mass(s) for s in ("Fe2O3", "Fe3O4", "FeO", "Fe")])
    Mh2, Mh2o = oracle.molar_mass("H2"), oracle.molar_mass("H2O")

    def moles(st):
        n = st[oracle.S_M:oracle.S_M + 4] / M[:, None]
        fe = 2 * n[0] + 3 * n[1] + n[2] + n[3]
        ox = 3 * n[0] + 4 * n[1] + n[2]
        return fe, ox

    fe0, ox0 = moles(o.state())
    h2o = 0.0
    h2 = 0.0
    dt = b.beds[0].dt
    for _ in range(40):
        o.step(1)
        dep = o.deposits()
        h2o += dep[:, 2].sum() / Mh2o * dt
        h2 += dep[:, 1].sum() / Mh2 * dt
    fe1, ox1 = moles(o.state())
    assert np.allclose(fe1, fe0, rtol=1e-13, atol=0)
    removed = (ox0 - ox1).sum()
    assert removed > 0
    assert abs(h2o - removed) < 1e-9 * removed
    assert abs(-h2 - removed) < 1e-9 * removed


def _bed1_gas():
    xh, xn = 0.7, 0.3
    M = xh * 2.016 + xn * 28.014
    return [xh * 2.016 / M, 0.0, xn * 28.014 / M]


def test_bed1_film_resistance_loose():
    # Sec. 5.1.1: mean gas-film resistance 0.048 s/m for Bed I (magnetite, 943 K, 70% H2);
    # at eps_g = 0.5 and the superficial velocity 0.18 m/s the oracle is within 30 %
    Y = _bed1_gas()
    cfg = synth.BedConfig(T_in=943.0, Y_in=tuple(Y), k0=synth.MAGNETITE_FIT[0], Ea=synth.MAGNETITE_FIT[1])
    k = oracle.kinetics(cfg, np.array([0, 0.6994, 0.3006, 0]) * 1e-7, 943.0, 100e-6, 1, 0.5,
                        0.18 / 0.5, 943.0, Y, 1e-5)
    assert abs(k["F"] - PV["film_resistance_bed1"]) < 0.3 * PV["film_resistance_bed1"]


def test_bed1_resistance_ordering_loose():
    # Sec. 5.1.1: A_mw > A_wFe > B_w > B_Fe > F during magnetite reduction
    Y = _bed1_gas()
    cfg = synth.BedConfig(T_in=943.0, Y_in=tuple(Y), k0=synth.MAGNETITE_FIT[0], Ea=synth.MAGNETITE_FIT[1])
    k = oracle.kinetics(cfg, np.array([0, 0.4, 0.4, 0.2]) * 1e-7, 943.0, 100e-6, 1, 0.5, 0.36,
                        943.0, Y, 1e-5)
    A, B, F = k["A"], k["B"], k["F"]
    assert A[1] > A[2] > B[1] > B[2] > F > 0
