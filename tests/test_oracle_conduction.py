"""Pins of the oracle's contact heat conduction (CPU only): eqs (3-14), (3-15), (3-15-1),
(3-15-2) with the coarse-grained scaling of eqs (3-42)..(3-48-2).

Checks: f(e) of eqs (3-43), (3-44) equals the maximum overlap of a simulated damped binary
collision in units of v/omega_0; the clamp of eq (3-45); the contact radius satisfies the
two spheres' Pythagorean relations; the fluid-lens integral of eq (3-15) against its closed
form for equal spheres and an independent adaptive quadrature (scipy) for unequal ones, the
wall's against its closed form; two equal spheres conduct 2 lambda a dT (Batchelor and
O'Brien's constriction result); pair conduction is antisymmetric, so a bed without walls
conserves the parcels' heat; two touching parcels exchange heat at the rate their conductance
fixes, the heat one gains being the heat the other loses.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth
from tests.helpers import ISOLATED, bed_from_arrays

LMIN = 1.013e-2 / 101325.0   # the gas mean free path of Sec. 2.3 for H2 at 1 atm, m


@pytest.mark.parametrize("e", [0.9, 0.5, 0.2])
def test_restitution_f_is_the_maximum_overlap_of_a_damped_collision(e):
    # head-on collision of two equal parcels with only the contact law acting; the largest
    # overlap reached, in units of v_rel / omega_0 (omega_0 = sqrt(k_n / m*)), is f(e)
    k = 1000.0
    cfg = synth.BedConfig(D=0.02, H=0.02, nx=2, ny=2, nz=2, cg_ratio=4.0, kn=k, restitution=e, mu_s=0.0,
                          flags=ISOLATED)
    d = 100e-6
    r = 0.5 * cfg.cg_ratio * d
    m = 5000.0 * math.pi / 6 * (2 * r) ** 3
    w0 = math.sqrt(k / (0.5 * m))
    tc = math.pi / w0
    cfg.dt = tc / 20000
    v0 = 0.05
    b = bed_from_arrays(cfg, [-r - 1e-9, r + 1e-9], 0.0, 0.01, v=[[v0 / 2, -v0 / 2], [0, 0], [0, 0]], d_real=d)
    o = oracle.Oracle(b)
    worst = 0.0
    for _ in range(20000):       # until the overlap passes its maximum
        o.step(1)
        st = o.state()
        ov = 2 * r - (st[0][1] - st[0][0])
        if worst > 0 and ov < worst:
            break
        worst = max(worst, ov)
    f = oracle.restitution_f(e)
    # the dashpot acts on the half-step velocity, an O(dt) shift of the damping (~3e-5 here)
    assert abs(worst / (v0 / w0) - f) < 1e-4 * f, (worst / (v0 / w0), f)


def test_restitution_f_limits_and_the_clamp_of_eq_3_45():
    assert oracle.restitution_f(1.0) == 1.0
    assert abs(oracle.restitution_f(0.0) - math.exp(-1.0)) < 1e-15
    fs = [oracle.restitution_f(e) for e in np.linspace(0.01, 0.99, 50)]
    assert all(b > a for a, b in zip(fs, fs[1:]))
    # eq (3-45): real below k = 1/(1 - e^2), clamped at 0 above it
    assert abs(oracle.e_cgp(0.9, 2.8) - math.sqrt(1 + 2.8 * (0.81 - 1))) < 1e-15
    assert oracle.e_cgp(0.9, 6.0) == 0.0 and oracle.e_cgp(0.9, 1.0) == 0.9


def _cfg(**kw):
    return synth.BedConfig(cg_ratio=6.0, flags=synth.CONDUCTION, **kw)


@pytest.mark.parametrize("delta", [1e-9, 1e-7, 3e-6, 2e-5])
def test_equal_spheres_against_closed_forms(delta):
    cfg = _cfg()
    R = 360e-6
    d = 2 * R - delta
    lam, lam_g = 2.5, 0.4
    q = oracle.conduction_pair(cfg, R, R, d, 1000.0, 1010.0, lam, lam, lam_g)
    # the contact circle of two equal spheres: R_c^2 = R^2 - (d/2)^2
    assert abs(q["Rc"] - math.sqrt(R * R - 0.25 * d * d)) < 1e-9 * q["Rc"]
    # eq (3-15) with u = sqrt(R^2 - r^2): int u du / (d - 2u) from 0 to (d - L_min)/2
    I = 0.25 * d * math.log(d / LMIN) - 0.25 * (d - LMIN)
    assert abs(q["I"] - I) < 1e-9 * I
    k = cfg.cg_ratio
    sc = k ** 0.75 * math.sqrt(oracle.restitution_f(0.9) / math.exp(-1.0))     # e_CGP clamped at 0
    # two equal spheres conduct 2 lambda a dT through their contact (lambda_e = lambda / 2)
    assert abs(q["Qpp"] - sc * 2 * lam * q["Rc"] * 10.0) < 1e-12 * abs(q["Qpp"])
    assert abs(q["Qpfp"] - k * k * 2 * math.pi * lam_g * 10.0 * I) < 1e-12 * abs(q["Qpfp"])


@pytest.mark.parametrize("Ra,Rb,delta", [(360e-6, 300e-6, 1e-8), (250e-6, 500e-6, 2e-6), (360e-6, 359e-6, 5e-7)])
def test_unequal_spheres_against_independent_quadrature(Ra, Rb, delta):
    from scipy.integrate import quad
    from scipy.optimize import brentq
    d = Ra + Rb - delta
    q = oracle.conduction_pair(_cfg(), Ra, Rb, d, 1000.0, 990.0, 2.0, 3.0, 0.4)
    # the contact circle: both spheres' Pythagorean relations with the centre distance
    xa, xb = math.sqrt(Ra * Ra - q["Rc"] ** 2), math.sqrt(Rb * Rb - q["Rc"] ** 2)
    assert abs(xa + xb - d) < 1e-12 * d
    L = lambda R: d - math.sqrt(Ra * Ra - R * R) - math.sqrt(Rb * Rb - R * R)
    Rin = brentq(lambda R: L(R) - LMIN, q["Rc"], min(Ra, Rb), xtol=1e-22, rtol=1e-15)
    I, _ = quad(lambda R: R / L(R), Rin, min(Ra, Rb), epsabs=0, epsrel=1e-12, limit=400)
    assert abs(q["I"] - I) < 1e-8 * I
    # lambda_e: the two constrictions in series
    sc = 6.0 ** 0.75 * math.sqrt(oracle.restitution_f(0.9) / math.exp(-1.0))
    assert abs(q["Qpp"] - sc * 4 * q["Rc"] * (2.0 * 3.0 / 5.0) * (-10.0)) < 1e-12 * abs(q["Qpp"])


@pytest.mark.parametrize("delta", [1e-9, 1e-6, 2e-5])
def test_wall_against_closed_forms(delta):
    cfg = _cfg(T_in=1100.0, lambda_wall=16.0)
    R = 360e-6
    h = R - delta
    q = oracle.conduction_wall(cfg, R, h, 1000.0, 2.5, 0.4)
    assert abs(q["Rc"] - math.sqrt(R * R - h * h)) < 1e-9 * q["Rc"]
    I = h * math.log(h / LMIN) - (h - LMIN)
    assert abs(q["I"] - I) < 1e-9 * I
    sc = 6.0 ** 0.75 * math.sqrt(oracle.restitution_f(0.9) / math.exp(-1.0))
    lam_e = 2.5 * 16.0 / 18.5
    assert abs(q["Qpp"] - sc * 4 * q["Rc"] * lam_e * 100.0) < 1e-12 * q["Qpp"]
    assert abs(q["Qpfp"] - 36.0 * 2 * math.pi * 0.4 * 100.0 * I) < 1e-12 * q["Qpfp"]


def _lattice(n_side, T, v_scale=0.0, seed=4, kn=1000.0, flags=0):
    cfg = synth.BedConfig(D=0.04, H=0.04, nx=8, ny=8, nz=8, dt=2e-6, cg_ratio=4.0, T_in=1000.0, kn=kn,
                          flags=flags)
    d = 100e-6
    p = cfg.cg_ratio * d * 0.999          # neighbours overlap by 0.1 % of a diameter
    g = (np.arange(n_side) - (n_side - 1) / 2) * p
    X, Y, Z = np.meshgrid(g, g, g + 0.02, indexing="ij")
    n = X.size
    u = synth.uniform(seed, 4 * n).reshape(4, n)
    return bed_from_arrays(cfg, X.ravel(), Y.ravel(), Z.ravel(), v=v_scale * (2 * u[:3] - 1), d_real=d,
                           T=T + 100.0 * u[3], comp=synth.COMP_MIXED)


def test_pair_conduction_conserves_the_parcels_heat():
    # a lattice in the middle of the bed (no wall contact), everything but the contacts and the
    # conduction switched off: the conduction terms of all parcels sum to zero
    b = _lattice(8, 950.0, v_scale=0.02, flags=ISOLATED | synth.CONDUCTION)
    o = oracle.Oracle(b)
    for _ in range(3):
        o.step(5)
        q = o.diag()[oracle.D_QCOND]
        assert np.count_nonzero(q) > 0.9 * b.n
        assert abs(q.sum()) < 1e-12 * np.abs(q).sum()
    cnt, partner, _ = o.contacts()
    assert cnt.mean() > 3
    assert (partner[np.arange(partner.shape[1])[None, :] < cnt[:, None]] >= 0).all()   # no wall contact


def test_two_touching_parcels_exchange_heat_at_their_conductance():
    # two equal parcels held in place (tiny spring, no other forces), 20 K apart: one explicit
    # step moves the colder one by dt G dT / (m c_p), G the pair conductance of eqs (3-14),
    # (3-15), (3-46), (3-48), and the hotter one by the same heat
    cfg = synth.BedConfig(D=0.04, H=0.04, nx=4, ny=4, nz=4, dt=1e-4, cg_ratio=4.0, kn=1e-6,
                          flags=ISOLATED | synth.CONDUCTION, T_in=1000.0)
    d = 100e-6
    r = 0.5 * cfg.cg_ratio * d
    gap = 2 * r - 1e-7
    b = bed_from_arrays(cfg, [-gap / 2, gap / 2], 0.0, 0.02, d_real=d, T=[990.0, 1010.0])
    o = oracle.Oracle(b)
    lam_g = oracle.gas_props(cfg, 1000.0, list(cfg.Y_in))["lam"]
    q = oracle.conduction_pair(cfg, r, r, gap, 990.0, 1010.0, cfg.lambda_p[0], cfg.lambda_p[0], lam_g)
    G = (q["Qpp"] + q["Qpfp"]) / 20.0
    m = b.m0[:, 0].sum()
    o.step(1)
    st = o.state()
    # the heat capacity at the start of the step (eq (3-9) with Table C1)
    cp = sum(b.m0[z, 0] / m * oracle.cp(3 + z, 990.0) for z in range(4))
    assert abs((st[9][0] - 990.0) - cfg.dt * G * 20.0 / (m * cp)) < 1e-10
    cp1 = sum(b.m0[z, 1] / m * oracle.cp(3 + z, 1010.0) for z in range(4))
    heat0, heat1 = m * cp * (st[9][0] - 990.0), m * cp1 * (st[9][1] - 1010.0)
    assert abs(heat0 + heat1) < 1e-12 * abs(heat0)          # what one gains, the other loses
