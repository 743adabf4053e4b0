"""Pins of the oracle's particle radiation, eqs (3-16), (3-17), (3-51) (CPU only).

* The neighbourhood mean T_se of eq (3-17) against brute force over all parcel pairs:
  sphere of radius 1.5 d_CGP around each parcel, the parcel itself included, the cell's
  eps_g and T_g, the temperatures before the step.
* An isolated parcel heated by radiation from the gas around it: the time the oracle takes
  to reach its final temperature equals the closed-form time of the grey-body law
  m c_p(T) dT/dt = k^3 sigma eta pi d^2 (T_se^4 - T^4), integrated by quadrature with the
  paper's printed sigma and emissivity (within the O(dt) error of explicit Euler).
* Radiation off: no T_se, no Q_rad, and the same trajectory as before the switch existed
  (the temperature update with Q_rad = 0).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2311_03908_gb300 import synth
from tests.helpers import ISOLATED, bed_from_arrays, paper_values


def _packed(flags, seed=5, n=400):
    b = synth.small_packed(seed=seed, n=n, v_scale=0.0, flags=flags)
    rng = np.random.default_rng(seed)
    b.T = 900.0 + 200.0 * rng.random(b.x.size)   # every parcel its own temperature
    return b


def test_tse_matches_brute_force_neighbourhood():
    flags = synth.NO_GRAVITY | synth.RADIATION
    b = _packed(flags)
    o = oracle.Oracle(b)
    gas0 = o.gas().copy()
    o.step(1)   # v = 0 and a = 0: the drift of the first step leaves the positions in place
    dg = o.diag()
    cfg = b.beds[0]
    R = 1.5 * cfg.cg_ratio * b.d_real
    dx = b.x[None, :] - b.x[:, None]
    dy = b.y[None, :] - b.y[:, None]
    dz = b.z[None, :] - b.z[:, None]
    inside = (dx * dx + dy * dy) + dz * dz < (R * R)[:, None]
    cnt = inside.sum(axis=1)
    assert cnt.min() >= 1 and cnt.max() > 5          # self always; packed: several neighbours
    assert (cnt < b.x.size).all()                    # a neighbourhood, not the bed
    cell = dg[oracle.D_CELL].astype(np.int64)
    eps, Tg = gas0[cell, oracle.G_EPS], gas0[cell, oracle.G_T]
    tse = eps * Tg + (1.0 - eps) * (inside * b.T[None, :]).sum(axis=1) / cnt
    assert np.abs(dg[oracle.D_TSE] - tse).max() < 1e-12 * tse.max()
    # the radiation of the parcel itself: the grey-body law with the printed constants
    pv = paper_values()
    q = cfg.cg_ratio ** 3 * pv["stefan_boltzmann"] * pv["emissivity"] * math.pi * b.d_real ** 2 * \
        (tse ** 4 - b.T ** 4)
    assert np.abs(dg[oracle.D_QRAD] - q).max() < 1e-9 * np.abs(q).max()


def test_isolated_parcel_relaxation_time():
    pv = paper_values()
    cfg = synth.BedConfig(U_in=0.0, T_in=1200.0, flags=ISOLATED | synth.RADIATION,
                          emissivity=pv["emissivity"])
    d, T0, nsteps = 100e-6, 900.0, 2000
    b = bed_from_arrays(cfg, [0.001], 0.002, 0.1, d_real=d, T=T0)
    o = oracle.Oracle(b)
    o.step(nsteps)
    T1 = o.state()[oracle.S_T, 0]
    assert T1 > T0 + 5.0                                            # heated noticeably
    cell = int(o.diag()[oracle.D_CELL, 0])
    eps, Tg = o.gas()[cell, oracle.G_EPS], o.gas()[cell, oracle.G_T]
    assert Tg == 1200.0 and 0.99 < eps < 1.0
    m = b.m0[:, 0].sum()
    k3A = cfg.cg_ratio ** 3 * math.pi * d ** 2
    sigma = pv["stefan_boltzmann"]

    def dt_dT(T):   # dt/dT of the grey-body law; the parcel is alone in its sphere (n = 1)
        te = eps * Tg + (1.0 - eps) * T
        return m * oracle.cp(3, T) / (k3A * sigma * pv["emissivity"] * (te ** 4 - T ** 4))

    t, _ = integrate.quad(dt_dT, T0, T1, epsabs=0.0, epsrel=1e-12)
    assert abs(t - nsteps * cfg.dt) < 1e-4 * nsteps * cfg.dt


def test_radiation_off_leaves_no_trace():
    b = _packed(synth.NO_GRAVITY)
    o = oracle.Oracle(b)
    o.step(3)
    dg = o.diag()
    assert not dg[oracle.D_TSE].any() and not dg[oracle.D_QRAD].any()


def test_adjoint_refuses_radiation():
    b = _packed(synth.RADIATION, n=50)
    o = oracle.Oracle(b)
    with pytest.raises(ValueError):
        o.adjoint(2)
