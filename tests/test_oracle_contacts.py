"""Pins of the oracle's pair search, contact law and time integration (CPU only).

Each check compares the oracle with something other than itself: brute force, the
closed-form linear spring-dashpot collision, energy conservation, exact free fall under
kick-drift-kick, and the textbook sliding-to-rolling transition of a sphere (v = 5/7 v0).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth
from tests.helpers import ISOLATED, bed_from_arrays


def _cloud(seed, n, box, rmin, rmax):
    u = synth.uniform(seed, 4 * n).reshape(4, n)
    return u[0] * box, u[1] * box, u[2] * box, rmin + (rmax - rmin) * u[3]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pairs_cells_equal_bruteforce(seed):
    x, y, z, r = _cloud(seed, 1500, 0.01, 1e-4, 3e-4)
    bf = oracle.pairs_bruteforce(x, y, z, r)
    cl = oracle.pairs_cells(x, y, z, r)
    assert len(bf) > 100
    assert np.array_equal(bf, cl)


def test_pairs_touching_lattice_strict():
    # spheres on a lattice at exactly twice their radius: d^2 == (2r)^2 is no contact
    r = 0.25
    g = np.arange(6, dtype=float)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = X.ravel() * 0.5, Y.ravel() * 0.5, Z.ravel() * 0.5
    rr = np.full(x.size, r)
    assert len(oracle.pairs_bruteforce(x, y, z, rr)) == 0
    assert len(oracle.pairs_cells(x, y, z, rr)) == 0
    # a hair closer: every lattice neighbour becomes a pair (3 * 6 * 6 * 5 = 540)
    rr2 = np.full(x.size, r * (1 + 1e-12))
    assert len(oracle.pairs_bruteforce(x, y, z, rr2)) == 540
    assert np.array_equal(oracle.pairs_bruteforce(x, y, z, rr2), oracle.pairs_cells(x, y, z, rr2))


def _two_body_cfg(e, dt, mu=0.3):
    return synth.BedConfig(D=0.02, H=0.02, nx=1, ny=1, nz=1, dt=dt, restitution=e, mu_s=mu,
                           cg_ratio=4.0, flags=ISOLATED)


def _tc(cfg, mstar):
    le = math.log(cfg.restitution)
    eta = -2 * le * math.sqrt(mstar * cfg.kn / (math.pi ** 2 + le * le))
    return math.pi / math.sqrt(cfg.kn / mstar - (eta / (2 * mstar)) ** 2)


def test_binary_collision_restitution_and_contact_time():
    d_real = 100e-6
    r = 0.5 * 4.0 * d_real
    m = 5000.0 * math.pi / 6.0 * (2 * r) ** 3
    cfg0 = _two_body_cfg(0.9, 1.0)
    tc = _tc(cfg0, 0.5 * m)
    dt = tc / 2000.0
    cfg = _two_body_cfg(0.9, dt)
    v0 = 0.1
    gap = 3 * v0 * dt
    x = np.array([-r - gap, r + gap])
    b = bed_from_arrays(cfg, x, 0.0, 0.01, v=[[v0, -v0], [0, 0], [0, 0]], d_real=d_real)
    o = oracle.Oracle(b)
    in_contact = 0
    started = False
    for _ in range(6000):
        o.step(1)
        c = o.diag()[oracle.D_NCONTACT]
        if c[0] > 0:
            in_contact += 1
            started = True
        elif started:
            break
    st = o.state()
    v_after = st[oracle.S_VX, 1] - st[oracle.S_VX, 0]
    e_meas = v_after / (2 * v0)
    assert abs(e_meas - 0.9) < 1e-3 * 0.9
    assert abs(in_contact * dt - tc) < 1e-3 * tc
    # momentum conserved exactly up to rounding
    assert abs(st[oracle.S_VX, 0] + st[oracle.S_VX, 1]) < 1e-12


def test_wall_bounce_restitution():
    d_real = 100e-6
    r = 0.5 * 4.0 * d_real
    m = 5000.0 * math.pi / 6.0 * (2 * r) ** 3
    tc = _tc(_two_body_cfg(0.8, 1.0), m)
    dt = tc / 2000.0
    cfg = _two_body_cfg(0.8, dt)
    v0 = 0.2
    b = bed_from_arrays(cfg, 0.0, 0.0, r + 2 * v0 * dt, v=[[0], [0], [-v0]], d_real=d_real)
    o = oracle.Oracle(b)
    for _ in range(8000):
        o.step(1)
        if o.state()[oracle.S_VZ, 0] > 0 and o.diag()[oracle.D_NCONTACT, 0] == 0:
            break
    vz = o.state()[oracle.S_VZ, 0]
    assert abs(vz / v0 - 0.8) < 1e-3 * 0.8


def test_free_fall_exact():
    dt = 1e-4
    cfg = synth.BedConfig(D=0.05, H=1.0, nx=1, ny=1, nz=4, dt=dt,
                          flags=ISOLATED & ~synth.NO_GRAVITY)
    z0, vz0 = 0.9, 0.3
    b = bed_from_arrays(cfg, 0.0, 0.0, z0, v=[[0], [0], [vz0]])
    o = oracle.Oracle(b)
    n = 300
    o.step(n)
    st = o.state()
    t = n * dt
    assert abs(st[oracle.S_Z, 0] - (z0 + vz0 * t - 0.5 * 9.81 * t * t)) < 1e-12
    assert abs(st[oracle.S_VZ, 0] - (vz0 - 9.81 * t)) < 1e-12


def test_energy_conserved_elastic_frictionless():
    # e = 1 and mu = 0: kinetic plus elastic energy (pairs and walls) is conserved
    d_real = 100e-6
    r = 0.5 * 4.0 * d_real
    m = 5000.0 * math.pi / 6.0 * (2 * r) ** 3
    tc = _tc(_two_body_cfg(0.999999, 1.0), 0.5 * m)
    dt = tc / 200.0
    cfg = synth.BedConfig(D=0.004, H=0.004, nx=1, ny=1, nz=1, dt=dt, restitution=1.0, mu_s=0.0,
                          cg_ratio=4.0, flags=ISOLATED)
    # 12 spheres on a jittered 3x2x2 lattice inside the small cylinder
    pts = [(i * 0.9e-3 - 0.9e-3, j * 0.9e-3 - 0.45e-3, 1.2e-3 + k * 0.9e-3)
           for i in range(3) for j in range(2) for k in range(2)]
    x, y, z = (np.array(a) for a in zip(*pts))
    u = synth.uniform(5, 3 * x.size).reshape(3, -1)
    v = 0.4 * (2 * u - 1)
    b = bed_from_arrays(cfg, x, y, z, v=v, d_real=d_real)
    o = oracle.Oracle(b)

    def energy():
        st = o.state()
        ke = 0.5 * m * (st[oracle.S_VX] ** 2 + st[oracle.S_VY] ** 2 + st[oracle.S_VZ] ** 2).sum()
        P = st[oracle.S_X:oracle.S_Z + 1].T
        pe = 0.0
        for i in range(len(P)):
            for j in range(i + 1, len(P)):
                d = np.linalg.norm(P[i] - P[j])
                if d < 2 * r:
                    pe += 0.5 * cfg.kn * (2 * r - d) ** 2
            dist, _ = oracle.wall_distance(cfg, *P[i])
            for dd in dist:
                if dd < r:
                    pe += 0.5 * cfg.kn * (r - dd) ** 2
        return ke + pe

    e0 = energy()
    ncontacts = 0
    worst = 0.0
    for _ in range(100):
        o.step(1000)
        ncontacts += int(o.diag()[oracle.D_NCONTACT].sum() > 0)
        worst = max(worst, abs(energy() - e0) / e0)
    assert worst < 1e-4
    assert ncontacts > 0


def test_sliding_sphere_reaches_five_sevenths():
    # a sphere launched along the floor slides with |F_t| = mu |F_n| until it rolls at 5/7 v0
    d_real = 100e-6
    r = 0.5 * 4.0 * d_real
    dt = 2e-7
    cfg = synth.BedConfig(D=0.05, H=0.01, nx=1, ny=1, nz=1, dt=dt, restitution=0.5, mu_s=0.3,
                          cg_ratio=4.0, flags=ISOLATED & ~synth.NO_GRAVITY)
    v0 = 0.05
    b = bed_from_arrays(cfg, -0.01, 0.0, r - 9.81 * 1.676e-7 / 1000.0, v=[[v0], [0], [0]],
                        d_real=d_real)
    o = oracle.Oracle(b)
    saturated = []
    for k in range(500):
        o.step(100)
        dg = o.diag()
        ft = math.hypot(dg[oracle.D_FC, 0], dg[oracle.D_FC + 1, 0])
        fn = abs(dg[oracle.D_FC + 2, 0])
        st = o.state()
        slip = st[oracle.S_VX, 0] + r * st[oracle.S_WY, 0] * -1.0  # contact-point velocity
        if 10 < k < 40 and abs(slip) > 1e-3:
            saturated.append(ft / fn)
    st = o.state()
    assert saturated and max(abs(s - 0.3) for s in saturated) < 1e-9
    t_slip = 2 * v0 / (7 * 0.3 * 9.81)
    assert 500 * 100 * dt > 1.5 * t_slip
    assert abs(st[oracle.S_VX, 0] - 5.0 / 7.0 * v0) < 0.01 * v0
