"""Pin of the oracle's adjoint reference: forward-mode dual numbers against central
finite differences of the same frozen-position drag-heat-reaction map (CPU only)."""
import numpy as np

import oracle
from paper_2311_03908_gb300 import synth


def test_dual_gradient_matches_central_differences():
    b = synth.config_adjoint_64k(n=300)
    o = oracle.Oracle(b)
    J0, _ = o.adjoint(200, mode=0)
    Jf, gf = o.adjoint(200, mode=1, rel=1e-6)
    Jd, gd = o.adjoint(200, mode=2)
    assert J0 > 0 and J0 == Jf == Jd
    # all three reactions run from t = 0 in the mixed ore, so every component is non-zero
    assert np.all(np.abs(gd) > 0)
    assert np.allclose(gd, gf, rtol=1e-4, atol=0)
    # k0 raises the rate, Ea lowers it
    assert np.all(gd[:3] > 0) and np.all(gd[3:] < 0)


def test_full_step_is_deterministic():
    b = synth.small_packed(seed=3, n=800, v_scale=0.2)
    o1 = oracle.Oracle(b)
    o2 = oracle.Oracle(b)
    o1.step(15)
    o2.step(15)
    assert np.array_equal(o1.state(), o2.state())
    assert np.array_equal(o1.gas(), o2.gas())


def test_observed_curves_agree_with_separate_horizons():
    # observing the map after 100, 200 and 300 sub-steps gives the plain J of each horizon,
    # and the dual gradient of a weighted sum of observations is that sum of the horizons'
    # gradients (and central differences of the weighted sum)
    b = synth.config_adjoint_64k(n=300)
    o = oracle.Oracle(b)
    w = np.array([[0.5], [-1.25], [2.0]])
    Jo, go = o.adjoint_obs(300, [100, 200, 300], weights=w, mode=2)
    parts = [o.adjoint(h, mode=2) for h in (100, 200, 300)]
    assert np.allclose(Jo[:, 0], [p[0] for p in parts], rtol=1e-14, atol=0)
    expect = sum(wk * p[1] for wk, p in zip(w[:, 0], parts))
    assert np.allclose(go, expect, rtol=1e-12, atol=0)
    # central differences of the weighted sum in each parameter
    k0, Ea = np.array(b.beds[0].k0), np.array(b.beds[0].Ea)
    th = np.concatenate([k0, Ea])
    for q in range(6):
        h = 1e-6 * th[q]
        vals = []
        for sgn in (1, -1):
            t = th.copy()
            t[q] += sgn * h
            o.set_kinetics(t[:3], t[3:])
            J, _ = o.adjoint_obs(300, [100, 200, 300])
            vals.append(float((w[:, 0] * J[:, 0]).sum()))
        o.set_kinetics(k0, Ea)
        assert abs((vals[0] - vals[1]) / (2 * h) - go[q]) < 1e-4 * abs(go[q]), q


def test_observed_curves_per_bed():
    # two beds at different temperatures: the bed means separate, the hotter reduces faster
    parts = [synth.config_adjoint_64k(n=150, seed=11), synth.config_adjoint_64k(n=150, seed=12)]
    parts[0].beds[0].T_in, parts[1].beds[0].T_in = 873.0, 1073.0
    parts[0].T[:] = 873.0
    cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
    bed = synth.Bed([p.beds[0] for p in parts], cat("x"), cat("y"), cat("z"), cat("vx"), cat("vy"), cat("vz"),
                    cat("d_real"), cat("T"), np.concatenate([p.m0 for p in parts], axis=1), cat("ore"),
                    np.repeat(np.arange(2, dtype=np.int32), 150), "two")
    o = oracle.Oracle(bed)
    Jo, _ = o.adjoint_obs(200, [50, 200])
    for k, h in enumerate((50, 200)):
        sub = [oracle.Oracle(p).adjoint(h)[0] for p in parts]
        assert np.allclose(Jo[k], sub, rtol=1e-14, atol=0)
    assert Jo[1, 1] > Jo[1, 0] > 0
