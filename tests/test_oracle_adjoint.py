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
