"""Hand-written adjoint (through the C ABI and torch.autograd) against the FP64 oracle's
dual-number gradient and central finite differences of the same map, on the GPU."""
import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

from paper_2311_03908_gb300 import binding  # noqa: E402
from paper_2311_03908_gb300.autograd import reduction_degree  # noqa: E402


def _ctx(bed, prec="fp64"):
    return binding.Context(bed, precision=prec, stream=torch.cuda.current_stream().cuda_stream)


def test_adjoint_gradient_matches_dual_numbers_and_central_differences():
    bed = synth.config_adjoint_64k(n=1500)
    ctx = _ctx(bed)
    J, g = ctx.dem_adjoint(300, 40)
    ref = oracle.Oracle(bed)
    Jd, gd = ref.adjoint(300, mode=2)
    Jf, gf = ref.adjoint(300, mode=1, rel=1e-6)
    assert J > 0
    assert abs(J - Jd) < 1e-9 * abs(Jd)
    assert np.all(np.abs(g - gd) <= 1e-4 * np.abs(gd)), (g, gd)
    assert np.all(np.abs(g - gf) <= 1e-4 * np.abs(gf)), (g, gf)
    # the checkpoint interval changes the recomputation, not the result
    J2, g2 = ctx.dem_adjoint(300, 7)
    assert J2 == J and np.allclose(g2, g, rtol=1e-12, atol=0)
    J3, g3 = ctx.dem_adjoint(300, 300)
    assert np.allclose(g3, g, rtol=1e-12, atol=0)
    # forward sweep only
    J4, none = ctx.dem_adjoint(300, 40, want_grad=False)
    assert none is None and J4 == J
    ctx.close()


def test_adjoint_split_context_and_magnetite_fit():
    bed = synth.config_adjoint_64k(n=800)
    for c in bed.beds:
        c.k0, c.Ea = synth.MAGNETITE_FIT
    ctx = _ctx(bed, "split")
    J, g = ctx.dem_adjoint(150, 50)
    ref = oracle.Oracle(bed)
    Jd, gd = ref.adjoint(150, mode=2)
    # the split context stores v and T in FP32; the sub-step itself runs in FP64
    assert abs(J - Jd) < 1e-5 * abs(Jd)
    assert np.all(np.abs(g - gd) <= 1e-3 * np.abs(gd)), (g, gd)
    ctx.close()


def test_autograd_function_returns_the_adjoint_gradient():
    bed = synth.config_adjoint_64k(n=600)
    ctx = _ctx(bed)
    k0, Ea = synth.TAKENAKA
    params = torch.tensor(list(k0) + list(Ea), dtype=torch.float64, requires_grad=True)
    J = reduction_degree(params, ctx, nsteps=100, ckpt_every=25)
    J.backward()
    Jr, gr = ctx.dem_adjoint(100, 25)
    assert float(J.detach()) == Jr
    assert np.allclose(params.grad.numpy(), gr, rtol=1e-13, atol=0)
    ctx.close()


def test_adjoint_at_the_benchmarked_size():
    # the adjoint workload as the bench times it: 64,000 parcels, 2,000 sub-steps, a
    # checkpoint every 100; the gradient against the oracle's FP64 dual numbers and central
    # differences (relative step 1e-6) of the same map, per component to 1e-4
    bed = synth.config_adjoint_64k()
    steps, ck = int(bed.meta["steps"]), int(bed.meta["ckpt"])
    ctx = _ctx(bed)
    J, g = ctx.dem_adjoint(steps, ck)
    ctx.close()
    ref = oracle.Oracle(bed)
    Jd, gd = ref.adjoint(steps, mode=2)
    assert abs(J - Jd) < 1e-9 * abs(Jd)
    assert np.all(np.abs(g - gd) <= 1e-4 * np.abs(gd)), (g, gd)
    Jf, gf = ref.adjoint(steps, mode=1, rel=1e-6)
    assert np.all(np.abs(g - gf) <= 1e-4 * np.abs(gf)), (g, gf)


def test_observed_curves_and_weighted_gradient_against_oracle():
    # four beds at different temperatures in one context: the bed curves at five observation
    # steps, and the gradient of an arbitrary weighted sum of them, against the oracle's
    # FP64 values and dual numbers; observations inside a checkpoint segment and at its end
    bed = synth.config_calibration(n_per_bed=200, n_beds=4, dt=1e-3)
    obs = [37, 100, 250, 399, 400]
    w = synth.uniform(5, 20).reshape(5, 4) * 2 - 1
    ctx = _ctx(bed)
    Jg, gg = ctx.dem_adjoint_obs(400, obs, w, 50)
    Jf, none = ctx.dem_adjoint_obs(400, obs, None, 50)
    assert none is None and np.array_equal(Jf, Jg)
    ref = oracle.Oracle(bed)
    Jo, go = ref.adjoint_obs(400, obs, w, mode=2)
    assert np.allclose(Jg, Jo, rtol=1e-9, atol=1e-15)
    assert np.all(np.abs(gg - go) <= 1e-6 * np.abs(go)), (gg, go)
    # the checkpoint interval changes the recomputation only
    _, g2 = ctx.dem_adjoint_obs(400, obs, w, 7)
    assert np.allclose(g2, gg, rtol=1e-12, atol=0)
    ctx.close()


def test_curve_autograd_and_calibration_recovers_the_kinetics():
    # synthetic measured curves from the oracle at known kinetics (Table 2) for eight beds at
    # 773..1073 K over 50 s of reduction at a chemistry time step of 5 ms (reduction degrees
    # 0.12..0.90); the fit starts from k0 off by factors 3, 0.4, 2.5 and Ea off by +4 %, -4 %,
    # +3 % and must recover all six (noise-free curves: to far below the stated 1e-6)
    from paper_2311_03908_gb300 import calibrate
    from paper_2311_03908_gb300.autograd import reduction_degree_curves
    nsteps = 10000
    obs = [nsteps * (k + 1) // 10 for k in range(10)]
    bed = synth.config_calibration()
    Jt, _ = oracle.Oracle(bed).adjoint_obs(nsteps, obs)
    ctx = _ctx(bed)
    k0t, Eat = np.array(synth.TAKENAKA[0]), np.array(synth.TAKENAKA[1])
    # the autograd function's backward is the weighted reverse sweep
    p = torch.tensor(np.concatenate([k0t, Eat]), dtype=torch.float64, requires_grad=True)
    J = reduction_degree_curves(p, ctx, nsteps, obs)
    assert np.allclose(J.detach().numpy(), Jt, rtol=1e-9, atol=1e-15)
    (J * torch.from_numpy(Jt)).sum().backward()
    _, g = ctx.dem_adjoint_obs(nsteps, obs, Jt, 200)
    assert np.allclose(p.grad.numpy(), g, rtol=1e-12, atol=0)
    r = calibrate.fit_kinetics(ctx, nsteps, obs, Jt, k0t * np.array([3.0, 0.4, 2.5]), Eat * np.array([1.04, 0.96, 1.03]))
    assert np.all(np.abs(r["k0"] / k0t - 1) < 1e-6), r
    assert np.all(np.abs(r["Ea"] / Eat - 1) < 1e-6), r
    ctx.close()
