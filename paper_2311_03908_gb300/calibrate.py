"""Fit of the kinetic parameters to observed reduction-degree curves with the adjoint.

Sec. 5.1.1 and Sec. 5.2.1 of the paper fit the pre-exponential factors (and use published
activation energies) of the interface rate constants k_r = k0 exp(-Ea / (R T_p)) (eq (2-13))
by comparing simulated reduction-degree curves with measured ones at several temperatures.
This module automates that fit: the curves come from the frozen-position drag-heat-reaction
map of dem_adjoint_obs (one context holding one bed per temperature), and the gradient of
the least-squares misfit from the library's hand-written reverse sweep, one call per
evaluation, fed to a quasi-Newton minimiser (L-BFGS-B).

Each reaction r is parametrised by u_r = ln k_r(T_ref) (the log rate constant at a reference
temperature inside the fitted range) and w_r = Ea_r / (R T_ref): over a range of temperatures
around T_ref these two are far less correlated than ln k0 and Ea, which the Arrhenius form
couples through ln k0 = u + w.
"""
from __future__ import annotations

import math

import numpy as np

R_GAS = 8.314   # J/mol/K, the gas constant of Sec. 2.1


def to_theta(k0, Ea, T_ref):
    k0, Ea = np.asarray(k0, float), np.asarray(Ea, float)
    w = Ea / (R_GAS * T_ref)
    return np.concatenate([np.log(k0) - w, w])


def from_theta(th, T_ref):
    u, w = th[:3], th[3:]
    return np.exp(u + w), w * R_GAS * T_ref


def misfit(ctx, th, nsteps, obs_steps, target, T_ref, ckpt, scale, want_grad=True):
    """0.5 sum((J_obs - target) / scale)^2 and its gradient in theta."""
    k0, Ea = from_theta(th, T_ref)
    ctx.dem_set_kinetics(k0, Ea)
    Jo, _ = ctx.dem_adjoint_obs(nsteps, obs_steps, None, ckpt)
    r = (Jo - target) / scale
    f = 0.5 * float(np.sum(r * r))
    if not want_grad:
        return f, None, Jo
    _, g = ctx.dem_adjoint_obs(nsteps, obs_steps, r / scale, ckpt)      # d f / d(k0, Ea)
    gk0, gEa = g[:3], g[3:]
    # chain rule: ln k0 = u + w, Ea = w R T_ref
    du = k0 * gk0
    dw = k0 * gk0 + R_GAS * T_ref * gEa
    return f, np.concatenate([du, dw]), Jo


def fit_kinetics(ctx, nsteps, obs_steps, target, k0_start, Ea_start, T_ref=900.0, ckpt=200, maxiter=300,
                 gtol=1e-14):
    """Minimise the curve misfit from a starting guess. Returns the fitted parameters, the
    final misfit, the number of misfit evaluations and the path of the misfit."""
    from scipy.optimize import minimize
    target = np.asarray(target, float)
    scale = float(np.abs(target).max())
    hist = []

    def fun(th):
        f, g, _ = misfit(ctx, th, nsteps, obs_steps, target, T_ref, ckpt, scale)
        hist.append(f)
        return f, g

    th0 = to_theta(k0_start, Ea_start, T_ref)
    # a box around the start keeps every trial rate constant finite and every Ea >= 0
    bounds = [(th0[q] - 12.0, th0[q] + 12.0) for q in range(3)] + \
             [(max(0.0, 0.5 * th0[q]), 2.0 * th0[q] + 1.0) for q in range(3, 6)]
    res = minimize(fun, th0, jac=True, method="L-BFGS-B", bounds=bounds,
                   options=dict(maxiter=maxiter, maxfun=3 * maxiter, ftol=1e-30, gtol=gtol))
    k0, Ea = from_theta(res.x, T_ref)
    return dict(k0=k0, Ea=Ea, misfit=float(res.fun), evaluations=len(hist), iterations=int(res.nit),
                history=hist, message=str(res.message))


def curve_jacobian(ctx, k0, Ea, nsteps, obs_steps, T_ref=900.0, ckpt=200, rel=1e-4):
    """Sensitivities of the observed curves to theta by central differences of the forward
    map: (n_obs * n_beds, 6); its singular values say how well the curves fix the six
    parameters."""
    th = to_theta(k0, Ea, T_ref)
    cols = []
    for q in range(6):
        h = rel * max(abs(th[q]), 1.0)
        vals = []
        for s in (1, -1):
            t = th.copy()
            t[q] += s * h
            kk, ee = from_theta(t, T_ref)
            ctx.dem_set_kinetics(kk, ee)
            Jo, _ = ctx.dem_adjoint_obs(nsteps, obs_steps, None, ckpt)
            vals.append(Jo.ravel())
        cols.append((vals[0] - vals[1]) / (2 * h))
    ctx.dem_set_kinetics(k0, Ea)
    return np.stack(cols, axis=1)
