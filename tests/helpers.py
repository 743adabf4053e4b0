"""Small bed builders shared by the tests (input construction only, no method arithmetic)."""
import math

import numpy as np

from paper_2311_03908_gb300 import synth


def bed_from_arrays(cfg, x, y, z, v=None, d_real=100e-6, T=873.0, comp=(1.0, 0.0, 0.0, 0.0),
                    rho=5000.0, ore=0, w=None):
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = x.size
    y = np.broadcast_to(np.asarray(y, dtype=float), (n,)).copy()
    z = np.broadcast_to(np.asarray(z, dtype=float), (n,)).copy()
    d = np.broadcast_to(np.asarray(d_real, dtype=float), (n,)).copy()
    dc = cfg.cg_ratio * d
    mass = rho * math.pi / 6.0 * dc ** 3
    comp = np.asarray(comp, dtype=float)
    if comp.ndim == 1:
        comp = np.repeat(comp[:, None], n, axis=1)
    m0 = mass[None, :] * comp
    v = np.zeros((3, n)) if v is None else np.asarray(v, dtype=float).reshape(3, n)
    T = np.broadcast_to(np.asarray(T, dtype=float), (n,)).copy()
    ore = np.broadcast_to(np.asarray(ore, dtype=np.int32), (n,)).copy()
    return synth.Bed([cfg], x.copy(), y, z, v[0].copy(), v[1].copy(), v[2].copy(), d, T, m0,
                     ore, np.zeros(n, dtype=np.int32), "explicit")


ISOLATED = (synth.NO_GRAVITY | synth.NO_DRAG | synth.NO_HEAT | synth.NO_KINETICS |
            synth.NO_GAS_UPDATE)


def paper_values():
    """Numbers printed in the paper (tests/golden/paper_printed_values.txt), by name."""
    return golden_values("paper_printed_values.txt")


def handbook_values():
    """Tabulated reference values independent of the paper (tests/golden/handbook_values.txt)."""
    return golden_values("handbook_values.txt")


def golden_values(fname):
    import os
    out = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", fname)
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            name, rest = line.split("=", 1)
            out[name.strip()] = float(rest.split("|", 1)[0])
    return out
