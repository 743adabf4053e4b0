"""Pins of the oracle's IBM wall geometry (CPU only): signed distances and normals of the
cone and of the perforated plate against a brute-force minimum over dense point samples
of each surface, and the solid-cell marking against a Monte-Carlo test of every cell.

The wall of the conical bed (Sec. 4, the reactor of Fig. 6 with an immersed boundary):
cylinder side, cone below the distributor plate, zero-thickness perforated plate with round
holes on a square lattice, lid. Distances are measured from the parcel centre.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_03908_gb300 import synth
from tests.helpers import ISOLATED, bed_from_arrays


def _cone_cfg(**kw):
    base = dict(D=0.1, H=0.6, wall_kind=synth.WALL_CONE, cone_half_angle=math.radians(45.0),
                cone_height=0.05, plate_z=0.05, hole_d=1e-3, hole_pitch=4e-3, nx=16, ny=16, nz=96)
    base.update(kw)
    return synth.BedConfig(**base)


def _cone_points(cfg, azimuth, n=400_001):
    """Dense sample of the cone's meridian at a given azimuth (the nearest point of a surface
    of revolution to a point lies in the point's own meridian half-plane)."""
    R = 0.5 * cfg.D
    al = cfg.cone_half_angle
    za = cfg.cone_height - R / math.tan(al)            # apex: the rim is at (R, cone_height)
    rho = np.linspace(0.0, 1.5 * R, n)
    return np.stack([rho * math.cos(azimuth), rho * math.sin(azimuth), za + rho / math.tan(al)], axis=1)


@pytest.mark.parametrize("alpha_deg", [45.0, 30.0, 60.0])
def test_cone_distance_and_normal_brute_force(alpha_deg):
    cfg = _cone_cfg(cone_half_angle=math.radians(alpha_deg))
    R = 0.5 * cfg.D
    za = cfg.cone_height - R / math.tan(cfg.cone_half_angle)
    u = synth.uniform(17, 3 * 40).reshape(3, 40)
    checked = 0
    for k in range(40):
        rho = 0.9 * R * u[0, k]
        th = 2 * math.pi * u[1, k]
        zsurf = za + rho / math.tan(cfg.cone_half_angle)
        z = zsurf + 3e-3 * u[2, k] + 1e-5          # inside the fluid, above the cone
        if z >= cfg.plate_z:
            continue
        x, y = rho * math.cos(th), rho * math.sin(th)
        dist, nrm = oracle.wall_distance(cfg, x, y, z)
        pts = _cone_points(cfg, th)
        dv = np.array([x, y, z])[None, :] - pts
        dd = np.sqrt((dv ** 2).sum(1))
        j = int(np.argmin(dd))
        assert abs(dist[1] - dd[j]) < 2e-7, (k, dist[1], dd[j])
        assert dist[1] > 0                            # positive on the fluid side
        assert np.allclose(nrm[1], dv[j] / dd[j], atol=5e-3)
        checked += 1
    assert checked > 20


def _plate_points(cfg, x, y, half=2.5e-3, h=4e-6, nphi=100_000):
    """Dense sample of the plate z = plate_z around (x, y): a grid over the solid part
    (holes removed) plus the rims of the nearby holes, each sampled along its circle."""
    g = np.arange(-half, half + h / 2, h)
    X, Y = np.meshgrid(x + g, y + g, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    p = cfg.hole_pitch
    hx = np.floor(X / p + 0.5) * p
    hy = np.floor(Y / p + 0.5) * p
    keep = np.hypot(X - hx, Y - hy) >= 0.5 * cfg.hole_d
    pts = [np.stack([X[keep], Y[keep], np.full(keep.sum(), cfg.plate_z)], axis=1)]
    phi = np.linspace(0.0, 2 * math.pi, nphi, endpoint=False)
    cx0, cy0 = math.floor(x / p + 0.5) * p, math.floor(y / p + 0.5) * p
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            rx = cx0 + a * p + 0.5 * cfg.hole_d * np.cos(phi)
            ry = cy0 + b * p + 0.5 * cfg.hole_d * np.sin(phi)
            pts.append(np.stack([rx, ry, np.full(nphi, cfg.plate_z)], axis=1))
    return np.concatenate(pts)


def test_perforated_plate_distance_and_normal_brute_force():
    cfg = _cone_cfg()
    u = synth.uniform(23, 3 * 30).reshape(3, 30)
    for k in range(30):
        # points near a hole (half of them inside the hole's cylinder), above or below the plate
        cx = (int(8 * u[0, k]) - 4) * cfg.hole_pitch
        cy = (int(8 * u[1, k]) - 4) * cfg.hole_pitch
        off = (0.25 + 0.8 * u[2, k]) * cfg.hole_d
        x, y = cx + off * math.cos(7.0 * k), cy + off * math.sin(7.0 * k)
        z = cfg.plate_z + (1 if k % 2 else -1) * (50e-6 + 400e-6 * ((k * 0.37) % 1.0))
        dist, nrm = oracle.wall_distance(cfg, x, y, z)
        pts = _plate_points(cfg, x, y)
        dv = np.array([x, y, z])[None, :] - pts
        dd = np.sqrt((dv ** 2).sum(1))
        j = int(np.argmin(dd))
        assert abs(dist[2] - dd[j]) < 1e-7 + 1e-3 * dd[j], (k, dist[2], dd[j])
        assert np.allclose(nrm[2], dv[j] / dd[j], atol=5e-3)


def test_side_and_lid_distances():
    cfg = _cone_cfg()
    dist, nrm = oracle.wall_distance(cfg, 0.03, 0.04, 0.2)
    assert abs(dist[0] - (0.05 - 0.05)) < 1e-15 and abs(dist[3] - 0.4) < 1e-15
    dist, nrm = oracle.wall_distance(cfg, 0.012, -0.005, 0.3)
    assert abs(dist[0] - (0.05 - 0.013)) < 1e-15
    assert np.allclose(nrm[0], [-0.012 / 0.013, 0.005 / 0.013, 0.0], atol=1e-15)


def _outside_fluid(cfg, x, y, z):
    """Independent inside/outside test of the conical bed: outside the cylinder, or below
    the cone surface (z below the apex height plus rho / tan(alpha))."""
    R = 0.5 * cfg.D
    rho = np.hypot(x, y)
    za = cfg.cone_height - R / math.tan(cfg.cone_half_angle)
    return (rho > R) | (z < za + rho / math.tan(cfg.cone_half_angle))


@pytest.mark.parametrize("wall", [synth.WALL_CONE, synth.WALL_FLAT])
def test_ibm_solid_cells_against_monte_carlo(wall):
    # a cell is marked solid when it lies wholly outside the fluid: every marked cell has
    # all of its Monte-Carlo points (and corners) outside, no cell with a point inside is
    # marked, and the marking misses only cells that touch the boundary within one diagonal
    cfg = _cone_cfg(wall_kind=wall, nx=12, ny=12, nz=40, H=0.2,
                    flags=ISOLATED)
    b = bed_from_arrays(cfg, [0.0], 0.0, 0.15)
    mark = oracle.Oracle(b).gas()[:, oracle.G_MARK]
    nx, ny, nz = cfg.nx, cfg.ny, cfg.nz
    hx, hy, hz = cfg.D / nx, cfg.D / ny, cfg.H / nz
    m = 64
    u = synth.uniform(31, 3 * m).reshape(3, m)
    corners = np.array([[a, b_, c] for a in (0, 1) for b_ in (0, 1) for c in (0, 1)], dtype=float).T
    samples = np.concatenate([u, corners], axis=1)
    n_out_all = 0
    for c in range(nx * ny * nz):
        ix, iy, iz = c % nx, (c // nx) % ny, c // (nx * ny)
        x = -0.5 * cfg.D + (ix + samples[0]) * hx
        y = -0.5 * cfg.D + (iy + samples[1]) * hy
        z = (iz + samples[2]) * hz
        out = _outside_fluid(cfg, x, y, z) if wall == synth.WALL_CONE else (np.hypot(x, y) > 0.5 * cfg.D)
        if mark[c] != 0:
            assert out.all(), c
        if not out.any():
            assert mark[c] == 0, c
        if out.all():
            n_out_all += 1
            if mark[c] == 0:
                # unmarked although wholly outside: its centre lies within a diagonal of the fluid
                xc, yc, zc = -0.5 * cfg.D + (ix + 0.5) * hx, -0.5 * cfg.D + (iy + 0.5) * hy, (iz + 0.5) * hz
                g = np.linspace(-1, 1, 41)
                diag = math.sqrt(hx * hx + hy * hy + hz * hz)
                G = np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1) * diag
                near = ~_outside_fluid(cfg, xc + G[0], yc + G[1], zc + G[2]) if wall == synth.WALL_CONE \
                    else np.hypot(xc + G[0], yc + G[1]) <= 0.5 * cfg.D
                assert near.any(), c
    assert mark.sum() > 0.5 * n_out_all
