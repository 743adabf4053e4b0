"""Seeded synthetic beds: the inputs that both the CUDA path and the CPU oracle consume.

This module only draws random numbers and places spheres; it holds none of the
method's arithmetic (no forces, no kinetics, no gas properties). Every array it
returns is plain numpy, so the same bed can be handed to the C-ABI library and to
the oracle.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based generator:
value i of stream s is mix(seed + golden * (s * 2**32 + i + 1)).

Workload shapes follow the paper's Table 3 (particle properties, bed geometry,
Sec. 4.3) and the five benchmark beds this library is measured on:
  * ``config_plain_2k``      2,000 parcels, D=0.05 m, H=0.3 m, 10x10x60 cells, 100 um, k=4
  * ``config_split_200k``    200,000 parcels, D=0.1 m, H=0.6 m, 40x40x240 cells, lognormal 100 um, k=6
  * ``config_ibm_2m``        2,000,000 parcels, two ore types, cone + perforated plate, 64x64x384
  * ``config_adjoint_64k``   64,000 parcels, packed, mixed composition, 1073 K
  * ``config_batched_32``    32 beds, 10k-200k parcels each, 773-1073 K, 0.2-0.5 m/s
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Wall kinds of a bed.
WALL_FLAT = 0   # cylinder side, flat bottom at z=0, lid at z=H
WALL_CONE = 1   # cylinder side, conical bottom, perforated distributor plate, lid

# Ore types (index into the per-ore arrays of a bed).
ORE_HEMATITE = 0
ORE_MAGNETITE = 1

# Physics switches (bit mask, identical meaning in the library and in the oracle).
NO_GRAVITY = 1 << 0
NO_DRAG = 1 << 1
NO_HEAT = 1 << 2
NO_KINETICS = 1 << 3
NO_GAS_UPDATE = 1 << 4
NO_FILM = 1 << 5
NO_LAYER = 1 << 6
NO_RXN_HEAT = 1 << 7
NO_CONTACTS = 1 << 8
RADIATION = 1 << 9   # switches ON the particle radiation (off by default)
CONDUCTION = 1 << 10  # switches ON the contact heat conduction (off by default)
GAS_SOLVER = 1 << 11  # the gas phase solved (momentum, energy, species) instead of the prescribed field

# Kinetic presets: (k0 [m/s], Ea [J/mol]) for R1 (h->m), R2 (m->w), R3 (w->Fe).
TAKENAKA = ((29.17, 15.56, 2858.0), (66974.0, 75345.0, 117204.0))        # Table 2
MAGNETITE_FIT = ((29.17, 8.0, 6000.0), (66974.0, 75345.0, 117204.0))      # Sec. 5.1.1
HEMATITE_FIT = ((10.0, 0.0007, 0.022), (42400.0, 19300.0, 33880.0))       # Sec. 5.2.1

# Initial solid mass fractions (Fe2O3, Fe3O4, FeO, Fe) of the two ores of Table 3.
COMP_BED2_HEMATITE = (0.9628, 0.0, 0.0372, 0.0)
COMP_BED1_MAGNETITE = (0.0, 0.6994, 0.3006, 0.0)
COMP_PURE_HEMATITE = (1.0, 0.0, 0.0, 0.0)
COMP_MIXED = tuple(0.5 * (a + b) for a, b in zip(COMP_BED2_HEMATITE, COMP_BED1_MAGNETITE))


def splitmix64(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n raw 64-bit SplitMix64 outputs of a counter-based stream."""
    with np.errstate(over="ignore"):
        ctr = np.arange(1, n + 1, dtype=np.uint64) + np.uint64((stream << 32) & 0xFFFFFFFFFFFFFFFF)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, n, stream) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform of two uniform streams."""
    u1 = uniform(seed, n, 2 * stream + 1000)
    u2 = uniform(seed, n, 2 * stream + 1001)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def lognormal_truncated(seed: int, n: int, median: float, sigma: float, nsig: float = 3.0,
                        stream: int = 0) -> np.ndarray:
    """Lognormal diameters, redrawn until inside +-nsig sigma of the median."""
    out = np.empty(n)
    todo = np.arange(n)
    s = stream
    while todo.size:
        z = normal(seed, todo.size, s)
        ok = np.abs(z) <= nsig
        out[todo[ok]] = median * np.exp(sigma * z[ok])
        todo = todo[~ok]
        s += 7
    return out


@dataclass
class BedConfig:
    """One bed: geometry, gas grid, contact law, kinetics (one row of the C struct)."""
    D: float = 0.05
    H: float = 0.3
    wall_kind: int = WALL_FLAT
    cone_half_angle: float = math.radians(45.0)
    cone_height: float = 0.05
    plate_z: float = 0.05
    hole_d: float = 1.0e-3
    hole_pitch: float = 4.0e-3
    nx: int = 10
    ny: int = 10
    nz: int = 60
    dt: float = 1.0e-5
    kn: float = 1000.0
    kt_over_kn: float = 2.0 / 7.0
    restitution: float = 0.9
    mu_s: float = 0.3
    mu_r: float = 0.0
    cg_ratio: float = 4.0
    coupling_interval: int = 1
    U_in: float = 0.3
    T_in: float = 873.0
    p0: float = 101325.0
    Y_in: tuple = (1.0, 0.0, 0.0)          # H2, H2O, N2 mass fractions
    k0: tuple = TAKENAKA[0]
    Ea: tuple = TAKENAKA[1]
    tortuosity: float = 2.0
    sphericity: tuple = (1.0, 1.0)          # per ore type
    xi0: tuple = (0.34, 0.29)               # initial porosity per ore type (Table 3)
    pore_d_cm: tuple = (3.3e-6, 9.5e-6)     # pore diameter per ore type, cm (Table 3)
    rho_true: tuple = (5300.0, 5180.0, 5390.0, 7900.0)  # Fe2O3, Fe3O4, FeO, Fe (Table 3)
    dpdz: float = 0.0                       # prescribed gas pressure gradient, Pa/m
    eps_min: float = 0.36                   # lower clamp of the gas volume fraction
    flags: int = 0                          # physics switches (NO_* bits, RADIATION)
    emissivity: float = 0.85                # particle emissivity (Table 3), used with RADIATION
    lambda_p: tuple = (2.5, 2.5)            # particle thermal conductivity per ore type, W/m/K (CONDUCTION)
    lambda_wall: float = 16.0               # reactor wall thermal conductivity, W/m/K (CONDUCTION)

    def as_dict(self) -> dict:
        return dict(self.__dict__)


@dataclass
class Bed:
    """A synthetic workload: bed configs plus the parcel arrays (input order = parcel index)."""
    beds: list
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    d_real: np.ndarray
    T: np.ndarray
    m0: np.ndarray            # (4, n) kg per parcel: Fe2O3, Fe3O4, FeO, Fe
    ore: np.ndarray           # int32
    bed: np.ndarray           # int32
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.size)

    def subset(self, idx: np.ndarray) -> "Bed":
        idx = np.asarray(idx)
        return Bed(self.beds, self.x[idx].copy(), self.y[idx].copy(), self.z[idx].copy(),
                   self.vx[idx].copy(), self.vy[idx].copy(), self.vz[idx].copy(),
                   self.d_real[idx].copy(), self.T[idx].copy(), self.m0[:, idx].copy(),
                   self.ore[idx].copy(), self.bed[idx].copy(), self.name + "-subset", dict(self.meta))


def _masses(d_cgp: np.ndarray, rho: float, comp: np.ndarray) -> np.ndarray:
    """Per-parcel species masses: density times sphere volume times mass fraction."""
    vol = (math.pi / 6.0) * d_cgp ** 3
    return (rho * vol)[None, :] * comp


def _stratified_lattice(seed: int, d: np.ndarray, R: float, z0: float, solid_fraction: float,
                        stream: int = 0, fill: float = 0.75, jitter: float = 1.0, compress: float = 0.0):
    """Overlap-free positions for spheres of diameters d inside a cylinder of radius R.

    Spheres are sorted by size and cut into strata of similar size; each stratum fills
    square-lattice layers (pitch = c * largest diameter of the stratum, c set by the
    target solid fraction) inside the disk, strata are stacked in random order from z0
    upward, and every sphere is jittered inside its own lattice box, so no two spheres
    overlap. fill is the fraction of a layer's sites a stratum of median spheres occupies;
    jitter scales the displacement inside the box (0: every sphere on its site); compress
    shrinks the pitch below the largest diameter by that fraction, so that neighbouring
    spheres overlap by up to compress times their diameter (a jammed packing). Returns x,
    y, z in the order of d.
    """
    n = d.size
    c = max(1.0, ((math.pi / 6.0) / solid_fraction) ** (1.0 / 3.0))
    order = np.argsort(d, kind="stable")
    # a stratum is roughly one full layer of the median sphere
    pitch_med = c * float(np.median(d))
    per_layer = max(1, int(math.pi * (R - pitch_med) ** 2 / pitch_med ** 2 * fill))
    strata = [order[i:i + per_layer] for i in range(0, n, per_layer)]
    perm = np.argsort(uniform(seed, len(strata), stream + 11), kind="stable")
    x = np.empty(n)
    y = np.empty(n)
    z = np.empty(n)
    zc = z0
    prev_pitch = None
    layer_no = 0
    ju = uniform(seed, 3 * n, stream + 12).reshape(3, n)
    for si in perm:
        members = strata[si]
        pitch = c * float(d[members].max()) * (1.0 - compress)
        # sites of a square lattice inside the disk of radius R - pitch/2
        m = int(math.floor(R / pitch)) + 1
        g = (np.arange(-m, m + 1) * pitch)
        gx, gy = np.meshgrid(g, g, indexing="ij")
        gx = gx.ravel()
        gy = gy.ravel()
        inside = np.hypot(gx, gy) <= R - 0.5 * pitch * 1.0001 - 1e-9
        sx = gx[inside]
        sy = gy[inside]
        if sx.size == 0:
            raise ValueError("bed too narrow for its spheres")
        pos = 0
        while pos < members.size:
            layer = members[pos:pos + sx.size]
            k = layer.size
            # consecutive layers are (p_prev + p)/2 apart, so boxes never overlap
            zc += 0.5 * pitch if prev_pitch is None else 0.5 * (pitch + prev_pitch)
            slack = 0.49 * jitter * np.maximum(pitch - d[layer], 0.0)
            sel = np.argsort(uniform(seed, sx.size, stream + 1000 + layer_no), kind="stable")[:k]
            x[layer] = sx[sel] + slack * (2.0 * ju[0, layer] - 1.0)
            y[layer] = sy[sel] + slack * (2.0 * ju[1, layer] - 1.0)
            z[layer] = zc + slack * (2.0 * ju[2, layer] - 1.0)
            prev_pitch = pitch
            layer_no += 1
            pos += k
    return x, y, z


def _uniform_cylinder(seed: int, d: np.ndarray, R: float, H: float, stream: int = 0):
    """Uniform random centres in the cylinder, redrawing any sphere that overlaps another
    or the wall (the dilute bed of the 2,000-parcel case)."""
    n = d.size
    r = 0.5 * d
    x = np.empty(n)
    y = np.empty(n)
    z = np.empty(n)
    placed = np.zeros(n, dtype=bool)
    s = stream
    for _ in range(200):
        todo = np.flatnonzero(~placed)
        if todo.size == 0:
            break
        u = uniform(seed, 3 * todo.size, s).reshape(3, -1)
        s += 1
        rad = (R - r[todo]) * np.sqrt(u[0])
        th = 2.0 * math.pi * u[1]
        x[todo] = rad * np.cos(th)
        y[todo] = rad * np.sin(th)
        z[todo] = r[todo] + (H - 2.0 * r[todo]) * u[2]
        placed[todo] = True
        # reject overlaps: keep the lower index of any overlapping pair
        idx = np.flatnonzero(placed)
        cell = 2.0 * r.max()
        key = np.floor(np.stack([x[idx], y[idx], z[idx]]) / cell).astype(np.int64)
        from collections import defaultdict
        grid = defaultdict(list)
        for t, (a, b, c) in enumerate(key.T):
            grid[(a, b, c)].append(idx[t])
        bad = set()
        for (a, b, c), members in grid.items():
            cand = []
            for da in (-1, 0, 1):
                for db in (-1, 0, 1):
                    for dc in (-1, 0, 1):
                        cand.extend(grid.get((a + da, b + db, c + dc), ()))
            for i in members:
                for j in cand:
                    if j <= i or j in bad or i in bad:
                        continue
                    dd = (x[i] - x[j]) ** 2 + (y[i] - y[j]) ** 2 + (z[i] - z[j]) ** 2
                    if dd < (r[i] + r[j]) ** 2 * 1.0001:
                        bad.add(j)
        if bad:
            placed[np.array(sorted(bad))] = False
    if not placed.all():
        raise RuntimeError("could not place all spheres")
    return x, y, z


def _assemble(beds, x, y, z, d_real, T, m0, ore, bedid, v=None, name="", meta=None) -> Bed:
    n = x.size
    vx = np.zeros(n) if v is None else v[0]
    vy = np.zeros(n) if v is None else v[1]
    vz = np.zeros(n) if v is None else v[2]
    return Bed(list(beds), x, y, z, vx, vy, vz, d_real, T, m0, ore.astype(np.int32),
               bedid.astype(np.int32), name, meta or {})


def _shuffle(seed: int, bed: Bed, stream: int = 99) -> Bed:
    perm = np.argsort(uniform(seed, bed.n, stream), kind="stable")
    return bed.subset(perm)


def _random_velocity(seed: int, n: int, scale: float, stream: int):
    if scale == 0.0:
        return None
    u = uniform(seed, 3 * n, stream).reshape(3, n)
    return scale * (2.0 * u - 1.0)


def config_plain_2k(seed: int = 2311039081, n: int = 2000) -> Bed:
    """2,000 parcels, uniform random in the cylinder; pure hematite at 873 K; FP64 form."""
    cfg = BedConfig(D=0.05, H=0.3, nx=10, ny=10, nz=60, dt=1e-5, cg_ratio=4.0, U_in=0.3,
                    T_in=873.0, Y_in=(1.0, 0.0, 0.0))
    d_real = np.full(n, 100e-6)
    d_cgp = cfg.cg_ratio * d_real
    x, y, z = _uniform_cylinder(seed, d_cgp, 0.5 * cfg.D, cfg.H)
    m0 = _masses(d_cgp, 5000.0, np.array(COMP_PURE_HEMATITE)[:, None])
    b = _assemble([cfg], x, y, z, d_real, np.full(n, 873.0), m0, np.zeros(n), np.zeros(n),
                  name="plain_2k", meta=dict(steps=200, rho=5000.0))
    return b


def packed_bed(seed: int, n: int, cfg: BedConfig, d_median: float, sigma: float,
               comp=COMP_PURE_HEMATITE, ore: int = ORE_HEMATITE, T0: float | None = None,
               rho: float = 5000.0, solid_fraction: float = 0.4, v_scale: float = 0.0,
               z0: float = 0.0, two_ores: bool = False, name: str = "packed",
               fill: float = 0.75, jitter: float = 1.0, compress: float = 0.0) -> Bed:
    """A packed bed of n parcels on the bottom of the bed (stratified jittered lattice)."""
    if sigma > 0.0:
        d_real = lognormal_truncated(seed, n, d_median, sigma)
    else:
        d_real = np.full(n, d_median)
    d_cgp = cfg.cg_ratio * d_real
    R = 0.5 * cfg.D
    x, y, z = _stratified_lattice(seed, d_cgp, R, z0, solid_fraction, fill=fill, jitter=jitter,
                                  compress=compress)
    if two_ores:
        # equal mass of the two ores: alternate parcels by a seeded coin so sizes stay mixed
        coin = uniform(seed, n, 31) < 0.5
        ores = np.where(coin, ORE_HEMATITE, ORE_MAGNETITE)
        comp_arr = np.where(coin[None, :], np.array(COMP_BED2_HEMATITE)[:, None],
                            np.array(COMP_BED1_MAGNETITE)[:, None])
    else:
        ores = np.full(n, ore)
        comp_arr = np.array(comp)[:, None]
    m0 = _masses(d_cgp, rho, comp_arr)
    T = np.full(n, cfg.T_in if T0 is None else T0)
    v = _random_velocity(seed, n, v_scale, 41)
    b = _assemble([cfg], x, y, z, d_real, T, m0, ores, np.zeros(n), v=v, name=name,
                  meta=dict(rho=rho, solid_fraction=solid_fraction))
    return _shuffle(seed, b)


def config_split_200k(seed: int = 2311039082, n: int = 200_000) -> Bed:
    cfg = BedConfig(D=0.1, H=0.6, nx=40, ny=40, nz=240, dt=1e-5, cg_ratio=6.0, U_in=0.3,
                    T_in=1023.0, Y_in=(1.0, 0.0, 0.0))
    b = packed_bed(seed, n, cfg, 100e-6, 0.25, name="split_200k")
    b.meta["steps"] = 1000
    return b


def config_ibm_2m(seed: int = 2311039083, n: int = 2_000_000, v_scale: float = 0.0,
                  solid_fraction: float = 0.4, U_in: float = 0.3, name: str = "ibm_2m",
                  fill: float = 0.75, jitter: float = 1.0, compress: float = 0.0, sigma: float = 0.25) -> Bed:
    cfg = BedConfig(D=0.1, H=0.6, wall_kind=WALL_CONE, cone_half_angle=math.radians(45.0),
                    cone_height=0.05, plate_z=0.05, hole_d=1e-3, hole_pitch=4e-3,
                    nx=64, ny=64, nz=384, dt=1e-5, cg_ratio=6.0, U_in=U_in, T_in=1023.0,
                    Y_in=(1.0, 0.0, 0.0), sphericity=(0.86, 0.85))
    b = packed_bed(seed, n, cfg, 120e-6, sigma, two_ores=True, z0=cfg.plate_z, name=name,
                   v_scale=v_scale, solid_fraction=solid_fraction, fill=fill, jitter=jitter, compress=compress)
    b.meta["steps"] = 500
    return b


def config_ibm_2m_dense(seed: int = 2311039086, n: int = 2_000_000, v_scale: float = 0.0,
                        U_in: float = 0.0, compress: float = 0.0, sigma: float = 0.0) -> Bed:
    """The 2M bed as a fixed packed bed: 120 um parcels (k = 6) of one size, every site of a
    square lattice filled, each sphere on its site and the pitch equal to the diameter, so
    that lattice neighbours touch; resting on the plate, the packing is compressed by its own
    weight within a few hundred steps into a static bed in which every parcel has its
    lattice contacts (the contact-dominated regime of a settled bed). No gas flow by
    default (U_in below about 0.03 m/s, minimum fluidisation of 120 um ore in H2 at 1023 K,
    keeps it packed)."""
    return config_ibm_2m(seed, n, v_scale=v_scale, solid_fraction=0.6, U_in=U_in, name="ibm_2m_dense",
                         fill=1.0, jitter=0.0, compress=compress, sigma=sigma)


def config_adjoint_64k(seed: int = 2311039084, n: int = 64_000) -> Bed:
    cfg = BedConfig(D=0.05, H=0.3, nx=10, ny=10, nz=60, dt=1e-5, cg_ratio=4.0, U_in=0.3,
                    T_in=1073.0, Y_in=(1.0, 0.0, 0.0))
    b = packed_bed(seed, n, cfg, 100e-6, 0.0, comp=COMP_MIXED, ore=ORE_HEMATITE,
                   name="adjoint_64k")
    b.meta.update(steps=2000, ckpt=100)
    return b


def config_batched_32(seed: int = 2311039085, n_beds: int = 32, n_min: int = 10_000,
                      n_max: int = 200_000, v_scale: float = 0.0) -> Bed:
    """32 independent beds of uneven size, temperature and inlet velocity."""
    counts = n_min + np.floor(uniform(seed, n_beds, 51) * (n_max - n_min + 1)).astype(np.int64)
    Us = 0.2 + 0.3 * uniform(seed, n_beds, 52)
    cfgs = []
    parts = []
    for b in range(n_beds):
        Tb = 773.0 + 300.0 * b / (n_beds - 1)
        cfg = BedConfig(D=0.05, H=0.3, nx=20, ny=20, nz=120, dt=1e-5, cg_ratio=6.0,
                        U_in=float(Us[b]), T_in=Tb, Y_in=(1.0, 0.0, 0.0))
        cfgs.append(cfg)
        parts.append(packed_bed(seed + 1000 * (b + 1), int(counts[b]), cfg, 100e-6, 0.25,
                                name=f"bed{b}", v_scale=v_scale))
    cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
    bedid = np.concatenate([np.full(p.n, i, dtype=np.int32) for i, p in enumerate(parts)])
    out = Bed(cfgs, cat("x"), cat("y"), cat("z"), cat("vx"), cat("vy"), cat("vz"),
              cat("d_real"), cat("T"), np.concatenate([p.m0 for p in parts], axis=1),
              cat("ore"), bedid, "batched_32", dict(steps=500, counts=counts.tolist()))
    return out


def small_packed(seed: int = 7, n: int = 3000, sigma: float = 0.2, v_scale: float = 0.05,
                 wall_kind: int = WALL_FLAT, T0: float = 1023.0, two_ores: bool = True,
                 nx: int = 8, nz: int = 48, D: float = 0.012, H: float = 0.072,
                 cg_ratio: float = 4.0, flags: int = 0) -> Bed:
    """A small dense bed for parity tests: several gas cells, many contacts, walls."""
    # dt = 5e-6 keeps omega_0 dt < 2 for the smallest parcels of the +-3 sigma size range
    cfg = BedConfig(D=D, H=H, nx=nx, ny=nx, nz=nz, dt=5e-6, cg_ratio=cg_ratio, U_in=0.3,
                    T_in=T0, Y_in=(0.9, 0.05, 0.05), wall_kind=wall_kind, flags=flags,
                    cone_half_angle=math.radians(45.0), cone_height=0.5 * D,
                    plate_z=0.5 * D, hole_d=0.6e-3, hole_pitch=1.5e-3, sphericity=(0.86, 0.85))
    z0 = cfg.plate_z if wall_kind == WALL_CONE else 0.0
    return packed_bed(seed, n, cfg, 100e-6, sigma, two_ores=two_ores, v_scale=v_scale, z0=z0,
                      T0=T0 - 30.0, name="small_packed")


def config_calibration(seed: int = 2311039087, n_per_bed: int = 128, n_beds: int = 8, T_lo: float = 773.0,
                       T_hi: float = 1073.0, dt: float = 5e-3, k0=TAKENAKA[0], Ea=TAKENAKA[1]) -> Bed:
    """Beds at n_beds evenly spaced temperatures for fitting the kinetics to reduction-degree
    curves over minutes (the frozen-position map of the adjoint; no contact is evaluated, so
    the contact stiffness is only a placeholder that keeps the time step admissible): each
    bed n_per_bed parcels of the mixed composition, packed, at its own temperature."""
    cfgs, parts = [], []
    for b in range(n_beds):
        Tb = T_lo + (T_hi - T_lo) * b / max(1, n_beds - 1)
        cfg = BedConfig(D=0.05, H=0.3, nx=10, ny=10, nz=60, dt=dt, cg_ratio=4.0, U_in=0.3, T_in=Tb,
                        Y_in=(1.0, 0.0, 0.0), kn=1e-6, flags=NO_CONTACTS, k0=tuple(k0), Ea=tuple(Ea))
        cfgs.append(cfg)
        parts.append(packed_bed(seed + 97 * b, n_per_bed, cfg, 100e-6, 0.0, comp=COMP_MIXED,
                                ore=ORE_HEMATITE, name=f"cal{b}"))
    cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
    bedid = np.repeat(np.arange(n_beds, dtype=np.int32), n_per_bed)
    return Bed(cfgs, cat("x"), cat("y"), cat("z"), cat("vx"), cat("vy"), cat("vz"), cat("d_real"), cat("T"),
               np.concatenate([p.m0 for p in parts], axis=1), cat("ore"), bedid, "calibration",
               dict(temperatures=[c.T_in for c in cfgs]))
