"""ctypes wrapper of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

The oracle is the plain, slow restatement of the paper's particle step that the CUDA
library is checked against. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package; the library itself never does.

Parity notes per function (pins live in tests/test_oracle_*.py):
  * pair search, contact law, integration: pinned (brute force, closed-form binary
    collision, energy conservation, free fall, Coulomb sliding).
  * kinetics: pinned (chemical-control law, oxygen/iron balance, Kirchhoff network
    against the printed closed forms, printed q values and densities, loose F_mean).
  * drag and convection: pinned by their textbook limits (Stokes drag, Nu = Sh = 2).
  * gas properties: pinned by invariants (Fuller scaling, Wilke binary limit, NASA
    dH/dT = C_p, standard enthalpies) and the absolute Fuller coefficients against measured
    binary diffusivities.
  * prescribed gas update: pinned by the upwind scheme's conservation, transport speed and
    monotonicity, the gas-parcel energy exchange and the exact mixing of the deposited
    mass (tests/test_oracle_gas_update.py).
  * porosity-dependent D_eff values: parity unpinned (the tortuosity is not printed).
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

# Index constants mirror dem_oracle.h (the oracle's own header).
NB = 0
_B = {}
for _i, _name in enumerate(
        ["D", "H", "WALL", "CONE_ALPHA", "CONE_H", "PLATE_Z", "HOLE_D", "HOLE_PITCH", "NX", "NY",
         "NZ", "DT", "KN", "KT_KN", "REST", "MU_S", "MU_R", "CG", "NCOUPLE", "U_IN", "T_IN", "P0",
         "Y_IN", "Y_IN1", "Y_IN2", "K0", "K01", "K02", "EA", "EA1", "EA2", "TAU", "PSI", "PSI1",
         "XI0", "XI01", "PORE", "PORE1", "RHOT", "RHOT1", "RHOT2", "RHOT3", "DPDZ", "EPS_MIN",
         "FLAGS", "EMISS", "LAMP", "LAMP1", "LAMW"]):
    _B[_name] = _i
NB = len(_B)

S_X, S_Y, S_Z, S_VX, S_VY, S_VZ, S_WX, S_WY, S_WZ, S_T = range(10)
S_M = 10
S_AX, S_AY, S_AZ, S_ALX, S_ALY, S_ALZ = range(14, 20)
NS = 20
STATE_NAMES = ["x", "y", "z", "vx", "vy", "vz", "wx", "wy", "wz", "T", "m_h", "m_m", "m_w",
               "m_fe", "ax", "ay", "az", "alx", "aly", "alz"]

D_FC, D_TC, D_FD, D_K, D_QCONV, D_QR, D_QRM = 0, 3, 6, 9, 10, 11, 12
D_XIDOT, D_MDOT, D_FFILM, D_A, D_B, D_SH, D_NU, D_RE, D_NCONTACT, D_CELL = 13, 16, 20, 21, 24, 27, 28, 29, 30, 31
D_TSE, D_QRAD, D_QCOND = 32, 33, 34
ND = 35

G_EPS, G_Y, G_T, G_MARK = 0, 1, 4, 5
NG = 6
NDEP = 14
DEP_NAMES = ["Vs", "SH2", "SH2O", "K", "Kvx", "Kvy", "Kvz", "hA", "hAT", "Qrm", "Qr", "EQ", "ES", "count"]

GP_RHO, GP_MU, GP_LAM, GP_CP, GP_X, GP_XP, GP_DM, GP_MG, GP_D12, GP_D13 = 0, 1, 2, 3, 4, 5, 8, 9, 10, 11
NGP = 12
K_XIDOT, K_MDOT, K_SH2, K_SH2O, K_QR, K_QRM, K_A, K_B, K_F, K_SH, K_F3, K_ACT, K_EQ, K_ES, K_DEFF, K_XI = \
    0, 3, 7, 8, 9, 10, 11, 14, 17, 18, 19, 22, 25, 26, 27, 30
NK = 33
MAX_CONTACTS = 24

SPECIES = ["H2", "H2O", "N2", "Fe2O3", "Fe3O4", "FeO", "Fe"]

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int32, dp, C.c_int32] + [dp] * 9 + [ip, ip, dp, dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_int32]
        L.orc_step.restype = C.c_int32
        for f in ("orc_get_state", "orc_get_diag", "orc_get_gas", "orc_get_deposits"):
            getattr(L, f).argtypes = [C.c_void_p, dp]
        L.orc_get_contacts.argtypes = [C.c_void_p, ip, ip, dp]
        L.orc_ncells.argtypes = [C.c_void_p]
        L.orc_ncells.restype = C.c_int64
        L.orc_reduction_degree.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_set_kinetics.argtypes = [C.c_void_p, dp, dp]
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_get_threads.restype = C.c_int32
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_adjoint.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_double, dp, dp]
        L.orc_adjoint.restype = C.c_int32
        L.orc_get_flow.argtypes = [C.c_void_p, dp]
        L.orc_get_faces.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        L.orc_pseudo_turbulence.argtypes = [C.c_double] * 5 + [dp, dp, C.c_double, dp]
        L.orc_adjoint_obs.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, ip, dp, dp, dp]
        L.orc_adjoint_obs.restype = C.c_int32
        L.orc_gas_props.argtypes = [dp, C.c_double, dp, C.c_double, dp]
        L.orc_network.argtypes = [dp, dp, C.c_double, ip, C.c_double, dp, dp, dp, ip]
        L.orc_kinetics.argtypes = [dp, dp, C.c_double, C.c_double, C.c_int32, C.c_double, C.c_double,
                                   C.c_double, dp, C.c_double, dp]
        L.orc_drag.argtypes = [dp, C.c_double, C.c_int32, C.c_double, C.c_double, C.c_double, dp, dp, dp]
        L.orc_heat.argtypes = [dp, C.c_double, C.c_double, C.c_double, C.c_double, dp, dp, dp]
        for f in ("orc_enthalpy", "orc_cp"):
            getattr(L, f).argtypes = [C.c_int32, C.c_double]
            getattr(L, f).restype = C.c_double
        L.orc_molar_mass.argtypes = [C.c_int32]
        L.orc_molar_mass.restype = C.c_double
        L.orc_layer_porosity.argtypes = [dp, C.c_int32, dp]
        for f in ("orc_pairs_bruteforce", "orc_pairs_cells"):
            getattr(L, f).argtypes = [C.c_int32, dp, dp, dp, dp, ip, C.c_int64]
            getattr(L, f).restype = C.c_int64
        L.orc_wall_distance.argtypes = [dp, C.c_double, C.c_double, C.c_double, dp, dp]
        L.orc_restitution_f.argtypes = [C.c_double]
        L.orc_restitution_f.restype = C.c_double
        L.orc_e_cgp.argtypes = [C.c_double, C.c_double]
        L.orc_e_cgp.restype = C.c_double
        L.orc_conduction_pair.argtypes = [dp] + [C.c_double] * 8 + [dp]
        L.orc_conduction_wall.argtypes = [dp] + [C.c_double] * 5 + [dp]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def bed_vector(cfg) -> np.ndarray:
    """Flatten a synth.BedConfig (or dict) into the oracle's per-bed parameter vector."""
    c = cfg if isinstance(cfg, dict) else cfg.as_dict()
    v = np.zeros(NB)
    v[_B["D"]] = c["D"]
    v[_B["H"]] = c["H"]
    v[_B["WALL"]] = c["wall_kind"]
    v[_B["CONE_ALPHA"]] = c["cone_half_angle"]
    v[_B["CONE_H"]] = c["cone_height"]
    v[_B["PLATE_Z"]] = c["plate_z"]
    v[_B["HOLE_D"]] = c["hole_d"]
    v[_B["HOLE_PITCH"]] = c["hole_pitch"]
    v[_B["NX"]], v[_B["NY"]], v[_B["NZ"]] = c["nx"], c["ny"], c["nz"]
    v[_B["DT"]] = c["dt"]
    v[_B["KN"]] = c["kn"]
    v[_B["KT_KN"]] = c["kt_over_kn"]
    v[_B["REST"]] = c["restitution"]
    v[_B["MU_S"]] = c["mu_s"]
    v[_B["MU_R"]] = c["mu_r"]
    v[_B["CG"]] = c["cg_ratio"]
    v[_B["NCOUPLE"]] = c["coupling_interval"]
    v[_B["U_IN"]] = c["U_in"]
    v[_B["T_IN"]] = c["T_in"]
    v[_B["P0"]] = c["p0"]
    v[_B["Y_IN"]:_B["Y_IN"] + 3] = c["Y_in"]
    v[_B["K0"]:_B["K0"] + 3] = c["k0"]
    v[_B["EA"]:_B["EA"] + 3] = c["Ea"]
    v[_B["TAU"]] = c["tortuosity"]
    v[_B["PSI"]:_B["PSI"] + 2] = c["sphericity"]
    v[_B["XI0"]:_B["XI0"] + 2] = c["xi0"]
    v[_B["PORE"]:_B["PORE"] + 2] = c["pore_d_cm"]
    v[_B["RHOT"]:_B["RHOT"] + 4] = c["rho_true"]
    v[_B["DPDZ"]] = c["dpdz"]
    v[_B["EPS_MIN"]] = c["eps_min"]
    v[_B["FLAGS"]] = c["flags"]
    v[_B["EMISS"]] = c["emissivity"]
    v[_B["LAMP"]:_B["LAMP"] + 2] = c["lambda_p"]
    v[_B["LAMW"]] = c["lambda_wall"]
    return v


class Oracle:
    """Stateful oracle over a synth.Bed (all beds, all parcels, input order)."""

    def __init__(self, bed, gasY=None, gasT=None):
        L = lib()
        self.n = bed.n
        self.nbeds = len(bed.beds)
        self._grids = [(c.nx, c.ny, c.nz) for c in bed.beds]
        self._keep = []
        bv, bp = _d(np.stack([bed_vector(c) for c in bed.beds]))
        arrs = [bed.x, bed.y, bed.z, bed.vx, bed.vy, bed.vz, bed.d_real, bed.T,
                np.ascontiguousarray(bed.m0).ravel()]
        ptrs = []
        for a in arrs:
            a2, p = _d(a)
            self._keep.append(a2)
            ptrs.append(p)
        ore, op = _i(bed.ore)
        bid, bidp = _i(bed.bed)
        gy = None if gasY is None else _d(gasY)
        gt = None if gasT is None else _d(gasT)
        self._keep += [bv, ore, bid]
        # m0 pointer takes the slot after T
        self.h = L.orc_create(self.nbeds, bp, self.n, *ptrs[:8], ptrs[8], op, bidp,
                              gy[1] if gy else None, gt[1] if gt else None)
        self.ncells = int(L.orc_ncells(self.h))

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().orc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def step(self, n: int = 1):
        lib().orc_step(self.h, int(n))

    def state(self) -> np.ndarray:
        out = np.zeros((NS, self.n))
        lib().orc_get_state(self.h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def diag(self) -> np.ndarray:
        out = np.zeros((ND, self.n))
        lib().orc_get_diag(self.h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def contacts(self):
        cnt = np.zeros(self.n, dtype=np.int32)
        partner = np.zeros((self.n, MAX_CONTACTS), dtype=np.int32)
        xi = np.zeros((self.n, MAX_CONTACTS, 3))
        lib().orc_get_contacts(self.h, cnt.ctypes.data_as(C.POINTER(C.c_int32)),
                               partner.ctypes.data_as(C.POINTER(C.c_int32)),
                               xi.ctypes.data_as(C.POINTER(C.c_double)))
        return cnt, partner, xi

    def gas(self) -> np.ndarray:
        out = np.zeros((self.ncells, NG))
        lib().orc_get_gas(self.h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def flow(self) -> np.ndarray:
        """Per gas cell: the cell-centre gas velocity (3) and the pressure relative to p0."""
        out = np.zeros((self.ncells, 4))
        lib().orc_get_flow(self.h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def faces(self, b: int = 0):
        """Face velocities of solved bed b, as arrays (nz, ny, nx+1), (nz, ny+1, nx), (nz+1, ny, nx)."""
        nx, ny, nz = self._grids[b]
        fu = np.zeros((nz, ny, nx + 1))
        fv = np.zeros((nz, ny + 1, nx))
        fw = np.zeros((nz + 1, ny, nx))
        lib().orc_get_faces(self.h, b, fu.ctypes.data_as(C.POINTER(C.c_double)),
                            fv.ctypes.data_as(C.POINTER(C.c_double)), fw.ctypes.data_as(C.POINTER(C.c_double)))
        return fu, fv, fw

    def deposits(self) -> np.ndarray:
        out = np.zeros((self.ncells, NDEP))
        lib().orc_get_deposits(self.h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def reduction_degree(self):
        mean = np.zeros(self.nbeds)
        oxy = np.zeros(self.nbeds)
        per = np.zeros(self.n)
        lib().orc_reduction_degree(self.h, mean.ctypes.data_as(C.POINTER(C.c_double)),
                                   oxy.ctypes.data_as(C.POINTER(C.c_double)),
                                   per.ctypes.data_as(C.POINTER(C.c_double)))
        return mean, oxy, per

    def set_kinetics(self, k0, Ea):
        a, ap = _d(k0)
        b, bp = _d(Ea)
        lib().orc_set_kinetics(self.h, ap, bp)

    def adjoint(self, nsteps: int, mode: int = 0, rel: float = 1e-6):
        J = np.zeros(1)
        g = np.zeros(6)
        st = lib().orc_adjoint(self.h, int(nsteps), int(mode), float(rel),
                               J.ctypes.data_as(C.POINTER(C.c_double)), g.ctypes.data_as(C.POINTER(C.c_double)))
        if st != 0:
            raise ValueError("the adjoint map is per parcel: not defined with radiation switched on")
        return float(J[0]), g


    def adjoint_obs(self, nsteps: int, obs_steps, weights=None, mode: int = 0):
        """Bed means of f_ov - f_ov(now) after each of obs_steps sub-steps of the frozen map,
        (n_obs, n_beds); mode 2 adds the dual-number gradient of sum(weights * J_obs)."""
        steps = np.ascontiguousarray(obs_steps, dtype=np.int32)
        nobs = int(steps.size)
        Jo = np.zeros((nobs, self.nbeds))
        g = np.zeros(6)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64).reshape(nobs, self.nbeds)
        st = lib().orc_adjoint_obs(self.h, int(nsteps), int(mode), nobs, steps.ctypes.data_as(C.POINTER(C.c_int32)),
                                   None if w is None else w.ctypes.data_as(C.POINTER(C.c_double)),
                                   Jo.ctypes.data_as(C.POINTER(C.c_double)), g.ctypes.data_as(C.POINTER(C.c_double)))
        if st != 0:
            raise ValueError("the adjoint map is per parcel: not defined with radiation or conduction")
        return Jo, (g if mode == 2 else None)


def set_threads(n: int):
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def gas_props(cfg, T, Y, p=None):
    bv, bp = _d(bed_vector(cfg))
    y, yp = _d(Y)
    out = np.zeros(NGP)
    lib().orc_gas_props(bp, float(T), yp, float(bv[_B["P0"]] if p is None else p),
                        out.ctypes.data_as(C.POINTER(C.c_double)))
    return dict(rho=out[GP_RHO], mu=out[GP_MU], lam=out[GP_LAM], cp=out[GP_CP], x=out[GP_X],
                xp=out[GP_XP:GP_XP + 3].copy(), Dm=out[GP_DM], Mg=out[GP_MG], D12=out[GP_D12],
                D13=out[GP_D13])


def network(A, B, F, active, x, xeq):
    a, ap = _d(A)
    b, bp = _d(B)
    act, actp = _i(active)
    xe, xep = _d(xeq)
    J = np.zeros(3)
    v = np.zeros(9)
    ao = np.zeros(3, dtype=np.int32)
    lib().orc_network(ap, bp, float(F), actp, float(x), xep, J.ctypes.data_as(C.POINTER(C.c_double)),
                      v.ctypes.data_as(C.POINTER(C.c_double)), ao.ctypes.data_as(C.POINTER(C.c_int32)))
    return J, v.reshape(3, 3), ao


def kinetics(cfg, m, Tp, d_real, ore, eps, slip, Tg, Y, dt_mass):
    bv, bp = _d(bed_vector(cfg))
    mm, mp = _d(m)
    y, yp = _d(Y)
    out = np.zeros(NK)
    lib().orc_kinetics(bp, mp, float(Tp), float(d_real), int(ore), float(eps), float(slip),
                       float(Tg), yp, float(dt_mass), out.ctypes.data_as(C.POINTER(C.c_double)))
    return dict(xidot=out[K_XIDOT:K_XIDOT + 3].copy(), mdot=out[K_MDOT:K_MDOT + 4].copy(),
                sH2=out[K_SH2], sH2O=out[K_SH2O], Qr=out[K_QR], Qrm=out[K_QRM],
                A=out[K_A:K_A + 3].copy(), B=out[K_B:K_B + 3].copy(), F=out[K_F], Sh=out[K_SH],
                f=out[K_F3:K_F3 + 3].copy(), act=out[K_ACT:K_ACT + 3].astype(int),
                EQ=out[K_EQ], ES=out[K_ES], Deff=out[K_DEFF:K_DEFF + 3].copy(),
                xi=out[K_XI:K_XI + 3].copy())


def drag(cfg, d_real, ore, eps, slip, Tg, Y):
    bv, bp = _d(bed_vector(cfg))
    y, yp = _d(Y)
    b = np.zeros(1)
    re = np.zeros(1)
    lib().orc_drag(bp, float(d_real), int(ore), float(eps), float(slip), float(Tg), yp,
                   b.ctypes.data_as(C.POINTER(C.c_double)), re.ctypes.data_as(C.POINTER(C.c_double)))
    return float(b[0]), float(re[0])


def heat(cfg, d_real, eps, slip, Tg, Y):
    bv, bp = _d(bed_vector(cfg))
    y, yp = _d(Y)
    nu = np.zeros(1)
    h = np.zeros(1)
    lib().orc_heat(bp, float(d_real), float(eps), float(slip), float(Tg), yp,
                   nu.ctypes.data_as(C.POINTER(C.c_double)), h.ctypes.data_as(C.POINTER(C.c_double)))
    return float(nu[0]), float(h[0])


def enthalpy(species, T):
    return lib().orc_enthalpy(SPECIES.index(species) if isinstance(species, str) else int(species), float(T))


def cp(species, T):
    return lib().orc_cp(SPECIES.index(species) if isinstance(species, str) else int(species), float(T))


def molar_mass(species):
    return lib().orc_molar_mass(SPECIES.index(species) if isinstance(species, str) else int(species))


def layer_porosity(cfg, ore):
    bv, bp = _d(bed_vector(cfg))
    out = np.zeros(3)
    lib().orc_layer_porosity(bp, int(ore), out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def _pairs(fn, x, y, z, r):
    n = len(x)
    xs = [_d(a) for a in (x, y, z, r)]
    cap = 64 * n + 16
    out = np.zeros(2 * cap, dtype=np.int32)
    np_ = fn(n, xs[0][1], xs[1][1], xs[2][1], xs[3][1], out.ctypes.data_as(C.POINTER(C.c_int32)), cap)
    if np_ > cap:
        raise RuntimeError("pair buffer too small")
    return out[:2 * np_].reshape(-1, 2)


def pairs_bruteforce(x, y, z, r):
    return _pairs(lib().orc_pairs_bruteforce, x, y, z, r)


def pairs_cells(x, y, z, r):
    return _pairs(lib().orc_pairs_cells, x, y, z, r)


def wall_distance(cfg, x, y, z):
    bv, bp = _d(bed_vector(cfg))
    dist = np.zeros(4)
    nrm = np.zeros(12)
    lib().orc_wall_distance(bp, float(x), float(y), float(z), dist.ctypes.data_as(C.POINTER(C.c_double)),
                            nrm.ctypes.data_as(C.POINTER(C.c_double)))
    return dist, nrm.reshape(4, 3)


def restitution_f(e):
    """f(e) of eqs (3-43), (3-44) (the reading: maximum overlap of a damped linear collision)."""
    return float(lib().orc_restitution_f(float(e)))


def e_cgp(e, k):
    """Restitution coefficient of a coarse-grained parcel, eq (3-45), clamped at 0."""
    return float(lib().orc_e_cgp(float(e), float(k)))


def conduction_pair(cfg, Ra, Rb, d, Ta, Tb, lam_a, lam_b, lam_g):
    """Heat into parcel a from parcel b in contact: dict(Qpp, Qpfp, Rc, I) (coarse-grained)."""
    bv, bp = _d(bed_vector(cfg))
    out = np.zeros(4)
    lib().orc_conduction_pair(bp, float(Ra), float(Rb), float(d), float(Ta), float(Tb), float(lam_a),
                              float(lam_b), float(lam_g), out.ctypes.data_as(C.POINTER(C.c_double)))
    return dict(Qpp=out[0], Qpfp=out[1], Rc=out[2], I=out[3])


def conduction_wall(cfg, R, h, Ta, lam_a, lam_g):
    """Heat into a parcel from the wall at distance h: dict(Qpp, Qpfp, Rc, I) (coarse-grained)."""
    bv, bp = _d(bed_vector(cfg))
    out = np.zeros(4)
    lib().orc_conduction_wall(bp, float(R), float(h), float(Ta), float(lam_a), float(lam_g),
                              out.ctypes.data_as(C.POINTER(C.c_double)))
    return dict(Qpp=out[0], Qpfp=out[1], Rc=out[2], I=out[3])


def pseudo_turbulence(eps, rho, mu, lam, cp, ug, up, dp):
    """Closures of eqs (3-28)..(3-37) for one cell: dict(Rpa, Rpe, apa, ape, s)."""
    a, ap = _d(ug)
    b, bp = _d(up)
    out = np.zeros(8)
    lib().orc_pseudo_turbulence(float(eps), float(rho), float(mu), float(lam), float(cp), ap, bp, float(dp),
                                out.ctypes.data_as(C.POINTER(C.c_double)))
    return dict(Rpa=out[0], Rpe=out[1], apa=out[2], ape=out[3], s=out[4:7].copy())
