"""ctypes binding of libdem_gb300.so: the C ABI of include/dem.h under the same names.

Argument marshalling only: every step of the particle path runs in the library's CUDA
kernels. PyTorch, where it is used, supplies device memory and the stream. If the
library is not built this module builds it (nvcc, sm_103a); if that fails the import
fails -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DEM_OK, DEM_EINVAL, DEM_ENOMEM, DEM_ECUDA, DEM_ECAPACITY, DEM_ENONFINITE, DEM_ETIMEOUT, DEM_ESTATE, DEM_EDOMAIN = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
DEM_PREC_FP64, DEM_PREC_SPLIT, DEM_PREC_SPLIT_KAHAN = 0, 1, 2
DEM_MAX_CONTACTS = 24
DEM_NSTATE, DEM_NGAS, DEM_NDEP, DEM_NDIAG, DEM_NFLOW = 20, 6, 14, 35, 4
DEM_NOALLOC_MAX_PARCELS = 8388608
PRECISIONS = {"fp64": DEM_PREC_FP64, "split": DEM_PREC_SPLIT, "split_kahan": DEM_PREC_SPLIT_KAHAN}
DEM_NTUNE = 11
TUNING_KEYS = ("neighbour_lists", "bs_key", "bs_restore", "bs_search", "bs_contacts", "bs_gas_particle", "bs_cells",
               "skin_permille", "restore_every", "gas_mg_sweeps", "gas_mg_weight_pct")

STATE_ROWS = ["x", "y", "z", "vx", "vy", "vz", "wx", "wy", "wz", "T", "m_h", "m_m", "m_w", "m_fe",
              "ax", "ay", "az", "alx", "aly", "alz"]
DIAG_ROWS = (["Fcx", "Fcy", "Fcz", "Tcx", "Tcy", "Tcz", "Fdx", "Fdy", "Fdz", "K", "Qconv", "Qr", "Qrm",
              "xidot0", "xidot1", "xidot2", "mdot0", "mdot1", "mdot2", "mdot3", "F_film", "A0", "A1",
              "A2", "B0", "B1", "B2", "Sh", "Nu", "Re", "ncontact", "cell", "Tse", "Qrad", "Qcond"])
SOURCE_ROWS = ["Vs", "SH2", "SH2O", "K", "Kvx", "Kvy", "Kvz", "hA", "hAT", "Qrm", "Qr", "EQ", "ES", "count"]


class DemBedConfig(C.Structure):
    _fields_ = [
        ("bed_D", C.c_double), ("bed_H", C.c_double), ("wall_kind", C.c_int32),
        ("cone_half_angle", C.c_double), ("cone_height", C.c_double), ("plate_z", C.c_double),
        ("hole_d", C.c_double), ("hole_pitch", C.c_double),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("dt", C.c_double), ("kn", C.c_double), ("kt_over_kn", C.c_double),
        ("restitution", C.c_double), ("mu_s", C.c_double), ("mu_r", C.c_double),
        ("cg_ratio", C.c_double), ("coupling_interval", C.c_int32),
        ("U_in", C.c_double), ("T_in", C.c_double), ("p0", C.c_double), ("Y_in", C.c_double * 3),
        ("k0", C.c_double * 3), ("Ea", C.c_double * 3), ("tortuosity", C.c_double),
        ("sphericity", C.c_double * 2), ("xi0", C.c_double * 2), ("pore_d_cm", C.c_double * 2),
        ("rho_true", C.c_double * 4), ("dpdz", C.c_double), ("eps_min", C.c_double),
        ("flags", C.c_uint32), ("emissivity", C.c_double),
        ("lambda_p", C.c_double * 2), ("lambda_wall", C.c_double),
    ]


class DemParcels(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("on_device", C.c_int32),
        ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
        ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p),
        ("d_real", C.c_void_p), ("T", C.c_void_p), ("m0", C.c_void_p * 4),
        ("ore_type", C.c_void_p), ("bed", C.c_void_p), ("id", C.c_void_p),
    ]


class DemGas(C.Structure):
    _fields_ = [("on_device", C.c_int32), ("Y", C.c_void_p), ("T", C.c_void_p)]


_lib = None


def lib() -> C.CDLL:
    """Load (building if needed) the CUDA library and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        path = _build.build()
    L = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)
    sig = {
        "dem_init": (C.c_int, [C.POINTER(DemBedConfig), C.c_int32, C.POINTER(DemParcels), C.POINTER(DemGas),
                               C.c_int32, vp, C.POINTER(vp)]),
        "dem_step": (C.c_int, [vp, C.c_int32]),
        "dem_step_graph": (C.c_int, [vp, C.c_int32]),
        "dem_sync": (C.c_int, [vp]),
        "dem_reduction_degree": (C.c_int, [vp, dp, dp, vp]),
        "dem_adjoint": (C.c_int, [vp, C.c_int32, C.c_int32, dp, dp]),
        "dem_adjoint_obs": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, ip, dp, dp, dp]),
        "dem_set_kinetics": (C.c_int, [vp, dp, dp]),
        "dem_get_state": (C.c_int, [vp, dp]),
        "dem_num_cells": (C.c_int64, [vp]),
        "dem_get_gas": (C.c_int, [vp, dp]),
        "dem_get_sources": (C.c_int, [vp, dp]),
        "dem_get_flow": (C.c_int, [vp, dp, C.POINTER(C.c_int32)]),
        "dem_get_sources_occupied": (C.c_int, [vp, C.c_int64, C.POINTER(C.c_int64), vp, vp]),
        "dem_get_contacts": (C.c_int, [vp, ip, ip, dp]),
        "dem_set_diagnostics": (C.c_int, [vp, C.c_int32]),
        "dem_get_diag": (C.c_int, [vp, dp]),
        "dem_autotune": (C.c_int, [vp, C.c_int32]),
        "dem_get_tuning": (C.c_int, [vp, C.POINTER(C.c_int32)]),
        "dem_set_tuning": (C.c_int, [vp, C.POINTER(C.c_int32)]),
        "dem_get_counters": (C.c_int, [vp, C.POINTER(C.c_int64)]),
        "dem_last_launch_count": (C.c_int64, [vp]),
        "dem_set_gas": (C.c_int, [vp, C.POINTER(DemGas)]),
        "dem_profile": (C.c_int, [vp, C.c_int32]),
        "dem_kernel_times": (C.c_int, [vp, C.c_int32, C.c_char_p, C.POINTER(C.c_int64), dp]),
        "dem_reduction_degree_noalloc": (C.c_int, [vp, vp, vp, vp, vp, C.c_int32, vp, vp]),
        "dem_strerror": (C.c_char_p, [C.c_int]),
        "dem_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class DemError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {lib().dem_strerror(status).decode()} ({status})")


def _check(status: int, what: str):
    if status != DEM_OK:
        raise DemError(status, what)


def bed_struct(cfg) -> DemBedConfig:
    c = cfg if isinstance(cfg, dict) else cfg.as_dict()
    s = DemBedConfig()
    s.bed_D, s.bed_H, s.wall_kind = c["D"], c["H"], c["wall_kind"]
    s.cone_half_angle, s.cone_height, s.plate_z = c["cone_half_angle"], c["cone_height"], c["plate_z"]
    s.hole_d, s.hole_pitch = c["hole_d"], c["hole_pitch"]
    s.nx, s.ny, s.nz = c["nx"], c["ny"], c["nz"]
    s.dt, s.kn, s.kt_over_kn = c["dt"], c["kn"], c["kt_over_kn"]
    s.restitution, s.mu_s, s.mu_r = c["restitution"], c["mu_s"], c["mu_r"]
    s.cg_ratio, s.coupling_interval = c["cg_ratio"], c["coupling_interval"]
    s.U_in, s.T_in, s.p0 = c["U_in"], c["T_in"], c["p0"]
    s.Y_in[:] = list(c["Y_in"])
    s.k0[:] = list(c["k0"])
    s.Ea[:] = list(c["Ea"])
    s.tortuosity = c["tortuosity"]
    s.sphericity[:] = list(c["sphericity"])
    s.xi0[:] = list(c["xi0"])
    s.pore_d_cm[:] = list(c["pore_d_cm"])
    s.rho_true[:] = list(c["rho_true"])
    s.dpdz, s.eps_min, s.flags = c["dpdz"], c["eps_min"], int(c["flags"])
    s.emissivity = c["emissivity"]
    s.lambda_p[:] = list(c["lambda_p"])
    s.lambda_wall = c["lambda_wall"]
    return s


def _ptr(a):
    """Data pointer of a numpy array or a torch tensor (no copy)."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Context:
    """One simulation: all beds and parcels of a synthetic or user workload.

    ``bed`` is a synth.Bed (numpy arrays, copied by dem_init). ``stream`` is a CUDA stream
    handle (int) or None for the legacy default stream.
    """

    def __init__(self, bed, precision="fp64", stream=None, gasY=None, gasT=None):
        L = lib()
        self.n = bed.n
        self.nbeds = len(bed.beds)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfgs = (DemBedConfig * self.nbeds)(*[bed_struct(c) for c in bed.beds])
        keep = []

        def arr(a, dt=np.float64):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data

        p = DemParcels()
        p.n = bed.n
        p.on_device = 0
        p.x, p.y, p.z = arr(bed.x), arr(bed.y), arr(bed.z)
        p.vx, p.vy, p.vz = arr(bed.vx), arr(bed.vy), arr(bed.vz)
        p.d_real, p.T = arr(bed.d_real), arr(bed.T)
        for q in range(4):
            p.m0[q] = arr(bed.m0[q])
        p.ore_type = arr(bed.ore, np.int32)
        p.bed = arr(bed.bed, np.int32)
        p.id = None
        g = None
        if gasY is not None:
            g = DemGas()
            g.on_device = 0
            g.Y = arr(gasY)
            g.T = arr(gasT)
        h = C.c_void_p()
        st = C.c_void_p(int(stream)) if stream else None
        rc = L.dem_init(cfgs, self.nbeds, C.byref(p), C.byref(g) if g is not None else None, prec, st,
                        C.byref(h))
        _check(rc, "dem_init")
        self.h = h
        self.ncells = int(L.dem_num_cells(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().dem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dem_step(self, n=1):
        _check(lib().dem_step(self.h, int(n)), "dem_step")

    def dem_step_graph(self, n=1):
        _check(lib().dem_step_graph(self.h, int(n)), "dem_step_graph")

    def dem_sync(self):
        _check(lib().dem_sync(self.h), "dem_sync")

    def dem_reduction_degree(self, per_parcel=None):
        """Bed means of f_ov (and removed-oxygen fractions); per_parcel: optional device
        tensor of n doubles that receives every parcel's f_ov in parcel-index order."""
        mean = np.zeros(self.nbeds)
        oxy = np.zeros(self.nbeds)
        _check(lib().dem_reduction_degree(self.h, mean.ctypes.data_as(C.POINTER(C.c_double)),
                                          oxy.ctypes.data_as(C.POINTER(C.c_double)),
                                          C.c_void_p(_ptr(per_parcel)) if per_parcel is not None else None),
               "dem_reduction_degree")
        return mean, oxy

    def dem_adjoint(self, nsteps, ckpt_every=100, want_grad=True):
        """(J, grad) of the frozen-position drag-heat-reaction map; grad is None when
        want_grad is False (forward sweep only)."""
        J = np.zeros(1)
        g = np.zeros(6)
        gp = g.ctypes.data_as(C.POINTER(C.c_double)) if want_grad else None
        _check(lib().dem_adjoint(self.h, int(nsteps), int(ckpt_every), J.ctypes.data_as(C.POINTER(C.c_double)), gp),
               "dem_adjoint")
        return float(J[0]), (g if want_grad else None)

    def dem_adjoint_obs(self, nsteps, obs_steps, weights=None, ckpt_every=100):
        """Observed bed reduction-degree curves J_obs (n_obs, n_beds) after obs_steps
        sub-steps of the frozen-position map, and (with weights, an (n_obs, n_beds) array)
        the gradient of sum(weights * J_obs) w.r.t. k0[3], Ea[3] (None without weights)."""
        steps = np.ascontiguousarray(obs_steps, dtype=np.int32)
        nobs = int(steps.size)
        Jo = np.zeros((nobs, self.nbeds))
        g = np.zeros(6) if weights is not None else None
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64).reshape(nobs, self.nbeds)
        _check(lib().dem_adjoint_obs(self.h, int(nsteps), int(ckpt_every), nobs,
                                     steps.ctypes.data_as(C.POINTER(C.c_int32)),
                                     None if w is None else w.ctypes.data_as(C.POINTER(C.c_double)),
                                     Jo.ctypes.data_as(C.POINTER(C.c_double)),
                                     None if g is None else g.ctypes.data_as(C.POINTER(C.c_double))),
               "dem_adjoint_obs")
        return Jo, g

    def dem_set_kinetics(self, k0, Ea):
        a = np.ascontiguousarray(k0, dtype=np.float64)
        b = np.ascontiguousarray(Ea, dtype=np.float64)
        _check(lib().dem_set_kinetics(self.h, a.ctypes.data_as(C.POINTER(C.c_double)),
                                      b.ctypes.data_as(C.POINTER(C.c_double))), "dem_set_kinetics")

    def dem_get_state(self):
        out = np.zeros((DEM_NSTATE, self.n))
        _check(lib().dem_get_state(self.h, out.ctypes.data_as(C.POINTER(C.c_double))), "dem_get_state")
        return out

    def dem_get_gas(self):
        out = np.zeros((self.ncells, DEM_NGAS))
        _check(lib().dem_get_gas(self.h, out.ctypes.data_as(C.POINTER(C.c_double))), "dem_get_gas")
        return out

    def dem_get_sources(self, out=None):
        """Cell sources of the last coupling step, (cells, DEM_NDEP) doubles. out: optional
        host buffer of that shape to fill (a page-locked torch tensor makes the copy fast)."""
        if out is None:
            out = np.zeros((self.ncells, DEM_NDEP))
        _check(lib().dem_get_sources(self.h, C.cast(C.c_void_p(_ptr(out)), C.POINTER(C.c_double))),
               "dem_get_sources")
        return out

    def dem_get_sources_occupied(self, cells=None, out=None):
        """Sources of the fluid cells that hold parcels: (cells int64 (k,), rows (k, DEM_NDEP)).
        cells, out: optional host buffers of capacity >= the count (page-locked torch tensors
        make the copies fast); views of their first k entries are returned."""
        cap = min(self.n, self.ncells)
        if cells is None:
            cells = np.zeros(cap, dtype=np.int64)
        if out is None:
            out = np.zeros((cap, DEM_NDEP))
        k = C.c_int64(0)
        cap_b = min(len(cells), len(out))
        _check(lib().dem_get_sources_occupied(self.h, cap_b, C.byref(k), C.c_void_p(_ptr(cells)),
                                              C.c_void_p(_ptr(out))), "dem_get_sources_occupied")
        return cells[:k.value], out[:k.value]

    def dem_get_flow(self):
        """Cell-centre gas velocity (3) and pressure relative to p0 of every cell,
        (cells, DEM_NFLOW) doubles, and the conjugate-gradient iterations of the last
        pressure solve (0 without the gas solver)."""
        out = np.zeros((self.ncells, DEM_NFLOW))
        it = C.c_int32(0)
        _check(lib().dem_get_flow(self.h, out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(it)), "dem_get_flow")
        return out, int(it.value)

    def dem_get_contacts(self):
        cnt = np.zeros(self.n, dtype=np.int32)
        partner = np.zeros((self.n, DEM_MAX_CONTACTS), dtype=np.int32)
        xi = np.zeros((self.n, DEM_MAX_CONTACTS, 3))
        _check(lib().dem_get_contacts(self.h, cnt.ctypes.data_as(C.POINTER(C.c_int32)),
                                      partner.ctypes.data_as(C.POINTER(C.c_int32)),
                                      xi.ctypes.data_as(C.POINTER(C.c_double))), "dem_get_contacts")
        return cnt, partner, xi

    def dem_set_diagnostics(self, on=True):
        _check(lib().dem_set_diagnostics(self.h, 1 if on else 0), "dem_set_diagnostics")

    def dem_get_diag(self):
        out = np.zeros((DEM_NDIAG, self.n))
        _check(lib().dem_get_diag(self.h, out.ctypes.data_as(C.POINTER(C.c_double))), "dem_get_diag")
        return out

    def dem_autotune(self, nsteps=30):
        _check(lib().dem_autotune(self.h, int(nsteps)), "dem_autotune")
        return self.dem_get_tuning()

    def dem_get_tuning(self):
        """Launch configuration: dict with the DEM_NTUNE values by name."""
        t = (C.c_int32 * DEM_NTUNE)()
        _check(lib().dem_get_tuning(self.h, t), "dem_get_tuning")
        return dict(zip(TUNING_KEYS, [int(v) for v in t]))

    def dem_set_tuning(self, **kw):
        """Change named entries of the launch configuration (see TUNING_KEYS)."""
        cur = self.dem_get_tuning()
        for k, v in kw.items():
            if k not in cur:
                raise KeyError(k)
            cur[k] = int(v)
        t = (C.c_int32 * DEM_NTUNE)(*[cur[k] for k in TUNING_KEYS])
        _check(lib().dem_set_tuning(self.h, t), "dem_set_tuning")

    def dem_get_counters(self):
        """(steps taken, neighbour-list builds, list entries at the last build) since dem_init."""
        v = (C.c_int64 * 3)()
        _check(lib().dem_get_counters(self.h, v), "dem_get_counters")
        return int(v[0]), int(v[1]), int(v[2])

    def dem_set_gas(self, Y, T):
        """Y: (cells, 3) mass fractions, T: (cells,) temperatures; numpy (host, ideally pinned)
        or torch CUDA tensors (device)."""
        g = DemGas()
        g.on_device = 1 if hasattr(Y, "is_cuda") and Y.is_cuda else 0
        g.Y = _ptr(Y)
        g.T = _ptr(T)
        _check(lib().dem_set_gas(self.h, C.byref(g)), "dem_set_gas")

    def dem_profile(self, on=True):
        _check(lib().dem_profile(self.h, 1 if on else 0), "dem_profile")

    def dem_kernel_times(self):
        """{kernel name: (launches, total ms)} since profiling was switched on."""
        m = 64
        names = C.create_string_buffer(32 * m)
        n = np.zeros(m, dtype=np.int64)
        t = np.zeros(m)
        k = lib().dem_kernel_times(self.h, m, names, n.ctypes.data_as(C.POINTER(C.c_int64)),
                                   t.ctypes.data_as(C.POINTER(C.c_double)))
        if k < 0:
            raise DemError(k, "dem_kernel_times")
        out = {}
        for i in range(k):
            nm = names.raw[32 * i:32 * (i + 1)].split(b"\0")[0].decode()
            out[nm] = (int(n[i]), float(t[i]))
        return out

    def dem_last_launch_count(self):
        return int(lib().dem_last_launch_count(self.h))
