// common.cuh -- device-side constants, per-bed parameters and the physics of one parcel.
//
// The arithmetic of forces, drag, heat and kinetics follows a precision policy P:
//   PrecF64   -- everything in FP64 (the all-FP64 form);
//   PrecSplit -- FP32 physics; FP64 positions, layer masses and cell-source sums;
//   PrecKahan -- as PrecSplit, but masses and cell sums as Kahan-compensated FP32 pairs.
// GB300 issues only a few FP64 operations per SM per clock, so in the FP32 forms every
// constant and table is prepared in FP32 on the host and the device code avoids FP64
// except where a result accumulates (positions, masses, cell sums, the gas state).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dem.h"
#include "pdl.cuh"

namespace dem {

constexpr int KMAX = DEM_MAX_CONTACTS;
// candidate list of the pair search (per thread, shared memory): live contacts plus the few
// extra candidates of the exact form's FP32 prefilter
constexpr int KLIST = KMAX + 8;
constexpr double kPI = 3.14159265358979323846;
constexpr double kRgas = 8.314;  // gas constant of Sec. 2.1
constexpr double kGrav = 9.81;
constexpr double kSigmaSB = 5.67e-8;   // Stefan-Boltzmann constant printed with eq (3-16), W/m^2/K^4

// kahan: layer masses and positions are compensated FP32 pairs (no FP64 arithmetic in the
// step); exact: the FP64 form, whose pair tests follow the oracle bit for bit
struct PrecF64 { using R = double; static constexpr bool kahan = false; static constexpr bool exact = true; };
struct PrecSplit { using R = float; static constexpr bool kahan = false; static constexpr bool exact = false; };
struct PrecKahan { using R = float; static constexpr bool kahan = true; static constexpr bool exact = false; };

enum : int { ERR_CAPACITY = 1, ERR_NONFINITE = 2, ERR_DOMAIN = 4, ERR_TIMEOUT = 8 };

// per-cell gas properties (derived from the gas state by gas_cell_props), stored cell by
// cell in records of GP_STRIDE words, so that a parcel reads its cell's record in a few
// vector loads; the gas velocity (GP_UX, GP_UY, GP_UZ) is the prescribed plug flow, or the
// cell-centre velocity of the solved gas
enum : int {
  GP_RHO = 0, GP_MU, GP_LAM, GP_CP, GP_X, GP_DM, GP_SC13, GP_PR13, GP_EPOW, GP_D0, GP_D1,
  GP_UZ, GP_EPS, GP_TG, GP_UX, GP_UY, GP_N, GP_STRIDE = 16
};
static_assert((int)GP_N <= (int)GP_STRIDE, "property record");
// gas state rows (double)
enum : int { GS_EPS = 0, GS_Y0, GS_Y1, GS_Y2, GS_T, GS_N };
// per-parcel source rows
enum : int {
  SR_VS = 0, SR_SH2, SR_SH2O, SR_K, SR_KVX, SR_KVY, SR_KVZ, SR_HA, SR_HAT, SR_QRM, SR_QR, SR_EQ,
  SR_ES, SR_CNT, SR_N
};
static_assert((int)SR_N == (int)DEM_NDEP, "source rows");
// diagnostics rows (same order as documented in dem.h)
enum : int {
  DG_FC = 0, DG_TC = 3, DG_FD = 6, DG_K = 9, DG_QCONV, DG_QR, DG_QRM, DG_XIDOT = 13, DG_MDOT = 16,
  DG_FFILM = 20, DG_A = 21, DG_B = 24, DG_SH = 27, DG_NU, DG_RE, DG_NCONTACT, DG_CELL, DG_TSE, DG_QRAD,
  DG_QCOND, DG_N
};
static_assert((int)DG_N == (int)DEM_NDIAG, "diag rows");

// Geometry of a bed in FP64 (positions, grid, walls, gas state). The gas cells are also
// the cell list of the contact search (init checks that no parcel is wider than a cell).
struct DevBed {
  double x0, y0, z0, dx, dy, dz, inv_dx, inv_dy, inv_dz, vcell, inv_vcell;
  int nx, ny, nz;
  long long cell_off;           // first global gas cell (and sort key) of this bed
  int pstart, pend;             // storage positions of this bed's parcels (fixed: beds are stored
                                // in bed order after the first binning and parcels never change bed)
  int corner_off;               // first entry of this bed in the cell-corner table
  int cornerp_off;              // the same in the FP32-pair table (nx+1, ny+1, nz+1 entries)
  float inv_nx_f, inv_nxy_f;    // 1/nx, 1/(nx ny): cell offsets from key differences
  int fast_offsets;             // nx, ny >= 5: offsets in [-2, 2] decode by rounding
  double R_bed, H, cos_a, sin_a, z_apex, plate_z, pitch, inv_pitch, r_hole;
  int wall;
  double dt, k;
  int ncouple;
  double U_in, T_in, p0, Y_in[3], eps_min;
  unsigned flags;
  long long fx_off, fy_off, fz_off;   // first x-, y-, z-face of this bed (solved gas)
};

// Physics parameters of a bed in the form's arithmetic type R (prepared on the host).
template <class R> struct BedP {
  R k, k3, inv_k3, dt, half_dt, kn, kt, eta_coef, eta_t_ratio, mu_s, mu_r;
  R x0, y0, z0, dx, dy, dz, inv_dx, inv_dy, inv_dz;   // grid (cell-local coordinates)
  R R_bed, H, cos_a, sin_a, z_apex, plate_z, pitch, inv_pitch, r_hole;   // walls
  R U_in, p0, T_in, Y_in[3], eps_min, inv_vcell;
  R k0[3], Ea_R[3], inv_tau;
  R psi[2], K1b[2], K2[2], wall_K1;   // Ganser constants; wall_K1 = 2.25 / D
  R xi[2][3];                   // product-layer porosity per ore: m, w, Fe (eqs (2-31)..(2-36))
  R pore_cm[2], DKc[2];         // pore diameter (cm) and 0.97 r_a of eq (2-28)
  R fuller12, fuller13, mfp_c;  // eq (2-26) without T and p; 1.013 / p of Sec. 2.3
  R rate_c;                     // pi p0 / R_g (molar-rate prefactor of eq (2-1) without d^2 / T)
  R dpdz, grav, dtg;
  R pf_margin;                  // prefilter margin of the exact (FP64) pair test, m
  R reach_max;                  // largest parcel radius of the bed (CGP), m
  R skin, half_skin2;           // neighbour-list skin (m) and (skin / 2)^2
  R rad_c;                      // k^3 sigma eta_p pi: eqs (3-16) and (3-51) without d_p^2 and the temperatures
  // contact conduction (eqs (3-14)..(3-15-2) with the scaling of eqs (3-46), (3-48)..(3-48-2)):
  R cond_pp;                    // 4 k^(3/4) sqrt(f(e) / f(e_CGP)): eq (3-46) times the 4 of eq (3-14)
  R cond_pf;                    // 2 pi k^2: eq (3-48) times the 2 pi of eq (3-15)
  R lam_e[2][2], lam_ew[2];     // series conductances lambda_a lambda_b / (lambda_a + lambda_b), and with the wall
  R lmin;                       // smallest conducting gap: 1.013 / p0 cm (Sec. 2.3), m
  unsigned flags;
  int ncouple, wall;
};

// Constant tables in the form's arithmetic type.
template <class R> struct Tab {
  R Mz[4], Mj[3], Ka[3], Kb[3], RMz[4], RMj[3];   // molar masses, Table 2, R_g / M
  R nasaT[7];
  R h[7][2][6];                 // Table C1: a1, a2/2, a3/3, a4/4, a5/5, a6 (enthalpy / R)
  R cp[7][2][5];                // Table C1: a1..a5 (heat capacity / R)
  R dcp[7][2][4];               // derivative of the heat-capacity polynomial
  R visc[3][3], cond[3][5];     // Tables C2, C3
};

// Molar masses (kg/mol): solids Fe2O3, Fe3O4, FeO, Fe; gases H2, H2O, N2.
constexpr double kMz[4] = {159.69e-3, 231.533e-3, 71.844e-3, 55.845e-3};
constexpr double kMj[3] = {2.016e-3, 18.015e-3, 28.014e-3};
constexpr double kKa[3] = {1433.4, -7393.9, -2023.8};   // Table 2: K_eq = exp(a / T + b)
constexpr double kKb[3] = {9.08, 7.56, 1.24};
// Table C1, two ranges per species (H2, H2O, N2, Fe2O3, Fe3O4, FeO, Fe); the Fe ranges
// 1000-1184 K are represented by the 298-1000 K range (see the design notes)
constexpr double kNasaT[7] = {1000.0, 1000.0, 1000.0, 960.0, 850.0, 1000.0, 1184.0};
constexpr double kNasa[7][2][6] = {
  {{2.3443, 7.98e-3, -1.95e-5, 2.02e-8, -7.38e-12, -9.179e2}, {2.9328, 8.27e-4, -1.46e-7, 1.54e-11, -6.89e-16, -8.131e2}},
  {{4.1986, -2.04e-3, 6.52e-6, -5.49e-9, 1.77e-12, -3.03e4}, {2.677, 2.97e-3, -7.74e-7, 9.44e-11, -4.27e-15, -2.989e4}},
  {{3.531, -1.24e-4, -5.03e-7, 2.44e-9, -1.41e-12, -1.047e3}, {2.9526, 1.40e-3, -4.93e-7, 7.86e-11, -4.61e-15, -9.239e2}},
  {{0.1522, 6.71e-2, -1.13e-4, 9.93e-8, -3.28e-11, -1.013e5}, {353.05, -0.9728, 1.05e-3, -4.96e-7, 8.74e-11, -1.96e5}},
  {{4.8445, 4.39e-2, 5.25e-5, -2.21e-7, 1.75e-10, -1.38e5}, {88.431, -0.149, 1.26e-4, -4.7e-8, 6.79e-12, -1.621e5}},
  {{5.3195, 2.21e-3, 1.07e-6, -2.79e-9, 1.33e-12, -3.441e4}, {5.8316, 1.43e-3, -9.32e-8, -6.6e-12, -2.25e-14, -3.457e4}},
  {{2.4134, -1.58e-3, 2.15e-5, -3.8e-8, 2.20e-11, -774.38}, {61.011, -0.161, 1.68e-4, -7.75e-8, 1.33e-11, -1.65e4}},
};
constexpr double kVisc[3][3] = {{2.85e-6, 2.16e-8, -3.78e-12}, {-4.44e-6, 4.52e-8, -3.20e-12}, {7.86e-6, 3.87e-8, -5.11e-12}};
constexpr double kCond[3][5] = {{3.07e-3, 8.09e-4, -8.52e-7, 7.2e-10, -2.21e-13},
                                {6.84e-3, 6.25e-6, 1.31e-7, -5.99e-11, 1.12e-14},
                                {2.51e-3, 8.92e-5, -4.00e-8, 1.62e-11, -2.61e-15}};

template <class R> constexpr Tab<R> make_tab() {
  Tab<R> t{};
  for (int z = 0; z < 4; ++z) { t.Mz[z] = (R)kMz[z]; t.RMz[z] = (R)(kRgas / kMz[z]); }
  for (int j = 0; j < 3; ++j) { t.Mj[j] = (R)kMj[j]; t.RMj[j] = (R)(kRgas / kMj[j]); }
  for (int r = 0; r < 3; ++r) { t.Ka[r] = (R)kKa[r]; t.Kb[r] = (R)kKb[r]; }
  for (int s = 0; s < 7; ++s) {
    t.nasaT[s] = (R)kNasaT[s];
    for (int g = 0; g < 2; ++g) {
      const double *a = kNasa[s][g];
      t.h[s][g][0] = (R)a[0];
      t.h[s][g][1] = (R)(a[1] / 2.0);
      t.h[s][g][2] = (R)(a[2] / 3.0);
      t.h[s][g][3] = (R)(a[3] / 4.0);
      t.h[s][g][4] = (R)(a[4] / 5.0);
      t.h[s][g][5] = (R)a[5];
      for (int k = 0; k < 5; ++k) t.cp[s][g][k] = (R)a[k];
      for (int k = 0; k < 4; ++k) t.dcp[s][g][k] = (R)((k + 1) * a[k + 1]);
    }
  }
  for (int j = 0; j < 3; ++j) {
    for (int k = 0; k < 3; ++k) t.visc[j][k] = (R)kVisc[j][k];
    for (int k = 0; k < 5; ++k) t.cond[j][k] = (R)kCond[j][k];
  }
  return t;
}

static __constant__ Tab<float> cTabF = make_tab<float>();
static __constant__ Tab<double> cTabD = make_tab<double>();
template <class R> __device__ __forceinline__ const Tab<R> &tab();
template <> __device__ __forceinline__ const Tab<float> &tab<float>() { return cTabF; }
template <> __device__ __forceinline__ const Tab<double> &tab<double>() { return cTabD; }

// ---------------------------------------------------------------------------------------
// Thermochemistry (eqs (3-22), (3-23)): molar enthalpy / R and molar heat capacity / R.
// Species index s: 0 H2, 1 H2O, 2 N2, 3 Fe2O3, 4 Fe3O4, 5 FeO, 6 Fe.
// ---------------------------------------------------------------------------------------
// Elementary functions in the form's arithmetic type. The FP64 form uses the libm
// functions and IEEE division; the FP32 forms use the hardware approximations (__expf,
// __logf, reciprocal-based division: errors of a few ulp, or ~1e-6 relative for exp of
// arguments up to ~20), far inside those forms' 1e-4 tolerance against the FP64 oracle.
template <class R> __device__ __forceinline__ R fexp(R x) {
  if constexpr (sizeof(R) == 8) return exp(x); else return __expf(x);
}
template <class R> __device__ __forceinline__ R flog(R x) {
  if constexpr (sizeof(R) == 8) return log(x); else return __logf(x);
}
// cube root of x >= 0 (FP32: exp(log(x) / 3))
template <class R> __device__ __forceinline__ R fcbrt(R x) {
  if constexpr (sizeof(R) == 8) return cbrt(x); else return __expf(__logf(x) * (1.0f / 3.0f));
}
template <class R> __device__ __forceinline__ R fdiv(R a, R b) {
  if constexpr (sizeof(R) == 8) return a / b; else return __fdividef(a, b);
}
template <class R> __device__ __forceinline__ R frcp(R x) {
  if constexpr (sizeof(R) == 8) return 1.0 / x; else return __fdividef(1.0f, x);
}

// The NASA polynomials of Table C1 (two temperature ranges per species). In the FP32 forms
// both ranges are evaluated and the result is selected: a range chosen before the loads would
// make the coefficients' constant-memory address differ between the threads of a warp (whose
// parcels straddle the range boundary) and serialise the loads, which took 15 % of the
// gas-particle kernel; with both ranges every load is warp-uniform. The arithmetic of the
// chosen range is the same either way, so are the results. The FP64 form, whose FP64 pipe
// is narrow, evaluates only the chosen range.
template <class R> __device__ __forceinline__ R h_poly(const R *a, R T) {
  return T * (a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])))) + a[5];
}
template <class R> __device__ __forceinline__ R cp_poly(const R *a, R T) {
  return a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
}
template <class R> __device__ __forceinline__ R dcp_poly(const R *a, R T) {
  return a[0] + T * (a[1] + T * (a[2] + T * a[3]));
}
template <class R> __device__ __forceinline__ R h_over_R(int s, R T) {
  const Tab<R> &t = tab<R>();
  if constexpr (sizeof(R) == 4) {
    const R lo = h_poly(t.h[s][0], T), hi = h_poly(t.h[s][1], T);
    return T <= t.nasaT[s] ? lo : hi;
  } else {
    return h_poly(t.h[s][T <= t.nasaT[s] ? 0 : 1], T);
  }
}
template <class R> __device__ __forceinline__ R cp_over_R(int s, R T) {
  const Tab<R> &t = tab<R>();
  if constexpr (sizeof(R) == 4) {
    const R lo = cp_poly(t.cp[s][0], T), hi = cp_poly(t.cp[s][1], T);
    return T <= t.nasaT[s] ? lo : hi;
  } else {
    return cp_poly(t.cp[s][T <= t.nasaT[s] ? 0 : 1], T);
  }
}
template <class R> __device__ __forceinline__ R dcp_over_R(int s, R T) {
  const Tab<R> &t = tab<R>();
  if constexpr (sizeof(R) == 4) {
    const R lo = dcp_poly(t.dcp[s][0], T), hi = dcp_poly(t.dcp[s][1], T);
    return T <= t.nasaT[s] ? lo : hi;
  } else {
    return dcp_poly(t.dcp[s][T <= t.nasaT[s] ? 0 : 1], T);
  }
}

// ---------------------------------------------------------------------------------------
// Gas-cell properties (eqs (2-1-1), (2-1-2), (2-26)..(2-29), (3-53)..(3-59)), once per cell.
// ---------------------------------------------------------------------------------------
template <class R> struct CellProps {
  R rho, mu, lam, cp, x, Dm, sc13, pr13, epow, D[2], uz, eps, T, ux, uy;
};

// mean molar mass, density (eq (3-53)) and heat capacity (eq (3-57)) of the gas: shared by the
// property record and by the gas update, which recomputes them instead of reading the record
template <class R> __device__ __forceinline__ R gas_molar_mass(const R Y[3]) {
  const Tab<R> &t = tab<R>();
  return frcp<R>(fdiv<R>(Y[0], t.Mj[0]) + fdiv<R>(Y[1], t.Mj[1]) + fdiv<R>(Y[2], t.Mj[2]));
}
template <class R> __device__ __forceinline__ R gas_density(const BedP<R> &B, R Mg, R T) {
  return fdiv<R>(Mg * B.p0, (R)kRgas * T);
}
template <class R> __device__ __forceinline__ R gas_heat_capacity(const R Y[3], R T) {
  const Tab<R> &t = tab<R>();
  R cp = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) cp += Y[j] * cp_over_R<R>(j, T) * t.RMj[j];
  return cp;
}

template <class R>
__device__ inline CellProps<R> gas_cell_props(const BedP<R> &B, R eps, const R Y[3], R T) {
  const Tab<R> &t = tab<R>();
  CellProps<R> o;
  const R p = B.p0;
  const R Mg = gas_molar_mass<R>(Y);
  const R xp0 = fdiv<R>(Y[0] * Mg, t.Mj[0]), xp1 = fdiv<R>(Y[1] * Mg, t.Mj[1]), xp2 = fdiv<R>(Y[2] * Mg, t.Mj[2]);
  const R den = xp0 + xp1;
  o.x = den > (R)0 ? fdiv<R>(xp0, den) : (R)0;
  o.rho = gas_density<R>(B, Mg, T);
  R mu = 0, lam = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    mu += Y[j] * (t.visc[j][0] + T * (t.visc[j][1] + T * t.visc[j][2]));
    lam += Y[j] * (t.cond[j][0] + T * (t.cond[j][1] + T * (t.cond[j][2] + T * (t.cond[j][3] + T * t.cond[j][4]))));
  }
  const R cp = gas_heat_capacity<R>(Y, T);
  o.mu = mu; o.lam = lam; o.cp = cp;
  // Fuller binary coefficients D(H2,H2O), D(H2,N2) (T^1.75 = T sqrt(T) sqrt(sqrt(T))) and
  // Wilke's rule for H2 (its 0/0 limit in pure H2 is the binary coefficient)
  const R sT = sqrt(T);
  const R tf = T * sT * sqrt(sT) * ((R)101325 / p) * (R)1e-7;
  const R D12 = tf * B.fuller12, D13 = tf * B.fuller13;
  const R rest = (R)1 - xp0;
  o.Dm = rest < (R)1e-12 ? D12 : fdiv<R>(rest, fdiv<R>(xp1, D12) + fdiv<R>(xp2, D13));
  o.sc13 = fcbrt<R>(fdiv<R>(mu, o.rho * o.Dm));
  o.pr13 = fcbrt<R>(fdiv<R>(cp * mu, lam));
  o.epow = fexp<R>((R)-2.65 * flog<R>(eps));
  // pore diffusion per ore: molecular, Knudsen, or Bosanquet by lambda / d_a (Sec. 2.3)
  const R mfp = o.x > (R)0 ? B.mfp_c / o.x : (R)3e38;
  const R sq = sqrt(T / (t.Mj[0] * (R)1e3));
#pragma unroll
  for (int ore = 0; ore < 2; ++ore) {
    const R DK = B.DKc[ore] * sq;
    const R ratio = mfp / B.pore_cm[ore];
    o.D[ore] = ratio <= (R)0.01 ? o.Dm : (ratio >= (R)10 ? DK : frcp<R>(frcp<R>(o.Dm) + frcp<R>(DK)));
  }
  o.uz = fdiv<R>(B.U_in, eps);
  o.ux = (R)0;
  o.uy = (R)0;
  o.eps = eps;
  o.T = T;
  return o;
}

// ---------------------------------------------------------------------------------------
// Per-parcel gas-side terms.
// ---------------------------------------------------------------------------------------
template <class R> struct Gas {   // a cell's properties in the parcel's arithmetic type
  R rho, mu, lam, cp, x, Dm, sc13, pr13, epow, D, uz, eps, T, ux, uy;
};

template <class R> __device__ __forceinline__ R pos_pow(R x, R e) {   // x^e for x >= 0
  return x > (R)0 ? fexp<R>(e * flog<R>(x)) : (R)0;
}

// Gunn correlation (eqs (2-22), (3-12)); c13 is Sc^(1/3) or Pr^(1/3), re02 = Re^0.2
template <class R> __device__ __forceinline__ R gunn(R eps, R re02, R re07, R c13) {
  return ((R)7 - (R)10 * eps + (R)5 * eps * eps) * ((R)1 + (R)0.7 * re02 * c13) +
         ((R)1.33 - (R)2.4 * eps + (R)1.2 * eps * eps) * re07 * c13;
}

// Gidaspow-Ganser drag coefficient divided by the solid fraction (eqs (3-5-2)..(3-5-5)):
// F_d = (beta / eps_p) V_p (u_g - v_p), the form of eq (3-5) with eps_p cancelled. The
// inertial Ergun term carries eps_p (Gidaspow's correlation, which eq (3-5-1) cites, and
// Ergun's fixed-bed pressure drop), so it is 1.75 rho |u - v| / (d psi) after the division.
// Contact conduction of a parcel pair (radii Ra, Rb, centre distance d, overlap
// delta = Ra + Rb - d > 0), into the parcel at temperature Ta from the one at Tb: the
// constriction term of eq (3-14) with the radius R_c of the circle in which the spheres
// meet, and the fluid lens of eq (3-15) over the smaller sphere's disk down to the gap lmin,
// both scaled by eqs (3-46), (3-48). The lens integral is taken in closed form: with
// v = d - L (L the gap between the surfaces) the printed integrand R dR / L becomes the
// rational (v^4 - D^2) / (4 v^3 (d - v)) dv, D = Rb^2 - Ra^2 (Ra the smaller radius), over
// v from sqrt(D) (the rim of the smaller sphere) to d - lmin.
template <class R>
__device__ __forceinline__ R lens_pair(R Ra, R Rb, R d, R lmin) {
  const R a = fmin(Ra, Rb), b = fmax(Ra, Rb);
  const R D = (b - a) * (b + a);
  const R v0 = sqrt(D), v1 = d - lmin;
  const R top = d - v0;                      // the gap at the rim of the smaller sphere
  if (!(top > lmin)) return (R)0;
  const R lg = log(top / lmin);              // ln((d - v0) / (d - v1))
  R I = d * lg - (v1 - v0);
  if (D > (R)0) {
    const R id = (R)1 / d, iv0 = (R)1 / v0, iv1 = (R)1 / v1;
    I -= D * D * (id * id * id * (log(v1 / v0) + lg) + id * id * (iv0 - iv1) +
                  (R)0.5 * id * (iv0 * iv0 - iv1 * iv1));
  }
  return (R)0.25 * I;
}
template <class R>
__device__ __forceinline__ R conduction_pair(const BedP<R> &B, R Ra, R Rb, R d, R delta, R Ta, R Tb, R lam_e,
                                             R lam_g) {
  const R Rc = sqrt(fmax(delta * (d + Ra + Rb) * ((d + Ra) - Rb) * ((d - Ra) + Rb), (R)0)) / ((R)2 * d);
  return (B.cond_pp * Rc * lam_e + B.cond_pf * lam_g * lens_pair<R>(Ra, Rb, d, B.lmin)) * (Tb - Ta);
}
// the same with a wall at distance h = Rp - delta (plane, cone or rim; delta taken in FP64 by
// the caller): R_c of the sphere's cut by the wall's tangent plane, the lens over the whole sphere's disk in closed form,
// h ln(h / lmin) - (h - lmin) (eqs (3-15-1), (3-15-2), (3-48-1), (3-48-2))
template <class R>
__device__ __forceinline__ R conduction_wall(const BedP<R> &B, R Rp, R h, R delta, R Ta, R lam_ew, R lam_g) {
  const R Rc = sqrt(fmax(delta * ((R)2 * Rp - delta), (R)0));
  const R I = h > B.lmin ? h * log(h / B.lmin) - (h - B.lmin) : (R)0;
  return (B.cond_pp * Rc * lam_ew + B.cond_pf * lam_g * I) * (B.T_in - Ta);
}

template <class R>
__device__ __forceinline__ R beta_over_epsp(const BedP<R> &B, int ore, R d, const Gas<R> &g, R slip, R Re) {
  const R eps = g.eps, ep = (R)1 - eps;
  const R psi = B.psi[ore];
  if (eps < (R)0.8)
    return fdiv<R>((R)150 * ep * g.mu, eps * d * d * psi * psi) + fdiv<R>((R)1.75 * g.rho * slip, d * psi);
  const R K1 = B.K1b[ore] - B.wall_K1 * d;
  const R K2 = B.K2[ore];
  if (Re > (R)0) {
    const R RK = Re * (K1 * K2);
    const R CD = fdiv<R>((R)24, Re * K1) * ((R)1 + (R)0.1118 * pos_pow(RK, (R)0.6567)) +
                 fdiv<R>((R)0.4305 * K2, (R)1 + fdiv<R>((R)3305, RK));
    return fdiv<R>((R)0.75 * CD * eps * g.rho * slip, d) * g.epow;
  }
  return (R)0.75 * fdiv<R>((R)24 * g.mu, K1 * d * d) * g.epow;
}

// ---------------------------------------------------------------------------------------
// USCM kinetics of one parcel (Sec. 2), per real particle, then scaled by k^3.
// The resistance network of Fig. 2(a) is solved in closed form in terms of the interface
// conductances g_kl = 1/A_kl (an inactive reaction has g = 0): these are eqs (2-2)..(2-10)
// multiplied through by g_hm g_mw g_wFe, with the three-reaction determinant as W.
// ---------------------------------------------------------------------------------------
template <class R> struct KinOut {
  R xidot[3], mdot[4], sH2, sH2O, Qr, Qrm, EQ, ES, A[3], B[3], F, Sh;
};

template <class R>
__device__ __forceinline__ void uscm(const BedP<R> &Bd, const R m[4], R Tp, R d, int ore,
                                     const Gas<R> &g, R re02, R re07, R dtm, KinOut<R> &o) {
  const Tab<R> &t = tab<R>();
  const unsigned fl = Bd.flags;
#pragma unroll
  for (int r = 0; r < 3; ++r) { o.xidot[r] = 0; o.A[r] = 0; o.B[r] = 0; }
#pragma unroll
  for (int z = 0; z < 4; ++z) o.mdot[z] = 0;
  o.sH2 = o.sH2O = o.Qr = o.Qrm = o.EQ = o.ES = o.F = o.Sh = 0;
  R n[4];
#pragma unroll
  for (int z = 0; z < 4; ++z) n[z] = fdiv<R>(m[z] * Bd.inv_k3, t.Mz[z]);
  const R nfe = (R)2 * n[0] + (R)3 * n[1] + n[2] + n[3];
  if (!(nfe > (R)0)) return;
  const R inv_nfe = frcp<R>(nfe);
  // 1 - f of eqs (2-15)..(2-17), written as the iron fractions still behind each front
  R om[3];
  om[0] = (R)2 * n[0] * inv_nfe;
  om[1] = ((R)2 * n[0] + (R)3 * n[1]) * inv_nfe;
  om[2] = ((R)2 * n[0] + (R)3 * n[1] + n[2]) * inv_nfe;
  const R invT = frcp<R>(Tp);
  R xeq[3], gk[3], c3[3];
  bool act[3];
  const bool kin = !(fl & DEM_NO_KINETICS);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const R K = fexp<R>(t.Ka[r] * invT + t.Kb[r]);             // Table 2
    xeq[r] = frcp<R>(K + (R)1);                                  // eq (2-1-3)
    const R kr = Bd.k0[r] * fexp<R>(-Bd.Ea_R[r] * invT);         // eq (2-13)
    c3[r] = fcbrt<R>(om[r]);
    act[r] = kin && n[r] > (R)0 && g.x > xeq[r] && Bd.k0[r] > (R)0;
    // 1/A of eq (2-12): k_r (1-f)^(2/3) (1 + K)/K
    gk[r] = act[r] ? kr * c3[r] * c3[r] * ((R)1 + frcp<R>(K)) : (R)0;
  }
  // product-layer resistances, eq (2-14), with D_eff of eq (2-30)
  const R rp_tau = fdiv<R>((R)0.5 * d, g.D * Bd.inv_tau);
  R Bm = 0, Bw = 0, BFe = 0;
  if (!(fl & DEM_NO_LAYER)) {
    const R ic0 = frcp<R>(c3[0]), ic1 = frcp<R>(c3[1]), ic2 = frcp<R>(c3[2]);
    if (act[0]) Bm = fdiv<R>(rp_tau, Bd.xi[ore][0]) * (ic0 - ic1);
    if ((act[0] || act[1]) && om[1] > (R)0) Bw = fdiv<R>(rp_tau, Bd.xi[ore][1]) * (ic1 - ic2);
    if (om[2] > (R)0) BFe = fdiv<R>(rp_tau, Bd.xi[ore][2]) * (ic2 - (R)1);
  }
  // gas film, eqs (2-20)..(2-24)
  o.Sh = gunn(g.eps, re02, re07, g.sc13);
  const R F = (fl & DEM_NO_FILM) ? (R)0 : fdiv<R>(d, o.Sh * g.Dm);
#pragma unroll
  for (int r = 0; r < 3; ++r) o.A[r] = gk[r] > (R)0 ? frcp<R>(gk[r]) : (R)0;
  // closed-form network; a reaction whose flux is negative is dropped and the rest re-solved
  const R S = F + BFe, BwS = Bw + S;
  R J[3] = {0, 0, 0}, vsum[3] = {0, 0, 0};
  for (int it = 0; it < 3; ++it) {
    const R g1 = gk[0], g2 = gk[1], g3 = gk[2];
    const R a1 = (R)1 + Bm * g1;
    const R W = a1 * ((R)1 + BwS * g2 + S * g3 * ((R)1 + Bw * g2)) + g1 * (BwS + Bw * S * g3);
    const R iW = frcp<R>(W);
    const R v11 = g1 * (((R)1 + BwS * g2) + S * g3 * ((R)1 + Bw * g2)) * iW;
    const R v12 = -g1 * g2 * (BwS + Bw * S * g3) * iW;
    const R v13 = -S * g1 * g3 * iW;
    const R v22 = g2 * (((R)1 + (Bm + Bw) * g1) * ((R)1 + S * g3) + S * g1) * iW;
    const R v23 = -S * g2 * g3 * a1 * iW;
    const R v33 = g3 * (a1 * ((R)1 + BwS * g2) + BwS * g1) * iW;
    const R d1 = g.x - xeq[0], d2 = g.x - xeq[1], d3 = g.x - xeq[2];
    J[0] = v11 * d1 + v12 * d2 + v13 * d3;
    J[1] = v12 * d1 + v22 * d2 + v23 * d3;
    J[2] = v13 * d1 + v23 * d2 + v33 * d3;
    vsum[0] = v11 + v12 + v13;
    vsum[1] = v12 + v22 + v23;
    vsum[2] = v13 + v23 + v33;
    bool neg = false;
#pragma unroll
    for (int r = 0; r < 3; ++r)
      if (gk[r] > (R)0 && J[r] < (R)0) { gk[r] = 0; neg = true; }
    if (!neg) break;
  }
  // molar rates per real particle (eq (2-1), eta = 1), limited by the reactant present
  const R c = Bd.rate_c * d * d * invT;
  const R inv_dtm = frcp<R>(dtm);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    R x = gk[r] > (R)0 ? c * J[r] : (R)0;
    const R cap = fdiv<R>(n[r], r == 0 ? (R)3 : (R)1) * inv_dtm;
    x = x < cap ? x : cap;
    o.xidot[r] = x > (R)0 ? x : (R)0;
  }
  const R k3 = Bd.k3;
  o.mdot[0] = -(R)3 * o.xidot[0] * t.Mz[0] * k3;
  o.mdot[1] = ((R)2 * o.xidot[0] - o.xidot[1]) * t.Mz[1] * k3;
  o.mdot[2] = ((R)3 * o.xidot[1] - o.xidot[2]) * t.Mz[2] * k3;
  o.mdot[3] = o.xidot[2] * t.Mz[3] * k3;
  const R tot = o.xidot[0] + o.xidot[1] + o.xidot[2];
  o.sH2 = -tot * t.Mj[0] * k3;
  o.sH2O = tot * t.Mj[1] * k3;
  if (!(fl & DEM_NO_RXN_HEAT)) {
    // eqs (3-19), (3-21) at T_p, with H in J/kg = R h / M
    R qr = 0;
#pragma unroll
    for (int z = 0; z < 4; ++z) qr += h_over_R<R>(3 + z, Tp) * t.RMz[z] * o.mdot[z];
    o.Qr = -qr;
    o.Qrm = -(h_over_R<R>(0, Tp) * t.RMj[0] * o.sH2 + h_over_R<R>(1, Tp) * t.RMj[1] * o.sH2O);
  }
  const R E = k3 * (R)kPI * d * d * invT;
  o.EQ = E * (vsum[0] + vsum[1] + vsum[2]);
  o.ES = E * (vsum[0] * xeq[0] + vsum[1] * xeq[1] + vsum[2] * xeq[2]);
  // report the resistances of the reactions that started the step active
  o.B[0] = Bm; o.B[1] = Bw; o.B[2] = BFe;
  o.F = F;
}

// ---------------------------------------------------------------------------------------
// Contact law (linear spring-dashpot, tangential spring with history, Coulomb cap).
// n: unit vector from the parcel to the partner; delta: overlap; vrel: contact-point
// velocity of the parcel relative to the partner.
// ---------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void contact_force(const BedP<R> &B, R mstar, R ri, const R n[3], R delta,
                                              const R vrel[3], const R xo[3], const R w[3],
                                              R F[3], R Tq[3], R xn[3]) {
  const R kn = B.kn, kt = B.kt;
  const R eta_n = B.eta_coef * sqrt(mstar * kn);
  const R eta_t = eta_n * B.eta_t_ratio;
  const R vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
  R vt[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) vt[q] = vrel[q] - vn * n[q];
  const R fn = kn * delta + eta_n * vn;
  const R sdot = xo[0] * n[0] + xo[1] * n[1] + xo[2] * n[2];
  R xr[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) xr[q] = xo[q] - sdot * n[q];
  const R mo2 = xo[0] * xo[0] + xo[1] * xo[1] + xo[2] * xo[2];
  const R mr2 = xr[0] * xr[0] + xr[1] * xr[1] + xr[2] * xr[2];
  if (mr2 > (R)0) {
    const R sc = sqrt(mo2 / mr2);
#pragma unroll
    for (int q = 0; q < 3; ++q) xr[q] *= sc;
  }
  const R dt = B.dt;
  R ft[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    xn[q] = xr[q] + vt[q] * dt;
    ft[q] = -kt * xn[q] - eta_t * vt[q];
  }
  const R ftm = sqrt(ft[0] * ft[0] + ft[1] * ft[1] + ft[2] * ft[2]);
  const R cap = B.mu_s * fabs(fn);
  if (ftm > cap) {
    const R sc = cap / ftm;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      ft[q] *= sc;
      xn[q] = -(ft[q] + eta_t * vt[q]) / kt;
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) F[q] = -fn * n[q] + ft[q];
  Tq[0] = ri * (n[1] * ft[2] - n[2] * ft[1]);
  Tq[1] = ri * (n[2] * ft[0] - n[0] * ft[2]);
  Tq[2] = ri * (n[0] * ft[1] - n[1] * ft[0]);
  if (B.mu_r > (R)0) {
    const R wm = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (wm > (R)0) {
      const R c = B.mu_r * fabs(fn) / wm;
#pragma unroll
      for (int q = 0; q < 3; ++q) Tq[q] -= c * w[q];
    }
  }
}

// Distances from a parcel centre to the four wall primitives (side, bottom or cone,
// plate, lid) and unit normals pointing from the wall to the centre; 1e30 = absent.
// T is double for the overlap of a touching wall and float for the pre-screen.
template <class T, class G>
__device__ __forceinline__ void wall_primitives(const G &B, T x, T y, T z, T dist[4], T nw[4][3]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) { dist[p] = (T)1e30; nw[p][0] = nw[p][1] = nw[p][2] = (T)0; }
  const T rho = sqrt(x * x + y * y);
  if (rho > (T)0) {
    dist[0] = (T)B.R_bed - rho;
    nw[0][0] = -x / rho;
    nw[0][1] = -y / rho;
  }
  if (B.wall == DEM_WALL_FLAT) {
    dist[1] = z;
    nw[1][2] = (T)1;
  } else {
    if (z < (T)B.plate_z) {   // the cone acts below the distributor plate
      dist[1] = (z - (T)B.z_apex) * (T)B.sin_a - rho * (T)B.cos_a;
      if (rho > (T)0) { nw[1][0] = -(T)B.cos_a * x / rho; nw[1][1] = -(T)B.cos_a * y / rho; }
      else nw[1][0] = -(T)B.cos_a;
      nw[1][2] = (T)B.sin_a;
    }
    const T hx = floor(x * (T)B.inv_pitch + (T)0.5) * (T)B.pitch;
    const T hy = floor(y * (T)B.inv_pitch + (T)0.5) * (T)B.pitch;
    const T ex = x - hx, ey = y - hy, ez = z - (T)B.plate_z;
    const T q = sqrt(ex * ex + ey * ey);
    if (q >= (T)B.r_hole) {
      dist[2] = fabs(ez);
      nw[2][2] = ez >= (T)0 ? (T)1 : (T)-1;
    } else {
      T ux = (T)1, uy = (T)0;
      if (q > (T)0) { ux = ex / q; uy = ey / q; }
      const T rx = -((T)B.r_hole - q) * ux, ry = -((T)B.r_hole - q) * uy;
      const T dd = sqrt(rx * rx + ry * ry + ez * ez);
      dist[2] = dd;
      if (dd > (T)0) { nw[2][0] = rx / dd; nw[2][1] = ry / dd; nw[2][2] = ez / dd; }
      else nw[2][2] = (T)1;
    }
  }
  dist[3] = (T)B.H - z;
  nw[3][2] = (T)-1;
}

__device__ __forceinline__ void set_error(int *err, int bit) { atomicOr(err, bit); }

// ---------------------------------------------------------------------------------------
// Layer masses: FP64 values (FP64 and split forms) or Kahan pairs (value, compensation) of
// FP32 stored in the same 8-byte slot (split-Kahan form).
// ---------------------------------------------------------------------------------------
template <class P> __device__ __forceinline__ typename P::R mass_r(const double *m, int i) {
  if constexpr (P::kahan) {
    const float2 v = reinterpret_cast<const float2 *>(m)[i];
    return v.x + v.y;
  } else {
    return (typename P::R)m[i];
  }
}
// the same from a mass word already loaded
template <class P> __device__ __forceinline__ typename P::R mass_word_r(double w) {
  if constexpr (P::kahan) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(w);
    return __uint_as_float((unsigned)u) + __uint_as_float((unsigned)(u >> 32));
  } else {
    return (typename P::R)w;
  }
}
template <class P> __device__ __forceinline__ double mass_d(const double *m, int i) {
  if constexpr (P::kahan) {
    const float2 v = reinterpret_cast<const float2 *>(m)[i];
    return (double)v.x + (double)v.y;
  } else {
    return m[i];
  }
}
// m += inc, not below zero (Kahan-compensated in the split-Kahan form)
template <class P> __device__ __forceinline__ void mass_add(double *m, int i, typename P::R inc) {
  if constexpr (P::kahan) {
    // value = hi + lo; lo carries what the FP32 sum hi could not hold (compensated summation,
    // Kahan 1965, with the compensation stored with the opposite sign)
    float2 v = reinterpret_cast<float2 *>(m)[i];
    const float y = inc + v.y;
    const float t = v.x + y;
    v.y = y - (t - v.x);
    v.x = t;
    if (v.x + v.y < 0.0f) { v.x = 0.0f; v.y = 0.0f; }
    reinterpret_cast<float2 *>(m)[i] = v;
  } else {
    const double mn = m[i] + (double)inc;
    m[i] = __double_as_longlong(mn) < 0 ? 0.0 : mn;   // max(mn, 0) by the sign bit: no FP64 compare
  }
}

// ---------------------------------------------------------------------------------------
// Gas state words: FP64 values in the FP64 form; in the FP32 forms a (value, compensation)
// pair of FP32 in the same 8-byte slot, so that the explicit update accumulates small
// increments without FP64 arithmetic (compensated summation).
// ---------------------------------------------------------------------------------------
template <class P> __device__ __forceinline__ typename P::R gas_r(const double *G, size_t k) {
  if constexpr (P::exact) {
    return G[k];
  } else {
    const float2 v = reinterpret_cast<const float2 *>(G)[k];
    return v.x + v.y;
  }
}
template <class P> __device__ __forceinline__ double gas_d(const double *G, size_t k) {
  if constexpr (P::exact) {
    return G[k];
  } else {
    const float2 v = reinterpret_cast<const float2 *>(G)[k];
    return (double)v.x + (double)v.y;
  }
}
// a value given in FP64 (inputs)
__device__ __forceinline__ void gas_put(double *G, size_t k, double v, bool pairs) {
  if (!pairs) {
    G[k] = v;
  } else {
    const float hi = (float)v;
    reinterpret_cast<float2 *>(G)[k] = make_float2(hi, (float)(v - (double)hi));
  }
}
// (hi, lo) + b with the rounding error of hi + b carried into lo (two-sum, Knuth), then
// renormalised; the pair keeps ~48 significant bits
__device__ __forceinline__ float2 pair_add_exact(float2 a, float b) {
  const float s = a.x + b;
  const float bb = s - a.x;
  const float err = (a.x - (s - bb)) + (b - bb);
  const float lo = a.y + err;
  const float hi = s + lo;
  return make_float2(hi, lo - (hi - s));
}
// position word of parcel i: FP64 value, or in the split-Kahan form a (hi, lo) pair of FP32
// relative to the bed's corner (origin)
template <class P> __device__ __forceinline__ double pos_abs(const double *x, int i, double origin) {
  if constexpr (P::kahan) {
    const float2 v = reinterpret_cast<const float2 *>(x)[i];
    return origin + ((double)v.x + (double)v.y);
  } else {
    return x[i];
  }
}
// (hi, lo) + inc, compensated
__device__ __forceinline__ float2 pair_add(float2 v, float inc) {
  const float y = inc + v.y;
  const float t = v.x + y;
  return make_float2(t, y - (t - v.x));
}

}  // namespace dem
