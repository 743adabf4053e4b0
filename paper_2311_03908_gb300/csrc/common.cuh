// common.cuh -- device-side constants, per-bed parameters and the physics of one parcel.
//
// Everything here is templated on R, the arithmetic type of forces, drag, heat and
// kinetics: double for the all-FP64 form, float for the split form. Positions, layer
// masses and cell-source sums are always double.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dem.h"

namespace dem {

constexpr int KMAX = DEM_MAX_CONTACTS;
constexpr double kPI = 3.14159265358979323846;
constexpr double kRgas = 8.314;  // gas constant of Sec. 2.1
constexpr double kGrav = 9.81;

enum : int { ERR_CAPACITY = 1, ERR_NONFINITE = 2, ERR_DOMAIN = 4, ERR_TIMEOUT = 8 };

// per-cell gas-property rows (derived from the gas state by gas_cell_props)
enum : int {
  GP_RHO = 0, GP_MU, GP_LAM, GP_CP, GP_X, GP_DM, GP_SC13, GP_PR13, GP_EPOW, GP_D0, GP_D1,
  GP_UZ, GP_EPS, GP_TG, GP_N
};
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
  DG_FFILM = 20, DG_A = 21, DG_B = 24, DG_SH = 27, DG_NU, DG_RE, DG_NCONTACT, DG_CELL, DG_N
};
static_assert((int)DG_N == (int)DEM_NDIAG, "diag rows");

// Bed parameters as the kernels need them (derived once on the host at dem_init).
struct DevBed {
  // gas grid: cell of a point = floor((x - x0) * inv_dx), clamped
  double x0, y0, z0, dx, dy, dz, inv_dx, inv_dy, inv_dz, vcell;
  int nx, ny, nz, s;            // s = DEM sub-cells per gas-cell edge
  long long cell_off;           // first global gas cell of this bed
  unsigned key_off;             // first global DEM-cell key of this bed
  float pf_margin;              // FP32 prefilter margin of the pair test, m
  // walls
  double R, H, cos_a, sin_a, z_apex, plate_z, pitch, r_hole;
  int wall;
  // contact law
  double dt, kn, kt, eta_coef, eta_t_ratio, mu_s, mu_r;
  double k, k3;
  int ncouple;
  // gas
  double U_in, T_in, p0, Y_in[3];
  double fuller12, fuller13;    // T- and p-free parts of eq (2-26)
  // kinetics
  double k0[3], Ea[3], tau;
  double psi[2], K1b[2], K2[2]; // Ganser constants per ore (K1 without the wall term)
  double xi[2][3];              // product-layer porosity per ore: m, w, Fe (eqs (2-31)..(2-36))
  double pore_cm[2];
  double dpdz, eps_min, bedD;
  unsigned flags;
};

// Molar masses (kg/mol): solids Fe2O3, Fe3O4, FeO, Fe; gases H2, H2O, N2.
__device__ __constant__ static const double cMz[4] = {159.69e-3, 231.533e-3, 71.844e-3, 55.845e-3};
__device__ __constant__ static const double cMj[3] = {2.016e-3, 18.015e-3, 28.014e-3};
// Table 2 equilibrium constants K = exp(a / T + b)
__device__ __constant__ static const double cKa[3] = {1433.4, -7393.9, -2023.8};
__device__ __constant__ static const double cKb[3] = {9.08, 7.56, 1.24};
// Table C1, two ranges per species (H2, H2O, N2, Fe2O3, Fe3O4, FeO, Fe); the Fe ranges
// 1000-1184 K are represented by the 298-1000 K range (see the design notes)
__device__ __constant__ static const double cNasaT[7] = {1000.0, 1000.0, 1000.0, 960.0, 850.0, 1000.0, 1184.0};
__device__ __constant__ static const double cNasa[7][2][6] = {
  {{2.3443, 7.98e-3, -1.95e-5, 2.02e-8, -7.38e-12, -9.179e2}, {2.9328, 8.27e-4, -1.46e-7, 1.54e-11, -6.89e-16, -8.131e2}},
  {{4.1986, -2.04e-3, 6.52e-6, -5.49e-9, 1.77e-12, -3.03e4}, {2.677, 2.97e-3, -7.74e-7, 9.44e-11, -4.27e-15, -2.989e4}},
  {{3.531, -1.24e-4, -5.03e-7, 2.44e-9, -1.41e-12, -1.047e3}, {2.9526, 1.40e-3, -4.93e-7, 7.86e-11, -4.61e-15, -9.239e2}},
  {{0.1522, 6.71e-2, -1.13e-4, 9.93e-8, -3.28e-11, -1.013e5}, {353.05, -0.9728, 1.05e-3, -4.96e-7, 8.74e-11, -1.96e5}},
  {{4.8445, 4.39e-2, 5.25e-5, -2.21e-7, 1.75e-10, -1.38e5}, {88.431, -0.149, 1.26e-4, -4.7e-8, 6.79e-12, -1.621e5}},
  {{5.3195, 2.21e-3, 1.07e-6, -2.79e-9, 1.33e-12, -3.441e4}, {5.8316, 1.43e-3, -9.32e-8, -6.6e-12, -2.25e-14, -3.457e4}},
  {{2.4134, -1.58e-3, 2.15e-5, -3.8e-8, 2.20e-11, -774.38}, {61.011, -0.161, 1.68e-4, -7.75e-8, 1.33e-11, -1.65e4}},
};
// Table C2 viscosity, Table C3 conductivity
__device__ __constant__ static const double cVisc[3][3] = {
  {2.85e-6, 2.16e-8, -3.78e-12}, {-4.44e-6, 4.52e-8, -3.20e-12}, {7.86e-6, 3.87e-8, -5.11e-12}};
__device__ __constant__ static const double cCond[3][5] = {
  {3.07e-3, 8.09e-4, -8.52e-7, 7.2e-10, -2.21e-13},
  {6.84e-3, 6.25e-6, 1.31e-7, -5.99e-11, 1.12e-14},
  {2.51e-3, 8.92e-5, -4.00e-8, 1.62e-11, -2.61e-15}};

// ---------------------------------------------------------------------------------------
// Thermochemistry (eqs (3-22), (3-23)): molar enthalpy / R and molar heat capacity / R.
// Species index s: 0 H2, 1 H2O, 2 N2, 3 Fe2O3, 4 Fe3O4, 5 FeO, 6 Fe.
// ---------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R h_over_R(int s, R T) {
  const int r = (double)T <= cNasaT[s] ? 0 : 1;
  const double *a = cNasa[s][r];
  const R c1 = (R)a[0], c2 = (R)(a[1] * 0.5), c3 = (R)(a[2] * (1.0 / 3.0)), c4 = (R)(a[3] * 0.25),
          c5 = (R)(a[4] * 0.2);
  return T * (c1 + T * (c2 + T * (c3 + T * (c4 + T * c5)))) + (R)a[5];
}
template <class R>
__device__ __forceinline__ R cp_over_R(int s, R T) {
  const int r = (double)T <= cNasaT[s] ? 0 : 1;
  const double *a = cNasa[s][r];
  return (R)a[0] + T * ((R)a[1] + T * ((R)a[2] + T * ((R)a[3] + T * (R)a[4])));
}

// ---------------------------------------------------------------------------------------
// Gas-cell properties (eqs (2-1-1), (2-1-2), (2-26)..(2-29), (3-53)..(3-59)) computed once
// per cell in double and stored in R: the parcel kernels then read finished numbers.
// ---------------------------------------------------------------------------------------
struct CellProps {
  double rho, mu, lam, cp, x, Dm, sc13, pr13, epow, D[2], uz, eps, T;
};

// Computed in the form's arithmetic type P (double in the FP64 form, float in the split
// form: GB300's FP64 rate is a small fraction of its FP32 rate); the gas state itself and
// the cell sums stay FP64.
template <class P>
__device__ inline CellProps gas_cell_props(const DevBed &B, double eps_d, const double Yd[3], double Td) {
  CellProps o;
  const P p = (P)B.p0, T = (P)Td, eps = (P)eps_d;
  const P Y[3] = {(P)Yd[0], (P)Yd[1], (P)Yd[2]};
  const P inv = Y[0] / (P)cMj[0] + Y[1] / (P)cMj[1] + Y[2] / (P)cMj[2];
  const P Mg = (P)1 / inv;
  const P xp0 = Y[0] * Mg / (P)cMj[0], xp1 = Y[1] * Mg / (P)cMj[1], xp2 = Y[2] * Mg / (P)cMj[2];
  const P den = xp0 + xp1;
  const P x = den > (P)0 ? xp0 / den : (P)0;
  const P rho = Mg * p / ((P)kRgas * T);
  P mu = 0, lam = 0, cp = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    mu += Y[j] * ((P)cVisc[j][0] + T * ((P)cVisc[j][1] + T * (P)cVisc[j][2]));
    lam += Y[j] * ((P)cCond[j][0] + T * ((P)cCond[j][1] + T * ((P)cCond[j][2] + T * ((P)cCond[j][3] + T * (P)cCond[j][4]))));
    cp += Y[j] * cp_over_R<P>(j, T) * (P)(kRgas / cMj[j]);
  }
  // Fuller binary coefficients D(H2,H2O), D(H2,N2) (T^1.75 = T sqrt(T) sqrt(sqrt(T))) and
  // Wilke's rule for H2
  const P sT = sqrt(T);
  const P tf = T * sT * sqrt(sT) * ((P)101325 / p) * (P)1e-7;
  const P D12 = tf * (P)B.fuller12, D13 = tf * (P)B.fuller13;
  const P rest = (P)1 - xp0;
  const P Dm = rest < (P)1e-12 ? D12 : rest / (xp1 / D12 + xp2 / D13);
  o.rho = rho; o.mu = mu; o.lam = lam; o.cp = cp; o.x = x; o.Dm = Dm;
  o.sc13 = cbrt(mu / (rho * Dm));
  o.pr13 = cbrt(cp * mu / lam);
  o.epow = exp((P)-2.65 * log(eps));
  // pore diffusion per ore: molecular, Knudsen, or Bosanquet by lambda / d_a (Sec. 2.3)
  const P mfp = x > (P)0 ? (P)1.013 / (p * x) : (P)3e38;
  const P sq = sqrt(T / (P)(cMj[0] * 1e3));
#pragma unroll
  for (int ore = 0; ore < 2; ++ore) {
    const P da = (P)B.pore_cm[ore];
    const P DK = (P)0.97 * ((P)0.5 * da) * sq;
    const P ratio = mfp / da;
    o.D[ore] = ratio <= (P)0.01 ? Dm : (ratio >= (P)10 ? DK : (P)1 / ((P)1 / Dm + (P)1 / DK));
  }
  o.uz = (P)B.U_in / eps;
  o.eps = eps_d;
  o.T = Td;
  return o;
}

// ---------------------------------------------------------------------------------------
// Per-parcel gas-side terms.
// ---------------------------------------------------------------------------------------
template <class R> struct Gas {   // a cell's properties in the parcel's arithmetic type
  R rho, mu, lam, cp, x, Dm, sc13, pr13, epow, D, uz, eps, T;
};

template <class R> __device__ __forceinline__ R pos_pow(R x, R e) {   // x^e for x >= 0
  return x > (R)0 ? exp(e * log(x)) : (R)0;
}

// Gunn correlation (eqs (2-22), (3-12)); c13 is Sc^(1/3) or Pr^(1/3), re02 = Re^0.2
template <class R> __device__ __forceinline__ R gunn(R eps, R re02, R re07, R c13) {
  return ((R)7 - (R)10 * eps + (R)5 * eps * eps) * ((R)1 + (R)0.7 * re02 * c13) +
         ((R)1.33 - (R)2.4 * eps + (R)1.2 * eps * eps) * re07 * c13;
}

// Gidaspow-Ganser drag coefficient divided by the solid fraction (eqs (3-5-2)..(3-5-5)):
// F_d = (beta / eps_p) V_p (u_g - v_p), the form of eq (3-5) with eps_p cancelled.
template <class R>
__device__ __forceinline__ R beta_over_epsp(const DevBed &B, int ore, R d, const Gas<R> &g, R slip, R Re) {
  const R eps = g.eps, ep = (R)1 - eps;
  const R psi = (R)B.psi[ore];
  if (eps < (R)0.8)
    return (R)150 * ep * g.mu / (eps * d * d * psi * psi) + (R)1.75 * eps * g.rho * slip / (d * psi * ep);
  const R K1 = (R)B.K1b[ore] - (R)2.25 * d / (R)B.bedD;
  const R K2 = (R)B.K2[ore];
  if (Re > (R)0) {
    const R RK = Re * (K1 * K2);
    const R CD = (R)24 / (Re * K1) * ((R)1 + (R)0.1118 * pos_pow(RK, (R)0.6567)) +
                 (R)0.4305 * K2 / ((R)1 + (R)3305 / RK);
    return (R)0.75 * CD * eps * g.rho * slip / d * g.epow;
  }
  return (R)0.75 * ((R)24 / K1) * g.mu / (d * d) * g.epow;
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
__device__ __forceinline__ void uscm(const DevBed &Bd, const double m[4], R Tp, R d, int ore,
                                     const Gas<R> &g, R re02, R re07, R dtm, KinOut<R> &o) {
  const unsigned fl = Bd.flags;
#pragma unroll
  for (int r = 0; r < 3; ++r) { o.xidot[r] = 0; o.A[r] = 0; o.B[r] = 0; }
#pragma unroll
  for (int z = 0; z < 4; ++z) o.mdot[z] = 0;
  o.sH2 = o.sH2O = o.Qr = o.Qrm = o.EQ = o.ES = o.F = o.Sh = 0;
  const R inv_k3 = (R)(1.0 / Bd.k3);
  R n[4];
#pragma unroll
  for (int z = 0; z < 4; ++z) n[z] = (R)m[z] * inv_k3 / (R)cMz[z];
  const R nfe = (R)2 * n[0] + (R)3 * n[1] + n[2] + n[3];
  if (!(nfe > (R)0)) return;
  const R inv_nfe = (R)1 / nfe;
  // 1 - f of eqs (2-15)..(2-17), written as the iron fractions still behind each front
  R om[3];
  om[0] = (R)2 * n[0] * inv_nfe;
  om[1] = ((R)2 * n[0] + (R)3 * n[1]) * inv_nfe;
  om[2] = ((R)2 * n[0] + (R)3 * n[1] + n[2]) * inv_nfe;
  const R invT = (R)1 / Tp;
  R xeq[3], gk[3], c3[3];
  bool act[3];
  const bool kin = !(fl & DEM_NO_KINETICS);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const R K = exp((R)cKa[r] * invT + (R)cKb[r]);                 // Table 2
    xeq[r] = (R)1 / (K + (R)1);                                       // eq (2-1-3)
    const R kr = (R)Bd.k0[r] * exp(-(R)(Bd.Ea[r] / kRgas) * invT);    // eq (2-13)
    c3[r] = cbrt(om[r]);
    act[r] = kin && n[r] > (R)0 && g.x > xeq[r] && Bd.k0[r] > 0.0;
    // 1/A of eq (2-12): k_r (1-f)^(2/3) (1 + K)/K
    gk[r] = act[r] ? kr * c3[r] * c3[r] * ((R)1 + (R)1 / K) : (R)0;
  }
  // product-layer resistances, eq (2-14), with D_eff of eq (2-30)
  const R D = g.D;
  const R rp = (R)0.5 * d;
  R Bm = 0, Bw = 0, BFe = 0;
  if (!(fl & DEM_NO_LAYER)) {
    const R inv_tau = (R)(1.0 / Bd.tau);
    if (act[0]) Bm = rp / (D * (R)Bd.xi[ore][0] * inv_tau) * ((R)1 / c3[0] - (R)1 / c3[1]);
    if ((act[0] || act[1]) && om[1] > (R)0) Bw = rp / (D * (R)Bd.xi[ore][1] * inv_tau) * ((R)1 / c3[1] - (R)1 / c3[2]);
    if (om[2] > (R)0) BFe = rp / (D * (R)Bd.xi[ore][2] * inv_tau) * ((R)1 / c3[2] - (R)1);
  }
  // gas film, eqs (2-20)..(2-24)
  o.Sh = gunn(g.eps, re02, re07, g.sc13);
  const R F = (fl & DEM_NO_FILM) ? (R)0 : d / (o.Sh * g.Dm);
  // closed-form network; a reaction whose flux is negative is dropped and the rest re-solved
  const R S = F + BFe, BwS = Bw + S;
#pragma unroll
  for (int r = 0; r < 3; ++r) o.A[r] = gk[r] > (R)0 ? (R)1 / gk[r] : (R)0;
  R J[3] = {0, 0, 0}, vsum[3] = {0, 0, 0};
  for (int it = 0; it < 3; ++it) {
    const R g1 = gk[0], g2 = gk[1], g3 = gk[2];
    const R a1 = (R)1 + Bm * g1;
    const R W = a1 * ((R)1 + BwS * g2 + S * g3 * ((R)1 + Bw * g2)) + g1 * (BwS + Bw * S * g3);
    const R iW = (R)1 / W;
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
  const R c = (R)kPI * d * d * (R)Bd.p0 * invT * (R)(1.0 / kRgas);
  const R inv_dtm = (R)1 / dtm;
  const R nu[3] = {3, 1, 1};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    R x = gk[r] > (R)0 ? c * J[r] : (R)0;
    const R cap = n[r] / nu[r] * inv_dtm;
    x = x < cap ? x : cap;
    o.xidot[r] = x > (R)0 ? x : (R)0;
  }
  const R k3 = (R)Bd.k3;
  o.mdot[0] = -(R)3 * o.xidot[0] * (R)cMz[0] * k3;
  o.mdot[1] = ((R)2 * o.xidot[0] - o.xidot[1]) * (R)cMz[1] * k3;
  o.mdot[2] = ((R)3 * o.xidot[1] - o.xidot[2]) * (R)cMz[2] * k3;
  o.mdot[3] = o.xidot[2] * (R)cMz[3] * k3;
  const R tot = o.xidot[0] + o.xidot[1] + o.xidot[2];
  o.sH2 = -tot * (R)cMj[0] * k3;
  o.sH2O = tot * (R)cMj[1] * k3;
  if (!(fl & DEM_NO_RXN_HEAT)) {
    // eqs (3-19), (3-21) at T_p, with H in J/kg = R h / M
    R qr = 0;
#pragma unroll
    for (int z = 0; z < 4; ++z) qr += h_over_R(3 + z, Tp) * (R)(kRgas / cMz[z]) * o.mdot[z];
    o.Qr = -qr;
    o.Qrm = -(h_over_R(0, Tp) * (R)(kRgas / cMj[0]) * o.sH2 + h_over_R(1, Tp) * (R)(kRgas / cMj[1]) * o.sH2O);
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
__device__ __forceinline__ void contact_force(const DevBed &B, R mstar, R ri, const R n[3], R delta,
                                              const R vrel[3], const R xo[3], const R w[3],
                                              R F[3], R Tq[3], R xn[3]) {
  const R kn = (R)B.kn, kt = (R)B.kt;
  const R eta_n = (R)B.eta_coef * sqrt(mstar * kn);
  const R eta_t = eta_n * (R)B.eta_t_ratio;
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
  const R dt = (R)B.dt;
  R ft[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    xn[q] = xr[q] + vt[q] * dt;
    ft[q] = -kt * xn[q] - eta_t * vt[q];
  }
  const R ftm = sqrt(ft[0] * ft[0] + ft[1] * ft[1] + ft[2] * ft[2]);
  const R cap = (R)B.mu_s * fabs(fn);
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
  if (B.mu_r > 0.0) {
    const R wm = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (wm > (R)0) {
      const R c = (R)B.mu_r * fabs(fn) / wm;
#pragma unroll
      for (int q = 0; q < 3; ++q) Tq[q] -= c * w[q];
    }
  }
}

// Distances from a parcel centre to the four wall primitives (side, bottom or cone,
// plate, lid) and unit normals pointing from the wall to the centre; 1e300 = absent.
__device__ inline void wall_primitives(const DevBed &B, double x, double y, double z,
                                       double dist[4], double nw[4][3]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) { dist[p] = 1e300; nw[p][0] = nw[p][1] = nw[p][2] = 0.0; }
  const double rho = sqrt(x * x + y * y);
  if (rho > 0.0) {
    dist[0] = B.R - rho;
    nw[0][0] = -x / rho;
    nw[0][1] = -y / rho;
  }
  if (B.wall == DEM_WALL_FLAT) {
    dist[1] = z;
    nw[1][2] = 1.0;
  } else {
    if (z < B.plate_z) {   // the cone acts below the distributor plate
      dist[1] = (z - B.z_apex) * B.sin_a - rho * B.cos_a;
      if (rho > 0.0) { nw[1][0] = -B.cos_a * x / rho; nw[1][1] = -B.cos_a * y / rho; }
      else nw[1][0] = -B.cos_a;
      nw[1][2] = B.sin_a;
    }
    const double hx = floor(x / B.pitch + 0.5) * B.pitch;
    const double hy = floor(y / B.pitch + 0.5) * B.pitch;
    const double ex = x - hx, ey = y - hy, ez = z - B.plate_z;
    const double q = sqrt(ex * ex + ey * ey);
    if (q >= B.r_hole) {
      dist[2] = fabs(ez);
      nw[2][2] = ez >= 0.0 ? 1.0 : -1.0;
    } else {
      double ux = 1.0, uy = 0.0;
      if (q > 0.0) { ux = ex / q; uy = ey / q; }
      const double rx = -(B.r_hole - q) * ux, ry = -(B.r_hole - q) * uy;
      const double dd = sqrt(rx * rx + ry * ry + ez * ez);
      dist[2] = dd;
      if (dd > 0.0) { nw[2][0] = rx / dd; nw[2][1] = ry / dd; nw[2][2] = ez / dd; }
      else nw[2][2] = 1.0;
    }
  }
  dist[3] = B.H - z;
  nw[3][2] = -1.0;
}

__device__ __forceinline__ void set_error(int *err, int bit) { atomicOr(err, bit); }

}  // namespace dem
