// dem_oracle.cpp -- TEST INFRASTRUCTURE ONLY (see dem_oracle.h).
//
// Plain FP64 restatement of the particle-side step of Lan et al. (arXiv 2311.03908).
// Each function names the section / equation / table of the paper it follows. Where
// the paper is silent or garbled, the reading taken is stated in a comment starting
// "Reading:"; the same readings are listed in the repository's design notes.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fopenmp -fPIC -shared  (no FMA
// contraction anywhere, so positions and the pair test are plain IEEE double ops).
#include "dem_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kRg = 8.314;      // gas constant used by the paper, Sec. 2.1
constexpr double kG = 9.81;        // gravity magnitude, -z
constexpr double kSigma = 5.67e-8;  // Stefan-Boltzmann constant as printed with eq (3-16), W/m^2/K^4

// Molar masses, kg/mol. Solids z: Fe2O3 (h), Fe3O4 (m), FeO (w), Fe; gases j: H2, H2O, N2.
constexpr double kMz[4] = {159.69e-3, 231.533e-3, 71.844e-3, 55.845e-3};
constexpr double kMj[3] = {2.016e-3, 18.015e-3, 28.014e-3};

// Table 2: K_eq = exp(a / T_p + b) for R1 (h->m), R2 (m->w), R3 (w->Fe).
constexpr double kKeqA[3] = {1433.4, -7393.9, -2023.8};
constexpr double kKeqB[3] = {9.08, 7.56, 1.24};

// Sec. 2.3: Fuller diffusion volumes, cm^3/mol (H2, H2O, N2).
constexpr double kVd[3] = {7.07, 12.7, 17.9};

// Table C1 (NASA-type coefficients a1..a6). Species order: H2, H2O, N2, Fe2O3, Fe3O4, FeO, Fe.
// Reading: the two Fe ranges 1000-1184 K are replaced by the 298-1000 K range (as printed
// they give a negative heat capacity and jumps of ~40 kJ/mol); at a range boundary the
// lower range is used (T <= boundary).
struct NasaRange { double tmax; double a[6]; };
struct NasaSpecies { int nr; NasaRange r[2]; };
const NasaSpecies kNasa[7] = {
  {2, {{1000.0, {2.3443, 7.98e-3, -1.95e-5, 2.02e-8, -7.38e-12, -9.179e2}},
       {1e30, {2.9328, 8.27e-4, -1.46e-7, 1.54e-11, -6.89e-16, -8.131e2}}}},
  {2, {{1000.0, {4.1986, -2.04e-3, 6.52e-6, -5.49e-9, 1.77e-12, -3.03e4}},
       {1e30, {2.677, 2.97e-3, -7.74e-7, 9.44e-11, -4.27e-15, -2.989e4}}}},
  {2, {{1000.0, {3.531, -1.24e-4, -5.03e-7, 2.44e-9, -1.41e-12, -1.047e3}},
       {1e30, {2.9526, 1.40e-3, -4.93e-7, 7.86e-11, -4.61e-15, -9.239e2}}}},
  {2, {{960.0, {0.1522, 6.71e-2, -1.13e-4, 9.93e-8, -3.28e-11, -1.013e5}},
       {1e30, {353.05, -0.9728, 1.05e-3, -4.96e-7, 8.74e-11, -1.96e5}}}},
  {2, {{850.0, {4.8445, 4.39e-2, 5.25e-5, -2.21e-7, 1.75e-10, -1.38e5}},
       {1e30, {88.431, -0.149, 1.26e-4, -4.7e-8, 6.79e-12, -1.621e5}}}},
  {2, {{1000.0, {5.3195, 2.21e-3, 1.07e-6, -2.79e-9, 1.33e-12, -3.441e4}},
       {1e30, {5.8316, 1.43e-3, -9.32e-8, -6.6e-12, -2.25e-14, -3.457e4}}}},
  {2, {{1184.0, {2.4134, -1.58e-3, 2.15e-5, -3.8e-8, 2.20e-11, -774.38}},
       {1e30, {61.011, -0.161, 1.68e-4, -7.75e-8, 1.33e-11, -1.65e4}}}},
};
const double kNasaM[7] = {kMj[0], kMj[1], kMj[2], kMz[0], kMz[1], kMz[2], kMz[3]};

// Table C2: gas viscosity mu = a1 + a2 T + a3 T^2 (Pa s).
constexpr double kMu[3][3] = {{2.85e-6, 2.16e-8, -3.78e-12},
                              {-4.44e-6, 4.52e-8, -3.20e-12},
                              {7.86e-6, 3.87e-8, -5.11e-12}};
// Table C3: gas conductivity lambda = a1 + a2 T + ... + a5 T^4 (W/m/K).
constexpr double kLam[3][5] = {{3.07e-3, 8.09e-4, -8.52e-7, 7.2e-10, -2.21e-13},
                               {6.84e-3, 6.25e-6, 1.31e-7, -5.99e-11, 1.12e-14},
                               {2.51e-3, 8.92e-5, -4.00e-8, 1.62e-11, -2.61e-15}};

// ---------------------------------------------------------------------------------------
// Forward-mode dual numbers with 6 tangents (derivatives w.r.t. k0[3], Ea[3]); used only
// by the adjoint reference. Every physics function below is a template over the scalar.
// ---------------------------------------------------------------------------------------
constexpr int kNT = 6;
struct Dual {
  double v = 0.0;
  double d[kNT] = {0, 0, 0, 0, 0, 0};
  Dual() = default;
  Dual(double x) : v(x) {}  // NOLINT: constants promote implicitly
};
inline double val(double x) { return x; }
inline double val(const Dual &x) { return x.v; }
inline Dual operator+(const Dual &a, const Dual &b) { Dual r(a.v + b.v); for (int i = 0; i < kNT; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
inline Dual operator-(const Dual &a, const Dual &b) { Dual r(a.v - b.v); for (int i = 0; i < kNT; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
inline Dual operator-(const Dual &a) { Dual r(-a.v); for (int i = 0; i < kNT; ++i) r.d[i] = -a.d[i]; return r; }
inline Dual operator*(const Dual &a, const Dual &b) { Dual r(a.v * b.v); for (int i = 0; i < kNT; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
inline Dual operator/(const Dual &a, const Dual &b) { Dual r(a.v / b.v); for (int i = 0; i < kNT; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v); return r; }
inline Dual operator+(const Dual &a, double b) { return a + Dual(b); }
inline Dual operator+(double a, const Dual &b) { return Dual(a) + b; }
inline Dual operator-(const Dual &a, double b) { return a - Dual(b); }
inline Dual operator-(double a, const Dual &b) { return Dual(a) - b; }
inline Dual operator*(const Dual &a, double b) { Dual r(a.v * b); for (int i = 0; i < kNT; ++i) r.d[i] = a.d[i] * b; return r; }
inline Dual operator*(double a, const Dual &b) { return b * a; }
inline Dual operator/(const Dual &a, double b) { Dual r(a.v / b); for (int i = 0; i < kNT; ++i) r.d[i] = a.d[i] / b; return r; }
inline Dual operator/(double a, const Dual &b) { return Dual(a) / b; }
inline Dual &operator+=(Dual &a, const Dual &b) { a = a + b; return a; }
inline Dual &operator-=(Dual &a, const Dual &b) { a = a - b; return a; }
inline Dual &operator*=(Dual &a, const Dual &b) { a = a * b; return a; }
inline Dual chain(const Dual &a, double f, double df) { Dual r(f); for (int i = 0; i < kNT; ++i) r.d[i] = df * a.d[i]; return r; }
inline Dual exp(const Dual &a) { double e = std::exp(a.v); return chain(a, e, e); }
inline Dual log(const Dual &a) { return chain(a, std::log(a.v), 1.0 / a.v); }
inline Dual sqrt(const Dual &a) { double s = std::sqrt(a.v); return chain(a, s, s > 0 ? 0.5 / s : 0.0); }
inline Dual pow(const Dual &a, double c) {
  double p = std::pow(a.v, c);
  return chain(a, p, a.v != 0.0 ? c * p / a.v : 0.0);
}
inline Dual fabs(const Dual &a) { return a.v < 0 ? -a : a; }
using std::exp; using std::log; using std::sqrt; using std::pow; using std::fabs;

template <class S> inline S smin(const S &a, const S &b) { return val(b) < val(a) ? b : a; }
template <class S> inline S smax(const S &a, const S &b) { return val(b) > val(a) ? b : a; }

inline int ib(const double *b, int k) { return (int)std::lround(b[k]); }

// ---------------------------------------------------------------------------------------
// Thermochemistry, Sec. 3.1 eqs (3-22), (3-23) with Table C1.
// ---------------------------------------------------------------------------------------
inline const double *nasa_coeffs(int s, double T) {
  const NasaSpecies &sp = kNasa[s];
  return (T <= sp.r[0].tmax) ? sp.r[0].a : sp.r[1].a;
}
template <class S> S nasa_H(int s, const S &T) {   // eq (3-22), J/kg
  const double *a = nasa_coeffs(s, val(T));
  S h = T * (a[0] + T * (a[1] / 2.0 + T * (a[2] / 3.0 + T * (a[3] / 4.0 + T * (a[4] / 5.0))))) + a[5];
  return kRg * h / kNasaM[s];
}
template <class S> S nasa_cp(int s, const S &T) {  // eq (3-23), J/kg/K
  const double *a = nasa_coeffs(s, val(T));
  S c = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
  return kRg * c / kNasaM[s];
}

// ---------------------------------------------------------------------------------------
// Gas properties of one cell (Sec. 2.1 eqs (2-1-1), (2-1-2); Sec. 2.3 eqs (2-26), (2-27);
// Sec. 3.4 eqs (3-53)..(3-59)). The gas is frozen within a step, so plain doubles.
// ---------------------------------------------------------------------------------------
struct GasProps {
  double T, p, rho, mu, lam, cp, x, xp[3], Dm, Mg, D12, D13;
};

double fuller(int i, int j, double T, double p) {  // eq (2-26), m^2/s; M in g/mol
  double Mi = kMj[i] * 1e3, Mj = kMj[j] * 1e3;
  double s = std::cbrt(kVd[i]) + std::cbrt(kVd[j]);
  return 1e-7 * std::pow(T, 1.75) * std::sqrt(1.0 / Mi + 1.0 / Mj) / ((p / 101325.0) * s * s);
}

GasProps gas_props(double T, const double Y[3], double p) {
  GasProps g{};
  g.T = T;
  g.p = p;
  double inv = 0.0;
  for (int j = 0; j < 3; ++j) inv += Y[j] / kMj[j];
  g.Mg = 1.0 / inv;                                         // eq (2-1-2)
  for (int j = 0; j < 3; ++j) g.xp[j] = Y[j] * g.Mg / kMj[j];  // eq (2-1-1)
  double den = g.xp[0] + g.xp[1];
  g.x = den > 0.0 ? g.xp[0] / den : 0.0;                    // H2 basis, Sec. 2.1
  g.rho = g.Mg * p / (kRg * T);                             // eq (3-53)
  g.mu = 0.0;
  g.lam = 0.0;
  g.cp = 0.0;
  for (int j = 0; j < 3; ++j) {
    g.mu += Y[j] * (kMu[j][0] + kMu[j][1] * T + kMu[j][2] * T * T);                   // (3-55,56)
    g.lam += Y[j] * (kLam[j][0] + T * (kLam[j][1] + T * (kLam[j][2] + T * (kLam[j][3] + T * kLam[j][4]))));  // (3-58,59)
    g.cp += Y[j] * nasa_cp(j, T);                                                      // (3-57)
  }
  g.D12 = fuller(0, 1, T, p);
  g.D13 = fuller(0, 2, T, p);
  // eq (2-27) for H2 on the true mole fractions. Reading: in (nearly) pure H2 the
  // expression is 0/0; its limit with no N2 present is the binary D(H2,H2O).
  double rest = 1.0 - g.xp[0];
  if (rest < 1e-12) g.Dm = g.D12;
  else g.Dm = rest / (g.xp[1] / g.D12 + g.xp[2] / g.D13);
  return g;
}

// Layer porosities xi_m, xi_w, xi_Fe, Sec. 2.3 eqs (2-31)..(2-36).
void layer_porosity(const double *bed, int ore, double xi[3]) {
  const double q_mh = 2.0 * kMz[1] / (3.0 * kMz[0]);   // eq (2-36) for R1
  const double q_wm = 3.0 * kMz[2] / kMz[1];           // R2
  const double q_few = kMz[3] / kMz[2];                // R3
  const double *rt = bed + ORC_B_RHOT;
  double xi0 = bed[ORC_B_XI0 + ore];
  double rho_m;
  if (ore == 0) {
    double rho_h = (1.0 - xi0) * rt[0];                // eq (2-32)
    rho_m = rho_h * q_mh;                              // eq (2-33)
  } else {
    rho_m = (1.0 - xi0) * rt[1];  // Reading: for a magnetite ore the core is Fe3O4
  }
  double rho_w = rho_m * q_wm;                         // eq (2-34)
  double rho_fe = rho_w * q_few;                       // eq (2-35)
  xi[0] = 1.0 - rho_m / rt[1];                         // eq (2-31)
  xi[1] = 1.0 - rho_w / rt[2];
  xi[2] = 1.0 - rho_fe / rt[3];
}

// Gunn correlation, eqs (2-22) and (3-12).
template <class S> S gunn(double eps, const S &Re, double X) {
  double c13 = std::cbrt(X);
  return (7.0 - 10.0 * eps + 5.0 * eps * eps) * (1.0 + 0.7 * pow(Re, 0.2) * c13) +
         (1.33 - 2.4 * eps + 1.2 * eps * eps) * pow(Re, 0.7) * c13;
}

// ---------------------------------------------------------------------------------------
// Resistance network of Fig. 2(a) by Kirchhoff's voltage law along the three paths from
// the bulk gas to the three reaction interfaces (Sec. 2.1). Unknowns: the H2 fluxes J
// (m/s x mole fraction) consumed by R1, R2, R3. Path to interface k crosses the gas film
// F, the product layers outside it and the interface resistance A_k:
//   x - x_eq^hm  = (F+B_Fe)(J1+J2+J3) + B_w(J1+J2) + (B_m + A_hm) J1
//   x - x_eq^mw  = (F+B_Fe)(J1+J2+J3) + (B_w + A_mw)(J1+J2) - A_mw J1 ... written as a
// symmetric resistance matrix R below; J = R^{-1} (x - x_eq). The v_i^{kl} of eqs
// (2-2)..(2-10) are the entries of R^{-1}; inactive reactions are removed from the system
// (their A is infinite). Reading: a reaction whose flux comes out negative is removed and
// the network solved again (every reaction is irreversible, assumption (i) of Sec. 2).
// ---------------------------------------------------------------------------------------
template <class S>
bool solve_small(int m, S a[3][3], S inv[3][3]) {  // Gauss-Jordan with partial pivoting
  S w[3][6];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < 2 * m; ++j) w[i][j] = j < m ? a[i][j] : S(j - m == i ? 1.0 : 0.0);
  for (int c = 0; c < m; ++c) {
    int p = c;
    for (int i = c + 1; i < m; ++i)
      if (std::fabs(val(w[i][c])) > std::fabs(val(w[p][c]))) p = i;
    if (val(w[p][c]) == 0.0) return false;
    if (p != c)
      for (int j = 0; j < 2 * m; ++j) std::swap(w[p][j], w[c][j]);
    S piv = w[c][c];
    for (int j = 0; j < 2 * m; ++j) w[c][j] = w[c][j] / piv;
    for (int i = 0; i < m; ++i) {
      if (i == c) continue;
      S f = w[i][c];
      for (int j = 0; j < 2 * m; ++j) w[i][j] = w[i][j] - f * w[c][j];
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) inv[i][j] = w[i][m + j];
  return true;
}

template <class S>
void network(const S A[3], const S B[3], const S &F, int act[3], double x, const S xeq[3],
             S J[3], S v[3][3]) {
  // B = {B_m, B_w, B_Fe}; order of reactions: hm, mw, wFe.
  S Sr = F + B[2];
  S R[3][3];
  R[0][0] = Sr + B[1] + B[0] + A[0];
  R[0][1] = Sr + B[1];
  R[0][2] = Sr;
  R[1][0] = R[0][1];
  R[1][1] = Sr + B[1] + A[1];
  R[1][2] = Sr;
  R[2][0] = Sr;
  R[2][1] = Sr;
  R[2][2] = Sr + A[2];
  for (int r = 0; r < 3; ++r) { J[r] = S(0.0); for (int c = 0; c < 3; ++c) v[r][c] = S(0.0); }
  for (int iter = 0; iter < 4; ++iter) {
    int idx[3], m = 0;
    for (int r = 0; r < 3; ++r) if (act[r]) idx[m++] = r;
    for (int r = 0; r < 3; ++r) { J[r] = S(0.0); for (int c = 0; c < 3; ++c) v[r][c] = S(0.0); }
    if (m == 0) return;
    S a[3][3], inv[3][3];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) a[i][j] = R[idx[i]][idx[j]];
    if (!solve_small(m, a, inv)) return;
    for (int i = 0; i < m; ++i) {
      S s(0.0);
      for (int j = 0; j < m; ++j) s = s + inv[i][j] * (x - xeq[idx[j]]);
      J[idx[i]] = s;
      for (int j = 0; j < m; ++j) v[idx[i]][idx[j]] = inv[i][j];
    }
    bool neg = false;
    for (int i = 0; i < m; ++i)
      if (val(J[idx[i]]) < 0.0) { act[idx[i]] = 0; neg = true; }
    if (!neg) return;
  }
}

// ---------------------------------------------------------------------------------------
// USCM kinetics of one coarse-grained parcel (Sec. 2, Sec. 3.3): rates per real particle,
// then the k^3 scaling of eqs (3-49), (3-50), (3-52).
// ---------------------------------------------------------------------------------------
template <class S> struct Kin {
  S xidot[3], mdot[4], sH2, sH2O, Qr, Qrm, A[3], B[3], F, Sh, f[3], EQ, ES, Deff[3];
  int act[3];
  double xi[3];
};

template <class S>
void kinetics(const double *bed, const S m[4], const S &Tp, double dreal, int ore,
              const GasProps &g, double eps, const S &slip, double dtm, const S k0[3],
              const S Ea[3], Kin<S> &o) {
  const unsigned flags = (unsigned)ib(bed, ORC_B_FLAGS);
  const double k = bed[ORC_B_CG];
  const double k3 = k * k * k;
  for (int r = 0; r < 3; ++r) {
    o.xidot[r] = S(0.0); o.A[r] = S(0.0); o.B[r] = S(0.0); o.f[r] = S(0.0); o.Deff[r] = S(0.0);
    o.act[r] = 0;
  }
  for (int z = 0; z < 4; ++z) o.mdot[z] = S(0.0);
  o.sH2 = o.sH2O = o.Qr = o.Qrm = o.F = o.Sh = o.EQ = o.ES = S(0.0);
  layer_porosity(bed, ore, o.xi);
  // moles of each solid in one real particle
  S n[4];
  for (int z = 0; z < 4; ++z) n[z] = m[z] / (k3 * kMz[z]);
  S nfe = 2.0 * n[0] + 3.0 * n[1] + n[2] + n[3];
  if (!(val(nfe) > 0.0)) return;
  // eqs (2-15)..(2-17)
  o.f[0] = (3.0 * n[1] + n[2] + n[3]) / nfe;
  o.f[1] = (n[2] + n[3]) / nfe;
  o.f[2] = n[3] / nfe;
  S one_f[3] = {1.0 - o.f[0], 1.0 - o.f[1], 1.0 - o.f[2]};
  // eq (2-1-3) with Table 2
  S Keq[3], xeq[3], kr[3];
  for (int r = 0; r < 3; ++r) {
    Keq[r] = exp(kKeqA[r] / Tp + kKeqB[r]);
    xeq[r] = 1.0 / (Keq[r] + 1.0);
    kr[r] = k0[r] * exp(-Ea[r] / (kRg * Tp));          // eq (2-13)
  }
  const double x = g.x;
  // Reading: reaction kl runs iff its reactant is present and the bulk H2 fraction exceeds
  // its equilibrium fraction (this reproduces the cases of Fig. 2(b)-(g) and Fig. 4).
  bool kin_on = !(flags & ORC_NO_KINETICS);
  for (int r = 0; r < 3; ++r)
    o.act[r] = kin_on && val(n[r]) > 0.0 && x > val(xeq[r]) && val(k0[r]) > 0.0;
  for (int r = 0; r < 3; ++r)
    if (o.act[r]) o.A[r] = (1.0 / kr[r]) * pow(one_f[r], -2.0 / 3.0) * Keq[r] / (1.0 + Keq[r]);  // eq (2-12)
  // diffusion, Sec. 2.3
  const double pore = bed[ORC_B_PORE + ore];                    // cm
  const double DK = 0.97 * (0.5 * pore) * std::sqrt(g.T / (kMj[0] * 1e3));  // eq (2-28), m^2/s
  const double lam = x > 0.0 ? 1.013 / (g.p * x) : 1e300;        // cm, Sec. 2.3
  const double ratio = lam / pore;
  double D;
  if (ratio <= 0.01) D = g.Dm;
  else if (ratio >= 10.0) D = DK;
  else D = 1.0 / (1.0 / g.Dm + 1.0 / DK);                        // eq (2-29)
  const double tau = bed[ORC_B_TAU];
  for (int l = 0; l < 3; ++l) o.Deff[l] = S(D * o.xi[l] / tau);   // eq (2-30)
  const double rp = 0.5 * dreal;
  // eq (2-14); reading: l-1 is the inner interface of layer l (m: h|m .. m|w, w: m|w ..
  // w|Fe, Fe: w|Fe .. surface). A layer is only evaluated when a reaction behind it runs.
  if (!(flags & ORC_NO_LAYER)) {
    if (o.act[0]) o.B[0] = (rp / o.Deff[0]) * (pow(one_f[0], -1.0 / 3.0) - pow(one_f[1], -1.0 / 3.0));
    if ((o.act[0] || o.act[1]) && val(one_f[1]) > 0.0)
      o.B[1] = (rp / o.Deff[1]) * (pow(one_f[1], -1.0 / 3.0) - pow(one_f[2], -1.0 / 3.0));
    if (val(one_f[2]) > 0.0) o.B[2] = (rp / o.Deff[2]) * (pow(one_f[2], -1.0 / 3.0) - 1.0);
  }
  // gas film, eqs (2-20)..(2-24), with D_eff,f from eq (2-27)
  S Re = g.rho * eps * dreal * slip / g.mu;
  double Sc = g.mu / (g.rho * g.Dm);
  o.Sh = gunn(eps, Re, Sc);
  if (!(flags & ORC_NO_FILM)) o.F = dreal / (o.Sh * g.Dm);
  S J[3], v[3][3];
  network(o.A, o.B, o.F, o.act, x, xeq, J, v);
  // eq (2-1): molar H2 rate per real particle (eta = 1 for every reaction of Table 1)
  const double Ap = kPi * dreal * dreal;
  S c = Ap * g.p / (kRg * Tp);
  for (int r = 0; r < 3; ++r) o.xidot[r] = c * J[r];
  // Reading: a reaction is limited so that its reactant cannot go negative within the
  // mass-update interval; the limited rate is the one applied and deposited.
  const double nu[3] = {3.0, 1.0, 1.0};
  for (int r = 0; r < 3; ++r) {
    S cap = n[r] / (nu[r] * dtm);
    o.xidot[r] = smin(o.xidot[r], cap);
    if (val(o.xidot[r]) < 0.0) o.xidot[r] = S(0.0);
  }
  // Table 1 stoichiometry; eq (2-25); k^3 scaling eq (3-52)
  o.mdot[0] = -3.0 * o.xidot[0] * (kMz[0] * k3);
  o.mdot[1] = (2.0 * o.xidot[0] - o.xidot[1]) * (kMz[1] * k3);
  o.mdot[2] = (3.0 * o.xidot[1] - o.xidot[2]) * (kMz[2] * k3);
  o.mdot[3] = o.xidot[2] * (kMz[3] * k3);
  S tot = o.xidot[0] + o.xidot[1] + o.xidot[2];
  o.sH2 = -tot * (kMj[0] * k3);
  o.sH2O = tot * (kMj[1] * k3);
  // eqs (3-18)..(3-21) with H from eq (3-22) at the particle temperature; (3-49), (3-50)
  if (!(flags & ORC_NO_RXN_HEAT)) {
    S qr(0.0);
    for (int z = 0; z < 4; ++z) qr = qr + nasa_H(3 + z, Tp) * o.mdot[z];
    o.Qr = -qr;
    o.Qrm = -(nasa_H(0, Tp) * o.sH2 + nasa_H(1, Tp) * o.sH2O);
  }
  // Sec. 4.2: E = eta A_p / T_p, Q = sum of v_i, S = sum of v_i x_eq^i (times k^3 here)
  S Q(0.0), Ssum(0.0);
  for (int i = 0; i < 3; ++i) {
    S vi(0.0);
    for (int r = 0; r < 3; ++r) vi = vi + v[r][i];
    Q = Q + vi;
    Ssum = Ssum + vi * xeq[i];
  }
  S E = k3 * Ap / Tp;
  o.EQ = E * Q;
  o.ES = E * Ssum;
}

// Gidaspow-Ganser drag, eqs (3-5), (3-5-2)..(3-5-5). Returns beta/eps_p, so that the
// force beta V/(1-eps_g) (u-v) of eq (3-5) is (beta/eps_p) V (u-v); eps_p cancels exactly,
// which keeps a parcel that entered an empty cell (eps_g = 1, lagged) finite.
// Reading: the inertial Ergun term takes eps_p, as in the Gidaspow correlation that eq (3-5-1)
// cites and as Ergun's fixed-bed pressure drop requires (beta (u-v) = eps_g dp/dL); the printed
// eps_g there is read as a misprint. Then beta/eps_p = 150 eps_p mu/(eps_g d^2 psi^2)
// + 1.75 rho |u-v| / (d psi).
template <class S>
S drag_beta_over_epsp(const double *bed, double dreal, int ore, double eps, const S &slip,
                      const GasProps &g, S *Re_out) {
  const double psi = bed[ORC_B_PSI + ore];
  const double ep = 1.0 - eps;
  S Re = g.rho * eps * dreal * slip / g.mu;                        // eq (2-23)
  if (Re_out) *Re_out = Re;
  if (eps < 0.8) {
    return 150.0 * ep * g.mu / (eps * dreal * dreal * psi * psi) +
           1.75 * g.rho * slip / (dreal * psi);
  }
  const double K1 = 1.0 / (1.0 / 3.0 + (2.0 / 3.0) / std::sqrt(psi)) - 2.25 * dreal / bed[ORC_B_D];  // (3-5-4)
  const double K2 = std::pow(10.0, 1.8148 * std::pow(-std::log10(psi), 0.5743));                  // (3-5-5)
  const double epow = std::pow(eps, -2.65);
  if (val(Re) > 0.0) {
    S RK = Re * (K1 * K2);
    S CD = 24.0 / (Re * K1) * (1.0 + 0.1118 * pow(RK, 0.6567)) + 0.4305 * K2 / (1.0 + 3305.0 / RK);  // (3-5-3)
    return 0.75 * CD * eps * g.rho * slip / dreal * epow;
  }
  return S(0.75 * (24.0 / K1) * g.mu / (dreal * dreal) * epow);   // Re -> 0 limit
}

// ---------------------------------------------------------------------------------------
// Walls: signed distances to the analytic primitives of the reactor (IBM wall).
// Primitive 0 cylinder side, 1 bottom (plane z=0, or the cone of the conical bed),
// 2 perforated distributor plate (conical bed only), 3 lid z=H. Returns the distance from
// the parcel centre to the surface and the unit normal pointing from the wall to the centre.
// ---------------------------------------------------------------------------------------
void wall_distance(const double *bed, double x, double y, double z, double dist[4], double nrm[4][3]) {
  const double R = 0.5 * bed[ORC_B_D];
  const double H = bed[ORC_B_H];
  const int kind = ib(bed, ORC_B_WALL);
  for (int k = 0; k < 4; ++k) { dist[k] = 1e300; nrm[k][0] = nrm[k][1] = nrm[k][2] = 0.0; }
  double rho = std::sqrt(x * x + y * y);
  if (rho > 0.0) {
    dist[0] = R - rho;
    nrm[0][0] = -x / rho; nrm[0][1] = -y / rho; nrm[0][2] = 0.0;
  }
  if (kind == 0) {
    dist[1] = z;
    nrm[1][2] = 1.0;
  } else {
    const double al = bed[ORC_B_CONE_ALPHA];
    const double za = bed[ORC_B_CONE_H] - R / std::tan(al);
    // Reading: the cone acts only below the distributor plate.
    if (z < bed[ORC_B_PLATE_Z]) {
      double ca = std::cos(al), sa = std::sin(al);
      dist[1] = (z - za) * sa - rho * ca;
      if (rho > 0.0) { nrm[1][0] = -ca * x / rho; nrm[1][1] = -ca * y / rho; }
      else { nrm[1][0] = -ca; nrm[1][1] = 0.0; }
      nrm[1][2] = sa;
    }
    // perforated plate: zero-thickness plane with round holes on a square lattice
    const double pz = bed[ORC_B_PLATE_Z];
    const double pitch = bed[ORC_B_HOLE_PITCH];
    const double rh = 0.5 * bed[ORC_B_HOLE_D];
    double hx = std::floor(x / pitch + 0.5) * pitch;
    double hy = std::floor(y / pitch + 0.5) * pitch;
    double dx = x - hx, dy = y - hy, dz = z - pz;
    double q = std::sqrt(dx * dx + dy * dy);
    if (q >= rh) {
      dist[2] = std::fabs(dz);
      nrm[2][2] = dz >= 0.0 ? 1.0 : -1.0;
    } else {
      double ux = 1.0, uy = 0.0;
      if (q > 0.0) { ux = dx / q; uy = dy / q; }
      double ex = -(rh - q) * ux, ey = -(rh - q) * uy;   // centre minus nearest rim point
      double dd = std::sqrt(ex * ex + ey * ey + dz * dz);
      dist[2] = dd;
      if (dd > 0.0) { nrm[2][0] = ex / dd; nrm[2][1] = ey / dd; nrm[2][2] = dz / dd; }
      else nrm[2][2] = 1.0;
    }
  }
  dist[3] = H - z;
  nrm[3][2] = -1.0;
}

// Gas cell marking (IBM): a cell is solid when it lies wholly outside the fluid region,
// i.e. the signed distance of its centre to the fluid boundary is below minus half its
// diagonal (cylinder side; cone for the conical bed). Reading of the IBM mark of Sec. 4.
bool cell_is_solid(const double *bed, double xc, double yc, double zc, double hd) {
  const double R = 0.5 * bed[ORC_B_D];
  double rho = std::sqrt(xc * xc + yc * yc);
  double sd = R - rho;
  if (ib(bed, ORC_B_WALL) == 1) {
    const double al = bed[ORC_B_CONE_ALPHA];
    const double za = bed[ORC_B_CONE_H] - R / std::tan(al);
    double sc = (zc - za) * std::sin(al) - rho * std::cos(al);
    sd = std::min(sd, sc);
  }
  return sd < -hd;
}

// ---------------------------------------------------------------------------------------
// Contact law: linear spring-dashpot normal force, tangential spring with history and a
// Coulomb cap (the paper defers the law to another paper; the parameters are those of
// the benchmark beds). n points from the parcel to the partner (or wall).
// ---------------------------------------------------------------------------------------
struct ContactOut { double F[3]; double Tq[3]; double xi[3]; };

void contact_law(const double *bed, double mstar, double ri, const double n[3], double delta,
                 const double vrel[3], const double xi_old[3], const double w[3], ContactOut &o) {
  const double kn = bed[ORC_B_KN];
  const double kt = bed[ORC_B_KT_KN] * kn;
  const double e = bed[ORC_B_REST];
  const double le = std::log(e);
  const double eta_n = -2.0 * le * std::sqrt(mstar * kn / (kPi * kPi + le * le));
  const double eta_t = eta_n * std::sqrt(bed[ORC_B_KT_KN]);
  const double mu = bed[ORC_B_MU_S];
  const double mur = bed[ORC_B_MU_R];
  const double dt = bed[ORC_B_DT];
  double vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
  double vt[3] = {vrel[0] - vn * n[0], vrel[1] - vn * n[1], vrel[2] - vn * n[2]};
  double fn = kn * delta + eta_n * vn;   // repulsive magnitude (no tensile clamp)
  // rotate the stored tangential displacement into the current tangent plane
  double s = xi_old[0] * n[0] + xi_old[1] * n[1] + xi_old[2] * n[2];
  double xr[3] = {xi_old[0] - s * n[0], xi_old[1] - s * n[1], xi_old[2] - s * n[2]};
  double m_old = std::sqrt(xi_old[0] * xi_old[0] + xi_old[1] * xi_old[1] + xi_old[2] * xi_old[2]);
  double m_rot = std::sqrt(xr[0] * xr[0] + xr[1] * xr[1] + xr[2] * xr[2]);
  if (m_rot > 0.0) { double sc = m_old / m_rot; xr[0] *= sc; xr[1] *= sc; xr[2] *= sc; }
  double xi[3] = {xr[0] + vt[0] * dt, xr[1] + vt[1] * dt, xr[2] + vt[2] * dt};
  double ft[3] = {-kt * xi[0] - eta_t * vt[0], -kt * xi[1] - eta_t * vt[1], -kt * xi[2] - eta_t * vt[2]};
  double ftm = std::sqrt(ft[0] * ft[0] + ft[1] * ft[1] + ft[2] * ft[2]);
  double cap = mu * std::fabs(fn);
  if (ftm > cap) {
    double sc = cap / ftm;
    for (int c = 0; c < 3; ++c) {
      ft[c] *= sc;
      xi[c] = -(ft[c] + eta_t * vt[c]) / kt;
    }
  }
  for (int c = 0; c < 3; ++c) o.F[c] = -fn * n[c] + ft[c];
  // torque of the tangential force about the centre, lever arm r_i n (eq (3-6))
  o.Tq[0] = ri * (n[1] * ft[2] - n[2] * ft[1]);
  o.Tq[1] = ri * (n[2] * ft[0] - n[0] * ft[2]);
  o.Tq[2] = ri * (n[0] * ft[1] - n[1] * ft[0]);
  // Reading of eq (3-6): rolling resistance torque -mu_r |F_n| w/|w| (mu_r a length).
  if (mur > 0.0) {
    double wm = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (wm > 0.0)
      for (int c = 0; c < 3; ++c) o.Tq[c] -= mur * std::fabs(fn) * w[c] / wm;
  }
  for (int c = 0; c < 3; ++c) o.xi[c] = xi[c];
}

// ---------------------------------------------------------------------------------------
// Contact heat conduction: particle-particle (eq (3-14)), particle-fluid-particle
// (eq (3-15)), particle-wall and particle-fluid-wall (eqs (3-15-1), (3-15-2)), with the
// coarse-grained scaling of Sec. 3.3 (eqs (3-42)..(3-48-2)). The paper takes the meaning
// of R_c, lambda_e and the integration limits from another paper; the readings:
//   * both sums run over the contacts of eq (3-3) (the same n_b parcels and walls);
//   * R_c is the radius of the circle in which the two overlapping spheres intersect (for
//     a wall: in which the sphere meets the wall's tangent plane);
//   * lambda_e is the series conductance of the two constrictions, lambda_a lambda_b /
//     (lambda_a + lambda_b) (for two equal spheres Q = 2 lambda a dT, the constriction
//     resistance 1/(4 lambda a) of each side in series); lambda_p per ore type and the
//     wall's lambda_w are bed parameters;
//   * the fluid lens of eq (3-15) spans the smaller sphere's projected disk (R_out =
//     min(R_a, R_b); a wall: r_out = R) and ends where the gap between the surfaces falls
//     below the gas mean free path of Sec. 2.3 for hydrogen at the bed pressure,
//     L_min = 1.013 / p cm (R_in, r_in); lambda_g is the mean of the two parcels' cells'
//     (a wall: the parcel's cell);
//   * the wall is at the bed's inlet temperature (Table 3 lists them equal);
//   * eq (3-43) as printed is garbled; it is read as the maximum overlap of a damped
//     linear spring-dashpot collision in units of v/omega_0,
//     f(e) = exp(-zeta arccos(zeta) / sqrt(1 - zeta^2)), zeta of eq (3-44);
//   * e_CGP of eq (3-45) has no real value for k >= 1/(1 - e^2) (5.26 at e = 0.9); it is
//     clamped at 0, where f takes its limit exp(-1) (critical damping).
// ---------------------------------------------------------------------------------------
double restitution_f(double e) {
  if (!(e > 0.0)) return std::exp(-1.0);
  if (e >= 1.0) return 1.0;
  const double le = std::log(e);
  const double zeta = -le / std::sqrt(kPi * kPi + le * le);         // eq (3-44)
  return std::exp(-zeta * std::acos(zeta) / std::sqrt(1.0 - zeta * zeta));   // eq (3-43)
}
double e_cgp(double e, double k) {                                   // eq (3-45)
  const double a = 1.0 + k * (e * e - 1.0);
  return a > 0.0 ? std::sqrt(a) : 0.0;
}
// adaptive Simpson quadrature of f over [a, b] to an absolute tolerance
template <class F> double simpson_rec(F &f, double a, double b, double fa, double fm, double fb, double whole,
                                      double tol, int depth) {
  const double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  const double flm = f(lm), frm = f(rm);
  const double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm), right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  const double diff = left + right - whole;
  if (depth <= 0 || std::fabs(diff) <= 15.0 * tol) return left + right + diff / 15.0;
  return simpson_rec(f, a, m, fa, flm, fm, left, 0.5 * tol, depth - 1) +
         simpson_rec(f, m, b, fm, frm, fb, right, 0.5 * tol, depth - 1);
}
template <class F> double simpson(F f, double a, double b, double tol) {
  const double fa = f(a), fb = f(b), fm = f(0.5 * (a + b));
  return simpson_rec(f, a, b, fa, fm, fb, (b - a) / 6.0 * (fa + 4.0 * fm + fb), tol, 48);
}
inline double gap_lmin(const double *bed) { return 1.013e-2 / bed[ORC_B_P0]; }   // m (Sec. 2.3, x = 1)
// eq (3-15): int_{R_in}^{R_out} R / (d - sqrt(Ra^2 - R^2) - sqrt(Rb^2 - R^2)) dR
double lens_integral_pair(double Ra, double Rb, double d, double Lmin) {
  auto L = [&](double R) { return d - std::sqrt(Ra * Ra - R * R) - std::sqrt(Rb * Rb - R * R); };
  const double Rout = std::min(Ra, Rb);
  if (!(L(Rout) > Lmin)) return 0.0;
  double lo = 0.0, hi = Rout;   // L increases with R: R_in where L(R_in) = L_min
  if (L(lo) < Lmin) {
    for (int it = 0; it < 200 && hi - lo > 1e-20; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (L(mid) < Lmin) lo = mid; else hi = mid;
    }
    lo = hi;
  }
  const double scale = Rout * Rout / Lmin;
  return simpson([&](double R) { return R / L(R); }, lo, Rout, 1e-13 * scale);
}
// eq (3-15-2): int_{r_in}^{r_out} r / L_w dr with L_w = h - sqrt(R^2 - r^2)
double lens_integral_wall(double R, double h, double Lmin) {
  if (!(h > Lmin)) return 0.0;
  const double u = h - Lmin;
  const double rin = u < R ? std::sqrt(R * R - u * u) : 0.0;
  const double scale = R * R / Lmin;
  return simpson([&](double r) { return r / (h - std::sqrt(R * R - r * r)); }, rin, R, 1e-13 * scale);
}
// Q into parcel a from a parcel b in contact (scaled to the coarse-grained system)
void conduction_pair(const double *bed, double Ra, double Rb, double d, double Ta, double Tb, double lam_a,
                     double lam_b, double lam_g, double out[4]) {
  const double k = bed[ORC_B_CG];
  const double e = bed[ORC_B_REST];
  const double delta = Ra + Rb - d;
  // radius of the intersection circle of the two spheres
  const double Rc = std::sqrt(delta * (d + Ra + Rb) * (d + Ra - Rb) * (d - Ra + Rb)) / (2.0 * d);
  const double lam_e = lam_a * lam_b / (lam_a + lam_b);
  const double Qpp = 4.0 * Rc * lam_e * (Tb - Ta);                              // eq (3-14)
  const double I = lens_integral_pair(Ra, Rb, d, gap_lmin(bed));
  const double Qpfp = 2.0 * kPi * lam_g * (Tb - Ta) * I;                        // eq (3-15)
  const double sc = std::pow(k, 0.75) * std::sqrt(restitution_f(e) / restitution_f(e_cgp(e, k)));
  out[0] = sc * Qpp;                                                            // eq (3-46)
  out[1] = k * k * Qpfp;                                                        // eq (3-48)
  out[2] = Rc;
  out[3] = I;
}
void conduction_wall(const double *bed, double R, double h, double Ta, double lam_a, double lam_g, double out[4]) {
  const double k = bed[ORC_B_CG];
  const double e = bed[ORC_B_REST];
  const double Tw = bed[ORC_B_T_IN];
  const double lam_w = bed[ORC_B_LAMW];
  const double delta = R - h;
  const double Rc = std::sqrt(delta * (2.0 * R - delta));
  const double lam_e = lam_a * lam_w / (lam_a + lam_w);
  const double Qpw = 4.0 * Rc * lam_e * (Tw - Ta);                              // eq (3-15-1)
  const double I = lens_integral_wall(R, h, gap_lmin(bed));
  const double Qpfw = 2.0 * kPi * lam_g * (Tw - Ta) * I;                        // eq (3-15-2)
  const double sc = std::pow(k, 0.75) * std::sqrt(restitution_f(e) / restitution_f(e_cgp(e, k)));
  out[0] = sc * Qpw;                                                            // eq (3-48-1)
  out[1] = k * k * Qpfw;                                                        // eq (3-48-2)
  out[2] = Rc;
  out[3] = I;
}

struct Contact { int32_t partner; double xi[3]; };

struct Grid {
  int nx, ny, nz;
  double x0, y0, z0, dx, dy, dz, ix, iy, iz;
};
Grid make_grid(const double *bed) {
  Grid g;
  g.nx = ib(bed, ORC_B_NX); g.ny = ib(bed, ORC_B_NY); g.nz = ib(bed, ORC_B_NZ);
  double D = bed[ORC_B_D], H = bed[ORC_B_H];
  g.x0 = -0.5 * D; g.y0 = -0.5 * D; g.z0 = 0.0;
  g.dx = D / g.nx; g.dy = D / g.ny; g.dz = H / g.nz;
  g.ix = 1.0 / g.dx; g.iy = 1.0 / g.dy; g.iz = 1.0 / g.dz;
  return g;
}
// cell containing a point: floor((x - x0) * (1/dx)), clamped to the grid
inline int64_t cell_of(const Grid &g, double x, double y, double z, bool *outside) {
  double fx = std::floor((x - g.x0) * g.ix), fy = std::floor((y - g.y0) * g.iy), fz = std::floor((z - g.z0) * g.iz);
  bool out = !(fx >= 0.0 && fx < g.nx && fy >= 0.0 && fy < g.ny && fz >= 0.0 && fz < g.nz);
  if (outside) *outside = out;
  int64_t ix = (int64_t)std::min(std::max(fx, 0.0), (double)(g.nx - 1));
  int64_t iy = (int64_t)std::min(std::max(fy, 0.0), (double)(g.ny - 1));
  int64_t iz = (int64_t)std::min(std::max(fz, 0.0), (double)(g.nz - 1));
  return (iz * g.ny + iy) * g.nx + ix;
}

// Pair search on a plain uniform cell list; contact iff d^2 < (r_i + r_j)^2 with
// d^2 = (dx*dx + dy*dy) + dz*dz, dx = x_j - x_i, in IEEE double without contraction.
inline bool touching(double xi, double yi, double zi, double xj, double yj, double zj, double rs) {
  double dx = xj - xi, dy = yj - yi, dz = zj - zi;
  double d2 = (dx * dx + dy * dy) + dz * dz;
  return d2 < rs * rs;
}

struct CellList {
  // cells of edge h over the bounding box of the parcels; (cell key, parcel) pairs sorted
  // by key, and neighbours found by binary search of the 27 surrounding keys
  double h, x0, y0, z0;
  int64_t nx, ny, nz;
  std::vector<std::pair<int64_t, int32_t>> items;
  void build(const std::vector<int32_t> &ids, const double *x, const double *y, const double *z,
             double hcell) {
    h = hcell;
    double mnx = 1e300, mny = 1e300, mnz = 1e300, mxx = -1e300, mxy = -1e300, mxz = -1e300;
    for (int32_t i : ids) {
      mnx = std::min(mnx, x[i]); mny = std::min(mny, y[i]); mnz = std::min(mnz, z[i]);
      mxx = std::max(mxx, x[i]); mxy = std::max(mxy, y[i]); mxz = std::max(mxz, z[i]);
    }
    if (ids.empty()) { mnx = mny = mnz = 0; mxx = mxy = mxz = 0; }
    x0 = mnx; y0 = mny; z0 = mnz;
    nx = (int64_t)((mxx - mnx) / h) + 1; ny = (int64_t)((mxy - mny) / h) + 1; nz = (int64_t)((mxz - mnz) / h) + 1;
    items.resize(ids.size());
    for (size_t t = 0; t < ids.size(); ++t) {
      int32_t i = ids[t];
      items[t] = {coord(x[i], y[i], z[i]), i};
    }
    std::sort(items.begin(), items.end());
  }
  int64_t cx(double v, double o, int64_t n) const {
    int64_t c = (int64_t)std::floor((v - o) / h);
    return std::min(std::max(c, (int64_t)0), n - 1);
  }
  int64_t coord(double x, double y, double z) const {
    return (cx(z, z0, nz) * ny + cx(y, y0, ny)) * nx + cx(x, x0, nx);
  }
  template <class F> void neighbours(double x, double y, double z, F f) const {
    int64_t a = cx(x, x0, nx), b = cx(y, y0, ny), c = cx(z, z0, nz);
    for (int64_t k = std::max<int64_t>(c - 1, 0); k <= std::min(c + 1, nz - 1); ++k)
      for (int64_t j = std::max<int64_t>(b - 1, 0); j <= std::min(b + 1, ny - 1); ++j)
        for (int64_t i = std::max<int64_t>(a - 1, 0); i <= std::min(a + 1, nx - 1); ++i) {
          int64_t cc = (k * ny + j) * nx + i;
          auto it = std::lower_bound(items.begin(), items.end(), std::make_pair(cc, INT32_MIN));
          for (; it != items.end() && it->first == cc; ++it) f(it->second);
        }
  }
};

// ---------------------------------------------------------------------------------------
// The stateful oracle.
// ---------------------------------------------------------------------------------------
struct Oracle {
  int nb = 0, n = 0;
  std::vector<double> beds;                  // nb * ORC_NB
  std::vector<double> s[ORC_NS];             // state rows
  std::vector<double> dreal;
  std::vector<int32_t> ore, bed;
  std::vector<std::vector<Contact>> hist;
  std::vector<double> diag;                  // ORC_ND * n
  std::vector<int64_t> cell_off;             // per bed offset into gas arrays
  std::vector<double> gas;                   // ORC_NG per cell
  std::vector<double> dep;                   // ORC_NDEP per cell
  std::vector<std::vector<int32_t>> members; // parcel ids of each bed
  int64_t step_no = 0;
  int64_t ncell_total = 0;
  // solved gas phase (beds with ORC_GAS_SOLVER): face velocities on a staggered grid and the
  // cell pressure relative to p0, per bed; eps of the previous coupling step per cell
  std::vector<std::vector<double>> fu, fv, fw, pr;
  const double *B(int b) const { return beds.data() + (size_t)b * ORC_NB; }
};

double parcel_mass(const Oracle &o, int i) {
  return o.s[ORC_S_M][i] + o.s[ORC_S_M + 1][i] + o.s[ORC_S_M + 2][i] + o.s[ORC_S_M + 3][i];
}

void deposit_volume_and_eps(Oracle &o) {
  // initial gas volume fraction from the parcel volumes in each cell (Sec. 3.2)
  std::fill(o.dep.begin(), o.dep.end(), 0.0);
  for (int b = 0; b < o.nb; ++b) {
    const double *bd = o.B(b);
    Grid g = make_grid(bd);
    double k = bd[ORC_B_CG];
    for (int32_t i : o.members[b]) {
      int64_t c = o.cell_off[b] + cell_of(g, o.s[0][i], o.s[1][i], o.s[2][i], nullptr);
      double dc = k * o.dreal[i];
      o.dep[c * ORC_NDEP + ORC_DEP_VS] += kPi / 6.0 * dc * dc * dc;
    }
    double V = g.dx * g.dy * g.dz;
    int64_t nc = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t c = 0; c < nc; ++c) {
      double *gc = &o.gas[(o.cell_off[b] + c) * ORC_NG];
      if (gc[ORC_G_MARK] != 0.0) { gc[ORC_G_EPS] = bd[ORC_B_EPS_MIN]; continue; }
      gc[ORC_G_EPS] = std::max(1.0 - o.dep[(o.cell_off[b] + c) * ORC_NDEP + ORC_DEP_VS] / V, bd[ORC_B_EPS_MIN]);
    }
  }
  std::fill(o.dep.begin(), o.dep.end(), 0.0);
}

// ---------------------------------------------------------------------------------------
// Gas phase solver (Sec. 3.2, Sec. 4.1, Sec. 4.2), in beds with ORC_GAS_SOLVER, once per
// coupling step with dt_CFD = n dt_DEM: continuity (eq (3-24)), momentum with the
// semi-implicit drag of eq (4-2), energy with the semi-implicit H0 of eq (4-6), the reducing
// gas with the semi-implicit C0, C1 of eq (4-9), the pseudo-turbulent stress and heat flux
// of eqs (3-28)..(3-37). Readings (the paper solves the gas with OpenFOAM's schemes, Table 4):
//   * staggered (MAC) grid on the gas cells: velocity components on the faces, scalars at
//     the centres; explicit Euler in time, first-order upwind convection (Table 4 uses
//     limitedLinear for velocity and species); species and energy first, with the mass
//     fluxes of the last projection; continuity in the low-Mach divergence form
//     div(eps u) = -d eps/dt + M / rho - eps D ln(rho)/Dt (eq (3-24) with rho = p M_g / (R T)
//     at fixed p0 and the material rates of the species and energy update, so that the
//     oxygen the reactions add to the gas raises its density instead of leaving as extra
//     volume flow); then momentum and an incremental pressure projection for that
//     divergence, solved by conjugate gradients; the inlet carries the inlet gas's density;
//   * momentum: convection in non-conservative form, viscous stress as div(eps mu grad u)
//     (the transpose and dilatation parts of eq (3-33) dropped), the divergence of the
//     pseudo-turbulent stress by its normal components, gravity, the drag of eq (4-2) with
//     K_gp u_g implicit and K_gp u_p explicit, where K_gp = -(1/V) sum beta V_p/(1 - eps_g)
//     and K_gp u_p = -(1/V) sum beta V_p/(1 - eps_g) v_p (the reaction to the parcels' drag);
//   * boundaries: immersed-boundary cells and the box sides are no-slip walls; a face below a
//     fluid cell whose lower neighbour is solid or outside takes the inlet gas at the
//     superficial velocity U_in (eps u = U_in, Y_in, T_in); the top is an outlet at p0; walls
//     hold the bed's inlet temperature (Table 3 lists them equal) and conduct heat to the gas;
//   * the reducing gas H2 with eqs (4-8)..(4-11) as printed (x_H2 = M_g Y_H2 / (M_H2 X),
//     M_g and X lagged), H2O produced at M_H2O / M_H2 times the H2 consumed (eq (2-25)), N2
//     by closure; molecular diffusion with D_H2,m of eq (2-27) for every species;
//   * the pseudo-turbulence closures with the cell's drag-weighted mean parcel velocity
//     (u_p = K_gp u_p / K_gp), the volume-mean real diameter of its parcels and
//     Re_m = eps rho |u_g - u_p| d_p / mu, evaluated as printed (Re_m capped at 100 and
//     eps_p at 0.5, the upper ends of the closures' ranges); R and alpha_PT are rotated to
//     the slip direction s: R = R_pe I + (R_pa - R_pe) s s^T (the Gram-Schmidt frame's
//     perpendicular axes drop out), and only their diagonal enters the fluxes (cross-
//     derivative terms dropped); D_PT = alpha_PT.
// ---------------------------------------------------------------------------------------
struct FlowGrid {
  int nx, ny, nz;
  double hx, hy, hz;
  int64_t off;
  const double *gas;
  int64_t cidx(int i, int j, int k) const { return ((int64_t)k * ny + j) * nx + i; }
  bool fluid(int i, int j, int k) const {
    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return false;
    return gas[(off + cidx(i, j, k)) * ORC_NG + ORC_G_MARK] == 0.0;
  }
  int64_t xf(int i, int j, int k) const { return ((int64_t)k * ny + j) * (nx + 1) + i; }
  int64_t yf(int i, int j, int k) const { return ((int64_t)k * (ny + 1) + j) * nx + i; }
  int64_t zf(int i, int j, int k) const { return ((int64_t)k * ny + j) * nx + i; }
};
// face kind: 0 wall, 1 open (fluid on both sides), 2 inlet, 3 outlet
int face_kind(const FlowGrid &g, int a, int i, int j, int k) {
  int di = a == 0, dj = a == 1, dk = a == 2;
  bool lo = g.fluid(i - di, j - dj, k - dk), hi = g.fluid(i, j, k);
  if (lo && hi) return 1;
  if (a == 2 && hi && !lo) return 2;
  if (a == 2 && lo && k == g.nz) return 3;
  return 0;
}
// pseudo-turbulence coefficients of a cell: R_pa, R_pe, alpha_pa, alpha_pe and the slip direction
struct PT { double Rpa, Rpe, apa, ape, s[3]; };
PT pseudo_turbulence(double eps, double rho, double mu, double lam, double cp, const double ug[3],
                     const double up[3], double dp) {
  PT t{0, 0, 0, 0, {0, 0, 0}};
  const double ep = 1.0 - eps;
  double sl[3] = {ug[0] - up[0], ug[1] - up[1], ug[2] - up[2]};
  const double sm = std::sqrt(sl[0] * sl[0] + sl[1] * sl[1] + sl[2] * sl[2]);
  if (!(ep > 0.0) || !(sm > 0.0) || !(dp > 0.0)) return t;
  for (int q = 0; q < 3; ++q) t.s[q] = sl[q] / sm;
  const double Rem = std::min(eps * rho * sm * dp / mu, 100.0);
  const double epc = std::min(ep, 0.5);
  const double Eg = 0.5 * sm * sm;                                                   // eq (3-30)
  const double kg = Eg * (2.0 * ep + 2.5 * ep * eps * eps * eps * std::exp(-ep * std::sqrt(Rem)));   // eq (3-29)
  const double bpa = 0.523 / (1.0 + 0.305 * std::exp(-0.114 * Rem)) *
                     std::exp(-3.511 * ep / (1.0 + 1.801 * std::exp(-0.005 * Rem)));  // eq (3-31)
  const double bpe = -0.5 * bpa;                                                     // eq (3-32)
  t.Rpa = 2.0 * kg * (bpa + 1.0 / 3.0);                                               // eq (3-28)
  t.Rpe = 2.0 * kg * (bpe + 1.0 / 3.0);
  const double Pr = cp * mu / lam;
  const double ag = lam / (rho * cp);
  const double Num = (-0.46 + 1.77 * eps + 0.69 * eps * eps) / (eps * eps * eps) +
                     (1.37 - 2.4 * eps + 1.2 * eps * eps) * std::pow(Rem, 0.7) * std::cbrt(Pr);   // eq (3-36)
  const double num = 1.4 * Rem * (Rem + 1.4) * Pr * std::exp(-0.002089 * Rem) *
                     (eps * (-5.11 * epc + 10.1 * epc * epc - 10.85 * epc * epc * epc) + 1.0 - std::exp(-10.96 * epc));
  const double den = 3.0 * kPi * eps * eps * Num *
                     (1.17 * epc - 0.2021 * std::sqrt(epc) + 0.08568 * std::pow(epc, 0.25)) *
                     (1.0 - 1.6 * epc * eps - 3.0 * epc * std::pow(eps, 4.0) * std::exp(-std::pow(Rem, 0.4) * epc));
  t.apa = den > 0.0 ? ag * num / den : 0.0;                                           // eq (3-35)
  t.ape = (3.0 * bpe + 1.0) / (3.0 * bpa + 1.0) * t.apa;                               // eq (3-37)
  return t;
}
inline double pt_diag(const PT &t, int a, bool heat) {
  const double pa = heat ? t.apa : t.Rpa, pe = heat ? t.ape : t.Rpe;
  return pe + (pa - pe) * t.s[a] * t.s[a];
}

// one gas step of bed b over dt, from the gas state and the parcels' cell sums in o.dep
void gas_solve(Oracle &o, int b, const std::vector<GasProps> &gp, double dt) {
  const double *bd = o.B(b);
  const Grid gg = make_grid(bd);
  FlowGrid g{gg.nx, gg.ny, gg.nz, gg.dx, gg.dy, gg.dz, o.cell_off[b], o.gas.data()};
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int64_t nc = (int64_t)nx * ny * nz, off = g.off;
  const double V = g.hx * g.hy * g.hz;
  const double h[3] = {g.hx, g.hy, g.hz};
  const double Af[3] = {g.hy * g.hz, g.hx * g.hz, g.hx * g.hy};
  const double k = bd[ORC_B_CG], k3 = k * k * k;
  const double Uin = bd[ORC_B_U_IN], Tin = bd[ORC_B_T_IN], p0 = bd[ORC_B_P0];
  const double grav = ((unsigned)ib(bd, ORC_B_FLAGS) & ORC_NO_GRAVITY) ? 0.0 : -kG;
  std::vector<double> &U = o.fu[b], &Vv = o.fv[b], &W = o.fw[b], &P = o.pr[b];
  auto comp = [&](int a) -> std::vector<double> & { return a == 0 ? U : (a == 1 ? Vv : W); };
  auto fidx = [&](int a, int i, int j, int kk) { return a == 0 ? g.xf(i, j, kk) : (a == 1 ? g.yf(i, j, kk) : g.zf(i, j, kk)); };
  // per-cell coefficients from the old state and the cell sums (eps: this coupling step's, from
  // the deposited parcel volume; epso: the last one's)
  std::vector<double> eps(nc), epso(nc), rho(nc), mu(nc), lam(nc), cp(nc), Dm(nc), Kc(nc), Kv(3 * nc), RT(3 * nc),
      AT(3 * nc), uc(3 * nc);
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int64_t c = g.cidx(i, j, kk);
        const double *gc = &o.gas[(off + c) * ORC_NG];
        const double *dp = &o.dep[(off + c) * ORC_NDEP];
        const GasProps &G = gp[off + c];
        epso[c] = gc[ORC_G_EPS];   // the last coupling step's
        eps[c] = g.fluid(i, j, kk) ? std::max(1.0 - dp[ORC_DEP_VS] / V, bd[ORC_B_EPS_MIN]) : bd[ORC_B_EPS_MIN];
        rho[c] = G.rho; mu[c] = G.mu; lam[c] = G.lam; cp[c] = G.cp; Dm[c] = G.Dm;
        Kc[c] = dp[ORC_DEP_K] / V;
        for (int q = 0; q < 3; ++q) Kv[3 * c + q] = dp[ORC_DEP_KV + q] / V;
        uc[3 * c + 0] = 0.5 * (U[g.xf(i, j, kk)] + U[g.xf(i + 1, j, kk)]);
        uc[3 * c + 1] = 0.5 * (Vv[g.yf(i, j, kk)] + Vv[g.yf(i, j + 1, kk)]);
        uc[3 * c + 2] = 0.5 * (W[g.zf(i, j, kk)] + W[g.zf(i, j, kk + 1)]);
        PT t{0, 0, 0, 0, {0, 0, 0}};
        if (g.fluid(i, j, kk) && dp[ORC_DEP_K] > 0.0 && dp[ORC_DEP_COUNT] > 0.0) {
          const double upv[3] = {dp[ORC_DEP_KV] / dp[ORC_DEP_K], dp[ORC_DEP_KV + 1] / dp[ORC_DEP_K],
                                 dp[ORC_DEP_KV + 2] / dp[ORC_DEP_K]};
          const double dpm = std::cbrt(6.0 * dp[ORC_DEP_VS] / (kPi * dp[ORC_DEP_COUNT] * k3));
          t = pseudo_turbulence(eps[c], rho[c], mu[c], lam[c], cp[c], &uc[3 * c], upv, dpm);
        }
        for (int a = 0; a < 3; ++a) { RT[3 * c + a] = pt_diag(t, a, false); AT[3 * c + a] = pt_diag(t, a, true); }
      }
  // face mass flux (kg/s along +axis) of velocity u through a face of kind kd, with the cell
  // densities r; the inlet carries the inlet gas (eps u = U_in at its density)
  const double Yin[3] = {bd[ORC_B_Y_IN], bd[ORC_B_Y_IN + 1], bd[ORC_B_Y_IN + 2]};
  const double rho_in = gas_props(Tin, Yin, p0).rho;
  auto face_flux = [&](int a, int i, int j, int kk, int kd, double u, const std::vector<double> &r) -> double {
    const int di = a == 0, dj = a == 1, dk = a == 2;
    if (kd == 0) return 0.0;
    if (kd == 2) return rho_in * Uin * Af[a];
    const int64_t cP = g.cidx(i - di, j - dj, kk - dk);
    if (kd == 3) return eps[cP] * r[cP] * u * Af[a];
    const int64_t cN = g.cidx(i, j, kk);
    return 0.5 * (eps[cP] + eps[cN]) * 0.5 * (r[cP] + r[cN]) * u * Af[a];
  };
  // 1. species (eq (4-9)) and energy (eq (4-6)) with the mass fluxes of the last projection
  //    (the current face velocities, the old densities); from their non-advective rates the
  //    velocity divergence that continuity (eq (3-24)) requires of the new flow: with
  //    rho = p M_g / (R T) (eq (3-53)) at fixed p0, d(eps rho)/dt + div(eps rho u) = M reads
  //    div(eps u) = -d eps/dt + M / rho - eps D ln(rho)/Dt, and
  //    D ln(rho)/Dt = -M_g sum_j (DY_j/Dt) / M_j - (DT/Dt) / T, DY_j/Dt and DT/Dt the changes
  //    of the update less its convective part (the low-Mach divergence form: an equimolar
  //    reaction, H2 to H2O, leaves the volume flow unchanged)
  std::vector<double> nxt(o.gas.begin() + off * ORC_NG, o.gas.begin() + (off + nc) * ORC_NG);
  const double MH2 = kMj[0], MH2O = kMj[1];
  std::vector<double> divg(nc, 0.0);
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if (!g.fluid(i, j, kk)) continue;
        const int64_t c = g.cidx(i, j, kk);
        const double *gc = &o.gas[(off + c) * ORC_NG];
        const double *dp = &o.dep[(off + c) * ORC_NDEP];
        const GasProps &G = gp[off + c];
        const double Y0 = gc[ORC_G_Y], Y1 = gc[ORC_G_Y + 1], T = gc[ORC_G_T];
        double cY0 = 0.0, cY1 = 0.0, cT = 0.0, dY0 = 0.0, dY1 = 0.0, dT = 0.0;
        for (int a = 0; a < 3; ++a) {
          const int di = a == 0, dj = a == 1, dk = a == 2;
          for (int side = 0; side < 2; ++side) {   // 0: low face, 1: high face
            const int fi = i + side * di, fj = j + side * dj, fk = kk + side * dk;
            const int kd = face_kind(g, a, fi, fj, fk);
            const double F = kd == 0 ? 0.0 : face_flux(a, fi, fj, fk, kd, comp(a)[fidx(a, fi, fj, fk)], rho);
            const double inflow = side == 0 ? F : -F;   // mass into the cell through this face
            const int ni = i + (side ? di : -di), nj = j + (side ? dj : -dj), nk = kk + (side ? dk : -dk);
            if (kd == 1) {
              const int64_t cn = g.cidx(ni, nj, nk);
              const double *gn = &o.gas[(off + cn) * ORC_NG];
              if (inflow > 0.0) {
                cY0 += inflow * (gn[ORC_G_Y] - Y0);
                cY1 += inflow * (gn[ORC_G_Y + 1] - Y1);
                cT += inflow * cp[c] * (gn[ORC_G_T] - T);
              }
              const double ef = 0.5 * (eps[c] + eps[cn]), rf = 0.5 * (rho[c] + rho[cn]);
              const double Df = 0.5 * (Dm[c] + Dm[cn]) + 0.5 * (AT[3 * c + a] + AT[3 * cn + a]);
              const double lf = 0.5 * (lam[c] + lam[cn]) + rf * 0.5 * (cp[c] + cp[cn]) * 0.5 * (AT[3 * c + a] + AT[3 * cn + a]);
              dY0 += ef * rf * Df * Af[a] / h[a] * (gn[ORC_G_Y] - Y0);
              dY1 += ef * rf * Df * Af[a] / h[a] * (gn[ORC_G_Y + 1] - Y1);
              dT += ef * lf * Af[a] / h[a] * (gn[ORC_G_T] - T);
            } else if (kd == 2) {                 // inlet gas
              if (inflow > 0.0) {
                cY0 += inflow * (Yin[0] - Y0);
                cY1 += inflow * (Yin[1] - Y1);
                cT += inflow * cp[c] * (Tin - T);
              }
            } else if (kd == 0) {                 // wall at the inlet temperature
              dT += eps[c] * lam[c] * Af[a] / (0.5 * h[a]) * (Tin - T);
            }                                     // outlet: zero gradient
          }
        }
        const double m = eps[c] * rho[c] * V;
        // eqs (4-8)..(4-11): H2 consumed at (M_H2 p / R)(x EQ - ES) with x = a Y_H2 (implicit in
        // Y_H2), H2O produced at M_H2O / M_H2 times that; in the non-conservative form the
        // net mass source takes Y (and c_p T) of the cell away
        const double X = G.xp[0] + G.xp[1];
        const double ax = X > 0.0 ? G.Mg / (MH2 * X) : 0.0;
        const double C0 = MH2 * p0 * ax * dp[ORC_DEP_EQ] / kRg, C1 = MH2 * p0 * dp[ORC_DEP_ES] / kRg;
        const double rq = MH2O / MH2 - 1.0;
        const double Y0n = (m * Y0 / dt + cY0 + dY0 + C1 * (1.0 + Y0 * rq)) / (m / dt + C0 * (1.0 + Y0 * rq));
        const double cons = C0 * Y0n - C1;                        // H2 consumed, kg/s
        const double Mnet = rq * cons;                            // net gas mass source, kg/s
        double Y0f = Y0n;
        double Y1f = Y1 + dt / m * (cY1 + dY1 + MH2O / MH2 * cons - Y1 * Mnet);
        Y0f = std::max(Y0f, 0.0);
        Y1f = std::max(Y1f, 0.0);
        double Y2f = std::max(1.0 - Y0f - Y1f, 0.0);
        const double ys = Y0f + Y1f + Y2f;
        double *nc_ = &nxt[c * ORC_NG];
        nc_[ORC_G_Y] = Y0f / ys;
        nc_[ORC_G_Y + 1] = Y1f / ys;
        nc_[ORC_G_Y + 2] = Y2f / ys;
        // energy: M_r of eq (3-39) with the parcels' species sources (as the prescribed update
        // takes it) and M_rm of eq (3-38): together the sensible enthalpy the species bring
        // from the parcels' temperature, so the temperature form needs no further mass-source
        // term
        const double Mr = -(nasa_H(0, T) * dp[ORC_DEP_SH2] + nasa_H(1, T) * dp[ORC_DEP_SH2O]);
        const double Mrm = -dp[ORC_DEP_QRM];
        const double mc = m * cp[c];
        nc_[ORC_G_T] = (mc * T / dt + cT + dT + dp[ORC_DEP_HAT] + Mr + Mrm) / (mc / dt + dp[ORC_DEP_HA]);
        const double Y2 = gc[ORC_G_Y + 2];
        const double DY0 = (nc_[ORC_G_Y] - Y0) / dt - cY0 / m, DY1 = (nc_[ORC_G_Y + 1] - Y1) / dt - cY1 / m;
        const double DY2 = (nc_[ORC_G_Y + 2] - Y2) / dt + (cY0 + cY1) / m;   // N2 carried in: -(cY0 + cY1)
        const double DT = (nc_[ORC_G_T] - T) / dt - cT / mc;
        const double Dlnrho = -G.Mg * (DY0 / kMj[0] + DY1 / kMj[1] + DY2 / kMj[2]) - DT / T;
        // M of eq (3-25) as the species update takes it (the H2 sink semi-implicit, eq (4-9))
        divg[c] = -(eps[c] - epso[c]) / dt + Mnet / (V * rho[c]) - eps[c] * Dlnrho;
      }
  // 2. momentum predictor on every face (eq (4-2)), with the old state's properties
  std::vector<double> Us[3] = {U, Vv, W};
  auto fval = [&](int a, int i, int j, int kk) -> double {
    // a face value seen from a neighbouring face: open, inlet and outlet faces carry theirs;
    // NaN for walls and faces off the grid (the caller applies the wall condition)
    const int nmax[3] = {nx + (a == 0), ny + (a == 1), nz + (a == 2)};
    if (i < 0 || j < 0 || kk < 0 || i >= nmax[0] || j >= nmax[1] || kk >= nmax[2]) return std::nan("");
    const int kd = face_kind(g, a, i, j, kk);
    return kd == 0 ? std::nan("") : comp(a)[fidx(a, i, j, kk)];
  };
  for (int a = 0; a < 3; ++a) {
    const int di = a == 0, dj = a == 1, dk = a == 2;
    for (int kk = 0; kk < nz + dk; ++kk)
      for (int j = 0; j < ny + dj; ++j)
        for (int i = 0; i < nx + di; ++i) {
          const int kd = face_kind(g, a, i, j, kk);
          const int64_t f = fidx(a, i, j, kk);
          if (kd == 0) { Us[a][f] = 0.0; continue; }
          if (kd == 2) { Us[a][f] = Uin / eps[g.cidx(i, j, kk)]; continue; }
          if (kd == 3) continue;   // outlet: after the interior faces (zero gradient)
          const int64_t cP = g.cidx(i - di, j - dj, kk - dk), cN = g.cidx(i, j, kk);
          const double ef = 0.5 * (eps[cP] + eps[cN]), rf = 0.5 * (rho[cP] + rho[cN]);
          const double mf = 0.5 * (mu[cP] + mu[cN]), Kf = 0.5 * (Kc[cP] + Kc[cN]);
          const double Kvf = 0.5 * (Kv[3 * cP + a] + Kv[3 * cN + a]);
          const double u0 = comp(a)[f];
          // the velocity at the face: its own component, the others from the four faces around
          double Uf[3];
          for (int bb = 0; bb < 3; ++bb) {
            if (bb == a) { Uf[bb] = u0; continue; }
            const int ei = bb == 0, ej = bb == 1, ek = bb == 2;
            // the bb-faces of cells P and N, low and high side
            double sum = 0.0;
            sum += comp(bb)[fidx(bb, i - di, j - dj, kk - dk)] + comp(bb)[fidx(bb, i - di + ei, j - dj + ej, kk - dk + ek)];
            sum += comp(bb)[fidx(bb, i, j, kk)] + comp(bb)[fidx(bb, i + ei, j + ej, kk + ek)];
            Uf[bb] = 0.25 * sum;
          }
          double conv = 0.0, visc = 0.0;
          for (int bb = 0; bb < 3; ++bb) {
            const int ei = bb == 0, ej = bb == 1, ek = bb == 2;
            double lo = fval(a, i - ei, j - ej, kk - ek), hi = fval(a, i + ei, j + ej, kk + ek);
            if (bb != a) {   // tangential neighbours: no-slip walls halfway between
              if (std::isnan(lo)) lo = -u0;
              if (std::isnan(hi)) hi = -u0;
            } else {         // normal neighbours: walls at rest
              if (std::isnan(lo)) lo = 0.0;
              if (std::isnan(hi)) hi = 0.0;
            }
            conv += Uf[bb] > 0.0 ? Uf[bb] * (u0 - lo) / h[bb] : Uf[bb] * (hi - u0) / h[bb];
            visc += (hi - 2.0 * u0 + lo) / (h[bb] * h[bb]);
          }
          const double ptrs = -(eps[cN] * rho[cN] * RT[3 * cN + a] - eps[cP] * rho[cP] * RT[3 * cP + a]) / h[a];
          const double rhs = ef * rf * u0 / dt - ef * rf * conv + ef * mf * visc + ptrs +
                             (a == 2 ? ef * rf * grav : 0.0) - ef * (P[cN] - P[cP]) / h[a] + Kvf;
          Us[a][f] = rhs / (ef * rf / dt + Kf);
        }
  }
  for (int j = 0; j < ny; ++j)   // outlet faces: the face below
    for (int i = 0; i < nx; ++i)
      if (face_kind(g, 2, i, j, nz) == 3) Us[2][g.zf(i, j, nz)] = Us[2][g.zf(i, j, nz - 1)];
  // 3. pressure correction (incremental projection): for each fluid cell
  //    sum_f c_f (p''_nb - p''_P) = sum_f s_f eps_f u*_f A_f - V div(eps u)
  //    c_f = eps_f beta_f A_f / h, beta_f = eps_f / (eps_f rho_f / dt + K_f) from eq (4-2)
  auto vflux = [&](int a, int i, int j, int kk, int kd, double u) -> double {   // eps u A of a face
    const int di = a == 0, dj = a == 1, dk = a == 2;
    if (kd == 0) return 0.0;
    if (kd == 2) return Uin * Af[a];
    const int64_t cP = g.cidx(i - di, j - dj, kk - dk);
    if (kd == 3) return eps[cP] * u * Af[a];
    return 0.5 * (eps[cP] + eps[g.cidx(i, j, kk)]) * u * Af[a];
  };
  auto face_c = [&](int a, int i, int j, int kk, int kd) -> double {   // c_f of an open or outlet face
    const int di = a == 0, dj = a == 1, dk = a == 2;
    const int64_t cP = g.cidx(i - di, j - dj, kk - dk);
    if (kd == 3) {
      const double beta = eps[cP] / (eps[cP] * rho[cP] / dt + Kc[cP]);
      return 2.0 * eps[cP] * beta * Af[a] / h[a];
    }
    const int64_t cN = g.cidx(i, j, kk);
    const double ef = 0.5 * (eps[cP] + eps[cN]), rf = 0.5 * (rho[cP] + rho[cN]), Kf = 0.5 * (Kc[cP] + Kc[cN]);
    const double beta = ef / (ef * rf / dt + Kf);
    return ef * beta * Af[a] / h[a];
  };
  std::vector<double> rhs(nc, 0.0), diagA(nc, 0.0);
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if (!g.fluid(i, j, kk)) continue;
        const int64_t c = g.cidx(i, j, kk);
        double net = 0.0, dsum = 0.0;
        for (int a = 0; a < 3; ++a) {
          const int di = a == 0, dj = a == 1, dk = a == 2;
          const int kl = face_kind(g, a, i, j, kk), kh = face_kind(g, a, i + di, j + dj, kk + dk);
          net += vflux(a, i + di, j + dj, kk + dk, kh, Us[a][fidx(a, i + di, j + dj, kk + dk)]) -
                 vflux(a, i, j, kk, kl, Us[a][fidx(a, i, j, kk)]);
          if (kl == 1) dsum += face_c(a, i, j, kk, kl);
          if (kh == 1 || kh == 3) dsum += face_c(a, i + di, j + dj, kk + dk, kh);
        }
        rhs[c] = net - V * divg[c];
        diagA[c] = dsum;
      }
  // apply L p = sum_f c_f (p_nb - p_P) (outlet neighbours at 0)
  auto applyL = [&](const std::vector<double> &x, std::vector<double> &y) {
    for (int kk = 0; kk < nz; ++kk)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const int64_t c = g.cidx(i, j, kk);
          if (!g.fluid(i, j, kk)) { y[c] = 0.0; continue; }
          double acc = 0.0;
          for (int a = 0; a < 3; ++a) {
            const int di = a == 0, dj = a == 1, dk = a == 2;
            const int kl = face_kind(g, a, i, j, kk), kh = face_kind(g, a, i + di, j + dj, kk + dk);
            if (kl == 1) acc += face_c(a, i, j, kk, kl) * (x[g.cidx(i - di, j - dj, kk - dk)] - x[c]);
            if (kh == 1) acc += face_c(a, i + di, j + dj, kk + dk, kh) * (x[g.cidx(i + di, j + dj, kk + dk)] - x[c]);
            if (kh == 3) acc += face_c(a, i + di, j + dj, kk + dk, kh) * (0.0 - x[c]);
          }
          y[c] = acc;
        }
  };
  // conjugate gradients on -L p'' = -rhs (Jacobi preconditioner), to a relative residual 1e-12
  std::vector<double> x(nc, 0.0), r(nc), z(nc), pp(nc), Ap(nc);
  double bnorm = 0.0;
  for (int64_t c = 0; c < nc; ++c) { r[c] = -rhs[c]; bnorm += r[c] * r[c]; }
  bnorm = std::sqrt(bnorm);
  if (bnorm > 0.0) {
    for (int64_t c = 0; c < nc; ++c) { z[c] = diagA[c] > 0.0 ? r[c] / diagA[c] : 0.0; pp[c] = z[c]; }
    double rz = 0.0;
    for (int64_t c = 0; c < nc; ++c) rz += r[c] * z[c];
    for (int it = 0; it < 20000; ++it) {
      applyL(pp, Ap);
      double pAp = 0.0;
      for (int64_t c = 0; c < nc; ++c) { Ap[c] = -Ap[c]; pAp += pp[c] * Ap[c]; }
      if (!(pAp > 0.0)) break;
      const double al = rz / pAp;
      double rn = 0.0;
      for (int64_t c = 0; c < nc; ++c) { x[c] += al * pp[c]; r[c] -= al * Ap[c]; rn += r[c] * r[c]; }
      if (std::sqrt(rn) < 1e-12 * bnorm) break;
      double rzn = 0.0;
      for (int64_t c = 0; c < nc; ++c) { z[c] = diagA[c] > 0.0 ? r[c] / diagA[c] : 0.0; rzn += r[c] * z[c]; }
      const double be = rzn / rz;
      rz = rzn;
      for (int64_t c = 0; c < nc; ++c) pp[c] = z[c] + be * pp[c];
    }
  }
  // correct the face velocities and the pressure
  for (int a = 0; a < 3; ++a) {
    const int di = a == 0, dj = a == 1, dk = a == 2;
    for (int kk = 0; kk < nz + dk; ++kk)
      for (int j = 0; j < ny + dj; ++j)
        for (int i = 0; i < nx + di; ++i) {
          const int kd = face_kind(g, a, i, j, kk);
          if (kd != 1 && kd != 3) continue;
          const int64_t f = fidx(a, i, j, kk), cP = g.cidx(i - di, j - dj, kk - dk);
          if (kd == 3) {
            const double beta = eps[cP] / (eps[cP] * rho[cP] / dt + Kc[cP]);
            Us[a][f] -= beta * (0.0 - x[cP]) / (0.5 * h[a]);
          } else {
            const int64_t cN = g.cidx(i, j, kk);
            const double ef = 0.5 * (eps[cP] + eps[cN]), rf = 0.5 * (rho[cP] + rho[cN]), Kf = 0.5 * (Kc[cP] + Kc[cN]);
            Us[a][f] -= ef / (ef * rf / dt + Kf) * (x[cN] - x[cP]) / h[a];
          }
        }
  }
  for (int64_t c = 0; c < nc; ++c) P[c] += x[c];
  U = Us[0]; Vv = Us[1]; W = Us[2];
  for (int64_t c = 0; c < nc; ++c) nxt[c * ORC_NG + ORC_G_EPS] = eps[c];
  std::copy(nxt.begin(), nxt.end(), o.gas.begin() + off * ORC_NG);
}

// initial gas flow of a solved bed: plug flow at the superficial velocity through every fluid
// column (eps w = U_in on the z-faces that carry gas), no cross flow, p = p0
void gas_flow_init(Oracle &o, int b) {
  const double *bd = o.B(b);
  const Grid gg = make_grid(bd);
  FlowGrid g{gg.nx, gg.ny, gg.nz, gg.dx, gg.dy, gg.dz, o.cell_off[b], o.gas.data()};
  o.fu[b].assign((size_t)(g.nx + 1) * g.ny * g.nz, 0.0);
  o.fv[b].assign((size_t)g.nx * (g.ny + 1) * g.nz, 0.0);
  o.fw[b].assign((size_t)g.nx * g.ny * (g.nz + 1), 0.0);
  o.pr[b].assign((size_t)g.nx * g.ny * g.nz, 0.0);
  for (int k = 0; k <= g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const int kd = face_kind(g, 2, i, j, k);
        if (kd == 0) continue;
        const int kc = kd == 3 ? k - 1 : k;
        o.fw[b][g.zf(i, j, k)] = bd[ORC_B_U_IN] / o.gas[(g.off + g.cidx(i, j, kc)) * ORC_NG + ORC_G_EPS];
      }
}


template <class S> S fov_of(const S m[4], int ore) {   // eqs (2-15)..(2-19)
  S n[4];
  for (int z = 0; z < 4; ++z) n[z] = m[z] / kMz[z];
  S nfe = 2.0 * n[0] + 3.0 * n[1] + n[2] + n[3];
  if (!(val(nfe) > 0.0)) return S(0.0);
  S fh = (3.0 * n[1] + n[2] + n[3]) / nfe, fm = (n[2] + n[3]) / nfe, fw = n[3] / nfe;
  if (ore == 0) return fh / 9.0 + 2.0 * fm / 9.0 + 6.0 * fw / 9.0;
  return fm / 4.0 + 3.0 * fw / 4.0;
}

// One full step of every bed (Sec. 3, Sec. 4; order: half kick and drift, contacts,
// gas-particle terms and kinetics, second half kick with T and mass update, deposition,
// gas update).
void step_once(Oracle &o) {
  const int n = o.n;
  // gas properties of every cell at the start of the step (frozen during the step)
  std::vector<GasProps> gp(o.ncell_total);
  for (int b = 0; b < o.nb; ++b) {
    const double *bd = o.B(b);
    Grid g = make_grid(bd);
    int64_t nc = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t c = 0; c < nc; ++c) {
      const double *gc = &o.gas[(o.cell_off[b] + c) * ORC_NG];
      gp[o.cell_off[b] + c] = gas_props(gc[ORC_G_T], gc + ORC_G_Y, bd[ORC_B_P0]);
    }
  }
  // cell-centre gas velocity of the beds whose gas is solved (the mean of the two faces)
  std::vector<double> ucell(3 * (size_t)o.ncell_total, 0.0);
  for (int b = 0; b < o.nb; ++b) {
    const double *bd = o.B(b);
    if (!((unsigned)ib(bd, ORC_B_FLAGS) & ORC_GAS_SOLVER)) continue;
    Grid gg = make_grid(bd);
    FlowGrid g{gg.nx, gg.ny, gg.nz, gg.dx, gg.dy, gg.dz, o.cell_off[b], o.gas.data()};
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          const int64_t c = o.cell_off[b] + g.cidx(i, j, k);
          ucell[3 * c] = 0.5 * (o.fu[b][g.xf(i, j, k)] + o.fu[b][g.xf(i + 1, j, k)]);
          ucell[3 * c + 1] = 0.5 * (o.fv[b][g.yf(i, j, k)] + o.fv[b][g.yf(i, j + 1, k)]);
          ucell[3 * c + 2] = 0.5 * (o.fw[b][g.zf(i, j, k)] + o.fw[b][g.zf(i, j, k + 1)]);
        }
  }
  // 1. half kick and drift (velocity Verlet, kick-drift-kick)
  for (int i = 0; i < n; ++i) {
    double dt = o.B(o.bed[i])[ORC_B_DT];
    for (int c = 0; c < 3; ++c) {
      o.s[ORC_S_VX + c][i] = o.s[ORC_S_VX + c][i] + o.s[ORC_S_AX + c][i] * (0.5 * dt);
      o.s[ORC_S_WX + c][i] = o.s[ORC_S_WX + c][i] + o.s[ORC_S_ALX + c][i] * (0.5 * dt);
      o.s[ORC_S_X + c][i] = o.s[ORC_S_X + c][i] + o.s[ORC_S_VX + c][i] * dt;
    }
  }
  std::fill(o.diag.begin(), o.diag.end(), 0.0);
  std::vector<char> coupled(o.nb);
  for (int b = 0; b < o.nb; ++b) {
    int nc = std::max(1, ib(o.B(b), ORC_B_NCOUPLE));
    coupled[b] = ((o.step_no + 1) % nc) == 0;
  }
  // 2. contacts, per bed (and the contact conduction of beds that switch it on)
  std::vector<double> Fc(3 * (size_t)n, 0.0), Tc(3 * (size_t)n, 0.0), Qcond(n, 0.0);
  std::vector<double> lamg(n, 0.0);   // gas conductivity of each parcel's cell (after the drift)
  for (int i = 0; i < n; ++i) {
    Grid g = make_grid(o.B(o.bed[i]));
    lamg[i] = gp[o.cell_off[o.bed[i]] + cell_of(g, o.s[0][i], o.s[1][i], o.s[2][i], nullptr)].lam;
  }
  for (int b = 0; b < o.nb; ++b) {
    const double *bd = o.B(b);
    const auto &ids = o.members[b];
    if ((unsigned)ib(bd, ORC_B_FLAGS) & ORC_NO_CONTACTS) {
      for (int32_t i : ids) o.hist[i].clear();
      continue;
    }
    const double k = bd[ORC_B_CG];
    const bool cond = ((unsigned)ib(bd, ORC_B_FLAGS) & ORC_CONDUCTION) != 0;
    double hmax = 0.0;
    for (int32_t i : ids) hmax = std::max(hmax, k * o.dreal[i]);
    CellList cl;
    cl.build(ids, o.s[0].data(), o.s[1].data(), o.s[2].data(), std::max(hmax, 1e-12));
    const double *X = o.s[0].data(), *Y = o.s[1].data(), *Z = o.s[2].data();
#pragma omp parallel for schedule(dynamic, 256)
    for (size_t t = 0; t < ids.size(); ++t) {
      int32_t i = ids[t];
      double ri = 0.5 * (k * o.dreal[i]);
      double mi = parcel_mass(o, i);
      struct Cand { int32_t id; double n[3]; double delta; double dist; double mstar; double vrel[3]; };
      std::vector<Cand> cands;
      cl.neighbours(X[i], Y[i], Z[i], [&](int32_t j) {
        if (j == i) return;
        double rj = 0.5 * (k * o.dreal[j]);
        double rs = ri + rj;
        if (!touching(X[i], Y[i], Z[i], X[j], Y[j], Z[j], rs)) return;
        double dx = X[j] - X[i], dy = Y[j] - Y[i], dz = Z[j] - Z[i];
        double d = std::sqrt((dx * dx + dy * dy) + dz * dz);
        Cand c;
        c.id = j;
        c.n[0] = dx / d; c.n[1] = dy / d; c.n[2] = dz / d;
        c.delta = rs - d;
        c.dist = d;
        double mj = parcel_mass(o, j);
        c.mstar = mi * mj / (mi + mj);
        double wsum[3];
        for (int q = 0; q < 3; ++q) wsum[q] = ri * o.s[ORC_S_WX + q][i] + rj * o.s[ORC_S_WX + q][j];
        double cr[3] = {wsum[1] * c.n[2] - wsum[2] * c.n[1], wsum[2] * c.n[0] - wsum[0] * c.n[2],
                        wsum[0] * c.n[1] - wsum[1] * c.n[0]};
        for (int q = 0; q < 3; ++q) c.vrel[q] = (o.s[ORC_S_VX + q][i] - o.s[ORC_S_VX + q][j]) + cr[q];
        cands.push_back(c);
      });
      double dist[4], nw[4][3];
      wall_distance(bd, X[i], Y[i], Z[i], dist, nw);
      for (int p = 0; p < 4; ++p) {
        if (!(dist[p] < ri)) continue;
        Cand c;
        c.id = -1 - p;
        for (int q = 0; q < 3; ++q) c.n[q] = -nw[p][q];
        c.delta = ri - dist[p];
        c.dist = dist[p];
        c.mstar = mi;
        double w[3] = {ri * o.s[ORC_S_WX][i], ri * o.s[ORC_S_WY][i], ri * o.s[ORC_S_WZ][i]};
        double cr[3] = {w[1] * c.n[2] - w[2] * c.n[1], w[2] * c.n[0] - w[0] * c.n[2], w[0] * c.n[1] - w[1] * c.n[0]};
        for (int q = 0; q < 3; ++q) c.vrel[q] = o.s[ORC_S_VX + q][i] + cr[q];
        cands.push_back(c);
      }
      std::sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b2) { return a.id < b2.id; });
      std::vector<Contact> nh;
      double w[3] = {o.s[ORC_S_WX][i], o.s[ORC_S_WY][i], o.s[ORC_S_WZ][i]};
      for (const Cand &c : cands) {
        double xo[3] = {0, 0, 0};
        for (const Contact &h : o.hist[i])
          if (h.partner == c.id) { xo[0] = h.xi[0]; xo[1] = h.xi[1]; xo[2] = h.xi[2]; break; }
        ContactOut co;
        contact_law(bd, c.mstar, ri, c.n, c.delta, c.vrel, xo, w, co);
        for (int q = 0; q < 3; ++q) { Fc[3 * (size_t)i + q] += co.F[q]; Tc[3 * (size_t)i + q] += co.Tq[q]; }
        if ((int)nh.size() < ORC_MAX_CONTACTS) nh.push_back(Contact{c.id, {co.xi[0], co.xi[1], co.xi[2]}});
        if (cond) {
          double q4[4];
          const double lam_a = bd[ORC_B_LAMP + o.ore[i]];
          if (c.id >= 0) {
            const int32_t j = c.id;
            const double rj = 0.5 * (k * o.dreal[j]);
            conduction_pair(bd, ri, rj, c.dist, o.s[ORC_S_T][i], o.s[ORC_S_T][j], lam_a,
                            bd[ORC_B_LAMP + o.ore[j]], 0.5 * (lamg[i] + lamg[j]), q4);
          } else {
            conduction_wall(bd, ri, c.dist, o.s[ORC_S_T][i], lam_a, lamg[i], q4);
          }
          Qcond[i] += q4[0] + q4[1];
        }
      }
      o.hist[i] = nh;
      o.diag[(size_t)ORC_D_NCONTACT * n + i] = (double)cands.size();
    }
  }
  // 2b. particle radiation, eqs (3-16), (3-17), (3-51), in beds that switch it on. T_se is
  // the mean temperature over a sphere of radius 1.5 d around the parcel, with these
  // readings: d is the parcel's own diameter k d_p (the neighbourhood is one of parcels);
  // the parcel itself is one of the n_p,Omega parcels averaged (so n >= 1); a parcel is in
  // the sphere when its centre is (d^2 < R^2, the pair test's expression); eps_g and T_g are
  // those of the parcel's gas cell (eps_g lagged as in the drag); the temperatures are the
  // ones before this step's update. The area is that of the real particle, pi d_p^2 (as in
  // the convective heat), and k^3 scales it to the parcel (eq 3-51).
  std::vector<double> Qrad(n, 0.0), Tse(n, 0.0);
  for (int b = 0; b < o.nb; ++b) {
    const double *bd = o.B(b);
    if (!((unsigned)ib(bd, ORC_B_FLAGS) & ORC_RADIATION)) continue;
    const auto &ids = o.members[b];
    const double k = bd[ORC_B_CG];
    double Rmax = 0.0;
    for (int32_t i : ids) Rmax = std::max(Rmax, 1.5 * (k * o.dreal[i]));
    const double *X = o.s[0].data(), *Y = o.s[1].data(), *Z = o.s[2].data();
    const double *Tp = o.s[ORC_S_T].data();
    CellList cl;   // cells of edge R_max: every centre within R lies in the 27 cells around
    cl.build(ids, X, Y, Z, std::max(Rmax, 1e-12));
    Grid g = make_grid(bd);
#pragma omp parallel for schedule(dynamic, 256)
    for (size_t t = 0; t < ids.size(); ++t) {
      int32_t i = ids[t];
      const double R = 1.5 * (k * o.dreal[i]);
      double sumT = 0.0;
      int64_t cnt = 0;
      cl.neighbours(X[i], Y[i], Z[i], [&](int32_t j) {
        if (!touching(X[i], Y[i], Z[i], X[j], Y[j], Z[j], R)) return;
        sumT += Tp[j];
        ++cnt;
      });
      bool outside = false;
      int64_t c = o.cell_off[b] + cell_of(g, X[i], Y[i], Z[i], &outside);
      const double eps = o.gas[c * ORC_NG + ORC_G_EPS];
      const double Ts = eps * gp[c].T + (1.0 - eps) * (sumT / (double)cnt);   // eq (3-17)
      const double dp = o.dreal[i];
      const double Qp = kSigma * bd[ORC_B_EMISS] * (kPi * dp * dp) *
                        (Ts * Ts * Ts * Ts - Tp[i] * Tp[i] * Tp[i] * Tp[i]);   // eq (3-16)
      Qrad[i] = k * k * k * Qp;                                                 // eq (3-51)
      Tse[i] = Ts;
    }
  }
  // 3. gas-particle terms, kinetics, second half kick, temperature and mass update
  std::vector<double> pdep((size_t)n * ORC_NDEP, 0.0);
  std::vector<int64_t> pcell(n, -1);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    int b = o.bed[i];
    const double *bd = o.B(b);
    const unsigned flags = (unsigned)ib(bd, ORC_B_FLAGS);
    Grid g = make_grid(bd);
    const double dt = bd[ORC_B_DT];
    const int ncpl = std::max(1, ib(bd, ORC_B_NCOUPLE));
    const double dtm = ncpl * dt;
    const double k = bd[ORC_B_CG];
    const double k3 = k * k * k;
    const double dc = k * o.dreal[i];
    const double r = 0.5 * dc;
    const double V = kPi / 6.0 * dc * dc * dc;
    bool outside = false;
    int64_t lc = cell_of(g, o.s[0][i], o.s[1][i], o.s[2][i], &outside);
    int64_t c = o.cell_off[b] + lc;
    pcell[i] = c;
    const double *gc = &o.gas[c * ORC_NG];
    const GasProps &G = gp[c];
    double eps = gc[ORC_G_EPS];
    double ug[3] = {0.0, 0.0, bd[ORC_B_U_IN] / eps};
    if (flags & ORC_GAS_SOLVER)
      for (int q = 0; q < 3; ++q) ug[q] = ucell[3 * c + q];   // the solved gas, cell centre
    double sv[3] = {ug[0] - o.s[ORC_S_VX][i], ug[1] - o.s[ORC_S_VY][i], ug[2] - o.s[ORC_S_VZ][i]};
    double slip = std::sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
    double Re = 0.0;
    double bo = drag_beta_over_epsp(bd, o.dreal[i], o.ore[i], eps, slip, G, &Re);
    double Kp = (flags & ORC_NO_DRAG) ? 0.0 : bo * V;        // beta V/(1-eps), eq (3-27a)
    double Fd[3] = {Kp * sv[0], Kp * sv[1], Kp * sv[2]};     // eq (3-5)
    double Fp[3] = {0.0, 0.0, -V * bd[ORC_B_DPDZ]};          // -V grad p, eq (3-3)
    // convective heat, eqs (3-10)..(3-13), (3-41)
    double Pr = G.cp * G.mu / G.lam;
    double Nu = gunn(eps, Re, Pr);
    double hcoef = Nu * G.lam / o.dreal[i];
    double hA = (flags & ORC_NO_HEAT) ? 0.0 : k3 * hcoef * kPi * o.dreal[i] * o.dreal[i];
    double Tp = o.s[ORC_S_T][i];
    double Qconv = hA * (G.T - Tp);
    double m[4] = {o.s[ORC_S_M][i], o.s[ORC_S_M + 1][i], o.s[ORC_S_M + 2][i], o.s[ORC_S_M + 3][i]};
    const double *k0 = bd + ORC_B_K0;
    const double *Ea = bd + ORC_B_EA;
    Kin<double> kn;
    kinetics(bd, m, Tp, o.dreal[i], o.ore[i], G, eps, slip, dtm, k0, Ea, kn);
    double mp = m[0] + m[1] + m[2] + m[3];
    double I = 0.4 * mp * r * r;                              // eq (3-7)
    double gz = (flags & ORC_NO_GRAVITY) ? 0.0 : -kG;
    double a[3], al[3];
    for (int q = 0; q < 3; ++q) {
      a[q] = (Fc[3 * (size_t)i + q] + Fd[q] + Fp[q]) / mp;    // eq (3-3)
      al[q] = Tc[3 * (size_t)i + q] / I;                      // eq (3-6)
    }
    a[2] += gz;
    for (int q = 0; q < 3; ++q) {
      o.s[ORC_S_VX + q][i] = o.s[ORC_S_VX + q][i] + a[q] * (0.5 * dt);
      o.s[ORC_S_WX + q][i] = o.s[ORC_S_WX + q][i] + al[q] * (0.5 * dt);
      o.s[ORC_S_AX + q][i] = a[q];
      o.s[ORC_S_ALX + q][i] = al[q];
    }
    // particle energy, eqs (3-8), (3-9); reading: d(m C_p)/dt T is not carried
    double cpp = 0.0;
    for (int z = 0; z < 4; ++z) cpp += (m[z] / mp) * nasa_cp(3 + z, Tp);
    double Qrx = kn.Qr + kn.Qrm;
    o.s[ORC_S_T][i] = Tp + dt * (Qconv + Qrx + Qrad[i] + Qcond[i]) / (mp * cpp);
    // eq (3-4): layer masses change only at coupling steps (Sec. 4)
    if (coupled[b])
      for (int z = 0; z < 4; ++z) o.s[ORC_S_M + z][i] = std::max(m[z] + kn.mdot[z] * dtm, 0.0);
    // per-parcel contributions to the cell sums (Sec. 3.2, Sec. 4.1, Sec. 4.2)
    double *pd = &pdep[(size_t)i * ORC_NDEP];
    pd[ORC_DEP_VS] = V;
    pd[ORC_DEP_SH2] = kn.sH2;
    pd[ORC_DEP_SH2O] = kn.sH2O;
    pd[ORC_DEP_K] = Kp;
    pd[ORC_DEP_HA] = hA;
    pd[ORC_DEP_HAT] = hA * Tp;
    pd[ORC_DEP_QRM] = kn.Qrm;
    pd[ORC_DEP_QR] = kn.Qr;
    pd[ORC_DEP_EQ] = kn.EQ;
    pd[ORC_DEP_ES] = kn.ES;
    pd[ORC_DEP_COUNT] = 1.0;
    // half-step velocity used in the drag (deposited with K)
    for (int q = 0; q < 3; ++q) pd[ORC_DEP_KV + q] = Kp * (ug[q] - sv[q]);
    // diagnostics
    double *dg = o.diag.data();
    for (int q = 0; q < 3; ++q) {
      dg[(size_t)(ORC_D_FC + q) * n + i] = Fc[3 * (size_t)i + q];
      dg[(size_t)(ORC_D_TC + q) * n + i] = Tc[3 * (size_t)i + q];
      dg[(size_t)(ORC_D_FD + q) * n + i] = Fd[q];
      dg[(size_t)(ORC_D_XIDOT + q) * n + i] = kn.xidot[q];
      dg[(size_t)(ORC_D_A + q) * n + i] = kn.A[q];
      dg[(size_t)(ORC_D_B + q) * n + i] = kn.B[q];
    }
    for (int z = 0; z < 4; ++z) dg[(size_t)(ORC_D_MDOT + z) * n + i] = kn.mdot[z];
    dg[(size_t)ORC_D_K * n + i] = Kp;
    dg[(size_t)ORC_D_QCONV * n + i] = Qconv;
    dg[(size_t)ORC_D_QR * n + i] = kn.Qr;
    dg[(size_t)ORC_D_QRM * n + i] = kn.Qrm;
    dg[(size_t)ORC_D_FFILM * n + i] = kn.F;
    dg[(size_t)ORC_D_SH * n + i] = kn.Sh;
    dg[(size_t)ORC_D_NU * n + i] = Nu;
    dg[(size_t)ORC_D_RE * n + i] = Re;
    dg[(size_t)ORC_D_CELL * n + i] = (double)lc;
    dg[(size_t)ORC_D_TSE * n + i] = Tse[i];
    dg[(size_t)ORC_D_QRAD * n + i] = Qrad[i];
    dg[(size_t)ORC_D_QCOND * n + i] = Qcond[i];
  }
  // 4. deposition: per-cell sums in parcel order (eqs (3-25), (3-27a), (3-38), (3-39),
  //    (4-4), (4-5), (4-10), (4-11)); only at coupling steps
  std::fill(o.dep.begin(), o.dep.end(), 0.0);
  for (int i = 0; i < n; ++i) {
    if (!coupled[o.bed[i]]) continue;
    int64_t c = pcell[i];
    if (o.gas[c * ORC_NG + ORC_G_MARK] != 0.0) continue;   // solid cells take no sources
    for (int f = 0; f < ORC_NDEP; ++f) o.dep[c * ORC_NDEP + f] += pdep[(size_t)i * ORC_NDEP + f];
  }
  // 5. gas update: the gas phase solver of beds that switch it on, else the prescribed field
  //    with its simple explicit update
  for (int b = 0; b < o.nb; ++b) {
    const double *bd = o.B(b);
    if (!coupled[b] || ((unsigned)ib(bd, ORC_B_FLAGS) & ORC_NO_GAS_UPDATE)) continue;
    if ((unsigned)ib(bd, ORC_B_FLAGS) & ORC_GAS_SOLVER) {
      gas_solve(o, b, gp, std::max(1, ib(bd, ORC_B_NCOUPLE)) * bd[ORC_B_DT]);
      continue;
    }
    Grid g = make_grid(bd);
    const double dtg = std::max(1, ib(bd, ORC_B_NCOUPLE)) * bd[ORC_B_DT];
    const double V = g.dx * g.dy * g.dz;
    const int64_t nc = (int64_t)g.nx * g.ny * g.nz;
    const int64_t off = o.cell_off[b];
    std::vector<double> nxt(o.gas.begin() + off * ORC_NG, o.gas.begin() + (off + nc) * ORC_NG);
    for (int64_t c = 0; c < nc; ++c) {
      const double *gc = &o.gas[(off + c) * ORC_NG];
      if (gc[ORC_G_MARK] != 0.0) continue;
      const double *dp = &o.dep[(off + c) * ORC_NDEP];
      const GasProps &G = gp[off + c];
      double eps = gc[ORC_G_EPS];
      double uz = bd[ORC_B_U_IN] / eps;
      // upwind neighbour: the cell below, or the inlet state for the lowest fluid cell
      double Yup[3] = {bd[ORC_B_Y_IN], bd[ORC_B_Y_IN + 1], bd[ORC_B_Y_IN + 2]};
      double Tup = bd[ORC_B_T_IN];
      if (c >= (int64_t)g.nx * g.ny) {
        const double *gb = &o.gas[(off + c - (int64_t)g.nx * g.ny) * ORC_NG];
        if (gb[ORC_G_MARK] == 0.0) {
          for (int j = 0; j < 3; ++j) Yup[j] = gb[ORC_G_Y + j];
          Tup = gb[ORC_G_T];
        }
      }
      double S[3] = {dp[ORC_DEP_SH2], dp[ORC_DEP_SH2O], 0.0};
      double Snet = S[0] + S[1] + S[2];
      double mg = eps * G.rho * V;   // gas mass in the cell
      double Y[3], ysum = 0.0;
      for (int j = 0; j < 3; ++j) {
        double y = gc[ORC_G_Y + j];
        y = y + dtg * (-uz * (y - Yup[j]) / g.dz + (S[j] - y * Snet) / mg);
        Y[j] = std::max(y, 0.0);
        ysum += Y[j];
      }
      for (int j = 0; j < 3; ++j) nxt[c * ORC_NG + ORC_G_Y + j] = ysum > 0.0 ? Y[j] / ysum : gc[ORC_G_Y + j];
      // energy, semi-implicit in H0 as in eq (4-6)
      double cap = eps * G.rho * G.cp;
      double H0 = dp[ORC_DEP_HA] / V, H1 = dp[ORC_DEP_HAT] / V;
      double Mrm = -dp[ORC_DEP_QRM] / V;                                    // eq (3-38)
      double Mr = -(nasa_H(0, G.T) * S[0] + nasa_H(1, G.T) * S[1]) / V;    // eq (3-39)
      double T = gc[ORC_G_T];
      double rhs = T + dtg * (-uz * (T - Tup) / g.dz + (H1 + Mr + Mrm) / cap);
      nxt[c * ORC_NG + ORC_G_T] = rhs / (1.0 + dtg * H0 / cap);
      nxt[c * ORC_NG + ORC_G_EPS] = std::max(1.0 - dp[ORC_DEP_VS] / V, bd[ORC_B_EPS_MIN]);
    }
    std::copy(nxt.begin(), nxt.end(), o.gas.begin() + off * ORC_NG);
  }
  o.step_no++;
}

// Frozen-position drag-heat-reaction sub-step used by the adjoint (positions, cells and
// the gas field held at their current values; per-parcel state v, T_p, m_z).
// With observations (nobs > 0): returns sum_k sum_i coef[k][bed i] (f_ov,i(obs[k]) - f_ov,i(0))
// and writes the values f_ov,i(obs[k]) - f_ov,i(0) to rec[k][i]; otherwise the mean over all
// parcels of f_ov(after nsteps) - f_ov(0).
template <class S>
S adjoint_J(const Oracle &o, const std::vector<GasProps> &gp, const std::vector<int64_t> &pcell,
            int nsteps, const S k0s[3], const S Eas[3], int nobs = 0, const int *obs = nullptr,
            const double *coef = nullptr, double *rec = nullptr) {
  S total(0.0);
  const int n = o.n;
  std::vector<S> part(n);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    const double *bd = o.B(o.bed[i]);
    const unsigned flags = (unsigned)ib(bd, ORC_B_FLAGS);
    const double dt = bd[ORC_B_DT];
    const double k = bd[ORC_B_CG], k3 = k * k * k;
    const double d = o.dreal[i], dc = k * d, V = kPi / 6.0 * dc * dc * dc;
    const int64_t c = pcell[i];
    const GasProps &G = gp[c];
    const double eps = o.gas[c * ORC_NG + ORC_G_EPS];
    const double ug[3] = {0.0, 0.0, bd[ORC_B_U_IN] / eps};
    S v[3], T, m[4];
    for (int q = 0; q < 3; ++q) v[q] = S(o.s[ORC_S_VX + q][i]);
    T = S(o.s[ORC_S_T][i]);
    for (int z = 0; z < 4; ++z) m[z] = S(o.s[ORC_S_M + z][i]);
    S f0 = fov_of(m, o.ore[i]);
    S wsum(0.0);
    int oi = 0;
    for (int st = 0; st < nsteps; ++st) {
      S sv[3] = {ug[0] - v[0], ug[1] - v[1], ug[2] - v[2]};
      S slip = sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
      S Re(0.0);
      S bo = drag_beta_over_epsp(bd, d, o.ore[i], eps, slip, G, &Re);
      S Kp = (flags & ORC_NO_DRAG) ? S(0.0) : bo * V;
      S mp = m[0] + m[1] + m[2] + m[3];
      double Pr = G.cp * G.mu / G.lam;
      S Nu = gunn(eps, Re, Pr);
      S hA = (flags & ORC_NO_HEAT) ? S(0.0) : k3 * Nu * G.lam / d * (kPi * d * d);
      S Qconv = hA * (G.T - T);
      Kin<S> kn;
      kinetics(bd, m, T, d, o.ore[i], G, eps, slip, dt, k0s, Eas, kn);
      S cpp(0.0);
      for (int z = 0; z < 4; ++z) cpp = cpp + (m[z] / mp) * nasa_cp(3 + z, T);
      S Tn = T + dt * (Qconv + kn.Qr + kn.Qrm) / (mp * cpp);
      for (int q = 0; q < 3; ++q) v[q] = v[q] + dt * Kp * sv[q] / mp;
      for (int z = 0; z < 4; ++z) m[z] = smax(m[z] + kn.mdot[z] * dt, S(0.0));
      T = Tn;
      if (oi < nobs && st + 1 == obs[oi]) {
        const S df = fov_of(m, o.ore[i]) - f0;
        rec[(size_t)oi * n + i] = val(df);
        wsum = wsum + coef[(size_t)oi * o.nb + o.bed[i]] * df;
        ++oi;
      }
    }
    part[i] = nobs > 0 ? wsum : fov_of(m, o.ore[i]) - f0;
  }
  for (int i = 0; i < n; ++i) total = total + part[i];
  return nobs > 0 ? total : total / (double)n;
}

}  // namespace

// =========================================================================================
// C API
// =========================================================================================
extern "C" {

int32_t orc_adjoint_obs(void *h, int32_t nsteps, int32_t mode, int32_t nobs, const int32_t *obs_steps,
                        const double *weights, double *J_obs, double *grad6) {
  Oracle *o = (Oracle *)h;
  for (int b = 0; b < o->nb; ++b)
    if ((unsigned)ib(o->B(b), ORC_B_FLAGS) & (ORC_RADIATION | ORC_CONDUCTION | ORC_GAS_SOLVER)) return -1;
  std::vector<GasProps> gp(o->ncell_total);
  for (int b = 0; b < o->nb; ++b) {
    const double *bd = o->B(b);
    for (int64_t c = o->cell_off[b]; c < o->cell_off[b + 1]; ++c)
      gp[c] = gas_props(o->gas[c * ORC_NG + ORC_G_T], &o->gas[c * ORC_NG + ORC_G_Y], bd[ORC_B_P0]);
  }
  std::vector<int64_t> pcell(o->n);
  std::vector<int> cnt(o->nb, 0);
  for (int i = 0; i < o->n; ++i) {
    const double *bd = o->B(o->bed[i]);
    Grid g = make_grid(bd);
    pcell[i] = o->cell_off[o->bed[i]] + cell_of(g, o->s[0][i], o->s[1][i], o->s[2][i], nullptr);
    cnt[o->bed[i]]++;
  }
  std::vector<int> obs(obs_steps, obs_steps + nobs);
  std::vector<double> coef((size_t)nobs * o->nb, 0.0);   // weight over the bed's parcel count
  for (int k = 0; k < nobs; ++k)
    for (int b = 0; b < o->nb; ++b)
      coef[(size_t)k * o->nb + b] = weights && cnt[b] ? weights[(size_t)k * o->nb + b] / cnt[b] : 0.0;
  std::vector<double> rec((size_t)nobs * o->n, 0.0);
  double th[6];
  for (int r = 0; r < 3; ++r) { th[r] = o->B(0)[ORC_B_K0 + r]; th[3 + r] = o->B(0)[ORC_B_EA + r]; }
  if (mode == 2) {
    Dual k0s[3], Eas[3];
    for (int r = 0; r < 3; ++r) {
      k0s[r] = Dual(th[r]); k0s[r].d[r] = 1.0;
      Eas[r] = Dual(th[3 + r]); Eas[r].d[3 + r] = 1.0;
    }
    Dual Jd = adjoint_J<Dual>(*o, gp, pcell, nsteps, k0s, Eas, nobs, obs.data(), coef.data(), rec.data());
    for (int q = 0; q < 6; ++q) grad6[q] = Jd.d[q];
  } else {
    double k0s[3] = {th[0], th[1], th[2]}, Eas[3] = {th[3], th[4], th[5]};
    adjoint_J<double>(*o, gp, pcell, nsteps, k0s, Eas, nobs, obs.data(), coef.data(), rec.data());
  }
  for (int k = 0; k < nobs; ++k)
    for (int b = 0; b < o->nb; ++b) {
      double sum = 0.0;
      for (int i = 0; i < o->n; ++i)
        if (o->bed[i] == b) sum += rec[(size_t)k * o->n + i];
      J_obs[(size_t)k * o->nb + b] = cnt[b] ? sum / cnt[b] : 0.0;
    }
  return 0;
}

void orc_set_threads(int32_t nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}
int32_t orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void *orc_create(int32_t nbeds, const double *beds, int32_t n, const double *x, const double *y,
                 const double *z, const double *vx, const double *vy, const double *vz,
                 const double *d_real, const double *T, const double *m0, const int32_t *ore,
                 const int32_t *bed, const double *gasY, const double *gasT) {
  Oracle *o = new Oracle();
  o->nb = nbeds;
  o->n = n;
  o->beds.assign(beds, beds + (size_t)nbeds * ORC_NB);
  for (int f = 0; f < ORC_NS; ++f) o->s[f].assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    o->s[ORC_S_X][i] = x[i]; o->s[ORC_S_Y][i] = y[i]; o->s[ORC_S_Z][i] = z[i];
    o->s[ORC_S_VX][i] = vx[i]; o->s[ORC_S_VY][i] = vy[i]; o->s[ORC_S_VZ][i] = vz[i];
    o->s[ORC_S_T][i] = T[i];
    for (int q = 0; q < 4; ++q) o->s[ORC_S_M + q][i] = m0[(size_t)q * n + i];
    // Reading: the stored acceleration starts as gravity alone (no contact or drag force
    // is known before the first step), so the first half kick is the body force.
    const double *bd = beds + (size_t)bed[i] * ORC_NB;
    o->s[ORC_S_AZ][i] = ((unsigned)ib(bd, ORC_B_FLAGS) & ORC_NO_GRAVITY) ? 0.0 : -kG;
  }
  o->dreal.assign(d_real, d_real + n);
  o->ore.assign(ore, ore + n);
  o->bed.assign(bed, bed + n);
  o->hist.assign(n, {});
  o->diag.assign((size_t)ORC_ND * n, 0.0);
  o->members.assign(nbeds, {});
  for (int i = 0; i < n; ++i) o->members[bed[i]].push_back(i);
  o->cell_off.assign(nbeds + 1, 0);
  for (int b = 0; b < nbeds; ++b) {
    const double *bd = o->B(b);
    o->cell_off[b + 1] = o->cell_off[b] + (int64_t)ib(bd, ORC_B_NX) * ib(bd, ORC_B_NY) * ib(bd, ORC_B_NZ);
  }
  o->ncell_total = o->cell_off[nbeds];
  o->gas.assign((size_t)o->ncell_total * ORC_NG, 0.0);
  o->dep.assign((size_t)o->ncell_total * ORC_NDEP, 0.0);
  for (int b = 0; b < nbeds; ++b) {
    const double *bd = o->B(b);
    Grid g = make_grid(bd);
    double hd = 0.5 * std::sqrt(g.dx * g.dx + g.dy * g.dy + g.dz * g.dz);
    for (int iz = 0; iz < g.nz; ++iz)
      for (int iy = 0; iy < g.ny; ++iy)
        for (int ix = 0; ix < g.nx; ++ix) {
          int64_t c = o->cell_off[b] + ((int64_t)iz * g.ny + iy) * g.nx + ix;
          double *gc = &o->gas[c * ORC_NG];
          for (int j = 0; j < 3; ++j) gc[ORC_G_Y + j] = gasY ? gasY[c * 3 + j] : bd[ORC_B_Y_IN + j];
          gc[ORC_G_T] = gasT ? gasT[c] : bd[ORC_B_T_IN];
          double xc = g.x0 + (ix + 0.5) * g.dx, yc = g.y0 + (iy + 0.5) * g.dy, zc = g.z0 + (iz + 0.5) * g.dz;
          gc[ORC_G_MARK] = cell_is_solid(bd, xc, yc, zc, hd) ? 1.0 : 0.0;
        }
  }
  deposit_volume_and_eps(*o);
  o->fu.resize(nbeds); o->fv.resize(nbeds); o->fw.resize(nbeds); o->pr.resize(nbeds);
  for (int b = 0; b < nbeds; ++b)
    if ((unsigned)ib(o->B(b), ORC_B_FLAGS) & ORC_GAS_SOLVER) gas_flow_init(*o, b);
  return o;
}

int32_t orc_step(void *h, int32_t nsteps) {
  Oracle *o = (Oracle *)h;
  for (int s = 0; s < nsteps; ++s) step_once(*o);
  return 0;
}

void orc_get_state(void *h, double *out) {
  Oracle *o = (Oracle *)h;
  for (int f = 0; f < ORC_NS; ++f) std::memcpy(out + (size_t)f * o->n, o->s[f].data(), sizeof(double) * o->n);
}
void orc_get_diag(void *h, double *out) {
  Oracle *o = (Oracle *)h;
  std::memcpy(out, o->diag.data(), sizeof(double) * o->diag.size());
}
void orc_get_contacts(void *h, int32_t *count, int32_t *partner, double *xi) {
  Oracle *o = (Oracle *)h;
  for (int i = 0; i < o->n; ++i) {
    count[i] = (int32_t)o->hist[i].size();
    for (int k = 0; k < ORC_MAX_CONTACTS; ++k) {
      bool live = k < (int)o->hist[i].size();
      partner[(size_t)i * ORC_MAX_CONTACTS + k] = live ? o->hist[i][k].partner : INT32_MIN;
      for (int q = 0; q < 3; ++q)
        xi[((size_t)i * ORC_MAX_CONTACTS + k) * 3 + q] = live ? o->hist[i][k].xi[q] : 0.0;
    }
  }
}
int64_t orc_ncells(void *h) { return ((Oracle *)h)->ncell_total; }
void orc_get_gas(void *h, double *out) {
  Oracle *o = (Oracle *)h;
  std::memcpy(out, o->gas.data(), sizeof(double) * o->gas.size());
}
void orc_get_deposits(void *h, double *out) {
  Oracle *o = (Oracle *)h;
  std::memcpy(out, o->dep.data(), sizeof(double) * o->dep.size());
}
void orc_reduction_degree(void *h, double *mean_per_bed, double *oxygen_per_bed, double *per_parcel) {
  Oracle *o = (Oracle *)h;
  std::vector<double> sum(o->nb, 0.0), on(o->nb, 0.0), omax(o->nb, 0.0);
  std::vector<int64_t> cnt(o->nb, 0);
  for (int i = 0; i < o->n; ++i) {
    double m[4] = {o->s[ORC_S_M][i], o->s[ORC_S_M + 1][i], o->s[ORC_S_M + 2][i], o->s[ORC_S_M + 3][i]};
    double f = fov_of(m, o->ore[i]);
    if (per_parcel) per_parcel[i] = f;
    int b = o->bed[i];
    sum[b] += f;
    cnt[b]++;
    double nn[4];
    for (int z = 0; z < 4; ++z) nn[z] = m[z] / kMz[z];
    double nfe = 2 * nn[0] + 3 * nn[1] + nn[2] + nn[3];
    on[b] += 3 * nn[0] + 4 * nn[1] + nn[2];
    omax[b] += (o->ore[i] == 0 ? 1.5 : 4.0 / 3.0) * nfe;
  }
  for (int b = 0; b < o->nb; ++b) {
    if (mean_per_bed) mean_per_bed[b] = cnt[b] ? sum[b] / cnt[b] : 0.0;
    if (oxygen_per_bed) oxygen_per_bed[b] = omax[b] > 0 ? 1.0 - on[b] / omax[b] : 0.0;
  }
}
void orc_set_kinetics(void *h, const double *k0, const double *Ea) {
  Oracle *o = (Oracle *)h;
  for (int b = 0; b < o->nb; ++b)
    for (int r = 0; r < 3; ++r) {
      o->beds[(size_t)b * ORC_NB + ORC_B_K0 + r] = k0[r];
      o->beds[(size_t)b * ORC_NB + ORC_B_EA + r] = Ea[r];
    }
}
void orc_destroy(void *h) { delete (Oracle *)h; }

int32_t orc_adjoint(void *h, int32_t nsteps, int32_t mode, double rel, double *J, double *grad6) {
  Oracle *o = (Oracle *)h;
  // the differentiated map is per parcel in a prescribed gas; radiation and conduction couple
  // parcels, and a solved gas is not the map's prescribed field
  for (int b = 0; b < o->nb; ++b)
    if ((unsigned)ib(o->B(b), ORC_B_FLAGS) & (ORC_RADIATION | ORC_CONDUCTION | ORC_GAS_SOLVER)) return -1;
  std::vector<GasProps> gp(o->ncell_total);
  for (int b = 0; b < o->nb; ++b) {
    const double *bd = o->B(b);
    for (int64_t c = o->cell_off[b]; c < o->cell_off[b + 1]; ++c)
      gp[c] = gas_props(o->gas[c * ORC_NG + ORC_G_T], &o->gas[c * ORC_NG + ORC_G_Y], bd[ORC_B_P0]);
  }
  std::vector<int64_t> pcell(o->n);
  for (int i = 0; i < o->n; ++i) {
    const double *bd = o->B(o->bed[i]);
    Grid g = make_grid(bd);
    pcell[i] = o->cell_off[o->bed[i]] + cell_of(g, o->s[0][i], o->s[1][i], o->s[2][i], nullptr);
  }
  // parameters are shared by all beds: take bed 0's values and apply them everywhere
  double th[6];
  for (int r = 0; r < 3; ++r) { th[r] = o->B(0)[ORC_B_K0 + r]; th[3 + r] = o->B(0)[ORC_B_EA + r]; }
  if (mode == 2) {
    Dual k0s[3], Eas[3];
    for (int r = 0; r < 3; ++r) {
      k0s[r] = Dual(th[r]); k0s[r].d[r] = 1.0;
      Eas[r] = Dual(th[3 + r]); Eas[r].d[3 + r] = 1.0;
    }
    Dual Jd = adjoint_J<Dual>(*o, gp, pcell, nsteps, k0s, Eas);
    *J = Jd.v;
    for (int q = 0; q < 6; ++q) grad6[q] = Jd.d[q];
    return 0;
  }
  auto evalJ = [&](const double t[6]) {
    double k0s[3] = {t[0], t[1], t[2]}, Eas[3] = {t[3], t[4], t[5]};
    return adjoint_J<double>(*o, gp, pcell, nsteps, k0s, Eas);
  };
  *J = evalJ(th);
  if (mode == 1) {
    for (int q = 0; q < 6; ++q) {
      double hq = rel * std::fabs(th[q]);
      double tp[6], tm[6];
      std::memcpy(tp, th, sizeof tp); std::memcpy(tm, th, sizeof tm);
      tp[q] += hq; tm[q] -= hq;
      grad6[q] = (evalJ(tp) - evalJ(tm)) / ((th[q] + hq) - (th[q] - hq));
    }
  }
  return 0;
}

// ---- single-call pieces ----
void orc_gas_props(const double *bed, double Tg, const double *Y, double p, double *out) {
  (void)bed;
  GasProps g = gas_props(Tg, Y, p);
  out[ORC_GP_RHO] = g.rho; out[ORC_GP_MU] = g.mu; out[ORC_GP_LAM] = g.lam; out[ORC_GP_CP] = g.cp;
  out[ORC_GP_X] = g.x;
  for (int j = 0; j < 3; ++j) out[ORC_GP_XP + j] = g.xp[j];
  out[ORC_GP_DM] = g.Dm; out[ORC_GP_MG] = g.Mg; out[ORC_GP_D12] = g.D12; out[ORC_GP_D13] = g.D13;
}

int32_t orc_network(const double *A, const double *B, double F, const int32_t *active_in, double x,
                    const double *xeq, double *J, double *v9, int32_t *active_out) {
  int act[3] = {active_in[0], active_in[1], active_in[2]};
  double Jv[3], v[3][3], Av[3] = {A[0], A[1], A[2]}, Bv[3] = {B[0], B[1], B[2]}, xe[3] = {xeq[0], xeq[1], xeq[2]};
  network(Av, Bv, F, act, x, xe, Jv, v);
  for (int r = 0; r < 3; ++r) {
    J[r] = Jv[r];
    active_out[r] = act[r];
    for (int c = 0; c < 3; ++c) v9[r * 3 + c] = v[r][c];
  }
  return 0;
}

void orc_kinetics(const double *bed, const double *m, double Tp, double d_real, int32_t ore,
                  double eps, double slip, double Tg, const double *Y, double dt_mass, double *out) {
  GasProps g = gas_props(Tg, Y, bed[ORC_B_P0]);
  Kin<double> k;
  double mm[4] = {m[0], m[1], m[2], m[3]};
  kinetics(bed, mm, Tp, d_real, ore, g, eps, slip, dt_mass, bed + ORC_B_K0, bed + ORC_B_EA, k);
  for (int r = 0; r < 3; ++r) {
    out[ORC_K_XIDOT + r] = k.xidot[r]; out[ORC_K_A + r] = k.A[r]; out[ORC_K_B + r] = k.B[r];
    out[ORC_K_F3 + r] = k.f[r]; out[ORC_K_ACT + r] = k.act[r]; out[ORC_K_DEFF + r] = k.Deff[r];
    out[ORC_K_XI + r] = k.xi[r];
  }
  for (int z = 0; z < 4; ++z) out[ORC_K_MDOT + z] = k.mdot[z];
  out[ORC_K_SH2] = k.sH2; out[ORC_K_SH2O] = k.sH2O; out[ORC_K_QR] = k.Qr; out[ORC_K_QRM] = k.Qrm;
  out[ORC_K_F] = k.F; out[ORC_K_SH] = k.Sh; out[ORC_K_EQ] = k.EQ; out[ORC_K_ES] = k.ES;
}

void orc_drag(const double *bed, double d_real, int32_t ore, double eps, double slip, double Tg,
              const double *Y, double *beta_over_epsp, double *Re) {
  GasProps g = gas_props(Tg, Y, bed[ORC_B_P0]);
  double re = 0.0;
  *beta_over_epsp = drag_beta_over_epsp(bed, d_real, ore, eps, slip, g, &re);
  *Re = re;
}

void orc_heat(const double *bed, double d_real, double eps, double slip, double Tg, const double *Y,
              double *Nu, double *h) {
  GasProps g = gas_props(Tg, Y, bed[ORC_B_P0]);
  double Re = g.rho * eps * d_real * slip / g.mu;
  double Pr = g.cp * g.mu / g.lam;
  *Nu = gunn(eps, Re, Pr);
  *h = *Nu * g.lam / d_real;
}

double orc_enthalpy(int32_t species, double T) { return nasa_H(species, T); }
double orc_cp(int32_t species, double T) { return nasa_cp(species, T); }
double orc_molar_mass(int32_t species) { return kNasaM[species]; }
void orc_layer_porosity(const double *bed, int32_t ore, double *xi3) { layer_porosity(bed, ore, xi3); }

int64_t orc_pairs_bruteforce(int32_t n, const double *x, const double *y, const double *z,
                             const double *r, int32_t *pairs, int64_t max_pairs) {
  int64_t np = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (touching(x[i], y[i], z[i], x[j], y[j], z[j], r[i] + r[j])) {
        if (np < max_pairs) { pairs[2 * np] = i; pairs[2 * np + 1] = j; }
        ++np;
      }
  return np;
}

int64_t orc_pairs_cells(int32_t n, const double *x, const double *y, const double *z,
                        const double *r, int32_t *pairs, int64_t max_pairs) {
  std::vector<int32_t> ids(n);
  double h = 0.0;
  for (int i = 0; i < n; ++i) { ids[i] = i; h = std::max(h, 2.0 * r[i]); }
  CellList cl;
  cl.build(ids, x, y, z, std::max(h, 1e-12));
  std::vector<std::pair<int32_t, int32_t>> out;
  for (int i = 0; i < n; ++i)
    cl.neighbours(x[i], y[i], z[i], [&](int32_t j) {
      if (j > i && touching(x[i], y[i], z[i], x[j], y[j], z[j], r[i] + r[j])) out.emplace_back(i, j);
    });
  std::sort(out.begin(), out.end());
  int64_t np = (int64_t)out.size();
  for (int64_t t = 0; t < std::min(np, max_pairs); ++t) { pairs[2 * t] = out[t].first; pairs[2 * t + 1] = out[t].second; }
  return np;
}

void orc_pseudo_turbulence(double eps, double rho, double mu, double lam, double cp, const double *ug,
                           const double *up, double dp, double *out8) {
  const PT t = pseudo_turbulence(eps, rho, mu, lam, cp, ug, up, dp);
  out8[0] = t.Rpa; out8[1] = t.Rpe; out8[2] = t.apa; out8[3] = t.ape;
  for (int q = 0; q < 3; ++q) out8[4 + q] = t.s[q];
  out8[7] = 0.0;
}

void orc_get_faces(void *h, int b, double *fu, double *fv, double *fw) {
  Oracle *o = (Oracle *)h;
  if (b < 0 || b >= o->nb) return;
  std::copy(o->fu[b].begin(), o->fu[b].end(), fu);
  std::copy(o->fv[b].begin(), o->fv[b].end(), fv);
  std::copy(o->fw[b].begin(), o->fw[b].end(), fw);
}

void orc_get_flow(void *h, double *out) {
  Oracle *o = (Oracle *)h;
  for (int b = 0; b < o->nb; ++b) {
    const double *bd = o->B(b);
    Grid gg = make_grid(bd);
    FlowGrid g{gg.nx, gg.ny, gg.nz, gg.dx, gg.dy, gg.dz, o->cell_off[b], o->gas.data()};
    const bool solved = ((unsigned)ib(bd, ORC_B_FLAGS) & ORC_GAS_SOLVER) != 0;
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          const int64_t c = o->cell_off[b] + g.cidx(i, j, k);
          double *r = out + c * ORC_NV;
          if (!solved) {
            r[0] = r[1] = 0.0;
            r[2] = bd[ORC_B_U_IN] / o->gas[c * ORC_NG + ORC_G_EPS];
            r[3] = 0.0;
            continue;
          }
          r[0] = 0.5 * (o->fu[b][g.xf(i, j, k)] + o->fu[b][g.xf(i + 1, j, k)]);
          r[1] = 0.5 * (o->fv[b][g.yf(i, j, k)] + o->fv[b][g.yf(i, j + 1, k)]);
          r[2] = 0.5 * (o->fw[b][g.zf(i, j, k)] + o->fw[b][g.zf(i, j, k + 1)]);
          r[3] = o->pr[b][g.cidx(i, j, k)];
        }
  }
}

double orc_restitution_f(double e) { return restitution_f(e); }
double orc_e_cgp(double e, double k) { return e_cgp(e, k); }
void orc_conduction_pair(const double *bed, double Ra, double Rb, double d, double Ta, double Tb,
                         double lam_a, double lam_b, double lam_g, double *out4) {
  conduction_pair(bed, Ra, Rb, d, Ta, Tb, lam_a, lam_b, lam_g, out4);
}
void orc_conduction_wall(const double *bed, double R, double h, double Ta, double lam_a, double lam_g,
                         double *out4) {
  conduction_wall(bed, R, h, Ta, lam_a, lam_g, out4);
}

void orc_wall_distance(const double *bed, double x, double y, double z, double *dist4, double *n12) {
  double nrm[4][3];
  wall_distance(bed, x, y, z, dist4, nrm);
  for (int k = 0; k < 4; ++k)
    for (int q = 0; q < 3; ++q) n12[k * 3 + q] = nrm[k][q];
}

}  // extern "C"
