// gas.cuh -- the gas phase solved on the GPU instead of the prescribed field (beds with
// DEM_GAS_SOLVER), once per coupling step with dt_CFD = n dt_DEM: continuity (eq (3-24)),
// momentum with the drag of eq (4-2) implicit in u_g and explicit in the parcels' velocities,
// energy with H0 implicit (eq (4-6)), the reducing gas with C0, C1 (eqs (4-8)..(4-11)), the
// pseudo-turbulent stress and heat flux (eqs (3-28)..(3-37)). FP64 in every precision form.
//
// Discretisation: the gas cells as a staggered grid (velocity components on the faces,
// scalars at the centres), explicit Euler, first-order upwind convection. Species and energy
// go first, with the mass fluxes of the last projection. Continuity is taken in the low-Mach
// divergence form: with rho = p M_g / (R T) (eq (3-53)) at fixed p0, eq (3-24) reads
// div(eps u) = -d eps/dt + M / rho - eps D ln(rho)/Dt, D ln(rho)/Dt from the material rates
// of the species and energy update (its change less the convective part), so that an
// equimolar reaction (H2 to H2O) leaves the volume flow unchanged. Then the momentum
// predictor and an incremental pressure projection for that divergence, solved by Jacobi-
// preconditioned conjugate gradients (one global system over all beds, in one cooperative
// kernel). Boundaries: immersed-boundary cells and the box sides are no-slip walls held at
// T_in; a z-face below a fluid cell whose lower neighbour is not fluid takes the inlet gas
// (eps u = U_in, Y_in, T_in); a z-face on top of the box above a fluid cell is an outlet at
// p0 (zero gradient). The pseudo-turbulent stress enters by its normal components in the
// slip frame, the heat flux by the diagonal of alpha_PT; H2O follows by stoichiometry and
// N2 by closure.
#pragma once
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace dem {

// per-cell coefficient rows of one gas step ([GC_N][ncells])
enum : int {
  GC_EPS = 0, GC_EPSO, GC_RHO, GC_MU, GC_LAM, GC_CP, GC_DM, GC_K, GC_KV, GC_RT = GC_KV + 3, GC_AT = GC_RT + 3,
  GC_AX = GC_AT + 3,            // x_H2 / Y_H2 of eq (4-8)
  GC_L = GC_AX + 1,             // pressure-equation coefficient of the cell's lower x-, y-, z-face where
                                // it is open, else 0 (an upper face's is the upper neighbour's lower one)
  GC_DIAG = GC_L + 3,           // the sum over the cell's open faces plus its outlet's
  GC_OUT = GC_DIAG + 1,         // the outlet's coefficient (0 below the top)
  GC_RHS = GC_OUT + 1,
  GC_DIV = GC_RHS + 1,          // div(eps u) that continuity requires of the new flow, 1/s
  GC_N
};
constexpr int GS_CG_MAXIT = 20000;
constexpr double GS_CG_TOL = 1e-12;   // relative residual of the pressure correction

// One level of the multigrid preconditioner of the pressure equation. Level 0 is the gas
// grid itself; level l + 1 aggregates the 2 x 2 x 2 cells (fewer at an odd edge) of level l,
// bed by bed, until every bed is one cell. Operators are Galerkin (P^T A P with P the
// piecewise-constant prolongation): a coarse cell's lower-face coefficient is the sum of its
// children's across that face, its diagonal the sum of its external faces' and outlets'.
constexpr int GS_MAXLEV = 16;
// The preconditioner runs in FP32 (level 0 holds FP32 copies of the FP64 pressure operator);
// the CG around it stays FP64 and takes the flexible (Polak-Ribiere) beta, so the FP32
// rounding of the V-cycle does not limit the FP64 solve.
struct GsLevel {
  long long n;                  // cells, all beds
  float *L;                     // [3][n] lower x-, y-, z-face coefficients
  float *diag, *out;            // diagonal; the outlet's part of it
  float *dinv;                  // GS_OMEGA / diag (0 for an empty cell), set with the operator
  float *b, *xa, *xb;           // right-hand side, two iterate buffers
  const int *bed;               // bed of each cell
  const int *parent;            // the cell of level l + 1 that holds each cell (none on the coarsest)
  int ux, uy;                   // nx, ny when every bed has the same dims at this level, else 0
};
struct GsLevelBed { int nx, ny, nz; long long off; };   // per level and bed: dims, first cell

struct GasView {
  double *fu, *fv, *fw;         // face velocities (x-, y-, z-faces of every bed, bed by bed)
  double *su, *sv, *sw;         // predicted face velocities
  double *pr;                   // pressure relative to p0 [ncells]
  double *co;                   // [GC_N][ncells]
  double *x, *r, *z, *pa, *pb, *Ap;   // CG vectors [ncells]
  double *part;                 // per-block partial sums [blocks][4]
  int *cg_iters;                // iterations of the last solve (diagnostic)
  double *dep;                  // cell sums of the coupling step [ncells][DEM_NDEP]
  const BedP<double> *bpd;
  long long nfx, nfy, nfz;
  // preconditioner: mg_nu = 0 Jacobi, else an FP32 multigrid V-cycle with mg_nu damped-
  // Jacobi sweeps before and after each coarse correction, the correction weighted by mg_alpha
  int mg_nu, nlev, nbeds;
  double mg_alpha;
  const GsLevel *lev;           // [nlev]
  const GsLevelBed *lb;         // [nlev][nbeds]
};

struct GsGrid {
  const DevBed *B;
  const unsigned char *mark;
  __device__ __forceinline__ long long cell(int i, int j, int k) const {
    return B->cell_off + ((long long)k * B->ny + j) * B->nx + i;
  }
  __device__ __forceinline__ bool fluid(int i, int j, int k) const {
    if (i < 0 || j < 0 || k < 0 || i >= B->nx || j >= B->ny || k >= B->nz) return false;
    return mark[cell(i, j, k)] == 0;
  }
  __device__ __forceinline__ long long face(int a, int i, int j, int k) const {
    const int nx = B->nx, ny = B->ny;
    if (a == 0) return B->fx_off + ((long long)k * ny + j) * (nx + 1) + i;
    if (a == 1) return B->fy_off + ((long long)k * (ny + 1) + j) * nx + i;
    return B->fz_off + ((long long)k * ny + j) * nx + i;
  }
  // 0 wall, 1 open, 2 inlet, 3 outlet
  __device__ __forceinline__ int kind(int a, int i, int j, int k) const {
    const int di = a == 0, dj = a == 1, dk = a == 2;
    const bool lo = fluid(i - di, j - dj, k - dk), hi = fluid(i, j, k);
    if (lo && hi) return 1;
    if (a == 2 && hi && !lo) return 2;
    if (a == 2 && lo && k == B->nz) return 3;
    return 0;
  }
  __device__ __forceinline__ void ijk(long long c, int &i, int &j, int &k) const {
    const long long l = c - B->cell_off;
    i = (int)(l % B->nx);
    j = (int)((l / B->nx) % B->ny);
    k = (int)(l / ((long long)B->nx * B->ny));
  }
};
__device__ __forceinline__ double *gs_comp(const GasView &S, int a, bool star) {
  return star ? (a == 0 ? S.su : (a == 1 ? S.sv : S.sw)) : (a == 0 ? S.fu : (a == 1 ? S.fv : S.fw));
}
// the bed of a face of axis a (beds hold their faces in bed order)
__device__ __forceinline__ int gs_face_bed(const DevBed *beds, int nbeds, int a, long long f) {
  int b = 0;
  for (int q = 1; q < nbeds; ++q) {
    const long long o = a == 0 ? beds[q].fx_off : (a == 1 ? beds[q].fy_off : beds[q].fz_off);
    if (f >= o) b = q; else break;
  }
  return b;
}
// the solver's beds share one coupling interval (checked at set-up): bed 0 decides
__device__ __forceinline__ bool gs_active(const DevBed *beds, const long long *ctr) {
  return coupled_step(beds[0].ncouple, ctr);
}

// pseudo-turbulence closures of a cell (eqs (3-28)..(3-37)) as the diagonals in the global
// frame of R_pe I + (R_pa - R_pe) s s^T and of the same form of alpha_PT (s: slip direction);
// Re_m capped at 100 and eps_p at 0.5, the upper ends of the closures' ranges
__device__ inline void gs_pt(double eps, double rho, double mu, double lam, double cp, const double ug[3],
                             const double up[3], double dp, double RT[3], double AT[3]) {
  for (int q = 0; q < 3; ++q) { RT[q] = 0.0; AT[q] = 0.0; }
  const double ep = 1.0 - eps;
  const double sl[3] = {ug[0] - up[0], ug[1] - up[1], ug[2] - up[2]};
  const double sm = sqrt(sl[0] * sl[0] + sl[1] * sl[1] + sl[2] * sl[2]);
  if (!(ep > 0.0) || !(sm > 0.0) || !(dp > 0.0)) return;
  const double Re = fmin(eps * rho * sm * dp / mu, 100.0);
  const double epc = fmin(ep, 0.5);
  const double kg = 0.5 * sm * sm * (2.0 * ep + 2.5 * ep * eps * eps * eps * exp(-ep * sqrt(Re)));   // (3-29), (3-30)
  const double bpa = 0.523 / (1.0 + 0.305 * exp(-0.114 * Re)) * exp(-3.511 * ep / (1.0 + 1.801 * exp(-0.005 * Re)));
  const double bpe = -0.5 * bpa;                                                                     // (3-31), (3-32)
  const double Rpa = 2.0 * kg * (bpa + 1.0 / 3.0), Rpe = 2.0 * kg * (bpe + 1.0 / 3.0);               // (3-28)
  const double Pr = cp * mu / lam, ag = lam / (rho * cp);
  const double Num = (-0.46 + 1.77 * eps + 0.69 * eps * eps) / (eps * eps * eps) +
                     (1.37 - 2.4 * eps + 1.2 * eps * eps) * pow(Re, 0.7) * cbrt(Pr);                 // (3-36)
  const double num = 1.4 * Re * (Re + 1.4) * Pr * exp(-0.002089 * Re) *
                     (eps * (-5.11 * epc + 10.1 * epc * epc - 10.85 * epc * epc * epc) + 1.0 - exp(-10.96 * epc));
  const double e4 = (eps * eps) * (eps * eps);
  const double den = 3.0 * kPI * eps * eps * Num * (1.17 * epc - 0.2021 * sqrt(epc) + 0.08568 * sqrt(sqrt(epc))) *
                     (1.0 - 1.6 * epc * eps - 3.0 * epc * e4 * exp(-pow(Re, 0.4) * epc));
  const double apa = den > 0.0 ? ag * num / den : 0.0;                                               // (3-35)
  const double ape = (3.0 * bpe + 1.0) / (3.0 * bpa + 1.0) * apa;                                     // (3-37)
  for (int q = 0; q < 3; ++q) {
    const double s2 = (sl[q] / sm) * (sl[q] / sm);
    RT[q] = Rpe + (Rpa - Rpe) * s2;
    AT[q] = ape + (apa - ape) * s2;
  }
}

// the properties the solver's equations need (rho, mu, lam, c_p, D_m), with the same
// expressions as gas_cell_props: the parcel-side ones (film and pore terms) are not evaluated
struct GsProps { double rho, mu, lam, cp, Dm; };
__device__ inline GsProps gs_props(const BedP<double> &B, const double Y[3], double T) {
  const Tab<double> &t = tab<double>();
  GsProps o;
  const double p = B.p0;
  const double inv = Y[0] / t.Mj[0] + Y[1] / t.Mj[1] + Y[2] / t.Mj[2];
  const double Mg = 1.0 / inv;
  const double xp0 = Y[0] * Mg / t.Mj[0], xp1 = Y[1] * Mg / t.Mj[1], xp2 = Y[2] * Mg / t.Mj[2];
  o.rho = Mg * p / (kRgas * T);
  double mu = 0, lam = 0, cp = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    mu += Y[j] * (t.visc[j][0] + T * (t.visc[j][1] + T * t.visc[j][2]));
    lam += Y[j] * (t.cond[j][0] + T * (t.cond[j][1] + T * (t.cond[j][2] + T * (t.cond[j][3] + T * t.cond[j][4]))));
    cp += Y[j] * cp_over_R<double>(j, T) * t.RMj[j];
  }
  o.mu = mu; o.lam = lam; o.cp = cp;
  const double sT = sqrt(T);
  const double tf = T * sT * sqrt(sT) * (101325.0 / p) * 1e-7;
  const double D12 = tf * B.fuller12, D13 = tf * B.fuller13;
  const double rest = 1.0 - xp0;
  o.Dm = rest < 1e-12 ? D12 : rest / (xp1 / D12 + xp2 / D13);
  return o;
}

// cell-centre gas velocity: the mean of the cell's two faces on each axis
__device__ __forceinline__ void gs_ucell(const GasView &S, const GsGrid &g, int i, int j, int k, double u[3]) {
  u[0] = 0.5 * (S.fu[g.face(0, i, j, k)] + S.fu[g.face(0, i + 1, j, k)]);
  u[1] = 0.5 * (S.fv[g.face(1, i, j, k)] + S.fv[g.face(1, i, j + 1, k)]);
  u[2] = 0.5 * (S.fw[g.face(2, i, j, k)] + S.fw[g.face(2, i, j, k + 1)]);
}

// 1. per cell, on coupling steps: the cell sums of this step's parcel sources, this step's
// eps (from the parcels' volume), the properties of the old gas state, the drag sums, the
// closures
template <class P>
__global__ void k_gs_coeffs(StepView<P> V, GasView S) {
  pdl_wait();
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells || !gs_active(V.beds, V.step_ctr)) return;
  const int b = V.cell_bed[c];
  const DevBed &B = V.beds[b];
  const size_t nc = (size_t)V.ncells;
  const bool fl = V.mark[c] == 0;
  CellSum<P> cs;
  cs.run(V.src, (size_t)V.cap, V.vals, V.cstart[c], V.cend[c]);
  double d[SR_N];
#pragma unroll
  for (int f = 0; f < SR_N; ++f) {
    d[f] = fl ? (double)cs.s[f] : 0.0;
    S.dep[(size_t)c * SR_N + f] = d[f];
  }
  const double Y[3] = {gas_d<P>(V.gas, GS_Y0 * nc + c), gas_d<P>(V.gas, GS_Y1 * nc + c),
                       gas_d<P>(V.gas, GS_Y2 * nc + c)};
  const double T = gas_d<P>(V.gas, GS_T * nc + c);
  const double eps = fl ? fmax(1.0 - d[SR_VS] * B.inv_vcell, B.eps_min) : B.eps_min;
  const GsProps p = gs_props(S.bpd[b], Y, T);
  double *co = S.co;
  co[GC_EPS * nc + c] = eps;
  co[GC_EPSO * nc + c] = gas_d<P>(V.gas, GS_EPS * nc + c);
  co[GC_RHO * nc + c] = p.rho; co[GC_MU * nc + c] = p.mu; co[GC_LAM * nc + c] = p.lam;
  co[GC_CP * nc + c] = p.cp; co[GC_DM * nc + c] = p.Dm;
  co[GC_K * nc + c] = d[SR_K] * B.inv_vcell;
  for (int q = 0; q < 3; ++q) co[(GC_KV + q) * nc + c] = d[SR_KVX + q] * B.inv_vcell;
  // x_H2 = M_g Y_H2 / (M_H2 X) with X = x'_H2 + x'_H2O (eq (4-8)): the factor of Y_H2
  const Tab<double> &td = tab<double>();
  const double yh = Y[0] / td.Mj[0] + Y[1] / td.Mj[1];
  co[GC_AX * nc + c] = yh > 0.0 ? 1.0 / (td.Mj[0] * yh) : 0.0;
  GsGrid g{&B, V.mark};
  int i, j, k;
  g.ijk(c, i, j, k);
  double RT[3] = {0, 0, 0}, AT[3] = {0, 0, 0};
  if (fl && d[SR_K] > 0.0 && d[SR_CNT] > 0.0) {
    // the drag-weighted mean parcel velocity and the volume-mean real diameter of the cell
    double ug[3];
    gs_ucell(S, g, i, j, k, ug);
    const double up[3] = {d[SR_KVX] / d[SR_K], d[SR_KVY] / d[SR_K], d[SR_KVZ] / d[SR_K]};
    const double dpm = cbrt(6.0 * d[SR_VS] / (kPI * d[SR_CNT] * B.k * B.k * B.k));
    gs_pt(eps, p.rho, p.mu, p.lam, p.cp, ug, up, dpm, RT, AT);
  }
  for (int q = 0; q < 3; ++q) { co[(GC_RT + q) * nc + c] = RT[q]; co[(GC_AT + q) * nc + c] = AT[q]; }
}

// 3. momentum predictor on every face (eq (4-2)), with the old state's properties: the faces of
// all three axes in one launch
template <class P>
__global__ void k_gs_predict(StepView<P> V, GasView S) {
  pdl_wait();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S.nfx + S.nfy + S.nfz || !gs_active(V.beds, V.step_ctr)) return;
  int a = 0;
  if (t >= S.nfx) { t -= S.nfx; a = 1; if (t >= S.nfy) { t -= S.nfy; a = 2; } }
  const DevBed &B = V.beds[gs_face_bed(V.beds, V.nbeds, a, t)];
  GsGrid g{&B, V.mark};
  const int di = a == 0, dj = a == 1, dk = a == 2;
  const int nxa = B.nx + di, nya = B.ny + dj;
  const long long l = t - (a == 0 ? B.fx_off : (a == 1 ? B.fy_off : B.fz_off));
  const int i = (int)(l % nxa), j = (int)((l / nxa) % nya), k = (int)(l / ((long long)nxa * nya));
  const int kd = g.kind(a, i, j, k);
  double *us = gs_comp(S, a, true);
  const size_t nc = (size_t)V.ncells;
  const double *co = S.co;
  if (kd == 0) { us[t] = 0.0; return; }
  if (kd == 2) { us[t] = B.U_in / co[GC_EPS * nc + g.cell(i, j, k)]; return; }
  if (kd == 3) return;   // outlet: the face below, taken with the pressure equation
  const double h[3] = {B.dx, B.dy, B.dz};
  const long long cP = g.cell(i - di, j - dj, k - dk), cN = g.cell(i, j, k);
  const double ef = 0.5 * (co[GC_EPS * nc + cP] + co[GC_EPS * nc + cN]);
  const double rf = 0.5 * (co[GC_RHO * nc + cP] + co[GC_RHO * nc + cN]);
  const double mf = 0.5 * (co[GC_MU * nc + cP] + co[GC_MU * nc + cN]);
  const double Kf = 0.5 * (co[GC_K * nc + cP] + co[GC_K * nc + cN]);
  const double Kvf = 0.5 * (co[(GC_KV + a) * nc + cP] + co[(GC_KV + a) * nc + cN]);
  const double *u = gs_comp(S, a, false);
  const double u0 = u[t];
  // the velocity at the face: its own component, the others from the four faces around it
  double Uf[3];
  for (int bb = 0; bb < 3; ++bb) {
    if (bb == a) { Uf[bb] = u0; continue; }
    const int ei = bb == 0, ej = bb == 1, ek = bb == 2;
    const double *w = gs_comp(S, bb, false);
    Uf[bb] = 0.25 * ((w[g.face(bb, i - di, j - dj, k - dk)] + w[g.face(bb, i - di + ei, j - dj + ej, k - dk + ek)]) +
                     (w[g.face(bb, i, j, k)] + w[g.face(bb, i + ei, j + ej, k + ek)]));
  }
  double conv = 0.0, visc = 0.0;
  for (int bb = 0; bb < 3; ++bb) {
    const int ei = bb == 0, ej = bb == 1, ek = bb == 2;
    double v2[2];
    for (int sd = 0; sd < 2; ++sd) {   // the neighbouring faces of this axis along bb
      const int s = sd ? 1 : -1;
      const int ii = i + s * ei, jj = j + s * ej, kk = k + s * ek;
      const bool in = ii >= 0 && jj >= 0 && kk >= 0 && ii < nxa && jj < nya && kk < B.nz + dk;
      if (in && g.kind(a, ii, jj, kk) != 0) v2[sd] = u[g.face(a, ii, jj, kk)];
      else v2[sd] = bb != a ? -u0 : 0.0;   // a no-slip wall halfway (tangential), at rest (normal)
    }
    const double lo = v2[0], hi = v2[1];
    conv += Uf[bb] > 0.0 ? Uf[bb] * (u0 - lo) / h[bb] : Uf[bb] * (hi - u0) / h[bb];
    visc += (hi - 2.0 * u0 + lo) / (h[bb] * h[bb]);
  }
  const double ptrs = -(co[GC_EPS * nc + cN] * co[GC_RHO * nc + cN] * co[(GC_RT + a) * nc + cN] -
                        co[GC_EPS * nc + cP] * co[GC_RHO * nc + cP] * co[(GC_RT + a) * nc + cP]) / h[a];
  const double dt = B.ncouple * B.dt;
  const double grav = (a == 2 && !(B.flags & DEM_NO_GRAVITY)) ? -kGrav : 0.0;
  const double rhs = ef * rf * u0 / dt - ef * rf * conv + ef * mf * visc + ptrs + ef * rf * grav -
                     ef * (S.pr[cN] - S.pr[cP]) / h[a] + Kvf;
  us[t] = rhs / (ef * rf / dt + Kf);
}

// projection coefficient c_f of an open face (cells P below, N above along its axis) or of
// an outlet face (P below; the outlet pressure half a cell away)
// c_f = eps_f beta_f A_f / h with beta_f = eps_f / (eps_f rho_f / dt + K_f) of eq (4-2)
__device__ __forceinline__ double gs_face_c(const double *co, size_t nc, long long cP, long long cN, bool outlet,
                                            double dt, double Af, double h) {
  if (outlet) {
    const double e = co[GC_EPS * nc + cP], r = co[GC_RHO * nc + cP];
    const double beta = e / (e * r / dt + co[GC_K * nc + cP]);
    return 2.0 * e * beta * Af / h;
  }
  const double ef = 0.5 * (co[GC_EPS * nc + cP] + co[GC_EPS * nc + cN]);
  const double rf = 0.5 * (co[GC_RHO * nc + cP] + co[GC_RHO * nc + cN]);
  const double Kf = 0.5 * (co[GC_K * nc + cP] + co[GC_K * nc + cN]);
  const double beta = ef / (ef * rf / dt + Kf);
  return ef * beta * Af / h;
}
// volume flux eps u A through a face of kind kd with velocity u (the inlet: U_in A)
__device__ __forceinline__ double gs_vflux(const double *co, size_t nc, const GsGrid &g, int a, int i, int j, int k,
                                           int kd, double u, double Af) {
  if (kd == 0) return 0.0;
  if (kd == 2) return g.B->U_in * Af;
  const int di = a == 0, dj = a == 1, dk = a == 2;
  const long long cP = g.cell(i - di, j - dj, k - dk);
  if (kd == 3) return co[GC_EPS * nc + cP] * u * Af;
  return 0.5 * (co[GC_EPS * nc + cP] + co[GC_EPS * nc + g.cell(i, j, k)]) * u * Af;
}
// density of the inlet gas (eq (3-53) at Y_in, T_in, p0)
__device__ __forceinline__ double gs_rho_in(const DevBed &B) {
  const Tab<double> &td = tab<double>();
  const double inv = B.Y_in[0] / td.Mj[0] + B.Y_in[1] / td.Mj[1] + B.Y_in[2] / td.Mj[2];
  return (1.0 / inv) * B.p0 / (kRgas * B.T_in);
}
// mass flux through a face (kg/s along +axis) of kind kd with velocity u and the densities of
// coefficient row rrow; the inlet carries the inlet gas (eps u = U_in at its density rho_in)
__device__ __forceinline__ double gs_face_flux(const double *co, size_t nc, const GsGrid &g, int a, int i, int j,
                                               int k, int kd, double u, double Af, int rrow, double rho_in) {
  if (kd == 0) return 0.0;
  if (kd == 2) return rho_in * g.B->U_in * Af;
  const int di = a == 0, dj = a == 1, dk = a == 2;
  const double *r = co + (size_t)rrow * nc;
  const long long cP = g.cell(i - di, j - dj, k - dk);
  if (kd == 3) return co[GC_EPS * nc + cP] * r[cP] * u * Af;
  const long long cN = g.cell(i, j, k);
  return 0.5 * (co[GC_EPS * nc + cP] + co[GC_EPS * nc + cN]) * 0.5 * (r[cP] + r[cN]) * u * Af;
}
__device__ __forceinline__ double gs_face_val(const GasView &S, const GsGrid &g, int a, int i, int j, int k, bool star) {
  return gs_comp(S, a, star)[g.face(a, i, j, k)];
}

// 4. the pressure equation of every fluid cell: sum_f c_f (p''_nb - p''_P) =
// net predicted volume outflow - V div(eps u); the outlet faces take the predicted velocity
// of the face below (zero gradient)
template <class P>
__global__ void k_gs_rhs(StepView<P> V, GasView S) {
  pdl_wait();
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells || !gs_active(V.beds, V.step_ctr)) return;
  const DevBed &B = V.beds[V.cell_bed[c]];
  const size_t nc = (size_t)V.ncells;
  double *co = S.co;
  for (int q = 0; q < 3; ++q) co[(GC_L + q) * nc + c] = 0.0;
  co[GC_OUT * nc + c] = 0.0;
  if (V.mark[c] != 0) { co[GC_DIAG * nc + c] = 0.0; co[GC_RHS * nc + c] = 0.0; return; }
  GsGrid g{&B, V.mark};
  int i, j, k;
  g.ijk(c, i, j, k);
  const double h[3] = {B.dx, B.dy, B.dz};
  const double Af[3] = {B.dy * B.dz, B.dx * B.dz, B.dx * B.dy};
  const double dt = B.ncouple * B.dt;
  double net = 0.0, dsum = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int di = a == 0, dj = a == 1, dk = a == 2;
    const int kl = g.kind(a, i, j, k), kh = g.kind(a, i + di, j + dj, k + dk);
    double uh = gs_face_val(S, g, a, i + di, j + dj, k + dk, true);
    if (kh == 3) {   // this cell owns the outlet face above it
      uh = gs_face_val(S, g, 2, i, j, k, true);
      S.sw[g.face(2, i, j, k + 1)] = uh;
    }
    const double ul = gs_face_val(S, g, a, i, j, k, true);
    net += gs_vflux(co, nc, g, a, i + di, j + dj, k + dk, kh, uh, Af[a]) - gs_vflux(co, nc, g, a, i, j, k, kl, ul, Af[a]);
    if (kl == 1) {
      const double cf = gs_face_c(co, nc, g.cell(i - di, j - dj, k - dk), c, false, dt, Af[a], h[a]);
      co[(GC_L + a) * nc + c] = cf;
      dsum += cf;
    }
    if (kh == 1 || kh == 3) {   // the same expression the upper neighbour stores for this face
      const double cf = gs_face_c(co, nc, c, kh == 1 ? g.cell(i + di, j + dj, k + dk) : c, kh == 3, dt, Af[a], h[a]);
      if (kh == 3) co[GC_OUT * nc + c] = cf;
      dsum += cf;
    }
  }
  co[GC_RHS * nc + c] = net - B.vcell * co[GC_DIV * nc + c];
  co[GC_DIAG * nc + c] = dsum;
}

// 5. preconditioned conjugate gradients on -L p'' = -rhs, from p'' = 0, to a relative
// residual GS_CG_TOL (at most GS_CG_MAXIT iterations): one cooperative kernel whose blocks
// meet at grid barriers. The preconditioner is Jacobi (mg_nu = 0) or one FP32 multigrid
// V-cycle (damped Jacobi before and after the coarse correction, the coarsest level of one
// cell per bed solved exactly) under the flexible form of CG; either converges to the same
// FP64 tolerance, so the answer differs from the Jacobi-preconditioned solve by rounding only. The search direction is
// double-buffered so that p_k = z_k + beta p_{k-1} is formed where -L p_k is (neighbours
// recomputed from z and p_{k-1}). Sums are per-block partials added in block order by every
// block: the same value in every block, reproducible run to run.
constexpr int GS_CG_BLOCK = 256;
constexpr double GS_OMEGA = 0.8;   // damping of the Jacobi smoother
__device__ __forceinline__ double gs_cg_dir(const double *z, const double *po, double beta, long long c) {
  return z[c] + beta * po[c];
}
template <int NV>
__device__ __forceinline__ void gs_block_sums(double (&v)[NV], double *part, int slot0, double *sh) {
#pragma unroll
  for (int q = 0; q < NV; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q * 32 + w] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[q * 32 + k];
      part[(size_t)blockIdx.x * 4 + slot0 + q] = s;
    }
  }
  __syncthreads();
}
// the grid's sums of slots [slot0, slot0 + NV), after a grid barrier
template <int NV>
__device__ __forceinline__ void gs_grid_sums(const double *part, int slot0, double *sh, double (&out)[NV]) {
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int k = threadIdx.x; k < (int)gridDim.x; k += 32) s += part[(size_t)k * 4 + slot0 + q];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) sh[128 + q] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = sh[128 + q];
  __syncthreads();
}

// (A x)_i of the operator of a level (A = -L: diag x_i - sum over open faces c_f x_nb), for
// x read through XV (a plain array, or one with a coarse correction added as it is read).
// The upper neighbour along an axis is i + stride: where that steps out of the row or the
// plane, the cell reached (same bed) has the box side as its lower face, coefficient 0;
// where every bed has the same dims the bed's top steps into the next bed's bottom cell,
// whose lower z-face coefficient is 0 too (an inlet or a wall), so only the array's end
// bounds it; otherwise the bed's end does.
template <class XV>
__device__ __forceinline__ float gs_apply(const GsLevel &Lv, long long sy, long long sz, long long end, long long i,
                                          const XV &xv) {
  const long long st[3] = {1, sy, sz};
  float acc = Lv.diag[i] * xv(i);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float cl = Lv.L[a * Lv.n + i];
    const float ch = i + st[a] < end ? Lv.L[a * Lv.n + i + st[a]] : 0.0f;
    if (cl != 0.0f) acc -= cl * xv(i - st[a]);
    if (ch != 0.0f) acc -= ch * xv(i + st[a]);
  }
  return acc;
}
// strides and end of cell i's bed at a level
__device__ __forceinline__ void gs_strides(const GasView &S, const GsLevel &Lv, int l, long long i, long long &sy,
                                           long long &sz, long long &end) {
  if (Lv.ux > 0) {
    sy = Lv.ux; sz = (long long)Lv.ux * Lv.uy; end = Lv.n;
  } else {
    const GsLevelBed g = S.lb[(size_t)l * S.nbeds + Lv.bed[i]];
    sy = g.nx; sz = (long long)g.nx * g.ny; end = g.off + sz * g.nz;
  }
}
__device__ __forceinline__ void gs_local(const GsLevelBed &g, long long i, int &x, int &y, int &z) {
  const int l = (int)(i - g.off);   // a bed has fewer than 2^30 cells
  const int q = l / g.nx;
  x = l - q * g.nx;
  z = q / g.ny;
  y = q - z * g.ny;
}
// levels of at most this many cells are smoothed and restricted by one block alone (block
// barriers instead of grid barriers)
constexpr long long GS_SMALL = 2048;

// level 0 of the preconditioner: FP32 copies of this step's pressure operator
__device__ __forceinline__ void gs_mg_level0(const GasView &S, const GsLevel &L0, long long c0, long long stride) {
  const size_t nc = (size_t)L0.n;
  const double *L = S.co + GC_L * nc, *dg = S.co + GC_DIAG * nc, *ot = S.co + GC_OUT * nc;
  for (long long c = c0; c < L0.n; c += stride) {
#pragma unroll
    for (int a = 0; a < 3; ++a) L0.L[a * nc + c] = (float)L[a * nc + c];
    const double d = dg[c];
    L0.diag[c] = (float)d;
    L0.out[c] = (float)ot[c];
    L0.dinv[c] = d > 0.0 ? (float)(GS_OMEGA / d) : 0.0f;
  }
}

// Galerkin coefficients of level l + 1 from level l: per coarse cell, over its children
static __device__ __noinline__ void gs_mg_setup(const GasView &S, const GsLevel *lev, int l, long long c0,
                                                long long stride) {
  const GsLevel &F = lev[l], &Cv = lev[l + 1];
  for (long long I = c0; I < Cv.n; I += stride) {
    const int b = Cv.bed[I];
    const GsLevelBed gf = S.lb[(size_t)l * S.nbeds + b], gc = S.lb[(size_t)(l + 1) * S.nbeds + b];
    int X, Y, Z;
    gs_local(gc, I, X, Y, Z);
    const int C[3] = {X, Y, Z}, nf[3] = {gf.nx, gf.ny, gf.nz};
    const long long st[3] = {1, gf.nx, (long long)gf.nx * gf.ny};
    float Lc[3] = {0.0f, 0.0f, 0.0f}, dc = 0.0f, oc = 0.0f;
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          const int f[3] = {2 * X + di, 2 * Y + dj, 2 * Z + dk};
          if (f[0] >= nf[0] || f[1] >= nf[1] || f[2] >= nf[2]) continue;
          const long long i = gf.off + ((long long)f[2] * nf[1] + f[1]) * nf[0] + f[0];
          oc += F.out[i];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if ((f[a] - 1) >> 1 != C[a] || f[a] == 0) {   // lower face external (or the box side)
              const float v = F.L[a * F.n + i];
              Lc[a] += v;
              dc += v;
            }
            if (f[a] + 1 < nf[a] && (f[a] + 1) >> 1 != C[a]) dc += F.L[a * F.n + i + st[a]];   // upper, external
          }
        }
#pragma unroll
    for (int a = 0; a < 3; ++a) Cv.L[a * Cv.n + I] = Lc[a];
    Cv.diag[I] = dc + oc;
    Cv.out[I] = oc;
    Cv.dinv[I] = dc + oc > 0.0f ? (float)GS_OMEGA / (dc + oc) : 0.0f;
  }
}

// A damped-Jacobi sweep of level l, x_dst = x' + omega D^-1 (b - A x'), with x' = x_src, or
// with CORR x' = x_src + w P x_c (the coarse correction applied as the values are read, so no
// barrier separates it from the sweep). FINAL (level 0): the result goes to the FP64 z of the
// CG, with the partial sums r . z and r . z_old.
template <bool CORR, bool FINAL>
__device__ __forceinline__ void gs_sweep(const GasView &S, const GsLevel *lev, int l, const float *src, float *dst,
                                         long long c0, long long stride, double *rz, double *rzo) {
  const GsLevel &Lv = lev[l];
  const float *__restrict__ xc = CORR ? lev[l + 1].xb : nullptr;
  const int *__restrict__ par = Lv.parent;
  const float w = (float)S.mg_alpha;
  auto xv = [&](long long k) -> float { return CORR ? src[k] + w * xc[par[k]] : src[k]; };
  for (long long i = c0; i < Lv.n; i += stride) {
    const float di = Lv.dinv[i];
    float v = 0.0f;
    if (di != 0.0f) {
      long long sy, sz, end;
      gs_strides(S, Lv, l, i, sy, sz, end);
      v = xv(i) + (Lv.b[i] - gs_apply(Lv, sy, sz, end, i, xv)) * di;
    }
    if constexpr (FINAL) {
      const double zo = S.z[i], rc = S.r[i];
      S.z[i] = (double)v;
      *rz += rc * (double)v;
      *rzo += rc * zo;
    } else {
      dst[i] = v;
    }
  }
}

// restriction of level l's residual b - A x (x: the iterate xf) to level l + 1's right-hand
// side, with the first sweep there (from 0), or the exact solve of the coarsest level (one
// cell per bed) into its xb
__device__ __forceinline__ void gs_mg_restrict(const GasView &S, const GsLevel *lev, int l, const float *xf,
                                               long long c0, long long stride) {
  const GsLevel &F = lev[l], &Cv = lev[l + 1];
  const bool coarsest = l + 2 == S.nlev;
  auto xv = [&](long long k) -> float { return xf[k]; };
  for (long long I = c0; I < Cv.n; I += stride) {
    const int b = Cv.bed[I];
    const GsLevelBed gf = S.lb[(size_t)l * S.nbeds + b], gc = S.lb[(size_t)(l + 1) * S.nbeds + b];
    int X, Y, Z;
    gs_local(gc, I, X, Y, Z);
    const long long sy = gf.nx, sz = (long long)gf.nx * gf.ny;
    const long long end = F.ux > 0 ? F.n : gf.off + sz * gf.nz;
    float sum = 0.0f;
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          const int fx = 2 * X + di, fy = 2 * Y + dj, fz = 2 * Z + dk;
          if (fx >= gf.nx || fy >= gf.ny || fz >= gf.nz) continue;
          const long long i = gf.off + ((long long)fz * gf.ny + fy) * gf.nx + fx;
          if (F.dinv[i] != 0.0f) sum += F.b[i] - gs_apply(F, sy, sz, end, i, xv);
        }
    Cv.b[I] = sum;
    const float w = Cv.dinv[I];
    if (coarsest) Cv.xb[I] = sum * (w * (float)(1.0 / GS_OMEGA));   // one cell per bed: exact
    else Cv.xa[I] = sum * w;
  }
}

// One V-cycle z = M r (r, z: the CG's FP64 vectors) and the grid's r . z and r . z_old. The
// sweep counts before and after each coarse correction are equal and the smoother is
// symmetric, so M is symmetric up to the FP32 rounding; every sweep after the first reads its
// neighbours, so a barrier separates the phases.
static __device__ __noinline__ void gs_vcycle(const GasView &S, const GsLevel *lev,
                                              cooperative_groups::grid_group &grid, long long c0, long long stride,
                                              double *sh, double (&out)[2]) {
  const int nu = S.mg_nu;
  double rz = 0.0, rzo = 0.0;
  const GsLevel &L0 = lev[0];
  if (S.nlev == 1) {   // one cell per bed: the exact solve
    for (long long i = c0; i < L0.n; i += stride) {
      const double rc = S.r[i], zo = S.z[i];
      const double v = rc * ((double)L0.dinv[i] * (1.0 / GS_OMEGA));
      S.z[i] = v;
      rz += rc * v;
      rzo += rc * zo;
    }
  } else {
    int ls = S.nlev;   // the first level that one block handles
    for (int l = 1; l < S.nlev; ++l)
      if (lev[l].n <= GS_SMALL) { ls = l; break; }
    for (long long i = c0; i < L0.n; i += stride) {   // level 0: b = r, first sweep from 0
      const float b = (float)S.r[i];
      L0.b[i] = b;
      L0.xa[i] = b * L0.dinv[i];
    }
    grid.sync();
    for (int l = 0; l < ls && l + 1 < S.nlev; ++l) {   // down: smooth, restrict (first sweep below fused)
      if (nu == 2) {
        gs_sweep<false, false>(S, lev, l, lev[l].xa, lev[l].xb, c0, stride, nullptr, nullptr);
        grid.sync();
      }
      gs_mg_restrict(S, lev, l, nu == 2 ? lev[l].xb : lev[l].xa, c0, stride);
      grid.sync();
    }
    if (ls + 1 < S.nlev) {   // the small levels, down and up, in block 0
      if (blockIdx.x == 0) {
        const long long t0 = threadIdx.x, ts = blockDim.x;
        for (int l = ls; l + 1 < S.nlev; ++l) {
          if (nu == 2) {
            gs_sweep<false, false>(S, lev, l, lev[l].xa, lev[l].xb, t0, ts, nullptr, nullptr);
            __syncthreads();
          }
          gs_mg_restrict(S, lev, l, nu == 2 ? lev[l].xb : lev[l].xa, t0, ts);
          __syncthreads();
        }
        for (int l = S.nlev - 2; l >= ls; --l) {
          if (nu == 2) {
            gs_sweep<true, false>(S, lev, l, lev[l].xb, lev[l].xa, t0, ts, nullptr, nullptr);
            __syncthreads();
            gs_sweep<false, false>(S, lev, l, lev[l].xa, lev[l].xb, t0, ts, nullptr, nullptr);
          } else {
            gs_sweep<true, false>(S, lev, l, lev[l].xa, lev[l].xb, t0, ts, nullptr, nullptr);
          }
          __syncthreads();
        }
      }
      grid.sync();
    }
    for (int l = (ls < S.nlev ? ls : S.nlev - 1) - 1; l >= 0; --l) {   // up: correct and smooth
      if (nu == 2) {
        gs_sweep<true, false>(S, lev, l, lev[l].xb, lev[l].xa, c0, stride, nullptr, nullptr);
        grid.sync();
        if (l > 0) gs_sweep<false, false>(S, lev, l, lev[l].xa, lev[l].xb, c0, stride, nullptr, nullptr);
        else gs_sweep<false, true>(S, lev, 0, lev[0].xa, nullptr, c0, stride, &rz, &rzo);
      } else {
        if (l > 0) gs_sweep<true, false>(S, lev, l, lev[l].xa, lev[l].xb, c0, stride, nullptr, nullptr);
        else gs_sweep<true, true>(S, lev, 0, lev[0].xa, nullptr, c0, stride, &rz, &rzo);
      }
      if (l > 0) grid.sync();
    }
  }
  double v[2] = {rz, rzo};
  gs_block_sums<2>(v, S.part, 2, sh);
  grid.sync();
  gs_grid_sums<2>(S.part, 2, sh, out);
}

template <class P>
__global__ void __launch_bounds__(GS_CG_BLOCK, 4) k_gs_cg(const DevBed *beds, const int *cell_bed,
                                                       const long long *ctr, long long ncells, GasView S) {
  namespace cg = cooperative_groups;
  if (!gs_active(beds, ctr)) return;   // the same answer in every block
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[4 * 32 + 8];
  __shared__ GsLevel lev[GS_MAXLEV];   // the level descriptors, read by every phase
  if (threadIdx.x < S.nlev) lev[threadIdx.x] = S.lev[threadIdx.x];
  __syncthreads();
  const size_t nc = (size_t)ncells;
  const double *diag = S.co + GC_DIAG * nc, *rhs = S.co + GC_RHS * nc;
  const double *L = S.co + GC_L * nc;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long c0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double *x = S.x, *r = S.r, *z = S.z, *Ap = S.Ap;
  double *po = S.pa, *pn = S.pb;
  const bool mg = S.mg_nu > 0;
  const int uxy[2] = {lev[0].ux, lev[0].uy};
  if (mg) {   // the preconditioner's operators of this step's coefficients (small levels in block 0)
    gs_mg_level0(S, lev[0], c0, stride);
    grid.sync();
    int l = 0;
    for (; l + 1 < S.nlev && lev[l + 1].n > GS_SMALL; ++l) {
      gs_mg_setup(S, lev, l, c0, stride);
      grid.sync();
    }
    if (l + 1 < S.nlev) {
      if (blockIdx.x == 0)
        for (; l + 1 < S.nlev; ++l) {
          gs_mg_setup(S, lev, l, threadIdx.x, blockDim.x);
          __syncthreads();
        }
      grid.sync();
    }
  }
  {
    double v[2] = {0.0, 0.0};
    for (long long c = c0; c < ncells; c += stride) {
      const double rc = -rhs[c];
      r[c] = rc; x[c] = 0.0; po[c] = 0.0;
      v[0] += rc * rc;
      const double zc = !mg && diag[c] > 0.0 ? rc / diag[c] : 0.0;
      z[c] = zc;
      v[1] += rc * zc;
    }
    gs_block_sums<2>(v, S.part, 1, sh);
  }
  grid.sync();
  double s2[2];
  gs_grid_sums<2>(S.part, 1, sh, s2);
  const double bnorm = sqrt(s2[0]);
  double rz = s2[1], beta = 0.0;
  int it = 0;
  if (bnorm > 0.0) {
    if (mg) {
      double o2[2];
      gs_vcycle(S, lev, grid, c0, stride, sh, o2);
      rz = o2[0];
    }
    for (; it < GS_CG_MAXIT; ++it) {
      // p_k and -L p_k
      double v1[1] = {0.0};
      for (long long c = c0; c < ncells; c += stride) {
        const double pc = gs_cg_dir(z, po, beta, c);
        pn[c] = pc;
        double acc = diag[c] * pc;
        if (diag[c] > 0.0) {
          long long st[3] = {1, uxy[0], (long long)uxy[0] * uxy[1]}, cend = ncells;   // uniform dims: see gs_apply
          if (uxy[0] == 0) {
            const DevBed &B = beds[cell_bed[c]];
            st[1] = B.nx; st[2] = (long long)B.nx * B.ny; cend = B.cell_off + st[2] * B.nz;
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const double cl = L[a * nc + c];
            const double ch = c + st[a] < cend ? L[a * nc + c + st[a]] : 0.0;
            if (cl != 0.0) acc -= cl * gs_cg_dir(z, po, beta, c - st[a]);
            if (ch != 0.0) acc -= ch * gs_cg_dir(z, po, beta, c + st[a]);
          }
        }
        Ap[c] = acc;
        v1[0] += pc * acc;
      }
      gs_block_sums<1>(v1, S.part, 0, sh);
      grid.sync();
      double pAp[1];
      gs_grid_sums<1>(S.part, 0, sh, pAp);
      if (!(pAp[0] > 0.0)) break;
      const double alpha = rz / pAp[0];
      double v2[2] = {0.0, 0.0};
      for (long long c = c0; c < ncells; c += stride) {
        x[c] += alpha * pn[c];
        const double rc = r[c] - alpha * Ap[c];
        r[c] = rc;
        v2[0] += rc * rc;
        if (!mg) {
          const double zc = diag[c] > 0.0 ? rc / diag[c] : 0.0;
          z[c] = zc;
          v2[1] += rc * zc;
        }
      }
      gs_block_sums<2>(v2, S.part, 1, sh);
      grid.sync();
      gs_grid_sums<2>(S.part, 1, sh, s2);
      if (sqrt(s2[0]) < GS_CG_TOL * bnorm) { ++it; break; }
      if (mg) {   // flexible beta: r_new . (z_new - z_old) / (r_old . z_old)
        double o2[2];
        gs_vcycle(S, lev, grid, c0, stride, sh, o2);
        beta = (o2[0] - o2[1]) / rz;
        rz = o2[0];
      } else {
        beta = s2[1] / rz;
        rz = s2[1];
      }
      double *t = po; po = pn; pn = t;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *S.cg_iters = it;
}

// 6. projection: the open and outlet faces corrected by the pressure-correction gradient, the
// others as predicted; the pressure updated
template <class P>
__global__ void k_gs_correct(StepView<P> V, GasView S) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nf = S.nfx + S.nfy + S.nfz;
  if (t >= nf + V.ncells || !gs_active(V.beds, V.step_ctr)) return;
  if (t >= nf) {
    const long long c = t - nf;
    S.pr[c] += S.x[c];
    return;
  }
  int a = 0;
  if (t >= S.nfx) { t -= S.nfx; a = 1; if (t >= S.nfy) { t -= S.nfy; a = 2; } }
  const DevBed &B = V.beds[gs_face_bed(V.beds, V.nbeds, a, t)];
  GsGrid g{&B, V.mark};
  const int di = a == 0, dj = a == 1, dk = a == 2;
  const int nxa = B.nx + di, nya = B.ny + dj;
  const long long l = t - (a == 0 ? B.fx_off : (a == 1 ? B.fy_off : B.fz_off));
  const int i = (int)(l % nxa), j = (int)((l / nxa) % nya), k = (int)(l / ((long long)nxa * nya));
  const int kd = g.kind(a, i, j, k);
  const double us = gs_comp(S, a, true)[t];
  double u = us;
  const size_t nc = (size_t)V.ncells;
  const double *co = S.co;
  const double dt = B.ncouple * B.dt;
  const double h = a == 0 ? B.dx : (a == 1 ? B.dy : B.dz);
  if (kd == 3) {
    const long long cP = g.cell(i, j, k - 1);
    const double e = co[GC_EPS * nc + cP], r = co[GC_RHO * nc + cP];
    const double beta = e / (e * r / dt + co[GC_K * nc + cP]);
    u = us - beta * (0.0 - S.x[cP]) / (0.5 * h);
  } else if (kd == 1) {
    const long long cP = g.cell(i - di, j - dj, k - dk), cN = g.cell(i, j, k);
    const double ef = 0.5 * (co[GC_EPS * nc + cP] + co[GC_EPS * nc + cN]);
    const double rf = 0.5 * (co[GC_RHO * nc + cP] + co[GC_RHO * nc + cN]);
    const double Kf = 0.5 * (co[GC_K * nc + cP] + co[GC_K * nc + cN]);
    u = us - ef / (ef * rf / dt + Kf) * (S.x[cN] - S.x[cP]) / h;
  }
  gs_comp(S, a, false)[t] = u;
}

// the cell's property record for the next steps: the properties of (eps, Y, T) in the form's
// type, and the cell-centre velocity of the solved faces
template <class P>
__device__ __forceinline__ void gs_store_props(StepView<P> &V, const GasView &S, const GsGrid &g, long long c,
                                               double eps, const double Y[3], double T) {
  using R = typename P::R;
  const BedP<R> &bp = V.bp[V.cell_bed[c]];
  const R Yr[3] = {(R)Y[0], (R)Y[1], (R)Y[2]};
  CellProps<R> p = gas_cell_props<R>(bp, (R)eps, Yr, (R)T);
  int i, j, k;
  g.ijk(c, i, j, k);
  double u[3];
  gs_ucell(S, g, i, j, k, u);
  p.ux = (R)u[0]; p.uy = (R)u[1]; p.uz = (R)u[2];
  store_props(V, c, p);
}
// the state in the form's storage: FP64 words or compensated FP32 pairs
template <class P> __device__ __forceinline__ double gs_get(const double *G, size_t k) { return gas_d<P>(G, k); }
template <class P> __device__ __forceinline__ void gs_put(double *G, size_t k, double v) { gas_put(G, k, v, !P::exact); }

// 2. species (eq (4-9)) and energy (eq (4-6)) with the mass fluxes of the last projection
// (the current faces, the old densities), every step: on coupling steps the update and the
// velocity divergence continuity requires, on the others a copy of the state
template <class P>
__global__ void k_gs_scalars(StepView<P> V, GasView S) {
  pdl_wait();
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells) return;
  const size_t nc = (size_t)V.ncells;
  const bool active = gs_active(V.beds, V.step_ctr);
  const double *G = V.gas;
  double *Gn = V.gas_new;
  if (!active) {   // a copy of the words (pairs stay pairs)
    for (int q = 0; q < GS_N; ++q) Gn[q * nc + c] = G[q * nc + c];
    return;
  }
  double Y[3] = {gs_get<P>(G, GS_Y0 * nc + c), gs_get<P>(G, GS_Y1 * nc + c), gs_get<P>(G, GS_Y2 * nc + c)};
  double T = gs_get<P>(G, GS_T * nc + c);
  const DevBed &B = V.beds[V.cell_bed[c]];
  GsGrid g{&B, V.mark};
  double *co = S.co;
  const double eps = co[GC_EPS * nc + c];
  const double rho = co[GC_RHO * nc + c];
  double div = 0.0;
  if (V.mark[c] == 0) {
    int i, j, k;
    g.ijk(c, i, j, k);
    const double h[3] = {B.dx, B.dy, B.dz};
    const double Af[3] = {B.dy * B.dz, B.dx * B.dz, B.dx * B.dy};
    const double Afh[3] = {Af[0] / h[0], Af[1] / h[1], Af[2] / h[2]};
    const double dt = B.ncouple * B.dt, idt = 1.0 / dt;
    const double rho_in = gs_rho_in(B);
    const double cp = co[GC_CP * nc + c], lam = co[GC_LAM * nc + c];
    const double Dm = co[GC_DM * nc + c];
    const double Y0 = Y[0], Y1 = Y[1], Y2o = Y[2];
    double cY0 = 0.0, cY1 = 0.0, cT = 0.0, dY0 = 0.0, dY1 = 0.0, dT = 0.0;
    for (int a = 0; a < 3; ++a) {
      const int di = a == 0, dj = a == 1, dk = a == 2;
      const double ATc = co[(GC_AT + a) * nc + c];
      for (int side = 0; side < 2; ++side) {
        const int fi = i + side * di, fj = j + side * dj, fk = k + side * dk;
        const int kd = g.kind(a, fi, fj, fk);
        const double F = kd == 0 ? 0.0
                                 : gs_face_flux(co, nc, g, a, fi, fj, fk, kd, gs_face_val(S, g, a, fi, fj, fk, false),
                                                Af[a], GC_RHO, rho_in);
        const double inflow = side == 0 ? F : -F;
        if (kd == 1) {
          const long long cn = g.cell(i + (side ? di : -di), j + (side ? dj : -dj), k + (side ? dk : -dk));
          const double yn0 = gs_get<P>(G, GS_Y0 * nc + cn), yn1 = gs_get<P>(G, GS_Y1 * nc + cn);
          const double tn = gs_get<P>(G, GS_T * nc + cn);
          if (inflow > 0.0) {
            cY0 += inflow * (yn0 - Y0);
            cY1 += inflow * (yn1 - Y1);
            cT += inflow * cp * (tn - T);
          }
          const double ef = 0.5 * (eps + co[GC_EPS * nc + cn]), rf = 0.5 * (rho + co[GC_RHO * nc + cn]);
          const double ATf = 0.5 * (ATc + co[(GC_AT + a) * nc + cn]);
          const double Df = 0.5 * (Dm + co[GC_DM * nc + cn]) + ATf;
          const double lf = 0.5 * (lam + co[GC_LAM * nc + cn]) + rf * (0.5 * (cp + co[GC_CP * nc + cn])) * ATf;
          const double gD = ef * rf * Df * Afh[a];
          dY0 += gD * (yn0 - Y0);
          dY1 += gD * (yn1 - Y1);
          dT += ef * lf * Afh[a] * (tn - T);
        } else if (kd == 2) {
          if (inflow > 0.0) {
            cY0 += inflow * (B.Y_in[0] - Y0);
            cY1 += inflow * (B.Y_in[1] - Y1);
            cT += inflow * cp * (B.T_in - T);
          }
        } else if (kd == 0) {   // a wall at the inlet temperature
          dT += eps * lam * (2.0 * Afh[a]) * (B.T_in - T);
        }                       // outlet: zero gradient
      }
    }
    const double *d = S.dep + (size_t)c * SR_N;
    const double m = eps * rho * B.vcell;
    // eqs (4-8)..(4-11): H2 consumed at (M_H2 p / R)(x EQ - ES) with x implicit in Y_H2; H2O
    // produced at M_H2O / M_H2 times that; the net mass source takes Y and c_p T of the cell
    const Tab<double> &td = tab<double>();
    const double MH2 = td.Mj[0], MH2O = td.Mj[1];
    const double C0 = MH2 * B.p0 * co[GC_AX * nc + c] * d[SR_EQ] / kRgas, C1 = MH2 * B.p0 * d[SR_ES] / kRgas;
    const double rq = MH2O / MH2 - 1.0;
    const double mdt = m * idt;
    const double Y0n = (mdt * Y0 + cY0 + dY0 + C1 * (1.0 + Y0 * rq)) / (mdt + C0 * (1.0 + Y0 * rq));
    const double cons = C0 * Y0n - C1;
    const double Mnet = rq * cons;
    const double Y0f = fmax(Y0n, 0.0);
    const double im = 1.0 / m;
    const double Y1f = fmax(Y1 + dt * im * (cY1 + dY1 + MH2O / MH2 * cons - Y1 * Mnet), 0.0);
    const double Y2f = fmax(1.0 - Y0f - Y1f, 0.0);
    const double ys = Y0f + Y1f + Y2f;
    const double iys = 1.0 / ys;
    Y[0] = Y0f * iys; Y[1] = Y1f * iys; Y[2] = Y2f * iys;
    // M_r of eq (3-39) with the parcels' species sources and M_rm of eq (3-38): together the
    // sensible enthalpy the species bring from the parcels' temperature
    const double Mr = -(h_over_R<double>(0, T) * td.RMj[0] * d[SR_SH2] + h_over_R<double>(1, T) * td.RMj[1] * d[SR_SH2O]);
    const double Mrm = -d[SR_QRM];
    const double mc = m * cp;
    const double mcdt = mc * idt;
    const double Tn = (mcdt * T + cT + dT + d[SR_HAT] + Mr + Mrm) / (mcdt + d[SR_HA]);
    // div(eps u) = -d eps/dt + M / rho - eps D ln(rho)/Dt (the material rates: the change less
    // its convective part; the N2 carried in is -(cY0 + cY1))
    const double DY0 = (Y[0] - Y0) * idt - cY0 * im, DY1 = (Y[1] - Y1) * idt - cY1 * im;
    const double DY2 = (Y[2] - Y2o) * idt + (cY0 + cY1) * im;
    const double DT = (Tn - T) * idt - cT * im / cp;
    const double iM[3] = {1.0 / td.Mj[0], 1.0 / td.Mj[1], 1.0 / td.Mj[2]};   // constants, folded
    const double Mg = 1.0 / (Y0 * iM[0] + Y1 * iM[1] + Y2o * iM[2]);
    const double Dlnrho = -Mg * (DY0 * iM[0] + DY1 * iM[1] + DY2 * iM[2]) - DT / T;
    div = -(eps - co[GC_EPSO * nc + c]) * idt + Mnet * im * eps - eps * Dlnrho;
    T = Tn;
  }
  gs_put<P>(Gn, GS_EPS * nc + c, eps);
  gs_put<P>(Gn, GS_Y0 * nc + c, Y[0]); gs_put<P>(Gn, GS_Y1 * nc + c, Y[1]); gs_put<P>(Gn, GS_Y2 * nc + c, Y[2]);
  gs_put<P>(Gn, GS_T * nc + c, T);
  co[GC_DIV * nc + c] = div;
}

// 7. on coupling steps, the cell's property record for the next steps from the updated state
// and the projected faces
template <class P>
__global__ void k_gs_props(StepView<P> V, GasView S) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells || !gs_active(V.beds, V.step_ctr)) return;
  const size_t nc = (size_t)V.ncells;
  const DevBed &B = V.beds[V.cell_bed[c]];
  GsGrid g{&B, V.mark};
  const double *Gn = V.gas_new;
  const double Y[3] = {gs_get<P>(Gn, GS_Y0 * nc + c), gs_get<P>(Gn, GS_Y1 * nc + c), gs_get<P>(Gn, GS_Y2 * nc + c)};
  gs_store_props(V, S, g, c, gs_get<P>(Gn, GS_EPS * nc + c), Y, gs_get<P>(Gn, GS_T * nc + c));
}

// initial flow of the solved beds: plug flow at the superficial velocity through every
// fluid column (eps w = U_in on the z-faces that carry gas), no cross flow, p = p0; then
// the property records with the cell-centre velocities of those faces
template <class P>
__global__ void k_gs_init_faces(StepView<P> V, GasView S) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nf = S.nfx + S.nfy + S.nfz;
  if (t >= nf + V.ncells) return;
  if (t >= nf) { S.pr[t - nf] = 0.0; return; }
  int a = 0;
  if (t >= S.nfx) { t -= S.nfx; a = 1; if (t >= S.nfy) { t -= S.nfy; a = 2; } }
  double *u = gs_comp(S, a, false);
  if (a != 2) { u[t] = 0.0; return; }
  const DevBed &B = V.beds[gs_face_bed(V.beds, V.nbeds, 2, t)];
  GsGrid g{&B, V.mark};
  const long long l = t - B.fz_off;
  const int i = (int)(l % B.nx), j = (int)((l / B.nx) % B.ny), k = (int)(l / ((long long)B.nx * B.ny));
  const int kd = g.kind(2, i, j, k);
  if (kd == 0) { u[t] = 0.0; return; }
  const long long cc = g.cell(i, j, kd == 3 ? k - 1 : k);
  u[t] = B.U_in / gs_get<P>(V.gas, GS_EPS * (size_t)V.ncells + cc);
}
template <class P>
__global__ void k_gs_init_props(StepView<P> V, GasView S) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells) return;
  const size_t nc = (size_t)V.ncells;
  const DevBed &B = V.beds[V.cell_bed[c]];
  GsGrid g{&B, V.mark};
  const double Y[3] = {gs_get<P>(V.gas, GS_Y0 * nc + c), gs_get<P>(V.gas, GS_Y1 * nc + c), gs_get<P>(V.gas, GS_Y2 * nc + c)};
  gs_store_props(V, S, g, c, gs_get<P>(V.gas, GS_EPS * nc + c), Y, gs_get<P>(V.gas, GS_T * nc + c));
}

// cell-centre gas velocity and pressure of every cell (dem_get_flow): the solved beds' faces,
// or the prescribed plug flow (0, 0, U_in / eps) and 0
template <class P>
__global__ void k_gs_flow(StepView<P> V, GasView S, int solved, double *out /* [ncells][4] */) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells) return;
  const DevBed &B = V.beds[V.cell_bed[c]];
  double *o = out + (size_t)c * 4;
  if (!solved) {
    o[0] = 0.0; o[1] = 0.0; o[2] = B.U_in / gs_get<P>(V.gas, GS_EPS * (size_t)V.ncells + c); o[3] = 0.0;
    return;
  }
  GsGrid g{&B, V.mark};
  int i, j, k;
  g.ijk(c, i, j, k);
  double u[3];
  gs_ucell(S, g, i, j, k, u);
  o[0] = u[0]; o[1] = u[1]; o[2] = u[2]; o[3] = S.pr[c];
}

}  // namespace dem
