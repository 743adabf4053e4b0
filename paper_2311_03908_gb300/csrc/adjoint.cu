// adjoint.cu -- hand-written adjoint of the frozen-position drag-heat-reaction sub-step.
//
// The map being differentiated (per parcel, positions, cells and the gas field frozen):
//   v'   = v + dt K_p (u_g - v) / m_p                      drag, eqs (3-5), (3-5-2)..(3-5-5)
//   T_p' = T_p + dt (Q_conv + Q_r + Q_rm) / sum_z m_z c_z    eqs (3-8)..(3-13), (3-18)..(3-23)
//   m_z' = max(m_z + dt mdot_z, 0)                          USCM, Sec. 2, eq (3-52)
// J = mean over parcels of f_ov(after n steps) - f_ov(now) (eqs (2-15)..(2-19)); the
// gradient is taken w.r.t. k0[3] and Ea[3] (eq (2-13)), the parameters of Sec. 5.
//
// One thread per parcel runs the whole time loop (parcels do not interact in this map):
// a forward sweep that stores a checkpoint every `ckpt` sub-steps, then, segment by segment
// from the last, a recompute of the segment that keeps every sub-step's state and forward
// intermediates in a device buffer, and the reverse sweep through them, back-propagating the
// adjoint by hand (two forward evaluations per sub-step in all, plus the reverse). The network's derivative uses the loop-matrix form:
// J = R^{-1}(x - x_eq) gives adj(R) = -(V adj(J)) J^T with V = R^{-1}.
#include "launch.cuh"

namespace dem {
namespace {

// moles of reactant per mole of H2 (Table 1): 3 Fe2O3, 1 Fe3O4, 1 FeO
__device__ __forceinline__ double nu_of(int r) { return r == 0 ? 3.0 : 1.0; }

struct Params6 { double v[6]; };              // k0[3], Ea[3]

struct Par {          // per-parcel constants of the frozen map (FP64)
  double d, k3, inv_k3, Vp, dt, uz, rho, mu, lam, eps, Tg, x, Dm, sc13, pr13, epow, D, p0;
  double cRe, aE, bE, cW, K1, K2, wlim, a1g, a2g, cB[3];
  bool ergun;
  int ore;
  unsigned flags;
};

struct Fwd {          // intermediates of one forward sub-step
  double sv[3], slip, Re, re02, re07, bo, Kp, mp, Nu, hA, Qc;
  double n[4], nfe, om[3], invT, K[3], xeq[3], kr[3], c3[3], g[3];
  bool act[3], fin[3], hasB[3];
  double Bm, Bw, BFe, Sh, F, J[3], V[3][3], c;
  int lim[3];         // 0: rate = c J, 1: capped by the reactant, 2: zero
  double xid[3], mdot[4], tot, Qx, C;
  bool clampm[4];
};

static_assert(sizeof(Fwd) % 8 == 0, "forward intermediates are stored as 8-byte words");
constexpr int kFwdWords = (int)(sizeof(Fwd) / 8);
constexpr int kSegWords = 8 + kFwdWords;   // per parcel and sub-step of a recomputed segment

__device__ inline double cz_mass(int s, double T, double M) { return cp_over_R<double>(s, T) * kRgas / M; }


__device__ void fwd(const Par &P, const double s[8], const double th[6], Fwd &F, double sn[8]) {
  const Tab<double> &td = tab<double>();
  const unsigned fl = P.flags;
  const double v[3] = {s[0], s[1], s[2]};
  const double T = s[3];
  const double *m = s + 4;
  // drag
  F.sv[0] = -v[0]; F.sv[1] = -v[1]; F.sv[2] = P.uz - v[2];
  F.slip = sqrt(F.sv[0] * F.sv[0] + F.sv[1] * F.sv[1] + F.sv[2] * F.sv[2]);
  F.Re = P.cRe * F.slip;
  F.re02 = F.Re > 0.0 ? exp(0.2 * log(F.Re)) : 0.0;
  F.re07 = F.re02 * sqrt(F.Re);
  if (P.ergun) {
    F.bo = P.aE + P.bE * F.slip;
  } else if (F.Re > 0.0) {
    const double RK = F.Re * (P.K1 * P.K2);
    const double CD = 24.0 / (F.Re * P.K1) * (1.0 + 0.1118 * exp(0.6567 * log(RK))) + 0.4305 * P.K2 / (1.0 + 3305.0 / RK);
    F.bo = P.cW * CD * F.slip;
  } else {
    F.bo = P.wlim;
  }
  F.Kp = (fl & DEM_NO_DRAG) ? 0.0 : F.bo * P.Vp;
  F.mp = m[0] + m[1] + m[2] + m[3];
  for (int q = 0; q < 3; ++q) sn[q] = v[q] + P.dt * F.Kp * F.sv[q] / F.mp;
  // convection
  F.Nu = P.a1g * (1.0 + 0.7 * F.re02 * P.pr13) + P.a2g * F.re07 * P.pr13;
  F.hA = (fl & DEM_NO_HEAT) ? 0.0 : P.k3 * kPI * P.d * P.lam * F.Nu;
  F.Qc = F.hA * (P.Tg - T);
  // kinetics (the same arithmetic as uscm<double>)
  for (int z = 0; z < 4; ++z) F.n[z] = m[z] * P.inv_k3 / td.Mz[z];
  F.nfe = 2.0 * F.n[0] + 3.0 * F.n[1] + F.n[2] + F.n[3];
  for (int r = 0; r < 3; ++r) { F.xid[r] = 0.0; F.J[r] = 0.0; F.g[r] = 0.0; F.act[r] = F.fin[r] = F.hasB[r] = false; F.lim[r] = 2; }
  for (int z = 0; z < 4; ++z) F.mdot[z] = 0.0;
  F.tot = F.Qx = 0.0;
  F.Bm = F.Bw = F.BFe = F.Sh = F.F = F.c = 0.0;
  F.invT = 1.0 / T;
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) F.V[i][j] = 0.0;
  const bool alive = F.nfe > 0.0;
  if (alive) {
    const double inv_nfe = 1.0 / F.nfe;
    F.om[0] = 2.0 * F.n[0] * inv_nfe;
    F.om[1] = (2.0 * F.n[0] + 3.0 * F.n[1]) * inv_nfe;
    F.om[2] = (2.0 * F.n[0] + 3.0 * F.n[1] + F.n[2]) * inv_nfe;
    const bool kin = !(fl & DEM_NO_KINETICS);
    for (int r = 0; r < 3; ++r) {
      F.K[r] = exp(td.Ka[r] * F.invT + td.Kb[r]);
      F.xeq[r] = 1.0 / (F.K[r] + 1.0);
      F.kr[r] = th[r] * exp(-(th[3 + r] / kRgas) * F.invT);
      F.c3[r] = cbrt(F.om[r]);
      F.act[r] = kin && F.n[r] > 0.0 && P.x > F.xeq[r] && th[r] > 0.0;
      F.g[r] = F.act[r] ? F.kr[r] * F.c3[r] * F.c3[r] * (1.0 + 1.0 / F.K[r]) : 0.0;
    }
    if (!(fl & DEM_NO_LAYER)) {
      if (F.act[0]) { F.hasB[0] = true; F.Bm = P.cB[0] * (1.0 / F.c3[0] - 1.0 / F.c3[1]); }
      if ((F.act[0] || F.act[1]) && F.om[1] > 0.0) { F.hasB[1] = true; F.Bw = P.cB[1] * (1.0 / F.c3[1] - 1.0 / F.c3[2]); }
      if (F.om[2] > 0.0) { F.hasB[2] = true; F.BFe = P.cB[2] * (1.0 / F.c3[2] - 1.0); }
    }
    F.Sh = P.a1g * (1.0 + 0.7 * F.re02 * P.sc13) + P.a2g * F.re07 * P.sc13;
    F.F = (fl & DEM_NO_FILM) ? 0.0 : P.d / (F.Sh * P.Dm);
    double gk[3] = {F.g[0], F.g[1], F.g[2]};
    const double S = F.F + F.BFe, BwS = F.Bw + S;
    for (int it = 0; it < 3; ++it) {
      const double g1 = gk[0], g2 = gk[1], g3 = gk[2];
      const double a1 = 1.0 + F.Bm * g1;
      const double W = a1 * (1.0 + BwS * g2 + S * g3 * (1.0 + F.Bw * g2)) + g1 * (BwS + F.Bw * S * g3);
      const double iW = 1.0 / W;
      F.V[0][0] = g1 * ((1.0 + BwS * g2) + S * g3 * (1.0 + F.Bw * g2)) * iW;
      F.V[0][1] = F.V[1][0] = -g1 * g2 * (BwS + F.Bw * S * g3) * iW;
      F.V[0][2] = F.V[2][0] = -S * g1 * g3 * iW;
      F.V[1][1] = g2 * ((1.0 + (F.Bm + F.Bw) * g1) * (1.0 + S * g3) + S * g1) * iW;
      F.V[1][2] = F.V[2][1] = -S * g2 * g3 * a1 * iW;
      F.V[2][2] = g3 * (a1 * (1.0 + BwS * g2) + BwS * g1) * iW;
      const double dd[3] = {P.x - F.xeq[0], P.x - F.xeq[1], P.x - F.xeq[2]};
      for (int r = 0; r < 3; ++r) F.J[r] = F.V[r][0] * dd[0] + F.V[r][1] * dd[1] + F.V[r][2] * dd[2];
      bool neg = false;
      for (int r = 0; r < 3; ++r)
        if (gk[r] > 0.0 && F.J[r] < 0.0) { gk[r] = 0.0; neg = true; }
      if (!neg) break;
    }
    for (int r = 0; r < 3; ++r) F.fin[r] = gk[r] > 0.0;
    F.c = kPI * P.d * P.d * P.p0 * F.invT / kRgas;
    for (int r = 0; r < 3; ++r) {
      // the reactant limiter of uscm: min(c J, n / (nu dt)), then not below zero
      const double x0 = F.fin[r] ? F.c * F.J[r] : 0.0;
      const double cap = F.n[r] / nu_of(r) / P.dt;
      const double xr = x0 < cap ? x0 : cap;
      F.xid[r] = xr > 0.0 ? xr : 0.0;
      F.lim[r] = !(xr > 0.0) ? 2 : (x0 < cap ? 0 : 1);
    }
    const double k3 = P.k3;
    F.mdot[0] = -3.0 * F.xid[0] * td.Mz[0] * k3;
    F.mdot[1] = (2.0 * F.xid[0] - F.xid[1]) * td.Mz[1] * k3;
    F.mdot[2] = (3.0 * F.xid[1] - F.xid[2]) * td.Mz[2] * k3;
    F.mdot[3] = F.xid[2] * td.Mz[3] * k3;
    F.tot = F.xid[0] + F.xid[1] + F.xid[2];
    if (!(fl & DEM_NO_RXN_HEAT)) {
      double q = 0.0;
      for (int z = 0; z < 4; ++z) q += h_over_R<double>(3 + z, T) * kRgas * F.mdot[z] / td.Mz[z];
      F.Qx = -q + F.tot * k3 * kRgas * (h_over_R<double>(0, T) - h_over_R<double>(1, T));
    }
  }
  // temperature
  F.C = 0.0;
  for (int z = 0; z < 4; ++z) F.C += m[z] * cz_mass(3 + z, T, td.Mz[z]);
  sn[3] = T + P.dt * (F.Qc + F.Qx) / F.C;
  // masses
  for (int z = 0; z < 4; ++z) {
    const double mn = m[z] + P.dt * F.mdot[z];
    F.clampm[z] = !(mn >= 0.0);
    sn[4 + z] = F.clampm[z] ? 0.0 : mn;
  }
}

// Reverse of fwd: given the adjoint ln of the outputs, write the adjoint l of the inputs
// and add this step's contribution to the parameter gradient g (k0[3], Ea[3]).
__device__ void bwd(const Par &P, const double s[8], const double th[6], const Fwd &F, const double ln[8],
                    double l[8], double g[6]) {
  const Tab<double> &td = tab<double>();
  const unsigned fl = P.flags;
  const double T = s[3];
  const double *m = s + 4;
  double lv[3] = {ln[0], ln[1], ln[2]};
  double lT = ln[3];
  double lm[4], lmdot[4];
  for (int z = 0; z < 4; ++z) {
    lm[z] = F.clampm[z] ? 0.0 : ln[4 + z];
    lmdot[z] = F.clampm[z] ? 0.0 : ln[4 + z] * P.dt;
  }
  // T' = T + dt (Qc + Qx) / C
  const double lQ = ln[3] * P.dt / F.C;
  const double lC = -ln[3] * P.dt * (F.Qc + F.Qx) / (F.C * F.C);
  double dC = 0.0;
  for (int z = 0; z < 4; ++z) {
    lm[z] += lC * cz_mass(3 + z, T, td.Mz[z]);
    dC += m[z] * dcp_over_R<double>(3 + z, T) * kRgas / td.Mz[z];
  }
  lT += lC * dC;
  // v' = v + dt Kp sv / mp
  double vsv = ln[0] * F.sv[0] + ln[1] * F.sv[1] + ln[2] * F.sv[2];
  const double lKp = P.dt * vsv / F.mp;
  double lsv[3] = {P.dt * F.Kp * ln[0] / F.mp, P.dt * F.Kp * ln[1] / F.mp, P.dt * F.Kp * ln[2] / F.mp};
  const double lmp = -P.dt * F.Kp * vsv / (F.mp * F.mp);
  for (int z = 0; z < 4; ++z) lm[z] += lmp;
  // Qc = hA (Tg - T), hA = k3 pi d lam Nu
  double lRe = 0.0;
  if (!(fl & DEM_NO_HEAT)) {
    lT += -lQ * F.hA;
    const double lNu = lQ * (P.Tg - T) * P.k3 * kPI * P.d * P.lam;
    if (F.Re > 0.0) lRe += lNu * (P.a1g * 0.7 * P.pr13 * 0.2 * F.re02 + P.a2g * P.pr13 * 0.7 * F.re07) / F.Re;
  }
  double ln_[4] = {0, 0, 0, 0};
  double linvT = 0.0;
  if (F.nfe > 0.0) {
    const double k3 = P.k3;
    double ltot = 0.0;
    if (!(fl & DEM_NO_RXN_HEAT)) {
      // Qx = -sum_z R h_z mdot_z / M_z + tot k3 R (h_H2 - h_H2O)
      double dQ = 0.0;
      for (int z = 0; z < 4; ++z) {
        lmdot[z] += -lQ * h_over_R<double>(3 + z, T) * kRgas / td.Mz[z];
        dQ += -cp_over_R<double>(3 + z, T) * kRgas * F.mdot[z] / td.Mz[z];
      }
      ltot = lQ * k3 * kRgas * (h_over_R<double>(0, T) - h_over_R<double>(1, T));
      dQ += F.tot * k3 * kRgas * (cp_over_R<double>(0, T) - cp_over_R<double>(1, T));
      lT += lQ * dQ;
    }
    double lx[3];
    lx[0] = k3 * (-3.0 * td.Mz[0] * lmdot[0] + 2.0 * td.Mz[1] * lmdot[1]) + ltot;
    lx[1] = k3 * (-td.Mz[1] * lmdot[1] + 3.0 * td.Mz[2] * lmdot[2]) + ltot;
    lx[2] = k3 * (-td.Mz[2] * lmdot[2] + td.Mz[3] * lmdot[3]) + ltot;
    double lJ[3] = {0, 0, 0}, lc = 0.0;
    for (int r = 0; r < 3; ++r) {
      if (F.lim[r] == 0) { lc += lx[r] * F.J[r]; lJ[r] = lx[r] * F.c; }
      else if (F.lim[r] == 1) ln_[r] += lx[r] / (nu_of(r) * P.dt);
    }
    linvT += lc * F.c / F.invT;
    // network on the final active set: J = V (x - xeq)
    double ld[3];
    for (int i = 0; i < 3; ++i) ld[i] = F.V[i][0] * lJ[0] + F.V[i][1] * lJ[1] + F.V[i][2] * lJ[2];
    double lxeq[3] = {-ld[0], -ld[1], -ld[2]};
    double LR[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) LR[i][j] = -ld[i] * F.J[j];
    double lA[3] = {LR[0][0], LR[1][1], LR[2][2]};
    const double lBm = LR[0][0];
    const double lBw = LR[0][0] + LR[1][1] + LR[0][1] + LR[1][0];
    double lS = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) lS += LR[i][j];
    double lg[3] = {0, 0, 0};
    for (int r = 0; r < 3; ++r)
      if (F.fin[r]) lg[r] = -lA[r] / (F.g[r] * F.g[r]);
    const double lF = (fl & DEM_NO_FILM) ? 0.0 : lS;
    const double lBFe = lS;
    // F = d / (Sh Dm), Sh = Gunn(Re)
    if (!(fl & DEM_NO_FILM) && F.Re > 0.0) {
      const double lSh = -lF * F.F / F.Sh;
      lRe += lSh * (P.a1g * 0.7 * P.sc13 * 0.2 * F.re02 + P.a2g * P.sc13 * 0.7 * F.re07) / F.Re;
    }
    double lc3[3] = {0, 0, 0};
    if (F.hasB[0]) { lc3[0] += -lBm * P.cB[0] / (F.c3[0] * F.c3[0]); lc3[1] += lBm * P.cB[0] / (F.c3[1] * F.c3[1]); }
    if (F.hasB[1]) { lc3[1] += -lBw * P.cB[1] / (F.c3[1] * F.c3[1]); lc3[2] += lBw * P.cB[1] / (F.c3[2] * F.c3[2]); }
    if (F.hasB[2]) { lc3[2] += -lBFe * P.cB[2] / (F.c3[2] * F.c3[2]); }
    double lK[3] = {0, 0, 0};
    for (int r = 0; r < 3; ++r) {
      if (F.act[r]) {
        const double q = 1.0 + 1.0 / F.K[r];
        const double lkr = lg[r] * F.c3[r] * F.c3[r] * q;
        lc3[r] += lg[r] * F.kr[r] * 2.0 * F.c3[r] * q;
        lK[r] += lg[r] * F.kr[r] * F.c3[r] * F.c3[r] * (-1.0 / (F.K[r] * F.K[r]));
        // kr = k0 exp(-Ea invT / R)
        g[r] += lkr * F.kr[r] / th[r];
        g[3 + r] += lkr * (-F.kr[r] * F.invT / kRgas);
        linvT += lkr * (-F.kr[r] * th[3 + r] / kRgas);
      }
      lK[r] += lxeq[r] * (-1.0 / ((F.K[r] + 1.0) * (F.K[r] + 1.0)));
      linvT += lK[r] * F.K[r] * td.Ka[r];
    }
    // c3 = cbrt(om); om = u / nfe
    double lom[3];
    for (int r = 0; r < 3; ++r) lom[r] = F.om[r] > 0.0 ? lc3[r] * F.c3[r] / (3.0 * F.om[r]) : 0.0;
    const double du[3][4] = {{2, 0, 0, 0}, {2, 3, 0, 0}, {2, 3, 1, 0}};
    const double dnfe[4] = {2, 3, 1, 1};
    for (int r = 0; r < 3; ++r)
      for (int z = 0; z < 4; ++z) ln_[z] += lom[r] * (du[r][z] - F.om[r] * dnfe[z]) / F.nfe;
    for (int z = 0; z < 4; ++z) lm[z] += ln_[z] * P.inv_k3 / td.Mz[z];
  }
  lT += -linvT * F.invT * F.invT;
  // drag: Kp = bo Vp; bo(slip) with Re = cRe slip; Nu and Sh contributions arrive via lRe
  double lslip = lRe * P.cRe;
  if (!(fl & DEM_NO_DRAG)) {
    const double lbo = lKp * P.Vp;
    double dbo = 0.0;
    if (P.ergun) dbo = P.bE;
    else if (F.Re > 0.0) {
      const double RK = F.Re * (P.K1 * P.K2);
      const double P1 = exp(0.6567 * log(RK));
      const double q = RK + 3305.0;
      dbo = P.cW * (24.0 * 0.1118 * (1.0 - 0.3433) * P1 / (P.K1 * F.Re) + 0.4305 * P.K2 * RK / q +
                    0.4305 * P.K2 * 3305.0 * RK / (q * q));
    }
    lslip += lbo * dbo;
  }
  if (F.slip > 0.0)
    for (int q = 0; q < 3; ++q) lsv[q] += lslip * F.sv[q] / F.slip;
  for (int q = 0; q < 3; ++q) lv[q] += -lsv[q];
  for (int q = 0; q < 3; ++q) l[q] = lv[q];
  l[3] = lT;
  for (int z = 0; z < 4; ++z) l[4 + z] = lm[z];
}

__device__ double fov(const double *m, int ore) {
  const Tab<double> &td = tab<double>();
  const double n0 = m[0] / td.Mz[0], n1 = m[1] / td.Mz[1], n2 = m[2] / td.Mz[2], n3 = m[3] / td.Mz[3];
  const double nfe = 2.0 * n0 + 3.0 * n1 + n2 + n3;
  if (!(nfe > 0.0)) return 0.0;
  const double fh = (3.0 * n1 + n2 + n3) / nfe, fm = (n2 + n3) / nfe, fw = n3 / nfe;
  return ore == 0 ? fh / 9.0 + 2.0 * fm / 9.0 + 6.0 * fw / 9.0 : 0.25 * fm + 0.75 * fw;
}

__device__ void dfov_dm(const double *m, int ore, double out[4]) {
  const Tab<double> &td = tab<double>();
  double n[4];
  for (int z = 0; z < 4; ++z) n[z] = m[z] / td.Mz[z];
  const double nfe = 2.0 * n[0] + 3.0 * n[1] + n[2] + n[3];
  for (int z = 0; z < 4; ++z) out[z] = 0.0;
  if (!(nfe > 0.0)) return;
  const double w[3] = {ore == 0 ? 1.0 / 9.0 : 0.0, ore == 0 ? 2.0 / 9.0 : 0.25, ore == 0 ? 6.0 / 9.0 : 0.75};
  const double du[3][4] = {{0, 3, 1, 1}, {0, 0, 1, 1}, {0, 0, 0, 1}};
  const double dnfe[4] = {2, 3, 1, 1};
  const double f = fov(m, ore);
  for (int z = 0; z < 4; ++z) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += w[k] * du[k][z];
    out[z] = (s - f * dnfe[z]) / nfe / td.Mz[z];
  }
}

template <class Pp>
__device__ void load_par(const StepView<Pp> &V, const BedP<double> *bpd, int i, Par &P, double s[8]) {
  const int meta = V.A.meta[i];
  const BedP<double> &B = bpd[meta >> 8];
  P.ore = meta & 255;
  P.flags = B.flags;
  P.d = (double)V.A.d[i];
  P.k3 = B.k3;
  P.inv_k3 = B.inv_k3;
  const double dc = B.k * P.d;
  P.Vp = kPI / 6.0 * dc * dc * dc;
  P.dt = B.dt;
  P.p0 = B.p0;
  const size_t nc = (size_t)V.ncells;
  const unsigned c = V.keyp[i];   // the parcel's gas cell (storage order)
  const double *G = V.gas;
  const double Y[3] = {gas_d<Pp>(G, GS_Y0 * nc + c), gas_d<Pp>(G, GS_Y1 * nc + c), gas_d<Pp>(G, GS_Y2 * nc + c)};
  const CellProps<double> cp = gas_cell_props<double>(B, gas_d<Pp>(G, GS_EPS * nc + c), Y, gas_d<Pp>(G, GS_T * nc + c));
  P.rho = cp.rho; P.mu = cp.mu; P.lam = cp.lam; P.eps = cp.eps; P.Tg = cp.T; P.x = cp.x; P.Dm = cp.Dm;
  P.sc13 = cp.sc13; P.pr13 = cp.pr13; P.epow = cp.epow; P.D = cp.D[P.ore]; P.uz = cp.uz;
  P.cRe = P.rho * P.eps * P.d / P.mu;
  const double ep = 1.0 - P.eps, psi = B.psi[P.ore];
  P.ergun = P.eps < 0.8;
  P.aE = 150.0 * ep * P.mu / (P.eps * P.d * P.d * psi * psi);
  P.bE = 1.75 * P.rho / (P.d * psi);
  P.K1 = B.K1b[P.ore] - B.wall_K1 * P.d;
  P.K2 = B.K2[P.ore];
  P.cW = 0.75 * P.eps * P.rho / P.d * P.epow;
  P.wlim = 0.75 * (24.0 / P.K1) * P.mu / (P.d * P.d) * P.epow;
  P.a1g = 7.0 - 10.0 * P.eps + 5.0 * P.eps * P.eps;
  P.a2g = 1.33 - 2.4 * P.eps + 1.2 * P.eps * P.eps;
  const double rp = 0.5 * P.d;
  for (int l = 0; l < 3; ++l) P.cB[l] = rp / (P.D * B.xi[P.ore][l] * B.inv_tau);
  for (int q = 0; q < 3; ++q)   // the whole-step velocity (the state holds the half-step one)
    s[q] = (double)half_kick_back(V.bp[meta >> 8].half_dt, B.dt, V.A.v[q][i], V.A.a[q][i]);
  s[3] = (double)V.A.T[i];
  for (int z = 0; z < 4; ++z) s[4 + z] = mass_d<Pp>(V.A.m[z], i);
}

// Observations of the reduction-degree curve (dem_adjoint_obs): after steps[k] sub-steps
// every parcel's f_ov - f_ov(0) goes to f[k][i], and the differentiated quantity is
// sum_k sum_i coef[k][bed of i] (f_ov,i(steps[k]) - f_ov,i(0)). nobs = 0: the plain J.
struct Obs {
  int nobs;
  const int *steps;       // ascending, in [1, nsteps]
  const double *coef;     // [nobs][nbeds]
  double *f;              // [nobs][n]
};

__device__ __forceinline__ void add_dfov(const double *m, int ore, double c, double lam[8]) {
  double d[4];
  dfov_dm(m, ore, d);
  for (int z = 0; z < 4; ++z) lam[4 + z] += c * d[z];
}

// grad == false: forward sweep only (J). partial: [grid][7] = J sum, then 6 gradient sums.
template <class Pp>
__global__ void __launch_bounds__(128) k_adjoint(StepView<Pp> V, const BedP<double> *bpd, int nsteps, int ckpt,
                                                 Params6 th6, double *cks, double *seg, bool grad, double *partial,
                                                 Obs ob) {
  __shared__ double sh[7][128];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  if (i < V.n) {
    Par P;
    double s[8], sn[8];
    load_par(V, bpd, i, P, s);
    const double *th = th6.v;
    const int ore = P.ore;
    const double f0 = fov(s + 4, ore);
    Fwd F;
    const size_t n = (size_t)V.n;
    const int bed = V.A.meta[i] >> 8;
    int oi = 0;
    for (int st = 0; st < nsteps; ++st) {
      if (grad && st % ckpt == 0)
        for (int q = 0; q < 8; ++q) cks[((size_t)(st / ckpt) * 8 + q) * n + i] = s[q];
      fwd(P, s, th, F, sn);
      for (int q = 0; q < 8; ++q) s[q] = sn[q];
      if (oi < ob.nobs && st + 1 == ob.steps[oi]) ob.f[(size_t)(oi++) * n + i] = fov(s + 4, ore) - f0;
    }
    acc[0] = fov(s + 4, ore) - f0;
    if (grad) {
      double lam[8] = {0, 0, 0, 0, 0, 0, 0, 0}, lout[8], g[6] = {0, 0, 0, 0, 0, 0};
      // the seed at the end of the horizon: the plain J, or the observation taken there
      oi = ob.nobs - 1;
      if (ob.nobs == 0) dfov_dm(s + 4, ore, lam + 4);
      else if (ob.steps[oi] == nsteps) add_dfov(s + 4, ore, ob.coef[(size_t)(oi--) * V.nbeds + bed], lam);
      const int nseg = (nsteps + ckpt - 1) / ckpt;
      for (int sg = nseg - 1; sg >= 0; --sg) {
        const int st0 = sg * ckpt, st1 = min(st0 + ckpt, nsteps);
        for (int q = 0; q < 8; ++q) s[q] = cks[((size_t)sg * 8 + q) * n + i];
        // recompute the segment, keeping each sub-step's state and forward intermediates
        for (int k = st0; k < st1; ++k) {
          double *slot = seg + (size_t)(k - st0) * kSegWords * n + i;
          for (int q = 0; q < 8; ++q) slot[(size_t)q * n] = s[q];
          fwd(P, s, th, F, sn);
          const unsigned long long *fw = reinterpret_cast<const unsigned long long *>(&F);
          unsigned long long *sw = reinterpret_cast<unsigned long long *>(slot + 8 * n);
          for (int q = 0; q < kFwdWords; ++q) sw[(size_t)q * n] = fw[q];
          for (int q = 0; q < 8; ++q) s[q] = sn[q];
        }
        for (int k = st1 - 1; k >= st0; --k) {
          // an observation of the state after sub-step k (k + 1 < nsteps): the adjoint of
          // that state takes its weight before the reverse of sub-step k
          if (oi >= 0 && ob.steps[oi] == k + 1) {
            const double *sk1 = k + 1 < st1 ? seg + (size_t)(k + 1 - st0) * kSegWords * n + i
                                            : cks + (size_t)(sg + 1) * 8 * n + i;
            double m1[4];
            for (int z = 0; z < 4; ++z) m1[z] = sk1[(size_t)(4 + z) * n];
            add_dfov(m1, ore, ob.coef[(size_t)(oi--) * V.nbeds + bed], lam);
          }
          const double *slot = seg + (size_t)(k - st0) * kSegWords * n + i;
          for (int q = 0; q < 8; ++q) s[q] = slot[(size_t)q * n];
          unsigned long long *fw = reinterpret_cast<unsigned long long *>(&F);
          const unsigned long long *sw = reinterpret_cast<const unsigned long long *>(slot + 8 * n);
          for (int q = 0; q < kFwdWords; ++q) fw[q] = sw[(size_t)q * n];
          bwd(P, s, th, F, lam, lout, g);
          for (int q = 0; q < 8; ++q) lam[q] = lout[q];
        }
      }
      for (int q = 0; q < 6; ++q) acc[1 + q] = g[q];
    }
  }
  for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off)
      for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x < 7) partial[(size_t)blockIdx.x * 7 + threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

template <class Pp>
int run_adjoint(dem_ctx *c, int nsteps, int ckpt, double *J, double *grad, int nobs, const int *obs_steps,
                const double *weights, double *J_obs) {
  const bool want_grad = grad != nullptr;
  const int n = c->n;
  const int nseg = (nsteps + ckpt - 1) / ckpt;
  const int bs = 128, grid = (n + bs - 1) / bs;
  const size_t obs_words = nobs > 0 ? (size_t)nobs * n + (size_t)nobs * c->nbeds + (size_t)nobs + 1 : 0;
  const size_t need = sizeof(double) * ((want_grad ? ((size_t)nseg * 8 * n + (size_t)ckpt * kSegWords * n) : 0) +
                                        (size_t)grid * 7 + obs_words);
  if (c->adj_bytes < need) {
    if (c->adj) cudaFree(c->adj);
    c->adj = nullptr;
    c->adj_bytes = 0;
    if (cudaMalloc(&c->adj, need) != cudaSuccess) return DEM_ENOMEM;
    c->adj_bytes = need;
  }
  double *cks = c->adj;
  double *seg = cks + (want_grad ? (size_t)nseg * 8 * n : 0);
  double *partial = seg + (want_grad ? (size_t)ckpt * kSegWords * n : 0);
  Obs ob{0, nullptr, nullptr, nullptr};
  std::vector<double> hcoef;
  std::vector<int> hcount(c->nbeds, 0);
  if (nobs > 0) {
    // coefficients per (observation, bed): the weight over the bed's parcel count, so that
    // the kernel's per-parcel seeds sum to the weighted bed means
    for (int b = 0; b < c->nbeds; ++b) hcount[b] = c->hbeds[b].pend - c->hbeds[b].pstart;
    hcoef.assign((size_t)nobs * c->nbeds, 0.0);
    for (int k = 0; k < nobs; ++k)
      for (int b = 0; b < c->nbeds; ++b)
        hcoef[(size_t)k * c->nbeds + b] =
            weights && hcount[b] > 0 ? weights[(size_t)k * c->nbeds + b] / hcount[b] : 0.0;
    double *of = partial + (size_t)grid * 7;
    double *oc = of + (size_t)nobs * n;
    int *os = reinterpret_cast<int *>(oc + (size_t)nobs * c->nbeds);
    if (cudaMemcpyAsync(oc, hcoef.data(), sizeof(double) * hcoef.size(), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(os, obs_steps, sizeof(int) * nobs, cudaMemcpyHostToDevice, c->st) != cudaSuccess)
      return DEM_ECUDA;
    ob = Obs{nobs, os, oc, of};
  }
  StepView<Pp> V = make_view<Pp>(c, false);
  Params6 th;
  for (int r = 0; r < 3; ++r) { th.v[r] = c->cfg[0].k0[r]; th.v[3 + r] = c->cfg[0].Ea[r]; }
  k_adjoint<Pp><<<grid, bs, 0, c->st>>>(V, c->dbp_d, nsteps, ckpt, th, cks, seg, want_grad, partial, ob);
  if (cudaPeekAtLastError() != cudaSuccess) return DEM_ECUDA;

  std::vector<double> h((size_t)grid * 7);
  if (cudaMemcpyAsync(h.data(), partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
    return DEM_ECUDA;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return DEM_ECUDA;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < grid; ++b)
    for (int q = 0; q < 7; ++q) acc[q] += h[(size_t)b * 7 + q];
  if (J) *J = acc[0] / n;
  if (want_grad)
    for (int q = 0; q < 6; ++q) grad[q] = nobs > 0 ? acc[1 + q] : acc[1 + q] / n;
  if (nobs > 0) {
    // the observed bed means: per-parcel values back to the host, summed bed by bed in
    // storage order (each bed's parcels occupy a fixed storage range)
    std::vector<double> hf((size_t)nobs * n);
    if (cudaMemcpy(hf.data(), partial + (size_t)grid * 7, sizeof(double) * hf.size(), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return DEM_ECUDA;
    for (int k = 0; k < nobs; ++k)
      for (int b = 0; b < c->nbeds; ++b) {
        double sum = 0.0;
        for (int i = c->hbeds[b].pstart; i < c->hbeds[b].pend; ++i) sum += hf[(size_t)k * n + i];
        J_obs[(size_t)k * c->nbeds + b] = hcount[b] > 0 ? sum / hcount[b] : 0.0;
      }
  }
  return DEM_OK;
}

template int run_adjoint<PrecF64>(dem_ctx *, int, int, double *, double *, int, const int *, const double *, double *);
template int run_adjoint<PrecSplit>(dem_ctx *, int, int, double *, double *, int, const int *, const double *, double *);
template int run_adjoint<PrecKahan>(dem_ctx *, int, int, double *, double *, int, const int *, const double *, double *);

}  // namespace dem
