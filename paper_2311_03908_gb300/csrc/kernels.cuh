// kernels.cuh -- the per-step kernels of the particle path, templated on the precision
// policy P (PrecF64, PrecSplit, PrecKahan; see common.cuh). Instantiated in inst_*.cu,
// launched by launch.cuh.
#pragma once
#include "common.cuh"

namespace dem {

// One parcel-state buffer, structure of arrays in the current sorted order.
template <class R> struct PState {
  double *x, *y, *z;
  R *v[3], *w[3], *a[3], *al[3], *T, *d;
  double *m[4];  // FP64 masses, or (value, compensation) FP32 pairs in the split-Kahan form
  int *meta;     // bed << 8 | ore
  int *orig;     // parcel index (input order)
};

// Contact-history table: count per parcel, then KMAX slots of partner index and 3-vector.
template <class R> struct Hist {
  unsigned char *cnt;
  int *id;     // [KMAX][cap]
  R *xi;       // [KMAX*3][cap]
};

// Everything a step's kernels touch.
template <class P> struct StepView {
  using R = typename P::R;
  int n, cap, nbeds;
  long long ncells;
  const DevBed *beds;
  const BedP<R> *bp;
  PState<R> A, B;               // A: state before the step, B: gather target
  Hist<R> H, Hn;                // H: current history, Hn: gather target
  unsigned *keys, *vals;        // sorted keys (global gas cell) and the permutation
  unsigned *cstart, *cend;      // parcel range of every gas cell (empty: 0, 0)
  float4 *xl;                   // FP32 position relative to the own cell's corner, radius
  R *mass;                      // parcel mass (new order)
  R *F[3], *Tq[3];              // contact force and torque
  R *src;                       // [SR_N][cap] per-parcel cell sources
  double *gas, *gas_new;        // [GS_N][ncells]
  R *gp;                        // [GP_N][ncells]
  unsigned char *mark;          // solid (IBM) cell mark
  int *cell_bed;                // bed of each gas cell
  double *diag;                 // [DG_N][cap] or null
  double *dep;                  // [ncells][SR_N] or null (written by k_sources)
  int *err;
  const long long *step_ctr;    // steps completed so far (device)
};

__device__ __forceinline__ bool coupled_step(int ncouple, const long long *ctr) {
  return ncouple == 1 || (((int)(*ctr % ncouple)) + 1) % ncouple == 0;
}

// ---------------------------------------------------------------------------------------
// half kick and drift of velocity Verlet (kick-drift-kick). The key kernel and the gather
// kernel both call this, so the new positions they see are the same bits.
// ---------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void kick_drift(R half_dt, R dt, double dt_d, double &x, R &v, R a) {
  if constexpr (sizeof(R) == 8) {
    const double vh = __dadd_rn((double)v, __dmul_rn((double)a, 0.5 * dt_d));
    x = __dadd_rn(x, __dmul_rn(vh, dt_d));
    v = (R)vh;
  } else {
    v = v + a * half_dt;
    x = x + (double)(v * dt);
  }
}

// Gas cell of a point: floor((x - x0) * (1/dx)) clamped, in FP64. The FP32 forms first try
// FP32 and fall back to FP64 only within 1e-3 of a cell face, so both agree.
__device__ __forceinline__ int cell_coord_d(double x, double x0, double inv, int n, bool &out) {
  const double f = floor((x - x0) * inv);
  if (!(f >= 0.0 && f < (double)n)) out = true;
  return (int)fmin(fmax(f, 0.0), (double)(n - 1));
}
template <class P>
__device__ __forceinline__ int cell_coord(double x, double x0, double inv, float x0f, float invf, int n, bool &out) {
  if constexpr (!P::exact) {
    const float u = ((float)x - x0f) * invf;
    const float fl = floorf(u);
    if (u - fl > 1e-3f && u - fl < 1.0f - 1e-3f && fl >= 0.0f && fl < (float)n) return (int)fl;
  }
  return cell_coord_d(x, x0, inv, n, out);
}

template <class P>
__device__ __forceinline__ unsigned point_key(const DevBed &B, const BedP<typename P::R> &bp, double x,
                                              double y, double z, bool &out) {
  out = false;
  const int ix = cell_coord<P>(x, B.x0, B.inv_dx, (float)bp.x0, (float)bp.inv_dx, B.nx, out);
  const int iy = cell_coord<P>(y, B.y0, B.inv_dy, (float)bp.y0, (float)bp.inv_dy, B.ny, out);
  const int iz = cell_coord<P>(z, B.z0, B.inv_dz, (float)bp.z0, (float)bp.inv_dz, B.nz, out);
  return (unsigned)(B.cell_off + ((long long)iz * B.ny + iy) * B.nx + ix);
}

template <class P>
__global__ void k_key(StepView<P> V, int drift) {
  using R = typename P::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int b = V.A.meta[i] >> 8;
  const DevBed &B = V.beds[b];
  const BedP<R> &bp = V.bp[b];
  double x = V.A.x[i], y = V.A.y[i], z = V.A.z[i];
  if (drift) {
    R vx = V.A.v[0][i], vy = V.A.v[1][i], vz = V.A.v[2][i];
    kick_drift<R>(bp.half_dt, bp.dt, B.dt, x, vx, V.A.a[0][i]);
    kick_drift<R>(bp.half_dt, bp.dt, B.dt, y, vy, V.A.a[1][i]);
    kick_drift<R>(bp.half_dt, bp.dt, B.dt, z, vz, V.A.a[2][i]);
  }
  bool out;
  V.keys[i] = point_key<P>(B, bp, x, y, z, out);
  V.vals[i] = (unsigned)i;
  if (out) set_error(V.err, ERR_DOMAIN);
}

// Gather the state into the sorted order, applying the half kick and drift; record the
// cell ranges by boundary detection on the sorted keys; copy the history slots.
template <class P>
__global__ void k_gather(StepView<P> V, int drift) {
  using R = typename P::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int j = (int)V.vals[i];
  const int meta = V.A.meta[j];
  const DevBed &B = V.beds[meta >> 8];
  const BedP<R> &bp = V.bp[meta >> 8];
  double x = V.A.x[j], y = V.A.y[j], z = V.A.z[j];
  R v[3] = {V.A.v[0][j], V.A.v[1][j], V.A.v[2][j]};
  R w[3] = {V.A.w[0][j], V.A.w[1][j], V.A.w[2][j]};
  R a[3] = {V.A.a[0][j], V.A.a[1][j], V.A.a[2][j]};
  R al[3] = {V.A.al[0][j], V.A.al[1][j], V.A.al[2][j]};
  if (drift) {
    kick_drift<R>(bp.half_dt, bp.dt, B.dt, x, v[0], a[0]);
    kick_drift<R>(bp.half_dt, bp.dt, B.dt, y, v[1], a[1]);
    kick_drift<R>(bp.half_dt, bp.dt, B.dt, z, v[2], a[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) w[q] = w[q] + al[q] * bp.half_dt;
  }
  V.B.x[i] = x; V.B.y[i] = y; V.B.z[i] = z;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    V.B.v[q][i] = v[q]; V.B.w[q][i] = w[q]; V.B.a[q][i] = a[q]; V.B.al[q][i] = al[q];
  }
  V.B.T[i] = V.A.T[j];
  const R d = V.A.d[j];
  V.B.d[i] = d;
  R msum = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double mq = V.A.m[q][j];   // copied bit for bit (FP64 value or Kahan pair)
    V.B.m[q][i] = mq;
    msum += mass_r<P>(V.B.m[q], i);
  }
  V.B.meta[i] = meta;
  V.B.orig[i] = V.A.orig[j];
  V.mass[i] = msum;
  // position relative to the own cell's corner (FP64 difference, then FP32)
  const unsigned k = V.keys[i];
  const long long l = (long long)k - B.cell_off;
  const int ix = (int)(l % B.nx), iy = (int)((l / B.nx) % B.ny), iz = (int)(l / ((long long)B.nx * B.ny));
  const float r = (float)(bp.k * d) * 0.5f;
  V.xl[i] = make_float4((float)(x - (B.x0 + ix * B.dx)), (float)(y - (B.y0 + iy * B.dy)),
                        (float)(z - (B.z0 + iz * B.dz)), r);
  // occupied ranges
  if (i == 0 || V.keys[i - 1] != k) V.cstart[k] = (unsigned)i;
  if (i == V.n - 1 || V.keys[i + 1] != k) V.cend[k] = (unsigned)(i + 1);
  // history slots travel with the parcel
  const int c = V.H.cnt[j];
  V.Hn.cnt[i] = (unsigned char)c;
  for (int s = 0; s < c; ++s) {
    V.Hn.id[(size_t)s * V.cap + i] = V.H.id[(size_t)s * V.cap + j];
#pragma unroll
    for (int q = 0; q < 3; ++q) V.Hn.xi[(size_t)(s * 3 + q) * V.cap + i] = V.H.xi[(size_t)(s * 3 + q) * V.cap + j];
  }
}

// ---------------------------------------------------------------------------------------
// Contacts: one thread per parcel over the 27 neighbouring cells. The pair test runs on
// FP32 cell-local coordinates (exact to ~1e-10 m); the FP64 form then re-tests the
// survivors on the FP64 positions with the oracle's expression, so its pair sets are
// bit-exact. Walls: FP32 pre-screen, FP64 distances for the primitives within reach.
// ---------------------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ void add_contact(const StepView<P> &V, int i, int cin, int pid, const BedP<typename P::R> &bp,
                                            typename P::R mstar, typename P::R ri, const typename P::R nrm[3],
                                            typename P::R delta, const typename P::R vrel[3],
                                            const typename P::R wi[3], typename P::R Fi[3], typename P::R Ti[3],
                                            int &cout) {
  using R = typename P::R;
  R xo[3] = {0, 0, 0};
  for (int sl = 0; sl < cin; ++sl)
    if (V.Hn.id[(size_t)sl * V.cap + i] == pid) {
#pragma unroll
      for (int q = 0; q < 3; ++q) xo[q] = V.Hn.xi[(size_t)(sl * 3 + q) * V.cap + i];
      break;
    }
  R Fc[3], Tc[3], xn[3];
  contact_force<R>(bp, mstar, ri, nrm, delta, vrel, xo, wi, Fc, Tc, xn);
#pragma unroll
  for (int q = 0; q < 3; ++q) { Fi[q] += Fc[q]; Ti[q] += Tc[q]; }
  if (cout < KMAX) {
    V.H.id[(size_t)cout * V.cap + i] = pid;
#pragma unroll
    for (int q = 0; q < 3; ++q) V.H.xi[(size_t)(cout * 3 + q) * V.cap + i] = xn[q];
    ++cout;
  } else {
    set_error(V.err, ERR_CAPACITY);
  }
}

template <class P>
__global__ void k_contacts(StepView<P> V) {
  using R = typename P::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int meta = V.B.meta[i];
  const int b = meta >> 8;
  const DevBed &B = V.beds[b];
  const BedP<R> &bp = V.bp[b];
  R Fi[3] = {0, 0, 0}, Ti[3] = {0, 0, 0};
  int cout = 0;
  const int cin = V.Hn.cnt[i];
  if (!(bp.flags & DEM_NO_CONTACTS)) {
    const float4 me = V.xl[i];
    const R di = V.B.d[i];
    const R mi = V.mass[i];
    const R vi[3] = {V.B.v[0][i], V.B.v[1][i], V.B.v[2][i]};
    const R wi[3] = {V.B.w[0][i], V.B.w[1][i], V.B.w[2][i]};
    const unsigned key = V.keys[i];
    const long long l = (long long)key - B.cell_off;
    const int X = (int)(l % B.nx), Y = (int)((l / B.nx) % B.ny), Z = (int)(l / ((long long)B.nx * B.ny));
    const float hx = (float)bp.dx, hy = (float)bp.dy, hz = (float)bp.dz;
    const float pm = (float)bp.pf_margin;
    double xi_d = 0, yi_d = 0, zi_d = 0, ri_d = 0;
    if constexpr (P::exact) {
      xi_d = V.B.x[i]; yi_d = V.B.y[i]; zi_d = V.B.z[i];
      ri_d = __dmul_rn(0.5, __dmul_rn(B.k, (double)di));
    }
    const R ri = P::exact ? (R)ri_d : (R)me.w;
    for (int dz = -1; dz <= 1; ++dz) {
      const int Z2 = Z + dz;
      if (Z2 < 0 || Z2 >= B.nz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int Y2 = Y + dy;
        if (Y2 < 0 || Y2 >= B.ny) continue;
        const unsigned krow = (unsigned)(B.cell_off + ((long long)Z2 * B.ny + Y2) * B.nx);
        const float oy = dy * hy - me.y, oz = dz * hz - me.z;
        for (int dx = -1; dx <= 1; ++dx) {
          const int X2 = X + dx;
          if (X2 < 0 || X2 >= B.nx) continue;
          const unsigned k2 = krow + (unsigned)X2;
          const unsigned jb = V.cstart[k2], je = V.cend[k2];
          const float ox = dx * hx - me.x;
          for (unsigned jj = jb; jj < je; ++jj) {
            const int j = (int)jj;
            if (j == i) continue;
            const float4 o = V.xl[j];
            const float ex = o.x + ox, ey = o.y + oy, ez = o.z + oz;   // x_j - x_i
            const float d2f = ex * ex + ey * ey + ez * ez;
            const float rsf = me.w + o.w;
            R nrm[3], delta;
            double rj_d = 0;
            if constexpr (P::exact) {
              const float rp = rsf + pm;
              if (d2f >= rp * rp) continue;
              const double dxd = V.B.x[j] - xi_d, dyd = V.B.y[j] - yi_d, dzd = V.B.z[j] - zi_d;
              rj_d = __dmul_rn(0.5, __dmul_rn(B.k, (double)V.B.d[j]));
              const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dxd, dxd), __dmul_rn(dyd, dyd)), __dmul_rn(dzd, dzd));
              const double rs = __dadd_rn(ri_d, rj_d);
              if (!(d2 < __dmul_rn(rs, rs))) continue;
              const double dd = sqrt(d2);
              nrm[0] = (R)(dxd / dd); nrm[1] = (R)(dyd / dd); nrm[2] = (R)(dzd / dd);
              delta = (R)(rs - dd);
            } else {
              if (!(d2f < rsf * rsf)) continue;
              const float df = sqrtf(d2f);
              const float inv = 1.0f / df;
              nrm[0] = (R)(ex * inv); nrm[1] = (R)(ey * inv); nrm[2] = (R)(ez * inv);
              delta = (R)((rsf * rsf - d2f) / (rsf + df));
            }
            const R rj = P::exact ? (R)rj_d : (R)o.w;
            const R mj = V.mass[j];
            const R mstar = mi * mj / (mi + mj);
            const R ws[3] = {ri * wi[0] + rj * V.B.w[0][j], ri * wi[1] + rj * V.B.w[1][j], ri * wi[2] + rj * V.B.w[2][j]};
            R vrel[3];
            vrel[0] = (vi[0] - V.B.v[0][j]) + (ws[1] * nrm[2] - ws[2] * nrm[1]);
            vrel[1] = (vi[1] - V.B.v[1][j]) + (ws[2] * nrm[0] - ws[0] * nrm[2]);
            vrel[2] = (vi[2] - V.B.v[2][j]) + (ws[0] * nrm[1] - ws[1] * nrm[0]);
            add_contact<P>(V, i, cin, V.B.orig[j], bp, mstar, ri, nrm, delta, vrel, wi, Fi, Ti, cout);
          }
        }
      }
    }
    // walls: FP32 pre-screen on the absolute position rebuilt from the cell corner
    const float xa = (float)bp.x0 + X * hx + me.x, ya = (float)bp.y0 + Y * hy + me.y, za = (float)bp.z0 + Z * hz + me.z;
    float distf[4], nwf[4][3];
    wall_primitives<float>(bp, xa, ya, za, distf, nwf);
    bool near = false;
#pragma unroll
    for (int p = 0; p < 4; ++p) near |= distf[p] < me.w + 1e-6f;
    if (near) {
      const double xd = V.B.x[i], yd = V.B.y[i], zd = V.B.z[i];
      const double rid = __dmul_rn(0.5, __dmul_rn(B.k, (double)di));
      double dist[4], nw[4][3];
      wall_primitives<double>(B, xd, yd, zd, dist, nw);
      for (int p = 0; p < 4; ++p) {
        const double gap = rid - dist[p];
        if (!(gap > 0.0)) continue;
        const R nrm[3] = {(R)-nw[p][0], (R)-nw[p][1], (R)-nw[p][2]};
        const R delta = (R)gap;
        const R wr[3] = {ri * wi[0], ri * wi[1], ri * wi[2]};
        R vrel[3];
        vrel[0] = vi[0] + (wr[1] * nrm[2] - wr[2] * nrm[1]);
        vrel[1] = vi[1] + (wr[2] * nrm[0] - wr[0] * nrm[2]);
        vrel[2] = vi[2] + (wr[0] * nrm[1] - wr[1] * nrm[0]);
        add_contact<P>(V, i, cin, -1 - p, bp, mi, ri, nrm, delta, vrel, wi, Fi, Ti, cout);
      }
    }
  }
  V.H.cnt[i] = (unsigned char)cout;
#pragma unroll
  for (int q = 0; q < 3; ++q) { V.F[q][i] = Fi[q]; V.Tq[q][i] = Ti[q]; }
  if (V.diag) V.diag[(size_t)DG_NCONTACT * V.cap + i] = (double)cout;
}

// ---------------------------------------------------------------------------------------
// Gas-particle terms, kinetics, second half kick, temperature and mass update; writes the
// parcel's contributions to its cell sums.
// ---------------------------------------------------------------------------------------
template <class P>
__global__ void k_gas_particle(StepView<P> V) {
  using R = typename P::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int meta = V.B.meta[i];
  const int ore = meta & 255;
  const BedP<R> &bp = V.bp[meta >> 8];
  const unsigned fl = bp.flags;
  const unsigned c = V.keys[i];
  const size_t nc = (size_t)V.ncells;
  Gas<R> g;
  g.rho = V.gp[GP_RHO * nc + c]; g.mu = V.gp[GP_MU * nc + c]; g.lam = V.gp[GP_LAM * nc + c];
  g.cp = V.gp[GP_CP * nc + c]; g.x = V.gp[GP_X * nc + c]; g.Dm = V.gp[GP_DM * nc + c];
  g.sc13 = V.gp[GP_SC13 * nc + c]; g.pr13 = V.gp[GP_PR13 * nc + c]; g.epow = V.gp[GP_EPOW * nc + c];
  g.D = V.gp[(ore ? GP_D1 : GP_D0) * nc + c]; g.uz = V.gp[GP_UZ * nc + c];
  g.eps = V.gp[GP_EPS * nc + c]; g.T = V.gp[GP_TG * nc + c];
  const R d = V.B.d[i];
  const R dc = bp.k * d;
  const R Vp = (R)(kPI / 6.0) * dc * dc * dc;
  const R r = (R)0.5 * dc;
  const R vh[3] = {V.B.v[0][i], V.B.v[1][i], V.B.v[2][i]};
  const R sv[3] = {-vh[0], -vh[1], g.uz - vh[2]};
  const R slip = sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
  const R Re = g.rho * g.eps * d * slip / g.mu;
  const R re02 = pos_pow(Re, (R)0.2);
  const R re07 = re02 * sqrt(Re);
  const R bo = beta_over_epsp<R>(bp, ore, d, g, slip, Re);
  const R Kp = (fl & DEM_NO_DRAG) ? (R)0 : bo * Vp;
  const R Fd[3] = {Kp * sv[0], Kp * sv[1], Kp * sv[2]};
  const R Nu = gunn(g.eps, re02, re07, g.pr13);
  const R hA = (fl & DEM_NO_HEAT) ? (R)0 : bp.k3 * Nu * g.lam / d * ((R)kPI * d * d);
  const R Tp = V.B.T[i];
  const R Qconv = hA * (g.T - Tp);
  R m[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) m[q] = mass_r<P>(V.B.m[q], i);
  const bool cpl = coupled_step(bp.ncouple, V.step_ctr);
  const R dtm = bp.dtg;
  KinOut<R> kn;
  uscm<R>(bp, m, Tp, d, ore, g, re02, re07, dtm, kn);
  const R mp = V.mass[i];
  const R I = (R)0.4 * mp * r * r;
  const R F[3] = {V.F[0][i], V.F[1][i], V.F[2][i]};
  const R Tq[3] = {V.Tq[0][i], V.Tq[1][i], V.Tq[2][i]};
  R a[3];
  a[0] = (F[0] + Fd[0]) / mp;
  a[1] = (F[1] + Fd[1]) / mp;
  a[2] = (F[2] + Fd[2] - Vp * bp.dpdz) / mp + bp.grav;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const R al = Tq[q] / I;
    V.B.v[q][i] = vh[q] + a[q] * bp.half_dt;
    V.B.w[q][i] = V.B.w[q][i] + al * bp.half_dt;
    V.B.a[q][i] = a[q];
    V.B.al[q][i] = al;
  }
  const Tab<R> &t = tab<R>();
  R cpp = 0;
  const R inv_mp = (R)1 / mp;
#pragma unroll
  for (int q = 0; q < 4; ++q) cpp += m[q] * inv_mp * cp_over_R<R>(3 + q, Tp) * t.RMz[q];
  const R Tn = Tp + bp.dt * (Qconv + kn.Qr + kn.Qrm) / (mp * cpp);
  V.B.T[i] = Tn;
  if (cpl) {
#pragma unroll
    for (int q = 0; q < 4; ++q) mass_add<P>(V.B.m[q], i, kn.mdot[q] * dtm);
  }
  if (!isfinite(Tn) || !isfinite(V.B.v[0][i] + V.B.v[1][i] + V.B.v[2][i])) set_error(V.err, ERR_NONFINITE);
  // contributions to the cell sums
  const size_t cp = (size_t)V.cap;
  R *s = V.src;
  s[SR_VS * cp + i] = Vp;
  s[SR_SH2 * cp + i] = kn.sH2;
  s[SR_SH2O * cp + i] = kn.sH2O;
  s[SR_K * cp + i] = Kp;
  s[SR_KVX * cp + i] = Kp * vh[0];
  s[SR_KVY * cp + i] = Kp * vh[1];
  s[SR_KVZ * cp + i] = Kp * vh[2];
  s[SR_HA * cp + i] = hA;
  s[SR_HAT * cp + i] = hA * Tp;
  s[SR_QRM * cp + i] = kn.Qrm;
  s[SR_QR * cp + i] = kn.Qr;
  s[SR_EQ * cp + i] = kn.EQ;
  s[SR_ES * cp + i] = kn.ES;
  s[SR_CNT * cp + i] = (R)1;
  if (V.diag) {
    double *dg = V.diag;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      dg[(DG_FC + q) * cp + i] = (double)F[q];
      dg[(DG_TC + q) * cp + i] = (double)Tq[q];
      dg[(DG_FD + q) * cp + i] = (double)Fd[q];
      dg[(DG_XIDOT + q) * cp + i] = (double)kn.xidot[q];
      dg[(DG_A + q) * cp + i] = (double)kn.A[q];
      dg[(DG_B + q) * cp + i] = (double)kn.B[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) dg[(DG_MDOT + q) * cp + i] = (double)kn.mdot[q];
    dg[DG_K * cp + i] = (double)Kp;
    dg[DG_QCONV * cp + i] = (double)Qconv;
    dg[DG_QR * cp + i] = (double)kn.Qr;
    dg[DG_QRM * cp + i] = (double)kn.Qrm;
    dg[DG_FFILM * cp + i] = (double)kn.F;
    dg[DG_SH * cp + i] = (double)kn.Sh;
    dg[DG_NU * cp + i] = (double)Nu;
    dg[DG_RE * cp + i] = (double)Re;
    dg[DG_CELL * cp + i] = (double)(c - V.beds[meta >> 8].cell_off);
  }
}

// ---------------------------------------------------------------------------------------
// Per gas cell: sum the sources of its parcels in sorted order, update the gas state
// (coupling steps), and recompute the cell's properties for the next step.
// ---------------------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ void store_props(StepView<P> &V, long long c, const CellProps<typename P::R> &p) {
  const size_t nc = (size_t)V.ncells;
  V.gp[GP_RHO * nc + c] = p.rho; V.gp[GP_MU * nc + c] = p.mu; V.gp[GP_LAM * nc + c] = p.lam;
  V.gp[GP_CP * nc + c] = p.cp; V.gp[GP_X * nc + c] = p.x; V.gp[GP_DM * nc + c] = p.Dm;
  V.gp[GP_SC13 * nc + c] = p.sc13; V.gp[GP_PR13 * nc + c] = p.pr13;
  V.gp[GP_EPOW * nc + c] = p.epow; V.gp[GP_D0 * nc + c] = p.D[0];
  V.gp[GP_D1 * nc + c] = p.D[1]; V.gp[GP_UZ * nc + c] = p.uz;
  V.gp[GP_EPS * nc + c] = p.eps; V.gp[GP_TG * nc + c] = p.T;
}

// sums of the per-parcel sources of [jb, je): FP64 or Kahan-compensated FP32
template <class P> struct CellSum {
  double s[SR_N];
  __device__ __forceinline__ void run(const typename P::R *src, size_t cp, unsigned jb, unsigned je) {
    if constexpr (P::kahan) {
      float v[SR_N], cc[SR_N];
#pragma unroll
      for (int f = 0; f < SR_N; ++f) { v[f] = 0.f; cc[f] = 0.f; }
      for (unsigned j = jb; j < je; ++j) {
#pragma unroll
        for (int f = 0; f < SR_N; ++f) {
          const float y = src[f * cp + j] - cc[f];
          const float t = v[f] + y;
          cc[f] = (t - v[f]) - y;
          v[f] = t;
        }
      }
#pragma unroll
      for (int f = 0; f < SR_N; ++f) s[f] = (double)v[f] - (double)cc[f];
    } else {
#pragma unroll
      for (int f = 0; f < SR_N; ++f) s[f] = 0.0;
      for (unsigned j = jb; j < je; ++j) {
#pragma unroll
        for (int f = 0; f < SR_N; ++f) s[f] += (double)src[f * cp + j];
      }
    }
  }
};

template <class P>
__global__ void k_cells(StepView<P> V, int mode /* 0 step, 1 eps init, 2 props only */) {
  using R = typename P::R;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells) return;
  const int b = V.cell_bed[c];
  const DevBed &B = V.beds[b];
  const BedP<R> &bp = V.bp[b];
  const size_t nc = (size_t)V.ncells;
  const double *G = V.gas;
  double *Gn = V.gas_new;
  double eps = G[GS_EPS * nc + c], Y[3] = {G[GS_Y0 * nc + c], G[GS_Y1 * nc + c], G[GS_Y2 * nc + c]};
  double T = G[GS_T * nc + c];
  const bool solid = V.mark[c] != 0;
  if (mode != 2) {
    const unsigned jb = V.cstart[c], je = V.cend[c];
    const size_t cp = (size_t)V.cap;
    if (mode == 1) {
      double vs = 0.0;
      for (unsigned j = jb; j < je; ++j) vs += (double)V.src[SR_VS * cp + j];
      eps = solid ? B.eps_min : fmax(1.0 - vs / B.vcell, B.eps_min);
    } else if (!solid && coupled_step(bp.ncouple, V.step_ctr) && !(bp.flags & DEM_NO_GAS_UPDATE)) {
      CellSum<P> S;
      S.run(V.src, cp, jb, je);
      const long long lc = c - B.cell_off;
      const long long layer = (long long)B.nx * B.ny;
      const bool up = lc >= layer && !V.mark[c - layer];
      if constexpr (sizeof(R) == 8) {
        // the all-FP64 form: the oracle's expressions
        const double dtg = B.ncouple * B.dt;
        const double rho = (double)V.gp[GP_RHO * nc + c], cpg = (double)V.gp[GP_CP * nc + c];
        const double uz = B.U_in / eps;
        double Yup[3] = {B.Y_in[0], B.Y_in[1], B.Y_in[2]}, Tup = B.T_in;
        if (up) {
          Yup[0] = G[GS_Y0 * nc + c - layer]; Yup[1] = G[GS_Y1 * nc + c - layer]; Yup[2] = G[GS_Y2 * nc + c - layer];
          Tup = G[GS_T * nc + c - layer];
        }
        const double Sj[3] = {S.s[SR_SH2], S.s[SR_SH2O], 0.0};
        const double Snet = Sj[0] + Sj[1];
        const double mg = eps * rho * B.vcell;
        double Yn[3], ys = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const double y = Y[j] + dtg * (-uz * (Y[j] - Yup[j]) / B.dz + (Sj[j] - Y[j] * Snet) / mg);
          Yn[j] = fmax(y, 0.0);
          ys += Yn[j];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) Yn[j] = ys > 0.0 ? Yn[j] / ys : Y[j];
        const double capc = eps * rho * cpg;
        const double H0 = S.s[SR_HA] / B.vcell, H1 = S.s[SR_HAT] / B.vcell;
        const double Mrm = -S.s[SR_QRM] / B.vcell;
        const Tab<double> &td = tab<double>();
        const double Mr = -(h_over_R<double>(0, T) * td.RMj[0] * Sj[0] + h_over_R<double>(1, T) * td.RMj[1] * Sj[1]) / B.vcell;
        const double rhs = T + dtg * (-uz * (T - Tup) / B.dz + (H1 + Mr + Mrm) / capc);
        T = rhs / (1.0 + dtg * H0 / capc);
        eps = fmax(1.0 - S.s[SR_VS] / B.vcell, B.eps_min);
#pragma unroll
        for (int j = 0; j < 3; ++j) Y[j] = Yn[j];
      } else {
        // FP32 forms: increments in FP32, accumulated into the FP64 state
        const Tab<R> &t = tab<R>();
        const R dtg = bp.dtg;
        const R rho = V.gp[GP_RHO * nc + c], cpg = V.gp[GP_CP * nc + c];
        const R eps_r = V.gp[GP_EPS * nc + c], T_r = V.gp[GP_TG * nc + c];
        const R uz = bp.U_in / eps_r;
        const R Yr[3] = {(R)Y[0], (R)Y[1], (R)Y[2]};
        R Yup[3] = {bp.Y_in[0], bp.Y_in[1], bp.Y_in[2]}, Tup = bp.T_in;
        if (up) {
          Yup[0] = (R)G[GS_Y0 * nc + c - layer]; Yup[1] = (R)G[GS_Y1 * nc + c - layer];
          Yup[2] = (R)G[GS_Y2 * nc + c - layer];
          Tup = (R)G[GS_T * nc + c - layer];   // the old state: props are rewritten in place
        }
        const R Sj[3] = {(R)S.s[SR_SH2], (R)S.s[SR_SH2O], (R)0};
        const R Snet = Sj[0] + Sj[1];
        const R inv_mg = bp.inv_vcell / (eps_r * rho);
        bool clamp = false;
        double Yn[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const R dy = dtg * (-uz * (Yr[j] - Yup[j]) * bp.inv_dz + (Sj[j] - Yr[j] * Snet) * inv_mg);
          Yn[j] = Y[j] + (double)dy;
          if (Yn[j] < 0.0) { Yn[j] = 0.0; clamp = true; }
        }
        if (clamp) {
          const double ys = Yn[0] + Yn[1] + Yn[2];
#pragma unroll
          for (int j = 0; j < 3; ++j) Yn[j] = ys > 0.0 ? Yn[j] / ys : Y[j];
        }
        const R capc = eps_r * rho * cpg;
        const R H0 = (R)S.s[SR_HA] * bp.inv_vcell, H1 = (R)S.s[SR_HAT] * bp.inv_vcell;
        const R Mrm = -(R)S.s[SR_QRM] * bp.inv_vcell;
        const R Mr = -(h_over_R<R>(0, T_r) * t.RMj[0] * Sj[0] + h_over_R<R>(1, T_r) * t.RMj[1] * Sj[1]) * bp.inv_vcell;
        // T' - T of the semi-implicit update (eq (4-6)), H1 - H0 T formed before dividing
        const R num = dtg * (-uz * (T_r - Tup) * bp.inv_dz + (H1 - H0 * T_r + Mr + Mrm) / capc);
        const R den = (R)1 + dtg * H0 / capc;
        T = T + (double)(num / den);
        const R epsn = (R)1 - (R)S.s[SR_VS] * bp.inv_vcell;
        eps = (double)(epsn > bp.eps_min ? epsn : bp.eps_min);
#pragma unroll
        for (int j = 0; j < 3; ++j) Y[j] = Yn[j];
      }
    }
  }
  Gn[GS_EPS * nc + c] = eps;
  Gn[GS_Y0 * nc + c] = Y[0]; Gn[GS_Y1 * nc + c] = Y[1]; Gn[GS_Y2 * nc + c] = Y[2];
  Gn[GS_T * nc + c] = T;
  const R Yr[3] = {(R)Y[0], (R)Y[1], (R)Y[2]};
  const CellProps<R> p = gas_cell_props<R>(bp, (R)eps, Yr, (R)T);
  store_props(V, c, p);
}

// Cell sums of the last step's per-parcel sources (dem_get_sources).
template <class P>
__global__ void k_sources(StepView<P> V) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells) return;
  const size_t cp = (size_t)V.cap;
  CellSum<P> S;
  S.run(V.src, cp, V.cstart[c], V.cend[c]);
  const bool solid = V.mark[c] != 0;
  for (int f = 0; f < SR_N; ++f) V.dep[(size_t)c * SR_N + f] = solid ? 0.0 : S.s[f];
}

// Initial per-parcel volume for the initial gas volume fraction.
template <class P>
__global__ void k_volume(StepView<P> V) {
  using R = typename P::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const BedP<R> &bp = V.bp[V.B.meta[i] >> 8];
  const R dc = bp.k * V.B.d[i];
  V.src[SR_VS * (size_t)V.cap + i] = (R)(kPI / 6.0) * dc * dc * dc;
}

// ---------------------------------------------------------------------------------------
// Reduction degree (eqs (2-15)..(2-19)) per parcel and per bed (deterministic two-pass).
// ---------------------------------------------------------------------------------------
template <class P>
__global__ void k_fov_parcel(StepView<P> V, double *per_parcel_orig, double *fv /* [3][n] */) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int ore = V.A.meta[i] & 255;
  const Tab<double> &td = tab<double>();
  double n[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) n[q] = mass_d<P>(V.A.m[q], i) / td.Mz[q];
  const double nfe = 2.0 * n[0] + 3.0 * n[1] + n[2] + n[3];
  double f = 0.0;
  if (nfe > 0.0) {
    const double fh = (3.0 * n[1] + n[2] + n[3]) / nfe, fm = (n[2] + n[3]) / nfe, fw = n[3] / nfe;
    f = ore == 0 ? fh / 9.0 + 2.0 * fm / 9.0 + 6.0 * fw / 9.0 : 0.25 * fm + 0.75 * fw;
  }
  if (per_parcel_orig) per_parcel_orig[V.A.orig[i]] = f;
  fv[i] = f;
  fv[(size_t)V.n + i] = 3.0 * n[0] + 4.0 * n[1] + n[2];
  fv[2 * (size_t)V.n + i] = (ore == 0 ? 1.5 : 4.0 / 3.0) * nfe;
}

// One block per bed: the bed's parcels are contiguous in the sorted order; sum them in a
// fixed order (strided per thread, then a shared-memory tree) so the result is
// reproducible bit for bit.
template <class P>
__global__ void k_fov_bed(StepView<P> V, const double *fv, double *out /* [nbeds][4] */) {
  __shared__ double sh[3][256];
  const int b = blockIdx.x;
  const unsigned klo = (unsigned)V.beds[b].cell_off;
  const unsigned khi = (b + 1 < V.nbeds) ? (unsigned)V.beds[b + 1].cell_off : 0xffffffffu;
  int lo = 0, hi = V.n;
  while (lo < hi) { int mid = (lo + hi) >> 1; if (V.keys[mid] < klo) lo = mid + 1; else hi = mid; }
  const int beg = lo;
  hi = V.n;
  while (lo < hi) { int mid = (lo + hi) >> 1; if (V.keys[mid] < khi) lo = mid + 1; else hi = mid; }
  const int end = lo;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int i = beg + (int)threadIdx.x; i < end; i += blockDim.x) {
    a0 += fv[i]; a1 += fv[(size_t)V.n + i]; a2 += fv[2 * (size_t)V.n + i];
  }
  sh[0][threadIdx.x] = a0; sh[1][threadIdx.x] = a1; sh[2][threadIdx.x] = a2;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[b * 4 + 0] = sh[0][0]; out[b * 4 + 1] = sh[1][0]; out[b * 4 + 2] = sh[2][0];
    out[b * 4 + 3] = (double)(end - beg);
  }
}

// ---------------------------------------------------------------------------------------
// Scatter helpers (sorted order -> parcel-index order) for the getters.
// ---------------------------------------------------------------------------------------
template <class P>
__global__ void k_scatter_state(StepView<P> V, double *out /* [DEM_NSTATE][n] */) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const size_t n = (size_t)V.n;
  const int o = V.A.orig[i];
  out[0 * n + o] = V.A.x[i]; out[1 * n + o] = V.A.y[i]; out[2 * n + o] = V.A.z[i];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    out[(3 + q) * n + o] = (double)V.A.v[q][i];
    out[(6 + q) * n + o] = (double)V.A.w[q][i];
    out[(14 + q) * n + o] = (double)V.A.a[q][i];
    out[(17 + q) * n + o] = (double)V.A.al[q][i];
  }
  out[9 * n + o] = (double)V.A.T[i];
#pragma unroll
  for (int q = 0; q < 4; ++q) out[(10 + q) * n + o] = mass_d<P>(V.A.m[q], i);
}

template <class P>
__global__ void k_scatter_diag(StepView<P> V, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int o = V.A.orig[i];
  for (int f = 0; f < DG_N; ++f) out[(size_t)f * V.n + o] = V.diag[(size_t)f * V.cap + i];
}

template <class P>
__global__ void k_scatter_hist(StepView<P> V, int *cnt, int *partner, double *xi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int o = V.A.orig[i];
  const int c = V.H.cnt[i];
  cnt[o] = c;
  for (int s = 0; s < KMAX; ++s) {
    const bool live = s < c;
    partner[(size_t)o * KMAX + s] = live ? V.H.id[(size_t)s * V.cap + i] : INT_MIN;
#pragma unroll
    for (int q = 0; q < 3; ++q)
      xi[((size_t)o * KMAX + s) * 3 + q] = live ? (double)V.H.xi[(size_t)(s * 3 + q) * V.cap + i] : 0.0;
  }
}

__global__ void k_mark_cells(const DevBed *beds, const int *cell_bed, unsigned char *mark, long long ncells);
__global__ void k_step_counter(long long *ctr);

}  // namespace dem
