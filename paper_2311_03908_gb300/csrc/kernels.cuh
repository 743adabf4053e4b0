// kernels.cuh -- the per-step kernels of the particle path, templated on the arithmetic
// type R (double: all-FP64 form; float: split form). Instantiated in inst_f64.cu and
// inst_f32.cu, launched by dem_api.cu.
#pragma once
#include "common.cuh"

namespace dem {

// One parcel-state buffer, structure of arrays in the current sorted order.
template <class R> struct PState {
  double *x, *y, *z;
  R *v[3], *w[3], *a[3], *al[3], *T, *d;
  double *m[4];
  int *meta;   // bed << 8 | ore
  int *orig;   // parcel index (input order)
};

// Contact-history table: count per parcel, then KMAX slots of partner index and 3-vector.
template <class R> struct Hist {
  unsigned char *cnt;
  int *id;     // [KMAX][cap]
  R *xi;       // [KMAX*3][cap]
};

// Everything a step's kernels touch.
template <class R> struct StepView {
  int n, cap, nbeds;
  long long ncells;
  const DevBed *beds;
  PState<R> A, B;               // A: state before the step, B: gather target
  Hist<R> H, Hn;                // H: current history, Hn: gather target
  unsigned *keys, *vals;        // sorted keys and the permutation (old index of new slot)
  unsigned *cstart, *cend;      // DEM-cell ranges
  unsigned *gstart, *gend;      // gas-cell ranges (alias of the DEM ranges when every s == 1)
  int *gcell;                   // global gas cell of each parcel (new order)
  float4 *xf;                   // FP32 bed-relative position and radius (new order)
  R *mass;                      // parcel mass (new order)
  R *F[3], *Tq[3];              // contact force and torque
  R *src;                       // [SR_N][cap] per-parcel cell sources
  double *gas, *gas_new;        // [GS_N][ncells]
  R *gp;                        // [GP_N][ncells]
  unsigned char *mark;          // solid (IBM) cell mark
  int *cell_bed;                // bed of each gas cell
  double *diag;                 // [DG_N][cap] or null
  double *dep;                  // [SR_N][ncells] or null (written by k_sources)
  int *err;
  const long long *step_ctr;    // steps completed so far (device)
};

__device__ __forceinline__ bool coupled_step(const DevBed &B, const long long *ctr) {
  return ((*ctr + 1) % B.ncouple) == 0;
}

// ---------------------------------------------------------------------------------------
// half kick and drift of velocity Verlet (kick-drift-kick). The key kernel and the gather
// kernel both call this, so the new positions they see are the same bits.
// ---------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void kick_drift(double dt, double &x, R &v, R a) {
  if (sizeof(R) == 8) {
    double vh = __dadd_rn((double)v, __dmul_rn((double)a, 0.5 * dt));
    x = __dadd_rn(x, __dmul_rn(vh, dt));
    v = (R)vh;
  } else {
    v = v + a * (R)(0.5 * dt);
    x = x + (double)v * dt;
  }
}

// Gas cell and DEM-cell key of a point (cell = floor((x - x0) * (1/dx)), clamped).
__device__ __forceinline__ unsigned point_key(const DevBed &B, double x, double y, double z,
                                              int &g_local, bool &outside) {
  const double fx = floor((x - B.x0) * B.inv_dx);
  const double fy = floor((y - B.y0) * B.inv_dy);
  const double fz = floor((z - B.z0) * B.inv_dz);
  outside = !(fx >= 0.0 && fx < (double)B.nx && fy >= 0.0 && fy < (double)B.ny && fz >= 0.0 &&
              fz < (double)B.nz);
  const int ix = (int)fmin(fmax(fx, 0.0), (double)(B.nx - 1));
  const int iy = (int)fmin(fmax(fy, 0.0), (double)(B.ny - 1));
  const int iz = (int)fmin(fmax(fz, 0.0), (double)(B.nz - 1));
  g_local = (iz * B.ny + iy) * B.nx + ix;
  if (B.s == 1) return B.key_off + (unsigned)g_local;
  const int s = B.s;
  const int sx = min(max((int)floor(((x - B.x0) * B.inv_dx - ix) * s), 0), s - 1);
  const int sy = min(max((int)floor(((y - B.y0) * B.inv_dy - iy) * s), 0), s - 1);
  const int sz = min(max((int)floor(((z - B.z0) * B.inv_dz - iz) * s), 0), s - 1);
  return B.key_off + (unsigned)g_local * (unsigned)(s * s * s) + (unsigned)((sz * s + sy) * s + sx);
}

template <class R>
__global__ void k_key(StepView<R> V, int drift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int b = V.A.meta[i] >> 8;
  const DevBed &B = V.beds[b];
  double x = V.A.x[i], y = V.A.y[i], z = V.A.z[i];
  if (drift) {
    R vx = V.A.v[0][i], vy = V.A.v[1][i], vz = V.A.v[2][i];
    kick_drift<R>(B.dt, x, vx, V.A.a[0][i]);
    kick_drift<R>(B.dt, y, vy, V.A.a[1][i]);
    kick_drift<R>(B.dt, z, vz, V.A.a[2][i]);
  }
  int gl;
  bool out;
  V.keys[i] = point_key(B, x, y, z, gl, out);
  V.vals[i] = (unsigned)i;
  if (out) set_error(V.err, ERR_DOMAIN);
}

// Gather the state into the sorted order, applying the half kick and drift; record the
// cell ranges by boundary detection on the sorted keys; copy the history slots.
template <class R>
__global__ void k_gather(StepView<R> V, int drift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int j = (int)V.vals[i];
  const int meta = V.A.meta[j];
  const DevBed &B = V.beds[meta >> 8];
  double x = V.A.x[j], y = V.A.y[j], z = V.A.z[j];
  R v[3] = {V.A.v[0][j], V.A.v[1][j], V.A.v[2][j]};
  R w[3] = {V.A.w[0][j], V.A.w[1][j], V.A.w[2][j]};
  R a[3] = {V.A.a[0][j], V.A.a[1][j], V.A.a[2][j]};
  R al[3] = {V.A.al[0][j], V.A.al[1][j], V.A.al[2][j]};
  if (drift) {
    kick_drift<R>(B.dt, x, v[0], a[0]);
    kick_drift<R>(B.dt, y, v[1], a[1]);
    kick_drift<R>(B.dt, z, v[2], a[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) w[q] = w[q] + al[q] * (R)(0.5 * B.dt);
  }
  V.B.x[i] = x; V.B.y[i] = y; V.B.z[i] = z;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    V.B.v[q][i] = v[q]; V.B.w[q][i] = w[q]; V.B.a[q][i] = a[q]; V.B.al[q][i] = al[q];
  }
  V.B.T[i] = V.A.T[j];
  const R d = V.A.d[j];
  V.B.d[i] = d;
  double msum = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) { const double mq = V.A.m[q][j]; V.B.m[q][i] = mq; msum += mq; }
  V.B.meta[i] = meta;
  V.B.orig[i] = V.A.orig[j];
  V.mass[i] = (R)msum;
  const double r = 0.5 * (B.k * (double)d);
  V.xf[i] = make_float4((float)(x - B.x0), (float)(y - B.y0), (float)(z - B.z0), (float)r);
  int gl;
  bool out;
  (void)point_key(B, x, y, z, gl, out);
  const int gc = (int)(B.cell_off + gl);
  V.gcell[i] = gc;
  // occupied ranges
  const unsigned k = V.keys[i];
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

// Gas-cell ranges when some bed uses DEM sub-cells (the gas cell is key / s^3).
template <class R>
__global__ void k_gas_ranges(StepView<R> V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int g = V.gcell[i];
  if (i == 0 || V.gcell[i - 1] != g) V.gstart[g] = (unsigned)i;
  if (i == V.n - 1 || V.gcell[i + 1] != g) V.gend[g] = (unsigned)(i + 1);
}

// ---------------------------------------------------------------------------------------
// Contacts: one thread per parcel over the 27 neighbouring DEM cells, FP32 prefilter on
// bed-relative coordinates, then the exact FP64 overlap test; walls last.
// ---------------------------------------------------------------------------------------
template <class R>
__global__ void k_contacts(StepView<R> V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int meta = V.B.meta[i];
  const DevBed &B = V.beds[meta >> 8];
  R Fi[3] = {0, 0, 0}, Ti[3] = {0, 0, 0};
  int cout = 0;
  const int cin = V.Hn.cnt[i];
  if (!(B.flags & DEM_NO_CONTACTS)) {
    const double xi = V.B.x[i], yi = V.B.y[i], zi = V.B.z[i];
    const float4 me = V.xf[i];
    const R di = V.B.d[i];
    const double ri_d = __dmul_rn(0.5, __dmul_rn(B.k, (double)di));
    const R ri = (R)ri_d;
    const R mi = V.mass[i];
    const R vi[3] = {V.B.v[0][i], V.B.v[1][i], V.B.v[2][i]};
    const R wi[3] = {V.B.w[0][i], V.B.w[1][i], V.B.w[2][i]};
    // DEM-cell coordinates of this parcel from its key
    const int s = B.s, s3 = s * s * s;
    const unsigned q = V.keys[i] - B.key_off;
    const int g = (int)(q / (unsigned)s3), sub = (int)(q - (unsigned)g * (unsigned)s3);
    const int ix = g % B.nx, iy = (g / B.nx) % B.ny, iz = g / (B.nx * B.ny);
    const int X = ix * s + sub % s, Y = iy * s + (sub / s) % s, Z = iz * s + sub / (s * s);
    const int NX = B.nx * s, NY = B.ny * s, NZ = B.nz * s;
    const float pm = B.pf_margin;
    for (int dz = -1; dz <= 1; ++dz) {
      const int Z2 = Z + dz;
      if (Z2 < 0 || Z2 >= NZ) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int Y2 = Y + dy;
        if (Y2 < 0 || Y2 >= NY) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int X2 = X + dx;
          if (X2 < 0 || X2 >= NX) continue;
          unsigned k2;
          if (s == 1) k2 = B.key_off + (unsigned)((Z2 * B.ny + Y2) * B.nx + X2);
          else k2 = B.key_off + (unsigned)(((Z2 / s) * B.ny + Y2 / s) * B.nx + X2 / s) * (unsigned)s3 +
                    (unsigned)(((Z2 % s) * s + Y2 % s) * s + X2 % s);
          const unsigned jb = V.cstart[k2], je = V.cend[k2];
          for (unsigned jj = jb; jj < je; ++jj) {
            const int j = (int)jj;
            if (j == i) continue;
            const float4 o = V.xf[j];
            const float ex = o.x - me.x, ey = o.y - me.y, ez = o.z - me.z;
            const float rsf = me.w + o.w + pm;
            if (ex * ex + ey * ey + ez * ez >= rsf * rsf) continue;
            // exact overlap from the FP64 positions
            const double dxd = V.B.x[j] - xi, dyd = V.B.y[j] - yi, dzd = V.B.z[j] - zi;
            const double rj_d = __dmul_rn(0.5, __dmul_rn(B.k, (double)V.B.d[j]));
            R nrm[3], delta;
            if (sizeof(R) == 8) {
              const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dxd, dxd), __dmul_rn(dyd, dyd)), __dmul_rn(dzd, dzd));
              const double rs = __dadd_rn(ri_d, rj_d);
              if (!(d2 < __dmul_rn(rs, rs))) continue;
              const double dd = sqrt(d2);
              nrm[0] = (R)(dxd / dd); nrm[1] = (R)(dyd / dd); nrm[2] = (R)(dzd / dd);
              delta = (R)(rs - dd);
            } else {
              const double d2 = dxd * dxd + dyd * dyd + dzd * dzd;
              const double rs = ri_d + rj_d;
              const double gap = rs * rs - d2;        // > 0 iff overlapping
              if (!(gap > 0.0)) continue;
              const float df = sqrtf((float)d2);
              const float inv = 1.0f / df;
              nrm[0] = (R)((float)dxd * inv); nrm[1] = (R)((float)dyd * inv); nrm[2] = (R)((float)dzd * inv);
              delta = (R)((float)gap / ((float)rs + df));
            }
            const R rj = (R)rj_d;
            const R mj = V.mass[j];
            const R mstar = mi * mj / (mi + mj);
            const R ws[3] = {ri * wi[0] + rj * V.B.w[0][j], ri * wi[1] + rj * V.B.w[1][j], ri * wi[2] + rj * V.B.w[2][j]};
            R vrel[3];
            vrel[0] = (vi[0] - V.B.v[0][j]) + (ws[1] * nrm[2] - ws[2] * nrm[1]);
            vrel[1] = (vi[1] - V.B.v[1][j]) + (ws[2] * nrm[0] - ws[0] * nrm[2]);
            vrel[2] = (vi[2] - V.B.v[2][j]) + (ws[0] * nrm[1] - ws[1] * nrm[0]);
            const int pid = V.B.orig[j];
            R xo[3] = {0, 0, 0};
            for (int sl = 0; sl < cin; ++sl)
              if (V.Hn.id[(size_t)sl * V.cap + i] == pid) {
#pragma unroll
                for (int qq = 0; qq < 3; ++qq) xo[qq] = V.Hn.xi[(size_t)(sl * 3 + qq) * V.cap + i];
                break;
              }
            R Fc[3], Tc[3], xn[3];
            contact_force<R>(B, mstar, ri, nrm, delta, vrel, xo, wi, Fc, Tc, xn);
#pragma unroll
            for (int qq = 0; qq < 3; ++qq) { Fi[qq] += Fc[qq]; Ti[qq] += Tc[qq]; }
            if (cout < KMAX) {
              V.H.id[(size_t)cout * V.cap + i] = pid;
#pragma unroll
              for (int qq = 0; qq < 3; ++qq) V.H.xi[(size_t)(cout * 3 + qq) * V.cap + i] = xn[qq];
              ++cout;
            } else {
              set_error(V.err, ERR_CAPACITY);
            }
          }
        }
      }
    }
    // walls: distances in FP64 (resting overlaps are far below FP32 resolution of the bed)
    double dist[4], nw[4][3];
    wall_primitives(B, xi, yi, zi, dist, nw);
    for (int p = 0; p < 4; ++p) {
      const double gap = ri_d - dist[p];
      if (!(gap > 0.0)) continue;
      R nrm[3] = {(R)-nw[p][0], (R)-nw[p][1], (R)-nw[p][2]};
      const R delta = (R)gap;
      const R wr[3] = {ri * wi[0], ri * wi[1], ri * wi[2]};
      R vrel[3];
      vrel[0] = vi[0] + (wr[1] * nrm[2] - wr[2] * nrm[1]);
      vrel[1] = vi[1] + (wr[2] * nrm[0] - wr[0] * nrm[2]);
      vrel[2] = vi[2] + (wr[0] * nrm[1] - wr[1] * nrm[0]);
      const int pid = -1 - p;
      R xo[3] = {0, 0, 0};
      for (int sl = 0; sl < cin; ++sl)
        if (V.Hn.id[(size_t)sl * V.cap + i] == pid) {
#pragma unroll
          for (int qq = 0; qq < 3; ++qq) xo[qq] = V.Hn.xi[(size_t)(sl * 3 + qq) * V.cap + i];
          break;
        }
      R Fc[3], Tc[3], xn[3];
      contact_force<R>(B, mi, ri, nrm, delta, vrel, xo, wi, Fc, Tc, xn);
#pragma unroll
      for (int qq = 0; qq < 3; ++qq) { Fi[qq] += Fc[qq]; Ti[qq] += Tc[qq]; }
      if (cout < KMAX) {
        V.H.id[(size_t)cout * V.cap + i] = pid;
#pragma unroll
        for (int qq = 0; qq < 3; ++qq) V.H.xi[(size_t)(cout * 3 + qq) * V.cap + i] = xn[qq];
        ++cout;
      } else {
        set_error(V.err, ERR_CAPACITY);
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
template <class R>
__global__ void k_gas_particle(StepView<R> V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int meta = V.B.meta[i];
  const int ore = meta & 255;
  const DevBed &B = V.beds[meta >> 8];
  const unsigned fl = B.flags;
  const int c = V.gcell[i];
  const size_t nc = (size_t)V.ncells;
  Gas<R> g;
  g.rho = V.gp[GP_RHO * nc + c]; g.mu = V.gp[GP_MU * nc + c]; g.lam = V.gp[GP_LAM * nc + c];
  g.cp = V.gp[GP_CP * nc + c]; g.x = V.gp[GP_X * nc + c]; g.Dm = V.gp[GP_DM * nc + c];
  g.sc13 = V.gp[GP_SC13 * nc + c]; g.pr13 = V.gp[GP_PR13 * nc + c]; g.epow = V.gp[GP_EPOW * nc + c];
  g.D = V.gp[(ore ? GP_D1 : GP_D0) * nc + c]; g.uz = V.gp[GP_UZ * nc + c];
  g.eps = V.gp[GP_EPS * nc + c]; g.T = V.gp[GP_TG * nc + c];
  const R d = V.B.d[i];
  const R k = (R)B.k, k3 = (R)B.k3;
  const R dc = k * d;
  const R Vp = (R)(kPI / 6.0) * dc * dc * dc;
  const R r = (R)0.5 * dc;
  R vh[3] = {V.B.v[0][i], V.B.v[1][i], V.B.v[2][i]};
  const R sv[3] = {-vh[0], -vh[1], g.uz - vh[2]};
  const R slip = sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
  const R Re = g.rho * g.eps * d * slip / g.mu;
  const R re02 = pos_pow(Re, (R)0.2);
  const R re07 = re02 * sqrt(Re);
  const R bo = beta_over_epsp<R>(B, ore, d, g, slip, Re);
  const R Kp = (fl & DEM_NO_DRAG) ? (R)0 : bo * Vp;
  const R Fd[3] = {Kp * sv[0], Kp * sv[1], Kp * sv[2]};
  const R Nu = gunn(g.eps, re02, re07, g.pr13);
  const R hA = (fl & DEM_NO_HEAT) ? (R)0 : k3 * Nu * g.lam / d * ((R)kPI * d * d);
  const R Tp = V.B.T[i];
  const R Qconv = hA * (g.T - Tp);
  double m[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) m[q] = V.B.m[q][i];
  const bool cpl = coupled_step(B, V.step_ctr);
  const R dt = (R)B.dt;
  const R dtm = (R)(B.ncouple * B.dt);
  KinOut<R> kn;
  uscm<R>(B, m, Tp, d, ore, g, re02, re07, dtm, kn);
  const R mp = V.mass[i];
  const R I = (R)0.4 * mp * r * r;
  R a[3], al[3];
  const R F[3] = {V.F[0][i], V.F[1][i], V.F[2][i]};
  const R Tq[3] = {V.Tq[0][i], V.Tq[1][i], V.Tq[2][i]};
  a[0] = (F[0] + Fd[0]) / mp;
  a[1] = (F[1] + Fd[1]) / mp;
  a[2] = (F[2] + Fd[2] - Vp * (R)B.dpdz) / mp + ((fl & DEM_NO_GRAVITY) ? (R)0 : (R)(-kGrav));
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    al[q] = Tq[q] / I;
    V.B.v[q][i] = vh[q] + a[q] * (R)(0.5 * B.dt);
    V.B.w[q][i] = V.B.w[q][i] + al[q] * (R)(0.5 * B.dt);
    V.B.a[q][i] = a[q];
    V.B.al[q][i] = al[q];
  }
  R cpp = 0;
  const R inv_mp = (R)1 / mp;
#pragma unroll
  for (int q = 0; q < 4; ++q) cpp += (R)m[q] * inv_mp * cp_over_R(3 + q, Tp) * (R)(kRgas / cMz[q]);
  const R Tn = Tp + dt * (Qconv + kn.Qr + kn.Qrm) / (mp * cpp);
  V.B.T[i] = Tn;
  bool bad = !isfinite((double)Tn) || !isfinite((double)V.B.v[0][i]) || !isfinite((double)V.B.v[2][i]);
  if (cpl) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double mn = fmax(m[q] + (double)kn.mdot[q] * (double)dtm, 0.0);
      V.B.m[q][i] = mn;
    }
  }
  if (bad) set_error(V.err, ERR_NONFINITE);
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
    dg[DG_CELL * cp + i] = (double)(c - B.cell_off);
  }
}

// ---------------------------------------------------------------------------------------
// Per gas cell: sum the sources of its parcels in sorted order (FP64), update the gas
// state (coupling steps), and recompute the cell's properties for the next step.
// ---------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void store_props(StepView<R> &V, int c, const CellProps &p) {
  const size_t nc = (size_t)V.ncells;
  V.gp[GP_RHO * nc + c] = (R)p.rho; V.gp[GP_MU * nc + c] = (R)p.mu; V.gp[GP_LAM * nc + c] = (R)p.lam;
  V.gp[GP_CP * nc + c] = (R)p.cp; V.gp[GP_X * nc + c] = (R)p.x; V.gp[GP_DM * nc + c] = (R)p.Dm;
  V.gp[GP_SC13 * nc + c] = (R)p.sc13; V.gp[GP_PR13 * nc + c] = (R)p.pr13;
  V.gp[GP_EPOW * nc + c] = (R)p.epow; V.gp[GP_D0 * nc + c] = (R)p.D[0];
  V.gp[GP_D1 * nc + c] = (R)p.D[1]; V.gp[GP_UZ * nc + c] = (R)p.uz;
  V.gp[GP_EPS * nc + c] = (R)p.eps; V.gp[GP_TG * nc + c] = (R)p.T;
}

template <class R>
__global__ void k_cells(StepView<R> V, int mode /* 0 step, 1 eps init, 2 props only */) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells) return;
  const int b = V.cell_bed[c];
  const DevBed &B = V.beds[b];
  const size_t nc = (size_t)V.ncells;
  const double *G = V.gas;
  double *Gn = V.gas_new;
  double eps = G[GS_EPS * nc + c], Y[3] = {G[GS_Y0 * nc + c], G[GS_Y1 * nc + c], G[GS_Y2 * nc + c]};
  double T = G[GS_T * nc + c];
  const bool solid = V.mark[c] != 0;
  if (mode != 2) {
    const unsigned jb = V.gstart[c], je = V.gend[c];
    const size_t cp = (size_t)V.cap;
    if (mode == 1) {
      double vs = 0.0;
      for (unsigned j = jb; j < je; ++j) vs += (double)V.src[SR_VS * cp + j];
      eps = solid ? B.eps_min : fmax(1.0 - vs / B.vcell, B.eps_min);
    } else if (!solid && coupled_step(B, V.step_ctr) && !(B.flags & DEM_NO_GAS_UPDATE)) {
      double S[SR_N];
#pragma unroll
      for (int f = 0; f < SR_N; ++f) S[f] = 0.0;
      for (unsigned j = jb; j < je; ++j) {
#pragma unroll
        for (int f = 0; f < SR_N; ++f) S[f] += (double)V.src[f * cp + j];
      }
      const double dtg = B.ncouple * B.dt;
      const double rho = (double)V.gp[GP_RHO * nc + c], cpg = (double)V.gp[GP_CP * nc + c];
      const double uz = B.U_in / eps;
      const long long lc = c - B.cell_off;
      const long long layer = (long long)B.nx * B.ny;
      double Yup[3] = {B.Y_in[0], B.Y_in[1], B.Y_in[2]}, Tup = B.T_in;
      if (lc >= layer && !V.mark[c - layer]) {
        Yup[0] = G[GS_Y0 * nc + c - layer]; Yup[1] = G[GS_Y1 * nc + c - layer]; Yup[2] = G[GS_Y2 * nc + c - layer];
        Tup = G[GS_T * nc + c - layer];
      }
      const double Sj[3] = {S[SR_SH2], S[SR_SH2O], 0.0};
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
      const double H0 = S[SR_HA] / B.vcell, H1 = S[SR_HAT] / B.vcell;
      const double Mrm = -S[SR_QRM] / B.vcell;
      const double Mr = -(h_over_R<double>(0, T) * (kRgas / cMj[0]) * Sj[0] +
                          h_over_R<double>(1, T) * (kRgas / cMj[1]) * Sj[1]) / B.vcell;
      const double rhs = T + dtg * (-uz * (T - Tup) / B.dz + (H1 + Mr + Mrm) / capc);
      T = rhs / (1.0 + dtg * H0 / capc);
      eps = fmax(1.0 - S[SR_VS] / B.vcell, B.eps_min);
#pragma unroll
      for (int j = 0; j < 3; ++j) Y[j] = Yn[j];
    }
  }
  Gn[GS_EPS * nc + c] = eps;
  Gn[GS_Y0 * nc + c] = Y[0]; Gn[GS_Y1 * nc + c] = Y[1]; Gn[GS_Y2 * nc + c] = Y[2];
  Gn[GS_T * nc + c] = T;
  const CellProps p = gas_cell_props<R>(B, eps, Y, T);
  store_props(V, (int)c, p);
}

// Cell sums of the last step's per-parcel sources (dem_get_sources).
template <class R>
__global__ void k_sources(StepView<R> V) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells) return;
  const size_t nc = (size_t)V.ncells, cp = (size_t)V.cap;
  const unsigned jb = V.gstart[c], je = V.gend[c];
  const bool solid = V.mark[c] != 0;
  for (int f = 0; f < SR_N; ++f) {
    double s = 0.0;
    if (!solid)
      for (unsigned j = jb; j < je; ++j) s += (double)V.src[f * cp + j];
    V.dep[(size_t)c * SR_N + f] = s;
  }
}

// Initial per-parcel volume for the initial gas volume fraction.
template <class R>
__global__ void k_volume(StepView<R> V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const DevBed &B = V.beds[V.B.meta[i] >> 8];
  const R dc = (R)B.k * V.B.d[i];
  V.src[SR_VS * (size_t)V.cap + i] = (R)(kPI / 6.0) * dc * dc * dc;
}

// ---------------------------------------------------------------------------------------
// Reduction degree (eqs (2-15)..(2-19)) per parcel and per bed (deterministic two-pass).
// ---------------------------------------------------------------------------------------
template <class R>
__global__ void k_fov_parcel(StepView<R> V, double *per_parcel_orig, double *fv /* [3][n] */) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int ore = V.A.meta[i] & 255;
  double n[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) n[q] = V.A.m[q][i] / cMz[q];
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
template <class R>
__global__ void k_fov_bed(StepView<R> V, const double *fv, double *out /* [nbeds][4] */) {
  __shared__ double sh[3][256];
  const int b = blockIdx.x;
  const unsigned klo = V.beds[b].key_off;
  const unsigned khi = (b + 1 < V.nbeds) ? V.beds[b + 1].key_off : 0xffffffffu;
  // first index with key >= klo, first with key >= khi
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
template <class R>
__global__ void k_scatter_state(StepView<R> V, double *out /* [DEM_NSTATE][n] */) {
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
  for (int q = 0; q < 4; ++q) out[(10 + q) * n + o] = V.A.m[q][i];
}

template <class R>
__global__ void k_scatter_diag(StepView<R> V, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const int o = V.A.orig[i];
  for (int f = 0; f < DG_N; ++f) out[(size_t)f * V.n + o] = V.diag[(size_t)f * V.cap + i];
}

template <class R>
__global__ void k_scatter_hist(StepView<R> V, int *cnt, int *partner, double *xi) {
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

// Solid (IBM) marks of the gas cells: a cell is solid when it lies wholly outside the fluid
// region (signed distance of its centre below minus half the cell diagonal).
__global__ void k_mark_cells(const DevBed *beds, const int *cell_bed, unsigned char *mark, long long ncells);

__global__ void k_step_counter(long long *ctr);

}  // namespace dem
