// dem_api.cu -- the C ABI declared in include/dem.h: validation, the device arena,
// initial binning, stepping (plain and CUDA-graph), getters and error handling.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "radix.cuh"

using dem::DevBed;

namespace dem {

__global__ void k_step_counter(StepEnd se) {
  pdl_wait();
  step_end(se);
}

// Solid (IBM-marked) gas cells, and the cells near a wall: those whose parcels may touch a
// wall primitive. Every primitive's distance is 1-Lipschitz in the position (the plate's
// is bounded below by |z - z_plate|), so a cell is far from all walls when each distance at
// its centre exceeds the half-diagonal plus the largest parcel radius plus a margin of
// 1e-5 m (far above the FP32 error of the contact kernels' wall pre-screen, which would
// then find nothing within reach either).
__global__ void k_mark_cells(const DevBed *beds, const BedP<double> *bps, const int *cell_bed, unsigned char *mark,
                             unsigned char *wnear, long long ncells) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const DevBed &B = beds[cell_bed[c]];
  const BedP<double> &bp = bps[cell_bed[c]];
  const long long l = c - B.cell_off;
  const int ix = (int)(l % B.nx), iy = (int)((l / B.nx) % B.ny), iz = (int)(l / ((long long)B.nx * B.ny));
  const double xc = B.x0 + (ix + 0.5) * B.dx, yc = B.y0 + (iy + 0.5) * B.dy, zc = B.z0 + (iz + 0.5) * B.dz;
  const double hd = 0.5 * sqrt(B.dx * B.dx + B.dy * B.dy + B.dz * B.dz);
  const double rho = sqrt(xc * xc + yc * yc);
  double sd = B.R_bed - rho;
  if (B.wall == DEM_WALL_CONE) sd = fmin(sd, (zc - B.z_apex) * B.sin_a - rho * B.cos_a);
  mark[c] = sd < -hd ? 1 : 0;
  const double far = hd + bp.reach_max + 1e-5;
  bool near = B.R_bed - rho < far || B.H - zc < far;
  if (B.wall == DEM_WALL_FLAT) {
    near |= zc < far;
  } else {
    if (zc - 0.5 * B.dz < B.plate_z) near |= (zc - B.z_apex) * B.sin_a - rho * B.cos_a < far;
    near |= fabs(zc - B.plate_z) < far;
  }
  wnear[c] = near ? 1 : 0;
}

// Initial parcel state in input order (accelerations start as gravity, spins at rest).
template <class P>
__global__ void k_load(int n, const double *const *src /* 8 + 4 arrays */, const int *ore,
                       const int *bed, const DevBed *beds, double *x, double *y, double *z,
                       typename P::R *const *rv /* v3 w3 a3 al3 T d */, double *const *m, int *meta, int *orig) {
  using R = typename P::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const DevBed &B = beds[bed[i]];
  if constexpr (P::kahan) {
    // FP32 pairs relative to the bed corner
    const double o[3] = {B.x0, B.y0, B.z0};
    double *const pd[3] = {x, y, z};
    for (int q = 0; q < 3; ++q) {
      const double rel = src[q][i] - o[q];
      const float hi = (float)rel;
      reinterpret_cast<float2 *>(pd[q])[i] = make_float2(hi, (float)(rel - (double)hi));
    }
  } else {
    x[i] = src[0][i]; y[i] = src[1][i]; z[i] = src[2][i];
  }
  for (int q = 0; q < 3; ++q) {
    rv[q][i] = (R)src[3 + q][i];
    rv[3 + q][i] = (R)0;
    rv[6 + q][i] = (R)0;
    rv[9 + q][i] = (R)0;
  }
  rv[8][i] = (B.flags & DEM_NO_GRAVITY) ? (R)0 : (R)(-kGrav);
  // the state holds the half-step velocity: the first half kick of the first step, with the
  // key kernel's expression and the stored acceleration (gravity)
  rv[2][i] = half_kick<R>((R)(0.5 * B.dt), B.dt, rv[2][i], rv[8][i]);
  rv[12][i] = (R)src[7][i];
  rv[13][i] = (R)src[6][i];
  for (int q = 0; q < 4; ++q) {
    if constexpr (P::kahan) {
      const float hi = (float)src[8 + q][i];
      reinterpret_cast<float2 *>(m[q])[i] = make_float2(hi, (float)(src[8 + q][i] - (double)hi));
    } else {
      m[q][i] = src[8 + q][i];
    }
  }
  meta[i] = (bed[i] << 8) | ore[i];
  orig[i] = i;
}

int prof_begin(dem_ctx *c, const char *name) {
  if (!c->prof_on) return -1;
  int id = -1;
  for (size_t k = 0; k < c->prof_names.size(); ++k)
    if (c->prof_names[k] == name) { id = (int)k; break; }
  if (id < 0) {
    c->prof_names.push_back(name);
    c->prof_ms.push_back(0.0);
    c->prof_n.push_back(0);
    id = (int)c->prof_names.size() - 1;
  }
  const int slot = (int)(2 * c->prof_marks.size());
  while ((int)c->ev_pool.size() < slot + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    c->ev_pool.push_back(e);
  }
  cudaEventRecord(c->ev_pool[slot], c->st);
  c->prof_marks.push_back({id, slot});
  return slot;
}

void prof_end(dem_ctx *c, int slot) {
  if (slot < 0) return;
  cudaEventRecord(c->ev_pool[slot + 1], c->st);
}

__global__ void k_gas_load(long long nc, const double *Y /* nc*3 */, const double *T, double *G, bool pairs) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  gas_put(G, GS_EPS * nc + c, 1.0, pairs);
  gas_put(G, GS_Y0 * nc + c, Y[c * 3 + 0], pairs);
  gas_put(G, GS_Y1 * nc + c, Y[c * 3 + 1], pairs);
  gas_put(G, GS_Y2 * nc + c, Y[c * 3 + 2], pairs);
  gas_put(G, GS_T * nc + c, T[c], pairs);
}

}  // namespace dem

namespace {

using namespace dem;

const double kMzH[4] = {159.69e-3, 231.533e-3, 71.844e-3, 55.845e-3};

#define CK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) { return fail(c, e_); }         \
  } while (0)

int fail(dem_ctx *c, cudaError_t e) {
  (void)c;
  if (e == cudaErrorMemoryAllocation) return DEM_ENOMEM;
  return DEM_ECUDA;
}

int status_from_bits(int bits) {
  if (bits & ERR_NONFINITE) return DEM_ENONFINITE;
  if (bits & ERR_CAPACITY) return DEM_ECAPACITY;
  if (bits & ERR_TIMEOUT) return DEM_ETIMEOUT;
  if (bits & ERR_DOMAIN) return DEM_EDOMAIN;
  return DEM_OK;
}

// observe a finished step's error word; block = wait for it
int poll(dem_ctx *c, bool block) {
  if (c->sticky != DEM_OK) return c->sticky;
  if (!c->pending) return DEM_OK;
  if (block) {
    if (cudaEventSynchronize(c->ev) != cudaSuccess) { c->sticky = DEM_ECUDA; return c->sticky; }
  } else {
    cudaError_t q = cudaEventQuery(c->ev);
    if (q == cudaErrorNotReady) return DEM_OK;
    if (q != cudaSuccess) { c->sticky = DEM_ECUDA; return c->sticky; }
  }
  c->pending = false;
  c->sticky = status_from_bits(*c->h_err);
  return c->sticky;
}

int mark_pending(dem_ctx *c) {
  CK(cudaMemcpyAsync(c->h_err, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaEventRecord(c->ev, c->st));
  c->pending = true;
  return DEM_OK;
}

// the context stream takes up a coupling input still crossing on its own stream
int join_gas(dem_ctx *c) {
  if (!c->gas_pending) return DEM_OK;
  if (cudaStreamWaitEvent(c->st, c->ev_gas, 0) != cudaSuccess) return DEM_ECUDA;
  c->gas_pending = false;
  return DEM_OK;
}

int sync_all(dem_ctx *c) {
  int s = poll(c, true);
  if (s != DEM_OK) return s;
  if (join_gas(c) != DEM_OK) return c->sticky = DEM_ECUDA;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return DEM_ECUDA;
  return DEM_OK;
}

// Layer porosities (Sec. 2.3): the core's effective density from the initial porosity, each
// product layer's effective density by the equivalent-mass ratios q of eq (2-36).
void layer_porosity_host(const dem_bed_config &b, int ore, double out[3]) {
  const double q_mh = 2.0 * kMzH[1] / (3.0 * kMzH[0]);
  const double q_wm = 3.0 * kMzH[2] / kMzH[1];
  const double q_few = kMzH[3] / kMzH[2];
  double rm = ore == 0 ? (1.0 - b.xi0[0]) * b.rho_true[0] * q_mh : (1.0 - b.xi0[1]) * b.rho_true[1];
  double rw = rm * q_wm, rfe = rw * q_few;
  out[0] = 1.0 - rm / b.rho_true[1];
  out[1] = 1.0 - rw / b.rho_true[2];
  out[2] = 1.0 - rfe / b.rho_true[3];
}

double fuller_const(double Mi, double Mj, double Vi, double Vj) {
  const double s = std::cbrt(Vi) + std::cbrt(Vj);
  return std::sqrt(1.0 / Mi + 1.0 / Mj) / (s * s);
}

int validate_bed(const dem_bed_config &b) {
  if (!(b.bed_D > 0 && b.bed_H > 0 && b.nx >= 1 && b.ny >= 1 && b.nz >= 1)) return DEM_EINVAL;
  if ((long long)b.nx * b.ny * b.nz > (1LL << 30)) return DEM_EINVAL;
  if (!(b.dt > 0 && b.kn > 0 && b.kt_over_kn > 0 && b.restitution > 0 && b.restitution <= 1)) return DEM_EINVAL;
  if (!(b.mu_s >= 0 && b.mu_r >= 0 && b.cg_ratio >= 1 && b.coupling_interval >= 1)) return DEM_EINVAL;
  if (!(b.T_in > 0 && b.p0 > 0 && b.U_in >= 0 && b.tortuosity > 0 && b.eps_min > 0 && b.eps_min < 1)) return DEM_EINVAL;
  double ys = b.Y_in[0] + b.Y_in[1] + b.Y_in[2];
  if (!(std::fabs(ys - 1.0) < 1e-9) || b.Y_in[0] < 0 || b.Y_in[1] < 0 || b.Y_in[2] < 0) return DEM_EINVAL;
  for (int o = 0; o < 2; ++o)
    if (!(b.sphericity[o] > 0 && b.sphericity[o] <= 1 && b.xi0[o] >= 0 && b.xi0[o] < 1 && b.pore_d_cm[o] > 0)) return DEM_EINVAL;
  for (int z = 0; z < 4; ++z) if (!(b.rho_true[z] > 0)) return DEM_EINVAL;
  for (int r = 0; r < 3; ++r) if (!(b.k0[r] >= 0 && b.Ea[r] >= 0)) return DEM_EINVAL;
  if (b.wall_kind != DEM_WALL_FLAT && b.wall_kind != DEM_WALL_CONE) return DEM_EINVAL;
  if ((b.flags & DEM_RADIATION) && !(b.emissivity >= 0 && b.emissivity <= 1)) return DEM_EINVAL;
  if ((b.flags & DEM_GAS_SOLVER) && (b.flags & DEM_NO_GAS_UPDATE)) return DEM_EINVAL;
  if ((b.flags & DEM_CONDUCTION) &&
      !(b.lambda_p[0] > 0 && b.lambda_p[1] > 0 && b.lambda_wall > 0 && std::isfinite(b.lambda_p[0]) &&
        std::isfinite(b.lambda_p[1]) && std::isfinite(b.lambda_wall)))
    return DEM_EINVAL;
  if (b.wall_kind == DEM_WALL_CONE &&
      !(b.cone_half_angle > 0 && b.cone_half_angle < 1.5707963 && b.cone_height > 0 && b.hole_pitch > 0 &&
        b.hole_d > 0 && b.hole_d < b.hole_pitch && b.plate_z > 0 && b.plate_z < b.bed_H))
    return DEM_EINVAL;
  return DEM_OK;
}

DevBed derive_bed(const dem_bed_config &b) {
  DevBed B;
  std::memset(&B, 0, sizeof B);
  B.nx = b.nx; B.ny = b.ny; B.nz = b.nz;
  B.x0 = -0.5 * b.bed_D; B.y0 = -0.5 * b.bed_D; B.z0 = 0.0;
  B.dx = b.bed_D / b.nx; B.dy = b.bed_D / b.ny; B.dz = b.bed_H / b.nz;
  B.inv_dx = 1.0 / B.dx; B.inv_dy = 1.0 / B.dy; B.inv_dz = 1.0 / B.dz;
  B.vcell = B.dx * B.dy * B.dz;
  B.inv_vcell = 1.0 / B.vcell;
  B.R_bed = 0.5 * b.bed_D; B.H = b.bed_H; B.wall = b.wall_kind;
  B.cos_a = std::cos(b.cone_half_angle); B.sin_a = std::sin(b.cone_half_angle);
  B.z_apex = b.wall_kind == DEM_WALL_CONE ? b.cone_height - B.R_bed / std::tan(b.cone_half_angle) : 0.0;
  B.plate_z = b.plate_z; B.pitch = b.hole_pitch > 0 ? b.hole_pitch : 1.0; B.inv_pitch = 1.0 / B.pitch;
  B.r_hole = 0.5 * b.hole_d;
  B.dt = b.dt; B.k = b.cg_ratio;
  B.ncouple = b.coupling_interval;
  B.U_in = b.U_in; B.T_in = b.T_in; B.p0 = b.p0;
  for (int j = 0; j < 3; ++j) B.Y_in[j] = b.Y_in[j];
  B.eps_min = b.eps_min;
  B.flags = b.flags;
  return B;
}

// Physics parameters of a bed, computed in FP64 and stored in the form's type.
template <class R>
BedP<R> derive_params(const dem_bed_config &b, const DevBed &G) {
  BedP<R> P{};
  std::memset(&P, 0, sizeof P);
  P.k = (R)b.cg_ratio; P.k3 = (R)(b.cg_ratio * b.cg_ratio * b.cg_ratio);
  P.inv_k3 = (R)(1.0 / (b.cg_ratio * b.cg_ratio * b.cg_ratio));
  P.dt = (R)b.dt; P.half_dt = (R)(0.5 * b.dt);
  P.kn = (R)b.kn; P.kt = (R)(b.kt_over_kn * b.kn);
  const double le = std::log(b.restitution);
  P.eta_coef = (R)(-2.0 * le / std::sqrt(kPI * kPI + le * le));
  P.eta_t_ratio = (R)std::sqrt(b.kt_over_kn);
  P.mu_s = (R)b.mu_s; P.mu_r = (R)b.mu_r;
  P.x0 = (R)G.x0; P.y0 = (R)G.y0; P.z0 = (R)G.z0;
  P.dx = (R)G.dx; P.dy = (R)G.dy; P.dz = (R)G.dz;
  P.inv_dx = (R)G.inv_dx; P.inv_dy = (R)G.inv_dy; P.inv_dz = (R)G.inv_dz;
  P.R_bed = (R)G.R_bed; P.H = (R)G.H; P.cos_a = (R)G.cos_a; P.sin_a = (R)G.sin_a; P.z_apex = (R)G.z_apex;
  P.plate_z = (R)G.plate_z; P.pitch = (R)G.pitch; P.inv_pitch = (R)G.inv_pitch; P.r_hole = (R)G.r_hole;
  P.U_in = (R)b.U_in; P.p0 = (R)b.p0; P.T_in = (R)b.T_in;
  for (int j = 0; j < 3; ++j) P.Y_in[j] = (R)b.Y_in[j];
  P.eps_min = (R)b.eps_min; P.inv_vcell = (R)G.inv_vcell;
  for (int r = 0; r < 3; ++r) { P.k0[r] = (R)b.k0[r]; P.Ea_R[r] = (R)(b.Ea[r] / kRgas); }
  P.inv_tau = (R)(1.0 / b.tortuosity);
  for (int o = 0; o < 2; ++o) {
    const double psi = b.sphericity[o];
    P.psi[o] = (R)psi;
    P.K1b[o] = (R)(1.0 / (1.0 / 3.0 + (2.0 / 3.0) / std::sqrt(psi)));
    P.K2[o] = (R)std::pow(10.0, 1.8148 * std::pow(-std::log10(psi), 0.5743));
    double xi[3];
    layer_porosity_host(b, o, xi);
    for (int l = 0; l < 3; ++l) P.xi[o][l] = (R)xi[l];
    P.pore_cm[o] = (R)b.pore_d_cm[o];
    P.DKc[o] = (R)(0.97 * 0.5 * b.pore_d_cm[o]);
  }
  P.wall_K1 = (R)(2.25 / b.bed_D);
  P.fuller12 = (R)fuller_const(2.016, 18.015, 7.07, 12.7);
  P.fuller13 = (R)fuller_const(2.016, 28.014, 7.07, 17.9);
  P.mfp_c = (R)(1.013 / b.p0);
  P.rate_c = (R)(kPI * b.p0 / kRgas);
  P.dpdz = (R)b.dpdz;
  P.grav = (b.flags & DEM_NO_GRAVITY) ? (R)0 : (R)(-kGrav);
  P.dtg = (R)(b.coupling_interval * b.dt);
  P.pf_margin = (R)1e-8;
  P.rad_c = (b.flags & DEM_RADIATION)
                ? (R)(b.cg_ratio * b.cg_ratio * b.cg_ratio * kSigmaSB * b.emissivity * kPI) : (R)0;
  if (b.flags & DEM_CONDUCTION) {
    // f(e) of eq (3-43): the maximum overlap of a damped linear collision in units of
    // v / omega_0, exp(-zeta arccos(zeta) / sqrt(1 - zeta^2)) with zeta of eq (3-44); e_CGP
    // of eq (3-45) clamped at 0, where f is exp(-1) (critical damping)
    auto f_of = [](double e) {
      if (!(e > 0.0)) return std::exp(-1.0);
      if (e >= 1.0) return 1.0;
      const double l = std::log(e), z = -l / std::sqrt(kPI * kPI + l * l);
      return std::exp(-z * std::acos(z) / std::sqrt(1.0 - z * z));
    };
    const double k = b.cg_ratio, e = b.restitution;
    const double ecg2 = 1.0 + k * (e * e - 1.0);
    const double ecg = ecg2 > 0.0 ? std::sqrt(ecg2) : 0.0;
    P.cond_pp = (R)(4.0 * std::pow(k, 0.75) * std::sqrt(f_of(e) / f_of(ecg)));
    P.cond_pf = (R)(2.0 * kPI * k * k);
    for (int o = 0; o < 2; ++o) {
      for (int q = 0; q < 2; ++q) P.lam_e[o][q] = (R)(b.lambda_p[o] * b.lambda_p[q] / (b.lambda_p[o] + b.lambda_p[q]));
      P.lam_ew[o] = (R)(b.lambda_p[o] * b.lambda_wall / (b.lambda_p[o] + b.lambda_wall));
    }
    P.lmin = (R)(1.013e-2 / b.p0);
  }
  P.flags = b.flags;
  P.ncouple = b.coupling_interval;
  P.wall = b.wall_kind;
  return P;
}

struct Bump {
  char *base = nullptr;
  size_t off = 0;
  template <class T> T *take(size_t count, size_t elem = sizeof(T)) {
    off = (off + 255) & ~(size_t)255;
    T *p = base ? (T *)(base + off) : nullptr;
    off += count * elem;
    return p;
  }
};

template <class R> void set_skin(BedP<R> &P, double skin) {
  P.skin = (R)skin;
  P.half_skin2 = (R)(0.49 * 0.49 * skin * skin);   // 2% below half the skin: FP32 displacements
}

// Lay out (or measure, when base is null) every arena buffer.
void layout(dem_ctx *c, Bump &m) {
  const size_t N = (size_t)c->cap, R = c->rsize, C = (size_t)c->ncells;
  for (int k = 0; k < 2; ++k) {
    for (int q = 0; q < 3; ++q) c->px[k][q] = m.take<double>(N);
    for (int q = 0; q < 3; ++q) {
      c->pv[k][q] = m.take<char>(N, R); c->pw[k][q] = m.take<char>(N, R);
      c->pa[k][q] = m.take<char>(N, R); c->pal[k][q] = m.take<char>(N, R);
    }
    c->pT[k] = m.take<char>(N, R);
    c->pd[k] = m.take<char>(N, R);
    for (int q = 0; q < 4; ++q) c->pm[k][q] = m.take<double>(N);
    c->pmeta[k] = m.take<int>(N);
    c->porig[k] = m.take<int>(N);
    for (int q = 0; q < 3; ++q) c->pdsp[k][q] = m.take<float>(N);
    c->hcnt[k] = m.take<unsigned char>(N);
    c->hid[k] = m.take<int>(N * KMAX);
    c->hxi[k] = m.take<char>(N * KMAX * 3, R);
  }
  c->keys = m.take<unsigned>(N); c->vals = m.take<unsigned>(N);
  c->keys2 = m.take<unsigned>(N); c->vals2 = m.take<unsigned>(N);
  for (int k = 0; k < 2; ++k) { c->skey[k] = m.take<unsigned>(N); c->sval[k] = m.take<unsigned>(N); }
  c->rsw = m.take<unsigned>(resort_words((int)N, &c->rs_pow2));
  c->inv = m.take<unsigned>(N);
  c->rhist = m.take<unsigned>(radix_hist_words((int)N));
  c->cstart = m.take<unsigned>(C); c->cend = m.take<unsigned>(C);
  c->xl = m.take<float4>(N);
  c->plist = m.take<int>(N * KLIST);
  c->pcode = m.take<unsigned char>(N * KLIST);
  c->pcnt = m.take<unsigned char>(N);
  c->nl = m.take<int>(N * KNL);
  c->nlc = m.take<unsigned char>(N);
  c->rebuild = m.take<int>(1);
  c->ovf = m.take<int>(N);
  c->novf = m.take<int>(1);
  c->work = m.take<uint2>(N);
  c->nwork = m.take<int>(1);
  const size_t Nr = c->any_rad ? N : 0;   // the radiation buffers exist only where a bed radiates
  c->qrad = m.take<char>(Nr, R);
  c->tsrt = m.take<char>(c->rsize == sizeof(double) ? Nr : 0, R);   // FP64 form only
  c->xr = m.take<float4>(Nr);
  c->qc = m.take<char>(c->any_cond ? N : 0, R);   // conduction heat of parcels in contact
  c->corner = m.take<double>(c->hcorner.size());
  c->cornerp = m.take<float2>(c->hcornerp.size());
  for (int q = 0; q < 3; ++q) { c->F[q] = m.take<char>(N, R); c->Tq[q] = m.take<char>(N, R); }
  c->src = m.take<char>(N * SR_CNT, R);
  c->gas[0] = m.take<double>(C * GS_N);
  c->gas[1] = m.take<double>(C * GS_N);
  c->gp = m.take<char>(C * GP_STRIDE, R);
  c->mark = m.take<unsigned char>(C);
  c->wnear = m.take<unsigned char>(C);
  c->cell_bed = m.take<int>(C);
  c->fv = m.take<double>((size_t)c->nbeds * FOV_CHUNKS * 4);
  c->fvbed = m.take<double>((size_t)c->nbeds * 4);
  c->err = m.take<int>(1);
  c->step_ctr = m.take<long long>(6);
  c->dbeds = m.take<DevBed>(c->nbeds);
  c->dbp_d = m.take<BedP<double>>(c->nbeds);
  c->dbp_f = m.take<BedP<float>>(c->nbeds);
  if (c->gas_solver) {   // the gas solver's faces, pressure, coefficients and CG vectors
    GasView &S = c->gsv;
    S.fu = m.take<double>(S.nfx); S.fv = m.take<double>(S.nfy); S.fw = m.take<double>(S.nfz);
    S.su = m.take<double>(S.nfx); S.sv = m.take<double>(S.nfy); S.sw = m.take<double>(S.nfz);
    S.pr = m.take<double>(C);
    S.co = m.take<double>(C * GC_N);
    S.x = m.take<double>(C); S.r = m.take<double>(C); S.z = m.take<double>(C);
    S.pa = m.take<double>(C); S.pb = m.take<double>(C); S.Ap = m.take<double>(C);
    S.part = m.take<double>((size_t)c->gs_grid * 4);
    S.cg_iters = m.take<int>(1);
    S.dep = m.take<double>(C * SR_N);
    S.bpd = c->dbp_d;
    // multigrid levels
    const int nl = (int)c->hlev.size();
    c->dlbed.assign(nl, nullptr);
    for (int l = 0; l < nl; ++l) {   // FP32 operators and iterates (level 0: copies of the FP64 one)
      GsLevel &Lv = c->hlev[l];
      if (l == 0) Lv.n = c->ncells;
      const size_t n = (size_t)Lv.n;
      Lv.L = m.take<float>(3 * n);
      Lv.diag = m.take<float>(n); Lv.out = m.take<float>(n); Lv.dinv = m.take<float>(n);
      Lv.b = m.take<float>(n); Lv.xa = m.take<float>(n); Lv.xb = m.take<float>(n);
      if (l > 0) {
        c->dlbed[l] = m.take<int>(n);
        Lv.bed = c->dlbed[l];
      } else {
        Lv.bed = c->cell_bed;
      }
    }
    c->dlpar.assign(nl, nullptr);
    for (int l = 0; l + 1 < nl; ++l) {
      c->dlpar[l] = m.take<int>((size_t)(l == 0 ? c->ncells : c->hlev[l].n));
      c->hlev[l].parent = c->dlpar[l];
    }
    for (int l = 0; l < nl; ++l) {   // uniform dims per level
      const GsLevelBed *g = &c->hlb[(size_t)l * c->nbeds];
      bool uni = true;
      for (int b = 1; b < c->nbeds; ++b) uni = uni && g[b].nx == g[0].nx && g[b].ny == g[0].ny && g[b].nz == g[0].nz;
      c->hlev[l].ux = uni ? g[0].nx : 0;
      c->hlev[l].uy = uni ? g[0].ny : 0;
    }
    c->dlev = m.take<GsLevel>(nl);
    c->dlb = m.take<GsLevelBed>(c->hlb.size());
    S.nlev = nl;
    S.nbeds = c->nbeds;
    S.lev = c->dlev;
    S.lb = c->dlb;
  }
}

int enqueue_steps_any(dem_ctx *c, int n) { return DEM_DISPATCH(c, enqueue_steps, c, n); }

// captured graphs bake launch shapes and pointers in
void drop_graphs(dem_ctx *c) {
  for (auto &kv : c->graphs) {
    cudaGraphExecDestroy(kv.second.second);
    cudaGraphDestroy(kv.second.first);
  }
  c->graphs.clear();
  c->graph_launches.clear();
}

void get_tuning(const dem_ctx *c, int32_t *t) {
  t[0] = c->use_lists;
  t[1] = c->bs_key; t[2] = c->bs_restore; t[3] = c->bs_search; t[4] = c->bs_contacts;
  t[5] = c->bs_gp; t[6] = c->bs_cells;
  t[7] = (int32_t)std::lround(c->skin_frac * 1000.0);
  t[8] = c->restore_every;
  t[9] = c->gsv.mg_nu;
  t[10] = (int32_t)std::lround(c->gsv.mg_alpha * 100.0);
}

int apply_tuning(dem_ctx *c, const int32_t *t) {
  if (t[0] != 0 && t[0] != 1) return DEM_EINVAL;
  int lim[6];
  if (DEM_DISPATCH(c, kernel_limits, lim) != 0) return DEM_ECUDA;
  for (int k = 1; k <= 6; ++k)
    if (t[k] < 32 || t[k] > 1024 || t[k] % 32 != 0 || t[k] > lim[k - 1]) return DEM_EINVAL;
  if (t[7] < 1 || t[7] > 1000) return DEM_EINVAL;
  if (t[8] < 1 || t[8] > 64) return DEM_EINVAL;
  if (t[9] < 0 || t[9] > 2 || t[10] < 50 || t[10] > 200) return DEM_EINVAL;
  c->use_lists = t[0];
  c->bs_key = t[1]; c->bs_restore = t[2]; c->bs_search = t[3]; c->bs_contacts = t[4];
  c->bs_gp = t[5]; c->bs_cells = t[6];
  c->skin_frac = t[7] / 1000.0;
  c->restore_every = t[8];
  c->gsv.mg_nu = t[9];
  c->gsv.mg_alpha = t[10] / 100.0;
  for (int b = 0; b < c->nbeds; ++b) {
    const double dmax = 2.0 * c->hbp_d[b].reach_max;
    set_skin(c->hbp_d[b], c->skin_frac * dmax);
    set_skin(c->hbp_f[b], c->skin_frac * dmax);
  }
  drop_graphs(c);
  if (cudaMemcpyAsync(c->dbp_d, c->hbp_d.data(), sizeof(BedP<double>) * c->nbeds, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
      cudaMemcpyAsync(c->dbp_f, c->hbp_f.data(), sizeof(BedP<float>) * c->nbeds, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
      cudaMemsetAsync(c->rebuild, 1, sizeof(int), c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess)
    return DEM_ECUDA;
  return DEM_OK;
}

}  // namespace

extern "C" {

const char *dem_strerror(int s) {
  switch (s) {
    case DEM_OK: return "ok";
    case DEM_EINVAL: return "invalid argument";
    case DEM_ENOMEM: return "out of memory";
    case DEM_ECUDA: return "CUDA runtime error";
    case DEM_ECAPACITY: return "contact-history capacity exceeded";
    case DEM_ENONFINITE: return "non-finite parcel state";
    case DEM_ETIMEOUT: return "bounded device wait timed out";
    case DEM_ESTATE: return "call not valid in this state";
    case DEM_EDOMAIN: return "parcel outside its gas grid";
    default: return "unknown status";
  }
}

void dem_destroy(dem_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  if (c->gst) cudaStreamDestroy(c->gst);
  if (c->sst) {
    cudaStreamSynchronize(c->sst);
    cudaStreamDestroy(c->sst);
  }
  if (c->ev_main) cudaEventDestroy(c->ev_main);
  if (c->ev_gas) cudaEventDestroy(c->ev_gas);
  for (auto &kv : c->graphs) {
    if (kv.second.second) cudaGraphExecDestroy(kv.second.second);
    if (kv.second.first) cudaGraphDestroy(kv.second.first);
  }
  if (c->arena) cudaFree(c->arena);
  if (c->diag) cudaFree(c->diag);
  if (c->dep) cudaFree(c->dep);
  if (c->scratch_out) cudaFree(c->scratch_out);
  if (c->adj) cudaFree(c->adj);
  if (c->gas_stage) cudaFree(c->gas_stage);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->ev) cudaEventDestroy(c->ev);
  delete c;
}

int dem_init(const dem_bed_config *beds, int32_t n_beds, const dem_parcels *p, const dem_gas *g,
             int32_t precision, void *cuda_stream, dem_ctx **out) {
  if (!out) return DEM_EINVAL;
  *out = nullptr;
  if (!beds || !p || n_beds < 1 || n_beds > DEM_MAX_BEDS || p->n <= 0) return DEM_EINVAL;
  if (precision != DEM_PREC_FP64 && precision != DEM_PREC_SPLIT && precision != DEM_PREC_SPLIT_KAHAN) return DEM_EINVAL;
  if (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz || !p->d_real || !p->T || !p->ore_type || !p->bed)
    return DEM_EINVAL;
  for (int q = 0; q < 4; ++q) if (!p->m0[q]) return DEM_EINVAL;
  for (int b = 0; b < n_beds; ++b) {
    int s = validate_bed(beds[b]);
    if (s != DEM_OK) return s;
  }
  const int n = p->n;
  // stage the parcel arrays on the host for validation
  std::vector<double> h[12];
  std::vector<int> hore(n), hbed(n);
  const double *srcs[12] = {p->x, p->y, p->z, p->vx, p->vy, p->vz, p->d_real, p->T, p->m0[0], p->m0[1], p->m0[2], p->m0[3]};
  for (int k = 0; k < 12; ++k) {
    h[k].resize(n);
    if (p->on_device) {
      if (cudaMemcpy(h[k].data(), srcs[k], sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return DEM_ECUDA;
    } else {
      std::memcpy(h[k].data(), srcs[k], sizeof(double) * n);
    }
  }
  if (p->on_device) {
    if (cudaMemcpy(hore.data(), p->ore_type, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return DEM_ECUDA;
    if (cudaMemcpy(hbed.data(), p->bed, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return DEM_ECUDA;
  } else {
    std::memcpy(hore.data(), p->ore_type, sizeof(int) * n);
    std::memcpy(hbed.data(), p->bed, sizeof(int) * n);
  }
  std::vector<double> dmax(n_beds, 0.0), mmin(n_beds, 1e300);
  std::vector<long long> nb(n_beds, 0);
  for (int i = 0; i < n; ++i) {
    const int b = hbed[i];
    if (b < 0 || b >= n_beds || (hore[i] != 0 && hore[i] != 1)) return DEM_EINVAL;
    const dem_bed_config &B = beds[b];
    for (int k = 0; k < 12; ++k) if (!std::isfinite(h[k][i])) return DEM_EINVAL;
    const double d = h[6][i];
    if (!(d > 0) || !(h[7][i] > 0)) return DEM_EINVAL;
    double m = 0.0;
    for (int q = 0; q < 4; ++q) { if (h[8 + q][i] < 0) return DEM_EINVAL; m += h[8 + q][i]; }
    if (!(m > 0)) return DEM_EINVAL;
    const double r = 0.5 * B.cg_ratio * d;
    const double rho = std::sqrt(h[0][i] * h[0][i] + h[1][i] * h[1][i]);
    if (!(rho <= 0.5 * B.bed_D && h[2][i] >= 0.0 && h[2][i] <= B.bed_H)) return DEM_EINVAL;
    (void)r;
    dmax[b] = std::max(dmax[b], B.cg_ratio * d);
    mmin[b] = std::min(mmin[b], m);
    nb[b]++;
  }
  dem_ctx *c = new dem_ctx();
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
      c->nsm = nsm;
  }
  c->n = n;
  c->cap = n;
  c->nbeds = n_beds;
  c->prec = precision;
  c->rsize = precision == DEM_PREC_FP64 ? sizeof(double) : sizeof(float);
  c->st = (cudaStream_t)cuda_stream;
  c->cfg.assign(beds, beds + n_beds);
  int nsolve = 0;
  for (int b = 0; b < n_beds; ++b) {
    c->any_rad = c->any_rad || (beds[b].flags & DEM_RADIATION) != 0;
    c->any_cond = c->any_cond || (beds[b].flags & DEM_CONDUCTION) != 0;
    if (beds[b].flags & DEM_GAS_SOLVER) {
      ++nsolve;
      if (beds[b].coupling_interval != beds[0].coupling_interval) { delete c; return DEM_EINVAL; }
    }
  }
  // the gas solver runs for every bed or for none, on one coupling interval
  if (nsolve != 0 && nsolve != n_beds) { delete c; return DEM_EINVAL; }
  c->gas_solver = nsolve > 0;
  // per-bed constants and grid offsets; the gas cells are the cell list of the contact
  // search, so no parcel may be wider than a cell edge
  long long coff = 0, pacc = 0;
  for (int b = 0; b < n_beds; ++b) {
    DevBed B = derive_bed(beds[b]);
    const double edge = std::min(B.dx, std::min(B.dy, B.dz));
    if (nb[b] > 0 && dmax[b] > edge) { delete c; return DEM_EINVAL; }
    // stability of the stiffest contact: omega_0 dt < 2 with m* = m_min / 2
    if (nb[b] > 0 && std::sqrt(beds[b].kn / (0.5 * mmin[b])) * beds[b].dt >= 2.0) { delete c; return DEM_EINVAL; }
    B.cell_off = coff;
    B.fx_off = c->gsv.nfx;
    B.fy_off = c->gsv.nfy;
    B.fz_off = c->gsv.nfz;
    c->gsv.nfx += (long long)(B.nx + 1) * B.ny * B.nz;
    c->gsv.nfy += (long long)B.nx * (B.ny + 1) * B.nz;
    c->gsv.nfz += (long long)B.nx * B.ny * (B.nz + 1);
    B.pstart = (int)pacc;
    pacc += nb[b];
    B.pend = (int)pacc;
    coff += (long long)B.nx * B.ny * B.nz;
    B.cornerp_off = (int)c->hcornerp.size();
    {
      const int nn[3] = {B.nx, B.ny, B.nz};
      const double hh[3] = {B.dx, B.dy, B.dz};
      for (int a = 0; a < 3; ++a)
        for (int q = 0; q <= nn[a]; ++q) {
          const double cv = q * hh[a];
          const float hi = (float)cv;
          c->hcornerp.push_back(make_float2(hi, (float)(cv - (double)hi)));
        }
    }
    B.corner_off = (int)c->hcorner.size();
    B.inv_nx_f = 1.0f / (float)B.nx;
    B.inv_nxy_f = 1.0f / (float)((long long)B.nx * B.ny);
    B.fast_offsets = (B.nx >= 5 && B.ny >= 5 && (long long)B.nx * B.ny < (1 << 22)) ? 1 : 0;
    for (int q = 0; q < B.nx; ++q) c->hcorner.push_back(B.x0 + q * B.dx);
    for (int q = 0; q < B.ny; ++q) c->hcorner.push_back(B.y0 + q * B.dy);
    for (int q = 0; q < B.nz; ++q) c->hcorner.push_back(B.z0 + q * B.dz);
    c->hbeds.push_back(B);
    c->hbp_d.push_back(derive_params<double>(beds[b], B));
    c->hbp_f.push_back(derive_params<float>(beds[b], B));
    c->hbp_d.back().reach_max = 0.5 * dmax[b];
    c->hbp_f.back().reach_max = (float)(0.5 * dmax[b]);
    set_skin(c->hbp_d.back(), c->skin_frac * dmax[b]);
    set_skin(c->hbp_f.back(), c->skin_frac * dmax[b]);
  }
  if (coff >= (1LL << 31)) { delete c; return DEM_EINVAL; }
  c->ncells = coff;
  c->key_bits = 1;
  while ((1LL << c->key_bits) < coff) ++c->key_bits;
  if (c->gas_solver) {
    // multigrid levels of the pressure preconditioner: halve every bed's dims (rounding up)
    // until each bed is one cell
    for (int b = 0; b < n_beds; ++b)
      c->hlb.push_back({c->hbeds[b].nx, c->hbeds[b].ny, c->hbeds[b].nz, c->hbeds[b].cell_off});
    c->hlev.assign(1, GsLevel{});
    for (;;) {
      const GsLevelBed *prev = &c->hlb[(c->hlev.size() - 1) * n_beds];
      bool single = true;
      for (int b = 0; b < n_beds; ++b) single = single && prev[b].nx == 1 && prev[b].ny == 1 && prev[b].nz == 1;
      if (single || (int)c->hlev.size() == GS_MAXLEV) break;
      long long off = 0;
      std::vector<GsLevelBed> nxt(n_beds);
      for (int b = 0; b < n_beds; ++b) {
        nxt[b] = {(prev[b].nx + 1) / 2, (prev[b].ny + 1) / 2, (prev[b].nz + 1) / 2, off};
        off += (long long)nxt[b].nx * nxt[b].ny * nxt[b].nz;
      }
      c->hlb.insert(c->hlb.end(), nxt.begin(), nxt.end());
      GsLevel Lv{};
      Lv.n = off;
      c->hlev.push_back(Lv);
    }
  }
  c->gsv.mg_nu = 2;        // preconditioner of the gas pressure solve (tuning entries 9, 10)
  c->gsv.mg_alpha = 1.5;   // the Galerkin aggregates' coarse correction falls short; over-correct
  if (c->gas_solver) {   // the cooperative pressure solve: no more blocks than fit at once
    int per_sm = 0;
    if (DEM_DISPATCH(c, gas_cg_occupancy, &per_sm) != 0 || per_sm < 1) { delete c; return DEM_ECUDA; }
    const long long need = (c->ncells + GS_CG_BLOCK - 1) / GS_CG_BLOCK;
    c->gs_grid = (int)std::max(1LL, std::min(need, (long long)per_sm * c->nsm));
  }
  // arena
  Bump meas;
  layout(c, meas);
  c->arena_bytes = meas.off + 256;
  if (cudaMalloc(&c->arena, c->arena_bytes) != cudaSuccess) { dem_destroy(c); return DEM_ENOMEM; }
  Bump real;
  real.base = c->arena;
  layout(c, real);
  if (cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) { dem_destroy(c); return DEM_ENOMEM; }
  *c->h_err = 0;
  if (cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_main, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_gas, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->sst, cudaStreamNonBlocking) != cudaSuccess) {
    dem_destroy(c);
    return DEM_ECUDA;
  }
  int rc = DEM_OK;
  auto ck = [&](cudaError_t e) { if (e != cudaSuccess && rc == DEM_OK) rc = e == cudaErrorMemoryAllocation ? DEM_ENOMEM : DEM_ECUDA; };
  ck(cudaMemcpyAsync(c->dbeds, c->hbeds.data(), sizeof(DevBed) * n_beds, cudaMemcpyHostToDevice, c->st));
  ck(cudaMemcpyAsync(c->dbp_d, c->hbp_d.data(), sizeof(BedP<double>) * n_beds, cudaMemcpyHostToDevice, c->st));
  ck(cudaMemcpyAsync(c->dbp_f, c->hbp_f.data(), sizeof(BedP<float>) * n_beds, cudaMemcpyHostToDevice, c->st));
  ck(cudaMemcpyAsync(c->corner, c->hcorner.data(), sizeof(double) * c->hcorner.size(), cudaMemcpyHostToDevice, c->st));
  ck(cudaMemcpyAsync(c->cornerp, c->hcornerp.data(), sizeof(float2) * c->hcornerp.size(), cudaMemcpyHostToDevice, c->st));
  // staging copies of the inputs (freed at the end of init)
  double *dsrc = nullptr;
  int *dint = nullptr;
  const double **dptrs = nullptr;
  ck(cudaMalloc(&dsrc, sizeof(double) * 12 * (size_t)n));
  ck(cudaMalloc(&dint, sizeof(int) * 2 * (size_t)n));
  ck(cudaMalloc(&dptrs, sizeof(double *) * 12));
  if (rc != DEM_OK) { cudaFree(dsrc); cudaFree(dint); cudaFree(dptrs); dem_destroy(c); return rc; }
  const double *hp[12];
  for (int k = 0; k < 12; ++k) {
    ck(cudaMemcpyAsync(dsrc + (size_t)k * n, h[k].data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
    hp[k] = dsrc + (size_t)k * n;
  }
  ck(cudaMemcpyAsync(dint, hore.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
  ck(cudaMemcpyAsync(dint + n, hbed.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
  ck(cudaMemcpyAsync(dptrs, hp, sizeof(hp), cudaMemcpyHostToDevice, c->st));
  const int bs = 256, gridn = (n + bs - 1) / bs;
  void **drv = nullptr;   // 14 state-row pointers and 4 mass pointers for k_load
  ck(cudaMalloc(&drv, sizeof(void *) * 18));
  {
    void *hrv[18] = {c->pv[0][0], c->pv[0][1], c->pv[0][2], c->pw[0][0], c->pw[0][1], c->pw[0][2],
                     c->pa[0][0], c->pa[0][1], c->pa[0][2], c->pal[0][0], c->pal[0][1], c->pal[0][2],
                     c->pT[0], c->pd[0], c->pm[0][0], c->pm[0][1], c->pm[0][2], c->pm[0][3]};
    ck(cudaMemcpyAsync(drv, hrv, sizeof(hrv), cudaMemcpyHostToDevice, c->st));
  }
  if (rc == DEM_OK) {
    if (c->prec == DEM_PREC_FP64)
      k_load<PrecF64><<<gridn, bs, 0, c->st>>>(n, dptrs, dint, dint + n, c->dbeds, c->px[0][0], c->px[0][1], c->px[0][2],
                                               (double *const *)drv, (double *const *)(drv + 14), c->pmeta[0], c->porig[0]);
    else if (c->prec == DEM_PREC_SPLIT)
      k_load<PrecSplit><<<gridn, bs, 0, c->st>>>(n, dptrs, dint, dint + n, c->dbeds, c->px[0][0], c->px[0][1], c->px[0][2],
                                                 (float *const *)drv, (double *const *)(drv + 14), c->pmeta[0], c->porig[0]);
    else
      k_load<PrecKahan><<<gridn, bs, 0, c->st>>>(n, dptrs, dint, dint + n, c->dbeds, c->px[0][0], c->px[0][1], c->px[0][2],
                                                 (float *const *)drv, (double *const *)(drv + 14), c->pmeta[0], c->porig[0]);
  }
  ck(cudaMemsetAsync(c->hcnt[0], 0, (size_t)n, c->st));
  ck(cudaMemsetAsync(c->hcnt[1], 0, (size_t)n, c->st));
  ck(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
  ck(cudaMemsetAsync(c->step_ctr, 0, 6 * sizeof(long long), c->st));
  if (c->gas_solver) {
    ck(cudaMemsetAsync(c->gsv.cg_iters, 0, sizeof(int), c->st));
    ck(cudaMemcpyAsync(c->dlev, c->hlev.data(), sizeof(GsLevel) * c->hlev.size(), cudaMemcpyHostToDevice, c->st));
    ck(cudaMemcpyAsync(c->dlb, c->hlb.data(), sizeof(GsLevelBed) * c->hlb.size(), cudaMemcpyHostToDevice, c->st));
    for (size_t l = 1; l < c->hlev.size(); ++l) {   // bed of each coarse cell
      std::vector<int> bl((size_t)c->hlev[l].n);
      for (int b = 0; b < n_beds; ++b) {
        const GsLevelBed &g = c->hlb[l * n_beds + b];
        std::fill(bl.begin() + g.off, bl.begin() + g.off + (long long)g.nx * g.ny * g.nz, b);
      }
      ck(cudaMemcpy(c->dlbed[l], bl.data(), sizeof(int) * bl.size(), cudaMemcpyHostToDevice));
    }
    for (size_t l = 0; l + 1 < c->hlev.size(); ++l) {   // the coarse cell holding each cell
      const long long nl = l == 0 ? c->ncells : c->hlev[l].n;
      std::vector<int> par((size_t)nl, 0);
      for (int b = 0; b < n_beds; ++b) {
        const GsLevelBed &g = c->hlb[l * n_beds + b], &gc = c->hlb[(l + 1) * n_beds + b];
        for (int z = 0; z < g.nz; ++z)
          for (int y = 0; y < g.ny; ++y)
            for (int x = 0; x < g.nx; ++x)
              par[g.off + ((long long)z * g.ny + y) * g.nx + x] =
                  (int)(gc.off + ((long long)(z / 2) * gc.ny + y / 2) * gc.nx + x / 2);
      }
      ck(cudaMemcpy(c->dlpar[l], par.data(), sizeof(int) * par.size(), cudaMemcpyHostToDevice));
    }
  }
  // neighbour lists: none yet (the first step builds them); no displacement
  ck(cudaMemsetAsync(c->rebuild, 1, sizeof(int), c->st));
  for (int k = 0; k < 2; ++k) {
    for (int q = 0; q < 3; ++q) ck(cudaMemsetAsync(c->pdsp[k][q], 0, sizeof(float) * (size_t)n, c->st));
  }
  ck(cudaMemsetAsync(c->nlc, 0, (size_t)n, c->st));
  ck(cudaMemsetAsync(c->nwork, 0, sizeof(int), c->st));
  ck(cudaMemsetAsync(resort_counts(c->rsw, c->rs_pow2, n), 0, sizeof(int) * (size_t)((n + 1023) / 1024 + 1), c->st));
  // gas: cell -> bed, marks, initial state
  {
    std::vector<int> cb(c->ncells);
    for (int b = 0; b < n_beds; ++b) {
      const long long ng = (long long)c->hbeds[b].nx * c->hbeds[b].ny * c->hbeds[b].nz;
      std::fill(cb.begin() + c->hbeds[b].cell_off, cb.begin() + c->hbeds[b].cell_off + ng, b);
    }
    ck(cudaMemcpyAsync(c->cell_bed, cb.data(), sizeof(int) * c->ncells, cudaMemcpyHostToDevice, c->st));
    std::vector<double> Y((size_t)c->ncells * 3), T(c->ncells);
    if (g && g->Y && g->T) {
      if (g->on_device) {
        ck(cudaMemcpy(Y.data(), g->Y, sizeof(double) * Y.size(), cudaMemcpyDeviceToHost));
        ck(cudaMemcpy(T.data(), g->T, sizeof(double) * T.size(), cudaMemcpyDeviceToHost));
      } else {
        std::memcpy(Y.data(), g->Y, sizeof(double) * Y.size());
        std::memcpy(T.data(), g->T, sizeof(double) * T.size());
      }
    } else {
      for (long long cc = 0; cc < c->ncells; ++cc) {
        const dem_bed_config &B = beds[cb[cc]];
        for (int j = 0; j < 3; ++j) Y[cc * 3 + j] = B.Y_in[j];
        T[cc] = B.T_in;
      }
    }
    double *dY = nullptr, *dT = nullptr;
    ck(cudaMalloc(&dY, sizeof(double) * Y.size()));
    ck(cudaMalloc(&dT, sizeof(double) * T.size()));
    if (rc == DEM_OK) {
      ck(cudaMemcpyAsync(dY, Y.data(), sizeof(double) * Y.size(), cudaMemcpyHostToDevice, c->st));
      ck(cudaMemcpyAsync(dT, T.data(), sizeof(double) * T.size(), cudaMemcpyHostToDevice, c->st));
      const int gg = (int)((c->ncells + 255) / 256);
      k_gas_load<<<gg, 256, 0, c->st>>>(c->ncells, dY, dT, c->gas[0], c->prec != DEM_PREC_FP64);
      k_mark_cells<<<gg, 256, 0, c->st>>>(c->dbeds, c->dbp_d, c->cell_bed, c->mark, c->wnear, c->ncells);
    }
    ck(cudaStreamSynchronize(c->st));
    cudaFree(dY);
    cudaFree(dT);
  }
  c->cur = 0;
  c->gcur = 0;
  if (rc == DEM_OK) {
    int e = DEM_DISPATCH(c, enqueue_init, c);
    if (!e && c->gas_solver) e = DEM_DISPATCH(c, enqueue_gas_solver_init, c);
    if (e) rc = DEM_ECUDA;
  }
  ck(cudaStreamSynchronize(c->st));
  cudaFree(dsrc);
  cudaFree(dint);
  cudaFree(dptrs);
  cudaFree(drv);
  if (rc == DEM_OK) {
    int herr = 0;
    ck(cudaMemcpy(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (rc == DEM_OK && herr) rc = status_from_bits(herr);
  }
  if (rc != DEM_OK) { dem_destroy(c); return rc; }
  *out = c;
  return DEM_OK;
}

int dem_step(dem_ctx *c, int32_t n_steps) {
  if (!c || n_steps < 0) return DEM_EINVAL;
  int s = poll(c, false);
  if (s != DEM_OK) return s;
  c->launches = 0;
  if (enqueue_steps_any(c, n_steps)) return c->sticky = DEM_ECUDA;
  return mark_pending(c);
}

int dem_step_graph(dem_ctx *c, int32_t n_steps) {
  if (!c || n_steps <= 0) return DEM_EINVAL;
  int s = poll(c, false);
  if (s != DEM_OK) return s;
  const auto key = std::make_tuple((int)n_steps, c->cur, c->gcur);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    // capture on a private non-blocking stream (the legacy default stream cannot capture);
    // capturing records the kernels without running them
    if (!c->gst && cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking) != cudaSuccess) return c->sticky = DEM_ECUDA;
    const int cur0 = c->cur, gcur0 = c->gcur;
    cudaStream_t user = c->st;
    c->st = c->gst;
    c->launches = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { c->st = user; return c->sticky = DEM_ECUDA; }
    int e = enqueue_steps_any(c, n_steps);
    cudaError_t ce = cudaStreamEndCapture(c->st, &graph);
    c->st = user;
    if (e || ce != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return c->sticky = DEM_ECUDA; }
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) { cudaGraphDestroy(graph); return c->sticky = DEM_ECUDA; }
    it = c->graphs.emplace(key, std::make_pair(graph, exec)).first;
    c->graph_launches[key] = c->launches;
    c->cur = cur0;
    c->gcur = gcur0;
  }
  // the host-side bookkeeping advances as the captured steps do (the sorted keys of a state
  // buffer live in the key buffer of the same parity)
  for (int k = 0; k < n_steps; ++k) {
    c->cur = 1 - c->cur;
    c->gcur = 1 - c->gcur;
  }
  if (cudaGraphLaunch(it->second.second, c->st) != cudaSuccess) return c->sticky = DEM_ECUDA;
  c->gas_pending = false;   // every captured step graph waits for the coupling input's event
  c->launches = c->graph_launches[key];
  return mark_pending(c);
}

int dem_sync(dem_ctx *c) {
  if (!c) return DEM_EINVAL;
  return sync_all(c);
}

int dem_set_kinetics(dem_ctx *c, const double k0[3], const double Ea[3]) {
  if (!c || !k0 || !Ea) return DEM_EINVAL;
  for (int r = 0; r < 3; ++r)
    if (!(k0[r] >= 0 && Ea[r] >= 0)) return DEM_EINVAL;   // nothing changed
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  for (int b = 0; b < c->nbeds; ++b)
    for (int r = 0; r < 3; ++r) {
      c->hbp_d[b].k0[r] = k0[r];
      c->hbp_d[b].Ea_R[r] = Ea[r] / kRgas;
      c->hbp_f[b].k0[r] = (float)k0[r];
      c->hbp_f[b].Ea_R[r] = (float)(Ea[r] / kRgas);
      c->cfg[b].k0[r] = k0[r];
      c->cfg[b].Ea[r] = Ea[r];
    }
  CK(cudaMemcpyAsync(c->dbp_d, c->hbp_d.data(), sizeof(BedP<double>) * c->nbeds, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->dbp_f, c->hbp_f.data(), sizeof(BedP<float>) * c->nbeds, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return DEM_OK;
}

static int ensure_scratch(dem_ctx *c, size_t bytes) {
  if (c->scratch_bytes >= bytes) return DEM_OK;
  if (c->scratch_out) cudaFree(c->scratch_out);
  c->scratch_out = nullptr;
  c->scratch_bytes = 0;
  if (cudaMalloc(&c->scratch_out, bytes) != cudaSuccess) return DEM_ENOMEM;
  c->scratch_bytes = bytes;
  return DEM_OK;
}

int dem_reduction_degree(dem_ctx *c, double *mean_per_bed, double *oxygen_per_bed, double *per_parcel) {
  if (!c || !mean_per_bed) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  int e = DEM_DISPATCH(c, enqueue_fov, c, per_parcel);
  if (e) return DEM_ECUDA;
  std::vector<double> hb((size_t)c->nbeds * 4);
  CK(cudaMemcpyAsync(hb.data(), c->fvbed, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int b = 0; b < c->nbeds; ++b) {
    const double cnt = hb[b * 4 + 3];
    mean_per_bed[b] = cnt > 0 ? hb[b * 4 + 0] / cnt : 0.0;
    if (oxygen_per_bed) oxygen_per_bed[b] = hb[b * 4 + 2] > 0 ? 1.0 - hb[b * 4 + 1] / hb[b * 4 + 2] : 0.0;
  }
  return DEM_OK;
}

int dem_get_state(dem_ctx *c, double *out_host) {
  if (!c || !out_host) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  const size_t bytes = sizeof(double) * DEM_NSTATE * (size_t)c->n;
  if ((s = ensure_scratch(c, bytes)) != DEM_OK) return s;
  int e = DEM_DISPATCH(c, enqueue_scatter_state, c, c->scratch_out);
  if (e) return DEM_ECUDA;
  CK(cudaMemcpyAsync(out_host, c->scratch_out, bytes, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return DEM_OK;
}

int64_t dem_num_cells(dem_ctx *c) { return c ? c->ncells : 0; }

int dem_get_gas(dem_ctx *c, double *out_host) {
  if (!c || !out_host) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  const size_t nc = (size_t)c->ncells;
  std::vector<double> G(nc * GS_N);
  std::vector<unsigned char> mk(nc);
  CK(cudaMemcpyAsync(G.data(), c->gas[c->gcur], sizeof(double) * G.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(mk.data(), c->mark, nc, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (size_t k = 0; k < nc; ++k) {
    for (int f = 0; f < GS_N; ++f) {
      double v = G[f * nc + k];
      if (c->prec != DEM_PREC_FP64) {   // FP32 forms: (value, compensation) pair of FP32
        float p[2];
        std::memcpy(p, &v, sizeof p);
        v = (double)p[0] + (double)p[1];
      }
      out_host[k * DEM_NGAS + f] = v;
    }
    out_host[k * DEM_NGAS + 5] = mk[k];
  }
  return DEM_OK;
}

int dem_get_sources(dem_ctx *c, double *out_host) {
  if (!c || !out_host) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  if (!c->dep && cudaMalloc(&c->dep, sizeof(double) * SR_N * (size_t)c->ncells) != cudaSuccess) return DEM_ENOMEM;
  int e = DEM_DISPATCH(c, enqueue_sources, c);
  if (e) return DEM_ECUDA;
  CK(cudaMemcpyAsync(out_host, c->dep, sizeof(double) * SR_N * (size_t)c->ncells, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return DEM_OK;
}

int dem_get_sources_occupied(dem_ctx *c, int64_t cap, int64_t *n_occupied, int64_t *cells_host, double *out_host) {
  if (!c || !n_occupied || cap < 0 || (cap > 0 && (!cells_host || !out_host))) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  const size_t nmax = (size_t)std::min<long long>(c->n, c->ncells);
  const int nb = (c->n + OCC_CHUNK - 1) / OCC_CHUNK;
  const size_t cells_off = ((sizeof(int) * (size_t)(nb + 1) + 255) / 256) * 256;
  const size_t out_off = cells_off + ((sizeof(long long) * nmax + 255) / 256) * 256;
  if ((s = ensure_scratch(c, out_off + sizeof(double) * SR_N * nmax)) != DEM_OK) return s;
  char *base = (char *)c->scratch_out;
  int *cnt = (int *)base;
  long long *dcells = (long long *)(base + cells_off);
  double *dout = (double *)(base + out_off);
  int e = DEM_DISPATCH(c, enqueue_sources_occupied, c, cnt, dcells, dout);
  if (e) return DEM_ECUDA;
  int n = 0;
  CK(cudaMemcpyAsync(&n, cnt + nb, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  *n_occupied = n;
  if (n > cap) return DEM_EINVAL;   // the count is reported; nothing else is written
  if (n > 0) {
    CK(cudaMemcpyAsync(cells_host, dcells, sizeof(long long) * (size_t)n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(out_host, dout, sizeof(double) * SR_N * (size_t)n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
  }
  return DEM_OK;
}

int dem_get_flow(dem_ctx *c, double *out_host, int32_t *iters) {
  if (!c || !out_host) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  const size_t bytes = sizeof(double) * 4 * (size_t)c->ncells;
  if ((s = ensure_scratch(c, bytes)) != DEM_OK) return s;
  int e = DEM_DISPATCH(c, enqueue_flow, c, c->scratch_out);
  if (e) return DEM_ECUDA;
  CK(cudaMemcpyAsync(out_host, c->scratch_out, bytes, cudaMemcpyDeviceToHost, c->st));
  int it = 0;
  if (c->gas_solver) CK(cudaMemcpyAsync(&it, c->gsv.cg_iters, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (iters) *iters = it;
  return DEM_OK;
}

int dem_get_contacts(dem_ctx *c, int32_t *count, int32_t *partner, double *xi) {
  if (!c || !count || !partner || !xi) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  const size_t n = (size_t)c->n;
  const size_t bytes = n * sizeof(int) + n * KMAX * sizeof(int) + n * KMAX * 3 * sizeof(double) + 512;
  if ((s = ensure_scratch(c, bytes)) != DEM_OK) return s;
  char *base = (char *)c->scratch_out;
  double *dxi = (double *)base;
  int *dcnt = (int *)(base + n * KMAX * 3 * sizeof(double));
  int *dpart = dcnt + n;
  int e = DEM_DISPATCH(c, enqueue_scatter_hist, c, dcnt, dpart, dxi);
  if (e) return DEM_ECUDA;
  CK(cudaMemcpyAsync(count, dcnt, n * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(partner, dpart, n * KMAX * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(xi, dxi, n * KMAX * 3 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  // slots sorted by partner
  for (size_t i = 0; i < n; ++i) {
    const int cnt = count[i];
    std::vector<std::pair<int, int>> ord(cnt);
    for (int k = 0; k < cnt; ++k) ord[k] = {partner[i * KMAX + k], k};
    std::sort(ord.begin(), ord.end());
    std::vector<int> p2(cnt);
    std::vector<double> x2((size_t)cnt * 3);
    for (int k = 0; k < cnt; ++k) {
      p2[k] = ord[k].first;
      for (int q = 0; q < 3; ++q) x2[(size_t)k * 3 + q] = xi[(i * KMAX + ord[k].second) * 3 + q];
    }
    for (int k = 0; k < cnt; ++k) {
      partner[i * KMAX + k] = p2[k];
      for (int q = 0; q < 3; ++q) xi[(i * KMAX + k) * 3 + q] = x2[(size_t)k * 3 + q];
    }
  }
  return DEM_OK;
}

int dem_set_diagnostics(dem_ctx *c, int32_t on) {
  if (!c) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  if (on && !c->diag) {
    if (cudaMalloc(&c->diag, sizeof(double) * DG_N * (size_t)c->cap) != cudaSuccess) return DEM_ENOMEM;
    CK(cudaMemset(c->diag, 0, sizeof(double) * DG_N * (size_t)c->cap));
  }
  if (c->diag_on != (on != 0)) {
    drop_graphs(c);   // captured graphs bake the diagnostics pointer in
  }
  c->diag_on = on != 0;
  return DEM_OK;
}

int dem_get_diag(dem_ctx *c, double *out_host) {
  if (!c || !out_host) return DEM_EINVAL;
  if (!c->diag) return DEM_ESTATE;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  const size_t bytes = sizeof(double) * DG_N * (size_t)c->n;
  if ((s = ensure_scratch(c, bytes)) != DEM_OK) return s;
  int e = DEM_DISPATCH(c, enqueue_scatter_diag, c, c->scratch_out);
  if (e) return DEM_ECUDA;
  CK(cudaMemcpyAsync(out_host, c->scratch_out, bytes, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return DEM_OK;
}

int64_t dem_last_launch_count(dem_ctx *c) { return c ? c->launches : 0; }

int dem_set_gas(dem_ctx *c, const dem_gas *g) {
  if (!c || !g || !g->Y || !g->T) return DEM_EINVAL;
  if (c->gas_solver) return DEM_EINVAL;   // the gas is solved here
  int s = poll(c, false);
  if (s != DEM_OK) return s;
  const size_t nc = (size_t)c->ncells;
  const double *Y = g->Y, *T = g->T;
  // on the input's own stream, after everything the context stream holds so far (the last
  // step's gas update): host arrays cross by a copy engine into the staging buffer (no SM is
  // needed, so the transfer overlaps the next step's binning and contact kernels), then one
  // kernel writes the gas state and the cell properties
  CK(cudaEventRecord(c->ev_main, c->st));
  CK(cudaStreamWaitEvent(c->sst, c->ev_main, 0));
  if (!g->on_device) {
    if (!c->gas_stage && cudaMalloc(&c->gas_stage, sizeof(double) * 4 * nc) != cudaSuccess) return DEM_ENOMEM;
    CK(cudaMemcpyAsync(c->gas_stage, g->Y, sizeof(double) * 3 * nc, cudaMemcpyHostToDevice, c->sst));
    CK(cudaMemcpyAsync(c->gas_stage + 3 * nc, g->T, sizeof(double) * nc, cudaMemcpyHostToDevice, c->sst));
    Y = c->gas_stage;
    T = c->gas_stage + 3 * nc;
  }
  int e = DEM_DISPATCH(c, enqueue_gas_set, c, Y, T, c->sst);
  if (e) return c->sticky = DEM_ECUDA;
  CK(cudaEventRecord(c->ev_gas, c->sst));
  c->gas_pending = true;
  return DEM_OK;
}

int dem_profile(dem_ctx *c, int32_t on) {
  if (!c) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  c->prof_on = on != 0;
  c->prof_marks.clear();
  c->prof_names.clear();
  c->prof_ms.clear();
  c->prof_n.clear();
  return DEM_OK;
}

int dem_kernel_times(dem_ctx *c, int32_t max_kernels, char *names, int64_t *launches, double *ms_total) {
  if (!c || max_kernels < 0) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  for (const auto &mk : c->prof_marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[mk.second], c->ev_pool[mk.second + 1]) != cudaSuccess) return DEM_ECUDA;
    c->prof_ms[mk.first] += ms;
    c->prof_n[mk.first] += 1;
  }
  c->prof_marks.clear();
  const int k = (int)c->prof_names.size();
  for (int i = 0; i < k && i < max_kernels; ++i) {
    if (names) {
      std::memset(names + 32 * i, 0, 32);
      std::strncpy(names + 32 * i, c->prof_names[i].c_str(), 31);
    }
    if (launches) launches[i] = c->prof_n[i];
    if (ms_total) ms_total[i] = c->prof_ms[i];
  }
  return k;
}

int dem_get_tuning(dem_ctx *c, int32_t *out) {
  if (!c || !out) return DEM_EINVAL;
  get_tuning(c, out);
  return DEM_OK;
}

int dem_set_tuning(dem_ctx *c, const int32_t *in) {
  if (!c || !in) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  return apply_tuning(c, in);
}

int dem_get_counters(dem_ctx *c, int64_t *out) {
  if (!c || !out) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  long long v[3];
  CK(cudaMemcpyAsync(v, c->step_ctr, sizeof v, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int k = 0; k < 3; ++k) out[k] = v[k];
  return DEM_OK;
}

int dem_autotune(dem_ctx *c, int32_t n_steps) {
  if (!c || n_steps < 1) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  void *snap = nullptr;
  if (cudaMalloc(&snap, c->arena_bytes) != cudaSuccess) return DEM_ENOMEM;
  CK(cudaMemcpyAsync(snap, c->arena, c->arena_bytes, cudaMemcpyDeviceToDevice, c->st));
  const int cur0 = c->cur, gcur0 = c->gcur;
  const bool prof0 = c->prof_on;
  int32_t best[DEM_NTUNE];
  get_tuning(c, best);
  int rc = DEM_OK;
  auto restore = [&]() {
    cudaMemcpyAsync(c->arena, snap, c->arena_bytes, cudaMemcpyDeviceToDevice, c->st);
    c->cur = cur0; c->gcur = gcur0;
  };
  // one candidate: per-kernel mean times (ms) and the total, or a negative total on error
  auto trial = [&](const int32_t *t, std::map<std::string, double> &per, int steps) -> double {
    restore();
    if (apply_tuning(c, t) != DEM_OK) return -1.0;
    c->prof_on = true;
    c->prof_marks.clear(); c->prof_names.clear(); c->prof_ms.clear(); c->prof_n.clear();
    if (enqueue_steps_any(c, steps) != 0) { c->prof_on = false; return -1.0; }
    if (cudaStreamSynchronize(c->st) != cudaSuccess) { c->prof_on = false; return -1.0; }
    c->prof_on = false;
    for (const auto &mk : c->prof_marks) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->ev_pool[mk.second], c->ev_pool[mk.second + 1]);
      c->prof_ms[mk.first] += ms;
      c->prof_n[mk.first] += 1;
    }
    double tot = 0.0;
    per.clear();
    for (size_t k = 0; k < c->prof_names.size(); ++k) {
      per[c->prof_names[k]] = c->prof_ms[k] / (double)std::max<long long>(1, c->prof_n[k]);
      tot += c->prof_ms[k];
    }
    return tot;
  };
  // 1) block sizes, every per-thread kernel at once, each kernel keeping its fastest
  const char *kname[6] = {"k_key", "k_restore", "k_pair_search", "k_contact_screen", "k_gas_particle", "k_cells"};
  double bt[6];
  for (int k = 0; k < 6; ++k) bt[k] = 1e300;
  int32_t tb[DEM_NTUNE];
  std::memcpy(tb, best, sizeof tb);
  tb[0] = 1;
  int lim[6];
  if (DEM_DISPATCH(c, kernel_limits, lim) != 0) rc = DEM_ECUDA;
  for (int bs : {64, 128, 256, 512}) {
    if (rc != DEM_OK) break;
    int32_t t[DEM_NTUNE];
    std::memcpy(t, tb, sizeof t);
    for (int k = 1; k <= 6; ++k) t[k] = std::min(bs, lim[k - 1] / 32 * 32);
    std::map<std::string, double> per;
    if (trial(t, per, n_steps) < 0) { rc = DEM_ECUDA; break; }
    for (int k = 0; k < 6; ++k) {
      auto it = per.find(kname[k]);
      if (it != per.end() && it->second < bt[k]) { bt[k] = it->second; best[1 + k] = t[1 + k]; }
    }
  }
  // 2) skin of the neighbour lists (whole-step time: rebuilds against list length)
  double best_tot = 1e300;
  if (rc == DEM_OK) {
    const int32_t skin0 = best[7];
    for (int sk : {25, 50, 100, 200}) {
      int32_t t[DEM_NTUNE];
      std::memcpy(t, best, sizeof t);
      t[0] = 1;
      t[7] = sk;
      std::map<std::string, double> per;
      const double tot = trial(t, per, 4 * n_steps);   // rebuilds amortise over long windows
      if (tot < 0) { rc = DEM_ECUDA; break; }
      if (tot < best_tot) { best_tot = tot; best[7] = sk; }
    }
    if (rc != DEM_OK) best[7] = skin0;
  }
  // 3) re-store interval (whole-step time over long windows, as the skin)
  if (rc == DEM_OK) {
    const int32_t re0 = best[8];
    double bt_re = 1e300;
    for (int re : {1, 2, 4, 8}) {
      int32_t t[DEM_NTUNE];
      std::memcpy(t, best, sizeof t);
      t[0] = 1;
      t[8] = re;
      std::map<std::string, double> per;
      const double tot = trial(t, per, 4 * n_steps);
      if (tot < 0) { rc = DEM_ECUDA; break; }
      if (tot < bt_re) { bt_re = tot; best[8] = re; }
    }
    if (rc != DEM_OK) best[8] = re0;
    else best_tot = bt_re;
  }
  // 4) the cell-list search every step (no lists) against the best list configuration
  best[0] = 1;
  if (rc == DEM_OK) {
    int32_t t[DEM_NTUNE];
    std::memcpy(t, best, sizeof t);
    t[0] = 0;
    std::map<std::string, double> per;
    const double tot = trial(t, per, 4 * n_steps);
    if (tot < 0) rc = DEM_ECUDA;
    else if (tot < best_tot) best[0] = 0;
  }
  restore();
  if (rc == DEM_OK) rc = apply_tuning(c, best);
  cudaStreamSynchronize(c->st);
  cudaFree(snap);
  c->prof_marks.clear(); c->prof_names.clear(); c->prof_ms.clear(); c->prof_n.clear();
  c->prof_on = prof0;
  if (rc != DEM_OK) c->sticky = rc;
  return rc;
}

int dem_adjoint(dem_ctx *c, int32_t n_steps, int32_t ckpt_every, double *J, double *grad) {
  if (!c || !J || n_steps < 0 || ckpt_every < 1) return DEM_EINVAL;
  // radiation and conduction couple the parcels (the map is per parcel); the gas solver
  // couples them through the gas
  if (c->any_rad || c->any_cond || c->gas_solver) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  return DEM_DISPATCH(c, run_adjoint, c, n_steps, ckpt_every, J, grad);
}

int dem_adjoint_obs(dem_ctx *c, int32_t n_steps, int32_t ckpt_every, int32_t n_obs, const int32_t *obs_steps,
                    const double *weights, double *J_obs, double *grad) {
  if (!c || n_steps < 1 || ckpt_every < 1 || n_obs < 1 || n_obs > DEM_MAX_OBS || !obs_steps || !J_obs)
    return DEM_EINVAL;
  if (grad && !weights) return DEM_EINVAL;
  for (int k = 0; k < n_obs; ++k)
    if (obs_steps[k] < 1 || obs_steps[k] > n_steps || (k > 0 && obs_steps[k] <= obs_steps[k - 1])) return DEM_EINVAL;
  if (weights)
    for (int k = 0; k < n_obs * c->nbeds; ++k)
      if (!std::isfinite(weights[k])) return DEM_EINVAL;
  if (c->any_rad || c->any_cond || c->gas_solver) return DEM_EINVAL;
  int s = sync_all(c);
  if (s != DEM_OK) return s;
  std::vector<int> st(obs_steps, obs_steps + n_obs);
  return DEM_DISPATCH(c, run_adjoint, c, n_steps, ckpt_every, nullptr, grad, n_obs, st.data(), weights, J_obs);
}

}  // extern "C"
