// kernels.cuh -- the per-step kernels of the particle path, templated on the precision
// policy P (PrecF64, PrecSplit, PrecKahan; see common.cuh). Instantiated in inst_*.cu,
// launched by launch.cuh.
#pragma once
#include "common.cuh"

namespace dem {

// One parcel-state buffer, structure of arrays. The parcels stay where they are between
// neighbour-list builds ("storage order"); each build re-stores them in the sorted order of
// that step, so the storage order is always the cell order of the last build, and parcels
// have moved less than half the skin since.
template <class R> struct PState {
  double *x, *y, *z;
  R *v[3], *w[3], *a[3], *al[3], *T, *d;
  double *m[4];  // FP64 masses, or (value, compensation) FP32 pairs in the split-Kahan form
  int *meta;     // bed << 8 | ore
  int *orig;     // parcel index (input order)
  float *dsp[3]; // displacement since the last list build (FP32)
};

// Verlet neighbour lists: slots per parcel, and the count that marks an overflowed list
constexpr int KNL = 32;
constexpr int NL_OVERFLOW = 255;

// Contact-history table: count per parcel, then KMAX slots of partner index and 3-vector.
template <class R> struct Hist {
  unsigned char *cnt;
  int *id;     // [KMAX][cap]
  R *xi;       // [KMAX*3][cap]
};

// Everything a step's kernels touch. Parcel arrays are indexed by storage position; the
// cell ranges and sorted keys by sorted position (vals maps sorted to storage positions).
template <class P> struct StepView {
  using R = typename P::R;
  int n, cap, nbeds;
  long long ncells;
  const DevBed *beds;
  const BedP<R> *bp;
  PState<R> A, S;               // A: the state (updated in place); S: scratch of a re-store
  Hist<R> H, Hn;                // H: history before the step, Hn: after it
  Hist<R> Hs;                   // scratch of a re-store
  unsigned *keyp;               // gas-cell key of each parcel (storage order)
  unsigned *keys, *vals;        // sorted keys and the storage position at each sorted position
  const unsigned *keys_prev, *vals_prev;   // the same for the previous step
  unsigned *knew;               // re-sort input: new keys in the previous sorted order
  unsigned *inv;                // sorted position of each storage position (previous sort until
                                // the ranges kernel of this step rewrites it)
  unsigned *cstart, *cend;      // sorted-position range of every gas cell (empty: 0, 0)
  float4 *xl;                   // FP32 position relative to the own cell's corner, radius
  R *F[3], *Tq[3];              // contact force and torque
  float4 *xls;                  // scratch of a re-store (aliases the per-parcel sources,
                                // which the gas-particle kernel rewrites later in the step)
  int *plist;                   // [KLIST][cap] partners in contact range this step
  unsigned char *pcode;         // [KLIST][cap] their cell offset codes
  unsigned char *pcnt;          // number of them per parcel
  int *nl;                      // [KNL][cap] neighbour lists (storage positions)
  unsigned char *nlc;           // list lengths (NL_OVERFLOW: none, search the cells)
  int *rebuild;                 // device flag: rebuild the lists (and re-store) this step
  int nolists;                  // search the cell list every step instead of using lists
  const double *corner;         // cell-corner coordinates (see DevBed::corner_off)
  const float2 *cornerp;        // cell corners relative to the bed corner, FP32 pairs
  int *moved;                   // per 1024 sorted positions: keys that changed (re-sort)
  R *src;                       // [SR_CNT][cap] per-parcel cell sources (the count is je - jb)
  double *gas, *gas_new;        // [GS_N][ncells]
  R *gp;                        // [GP_N][ncells]
  unsigned char *mark;          // solid (IBM) cell mark
  int *cell_bed;                // bed of each gas cell
  double *diag;                 // [DG_N][cap] or null
  double *dep;                  // [ncells][SR_N] or null (written by k_sources)
  int *err;
  const long long *step_ctr;    // steps completed so far (device); [4] list builds since the last re-store
  int restore_every;            // the state is re-stored in cell order at every k-th list build
  unsigned long long *list_acc; // list entries of the build in progress
  int *ovf, *novf;              // parcels whose list overflowed at the last build, and their count
  uint2 *work;                  // contact work list: (parcel, list-hit mask) ...
  int *nwork;                   // ... and its length (reset by the step counter)
  const unsigned char *wnear;   // per cell: a wall may be within a parcel's reach
  R *qrad;                      // radiation heat of each parcel this step (radiating beds)
  float4 *xr;                   // radiation: local coordinates in sorted order, w = T (FP32 forms)
  R *tsrt;                      // radiation, FP64 form: temperatures in sorted order
  int rad;                      // some bed radiates: k_ranges writes the sorted copies every step
  R *qc;                        // contact conduction heat of each parcel in contact (conducting beds)
};

// total layer mass of parcel i in the form's type (the same sum everywhere it is needed)
template <class P> __device__ __forceinline__ typename P::R parcel_mass(const PState<typename P::R> &A, int i) {
  typename P::R s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) s += mass_r<P>(A.m[q], i);
  return s;
}

// whether this step re-stores the state in cell order: a list-build step that completes
// restore_every builds since the last re-store (the same answer in every kernel of the step)
template <class P> __device__ __forceinline__ bool restore_now(const StepView<P> &V) {
  return *V.rebuild != 0 && V.step_ctr[4] + 1 >= V.restore_every;
}

__device__ __forceinline__ bool coupled_step(int ncouple, const long long *ctr) {
  return ncouple == 1 || (((int)(*ctr % ncouple)) + 1) % ncouple == 0;
}

// The end of a step (k_step_counter, one thread, after every other kernel of the step): the
// step counter, the list-build and re-store counters, the next step's empty contact work
// list. ctr[0] steps, [1] list builds, [2] list entries of the last build, [3] those of the
// build in progress, [4] builds since the last re-store, [5] a coupling input arrived.
struct StepEnd {
  long long *ctr;
  int *rebuild;
  int *nwork;
  int lists, restore_every;
};
__device__ __forceinline__ void step_end(const StepEnd &e) {
  long long *ctr = e.ctr;
  ctr[0] += 1;
  *e.nwork = 0;   // the next step's contact work list starts empty
  if (*e.rebuild) ctr[4] = ctr[4] + 1 >= e.restore_every ? 0 : ctr[4] + 1;   // builds since the last re-store
  if (e.lists && *e.rebuild) {   // neighbour-list builds, and the list entries of the last one
    ctr[1] += 1;
    ctr[2] = ctr[3];
    ctr[3] = 0;
  }
  *e.rebuild = 0;   // the lists built this step (if any) are current
  ctr[5] = 0;       // the gas buffers agree after this step's k_cells (a copy step, if needed)
}

// ---------------------------------------------------------------------------------------
// Velocity Verlet (kick-drift-kick). The state holds the half-step velocity: the key kernel
// drifts the positions with it, the contact and gas-particle kernels read it, and the
// gas-particle kernel applies this step's second half kick and then the next step's first.
// ---------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R half_kick(R half_dt, double dt_d, R v, R a) {
  if constexpr (sizeof(R) == 8) return __dadd_rn(v, __dmul_rn(a, 0.5 * dt_d));
  else return v + a * half_dt;
}
// the whole-step velocity from the half-step one the state holds (within an ulp of the
// velocity the half kick started from)
template <class R>
__device__ __forceinline__ R half_kick_back(R half_dt, double dt_d, R u, R a) {
  if constexpr (sizeof(R) == 8) return __dsub_rn(u, __dmul_rn(a, 0.5 * dt_d));
  else return u - a * half_dt;
}

// Gas cell of a point: floor((x - x0) * (1/dx)) clamped, in FP64.
__device__ __forceinline__ int cell_coord_d(double x, double x0, double inv, int n, bool &out) {
  const double f = floor((x - x0) * inv);
  if (!(f >= 0.0 && f < (double)n)) out = true;
  return (int)fmin(fmax(f, 0.0), (double)(n - 1));
}

static __device__ __noinline__ unsigned point_key_d(const DevBed &B, double x, double y, double z, bool &out) {
  out = false;
  const int ix = cell_coord_d(x, B.x0, B.inv_dx, B.nx, out);
  const int iy = cell_coord_d(y, B.y0, B.inv_dy, B.ny, out);
  const int iz = cell_coord_d(z, B.z0, B.inv_dz, B.nz, out);
  return (unsigned)(B.cell_off + ((long long)iz * B.ny + iy) * B.nx + ix);
}

// cell coordinates of a key within its bed (32-bit arithmetic: keys are below 2^31)
__device__ __forceinline__ void key_cell(const DevBed &B, unsigned key, int &ix, int &iy, int &iz) {
  const unsigned l = key - (unsigned)B.cell_off;
  const unsigned nx = (unsigned)B.nx, ny = (unsigned)B.ny;
  const unsigned row = l / nx;
  ix = (int)(l - row * nx);
  iz = (int)(row / ny);
  iy = (int)(row - (unsigned)iz * ny);
}

// Half kick + drift (written back to the FP64 positions), the sort key, and the FP32
// cell-local coordinates. The FP32 forms take the key from the previous cell when the
// parcel stays more than 1e-3 of an edge inside it (the local coordinates then decide
// it exactly, their error being ~1e-10 m); otherwise, and always in the FP64 form, the key
// is the FP64 definition.
// Cell of a position given as an FP32 pair p relative to the bed corner (split-Kahan form):
// the q with corner[q] <= p < corner[q+1], corners being FP32 pairs too; the differences
// hi - c_hi are exact (Sterbenz), so the test and the local coordinate agree.
__device__ __forceinline__ float pair_minus(float2 p, float2 c) { return (p.x - c.x) + (p.y - c.y); }
__device__ __forceinline__ int pair_cell(float2 p, const float2 *c, float inv_h, int n, bool &out) {
  int q = (int)floorf(p.x * inv_h);
  q = min(max(q, 0), n - 1);
  if (pair_minus(p, c[q]) < 0.f && q > 0) --q;
  else if (pair_minus(p, c[q + 1]) >= 0.f && q < n - 1) ++q;
  if (pair_minus(p, c[q]) < 0.f || pair_minus(p, c[q + 1]) >= 0.f) out = true;
  return q;
}

// FP32 position relative to the corner of cell (ix, iy, iz) and the radius
template <class P>
__device__ __forceinline__ float4 local_coords(const StepView<P> &V, const DevBed &B, int ix, int iy, int iz,
                                               double x, double y, double z, const float2 *p2, float r) {
  if constexpr (P::kahan) {
    const float2 *cp = V.cornerp + B.cornerp_off;
    const float2 *cy = cp + B.nx + 1, *cz = cy + B.ny + 1;
    return make_float4(pair_minus(p2[0], cp[ix]), pair_minus(p2[1], cy[iy]), pair_minus(p2[2], cz[iz]), r);
  } else {
    const double *cn = V.corner + B.corner_off;
    return make_float4((float)(x - cn[ix]), (float)(y - cn[B.nx + iy]), (float)(z - cn[B.nx + B.ny + iz]), r);
  }
}

// one parcel's inputs of the key kernel, loaded before any of its work, so that a thread's
// two parcels have all their loads in flight together
template <class P> struct KeyIn {
  typename P::R v[3], d;
  double x, y, z;
  float2 p2[3];
  float dsp[3];
  float4 xl;
  unsigned keyp, inv, kprev, kprev1;
  int meta;
};

template <class P>
__device__ __forceinline__ void key_load(const StepView<P> &V, int i, int drift, KeyIn<P> &in) {
  if (drift) {
    in.kprev = V.keys_prev[i];
    in.kprev1 = i > 0 ? V.keys_prev[i - 1] : ~in.kprev;
  }
  in.meta = V.A.meta[i];
  if constexpr (P::kahan) {
#pragma unroll
    for (int q = 0; q < 3; ++q) in.p2[q] = reinterpret_cast<const float2 *>(q == 0 ? V.A.x : q == 1 ? V.A.y : V.A.z)[i];
    in.x = in.y = in.z = 0.0;
  } else {
    in.x = V.A.x[i]; in.y = V.A.y[i]; in.z = V.A.z[i];
  }
  if (drift) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      in.v[q] = V.A.v[q][i];
      in.dsp[q] = V.A.dsp[q][i];
    }
    in.inv = V.inv[i];
    if constexpr (!P::exact) in.xl = V.xl[i];
  }
  in.keyp = V.keyp[i];
  in.d = V.A.d[i];
}

// Drift of velocity Verlet with the half-step velocity the state holds (the gas-particle
// kernel of the last step applied this step's first half kick after its second one, with the
// same expression), the gas cell of the new position, and the FP32 cell-local coordinates;
// in place, storage order.
// The FP32 forms take the key from the previous cell when the parcel stays more than 1e-3 of
// an edge inside it (the local coordinates then decide it exactly, their error being
// ~1e-10 m); otherwise, and always in the FP64 form, the key is recomputed from the
// position: FP64 floor((x - x0) / dx), or in the split-Kahan form the pair comparison.
template <class P>
__device__ __forceinline__ void key_work(const StepView<P> &V, int i, int drift, KeyIn<P> &in) {
  using R = typename P::R;
  if (drift && in.kprev1 != in.kprev) {   // empty the previous step's cell ranges (k_ranges writes this step's)
    V.cstart[in.kprev] = 0u;
    V.cend[in.kprev] = 0u;
  }
  const int b = in.meta >> 8;
  const DevBed &B = V.beds[b];
  const BedP<R> &bp = V.bp[b];
  double x = in.x, y = in.y, z = in.z;
  float2 p2[3] = {in.p2[0], in.p2[1], in.p2[2]};
  bool fast = false;
  unsigned key = 0;
  int ix = 0, iy = 0, iz = 0;
  if (drift) {
    R disp[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const R vh = in.v[q];
      if constexpr (sizeof(R) == 8) disp[q] = __dmul_rn(vh, B.dt);
      else disp[q] = vh * bp.dt;
    }
    if constexpr (P::kahan) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        p2[q] = pair_add_exact(p2[q], (float)disp[q]);
        reinterpret_cast<float2 *>(q == 0 ? V.A.x : q == 1 ? V.A.y : V.A.z)[i] = p2[q];
      }
    } else {
      if constexpr (sizeof(R) == 8) {
        x = __dadd_rn(x, disp[0]); y = __dadd_rn(y, disp[1]); z = __dadd_rn(z, disp[2]);
      } else {
        x = x + (double)disp[0]; y = y + (double)disp[1]; z = z + (double)disp[2];
      }
      V.A.x[i] = x; V.A.y[i] = y; V.A.z[i] = z;
    }
    // displacement since the neighbour lists were built; past half the skin they are rebuilt
    float s2 = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float dq = in.dsp[q] + (float)disp[q];
      V.A.dsp[q][i] = dq;
      s2 += dq * dq;
    }
    if (s2 > (float)bp.half_skin2) atomicOr(V.rebuild, 1);
    if constexpr (!P::exact) {
      const float4 o = in.xl;
      const float hx = (float)bp.dx, hy = (float)bp.dy, hz = (float)bp.dz;
      const float ux = o.x + (float)disp[0], uy = o.y + (float)disp[1], uz = o.z + (float)disp[2];
      fast = ux > 1e-3f * hx && ux < 0.999f * hx && uy > 1e-3f * hy && uy < 0.999f * hy &&
             uz > 1e-3f * hz && uz < 0.999f * hz;
      if (fast) {
        key = in.keyp;
        key_cell(B, key, ix, iy, iz);
      }
    }
  }
  if (!fast) {
    bool out = false;
    if constexpr (P::kahan) {
      const float2 *cp = V.cornerp + B.cornerp_off;
      const float2 *cy = cp + B.nx + 1, *cz = cy + B.ny + 1;
      ix = pair_cell(p2[0], cp, (float)bp.inv_dx, B.nx, out);
      iy = pair_cell(p2[1], cy, (float)bp.inv_dy, B.ny, out);
      iz = pair_cell(p2[2], cz, (float)bp.inv_dz, B.nz, out);
      key = (unsigned)(B.cell_off + ((long long)iz * B.ny + iy) * B.nx + ix);
    } else {
      key = point_key_d(B, x, y, z, out);
      key_cell(B, key, ix, iy, iz);
    }
    if (out) set_error(V.err, ERR_DOMAIN);
  }
  if (drift) {
    // the re-sort's input: the new key at the parcel's previous sorted position, and the
    // count of changed keys per 1024 sorted positions
    V.knew[in.inv] = key;
    if (key != in.keyp) atomicAdd(V.moved + (in.inv >> 10), 1);
  }
  V.keyp[i] = key;
  V.xl[i] = local_coords<P>(V, B, ix, iy, iz, x, y, z, p2, (float)(bp.k * in.d) * 0.5f);
}

// Two parcels per thread, 32 apart (each load instruction of a warp stays coalesced); all
// the loads of both come first.
template <class P>
__global__ void k_key(StepView<P> V, int drift) {
  pdl_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i0 = (t >> 5) * 64 + (t & 31), i1 = i0 + 32;
  if (i0 >= V.n) return;
  const bool two = i1 < V.n;
  KeyIn<P> a, b;
  key_load<P>(V, i0, drift, a);
  if (two) key_load<P>(V, i1, drift, b);
  key_work<P>(V, i0, drift, a);
  if (two) key_work<P>(V, i1, drift, b);
}

// Re-store (list-build steps, and the first binning): copy every parcel's record, local
// coordinates, key and history to its sorted position in the scratch buffers ...
template <class P>
__device__ __forceinline__ void restore_out_one(const StepView<P> &V, int i) {
  const int j = (int)__ldg(V.vals + i);
  const double x = __ldg(V.A.x + j), y = __ldg(V.A.y + j), z = __ldg(V.A.z + j);
  V.S.x[i] = x; V.S.y[i] = y; V.S.z[i] = z;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    V.S.v[q][i] = __ldg(V.A.v[q] + j); V.S.w[q][i] = __ldg(V.A.w[q] + j);
    V.S.a[q][i] = __ldg(V.A.a[q] + j); V.S.al[q][i] = __ldg(V.A.al[q] + j);
    V.S.dsp[q][i] = __ldg(V.A.dsp[q] + j);
  }
  V.S.T[i] = __ldg(V.A.T + j);
  V.S.d[i] = __ldg(V.A.d + j);
#pragma unroll
  for (int q = 0; q < 4; ++q) V.S.m[q][i] = __ldg(V.A.m[q] + j);
  V.S.meta[i] = __ldg(V.A.meta + j);
  V.S.orig[i] = __ldg(V.A.orig + j);
  V.xls[i] = __ldg(V.xl + j);
  const int c = __ldg(V.H.cnt + j);
  V.Hs.cnt[i] = (unsigned char)c;
  for (int s = 0; s < c; ++s) {
    V.Hs.id[(size_t)s * V.cap + i] = V.H.id[(size_t)s * V.cap + j];
#pragma unroll
    for (int q = 0; q < 3; ++q) V.Hs.xi[(size_t)(s * 3 + q) * V.cap + i] = V.H.xi[(size_t)(s * 3 + q) * V.cap + j];
  }
}

// Sorted-position range of every occupied cell, and the sorted position of every storage
// position (the next step's key kernel scatters its keys through it). Four consecutive
// sorted positions per thread (vector loads of keys and permutation). On a re-store step
// (or with force, at the first binning) also the first half of the re-store: every record
// copied to its sorted position in the scratch buffers (k_restore_in, after the whole grid,
// copies them back).
template <class P>
__global__ void k_ranges(StepView<P> V, int force) {
  pdl_wait();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int i0 = 4 * q;
  if (i0 >= V.n) return;
  if (force || restore_now(V)) {
    const int ce = min(i0 + 4, V.n);
    for (int i = i0; i < ce; ++i) restore_out_one<P>(V, i);
  }
  if (q == 0 && *V.rebuild) *V.novf = 0;   // a list build lists the overflowed parcels anew
  if (q < (V.n + 1023) / 1024) V.moved[q] = 0;   // the re-sort is done with the counts: zero for the next step
  // a search of every parcel without a re-store reads the local coordinates in sorted order
  const bool copy = (*V.rebuild || V.nolists) && !restore_now(V);
  const int cnt = min(4, V.n - i0);
  unsigned k[4], j[4];
  if (cnt == 4) {
    const uint4 kk = *reinterpret_cast<const uint4 *>(V.keys + i0);
    const uint4 jj = *reinterpret_cast<const uint4 *>(V.vals + i0);
    k[0] = kk.x; k[1] = kk.y; k[2] = kk.z; k[3] = kk.w;
    j[0] = jj.x; j[1] = jj.y; j[2] = jj.z; j[3] = jj.w;
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      k[u] = u < cnt ? V.keys[i0 + u] : 0u;
      j[u] = u < cnt ? V.vals[i0 + u] : 0u;
    }
  }
  const bool has_prev = i0 > 0, has_next = i0 + cnt < V.n;
  const unsigned kprev = has_prev ? V.keys[i0 - 1] : 0u, knext = has_next ? V.keys[i0 + cnt] : 0u;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (u >= cnt) break;
    const int i = i0 + u;
    const bool first = u == 0 ? (!has_prev || kprev != k[0]) : k[u - 1] != k[u];
    const bool last = u == cnt - 1 ? (!has_next || knext != k[u]) : k[u + 1] != k[u];
    if (first) V.cstart[k[u]] = (unsigned)i;
    if (last) V.cend[k[u]] = (unsigned)(i + 1);
    V.inv[j[u]] = (unsigned)i;
    if (copy) V.xls[i] = V.xl[j[u]];
    if (V.rad) {   // the radiation kernel's candidates: coordinates and temperature, sorted order
      const float4 o = V.xl[j[u]];
      const typename P::R t = V.A.T[j[u]];
      V.xr[i] = make_float4(o.x, o.y, o.z, (float)t);
      if constexpr (P::exact) V.tsrt[i] = t;
    }
  }
}

// ... and back into the state, which is then in sorted order (storage = sorted position).
template <class P>
__device__ __forceinline__ void restore_in_one(const StepView<P> &V, int i) {
  V.A.x[i] = V.S.x[i]; V.A.y[i] = V.S.y[i]; V.A.z[i] = V.S.z[i];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    V.A.v[q][i] = V.S.v[q][i]; V.A.w[q][i] = V.S.w[q][i];
    V.A.a[q][i] = V.S.a[q][i]; V.A.al[q][i] = V.S.al[q][i];
    V.A.dsp[q][i] = V.S.dsp[q][i];
  }
  V.A.T[i] = V.S.T[i];
  V.A.d[i] = V.S.d[i];
#pragma unroll
  for (int q = 0; q < 4; ++q) V.A.m[q][i] = V.S.m[q][i];
  V.A.meta[i] = V.S.meta[i];
  V.A.orig[i] = V.S.orig[i];
  V.xl[i] = V.xls[i];
  V.keyp[i] = V.keys[i];
  V.vals[i] = (unsigned)i;
  V.inv[i] = (unsigned)i;
  const int c = V.Hs.cnt[i];
  V.H.cnt[i] = (unsigned char)c;
  for (int s = 0; s < c; ++s) {
    V.H.id[(size_t)s * V.cap + i] = V.Hs.id[(size_t)s * V.cap + i];
#pragma unroll
    for (int q = 0; q < 3; ++q) V.H.xi[(size_t)(s * 3 + q) * V.cap + i] = V.Hs.xi[(size_t)(s * 3 + q) * V.cap + i];
  }
}

template <class P>
__global__ void k_restore_in(StepView<P> V, int force) {
  pdl_wait();
  if (!force && !restore_now(V)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V.n; i += gridDim.x * blockDim.x)
    restore_in_one<P>(V, i);
}

// ---------------------------------------------------------------------------------------
// Contacts: one thread per parcel over the 27 neighbouring cells. The pair test runs on
// FP32 cell-local coordinates (exact to ~1e-10 m); the FP64 form then re-tests the
// survivors on the FP64 positions with the oracle's expression, so its pair sets are
// bit-exact. Walls: FP32 pre-screen, FP64 distances for the primitives within reach.
// ---------------------------------------------------------------------------------------
// the parcel's contact history before the step: its count and the first partners, loaded
// once per parcel (the rest, if any, are read from memory)
constexpr int HPRE = 4;
struct HistIn {
  int cin;
  int id[HPRE];
};

template <class P>
__device__ __forceinline__ void add_contact(const StepView<P> &V, int i, const HistIn &hin, int pid,
                                            const BedP<typename P::R> &bp,
                                            typename P::R mstar, typename P::R ri, const typename P::R nrm[3],
                                            typename P::R delta, const typename P::R vrel[3],
                                            const typename P::R wi[3], typename P::R Fi[3], typename P::R Ti[3],
                                            int &cout) {
  using R = typename P::R;
  R xo[3] = {0, 0, 0};
  int found = -1;
#pragma unroll
  for (int sl = 0; sl < HPRE; ++sl)
    if (found < 0 && sl < hin.cin && hin.id[sl] == pid) found = sl;
  for (int sl = HPRE; found < 0 && sl < hin.cin; ++sl)
    if (V.H.id[(size_t)sl * V.cap + i] == pid) found = sl;
  if (found >= 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) xo[q] = V.H.xi[(size_t)(found * 3 + q) * V.cap + i];
  }
  R Fc[3], Tc[3], xn[3];
  contact_force<R>(bp, mstar, ri, nrm, delta, vrel, xo, wi, Fc, Tc, xn);
#pragma unroll
  for (int q = 0; q < 3; ++q) { Fi[q] += Fc[q]; Ti[q] += Tc[q]; }
  if (cout < KMAX) {
    V.Hn.id[(size_t)cout * V.cap + i] = pid;
#pragma unroll
    for (int q = 0; q < 3; ++q) V.Hn.xi[(size_t)(cout * 3 + q) * V.cap + i] = xn[q];
    ++cout;
  } else {
    set_error(V.err, ERR_CAPACITY);
  }
}

// ---------------------------------------------------------------------------------------
// Contacts, one thread per parcel.
// k_pair_search (list builds, overflowed lists, no lists): for each of the 9 neighbour rows
// (dy, dz) the cells X-1..X+1 hold one contiguous run of sorted positions; rows and end cells
// farther than r_i + r_max (+ skin) from the parcel are skipped. Every candidate is tested on
// the FP32 cell-local coordinates (the exact form with a small margin); the hits go, in
// visiting order (dz, dy, dx, sorted position), to a per-parcel hit list, and on build steps
// the partners within r_i + r_j + skin to the parcel's neighbour list. Few registers, so many
// warps hide the load latency of the pair loop.
// k_contact_screen / k_contact_forces: the list test between builds, the contact law for the
// pairs (the FP64 form first re-tests each pair on the FP64 positions with the oracle's
// expression, so its pair sets are bit-exact), and the walls.
// ---------------------------------------------------------------------------------------
// cell offsets (dx, dy, dz) of the cell with key k2 relative to the cell with key k1
__device__ __forceinline__ void key_offset(const DevBed &B, unsigned k1, unsigned k2, int &dx, int &dy, int &dz) {
  if (B.fast_offsets) {
    // k2 - k1 = dz nx ny + dy nx + dx with |dx|, |dy|, |dz| <= 2 and nx, ny >= 5, so rounding
    // recovers each term with a margin of 0.05 in units of the divisor
    const int dk = (int)(k2 - k1);
    const int nxy = B.nx * B.ny;
    dz = __float2int_rn((float)dk * B.inv_nxy_f);
    const int r = dk - dz * nxy;
    dy = __float2int_rn((float)r * B.inv_nx_f);
    dx = r - dy * B.nx;
  } else {
    int x1, y1, z1, x2, y2, z2;
    key_cell(B, k1, x1, y1, z1);
    key_cell(B, k2, x2, y2, z2);
    dx = x2 - x1; dy = y2 - y1; dz = z2 - z1;
  }
}

template <class P>
__device__ __forceinline__ void pair_search(const StepView<P> &V, int i, bool rebuild, bool restored, bool copy) {
  const int b = V.A.meta[i] >> 8;
  const DevBed &B = V.beds[b];
  const BedP<typename P::R> &bp = V.bp[b];
  const size_t cap = (size_t)V.cap;
  const bool build = rebuild && !V.nolists;
  int nh = 0, nn = 0;
  if (!(bp.flags & DEM_NO_CONTACTS)) {
    const float4 me = V.xl[i];
    const unsigned key = V.keyp[i];
    const int si = (int)V.inv[i];   // the parcel's own sorted position
    const float hx = (float)bp.dx, hy = (float)bp.dy, hz = (float)bp.dz;
    const float pm = P::exact ? (float)bp.pf_margin : 0.f;
    // the candidates' records in sorted order: the state itself just after a re-store, else
    // the copy k_ranges gathered on a search-all step; otherwise through the permutation
    const float4 *xs = restored ? V.xl : V.xls;
    {
      // cell-list path (list rebuild, or a parcel whose list overflowed)
      const float skin = build ? (float)bp.skin : 0.f;
      int X, Y, Z;
      key_cell(B, key, X, Y, Z);
      // no partner centre lies farther than r_i + r_max (+ skin); the margin is far above
      // the ~1e-10 m resolution of the local coordinates
      const float reach = (me.w + (float)bp.reach_max + skin) * 1.0001f + pm + 1e-9f;
      const int xlo = (X > 0 && me.x < reach) ? -1 : 0, xhi = (X < B.nx - 1 && hx - me.x < reach) ? 1 : 0;
      const int ylo = (Y > 0 && me.y < reach) ? -1 : 0, yhi = (Y < B.ny - 1 && hy - me.y < reach) ? 1 : 0;
      const int zlo = (Z > 0 && me.z < reach) ? -1 : 0, zhi = (Z < B.nz - 1 && hz - me.z < reach) ? 1 : 0;
      for (int dz = zlo; dz <= zhi; ++dz) {
        const float gz = dz < 0 ? me.z : (dz > 0 ? hz - me.z : 0.0f);   // distance to the row
        for (int dy = ylo; dy <= yhi; ++dy) {
          const float gy = dy < 0 ? me.y : (dy > 0 ? hy - me.y : 0.0f);
          if (gy * gy + gz * gz >= reach * reach) continue;
          const unsigned krow = key + (unsigned)(dy * B.nx) + (unsigned)(dz * B.nx * B.ny);
          const float oy = dy * hy - me.y, oz = dz * hz - me.z;
          for (int dx = xlo; dx <= xhi; ++dx) {
            const unsigned jb = __ldg(V.cstart + krow + dx), je = __ldg(V.cend + krow + dx);
            const float ox = dx * hx - me.x;
            const unsigned char code = (unsigned char)((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1));
// test of the candidate at sorted position s, storage position js
#define DEM_PAIR_TEST(o, s, js)                                                       \
  do {                                                                                \
    const float ex = (o).x + ox, ey = (o).y + oy, ez = (o).z + oz; /* x_j - x_i */   \
    const float d2 = ex * ex + ey * ey + ez * ez;                                     \
    const float rs = me.w + (o).w;                                                    \
    const float lim = rs + pm, liml = rs + skin;                                      \
    const bool inl = build && d2 < liml * liml, inh = d2 < lim * lim;                 \
    if ((inl || inh) && (s) != si) {                                                  \
      const int j = (js);                                                             \
      if (inl) {                                                                      \
        if (nn < KNL) V.nl[nn * cap + i] = j;                                         \
        ++nn;                                                                         \
      }                                                                               \
      if (inh) {                                                                      \
        if (nh < KLIST) {                                                             \
          V.plist[nh * cap + i] = j;                                                  \
          V.pcode[nh * cap + i] = code;                                               \
        }                                                                             \
        ++nh;                                                                         \
      }                                                                               \
    }                                                                                 \
  } while (0)
            int jj = (int)jb;
            if (restored) {
              for (; jj + 4 <= (int)je; jj += 4) {
                const float4 o0 = __ldg(xs + jj), o1 = __ldg(xs + jj + 1);
                const float4 o2 = __ldg(xs + jj + 2), o3 = __ldg(xs + jj + 3);
                DEM_PAIR_TEST(o0, jj, jj);
                DEM_PAIR_TEST(o1, jj + 1, jj + 1);
                DEM_PAIR_TEST(o2, jj + 2, jj + 2);
                DEM_PAIR_TEST(o3, jj + 3, jj + 3);
              }
              for (; jj < (int)je; ++jj) {
                const float4 o0 = __ldg(xs + jj);
                DEM_PAIR_TEST(o0, jj, jj);
              }
            } else if (copy) {
              // the storage positions are loaded with the records, not after a hit
              for (; jj + 4 <= (int)je; jj += 4) {
                const float4 o0 = __ldg(xs + jj), o1 = __ldg(xs + jj + 1);
                const float4 o2 = __ldg(xs + jj + 2), o3 = __ldg(xs + jj + 3);
                const int j0 = (int)__ldg(V.vals + jj), j1 = (int)__ldg(V.vals + jj + 1);
                const int j2 = (int)__ldg(V.vals + jj + 2), j3 = (int)__ldg(V.vals + jj + 3);
                DEM_PAIR_TEST(o0, jj, j0);
                DEM_PAIR_TEST(o1, jj + 1, j1);
                DEM_PAIR_TEST(o2, jj + 2, j2);
                DEM_PAIR_TEST(o3, jj + 3, j3);
              }
              for (; jj < (int)je; ++jj) {
                const float4 o0 = __ldg(xs + jj);
                const int j0 = (int)__ldg(V.vals + jj);
                DEM_PAIR_TEST(o0, jj, j0);
              }
            } else {
              // overflowed lists between builds: through the permutation, four at a time
              for (; jj + 4 <= (int)je; jj += 4) {
                const int j0 = (int)__ldg(V.vals + jj), j1 = (int)__ldg(V.vals + jj + 1);
                const int j2 = (int)__ldg(V.vals + jj + 2), j3 = (int)__ldg(V.vals + jj + 3);
                const float4 o0 = __ldg(V.xl + j0), o1 = __ldg(V.xl + j1);
                const float4 o2 = __ldg(V.xl + j2), o3 = __ldg(V.xl + j3);
                DEM_PAIR_TEST(o0, jj, j0);
                DEM_PAIR_TEST(o1, jj + 1, j1);
                DEM_PAIR_TEST(o2, jj + 2, j2);
                DEM_PAIR_TEST(o3, jj + 3, j3);
              }
              for (; jj < (int)je; ++jj) {
                const int j0 = (int)__ldg(V.vals + jj);
                const float4 o0 = __ldg(V.xl + j0);
                DEM_PAIR_TEST(o0, jj, j0);
              }
            }
#undef DEM_PAIR_TEST
          }
        }
      }
    }
  }
  if (rebuild) {
#pragma unroll
    for (int q = 0; q < 3; ++q) V.A.dsp[q][i] = 0.f;   // displacements count from this build
  }
  if (build) {
    V.nlc[i] = (unsigned char)(nn > KNL ? NL_OVERFLOW : nn);
    if (nn > KNL) V.ovf[atomicAdd(V.novf, 1)] = i;   // searched again every step until the next build
    const unsigned am = __activemask();   // one atomic per group of lanes running together
    const unsigned tot = __reduce_add_sync(am, (unsigned)min(nn, KNL));
    if ((threadIdx.x & 31) == __ffs(am) - 1) atomicAdd(V.list_acc, (unsigned long long)tot);
  }
  if (nh > KLIST) { set_error(V.err, ERR_CAPACITY); nh = KLIST; }
  V.pcnt[i] = (unsigned char)nh;
}

// The cell-list search: every parcel on list-build steps (and every step with the lists
// off), otherwise only the parcels whose list overflowed at the last build (their storage
// positions do not change between builds). Grid-stride over at most one wave of blocks, so
// that the steps between builds cost one flag read per block.
template <class P>
__global__ void k_pair_search(StepView<P> V) {
  pdl_wait();
  const bool rebuild = *V.rebuild != 0;
  const bool restored = restore_now(V);
  const bool all = rebuild || V.nolists;
  const int cnt = all ? V.n : *V.novf;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x)
    pair_search<P>(V, all ? t : V.ovf[t], rebuild, restored, all && !restored);
}

// Contact of parcel i with partner j (storage positions; code = cell offset of j's cell):
// the FP64 form re-tests the pair on the FP64 positions with the oracle's expression.
template <class P>
__device__ __forceinline__ void pair_contact(const StepView<P> &V, int i, int j, int code, const DevBed &B,
                                             const BedP<typename P::R> &bp, const float4 &me, float hx, float hy,
                                             float hz, const double *xi_d, double ri_d, typename P::R ri,
                                             typename P::R mi, const typename P::R vi[3], const typename P::R wi[3],
                                             const HistIn &hin, typename P::R Fi[3], typename P::R Ti[3], int &cout,
                                             const typename P::R cth[3], typename P::R &Qc) {
  using R = typename P::R;
  R nrm[3], delta, dist;
  double rj_d = 0;
  if constexpr (P::exact) {
    const double dxd = V.A.x[j] - xi_d[0], dyd = V.A.y[j] - xi_d[1], dzd = V.A.z[j] - xi_d[2];
    rj_d = __dmul_rn(0.5, __dmul_rn(B.k, (double)V.A.d[j]));
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dxd, dxd), __dmul_rn(dyd, dyd)), __dmul_rn(dzd, dzd));
    const double rs = __dadd_rn(ri_d, rj_d);
    if (!(d2 < __dmul_rn(rs, rs))) return;
    const double dd = sqrt(d2);
    nrm[0] = (R)(dxd / dd); nrm[1] = (R)(dyd / dd); nrm[2] = (R)(dzd / dd);
    delta = (R)(rs - dd);
    dist = (R)dd;
  } else {
    const int cdx = code % 3 - 1, cdy = (code / 3) % 3 - 1, cdz = code / 9 - 1;
    const float4 o = __ldg(V.xl + j);
    const float ex = o.x + (cdx * hx - me.x), ey = o.y + (cdy * hy - me.y), ez = o.z + (cdz * hz - me.z);
    const float d2f = ex * ex + ey * ey + ez * ez;
    const float rsf = me.w + o.w;
    const float df = sqrtf(d2f);
    const float inv = 1.0f / df;
    nrm[0] = (R)(ex * inv); nrm[1] = (R)(ey * inv); nrm[2] = (R)(ez * inv);
    delta = (R)((rsf * rsf - d2f) / (rsf + df));
    dist = (R)df;
  }
  const R rj = P::exact ? (R)rj_d : (R)__ldg(&V.xl[j].w);
  if (bp.flags & DEM_CONDUCTION) {
    // cth: own temperature, own ore, own cell's gas conductivity
    const int orej = V.A.meta[j] & 255;
    const R lamg_j = V.gp[(size_t)V.keyp[j] * GP_STRIDE + GP_LAM];
    Qc += conduction_pair<R>(bp, ri, rj, dist, delta, cth[0], V.A.T[j], bp.lam_e[(int)cth[1]][orej],
                             (R)0.5 * (cth[2] + lamg_j));
  }
  const R mj = parcel_mass<P>(V.A, j);
  const R mstar = mi * mj / (mi + mj);
  const R ws[3] = {ri * wi[0] + rj * V.A.w[0][j], ri * wi[1] + rj * V.A.w[1][j], ri * wi[2] + rj * V.A.w[2][j]};
  R vrel[3];
  vrel[0] = (vi[0] - V.A.v[0][j]) + (ws[1] * nrm[2] - ws[2] * nrm[1]);
  vrel[1] = (vi[1] - V.A.v[1][j]) + (ws[2] * nrm[0] - ws[0] * nrm[2]);
  vrel[2] = (vi[2] - V.A.v[2][j]) + (ws[0] * nrm[1] - ws[1] * nrm[0]);
  add_contact<P>(V, i, hin, V.A.orig[j], bp, mstar, ri, nrm, delta, vrel, wi, Fi, Ti, cout);
}

// Contacts in two passes. The screen pass runs over every parcel: the neighbour-list test
// (between list builds; hits kept as a mask over the list entries), the search hits of
// build steps (and of overflowed lists, or with the lists off), and an FP32 wall
// pre-screen in the cells that may hold a parcel within reach of a wall. Parcels with none
// of these get an empty contact history at once; the others are appended to a work list,
// so that the force pass runs on dense warps of parcels that have something to evaluate (a
// few per cent of them) instead of leaving most lanes of most warps idle. Results do not
// depend on the order of the work list: each entry writes only its own parcel's forces and
// history.
template <class P>
__device__ __forceinline__ bool wall_near(const StepView<P> &V, const DevBed &B, const BedP<typename P::R> &bp,
                                          unsigned key, const float4 &me) {
  if (!V.wnear[key]) return false;
  int X, Y, Z;
  key_cell(B, key, X, Y, Z);
  const float hx = (float)bp.dx, hy = (float)bp.dy, hz = (float)bp.dz;
  const float xa = (float)bp.x0 + X * hx + me.x, ya = (float)bp.y0 + Y * hy + me.y, za = (float)bp.z0 + Z * hz + me.z;
  float distf[4], nwf[4][3];
  wall_primitives<float>(bp, xa, ya, za, distf, nwf);
  bool near = false;
#pragma unroll
  for (int p = 0; p < 4; ++p) near |= distf[p] < me.w + 1e-6f;
  return near;
}

template <class P>
__device__ __forceinline__ bool contact_screen(const StepView<P> &V, int i, unsigned &hits) {
  // the parcel's own loads first, all in flight together (3 % faster than issuing them after
  // the bed's switches are read)
  const int meta = V.A.meta[i];
  const float4 me = V.xl[i];
  const unsigned key = V.keyp[i];
  const int listed = V.nlc[i];
  const DevBed &B = V.beds[meta >> 8];
  const BedP<typename P::R> &bp = V.bp[meta >> 8];
  hits = 0u;
  if (bp.flags & DEM_NO_CONTACTS) return false;
  const bool near = wall_near<P>(V, B, bp, key, me);
  const bool searched = *V.rebuild || V.nolists || listed == NL_OVERFLOW;
  if (searched) return near || V.pcnt[i] != 0;
  const float hx = (float)bp.dx, hy = (float)bp.dy, hz = (float)bp.dz;
  const size_t cap = (size_t)V.cap;
  const float pm = P::exact ? (float)bp.pf_margin : 0.f;
  for (int k0 = 0; k0 < listed; k0 += 4) {
    int j[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) j[u] = k0 + u < listed ? V.nl[(k0 + u) * cap + i] : -1;
    unsigned kj[4];
    float4 o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      kj[u] = j[u] >= 0 ? V.keyp[j[u]] : key;
      o[u] = j[u] >= 0 ? __ldg(V.xl + j[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (j[u] < 0) continue;
      int dx, dy, dz;
      key_offset(B, key, kj[u], dx, dy, dz);
      if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) continue;   // cannot touch
      const float ex = o[u].x + (dx * hx - me.x), ey = o[u].y + (dy * hy - me.y), ez = o[u].z + (dz * hz - me.z);
      const float d2 = ex * ex + ey * ey + ez * ez;
      const float lim = me.w + o[u].w + pm;
      if (d2 < lim * lim) hits |= 1u << (k0 + u);
    }
  }
  return near || hits != 0u;
}

// All contact forces on a parcel of the work list: its partners (the list hits in list
// order, or the search hits), then the walls (FP64 distances for the primitives within
// reach). Writes the parcel's new contact history; returns its number of contacts.
template <class P>
__device__ __forceinline__ int contact_forces(const StepView<P> &V, int i, unsigned hits, typename P::R Fi[3],
                                              typename P::R Ti[3], typename P::R &Qc) {
  using R = typename P::R;
  const int meta = V.A.meta[i];
  const DevBed &B = V.beds[meta >> 8];
  const BedP<R> &bp = V.bp[meta >> 8];
#pragma unroll
  for (int q = 0; q < 3; ++q) { Fi[q] = 0; Ti[q] = 0; }
  Qc = 0;
  // contact conduction (eqs (3-14)..(3-15-2)): own temperature, ore and cell's gas conductivity
  R cth[3] = {0, 0, 0};
  if (bp.flags & DEM_CONDUCTION) {
    cth[0] = V.A.T[i];
    cth[1] = (R)(meta & 255);
    cth[2] = V.gp[(size_t)V.keyp[i] * GP_STRIDE + GP_LAM];
  }
  int cout = 0;
  HistIn hin;
  hin.cin = V.H.cnt[i];
#pragma unroll
  for (int sl = 0; sl < HPRE; ++sl) hin.id[sl] = sl < hin.cin ? V.H.id[(size_t)sl * V.cap + i] : 0;
  const float4 me = V.xl[i];
  const unsigned key = V.keyp[i];
  const float hx = (float)bp.dx, hy = (float)bp.dy, hz = (float)bp.dz;
  const size_t cap = (size_t)V.cap;
  const int listed = V.nlc[i];
  const bool searched = *V.rebuild || V.nolists || listed == NL_OVERFLOW;
  const int nsearch = searched ? (int)V.pcnt[i] : 0;
  const R di = V.A.d[i];
  const R mi = parcel_mass<P>(V.A, i);
  const R vi[3] = {V.A.v[0][i], V.A.v[1][i], V.A.v[2][i]};
  const R wi[3] = {V.A.w[0][i], V.A.w[1][i], V.A.w[2][i]};
  double xi_d[3] = {0, 0, 0}, ri_d = 0;
  if constexpr (P::exact) {
    xi_d[0] = V.A.x[i]; xi_d[1] = V.A.y[i]; xi_d[2] = V.A.z[i];
    ri_d = __dmul_rn(0.5, __dmul_rn(B.k, (double)di));
  }
  const R ri = P::exact ? (R)ri_d : (R)me.w;
  for (int h = 0; h < nsearch; ++h)
    pair_contact<P>(V, i, V.plist[h * cap + i], V.pcode[h * cap + i], B, bp, me, hx, hy, hz, xi_d, ri_d, ri, mi,
                    vi, wi, hin, Fi, Ti, cout, cth, Qc);
  while (hits) {   // list order
    const int k = __ffs(hits) - 1;
    hits &= hits - 1u;
    const int j = V.nl[k * cap + i];
    int dx, dy, dz;
    key_offset(B, key, V.keyp[j], dx, dy, dz);
    pair_contact<P>(V, i, j, (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1), B, bp, me, hx, hy, hz, xi_d, ri_d, ri, mi,
                    vi, wi, hin, Fi, Ti, cout, cth, Qc);
  }
  // walls: the FP32 pre-screen again, FP64 distances for the primitives within reach
  if (!(bp.flags & DEM_NO_CONTACTS) && wall_near<P>(V, B, bp, key, me)) {
    const double xd = pos_abs<P>(V.A.x, i, B.x0), yd = pos_abs<P>(V.A.y, i, B.y0), zd = pos_abs<P>(V.A.z, i, B.z0);
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
      add_contact<P>(V, i, hin, -1 - p, bp, mi, ri, nrm, delta, vrel, wi, Fi, Ti, cout);
      if (bp.flags & DEM_CONDUCTION)
        Qc += conduction_wall<R>(bp, (R)rid, (R)dist[p], delta, cth[0], bp.lam_ew[(int)cth[1]], cth[2]);
    }
  }
  V.Hn.cnt[i] = (unsigned char)cout;
  if (V.diag) V.diag[(size_t)DG_NCONTACT * V.cap + i] = (double)cout;
  return cout;
}

// Screen pass: one thread per parcel; a warp appends its parcels with work in one atomic.
// Held to 48 registers in the FP32 forms (five 256-thread blocks per SM): more warps to
// hide the latency of the list loads.
template <class P>
__global__ void __launch_bounds__(256, P::exact ? 1 : 5) k_contact_screen(StepView<P> V) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned hits = 0u;
  bool work = false;
  if (i < V.n) {
    work = contact_screen<P>(V, i, hits);
    if (!work) {
      V.Hn.cnt[i] = 0;
      if (V.diag) V.diag[(size_t)DG_NCONTACT * V.cap + i] = 0.0;
    }
  }
  const unsigned bal = __ballot_sync(0xffffffffu, work);
  if (bal == 0u) return;
  const int lane = threadIdx.x & 31, lead = __ffs(bal) - 1;
  int base = 0;
  if (lane == lead) base = atomicAdd(V.nwork, __popc(bal));
  base = __shfl_sync(0xffffffffu, base, lead);
  if (work) V.work[base + __popc(bal & ((1u << lane) - 1u))] = make_uint2((unsigned)i, hits);
}

// Force pass over the work list (grid-stride over at most one wave of blocks). Force and
// torque are written only for parcels in contact; k_gas_particle reads them only there.
template <class P>
__global__ void k_contact_forces(StepView<P> V) {
  pdl_wait();
  using R = typename P::R;
  const int cnt = *V.nwork;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
    const uint2 w = V.work[t];
    const int i = (int)w.x;
    R F[3], Tq[3], Qc;
    if (contact_forces<P>(V, i, w.y, F, Tq, Qc) == 0) continue;
#pragma unroll
    for (int q = 0; q < 3; ++q) { V.F[q][i] = F[q]; V.Tq[q][i] = Tq[q]; }
    if (V.bp[V.A.meta[i] >> 8].flags & DEM_CONDUCTION) V.qc[i] = Qc;
  }
}

// ---------------------------------------------------------------------------------------
// Particle radiation, eqs (3-16), (3-17), (3-51), in beds with DEM_RADIATION: one thread
// per sorted position, so the threads of a warp work on a few neighbouring cells and read
// the same candidates. T_se averages the temperatures of the parcels whose centres lie
// within R = 1.5 k d_p of the parcel's centre, the parcel itself included, weighted with the
// gas cell's eps_g and T_g. No parcel is wider than a cell edge, so R < 2 edges and the
// sphere lies in the 5 x 5 x 5 cells around the parcel's own; only the cells within R are
// visited. Candidates come in sorted order from the contiguous copy k_ranges writes (local
// coordinates with the temperature as w, one 16-byte load; the FP64 form reads its FP64
// temperatures from a second copy), with no indirection. They are tested on the FP32
// cell-local coordinates;
// the FP64 form re-tests every candidate within R plus a margin on the FP64 positions with
// the oracle's expression, so its neighbourhoods are exact. The temperatures are the ones
// before this step's update (k_gas_particle runs after this kernel). Writes Q_rad and, with
// diagnostics, T_se, at the parcel's storage position. T_se^4 - T_p^4 is evaluated as
// (T_se - T_p)(T_se + T_p)(T_se^2 + T_p^2), which keeps the FP32 forms accurate when T_se is
// close to T_p.
// ---------------------------------------------------------------------------------------
template <class P>
__global__ void __launch_bounds__(128, 8) k_radiation(StepView<P> V) {
  pdl_wait();
  using R = typename P::R;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;   // sorted position
  if (s >= V.n) return;
  const unsigned key = V.keys[s];
  const int b = V.cell_bed[key];
  const BedP<R> &bp = V.bp[b];
  if (!(bp.flags & DEM_RADIATION)) return;
  const bool restored = restore_now(V);   // storage order is sorted order after a re-store
  const float4 *xs = V.xr;
  const int i = restored ? s : (int)__ldg(V.vals + s);   // storage position
  const DevBed &B = V.beds[b];
  const float4 me = xs[s];
  R Tp;
  if constexpr (P::exact) Tp = V.tsrt[s]; else Tp = me.w;
  const float hx = (float)bp.dx, hy = (float)bp.dy, hz = (float)bp.dz;
  const R d = V.A.d[i];
  double Rd = 0.0, xi_d[3] = {0.0, 0.0, 0.0};
  if constexpr (P::exact) {
    Rd = __dmul_rn(1.5, __dmul_rn(B.k, (double)d));
    xi_d[0] = V.A.x[i]; xi_d[1] = V.A.y[i]; xi_d[2] = V.A.z[i];
  }
  const float rf = 1.5f * ((float)bp.k * (float)d);
  const float hi = P::exact ? rf + (float)bp.pf_margin : rf;   // FP32 screen (with margin in FP64)
  const float hi2 = hi * hi;
  const float reach = hi * 1.0001f + 1e-9f;                    // cell pruning, with a margin
  int X, Y, Z;
  key_cell(B, key, X, Y, Z);
  R sumT = 0;
  int cnt = 0;
  float ox = 0.f, oy = 0.f, oz = 0.f;   // offset of the candidate's cell corner from the parcel
  // one candidate at sorted position q
  auto test = [&](const float4 &o, unsigned q) {
    const float ex = o.x + ox, ey = o.y + oy, ez = o.z + oz;
    bool in = ex * ex + ey * ey + ez * ez < hi2;
    if constexpr (P::exact) {
      if (in) {
        const int j = restored ? (int)q : (int)__ldg(V.vals + q);
        const double dxd = V.A.x[j] - xi_d[0], dyd = V.A.y[j] - xi_d[1], dzd = V.A.z[j] - xi_d[2];
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dxd, dxd), __dmul_rn(dyd, dyd)), __dmul_rn(dzd, dzd));
        in = d2 < __dmul_rn(Rd, Rd);
      }
    }
    if (in) {
      if constexpr (P::exact) sumT += __ldg(V.tsrt + q); else sumT += o.w;
      ++cnt;
    }
  };
  // the cell offsets along one axis that the sphere can reach (within the grid)
  auto lo_of = [reach](float m, float h, int c) {
    return (c > 0 && m < reach) ? ((c > 1 && m + h < reach) ? -2 : -1) : 0;
  };
  auto hi_of = [reach](float m, float h, int c, int nc) {
    return (c < nc - 1 && h - m < reach) ? ((c < nc - 2 && 2.f * h - m < reach) ? 2 : 1) : 0;
  };
  const int xlo = lo_of(me.x, hx, X), xhi = hi_of(me.x, hx, X, B.nx);
  const int ylo = lo_of(me.y, hy, Y), yhi = hi_of(me.y, hy, Y, B.ny);
  const int zlo = lo_of(me.z, hz, Z), zhi = hi_of(me.z, hz, Z, B.nz);
  for (int dz = zlo; dz <= zhi; ++dz) {
    const float gz = fmaxf(0.f, dz < 0 ? me.z - (dz + 1) * hz : dz * hz - me.z);   // gap to the layer
    oz = dz * hz - me.z;
    for (int dy = ylo; dy <= yhi; ++dy) {
      const float gy = fmaxf(0.f, dy < 0 ? me.y - (dy + 1) * hy : dy * hy - me.y);
      if (gy * gy + gz * gz >= reach * reach) continue;
      oy = dy * hy - me.y;
      const unsigned krow = key + (unsigned)(dy * B.nx) + (unsigned)(dz * B.nx * B.ny);
      for (int dx = xlo; dx <= xhi; ++dx) {
        const float gx = fmaxf(0.f, dx < 0 ? me.x - (dx + 1) * hx : dx * hx - me.x);
        if (gx * gx + gy * gy + gz * gz >= reach * reach) continue;
        ox = dx * hx - me.x;
        const unsigned jb = __ldg(V.cstart + krow + dx), je = __ldg(V.cend + krow + dx);
        unsigned q = jb;
        for (; q + 4 <= je; q += 4) {   // four candidates' loads in flight before their tests
          const float4 o0 = __ldg(xs + q), o1 = __ldg(xs + q + 1), o2 = __ldg(xs + q + 2), o3 = __ldg(xs + q + 3);
          test(o0, q); test(o1, q + 1); test(o2, q + 2); test(o3, q + 3);
        }
        for (; q < je; ++q) test(__ldg(xs + q), q);
      }
    }
  }
  const R *gv = V.gp + (size_t)key * GP_STRIDE;
  const R eps = gv[GP_EPS], Tg = gv[GP_TG];
  // the parcel is in its own sphere, so cnt >= 1
  const R Tse = eps * Tg + ((R)1 - eps) * (sumT / (R)max(cnt, 1));
  const R Q = bp.rad_c * d * d * ((Tse - Tp) * (Tse + Tp) * (Tse * Tse + Tp * Tp));
  V.qrad[i] = Q;
  if (V.diag) V.diag[(size_t)DG_TSE * V.cap + i] = (double)Tse;
}

// The diagnostics rows of parcel i (dem_set_diagnostics), as a call of its own: inlined, its
// FP64 conversions were scheduled ahead of the branch and ran for every parcel without
// diagnostics too, on GB300's narrow FP64 pipe.
template <class R>
__device__ __noinline__ void gp_write_diag(double *dg, size_t cp, int i, const R F[3], const R Tq[3], const R Fd[3],
                                           const KinOut<R> &kn, R Kp, R Qconv, R Nu, R Re, long long cell, R Qrad,
                                           R Qcond, bool no_tse) {
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
  dg[DG_CELL * cp + i] = (double)cell;
  dg[DG_QRAD * cp + i] = (double)Qrad;
  dg[DG_QCOND * cp + i] = (double)Qcond;
  if (no_tse) dg[DG_TSE * cp + i] = 0.0;
}

// ---------------------------------------------------------------------------------------
// Per parcel (storage order): gas-particle terms, kinetics, second half kick, temperature
// and mass update; writes the parcel's contributions to its cell sums.
// ---------------------------------------------------------------------------------------
// The FP32 forms are held to 64 registers (4 blocks of 256 threads per SM): a few spills
// to L1 cost less than the latency the extra occupancy hides (ncu: 33 % -> 50 % warps).
// RAD: some bed has radiation (the variant that adds k_radiation's Q_rad to the heat balance).
template <class P, bool RAD>
// full: this is the last step of a stepping call (or the gas is solved): the accelerations,
// which only the state output and the adjoint read (to report whole-step velocities), and
// the source rows only dem_get_sources and the gas solver read (K, K v, Q_r, E Q, E S) are
// stored; the prescribed gas update reads the other six every step
__global__ void __launch_bounds__(256, P::exact ? 1 : 4) k_gas_particle(StepView<P> V, int full) {
  pdl_wait();
  using R = typename P::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  // every load of the parcel's own record first, so that they are all in flight together
  // (the compiler, held to 64 registers, would otherwise issue some only where they are used)
  const int meta = V.A.meta[i];
  const unsigned c = V.keyp[i];
  const R d = V.A.d[i];
  const R vh[3] = {V.A.v[0][i], V.A.v[1][i], V.A.v[2][i]};
  const R Tp = V.A.T[i];
  R m[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) m[q] = mass_r<P>(V.A.m[q], i);
  const R wv[3] = {V.A.w[0][i], V.A.w[1][i], V.A.w[2][i]};
  R F[3] = {0, 0, 0}, Tq[3] = {0, 0, 0};
  const bool touching = V.Hn.cnt[i] != 0;
  if (touching) {   // the contact kernel wrote them only for parcels in contact
#pragma unroll
    for (int q = 0; q < 3; ++q) { F[q] = V.F[q][i]; Tq[q] = V.Tq[q][i]; }
  }
  const int ore = meta & 255;
  const BedP<R> &bp = V.bp[meta >> 8];
  const unsigned fl = bp.flags;
  const R Qcond = (touching && (fl & DEM_CONDUCTION)) ? V.qc[i] : (R)0;   // contact conduction, this step
  const size_t nc = (size_t)V.ncells;
  Gas<R> g;
  R gv[GP_STRIDE];   // the cell's property record, in vector loads
  if constexpr (sizeof(R) == 4) {
    const float4 *q = reinterpret_cast<const float4 *>(V.gp + (size_t)c * GP_STRIDE);
#pragma unroll
    for (int k = 0; k < GP_STRIDE / 4; ++k) {
      const float4 t = __ldg(q + k);
      gv[4 * k] = t.x; gv[4 * k + 1] = t.y; gv[4 * k + 2] = t.z; gv[4 * k + 3] = t.w;
    }
  } else {
    const double2 *q = reinterpret_cast<const double2 *>(V.gp + (size_t)c * GP_STRIDE);
#pragma unroll
    for (int k = 0; k < GP_N / 2; ++k) {
      const double2 t = __ldg(q + k);
      gv[2 * k] = t.x; gv[2 * k + 1] = t.y;
    }
  }
  g.rho = gv[GP_RHO]; g.mu = gv[GP_MU]; g.lam = gv[GP_LAM]; g.cp = gv[GP_CP]; g.x = gv[GP_X];
  g.Dm = gv[GP_DM]; g.sc13 = gv[GP_SC13]; g.pr13 = gv[GP_PR13]; g.epow = gv[GP_EPOW];
  g.D = ore ? gv[GP_D1] : gv[GP_D0]; g.uz = gv[GP_UZ]; g.eps = gv[GP_EPS]; g.T = gv[GP_TG];
  g.ux = gv[GP_UX]; g.uy = gv[GP_UY];
  const R dc = bp.k * d;
  const R Vp = (R)(kPI / 6.0) * dc * dc * dc;
  const R r = (R)0.5 * dc;
  const R sv[3] = {g.ux - vh[0], g.uy - vh[1], g.uz - vh[2]};
  const R slip = sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
  const R Re = fdiv<R>(g.rho * g.eps * d * slip, g.mu);
  const R re02 = pos_pow(Re, (R)0.2);
  const R re07 = re02 * sqrt(Re);
  const R bo = beta_over_epsp<R>(bp, ore, d, g, slip, Re);
  const R Kp = (fl & DEM_NO_DRAG) ? (R)0 : bo * Vp;
  const R Fd[3] = {Kp * sv[0], Kp * sv[1], Kp * sv[2]};
  const R Nu = gunn(g.eps, re02, re07, g.pr13);
  const R hA = (fl & DEM_NO_HEAT) ? (R)0 : fdiv<R>(bp.k3 * Nu * g.lam, d) * ((R)kPI * d * d);
  const R Qconv = hA * (g.T - Tp);
  const bool cpl = coupled_step(bp.ncouple, V.step_ctr);
  const R dtm = bp.dtg;
  KinOut<R> kn;
  uscm<R>(bp, m, Tp, d, ore, g, re02, re07, dtm, kn);
  R mp = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) mp += m[q];   // the same sum as parcel_mass
  const R I = (R)0.4 * mp * r * r;
  R a[3];
  a[0] = fdiv<R>(F[0] + Fd[0], mp);
  a[1] = fdiv<R>(F[1] + Fd[1], mp);
  a[2] = fdiv<R>(F[2] + Fd[2] - Vp * bp.dpdz, mp) + bp.grav;
  // second half kick (the whole-step velocity and spin), then the first half kick of the next
  // step with the key kernel's expression: the state keeps the half-step velocity and spin,
  // so the next step's drift reads neither the accelerations nor writes the velocities back
  const double dt_d = V.beds[meta >> 8].dt;
  R vnew[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const R al = fdiv<R>(Tq[q], I);
    const R v1 = vh[q] + a[q] * bp.half_dt, w1 = wv[q] + al * bp.half_dt;
    vnew[q] = half_kick<R>(bp.half_dt, dt_d, v1, a[q]);
    V.A.v[q][i] = vnew[q];
    V.A.w[q][i] = w1 + al * bp.half_dt;
    if (full) {
      V.A.a[q][i] = a[q];
      V.A.al[q][i] = al;
    }
  }
  const Tab<R> &t = tab<R>();
  R cpp = 0;
  const R inv_mp = frcp<R>(mp);
#pragma unroll
  for (int q = 0; q < 4; ++q) cpp += m[q] * inv_mp * cp_over_R<R>(3 + q, Tp) * t.RMz[q];
  R Qrad = 0;
  if constexpr (RAD) Qrad = (fl & DEM_RADIATION) ? V.qrad[i] : (R)0;   // k_radiation, this step
  const R Tn = RAD ? Tp + fdiv<R>(bp.dt * (Qconv + kn.Qr + kn.Qrm + Qrad + Qcond), mp * cpp)
                   : Tp + fdiv<R>(bp.dt * (Qconv + kn.Qr + kn.Qrm + Qcond), mp * cpp);
  V.A.T[i] = Tn;
  if (cpl) {
#pragma unroll
    for (int q = 0; q < 4; ++q) mass_add<P>(V.A.m[q], i, kn.mdot[q] * dtm);
  }
  if (!isfinite(Tn) || !isfinite(vnew[0] + vnew[1] + vnew[2])) set_error(V.err, ERR_NONFINITE);
  // contributions to the cell sums: the rows the gas update reads at coupling steps (and on
  // a call's last step, for dem_get_sources), the others on a call's last step
  const size_t cp = (size_t)V.cap;
  R *s = V.src;
  if (cpl || full) {
    s[SR_VS * cp + i] = Vp;
    s[SR_SH2 * cp + i] = kn.sH2;
    s[SR_SH2O * cp + i] = kn.sH2O;
    s[SR_HA * cp + i] = hA;
    s[SR_HAT * cp + i] = hA * Tp;
    s[SR_QRM * cp + i] = kn.Qrm;
  }
  if (full) {
    s[SR_K * cp + i] = Kp;
    s[SR_KVX * cp + i] = Kp * vh[0];
    s[SR_KVY * cp + i] = Kp * vh[1];
    s[SR_KVZ * cp + i] = Kp * vh[2];
    s[SR_QR * cp + i] = kn.Qr;
    s[SR_EQ * cp + i] = kn.EQ;
    s[SR_ES * cp + i] = kn.ES;
  }
  if (V.diag)
    gp_write_diag<R>(V.diag, cp, i, F, Tq, Fd, kn, Kp, Qconv, Nu, Re, (long long)c - V.beds[meta >> 8].cell_off, Qrad,
                     Qcond, !RAD || !(fl & DEM_RADIATION));
}

// ---------------------------------------------------------------------------------------
// Per gas cell: sum the sources of its parcels in sorted order, update the gas state
// (coupling steps), and recompute the cell's properties for the next step.
// ---------------------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ void store_props(StepView<P> &V, long long c, const CellProps<typename P::R> &p) {
  using R = typename P::R;
  R r[GP_STRIDE];
  r[GP_RHO] = p.rho; r[GP_MU] = p.mu; r[GP_LAM] = p.lam; r[GP_CP] = p.cp; r[GP_X] = p.x; r[GP_DM] = p.Dm;
  r[GP_SC13] = p.sc13; r[GP_PR13] = p.pr13; r[GP_EPOW] = p.epow; r[GP_D0] = p.D[0]; r[GP_D1] = p.D[1];
  r[GP_UZ] = p.uz; r[GP_EPS] = p.eps; r[GP_TG] = p.T; r[GP_UX] = p.ux; r[GP_UY] = p.uy;
  // the record in vector stores (a warp writes whole sectors)
  if constexpr (sizeof(R) == 4) {
    float4 *q = reinterpret_cast<float4 *>(V.gp + (size_t)c * GP_STRIDE);
#pragma unroll
    for (int k = 0; k < GP_STRIDE / 4; ++k) q[k] = make_float4(r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
  } else {
    double2 *q = reinterpret_cast<double2 *>(V.gp + (size_t)c * GP_STRIDE);
#pragma unroll
    for (int k = 0; k < GP_N / 2; ++k) q[k] = make_double2(r[2 * k], r[2 * k + 1]);
  }
}

// sums of the per-parcel sources of [jb, je): FP64 in the FP64 form, compensated FP32
// (Kahan) in the FP32 forms; MASK selects the rows summed (the others stay 0)
constexpr unsigned SR_ALL = (1u << SR_CNT) - 1u;
// the rows the prescribed gas update reads
constexpr unsigned SR_GAS = (1u << SR_VS) | (1u << SR_SH2) | (1u << SR_SH2O) | (1u << SR_HA) | (1u << SR_HAT) |
                            (1u << SR_QRM);
template <class P> struct CellSum {
  using S = typename P::R;
  S s[SR_N];
  template <unsigned MASK = SR_ALL>
  __device__ __forceinline__ void run(const S *src, size_t cp, const unsigned *vals, unsigned jb, unsigned je) {
    if constexpr (!P::exact) {
      float cc[SR_CNT];
#pragma unroll
      for (int f = 0; f < SR_CNT; ++f) { s[f] = 0.f; cc[f] = 0.f; }
      for (unsigned jj = jb; jj < je; ++jj) {
        const unsigned j = vals[jj];
#pragma unroll
        for (int f = 0; f < SR_CNT; ++f) {
          if (!((MASK >> f) & 1u)) continue;
          const float y = src[f * cp + j] - cc[f];
          const float t = s[f] + y;
          cc[f] = (t - s[f]) - y;
          s[f] = t;
        }
      }
#pragma unroll
      for (int f = 0; f < SR_CNT; ++f) s[f] -= cc[f];
    } else {
#pragma unroll
      for (int f = 0; f < SR_CNT; ++f) s[f] = 0.0;
      for (unsigned jj = jb; jj < je; ++jj) {
        const unsigned j = vals[jj];
#pragma unroll
        for (int f = 0; f < SR_CNT; ++f)
          if ((MASK >> f) & 1u) s[f] += src[f * cp + j];
      }
    }
    s[SR_CNT] = (S)(je - jb);
  }
};

template <class P>
__device__ __forceinline__ void cell_step(StepView<P> &V, long long c, int mode /* 0 step, 1 eps init */) {
  using R = typename P::R;
  const int b = V.cell_bed[c];
  const DevBed &B = V.beds[b];
  const BedP<R> &bp = V.bp[b];
  const size_t nc = (size_t)V.ncells;
  const double *G = V.gas;
  double *Gn = V.gas_new;
  const bool solid = V.mark[c] != 0;
  const size_t cp = (size_t)V.cap;
  const long long layer = (long long)B.nx * B.ny;
  const bool cpl = coupled_step(bp.ncouple, V.step_ctr);
  // Between coupling steps the gas state does not change, and the other buffer already holds
  // it, unless the last step was a coupling step (or the first after dem_init) or an input
  // arrived since (dem_set_gas sets step_ctr[5]; the step counter clears it): then it is
  // copied across once. The stored property records are those of the unchanged state.
  if (mode == 0 && !cpl && V.step_ctr[0] % bp.ncouple != 0 && V.step_ctr[5] == 0) return;
  const bool update = mode == 0 && !solid && cpl && !(bp.flags & DEM_NO_GAS_UPDATE);
  if constexpr (P::exact) {
    // the all-FP64 form: the oracle's expressions
    double eps = G[GS_EPS * nc + c], Y[3] = {G[GS_Y0 * nc + c], G[GS_Y1 * nc + c], G[GS_Y2 * nc + c]};
    double T = G[GS_T * nc + c];
    if (mode == 1) {
      double vs = 0.0;
      for (unsigned j = V.cstart[c]; j < V.cend[c]; ++j) vs += (double)V.src[SR_VS * cp + V.vals[j]];
      eps = solid ? B.eps_min : fmax(1.0 - vs / B.vcell, B.eps_min);
    } else if (update) {
      CellSum<P> S;
      S.run<SR_GAS>(V.src, cp, V.vals, V.cstart[c], V.cend[c]);
      const bool up = c - B.cell_off >= layer && !V.mark[c - layer];
      const double dtg = B.ncouple * B.dt;
      const double rho = (double)V.gp[(size_t)c * GP_STRIDE + GP_RHO], cpg = (double)V.gp[(size_t)c * GP_STRIDE + GP_CP];
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
    }
    Gn[GS_EPS * nc + c] = eps;
    Gn[GS_Y0 * nc + c] = Y[0]; Gn[GS_Y1 * nc + c] = Y[1]; Gn[GS_Y2 * nc + c] = Y[2];
    Gn[GS_T * nc + c] = T;
    const CellProps<double> p = gas_cell_props<double>(bp, eps, Y, T);
    store_props(V, c, p);
  } else {
    // FP32 forms: FP32 increments added to compensated FP32 pairs; no FP64 arithmetic
    const float2 *G2 = reinterpret_cast<const float2 *>(G);
    float2 *Gn2 = reinterpret_cast<float2 *>(Gn);
    float2 eps2 = G2[GS_EPS * nc + c], T2 = G2[GS_T * nc + c];
    float2 Y2[3] = {G2[GS_Y0 * nc + c], G2[GS_Y1 * nc + c], G2[GS_Y2 * nc + c]};
    if (mode == 1) {
      float vs = 0.f, cc = 0.f;
      for (unsigned j = V.cstart[c]; j < V.cend[c]; ++j) {
        const float y = V.src[SR_VS * cp + V.vals[j]] - cc, t = vs + y;
        cc = (t - vs) - y;
        vs = t;
      }
      const float e = (float)1 - (vs - cc) * bp.inv_vcell;
      eps2 = make_float2(solid ? bp.eps_min : (e > bp.eps_min ? e : bp.eps_min), 0.f);
    } else if (update) {
      CellSum<P> S;
      S.run<SR_GAS>(V.src, cp, V.vals, V.cstart[c], V.cend[c]);
      const bool up = c - B.cell_off >= layer && !V.mark[c - layer];
      const Tab<R> &t = tab<R>();
      const R dtg = bp.dtg;
      const R eps_r = eps2.x + eps2.y, T_r = T2.x + T2.y;
      const R uz = bp.U_in / eps_r;
      const R Yr[3] = {Y2[0].x + Y2[0].y, Y2[1].x + Y2[1].y, Y2[2].x + Y2[2].y};
      // the density and heat capacity of the old state, computed as its property record holds
      // them (the record is a function of these FP32 values), instead of read from the record
      const R rho = gas_density<R>(bp, gas_molar_mass<R>(Yr), T_r), cpg = gas_heat_capacity<R>(Yr, T_r);
      R Yup[3] = {bp.Y_in[0], bp.Y_in[1], bp.Y_in[2]}, Tup = bp.T_in;
      if (up) {   // the old state of the cell below
        Yup[0] = gas_r<P>(G, GS_Y0 * nc + c - layer); Yup[1] = gas_r<P>(G, GS_Y1 * nc + c - layer);
        Yup[2] = gas_r<P>(G, GS_Y2 * nc + c - layer);
        Tup = gas_r<P>(G, GS_T * nc + c - layer);
      }
      const R Sj[3] = {S.s[SR_SH2], S.s[SR_SH2O], (R)0};
      const R Snet = Sj[0] + Sj[1];
      const R inv_mg = bp.inv_vcell / (eps_r * rho);
      bool clamp = false;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const R dy = dtg * (-uz * (Yr[j] - Yup[j]) * bp.inv_dz + (Sj[j] - Yr[j] * Snet) * inv_mg);
        Y2[j] = pair_add(Y2[j], dy);
        if (Y2[j].x + Y2[j].y < 0.f) { Y2[j] = make_float2(0.f, 0.f); clamp = true; }
      }
      if (clamp) {
        const float ys = (Y2[0].x + Y2[0].y) + (Y2[1].x + Y2[1].y) + (Y2[2].x + Y2[2].y);
#pragma unroll
        for (int j = 0; j < 3; ++j) Y2[j] = make_float2(ys > 0.f ? (Y2[j].x + Y2[j].y) / ys : Yr[j], 0.f);
      }
      const R capc = eps_r * rho * cpg;
      const R H0 = S.s[SR_HA] * bp.inv_vcell, H1 = S.s[SR_HAT] * bp.inv_vcell;
      const R Mrm = -S.s[SR_QRM] * bp.inv_vcell;
      const R Mr = -(h_over_R<R>(0, T_r) * t.RMj[0] * Sj[0] + h_over_R<R>(1, T_r) * t.RMj[1] * Sj[1]) * bp.inv_vcell;
      // T' - T of the semi-implicit update (eq (4-6)), H1 - H0 T formed before dividing
      const R num = dtg * (-uz * (T_r - Tup) * bp.inv_dz + (H1 - H0 * T_r + Mr + Mrm) / capc);
      const R den = (R)1 + dtg * H0 / capc;
      T2 = pair_add(T2, num / den);
      const R epsn = (R)1 - S.s[SR_VS] * bp.inv_vcell;
      eps2 = make_float2(epsn > bp.eps_min ? epsn : bp.eps_min, 0.f);
    }
    Gn2[GS_EPS * nc + c] = eps2;
    Gn2[GS_Y0 * nc + c] = Y2[0]; Gn2[GS_Y1 * nc + c] = Y2[1]; Gn2[GS_Y2 * nc + c] = Y2[2];
    Gn2[GS_T * nc + c] = T2;
    const R Yr[3] = {Y2[0].x + Y2[0].y, Y2[1].x + Y2[1].y, Y2[2].x + Y2[2].y};
    const R epsr = eps2.x + eps2.y, Tr = T2.x + T2.y;
    if (mode == 0) {
      // the properties are a function of the FP32 values of (eps, Y, T): when none of them
      // changed in this step, the stored properties are already the ones they give
      const float2 eo = G2[GS_EPS * nc + c], to = G2[GS_T * nc + c];
      const float2 y0 = G2[GS_Y0 * nc + c], y1 = G2[GS_Y1 * nc + c], y2 = G2[GS_Y2 * nc + c];
      if (epsr == eo.x + eo.y && Tr == to.x + to.y && Yr[0] == y0.x + y0.y && Yr[1] == y1.x + y1.y &&
          Yr[2] == y2.x + y2.y)
        return;
    }
    const CellProps<R> p = gas_cell_props<R>(bp, epsr, Yr, Tr);
    store_props(V, c, p);
  }
}

// One thread per gas cell (48 registers in the FP32 forms, as the screen pass).
template <class P>
__global__ void __launch_bounds__(256, P::exact ? 1 : 5) k_cells(StepView<P> V, int mode) {
  pdl_wait();
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < V.ncells) cell_step<P>(V, c, mode);
}

// The coupling input (dem_set_gas): the gas composition and temperature of every cell from
// the caller (FP64; device memory, or mapped pinned host memory read directly), written to
// the other gas-state buffer with the volume fraction kept, and the cell's property record
// for the next step; in the FP32 forms only where the FP32 state changed (as in k_cells).
template <class P>
__global__ void k_gas_set_props(StepView<P> V, const double *__restrict__ Yin /* ncells*3 */,
                                const double *__restrict__ Tin, long long *ctr) {
  using R = typename P::R;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells) return;
  if (c == 0) ctr[5] = 1;   // the buffers differ: the next step's k_cells copies
  const BedP<R> &bp = V.bp[V.cell_bed[c]];
  const size_t nc = (size_t)V.ncells;
  const double y0 = Yin[c * 3], y1 = Yin[c * 3 + 1], y2 = Yin[c * 3 + 2], tg = Tin[c];
  if constexpr (P::exact) {
    const double eps = V.gas[GS_EPS * nc + c];
    V.gas_new[GS_EPS * nc + c] = eps;
    V.gas_new[GS_Y0 * nc + c] = y0; V.gas_new[GS_Y1 * nc + c] = y1; V.gas_new[GS_Y2 * nc + c] = y2;
    V.gas_new[GS_T * nc + c] = tg;
    const double Y[3] = {y0, y1, y2};
    store_props(V, c, gas_cell_props<double>(bp, eps, Y, tg));
  } else {
    const float2 *G2 = reinterpret_cast<const float2 *>(V.gas);
    const float2 eps2 = G2[GS_EPS * nc + c];
    V.gas_new[GS_EPS * nc + c] = V.gas[GS_EPS * nc + c];
    gas_put(V.gas_new, GS_Y0 * nc + c, y0, true);
    gas_put(V.gas_new, GS_Y1 * nc + c, y1, true);
    gas_put(V.gas_new, GS_Y2 * nc + c, y2, true);
    gas_put(V.gas_new, GS_T * nc + c, tg, true);
    const float2 *N2 = reinterpret_cast<const float2 *>(V.gas_new);
    const float2 n0 = N2[GS_Y0 * nc + c], n1 = N2[GS_Y1 * nc + c], n2 = N2[GS_Y2 * nc + c], nt = N2[GS_T * nc + c];
    const R Yr[3] = {n0.x + n0.y, n1.x + n1.y, n2.x + n2.y};
    const R Tr = nt.x + nt.y, epsr = eps2.x + eps2.y;
    const float2 to = G2[GS_T * nc + c], o0 = G2[GS_Y0 * nc + c], o1 = G2[GS_Y1 * nc + c], o2 = G2[GS_Y2 * nc + c];
    if (Tr == to.x + to.y && Yr[0] == o0.x + o0.y && Yr[1] == o1.x + o1.y && Yr[2] == o2.x + o2.y) return;
    store_props(V, c, gas_cell_props<R>(bp, epsr, Yr, Tr));
  }
}

// Cell sums of the last step's per-parcel sources (dem_get_sources).
template <class P>
__global__ void k_sources(StepView<P> V) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= V.ncells) return;
  const size_t cp = (size_t)V.cap;
  CellSum<P> S;
  S.run(V.src, cp, V.vals, V.cstart[c], V.cend[c]);
  const bool solid = V.mark[c] != 0;
  for (int f = 0; f < SR_N; ++f) V.dep[(size_t)c * SR_N + f] = solid ? 0.0 : (double)S.s[f];
}

// Cell sums of the last step's per-parcel sources for the fluid cells that hold parcels
// (dem_get_sources_occupied), compacted in increasing cell order: the occupied cells are the
// starts of the runs of equal keys in the sorted order. Three passes, deterministic: a count
// per chunk of OCC_CHUNK sorted positions, an exclusive scan of the counts in one block, and
// the writes (each chunk's block ranks its run starts with a block-wide scan).
constexpr int OCC_BLOCK = 256;
constexpr int OCC_PER_THREAD = 4;
constexpr int OCC_CHUNK = OCC_BLOCK * OCC_PER_THREAD;
template <class P>
__device__ __forceinline__ bool occ_start(const StepView<P> &V, int s) {
  if (s >= V.n) return false;
  const unsigned k = V.keys[s];
  return (s == 0 || V.keys[s - 1] != k) && V.mark[k] == 0;
}
template <class P>
__global__ void __launch_bounds__(OCC_BLOCK) k_occ_count(StepView<P> V, int *cnt) {
  const int s0 = blockIdx.x * OCC_CHUNK + threadIdx.x * OCC_PER_THREAD;
  int m = 0;
#pragma unroll
  for (int q = 0; q < OCC_PER_THREAD; ++q) m += occ_start(V, s0 + q) ? 1 : 0;
  m = __reduce_add_sync(0xffffffffu, m);
  __shared__ int w[OCC_BLOCK / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < OCC_BLOCK / 32; ++k) t += w[k];
    cnt[blockIdx.x] = t;
  }
}
// exclusive scan of nb counts in place, total in cnt[nb] (one block)
static __global__ void __launch_bounds__(1024) k_occ_scan(int *cnt, int nb) {
  __shared__ int carry;
  __shared__ int ws[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? cnt[i] : 0;
    int x = v;   // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      int t = ws[threadIdx.x];
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (threadIdx.x >= o) t += y;
      }
      ws[threadIdx.x] = t;
    }
    __syncthreads();
    const int incl = x + ((threadIdx.x >> 5) ? ws[(threadIdx.x >> 5) - 1] : 0);
    if (i < nb) cnt[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[nb] = carry;
}
template <class P>
__global__ void __launch_bounds__(OCC_BLOCK) k_occ_write(StepView<P> V, const int *off, long long *cells,
                                                         double *out /* [occupied][SR_N] */) {
  const int s0 = blockIdx.x * OCC_CHUNK + threadIdx.x * OCC_PER_THREAD;
  bool f[OCC_PER_THREAD];
  int m = 0;
#pragma unroll
  for (int q = 0; q < OCC_PER_THREAD; ++q) { f[q] = occ_start(V, s0 + q); m += f[q] ? 1 : 0; }
  // exclusive block scan of m
  int x = m;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) >= o) x += y;
  }
  __shared__ int ws[OCC_BLOCK / 32];
  if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
  __syncthreads();
  int before = 0;
  for (int k = 0; k < (int)(threadIdx.x >> 5); ++k) before += ws[k];
  int pos = off[blockIdx.x] + before + x - m;
  const size_t cp = (size_t)V.cap;
#pragma unroll
  for (int q = 0; q < OCC_PER_THREAD; ++q) {
    if (!f[q]) continue;
    const unsigned c = V.keys[s0 + q];
    CellSum<P> S;
    S.run(V.src, cp, V.vals, V.cstart[c], V.cend[c]);
    cells[pos] = (long long)c;
    for (int g = 0; g < SR_N; ++g) out[(size_t)pos * SR_N + g] = (double)S.s[g];
    ++pos;
  }
}

// Initial per-parcel volume for the initial gas volume fraction.
template <class P>
__global__ void k_volume(StepView<P> V) {
  using R = typename P::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const BedP<R> &bp = V.bp[V.A.meta[i] >> 8];
  const R dc = bp.k * V.A.d[i];
  V.src[SR_VS * (size_t)V.cap + i] = (R)(kPI / 6.0) * dc * dc * dc;
}

// ---------------------------------------------------------------------------------------
// Reduction degree (eqs (2-15)..(2-19)) per parcel and per bed (deterministic two-pass).
// ---------------------------------------------------------------------------------------
constexpr int FOV_CHUNKS = 1024;  // blocks per bed of the reduction-degree sums
constexpr int FOV_BLOCK = 128;    // threads per block of k_fov_chunks
static_assert(FOV_CHUNKS % 256 == 0, "k_fov_beds adds FOV_CHUNKS / 256 slices per thread");

// Each bed's parcels occupy a fixed range of storage positions; block (bed, chunk) sums a
// fixed slice of them (strided per thread, then a shared-memory tree in FP64), and k_fov_beds
// adds the slices in a fixed order, so the result is reproducible bit for bit. The FP64 form
// evaluates f_ov in FP64; the FP32 forms in FP32 (relative error ~1e-7 per parcel) with
// compensated per-thread sums.
template <class P>
__global__ void k_fov_chunks(StepView<P> V, double *per_parcel_orig, double *part /* [nbeds][FOV_CHUNKS][4] */) {
  __shared__ double sh[3][FOV_BLOCK];
  const int b = blockIdx.x / FOV_CHUNKS, ch = blockIdx.x % FOV_CHUNKS;
  const int p0 = V.beds[b].pstart;
  const long long len = V.beds[b].pend - p0;
  const int c0 = p0 + (int)(len * ch / FOV_CHUNKS), c1 = p0 + (int)(len * (ch + 1) / FOV_CHUNKS);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  if constexpr (P::exact) {
    const Tab<double> &td = tab<double>();
    for (int i = c0 + (int)threadIdx.x; i < c1; i += blockDim.x) {
      const int ore = V.A.meta[i] & 255;
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
      a0 += f;
      a1 += 3.0 * n[0] + 4.0 * n[1] + n[2];
      a2 += (ore == 0 ? 1.5 : 4.0 / 3.0) * nfe;
    }
  } else {
    const Tab<float> &tf = tab<float>();
    float iM[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) iM[q] = 1.0f / tf.Mz[q];
    float s[3] = {0.f, 0.f, 0.f}, cc[3] = {0.f, 0.f, 0.f};
    for (int i = c0 + (int)threadIdx.x; i < c1; i += blockDim.x) {
      const int ore = V.A.meta[i] & 255;
      float n[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) n[q] = mass_r<P>(V.A.m[q], i) * iM[q];
      const float nfe = 2.f * n[0] + 3.f * n[1] + n[2] + n[3];
      float f = 0.f;
      if (nfe > 0.f) {
        const float inv = 1.0f / nfe;
        const float fh = (3.f * n[1] + n[2] + n[3]) * inv, fm = (n[2] + n[3]) * inv, fw = n[3] * inv;
        f = ore == 0 ? (fh + 2.f * fm + 6.f * fw) * (1.0f / 9.0f) : 0.25f * fm + 0.75f * fw;
      }
      if (per_parcel_orig) per_parcel_orig[V.A.orig[i]] = (double)f;
      const float v[3] = {f, 3.f * n[0] + 4.f * n[1] + n[2], (ore == 0 ? 1.5f : 4.0f / 3.0f) * nfe};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float y = v[q] - cc[q], t = s[q] + y;
        cc[q] = (t - s[q]) - y;
        s[q] = t;
      }
    }
    a0 = (double)s[0] - (double)cc[0];
    a1 = (double)s[1] - (double)cc[1];
    a2 = (double)s[2] - (double)cc[2];
  }
  sh[0][threadIdx.x] = a0; sh[1][threadIdx.x] = a1; sh[2][threadIdx.x] = a2;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double *o = part + (size_t)blockIdx.x * 4;
    o[0] = sh[0][0]; o[1] = sh[1][0]; o[2] = sh[2][0]; o[3] = (double)(c1 - c0);
  }
}

// One block per bed: each thread adds FOV_CHUNKS / 256 consecutive slices in order, then a
// fixed shared-memory tree.
static __global__ void __launch_bounds__(256) k_fov_beds(const double *part, int nbeds, double *out /* [nbeds][4] */) {
  __shared__ double sh[4][256];
  const int b = blockIdx.x;
  constexpr int per = FOV_CHUNKS / 256;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < per; ++k) {
    const double *p = part + ((size_t)b * FOV_CHUNKS + threadIdx.x * per + k) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += p[q];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[b * 4 + threadIdx.x] = sh[threadIdx.x][0];
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
  const DevBed &B = V.beds[V.A.meta[i] >> 8];
  const auto &bp = V.bp[V.A.meta[i] >> 8];
  out[0 * n + o] = pos_abs<P>(V.A.x, i, B.x0); out[1 * n + o] = pos_abs<P>(V.A.y, i, B.y0);
  out[2 * n + o] = pos_abs<P>(V.A.z, i, B.z0);
#pragma unroll
  for (int q = 0; q < 3; ++q) {   // the whole-step velocity and spin (the state holds the half-step ones)
    out[(3 + q) * n + o] = (double)half_kick_back(bp.half_dt, B.dt, V.A.v[q][i], V.A.a[q][i]);
    out[(6 + q) * n + o] = (double)half_kick_back(bp.half_dt, B.dt, V.A.w[q][i], V.A.al[q][i]);
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

__global__ void k_mark_cells(const DevBed *beds, const BedP<double> *bps, const int *cell_bed, unsigned char *mark,
                             unsigned char *wnear, long long ncells);
__global__ void k_step_counter(StepEnd se);

}  // namespace dem
