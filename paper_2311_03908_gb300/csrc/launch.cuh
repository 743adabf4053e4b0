// launch.cuh -- host-side orchestration of the per-step kernels for one arithmetic type.
// Included by inst_f64.cu, inst_f32.cu and inst_kahan.cu, which instantiate it per precision form.
#pragma once
#include "ctx.cuh"
#include "radix.cuh"

namespace dem {

inline int grid_for(long long n, int bs) { return (int)((n + bs - 1) / bs); }
// grid of a grid-stride kernel: at most one wave of full-occupancy blocks
inline int grid_wave(const dem_ctx *c, long long n, int bs) {
  const int g = grid_for(n, bs), w = c->nsm * (2048 / bs);
  return g < w ? g : w;
}

template <class P>
StepView<P> make_view(dem_ctx *c, bool for_step) {
  using R = typename P::R;
  StepView<P> V;
  V.n = c->n;
  V.cap = c->cap;
  V.nbeds = c->nbeds;
  V.ncells = c->ncells;
  V.beds = c->dbeds;
  if constexpr (sizeof(R) == 8) V.bp = c->dbp_d; else V.bp = c->dbp_f;
  // a: buffers of the state before the step (the current ones between steps), b: after it
  const int a = c->cur, b = for_step ? 1 - c->cur : c->cur;
  auto fill = [&](PState<R> &Pp, int k) {
    Pp.x = c->px[k][0]; Pp.y = c->px[k][1]; Pp.z = c->px[k][2];
    for (int q = 0; q < 3; ++q) {
      Pp.v[q] = (R *)c->pv[k][q]; Pp.w[q] = (R *)c->pw[k][q];
      Pp.a[q] = (R *)c->pa[k][q]; Pp.al[q] = (R *)c->pal[k][q];
    }
    Pp.T = (R *)c->pT[k];
    Pp.d = (R *)c->pd[k];
    for (int q = 0; q < 4; ++q) Pp.m[q] = c->pm[k][q];
    Pp.meta = c->pmeta[k];
    Pp.orig = c->porig[k];
    for (int q = 0; q < 3; ++q) Pp.dsp[q] = c->pdsp[k][q];
  };
  fill(V.A, 0);   // the state, always in buffer 0
  fill(V.S, 1);   // scratch of a re-store
  V.H.cnt = c->hcnt[a]; V.H.id = c->hid[a]; V.H.xi = (R *)c->hxi[a];
  V.Hn.cnt = c->hcnt[b]; V.Hn.id = c->hid[b]; V.Hn.xi = (R *)c->hxi[b];
  V.Hs = V.Hn;    // the re-store runs before the contacts write the new history
  V.keyp = c->keys;
  V.keys = c->skey[b];
  V.vals = c->sval[b];
  V.keys_prev = c->skey[a];
  V.vals_prev = c->sval[a];
  V.knew = c->keys2;
  V.inv = c->inv;
  V.cstart = c->cstart; V.cend = c->cend;
  V.xl = c->xl;
  for (int q = 0; q < 3; ++q) { V.F[q] = (R *)c->F[q]; V.Tq[q] = (R *)c->Tq[q]; }
  V.xls = reinterpret_cast<float4 *>(c->src);
  V.plist = c->plist;
  V.pcode = c->pcode;
  V.pcnt = c->pcnt;
  V.nl = c->nl;
  V.nlc = c->nlc;
  V.rebuild = c->rebuild;
  V.nolists = c->use_lists ? 0 : 1;
  V.corner = c->corner;
  V.cornerp = c->cornerp;
  V.moved = resort_counts(c->rsw, c->rs_pow2, c->n);
  V.src = (R *)c->src;
  V.gas = c->gas[c->gcur];
  V.gas_new = c->gas[1 - c->gcur];
  V.gp = (R *)c->gp;
  V.mark = c->mark;
  V.cell_bed = c->cell_bed;
  V.diag = c->diag_on ? c->diag : nullptr;
  V.dep = c->dep;
  V.err = c->err;
  V.step_ctr = c->step_ctr;
  V.restore_every = c->restore_every;
  V.list_acc = (unsigned long long *)(c->step_ctr + 3);
  V.ovf = c->ovf;
  V.novf = c->novf;
  V.work = c->work;
  V.nwork = c->nwork;
  V.wnear = c->wnear;
  V.qrad = (R *)c->qrad;
  V.tsrt = (R *)c->tsrt;
  V.xr = c->xr;
  V.rad = c->any_rad ? 1 : 0;
  V.qc = (R *)c->qc;
  return V;
}

// storage positions 0..n-1 (the radix sort's values at the first binning)
static __global__ void k_iota(unsigned *v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (unsigned)i;
}

// Binning: drift and keys in storage order, then the sorted order of the keys (incremental
// re-sort from the previous step's; LSD radix sort at the first binning), the cell ranges,
// and on list-build steps a re-store of the parcels in that order.
template <class P>
int enqueue_binning(dem_ctx *c, int drift) {
  cudaStream_t st = c->st;
  StepView<P> V = make_view<P>(c, true);
  // the per-1024 counts of changed keys start at zero (k_ranges clears them after use)
  const bool pdl = !c->prof_on;   // per-kernel event timing wants plain stream order
  int ps = prof_begin(c, "k_key");
  // two parcels per thread, 32 apart: ceil(n / 64) warps
  launch_k(pdl, k_key<P>, grid_for(((long long)c->n + 63) / 64 * 32, c->bs_key), c->bs_key, st, V, drift);
  prof_end(c, ps);
  ++c->launches;
  const int nxt = 1 - c->cur;
  if (drift) {
    ps = prof_begin(c, "resort");
    int e = resort_pairs(c->skey[c->cur], c->keys2, c->sval[c->cur], c->skey[nxt], c->sval[nxt], c->rsw, c->rs_pow2,
                         c->n, st, &c->launches, pdl);
    if (e) return e;
    prof_end(c, ps);
    ps = prof_begin(c, "k_ranges");   // the key kernel emptied the previous step's ranges
    launch_k(pdl, k_ranges<P>, grid_for((c->n + 3) / 4, c->bs_restore), c->bs_restore, st, V, 0);
    prof_end(c, ps);
    ++c->launches;
  } else {
    // first binning: LSD radix sort of (key, storage position)
    ps = prof_begin(c, "radix_sort");
    cudaMemcpyAsync(c->keys2, c->keys, sizeof(unsigned) * c->n, cudaMemcpyDeviceToDevice, st);
    k_iota<<<grid_for(c->n, 256), 256, 0, st>>>(c->vals2, c->n);
    unsigned *kr = nullptr, *vr = nullptr;
    int e = radix_sort_pairs(c->keys2, c->vals2, c->skey[nxt], c->sval[nxt], c->rhist, c->n, c->key_bits, st,
                             &kr, &vr, &c->launches);
    if (e) return e;
    if (kr != c->skey[nxt]) {
      cudaMemcpyAsync(c->skey[nxt], kr, sizeof(unsigned) * c->n, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(c->sval[nxt], vr, sizeof(unsigned) * c->n, cudaMemcpyDeviceToDevice, st);
    }
    cudaMemsetAsync(c->cstart, 0, sizeof(unsigned) * c->ncells, st);
    cudaMemsetAsync(c->cend, 0, sizeof(unsigned) * c->ncells, st);
    k_ranges<P><<<grid_for((c->n + 3) / 4, 256), 256, 0, st>>>(V, 1);
    prof_end(c, ps);
    c->launches += 2;
  }
  // the re-store's second half (k_ranges copied the records out)
  ps = prof_begin(c, "k_restore");
  launch_k(pdl, k_restore_in<P>, grid_wave(c, c->n, c->bs_restore), c->bs_restore, st, V, drift ? 0 : 1);
  prof_end(c, ps);
  ++c->launches;
  return (int)cudaPeekAtLastError();
}

// The gas solver's kernels of one step (beds with DEM_GAS_SOLVER), in place of k_cells: on
// coupling steps the cell sums and coefficients, the species and energy update (and the new
// densities), the momentum predictor, the pressure equation, the cooperative conjugate-
// gradient solve, the projection and the cells' property records; on the other steps the
// species kernel copies the state and the others return at once.
template <class P>
int enqueue_gas_solve(dem_ctx *c, StepView<P> &V, bool pdl) {
  cudaStream_t st = c->st;
  const GasView &S = c->gsv;
  const long long nf = S.nfx + S.nfy + S.nfz;
  int ps = prof_begin(c, "k_gs_coeffs");
  launch_k(pdl, k_gs_coeffs<P>, grid_for(c->ncells, 256), 256, st, V, S);
  prof_end(c, ps);
  ps = prof_begin(c, "k_gs_scalars");
  launch_k(pdl, k_gs_scalars<P>, grid_for(c->ncells, 256), 256, st, V, S);
  prof_end(c, ps);
  ps = prof_begin(c, "k_gs_predict");
  launch_k(pdl, k_gs_predict<P>, grid_for(nf, 256), 256, st, V, S);
  prof_end(c, ps);
  ps = prof_begin(c, "k_gs_rhs");
  launch_k(pdl, k_gs_rhs<P>, grid_for(c->ncells, 256), 256, st, V, S);
  prof_end(c, ps);
  ps = prof_begin(c, "k_gs_cg");
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c->gs_grid);
    cfg.blockDim = dim3(GS_CG_BLOCK);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_gs_cg<P>, (const DevBed *)c->dbeds, (const int *)c->cell_bed,
                           (const long long *)c->step_ctr, c->ncells, S) != cudaSuccess)
      return -1;
  }
  prof_end(c, ps);
  ps = prof_begin(c, "k_gs_correct");
  k_gs_correct<P><<<grid_for(nf + c->ncells, 256), 256, 0, st>>>(V, S);
  prof_end(c, ps);
  ps = prof_begin(c, "k_gs_props");
  k_gs_props<P><<<grid_for(c->ncells, 256), 256, 0, st>>>(V, S);
  prof_end(c, ps);
  c->launches += 7;
  return (int)cudaPeekAtLastError();
}

template <class P>
int enqueue_steps(dem_ctx *c, int nsteps) {
  cudaStream_t st = c->st;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return -1;
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  for (int s = 0; s < nsteps; ++s) {
    int e = enqueue_binning<P>(c, 1);
    if (e) return e;
    StepView<P> V = make_view<P>(c, true);
    const bool pdl = !c->prof_on;
    int ps;
    // the cell-list search (list builds, overflowed lists, no lists; otherwise a no-op), the
    // contact forces (with the list test between builds), then the gas-particle terms
    ps = prof_begin(c, "k_pair_search");
    launch_k(pdl, k_pair_search<P>, grid_wave(c, c->n, c->bs_search), c->bs_search, st, V);
    prof_end(c, ps);
    ps = prof_begin(c, "k_contact_screen");
    launch_k(pdl, k_contact_screen<P>, grid_for(c->n, c->bs_contacts), c->bs_contacts, st, V);
    prof_end(c, ps);
    ps = prof_begin(c, "k_contact_forces");
    launch_k(pdl, k_contact_forces<P>, grid_wave(c, c->n, 128), 128, st, V);
    prof_end(c, ps);
    // the first kernel that reads the gas state or the cell properties waits for a coupling
    // input still crossing on its own stream (dem_set_gas); a captured graph always carries
    // the wait, as an external-event node, since a later replay may follow a new input
    bool waited = false;
    if (s == 0 && (c->gas_pending || capturing)) {
      if (cudaStreamWaitEvent(st, c->ev_gas, capturing ? cudaEventWaitExternal : 0) != cudaSuccess) return -1;
      c->gas_pending = false;
      waited = true;
    }
    if (c->any_rad) {   // particle radiation, from the temperatures before the update
      ps = prof_begin(c, "k_radiation");
      launch_k(pdl && !waited, k_radiation<P>, grid_for(c->n, 128), 128, st, V);
      prof_end(c, ps);
      ++c->launches;
      waited = false;
    }
    ps = prof_begin(c, "k_gas_particle");
    // the accelerations and the sources only dem_get_sources and the gas solver read are
    // stored on a call's last step (every step when the gas is solved)
    const int last = (s == nsteps - 1 || c->gas_solver) ? 1 : 0;
    if (c->any_rad) launch_k(pdl && !waited, k_gas_particle<P, true>, grid_for(c->n, c->bs_gp), c->bs_gp, st, V, last);
    else launch_k(pdl && !waited, k_gas_particle<P, false>, grid_for(c->n, c->bs_gp), c->bs_gp, st, V, last);
    prof_end(c, ps);
    StepEnd se;   // the end of the step: its counters
    se.ctr = c->step_ctr;
    se.rebuild = c->rebuild;
    se.nwork = c->nwork;
    se.lists = c->use_lists;
    se.restore_every = c->restore_every;
    if (c->gas_solver) {
      e = enqueue_gas_solve<P>(c, V, pdl);
      if (e) return e;
    } else {
      ps = prof_begin(c, "k_cells");
      launch_k(pdl, k_cells<P>, grid_for(c->ncells, c->bs_cells), c->bs_cells, st, V, 0);
      prof_end(c, ps);
      ++c->launches;
    }
    launch_k(pdl, k_step_counter, 1, 1, st, se);
    c->launches += 5;
    e = (int)cudaPeekAtLastError();
    if (e) return e;
    c->cur = 1 - c->cur;
    c->gcur = 1 - c->gcur;
  }
  return 0;
}

template <class P>
int enqueue_init(dem_ctx *c) {
  cudaStream_t st = c->st;
  int e = enqueue_binning<P>(c, 0);
  if (e) return e;
  StepView<P> V = make_view<P>(c, true);
  k_volume<P><<<grid_for(c->n, 256), 256, 0, st>>>(V);
  k_cells<P><<<grid_for(c->ncells, 256), 256, 0, st>>>(V, 1);
  c->cur = 1 - c->cur;
  c->gcur = 1 - c->gcur;
  return (int)cudaPeekAtLastError();
}

template <class P>
int enqueue_fov(dem_ctx *c, double *per_parcel_dev) {
  StepView<P> V = make_view<P>(c, false);
  k_fov_chunks<P><<<c->nbeds * FOV_CHUNKS, FOV_BLOCK, 0, c->st>>>(V, per_parcel_dev, c->fv);
  k_fov_beds<<<c->nbeds, 256, 0, c->st>>>(c->fv, c->nbeds, c->fvbed);
  return (int)cudaPeekAtLastError();
}

template <class P>
int enqueue_scatter_state(dem_ctx *c, double *out_dev) {
  StepView<P> V = make_view<P>(c, false);
  k_scatter_state<P><<<grid_for(c->n, 256), 256, 0, c->st>>>(V, out_dev);
  return (int)cudaPeekAtLastError();
}

template <class P>
int enqueue_scatter_diag(dem_ctx *c, double *out_dev) {
  StepView<P> V = make_view<P>(c, false);
  V.diag = c->diag;
  k_scatter_diag<P><<<grid_for(c->n, 256), 256, 0, c->st>>>(V, out_dev);
  return (int)cudaPeekAtLastError();
}

template <class P>
int enqueue_scatter_hist(dem_ctx *c, int *cnt, int *partner, double *xi) {
  StepView<P> V = make_view<P>(c, false);
  k_scatter_hist<P><<<grid_for(c->n, 256), 256, 0, c->st>>>(V, cnt, partner, xi);
  return (int)cudaPeekAtLastError();
}

template <class P>
int enqueue_sources(dem_ctx *c) {
  StepView<P> V = make_view<P>(c, false);
  V.dep = c->dep;
  k_sources<P><<<grid_for(c->ncells, 256), 256, 0, c->st>>>(V);
  return (int)cudaPeekAtLastError();
}

// the occupied cells' source sums: counts per chunk into cnt[0..nb), their scan (total in
// cnt[nb]), then the compacted cells and sums
template <class P>
int enqueue_sources_occupied(dem_ctx *c, int *cnt, long long *cells, double *out) {
  StepView<P> V = make_view<P>(c, false);
  const int nb = (c->n + OCC_CHUNK - 1) / OCC_CHUNK;
  k_occ_count<P><<<nb, OCC_BLOCK, 0, c->st>>>(V, cnt);
  k_occ_scan<<<1, 1024, 0, c->st>>>(cnt, nb);
  k_occ_write<P><<<nb, OCC_BLOCK, 0, c->st>>>(V, cnt, cells, out);
  return (int)cudaPeekAtLastError();
}

template <class P>
int enqueue_gas_set(dem_ctx *c, const double *Y, const double *T, cudaStream_t st) {
  StepView<P> V = make_view<P>(c, false);
  V.gas = c->gas[c->gcur];
  V.gas_new = c->gas[1 - c->gcur];
  k_gas_set_props<P><<<grid_for(c->ncells, 256), 256, 0, st>>>(V, Y, T, c->step_ctr);
  c->gcur = 1 - c->gcur;
  return (int)cudaPeekAtLastError();
}

// the solved beds' initial flow and property records (after enqueue_init)
template <class P>
int enqueue_gas_solver_init(dem_ctx *c) {
  StepView<P> V = make_view<P>(c, false);
  const GasView &S = c->gsv;
  const long long nf = S.nfx + S.nfy + S.nfz;
  k_gs_init_faces<P><<<grid_for(nf + c->ncells, 256), 256, 0, c->st>>>(V, S);
  k_gs_init_props<P><<<grid_for(c->ncells, 256), 256, 0, c->st>>>(V, S);
  return (int)cudaPeekAtLastError();
}

template <class P>
int enqueue_flow(dem_ctx *c, double *out_dev) {
  StepView<P> V = make_view<P>(c, false);
  k_gs_flow<P><<<grid_for(c->ncells, 256), 256, 0, c->st>>>(V, c->gsv, c->gas_solver ? 1 : 0, out_dev);
  return (int)cudaPeekAtLastError();
}

template <class P>
int gas_cg_occupancy(int *blocks_per_sm) {
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_gs_cg<P>, GS_CG_BLOCK, 0);
}

// largest block each tunable kernel can launch with (registers per thread decide it)
template <class P>
int kernel_limits(int *lim) {
  const void *fn[6] = {(const void *)k_key<P>, (const void *)k_ranges<P>, (const void *)k_pair_search<P>,
                       (const void *)k_contact_screen<P>, (const void *)k_gas_particle<P, false>, (const void *)k_cells<P>};
  for (int k = 0; k < 6; ++k) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, fn[k]) != cudaSuccess) return -1;
    lim[k] = a.maxThreadsPerBlock;
  }
  cudaFuncAttributes a;   // the re-store block size serves k_ranges and k_restore_in
  if (cudaFuncGetAttributes(&a, (const void *)k_restore_in<P>) != cudaSuccess) return -1;
  lim[1] = lim[1] < a.maxThreadsPerBlock ? lim[1] : a.maxThreadsPerBlock;
  return 0;
}

#define DEM_INSTANTIATE(P)                                                             \
  template int kernel_limits<P>(int *);                                                 \
  template StepView<P> make_view<P>(dem_ctx *, bool);                                   \
  template int enqueue_steps<P>(dem_ctx *, int);                                        \
  template int enqueue_init<P>(dem_ctx *);                                              \
  template int enqueue_fov<P>(dem_ctx *, double *);                                     \
  template int enqueue_scatter_state<P>(dem_ctx *, double *);                           \
  template int enqueue_scatter_diag<P>(dem_ctx *, double *);                            \
  template int enqueue_scatter_hist<P>(dem_ctx *, int *, int *, double *);              \
  template int enqueue_sources<P>(dem_ctx *);                                           \
  template int enqueue_sources_occupied<P>(dem_ctx *, int *, long long *, double *);      \
  template int enqueue_gas_set<P>(dem_ctx *, const double *, const double *, cudaStream_t); \
  template int enqueue_gas_solver_init<P>(dem_ctx *);                                   \
  template int enqueue_flow<P>(dem_ctx *, double *);                                    \
  template int gas_cg_occupancy<P>(int *);

}  // namespace dem
