// launch.cuh -- host-side orchestration of the per-step kernels for one arithmetic type.
// Included by inst_f64.cu and inst_f32.cu, which instantiate it for double and float.
#pragma once
#include "ctx.cuh"
#include "radix.cuh"

namespace dem {

inline int grid_for(long long n, int bs) { return (int)((n + bs - 1) / bs); }

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
    Pp.bidx = c->pbidx[k];
    for (int q = 0; q < 3; ++q) Pp.dsp[q] = c->pdsp[k][q];
  };
  fill(V.A, a);
  fill(V.B, b);
  V.H.cnt = c->hcnt[0]; V.H.id = c->hid[0]; V.H.xi = (R *)c->hxi[0];
  V.Hn.cnt = c->hcnt[1]; V.Hn.id = c->hid[1]; V.Hn.xi = (R *)c->hxi[1];
  V.keys = c->skey[b];
  V.vals = c->sval[b];
  V.cstart = c->cstart; V.cend = c->cend;
  V.xl = c->xl;
  V.plist = c->plist;
  V.pcode = c->pcode;
  V.pcnt = c->pcnt;
  V.nl = c->nl;
  V.nlc = c->nlc;
  V.cur = c->curpos;
  V.rebuild = c->rebuild;
  V.corner = c->corner;
  V.cornerp = c->cornerp;
  V.kprev = c->skey[a];
  V.mass = (R *)c->mass;
  for (int q = 0; q < 3; ++q) { V.F[q] = (R *)c->F[q]; V.Tq[q] = (R *)c->Tq[q]; }
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
  V.list_acc = (unsigned long long *)(c->step_ctr + 3);
  return V;
}

// binning: keys of the (drifted) positions, radix sort, gather into the sorted order
template <class P>
int enqueue_binning(dem_ctx *c, int drift) {
  cudaStream_t st = c->st;
  StepView<P> V = make_view<P>(c, true);
  V.keys = c->keys;
  V.vals = c->vals;
  V.moved = resort_counts(c->rsw, c->rs_pow2, c->n);
  if (drift) cudaMemsetAsync(V.moved, 0, sizeof(int) * (size_t)((c->n + 1023) / 1024 + 1), st);
  int ps = prof_begin(c, "k_key");
  k_key<P><<<grid_for(c->n, c->bs_key), c->bs_key, 0, st>>>(V, drift);
  prof_end(c, ps);
  ++c->launches;
  const int nxt = 1 - c->cur;
  if (drift) {
    // few keys change per step: re-sort incrementally from the previous sorted order
    ps = prof_begin(c, "resort");
    int e = resort_pairs(c->skey[c->cur], c->keys, c->skey[nxt], c->sval[nxt], c->rsw, c->rs_pow2, c->n, st,
                         &c->launches);
    prof_end(c, ps);
    if (e) return e;
  } else {
    // first binning: full LSD radix sort of (key, index)
    unsigned *kr = nullptr, *vr = nullptr;
    ps = prof_begin(c, "radix_sort");
    int e = radix_sort_pairs(c->keys, c->vals, c->keys2, c->vals2, c->rhist, c->n, c->key_bits, st,
                             &kr, &vr, &c->launches);
    prof_end(c, ps);
    if (e) return e;
    c->kres = kr;
    c->vres = vr;
    cudaMemcpyAsync(c->skey[nxt], kr, sizeof(unsigned) * c->n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(c->sval[nxt], vr, sizeof(unsigned) * c->n, cudaMemcpyDeviceToDevice, st);
  }
  V.keys = c->skey[nxt];
  V.vals = c->sval[nxt];
  cudaMemsetAsync(c->cstart, 0, sizeof(unsigned) * c->ncells, st);
  cudaMemsetAsync(c->cend, 0, sizeof(unsigned) * c->ncells, st);
  ps = prof_begin(c, "k_gather");
  k_gather<P><<<grid_for(c->n, c->bs_gather), c->bs_gather, 0, st>>>(V, drift);
  prof_end(c, ps);
  ++c->launches;
  return (int)cudaPeekAtLastError();
}

template <class P>
int enqueue_steps(dem_ctx *c, int nsteps) {
  cudaStream_t st = c->st;
  for (int s = 0; s < nsteps; ++s) {
    int e = enqueue_binning<P>(c, 1);
    if (e) return e;
    StepView<P> V = make_view<P>(c, true);
    int ps;
    if (c->contact_mode == 1) {
      ps = prof_begin(c, "k_contacts_cell");
      k_contacts_cell<P><<<grid_for(c->n, CW_WARPS * 32), CW_WARPS * 32, 0, st>>>(V);
      prof_end(c, ps);
    } else {
      ps = prof_begin(c, "k_pair_list");
      k_pair_list<P><<<grid_for(c->n, c->bs_search), c->bs_search, 0, st>>>(V);
      prof_end(c, ps);
      ps = prof_begin(c, "k_pair_search");
      k_pair_search<P><<<grid_for(c->n, c->bs_search), c->bs_search, 0, st>>>(V);
      prof_end(c, ps);
      ps = prof_begin(c, "k_pair_forces");
      k_pair_forces<P><<<grid_for(c->n, c->bs_contacts), c->bs_contacts, 0, st>>>(V);
      prof_end(c, ps);
      c->launches += 2;
    }
    ps = prof_begin(c, "k_gas_particle");
    k_gas_particle<P><<<grid_for(c->n, c->bs_gp), c->bs_gp, 0, st>>>(V);
    prof_end(c, ps);
    ps = prof_begin(c, "k_cells");
    k_cells<P><<<grid_for(c->ncells, c->bs_cells), c->bs_cells, 0, st>>>(V, 0);
    prof_end(c, ps);
    k_step_counter<<<1, 1, 0, st>>>(c->step_ctr, c->rebuild, c->contact_mode == 0);
    c->launches += 4;
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
  k_fov_chunks<P><<<c->nbeds * FOV_CHUNKS, 256, 0, c->st>>>(V, per_parcel_dev, c->fv);
  k_fov_beds<<<(c->nbeds + 63) / 64, 64, 0, c->st>>>(c->fv, c->nbeds, c->fvbed);
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

template <class P>
int enqueue_props(dem_ctx *c) {
  StepView<P> V = make_view<P>(c, false);
  V.gas = c->gas[c->gcur];
  V.gas_new = c->gas[1 - c->gcur];
  k_cells<P><<<grid_for(c->ncells, 256), 256, 0, c->st>>>(V, 2);
  c->gcur = 1 - c->gcur;
  return (int)cudaPeekAtLastError();
}

// largest block each tunable kernel can launch with (registers per thread decide it)
template <class P>
int kernel_limits(int *lim) {
  const void *fn[6] = {(const void *)k_key<P>, (const void *)k_gather<P>, (const void *)k_pair_search<P>,
                       (const void *)k_pair_forces<P>, (const void *)k_gas_particle<P>, (const void *)k_cells<P>};
  for (int k = 0; k < 6; ++k) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, fn[k]) != cudaSuccess) return -1;
    lim[k] = a.maxThreadsPerBlock;
  }
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
  template int enqueue_props<P>(dem_ctx *);

}  // namespace dem
