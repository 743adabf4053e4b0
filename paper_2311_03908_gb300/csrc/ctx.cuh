// ctx.cuh -- the library's context: one device arena holding every array of the particle
// path, plus the host-side bookkeeping (which ping-pong buffer is current, cached graphs).
#pragma once
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "gas.cuh"

struct dem_ctx {
  int n = 0, cap = 0, nbeds = 0, prec = DEM_PREC_FP64;
  long long ncells = 0;
  int key_bits = 1;
  cudaStream_t st = nullptr;
  std::vector<dem::DevBed> hbeds;
  std::vector<dem::BedP<double>> hbp_d;
  std::vector<dem::BedP<float>> hbp_f;
  std::vector<dem_bed_config> cfg;
  dem::DevBed *dbeds = nullptr;
  dem::BedP<double> *dbp_d = nullptr;
  dem::BedP<float> *dbp_f = nullptr;
  // one device arena
  char *arena = nullptr;
  size_t arena_bytes = 0;
  size_t rsize = 8;                 // sizeof(R)
  // parcel state: buffer 0 the state (in place), buffer 1 the scratch of a re-store
  double *px[2][3] = {};
  void *pv[2][3] = {}, *pw[2][3] = {}, *pa[2][3] = {}, *pal[2][3] = {}, *pT[2] = {}, *pd[2] = {};
  double *pm[2][4] = {};
  int *pmeta[2] = {}, *porig[2] = {};
  float *pdsp[2][3] = {};
  // contact history, double-buffered by step parity: before the step and after it (the
  // latter is also the re-store's scratch)
  unsigned char *hcnt[2] = {};
  int *hid[2] = {};
  void *hxi[2] = {};
  // binning
  unsigned *keys = nullptr, *vals = nullptr, *keys2 = nullptr, *vals2 = nullptr, *rhist = nullptr;
  unsigned *skey[2] = {}, *sval[2] = {};       // sorted keys / permutation, by step parity
  unsigned *inv = nullptr;                     // sorted position of each storage position
  unsigned *rsw = nullptr;                     // scratch of the incremental re-sort
  int rs_pow2 = 1;
  unsigned *cstart = nullptr, *cend = nullptr;
  float4 *xl = nullptr;             // cell-local position and radius, sorted order
  int *plist = nullptr;             // pair-search hit lists [KLIST][cap]
  unsigned char *pcode = nullptr, *pcnt = nullptr;
  int *nl = nullptr, *rebuild = nullptr;   // neighbour lists (storage positions), build flag
  unsigned char *nlc = nullptr;
  double skin_frac = 0.1;         // neighbour-list skin as a fraction of the largest diameter
  int restore_every = 1;          // re-store the state in cell order at every k-th list build
  double *corner = nullptr;         // cell-corner coordinates: per bed x0+i dx, y0+j dy, z0+k dz
  std::vector<double> hcorner;
  float2 *cornerp = nullptr;        // cell corners relative to the bed corner as FP32 pairs
  std::vector<float2> hcornerp;
  void *F[3] = {}, *Tq[3] = {}, *src = nullptr;
  // gas: two state buffers (gcur = current), properties, marks
  double *gas[2] = {};
  void *gp = nullptr;
  unsigned char *mark = nullptr;
  int *cell_bed = nullptr;
  double *fv = nullptr, *fvbed = nullptr;
  int *err = nullptr;
  long long *step_ctr = nullptr;
  int cur = 0, gcur = 0;
  // optional buffers (cudaMalloc on first use, outside the arena)
  double *diag = nullptr, *dep = nullptr, *scratch_out = nullptr;
  size_t scratch_bytes = 0;
  bool diag_on = false;
  // host-side status
  int *h_err = nullptr;             // pinned
  cudaEvent_t ev = nullptr;
  bool pending = false;
  int sticky = DEM_OK;
  long long launches = 0;
  int bs_contacts = 128, bs_gp = 128, bs_restore = 256, bs_cells = 256, bs_key = 256;
  int use_lists = 1;               // 1: Verlet neighbour lists, 0: cell-list search every step
  int bs_search = 256;
  int nsm = 152;                   // SMs of the device (one wave of a grid-stride launch)
  unsigned char *wnear = nullptr;   // per cell: a wall primitive may be within a parcel's reach
  int *ovf = nullptr, *novf = nullptr;   // parcels whose neighbour list overflowed, and their count
  uint2 *work = nullptr;           // contact work list (parcel, list-hit mask)
  int *nwork = nullptr;            // its length
  char *qrad = nullptr;            // radiation heat of each parcel this step (form's type)
  char *tsrt = nullptr;            // FP64 temperatures in sorted order for the radiation kernel
  float4 *xr = nullptr;            // local coordinates and temperature in sorted order (radiation)
  bool any_rad = false;            // some bed has DEM_RADIATION: the radiation kernel runs
  bool any_cond = false;           // some bed has DEM_CONDUCTION
  bool gas_solver = false;         // every bed has DEM_GAS_SOLVER: the gas kernels replace k_cells
  dem::GasView gsv = {};           // the solver's arrays (in the arena)
  int gs_grid = 1;                 // blocks of the cooperative pressure solve (all co-resident)
  // multigrid levels of the pressure preconditioner: per level the arrays (level 0: the gas
  // grid's coefficient rows and CG vectors), per level and bed the dims and first cell
  std::vector<dem::GsLevel> hlev;
  std::vector<dem::GsLevelBed> hlb;
  std::vector<int *> dlbed;        // bed of each cell, levels >= 1 (arena)
  std::vector<int *> dlpar;        // the coarse cell holding each cell, levels below the coarsest (arena)
  dem::GsLevel *dlev = nullptr;
  dem::GsLevelBed *dlb = nullptr;
  char *qc = nullptr;              // contact conduction heat of each parcel in contact (form's type)
  std::map<std::tuple<int, int, int>, std::pair<cudaGraph_t, cudaGraphExec_t>> graphs;
  std::map<std::tuple<int, int, int>, long long> graph_launches;
  cudaStream_t gst = nullptr;     // private stream used to capture graphs
  // the coupling input (dem_set_gas) runs on its own stream: the host arrays cross by a
  // copy engine into gas_stage while the next step's binning and contact kernels run (those
  // read no gas state); the step's first kernel that reads the gas waits for ev_gas
  cudaStream_t sst = nullptr;
  cudaEvent_t ev_main = nullptr, ev_gas = nullptr;
  bool gas_pending = false;
  // per-kernel event timing
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> prof_marks;   // (kernel id, index of its start event)
  std::vector<std::string> prof_names;
  std::vector<double> prof_ms;
  std::vector<long long> prof_n;
  double *gas_stage = nullptr;
  // adjoint buffers
  double *adj = nullptr;
  size_t adj_bytes = 0;
};

namespace dem {

template <class P> int kernel_limits(int *lim);
template <class P> StepView<P> make_view(dem_ctx *c, bool for_step);
template <class P> int enqueue_steps(dem_ctx *c, int nsteps);
template <class P> int enqueue_init(dem_ctx *c);
template <class P> int enqueue_fov(dem_ctx *c, double *per_parcel_dev);
template <class P> int enqueue_scatter_state(dem_ctx *c, double *out_dev);
template <class P> int enqueue_scatter_diag(dem_ctx *c, double *out_dev);
template <class P> int enqueue_scatter_hist(dem_ctx *c, int *cnt, int *partner, double *xi);
template <class P> int enqueue_sources(dem_ctx *c);
template <class P> int enqueue_sources_occupied(dem_ctx *c, int *cnt, long long *cells, double *out);
template <class P> int enqueue_gas_set(dem_ctx *c, const double *Y, const double *T, cudaStream_t st);
template <class P> int enqueue_gas_solver_init(dem_ctx *c);
template <class P> int enqueue_flow(dem_ctx *c, double *out_dev);
template <class P> int gas_cg_occupancy(int *blocks_per_sm);
template <class P> int run_adjoint(dem_ctx *c, int nsteps, int ckpt, double *J, double *grad, int nobs = 0,
                                   const int *obs_steps = nullptr, const double *weights = nullptr,
                                   double *J_obs = nullptr);

// event pair around one kernel when profiling is on (returns the start-event slot or -1)
int prof_begin(dem_ctx *c, const char *name);
void prof_end(dem_ctx *c, int slot);

// call FN<P>(args...) with the context's precision policy P
#define DEM_DISPATCH(c, FN, ...)                                                         \
  ((c)->prec == DEM_PREC_FP64 ? FN<::dem::PrecF64>(__VA_ARGS__)                         \
                              : (c)->prec == DEM_PREC_SPLIT ? FN<::dem::PrecSplit>(__VA_ARGS__) \
                                                            : FN<::dem::PrecKahan>(__VA_ARGS__))

}  // namespace dem
