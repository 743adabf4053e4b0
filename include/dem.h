/*
 * dem.h -- C ABI of the GB300 (sm_103a) particle-side step of the coarse-grained
 * CFD-DEM-IBM method for hydrogen reduction of iron ore of Lan et al. (arXiv 2311.03908).
 *
 * One call of dem_step advances every coarse-grained parcel of every bed by one DEM time
 * step, entirely on the GPU:
 *   1. half kick and drift (velocity Verlet of eq (3-3) and eq (3-6));
 *   2. binning of the parcels on their cell key: an LSD radix sort at the first binning,
 *      then each step an incremental re-sort of the keys and the permutation (the same
 *      permutation bit for bit);
 *   3. occupied-cell ranges; the parcel state re-stored in cell order at every k-th
 *      neighbour-list build (it stays in place in between);
 *   4. soft-sphere contacts with the neighbouring parcels (linear spring-dashpot normal
 *      force, tangential spring with a contact-history table and a Coulomb cap) and with
 *      the analytic reactor wall (cylinder, flat bottom or cone, perforated plate, lid);
 *   5. gas-particle terms of the containing gas cell: Gidaspow-Ganser drag (eqs (3-5),
 *      (3-5-2)..(3-5-5)), Gunn convection (eqs (3-10)..(3-13)), the multi-path unreacted
 *      shrinking core model (Sec. 2: eqs (2-1)..(2-36)) with the coarse-graining k^3
 *      scaling (eqs (3-41), (3-49), (3-50), (3-52));
 *   6. second half kick, particle temperature (eqs (3-8), (3-9)) and, at coupling steps
 *      (every n = coupling_interval steps, Sec. 4), the layer masses (eq (3-4));
 *   7. at coupling steps, deposition of the cell sources by a segmented reduction over the
 *      sorted parcels (eqs (3-25), (3-27a), (3-38), (3-39), (4-4), (4-5), (4-10), (4-11));
 *   8. at coupling steps, a simple explicit update of the prescribed gas field (volume
 *      fraction, species, temperature; semi-implicit in the convective coefficient as in
 *      eq (4-6)), which is otherwise left unchanged.
 *
 * Conventions (every entry point):
 *   - returns int status: DEM_OK (0) or a negative DEM_E* code; never aborts or exits;
 *   - host pointers are read during the call only (the library copies what it keeps);
 *     device pointers (when a struct says on_device = 1) must stay valid for the call;
 *   - all work is enqueued on the stream given to dem_init; a fault detected on the device
 *     (contact-table overflow, non-finite state, a parcel outside its grid) is sticky: it
 *     is returned by the next call that observes it (dem_sync always observes it);
 *   - units are SI; arrays of parcels are indexed in input order (the "parcel index").
 */
#ifndef DEM_H
#define DEM_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum {
  DEM_OK = 0,
  DEM_EINVAL = -1,      /* bad argument (sizes, ranges, geometry, stability) */
  DEM_ENOMEM = -2,      /* device or pinned allocation failed */
  DEM_ECUDA = -3,       /* a CUDA runtime call failed */
  DEM_ECAPACITY = -4,   /* a parcel had more contacts than DEM_MAX_CONTACTS */
  DEM_ENONFINITE = -5,  /* a parcel state became NaN or Inf */
  DEM_ETIMEOUT = -6,    /* a bounded device wait gave up */
  DEM_ESTATE = -7,      /* call not valid in the context's state */
  DEM_EDOMAIN = -8      /* a parcel centre left its bed's gas grid (clamped) */
};

enum { DEM_PREC_FP64 = 0, DEM_PREC_SPLIT = 1, DEM_PREC_SPLIT_KAHAN = 2 };

/* physics switches (bit mask in dem_bed_config.flags); 0 = the full method without
 * radiation and contact conduction. DEM_CONDUCTION switches ON the contact heat conduction
 * of eqs (3-14), (3-15) (parcel-parcel and parcel-fluid-parcel) and (3-15-1), (3-15-2)
 * (parcel-wall and parcel-fluid-wall), scaled to the coarse-grained parcels by eqs (3-46),
 * (3-48), (3-48-1), (3-48-2), over the contacts of eq (3-3): R_c is the radius of the
 * circle in which the overlapping spheres (or a sphere and the wall's tangent plane) meet;
 * lambda_e = lambda_a lambda_b / (lambda_a + lambda_b) with the per-ore lambda_p and the
 * wall's lambda_wall; the fluid lens spans the smaller sphere's disk down to a gap of
 * 1.013 / p0 cm (the Sec. 2.3 mean free path of H2), with the mean lambda_g of the two
 * parcels' cells (a wall: the parcel's); walls are at T_in; f(e) of eq (3-43) is
 * exp(-zeta arccos(zeta) / sqrt(1 - zeta^2)) with zeta of eq (3-44), and e_CGP of
 * eq (3-45) is clamped at 0. The heat enters each parcel's balance (eq (3-8)), not the gas.
 * Radiation: DEM_RADIATION switches ON the particle radiation of eqs (3-16), (3-17) and
 * (3-51): Q_rad = k^3 sigma eta_p pi d_p^2 (T_se^4 - T_p^4), T_se = eps_g T_g + (1 - eps_g)
 * times the mean temperature of the parcels whose centres lie within 1.5 k d_p of the
 * parcel's centre (the parcel itself included), eps_g and T_g those of the parcel's gas
 * cell, all temperatures from before the step's update; Q_rad adds to the parcel's heat
 * balance (eq 3-8) and, as the paper neglects gas radiation, not to the gas.
 * Gas solver: DEM_GAS_SOLVER replaces the prescribed gas field (plug flow U_in / eps_g along
 * z, no cross flow, the explicit upwind update of Y and T along z) with the gas phase solved
 * on the bed's grid every coupling step, in FP64 in every precision form: continuity
 * (eq (3-24)) with the mass source of eq (3-25), momentum with the drag of eq (4-2)
 * (K_gp u_g implicit, K_gp u_p explicit from the parcels' sums), energy with H0 implicit
 * (eq (4-6)) and the reducing gas with C0, C1 (eqs (4-8)..(4-11)), the pseudo-turbulent
 * stress and heat flux of eqs (3-28)..(3-37). Readings (the paper solves this with a
 * finite-volume code and gives no discretisation): a staggered grid with the velocity
 * components on the cell faces, explicit Euler in dt_CFD = n dt_DEM, first-order upwind
 * convection; species and energy first, with the mass fluxes of the last projection, which
 * gives the new density rho' (eq (3-53)); then the momentum predictor and an incremental
 * pressure projection in which continuity takes d(eps rho)/dt = (eps rho' - eps_old rho)/dt
 * and rho' in the mass fluxes (so the oxygen the reactions add raises the gas density
 * instead of leaving as extra volume flow), solved by Jacobi-preconditioned conjugate
 * gradients to a relative residual of 1e-12; immersed-boundary cells and the box sides are
 * no-slip walls held at T_in (Table 3 lists the wall and inlet temperatures equal); a
 * z-face below a fluid cell whose lower neighbour is not fluid carries the inlet gas
 * (eps u = U_in at the inlet gas's density, Y_in, T_in); z-faces on top of the box are an outlet at p0 with zero
 * gradient; the pseudo-turbulent stress enters by its normal components and the heat flux
 * by the diagonal of alpha_PT, both rotated to the slip direction of the cell's drag-
 * weighted parcel velocity, with Re_m capped at 100 and eps_p at 0.5; H2O follows the H2
 * consumed by stoichiometry (eq (2-25)) and N2 by closure; molecular diffusion takes
 * D_H2,m of eq (2-27) for every species. Parcels see the cell-centre velocity of the solved
 * faces; their pressure force keeps the prescribed dpdz. The flow starts as plug flow at
 * U_in through every fluid column. Either every bed of a context has DEM_GAS_SOLVER, with
 * one coupling interval for all, or none; it excludes DEM_NO_GAS_UPDATE, and a solving
 * context takes no dem_set_gas input and no adjoint (DEM_EINVAL). */
enum {
  DEM_NO_GRAVITY = 1, DEM_NO_DRAG = 2, DEM_NO_HEAT = 4, DEM_NO_KINETICS = 8,
  DEM_NO_GAS_UPDATE = 16, DEM_NO_FILM = 32, DEM_NO_LAYER = 64, DEM_NO_RXN_HEAT = 128,
  DEM_NO_CONTACTS = 256, DEM_RADIATION = 512, DEM_CONDUCTION = 1024, DEM_GAS_SOLVER = 2048
};

enum { DEM_WALL_FLAT = 0, DEM_WALL_CONE = 1 };
enum { DEM_ORE_HEMATITE = 0, DEM_ORE_MAGNETITE = 1 };

#define DEM_MAX_CONTACTS 24   /* contact-history slots per parcel (walls included) */
#define DEM_MAX_BEDS 1024

/*
 * One bed (Table 3 of the paper lists the physical parameters; the benchmark beds fix the
 * rest). Geometry: a cylinder of diameter bed_D and height bed_H standing on z = 0, the
 * gas grid nx*ny*nz covering [-D/2, D/2]^2 x [0, H]. wall_kind DEM_WALL_CONE adds a cone
 * of half angle cone_half_angle (rad) whose rim meets the cylinder at z = cone_height,
 * and a zero-thickness distributor plate at z = plate_z with round holes of diameter
 * hole_d on a square lattice of pitch hole_pitch centred on the axis.
 * Gas cells that lie wholly outside the fluid region are marked solid (immersed
 * boundary): they take no sources and keep their state.
 */
typedef struct {
  double bed_D, bed_H;
  int32_t wall_kind;
  double cone_half_angle, cone_height, plate_z, hole_d, hole_pitch;
  int32_t nx, ny, nz;
  double dt;              /* DEM time step, s */
  double kn;              /* normal spring stiffness, N/m */
  double kt_over_kn;      /* tangential / normal stiffness; tangential damping scales by its sqrt */
  double restitution;     /* restitution coefficient of a parcel-parcel or parcel-wall contact */
  double mu_s;            /* sliding friction coefficient (Coulomb cap) */
  double mu_r;            /* rolling friction length, m (0 = off) */
  double cg_ratio;        /* coarse-graining ratio k = d_CGP / d_p (Sec. 3.3) */
  int32_t coupling_interval;  /* n = dt_CFD / dt_DEM (Sec. 4): masses, sources, gas every n steps */
  double U_in, T_in, p0;  /* superficial inlet velocity (m/s), inlet temperature (K), pressure (Pa) */
  double Y_in[3];         /* inlet mass fractions of H2, H2O, N2 */
  double k0[3], Ea[3];    /* pre-exponential factor (m/s) and activation energy (J/mol) of R1..R3 */
  double tortuosity;      /* tau of eq (2-30) (not printed in the paper) */
  double sphericity[2];   /* psi of eqs (3-5-2)..(3-5-5), per ore type */
  double xi0[2];          /* initial porosity per ore type (Table 3) */
  double pore_d_cm[2];    /* pore diameter per ore type, cm (Table 3) */
  double rho_true[4];     /* true densities of Fe2O3, Fe3O4, FeO, Fe (Table 3) */
  double dpdz;            /* prescribed gas pressure gradient along z, Pa/m (force -V dp/dz) */
  double eps_min;         /* lower clamp of the gas volume fraction */
  uint32_t flags;         /* DEM_NO_* switches, DEM_RADIATION, DEM_CONDUCTION, DEM_GAS_SOLVER */
  double emissivity;      /* particle emissivity eta_p of eq (3-16), in [0, 1] (Table 3: 0.85);
                             read only with DEM_RADIATION */
  double lambda_p[2];     /* particle thermal conductivity per ore type, W/m/K (> 0); read only
                             with DEM_CONDUCTION (not printed in the paper) */
  double lambda_wall;     /* reactor wall thermal conductivity, W/m/K (> 0); DEM_CONDUCTION */
} dem_bed_config;

/*
 * Parcels (coarse-grained particles). x, y, z, vx, vy, vz, d_real, T and m0[4] are n doubles
 * each; ore_type and bed are n int32 (bed indexes the dem_bed_config array). d_real is the
 * real particle diameter d_p (the parcel diameter is cg_ratio * d_real); m0 are the parcel
 * masses of Fe2O3, Fe3O4, FeO and Fe (kg). id (nullable) is carried for the caller only.
 * on_device = 1: every pointer is a device pointer; 0: host pointers.
 */
typedef struct {
  int32_t n;
  int32_t on_device;
  const double *x, *y, *z, *vx, *vy, *vz, *d_real, *T;
  const double *m0[4];
  const int32_t *ore_type, *bed;
  const int64_t *id;
} dem_parcels;

/*
 * Initial gas field (nullable: uniform inlet state). Y is (total cells) x 3 mass fractions
 * (H2, H2O, N2) and T the temperatures, cells ordered bed by bed, then x fastest, then y,
 * then z.
 */
typedef struct {
  int32_t on_device;
  const double *Y, *T;
} dem_gas;

typedef struct dem_ctx dem_ctx;

/* Create a context: validates the inputs, allocates one device arena, copies the parcels
 * and bins them once. The validation follows the paper's statement of the problem: a
 * coarse-grained parcel of diameter k d_p (Sec. 3.3, eq (3-41)) must fit inside one gas
 * cell, since the particle-to-gas coupling of Sec. 3.2 (eqs (3-24), (3-25)) assigns each
 * parcel to the single cell that holds its centre; the soft-sphere contact of eq (3-3) is
 * integrated explicitly, so the DEM step must resolve the stiffest contact (omega_0 dt < 2
 * with omega_0 = sqrt(k_n / m*)); and masses are updated every n = dt_CFD / dt_DEM steps
 * (Sec. 4), so n >= 1. cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * precision: DEM_PREC_FP64 (everything FP64), DEM_PREC_SPLIT (FP32 contact geometry,
 * forces, drag, heat, kinetics and velocities; FP64 positions and layer masses; cell-source
 * sums and the gas state in Kahan-compensated FP32) or DEM_PREC_SPLIT_KAHAN (as SPLIT but
 * positions and layer masses as Kahan-compensated FP32 pairs too: no FP64 arithmetic in
 * the step).
 * Errors: DEM_EINVAL for n <= 0, n_beds outside [1, DEM_MAX_BEDS], a bad grid, a parcel
 * outside its bed, coupling_interval < 1, k*d_p larger than a gas cell, or a time step at
 * or above the stability limit omega_0 dt >= 2 of the stiffest pair; DEM_ENOMEM/DEM_ECUDA. */
int dem_init(const dem_bed_config *beds, int32_t n_beds, const dem_parcels *p,
             const dem_gas *g, int32_t precision, void *cuda_stream, dem_ctx **out);

/* Advance n_steps steps (asynchronous on the context stream). */
int dem_step(dem_ctx *c, int32_t n_steps);

/* Advance n_steps steps by replaying a CUDA graph of those steps (captured on first use
 * for this n_steps and kept; one graph launch per call). */
int dem_step_graph(dem_ctx *c, int32_t n_steps);

/* Wait for the context stream and return any sticky device error. */
int dem_sync(dem_ctx *c);

/* Overall reduction degree (eqs (2-15)..(2-19)): mean_per_bed (host, n_beds doubles) gets
 * the arithmetic mean of the parcels' f_ov in each bed; oxygen_per_bed (host, nullable)
 * the bed's removed-oxygen fraction; per_parcel (nullable, device, n doubles) each
 * parcel's f_ov in parcel-index order. Synchronous. */
int dem_reduction_degree(dem_ctx *c, double *mean_per_bed, double *oxygen_per_bed,
                         double *per_parcel);

/* Adjoint of the frozen-position drag-heat-reaction sub-step: from the current state,
 * J = mean over all parcels of f_ov after n_steps sub-steps minus f_ov now, with positions,
 * cells and the gas field held fixed and (v, T_p, m_z) integrated by explicit Euler with
 * the bed time step. grad (host, 6 doubles) gets dJ/dk0[0..2] and dJ/dEa[0..2], the
 * parameters applied to every bed. The forward pass stores a checkpoint every
 * ckpt_every sub-steps; the reverse pass recomputes each segment and runs the hand-written
 * adjoint kernel back through it. The context's state is not changed. Synchronous.
 * grad may be NULL: then only the forward sweep runs and only J is written. The sub-step
 * is evaluated in FP64 whatever the context's precision. Errors: DEM_EINVAL for n_steps < 0
 * or ckpt_every < 1, and when a bed has DEM_RADIATION or DEM_CONDUCTION (they couple the
 * parcels' temperatures, and the differentiated map is per parcel); DEM_ENOMEM when the checkpoint and segment buffers (8 doubles per
 * parcel per checkpoint and per sub-step of a segment) cannot be allocated. */
int dem_adjoint(dem_ctx *c, int32_t n_steps, int32_t ckpt_every, double *J, double *grad);

/* Observed reduction-degree curves and the gradient of a weighted sum of them, for fitting
 * the kinetic parameters to measured curves as Sec. 5.1.1 and Sec. 5.2.1 do (there by
 * hand): the frozen-position sub-step of dem_adjoint is run for n_steps; after obs_steps[k]
 * sub-steps (1 <= obs_steps[0] < ... < obs_steps[n_obs-1] <= n_steps, n_obs <= DEM_MAX_OBS)
 * J_obs[k * n_beds + b] (host) gets the mean over bed b's parcels of f_ov - f_ov(now)
 * (eqs (2-15)..(2-19)). With grad (host, 6 doubles; needs weights, host n_obs x n_beds):
 * the derivative of sum_k sum_b weights[k * n_beds + b] J_obs[k * n_beds + b] w.r.t. k0[0..2]
 * and Ea[0..2] (eq (2-13)), by the same checkpointed reverse sweep (a least-squares fit's
 * gradient is one call with weights 2 (J_obs - target), after a call without grad for J_obs).
 * State unchanged; synchronous. Errors as dem_adjoint, and DEM_EINVAL for unordered or
 * out-of-range observation steps, non-finite weights, or grad without weights. */
#define DEM_MAX_OBS 4096
int dem_adjoint_obs(dem_ctx *c, int32_t n_steps, int32_t ckpt_every, int32_t n_obs, const int32_t *obs_steps,
                    const double *weights, double *J_obs, double *grad);

/* Replace the kinetic parameters of every bed: the pre-exponential factors k0 (m/s) and
 * activation energies Ea (J/mol) of the interface rate constants k_r = k0 exp(-Ea / (R T_p))
 * of eq (2-13) for R1 (Fe2O3 -> Fe3O4), R2 (Fe3O4 -> FeO), R3 (FeO -> Fe) (Table 2 lists
 * one set; Sec. 5.1.1 and Sec. 5.2.1 fit others). Host arrays of 3 doubles, k0 >= 0 and
 * Ea >= 0 (DEM_EINVAL otherwise, NaN included). Waits for the context stream, then takes
 * effect from the next step (captured step graphs read the parameters from device memory). */
int dem_set_kinetics(dem_ctx *c, const double k0[3], const double Ea[3]);

/* Per-parcel state in parcel-index order, DEM_NSTATE rows of n doubles (host): the
 * position and velocity of the translational equation (3-3), the angular velocity of the
 * rotational equation (3-6), the temperature of the energy equation (3-8), the layer masses
 * m_z of eqs (3-1), (3-2), (3-4), and the accelerations of eqs (3-3) and (3-6) at the end of
 * the last step: x y z vx vy vz wx wy wz T m_Fe2O3 m_Fe3O4 m_FeO m_Fe ax ay az alx aly alz.
 * Synchronous. */
enum { DEM_NSTATE = 20 };
int dem_get_state(dem_ctx *c, double *out_host);

/* Per-gas-cell state, DEM_NGAS doubles per cell (host): eps Y_H2 Y_H2O Y_N2 T solid_mark. */
enum { DEM_NGAS = 6 };
int64_t dem_num_cells(dem_ctx *c);
int dem_get_gas(dem_ctx *c, double *out_host);

/* Cell sources of the last step taken (the coupling output of Sec. 4 when that step is a
 * coupling step), DEM_NDEP doubles per cell (host): V_s, S_H2,
 * S_H2O (kg/s into the gas), K, K v_x, K v_y, K v_z (eq (3-27a)), hA, hA T_p (eqs (4-4),
 * (4-5)), Q_rm, Q_r (eqs (3-38), (3-49), (3-50)), E Q, E S (eqs (4-10), (4-11)), count.
 * Recomputed from the per-parcel sources kept from the last step. Synchronous. */
enum { DEM_NDEP = 14 };
int dem_get_sources(dem_ctx *c, double *out_host);

/* The same sources for only the fluid cells that hold parcels (the others' are all zero), in
 * increasing cell order: the coupling output of Sec. 4 without the empty cells, for a gas
 * solver that takes sparse sources (no counterpart in the paper: it only changes how much
 * crosses the link). *n_occupied (host) receives the number of such cells; cells_host (host,
 * cap int64) their global cell indices and out_host (host, cap x DEM_NDEP doubles) their rows,
 * identical to the rows dem_get_sources returns for them. If n_occupied exceeds cap, nothing
 * else is written and DEM_EINVAL is returned (the count is, so the caller can size its
 * buffers; at most min(parcels, cells)). Synchronous. */
int dem_get_sources_occupied(dem_ctx *c, int64_t cap, int64_t *n_occupied, int64_t *cells_host, double *out_host);

/* Gas flow of every cell, DEM_NFLOW doubles per cell (host): the cell-centre gas velocity
 * u_x u_y u_z (m/s; the mean of the cell's two faces on each axis where the gas is solved,
 * (0, 0, U_in / eps_g) where it is prescribed) and the pressure relative to p0 (Pa; 0 where
 * prescribed), and the number of conjugate-gradient iterations of the last pressure solve
 * in iters (nullable; 0 without DEM_GAS_SOLVER). Synchronous. */
enum { DEM_NFLOW = 4 };
int dem_get_flow(dem_ctx *c, double *out_host, int32_t *iters);

/* Contact-history table in parcel-index order (host): count[n]; partner[n*DEM_MAX_CONTACTS]
 * (parcel index of the partner, or -1-p for wall primitive p: 0 side, 1 bottom or cone,
 * 2 plate, 3 lid; INT32_MIN in unused slots); xi[n*DEM_MAX_CONTACTS*3] tangential
 * displacements. Slots are sorted by partner. Synchronous. */
int dem_get_contacts(dem_ctx *c, int32_t *count, int32_t *partner, double *xi);

/* Per-parcel diagnostics of the last step (enable with dem_set_diagnostics before stepping),
 * DEM_NDIAG rows of n doubles (host), parcel-index order:
 * Fc(3) Tc(3) Fd(3) K Qconv Qr Qrm xidot(3) mdot(4) F_film A(3) B(3) Sh Nu Re ncontact cell
 * T_se Q_rad Q_cond (T_se and Q_rad are 0 in beds without DEM_RADIATION, Q_cond in beds
 * without DEM_CONDUCTION) */
enum { DEM_NDIAG = 35 };
int dem_set_diagnostics(dem_ctx *c, int32_t on);
int dem_get_diag(dem_ctx *c, double *out_host);

/* Launch configuration of the step kernels (no counterpart in the paper: it only changes how
 * the same step is computed), DEM_NTUNE int32 values:
 *   [0] contact search: 1 = Verlet neighbour lists rebuilt from the cell list when a parcel
 *       has moved half the skin (default), 0 = the cell-list search every step;
 *   [1]..[6] block sizes of the key, re-store, pair-search, contact, gas-particle and
 *       gas-cell kernels (multiples of 32 in [32, 1024], and no larger than the kernel's
 *       launch bounds and register use allow: the gas-particle kernel stops at 256);
 *   [7] neighbour-list skin in thousandths of the bed's largest parcel diameter (1..1000);
 *   [8] re-store the parcel state in cell order at every k-th neighbour-list build (1..64;
 *       1 = every build): between re-stores the records stay where they are and the
 *       search reads them through the sort's permutation;
 *   [9] preconditioner of the gas solver's pressure equation (DEM_GAS_SOLVER): 0 = Jacobi,
 *       1 or 2 = an FP32 multigrid V-cycle (under the flexible form of the FP64 conjugate
 *       gradients) with that many damped-Jacobi sweeps before and after each coarse
 *       correction (default 2; Galerkin coarse levels of 2 x 2 x 2 aggregates, down to one
 *       cell per bed); the solve converges to the same FP64 tolerance either way;
 *   [10] weight of the multigrid coarse correction in percent (50..200, default 150: the
 *        piecewise-constant aggregates' correction falls short, and over-correcting it
 *        halves the iterations).
 * dem_set_tuning validates every value (DEM_EINVAL, nothing changed), drops captured graphs
 * and makes the next step rebuild the neighbour lists; results can then differ from an
 * untuned run in the last bits (order of the force sums), never in the pair sets. */
enum { DEM_NTUNE = 11 };
int dem_get_tuning(dem_ctx *c, int32_t *out);
int dem_set_tuning(dem_ctx *c, const int32_t *in);

/* Pick the tuning above by timing candidates, each over n_steps steps started from the same
 * saved state (block sizes, skin, lists or not). The state is restored afterwards and the
 * chosen tuning applied (as dem_set_tuning). Needs a temporary device copy of the context's
 * arena (DEM_ENOMEM if it cannot be allocated); clears the dem_profile record. Synchronous. */
int dem_autotune(dem_ctx *c, int32_t n_steps);

/* Counters since dem_init (3 values, host): steps taken, neighbour-list builds, and the total
 * number of list entries at the last build (their mean length is that over n). Synchronous. */
int dem_get_counters(dem_ctx *c, int64_t *out);

/* Number of kernels launched by the last dem_step/dem_step_graph call (for accounting). */
int64_t dem_last_launch_count(dem_ctx *c);

/* Replace the gas field (the coupling input of Sec. 4, Fig. 5: cell fields from the gas
 * solver). g->Y is (total cells) x 3 mass fractions, g->T the temperatures (host or device
 * by g->on_device); the gas volume fraction is kept; the cells' derived properties are
 * recomputed. Asynchronous: the input is taken on a stream of the context's own, after the
 * work already enqueued on the context stream; host arrays are copied by a copy engine
 * (page-locked host memory at the link's rate, without occupying the GPU's SMs), so the
 * transfer runs beside the next step's binning and contact kernels, which read no gas
 * state; the step's first kernel that does read it waits for the input. Host buffers must
 * stay unchanged until the next call that synchronises with the context (as for any
 * asynchronous copy); device buffers likewise. */
int dem_set_gas(dem_ctx *c, const dem_gas *g);

/* Per-kernel timing: while on, every kernel that dem_step launches is bracketed by CUDA
 * events on the context stream; dem_kernel_times (synchronous) returns, per kernel name,
 * the number of launches and their total device time since profiling was switched on.
 * names receives up to max_kernels NUL-terminated names of 32 bytes each. Returns the
 * number of kernel names (>= 0) or a negative status. */
int dem_profile(dem_ctx *c, int32_t on);
int dem_kernel_times(dem_ctx *c, int32_t max_kernels, char *names, int64_t *launches, double *ms_total);

/* Reduction degree of parcel arrays the caller owns, without allocating anything.
 * The paper has no counterpart: this serves callers that cannot call cudaMalloc -- code
 * whose device memory is all handed out by another framework's allocator, or a
 * latency-critical loop that cannot take cudaMalloc's implicit device-wide
 * synchronisation -- and that keep their parcels in their own device arrays.
 * Inputs (device, n each): the parcel masses of Fe2O3, Fe3O4, FeO, Fe (kg) and the ore type
 * (0 hematite, 1 magnetite). Output (device, 2 doubles): out[0] the arithmetic mean of the
 * parcels' f_ov (eqs (2-15)..(2-19), as dem_reduction_degree), out[1] the removed-oxygen
 * fraction. Asynchronous on cuda_stream (NULL = legacy default stream).
 * Scratch: a file-scope __device__ array of 4096 x 3 doubles (96 KiB) that every GPU loading
 * the library holds until the process exits; n is limited to DEM_NOALLOC_MAX_PARCELS and a
 * larger n returns DEM_EINVAL before any work is enqueued. No cudaMalloc, cudaFree or
 * allocating library routine is called. Every call made outside a stream capture (with its
 * device current) looks up the array's device address with cudaGetSymbolAddress; a call
 * made while cuda_stream is capturing uses the address found by the last uncaptured call on
 * that device, and returns DEM_ESTATE if there was none. So make one uncaptured call on a
 * device before capturing a call, and again after anything that tears the device's context
 * down and creates it anew (cudaDeviceReset). Every call shares the array and overwrites
 * the rows it reads, so the array keeps the last call's partial sums; calls that overlap on
 * the GPU (other streams, other threads) race on it and must be ordered by the caller.
 * DEM_ECUDA reports a failure of this call's own lookups or launches only, not an error
 * that other code left pending. */
#define DEM_NOALLOC_MAX_PARCELS 8388608
int dem_reduction_degree_noalloc(const double *m_fe2o3, const double *m_fe3o4, const double *m_feo,
                                 const double *m_fe, const int32_t *ore_type, int32_t n,
                                 double *out, void *cuda_stream);

/* Human-readable text of a status code (static storage). */
const char *dem_strerror(int status);

/* Release everything (safe on NULL and after any error). */
void dem_destroy(dem_ctx *c);

#ifdef __cplusplus
}
#endif
#endif
