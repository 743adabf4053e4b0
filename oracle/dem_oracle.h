/*
 * dem_oracle.h -- plain, slow, FP64 CPU restatement of the particle-side step of
 * Lan et al., "Direct reduction of iron-ore with hydrogen in fluidized beds: a
 * coarse-grained CFD-DEM-IBM study" (arXiv 2311.03908).
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA library against
 * the paper. It shares no code, header, table or helper with the CUDA path; only the
 * tests, the package's smoke() and the benchmark's CPU-baseline leg may load it.
 *
 * Every entry point uses flat arrays: a bed is ORC_NB doubles (integers stored as
 * doubles) in the order of the ORC_B_* indices below; parcel arrays are in input order.
 * Functions whose parity is not pinned by an independent check say so in their comment.
 */
#ifndef DEM_ORACLE_H
#define DEM_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* per-bed parameter vector */
enum {
  ORC_B_D = 0, ORC_B_H, ORC_B_WALL, ORC_B_CONE_ALPHA, ORC_B_CONE_H, ORC_B_PLATE_Z,
  ORC_B_HOLE_D, ORC_B_HOLE_PITCH, ORC_B_NX, ORC_B_NY, ORC_B_NZ, ORC_B_DT, ORC_B_KN,
  ORC_B_KT_KN, ORC_B_REST, ORC_B_MU_S, ORC_B_MU_R, ORC_B_CG, ORC_B_NCOUPLE, ORC_B_U_IN,
  ORC_B_T_IN, ORC_B_P0, ORC_B_Y_IN /* 3 */, ORC_B_K0 = ORC_B_Y_IN + 3, ORC_B_EA = ORC_B_K0 + 3,
  ORC_B_TAU = ORC_B_EA + 3, ORC_B_PSI /* 2 */, ORC_B_XI0 = ORC_B_PSI + 2,
  ORC_B_PORE = ORC_B_XI0 + 2, ORC_B_RHOT = ORC_B_PORE + 2, ORC_B_DPDZ = ORC_B_RHOT + 4,
  ORC_B_EPS_MIN, ORC_B_FLAGS, ORC_B_EMISS /* particle emissivity, eq (3-16) */,
  ORC_B_LAMP /* 2: particle thermal conductivity per ore, W/m/K */, ORC_B_LAMW = ORC_B_LAMP + 2 /* wall, W/m/K */,
  ORC_NB
};

/* physics switches (bit mask in ORC_B_FLAGS) */
enum {
  ORC_NO_GRAVITY = 1, ORC_NO_DRAG = 2, ORC_NO_HEAT = 4, ORC_NO_KINETICS = 8,
  ORC_NO_GAS_UPDATE = 16, ORC_NO_FILM = 32, ORC_NO_LAYER = 64, ORC_NO_RXN_HEAT = 128,
  ORC_NO_CONTACTS = 256,
  ORC_RADIATION = 512,  /* switch ON the particle radiation of eqs (3-16), (3-17), (3-51) */
  ORC_CONDUCTION = 1024, /* switch ON the contact conduction of eqs (3-14)..(3-15-2), (3-42)..(3-48-2) */
  ORC_GAS_SOLVER = 2048  /* the gas phase solved by eqs (3-24), (4-2), (4-6), (4-9) instead of the prescribed field */
};

/* per-parcel state returned by orc_get_state: ORC_NS rows of n doubles */
enum {
  ORC_S_X = 0, ORC_S_Y, ORC_S_Z, ORC_S_VX, ORC_S_VY, ORC_S_VZ, ORC_S_WX, ORC_S_WY, ORC_S_WZ,
  ORC_S_T, ORC_S_M /* 4 */, ORC_S_AX = ORC_S_M + 4, ORC_S_AY, ORC_S_AZ, ORC_S_ALX, ORC_S_ALY,
  ORC_S_ALZ, ORC_NS
};

/* per-parcel diagnostics of the last step: ORC_ND rows of n doubles */
enum {
  ORC_D_FC = 0 /* 3 contact force */, ORC_D_TC = 3 /* 3 contact torque */,
  ORC_D_FD = 6 /* 3 drag force */, ORC_D_K = 9, ORC_D_QCONV, ORC_D_QR, ORC_D_QRM,
  ORC_D_XIDOT /* 3, mol/s per real particle, after limiting */ = 13,
  ORC_D_MDOT = 16 /* 4, kg/s per parcel */, ORC_D_FFILM = 20, ORC_D_A = 21 /* 3 */,
  ORC_D_B = 24 /* 3 */, ORC_D_SH = 27, ORC_D_NU, ORC_D_RE, ORC_D_NCONTACT, ORC_D_CELL,
  ORC_D_TSE /* eq (3-17), 0 without radiation */, ORC_D_QRAD /* eq (3-51), W per parcel */,
  ORC_D_QCOND /* contact conduction with parcels and walls, W per parcel, 0 when off */, ORC_ND
};

/* gas velocity of the solved gas phase (beds with ORC_GAS_SOLVER): per cell ORC_NV doubles,
 * the cell-centre velocity (3) and the pressure relative to p0 */
enum { ORC_V_U = 0, ORC_V_P = 3, ORC_NV };
void orc_get_flow(void *h, double *out);
// face velocities of a solved bed b: (nx+1) ny nz x-faces, nx (ny+1) nz y-faces, nx ny (nz+1)
// z-faces, x fastest (zeros before the first step of a bed that is not solved)
void orc_get_faces(void *h, int b, double *fu, double *fv, double *fw);
/* pseudo-turbulence closures of one cell (eqs (3-28)..(3-37)): out8 = R_pa, R_pe, alpha_pa,
 * alpha_pe, slip direction (3), 0 */
void orc_pseudo_turbulence(double eps, double rho, double mu, double lam, double cp, const double *ug,
                           const double *up, double dp, double *out8);

/* per gas cell: ORC_NG doubles */
enum { ORC_G_EPS = 0, ORC_G_Y /* 3 */, ORC_G_T = 4, ORC_G_MARK, ORC_NG };

/* per gas cell deposits (sums over the parcels in the cell): ORC_NDEP doubles */
enum {
  ORC_DEP_VS = 0, ORC_DEP_SH2, ORC_DEP_SH2O, ORC_DEP_K, ORC_DEP_KV /* 3 */,
  ORC_DEP_HA = 7, ORC_DEP_HAT, ORC_DEP_QRM, ORC_DEP_QR, ORC_DEP_EQ, ORC_DEP_ES, ORC_DEP_COUNT,
  ORC_NDEP
};

/* gas-property vector of orc_gas_props */
enum {
  ORC_GP_RHO = 0, ORC_GP_MU, ORC_GP_LAM, ORC_GP_CP, ORC_GP_X, ORC_GP_XP /* 3 */,
  ORC_GP_DM = 8, ORC_GP_MG, ORC_GP_D12, ORC_GP_D13, ORC_NGP
};

/* single-parcel kinetics vector of orc_kinetics */
enum {
  ORC_K_XIDOT = 0 /* 3 */, ORC_K_MDOT = 3 /* 4 */, ORC_K_SH2 = 7, ORC_K_SH2O, ORC_K_QR, ORC_K_QRM,
  ORC_K_A = 11 /* 3 */, ORC_K_B = 14 /* 3 */, ORC_K_F = 17, ORC_K_SH, ORC_K_F3 = 19 /* f_h,f_m,f_w */,
  ORC_K_ACT = 22 /* 3 */, ORC_K_EQ = 25, ORC_K_ES, ORC_K_DEFF = 27 /* 3 */, ORC_K_XI = 30 /* 3 */,
  ORC_NK = 33
};

#define ORC_MAX_CONTACTS 24

/* ---- stateful stepping ---- */
void *orc_create(int32_t nbeds, const double *beds, int32_t n, const double *x, const double *y,
                 const double *z, const double *vx, const double *vy, const double *vz,
                 const double *d_real, const double *T, const double *m0 /* 4*n, species-major */,
                 const int32_t *ore, const int32_t *bed, const double *gasY /* nullable */,
                 const double *gasT /* nullable */);
int32_t orc_step(void *h, int32_t nsteps);
void orc_get_state(void *h, double *out);
void orc_get_diag(void *h, double *out);
void orc_get_contacts(void *h, int32_t *count, int32_t *partner, double *xi);
int64_t orc_ncells(void *h);
void orc_get_gas(void *h, double *out);
void orc_get_deposits(void *h, double *out);
void orc_reduction_degree(void *h, double *mean_per_bed, double *oxygen_per_bed, double *per_parcel);
void orc_set_kinetics(void *h, const double *k0, const double *Ea);
void orc_set_threads(int32_t nthreads);
int32_t orc_get_threads(void);
void orc_destroy(void *h);

/* adjoint reference: J = mean over parcels of f_ov(after n sub-steps) - f_ov(now) for the
 * frozen-position drag-heat-reaction sub-step; mode 0 = J only, 1 = central finite
 * differences with relative step rel, 2 = forward-mode dual numbers. */
int32_t orc_adjoint(void *h, int32_t nsteps, int32_t mode, double rel, double *J, double *grad6);
/* the same map observed after obs_steps[k] sub-steps: J_obs[k * nbeds + b] = mean over bed b
 * of f_ov - f_ov(now); mode 2 also writes the dual-number gradient of
 * sum_k sum_b weights[k * nbeds + b] J_obs[k * nbeds + b] to grad6 (weights nullable: zero) */
int32_t orc_adjoint_obs(void *h, int32_t nsteps, int32_t mode, int32_t nobs, const int32_t *obs_steps,
                        const double *weights, double *J_obs, double *grad6);

/* ---- single-call pieces for the pins ---- */
void orc_gas_props(const double *bed, double Tg, const double *Y, double p, double *out);
int32_t orc_network(const double *A, const double *B, double F, const int32_t *active_in,
                    double x, const double *xeq, double *J, double *v9, int32_t *active_out);
void orc_kinetics(const double *bed, const double *m, double Tp, double d_real, int32_t ore,
                  double eps, double slip, double Tg, const double *Y, double dt_mass,
                  double *out);
void orc_drag(const double *bed, double d_real, int32_t ore, double eps, double slip,
              double Tg, const double *Y, double *beta_over_epsp, double *Re);
void orc_heat(const double *bed, double d_real, double eps, double slip, double Tg,
              const double *Y, double *Nu, double *h);
double orc_enthalpy(int32_t species, double T);  /* J/kg, Table C1 order H2,H2O,N2,Fe2O3,Fe3O4,FeO,Fe */
double orc_cp(int32_t species, double T);        /* J/kg/K */
double orc_molar_mass(int32_t species);          /* kg/mol, same order */
void orc_layer_porosity(const double *bed, int32_t ore, double *xi3);
int64_t orc_pairs_bruteforce(int32_t n, const double *x, const double *y, const double *z,
                             const double *r, int32_t *pairs, int64_t max_pairs);
int64_t orc_pairs_cells(int32_t n, const double *x, const double *y, const double *z,
                        const double *r, int32_t *pairs, int64_t max_pairs);
void orc_wall_distance(const double *bed, double x, double y, double z, double *dist4, double *n12);
/* contact conduction pieces: f(e) of eqs (3-43), (3-44); e_CGP of eq (3-45) (clamped at 0);
 * one parcel pair (radii, centre distance, temperatures, particle and gas conductivities)
 * -> out[0] Q_pp' and out[1] Q_pfp' into parcel a (eqs (3-14), (3-15), (3-46), (3-48)),
 * out[2] the contact radius R_c, out[3] the lens integral of eq (3-15); one parcel and a
 * wall at distance h -> the same for eqs (3-15-1), (3-15-2), (3-48-1), (3-48-2). */
double orc_restitution_f(double e);
double orc_e_cgp(double e, double k);
void orc_conduction_pair(const double *bed, double Ra, double Rb, double d, double Ta, double Tb,
                         double lam_a, double lam_b, double lam_g, double *out4);
void orc_conduction_wall(const double *bed, double R, double h, double Ta, double lam_a, double lam_g,
                         double *out4);

#ifdef __cplusplus
}
#endif
#endif
