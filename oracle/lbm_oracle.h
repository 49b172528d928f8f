/*
 * lbm_oracle.h -- plain FP64 CPU oracle of the CooLBM per-time-step update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no header, table or helper with
 * the CUDA path (paper_2502_12955_gb300/csrc); the two are written
 * independently from the paper.
 *
 * Node index n = x + nx*(y + ny*z), x fastest; 2D runs use nz == 1.
 * Flags: 0 fluid, 1 inert solid, 2 reactive solid.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
  int32_t dim;                 /* 2 -> D2Q9 flow + D2Q5 scalars; 3 -> D3Q19 + D3Q7 */
  int32_t nx, ny, nz;
  int32_t n_comp;              /* fluid components sigma, 1..2 */
  double tau[2];               /* relaxation time per component (Eq. 1.16) */
  double G[2][2];              /* cohesion G_{sigma,sigma~} (Eq. 1.12-1.14) */
  double G_ads[2];             /* adhesion G_ads,sigma (Eq. 1.15) */
  double rho_solid;            /* psi(rho_s) used for solid neighbours (Eq. 1.13) */
  int32_t psi_kind;            /* 0: psi = rho0 (1 - exp(-rho/rho0)) (Eq. 1.11); 1: psi = rho */
  double rho0;                 /* reference density in Eq. 1.11 */
  int32_t forcing;             /* 0: Guo (Sec. 2.1.3); 1: Shan-Chen velocity shift (Sec. 2.1.2) */
  double g[3];                 /* body acceleration; F_body^sigma = rho^sigma g */
  int32_t collision;           /* 0: BGK; 1: MRT (Gram-Schmidt moment basis) */
  double s_e, s_eps, s_q, s_pi, s_m;   /* MRT rates of the non-hydrodynamic moment groups */
  int32_t n_scal;              /* advection-diffusion lattices, 0..2; scalar 0 reacts (the product
                                  lattice, if any, comes after them) */
  double tau_c[2];             /* scalar relaxation times (Eq. therpop_species) */
  double J0;                   /* rest weight of D2Q5 / D3Q7 */
  double k_react;              /* first-order surface rate k of scalar 0 (Eq. reactO2, wetnode9) */
  int32_t ade_open_x;          /* 1: scalars have inlet at x=0 (C_in) and zero-gradient outlet at x=nx-1 */
  double C_in[2];
  int32_t periodic[3];         /* flow-lattice periodicity per axis */
  int32_t geo_mode;            /* 0 none, 1 dissolution, 2 deposition */
  double V_m;                  /* solid mass removed per unit of reacted scalar */
  double m_s0;                 /* initial solid mass of a reactive node */
  double DP;                   /* deposition probability (Eq. surface_deposition) */
  int32_t deposit_conservative;/* 1: deposited particle mass leaves the populations */
  int32_t N_geo;               /* geometry flips evaluated every N_geo steps */
  double u_wall_ymax[3];       /* velocity of the closed face beyond y = ny-1 (moving-wall
                                  bounce-back, Sec. 3.1.1 Couette flow); needs periodic[1] == 0 */
  int32_t flow_open_x;         /* 1: flow velocity inlet at x = 0 and zero-gradient outlet at
                                  x = nx-1 (Sec. 3.4); needs periodic[0] == periodic[1] == 0 and
                                  one component without Shan-Chen forces */
  double u_in;                 /* mean inlet velocity U of the profile u_x = 6 U s (1 - s),
                                  s = (y + 1/2) / ny */
  int32_t arrhenius;           /* 1: scalar 1 is the temperature T; the surface rate of scalar 0 is
                                  k(T_b) = A exp(-Ta / T_b) at each reactive link's interface
                                  temperature, and the reaction releases heat into T (Sec. 2.1.5,
                                  Eq. reactO2, reacRate, fluxCon; an adiabatic solid unless
                                  conjugate is set) */
  double arr_A;                /* pre-exponential factor A */
  double arr_Ta;               /* activation temperature E / R_u */
  double heat_release;         /* h_r: heat flux released per unit reaction rate */
  int32_t n_it;                /* fixed-point iterations of the C_b - T_b coupling per link */
  int32_t conjugate;           /* 1 (with arrhenius): heat conduction in the solid on its own scalar
                                  lattice, exchanged with the fluid temperature link by link
                                  (Sec. 2.1.5, Eq. therpop_solid, tempCon, fluxCon, reacRate);
                                  not with deposition */
  double tau_s;                /* relaxation time of the solid thermal lattice (tau_e,s) */
  double c_fs;                 /* heat-capacity ratio (rho c_p)_f / (rho c_p)_s */
  int32_t product;             /* 1: one more scalar lattice after the n_scal ones, the product (CO2)
                                  of the surface reaction: at each reactive link it gains what the
                                  reaction takes from scalar 0 (Sec. 2.1.5, Eq. react, reactCO2) */
  double tau_p;                /* relaxation time of the product lattice (tau_d,CO2) */
  double C_in_p;               /* product value of the inlet ghost (with ade_open_x) */
} orc_params;

/* Monitor vector layout (doubles). */
enum {
  ORC_MON_STEP = 0,
  ORC_MON_MASS = 1,        /* 2 entries: sum of populations per component over fluid nodes */
  ORC_MON_MOM = 3,         /* 3 entries: sum_sigma sum_i c_i f_i over fluid nodes */
  ORC_MON_SPECIES = 6,     /* 2 entries */
  ORC_MON_REACTED = 8,     /* cumulative reaction k C_b summed over reactive links, scalar 0 */
  ORC_MON_INFLOW = 9,      /* 2 entries, cumulative */
  ORC_MON_OUTFLOW = 11,    /* 2 entries, cumulative */
  ORC_MON_INJ_MASS = 13,   /* 2 entries, cumulative mass injected by dissolution flips */
  ORC_MON_INJ_SPEC = 15,   /* 2 */
  ORC_MON_REM_MASS = 17,   /* 2, removed by deposition flips */
  ORC_MON_REM_SPEC = 19,   /* 2 */
  ORC_MON_DEPOSITED = 21,  /* cumulative deposited particle mass */
  ORC_MON_NSOLID = 22,
  ORC_MON_NFLUID = 23,
  ORC_MON_NONFINITE = 24,
  ORC_MON_WALLX = 25,      /* cumulative scalar-0 population loss through reactive links */
  ORC_MON_HEAT = 26,       /* cumulative temperature-population gain through reactive links
                              (conjugate: through every solid link, fluid side) */
  ORC_MON_TSOLID = 27,     /* conjugate: sum of the stored solid temperature populations */
  ORC_MON_HEAT_S = 28,     /* conjugate: cumulative solid-population gain through solid links */
  ORC_MON_HEAT_SRC = 29,   /* conjugate: cumulative reaction heat put into the link exchanges,
                              in units of the fluid's rho c_p */
  ORC_MON_SOLID_REM = 30,  /* conjugate: cumulative solid populations removed by dissolution */
  ORC_MON_SPECIES_P = 31,  /* product lattice: the entries that scalars 0 and 1 have above */
  ORC_MON_INFLOW_P = 32,
  ORC_MON_OUTFLOW_P = 33,
  ORC_MON_INJ_SPEC_P = 34,
  ORC_MON_REM_SPEC_P = 35,
  ORC_MON_PRODUCED = 36,   /* cumulative product-population gain through reactive links */
  ORC_MON_COUNT = 37
};

typedef struct orc_ctx orc_ctx;

orc_ctx* orc_create(const orc_params* p, int* status);
void orc_destroy(orc_ctx* c);
int orc_set_geometry(orc_ctx* c, const uint8_t* flags);
/* rho: [n_comp][N], u: [3][N] (2D: uz ignored), C: [n_scal + product][N] (the product last);
   NULL C allowed if there is no scalar lattice */
int orc_set_fields(orc_ctx* c, const double* rho, const double* u, const double* C);
int orc_step(orc_ctx* c, int64_t nsteps);
/* rho [n_comp][N], u [3][N] physical velocity, C [n_scal + product][N], flags [N], acc [N]; any
   may be NULL */
int orc_get_fields(orc_ctx* c, double* rho, double* u, double* C, uint8_t* flags, double* acc);
/* pre-collision populations at the current time: f [n_comp][Qf][N], h [n_scal + product][Qc][N] */
int orc_get_pops(orc_ctx* c, double* f, double* h);
int orc_set_pops(orc_ctx* c, const double* f, const double* h);
int orc_get_monitors(orc_ctx* c, double* out /* ORC_MON_COUNT */);
/* relative L2 change of u and C since the previous call over fluid nodes (max of the two);
   the first call returns -1 */
double orc_residual(orc_ctx* c);
/* MRT moment matrix M [Q][Q] (row-major) and rate vector S [Q] as built by Gram-Schmidt */
int orc_get_mrt(orc_ctx* c, double* M, double* S);
int orc_lattice(orc_ctx* c, int which /*0 flow, 1 scalar*/, int* q, int* cvec /*[Q][3]*/, double* w);

#ifdef __cplusplus
}
#endif
#endif
