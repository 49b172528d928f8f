/*
 * lbm.h -- C ABI of the GB300 (sm_103a) reactive multi-component lattice Boltzmann step.
 *
 * The library advances the coupled CooLBM models (Alamian, Nayak, Shadloo, arXiv 2502.12955)
 * on one GPU: a D2Q9 / D3Q19 flow lattice per fluid component with the Shan-Chen
 * pseudopotential force (Sec. 2.1.1, Eq. 1.11-1.16), Guo or Shan-Chen velocity-shift forcing
 * (Sec. 2.1.2-2.1.3, Eq. 1.17-1.21), D2Q5 / D3Q7 advection-diffusion lattices for solute and
 * temperature (Sec. 2.1.5, Eq. therpop_species, therpopeq_species), halfway bounce-back, the
 * Kang wet-node reactive boundary (Eq. wetnode9), and the geometry update driven by reaction
 * (solid consumption, Sec. 2.1.5) or deposition (Sec. 3.3, Eq. surface_deposition).
 *
 * Conventions shared by every call:
 *  - Node index n = x + nx*(y + ny*z), x fastest; 2D domains use nz == 1.
 *  - Flags: 0 fluid, 1 inert solid, 2 reactive solid.
 *  - The library owns all device memory.  Host pointers belong to the caller and are only
 *    read or written during the call.  Fields cross the boundary in FP64.
 *  - Every call returns an lbm_status; no call aborts the process.  On error,
 *    lbm_last_error() holds a one-line message.
 *  - Work is enqueued on params.stream (a cudaStream_t, NULL for the legacy default stream).
 *    lbm_step returns after enqueueing.  Calls that return data synchronise that stream.
 *  - One context is used by one host thread at a time.
 *  - The device named by params.device must be the current device of the calling thread for
 *    every call on a context (lbm_get_pops_noalloc alone switches to it and back).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbm_status {
  LBM_OK = 0,
  LBM_ERR_INVALID_ARG = -1,  /* argument out of range; nothing was changed */
  LBM_ERR_OOM = -2,          /* device or host allocation failed */
  LBM_ERR_CUDA = -3,         /* a CUDA runtime call failed (message in lbm_last_error) */
  LBM_ERR_NONFINITE = -4,    /* a monitor evaluation found non-finite populations */
  LBM_ERR_TIMEOUT = -5,      /* a bounded device wait ran out */
  LBM_ERR_STATE = -6,        /* call out of order (e.g. step before fields were set) */
  LBM_ERR_CAPACITY = -7,     /* a device work list overflowed; results after it are invalid.
                                From lbm_get_pops_noalloc: the request exceeds its fixed
                                scratch array; nothing ran and the context is unchanged */
  LBM_ERR_BOUNDS = -8        /* bounds-checked build only (-DLBM_BOUNDS_CHECK): a step kernel
                                computed an index outside its buffer and used 0 instead */
} lbm_status;

typedef enum lbm_lattice {
  LBM_D2Q9_D2Q5 = 2,   /* D2Q9 flow (Table D2Q9, axis weights 1/9) + D2Q5 scalars (Table D2Q5) */
  LBM_D3Q19_D3Q7 = 3   /* D3Q19 flow (Table D3Q19) + D3Q7 scalars */
} lbm_lattice;

typedef enum lbm_precision {
  LBM_FP64 = 0,          /* populations and arithmetic in FP64 */
  LBM_FP32 = 1,          /* populations and arithmetic in FP32 */
  LBM_FP16_SHIFTED = 2,  /* stored as FP16 deviation from w_i * reference, FP32 arithmetic */
  LBM_BF16_SHIFTED = 3,  /* stored as BF16 deviation from w_i * reference, FP32 arithmetic */
  LBM_FP16_SHIFTED_S32 = 4,  /* flow populations as in LBM_FP16_SHIFTED, scalar populations in FP32
                                (deviations from w_j * C_ref): scalars that vary by O(1) across the
                                domain keep FP32 rounding */
  LBM_BF16_SHIFTED_S32 = 5   /* flow populations as in LBM_BF16_SHIFTED, scalars in FP32 */
} lbm_precision;

enum { LBM_FORCING_GUO = 0, LBM_FORCING_SC_SHIFT = 1 };
enum { LBM_COLLISION_BGK = 0, LBM_COLLISION_MRT = 1 };
enum { LBM_PSI_EXP = 0, LBM_PSI_IDENTITY = 1 };
enum { LBM_GEO_NONE = 0, LBM_GEO_DISSOLVE = 1, LBM_GEO_DEPOSIT = 2 };

/* Case parameters (the paper's problem statement: lattice, relaxation times, forces,
   reaction constants, boundary values).  Fill with lbm_params_default() first. */
typedef struct lbm_params {
  int32_t precision;          /* lbm_precision */
  int32_t n_comp;             /* fluid components sigma: 1 or 2 */
  double tau[2];              /* relaxation time per component, > 0.5 (Eq. 1.16) */
  double G[2][2];             /* cohesion G_{sigma,sigma~} (Eq. 1.12-1.14); all zero disables it */
  double G_ads[2];            /* adhesion G_ads,sigma (Eq. 1.15) */
  double rho_solid;           /* density whose psi solid neighbours carry (Eq. 1.13) */
  int32_t psi_kind;           /* LBM_PSI_EXP (Eq. 1.11, rho0) or LBM_PSI_IDENTITY (psi = rho) */
  double rho0;                /* reference density of Eq. 1.11 */
  int32_t forcing;            /* LBM_FORCING_GUO (Eq. 1.19-1.21) or LBM_FORCING_SC_SHIFT (1.17-1.18) */
  double g[3];                /* body acceleration: F_body^sigma = rho^sigma g */
  int32_t collision;          /* LBM_COLLISION_BGK or LBM_COLLISION_MRT (single component, Guo) */
  double s_e, s_eps, s_q, s_pi, s_m;  /* MRT rates of the energy, energy-square, heat-flux,
                                          ghost-stress and cubic moment groups; stress uses 1/tau */
  int32_t n_scal;             /* advection-diffusion lattices: 0, 1 or 2; scalar 0 reacts */
  double tau_c[2];            /* scalar relaxation times, > 0.5 (Eq. therpop_species) */
  double J0;                  /* rest weight of D2Q5 / D3Q7, in [0, 1) */
  double k_react;             /* first-order surface rate k of scalar 0 at reactive links */
  int32_t ade_open_x;         /* 1: scalar inlet at x = 0 (value C_in) and zero-gradient outlet
                                 at x = nx-1; the flow lattice keeps its own periodicity */
  double C_in[2];
  int32_t periodic[3];        /* flow-lattice periodicity per axis; a closed axis has walls */
  int32_t geo_mode;           /* LBM_GEO_NONE / DISSOLVE / DEPOSIT */
  double V_m;                 /* solid mass per unit reacted (dissolution) */
  double m_s0;                /* solid mass of a reactive node (dissolution threshold) */
  double DP;                  /* deposition probability (Eq. surface_deposition) */
  int32_t deposit_conservative; /* 1: deposited particle mass leaves the populations */
  int32_t N_geo;              /* geometry flips every N_geo steps (>= 1) */
  int32_t N_mon;              /* automatic monitor + residual every N_mon steps (0: never) */
  double rho_ref[2];          /* storage shift references for 16-bit modes (flow) */
  double C_ref[2];            /* storage shift references for 16-bit modes (scalars) */
  void* stream;               /* cudaStream_t for all work of this context */
  int32_t block_x;            /* threads per block of the step kernel: 0 (automatic: 256) or a
                                 multiple of 32 up to 256 */
  int32_t device;             /* CUDA device ordinal */
  int32_t l2_fetch_bytes;     /* L2 fetch granularity hint for this process's context
                                 (cudaLimitMaxL2FetchGranularity: 32, 64 or 128; 0, the default,
                                 leaves the context's current value).  Smaller fetches move fewer
                                 bytes on porous geometries but expose more latency. */
  double u_wall_ymax[3];      /* velocity of the closed face beyond y = ny-1 (moving top plate,
                                 Sec. 3.1.1 Couette flow): its links reflect with Ladd's momentum
                                 term 2 w_i rho (c_i . u) / c_s^2.  Needs periodic[1] == 0 and a
                                 tangential velocity (component 1 zero); zero disables it. */
  int32_t flow_open_x;        /* 1: the flow lattice has a velocity inlet at x = 0 and a zero-gradient
                                 outlet at x = nx-1 (Sec. 3.4).  Links leaving through x = 0
                                 reflect off a face moving with u_x = 6 u_in s (1 - s),
                                 s = (y + 1/2) / ny (Ladd's term 2 w_i rho (c_i . u) / c_s^2); the
                                 population entering through x = nx-1 repeats the node's own
                                 post-collision value.  Needs periodic[0] == periodic[1] == 0,
                                 nx >= 2 and one component without Shan-Chen or adhesion forces. */
  double u_in;                /* mean velocity U of the inlet profile (flow_open_x only) */
  int32_t arrhenius;          /* 1: scalar 1 is the temperature T.  The surface rate of scalar 0 at
                                 each reactive link is k(T_b) = arr_A exp(-arr_Ta / T_b) at the
                                 link's interface temperature, and the reaction releases the heat
                                 flux heat_release * k C_b into T (Sec. 2.1.5, Eq. reactO2, reacRate,
                                 fluxCon with an adiabatic solid).  C_b and T_b are solved together
                                 per link by n_it fixed-point iterations from the zero-flux value.
                                 Needs n_scal == 2; k_react is not used. */
  double arr_A;               /* pre-exponential factor A (>= 0) */
  double arr_Ta;              /* activation temperature E / R_u (>= 0) */
  double heat_release;        /* h_r: heat flux per unit reaction rate */
  int32_t n_it;               /* iterations of the C_b - T_b coupling, 0..64 (default 16) */
  int32_t product;            /* 1: one more scalar lattice after the n_scal given ones carries the
                                 product of the surface reaction (CO2; Sec. 2.1.5, Eq. react,
                                 reactCO2).  At each reactive link it gains what the reaction takes
                                 from scalar 0 there, r = k C_b: the per-link wet-node ansatz with
                                 the flux reversed gives h_P,i = h_P,opp(i) + r tau_p / (tau_p - 1/2).
                                 Fields and populations then carry n_scal + 1 scalar rows, the
                                 product last; its 16-bit storage reference is 0.  Needs n_scal >= 1,
                                 no deposition, one component when n_scal == 2; not in ensembles. */
  double tau_p;               /* relaxation time of the product lattice (> 0.5) */
  double C_in_p;              /* product value of the inlet ghost (with ade_open_x) */
  int32_t conjugate;          /* 1 (with arrhenius): heat conduction in the solid on its own D3Q7 /
                                 D2Q5 lattice, g_s,eq = w T_s (Sec. 2.1.5, Eq. therpop_solid,
                                 macroreacb_solid), exchanged with the fluid temperature link by
                                 link after each step (Eq. tempCon, fluxCon, reacRate): at a fluid-
                                 solid link the two post-collision populations meet at
                                 T_b = (c_fs ho + go + c_fs Qp / 2) / (w (c_fs + 1)) and each side
                                 receives 2 w T_b minus what it sent; Qp = heat_release k(T_b) C_b
                                 at a reactive link, whose k the next step's species closure uses.
                                 Faces that are not periodic for the scalars reflect.  Row 1 of the
                                 fields (set and get) is the solid temperature at solid nodes.  Not
                                 with deposition or in ensembles; checkpoints carry the solid lattice. */
  double tau_s;               /* relaxation time of the solid thermal lattice (> 0.5) */
  double c_fs;                /* heat-capacity ratio (rho c_p)_fluid / (rho c_p)_solid (> 0) */
} lbm_params;

/* Monitors, all FP64.  Cumulative entries count from the last lbm_set_fields. */
typedef struct lbm_monitors {
  double step;                /* completed steps */
  double mass[2];             /* sum of stored populations per component over fluid nodes */
  double momentum[3];         /* sum_sigma sum_i c_i f_i over fluid nodes */
  double species[2];          /* sum of stored scalar populations over fluid nodes */
  double reacted;             /* cumulative reaction k C_b over reactive links (scalar 0) */
  double inflow[2];           /* cumulative scalar entering through the inlet */
  double outflow[2];          /* cumulative scalar leaving through the outlet */
  double injected_mass[2];    /* added by dissolution flips */
  double injected_species[2];
  double removed_mass[2];     /* removed by deposition flips */
  double removed_species[2];
  double deposited;           /* cumulative deposited particle mass */
  double n_solid;
  double n_fluid;
  double nonfinite;           /* fluid nodes holding a non-finite population */
  double wall_exchange;       /* cumulative scalar-0 population loss through reactive links */
  double residual;            /* last automatic residual (-1 if none yet) */
  double heat;                /* cumulative temperature-population gain through reactive links
                                 (arrhenius only; with conjugate, through every fluid-solid link) */
  double species_p;           /* product lattice (product only): sum of its stored populations */
  double inflow_p;            /* cumulative product entering through the inlet */
  double outflow_p;           /* cumulative product leaving through the outlet */
  double injected_species_p;  /* product added by dissolution flips */
  double removed_species_p;   /* always 0 (the product is not combined with deposition) */
  double produced;            /* cumulative product-population gain through reactive links */
  double t_solid;             /* conjugate only: sum of the solid lattice's populations */
  double heat_solid;          /* cumulative solid-population gain through fluid-solid links
                                 (conjugate; heat holds the fluid side's gain there) */
  double heat_source;         /* cumulative reaction heat put into the link exchanges (conjugate) */
  double solid_removed;       /* cumulative solid populations taken by dissolution (conjugate) */
} lbm_monitors;

typedef struct lbm_ctx lbm_ctx;

/* Fill *p with defaults: FP32, one component, tau 1, no forces, BGK, Guo, no scalars,
   periodic box, no geometry update, N_geo 1, N_mon 0, device 0, l2_fetch_bytes 0. */
lbm_status lbm_params_default(lbm_params* p);

/* Allocate a context for an nx x ny x nz domain (Sec. 2.1.4 lattices).  Validates every
   parameter (tau > 0.5, n_comp, n_scal, J0, MRT only with one component and Guo forcing,
   nz == 1 for 2D, nx >= 2 with ade_open_x).  Device memory: populations in SoA planes
   pop[q][n], one in-place copy per lattice, plus flags, link masks and FP64 bookkeeping.
   *out is NULL on error; lbm_last_error(NULL) then holds the reason. */
lbm_status lbm_create(lbm_lattice lattice, int32_t nx, int32_t ny, int32_t nz,
                      const lbm_params* params, lbm_ctx** out);

/* Copy the geometry (flags[n], n = nx*ny*nz bytes, host) and rebuild the link masks.  Resets
   the per-node bookkeeping (consumed / deposited amounts) to zero.  Values above 2 are
   rejected.  Call lbm_set_fields afterwards. */
lbm_status lbm_set_geometry(lbm_ctx* ctx, const uint8_t* flags, size_t n);

/* Initialise populations at equilibrium (Eq. 6, Eq. therpopeq_species) from host FP64 fields:
   rho [n_comp][N], u [3][N] (2D: the z row is ignored), C [n_scal + product][N] (NULL when
   n_scal == 0; the product's row last).  Solid nodes are ignored, except with conjugate, where
   row 1 at a solid node is its initial temperature (the solid lattice starts at rest
   equilibrium).  Resets the step counter and all monitors. */
lbm_status lbm_set_fields(lbm_ctx* ctx, const double* rho, const double* u, const double* C,
                          size_t n);

/* Enqueue nsteps time steps (Sec. 2.1: collide-stream of every lattice, reactive closure,
   geometry update every N_geo steps, monitors every N_mon steps). */
lbm_status lbm_step(lbm_ctx* ctx, int64_t nsteps);

/* Wait for the context's stream; report device-side errors (LBM_ERR_CAPACITY,
   LBM_ERR_NONFINITE from the automatic monitor). */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Copy macroscopic fields at the current time into caller buffers (any may be NULL):
   rho [n_comp][N]; u [3][N], the physical velocity sum_sigma (j^sigma + F^sigma/2) / rho
   (Eq. 1.19); C [n_scal][N] with the wet-node closure applied; flags [N]; acc [N], the
   per-node consumed amount (reactive solids) or deposited fraction (deposition).  With the
   reaction product, C has n_scal + 1 rows (the product last), as in lbm_set_fields.  With
   conjugate, row 1 at a solid node holds the solid temperature (Eq. macroreacb_solid). */
lbm_status lbm_get_fields(lbm_ctx* ctx, double* rho, double* u, double* C, uint8_t* flags,
                          double* acc);

/* The same fields left on the device: computes them into the context's FP64 staging arrays and
   returns device pointers (any output may be NULL): rho [n_comp][N], u [3][N], C [n_scal +
   product][N] (NULL without scalars), flags [N] (uint8), acc [N], in the layouts of
   lbm_get_fields.  The context owns the memory.  The arrays hold this call's values until the
   next lbm_get_fields, lbm_get_fields_device or lbm_set_fields (which stage through them), the
   flags and acc until the next step or geometry call.  The context's stream is synchronised
   before return, so readers on any stream see complete values.  No host copy is made. */
lbm_status lbm_get_fields_device(lbm_ctx* ctx, const double** rho, const double** u, const double** C,
                                 const uint8_t** flags, const double** acc);

/* Pre-collision populations at the current time, FP64, [n_comp][Qf][N] and
   [n_scal + product][Qc][N] (either may be NULL).  Reactive-link scalar slots hold the stored bounce-back value. */
lbm_status lbm_get_pops(lbm_ctx* ctx, double* f, double* h);
lbm_status lbm_set_pops(lbm_ctx* ctx, const double* f, const double* h);

/* Same result as lbm_get_pops, without allocating device memory.  The paper has no counterpart;
   this entry point exists for callers that cannot call cudaMalloc: code whose device memory is
   fully reserved by another allocator (for example a framework's caching pool), or code that
   must not trigger the implicit device-wide synchronisation of cudaMalloc / cudaFree.
   The populations are staged through a fixed device scratch array of
   LBM_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading this library holds until the
   process exits.  A request of more than that many bytes, (n_comp*Qf [if f] + n_scal*Qc [if h])
   * N * 8, is rejected with LBM_ERR_CAPACITY before anything runs.  All calls share that array:
   calls on different contexts or streams that overlap on the GPU race on it, so serialise
   them.  The first call on a device looks up the array's device address
   (cudaGetSymbolAddress) and keeps it for the life of the process; make that first call before
   any stream capture, and make no call after cudaDeviceReset, which would leave the kept
   address stale.  Outputs are host buffers as in lbm_get_pops; the call synchronises the
   stream. */
#define LBM_NOALLOC_SCRATCH_BYTES (16u << 20)
lbm_status lbm_get_pops_noalloc(lbm_ctx* ctx, double* f, double* h);

/* Evaluate the monitors now (FP64 reductions on the device) and copy them to *out. */
lbm_status lbm_get_monitors(lbm_ctx* ctx, lbm_monitors* out);

/* Relative L2 change of u and C (max of the two) over fluid nodes since the previous call;
   -1 on the first call.  Replaces the stored snapshot. */
lbm_status lbm_residual(lbm_ctx* ctx, double* r);

/* Checkpoint: raw populations in storage precision, flags, bookkeeping, step counter (which
   fixes the in-place layout parity) and cumulative monitors.  With host == NULL, *nbytes
   receives the required size.  lbm_set_state restores a checkpoint of the same shape and
   parameters bit for bit. */
lbm_status lbm_get_state(lbm_ctx* ctx, void* host, size_t* nbytes);
lbm_status lbm_set_state(lbm_ctx* ctx, const void* host, size_t nbytes);

/* Device time of the population pass of each step: when enabled, lbm_step brackets the fused
   step kernel, together with the psi pass that precedes it when Shan-Chen forces are on, with
   CUDA events on the context's stream.  lbm_profile_read synchronises and returns the summed
   milliseconds and the number of bracketed steps since the last read. */
lbm_status lbm_profile_enable(lbm_ctx* ctx, int32_t on);
lbm_status lbm_profile_read(lbm_ctx* ctx, double* ms, int64_t* launches);

/* Kernel launches enqueued by this context since creation (all kernels of the library). */
lbm_status lbm_launch_count(lbm_ctx* ctx, int64_t* launches);

/* Message of the last failed call on ctx; with ctx == NULL, of the last failed lbm_create on
   the calling thread. */
const char* lbm_last_error(const lbm_ctx* ctx);
void lbm_destroy(lbm_ctx* ctx);

/* ---------------------------------------------------------------- ensembles
 *
 * Many independent domains of one lattice, possibly of different sizes, advanced together: one
 * persistent kernel walks a work list of tiles (blocks of consecutive fluid-list entries of one
 * member) across all active members, and even + odd step pairs replay as one CUDA graph.  This
 * is the batched form of the same per-step update (Sec. 2.1 Eq. 1.16 / 1.21 with Sec. 2.1.5),
 * for sweeps of geometries run to steady state.
 *
 * Members share precision, n_comp, n_scal, collision, block_x, device and stream; each has its
 * own size, geometry, relaxation times, forces and scalar parameters.  Ensembles keep their
 * geometry (geo_mode LBM_GEO_NONE) and use Guo forcing without Shan-Chen forces; other
 * parameters are rejected with LBM_ERR_INVALID_ARG.
 */
typedef struct lbm_ensemble lbm_ensemble;

/* n members; member k has size dims[3k], dims[3k+1], dims[3k+2] and parameters params[k].
   Allocates every member's device memory; on failure nothing is left allocated and
   lbm_ensemble_last_error(NULL) says which member failed. */
lbm_status lbm_ensemble_create(lbm_lattice lattice, int32_t n, const int32_t* dims,
                               const lbm_params* params, lbm_ensemble** out);

/* Context of member k, owned by the ensemble (do not lbm_destroy it): set its geometry and
   fields, read fields, monitors and the residual through the single-domain calls.  Stepping a
   member with lbm_step is allowed but leaves it out of step with the others. */
lbm_status lbm_ensemble_member(lbm_ensemble* e, int32_t k, lbm_ctx** out);

/* Advance every active member by nsteps.  Active members must share one step count
   (LBM_ERR_STATE otherwise) and have their fields set.  Each member's monitors and residual
   are evaluated every N_mon of its steps, as lbm_step does. */
lbm_status lbm_ensemble_step(lbm_ensemble* e, int64_t nsteps);

/* Step until every active member's residual (evaluated every N_mon steps; one common
   N_mon > 0 is required) is <= r_tol, or max_steps have been taken.  A member that reaches the
   tolerance stops stepping (leaves the work list).  Returns the steps taken and how many
   members have stopped. */
lbm_status lbm_ensemble_run_to_steady(lbm_ensemble* e, double r_tol, int64_t max_steps,
                                      int64_t* steps_done, int32_t* n_converged);

/* Time `steps` (even, >= 2) real steps of the ensemble with each tile size of 64, 128 and 256
   entries and keep the fastest; the steps advance the simulation.  threads_out may be NULL. */
lbm_status lbm_ensemble_autotune(lbm_ensemble* e, int32_t steps, int32_t* threads_out);

/* Kernel launches of the ensemble and its members since creation. */
lbm_status lbm_ensemble_launch_count(lbm_ensemble* e, int64_t* launches);

/* Message of the last failed ensemble call; with e == NULL, of the last failed
   lbm_ensemble_create on the calling thread. */
const char* lbm_ensemble_last_error(const lbm_ensemble* e);
void lbm_ensemble_destroy(lbm_ensemble* e);

#ifdef __cplusplus
}
#endif
#endif
