/*
 * lbm_oracle.c -- plain, slow, FP64 CPU oracle of the CooLBM per-step update.
 *
 * TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).  Written from the paper
 * (Alamian, Nayak, Shadloo, "CooLBM", arXiv 2502.12955):
 *   Sec. 2.1    LBGK collision and streaming (Eq. 3-6), moments (Eq. 1.7, 1.8)
 *   Sec. 2.1.1  Shan-Chen pseudopotential force (Eq. 1.11-1.16)
 *   Sec. 2.1.2  Shan-Chen velocity-shift forcing (Eq. 1.17, 1.18)
 *   Sec. 2.1.3  Guo forcing, barycentric velocity (Eq. 1.19-1.21)
 *   Sec. 2.1.4  velocity sets (Tables D3Q19, D2Q9, D2Q5)
 *   Sec. 2.1.5  species advection-diffusion LBGK (Eq. therpop_species,
 *               therpopeq_species) and the Kang wet-node reactive boundary
 *               (Eq. wetnode9)
 *   Sec. 2.1.5  temperature-dependent rate and reaction heat (Eq. reactO2,
 *               reacRate, fluxCon); conduction in the solid and its link
 *               exchange with the fluid temperature (Eq. therpop_solid,
 *               macroreacb_solid, tempCon, fluxCon, unknownpopTempS); the
 *               reaction product (Eq. react, reactCO2)
 *   Sec. 3.1.1  moving plate; Sec. 3.4 velocity inlet and outlet
 *   Sec. 3.3    particle deposition (Eq. surface_deposition)
 * Where the paper is silent or garbled this file takes these readings: D2Q9
 * weights normalised; D3Q7 for 3D scalars; the wet node applied per link;
 * dissolution by solid-mass bookkeeping; synchronous psi evaluation; the
 * solid-fluid heat exchange in a per-link, energy-conserving form (at
 * exchange_solid).
 *
 * Every step is a full sweep with two population arrays (pull streaming):
 *   A. wet-node closure of the unknown scalar populations at reactive links
 *      (Eq. wetnode9, applied to the gathered populations) with reaction
 *      bookkeeping; then deposition at near-substrate fluid nodes
 *   B. rho, psi for ALL nodes, then forces, then velocities
 *   C. flow collision (BGK or MRT, Guo or velocity shift); scalar collision
 *   D. pull streaming with halfway bounce-back at walls (reactive links keep
 *      the bounce-back value until the next closure), inlet/outlet, periodic wrap;
 *      with conduction in the solid, the solid collision comes after C, and the
 *      exchange across solid links of the temperature and the streaming inside
 *      the solid after D
 *   E. geometry flips (every N_geo steps), effective from the next step
 * No blocking, fusion or reordering beyond that; sums run i = 0..Q-1.
 * Compile with -ffp-contract=off.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define QMAX 19

typedef struct {
  int q;
  int c[QMAX][3];
  double w[QMAX];
  int opp[QMAX];
  double cs2;
} lattice_t;

struct orc_ctx {
  orc_params p;
  int64_t N;
  lattice_t lf, lc;               /* flow and scalar lattices */
  int per_c[3];                   /* scalar-lattice periodicity */
  double* f[2];                   /* [N][Qf] pre-collision, per component */
  double* fp[2];                  /* post-collision */
  double* h[3];                   /* [N][Qc] stored state (reactive links hold bounce-back value);
                                     scalars 0 .. n_scal-1, then the product lattice */
  double* hc[3];                  /* [N][Qc] state after the wet-node closure (per-step scratch) */
  double* hp[3];
  uint8_t* flag;
  double* acc;                    /* reacted amount (solid) / deposited fraction (fluid) */
  double* rho[2];
  double* jm[2];                  /* [N][3] bare momentum sum_i c_i f_i */
  double* psi[2];
  double* F[2];                   /* [N][3] total force per component */
  double* ub;                     /* [N][3] barycentric / physical velocity */
  double* Cs[3];                  /* scalar value per node */
  double* gs;                     /* [N][Qc] solid thermal populations, stored (conjugate) */
  double* gsp;                    /* post-collision */
  double* kb;                     /* [N][Qc] rate constant k(T_b) of each fluid node's reactive
                                     link, set by the last exchange (conjugate) */
  uint8_t* kb_ok;                 /* 1 once kb of the link was set by an exchange */
  double mon[ORC_MON_COUNT];
  int64_t t;
  double* snap_u;
  double* snap_C;
  int have_snap;
  double M[QMAX][QMAX];
  double Minv[QMAX][QMAX];
  double S[QMAX];
};

/* ---------------------------------------------------------------- tables */

/* Table D3Q19 (Sec. 2.1.4), velocity order as printed. */
static const int D3Q19_C[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, 0, 1},  {-1, 0, -1}, {0, 1, 1},  {0, -1, -1}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}, {0, 1, -1}, {0, -1, 1}};
/* Table D2Q9 (Sec. 2.1.4), velocity order as printed. */
static const int D2Q9_C[9][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};

static void finish_lattice(lattice_t* L) {
  for (int i = 0; i < L->q; ++i) {
    L->opp[i] = -1;
    for (int j = 0; j < L->q; ++j)
      if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
        L->opp[i] = j;
  }
  /* c_s^2 from its definition sum_i w_i c_ix^2 */
  double s = 0.0;
  for (int i = 0; i < L->q; ++i) s += L->w[i] * (double)(L->c[i][0] * L->c[i][0]);
  L->cs2 = s;
}

static void make_lattices(orc_ctx* c) {
  lattice_t* L = &c->lf;
  if (c->p.dim == 3) {
    L->q = 19;
    for (int i = 0; i < 19; ++i) {
      for (int a = 0; a < 3; ++a) L->c[i][a] = D3Q19_C[i][a];
      L->w[i] = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
  } else {
    L->q = 9;
    for (int i = 0; i < 9; ++i) {
      for (int a = 0; a < 3; ++a) L->c[i][a] = D2Q9_C[i][a];
      /* printed w_4 = 1/36 does not normalise; the axis weights are 1/9 */
      L->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
  }
  finish_lattice(L);
  /* scalar lattice: D2Q5 (Table D2Q5, w0 = J0) or D3Q7 (same rule in 3D) */
  lattice_t* K = &c->lc;
  int qc = (c->p.dim == 3) ? 7 : 5;
  K->q = qc;
  for (int i = 0; i < qc; ++i) {
    for (int a = 0; a < 3; ++a) K->c[i][a] = (c->p.dim == 3) ? D3Q19_C[i][a] : D2Q9_C[i][a];
    K->w[i] = (i == 0) ? c->p.J0 : (1.0 - c->p.J0) / (double)(qc - 1);
  }
  finish_lattice(K);
}

/* ------------------------------------------------------------ MRT basis */

enum { GRP_CONS = 0, GRP_E, GRP_EPS, GRP_Q, GRP_NU, GRP_PI, GRP_M };

/* Monomial k of velocity c, d'Humieres (3D) / Lallemand-Luo (2D) ordering. */
static double monomial(int dim, int k, const int* cv, int* grp) {
  double x = cv[0], y = cv[1], z = cv[2];
  double c2 = x * x + y * y + z * z;
  if (dim == 2) {
    switch (k) {
      case 0: *grp = GRP_CONS; return 1.0;
      case 1: *grp = GRP_E; return c2;
      case 2: *grp = GRP_EPS; return c2 * c2;
      case 3: *grp = GRP_CONS; return x;
      case 4: *grp = GRP_Q; return c2 * x;
      case 5: *grp = GRP_CONS; return y;
      case 6: *grp = GRP_Q; return c2 * y;
      case 7: *grp = GRP_NU; return x * x - y * y;
      default: *grp = GRP_NU; return x * y;
    }
  }
  switch (k) {
    case 0: *grp = GRP_CONS; return 1.0;
    case 1: *grp = GRP_E; return c2;
    case 2: *grp = GRP_EPS; return c2 * c2;
    case 3: *grp = GRP_CONS; return x;
    case 4: *grp = GRP_Q; return c2 * x;
    case 5: *grp = GRP_CONS; return y;
    case 6: *grp = GRP_Q; return c2 * y;
    case 7: *grp = GRP_CONS; return z;
    case 8: *grp = GRP_Q; return c2 * z;
    case 9: *grp = GRP_NU; return 3.0 * x * x - c2;
    case 10: *grp = GRP_PI; return c2 * (3.0 * x * x - c2);
    case 11: *grp = GRP_NU; return y * y - z * z;
    case 12: *grp = GRP_PI; return c2 * (y * y - z * z);
    case 13: *grp = GRP_NU; return x * y;
    case 14: *grp = GRP_NU; return y * z;
    case 15: *grp = GRP_NU; return x * z;
    case 16: *grp = GRP_M; return x * (y * y - z * z);
    case 17: *grp = GRP_M; return y * (z * z - x * x);
    default: *grp = GRP_M; return z * (x * x - y * y);
  }
}

/* Gram-Schmidt on the monomials (unweighted inner product over directions),
   Gauss-Jordan inverse, and the rate of each row's group. */
static int build_mrt(orc_ctx* c) {
  int Q = c->lf.q;
  int grp[QMAX];
  double A[QMAX][QMAX];
  for (int k = 0; k < Q; ++k) {
    for (int i = 0; i < Q; ++i) A[k][i] = monomial(c->p.dim, k, c->lf.c[i], &grp[k]);
    for (int j = 0; j < k; ++j) {
      double num = 0.0, den = 0.0;
      for (int i = 0; i < Q; ++i) {
        num += A[k][i] * c->M[j][i];
        den += c->M[j][i] * c->M[j][i];
      }
      double r = num / den;
      for (int i = 0; i < Q; ++i) A[k][i] -= r * c->M[j][i];
    }
    for (int i = 0; i < Q; ++i) c->M[k][i] = A[k][i];
  }
  /* Gauss-Jordan with partial pivoting on [M | I] */
  double W[QMAX][2 * QMAX];
  for (int r = 0; r < Q; ++r)
    for (int s = 0; s < 2 * Q; ++s) W[r][s] = (s < Q) ? c->M[r][s] : (s - Q == r ? 1.0 : 0.0);
  for (int col = 0; col < Q; ++col) {
    int piv = col;
    for (int r = col + 1; r < Q; ++r)
      if (fabs(W[r][col]) > fabs(W[piv][col])) piv = r;
    if (fabs(W[piv][col]) < 1e-12) return -1;
    if (piv != col)
      for (int s = 0; s < 2 * Q; ++s) {
        double t = W[col][s];
        W[col][s] = W[piv][s];
        W[piv][s] = t;
      }
    double d = W[col][col];
    for (int s = 0; s < 2 * Q; ++s) W[col][s] /= d;
    for (int r = 0; r < Q; ++r) {
      if (r == col) continue;
      double m = W[r][col];
      if (m == 0.0) continue;
      for (int s = 0; s < 2 * Q; ++s) W[r][s] -= m * W[col][s];
    }
  }
  for (int r = 0; r < Q; ++r)
    for (int s = 0; s < Q; ++s) c->Minv[r][s] = W[r][Q + s];
  for (int k = 0; k < Q; ++k) {
    double s_nu = 1.0 / c->p.tau[0]; /* replaced per component in collide */
    switch (grp[k]) {
      case GRP_E: c->S[k] = c->p.s_e; break;
      case GRP_EPS: c->S[k] = c->p.s_eps; break;
      case GRP_Q: c->S[k] = c->p.s_q; break;
      case GRP_PI: c->S[k] = c->p.s_pi; break;
      case GRP_M: c->S[k] = c->p.s_m; break;
      default: c->S[k] = -1.0; (void)s_nu; break; /* -1 marks "viscous rate 1/tau" */
    }
  }
  return 0;
}

/* ------------------------------------------------------------- helpers */

static inline int64_t idx3(const orc_ctx* c, int x, int y, int z) {
  return (int64_t)x + (int64_t)c->p.nx * ((int64_t)y + (int64_t)c->p.ny * (int64_t)z);
}

/* Index of (x+dx, y+dy, z+dz) under periodicity per[]; -1 if outside the box. */
static int64_t nbr(const orc_ctx* c, int x, int y, int z, int dx, int dy, int dz, const int* per) {
  int X = x + dx, Y = y + dy, Z = z + dz;
  int n3[3] = {c->p.nx, c->p.ny, c->p.nz};
  int v[3] = {X, Y, Z};
  for (int a = 0; a < 3; ++a) {
    if (v[a] < 0 || v[a] >= n3[a]) {
      if (!per[a]) return -1;
      v[a] = ((v[a] % n3[a]) + n3[a]) % n3[a];
    }
  }
  return idx3(c, v[0], v[1], v[2]);
}

static inline void coords(const orc_ctx* c, int64_t n, int* x, int* y, int* z) {
  *x = (int)(n % c->p.nx);
  *y = (int)((n / c->p.nx) % c->p.ny);
  *z = (int)(n / ((int64_t)c->p.nx * c->p.ny));
}

/* Eq. 1.11 / pseudo-potential_multicomponent, or psi = rho */
static double psi_of(const orc_ctx* c, double rho) {
  if (c->p.psi_kind == 1) return rho;
  return c->p.rho0 * (1.0 - exp(-rho / c->p.rho0));
}

/* Eq. 6: f_i^eq = w_i rho (1 + u.c/cs2 + u_a u_b Q_iab / (2 cs2^2)),
   Q_iab = c_ia c_ib - cs2 delta_ab. */
static double feq(const lattice_t* L, int i, double rho, const double* u) {
  double cu = 0.0, uQu = 0.0;
  for (int a = 0; a < 3; ++a) cu += u[a] * (double)L->c[i][a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double Q = (double)(L->c[i][a] * L->c[i][b]) - (a == b ? L->cs2 : 0.0);
      uQu += u[a] * u[b] * Q;
    }
  return L->w[i] * rho * (1.0 + cu / L->cs2 + uQu / (2.0 * L->cs2 * L->cs2));
}

/* Eq. 1.21: F_i = w_i [c_ia / cs2 + (c_ia c_ib - cs2 delta_ab) u_b / cs2^2] F_a */
static double guo_term(const lattice_t* L, int i, const double* u, const double* F) {
  double s = 0.0;
  for (int a = 0; a < 3; ++a) {
    double t = (double)L->c[i][a] / L->cs2;
    for (int b = 0; b < 3; ++b) {
      double Q = (double)(L->c[i][a] * L->c[i][b]) - (a == b ? L->cs2 : 0.0);
      t += Q * u[b] / (L->cs2 * L->cs2);
    }
    s += t * F[a];
  }
  return L->w[i] * s;
}

/* Eq. therpopeq_species: h_i^eq = w_i C (1 + c_i.u / cs2) */
static double heq(const lattice_t* K, int i, double C, const double* u) {
  double cu = 0.0;
  for (int a = 0; a < 3; ++a) cu += u[a] * (double)K->c[i][a];
  return K->w[i] * C * (1.0 + cu / K->cs2);
}

/* ----------------------------------------------------------- lifecycle */

static void* zalloc(size_t n) { return calloc(n ? n : 1, 1); }

/* scalar lattices: the n_scal given ones, then the product lattice if there is one */
static inline int n_lat(const orc_ctx* c) { return c->p.n_scal + (c->p.product ? 1 : 0); }
static inline double tau_of(const orc_ctx* c, int s) { return s < c->p.n_scal ? c->p.tau_c[s] : c->p.tau_p; }
static inline double cin_of(const orc_ctx* c, int s) { return s < c->p.n_scal ? c->p.C_in[s] : c->p.C_in_p; }

/* monitor entry of scalar s for a per-scalar quantity: the product lattice has its own */
static int mon_of(const orc_ctx* c, int base, int s) {
  if (s < c->p.n_scal) return base + s;
  switch (base) {
    case ORC_MON_SPECIES: return ORC_MON_SPECIES_P;
    case ORC_MON_INFLOW: return ORC_MON_INFLOW_P;
    case ORC_MON_OUTFLOW: return ORC_MON_OUTFLOW_P;
    case ORC_MON_INJ_SPEC: return ORC_MON_INJ_SPEC_P;
    default: return ORC_MON_REM_SPEC_P;
  }
}

orc_ctx* orc_create(const orc_params* p, int* status) {
  int st = 0;
  if (!p || (p->dim != 2 && p->dim != 3) || p->nx < 1 || p->ny < 1 || p->nz < 1 ||
      (p->dim == 2 && p->nz != 1) || p->n_comp < 1 || p->n_comp > 2 || p->n_scal < 0 ||
      p->n_scal > 2 || p->N_geo < 1 || (p->collision == 1 && p->forcing == 1))
    st = -1;
  for (int s = 0; p && !st && s < p->n_comp; ++s)
    if (!(p->tau[s] > 0.5)) st = -1;
  for (int s = 0; p && !st && s < p->n_scal; ++s)
    if (!(p->tau_c[s] > 0.5)) st = -1;
  if (p && !st && p->n_scal > 0 && !(p->J0 >= 0.0 && p->J0 < 1.0)) st = -1;
  if (p && !st && p->ade_open_x && p->nx < 2) st = -1;
  /* a moving top plate needs a closed y axis and moves in its own plane */
  if (p && !st && (p->u_wall_ymax[0] != 0.0 || p->u_wall_ymax[1] != 0.0 || p->u_wall_ymax[2] != 0.0) &&
      (p->periodic[1] || p->u_wall_ymax[1] != 0.0))
    st = -1;
  /* the temperature-dependent rate needs the temperature as scalar 1, a positive temperature
     scale and a bounded iteration */
  if (p && !st && p->arrhenius &&
      (p->n_scal != 2 || !(p->arr_A >= 0.0) || !(p->arr_Ta >= 0.0) || p->n_it < 0 || p->n_it > 64))
    st = -1;
  /* conduction in the solid couples to the temperature scalar of the temperature-dependent mode */
  if (p && !st && p->conjugate &&
      (!p->arrhenius || !(p->tau_s > 0.5) || !(p->c_fs > 0.0) || p->geo_mode == 2))
    st = -1;
  /* the product needs the reacting scalar 0; deposition has no reaction to produce it */
  if (p && !st && p->product && (p->n_scal < 1 || !(p->tau_p > 0.5) || p->geo_mode == 2)) st = -1;
  /* the velocity inlet / zero-gradient outlet closes the x axis of the flow lattice, needs the
     channel walls on y, and is defined for one component without Shan-Chen forces */
  if (p && !st && p->flow_open_x &&
      (p->periodic[0] || p->periodic[1] || p->nx < 2 || p->n_comp != 1 || p->G[0][0] != 0.0 ||
       p->G_ads[0] != 0.0 || p->rho_solid != 0.0))
    st = -1;
  if (st) {
    if (status) *status = st;
    return NULL;
  }
  orc_ctx* c = (orc_ctx*)zalloc(sizeof(orc_ctx));
  c->p = *p;
  c->N = (int64_t)p->nx * p->ny * p->nz;
  make_lattices(c);
  c->per_c[0] = p->ade_open_x ? 0 : p->periodic[0];
  c->per_c[1] = p->periodic[1];
  c->per_c[2] = p->periodic[2];
  size_t N = (size_t)c->N;
  for (int s = 0; s < p->n_comp; ++s) {
    c->f[s] = (double*)zalloc(sizeof(double) * N * c->lf.q);
    c->fp[s] = (double*)zalloc(sizeof(double) * N * c->lf.q);
    c->rho[s] = (double*)zalloc(sizeof(double) * N);
    c->jm[s] = (double*)zalloc(sizeof(double) * N * 3);
    c->psi[s] = (double*)zalloc(sizeof(double) * N);
    c->F[s] = (double*)zalloc(sizeof(double) * N * 3);
  }
  for (int s = 0; s < n_lat(c); ++s) {
    c->h[s] = (double*)zalloc(sizeof(double) * N * c->lc.q);
    c->hc[s] = (double*)zalloc(sizeof(double) * N * c->lc.q);
    c->hp[s] = (double*)zalloc(sizeof(double) * N * c->lc.q);
    if (s == 1 && p->conjugate) {
      c->gs = (double*)zalloc(sizeof(double) * N * c->lc.q);
      c->gsp = (double*)zalloc(sizeof(double) * N * c->lc.q);
      c->kb = (double*)zalloc(sizeof(double) * N * c->lc.q);
      c->kb_ok = (uint8_t*)zalloc(N * c->lc.q);
    }
    c->Cs[s] = (double*)zalloc(sizeof(double) * N);
  }
  c->flag = (uint8_t*)zalloc(N);
  c->acc = (double*)zalloc(sizeof(double) * N);
  c->ub = (double*)zalloc(sizeof(double) * N * 3);
  c->snap_u = (double*)zalloc(sizeof(double) * N * 3);
  c->snap_C = (double*)zalloc(sizeof(double) * N);
  if (p->collision == 1 && build_mrt(c) != 0) {
    orc_destroy(c);
    if (status) *status = -2;
    return NULL;
  }
  if (status) *status = 0;
  return c;
}

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  for (int s = 0; s < 2; ++s) {
    free(c->f[s]); free(c->fp[s]); free(c->rho[s]); free(c->jm[s]); free(c->psi[s]); free(c->F[s]);
  }
  for (int s = 0; s < 3; ++s) {
    free(c->h[s]); free(c->hc[s]); free(c->hp[s]); free(c->Cs[s]);
  }
  free(c->gs); free(c->gsp); free(c->kb); free(c->kb_ok);
  free(c->flag); free(c->acc); free(c->ub); free(c->snap_u); free(c->snap_C);
  free(c);
}

int orc_set_geometry(orc_ctx* c, const uint8_t* flags) {
  for (int64_t n = 0; n < c->N; ++n) {
    if (flags[n] > 2) return -1;
  }
  memcpy(c->flag, flags, (size_t)c->N);
  for (int64_t n = 0; n < c->N; ++n) c->acc[n] = 0.0;
  return 0;
}

int orc_set_fields(orc_ctx* c, const double* rho, const double* u, const double* C) {
  int64_t N = c->N;
  int Qf = c->lf.q, Qc = c->lc.q;
  for (int64_t n = 0; n < N; ++n) {
    double un[3] = {u[n], u[N + n], c->p.dim == 3 ? u[2 * N + n] : 0.0};
    int fluid = (c->flag[n] == 0);
    for (int s = 0; s < c->p.n_comp; ++s)
      for (int i = 0; i < Qf; ++i) c->f[s][n * Qf + i] = fluid ? feq(&c->lf, i, rho[s * N + n], un) : 0.0;
    for (int s = 0; s < n_lat(c); ++s)
      for (int i = 0; i < Qc; ++i) c->h[s][n * Qc + i] = fluid ? heq(&c->lc, i, C[s * N + n], un) : 0.0;
    if (c->p.conjugate) {
      /* the solid starts at rest equilibrium with the temperature given for it */
      double zero[3] = {0.0, 0.0, 0.0};
      for (int i = 0; i < Qc; ++i) {
        c->gs[n * Qc + i] = fluid ? 0.0 : heq(&c->lc, i, C[N + n], zero);
        c->kb_ok[n * Qc + i] = 0;
        c->kb[n * Qc + i] = 0.0;
      }
    }
  }
  memset(c->mon, 0, sizeof(c->mon));
  c->t = 0;
  c->have_snap = 0;
  return 0;
}

/* ------------------------------------------------------ step, part B */

static int is_fluid_idx(const orc_ctx* c, int64_t m) { return m >= 0 && c->flag[m] == 0; }

/* rho^sigma, bare momentum, psi for all fluid nodes; then forces; then u^b. */
static void macros(orc_ctx* c) {
  int64_t N = c->N;
  int Qf = c->lf.q;
  const lattice_t* L = &c->lf;
  for (int64_t n = 0; n < N; ++n) {
    for (int s = 0; s < c->p.n_comp; ++s) {
      double r = 0.0, j[3] = {0.0, 0.0, 0.0};
      if (c->flag[n] == 0) {
        for (int i = 0; i < Qf; ++i) {
          double fi = c->f[s][n * Qf + i];
          r += fi;                                     /* Eq. 1.7 */
          for (int a = 0; a < 3; ++a) j[a] += (double)L->c[i][a] * fi;   /* Eq. 1.8 */
        }
      }
      c->rho[s][n] = r;
      for (int a = 0; a < 3; ++a) c->jm[s][n * 3 + a] = j[a];
      c->psi[s][n] = (c->flag[n] == 0) ? psi_of(c, r) : 0.0;
    }
  }
  double psi_wall = psi_of(c, c->p.rho_solid);
  for (int64_t n = 0; n < N; ++n) {
    int x, y, z;
    coords(c, n, &x, &y, &z);
    for (int s = 0; s < c->p.n_comp; ++s)
      for (int a = 0; a < 3; ++a) c->F[s][n * 3 + a] = 0.0;
    if (c->flag[n] != 0) continue;
    for (int s = 0; s < c->p.n_comp; ++s) {
      double Fs[3] = {0.0, 0.0, 0.0};
      /* Eq. 1.13 / 1.14: -psi^s(x) sum_s~ G_ss~ sum_i w_i psi^s~(x + c_i) c_i */
      for (int s2 = 0; s2 < c->p.n_comp; ++s2) {
        double Gss = c->p.G[s][s2];
        if (Gss == 0.0) continue;
        double sum[3] = {0.0, 0.0, 0.0};
        for (int i = 1; i < Qf; ++i) {
          int64_t m = nbr(c, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2], c->p.periodic);
          double ps = is_fluid_idx(c, m) ? c->psi[s2][m] : psi_wall;
          for (int a = 0; a < 3; ++a) sum[a] += L->w[i] * ps * (double)L->c[i][a];
        }
        for (int a = 0; a < 3; ++a) Fs[a] += -c->psi[s][n] * Gss * sum[a];
      }
      /* Eq. 1.15: -G_ads,s rho^s sum_i w_i s(x + c_i) c_i */
      if (c->p.G_ads[s] != 0.0) {
        double sum[3] = {0.0, 0.0, 0.0};
        for (int i = 1; i < Qf; ++i) {
          int64_t m = nbr(c, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2], c->p.periodic);
          double sw = is_fluid_idx(c, m) ? 0.0 : 1.0;
          for (int a = 0; a < 3; ++a) sum[a] += L->w[i] * sw * (double)L->c[i][a];
        }
        for (int a = 0; a < 3; ++a) Fs[a] += -c->p.G_ads[s] * c->rho[s][n] * sum[a];
      }
      /* external body force added to the SC force (Sec. 3.2.3) */
      for (int a = 0; a < 3; ++a) Fs[a] += c->rho[s][n] * c->p.g[a];
      for (int a = 0; a < 3; ++a) c->F[s][n * 3 + a] = Fs[a];
    }
    /* Eq. 1.19 / Shan_Chen_forcing_actual_velocity: u = sum_s (j^s + F^s/2) / rho */
    double rt = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int s = 0; s < c->p.n_comp; ++s) {
      rt += c->rho[s][n];                                         /* Eq. 1.20 */
      for (int a = 0; a < 3; ++a) m[a] += c->jm[s][n * 3 + a] + 0.5 * c->F[s][n * 3 + a];
    }
    for (int a = 0; a < 3; ++a) c->ub[n * 3 + a] = m[a] / rt;
  }
  for (int s = 0; s < n_lat(c); ++s)
    for (int64_t n = 0; n < N; ++n) {
      double C = 0.0;
      if (c->flag[n] == 0)
        for (int i = 0; i < c->lc.q; ++i) C += c->hc[s][n * c->lc.q + i];  /* Eq. macroreacb_species */
      c->Cs[s][n] = C;
    }
  if (c->p.conjugate)
    for (int64_t n = 0; n < N; ++n) {
      if (c->flag[n] == 0) continue;
      double T = 0.0;
      for (int i = 0; i < c->lc.q; ++i) T += c->gs[n * c->lc.q + i];
      c->Cs[1][n] = T;   /* the solid temperature (Eq. macroreacb_solid, per unit rho c_p) */
    }
}

/* ------------------------------------------------------ step, part C */

static void collide(orc_ctx* c) {
  int64_t N = c->N;
  int Qf = c->lf.q, Qc = c->lc.q;
  const lattice_t* L = &c->lf;
  for (int64_t n = 0; n < N; ++n) {
    if (c->flag[n] != 0) continue;
    const double* u = &c->ub[n * 3];
    if (c->p.forcing == 1) {
      /* Eq. 1.18: u' = sum_s rho^s u^s / tau^s / sum_s rho^s / tau^s (rho^s u^s = j^s) */
      double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
      for (int s = 0; s < c->p.n_comp; ++s) {
        for (int a = 0; a < 3; ++a) num[a] += c->jm[s][n * 3 + a] / c->p.tau[s];
        den += c->rho[s][n] / c->p.tau[s];
      }
      for (int s = 0; s < c->p.n_comp; ++s) {
        double ueq[3];
        for (int a = 0; a < 3; ++a)   /* Eq. 1.17 */
          ueq[a] = num[a] / den + c->p.tau[s] * c->F[s][n * 3 + a] / c->rho[s][n];
        for (int i = 0; i < Qf; ++i) {
          double fi = c->f[s][n * Qf + i];
          c->fp[s][n * Qf + i] = fi - (fi - feq(L, i, c->rho[s][n], ueq)) / c->p.tau[s];  /* Eq. 1.16, F_i = 0 */
        }
      }
    } else if (c->p.collision == 0) {
      for (int s = 0; s < c->p.n_comp; ++s) {
        const double* F = &c->F[s][n * 3];
        double tau = c->p.tau[s];
        for (int i = 0; i < Qf; ++i) {
          double fi = c->f[s][n * Qf + i];
          /* Eq. 1.16 with u^eq = u^b and F_i from Eq. 1.21 */
          c->fp[s][n * Qf + i] = fi - (fi - feq(L, i, c->rho[s][n], u)) / tau +
                                 (1.0 - 1.0 / (2.0 * tau)) * guo_term(L, i, u, F);
        }
      }
    } else {
      /* MRT: m* = m - S (m - m_eq) + (I - S/2) M F_i ;  f* = M^-1 m* */
      for (int s = 0; s < c->p.n_comp; ++s) {
        const double* F = &c->F[s][n * 3];
        double fv[QMAX], fe[QMAX], fF[QMAX], mp[QMAX];
        for (int i = 0; i < Qf; ++i) {
          fv[i] = c->f[s][n * Qf + i];
          fe[i] = feq(L, i, c->rho[s][n], u);
          fF[i] = guo_term(L, i, u, F);
        }
        for (int k = 0; k < Qf; ++k) {
          double m = 0.0, me = 0.0, mf = 0.0;
          for (int i = 0; i < Qf; ++i) {
            m += c->M[k][i] * fv[i];
            me += c->M[k][i] * fe[i];
            mf += c->M[k][i] * fF[i];
          }
          double rate = (c->S[k] < 0.0) ? 1.0 / c->p.tau[s] : c->S[k];
          mp[k] = m - rate * (m - me) + (1.0 - 0.5 * rate) * mf;
        }
        for (int i = 0; i < Qf; ++i) {
          double v = 0.0;
          for (int k = 0; k < Qf; ++k) v += c->Minv[i][k] * mp[k];
          c->fp[s][n * Qf + i] = v;
        }
      }
    }
    /* Eq. therpop_species with Eq. therpopeq_species, u = physical velocity */
    for (int s = 0; s < n_lat(c); ++s) {
      double C = c->Cs[s][n];
      for (int i = 0; i < Qc; ++i) {
        double hi = c->hc[s][n * Qc + i];
        c->hp[s][n * Qc + i] = hi - (hi - heq(&c->lc, i, C, u)) / tau_of(c, s);
      }
    }
  }
}

/* Eq. therpop_solid with Eq. therpopeq_solid: conduction in the solid, g_s^eq = w T_s */
static void collide_solid(orc_ctx* c) {
  if (!c->p.conjugate) return;
  int Qc = c->lc.q;
  double zero[3] = {0.0, 0.0, 0.0};
  for (int64_t n = 0; n < c->N; ++n) {
    if (c->flag[n] == 0) continue;
    const double T = c->Cs[1][n];
    for (int i = 0; i < Qc; ++i) {
      const double gi = c->gs[n * Qc + i];
      c->gsp[n * Qc + i] = gi - (gi - heq(&c->lc, i, T, zero)) / c->p.tau_s;
    }
  }
}

/* The exchange across a solid link (Sec. 2.1.5, Eq. tempCon, fluxCon, reacRate), after the
   streaming of every fluid population.  For fluid node n and direction i whose source
   s = n - c_i is solid, the fluid temperature population ho = h*_T,opp(i)(n) leaving n toward s
   and the solid population go = g*_s,i(s) leaving s toward n meet at one interface temperature
   T_b.  Each side receives 2 w T_b minus what it sent (anti-bounce-back on the common T_b), and
   the energy of the link, in units of the fluid's rho c_p, grows by the reaction heat Qp:
       (h_T,i - ho) + (g_s,opp(i) - go) / c_fs = Qp,
       h_T,i = 2 w T_b - ho,   g_s,opp(i) = 2 w T_b - go,
   so that T_b = (c_fs ho + go + c_fs Qp / 2) / (w (c_fs + 1)).  With c_fs = 1, tau_s = tau_T
   and Qp = 0 this is plain streaming (h_T,i = go, g_s,opp(i) = ho).  At a reactive link
   Qp = h_r k(T_b) C_b, the heat release of Eq. reacRate: ho and go are post-collision, so what
   the link adds to the populations in one step is the heat that crosses it, the physical flux
   that Eq. fluxCon balances (the factor tau / (tau - 1/2) of Eq. unknownpopTempS belongs to a
   closure written on pre-collision populations).  C_b = 2 hb / (2 w + k tau_c / (tau_c - 1/2))
   is the closure of the species population hb = h_C,opp(i)(n) that has just streamed in; T_b and C_b are solved
   together by n_it fixed-point iterations from the source-free T_b, and k is kept for the
   species closure of the next step, which then finds the same C_b. */
static void exchange_solid(orc_ctx* c) {
  if (!c->p.conjugate) return;
  int Qc = c->lc.q;
  const lattice_t* K = &c->lc;
  const double cf = c->p.c_fs;
  const double fc = c->p.tau_c[0] / (c->p.tau_c[0] - 0.5);
  for (int64_t n = 0; n < c->N; ++n) {
    if (c->flag[n] != 0) continue;
    int x, y, z;
    coords(c, n, &x, &y, &z);
    for (int i = 1; i < Qc; ++i) {
      int64_t src = nbr(c, x, y, z, -K->c[i][0], -K->c[i][1], -K->c[i][2], c->per_c);
      if (src < 0 || c->flag[src] == 0) continue;
      const double w = K->w[i];
      const double ho = c->hp[1][n * Qc + K->opp[i]];
      const double go = c->gsp[src * Qc + i];
      double Tb = (cf * ho + go) / (w * (cf + 1.0));
      double Qp = 0.0;
      if (c->flag[src] == 2) {
        const double hb = c->h[0][n * Qc + K->opp[i]];
        double k = 0.0;
        for (int it = 0; it <= c->p.n_it; ++it) {
          k = c->p.arr_A * exp(-c->p.arr_Ta / Tb);
          const double Cb = 2.0 * hb / (2.0 * w + k * fc);
          Qp = c->p.heat_release * k * Cb;
          Tb = (cf * ho + go + 0.5 * cf * Qp) / (w * (cf + 1.0));
        }
        c->kb[n * Qc + i] = k;
        c->kb_ok[n * Qc + i] = 1;
      }
      const double hin = 2.0 * w * Tb - ho;
      const double gin = 2.0 * w * Tb - go;
      c->h[1][n * Qc + i] = hin;
      c->gs[src * Qc + K->opp[i]] = gin;
      c->mon[ORC_MON_HEAT] += hin - ho;
      c->mon[ORC_MON_HEAT_S] += gin - go;
      c->mon[ORC_MON_HEAT_SRC] += Qp;
    }
  }
}

/* Streaming inside the solid; populations arriving from a fluid node were set by the exchange,
   closed faces reflect. */
static void stream_solid(orc_ctx* c) {
  if (!c->p.conjugate) return;
  int Qc = c->lc.q;
  const lattice_t* K = &c->lc;
  for (int64_t n = 0; n < c->N; ++n) {
    if (c->flag[n] == 0) continue;
    int x, y, z;
    coords(c, n, &x, &y, &z);
    for (int i = 0; i < Qc; ++i) {
      int64_t src = nbr(c, x, y, z, -K->c[i][0], -K->c[i][1], -K->c[i][2], c->per_c);
      if (src >= 0 && c->flag[src] == 0) continue;
      c->gs[n * Qc + i] = (src >= 0) ? c->gsp[src * Qc + i] : c->gsp[n * Qc + K->opp[i]];
    }
  }
}

/* ------------------------------------------------------ step, part D */

static void stream(orc_ctx* c) {
  int64_t N = c->N;
  int Qf = c->lf.q, Qc = c->lc.q;
  const lattice_t* L = &c->lf;
  const lattice_t* K = &c->lc;
  for (int64_t n = 0; n < N; ++n) {
    if (c->flag[n] != 0) continue;
    int x, y, z;
    coords(c, n, &x, &y, &z);
    for (int s = 0; s < c->p.n_comp; ++s)
      for (int i = 0; i < Qf; ++i) {
        int64_t src = nbr(c, x, y, z, -L->c[i][0], -L->c[i][1], -L->c[i][2], c->p.periodic);
        if (is_fluid_idx(c, src)) {
          c->f[s][n * Qf + i] = c->fp[s][src * Qf + i];          /* Eq. 5 */
        } else if (src < 0 && c->p.flow_open_x && x - L->c[i][0] < 0) {
          /* velocity inlet (Sec. 3.4): bounce-back off a face moving with the inlet profile
             u_x = 6 U s (1 - s), s = (y + 1/2) / ny, carrying 2 w rho (c . u) / c_s^2 */
          const double sy = ((double)y + 0.5) / (double)c->p.ny;
          const double ux = 6.0 * c->p.u_in * sy * (1.0 - sy);
          c->f[s][n * Qf + i] =
              c->fp[s][n * Qf + L->opp[i]] + 6.0 * L->w[i] * c->rho[s][n] * ((double)L->c[i][0] * ux);
        } else if (src < 0 && c->p.flow_open_x && x - L->c[i][0] >= c->p.nx) {
          /* zero-gradient outlet: f_i(nx-1) takes the post-collision f_i of the node itself,
             as the scalar outlet does */
          c->f[s][n * Qf + i] = c->fp[s][n * Qf + i];
        } else {
          double v = c->fp[s][n * Qf + L->opp[i]];                /* halfway bounce-back */
          if (src < 0 && y - L->c[i][1] >= c->p.ny) {
            /* moving top plate (Sec. 3.1.1): the reflected population carries the momentum
               exchange 2 w rho (c . u_wall) / c_s^2, c_s^2 = 1/3, rho the node's density */
            double cu = 0.0;
            for (int a = 0; a < 3; ++a) cu += (double)L->c[i][a] * c->p.u_wall_ymax[a];
            v += 6.0 * L->w[i] * c->rho[s][n] * cu;
          }
          c->f[s][n * Qf + i] = v;
        }
      }
    for (int s = 0; s < n_lat(c); ++s)
      for (int i = 0; i < Qc; ++i) {
        int64_t src = nbr(c, x, y, z, -K->c[i][0], -K->c[i][1], -K->c[i][2], c->per_c);
        double hout = c->hp[s][n * Qc + K->opp[i]];
        double hin;
        int xs = x - K->c[i][0];
        if (is_fluid_idx(c, src)) {
          hin = c->hp[s][src * Qc + i];
        } else if (src < 0 && c->p.ade_open_x && xs < 0) {
          /* inlet ghost at equilibrium with C_in and the node's own velocity */
          hin = heq(K, i, cin_of(c, s), &c->ub[n * 3]);
          c->mon[mon_of(c, ORC_MON_INFLOW, s)] += hin - hout;
        } else if (src < 0 && c->p.ade_open_x && xs >= c->p.nx) {
          /* zero-gradient outlet: h_i(nx-1) = h_i(nx-2) = own post-collision h_i */
          hin = c->hp[s][n * Qc + i];
          c->mon[mon_of(c, ORC_MON_OUTFLOW, s)] += hout - hin;
        } else {
          /* wall: bounce-back; at a reactive link of scalar 0 this value is
             replaced by the wet-node closure at the start of the next step, and at a
             solid link of the temperature with conduction in the solid, by the
             exchange that follows the streaming */
          hin = hout;
        }
        c->h[s][n * Qc + i] = hin;
      }
  }
}

/* Kang wet-node closure (Sec. 2.1.5, Eq. wetnode9) applied per link: for fluid
   node n and scalar-0 direction i whose source n - c_i is a reactive solid, the
   population h_i arriving from the wall is unknown after streaming.  With
   K = k tau_c / (tau_c - 1/2) and hb the gathered population moving toward the
   wall (direction opposite to i):
       C_b = 2 hb / (2 w_i + K),   h_i = 2 w_i C_b - hb.
   For D2Q5 with J0 = 0.4, 2 w_i = (1 - J0)/2, the printed denominator.  Every
   closure of a node reads the values before any closure.  dst gets the closed
   populations of node n.  When book != 0 the reaction rate k C_b of each link is
   added to acc of that solid node and to the reacted total, and the stored-minus-
   closed value (what left the lattice through the link) to the wall exchange. */
static void close_node(orc_ctx* c, int s, int64_t n, double* dst, int book, double* rl) {
  int Qc = c->lc.q;
  const lattice_t* K = &c->lc;
  const double* hs = &c->h[s][n * Qc];
  for (int i = 0; i < Qc; ++i) dst[i] = hs[i];
  if (s != 0 || c->flag[n] != 0) return;
  double Kr = c->p.k_react * c->p.tau_c[0] / (c->p.tau_c[0] - 0.5);
  int x, y, z;
  coords(c, n, &x, &y, &z);
  for (int i = 1; i < Qc; ++i) {
    int64_t src = nbr(c, x, y, z, -K->c[i][0], -K->c[i][1], -K->c[i][2], c->per_c);
    if (src < 0 || c->flag[src] != 2) continue;
    double hb = hs[K->opp[i]];
    double Cb = 2.0 * hb / (2.0 * K->w[i] + Kr);
    double hin = 2.0 * K->w[i] * Cb - hb;
    dst[i] = hin;
    if (rl) rl[i] = c->p.k_react * Cb;
    if (book) {
      /* reaction rate at the wall, Eq. reactO2: k C_b (= (1 - 1/(2 tau_c)) (hb - h_i)) */
      double r = c->p.k_react * Cb;
      c->acc[src] += r;
      c->mon[ORC_MON_REACTED] += r;
      /* populations that left the lattice through this link (closes the species budget) */
      c->mon[ORC_MON_WALLX] += hs[i] - hin;
    }
  }
}

/* Reactive link with a temperature-dependent rate and heat release (Sec. 2.1.5): scalar 0 is
   the reacting species (C), scalar 1 the temperature (T).  At a link whose source n - c_i is a
   reactive solid, with hb, gb the gathered C and T populations moving toward the wall and w the
   link weight, the interface values satisfy
       C_b = 2 hb / (2 w + k(T_b) tau_c / (tau_c - 1/2)),      k(T) = A exp(-Ta / T)  (Eq. reactO2)
       Q   = h_r k(T_b) C_b                                                             (Eq. reacRate)
       T_b = (2 gb + Q tau_T / (tau_T - 1/2)) / (2 w),
   the last from the same per-link wet-node ansatz as the species closure: h_T,i + gb = 2 w T_b
   and (1 - 1/(2 tau_T)) (h_T,i - gb) = Q, the heat flux entering the fluid through the link
   (Eq. fluxCon with an adiabatic solid).  The coupled pair is solved by n_it fixed-point
   iterations from the zero-flux value T_b = gb / w; then
       h_C,i = 2 w C_b - hb,      h_T,i = gb + Q tau_T / (tau_T - 1/2). */
static void close_node_thermal(orc_ctx* c, int64_t n, double* dst0, double* dst1, int book,
                               double* rl) {
  int Qc = c->lc.q;
  const lattice_t* K = &c->lc;
  const double* h0 = &c->h[0][n * Qc];
  const double* h1 = &c->h[1][n * Qc];
  for (int i = 0; i < Qc; ++i) {
    dst0[i] = h0[i];
    dst1[i] = h1[i];
  }
  if (c->flag[n] != 0) return;
  const double fc = c->p.tau_c[0] / (c->p.tau_c[0] - 0.5);
  const double fT = c->p.tau_c[1] / (c->p.tau_c[1] - 0.5);
  int x, y, z;
  coords(c, n, &x, &y, &z);
  for (int i = 1; i < Qc; ++i) {
    int64_t src = nbr(c, x, y, z, -K->c[i][0], -K->c[i][1], -K->c[i][2], c->per_c);
    if (src < 0 || c->flag[src] != 2) continue;
    const double w = K->w[i];
    const double hb = h0[K->opp[i]];
    const double gb = h1[K->opp[i]];
    double Tb = gb / w;
    for (int it = 0; it < c->p.n_it; ++it) {
      const double k = c->p.arr_A * exp(-c->p.arr_Ta / Tb);
      const double Cb = 2.0 * hb / (2.0 * w + k * fc);
      const double Q = c->p.heat_release * k * Cb;
      Tb = (2.0 * gb + Q * fT) / (2.0 * w);
    }
    const double k = c->p.arr_A * exp(-c->p.arr_Ta / Tb);
    const double Cb = 2.0 * hb / (2.0 * w + k * fc);
    const double Q = c->p.heat_release * k * Cb;
    dst0[i] = 2.0 * w * Cb - hb;
    dst1[i] = gb + Q * fT;
    rl[i] = k * Cb;
    if (book) {
      const double r = k * Cb;
      c->acc[src] += r;
      c->mon[ORC_MON_REACTED] += r;
      c->mon[ORC_MON_WALLX] += h0[i] - dst0[i];
      c->mon[ORC_MON_HEAT] += dst1[i] - h1[i];
    }
  }
}

/* Species closure with conduction in the solid: the wet-node closure of close_node at each
   reactive link, with the rate constant k(T_b) that the link's last exchange (exchange_solid)
   found together with C_b; before a link's first exchange k is taken at the heat-capacity-
   weighted mean of the two sides' temperatures.  The heat of the reaction was put into the
   temperature fields by that exchange, so the closure leaves the temperature unchanged. */
static void close_node_conjugate(orc_ctx* c, int64_t n, double* dst0, double* dst1, int book,
                                 double* rl) {
  int Qc = c->lc.q;
  const lattice_t* K = &c->lc;
  const double* h0 = &c->h[0][n * Qc];
  const double* h1 = &c->h[1][n * Qc];
  for (int i = 0; i < Qc; ++i) {
    dst0[i] = h0[i];
    dst1[i] = h1[i];
  }
  if (c->flag[n] != 0) return;
  const double fc = c->p.tau_c[0] / (c->p.tau_c[0] - 0.5);
  int x, y, z;
  coords(c, n, &x, &y, &z);
  for (int i = 1; i < Qc; ++i) {
    int64_t src = nbr(c, x, y, z, -K->c[i][0], -K->c[i][1], -K->c[i][2], c->per_c);
    if (src < 0 || c->flag[src] != 2) continue;
    double k = c->kb[n * Qc + i];
    if (!c->kb_ok[n * Qc + i]) {
      double Tf = 0.0, Ts = 0.0;
      for (int j = 0; j < Qc; ++j) {
        Tf += h1[j];
        Ts += c->gs[src * Qc + j];
      }
      k = c->p.arr_A * exp(-c->p.arr_Ta / ((c->p.c_fs * Tf + Ts) / (c->p.c_fs + 1.0)));
    }
    const double w = K->w[i];
    const double hb = h0[K->opp[i]];
    const double Cb = 2.0 * hb / (2.0 * w + k * fc);
    dst0[i] = 2.0 * w * Cb - hb;
    rl[i] = k * Cb;
    if (book) {
      const double r = k * Cb;
      c->acc[src] += r;
      c->mon[ORC_MON_REACTED] += r;
      c->mon[ORC_MON_WALLX] += h0[i] - dst0[i];
    }
  }
}

/* The product of the surface reaction (Sec. 2.1.5, Eq. react, reactCO2): at each reactive link
   the product enters the fluid at the rate the reaction takes scalar 0, r = k C_b of that link.
   The same per-link wet-node ansatz as the species closure, with the sign of the flux reversed,
   (1 - 1/(2 tau_p)) (h_P,i - h_P,opp(i)) = r, gives h_P,i = h_P,opp(i) + r tau_p / (tau_p - 1/2).
   rl holds the link rates of scalar 0 from its closure at this node. */
static void close_node_product(orc_ctx* c, int64_t n, double* dst, int book, const double* rl) {
  int Qc = c->lc.q;
  const lattice_t* K = &c->lc;
  const double* hs = &c->h[c->p.n_scal][n * Qc];
  for (int i = 0; i < Qc; ++i) dst[i] = hs[i];
  if (c->flag[n] != 0) return;
  const double fp = c->p.tau_p / (c->p.tau_p - 0.5);
  int x, y, z;
  coords(c, n, &x, &y, &z);
  for (int i = 1; i < Qc; ++i) {
    int64_t src = nbr(c, x, y, z, -K->c[i][0], -K->c[i][1], -K->c[i][2], c->per_c);
    if (src < 0 || c->flag[src] != 2) continue;
    dst[i] = hs[K->opp[i]] + rl[i] * fp;
    if (book) c->mon[ORC_MON_PRODUCED] += dst[i] - hs[i];
  }
}

/* Every scalar closure of node n, into dst[s] for each scalar lattice s. */
static void close_node_all(orc_ctx* c, int64_t n, double* const* dst, int book) {
  double rl[QMAX];
  for (int i = 0; i < QMAX; ++i) rl[i] = 0.0;
  if (c->p.conjugate) {
    close_node_conjugate(c, n, dst[0], dst[1], book, rl);
  } else if (c->p.arrhenius) {
    close_node_thermal(c, n, dst[0], dst[1], book, rl);
  } else {
    for (int s = 0; s < c->p.n_scal; ++s) close_node(c, s, n, dst[s], book, s == 0 ? rl : NULL);
  }
  if (c->p.product) close_node_product(c, n, dst[c->p.n_scal], book, rl);
}

static void close_all(orc_ctx* c, int book) {
  int Qc = c->lc.q;
  for (int64_t n = 0; n < c->N; ++n) {
    double* dst[3] = {NULL, NULL, NULL};
    for (int s = 0; s < n_lat(c); ++s) dst[s] = &c->hc[s][n * Qc];
    close_node_all(c, n, dst, book);
  }
}

/* ---------------------------------------------- step, part A and E */

static int scalar_link_is_wall(const orc_ctx* c, int x, int y, int z, int i) {
  const lattice_t* K = &c->lc;
  int64_t m = nbr(c, x, y, z, K->c[i][0], K->c[i][1], K->c[i][2], c->per_c);
  if (m >= 0) return c->flag[m] != 0;
  int xs = x + K->c[i][0];
  if (c->p.ade_open_x && (xs < 0 || xs >= c->p.nx)) return 0;  /* open face */
  return 1;
}

static void deposit(orc_ctx* c) {
  if (c->p.geo_mode != 2 || c->p.n_scal < 1) return;
  int Qc = c->lc.q;
  for (int64_t n = 0; n < c->N; ++n) {
    if (c->flag[n] != 0) continue;
    int x, y, z;
    coords(c, n, &x, &y, &z);
    int near = 0;
    for (int i = 1; i < Qc; ++i) near |= scalar_link_is_wall(c, x, y, z, i);
    if (!near) continue;
    /* Eq. surface_deposition: C_p,s += DP sum_i h_p,i */
    double sum = 0.0;
    for (int i = 0; i < Qc; ++i) sum += c->hc[0][n * Qc + i];
    double dep = c->p.DP * sum;
    c->acc[n] += dep;
    c->mon[ORC_MON_DEPOSITED] += dep;
    if (c->p.deposit_conservative)
      for (int i = 0; i < Qc; ++i) c->hc[0][n * Qc + i] *= (1.0 - c->p.DP);
  }
}

static void flips(orc_ctx* c) {
  if (c->p.geo_mode == 0 || ((c->t + 1) % c->p.N_geo) != 0) return;
  int64_t N = c->N;
  int Qf = c->lf.q, Qc = c->lc.q;
  const lattice_t* L = &c->lf;
  int64_t* list = (int64_t*)zalloc(sizeof(int64_t) * (size_t)N);
  int64_t cnt = 0;
  /* a reactive node has consumed its solid mass once V_m acc >= m_s0: the remaining mass
     m_s0 - V_m acc has reached zero (solid consumption, Sec. 2.1.5) */
  for (int64_t n = 0; n < N; ++n) {
    if (c->p.geo_mode == 1 && c->flag[n] == 2 && c->p.V_m * c->acc[n] >= c->p.m_s0) list[cnt++] = n;
    if (c->p.geo_mode == 2 && c->flag[n] == 0 && c->acc[n] > 1.0) list[cnt++] = n;
  }
  if (c->p.geo_mode == 1) {
    /* dissolution: new fluid node at rest equilibrium with the mean density and
       concentration of its fluid neighbours (values after this step's streaming) */
    /* per new node: the mean density of each component, then the mean of each scalar */
    double* mean = (double*)zalloc(sizeof(double) * (size_t)(cnt * 5 + 1));
    int* ok = (int*)zalloc(sizeof(int) * (size_t)(cnt + 1));
    for (int64_t k = 0; k < cnt; ++k) {
      int64_t n = list[k];
      int x, y, z;
      coords(c, n, &x, &y, &z);
      double sr[2] = {0.0, 0.0}, sc[3] = {0.0, 0.0, 0.0};
      int m_count = 0;
      for (int i = 1; i < Qf; ++i) {
        int64_t m = nbr(c, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2], c->p.periodic);
        if (!is_fluid_idx(c, m)) continue;
        m_count++;
        for (int s = 0; s < c->p.n_comp; ++s) {
          double r = 0.0;
          for (int j = 0; j < Qf; ++j) r += c->f[s][m * Qf + j];
          sr[s] += r;
        }
        /* the neighbour's scalars after its closure (the same closure the step applies) */
        double hm[3][QMAX];
        double* dst[3] = {hm[0], hm[1], hm[2]};
        close_node_all(c, m, dst, 0);
        for (int s = 0; s < n_lat(c); ++s) {
          double C = 0.0;
          for (int j = 0; j < Qc; ++j) C += hm[s][j];
          sc[s] += C;
        }
      }
      ok[k] = m_count > 0;
      for (int s = 0; s < 2; ++s) mean[k * 5 + s] = m_count ? sr[s] / (double)m_count : 0.0;
      for (int s = 0; s < 3; ++s) mean[k * 5 + 2 + s] = m_count ? sc[s] / (double)m_count : 0.0;
    }
    double zero[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k < cnt; ++k) {
      if (!ok[k]) continue;
      int64_t n = list[k];
      for (int s = 0; s < c->p.n_comp; ++s) {
        double r = mean[k * 5 + s];
        for (int i = 0; i < Qf; ++i) c->f[s][n * Qf + i] = feq(L, i, r, zero);
        c->mon[ORC_MON_INJ_MASS + s] += r;
      }
      for (int s = 0; s < n_lat(c); ++s) {
        double C = mean[k * 5 + 2 + s];
        if (s == 1 && c->p.conjugate) {
          /* with conduction in the solid the node keeps its own temperature; its solid
             populations leave the solid lattice */
          C = 0.0;
          for (int i = 0; i < Qc; ++i) {
            C += c->gs[n * Qc + i];
            c->gs[n * Qc + i] = 0.0;
          }
          c->mon[ORC_MON_SOLID_REM] += C;
        }
        for (int i = 0; i < Qc; ++i) c->h[s][n * Qc + i] = heq(&c->lc, i, C, zero);
        c->mon[mon_of(c, ORC_MON_INJ_SPEC, s)] += C;
      }
      c->flag[n] = 0;
    }
    free(mean);
    free(ok);
  } else {
    /* deposition: node becomes an inert solid; its populations are removed */
    for (int64_t k = 0; k < cnt; ++k) {
      int64_t n = list[k];
      for (int s = 0; s < c->p.n_comp; ++s) {
        double r = 0.0;
        for (int i = 0; i < Qf; ++i) {
          r += c->f[s][n * Qf + i];
          c->f[s][n * Qf + i] = 0.0;
        }
        c->mon[ORC_MON_REM_MASS + s] += r;
      }
      for (int s = 0; s < n_lat(c); ++s) {
        double C = 0.0;
        for (int i = 0; i < Qc; ++i) {
          C += c->h[s][n * Qc + i];
          c->h[s][n * Qc + i] = 0.0;
        }
        c->mon[mon_of(c, ORC_MON_REM_SPEC, s)] += C;
      }
      c->flag[n] = 1;
    }
  }
  free(list);
}

int orc_step(orc_ctx* c, int64_t nsteps) {
  for (int64_t k = 0; k < nsteps; ++k) {
    close_all(c, 1);
    deposit(c);
    macros(c);
    collide(c);
    collide_solid(c);
    stream(c);
    exchange_solid(c);
    stream_solid(c);
    flips(c);
    c->t += 1;
  }
  return 0;
}

/* ------------------------------------------------------------ queries */

int orc_get_fields(orc_ctx* c, double* rho, double* u, double* C, uint8_t* flags, double* acc) {
  close_all(c, 0);
  macros(c);
  int64_t N = c->N;
  for (int64_t n = 0; n < N; ++n) {
    for (int s = 0; s < c->p.n_comp; ++s)
      if (rho) rho[s * N + n] = c->rho[s][n];
    if (u)
      for (int a = 0; a < 3; ++a) u[a * N + n] = (c->flag[n] == 0) ? c->ub[n * 3 + a] : 0.0;
    for (int s = 0; s < n_lat(c); ++s)
      if (C) C[s * N + n] = c->Cs[s][n];
    if (flags) flags[n] = c->flag[n];
    if (acc) acc[n] = c->acc[n];
  }
  return 0;
}

int orc_get_pops(orc_ctx* c, double* f, double* h) {
  int64_t N = c->N;
  int Qf = c->lf.q, Qc = c->lc.q;
  for (int s = 0; s < c->p.n_comp; ++s)
    for (int i = 0; i < Qf; ++i)
      for (int64_t n = 0; n < N; ++n)
        if (f) f[((int64_t)s * Qf + i) * N + n] = c->f[s][n * Qf + i];
  for (int s = 0; s < n_lat(c); ++s)
    for (int i = 0; i < Qc; ++i)
      for (int64_t n = 0; n < N; ++n)
        if (h) h[((int64_t)s * Qc + i) * N + n] = c->h[s][n * Qc + i];
  return 0;
}

int orc_set_pops(orc_ctx* c, const double* f, const double* h) {
  int64_t N = c->N;
  int Qf = c->lf.q, Qc = c->lc.q;
  for (int s = 0; s < c->p.n_comp; ++s)
    for (int i = 0; i < Qf; ++i)
      for (int64_t n = 0; n < N; ++n)
        if (f) c->f[s][n * Qf + i] = f[((int64_t)s * Qf + i) * N + n];
  for (int s = 0; s < n_lat(c); ++s)
    for (int i = 0; i < Qc; ++i)
      for (int64_t n = 0; n < N; ++n)
        if (h) c->h[s][n * Qc + i] = h[((int64_t)s * Qc + i) * N + n];
  return 0;
}

int orc_get_monitors(orc_ctx* c, double* out) {
  int64_t N = c->N;
  int Qf = c->lf.q, Qc = c->lc.q;
  const lattice_t* L = &c->lf;
  double mass[2] = {0.0, 0.0}, mom[3] = {0.0, 0.0, 0.0}, spec[3] = {0.0, 0.0, 0.0};
  double nsolid = 0.0, nfluid = 0.0, nonfinite = 0.0;
  for (int64_t n = 0; n < N; ++n) {
    if (c->flag[n] != 0) {
      nsolid += 1.0;
      continue;
    }
    nfluid += 1.0;
    int bad = 0;
    for (int s = 0; s < c->p.n_comp; ++s)
      for (int i = 0; i < Qf; ++i) {
        double fi = c->f[s][n * Qf + i];
        mass[s] += fi;
        for (int a = 0; a < 3; ++a) mom[a] += (double)L->c[i][a] * fi;
        if (!isfinite(fi)) bad = 1;
      }
    for (int s = 0; s < n_lat(c); ++s)
      for (int i = 0; i < Qc; ++i) {
        double hi = c->h[s][n * Qc + i];
        spec[s] += hi;
        if (!isfinite(hi)) bad = 1;
      }
    nonfinite += bad;
  }
  for (int k = 0; k < ORC_MON_COUNT; ++k) out[k] = c->mon[k];
  out[ORC_MON_STEP] = (double)c->t;
  for (int s = 0; s < 2; ++s) out[ORC_MON_MASS + s] = mass[s];
  for (int a = 0; a < 3; ++a) out[ORC_MON_MOM + a] = mom[a];
  for (int s = 0; s < n_lat(c); ++s) out[mon_of(c, ORC_MON_SPECIES, s)] = spec[s];
  out[ORC_MON_NSOLID] = nsolid;
  out[ORC_MON_NFLUID] = nfluid;
  out[ORC_MON_NONFINITE] = nonfinite;
  double ts = 0.0;
  if (c->p.conjugate)
    for (int64_t n = 0; n < N; ++n)
      if (c->flag[n] != 0)
        for (int i = 0; i < Qc; ++i) ts += c->gs[n * Qc + i];
  out[ORC_MON_TSOLID] = ts;
  return 0;
}

double orc_residual(orc_ctx* c) {
  close_all(c, 0);
  macros(c);
  int64_t N = c->N;
  double du = 0.0, nu = 0.0, dc = 0.0, nc = 0.0;
  for (int64_t n = 0; n < N; ++n) {
    if (c->flag[n] != 0) continue;
    for (int a = 0; a < 3; ++a) {
      double v = c->ub[n * 3 + a];
      double d = v - c->snap_u[n * 3 + a];
      du += d * d;
      nu += v * v;
      c->snap_u[n * 3 + a] = v;
    }
    if (c->p.n_scal > 0) {
      double v = c->Cs[0][n];
      double d = v - c->snap_C[n];
      dc += d * d;
      nc += v * v;
      c->snap_C[n] = v;
    }
  }
  int first = !c->have_snap;
  c->have_snap = 1;
  if (first) return -1.0;
  double r = (nu > 0.0) ? sqrt(du / nu) : 0.0;
  if (nc > 0.0) {
    double rc = sqrt(dc / nc);
    if (rc > r) r = rc;
  }
  return r;
}

int orc_get_mrt(orc_ctx* c, double* M, double* S) {
  int Q = c->lf.q;
  if (c->p.collision != 1) return -1;
  for (int k = 0; k < Q; ++k) {
    for (int i = 0; i < Q; ++i) M[k * Q + i] = c->M[k][i];
    S[k] = c->S[k];
  }
  return 0;
}

int orc_lattice(orc_ctx* c, int which, int* q, int* cvec, double* w) {
  const lattice_t* L = which ? &c->lc : &c->lf;
  *q = L->q;
  for (int i = 0; i < L->q; ++i) {
    for (int a = 0; a < 3; ++a) cvec[i * 3 + a] = L->c[i][a];
    w[i] = L->w[i];
  }
  return 0;
}
