// kernels.cuh -- sm_103a kernels of the reactive multi-component LBM step.
//
// Storage: structure of arrays, one plane per direction, pop[i * pitch + slot[n]], node
// n = x + nx*(y + ny*z).  The slot map puts the fluid nodes first, in list order, so a warp's
// lanes touch consecutive slots in every plane and no cache line carries solid-node bytes; the
// cells named (n, i) below are pop[i * pitch + slot[n]].
// Every lattice keeps ONE copy of its populations and streams in place with the A-A pattern:
//   even steps (parity 0) read f_i(n) from slot (n, i) and write the post-collision f*_i to
//   slot (n, opp i); odd steps (parity 1) read f_i(n) from (n - c_i, opp i) and write f*_i to
//   (n + c_i, i).  A population that meets a wall is written to (n, opp i) at either parity
//   (halfway bounce-back), and read back from (n, i).  Each slot is read and then written by
//   the same thread within a step, so one pass reads and writes every population exactly once.
// After an even number of steps the layout is natural (f_i(n) at (n, i)); after an odd number
// it is swapped.  Every reader of the state (moments, monitors, flips, checkpoints) follows
// the same rule.
//
// The reactive wet-node closure of scalar 0 (Eq. wetnode9) is applied when a node gathers its
// populations: the stored value of a reactive link is the bounce-back value, and the closure
// computes the unknown population from the gathered one moving toward the wall.
//
// Populations are stored as deviations from w_i * ref (ref = 0 in FP64 mode, the configured
// reference density / concentration otherwise), and the collision works on deviations, so
// the large w_i * ref part never enters a difference in reduced precision.  All parameter
// arithmetic is done on the host (Coef<T>): the kernels see only compute-type constants.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

#include "lattice.cuh"

namespace lbm {

// ------------------------------------------------------------------ storage

template <class S>
struct Store;
template <>
struct Store<double> {
  using T = double;
  __device__ static T ld(const double* p) { return __ldg(p); }
  __device__ static T ldv(const double* p) { return *p; }
  __device__ static void st(double* p, T v) { *p = v; }
};
template <>
struct Store<float> {
  using T = float;
  __device__ static T ld(const float* p) { return __ldg(p); }
  __device__ static T ldv(const float* p) { return *p; }
  __device__ static void st(float* p, T v) { *p = v; }
};
template <>
struct Store<__half> {
  using T = float;
  __device__ static T ld(const __half* p) { return __half2float(__ldg(p)); }
  __device__ static T ldv(const __half* p) { return __half2float(*p); }
  __device__ static void st(__half* p, T v) { *p = __float2half_rn(v); }
};
template <>
struct Store<__nv_bfloat16> {
  using T = float;
  __device__ static T ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  __device__ static T ldv(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ static void st(__nv_bfloat16* p, T v) { *p = __float2bfloat16_rn(v); }
};

// Mixed storage: 16-bit flow populations with the scalar lattices in FP32.  The tag types are
// the flow's storage element (2 bytes, loaded and stored like the plain 16-bit types); the scalar
// lattices of every storage type S are stored as ScalarOf<S>.
struct half_s32 {
  __half v;
};
struct bf16_s32 {
  __nv_bfloat16 v;
};
template <>
struct Store<half_s32> {
  using T = float;
  __device__ static T ld(const half_s32* p) { return __half2float(__ldg(&p->v)); }
  __device__ static T ldv(const half_s32* p) { return __half2float(p->v); }
  __device__ static void st(half_s32* p, T v) { p->v = __float2half_rn(v); }
};
template <>
struct Store<bf16_s32> {
  using T = float;
  __device__ static T ld(const bf16_s32* p) { return __bfloat162float(__ldg(&p->v)); }
  __device__ static T ldv(const bf16_s32* p) { return __bfloat162float(p->v); }
  __device__ static void st(bf16_s32* p, T v) { p->v = __float2bfloat16_rn(v); }
};
template <class S>
struct ScalarOf {
  using type = S;
};
template <>
struct ScalarOf<half_s32> {
  using type = float;
};
template <>
struct ScalarOf<bf16_s32> {
  using type = float;
};

// ------------------------------------------------------------- arguments

enum : int { ERR_CAPACITY = 1, ERR_NONFINITE = 2, ERR_CAS = 4, ERR_BOUNDS = 8 };
enum : int { GEO_NONE = 0, GEO_DISSOLVE = 1, GEO_DEPOSIT = 2 };
enum : uint8_t { FL_FLUID = 0, FL_SOLID = 1, FL_REACTIVE = 2, FL_FLIPPING = 3 };

// Floor division by a fixed divisor d through a rounded-up reciprocal (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): with l = ceil(log2 d) and
// M = ceil(2^(31 + l) / d), floor(n / d) = (n * M) >> (31 + l) for every n < 2^31 and
// 1 <= d < 2^31.  The host builds M and the shift and checks them at every quotient boundary.
struct FastDiv {
  uint32_t M;
  int sh;
};
__host__ __device__ __forceinline__ unsigned int fast_div(unsigned int n, FastDiv d) {
  return (unsigned int)(((unsigned long long)n * d.M) >> d.sh);
}

// Everything a kernel needs, in double; kernels convert to their compute type.
struct Args {
  void* f[2];
  void* h[3];                // scalar lattices: the given scalars, then the reaction product (if any)
  void* fplane[2][19];       // base pointer of every population plane (host-computed)
  void* hplane[3][7];
  void* psi[2];              // compute-type psi per component (Shan-Chen only)
  uint8_t* flags;
  uint32_t* mask;
  double* acc;               // consumed (reactive solid) / deposited (fluid) per node
  uint32_t* fluid_list;       // fluid node indices (sorted at each rebuild, appended by flips)
  unsigned int* fluid_count;  // [0] list length, [1] length at the last rebuild (see slot)
  // Storage slot of every node: populations of node n live at plane * pitch + slot[n].  Each
  // rebuild renumbers the fluid nodes to slots 0 .. F-1 in list order (so list entry e < F has
  // slot e) and the solid nodes to F .. N-1; nodes that become fluid later keep their slot.
  uint32_t* slot;
  uint32_t* slot_new;         // rebuild scratch
  unsigned int* block_counts; // ordered-compaction scratch [chunks + 1]
  unsigned int* block_counts_v;   // the same for the in-domain positions of the fluid-list order
  double* wallx_slot;        // [NBANKS][WALLX_SLOTS] wall-exchange accumulators
  uint32_t* iface_list;       // reactive solids with a fluid scalar-lattice neighbour
  unsigned int* iface_count;
  uint8_t* listed;           // 1 once a node is in iface_list
  uint32_t* flip_list;
  unsigned int* flip_count;
  unsigned int flip_cap;
  double* flip_scratch;      // [flip_cap][5]: new node's mean density (2) and scalars (3)
  double* flip_mon;          // [11] inj_mass[2], inj_spec[3], rem_mass[2], rem_spec[3], solid_rem
  int* err;
  double* inflow_row;        // [3][rows]
  double* outflow_row;       // [3][rows]
  double* partials;          // monitor partial sums [blocks][NMON]
  double* mon_out;           // [NMON]
  double* d_rho;             // FP64 staging [n_comp][N]
  double* d_u;               // [3][N]
  double* d_C;               // [n_scal][N]
  void* snap;                // compute-type residual snapshots [4][pitch] by slot: u_x, u_y, u_z, C
  long long pitch;           // elements per population plane (>= N, multiple of 32)
  long long N;
  int nx, ny, nz;
  int n_comp, n_scal;        // n_scal: scalar lattices, the product included
  int product;               // the last scalar lattice is the reaction product (Eq. reactCO2)
  int per[3];                // flow periodicity
  int open_x;                // scalar inlet / outlet on the x faces
  int sc_on, ads_on, shift_forcing, psi_identity;
  int geo_mode, deposit_conservative;
  double tau[2], G[2][2], G_ads[2], psi_wall, rho0, g[3];
  double s_grp[5];           // MRT rates: e, eps, q, pi, m
  double tau_c[3], J0, k_react, C_in[3];
  double V_m, m_s0, DP;
  double rho_ref[2], C_ref[3];
  int bx, by;                // step-kernel block shape
  FastDiv div_x, div_y;      // node index / nx, (node index / nx) / ny
  double u_wall[3];          // velocity of the top plate beyond y = ny - 1
  int moving_wall;           // the top plate moves (closed y axis)
  int flow_open_x;           // flow velocity inlet at x = 0, zero-gradient outlet at x = nx - 1
  double* u_in_row;          // [ny] inlet velocity u_x(y)
  int voff_ok;               // 3 * pitch < 2^31: wall links can be addressed by 32-bit offsets
  int arrhenius;             // scalar 1 is the temperature: rate k(T_b), reaction heat into T
  int n_it;                  // fixed-point iterations of the C_b - T_b coupling per link
  double arr_A, arr_Ta, heat_release;
  // conduction in the solid (with arrhenius): the solid thermal lattice in two compute-type
  // buffers [QC][N] by node (full values); step t reads gs[t & 1] and writes gs[(t + 1) & 1]
  int conjugate;
  double tau_s, c_fs;
  void* gs[2];
  void* kb;                  // compute-type [QC - 1][N]: k(T_b) of the link arriving in
                             // direction j at node n from the last exchange; NaN before one
};

// Index guard of the bounds-checked build (-DLBM_BOUNDS_CHECK): an index outside [0, bound)
// sets ERR_BOUNDS and is replaced by 0, so the access stays inside its buffer.  In normal
// builds LBM_CHK is the bare index expression and the generated code is unchanged.
#ifdef LBM_BOUNDS_CHECK
__device__ __forceinline__ long long chk_index(int* err, long long i, long long bound) {
  if (i < 0 || i >= bound) {
    atomicOr(err, ERR_BOUNDS);
    return 0;
  }
  return i;
}
#define LBM_CHK(err, i, bound) chk_index((err), (long long)(i), (long long)(bound))
#else
#define LBM_CHK(err, i, bound) (i)
#endif

// Compute-type constants derived on the host from Args (see make_coef).
template <class T>
struct Coef {
  T om[2];          // 1 / tau
  T tau[2];
  T G[2][2], G_ads[2], psi_wall, rho0, g[3];
  T mrt_g[10];      // (s_k - 1/tau) / |R_k|^2 of the MRT rows (one component)
  T omc[3];         // 1 / tau_c
  T wc0, wca;       // scalar weights: rest, axis
  T ics2c;          // 1 / c_s^2 of the scalar lattice
  T icb;            // 1 / (2 w_a + K), K = k tau_c / (tau_c - 1/2): wet-node closure
  T kr;             // k
  T C_in[3];
  T DP, keep;       // deposition probability, 1 - DP
  T rref[2], cref[3];   // storage references (0 in FP64 mode)
  T fp;             // tau_P / (tau_P - 1/2) of the product lattice
  T uw6[3];         // 6 u_wall = 2 u_wall / c_s^2 of the moving top plate
  T arrA, arrTa;    // temperature-dependent rate A exp(-Ta / T)
  T fc, fT;         // tau / (tau - 1/2) of scalar 0 and of the temperature (scalar 1)
  T hr;             // reaction heat per unit rate
  T oms;            // 1 / tau_s of the solid thermal lattice
  T cfs;            // heat-capacity ratio (rho c_p)_f / (rho c_p)_s
};

constexpr int NMON = 25;
constexpr int WALLX_SLOTS = 4096;
// partial-sum slots
enum : int {
  M_MASS = 0, M_MOM = 2, M_SPEC = 5, M_REACT = 7, M_DEPO = 8, M_IN = 9, M_OUT = 11,
  M_WALLX = 13, M_NSOLID = 14, M_NFLUID = 15, M_NONFIN = 16, M_HEAT = 17,
  M_SPEC2 = 18, M_IN2 = 19, M_OUT2 = 20, M_PROD = 21,  // the third scalar lattice; product gained
  M_TSOLID = 22, M_HEAT_S = 23, M_HEAT_SRC = 24         // conduction in the solid
};
// banks of the wall-exchange accumulators (WALLX_SLOTS doubles each)
enum : int { BANK_WALLX = 0, BANK_HEAT = 1, BANK_PROD = 2, BANK_HEAT_S = 3, BANK_HEAT_SRC = 4, NBANKS = 5 };
// monitor slots of scalar lattice s (0 .. 2)
__host__ __device__ constexpr int mon_spec(int s) { return s < 2 ? M_SPEC + s : M_SPEC2; }
__host__ __device__ constexpr int mon_in(int s) { return s < 2 ? M_IN + s : M_IN2; }
__host__ __device__ constexpr int mon_out(int s) { return s < 2 ? M_OUT + s : M_OUT2; }

// ------------------------------------------------------------- indexing

struct Nbr {
  int n;                              // linear node index
  int oxm, oxp, oym, oyp, ozm, ozp;   // linear offsets to the -/+ neighbours, periodic wrap
  __device__ __forceinline__ int at(int dx, int dy, int dz) const {
    return n + (dx < 0 ? oxm : (dx > 0 ? oxp : 0)) + (dy < 0 ? oym : (dy > 0 ? oyp : 0)) +
           (dz < 0 ? ozm : (dz > 0 ? ozp : 0));
  }
};

__device__ __forceinline__ Nbr make_nbr(const Args& a, int x, int y, int z) {
  Nbr b;
  const int sy = a.nx, sz = a.nx * a.ny;
  b.n = x + sy * y + sz * z;
  // always wrap: walls on closed axes are excluded by the link masks before any access
  b.oxm = x == 0 ? a.nx - 1 : -1;
  b.oxp = x == a.nx - 1 ? 1 - a.nx : 1;
  b.oym = y == 0 ? (a.ny - 1) * sy : -sy;
  b.oyp = y == a.ny - 1 ? (1 - a.ny) * sy : sy;
  b.ozm = z == 0 ? (a.nz - 1) * sz : -sz;
  b.ozp = z == a.nz - 1 ? (1 - a.nz) * sz : sz;
  return b;
}

template <class L>
__device__ __forceinline__ bool flow_wall(uint32_t m, int i) { return (m >> i) & 1u; }

// ------------------------------------------------------------- gathers

// Pre-collision flow populations of node n (as stored; shift added for 16-bit storage).
// Stored (deviation) values of the pre-collision flow populations of node n.
// sn is the node's storage slot; neighbour slots come from the slot map.
template <class L, class S>
__device__ __forceinline__ void gather_flow(const S* __restrict__ f, long long pitch, long long sn,
                                            const uint32_t* __restrict__ slot, uint32_t m,
                                            const Nbr& nb, int parity, typename Store<S>::T* out) {
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const S* p;
    if (parity == 0 || i == 0 || flow_wall<L>(m, L::opp(i))) {
      p = f + (long long)i * pitch + sn;
    } else {
      p = f + (long long)L::opp(i) * pitch + __ldg(slot + nb.at(-L::cx(i), -L::cy(i), -L::cz(i)));
    }
    out[i] = Store<S>::ld(p);
  }
}

// Same as gather_flow, addressing through per-plane base pointers with 64-bit node offsets
// (no multiply by the plane pitch in the kernel).
template <class L, class S>
__device__ __forceinline__ void gather_flow_pl(void* const* planes, long long sn,
                                               const uint32_t* __restrict__ slot, uint32_t m,
                                               const Nbr& nb, int parity, typename Store<S>::T* out,
                                               int* err, long long n_nodes, long long pitch) {
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const S* p;
    if (parity == 0 || i == 0 || flow_wall<L>(m, L::opp(i)))
      p = reinterpret_cast<const S*>(planes[i]) + LBM_CHK(err, sn, pitch);
    else
      p = reinterpret_cast<const S*>(planes[L::opp(i)]) +
          (long long)LBM_CHK(err, __ldg(slot + LBM_CHK(err, nb.at(-L::cx(i), -L::cy(i), -L::cz(i)), n_nodes)), pitch);
    out[i] = Store<S>::ld(p);
  }
}

template <class L, class S>
__device__ __forceinline__ void gather_scal_pl(void* const* planes, long long sn,
                                               const uint32_t* __restrict__ slot, uint32_t m,
                                               const Nbr& nb, int parity, typename Store<S>::T* out,
                                               int* err, long long n_nodes, long long pitch) {
#pragma unroll
  for (int j = 0; j < L::QC; ++j) {
    const S* p;
    if (parity == 0 || j == 0 || MaskBits<L>::code(m, L::opp(j)) != 0)
      p = reinterpret_cast<const S*>(planes[j]) + LBM_CHK(err, sn, pitch);
    else
      p = reinterpret_cast<const S*>(planes[L::opp(j)]) +
          (long long)LBM_CHK(err, __ldg(slot + LBM_CHK(err, nb.at(-L::cx(j), -L::cy(j), -L::cz(j)), n_nodes)), pitch);
    out[j] = Store<S>::ld(p);
  }
}

template <class T>
__device__ __forceinline__ T scal_w(int j, const Coef<T>& k) { return j == 0 ? k.wc0 : k.wca; }

template <class L, class S>
__device__ __forceinline__ void gather_scal(const S* __restrict__ h, long long pitch, long long sn,
                                            const uint32_t* __restrict__ slot, uint32_t m,
                                            const Nbr& nb, int parity, typename Store<S>::T* out) {
#pragma unroll
  for (int j = 0; j < L::QC; ++j) {
    const S* p;
    if (parity == 0 || j == 0 || MaskBits<L>::code(m, L::opp(j)) != 0) {
      p = h + (long long)j * pitch + sn;
    } else {
      p = h + (long long)L::opp(j) * pitch + __ldg(slot + nb.at(-L::cx(j), -L::cy(j), -L::cz(j)));
    }
    out[j] = Store<S>::ld(p);
  }
}

// Wet-node closure (Eq. wetnode9 per link).  For direction j whose source n - c_j is a
// reactive solid: C_b = 2 hb / (2 w + K), h_j = 2 w C_b - hb, hb = gathered h_{opp j}.
// All closures use the values before closure.  Returns, through the callbacks' arguments,
// the reaction rate k C_b per link and the stored-minus-closed exchange.
// h holds deviations from w_j * cref; the closure works on full values at reactive links.
template <class L, class T, class OnLink>
__device__ __forceinline__ void close_scalar(T* h, uint32_t m, const Coef<T>& k, OnLink on_link) {
  T old[L::QC];
#pragma unroll
  for (int j = 0; j < L::QC; ++j) old[j] = h[j];
  const T sh = k.wca * k.cref[0];
#pragma unroll
  for (int j = 1; j < L::QC; ++j) {
    if (MaskBits<L>::code(m, L::opp(j)) == 2u) {
      const T hb = old[L::opp(j)] + sh;
      const T Cb = T(2) * hb * k.icb;
      const T hn = T(2) * k.wca * Cb - hb - sh;
      h[j] = hn;
      on_link(j, Cb, old[j] - hn);
    }
  }
}

// Reactive link with a temperature-dependent rate and reaction heat (Sec. 2.1.5, Eq. reactO2,
// reacRate, fluxCon with an adiabatic solid): scalar 0 is the reacting species, scalar 1 the
// temperature.  With hb, gb the gathered species and temperature populations moving toward the
// wall (full values), per link
//   C_b = 2 hb / (2 w + k(T_b) fc),  k(T) = A exp(-Ta / T),  Q = h_r k(T_b) C_b,
//   T_b = (2 gb + Q fT) / (2 w),     fc, fT = tau / (tau - 1/2) of the two scalars,
// solved by n_it fixed-point iterations from the zero-flux value T_b = gb / w; then
//   h_C = 2 w C_b - hb and h_T = gb + Q fT.  All closures of a node read the values before
// any closure.  on_link(j, rate k C_b, species exchange, heat exchange) does the bookkeeping.
template <class L, class T, class OnLink>
__device__ __forceinline__ void close_thermal(T* h0, T* h1, uint32_t m, const Coef<T>& k, int n_it,
                                              OnLink on_link) {
  T old0[L::QC], old1[L::QC];
#pragma unroll
  for (int j = 0; j < L::QC; ++j) {
    old0[j] = h0[j];
    old1[j] = h1[j];
  }
  const T sh0 = k.wca * k.cref[0], sh1 = k.wca * k.cref[1];
  const T w2 = T(2) * k.wca;
#pragma unroll
  for (int j = 1; j < L::QC; ++j) {
    if (MaskBits<L>::code(m, L::opp(j)) == 2u) {
      const T hb = old0[L::opp(j)] + sh0;
      const T gb = old1[L::opp(j)] + sh1;
      T Tb = gb / k.wca;
      for (int it = 0; it < n_it; ++it) {
        const T kt = k.arrA * exp(-k.arrTa / Tb);
        const T Cb = T(2) * hb / (w2 + kt * k.fc);
        const T Q = k.hr * kt * Cb;
        Tb = (T(2) * gb + Q * k.fT) / w2;
      }
      const T kt = k.arrA * exp(-k.arrTa / Tb);
      const T Cb = T(2) * hb / (w2 + kt * k.fc);
      const T Q = k.hr * kt * Cb;
      const T hn0 = w2 * Cb - hb - sh0;
      const T hn1 = gb + Q * k.fT - sh1;
      h0[j] = hn0;
      h1[j] = hn1;
      on_link(j, kt * Cb, old0[j] - hn0, hn1 - old1[j]);
    }
  }
}

// Species closure with conduction in the solid (Sec. 2.1.5, Eq. reactO2, reacRate): the wet-node
// closure at each reactive link with the rate constant k(T_b) that the link's last exchange
// (k_exchange) found together with C_b, kept in kb[(j - 1) N + n] for the link arriving in direction
// j.  Before a link's first exchange (NaN entry) k is taken at the heat-capacity-weighted mean
// c_fs T_f + T_s over c_fs + 1 of the node's own temperature T_f and the solid's T_s.  The
// reaction heat entered the temperature through that exchange, so the temperature is not closed
// here.  h0 and h1 hold deviations from w cref; gsrc is the solid lattice the step reads.
template <class L, class T, class OnLink>
__device__ __forceinline__ void close_conjugate(T* h0, const T* h1, uint32_t m, const Coef<T>& k, const Args& a,
                                                const Nbr& nb, const T* gsrc, OnLink on_link) {
  T old[L::QC];
#pragma unroll
  for (int j = 0; j < L::QC; ++j) old[j] = h0[j];
  const T sh0 = k.wca * k.cref[0];
  const T w2 = T(2) * k.wca;
  const T* kb = reinterpret_cast<const T*>(a.kb);
#pragma unroll
  for (int j = 1; j < L::QC; ++j) {
    if (MaskBits<L>::code(m, L::opp(j)) == 2u) {
      T kt = kb[(long long)(j - 1) * a.N + nb.n];
      if (!(kt >= T(0))) {
        const int src = nb.at(-L::cx(j), -L::cy(j), -L::cz(j));
        T Tf = k.cref[1], Ts = T(0);
#pragma unroll
        for (int q = 0; q < L::QC; ++q) {
          Tf += h1[q];
          Ts += gsrc[(long long)q * a.N + src];
        }
        kt = k.arrA * exp(-k.arrTa / ((k.cfs * Tf + Ts) / (k.cfs + T(1))));
      }
      const T hb = old[L::opp(j)] + sh0;
      const T Cb = T(2) * hb / (w2 + kt * k.fc);
      const T hn = w2 * Cb - hb - sh0;
      h0[j] = hn;
      on_link(j, kt * Cb, old[j] - hn);
    }
  }
}

// The reaction product (Sec. 2.1.5, Eq. react, reactCO2): at each reactive link the product lattice
// gains what the reaction takes from scalar 0 there, r = k C_b of that link's closure.  The per-link
// wet-node ansatz of the species closure with the flux reversed, (1 - 1/(2 tau_P)) (h_P,j -
// h_P,opp j) = r, gives h_P,j = h_P,opp j + r tau_P / (tau_P - 1/2).  All closures of a node use the
// values before any closure; hp holds deviations from w C_ref,P on both sides of the link, so the
// shift cancels.  gain accumulates what the closure adds to the populations.
template <class L, class T>
__device__ __forceinline__ void close_product(T* hp, uint32_t m, const Coef<T>& k, const T* rl, T& gain) {
  T old[L::QC];
#pragma unroll
  for (int j = 0; j < L::QC; ++j) old[j] = hp[j];
#pragma unroll
  for (int j = 1; j < L::QC; ++j) {
    if (MaskBits<L>::code(m, L::opp(j)) == 2u) {
      hp[j] = old[L::opp(j)] + rl[j] * k.fp;
      gain += hp[j] - old[j];
    }
  }
}

// ---------------------------------------------------------- equilibria

template <class L, class T>
__device__ __forceinline__ T feq(int i, T rho, T ux, T uy, T uz) {
  const T cu = T(L::cx(i)) * ux + T(L::cy(i)) * uy + T(L::cz(i)) * uz;
  const T uu = ux * ux + uy * uy + uz * uz;
  return T(L::w(i)) * rho * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
}

// f_i^eq - w_i rref, given drho = rho - rref (Eq. 6 written as a deviation)
template <class L, class T>
__device__ __forceinline__ T feq_dev(int i, T rho, T drho, T ux, T uy, T uz) {
  const T cu = T(L::cx(i)) * ux + T(L::cy(i)) * uy + T(L::cz(i)) * uz;
  const T uu = ux * ux + uy * uy + uz * uz;
  return T(L::w(i)) * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
}

// Guo forcing term (Eq. 1.21) with c_s^2 = 1/3
template <class L, class T>
__device__ __forceinline__ T guo(int i, T ux, T uy, T uz, T Fx, T Fy, T Fz) {
  const T cx = T(L::cx(i)), cy = T(L::cy(i)), cz = T(L::cz(i));
  const T cu = cx * ux + cy * uy + cz * uz;
  const T cF = cx * Fx + cy * Fy + cz * Fz;
  const T uF = ux * Fx + uy * Fy + uz * Fz;
  return T(L::w(i)) * (T(3) * (cF - uF) + T(9) * cu * cF);
}

// -------------------------------------------------------- flip list append

__device__ __forceinline__ void push_flip(const Args& a, int n) {
  const unsigned int k = atomicAdd(a.flip_count, 1u);
  if (k < a.flip_cap)
    a.flip_list[k] = (uint32_t)n;
  else
    atomicOr(a.err, ERR_CAPACITY);
}

// A reactive solid node has consumed its solid mass once V_m acc >= m_s0, i.e. its remaining
// mass m_s0 - V_m acc has reached zero (solid consumption, Sec. 2.1.5).  The product is formed
// in FP64 exactly as written; a node whose V_m acc lies within rounding of m_s0 may flip one
// geometry update earlier or later than in a run that summed its links in another order.
__device__ __forceinline__ bool consumed(const Args& a, double acc) { return a.V_m * acc >= a.m_s0; }

// Exact float -> double widening by re-biasing the IEEE-754 fields with integer operations; the
// conversion instruction itself runs on the FP64 unit, which is narrow on this GPU.  Zero keeps
// its sign; subnormal, infinite and NaN inputs (never produced on the hot path) take the
// conversion instruction.
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) {
  const unsigned int b = __float_as_uint(v);
  const unsigned int ex = (b >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  if ((b << 1) == 0u) return __longlong_as_double((long long)sign);
  if (ex == 0u || ex == 0xffu) return double(v);
  return __longlong_as_double((long long)(sign | ((unsigned long long)(ex + (1023u - 127u)) << 52) |
                                          ((unsigned long long)(b & 0x7fffffu) << 29)));
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ================================================================ step

// One fused time step for every fluid node: gather (A-A parity), wet-node closure and its
// bookkeeping, deposition, moments, forces, velocity, flow collision (BGK / MRT, Guo or
// velocity shift), scalar collision, in-place scatter with bounce-back / inlet / outlet.
// Registers hold deviations from w_i * ref throughout.
#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 3   // resident 256-thread blocks per SM, one component in FP32 math (80 registers)
#endif
#ifndef LBM_STEP_MIN_BLOCKS_ODD
#define LBM_STEP_MIN_BLOCKS_ODD 3   // k_step's odd parity: the slot prefetch hides the lookups, registers pay
#endif
#ifndef LBM_TILES_MIN_BLOCKS_ODD
#define LBM_TILES_MIN_BLOCKS_ODD 3  // k_step_tiles: odd parity, slots prefetched a tile ahead (as k_step)
#endif

// Neighbour offsets of fluid node n from its coordinates (fast divisions by nx and ny).
__device__ __forceinline__ Nbr nbr_of(const Args& a, int n) {
  const unsigned int q = fast_div(unsigned(n), a.div_x);
  const unsigned int z = fast_div(q, a.div_y);
  return make_nbr(a, n - int(q) * a.nx, int(q - z * unsigned(a.ny)), int(z));
}

// Stored populations of list entry e (node n, link mask m) as the node gathers them.
template <class L, class S, int NC, int NS, int parity>
__device__ __forceinline__ void gather_entry(const Args& a, unsigned int e, unsigned int base, int n,
                                             uint32_t m, typename Store<S>::T (&f)[NC][L::Q],
                                             typename Store<S>::T (&h)[NS > 0 ? NS : 1][L::QC]) {
  const long long sn = e < base ? (long long)e : (long long)__ldg(a.slot + n);
  const Nbr nb = parity ? nbr_of(a, n) : Nbr{};
#pragma unroll
  for (int s = 0; s < NC; ++s) gather_flow_pl<L, S>(a.fplane[s], sn, a.slot, m, nb, parity, f[s], a.err, a.N, a.pitch);
#pragma unroll
  for (int s = 0; s < NS; ++s)
    gather_scal_pl<L, typename ScalarOf<S>::type>(a.hplane[s], sn, a.slot, m, nb, parity, h[s], a.err, a.N, a.pitch);
}

// Neighbour-slot cache of the odd step.  An odd step reads cell (n - c_i, opp i) and writes
// cell (n + c_i, i): every neighbour slot it needs on the way in, it needs again on the way out,
// and the scalar lattice's axis links use the flow lattice's neighbours.  The gather of the first
// flow component looks each slot up once and keeps it in shared memory, entry i - 1 for the
// neighbour n + c_i; the later gathers and the scatters read it back.  A scalar link to a fluid
// neighbour is always a fluid flow link too, so every entry they read was written.
#ifndef LBM_ODD_SLOT_CACHE
#define LBM_ODD_SLOT_CACHE 1
#endif
// k_step keeps the cache as rows of LBM_STEP_CACHE_STRIDE threads per direction (consecutive
// threads in consecutive words; its blocks have at most that many threads); the ensemble's
// tile kernel gives each thread Q consecutive words of dynamic shared memory instead, sized
// to its block (Q - 1 used; the odd stride puts the threads of a warp on distinct banks).
#define LBM_STEP_CACHE_STRIDE 256
#ifndef LBM_ODD_SLOT_PREFETCH
#define LBM_ODD_SLOT_PREFETCH 1   // k_step: the slots of the next node are copied in while this one runs
#endif
// Asynchronous copies (cp.async, sm_80 and later) of one 4-byte word from global to shared
// memory; a thread waits for its own groups with cp_async_wait.
__device__ __forceinline__ void cp_async4(uint32_t* smem, const uint32_t* gmem) {
  const unsigned int s = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Start copying the slots of all Q - 1 neighbours n + c_i of node n into the cache rows (row i
// for n + c_i), one step of the grid-stride loop ahead of their use.  Links into walls copy a
// slot that is never read (the periodic image is always a valid node).
template <class L, int CS>
__device__ __forceinline__ void prefetch_slots(const Args& a, int n, uint32_t* cache) {
  const Nbr nb = nbr_of(a, n);
#pragma unroll
  for (int i = 1; i < L::Q; ++i)
    cp_async4(cache + (i - 1) * CS, a.slot + LBM_CHK(a.err, nb.at(L::cx(i), L::cy(i), L::cz(i)), a.N));
}

// Flow links into walls read and write the node's own cell: (n, i) for the population arriving
// in direction i, which sits in plane i while a fluid link's cell sits in plane opp(i).  Writing
// into a wall link's cache entry the offset of that own cell relative to the neighbour's plane,
// slot + (opp(k) - k) * pitch, lets every flow access take plane + entry without testing the
// link (signed 32-bit: needs 3 * pitch < 2^31, checked on the host).
template <class L, int CS>
__device__ __forceinline__ void wall_offsets(const Args& a, long long sn, uint32_t m, uint32_t* cache) {
#pragma unroll
  for (int k = 1; k < L::Q; ++k)
    if (flow_wall<L>(m, k)) cache[(k - 1) * CS] = (uint32_t)(int)(sn + (long long)(L::opp(k) - k) * a.pitch);
}

template <class L, class S, int NC, int NS, int CS, bool PREFETCHED = false, bool VOFF = false>
__device__ __forceinline__ void gather_entry_odd_cached(const Args& a, long long sn, int n, uint32_t m,
                                                        uint32_t* cache, typename Store<S>::T (&f)[NC][L::Q],
                                                        typename Store<S>::T (&h)[NS > 0 ? NS : 1][L::QC]) {
  const Nbr nb = PREFETCHED ? Nbr{} : nbr_of(a, n);
#pragma unroll
  for (int s = 0; s < NC; ++s) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const S* p;
      if (VOFF && i != 0) {
        // the entry holds the plane-relative offset of the cell, own or neighbour (see
        // wall_offsets)
        const long long off = (long long)(int)cache[(L::opp(i) - 1) * CS];
        const long long base_k = (long long)L::opp(i) * a.pitch;   // the plane's start in the array
        p = reinterpret_cast<const S*>(a.fplane[s][L::opp(i)]) +
            (LBM_CHK(a.err, off + base_k, (long long)L::Q * a.pitch) - base_k);
      } else if (i == 0 || flow_wall<L>(m, L::opp(i))) {
        p = reinterpret_cast<const S*>(a.fplane[s][i]) + LBM_CHK(a.err, sn, a.pitch);
      } else {
        uint32_t q;
        if (s == 0 && PREFETCHED) {
          q = (uint32_t)LBM_CHK(a.err, cache[(L::opp(i) - 1) * CS], a.pitch);
        } else if (s == 0) {
          q = (uint32_t)LBM_CHK(a.err, __ldg(a.slot + LBM_CHK(a.err, nb.at(-L::cx(i), -L::cy(i), -L::cz(i)), a.N)),
                                a.pitch);
          cache[(L::opp(i) - 1) * CS] = q;
        } else {
          q = cache[(L::opp(i) - 1) * CS];
        }
        p = reinterpret_cast<const S*>(a.fplane[s][L::opp(i)]) + q;
      }
      f[s][i] = Store<S>::ld(p);
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
#pragma unroll
    for (int j = 0; j < L::QC; ++j) {
      using SC = typename ScalarOf<S>::type;
      const SC* p;
      if (j == 0 || MaskBits<L>::code(m, L::opp(j)) != 0)
        p = reinterpret_cast<const SC*>(a.hplane[s][j]) + LBM_CHK(a.err, sn, a.pitch);
      else
        p = reinterpret_cast<const SC*>(a.hplane[s][L::opp(j)]) + cache[(L::opp(j) - 1) * CS];
      h[s][j] = Store<SC>::ld(p);
    }
  }
}

// ------------------------------------------------------------- collision helpers

// Fused multiply-add of the compute types.
__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }

// MRT correction on top of the BGK update: with n = f - f_eq + F_i / 2 split into pair sums sp
// and differences dp (indexed by the first member of each opposite pair, sp[0] = n_0),
// f_i -= sum_k R_k(c_i) g_k m_k, m_k = sum_i R_k(c_i) n_i, g_k = (s_k - 1/tau) / |R_k|^2.
// Generic form, row by row.
template <class L, class T, class G>
__device__ __forceinline__ void mrt_correct_rows(T* f, const T* sp, const T* dp, const G* g) {
  T coef[L::NMRT];
#pragma unroll
  for (int kk = 0; kk < L::NMRT; ++kk) {
    T mk = T(0);
    if (!mrt_odd<L>(kk)) {
      const int r0 = Mrt<L>::row(kk, 0);
      if (r0 != 0) mk += T(r0) * sp[0];
    }
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
      if (i > L::opp(i)) continue;
      const int r = Mrt<L>::row(kk, i);
      if (r != 0) mk += T(r) * (mrt_odd<L>(kk) ? dp[i] : sp[i]);
    }
    coef[kk] = T(g[kk]) * mk;
  }
  {
    T c = T(0);
#pragma unroll
    for (int kk = 0; kk < L::NMRT; ++kk) {
      const int r = Mrt<L>::row(kk, 0);
      if (r != 0 && !mrt_odd<L>(kk)) c += T(r) * coef[kk];
    }
    f[0] -= c;
  }
#pragma unroll
  for (int i = 1; i < L::Q; ++i) {
    if (i > L::opp(i)) continue;
    T ce = T(0), co = T(0);
#pragma unroll
    for (int kk = 0; kk < L::NMRT; ++kk) {
      const int r = Mrt<L>::row(kk, i);
      if (r == 0) continue;
      if (mrt_odd<L>(kk)) co += T(r) * coef[kk];
      else ce += T(r) * coef[kk];
    }
    f[i] -= ce + co;
    f[L::opp(i)] -= ce - co;
  }
}

// D3Q19: the same rows (d'Humieres et al. 2002) evaluated through the sums their polynomials
// share: axis pairs 1, 3, 5 (x, y, z), diagonal classes xy {7, 13}, xz {9, 15}, yz {11, 17}.
template <class T, class G>
__device__ __forceinline__ void mrt_correct_d3q19(T* f, const T* sp, const T* dp, const G* g) {
  // even moments (e, eps, 3 pi_xx, pi_ww) from pair sums
  const T A = sp[1] + sp[3] + sp[5];
  const T Dxy = sp[7] + sp[13], Dxz = sp[9] + sp[15], Dyz = sp[11] + sp[17];
  const T D = Dxy + Dxz + Dyz;
  const T m_e = fmad(T(-30), sp[0], fmad(T(-11), A, T(8) * D));
  const T m_eps = fmad(T(12), sp[0], fmad(T(-4), A, D));
  const T m_pxx = fmad(T(-4), sp[1], fmad(T(2), sp[3] + sp[5], fmad(T(-2), Dyz, Dxy + Dxz)));
  const T m_pww = fmad(T(2), sp[5] - sp[3], Dxy - Dxz);
  // odd moments (q, m) from pair differences
  const T P = dp[7] + dp[13], Mxy = dp[7] - dp[13];
  const T R = dp[9] + dp[15], Mxz = dp[9] - dp[15];
  const T S = dp[11] + dp[17], Myz = dp[11] - dp[17];
  const T m_qx = fmad(T(-4), dp[1], P + R), m_mx = P - R;
  const T m_qy = fmad(T(-4), dp[3], Mxy + S), m_my = S - Mxy;
  const T m_qz = fmad(T(-4), dp[5], Mxz + Myz), m_mz = Mxz - Myz;
  // row order of g: e, eps, q_x, q_y, q_z, 3 pi_xx, pi_ww, m_x, m_y, m_z
  const T ce = T(g[0]) * m_e, cs = T(g[1]) * m_eps;
  const T cqx = T(g[2]) * m_qx, cqy = T(g[3]) * m_qy, cqz = T(g[4]) * m_qz;
  const T cpx = T(g[5]) * m_pxx, cpw = T(g[6]) * m_pww;
  const T cmx = T(g[7]) * m_mx, cmy = T(g[8]) * m_my, cmz = T(g[9]) * m_mz;
  // redistribution: even part E of each pair, odd part O; f_i -= E + O, f_opp -= E - O
  f[0] = fmad(T(30), ce, fmad(T(-12), cs, f[0]));
  const T a0 = fmad(T(-11), ce, T(-4) * cs);
  const T Ex = fmad(T(-4), cpx, a0);
  const T t = fmad(T(2), cpx, a0);
  const T Ey = fmad(T(-2), cpw, t), Ez = fmad(T(2), cpw, t);
  f[1] = fmad(T(4), cqx, f[1] - Ex);
  f[2] = fmad(T(-4), cqx, f[2] - Ex);
  f[3] = fmad(T(4), cqy, f[3] - Ey);
  f[4] = fmad(T(-4), cqy, f[4] - Ey);
  f[5] = fmad(T(4), cqz, f[5] - Ez);
  f[6] = fmad(T(-4), cqz, f[6] - Ez);
  const T d0 = fmad(T(8), ce, cs);
  const T Exy = d0 + (cpx + cpw), Exz = d0 + (cpx - cpw), Eyz = fmad(T(-2), cpx, d0);
  const T u1 = cqx + cmx, v1 = cqy - cmy;   // pairs 7 (+x+y): u1 + v1, 13 (+x-y): u1 - v1
  const T u2 = cqx - cmx, v2 = cqz + cmz;   // pairs 9 (+x+z): u2 + v2, 15 (+x-z): u2 - v2
  const T u3 = cqy + cmy, v3 = cqz - cmz;   // pairs 11 (+y+z): u3 + v3, 17 (+y-z): u3 - v3
  const T O7 = u1 + v1, O13 = u1 - v1, O9 = u2 + v2, O15 = u2 - v2, O11 = u3 + v3, O17 = u3 - v3;
  f[7] = (f[7] - Exy) - O7;
  f[8] = (f[8] - Exy) + O7;
  f[13] = (f[13] - Exy) - O13;
  f[14] = (f[14] - Exy) + O13;
  f[9] = (f[9] - Exz) - O9;
  f[10] = (f[10] - Exz) + O9;
  f[15] = (f[15] - Exz) - O15;
  f[16] = (f[16] - Exz) + O15;
  f[11] = (f[11] - Eyz) - O11;
  f[12] = (f[12] - Eyz) + O11;
  f[17] = (f[17] - Eyz) - O17;
  f[18] = (f[18] - Eyz) + O17;
}
template <class L, class T, class G>
__device__ __forceinline__ void mrt_correct(T* f, const T* sp, const T* dp, const G* g) {
  if constexpr (L::Q == 19) mrt_correct_d3q19<T, G>(f, sp, dp, g);
  else mrt_correct_rows<L, T, G>(f, sp, dp, g);
}

// Everything after the gather for one fluid node: wet-node closure and its bookkeeping,
// deposition, moments, forces, velocity, flow and scalar collision, in-place scatter.
template <class L, class S, int NC, int NS, int COLL, int parity, bool BND, bool CACHE = false, int CS = 1,
          bool VOFF = false>
__device__ __forceinline__ void collide_scatter(const Args& a, const Coef<typename Store<S>::T>& k, int n,
                                                uint32_t m, long long sn,
                                                typename Store<S>::T (&f)[NC][L::Q],
                                                typename Store<S>::T (&h)[NS > 0 ? NS : 1][L::QC],
                                                typename Store<S>::T& wallx, typename Store<S>::T& heatx,
                                                typename Store<S>::T& prodx, const uint32_t* cache = nullptr) {
  using T = typename Store<S>::T;
  constexpr int Q = L::Q, QC = L::QC;
  const Nbr nb = nbr_of(a, n);
  // ---- wet-node closure of scalar 0 and reaction bookkeeping (Eq. wetnode9, reactO2)
  if (NS > 0) {
    // the consumed totals are reductions (no value returned): the threshold test runs in
    // k_detect over the interface list before the geometry update; rl keeps each link's rate
    // for the product lattice's closure
    T rl[QC];
#pragma unroll
    for (int j = 0; j < QC; ++j) rl[j] = T(0);
    if (BND && NS > 1 && a.conjugate) {
      // conduction in the solid: the rate constant of the link's last exchange
      close_conjugate<L, T>(h[0], h[NS > 1 ? 1 : 0], m, k, a, nb,
                            reinterpret_cast<const T*>(a.gs[parity]), [&](int j, T r, T exch) {
        const int src = LBM_CHK(a.err, nb.at(-L::cx(j), -L::cy(j), -L::cz(j)), a.N);
        atomicAdd(a.acc + src, widen(r));
        wallx += exch;
        rl[j] = r;
      });
    } else if (BND && NS > 1 && a.arrhenius) {
      // temperature-dependent rate and reaction heat (the full kernel variant only)
      close_thermal<L, T>(h[0], h[NS > 1 ? 1 : 0], m, k, a.n_it, [&](int j, T r, T exch, T heat) {
        const int src = LBM_CHK(a.err, nb.at(-L::cx(j), -L::cy(j), -L::cz(j)), a.N);
        atomicAdd(a.acc + src, widen(r));
        wallx += exch;
        heatx += heat;
        rl[j] = r;
      });
    } else {
      close_scalar<L, T>(h[0], m, k, [&](int j, T Cb, T exch) {
        const int src = LBM_CHK(a.err, nb.at(-L::cx(j), -L::cy(j), -L::cz(j)), a.N);
        atomicAdd(a.acc + src, widen(k.kr * Cb));
        wallx += exch;
        rl[j] = k.kr * Cb;
      });
    }
    if (NS > 1 && a.product) close_product<L, T>(h[NS - 1], m, k, rl, prodx);
    // ---- deposition at near-substrate nodes (Eq. surface_deposition)
    if (a.geo_mode == GEO_DEPOSIT) {
      bool near = false;
#pragma unroll
      for (int j = 1; j < QC; ++j) {
        const uint32_t c = MaskBits<L>::code(m, j);
        near |= (c == 1u || c == 2u);
      }
      if (near) {
        T sum = k.cref[0];
#pragma unroll
        for (int j = 0; j < QC; ++j) sum += h[0][j];
        const double dep = double(k.DP * sum);
        const double old = a.acc[n];
        a.acc[n] = old + dep;
        if (old <= 1.0 && old + dep > 1.0) push_flip(a, n);
        if (a.deposit_conservative) {
#pragma unroll
          for (int j = 0; j < QC; ++j) h[0][j] = h[0][j] * k.keep - scal_w<T>(j, k) * k.cref[0] * k.DP;
        }
      }
    }
  }
  // ---- moments (Eq. 1.7, 1.8): rho = rref + sum of deviations
  T drho[NC], rho[NC], jx[NC], jy[NC], jz[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    T r = T(0), ax = T(0), ay = T(0), az = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      r += f[s][i];
      if (L::cx(i)) ax += T(L::cx(i)) * f[s][i];
      if (L::cy(i)) ay += T(L::cy(i)) * f[s][i];
      if (L::cz(i)) az += T(L::cz(i)) * f[s][i];
    }
    drho[s] = r;
    rho[s] = k.rref[s] + r;
    jx[s] = ax; jy[s] = ay; jz[s] = az;
  }
  // ---- forces: Shan-Chen cohesion / solid psi (Eq. 1.13, 1.14), adhesion (1.15), body
  T Fx[NC], Fy[NC], Fz[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    Fx[s] = rho[s] * k.g[0];
    Fy[s] = rho[s] * k.g[1];
    Fz[s] = rho[s] * k.g[2];
  }
  if (a.sc_on) {
    T sx[NC], sy[NC], sz[NC];
#pragma unroll
    for (int s2 = 0; s2 < NC; ++s2) {
      const T* ps = reinterpret_cast<const T*>(a.psi[s2]);
      T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const T pv = flow_wall<L>(m, i) ? k.psi_wall : ps[nb.at(L::cx(i), L::cy(i), L::cz(i))];
        const T wp = T(L::w(i)) * pv;
        if (L::cx(i)) ax += T(L::cx(i)) * wp;
        if (L::cy(i)) ay += T(L::cy(i)) * wp;
        if (L::cz(i)) az += T(L::cz(i)) * wp;
      }
      sx[s2] = ax; sy[s2] = ay; sz[s2] = az;
    }
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      const T pself = reinterpret_cast<const T*>(a.psi[s])[n];
#pragma unroll
      for (int s2 = 0; s2 < NC; ++s2) {
        const T Gss = k.G[s][s2];
        Fx[s] -= pself * Gss * sx[s2];
        Fy[s] -= pself * Gss * sy[s2];
        Fz[s] -= pself * Gss * sz[s2];
      }
    }
  }
  if (a.ads_on) {
    T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (flow_wall<L>(m, i)) {
        ax += T(L::w(i)) * T(L::cx(i));
        ay += T(L::w(i)) * T(L::cy(i));
        az += T(L::w(i)) * T(L::cz(i));
      }
    }
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      const T ga = k.G_ads[s] * rho[s];
      Fx[s] -= ga * ax; Fy[s] -= ga * ay; Fz[s] -= ga * az;
    }
  }
  // ---- physical / barycentric velocity (Eq. 1.19, 1.20)
  T rt = T(0), mx = T(0), my = T(0), mz = T(0);
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    rt += rho[s];
    mx += jx[s] + T(0.5) * Fx[s];
    my += jy[s] + T(0.5) * Fy[s];
    mz += jz[s] + T(0.5) * Fz[s];
  }
  const T irt = T(1) / rt;
  const T ux = mx * irt, uy = my * irt, uz = mz * irt;
  // ---- flow collision
  if (a.shift_forcing) {
    // Shan-Chen velocity shift (Eq. 1.17, 1.18), BGK, F_i = 0
    T nxs = T(0), nys = T(0), nzs = T(0), den = T(0);
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      nxs += jx[s] * k.om[s]; nys += jy[s] * k.om[s]; nzs += jz[s] * k.om[s];
      den += rho[s] * k.om[s];
    }
    const T iden = T(1) / den;
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      const T ir = T(1) / rho[s];
      const T ex = nxs * iden + k.tau[s] * Fx[s] * ir;
      const T ey = nys * iden + k.tau[s] * Fy[s] * ir;
      const T ez = nzs * iden + k.tau[s] * Fz[s] * ir;
#pragma unroll
      for (int i = 0; i < Q; ++i)
        f[s][i] -= k.om[s] * (f[s][i] - feq_dev<L, T>(i, rho[s], drho[s], ex, ey, ez));
    }
  } else {
    // Eq. 1.16 with Guo forcing (Eq. 1.21): f* = f + F_i - omega (f - f_eq + F_i / 2), for BGK;
    // MRT adds the projections of n = f - f_eq + F_i / 2 on the non-hydrodynamic groups with
    // rate (s_g - 1/tau).  Opposite directions are handled as pairs: the equilibrium and the
    // Guo term split into even and odd parts, even MRT rows see n_i + n_opp(i), odd rows see
    // n_i - n_opp(i).
    const T uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      const T om = k.om[s];
      const T uF = ux * Fx[s] + uy * Fy[s] + uz * Fz[s];
      T sp[Q], dp[Q];   // pair sums / differences of n (MRT only), index of the first member
      {
        // rest population
        const T w0 = T(L::w(0));
        const T fe = w0 * (drho[s] - rho[s] * T(1.5) * uu);
        const T Fi = w0 * (T(-3) * uF);
        const T nq = f[s][0] - fe + T(0.5) * Fi;
        if (COLL == 1) sp[0] = nq;
        f[s][0] = f[s][0] + Fi - om * nq;
      }
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (i > L::opp(i)) continue;
        const int o = L::opp(i);
        const T w = T(L::w(i));
        const T cu = T(L::cx(i)) * ux + T(L::cy(i)) * uy + T(L::cz(i)) * uz;
        const T cF = T(L::cx(i)) * Fx[s] + T(L::cy(i)) * Fy[s] + T(L::cz(i)) * Fz[s];
        const T fe_e = w * (drho[s] + rho[s] * (T(4.5) * cu * cu - T(1.5) * uu));
        const T fe_o = w * (T(3) * rho[s] * cu);
        const T Fi_e = w * (T(9) * cu * cF - T(3) * uF);
        const T Fi_o = w * (T(3) * cF);
        const T nq_i = f[s][i] - (fe_e + fe_o) + T(0.5) * (Fi_e + Fi_o);
        const T nq_o = f[s][o] - (fe_e - fe_o) + T(0.5) * (Fi_e - Fi_o);
        if (COLL == 1) {
          sp[i] = nq_i + nq_o;
          dp[i] = nq_i - nq_o;
        }
        f[s][i] = f[s][i] + (Fi_e + Fi_o) - om * nq_i;
        f[s][o] = f[s][o] + (Fi_e - Fi_o) - om * nq_o;
      }
      if (COLL == 1) mrt_correct<L>(f[s], sp, dp, k.mrt_g);
    }
  }
  // ---- scalar collision (Eq. therpop_species, therpopeq_species), u = physical velocity
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    T dC = T(0);
#pragma unroll
    for (int j = 0; j < QC; ++j) dC += h[s][j];
    const T C = k.cref[s] + dC;
#pragma unroll
    for (int j = 0; j < QC; ++j) {
      const T cu = T(L::cx(j)) * ux + T(L::cy(j)) * uy + T(L::cz(j)) * uz;
      const T he = scal_w<T>(j, k) * (dC + C * cu * k.ics2c);
      h[s][j] -= k.omc[s] * (h[s][j] - he);
    }
  }
  // ---- scatter flow
  // a node under a moving top plate (Sec. 3.1.1): links through the face beyond y = ny - 1
  // reflect with Ladd's momentum exchange 2 w_i rho (c_i . u_wall) / c_s^2
  // a node on the inlet face (Sec. 3.4): links leaving through x = 0 reflect off a face moving
  // with the inlet profile (the same momentum exchange); on the outlet face the population
  // entering through x = nx - 1 repeats the node's own post-collision value (zero gradient)
  // (BND: the kernel variant for contexts with a moving plate or a velocity inlet)
  bool top = false, xin = false, xout = false;
  T uin = T(0);
  if (BND && (a.moving_wall || a.flow_open_x)) {
    const unsigned int q = fast_div(unsigned(n), a.div_x);
    const int yy = int(q - fast_div(q, a.div_y) * unsigned(a.ny));
    top = a.moving_wall && yy == a.ny - 1;
    if (a.flow_open_x) {
      const int xx = n - int(q) * a.nx;
      xin = xx == 0;
      xout = xx == a.nx - 1;
      if (xin) uin = T(a.u_in_row[yy]);
    }
  }
#pragma unroll
  for (int s = 0; s < NC; ++s) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      S* p;
      T v = f[s][i];
      bool keep = true;
      if (VOFF && i != 0) {
        const long long off = (long long)(int)cache[(i - 1) * CS];
        const long long base_k = (long long)i * a.pitch;   // the plane's start in the array
        p = reinterpret_cast<S*>(a.fplane[s][i]) + (LBM_CHK(a.err, off + base_k, (long long)L::Q * a.pitch) - base_k);
      } else if (parity == 0 || i == 0 || flow_wall<L>(m, i)) {
        p = reinterpret_cast<S*>(a.fplane[s][L::opp(i)]) + LBM_CHK(a.err, sn, a.pitch);
        if (BND) {
          if (L::cx(i) < 0 && xin && flow_wall<L>(m, i))
            v += T(6.0 * L::w(i)) * rho[s] * uin;
          else if (L::cx(i) > 0 && xout)
            keep = false;   // leaves through the outlet; the cell is written below with opp(i)
          else if (L::cy(i) > 0 && top && flow_wall<L>(m, i))
            v -= T(L::w(i)) * rho[s] * (T(L::cx(i)) * k.uw6[0] + T(L::cz(i)) * k.uw6[2] + k.uw6[1]);
        }
      } else {
        if (CACHE)
          p = reinterpret_cast<S*>(a.fplane[s][i]) + cache[(i - 1) * CS];
        else
          p = reinterpret_cast<S*>(a.fplane[s][i]) +
              LBM_CHK(a.err, (long long)__ldg(a.slot + LBM_CHK(a.err, nb.at(L::cx(i), L::cy(i), L::cz(i)), a.N)), a.pitch);
      }
      if (keep) Store<S>::st(p, v);
      // zero-gradient outlet: the population entering through x = nx - 1 with direction i
      // repeats the node's own post-collision f_i, in the cell where link opp(i) reflects
      if (BND && L::cx(i) < 0 && xout)
        Store<S>::st(reinterpret_cast<S*>(a.fplane[s][i]) + LBM_CHK(a.err, sn, a.pitch), f[s][i]);
    }
  }
  // ---- scatter scalars: bounce-back at walls, inlet ghost / zero-gradient outlet at open faces
#pragma unroll
  for (int s = 0; s < NS; ++s) {
#pragma unroll
    for (int j = 0; j < QC; ++j) {
      using SC = typename ScalarOf<S>::type;
      const uint32_t code = j == 0 ? 0u : MaskBits<L>::code(m, j);
      T v = h[s][j];
      SC* p;
      if (code == 3u) {
        // open face: the population arriving from outside replaces the one leaving
        const int jb = L::opp(j);
        T b;
        const T sh = k.wca * k.cref[s];
        if (L::cx(j) < 0) {
          const T cu = T(L::cx(jb)) * ux + T(L::cy(jb)) * uy + T(L::cz(jb)) * uz;
          b = k.wca * k.C_in[s] * (T(1) + cu * k.ics2c) - sh;
          a.inflow_row[LBM_CHK(a.err, s * (a.ny * a.nz) + int(fast_div(unsigned(n), a.div_x)), 3ll * a.ny * a.nz)] +=
              widen(b) - widen(v);
        } else {
          b = h[s][jb];
          a.outflow_row[LBM_CHK(a.err, s * (a.ny * a.nz) + int(fast_div(unsigned(n), a.div_x)), 3ll * a.ny * a.nz)] +=
              widen(v) - widen(b);
        }
        v = b;
        p = reinterpret_cast<SC*>(a.hplane[s][jb]) + LBM_CHK(a.err, sn, a.pitch);
      } else if (parity == 0 || j == 0 || code != 0u) {
        p = reinterpret_cast<SC*>(a.hplane[s][L::opp(j)]) + LBM_CHK(a.err, sn, a.pitch);
      } else {
        if (CACHE)
          p = reinterpret_cast<SC*>(a.hplane[s][j]) + cache[(j - 1) * CS];
        else
          p = reinterpret_cast<SC*>(a.hplane[s][j]) +
              LBM_CHK(a.err, (long long)__ldg(a.slot + LBM_CHK(a.err, nb.at(L::cx(j), L::cy(j), L::cz(j)), a.N)), a.pitch);
      }
      Store<SC>::st(p, v);
    }
  }
}

// One fused time step for every fluid node: gather (A-A parity), wet-node closure and its
// bookkeeping, deposition, moments, forces, velocity, flow collision (BGK / MRT, Guo or
// velocity shift), scalar collision, in-place scatter with bounce-back / inlet / outlet.
// Registers hold deviations from w_i * ref throughout.
template <class L, class S, int NC, int NS, int COLL, int parity, bool BND>
__global__ void __launch_bounds__(256, (NC == 1 && sizeof(typename Store<S>::T) == 4 ? (parity ? LBM_STEP_MIN_BLOCKS_ODD : LBM_STEP_MIN_BLOCKS) : 2)) k_step(const Args a, const Coef<typename Store<S>::T> k) {
  using T = typename Store<S>::T;
  constexpr int Q = L::Q, QC = L::QC, NSD = NS > 0 ? NS : 1;
  T wallx = T(0), heatx = T(0), prodx = T(0);
  const unsigned int count = a.fluid_count[0];
  const unsigned int base = a.fluid_count[1];   // entries below it have slot == entry
  const unsigned int stride = gridDim.x * blockDim.x;
  unsigned int e = blockIdx.x * blockDim.x + threadIdx.x;
  // Odd parity with two cache buffers: the neighbour slots of the next entry are copied
  // asynchronously into one while the current entry works from the other.
  constexpr bool kPrefetch = LBM_ODD_SLOT_CACHE && LBM_ODD_SLOT_PREFETCH && parity == 1;
#if LBM_ODD_SLOT_CACHE && LBM_ODD_SLOT_PREFETCH
  if (kPrefetch) {
    __shared__ uint32_t slot_buf[kPrefetch ? 2 * (L::Q - 1) * LBM_STEP_CACHE_STRIDE : 1];
    uint32_t* cb = slot_buf + threadIdx.x;
    uint32_t* cn = slot_buf + (L::Q - 1) * LBM_STEP_CACHE_STRIDE + threadIdx.x;
    int n_cur = e < count ? int(LBM_CHK(a.err, a.fluid_list[e], a.N)) : 0;
    int n_nx = e + stride < count ? int(LBM_CHK(a.err, a.fluid_list[e + stride], a.N)) : 0;
    uint32_t m_cur = e < count ? a.mask[n_cur] : 0u;
    if (e < count) prefetch_slots<L, LBM_STEP_CACHE_STRIDE>(a, n_cur, cb);
    cp_async_commit();
    for (; e < count; e += stride) {
      const int n = n_cur;
      const uint32_t m = m_cur;
      if (e + stride < count) {
        n_cur = n_nx;
        m_cur = a.mask[n_cur];
        prefetch_slots<L, LBM_STEP_CACHE_STRIDE>(a, n_cur, cn);
      }
      if (e + 2 * stride < count) n_nx = int(LBM_CHK(a.err, a.fluid_list[e + 2 * stride], a.N));
      cp_async_commit();
      cp_async_wait<1>();   // this entry's slots have arrived
      if (m & 1u) {
        T f[NC][Q], h[NSD][QC];
        const long long sn = e < base ? (long long)e : (long long)__ldg(a.slot + n);
        // the plain variant addresses every flow link through its cache entry (wall_offsets);
        // the full variant keeps the per-link tests its boundary rules need
        if (!BND) wall_offsets<L, LBM_STEP_CACHE_STRIDE>(a, sn, m, cb);
        gather_entry_odd_cached<L, S, NC, NS, LBM_STEP_CACHE_STRIDE, true, !BND>(a, sn, n, m, cb, f, h);
        collide_scatter<L, S, NC, NS, COLL, parity, BND, true, LBM_STEP_CACHE_STRIDE, !BND>(a, k, n, m, sn, f, h, wallx,
                                                                                          heatx, prodx, cb);
      }
      uint32_t* t = cb;
      cb = cn;
      cn = t;
    }
    cp_async_wait<0>();
  } else
#endif
  {
#if LBM_ODD_SLOT_CACHE
  __shared__ uint32_t slot_cache[(parity && !kPrefetch) ? (L::Q - 1) * LBM_STEP_CACHE_STRIDE : 1];
  uint32_t* cache = slot_cache + threadIdx.x;
#endif
  // the list entry is fetched two iterations and the link mask one iteration ahead
  int n_next = e < count ? int(LBM_CHK(a.err, a.fluid_list[e], a.N)) : 0;
  int n_next2 = e + stride < count ? int(LBM_CHK(a.err, a.fluid_list[e + stride], a.N)) : 0;
  uint32_t m_next = e < count ? a.mask[n_next] : 0u;
  for (; e < count; e += stride) {
    const int n = n_next;
    const uint32_t m = m_next;
    n_next = n_next2;
    if (e + stride < count) m_next = a.mask[n_next];
    if (e + 2 * stride < count) n_next2 = int(LBM_CHK(a.err, a.fluid_list[e + 2 * stride], a.N));
    if (!(m & 1u)) continue;   // a node removed by deposition since the last list rebuild
    T f[NC][Q], h[NSD][QC];
#if LBM_ODD_SLOT_CACHE
    if (parity) {
      const long long sn = e < base ? (long long)e : (long long)__ldg(a.slot + n);
      gather_entry_odd_cached<L, S, NC, NS, LBM_STEP_CACHE_STRIDE>(a, sn, n, m, cache, f, h);
      collide_scatter<L, S, NC, NS, COLL, parity, BND, true, LBM_STEP_CACHE_STRIDE>(a, k, n, m, sn, f, h, wallx, heatx,
                                                                                    prodx, cache);
      continue;
    }
#endif
    gather_entry<L, S, NC, NS, parity>(a, e, base, n, m, f, h);
    const long long sn = e < base ? (long long)e : (long long)__ldg(a.slot + n);
    collide_scatter<L, S, NC, NS, COLL, parity, BND>(a, k, n, m, sn, f, h, wallx, heatx, prodx);
  }
  }
  // ---- wall-exchange monitor: one reduction per warp that saw a reactive link
  if (NS > 0) {
    const unsigned int any = __ballot_sync(0xffffffffu, wallx != T(0));
    if (any) {
      const T w = warp_sum(wallx);
      if ((threadIdx.x & 31) == 0)
        atomicAdd(a.wallx_slot + ((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % WALLX_SLOTS),
                  widen(w));
    }
  }
  // ---- reaction heat monitor (second bank of the slots)
  if (BND && NS > 1) {
    const unsigned int any = __ballot_sync(0xffffffffu, heatx != T(0));
    if (any) {
      const T w = warp_sum(heatx);
      if ((threadIdx.x & 31) == 0)
        atomicAdd(a.wallx_slot + WALLX_SLOTS +
                      ((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % WALLX_SLOTS),
                  widen(w));
    }
  }
  // ---- reaction product monitor (third bank)
  if (NS > 1) {
    const unsigned int any = __ballot_sync(0xffffffffu, prodx != T(0));
    if (any) {
      const T w = warp_sum(prodx);
      if ((threadIdx.x & 31) == 0)
        atomicAdd(a.wallx_slot + 2 * WALLX_SLOTS +
                      ((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % WALLX_SLOTS),
                  widen(w));
    }
  }
}

// ================================================================ ensembles

#ifndef LBM_TILE_CHUNK
#define LBM_TILE_CHUNK 8
#endif
// Work tile of an ensemble step: blockDim consecutive fluid-list entries of one member.
struct Tile {
  unsigned int member, first;
};

// One time step of every member of an ensemble in one launch.  Blocks take chunks of the work
// list of tiles in turn; whenever a block enters another member it stages that member's
// arguments and constants in shared memory, and for each tile it updates entries first ..
// first + blockDim - 1 exactly as k_step updates them.
template <class L, class S, int NC, int NS, int COLL, int parity, bool BND>
__global__ void __launch_bounds__(256, (NC == 1 && sizeof(typename Store<S>::T) == 4 ? (parity ? LBM_TILES_MIN_BLOCKS_ODD : LBM_STEP_MIN_BLOCKS) : 2)) k_step_tiles(
    const Args* __restrict__ args, const Coef<typename Store<S>::T>* __restrict__ coefs,
    const Tile* __restrict__ tiles, unsigned int ntiles) {
  using T = typename Store<S>::T;
  constexpr int Q = L::Q, QC = L::QC, NSD = NS > 0 ? NS : 1;
  static_assert(sizeof(Args) % 4 == 0 && sizeof(Coef<T>) % 4 == 0, "word copies");
  __shared__ Args sa;
  __shared__ Coef<T> sk;
#if LBM_ODD_SLOT_CACHE
  extern __shared__ uint32_t slot_smem[];   // blockDim.x * Q words at odd parity (launcher)
  uint32_t* cache = slot_smem + threadIdx.x * L::Q;
#endif
  // blocks take chunks of LBM_TILE_CHUNK consecutive tiles in turn: the work list holds each
  // member's tiles together, so a chunk mostly stays within one member and its arguments are
  // staged again only when the chunk crosses into another; taking chunks in turn keeps a mix of
  // 2D and 3D members on every block
  auto next_tile = [&](unsigned int t) {
    return t + ((t % LBM_TILE_CHUNK == LBM_TILE_CHUNK - 1) ? (gridDim.x - 1) * LBM_TILE_CHUNK + 1 : 1);
  };
#if LBM_ODD_SLOT_CACHE
  // odd parity: two slot buffers, the next tile's neighbour slots are copied in (cp.async)
  // while this tile computes, as in k_step; the next tile's list entry and link mask are loaded
  // one tile ahead at both parities whenever it belongs to the member already staged
  uint32_t* cn = slot_smem + (blockDim.x + threadIdx.x) * L::Q;
#endif
  bool have_next = false;
  int n_pf = 0;
  uint32_t m_pf = 0u;
  unsigned int staged = 0xffffffffu;
  for (unsigned int t = blockIdx.x * LBM_TILE_CHUNK; t < ntiles; t = next_tile(t)) {
    const Tile tile = tiles[t];
    if (tile.member != staged) {   // block-uniform
      __syncthreads();   // the previous member's tiles are done with sa / sk
      const uint32_t* src = reinterpret_cast<const uint32_t*>(args + tile.member);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sa);
      for (unsigned int i = threadIdx.x; i < sizeof(Args) / 4; i += blockDim.x) dst[i] = src[i];
      const uint32_t* ksrc = reinterpret_cast<const uint32_t*>(coefs + tile.member);
      uint32_t* kdst = reinterpret_cast<uint32_t*>(&sk);
      for (unsigned int i = threadIdx.x; i < sizeof(Coef<T>) / 4; i += blockDim.x) kdst[i] = ksrc[i];
      __syncthreads();
      staged = tile.member;
      have_next = false;
    }
    const Args& a = sa;
    T wallx = T(0), heatx = T(0), prodx = T(0);
    const unsigned int e = tile.first + threadIdx.x;
    const unsigned int count = a.fluid_count[0];
    int n = 0;
    uint32_t m = 0u;
    if (have_next) {
      n = n_pf;
      m = m_pf;
    } else if (e < count) {
      n = int(LBM_CHK(a.err, a.fluid_list[e], a.N));
      m = a.mask[n];
#if LBM_ODD_SLOT_CACHE
      if (parity) prefetch_slots<L, 1>(a, n, cache);
#endif
    }
#if LBM_ODD_SLOT_CACHE
    if (parity) cp_async_commit();
#endif
    // the next tile of this block, if it belongs to the staged member
    have_next = false;
    const unsigned int tn = next_tile(t);
    if (tn < ntiles) {
      const Tile tile2 = tiles[tn];
      if (tile2.member == staged) {
        const unsigned int e2 = tile2.first + threadIdx.x;
        n_pf = 0;
        m_pf = 0u;
        if (e2 < count) {
          n_pf = int(LBM_CHK(a.err, a.fluid_list[e2], a.N));
          m_pf = a.mask[n_pf];
#if LBM_ODD_SLOT_CACHE
          if (parity) prefetch_slots<L, 1>(a, n_pf, cn);
#endif
        }
        have_next = true;
      }
    }
#if LBM_ODD_SLOT_CACHE
    if (parity) {
      cp_async_commit();
      cp_async_wait<1>();   // this tile's slots have arrived
    }
#endif
    if (e < count && (m & 1u)) {
      const unsigned int base = a.fluid_count[1];
      T f[NC][Q], h[NSD][QC];
      const long long sn = e < base ? (long long)e : (long long)__ldg(a.slot + n);
#if LBM_ODD_SLOT_CACHE
      if (parity) {
        // the plain variant addresses every flow link through its cache entry (wall_offsets)
        if (!BND) wall_offsets<L, 1>(a, sn, m, cache);
        gather_entry_odd_cached<L, S, NC, NS, 1, true, !BND>(a, sn, n, m, cache, f, h);
        collide_scatter<L, S, NC, NS, COLL, parity, BND, true, 1, !BND>(a, sk, n, m, sn, f, h, wallx, heatx, prodx,
                                                                         cache);
      } else
#endif
      {
        gather_entry<L, S, NC, NS, parity>(a, e, base, n, m, f, h);
        collide_scatter<L, S, NC, NS, COLL, parity, BND>(a, sk, n, m, sn, f, h, wallx, heatx, prodx);
      }
    }
#if LBM_ODD_SLOT_CACHE
    if (parity) {
      uint32_t* tmp = cache;
      cache = cn;
      cn = tmp;
    }
#endif
    if (NS > 0) {
      const unsigned int any = __ballot_sync(0xffffffffu, wallx != T(0));
      if (any) {
        const T w = warp_sum(wallx);
        if ((threadIdx.x & 31) == 0)
          atomicAdd(a.wallx_slot + ((t * (blockDim.x >> 5) + (threadIdx.x >> 5)) % WALLX_SLOTS), widen(w));
      }
    }
    if (BND && NS > 1) {
      const unsigned int any = __ballot_sync(0xffffffffu, heatx != T(0));
      if (any) {
        const T w = warp_sum(heatx);
        if ((threadIdx.x & 31) == 0)
          atomicAdd(a.wallx_slot + WALLX_SLOTS + ((t * (blockDim.x >> 5) + (threadIdx.x >> 5)) % WALLX_SLOTS),
                    widen(w));
      }
    }
    if (NS > 1) {
      const unsigned int any = __ballot_sync(0xffffffffu, prodx != T(0));
      if (any) {
        const T w = warp_sum(prodx);
        if ((threadIdx.x & 31) == 0)
          atomicAdd(a.wallx_slot + 2 * WALLX_SLOTS + ((t * (blockDim.x >> 5) + (threadIdx.x >> 5)) % WALLX_SLOTS),
                    widen(w));
      }
    }
  }
#if LBM_ODD_SLOT_CACHE
  if (parity) cp_async_wait<0>();
#endif
}

// ================================================================ psi

template <class L, class S, int NC, int parity>
__global__ void __launch_bounds__(256) k_psi(const Args a, const Coef<typename Store<S>::T> k) {
  // Walks the fluid list in slot order, as k_step does: at parity 0 every population of the
  // node sits in its own cell (coalesced); at parity 1 population i sits in cell (n - c_i, opp i),
  // whose slot is looked up once for all components.  Sums in population order 0 .. Q-1 from
  // rho_ref, the order the gather of the step uses.
  using T = typename Store<S>::T;
  const unsigned int count = a.fluid_count[0];
  const unsigned int base = a.fluid_count[1];   // entries below it have slot == entry
  const unsigned int stride = gridDim.x * blockDim.x;
  for (unsigned int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += stride) {
    const int n = int(LBM_CHK(a.err, a.fluid_list[e], a.N));
    const uint32_t m = a.mask[n];
    if (!(m & 1u)) continue;   // a node removed by deposition since the last list rebuild
    const long long sn = e < base ? (long long)e : (long long)__ldg(a.slot + n);
    long long cell[L::Q];   // slot of the cell holding population i
    const Nbr nb = parity ? nbr_of(a, n) : Nbr{};
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      cell[i] = (parity == 0 || i == 0 || flow_wall<L>(m, L::opp(i)))
                    ? sn
                    : (long long)__ldg(a.slot + LBM_CHK(a.err, nb.at(-L::cx(i), -L::cy(i), -L::cz(i)), a.N));
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      T r = k.rref[s];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        // the own cell in plane i, a neighbour's in plane opp(i)
        const bool own = parity == 0 || i == 0 || flow_wall<L>(m, L::opp(i));
        const S* p = reinterpret_cast<const S*>(own ? a.fplane[s][i] : a.fplane[s][L::opp(i)]);
        r += Store<S>::ld(p + LBM_CHK(a.err, cell[i], a.pitch));
      }
      T p;
      if (a.psi_identity) p = r;
      else p = k.rho0 * (T(1) - exp(-r / k.rho0));   // Eq. 1.11
      reinterpret_cast<T*>(a.psi[s])[n] = p;
    }
  }
}

// ================================================================ monitors

template <int K>
__device__ __forceinline__ void block_reduce_store(double (&v)[K], double* out) {
  __shared__ double sh[32][K];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, wid = tid >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double s = warp_sum(v[q]);
    if (lane == 0) sh[wid][q] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double s = lane < nw ? sh[lane][q] : 0.0;
      s = warp_sum(s);
      if (lane == 0) out[q] = s;
    }
  }
}

// Monitors, one wave of blocks: population sums over the fluid list in the compute type
// (deviations from the reference, so the sums stay accurate), bookkeeping sums over all nodes
// in FP64, per-block partials in FP64 (summed in fixed order by k_reduce_partials).
template <class L, class S, int NC, int NS>
__global__ void __launch_bounds__(256) k_monitor(const Args a, const Coef<typename Store<S>::T> k,
                                                 const int parity) {
  using T = typename Store<S>::T;
  constexpr int Q = L::Q, QC = L::QC;
  const unsigned int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned int nthr = gridDim.x * blockDim.x;
  T dm[NC > 0 ? NC : 1], mom[3] = {T(0), T(0), T(0)}, dsp[NS > 0 ? NS : 1];
#pragma unroll
  for (int s = 0; s < NC; ++s) dm[s] = T(0);
#pragma unroll
  for (int s = 0; s < NS; ++s) dsp[s] = T(0);
  unsigned int nfluid = 0, nonfin = 0;
  const unsigned int count = a.fluid_count[0], base = a.fluid_count[1];
  for (unsigned int e = tid; e < count; e += nthr) {
    const int n = int(a.fluid_list[e]);
    const uint32_t m = a.mask[n];
    if (!(m & 1u)) continue;
    ++nfluid;
    const Nbr nb = parity ? nbr_of(a, n) : Nbr{};
    const long long sn = e < base ? (long long)e : (long long)a.slot[n];
    bool bad = false;
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      T f[Q];
      gather_flow_pl<L, S>(a.fplane[s], sn, a.slot, m, nb, parity, f, a.err, a.N, a.pitch);
      T r = T(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        r += f[i];
        if (L::cx(i)) mom[0] += T(L::cx(i)) * f[i];
        if (L::cy(i)) mom[1] += T(L::cy(i)) * f[i];
        if (L::cz(i)) mom[2] += T(L::cz(i)) * f[i];
      }
      bad |= !isfinite(r);
      dm[s] += r;
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      T h[QC];
      gather_scal_pl<L, typename ScalarOf<S>::type>(a.hplane[s], sn, a.slot, m, nb, parity, h, a.err, a.N, a.pitch);
      T c = T(0);
#pragma unroll
      for (int j = 0; j < QC; ++j) c += h[j];
      bad |= !isfinite(c);
      dsp[s] += c;
    }
    nonfin += bad ? 1u : 0u;
  }
  double v[NMON];
#pragma unroll
  for (int q = 0; q < NMON; ++q) v[q] = 0.0;
  for (int s = 0; s < NC; ++s) v[M_MASS + s] = double(dm[s]) + double(k.rref[s]) * double(nfluid);
  for (int c = 0; c < 3; ++c) v[M_MOM + c] = double(mom[c]);
  for (int s = 0; s < NS; ++s) v[mon_spec(s)] = double(dsp[s]) + double(k.cref[s]) * double(nfluid);
  v[M_NFLUID] = double(nfluid);
  v[M_NONFIN] = double(nonfin);
  // bookkeeping over every node
  const bool dep = a.geo_mode == GEO_DEPOSIT;
  double react = 0.0, depo = 0.0, nsolid = 0.0, tsolid = 0.0;
  const T* gcur = a.conjugate ? reinterpret_cast<const T*>(a.gs[parity]) : nullptr;
  for (long long n = tid; n < a.N; n += nthr) {
    const uint8_t fl = a.flags[n];
    nsolid += fl != FL_FLUID ? 1.0 : 0.0;
    const double acc = a.acc[n];
    if (acc != 0.0) {
      if (dep && fl != FL_REACTIVE) depo += acc; else react += acc;
    }
    if (gcur && fl != FL_FLUID) {
      T t = T(0);
#pragma unroll
      for (int q = 0; q < QC; ++q) t += gcur[(long long)q * a.N + n];
      tsolid += double(t);
    }
  }
  v[M_REACT] = react;
  v[M_DEPO] = depo;
  v[M_NSOLID] = nsolid;
  v[M_TSOLID] = tsolid;
  const int rows = a.ny * a.nz;
  for (int r = tid; r < rows; r += nthr)
    for (int s = 0; s < NS; ++s) {
      v[mon_in(s)] += a.inflow_row[s * rows + r];
      v[mon_out(s)] += a.outflow_row[s * rows + r];
    }
  for (int q = tid; q < WALLX_SLOTS; q += nthr) {
    v[M_WALLX] += a.wallx_slot[BANK_WALLX * WALLX_SLOTS + q];
    v[M_HEAT] += a.wallx_slot[BANK_HEAT * WALLX_SLOTS + q];
    v[M_PROD] += a.wallx_slot[BANK_PROD * WALLX_SLOTS + q];
    v[M_HEAT_S] += a.wallx_slot[BANK_HEAT_S * WALLX_SLOTS + q];
    v[M_HEAT_SRC] += a.wallx_slot[BANK_HEAT_SRC * WALLX_SLOTS + q];
  }
  block_reduce_store<NMON>(v, a.partials + (long long)blockIdx.x * NMON);
}

// ================================================================ node macroscopics

// rho^sigma, physical velocity (Eq. 1.19) and closed scalars of fluid node n; psi arrays must be
// current when Shan-Chen forces are on.
template <class L, class S, int NC, int NS>
__device__ __forceinline__ void node_macros(const Args& a, const Coef<typename Store<S>::T>& k, int n,
                                            uint32_t m, long long sn, int parity, typename Store<S>::T* rho_out,
                                            typename Store<S>::T* u_out, typename Store<S>::T* C_out) {
  using T = typename Store<S>::T;
  constexpr int Q = L::Q, QC = L::QC;
  const Nbr nb = nbr_of(a, n);
  T rho[NC], jx[NC], jy[NC], jz[NC], Fx[NC], Fy[NC], Fz[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    T f[Q];
    gather_flow_pl<L, S>(a.fplane[s], sn, a.slot, m, nb, parity, f, a.err, a.N, a.pitch);
    T r = T(0), ax = T(0), ay = T(0), az = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      r += f[i];
      ax += T(L::cx(i)) * f[i];
      ay += T(L::cy(i)) * f[i];
      az += T(L::cz(i)) * f[i];
    }
    r += k.rref[s];
    rho[s] = r; jx[s] = ax; jy[s] = ay; jz[s] = az;
    Fx[s] = r * k.g[0]; Fy[s] = r * k.g[1]; Fz[s] = r * k.g[2];
  }
  if (a.sc_on) {
    for (int s = 0; s < NC; ++s) {
      const T pself = reinterpret_cast<const T*>(a.psi[s])[n];
      for (int s2 = 0; s2 < NC; ++s2) {
        const T* ps = reinterpret_cast<const T*>(a.psi[s2]);
        T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          const T pv = flow_wall<L>(m, i) ? k.psi_wall : ps[nb.at(L::cx(i), L::cy(i), L::cz(i))];
          ax += T(L::w(i)) * pv * T(L::cx(i));
          ay += T(L::w(i)) * pv * T(L::cy(i));
          az += T(L::w(i)) * pv * T(L::cz(i));
        }
        const T Gss = k.G[s][s2];
        Fx[s] -= pself * Gss * ax; Fy[s] -= pself * Gss * ay; Fz[s] -= pself * Gss * az;
      }
    }
  }
  if (a.ads_on) {
    T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (flow_wall<L>(m, i)) {
        ax += T(L::w(i)) * T(L::cx(i));
        ay += T(L::w(i)) * T(L::cy(i));
        az += T(L::w(i)) * T(L::cz(i));
      }
    for (int s = 0; s < NC; ++s) {
      const T ga = k.G_ads[s] * rho[s];
      Fx[s] -= ga * ax; Fy[s] -= ga * ay; Fz[s] -= ga * az;
    }
  }
  T rt = T(0), mx = T(0), my = T(0), mz = T(0);
  for (int s = 0; s < NC; ++s) {
    rt += rho[s];
    mx += jx[s] + T(0.5) * Fx[s];
    my += jy[s] + T(0.5) * Fy[s];
    mz += jz[s] + T(0.5) * Fz[s];
  }
  for (int s = 0; s < NC; ++s) rho_out[s] = rho[s];
  u_out[0] = mx / rt;
  u_out[1] = my / rt;
  u_out[2] = mz / rt;
  T hh[NS > 0 ? NS : 1][QC];
#pragma unroll
  for (int s = 0; s < NS; ++s)
    gather_scal_pl<L, typename ScalarOf<S>::type>(a.hplane[s], sn, a.slot, m, nb, parity, hh[s], a.err, a.N, a.pitch);
  T rl[QC], gain = T(0);
#pragma unroll
  for (int j = 0; j < QC; ++j) rl[j] = T(0);
  if (NS > 1 && a.conjugate)
    close_conjugate<L, T>(hh[0], hh[NS > 1 ? 1 : 0], m, k, a, nb, reinterpret_cast<const T*>(a.gs[parity]),
                          [&](int j, T r, T) { rl[j] = r; });
  else if (NS > 1 && a.arrhenius)
    close_thermal<L, T>(hh[0], hh[NS > 1 ? 1 : 0], m, k, a.n_it, [&](int j, T r, T, T) { rl[j] = r; });
  else if (NS > 0)
    close_scalar<L, T>(hh[0], m, k, [&](int j, T Cb, T) { rl[j] = k.kr * Cb; });
  if (NS > 1 && a.product) close_product<L, T>(hh[NS - 1], m, k, rl, gain);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    T C = k.cref[s];
#pragma unroll
    for (int j = 0; j < QC; ++j) C += hh[s][j];
    C_out[s] = C;
  }
}

// Macroscopic fields of every node into FP64 staging (solid nodes read 0).
template <class L, class S, int NC, int NS>
__global__ void __launch_bounds__(256) k_moments(const Args a, const Coef<typename Store<S>::T> k,
                                                 const int parity) {
  using T = typename Store<S>::T;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const long long N = a.N;
  const uint32_t m = a.mask[n];
  T rho[NC], u[3], C[NS > 0 ? NS : 1];
  if (m & 1u) {
    node_macros<L, S, NC, NS>(a, k, int(n), m, (long long)a.slot[n], parity, rho, u, C);
  } else {
    for (int s = 0; s < NC; ++s) rho[s] = T(0);
    u[0] = u[1] = u[2] = T(0);
    for (int s = 0; s < NS; ++s) C[s] = T(0);
    if (NS > 1 && a.conjugate) {
      // the solid temperature (Eq. macroreacb_solid)
      const T* g = reinterpret_cast<const T*>(a.gs[parity]);
      T t = T(0);
#pragma unroll
      for (int q = 0; q < L::QC; ++q) t += g[(long long)q * N + n];
      C[NS > 1 ? 1 : 0] = t;
    }
  }
  for (int s = 0; s < NC; ++s) a.d_rho[s * N + n] = double(rho[s]);
  for (int c = 0; c < 3; ++c) a.d_u[c * N + n] = double(u[c]);
  for (int s = 0; s < NS; ++s) a.d_C[s * N + n] = double(C[s]);
}

// Residual partials over the fluid list against compute-type snapshots [4][pitch] (u, C) held
// at the nodes' storage slots, which are replaced: sum (u - u_s)^2, sum u^2, sum (C - C_s)^2,
// sum C^2.  (A re-slotting invalidates the snapshots; the runtime then skips one evaluation.)
template <class L, class S, int NC, int NS>
__global__ void __launch_bounds__(256) k_resid(const Args a, const Coef<typename Store<S>::T> k,
                                               const int parity) {
  using T = typename Store<S>::T;
  T* snap = reinterpret_cast<T*>(a.snap);
  const long long P = a.pitch;
  T du = T(0), uu = T(0), dc = T(0), cc = T(0);
  const unsigned int count = a.fluid_count[0], base = a.fluid_count[1];
  for (unsigned int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    const int n = int(a.fluid_list[e]);
    const uint32_t m = a.mask[n];
    if (!(m & 1u)) continue;
    const long long sn = e < base ? (long long)e : (long long)a.slot[n];
    T rho[NC], u[3], C[NS > 0 ? NS : 1];
    node_macros<L, S, NC, NS>(a, k, n, m, sn, parity, rho, u, C);
    for (int c = 0; c < 3; ++c) {
      const T d = u[c] - snap[c * P + sn];
      du += d * d;
      uu += u[c] * u[c];
      snap[c * P + sn] = u[c];
    }
    if (NS > 0) {
      const T d = C[0] - snap[3 * P + sn];
      dc += d * d;
      cc += C[0] * C[0];
      snap[3 * P + sn] = C[0];
    }
  }
  double v[4] = {double(du), double(uu), double(dc), double(cc)};
  block_reduce_store<4>(v, a.partials + (long long)blockIdx.x * 4);
}

// ================================================================ init / pop I/O

// Equilibrium populations from FP64 staging fields (Eq. 6, Eq. therpopeq_species), natural
// layout, computed in the compute type.
template <class L, class S, int NC, int NS>
__global__ void __launch_bounds__(256) k_init(const Args a, const Coef<typename Store<S>::T> k) {
  using T = typename Store<S>::T;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const bool fluid = a.flags[n] == FL_FLUID;
  const long long sn = a.slot[n];
  const T ux = T(a.d_u[n]), uy = T(a.d_u[a.N + n]), uz = (L::D == 3) ? T(a.d_u[2 * a.N + n]) : T(0);
  for (int s = 0; s < NC; ++s) {
    S* fs = reinterpret_cast<S*>(a.f[s]);
    const T r = T(a.d_rho[s * a.N + n]);
    const T dr = T(a.d_rho[s * a.N + n] - double(k.rref[s]));
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const T v = fluid ? feq_dev<L, T>(i, r, dr, ux, uy, uz) : T(0);
      Store<S>::st(fs + (long long)i * a.pitch + sn, v);
    }
  }
  for (int s = 0; s < NS; ++s) {
    using SC = typename ScalarOf<S>::type;
    SC* hs = reinterpret_cast<SC*>(a.h[s]);
    const T C = T(a.d_C[s * a.N + n]);
    const T dC = T(a.d_C[s * a.N + n] - double(k.cref[s]));
#pragma unroll
    for (int j = 0; j < L::QC; ++j) {
      const T cu = T(L::cx(j)) * ux + T(L::cy(j)) * uy + T(L::cz(j)) * uz;
      const T wj = scal_w<T>(j, k);
      const T v = fluid ? wj * (dC + C * cu * k.ics2c) : T(0);
      Store<SC>::st(hs + (long long)j * a.pitch + sn, v);
    }
  }
}

// Natural-order FP64 copy of the pre-collision populations (dir = 0: device state -> out,
// dir = 1: in -> device state at the current layout parity).  Full values (reference added
// back).  Solid nodes read as 0.
template <class L, class S, int NC, int NS>
__global__ void __launch_bounds__(256) k_pops_io(const Args a, const Coef<typename Store<S>::T> k,
                                                 const int parity, const int dir, double* fio,
                                                 double* hio) {
  using T = typename Store<S>::T;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  const int n = x + a.nx * (y + a.ny * z);
  const uint32_t m = a.mask[n];
  const bool fluid = (m & 1u) != 0u;
  const Nbr nb = make_nbr(a, x, y, z);
  const long long N = a.N, P = a.pitch;
  const long long sn = a.slot[n];
  if (fio) {
    for (int s = 0; s < NC; ++s) {
      S* fs = reinterpret_cast<S*>(a.f[s]);
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        double* io = fio + ((long long)s * L::Q + i) * N + n;
        if (!fluid) {
          if (dir == 0) *io = 0.0;
          continue;
        }
        S* p;
        if (parity == 0 || i == 0 || flow_wall<L>(m, L::opp(i)))
          p = fs + (long long)i * P + sn;
        else
          p = fs + (long long)L::opp(i) * P + a.slot[nb.at(-L::cx(i), -L::cy(i), -L::cz(i))];
        const double sh = L::w(i) * double(k.rref[s]);
        if (dir == 0) *io = double(Store<S>::ldv(p)) + sh;
        else Store<S>::st(p, T(*io - sh));
      }
    }
  }
  if (hio) {
    using SC = typename ScalarOf<S>::type;
    for (int s = 0; s < NS; ++s) {
      SC* hs = reinterpret_cast<SC*>(a.h[s]);
#pragma unroll
      for (int j = 0; j < L::QC; ++j) {
        double* io = hio + ((long long)s * L::QC + j) * N + n;
        if (!fluid) {
          if (dir == 0) *io = 0.0;
          continue;
        }
        SC* p;
        if (parity == 0 || j == 0 || MaskBits<L>::code(m, L::opp(j)) != 0u)
          p = hs + (long long)j * P + sn;
        else
          p = hs + (long long)L::opp(j) * P + a.slot[nb.at(-L::cx(j), -L::cy(j), -L::cz(j))];
        const double sh = double(scal_w<T>(j, k)) * double(k.cref[s]);
        if (dir == 0) *io = double(Store<SC>::ldv(p)) + sh;
        else Store<SC>::st(p, T(*io - sh));
      }
    }
  }
}

// ================================================================ link masks

// Neighbour of (x, y, z) in direction (dx, dy, dz) under per-axis periodicity: -1 if outside.
// *axis_out receives the first axis that left the box (0, 1, 2) or -1.
__device__ __forceinline__ long long nbr_checked(const Args& a, int x, int y, int z, int dx, int dy,
                                                 int dz, const int* per, int* axis_out) {
  int v[3] = {x + dx, y + dy, z + dz};
  const int n3[3] = {a.nx, a.ny, a.nz};
  *axis_out = -1;
  for (int c = 0; c < 3; ++c) {
    if (v[c] < 0 || v[c] >= n3[c]) {
      if (!per[c]) {
        *axis_out = c;
        return -1;
      }
      v[c] = v[c] < 0 ? v[c] + n3[c] : v[c] - n3[c];
    }
  }
  return v[0] + (long long)a.nx * (v[1] + (long long)a.ny * v[2]);
}

template <class L>
__device__ uint32_t compute_mask(const Args& a, int x, int y, int z) {
  const long long n = x + (long long)a.nx * (y + (long long)a.ny * z);
  if (a.flags[n] != FL_FLUID) return 0u;
  uint32_t m = 1u;
  int ax;
  for (int i = 1; i < L::Q; ++i) {
    const long long q = nbr_checked(a, x, y, z, L::cx(i), L::cy(i), L::cz(i), a.per, &ax);
    if (q < 0 || a.flags[q] != FL_FLUID) m |= 1u << i;
  }
  const int perc[3] = {a.open_x ? 0 : a.per[0], a.per[1], a.per[2]};
  for (int j = 1; j < L::QC; ++j) {
    const long long q = nbr_checked(a, x, y, z, L::cx(j), L::cy(j), L::cz(j), perc, &ax);
    uint32_t code;
    if (q < 0) code = (ax == 0 && a.open_x) ? 3u : 1u;
    else {
      const uint8_t fl = a.flags[q];
      code = fl == FL_FLUID ? 0u : (fl == FL_REACTIVE ? 2u : 1u);
    }
    m |= code << (MaskBits<L>::SC_BASE + 2 * (j - 1));
  }
  return m;
}

template <class L>
__global__ void __launch_bounds__(256) k_masks(const Args a) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const int x = int(n % a.nx);
  const int y = int((n / a.nx) % a.ny);
  const int z = int(n / ((long long)a.nx * a.ny));
  a.mask[n] = compute_mask<L>(a, x, y, z);
}

// ================================================================ node lists

// Ordered stream compaction of the nodes that satisfy a predicate, in chunks of 1024 positions:
// count, scan, write.  PRED 0: fluid nodes (the step kernel's work list), in brick order (below);
// also assigns the storage slots.  PRED 1: reactive solids touching the fluid through a scalar
// link (the dissolution interface list, node order; also marks listed[]).
//
// Brick order: the domain is cut into bricks of BX x BY x BZ nodes, visited x-fastest, with the
// nodes x-fastest inside a brick.  A warp's 32 consecutive list entries then lie in a compact
// block, so the neighbour cells an odd step reads and writes fall in a few nearby slot ranges
// instead of nine distant rows.
#ifndef LBM_BRICK_X
#define LBM_BRICK_X 32
#endif
#ifndef LBM_BRICK_Y
#define LBM_BRICK_Y 8
#endif
#ifndef LBM_BRICK_Z
#define LBM_BRICK_Z 4
#endif
template <class L>
struct Brick {
  static constexpr int X = LBM_BRICK_X, Y = LBM_BRICK_Y, Z = L::D == 3 ? LBM_BRICK_Z : 1;
  static constexpr long long V = (long long)X * Y * Z;
};

// node at position t of the brick order, or -1 for a position outside the domain
template <class L>
__device__ __forceinline__ long long brick_node(const Args& a, long long t) {
  using B = Brick<L>;
  const long long b = t / B::V;
  const int l = int(t - b * B::V);
  const long long nbx = (a.nx + B::X - 1) / B::X, nby = (a.ny + B::Y - 1) / B::Y;
  const long long x = (b % nbx) * B::X + l % B::X;
  const long long y = ((b / nbx) % nby) * B::Y + (l / B::X) % B::Y;
  const long long z = (b / (nbx * nby)) * B::Z + l / (B::X * B::Y);
  if (x >= a.nx || y >= a.ny || z >= a.nz) return -1;
  return x + a.nx * (y + a.ny * z);
}

template <class L>
__device__ __forceinline__ bool has_fluid_scalar_neighbour(const Args& a, int x, int y, int z);

// node of position t in the order of list PRED (-1: no node), and whether it enters the list
template <class L, int PRED>
__device__ __forceinline__ bool list_pred(const Args& a, long long t, long long* node) {
  const long long n = PRED == 0 ? brick_node<L>(a, t) : (t < a.N ? t : -1);
  *node = n;
  if (n < 0) return false;
  if (PRED == 0) return a.flags[n] == FL_FLUID;
  if (a.flags[n] != FL_REACTIVE) return false;
  return has_fluid_scalar_neighbour<L>(a, int(n % a.nx), int((n / a.nx) % a.ny),
                                       int(n / ((long long)a.nx * a.ny)));
}

__device__ __forceinline__ unsigned int block_count(unsigned int b, unsigned int* wsum) {
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  unsigned int v = 0;
  if (threadIdx.x < 32) {
    v = wsum[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

template <class L, int PRED>
__global__ void __launch_bounds__(1024) k_list_count(const Args a) {
  __shared__ unsigned int wsum[32];
  const long long t = blockIdx.x * 1024ll + threadIdx.x;
  long long n;
  const bool f = list_pred<L, PRED>(a, t, &n);
  const unsigned int cf = block_count(__ballot_sync(0xffffffffu, f), wsum);
  if (threadIdx.x == 0) a.block_counts[blockIdx.x] = cf;
  if (PRED == 0) {
    const unsigned int cv = block_count(__ballot_sync(0xffffffffu, n >= 0), wsum);
    if (threadIdx.x == 0) a.block_counts_v[blockIdx.x] = cv;
  }
}

// exclusive scan of the chunk counts by one block; the total goes to count[0] and count[1]
template <int DUMMY = 0>
__global__ void __launch_bounds__(1024) k_list_scan(unsigned int* counts, unsigned int nchunks,
                                                    unsigned int* count) {
  __shared__ unsigned int part[1024];
  __shared__ unsigned int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (unsigned int base = 0; base < nchunks; base += 1024) {
    const unsigned int i = base + threadIdx.x;
    const unsigned int v = i < nchunks ? counts[i] : 0u;
    part[threadIdx.x] = v;
    __syncthreads();
    for (unsigned int o = 1; o < 1024; o <<= 1) {
      const unsigned int t = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
      __syncthreads();
      part[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nchunks) counts[i] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    count[0] = carry;
    count[1] = carry;
  }
}

// exclusive prefix of ballot b over the block (chunk offset off added)
__device__ __forceinline__ unsigned int block_prefix(unsigned int b, unsigned int off, unsigned int* wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wsum[wid] = __popc(b);
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned int v = wsum[threadIdx.x], incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (threadIdx.x >= o) incl += t;
    }
    wsum[threadIdx.x] = incl - v;
  }
  __syncthreads();
  const unsigned int pos = off + wsum[wid] + __popc(b & ((1u << lane) - 1u));
  __syncthreads();
  return pos;
}

// PRED 0 also assigns the new storage slots: fluid nodes take their list position, solid nodes
// follow the fluid total in brick order (slot_new).
template <class L, int PRED>
__global__ void __launch_bounds__(1024) k_list_write(const Args a, uint32_t* list) {
  __shared__ unsigned int wsum[32];
  const long long t = blockIdx.x * 1024ll + threadIdx.x;
  long long n;
  const bool f = list_pred<L, PRED>(a, t, &n);
  const unsigned int pos = block_prefix(__ballot_sync(0xffffffffu, f), a.block_counts[blockIdx.x], wsum);
  if (PRED == 0) {
    const unsigned int vpos = block_prefix(__ballot_sync(0xffffffffu, n >= 0), a.block_counts_v[blockIdx.x], wsum);
    if (n >= 0) a.slot_new[n] = f ? pos : a.fluid_count[0] + (vpos - pos);
  }
  if (f) {
    list[pos] = (uint32_t)n;
    if (PRED == 1) a.listed[n] = 1;
  }
}

// ================================================================ interface list

template <class L>
__device__ __forceinline__ bool has_fluid_scalar_neighbour(const Args& a, int x, int y, int z) {
  const int perc[3] = {a.open_x ? 0 : a.per[0], a.per[1], a.per[2]};
  int ax;
  for (int j = 1; j < L::QC; ++j) {
    const long long q = nbr_checked(a, x, y, z, L::cx(j), L::cy(j), L::cz(j), perc, &ax);
    if (q >= 0 && a.flags[q] == FL_FLUID) return true;
  }
  return false;
}

__device__ __forceinline__ void push_iface(const Args& a, long long n) {
  const unsigned int e = atomicAdd(a.iface_count, 1u);
  if (e < a.N) a.iface_list[e] = (uint32_t)n;
  else atomicOr(a.err, ERR_CAPACITY);
}

// ================================================================ geometry flips

__device__ __forceinline__ bool cas_flag(uint8_t* flags, long long n, uint8_t expect, uint8_t desired,
                                         int* err) {
  unsigned int* w = reinterpret_cast<unsigned int*>(flags + (n & ~3ll));
  const int sh = int(n & 3) * 8;
  unsigned int old = atomicAdd(w, 0u);
  for (int it = 0; it < 64; ++it) {
    if (((old >> sh) & 0xffu) != expect) return false;
    const unsigned int nw = (old & ~(0xffu << sh)) | (unsigned(desired) << sh);
    const unsigned int prev = atomicCAS(w, old, nw);
    if (prev == old) return true;
    old = prev;
  }
  atomicOr(err, ERR_CAS);
  return false;
}

// FLIPPING (0b11) -> v in {FLUID 0b00, SOLID 0b01, REACTIVE 0b10} with one atomic operation,
// so a concurrent reader never sees an intermediate value.
__device__ __forceinline__ void leave_flipping(uint8_t* flags, long long n, uint8_t v) {
  unsigned int* w = reinterpret_cast<unsigned int*>(flags + (n & ~3ll));
  const int sh = int(n & 3) * 8;
  atomicAnd(w, ~((3u ^ unsigned(v)) << sh));
}

__device__ __forceinline__ void coords_of(const Args& a, long long n, int* x, int* y, int* z) {
  *x = int(n % a.nx);
  *y = int((n / a.nx) % a.ny);
  *z = int(n / ((long long)a.nx * a.ny));
}

// One block processes the whole flip list in phases separated by __syncthreads:
//   0 claim entries (validate, mark FLIPPING, drop duplicates)
//   1 dissolution: neighbour means (flags before the flip);  deposition: removed sums
//   2 write populations of the new fluid nodes / hand populations to remaining neighbours
//   3 final flags;  4 link masks of every node around a flipped one;  5 clear the list
// parity_next is the layout parity of the state the flips act on (steps completed & 1).
template <class L, class S, int NC, int NS>
__global__ void __launch_bounds__(1024) k_flip(const Args a, const Coef<typename Store<S>::T> k,
                                               const int parity_next) {
  using T = typename Store<S>::T;
  using SC = typename ScalarOf<S>::type;   // scalar lattices' storage
  constexpr int Q = L::Q, QC = L::QC;
  const unsigned int cnt_raw = *a.flip_count;
  const unsigned int cnt = cnt_raw < a.flip_cap ? cnt_raw : a.flip_cap;
  if (cnt == 0) return;
  const int percf[3] = {a.per[0], a.per[1], a.per[2]};
  const int percs[3] = {a.open_x ? 0 : a.per[0], a.per[1], a.per[2]};
  const long long P = a.pitch;
  const bool dissolve = a.geo_mode == GEO_DISSOLVE;
  // flip monitors: injected mass [0, 2), injected scalars [2, 5), removed mass [5, 7), removed
  // scalars [7, 10), solid temperature taken from the solid lattice [10]
  __shared__ double sred[11];
  if (threadIdx.x < 11) sred[threadIdx.x] = 0.0;
  // ---- phase 0: claim
  for (unsigned int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const long long s = a.flip_list[e];
    bool ok;
    if (dissolve)
      ok = a.flags[s] == FL_REACTIVE && consumed(a, a.acc[s]) &&
           cas_flag(a.flags, s, FL_REACTIVE, FL_FLIPPING, a.err);
    else
      ok = a.flags[s] == FL_FLUID && a.acc[s] > 1.0 && cas_flag(a.flags, s, FL_FLUID, FL_FLIPPING, a.err);
    if (!ok) a.flip_list[e] = 0xffffffffu;
  }
  __syncthreads();
  // ---- phase 1
  for (unsigned int e = threadIdx.x; e < cnt; e += blockDim.x) {
    if (a.flip_list[e] == 0xffffffffu) continue;
    const long long s = a.flip_list[e];
    int x, y, z;
    coords_of(a, s, &x, &y, &z);
    if (dissolve) {
      double sr[2] = {0.0, 0.0}, sc[3] = {0.0, 0.0, 0.0};
      int count = 0;
      int ax;
      for (int i = 1; i < Q; ++i) {
        const long long q = nbr_checked(a, x, y, z, L::cx(i), L::cy(i), L::cz(i), percf, &ax);
        if (q < 0 || a.flags[q] != FL_FLUID) continue;
        ++count;
        int qx, qy, qz;
        coords_of(a, q, &qx, &qy, &qz);
        const Nbr nq = make_nbr(a, qx, qy, qz);
        const uint32_t mq = a.mask[q];
        for (int c = 0; c < NC; ++c) {
          T f[Q];
          gather_flow<L, S>(reinterpret_cast<const S*>(a.f[c]), P, a.slot[q], a.slot, mq, nq, parity_next, f);
          double r = double(k.rref[c]);
          for (int j = 0; j < Q; ++j) r += double(f[j]);
          sr[c] += r;
        }
        T hh[NS > 0 ? NS : 1][QC];
        for (int c = 0; c < NS; ++c)
          gather_scal<L, SC>(reinterpret_cast<const SC*>(a.h[c]), P, a.slot[q], a.slot, mq, nq, parity_next, hh[c]);
        T rl[QC], gain = T(0);
        for (int j = 0; j < QC; ++j) rl[j] = T(0);
        if (NS > 1 && a.conjugate)
          close_conjugate<L, T>(hh[0], hh[NS > 1 ? 1 : 0], mq, k, a, nq,
                                reinterpret_cast<const T*>(a.gs[parity_next]), [&](int j, T r, T) { rl[j] = r; });
        else if (NS > 1 && a.arrhenius)
          close_thermal<L, T>(hh[0], hh[NS > 1 ? 1 : 0], mq, k, a.n_it, [&](int j, T r, T, T) { rl[j] = r; });
        else if (NS > 0)
          close_scalar<L, T>(hh[0], mq, k, [&](int j, T Cb, T) { rl[j] = k.kr * Cb; });
        if (NS > 1 && a.product) close_product<L, T>(hh[NS - 1], mq, k, rl, gain);
        for (int c = 0; c < NS; ++c) {
          double C = double(k.cref[c]);
          for (int j = 0; j < QC; ++j) C += double(hh[c][j]);
          sc[c] += C;
        }
      }
      double* sc4 = a.flip_scratch + 5ll * e;
      if (count == 0) {
        leave_flipping(a.flags, s, FL_REACTIVE);   // nothing to average: stays solid
        a.flip_list[e] = 0xffffffffu;
        continue;
      }
      for (int c = 0; c < 2; ++c) sc4[c] = sr[c] / count;
      for (int c = 0; c < 3; ++c) sc4[2 + c] = sc[c] / count;
    } else {
      const Nbr ns = make_nbr(a, x, y, z);
      const uint32_t ms = a.mask[s];
      for (int c = 0; c < NC; ++c) {
        T f[Q];
        gather_flow<L, S>(reinterpret_cast<const S*>(a.f[c]), P, a.slot[s], a.slot, ms, ns, parity_next, f);
        double r = double(k.rref[c]);
        for (int j = 0; j < Q; ++j) r += double(f[j]);
        atomicAdd(&sred[5 + c], r);
      }
      for (int c = 0; c < NS; ++c) {
        T h[QC];
        gather_scal<L, SC>(reinterpret_cast<const SC*>(a.h[c]), P, a.slot[s], a.slot, ms, ns, parity_next, h);
        double C = double(k.cref[c]);
        for (int j = 0; j < QC; ++j) C += double(h[j]);
        atomicAdd(&sred[7 + c], C);
      }
    }
  }
  __syncthreads();
  // ---- phase 2
  for (unsigned int e = threadIdx.x; e < cnt; e += blockDim.x) {
    if (a.flip_list[e] == 0xffffffffu) continue;
    const long long s = a.flip_list[e];
    const long long ss = a.slot[s];   // storage slot of the flipping node
    int x, y, z;
    coords_of(a, s, &x, &y, &z);
    int ax;
    if (dissolve) {
      const double* sc4 = a.flip_scratch + 5ll * e;
      for (int c = 0; c < NC; ++c) {
        S* fs = reinterpret_cast<S*>(a.f[c]);
        const double r = sc4[c];
        atomicAdd(&sred[c], r);
        for (int j = 0; j < Q; ++j) {
          const T tv = T(L::w(j) * (r - double(k.rref[c])));   // f_eq(rho_bar, u = 0) - w rref
          if (parity_next == 0 || j == 0) {
            Store<S>::st(fs + (long long)j * P + ss, tv);
            continue;
          }
          const long long src = nbr_checked(a, x, y, z, -L::cx(j), -L::cy(j), -L::cz(j), percf, &ax);
          const uint8_t fl = src < 0 ? FL_SOLID : a.flags[src];
          if (fl == FL_FLUID) {
            S* from = fs + (long long)L::opp(j) * P + a.slot[src];
            *(fs + (long long)j * P + ss) = *from;     // neighbour's bounced value moves
            Store<S>::st(from, tv);
          } else if (fl == FL_FLIPPING) {
            Store<S>::st(fs + (long long)L::opp(j) * P + a.slot[src], tv);
          } else {
            Store<S>::st(fs + (long long)j * P + ss, tv);
          }
        }
      }
      for (int c = 0; c < NS; ++c) {
        SC* hs = reinterpret_cast<SC*>(a.h[c]);
        double C = sc4[2 + c];
        if (c == 1 && a.conjugate) {
          // with conduction in the solid the new fluid node keeps its own temperature: its solid
          // populations leave the solid lattice
          T* g = reinterpret_cast<T*>(a.gs[parity_next]);
          C = 0.0;
          for (int q = 0; q < QC; ++q) {
            C += double(g[(long long)q * a.N + s]);
            g[(long long)q * a.N + s] = T(0);
          }
          atomicAdd(&sred[10], C);
        }
        atomicAdd(&sred[2 + c], C);
        for (int j = 0; j < QC; ++j) {
          const double wj = double(scal_w<T>(j, k));
          const T tv = T(wj * (C - double(k.cref[c])));       // h_eq(C_bar, u = 0) - w cref
          if (parity_next == 0 || j == 0) {
            Store<SC>::st(hs + (long long)j * P + ss, tv);
            continue;
          }
          const long long src = nbr_checked(a, x, y, z, -L::cx(j), -L::cy(j), -L::cz(j), percs, &ax);
          const uint8_t fl = src < 0 ? FL_SOLID : a.flags[src];
          if (fl == FL_FLUID) {
            SC* from = hs + (long long)L::opp(j) * P + a.slot[src];
            *(hs + (long long)j * P + ss) = *from;
            Store<SC>::st(from, tv);
          } else if (fl == FL_FLIPPING) {
            Store<SC>::st(hs + (long long)L::opp(j) * P + a.slot[src], tv);
          } else {
            Store<SC>::st(hs + (long long)j * P + ss, tv);
          }
        }
      }
    } else if (parity_next == 1) {
      // deposition in the swapped layout: a remaining fluid neighbour y = s + c_d now reads its
      // population from the new wall at (y, d); give it what s streamed toward it, (s, opp d)
      for (int c = 0; c < NC; ++c) {
        S* fs = reinterpret_cast<S*>(a.f[c]);
        for (int d = 1; d < Q; ++d) {
          const long long yn = nbr_checked(a, x, y, z, L::cx(d), L::cy(d), L::cz(d), percf, &ax);
          if (yn < 0 || a.flags[yn] != FL_FLUID) continue;
          *(fs + (long long)d * P + a.slot[yn]) = *(fs + (long long)L::opp(d) * P + ss);
        }
      }
      for (int c = 0; c < NS; ++c) {
        SC* hs = reinterpret_cast<SC*>(a.h[c]);
        for (int d = 1; d < QC; ++d) {
          const long long yn = nbr_checked(a, x, y, z, L::cx(d), L::cy(d), L::cz(d), percs, &ax);
          if (yn < 0 || a.flags[yn] != FL_FLUID) continue;
          *(hs + (long long)d * P + a.slot[yn]) = *(hs + (long long)L::opp(d) * P + ss);
        }
      }
    }
  }
  __syncthreads();
  // ---- phase 3: final flags; new fluid nodes join the fluid list (removed ones are skipped by
  // their mask until the next rebuild)
  for (unsigned int e = threadIdx.x; e < cnt; e += blockDim.x) {
    if (a.flip_list[e] == 0xffffffffu) continue;
    leave_flipping(a.flags, a.flip_list[e], dissolve ? FL_FLUID : FL_SOLID);
    if (dissolve) {
      const unsigned int pos = atomicAdd(a.fluid_count, 1u);
      if (pos < a.N) a.fluid_list[pos] = a.flip_list[e];
      else atomicOr(a.err, ERR_CAPACITY);
    }
  }
  __syncthreads();
  // ---- phase 4: masks around every flipped node
  for (unsigned int e = threadIdx.x; e < cnt; e += blockDim.x) {
    if (a.flip_list[e] == 0xffffffffu) continue;
    const long long s = a.flip_list[e];
    int x, y, z, ax;
    coords_of(a, s, &x, &y, &z);
    a.mask[s] = compute_mask<L>(a, x, y, z);
    for (int i = 1; i < Q; ++i) {
      const long long q = nbr_checked(a, x, y, z, L::cx(i), L::cy(i), L::cz(i), percf, &ax);
      if (q < 0) continue;
      int qx, qy, qz;
      coords_of(a, q, &qx, &qy, &qz);
      a.mask[q] = compute_mask<L>(a, qx, qy, qz);
    }
    if (dissolve) {
      // reactive solids that now touch the new fluid node join the interface list
      for (int j = 1; j < QC; ++j) {
        const long long q = nbr_checked(a, x, y, z, L::cx(j), L::cy(j), L::cz(j), percs, &ax);
        if (q >= 0 && a.flags[q] == FL_REACTIVE && cas_flag(a.listed, q, 0, 1, a.err)) push_iface(a, q);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 11 && sred[threadIdx.x] != 0.0) atomicAdd(a.flip_mon + threadIdx.x, sred[threadIdx.x]);
  if (threadIdx.x == 0) *a.flip_count = 0u;
}

// ================================================================ conduction in the solid

// Solid thermal lattice (Sec. 2.1.5, Eq. therpop_solid with g_s^eq = w T_s, Eq. macroreacb_solid):
// collision and streaming of every solid node, from gs[parity] into gs[parity ^ 1] (node-indexed
// planes, full values).  A population leaving toward another solid node streams there; one
// leaving toward a fluid node or through a face that is not periodic for the scalars is kept at
// the node as the arriving population of the opposite direction: at a closed face that is the
// reflection, at a fluid neighbour it is the solid side of the link that k_exchange replaces.
template <class L, class S>
__global__ void __launch_bounds__(256) k_solid(const Args a, const Coef<typename Store<S>::T> k,
                                               const int parity) {
  using T = typename Store<S>::T;
  constexpr int QC = L::QC;
  const T* gin = reinterpret_cast<const T*>(a.gs[parity]);
  T* gout = reinterpret_cast<T*>(a.gs[parity ^ 1]);
  const int perc[3] = {a.open_x ? 0 : a.per[0], a.per[1], a.per[2]};
  const long long N = a.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    if (a.flags[n] == FL_FLUID) continue;
    T g[QC];
    T Ts = T(0);
#pragma unroll
    for (int q = 0; q < QC; ++q) {
      g[q] = gin[(long long)q * N + n];
      Ts += g[q];
    }
    int x, y, z, ax;
    coords_of(a, n, &x, &y, &z);
#pragma unroll
    for (int q = 0; q < QC; ++q) {
      const T v = g[q] - (g[q] - scal_w<T>(q, k) * Ts) * k.oms;
      if (q == 0) {
        gout[n] = v;
        continue;
      }
      const long long d = nbr_checked(a, x, y, z, L::cx(q), L::cy(q), L::cz(q), perc, &ax);
      if (d >= 0 && a.flags[d] != FL_FLUID) gout[(long long)q * N + d] = v;
      else gout[(long long)L::opp(q) * N + n] = v;
    }
  }
}

// The exchange across every solid link of the temperature (Sec. 2.1.5, Eq. tempCon, fluxCon,
// reacRate), after the fluid step and the solid lattice's streaming.  For fluid node n and a
// direction j toward a solid node s = n + c_j (arriving direction i = opp(j)): the fluid
// population ho = h*_T,j that left n toward s (kept at n by the bounce-back of the step, in plane
// i) and the solid population go = g*_s,i that left s toward n (kept at s in plane j by k_solid)
// meet at one interface temperature T_b.  Each side receives 2 w T_b minus what it sent, and the
// link's energy in units of the fluid's rho c_p grows by the reaction heat Qp:
//     T_b = (c_fs ho + go + c_fs Qp / 2) / (w (c_fs + 1)).
// Qp = h_r k(T_b) C_b at a reactive link, where C_b = 2 hb / (2 w + k tau_c / (tau_c - 1/2)) closes
// the species population hb = h_C,j that has just streamed into n (read as the next step's
// gather reads it); T_b and C_b come from n_it + 1 fixed-point updates starting at the value
// without reaction, and k is kept for the next step's species closure.  Monitors: heat gained by
// the fluid side (bank HEAT), by the solid side (HEAT_S), reaction heat (HEAT_SRC).
template <class L, class S>
__global__ void __launch_bounds__(256) k_exchange(const Args a, const Coef<typename Store<S>::T> k,
                                                  const int parity_next) {
  using T = typename Store<S>::T;
  using SC = typename ScalarOf<S>::type;
  constexpr int QC = L::QC;
  T* g = reinterpret_cast<T*>(a.gs[parity_next]);
  T* kb = reinterpret_cast<T*>(a.kb);
  const int perc[3] = {a.open_x ? 0 : a.per[0], a.per[1], a.per[2]};
  const T sh0 = k.wca * k.cref[0], sh1 = k.wca * k.cref[1];
  const T w = k.wca, cf = k.cfs;
  const T den = w * (cf + T(1));
  T heat = T(0), heat_s = T(0), src_q = T(0);
  const unsigned int count = a.fluid_count[0], base = a.fluid_count[1];
  for (unsigned int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    const int n = int(LBM_CHK(a.err, a.fluid_list[e], a.N));
    const uint32_t m = a.mask[n];
    if (!(m & 1u)) continue;
    bool any = false;
#pragma unroll
    for (int j = 1; j < QC; ++j) {
      const uint32_t c = MaskBits<L>::code(m, j);
      any |= (c == 1u || c == 2u);
    }
    if (!any) continue;
    const long long sn = e < base ? (long long)e : (long long)a.slot[n];
    int x, y, z, ax;
    coords_of(a, n, &x, &y, &z);
    const Nbr nb = make_nbr(a, x, y, z);
#pragma unroll
    for (int j = 1; j < QC; ++j) {
      const uint32_t c = MaskBits<L>::code(m, j);
      if (c != 1u && c != 2u) continue;
      const long long s = nbr_checked(a, x, y, z, L::cx(j), L::cy(j), L::cz(j), perc, &ax);
      if (s < 0) continue;   // a closed face: plain bounce-back
      const int i = L::opp(j);
      SC* hp = reinterpret_cast<SC*>(a.hplane[1][i]) + LBM_CHK(a.err, sn, a.pitch);
      T* gp = g + (long long)j * a.N + s;
      const T ho = Store<SC>::ld(hp) + sh1;
      const T go = *gp;
      T Tb = (cf * ho + go) / den;
      T Qp = T(0);
      if (c == 2u) {
        // the species population moving toward the wall, where the next step gathers it
        const SC* bp;
        if (parity_next == 0 || MaskBits<L>::code(m, i) != 0u)
          bp = reinterpret_cast<const SC*>(a.hplane[0][j]) + LBM_CHK(a.err, sn, a.pitch);
        else
          bp = reinterpret_cast<const SC*>(a.hplane[0][i]) +
               LBM_CHK(a.err, (long long)__ldg(a.slot + LBM_CHK(a.err, nb.at(-L::cx(j), -L::cy(j), -L::cz(j)), a.N)),
                       a.pitch);
        const T hb = Store<SC>::ld(bp) + sh0;
        T kt = T(0);
        for (int it = 0; it <= a.n_it; ++it) {
          kt = k.arrA * exp(-k.arrTa / Tb);
          const T Cb = T(2) * hb / (T(2) * w + kt * k.fc);
          Qp = k.hr * kt * Cb;
          Tb = (cf * ho + go + T(0.5) * cf * Qp) / den;
        }
        kb[(long long)(i - 1) * a.N + n] = kt;
      }
      const T hn = T(2) * w * Tb - ho;
      const T gn = T(2) * w * Tb - go;
      Store<SC>::st(hp, hn - sh1);
      *gp = gn;
      heat += hn - ho;
      heat_s += gn - go;
      src_q += Qp;
    }
  }
  const int lane_slot = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % WALLX_SLOTS;
  const T vals[3] = {heat, heat_s, src_q};
  const int banks[3] = {BANK_HEAT, BANK_HEAT_S, BANK_HEAT_SRC};
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (__ballot_sync(0xffffffffu, vals[b] != T(0))) {
      const T v = warp_sum(vals[b]);
      if ((threadIdx.x & 31) == 0) atomicAdd(a.wallx_slot + banks[b] * WALLX_SLOTS + lane_slot, widen(v));
    }
  }
}

// The solid thermal lattice at rest equilibrium with the temperature given for each solid node
// (row 1 of the staged scalar fields): g_q = w_q T into gs[0]; gs[1] and the exchange's rate
// constants cleared (NaN: no exchange yet).
template <class L, class S>
__global__ void __launch_bounds__(256) k_solid_init(const Args a, const Coef<typename Store<S>::T> k) {
  using T = typename Store<S>::T;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  T* g0 = reinterpret_cast<T*>(a.gs[0]);
  T* g1 = reinterpret_cast<T*>(a.gs[1]);
  T* kb = reinterpret_cast<T*>(a.kb);
  const bool solid = a.flags[n] != FL_FLUID;
  const double Tn = a.d_C[a.N + n];
#pragma unroll
  for (int q = 0; q < L::QC; ++q) {
    g0[(long long)q * a.N + n] = solid ? T(double(scal_w<T>(q, k)) * Tn) : T(0);
    g1[(long long)q * a.N + n] = T(0);
    if (q > 0) kb[(long long)(q - 1) * a.N + n] = T(NAN);
  }
}

}  // namespace lbm
