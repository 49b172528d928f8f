// runtime.cu -- context, device memory, step sequencing and the C ABI of include/lbm.h.
//
// One lbm_ctx owns every device buffer of one domain on one GPU.  lbm_step enqueues, per time
// step: the psi pass (Shan-Chen runs only), the fused step kernel, the geometry-flip kernel
// every N_geo steps, and the monitor / residual kernels every N_mon steps.  Nothing here falls
// back to host arithmetic: every step of the update runs in the kernels of kernels.cuh.
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "launch.cuh"

using namespace lbm;

struct lbm_ctx {
  int lattice = 0;
  int nx = 0, ny = 0, nz = 0;
  long long N = 0, pitch = 0;
  int Qf = 0, Qc = 0;
  lbm_params p{};
  cudaStream_t stream = nullptr;
  const KernelSet* ks = nullptr;
  size_t elem = 0;                 // bytes per stored flow population
  size_t elem_h = 0;               // bytes per stored scalar population
  Args a{};
  long long step = 0;
  bool fields_set = false;
  bool have_snap = false;
  int res_evals = 0;               // residual evaluations since the fields were set
  long long launches = 0;
  bool profile = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used;
  std::string err;
  std::vector<void*> allocs;
  double* mon_host = nullptr;      // pinned [NMON + 12]: monitors, then the 11 flip monitors
  void* f_alt[2] = {nullptr, nullptr};   // second population buffers: targets of re-slotting
  void* h_alt[3] = {nullptr, nullptr, nullptr};
  int nlat = 0;                    // scalar lattices: the given scalars, then the product if any
  // CUDA graphs of one even + odd step pair, keyed by which of the two steps end with a
  // geometry update; rebuilt whenever the kernel arguments change (re-slotting)
  cudaStream_t cap_stream = nullptr;
  long long gen = 0;               // bumped whenever the arguments or the fluid list change
  cudaGraphExec_t pair_exec[4] = {nullptr, nullptr, nullptr, nullptr};
  long long pair_launches[4] = {0, 0, 0, 0};
  bool graphs_ok = true;
};

namespace {

thread_local std::string g_create_err;   // message of the last failed lbm_create on this thread

lbm_status fail(lbm_ctx* c, lbm_status st, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return st;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
  return fail(c, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                               \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);     \
  } while (0)

#define LAUNCH(call)                                           \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    c->launches += 1;                                          \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);     \
  } while (0)

lbm_status dalloc(lbm_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LBM_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  return LBM_OK;
}

const KernelSet* pick(int lattice, int precision) {
  if (lattice == LBM_D2Q9_D2Q5) {
    switch (precision) {
      case LBM_FP64: return &kernels_d2_f64();
      case LBM_FP32: return &kernels_d2_f32();
      case LBM_FP16_SHIFTED: return &kernels_d2_f16();
      case LBM_BF16_SHIFTED: return &kernels_d2_bf16();
      case LBM_FP16_SHIFTED_S32: return &kernels_d2_f16s32();
      case LBM_BF16_SHIFTED_S32: return &kernels_d2_bf16s32();
    }
  } else {
    switch (precision) {
      case LBM_FP64: return &kernels_d3_f64();
      case LBM_FP32: return &kernels_d3_f32();
      case LBM_FP16_SHIFTED: return &kernels_d3_f16();
      case LBM_BF16_SHIFTED: return &kernels_d3_bf16();
      case LBM_FP16_SHIFTED_S32: return &kernels_d3_f16s32();
      case LBM_BF16_SHIFTED_S32: return &kernels_d3_bf16s32();
    }
  }
  return nullptr;
}

double psi_of(const lbm_params& p, double rho) {
  return p.psi_kind == LBM_PSI_IDENTITY ? rho : p.rho0 * (1.0 - std::exp(-rho / p.rho0));
}

lbm_status validate(lbm_ctx* c, int lattice, int nx, int ny, int nz, const lbm_params* p) {
  if (!p) return fail(c, LBM_ERR_INVALID_ARG, "params is NULL");
  if (lattice != LBM_D2Q9_D2Q5 && lattice != LBM_D3Q19_D3Q7) return fail(c, LBM_ERR_INVALID_ARG, "unknown lattice %d", lattice);
  if (nx < 1 || ny < 1 || nz < 1) return fail(c, LBM_ERR_INVALID_ARG, "domain %dx%dx%d", nx, ny, nz);
  if (lattice == LBM_D2Q9_D2Q5 && nz != 1) return fail(c, LBM_ERR_INVALID_ARG, "2D lattice needs nz == 1");
  if ((long long)nx * ny * nz >= (1ll << 31)) return fail(c, LBM_ERR_INVALID_ARG, "more than 2^31 nodes");
  if (ny > 65535 || nz > 65535) return fail(c, LBM_ERR_INVALID_ARG, "ny and nz must not exceed 65535");
  if (p->precision < 0 || p->precision > 5) return fail(c, LBM_ERR_INVALID_ARG, "precision %d", p->precision);
  if (p->n_comp < 1 || p->n_comp > 2) return fail(c, LBM_ERR_INVALID_ARG, "n_comp %d", p->n_comp);
  for (int s = 0; s < p->n_comp; ++s)
    if (!(p->tau[s] > 0.5)) return fail(c, LBM_ERR_INVALID_ARG, "tau[%d] = %g must exceed 0.5", s, p->tau[s]);
  if (p->n_scal < 0 || p->n_scal > 2) return fail(c, LBM_ERR_INVALID_ARG, "n_scal %d", p->n_scal);
  for (int s = 0; s < p->n_scal; ++s)
    if (!(p->tau_c[s] > 0.5)) return fail(c, LBM_ERR_INVALID_ARG, "tau_c[%d] = %g must exceed 0.5", s, p->tau_c[s]);
  if (p->n_scal > 0 && !(p->J0 >= 0.0 && p->J0 < 1.0)) return fail(c, LBM_ERR_INVALID_ARG, "J0 %g", p->J0);
  if (p->forcing != LBM_FORCING_GUO && p->forcing != LBM_FORCING_SC_SHIFT) return fail(c, LBM_ERR_INVALID_ARG, "forcing");
  if (p->collision != LBM_COLLISION_BGK && p->collision != LBM_COLLISION_MRT) return fail(c, LBM_ERR_INVALID_ARG, "collision");
  if (p->collision == LBM_COLLISION_MRT && (p->n_comp != 1 || p->forcing != LBM_FORCING_GUO))
    return fail(c, LBM_ERR_INVALID_ARG, "MRT needs one component and Guo forcing");
  if (p->psi_kind != LBM_PSI_EXP && p->psi_kind != LBM_PSI_IDENTITY) return fail(c, LBM_ERR_INVALID_ARG, "psi_kind");
  if (p->psi_kind == LBM_PSI_EXP && !(p->rho0 > 0.0)) return fail(c, LBM_ERR_INVALID_ARG, "rho0");
  if (p->geo_mode < 0 || p->geo_mode > 2) return fail(c, LBM_ERR_INVALID_ARG, "geo_mode");
  if (p->geo_mode != LBM_GEO_NONE && p->n_scal < 1) return fail(c, LBM_ERR_INVALID_ARG, "geometry update needs a scalar");
  if (p->N_geo < 1) return fail(c, LBM_ERR_INVALID_ARG, "N_geo must be >= 1");
  if (p->N_mon < 0) return fail(c, LBM_ERR_INVALID_ARG, "N_mon must be >= 0");
  if (p->ade_open_x && nx < 2) return fail(c, LBM_ERR_INVALID_ARG, "inlet/outlet needs nx >= 2");
  if (p->l2_fetch_bytes != 0 && p->l2_fetch_bytes != 32 && p->l2_fetch_bytes != 64 && p->l2_fetch_bytes != 128)
    return fail(c, LBM_ERR_INVALID_ARG, "l2_fetch_bytes must be 0, 32, 64 or 128");
  if (p->block_x < 0 || p->block_x > 256 || (p->block_x % 32) != 0)
    return fail(c, LBM_ERR_INVALID_ARG, "block_x must be a multiple of 32 in [0, 256]");
  if (p->u_wall_ymax[0] != 0.0 || p->u_wall_ymax[1] != 0.0 || p->u_wall_ymax[2] != 0.0) {
    if (p->periodic[1]) return fail(c, LBM_ERR_INVALID_ARG, "a moving top plate needs a closed y axis");
    if (p->u_wall_ymax[1] != 0.0) return fail(c, LBM_ERR_INVALID_ARG, "the top plate moves in its own plane");
  }
  if (p->arrhenius) {
    if (p->n_scal != 2) return fail(c, LBM_ERR_INVALID_ARG, "the temperature-dependent rate needs n_scal == 2 (temperature)");
    if (!(p->arr_A >= 0.0) || !(p->arr_Ta >= 0.0)) return fail(c, LBM_ERR_INVALID_ARG, "arr_A and arr_Ta must be >= 0");
    if (p->n_it < 0 || p->n_it > 64) return fail(c, LBM_ERR_INVALID_ARG, "n_it must be in [0, 64]");
  }
  if (p->flow_open_x) {
    if (p->periodic[0] || p->periodic[1])
      return fail(c, LBM_ERR_INVALID_ARG, "a velocity inlet needs closed x and y axes");
    if (nx < 2) return fail(c, LBM_ERR_INVALID_ARG, "a velocity inlet needs nx >= 2");
    if (p->n_comp != 1 || p->G[0][0] != 0.0 || p->G_ads[0] != 0.0 || p->rho_solid != 0.0)
      return fail(c, LBM_ERR_INVALID_ARG, "a velocity inlet needs one component without Shan-Chen forces");
  }
  if (p->conjugate != 0 && p->conjugate != 1) return fail(c, LBM_ERR_INVALID_ARG, "conjugate must be 0 or 1");
  if (p->conjugate) {
    if (!p->arrhenius)
      return fail(c, LBM_ERR_INVALID_ARG, "conduction in the solid couples to the temperature of the temperature-dependent rate (arrhenius)");
    if (!(p->tau_s > 0.5)) return fail(c, LBM_ERR_INVALID_ARG, "tau_s = %g must exceed 0.5", p->tau_s);
    if (!(p->c_fs > 0.0)) return fail(c, LBM_ERR_INVALID_ARG, "c_fs = %g must be positive", p->c_fs);
    if (p->geo_mode == LBM_GEO_DEPOSIT) return fail(c, LBM_ERR_INVALID_ARG, "conduction in the solid is not combined with deposition");
  }
  if (p->product != 0 && p->product != 1) return fail(c, LBM_ERR_INVALID_ARG, "product must be 0 or 1");
  if (p->product) {
    if (p->n_scal < 1) return fail(c, LBM_ERR_INVALID_ARG, "the reaction product needs the reacting scalar (n_scal >= 1)");
    if (!(p->tau_p > 0.5)) return fail(c, LBM_ERR_INVALID_ARG, "tau_p = %g must exceed 0.5", p->tau_p);
    if (p->geo_mode == LBM_GEO_DEPOSIT) return fail(c, LBM_ERR_INVALID_ARG, "the reaction product is not combined with deposition");
    if (p->n_scal == 2 && p->n_comp != 1) return fail(c, LBM_ERR_INVALID_ARG, "three scalar lattices need one component");
  }
  return LBM_OK;
}

FastDiv make_fast_div(long long d) {
  int l = 0;
  while ((1ll << l) < d) ++l;
  const unsigned long long num = 1ull << (31 + l);
  FastDiv f;
  f.M = (uint32_t)((num + (unsigned long long)d - 1) / (unsigned long long)d);
  f.sh = 31 + l;
  return f;
}

// The quotient of a monotone approximation is exact everywhere once it is exact on both sides
// of every quotient boundary q * d below the limit.
bool fast_div_exact(FastDiv f, long long d, long long limit) {
  for (long long n = d; n < limit; n += d) {
    const long long q = n / d;
    if (fast_div((unsigned int)(n - 1), f) != (unsigned int)(q - 1) || fast_div((unsigned int)n, f) != (unsigned int)q)
      return false;
  }
  return limit <= 1 || fast_div((unsigned int)(limit - 1), f) == (unsigned int)((limit - 1) / d);
}

void fill_args(lbm_ctx* c) {
  Args& a = c->a;
  const lbm_params& p = c->p;
  a.pitch = c->pitch;
  a.voff_ok = 3ll * c->pitch < (1ll << 31) ? 1 : 0;
  a.N = c->N;
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
  a.n_comp = p.n_comp;
  a.n_scal = c->nlat;                 // scalar lattices, the product (if any) last
  a.product = p.product ? 1 : 0;
  for (int k = 0; k < 3; ++k) a.per[k] = p.periodic[k] ? 1 : 0;
  a.open_x = p.ade_open_x ? 1 : 0;
  bool sc = false;
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) {
      a.G[s][t] = (s < p.n_comp && t < p.n_comp) ? p.G[s][t] : 0.0;
      sc |= a.G[s][t] != 0.0;
    }
  a.sc_on = sc ? 1 : 0;
  a.ads_on = 0;
  for (int s = 0; s < p.n_comp; ++s) {
    a.G_ads[s] = p.G_ads[s];
    a.ads_on |= p.G_ads[s] != 0.0;
  }
  a.shift_forcing = p.forcing == LBM_FORCING_SC_SHIFT;
  a.psi_identity = p.psi_kind == LBM_PSI_IDENTITY;
  a.psi_wall = psi_of(p, p.rho_solid);
  a.rho0 = p.rho0;
  for (int s = 0; s < 2; ++s) {
    a.tau[s] = p.tau[s] > 0.5 ? p.tau[s] : 1.0;
    a.rho_ref[s] = p.rho_ref[s];
  }
  for (int s = 0; s < 3; ++s) {
    a.tau_c[s] = 1.0;
    a.C_in[s] = 0.0;
    a.C_ref[s] = 0.0;
  }
  for (int s = 0; s < p.n_scal; ++s) {
    a.tau_c[s] = p.tau_c[s] > 0.5 ? p.tau_c[s] : 1.0;
    a.C_in[s] = p.C_in[s];
    a.C_ref[s] = p.C_ref[s];
  }
  if (p.product) {   // the product lattice: its own relaxation time and inlet value, shift 0
    a.tau_c[p.n_scal] = p.tau_p > 0.5 ? p.tau_p : 1.0;
    a.C_in[p.n_scal] = p.C_in_p;
  }
  for (int k = 0; k < 3; ++k) a.g[k] = (k < 2 || c->lattice == LBM_D3Q19_D3Q7) ? p.g[k] : 0.0;
  a.s_grp[0] = p.s_e; a.s_grp[1] = p.s_eps; a.s_grp[2] = p.s_q; a.s_grp[3] = p.s_pi; a.s_grp[4] = p.s_m;
  a.J0 = p.J0;
  a.k_react = p.k_react;
  a.geo_mode = p.geo_mode;
  a.deposit_conservative = p.deposit_conservative ? 1 : 0;
  a.V_m = p.V_m; a.m_s0 = p.m_s0; a.DP = p.DP;
  int bx = p.block_x;
  if (bx == 0) bx = 256;   // the step kernel walks the fluid list: the block shape is not tied to nx
  a.bx = bx;
  a.by = 1;
  a.div_x = make_fast_div(c->nx);
  a.div_y = make_fast_div(c->ny);
  for (int k = 0; k < 3; ++k) a.u_wall[k] = p.u_wall_ymax[k];
  a.moving_wall = (p.u_wall_ymax[0] != 0.0 || p.u_wall_ymax[2] != 0.0) ? 1 : 0;
  a.flow_open_x = p.flow_open_x ? 1 : 0;
  a.arrhenius = p.arrhenius ? 1 : 0;
  a.n_it = p.n_it;
  a.arr_A = p.arr_A;
  a.arr_Ta = p.arr_Ta;
  a.heat_release = p.heat_release;
  a.conjugate = p.conjugate ? 1 : 0;
  a.tau_s = p.tau_s;
  a.c_fs = p.c_fs;
}

int parity_of(long long step) { return int(step & 1); }

constexpr long long kListRebuild = 1024;   // steps between sorted rebuilds of the fluid list
#ifndef LBM_STEP_GRAPHS
#define LBM_STEP_GRAPHS 1
#endif

void set_planes(lbm_ctx* c) {
  for (int s = 0; s < c->p.n_comp; ++s)
    for (int i = 0; i < c->Qf; ++i)
      c->a.fplane[s][i] = static_cast<char*>(c->a.f[s]) + (size_t)i * c->pitch * c->elem;
  for (int s = 0; s < c->nlat; ++s)
    for (int j = 0; j < c->Qc; ++j)
      c->a.hplane[s][j] = static_cast<char*>(c->a.h[s]) + (size_t)j * c->pitch * c->elem_h;
}

// Copies the populations of every fluid node between two population buffers.  A NULL map
// means node order; otherwise the map gives the slot of each node.
lbm_status move_pops(lbm_ctx* c, void* const* src_f, void* const* dst_f, void* const* src_h,
                     void* const* dst_h, const uint32_t* from, const uint32_t* to) {
  for (int s = 0; s < c->p.n_comp; ++s)
    LAUNCH(launch_permute(src_f[s], dst_f[s], (int)c->elem, c->pitch, c->Qf, c->a.flags, c->N, from, to,
                          c->stream));
  for (int s = 0; s < c->nlat; ++s)
    LAUNCH(launch_permute(src_h[s], dst_h[s], (int)c->elem_h, c->pitch, c->Qc, c->a.flags, c->N, from, to,
                          c->stream));
  return LBM_OK;
}

// Ordered rebuild of the fluid and interface lists and of the slot map (fluid nodes first, in
// list order).  With carry, the populations follow their nodes into the new slots.
void drop_graphs(lbm_ctx* c) {
  for (auto& g : c->pair_exec) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

lbm_status relist(lbm_ctx* c, bool carry) {
  drop_graphs(c);   // the captured launches hold the old buffer pointers
  c->gen += 1;
  // residual snapshots sit at the old slots: the next evaluation starts a new pair
  c->have_snap = false;
  c->res_evals = 0;
  CK(cudaMemsetAsync(c->a.listed, 0, (c->N + 3) / 4 * 4, c->stream));
  LAUNCH(c->ks->lists(c->a, 3, c->stream));
  if (carry) {
    lbm_status st = move_pops(c, c->a.f, c->f_alt, c->a.h, c->h_alt, c->a.slot, c->a.slot_new);
    if (st != LBM_OK) return st;
    for (int s = 0; s < 2; ++s) {
      std::swap(c->a.f[s], c->f_alt[s]);
      std::swap(c->a.h[s], c->h_alt[s]);
    }
    set_planes(c);
  }
  std::swap(c->a.slot, c->a.slot_new);
  return LBM_OK;
}

lbm_status rebuild_geometry(lbm_ctx* c, bool carry) {
  LAUNCH(c->ks->masks(c->a, c->stream));
  return relist(c, carry);
}

lbm_status run_monitor(lbm_ctx* c) {
  long long nb = 0;
  LAUNCH(c->ks->monitor(c->a, parity_of(c->step), c->stream, &nb));
  LAUNCH(launch_reduce(c->a.partials, nb, NMON, c->a.mon_out, c->a.err, M_NONFIN, c->stream));
  return LBM_OK;
}

lbm_status run_moments(lbm_ctx* c) {
  if (c->a.sc_on) LAUNCH(c->ks->psi(c->a, parity_of(c->step), c->stream));
  LAUNCH(c->ks->moments(c->a, parity_of(c->step), c->stream));
  return LBM_OK;
}

// residual partials land in partials[0 .. 4*nb); summed into mon_out[NMON .. NMON+4)
lbm_status run_residual(lbm_ctx* c) {
  if (c->a.sc_on) LAUNCH(c->ks->psi(c->a, parity_of(c->step), c->stream));
  long long nb = 0;
  LAUNCH(c->ks->resid(c->a, parity_of(c->step), c->stream, &nb));
  LAUNCH(launch_reduce(c->a.partials, nb, 4, c->a.mon_out + NMON, c->a.err, -1, c->stream));
  return LBM_OK;
}

double residual_from(const double* r4) {
  double r = r4[1] > 0.0 ? std::sqrt(r4[0] / r4[1]) : 0.0;
  if (r4[3] > 0.0) {
    const double rc = std::sqrt(r4[2] / r4[3]);
    if (rc > r) r = rc;
  }
  return r;
}

lbm_status check_err(lbm_ctx* c) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, c->a.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (e & ERR_BOUNDS) return fail(c, LBM_ERR_BOUNDS, "a step kernel index left its buffer");
  if (e & ERR_CAPACITY) return fail(c, LBM_ERR_CAPACITY, "geometry flip list overflowed");
  if (e & ERR_CAS) return fail(c, LBM_ERR_TIMEOUT, "flag update retry limit reached");
  if (e & ERR_NONFINITE) return fail(c, LBM_ERR_NONFINITE, "non-finite populations detected");
  return LBM_OK;
}

}  // namespace

namespace lbm {

// Fixed-order sum of the per-block partials (deterministic): each thread adds a fixed set of
// blocks for all K values at once (K <= 32), then warp shuffles and one pass over the warps.
__global__ void __launch_bounds__(256) k_reduce_partials(const double* __restrict__ partials,
                                                         long long nblocks, int K,
                                                         double* __restrict__ out, int* err,
                                                         int nonfin_slot) {
  __shared__ double sh[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double acc[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) acc[k] = 0.0;
  for (long long b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if (k < K) acc[k] += partials[b * K + k];
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k >= K) break;
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][k] = v;
  }
  __syncthreads();
  if (wid == 0 && lane < K) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][lane];
    out[lane] = v;
    if (nonfin_slot == lane && v > 0.0) atomicOr(err, ERR_NONFINITE);
  }
}

cudaError_t launch_reduce(const double* partials, long long nblocks, int K, double* out, int* err,
                          int nonfin_slot, cudaStream_t st) {
  if (K > 32) return cudaErrorInvalidValue;
  k_reduce_partials<<<1, 256, 0, st>>>(partials, nblocks, K, out, err, nonfin_slot);
  return cudaGetLastError();
}

// Dissolution test (V_m acc >= m_s0) over the interface list.
__global__ void __launch_bounds__(256) k_detect(const Args a) {
  const unsigned int cnt = *a.iface_count;
  for (unsigned int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const long long n = a.iface_list[e];
    // the flag is read only for the few nodes past the threshold (most of them flipped already)
    if (consumed(a, a.acc[n]) && a.flags[n] == FL_REACTIVE) push_flip(a, int(n));
  }
}

// Population copy of every fluid node between buffers of one lattice: dst[i][to(n)] =
// src[i][from(n)], where a NULL map is node order.
template <class E>
__global__ void __launch_bounds__(256) k_permute(const E* __restrict__ src, E* __restrict__ dst, long long pitch,
                                                 int planes, const uint8_t* __restrict__ flags, long long N,
                                                 const uint32_t* __restrict__ from, const uint32_t* __restrict__ to) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N || flags[n] != FL_FLUID) return;
  const long long s = from ? (long long)from[n] : n;
  const long long d = to ? (long long)to[n] : n;
  for (int i = 0; i < planes; ++i) dst[i * pitch + d] = src[i * pitch + s];
}

cudaError_t launch_permute(const void* src, void* dst, int elem, long long pitch, int planes,
                           const uint8_t* flags, long long N, const uint32_t* from, const uint32_t* to,
                           cudaStream_t st) {
  const unsigned int nb = (unsigned int)((N + 255) / 256);
  switch (elem) {
    case 2:
      k_permute<uint16_t><<<nb, 256, 0, st>>>(static_cast<const uint16_t*>(src), static_cast<uint16_t*>(dst),
                                              pitch, planes, flags, N, from, to);
      break;
    case 4:
      k_permute<uint32_t><<<nb, 256, 0, st>>>(static_cast<const uint32_t*>(src), static_cast<uint32_t*>(dst),
                                              pitch, planes, flags, N, from, to);
      break;
    default:
      k_permute<unsigned long long><<<nb, 256, 0, st>>>(static_cast<const unsigned long long*>(src),
                                                        static_cast<unsigned long long*>(dst), pitch, planes,
                                                        flags, N, from, to);
  }
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_iota(uint32_t* __restrict__ v, long long N) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n < N) v[n] = (uint32_t)n;
}

cudaError_t launch_iota(uint32_t* v, long long N, cudaStream_t st) {
  k_iota<<<(unsigned int)((N + 255) / 256), 256, 0, st>>>(v, N);
  return cudaGetLastError();
}

cudaError_t launch_detect(const Args& a, cudaStream_t st) {
  long long nb = (a.N / 8 + 255) / 256;
  if (nb < 1) nb = 1;
  if (nb > 152 * 16) nb = 152 * 16;
  k_detect<<<(unsigned int)nb, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lbm

// ====================================================================== C ABI

extern "C" {

lbm_status lbm_params_default(lbm_params* p) {
  if (!p) return LBM_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->precision = LBM_FP32;
  p->n_comp = 1;
  p->tau[0] = p->tau[1] = 1.0;
  p->rho0 = 1.0;
  p->forcing = LBM_FORCING_GUO;
  p->collision = LBM_COLLISION_BGK;
  p->s_e = 1.19; p->s_eps = 1.4; p->s_q = 1.2; p->s_pi = 1.0; p->s_m = 1.98;
  p->tau_c[0] = p->tau_c[1] = 1.0;
  p->J0 = 0.25;
  p->periodic[0] = p->periodic[1] = p->periodic[2] = 1;
  p->V_m = 1.0; p->m_s0 = 1.0;
  p->deposit_conservative = 1;
  p->N_geo = 1;
  p->rho_ref[0] = p->rho_ref[1] = 1.0;
  p->l2_fetch_bytes = 0;
  p->n_it = 16;
  p->tau_p = 1.0;
  p->tau_s = 1.0;
  p->c_fs = 1.0;
  return LBM_OK;
}

lbm_status lbm_create(lbm_lattice lattice, int32_t nx, int32_t ny, int32_t nz, const lbm_params* params,
                      lbm_ctx** out) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  lbm_ctx tmp;
  lbm_status st = validate(&tmp, lattice, nx, ny, nz, params);
  if (st != LBM_OK) {
    g_create_err = tmp.err;
    return st;
  }
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_OOM;
  c->lattice = lattice;
  c->nx = nx; c->ny = ny; c->nz = nz;
  c->N = (long long)nx * ny * nz;
  c->pitch = (c->N + 31) / 32 * 32;
  c->p = *params;
  c->nlat = params->n_scal + (params->product ? 1 : 0);
  c->Qf = lattice == LBM_D3Q19_D3Q7 ? 19 : 9;
  c->Qc = lattice == LBM_D3Q19_D3Q7 ? 7 : 5;
  c->stream = reinterpret_cast<cudaStream_t>(params->stream);
  c->ks = pick(lattice, params->precision);
  c->elem = params->precision == LBM_FP64 ? 8 : (params->precision == LBM_FP32 ? 4 : 2);
  c->elem_h = (params->precision == LBM_FP16_SHIFTED_S32 || params->precision == LBM_BF16_SHIFTED_S32) ? 4 : c->elem;
  auto bail = [&](lbm_status s) {
    g_create_err = c->err;    // reachable through lbm_last_error(NULL)
    lbm_destroy(c);
    return s;
  };
  cudaError_t e = cudaSetDevice(params->device);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaSetDevice"));
  if (params->l2_fetch_bytes > 0) {
    e = cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)params->l2_fetch_bytes);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaDeviceSetLimit(MaxL2FetchGranularity)"));
  }
  fill_args(c);
  if (!fast_div_exact(c->a.div_x, nx, c->N) || !fast_div_exact(c->a.div_y, ny, (long long)ny * nz))
    return bail(fail(c, LBM_ERR_INVALID_ARG, "internal: node-index division check failed"));
  Args& a = c->a;
  const long long N = c->N, P = c->pitch;
  const long long rows = (long long)ny * nz;
  void* v;
#define DA(ptr, bytes)                                      \
  do {                                                      \
    st = dalloc(c, &v, (size_t)(bytes));                    \
    if (st != LBM_OK) return bail(st);                      \
    ptr = reinterpret_cast<decltype(ptr)>(v);               \
  } while (0)
  for (int s = 0; s < params->n_comp; ++s) DA(a.f[s], P * c->Qf * c->elem);
  for (int s = 0; s < c->nlat; ++s) DA(a.h[s], P * c->Qc * c->elem_h);
  for (int s = 0; s < params->n_comp; ++s) DA(c->f_alt[s], P * c->Qf * c->elem);
  for (int s = 0; s < c->nlat; ++s) DA(c->h_alt[s], P * c->Qc * c->elem_h);
  set_planes(c);
  DA(a.slot, N * 4);
  DA(a.slot_new, N * 4);
  if (a.sc_on)
    for (int s = 0; s < params->n_comp; ++s) DA(a.psi[s], P * c->ks->psi_bytes);
  DA(a.flags, (N + 3) / 4 * 4);
  DA(a.mask, N * 4);
  DA(a.acc, N * 8);
  unsigned int cap = (unsigned int)std::min<long long>(std::max<long long>(4096, N / 16), 1ll << 22);
  a.flip_cap = cap;
  DA(a.fluid_list, N * 4);
  DA(a.fluid_count, 16);
  {
    // positions of the brick order: the domain padded to whole bricks
    const long long bz = lattice == LBM_D3Q19_D3Q7 ? LBM_BRICK_Z : 1;
    const long long pos = std::max<long long>(
        N, ((nx + LBM_BRICK_X - 1) / LBM_BRICK_X) * (long long)LBM_BRICK_X * ((ny + LBM_BRICK_Y - 1) / LBM_BRICK_Y) *
               LBM_BRICK_Y * ((nz + bz - 1) / bz) * bz);
    DA(a.block_counts, ((pos + 1023) / 1024 + 1) * 4);
    DA(a.block_counts_v, ((pos + 1023) / 1024 + 1) * 4);
  }
  DA(a.wallx_slot, NBANKS * WALLX_SLOTS * 8);
  if (params->conjugate) {
    // the solid thermal lattice (two node-indexed copies) and the exchange's rate constants
    for (int b = 0; b < 2; ++b) DA(a.gs[b], N * c->Qc * c->ks->psi_bytes);
    DA(a.kb, N * (c->Qc - 1) * c->ks->psi_bytes);
  }
  DA(a.u_in_row, ny * 8);
  DA(a.iface_list, N * 4);
  DA(a.iface_count, 16);
  DA(a.listed, (N + 3) / 4 * 4);
  DA(a.flip_list, (size_t)cap * 4);
  DA(a.flip_count, 16);
  DA(a.flip_scratch, (size_t)cap * 5 * 8);
  DA(a.flip_mon, 11 * 8);
  DA(a.err, 16);
  DA(a.inflow_row, 3 * rows * 8);
  DA(a.outflow_row, 3 * rows * 8);
  // monitor partials: the monitor grid uses 128-thread blocks over x; the residual 256 over N
  DA(a.partials, (long long)wave_blocks() * NMON * 8);
  DA(a.mon_out, (NMON + 8) * 8);
  DA(a.d_rho, 2 * N * 8);
  DA(a.d_u, 3 * N * 8);
  DA(a.d_C, std::max<long long>(1, c->nlat) * N * 8);
  DA(a.snap, 4 * P * c->ks->psi_bytes);
#undef DA
  e = cudaMallocHost(reinterpret_cast<void**>(&c->mon_host), (NMON + 12) * sizeof(double));
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMallocHost"));
  // zero everything the kernels accumulate into
  e = cudaMemsetAsync(a.flags, 0, (N + 3) / 4 * 4, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.mask, 0, N * 4, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.acc, 0, N * 8, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.flip_count, 0, 16, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.iface_count, 0, 16, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.listed, 0, (N + 3) / 4 * 4, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.flip_mon, 0, 88, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.err, 0, 16, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.wallx_slot, 0, NBANKS * WALLX_SLOTS * 8, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.fluid_count, 0, 16, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.inflow_row, 0, 3 * rows * 8, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.outflow_row, 0, 3 * rows * 8, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.mon_out, 0, (NMON + 8) * 8, c->stream);
  for (int s = 0; s < params->n_comp && e == cudaSuccess; ++s) e = cudaMemsetAsync(a.f[s], 0, P * c->Qf * c->elem, c->stream);
  for (int s = 0; s < c->nlat && e == cudaSuccess; ++s) e = cudaMemsetAsync(a.h[s], 0, P * c->Qc * c->elem_h, c->stream);
  if (e == cudaSuccess) e = launch_iota(a.slot, N, c->stream);   // node order until a geometry is set
  if (e == cudaSuccess) {
    // inlet profile u_x(y) = 6 U s (1 - s), s = (y + 1/2) / ny (zero without a velocity inlet)
    std::vector<double> row(ny, 0.0);
    if (params->flow_open_x)
      for (int y = 0; y < ny; ++y) {
        const double sy = ((double)y + 0.5) / (double)ny;
        row[y] = 6.0 * params->u_in * sy * (1.0 - sy);
      }
    e = cudaMemcpyAsync(a.u_in_row, row.data(), ny * 8, cudaMemcpyHostToDevice, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "initial memset"));
  *out = c;
  return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx* c, const uint8_t* flags, size_t n) {
  if (!c || !flags) return LBM_ERR_INVALID_ARG;
  if ((long long)n != c->N) return fail(c, LBM_ERR_INVALID_ARG, "geometry has %zu entries, domain %lld", n, c->N);
  // the largest flag first (a loop without an early exit, which the compiler vectorises), the
  // offending node only when there is one
  uint8_t fmax = 0;
  for (size_t k = 0; k < n; ++k) fmax = flags[k] > fmax ? flags[k] : fmax;
  if (fmax > 2)
    for (size_t k = 0; k < n; ++k)
      if (flags[k] > 2) return fail(c, LBM_ERR_INVALID_ARG, "flag %u at node %zu", flags[k], k);
  CK(cudaMemcpyAsync(c->a.flags, flags, n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->a.acc, 0, c->N * 8, c->stream));
  lbm_status st = rebuild_geometry(c, false);
  if (st != LBM_OK) return st;
  CK(cudaStreamSynchronize(c->stream));
  c->fields_set = false;
  return LBM_OK;
}

lbm_status lbm_set_fields(lbm_ctx* c, const double* rho, const double* u, const double* C, size_t n) {
  if (!c || !rho || !u) return LBM_ERR_INVALID_ARG;
  if ((long long)n != c->N) return fail(c, LBM_ERR_INVALID_ARG, "fields have %zu nodes, domain %lld", n, c->N);
  if (c->nlat > 0 && !C) return fail(c, LBM_ERR_INVALID_ARG, "C is NULL with n_scal > 0");
  const size_t N = (size_t)c->N;
  CK(cudaMemcpyAsync(c->a.d_rho, rho, c->p.n_comp * N * 8, cudaMemcpyHostToDevice, c->stream));
  const int ud = c->lattice == LBM_D3Q19_D3Q7 ? 3 : 2;
  CK(cudaMemcpyAsync(c->a.d_u, u, ud * N * 8, cudaMemcpyHostToDevice, c->stream));
  if (ud == 2) CK(cudaMemsetAsync(c->a.d_u + 2 * N, 0, N * 8, c->stream));
  if (c->nlat > 0) CK(cudaMemcpyAsync(c->a.d_C, C, c->nlat * N * 8, cudaMemcpyHostToDevice, c->stream));
  LAUNCH(c->ks->init(c->a, c->stream));
  if (c->p.conjugate) LAUNCH(c->ks->solid_init(c->a, c->stream));
  const long long rows = (long long)c->ny * c->nz;
  CK(cudaMemsetAsync(c->a.flip_count, 0, 16, c->stream));
  CK(cudaMemsetAsync(c->a.flip_mon, 0, 88, c->stream));
  CK(cudaMemsetAsync(c->a.err, 0, 16, c->stream));
  CK(cudaMemsetAsync(c->a.wallx_slot, 0, NBANKS * WALLX_SLOTS * 8, c->stream));
  CK(cudaMemsetAsync(c->a.inflow_row, 0, 3 * rows * 8, c->stream));
  CK(cudaMemsetAsync(c->a.outflow_row, 0, 3 * rows * 8, c->stream));
  CK(cudaMemsetAsync(c->a.acc, 0, c->N * 8, c->stream));
  CK(cudaMemsetAsync(c->a.snap, 0, 4 * c->pitch * c->ks->psi_bytes, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->step = 0;
  c->fields_set = true;
  c->have_snap = false;
  c->res_evals = 0;
  return LBM_OK;
}

}  // extern "C"

namespace {

bool geo_after(const lbm_ctx* c, long long step_done) {
  return c->p.geo_mode != LBM_GEO_NONE && (step_done % c->p.N_geo) == 0;
}

// The kernels of one time step (the psi pass, the fused step, the geometry update when due)
// on stream st; the step counter is not advanced.
lbm_status enqueue_step(lbm_ctx* c, long long step, cudaStream_t st, bool timed) {
  const int par = parity_of(step);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (timed) {
    if (c->ev_free.size() < 2) {
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
    } else {
      e0 = c->ev_free.back(); c->ev_free.pop_back();
      e1 = c->ev_free.back(); c->ev_free.pop_back();
    }
    CK(cudaEventRecord(e0, st));
  }
  // the psi pass (Shan-Chen forces) is part of the timed step: it reads every population too
  if (c->a.sc_on) LAUNCH(c->ks->psi(c->a, par, st));
  LAUNCH(c->ks->step(c->a, par, c->p.collision, st));
  if (c->p.conjugate) {
    // conduction in the solid: the solid lattice's step, then the exchange across its links
    LAUNCH(c->ks->solid(c->a, par, st));
    LAUNCH(c->ks->exchange(c->a, par ^ 1, st));
  }
  if (timed) {
    CK(cudaEventRecord(e1, st));
    c->ev_used.push_back({e0, e1});
  }
  if (geo_after(c, step + 1)) {
    if (c->p.geo_mode == LBM_GEO_DISSOLVE) LAUNCH(launch_detect(c->a, st));
    LAUNCH(c->ks->flip(c->a, parity_of(step + 1), st));
  }
  return LBM_OK;
}

// Steps step+1 and step+2 complete neither a list rebuild nor a monitor evaluation.
bool plain_pair(const lbm_ctx* c, long long step) {
  for (long long d = step + 1; d <= step + 2; ++d) {
    if (c->p.geo_mode != LBM_GEO_NONE && (d % kListRebuild) == 0) return false;
    if (c->p.N_mon > 0 && (d % c->p.N_mon) == 0) return false;
  }
  return true;
}

// Captures an even + odd step pair into a graph (once per geometry-update pattern).
lbm_status pair_graph(lbm_ctx* c, long long step, cudaGraphExec_t* out, long long* launches) {
  const int key = (geo_after(c, step + 1) ? 1 : 0) | (geo_after(c, step + 2) ? 2 : 0);
  if (!c->pair_exec[key]) {
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const long long l0 = c->launches;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    lbm_status st = enqueue_step(c, step, c->cap_stream, false);
    if (st == LBM_OK) st = enqueue_step(c, step + 1, c->cap_stream, false);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (st != LBM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    const cudaError_t ei = cudaGraphInstantiate(&c->pair_exec[key], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      c->pair_exec[key] = nullptr;
      return cuda_fail(c, ei, "cudaGraphInstantiate");
    }
    c->pair_launches[key] = c->launches - l0;
    c->launches = l0;
  }
  *out = c->pair_exec[key];
  *launches = c->pair_launches[key];
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_step(lbm_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return LBM_ERR_INVALID_ARG;
  if (!c->fields_set) return fail(c, LBM_ERR_STATE, "lbm_set_fields must precede lbm_step");
  for (int64_t k = 0; k < nsteps;) {
    // two plain steps from an even step: one graph launch
    if (LBM_STEP_GRAPHS && c->graphs_ok && !c->profile && (c->step & 1) == 0 && nsteps - k >= 2 &&
        plain_pair(c, c->step)) {
      cudaGraphExec_t g = nullptr;
      long long nl = 0;
      if (pair_graph(c, c->step, &g, &nl) == LBM_OK) {
        CK(cudaGraphLaunch(g, c->stream));
        c->launches += nl;
        c->step += 2;
        k += 2;
        continue;
      }
      c->graphs_ok = false;   // capture unavailable: launch the kernels one by one from now on
    }
    lbm_status st = enqueue_step(c, c->step, c->stream, c->profile);
    if (st != LBM_OK) return st;
    c->step += 1;
    k += 1;
    // geometry updates append new fluid nodes to the list (they keep their old slots); now and
    // then restore the sorted order and the fluid-first slots
    if (c->p.geo_mode != LBM_GEO_NONE && (c->step % kListRebuild) == 0) {
      st = relist(c, true);
      if (st != LBM_OK) return st;
    }
    if (c->p.N_mon > 0 && (c->step % c->p.N_mon) == 0) {
      st = run_monitor(c);
      if (st != LBM_OK) return st;
      st = run_residual(c);
      if (st != LBM_OK) return st;
      c->have_snap = true;
      c->res_evals += 1;
    }
  }
  return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c) {
  if (!c) return LBM_ERR_INVALID_ARG;
  return check_err(c);
}

lbm_status lbm_get_fields(lbm_ctx* c, double* rho, double* u, double* C, uint8_t* flags, double* acc) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!c->fields_set) return fail(c, LBM_ERR_STATE, "fields were never set");
  lbm_status st = run_moments(c);
  if (st != LBM_OK) return st;
  const size_t N = (size_t)c->N;
  if (rho) CK(cudaMemcpyAsync(rho, c->a.d_rho, c->p.n_comp * N * 8, cudaMemcpyDeviceToHost, c->stream));
  if (u) CK(cudaMemcpyAsync(u, c->a.d_u, 3 * N * 8, cudaMemcpyDeviceToHost, c->stream));
  if (C && c->nlat > 0) CK(cudaMemcpyAsync(C, c->a.d_C, c->nlat * N * 8, cudaMemcpyDeviceToHost, c->stream));
  if (flags) CK(cudaMemcpyAsync(flags, c->a.flags, N, cudaMemcpyDeviceToHost, c->stream));
  if (acc) CK(cudaMemcpyAsync(acc, c->a.acc, N * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_get_fields_device(lbm_ctx* c, const double** rho, const double** u, const double** C,
                                 const uint8_t** flags, const double** acc) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!c->fields_set) return fail(c, LBM_ERR_STATE, "fields were never set");
  lbm_status st = run_moments(c);
  if (st != LBM_OK) return st;
  CK(cudaStreamSynchronize(c->stream));
  if (rho) *rho = c->a.d_rho;
  if (u) *u = c->a.d_u;
  if (C) *C = c->nlat > 0 ? c->a.d_C : nullptr;
  if (flags) *flags = c->a.flags;
  if (acc) *acc = c->a.acc;
  return LBM_OK;
}

lbm_status lbm_get_pops(lbm_ctx* c, double* f, double* h) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const size_t N = (size_t)c->N;
  double* df = nullptr;
  double* dh = nullptr;
  if (f) CK(cudaMalloc(&df, c->p.n_comp * c->Qf * N * 8));
  if (h && c->nlat > 0) CK(cudaMalloc(&dh, c->nlat * c->Qc * N * 8));
  cudaError_t e = c->ks->pops_io(c->a, parity_of(c->step), 0, df, dh, c->stream);
  c->launches += 1;
  if (e == cudaSuccess && df) e = cudaMemcpyAsync(f, df, c->p.n_comp * c->Qf * N * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && dh) e = cudaMemcpyAsync(h, dh, c->nlat * c->Qc * N * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(df);
  cudaFree(dh);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_get_pops");
  return LBM_OK;
}

}  // extern "C"

// Scratch of lbm_get_pops_noalloc: a fixed device array, so the call allocates nothing.  In host
// code this name is only a stand-in; kernels get the device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LBM_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
// device address of g_noalloc_scratch, per device; racing first calls store the same value
std::atomic<void*> g_noalloc_ptr[kMaxDevices] = {};

// Looks up the scratch array's device address once per device (the device must be current).
lbm_status noalloc_scratch(lbm_ctx* c, void** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(c, LBM_ERR_INVALID_ARG, "device ordinal %d", dev);
  void* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return LBM_OK;
}
}  // namespace

extern "C" {

lbm_status lbm_get_pops_noalloc(lbm_ctx* c, double* f, double* h) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const size_t N = (size_t)c->N;
  const size_t nf = f ? (size_t)c->p.n_comp * c->Qf * N : 0;
  const size_t nh = (h && c->nlat > 0) ? (size_t)c->nlat * c->Qc * N : 0;
  const size_t need = (nf + nh) * sizeof(double);
  if (need > LBM_NOALLOC_SCRATCH_BYTES)
    return fail(c, LBM_ERR_CAPACITY, "lbm_get_pops_noalloc needs %zu bytes of scratch, the fixed array holds %u",
                need, (unsigned)LBM_NOALLOC_SCRATCH_BYTES);
  int prev = 0;
  CK(cudaGetDevice(&prev));
  if (prev != c->p.device) CK(cudaSetDevice(c->p.device));
  void* scratch = nullptr;
  lbm_status st = noalloc_scratch(c, &scratch);
  if (st == LBM_OK) {
    double* df = nf ? static_cast<double*>(scratch) : nullptr;
    double* dh = nh ? static_cast<double*>(scratch) + nf : nullptr;
    cudaError_t e = c->ks->pops_io(c->a, parity_of(c->step), 0, df, dh, c->stream);
    c->launches += 1;
    if (e == cudaSuccess && df) e = cudaMemcpyAsync(f, df, nf * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && dh) e = cudaMemcpyAsync(h, dh, nh * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = cuda_fail(c, e, "lbm_get_pops_noalloc");
  }
  if (prev != c->p.device) cudaSetDevice(prev);
  return st;
}

lbm_status lbm_set_pops(lbm_ctx* c, const double* f, const double* h) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const size_t N = (size_t)c->N;
  double* df = nullptr;
  double* dh = nullptr;
  cudaError_t e = cudaSuccess;
  if (f) e = cudaMalloc(&df, c->p.n_comp * c->Qf * N * 8);
  if (e == cudaSuccess && h && c->nlat > 0) e = cudaMalloc(&dh, c->nlat * c->Qc * N * 8);
  if (e == cudaSuccess && df) e = cudaMemcpyAsync(df, f, c->p.n_comp * c->Qf * N * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && dh) e = cudaMemcpyAsync(dh, h, c->nlat * c->Qc * N * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    e = c->ks->pops_io(c->a, parity_of(c->step), 1, df, dh, c->stream);
    c->launches += 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(df);
  cudaFree(dh);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_set_pops");
  c->fields_set = true;
  return LBM_OK;
}

lbm_status lbm_get_monitors(lbm_ctx* c, lbm_monitors* out) {
  if (!c || !out) return LBM_ERR_INVALID_ARG;
  if (!c->fields_set) return fail(c, LBM_ERR_STATE, "fields were never set");
  lbm_status st = run_monitor(c);
  if (st != LBM_OK) return st;
  double* hm = c->mon_host;
  CK(cudaMemcpyAsync(hm, c->a.mon_out, NMON * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hm + NMON, c->a.flip_mon, 11 * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::memset(out, 0, sizeof(*out));
  out->step = double(c->step);
  out->mass[0] = hm[M_MASS]; out->mass[1] = hm[M_MASS + 1];
  for (int k = 0; k < 3; ++k) out->momentum[k] = hm[M_MOM + k];
  out->reacted = hm[M_REACT];
  out->deposited = hm[M_DEPO];
  // flip monitors: injected mass [0, 2), injected scalars [2, 5), removed mass [5, 7), removed
  // scalars [7, 10); the product lattice, when there is one, is scalar lattice n_scal
  double sp[3], in[3], outf[3], inj[3], rem[3];
  for (int s = 0; s < 3; ++s) {
    sp[s] = hm[mon_spec(s)];
    in[s] = hm[mon_in(s)];
    outf[s] = hm[mon_out(s)];
    inj[s] = hm[NMON + 2 + s];
    rem[s] = hm[NMON + 7 + s];
  }
  for (int s = 0; s < 2; ++s) {
    out->injected_mass[s] = hm[NMON + s];
    out->removed_mass[s] = hm[NMON + 5 + s];
  }
  const int ns = c->p.n_scal;
  for (int s = 0; s < 2; ++s) {
    const bool given = s < ns;
    out->species[s] = given ? sp[s] : 0.0;
    out->inflow[s] = given ? in[s] : 0.0;
    out->outflow[s] = given ? outf[s] : 0.0;
    out->injected_species[s] = given ? inj[s] : 0.0;
    out->removed_species[s] = given ? rem[s] : 0.0;
  }
  if (c->p.product) {
    out->species_p = sp[ns];
    out->inflow_p = in[ns];
    out->outflow_p = outf[ns];
    out->injected_species_p = inj[ns];
    out->removed_species_p = rem[ns];
    out->produced = hm[M_PROD];
  }
  out->wall_exchange = hm[M_WALLX];
  out->heat = hm[M_HEAT];
  if (c->p.conjugate) {
    out->t_solid = hm[M_TSOLID];
    out->heat_solid = hm[M_HEAT_S];
    out->heat_source = hm[M_HEAT_SRC];
    out->solid_removed = hm[NMON + 10];
  }
  out->n_solid = hm[M_NSOLID];
  out->n_fluid = hm[M_NFLUID];
  out->nonfinite = hm[M_NONFIN];
  // latest residual evaluation (automatic every N_mon steps, or lbm_residual)
  out->residual = -1.0;
  if (c->res_evals >= 2) {
    double r4[4];
    CK(cudaMemcpyAsync(r4, c->a.mon_out + NMON, 32, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out->residual = residual_from(r4);
  }
  return LBM_OK;
}

lbm_status lbm_residual(lbm_ctx* c, double* r) {
  if (!c || !r) return LBM_ERR_INVALID_ARG;
  if (!c->fields_set) return fail(c, LBM_ERR_STATE, "fields were never set");
  lbm_status st = run_residual(c);
  if (st != LBM_OK) return st;
  double r4[4];
  CK(cudaMemcpyAsync(r4, c->a.mon_out + NMON, 32, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *r = c->have_snap ? residual_from(r4) : -1.0;
  c->have_snap = true;
  c->res_evals += 1;
  return LBM_OK;
}

// ---------------------------------------------------------------- checkpoint

namespace {
struct StateHeader {
  char magic[8];
  int32_t version, lattice, precision, n_comp, n_scal, nx, ny, nz;
  int64_t step;
};
// bytes of the solid thermal lattice's state (conduction in the solid): both node-indexed copies,
// the exchange's rate constants, the two heat banks and the removed-solid monitor
size_t solid_state_bytes(const lbm_ctx* c) {
  if (!c->p.conjugate) return 0;
  const size_t N = (size_t)c->N, e = (size_t)c->ks->psi_bytes;
  return (2 * c->Qc + (c->Qc - 1)) * N * e + 2 * WALLX_SLOTS * 8 + 8;
}
size_t state_bytes(const lbm_ctx* c) {
  const size_t N = (size_t)c->N, P = (size_t)c->pitch, rows = (size_t)c->ny * c->nz;
  return sizeof(StateHeader) + (c->p.n_comp * c->Qf * c->elem + c->nlat * c->Qc * c->elem_h) * P +
         (N + 3) / 4 * 4 + N * 8 + 3 * WALLX_SLOTS * 8 + 6 * rows * 8 + 10 * 8 + solid_state_bytes(c);
}
}  // namespace

lbm_status lbm_get_state(lbm_ctx* c, void* host, size_t* nbytes) {
  if (!c || !nbytes) return LBM_ERR_INVALID_ARG;
  const size_t need = state_bytes(c);
  if (!host) {
    *nbytes = need;
    return LBM_OK;
  }
  if (*nbytes < need) return fail(c, LBM_ERR_INVALID_ARG, "state buffer %zu < %zu bytes", *nbytes, need);
  uint8_t* o = static_cast<uint8_t*>(host);
  StateHeader hd{};
  std::memcpy(hd.magic, "LBMSTAT2", 8);   // format 2: three scalar lattices' worth of bookkeeping
  hd.version = 2; hd.lattice = c->lattice; hd.precision = c->p.precision;
  hd.n_comp = c->p.n_comp; hd.n_scal = c->nlat; hd.nx = c->nx; hd.ny = c->ny; hd.nz = c->nz;
  hd.step = c->step;
  std::memcpy(o, &hd, sizeof hd);
  o += sizeof hd;
  const size_t P = (size_t)c->pitch, N = (size_t)c->N, rows = (size_t)c->ny * c->nz;
  // populations in node order (solid nodes 0), staged in the second population buffers
  for (int s = 0; s < c->p.n_comp; ++s) CK(cudaMemsetAsync(c->f_alt[s], 0, c->Qf * P * c->elem, c->stream));
  for (int s = 0; s < c->nlat; ++s) CK(cudaMemsetAsync(c->h_alt[s], 0, c->Qc * P * c->elem_h, c->stream));
  lbm_status st = move_pops(c, c->a.f, c->f_alt, c->a.h, c->h_alt, c->a.slot, nullptr);
  if (st != LBM_OK) return st;
  for (int s = 0; s < c->p.n_comp; ++s) {
    CK(cudaMemcpyAsync(o, c->f_alt[s], c->Qf * P * c->elem, cudaMemcpyDeviceToHost, c->stream));
    o += c->Qf * P * c->elem;
  }
  for (int s = 0; s < c->nlat; ++s) {
    CK(cudaMemcpyAsync(o, c->h_alt[s], c->Qc * P * c->elem_h, cudaMemcpyDeviceToHost, c->stream));
    o += c->Qc * P * c->elem_h;
  }
  CK(cudaMemcpyAsync(o, c->a.flags, (N + 3) / 4 * 4, cudaMemcpyDeviceToHost, c->stream)); o += (N + 3) / 4 * 4;
  CK(cudaMemcpyAsync(o, c->a.acc, N * 8, cudaMemcpyDeviceToHost, c->stream)); o += N * 8;
  CK(cudaMemcpyAsync(o, c->a.wallx_slot, 3 * WALLX_SLOTS * 8, cudaMemcpyDeviceToHost, c->stream)); o += 3 * WALLX_SLOTS * 8;
  CK(cudaMemcpyAsync(o, c->a.inflow_row, 3 * rows * 8, cudaMemcpyDeviceToHost, c->stream)); o += 3 * rows * 8;
  CK(cudaMemcpyAsync(o, c->a.outflow_row, 3 * rows * 8, cudaMemcpyDeviceToHost, c->stream)); o += 3 * rows * 8;
  CK(cudaMemcpyAsync(o, c->a.flip_mon, 80, cudaMemcpyDeviceToHost, c->stream)); o += 80;
  if (c->p.conjugate) {
    const size_t gsb = (size_t)c->Qc * N * c->ks->psi_bytes, kbb = (size_t)(c->Qc - 1) * N * c->ks->psi_bytes;
    for (int b = 0; b < 2; ++b) {
      CK(cudaMemcpyAsync(o, c->a.gs[b], gsb, cudaMemcpyDeviceToHost, c->stream)); o += gsb;
    }
    CK(cudaMemcpyAsync(o, c->a.kb, kbb, cudaMemcpyDeviceToHost, c->stream)); o += kbb;
    CK(cudaMemcpyAsync(o, c->a.wallx_slot + BANK_HEAT_S * WALLX_SLOTS, 2 * WALLX_SLOTS * 8, cudaMemcpyDeviceToHost,
                       c->stream)); o += 2 * WALLX_SLOTS * 8;
    CK(cudaMemcpyAsync(o, c->a.flip_mon + 10, 8, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  *nbytes = need;
  return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx* c, const void* host, size_t nbytes) {
  if (!c || !host) return LBM_ERR_INVALID_ARG;
  const size_t need = state_bytes(c);
  if (nbytes != need) return fail(c, LBM_ERR_INVALID_ARG, "state has %zu bytes, expected %zu", nbytes, need);
  const uint8_t* o = static_cast<const uint8_t*>(host);
  StateHeader hd;
  std::memcpy(&hd, o, sizeof hd);
  if (std::memcmp(hd.magic, "LBMSTAT2", 8) != 0 || hd.lattice != c->lattice || hd.precision != c->p.precision ||
      hd.n_comp != c->p.n_comp || hd.n_scal != c->nlat || hd.nx != c->nx || hd.ny != c->ny || hd.nz != c->nz)
    return fail(c, LBM_ERR_INVALID_ARG, "checkpoint does not match this context");
  o += sizeof hd;
  const size_t P = (size_t)c->pitch, N = (size_t)c->N, rows = (size_t)c->ny * c->nz;
  // node-order populations go to the second buffers; they move to their slots once the slot
  // map of the restored geometry exists
  for (int s = 0; s < c->p.n_comp; ++s) {
    CK(cudaMemcpyAsync(c->f_alt[s], o, c->Qf * P * c->elem, cudaMemcpyHostToDevice, c->stream));
    o += c->Qf * P * c->elem;
  }
  for (int s = 0; s < c->nlat; ++s) {
    CK(cudaMemcpyAsync(c->h_alt[s], o, c->Qc * P * c->elem_h, cudaMemcpyHostToDevice, c->stream));
    o += c->Qc * P * c->elem_h;
  }
  CK(cudaMemcpyAsync(c->a.flags, o, (N + 3) / 4 * 4, cudaMemcpyHostToDevice, c->stream)); o += (N + 3) / 4 * 4;
  CK(cudaMemcpyAsync(c->a.acc, o, N * 8, cudaMemcpyHostToDevice, c->stream)); o += N * 8;
  CK(cudaMemcpyAsync(c->a.wallx_slot, o, 3 * WALLX_SLOTS * 8, cudaMemcpyHostToDevice, c->stream)); o += 3 * WALLX_SLOTS * 8;
  CK(cudaMemcpyAsync(c->a.inflow_row, o, 3 * rows * 8, cudaMemcpyHostToDevice, c->stream)); o += 3 * rows * 8;
  CK(cudaMemcpyAsync(c->a.outflow_row, o, 3 * rows * 8, cudaMemcpyHostToDevice, c->stream)); o += 3 * rows * 8;
  CK(cudaMemcpyAsync(c->a.flip_mon, o, 80, cudaMemcpyHostToDevice, c->stream)); o += 80;
  if (c->p.conjugate) {
    const size_t gsb = (size_t)c->Qc * N * c->ks->psi_bytes, kbb = (size_t)(c->Qc - 1) * N * c->ks->psi_bytes;
    for (int b = 0; b < 2; ++b) {
      CK(cudaMemcpyAsync(c->a.gs[b], o, gsb, cudaMemcpyHostToDevice, c->stream)); o += gsb;
    }
    CK(cudaMemcpyAsync(c->a.kb, o, kbb, cudaMemcpyHostToDevice, c->stream)); o += kbb;
    CK(cudaMemcpyAsync(c->a.wallx_slot + BANK_HEAT_S * WALLX_SLOTS, o, 2 * WALLX_SLOTS * 8, cudaMemcpyHostToDevice,
                       c->stream)); o += 2 * WALLX_SLOTS * 8;
    CK(cudaMemcpyAsync(c->a.flip_mon + 10, o, 8, cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaMemsetAsync(c->a.flip_count, 0, 16, c->stream));
  CK(cudaMemsetAsync(c->a.err, 0, 16, c->stream));
  lbm_status st = rebuild_geometry(c, false);
  if (st != LBM_OK) return st;
  st = move_pops(c, c->f_alt, c->a.f, c->h_alt, c->a.h, nullptr, c->a.slot);
  if (st != LBM_OK) return st;
  CK(cudaStreamSynchronize(c->stream));
  c->step = hd.step;
  c->fields_set = true;
  c->have_snap = false;
  c->res_evals = 0;
  return LBM_OK;
}

lbm_status lbm_profile_enable(lbm_ctx* c, int32_t on) {
  if (!c) return LBM_ERR_INVALID_ARG;
  c->profile = on != 0;
  return LBM_OK;
}

lbm_status lbm_profile_read(lbm_ctx* c, double* ms, int64_t* launches) {
  if (!c || !ms || !launches) return LBM_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(c->stream));
  double total = 0.0;
  for (auto& pr : c->ev_used) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, pr.first, pr.second));
    total += t;
    c->ev_free.push_back(pr.first);
    c->ev_free.push_back(pr.second);
  }
  *launches = (int64_t)c->ev_used.size();
  c->ev_used.clear();
  *ms = total;
  return LBM_OK;
}

lbm_status lbm_launch_count(lbm_ctx* c, int64_t* launches) {
  if (!c || !launches) return LBM_ERR_INVALID_ARG;
  *launches = c->launches;
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (void* p : c->allocs) cudaFree(p);
  for (auto& pr : c->ev_used) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (auto e : c->ev_free) cudaEventDestroy(e);
  if (c->mon_host) cudaFreeHost(c->mon_host);
  delete c;
}

}  // extern "C"

// ====================================================================== ensembles

struct lbm_ensemble {
  int lattice = 0;
  std::vector<lbm_ctx*> m;
  std::vector<char> active;
  std::vector<long long> built_gen;   // member generations the device work list was built from
  cudaStream_t stream = nullptr;
  int device = 0;
  const KernelSet* ks = nullptr;
  int threads = 256;
  Args* d_args = nullptr;
  void* d_coefs = nullptr;
  Tile* d_tiles = nullptr;
  size_t tile_cap = 0;
  unsigned int ntiles = 0;
  bool dirty = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t pair = nullptr;
  long long pair_launches = 0;
  long long launches = 0;
  std::string err;
};

namespace {

thread_local std::string g_ens_create_err;

lbm_status efail(lbm_ensemble* e, lbm_status st, const char* fmt, ...) {
  if (e) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    e->err = buf;
  }
  return st;
}

#define ECK(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return efail(e, LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

void ens_drop_graph(lbm_ensemble* e) {
  if (e->pair) cudaGraphExecDestroy(e->pair);
  e->pair = nullptr;
}

// (Re)build the device work list: one tile of `threads` entries at a time over every active
// member's fluid list, plus the members' arguments and constants.
lbm_status ens_prepare(lbm_ensemble* e) {
  bool stale = e->dirty;
  for (size_t k = 0; k < e->m.size(); ++k) stale |= e->built_gen[k] != e->m[k]->gen;
  if (!stale) return LBM_OK;
  ens_drop_graph(e);
  const int n = (int)e->m.size();
  std::vector<Args> args(n);
  std::vector<unsigned int> counts(n, 0);
  for (int k = 0; k < n; ++k) {
    lbm_ctx* c = e->m[k];
    args[k] = c->a;
    if (!e->active[k]) continue;
    ECK(cudaMemcpyAsync(&counts[k], c->a.fluid_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream));
  }
  for (int k = 0; k < n; ++k) ECK(cudaStreamSynchronize(e->m[k]->stream));
  std::vector<Tile> tiles;
  for (int k = 0; k < n; ++k) {
    if (!e->active[k]) continue;
    for (unsigned int f = 0; f < counts[k]; f += (unsigned int)e->threads) tiles.push_back(Tile{(unsigned int)k, f});
  }
  std::vector<char> coefs((size_t)n * e->ks->coef_bytes);
  e->ks->coefs(args.data(), n, coefs.data());
  if (!e->d_args) {
    ECK(cudaMalloc(&e->d_args, n * sizeof(Args)));
    ECK(cudaMalloc(&e->d_coefs, coefs.size()));
  }
  if (tiles.size() > e->tile_cap) {
    if (e->d_tiles) cudaFree(e->d_tiles);
    e->d_tiles = nullptr;
    ECK(cudaMalloc(&e->d_tiles, std::max<size_t>(1, tiles.size()) * sizeof(Tile)));
    e->tile_cap = tiles.size();
  }
  ECK(cudaMemcpyAsync(e->d_args, args.data(), n * sizeof(Args), cudaMemcpyHostToDevice, e->stream));
  ECK(cudaMemcpyAsync(e->d_coefs, coefs.data(), coefs.size(), cudaMemcpyHostToDevice, e->stream));
  if (!tiles.empty())
    ECK(cudaMemcpyAsync(e->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, e->stream));
  ECK(cudaStreamSynchronize(e->stream));
  e->ntiles = (unsigned int)tiles.size();
  for (int k = 0; k < n; ++k) e->built_gen[k] = e->m[k]->gen;
  e->dirty = false;
  return LBM_OK;
}

lbm_status ens_launch(lbm_ensemble* e, int parity, cudaStream_t st) {
  if (e->ntiles == 0) return LBM_OK;
  const lbm_params& p = e->m[0]->p;
  int bnd = 0;   // the boundary-rule kernel variant when any member has a moving plate or an inlet
  // (or a domain too large for the plain variant's 32-bit wall offsets)
  for (size_t k = 0; k < e->m.size(); ++k)
    bnd |= e->m[k]->a.moving_wall | e->m[k]->a.flow_open_x | e->m[k]->a.arrhenius | !e->m[k]->a.voff_ok;
  const cudaError_t r = e->ks->step_tiles(e->d_args, e->d_coefs, e->d_tiles, e->ntiles, p.n_comp, p.n_scal,
                                          p.collision, parity, bnd, e->threads, st);
  e->launches += 1;
  if (r != cudaSuccess) return efail(e, LBM_ERR_CUDA, "ensemble step: %s", cudaGetErrorString(r));
  return LBM_OK;
}

// after a step: the members' counters, and their monitors when due
lbm_status ens_after_step(lbm_ensemble* e) {
  for (size_t k = 0; k < e->m.size(); ++k) {
    if (!e->active[k]) continue;
    lbm_ctx* c = e->m[k];
    c->step += 1;
    if (c->p.N_mon > 0 && (c->step % c->p.N_mon) == 0) {
      lbm_status st = run_monitor(c);
      if (st == LBM_OK) st = run_residual(c);
      if (st != LBM_OK) return efail(e, st, "member %zu: %s", k, c->err.c_str());
      c->have_snap = true;
      c->res_evals += 1;
    }
  }
  return LBM_OK;
}

bool ens_plain_pair(const lbm_ensemble* e, long long step) {
  for (size_t k = 0; k < e->m.size(); ++k) {
    if (!e->active[k]) continue;
    const long long Nm = e->m[k]->p.N_mon;
    if (Nm > 0 && ((step + 1) % Nm == 0 || (step + 2) % Nm == 0)) return false;
  }
  return true;
}

long long ens_step_of(const lbm_ensemble* e) {
  for (size_t k = 0; k < e->m.size(); ++k)
    if (e->active[k]) return e->m[k]->step;
  return 0;
}

}  // namespace

extern "C" {

lbm_status lbm_ensemble_create(lbm_lattice lattice, int32_t n, const int32_t* dims, const lbm_params* params,
                               lbm_ensemble** out) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  g_ens_create_err.clear();
  if (n < 1 || !dims || !params) {
    g_ens_create_err = "ensemble needs n >= 1, dims and params";
    return LBM_ERR_INVALID_ARG;
  }
  const lbm_params& p0 = params[0];
  for (int k = 0; k < n; ++k) {
    const lbm_params& p = params[k];
    const char* why = nullptr;
    if (p.precision != p0.precision) why = "precision differs from member 0";
    else if (p.n_comp != p0.n_comp || p.n_scal != p0.n_scal) why = "n_comp / n_scal differ from member 0";
    else if (p.product) why = "the reaction product lattice is not supported in ensembles";
    else if (p.conjugate) why = "conduction in the solid is not supported in ensembles";
    else if (p.collision != p0.collision) why = "collision differs from member 0";
    else if (p.device != p0.device || p.stream != p0.stream) why = "device / stream differ from member 0";
    else if (p.geo_mode != LBM_GEO_NONE) why = "ensemble members keep their geometry (geo_mode none)";
    else if (p.block_x != p0.block_x) why = "block_x differs from member 0";
    else {
      bool sc = false;
      for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t) sc |= (s < p.n_comp && t < p.n_comp) && p.G[s][t] != 0.0;
      if (sc) why = "Shan-Chen forces are not available in ensembles";
      else if (p.forcing != LBM_FORCING_GUO) why = "ensembles use Guo forcing";
    }
    if (why) {
      char buf[160];
      snprintf(buf, sizeof buf, "member %d: %s", k, why);
      g_ens_create_err = buf;
      return LBM_ERR_INVALID_ARG;
    }
  }
  lbm_ensemble* e = new (std::nothrow) lbm_ensemble();
  if (!e) return LBM_ERR_OOM;
  e->lattice = lattice;
  e->stream = reinterpret_cast<cudaStream_t>(p0.stream);
  e->device = p0.device;
  for (int k = 0; k < n; ++k) {
    lbm_ctx* c = nullptr;
    const lbm_status st = lbm_create(lattice, dims[3 * k], dims[3 * k + 1], dims[3 * k + 2], &params[k], &c);
    if (st != LBM_OK) {
      char buf[600];
      snprintf(buf, sizeof buf, "member %d: %s", k, g_create_err.c_str());
      g_ens_create_err = buf;
      lbm_ensemble_destroy(e);
      return st;
    }
    e->m.push_back(c);
  }
  e->active.assign(n, 1);
  e->built_gen.assign(n, -1);
  e->ks = e->m[0]->ks;
  e->threads = e->m[0]->a.bx;
  *out = e;
  return LBM_OK;
}

lbm_status lbm_ensemble_member(lbm_ensemble* e, int32_t k, lbm_ctx** out) {
  if (!e || !out || k < 0 || k >= (int32_t)e->m.size()) return LBM_ERR_INVALID_ARG;
  *out = e->m[k];
  return LBM_OK;
}

lbm_status lbm_ensemble_step(lbm_ensemble* e, int64_t nsteps) {
  if (!e || nsteps < 0) return LBM_ERR_INVALID_ARG;
  long long step = -1;
  for (size_t k = 0; k < e->m.size(); ++k) {
    if (!e->active[k]) continue;
    if (!e->m[k]->fields_set) return efail(e, LBM_ERR_STATE, "member %zu: fields were never set", k);
    if (step < 0) step = e->m[k]->step;
    else if (e->m[k]->step != step) return efail(e, LBM_ERR_STATE, "active members must share one step count");
  }
  if (step < 0) return LBM_OK;   // nothing active
  lbm_status st = ens_prepare(e);
  if (st != LBM_OK) return st;
  for (int64_t k = 0; k < nsteps;) {
    const long long s = ens_step_of(e);
    if ((s & 1) == 0 && nsteps - k >= 2 && ens_plain_pair(e, s)) {
      if (!e->pair) {
        if (!e->cap_stream) ECK(cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking));
        const long long l0 = e->launches;
        ECK(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
        st = ens_launch(e, 0, e->cap_stream);
        if (st == LBM_OK) st = ens_launch(e, 1, e->cap_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(e->cap_stream, &g);
        if (st != LBM_OK) {
          if (g) cudaGraphDestroy(g);
          return st;
        }
        if (ec != cudaSuccess) return efail(e, LBM_ERR_CUDA, "capture: %s", cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&e->pair, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
          e->pair = nullptr;
          return efail(e, LBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ei));
        }
        e->pair_launches = e->launches - l0;
        e->launches = l0;
      }
      ECK(cudaGraphLaunch(e->pair, e->stream));
      e->launches += e->pair_launches;
      for (int r = 0; r < 2; ++r) {
        st = ens_after_step(e);
        if (st != LBM_OK) return st;
      }
      k += 2;
      continue;
    }
    st = ens_launch(e, int(s & 1), e->stream);
    if (st == LBM_OK) st = ens_after_step(e);
    if (st != LBM_OK) return st;
    k += 1;
  }
  return LBM_OK;
}

lbm_status lbm_ensemble_run_to_steady(lbm_ensemble* e, double r_tol, int64_t max_steps, int64_t* steps_done,
                                      int32_t* n_converged) {
  if (!e || !(r_tol > 0.0) || max_steps < 0) return LBM_ERR_INVALID_ARG;
  const long long Nm = e->m[0]->p.N_mon;
  for (auto* c : e->m)
    if (c->p.N_mon != Nm || Nm <= 0)
      return efail(e, LBM_ERR_INVALID_ARG, "run_to_steady needs one common N_mon > 0");
  long long done = 0;
  while (done < max_steps) {
    bool any = false;
    for (char a : e->active) any |= a != 0;
    if (!any) break;
    const long long s = ens_step_of(e);
    const long long chunk = std::min<long long>(Nm - (s % Nm), max_steps - done);
    lbm_status st = lbm_ensemble_step(e, chunk);
    if (st != LBM_OK) return st;
    done += chunk;
    if ((ens_step_of(e) % Nm) != 0) continue;
    // per-member exit: a member whose residual reached the tolerance stops stepping
    for (size_t k = 0; k < e->m.size(); ++k) {
      if (!e->active[k]) continue;
      lbm_monitors mon;
      st = lbm_get_monitors(e->m[k], &mon);
      if (st != LBM_OK) return efail(e, st, "member %zu: %s", k, e->m[k]->err.c_str());
      if (mon.residual >= 0.0 && mon.residual <= r_tol) {
        e->active[k] = 0;
        e->dirty = true;
      }
    }
  }
  int32_t conv = 0;
  for (char a : e->active) conv += a ? 0 : 1;
  if (steps_done) *steps_done = done;
  if (n_converged) *n_converged = conv;
  return LBM_OK;
}

lbm_status lbm_ensemble_autotune(lbm_ensemble* e, int32_t steps, int32_t* threads_out) {
  if (!e || steps < 2) return LBM_ERR_INVALID_ARG;
  const int cand[3] = {64, 128, 256};
  float best = -1.f;
  int best_t = e->threads;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  ECK(cudaEventCreate(&t0));
  ECK(cudaEventCreate(&t1));
  lbm_status st = LBM_OK;
  for (int c : cand) {
    e->threads = c;
    e->dirty = true;
    st = ens_prepare(e);
    if (st == LBM_OK) st = lbm_ensemble_step(e, 2);   // warm-up, graph capture
    if (st != LBM_OK) break;
    cudaEventRecord(t0, e->stream);
    st = lbm_ensemble_step(e, steps & ~1);
    if (st != LBM_OK) break;
    cudaEventRecord(t1, e->stream);
    cudaEventSynchronize(t1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (best < 0.f || ms < best) {
      best = ms;
      best_t = c;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (st != LBM_OK) return st;
  e->threads = best_t;
  e->dirty = true;
  if (threads_out) *threads_out = best_t;
  return LBM_OK;
}

lbm_status lbm_ensemble_launch_count(lbm_ensemble* e, int64_t* launches) {
  if (!e || !launches) return LBM_ERR_INVALID_ARG;
  long long total = e->launches;
  for (auto* c : e->m) total += c->launches;
  *launches = total;
  return LBM_OK;
}

const char* lbm_ensemble_last_error(const lbm_ensemble* e) {
  return e ? e->err.c_str() : g_ens_create_err.c_str();
}

void lbm_ensemble_destroy(lbm_ensemble* e) {
  if (!e) return;
  if (e->stream || !e->m.empty()) cudaStreamSynchronize(e->stream);
  ens_drop_graph(e);
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  for (auto* c : e->m) lbm_destroy(c);
  if (e->d_args) cudaFree(e->d_args);
  if (e->d_coefs) cudaFree(e->d_coefs);
  if (e->d_tiles) cudaFree(e->d_tiles);
  delete e;
}

}  // extern "C"
