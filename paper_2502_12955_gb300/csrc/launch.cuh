// launch.cuh -- host launchers for one (lattice, storage) pair.  Each inst_*.cu includes this
// file once and exports a KernelSet; the runtime picks the set at lbm_create.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "kernels.cuh"

namespace lbm {

struct KernelSet {
  cudaError_t (*step)(const Args&, int parity, int coll, cudaStream_t);
  cudaError_t (*psi)(const Args&, int parity, cudaStream_t);
  cudaError_t (*moments)(const Args&, int parity, cudaStream_t);
  cudaError_t (*monitor)(const Args&, int parity, cudaStream_t, long long* nblocks);
  cudaError_t (*init)(const Args&, cudaStream_t);
  cudaError_t (*pops_io)(const Args&, int parity, int dir, double* f, double* h, cudaStream_t);
  cudaError_t (*flip)(const Args&, int parity_next, cudaStream_t);
  cudaError_t (*masks)(const Args&, cudaStream_t);
  cudaError_t (*lists)(const Args&, int which, cudaStream_t);   // which: 1 fluid, 2 interface, 3 both
  cudaError_t (*resid)(const Args&, int parity, cudaStream_t, long long* nblocks);
  // conduction in the solid: the solid lattice's step, the link exchange after the fluid step
  // (parity of the next step), and the solid's initial state from the staged fields
  cudaError_t (*solid)(const Args&, int parity, cudaStream_t);
  cudaError_t (*exchange)(const Args&, int parity_next, cudaStream_t);
  cudaError_t (*solid_init)(const Args&, cudaStream_t);
  // ensembles: compute-type constants of n members into host memory (coef_bytes each), and one
  // step of every tile
  void (*coefs)(const Args* a, int n, void* out);
  cudaError_t (*step_tiles)(const Args* d_args, const void* d_coefs, const Tile* d_tiles, unsigned int ntiles,
                            int n_comp, int n_scal, int coll, int parity, int bnd, int threads, cudaStream_t);
  int psi_bytes;   // bytes per psi element (compute type)
  int coef_bytes;
};

inline dim3 node_grid(const Args& a, dim3 blk) {
  return dim3((a.nx + blk.x - 1) / blk.x, (a.ny + blk.y - 1) / blk.y, a.nz);
}

inline dim3 step_block(const Args& a) { return dim3(a.bx, a.by, 1); }

// positions of the brick order (whole bricks, so at least N)
template <class L>
long long brick_positions(const Args& a) {
  using B = Brick<L>;
  return ((a.nx + B::X - 1) / B::X) * (long long)((a.ny + B::Y - 1) / B::Y) * ((a.nz + B::Z - 1) / B::Z) * B::V;
}

// blocks of 256 threads for one resident wave (4 per SM) of the reduction kernels
inline unsigned int wave_blocks() {
  static unsigned int cached = 0;
  if (!cached) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached = (unsigned int)((sms > 0 ? sms : 1) * 4);
  }
  return cached;
}

// Host-side derivation of every constant the kernels use, in their compute type.
template <class L, class T>
Coef<T> make_coef(const Args& a, bool shifted) {
  Coef<T> k{};
  for (int s = 0; s < 2; ++s) {
    k.om[s] = T(1.0 / a.tau[s]);
    k.tau[s] = T(a.tau[s]);
    k.G_ads[s] = T(a.G_ads[s]);
    for (int t = 0; t < 2; ++t) k.G[s][t] = T(a.G[s][t]);
    k.rref[s] = shifted ? T(a.rho_ref[s]) : T(0);
  }
  for (int s = 0; s < 3; ++s) {
    k.omc[s] = T(1.0 / a.tau_c[s]);
    k.C_in[s] = T(a.C_in[s]);
    k.cref[s] = shifted ? T(a.C_ref[s]) : T(0);
  }
  // the product lattice is the last one (tau_c[n_scal - 1] when a.product)
  {
    const double tp = a.product && a.n_scal > 0 ? a.tau_c[a.n_scal - 1] : 1.0;
    k.fp = T(tp / (tp - 0.5));
  }
  k.psi_wall = T(a.psi_wall);
  k.rho0 = T(a.rho0);
  for (int c = 0; c < 3; ++c) k.g[c] = T(a.g[c]);
  for (int q = 0; q < 10; ++q)
    k.mrt_g[q] = q < L::NMRT ? T((a.s_grp[Mrt<L>::group(q)] - 1.0 / a.tau[0]) / double(mrt_norm2<L>(q))) : T(0);
  k.wc0 = T(a.J0);
  k.wca = T((1.0 - a.J0) / double(L::QC - 1));
  k.ics2c = T(double(L::QC - 1) / (2.0 * (1.0 - a.J0)));
  k.icb = T(1.0 / (2.0 * (1.0 - a.J0) / double(L::QC - 1) + a.k_react * a.tau_c[0] / (a.tau_c[0] - 0.5)));
  k.kr = T(a.k_react);
  k.DP = T(a.DP);
  k.keep = T(1.0 - a.DP);
  for (int c = 0; c < 3; ++c) k.uw6[c] = T(6.0 * a.u_wall[c]);
  k.arrA = T(a.arr_A);
  k.arrTa = T(a.arr_Ta);
  k.hr = T(a.heat_release);
  k.oms = T(a.conjugate ? 1.0 / a.tau_s : 1.0);
  k.cfs = T(a.c_fs);
  k.fc = T(a.tau_c[0] / (a.tau_c[0] - 0.5));
  k.fT = T(a.tau_c[1] / (a.tau_c[1] - 0.5));
  return k;
}

template <class L, class S>
struct Launchers {
  using T = typename Store<S>::T;
  static constexpr bool kShifted = !std::is_same<S, double>::value;
  static Coef<T> coef(const Args& a) { return make_coef<L, T>(a, kShifted); }

  // one resident wave of blocks; the kernel walks the fluid list with a grid-stride loop
  // dynamic shared memory of the tile kernel's odd-step neighbour-slot caches: two buffers of Q
  // words per thread (the current tile's and the next tile's)
  static size_t slot_smem_bytes(int parity, int threads) {
    if (!parity || !LBM_ODD_SLOT_CACHE) return 0;
    return 2 * (size_t)threads * L::Q * sizeof(uint32_t);
  }

  template <int NC, int NS, int COLL, int PAR, bool BND>
  static cudaError_t step_p(const Args& a, cudaStream_t st) {
    const int threads = a.bx;
    static int cached_threads = -1, cached_blocks = 0;
    if (cached_threads != threads) {
      int dev = 0, sms = 0, occ = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step<L, S, NC, NS, COLL, PAR, BND>, threads, 0);
      cached_blocks = (occ > 0 ? occ : 1) * (sms > 0 ? sms : 1);
      cached_threads = threads;
    }
    long long need = (a.N + threads - 1) / threads;
    const unsigned int blocks = (unsigned int)(need < cached_blocks ? need : cached_blocks);
    k_step<L, S, NC, NS, COLL, PAR, BND><<<blocks > 0 ? blocks : 1, threads, 0, st>>>(a, coef(a));
    return cudaGetLastError();
  }
  // BND: a moving plate, a velocity inlet or the temperature-dependent reaction needs the full
  // variant of the step kernel, and so does a domain too large for the plain variant's 32-bit
  // wall offsets
  template <int NC, int NS, int COLL>
  static cudaError_t step_t(const Args& a, int parity, cudaStream_t st) {
    if (a.moving_wall || a.flow_open_x || a.arrhenius || !a.voff_ok)
      return parity ? step_p<NC, NS, COLL, 1, true>(a, st) : step_p<NC, NS, COLL, 0, true>(a, st);
    return parity ? step_p<NC, NS, COLL, 1, false>(a, st) : step_p<NC, NS, COLL, 0, false>(a, st);
  }
  template <int NC, int NS>
  static cudaError_t step_c(const Args& a, int parity, int coll, cudaStream_t st) {
    if (coll == 1) {
      if (NC != 1) return cudaErrorInvalidValue;
      return step_t<1, NS, 1>(a, parity, st);
    }
    return step_t<NC, NS, 0>(a, parity, st);
  }
  template <int NC>
  static cudaError_t step_s(const Args& a, int parity, int coll, cudaStream_t st) {
    switch (a.n_scal) {
      case 0: return step_c<NC, 0>(a, parity, coll, st);
      case 1: return step_c<NC, 1>(a, parity, coll, st);
      case 2: return step_c<NC, 2>(a, parity, coll, st);
      default:
        // three scalar lattices (two scalars and the reaction product): one component only
        if constexpr (NC == 1) return step_c<1, 3>(a, parity, coll, st);
        else return cudaErrorInvalidValue;
    }
  }
  static cudaError_t step(const Args& a, int parity, int coll, cudaStream_t st) {
    return a.n_comp == 1 ? step_s<1>(a, parity, coll, st) : step_s<2>(a, parity, coll, st);
  }

  // psi pass: resident waves of 256-thread blocks over the fluid list (grid-stride)
  template <int NC, int PAR>
  static cudaError_t psi_p(const Args& a, cudaStream_t st) {
    static int cached_blocks = 0;
    if (!cached_blocks) {
      int dev = 0, sms = 0, occ = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_psi<L, S, NC, PAR>, 256, 0);
      cached_blocks = (occ > 0 ? occ : 1) * (sms > 0 ? sms : 1);
    }
    const long long need = (a.N + 255) / 256;
    const unsigned int blocks = (unsigned int)(need < cached_blocks ? need : cached_blocks);
    k_psi<L, S, NC, PAR><<<blocks > 0 ? blocks : 1, 256, 0, st>>>(a, coef(a));
    return cudaGetLastError();
  }
  static cudaError_t psi(const Args& a, int parity, cudaStream_t st) {
    if (a.n_comp == 1) return parity ? psi_p<1, 1>(a, st) : psi_p<1, 0>(a, st);
    return parity ? psi_p<2, 1>(a, st) : psi_p<2, 0>(a, st);
  }

  template <class F>
  static void by_nc_ns(const Args& a, F&& fn) {
    // dispatch on (n_comp, n_scal) with a generic lambda taking integral constants
    if (a.n_comp == 1) {
      if (a.n_scal == 0) fn(std::integral_constant<int, 1>(), std::integral_constant<int, 0>());
      else if (a.n_scal == 1) fn(std::integral_constant<int, 1>(), std::integral_constant<int, 1>());
      else if (a.n_scal == 2) fn(std::integral_constant<int, 1>(), std::integral_constant<int, 2>());
      else fn(std::integral_constant<int, 1>(), std::integral_constant<int, 3>());
    } else {
      if (a.n_scal == 0) fn(std::integral_constant<int, 2>(), std::integral_constant<int, 0>());
      else if (a.n_scal == 1) fn(std::integral_constant<int, 2>(), std::integral_constant<int, 1>());
      else fn(std::integral_constant<int, 2>(), std::integral_constant<int, 2>());
    }
  }

  static cudaError_t moments(const Args& a, int parity, cudaStream_t st) {
    const unsigned int nb = (unsigned int)((a.N + 255) / 256);
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_moments<L, S, decltype(nc)::value, decltype(ns)::value><<<nb, 256, 0, st>>>(a, coef(a), parity);
    });
    return cudaGetLastError();
  }

  static cudaError_t monitor(const Args& a, int parity, cudaStream_t st, long long* nblocks) {
    const unsigned int grd = wave_blocks();
    *nblocks = grd;
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_monitor<L, S, decltype(nc)::value, decltype(ns)::value><<<grd, 256, 0, st>>>(a, coef(a), parity);
    });
    return cudaGetLastError();
  }

  static cudaError_t resid(const Args& a, int parity, cudaStream_t st, long long* nblocks) {
    const unsigned int grd = wave_blocks();
    *nblocks = grd;
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_resid<L, S, decltype(nc)::value, decltype(ns)::value><<<grd, 256, 0, st>>>(a, coef(a), parity);
    });
    return cudaGetLastError();
  }

  static cudaError_t init(const Args& a, cudaStream_t st) {
    const unsigned int nb = (unsigned int)((a.N + 255) / 256);
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_init<L, S, decltype(nc)::value, decltype(ns)::value><<<nb, 256, 0, st>>>(a, coef(a));
    });
    return cudaGetLastError();
  }

  static cudaError_t pops_io(const Args& a, int parity, int dir, double* f, double* h, cudaStream_t st) {
    const dim3 blk(128, 1, 1);
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_pops_io<L, S, decltype(nc)::value, decltype(ns)::value>
          <<<node_grid(a, blk), blk, 0, st>>>(a, coef(a), parity, dir, f, h);
    });
    return cudaGetLastError();
  }

  static cudaError_t flip(const Args& a, int parity_next, cudaStream_t st) {
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_flip<L, S, decltype(nc)::value, decltype(ns)::value><<<1, 1024, 0, st>>>(a, coef(a), parity_next);
    });
    return cudaGetLastError();
  }

  // grid-stride kernels over the box (k_solid) and the fluid list (k_exchange): two waves of
  // blocks, fewer on a small domain
  static unsigned int box_blocks(const Args& a) {
    const long long need = (a.N + 255) / 256, cap = 2ll * wave_blocks();
    return (unsigned int)(need < cap ? (need > 0 ? need : 1) : cap);
  }
  static cudaError_t solid(const Args& a, int parity, cudaStream_t st) {
    k_solid<L, S><<<box_blocks(a), 256, 0, st>>>(a, coef(a), parity);
    return cudaGetLastError();
  }
  static cudaError_t exchange(const Args& a, int parity_next, cudaStream_t st) {
    k_exchange<L, S><<<box_blocks(a), 256, 0, st>>>(a, coef(a), parity_next);
    return cudaGetLastError();
  }
  static cudaError_t solid_init(const Args& a, cudaStream_t st) {
    const unsigned int nb = (unsigned int)((a.N + 255) / 256);
    k_solid_init<L, S><<<nb, 256, 0, st>>>(a, coef(a));
    return cudaGetLastError();
  }

  static cudaError_t masks(const Args& a, cudaStream_t st) {
    const unsigned int nb = (unsigned int)((a.N + 255) / 256);
    k_masks<L><<<nb, 256, 0, st>>>(a);
    return cudaGetLastError();
  }

  // ordered rebuild of the fluid list (which & 1) and the interface list (which & 2)
  static cudaError_t lists(const Args& a, int which, cudaStream_t st) {
    const unsigned int chunks = (unsigned int)((a.N + 1023) / 1024);
    if (which & 1) {
      const unsigned int bchunks = (unsigned int)((brick_positions<L>(a) + 1023) / 1024);
      k_list_count<L, 0><<<bchunks, 1024, 0, st>>>(a);
      k_list_scan<<<1, 1024, 0, st>>>(a.block_counts, bchunks, a.fluid_count);
      k_list_scan<<<1, 1024, 0, st>>>(a.block_counts_v, bchunks, a.fluid_count + 2);
      k_list_write<L, 0><<<bchunks, 1024, 0, st>>>(a, a.fluid_list);
    }
    if (which & 2) {
      k_list_count<L, 1><<<chunks, 1024, 0, st>>>(a);
      k_list_scan<<<1, 1024, 0, st>>>(a.block_counts, chunks, a.iface_count);
      k_list_write<L, 1><<<chunks, 1024, 0, st>>>(a, a.iface_list);
    }
    return cudaGetLastError();
  }

  static void coefs(const Args* a, int n, void* out) {
    Coef<T>* o = static_cast<Coef<T>*>(out);
    for (int i = 0; i < n; ++i) o[i] = coef(a[i]);
  }
  template <int NC, int NS, int COLL, int PAR, bool BND>
  static cudaError_t step_tiles_p(const Args* d_args, const void* d_coefs, const Tile* d_tiles, unsigned int ntiles,
                                  int threads, cudaStream_t st) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = slot_smem_bytes(PAR, threads);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_tiles<L, S, NC, NS, COLL, PAR, BND>, threads, smem);
    const unsigned int wave = (unsigned int)((occ > 0 ? occ : 1) * (sms > 0 ? sms : 1));
    const unsigned int blocks = ntiles < wave ? (ntiles > 0 ? ntiles : 1) : wave;
    k_step_tiles<L, S, NC, NS, COLL, PAR, BND><<<blocks, threads, smem, st>>>(
        d_args, static_cast<const Coef<T>*>(d_coefs), d_tiles, ntiles);
    return cudaGetLastError();
  }
  template <int NC, int NS, int COLL>
  static cudaError_t step_tiles_b(const Args* d, const void* k, const Tile* t, unsigned int nt, int parity, int bnd,
                                  int threads, cudaStream_t st) {
    if (bnd)
      return parity ? step_tiles_p<NC, NS, COLL, 1, true>(d, k, t, nt, threads, st)
                    : step_tiles_p<NC, NS, COLL, 0, true>(d, k, t, nt, threads, st);
    return parity ? step_tiles_p<NC, NS, COLL, 1, false>(d, k, t, nt, threads, st)
                  : step_tiles_p<NC, NS, COLL, 0, false>(d, k, t, nt, threads, st);
  }
  template <int NC, int NS>
  static cudaError_t step_tiles_c(const Args* d, const void* k, const Tile* t, unsigned int nt, int coll, int parity,
                                  int bnd, int threads, cudaStream_t st) {
    if (coll == 1) {
      if (NC != 1) return cudaErrorInvalidValue;
      return step_tiles_b<1, NS, 1>(d, k, t, nt, parity, bnd, threads, st);
    }
    return step_tiles_b<NC, NS, 0>(d, k, t, nt, parity, bnd, threads, st);
  }
  static cudaError_t step_tiles(const Args* d, const void* k, const Tile* t, unsigned int nt, int n_comp, int n_scal,
                                int coll, int parity, int bnd, int threads, cudaStream_t st) {
    if (n_comp == 1) {
      if (n_scal == 0) return step_tiles_c<1, 0>(d, k, t, nt, coll, parity, bnd, threads, st);
      if (n_scal == 1) return step_tiles_c<1, 1>(d, k, t, nt, coll, parity, bnd, threads, st);
      return step_tiles_c<1, 2>(d, k, t, nt, coll, parity, bnd, threads, st);
    }
    if (n_scal == 0) return step_tiles_c<2, 0>(d, k, t, nt, coll, parity, bnd, threads, st);
    if (n_scal == 1) return step_tiles_c<2, 1>(d, k, t, nt, coll, parity, bnd, threads, st);
    return step_tiles_c<2, 2>(d, k, t, nt, coll, parity, bnd, threads, st);
  }

  static KernelSet make() {
    KernelSet k;
    k.coefs = &coefs;
    k.step_tiles = &step_tiles;
    k.coef_bytes = (int)sizeof(Coef<T>);
    k.step = &step;
    k.psi = &psi;
    k.moments = &moments;
    k.monitor = &monitor;
    k.init = &init;
    k.pops_io = &pops_io;
    k.flip = &flip;
    k.masks = &masks;
    k.lists = &lists;
    k.resid = &resid;
    k.solid = &solid;
    k.exchange = &exchange;
    k.solid_init = &solid_init;
    k.psi_bytes = (int)sizeof(typename Store<S>::T);
    return k;
  }
};

// Defined in inst_<lattice>_<storage>.cu
const KernelSet& kernels_d2_f64();
const KernelSet& kernels_d2_f32();
const KernelSet& kernels_d2_f16();
const KernelSet& kernels_d2_bf16();
const KernelSet& kernels_d3_f64();
const KernelSet& kernels_d3_f32();
const KernelSet& kernels_d3_f16();
const KernelSet& kernels_d3_bf16();
const KernelSet& kernels_d2_f16s32();
const KernelSet& kernels_d2_bf16s32();
const KernelSet& kernels_d3_f16s32();
const KernelSet& kernels_d3_bf16s32();

// Storage-independent kernels (runtime.cu)
cudaError_t launch_reduce(const double* partials, long long nblocks, int K, double* out, int* err,
                          int nonfin_slot, cudaStream_t st);
cudaError_t launch_detect(const Args& a, cudaStream_t st);
cudaError_t launch_permute(const void* src, void* dst, int elem, long long pitch, int planes,
                           const uint8_t* flags, long long N, const uint32_t* from, const uint32_t* to,
                           cudaStream_t st);
cudaError_t launch_iota(uint32_t* v, long long N, cudaStream_t st);

}  // namespace lbm
