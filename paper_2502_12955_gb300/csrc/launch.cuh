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
  int psi_bytes;   // bytes per psi element (compute type)
};

inline dim3 node_grid(const Args& a, dim3 blk) {
  return dim3((a.nx + blk.x - 1) / blk.x, (a.ny + blk.y - 1) / blk.y, a.nz);
}

inline dim3 step_block(const Args& a) { return dim3(a.bx, a.by, 1); }

template <class L, class S>
struct Launchers {
  template <int NC, int NS, int COLL>
  static cudaError_t step_t(const Args& a, int parity, cudaStream_t st) {
    const dim3 blk = step_block(a);
    k_step<L, S, NC, NS, COLL><<<node_grid(a, blk), blk, 0, st>>>(a, parity);
    return cudaGetLastError();
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
      default: return step_c<NC, 2>(a, parity, coll, st);
    }
  }
  static cudaError_t step(const Args& a, int parity, int coll, cudaStream_t st) {
    return a.n_comp == 1 ? step_s<1>(a, parity, coll, st) : step_s<2>(a, parity, coll, st);
  }

  static cudaError_t psi(const Args& a, int parity, cudaStream_t st) {
    const dim3 blk(128, 1, 1);
    if (a.n_comp == 1) k_psi<L, S, 1><<<node_grid(a, blk), blk, 0, st>>>(a, parity);
    else k_psi<L, S, 2><<<node_grid(a, blk), blk, 0, st>>>(a, parity);
    return cudaGetLastError();
  }

  template <class F>
  static void by_nc_ns(const Args& a, F&& fn) {
    // dispatch on (n_comp, n_scal) with a generic lambda taking integral constants
    if (a.n_comp == 1) {
      if (a.n_scal == 0) fn(std::integral_constant<int, 1>(), std::integral_constant<int, 0>());
      else if (a.n_scal == 1) fn(std::integral_constant<int, 1>(), std::integral_constant<int, 1>());
      else fn(std::integral_constant<int, 1>(), std::integral_constant<int, 2>());
    } else {
      if (a.n_scal == 0) fn(std::integral_constant<int, 2>(), std::integral_constant<int, 0>());
      else if (a.n_scal == 1) fn(std::integral_constant<int, 2>(), std::integral_constant<int, 1>());
      else fn(std::integral_constant<int, 2>(), std::integral_constant<int, 2>());
    }
  }

  static cudaError_t moments(const Args& a, int parity, cudaStream_t st) {
    const dim3 blk(128, 1, 1);
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_moments<L, S, decltype(nc)::value, decltype(ns)::value><<<node_grid(a, blk), blk, 0, st>>>(a, parity);
    });
    return cudaGetLastError();
  }

  static cudaError_t monitor(const Args& a, int parity, cudaStream_t st, long long* nblocks) {
    const dim3 blk(128, 1, 1);
    const dim3 grd = node_grid(a, blk);
    *nblocks = (long long)grd.x * grd.y * grd.z;
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_monitor<L, S, decltype(nc)::value, decltype(ns)::value><<<grd, blk, 0, st>>>(a, parity);
    });
    return cudaGetLastError();
  }

  static cudaError_t init(const Args& a, cudaStream_t st) {
    const unsigned int nb = (unsigned int)((a.N + 255) / 256);
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_init<L, S, decltype(nc)::value, decltype(ns)::value><<<nb, 256, 0, st>>>(a);
    });
    return cudaGetLastError();
  }

  static cudaError_t pops_io(const Args& a, int parity, int dir, double* f, double* h, cudaStream_t st) {
    const dim3 blk(128, 1, 1);
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_pops_io<L, S, decltype(nc)::value, decltype(ns)::value>
          <<<node_grid(a, blk), blk, 0, st>>>(a, parity, dir, f, h);
    });
    return cudaGetLastError();
  }

  static cudaError_t flip(const Args& a, int parity_next, cudaStream_t st) {
    by_nc_ns(a, [&](auto nc, auto ns) {
      k_flip<L, S, decltype(nc)::value, decltype(ns)::value><<<1, 1024, 0, st>>>(a, parity_next);
    });
    return cudaGetLastError();
  }

  static cudaError_t masks(const Args& a, cudaStream_t st) {
    const unsigned int nb = (unsigned int)((a.N + 255) / 256);
    k_masks<L><<<nb, 256, 0, st>>>(a);
    return cudaGetLastError();
  }

  static KernelSet make() {
    KernelSet k;
    k.step = &step;
    k.psi = &psi;
    k.moments = &moments;
    k.monitor = &monitor;
    k.init = &init;
    k.pops_io = &pops_io;
    k.flip = &flip;
    k.masks = &masks;
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

// Storage-independent kernels (runtime.cu)
cudaError_t launch_reduce(const double* partials, long long nblocks, int K, double* out, int* err,
                          int nonfin_slot, cudaStream_t st);
cudaError_t launch_residual(const Args& a, int has_c, cudaStream_t st, long long* nblocks);

}  // namespace lbm
