// lattice.cuh -- compile-time velocity sets and MRT moment rows for the CUDA path.
//
// Velocity orders follow the paper's Tables D3Q19 and D2Q9 (Sec. 2.1.4); the D2Q9 axis
// weights are 1/9 (the printed 1/36 for direction 4 does not normalise).  Scalar lattices
// D2Q5 (Table D2Q5, rest weight J0) and D3Q7 reuse the first 5 / 7 directions of the flow
// sets, so a scalar direction j is the flow direction j.
//
// MRT rows are the d'Humieres et al. (2002) D3Q19 and Lallemand & Luo (2000) D2Q9
// polynomials of the non-hydrodynamic groups (energy e, energy square eps, heat flux q,
// ghost stress pi, cubic m); the stress group relaxes with 1/tau like BGK.
#pragma once
#include <cstdint>

namespace lbm {

struct D2 {
  static constexpr int D = 2;
  static constexpr int Q = 9;
  static constexpr int QC = 5;
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  // opposite direction
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
  }
  // number of MRT correction rows (e, eps, q_x, q_y)
  static constexpr int NMRT = 4;
};

struct D3 {
  static constexpr int D = 3;
  static constexpr int Q = 19;
  static constexpr int QC = 7;
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 13 || i == 15) ? 1
           : ((i == 2 || i == 8 || i == 10 || i == 14 || i == 16) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 11 || i == 14 || i == 17) ? 1
           : ((i == 4 || i == 8 || i == 12 || i == 13 || i == 18) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cz(int i) {
    return (i == 5 || i == 9 || i == 11 || i == 16 || i == 18) ? 1
           : ((i == 6 || i == 10 || i == 12 || i == 15 || i == 17) ? -1 : 0);
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  // pairs (1,2) (3,4) ... (17,18)
  __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
  // number of MRT correction rows (e, eps, q x3, pi x2, m x3)
  static constexpr int NMRT = 10;
};

// MRT correction rows R_k(c) (integer valued) and their group: 0 e, 1 eps, 2 q, 3 pi, 4 m.
template <class L>
struct Mrt;

template <>
struct Mrt<D3> {
  __host__ __device__ static constexpr int group(int k) {
    return k == 0 ? 0 : (k == 1 ? 1 : (k <= 4 ? 2 : (k <= 6 ? 3 : 4)));
  }
  __host__ __device__ static constexpr int row(int k, int i) {
    const int x = D3::cx(i), y = D3::cy(i), z = D3::cz(i);
    const int c2 = x * x + y * y + z * z;
    switch (k) {
      case 0: return 19 * c2 - 30;                                  // e
      case 1: return (21 * c2 * c2 - 53 * c2 + 24) / 2;             // eps
      case 2: return (5 * c2 - 9) * x;                              // q_x
      case 3: return (5 * c2 - 9) * y;                              // q_y
      case 4: return (5 * c2 - 9) * z;                              // q_z
      case 5: return (3 * c2 - 5) * (3 * x * x - c2);               // 3 pi_xx
      case 6: return (3 * c2 - 5) * (y * y - z * z);                // pi_ww
      case 7: return x * (y * y - z * z);                           // m_x
      case 8: return y * (z * z - x * x);                           // m_y
      default: return z * (x * x - y * y);                          // m_z
    }
  }
};

template <>
struct Mrt<D2> {
  __host__ __device__ static constexpr int group(int k) { return k == 0 ? 0 : (k == 1 ? 1 : 2); }
  __host__ __device__ static constexpr int row(int k, int i) {
    const int x = D2::cx(i), y = D2::cy(i);
    const int c2 = x * x + y * y;
    switch (k) {
      case 0: return 3 * c2 - 4;                                    // e
      case 1: return (8 - 21 * c2 + 9 * c2 * c2) / 2;               // eps
      case 2: return (3 * c2 - 5) * x;                              // q_x
      default: return (3 * c2 - 5) * y;                             // q_y
    }
  }
};

// odd rows (heat flux q, cubic m) change sign under c -> -c; the others are even
template <class L>
__host__ __device__ constexpr bool mrt_odd(int k) {
  return Mrt<L>::group(k) == 2 || Mrt<L>::group(k) == 4;
}

template <class L>
__host__ __device__ constexpr int mrt_norm2(int k) {
  int s = 0;
  for (int i = 0; i < L::Q; ++i) s += Mrt<L>::row(k, i) * Mrt<L>::row(k, i);
  return s;
}

// Link-mask layout (uint32 per node):
//   bit 0                  node is fluid
//   bit i (1..Q-1)         flow neighbour x + c_i is a wall (solid, or outside a closed axis)
//   bits MB + 2(j-1), +1   scalar code of neighbour x + c_j, j = 1..QC-1:
//                          0 fluid, 1 inert wall, 2 reactive solid, 3 open face (inlet/outlet)
template <class L>
struct MaskBits {
  static constexpr int SC_BASE = L::Q;  // 19 (3D) or 9 (2D)
  __host__ __device__ static constexpr uint32_t code(uint32_t m, int j) {
    return (m >> (SC_BASE + 2 * (j - 1))) & 3u;
  }
};

}  // namespace lbm
