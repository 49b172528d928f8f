// nn.cu -- sm_103a kernels of the warm-start network (3D convolutional encoder-decoder).
//
// The paper has no network; its steady states come from running the method to convergence
// (Sec. 3.4).  The network predicts those steady fields from the geometry so the lattice
// Boltzmann step starts close to them; the step's own residual decides convergence.  The
// operations are defined, in FP64, by oracle/nn_oracle.py's counterparts (the test suite's
// reference); here they run in BF16 storage with FP32 accumulation.
//
// Layouts: activations are channel-last, x[v][c] with voxel v = x + W (y + H z); a 3^3
// convolution is a GEMM over im2col rows, col[v][k] with k = tap * C + c and
// tap = (dz + 1) 9 + (dy + 1) 3 + (dx + 1), zero outside the domain and for k >= 27 C (K is padded
// to a multiple of 128).  The contraction runs on the 5th-generation tensor cores:
//   - C[M][N] = A[M][K] B[N][K]^T, A and B BF16 with K contiguous ("TN"), FP32 accumulation;
//   - one CTA of 4 warps per 128 x BN output tile (BN = 16 .. 256, N tiles fastest across the grid
//     so that CTAs resident together share A tiles in L2); a TMA unit loads 128 x 64 and BN x 64 tiles
//     (128-byte swizzle) into a 4-stage shared-memory ring; one thread issues tcgen05.mma into
//     a TMEM accumulator (128 lanes x BN columns); all four warps read it back with tcgen05.ld;
//   - forward:       Y[v][o]  = col(X)[v][k]  W[o][k]            (bias, ReLU in the epilogue)
//     input grad:    dX[v][c] = col(dY)[v][k'] Wt[c][k']          (Wt: the kernel flipped, k' = tap C_out + o)
//     weight grad:   dW[k][o] = colT(X)[k][v] dYT[o][v]            (split over v, partial sums in FP32)
// Every wait on an mbarrier is bounded; a wait that runs out sets the error word (the entry point
// then returns LBM_ERR_TIMEOUT) and the kernel still releases its TMEM before it returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "../../include/lbm_nn.h"

namespace lbmnn {

using bf16 = __nv_bfloat16;

constexpr int BM = 128;         // output rows per CTA (TMEM lanes)
constexpr int BK = 64;          // K per stage: 64 BF16 = one 128-byte swizzle row
constexpr int STAGES = 4;
constexpr unsigned kWaitLimit = 1u << 22;   // polls of an mbarrier before a wait gives up

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// 2D tiled TMA load of box {x .. x + 63, y .. y + rows - 1} into shared memory, counted on bar
__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, void* dst, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile written by TMA with the 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset); the leading byte offset
// is not used by this layout.  Bits: start address >> 4 [0, 14), leading offset >> 4 [16, 30),
// stride offset >> 4 [32, 46), descriptor version 1 [46, 48), layout 2 = 128-byte swizzle [61, 64).
__device__ __forceinline__ uint64_t desc_sw128(const void* p) {
  uint64_t d = (uint64_t)((saddr(p) >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator [4, 6) = 1, A and B BF16 [7, 10) = 1,
// [10, 13) = 1, both K-major (bits 15, 16 clear), N >> 3 at [17, 23), M >> 4 at [24, 29).
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on bar once every tcgen05 operation this thread issued before has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(saddr(bar))
               : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ GEMM

struct GemmOut {
  void* c;            // FP32 [splits][M][ldc] or BF16 [M][ldc]
  long long ldc;
  long long split_stride;   // elements between the partial sums of consecutive splits
  const float* bias;  // [N] or null (BF16 output only)
  int kind;           // LBM_NN_OUT_*
};

template <int BN>
struct GemmSmem {
  static constexpr size_t a_bytes = (size_t)BM * BK * 2, b_bytes = (size_t)BN * BK * 2;
  static constexpr size_t tiles = STAGES * (a_bytes + b_bytes);
  static constexpr size_t bytes = 1024 + tiles + (2 * STAGES + 1) * 8 + 16;   // + alignment slack
  static constexpr int tmem_cols = BN < 32 ? 32 : BN;
};

template <int BN>
__global__ void __launch_bounds__(128, 1) k_gemm_tn(const __grid_constant__ CUtensorMap ta,
                                                    const __grid_constant__ CUtensorMap tb, int K, int kb_per_split,
                                                    GemmOut out, int* err) {
  using SM = GemmSmem<BN>;
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment of the shared-memory offset (the 128-byte swizzle pattern repeats every 1024 bytes)
  const uint32_t s0 = saddr(smem_raw);
  unsigned char* base = smem_raw + (((s0 + 1023u) & ~1023u) - s0);
  bf16* sA = reinterpret_cast<bf16*>(base);
  bf16* sB = reinterpret_cast<bf16*>(base + STAGES * SM::a_bytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + SM::tiles);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // N tiles vary fastest across the grid, so CTAs running at the same time share their A tiles in L2
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nkb_all = K / BK;
  const int kb0 = blockIdx.z * kb_per_split;
  const int kb1 = min(nkb_all, kb0 + kb_per_split);
  const int nkb = kb1 > kb0 ? kb1 - kb0 : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                 "r"(SM::tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // producer: TMA loads of the A and B tiles of every K block into the stage ring
    for (int i = 0; i < nkb && ok; ++i) {
      const int s = i % STAGES;
      const unsigned ph = (unsigned)(i / STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        ok = false;
        break;
      }
      mbar_expect_tx(&full[s], (unsigned)(SM::a_bytes + SM::b_bytes));
      tma_load_2d(&ta, sA + (size_t)s * BM * BK, &full[s], (kb0 + i) * BK, m0);
      tma_load_2d(&tb, sB + (size_t)s * BN * BK, &full[s], (kb0 + i) * BK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 MMAs of K = 16 per stage, accumulating in TMEM
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int i = 0; i < nkb && ok; ++i) {
      const int s = i % STAGES;
      const unsigned ph = (unsigned)(i / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t ad = desc_sw128(sA + (size_t)s * BM * BK + kk * 16);
        const uint64_t bd = desc_sw128(sB + (size_t)s * BN * BK + kk * 16);
        mma_bf16(tmem, ad, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);   // the stage is free once these MMAs have read it
    }
    mma_commit(done);
  }
  __syncwarp();
  // epilogue: warp w reads TMEM lanes 32w .. 32w + 31 (rows of the tile)
  if (!mbar_wait(done, 0)) ok = false;
  tc_fence_after();
  const long long row = (long long)m0 + warp * 32 + lane;
#pragma unroll 1
  for (int c = 0; c < BN; c += 16) {
    float v[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
    if (nkb == 0) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
    }
    if (out.kind == LBM_NN_OUT_F32) {
      float* dst = static_cast<float*>(out.c) + blockIdx.z * out.split_stride + row * out.ldc + n0 + c;
#pragma unroll
      for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else {
      bf16* dst = static_cast<bf16*>(out.c) + row * out.ldc + n0 + c;
      __align__(16) bf16 o[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float x = v[i] + (out.bias ? out.bias[n0 + c + i] : 0.f);
        if (out.kind == LBM_NN_OUT_BF16_RELU) x = fmaxf(x, 0.f);
        o[i] = __float2bfloat16_rn(x);
      }
      *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(o);
      *reinterpret_cast<uint4*>(dst + 8) = *reinterpret_cast<const uint4*>(o + 8);
    }
  }
  if (!ok) atomicOr(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(SM::tmem_cols) : "memory");
}

// ------------------------------------------------------------------ data movement

// col[v][k] (or colT[k][v]) = x[v + tap][c], k = tap * C + c; zero outside the domain and for
// k >= 27 C.  One thread per (v, k) element; consecutive threads take consecutive k (row layout)
// or consecutive v (transposed layout), so the writes are coalesced.
__global__ void k_im2col(const bf16* __restrict__ x, bf16* __restrict__ col, int D, int H, int W, int C, int Kp,
                         int transposed) {
  const long long V = (long long)D * H * W;
  const long long total = V * Kp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    long long v;
    int k;
    if (transposed) {
      k = (int)(i / V);
      v = i - (long long)k * V;
    } else {
      v = i / Kp;
      k = (int)(i - v * Kp);
    }
    bf16 val = __float2bfloat16_rn(0.f);
    if (k < 27 * C) {
      const int tap = k / C, c = k - tap * C;
      const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
      const int xx = (int)(v % W), yy = (int)((v / W) % H), zz = (int)(v / ((long long)W * H));
      const int x2 = xx + dx, y2 = yy + dy, z2 = zz + dz;
      if (x2 >= 0 && x2 < W && y2 >= 0 && y2 < H && z2 >= 0 && z2 < D)
        val = x[((long long)(z2 * H + y2) * W + x2) * C + c];
    }
    col[i] = val;
  }
}

// Row layout for C % 8 == 0: one thread per 8 consecutive k of one row (16 bytes, always inside
// one tap since C is a multiple of 8), copied with one 16-byte load and store.
__global__ void k_im2col_vec(const bf16* __restrict__ x, bf16* __restrict__ col, int D, int H, int W, int C, int Kp) {
  const long long V = (long long)D * H * W;
  const int CH = Kp / 8;
  const long long total = V * CH;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / CH;
    const int k0 = (int)(i - v * CH) * 8;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (k0 < 27 * C) {
      const int tap = k0 / C, c = k0 - tap * C;
      const int xx = (int)(v % W), yy = (int)((v / W) % H), zz = (int)(v / ((long long)W * H));
      const int x2 = xx + tap % 3 - 1, y2 = yy + (tap / 3) % 3 - 1, z2 = zz + tap / 9 - 1;
      if (x2 >= 0 && x2 < W && y2 >= 0 && y2 < H && z2 >= 0 && z2 < D)
        val = *reinterpret_cast<const uint4*>(x + ((long long)(z2 * H + y2) * W + x2) * C + c);
    }
    *reinterpret_cast<uint4*>(col + v * Kp + k0) = val;
  }
}

// Transposed layout from a channel-major copy xT [C][V] (W % 8 == 0): colT[k][v] = xT[c][v + tap],
// one thread per 8 consecutive voxels of one row k (same y and z), one 16-byte store.
__global__ void k_im2col_cv(const bf16* __restrict__ xT, bf16* __restrict__ colT, int D, int H, int W, int C,
                            int Kp) {
  const long long V = (long long)D * H * W;
  const long long VC = V / 8;
  const long long total = (long long)Kp * VC;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / VC);
    const long long v0 = (i - (long long)k * VC) * 8;
    __align__(16) bf16 o[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) o[e] = __float2bfloat16_rn(0.f);
    if (k < 27 * C) {
      const int tap = k / C, c = k - tap * C;
      const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
      const int x0 = (int)(v0 % W), yy = (int)((v0 / W) % H), zz = (int)(v0 / ((long long)W * H));
      const int y2 = yy + dy, z2 = zz + dz;
      if (y2 >= 0 && y2 < H && z2 >= 0 && z2 < D) {
        const bf16* row = xT + (long long)c * V + (long long)(z2 * H + y2) * W;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int x2 = x0 + e + dx;
          if (x2 >= 0 && x2 < W) o[e] = row[x2];
        }
      }
    }
    *reinterpret_cast<uint4*>(colT + (long long)k * V + v0) = *reinterpret_cast<const uint4*>(o);
  }
}

// y[c][r] = x[r][c]
__global__ void k_transpose(const bf16* __restrict__ x, bf16* __restrict__ y, long long R, int Cc) {
  __shared__ bf16 t[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const long long r = r0 + j;
    const int c = c0 + threadIdx.x;
    if (r < R && c < Cc) t[j][threadIdx.x] = x[r * Cc + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j;
    const long long r = r0 + threadIdx.x;
    if (r < R && c < Cc) y[(long long)c * R + r] = t[threadIdx.x][j];
  }
}

__global__ void k_reduce_splits(const float* __restrict__ part, float* __restrict__ out, long long n, int splits,
                                long long stride) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[z * stride + i];
    out[i] = s;
  }
}

// dx = dy where y > 0, else 0 (gradient through y = relu(x))
__global__ void k_relu_grad(const bf16* __restrict__ y, const bf16* __restrict__ dy, bf16* __restrict__ dx, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dx[i] = __bfloat162float(y[i]) > 0.f ? dy[i] : __float2bfloat16_rn(0.f);
}

// 2x average pooling (forward: x fine -> y coarse) and its gradient (dy coarse -> dx fine)
__global__ void k_pool2(const bf16* __restrict__ in, bf16* __restrict__ out, int D, int H, int W, int C, int backward) {
  const int d = D / 2, h = H / 2, w = W / 2;
  const long long total = backward ? (long long)D * H * W * C : (long long)d * h * w * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long v = i / C;
    if (backward) {
      const int xx = (int)(v % W), yy = (int)((v / W) % H), zz = (int)(v / ((long long)W * H));
      const long long vc = ((long long)(zz / 2) * h + yy / 2) * w + xx / 2;
      out[i] = __float2bfloat16_rn(__bfloat162float(in[vc * C + c]) * 0.125f);
    } else {
      const int xx = (int)(v % w), yy = (int)((v / w) % h), zz = (int)(v / ((long long)w * h));
      float s = 0.f;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          for (int e = 0; e < 2; ++e)
            s += __bfloat162float(in[(((long long)(2 * zz + a) * H + 2 * yy + b) * W + 2 * xx + e) * C + c]);
      out[i] = __float2bfloat16_rn(s * 0.125f);
    }
  }
}

// 2x nearest upsampling (forward: coarse -> fine) and its gradient (fine -> coarse block sums);
// D, H, W are the coarse sizes
__global__ void k_up2(const bf16* __restrict__ in, bf16* __restrict__ out, int D, int H, int W, int C, int backward) {
  const int D2 = 2 * D, H2 = 2 * H, W2 = 2 * W;
  const long long total = backward ? (long long)D * H * W * C : (long long)D2 * H2 * W2 * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long v = i / C;
    if (backward) {
      const int xx = (int)(v % W), yy = (int)((v / W) % H), zz = (int)(v / ((long long)W * H));
      float s = 0.f;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          for (int e = 0; e < 2; ++e)
            s += __bfloat162float(in[(((long long)(2 * zz + a) * H2 + 2 * yy + b) * W2 + 2 * xx + e) * C + c]);
      out[i] = __float2bfloat16_rn(s);
    } else {
      const int xx = (int)(v % W2), yy = (int)((v / W2) % H2), zz = (int)(v / ((long long)W2 * H2));
      out[i] = in[(((long long)(zz / 2) * H + yy / 2) * W + xx / 2) * C + c];
    }
  }
}

// out[v] = [a[v] (Ca channels), b[v] (Cb channels)]; backward splits out into a and b
__global__ void k_concat(bf16* __restrict__ a, int Ca, bf16* __restrict__ b, int Cb, bf16* __restrict__ out,
                         long long V, int backward) {
  const int Cc = Ca + Cb;
  const long long total = V * Cc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / Cc;
    const int c = (int)(i - v * Cc);
    bf16* src = c < Ca ? a + v * Ca + c : b + v * Cb + (c - Ca);
    if (backward) *src = out[i];
    else out[i] = *src;
  }
}

// Column sums of a [V][C] BF16 array into FP32 (bias gradient; out zeroed first): per block a
// chunk of voxels, warps over 32 consecutive columns (coalesced rows), a shared-memory reduction
// over the block's 8 warps and one atomic per block and column.
__global__ void k_colsum(const bf16* __restrict__ x, float* __restrict__ out, long long V, int C, long long chunk) {
  __shared__ float red[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long v0 = blockIdx.x * chunk, v1 = min(V, v0 + chunk);
  for (int c0 = 0; c0 < C; c0 += 32) {
    const int c = c0 + tx;
    float sum = 0.f;
    if (c < C)
      for (long long v = v0 + ty; v < v1; v += 8) sum += __bfloat162float(x[v * C + c]);
    red[ty][tx] = sum;
    __syncthreads();
    if (ty == 0) {
      float t = 0.f;
      for (int r = 0; r < 8; ++r) t += red[r][tx];
      if (c < C) atomicAdd(&out[c], t);
    }
    __syncthreads();
  }
}

// Head (1x1 convolution, C -> Co, FP32 output): y[v][o] = b[o] + sum_c w[o][c] h[v][c]
__global__ void k_head_fwd(const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ b,
                           float* __restrict__ y, long long V, int C, int Co) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x)
    for (int o = 0; o < Co; ++o) {
      float s = b[o];
      for (int c = 0; c < C; ++c) s = fmaf(w[o * C + c], __bfloat162float(h[v * C + c]), s);
      y[v * Co + o] = s;
    }
}

// Head gradients: dh[v][c] = sum_o w[o][c] dy[v][o] (BF16); dw[o][c] = sum_v dy[v][o] h[v][c] and
// db[o] = sum_v dy[v][o] (FP32: per-thread sums, then one warp reduction and one atomic per warp and
// entry; dw, db zeroed first).  C and Co are the head's fixed sizes.
template <int C, int Co>
__global__ void __launch_bounds__(256) k_head_bwd(const bf16* __restrict__ h, const float* __restrict__ w,
                                                  const float* __restrict__ dy, bf16* __restrict__ dh,
                                                  float* __restrict__ dw, float* __restrict__ db, long long V) {
  float acc[Co * (C + 1)];
#pragma unroll
  for (int i = 0; i < Co * (C + 1); ++i) acc[i] = 0.f;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    float g[Co], hv[C];
#pragma unroll
    for (int o = 0; o < Co; ++o) g[o] = dy[v * Co + o];
#pragma unroll
    for (int c = 0; c < C; ++c) hv[c] = __bfloat162float(h[v * C + c]);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float s = 0.f;
#pragma unroll
      for (int o = 0; o < Co; ++o) s = fmaf(w[o * C + c], g[o], s);
      if (dh) dh[v * C + c] = __float2bfloat16_rn(s);
    }
#pragma unroll
    for (int o = 0; o < Co; ++o) {
#pragma unroll
      for (int c = 0; c < C; ++c) acc[o * (C + 1) + c] = fmaf(g[o], hv[c], acc[o * (C + 1) + c]);
      acc[o * (C + 1) + C] += g[o];
    }
  }
#pragma unroll
  for (int i = 0; i < Co * (C + 1); ++i) {
    float s = acc[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) {
      const int o = i / (C + 1), c = i % (C + 1);
      atomicAdd(c < C ? &dw[o * C + c] : &db[o], s);
    }
  }
}

// Masked mean squared error over fluid voxels: loss += sum (y - t)^2 / (n_fluid Co) and
// dy = 2 (y - t) / (n_fluid Co) on fluid voxels, 0 elsewhere (loss zeroed first)
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, const uint8_t* __restrict__ fluid,
                      float* __restrict__ dy, double* __restrict__ loss, long long V, int Co, double inv_n) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V * Co; i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / Co;
    const float d = fluid[v] ? y[i] - t[i] : 0.f;
    s += (double)d * d;
    dy[i] = (float)(2.0 * d * inv_n);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv_n);
}

// Adam (Kingma and Ba 2015) on FP32 master weights
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// Weights w[o][c][tap] (FP32) -> wk[o][k] (k = tap Ci + c) and the flipped transpose
// wt[c][k'] (k' = tap' Co + o, tap' = 26 - tap), BF16, zero in the K padding
__global__ void k_pack_w(const float* __restrict__ w, bf16* __restrict__ wk, bf16* __restrict__ wt, int Co, int Ci,
                         int Kp, int Kpt) {
  const long long n1 = (long long)Co * Kp, n2 = (long long)Ci * Kpt;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n1 + n2; i += (long long)gridDim.x * blockDim.x) {
    if (i < n1) {
      const int o = (int)(i / Kp), k = (int)(i % Kp);
      float val = 0.f;
      if (k < 27 * Ci) val = w[((long long)o * Ci + k % Ci) * 27 + k / Ci];
      wk[i] = __float2bfloat16_rn(val);
    } else if (wt) {
      const long long j = i - n1;
      const int c = (int)(j / Kpt), k = (int)(j % Kpt);
      float val = 0.f;
      if (k < 27 * Co) val = w[((long long)(k % Co) * Ci + c) * 27 + (26 - k / Co)];
      wt[j] = __float2bfloat16_rn(val);
    }
  }
}

// dwcol[k][o] (FP32, k = tap Ci + c) -> dw[o][c][tap]
__global__ void k_unpack_dw(const float* __restrict__ dwcol, float* __restrict__ dw, int Co, int Ci) {
  const long long n = (long long)Co * Ci * 27;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int tap = (int)(i % 27);
    const int c = (int)((i / 27) % Ci), o = (int)(i / (27LL * Ci));
    dw[i] = dwcol[(long long)(tap * Ci + c) * Co + o];
  }
}

__global__ void k_add(const bf16* __restrict__ a, const bf16* __restrict__ b, bf16* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

__global__ void k_cast(const float* __restrict__ x, bf16* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// ------------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q{};
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// tensor map of a row-major BF16 matrix [rows][cols] read in boxes of 64 columns x box_rows rows
bool make_map(CUtensorMap* m, const void* ptr, unsigned long long rows, unsigned long long cols, unsigned box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int* err_word() {
  static int* d = nullptr;
  if (!d) {
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return nullptr;
    cudaMemset(d, 0, sizeof(int));
  }
  return d;
}

template <int BN>
cudaError_t launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, int splits, int kbs,
                        const GemmOut& o, cudaStream_t st) {
  using SM = GemmSmem<BN>;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_gemm_tn<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid(N / BN, M / BM, splits);
  k_gemm_tn<BN><<<grid, 128, SM::bytes, st>>>(ta, tb, K, kbs, o, err_word());
  return cudaGetLastError();
}

unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace lbmnn

using namespace lbmnn;

#define NN_CK(x)                                 \
  do {                                           \
    if ((x) != cudaSuccess) return LBM_ERR_CUDA; \
  } while (0)

extern "C" {

lbm_status lbm_nn_gemm_tn(const void* A, const void* B, void* C, int64_t ldc, int32_t M, int32_t N, int32_t K,
                          int32_t splits, int32_t out_kind, const float* bias, void* stream) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || (M % BM) || (K % BK) || (N % 16) || splits < 1)
    return LBM_ERR_INVALID_ARG;
  if (out_kind != LBM_NN_OUT_F32 && splits != 1) return LBM_ERR_INVALID_ARG;
  if (M / BM > 65535 || splits > 65535) return LBM_ERR_INVALID_ARG;   // grid y and z limits
  if (out_kind < LBM_NN_OUT_F32 || out_kind > LBM_NN_OUT_BF16_RELU || ldc < N || (ldc % 8)) return LBM_ERR_INVALID_ARG;
  const int BN = N % 256 == 0 ? 256 : (N % 128 == 0 ? 128 : (N % 64 == 0 ? 64 : (N % 32 == 0 ? 32 : 16)));
  const int nkb = K / BK;
  if (splits > nkb) splits = nkb;
  const int kbs = (nkb + splits - 1) / splits;
  splits = (nkb + kbs - 1) / kbs;   // every split gets at least one K block
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, (unsigned long long)M, (unsigned long long)K, BM) ||
      !make_map(&tb, B, (unsigned long long)N, (unsigned long long)K, (unsigned)BN))
    return LBM_ERR_CUDA;
  GemmOut o{C, ldc, (long long)M * ldc, bias, out_kind};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (BN) {
    case 256: e = launch_gemm<256>(ta, tb, M, N, K, splits, kbs, o, st); break;
    case 128: e = launch_gemm<128>(ta, tb, M, N, K, splits, kbs, o, st); break;
    case 64: e = launch_gemm<64>(ta, tb, M, N, K, splits, kbs, o, st); break;
    case 32: e = launch_gemm<32>(ta, tb, M, N, K, splits, kbs, o, st); break;
    default: e = launch_gemm<16>(ta, tb, M, N, K, splits, kbs, o, st); break;
  }
  return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int32_t lbm_nn_gemm_splits(int32_t K, int32_t splits) {
  const int nkb = K / BK;
  if (nkb <= 0) return 0;
  if (splits > nkb) splits = nkb;
  if (splits < 1) splits = 1;
  const int kbs = (nkb + splits - 1) / splits;
  return (nkb + kbs - 1) / kbs;
}

lbm_status lbm_nn_status(void* stream) {
  int* d = err_word();
  if (!d) return LBM_ERR_CUDA;
  int h = 0;
  NN_CK(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)));
  NN_CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  if (h) {
    cudaMemsetAsync(d, 0, sizeof(int), static_cast<cudaStream_t>(stream));
    return LBM_ERR_TIMEOUT;
  }
  return LBM_OK;
}

lbm_status lbm_nn_im2col(const void* x, void* col, int32_t D, int32_t H, int32_t W, int32_t C, int32_t Kp,
                         int32_t transposed, void* stream) {
  if (!x || !col || D <= 0 || H <= 0 || W <= 0 || C <= 0 || Kp < 27 * C) return LBM_ERR_INVALID_ARG;
  const long long n = (long long)D * H * W * Kp;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!transposed && C % 8 == 0 && Kp % 8 == 0)
    k_im2col_vec<<<grid_for(n / 8), 256, 0, st>>>(static_cast<const bf16*>(x), static_cast<bf16*>(col), D, H, W, C, Kp);
  else
    k_im2col<<<grid_for(n), 256, 0, st>>>(static_cast<const bf16*>(x), static_cast<bf16*>(col), D, H, W, C, Kp,
                                          transposed);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_im2col_cv(const void* xT, void* colT, int32_t D, int32_t H, int32_t W, int32_t C, int32_t Kp,
                            void* stream) {
  if (!xT || !colT || D <= 0 || H <= 0 || W <= 0 || (W % 8) || C <= 0 || Kp < 27 * C) return LBM_ERR_INVALID_ARG;
  const long long n = (long long)D * H * W * Kp / 8;
  k_im2col_cv<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(xT),
                                                                          static_cast<bf16*>(colT), D, H, W, C, Kp);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_transpose(const void* x, void* y, int64_t R, int32_t Cc, void* stream) {
  if (!x || !y || R <= 0 || Cc <= 0) return LBM_ERR_INVALID_ARG;
  dim3 grid((unsigned)((R + 31) / 32), (unsigned)((Cc + 31) / 32));
  k_transpose<<<grid, dim3(32, 8), 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(x),
                                                                          static_cast<bf16*>(y), R, Cc);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_reduce_splits(const float* part, float* out, int64_t n, int32_t splits, int64_t stride, void* stream) {
  if (!part || !out || n <= 0 || splits < 1 || stride < n) return LBM_ERR_INVALID_ARG;
  k_reduce_splits<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(part, out, n, splits, stride);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_relu_grad(const void* y, const void* dy, void* dx, int64_t n, void* stream) {
  if (!y || !dy || !dx || n <= 0) return LBM_ERR_INVALID_ARG;
  k_relu_grad<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(y), static_cast<const bf16*>(dy), static_cast<bf16*>(dx), n);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_pool2(const void* in, void* out, int32_t D, int32_t H, int32_t W, int32_t C, int32_t backward,
                        void* stream) {
  if (!in || !out || D < 2 || H < 2 || W < 2 || (D | H | W) & 1 || C <= 0) return LBM_ERR_INVALID_ARG;
  const long long n = (long long)D * H * W * C;
  k_pool2<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(in),
                                                                      static_cast<bf16*>(out), D, H, W, C, backward);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_up2(const void* in, void* out, int32_t D, int32_t H, int32_t W, int32_t C, int32_t backward,
                      void* stream) {
  if (!in || !out || D <= 0 || H <= 0 || W <= 0 || C <= 0) return LBM_ERR_INVALID_ARG;
  const long long n = 8LL * D * H * W * C;
  k_up2<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(in), static_cast<bf16*>(out),
                                                                    D, H, W, C, backward);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_concat(void* a, int32_t Ca, void* b, int32_t Cb, void* out, int64_t V, int32_t backward,
                         void* stream) {
  if (!a || !b || !out || Ca <= 0 || Cb <= 0 || V <= 0) return LBM_ERR_INVALID_ARG;
  k_concat<<<grid_for(V * (Ca + Cb)), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<bf16*>(a), Ca, static_cast<bf16*>(b), Cb, static_cast<bf16*>(out), V, backward);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_colsum(const void* x, float* out, int64_t V, int32_t C, void* stream) {
  if (!x || !out || V <= 0 || C <= 0) return LBM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NN_CK(cudaMemsetAsync(out, 0, sizeof(float) * C, st));
  long long blocks = V / 2048 + 1;
  if (blocks > 152 * 8) blocks = 152 * 8;
  const long long chunk = (V + blocks - 1) / blocks;
  k_colsum<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const bf16*>(x), out, V, C, chunk);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_head_fwd(const void* h, const float* w, const float* b, float* y, int64_t V, int32_t C, int32_t Co,
                           void* stream) {
  if (!h || !w || !b || !y || V <= 0 || C <= 0 || Co <= 0) return LBM_ERR_INVALID_ARG;
  k_head_fwd<<<grid_for(V), 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(h), w, b, y, V, C, Co);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_head_bwd(const void* h, const float* w, const float* dy, void* dh, float* dw, float* db, int64_t V,
                           int32_t C, int32_t Co, void* stream) {
  if (!h || !w || !dy || !dw || !db || V <= 0 || C != 16 || Co != 4) return LBM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NN_CK(cudaMemsetAsync(dw, 0, sizeof(float) * Co * C, st));
  NN_CK(cudaMemsetAsync(db, 0, sizeof(float) * Co, st));
  unsigned g = grid_for(V);
  if (g > 152 * 4) g = 152 * 4;
  k_head_bwd<16, 4><<<g, 256, 0, st>>>(static_cast<const bf16*>(h), w, dy, static_cast<bf16*>(dh), dw, db, V);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_mse(const float* y, const float* t, const uint8_t* fluid, float* dy, double* loss, int64_t V,
                      int32_t Co, int64_t n_fluid, void* stream) {
  if (!y || !t || !fluid || !dy || !loss || V <= 0 || Co <= 0) return LBM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NN_CK(cudaMemsetAsync(loss, 0, sizeof(double), st));
  const double inv_n = 1.0 / ((double)(n_fluid > 0 ? n_fluid : 1) * Co);
  k_mse<<<grid_for(V * Co), 256, 0, st>>>(y, t, fluid, dy, loss, V, Co, inv_n);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                       int32_t step, void* stream) {
  if (!w || !g || !m || !v || n <= 0 || step < 1) return LBM_ERR_INVALID_ARG;
  const float c1 = 1.f / (1.f - powf(b1, (float)step)), c2 = 1.f / (1.f - powf(b2, (float)step));
  k_adam<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_pack_weights(const float* w, void* wk, void* wt, int32_t Co, int32_t Ci, int32_t Kp, int32_t Kpt,
                               void* stream) {
  if (!w || !wk || Co <= 0 || Ci <= 0 || Kp < 27 * Ci || (wt && Kpt < 27 * Co)) return LBM_ERR_INVALID_ARG;
  const long long n = (long long)Co * Kp + (wt ? (long long)Ci * Kpt : 0);
  k_pack_w<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(w, static_cast<bf16*>(wk), static_cast<bf16*>(wt),
                                                                       Co, Ci, Kp, Kpt);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_unpack_wgrad(const float* dwcol, float* dw, int32_t Co, int32_t Ci, void* stream) {
  if (!dwcol || !dw || Co <= 0 || Ci <= 0) return LBM_ERR_INVALID_ARG;
  k_unpack_dw<<<grid_for(27LL * Co * Ci), 256, 0, static_cast<cudaStream_t>(stream)>>>(dwcol, dw, Co, Ci);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_cast_bf16(const float* x, void* y, int64_t n, void* stream) {
  if (!x || !y || n <= 0) return LBM_ERR_INVALID_ARG;
  k_cast<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, static_cast<bf16*>(y), n);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_nn_add(const void* a, const void* b, void* y, int64_t n, void* stream) {
  if (!a || !b || !y || n <= 0) return LBM_ERR_INVALID_ARG;
  k_add<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(a),
                                                                    static_cast<const bf16*>(b), static_cast<bf16*>(y), n);
  NN_CK(cudaGetLastError());
  return LBM_OK;
}

}  // extern "C"
