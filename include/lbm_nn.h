/*
 * lbm_nn.h -- C ABI of the warm-start network kernels (sm_103a): BF16 3D convolutions on the
 * 5th-generation tensor cores and the data movement around them.
 *
 * The paper has no counterpart: it reaches steady states by running the method (Sec. 3.4).  These
 * calls train and run a small convolutional encoder-decoder that predicts the steady velocity and
 * concentration from the geometry, so the lattice Boltzmann step (lbm.h) can start from that
 * prediction instead of from rest; the step's own residual still decides convergence.  Every
 * operation's definition is the FP64 reference of the test suite (oracle/nn_oracle.py).
 *
 * Conventions shared by every call:
 *  - Pointers are DEVICE pointers owned by the caller; nothing is allocated except one 4-byte
 *    error word per process (lbm_nn_gemm_tn's bounded waits) on first use.
 *  - Activations are channel-last BF16, x[v][c], voxel v = x + W (y + H z).
 *  - A 3^3 convolution ("same", zero outside) uses im2col rows col[v][k], k = tap C + c,
 *    tap = (dz+1) 9 + (dy+1) 3 + (dx+1), zero for k >= 27 C up to the padded width Kp.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default); no call synchronises
 *    except lbm_nn_status.  Invalid sizes or pointers return LBM_ERR_INVALID_ARG before anything
 *    runs; a launch failure returns LBM_ERR_CUDA.
 */
#ifndef LBM_NN_H
#define LBM_NN_H

#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { LBM_NN_OUT_F32 = 0, LBM_NN_OUT_BF16 = 1, LBM_NN_OUT_BF16_RELU = 2 };

/* C = A B^T on the tensor cores (tcgen05.mma, FP32 accumulation in TMEM, TMA tile loads).
   A: BF16 [M][K], B: BF16 [N][K] (K contiguous, 16-byte aligned rows).  M % 128 == 0,
   M <= 65535 * 128, K % 64 == 0, N % 16 == 0, ldc % 8 == 0, ldc >= N.
   out_kind LBM_NN_OUT_F32: C is FP32 [splits][M][ldc]; the K blocks are divided among `splits`
   partial products (lbm_nn_gemm_splits gives the count actually used) to be summed with
   lbm_nn_reduce_splits.  LBM_NN_OUT_BF16 (_RELU): splits must be 1, C is BF16 [M][ldc] holding
   A B^T + bias (bias FP32 [N] or NULL), then max(., 0) for _RELU. */
lbm_status lbm_nn_gemm_tn(const void* A, const void* B, void* C, int64_t ldc, int32_t M, int32_t N, int32_t K,
                          int32_t splits, int32_t out_kind, const float* bias, void* stream);
/* Number of partial products lbm_nn_gemm_tn writes for this K and requested split count. */
int32_t lbm_nn_gemm_splits(int32_t K, int32_t splits);
/* Synchronises `stream`; LBM_ERR_TIMEOUT if a GEMM gave up waiting on its copies since the last
   call (the word is then cleared). */
lbm_status lbm_nn_status(void* stream);

/* im2col of x [D*H*W][C] into col [V][Kp] (transposed = 0) or [Kp][V] (transposed = 1). */
lbm_status lbm_nn_im2col(const void* x, void* col, int32_t D, int32_t H, int32_t W, int32_t C, int32_t Kp,
                         int32_t transposed, void* stream);
/* The transposed im2col colT [Kp][V] from a channel-major copy xT [C][V] of the input (W % 8 == 0):
   the same values as lbm_nn_im2col with transposed = 1, with coalesced reads and writes. */
lbm_status lbm_nn_im2col_cv(const void* xT, void* colT, int32_t D, int32_t H, int32_t W, int32_t C, int32_t Kp,
                            void* stream);
/* y [Cc][R] = x [R][Cc] (BF16). */
lbm_status lbm_nn_transpose(const void* x, void* y, int64_t R, int32_t Cc, void* stream);
/* out[i] = sum_z part[z * stride + i], i < n (FP32). */
lbm_status lbm_nn_reduce_splits(const float* part, float* out, int64_t n, int32_t splits, int64_t stride, void* stream);
/* dx = dy where y > 0, else 0 (gradient through y = relu(x)); n BF16 elements. */
lbm_status lbm_nn_relu_grad(const void* y, const void* dy, void* dx, int64_t n, void* stream);
/* 2x average pooling of in [D*H*W][C] into out [D/2*H/2*W/2][C] (D, H, W even), or with
   backward = 1 its gradient: in = dL/dout (coarse), out = dL/din (fine, D*H*W). */
lbm_status lbm_nn_pool2(const void* in, void* out, int32_t D, int32_t H, int32_t W, int32_t C, int32_t backward,
                        void* stream);
/* 2x nearest upsampling of in [D*H*W][C] (coarse sizes) into out [2D*2H*2W][C], or with
   backward = 1 its gradient (fine in, coarse out: sums over each 2x2x2 block). */
lbm_status lbm_nn_up2(const void* in, void* out, int32_t D, int32_t H, int32_t W, int32_t C, int32_t backward,
                      void* stream);
/* out [V][Ca+Cb] = [a [V][Ca], b [V][Cb]]; backward = 1 splits out back into a and b. */
lbm_status lbm_nn_concat(void* a, int32_t Ca, void* b, int32_t Cb, void* out, int64_t V, int32_t backward,
                         void* stream);
/* out[c] = sum_v x[v][c] (bias gradient), FP32, overwritten. */
lbm_status lbm_nn_colsum(const void* x, float* out, int64_t V, int32_t C, void* stream);
/* Head (1x1 convolution, FP32 weights w [Co][C], bias b [Co]): y [V][Co] FP32 from h [V][C]. */
lbm_status lbm_nn_head_fwd(const void* h, const float* w, const float* b, float* y, int64_t V, int32_t C, int32_t Co,
                           void* stream);
/* Head gradients from dy [V][Co] FP32: dh [V][C] BF16 (may be NULL), dw [Co][C], db [Co] FP32
   (overwritten).  C == 16 and Co == 4 only. */
lbm_status lbm_nn_head_bwd(const void* h, const float* w, const float* dy, void* dh, float* dw, float* db, int64_t V,
                           int32_t C, int32_t Co, void* stream);
/* Masked mean squared error over fluid voxels (fluid [V] nonzero): *loss (FP64, overwritten) =
   sum (y - t)^2 / (n_fluid Co); dy [V][Co] = its gradient (0 on solid voxels). */
lbm_status lbm_nn_mse(const float* y, const float* t, const uint8_t* fluid, float* dy, double* loss, int64_t V,
                      int32_t Co, int64_t n_fluid, void* stream);
/* One Adam step (Kingma and Ba 2015) of n FP32 weights w with gradient g and moments m, v;
   step >= 1 is the step count for the bias corrections. */
lbm_status lbm_nn_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                       int32_t step, void* stream);
/* 3^3 weights w [Co][Ci][27] (FP32) -> wk [Co][Kp] BF16 (k = tap Ci + c) and, if wt is not NULL,
   the flipped transpose wt [Ci][Kpt] (k' = tap' Co + o holds w[o][c][26 - tap']) that turns the
   input gradient into a convolution of dL/dy; zero in the K padding. */
lbm_status lbm_nn_pack_weights(const float* w, void* wk, void* wt, int32_t Co, int32_t Ci, int32_t Kp, int32_t Kpt,
                               void* stream);
/* dwcol [27 Ci][Co] (k = tap Ci + c, FP32) -> dw [Co][Ci][27]. */
lbm_status lbm_nn_unpack_wgrad(const float* dwcol, float* dw, int32_t Co, int32_t Ci, void* stream);
/* y = a + b, n BF16 elements. */
lbm_status lbm_nn_add(const void* a, const void* b, void* y, int64_t n, void* stream);
/* y = BF16(x), n elements. */
lbm_status lbm_nn_cast_bf16(const float* x, void* y, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif
