/*
 * surrogate.h -- C ABI of the kernels behind the learned surrogate: a convolutional U-Net that
 * maps (phi, ux, uy) of a periodic lattice at one time level to a later one (many lattice
 * Boltzmann steps at once).  The paper has no counterpart; the LB solver (lbm.h) stays the judge
 * of every prediction and the fallback when a prediction is rejected.
 *
 * Conventions
 *   - All pointers are device pointers (caller-owned, typically torch tensors), 16-byte aligned.
 *   - Activations are NHWC: element (b, y, x, c) at ((b*H + y)*W + x)*C + c, BF16 unless the
 *     argument says float.  Images are periodic in x and y.
 *   - 3x3 weights are [tap][Cin][Cout] BF16 with tap = 3*(dy+1) + (dx+1), dy, dx in {-1, 0, 1};
 *     biases and gradients of weights/biases are FP32.
 *   - Channel counts must be multiples of 16.  Every call is asynchronous on `stream` (NULL =
 *     legacy default stream) and returns a sur_status.
 */
#ifndef SURROGATE_H
#define SURROGATE_H

#include <stddef.h>

#if defined(__GNUC__)
#define SUR_API __attribute__((visibility("default")))
#else
#define SUR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { SUR_OK = 0, SUR_ERR_PARAM = -1, SUR_ERR_CUDA = -3, SUR_ERR_TIMEOUT = -5 } sur_status;

/* Periodic 3x3 convolution as an implicit GEMM on the BF16 tensor cores, FP32 accumulation:
 *   y[p][n] = sum_tap sum_k x[p + sgn*off(tap)][k] * w'(tap, k, n) (+ bias[n]) (then ReLU if relu)
 * with w'(tap, k, n) = w[tap][k][n] (transposed_weights = 0: the forward pass, K = Cin, N = Cout,
 * sgn = +1) or w[tap][n][k] (transposed_weights = 1, sgn = -1: the gradient with respect to the
 * input, x = dL/dy with K = Cout, N = Cin).  bias may be NULL.  y is FP32 when out_f32, else BF16.
 * K, N multiples of 16; batch*H*W <= 2^30. */
SUR_API int sur_conv3x3(const void* x, const void* w, const float* bias, void* y, int batch, int H, int W, int K,
                        int N, int transposed_weights, int sgn, int relu, int out_f32, void* stream);

/* The same forward convolution on the 5th-generation tensor cores (tcgen05.mma, FP32 accumulator
 * in tensor memory): y[p][n] = sum_tap sum_k x[p + off(tap)][k] * wt[tap][n][k] (+ bias[n])
 * (+ addend[p][n]) (then ReLU if relu), BF16 operands, y BF16 or FP32 (out_f32).  wt holds the
 * weights K-major, [tap][N][K] (sur_transpose_taps makes it from the [tap][K][N] layout).
 * upsampled = 1: x is the coarse (batch, H/2, W/2, K) image read through the 2x nearest
 * upsampling (the decoder), as sur_conv3x3_up_add.  bias and addend may be NULL; an addend needs
 * BF16 output.  The kernel tiles 128 pixels (R rows of TW = min(W, 128) columns) by up to 128
 * output channels: W must be a multiple of 128 or a power of two from 2 to 64, H a multiple of
 * 128 / TW (H, W even
 * when upsampled), K and N multiples of 16, N <= 128 or a multiple of 128;
 * sur_conv3x3_tc_supported (1 / 0) says whether a shape qualifies.  Errors: SUR_ERR_PARAM (a shape
 * it cannot serve, NULL or misaligned pointers), SUR_ERR_CUDA.  Its waits are bounded: see
 * sur_check. */
SUR_API int sur_conv3x3_tc(const void* x, const void* wt, const float* bias, const void* addend, void* y, int batch,
                           int H, int W, int K, int N, int relu, int out_f32, int upsampled, void* stream);
SUR_API int sur_conv3x3_tc_supported(int batch, int H, int W, int K, int N, int upsampled);

/* wt[tap][n][k] = w[tap][k][n] for 9 taps (BF16). */
SUR_API int sur_transpose_taps(const void* w, void* wt, int K, int N, void* stream);

/* Synchronise `stream` and report whether a bounded wait of a tensor-core kernel gave up since the
 * last call (SUR_ERR_TIMEOUT; that launch wrote no output for the CTAs concerned), clearing it. */
SUR_API int sur_check(void* stream);

/* Gradient of the weights: dw[tap][ci][co] += sum_p x[p + off(tap)][ci] * dy[p][co] (FP32 atomics,
 * so dw must be zeroed first).  Cin, Cout multiples of 16; batch*H*W <= 7.4e6. */
SUR_API int sur_conv3x3_wgrad(const void* x, const void* dy, float* dw, int batch, int H, int W, int Cin, int Cout,
                              void* stream);

/* Decoder convolution fused with its neighbours: y = conv3x3(up2(xc)) + bias + addend (BF16, no
 * activation), where xc is the coarse (batch, H/2, W/2, K) image, up2 its 2x nearest upsampling to
 * H x W (never materialised) and addend (may be NULL) a BF16 (batch, H, W, N) tensor.  Forward
 * weights [tap][K][N]; H, W even; K, N multiples of 16.  Equals sur_up2 + sur_conv3x3 + sur_add
 * up to one BF16 rounding of the convolution output. */
SUR_API int sur_conv3x3_up_add(const void* xc, const void* w, const float* bias, const void* addend, void* y,
                               int batch, int H, int W, int K, int N, void* stream);

/* Weight gradient of that convolution: as sur_conv3x3_wgrad with x = up2(xc), read from the coarse
 * (batch, H/2, W/2, Cin) image xc. */
SUR_API int sur_conv3x3_wgrad_up(const void* xc, const void* dy, float* dw, int batch, int H, int W, int Cin,
                                 int Cout, void* stream);

/* ReLU backward from the post-activation y: dx = dy where y > 0, else 0 (n elements). */
SUR_API int sur_relu_bwd(const void* y, const void* dy, void* dx, size_t n, void* stream);

/* db[c] += sum over npix pixels of dy[p][c] (FP32 atomics; zero db first). */
SUR_API int sur_bias_grad(const void* dy, float* db, int npix, int C, void* stream);

/* 2x2 average pooling (H, W even) and its gradient; 2x nearest upsampling and its gradient.
 * H, W are the sizes of the FINER image for pool2 / pool2_bwd and of the COARSER one for up2 /
 * up2_bwd. */
SUR_API int sur_pool2(const void* x, void* y, int batch, int H, int W, int C, void* stream);
SUR_API int sur_pool2_bwd(const void* dy, void* dx, int batch, int H, int W, int C, void* stream);
SUR_API int sur_up2(const void* x, void* y, int batch, int H, int W, int C, void* stream);
SUR_API int sur_up2_bwd(const void* dy, void* dx, int batch, int H, int W, int C, void* stream);

/* y = a + b (n BF16 elements). */
SUR_API int sur_add(const void* a, const void* b, void* y, size_t n, void* stream);

/* Residual mean-squared error on the first `used` of C channels: prediction = xin + out,
 * *loss += mean((prediction - target)^2) (target: npix x used FP32), dout = dL/dout (BF16,
 * channels >= used set to 0). */
SUR_API int sur_mse(const float* out, const void* xin, const float* target, void* dout, float* loss, int npix, int C,
                    int used, void* stream);

/* One Adam step (Kingma & Ba) on FP32 master weights w with moments m, v (step >= 1 counts from
 * 1); wb (may be NULL) receives the BF16 copy used by the forward pass. */
SUR_API int sur_adam(float* w, const float* grad, float* m, float* v, void* wb, size_t n, float lr, float b1,
                     float b2, float eps, int step, void* stream);

/* Conservative output of the network: from its FP32 output `out` (C >= 4 channels: Jx, Jy,
 * dux, duy) and the FP32 state base (npix x 3: phi, ux, uy) the prediction pred (npix x 3 FP32)
 * is phi - [Jx(x,y) - Jx(x-1,y) + Jy(x,y) - Jy(x,y-1)], ux + dux, uy + duy.  The
 * periodic divergence telescopes, so sum phi is conserved up to FP32 rounding: the Cahn-Hilliard
 * equation (Eq. 1) is a conservation law and the predicted phi change is the divergence of a flux.
 * sur_flux_update_bwd maps dL/dpred to dL/dout (BF16, channels >= 4 zero). */
SUR_API int sur_flux_update(const float* out, const float* base, float* pred, int batch, int H, int W, int C,
                            void* stream);
SUR_API int sur_flux_update_bwd(const float* dpred, void* dout, int batch, int H, int W, int C, void* stream);

/* *loss += mean((pred - target)^2) over n FP32 values; dpred (may be NULL) = dL/dpred. */
SUR_API int sur_mse3(const float* pred, const float* target, float* dpred, float* loss, size_t n, void* stream);

/* Zero `bytes` bytes of device memory (cudaMemsetAsync). */
SUR_API int sur_zero(void* p, size_t bytes, void* stream);

/* y = bf16(x) (n elements). */
SUR_API int sur_cast_bf16(const float* x, void* y, size_t n, void* stream);

/* The solver's state and the network's: `state` is npix x 3 FP32 (phi, ux, uy per pixel, the layout
 * of lbm_batch_get_state); x the BF16 network input (npix x C: phi, u_scale ux, u_scale uy, then
 * zeros) and base the FP32 state the prediction advances (npix x 3: phi, u_scale ux, u_scale uy).
 * sur_unpack_state maps a prediction (npix x 3, velocities scaled) back to a solver state.
 * u_scale != 0; C >= 3. */
SUR_API int sur_pack_state(const float* state, void* x, float* base, size_t npix, int C, float u_scale, void* stream);
SUR_API int sur_unpack_state(const float* pred, float* state, size_t npix, float u_scale, void* stream);

/* Judge reductions, per image b of a batch of `batch` images of npix pixels and C channels (FP32),
 * in FP64 and in a fixed order (the same bits for the same input): sums[b] = sum over pixels of
 * channel 0 (phi), or for sur_phi_sq_diff the sum of (a - b)^2 over channel 0.  sums: device,
 * `batch` doubles.  A non-finite value makes its image's sum non-finite. */
SUR_API int sur_phi_sums(const float* state, int batch, int npix, int C, double* sums, void* stream);
SUR_API int sur_phi_sq_diff(const float* a, const float* b, int batch, int npix, int C, double* sums, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SURROGATE_H */
