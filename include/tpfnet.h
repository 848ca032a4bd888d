/*
 * tpfnet — the tensor-core kernels of the warm-start U-Net (training and inference).
 *
 * The paper has no network: this is the learned warm start that predicts steady
 * (phi, u, T) fields of the heated microchannel so that tpflbm_step converges in
 * fewer steps.  Every call is asynchronous on `stream` (cudaStream_t, NULL = legacy
 * default stream), takes device pointers the caller owns, allocates nothing, and
 * returns TPF_OK, TPF_ERR_INVALID_ARG (bad sizes) or TPF_ERR_CUDA (launch failure).
 *
 * Layouts: activations NHWC bfloat16 ("bf16": 2-byte storage); 3x3 weights bf16
 * [9][Cout][Cin] with tap = (dh + 1) * 3 + (dw + 1); biases, the 1x1 head, losses,
 * gradients and Adam state float32.  Convolutions use zero padding 1, stride 1, and
 * accumulate in float32 on the tensor cores.
 */
#ifndef TPFNET_H
#define TPFNET_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* y = act(bias + conv3x3(x, wt)); act = ReLU when relu != 0.  Cin % 32 == 0,
 * Cout % 32 == 0; bias may be NULL. */
int tpfnet_conv3x3(const void *x, int N, int H, int W, int Cin, const void *wt, const float *bias, int Cout,
                   int relu, void *y, void *stream);

/* Which kernel tpfnet_conv3x3 (and tpfnet_conv3x3_dgrad, with Cin and Cout swapped)
 * runs for a shape, given 16-byte aligned tensors: the width in output channels of the
 * tcgen05 kernel's tiles (32, 64, 128 or 256), or 0 for the mma.sync kernel.  The
 * tcgen05 kernel takes pixel blocks of 128 = BW x BH with BW = min(W, 128) dividing
 * both 128 and W and BH dividing H; it stages operands with TMA and accumulates in
 * tensor memory. */
int tpfnet_conv3x3_tcgen05(int N, int H, int W, int Cin, int Cout);

/* 1 when tpfnet_conv3x3_wgrad runs the tcgen05 kernel for a shape (W a multiple of 64,
 * 16-byte aligned tensors), 0 for the mma.sync kernel.  The tcgen05 weight gradient
 * reduces over pixels with both operands staged MN-major by TMA (one pixel's channels
 * per 128-byte row) and adds each CTA's FP32 partial sums into dw with atomics. */
int tpfnet_conv3x3_wgrad_tcgen05(int N, int H, int W, int Cin, int Cout);

/* TPF_OK, or TPF_ERR_TIMEOUT once a bounded wait of a tcgen05 kernel has run
 * out in this process (its output is then not to be trusted; the flag stays set);
 * TPF_ERR_CUDA if the flag cannot be read.  Synchronises with the device. */
int tpfnet_status(void);

/* Data gradient of conv3x3: dx = conv3x3 of dz (the gradient at the convolution's
 * output, ReLU mask already applied) with the flipped, transposed weights, which are
 * written to wflip (9 * Cin * Cout bf16 of caller scratch). */
int tpfnet_conv3x3_dgrad(const void *dz, int N, int H, int W, int Cout, const void *wt, int Cin, void *wflip,
                         void *dx, void *stream);

/* Weight and bias gradients of conv3x3, ADDED to dw ([9][Cout][Cin] float32) and db
 * (Cout float32, or NULL).  Cin % 32 == 0, Cout % 32 == 0. */
int tpfnet_conv3x3_wgrad(const void *x, const void *dz, int N, int H, int W, int Cin, int Cout, float *dw,
                         float *db, void *stream);

/* d[k] = 0 where y[k] <= 0 (ReLU backward on bf16 tensors of `count` elements). */
int tpfnet_relu_mask(void *d, const void *y, long long count, void *stream);

/* 2 x 2 average pooling (H, W even) and its adjoint (dx = dy / 4 spread over each
 * 2 x 2 block, added to dx when accumulate != 0). */
int tpfnet_pool(const void *x, int N, int H, int W, int C, void *y, void *stream);
int tpfnet_pool_back(const void *dy, int N, int H, int W, int C, void *dx, int accumulate, void *stream);

/* Nearest 2 x 2 upsampling of x (N, H/2, W/2, C) into channels [cofs, cofs + C) of
 * y (N, H, W, Ctot), and its adjoint (sum over each 2 x 2 block into dx (N, H/2, W/2, C)). */
int tpfnet_up_into(const void *x, int N, int H, int W, int C, void *y, int Ctot, int cofs, void *stream);
int tpfnet_up_back(const void *dy, int N, int H, int W, int Ctot, int cofs, int C, void *dx, void *stream);

/* Copy channels [sofs, sofs + C) of src (pixels x Sc) into channels [dofs, dofs + C)
 * of dst (pixels x Dc), adding when accumulate != 0 (concatenation and its adjoint). */
int tpfnet_channels(const void *src, int Sc, int sofs, long long pixels, int C, void *dst, int Dc, int dofs,
                    int accumulate, void *stream);

/* 1 x 1 head: out[p][o] = b[o] + sum_c x[p][c] Wt[c][o] (Wt, b, out float32), and its
 * gradients: dx (bf16) overwritten, dW and db ADDED.  C * Cout + Cout <= 12288. */
int tpfnet_head(const void *x, long long pixels, int C, const float *Wt, const float *b, int Cout, float *out,
                void *stream);
int tpfnet_head_back(const void *x, const float *dout, long long pixels, int C, const float *Wt, int Cout,
                     void *dx, float *dW, float *db, void *stream);

/* loss += mean_k (pred[k] - target[k])^2 wch[k % C] (FP64, device); grad[k] = d loss /
 * d pred[k] (or NULL to skip); wch may be NULL (all ones). */
int tpfnet_mse(const float *pred, const float *target, const float *wch, long long count, int C, float *grad,
               double *loss, void *stream);

/* One Adam step (bias-corrected, step >= 1) on float32 parameters p with gradient g and
 * moments m, v; writes the bf16 copy pb as well when pb != NULL. */
int tpfnet_adam(float *p, const float *g, float *m, float *v, long long count, float lr, float b1, float b2,
                float eps, int step, void *pb, void *stream);

/* Planar fields to an interleaved tensor and back, with a per-channel affine map
 * (scale, shift: host arrays of C floats, NULL = 1 and 0; 1 <= C <= 8) and optional
 * base planes (device, same layout as the planar side, NULL = 0):
 *   pack:   dst[p * Cd + c] = (src[c * plane + p] - base[c * plane + p]) * scale[c] + shift[c]
 *           for c < C (float32 dst, or bf16 when dst_bf16 != 0; channels C..Cd-1 untouched);
 *   unpack: dst[c * plane + p] = src[p * C + c] * scale[c] + shift[c] + base[c * plane + p]. */
int tpfnet_pack(const float *src, const float *base, long long plane, int C, long long pixels, const float *scale,
                const float *shift, void *dst, int Cd, int dst_bf16, void *stream);
int tpfnet_unpack(const float *src, long long pixels, int C, const float *scale, const float *shift,
                  const float *base, float *dst, long long plane, void *stream);

/* y = bf16(x). */
int tpfnet_to_bf16(const float *x, long long count, void *y, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TPFNET_H */
