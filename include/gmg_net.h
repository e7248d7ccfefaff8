/*
 * gmg_net.h -- C ABI of the learned warm start: the kernels of a small 3D
 * convolutional network that predicts the initial guess of a pressure solve.
 *
 * The paper has no learned component; this network is an addition on top of
 * its method (the solver of Sec. 3 then iterates from the network's guess to
 * the same tolerance, so it both uses and judges the prediction).
 *
 * Layout.  Activations and activation gradients are BF16, channels last:
 * element (z, y, x, c) of a D x H x W grid with channel stride cs sits at
 * ((z * H + y) * W + x) * cs + c.  Channel counts of convolution inputs and
 * outputs are multiples of 16 (pad with zero channels).  Packed 3x3x3 weights
 * are [27][co][ci] (tap t = 9 dz + 3 dy + dx, offsets dz-1, dy-1, dx-1);
 * the "flipped" copy used for input gradients is [27][ci][co] with tap
 * 26 - t.  Master weights, gradients and optimiser state are FP32 in the
 * packed layout.  Every pointer is device memory (except the `periodic` flags
 * of gmg_net_pack_input, a host array); every call is asynchronous
 * on `stream` and returns 0, or 1 for a bad argument, or 2 for a CUDA error.
 * Arithmetic: products of BF16 operands on the tensor cores, FP32 sums.
 */
#ifndef GMG_NET_H
#define GMG_NET_H

#ifdef __cplusplus
extern "C" {
#endif

typedef unsigned short gmg_bf16;   /* bit pattern of a bfloat16 */

/*
 * y[:, :, :, yoff + o] = act(b[o] + sum over taps and ci of w[t][o][ci] x(shifted)[ci]),
 * zero padding outside the grid; act = ReLU if relu != 0.  ci, co multiples
 * of 16 (co <= 96); cx >= ci and cy >= yoff + co are the channel strides.
 * bias may be NULL.  With the flipped weights, no bias and no ReLU this is
 * the input gradient of the convolution.
 */
int gmg_net_conv3(int D, int H, int W, const gmg_bf16* x, int cx, int ci, const gmg_bf16* w, const float* bias,
                  int co, int relu, gmg_bf16* y, int cy, int yoff, void* stream);

/*
 * Weight and bias gradients: dw[t][o][ci] += sum over cells of g[o] x(shifted by t)[ci],
 * db[o] += sum over cells of g[o] (db may be NULL).  g has co channels at
 * stride cg; x has ci channels at stride cx.  dw and db accumulate (FP32).
 */
int gmg_net_conv3_wgrad(int D, int H, int W, const gmg_bf16* x, int cx, int ci, const gmg_bf16* g, int cg,
                        int co, float* dw, float* db, void* stream);

/* g[c] = 0 where y[c] <= 0 (ReLU backward, in place); C channels at strides cg, cy. */
int gmg_net_relu_backward(int D, int H, int W, gmg_bf16* g, int cg, const gmg_bf16* y, int cy, int C,
                          void* stream);

/* y[:, :, :, yoff + c] = mean of each 2x2x2 block of x (output grid D/2 x H/2 x W/2). */
int gmg_net_pool2(int D, int H, int W, const gmg_bf16* x, int cx, int C, gmg_bf16* y, int cy, int yoff,
                  void* stream);

/*
 * Adjoint of pool2 plus an optional second gradient: gx[c] = gy[block][c] / 8
 * (+ add[addoff + c] if add is not NULL).  D, H, W are the fine dimensions.
 */
int gmg_net_pool2_backward(int D, int H, int W, const gmg_bf16* gy, int cgy, int C, gmg_bf16* gx, int cgx,
                           const gmg_bf16* add, int cadd, int addoff, void* stream);

/* Nearest 2x upsampling: y (2D x 2H x 2W)[:, :, :, yoff + c] = x[c]; D, H, W coarse dimensions. */
int gmg_net_up2(int D, int H, int W, const gmg_bf16* x, int cx, int C, gmg_bf16* y, int cy, int yoff,
                void* stream);

/* Adjoint of up2: gx[c] = sum over the 8 children of gy[goff + c]; D, H, W coarse dimensions. */
int gmg_net_up2_backward(int D, int H, int W, const gmg_bf16* gy, int cgy, int goff, int C, gmg_bf16* gx,
                         int cgx, void* stream);

/*
 * Network input, 16 channels: (b / s, mean of the six face coefficients,
 * p_prev / s, r / s, 0, ...) with r = b - A p_prev the residual of the
 * previous pressure (difference form of the solver's operator, FP32) and
 * s = RMS of b, written to s_out[0]; s_out[1] receives RMS of r (device
 * float[2]; each 1 where zero).  b, p_prev (may be NULL: zero, then r = b), bx,
 * by, bz are FP32 [D][H][W] arrays in the solver's layout; periodic: host array
 * of 3 flags for (x, y, z) (NULL: walls).  Uses the scratch `red` (device
 * double[2]).
 */
int gmg_net_pack_input(int D, int H, int W, const float* b, const float* p_prev, const float* bx,
                       const float* by, const float* bz, const int* periodic, gmg_bf16* x0, float* s_out,
                       double* red, void* stream);

/* out[cell] = sum_c w[c] h[c] + b[0] (1x1x1 convolution of 16 channels, FP32 out). */
int gmg_net_head(int D, int H, int W, const gmg_bf16* h, int ch, const float* w, const float* b, float* out,
                 void* stream);

/*
 * Loss of the prediction q = out + p_prev / s against t = target / s:
 * |(q - mean q) - (t - mean t)|^2 / |t - mean t|^2 (target and p_prev FP32,
 * p_prev may be NULL: zero; s device float, the output scale: s_out[0] of
 * gmg_net_pack_input).  Writes the loss to *loss (device double) and
 * d(loss)/d(out) to gout.  Uses scratch red (device double[4]).
 */
int gmg_net_loss(int D, int H, int W, const float* out, const float* target, const float* p_prev, const float* s,
                 float* gout, double* loss, double* red, void* stream);

/*
 * Residual loss of the prediction p0 = p_prev + s out (s the output scale,
 * device float; p_prev may be NULL: zero) against the source b:
 * L = |b - A p0|^2 / |b|^2 with A the solver's operator (difference form,
 * FP32; walls or periodic axes as in gmg_net_pack_input; periodic is a host
 * array or NULL), written to *loss (device double), and
 * d(L)/d(out) = s * (-2 A (b - A p0) / |b|^2) to gout (A is symmetric).
 * work: device scratch of 2 D H W floats; red: device double[2].
 */
int gmg_net_residual_loss(int D, int H, int W, const float* out, const float* p_prev, const float* s, const float* b,
                          const float* bx, const float* by, const float* bz, const int* periodic, float* work,
                          float* gout, double* loss, double* red, void* stream);

/* Head backward: gh[c] = w[c] gout, dw[c] += sum gout h[c], db[0] += sum gout. */
int gmg_net_head_backward(int D, int H, int W, const float* gout, const gmg_bf16* h, int ch, const float* w,
                          gmg_bf16* gh, float* dw, float* db, void* stream);

/* p0 = s * out + p_prev (the prediction: the network gives the increment over
 * the previous pressure in units of the output scale s, s_out[0] of
 * gmg_net_pack_input; p_prev may be NULL: zero). */
int gmg_net_unscale(long long n, const float* out, const float* s, const float* p_prev, float* p0, void* stream);

/*
 * Adam on n FP32 parameters (step number t >= 1, bias-corrected moments).
 * If wb is not NULL the updated values are also written as BF16 to wb and,
 * for 3x3x3 weights (ci > 0), the flipped transposed copy to wt: the
 * parameters are then packed [27][co][ci].
 */
int gmg_net_adam(long long n, float* w, const float* g, float* m, float* v, int t, float lr, float b1, float b2,
                 float eps, gmg_bf16* wb, gmg_bf16* wt, int co, int ci, void* stream);

/* n FP32 values set to zero (gradient buffers). */
int gmg_net_zero(long long n, float* a, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GMG_NET_H */
