/* C ABI of the learned warm start's network kernels (libfdlbm.so).
 *
 * The paper has no counterpart: these layers serve a small 3D convolutional U-Net that
 * predicts steady velocity, mole-fraction and temperature fields of a porous geometry
 * from its solid mask and inlet state; the solver uses the prediction only as the initial
 * state of a run (fdlbm_set_fields), which then proceeds to the steady-state residual as
 * usual.
 *
 * Tensors are device pointers owned by the caller. Activations are NDHWC bf16
 * ([batch][z][y][x][channels], channels innermost), 16-byte aligned; a volume is (N, D,
 * H, W) = (batch, z, y, x). 3x3x3 weights are bf16 [c_out][27][c_in] with the tap index
 * 9 dz + 3 dy + dx (offsets dz - 1, dy - 1, dx - 1); biases, 1x1x1 head weights,
 * gradients and optimiser state are float32. Every call is asynchronous on `stream` (a
 * cudaStream_t; NULL: the legacy default stream) and returns FDLBM_EINVAL for bad
 * arguments (nothing is launched) or FDLBM_ECUDA for a failed launch; the message is in
 * fdlbm_net_last_error(). The convolution kernels give up on a stalled pipeline after a
 * time limit and raise a device-side flag that fdlbm_net_check reports as
 * FDLBM_ETIMEOUT. */
#ifndef FDLBM_NET_H
#define FDLBM_NET_H

#include "fdlbm.h"

#ifdef __cplusplus
extern "C" {
#endif

const char* fdlbm_net_last_error(void);

/* Wait for `stream` and report (then clear) the device-side error flag of the
 * convolution kernels: FDLBM_ETIMEOUT if a pipeline wait ran out. */
fdlbm_status fdlbm_net_check(void* stream);

/* 3x3x3 same-size convolution with zero padding on the tensor cores:
 * y[v][o] = bias[o] + sum_{tap, c} w[o][tap][c] x[v + tap - 1][c], x being the channel
 * concatenation of x0 (c0 channels) and x1 (c1 channels, 0 for none); optionally ReLU
 * (relu != 0), then a ReLU-backward mask: y[v][o] = 0 where mask[v][o] <= 0 (mask NULL:
 * none). c0, c1: multiples of 16; c_out: 16..128, a multiple of 16; D, H, W: multiples of
 * 4, 4, 8. With the flipped weights of fdlbm_conv3_flip_weights and the output gradient
 * as x, it returns the input gradient (no bias, no ReLU; the mask applies the ReLU
 * backward of the layer that produced the input). */
fdlbm_status fdlbm_conv3_fwd(const void* x0, int c0, const void* x1, int c1, int N, int D, int H, int W,
                             const void* w, const float* bias, int c_out, int relu, const void* mask, void* y,
                             void* stream);

/* wf[c][26 - tap][o] = w[o][tap][c]: the weights of the input-gradient convolution. */
fdlbm_status fdlbm_conv3_flip_weights(const void* w, int c_out, int c_in, void* wf, void* stream);

/* Weight and bias gradients of the 3x3x3 convolution on the tensor cores:
 * gw[o][tap][c] = sum_v gy[v][o] x[v + tap - 1][c] (x = concat(x0, x1), zero outside the
 * volume), gb[o] = sum_v gy[v][o] (gb may be NULL). gw and gb are overwritten. c0, c1:
 * multiples of 16; c_out: 8..128, a multiple of 8. */
fdlbm_status fdlbm_conv3_wgrad(const void* x0, int c0, const void* x1, int c1, int N, int D, int H, int W,
                               const void* gy, int c_out, float* gw, float* gb, void* stream);

/* Mean over 2x2x2 blocks: y has (D/2, H/2, W/2); and its gradient gx = gy / 8 repeated
 * over each block, zero where mask <= 0 (mask: NULL or the fine-grid activation). */
fdlbm_status fdlbm_net_avgpool2(const void* x, int c, int N, int D, int H, int W, void* y, void* stream);
fdlbm_status fdlbm_net_avgpool2_bwd(const void* gy, int c, int N, int D, int H, int W, const void* mask, void* gx,
                                    void* stream);

/* Decoder input on the fine grid (D, H, W): out[v] = [h[v / 2] (cu channels, nearest
 * upsampling of the coarse h), skip[v] (cs channels; cs = 0 and skip NULL for the
 * upsampling alone)]; and its gradient: gh[v'] = sum of
 * g[v][0:cu] over the 8 fine voxels of v' (zero where mask_h <= 0), gskip = (gskip +
 * g[v][cu:]) zeroed where mask_skip <= 0. */
fdlbm_status fdlbm_net_up2cat(const void* h, int cu, const void* skip, int cs, int N, int D, int H, int W, void* out,
                              void* stream);
fdlbm_status fdlbm_net_up2cat_bwd(const void* g, int cu, int cs, int N, int D, int H, int W, const void* mask_h,
                                  void* gh, const void* mask_skip, void* gskip, void* stream);

/* dst += src (bf16, count elements). */
fdlbm_status fdlbm_net_add(void* dst, const void* src, long long count, void* stream);

/* 1x1x1 output head: y[v][o] = b[o] + sum_c w[o][c] h[v][c] (y, w, b float32), and its
 * gradients: gh[v][c] = sum_o w[o][c] gy[v][o] zeroed where h <= 0 (the head reads a ReLU
 * output), gw, gb overwritten. */
fdlbm_status fdlbm_net_conv1(const void* h, int c, const float* w, const float* b, int c_out, long long nvox, float* y,
                             void* stream);
fdlbm_status fdlbm_net_conv1_bwd(const float* gy, int c_out, const float* w, int c, const void* h, long long nvox,
                                 void* gh, float* gw, float* gb, void* stream);

/* Weighted mean-squared error: *loss = sum_{v, o} wgt[v] (y - t)^2 / (c_out nvox) (FP64,
 * device), gy = 2 wgt (y - t) / (c_out nvox); wgt NULL: 1. */
fdlbm_status fdlbm_net_mse(const float* y, const float* t, const float* wgt, int c_out, long long nvox, double* loss,
                           float* gy, void* stream);

/* One Adam step (Kingma and Ba) of step number t >= 1 on count parameters: m, v moment
 * estimates updated in place, p -= lr m_hat / (sqrt(v_hat) + eps); p_bf16 (optional)
 * receives the updated parameters in bf16. */
fdlbm_status fdlbm_net_adam(float* p, const float* g, float* m, float* v, long long count, int t, float lr, float b1,
                            float b2, float eps, void* p_bf16, void* stream);

/* y = bf16(x), count elements. */
fdlbm_status fdlbm_net_to_bf16(const float* x, long long count, void* y, void* stream);

#ifdef __cplusplus
}
#endif
#endif
