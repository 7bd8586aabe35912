/*
 * bpm_corrector.h - C ABI of the learned coarse-step corrector (libbpm.so).
 *
 * Coarse split-steps of length 4 dz (index screen averaged over the four fine
 * slices, bpm_coarsen_index) cost a quarter of the fine steps but add a
 * splitting error.  The corrector is a small convolutional network f applied
 * after each coarse step, E <- E + f(E): four 3x3 convolutions with circular
 * padding (C_in -> 32 -> 32 -> 32 -> 2, ReLU between), input channels
 * Re E, Im E and optionally the averaged index step (times a caller scale),
 * output the correction of Re E and Im E (times a fixed residual scale).  It is trained on pairs (one coarse
 * step from a fine-step field at plane 4j, the fine-step field at plane 4j+4)
 * that the propagation itself generates.  The paper has no network: it only
 * motivates wave-optical simulations as training data for machine learning
 * (introduction); this is an addition of the library, checked against an
 * FP64 CPU implementation of the same network.
 *
 * Numerics: FP32 master weights and Adam moments (beta1 0.9, beta2 0.999,
 * eps 1e-8); the convolutions use the weights rounded to BF16 and accumulate
 * in FP32.  Tensors are float, [batch][channel][y][x], H and W multiples of 16.
 * Parameters are one flat float vector [W1, b1, W2, b2, W3, b3, W4, b4] with
 * weights [C_out][C_in][3][3].  Device pointers d_*, host pointers h_*; work is
 * asynchronous on the stream unless a host result is requested.  Status codes
 * as in bpm.h; bpm_corrector_last_error() gives the message.
 */
#ifndef BPM_CORRECTOR_H
#define BPM_CORRECTOR_H

#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bpm_corrector_s *bpm_corrector_t;

/* Create a corrector with in_channels 2 (field only) or 3 (field and index),
 * and device buffers for batches up to max_batch of max_h x max_w (multiples
 * of 16).  Parameters start at zero; set them with bpm_corrector_set_params.
 * Owns about (7 * 32 + 8) * max_batch * max_h * max_w floats of activations. */
int bpm_corrector_create(bpm_corrector_t *out, int in_channels, int max_batch, int max_h, int max_w,
                         cudaStream_t stream);

/* Number of parameters (flat vector length). */
int bpm_corrector_param_count(bpm_corrector_t c);

/* Residual scale sigma (default 1): the network output is
 * x[:, :2] + sigma f(x).  Set it to the RMS size of the corrections to be
 * learned so that f is of order one. */
int bpm_corrector_set_residual_scale(bpm_corrector_t c, float sigma);

/* Load FP32 master parameters (n = param count), reset the Adam moments and
 * the step counter; synchronises the stream. */
int bpm_corrector_set_params(bpm_corrector_t c, const float *h_params, int n, cudaStream_t stream);

/* Copy parameters to the host: which = 0 FP32 masters, 1 the BF16-rounded
 * working copy, 2 the gradient of the last bpm_corrector_loss_grad;
 * synchronises the stream. */
int bpm_corrector_get_params(bpm_corrector_t c, float *h_params, int n, int which, cudaStream_t stream);

/* d_out[b] = d_x[b][0:2] + sigma f(d_x[b]); d_x [batch][C_in][h][w], d_out [batch][2][h][w]. */
int bpm_corrector_forward(bpm_corrector_t c, const float *d_x, float *d_out, int batch, int h, int w,
                          cudaStream_t stream);

/* Mean squared error L = sum (x[:, :2] + sigma f(x) - target)^2 / numel(target) and
 * its gradient with respect to every parameter (kept in the corrector);
 * h_loss (nullable) receives L, which synchronises the stream. */
int bpm_corrector_loss_grad(bpm_corrector_t c, const float *d_x, const float *d_target, int batch, int h, int w,
                            float *h_loss, cudaStream_t stream);

/* One Adam step with learning rate lr on the gradient of the last
 * bpm_corrector_loss_grad. */
int bpm_corrector_adam(bpm_corrector_t c, float lr, cudaStream_t stream);

/* bpm_corrector_loss_grad followed by bpm_corrector_adam. */
int bpm_corrector_train_step(bpm_corrector_t c, const float *d_x, const float *d_target, int batch, int h, int w,
                             float lr, float *h_loss, cudaStream_t stream);

/* Pack complex float fields [batch][h][w] into the network layout d_x
 * [batch][C_in][h][w]: each field divided by its RMS amplitude a_b (so the
 * correction scales linearly with the field, as the splitting error does),
 * and for 3 input channels the FP16 index plane of the field times dn_scale
 * (zeros when d_dn is NULL).  When d_targets (complex [batch][h][w]) is given,
 * d_t [batch][2][h][w] receives the targets divided by the same a_b.
 * batch <= the corrector's max_batch. */
int bpm_corrector_pack(bpm_corrector_t c, const void *d_fields, const void *d_targets, const void *d_dn,
                       float dn_scale, float *d_x, float *d_t, int batch, int h, int w, cudaStream_t stream);

/* In place on one complex float field [h][w]: E <- E + a sigma f(E / a),
 * a the RMS amplitude of E (d_dn: the coarse step's averaged index plane for
 * 3-channel correctors, else NULL). */
int bpm_corrector_apply(bpm_corrector_t c, void *d_field, const void *d_dn, float dn_scale, int h, int w,
                        cudaStream_t stream);

/* Averaged index volume of coarse steps: d_out[zc] = FP16(mean of d_dn[zc *
 * factor + k], k < factor), zc < nz / factor; volumes [z][ny][nx] FP16. */
int bpm_coarsen_index(const void *d_dn, int nz, int ny, int nx, int factor, void *d_out, cudaStream_t stream);

/* Inference engine of bpm_corrector_forward and bpm_corrector_apply: on != 0
 * (the default) runs the four convolutions on the tensor cores (tcgen05
 * kind::f16: BF16 activations and weights in shared memory, FP32 accumulators
 * in tensor memory, one 128-pixel row segment per MMA tile) whenever w is a
 * multiple of 128, else on the FP32 pipes; on = 0 always uses the FP32 pipes
 * (FP32 activations), as training does. */
int bpm_corrector_set_tensor_cores(bpm_corrector_t c, int on);

/* Training engine of bpm_corrector_loss_grad and bpm_corrector_train_step:
 * on != 0 computes the loss and every gradient on the tensor cores whenever
 * w is a multiple of 128 and h even (tcgen05 kind::f16: the forward pass keeps
 * BF16 activations; per layer the weight and bias gradients are a GEMM over
 * the pixels with taps x input channels as rows, and the data gradient of the
 * layer below is the adjoint convolution with the ReLU mask; BF16 operands,
 * FP32 accumulation, FP32 master weights and Adam as before).  on = 0 (the
 * default) trains on the FP32 pipes with FP32 activations and gradients, the
 * path checked against the FP64 oracle to 1e-4. */
int bpm_corrector_set_train_tensor_cores(bpm_corrector_t c, int on);

/* Synchronise the stream and report a device error of the tensor-core path
 * (BPM_ERR_TIMEOUT when a bounded wait gave up). */
int bpm_corrector_check(bpm_corrector_t c, cudaStream_t stream);

int bpm_corrector_free(bpm_corrector_t c);
const char *bpm_corrector_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BPM_CORRECTOR_H */
