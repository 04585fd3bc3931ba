/*
 * dgsurrogate.h -- C ABI of the learned covariance surrogate.
 *
 * A small CNN maps the occupancy raster of an axon substrate (Sec. 2.2: the
 * disks of a periodic cell, 1 inside a disk) and the conditioning (D, Delta)
 * to the covariance of the Sigma scheme (Sec. 4.1) in units of the free
 * value, y = {Sxx, Sxy, Syy} / (2 D Delta).  The paper has no learned part:
 * the network is trained on Sigma values that the DG solver of dgsigma.h
 * produces, and the DG solve stays its fallback and the reference for its error.
 *
 * Network: input 1 x 128 x 128; four blocks of 3x3 convolution (zero
 * padding) + ReLU + 2x2 average pooling with 48, 96, 192, 384 channels;
 * global average -> 384 features, concatenated with c = (log(D Delta /
 * um^2), D); dense 386 -> 256 + ReLU; dense 256 -> 3 (971,907 parameters).
 * Weights and activations in BF16 (channels-last on the device), all sums
 * accumulated in FP32; FP32 master weights, gradients and Adam.  The
 * convolutions and their input and weight gradients run as implicit GEMMs
 * on the tensor cores (tcgen05.mma, BF16 operands, FP32 accumulators in
 * tensor memory); the gradient of a convolution's output enters them
 * rounded to BF16.
 *
 * Parameter vector (FP32, sg_param_count values), in this order: for each
 * convolution l = 1..4 its weights [Cout][Cin][3][3] then biases [Cout];
 * dense 1 weights [256][386], biases [256]; dense 2 weights [3][256],
 * biases [3].
 *
 * Batches are device pointers: occ [B][128][128] bytes, cond [B][2] FP32,
 * target/out [B][3] FP32, 1 <= B <= max_batch.  Calls synchronise the
 * network's own stream before returning.  Status codes are those of
 * dgsigma.h; DG_ETIMEOUT if a tensor-core kernel's bounded wait for its MMAs
 * ran out (the network's outputs are then undefined; the network stays
 * usable).
 */
#ifndef DGSURROGATE_H
#define DGSURROGATE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_net sg_net;

/* New network with He-uniform weights drawn from a counter-based generator
 * seeded by seed, zero biases, on device (-1 = current). */
int sg_create(int max_batch, unsigned long long seed, int device, sg_net **out);
void sg_destroy(sg_net *net);
const char *sg_last_error(const sg_net *net);

int sg_param_count(sg_net *net, size_t *count);
/* FP32 master parameters to / from host memory (sg_param_count floats). */
int sg_get_params(sg_net *net, float *host);
int sg_set_params(sg_net *net, const float *host);

/* Forward pass: out[B][3] (device) = y for the batch. */
int sg_predict(sg_net *net, const uint8_t *occ, const float *cond, int B, float *out);

/* Loss mean_b,o (y - target)^2 and its gradient with respect to every
 * parameter (host buffers; either may be NULL), without an update. */
int sg_gradients(sg_net *net, const uint8_t *occ, const float *cond, const float *target, int B,
                 float *loss_host, float *grad_host);

/* One Adam step (beta 0.9, 0.999, eps 1e-8) with learning rate lr on the
 * mean squared error; loss_host (may be NULL) receives the loss before the
 * update. */
int sg_train_step(sg_net *net, const uint8_t *occ, const float *cond, const float *target, int B,
                  float lr, float *loss_host);

#ifdef __cplusplus
}
#endif

#endif /* DGSURROGATE_H */
