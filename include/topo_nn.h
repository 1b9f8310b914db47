/*
 * topo_nn.h -- the learned PCG warm start of libtopo.so (C-ABI).
 *
 * The paper solves every state equation from scratch (Section 4.3, sparse LU).
 * This part adds a small 3D convolutional network that predicts the shape of
 * the displacement field of a 3D problem from its densities, supports and
 * loads; the prediction, scaled by the energy-optimal factor, starts the
 * Jacobi-PCG solve of tp_solve.  The true FP64 residual judges the result: a
 * start worse than u = 0 is dropped (tp_solve_info.warm_fallback).
 *
 * Network (a 4-level U-Net with additive skips; widths c0..c3, c3 == c2):
 *   enc0 conv(in,c0) conv(c0,c0)=s0 pool | enc1 conv(c0,c1) conv(c1,c1)=s1 pool |
 *   enc2 conv(c1,c2) conv(c2,c2)=s2 pool | mid conv(c2,c3) up +s2 |
 *   dec2 conv(c3,c1) up +s1 | dec1 conv(c1,c0) up +s0 | dec0 conv(c0,c0) |
 *   head conv(c0,out)
 * Every conv is 3 x 3 x 3 with zero padding 1 and a bias, followed by ReLU
 * except the head; pool = 2 x 2 x 2 average; up = nearest, factor 2.
 * Numerics: weights and stored activations bfloat16 (round to nearest even),
 * every product accumulated in FP32, gradients FP32, Adam on FP32 master
 * weights.
 *
 * Layouts: tensors [n][C][D][H][W] (W fastest; D = z, H = y, W = x of the
 * element grid).  Parameters are packed per layer in network order as
 * [w (c_out * c_in * 27) | b (c_out)], weights w[c_out][c_in][27] with tap
 * t = (dz+1)*9 + (dy+1)*3 + (dx+1).
 * Pointers named *_bf16 carry bfloat16 bit patterns (uint16).  Tensor
 * arguments of tpnn_forward / tpnn_backward / tpnn_mse / tpnn_train_step are
 * DEVICE pointers on the network's device; parameter arrays of
 * tpnn_set_params / tpnn_get_params / tpnn_get_grads are HOST pointers.
 * Errors follow topo.h: a tp_status is returned, tpnn_last_error describes it,
 * and the handle stays valid.  All work runs on the stream given at creation.
 */
#ifndef TOPO_NN_H
#define TOPO_NN_H

#include "topo.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tpnn tpnn;

/* Input channels of the warm-start features (tpnn_features). */
#define TPNN_FEATURES 8

/* Create a network with c_in input channels (1..64), c_out = 3 output channels
 * and widths[4] in {16, 32, 64} with widths[3] == widths[2].  Parameters start
 * at zero; set them with tpnn_set_params. */
tp_status tpnn_create(int c_in, int c_out, const int* widths, void* cuda_stream, tpnn** out);
void tpnn_destroy(tpnn* m);
const char* tpnn_last_error(const tpnn* m);
/* Number of packed FP32 parameters. */
long long tpnn_param_count(const tpnn* m);
/* Outputs (each may be NULL): c_in, c_out, widths[4]. */
tp_status tpnn_info(const tpnn* m, int* c_in, int* c_out, int* widths);
/* Host FP32 parameter vector in, out; set also resets the Adam state. */
tp_status tpnn_set_params(tpnn* m, const float* src);
tp_status tpnn_get_params(tpnn* m, float* dst);
/* Host copy of the accumulated gradients (same packing as the parameters). */
tp_status tpnn_get_grads(tpnn* m, float* dst);

/* y[n][c_out][D][H][W] (FP32, device) = net(x[n][c_in][D][H][W] (bf16, device)).
 * D, H, W must be >= 8 and multiples of 8 (three poolings).  x must stay valid
 * until the next forward (the backward reads it). */
tp_status tpnn_forward(tpnn* m, const void* x_bf16, int n, int D, int H, int W, float* y);
/* Accumulate into the gradient buffer the gradients of sum(gy * y) with
 * respect to every parameter, for the input of the last tpnn_forward;
 * gy[n][c_out][D][H][W] FP32 device.  TP_ERR_STATE without a forward. */
tp_status tpnn_backward(tpnn* m, const float* gy);
tp_status tpnn_zero_grad(tpnn* m);
/* One Adam step (bias-corrected) on the accumulated gradients. */
tp_status tpnn_adam(tpnn* m, float lr, float beta1, float beta2, float eps);
/* Mean squared error of y (FP32) against t (bf16), count values: writes
 * gy = 2 (y - t) / count and, if loss != NULL, the mean (host, synchronises). */
tp_status tpnn_mse(tpnn* m, const float* y, const void* t_bf16, long long count, float* gy, double* loss);
/* zero_grad, forward, mse, backward, Adam(lr, 0.9, 0.999, 1e-8) in one call. */
tp_status tpnn_train_step(tpnn* m, const void* x_bf16, const void* t_bf16, int n, int D, int H, int W, float lr,
                          double* loss);

/* ---------------------------------------------------------------------------
 * Problem-side helpers (3D problems only; nelx, nely, nelz multiples of 8).
 *
 * tpnn_features writes the network input of each load case k to
 * dst_bf16[k][8][nelz][nely][nelx] (device): per element
 *   0  the density rho_e,
 *   1  the fraction of the element's 8 nodes that have a fixed DOF,
 *   2-4 the element's share of the load, sum over its nodes of f_k / (8 max|f_k|),
 *   5-7 the element centre's coordinates divided by (nelx, nely, nelz).
 * tpnn_targets writes the training target of each case from the current
 * displacement u_k: per element the mean of u_k over its 8 nodes, divided by
 * the largest magnitude of those means over all elements and components of
 * the case: dst_bf16[k][3][nelz][nely][nelx] (device).  TP_ERR_STATE without a
 * solution.
 * tp_warm_start_nn runs the network on the features, averages its per-element
 * output onto the nodes (mean over the adjacent elements, zero on fixed DOFs)
 * to get u^_k, and stores u_k = alpha_k u^_k with alpha_k = f_k^T u^_k /
 * u^_k^T K u^_k (the factor minimising the energy norm of the error) as the
 * start of the next tp_solve with warm_start = TP_WARM_USER.  alpha (host,
 * n_cases doubles, may be NULL) receives the factors, ms (host, may be NULL)
 * the device time of the whole warm start.  The network must have
 * c_in = TPNN_FEATURES and c_out = 3. */
tp_status tpnn_features(tp_problem* p, void* dst_bf16);
tp_status tpnn_targets(tp_problem* p, void* dst_bf16);
tp_status tp_warm_start_nn(tp_problem* p, tpnn* net, double* alpha, double* ms);
/* Training loss of the warm start: for the network output y[n_cases][3][nelz]
 * [nely][nelx] (FP32, device) of this problem, u^ = node average of y (as in
 * tp_warm_start_nn) and
 *   L_k = ||u*_k - alpha_k u^_k||_K^2 / c_k = 1 - (f_k^T u^_k)^2 / ((u^_k^T K u^_k) c_k),
 * the energy-norm error of the best multiple of u^_k relative to the energy
 * c_k = f_k^T u*_k of the solution (the case's compliance, host, > 0).  Writes
 * dL_k/dy to gy (FP32, device, same layout as y); loss (host, n_cases, may be
 * NULL) receives L_k.  dL/du^ = -(2 alpha / c)(f - alpha K u^): the scaled
 * residual of the start. */
tp_status tpnn_energy_grad(tp_problem* p, const float* y, const double* comp, float* gy, double* loss);

#ifdef __cplusplus
}
#endif
#endif /* TOPO_NN_H */
