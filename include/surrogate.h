/*
 * surrogate.h -- C ABI of the kernels behind the learned warm start of lb_steady: a small
 * 3D convolutional encoder-decoder that maps a porous medium to an estimate of its steady
 * flow and density, used only as the starting state (u_init, rho_init) of lb_steady (the
 * plain LB runs to the same residual from there, so it alone decides convergence). The paper
 * has no counterpart; it solves the LB from rest (Sec. "Introduction", Eq. lb_evolution).
 *
 * Conventions (in addition to those of mp.h, whose status codes and mp_last_error() these
 * functions share; they are exported by the same library, libmp):
 *  - Activations are BF16, channels last: x[b][v][c], v = x + W*(y + H*z) over a periodic
 *    D x H x W box (every axis periodic), c fastest. Channel counts are multiples of 16.
 *  - Convolutions are 3x3x3, stride 1, periodic ("circular") padding. Weights are BF16 in
 *    [27][N][K] order (tap-major; tap = 9*(dz+1) + 3*(dy+1) + (dx+1)): N output channels by
 *    K input channels for the forward pass. Master weights and gradients are FP32 in
 *    [27][Cin][Cout] order. Biases are FP32.
 *  - Products run on the tensor cores (mma.sync m16n8k16, BF16 inputs, FP32 accumulation).
 *  - Every pointer is device memory; every call is asynchronous on `stream` (a
 *    cudaStream_t, NULL = legacy default stream) and returns MP_OK or MP_EINVAL/MP_ECUDA.
 */
#ifndef SURROGATE_H
#define SURROGATE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * sg_conv3d -- y[b][v][n] = act(bias[n] + sum_{tap, k} x[b][v + sign*o_tap][k] w[tap][n][k]).
 *  x        BF16 [B][V][K];  w  BF16 [27][N][K];  bias FP32 [N] or NULL.
 *  y        BF16 [B][V][N] output or NULL;  yf  FP32 [B][V][N] output or NULL (one required).
 *  sign     +1 for the forward convolution; -1 gives the transposed convolution used for the
 *           gradient with respect to the input (with w in [27][Cin][Cout] order, N = Cin,
 *           K = Cout).
 *  relu     nonzero: act = max(0, .), else identity.
 * Needs K and N multiples of 16, D, H, W >= 1. Runs on the 5th-generation tensor cores
 * (tcgen05.mma, FP32 accumulators in tensor memory): blocks of 128 voxels x up to 256 output
 * channels. Its waits are bounded; sg_check reports one that gave up.
 */
int sg_conv3d(const void* x, const void* w, const float* bias, void* y, float* yf, int B, int D, int H,
              int W, int K, int N, int sign, int relu, void* stream);

/*
 * sg_check -- synchronises the stream and returns MP_ETIMEOUT (clearing the record) when a
 * bounded wait inside a tensor-core convolution launched since the last check gave up, so
 * that its output is not valid; MP_OK otherwise. (No counterpart in the paper.)
 */
int sg_check(void* stream);

/*
 * sg_conv3d_wgrad -- dw[tap][ci][co] += sum_{b, v} x[b][v + o_tap][ci] dy[b][v][co] and, when
 * dbias is not NULL, dbias[co] += sum_{b, v} dy[b][v][co] (FP32 accumulation; the caller
 * zeroes dw and dbias before the first call of a step). x BF16 [B][V][Cin], dy BF16
 * [B][V][Cout]. Summation order varies between runs (atomic adds).
 */
int sg_conv3d_wgrad(const void* x, const void* dy, float* dw, float* dbias, int B, int D, int H, int W, int Cin,
                    int Cout, void* stream);

/* sg_pool2 -- 2x2x2 average pooling, x [B][D][H][W][C] -> y [B][D/2][H/2][W/2][C] (even
 * D, H, W); sg_pool2_grad -- dx[child] = dy[parent] / 8. */
int sg_pool2(const void* x, void* y, int B, int D, int H, int W, int C, void* stream);
int sg_pool2_grad(const void* dy, void* dx, int B, int D, int H, int W, int C, void* stream);

/* sg_up2 -- nearest-neighbour 2x upsampling, x [B][D][H][W][C] -> y [B][2D][2H][2W][C];
 * sg_up2_grad -- dx[parent] = sum of dy over its 8 children. (D, H, W are the coarse sizes.) */
int sg_up2(const void* x, void* y, int B, int D, int H, int W, int C, void* stream);
int sg_up2_grad(const void* dy, void* dx, int B, int D, int H, int W, int C, void* stream);

/* sg_add -- y = a + b (BF16, n values; y may alias a or b).
 * sg_relu_grad -- g[i] = 0 where act[i] <= 0 (in place; the post-activation output marks
 * where the unit was active). */
int sg_add(const void* a, const void* b, void* y, int64_t n, void* stream);
int sg_relu_grad(const void* act, void* g, int64_t n, void* stream);

/*
 * sg_pack_input -- network input from node classes (mp_classify's encoding: 0 solid,
 * 1 fluid, 2 interfacial, +4 in the largest fluid cluster), for the flow driven along axis
 * `axis` (0 = x, 1 = y, 2 = z): the network is trained for a force along its first axis,
 * so the box is read with that axis moved first. x BF16 [V][16]: channel 0 = fluid,
 * channel 1 = in the forced cluster, the rest 0. cls u8 [nz][ny][nx] of the original box.
 */
int sg_pack_input(const uint8_t* cls, void* x, int nx, int ny, int nz, int axis, void* stream);

/*
 * sg_unpack_output -- on the nodes of the forced cluster of the original box only:
 * u[c][n] += scale_u * y[v][c'] with the network's axes mapped back (c' is the network
 * channel of lattice component c for a force along `axis`), and, when rho is not NULL,
 * rho[n] += scale_rho * (y[v][3] - m) with m the mean of y[.][3] over the forced cluster, so
 * the added density has zero mean there (the LB conserves each region's mass, and a cold
 * start has mean density 1). y FP32 [V][ldy] (ldy >= 4 with rho), u FP32 SoA [3][N], rho
 * FP32 [N].
 */
int sg_unpack_output(const float* y, int ldy, const uint8_t* cls, float* u, float* rho, int nx, int ny, int nz,
                     int axis, float scale_u, float scale_rho, void* stream);

/*
 * sg_pack_target -- training target (FP32 [V][4], network axes for a force along `axis`):
 * t[v][c] = scale_u * u[c'][n] for c < 3 and t[v][3] = scale_rho * (rho[n] - 1) on fluid
 * nodes (0 on solids), from an LB steady state u (FP32 SoA [3][N]) and rho (FP32 [N]).
 */
int sg_pack_target(const float* u, const float* rho, float* t, int nx, int ny, int nz, int axis, float scale_u,
                   float scale_rho, void* stream);

/*
 * sg_mse -- masked mean squared error of y (FP32 [B][V][ldy], channels 0..nc-1) against t
 * (FP32 [B][V][nc]) over fluid voxels (x channel 0 of the packed input, BF16 [B][V][16]);
 * writes the loss (FP64, accumulated into *loss, zeroed by the caller) and the BF16 gradient
 * dy [B][V][ldy] = 2 (y - t) / (nc n_fluid) on fluid voxels and channels below nc, 0
 * elsewhere. n_fluid is the number of fluid voxels over the batch; 1 <= nc <= ldy.
 */
int sg_mse(const float* y, int ldy, const float* t, int nc, const void* x, void* dy, double* loss, int B, int V,
           double n_fluid, void* stream);

/*
 * sg_adam -- one Adam step (Kingma and Ba, 2015) on n FP32 parameters p with gradient g and
 * moments m, v (bias-corrected with step t >= 1), then the BF16 copies: when wf is not NULL
 * the parameters are conv weights [27][cin][cout] and are written to wf in forward order
 * [27][cout][cin] and to wb in the order of the transposed convolution [27][cin][cout];
 * otherwise (biases) nothing else is written.
 */
int sg_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps, int t,
            void* wf, void* wb, int cin, int cout, void* stream);

#ifdef __cplusplus
}
#endif
#endif
