/*
 * hom_net.h -- C ABI of the learned warm start: a small BF16 3-D
 * convolutional network that predicts the initial strain fluctuation of the
 * homogenization solve from the phase map phi and the macro strain.
 *
 * The paper has no learned component.  Its hook is the initial iterate: in
 * the non-linear Galerkin extension (section 2.1.1) the previous load step's
 * strain starts the next solve.  Here the network's prediction is passed to
 * hom_solve as `warm_start`; hom_solve projects it onto compatible fields and
 * the FP64 true residual of eq. (galres) decides convergence, so a poor
 * prediction costs iterations, never accuracy.
 *
 * Network: periodic 3x3x3 convolutions with ReLU, a 4-level U-Net (channel
 * widths 16, 32, 48, 64; 2x2x2 average pooling down, nearest-neighbour
 * upsampling and skip concatenation up), a head with 36 output channels
 * M[6c+J], and the prediction x0_c = sum_J M[6c+J] E_J (Mandel components),
 * linear in the macro strain like the cell problem itself.  Activations and
 * weights are BF16 on the tensor cores with FP32 accumulation; master
 * weights, gradients and Adam moments are FP32.
 *
 * Conventions: grids are n1 x n2 x n3, C order, n3 fastest; each n_p a
 * multiple of 8 (three poolings).  Fields are FP32 device pointers laid out
 * [batch or case][6][voxels] in TENSOR components (e11, e22, e33, e23, e13,
 * e12), the convention of hom_fields and hom_solve's warm_start.  Macro
 * strains are host arrays [batch][6] of tensor components.  Calls are
 * stream-ordered on the stream given at creation and return when the result
 * is on the device (the loss is copied to the host).  Errors: HOM_EINVAL for
 * bad arguments, HOM_EUNSUPPORTED_GRID, HOM_ENOMEM, HOM_ECUDA (codes of
 * hom.h); hom_net_last_error gives a message.
 *
 * Parameter order (get/set/gradients): layers e1a, e1b, e2a, e2b, e3a, e3b,
 * bna, bnb, d3a, d3b, d2a, d2b, d1a, d1b, head; each as W[27][c_out][c_in]
 * (tap t = 9(dz+1) + 3(dy+1) + (dx+1) reads the input at offset (dz, dy, dx))
 * followed by b[c_out].
 */
#ifndef HOM_NET_H
#define HOM_NET_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hom_net hom_net;   /* opaque, owned by the library */

/* Create a network with He-initialised weights from `seed` (the head scaled
 * by 0.1) and zero biases, on the current CUDA device.  stream: cudaStream_t
 * or NULL (a stream the network creates). */
int hom_net_create(hom_net **out, unsigned long long seed, void *stream);
void hom_net_destroy(hom_net *net);
const char *hom_net_last_error(void);

/* Number of FP32 parameters; copy them to / from a host array in the order
 * above.  Setting resets nothing else (Adam moments are kept). */
long long hom_net_param_count(const hom_net *net);
int hom_net_get_params(const hom_net *net, float *host);
int hom_net_set_params(hom_net *net, const float *host);

/* Save / load parameters (and the Adam state) to / from a file. */
int hom_net_save(const hom_net *net, const char *path);
int hom_net_load(hom_net *net, const char *path);

/* Prediction at the network's own resolution: phi [batch][V] FP32 device,
 * macro [batch][6] host, x0 [batch][6][V] FP32 device. */
int hom_net_forward(hom_net *net, int batch, const int grid[3], const float *phi, const double *macro, float *x0);

/* One training step: forward, mean squared error against `target`
 * ([batch][6][V] FP32 device, tensor components; the error is taken in
 * Mandel components), backward, Adam (beta 0.9 / 0.999, eps 1e-8) with
 * learning rate lr.  *loss (may be NULL) receives the loss before the step. */
int hom_net_train_step(hom_net *net, int batch, const int grid[3], const float *phi, const double *macro,
                       const float *target, float lr, double *loss);

/* Weight of the squared error per voxel: vw + (1 - vw) phi, i.e. 1 in the
 * solid and vw in empty space (default vw = 1: plain mean squared error).
 * Strains in empty voxels are not unique (only the zero-start MINRES iterate
 * defines them), so vw < 1 lets the network spend its capacity on the solid. */
int hom_net_set_void_weight(hom_net *net, double void_weight);

/* Loss and parameter gradients (host array in parameter order) without a
 * step: for checks against an independent implementation. */
int hom_net_gradients(hom_net *net, int batch, const int grid[3], const float *phi, const double *macro,
                      const float *target, float *grads, double *loss);

/* Warm start for a solve on a grid `grid` (each n_p = s m_p, m_p a multiple
 * of 8): phi [V] FP32 device is averaged over s^3 blocks, the network runs on
 * the m grid, and its 36 head channels are interpolated back trilinearly
 * (periodic) before the contraction with each of the ncase macro strains
 * (host [ncase][6]).  x0 [ncase][6][V] FP32 device.  s = 1 runs the network
 * on the full grid. */
int hom_net_warm_start(hom_net *net, const int grid[3], int s, const float *phi, int ncase, const double *macro,
                       float *x0);

/* Number of this library's kernels the network has launched. */
long long hom_net_kernel_launches(const hom_net *net);

/* Step-level entry points (for parity tests and timing), device pointers,
 * BF16 values passed as their 16-bit patterns:
 *   out[v][co] = act(bias[co] + sum_t sum_ci W[t][co][ci] in[v + d_t][ci])
 * with in = [src0 (c0s channels), src1 (c1s channels at half resolution,
 * nearest-neighbour upsampled)], periodic wrap; c0s, c1s, cout multiples of
 * 16; bias may be NULL; out_f32 selects an FP32 output. */
int hom_net_conv3d(int batch, const int grid[3], const unsigned short *src0, int c0s, const unsigned short *src1,
                   int c1s, const unsigned short *W, const float *bias, int relu, int cout, void *out, int out_f32,
                   void *stream);
/* dW[t][co][ci] = sum_v G[v][co] in[v + d_t][ci] (FP32 [27][cout][c0s+c1s]),
 * cout <= 64. */
int hom_net_conv3d_wgrad(int batch, const int grid[3], const unsigned short *G, int cout, const unsigned short *src0,
                         int c0s, const unsigned short *src1, int c1s, float *dW, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HOM_NET_H */
