// hom_internal.h -- shared declarations of the library's kernels and context.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hom_fft.cuh"

namespace hom {

// Scalars of one MINRES solve, resident in device memory.  Written only by
// the single-thread scalar kernels; read by the field kernels.  FP64 always.
struct MinresState {
    double beta1;      // ||b||
    double beta;       // beta_k: coefficient of v_{k-1} in the next Lanczos step
    double alpha;      // alpha_k
    double c, s;       // previous Givens rotation
    double dbar;       // delta-bar_{k+1}
    double eps;        // epsilon_{k+1}
    double phibar;     // phi-bar_k
    double tol;
    // coefficients of the w / x / v update of the current iteration
    double u_delta, u_eps, u_inv_gamma, u_tau, u_inv_beta;
    double est;        // phibar_k / beta_1
    int k;             // iterations done
    int max_it;
    int done;          // no further operator / Lanczos work
    int done_update;   // the last w/x update has been applied
    int status;        // 0 ok, 1 max_it, -5 NaN
    int pad;
};

// Kernel-side description of the three axis transforms and the frequency
// tables of one context (one precision).
struct Geometry {
    int n1, n2, n3, h;      // h = n3/2 + 1
    long long V, S;         // voxels, half-spectrum points per component
    AxisPlan ax[3];
    const void *D[3];       // per axis: difference symbol (complex, length n_p)
    const void *M[3];       // per axis: averaging factor (complex, length n_p)
    // launch shapes
    int rows3, tile2, tile1;
    size_t smem3, smem2, smem1;
};

enum X3FwdMode { X3F_RAW = 0, X3F_MATERIAL = 1, X3F_MACRO = 2 };
enum X3InvMode { X3I_STORE = 0, X3I_STORE_NORM2 = 1, X3I_STORE_DOT = 2 };
enum X1Flags { X1_FWD = 1, X1_GAMMA = 2, X1_INV = 4 };

constexpr int kEwBlocks = 152 * 8;   // grid of the element-wise Krylov kernels
constexpr int kEwThreads = 256;

template <typename R> struct Launch {
    static void x3_fwd(const Geometry &g, cudaStream_t st, int mode, const R *in, const R *phi,
                       double lam, double mu, const double *macro_mandel, cpx<R> *spec,
                       const MinresState *state);
    static void x2(const Geometry &g, cudaStream_t st, int inverse, cpx<R> *spec,
                   const MinresState *state);
    static void x1(const Geometry &g, cudaStream_t st, int flags, cpx<R> *spec,
                   const MinresState *state);
    static void x3_inv(const Geometry &g, cudaStream_t st, int mode, const cpx<R> *spec, R *out,
                       double scale, const R *dotv, double *partials, const MinresState *state);
    // p -= alpha v + beta vprev ; partial ||p||^2
    static void lanczos(long long n, cudaStream_t st, R *p, const R *v, const R *vprev,
                        const MinresState *state, double *partials);
    // w2 <- (v - delta w1 - eps w2)/gamma ; x += tau w2 ; p <- p / beta_next
    static void update(long long n, cudaStream_t st, R *p, const R *v, const R *w1, R *w2, R *x,
                       MinresState *state);
    // y = a*x (+ b*y if accumulate)
    static void axpby(long long n, cudaStream_t st, double a, const R *x, double b, R *y);
    static void norm2(long long n, cudaStream_t st, const R *x, double *partials);
    static void mean_stress(long long V, cudaStream_t st, const R *x, const R *phi, double lam,
                            double mu, const double *macro_mandel, double *partials);
    static void fields(long long V, cudaStream_t st, const R *x, const R *phi, double lam,
                       double mu, double Escale, const double *macro_mandel, R *strain, R *stress);
    static void table_init(const Geometry &g);
};

// Conversions between precisions: out[i] = (To) in[i] (+ out[i] if acc)
void convert_f2d(long long n, cudaStream_t st, const float *in, double *out, int acc);
void convert_d2f(long long n, cudaStream_t st, const double *in, float *out);
// r = b - ax (double), partial ||r||^2
void residual64(long long n, cudaStream_t st, const double *b, const double *ax, double *r,
                double *partials);
// tensor <-> Mandel on a 6 x V field (scale the shear components)
template <typename R> void mandel_scale(long long V, cudaStream_t st, R *f, double s);
// phi conversion from the user's input kind into R precision; nonzero flag
// written to *bad on NaN or values outside [0,1]
template <typename R> void phi_convert(long long V, cudaStream_t st, const void *in, int kind,
                                       R *out, int *bad);

// single-thread scalar kernels
void scalar_start(cudaStream_t st, MinresState *s, const double *partials, int np, double tol,
                  int max_it);
void scalar_alpha(cudaStream_t st, MinresState *s, const double *partials, int np);
void scalar_givens(cudaStream_t st, MinresState *s, const double *partials, int np);
void reduce_to(cudaStream_t st, const double *partials, int np, double *out);

}  // namespace hom
