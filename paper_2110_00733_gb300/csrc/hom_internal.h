// hom_internal.h -- shared declarations of the library's kernels.
//
// Data layout in device memory
//   real field     : 6 x V, component-major (Mandel components), C order voxels
//   half spectrum  : n1 x n2 x h x 6 complex, h = n3/2 + 1, component fastest
//                    (the six components of one frequency are adjacent, which
//                    the projector and the n1 pass read together)
// The MINRES vectors live in the half-spectrum space: MINRES runs on
//   A^(v) = G F C F^-1 G v,
// the operator of eq. (linearOp) conjugated by the DFT, with the projector
// applied on the input as well as on the output, under the Parseval inner
// product <a,b> = sum_k w(k3) Re(conj(a_k) b_k) with w = 1 on the self-
// conjugate planes k3 = 0 and k3 = n3/2 (even n3) and 2 elsewhere.  On
// compatible fields this is the same iteration as MINRES on A(e) in real space.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hom_fft.cuh"
#include "hom_tma.cuh"

namespace hom {

// Scalars of one MINRES solve, resident in device memory.  Written only by
// the single-CTA scalar kernels; read by the field kernels.  FP64 always.
struct MinresState {
    int done;          // no further operator / Krylov work (first field: the
                       // pass kernels read it through any solver's state)
    int done_update;   // set with done on a NaN: keep the last finite iterate (no flush)
    int k;             // iterations done
    int max_it;
    int status;        // 0 ok, 1 max_it, -5 NaN
    int pad;
    double beta1;      // ||b||
    double beta;       // beta_k = ||u_k||: the stored Lanczos vector u_k = beta_k v_k
    double beta_prev;  // beta_{k-1} (0 before the second step: no v_0 term)
    double alpha;      // alpha_k
    double c, s;       // previous Givens rotation
    double dbar;       // delta-bar_{k+1}
    double eps;        // epsilon_{k+1}
    double phibar;     // phi-bar_k
    double tol;
    // coefficients of the w / x update of the last finished iteration k,
    // applied one iteration later: w_k = (u_k u_inv_beta - u_delta w_{k-1}
    // - u_eps w_{k-2}) u_inv_gamma, x += u_tau w_k
    double u_delta, u_eps, u_inv_gamma, u_tau, u_inv_beta;
    // tau_{k-1}, tau_{k-2}: the fused MINRES step adds tau_j w_j to x for
    // three j at once, every third iteration (x is read and written a third
    // as often)
    double u_tau1, u_tau2;
    double est;        // phibar_k / beta_1
    int bodies;        // captured bodies run by the device-side loop
    int max_bodies;    // hard cap of that loop
};

// alpha_k = <v_k, A v_k> = <u_k, A u_k> / beta_k^2 from sum = <u_k, A u_k> / scale
__device__ __forceinline__ void alpha_step(MinresState *st, double sum, double scale) {
    if (st->done) return;
    st->alpha = scale * sum / (st->beta * st->beta);
}

// MINRES step k (one thread): apply the previous Givens rotation to the new
// column of the Lanczos tridiagonal, form the next rotation and the
// coefficients of the w_k / x_k update (applied by the next step's kernel,
// or by the flush after the loop); stop when phibar_k / beta_1 <= tol,
// beta_{k+1} = 0, or k reaches max_it.  bn2 = ||u_{k+1}||^2.
__device__ __forceinline__ void givens_step(MinresState *st, double bn2) {
    if (st->done) return;
    const double beta_next = sqrt(bn2 > 0 ? bn2 : 0.0);
    const double alpha = st->alpha, c = st->c, s = st->s, dbar = st->dbar;
    const double delta = c * dbar + s * alpha;
    const double gbar = s * dbar - c * alpha;
    const double eps_next = s * beta_next;
    const double dbar_next = -c * beta_next;
    double gamma = hypot(gbar, beta_next);
    if (gamma == 0.0) gamma = 1e-300;
    const double cn = gbar / gamma, sn = beta_next / gamma;
    const double tau = cn * st->phibar;
    const double phibar = sn * st->phibar;
    st->u_delta = delta;
    st->u_eps = st->eps;            // epsilon_k multiplies w_{k-2}
    st->u_inv_gamma = 1.0 / gamma;
    st->u_tau2 = st->u_tau1;
    st->u_tau1 = st->u_tau;
    st->u_tau = tau;
    st->u_inv_beta = 1.0 / st->beta;   // v_k = u_k / beta_k in the lagged update
    st->c = cn;
    st->s = sn;
    st->dbar = dbar_next;
    st->eps = eps_next;
    st->phibar = phibar;
    st->beta_prev = st->beta;
    st->beta = beta_next;
    st->k += 1;
    st->est = phibar / st->beta1;
    if (!isfinite(alpha) || !isfinite(beta_next) || !isfinite(phibar)) {
        st->status = -5;
        st->done = 1;
        st->done_update = 1;        // keep the last finite iterate
        return;
    }
    if (st->est <= st->tol || beta_next == 0.0) {
        st->done = 1;               // the flush still applies this step's update
    } else if (st->k >= st->max_it) {
        st->status = 1;
        st->done = 1;
    }
}

// Scalars of one preconditioned CG solve (MoDBFFT, section 2.2); same
// leading flags as MinresState.
struct CgState {
    int done, done_update, k, max_it, status, pad;
    double rho;        // <r, M r>
    double rr0;        // ||r_0||^2
    double rr;         // ||r_k||^2
    double a, b;       // step length and direction update of this iteration
    double tol;
    double est;        // ||r_k|| / ||r_0||
};

// Kernel-side description of one cell for one precision.
struct Geometry {
    int n1, n2, n3, h;      // h = n3/2 + 1
    long long V, S;         // voxels, half-spectrum points per component
    AxisPlan ax[3];
    const void *D[3];       // per axis: difference symbol (complex, length n_p)
    const void *M[3];       // per axis: averaging factor (complex, length n_p)
    // launch shapes: rows per CTA of the n3 pass, columns per CTA of the n2
    // and n1 passes, threads per CTA, dynamic shared memory, and whether the
    // axis uses the compile-time register FFT (its length, or 0)
    int rows3, tile2, tile1;
    int threads3, threads2, threads1;
    size_t smem3, smem2, smem1;
    int fast[3];
    int nc;                 // complex components per frequency in the spectrum (6, or 10 for MoDBFFT)
    // load cases stacked along k1 in one launch of the MINRES kernels (work
    // spectrum nb x n1 x n2 x h x nc, Krylov vectors nb blocks of kvec, one
    // MinresState per case); 1 everywhere else
    int nb = 1;
    // nonzero: the MINRES passes launch with programmatic stream serialization
    // (set for the stacked graph's body; the kernels wait on their
    // predecessor with griddepcontrol before touching memory)
    int pdl = 0;
    int mask0;              // stress-controlled Mandel components (bit c): the projector keeps them at xi = 0
    // persistent TMA-staged n2 / n1 passes (FP32, register-FFT n in [64, 512]):
    // enabled flag, persistent grid sizes, shared memory, host-side cache of
    // tensor maps (never dereferenced on the device) and the device word a
    // pass sets when a bounded wait gives up
    int tma;
    // fused MINRES chain: complex elements of one Krylov vector stored in
    // n1-tile order (tiles of tile1 (k2,k3) columns, each tile a contiguous
    // n1 x 6 tile1 block laid out as the pass's shared-memory tile)
    long long kvec;
    // register-resident n3 pass (k_x3r: FP32, n3 in {64, 128, 256}) for
    // spectrum-to-spectrum applications
    int x3r;
    int grid2_tma, grid1_tma, grid1d_tma;
    int grid1l_tma;         // persistent grid of the fused MINRES n1 pass (0: plain-load form)
    size_t smem2_tma, smem1_tma, smem1d_tma;
    int grid3r = 0;         // persistent grid of the register n3 pass
    int x2_stages = 2;      // TMA ring stages of the persistent n2 pass
    int x1_l2pf = 1;        // fused n1 pass: L2 prefetch of each tile's u_k, u_{k-1} blocks
    size_t smem1l_tma = 0;  // fused MINRES n1 pass: work-tile stages + lagged-update ring
    int x1_lag_stages = 0;  // stages of that ring (kX1LagChunk bytes of each of 4 operands)
    void *tma_cache;
    int *err;
};

// register-resident n3 pass (k_x3r): supported lengths, rows per 128-thread
// CTA, and its shared memory (per row, the transpose slab of 3 lines x Q x
// (P + 1) complex values, N = P Q)
__host__ __device__ constexpr bool x3r_length(int n) { return n == 64 || n == 128 || n == 256; }
// register n3 pass: rows per warp (32 / lanes per row), and per warp the
// prefetch buffer of a row group (its rows' half spectra, then phi) and one
// transpose slab per row; four warps per CTA
__host__ __device__ constexpr int x3r_row_lanes(int n) { return n == 256 ? 16 : 8; }
__host__ __device__ constexpr int x3r_rows_per_warp(int n) { return 32 / x3r_row_lanes(n); }
__host__ __device__ constexpr size_t x3r_in_bytes(int n) {
    return (size_t)x3r_rows_per_warp(n) * (n / 2 + 1) * 6 * sizeof(float2);
}
// phi is prefetched with the rows except at n = 128, where its 2 KB per
// warp would leave room for two CTAs per SM instead of three (it is read
// from L2 there)
__host__ __device__ constexpr bool x3r_phi_prefetch(int n) { return n != 128; }
__host__ __device__ constexpr size_t x3r_phi_bytes(int n) {
    return x3r_phi_prefetch(n) ? (size_t)x3r_rows_per_warp(n) * n * sizeof(float) : 0;
}
__host__ __device__ constexpr size_t x3r_slab_elems(int n) {
    return (size_t)(n / x3r_row_lanes(n)) * (x3r_row_lanes(n) + 1);
}
__host__ __device__ constexpr size_t x3r_warp_bytes(int n) {
    return x3r_in_bytes(n) + x3r_phi_bytes(n) + (size_t)x3r_rows_per_warp(n) * x3r_slab_elems(n) * sizeof(float2);
}
constexpr int kX3rWarps = 4;
__host__ __device__ constexpr size_t x3r_smem(int n) { return kX3rWarps * x3r_warp_bytes(n); }

// A kernel launch, with programmatic stream serialization when pdl != 0.
template <typename... KArgs, typename... Args>
inline void launch_k(int pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args... args) {
    if (!pdl) {
        k<<<grid, block, smem, st>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

// tensor-map kinds of the TMA passes
enum TmaKind { TMA_X2 = 0, TMA_X1 = 1 };
// Host: the cached tensor map of `ptr` (a half spectrum of this geometry) for
// the given pass; nullptr if the driver entry point is unavailable.
const CUtensorMap *tma_map(const Geometry &g, const void *ptr, int kind, int elem_units);
void *tma_cache_new();
bool tma_available();
void tma_cache_free(void *cache);

// n3 pass (x3): input, middle and output stages
enum X3In { X3_IN_SPEC = 0, X3_IN_REAL = 1, X3_IN_MACRO = 2 };
enum X3Mid { X3_MID_NONE = 0, X3_MID_MATERIAL = 1,
             X3_MID_MODB = 2 };   // 10 components: tau = phi C_m eps (0-5), chi_v g (6-8), 0 (9)
enum X3Out { X3_OUT_SPEC = 0, X3_OUT_REAL = 1 };
// n1 pass (x1) flags
enum X1Flags { X1_FWD = 1, X1_GAMMA_IN = 2, X1_GAMMA_OUT = 4, X1_DOT = 8 };

constexpr int kEwBlocks = 152 * 8;   // grid of the element-wise Krylov kernels
constexpr int kNbMax = 8;            // load cases of one stacked MINRES batch
// threads of the persistent fused n1 pass: the transform group (the fast
// lengths' n1 tiles take 192 threads) and the lagged-update warps
constexpr int kX1Group = 192;
constexpr int kX1LagThreads = 64;
constexpr int kX1LagChunk = 4096;      // bytes of one operand per ring stage
constexpr int kX1LagMaxStages = 3;
constexpr int kX2MaxStages = 4;        // TMA ring of the persistent n2 pass
constexpr int kEwThreads = 256;

struct Mac6 { double v[6]; };

// The MINRES scalar steps folded into the pass that produces their partial
// sums: every CTA of a group counts itself on a counter after writing its
// partial, and the last one reduces the group's partials (fixed order) and
// applies the step to the FP64 state, then resets the counter for the next
// launch.  cnt == nullptr: no folding (a separate scalar kernel does the step).
// Counters: cnt[c] the n3 pass's CTAs of case c, cnt[kNbMax + c] the plain
// n1 pass's CTAs of case c, cnt[2 kNbMax] the persistent n1 pass's CTAs.
struct Fold {
    int *cnt;
    MinresState *st;     // the states (one per case)
    double scale;        // alpha: the partials sum to <u, A^ u> / scale
};
constexpr int kFoldCounters = 2 * kNbMax + 1;

template <typename R> struct Launch {
    // n3 pass: C2R (SPEC in) or real / macro input, optional material law
    // tau = phi C_m e, R2C (SPEC out) or real output; scale applied to the
    // real-space values (1/V for SPEC in is included automatically).
    // epart (6-component spectra only): per-CTA sums of the strain energy
    // e : C : e of the scaled real-space input (x3_grid(g) values).
    // fold: the alpha step folded into the pass (see Fold in hom_passes.cuh)
    // tsum (shared-memory pass with the material law only): per-CTA partial
    // sums over the voxels of the six stress components it forms,
    // tsum[c * x3_grid(g) + block]
    static void x3(const Geometry &g, cudaStream_t st, int in_mode, const void *in, int mid, double lam, double mu,
                   const double *macro_mandel, double scale, int out_mode, void *out, const R *phi,
                   const MinresState *state, double *epart = nullptr, Fold fold = Fold{}, double *tsum = nullptr);
    // n2 pass, in place on the half spectrum
    static void x2(const Geometry &g, cudaStream_t st, int inverse, cpx<R> *spec, const MinresState *state);
    // n1 pass: in -> out (may alias), optional projector before / after, and
    // the weighted partial sum <dotv, out> per CTA
    static void x1(const Geometry &g, cudaStream_t st, int flags, const cpx<R> *in, cpx<R> *out,
                   const cpx<R> *dotv, double *partials, const MinresState *state);
    // MoDBFFT: forward n1 pass of the 10-component spectrum in10 with the
    // contraction to 3 components fused (out3 = tau xi + g, eq. modbfftfop;
    // with dot3, the weighted <dot3, out3> partials).  Returns the number of
    // partials written, or 0 without launching where the fused form does not
    // apply (not the TMA-staged FP32 pass, or more partials than max_partials).
    static int x1_modb_contract(const Geometry &g, cudaStream_t st, const cpx<R> *in10, cpx<R> *out3,
                                const cpx<R> *dot3, double *partials, int max_partials, const MinresState *state);
    // MoDBFFT: the expansion of u3 to 10 components with the penalty alpha
    // (modb_expand) and the inverse n1 pass as one TMA-staged FP32 pass into
    // out10.  Returns false without launching where the fused form does not
    // apply (not the TMA-staged FP32 pass).
    static bool x1_modb_expand(const Geometry &g, cudaStream_t st, double alpha, const cpx<R> *u3, cpx<R> *out10,
                               const MinresState *state);
    // MINRES step k on unnormalised Lanczos vectors u_j = beta_j v_j, p = A u_k:
    //   um <- (p - alpha u_k - beta_k^2/beta_{k-1} um) / beta_k   (= u_{k+1}),
    //   weighted partial ||u_{k+1}||^2, and the lagged update of step k-1
    //   (k > 1): wb <- (um_old/beta_{k-1} - delta wa - eps wb) / gamma,
    //   x += tau wb.  wa = w_{k-2}, wb = w_{k-3} on entry.
    static void lanczos_update(const Geometry &g, cudaStream_t st, const cpx<R> *p, const cpx<R> *uk, cpx<R> *um,
                               const cpx<R> *wa, cpx<R> *wb, cpx<R> *x, const MinresState *state, double *partials);
    // fused n1 pass of a MINRES step (see k_x1_lanczos): spec holds the
    // forward n3 / n2 transforms of C e_k on entry and the inverse n1
    // transform of G u_{k+1} on exit; u_{k+1} is written to un (a third
    // buffer, neither uk nor um); wb, x as for lanczos_update;
    // x1_lanczos_grid(g) partials of ||u_{k+1}||^2
    // (fold: the Givens step folded into the pass)
    static void x1_lanczos(const Geometry &g, cudaStream_t st, cpx<R> *spec, const cpx<R> *uk, const cpx<R> *um,
                           cpx<R> *un, const cpx<R> *wa, cpx<R> *wb, cpx<R> *x, const MinresState *state,
                           double *partials, Fold fold = Fold{});
    static int x1_lanczos_grid(const Geometry &g);
    // standard half-spectrum order <-> n1-tile order of the fused chain's
    // Krylov vectors (the tile order's padding is left untouched)
    static void to_tiles(const Geometry &g, cudaStream_t st, const cpx<R> *in, cpx<R> *out);
    static void from_tiles(const Geometry &g, cudaStream_t st, const cpx<R> *in, cpx<R> *out);
    // the lagged update of the last step K after the loop; u_K sits in
    // buffer K mod 3 of (ua, ub, uc), or without uc (two Lanczos buffers) in
    // ub for odd K, in ua for even K; w_{K-1} in wd for even K, wc for odd K
    static void minres_flush(const Geometry &g, cudaStream_t st, const cpx<R> *ua, const cpx<R> *ub,
                             const cpx<R> *uc, cpx<R> *wc, cpx<R> *wd, cpx<R> *x, MinresState *state, long long n);
    // Parseval partials of <phi, (G x^)_c>, c = 0..5 (see k_phi_dot); returns
    // the number of blocks (partials[c * nb + block])
    static int phi_dot(const Geometry &g, cudaStream_t st, const cpx<R> *x, const cpx<R> *phihat, double *partials);
    // b^ = -G (phi^ tau) for the constant tensor tau = C_m : E_bar (Mandel)
    // sbar_v: V times the prescribed mean stress of the stress-controlled
    // components (Mandel, units of E), added at xi = 0; nullptr for none
    static void rhs_phihat(const Geometry &g, cudaStream_t st, const cpx<R> *phihat, const double *tau,
                           const double *sbar_v, cpx<R> *out);
    // out10 = (-phi^ tau, 0, 0, 0, 0): the MoDBFFT stress input of C : E_bar
    static void phihat_tau10(const Geometry &g, cudaStream_t st, const cpx<R> *phihat, const double *tau,
                             cpx<R> *out10);
    // y = a x + b y over n reals
    static void axpby(long long n, cudaStream_t st, double a, const R *x, double b, R *y);
    // weighted partial ||x||^2 of a spectral vector with nc components per frequency
    static void norm2w(const Geometry &g, cudaStream_t st, const cpx<R> *x, double *partials, int nc = 6);
    // MoDBFFT point-wise kernels (hom_modb.cuh); 3-component half spectra
    static void modb_expand(const Geometry &g, cudaStream_t st, double alpha, int with_penalty, const cpx<R> *u,
                            cpx<R> *out, int nc_out, const MinresState *state);
    static void modb_contract(const Geometry &g, cudaStream_t st, const cpx<R> *in10, cpx<R> *out3,
                              const cpx<R> *dotv, double *partials, const MinresState *state);
    static void modb_precond(const Geometry &g, cudaStream_t st, double lam_b, double mu_b, const cpx<R> *in,
                             cpx<R> *out);
    static void cg_xr(const Geometry &g, cudaStream_t st, double lam_b, double mu_b, cpx<R> *x, cpx<R> *r,
                      const cpx<R> *p, const cpx<R> *q, cpx<R> *z, const CgState *state, double *partials);
    static void cg_p(const Geometry &g, cudaStream_t st, cpx<R> *p, const cpx<R> *z, const CgState *state);
    static int ew_grid(long long n);
    static void table_init(const Geometry &g);
    static int x3_grid(const Geometry &g);
    static int x3_epart_grid(const Geometry &g);
    // resident CTAs x SMs of the persistent register n3 pass (0: it cannot run)
    static int x3r_grid(const Geometry &g);
    static int x1_grid(const Geometry &g);
    static int tma_grids(Geometry &g);
};

// FP64 helpers on spectral vectors (double2) and real fields
void spec_residual64(const Geometry &g, cudaStream_t st, const double2 *b, const double2 *ax, double2 *r,
                     double *partials, int nc = 6);             // r = b - ax, weighted ||r||^2
void spec_residual_mixed(const Geometry &g, cudaStream_t st, const double2 *b, const float2 *ax, double2 *r,
                         double *partials);                     // r = b - ax (ax FP32), weighted ||r||^2
void spec_d2f(long long ncplx, cudaStream_t st, const double2 *in, float2 *out);
void spec_f2d_acc(long long ncplx, cudaStream_t st, const float2 *in, double2 *out,
                  double a = 1.0);   // out += a in
void mean_stress64(long long V, cudaStream_t st, const double *x, const double *phi, double lam, double mu,
                   const double *macro_mandel, double *partials);   // partials[6][ew_grid(V)]
template <typename Ro>
void fields_from64(long long V, cudaStream_t st, const double *x, const double *phi, double lam, double mu,
                   double Escale, const double *macro_mandel, Ro *strain, Ro *stress);
void real_convert_f2d(long long n, cudaStream_t st, const float *in, double *out);
void real_convert_d2f(long long n, cudaStream_t st, const double *in, float *out);
void mandel_scale64(long long V, cudaStream_t st, double *f, double s);
template <typename R>
void phi_convert(long long V, cudaStream_t st, const void *in, int kind, R *out, int *bad);
int ew_blocks(long long n);
// sets the message hom_last_error(NULL) returns
void hom_set_error(const char *msg);

// single-CTA scalar kernels
void scalar_start(cudaStream_t st, MinresState *s, const double *partials, int np, double tol, int max_it,
                  int max_bodies = 0);
// end of a captured MINRES body inside a WHILE graph node: count the body and
// keep looping while one of the nb states is not done and the cap (of the
// first state) is not reached
void loop_cond(cudaStream_t st, cudaGraphConditionalHandle h, MinresState *s, int nb = 1);
// alpha_k from partials summing to <u_k, A^ u_k> / scale.  The scalar
// kernels of a stacked batch run one CTA per case c, on s[c] and the
// partials at c * np.
void scalar_alpha(cudaStream_t st, MinresState *s, const double *partials, int np, double scale = 1.0, int nb = 1,
                  int pdl = 0);
void scalar_givens(cudaStream_t st, MinresState *s, const double *partials, int np, int nb = 1);
// PCG scalars (MoDBFFT): start from <r0,z0>, ||r0||^2; step length; direction
void scalar_cg_start(cudaStream_t st, CgState *s, const double *partials, int np, double tol, int max_it);
void scalar_cg_alpha(cudaStream_t st, CgState *s, const double *partials, int np);
void scalar_cg_beta(cudaStream_t st, CgState *s, const double *partials, int np);
void reduce_to(cudaStream_t st, const double *partials, int np, double *out);

}  // namespace hom
