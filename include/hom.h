/*
 * hom.h -- C ABI of the GB300 Galerkin-FFT homogenization library (libhom.so).
 *
 * The library solves the periodic cell problem of section 2.1 of Lucarini et
 * al., "Adaptation and validation of FFT methods for homogenization of
 * lattice based materials" (arXiv 2110.00733):
 *
 *   find the strain fluctuation e~ with  A(e~) = b,                eq. (gallin)
 *   A(e) = F^-1{ G(xi) : F{ C(x) : e } },                          eq. (linearOp)
 *   b    = -F^-1{ G(xi) : F{ C(x) : E_bar } }   (strain control),
 *
 * with C(x) = phi(x) C_m (isotropic E, nu scaled by the per-voxel solid
 * fraction phi, Voigt rule of section 3.3; phi = 0 is empty space), G the
 * compatible-strain projector of eq. (galop) built from the continuous
 * frequencies of eq. (freq) or the rotated finite-difference frequencies of
 * eq. (freqrot), solved by MINRES (section 2.1) to the relative residual of
 * eq. (galres).  The effective stiffness is the volume average of the stress
 * over the six unit macro strains (section 4.3).
 *
 * Conventions shared by every entry point
 *   - grid n1 x n2 x n3, C order (index n3 fastest), unit cell edges;
 *     each n_p in [2, 512] and of the form 2^a 3^b 5^c.
 *   - V = n1*n2*n3.  A "field" is 6 x V values, component-major
 *     (field[c*V + voxel]).  Entry points marked MANDEL use Mandel components
 *     (e11, e22, e33, sqrt2 e23, sqrt2 e13, sqrt2 e12); the others use tensor
 *     components (e11, e22, e33, e23, e13, e12).
 *   - A "spectrum" is the half spectrum of 6 real components:
 *     n1 x n2 x (n3/2+1) x 6 complex values (re, im interleaved), the six
 *     components of one frequency adjacent, unnormalised forward DFT with
 *     kernel exp(-2 pi i k n / N).
 *   - MINRES (section 2.1) runs on the DFT of the strain fluctuation: on
 *     A^ = G F C F^-1 G with the Parseval inner product, which on compatible
 *     fields is the same iteration as MINRES on A of eq. (linearOp); applying
 *     G to the input too keeps rounding from driving the iterate out of the
 *     compatible subspace.
 *   - Field and spectrum buffers are float (HOM_PREC_FP32_FIELDS) or double
 *     (HOM_PREC_FP64) as chosen at create time.  They are host pointers unless
 *     hom_options.device_ptrs is set, in which case they are device pointers
 *     on the context's device, used on the context's stream.
 *   - The caller owns every buffer it passes; the library copies what it
 *     keeps.  The context owns its device workspace (allocated by hom_create,
 *     freed by hom_destroy).
 *   - Stiffness, stress and the outputs of hom_apply / hom_rhs: hom_apply and
 *     hom_rhs use C_m / E (units of E); hom_solve_info.sigma_mean,
 *     hom_effective_stiffness and hom_fields' stress are in the units of E.
 *   - Entry points return after their device work has completed (except
 *     hom_apply_noalloc, which only enqueues it).
 *   - Return value: HOM_OK (0), a positive warning (result valid), or a
 *     negative error, in which case no output buffer has been written;
 *     hom_last_error() then describes the failure.
 *   - A context is not thread-safe: one host thread at a time.
 *   - HOM_PDL=1 in the environment at hom_create makes the kernels of a
 *     MINRES sweep's graph use programmatic dependent launch (each starts
 *     while its predecessor drains and waits for it before touching
 *     memory); off by default, where it measured slower.
 *   - HOM_X2_STAGES=2..4 in the environment at hom_create sets the depth of
 *     the TMA ring of the FP32 n2 pass (default 3 at n2 >= 256, else 2).
 *   - HOM_X1_L2PF=0 in the environment at hom_create turns off the L2
 *     prefetch of each tile's Lanczos blocks in the fused FP32 n1 pass.
 *   - HOM_FOLD_ALPHA=1 in the environment at the first solve folds the
 *     MINRES alpha reduction into the register n3 pass (one launch fewer
 *     per step; off by default).
 */
#ifndef HOM_H
#define HOM_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HOM_OK = 0,
    HOM_NOT_CONVERGED = 1,          /* max_it reached; best iterate returned */
    HOM_EINVAL = -1,                /* bad argument */
    HOM_EUNSUPPORTED_GRID = -2,     /* a grid size outside [2,512] or not 2^a3^b5^c */
    HOM_ENOMEM = -3,                /* device allocation failed */
    HOM_ECUDA = -4,                 /* CUDA runtime error */
    HOM_ENAN = -5,                  /* NaN/Inf met in the input or a Krylov scalar */
    HOM_ETIMEOUT = -6               /* a bounded device wait (TMA completion) gave up */
};

enum { HOM_INPUT_PHASE_U8 = 0,      /* uint8 phase id: 0 empty, nonzero solid */
       HOM_INPUT_FRACTION_F32 = 1,  /* float solid fraction phi in [0,1] */
       HOM_INPUT_FRACTION_F64 = 2 };/* double solid fraction phi in [0,1] */
enum { HOM_SMOOTH_NONE = 0 };       /* phi used as given (plain, Voigt-smoothed, or the
                                       phase-field map of hom_pfs) */
enum { HOM_DERIV_CONTINUOUS = 0,    /* xi_p = i q_p N_p, eq. (freq) */
       HOM_DERIV_ROTATED = 1 };     /* rotated forward difference, eq. (freqrot) */
enum { HOM_SOLVER_GALERKIN_MINRES = 0,   /* section 2.1 */
       HOM_SOLVER_MODBFFT_CG = 1,        /* section 2.2: penalised displacement FFT, PCG */
       HOM_SOLVER_GALERKIN_CG = 2 };     /* section 2.1: CG on the Galerkin system, the
                                            solver the paper names for cells without void
                                            and reports failing with empty voxels; kept for
                                            that comparison (same operator, refinement
                                            sweeps and outputs as MINRES) */
enum { HOM_PREC_FP32_FIELDS = 0,    /* FP32 fields and FFTs, FP64 Krylov scalars */
       HOM_PREC_FP64 = 1 };         /* FP64 everywhere */

typedef struct hom_ctx hom_ctx;     /* opaque, owned by the library */

typedef struct {
    int solver;         /* HOM_SOLVER_GALERKIN_MINRES */
    int precision;      /* HOM_PREC_FP32_FIELDS (default) or HOM_PREC_FP64 */
    int device_ptrs;    /* nonzero: buffer arguments are device pointers */
    void *stream;       /* cudaStream_t to run on; NULL: a stream the context creates */
    int device;         /* CUDA device ordinal; -1: the current device */
    int refine;         /* FP32 fields: max FP64 iterative-refinement sweeps (default 3) */
    int rows3;          /* launch shape: n3-pass rows per CTA (0 = automatic, <= 64) */
    int tile2;          /* launch shape: n2-pass columns per CTA (0 = automatic; power of 2, <= 32) */
    int tile1;          /* launch shape: n1-pass columns per CTA (0 = automatic, <= 16) */
    int staging;        /* 0: persistent TMA-staged n1/n2 passes where supported
                           (FP32, n1 and n2 in {64, 96, 128, 160, 256, 512});
                           1: plain loads */
    double alpha;       /* MoDBFFT penalty alpha / E (0: 1e-4, section 4.2) */
    int autotune;       /* nonzero (and no explicit rows3/tile2/tile1): launch
                           shapes from hom_autotune for this grid and precision */
    int host_loop;      /* nonzero: the host replays the captured loop body
                           (six iterations per launch, a state read every
                           four launches) instead of one device-side WHILE
                           graph per sweep; the same kernels, for tools that
                           cannot see kernels inside conditional graphs */
    double sweep_floor; /* FP32 fields: smallest relative residual reduction one
                           refinement sweep is asked for (0: 1e-6 for MINRES,
                           5e-7 for its first sweep from a zero start; under
                           stress control 1e-4 for the first sweep and 1e-2
                           for later ones; 1e-3 for PCG); a sweep aims at
                           half the remaining
                           tolerance, and the FP64 true residual is recomputed
                           after every sweep */
} hom_options;

typedef struct {
    int iterations;        /* MINRES iterations (summed over refinement sweeps) */
    int status;            /* HOM_OK, HOM_NOT_CONVERGED or a negative error */
    int sweeps;            /* refinement sweeps taken (1 = none) */
    int reserved;
    double est_residual;   /* MINRES estimate phibar_k / beta_1 at exit */
    double true_residual;  /* ||A(e~) - b|| / ||b|| evaluated in FP64, eq. (galres) */
    double sigma_mean[6];  /* volume-averaged stress, tensor components, same units as E */
    double time_ms;        /* device time of this case */
    double eps_mean[6];    /* volume-averaged strain, tensor components: the macro
                              strain, with the solved mean of the stress-controlled
                              components of hom_solve_mixed */
} hom_solve_info;

/* Fill *opt with the defaults. */
void hom_default_options(hom_options *opt);

/* Create a context for one cell.
 *   grid[3]     n1, n2, n3 (see conventions).
 *   phase       V values of the kind given by input_kind, C order; host
 *               pointer, or device pointer if opt->device_ptrs.  Copied.
 *   E, nu       isotropic lattice material (section 4.1), E > 0, -1 < nu < 0.5.
 *   smoothing   HOM_SMOOTH_NONE.
 *   derivative  HOM_DERIV_CONTINUOUS or HOM_DERIV_ROTATED.
 *   opt         NULL for defaults.
 * Errors: HOM_EINVAL (bad pointer, E, nu, enum, phi outside [0,1] or NaN),
 * HOM_EUNSUPPORTED_GRID, HOM_ENOMEM, HOM_ECUDA. */
int hom_create(hom_ctx **out, const int grid[3], const void *phase, int input_kind,
               double E, double nu, int smoothing, int derivative,
               const hom_options *opt);

/* Solve eq. (gallin) for ncase macro strains (strain control) -- or, for a
 * context created with HOM_SOLVER_MODBFFT_CG, the MoDBFFT system of
 * eqs. (modbfftf)/(modbfftfop) by preconditioned CG (section 2.2), with
 * est_residual / true_residual the ratio of eq. (modbfftresres).
 *   macro_strain  ncase x 6 tensor components, host memory.
 *   tol           relative residual of eq. (galres), e.g. 1e-6.
 *   max_it        MINRES iteration cap per case (per refinement sweep; the
 *                 MoDBFFT sweeps share it).
 *   warm_start    NULL (zero start) or ncase x 6 x V fluctuation fields, tensor
 *                 components, host or device per device_ptrs; it is projected
 *                 onto compatible fields before use (with FP32 fields the
 *                 projection and the first residual use the FP32 operator; a
 *                 start within 1e-3 of b gets the FP64 residual instead).
 *   info          NULL or ncase records.
 * Returns HOM_OK if every case met tol, HOM_NOT_CONVERGED if one hit max_it,
 * or a negative error.  The solutions stay in the context for
 * hom_fields / hom_effective_stiffness until the next hom_solve.
 * A right-hand side that vanishes up to round-off (e.g. a homogeneous cell)
 * gives the zero fluctuation with 0 iterations.
 * Precision: with HOM_PREC_FP32_FIELDS the fields and transforms are FP32;
 * the Krylov scalars, the right-hand side, the true residual after every
 * refinement sweep and the mean stress (by Parseval from the FP64 DFT of phi)
 * are FP64.  Each MINRES sweep runs on the device as one graph launch.
 * Not thread-safe for one context; distinct contexts may be used from
 * distinct threads (see hom_solve_batch). */
int hom_solve(hom_ctx *ctx, const double *macro_strain, int ncase, double tol,
              int max_it, const void *warm_start, hom_solve_info *info);

/* Phase-field smoothening (section 3.2): the phase map of eq. (phase), solved
 * in Fourier space by eq. (phase3), phi^(xi) = omega^(xi) / (1 + (ell^2/eps)
 * |xi|^2) with the continuous frequencies of eq. (freq), on a fine grid, then
 * averaged over ratio^3 blocks onto the simulation grid fine / ratio, values
 * below threshold set to 0 (the paper: ell = half a coarse voxel, eps = 1,
 * threshold 0.05, ratio 2..20).
 *   fine         fine grid, each size a multiple of ratio and supported by
 *                hom_create.
 *   omega        the indicator (or any phase map in [0, 1]) on the fine grid,
 *                C order, of input_kind (HOM_INPUT_*); host memory, or device
 *                memory if device_ptrs is nonzero.
 *   ell          length in fine voxels (ratio / 2 for half a coarse voxel).
 *   phi_out      (fine/ratio)^3 doubles, C order, host or device per
 *                device_ptrs; pass it to hom_create as HOM_INPUT_FRACTION_F64.
 * Runs on a temporary FP64 context of the fine grid (about 100 bytes per fine
 * voxel of device memory while it runs).  Returns HOM_OK or a negative error;
 * hom_last_error(NULL) has the message.  The mean of phi_out equals the mean
 * of omega when threshold is 0 (the filter keeps xi = 0). */
int hom_pfs(const int fine[3], const void *omega, int input_kind, int ratio, double ell, double eps,
            double threshold, int device_ptrs, double *phi_out);

/* Galerkin-MINRES under mixed macroscopic control (section 2.1, eq. (galop)
 * and eq. (gallin)): the Mandel components whose bit is set in stress_mask
 * (bit 0..5 = 11, 22, 33, 23, 13, 12) are stress-controlled, the others
 * strain-controlled.  The projector at xi = 0 is the identity on the stress-
 * controlled components KL and zero on the strain-controlled kl, and the
 * right-hand side is b = -G : F{C : E_bar - S_bar}; the solution's mean then
 * carries the unknown mean strain of the KL components, reported in
 * info[].eps_mean and included in hom_fields.
 *   macro_strain  ncase x 6 tensor components: prescribed mean strain of the
 *                 kl components (entries of KL components ignored).
 *   macro_stress  ncase x 6 tensor components, same units as E: prescribed
 *                 mean stress of the KL components (kl entries ignored).
 *   stress_mask   0..63; 0 is pure strain control (as hom_solve); 63 with
 *                 macro_stress = s e1 (x) e1 is uniaxial stress, whose mean
 *                 strain gives E = s / e11 and nu = -e22 / e11 (section 4.3).
 * tol, max_it, warm_start and info as for hom_solve (warm_start must be NULL
 * unless stress_mask is 0).  Galerkin contexts only (HOM_EINVAL for MoDBFFT).
 * Returns as hom_solve. */
int hom_solve_mixed(hom_ctx *ctx, const double *macro_strain, const double *macro_stress, int stress_mask,
                    int ncase, double tol, int max_it, const void *warm_start, hom_solve_info *info);

/* Elastoplastic cells: the Newton extension of the Galerkin scheme (section
 * 2.1.1) for small-strain von Mises (J2) plasticity with linear isotropic
 * hardening, the lattice material of section 5 (hardening = 0 is perfect
 * plasticity).  A voxel's stress and consistent tangent are those of the
 * material (radial return, Simo & Hughes 1998, section 3.3) times phi.
 * Galerkin-MINRES contexts only (HOM_EINVAL for the other solvers).  Strains,
 * history, stresses and the Newton right-hand sides are FP64 in either
 * precision; with HOM_PREC_FP32_FIELDS the Newton systems are solved by FP32
 * MINRES sweeps with an FP32 copy of the tangent, refined (up to
 * hom_options.refine more sweeps) against the FP64 residual of the tangent
 * system, which decides whether a solve met tol_lin; with HOM_PREC_FP64 by
 * FP64 MINRES.
 *
 * hom_j2_begin allocates the history on the device (total and plastic
 * strain, hardening variable, tangent, Newton work fields: 584 bytes per
 * voxel with FP64 fields, about 540 with FP32) and zeroes it (virgin, unstrained cell); calling it again
 * resets the history.  yield_stress > 0 and hardening >= 0, same units as E. */
int hom_j2_begin(hom_ctx *ctx, double yield_stress, double hardening);

typedef struct {
    int status;            /* HOM_OK, or HOM_NOT_CONVERGED when max_newton ran out */
    int newton;            /* Newton iterations of the increment */
    int linear;            /* MINRES iterations over those Newton iterations (max_lin bounds
                              each Newton system, refinement sweeps included) */
    int backtracks;        /* step halvings of the line search over the increment */
    double r_newton;       /* ||d eps||_inf / ||eps^i - eps^t||_inf of the last step, eq. (galrnewton) */
    double residual;       /* ||b_i|| / ||b_0|| at exit (right-hand side of eq. (galnonlin)) */
    double sigma_mean[6];  /* mean stress at the end of the increment, tensor components, same units as E */
    double eps_mean[6];    /* mean total strain, tensor components */
    double time_ms;        /* device time of the increment */
} hom_j2_info;

/* One load increment t -> t + dt by an inexact damped Newton method.
 *   macro_strain  6 tensor components: the mean strain at t + dt of the
 *                 strain-controlled components (the first iterate adds the
 *                 change from the previous increment's macro_strain, zero
 *                 after hom_j2_begin, uniformly).
 *   macro_stress  6 tensor components, same units as E: the mean stress at t + dt
 *                 of the components set in stress_mask (bits as for
 *                 hom_solve_mixed).
 * Each Newton iteration solves eq. (galnonlin) with the tangent at the
 * current iterate by MINRES to ||A dE - b_i|| <= tol_lin ||b_0|| (eq. galrlin;
 * the relative tolerance a MINRES call is given is capped at 0.5), then
 * halves the step (at most 7 times) until ||b|| falls by the factor
 * 1 - 1e-4 t.  The increment is accepted when ||dE||_inf <= tol_newton
 * ||eps^i - eps^t||_inf (eq. galrnewton) after a step whose linear solve met
 * tol_lin; the plastic history then moves to t + dt.  When max_newton runs
 * out the last iterate is taken all the same and the status says so.
 * Returns HOM_OK, HOM_NOT_CONVERGED or a negative error, after which the
 * history is that of t (the increment is not applied). */
int hom_j2_increment(hom_ctx *ctx, const double macro_strain[6], const double macro_stress[6], int stress_mask,
                     double tol_lin, double tol_newton, int max_newton, int max_lin, hom_j2_info *info);

/* Total strain, plastic strain (each 6 x V tensor components, double) and
 * hardening variable (V doubles) of the history; host or device pointers
 * per device_ptrs; any may be NULL. */
int hom_j2_state(hom_ctx *ctx, double *strain, double *plastic_strain, double *alpha);

/* Frees the history (also done by hom_destroy). */
int hom_j2_end(hom_ctx *ctx);

/* 6x6 Voigt effective stiffness, row-major, sigma = C (e11,e22,e33,2e23,2e13,2e12),
 * same units as E, fitted to the mean stresses and mean strains of the last
 * hom_solve or hom_solve_mixed.  That solve must have had ncase >= 6 cases
 * whose mean strains span all six directions; otherwise HOM_EINVAL.  Section
 * 4.3 extracts E and nu from such averages. */
int hom_effective_stiffness(hom_ctx *ctx, double C[36]);

/* Total strain E_bar + e~ and stress C(x):(E_bar + e~) of case icase of the
 * last solve, each 6 x V tensor components (float or double per precision).
 * Either pointer may be NULL. */
int hom_fields(hom_ctx *ctx, int icase, void *strain, void *stress);

/* Step entry points (one pass of the hot path each; used by parity tests). */

/* out = A(eps), eq. (linearOp); eps and out are MANDEL fields. */
int hom_apply(hom_ctx *ctx, const void *eps, void *out);

/* out = b for one macro strain (6 tensor components, host), MANDEL field. */
int hom_rhs(hom_ctx *ctx, const double macro_strain[6], void *out);

/* Forward 3-D real-to-complex DFT of the 6 components of a field (no material,
 * no projection): field 6 x V  ->  spectrum (see conventions). */
int hom_fft_forward(hom_ctx *ctx, const void *field, void *spectrum);

/* Inverse of hom_fft_forward including the 1/V factor (complex-to-real; the
 * imaginary parts of the self-conjugate k3 = 0 and k3 = n3/2 planes are
 * dropped as a real transform does). */
int hom_fft_inverse(hom_ctx *ctx, const void *spectrum, void *field);

/* out = F^-1{ G : F{ in } }: the projection of eq. (galop) alone (no
 * material), MANDEL fields. */
int hom_project(hom_ctx *ctx, const void *in, void *out);

/* out = G F C F^-1 G in on spectra (see conventions): the operator of
 * eq. (linearOp) conjugated by the DFT, with the projector of eq. (galop) on
 * the input as well, as the MINRES iteration applies it (section 2.1).
 * Mandel components; units of E. */
int hom_apply_spectrum(hom_ctx *ctx, const void *in_spectrum, void *out_spectrum);

/* Average device time in milliseconds of each kernel of one MINRES iteration
 * of this context, each launched `reps` times back to back on the context's
 * stream between two CUDA events, on the workspace's current contents (an
 * instrument for roofline measurements; it changes no solver state that a
 * later hom_solve reads).  ms[0..5], the elastic MINRES step in launch
 * order: n2 inverse, n3 pass (C2R + material law with the strain-energy sums
 * of alpha + R2C), alpha reduction, n2 forward, fused n1 pass (forward +
 * projector, Lanczos step + norm, lagged w/x update, projector + inverse of
 * the next Lanczos vector), Givens step.  The fused n1 pass is launched a
 * multiple of 3 times (reps rounded up), cycling through the three steps of
 * its deferred x update (x is read and written on one of them), and ms[4]
 * is their mean.  Returns the number of entries written (<= nmax). */
int hom_time_kernels(hom_ctx *ctx, int reps, double *ms, int nmax);

/* Average device time in milliseconds of the kernels of the J2 Newton
 * extension (section 2.1.1) at the context's current iterate, each launched
 * `reps` times back to back on the context's stream between two CUDA events
 * (an instrument for roofline measurements; hom_j2_begin first; it changes no
 * state a later increment reads).  ms[0] radial return with the consistent
 * tangent at every voxel, ms[1] tangent application C_t : x at every voxel,
 * ms[2] and ms[3] the tangent operator's n3 passes (C2R to a real field,
 * R2C from one).  Returns the number of entries written (<= nmax). */
int hom_j2_time_kernels(hom_ctx *ctx, int reps, double *ms, int nmax);

/* A(eps) of hom_apply for a small cell, allocating no device memory.  The
 * paper has no counterpart: this is a calling convention for callers that
 * must not call cudaMalloc -- an application whose device memory belongs to
 * its own pool or is reserved up front (a framework's caching allocator, a
 * real-time or embedded system that forbids allocations after start-up), or
 * a latency-critical loop in which cudaMalloc, which may synchronise the
 * device, is not acceptable.  hom_create allocates its workspace, so those
 * callers use this entry point instead.
 *   grid[3]     n1, n2, n3, each in [2, 64] and 2^a 3^b 5^c, with
 *               n1 n2 n3 <= 32768 (for example 32^3); larger grids give
 *               HOM_EUNSUPPORTED_GRID.
 *   phi         device pointer, V floats in [0,1] (not checked here).
 *   E, nu       as hom_create; the operator uses C_m / E (units of E).
 *   derivative  HOM_DERIV_CONTINUOUS or HOM_DERIV_ROTATED.
 *   eps, out    device pointers, 6 x V floats, MANDEL fields; FP32.
 *   stream      cudaStream_t (NULL: the legacy default stream).  Unlike the
 *               other entry points, the call only enqueues its kernels on
 *               this stream and returns without waiting for them: the caller
 *               synchronises the stream (or orders its later work after it)
 *               before reading out.
 * The work spectrum and the FFT tables live in fixed file-scope device arrays
 * (about 1.6 MB, held on every GPU that loads the library until the process
 * exits).  The first call on a device looks up their device addresses
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the arrays and each call
 * rewrites what it reads: calls whose device work overlaps in time (on two
 * streams, or two host threads) race and must not be issued.  Errors:
 * HOM_EINVAL, HOM_EUNSUPPORTED_GRID, HOM_ECUDA (launch failures, or a CUDA
 * error already pending before the call, which is left pending), with
 * hom_last_error(NULL) describing them. */
int hom_apply_noalloc(const int grid[3], const float *phi, double E, double nu, int derivative,
                      const float *eps, float *out, void *stream);

/* MoDBFFT step entry points (contexts created with HOM_SOLVER_MODBFFT_CG).
 * A "displacement spectrum" is n1 x n2 x (n3/2+1) x 3 complex values: the
 * DFT of a real displacement fluctuation, with continuous frequencies
 * (eq. freq) whose Nyquist components are 0; frequencies with xi = 0 carry
 * no unknown.  Units of E. */

/* out = A^alpha(u), eq. (modbfftfop) with strain control. */
int hom_modb_apply(hom_ctx *ctx, const void *u_spectrum, void *out_spectrum);

/* out = b^alpha for one macro strain (6 tensor components), eq. (modbfftfrhs). */
int hom_modb_rhs(hom_ctx *ctx, const double macro_strain[6], void *out_spectrum);

/* out = [xi . Cbar . xi]^-1 in, eq. (precf) with Cbar = <phi> C_m (eq. avstiff). */
int hom_modb_precond(hom_ctx *ctx, const void *in_spectrum, void *out_spectrum);

/* Solve the same ncase macro strains on ncell cells at once (the cell studies
 * of section 4.3 scaled out).  ctxs[i] are independent contexts (own streams
 * and workspaces, any grid sizes).  When every context is a Galerkin-MINRES
 * context of one precision on the current device and ncase <= 8 cases fit in
 * device memory as one stacked batch per cell, each refinement sweep of all
 * cells is one graph launch: every cell's cases are stacked in its MINRES
 * kernels, the cells' steps are parallel branches of the graph's body, and
 * the body repeats on the device until every case has converged; the FP64
 * right-hand sides and true residuals run between sweeps.  Otherwise the
 * cells are solved one after another.  info: NULL or ncell x ncase records
 * (cell-major; time_ms is the whole batch's).  Returns the worst status over
 * the cells (negative errors first).  Each context then holds its own
 * solutions as after hom_solve. */
int hom_solve_batch(hom_ctx *const *ctxs, int ncell, const double *macro_strain, int ncase, double tol,
                    int max_it, hom_solve_info *info);

/* Launch-shape autotuner: for a grid and precision, time the kernels of one
 * MINRES iteration (scratch contexts, random phase map, CUDA events) for
 * candidate tiles of each FFT pass and write the fastest
 * (rows3, tile2, tile1) to shape[3].  Cached per process and, when the
 * environment variable HOM_TUNE_CACHE names a file, on disk.  Allocates and
 * frees scratch contexts. */
int hom_autotune(const int grid[3], int precision, int shape[3]);

/* Grid, precision and workspace size of a context. */
int hom_get_info(const hom_ctx *ctx, int grid[3], int *precision, long long *workspace_bytes);

/* Number of kernels the library has launched on this context so far. */
long long hom_kernel_launches(const hom_ctx *ctx);

void hom_destroy(hom_ctx *ctx);

/* Message of the last error on ctx (or of the last failed hom_create when ctx
 * is NULL).  Valid until the next call on the same context. */
const char *hom_last_error(const hom_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HOM_H */
