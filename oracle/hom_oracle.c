/*
 * hom_oracle.c -- plain FP64 CPU oracle of the Galerkin-FFT homogenization
 * method of Lucarini, Cobian, Vilchez-Morales, Segurado, "Adaptation and
 * validation of FFT methods for homogenization of lattice based materials"
 * (arXiv 2110.00733).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously correct reference
 * that the GPU library is checked against.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the GPU library.
 *
 * Conventions (each a reading of the paper, listed in the design notes):
 *   - grid n[0] x n[1] x n[2], C order (index n3 fastest), cell edges L_p = 1
 *     (the projector is invariant under a rescaling of each xi_p by the same
 *     factor, and all cells in the paper are cubic);
 *   - strain/stress fields are stored as 6 Mandel components per voxel,
 *     component-major: field[c*V + voxel], Mandel order
 *     (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12), so that the Euclidean inner
 *     product of two fields is the Frobenius product summed over voxels;
 *   - forward DFT uses exp(-2 pi i k n / N), no normalisation; inverse uses
 *     exp(+...) and the oracle divides by V itself.
 *
 * Nothing here is blocked, fused or reordered beyond the definitions: every
 * step is the paper's formula written out with plain loops.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* 1-D DFT: recursive mixed-radix Cooley-Tukey, direct DFT for prime lengths. */
/* Section 2.1: the transforms of eq. (gal) are discrete Fourier transforms   */
/* evaluated with an FFT; this is a textbook decimation-in-time FFT.          */
/* ------------------------------------------------------------------------ */

static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* out[k] = sum_j in[j*stride] * w[(j*k*(N/n)) mod N]   for k < n,
 * where w[t] = exp(sign * 2 pi i t / N) is a table of the N-th roots of unity
 * and n divides N.  scratch must hold n values. */
static void dft_rec(const cplx *in, int stride, cplx *out, int n,
                    const cplx *w, int N, cplx *scratch) {
    if (n == 1) { out[0] = in[0]; return; }
    int p = smallest_factor(n);
    int step = N / n;                  /* w[step*t] = exp(sign 2 pi i t / n) */
    if (p == n) {                      /* prime length: plain DFT */
        for (int k = 0; k < n; ++k) {
            cplx s = 0;
            for (int j = 0; j < n; ++j)
                s += in[(long)j * stride] * w[(long)step * ((long)j * k % n)];
            out[k] = s;
        }
        return;
    }
    int m = n / p;
    /* p sub-transforms of length m over the decimated sequences in[r + p j] */
    for (int r = 0; r < p; ++r)
        dft_rec(in + (long)r * stride, stride * p, out + r * m, m, w, N, scratch);
    /* combine: X[k + q m] = sum_r exp(sign 2 pi i r (k + q m)/n) Y_r[k] */
    for (int k = 0; k < m; ++k) {
        for (int q = 0; q < p; ++q) {
            cplx s = 0;
            int kk = k + q * m;
            for (int r = 0; r < p; ++r)
                s += out[r * m + k] * w[(long)step * ((long)r * kk % n)];
            scratch[kk] = s;
        }
    }
    memcpy(out, scratch, sizeof(cplx) * n);
}

static cplx *roots_of_unity(int n, int sign) {
    cplx *w = (cplx *)malloc(sizeof(cplx) * n);
    for (int t = 0; t < n; ++t) {
        double a = sign * 2.0 * PI * (double)t / (double)n;
        w[t] = cos(a) + I * sin(a);
    }
    return w;
}

/* In-place unnormalised 3-D DFT of a complex array of shape n[0] x n[1] x n[2]
 * (C order), sign = -1 forward, +1 inverse.  Applied axis by axis. */
void orc_fft3d(const int n[3], double *data_ri, int sign) {
    cplx *data = (cplx *)data_ri;
    long V = (long)n[0] * n[1] * n[2];
    long strides[3] = {(long)n[1] * n[2], n[2], 1};
    for (int ax = 0; ax < 3; ++ax) {
        int N = n[ax];
        if (N == 1) continue;
        cplx *w = roots_of_unity(N, sign);
        long nlines = V / N;
        long st = strides[ax];
#pragma omp parallel
        {
            cplx *line = (cplx *)malloc(sizeof(cplx) * N);
            cplx *res = (cplx *)malloc(sizeof(cplx) * N);
            cplx *scr = (cplx *)malloc(sizeof(cplx) * N);
#pragma omp for schedule(static)
            for (long l = 0; l < nlines; ++l) {
                /* line l: all indices except axis ax; base offset */
                long outer = l / st, inner = l % st;
                long base = outer * st * N + inner;
                for (int j = 0; j < N; ++j) line[j] = data[base + j * st];
                dft_rec(line, 1, res, N, w, N, scr);
                for (int j = 0; j < N; ++j) data[base + j * st] = res[j];
            }
            free(line); free(res); free(scr);
        }
        free(w);
    }
}

/* 1-D transform exposed for the FFT pins. */
void orc_fft1d(int N, double *data_ri, int sign) {
    int n[3] = {1, 1, N};
    orc_fft3d(n, data_ri, sign);
}

/* ------------------------------------------------------------------------ */
/* Frequencies, eq. (freq) and the rotated scheme, eq. (freqrot).             */
/* ------------------------------------------------------------------------ */

/* Signed frequency index of FFT index k on an axis of N points:
 * m = k for k < N/2, k - N otherwise (for even N, k = N/2 gives -N/2, the
 * paper's n - N/2 = -N/2 end of [-pi, pi]). */
static int signed_index(int k, int N) { return (2 * k < N) ? k : k - N; }

static int is_nyquist(int k, int N) { return (N % 2 == 0) && (2 * k == N); }

/* Frequency vector at FFT index (k1,k2,k3).
 * deriv = 0: continuous, xi_p = i q_p N_p / L_p                (eq. freq)
 * deriv = 1: rotated forward difference (Willot), eq. (freqrot):
 *     xi'_p = i 2 (N_p/L_p) tan(q_p/2) prod_r 1/2 (1 + e^{i q_r}),
 *   evaluated in the equivalent form
 *     xi'_p = N_p (e^{i q_p} - 1) prod_{r != p} 1/2 (1 + e^{i q_r}),
 *   since tan(q/2) (1 + e^{iq}) = -i (e^{iq} - 1); this form is finite at
 *   q = +-pi where the tan form is infinity times zero. */
void orc_frequency(const int n[3], const int k[3], int deriv, double xi_ri[6]) {
    cplx xi[3];
    double q[3];
    for (int p = 0; p < 3; ++p) q[p] = 2.0 * PI * signed_index(k[p], n[p]) / n[p];
    for (int p = 0; p < 3; ++p) {
        if (deriv == 0) {
            xi[p] = I * q[p] * n[p];
        } else {
            cplx v = n[p] * (cexp(I * q[p]) - 1.0);
            for (int r = 0; r < 3; ++r)
                if (r != p) v *= 0.5 * (1.0 + cexp(I * q[r]));
            xi[p] = v;
        }
    }
    for (int p = 0; p < 3; ++p) { xi_ri[2 * p] = creal(xi[p]); xi_ri[2 * p + 1] = cimag(xi[p]); }
}

/* ------------------------------------------------------------------------ */
/* Mandel <-> tensor                                                          */
/* ------------------------------------------------------------------------ */

static const int MI[6] = {0, 1, 2, 1, 0, 0};  /* row of Mandel component c */
static const int MJ[6] = {0, 1, 2, 2, 2, 1};  /* column                    */

static void mandel_to_tensor(const cplx m[6], cplx t[3][3]) {
    const double r2 = sqrt(2.0);
    for (int c = 0; c < 6; ++c) {
        cplx v = (c < 3) ? m[c] : m[c] / r2;
        t[MI[c]][MJ[c]] = v;
        t[MJ[c]][MI[c]] = v;
    }
}

static void tensor_to_mandel(cplx t[3][3], cplx m[6]) {
    const double r2 = sqrt(2.0);
    for (int c = 0; c < 6; ++c) {
        /* symmetric part of the (i,j) entry */
        cplx v = 0.5 * (t[MI[c]][MJ[c]] + t[MJ[c]][MI[c]]);
        m[c] = (c < 3) ? v : v * r2;
    }
}

/* ------------------------------------------------------------------------ */
/* Galerkin projector, eq. (galop).                                           */
/* ------------------------------------------------------------------------ */

/* Solve the 3x3 complex system K u = v by Gaussian elimination with partial
 * pivoting.  Returns 0 if K is singular. */
static int solve3(cplx K[3][3], cplx v[3], cplx u[3]) {
    cplx A[3][4];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) A[i][j] = K[i][j];
        A[i][3] = v[i];
    }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (cabs(A[r][c]) > cabs(A[piv][c])) piv = r;
        if (cabs(A[piv][c]) == 0.0) return 0;
        if (piv != c)
            for (int j = 0; j < 4; ++j) { cplx t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t; }
        for (int r = c + 1; r < 3; ++r) {
            cplx f = A[r][c] / A[c][c];
            for (int j = c; j < 4; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int i = 2; i >= 0; --i) {
        cplx s = A[i][3];
        for (int j = i + 1; j < 3; ++j) s -= A[i][j] * u[j];
        u[i] = s / A[i][i];
    }
    return 1;
}

/* Projection of one frequency's 3x3 symmetric tensor onto the compatible
 * strains {sym(u (x) xi)} at that frequency, orthogonal in the Hermitian
 * Frobenius product -- the reading of the fourth branch of eq. (galop),
 * [I^s_ijkl xi_j xi_l]^-1 xi_j xi_l, with the conjugate placed where a
 * complex (rotated) xi needs it:
 *   K_ik = I^s_ijkl conj(xi_j) xi_l = 1/2 (|xi|^2 delta_ik + xi_i conj(xi_k)),
 *   v_i  = tau_ij conj(xi_j),   K u = v,   (G tau)_ij = 1/2 (u_i xi_j + u_j xi_i).
 * Mandel components in and out (6 complex as re,im pairs).  xi = 0 gives 0,
 * the strain-controlled branch of eq. (galop). */
void orc_gamma_apply(const double xi_ri[6], const double tau_ri[12], double out_ri[12]) {
    cplx xi[3], tm[6], t[3][3], K[3][3], v[3], u[3], o[3][3], om[6];
    for (int p = 0; p < 3; ++p) xi[p] = xi_ri[2 * p] + I * xi_ri[2 * p + 1];
    for (int c = 0; c < 6; ++c) tm[c] = tau_ri[2 * c] + I * tau_ri[2 * c + 1];
    double n2 = 0;
    for (int p = 0; p < 3; ++p) n2 += creal(xi[p] * conj(xi[p]));
    if (n2 == 0.0) {
        for (int c = 0; c < 12; ++c) out_ri[c] = 0.0;
        return;
    }
    mandel_to_tensor(tm, t);
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
            K[i][k] = 0.5 * ((i == k ? n2 : 0.0) + xi[i] * conj(xi[k]));
    for (int i = 0; i < 3; ++i) {
        v[i] = 0;
        for (int j = 0; j < 3; ++j) v[i] += t[i][j] * conj(xi[j]);
    }
    if (!solve3(K, v, u)) {
        for (int c = 0; c < 12; ++c) out_ri[c] = 0.0;
        return;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) o[i][j] = 0.5 * (u[i] * xi[j] + u[j] * xi[i]);
    tensor_to_mandel(o, om);
    for (int c = 0; c < 6; ++c) { out_ri[2 * c] = creal(om[c]); out_ri[2 * c + 1] = cimag(om[c]); }
}

/* ------------------------------------------------------------------------ */
/* Material, operator A and right-hand side b (eqs. gallin, linearOp).        */
/* ------------------------------------------------------------------------ */

/* Isotropic stiffness C_m as a 6x6 Mandel matrix (lambda in the upper-left
 * 3x3 block, 2 mu on the diagonal).  The local stiffness is C(x) = phi(x) C_m
 * (Voigt rule, section 3.3). */
void orc_stiffness_mandel(double E, double nu, double Cm[36]) {
    double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double mu = E / (2.0 * (1.0 + nu));
    for (int i = 0; i < 36; ++i) Cm[i] = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Cm[i * 6 + j] = lam;
    for (int i = 0; i < 6; ++i) Cm[i * 6 + i] += 2.0 * mu;
}

typedef struct {
    int n[3];
    const double *phi;     /* V values in [0,1] */
    double Cm[36];         /* Mandel stiffness of the lattice material */
    int deriv;             /* 0 continuous, 1 rotated */
    int mask;              /* stress-controlled Mandel components KL (bit c) */
} orc_problem;

/* tau = C(x) : eps at every voxel (eps, tau: 6 x V Mandel). If eps_is_macro,
 * eps points to a single 6-vector used at every voxel. */
static void constitutive(const orc_problem *P, const double *eps, int eps_is_macro, cplx *tau) {
    long V = (long)P->n[0] * P->n[1] * P->n[2];
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        double e[6];
        for (int c = 0; c < 6; ++c) e[c] = eps_is_macro ? eps[c] : eps[(long)c * V + x];
        for (int i = 0; i < 6; ++i) {
            double s = 0;
            for (int j = 0; j < 6; ++j) s += P->Cm[i * 6 + j] * e[j];
            tau[(long)i * V + x] = P->phi[x] * s;
        }
    }
}

/* out = F^-1 { G(xi) : F{ tau } }  (real part), tau: 6 x V complex, overwritten. */
static void project_field(const orc_problem *P, cplx *tau, double *out) {
    long V = (long)P->n[0] * P->n[1] * P->n[2];
    for (int c = 0; c < 6; ++c) orc_fft3d(P->n, (double *)(tau + (long)c * V), -1);
    int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
#pragma omp parallel for schedule(static)
    for (long f = 0; f < V; ++f) {
        int k[3] = {(int)(f / ((long)n2 * n3)), (int)((f / n3) % n2), (int)(f % n3)};
        double o[12], t[12], xi[6];
        int nyq = is_nyquist(k[0], n1) || is_nyquist(k[1], n2) || is_nyquist(k[2], n3);
        if (k[0] == 0 && k[1] == 0 && k[2] == 0) {
            /* eq. (galop) at xi = 0: the symmetric identity on the stress-
             * controlled components KL, 0 on the strain-controlled kl */
            for (int c = 0; c < 6; ++c)
                if (!((P->mask >> c) & 1)) tau[(long)c * V + f] = 0;
            continue;
        }
        if (nyq) {
            /* eq. (galop): 0 at the Nyquist frequencies */
            for (int c = 0; c < 6; ++c) tau[(long)c * V + f] = 0;
            continue;
        }
        orc_frequency(P->n, k, P->deriv, xi);
        for (int c = 0; c < 6; ++c) {
            t[2 * c] = creal(tau[(long)c * V + f]);
            t[2 * c + 1] = cimag(tau[(long)c * V + f]);
        }
        orc_gamma_apply(xi, t, o);
        for (int c = 0; c < 6; ++c) tau[(long)c * V + f] = o[2 * c] + I * o[2 * c + 1];
    }
    for (int c = 0; c < 6; ++c) orc_fft3d(P->n, (double *)(tau + (long)c * V), +1);
    for (long i = 0; i < 6 * V; ++i) out[i] = creal(tau[i]) / (double)V;
}

/* A(eps) = F^-1{ G : F{ C : eps } },  eq. (linearOp), with the projector of
 * eq. (galop) for the stress-controlled components in mask (bit c = Mandel
 * component c; 0 = pure strain control). */
void orc_apply_mixed(const int n[3], const double *phi, double E, double nu, int deriv, int mask,
                     const double *eps, double *out) {
    orc_problem P;
    memcpy(P.n, n, sizeof P.n);
    P.phi = phi; P.deriv = deriv; P.mask = mask;
    orc_stiffness_mandel(E, nu, P.Cm);
    long V = (long)n[0] * n[1] * n[2];
    cplx *tau = (cplx *)malloc(sizeof(cplx) * 6 * V);
    constitutive(&P, eps, 0, tau);
    project_field(&P, tau, out);
    free(tau);
}

void orc_apply(const int n[3], const double *phi, double E, double nu, int deriv,
               const double *eps, double *out) {
    orc_apply_mixed(n, phi, E, nu, deriv, 0, eps, out);
}

/* b = -F^-1{ G : F{ C : Ebar - sigma_bar } }, eq. (gallin): Ebar carries the
 * prescribed strain components kl (its KL entries are ignored) and Sbar the
 * prescribed stress components KL (its kl entries are ignored), both Mandel. */
void orc_rhs_mixed(const int n[3], const double *phi, double E, double nu, int deriv, int mask,
                   const double Ebar[6], const double Sbar[6], double *out) {
    orc_problem P;
    memcpy(P.n, n, sizeof P.n);
    P.phi = phi; P.deriv = deriv; P.mask = mask;
    orc_stiffness_mandel(E, nu, P.Cm);
    long V = (long)n[0] * n[1] * n[2];
    double Ekl[6];
    for (int c = 0; c < 6; ++c) Ekl[c] = ((mask >> c) & 1) ? 0.0 : Ebar[c];
    cplx *tau = (cplx *)malloc(sizeof(cplx) * 6 * V);
    constitutive(&P, Ekl, 1, tau);
    for (int c = 0; c < 6; ++c)
        if ((mask >> c) & 1)
            for (long x = 0; x < V; ++x) tau[(long)c * V + x] -= Sbar[c];
    project_field(&P, tau, out);
    for (long i = 0; i < 6 * V; ++i) out[i] = -out[i];
    free(tau);
}

/* b for pure strain control (sigma_bar = 0). */
void orc_rhs(const int n[3], const double *phi, double E, double nu, int deriv,
             const double Ebar[6], double *out) {
    const double zero[6] = {0, 0, 0, 0, 0, 0};
    orc_rhs_mixed(n, phi, E, nu, deriv, 0, Ebar, zero, out);
}

/* Projection alone, F^-1 G F applied to a real 6 x V field (no material). */
void orc_project(const int n[3], int deriv, const double *in, double *out) {
    orc_problem P;
    memcpy(P.n, n, sizeof P.n);
    P.phi = NULL; P.deriv = deriv; P.mask = 0;
    long V = (long)n[0] * n[1] * n[2];
    cplx *tau = (cplx *)malloc(sizeof(cplx) * 6 * V);
    for (long i = 0; i < 6 * V; ++i) tau[i] = in[i];
    project_field(&P, tau, out);
    free(tau);
}

/* ------------------------------------------------------------------------ */
/* MINRES (Paige & Saunders 1975), the Krylov solver the paper uses for the   */
/* singular Galerkin system (section 2.1).  Written in the recurrence form of */
/* Choi, Paige & Saunders (2011); x0 = 0; stops when the estimated relative   */
/* residual phibar_k / beta_1 <= tol (eq. galres uses the true residual; the  */
/* caller confirms it).                                                       */
/* ------------------------------------------------------------------------ */

typedef void (*orc_matvec_fn)(void *ctx, const double *x, double *y);

static double dot(long n, const double *a, const double *b) {
    double s = 0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Returns the number of iterations; *rel_res receives phibar_k / beta_1.
 * hist (optional, max_it+1 entries) receives the estimated relative residual
 * after each iteration (hist[0] = 1). */
int orc_minres(long n, orc_matvec_fn A, void *ctx, const double *b, double *x,
               double tol, int max_it, double *rel_res, double *hist) {
    double *v_prev = (double *)calloc(n, sizeof(double));
    double *v = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *w1 = (double *)calloc(n, sizeof(double));  /* w_{k-1} */
    double *w2 = (double *)calloc(n, sizeof(double));  /* w_{k-2} */
    for (long i = 0; i < n; ++i) x[i] = 0.0;
    double beta1 = sqrt(dot(n, b, b));
    if (hist) hist[0] = 1.0;
    if (beta1 == 0.0) {
        *rel_res = 0.0;
        free(v_prev); free(v); free(p); free(w1); free(w2);
        return 0;
    }
    for (long i = 0; i < n; ++i) v[i] = b[i] / beta1;
    double beta = beta1;          /* beta_k (beta_1 for the first step) */
    double phibar = beta1, c = -1.0, s = 0.0, dbar = 0.0, eps = 0.0;
    int k = 0;
    *rel_res = 1.0;
    while (k < max_it) {
        ++k;
        A(ctx, v, p);                                         /* p = A v_k */
        double alpha = dot(n, v, p);
        double bk = (k == 1) ? 0.0 : beta;                    /* beta_k v_{k-1} term */
        for (long i = 0; i < n; ++i) p[i] -= alpha * v[i] + bk * v_prev[i];
        double beta_next = sqrt(dot(n, p, p));
        /* apply the previous rotation, then make the new one */
        double delta = c * dbar + s * alpha;
        double gbar = s * dbar - c * alpha;
        double eps_next = s * beta_next;
        double dbar_next = -c * beta_next;
        double gamma = hypot(gbar, beta_next);
        if (gamma == 0.0) gamma = 1e-300;
        c = gbar / gamma;
        s = beta_next / gamma;
        double tau = c * phibar;
        phibar = s * phibar;
        for (long i = 0; i < n; ++i) {
            double wn = (v[i] - delta * w1[i] - eps * w2[i]) / gamma;
            w2[i] = w1[i];
            w1[i] = wn;
            x[i] += tau * wn;
        }
        eps = eps_next;
        dbar = dbar_next;
        *rel_res = phibar / beta1;
        if (hist) hist[k] = *rel_res;
        if (*rel_res <= tol || beta_next == 0.0) break;
        for (long i = 0; i < n; ++i) {
            double vn = p[i] / beta_next;
            v_prev[i] = v[i];
            v[i] = vn;
        }
        beta = beta_next;
    }
    free(v_prev); free(v); free(p); free(w1); free(w2);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradients (Hestenes & Stiefel 1952), the solver the paper names */
/* for the Galerkin system of a cell without void (section 2.1) and shows to */
/* fail once empty voxels make the system singular.  x0 = 0; stops when the  */
/* recursively updated relative residual ||r_k|| / ||b|| <= tol.             */
/* ------------------------------------------------------------------------ */
int orc_cg(long n, orc_matvec_fn A, void *ctx, const double *b, double *x,
           double tol, int max_it, double *rel_res, double *hist) {
    double *r = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n);
    for (long i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; p[i] = b[i]; }
    double rho = dot(n, r, r);
    const double nb = sqrt(rho);
    if (hist) hist[0] = 1.0;
    *rel_res = 1.0;
    int k = 0;
    if (nb == 0.0) {
        *rel_res = 0.0;
        free(r); free(p); free(q);
        return 0;
    }
    while (k < max_it) {
        ++k;
        A(ctx, p, q);                                          /* q = A p_k */
        const double pq = dot(n, p, q);
        if (!(pq > 0.0)) break;                                /* not positive definite on p */
        const double alpha = rho / pq;
        for (long i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        const double rho_next = dot(n, r, r);
        *rel_res = sqrt(rho_next) / nb;
        if (hist) hist[k] = *rel_res;
        if (*rel_res <= tol) break;
        const double beta = rho_next / rho;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rho = rho_next;
    }
    free(r); free(p); free(q);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Full solve: b, MINRES, true residual (eq. galres), mean stress.           */
/* ------------------------------------------------------------------------ */

/* Relative size of ||b|| / ||C : Ebar|| below which the right-hand side is
 * FFT round-off and is taken as zero (the paper is silent on this case). */
#define ORC_RHS_ZERO 1e-12

typedef struct {
    const int *n;
    const double *phi;
    double E, nu;
    int deriv;
    int mask;
} apply_ctx;

static void apply_cb(void *ctx, const double *x, double *y) {
    apply_ctx *a = (apply_ctx *)ctx;
    orc_apply_mixed(a->n, a->phi, a->E, a->nu, a->deriv, a->mask, x, y);
}

/* Solves A(eps_tilde) = b of eq. (gallin) under mixed control: the Mandel
 * components in mask (bit c) are stress-controlled with prescribed mean
 * stress Sbar[c], the others strain-controlled with prescribed mean strain
 * Ebar[c] (mask = 0: pure strain control); method 0 MINRES, 1 CG.  Writes the solution eps_tilde
 * (6 x V Mandel; its mean carries the unknown mean strain of the stress-
 * controlled components), the volume-averaged stress <C : (Ebar_kl +
 * eps_tilde)> (sig_mean[6]) and strain Ebar_kl + <eps_tilde> (eps_mean[6],
 * may be NULL), all Mandel, and, in info[0..2], the iteration count, the
 * estimated and the true relative residual. */
int orc_solve_mixed(const int n[3], const double *phi, double E, double nu, int deriv, int mask,
                    const double Ebar[6], const double Sbar[6], int method, double tol, int max_it,
                    double *eps_tilde, double sig_mean[6], double eps_mean[6], double info[3], double *hist) {
    long V = (long)n[0] * n[1] * n[2];
    long N6 = 6 * V;
    double *b = (double *)malloc(sizeof(double) * N6);
    double *r = (double *)malloc(sizeof(double) * N6);
    double Ekl[6];
    for (int c = 0; c < 6; ++c) Ekl[c] = ((mask >> c) & 1) ? 0.0 : Ebar[c];
    orc_rhs_mixed(n, phi, E, nu, deriv, mask, Ebar, Sbar, b);
    apply_ctx ctx = {n, phi, E, nu, deriv, mask};
    double Cm[36];
    orc_stiffness_mandel(E, nu, Cm);
    /* scale of the right-hand side: ||C : Ebar_kl|| over the grid plus
     * ||sigma_bar_KL|| over the grid */
    double ce2 = 0.0, phi2 = 0.0, s2 = 0.0;
    for (int i = 0; i < 6; ++i) {
        double s = 0;
        for (int j = 0; j < 6; ++j) s += Cm[i * 6 + j] * Ekl[j];
        ce2 += s * s;
        if ((mask >> i) & 1) s2 += Sbar[i] * Sbar[i];
    }
    for (long x = 0; x < V; ++x) phi2 += phi[x] * phi[x];
    double ntau = sqrt(ce2 * phi2) + sqrt(s2 * (double)V);
    double est;
    int it;
    if (sqrt(dot(N6, b, b)) <= ORC_RHS_ZERO * ntau) {
        /* b vanishes up to FFT round-off (e.g. a homogeneous cell under strain
         * control, or a load the layout carries without any fluctuation):
         * eps_tilde = 0. */
        for (long i = 0; i < N6; ++i) { eps_tilde[i] = 0.0; b[i] = 0.0; }
        if (hist) hist[0] = 0.0;
        est = 0.0;
        it = 0;
    } else {
        it = (method == 1) ? orc_cg(N6, apply_cb, &ctx, b, eps_tilde, tol, max_it, &est, hist)
                           : orc_minres(N6, apply_cb, &ctx, b, eps_tilde, tol, max_it, &est, hist);
    }
    /* true residual ||A eps - b|| / ||b|| */
    orc_apply_mixed(n, phi, E, nu, deriv, mask, eps_tilde, r);
    double nb = sqrt(dot(N6, b, b)), nr = 0;
    for (long i = 0; i < N6; ++i) { double d = r[i] - b[i]; nr += d * d; }
    nr = sqrt(nr);
    info[0] = it;
    info[1] = est;
    info[2] = (nb > 0) ? nr / nb : 0.0;
    /* mean stress and mean strain */
    for (int i = 0; i < 6; ++i) sig_mean[i] = 0.0;
    double em[6] = {0, 0, 0, 0, 0, 0};
    for (long x = 0; x < V; ++x) {
        for (int i = 0; i < 6; ++i) {
            double s = 0;
            for (int j = 0; j < 6; ++j) s += Cm[i * 6 + j] * (Ekl[j] + eps_tilde[(long)j * V + x]);
            sig_mean[i] += phi[x] * s;
            em[i] += eps_tilde[(long)i * V + x];
        }
    }
    for (int i = 0; i < 6; ++i) sig_mean[i] /= (double)V;
    if (eps_mean)
        for (int i = 0; i < 6; ++i) eps_mean[i] = Ekl[i] + em[i] / (double)V;
    free(b); free(r);
    return it;
}

/* Pure strain control: orc_solve_mixed with no stress-controlled component. */
int orc_solve(const int n[3], const double *phi, double E, double nu, int deriv,
              const double Ebar[6], double tol, int max_it,
              double *eps_tilde, double sig_mean[6], double info[3], double *hist) {
    const double zero[6] = {0, 0, 0, 0, 0, 0};
    return orc_solve_mixed(n, phi, E, nu, deriv, 0, Ebar, zero, 0, tol, max_it, eps_tilde, sig_mean, NULL, info,
                           hist);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* MoDBFFT (section 2.2): penalised displacement FFT, strain control.         */
/* Unknown: the DFT of the displacement fluctuation, 3 complex components per */
/* frequency (full spectrum here), continuous frequencies of eq. (freq) with  */
/* the Nyquist component of xi set to 0.  Frequencies with xi = 0 carry no    */
/* unknown (u^ = 0 there) and no equation.                                    */
/* ------------------------------------------------------------------------ */

/* continuous xi with the Nyquist components zeroed */
static void modb_xi(const int n[3], const int k[3], cplx xi[3]) {
    for (int p = 0; p < 3; ++p) {
        double q = 2.0 * PI * signed_index(k[p], n[p]) / n[p];
        xi[p] = is_nyquist(k[p], n[p]) ? 0.0 : I * q * n[p];
    }
}

static int xi_zero(const cplx xi[3]) { return xi[0] == 0.0 && xi[1] == 0.0 && xi[2] == 0.0; }

/* out = A^alpha(u^), eq. (modbfftfop) without the stress-control rows:
 *   F{ (1 - chi_v) C : F^-1{ u^ (x)^s xi } } . xi + F{ chi_v F^-1{ alpha (u^ (x)^s xi) . xi } }
 * with chi_v = [phi == 0] (eq. indicator) and C = phi C_m.  u, out: 3 x V
 * complex (re,im), full spectrum.  alpha in the units of E. */
void orc_modb_apply(const int n[3], const double *phi, double E, double nu, double alpha,
                    const double *u_ri, double *out_ri) {
    long V = (long)n[0] * n[1] * n[2];
    const cplx *u = (const cplx *)u_ri;
    cplx *out = (cplx *)out_ri;
    double Cm[36];
    orc_stiffness_mandel(E, nu, Cm);
    cplx *eps = (cplx *)malloc(sizeof(cplx) * 6 * V);   /* Mandel */
    cplx *g = (cplx *)malloc(sizeof(cplx) * 3 * V);
    const double r2 = sqrt(2.0);
    /* strain sym(u (x) xi) and penalty vector alpha sym(u (x) xi) . xi per frequency */
    for (long f = 0; f < V; ++f) {
        int k[3] = {(int)(f / ((long)n[1] * n[2])), (int)((f / n[2]) % n[1]), (int)(f % n[2])};
        cplx xi[3], uu[3], e[3][3];
        modb_xi(n, k, xi);
        int zero = xi_zero(xi);
        for (int i = 0; i < 3; ++i) uu[i] = zero ? 0.0 : u[(long)i * V + f];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) e[i][j] = 0.5 * (uu[i] * xi[j] + uu[j] * xi[i]);
        for (int c = 0; c < 6; ++c) eps[(long)c * V + f] = (c < 3) ? e[MI[c]][MJ[c]] : r2 * e[MI[c]][MJ[c]];
        for (int i = 0; i < 3; ++i) {
            cplx s = 0;
            for (int j = 0; j < 3; ++j) s += e[i][j] * xi[j];
            g[(long)i * V + f] = alpha * s;
        }
    }
    for (int c = 0; c < 6; ++c) orc_fft3d(n, (double *)(eps + (long)c * V), +1);
    for (int c = 0; c < 3; ++c) orc_fft3d(n, (double *)(g + (long)c * V), +1);
    /* real space: tau = phi C_m : eps, h = chi_v g  (the 1/V of the inverse DFT applied here) */
    for (long x = 0; x < V; ++x) {
        double ev[6], tv[6];
        for (int c = 0; c < 6; ++c) ev[c] = creal(eps[(long)c * V + x]) / (double)V;
        for (int i = 0; i < 6; ++i) {
            double s = 0;
            for (int j = 0; j < 6; ++j) s += Cm[i * 6 + j] * ev[j];
            tv[i] = phi[x] * s;
        }
        for (int c = 0; c < 6; ++c) eps[(long)c * V + x] = tv[c];
        double chi = (phi[x] == 0.0) ? 1.0 : 0.0;
        for (int c = 0; c < 3; ++c) g[(long)c * V + x] = chi * creal(g[(long)c * V + x]) / (double)V;
    }
    for (int c = 0; c < 6; ++c) orc_fft3d(n, (double *)(eps + (long)c * V), -1);
    for (int c = 0; c < 3; ++c) orc_fft3d(n, (double *)(g + (long)c * V), -1);
    /* out = tau^ . xi + h^, zero where xi = 0 */
    for (long f = 0; f < V; ++f) {
        int k[3] = {(int)(f / ((long)n[1] * n[2])), (int)((f / n[2]) % n[1]), (int)(f % n[2])};
        cplx xi[3], tm[6], t[3][3];
        modb_xi(n, k, xi);
        if (xi_zero(xi)) {
            for (int i = 0; i < 3; ++i) out[(long)i * V + f] = 0.0;
            continue;
        }
        for (int c = 0; c < 6; ++c) tm[c] = eps[(long)c * V + f];
        mandel_to_tensor(tm, t);
        for (int i = 0; i < 3; ++i) {
            cplx s = g[(long)i * V + f];
            for (int j = 0; j < 3; ++j) s += t[i][j] * xi[j];
            out[(long)i * V + f] = s;
        }
    }
    free(eps);
    free(g);
}

/* b^ = -F{ C : E_bar } . xi  (eq. modbfftfrhs, sigma_bar = 0), 3 x V complex */
void orc_modb_rhs(const int n[3], const double *phi, double E, double nu, const double Ebar[6],
                  double *out_ri) {
    long V = (long)n[0] * n[1] * n[2];
    cplx *out = (cplx *)out_ri;
    double Cm[36], s[6];
    orc_stiffness_mandel(E, nu, Cm);
    for (int i = 0; i < 6; ++i) {
        s[i] = 0;
        for (int j = 0; j < 6; ++j) s[i] += Cm[i * 6 + j] * Ebar[j];
    }
    cplx *tau = (cplx *)malloc(sizeof(cplx) * 6 * V);
    for (int c = 0; c < 6; ++c)
        for (long x = 0; x < V; ++x) tau[(long)c * V + x] = phi[x] * s[c];
    for (int c = 0; c < 6; ++c) orc_fft3d(n, (double *)(tau + (long)c * V), -1);
    for (long f = 0; f < V; ++f) {
        int k[3] = {(int)(f / ((long)n[1] * n[2])), (int)((f / n[2]) % n[1]), (int)(f % n[2])};
        cplx xi[3], tm[6], t[3][3];
        modb_xi(n, k, xi);
        for (int c = 0; c < 6; ++c) tm[c] = tau[(long)c * V + f];
        mandel_to_tensor(tm, t);
        for (int i = 0; i < 3; ++i) {
            cplx v = 0;
            if (!xi_zero(xi))
                for (int j = 0; j < 3; ++j) v += t[i][j] * xi[j];
            out[(long)i * V + f] = -v;
        }
    }
    free(tau);
}

/* Preconditioner of eq. (precf): out(k) = [xi . Cbar . xi]^-1 in(k), Cbar =
 * <phi> C_m (eq. avstiff), solved per frequency by Gaussian elimination;
 * zero where xi = 0. */
void orc_modb_precond(const int n[3], double phibar, double E, double nu, const double *in_ri,
                      double *out_ri) {
    long V = (long)n[0] * n[1] * n[2];
    const cplx *in = (const cplx *)in_ri;
    cplx *out = (cplx *)out_ri;
    double lam = phibar * E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double mu = phibar * E / (2.0 * (1.0 + nu));
    for (long f = 0; f < V; ++f) {
        int k[3] = {(int)(f / ((long)n[1] * n[2])), (int)((f / n[2]) % n[1]), (int)(f % n[2])};
        cplx xi[3], K[3][3], v[3], u[3];
        modb_xi(n, k, xi);
        if (xi_zero(xi)) {
            for (int i = 0; i < 3; ++i) out[(long)i * V + f] = 0.0;
            continue;
        }
        /* (xi . C . xi)_ik = sum_jl xi_j C_ijkl xi_l, isotropic C */
        cplx xx = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
        for (int i = 0; i < 3; ++i)
            for (int kk = 0; kk < 3; ++kk)
                K[i][kk] = (lam + mu) * xi[i] * xi[kk] + (i == kk ? mu * xx : 0.0);
        for (int i = 0; i < 3; ++i) v[i] = in[(long)i * V + f];
        if (!solve3(K, v, u)) u[0] = u[1] = u[2] = 0.0;
        for (int i = 0; i < 3; ++i) out[(long)i * V + f] = u[i];
    }
}

/* Fluctuation strain F^-1{ u^ (x)^s xi } (6 x V Mandel, real part) and the
 * mean stress <C : (E_bar + eps)> (Mandel) of a MoDBFFT solution. */
void orc_modb_fields(const int n[3], const double *phi, double E, double nu, const double Ebar[6],
                     const double *u_ri, double *eps_out, double sig_mean[6]) {
    long V = (long)n[0] * n[1] * n[2];
    const cplx *u = (const cplx *)u_ri;
    cplx *e6 = (cplx *)malloc(sizeof(cplx) * 6 * V);
    const double r2 = sqrt(2.0);
    for (long f = 0; f < V; ++f) {
        int k[3] = {(int)(f / ((long)n[1] * n[2])), (int)((f / n[2]) % n[1]), (int)(f % n[2])};
        cplx xi[3], uu[3];
        modb_xi(n, k, xi);
        int zero = xi_zero(xi);
        for (int i = 0; i < 3; ++i) uu[i] = zero ? 0.0 : u[(long)i * V + f];
        for (int c = 0; c < 6; ++c) {
            cplx v = 0.5 * (uu[MI[c]] * xi[MJ[c]] + uu[MJ[c]] * xi[MI[c]]);
            e6[(long)c * V + f] = (c < 3) ? v : r2 * v;
        }
    }
    for (int c = 0; c < 6; ++c) orc_fft3d(n, (double *)(e6 + (long)c * V), +1);
    double Cm[36];
    orc_stiffness_mandel(E, nu, Cm);
    for (int i = 0; i < 6; ++i) sig_mean[i] = 0.0;
    for (long x = 0; x < V; ++x) {
        double ev[6];
        for (int c = 0; c < 6; ++c) {
            ev[c] = creal(e6[(long)c * V + x]) / (double)V;
            eps_out[(long)c * V + x] = ev[c];
        }
        for (int i = 0; i < 6; ++i) {
            double s = 0;
            for (int j = 0; j < 6; ++j) s += Cm[i * 6 + j] * (Ebar[j] + ev[j]);
            sig_mean[i] += phi[x] * s;
        }
    }
    for (int i = 0; i < 6; ++i) sig_mean[i] /= (double)V;
    free(e6);
}

/* ------------------------------------------------------------------------ */
/* Phase-field smoothening (PFS, section 3.2).  The phase map minimises       */
/* eq. (phase); its Euler-Lagrange equation (phase2) is solved in Fourier     */
/* space, eq. (phase3): phi^(xi) = omega^(xi) / (1 + (l^2/eps) |xi|^2) with   */
/* the continuous frequencies of eq. (freq) (xi = i q N / L, so xi . xi =     */
/* -|q N / L|^2).  The indicator omega is given on a fine grid (ratio r times */
/* the simulation grid along every axis); with voxel size d on the fine grid */
/* and l in units of d, (l^2/eps) |xi|^2 = (l^2/eps) sum_p q_p^2 with         */
/* q_p = 2 pi m_p / N_p, m_p the signed frequency index.  The fine phase map  */
/* is averaged over r^3 blocks onto the simulation grid, values below the     */
/* threshold (5 % in the paper) are set to 0, and round-off above 1 to 1.     */
/* ------------------------------------------------------------------------ */
void orc_pfs(const int nf[3], const double *omega, int ratio, double ell, double eps, double threshold,
             double *phi_coarse) {
    long Vf = (long)nf[0] * nf[1] * nf[2];
    cplx *w = (cplx *)malloc(sizeof(cplx) * Vf);
    for (long i = 0; i < Vf; ++i) w[i] = omega[i];
    orc_fft3d(nf, (double *)w, -1);
    const double c = ell * ell / eps;
    for (long f = 0; f < Vf; ++f) {
        int k[3] = {(int)(f / ((long)nf[1] * nf[2])), (int)((f / nf[2]) % nf[1]), (int)(f % nf[2])};
        double q2 = 0.0;
        for (int p = 0; p < 3; ++p) {
            double q = 2.0 * PI * (double)signed_index(k[p], nf[p]) / (double)nf[p];
            q2 += q * q;
        }
        w[f] /= (1.0 + c * q2);
    }
    orc_fft3d(nf, (double *)w, +1);
    const int nc[3] = {nf[0] / ratio, nf[1] / ratio, nf[2] / ratio};
    const double inv = 1.0 / ((double)ratio * ratio * ratio * (double)Vf);
    for (long i = 0; i < (long)nc[0] * nc[1] * nc[2]; ++i) phi_coarse[i] = 0.0;
    for (long f = 0; f < Vf; ++f) {
        int x[3] = {(int)(f / ((long)nf[1] * nf[2])), (int)((f / nf[2]) % nf[1]), (int)(f % nf[2])};
        long cidx = ((long)(x[0] / ratio) * nc[1] + x[1] / ratio) * nc[2] + x[2] / ratio;
        phi_coarse[cidx] += creal(w[f]) * inv;
    }
    for (long i = 0; i < (long)nc[0] * nc[1] * nc[2]; ++i) {
        if (phi_coarse[i] < threshold) phi_coarse[i] = 0.0;
        if (phi_coarse[i] > 1.0) phi_coarse[i] = 1.0;   /* phi lies in [0, 1]; FFT round-off */
    }
    free(w);
}

/* ------------------------------------------------------------------------ */
/* J2 plasticity and the Newton extension of the Galerkin scheme (section     */
/* 2.1.1).  The lattice material is small-strain von Mises plasticity with    */
/* linear isotropic hardening H (H = 0: the perfectly plastic law of section */
/* 5); a voxel's stress and tangent are those of the pristine material times */
/* phi (section 3.2).  Return mapping and consistent tangent are the radial  */
/* return of Simo & Hughes (Computational Inelasticity, 1998, section 3.3),  */
/* in Mandel components with m = (1,1,1,0,0,0).                               */
/* ------------------------------------------------------------------------ */
void orc_j2_point(double E, double nu, double sy, double H, double phi, const double eps[6],
                  const double epsp_n[6], double alpha_n, double sig[6], double Ct[36], double epsp[6],
                  double *alpha) {
    const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = E / (2.0 * (1.0 + nu));
    const double kappa = lam + 2.0 * mu / 3.0;
    const double m[6] = {1, 1, 1, 0, 0, 0};
    double ee[6], st[6], s[6], n[6] = {0, 0, 0, 0, 0, 0};
    for (int c = 0; c < 6; ++c) ee[c] = eps[c] - epsp_n[c];
    const double tr = ee[0] + ee[1] + ee[2];
    for (int c = 0; c < 6; ++c) st[c] = lam * tr * m[c] + 2.0 * mu * ee[c];        /* trial stress */
    const double p = (st[0] + st[1] + st[2]) / 3.0;
    double ns = 0.0;
    for (int c = 0; c < 6; ++c) { s[c] = st[c] - p * m[c]; ns += s[c] * s[c]; }
    ns = sqrt(ns);
    const double f = ns - sqrt(2.0 / 3.0) * (sy + H * alpha_n);                     /* trial yield function */
    double theta = 1.0, thetab = 0.0;
    for (int c = 0; c < 6; ++c) { sig[c] = st[c]; epsp[c] = epsp_n[c]; }
    *alpha = alpha_n;
    if (f > 0.0 && ns > 0.0) {
        const double dg = f / (2.0 * mu + 2.0 * H / 3.0);                              /* consistency */
        for (int c = 0; c < 6; ++c) {
            n[c] = s[c] / ns;
            sig[c] = st[c] - 2.0 * mu * dg * n[c];
            epsp[c] = epsp_n[c] + dg * n[c];
        }
        *alpha = alpha_n + sqrt(2.0 / 3.0) * dg;
        theta = 1.0 - 2.0 * mu * dg / ns;
        thetab = 1.0 / (1.0 + H / (3.0 * mu)) - (1.0 - theta);
    }
    /* C = kappa m (x) m + 2 mu theta (I - m (x) m / 3) - 2 mu thetab n (x) n */
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
            Ct[i * 6 + j] = phi * (kappa * m[i] * m[j] + 2.0 * mu * theta * ((i == j) - m[i] * m[j] / 3.0) -
                                   2.0 * mu * thetab * n[i] * n[j]);
    for (int c = 0; c < 6; ++c) sig[c] *= phi;
}

typedef struct {
    const int *n;
    const double *Ct;       /* 36 per voxel: the tangent of the last return mapping */
    int deriv, mask;
} tangent_ctx;

/* A_i(v) = F^-1{ G : F{ C^{i-1}(x) : v } } with the mixed projector, eq. (galnonlin) */
static void tangent_cb(void *c, const double *x, double *y) {
    tangent_ctx *t = (tangent_ctx *)c;
    orc_problem P;
    memcpy(P.n, t->n, sizeof P.n);
    P.phi = NULL; P.deriv = t->deriv; P.mask = t->mask;
    long V = (long)P.n[0] * P.n[1] * P.n[2];
    cplx *tau = (cplx *)malloc(sizeof(cplx) * 6 * V);
#pragma omp parallel for schedule(static)
    for (long v = 0; v < V; ++v)
        for (int i = 0; i < 6; ++i) {
            double s = 0;
            for (int j = 0; j < 6; ++j) s += t->Ct[v * 36 + i * 6 + j] * x[(long)j * V + v];
            tau[(long)i * V + v] = s;
        }
    project_field(&P, tau, y);
    free(tau);
}

typedef struct {
    const int *n;
    const double *phi;
    double E, nu, sy, H;
    int deriv, mask;
    const double *epsp, *alpha, *Sbar;
} j2_problem;

/* stress and tangent at eps (history at t) and b = -F^-1{ G : F{ sigma - Sbar } }
 * (right-hand side of eq. galnonlin); returns ||b|| */
static double j2_residual(const j2_problem *J, const double *eps, double *sig, double *Ct, double *b) {
    long V = (long)J->n[0] * J->n[1] * J->n[2], N6 = 6 * V;
#pragma omp parallel for schedule(static)
    for (long v = 0; v < V; ++v) {
        double e[6], ep[6], s6[6], epn[6], aln;
        for (int c = 0; c < 6; ++c) { e[c] = eps[(long)c * V + v]; ep[c] = J->epsp[(long)c * V + v]; }
        orc_j2_point(J->E, J->nu, J->sy, J->H, J->phi[v], e, ep, J->alpha[v], s6, Ct + v * 36, epn, &aln);
        for (int c = 0; c < 6; ++c) sig[(long)c * V + v] = s6[c];
    }
    orc_problem P;
    memcpy(P.n, J->n, sizeof P.n);
    P.phi = NULL; P.deriv = J->deriv; P.mask = J->mask;
    cplx *tau = (cplx *)malloc(sizeof(cplx) * N6);
    for (int c = 0; c < 6; ++c)
        for (long v = 0; v < V; ++v)
            tau[(long)c * V + v] = sig[(long)c * V + v] - (((J->mask >> c) & 1) ? J->Sbar[c] : 0.0);
    project_field(&P, tau, b);
    free(tau);
    for (long i = 0; i < N6; ++i) b[i] = -b[i];
    return sqrt(dot(N6, b, b));
}

/* One load increment t -> t + dt by an inexact damped Newton method (section
 * 2.1.1).  eps: total strain field (6 x V Mandel) at t on entry, at t + dt on
 * return; epsp (6 x V) and alpha (V): plastic history at t, updated on
 * return.  The kl components follow the macro strain from Ebar_t to Ebar_n
 * (the first iterate adds the difference uniformly), the KL components in
 * mask carry the mean stress Sbar_n.  Each Newton step solves eq.
 * (galnonlin) by MINRES to ||A dE - b_i|| <= tol_lin ||b_0|| (eq. galrlin)
 * and is damped by halving its length (at most 7 times) until ||b|| falls;
 * the increment is accepted when ||dE||_inf <= tol_newton ||eps^i - eps^t||_inf
 * (eq. galrnewton) after a step whose linear residual met tol_lin.  info:
 * Newton iterations, linear iterations, last r_newton, ||b|| / ||b_0|| at
 * exit, accepted (1/0). */
int orc_j2_increment(const int n[3], const double *phi, double E, double nu, double sy, double H, int deriv,
                     int mask, double *eps, double *epsp, double *alpha, const double Ebar_t[6],
                     const double Ebar_n[6], const double Sbar_n[6], double tol_lin, double tol_newton,
                     int max_newton, int max_lin, double sig_mean[6], double eps_mean[6], double info[5]) {
    long V = (long)n[0] * n[1] * n[2], N6 = 6 * V;
    double *eps_t = (double *)malloc(sizeof(double) * N6);
    double *sig = (double *)malloc(sizeof(double) * N6);
    double *Ct = (double *)malloc(sizeof(double) * 36 * V);
    double *b = (double *)malloc(sizeof(double) * N6);
    double *de = (double *)malloc(sizeof(double) * N6);
    double *etry = (double *)malloc(sizeof(double) * N6);
    double *btry = (double *)malloc(sizeof(double) * N6);
    double *Ctry = (double *)malloc(sizeof(double) * 36 * V);
    memcpy(eps_t, eps, sizeof(double) * N6);
    for (int c = 0; c < 6; ++c)
        if (!((mask >> c) & 1))
            for (long v = 0; v < V; ++v) eps[(long)c * V + v] += Ebar_n[c] - Ebar_t[c];
    j2_problem J = {n, phi, E, nu, sy, H, deriv, mask, epsp, alpha, Sbar_n};
    double nb = j2_residual(&J, eps, sig, Ct, b);
    const double b0 = nb;
    double rn = 0.0;
    int it = 0, lin = 0, done = (nb == 0.0);
    while (!done && it < max_newton) {
        ++it;
        tangent_ctx tc = {n, Ct, deriv, mask};
        double est;
        const double tol_i = tol_lin * b0 / nb;
        const int k = orc_minres(N6, tangent_cb, &tc, b, de, tol_i < 0.5 ? tol_i : 0.5, max_lin, &est, NULL);
        lin += k;
        const int lin_ok = est * nb <= tol_lin * b0 * (1.0 + 1e-9) || tol_i >= 0.5;
        double t = 1.0, nt = 0.0;
        for (int tries = 0; tries < 8; ++tries) {
            for (long i = 0; i < N6; ++i) etry[i] = eps[i] + t * de[i];
            nt = j2_residual(&J, etry, sig, Ctry, btry);
            if (nt < (1.0 - 1e-4 * t) * nb || tries == 7) break;
            t *= 0.5;
        }
        double dmax = 0.0, emax = 0.0;
        for (long i = 0; i < N6; ++i) {
            const double d = fabs(etry[i] - eps[i]), e = fabs(etry[i] - eps_t[i]);
            if (d > dmax) dmax = d;
            if (e > emax) emax = e;
        }
        memcpy(eps, etry, sizeof(double) * N6);
        memcpy(b, btry, sizeof(double) * N6);
        memcpy(Ct, Ctry, sizeof(double) * 36 * V);
        nb = nt;
        rn = emax > 0.0 ? dmax / emax : 0.0;
        if (lin_ok && rn <= tol_newton) done = 1;
    }
    /* history, mean stress and strain at the accepted iterate */
    double *ep_new = de, *al_new = (double *)malloc(sizeof(double) * V);
    for (int c = 0; c < 6; ++c) { sig_mean[c] = 0.0; eps_mean[c] = 0.0; }
    for (long v = 0; v < V; ++v) {
        double e[6], ep[6], s6[6], ct[36], epn[6], aln;
        for (int c = 0; c < 6; ++c) { e[c] = eps[(long)c * V + v]; ep[c] = epsp[(long)c * V + v]; }
        orc_j2_point(E, nu, sy, H, phi[v], e, ep, alpha[v], s6, ct, epn, &aln);
        for (int c = 0; c < 6; ++c) {
            ep_new[(long)c * V + v] = epn[c];
            sig_mean[c] += s6[c];
            eps_mean[c] += e[c];
        }
        al_new[v] = aln;
    }
    memcpy(epsp, ep_new, sizeof(double) * N6);
    memcpy(alpha, al_new, sizeof(double) * V);
    for (int c = 0; c < 6; ++c) { sig_mean[c] /= (double)V; eps_mean[c] /= (double)V; }
    info[0] = it; info[1] = lin; info[2] = rn; info[3] = b0 > 0.0 ? nb / b0 : 0.0; info[4] = done;
    free(eps_t); free(sig); free(Ct); free(b); free(de); free(etry); free(btry); free(Ctry); free(al_new);
    return it;
}
