// hom_modb.cuh -- point-wise kernels of the MoDBFFT solver (section 2.2):
// the displacement unknown u^ (3 complex components per frequency of the
// half spectrum) is expanded into the strain sym(u^ (x) xi) and the penalty
// vector alpha sym(u^ (x) xi) . xi before the inverse transform, and the
// transformed stress / penalty fields are contracted back, eq. (modbfftfop):
//   A^alpha(u^) = F{ (1-chi_v) C : F^-1{ u^ (x)^s xi } } . xi
//               + F{ chi_v F^-1{ alpha (u^ (x)^s xi) . xi } }.
// Frequencies are the continuous ones of eq. (freq), xi_p = i 2 pi m_p (unit
// cell), with the Nyquist component set to 0; where xi = 0 there is no
// unknown and no equation.  The preconditioner is eq. (precf) with the mean
// stiffness of eq. (avstiff).
#pragma once
#include "hom_internal.h"

namespace hom {

// frequency index of half-spectrum point f and its continuous xi / (i 2 pi)
__device__ __forceinline__ void modb_freq(const Geometry &g, int f, double q[3], int &k3) {
    const int hh = g.h;
    k3 = f % hh;
    const int rest = f / hh;
    const int k2 = rest % g.n2, k1 = rest / g.n2;
    const int ks[3] = {k1, k2, k3}, ns[3] = {g.n1, g.n2, g.n3};
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int n = ns[p], k = ks[p];
        q[p] = ((n & 1) == 0 && 2 * k == n) ? 0.0 : (double)((2 * k < n) ? k : k - n);
    }
}

// out10 = (sym(u (x) xi) Mandel, alpha sym(u (x) xi) . xi, 0), or the first
// six with nc_out = 6 (modb_expand_at)
template <typename R>
__global__ void k_modb_expand(Geometry g, R alpha, int with_penalty, const cpx<R> *__restrict__ u,
                              cpx<R> *__restrict__ out, int nc_out, const MinresState *state) {
    if (state && state->done) return;
    const int hh = g.h;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < (int)g.S; f += gridDim.x * blockDim.x) {
        const int k3 = f % hh, rest = f / hh;
        const int k2 = rest % g.n2, k1 = rest / g.n2;
        modb_expand_at<R>(g, k1, k2, k3, u + 3 * (size_t)f, alpha, with_penalty, nc_out, out + (size_t)f * nc_out);
    }
}

// out3 = tau^ . xi + h^ (10-component input), 0 where xi = 0; with dotv,
// the weighted partial sum <dotv, out3> per CTA
template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_modb_contract(Geometry g, const cpx<R> *__restrict__ in,
                                                              cpx<R> *__restrict__ out,
                                                              const cpx<R> *__restrict__ dotv, double *partials,
                                                              const MinresState *state) {
    if (state && state->done) return;
    const R tp = (R)6.28318530717958647692;
    const R r2 = (R)0.70710678118654752440;
    double acc = 0.0;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < (int)g.S; f += gridDim.x * blockDim.x) {
        double qd[3];
        int k3;
        modb_freq(g, f, qd, k3);
        cpx<R> r[3] = {mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0)};
        if (!(qd[0] == 0.0 && qd[1] == 0.0 && qd[2] == 0.0)) {
            const R s[3] = {tp * (R)qd[0], tp * (R)qd[1], tp * (R)qd[2]};
            const cpx<R> *t = in + (size_t)f * 10;
            const cpx<R> T[3][3] = {{t[0], scale<R>(t[5], r2), scale<R>(t[4], r2)},
                                    {scale<R>(t[5], r2), t[1], scale<R>(t[3], r2)},
                                    {scale<R>(t[4], r2), scale<R>(t[3], r2), t[2]}};
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                // (tau xi)_i = i sum_j tau_ij s_j
                const cpx<R> a = add<R>(add<R>(scale<R>(T[i][0], s[0]), scale<R>(T[i][1], s[1])), scale<R>(T[i][2], s[2]));
                r[i] = add<R>(mk<R>(-a.y, a.x), t[6 + i]);
            }
        }
        const double w = (k3 == 0 || 2 * k3 == g.n3) ? 1.0 : 2.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            out[3 * f + i] = r[i];
            if (dotv) {
                const cpx<R> d = dotv[3 * f + i];
                acc += w * ((double)d.x * (double)r[i].x + (double)d.y * (double)r[i].y);
            }
        }
    }
    if (dotv) {
        const double sum = block_sum(acc);
        if (threadIdx.x == 0) partials[blockIdx.x] = sum;
    }
}

// out3 = [xi . Cbar . xi]^-1 in3, Cbar isotropic (lam_b, mu_b): with xi = i s,
// xi.Cbar.xi = -((lam+mu) s s^T + mu |s|^2 I), inverse in closed form.
template <typename R>
__device__ __forceinline__ void modb_precond_point(double lam_b, double mu_b, const double qd[3], const cpx<R> *in,
                                                   cpx<R> *out) {
    if (qd[0] == 0.0 && qd[1] == 0.0 && qd[2] == 0.0) {
        out[0] = out[1] = out[2] = mk<R>(0, 0);
        return;
    }
    const double tp = 6.28318530717958647692;
    const double s0 = tp * qd[0], s1 = tp * qd[1], s2 = tp * qd[2];
    const double ss = s0 * s0 + s1 * s1 + s2 * s2;
    const double a = -1.0 / (mu_b * ss), b = (lam_b + mu_b) / ((lam_b + 2.0 * mu_b) * ss);
    const cpx<R> v0 = in[0], v1 = in[1], v2 = in[2];
    const double dre = s0 * v0.x + s1 * v1.x + s2 * v2.x, dim = s0 * v0.y + s1 * v1.y + s2 * v2.y;
    const double sv[3] = {s0, s1, s2};
    const cpx<R> vv[3] = {v0, v1, v2};
#pragma unroll
    for (int i = 0; i < 3; ++i)
        out[i] = mk<R>((R)(a * (vv[i].x - b * sv[i] * dre)), (R)(a * (vv[i].y - b * sv[i] * dim)));
}

template <typename R>
__global__ void k_modb_precond(Geometry g, double lam_b, double mu_b, const cpx<R> *__restrict__ in,
                               cpx<R> *__restrict__ out) {
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < (int)g.S; f += gridDim.x * blockDim.x) {
        double qd[3];
        int k3;
        modb_freq(g, f, qd, k3);
        modb_precond_point<R>(lam_b, mu_b, qd, in + 3 * f, out + 3 * f);
    }
}

// PCG step: x += a p; r -= a q; z = M r; partials <r,z> (first half) and
// <r,r> (second half), Parseval-weighted
template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_cg_xr(Geometry g, double lam_b, double mu_b, cpx<R> *__restrict__ x,
                                                      cpx<R> *__restrict__ r, const cpx<R> *__restrict__ p,
                                                      const cpx<R> *__restrict__ q, cpx<R> *__restrict__ z,
                                                      const CgState *st, double *partials) {
    if (st->done) return;
    const R a = (R)st->a;
    double rz = 0.0, rr = 0.0;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < (int)g.S; f += gridDim.x * blockDim.x) {
        double qd[3];
        int k3;
        modb_freq(g, f, qd, k3);
        cpx<R> rv[3], zv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const cpx<R> pp = p[3 * f + i], qq = q[3 * f + i], xx = x[3 * f + i], rr0 = r[3 * f + i];
            x[3 * f + i] = mk<R>(xx.x + a * pp.x, xx.y + a * pp.y);
            rv[i] = mk<R>(rr0.x - a * qq.x, rr0.y - a * qq.y);
            r[3 * f + i] = rv[i];
        }
        modb_precond_point<R>(lam_b, mu_b, qd, rv, zv);
        const double w = (k3 == 0 || 2 * k3 == g.n3) ? 1.0 : 2.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            z[3 * f + i] = zv[i];
            rz += w * ((double)rv[i].x * zv[i].x + (double)rv[i].y * zv[i].y);
            rr += w * ((double)rv[i].x * rv[i].x + (double)rv[i].y * rv[i].y);
        }
    }
    const double s1 = block_sum(rz);
    if (threadIdx.x == 0) partials[blockIdx.x] = s1;
    const double s2 = block_sum(rr);
    if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = s2;
}

// PCG direction: p = z + b p
template <typename R>
__global__ void k_cg_p(int n, cpx<R> *__restrict__ p, const cpx<R> *__restrict__ z, const CgState *st) {
    if (st->done) return;
    const R b = (R)st->b;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const cpx<R> pp = p[i], zz = z[i];
        p[i] = mk<R>(zz.x + b * pp.x, zz.y + b * pp.y);
    }
}

// ----- launchers ------------------------------------------------------------
template <typename R>
void Launch<R>::modb_expand(const Geometry &g, cudaStream_t st, double alpha, int with_penalty, const cpx<R> *u,
                            cpx<R> *out, int nc_out, const MinresState *state) {
    k_modb_expand<R><<<ew_grid(g.S), kEwThreads, 0, st>>>(g, (R)alpha, with_penalty, u, out, nc_out, state);
}
template <typename R>
void Launch<R>::modb_contract(const Geometry &g, cudaStream_t st, const cpx<R> *in10, cpx<R> *out3, const cpx<R> *dotv,
                              double *partials, const MinresState *state) {
    k_modb_contract<R><<<ew_grid(g.S), kEwThreads, 0, st>>>(g, in10, out3, dotv, partials, state);
}
template <typename R>
void Launch<R>::modb_precond(const Geometry &g, cudaStream_t st, double lam_b, double mu_b, const cpx<R> *in,
                             cpx<R> *out) {
    k_modb_precond<R><<<ew_grid(g.S), kEwThreads, 0, st>>>(g, lam_b, mu_b, in, out);
}
template <typename R>
void Launch<R>::cg_xr(const Geometry &g, cudaStream_t st, double lam_b, double mu_b, cpx<R> *x, cpx<R> *r,
                      const cpx<R> *p, const cpx<R> *q, cpx<R> *z, const CgState *state, double *partials) {
    k_cg_xr<R><<<ew_grid(g.S), kEwThreads, 0, st>>>(g, lam_b, mu_b, x, r, p, q, z, state, partials);
}
template <typename R>
void Launch<R>::cg_p(const Geometry &g, cudaStream_t st, cpx<R> *p, const cpx<R> *z, const CgState *state) {
    const int n = (int)(3 * g.S);
    k_cg_p<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, p, z, state);
}

}  // namespace hom
