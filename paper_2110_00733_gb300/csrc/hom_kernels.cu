// hom_kernels.cu -- sm_103a kernels of the Galerkin-FFT operator and of MINRES.
//
// One application of the operator of eq. (linearOp),
//     A(e) = F^-1{ G(xi) : F{ phi C_m : e } },
// is five passes over HBM:
//   x3_fwd : constitutive law (Voigt-scaled isotropic, section 3.3) fused with
//            the real-to-complex transform along the contiguous axis n3
//            (two real components packed into one complex line);
//   x2     : complex transform along n2 (forward);
//   x1     : complex transform along n1, the projector G of eq. (galop) at
//            every frequency (all 6 components of a frequency are in shared
//            memory together), and the inverse transform along n1;
//   x2     : inverse along n2;
//   x3_inv : complex-to-real along n3, scaling by 1/V, with the Krylov dot
//            product of the MINRES step fused into the store.
// The MINRES recurrences (section 2.1; Paige-Saunders) run in FP64 on one
// CTA; field updates are element-wise kernels with FP64 (float-float for FP32
// fields) partial sums and a deterministic two-level reduction.
#include <math.h>

#include "hom_internal.h"

namespace hom {

// ---------------------------------------------------------------------------
// Block-level reduction helpers.
// ---------------------------------------------------------------------------

// Per-thread accumulator of products: float-float (an error-free product and
// a compensated sum, ~44 significant bits) for FP32 data, plain FP64 for FP64
// data.  Either way the block sum is formed in FP64.
template <typename R> struct Acc;
template <> struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        float p = a * b;
        float e = fmaf(a, b, -p);
        float s = hi + p;
        float bp = s - hi;
        float err = (hi - (s - bp)) + (p - bp);
        hi = s;
        lo += err + e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <> struct Acc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ double value() const { return v; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; the result is valid in thread 0.  Fixed order.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = (lane < nw) ? red[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

__device__ __forceinline__ bool skip(const MinresState *s) { return s != nullptr && s->done; }

// ---------------------------------------------------------------------------
// Projector of eq. (galop) at one frequency, in closed form.  xi may be
// complex (rotated scheme).  With e = xi/|xi|, the orthogonal projection of a
// symmetric tau onto {sym(u (x) xi)} is sym(u (x) e) with
//     u = 2 tau conj(e) - e (conj(e) . tau conj(e))
// (Sherman-Morrison inverse of the acoustic tensor 1/2 (I + e e^H)).
// t[6] holds Mandel components, overwritten.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void gamma_project(cpx<R> *t, cpx<R> x0, cpx<R> x1, cpx<R> x2) {
    const R n2 = x0.x * x0.x + x0.y * x0.y + x1.x * x1.x + x1.y * x1.y + x2.x * x2.x + x2.y * x2.y;
    if (!(n2 > (R)0)) {
#pragma unroll
        for (int c = 0; c < 6; ++c) t[c] = mk<R>(0, 0);
        return;
    }
    const R inv = (R)1 / sqrt(n2);
    const cpx<R> e0 = scale<R>(x0, inv), e1 = scale<R>(x1, inv), e2 = scale<R>(x2, inv);
    const cpx<R> c0 = conjc<R>(e0), c1 = conjc<R>(e1), c2 = conjc<R>(e2);
    const R r2 = (R)0.70710678118654752440;   // 1/sqrt(2)
    const cpx<R> T11 = t[0], T22 = t[1], T33 = t[2];
    const cpx<R> T23 = scale<R>(t[3], r2), T13 = scale<R>(t[4], r2), T12 = scale<R>(t[5], r2);
    const cpx<R> v0 = add<R>(add<R>(mul<R>(T11, c0), mul<R>(T12, c1)), mul<R>(T13, c2));
    const cpx<R> v1 = add<R>(add<R>(mul<R>(T12, c0), mul<R>(T22, c1)), mul<R>(T23, c2));
    const cpx<R> v2 = add<R>(add<R>(mul<R>(T13, c0), mul<R>(T23, c1)), mul<R>(T33, c2));
    const cpx<R> s = add<R>(add<R>(mul<R>(c0, v0), mul<R>(c1, v1)), mul<R>(c2, v2));
    const cpx<R> u0 = sub<R>(scale<R>(v0, (R)2), mul<R>(e0, s));
    const cpx<R> u1 = sub<R>(scale<R>(v1, (R)2), mul<R>(e1, s));
    const cpx<R> u2 = sub<R>(scale<R>(v2, (R)2), mul<R>(e2, s));
    t[0] = mul<R>(u0, e0);
    t[1] = mul<R>(u1, e1);
    t[2] = mul<R>(u2, e2);
    t[3] = scale<R>(add<R>(mul<R>(u1, e2), mul<R>(u2, e1)), r2);
    t[4] = scale<R>(add<R>(mul<R>(u0, e2), mul<R>(u2, e0)), r2);
    t[5] = scale<R>(add<R>(mul<R>(u0, e1), mul<R>(u1, e0)), r2);
}

// ---------------------------------------------------------------------------
// Pass 1: constitutive law + R2C along n3.
// ---------------------------------------------------------------------------
struct Mac6 { double v[6]; };

template <typename R>
__global__ void __launch_bounds__(256) k_x3_fwd(Geometry g, int mode, const R *__restrict__ in,
                                                const R *__restrict__ phi, R lam, R mu2, Mac6 mac,
                                                cpx<R> *__restrict__ spec, const MinresState *state) {
    if (skip(state)) {
        // the iteration after convergence: no further w/x update either
        if (blockIdx.x == 0 && threadIdx.x == 0) const_cast<MinresState *>(state)->done_update = 1;
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = g.n3, ROWS = g.rows3, L = 3 * ROWS, H = g.h;
    cpx<R> *bufA = reinterpret_cast<cpx<R> *>(smem_raw);
    cpx<R> *bufB = bufA + N * L;
    const long long nrows = (long long)g.n1 * g.n2;
    const long long row0 = (long long)blockIdx.x * ROWS;
    const long long V = g.V;
    for (int idx = threadIdx.x; idx < ROWS * N; idx += blockDim.x) {
        const int r = idx / N, e = idx - r * N;
        const long long row = row0 + r;
        R t[6];
        if (row < nrows) {
            const long long vox = row * N + e;
            if (mode == X3F_RAW) {
#pragma unroll
                for (int c = 0; c < 6; ++c) t[c] = in[c * V + vox];
            } else {
                R ev[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) ev[c] = (mode == X3F_MACRO) ? (R)mac.v[c] : in[c * V + vox];
                const R ph = phi[vox];
                const R tr = lam * (ev[0] + ev[1] + ev[2]);
#pragma unroll
                for (int c = 0; c < 6; ++c) t[c] = ph * ((c < 3 ? tr : (R)0) + mu2 * ev[c]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) t[c] = 0;
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) bufA[e * L + p * ROWS + r] = mk<R>(t[2 * p], t[2 * p + 1]);
    }
    __syncthreads();
    cpx<R> *res = fft_lines<R, -1>(bufA, bufB, L, g.ax[2]);
    // unpack the two real transforms of each packed line:
    //   X_a[k] = (Z[k] + conj Z[N-k]) / 2,  X_b[k] = (Z[k] - conj Z[N-k]) / (2i)
    for (int idx = threadIdx.x; idx < ROWS * 3 * H; idx += blockDim.x) {
        const int k = idx % H;
        const int rest = idx / H;
        const int p = rest % 3, r = rest / 3;
        const long long row = row0 + r;
        if (row >= nrows) continue;
        const int km = (k == 0) ? 0 : N - k;
        const cpx<R> z = res[k * L + p * ROWS + r];
        const cpx<R> zm = conjc<R>(res[km * L + p * ROWS + r]);
        const cpx<R> xa = mk<R>((R)0.5 * (z.x + zm.x), (R)0.5 * (z.y + zm.y));
        const cpx<R> xb = mk<R>((R)0.5 * (z.y - zm.y), (R)-0.5 * (z.x - zm.x));
        spec[((long long)(2 * p) * nrows + row) * H + k] = xa;
        spec[((long long)(2 * p + 1) * nrows + row) * H + k] = xb;
    }
}

// ---------------------------------------------------------------------------
// Pass 2/4: complex transform along n2, in place on the half spectrum.
// Columns are (component, k1, k3) flattened; a CTA takes tile2 consecutive ones.
// ---------------------------------------------------------------------------
template <typename R, int S>
__global__ void __launch_bounds__(256) k_x2(Geometry g, cpx<R> *__restrict__ spec, const MinresState *state) {
    if (skip(state)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = g.n2, T = g.tile2, H = g.h;
    cpx<R> *bufA = reinterpret_cast<cpx<R> *>(smem_raw);
    cpx<R> *bufB = bufA + N * T;
    const long long total = 6LL * g.n1 * H;
    const long long f0 = (long long)blockIdx.x * T;
    for (int idx = threadIdx.x; idx < N * T; idx += blockDim.x) {
        const int e = idx / T, t = idx - e * T;
        const long long f = f0 + t;
        cpx<R> v = mk<R>(0, 0);
        if (f < total) {
            const long long q = f / H, k3 = f - q * H;
            v = spec[(q * N + e) * H + k3];
        }
        bufA[e * T + t] = v;
    }
    __syncthreads();
    cpx<R> *res = fft_lines<R, S>(bufA, bufB, T, g.ax[1]);
    for (int idx = threadIdx.x; idx < N * T; idx += blockDim.x) {
        const int e = idx / T, t = idx - e * T;
        const long long f = f0 + t;
        if (f < total) {
            const long long q = f / H, k3 = f - q * H;
            spec[(q * N + e) * H + k3] = res[e * T + t];
        }
    }
}

// ---------------------------------------------------------------------------
// Pass 3: transform along n1, projector G(xi), inverse along n1.
// Columns are (k2, k3) flattened; 6 components per column.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_x1(Geometry g, int flags, cpx<R> *__restrict__ spec,
                                            const MinresState *state) {
    if (skip(state)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = g.n1, T = g.tile1, H = g.h, L = 6 * T;
    cpx<R> *bufA = reinterpret_cast<cpx<R> *>(smem_raw);
    cpx<R> *bufB = bufA + N * L;
    const long long cols = (long long)g.n2 * H;
    const long long g0 = (long long)blockIdx.x * T;
    const long long sK1 = cols;        // stride between consecutive k1
    const long long sC = g.S;          // stride between components
    for (int idx = threadIdx.x; idx < N * L; idx += blockDim.x) {
        const int t = idx % T;
        const int rest = idx / T;
        const int c = rest % 6, e = rest / 6;
        const long long col = g0 + t;
        bufA[e * L + c * T + t] = (col < cols) ? spec[c * sC + e * sK1 + col] : mk<R>(0, 0);
    }
    __syncthreads();
    cpx<R> *cur = bufA, *oth = bufB;
    if (flags & X1_FWD) {
        cur = fft_lines<R, -1>(bufA, bufB, L, g.ax[0]);
        oth = (cur == bufA) ? bufB : bufA;
    }
    if (flags & X1_GAMMA) {
        const cpx<R> *D0 = reinterpret_cast<const cpx<R> *>(g.D[0]);
        const cpx<R> *D1 = reinterpret_cast<const cpx<R> *>(g.D[1]);
        const cpx<R> *D2 = reinterpret_cast<const cpx<R> *>(g.D[2]);
        const cpx<R> *M0 = reinterpret_cast<const cpx<R> *>(g.M[0]);
        const cpx<R> *M1 = reinterpret_cast<const cpx<R> *>(g.M[1]);
        const cpx<R> *M2 = reinterpret_cast<const cpx<R> *>(g.M[2]);
        for (int idx = threadIdx.x; idx < N * T; idx += blockDim.x) {
            const int e = idx / T, t = idx - e * T;
            const long long col = g0 + t;
            if (col >= cols) continue;
            const int k1 = e;
            const int k2 = (int)(col / H), k3 = (int)(col - (long long)k2 * H);
            cpx<R> tv[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) tv[c] = cur[e * L + c * T + t];
            // eq. (galop): zero at xi = 0 (strain control) and at every
            // frequency with a Nyquist index
            const bool nyq = ((g.n1 & 1) == 0 && 2 * k1 == g.n1) || ((g.n2 & 1) == 0 && 2 * k2 == g.n2) ||
                             ((g.n3 & 1) == 0 && 2 * k3 == g.n3);
            if (nyq || (k1 == 0 && k2 == 0 && k3 == 0)) {
#pragma unroll
                for (int c = 0; c < 6; ++c) tv[c] = mk<R>(0, 0);
            } else {
                const cpx<R> m0 = __ldg(&M0[k1]), m1 = __ldg(&M1[k2]), m2 = __ldg(&M2[k3]);
                const cpx<R> x0 = mul<R>(__ldg(&D0[k1]), mul<R>(m1, m2));
                const cpx<R> x1 = mul<R>(__ldg(&D1[k2]), mul<R>(m0, m2));
                const cpx<R> x2 = mul<R>(__ldg(&D2[k3]), mul<R>(m0, m1));
                gamma_project<R>(tv, x0, x1, x2);
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) cur[e * L + c * T + t] = tv[c];
        }
        __syncthreads();
    }
    if (flags & X1_INV) cur = fft_lines<R, 1>(cur, oth, L, g.ax[0]);
    for (int idx = threadIdx.x; idx < N * L; idx += blockDim.x) {
        const int t = idx % T;
        const int rest = idx / T;
        const int c = rest % 6, e = rest / 6;
        const long long col = g0 + t;
        if (col < cols) spec[c * sC + e * sK1 + col] = cur[e * L + c * T + t];
    }
}

// ---------------------------------------------------------------------------
// Pass 5: C2R along n3 with 1/V scaling and a fused reduction.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_x3_inv(Geometry g, int mode, const cpx<R> *__restrict__ spec,
                                                R *__restrict__ out, R scl, const R *__restrict__ dotv,
                                                double *__restrict__ partials, const MinresState *state) {
    if (skip(state)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = g.n3, ROWS = g.rows3, L = 3 * ROWS, H = g.h;
    cpx<R> *bufA = reinterpret_cast<cpx<R> *>(smem_raw);
    cpx<R> *bufB = bufA + N * L;
    const long long nrows = (long long)g.n1 * g.n2;
    const long long row0 = (long long)blockIdx.x * ROWS;
    const long long V = g.V;
    // pack two half spectra into one full complex line: Z = X_a + i X_b,
    // Z[N-k] = conj X_a[k] + i conj X_b[k]; the self-conjugate bins keep
    // their real parts only, as a complex-to-real transform does.
    for (int idx = threadIdx.x; idx < ROWS * 3 * H; idx += blockDim.x) {
        const int k = idx % H;
        const int rest = idx / H;
        const int p = rest % 3, r = rest / 3;
        const long long row = row0 + r;
        cpx<R> xa = mk<R>(0, 0), xb = mk<R>(0, 0);
        if (row < nrows) {
            xa = spec[((long long)(2 * p) * nrows + row) * H + k];
            xb = spec[((long long)(2 * p + 1) * nrows + row) * H + k];
        }
        const bool selfc = (k == 0) || (2 * k == N);
        if (selfc) { xa.y = 0; xb.y = 0; }
        bufA[k * L + p * ROWS + r] = mk<R>(xa.x - xb.y, xa.y + xb.x);
        if (!selfc) bufA[(N - k) * L + p * ROWS + r] = mk<R>(xa.x + xb.y, xb.x - xa.y);
    }
    __syncthreads();
    cpx<R> *res = fft_lines<R, 1>(bufA, bufB, L, g.ax[2]);
    Acc<R> acc;
    for (int idx = threadIdx.x; idx < ROWS * N; idx += blockDim.x) {
        const int r = idx / N, e = idx - r * N;
        const long long row = row0 + r;
        if (row >= nrows) continue;
        const long long vox = row * N + e;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const cpx<R> z = res[e * L + p * ROWS + r];
            const R a = z.x * scl, b = z.y * scl;
            const long long ia = (long long)(2 * p) * V + vox, ib = ia + V;
            out[ia] = a;
            out[ib] = b;
            if (mode == X3I_STORE_NORM2) { acc.add_prod(a, a); acc.add_prod(b, b); }
            else if (mode == X3I_STORE_DOT) { acc.add_prod(a, dotv[ia]); acc.add_prod(b, dotv[ib]); }
        }
    }
    if (mode != X3I_STORE) {
        const double s = block_sum(acc.value());
        if (threadIdx.x == 0) partials[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// Element-wise Krylov kernels (grid-stride, fixed grid of kEwBlocks).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_lanczos(long long n, R *__restrict__ p, const R *__restrict__ v,
                                                        const R *__restrict__ vprev, const MinresState *st,
                                                        double *__restrict__ partials) {
    if (skip(st)) return;
    const R a = (R)st->alpha, b = (R)st->beta;
    Acc<R> acc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const R q = p[i] - a * v[i] - b * vprev[i];
        p[i] = q;
        acc.add_prod(q, q);
    }
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_update(long long n, R *__restrict__ p, const R *__restrict__ v,
                                                       const R *__restrict__ w1, R *__restrict__ w2,
                                                       R *__restrict__ x, const MinresState *st) {
    if (st->done_update) return;
    const R d = (R)st->u_delta, e = (R)st->u_eps, ig = (R)st->u_inv_gamma, tau = (R)st->u_tau,
            ib = (R)st->u_inv_beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const R wn = (v[i] - d * w1[i] - e * w2[i]) * ig;
        w2[i] = wn;
        x[i] += tau * wn;
        p[i] *= ib;
    }
}

template <typename R>
__global__ void k_axpby(long long n, R a, const R *__restrict__ x, R b, R *__restrict__ y) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + (b != (R)0 ? b * y[i] : (R)0);
}

template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_norm2(long long n, const R *__restrict__ x, double *partials) {
    Acc<R> acc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc.add_prod(x[i], x[i]);
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// <phi C_m : (E_bar + x)> per Mandel component: partials[c * gridDim.x + block]
template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_mean_stress(long long V, const R *__restrict__ x,
                                                            const R *__restrict__ phi, double lam, double mu2,
                                                            Mac6 mac, double *partials) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        double e[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] = mac.v[c] + (double)x[c * V + i];
        const double ph = (double)phi[i];
        const double tr = lam * (e[0] + e[1] + e[2]);
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += ph * ((c < 3 ? tr : 0.0) + mu2 * e[c]);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const double s = block_sum(acc[c]);
        if (threadIdx.x == 0) partials[c * gridDim.x + blockIdx.x] = s;
    }
}

// total strain and stress in tensor components (shear / sqrt2), stress x Escale
template <typename R>
__global__ void k_fields(long long V, const R *__restrict__ x, const R *__restrict__ phi, R lam, R mu2, R Escale,
                         Mac6 mac, R *__restrict__ strain, R *__restrict__ stress) {
    const R r2 = (R)0.70710678118654752440;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        R e[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] = (R)mac.v[c] + x[c * V + i];
        if (strain) {
#pragma unroll
            for (int c = 0; c < 6; ++c) strain[c * V + i] = (c < 3) ? e[c] : e[c] * r2;
        }
        if (stress) {
            const R ph = phi[i];
            const R tr = lam * (e[0] + e[1] + e[2]);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const R s = Escale * ph * ((c < 3 ? tr : (R)0) + mu2 * e[c]);
                stress[c * V + i] = (c < 3) ? s : s * r2;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Scalar kernels: one CTA, deterministic reduction of the partials, then the
// FP64 recurrences on thread 0.
// ---------------------------------------------------------------------------
__device__ double reduce_partials(const double *partials, int np) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += partials[i];
    return block_sum(s);
}

__global__ void k_reduce_to(const double *partials, int np, double *out) {
    const double s = reduce_partials(partials, np);
    if (threadIdx.x == 0) *out = s;
}

// Set up the solve from ||b||^2: beta_1, phibar_0 = beta_1, c_0 = -1, s_0 = 0,
// delta-bar_1 = 0, epsilon_1 = 0; the v_1 = b / beta_1 scaling is the next kernel.
__global__ void k_scalar_start(MinresState *st, const double *partials, int np, double tol, int max_it) {
    const double b2 = reduce_partials(partials, np);
    if (threadIdx.x != 0) return;
    const double beta1 = sqrt(b2 > 0 ? b2 : 0.0);
    st->beta1 = beta1;
    st->beta = 0.0;     // no v_0 term in the first Lanczos step
    st->alpha = 0.0;
    st->c = -1.0;
    st->s = 0.0;
    st->dbar = 0.0;
    st->eps = 0.0;
    st->phibar = beta1;
    st->tol = tol;
    st->u_delta = st->u_eps = st->u_tau = 0.0;
    st->u_inv_gamma = st->u_inv_beta = 0.0;
    st->est = 1.0;
    st->k = 0;
    st->max_it = max_it;
    st->done = (beta1 == 0.0 || max_it <= 0) ? 1 : 0;
    st->done_update = st->done;
    st->status = isfinite(beta1) ? 0 : -5;
    if (!isfinite(beta1)) { st->done = 1; st->done_update = 1; }
}

__global__ void k_scalar_alpha(MinresState *st, const double *partials, int np) {
    if (st->done) return;
    const double a = reduce_partials(partials, np);
    if (threadIdx.x == 0) st->alpha = a;
}

// Paige-Saunders MINRES step k: apply the previous Givens rotation, form the
// new one, and the coefficients of w_k, x_k and v_{k+1}.
__global__ void k_scalar_givens(MinresState *st, const double *partials, int np) {
    if (st->done) return;
    const double bn2 = reduce_partials(partials, np);
    if (threadIdx.x != 0) return;
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
    st->u_tau = tau;
    st->u_inv_beta = (beta_next > 0.0) ? 1.0 / beta_next : 0.0;
    st->c = cn;
    st->s = sn;
    st->dbar = dbar_next;
    st->eps = eps_next;
    st->phibar = phibar;
    st->beta = beta_next;
    st->k += 1;
    st->est = phibar / st->beta1;
    const bool bad = !isfinite(alpha) || !isfinite(beta_next) || !isfinite(phibar);
    if (bad) {
        st->status = -5;
        st->done = 1;
        st->done_update = 1;        // keep the last finite iterate
        return;
    }
    if (st->est <= st->tol || beta_next == 0.0) {
        st->done = 1;               // this iteration's update still runs
    } else if (st->k >= st->max_it) {
        st->status = 1;
        st->done = 1;
    }
}

// ---------------------------------------------------------------------------
// Conversions and small helpers.
// ---------------------------------------------------------------------------
__global__ void k_f2d(long long n, const float *in, double *out, int acc) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i] + (acc ? out[i] : 0.0);
}
__global__ void k_d2f(long long n, const double *in, float *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
__global__ void __launch_bounds__(kEwThreads) k_residual64(long long n, const double *b, const double *ax, double *r,
                                                           double *partials) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = b[i] - ax[i];
        r[i] = d;
        acc = fma(d, d, acc);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}
template <typename R>
__global__ void k_mandel_scale(long long V, R *f, R s) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * V; i += (long long)gridDim.x * blockDim.x)
        f[3 * V + i] *= s;
}
template <typename R>
__global__ void k_phi_convert(long long V, const void *in, int kind, R *out, int *bad) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        double v;
        if (kind == 0) v = ((const unsigned char *)in)[i] ? 1.0 : 0.0;
        else if (kind == 1) v = (double)((const float *)in)[i];
        else v = ((const double *)in)[i];
        if (!(v >= 0.0 && v <= 1.0)) { atomicExch(bad, 1); v = 0.0; }
        out[i] = (R)v;
    }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
static inline int ew_grid(long long n) {
    long long b = (n + kEwThreads - 1) / kEwThreads;
    return (int)(b < kEwBlocks ? (b > 0 ? b : 1) : kEwBlocks);
}

// The dynamic shared-memory limit of each pass kernel is raised to the
// device's opt-in maximum (a per-function setting shared by all contexts; the
// launch's own size still decides occupancy).
template <typename R>
void Launch<R>::table_init(const Geometry &) {
    int dev = 0, lim = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    lim -= 1024;   // static shared memory of the reductions
    cudaFuncSetAttribute(k_x3_fwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_x3_inv<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_x2<R, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_x2<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_x1<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <typename R>
void Launch<R>::x3_fwd(const Geometry &g, cudaStream_t st, int mode, const R *in, const R *phi, double lam,
                       double mu, const double *macro, cpx<R> *spec, const MinresState *state) {
    Mac6 m{};
    if (macro) for (int c = 0; c < 6; ++c) m.v[c] = macro[c];
    const long long nrows = (long long)g.n1 * g.n2;
    const int grid = (int)((nrows + g.rows3 - 1) / g.rows3);
    k_x3_fwd<R><<<grid, 256, g.smem3, st>>>(g, mode, in, phi, (R)lam, (R)(2.0 * mu), m, spec, state);
}

template <typename R>
void Launch<R>::x2(const Geometry &g, cudaStream_t st, int inverse, cpx<R> *spec, const MinresState *state) {
    const long long total = 6LL * g.n1 * g.h;
    const int grid = (int)((total + g.tile2 - 1) / g.tile2);
    if (inverse) k_x2<R, 1><<<grid, 256, g.smem2, st>>>(g, spec, state);
    else k_x2<R, -1><<<grid, 256, g.smem2, st>>>(g, spec, state);
}

template <typename R>
void Launch<R>::x1(const Geometry &g, cudaStream_t st, int flags, cpx<R> *spec, const MinresState *state) {
    const long long cols = (long long)g.n2 * g.h;
    const int grid = (int)((cols + g.tile1 - 1) / g.tile1);
    k_x1<R><<<grid, 256, g.smem1, st>>>(g, flags, spec, state);
}

template <typename R>
void Launch<R>::x3_inv(const Geometry &g, cudaStream_t st, int mode, const cpx<R> *spec, R *out, double scl,
                       const R *dotv, double *partials, const MinresState *state) {
    const long long nrows = (long long)g.n1 * g.n2;
    const int grid = (int)((nrows + g.rows3 - 1) / g.rows3);
    k_x3_inv<R><<<grid, 256, g.smem3, st>>>(g, mode, spec, out, (R)scl, dotv, partials, state);
}

template <typename R>
void Launch<R>::lanczos(long long n, cudaStream_t st, R *p, const R *v, const R *vprev, const MinresState *state,
                        double *partials) {
    k_lanczos<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, p, v, vprev, state, partials);
}

template <typename R>
void Launch<R>::update(long long n, cudaStream_t st, R *p, const R *v, const R *w1, R *w2, R *x, MinresState *state) {
    k_update<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, p, v, w1, w2, x, state);
}

template <typename R>
void Launch<R>::axpby(long long n, cudaStream_t st, double a, const R *x, double b, R *y) {
    k_axpby<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, (R)a, x, (R)b, y);
}

template <typename R>
void Launch<R>::norm2(long long n, cudaStream_t st, const R *x, double *partials) {
    k_norm2<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, x, partials);
}

template <typename R>
void Launch<R>::mean_stress(long long V, cudaStream_t st, const R *x, const R *phi, double lam, double mu,
                            const double *macro, double *partials) {
    Mac6 m{};
    for (int c = 0; c < 6; ++c) m.v[c] = macro[c];
    k_mean_stress<R><<<ew_grid(V), kEwThreads, 0, st>>>(V, x, phi, lam, 2.0 * mu, m, partials);
}

template <typename R>
void Launch<R>::fields(long long V, cudaStream_t st, const R *x, const R *phi, double lam, double mu, double Escale,
                       const double *macro, R *strain, R *stress) {
    Mac6 m{};
    for (int c = 0; c < 6; ++c) m.v[c] = macro[c];
    k_fields<R><<<ew_grid(V), kEwThreads, 0, st>>>(V, x, phi, (R)lam, (R)(2.0 * mu), (R)Escale, m, strain, stress);
}

template struct Launch<float>;
template struct Launch<double>;

void convert_f2d(long long n, cudaStream_t st, const float *in, double *out, int acc) {
    k_f2d<<<ew_grid(n), kEwThreads, 0, st>>>(n, in, out, acc);
}
void convert_d2f(long long n, cudaStream_t st, const double *in, float *out) {
    k_d2f<<<ew_grid(n), kEwThreads, 0, st>>>(n, in, out);
}
void residual64(long long n, cudaStream_t st, const double *b, const double *ax, double *r, double *partials) {
    k_residual64<<<ew_grid(n), kEwThreads, 0, st>>>(n, b, ax, r, partials);
}
template <typename R>
void mandel_scale(long long V, cudaStream_t st, R *f, double s) {
    k_mandel_scale<R><<<ew_grid(3 * V), kEwThreads, 0, st>>>(V, f, (R)s);
}
template void mandel_scale<float>(long long, cudaStream_t, float *, double);
template void mandel_scale<double>(long long, cudaStream_t, double *, double);
template <typename R>
void phi_convert(long long V, cudaStream_t st, const void *in, int kind, R *out, int *bad) {
    k_phi_convert<R><<<ew_grid(V), kEwThreads, 0, st>>>(V, in, kind, out, bad);
}
template void phi_convert<float>(long long, cudaStream_t, const void *, int, float *, int *);
template void phi_convert<double>(long long, cudaStream_t, const void *, int, double *, int *);

void scalar_start(cudaStream_t st, MinresState *s, const double *partials, int np, double tol, int max_it) {
    k_scalar_start<<<1, 1024, 0, st>>>(s, partials, np, tol, max_it);
}
void scalar_alpha(cudaStream_t st, MinresState *s, const double *partials, int np) {
    k_scalar_alpha<<<1, 1024, 0, st>>>(s, partials, np);
}
void scalar_givens(cudaStream_t st, MinresState *s, const double *partials, int np) {
    k_scalar_givens<<<1, 1024, 0, st>>>(s, partials, np);
}
void reduce_to(cudaStream_t st, const double *partials, int np, double *out) {
    k_reduce_to<<<1, 1024, 0, st>>>(partials, np, out);
}

}  // namespace hom
