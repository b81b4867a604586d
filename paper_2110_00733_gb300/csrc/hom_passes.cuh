// hom_passes.cuh -- the FFT passes of the Galerkin operator and the Krylov
// vector kernels, templated on the field precision R (float or double).
//
// One application of the spectral operator  A^(v) = G F C F^-1 G v  (the
// operator of eq. (linearOp) seen through the DFT) is five passes, each one
// read and one write of the half spectrum:
//   x1(inverse, G on input)   projector of eq. (galop) + inverse along n1
//   x2(inverse)               inverse along n2
//   x3(spec -> spec)          C2R along n3, tau = phi C_m e (Voigt-scaled
//                             isotropic law, section 3.3), R2C along n3;
//                             the real-space fields never reach HBM
//   x2(forward)               forward along n2
//   x1(forward, G on output)  forward along n1 + projector, with the MINRES
//                             dot product <v, A^ v> fused into the store
// Lengths 8..512 that are powers of two use the compile-time register FFT
// (fast_fft); other 2^a 3^b 5^c lengths use the runtime Stockham engine.
#pragma once
#include <math.h>

#include <type_traits>

#include "hom_internal.h"

namespace hom {

// ---------------------------------------------------------------------------
// Reductions.
// ---------------------------------------------------------------------------

// Per-thread accumulator of products: float-float (error-free product and a
// compensated sum, ~44 significant bits) for FP32 data, plain FP64 for FP64
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

// Sum over the block in a fixed order; the result is valid in thread 0.
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
// load case c of a stacked batch (state points to g.nb states, or is null)
__device__ __forceinline__ bool skip_case(const MinresState *s, int c) { return s != nullptr && s[c].done; }

// true in every thread of the last CTA of a group of `count`; all threads
// of the CTA call it after thread 0 wrote the CTA's partial
__device__ __forceinline__ bool last_of(int *cnt, int count) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();   // the partial is visible before the count
        s_last = atomicAdd(cnt, 1) == count - 1;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// fixed-order sum of count partials written by other CTAs (read at L2)
__device__ __forceinline__ double sum_partials(const double *part, int count) {
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) v += __ldcg(part + i);
    return block_sum(v);
}

// Parseval weight of the half-spectrum plane k3
__device__ __forceinline__ int pweight(int k3, int n3) { return (k3 == 0 || 2 * k3 == n3) ? 1 : 2; }

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

// The projector of eq. (galop) at one frequency, split into the part that
// depends on the frequency only (mode and unit vector e = xi / |xi|) and its
// application, so that a pass projecting two tensors at the same frequency
// builds xi once.  mode 0: G = 0 (a Nyquist index, or xi = 0 numerically);
// 1: the projection; 2: xi = 0 (the identity on the stress-controlled
// components g.mask0, zero on the others).
template <typename R> struct GammaE {
    cpx<R> e0, e1, e2;
    int mode;
};

template <typename R>
__device__ __forceinline__ GammaE<R> gamma_e(const Geometry &g, int k1, int k2, int k3) {
    GammaE<R> q;
    q.mode = 0;
    if (k1 == 0 && k2 == 0 && k3 == 0) {
        q.mode = 2;
        return q;
    }
    const bool nyq = ((g.n1 & 1) == 0 && 2 * k1 == g.n1) || ((g.n2 & 1) == 0 && 2 * k2 == g.n2) ||
                     ((g.n3 & 1) == 0 && 2 * k3 == g.n3);
    if (nyq) return q;
    const cpx<R> *D0 = reinterpret_cast<const cpx<R> *>(g.D[0]);
    const cpx<R> *D1 = reinterpret_cast<const cpx<R> *>(g.D[1]);
    const cpx<R> *D2 = reinterpret_cast<const cpx<R> *>(g.D[2]);
    const cpx<R> *M0 = reinterpret_cast<const cpx<R> *>(g.M[0]);
    const cpx<R> *M1 = reinterpret_cast<const cpx<R> *>(g.M[1]);
    const cpx<R> *M2 = reinterpret_cast<const cpx<R> *>(g.M[2]);
    const cpx<R> m0 = __ldg(&M0[k1]), m1 = __ldg(&M1[k2]), m2 = __ldg(&M2[k3]);
    // xi_p = D_p(k_p) prod_{r != p} M_r(k_r): N_p (e^{iq_p} - 1) prod (1 + e^{iq_r})/2
    // for the rotated scheme of eq. (freqrot), i q_p N_p for eq. (freq)
    const cpx<R> x0 = mul<R>(__ldg(&D0[k1]), mul<R>(m1, m2));
    const cpx<R> x1 = mul<R>(__ldg(&D1[k2]), mul<R>(m0, m2));
    const cpx<R> x2 = mul<R>(__ldg(&D2[k3]), mul<R>(m0, m1));
    const R n2 = x0.x * x0.x + x0.y * x0.y + x1.x * x1.x + x1.y * x1.y + x2.x * x2.x + x2.y * x2.y;
    if (!(n2 > (R)0)) return q;
    const R inv = (R)1 / sqrt(n2);
    q.e0 = scale<R>(x0, inv);
    q.e1 = scale<R>(x1, inv);
    q.e2 = scale<R>(x2, inv);
    q.mode = 1;
    return q;
}

// Orthogonal projection of a symmetric tau (Mandel, t[6], overwritten) onto
// {sym(u (x) e)}, |e| = 1: sym(u (x) e) with u = 2 tau conj(e) - e (conj(e) .
// tau conj(e)) (Sherman-Morrison inverse of the acoustic tensor 1/2 (I + e e^H)).
template <typename R>
__device__ __forceinline__ void gamma_apply(const Geometry &g, const GammaE<R> &q, cpx<R> *t) {
    if (q.mode != 1) {
#pragma unroll
        for (int c = 0; c < 6; ++c)
            if (q.mode == 0 || !((g.mask0 >> c) & 1)) t[c] = mk<R>(0, 0);
        return;
    }
    const cpx<R> e0 = q.e0, e1 = q.e1, e2 = q.e2;
    const cpx<R> c0 = conjc<R>(e0), c1 = conjc<R>(e1), c2 = conjc<R>(e2);
    const R r2 = (R)0.70710678118654752440;   // 1/sqrt(2)
    const cpx<R> T11 = t[0], T22 = t[1], T33 = t[2];
    const cpx<R> T23 = scale<R>(t[3], r2), T13 = scale<R>(t[4], r2), T12 = scale<R>(t[5], r2);
    const cpx<R> v0 = add<R>(add<R>(mul<R>(T11, c0), mul<R>(T12, c1)), mul<R>(T13, c2));
    const cpx<R> v1 = add<R>(add<R>(mul<R>(T12, c0), mul<R>(T22, c1)), mul<R>(T23, c2));
    const cpx<R> v2 = add<R>(add<R>(mul<R>(T13, c0), mul<R>(T23, c1)), mul<R>(T33, c2));
    const cpx<R> sc = add<R>(add<R>(mul<R>(c0, v0), mul<R>(c1, v1)), mul<R>(c2, v2));
    const cpx<R> u0 = sub<R>(scale<R>(v0, (R)2), mul<R>(e0, sc));
    const cpx<R> u1 = sub<R>(scale<R>(v1, (R)2), mul<R>(e1, sc));
    const cpx<R> u2 = sub<R>(scale<R>(v2, (R)2), mul<R>(e2, sc));
    t[0] = mul<R>(u0, e0);
    t[1] = mul<R>(u1, e1);
    t[2] = mul<R>(u2, e2);
    t[3] = scale<R>(add<R>(mul<R>(u1, e2), mul<R>(u2, e1)), r2);
    t[4] = scale<R>(add<R>(mul<R>(u0, e2), mul<R>(u2, e0)), r2);
    t[5] = scale<R>(add<R>(mul<R>(u0, e1), mul<R>(u1, e0)), r2);
}

// G at frequency (k1,k2,k3) on the 6 Mandel components at p[0..5] (stride 1)
template <typename R>
__device__ __forceinline__ void gamma_at(const Geometry &g, int k1, int k2, int k3, cpx<R> *t) {
    const GammaE<R> q = gamma_e<R>(g, k1, k2, k3);
    gamma_apply<R>(g, q, t);
}

// Run the transform of the L lines in buf.  Fast engine: in place, returns
// buf.  Generic engine: ping-pong with buf2, returns the buffer holding the
// result.
// nsync != 0 (fast engine only): the first nsync threads run it on named
// barrier 1.
template <typename R, int S, int NF, int PAD = 0, typename Plan = FastPlan<NF>>
__device__ __forceinline__ cpx<R> *run_fft(cpx<R> *buf, cpx<R> *buf2, int L, int ES, const AxisPlan &p, int nsync = 0) {
    if constexpr (NF > 0) {
        fast_fft<R, S, NF, PAD, Plan>(buf, L, ES, reinterpret_cast<const cpx<R> *>(p.tw), nsync);
        return buf;
    } else {
        return fft_lines<R, S>(buf, buf2, L, ES, p);
    }
}

// Six adjacent complex values (one frequency, or one k of a row) as 16-byte
// accesses: pairs (2p, 2p+1) for FP32, single values for FP64.
template <typename R> struct Six;
template <> struct Six<float> {
    __device__ static void load_pair(const float2 *src, int p, float2 &a, float2 &b) {
        const float4 v = reinterpret_cast<const float4 *>(src)[p];
        a = make_float2(v.x, v.y);
        b = make_float2(v.z, v.w);
    }
    __device__ static void store_pair(float2 *dst, int p, float2 a, float2 b) {
        reinterpret_cast<float4 *>(dst)[p] = make_float4(a.x, a.y, b.x, b.y);
    }
};
template <> struct Six<double> {
    __device__ static void load_pair(const double2 *src, int p, double2 &a, double2 &b) {
        a = src[2 * p];
        b = src[2 * p + 1];
    }
    __device__ static void store_pair(double2 *dst, int p, double2 a, double2 b) {
        dst[2 * p] = a;
        dst[2 * p + 1] = b;
    }
};

// Register cap of the pass kernels: FP32 kernels are held to 64 registers
// (two 512-thread CTAs' worth per SM) so that more CTAs stay resident to hide
// HBM latency; FP64 kernels keep their data in registers instead.
#define HOM_PASS_BOUNDS(R) __launch_bounds__(512, sizeof(R) == 4 ? 2 : 1)
// the same, except for the register FFT lengths with more than 16 elements
// per thread (160: 20), which keep their elements in registers instead
#define HOM_PASS_BOUNDS_NF(R, NF) __launch_bounds__(512, (sizeof(R) == 4 && fast_elems(NF) <= 16) ? 2 : 1)
// the n3 pass, by its own plan's elements per thread
#define HOM_PASS_BOUNDS_N3(R, NF) __launch_bounds__(512, (sizeof(R) == 4 && fast_elems_n3(NF) <= 16) ? 2 : 1)

// ---------------------------------------------------------------------------
// n3 pass.  A CTA owns rows (k1,k2) [row0, row0+rows3); lines are the three
// component pairs (2p, 2p+1) of each row packed as one complex line
// Z = X_2p + i X_2p+1, line index p*rows3 + r.
// ---------------------------------------------------------------------------
template <typename R, int NF, int NP>
__global__ void HOM_PASS_BOUNDS_N3(R, NF) k_x3(Geometry g, int in_mode, const void *__restrict__ in_, int mid, R lam,
                                        R mu2, Mac6 mac, R scl, int out_mode, void *__restrict__ out_,
                                        const R *__restrict__ phi, const MinresState *state,
                                        double *__restrict__ epart, Fold fold, double *__restrict__ tsum) {
    pdl_release();
    pdl_wait();   // predecessor complete (programmatic launch in the MINRES graph)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // element stride ES = L rounded up to odd: the per-element phases below
    // stride by ES across a warp and stay free of bank conflicts; the fast
    // engine also skips one slot every 16 elements (PAD)
    constexpr int PAD = NF > 0 ? 1 : 0;
    constexpr int NC = 2 * NP;   // components per frequency
    const int N = g.n3, ROWS = g.rows3, L = NP * ROWS, ES = L | 1, H = g.h;
    auto ep = [ES](int e) { return epos<PAD>(e, ES); };
    cpx<R> *buf = reinterpret_cast<cpx<R> *>(smem_raw);
    cpx<R> *buf2 = buf + ep(N);   // second buffer of the generic engine only
    const int nrows = g.n1 * g.n2;
    // a CTA never straddles two load cases of a stacked batch
    const int bpc = (nrows + ROWS - 1) / ROWS;
    const int cs = blockIdx.x / bpc;
    if (skip_case(state, cs)) return;
    const int row0 = (blockIdx.x - cs * bpc) * ROWS;   // row within the case
    const int V = (int)g.V;
    const int nr = min(ROWS, nrows - row0);
    // stacked cases: spectrum rows and (real input / output) fields of case cs
    if (in_mode == X3_IN_SPEC) in_ = reinterpret_cast<const cpx<R> *>(in_) + (size_t)cs * nrows * H * NC;
    else if (in_mode == X3_IN_REAL) in_ = reinterpret_cast<const R *>(in_) + (size_t)cs * 6 * g.V;
    if (out_mode == X3_OUT_SPEC) out_ = reinterpret_cast<cpx<R> *>(out_) + (size_t)cs * nrows * H * NC;
    else out_ = reinterpret_cast<R *>(out_) + (size_t)cs * 6 * g.V;
    // ---- input
    if (in_mode == X3_IN_SPEC) {
        // Z[k] = X_a[k] + i X_b[k] and Z[N-k] = conj X_a[k] + i conj X_b[k];
        // the self-conjugate bins keep their real parts, as a C2R does
        const cpx<R> *spec = reinterpret_cast<const cpx<R> *>(in_);
        for (int r = 0; r < ROWS; ++r) {
            const cpx<R> *row = spec + (size_t)(row0 + r) * H * NC;
            for (int k = threadIdx.x; k < H; k += blockDim.x) {
                const bool selfc = (k == 0) || (2 * k == N);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    cpx<R> xa = mk<R>(0, 0), xb = mk<R>(0, 0);
                    if (r < nr) Six<R>::load_pair(row + NC * k, p, xa, xb);
                    if (selfc) { xa.y = 0; xb.y = 0; }
                    buf[ep(k) + p * ROWS + r] = mk<R>(xa.x - xb.y, xa.y + xb.x);
                    if (!selfc) buf[ep(N - k) + p * ROWS + r] = mk<R>(xa.x + xb.y, xb.x - xa.y);
                }
            }
        }
        __syncthreads();
        cpx<R> *res = run_fft<R, 1, NF, PAD, PlanN3<R, NF>>(buf, buf2, L, ES, g.ax[2]);
        if (res != buf) {   // generic engine ended in the second buffer
            for (int i = threadIdx.x; i < N * ES; i += blockDim.x) buf[i] = res[i];
            __syncthreads();
        }
    } else {
        const R *real = reinterpret_cast<const R *>(in_);
        for (int r = 0; r < ROWS; ++r) {
            const int vbase = (row0 + r) * N;
            for (int e = threadIdx.x; e < N; e += blockDim.x) {
                R t[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    t[c] = (r >= nr || c >= 6) ? (R)0
                                               : (in_mode == X3_IN_MACRO ? (R)mac.v[c] : real[c * V + vbase + e]);
#pragma unroll
                for (int p = 0; p < NP; ++p) buf[ep(e) + p * ROWS + r] = mk<R>(t[2 * p], t[2 * p + 1]);
            }
        }
        __syncthreads();
    }
    // ---- scaling and material law on the real-space values
    const R s_in = (in_mode == X3_IN_SPEC) ? (R)(1.0 / (double)g.V) : (R)1;
    const R s_all = s_in * scl;
    // strain energy sum_x e : C : e of the real-space input (epart): with
    // e = F^-1 G u this is <u, A^ u> / V, the MINRES alpha numerator, so the
    // n1 pass needs no dot product with u
    R en = 0;   // non-negative terms: a short per-thread sum in R is accurate to ~1e-6
    double ts[6] = {0, 0, 0, 0, 0, 0};   // stress sums (tsum)
    for (int r = 0; r < nr; ++r) {
        const int vbase = (row0 + r) * N;
        for (int e = threadIdx.x; e < N; e += blockDim.x) {
            cpx<R> *q = buf + ep(e) + r;
            R t[NC];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const cpx<R> z = q[p * ROWS];
                t[2 * p] = z.x * s_all;
                t[2 * p + 1] = z.y * s_all;
            }
            if (mid == X3_MID_MATERIAL || mid == X3_MID_MODB) {
                const R ph = phi[vbase + e];
                const R sum = t[0] + t[1] + t[2];
                const R tr = lam * sum;
                if (epart) {
                    R ee = t[0] * t[0];
#pragma unroll
                    for (int c = 1; c < 6; ++c) ee += t[c] * t[c];
                    en += ph * (tr * sum + mu2 * ee);
                }
#pragma unroll
                for (int c = 0; c < 6; ++c) t[c] = ph * ((c < 3 ? tr : (R)0) + mu2 * t[c]);
                if (tsum) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) ts[c] += (double)t[c];
                }
                if constexpr (NC == 10) {
                    // MoDBFFT penalty vector on the empty phase: chi_v g, eq. (modbfftfop)
                    const R chi = (ph == (R)0) ? (R)1 : (R)0;
                    t[6] *= chi;
                    t[7] *= chi;
                    t[8] *= chi;
                    t[9] = 0;
                }
            }
            if (out_mode == X3_OUT_REAL) {
                R *real = reinterpret_cast<R *>(out_);
#pragma unroll
                for (int c = 0; c < 6; ++c) real[c * V + vbase + e] = t[c];   // (NC == 6 only)
            } else {
#pragma unroll
                for (int p = 0; p < NP; ++p) q[p * ROWS] = mk<R>(t[2 * p], t[2 * p + 1]);
            }
        }
    }
    if (tsum) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double sum = block_sum(ts[c]);
            if (threadIdx.x == 0) tsum[(size_t)c * gridDim.x + blockIdx.x] = sum;
        }
    }
    if (epart) {
        const double sum = block_sum((double)en);
        if (threadIdx.x == 0) epart[blockIdx.x] = sum;
        if (fold.cnt && last_of(fold.cnt + cs, bpc)) {   // alpha of case cs
            const double tot = sum_partials(epart + (size_t)cs * bpc, bpc);
            if (threadIdx.x == 0) {
                alpha_step(fold.st + cs, tot, fold.scale);
                fold.cnt[cs] = 0;
            }
        }
    }
    if (out_mode == X3_OUT_REAL) return;
    // rows beyond nrows hold zeros already (their inputs were zero)
    __syncthreads();
    cpx<R> *res = run_fft<R, -1, NF, PAD, PlanN3<R, NF>>(buf, buf2, L, ES, g.ax[2]);
    // unpack the two real transforms of each packed line:
    //   X_a[k] = (Z[k] + conj Z[N-k]) / 2,  X_b[k] = (Z[k] - conj Z[N-k]) / (2i)
    cpx<R> *spec = reinterpret_cast<cpx<R> *>(out_);
    for (int r = 0; r < nr; ++r) {
        cpx<R> *row = spec + (size_t)(row0 + r) * H * NC;
        for (int k = threadIdx.x; k < H; k += blockDim.x) {
            const int km = (k == 0) ? 0 : N - k;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const cpx<R> z = res[ep(k) + p * ROWS + r];
                const cpx<R> zm = conjc<R>(res[ep(km) + p * ROWS + r]);
                Six<R>::store_pair(row + NC * k, p, mk<R>((R)0.5 * (z.x + zm.x), (R)0.5 * (z.y + zm.y)),
                                   mk<R>((R)0.5 * (z.y - zm.y), (R)-0.5 * (z.x - zm.x)));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Register-resident n3 pass (FP32, n3 in {64, 128, 256}, 6-component spectra,
// spectrum in and out): the C2R of a row, the material law with the strain-
// energy sums, and the R2C, with the row's data in registers.
//
// A row is handled by P lanes of one warp; lane j owns the elements j + P m,
// m < Q, of the three packed lines Z_p = X_2p + i X_2p+1 (N = P Q).  Each
// transform is two radix stages held in registers -- a length-Q DFT over m,
// a twiddle, a transpose through a padded per-row shared-memory slab, and
// length-P DFTs of Q/P columns -- after which lane j again owns the
// elements j + P m (the inverse maps frequencies j + P m to voxels j + P m,
// the forward voxels to frequencies).  The other half of the Hermitian
// spectrum (Z[N-k] from X[k]) and the unpacking of the result come from the
// partner lane P - j by warp shuffles.  The law needs all six components of
// a voxel, which lane j holds.
//
// Persistent and warp-independent: each warp takes groups of 32 / P
// consecutive rows (one contiguous block of the stacked spectrum) in turn.
// The group's rows and phi come from a per-warp shared-memory buffer, filled
// by cp.async while the warp computes the previous group's R2C and stores
// it, so the HBM latency is off the warp's critical path.  Only warp-level
// synchronisation is used until the final energy reduction.
// ---------------------------------------------------------------------------
template <int N> struct X3RPlan;
template <> struct X3RPlan<64>  { static constexpr int P = 8,  Q = 8,  ROWS = 16; };
template <> struct X3RPlan<128> { static constexpr int P = 8,  Q = 16, ROWS = 16; };
template <> struct X3RPlan<256> { static constexpr int P = 16, Q = 16, ROWS = 8; };


template <int P>
__device__ __forceinline__ float2 shfl_partner(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// stage 2 of a transform: lane t takes the Q/P columns t + P i of the slab
// (line p), a length-P DFT each, and returns element i + (Q/P) n of
// column i's output n in z[i + (Q/P) n]
template <int S, int P, int Q>
__device__ __forceinline__ void x3r_stage2(const float2 *slab, int t, float2 (&z)[Q]) {
    constexpr int C = Q / P;
#pragma unroll
    for (int i = 0; i < C; ++i) {
        float2 v[P];
        const float2 *col = slab + (t + P * i) * (P + 1);
#pragma unroll
        for (int k = 0; k < P; ++k) v[k] = col[k];
        dft<float, S, P>(v);
#pragma unroll
        for (int n = 0; n < P; ++n) z[i + C * n] = v[n];
    }
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// a twiddle factor, loaded where it is used (volatile: not hoisted out of
// the persistent loop, where the 2 Q of them would stay live in registers)
__device__ __forceinline__ float2 tw_load(const float2 *p) {
    float2 v;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

template <int N>
__global__ void __launch_bounds__(kX3rWarps * 32, N == 64 ? 5 : 3)
    k_x3r(Geometry g, const float2 *__restrict__ in, float2 *__restrict__ out, int material, float lam, float mu2,
          const float *__restrict__ phi, const MinresState *state, double *__restrict__ epart, Fold fold) {
    pdl_release();
    pdl_wait();   // predecessor complete (programmatic launch in the MINRES graph)
    using PL = X3RPlan<N>;
    constexpr int P = PL::P, Q = PL::Q, H = N / 2 + 1, NC = 6;
    constexpr int RW = 32 / P;                  // rows per warp group
    constexpr int TS = Q * (P + 1);             // one line's transpose slab
    static_assert(P == x3r_row_lanes(N) && TS == (int)x3r_slab_elems(N), "x3r layout");
    extern __shared__ __align__(16) unsigned char x3r_smem_raw[];
    __shared__ double sacc[kNbMax * kX3rWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rw = lane / P, j = lane % P;
    unsigned char *wbase = x3r_smem_raw + (size_t)warp * x3r_warp_bytes(N);
    // per warp: [rows of the group | one slab per row | phi]; the inverse
    // transform, which runs between reading the rows and prefetching the next
    // group, transposes its three lines at once through 3 RW slabs laid over
    // the first two regions
    float2 *inb = reinterpret_cast<float2 *>(wbase);                               // RW rows x H x 6
    float2 *tb = reinterpret_cast<float2 *>(wbase + x3r_in_bytes(N)) + rw * TS;    // the forward's slab
    float *phb = reinterpret_cast<float *>(wbase + x3r_in_bytes(N) + (size_t)RW * TS * sizeof(float2));
    float2 *tb3 = reinterpret_cast<float2 *>(wbase) + rw * TS;                     // line p at tb3 + p RW TS
    static_assert(2 * RW * TS * sizeof(float2) <= x3r_in_bytes(N), "three inverse slabs over rows + slab");
    const int nrows = g.n1 * g.n2;
    const int gpc = nrows / RW;                  // row groups per case (nrows is a multiple of RW)
    const int ngroups = gpc * g.nb;
    const int gstride = gridDim.x * kX3rWarps;
    if (threadIdx.x < kNbMax * kX3rWarps) sacc[threadIdx.x] = 0.0;
    __syncthreads();
    auto live_from = [&](int q) {
        while (q < ngroups && skip_case(state, q / gpc)) q += gstride;
        return q;
    };
    // the group's rows (contiguous) and, with the law, its phi rows
    auto prefetch = [&](int q) {
        const int cs = q / gpc, rowc = (q - cs * gpc) * RW;
        const char *src = reinterpret_cast<const char *>(in + ((size_t)cs * nrows + rowc) * H * NC);
        constexpr int nin = (int)(x3r_in_bytes(N) / 16);
#pragma unroll 1
        for (int i = lane; i < nin; i += 32) cp_async16(reinterpret_cast<char *>(inb) + 16 * i, src + 16 * i);
        if (material && x3r_phi_prefetch(N)) {
            const char *ps = reinterpret_cast<const char *>(phi + (size_t)rowc * N);
            constexpr int nph = (int)(x3r_phi_bytes(N) / 16);
#pragma unroll 1
            for (int i = lane; i < nph; i += 32) cp_async16(reinterpret_cast<char *>(phb) + 16 * i, ps + 16 * i);
        }
        cp_async_commit();
    };
    const float2 *tw = reinterpret_cast<const float2 *>(g.ax[2].tw);   // exp(-2 pi i t / N)
    const int lane0 = lane & ~(P - 1);
    const int partner = lane0 + ((P - j) & (P - 1));
    const float sV = 1.0f / (float)g.V;
    int q = live_from(blockIdx.x * kX3rWarps + warp);
    if (q < ngroups) prefetch(q);
    while (q < ngroups) {
        const int qn = live_from(q + gstride);
        const int cs = q / gpc;
        const size_t row = (size_t)cs * nrows + (size_t)(q - cs * gpc) * RW + rw;   // row of the stacked spectrum
        cp_async_wait_all();
        __syncwarp();
        // this group's twiddle row j (opaque to the compiler, so that the Q
        // twiddle addresses are formed here, not kept live across the loop)
        const float2 *twj;
        asm volatile("mov.b64 %0, %1;" : "=l"(twj) : "l"(tw + j));
        float2 z[3][Q];
        // ---- input, one line at a time: own frequencies k = j + P m <= N/2
        // (m < Q/2, and m = Q/2 for j = 0); the upper half m > Q/2 (and m = Q/2
        // for j != 0) is Z[j + P m] = Zc[N - j - P m], held by the partner at
        // m' = Q - 1 - m (by lane 0 itself at Q - m)
        const float2 *rp = inb + (size_t)rw * H * NC;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            float2 zc[Q / 2 + 1];   // conj X_a[k] + i conj X_b[k] = Z[N - k], for the partner
#pragma unroll
            for (int m = 0; m <= Q / 2; ++m) {
                const int k = j + P * m;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (m < Q / 2 || j == 0) v = reinterpret_cast<const float4 *>(rp + NC * k)[p];
                if (k == 0 || 2 * k == N) { v.y = 0.f; v.w = 0.f; }   // self-conjugate bins: real parts
                // a = (v.x, v.y), b = (v.z, v.w): Z = a + i b, Zc = conj a + i conj b
                z[p][m] = make_float2(v.x - v.w, v.y + v.z);
                zc[m] = make_float2(v.x + v.w, v.z - v.y);
            }
#pragma unroll
            for (int s = 0; s < Q / 2; ++s) {
                const float2 got = shfl_partner<P>(zc[s], partner);
                const int m = Q - 1 - s;
                z[p][m] = (j == 0) ? (m > Q / 2 ? zc[Q - m] : z[p][m]) : got;
            }
        }
        // ---- inverse transform (C2R part of eq. linearOp): the three
        // lines' transposes at once, over the rows just read
        __syncwarp();
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            dft<float, 1, Q>(z[p]);
#pragma unroll
            for (int n = 0; n < Q; ++n) {
                float2 w = tw_load(twj + (j * n - j));
                w.y = -w.y;
                tb3[p * RW * TS + n * (P + 1) + j] = mul<float>(z[p][n], w);
            }
        }
        __syncwarp();
#pragma unroll
        for (int p = 0; p < 3; ++p) x3r_stage2<1, P, Q>(tb3 + p * RW * TS, j, z[p]);
        __syncwarp();
        // ---- material law on voxels j + P m (scaled by 1/V), strain energy
        float en = 0.f;
        if (material) {
            const float *ph_row = x3r_phi_prefetch(N) ? phb + rw * N
                                                      : phi + ((size_t)(q - cs * gpc) * RW + rw) * N;
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                const float ph = x3r_phi_prefetch(N) ? ph_row[j + P * m] : __ldg(&ph_row[j + P * m]);
                float t[6];
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    t[2 * p] = z[p][m].x * sV;
                    t[2 * p + 1] = z[p][m].y * sV;
                }
                const float sum = t[0] + t[1] + t[2];
                const float tr = lam * sum;
                float ee = t[0] * t[0];
#pragma unroll
                for (int c = 1; c < 6; ++c) ee += t[c] * t[c];
                en += ph * (tr * sum + mu2 * ee);
#pragma unroll
                for (int c = 0; c < 6; ++c) t[c] = ph * ((c < 3 ? tr : 0.f) + mu2 * t[c]);
#pragma unroll
                for (int p = 0; p < 3; ++p) z[p][m] = make_float2(t[2 * p], t[2 * p + 1]);
            }
        } else {
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int m = 0; m < Q; ++m) z[p][m] = make_float2(z[p][m].x * sV, z[p][m].y * sV);
        }
        // the buffer is read: bring in the next group while this one finishes
        __syncwarp();
        if (qn < ngroups) prefetch(qn);
        // ---- forward transform (R2C)
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            dft<float, -1, Q>(z[p]);
#pragma unroll
            for (int n = 0; n < Q; ++n) tb[n * (P + 1) + j] = mul<float>(z[p][n], tw_load(twj + (j * n - j)));
            __syncwarp();
            x3r_stage2<-1, P, Q>(tb, j, z[p]);
            __syncwarp();
        }
        // ---- unpack and store own frequencies k = j + P m <= N/2:
        //   X_a[k] = (W[k] + conj W[N-k]) / 2,  X_b[k] = (W[k] - conj W[N-k]) / (2i),
        //   W[N-k] from the partner's register Q - 1 - m (lane 0: its own Q - m)
        float2 *op = out + row * H * NC;
#pragma unroll
        for (int m = 0; m <= Q / 2; ++m) {
            float2 wm[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const float2 got = shfl_partner<P>(z[p][(Q - 1 - m + Q) % Q], partner);
                wm[p] = (j == 0) ? z[p][(Q - m) % Q] : got;
            }
            const int k = j + P * m;
            if (m < Q / 2 || j == 0) {
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    const float2 w = z[p][m % Q];
                    const float2 c = make_float2(wm[p].x, -wm[p].y);
                    reinterpret_cast<float4 *>(op + NC * k)[p] =
                        make_float4(0.5f * (w.x + c.x), 0.5f * (w.y + c.y), 0.5f * (w.y - c.y), -0.5f * (w.x - c.x));
                }
            }
        }
        if (epart) {
            const double ws = warp_sum((double)en);
            if (lane == 0) sacc[cs * kX3rWarps + warp] += ws;
        }
        q = qn;
    }
    cp_async_wait_all();
    if (epart) {
        __syncthreads();
        if (threadIdx.x < g.nb) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < kX3rWarps; ++w) t += sacc[threadIdx.x * kX3rWarps + w];
            epart[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = t;   // = epart[case * grid + block]
        }
        if (fold.cnt && last_of(fold.cnt, gridDim.x)) {   // alpha of every case
            for (int cc = 0; cc < g.nb; ++cc) {
                const double tot = sum_partials(epart + (size_t)cc * gridDim.x, gridDim.x);
                if (threadIdx.x == 0) alpha_step(fold.st + cc, tot, fold.scale);
            }
            if (threadIdx.x == 0) fold.cnt[0] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// n2 pass, in place.  Columns are (k1, k3, c) flattened, f = k1 * 6h + q;
// element k2 of column f is at (k1 n2 + k2) 6h + q.  tile2 consecutive
// columns per CTA (contiguous runs of tile2 complex values).
// ---------------------------------------------------------------------------
template <typename R, int S, int NF>
__global__ void HOM_PASS_BOUNDS_NF(R, NF) k_x2(Geometry g, cpx<R> *__restrict__ spec, const MinresState *state) {
    pdl_release();
    pdl_wait();   // predecessor complete (programmatic launch in the MINRES graph)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int N = g.n2, T = g.tile2, H6 = g.nc * g.h;
    cpx<R> *buf = reinterpret_cast<cpx<R> *>(smem_raw);
    cpx<R> *buf2 = buf + N * T;
    const int total = g.n1 * g.nb * H6;   // stacked cases along k1
    const int t = threadIdx.x % T, e0 = threadIdx.x / T, es = blockDim.x / T;
    const int f = blockIdx.x * T + t;
    const bool live = f < total && !skip_case(state, f / (g.n1 * H6));
    const int k1 = live ? f / H6 : 0;
    cpx<R> *col = spec + (size_t)k1 * N * H6 + (f - k1 * H6);   // element e at col[e * H6]
    for (int e = e0; e < N; e += es) buf[e * T + t] = live ? col[(size_t)e * H6] : mk<R>(0, 0);
    __syncthreads();
    cpx<R> *res = run_fft<R, S, NF>(buf, buf2, T, T, g.ax[1]);
    if (live)
        for (int e = e0; e < N; e += es) col[(size_t)e * H6] = res[e * T + t];
}

// ---------------------------------------------------------------------------
// n1 pass.  Columns are (k2, k3) flattened, g = k2 h + k3; tile1 consecutive
// columns per CTA with all 6 components: line l = t*6 + c (so that a row of
// the tile is one contiguous run of 6 tile1 complex values).
// ---------------------------------------------------------------------------
template <typename R, int NF>
__global__ void HOM_PASS_BOUNDS_NF(R, NF) k_x1(Geometry g, int flags, const cpx<R> *__restrict__ in,
                                            cpx<R> *__restrict__ out, const cpx<R> *__restrict__ dotv,
                                            double *__restrict__ partials, const MinresState *state) {
    if (skip(state)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int NC = g.nc, N = g.n1, T = g.tile1, H = g.h, L = NC * T;
    cpx<R> *buf = reinterpret_cast<cpx<R> *>(smem_raw);
    cpx<R> *buf2 = buf + N * L;
    const int cols = g.n2 * H;
    const int g0 = blockIdx.x * T;
    const size_t sK1 = (size_t)cols * NC;   // stride between consecutive k1
    // each thread keeps one line l (blockDim is a multiple of L)
    const int lt = threadIdx.x % L, e0 = threadIdx.x / L, es = blockDim.x / L;
    const int tl = lt / NC;
    const bool live = g0 + tl < cols;
    {
        const cpx<R> *src = in + (size_t)g0 * NC + lt;
        for (int e = e0; e < N; e += es) buf[e * L + lt] = live ? src[e * sK1] : mk<R>(0, 0);
    }
    __syncthreads();
    // projector on whole frequencies: thread keeps one column t (blockDim % T == 0)
    const int tg = threadIdx.x % T, eg0 = threadIdx.x / T, egs = blockDim.x / T;
    const int colg = g0 + tg;
    const int k2g = colg / H, k3g = colg - k2g * H;
    if (flags & X1_GAMMA_IN) {
        if (colg < cols)
            for (int e = eg0; e < N; e += egs) gamma_at<R>(g, e, k2g, k3g, buf + e * L + tg * NC);
        __syncthreads();
    }
    cpx<R> *res = (flags & X1_FWD) ? run_fft<R, -1, NF>(buf, buf2, L, L, g.ax[0])
                                   : run_fft<R, 1, NF>(buf, buf2, L, L, g.ax[0]);
    if (flags & X1_GAMMA_OUT) {
        if (colg < cols)
            for (int e = eg0; e < N; e += egs) gamma_at<R>(g, e, k2g, k3g, res + e * L + tg * NC);
        __syncthreads();
    }
    Acc<R> acc;
    if (live) {
        const int colt = g0 + tl;
        const int k3 = colt - (colt / H) * H;
        const R w = (R)pweight(k3, g.n3);
        cpx<R> *dst = out + (size_t)g0 * NC + lt;
        const cpx<R> *dv = dotv + (size_t)g0 * NC + lt;
        for (int e = e0; e < N; e += es) {
            const cpx<R> z = res[e * L + lt];
            dst[e * sK1] = z;
            if (flags & X1_DOT) {
                const cpx<R> d = dv[e * sK1];
                acc.add_prod(w * z.x, d.x);
                acc.add_prod(w * z.y, d.y);
            }
        }
    }
    if (flags & X1_DOT) {
        const double s = block_sum(acc.value());
        if (threadIdx.x == 0) partials[blockIdx.x] = s;
    }
}

// A TMA box dimension holds at most 256 elements: a tile of n > 256 rows
// (n = 512) moves as consecutive boxes of 256 rows; rowb is the bytes of one
// row of the tile in shared memory.
constexpr int kBoxRows = 256;
__device__ __forceinline__ void tma_load_rows_3d(void *dst, const CUtensorMap *tm, int x, int n, int z, int rowb,
                                                 uint64_t *bar) {
    for (int y0 = 0; y0 < n; y0 += kBoxRows) tma_load_3d((char *)dst + (size_t)y0 * rowb, tm, x, y0, z, bar);
}
__device__ __forceinline__ void tma_store_rows_3d(const CUtensorMap *tm, int x, int n, int z, const void *src, int rowb) {
    for (int y0 = 0; y0 < n; y0 += kBoxRows) tma_store_3d(tm, x, y0, z, (const char *)src + (size_t)y0 * rowb);
}
__device__ __forceinline__ void tma_load_rows_2d(void *dst, const CUtensorMap *tm, int x, int y, int n, int rowb,
                                                 uint64_t *bar) {
    for (int y0 = 0; y0 < n; y0 += kBoxRows) tma_load_2d((char *)dst + (size_t)y0 * rowb, tm, x, y + y0, bar);
}
__device__ __forceinline__ void tma_store_rows_2d(const CUtensorMap *tm, int x, int y, int n, const void *src, int rowb) {
    for (int y0 = 0; y0 < n; y0 += kBoxRows) tma_store_2d(tm, x, y + y0, (const char *)src + (size_t)y0 * rowb);
}

// ---------------------------------------------------------------------------
// Persistent TMA-staged n2 and n1 passes (FP32, register-FFT n in [64, 512]).
// Each CTA loops over tiles with two shared-memory stages: while the FFT runs
// on stage s, the TMA load of the next tile fills stage s^1; results leave by
// TMA store.  One thread issues all copies; completion is tracked by one
// mbarrier per stage.  Every wait is bounded: on time-out the CTA records
// the failure in *g.err, waits (bounded) for its own load in flight and
// returns, and the host reports HOM_ETIMEOUT.
// ---------------------------------------------------------------------------
template <typename R, int S, int NF>
__global__ void HOM_PASS_BOUNDS_NF(R, NF) k_x2_tma(Geometry g, const __grid_constant__ CUtensorMap tm, int qtiles,
                                            const MinresState *state) {
    pdl_release();
    pdl_wait();   // predecessor complete (programmatic launch in the MINRES graph)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[kX2MaxStages];
    const int N = g.n2, T = g.tile2, NS = g.x2_stages;
    const int ntiles = g.n1 * g.nb * qtiles;   // stacked cases along k1
    const int tpc = g.n1 * qtiles;             // tiles per case
    // next tile of this CTA's sequence whose case is still iterating
    auto live_from = [&](int t) {
        while (t < ntiles && skip_case(state, t / tpc)) t += gridDim.x;
        return t;
    };
    cpx<R> *const base = reinterpret_cast<cpx<R> *>(smem_raw);
    const int per = N * T;   // stage s starts at base + s * per
    const uint32_t bytes = (uint32_t)(per * sizeof(cpx<R>));
    const bool leader = threadIdx.x == 0;
    if (leader) {
        for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // NS-stage ring: the leader keeps NS - 1 tiles in flight ahead of the one
    // being transformed (tile j of the sequence in stage j mod NS)
    int tile = live_from(blockIdx.x);
    int ahead = tile, issued = 0;   // next tile to load, tiles loaded (leader)
    auto issue = [&]() {
        const int q = issued % NS;
        mbar_expect_tx(&bar[q], bytes);
        tma_load_rows_3d(base + q * per, &tm, (ahead % qtiles) * T, N, ahead / qtiles, T * (int)sizeof(cpx<R>),
                         &bar[q]);
        ++issued;
        ahead = live_from(ahead + gridDim.x);
    };
    if (leader)
        for (int q = 0; q < NS - 1 && ahead < ntiles; ++q) issue();
    const cpx<R> *tw = reinterpret_cast<const cpx<R> *>(g.ax[1].tw);
    for (int i = 0; tile < ntiles; ++i) {
        const int q = i % NS;
        if (leader && ahead < ntiles) {
            bulk_wait_read_all();   // the store of the tile that used this stage has read it
            issue();
        }
        const bool ok = mbar_wait_bounded(&bar[q], (uint32_t)(i / NS) & 1u);
        if (__syncthreads_or(!ok)) {
            if (leader) {   // record, then wait (bounded) for this CTA's loads in flight
                atomicExch(g.err, 1);
                for (int m = i; m < issued; ++m) mbar_wait_bounded(&bar[m % NS], (uint32_t)(m / NS) & 1u);
                bulk_wait_all();
            }
            return;
        }
        cpx<R> *buf = base + q * per;
        fast_fft<R, S, NF>(buf, T, T, tw);
        fence_proxy_async_smem();
        __syncthreads();
        if (leader) {
            tma_store_rows_3d(&tm, (tile % qtiles) * T, N, tile / qtiles, buf, T * (int)sizeof(cpx<R>));
            bulk_commit();
        }
        tile = live_from(tile + gridDim.x);
    }
    if (leader) bulk_wait_all();
}

// MoDBFFT contraction at frequency (k1, k2, k3) of the 10-component
// forward transform t (the stress tau and the penalty vector g), eq.
// (modbfftfop): r = tau xi + g with xi = i 2 pi q, q the integer frequency (0
// on a Nyquist index); r = 0 at xi = 0.  The same arithmetic as the
// contraction kernel of the MoDBFFT operator.
template <typename R>
__device__ __forceinline__ void modb_contract_at(const Geometry &g, int k1, int k2, int k3, const cpx<R> *t,
                                                 cpx<R> r[3]) {
    const int ks[3] = {k1, k2, k3}, ns[3] = {g.n1, g.n2, g.n3};
    double q[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int n = ns[p], k = ks[p];
        q[p] = ((n & 1) == 0 && 2 * k == n) ? 0.0 : (double)((2 * k < n) ? k : k - n);
    }
    r[0] = r[1] = r[2] = mk<R>(0, 0);
    if (q[0] == 0.0 && q[1] == 0.0 && q[2] == 0.0) return;
    const R tp = (R)6.28318530717958647692;
    const R r2 = (R)0.70710678118654752440;
    const R sv[3] = {tp * (R)q[0], tp * (R)q[1], tp * (R)q[2]};
    const cpx<R> T[3][3] = {{t[0], scale<R>(t[5], r2), scale<R>(t[4], r2)},
                            {scale<R>(t[5], r2), t[1], scale<R>(t[3], r2)},
                            {scale<R>(t[4], r2), scale<R>(t[3], r2), t[2]}};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const cpx<R> a = add<R>(add<R>(scale<R>(T[i][0], sv[0]), scale<R>(T[i][1], sv[1])), scale<R>(T[i][2], sv[2]));
        r[i] = add<R>(mk<R>(-a.y, a.x), t[6 + i]);
    }
}

// MoDBFFT expansion at frequency (k1, k2, k3) of the displacement u (3
// components), eq. (modbfftfop): o = sym(u (x) xi) in Mandel order and, with
// nc_out = 10, the penalty vector alpha sym(u (x) xi) . xi (0 without the
// penalty) and a zero pad; xi = i 2 pi q, q the integer frequency (0 on a
// Nyquist index); o = 0 at xi = 0.  The point-wise expansion kernel and the
// inverse n1 pass with the expansion fused both take it from here.
template <typename R>
__device__ __forceinline__ void modb_expand_at(const Geometry &g, int k1, int k2, int k3, const cpx<R> *u, R alpha,
                                               int with_penalty, int nc_out, cpx<R> *o) {
    const int ks[3] = {k1, k2, k3}, ns[3] = {g.n1, g.n2, g.n3};
    double qd[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int n = ns[p], k = ks[p];
        qd[p] = ((n & 1) == 0 && 2 * k == n) ? 0.0 : (double)((2 * k < n) ? k : k - n);
    }
    if (qd[0] == 0.0 && qd[1] == 0.0 && qd[2] == 0.0) {
        for (int c = 0; c < nc_out; ++c) o[c] = mk<R>(0, 0);
        return;
    }
    const R tp = (R)6.28318530717958647692;   // 2 pi
    const R r2 = (R)1.41421356237309504880;
    // xi = i s, s = 2 pi q (real): sym(u (x) xi)_ij = i/2 (u_i s_j + u_j s_i)
    const R s0 = tp * (R)qd[0], s1 = tp * (R)qd[1], s2 = tp * (R)qd[2];
    const cpx<R> u0 = u[0], u1 = u[1], u2 = u[2];
    auto isym = [](cpx<R> a, R sa, cpx<R> b, R sb) {   // i/2 (a sb + b sa)
        const R re = (R)0.5 * (a.x * sb + b.x * sa), im = (R)0.5 * (a.y * sb + b.y * sa);
        return mk<R>(-im, re);
    };
    const cpx<R> e00 = isym(u0, s0, u0, s0), e11 = isym(u1, s1, u1, s1), e22 = isym(u2, s2, u2, s2);
    const cpx<R> e12 = isym(u1, s1, u2, s2), e02 = isym(u0, s0, u2, s2), e01 = isym(u0, s0, u1, s1);
    o[0] = e00;
    o[1] = e11;
    o[2] = e22;
    o[3] = scale<R>(e12, r2);
    o[4] = scale<R>(e02, r2);
    o[5] = scale<R>(e01, r2);
    if (nc_out == 10) {
        // g_i = alpha sum_j e_ij xi_j = alpha i sum_j e_ij s_j
        const cpx<R> E[3][3] = {{e00, e01, e02}, {e01, e11, e12}, {e02, e12, e22}};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const cpx<R> t = add<R>(add<R>(scale<R>(E[i][0], s0), scale<R>(E[i][1], s1)), scale<R>(E[i][2], s2));
            o[6 + i] = with_penalty ? mk<R>(-alpha * t.y, alpha * t.x) : mk<R>(0, 0);
        }
        o[9] = mk<R>(0, 0);
    }
}

// With MC (MoDBFFT, 10 components, forward): instead of storing the
// transformed tile, contract each frequency to the 3-component result
// (modb_contract_at) and write it to out3, with the weighted dot product
// against dot3 (if given) in the partials.
template <typename R, int NF, bool MC = false>
__global__ void HOM_PASS_BOUNDS_NF(R, NF) k_x1_tma(Geometry g, int flags, const __grid_constant__ CUtensorMap tin,
                                            const __grid_constant__ CUtensorMap tout,
                                            const __grid_constant__ CUtensorMap tdot, double *__restrict__ partials,
                                            const MinresState *state, cpx<R> *__restrict__ out3,
                                            const cpx<R> *__restrict__ dot3) {
    if (skip(state)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    const int NC = g.nc, N = g.n1, T = g.tile1, H = g.h, L = NC * T;
    const int cols = g.n2 * H;
    const int ntiles = (cols + T - 1) / T;
    const bool dot = (flags & X1_DOT) != 0;
    const int tile_elems = N * L;
    cpx<R> *base = reinterpret_cast<cpx<R> *>(smem_raw);
    // stage s: data tile at base + s * per, dot tile (if any) right after it
    const int per = tile_elems * (dot ? 2 : 1);
    const uint32_t bytes = (uint32_t)(tile_elems * sizeof(cpx<R>)) * (dot ? 2u : 1u);
    const bool leader = threadIdx.x == 0;
    if (leader) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t, int s) {
        mbar_expect_tx(&bar[s], bytes);
        tma_load_rows_2d(base + s * per, &tin, NC * T * t, 0, N, L * (int)sizeof(cpx<R>), &bar[s]);
        if (dot) tma_load_rows_2d(base + s * per + tile_elems, &tdot, NC * T * t, 0, N, L * (int)sizeof(cpx<R>), &bar[s]);
    };
    int tile = blockIdx.x;
    if (leader && tile < ntiles) issue(tile, 0);
    const cpx<R> *tw = reinterpret_cast<const cpx<R> *>(g.ax[0].tw);
    const int lt = threadIdx.x % L, e0 = threadIdx.x / L, es = blockDim.x / L;
    const int tg = threadIdx.x % T, eg0 = threadIdx.x / T, egs = blockDim.x / T;
    Acc<R> acc;
    for (int i = 0; tile < ntiles; ++i, tile += gridDim.x) {
        const int s = i & 1;
        const int next = tile + gridDim.x;
        if (leader && next < ntiles) {
            bulk_wait_read_all();
            issue(next, s ^ 1);
        }
        const bool ok = mbar_wait_bounded(&bar[s], (i >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (leader) {   // record, then wait (bounded) for this CTA's loads in flight
                atomicExch(g.err, 1);
                mbar_wait_bounded(&bar[s], (i >> 1) & 1);
                if (next < ntiles) mbar_wait_bounded(&bar[s ^ 1], ((i + 1) >> 1) & 1);
                bulk_wait_all();
            }
            return;
        }
        cpx<R> *buf = base + s * per;
        const int g0 = tile * T;
        const int colg = g0 + tg;
        const int k2g = colg / H, k3g = colg - k2g * H;
        if (flags & X1_GAMMA_IN) {
            if (colg < cols)
                for (int e = eg0; e < N; e += egs) gamma_at<R>(g, e, k2g, k3g, buf + e * L + tg * NC);
            __syncthreads();
        }
        if (flags & X1_FWD) fast_fft<R, -1, NF>(buf, L, L, tw);
        else fast_fft<R, 1, NF>(buf, L, L, tw);
        if (flags & X1_GAMMA_OUT) {
            if (colg < cols)
                for (int e = eg0; e < N; e += egs) gamma_at<R>(g, e, k2g, k3g, buf + e * L + tg * NC);
            __syncthreads();
        }
        if constexpr (MC) {   // MoDBFFT contraction in place of the store
            if (colg < cols) {
                const R w = (R)pweight(k3g, g.n3);
                for (int e = eg0; e < N; e += egs) {
                    cpx<R> r[3];
                    modb_contract_at<R>(g, e, k2g, k3g, buf + e * L + tg * NC, r);
                    const size_t f = ((size_t)e * g.n2 + k2g) * H + k3g;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        out3[3 * f + c] = r[c];
                        if (dot3) {
                            const cpx<R> d = dot3[3 * f + c];
                            acc.add_prod(w * r[c].x, d.x);
                            acc.add_prod(w * r[c].y, d.y);
                        }
                    }
                }
            }
            __syncthreads();   // the stage is read before the next load into it
            continue;
        }
        if (dot) {
            const int colt = g0 + lt / NC;
            if (colt < cols) {
                const int k3 = colt % H;
                const R w = (R)pweight(k3, g.n3);
                const cpx<R> *dv = buf + tile_elems;
                for (int e = e0; e < N; e += es) {
                    const cpx<R> z = buf[e * L + lt], d = dv[e * L + lt];
                    acc.add_prod(w * z.x, d.x);
                    acc.add_prod(w * z.y, d.y);
                }
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (leader) {
            tma_store_rows_2d(&tout, NC * T * tile, 0, N, buf, L * (int)sizeof(cpx<R>));
            bulk_commit();
        }
    }
    if (leader) bulk_wait_all();
    if (dot || (MC && dot3)) {
        const double sum = block_sum(acc.value());
        if (threadIdx.x == 0) partials[blockIdx.x] = sum;
    }
}

// MoDBFFT inverse n1 pass with the expansion fused (TMA-staged, FP32, 10
// components): each tile is formed in shared memory from u (3 components,
// plain loads) by modb_expand_at with the penalty, transformed (inverse DFT
// along n1) and stored by TMA, so that the 10-component spectrum is written
// once instead of being written by the expansion kernel and read back by the
// pass.  Two stage buffers: a tile is expanded into one while the store of
// the previous tile still reads the other.
template <typename R, int NF>
__global__ void HOM_PASS_BOUNDS_NF(R, NF) k_x1_tma_expand(Geometry g, const __grid_constant__ CUtensorMap tout,
                                                   const cpx<R> *__restrict__ u3, R alpha,
                                                   const MinresState *state) {
    if (skip(state)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int NC = g.nc, N = g.n1, T = g.tile1, H = g.h, L = NC * T;
    const int cols = g.n2 * H;
    const int ntiles = (cols + T - 1) / T;
    const int tile_elems = N * L;
    cpx<R> *base = reinterpret_cast<cpx<R> *>(smem_raw);
    const bool leader = threadIdx.x == 0;
    const cpx<R> *tw = reinterpret_cast<const cpx<R> *>(g.ax[0].tw);
    const int tg = threadIdx.x % T, eg0 = threadIdx.x / T, egs = blockDim.x / T;
    for (int i = 0, tile = blockIdx.x; tile < ntiles; ++i, tile += gridDim.x) {
        cpx<R> *buf = base + (i & 1) * tile_elems;
        // the store issued from this stage two tiles ago has read its source
        if (leader) bulk_wait_read_1();
        __syncthreads();
        const int colg = tile * T + tg;
        const int k2g = colg / H, k3g = colg - k2g * H;
        for (int e = eg0; e < N; e += egs) {
            cpx<R> *o = buf + e * L + tg * NC;
            if (colg < cols)
                modb_expand_at<R>(g, e, k2g, k3g, u3 + 3 * (((size_t)e * g.n2 + k2g) * H + k3g), alpha, 1, NC, o);
            else
                for (int c = 0; c < NC; ++c) o[c] = mk<R>(0, 0);
        }
        __syncthreads();
        fast_fft<R, 1, NF>(buf, L, L, tw);
        fence_proxy_async_smem();
        __syncthreads();
        if (leader) {
            tma_store_rows_2d(&tout, NC * T * tile, 0, N, buf, L * (int)sizeof(cpx<R>));
            bulk_commit();
        }
    }
    if (leader) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Fused n1 pass of one MINRES step (6-component spectra).  With the work
// spectrum holding F_3 F_2 of tau = C e_k (the forward n3 and n2 passes of
// A^ u_k) and alpha_k already known from the n3 pass's strain energy, one
// pass over each n1 tile
//   1. finishes p = A^ u_k: forward DFT along n1 and the projector G;
//   2. takes the Lanczos step on unnormalised vectors,
//        u_{k+1} = p / beta_k - (alpha_k / beta_k) u_k - (beta_k / beta_{k-1}) u_{k-1},
//      into a third buffer, with the weighted partial ||u_{k+1}||^2, and the
//      lagged w update of step k-1 (w_{k-1} over w_{k-3});
//   3. starts A^ u_{k+1}: G on u_{k+1} and the inverse DFT along n1, written
//      back over the tile of the work spectrum for the next step's n2 pass.
// p never reaches HBM, and u_k is read once per step instead of three times.
// x is updated every third step only, with the three newest w at once,
//   x += tau_{k-3} w_{k-3} + tau_{k-2} w_{k-2} + tau_{k-1} w_{k-1},
// which the two w buffers still hold at that step (w_{k-3} is read before
// w_{k-1} replaces it); the flush after the loop adds what is pending.  The
// sum is the same as one update per step, rounded in another order.
// ---------------------------------------------------------------------------
template <typename R> struct LzCoef {
    R cp, cu, cv;            // 1/beta_k, -alpha_k/beta_k, -beta_k/beta_{k-1}
    R d, e, ig, tau, ib;     // lagged update of step k-1
    R t1, t2;                // tau of the two steps before
    bool lagged;
    bool xstep;              // this step updates x
};

// x is updated when the iterations done (the state's k) are a multiple of 3
__host__ __device__ constexpr bool minres_xstep(int k) { return k > 0 && k % 3 == 0; }

template <typename R>
__device__ __forceinline__ LzCoef<R> lz_coef(const MinresState *st) {
    LzCoef<R> c;
    const double bk = st->beta, bkm = st->beta_prev;
    c.cp = (R)(1.0 / bk);
    c.cu = (R)(-st->alpha / bk);
    c.cv = (R)(bkm > 0.0 ? -bk / bkm : 0.0);
    c.lagged = st->k > 0;
    c.d = (R)st->u_delta;
    c.e = (R)st->u_eps;
    c.ig = (R)st->u_inv_gamma;
    c.tau = (R)st->u_tau;
    c.ib = (R)st->u_inv_beta;
    c.t1 = (R)st->u_tau1;
    c.t2 = (R)st->u_tau2;
    c.xstep = minres_xstep(st->k);
    return c;
}

// Steps 1-3 on the tile of columns [g0, g0 + T) held in buf (element e of
// line l at buf[e * L + l], L = 6 T); returns the buffer holding the inverse
// transform (buf for the register engine).  The CTA's threads (nsync = 0) or
// its first nsync threads (named barrier 1) call it.  Between the two
// transforms one loop over the tile's frequencies builds xi once per
// frequency and applies the projector to p and to u_{k+1}; the Krylov
// vectors are stored in tile order, so the six components of a frequency
// are 48 contiguous bytes of each vector and a warp reads and writes a
// contiguous block.  u_{k+1} goes to un, a third buffer (u_{k-1} stays
// readable for the lagged update); with LAG the lagged w / x update of step
// k-1 is done here too, else by other warps (x1_lagged_block).
template <typename R, int NF, bool LAG>
__device__ __forceinline__ cpx<R> *x1_lanczos_tile(const Geometry &g, cpx<R> *buf, cpx<R> *buf2, int g0,
                                                   const LzCoef<R> &c, const cpx<R> *__restrict__ uk,
                                                   const cpx<R> *__restrict__ um, cpx<R> *__restrict__ un,
                                                   const cpx<R> *__restrict__ wa, cpx<R> *__restrict__ wb,
                                                   cpx<R> *__restrict__ x, Acc<R> &acc, int nsync) {
    constexpr int NC = 6;
    const int N = g.n1, T = g.tile1, H = g.h, L = NC * T;
    const int cols = g.n2 * H;
    const int nthr = nsync ? nsync : (int)blockDim.x;
    // 1. forward DFT along n1
    cpx<R> *res = run_fft<R, -1, NF>(buf, buf2, L, L, g.ax[0], nsync);
    // 2. per frequency: p = G (.), Lanczos step, lagged update, G u_{k+1}
    const size_t kb = (size_t)(g0 / T) * (size_t)(N * L);
    for (int f = threadIdx.x; f < N * T; f += nthr) {
        const int e = f / T, t = f - e * T;
        const int col = g0 + t;
        cpx<R> *sp = res + e * L + t * NC;
        if (col >= cols) {
#pragma unroll
            for (int q = 0; q < NC; ++q) sp[q] = mk<R>(0, 0);
            continue;
        }
        const int k2 = col / H, k3 = col - k2 * H;
        const size_t i = kb + (size_t)f * NC;
        cpx<R> v[NC], u[NC], uo[NC];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            Six<R>::load_pair(sp, p, v[2 * p], v[2 * p + 1]);
            Six<R>::load_pair(uk + i, p, u[2 * p], u[2 * p + 1]);
            Six<R>::load_pair(um + i, p, uo[2 * p], uo[2 * p + 1]);
        }
        const GammaE<R> ge = gamma_e<R>(g, e, k2, k3);
        gamma_apply<R>(g, ge, v);
        const R w = (R)pweight(k3, g.n3);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            v[q] = mk<R>(c.cp * v[q].x + c.cu * u[q].x + c.cv * uo[q].x, c.cp * v[q].y + c.cu * u[q].y + c.cv * uo[q].y);
            acc.add_prod(w * v[q].x, v[q].x);
            acc.add_prod(w * v[q].y, v[q].y);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) Six<R>::store_pair(un + i, p, v[2 * p], v[2 * p + 1]);
        if (LAG && c.lagged) {
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                cpx<R> a[2], b[2], wn[2];
                Six<R>::load_pair(wa + i, p, a[0], a[1]);
                Six<R>::load_pair(wb + i, p, b[0], b[1]);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const cpx<R> &o = uo[2 * p + q];
                    wn[q] = mk<R>((o.x * c.ib - c.d * a[q].x - c.e * b[q].x) * c.ig,
                                  (o.y * c.ib - c.d * a[q].y - c.e * b[q].y) * c.ig);
                }
                Six<R>::store_pair(wb + i, p, wn[0], wn[1]);
                if (c.xstep) {
                    cpx<R> xx[2];
                    Six<R>::load_pair(x + i, p, xx[0], xx[1]);
#pragma unroll
                    for (int q = 0; q < 2; ++q)
                        xx[q] = mk<R>(xx[q].x + c.t2 * b[q].x + c.t1 * a[q].x + c.tau * wn[q].x,
                                      xx[q].y + c.t2 * b[q].y + c.t1 * a[q].y + c.tau * wn[q].y);
                    Six<R>::store_pair(x + i, p, xx[0], xx[1]);
                }
            }
        }
        gamma_apply<R>(g, ge, v);
#pragma unroll
        for (int p = 0; p < 3; ++p) Six<R>::store_pair(sp, p, v[2 * p], v[2 * p + 1]);
    }
    group_sync(nsync);
    // 3. inverse DFT along n1 of G u_{k+1}
    return run_fft<R, 1, NF>(res, res == buf ? buf2 : buf, L, L, g.ax[0], nsync);
}

// At most 384 threads per CTA (set_shapes enforces it): the fused pass keeps
// the Lanczos operands of a frequency (five Krylov vectors, 60 values) in
// registers, so it is not held to a register cap that would spill them.
#define HOM_X1L_BOUNDS(R) __launch_bounds__(384, 1)

// plain-load form: one tile per CTA, the lagged update inline
template <typename R, int NF>
__global__ void HOM_X1L_BOUNDS(R) k_x1_lanczos(Geometry g, cpx<R> *__restrict__ spec, const cpx<R> *__restrict__ uk,
                                                const cpx<R> *__restrict__ um, cpx<R> *__restrict__ un,
                                                const cpx<R> *__restrict__ wa, cpx<R> *__restrict__ wb,
                                                cpx<R> *__restrict__ x, const MinresState *state,
                                                double *__restrict__ partials, Fold fold) {
    pdl_release();
    pdl_wait();   // predecessor complete (programmatic launch in the MINRES graph)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int NC = 6;
    const int N = g.n1, T = g.tile1, H = g.h, L = NC * T;
    cpx<R> *buf = reinterpret_cast<cpx<R> *>(smem_raw);
    cpx<R> *buf2 = buf + N * L;
    const int cols = g.n2 * H;
    // load case cs of a stacked batch, tile tc of that case
    const int tpc = (cols + T - 1) / T;
    const int cs = blockIdx.x / tpc, tc = blockIdx.x - cs * tpc;
    if (skip_case(state, cs)) return;
    const size_t ko = (size_t)cs * g.kvec;      // the case's Krylov block
    spec += (size_t)cs * NC * g.S;               // the case's work spectrum
    const int g0 = tc * T;
    const size_t sK1 = (size_t)cols * NC;
    const int lt = threadIdx.x % L, e0 = threadIdx.x / L, es = blockDim.x / L;
    const bool live = g0 + lt / NC < cols;
    const LzCoef<R> c = lz_coef<R>(state + cs);
    {
        const cpx<R> *src = spec + (size_t)g0 * NC + lt;
        for (int e = e0; e < N; e += es) buf[e * L + lt] = live ? src[e * sK1] : mk<R>(0, 0);
    }
    __syncthreads();
    Acc<R> acc;
    cpx<R> *res = x1_lanczos_tile<R, NF, true>(g, buf, buf2, g0, c, uk + ko, um + ko, un + ko, wa + ko, wb + ko,
                                               x + ko, acc, 0);
    if (live) {
        cpx<R> *dst = spec + (size_t)g0 * NC + lt;
        for (int e = e0; e < N; e += es) dst[e * sK1] = res[e * L + lt];
    }
    const double sum = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = sum;   // = partials[cs * tpc + tc]
    if (fold.cnt && last_of(fold.cnt + kNbMax + cs, tpc)) {   // Givens step of case cs
        const double tot = sum_partials(partials + (size_t)cs * tpc, tpc);
        if (threadIdx.x == 0) {
            givens_step(fold.st + cs, tot);
            fold.cnt[kNbMax + cs] = 0;
        }
    }
}

// OR of a predicate over the n threads that use named barrier ID
template <int ID>
__device__ __forceinline__ bool group_or(bool v, int n) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(ID), "r"(n)
        : "memory");
    return r != 0;
}

// The lagged update of step k-1 by the lagged-update warps (named barrier
// 2) of the fused n1 pass, over the Krylov blocks of the CTA's tiles whose
// case has one:
//   w_{k-1} = (u_{k-1} / beta_{k-1} - delta w_{k-2} - eps w_{k-3}) / gamma
// over the slot of w_{k-3}, and on every third step the deferred x update.
// The blocks are cut into items of kX1LagChunk bytes; one thread brings an
// item's operands (u_{k-1}, w_{k-2}, w_{k-3}, and x on an x step) into a
// ring of S stages with untiled bulk copies, S items ahead, and the warps
// update it from shared memory and store w_{k-1} (and x) to HBM.  The update is the same on every real number,
// so it runs on 16-byte vectors.  Returns false after a bounded wait ran
// out (the copies in flight have been waited for, bounded).
template <typename R, typename LiveFrom>
__device__ __forceinline__ bool x1_lagged(const Geometry &g, const LzCoef<R> *scoef, LiveFrom live_from, int ntiles,
                                          int tpc, int per, unsigned char *ring, uint64_t *lbar,
                                          const cpx<R> *__restrict__ um, const cpx<R> *__restrict__ wa,
                                          cpx<R> *__restrict__ wb, cpx<R> *__restrict__ x) {
    using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
    constexpr int NR = 16 / sizeof(R);
    const int S = g.x1_lag_stages;
    const int lt = threadIdx.x - kX1Group;
    const long long pbytes = (long long)per * sizeof(cpx<R>);
    auto next_tile = [&](int t) {
        t = live_from(t);
        while (t < ntiles && !scoef[t / tpc].lagged) t = live_from(t + gridDim.x);
        return t;
    };
    auto base_of = [&](int t) {   // byte offset of tile t's block in each Krylov vector
        return ((long long)(t / tpc) * g.kvec + (long long)(t % tpc) * per) * (long long)sizeof(cpx<R>);
    };
    int pt = next_tile(blockIdx.x), ct = pt;   // producer / consumer cursors (tile, byte offset)
    long long po = 0, co = 0;
    int issued = 0;                            // items issued (thread lt = 0)
    auto issue = [&]() {
        const int s = issued % S;
        const uint32_t nb = (uint32_t)(pbytes - po < kX1LagChunk ? pbytes - po : kX1LagChunk);
        const long long o = base_of(pt) + po;
        unsigned char *st = ring + (size_t)s * 4 * kX1LagChunk;
        const bool xs = scoef[pt / tpc].xstep;
        mbar_expect_tx(&lbar[s], (xs ? 4 : 3) * nb);
        bulk_load(st, reinterpret_cast<const char *>(um) + o, nb, &lbar[s]);
        bulk_load(st + kX1LagChunk, reinterpret_cast<const char *>(wa) + o, nb, &lbar[s]);
        bulk_load(st + 2 * kX1LagChunk, reinterpret_cast<const char *>(wb) + o, nb, &lbar[s]);
        if (xs) bulk_load(st + 3 * kX1LagChunk, reinterpret_cast<const char *>(x) + o, nb, &lbar[s]);
        ++issued;
        po += kX1LagChunk;
        if (po >= pbytes) {
            po = 0;
            pt = next_tile(pt + gridDim.x);
        }
    };
    if (lt == 0)
        for (int s = 0; s < S && pt < ntiles; ++s) issue();
    int n = 0;
    for (; ct < ntiles; ++n) {
        const int s = n % S;
        const bool got = mbar_wait_bounded(&lbar[s], (uint32_t)(n / S) & 1u);
        if (group_or<2>(!got, kX1LagThreads)) {
            if (lt == 0) {   // record, then wait (bounded) for the items in flight
                atomicExch(g.err, 1);
                for (int m = n; m < issued; ++m) mbar_wait_bounded(&lbar[m % S], (uint32_t)(m / S) & 1u);
            }
            return false;
        }
        const LzCoef<R> c = scoef[ct / tpc];
        const int nv = (int)((pbytes - co < kX1LagChunk ? pbytes - co : kX1LagChunk) / 16);
        const long long o = base_of(ct) + co;
        const V *su = reinterpret_cast<const V *>(ring + (size_t)s * 4 * kX1LagChunk);
        const V *sa = su + kX1LagChunk / 16, *sb = su + 2 * (kX1LagChunk / 16), *sx = su + 3 * (kX1LagChunk / 16);
        V *gb = reinterpret_cast<V *>(reinterpret_cast<char *>(wb) + o);
        V *gx = reinterpret_cast<V *>(reinterpret_cast<char *>(x) + o);
        if (c.xstep) {
            for (int j = lt; j < nv; j += kX1LagThreads) {
                V vu = su[j], va = sa[j], vb = sb[j], vx = sx[j], vn;
                const R *u = reinterpret_cast<const R *>(&vu);
                const R *a = reinterpret_cast<const R *>(&va);
                const R *b = reinterpret_cast<const R *>(&vb);
                R *wn = reinterpret_cast<R *>(&vn);
                R *xx = reinterpret_cast<R *>(&vx);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    wn[r] = (u[r] * c.ib - c.d * a[r] - c.e * b[r]) * c.ig;
                    xx[r] += c.t2 * b[r] + c.t1 * a[r] + c.tau * wn[r];
                }
                gb[j] = vn;
                gx[j] = vx;
            }
        } else {
            for (int j = lt; j < nv; j += kX1LagThreads) {
                V vu = su[j], va = sa[j], vb = sb[j];
                const R *u = reinterpret_cast<const R *>(&vu);
                const R *a = reinterpret_cast<const R *>(&va);
                R *b = reinterpret_cast<R *>(&vb);
#pragma unroll
                for (int r = 0; r < NR; ++r) b[r] = (u[r] * c.ib - c.d * a[r] - c.e * b[r]) * c.ig;
                gb[j] = vb;
            }
        }
        co += kX1LagChunk;
        if (co >= pbytes) {
            co = 0;
            ct = next_tile(ct + gridDim.x);
        }
        asm volatile("bar.sync 2, %0;" ::"n"(kX1LagThreads) : "memory");   // stage s is read
        if (lt == 0 && pt < ntiles) issue();
    }
    return true;
}

// persistent TMA-staged form (FP32, register FFT lengths 64..512), warp-
// specialised.  The first g.threads1 threads (the transform group, named
// barrier 1) take the work tiles: each comes and goes by TMA, double-
// buffered as in k_x1_tma, and the Lanczos step reads u_k and u_{k-1}
// (bulk-prefetched into L2 at the tile's start) and writes u_{k+1} with
// plain coalesced accesses.  The last kX1LagThreads threads (two warps) run
// the lagged w update (and on one step in three the deferred x update) on
// the same tiles' Krylov blocks, streaming u_{k-1}, w_{k-2}, w_{k-3} (and x)
// while the transform group works in shared memory; the two groups share no
// written data (u_{k+1} has its own buffer), so they never wait on each
// other.  (Prefetching the next tile's blocks into L2 was measured to double
// the DRAM reads: the lines were evicted before use; the current tile's are
// used within microseconds.)  Tiles are numbered case-major over the stacked
// batch; tiles of converged cases are skipped; each transform thread keeps
// one running sum per case in shared memory, and the CTA writes one partial
// per case (partials[case * gridDim + block]).
template <typename R, int NF>
__global__ void __launch_bounds__(kX1Group + kX1LagThreads, 2)
    k_x1_lanczos_tma(Geometry g, const __grid_constant__ CUtensorMap tspec, const cpx<R> *__restrict__ uk,
                     const cpx<R> *__restrict__ um, cpx<R> *__restrict__ un, const cpx<R> *__restrict__ wa,
                     cpx<R> *__restrict__ wb, cpx<R> *__restrict__ x, const MinresState *state,
                     double *__restrict__ partials, Fold fold) {
    pdl_release();
    pdl_wait();   // predecessor complete (programmatic launch in the MINRES graph)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ __align__(8) uint64_t lbar[kX1LagMaxStages];
    __shared__ double sacc[kNbMax * kX1Group];
    __shared__ LzCoef<R> scoef[kNbMax];   // each case's coefficients, converted once
    constexpr int NC = 6;
    const int N = g.n1, T = g.tile1, L = NC * T;
    const int cols = g.n2 * g.h;
    const int tpc = (cols + T - 1) / T;   // tiles per case
    const int ntiles = tpc * g.nb;
    const int per = N * L;
    const uint32_t bytes = (uint32_t)(per * sizeof(cpx<R>));
    cpx<R> *base = reinterpret_cast<cpx<R> *>(smem_raw);
    const bool leader = threadIdx.x == 0;
    const bool xform = threadIdx.x < kX1Group;
    auto live_from = [&](int t) {
        while (t < ntiles && skip_case(state, t / tpc)) t += gridDim.x;
        return t;
    };
    if (xform)
        for (int cc = 0; cc < g.nb; ++cc) sacc[cc * kX1Group + threadIdx.x] = 0.0;
    if (threadIdx.x < g.nb) scoef[threadIdx.x] = lz_coef<R>(state + threadIdx.x);
    if (leader) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        for (int q = 0; q < kX1LagMaxStages; ++q) mbar_init(&lbar[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (!xform) {
        x1_lagged<R>(g, scoef, live_from, ntiles, tpc, per, smem_raw + g.smem1_tma, lbar, um, wa, wb, x);
    } else {
        int tile = live_from(blockIdx.x);
        if (leader && tile < ntiles) {
            mbar_expect_tx(&bar[0], bytes);
            tma_load_rows_2d(base, &tspec, NC * T * (tile % tpc), N * (tile / tpc), N, L * (int)sizeof(cpx<R>),
                             &bar[0]);
        }
        for (int i = 0; tile < ntiles; ++i) {
            const int s = i & 1;
            const int next = live_from(tile + gridDim.x);
            if (leader && next < ntiles) {
                bulk_wait_read_all();   // the store of the tile that used stage s^1 has read it
                mbar_expect_tx(&bar[s ^ 1], bytes);
                tma_load_rows_2d(base + (s ^ 1) * per, &tspec, NC * T * (next % tpc), N * (next / tpc), N,
                                 L * (int)sizeof(cpx<R>), &bar[s ^ 1]);
            }
            const bool ok = mbar_wait_bounded(&bar[s], (i >> 1) & 1);
            if (group_or<1>(!ok, kX1Group)) {
                if (leader) {   // record, then wait (bounded) for this CTA's loads in flight
                    atomicExch(g.err, 1);
                    mbar_wait_bounded(&bar[s], (i >> 1) & 1);
                    if (next < ntiles) mbar_wait_bounded(&bar[s ^ 1], ((i + 1) >> 1) & 1);
                }
                break;
            }
            const int cs = tile / tpc, tc = tile - cs * tpc;
            const size_t ko = (size_t)cs * g.kvec;
            if (leader && g.x1_l2pf) {   // this tile's u_k and u_{k-1} blocks into L2 for the Lanczos step
                bulk_prefetch_l2(uk + ko + (size_t)tc * per, bytes);
                bulk_prefetch_l2(um + ko + (size_t)tc * per, bytes);
            }
            const LzCoef<R> c = scoef[cs];
            Acc<R> acc;
            cpx<R> *buf = base + s * per;
            cpx<R> *res = x1_lanczos_tile<R, NF, false>(g, buf, buf, tc * T, c, uk + ko, um + ko, un + ko, wa + ko,
                                                        wb + ko, x + ko, acc, kX1Group);
            sacc[cs * kX1Group + threadIdx.x] += acc.value();
            fence_proxy_async_smem();
            group_sync(kX1Group);
            if (leader) {
                tma_store_rows_2d(&tspec, NC * T * tc, N * cs, N, res, L * (int)sizeof(cpx<R>));
                bulk_commit();
            }
            tile = next;
        }
        if (leader) bulk_wait_all();
    }
    __syncthreads();   // both groups done
    for (int cc = 0; cc < g.nb; ++cc) {
        const double sum = block_sum(xform ? sacc[cc * kX1Group + threadIdx.x] : 0.0);
        if (threadIdx.x == 0) partials[cc * gridDim.x + blockIdx.x] = sum;
    }
    if (fold.cnt && last_of(fold.cnt + 2 * kNbMax, gridDim.x)) {   // Givens step of every case
        for (int cc = 0; cc < g.nb; ++cc) {
            const double tot = sum_partials(partials + (size_t)cc * gridDim.x, gridDim.x);
            if (threadIdx.x == 0) givens_step(fold.st + cc, tot);
        }
        if (threadIdx.x == 0) fold.cnt[2 * kNbMax] = 0;
    }
}

// ---------------------------------------------------------------------------
// Krylov vector kernels on half spectra (n = 6 S complex values).  The
// Parseval weight of element i depends on k3 = (i / 6) mod h.
// ---------------------------------------------------------------------------
// MINRES step on unnormalised Lanczos vectors (see Launch::lanczos_update).
// Scalars come from the FP64 state: beta_k, beta_{k-1}, alpha_k, and the
// coefficients of the lagged w / x update of step k-1.
template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_lanczos_update(int n, int h, int n3, const cpx<R> *__restrict__ p,
                                                               const cpx<R> *__restrict__ uk, cpx<R> *__restrict__ um,
                                                               const cpx<R> *__restrict__ wa, cpx<R> *__restrict__ wb,
                                                               cpx<R> *__restrict__ x, const MinresState *st,
                                                               double *__restrict__ partials) {
    if (skip(st)) return;
    const double bk = st->beta, bkm = st->beta_prev;
    const R cp = (R)(1.0 / bk), cu = (R)(-st->alpha / bk), cv = (R)(bkm > 0.0 ? -bk / bkm : 0.0);
    const bool lagged = st->k > 0;
    const R d = (R)st->u_delta, e = (R)st->u_eps, ig = (R)st->u_inv_gamma, tau = (R)st->u_tau,
            ib = (R)st->u_inv_beta;
    Acc<R> acc;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const cpx<R> pp = p[i], u = uk[i], uo = um[i];
        const cpx<R> q = mk<R>(cp * pp.x + cu * u.x + cv * uo.x, cp * pp.y + cu * u.y + cv * uo.y);
        um[i] = q;
        if (lagged) {
            const cpx<R> a = wa[i], b = wb[i], xx = x[i];
            const cpx<R> wn = mk<R>((uo.x * ib - d * a.x - e * b.x) * ig, (uo.y * ib - d * a.y - e * b.y) * ig);
            wb[i] = wn;
            x[i] = mk<R>(xx.x + tau * wn.x, xx.y + tau * wn.y);
        }
        const R w = (R)pweight((i / 6) % h, n3);
        acc.add_prod(w * q.x, q.x);
        acc.add_prod(w * q.y, q.y);
    }
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// standard half-spectrum order <-> n1-tile order (see Geometry::kvec):
// element (k1, col, c) of the standard order, col = k2 h + k3, sits in the
// tile order at (col / T) n1 6T + k1 6T + (col % T) 6 + c
template <typename R>
__global__ void k_tiles(long long n, int n1, int cols, int T, int to_tiles, const cpx<R> *__restrict__ in,
                        cpx<R> *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % 6);
        const long long f = i / 6;
        const int col = (int)(f % cols), k1 = (int)(f / cols);
        const long long t = (long long)(col / T) * n1 * 6 * T + (long long)k1 * 6 * T + (col % T) * 6 + c;
        if (to_tiles) out[t] = in[i];
        else out[i] = in[t];
    }
}

// The lagged w / x update of the last step K; skipped when there is none
// or the state kept the last finite iterate.
// With three Lanczos buffers (the fused step) x has been updated every
// third step, and the flush also adds the pending tau_j w_j of the steps
// since the last x update (in the two w buffers).
template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_minres_flush(long long n, long long per_case, const cpx<R> *__restrict__ ua,
                                                             const cpx<R> *__restrict__ ub, const cpx<R> *__restrict__ uc,
                                                             cpx<R> *__restrict__ wc, cpx<R> *__restrict__ wd,
                                                             cpx<R> *__restrict__ x, const MinresState *sts) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const MinresState *st = sts + i / per_case;   // the element's load case
        const int K = st->k;
        if (st->done_update || K <= 0) continue;
        // u_K: buffer K mod 3 of (ua, ub, uc), or K mod 2 of (ua, ub) without uc
        const cpx<R> *u = uc ? (K % 3 == 0 ? ua : (K % 3 == 1 ? ub : uc)) : ((K & 1) ? ub : ua);
        const cpx<R> *wa = (K & 1) ? wc : wd;      // w_{K-1}
        cpx<R> *wb = (K & 1) ? wd : wc;            // w_{K-2}, overwritten by w_K
        const R d = (R)st->u_delta, e = (R)st->u_eps, ig = (R)st->u_inv_gamma, tau = (R)st->u_tau,
                ib = (R)st->u_inv_beta;
        const cpx<R> uu = u[i], a = wa[i], b = wb[i], xx = x[i];
        const cpx<R> wn = mk<R>((uu.x * ib - d * a.x - e * b.x) * ig, (uu.y * ib - d * a.y - e * b.y) * ig);
        wb[i] = wn;
        // pending with the deferred update: w_{K-1} (r >= 1) and w_{K-2} (r = 2)
        const int r = uc ? (K - 1) % 3 : 0;
        const R t1 = r >= 1 ? (R)st->u_tau1 : (R)0, t2 = r == 2 ? (R)st->u_tau2 : (R)0;
        x[i] = mk<R>(xx.x + t2 * b.x + t1 * a.x + tau * wn.x, xx.y + t2 * b.y + t1 * a.y + tau * wn.y);
    }
}

// Parseval sums for the mean of phi times the projected fluctuation:
// partials[c][block] = sum over half-spectrum points of w Re(conj(phi^) (G x^)_c),
// w the half-spectrum weight; (1/V^2) times the total is <phi eps~_c>.
template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_phi_dot(Geometry g, const cpx<R> *__restrict__ x,
                                                        const cpx<R> *__restrict__ phihat, double *__restrict__ partials) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < g.S; f += (long long)gridDim.x * blockDim.x) {
        const int k3 = (int)(f % g.h);
        const long long r = f / g.h;
        const int k2 = (int)(r % g.n2), k1 = (int)(r / g.n2);
        cpx<R> t[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) t[c] = x[6 * f + c];
        gamma_at<R>(g, k1, k2, k3, t);
        const cpx<R> ph = phihat[f];
        const double w = (double)pweight(k3, g.n3);
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += w * ((double)ph.x * (double)t[c].x + (double)ph.y * (double)t[c].y);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const double sum = block_sum(acc[c]);
        if (threadIdx.x == 0) partials[c * gridDim.x + blockIdx.x] = sum;
    }
}

// Right-hand side from the DFT of phi: F{phi C_m : E_bar} = phi^ tau with the
// constant tau = C_m : E_bar, so b^ = -G (phi^ tau), eq. (gallin), one point-wise
// pass (tau: Mandel, units of E).
template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_rhs_phihat(Geometry g, const cpx<R> *__restrict__ phihat, Mac6 tau,
                                                           Mac6 sbar_v, cpx<R> *__restrict__ out) {
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < g.S; f += (long long)gridDim.x * blockDim.x) {
        const int k3 = (int)(f % g.h);
        const long long r = f / g.h;
        const int k2 = (int)(r % g.n2), k1 = (int)(r / g.n2);
        const cpx<R> ph = phihat[f];
        cpx<R> t[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) t[c] = mk<R>(-(R)tau.v[c] * ph.x, -(R)tau.v[c] * ph.y);
        // F{sigma_bar} = V sigma_bar at xi = 0 only: b^ = -G (phi^ tau - F{sigma_bar})
        if (f == 0) {
#pragma unroll
            for (int c = 0; c < 6; ++c) t[c].x += (R)sbar_v.v[c];
        }
        gamma_at<R>(g, k1, k2, k3, t);
#pragma unroll
        for (int c = 0; c < 6; ++c) out[6 * f + c] = t[c];
    }
}

// 10-component MoDBFFT input whose stress part is F{phi C_m : E_bar} =
// phi^ tau (times -1) and whose penalty part is zero
template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_phihat_tau10(long long S, const cpx<R> *__restrict__ phihat, Mac6 tau,
                                                             cpx<R> *__restrict__ out10) {
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < S; f += (long long)gridDim.x * blockDim.x) {
        const cpx<R> ph = phihat[f];
#pragma unroll
        for (int c = 0; c < 6; ++c) out10[10 * f + c] = mk<R>(-(R)tau.v[c] * ph.x, -(R)tau.v[c] * ph.y);
#pragma unroll
        for (int c = 6; c < 10; ++c) out10[10 * f + c] = mk<R>(0, 0);
    }
}

template <typename R>
__global__ void k_axpby(long long n, R a, const R *__restrict__ x, R b, R *__restrict__ y) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + (b != (R)0 ? b * y[i] : (R)0);
}

template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_norm2w(int n, int h, int n3, int nc, const cpx<R> *__restrict__ x,
                                                       double *partials) {
    Acc<R> acc;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const cpx<R> q = x[i];
        const R w = (R)pweight((i / nc) % h, n3);
        acc.add_prod(w * q.x, q.x);
        acc.add_prod(w * q.y, q.y);
    }
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
template <typename R>
int Launch<R>::ew_grid(long long n) {
    long long b = (n + kEwThreads - 1) / kEwThreads;
    return (int)(b < kEwBlocks ? (b > 0 ? b : 1) : kEwBlocks);
}
// CTAs of the n3 pass per load case (the grid is nb times this)
template <typename R>
int Launch<R>::x3_grid(const Geometry &g) { return (g.n1 * g.n2 + g.rows3 - 1) / g.rows3; }
// partials per load case written by the n3 pass of the fused chain
// (spectrum in and out): case c's are at [c * count, (c + 1) * count)
template <typename R>
int Launch<R>::x3_epart_grid(const Geometry &g) {
    if (sizeof(R) == 4 && g.x3r) return g.grid3r;
    return x3_grid(g);
}
template <typename R>
int Launch<R>::x3r_grid(const Geometry &g) {
    if constexpr (sizeof(R) != 4) {
        return 0;
    } else {
        int dev = 0, sms = 0, nb = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const size_t sm = x3r_smem(g.n3);
        switch (g.n3) {
            case 64: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_x3r<64>, kX3rWarps * 32, sm); break;
            case 128: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_x3r<128>, kX3rWarps * 32, sm); break;
            case 256: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_x3r<256>, kX3rWarps * 32, sm); break;
            default: return 0;
        }
        return nb * sms;
    }
}
// number of partial sums the dot-product variant of the n1 pass writes
template <typename R>
int Launch<R>::x1_grid(const Geometry &g) {
    return g.tma ? g.grid1d_tma : (g.n2 * g.h + g.tile1 - 1) / g.tile1;
}

#define HOM_FAST_SWITCH(n, CALL)                   \
    switch (n) {                                   \
        case 8: CALL(8); break;                    \
        case 16: CALL(16); break;                  \
        case 32: CALL(32); break;                  \
        case 64: CALL(64); break;                  \
        case 96: CALL(96); break;                  \
        case 128: CALL(128); break;                \
        case 160: CALL(160); break;                \
        case 256: CALL(256); break;                \
        case 512: CALL(512); break;                \
        default: CALL(0); break;                   \
    }

template <typename R>
void Launch<R>::table_init(const Geometry &) {
    // The dynamic shared-memory limit of each pass kernel is raised to the
    // device's opt-in maximum (a per-function setting shared by all contexts;
    // the launch's own size still decides occupancy).
    int dev = 0, lim = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // (the opt-in limit covers static plus dynamic shared memory, so each
    // kernel's own static share is taken off), and the L1/shared carve-out to
    // the largest shared share, so that the number of resident CTAs is set by
    // registers, not by a small carve-out
#define HOM_SET_ATTR1(K)                                                                        \
    {                                                                                           \
        cudaFuncAttributes fa_{};                                                               \
        cudaFuncGetAttributes(&fa_, K);                                                         \
        cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize,                    \
                             lim - (int)fa_.sharedSizeBytes);                                   \
        cudaFuncSetAttribute(K, cudaFuncAttributePreferredSharedMemoryCarveout,                 \
                             cudaSharedmemCarveoutMaxShared);                                   \
    }
#define HOM_SET_ATTR(NF)                \
    HOM_SET_ATTR1((k_x3<R, NF, 3>))     \
    HOM_SET_ATTR1((k_x3<R, NF, 5>))     \
    HOM_SET_ATTR1((k_x2<R, -1, NF>))    \
    HOM_SET_ATTR1((k_x2<R, 1, NF>))     \
    HOM_SET_ATTR1((k_x1<R, NF>))        \
    HOM_SET_ATTR1((k_x1_lanczos<R, NF>))
    HOM_SET_ATTR(0) HOM_SET_ATTR(8) HOM_SET_ATTR(16) HOM_SET_ATTR(32) HOM_SET_ATTR(64) HOM_SET_ATTR(96)
    HOM_SET_ATTR(128) HOM_SET_ATTR(160) HOM_SET_ATTR(256) HOM_SET_ATTR(512)
    if constexpr (sizeof(R) == 4) {
#define HOM_SET_TMA(NF)                   \
    HOM_SET_ATTR1((k_x2_tma<R, -1, NF>))  \
    HOM_SET_ATTR1((k_x2_tma<R, 1, NF>))   \
    HOM_SET_ATTR1((k_x1_tma<R, NF>))      \
    HOM_SET_ATTR1((k_x1_tma<R, NF, true>)) \
    HOM_SET_ATTR1((k_x1_tma_expand<R, NF>)) \
    HOM_SET_ATTR1((k_x1_lanczos_tma<R, NF>))
        HOM_SET_TMA(64) HOM_SET_TMA(96) HOM_SET_TMA(128) HOM_SET_TMA(160) HOM_SET_TMA(256) HOM_SET_TMA(512)
#undef HOM_SET_TMA
        HOM_SET_ATTR1((k_x3r<64>))
        HOM_SET_ATTR1((k_x3r<128>))
        HOM_SET_ATTR1((k_x3r<256>))
    }
#undef HOM_SET_ATTR
#undef HOM_SET_ATTR1
}

// persistent-grid sizes of the TMA passes: resident CTAs per SM x SMs
template <typename R>
int Launch<R>::tma_grids(Geometry &g) {
    if constexpr (sizeof(R) != 4) {
        g.tma = 0;
        return 0;
    } else {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int b2 = 0, b1 = 0, b1d = 0;
        auto occ = [&](auto kern, int threads, size_t smem) {
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
            return nb;
        };
        switch (g.fast[1]) {
            case 64: b2 = occ(k_x2_tma<R, -1, 64>, g.threads2, g.smem2_tma); break;
            case 96: b2 = occ(k_x2_tma<R, -1, 96>, g.threads2, g.smem2_tma); break;
            case 160: b2 = occ(k_x2_tma<R, -1, 160>, g.threads2, g.smem2_tma); break;
            case 512: b2 = occ(k_x2_tma<R, -1, 512>, g.threads2, g.smem2_tma); break;
            case 128: b2 = occ(k_x2_tma<R, -1, 128>, g.threads2, g.smem2_tma); break;
            default: b2 = occ(k_x2_tma<R, -1, 256>, g.threads2, g.smem2_tma); break;
        }
        switch (g.fast[0]) {
            case 64: b1 = occ(k_x1_tma<R, 64>, g.threads1, g.smem1_tma);
                     b1d = occ(k_x1_tma<R, 64>, g.threads1, g.smem1d_tma); break;
            case 96: b1 = occ(k_x1_tma<R, 96>, g.threads1, g.smem1_tma);
                     b1d = occ(k_x1_tma<R, 96>, g.threads1, g.smem1d_tma); break;
            case 160: b1 = occ(k_x1_tma<R, 160>, g.threads1, g.smem1_tma);
                      b1d = occ(k_x1_tma<R, 160>, g.threads1, g.smem1d_tma); break;
            case 512: b1 = occ(k_x1_tma<R, 512>, g.threads1, g.smem1_tma);
                      b1d = occ(k_x1_tma<R, 512>, g.threads1, g.smem1d_tma); break;
            case 128: b1 = occ(k_x1_tma<R, 128>, g.threads1, g.smem1_tma);
                      b1d = occ(k_x1_tma<R, 128>, g.threads1, g.smem1d_tma); break;
            default: b1 = occ(k_x1_tma<R, 256>, g.threads1, g.smem1_tma);
                     b1d = occ(k_x1_tma<R, 256>, g.threads1, g.smem1d_tma); break;
        }
        if (b2 < 1 || b1 < 1 || b1d < 1) {
            g.tma = 0;
            return 0;
        }
        // the fused MINRES n1 pass: a transform group of exactly kX1Group
        // threads plus the lagged-update warps, whose ring takes as many
        // stages (up to kX1LagMaxStages) as leave room for two CTAs per SM
        int b1l = 0;
        if (g.nc == 6 && g.threads1 == kX1Group) {
            const int t = kX1Group + kX1LagThreads;
            int smem_sm = 0;
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            const size_t ring = 4 * (size_t)kX1LagChunk, fixed = 15 * 1024;   // static + reserved per CTA
            int st = kX1LagMaxStages;
            while (st > 1 && 2 * (g.smem1_tma + st * ring + fixed) > (size_t)smem_sm) --st;
            g.x1_lag_stages = st;
            g.smem1l_tma = g.smem1_tma + st * ring;
            switch (g.fast[0]) {
                case 64: b1l = occ(k_x1_lanczos_tma<R, 64>, t, g.smem1l_tma); break;
                case 96: b1l = occ(k_x1_lanczos_tma<R, 96>, t, g.smem1l_tma); break;
                case 160: b1l = occ(k_x1_lanczos_tma<R, 160>, t, g.smem1l_tma); break;
                case 512: b1l = occ(k_x1_lanczos_tma<R, 512>, t, g.smem1l_tma); break;
                case 128: b1l = occ(k_x1_lanczos_tma<R, 128>, t, g.smem1l_tma); break;
                default: b1l = occ(k_x1_lanczos_tma<R, 256>, t, g.smem1l_tma); break;
            }
        }
        g.grid1l_tma = b1l * sms;
        g.grid2_tma = b2 * sms;
        g.grid1_tma = b1 * sms;
        g.grid1d_tma = b1d * sms;
        return 1;
    }
}

template <typename R>
void Launch<R>::x3(const Geometry &g, cudaStream_t st, int in_mode, const void *in, int mid, double lam, double mu,
                   const double *macro, double scl, int out_mode, void *out, const R *phi,
                   const MinresState *state, double *epart, Fold fold, double *tsum) {
    if constexpr (sizeof(R) == 4) {
        if (!tsum && g.x3r && g.nc == 6 && in_mode == X3_IN_SPEC && out_mode == X3_OUT_SPEC && scl == 1.0 &&
            (mid == X3_MID_MATERIAL || mid == X3_MID_NONE)) {
            const int grid = g.grid3r;   // persistent: every case's row groups
            const size_t sm = x3r_smem(g.n3);
            const int mat = mid == X3_MID_MATERIAL;
            const float2 *fi = reinterpret_cast<const float2 *>(in);
            float2 *fo = reinterpret_cast<float2 *>(out);
            switch (g.n3) {
                case 64: launch_k(g.pdl, k_x3r<64>, grid, 128, sm, st, g, fi, fo, mat, (float)lam, (float)(2.0 * mu),
                                                          (const float *)phi, state, epart, fold); break;
                case 128: launch_k(g.pdl, k_x3r<128>, grid, 128, sm, st, g, fi, fo, mat, (float)lam, (float)(2.0 * mu),
                                                            (const float *)phi, state, epart, fold); break;
                default: launch_k(g.pdl, k_x3r<256>, grid, 128, sm, st, g, fi, fo, mat, (float)lam, (float)(2.0 * mu),
                                                            (const float *)phi, state, epart, fold); break;
            }
            return;
        }
    }
    Mac6 m{};
    if (macro)
        for (int c = 0; c < 6; ++c) m.v[c] = macro[c];
    const int grid = x3_grid(g) * g.nb;
#define HOM_X3(NF)                                                                                          \
    if (g.nc == 10)                                                                                         \
        launch_k(g.pdl, k_x3<R, NF, 5>, grid, g.threads3, g.smem3, st, g, in_mode, in, mid, (R)lam, (R)(2.0 * mu), m, \
                                                            (R)scl, out_mode, out, phi, state, nullptr, Fold{}, nullptr); \
    else                                                                                                    \
        launch_k(g.pdl, k_x3<R, NF, 3>, grid, g.threads3, g.smem3, st, g, in_mode, in, mid, (R)lam, (R)(2.0 * mu), m, \
                                                            (R)scl, out_mode, out, phi, state, epart, fold, tsum)
    HOM_FAST_SWITCH(g.fast[2], HOM_X3)
#undef HOM_X3
}

template <typename R>
void Launch<R>::x2(const Geometry &g, cudaStream_t st, int inverse, cpx<R> *spec, const MinresState *state) {
    if constexpr (sizeof(R) == 4) {
        if (g.tma) {
            const CUtensorMap *tm = tma_map(g, spec, TMA_X2, 1);
            const int qtiles = (g.nc * g.h + g.tile2 - 1) / g.tile2;
#define HOM_X2T(NF)                                                                                         \
    if (inverse) launch_k(g.pdl, k_x2_tma<R, 1, NF>, g.grid2_tma, g.threads2, g.smem2_tma, st, g, *tm, qtiles, state); \
    else launch_k(g.pdl, k_x2_tma<R, -1, NF>, g.grid2_tma, g.threads2, g.smem2_tma, st, g, *tm, qtiles, state)
            switch (g.fast[1]) {
                case 64: HOM_X2T(64); break;
                case 96: HOM_X2T(96); break;
                case 160: HOM_X2T(160); break;
                case 512: HOM_X2T(512); break;
                case 128: HOM_X2T(128); break;
                default: HOM_X2T(256); break;
            }
#undef HOM_X2T
            return;
        }
    }
    const int grid = (g.n1 * g.nb * g.nc * g.h + g.tile2 - 1) / g.tile2;
#define HOM_X2(NF)                                                                  \
    if (inverse) launch_k(g.pdl, k_x2<R, 1, NF>, grid, g.threads2, g.smem2, st, g, spec, state); \
    else launch_k(g.pdl, k_x2<R, -1, NF>, grid, g.threads2, g.smem2, st, g, spec, state)
    HOM_FAST_SWITCH(g.fast[1], HOM_X2)
#undef HOM_X2
}

template <typename R>
void Launch<R>::x1(const Geometry &g, cudaStream_t st, int flags, const cpx<R> *in, cpx<R> *out, const cpx<R> *dotv,
                   double *partials, const MinresState *state) {
    if constexpr (sizeof(R) == 4) {
        if (g.tma) {
            const bool dot = (flags & X1_DOT) != 0;
            const CUtensorMap *ti = tma_map(g, in, TMA_X1, 1);
            const CUtensorMap *to = tma_map(g, out, TMA_X1, 1);
            const CUtensorMap *td = dot ? tma_map(g, dotv, TMA_X1, 1) : ti;
            const int grid = dot ? g.grid1d_tma : g.grid1_tma;
            const size_t sm = dot ? g.smem1d_tma : g.smem1_tma;
#define HOM_X1T(NF) k_x1_tma<R, NF><<<grid, g.threads1, sm, st>>>(g, flags, *ti, *to, *td, partials, state, nullptr, nullptr)
            switch (g.fast[0]) {
                case 64: HOM_X1T(64); break;
                case 96: HOM_X1T(96); break;
                case 160: HOM_X1T(160); break;
                case 512: HOM_X1T(512); break;
                case 128: HOM_X1T(128); break;
                default: HOM_X1T(256); break;
            }
#undef HOM_X1T
            return;
        }
    }
    const int grid = (g.n2 * g.h + g.tile1 - 1) / g.tile1;
#define HOM_X1(NF) k_x1<R, NF><<<grid, g.threads1, g.smem1, st>>>(g, flags, in, out, dotv, partials, state)
    HOM_FAST_SWITCH(g.fast[0], HOM_X1)
#undef HOM_X1
}

template <typename R>
int Launch<R>::x1_modb_contract(const Geometry &g, cudaStream_t st, const cpx<R> *in10, cpx<R> *out3,
                                const cpx<R> *dot3, double *partials, int max_partials, const MinresState *state) {
    if constexpr (sizeof(R) == 4) {
        if (g.tma && g.nc == 10 && g.grid1_tma > 0 && (!dot3 || g.grid1_tma <= max_partials)) {
            const CUtensorMap *ti = tma_map(g, in10, TMA_X1, 1);
#define HOM_X1C(NF)                                                                                              \
    k_x1_tma<R, NF, true><<<g.grid1_tma, g.threads1, g.smem1_tma, st>>>(g, X1_FWD, *ti, *ti, *ti, partials, state, \
                                                                      out3, dot3)
            switch (g.fast[0]) {
                case 64: HOM_X1C(64); break;
                case 96: HOM_X1C(96); break;
                case 160: HOM_X1C(160); break;
                case 512: HOM_X1C(512); break;
                case 128: HOM_X1C(128); break;
                default: HOM_X1C(256); break;
            }
#undef HOM_X1C
            return g.grid1_tma;
        }
    }
    return 0;
}

template <typename R>
bool Launch<R>::x1_modb_expand(const Geometry &g, cudaStream_t st, double alpha, const cpx<R> *u3, cpx<R> *out10,
                               const MinresState *state) {
    if constexpr (sizeof(R) == 4) {
        if (g.tma && g.nc == 10 && g.grid1_tma > 0) {
            const CUtensorMap *to = tma_map(g, out10, TMA_X1, 1);
            if (!to) return false;
#define HOM_X1E(NF) \
    k_x1_tma_expand<R, NF><<<g.grid1_tma, g.threads1, g.smem1_tma, st>>>(g, *to, u3, (R)alpha, state)
            switch (g.fast[0]) {
                case 64: HOM_X1E(64); break;
                case 96: HOM_X1E(96); break;
                case 160: HOM_X1E(160); break;
                case 512: HOM_X1E(512); break;
                case 128: HOM_X1E(128); break;
                default: HOM_X1E(256); break;
            }
#undef HOM_X1E
            return true;
        }
    }
    return false;
}

// partials per load case written by the fused n1 pass (case c's at c * count)
template <typename R>
int Launch<R>::x1_lanczos_grid(const Geometry &g) {
    return (g.tma && g.grid1l_tma > 0) ? g.grid1l_tma : (g.n2 * g.h + g.tile1 - 1) / g.tile1;
}

template <typename R>
void Launch<R>::x1_lanczos(const Geometry &g, cudaStream_t st, cpx<R> *spec, const cpx<R> *uk, const cpx<R> *um,
                           cpx<R> *un, const cpx<R> *wa, cpx<R> *wb, cpx<R> *x, const MinresState *state,
                           double *partials, Fold fold) {
    if constexpr (sizeof(R) == 4) {
        if (g.tma && g.grid1l_tma > 0) {
            const CUtensorMap *ts = tma_map(g, spec, TMA_X1, 1);
#define HOM_X1LT(NF)                                                                                         \
    launch_k(g.pdl, k_x1_lanczos_tma<R, NF>, g.grid1l_tma, kX1Group + kX1LagThreads, g.smem1l_tma, st, g, *ts, uk, um, \
             un, wa, wb, x, state, partials, fold)
            switch (g.fast[0]) {
                case 64: HOM_X1LT(64); break;
                case 96: HOM_X1LT(96); break;
                case 160: HOM_X1LT(160); break;
                case 512: HOM_X1LT(512); break;
                case 128: HOM_X1LT(128); break;
                default: HOM_X1LT(256); break;
            }
#undef HOM_X1LT
            return;
        }
    }
    const int grid = (g.n2 * g.h + g.tile1 - 1) / g.tile1 * g.nb;
#define HOM_X1L(NF) \
    launch_k(g.pdl, k_x1_lanczos<R, NF>, grid, g.threads1, g.smem1, st, g, spec, uk, um, un, wa, wb, x, state, partials, \
             fold)
    HOM_FAST_SWITCH(g.fast[0], HOM_X1L)
#undef HOM_X1L
}

template <typename R>
void Launch<R>::to_tiles(const Geometry &g, cudaStream_t st, const cpx<R> *in, cpx<R> *out) {
    const long long n = 6 * g.S;
    k_tiles<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, g.n1, g.n2 * g.h, g.tile1, 1, in, out);
}

template <typename R>
void Launch<R>::from_tiles(const Geometry &g, cudaStream_t st, const cpx<R> *in, cpx<R> *out) {
    const long long n = 6 * g.S;
    k_tiles<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, g.n1, g.n2 * g.h, g.tile1, 0, in, out);
}

template <typename R>
void Launch<R>::lanczos_update(const Geometry &g, cudaStream_t st, const cpx<R> *p, const cpx<R> *uk, cpx<R> *um,
                               const cpx<R> *wa, cpx<R> *wb, cpx<R> *x, const MinresState *state, double *partials) {
    const int n = (int)(6 * g.S);
    k_lanczos_update<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, g.h, g.n3, p, uk, um, wa, wb, x, state, partials);
}

template <typename R>
void Launch<R>::minres_flush(const Geometry &g, cudaStream_t st, const cpx<R> *ua, const cpx<R> *ub, const cpx<R> *uc,
                             cpx<R> *wc, cpx<R> *wd, cpx<R> *x, MinresState *state, long long per_case) {
    const long long n = per_case * g.nb;
    k_minres_flush<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, per_case, ua, ub, uc, wc, wd, x, state);
}

template <typename R>
int Launch<R>::phi_dot(const Geometry &g, cudaStream_t st, const cpx<R> *x, const cpx<R> *phihat, double *partials) {
    const int nb = ew_grid(g.S);
    k_phi_dot<R><<<nb, kEwThreads, 0, st>>>(g, x, phihat, partials);
    return nb;
}

template <typename R>
void Launch<R>::rhs_phihat(const Geometry &g, cudaStream_t st, const cpx<R> *phihat, const double *tau,
                           const double *sbar_v, cpx<R> *out) {
    Mac6 m{}, sv{};
    for (int c = 0; c < 6; ++c) {
        m.v[c] = tau[c];
        sv.v[c] = sbar_v ? sbar_v[c] : 0.0;
    }
    k_rhs_phihat<R><<<ew_grid(g.S), kEwThreads, 0, st>>>(g, phihat, m, sv, out);
}

template <typename R>
void Launch<R>::phihat_tau10(const Geometry &g, cudaStream_t st, const cpx<R> *phihat, const double *tau, cpx<R> *out10) {
    Mac6 m{};
    for (int c = 0; c < 6; ++c) m.v[c] = tau[c];
    k_phihat_tau10<R><<<ew_grid(g.S), kEwThreads, 0, st>>>(g.S, phihat, m, out10);
}

template <typename R>
void Launch<R>::axpby(long long n, cudaStream_t st, double a, const R *x, double b, R *y) {
    k_axpby<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, (R)a, x, (R)b, y);
}

template <typename R>
void Launch<R>::norm2w(const Geometry &g, cudaStream_t st, const cpx<R> *x, double *partials, int nc) {
    const int n = (int)(nc * g.S);
    k_norm2w<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, g.h, g.n3, nc, x, partials);
}

}  // namespace hom

#include "hom_modb.cuh"
