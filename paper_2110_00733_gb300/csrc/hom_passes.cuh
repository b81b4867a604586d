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

// G at frequency (k1,k2,k3) on the 6 Mandel components at p[0..5] (stride 1)
template <typename R>
__device__ __forceinline__ void gamma_at(const Geometry &g, int k1, int k2, int k3, cpx<R> *t) {
    // eq. (galop): at xi = 0 the identity on the stress-controlled components
    // (g.mask0) and zero on the strain-controlled ones; zero at every
    // frequency with a Nyquist index
    if (k1 == 0 && k2 == 0 && k3 == 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c)
            if (!((g.mask0 >> c) & 1)) t[c] = mk<R>(0, 0);
        return;
    }
    const bool nyq = ((g.n1 & 1) == 0 && 2 * k1 == g.n1) || ((g.n2 & 1) == 0 && 2 * k2 == g.n2) ||
                     ((g.n3 & 1) == 0 && 2 * k3 == g.n3);
    if (nyq) {
#pragma unroll
        for (int c = 0; c < 6; ++c) t[c] = mk<R>(0, 0);
        return;
    }
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
    gamma_project<R>(t, x0, x1, x2);
}

// Run the transform of the L lines in buf.  Fast engine: in place, returns
// buf.  Generic engine: ping-pong with buf2, returns the buffer holding the
// result.
template <typename R, int S, int NF, int PAD = 0>
__device__ __forceinline__ cpx<R> *run_fft(cpx<R> *buf, cpx<R> *buf2, int L, int ES, const AxisPlan &p) {
    if constexpr (NF > 0) {
        fast_fft<R, S, NF, PAD>(buf, L, ES, reinterpret_cast<const cpx<R> *>(p.tw));
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

// ---------------------------------------------------------------------------
// n3 pass.  A CTA owns rows (k1,k2) [row0, row0+rows3); lines are the three
// component pairs (2p, 2p+1) of each row packed as one complex line
// Z = X_2p + i X_2p+1, line index p*rows3 + r.
// ---------------------------------------------------------------------------
template <typename R, int NF, int NP>
__global__ void HOM_PASS_BOUNDS(R) k_x3(Geometry g, int in_mode, const void *__restrict__ in_, int mid, R lam,
                                        R mu2, Mac6 mac, R scl, int out_mode, void *__restrict__ out_,
                                        const R *__restrict__ phi, const MinresState *state) {
    if (skip(state)) return;
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
    const int row0 = blockIdx.x * ROWS;
    const int V = (int)g.V;
    const int nr = min(ROWS, nrows - row0);
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
        cpx<R> *res = run_fft<R, 1, NF, PAD>(buf, buf2, L, ES, g.ax[2]);
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
                const R tr = lam * (t[0] + t[1] + t[2]);
#pragma unroll
                for (int c = 0; c < 6; ++c) t[c] = ph * ((c < 3 ? tr : (R)0) + mu2 * t[c]);
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
    if (out_mode == X3_OUT_REAL) return;
    // rows beyond nrows hold zeros already (their inputs were zero)
    __syncthreads();
    cpx<R> *res = run_fft<R, -1, NF, PAD>(buf, buf2, L, ES, g.ax[2]);
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
// n2 pass, in place.  Columns are (k1, k3, c) flattened, f = k1 * 6h + q;
// element k2 of column f is at (k1 n2 + k2) 6h + q.  tile2 consecutive
// columns per CTA (contiguous runs of tile2 complex values).
// ---------------------------------------------------------------------------
template <typename R, int S, int NF>
__global__ void HOM_PASS_BOUNDS(R) k_x2(Geometry g, cpx<R> *__restrict__ spec, const MinresState *state) {
    if (skip(state)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int N = g.n2, T = g.tile2, H6 = g.nc * g.h;
    cpx<R> *buf = reinterpret_cast<cpx<R> *>(smem_raw);
    cpx<R> *buf2 = buf + N * T;
    const int total = g.n1 * H6;
    const int t = threadIdx.x % T, e0 = threadIdx.x / T, es = blockDim.x / T;
    const int f = blockIdx.x * T + t;
    const bool live = f < total;
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
__global__ void HOM_PASS_BOUNDS(R) k_x1(Geometry g, int flags, const cpx<R> *__restrict__ in,
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

// ---------------------------------------------------------------------------
// Persistent TMA-staged n2 and n1 passes (FP32, n <= 256, fast engine).
// Each CTA loops over tiles with two shared-memory stages: while the FFT runs
// on stage s, the TMA load of the next tile fills stage s^1; results leave by
// TMA store.  One thread issues all copies; completion is tracked by one
// mbarrier per stage.  Every wait is bounded: on time-out the CTA records
// the failure in *g.err, waits (bounded) for its own load in flight and
// returns, and the host reports HOM_ETIMEOUT.
// ---------------------------------------------------------------------------
template <typename R, int S, int NF>
__global__ void HOM_PASS_BOUNDS(R) k_x2_tma(Geometry g, const __grid_constant__ CUtensorMap tm, int qtiles,
                                            const MinresState *state) {
    if (skip(state)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    const int N = g.n2, T = g.tile2;
    const int ntiles = g.n1 * qtiles;
    cpx<R> *const base = reinterpret_cast<cpx<R> *>(smem_raw);
    const int per = N * T;   // stage s starts at base + s * per
    const uint32_t bytes = (uint32_t)(per * sizeof(cpx<R>));
    const bool leader = threadIdx.x == 0;
    if (leader) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int tile = blockIdx.x;
    if (leader && tile < ntiles) {
        mbar_expect_tx(&bar[0], bytes);
        tma_load_3d(base, &tm, (tile % qtiles) * T, 0, tile / qtiles, &bar[0]);
    }
    const cpx<R> *tw = reinterpret_cast<const cpx<R> *>(g.ax[1].tw);
    for (int i = 0; tile < ntiles; ++i, tile += gridDim.x) {
        const int s = i & 1;
        const int next = tile + gridDim.x;
        if (leader && next < ntiles) {
            bulk_wait_read_all();   // the store of the tile that used stage s^1 has read it
            mbar_expect_tx(&bar[s ^ 1], bytes);
            tma_load_3d(base + (s ^ 1) * per, &tm, (next % qtiles) * T, 0, next / qtiles, &bar[s ^ 1]);
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
        fast_fft<R, S, NF>(buf, T, T, tw);
        fence_proxy_async_smem();
        __syncthreads();
        if (leader) {
            tma_store_3d(&tm, (tile % qtiles) * T, 0, tile / qtiles, buf);
            bulk_commit();
        }
    }
    if (leader) bulk_wait_all();
}

template <typename R, int NF>
__global__ void HOM_PASS_BOUNDS(R) k_x1_tma(Geometry g, int flags, const __grid_constant__ CUtensorMap tin,
                                            const __grid_constant__ CUtensorMap tout,
                                            const __grid_constant__ CUtensorMap tdot, double *__restrict__ partials,
                                            const MinresState *state) {
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
        tma_load_2d(base + s * per, &tin, NC * T * t, 0, &bar[s]);
        if (dot) tma_load_2d(base + s * per + tile_elems, &tdot, NC * T * t, 0, &bar[s]);
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
            tma_store_2d(&tout, NC * T * tile, 0, buf);
            bulk_commit();
        }
    }
    if (leader) bulk_wait_all();
    if (dot) {
        const double sum = block_sum(acc.value());
        if (threadIdx.x == 0) partials[blockIdx.x] = sum;
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

// The lagged w / x update of the last step K; skipped when there is none
// or the state kept the last finite iterate.
template <typename R>
__global__ void __launch_bounds__(kEwThreads) k_minres_flush(int n, const cpx<R> *__restrict__ ua,
                                                             const cpx<R> *__restrict__ ub, cpx<R> *__restrict__ wc,
                                                             cpx<R> *__restrict__ wd, cpx<R> *__restrict__ x,
                                                             const MinresState *st) {
    const int K = st->k;
    if (st->done_update || K <= 0) return;
    const cpx<R> *u = (K & 1) ? ub : ua;
    const cpx<R> *wa = (K & 1) ? wc : wd;      // w_{K-1}
    cpx<R> *wb = (K & 1) ? wd : wc;            // w_{K-2}, overwritten by w_K
    const R d = (R)st->u_delta, e = (R)st->u_eps, ig = (R)st->u_inv_gamma, tau = (R)st->u_tau,
            ib = (R)st->u_inv_beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const cpx<R> uu = u[i], a = wa[i], b = wb[i], xx = x[i];
        const cpx<R> wn = mk<R>((uu.x * ib - d * a.x - e * b.x) * ig, (uu.y * ib - d * a.y - e * b.y) * ig);
        wb[i] = wn;
        x[i] = mk<R>(xx.x + tau * wn.x, xx.y + tau * wn.y);
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
template <typename R>
int Launch<R>::x3_grid(const Geometry &g) { return (g.n1 * g.n2 + g.rows3 - 1) / g.rows3; }
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
        case 128: CALL(128); break;                \
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
    lim -= 1024;   // static shared memory of the reductions
    // and the L1/shared carve-out to the largest shared share, so that the
    // number of resident CTAs is set by registers, not by a small carve-out
#define HOM_SET_ATTR1(K)                                                                        \
    cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);                  \
    cudaFuncSetAttribute(K, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
#define HOM_SET_ATTR(NF)                \
    HOM_SET_ATTR1((k_x3<R, NF, 3>))     \
    HOM_SET_ATTR1((k_x3<R, NF, 5>))     \
    HOM_SET_ATTR1((k_x2<R, -1, NF>))    \
    HOM_SET_ATTR1((k_x2<R, 1, NF>))     \
    HOM_SET_ATTR1((k_x1<R, NF>))
    HOM_SET_ATTR(0) HOM_SET_ATTR(8) HOM_SET_ATTR(16) HOM_SET_ATTR(32) HOM_SET_ATTR(64) HOM_SET_ATTR(128)
    HOM_SET_ATTR(256) HOM_SET_ATTR(512)
    if constexpr (sizeof(R) == 4) {
#define HOM_SET_TMA(NF)                   \
    HOM_SET_ATTR1((k_x2_tma<R, -1, NF>))  \
    HOM_SET_ATTR1((k_x2_tma<R, 1, NF>))   \
    HOM_SET_ATTR1((k_x1_tma<R, NF>))
        HOM_SET_TMA(64) HOM_SET_TMA(128) HOM_SET_TMA(256)
#undef HOM_SET_TMA
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
            case 128: b2 = occ(k_x2_tma<R, -1, 128>, g.threads2, g.smem2_tma); break;
            default: b2 = occ(k_x2_tma<R, -1, 256>, g.threads2, g.smem2_tma); break;
        }
        switch (g.fast[0]) {
            case 64: b1 = occ(k_x1_tma<R, 64>, g.threads1, g.smem1_tma);
                     b1d = occ(k_x1_tma<R, 64>, g.threads1, g.smem1d_tma); break;
            case 128: b1 = occ(k_x1_tma<R, 128>, g.threads1, g.smem1_tma);
                      b1d = occ(k_x1_tma<R, 128>, g.threads1, g.smem1d_tma); break;
            default: b1 = occ(k_x1_tma<R, 256>, g.threads1, g.smem1_tma);
                     b1d = occ(k_x1_tma<R, 256>, g.threads1, g.smem1d_tma); break;
        }
        if (b2 < 1 || b1 < 1 || b1d < 1) {
            g.tma = 0;
            return 0;
        }
        g.grid2_tma = b2 * sms;
        g.grid1_tma = b1 * sms;
        g.grid1d_tma = b1d * sms;
        return 1;
    }
}

template <typename R>
void Launch<R>::x3(const Geometry &g, cudaStream_t st, int in_mode, const void *in, int mid, double lam, double mu,
                   const double *macro, double scl, int out_mode, void *out, const R *phi,
                   const MinresState *state) {
    Mac6 m{};
    if (macro)
        for (int c = 0; c < 6; ++c) m.v[c] = macro[c];
    const int grid = x3_grid(g);
#define HOM_X3(NF)                                                                                          \
    if (g.nc == 10)                                                                                         \
        k_x3<R, NF, 5><<<grid, g.threads3, g.smem3, st>>>(g, in_mode, in, mid, (R)lam, (R)(2.0 * mu), m,       \
                                                            (R)scl, out_mode, out, phi, state);                \
    else                                                                                                    \
        k_x3<R, NF, 3><<<grid, g.threads3, g.smem3, st>>>(g, in_mode, in, mid, (R)lam, (R)(2.0 * mu), m,       \
                                                            (R)scl, out_mode, out, phi, state)
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
    if (inverse) k_x2_tma<R, 1, NF><<<g.grid2_tma, g.threads2, g.smem2_tma, st>>>(g, *tm, qtiles, state);    \
    else k_x2_tma<R, -1, NF><<<g.grid2_tma, g.threads2, g.smem2_tma, st>>>(g, *tm, qtiles, state)
            switch (g.fast[1]) {
                case 64: HOM_X2T(64); break;
                case 128: HOM_X2T(128); break;
                default: HOM_X2T(256); break;
            }
#undef HOM_X2T
            return;
        }
    }
    const int grid = (g.n1 * g.nc * g.h + g.tile2 - 1) / g.tile2;
#define HOM_X2(NF)                                                                  \
    if (inverse) k_x2<R, 1, NF><<<grid, g.threads2, g.smem2, st>>>(g, spec, state); \
    else k_x2<R, -1, NF><<<grid, g.threads2, g.smem2, st>>>(g, spec, state)
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
#define HOM_X1T(NF) k_x1_tma<R, NF><<<grid, g.threads1, sm, st>>>(g, flags, *ti, *to, *td, partials, state)
            switch (g.fast[0]) {
                case 64: HOM_X1T(64); break;
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
void Launch<R>::lanczos_update(const Geometry &g, cudaStream_t st, const cpx<R> *p, const cpx<R> *uk, cpx<R> *um,
                               const cpx<R> *wa, cpx<R> *wb, cpx<R> *x, const MinresState *state, double *partials) {
    const int n = (int)(6 * g.S);
    k_lanczos_update<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, g.h, g.n3, p, uk, um, wa, wb, x, state, partials);
}

template <typename R>
void Launch<R>::minres_flush(const Geometry &g, cudaStream_t st, const cpx<R> *ua, const cpx<R> *ub, cpx<R> *wc,
                             cpx<R> *wd, cpx<R> *x, MinresState *state) {
    const int n = (int)(6 * g.S);
    k_minres_flush<R><<<ew_grid(n), kEwThreads, 0, st>>>(n, ua, ub, wc, wd, x, state);
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
