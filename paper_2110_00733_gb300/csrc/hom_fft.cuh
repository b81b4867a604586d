// hom_fft.cuh -- shared-memory mixed-radix FFT engine for the batched 3-D
// real FFTs of the Galerkin operator (section 2.1: the transforms of
// eq. (gal) are discrete Fourier transforms evaluated with an FFT).
//
// A CTA holds a batch of L lines of one axis in shared memory, element e of
// line l at buf[e*ES + l] with ES >= L (lines interleaved, so that the threads
// of a warp touch consecutive words whatever the stage's index pattern), and runs
// Stockham auto-sort stages between two buffers.  Each stage applies radix-R
// butterflies (R in {2,3,4,5,8,16}) held in registers; twiddles come from a
// per-axis table w[t] = exp(-2 pi i t / N) computed on the host in double.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hom {

template <typename R> struct cpx_t;
template <> struct cpx_t<float> { using type = float2; };
template <> struct cpx_t<double> { using type = double2; };
template <typename R> using cpx = typename cpx_t<R>::type;

template <typename R> __device__ __forceinline__ cpx<R> mk(R x, R y) { cpx<R> c; c.x = x; c.y = y; return c; }
template <typename R> __device__ __forceinline__ cpx<R> add(cpx<R> a, cpx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R> __device__ __forceinline__ cpx<R> sub(cpx<R> a, cpx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R> __device__ __forceinline__ cpx<R> mul(cpx<R> a, cpx<R> b) {
    return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R> __device__ __forceinline__ cpx<R> conjc(cpx<R> a) { return mk<R>(a.x, -a.y); }
template <typename R> __device__ __forceinline__ cpx<R> scale(cpx<R> a, R s) { return mk<R>(a.x * s, a.y * s); }
// multiply by s*i (s = +1 or -1)
template <typename R> __device__ __forceinline__ cpx<R> mul_si(cpx<R> a, int s) {
    return s > 0 ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x);
}

constexpr int kMaxStages = 8;

struct AxisPlan {
    int n;                    // transform length
    int nstages;
    int radix[kMaxStages];
    const void *tw;           // n complex values exp(-2 pi i t / n) (float2 or double2)
};

// ---------------------------------------------------------------------------
// In-register DFT codelets, kernel exp(S * 2 pi i j k / R), S = -1 forward.
// Constants are closed-form values: cos(2pi/5) = (sqrt5-1)/4, etc.
// ---------------------------------------------------------------------------
template <typename R, int S> __device__ __forceinline__ void dft2(cpx<R> &a, cpx<R> &b) {
    cpx<R> t = a;
    a = add<R>(t, b);
    b = sub<R>(t, b);
}

template <typename R, int S> __device__ __forceinline__ void dft3(cpx<R> *v) {
    const R h = (R)0.86602540378443864676;  // sqrt(3)/2
    cpx<R> t = add<R>(v[1], v[2]), u = sub<R>(v[1], v[2]);
    cpx<R> m = sub<R>(v[0], scale<R>(t, (R)0.5));
    cpx<R> r = mul_si<R>(scale<R>(u, h), S);
    v[0] = add<R>(v[0], t);
    v[1] = add<R>(m, r);
    v[2] = sub<R>(m, r);
}

template <typename R, int S> __device__ __forceinline__ void dft4(cpx<R> *v) {
    cpx<R> a = add<R>(v[0], v[2]), b = sub<R>(v[0], v[2]);
    cpx<R> c = add<R>(v[1], v[3]), d = mul_si<R>(sub<R>(v[1], v[3]), S);
    v[0] = add<R>(a, c);
    v[2] = sub<R>(a, c);
    v[1] = add<R>(b, d);
    v[3] = sub<R>(b, d);
}

template <typename R, int S> __device__ __forceinline__ void dft5(cpx<R> *v) {
    const R c1 = (R)0.30901699437494742410;   // cos(2pi/5)
    const R c2 = (R)-0.80901699437494742410;  // cos(4pi/5)
    const R s1 = (R)0.95105651629515357212;   // sin(2pi/5)
    const R s2 = (R)0.58778525229247312917;   // sin(4pi/5)
    cpx<R> t1 = add<R>(v[1], v[4]), t2 = add<R>(v[2], v[3]);
    cpx<R> u1 = sub<R>(v[1], v[4]), u2 = sub<R>(v[2], v[3]);
    cpx<R> a = v[0];
    cpx<R> m1 = mk<R>(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
    cpx<R> m2 = mk<R>(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
    cpx<R> n1 = mul_si<R>(mk<R>(s1 * u1.x + s2 * u2.x, s1 * u1.y + s2 * u2.y), S);
    cpx<R> n2 = mul_si<R>(mk<R>(s2 * u1.x - s1 * u2.x, s2 * u1.y - s1 * u2.y), S);
    v[0] = add<R>(a, add<R>(t1, t2));
    v[1] = add<R>(m1, n1);
    v[4] = sub<R>(m1, n1);
    v[2] = add<R>(m2, n2);
    v[3] = sub<R>(m2, n2);
}

// exp(S * 2 pi i k / 16) for k = 0..7
template <typename R, int S> __device__ __forceinline__ cpx<R> w16(int k) {
    const R c = (R)0.92387953251128675613;   // cos(pi/8)
    const R s = (R)0.38268343236508977173;   // sin(pi/8)
    const R h = (R)0.70710678118654752440;   // sqrt(1/2)
    R re, im;
    switch (k) {
        case 0: re = 1; im = 0; break;
        case 1: re = c; im = s; break;
        case 2: re = h; im = h; break;
        case 3: re = s; im = c; break;
        case 4: re = 0; im = 1; break;
        case 5: re = -s; im = c; break;
        case 6: re = -h; im = h; break;
        default: re = -c; im = s; break;
    }
    return mk<R>(re, S * im);
}

// a * exp(S 2 pi i k / 16) with the trivial factors spelled out: k = 4 is a
// multiplication by S i, k = 2 and 6 by sqrt(1/2) (+-1 + S i).  (IEEE rules
// keep a compiler from dropping the products with 0 and 1 by itself.)
template <typename R, int S> __device__ __forceinline__ cpx<R> mul_w16(cpx<R> a, int k) {
    const R h = (R)0.70710678118654752440;
    if (k == 0) return a;
    if (k == 4) return mul_si<R>(a, S);
    if (k == 2) return mk<R>(h * (a.x - (R)S * a.y), h * (a.y + (R)S * a.x));
    if (k == 6) return mk<R>(-h * (a.x + (R)S * a.y), h * ((R)S * a.x - a.y));
    return mul<R>(a, w16<R, S>(k));
}

template <typename R, int S> __device__ __forceinline__ void dft8(cpx<R> *v) {
    cpx<R> e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4<R, S>(e);
    dft4<R, S>(o);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const cpx<R> t = mul_w16<R, S>(o[k], 2 * k);
        v[k] = add<R>(e[k], t);
        v[k + 4] = sub<R>(e[k], t);
    }
}

template <typename R, int S> __device__ __forceinline__ void dft16(cpx<R> *v) {
    cpx<R> e[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { e[k] = v[2 * k]; o[k] = v[2 * k + 1]; }
    dft8<R, S>(e);
    dft8<R, S>(o);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const cpx<R> t = mul_w16<R, S>(o[k], k);
        v[k] = add<R>(e[k], t);
        v[k + 8] = sub<R>(e[k], t);
    }
}

// exp(S 2 pi i e / N) for N = 12 or 20 (e known at compile time after
// unrolling): cosines of multiples of 30 and 18 degrees
template <typename R, int N> __device__ __forceinline__ R cos_n(int e) {
    e %= N;
    if constexpr (N == 12) {
        const R c30 = (R)0.86602540378443864676;   // cos(pi/6)
        const R t[12] = {1, c30, (R)0.5, 0, (R)-0.5, -c30, -1, -c30, (R)-0.5, 0, (R)0.5, c30};
        return t[e];
    } else {
        const R a = (R)0.95105651629515357212, b = (R)0.80901699437494742410;   // cos(pi/10), cos(pi/5)
        const R c = (R)0.58778525229247312917, d = (R)0.30901699437494742410;   // cos(3pi/10), cos(2pi/5)
        const R t[20] = {1, a, b, c, d, 0, -d, -c, -b, -a, -1, -a, -b, -c, -d, 0, d, c, b, a};
        return t[e];
    }
}
template <typename R, int S, int N> __device__ __forceinline__ cpx<R> w_n(int e) {
    // sin(2 pi e / N) = cos(2 pi (e - N/4) / N)
    return mk<R>(cos_n<R, N>(e), (R)S * cos_n<R, N>(e + 3 * N / 4));
}

// Composite DFT of length N1 N2 in registers (Cooley-Tukey): DFT-N1 over n1
// for each n2 on x[N2 n1 + n2], the twiddle w_N^(n2 k1), DFT-N2 over n2 for
// each k1, output X[k1 + N1 k2].
template <typename R, int S, int N1, int N2> __device__ __forceinline__ void dft_ct(cpx<R> *v);

template <typename R, int S, int RAD> __device__ __forceinline__ void dft(cpx<R> *v) {
    if constexpr (RAD == 2) dft2<R, S>(v[0], v[1]);
    else if constexpr (RAD == 3) dft3<R, S>(v);
    else if constexpr (RAD == 4) dft4<R, S>(v);
    else if constexpr (RAD == 5) dft5<R, S>(v);
    else if constexpr (RAD == 8) dft8<R, S>(v);
    else if constexpr (RAD == 12) dft_ct<R, S, 4, 3>(v);
    else if constexpr (RAD == 20) dft_ct<R, S, 4, 5>(v);
    else dft16<R, S>(v);
}

template <typename R, int S, int N1, int N2> __device__ __forceinline__ void dft_ct(cpx<R> *v) {
    constexpr int N = N1 * N2;
    cpx<R> y[N];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
        cpx<R> a[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) a[n1] = v[N2 * n1 + n2];
        dft<R, S, N1>(a);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) y[N2 * k1 + n2] = (n2 * k1 == 0) ? a[k1] : mul<R>(a[k1], w_n<R, S, N>(n2 * k1));
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
        cpx<R> b[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) b[n2] = y[N2 * k1 + n2];
        dft<R, S, N2>(b);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k1 + N1 * k2] = b[k2];
    }
}

// ---------------------------------------------------------------------------
// One Stockham stage over L interleaved lines: src -> dst.
// Butterfly j (0 <= j < N/RAD) reads src[j + r N/RAD], multiplies input r by
// w_{Ns RAD}^{(j mod Ns) r}, and writes dst[(j/Ns) Ns RAD + (j mod Ns) + r Ns].
// ---------------------------------------------------------------------------
template <typename R, int S, int RAD>
__device__ __forceinline__ void stockham_stage(const cpx<R> *__restrict__ src, cpx<R> *__restrict__ dst,
                                               int N, int Ns, int L, int ES, const cpx<R> *__restrict__ tw) {
    const int nb = N / RAD;
    const int total = nb * L;
    const int twstep = N / (Ns * RAD);
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
        const int j = b / L;
        const int l = b - j * L;
        cpx<R> v[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[r] = src[(j + r * nb) * ES + l];
        const int jm = j % Ns;
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                cpx<R> w = __ldg(&tw[jm * r * twstep]);
                if (S > 0) w.y = -w.y;
                v[r] = mul<R>(v[r], w);
            }
        }
        dft<R, S, RAD>(v);
        const int o = (j - jm) * RAD + jm;
#pragma unroll
        for (int r = 0; r < RAD; ++r) dst[(o + r * Ns) * ES + l] = v[r];
    }
}

// Full transform of L interleaved lines held in bufA.  Returns the buffer
// holding the result (bufA or bufB).  All threads of the block must call it.
template <typename R, int S>
__device__ cpx<R> *fft_lines(cpx<R> *bufA, cpx<R> *bufB, int L, int ES, const AxisPlan &p) {
    cpx<R> *src = bufA, *dst = bufB;
    const cpx<R> *tw = reinterpret_cast<const cpx<R> *>(p.tw);
    int Ns = 1;
    for (int s = 0; s < p.nstages; ++s) {
        const int rad = p.radix[s];
        switch (rad) {
            case 2: stockham_stage<R, S, 2>(src, dst, p.n, Ns, L, ES, tw); break;
            case 3: stockham_stage<R, S, 3>(src, dst, p.n, Ns, L, ES, tw); break;
            case 4: stockham_stage<R, S, 4>(src, dst, p.n, Ns, L, ES, tw); break;
            case 5: stockham_stage<R, S, 5>(src, dst, p.n, Ns, L, ES, tw); break;
            case 8: stockham_stage<R, S, 8>(src, dst, p.n, Ns, L, ES, tw); break;
            default: stockham_stage<R, S, 16>(src, dst, p.n, Ns, L, ES, tw); break;
        }
        __syncthreads();
        Ns *= rad;
        cpx<R> *t = src; src = dst; dst = t;
    }
    return src;
}

// ---------------------------------------------------------------------------
// Register-resident engine for lengths known at compile time (powers of two,
// and 96 and 160, the mixed lengths of the batched cell studies).
// Every thread owns E elements of one line for the whole transform (BPT =
// E/RAD butterflies per stage), so a stage is: load the thread's butterfly
// inputs from the single shared buffer into registers, barrier, compute,
// store the outputs in place, barrier.  One buffer instead of two, all index
// arithmetic on compile-time powers of two.  The CTA must have exactly
// L * N / E threads; thread t works on line t % L.
// ---------------------------------------------------------------------------
// Stages in order R0, R1, R2, R3 (NS of them); E is a multiple of every
// stage's radix.  The mixed lengths 96 = 4 4 2 3 and 160 = 4 4 2 5 put the
// odd radix last, so that the sub-transform length before every stage is a
// power of two.
template <int N> struct FastPlan;
template <> struct FastPlan<8>   { static constexpr int E = 8,  NS = 1, R0 = 8,  R1 = 1,  R2 = 1, R3 = 1; };
template <> struct FastPlan<16>  { static constexpr int E = 16, NS = 1, R0 = 16, R1 = 1,  R2 = 1, R3 = 1; };
template <> struct FastPlan<32>  { static constexpr int E = 8,  NS = 2, R0 = 8,  R1 = 4,  R2 = 1, R3 = 1; };
template <> struct FastPlan<64>  { static constexpr int E = 8,  NS = 2, R0 = 8,  R1 = 8,  R2 = 1, R3 = 1; };
template <> struct FastPlan<96>  { static constexpr int E = 12, NS = 4, R0 = 4,  R1 = 4,  R2 = 2, R3 = 3; };
template <> struct FastPlan<128> { static constexpr int E = 16, NS = 2, R0 = 16, R1 = 8,  R2 = 1, R3 = 1; };
template <> struct FastPlan<160> { static constexpr int E = 20, NS = 4, R0 = 4,  R1 = 4,  R2 = 2, R3 = 5; };
template <> struct FastPlan<256> { static constexpr int E = 16, NS = 2, R0 = 16, R1 = 16, R2 = 1, R3 = 1; };
template <> struct FastPlan<512> { static constexpr int E = 16, NS = 3, R0 = 16, R1 = 16, R2 = 2, R3 = 1; };

// The n3 pass (shared-memory form) takes 96 and 160 in two stages instead
// of four, with radix-12 and radix-20 butterflies in registers (24 and 40
// elements per thread): 96 = 8 12, 160 = 8 20.  Other lengths as FastPlan.
template <int N> struct FastPlanN3 : FastPlan<N> {};
template <> struct FastPlanN3<96>  { static constexpr int E = 24, NS = 2, R0 = 8, R1 = 12, R2 = 1, R3 = 1; };
template <> struct FastPlanN3<160> { static constexpr int E = 40, NS = 2, R0 = 8, R1 = 20, R2 = 1, R3 = 1; };

__host__ __device__ constexpr bool is_fast_length(int n) {
    return n == 8 || n == 16 || n == 32 || n == 64 || n == 96 || n == 128 || n == 160 || n == 256 || n == 512;
}
__host__ __device__ constexpr int fast_elems(int n) {
    return (n == 8 || n == 32 || n == 64) ? 8 : (n == 96 ? 12 : (n == 160 ? 20 : 16));
}
__host__ __device__ constexpr int fast_elems_n3(int n) { return n == 96 ? 24 : (n == 160 ? 40 : fast_elems(n)); }
// the n3 pass's plan by precision: the two-stage plans in FP32 only (FP64
// elements would not fit in registers)
template <typename R, int N>
using PlanN3 = typename std::conditional<sizeof(R) == 4, FastPlanN3<N>, FastPlan<N>>::type;
template <typename R> __host__ __device__ constexpr int fast_elems_n3r(int n) {
    return sizeof(R) == 4 ? fast_elems_n3(n) : fast_elems(n);
}

// Position of element e of a line in a tile with element stride ES; with
// PAD, one slot is skipped every 16 elements so that the stride-16 writes of
// a radix-16 stage spread over the shared-memory banks.
template <int PAD> __device__ __forceinline__ int epos(int e, int ES) { return e * ES + (PAD ? (e >> 4) : 0); }

// Barrier of the threads that run a transform: the whole CTA (n = 0), or
// the first n threads on named barrier 1 (n a multiple of 32).
__device__ __forceinline__ void group_sync(int n) {
    if (n == 0) __syncthreads();
    else asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
}

template <typename R, int S, int N, int RAD, int NS_BEFORE, int PAD, typename Plan = FastPlan<N>>
__device__ __forceinline__ void fast_stage(cpx<R> *buf, int ES, int l, int j0, const cpx<R> *__restrict__ tw,
                                           int nsync) {
    constexpr int E = Plan::E;
    constexpr int BPT = E / RAD;
    constexpr int nb = N / RAD;
    constexpr int jstep = N / E;
    constexpr int twstep = N / (NS_BEFORE * RAD);
    cpx<R> v[BPT][RAD];
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int j = j0 + i * jstep;
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[i][r] = buf[epos<PAD>(j + r * nb, ES) + l];
    }
    group_sync(nsync);
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int j = j0 + i * jstep;
        const int jm = j & (NS_BEFORE - 1);
        if (NS_BEFORE > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                cpx<R> w = __ldg(&tw[jm * r * twstep]);
                if (S > 0) w.y = -w.y;
                v[i][r] = mul<R>(v[i][r], w);
            }
        }
        dft<R, S, RAD>(v[i]);
        const int o = (j - jm) * RAD + jm;
#pragma unroll
        for (int r = 0; r < RAD; ++r) buf[epos<PAD>(o + r * NS_BEFORE, ES) + l] = v[i][r];
    }
    group_sync(nsync);
}

// Transform of L interleaved lines in buf (in place), element e of line l
// at buf[epos<PAD>(e, ES) + l] (ES >= L).  With nsync = 0 the CTA must have
// exactly L * N / E threads (every thread takes part in every barrier);
// otherwise threads 0 .. nsync-1 (= L * N / E) run it and synchronise on
// named barrier 1, and the CTA's other warps are free for other work.
template <typename R, int S, int N, int PAD = 0, typename P = FastPlan<N>>
__device__ __forceinline__ void fast_fft(cpx<R> *buf, int L, int ES, const cpx<R> *__restrict__ tw, int nsync = 0) {
    const int l = (int)threadIdx.x % L;
    const int j0 = (int)threadIdx.x / L;
    fast_stage<R, S, N, P::R0, 1, PAD, P>(buf, ES, l, j0, tw, nsync);
    if constexpr (P::NS > 1) fast_stage<R, S, N, P::R1, P::R0, PAD, P>(buf, ES, l, j0, tw, nsync);
    if constexpr (P::NS > 2) fast_stage<R, S, N, P::R2, P::R0 * P::R1, PAD, P>(buf, ES, l, j0, tw, nsync);
    if constexpr (P::NS > 3) fast_stage<R, S, N, P::R3, P::R0 * P::R1 * P::R2, PAD, P>(buf, ES, l, j0, tw, nsync);
}

}  // namespace hom
