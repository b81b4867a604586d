// hom_cg.cu -- conjugate gradients on the Galerkin system (section 2.1: the
// solver the paper names for cells without void, and shows to fail once
// empty voxels make the system singular; MINRES with the rotated scheme is
// the method).  The vectors live in the projected half-spectrum space of the
// MINRES solver, under the same Parseval inner product; the operator
// application is shared with it.  The scalars (step a = rho / <p, A p>,
// direction b = rho' / rho, rho = ||r||^2, the stop test on ||r|| / ||r_0||)
// are the CgState kernels of the MoDBFFT solver, whose preconditioned
// <r, z> is here ||r||^2 itself.
#include <cuda_runtime.h>

#include "hom_cg.h"

namespace hom {
namespace {

constexpr int kCgThreads = 256;

// Parseval weight of the half-spectrum plane k3 (1 on the self-conjugate
// planes k3 = 0 and k3 = n3/2, 2 elsewhere)
__device__ __forceinline__ double plane_weight(int k3, int n3) { return (k3 == 0 || 2 * k3 == n3) ? 1.0 : 2.0; }

__device__ __forceinline__ double block_total(double v) {
    __shared__ double part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = (lane < (int)(blockDim.x >> 5)) ? part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

// x += a p, r -= a q; partial sums of ||r||^2 into partials[0, np) and, as
// the unpreconditioned <r, z>, into partials[np, 2 np)
template <typename R>
__global__ void __launch_bounds__(kCgThreads) k_gcg_xr(long long n, int h, int n3, const cpx<R> *__restrict__ p,
                                                       const cpx<R> *__restrict__ q, cpx<R> *__restrict__ x,
                                                       cpx<R> *__restrict__ r, const CgState *st, double *partials,
                                                       int np) {
    if (st->done) return;
    const R a = (R)st->a;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const cpx<R> pv = p[i], qv = q[i];
        cpx<R> xv = x[i], rv = r[i];
        xv.x += a * pv.x;
        xv.y += a * pv.y;
        rv.x -= a * qv.x;
        rv.y -= a * qv.y;
        x[i] = xv;
        r[i] = rv;
        acc += plane_weight((int)((i / 6) % h), n3) * ((double)rv.x * rv.x + (double)rv.y * rv.y);
    }
    const double s = block_total(acc);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        partials[np + blockIdx.x] = s;
    }
}

// p = r + b p
template <typename R>
__global__ void __launch_bounds__(kCgThreads) k_gcg_p(long long n, const cpx<R> *__restrict__ r, cpx<R> *__restrict__ p,
                                                      const CgState *st) {
    if (st->done) return;
    const R b = (R)st->b;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const cpx<R> rv = r[i];
        cpx<R> pv = p[i];
        pv.x = rv.x + b * pv.x;
        pv.y = rv.y + b * pv.y;
        p[i] = pv;
    }
}

}  // namespace

int gcg_blocks(long long n) {
    const long long b = (n + kCgThreads - 1) / kCgThreads;
    return (int)(b < 1 ? 1 : (b > kGcgMaxBlocks ? kGcgMaxBlocks : b));
}

template <typename R>
void gcg_xr(long long n, int h, int n3, cudaStream_t s, const cpx<R> *p, const cpx<R> *q, cpx<R> *x, cpx<R> *r,
            const CgState *st, double *partials) {
    const int nb = gcg_blocks(n);
    k_gcg_xr<R><<<nb, kCgThreads, 0, s>>>(n, h, n3, p, q, x, r, st, partials, nb);
}

template <typename R>
void gcg_p(long long n, cudaStream_t s, const cpx<R> *r, cpx<R> *p, const CgState *st) {
    k_gcg_p<R><<<gcg_blocks(n), kCgThreads, 0, s>>>(n, r, p, st);
}

template void gcg_xr<float>(long long, int, int, cudaStream_t, const float2 *, const float2 *, float2 *, float2 *,
                            const CgState *, double *);
template void gcg_xr<double>(long long, int, int, cudaStream_t, const double2 *, const double2 *, double2 *,
                             double2 *, const CgState *, double *);
template void gcg_p<float>(long long, cudaStream_t, const float2 *, float2 *, const CgState *);
template void gcg_p<double>(long long, cudaStream_t, const double2 *, double2 *, const CgState *);

}  // namespace hom
