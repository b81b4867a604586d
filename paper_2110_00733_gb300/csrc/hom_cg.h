// hom_cg.h -- conjugate gradients on the Galerkin system (hom_cg.cu).
#pragma once
#include <cuda_runtime.h>

#include "hom_internal.h"

namespace hom {

// blocks of the element-wise CG kernels (each writes one partial sum, twice)
constexpr int kGcgMaxBlocks = 152 * 4;
int gcg_blocks(long long n);

// x += a p, r -= a q over n complex values (6 per frequency, h = n3/2 + 1
// frequencies per k3 row); partial sums of ||r||^2 (Parseval) into
// partials[0, nb) and partials[nb, 2 nb), nb = gcg_blocks(n)
template <typename R>
void gcg_xr(long long n, int h, int n3, cudaStream_t s, const cpx<R> *p, const cpx<R> *q, cpx<R> *x, cpx<R> *r,
            const CgState *st, double *partials);

// p = r + b p
template <typename R>
void gcg_p(long long n, cudaStream_t s, const cpx<R> *r, cpx<R> *p, const CgState *st);

}  // namespace hom
