// hom_j2.h -- J2 plasticity kernels of the Newton extension (hom_j2.cu).
#pragma once
#include <cuda_runtime.h>

namespace hom {

struct J2Material {
    double E, nu, sy, H;    // Young's modulus, Poisson ratio, yield stress, isotropic hardening (Pa)
};

// radial return at every voxel (fields 6 x V Mandel, component-major):
// sig = phi sigma_J2(eps; epsp, alpha) and, if Ct is not null, the consistent
// tangent in T (36 x V: entry (i, j) of voxel v at (6 i + j) V + v, times phi);
// commit != 0 writes the updated plastic strain and hardening variable back
// into epsp and alpha
template <typename T>
void j2_return(long long V, const J2Material &m, const double *phi, const double *eps, double *epsp, double *alpha,
               double *sig, T *Ct, int commit, cudaStream_t s);
// out = Ct : v at every voxel (tangent in Tc, fields and arithmetic in Tf)
template <typename Tc, typename Tf>
void j2_tangent_apply(long long V, const Tc *Ct, const Tf *v, Tf *out, cudaStream_t s);
// eps[c] += d[c] at every voxel
void j2_add_uniform(long long V, double *eps, const double d[6], cudaStream_t s);
// b = -b over n complex values, plus sbar_v[c] at frequency 0 (component c)
void j2_negate_add_dc(long long n, double2 *b, const double sbar_v[6], cudaStream_t s);
// host: max |a| over n values (a - b if b is not null)
double j2_absmax(long long n, const double *a, const double *b, double *partials, double *h_partials, cudaStream_t s);
// host: the six component means of a 6 x V field
void j2_means(long long V, const double *f, double *partials, double *h_partials, double out[6], cudaStream_t s);
// partial buffer sizes the two host reductions need (doubles)
constexpr int kJ2Blocks = 152 * 4;

}  // namespace hom
