// hom_pfs.h -- kernels of the phase-field smoothening (hom_pfs.cu).
#pragma once
#include <cuda_runtime.h>

namespace hom {

// spec (n1 x n2 x (n3/2+1) complex, one component) *= 1 / (1 + c |q|^2)
void pfs_filter(int n1, int n2, int n3, double c, double2 *spec, cudaStream_t s);
// partial sums of phi into partials[0, nb) and of phi^2 into partials[nb, 2 nb);
// returns nb (at most 1216)
int phi_sums(long long V, const double *phi, double *partials, cudaStream_t s);
// coarse (n/r voxels) = r^3 block means of fine (n voxels), zeroed below threshold
void pfs_coarsen(int n1, int n2, int n3, int r, double threshold, const double *fine, double *coarse, cudaStream_t s);

}  // namespace hom
