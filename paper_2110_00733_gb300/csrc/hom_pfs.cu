// hom_pfs.cu -- phase-field smoothening (section 3.2): the spectral filter of
// eq. (phase3) on a half spectrum and the block average with threshold that
// carries the fine phase map onto the simulation grid.
#include <cuda_runtime.h>

#include "hom_pfs.h"

namespace hom {
namespace {

constexpr int kPfsThreads = 256;
constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ int signed_freq(int k, int n) { return (2 * k < n) ? k : k - n; }

// phi^ /= 1 + c |q|^2 with q_p = 2 pi m_p / N_p (half spectrum: m_3 = k3)
__global__ void __launch_bounds__(kPfsThreads) k_pfs_filter(int n1, int n2, int n3, double c, double2 *spec) {
    const int h = n3 / 2 + 1;
    const long long S = (long long)n1 * n2 * h;
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < S; f += (long long)gridDim.x * blockDim.x) {
        const int k3 = (int)(f % h);
        const long long r = f / h;
        const int k2 = (int)(r % n2), k1 = (int)(r / n2);
        const double q1 = kTwoPi * signed_freq(k1, n1) / n1, q2 = kTwoPi * signed_freq(k2, n2) / n2;
        const double q3 = kTwoPi * k3 / n3;
        const double g = 1.0 / (1.0 + c * (q1 * q1 + q2 * q2 + q3 * q3));
        double2 v = spec[f];
        v.x *= g;
        v.y *= g;
        spec[f] = v;
    }
}

// coarse voxel = mean of its r^3 fine voxels (component 0 of a Mandel field,
// fine voxels C order); values below the threshold become 0, values above 1
// (round-off) become 1
__global__ void __launch_bounds__(kPfsThreads) k_pfs_coarsen(int n1, int n2, int n3, int r, double threshold,
                                                             const double *fine, double *coarse) {
    const int c1 = n1 / r, c2 = n2 / r, c3 = n3 / r;
    const long long Vc = (long long)c1 * c2 * c3;
    const double inv = 1.0 / ((double)r * r * r);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Vc; i += (long long)gridDim.x * blockDim.x) {
        const int x3 = (int)(i % c3);
        const long long t = i / c3;
        const int x2 = (int)(t % c2), x1 = (int)(t / c2);
        double s = 0.0;
        for (int a = 0; a < r; ++a)
            for (int b = 0; b < r; ++b)
                for (int d = 0; d < r; ++d)
                    s += fine[((long long)(x1 * r + a) * n2 + (x2 * r + b)) * n3 + (x3 * r + d)];
        s *= inv;
        // a phase map lies in [0, 1]; transform round-off can step a few ulps past 1
        coarse[i] = s < threshold ? 0.0 : (s > 1.0 ? 1.0 : s);
    }
}

// partial sums of phi and phi^2 (FP64): partials[b] and partials[nb + b]
__global__ void __launch_bounds__(kPfsThreads) k_phi_sums(long long V, const double *__restrict__ phi,
                                                          double *partials) {
    __shared__ double red[2][kPfsThreads / 32];
    double s1 = 0.0, s2 = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        const double p = phi[i];
        s1 += p;
        s2 += p * p;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = s1;
        red[1][wid] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kPfsThreads / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        partials[blockIdx.x] = a;
        partials[gridDim.x + blockIdx.x] = b;
    }
}

int pfs_blocks(long long n) {
    const long long b = (n + kPfsThreads - 1) / kPfsThreads;
    return (int)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

}  // namespace

int phi_sums(long long V, const double *phi, double *partials, cudaStream_t s) {
    const int nb = pfs_blocks(V);
    k_phi_sums<<<nb, kPfsThreads, 0, s>>>(V, phi, partials);
    return nb;
}

void pfs_filter(int n1, int n2, int n3, double c, double2 *spec, cudaStream_t s) {
    const long long S = (long long)n1 * n2 * (n3 / 2 + 1);
    k_pfs_filter<<<pfs_blocks(S), kPfsThreads, 0, s>>>(n1, n2, n3, c, spec);
}

void pfs_coarsen(int n1, int n2, int n3, int r, double threshold, const double *fine, double *coarse, cudaStream_t s) {
    const long long Vc = (long long)(n1 / r) * (n2 / r) * (n3 / r);
    k_pfs_coarsen<<<pfs_blocks(Vc), kPfsThreads, 0, s>>>(n1, n2, n3, r, threshold, fine, coarse);
}

}  // namespace hom
