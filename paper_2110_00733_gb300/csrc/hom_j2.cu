// hom_j2.cu -- small-strain von Mises plasticity with linear isotropic
// hardening for the Newton extension of the Galerkin scheme (section 2.1.1):
// the radial return and its consistent tangent (Simo & Hughes 1998, section
// 3.3) at every voxel, stress and tangent times phi (section 3.2), and the
// point-wise helpers of the Newton loop.  The return map and the helpers run
// in FP64; the tangent is stored in FP64, or in FP32 for the FP32 MINRES
// solves of the Newton systems, and applied in the precision of the field.
#include <cuda_runtime.h>

#include "hom_j2.h"

namespace hom {
namespace {

constexpr int kJ2Threads = 256;

int j2_blocks(long long n) {
    const long long b = (n + kJ2Threads - 1) / kJ2Threads;
    return (int)(b < 1 ? 1 : (b > kJ2Blocks ? kJ2Blocks : b));
}

template <typename T>
__global__ void __launch_bounds__(kJ2Threads) k_j2_return(long long V, J2Material m, const double *__restrict__ phi,
                                                          const double *__restrict__ eps, double *epsp,
                                                          double *alpha, double *__restrict__ sig,
                                                          T *__restrict__ Ct, int commit) {
    const double lam = m.E * m.nu / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu)), mu = m.E / (2.0 * (1.0 + m.nu));
    const double kappa = lam + 2.0 * mu / 3.0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        double ee[6], st[6], s[6], n[6] = {0, 0, 0, 0, 0, 0}, epn[6];
        for (int c = 0; c < 6; ++c) {
            epn[c] = epsp[c * V + v];
            ee[c] = eps[c * V + v] - epn[c];
        }
        const double tr = ee[0] + ee[1] + ee[2];
        for (int c = 0; c < 6; ++c) st[c] = (c < 3 ? lam * tr : 0.0) + 2.0 * mu * ee[c];   // trial stress
        const double p = (st[0] + st[1] + st[2]) / 3.0;
        double ns = 0.0;
        for (int c = 0; c < 6; ++c) {
            s[c] = st[c] - (c < 3 ? p : 0.0);
            ns += s[c] * s[c];
        }
        ns = sqrt(ns);
        const double a0 = alpha[v];
        const double f = ns - sqrt(2.0 / 3.0) * (m.sy + m.H * a0);                             // trial yield function
        double theta = 1.0, thetab = 0.0, a1 = a0;
        if (f > 0.0 && ns > 0.0) {
            const double dg = f / (2.0 * mu + 2.0 * m.H / 3.0);                                  // consistency
            for (int c = 0; c < 6; ++c) {
                n[c] = s[c] / ns;
                st[c] -= 2.0 * mu * dg * n[c];
                epn[c] += dg * n[c];
            }
            a1 = a0 + sqrt(2.0 / 3.0) * dg;
            theta = 1.0 - 2.0 * mu * dg / ns;
            thetab = 1.0 / (1.0 + m.H / (3.0 * mu)) - (1.0 - theta);
        }
        const double ph = phi[v];
        for (int c = 0; c < 6; ++c) sig[c * V + v] = ph * st[c];
        if (Ct) {
            // C = kappa m (x) m + 2 mu theta (I - m (x) m / 3) - 2 mu thetab n (x) n, m = (1,1,1,0,0,0)
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    const double mm = (i < 3 && j < 3) ? 1.0 : 0.0;
                    const double cij = kappa * mm + 2.0 * mu * theta * ((i == j ? 1.0 : 0.0) - mm / 3.0) -
                                       2.0 * mu * thetab * n[i] * n[j];
                    Ct[(i * 6 + j) * V + v] = (T)(ph * cij);
                }
        }
        if (commit) {
            for (int c = 0; c < 6; ++c) epsp[c * V + v] = epn[c];
            alpha[v] = a1;
        }
    }
}

template <typename Tc, typename Tf>
__global__ void __launch_bounds__(kJ2Threads) k_j2_tangent_apply(long long V, const Tc *__restrict__ Ct,
                                                                 const Tf *__restrict__ x, Tf *__restrict__ y) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        Tf xv[6];
        for (int c = 0; c < 6; ++c) xv[c] = x[c * V + v];
        for (int i = 0; i < 6; ++i) {
            Tf s = 0;
            for (int j = 0; j < 6; ++j) s += (Tf)Ct[(i * 6 + j) * V + v] * xv[j];
            y[i * V + v] = s;
        }
    }
}

__global__ void __launch_bounds__(kJ2Threads) k_j2_add_uniform(long long V, double *eps, double d0, double d1,
                                                               double d2, double d3, double d4, double d5) {
    const double d[6] = {d0, d1, d2, d3, d4, d5};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 6 * V; i += (long long)gridDim.x * blockDim.x)
        eps[i] += d[i / V];
}

__global__ void __launch_bounds__(kJ2Threads) k_j2_negate_add_dc(long long n, double2 *b, double s0, double s1,
                                                                 double s2, double s3, double s4, double s5) {
    const double sv[6] = {s0, s1, s2, s3, s4, s5};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 v = b[i];
        v.x = -v.x + (i < 6 ? sv[i] : 0.0);
        v.y = -v.y;
        b[i] = v;
    }
}

__device__ __forceinline__ double block_max(double v) {
    __shared__ double part[kJ2Threads / 32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kJ2Threads / 32; ++w) v = fmax(v, part[w]);
    return v;
}

__device__ __forceinline__ double block_add(double v) {
    __shared__ double part[kJ2Threads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kJ2Threads / 32; ++w) v += part[w];
    return v;
}

__global__ void __launch_bounds__(kJ2Threads) k_j2_absmax(long long n, const double *__restrict__ a,
                                                          const double *__restrict__ b, double *partials) {
    double mx = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        mx = fmax(mx, fabs(b ? a[i] - b[i] : a[i]));
    mx = block_max(mx);
    if (threadIdx.x == 0) partials[blockIdx.x] = mx;
}

__global__ void __launch_bounds__(kJ2Threads) k_j2_means(long long V, const double *__restrict__ f, double *partials) {
    for (int c = 0; c < 6; ++c) {
        double s = 0.0;
        for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x)
            s += f[c * V + v];
        s = block_add(s);
        if (threadIdx.x == 0) partials[c * gridDim.x + blockIdx.x] = s;
    }
}

}  // namespace

template <typename T>
void j2_return(long long V, const J2Material &m, const double *phi, const double *eps, double *epsp, double *alpha,
               double *sig, T *Ct, int commit, cudaStream_t s) {
    k_j2_return<T><<<j2_blocks(V), kJ2Threads, 0, s>>>(V, m, phi, eps, epsp, alpha, sig, Ct, commit);
}
template void j2_return<float>(long long, const J2Material &, const double *, const double *, double *, double *,
                               double *, float *, int, cudaStream_t);
template void j2_return<double>(long long, const J2Material &, const double *, const double *, double *, double *,
                                double *, double *, int, cudaStream_t);

template <typename Tc, typename Tf>
void j2_tangent_apply(long long V, const Tc *Ct, const Tf *v, Tf *out, cudaStream_t s) {
    k_j2_tangent_apply<Tc, Tf><<<j2_blocks(V), kJ2Threads, 0, s>>>(V, Ct, v, out);
}
template void j2_tangent_apply<float, float>(long long, const float *, const float *, float *, cudaStream_t);
template void j2_tangent_apply<double, double>(long long, const double *, const double *, double *, cudaStream_t);
template void j2_tangent_apply<float, double>(long long, const float *, const double *, double *, cudaStream_t);

void j2_add_uniform(long long V, double *eps, const double d[6], cudaStream_t s) {
    k_j2_add_uniform<<<j2_blocks(6 * V), kJ2Threads, 0, s>>>(V, eps, d[0], d[1], d[2], d[3], d[4], d[5]);
}

void j2_negate_add_dc(long long n, double2 *b, const double sv[6], cudaStream_t s) {
    k_j2_negate_add_dc<<<j2_blocks(n), kJ2Threads, 0, s>>>(n, b, sv[0], sv[1], sv[2], sv[3], sv[4], sv[5]);
}

double j2_absmax(long long n, const double *a, const double *b, double *partials, double *h_partials, cudaStream_t s) {
    const int nb = j2_blocks(n);
    k_j2_absmax<<<nb, kJ2Threads, 0, s>>>(n, a, b, partials);
    cudaMemcpyAsync(h_partials, partials, sizeof(double) * nb, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    double mx = 0.0;
    for (int i = 0; i < nb; ++i) mx = h_partials[i] > mx ? h_partials[i] : mx;
    return mx;
}

void j2_means(long long V, const double *f, double *partials, double *h_partials, double out[6], cudaStream_t s) {
    const int nb = j2_blocks(V);
    k_j2_means<<<nb, kJ2Threads, 0, s>>>(V, f, partials);
    cudaMemcpyAsync(h_partials, partials, sizeof(double) * 6 * nb, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (int c = 0; c < 6; ++c) {
        double t = 0.0;
        for (int i = 0; i < nb; ++i) t += h_partials[c * nb + i];
        out[c] = t / (double)V;
    }
}

}  // namespace hom
