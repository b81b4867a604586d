// net.cu -- the warm-start network: point-wise kernels, the U-Net forward and
// backward passes over the convolution kernels of net_kernels.cu, Adam, and
// the C ABI of hom_net.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hom.h"
#include "../../include/hom_net.h"
#include "net_internal.h"

using namespace hnet;
using bf16 = __nv_bfloat16;

namespace {

thread_local std::string g_err;

int set_err(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define NCU(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return set_err(HOM_ECUDA, cudaGetErrorString(e_));        \
    } while (0)

constexpr int kEw = 256;
constexpr float kSqrt2 = 1.41421356237309505f;

int ew_blocks(long long n) {
    long long b = (n + kEw - 1) / kEw;
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ float bf(bf16 v) { return __bfloat162float(v); }

// ------------------------------------------------------------ point-wise
// network input: channel 0 = mean of phi over s^3 blocks, channels 1..15 = 0
__global__ void k_prep_input(int B, int m1, int m2, int m3, int s, const float *__restrict__ phi, bf16 *__restrict__ x) {
    const long long Vc = (long long)m1 * m2 * m3, total = Vc * B;
    const int n2 = m2 * s, n3 = m3 * s;
    const long long Vf = Vc * s * s * s;
    const float inv = 1.f / (float)(s * s * s);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long r = i;
        const int c3 = (int)(r % m3); r /= m3;
        const int c2 = (int)(r % m2); r /= m2;
        const int c1 = (int)(r % m1);
        const int b = (int)(r / m1);
        float acc = 0.f;
        for (int a = 0; a < s; ++a)
            for (int bb = 0; bb < s; ++bb)
                for (int cc = 0; cc < s; ++cc)
                    acc += phi[b * Vf + ((long long)(c1 * s + a) * n2 + c2 * s + bb) * n3 + c3 * s + cc];
        // the voxel's 16 channels as two 16-byte stores
        const unsigned short h0 = __bfloat16_as_ushort(__float2bfloat16(acc * inv));
        uint4 *o = reinterpret_cast<uint4 *>(x + i * 16);
        o[0] = make_uint4(h0, 0u, 0u, 0u);
        o[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// 2x2x2 average pooling, [B][n1][n2][n3][C] -> half resolution
__global__ void k_avgpool2(int B, int n1, int n2, int n3, int C, const bf16 *__restrict__ in, bf16 *__restrict__ out) {
    const int h1 = n1 / 2, h2 = n2 / 2, h3 = n3 / 2;
    const long long total = (long long)h1 * h2 * h3 * B * C;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long r = i / C;
        const int x = (int)(r % h3); r /= h3;
        const int y = (int)(r % h2); r /= h2;
        const int z = (int)(r % h1);
        const int b = (int)(r / h1);
        float acc = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int bb = 0; bb < 2; ++bb)
                for (int cc = 0; cc < 2; ++cc)
                    acc += bf(in[((((long long)b * n1 + 2 * z + a) * n2 + 2 * y + bb) * n3 + 2 * x + cc) * C + c]);
        out[i] = __float2bfloat16(acc * 0.125f);
    }
}

// Prediction x0[k][c][v] (tensor components) = sum_J M[6c+J] E_k[J] with M
// interpolated trilinearly (periodic) from the m grid to the s-times finer
// grid; case k uses M of batch (per_batch ? k : 0).
__global__ void k_predict(int ncase, int per_batch, int m1, int m2, int m3, int s, const float *__restrict__ M,
                          const float *__restrict__ E, float *__restrict__ x0) {
    const int n1 = m1 * s, n2 = m2 * s, n3 = m3 * s;
    const long long Vf = (long long)n1 * n2 * n3, Vc = (long long)m1 * m2 * m3;
    const long long total = Vf * ncase;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / Vf);
        const long long v = i - k * Vf;
        long long r = v;
        const int f3 = (int)(r % n3); r /= n3;
        const int f2 = (int)(r % n2);
        const int f1 = (int)(r / n2);
        const float *Mb = M + (per_batch ? (long long)k * Vc * 48 : 0);
        int i0[3], i1[3];
        float t[3];
        const int f[3] = {f1, f2, f3}, m[3] = {m1, m2, m3};
        for (int a = 0; a < 3; ++a) {
            const float p = ((float)f[a] + 0.5f) / (float)s - 0.5f;
            const float fl = floorf(p);
            t[a] = p - fl;
            int q = (int)fl;
            q = q < 0 ? q + m[a] : q;
            i0[a] = q;
            i1[a] = q + 1 == m[a] ? 0 : q + 1;
        }
        float e[6];
        for (int j = 0; j < 6; ++j) e[j] = E[k * 6 + j];
        float out[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int corner = 0; corner < 8; ++corner) {
            const int z = (corner & 4) ? i1[0] : i0[0], y = (corner & 2) ? i1[1] : i0[1], x = (corner & 1) ? i1[2] : i0[2];
            const float w = ((corner & 4) ? t[0] : 1.f - t[0]) * ((corner & 2) ? t[1] : 1.f - t[1]) *
                            ((corner & 1) ? t[2] : 1.f - t[2]);
            if (w == 0.f) continue;
            const float *mv = Mb + (((long long)z * m2 + y) * m3 + x) * 48;
            for (int c = 0; c < 6; ++c) {
                float acc = 0.f;
                for (int j = 0; j < 6; ++j) acc += mv[6 * c + j] * e[j];
                out[c] += w * acc;
            }
        }
        for (int c = 0; c < 6; ++c) x0[((long long)k * 6 + c) * Vf + v] = (c < 3) ? out[c] : out[c] / kSqrt2;
    }
}

__device__ __forceinline__ double block_sum_d(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < (int)((blockDim.x + 31) >> 5)) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    return r;
}

// Loss and head gradient: d_c = x0_c - target_c (Mandel), loss partials of
// sum w d^2 with the voxel weight w = vw + (1 - vw) phi (1 everywhere for
// vw = 1), G[v][6c+J] = scale w d_c E_J (channels 36..47 zero).  Six
// consecutive threads take the six components of one voxel, so a warp reads
// and writes contiguous runs of M and G.
__global__ void k_loss_grad(int B, long long V, const float *__restrict__ M, const float *__restrict__ E,
                            const float *__restrict__ target, const float *__restrict__ phi, float vw, float scale,
                            bf16 *__restrict__ G, double *__restrict__ partials) {
    double acc = 0.0;
    const long long total = V * B * 6;
    for (long long i6 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i6 < total;
         i6 += (long long)gridDim.x * blockDim.x) {
        const long long i = i6 / 6;
        const int c = (int)(i6 - i * 6);
        const int b = (int)(i / V);
        const long long v = i - b * V;
        const float2 *m = reinterpret_cast<const float2 *>(M + i * 48 + 6 * c);
        const float *e = E + b * 6;
        const float2 m0 = m[0], m1 = m[1], m2 = m[2];
        const float x = m0.x * e[0] + m0.y * e[1] + m1.x * e[2] + m1.y * e[3] + m2.x * e[4] + m2.y * e[5];
        float tv = target[((long long)b * 6 + c) * V + v];
        if (c >= 3) tv *= kSqrt2;
        const float w = vw + (1.f - vw) * phi[i];
        const float d = x - tv;
        acc += (double)w * d * d;
        const float g = scale * w * d;
        __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(G + i * 48 + 6 * c);
        o[0] = __floats2bfloat162_rn(g * e[0], g * e[1]);
        o[1] = __floats2bfloat162_rn(g * e[2], g * e[3]);
        o[2] = __floats2bfloat162_rn(g * e[4], g * e[5]);
        if (c == 5) {
            uint2 *z = reinterpret_cast<uint2 *>(G + i * 48 + 36);
            z[0] = z[1] = z[2] = make_uint2(0u, 0u);
        }
    }
    const double s = block_sum_d(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_sum_partials(const double *p, int n, double *out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
    s = block_sum_d(s);
    if (threadIdx.x == 0) *out = s;
}

// Gradient w.r.t. a layer output, masked by the ReLU and stored in BF16:
// G = [Y > 0] (A[., a_off + c] + sum of the 8 children in U[., u_off + c]
// on the 2x finer grid + P[parent, c] / 8 on the 2x coarser grid).
struct Assemble {
    int B, n1, n2, n3, C;
    const bf16 *Y;
    const bf16 *A;
    int a_stride, a_off;
    const bf16 *U;
    int u_stride, u_off;
    const bf16 *P;
    int p_stride;
    bf16 *G;
};

__device__ __forceinline__ void add8(float *g, const bf16 *p, float w) {
    const uint4 v = *reinterpret_cast<const uint4 *>(p);
    const bf16 *h = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] += w * bf(h[k]);
}

// one thread per voxel and 8 channels (channel counts, strides and offsets
// are multiples of 8, so every access is one 16-byte load or store)
__global__ void k_assemble(Assemble a) {
    const long long V = (long long)a.n1 * a.n2 * a.n3;
    const int C8 = a.C >> 3;
    const long long total = V * a.B * C8;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / C8;    // voxel (b, z, y, x) on this grid
        const int c = (int)(i - r * C8) * 8;
        float g[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (a.A) add8(g, a.A + r * a.a_stride + a.a_off + c, 1.f);
        if (a.U || a.P) {
            long long q = r;
            const int x = (int)(q % a.n3); q /= a.n3;
            const int y = (int)(q % a.n2); q /= a.n2;
            const int z = (int)(q % a.n1);
            const int b = (int)(q / a.n1);
            if (a.U) {
                const int f1 = 2 * a.n1, f2 = 2 * a.n2, f3 = 2 * a.n3;
                float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            const long long fv = (((long long)b * f1 + 2 * z + dz) * f2 + 2 * y + dy) * f3 + 2 * x + dx;
                            add8(s, a.U + fv * a.u_stride + a.u_off + c, 1.f);
                        }
#pragma unroll
                for (int k = 0; k < 8; ++k) g[k] += s[k];
            }
            if (a.P) {
                const int h1 = a.n1 / 2, h2 = a.n2 / 2, h3 = a.n3 / 2;
                const long long pv = (((long long)b * h1 + z / 2) * h2 + y / 2) * h3 + x / 2;
                const uint4 pw = *reinterpret_cast<const uint4 *>(a.P + pv * a.p_stride + c);
                const bf16 *ph = reinterpret_cast<const bf16 *>(&pw);
#pragma unroll
                for (int k = 0; k < 8; ++k) g[k] += bf(ph[k]) * 0.125f;
            }
        }
        if (a.Y) {
            const uint4 yw = *reinterpret_cast<const uint4 *>(a.Y + r * a.C + c);
            const bf16 *yh = reinterpret_cast<const bf16 *>(&yw);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (!(bf(yh[k]) > 0.f)) g[k] = 0.f;
        }
        __nv_bfloat162 o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = __floats2bfloat162_rn(g[2 * k], g[2 * k + 1]);
        *reinterpret_cast<uint4 *>(a.G + r * a.C + c) = *reinterpret_cast<const uint4 *>(o);
    }
}

// column sums of G [rows][C] -> partials [gridDim.x][C]
__global__ void k_colsum(long long rows, int C, const bf16 *__restrict__ G, float *__restrict__ partials) {
    extern __shared__ float sh[];
    const int per = blockDim.x / C;           // rows handled at once
    const int c = threadIdx.x % C, sub = threadIdx.x / C;
    float acc = 0.f;
    if (sub < per)
        for (long long r = (long long)blockIdx.x * per + sub; r < rows; r += (long long)gridDim.x * per)
            acc += bf(G[r * C + c]);
    sh[threadIdx.x] = (sub < per) ? acc : 0.f;
    __syncthreads();
    if (threadIdx.x < C) {
        float s = 0.f;
        for (int k = 0; k < per; ++k) s += sh[k * C + threadIdx.x];
        partials[(long long)blockIdx.x * C + threadIdx.x] = s;
    }
}

// one warp per column: lanes stride over the partials, then a warp sum
__global__ void k_colsum_reduce(int nb, int C, int cout, const float *partials, float *out) {
    const int c = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)), lane = threadIdx.x & 31;
    if (c >= cout) return;
    float s = 0.f;
    for (int b = lane; b < nb; b += 32) s += partials[(long long)b * C + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[c] = s;
}

// dW[t][co][ci] (logical sizes) = sum over splits of the padded partials
__global__ void k_wgrad_reduce(int S, int cout_p, int cin_s, int cout, int cin, const float *__restrict__ partial,
                               float *__restrict__ dW) {
    const long long total = 27LL * cout * cin;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cin);
        const long long r = i / cin;
        const int co = (int)(r % cout), t = (int)(r / cout);
        float s = 0.f;
        for (int k = 0; k < S; ++k) s += partial[(((long long)k * 27 + t) * cout_p + co) * cin_s + ci];
        dW[i] = s;
    }
}

__global__ void k_adam(long long n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// BF16 copies of one layer: Wf[t][co][ci] (padded), Wb[t][ci][co] =
// W[26-t][co][ci] for the input gradient, FP32 padded bias.
__global__ void k_pack(int cout, int cin, int cout_p, int cin_s, const float *__restrict__ w, bf16 *__restrict__ Wf,
                       bf16 *__restrict__ Wb, float *__restrict__ bias) {
    const long long total = 27LL * cout_p * cin_s;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cin_s);
        const long long r = i / cin_s;
        const int co = (int)(r % cout_p), t = (int)(r / cout_p);
        const float val = (co < cout && ci < cin) ? w[((long long)t * cout + co) * cin + ci] : 0.f;
        Wf[i] = __float2bfloat16(val);
        Wb[((long long)(26 - t) * cin_s + ci) * cout_p + co] = __float2bfloat16(val);
        if (t == 0 && ci == 0) bias[co] = co < cout ? w[27LL * cout * cin + co] : 0.f;
    }
}

// ------------------------------------------------------------ architecture
struct LayerDef {
    const char *name;
    int cin, cout, relu, level;
};
enum { E1A, E1B, E2A, E2B, E3A, E3B, BNA, BNB, D3A, D3B, D2A, D2B, D1A, D1B, HEAD, NL };
const LayerDef kDefs[NL] = {
    {"e1a", 1, 16, 1, 0},  {"e1b", 16, 16, 1, 0}, {"e2a", 16, 32, 1, 1}, {"e2b", 32, 32, 1, 1},
    {"e3a", 32, 48, 1, 2}, {"e3b", 48, 48, 1, 2}, {"bna", 48, 64, 1, 3}, {"bnb", 64, 64, 1, 3},
    {"d3a", 112, 48, 1, 2}, {"d3b", 48, 48, 1, 2}, {"d2a", 80, 32, 1, 1}, {"d2b", 32, 32, 1, 1},
    {"d1a", 48, 16, 1, 0}, {"d1b", 16, 16, 1, 0}, {"head", 16, 36, 0, 0}};

int pad16(int c) { return (c + 15) / 16 * 16; }

struct Layer {
    LayerDef d;
    int cin_s, cout_p;
    long long off;        // W offset in the flat parameter array; bias follows
    bf16 *Wf = nullptr, *Wb = nullptr;
    float *bias = nullptr;
};

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
double normal01(uint64_t &s) {   // Box-Muller from two 53-bit uniforms
    const double u1 = ((splitmix64(s) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

struct hom_net {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Layer L[NL];
    long long nparam = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    int step = 0;
    long long launches = 0;
    // workspace for (B, n1, n2, n3)
    int wB = 0, wn[3] = {0, 0, 0};
    std::vector<void *> bufs;
    bf16 *x = nullptr, *act[NL] = {}, *pool[3] = {}, *G[NL] = {}, *dX[NL] = {};
    float *M = nullptr, *partial = nullptr, *colpart = nullptr, *dE = nullptr, *Mw = nullptr;
    size_t partial_floats = 0, colpart_floats = 0, mw_floats = 0;
    double *losspart = nullptr, *dloss = nullptr;
    int ecap = 0;
    float void_weight = 1.f;
};

namespace {

void free_ws(hom_net *n) {
    for (void *p : n->bufs) cudaFree(p);
    n->bufs.clear();
    n->wB = 0;
    n->wn[0] = n->wn[1] = n->wn[2] = 0;
}

template <typename T>
int alloc(hom_net *n, T **p, size_t count) {
    void *q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) return set_err(HOM_ENOMEM, "device allocation failed");
    n->bufs.push_back(q);
    *p = static_cast<T *>(q);
    return HOM_OK;
}

long long level_vox(const hom_net *n, int B, const int g[3], int level) {
    return (long long)B * (g[0] >> level) * (g[1] >> level) * (g[2] >> level);
}

int wgrad_splits(long long vox) {
    long long s = (vox + 4095) / 4096;
    return (int)(s < 1 ? 1 : (s > 256 ? 256 : s));
}

int ensure_ws(hom_net *n, int B, const int g[3]) {
    if (n->wB == B && n->wn[0] == g[0] && n->wn[1] == g[1] && n->wn[2] == g[2]) return HOM_OK;
    free_ws(n);
    int rc = alloc(n, &n->x, (size_t)level_vox(n, B, g, 0) * 16);
    for (int l = 0; l < NL && !rc; ++l) {
        const Layer &L = n->L[l];
        const long long vox = level_vox(n, B, g, L.d.level);
        if (l == HEAD) rc = alloc(n, &n->M, (size_t)vox * 48);
        else rc = alloc(n, &n->act[l], (size_t)vox * L.cout_p);
        if (!rc) rc = alloc(n, &n->G[l], (size_t)vox * L.cout_p);
        if (!rc && l != E1A) rc = alloc(n, &n->dX[l], (size_t)vox * L.cin_s);
        const size_t pf = (size_t)wgrad_splits(vox) * 27 * L.cout_p * L.cin_s;
        if (pf > n->partial_floats) n->partial_floats = pf;
    }
    for (int k = 0; k < 3 && !rc; ++k) {
        const int c = k == 0 ? 16 : (k == 1 ? 32 : 48);
        rc = alloc(n, &n->pool[k], (size_t)level_vox(n, B, g, k + 1) * c);
    }
    if (!rc) rc = alloc(n, &n->partial, n->partial_floats);
    n->colpart_floats = (size_t)ew_blocks(level_vox(n, B, g, 0)) * 64;
    if (!rc) rc = alloc(n, &n->colpart, n->colpart_floats);
    if (!rc) rc = alloc(n, &n->losspart, (size_t)ew_blocks(level_vox(n, B, g, 0)));
    if (!rc) rc = alloc(n, &n->dloss, 1);
    if (rc) {
        free_ws(n);
        return rc;
    }
    n->wB = B;
    n->wn[0] = g[0];
    n->wn[1] = g[1];
    n->wn[2] = g[2];
    return HOM_OK;
}

int ensure_e(hom_net *n, int count) {
    if (count <= n->ecap) return HOM_OK;
    if (n->dE) cudaFree(n->dE);
    n->dE = nullptr;
    if (cudaMalloc(&n->dE, sizeof(float) * 6 * count) != cudaSuccess) return set_err(HOM_ENOMEM, "allocation failed");
    n->ecap = count;
    return HOM_OK;
}

// macro strains (tensor components, host) -> Mandel FP32 on the device
int upload_macro(hom_net *n, const double *macro, int count) {
    int rc = ensure_e(n, count);
    if (rc) return rc;
    std::vector<float> h(6 * count);
    for (int k = 0; k < count; ++k)
        for (int c = 0; c < 6; ++c) h[6 * k + c] = (float)(c < 3 ? macro[6 * k + c] : macro[6 * k + c] * std::sqrt(2.0));
    NCU(cudaMemcpyAsync(n->dE, h.data(), sizeof(float) * 6 * count, cudaMemcpyHostToDevice, n->stream));
    NCU(cudaStreamSynchronize(n->stream));
    return HOM_OK;
}

int pack_all(hom_net *n) {
    for (int l = 0; l < NL; ++l) {
        const Layer &L = n->L[l];
        k_pack<<<ew_blocks(27LL * L.cout_p * L.cin_s), kEw, 0, n->stream>>>(L.d.cout, L.d.cin, L.cout_p, L.cin_s,
                                                                            n->params + L.off, L.Wf, L.Wb, L.bias);
        ++n->launches;
    }
    NCU(cudaGetLastError());
    return HOM_OK;
}

// forward sources of layer l on the workspace
ConvArgs layer_args(hom_net *n, int l, int B, const int g[3]) {
    const Layer &L = n->L[l];
    ConvArgs a{};
    a.B = B;
    a.n1 = g[0] >> L.d.level;
    a.n2 = g[1] >> L.d.level;
    a.n3 = g[2] >> L.d.level;
    a.W = L.Wf;
    a.bias = L.bias;
    a.cout = L.cout_p;
    a.relu = L.d.relu;
    auto src = [&](const bf16 *p, int c) {
        a.src0 = p;
        a.c0s = c;
    };
    switch (l) {
        case E1A: src(n->x, 16); break;
        case E2A: src(n->pool[0], 16); break;
        case E3A: src(n->pool[1], 32); break;
        case BNA: src(n->pool[2], 48); break;
        case D3A: src(n->act[E3B], 48); a.src1 = n->act[BNB]; a.c1s = 64; break;
        case D2A: src(n->act[E2B], 32); a.src1 = n->act[D3B]; a.c1s = 48; break;
        case D1A: src(n->act[E1B], 16); a.src1 = n->act[D2B]; a.c1s = 32; break;
        default: src(n->act[l - 1], n->L[l - 1].cout_p); break;
    }
    if (l == HEAD) a.out_f32 = n->M;
    else a.out_bf16 = n->act[l];
    return a;
}

int run_conv(hom_net *n, const ConvArgs &a) {
    if (conv3_forward_tc(a, n->stream)) return set_err(HOM_EINVAL, "convolution shape not supported");
    ++n->launches;
    return HOM_OK;
}

// after a synchronisation: a tensor-core convolution that gave up a bounded wait
int tc_status() {
    if (conv3_tc_error(1)) return set_err(HOM_ETIMEOUT, "a bounded wait in a tensor-core convolution gave up");
    return HOM_OK;
}

int forward(hom_net *n, int B, const int g[3]) {
    for (int l = 0; l < NL; ++l) {
        if (l == E2A || l == E3A || l == BNA) {
            const int k = l == E2A ? 0 : (l == E3A ? 1 : 2);
            const int src = l == E2A ? E1B : (l == E3A ? E2B : E3B);
            const int lv = n->L[src].d.level;
            const long long out = level_vox(n, B, g, lv + 1) * n->L[src].cout_p;
            k_avgpool2<<<ew_blocks(out), kEw, 0, n->stream>>>(B, g[0] >> lv, g[1] >> lv, g[2] >> lv,
                                                               n->L[src].cout_p, n->act[src], n->pool[k]);
            ++n->launches;
        }
        int rc = run_conv(n, layer_args(n, l, B, g));
        if (rc) return rc;
    }
    NCU(cudaGetLastError());
    return HOM_OK;
}

int assemble(hom_net *n, int l, int B, const int g[3], const bf16 *A, int a_stride, int a_off, const bf16 *U,
             int u_stride, int u_off, const bf16 *P, int p_stride) {
    const Layer &L = n->L[l];
    Assemble a{};
    a.B = B;
    a.n1 = g[0] >> L.d.level;
    a.n2 = g[1] >> L.d.level;
    a.n3 = g[2] >> L.d.level;
    a.C = L.cout_p;
    a.Y = L.d.relu ? n->act[l] : nullptr;
    a.A = A;
    a.a_stride = a_stride;
    a.a_off = a_off;
    a.U = U;
    a.u_stride = u_stride;
    a.u_off = u_off;
    a.P = P;
    a.p_stride = p_stride;
    a.G = n->G[l];
    if ((a.C | a_stride | a_off | u_stride | u_off | p_stride) & 7)
        return set_err(HOM_EINVAL, "channel layout not a multiple of 8");
    k_assemble<<<ew_blocks(level_vox(n, B, g, L.d.level) * L.cout_p / 8), kEw, 0, n->stream>>>(a);
    ++n->launches;
    return HOM_OK;
}

// weight and bias gradients of layer l from G[l]; input gradient into dX[l]
int layer_back(hom_net *n, int l, int B, const int g[3]) {
    const Layer &L = n->L[l];
    const ConvArgs in = layer_args(n, l, B, g);
    const long long vox = level_vox(n, B, g, L.d.level);
    WgradArgs w{};
    w.in = in;
    w.G = n->G[l];
    w.cout = L.cout_p;
    w.partial = n->partial;
    w.S = wgrad_splits(vox);
    if (conv3_wgrad(w, n->stream)) return set_err(HOM_EINVAL, "weight-gradient shape not supported");
    k_wgrad_reduce<<<ew_blocks(27LL * L.d.cout * L.d.cin), kEw, 0, n->stream>>>(
        w.S, L.cout_p, L.cin_s, L.d.cout, L.d.cin, n->partial, n->grads + L.off);
    const int nb = ew_blocks(vox);
    k_colsum<<<nb, kEw, kEw * sizeof(float), n->stream>>>(vox, L.cout_p, n->G[l], n->colpart);
    k_colsum_reduce<<<(L.d.cout + 7) / 8, 256, 0, n->stream>>>(nb, L.cout_p, L.d.cout, n->colpart,
                                             n->grads + L.off + 27LL * L.d.cout * L.d.cin);
    n->launches += 4;
    if (l != E1A) {
        ConvArgs d{};
        d.B = B;
        d.n1 = in.n1;
        d.n2 = in.n2;
        d.n3 = in.n3;
        d.src0 = n->G[l];
        d.c0s = L.cout_p;
        d.W = L.Wb;
        d.cout = L.cin_s;
        d.out_bf16 = n->dX[l];
        int rc = run_conv(n, d);
        if (rc) return rc;
    }
    NCU(cudaGetLastError());
    return HOM_OK;
}

int backward(hom_net *n, int B, const int g[3]) {
    int rc = 0;
    auto back = [&](int l) { if (!rc) rc = layer_back(n, l, B, g); };
    auto asm_ = [&](int l, const bf16 *A, int as, int ao, const bf16 *U, int us, int uo, const bf16 *P, int ps) {
        if (!rc) rc = assemble(n, l, B, g, A, as, ao, U, us, uo, P, ps);
    };
    back(HEAD);                                                    // G[HEAD] from the loss
    asm_(D1B, n->dX[HEAD], 16, 0, nullptr, 0, 0, nullptr, 0);
    back(D1B);
    asm_(D1A, n->dX[D1B], 16, 0, nullptr, 0, 0, nullptr, 0);
    back(D1A);                                                     // dX: [s1 16 | up(d2) 32]
    asm_(D2B, nullptr, 0, 0, n->dX[D1A], 48, 16, nullptr, 0);
    back(D2B);
    asm_(D2A, n->dX[D2B], 32, 0, nullptr, 0, 0, nullptr, 0);
    back(D2A);                                                     // [s2 32 | up(d3) 48]
    asm_(D3B, nullptr, 0, 0, n->dX[D2A], 80, 32, nullptr, 0);
    back(D3B);
    asm_(D3A, n->dX[D3B], 48, 0, nullptr, 0, 0, nullptr, 0);
    back(D3A);                                                     // [s3 48 | up(bn) 64]
    asm_(BNB, nullptr, 0, 0, n->dX[D3A], 112, 48, nullptr, 0);
    back(BNB);
    asm_(BNA, n->dX[BNB], 64, 0, nullptr, 0, 0, nullptr, 0);
    back(BNA);                                                     // d pool3
    asm_(E3B, n->dX[D3A], 112, 0, nullptr, 0, 0, n->dX[BNA], 48);
    back(E3B);
    asm_(E3A, n->dX[E3B], 48, 0, nullptr, 0, 0, nullptr, 0);
    back(E3A);                                                     // d pool2
    asm_(E2B, n->dX[D2A], 80, 0, nullptr, 0, 0, n->dX[E3A], 32);
    back(E2B);
    asm_(E2A, n->dX[E2B], 32, 0, nullptr, 0, 0, nullptr, 0);
    back(E2A);                                                     // d pool1
    asm_(E1B, n->dX[D1A], 48, 0, nullptr, 0, 0, n->dX[E2A], 16);
    back(E1B);
    asm_(E1A, n->dX[E1B], 16, 0, nullptr, 0, 0, nullptr, 0);
    back(E1A);
    return rc;
}

int check_grid(const int g[3], int B) {
    if (!g || B <= 0) return set_err(HOM_EINVAL, "null grid or batch <= 0");
    for (int p = 0; p < 3; ++p)
        if (g[p] < 8 || g[p] % 8) return set_err(HOM_EUNSUPPORTED_GRID, "each grid size must be a positive multiple of 8");
    return HOM_OK;
}

int loss_and_head_grad(hom_net *n, int B, const int g[3], const float *phi, const float *target, double *loss) {
    const long long V = (long long)g[0] * g[1] * g[2];
    const int nb = ew_blocks(V * B);
    const float scale = (float)(2.0 / (6.0 * (double)V * B));
    k_loss_grad<<<nb, kEw, 0, n->stream>>>(B, V, n->M, n->dE, target, phi, n->void_weight, scale, n->G[HEAD],
                                           n->losspart);
    k_sum_partials<<<1, 256, 0, n->stream>>>(n->losspart, nb, n->dloss);
    n->launches += 2;
    NCU(cudaGetLastError());
    double h = 0.0;
    NCU(cudaMemcpyAsync(&h, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    NCU(cudaStreamSynchronize(n->stream));
    if (loss) *loss = h / (6.0 * (double)V * B);
    return HOM_OK;
}

int train_common(hom_net *n, int B, const int g[3], const float *phi, const double *macro, const float *target,
                 double *loss) {
    int rc = check_grid(g, B);
    if (rc) return rc;
    if (!phi || !macro || !target) return set_err(HOM_EINVAL, "null argument");
    cudaSetDevice(n->device);
    if ((rc = ensure_ws(n, B, g))) return rc;
    if ((rc = upload_macro(n, macro, B))) return rc;
    k_prep_input<<<ew_blocks(level_vox(n, B, g, 0)), kEw, 0, n->stream>>>(B, g[0], g[1], g[2], 1, phi, n->x);
    ++n->launches;
    if ((rc = forward(n, B, g))) return rc;
    if ((rc = loss_and_head_grad(n, B, g, phi, target, loss))) return rc;
    return backward(n, B, g);
}

}  // namespace

// ------------------------------------------------------------------ C ABI
const char *hom_net_last_error(void) { return g_err.c_str(); }

int hom_net_create(hom_net **out, unsigned long long seed, void *stream) {
    if (!out) return set_err(HOM_EINVAL, "null output");
    *out = nullptr;
    hom_net *n = new hom_net();
    cudaGetDevice(&n->device);
    long long off = 0;
    for (int l = 0; l < NL; ++l) {
        Layer &L = n->L[l];
        L.d = kDefs[l];
        L.cin_s = pad16(L.d.cin);
        L.cout_p = pad16(L.d.cout);
        L.off = off;
        off += 27LL * L.d.cout * L.d.cin + L.d.cout;
    }
    n->nparam = off;
    auto fail = [&](int code, const char *msg) {
        hom_net_destroy(n);
        return set_err(code, msg);
    };
    if (stream) n->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(HOM_ECUDA, "stream creation failed");
        n->own_stream = true;
    }
    const size_t pb = sizeof(float) * n->nparam;
    if (cudaMalloc(&n->params, pb) != cudaSuccess || cudaMalloc(&n->grads, pb) != cudaSuccess ||
        cudaMalloc(&n->m, pb) != cudaSuccess || cudaMalloc(&n->v, pb) != cudaSuccess)
        return fail(HOM_ENOMEM, "parameter allocation failed");
    for (int l = 0; l < NL; ++l) {
        Layer &L = n->L[l];
        const size_t wb = sizeof(bf16) * 27 * L.cout_p * L.cin_s;
        if (cudaMalloc(&L.Wf, wb) != cudaSuccess || cudaMalloc(&L.Wb, wb) != cudaSuccess ||
            cudaMalloc(&L.bias, sizeof(float) * L.cout_p) != cudaSuccess)
            return fail(HOM_ENOMEM, "weight allocation failed");
    }
    // He-normal weights, zero biases (host, splitmix64 + Box-Muller)
    std::vector<float> h(n->nparam, 0.f);
    uint64_t s = seed;
    for (int l = 0; l < NL; ++l) {
        const Layer &L = n->L[l];
        const double stdv = std::sqrt(2.0 / (27.0 * L.d.cin)) * (L.d.relu ? 1.0 : 0.1);
        for (long long i = 0; i < 27LL * L.d.cout * L.d.cin; ++i) h[L.off + i] = (float)(stdv * normal01(s));
    }
    if (cudaMemcpy(n->params, h.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->m, 0, pb) != cudaSuccess || cudaMemset(n->v, 0, pb) != cudaSuccess ||
        cudaMemset(n->grads, 0, pb) != cudaSuccess)
        return fail(HOM_ECUDA, "parameter upload failed");
    if (pack_all(n) || cudaStreamSynchronize(n->stream) != cudaSuccess) return fail(HOM_ECUDA, "weight packing failed");
    *out = n;
    return HOM_OK;
}

void hom_net_destroy(hom_net *n) {
    if (!n) return;
    cudaSetDevice(n->device);
    if (n->stream) cudaStreamSynchronize(n->stream);
    free_ws(n);
    for (int l = 0; l < NL; ++l) {
        cudaFree(n->L[l].Wf);
        cudaFree(n->L[l].Wb);
        cudaFree(n->L[l].bias);
    }
    cudaFree(n->params);
    cudaFree(n->grads);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->dE);
    cudaFree(n->Mw);
    if (n->own_stream) cudaStreamDestroy(n->stream);
    delete n;
}

long long hom_net_param_count(const hom_net *n) { return n ? n->nparam : 0; }

int hom_net_set_void_weight(hom_net *n, double void_weight) {
    if (!n || !(void_weight >= 0.0 && void_weight <= 1.0)) return set_err(HOM_EINVAL, "void weight must be in [0, 1]");
    n->void_weight = (float)void_weight;
    return HOM_OK;
}
long long hom_net_kernel_launches(const hom_net *n) { return n ? n->launches : 0; }

int hom_net_get_params(const hom_net *n, float *host) {
    if (!n || !host) return set_err(HOM_EINVAL, "null argument");
    cudaSetDevice(n->device);
    NCU(cudaStreamSynchronize(n->stream));
    NCU(cudaMemcpy(host, n->params, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost));
    return HOM_OK;
}

int hom_net_set_params(hom_net *n, const float *host) {
    if (!n || !host) return set_err(HOM_EINVAL, "null argument");
    cudaSetDevice(n->device);
    NCU(cudaStreamSynchronize(n->stream));
    NCU(cudaMemcpy(n->params, host, sizeof(float) * n->nparam, cudaMemcpyHostToDevice));
    int rc = pack_all(n);
    if (rc) return rc;
    NCU(cudaStreamSynchronize(n->stream));
    return HOM_OK;
}

int hom_net_save(const hom_net *n, const char *path) {
    if (!n || !path) return set_err(HOM_EINVAL, "null argument");
    std::vector<float> p(n->nparam), m(n->nparam), v(n->nparam);
    cudaSetDevice(n->device);
    NCU(cudaStreamSynchronize(n->stream));
    NCU(cudaMemcpy(p.data(), n->params, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost));
    NCU(cudaMemcpy(m.data(), n->m, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost));
    NCU(cudaMemcpy(v.data(), n->v, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost));
    FILE *f = std::fopen(path, "wb");
    if (!f) return set_err(HOM_EINVAL, "cannot open file for writing");
    const char magic[8] = {'H', 'O', 'M', 'N', 'E', 'T', '0', '1'};
    const long long cnt = n->nparam;
    const int step = n->step;
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&cnt, sizeof(cnt), 1, f) == 1 &&
              std::fwrite(&step, sizeof(step), 1, f) == 1 &&
              std::fwrite(p.data(), sizeof(float), cnt, f) == (size_t)cnt &&
              std::fwrite(m.data(), sizeof(float), cnt, f) == (size_t)cnt &&
              std::fwrite(v.data(), sizeof(float), cnt, f) == (size_t)cnt;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? HOM_OK : set_err(HOM_EINVAL, "write failed");
}

int hom_net_load(hom_net *n, const char *path) {
    if (!n || !path) return set_err(HOM_EINVAL, "null argument");
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_err(HOM_EINVAL, "cannot open file");
    char magic[8];
    long long cnt = 0;
    int step = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "HOMNET01", 8) == 0 &&
              std::fread(&cnt, sizeof(cnt), 1, f) == 1 && cnt == n->nparam && std::fread(&step, sizeof(step), 1, f) == 1;
    std::vector<float> p(ok ? cnt : 0), m(ok ? cnt : 0), v(ok ? cnt : 0);
    ok = ok && std::fread(p.data(), sizeof(float), cnt, f) == (size_t)cnt &&
         std::fread(m.data(), sizeof(float), cnt, f) == (size_t)cnt &&
         std::fread(v.data(), sizeof(float), cnt, f) == (size_t)cnt;
    std::fclose(f);
    if (!ok) return set_err(HOM_EINVAL, "not a parameter file of this network");
    cudaSetDevice(n->device);
    NCU(cudaMemcpy(n->m, m.data(), sizeof(float) * cnt, cudaMemcpyHostToDevice));
    NCU(cudaMemcpy(n->v, v.data(), sizeof(float) * cnt, cudaMemcpyHostToDevice));
    n->step = step;
    return hom_net_set_params(n, p.data());
}

int hom_net_forward(hom_net *n, int B, const int g[3], const float *phi, const double *macro, float *x0) {
    if (!n || !phi || !macro || !x0) return set_err(HOM_EINVAL, "null argument");
    int rc = check_grid(g, B);
    if (rc) return rc;
    cudaSetDevice(n->device);
    if ((rc = ensure_ws(n, B, g))) return rc;
    if ((rc = upload_macro(n, macro, B))) return rc;
    k_prep_input<<<ew_blocks(level_vox(n, B, g, 0)), kEw, 0, n->stream>>>(B, g[0], g[1], g[2], 1, phi, n->x);
    ++n->launches;
    if ((rc = forward(n, B, g))) return rc;
    k_predict<<<ew_blocks(level_vox(n, B, g, 0)), kEw, 0, n->stream>>>(B, 1, g[0], g[1], g[2], 1, n->M, n->dE, x0);
    ++n->launches;
    NCU(cudaGetLastError());
    NCU(cudaStreamSynchronize(n->stream));
    return tc_status();
}

int hom_net_train_step(hom_net *n, int B, const int g[3], const float *phi, const double *macro, const float *target,
                       float lr, double *loss) {
    if (!n) return set_err(HOM_EINVAL, "null network");
    if (!(lr > 0.f) || !std::isfinite(lr)) return set_err(HOM_EINVAL, "learning rate must be positive");
    int rc = train_common(n, B, g, phi, macro, target, loss);
    if (rc) return rc;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - std::pow(b1, (float)n->step), bc2 = 1.f - std::pow(b2, (float)n->step);
    k_adam<<<ew_blocks(n->nparam), kEw, 0, n->stream>>>(n->nparam, n->params, n->grads, n->m, n->v, lr, b1, b2, 1e-8f,
                                                         bc1, bc2);
    ++n->launches;
    if ((rc = pack_all(n))) return rc;
    NCU(cudaStreamSynchronize(n->stream));
    return tc_status();
}

int hom_net_gradients(hom_net *n, int B, const int g[3], const float *phi, const double *macro, const float *target,
                      float *grads, double *loss) {
    if (!n || !grads) return set_err(HOM_EINVAL, "null argument");
    int rc = train_common(n, B, g, phi, macro, target, loss);
    if (rc) return rc;
    NCU(cudaStreamSynchronize(n->stream));
    NCU(cudaMemcpy(grads, n->grads, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost));
    return tc_status();
}

int hom_net_warm_start(hom_net *n, const int grid[3], int s, const float *phi, int ncase, const double *macro,
                       float *x0) {
    if (!n || !grid || !phi || !macro || !x0 || ncase <= 0 || s <= 0) return set_err(HOM_EINVAL, "bad argument");
    int g[3];
    for (int p = 0; p < 3; ++p) {
        if (grid[p] % s) return set_err(HOM_EUNSUPPORTED_GRID, "grid sizes must be multiples of s");
        g[p] = grid[p] / s;
    }
    int rc = check_grid(g, 1);
    if (rc) return rc;
    cudaSetDevice(n->device);
    if ((rc = ensure_ws(n, 1, g))) return rc;
    if ((rc = upload_macro(n, macro, ncase))) return rc;
    k_prep_input<<<ew_blocks(level_vox(n, 1, g, 0)), kEw, 0, n->stream>>>(1, g[0], g[1], g[2], s, phi, n->x);
    ++n->launches;
    if ((rc = forward(n, 1, g))) return rc;
    const long long Vf = (long long)grid[0] * grid[1] * grid[2];
    k_predict<<<ew_blocks(Vf * ncase), kEw, 0, n->stream>>>(ncase, 0, g[0], g[1], g[2], s, n->M, n->dE, x0);
    ++n->launches;
    NCU(cudaGetLastError());
    NCU(cudaStreamSynchronize(n->stream));
    return tc_status();
}

int hom_net_conv3d(int batch, const int grid[3], const unsigned short *src0, int c0s, const unsigned short *src1,
                   int c1s, const unsigned short *W, const float *bias, int relu, int cout, void *out, int out_f32,
                   void *stream) {
    if (!grid || batch <= 0 || !src0 || !W || !out || (c1s && !src1)) return set_err(HOM_EINVAL, "bad argument");
    ConvArgs a{};
    a.B = batch;
    a.n1 = grid[0];
    a.n2 = grid[1];
    a.n3 = grid[2];
    a.src0 = reinterpret_cast<const bf16 *>(src0);
    a.c0s = c0s;
    a.src1 = reinterpret_cast<const bf16 *>(src1);
    a.c1s = c1s;
    a.W = reinterpret_cast<const bf16 *>(W);
    a.bias = bias;
    a.relu = relu;
    a.cout = cout;
    if (out_f32) a.out_f32 = static_cast<float *>(out);
    else a.out_bf16 = static_cast<bf16 *>(out);
    if (grid[0] <= 0 || grid[1] <= 0 || grid[2] <= 0) return set_err(HOM_EUNSUPPORTED_GRID, "empty grid");
    if (conv3_forward_tc(a, (cudaStream_t)stream))
        return set_err(HOM_EINVAL, "channel counts must be multiples of 16 (cout <= 256)");
    NCU(cudaGetLastError());
    NCU(cudaStreamSynchronize((cudaStream_t)stream));
    return tc_status();
}

int hom_net_conv3d_wgrad(int batch, const int grid[3], const unsigned short *G, int cout, const unsigned short *src0,
                         int c0s, const unsigned short *src1, int c1s, float *dW, void *stream) {
    if (!grid || batch <= 0 || !G || !src0 || !dW || (c1s && !src1)) return set_err(HOM_EINVAL, "bad argument");
    if (grid[0] <= 0 || grid[1] <= 0 || grid[2] <= 0) return set_err(HOM_EUNSUPPORTED_GRID, "empty grid");
    WgradArgs w{};
    w.in.B = batch;
    w.in.n1 = grid[0];
    w.in.n2 = grid[1];
    w.in.n3 = grid[2];
    w.in.src0 = reinterpret_cast<const bf16 *>(src0);
    w.in.c0s = c0s;
    w.in.src1 = reinterpret_cast<const bf16 *>(src1);
    w.in.c1s = c1s;
    w.G = reinterpret_cast<const bf16 *>(G);
    w.cout = cout;
    const long long vox = (long long)batch * grid[0] * grid[1] * grid[2];
    w.S = wgrad_splits(vox);
    const int cin_s = c0s + c1s;
    float *partial = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    NCU(cudaMalloc(&partial, sizeof(float) * w.S * 27 * cout * cin_s));
    w.partial = partial;
    if (conv3_wgrad(w, st)) {
        cudaFree(partial);
        return set_err(HOM_EINVAL, "channel counts must be multiples of 16, cout <= 64");
    }
    k_wgrad_reduce<<<ew_blocks(27LL * cout * cin_s), kEw, 0, st>>>(w.S, cout, cin_s, cout, cin_s, partial, dW);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(partial);
    if (e != cudaSuccess) return set_err(HOM_ECUDA, cudaGetErrorString(e));
    return HOM_OK;
}
