// net_kernels.cu -- weight gradients of the warm-start network's periodic
// 3x3x3 convolutions on the BF16 tensor cores (mma.sync m16n8k16, FP32
// accumulation; the forward and input-gradient convolutions run on tcgen05 in
// net_tc.cu).
//
// Tensors are channels-last BF16, [batch][n1][n2][n3][C] with C a multiple
// of 16 (padding channels hold zeros).  A convolution output voxel v and tap
// t = 9 (dz+1) + 3 (dy+1) + (dx+1) read the input at v + (dz, dy, dx), wrapped
// periodically.  Forward:  y[v, co] = sum_t sum_ci W[t, co, ci] x[v + d_t, ci].
// The input gradient is the same operation with W'[t, ci, co] = W[26-t, co, ci].
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "net_internal.h"

namespace hnet {

namespace {

constexpr int kConvThreads = 128;     // 4 warps
constexpr int kRowA = 24;             // smem row of a 16-channel chunk: 16 + 8 pad (48 B, odd 16-B count)

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous copy; src_bytes = 0 fills the destination with zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// D += A B, A 16x16 (row), B 16x8 (col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16816(float *c, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Input row for output voxel (b, z, y, x), tap offsets (dz, dy, dx), channel
// chunk kc (16 channels): the first source at full resolution, or the second
// at half resolution (nearest-neighbour upsampling).
__device__ __forceinline__ const __nv_bfloat16 *conv_row(const ConvArgs &a, int b, int z, int y, int x, int dz,
                                                         int dy, int dx, int kc) {
    const int zz = wrap(z + dz, a.n1), yy = wrap(y + dy, a.n2), xx = wrap(x + dx, a.n3);
    const int k0 = a.c0s >> 4;
    if (kc < k0) {
        const long long v = (((long long)b * a.n1 + zz) * a.n2 + yy) * a.n3 + xx;
        return a.src0 + v * a.c0s + kc * 16;
    }
    // second source at half resolution, read with nearest-neighbour upsampling
    const int h1 = a.n1 >> 1, h2 = a.n2 >> 1, h3 = a.n3 >> 1;
    const long long v = (((long long)b * h1 + (zz >> 1)) * h2 + (yy >> 1)) * h3 + (xx >> 1);
    return a.src1 + v * a.c1s + (kc - k0) * 16;
}

// Weight gradient: partial[s][t][co][ci] = sum over the voxels of split s of
// G[v, co] X[v + d_t, ci].  GEMM with M = cout (all, m16 tiles), N = 16 input
// channels (blockIdx.z chunk), K = voxels; the 4 warps take interleaved
// 16-voxel slices of each 64-voxel stage and are summed at the end.
constexpr int kWgVox = 64;
constexpr int kWgStages = 3;

template <int MT>
__global__ void __launch_bounds__(kConvThreads) k_wgrad3(WgradArgs a) {
    constexpr int kRowG = 16 * MT + 8;   // an odd count of 16-byte units per row
    constexpr int kGBytes = kWgStages * kWgVox * kRowG * 2;
    static_assert(kGBytes >= 4 * MT * 16 * 16 * 4, "the reduction buffer reuses the G ring");
    __shared__ __align__(128) unsigned char sGraw[kGBytes];
    __shared__ __align__(128) __nv_bfloat16 sX[kWgStages][kWgVox * kRowA];
    auto sG = reinterpret_cast<__nv_bfloat16(*)[kWgVox * kRowG]>(sGraw);
    auto red = reinterpret_cast<float(*)[MT * 16 * 16]>(sGraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long V = (long long)a.in.n1 * a.in.n2 * a.in.n3;
    const long long total = V * a.in.B;
    const int s = blockIdx.x, t = blockIdx.y, kc = blockIdx.z;
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const long long per = (total + a.S - 1) / a.S;
    const long long v0 = (long long)s * per;
    const long long v1 = (v0 + per < total) ? v0 + per : total;
    const int nst = (int)((v1 > v0 ? v1 - v0 : 0) + kWgVox - 1) / kWgVox;
    const int gch = 2 * MT;              // 16-byte chunks per G row
    const ConvArgs &ca = a.in;

    auto stage_load = [&](int st, int buf) {
        const long long vb = v0 + (long long)st * kWgVox;
        // G rows: kWgVox x gch chunks
        for (int i = tid; i < kWgVox * gch; i += kConvThreads) {
            const int r = i / gch, c = i - r * gch;
            const long long v = vb + r;
            const bool ok = v < v1;
            const __nv_bfloat16 *src = a.G + (ok ? v : 0) * (16 * MT) + c * 8;
            cp_async16(smem_addr(&sG[buf][r * kRowG + c * 8]), src, ok ? 16 : 0);
        }
        // X rows at the tap offset: kWgVox x 2 chunks
        {
            const int r = tid >> 1, h = tid & 1;
            const long long v = vb + r;
            const bool ok = v < v1;
            const __nv_bfloat16 *src = ca.src0;
            if (ok) {
                long long q = v;
                const int x = (int)(q % ca.n3); q /= ca.n3;
                const int y = (int)(q % ca.n2); q /= ca.n2;
                const int z = (int)(q % ca.n1);
                const int b = (int)(q / ca.n1);
                src = conv_row(ca, b, z, y, x, dz, dy, dx, kc);
            }
            cp_async16(smem_addr(&sX[buf][r * kRowA + h * 8]), src + h * 8, ok ? 16 : 0);
        }
    };

    float acc[MT][2][4];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

#pragma unroll
    for (int st = 0; st < kWgStages - 1; ++st) {
        if (st < nst) stage_load(st, st);
        cp_async_commit();
    }
    for (int st = 0; st < nst; ++st) {
        cp_async_wait<kWgStages - 2>();
        __syncthreads();
        const int nxt = st + kWgStages - 1;
        if (nxt < nst) stage_load(nxt, nxt % kWgStages);
        cp_async_commit();
        const int buf = st % kWgStages;
        const int vb = warp * 16;       // this warp's 16 voxels of the stage
        uint32_t bx[4];
        {
            const int v = vb + (lane & 7) + (((lane >> 3) & 1) << 3);
            ldsm_x4_t(smem_addr(&sX[buf][v * kRowA + (lane >> 4) * 8]), bx[0], bx[1], bx[2], bx[3]);
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            uint32_t af[4];
            const int v = vb + (lane & 7) + ((lane >> 4) << 3);
            ldsm_x4_t(smem_addr(&sG[buf][v * kRowG + mt * 16 + ((lane >> 3) & 1) * 8]), af[0], af[1], af[2], af[3]);
            mma16816(acc[mt][0], af, bx[0], bx[1]);
            mma16816(acc[mt][1], af, bx[2], bx[3]);
        }
    }
    cp_async_wait<0>();
    __syncthreads();                      // the G ring becomes the reduction buffer
    // sum the four warps' partial products
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int co = mt * 16 + g + (k >> 1) * 8, ci = nt * 8 + 2 * tq + (k & 1);
                red[warp][co * 16 + ci] = acc[mt][nt][k];
            }
    __syncthreads();
    const int cout = 16 * MT;
    const int cin_s = ca.c0s + ca.c1s;
    for (int i = tid; i < cout * 16; i += kConvThreads) {
        const float v = red[0][i] + red[1][i] + red[2][i] + red[3][i];
        const int co = i >> 4, ci = i & 15;
        a.partial[(((long long)s * 27 + t) * cout + co) * cin_s + kc * 16 + ci] = v;
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
int conv3_wgrad(const WgradArgs &a, cudaStream_t st) {
    if (conv3_wgrad_tc(a, st) == 0) return 0;
    const ConvArgs &c = a.in;
    if ((a.cout & 15) || a.cout > 64 || (c.c0s & 15) || (c.c1s & 15) || a.S <= 0) return -1;
    const dim3 grid(a.S, 27, (c.c0s + c.c1s) / 16);
    switch (a.cout / 16) {
        case 1: k_wgrad3<1><<<grid, kConvThreads, 0, st>>>(a); break;
        case 2: k_wgrad3<2><<<grid, kConvThreads, 0, st>>>(a); break;
        case 3: k_wgrad3<3><<<grid, kConvThreads, 0, st>>>(a); break;
        case 4: k_wgrad3<4><<<grid, kConvThreads, 0, st>>>(a); break;
        default: return -1;
    }
    return 0;
}

}  // namespace hnet
