// net_tc.cu -- periodic 3x3x3 convolution as an implicit GEMM on the 5th-
// generation tensor cores: tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulator in tensor memory), issued by one thread, completion tracked on
// mbarriers with tcgen05.commit, the result read back with tcgen05.ld.
//
// CTA tile: M = 128 output voxels x N = all output channels (<= 256, a
// multiple of 16) x K = 27 taps x input channels, consumed 64 K at a time
// through a 4-stage ring.  Warp-specialised: four producer warps gather the
// operands with cp.async (two chunks in flight per thread), fence them for
// the tensor core and arrive on the stage's "full" barrier; a fifth warp
// waits on it, issues the MMAs and commits to the stage's "empty" barrier,
// which the producers wait on before reusing the stage.
// Each K chunk is staged by cp.async (16-byte rows, the gathered input rows
// with periodic wrap and the half-resolution second source as in the
// mma.sync kernel) into the canonical no-swizzle K-major layout of the MMA:
// core matrices of 8 rows x 16 bytes, K-adjacent core matrices LBO = 128 B
// apart, 8-row groups SBO = 1024 B apart.
//
// Every wait is bounded; on a timeout the kernel records it in g_tc_err,
// waits (bounded) for its own MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "net_internal.h"

namespace hnet {

__device__ int g_tc_err;

namespace {

constexpr int kProducers = 128;   // 4 warps: operand staging, then the epilogue (one TMEM lane quarter each)
constexpr int kThreads = kProducers + 32;   // + 1 warp that issues the MMAs
constexpr int kBM = 128;          // M per CTA (tcgen05 M = 128, cta_group::1)
constexpr int kBK = 64;           // K elements per stage (4 MMAs of K = 16)
constexpr int kStages = 4;
constexpr int kLBO = 128;         // K-adjacent core matrices
constexpr int kSBO = kBK / 8 * 128;   // 8-row groups (kBK/8 K-chunks of 128 B)
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// shared-memory matrix descriptor: start >> 4, LBO >> 4, SBO >> 4, version 1
// (bit 46), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((kLBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((kSBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t instr_desc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// 8 input channels (16 bytes) of K chunk q (K = 8q .. 8q+7) for voxel (b,z,y,x)
__device__ __forceinline__ const __nv_bfloat16 *k8_src(const ConvArgs &a, int cin_s, int b, int z, int y, int x,
                                                      int q) {
    const int k = 8 * q;
    const int t = k / cin_s, ci = k - t * cin_s;
    const int zz = wrapi(z + t / 9 - 1, a.n1), yy = wrapi(y + (t / 3) % 3 - 1, a.n2), xx = wrapi(x + t % 3 - 1, a.n3);
    if (ci < a.c0s) {
        const long long v = (((long long)b * a.n1 + zz) * a.n2 + yy) * a.n3 + xx;
        return a.src0 + v * a.c0s + ci;
    }
    const long long v = (((long long)b * (a.n1 >> 1) + (zz >> 1)) * (a.n2 >> 1) + (yy >> 1)) * (a.n3 >> 1) + (xx >> 1);
    return a.src1 + v * a.c1s + (ci - a.c0s);
}

__global__ void __launch_bounds__(kThreads) k_conv3_tc(ConvArgs a, int ncols) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.cout;
    const int cin_s = a.c0s + a.c1s;
    const int ktot = 27 * cin_s;                       // multiple of 16
    const int nk = (ktot + kBK - 1) / kBK;
    const int a_bytes = kBM / 8 * kSBO;                // 16 KB
    const int b_bytes = N / 8 * kSBO;
    const int stage_bytes = a_bytes + b_bytes;
    const long long V = (long long)a.n1 * a.n2 * a.n3;
    const long long total = V * a.B;
    const long long m0 = (long long)blockIdx.x * kBM;
    constexpr int kMma = kProducers / 32;              // the MMA warp

    if (warp == kMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], kProducers);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == kMma) {
        // ---- MMA issue (one thread)
        if (lane == 0) {
            int ncommit[kStages] = {};
            const uint32_t idesc = instr_desc(N);
            bool ok = true;
            for (int c = 0; c < nk && ok; ++c) {
                const int s = c % kStages;
                ok = mbar_wait(&full[s], (uint32_t)(c / kStages) & 1u) && !abort_flag;
                if (!ok) break;
                tc_fence_after();
                const uint32_t ab = saddr(smem + s * stage_bytes), bb = ab + a_bytes;
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)
                    mma_bf16(tmem, smem_desc(ab + kk * 2 * kLBO), smem_desc(bb + kk * 2 * kLBO), idesc,
                             (c > 0 || kk > 0) ? 1u : 0u);
                mma_commit(&empty[s]);
                ++ncommit[s];
            }
            if (ok) {
                mma_commit(&done);
            } else {
                abort_flag = 1;
                atomicExch(&g_tc_err, 1);
                // let the issued MMAs drain (bounded) before the accumulator is freed
                for (int s = 0; s < kStages; ++s)
                    if (ncommit[s] > 0) mbar_wait(&empty[s], (uint32_t)(ncommit[s] - 1) & 1u);
            }
        }
        __syncwarp();
    } else {
        // ---- producers: operand staging
        const long long mrow = m0 + tid;
        const bool row_ok = mrow < total;
        int rb = 0, rz = 0, ry = 0, rx = 0;
        if (row_ok) {
            long long r = mrow;
            rx = (int)(r % a.n3); r /= a.n3;
            ry = (int)(r % a.n2); r /= a.n2;
            rz = (int)(r % a.n1); rb = (int)(r / a.n1);
        }
        bool ok = true;
        for (int c = 0; c < nk + kStages - 2 && ok; ++c) {
            if (c < nk) {
                const int s = c % kStages;
                if (c >= kStages) ok = mbar_wait(&empty[s], (uint32_t)(c / kStages - 1) & 1u) && !abort_flag;
                if (!ok) break;
                unsigned char *base = smem + s * stage_bytes;
                const uint32_t ab = saddr(base), bb = saddr(base + a_bytes);
#pragma unroll
                for (int j = 0; j < kBK / 8; ++j) {
                    const int q = c * (kBK / 8) + j;
                    const bool in = row_ok && 8 * q < ktot;
                    const __nv_bfloat16 *src = in ? k8_src(a, cin_s, rb, rz, ry, rx, q) : a.src0;
                    cp_async16(ab + (tid >> 3) * kSBO + j * kLBO + (tid & 7) * 16, src, in ? 16 : 0);
                }
                for (int i = tid; i < N * (kBK / 8); i += kProducers) {
                    const int n = i / (kBK / 8), j = i - n * (kBK / 8);
                    const int k = 8 * (c * (kBK / 8) + j);
                    const bool in = k < ktot;
                    const int t = in ? k / cin_s : 0, ci = in ? k - t * cin_s : 0;
                    const __nv_bfloat16 *src = a.W + ((long long)t * N + n) * cin_s + ci;
                    cp_async16(bb + (n >> 3) * kSBO + j * kLBO + (n & 7) * 16, src, in ? 16 : 0);
                }
            }
            cp_async_commit();
            // chunk c - (kStages - 2) has landed for this thread: fence it for
            // the tensor core and report it
            cp_async_wait<kStages - 2>();
            const int r = c - (kStages - 2);
            if (r >= 0 && r < nk) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&full[r % kStages])) : "memory");
            }
        }
        cp_async_wait<0>();
        if (!ok) abort_flag = 1;
        // ---- epilogue: all MMAs done -> TMEM -> bias, ReLU -> global
        if (ok) ok = mbar_wait(&done, 0u) && !abort_flag;
        if (ok) {
            tc_fence_after();
            const long long m = m0 + tid;
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
                if (m < total) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        if (a.bias) v[i] += a.bias[c0 + i];
                        if (a.relu) v[i] = fmaxf(v[i], 0.f);
                    }
                    if (a.out_f32) {
                        float4 *o = reinterpret_cast<float4 *>(a.out_f32 + m * N + c0);
#pragma unroll
                        for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                    } else {
                        __nv_bfloat162 h[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                        uint4 *o = reinterpret_cast<uint4 *>(a.out_bf16 + m * N + c0);
                        o[0] = *reinterpret_cast<uint4 *>(&h[0]);
                        o[1] = *reinterpret_cast<uint4 *>(&h[4]);
                    }
                }
            }
        } else if (tid == 0) {
            atomicExch(&g_tc_err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMma)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}


// ---------------------------------------------------------------------------
// Halo-tile variant for grids that a 4 x 4 x 8 brick tiles: the CTA's 128
// output voxels are one brick; for each 16-channel chunk of the input the
// periodic 6 x 6 x 10 halo is loaded once (cp.async), and each tap's A
// operand (128 rows x 16 K) is copied out of it in shared memory, so every
// input row leaves L2 once per CTA instead of once per tap.  One MMA
// (K = 16) per (chunk, tap) stage; A/B in the no-swizzle K-major layout with
// LBO = 128 B, SBO = 256 B.
// ---------------------------------------------------------------------------
constexpr int kHZ = 6, kHY = 6, kHX = 10, kHalo = kHZ * kHY * kHX;   // halo rows
constexpr int kHSt = 4;                      // stage ring
constexpr int kHLag = 2;                     // stages of B loads in flight per thread
constexpr int kHSBO = 256;                   // K = 16: two K core matrices per 8-row group

__device__ __forceinline__ uint64_t smem_desc_h(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((kLBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((kHSBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void bar_producers() { asm volatile("bar.sync 1, %0;" ::"n"(kProducers) : "memory"); }

__global__ void __launch_bounds__(kThreads) k_conv3_tch(ConvArgs a, int ncols) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kHSt], empty[kHSt], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.cout;
    const int cin_s = a.c0s + a.c1s;
    const int nch = cin_s / 16;
    const int nst = nch * 27;                          // stages: (chunk, tap)
    const int a_bytes = kBM / 8 * kHSBO;               // 4 KB
    const int b_bytes = N / 8 * kHSBO;
    const int stage_bytes = a_bytes + b_bytes;
    unsigned char *halo = smem;                        // kHalo rows x 32 B
    unsigned char *ring = smem + kHalo * 32;
    // this CTA's brick
    const int bx3 = a.n3 / 8, by2 = a.n2 / 4, bz1 = a.n1 / 4;
    int r = blockIdx.x;
    const int xb = r % bx3; r /= bx3;
    const int yb = r % by2; r /= by2;
    const int zb = r % bz1;
    const int b = r / bz1;
    const int z0 = zb * 4, y0 = yb * 4, x0 = xb * 8;
    constexpr int kMma = kProducers / 32;

    if (warp == kMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < kHSt; ++q) {
            mbar_init(&full[q], kProducers);
            mbar_init(&empty[q], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == kMma) {
        if (lane == 0) {
            int ncommit[kHSt] = {};
            const uint32_t idesc = instr_desc(N);
            bool ok = true;
            for (int c = 0; c < nst && ok; ++c) {
                const int q = c % kHSt;
                ok = mbar_wait(&full[q], (uint32_t)(c / kHSt) & 1u) && !abort_flag;
                if (!ok) break;
                tc_fence_after();
                const uint32_t ab = saddr(ring + q * stage_bytes), bb = ab + a_bytes;
                mma_bf16(tmem, smem_desc_h(ab), smem_desc_h(bb), idesc, c > 0 ? 1u : 0u);
                mma_commit(&empty[q]);
                ++ncommit[q];
            }
            if (ok) {
                mma_commit(&done);
            } else {
                abort_flag = 1;
                atomicExch(&g_tc_err, 1);
                for (int q = 0; q < kHSt; ++q)
                    if (ncommit[q] > 0) mbar_wait(&empty[q], (uint32_t)(ncommit[q] - 1) & 1u);
            }
        }
        __syncwarp();
    } else {
        // my output row m = tid: brick offsets (bz, by, bx)
        const int bz = tid >> 5, by = (tid >> 3) & 3, bx = tid & 7;
        bool ok = true;
        int stage = 0, arrived = 0;
        auto arrive_upto = [&](int upto) {   // stages [arrived, upto) have landed
            if (arrived < upto) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (; arrived < upto; ++arrived)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&full[arrived % kHSt]))
                             : "memory");
        };
        // every producer passes the same named barriers: after a failed wait a
        // thread keeps going through them and only skips the work
        for (int cc = 0; cc < nch; ++cc) {
            // the halo of channel chunk cc (all earlier copies out of it are done)
            bar_producers();
            if (ok) {
                const bool first = cc * 16 < a.c0s;
                for (int h = tid; h < kHalo; h += kProducers) {
                    const int hx = h % kHX, hy = (h / kHX) % kHY, hz = h / (kHX * kHY);
                    const int zz = wrapi(z0 - 1 + hz, a.n1), yy = wrapi(y0 - 1 + hy, a.n2),
                              xx = wrapi(x0 - 1 + hx, a.n3);
                    const __nv_bfloat16 *src;
                    if (first) {
                        const long long v = (((long long)b * a.n1 + zz) * a.n2 + yy) * a.n3 + xx;
                        src = a.src0 + v * a.c0s + cc * 16;
                    } else {
                        const long long v = (((long long)b * (a.n1 >> 1) + (zz >> 1)) * (a.n2 >> 1) + (yy >> 1)) *
                                                (a.n3 >> 1) + (xx >> 1);
                        src = a.src1 + v * a.c1s + (cc * 16 - a.c0s);
                    }
                    cp_async16(saddr(halo + h * 32), src, 16);
                    cp_async16(saddr(halo + h * 32 + 16), src + 8, 16);
                }
            }
            cp_async_commit();
            asm volatile("cp.async.wait_all;" ::: "memory");
            if (ok) arrive_upto(stage);         // B loads of earlier stages completed too
            bar_producers();
            for (int t = 0; t < 27; ++t, ++stage) {
                if (!ok) continue;
                const int q = stage % kHSt;
                if (stage >= kHSt) ok = mbar_wait(&empty[q], (uint32_t)(stage / kHSt - 1) & 1u) && !abort_flag;
                if (!ok) continue;
                unsigned char *base = ring + q * stage_bytes;
                // A: my row's 16 channels at the tap's halo position
                const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
                const int h = ((bz + dz) * kHY + (by + dy)) * kHX + (bx + dx);
                const uint4 lo = *reinterpret_cast<const uint4 *>(halo + h * 32);
                const uint4 hi = *reinterpret_cast<const uint4 *>(halo + h * 32 + 16);
                *reinterpret_cast<uint4 *>(base + (tid >> 3) * kHSBO + (tid & 7) * 16) = lo;
                *reinterpret_cast<uint4 *>(base + (tid >> 3) * kHSBO + kLBO + (tid & 7) * 16) = hi;
                // B: W[t][n][cc*16 .. +16]
                const uint32_t bb = saddr(base + a_bytes);
                for (int i = tid; i < N * 2; i += kProducers) {
                    const int n = i >> 1, j = i & 1;
                    const __nv_bfloat16 *src = a.W + ((long long)t * N + n) * cin_s + cc * 16 + j * 8;
                    cp_async16(bb + (n >> 3) * kHSBO + j * kLBO + (n & 7) * 16, src, 16);
                }
                cp_async_commit();
                cp_async_wait<kHLag>();
                arrive_upto(stage + 1 - kHLag);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (ok) arrive_upto(nst);
        if (!ok) abort_flag = 1;
        if (ok) ok = mbar_wait(&done, 0u) && !abort_flag;
        if (ok) {
            tc_fence_after();
            const long long m = (((long long)b * a.n1 + z0 + bz) * a.n2 + y0 + by) * a.n3 + x0 + bx;
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    if (a.bias) v[i] += a.bias[c0 + i];
                    if (a.relu) v[i] = fmaxf(v[i], 0.f);
                }
                if (a.out_f32) {
                    float4 *o = reinterpret_cast<float4 *>(a.out_f32 + m * N + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                } else {
                    __nv_bfloat162 hv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) hv[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                    uint4 *o = reinterpret_cast<uint4 *>(a.out_bf16 + m * N + c0);
                    o[0] = *reinterpret_cast<uint4 *>(&hv[0]);
                    o[1] = *reinterpret_cast<uint4 *>(&hv[4]);
                }
            }
        } else if (tid == 0) {
            atomicExch(&g_tc_err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMma)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}


// ---------------------------------------------------------------------------
// Halo tiles read in place.  The halo of a 16-channel chunk is stored as
// three copies, one per tap offset dy, each [6 z][4 y][10 x] rows of 16 bytes
// (channels 0-7 and 8-15 in two planes).  In copy dy the row of voxel
// (bz, by, bx) at tap (dz, dy, dx) is (bz + dz) * 40 + by * 10 + bx + dx: the
// 8 voxels of a brick row are 8 consecutive rows (one core matrix), the 16
// row groups (bz, by) lie 160 B apart, and the tap only moves the start.  So
// the A operand of every tap is a canonical K-major layout (SBO = 160 B,
// LBO = one plane) read straight from the halo: no per-tap copies, and the
// 27 MMAs of a chunk follow one another with one handoff per chunk.  B holds
// the chunk's weights for all 27 taps (K-major, N x 32 bytes per tap).
// ---------------------------------------------------------------------------
constexpr int kDY = 4;                           // y rows of one copy
constexpr int kDRows = kHZ * kDY * kHX;          // 240 rows per copy
constexpr int kDPlane = kDRows * 16;             // one channel half of one copy
constexpr int kDHalo = 3 * 2 * kDPlane;          // 23040 B
constexpr int kDSBO = kHX * 16;                  // (bz, by) row groups

__device__ __forceinline__ uint64_t smem_desc_d(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((kDPlane >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((kDSBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// the 27 tap MMAs of one chunk: A read in place from the halo copies, B the
// chunk's weights (32 N bytes per tap).  The descriptors are built once; a
// tap only adds its start offset (>> 4) to the address field, which stays
// inside its 14 bits because shared memory ends below 256 KB.
__device__ __forceinline__ void tap_mmas(uint32_t d, uint32_t ab, uint32_t bb, int N, uint32_t idesc, bool acc) {
    const uint64_t ad = smem_desc_d(ab), bd = smem_desc_h(bb);
    const uint64_t bstep = (uint64_t)(2 * N);          // 32 N bytes >> 4
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        constexpr int kRow = kDY * kHX;
        const int off = ((t / 3) % 3) * 2 * kDPlane + ((t / 9) * kRow + t % 3) * 16;
        mma_bf16(d, ad + (uint64_t)(off >> 4), bd + bstep * t, idesc, (acc || t > 0) ? 1u : 0u);
    }
}

__global__ void __launch_bounds__(kThreads) k_conv3_tcd(ConvArgs a, int ncols, int ring) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[2], empty[2], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.cout;
    const int cin_s = a.c0s + a.c1s;
    const int nch = cin_s / 16;
    const int b_bytes = 27 * 32 * N;
    const int stage_bytes = kDHalo + b_bytes;
    const int bx3 = a.n3 / 8, by2 = a.n2 / 4, bz1 = a.n1 / 4;
    int r = blockIdx.x;
    const int xb = r % bx3; r /= bx3;
    const int yb = r % by2; r /= by2;
    const int zb = r % bz1;
    const int b = r / bz1;
    const int z0 = zb * 4, y0 = yb * 4, x0 = xb * 8;
    constexpr int kMma = kProducers / 32;

    if (warp == kMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            mbar_init(&full[q], kProducers);
            mbar_init(&empty[q], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == kMma) {
        if (lane == 0) {
            int ncommit[2] = {0, 0};
            const uint32_t idesc = instr_desc(N);
            bool ok = true;
            for (int cc = 0; cc < nch && ok; ++cc) {
                const int q = cc % ring;
                ok = mbar_wait(&full[q], (uint32_t)(cc / ring) & 1u) && !abort_flag;
                if (!ok) break;
                tc_fence_after();
                const uint32_t ab = saddr(smem + q * stage_bytes), bb = ab + kDHalo;
                tap_mmas(tmem, ab, bb, N, idesc, cc > 0);
                mma_commit(&empty[q]);
                ++ncommit[q];
            }
            if (ok) {
                mma_commit(&done);
            } else {
                abort_flag = 1;
                atomicExch(&g_tc_err, 1);
                for (int q = 0; q < 2; ++q)
                    if (ncommit[q] > 0) mbar_wait(&empty[q], (uint32_t)(ncommit[q] - 1) & 1u);
            }
        }
        __syncwarp();
    } else {
        // my halo rows: (copy, row) pairs tid + 128 k of the 3 x 240, with the
        // periodic source voxel of each (full resolution and half resolution)
        constexpr int kMine = (3 * kDRows + kProducers - 1) / kProducers;   // 6
        int vfull[kMine], vhalf[kMine], dst[kMine];
        const int h1 = a.n1 >> 1, h2 = a.n2 >> 1, h3 = a.n3 >> 1;
#pragma unroll
        for (int k = 0; k < kMine; ++k) {
            const int i = tid + k * kProducers;
            const int dy = i / kDRows, row = i - dy * kDRows;
            const int xr = row % kHX, yr = (row / kHX) % kDY, zr = row / (kHX * kDY);
            const int zz = wrapi(z0 - 1 + zr, a.n1), yy = wrapi(y0 - 1 + yr + dy, a.n2),
                      xx = wrapi(x0 - 1 + xr, a.n3);
            vfull[k] = (zz * a.n2 + yy) * a.n3 + xx;
            vhalf[k] = ((zz >> 1) * h2 + (yy >> 1)) * h3 + (xx >> 1);
            dst[k] = dy * 2 * kDPlane + row * 16;
        }
        const __nv_bfloat16 *s0 = a.src0 + (long long)b * a.n1 * a.n2 * a.n3 * a.c0s;
        const __nv_bfloat16 *s1 = a.c1s ? a.src1 + (long long)b * h1 * h2 * h3 * a.c1s : nullptr;
        bool ok = true;
        for (int cc = 0; cc < nch; ++cc) {
            const int q = cc % ring;
            if (!ok) continue;
            if (cc >= ring) ok = mbar_wait(&empty[q], (uint32_t)(cc / ring - 1) & 1u) && !abort_flag;
            if (!ok) continue;
            unsigned char *st = smem + q * stage_bytes;
            const bool first = cc * 16 < a.c0s;
#pragma unroll
            for (int k = 0; k < kMine; ++k) {
                if (tid + k * kProducers < 3 * kDRows) {
                    const __nv_bfloat16 *src = first ? s0 + (long long)vfull[k] * a.c0s + cc * 16
                                                     : s1 + (long long)vhalf[k] * a.c1s + (cc * 16 - a.c0s);
                    cp_async16(saddr(st + dst[k]), src, 16);
                    cp_async16(saddr(st + dst[k] + kDPlane), src + 8, 16);
                }
            }
            // weights of the chunk, all 27 taps: W[t][n][cc*16 .. +16]
            const uint32_t bb = saddr(st + kDHalo);
            for (int i = tid; i < 54 * N; i += kProducers) {
                const int t = i / (2 * N), rem = i - t * 2 * N, n = rem >> 1, j = rem & 1;
                const __nv_bfloat16 *src = a.W + ((long long)t * N + n) * cin_s + cc * 16 + j * 8;
                cp_async16(bb + t * 32 * N + (n >> 3) * kHSBO + j * kLBO + (n & 7) * 16, src, 16);
            }
            cp_async_commit();
            asm volatile("cp.async.wait_all;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&full[q])) : "memory");
        }
        if (!ok) abort_flag = 1;
        if (ok) ok = mbar_wait(&done, 0u) && !abort_flag;
        if (ok) {
            tc_fence_after();
            const int bz = tid >> 5, by = (tid >> 3) & 3, bx = tid & 7;
            const long long m = (((long long)b * a.n1 + z0 + bz) * a.n2 + y0 + by) * a.n3 + x0 + bx;
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    if (a.bias) v[i] += a.bias[c0 + i];
                    if (a.relu) v[i] = fmaxf(v[i], 0.f);
                }
                if (a.out_f32) {
                    float4 *o = reinterpret_cast<float4 *>(a.out_f32 + m * N + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                } else {
                    __nv_bfloat162 hv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) hv[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                    uint4 *o = reinterpret_cast<uint4 *>(a.out_bf16 + m * N + c0);
                    o[0] = *reinterpret_cast<uint4 *>(&hv[0]);
                    o[1] = *reinterpret_cast<uint4 *>(&hv[4]);
                }
            }
        } else if (tid == 0) {
            atomicExch(&g_tc_err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMma)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// Persistent form of the in-place halo convolution: a CTA keeps the weights
// of all its chunks in shared memory and walks bricks blockIdx.x, +gridDim.x,
// ...  Halo stages (brick, chunk) go through a 2-slot ring and the brick's
// accumulator alternates between two TMEM column ranges, so the loads of
// brick j overlap the MMAs of brick j-1 and the epilogue of brick j-1 runs
// while the loads of brick j are in flight.  Barriers: hfull/hempty per halo
// slot (producers / MMA commit), afull/aempty per accumulator (MMA commit /
// producers after reading it).
__global__ void __launch_bounds__(kThreads) k_conv3_tcp(ConvArgs a, int ncols) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t hfull[2], hempty[2], afull[2], aempty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.cout;
    const int cin_s = a.c0s + a.c1s;
    const int nch = cin_s / 16;
    const int w_bytes = nch * 27 * 32 * N;
    unsigned char *halo = smem + w_bytes;              // 2 slots of kDHalo
    const int bx3 = a.n3 / 8, by2 = a.n2 / 4, bz1 = a.n1 / 4;
    const int nbricks = bx3 * by2 * bz1 * a.B;
    const int nb = blockIdx.x < nbricks ? (nbricks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    constexpr int kMma = kProducers / 32;
    if (nb == 0) return;

    if (warp == kMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            mbar_init(&hfull[q], kProducers);
            mbar_init(&hempty[q], 1);
            mbar_init(&afull[q], 1);
            mbar_init(&aempty[q], kProducers);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == kMma) {
        if (lane == 0) {
            int nh[2] = {0, 0}, na[2] = {0, 0};   // commits per barrier
            const uint32_t idesc = instr_desc(N);
            const uint32_t wb = saddr(smem);
            bool ok = true;
            for (int j = 0; j < nb && ok; ++j) {
                const int s = j & 1;
                if (j >= 2) ok = mbar_wait(&aempty[s], (uint32_t)((j >> 1) - 1) & 1u) && !abort_flag;
                if (!ok) break;
                tc_fence_after();
                for (int cc = 0; cc < nch && ok; ++cc) {
                    const int k = j * nch + cc, q = k & 1;
                    ok = mbar_wait(&hfull[q], (uint32_t)(k >> 1) & 1u) && !abort_flag;
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t ab = saddr(halo + q * kDHalo), bb = wb + cc * 27 * 32 * N;
                    tap_mmas(tmem + (uint32_t)(s * N), ab, bb, N, idesc, cc > 0);
                    mma_commit(&hempty[q]);
                    ++nh[q];
                }
                if (!ok) break;
                mma_commit(&afull[s]);
                ++na[s];
            }
            if (!ok) {
                abort_flag = 1;
                atomicExch(&g_tc_err, 1);
                for (int q = 0; q < 2; ++q) {
                    if (nh[q] > 0) mbar_wait(&hempty[q], (uint32_t)(nh[q] - 1) & 1u);
                    if (na[q] > 0) mbar_wait(&afull[q], (uint32_t)(na[q] - 1) & 1u);
                }
            }
        }
        __syncwarp();
    } else {
        // my halo rows: (copy, row) pairs tid + 128 k of the 3 x 240
        constexpr int kMine = (3 * kDRows + kProducers - 1) / kProducers;   // 6
        int rz[kMine], ry[kMine], rx[kMine], dst[kMine];
#pragma unroll
        for (int k = 0; k < kMine; ++k) {
            const int i = tid + k * kProducers;
            const int dy = i / kDRows, row = i - dy * kDRows;
            rx[k] = row % kHX - 1;
            ry[k] = (row / kHX) % kDY + dy - 1;
            rz[k] = row / (kHX * kDY) - 1;
            dst[k] = dy * 2 * kDPlane + row * 16;
        }
        const int h1 = a.n1 >> 1, h2 = a.n2 >> 1, h3 = a.n3 >> 1;
        const int bz = tid >> 5, by = (tid >> 3) & 3, bx = tid & 7;
        // weights of every chunk and tap: W[t][n][cc*16 .. +16], joined to the first halo group
        {
            const uint32_t wb = saddr(smem);
            for (int i = tid; i < 54 * N * nch; i += kProducers) {
                const int cc = i / (54 * N), i2 = i - cc * 54 * N;
                const int t = i2 / (2 * N), rem = i2 - t * 2 * N, n = rem >> 1, jj = rem & 1;
                const __nv_bfloat16 *src = a.W + ((long long)t * N + n) * cin_s + cc * 16 + jj * 8;
                cp_async16(wb + (cc * 27 + t) * 32 * N + (n >> 3) * kHSBO + jj * kLBO + (n & 7) * 16, src, 16);
            }
        }
        bool ok = true;
        int vfull[kMine], vhalf[kMine];
        int pb = 0, pz0 = 0, py0 = 0, px0 = 0;              // the previous brick, for its epilogue
        auto epilogue = [&](int j) {                        // brick j's accumulator to the output
            const int s = j & 1;
            ok = mbar_wait(&afull[s], (uint32_t)(j >> 1) & 1u) && !abort_flag;
            if (!ok) return;
            tc_fence_after();
            const long long m = (((long long)pb * a.n1 + pz0 + bz) * a.n2 + py0 + by) * a.n3 + px0 + bx;
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * N + c0), v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    if (a.bias) v[i] += a.bias[c0 + i];
                    if (a.relu) v[i] = fmaxf(v[i], 0.f);
                }
                if (a.out_f32) {
                    float4 *o = reinterpret_cast<float4 *>(a.out_f32 + m * N + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                } else {
                    __nv_bfloat162 hv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) hv[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                    uint4 *o = reinterpret_cast<uint4 *>(a.out_bf16 + m * N + c0);
                    o[0] = *reinterpret_cast<uint4 *>(&hv[0]);
                    o[1] = *reinterpret_cast<uint4 *>(&hv[4]);
                }
            }
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&aempty[s])) : "memory");
        };
        for (int j = 0; j < nb && ok; ++j) {
            int r = (int)blockIdx.x + j * (int)gridDim.x;
            const int xb = r % bx3; r /= bx3;
            const int yb = r % by2; r /= by2;
            const int zb = r % bz1;
            const int b = r / bz1;
            const int z0 = zb * 4, y0 = yb * 4, x0 = xb * 8;
#pragma unroll
            for (int k = 0; k < kMine; ++k) {
                const int zz = wrapi(z0 + rz[k], a.n1), yy = wrapi(y0 + ry[k], a.n2), xx = wrapi(x0 + rx[k], a.n3);
                vfull[k] = (zz * a.n2 + yy) * a.n3 + xx;
                vhalf[k] = ((zz >> 1) * h2 + (yy >> 1)) * h3 + (xx >> 1);
            }
            const __nv_bfloat16 *s0 = a.src0 + (long long)b * a.n1 * a.n2 * a.n3 * a.c0s;
            const __nv_bfloat16 *s1 = a.c1s ? a.src1 + (long long)b * h1 * h2 * h3 * a.c1s : nullptr;
            for (int cc = 0; cc < nch && ok; ++cc) {
                const int k = j * nch + cc, q = k & 1;
                if (k >= 2) ok = mbar_wait(&hempty[q], (uint32_t)((k >> 1) - 1) & 1u) && !abort_flag;
                if (!ok) break;
                unsigned char *st = halo + q * kDHalo;
                const bool first = cc * 16 < a.c0s;
#pragma unroll
                for (int kk = 0; kk < kMine; ++kk) {
                    if (tid + kk * kProducers < 3 * kDRows) {
                        const __nv_bfloat16 *src = first ? s0 + (long long)vfull[kk] * a.c0s + cc * 16
                                                         : s1 + (long long)vhalf[kk] * a.c1s + (cc * 16 - a.c0s);
                        cp_async16(saddr(st + dst[kk]), src, 16);
                        cp_async16(saddr(st + dst[kk] + kDPlane), src + 8, 16);
                    }
                }
                cp_async_commit();
                if (cc == 0 && j > 0) epilogue(j - 1);   // overlaps the loads just issued
                asm volatile("cp.async.wait_all;" ::: "memory");
                if (!ok) break;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&hfull[q])) : "memory");
            }
            pb = b; pz0 = z0; py0 = y0; px0 = x0;
        }
        if (ok) epilogue(nb - 1);
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (!ok) {
            abort_flag = 1;
            if (tid == 0) atomicExch(&g_tc_err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMma)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------
// Weight gradient on tcgen05: dW[t][co][ci] = sum_v G[v][co] X[v + d_t][ci].
// D rows are (tap, input channel) pairs, 8 taps x 16 channels = 128 per tap
// group (4 groups cover 27 taps), N = c_out, K = the 128 voxels of a brick.
// Both operands are MN-major, which is their natural layout: a 16-byte row
// of a core matrix is 8 channels of one voxel (X rows out of the halo, G
// rows out of the output gradient), 8 voxels per core matrix; MN-adjacent
// core matrices 2048 B apart, K-adjacent ones 128 B.  Without swizzling the
// descriptor of an MN-major operand takes the K-direction stride as its
// leading byte offset and the MN-direction stride as its stride byte offset
// (as for K-major operands, where the 8-row groups run along MN).  A CTA takes
// one 16-channel chunk of the input and a range of bricks, keeps the four
// group accumulators in tensor memory, and writes its split's partial sums.
// ---------------------------------------------------------------------------
constexpr int kWgMn = 2048;        // MN-adjacent core matrices (16 K-groups x 128 B): SBO
constexpr int kWgK = 128;          // K-adjacent core matrices: LBO
constexpr int kWgATile = 16 * kWgMn;   // 128 rows x 128 K, 32 KB

__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((kWgK >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((kWgMn >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::f16, FP32 accumulator, BF16 A and B, both MN-major (bits 15, 16)
__device__ __forceinline__ uint32_t instr_desc_mn(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kBM >> 4) << 24);
}

// A tile of tap group GRP for one voxel: rows (tap, channel half) of the
// voxel's column, taken from the two halo planes at the taps' offsets (all
// loads issued before the stores)
template <int GRP>
__device__ __forceinline__ void wg_copy(unsigned char *at, const unsigned char *hv) {
    constexpr int kNt = GRP < 3 ? 8 : 3;
    constexpr int kPlane = kHalo * 16;
    uint4 r[2 * kNt];
#pragma unroll
    for (int k = 0; k < kNt; ++k) {
        const int t = GRP * 8 + k;
        const int off = (((t / 9) * kHY + (t / 3) % 3) * kHX + t % 3) * 16;
        r[2 * k] = *reinterpret_cast<const uint4 *>(hv + off);
        r[2 * k + 1] = *reinterpret_cast<const uint4 *>(hv + kPlane + off);
    }
#pragma unroll
    for (int m = 0; m < 2 * kNt; ++m) *reinterpret_cast<uint4 *>(at + m * kWgMn) = r[m];
}

__global__ void __launch_bounds__(kThreads) k_wgrad3_tc(WgradArgs w, int ncols, int bricks_per_cta) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[2], empty[2], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const ConvArgs &a = w.in;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = w.cout;
    const int cin_s = a.c0s + a.c1s;
    const int cc = blockIdx.y;
    const int split = blockIdx.x;
    const int bx3 = a.n3 / 8, by2 = a.n2 / 4, bz1 = a.n1 / 4;
    const long long nbricks = (long long)bx3 * by2 * bz1 * a.B;
    const long long bb0 = (long long)split * bricks_per_cta;
    const long long bb1 = bb0 + bricks_per_cta < nbricks ? bb0 + bricks_per_cta : nbricks;
    constexpr int kMma = kProducers / 32;
    if (bb0 >= bb1) {   // no voxels in this split: its partial sums are zero
        for (int i = tid; i < 27 * N * 16; i += kThreads) {
            const int ci = i % 16, r = i / 16, co = r % N, t = r / N;
            w.partial[(((long long)split * 27 + t) * N + co) * cin_s + cc * 16 + ci] = 0.f;
        }
        return;
    }
    // two bricks in flight: halo[2] (two planes of 16-byte rows, channels
    // 0-7 and 8-15), G tile[2], and the two A-tile stages
    constexpr int kPlane = kHalo * 16;
    const int gbytes = (N / 8) * kWgMn;
    unsigned char *halo = smem;                              // 2 x 2 planes
    unsigned char *gt = smem + 4 * kPlane;                   // 2 x G tile
    unsigned char *ring = gt + 2 * gbytes;                   // 2 x A tile

    if (warp == kMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            mbar_init(&full[q], kProducers);
            mbar_init(&empty[q], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int nst = (int)(bb1 - bb0) * 4;                    // (brick, tap group) stages

    if (warp == kMma) {
        if (lane == 0) {
            int ncommit[2] = {0, 0};
            const uint32_t idesc = instr_desc_mn(N);
            bool ok = true;
            for (int c = 0; c < nst && ok; ++c) {
                const int q = c & 1, grp = c & 3;
                ok = mbar_wait(&full[q], (uint32_t)(c >> 1) & 1u) && !abort_flag;
                if (!ok) break;
                tc_fence_after();
                const uint32_t ab = saddr(ring + q * kWgATile);
                const uint32_t gb = saddr(gt + ((c >> 2) & 1) * gbytes);
#pragma unroll
                for (int j = 0; j < 8; ++j)   // K = 16 voxels = 2 K-adjacent core matrices per MMA
                    mma_bf16(tmem + (uint32_t)(grp * N), smem_desc_mn(ab + j * 2 * kWgK),
                             smem_desc_mn(gb + j * 2 * kWgK), idesc, (c >= 4 || j > 0) ? 1u : 0u);
                mma_commit(&empty[q]);
                ++ncommit[q];
            }
            if (ok) {
                mma_commit(&done);
            } else {
                abort_flag = 1;
                atomicExch(&g_tc_err, 1);
                for (int q = 0; q < 2; ++q)
                    if (ncommit[q] > 0) mbar_wait(&empty[q], (uint32_t)(ncommit[q] - 1) & 1u);
            }
        }
        __syncwarp();
    } else {
        // producer row = voxel tid of the brick: offsets (bz, by, bx)
        const int bz = tid >> 5, by = (tid >> 3) & 3, bx = tid & 7;
        const int hrow = ((bz * kHY + by) * kHX + bx) * 16;   // my voxel's halo row at tap offset 0
        const bool first = cc * 16 < a.c0s;
        // my halo rows (at most 3 of the 360) and their positions in the halo
        int hz[3], hy[3], hx[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int h = tid + r * kProducers;
            hx[r] = h % kHX;
            hy[r] = (h / kHX) % kHY;
            hz[r] = h / (kHX * kHY);
        }
        // the chunk's source: full resolution, or the half-resolution second
        // source read with nearest-neighbour upsampling
        const int sh = first ? 0 : 1;
        const int m1 = a.n1 >> sh, m2 = a.n2 >> sh, m3 = a.n3 >> sh;
        const int cs = first ? a.c0s : a.c1s;
        const __nv_bfloat16 *sbase = first ? a.src0 + cc * 16 : a.src1 + (cc * 16 - a.c0s);
        // halo of brick br into halo buffer hb, my G row into G buffer hb
        auto load_brick = [&](long long br, int hb) {
            long long rr = br;
            const int xb = (int)(rr % bx3); rr /= bx3;
            const int yb = (int)(rr % by2); rr /= by2;
            const int zb = (int)(rr % bz1);
            const int b = (int)(rr / bz1);
            const int z0 = zb * 4, y0 = yb * 4, x0 = xb * 8;
            const __nv_bfloat16 *src_b = sbase + (long long)b * m1 * m2 * m3 * cs;
            unsigned char *hp = halo + hb * 2 * kPlane + tid * 16;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                if (tid + r * kProducers < kHalo) {
                    const int zz = wrapi(z0 - 1 + hz[r], a.n1) >> sh, yy = wrapi(y0 - 1 + hy[r], a.n2) >> sh,
                              xx = wrapi(x0 - 1 + hx[r], a.n3) >> sh;
                    const __nv_bfloat16 *src = src_b + (long long)((zz * m2 + yy) * m3 + xx) * cs;
                    cp_async16(saddr(hp + r * kProducers * 16), src, 16);
                    cp_async16(saddr(hp + kPlane + r * kProducers * 16), src + 8, 16);
                }
            }
            const long long v = (((long long)b * a.n1 + z0 + bz) * a.n2 + y0 + by) * a.n3 + x0 + bx;
            const __nv_bfloat16 *g = w.G + v * N;
            unsigned char *gp = gt + hb * gbytes + (tid >> 3) * kWgK + (tid & 7) * 16;
            for (int ng = 0; ng < N / 8; ++ng) cp_async16(saddr(gp + ng * kWgMn), g + ng * 8, 16);
            cp_async_commit();
        };
        bool ok = true;
        load_brick(bb0, 0);
        for (long long br = bb0; br < bb1; ++br) {
            const int i = (int)(br - bb0), hb = i & 1;
            asm volatile("cp.async.wait_all;" ::: "memory");
            bar_producers();     // brick br's halo and G tile are in; brick br-1's copies are done
            const unsigned char *hp = halo + hb * 2 * kPlane;
            for (int grp = 0; grp < 4; ++grp) {
                const int c = 4 * i + grp, q = c & 1;
                if (!ok) continue;
                if (c >= 2) ok = mbar_wait(&empty[q], (uint32_t)((c >> 1) - 1) & 1u) && !abort_flag;
                if (!ok) continue;
                // stage c-2 is the last MMA of brick br-1: its buffers take brick br+1
                if (grp == 1 && br + 1 < bb1) load_brick(br + 1, hb ^ 1);
                unsigned char *at = ring + q * kWgATile + (tid >> 3) * kWgK + (tid & 7) * 16;
                switch (grp) {
                    case 0: wg_copy<0>(at, hp + hrow); break;
                    case 1: wg_copy<1>(at, hp + hrow); break;
                    case 2: wg_copy<2>(at, hp + hrow); break;
                    default: wg_copy<3>(at, hp + hrow); break;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&full[q])) : "memory");
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (!ok) abort_flag = 1;
        if (ok) ok = mbar_wait(&done, 0u) && !abort_flag;
        if (ok) {
            tc_fence_after();
            const int row = warp * 32 + lane;               // (tap in group, channel)
            const int tl = row >> 4, ci = row & 15;
            for (int grp = 0; grp < 4; ++grp) {
                const int t = grp * 8 + tl;
                for (int c0 = 0; c0 < N; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(grp * N + c0), v);
                    if (t < 27) {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            w.partial[(((long long)split * 27 + t) * N + c0 + i) * cin_s + cc * 16 + ci] = v[i];
                    }
                }
            }
        } else if (tid == 0) {
            atomicExch(&g_tc_err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMma)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace

int conv3_forward_tc(const ConvArgs &a, cudaStream_t st) {
    if ((a.cout & 15) || a.cout > 256 || a.cout < 16 || (a.c0s & 15) || (a.c1s & 15) || a.c0s <= 0) return -1;
    if (a.c1s && (!a.src1 || (a.n1 | a.n2 | a.n3) & 1)) return -1;
    int ncols = 32;
    while (ncols < a.cout) ncols <<= 1;
    static bool attr = false;
    if (!attr) {
        int dev = 0, lim = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncSetAttribute(k_conv3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - 1024);
        cudaFuncSetAttribute(k_conv3_tch, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - 1024);
        cudaFuncSetAttribute(k_conv3_tcd, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - 1024);
        cudaFuncSetAttribute(k_conv3_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - 1024);
        // all of the unified L1/shared array as shared memory, so that the
        // CTAs that the shared-memory budget allows are resident together
        cudaFuncSetAttribute(k_conv3_tcd, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_conv3_tcp, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_conv3_tch, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        attr = true;
    }
    const bool bricks_tile = a.n1 % 4 == 0 && a.n2 % 4 == 0 && a.n3 % 8 == 0;
    const size_t w_bytes = (size_t)(a.c0s + a.c1s) / 16 * 27 * 32 * a.cout;
    if (bricks_tile && a.cout <= 128 && w_bytes <= 96 * 1024) {
        // persistent CTAs with the weights resident; two TMEM accumulators
        int ncols2 = 32;
        while (ncols2 < 2 * a.cout) ncols2 <<= 1;
        size_t smem = w_bytes + 2 * (size_t)kDHalo;
        const size_t floor = 233472 / (512 / ncols2 + 1) + 1024;
        if (smem < floor) smem = floor;
        static int nsm = 0;
        if (!nsm) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        }
        // CTAs per SM that shared memory, registers and tensor memory allow
        static int regs = 0;
        if (!regs) {
            cudaFuncAttributes fa{};
            cudaFuncGetAttributes(&fa, k_conv3_tcp);
            regs = fa.numRegs > 0 ? (fa.numRegs + 7) / 8 * 8 : 255;
        }
        int per_sm = (int)(233472 / (smem + 2048));
        per_sm = per_sm < 65536 / (regs * kThreads) ? per_sm : 65536 / (regs * kThreads);
        per_sm = per_sm < 512 / ncols2 ? per_sm : 512 / ncols2;
        if (per_sm < 1) per_sm = 1;
        const long long bricks = (long long)(a.n1 / 4) * (a.n2 / 4) * (a.n3 / 8) * a.B;
        const long long grid = bricks < (long long)per_sm * nsm ? bricks : (long long)per_sm * nsm;
        k_conv3_tcp<<<(unsigned)grid, kThreads, smem, st>>>(a, ncols2);
        return 0;
    }
    if (bricks_tile && a.cout <= 128) {
        // halo tiles read in place: two chunk stages where they fit in about
        // half of the shared memory, else one
        const size_t stage = (size_t)kDHalo + 27 * 32 * (size_t)a.cout;
        const int ring = (a.c0s + a.c1s > 16 && 2 * stage <= 116 * 1024) ? 2 : 1;
        size_t smem = ring * stage;
        const size_t floor = 233472 / (512 / ncols + 1) + 1024;
        if (smem < floor) smem = floor;
        const long long bricks = (long long)(a.n1 / 4) * (a.n2 / 4) * (a.n3 / 8) * a.B;
        k_conv3_tcd<<<(unsigned)bricks, kThreads, smem, st>>>(a, ncols, ring);
        return 0;
    }
    if (a.n1 % 4 == 0 && a.n2 % 4 == 0 && a.n3 % 8 == 0) {
        // halo tiles; at least enough shared memory per CTA that the CTAs
        // resident on an SM never ask for more than its 512 TMEM columns
        size_t smem = (size_t)kHalo * 32 + (size_t)kHSt * (kBM / 8 * kHSBO + a.cout / 8 * kHSBO);
        const size_t floor = 233472 / (512 / ncols + 1) + 1024;
        if (smem < floor) smem = floor;
        const long long bricks = (long long)(a.n1 / 4) * (a.n2 / 4) * (a.n3 / 8) * a.B;
        k_conv3_tch<<<(unsigned)bricks, kThreads, smem, st>>>(a, ncols);
        return 0;
    }
    const size_t smem = (size_t)kStages * (kBM / 8 * kSBO + a.cout / 8 * kSBO);
    const long long total = (long long)a.n1 * a.n2 * a.n3 * a.B;
    k_conv3_tc<<<(unsigned)((total + kBM - 1) / kBM), kThreads, smem, st>>>(a, ncols);
    return 0;
}

int conv3_wgrad_tc(const WgradArgs &w, cudaStream_t st) {
    const ConvArgs &a = w.in;
    if ((w.cout & 15) || w.cout > 64 || w.cout < 16 || (a.c0s & 15) || (a.c1s & 15) || w.S <= 0) return -1;
    if (a.n1 % 4 || a.n2 % 4 || a.n3 % 8) return -1;
    int ncols = 32;
    while (ncols < 4 * w.cout) ncols <<= 1;
    static bool attr = false;
    if (!attr) {
        int dev = 0, lim = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncSetAttribute(k_wgrad3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - 1024);
        cudaFuncSetAttribute(k_wgrad3_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        attr = true;
    }
    size_t smem = 2 * ((size_t)kHalo * 32 + (size_t)(w.cout / 8) * kWgMn) + 2 * (size_t)kWgATile;
    const size_t floor = 233472 / (512 / ncols + 1) + 1024;    // TMEM columns per SM stay <= 512
    if (smem < floor) smem = floor;
    const long long nbricks = (long long)(a.n1 / 4) * (a.n2 / 4) * (a.n3 / 8) * a.B;
    const int bpc = (int)((nbricks + w.S - 1) / w.S);
    const dim3 grid(w.S, (a.c0s + a.c1s) / 16);
    k_wgrad3_tc<<<grid, kThreads, smem, st>>>(w, ncols, bpc);
    return 0;
}

int conv3_tc_error(int clear) {
    int e = 0;
    cudaMemcpyFromSymbol(&e, g_tc_err, sizeof(int));
    if (clear && e) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tc_err, &z, sizeof(int));
    }
    return e;
}

}  // namespace hnet
