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
    unsigned char *halo = smem;                              // kHalo rows x 32 B
    unsigned char *gt = smem + kHalo * 32;                   // G tile: N/8 x 2048 B
    unsigned char *ring = gt + (N / 8) * kWgMn;           // two A tiles

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
            const uint32_t gb = saddr(gt);
            bool ok = true;
            for (int c = 0; c < nst && ok; ++c) {
                const int q = c & 1, grp = c & 3;
                ok = mbar_wait(&full[q], (uint32_t)(c >> 1) & 1u) && !abort_flag;
                if (!ok) break;
                tc_fence_after();
                const uint32_t ab = saddr(ring + q * kWgATile);
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
        const bool first = cc * 16 < a.c0s;
        bool ok = true;
        int c = 0;
        for (long long br = bb0; br < bb1; ++br) {
            long long rr = br;
            const int xb = (int)(rr % bx3); rr /= bx3;
            const int yb = (int)(rr % by2); rr /= by2;
            const int zb = (int)(rr % bz1);
            const int b = (int)(rr / bz1);
            const int z0 = zb * 4, y0 = yb * 4, x0 = xb * 8;
            // the previous brick's MMAs read the G tile: wait for the last of them
            if (ok && c > 0) ok = mbar_wait(&empty[(c - 1) & 1], (uint32_t)((c - 1) >> 1) & 1u) && !abort_flag;
            bar_producers();
            if (ok) {
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
                // G rows of my voxel: N/8 chunks of 8 output channels
                const long long v = (((long long)b * a.n1 + z0 + bz) * a.n2 + y0 + by) * a.n3 + x0 + bx;
                const __nv_bfloat16 *g = w.G + v * N;
                for (int ng = 0; ng < N / 8; ++ng)
                    cp_async16(saddr(gt + ng * kWgMn + (tid >> 3) * kWgK + (tid & 7) * 16), g + ng * 8, 16);
            }
            cp_async_commit();
            asm volatile("cp.async.wait_all;" ::: "memory");
            bar_producers();
            for (int grp = 0; grp < 4; ++grp, ++c) {
                if (!ok) continue;
                const int q = c & 1;
                if (c >= 2) ok = mbar_wait(&empty[q], (uint32_t)((c >> 1) - 1) & 1u) && !abort_flag;
                if (!ok) continue;
                unsigned char *at = ring + q * kWgATile;
                // A rows (tap, channel half) x K = my voxel: 16 bytes each
#pragma unroll
                for (int mg = 0; mg < 16; ++mg) {
                    const int t = grp * 8 + (mg >> 1);
                    if (t < 27) {
                        const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
                        const int h = ((bz + dz) * kHY + (by + dy)) * kHX + (bx + dx);
                        *reinterpret_cast<uint4 *>(at + mg * kWgMn + (tid >> 3) * kWgK + (tid & 7) * 16) =
                            *reinterpret_cast<const uint4 *>(halo + h * 32 + (mg & 1) * 16);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&full[q])) : "memory");
            }
        }
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
        attr = true;
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
        attr = true;
    }
    size_t smem = (size_t)kHalo * 32 + (size_t)(w.cout / 8) * kWgMn + 2 * (size_t)kWgATile;
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
