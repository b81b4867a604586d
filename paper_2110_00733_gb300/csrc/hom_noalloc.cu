// hom_noalloc.cu -- hom_apply_noalloc: A(eps) for small cells without any
// device allocation.
//
// Who needs this: callers that must not call cudaMalloc.  An application whose
// device memory is owned by its own pool (a framework's caching allocator, a
// real-time or embedded system that reserves all of its memory at start-up
// and forbids allocations afterwards) cannot let a library allocate behind
// its back; and in a latency-critical loop cudaMalloc, which may synchronise
// the device, is not acceptable either.  hom_create allocates its workspace,
// so those callers cannot use it.
//
// Here the work spectrum and the FFT / frequency tables live in file-scope
// __device__ arrays of fixed size.  Every GPU that loads the library holds
// them (about 1.6 MB) until the process exits.  The host code obtains their
// device addresses with cudaGetSymbolAddress once per device, on the first
// call made with that device current; that first call should therefore come
// before any stream capture.  All calls share the arrays, so calls whose
// device work overlaps (for example on two streams) race with each other.
// Nothing needs to start at zero: each call rewrites the tables and every
// spectrum entry it reads.
//
// The call only enqueues its kernels on the caller's stream and returns; the
// caller synchronises that stream (or orders later work after it) before
// reading `out`.
#include <math.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/hom.h"
#include "hom_internal.h"

using namespace hom;

namespace {

constexpr int kMaxN = 64;          // largest grid size along any axis
constexpr int kMaxV = 32768;       // largest voxel count (for example 32^3)
constexpr int kMaxDevices = 64;

// work half spectrum: n1 n2 (n3/2+1) <= V for n3 >= 2, times 6 components
static __device__ __align__(256) float2 g_scratch_spec[6 * kMaxV];
// per axis: twiddles exp(-2 pi i t/N), difference symbol D, averaging factor M
static __device__ __align__(256) float2 g_scratch_tab[3][3][kMaxN];

struct DevicePtrs {
    float2 *spec = nullptr;
    float2 *tab = nullptr;
    bool ready = false;
};
DevicePtrs g_dev[kMaxDevices];
std::mutex g_mu;

// Frequency tables on the device, FP64 with sincospi, stored in FP32:
// tw[t] = exp(-2 pi i t/N); D, M of the continuous (eq. freq) or rotated
// (eq. freqrot) scheme, as in the context-based path.
__global__ void k_noalloc_tables(int n1, int n2, int n3, int deriv, float2 *tab) {
    const int ns[3] = {n1, n2, n3};
    for (int p = 0; p < 3; ++p) {
        const int N = ns[p];
        float2 *tw = tab + (p * 3 + 0) * kMaxN;
        float2 *D = tab + (p * 3 + 1) * kMaxN;
        float2 *M = tab + (p * 3 + 2) * kMaxN;
        for (int t = threadIdx.x; t < N; t += blockDim.x) {
            double s, c;
            sincospi(2.0 * (double)t / (double)N, &s, &c);
            tw[t] = make_float2((float)c, (float)-s);
            const int m = (2 * t < N) ? t : t - N;
            double sq, cq;
            sincospi(2.0 * (double)m / (double)N, &sq, &cq);
            if (deriv == HOM_DERIV_CONTINUOUS) {
                D[t] = make_float2(0.f, (float)(2.0 * 3.14159265358979323846 * m));   // i q N with q = 2 pi m / N
                M[t] = make_float2(1.f, 0.f);
            } else {
                D[t] = make_float2((float)(N * (cq - 1.0)), (float)(N * sq));
                M[t] = make_float2((float)(0.5 * (1.0 + cq)), (float)(0.5 * sq));
            }
        }
    }
}

bool radices(int n, AxisPlan &p) {
    int a = 0, m = n;
    while (m % 2 == 0) { m /= 2; ++a; }
    int b = 0;
    while (m % 3 == 0) { m /= 3; ++b; }
    int c = 0;
    while (m % 5 == 0) { m /= 5; ++c; }
    if (m != 1) return false;
    int ns = 0;
    if (a > 0) {
        int st2 = (a + 3) / 4;
        int base = a / st2, extra = a % st2;
        for (int i = 0; i < st2; ++i) p.radix[ns++] = 1 << (base + (i < extra ? 1 : 0));
    }
    for (int i = 0; i < b; ++i) p.radix[ns++] = 3;
    for (int i = 0; i < c; ++i) p.radix[ns++] = 5;
    if (ns > kMaxStages) return false;
    p.nstages = ns;
    p.n = n;
    return true;
}

int setup_device(int dev, DevicePtrs **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= kMaxDevices) {
        hom_set_error("hom_apply_noalloc: device ordinal beyond the 64 devices this entry point serves");
        return HOM_EINVAL;
    }
    DevicePtrs &d = g_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch_spec);
        if (e == cudaSuccess) {
            d.spec = static_cast<float2 *>(p);
            p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch_tab);
        }
        if (e != cudaSuccess) {
            hom_set_error((std::string("hom_apply_noalloc: device set-up (cudaGetSymbolAddress) failed: ") +
                           cudaGetErrorString(e)).c_str());
            return HOM_ECUDA;
        }
        d.tab = static_cast<float2 *>(p);
        Geometry g{};
        Launch<float>::table_init(g);   // shared-memory limits of the pass kernels
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            hom_set_error((std::string("hom_apply_noalloc: device set-up failed: ") + cudaGetErrorString(e)).c_str());
            return HOM_ECUDA;
        }
        d.ready = true;
    }
    *out = &d;
    return HOM_OK;
}

}  // namespace

int hom_apply_noalloc(const int grid[3], const float *phi, double E, double nu, int derivative, const float *eps,
                      float *out, void *stream) {
    if (!grid || !phi || !eps || !out) {
        hom_set_error("hom_apply_noalloc: null argument");
        return HOM_EINVAL;
    }
    if (!(E > 0.0) || !std::isfinite(E) || !(nu > -1.0 && nu < 0.5) ||
        (derivative != HOM_DERIV_CONTINUOUS && derivative != HOM_DERIV_ROTATED)) {
        hom_set_error("hom_apply_noalloc: need E > 0, -1 < nu < 0.5 and a valid derivative");
        return HOM_EINVAL;
    }
    Geometry g{};
    long long V = 1;
    for (int p = 0; p < 3; ++p) {
        if (grid[p] < 2 || grid[p] > kMaxN || !radices(grid[p], g.ax[p])) {
            hom_set_error("hom_apply_noalloc: each grid size must be in [2, 64] and of the form 2^a 3^b 5^c");
            return HOM_EUNSUPPORTED_GRID;
        }
        V *= grid[p];
    }
    if (V > kMaxV) {
        hom_set_error("hom_apply_noalloc: n1 n2 n3 must not exceed 32768 voxels");
        return HOM_EUNSUPPORTED_GRID;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        hom_set_error("hom_apply_noalloc: no CUDA device");
        return HOM_ECUDA;
    }
    // an error left pending by the caller's own earlier work is reported as
    // such (and left pending), so that it is neither taken for this call's
    // nor cleared
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        hom_set_error((std::string("hom_apply_noalloc: a CUDA error was already pending before the call: ") +
                       cudaGetErrorString(pending)).c_str());
        return HOM_ECUDA;
    }
    DevicePtrs *d = nullptr;
    int rc = setup_device(dev, &d);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    g.n1 = grid[0];
    g.n2 = grid[1];
    g.n3 = grid[2];
    g.h = g.n3 / 2 + 1;
    g.V = V;
    g.S = (long long)g.n1 * g.n2 * g.h;
    for (int p = 0; p < 3; ++p) {
        g.fast[p] = is_fast_length(grid[p]) ? grid[p] : 0;
        g.ax[p].tw = d->tab + (p * 3 + 0) * kMaxN;
        g.D[p] = d->tab + (p * 3 + 1) * kMaxN;
        g.M[p] = d->tab + (p * 3 + 2) * kMaxN;
    }
    // launch shapes, the same rules as a context's FP32 engine (plain loads)
    const size_t cs = sizeof(float2);
    auto round32 = [](int v) { return (v + 31) / 32 * 32; };
    auto clampt = [](int v) { return v < 128 ? 128 : (v > 512 ? 512 : v); };
    int rows, t2, t1;
    if (g.fast[2]) {
        rows = 48 / (3 * (g.n3 / fast_elems_n3(g.n3)));
        rows = rows < 1 ? 1 : (rows > 64 ? 64 : rows);
    } else {
        rows = 16;
        while (rows > 1 && 2ull * g.n3 * 3 * rows * cs > 48 * 1024) rows >>= 1;
    }
    if (g.fast[1]) t2 = g.n2 >= 128 ? 16 : 32;
    else {
        t2 = 32;
        while (t2 > 1 && 2ull * g.n2 * t2 * cs > 64 * 1024) t2 >>= 1;
    }
    if (g.fast[0]) {
        t1 = 192 * fast_elems(g.n1) / (6 * g.n1);
        t1 = t1 < 1 ? 1 : (t1 > 16 ? 16 : t1);
    } else {
        t1 = 16;
        while (t1 > 1 && 2ull * g.n1 * 6 * t1 * cs > 96 * 1024) t1 >>= 1;
    }
    g.rows3 = rows;
    g.tile2 = t2;
    g.tile1 = t1;
    const int es3 = (3 * rows) | 1;
    if (g.fast[2]) {
        g.threads3 = 3 * rows * (g.n3 / fast_elems_n3(g.n3));
        g.smem3 = ((size_t)es3 * g.n3 + g.n3 / 16 + 1) * cs;
    } else {
        g.threads3 = clampt(round32(3 * rows * g.n3 / 16));
        g.smem3 = 2ull * es3 * g.n3 * cs;
    }
    if (g.fast[1]) {
        g.threads2 = t2 * (g.n2 / fast_elems(g.n2));
        g.smem2 = (size_t)t2 * g.n2 * cs;
    } else {
        g.threads2 = clampt(round32(t2 * g.n2 / 16));
        g.smem2 = 2ull * t2 * g.n2 * cs;
    }
    const int L1 = 6 * t1;
    if (g.fast[0]) {
        g.threads1 = L1 * (g.n1 / fast_elems(g.n1));
        g.smem1 = (size_t)L1 * g.n1 * cs;
    } else {
        const int m = 256 / L1;
        g.threads1 = L1 * (m < 1 ? 1 : m);
        g.smem1 = 2ull * L1 * g.n1 * cs;
    }
    g.nc = 6;
    g.tma = 0;
    g.tma_cache = nullptr;
    g.err = nullptr;
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));   // lambda / E
    const double mu = 1.0 / (2.0 * (1.0 + nu));                // mu / E
    float2 *spec = d->spec;
    k_noalloc_tables<<<1, 64, 0, st>>>(g.n1, g.n2, g.n3, derivative, d->tab);
    // A(eps) = F^-1 G F (phi C_m : eps), eq. (linearOp), C_m in units of E
    Launch<float>::x3(g, st, X3_IN_REAL, eps, X3_MID_MATERIAL, lam, mu, nullptr, 1.0, X3_OUT_SPEC, spec, phi, nullptr);
    Launch<float>::x2(g, st, 0, spec, nullptr);
    Launch<float>::x1(g, st, X1_FWD | X1_GAMMA_OUT, spec, spec, nullptr, nullptr, nullptr);
    Launch<float>::x1(g, st, 0, spec, spec, nullptr, nullptr, nullptr);
    Launch<float>::x2(g, st, 1, spec, nullptr);
    Launch<float>::x3(g, st, X3_IN_SPEC, spec, X3_MID_NONE, lam, mu, nullptr, 1.0, X3_OUT_REAL, out, phi, nullptr);
    // launch errors only: the call does not wait for its kernels
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        hom_set_error(cudaGetErrorString(e));
        return HOM_ECUDA;
    }
    return HOM_OK;
}
