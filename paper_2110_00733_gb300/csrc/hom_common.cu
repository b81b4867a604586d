// hom_common.cu -- MINRES scalar recurrences (FP64, one CTA), FP64 helpers of
// the refinement and post-processing, and input conversion.
#include <math.h>

#include <mutex>
#include <vector>

#include "hom_internal.h"

namespace hom {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = (lane < nw) ? red[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

__device__ __forceinline__ int pweight(int k3, int n3) { return (k3 == 0 || 2 * k3 == n3) ? 1 : 2; }

// deterministic reduction of the partials by one CTA (fixed order)
__device__ double reduce_partials(const double *partials, int np) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += partials[i];
    return block_sum(s);
}

__global__ void k_reduce_to(const double *partials, int np, double *out) {
    const double s = reduce_partials(partials, np);
    if (threadIdx.x == 0) *out = s;
}

// MINRES set-up from ||b||^2: beta_1, phibar_0 = beta_1, c_0 = -1, s_0 = 0,
// delta-bar_1 = 0, epsilon_1 = 0 (Paige-Saunders).  The Lanczos vectors are
// kept unnormalised, u_k = beta_k v_k, so u_1 = b and beta_0 = 0.
__global__ void k_scalar_start(MinresState *st, const double *partials, int np, double tol, int max_it,
                               int max_bodies) {
    const double b2 = reduce_partials(partials, np);
    if (threadIdx.x != 0) return;
    const double beta1 = sqrt(b2 > 0 ? b2 : 0.0);
    st->beta1 = beta1;
    st->beta = beta1;
    st->beta_prev = 0.0;   // no v_0 term in the first Lanczos step
    st->alpha = 0.0;
    st->c = -1.0;
    st->s = 0.0;
    st->dbar = 0.0;
    st->eps = 0.0;
    st->phibar = beta1;
    st->tol = tol;
    st->u_delta = st->u_eps = st->u_tau = st->u_tau1 = st->u_tau2 = 0.0;
    st->u_inv_gamma = st->u_inv_beta = 0.0;
    st->est = 1.0;
    st->k = 0;
    st->max_it = max_it;
    st->bodies = 0;
    st->max_bodies = max_bodies;
    st->done = (beta1 == 0.0 || max_it <= 0) ? 1 : 0;
    st->done_update = st->done;
    st->status = 0;
    if (!isfinite(beta1)) { st->status = -5; st->done = 1; st->done_update = 1; }
}

// alpha_k = <v_k, A v_k> = <u_k, A u_k> / beta_k^2; the partials sum to
// <u_k, A u_k> / scale (scale = V for the strain-energy sums of the n3 pass)
__global__ void k_scalar_alpha(MinresState *st, const double *partials, int np, double scale) {
    pdl_release();
    pdl_wait();                    // the n3 pass's partials (programmatic launch in the MINRES graph)
    st += blockIdx.x;              // load case of a stacked batch (one CTA each)
    partials += (size_t)blockIdx.x * np;
    if (st->done) return;
    const double a = reduce_partials(partials, np);
    if (threadIdx.x == 0) alpha_step(st, a, scale);
}

// MINRES step k: apply the previous Givens rotation to the new column of the
// Lanczos tridiagonal, form the next rotation, and the coefficients of the
// w_k / x_k update (applied by the next step's kernel, or by the flush after
// the loop); stop when phibar_k / beta_1 <= tol, beta_{k+1} = 0, or k reaches
// max_it.
__global__ void k_scalar_givens(MinresState *st, const double *partials, int np) {
    st += blockIdx.x;              // load case of a stacked batch (one CTA each)
    partials += (size_t)blockIdx.x * np;
    if (st->done) return;
    const double bn2 = reduce_partials(partials, np);
    if (threadIdx.x == 0) givens_step(st, bn2);
}

// Condition of the device-side MINRES loop: one more body while not done
// and below the cap (the cap ends the loop even if done were never set).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, MinresState *st, int nb) {
    if (threadIdx.x != 0) return;
    st->bodies += 1;   // counted on the first case's state
    int active = 0;
    for (int c = 0; c < nb; ++c) active |= !st[c].done;
    cudaGraphSetConditional(h, (active && st->bodies < st->max_bodies) ? 1u : 0u);
}

// PCG (MoDBFFT, section 2.2): rho_0 = <r0, M r0>, ||r0||^2 from the two
// halves of the partials; p_0 = z_0 is copied by the caller.
__global__ void k_scalar_cg_start(CgState *st, const double *partials, int np, double tol, int max_it) {
    const double rz = reduce_partials(partials, np);
    const double rr = reduce_partials(partials + np, np);
    if (threadIdx.x != 0) return;
    st->rho = rz;
    st->rr0 = rr;
    st->rr = rr;
    st->a = st->b = 0.0;
    st->tol = tol;
    st->est = 1.0;
    st->k = 0;
    st->max_it = max_it;
    st->status = isfinite(rz) && isfinite(rr) ? 0 : -5;
    st->done = (rr == 0.0 || max_it <= 0 || st->status) ? 1 : 0;
    st->done_update = st->done;
}

// step length a = rho / <p, A p>
__global__ void k_scalar_cg_alpha(CgState *st, const double *partials, int np) {
    if (st->done) return;
    const double pq = reduce_partials(partials, np);
    if (threadIdx.x != 0) return;
    const double a = st->rho / pq;
    if (!isfinite(a)) { st->status = -5; st->done = 1; return; }
    st->a = a;
}

// after x, r, z: rho' = <r, z>, b = rho'/rho; stop at ||r||/||r0|| <= tol
__global__ void k_scalar_cg_beta(CgState *st, const double *partials, int np) {
    if (st->done) return;
    const double rz = reduce_partials(partials, np);
    const double rr = reduce_partials(partials + np, np);
    if (threadIdx.x != 0) return;
    st->k += 1;
    st->rr = rr;
    st->est = sqrt(rr / st->rr0);
    if (!isfinite(rz) || !isfinite(rr)) { st->status = -5; st->done = 1; return; }
    st->b = rz / st->rho;
    st->rho = rz;
    if (st->est <= st->tol) st->done = 1;
    else if (st->k >= st->max_it) { st->status = 1; st->done = 1; }
}

// r = b - ax with ax from an FP32 operator (the residual that starts an FP32
// sweep from a warm start)
__global__ void __launch_bounds__(kEwThreads) k_spec_residual_mixed(int n, int h, int n3, int nc, const double2 *b,
                                                                    const float2 *ax, double2 *r, double *partials) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double2 bb = b[i];
        const float2 aa = ax[i];
        const double2 d = make_double2(bb.x - (double)aa.x, bb.y - (double)aa.y);
        r[i] = d;
        acc += pweight((i / nc) % h, n3) * (d.x * d.x + d.y * d.y);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kEwThreads) k_spec_residual64(int n, int h, int n3, int nc, const double2 *b,
                                                                const double2 *ax, double2 *r, double *partials) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double2 bb = b[i], aa = ax[i];
        const double2 d = make_double2(bb.x - aa.x, bb.y - aa.y);
        r[i] = d;
        acc += pweight((i / nc) % h, n3) * (d.x * d.x + d.y * d.y);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_spec_d2f(long long n, const double2 *in, float2 *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

__global__ void k_spec_f2d_acc(long long n, const float2 *in, double2 *out, double a) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 o = out[i];
        out[i] = make_double2(o.x + a * (double)in[i].x, o.y + a * (double)in[i].y);
    }
}

// <phi C_m : (E_bar + x)> per Mandel component: partials[c * gridDim.x + block]
__global__ void __launch_bounds__(kEwThreads) k_mean_stress64(long long V, const double *x, const double *phi,
                                                              double lam, double mu2, Mac6 mac, double *partials) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        double e[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] = mac.v[c] + x[c * V + i];
        const double ph = phi[i];
        const double tr = lam * (e[0] + e[1] + e[2]);
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += ph * ((c < 3 ? tr : 0.0) + mu2 * e[c]);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const double s = block_sum(acc[c]);
        if (threadIdx.x == 0) partials[c * gridDim.x + blockIdx.x] = s;
    }
}

// total strain and stress in tensor components (shear / sqrt2), stress x Escale
template <typename Ro>
__global__ void k_fields64(long long V, const double *x, const double *phi, double lam, double mu2, double Escale,
                           Mac6 mac, Ro *strain, Ro *stress) {
    const double r2 = 0.70710678118654752440;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        double e[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] = mac.v[c] + x[c * V + i];
        if (strain) {
#pragma unroll
            for (int c = 0; c < 6; ++c) strain[c * V + i] = (Ro)((c < 3) ? e[c] : e[c] * r2);
        }
        if (stress) {
            const double ph = phi[i];
            const double tr = lam * (e[0] + e[1] + e[2]);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const double s = Escale * ph * ((c < 3 ? tr : 0.0) + mu2 * e[c]);
                stress[c * V + i] = (Ro)((c < 3) ? s : s * r2);
            }
        }
    }
}

__global__ void k_f2d(long long n, const float *in, double *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}
__global__ void k_d2f(long long n, const double *in, float *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
__global__ void k_mandel_scale64(long long V, double *f, double s) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * V; i += (long long)gridDim.x * blockDim.x)
        f[3 * V + i] *= s;
}
template <typename R>
__global__ void k_phi_convert(long long V, const void *in, int kind, R *out, int *bad) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        double v;
        if (kind == 0) v = ((const unsigned char *)in)[i] ? 1.0 : 0.0;
        else if (kind == 1) v = (double)((const float *)in)[i];
        else v = ((const double *)in)[i];
        if (!(v >= 0.0 && v <= 1.0)) { atomicExch(bad, 1); v = 0.0; }
        out[i] = (R)v;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Tensor maps of the TMA passes (host).  The encoder is the driver's
// cuTensorMapEncodeTiled, reached through the runtime's entry-point query so
// the library does not link libcuda directly.
// ---------------------------------------------------------------------------
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}
struct TmaEntry {
    const void *ptr;
    int kind;
    CUtensorMap map;
};
struct TmaCache {
    std::vector<TmaEntry *> entries;
};
}  // namespace

bool tma_available() { return encoder() != nullptr; }

void *tma_cache_new() { return new TmaCache(); }

void tma_cache_free(void *c) {
    TmaCache *tc = static_cast<TmaCache *>(c);
    if (!tc) return;
    for (TmaEntry *e : tc->entries) delete e;
    delete tc;
}

// Half spectrum n1 x n2 x h x 6 of 8-byte units (elem_units per complex).
//  TMA_X2: 3-D (6h, n2, n1), box (tile2, n2, 1): one tile2-wide run of
//          columns over all k2 of one k1 plane.
//  TMA_X1: 2-D (6 n2 h, n1), box (6 tile1, n1): tile1 (k2,k3) columns with
//          their 6 components over all k1.
const CUtensorMap *tma_map(const Geometry &g, const void *ptr, int kind, int units) {
    TmaCache *tc = static_cast<TmaCache *>(g.tma_cache);
    for (TmaEntry *e : tc->entries)
        if (e->ptr == ptr && e->kind == kind) return &e->map;
    EncodeTiledFn fn = encoder();
    if (!fn) return nullptr;
    TmaEntry *e = new TmaEntry();
    e->ptr = ptr;
    e->kind = kind;
    const cuuint64_t u = (cuuint64_t)units;
    const cuuint64_t h6 = (cuuint64_t)g.nc * g.h * u;   // components x h, in 8-byte units
    CUresult r;
    if (kind == TMA_X2) {
        cuuint64_t dims[3] = {h6, (cuuint64_t)g.n2, (cuuint64_t)g.n1 * g.nb};
        cuuint64_t strides[2] = {h6 * 8, h6 * 8 * g.n2};
        // box dimensions hold at most 256 elements: longer columns move in
        // boxes of 256 rows (the kernels issue one copy per box)
        cuuint32_t box[3] = {(cuuint32_t)(g.tile2 * units), (cuuint32_t)(g.n2 < 256 ? g.n2 : 256), 1};
        cuuint32_t es[3] = {1, 1, 1};
        r = fn(&e->map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void *>(ptr), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        cuuint64_t dims[2] = {h6 * g.n2, (cuuint64_t)g.n1 * g.nb};
        cuuint64_t strides[1] = {h6 * g.n2 * 8};
        cuuint32_t box[2] = {(cuuint32_t)(g.nc * g.tile1 * units), (cuuint32_t)(g.n1 < 256 ? g.n1 : 256)};
        cuuint32_t es[2] = {1, 1};
        r = fn(&e->map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(ptr), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) {
        delete e;
        return nullptr;
    }
    tc->entries.push_back(e);
    return &e->map;
}

int ew_blocks(long long n) {
    long long b = (n + kEwThreads - 1) / kEwThreads;
    return (int)(b < kEwBlocks ? (b > 0 ? b : 1) : kEwBlocks);
}

void spec_residual64(const Geometry &g, cudaStream_t st, const double2 *b, const double2 *ax, double2 *r,
                     double *partials, int nc) {
    const int n = (int)(nc * g.S);
    k_spec_residual64<<<ew_blocks(n), kEwThreads, 0, st>>>(n, g.h, g.n3, nc, b, ax, r, partials);
}
void spec_residual_mixed(const Geometry &g, cudaStream_t st, const double2 *b, const float2 *ax, double2 *r,
                         double *partials) {
    const int n = (int)(6 * g.S);
    k_spec_residual_mixed<<<ew_blocks(n), kEwThreads, 0, st>>>(n, g.h, g.n3, 6, b, ax, r, partials);
}
void spec_d2f(long long n, cudaStream_t st, const double2 *in, float2 *out) {
    k_spec_d2f<<<ew_blocks(n), kEwThreads, 0, st>>>(n, in, out);
}
void spec_f2d_acc(long long n, cudaStream_t st, const float2 *in, double2 *out, double a) {
    k_spec_f2d_acc<<<ew_blocks(n), kEwThreads, 0, st>>>(n, in, out, a);
}
void mean_stress64(long long V, cudaStream_t st, const double *x, const double *phi, double lam, double mu,
                   const double *macro, double *partials) {
    Mac6 m{};
    for (int c = 0; c < 6; ++c) m.v[c] = macro[c];
    k_mean_stress64<<<ew_blocks(V), kEwThreads, 0, st>>>(V, x, phi, lam, 2.0 * mu, m, partials);
}
template <typename Ro>
void fields_from64(long long V, cudaStream_t st, const double *x, const double *phi, double lam, double mu,
                   double Escale, const double *macro, Ro *strain, Ro *stress) {
    Mac6 m{};
    for (int c = 0; c < 6; ++c) m.v[c] = macro[c];
    k_fields64<Ro><<<ew_blocks(V), kEwThreads, 0, st>>>(V, x, phi, lam, 2.0 * mu, Escale, m, strain, stress);
}
template void fields_from64<float>(long long, cudaStream_t, const double *, const double *, double, double, double,
                                   const double *, float *, float *);
template void fields_from64<double>(long long, cudaStream_t, const double *, const double *, double, double, double,
                                    const double *, double *, double *);
void real_convert_f2d(long long n, cudaStream_t st, const float *in, double *out) {
    k_f2d<<<ew_blocks(n), kEwThreads, 0, st>>>(n, in, out);
}
void real_convert_d2f(long long n, cudaStream_t st, const double *in, float *out) {
    k_d2f<<<ew_blocks(n), kEwThreads, 0, st>>>(n, in, out);
}
void mandel_scale64(long long V, cudaStream_t st, double *f, double s) {
    k_mandel_scale64<<<ew_blocks(3 * V), kEwThreads, 0, st>>>(V, f, s);
}
template <typename R>
void phi_convert(long long V, cudaStream_t st, const void *in, int kind, R *out, int *bad) {
    k_phi_convert<R><<<ew_blocks(V), kEwThreads, 0, st>>>(V, in, kind, out, bad);
}
template void phi_convert<float>(long long, cudaStream_t, const void *, int, float *, int *);
template void phi_convert<double>(long long, cudaStream_t, const void *, int, double *, int *);

void scalar_start(cudaStream_t st, MinresState *s, const double *partials, int np, double tol, int max_it,
                  int max_bodies) {
    k_scalar_start<<<1, 1024, 0, st>>>(s, partials, np, tol, max_it, max_bodies);
}
void loop_cond(cudaStream_t st, cudaGraphConditionalHandle h, MinresState *s, int nb) {
    k_loop_cond<<<1, 32, 0, st>>>(h, s, nb);
}
void scalar_alpha(cudaStream_t st, MinresState *s, const double *partials, int np, double scale, int nb, int pdl) {
    launch_k(pdl, k_scalar_alpha, nb, 1024, 0, st, s, partials, np, scale);
}
void scalar_givens(cudaStream_t st, MinresState *s, const double *partials, int np, int nb) {
    k_scalar_givens<<<nb, 1024, 0, st>>>(s, partials, np);
}
void scalar_cg_start(cudaStream_t st, CgState *s, const double *partials, int np, double tol, int max_it) {
    k_scalar_cg_start<<<1, 1024, 0, st>>>(s, partials, np, tol, max_it);
}
void scalar_cg_alpha(cudaStream_t st, CgState *s, const double *partials, int np) {
    k_scalar_cg_alpha<<<1, 1024, 0, st>>>(s, partials, np);
}
void scalar_cg_beta(cudaStream_t st, CgState *s, const double *partials, int np) {
    k_scalar_cg_beta<<<1, 1024, 0, st>>>(s, partials, np);
}
void reduce_to(cudaStream_t st, const double *partials, int np, double *out) {
    k_reduce_to<<<1, 1024, 0, st>>>(partials, np, out);
}

}  // namespace hom
