// hom_api.cu -- the C ABI of include/hom.h: contexts, FFT plans, the
// operator of eq. (linearOp) in its spectral form, MINRES (section 2.1) as a
// captured CUDA graph, the FP64 true residual of eq. (galres) with iterative
// refinement for FP32 fields, and the volume-averaged stress of section 4.3.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/hom.h"
#include "hom_internal.h"
#include "hom_cg.h"
#include "hom_pfs.h"
#include "hom_j2.h"

using namespace hom;

namespace {

thread_local std::string g_create_error;

// smallest relative residual reduction one FP32-field MINRES sweep is asked for
constexpr double kFp32SweepFloor = 1e-6;
// ... except the first sweep of a zero start (its right-hand side is b
// itself), which may aim at 5e-7
constexpr double kFp32FirstSweepFloor = 5e-7;
// a sweep aims below the tolerance by this factor: the FP64 true residual
// after an FP32 sweep differs a little from the recurrence's estimate, and
// landing just above tol costs a restarted sweep
constexpr double kSweepTarget = 0.5;
// PCG on A^alpha (not symmetric where chi_v is non-zero) in FP32 drifts away
// from the FP64 residual sooner than MINRES: shorter sweeps, restarted from
// the FP64 true residual, keep it converging
constexpr double kFp32CgSweepFloor = 1e-3;
// Under stress control (hom_solve_mixed) the solution carries the mean strain
// of a compliant lattice, large against the right-hand side, and an FP32
// MINRES sweep on a cell with void loses track of its true residual below
// about 1e-5 (its estimate keeps falling while the FP64 residual stalls):
// the first FP32 sweep asks for a reduction of 1e-4, later sweeps, whose
// right-hand side is the residual FP32 left behind, for 1e-2, and the FP64
// true residual restarts each.
constexpr double kFp32MixedSweepFloor = 1e-4;
constexpr double kFp32MixedLaterSweepFloor = 1e-2;
// a warm start whose FP32-estimated residual is below this gets the FP64 one
constexpr double kWarmFp64Below = 1e-3;
// relative size of ||b|| / ||C : E_bar|| below which the right-hand side is
// FFT round-off and is taken as zero (the paper is silent on this case)
constexpr double kRhsZero = 1e-12;

struct Status {
    int code = HOM_OK;
    std::string msg;
};

// Per-precision engine: tables, phase map and spectrum workspace of one cell.
template <typename R> struct Engine {
    Geometry g{};
    Geometry gm{};             // MoDBFFT chain: 10 components per frequency
    R *phi = nullptr;
    cpx<R> *spec = nullptr;
    cpx<R> *spec10 = nullptr;  // MoDBFFT work spectrum
    void *tw[3] = {nullptr, nullptr, nullptr};
    void *D[3] = {nullptr, nullptr, nullptr};
    void *M[3] = {nullptr, nullptr, nullptr};
};

// History and Newton work fields of an elastoplastic cell (hom_j2_*), FP64
// real fields 6 x V Mandel, component-major.
struct J2State {
    bool active = false;
    J2Material mat{};          // units of E (E = 1)
    double *eps = nullptr;     // total strain at the current iterate
    double *eps_t = nullptr;   // total strain at t
    double *etry = nullptr;    // line-search trial
    double *epsp = nullptr;    // plastic strain at t
    double *alpha = nullptr;   // hardening variable at t (V)
    double *sig = nullptr;     // stress; inverse-FFT scratch inside the operator
    double *de = nullptr;      // Newton step (real); tangent output inside the operator
    double *Ct = nullptr;      // consistent tangent at the current iterate (36 V; FP64 fields)
    float *Ct32 = nullptr;     // the same in FP32 (FP32 fields: the MINRES operator is FP32)
    float *sig32 = nullptr, *de32 = nullptr;   // FP32 operator scratch (6 V each)
    double2 *x64 = nullptr;    // FP32 fields: the Newton step accumulated over refinement sweeps (spectral)
    double *partials = nullptr;
    double *h_partials = nullptr;   // pinned
    double Ebar[6] = {0, 0, 0, 0, 0, 0};   // macro strain of the last increment (Mandel)
    bool moved = false;        // the running increment has changed eps (eps_t holds t)
};

}  // namespace

struct hom_ctx {
    int n[3];
    long long V = 0, S = 0;
    int prec = HOM_PREC_FP32_FIELDS;
    int deriv = HOM_DERIV_ROTATED;
    double E = 1.0, nu = 0.3, lam = 0.0, mu = 0.0;   // lam, mu in units of E
    double phi2_sum = 0.0;                            // sum phi^2 (zero-rhs test)
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device_ptrs = 0;
    int refine = 3;
    double sweep_floor = kFp32SweepFloor;
    int shape[3] = {0, 0, 0};   // launch-shape overrides (rows3, tile2, tile1)
    int staging = 0;            // 0: TMA-staged passes where supported, 1: plain loads
    int solver = HOM_SOLVER_GALERKIN_MINRES;
    double alpha = 1e-4;        // MoDBFFT penalty / E
    double phibar = 0.0;        // mean of phi (MoDBFFT preconditioner, eq. avstiff)
    CgState *d_cg = nullptr;
    CgState *h_cg = nullptr;    // pinned
    cudaGraphExec_t cg_graph = nullptr;
    long long cg_graph_kernels = 0;
    int *d_err = nullptr;       // set by a pass whose bounded wait gave up
    Engine<float> e32;
    Engine<double> e64;
    // MINRES workspace in the solve precision (half spectra, float2 or double2)
    void *vbuf[3] = {nullptr, nullptr, nullptr};
    void *wbuf[2] = {nullptr, nullptr};
    void *xs = nullptr;     // MINRES iterate of the current sweep
    long long krylov_reals = 0;   // reals allocated per Krylov buffer (vbuf, wbuf, xs)
    void *rhs = nullptr;    // MINRES right-hand side of the current sweep
    double2 *b64 = nullptr, *r64 = nullptr;   // FP64 right-hand side and residual spectra
    double2 *phihat = nullptr;                // FP64 DFT of phi (half spectrum, one component)
    std::vector<double2 *> x64;     // per-case solutions (spectral, FP64 master copy)
    std::vector<double> macros;     // per-case prescribed macro strains (Mandel; 0 on stress-controlled components)
    std::vector<double> eps_means;  // per-case mean strains (Mandel, including solved stress-controlled means)
    std::vector<double> sig_mean;   // per-case mean stress (tensor comps, units of E)
    int ncase = 0;
    double *partials = nullptr;
    int npartials = 0;
    MinresState *d_state = nullptr;
    MinresState *h_state = nullptr;  // pinned
    double *d_scalar = nullptr;
    double *h_scalar = nullptr;      // pinned
    double *tsum_part = nullptr;     // per-CTA stress sums of the FP64 n3 pass (6 x x3_grid)
    int *d_flag = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool graph_loops = false;        // graph is a device-side WHILE loop over the body
    bool host_loop = false;          // asked for the host-replayed body
    int pdl = 0;                     // programmatic launches inside the stacked MINRES graph
    bool tangent_op = false;         // operator of eq. (galnonlin) with the J2 tangent (FP64)
    bool graph_tangent = false;      // the captured graph applies the tangent operator
    J2State j2;
    // Elastic MINRES on a stacked batch of load cases (the solve path of
    // hom_solve): capacity in cases, the stacked geometry of the captured
    // graph and its TMA cache, work spectra and Krylov vectors of every case,
    // FP64 right-hand sides and residuals, one state per case, partials, graph.
    int bcap = 0;
    Geometry bg{};
    void *btma = nullptr;
    void *bspec = nullptr;                       // bcap x 6S, solve precision
    void *bv[3] = {nullptr, nullptr, nullptr};   // bcap x kvec each (n1-tile order): u_k in bv[k mod 3]
    void *bw[2] = {nullptr, nullptr};
    void *bx = nullptr;
    void *brhs = nullptr;                        // bcap x 6S: right-hand sides, then iterates
    double2 *bb64 = nullptr, *br64 = nullptr;    // bcap x 6S
    MinresState *d_bst = nullptr, *h_bst = nullptr;
    double *bpart = nullptr;
    int *bcnt = nullptr;                         // kFoldCounters counters of the folded scalar steps
    cudaGraphExec_t bgraph = nullptr;
    int bgraph_nb = 0;
    bool bgraph_loops = false;
    long long bgraph_kernels = 0;
    int graph_iters = 6;
    long long graph_kernels = 0;
    long long launches = 0;
    long long workspace = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string err;
};

static void batch_free(hom_ctx *ctx);
static void set_stress_mask(hom_ctx *ctx, int mask);

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// message for hom_last_error(NULL) from entry points that take no context
namespace hom {
void hom_set_error(const char *msg) { g_create_error = msg ? msg : ""; }
}  // namespace hom

static int fail(hom_ctx *c, int code, const std::string &m) {
    if (c) c->err = m;
    else g_create_error = m;
    return code;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? HOM_ENOMEM : HOM_ECUDA,   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));            \
        }                                                                               \
    } while (0)

static bool factor_radices(int n, AxisPlan &p) {
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

template <typename R> static size_t cpx_size() { return sizeof(R) * 2; }

// Launch shapes of the three passes for a spectrum with nc components per
// frequency (defaults; hom_options may override them -- autotuner hook).
//  fast engine: threads = lines * n / E, one buffer of lines * n values
//  generic engine: Stockham ping-pong, two buffers
template <typename R>
static int set_shapes(hom_ctx *ctx, Geometry &g, int nc) {
    const size_t cs = cpx_size<R>();
    const int np = nc / 2;   // component pairs of the n3 pass
    g.nc = nc;
    int rows, t2, t1;
    if (g.fast[2]) {
        rows = 48 / (np * (g.n3 / fast_elems_n3r<R>(g.n3)));
        rows = rows < 1 ? 1 : (rows > 64 ? 64 : rows);
        // the two-stage FP32 plans at 96 and 160, measured (6-component
        // spectra): 8 rows at 160 (0.123 against 0.136 ms at 160^3), 2 at 96
        // (0.027 against 0.029 ms at 96^3)
        if (fast_elems_n3r<R>(g.n3) != fast_elems(g.n3) && nc == 6) rows = g.n3 == 160 ? 8 : 2;
    } else {
        rows = 16;
        while (rows > 1 && 2ull * g.n3 * np * rows * cs > 48 * 1024) rows >>= 1;
    }
    if (g.fast[1]) {
        t2 = g.n2 >= 512 ? 8 : (g.n2 >= 128 ? 16 : 32);
    } else {
        t2 = 32;
        while (t2 > 1 && 2ull * g.n2 * t2 * cs > 64 * 1024) t2 >>= 1;
    }
    if (g.fast[0]) {
        t1 = 192 * fast_elems(g.n1) / (nc * g.n1);
        t1 = t1 < 1 ? 1 : (t1 > 16 ? 16 : t1);
    } else {
        t1 = 16;
        while (t1 > 1 && 2ull * g.n1 * nc * t1 * cs > 96 * 1024) t1 >>= 1;
    }
    if (nc == 6) {
        if (ctx->shape[0] > 0) rows = ctx->shape[0];
        if (ctx->shape[1] > 0) t2 = ctx->shape[1];
        if (ctx->shape[2] > 0) t1 = ctx->shape[2];
    }
    g.rows3 = rows;
    g.tile2 = t2;
    g.tile1 = t1;
    auto round32 = [](int v) { return (v + 31) / 32 * 32; };
    auto clampt = [](int v) { return v < 128 ? 128 : (v > 512 ? 512 : v); };
    const int es3 = (np * rows) | 1;   // element stride of the n3 tile (odd)
    if (g.fast[2]) {
        g.threads3 = np * rows * (g.n3 / fast_elems_n3r<R>(g.n3));
        g.smem3 = ((size_t)es3 * g.n3 + g.n3 / 16 + 1) * cs;   // + one pad slot per 16 elements
    } else {
        g.threads3 = clampt(round32(np * rows * g.n3 / 16));
        g.smem3 = 2ull * es3 * g.n3 * cs;
    }
    if (g.fast[1]) {
        g.threads2 = t2 * (g.n2 / fast_elems(g.n2));
        g.smem2 = (size_t)t2 * g.n2 * cs;
    } else {
        g.threads2 = clampt(round32(t2 * g.n2 / 16));
        g.smem2 = 2ull * t2 * g.n2 * cs;
    }
    const int L1 = nc * t1;
    if (g.fast[0]) {
        g.threads1 = L1 * (g.n1 / fast_elems(g.n1));
        g.smem1 = (size_t)L1 * g.n1 * cs;
    } else {
        const int m = 256 / L1;
        g.threads1 = L1 * (m < 1 ? 1 : m);
        g.smem1 = 2ull * L1 * g.n1 * cs;
    }
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if (g.smem3 + 1024 > (size_t)dev_smem || g.smem2 + 1024 > (size_t)dev_smem || g.smem1 + 1024 > (size_t)dev_smem)
        return fail(ctx, HOM_EINVAL, "launch shape needs more shared memory than the device has");
    if (g.threads1 > 512 || g.threads2 > 512 || g.threads3 > 512 || g.threads1 < 1 || g.threads2 < 1 || g.threads3 < 1)
        return fail(ctx, HOM_EINVAL, "launch shape needs more than 512 threads per CTA");
    if ((t2 & (t2 - 1)) != 0 || g.threads2 % t2 != 0) return fail(ctx, HOM_EINVAL, "tile2 must be a power of two");
    if (nc == 6 && g.threads1 > 384)
        return fail(ctx, HOM_EINVAL, "launch shape needs more than 384 threads per CTA in the fused n1 pass");
    g.kvec = (long long)((g.n2 * g.h + t1 - 1) / t1) * g.n1 * nc * t1;
    g.x3r = (sizeof(R) == 4 && nc == 6 && x3r_length(g.n3) && ctx->shape[0] == 0 &&
             x3r_smem(g.n3) + 1024 <= (size_t)dev_smem && (g.n1 * g.n2) % x3r_rows_per_warp(g.n3) == 0) ? 1 : 0;
    g.grid3r = g.x3r ? Launch<R>::x3r_grid(g) : 0;
    if (g.grid3r <= 0) g.x3r = 0;
    // persistent TMA-staged n2 / n1 passes: FP32, register-FFT lengths <= 256
    g.tma = 0;
    g.err = ctx->d_err;
    g.tma_cache = nullptr;
    if (sizeof(R) == 4 && ctx->staging == 0 && tma_available() && g.fast[0] >= 64 && g.fast[0] <= 512 &&
        g.fast[1] >= 64 && g.fast[1] <= 512 && g.tile2 % 2 == 0) {
        g.tma = 1;
        // n2 ring stages: 3 at n2 >= 256 (0.143 against 0.148 ms per pass at
        // 256^3; 0.280 against 0.36 ms on 256 x 512 x 256), 2 below (at 128^3
        // three were slower: 0.0185 against 0.0165 ms); HOM_X2_STAGES (2..4)
        // overrides
        {
            const char *e = getenv("HOM_X2_STAGES");
            const int v = e ? atoi(e) : (g.n2 >= 256 ? 3 : 2);
            g.x2_stages = v < 2 ? 2 : (v > kX2MaxStages ? kX2MaxStages : v);
        }
        g.smem2_tma = (size_t)g.x2_stages * g.n2 * g.tile2 * cs;
        // fused n1 pass: bulk L2 prefetch of each tile's u_k and u_{k-1}
        // blocks at the tile's start (0.625 against 0.647 ms at 256^3; the
        // two warp groups' reads of u_{k-1} then both hit L2); HOM_X1_L2PF=0
        // turns it off
        {
            const char *e = getenv("HOM_X1_L2PF");
            g.x1_l2pf = e ? atoi(e) : 1;
        }
        g.smem1_tma = 2ull * nc * g.tile1 * g.n1 * cs;
        g.smem1d_tma = 2 * g.smem1_tma;
        if (g.smem1d_tma + 1024 > (size_t)dev_smem || g.smem2_tma + 1024 > (size_t)dev_smem) g.tma = 0;
        if (g.tma && Launch<R>::tma_grids(g)) g.tma_cache = tma_cache_new();
        else g.tma = 0;
    }
    return HOM_OK;
}

template <typename R>
static int engine_init(hom_ctx *ctx, Engine<R> &E) {
    Geometry &g = E.g;
    g.n1 = ctx->n[0];
    g.n2 = ctx->n[1];
    g.n3 = ctx->n[2];
    g.h = g.n3 / 2 + 1;
    g.V = ctx->V;
    g.S = ctx->S;
    const size_t cs = cpx_size<R>();
    for (int p = 0; p < 3; ++p) g.fast[p] = is_fast_length(ctx->n[p]) ? ctx->n[p] : 0;
    const double PI = 3.14159265358979323846;
    for (int p = 0; p < 3; ++p) {
        const int N = ctx->n[p];
        if (!factor_radices(N, g.ax[p])) return fail(ctx, HOM_EUNSUPPORTED_GRID, "grid size not 2^a3^b5^c");
        std::vector<R> tw(2 * N), D(2 * N), M(2 * N);
        for (int t = 0; t < N; ++t) {
            const double ang = 2.0 * PI * (double)t / (double)N;
            tw[2 * t] = (R)std::cos(ang);
            tw[2 * t + 1] = (R)-std::sin(ang);
            const int m = (2 * t < N) ? t : t - N;        // signed frequency index
            const double q = 2.0 * PI * (double)m / (double)N;
            if (ctx->deriv == HOM_DERIV_CONTINUOUS) {      // xi_p = i q_p N_p, eq. (freq)
                D[2 * t] = 0;
                D[2 * t + 1] = (R)(q * N);
                M[2 * t] = 1;
                M[2 * t + 1] = 0;
            } else {   // rotated scheme, eq. (freqrot): N (e^{iq}-1) and (1+e^{iq})/2
                D[2 * t] = (R)(N * (std::cos(q) - 1.0));
                D[2 * t + 1] = (R)(N * std::sin(q));
                M[2 * t] = (R)(0.5 * (1.0 + std::cos(q)));
                M[2 * t + 1] = (R)(0.5 * std::sin(q));
            }
        }
        CU(cudaMalloc(&E.tw[p], cs * N));
        CU(cudaMalloc(&E.D[p], cs * N));
        CU(cudaMalloc(&E.M[p], cs * N));
        CU(cudaMemcpy(E.tw[p], tw.data(), cs * N, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(E.D[p], D.data(), cs * N, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(E.M[p], M.data(), cs * N, cudaMemcpyHostToDevice));
        g.ax[p].tw = E.tw[p];
        g.D[p] = E.D[p];
        g.M[p] = E.M[p];
        ctx->workspace += 3 * (long long)cs * N;
    }
    CU(cudaMalloc(&E.phi, sizeof(R) * ctx->V));
    CU(cudaMalloc(&E.spec, cs * 6 * ctx->S));
    ctx->workspace += sizeof(R) * ctx->V + cs * 6 * ctx->S;
    Launch<R>::table_init(g);
    int rc = set_shapes<R>(ctx, g, 6);
    if (rc) return rc;
    CU(cudaGetLastError());
    return HOM_OK;
}

template <typename R>
static void engine_free(Engine<R> &E) {
    tma_cache_free(E.g.tma_cache);
    E.g.tma_cache = nullptr;
    tma_cache_free(E.gm.tma_cache);
    E.gm.tma_cache = nullptr;
    cudaFree(E.spec10);
    for (int p = 0; p < 3; ++p) {
        cudaFree(E.tw[p]);
        cudaFree(E.D[p]);
        cudaFree(E.M[p]);
    }
    cudaFree(E.phi);
    cudaFree(E.spec);
}

// p = A^ v = G F C F^-1 G v (spectral vectors); optional <v, p> partials.
template <typename R>
static void op_spec(hom_ctx *ctx, Engine<R> &E, const cpx<R> *v, cpx<R> *p, bool dot, double *partials,
                    const MinresState *st, double *tsum = nullptr) {
    cudaStream_t s = ctx->stream;
    Launch<R>::x1(E.g, s, X1_GAMMA_IN, v, E.spec, nullptr, nullptr, st);
    Launch<R>::x2(E.g, s, 1, E.spec, st);
    if (ctx->tangent_op) {
        // A_i v = G F (C^{i-1}(x) : F^-1 G v), eq. (galnonlin): the point-wise
        // 6x6 tangent between an inverse and a forward n3 pass (applying it
        // inside the n3 pass was measured slower: 0.199 against 0.152 ms at
        // 128^3, the pass's small CTAs do not stream the 36-entry tangent)
        R *tin, *tout;
        if constexpr (std::is_same<R, double>::value) {
            tin = ctx->j2.sig; tout = ctx->j2.de;
        } else {
            tin = ctx->j2.sig32; tout = ctx->j2.de32;
        }
        Launch<R>::x3(E.g, s, X3_IN_SPEC, E.spec, X3_MID_NONE, ctx->lam, ctx->mu, nullptr, 1.0, X3_OUT_REAL, tin,
                      E.phi, st);
        // FP64 operator of FP32 fields (their true residual): the FP32 tangent in FP64 arithmetic
        if constexpr (std::is_same<R, double>::value) {
            if (ctx->j2.Ct) j2_tangent_apply<double, double>(ctx->V, ctx->j2.Ct, tin, tout, s);
            else j2_tangent_apply<float, double>(ctx->V, ctx->j2.Ct32, tin, tout, s);
        } else {
            j2_tangent_apply<float, float>(ctx->V, ctx->j2.Ct32, tin, tout, s);
        }
        Launch<R>::x3(E.g, s, X3_IN_REAL, tout, X3_MID_NONE, ctx->lam, ctx->mu, nullptr, 1.0, X3_OUT_SPEC, E.spec,
                      E.phi, st);
        ctx->launches += 2;
    } else {
        Launch<R>::x3(E.g, s, X3_IN_SPEC, E.spec, X3_MID_MATERIAL, ctx->lam, ctx->mu, nullptr, 1.0, X3_OUT_SPEC,
                      E.spec, E.phi, st, nullptr, Fold{}, tsum);
    }
    Launch<R>::x2(E.g, s, 0, E.spec, st);
    Launch<R>::x1(E.g, s, X1_FWD | X1_GAMMA_OUT | (dot ? X1_DOT : 0), E.spec, p, dot ? v : nullptr, partials, st);
    ctx->launches += 5;
}

// b^ = -G F (C : E_bar) (spectral), eq. (gallin) with sigma_bar = 0
template <typename R>
static void rhs_spec(hom_ctx *ctx, Engine<R> &E, const double *macro_mandel, cpx<R> *b) {
    cudaStream_t s = ctx->stream;
    Launch<R>::x3(E.g, s, X3_IN_MACRO, nullptr, X3_MID_MATERIAL, ctx->lam, ctx->mu, macro_mandel, -1.0, X3_OUT_SPEC,
                  E.spec, E.phi, nullptr);
    Launch<R>::x2(E.g, s, 0, E.spec, nullptr);
    Launch<R>::x1(E.g, s, X1_FWD | X1_GAMMA_OUT, E.spec, b, nullptr, nullptr, nullptr);
    ctx->launches += 3;
}

// real Mandel field -> spectrum (optionally material law, optionally projector)
template <typename R>
static void real_to_spec(hom_ctx *ctx, Engine<R> &E, const R *in, int mid, bool gamma, cpx<R> *out) {
    cudaStream_t s = ctx->stream;
    Launch<R>::x3(E.g, s, X3_IN_REAL, in, mid, ctx->lam, ctx->mu, nullptr, 1.0, X3_OUT_SPEC, E.spec, E.phi, nullptr);
    Launch<R>::x2(E.g, s, 0, E.spec, nullptr);
    Launch<R>::x1(E.g, s, X1_FWD | (gamma ? X1_GAMMA_OUT : 0), E.spec, out, nullptr, nullptr, nullptr);
    ctx->launches += 3;
}

// spectrum -> real Mandel field (optionally projecting first), times scale
template <typename R>
static void spec_to_real(hom_ctx *ctx, Engine<R> &E, const cpx<R> *in, bool gamma, double scl, R *out) {
    cudaStream_t s = ctx->stream;
    Launch<R>::x1(E.g, s, gamma ? X1_GAMMA_IN : 0, in, E.spec, nullptr, nullptr, nullptr);
    Launch<R>::x2(E.g, s, 1, E.spec, nullptr);
    Launch<R>::x3(E.g, s, X3_IN_SPEC, E.spec, X3_MID_NONE, ctx->lam, ctx->mu, nullptr, scl, X3_OUT_REAL, out, E.phi,
                  nullptr);
    ctx->launches += 3;
}

// weighted ||v||^2 of a spectral vector; synchronous.
template <typename R>
static int spec_norm2(hom_ctx *ctx, Engine<R> &E, const cpx<R> *v, double *out) {
    Launch<R>::norm2w(E.g, ctx->stream, v, ctx->partials);
    reduce_to(ctx->stream, ctx->partials, Launch<R>::ew_grid(6 * ctx->S), ctx->d_scalar);
    ctx->launches += 2;
    CU(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *out = *ctx->h_scalar;
    return HOM_OK;
}

// Capture graph_iters MINRES iterations of the tangent operator (the J2
// Newton systems; the elastic operator runs as a stacked batch, see
// capture_bbody) once (graph_iters even: the buffer roles repeat every 2
// steps).  Unnormalised Lanczos vectors u_k = beta_k v_k alternate between
// vbuf[1] (odd k) and vbuf[0] (even k); p = A^ u_k is vbuf[2]; w_j sits in
// wbuf[0] for even j and wbuf[1] for odd j.  A step is op_spec with the dot
// product <u_k, p>, the alpha reduction, the Lanczos step fused with the
// lagged w / x update, and the Givens step.
template <typename R>
static void capture_body(hom_ctx *ctx, Engine<R> &E) {
    cpx<R> *ua = (cpx<R> *)ctx->vbuf[0], *ub = (cpx<R> *)ctx->vbuf[1], *p = (cpx<R> *)ctx->vbuf[2];
    cpx<R> *wc = (cpx<R> *)ctx->wbuf[0], *wd = (cpx<R> *)ctx->wbuf[1];
    cpx<R> *x = (cpx<R> *)ctx->xs;
    const int np1 = Launch<R>::x1_grid(E.g), npe = Launch<R>::ew_grid(6 * ctx->S);
    cudaStream_t s = ctx->stream;
    for (int it = 0; it < ctx->graph_iters; ++it) {
        const bool odd = (it % 2) == 0;          // step k = it + 1 (mod 2)
        cpx<R> *uk = odd ? ub : ua, *um = odd ? ua : ub;
        cpx<R> *wa = odd ? wd : wc, *wb = odd ? wc : wd;   // w_{k-2}, w_{k-3}
        op_spec<R>(ctx, E, uk, p, true, ctx->partials, ctx->d_state);
        scalar_alpha(s, ctx->d_state, ctx->partials, np1);
        Launch<R>::lanczos_update(E.g, s, p, uk, um, wa, wb, x, ctx->d_state, ctx->partials);
        scalar_givens(s, ctx->d_state, ctx->partials, npe);
        ctx->launches += 3;
    }
}

// The solve loop as one graph: a WHILE node whose body is graph_iters
// iterations plus the loop condition, so a whole MINRES sweep is one graph
// launch with no host polling; where conditional nodes are not available,
// a graph of the body alone that the host replays.
template <typename R>
static int build_graph(hom_ctx *ctx, Engine<R> &E) {
    if (ctx->graph && ctx->graph_tangent == ctx->tangent_op) return HOM_OK;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    const long long before = ctx->launches;
    cudaGraph_t graph = nullptr;
    bool loops = false;
    if (!ctx->host_loop && cudaGraphCreate(&graph, 0) == cudaSuccess) {
        cudaGraphConditionalHandle h;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        cudaGraphNode_t node;
        if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess) {
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess) {
                cudaGraph_t body = np.conditional.phGraph_out[0];
                CU(cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
                capture_body<R>(ctx, E);
                loop_cond(ctx->stream, h, ctx->d_state);
                ctx->launches += 1;
                cudaError_t e = cudaStreamEndCapture(ctx->stream, &body);
                if (e != cudaSuccess) {
                    cudaGraphDestroy(graph);
                    return fail(ctx, HOM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
                }
                loops = true;
            }
        }
        if (!loops) {
            cudaGetLastError();
            cudaGraphDestroy(graph);
            graph = nullptr;
        }
    }
    if (!loops) {
        CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        capture_body<R>(ctx, E);
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
        if (e != cudaSuccess) return fail(ctx, HOM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    ctx->graph_kernels = ctx->launches - before;
    ctx->launches = before;   // counted per body run instead
    cudaError_t e = cudaGraphInstantiate(&ctx->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, HOM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    ctx->graph_loops = loops;
    ctx->graph_tangent = ctx->tangent_op;
    return HOM_OK;
}

// MINRES on A^ x = rhs (rhs in ctx->rhs, solution in ctx->xs, precision R),
// zero start.
template <typename R>
static int run_minres(hom_ctx *ctx, Engine<R> &E, double tol, int max_it, int *iters, double *est, int *status) {
    const long long nr = 12 * ctx->S;   // reals per spectral vector
    cudaStream_t s = ctx->stream;
    int rc = build_graph<R>(ctx, E);
    if (rc) return rc;
    const int max_replays = (max_it + ctx->graph_iters - 1) / ctx->graph_iters + 1;
    Launch<R>::norm2w(E.g, s, (const cpx<R> *)ctx->rhs, ctx->partials);
    scalar_start(s, ctx->d_state, ctx->partials, Launch<R>::ew_grid(6 * ctx->S), tol, max_it, max_replays);
    ctx->launches += 2;
    CU(cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(MinresState), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const double beta1 = ctx->h_state->beta1;
    CU(cudaMemsetAsync(ctx->xs, 0, sizeof(R) * nr, s));
    if (!(beta1 > 0.0) || !std::isfinite(beta1)) {
        *iters = 0;
        *est = 0.0;
        *status = std::isfinite(beta1) ? 0 : HOM_ENAN;
        CU(cudaStreamSynchronize(s));
        return HOM_OK;
    }
    // u_0 = 0, u_1 = rhs (= beta_1 v_1), w_0 = w_{-1} = 0
    CU(cudaMemsetAsync(ctx->vbuf[0], 0, sizeof(R) * nr, s));
    CU(cudaMemcpyAsync(ctx->vbuf[1], ctx->rhs, sizeof(R) * nr, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemsetAsync(ctx->wbuf[0], 0, sizeof(R) * nr, s));
    CU(cudaMemsetAsync(ctx->wbuf[1], 0, sizeof(R) * nr, s));
    if (ctx->graph_loops) {
        // one launch: the device repeats the body until done (or the cap)
        CU(cudaGraphLaunch(ctx->graph, s));
        CU(cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(MinresState), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        ctx->launches += (long long)ctx->h_state->bodies * ctx->graph_kernels;
    } else {
        // replay the captured body until the state says done
        const int per_check = 4;
        int replays = 0;
        while (true) {
            for (int r = 0; r < per_check && replays < max_replays; ++r, ++replays) {
                CU(cudaGraphLaunch(ctx->graph, s));
                ctx->launches += ctx->graph_kernels;
            }
            CU(cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(MinresState), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            if (ctx->h_state->done || replays >= max_replays) break;
        }
    }
    // the last step's lagged w / x update
    Launch<R>::minres_flush(E.g, s, (const cpx<R> *)ctx->vbuf[0], (const cpx<R> *)ctx->vbuf[1], nullptr, (cpx<R> *)ctx->wbuf[0],
                            (cpx<R> *)ctx->wbuf[1], (cpx<R> *)ctx->xs, ctx->d_state, 6 * ctx->S);
    ctx->launches += 1;
    *iters = ctx->h_state->k;
    *est = ctx->h_state->est;
    *status = ctx->h_state->status == -5 ? HOM_ENAN : (ctx->h_state->status == 1 ? HOM_NOT_CONVERGED : HOM_OK);
    return HOM_OK;
}

// ---------------------------------------------------------------------------
// MoDBFFT (section 2.2)
// ---------------------------------------------------------------------------
template <typename R>
static int engine_init_modb(hom_ctx *ctx, Engine<R> &E) {
    E.gm = E.g;
    E.gm.tma_cache = nullptr;
    int rc = set_shapes<R>(ctx, E.gm, 10);
    if (rc) return rc;
    CU(cudaMalloc(&E.spec10, cpx_size<R>() * 10 * ctx->S));
    ctx->workspace += cpx_size<R>() * 10 * ctx->S;
    return HOM_OK;
}

// out3 = A^alpha(u3), eq. (modbfftfop); optional <dotv, out3> partials
template <typename R>
static int op_modb(hom_ctx *ctx, Engine<R> &E, const cpx<R> *u, cpx<R> *out, const cpx<R> *dotv, double *partials,
                   const MinresState *st) {
    // returns the number of dot partials written (with dotv)
    cudaStream_t s = ctx->stream;
    const Geometry &g = E.gm;
    // the expansion fused into the inverse n1 pass where it is TMA-staged
    int nl = 4;   // launches before the forward n1 pass
    if (!Launch<R>::x1_modb_expand(g, s, ctx->alpha, u, E.spec10, st)) {
        Launch<R>::modb_expand(g, s, ctx->alpha, 1, u, E.spec10, 10, st);
        Launch<R>::x1(g, s, 0, E.spec10, E.spec10, nullptr, nullptr, st);
        nl += 1;
    }
    Launch<R>::x2(g, s, 1, E.spec10, st);
    Launch<R>::x3(g, s, X3_IN_SPEC, E.spec10, X3_MID_MODB, ctx->lam, ctx->mu, nullptr, 1.0, X3_OUT_SPEC, E.spec10,
                  E.phi, st);
    Launch<R>::x2(g, s, 0, E.spec10, st);
    // the forward n1 pass with the contraction fused where it is TMA-staged
    int np = Launch<R>::x1_modb_contract(g, s, E.spec10, out, dotv, partials, ctx->npartials, st);
    if (np > 0) {
        ctx->launches += nl + 1;
        return np;
    }
    Launch<R>::x1(g, s, X1_FWD, E.spec10, E.spec10, nullptr, nullptr, st);
    Launch<R>::modb_contract(g, s, E.spec10, out, dotv, partials, st);
    ctx->launches += nl + 2;
    return Launch<R>::ew_grid(g.S);
}

// b3 = -F{C : E_bar} . xi, eq. (modbfftfrhs) with sigma_bar = 0
template <typename R>
static void rhs_modb(hom_ctx *ctx, Engine<R> &E, const double *macro_mandel, cpx<R> *b) {
    cudaStream_t s = ctx->stream;
    const Geometry &g = E.gm;
    if constexpr (sizeof(R) == 8) {
        // F{C : E_bar} = phi^ (C_m : E_bar): no transform needed
        double tau[6];
        const double tr = macro_mandel[0] + macro_mandel[1] + macro_mandel[2];
        for (int c = 0; c < 6; ++c) tau[c] = (c < 3 ? ctx->lam * tr : 0.0) + 2.0 * ctx->mu * macro_mandel[c];
        Launch<R>::phihat_tau10(g, s, ctx->phihat, tau, E.spec10);
        ctx->launches += 1;
    } else {
        Launch<R>::x3(g, s, X3_IN_MACRO, nullptr, X3_MID_MATERIAL, ctx->lam, ctx->mu, macro_mandel, -1.0,
                      X3_OUT_SPEC, E.spec10, E.phi, nullptr);
        Launch<R>::x2(g, s, 0, E.spec10, nullptr);
        Launch<R>::x1(g, s, X1_FWD, E.spec10, E.spec10, nullptr, nullptr, nullptr);
        ctx->launches += 3;
    }
    Launch<R>::modb_contract(g, s, E.spec10, b, nullptr, nullptr, nullptr);
    ctx->launches += 1;
}

// mean stiffness of eq. (avstiff) in units of E
static void cbar(const hom_ctx *ctx, double *lam_b, double *mu_b) {
    *lam_b = ctx->phibar * ctx->lam;
    *mu_b = ctx->phibar * ctx->mu;
}

// One PCG iteration per graph replay: q = A p (with <p, q>), step, x/r/z,
// direction.  Buffers: x = xs, r = vbuf[0], p = vbuf[1], q = vbuf[2], z = wbuf[0].
template <typename R>
static int build_cg_graph(hom_ctx *ctx, Engine<R> &E) {
    if (ctx->cg_graph) return HOM_OK;
    cpx<R> *x = (cpx<R> *)ctx->xs, *r = (cpx<R> *)ctx->vbuf[0], *p = (cpx<R> *)ctx->vbuf[1];
    cpx<R> *q = (cpx<R> *)ctx->vbuf[2], *z = (cpx<R> *)ctx->wbuf[0];
    const int np = Launch<R>::ew_grid(E.g.S);
    const MinresState *flags = reinterpret_cast<const MinresState *>(ctx->d_cg);
    double lam_b, mu_b;
    cbar(ctx, &lam_b, &mu_b);
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const long long before = ctx->launches;
    for (int it = 0; it < 4; ++it) {
        const int npq = op_modb<R>(ctx, E, p, q, p, ctx->partials, flags);
        scalar_cg_alpha(ctx->stream, ctx->d_cg, ctx->partials, npq);
        Launch<R>::cg_xr(E.g, ctx->stream, lam_b, mu_b, x, r, p, q, z, ctx->d_cg, ctx->partials);
        scalar_cg_beta(ctx->stream, ctx->d_cg, ctx->partials, np);
        Launch<R>::cg_p(E.g, ctx->stream, p, z, ctx->d_cg);
        ctx->launches += 4;
    }
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (e != cudaSuccess) return fail(ctx, HOM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    ctx->cg_graph_kernels = ctx->launches - before;
    ctx->launches = before;
    e = cudaGraphInstantiate(&ctx->cg_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, HOM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return HOM_OK;
}

// PCG on A^alpha x = rhs (ctx->rhs, 3-component spectrum), zero start;
// solution in ctx->xs.  As the paper does (section 2.2) the preconditioned CG
// recurrences are used although A^alpha is not symmetric where chi_v is
// non-zero; the FP64 true residual checks the result.
template <typename R>
static int run_cg(hom_ctx *ctx, Engine<R> &E, double tol, int max_it, int *iters, double *est, int *status) {
    const long long nr = 6 * ctx->S;   // reals per 3-component spectral vector
    cudaStream_t s = ctx->stream;
    int rc = build_cg_graph<R>(ctx, E);
    if (rc) return rc;
    cpx<R> *x = (cpx<R> *)ctx->xs, *r = (cpx<R> *)ctx->vbuf[0], *p = (cpx<R> *)ctx->vbuf[1];
    cpx<R> *q = (cpx<R> *)ctx->vbuf[2], *z = (cpx<R> *)ctx->wbuf[0];
    double lam_b, mu_b;
    cbar(ctx, &lam_b, &mu_b);
    CU(cudaMemsetAsync(x, 0, sizeof(R) * nr, s));
    CU(cudaMemsetAsync(p, 0, sizeof(R) * nr, s));
    CU(cudaMemsetAsync(q, 0, sizeof(R) * nr, s));
    CU(cudaMemcpyAsync(r, ctx->rhs, sizeof(R) * nr, cudaMemcpyDeviceToDevice, s));
    // z0 = M r0 and <r0, z0>, ||r0||^2 through one step of length 0
    memset(ctx->h_cg, 0, sizeof(CgState));
    CU(cudaMemcpyAsync(ctx->d_cg, ctx->h_cg, sizeof(CgState), cudaMemcpyHostToDevice, s));
    const int np = Launch<R>::ew_grid(E.g.S);
    Launch<R>::cg_xr(E.g, s, lam_b, mu_b, x, r, p, q, z, ctx->d_cg, ctx->partials);
    scalar_cg_start(s, ctx->d_cg, ctx->partials, np, tol, max_it);
    Launch<R>::cg_p(E.g, s, p, z, ctx->d_cg);   // p0 = z0 (b = 0)
    ctx->launches += 3;
    CU(cudaMemcpyAsync(ctx->h_cg, ctx->d_cg, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (ctx->h_cg->done) {
        *iters = 0;
        *est = 0.0;
        *status = ctx->h_cg->status == -5 ? HOM_ENAN : HOM_OK;
        return HOM_OK;
    }
    const int per_check = 4;
    int replays = 0;
    const int max_replays = (max_it + 3) / 4 + 1;
    while (true) {
        for (int k = 0; k < per_check && replays < max_replays; ++k, ++replays) {
            CU(cudaGraphLaunch(ctx->cg_graph, s));
            ctx->launches += ctx->cg_graph_kernels;
        }
        CU(cudaMemcpyAsync(ctx->h_cg, ctx->d_cg, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (ctx->h_cg->done || replays >= max_replays) break;
    }
    *iters = ctx->h_cg->k;
    *est = ctx->h_cg->est;
    *status = ctx->h_cg->status == -5 ? HOM_ENAN : (ctx->h_cg->status == 1 ? HOM_NOT_CONVERGED : HOM_OK);
    return HOM_OK;
}

// Galerkin CG (section 2.1): graph_iters iterations per captured graph,
// replayed by the host.  Buffers: x = xs, r = vbuf[0], p = vbuf[1],
// q = A^ p = vbuf[2]; the scalars are the CgState kernels (no preconditioner).
template <typename R>
static int build_gcg_graph(hom_ctx *ctx, Engine<R> &E) {
    if (ctx->cg_graph) return HOM_OK;
    cpx<R> *x = (cpx<R> *)ctx->xs, *r = (cpx<R> *)ctx->vbuf[0], *p = (cpx<R> *)ctx->vbuf[1];
    cpx<R> *q = (cpx<R> *)ctx->vbuf[2];
    const long long n = 6 * ctx->S;
    const int np1 = Launch<R>::x1_grid(E.g), npc = gcg_blocks(n);
    const MinresState *flags = reinterpret_cast<const MinresState *>(ctx->d_cg);
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const long long before = ctx->launches;
    for (int it = 0; it < ctx->graph_iters; ++it) {
        op_spec<R>(ctx, E, p, q, true, ctx->partials, flags);   // q = A^ p, partial <p, q>
        scalar_cg_alpha(ctx->stream, ctx->d_cg, ctx->partials, np1);
        gcg_xr<R>(n, E.g.h, E.g.n3, ctx->stream, p, q, x, r, ctx->d_cg, ctx->partials);
        scalar_cg_beta(ctx->stream, ctx->d_cg, ctx->partials, npc);
        gcg_p<R>(n, ctx->stream, r, p, ctx->d_cg);
        ctx->launches += 4;
    }
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (e != cudaSuccess) return fail(ctx, HOM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    ctx->cg_graph_kernels = ctx->launches - before;
    ctx->launches = before;
    e = cudaGraphInstantiate(&ctx->cg_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, HOM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return HOM_OK;
}

// CG on A^ x = rhs from x = 0; stops at ||r_k|| / ||r_0|| <= tol (recursive
// residual) or max_it
template <typename R>
static int run_gcg(hom_ctx *ctx, Engine<R> &E, double tol, int max_it, int *iters, double *est, int *status) {
    const long long n = 6 * ctx->S, nr = 2 * n;
    cudaStream_t s = ctx->stream;
    int rc = build_gcg_graph<R>(ctx, E);
    if (rc) return rc;
    cpx<R> *x = (cpx<R> *)ctx->xs, *r = (cpx<R> *)ctx->vbuf[0], *p = (cpx<R> *)ctx->vbuf[1];
    cpx<R> *q = (cpx<R> *)ctx->vbuf[2];
    CU(cudaMemsetAsync(x, 0, sizeof(R) * nr, s));
    CU(cudaMemsetAsync(p, 0, sizeof(R) * nr, s));
    CU(cudaMemsetAsync(q, 0, sizeof(R) * nr, s));
    CU(cudaMemcpyAsync(r, ctx->rhs, sizeof(R) * nr, cudaMemcpyDeviceToDevice, s));
    // ||r_0||^2 through one step of length 0, then p_0 = r_0 (b = 0)
    memset(ctx->h_cg, 0, sizeof(CgState));
    CU(cudaMemcpyAsync(ctx->d_cg, ctx->h_cg, sizeof(CgState), cudaMemcpyHostToDevice, s));
    gcg_xr<R>(n, E.g.h, E.g.n3, s, p, q, x, r, ctx->d_cg, ctx->partials);
    scalar_cg_start(s, ctx->d_cg, ctx->partials, gcg_blocks(n), tol, max_it);
    gcg_p<R>(n, s, r, p, ctx->d_cg);
    ctx->launches += 3;
    CU(cudaMemcpyAsync(ctx->h_cg, ctx->d_cg, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (ctx->h_cg->done) {
        *iters = 0;
        *est = 0.0;
        *status = ctx->h_cg->status == -5 ? HOM_ENAN : HOM_OK;
        return HOM_OK;
    }
    const int per_check = 4;
    int replays = 0;
    const int max_replays = (max_it + ctx->graph_iters - 1) / ctx->graph_iters + 1;
    while (true) {
        for (int k = 0; k < per_check && replays < max_replays; ++k, ++replays) {
            CU(cudaGraphLaunch(ctx->cg_graph, s));
            ctx->launches += ctx->cg_graph_kernels;
        }
        CU(cudaMemcpyAsync(ctx->h_cg, ctx->d_cg, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (ctx->h_cg->done || replays >= max_replays) break;
    }
    *iters = ctx->h_cg->k;
    *est = ctx->h_cg->est;
    *status = ctx->h_cg->status == -5 ? HOM_ENAN : (ctx->h_cg->status == 1 ? HOM_NOT_CONVERGED : HOM_OK);
    return HOM_OK;
}

// the Krylov solver of a Galerkin context
template <typename R>
static int run_krylov(hom_ctx *ctx, Engine<R> &E, double tol, int max_it, int *iters, double *est, int *status) {
    return ctx->solver == HOM_SOLVER_GALERKIN_CG ? run_gcg<R>(ctx, E, tol, max_it, iters, est, status)
                                                 : run_minres<R>(ctx, E, tol, max_it, iters, est, status);
}

static void macro_to_mandel(const double *t, double *m) {
    const double r2 = std::sqrt(2.0);
    for (int c = 0; c < 6; ++c) m[c] = (c < 3) ? t[c] : t[c] * r2;
}

// host <-> device staging for user buffers
static int stage_in(hom_ctx *ctx, const void *user, size_t bytes, void *dev) {
    if (ctx->device_ptrs) CU(cudaMemcpyAsync(dev, user, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    else CU(cudaMemcpyAsync(dev, user, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return HOM_OK;
}
static int stage_out(hom_ctx *ctx, void *user, size_t bytes, const void *dev) {
    if (ctx->device_ptrs) CU(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    else CU(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return HOM_OK;
}

static int finish(hom_ctx *ctx) {
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(ctx->stream));
    int e = 0;
    CU(cudaMemcpy(&e, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        CU(cudaMemset(ctx->d_err, 0, sizeof(int)));
        return fail(ctx, HOM_ETIMEOUT, "a bounded device wait gave up (TMA copy did not complete)");
    }
    return HOM_OK;
}

// ---------------------------------------------------------------------------
// C ABI (C linkage comes from the declarations in hom.h)
// ---------------------------------------------------------------------------

void hom_default_options(hom_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->solver = HOM_SOLVER_GALERKIN_MINRES;
    opt->precision = HOM_PREC_FP32_FIELDS;
    opt->device_ptrs = 0;
    opt->stream = nullptr;
    opt->device = -1;
    opt->refine = 3;
}

const char *hom_last_error(const hom_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

static void j2_free(hom_ctx *ctx) {
    J2State &j = ctx->j2;
    double *bufs[] = {j.eps, j.eps_t, j.etry, j.epsp, j.alpha, j.sig, j.de, j.Ct, j.partials};
    for (double *p : bufs) cudaFree(p);
    float *fbufs[] = {j.Ct32, j.sig32, j.de32};
    for (float *p : fbufs) cudaFree(p);
    cudaFree(j.x64);
    if (j.h_partials) cudaFreeHost(j.h_partials);
    j = J2State{};
    ctx->tangent_op = false;
    if (ctx->graph && ctx->graph_tangent) {   // it holds the freed buffers
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
}

void hom_destroy(hom_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    j2_free(ctx);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->cg_graph) cudaGraphExecDestroy(ctx->cg_graph);
    batch_free(ctx);
    cudaFree(ctx->d_cg);
    if (ctx->h_cg) cudaFreeHost(ctx->h_cg);
    engine_free(ctx->e32);
    engine_free(ctx->e64);
    for (int i = 0; i < 3; ++i) cudaFree(ctx->vbuf[i]);
    for (int i = 0; i < 2; ++i) cudaFree(ctx->wbuf[i]);
    cudaFree(ctx->xs);
    cudaFree(ctx->rhs);
    cudaFree(ctx->b64);
    cudaFree(ctx->r64);
    cudaFree(ctx->phihat);
    for (double2 *p : ctx->x64) cudaFree(p);
    cudaFree(ctx->partials);
    cudaFree(ctx->d_state);
    cudaFree(ctx->d_scalar);
    cudaFree(ctx->tsum_part);
    cudaFree(ctx->d_flag);
    cudaFree(ctx->d_err);
    if (ctx->h_state) cudaFreeHost(ctx->h_state);
    if (ctx->h_scalar) cudaFreeHost(ctx->h_scalar);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

static int create_impl(hom_ctx *ctx, const int grid[3], const void *phase, int input_kind) {
    {   // HOM_PDL=1 in the environment: programmatic launches in the MINRES
        // graph (measured 1.591 against 1.546 ms per step at 256^3: the early
        // successors' CTAs hold SM resources while the predecessor drains)
        const char *e = std::getenv("HOM_PDL");
        ctx->pdl = (e && e[0] == '1') ? 1 : 0;
    }
    for (int p = 0; p < 3; ++p) {
        AxisPlan tmp{};
        if (grid[p] < 2 || grid[p] > 512 || !factor_radices(grid[p], tmp))
            return fail(ctx, HOM_EUNSUPPORTED_GRID, "each grid size must be in [2,512] and of the form 2^a3^b5^c");
        ctx->n[p] = grid[p];
    }
    ctx->V = (long long)grid[0] * grid[1] * grid[2];
    ctx->S = (long long)grid[0] * grid[1] * (grid[2] / 2 + 1);
    if (12 * ctx->S >= (1LL << 31)) return fail(ctx, HOM_EUNSUPPORTED_GRID, "12 S must stay below 2^31");
    CU(cudaSetDevice(ctx->device));
    if (!ctx->stream) {
        CU(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    CU(cudaEventCreate(&ctx->ev0));
    CU(cudaEventCreate(&ctx->ev1));
    CU(cudaMalloc(&ctx->d_err, sizeof(int)));
    CU(cudaMemset(ctx->d_err, 0, sizeof(int)));
    int rc = engine_init<double>(ctx, ctx->e64);
    if (rc) return rc;
    if (ctx->prec == HOM_PREC_FP32_FIELDS) {
        rc = engine_init<float>(ctx, ctx->e32);
        if (rc) return rc;
    }
    if (ctx->solver == HOM_SOLVER_MODBFFT_CG) {
        rc = engine_init_modb<double>(ctx, ctx->e64);
        if (rc) return rc;
        if (ctx->prec == HOM_PREC_FP32_FIELDS) {
            rc = engine_init_modb<float>(ctx, ctx->e32);
            if (rc) return rc;
        }
    }
    if (ctx->solver != HOM_SOLVER_GALERKIN_MINRES) {
        CU(cudaMalloc(&ctx->d_cg, sizeof(CgState)));
        CU(cudaMallocHost(&ctx->h_cg, sizeof(CgState)));
    }
    const long long nr = 12 * ctx->S;   // reals per spectral vector (>= 6 V)
    const size_t rs = (ctx->prec == HOM_PREC_FP64) ? sizeof(double) : sizeof(float);
    // single-case Krylov vectors (half spectra): the tangent operator's MINRES,
    // CG / PCG, and scratch of the step entry points and the timing instrument
    // (which runs the fused chain on one case: the padded n1-tile order)
    const long long kv = (ctx->prec == HOM_PREC_FP64) ? ctx->e64.g.kvec : ctx->e32.g.kvec;
    const long long nk = std::max(nr, 2 * kv);
    for (int i = 0; i < 3; ++i) CU(cudaMalloc(&ctx->vbuf[i], rs * nk));
    for (int i = 0; i < 2; ++i) CU(cudaMalloc(&ctx->wbuf[i], rs * nk));
    CU(cudaMalloc(&ctx->xs, rs * nk));
    ctx->krylov_reals = nk;
    CU(cudaMalloc(&ctx->rhs, rs * nr));
    CU(cudaMalloc(&ctx->b64, sizeof(double) * nr));
    CU(cudaMalloc(&ctx->phihat, sizeof(double2) * ctx->S));
    CU(cudaMalloc(&ctx->r64, sizeof(double) * nr));
    ctx->workspace += 6 * (long long)rs * nk + (long long)rs * nr + 2 * (long long)sizeof(double) * nr;
    long long np = 8LL * kEwBlocks;
    np = std::max(np, (long long)Launch<double>::x1_grid(ctx->e64.g));
    np = std::max(np, (long long)Launch<double>::x3_grid(ctx->e64.g));
    np = std::max(np, (long long)Launch<double>::x1_lanczos_grid(ctx->e64.g));
    if (ctx->prec == HOM_PREC_FP32_FIELDS) {
        np = std::max(np, (long long)Launch<float>::x1_grid(ctx->e32.g));
        np = std::max(np, (long long)Launch<float>::x3_grid(ctx->e32.g));
        np = std::max(np, (long long)Launch<float>::x1_lanczos_grid(ctx->e32.g));
    }
    ctx->npartials = (int)np;
    CU(cudaMalloc(&ctx->partials, sizeof(double) * ctx->npartials));
    CU(cudaMalloc(&ctx->d_state, sizeof(MinresState)));
    CU(cudaMalloc(&ctx->d_scalar, sizeof(double) * 8));
    CU(cudaMalloc(&ctx->tsum_part, sizeof(double) * 6 * Launch<double>::x3_grid(ctx->e64.g)));
    CU(cudaMalloc(&ctx->d_flag, sizeof(int)));
    CU(cudaMallocHost(&ctx->h_state, sizeof(MinresState)));
    CU(cudaMallocHost(&ctx->h_scalar, sizeof(double) * 8));
    // phase map -> phi (FP64 copy always; FP32 copy for FP32 fields)
    const size_t in_bytes = (input_kind == HOM_INPUT_PHASE_U8 ? 1 : input_kind == HOM_INPUT_FRACTION_F32 ? 4 : 8);
    void *dev_in = ctx->xs;   // staging (xs holds >= 6 V reals of the solve precision >= V * 8 bytes)
    rc = stage_in(ctx, phase, in_bytes * ctx->V, dev_in);
    if (rc) return rc;
    CU(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    phi_convert<double>(ctx->V, ctx->stream, dev_in, input_kind, ctx->e64.phi, ctx->d_flag);
    if (ctx->prec == HOM_PREC_FP32_FIELDS)
        phi_convert<float>(ctx->V, ctx->stream, dev_in, input_kind, ctx->e32.phi, ctx->d_flag);
    ctx->launches += 2;
    int bad = 0;
    CU(cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (bad) return fail(ctx, HOM_EINVAL, "phase values must be finite and in [0,1]");
    // sum phi and phi^2 (mean density, scale of the zero right-hand-side
    // test): FP64 reductions on the device
    {
        const int nb = phi_sums(ctx->V, ctx->e64.phi, ctx->partials, ctx->stream);
        reduce_to(ctx->stream, ctx->partials, nb, ctx->d_scalar);
        reduce_to(ctx->stream, ctx->partials + nb, nb, ctx->d_scalar + 1);
        ctx->launches += 3;
        CU(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        ctx->phibar = ctx->h_scalar[0] / (double)ctx->V;
        ctx->phi2_sum = ctx->h_scalar[1];
    }
    // phi^ = F{phi} (FP64): the field [phi, 0, 0, 0, 0, 0] through the forward
    // passes, component 0 kept
    {
        double *f6 = (double *)ctx->r64;
        CU(cudaMemsetAsync(f6, 0, sizeof(double) * 6 * ctx->V, ctx->stream));
        CU(cudaMemcpyAsync(f6, ctx->e64.phi, sizeof(double) * ctx->V, cudaMemcpyDeviceToDevice, ctx->stream));
        real_to_spec<double>(ctx, ctx->e64, f6, X3_MID_NONE, false, ctx->b64);
        CU(cudaMemcpy2DAsync(ctx->phihat, sizeof(double2), ctx->b64, 6 * sizeof(double2), sizeof(double2), ctx->S,
                             cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return finish(ctx);
}

int hom_create(hom_ctx **out, const int grid[3], const void *phase, int input_kind, double E, double nu,
               int smoothing, int derivative, const hom_options *opt) {
    if (!out || !grid || !phase) return fail(nullptr, HOM_EINVAL, "null argument");
    *out = nullptr;
    if (!(E > 0.0) || !std::isfinite(E) || !(nu > -1.0 && nu < 0.5))
        return fail(nullptr, HOM_EINVAL, "need E > 0 and -1 < nu < 0.5");
    if (input_kind < 0 || input_kind > 2) return fail(nullptr, HOM_EINVAL, "bad input_kind");
    if (smoothing != HOM_SMOOTH_NONE) return fail(nullptr, HOM_EINVAL, "bad smoothing");
    if (derivative != HOM_DERIV_CONTINUOUS && derivative != HOM_DERIV_ROTATED)
        return fail(nullptr, HOM_EINVAL, "bad derivative");
    hom_options o;
    hom_default_options(&o);
    if (opt) o = *opt;
    if (o.autotune && o.rows3 == 0 && o.tile2 == 0 && o.tile1 == 0) {
        int shp[3] = {0, 0, 0};
        if (hom_autotune(grid, o.precision, shp) == HOM_OK) {
            o.rows3 = shp[0];
            o.tile2 = shp[1];
            o.tile1 = shp[2];
        }
    }
    if (o.solver != HOM_SOLVER_GALERKIN_MINRES && o.solver != HOM_SOLVER_MODBFFT_CG &&
        o.solver != HOM_SOLVER_GALERKIN_CG)
        return fail(nullptr, HOM_EINVAL, "bad solver");
    if (!(o.alpha >= 0.0) || !std::isfinite(o.alpha)) return fail(nullptr, HOM_EINVAL, "bad alpha");
    if (o.precision != HOM_PREC_FP32_FIELDS && o.precision != HOM_PREC_FP64)
        return fail(nullptr, HOM_EINVAL, "bad precision");
    if (o.rows3 < 0 || o.rows3 > 64 || o.tile2 < 0 || o.tile2 > 32 || o.tile1 < 0 || o.tile1 > 16)
        return fail(nullptr, HOM_EINVAL, "bad launch-shape override");
    if (!(o.sweep_floor >= 0.0 && o.sweep_floor < 1.0))
        return fail(nullptr, HOM_EINVAL, "sweep_floor must be in [0, 1)");
    hom_ctx *ctx = new hom_ctx();
    ctx->prec = o.precision;
    ctx->deriv = derivative;
    ctx->E = E;
    ctx->nu = nu;
    ctx->lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));   // lambda / E
    ctx->mu = 1.0 / (2.0 * (1.0 + nu));                // mu / E
    ctx->device_ptrs = o.device_ptrs;
    ctx->refine = o.refine < 0 ? 0 : o.refine;
    ctx->sweep_floor = o.sweep_floor > 0.0 ? o.sweep_floor
                                            : (o.solver == HOM_SOLVER_MODBFFT_CG ? kFp32CgSweepFloor : kFp32SweepFloor);
    ctx->shape[0] = o.rows3;
    ctx->shape[1] = o.tile2;
    ctx->shape[2] = o.tile1;
    ctx->staging = o.staging;
    ctx->host_loop = o.host_loop != 0;
    ctx->solver = o.solver;
    ctx->alpha = (o.alpha > 0.0) ? o.alpha : 1e-4;
    ctx->stream = (cudaStream_t)o.stream;
    if (o.device >= 0) ctx->device = o.device;
    else if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        delete ctx;
        return fail(nullptr, HOM_ECUDA, "no CUDA device");
    }
    int rc = create_impl(ctx, grid, phase, input_kind);
    if (rc) {
        g_create_error = ctx->err;
        hom_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return HOM_OK;
}

// Phase-field smoothening (section 3.2) on a temporary FP64 context of the
// fine grid: its creation already holds phi^ = F{omega}; filter it (eq.
// (phase3), continuous frequencies), transform back as component 0 of a
// Mandel spectrum, and average r^3 blocks with the threshold.
static int pfs_impl(hom_ctx *ctx, const int fine[3], int ratio, double ell, double eps, double threshold,
                    double *phi_out) {
    cudaStream_t s = ctx->stream;
    pfs_filter(fine[0], fine[1], fine[2], ell * ell / eps, ctx->phihat, s);
    CU(cudaMemsetAsync(ctx->b64, 0, sizeof(double2) * 6 * ctx->S, s));
    CU(cudaMemcpy2DAsync(ctx->b64, 6 * sizeof(double2), ctx->phihat, sizeof(double2), sizeof(double2), ctx->S,
                         cudaMemcpyDeviceToDevice, s));
    spec_to_real<double>(ctx, ctx->e64, (const cpx<double> *)ctx->b64, false, 1.0, (double *)ctx->r64);
    double *coarse = (double *)ctx->vbuf[0];
    pfs_coarsen(fine[0], fine[1], fine[2], ratio, threshold, (const double *)ctx->r64, coarse, s);
    ctx->launches += 2;
    const long long Vc = (long long)(fine[0] / ratio) * (fine[1] / ratio) * (fine[2] / ratio);
    int rc = stage_out(ctx, phi_out, sizeof(double) * Vc, coarse);
    if (rc) return rc;
    return finish(ctx);
}

int hom_pfs(const int fine[3], const void *omega, int input_kind, int ratio, double ell, double eps,
            double threshold, int device_ptrs, double *phi_out) {
    if (!fine || !omega || !phi_out) return fail(nullptr, HOM_EINVAL, "null argument");
    if (ratio < 1 || fine[0] % ratio || fine[1] % ratio || fine[2] % ratio)
        return fail(nullptr, HOM_EINVAL, "every fine grid size must be a multiple of ratio");
    if (!(ell >= 0.0) || !std::isfinite(ell) || !(eps > 0.0) || !std::isfinite(eps) || !std::isfinite(threshold))
        return fail(nullptr, HOM_EINVAL, "need ell >= 0, eps > 0 and a finite threshold");
    hom_options o;
    hom_default_options(&o);
    o.precision = HOM_PREC_FP64;
    o.device_ptrs = device_ptrs;
    hom_ctx *ctx = nullptr;
    int rc = hom_create(&ctx, fine, omega, input_kind, 1.0, 0.3, HOM_SMOOTH_NONE, HOM_DERIV_CONTINUOUS, &o);
    if (rc) return rc;
    rc = pfs_impl(ctx, fine, ratio, ell, eps, threshold, phi_out);
    if (rc) g_create_error = ctx->err;
    hom_destroy(ctx);
    return rc;
}

int hom_get_info(const hom_ctx *ctx, int grid[3], int *precision, long long *workspace_bytes) {
    if (!ctx) return HOM_EINVAL;
    if (grid) for (int p = 0; p < 3; ++p) grid[p] = ctx->n[p];
    if (precision) *precision = ctx->prec;
    if (workspace_bytes) *workspace_bytes = ctx->workspace + (long long)ctx->x64.size() * 12 * ctx->S * 8;
    return HOM_OK;
}

long long hom_kernel_launches(const hom_ctx *ctx) { return ctx ? ctx->launches : 0; }

// ----- step entry points ----------------------------------------------------
template <typename R>
static int step_impl(hom_ctx *ctx, Engine<R> &E, int which, const void *in, void *out, const double *macro) {
    const long long n = 6 * ctx->V;
    R *din = (R *)ctx->vbuf[0], *dout = (R *)ctx->vbuf[1];
    cpx<R> *spec = (cpx<R> *)ctx->vbuf[2];
    int rc;
    switch (which) {
        case 0:  // apply (Mandel): A(e) = F^-1 G F C e
            rc = stage_in(ctx, in, sizeof(R) * n, din);
            if (rc) return rc;
            real_to_spec<R>(ctx, E, din, X3_MID_MATERIAL, true, spec);
            spec_to_real<R>(ctx, E, spec, false, 1.0, dout);
            return stage_out(ctx, out, sizeof(R) * n, dout);
        case 1: {  // rhs (Mandel)
            double m[6];
            macro_to_mandel(macro, m);
            rhs_spec<R>(ctx, E, m, spec);
            spec_to_real<R>(ctx, E, spec, false, 1.0, dout);
            return stage_out(ctx, out, sizeof(R) * n, dout);
        }
        case 2:  // forward FFT
            rc = stage_in(ctx, in, sizeof(R) * n, din);
            if (rc) return rc;
            real_to_spec<R>(ctx, E, din, X3_MID_NONE, false, spec);
            return stage_out(ctx, out, cpx_size<R>() * 6 * ctx->S, spec);
        case 5: {  // spectral operator A^ = G F C F^-1 G on a spectrum
            cpx<R> *sout = (cpx<R> *)ctx->vbuf[0];
            rc = stage_in(ctx, in, cpx_size<R>() * 6 * ctx->S, spec);
            if (rc) return rc;
            op_spec<R>(ctx, E, spec, sout, false, nullptr, nullptr);
            return stage_out(ctx, out, cpx_size<R>() * 6 * ctx->S, sout);
        }
        case 3:  // inverse FFT
            rc = stage_in(ctx, in, cpx_size<R>() * 6 * ctx->S, spec);
            if (rc) return rc;
            spec_to_real<R>(ctx, E, spec, false, 1.0, dout);
            return stage_out(ctx, out, sizeof(R) * n, dout);
        default:  // projection (Mandel)
            rc = stage_in(ctx, in, sizeof(R) * n, din);
            if (rc) return rc;
            real_to_spec<R>(ctx, E, din, X3_MID_NONE, true, spec);
            spec_to_real<R>(ctx, E, spec, false, 1.0, dout);
            return stage_out(ctx, out, sizeof(R) * n, dout);
    }
}

static int step(hom_ctx *ctx, int which, const void *in, void *out, const double *macro) {
    if (!ctx || !out || (which != 1 && !in) || (which == 1 && !macro)) return fail(ctx, HOM_EINVAL, "null argument");
    cudaSetDevice(ctx->device);
    int rc = (ctx->prec == HOM_PREC_FP64) ? step_impl<double>(ctx, ctx->e64, which, in, out, macro)
                                          : step_impl<float>(ctx, ctx->e32, which, in, out, macro);
    if (rc) return rc;
    return finish(ctx);
}

template <typename R>
static int modb_step_impl(hom_ctx *ctx, Engine<R> &E, int which, const void *in, void *out, const double *macro) {
    const size_t bytes = cpx_size<R>() * 3 * ctx->S;
    cpx<R> *din = (cpx<R> *)ctx->vbuf[0], *dout = (cpx<R> *)ctx->vbuf[1];
    int rc;
    if (which == 0) {
        rc = stage_in(ctx, in, bytes, din);
        if (rc) return rc;
        op_modb<R>(ctx, E, din, dout, nullptr, nullptr, nullptr);
    } else if (which == 1) {
        double m[6];
        macro_to_mandel(macro, m);
        rhs_modb<R>(ctx, E, m, dout);
    } else {
        rc = stage_in(ctx, in, bytes, din);
        if (rc) return rc;
        double lam_b, mu_b;
        cbar(ctx, &lam_b, &mu_b);
        Launch<R>::modb_precond(E.g, ctx->stream, lam_b, mu_b, din, dout);
        ctx->launches += 1;
    }
    return stage_out(ctx, out, bytes, dout);
}

static int modb_step(hom_ctx *ctx, int which, const void *in, void *out, const double *macro) {
    if (!ctx || !out || (which != 1 && !in) || (which == 1 && !macro)) return fail(ctx, HOM_EINVAL, "null argument");
    if (ctx->solver != HOM_SOLVER_MODBFFT_CG) return fail(ctx, HOM_EINVAL, "context was not created for MoDBFFT");
    cudaSetDevice(ctx->device);
    int rc = (ctx->prec == HOM_PREC_FP64) ? modb_step_impl<double>(ctx, ctx->e64, which, in, out, macro)
                                          : modb_step_impl<float>(ctx, ctx->e32, which, in, out, macro);
    if (rc) return rc;
    return finish(ctx);
}

int hom_modb_apply(hom_ctx *ctx, const void *u, void *out) { return modb_step(ctx, 0, u, out, nullptr); }
int hom_modb_rhs(hom_ctx *ctx, const double macro_strain[6], void *out) { return modb_step(ctx, 1, nullptr, out, macro_strain); }
int hom_modb_precond(hom_ctx *ctx, const void *in, void *out) { return modb_step(ctx, 2, in, out, nullptr); }

int hom_apply(hom_ctx *ctx, const void *eps, void *out) { return step(ctx, 0, eps, out, nullptr); }
int hom_rhs(hom_ctx *ctx, const double macro_strain[6], void *out) { return step(ctx, 1, nullptr, out, macro_strain); }
int hom_fft_forward(hom_ctx *ctx, const void *field, void *spectrum) { return step(ctx, 2, field, spectrum, nullptr); }
int hom_fft_inverse(hom_ctx *ctx, const void *spectrum, void *field) { return step(ctx, 3, spectrum, field, nullptr); }
int hom_project(hom_ctx *ctx, const void *in, void *out) { return step(ctx, 4, in, out, nullptr); }
int hom_apply_spectrum(hom_ctx *ctx, const void *in, void *out) { return step(ctx, 5, in, out, nullptr); }

// ----- stacked-batch MINRES ---------------------------------------------------------
static void batch_free(hom_ctx *ctx) {
    if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
    ctx->bgraph = nullptr;
    ctx->bgraph_nb = 0;
    tma_cache_free(ctx->btma);
    ctx->btma = nullptr;
    for (void *p : {ctx->bspec, ctx->bv[0], ctx->bv[1], ctx->bv[2], ctx->bw[0], ctx->bw[1], ctx->bx, ctx->brhs}) cudaFree(p);
    cudaFree(ctx->bb64);
    cudaFree(ctx->br64);
    cudaFree(ctx->d_bst);
    cudaFree(ctx->bpart);
    cudaFree(ctx->bcnt);
    ctx->bcnt = nullptr;
    if (ctx->h_bst) cudaFreeHost(ctx->h_bst);
    ctx->bspec = ctx->bv[0] = ctx->bv[1] = ctx->bv[2] = ctx->bw[0] = ctx->bw[1] = ctx->bx = ctx->brhs = nullptr;
    ctx->bb64 = ctx->br64 = nullptr;
    ctx->d_bst = ctx->h_bst = nullptr;
    ctx->bpart = nullptr;
    ctx->bcap = 0;
    ctx->bg.nb = 0;
}

// device bytes of one load case of a stacked batch
static long long batch_case_bytes(const hom_ctx *ctx) {
    const long long n6 = 6 * ctx->S;
    const bool f64 = ctx->prec == HOM_PREC_FP64;
    const long long cs = f64 ? 16 : 8;
    const long long kv = f64 ? ctx->e64.g.kvec : ctx->e32.g.kvec;
    return cs * (2 * n6 + 6 * kv) + 2 * 16 * n6;
}

// room for nb load cases (frees and reallocates when it grows)
static int batch_reserve(hom_ctx *ctx, int nb) {
    if (ctx->bcap >= nb) return HOM_OK;
    batch_free(ctx);
    const long long n6 = 6 * ctx->S;
    const bool f64 = ctx->prec == HOM_PREC_FP64;
    const size_t cs = f64 ? sizeof(double2) : sizeof(float2);
    const long long kv = f64 ? ctx->e64.g.kvec : ctx->e32.g.kvec;
    CU(cudaMalloc(&ctx->bspec, cs * n6 * nb));
    for (int i = 0; i < 3; ++i) CU(cudaMalloc(&ctx->bv[i], cs * kv * nb));
    for (int i = 0; i < 2; ++i) CU(cudaMalloc(&ctx->bw[i], cs * kv * nb));
    CU(cudaMalloc(&ctx->bx, cs * kv * nb));
    CU(cudaMalloc(&ctx->brhs, cs * n6 * nb));
    CU(cudaMalloc(&ctx->bb64, sizeof(double2) * n6 * nb));
    CU(cudaMalloc(&ctx->br64, sizeof(double2) * n6 * nb));
    CU(cudaMalloc(&ctx->d_bst, sizeof(MinresState) * nb));
    CU(cudaMallocHost(&ctx->h_bst, sizeof(MinresState) * nb));
    long long np = Launch<double>::ew_grid(n6);
    if (f64) {
        np = std::max(np, (long long)Launch<double>::x3_epart_grid(ctx->e64.g));
        np = std::max(np, (long long)Launch<double>::x1_lanczos_grid(ctx->e64.g));
    } else {
        np = std::max(np, (long long)Launch<float>::x3_epart_grid(ctx->e32.g));
        np = std::max(np, (long long)Launch<float>::x1_lanczos_grid(ctx->e32.g));
    }
    CU(cudaMalloc(&ctx->bpart, sizeof(double) * np * nb));
    CU(cudaMalloc(&ctx->bcnt, sizeof(int) * kFoldCounters));
    CU(cudaMemset(ctx->bcnt, 0, sizeof(int) * kFoldCounters));
    ctx->bcap = nb;
    return HOM_OK;
}

// Load cases per stacked batch: at most kNbMax and ncase, as many as fit
// in the free device memory (at least one).
static int batch_width(hom_ctx *ctx, int ncase) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const long long per = batch_case_bytes(ctx);
    const long long avail = (long long)(0.9 * (double)fr) + (long long)ctx->bcap * per;
    long long fit = per > 0 ? avail / per : 1;
    int nb = std::min(ncase, kNbMax);
    if (fit < nb) nb = (int)std::max(1LL, fit);
    return nb;
}

// One step of the fused chain for every case of the stacked batch (see the
// kernels in hom_passes.cuh), five launches: n2 inverse; n3 pass with the
// material law and the strain-energy sums; alpha (one CTA per case); n2
// forward; fused n1 pass (projector, Lanczos step, lagged w / x update,
// projector and inverse of u_{k+1}), whose last CTA takes the Givens step of
// every case.  Buffer roles as in capture_body.
template <typename R>
static void capture_bbody(hom_ctx *ctx, Engine<R> &E) {
    const Geometry &g = ctx->bg;
    const int nb = g.nb;
    cpx<R> *u3[3] = {(cpx<R> *)ctx->bv[0], (cpx<R> *)ctx->bv[1], (cpx<R> *)ctx->bv[2]};
    cpx<R> *wc = (cpx<R> *)ctx->bw[0], *wd = (cpx<R> *)ctx->bw[1];
    cpx<R> *x = (cpx<R> *)ctx->bx, *spec = (cpx<R> *)ctx->bspec;
    // the Givens step folded into the n1 pass (its last CTA sums one partial
    // per CTA of a persistent grid); alpha folded into the persistent
    // register n3 pass when HOM_FOLD_ALPHA=1 (one partial per CTA), else in
    // its own kernel (the fold measured within noise of it: 13.18 G
    // voxel-iterations/s either way at 256^3)
    const Fold fold{ctx->bcnt, ctx->d_bst, (double)ctx->V};
    const char *fa = std::getenv("HOM_FOLD_ALPHA");
    const bool fold_alpha = g.x3r && fa && std::atoi(fa) == 1;
    const Fold fold3 = fold_alpha ? Fold{ctx->bcnt, ctx->d_bst, (double)ctx->V} : Fold{nullptr, nullptr, 0.0};
    const int np3 = Launch<R>::x3_epart_grid(g);
    cudaStream_t s = ctx->stream;
    // step it of the body is step k = 1 + it (mod graph_iters, a multiple of
    // 6) of the sweep: u_k in bv[k mod 3] (u_{k+1} into the third buffer, so
    // that u_{k-1} stays readable for the lagged update), w by parity
    for (int it = 0; it < ctx->graph_iters; ++it) {
        const bool odd = (it % 2) == 0;
        cpx<R> *uk = u3[(it + 1) % 3], *um = u3[it % 3], *un = u3[(it + 2) % 3];
        cpx<R> *wa = odd ? wd : wc, *wb = odd ? wc : wd;
        Launch<R>::x2(g, s, 1, spec, ctx->d_bst);
        Launch<R>::x3(g, s, X3_IN_SPEC, spec, X3_MID_MATERIAL, ctx->lam, ctx->mu, nullptr, 1.0, X3_OUT_SPEC, spec,
                      E.phi, ctx->d_bst, ctx->bpart, fold3);
        if (!fold3.cnt) scalar_alpha(s, ctx->d_bst, ctx->bpart, np3, (double)ctx->V, g.nb, g.pdl);
        Launch<R>::x2(g, s, 0, spec, ctx->d_bst);
        Launch<R>::x1_lanczos(g, s, spec, uk, um, un, wa, wb, x, ctx->d_bst, ctx->bpart, fold);
        ctx->launches += fold3.cnt ? 4 : 5;
    }
}

// the stacked batch's solve graph for nb cases: a device-side WHILE loop
// over graph_iters steps, or (host_loop / no conditional nodes) the body
// alone, replayed by the host
// the stacked geometry for nb cases (own TMA cache: its tensor maps span nb
// cases); a change of nb drops the cell's stacked graph
template <typename R>
static void set_bgeom(hom_ctx *ctx, Engine<R> &E, int nb) {
    if (ctx->bg.nb == nb && ctx->bg.n1 == E.g.n1 && ctx->bg.mask0 == E.g.mask0 && (ctx->btma || !E.g.tma)) return;
    if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
    ctx->bgraph = nullptr;
    ctx->bgraph_nb = 0;
    tma_cache_free(ctx->btma);
    ctx->btma = E.g.tma ? tma_cache_new() : nullptr;
    ctx->bg = E.g;
    ctx->bg.nb = nb;
    ctx->bg.tma_cache = ctx->btma;
    ctx->bg.pdl = ctx->pdl;
}

template <typename R>
static int build_bgraph(hom_ctx *ctx, Engine<R> &E, int nb) {
    set_bgeom<R>(ctx, E, nb);
    if (ctx->bgraph && ctx->bgraph_nb == nb) return HOM_OK;
    const long long before = ctx->launches;
    cudaGraph_t graph = nullptr;
    bool loops = false;
    if (!ctx->host_loop && cudaGraphCreate(&graph, 0) == cudaSuccess) {
        cudaGraphConditionalHandle h;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        cudaGraphNode_t node;
        if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess) {
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess) {
                cudaGraph_t body = np.conditional.phGraph_out[0];
                CU(cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
                capture_bbody<R>(ctx, E);
                loop_cond(ctx->stream, h, ctx->d_bst, nb);
                ctx->launches += 1;
                cudaError_t e = cudaStreamEndCapture(ctx->stream, &body);
                if (e != cudaSuccess) {
                    cudaGraphDestroy(graph);
                    return fail(ctx, HOM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
                }
                loops = true;
            }
        }
        if (!loops) {
            cudaGetLastError();
            cudaGraphDestroy(graph);
            graph = nullptr;
        }
    }
    if (!loops) {
        CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        capture_bbody<R>(ctx, E);
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
        if (e != cudaSuccess) return fail(ctx, HOM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    ctx->bgraph_kernels = ctx->launches - before;
    ctx->launches = before;
    cudaError_t e = cudaGraphInstantiate(&ctx->bgraph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, HOM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    ctx->bgraph_loops = loops;
    ctx->bgraph_nb = nb;
    return HOM_OK;
}

// MINRES from a zero start on the nb stacked right-hand sides in ctx->brhs
// (standard order, solve precision); case j runs with tolerance tol[j] and
// at most maxit[j] iterations (0: the case sits this sweep out).  In three
// parts so that several cells can share one graph launch:
//   batch_begin  per-case norms and FP64 states, Krylov vectors in tile
//                order, the first inverse n1 transform; *any = some case runs
//   (the stacked graph, see build_bgraph / hom_solve_batch)
//   batch_end    the last lagged update, the iterates back in the standard
//                order over ctx->brhs (zero for cases that did not run), and
//                the per-case iterations, estimated residual and status.
template <typename R>
static int batch_begin(hom_ctx *ctx, Engine<R> &E, int nb, const double *tol, const int *maxit, int max_bodies,
                       bool *any) {
    cudaStream_t s = ctx->stream;
    const long long n6 = 6 * ctx->S, kv = E.g.kvec;
    const int npe = Launch<R>::ew_grid(n6);
    cpx<R> *rhs = (cpx<R> *)ctx->brhs, *spec = (cpx<R> *)ctx->bspec;
    for (int j = 0; j < nb; ++j) {
        Launch<R>::norm2w(E.g, s, rhs + j * n6, ctx->bpart + (size_t)j * npe);
        scalar_start(s, ctx->d_bst + j, ctx->bpart + (size_t)j * npe, npe, tol[j], maxit[j], max_bodies);
    }
    ctx->launches += 2 * nb;
    CU(cudaMemcpyAsync(ctx->h_bst, ctx->d_bst, sizeof(MinresState) * nb, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *any = false;
    for (int j = 0; j < nb; ++j) *any = *any || !ctx->h_bst[j].done;
    CU(cudaMemsetAsync(ctx->bx, 0, sizeof(cpx<R>) * kv * nb, s));
    if (!*any) return HOM_OK;
    // the folded scalar steps' counters start at zero (each last CTA resets
    // its own; this also clears any left by a sweep that stopped on an error)
    CU(cudaMemsetAsync(ctx->bcnt, 0, sizeof(int) * kFoldCounters, s));
    // u_0 = 0, u_1 = rhs (= beta_1 v_1), w_0 = w_{-1} = 0, in tile order; the
    // work spectrum enters each step holding F_1^-1 G u_k
    CU(cudaMemsetAsync(ctx->bv[0], 0, sizeof(cpx<R>) * kv * nb, s));
    CU(cudaMemsetAsync(ctx->bv[1], 0, sizeof(cpx<R>) * kv * nb, s));
    CU(cudaMemsetAsync(ctx->bv[2], 0, sizeof(cpx<R>) * kv * nb, s));
    CU(cudaMemsetAsync(ctx->bw[0], 0, sizeof(cpx<R>) * kv * nb, s));
    CU(cudaMemsetAsync(ctx->bw[1], 0, sizeof(cpx<R>) * kv * nb, s));
    for (int j = 0; j < nb; ++j) {
        if (ctx->h_bst[j].done) continue;
        Launch<R>::to_tiles(E.g, s, rhs + j * n6, (cpx<R> *)ctx->bv[1] + j * kv);
        Launch<R>::x1(E.g, s, X1_GAMMA_IN, rhs + j * n6, spec + j * n6, nullptr, nullptr, nullptr);
        ctx->launches += 2;
    }
    return HOM_OK;
}

template <typename R>
static int batch_end(hom_ctx *ctx, Engine<R> &E, int nb, const int *maxit, bool ran, int *its, double *est, int *st) {
    cudaStream_t s = ctx->stream;
    const long long n6 = 6 * ctx->S, kv = E.g.kvec;
    cpx<R> *rhs = (cpx<R> *)ctx->brhs;
    if (ran) {
        Launch<R>::minres_flush(ctx->bg, s, (const cpx<R> *)ctx->bv[0], (const cpx<R> *)ctx->bv[1],
                                (const cpx<R> *)ctx->bv[2], (cpx<R> *)ctx->bw[0], (cpx<R> *)ctx->bw[1], (cpx<R> *)ctx->bx, ctx->d_bst, kv);
        ctx->launches += 1;
    }
    for (int j = 0; j < nb; ++j) Launch<R>::from_tiles(E.g, s, (const cpx<R> *)ctx->bx + j * kv, rhs + j * n6);
    ctx->launches += nb;
    CU(cudaMemcpyAsync(ctx->h_bst, ctx->d_bst, sizeof(MinresState) * nb, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (int j = 0; j < nb; ++j) {
        const MinresState &h = ctx->h_bst[j];
        its[j] = h.k;
        est[j] = h.est;
        st[j] = !std::isfinite(h.beta1) || h.status == -5 ? HOM_ENAN : (h.status == 1 ? HOM_NOT_CONVERGED : HOM_OK);
        if (maxit[j] <= 0 || h.beta1 == 0.0) est[j] = 0.0;
    }
    return HOM_OK;
}

// the stacked graph of one cell, launched until its states are done
template <typename R>
static int batch_launch(hom_ctx *ctx, Engine<R> &E, int nb, int max_bodies) {
    cudaStream_t s = ctx->stream;
    int rc = build_bgraph<R>(ctx, E, nb);
    if (rc) return rc;
    if (ctx->bgraph_loops) {
        CU(cudaGraphLaunch(ctx->bgraph, s));
        CU(cudaMemcpyAsync(ctx->h_bst, ctx->d_bst, sizeof(MinresState), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        ctx->launches += (long long)ctx->h_bst[0].bodies * ctx->bgraph_kernels;
        return HOM_OK;
    }
    const int per_check = 4;
    int replays = 0;
    while (true) {
        for (int r = 0; r < per_check && replays < max_bodies; ++r, ++replays) {
            CU(cudaGraphLaunch(ctx->bgraph, s));
            ctx->launches += ctx->bgraph_kernels;
        }
        CU(cudaMemcpyAsync(ctx->h_bst, ctx->d_bst, sizeof(MinresState) * nb, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        bool live = false;
        for (int j = 0; j < nb; ++j) live = live || !ctx->h_bst[j].done;
        if (!live || replays >= max_bodies) break;
    }
    return HOM_OK;
}

// graph bodies for a sweep with iteration cap mx
static int max_bodies_for(const hom_ctx *ctx, int mx) { return (mx + ctx->graph_iters - 1) / ctx->graph_iters + 1; }

// ----- solve -------------------------------------------------------------------
// ||A^ x - b^||_w / ||b^||_w in FP64 (Parseval: the real-space ratio of
// eq. (galres)); leaves b^ - A^ x in r64.
// r = b - A^ x in FP64 and |r| / |b|.  With tau (elastic Galerkin operator
// only), also the mean over the voxels of the stress phi C_m : eps~ formed by
// its n3 pass, eps~ = F^-1 G x: with the constant part this is the mean stress
// of the solution x (tau[c], Mandel, units of E), taken here instead of in a
// separate pass over the spectrum.
static int true_residual(hom_ctx *ctx, const double2 *x, const double2 *b, double2 *r, double bnorm, double *res,
                         double *tau = nullptr) {
    const bool ts = tau && !ctx->tangent_op;
    op_spec<double>(ctx, ctx->e64, x, r, false, nullptr, nullptr, ts ? ctx->tsum_part : nullptr);
    spec_residual64(ctx->e64.g, ctx->stream, b, r, r, ctx->partials);
    reduce_to(ctx->stream, ctx->partials, ew_blocks(6 * ctx->S), ctx->d_scalar);
    ctx->launches += 2;
    if (ts) {
        const int n3 = Launch<double>::x3_grid(ctx->e64.g);
        for (int c = 0; c < 6; ++c) reduce_to(ctx->stream, ctx->tsum_part + (size_t)c * n3, n3, ctx->d_scalar + 1 + c);
        ctx->launches += 6;
    }
    CU(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, (ts ? 7 : 1) * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *res = (bnorm > 0) ? std::sqrt(*ctx->h_scalar) / bnorm : 0.0;
    if (ts)
        for (int c = 0; c < 6; ++c) tau[c] = ctx->h_scalar[1 + c] / (double)ctx->V;
    return HOM_OK;
}

// real FP64 fluctuation strain of case icase (Mandel) into ctx->r64 (as 6 V doubles):
// Galerkin: F^-1 G x^;  MoDBFFT: F^-1 sym(u^ (x) xi)
static double *fluctuation64(hom_ctx *ctx, int icase) {
    double *eps = (double *)ctx->r64;
    if (ctx->solver == HOM_SOLVER_MODBFFT_CG) {
        Launch<double>::modb_expand(ctx->e64.g, ctx->stream, 0.0, 0, ctx->x64[icase], ctx->e64.spec, 6, nullptr);
        ctx->launches += 1;
        spec_to_real<double>(ctx, ctx->e64, ctx->e64.spec, false, 1.0, eps);
    } else {
        spec_to_real<double>(ctx, ctx->e64, ctx->x64[icase], true, 1.0, eps);
    }
    return eps;
}

// MoDBFFT solve of one case (section 2.2): FP64 right-hand side and true
// residual of eq. (modbfftresres); PCG sweeps in the field precision,
// refined against the FP64 residual.
static int solve_case_modb(hom_ctx *ctx, int icase, const double *m, double tol, int max_it, double2 *x,
                           hom_solve_info *inf, int *status_out) {
    const long long nc3 = 3 * ctx->S;   // complex values per displacement spectrum
    cudaStream_t s = ctx->stream;
    rhs_modb<double>(ctx, ctx->e64, m, ctx->b64);
    Launch<double>::norm2w(ctx->e64.g, s, ctx->b64, ctx->partials, 3);
    reduce_to(s, ctx->partials, ew_blocks(3 * ctx->S), ctx->d_scalar);
    ctx->launches += 2;
    CU(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaMemsetAsync(x, 0, sizeof(double2) * nc3, s));
    CU(cudaStreamSynchronize(s));
    const double bnorm = std::sqrt(*ctx->h_scalar);
    // scale of the right-hand side: ||C : E_bar|| max|xi| sqrt(V) (Parseval)
    double ce2 = 0.0;
    for (int i = 0; i < 6; ++i) {
        double sv = 2.0 * ctx->mu * m[i] + (i < 3 ? ctx->lam * (m[0] + m[1] + m[2]) : 0.0);
        ce2 += sv * sv;
    }
    const double nmax = std::max(ctx->n[0], std::max(ctx->n[1], ctx->n[2]));
    const double scale = std::sqrt(ce2 * ctx->phi2_sum * (double)ctx->V) * 3.14159265358979323846 * nmax;
    int status = HOM_OK;
    if (!std::isfinite(bnorm)) {
        *status_out = HOM_ENAN;
        return HOM_OK;
    }
    if (bnorm <= kRhsZero * scale) {
        inf->sweeps = 0;
        *status_out = HOM_OK;
        return HOM_OK;
    }
    auto residual = [&](double *res) -> int {
        op_modb<double>(ctx, ctx->e64, x, ctx->r64, nullptr, nullptr, nullptr);
        spec_residual64(ctx->e64.g, s, ctx->b64, ctx->r64, ctx->r64, ctx->partials, 3);
        reduce_to(s, ctx->partials, ew_blocks(3 * ctx->S), ctx->d_scalar);
        ctx->launches += 2;
        CU(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        *res = std::sqrt(*ctx->h_scalar) / bnorm;
        return HOM_OK;
    };
    double tres = 1.0;   // x = 0: r = b
    CU(cudaMemcpyAsync(ctx->r64, ctx->b64, sizeof(double2) * nc3, cudaMemcpyDeviceToDevice, s));
    int rc = HOM_OK;
    // FP32 fields: sweeps share the iteration budget; a sweep that raised the
    // FP64 true residual is taken back and ends the solve
    const int sweeps_max = (ctx->prec == HOM_PREC_FP64) ? 1 : 1 + ctx->refine;
    int budget = max_it;
    for (int sw = 0; sw < sweeps_max && tres > tol && budget > 0; ++sw) {
        double sweep_tol = tol / tres;
        if (sweep_tol > 0.5) sweep_tol = 0.5;
        if (ctx->prec == HOM_PREC_FP32_FIELDS && sweep_tol < ctx->sweep_floor) sweep_tol = ctx->sweep_floor;
        int it = 0, st = 0;
        double est = 0.0;
        if (ctx->prec == HOM_PREC_FP64) {
            CU(cudaMemcpyAsync(ctx->rhs, ctx->r64, sizeof(double2) * nc3, cudaMemcpyDeviceToDevice, s));
            rc = run_cg<double>(ctx, ctx->e64, sweep_tol, budget, &it, &est, &st);
            if (rc) return rc;
            Launch<double>::axpby(2 * nc3, s, 1.0, (const double *)ctx->xs, 1.0, (double *)x);
        } else {
            spec_d2f(nc3, s, ctx->r64, (float2 *)ctx->rhs);
            rc = run_cg<float>(ctx, ctx->e32, sweep_tol, budget, &it, &est, &st);
            if (rc) return rc;
            spec_f2d_acc(nc3, s, (const float2 *)ctx->xs, x);
        }
        ctx->launches += 2;
        budget -= it;
        inf->iterations += it;
        inf->est_residual = est * tres;
        inf->sweeps = sw + 1;
        const double prev = tres;
        rc = residual(&tres);
        if (rc) return rc;
        if (st == HOM_ENAN) { status = HOM_ENAN; break; }
        if (ctx->prec == HOM_PREC_FP32_FIELDS && !(tres < prev)) {
            spec_f2d_acc(nc3, s, (const float2 *)ctx->xs, x, -1.0);
            ctx->launches += 1;
            rc = residual(&tres);
            if (rc) return rc;
            status = HOM_NOT_CONVERGED;
            break;
        }
        if (st == HOM_NOT_CONVERGED && tres > tol && ctx->prec == HOM_PREC_FP64) { status = HOM_NOT_CONVERGED; break; }
    }
    inf->true_residual = tres;
    if (status == HOM_OK && tres > tol) status = HOM_NOT_CONVERGED;
    *status_out = status;
    return HOM_OK;
}

// mean stress <phi C_m : (E_bar + e~)> in FP64, timing, info record
static int finish_case(hom_ctx *ctx, int icase, const double *m, double2 *x, hom_solve_info *inf, int status,
                       hom_solve_info *info, const double *tau = nullptr) {
    cudaStream_t s = ctx->stream;
    const double r2 = std::sqrt(2.0);
    double sig[6];
    if (ctx->solver != HOM_SOLVER_MODBFFT_CG && tau) {
        // <sigma> = phibar C_m : E_bar + <phi C_m : eps~>, the second term from
        // the n3 pass of the last true residual (taken on this x)
        const double trE = m[0] + m[1] + m[2];
        for (int c = 0; c < 6; ++c)
            sig[c] = ctx->phibar * ((c < 3 ? ctx->lam * trE : 0.0) + 2.0 * ctx->mu * m[c]) + tau[c];
        CU(cudaEventRecord(ctx->ev1, s));
        CU(cudaEventSynchronize(ctx->ev1));
    } else if (ctx->solver != HOM_SOLVER_MODBFFT_CG) {
        // <sigma> = phibar C_m : E_bar + C_m : <phi eps~>, with <phi eps~> by
        // Parseval from phi^ and the projected spectrum: one point-wise pass
        const int nb = Launch<double>::phi_dot(ctx->e64.g, s, x, ctx->phihat, ctx->partials);
        for (int c = 0; c < 6; ++c) reduce_to(s, ctx->partials + c * nb, nb, ctx->d_scalar + c);
        ctx->launches += 7;
        CU(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaEventRecord(ctx->ev1, s));
        CU(cudaStreamSynchronize(s));
        const double VV = (double)ctx->V * (double)ctx->V;
        double mf[6];
        for (int c = 0; c < 6; ++c) mf[c] = ctx->h_scalar[c] / VV;
        const double trE = m[0] + m[1] + m[2], trF = mf[0] + mf[1] + mf[2];
        for (int c = 0; c < 6; ++c)
            sig[c] = ctx->phibar * ((c < 3 ? ctx->lam * trE : 0.0) + 2.0 * ctx->mu * m[c]) +
                     (c < 3 ? ctx->lam * trF : 0.0) + 2.0 * ctx->mu * mf[c];
    } else {
        const double *eps = fluctuation64(ctx, icase);
        mean_stress64(ctx->V, s, eps, ctx->e64.phi, ctx->lam, ctx->mu, m, ctx->partials);
        const int nb = ew_blocks(ctx->V);
        for (int c = 0; c < 6; ++c) reduce_to(s, ctx->partials + c * nb, nb, ctx->d_scalar + c);
        ctx->launches += 7;
        CU(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaEventRecord(ctx->ev1, s));
        CU(cudaStreamSynchronize(s));
        for (int c = 0; c < 6; ++c) sig[c] = ctx->h_scalar[c] / (double)ctx->V;
    }
    for (int c = 0; c < 6; ++c) {
        double v = sig[c] * ctx->E;
        if (c >= 3) v /= r2;
        inf->sigma_mean[c] = v;
        ctx->sig_mean[6 * icase + c] = v;
    }
    // mean strain: the prescribed components, plus x^(0) / V (the solved mean)
    // on the stress-controlled ones, which the projector keeps at xi = 0
    double em[6];
    for (int c = 0; c < 6; ++c) em[c] = m[c];
    const int mask = ctx->e64.g.mask0;
    if (mask && ctx->solver != HOM_SOLVER_MODBFFT_CG) {
        double2 x0[6];
        CU(cudaMemcpyAsync(x0, x, sizeof(x0), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        for (int c = 0; c < 6; ++c)
            if ((mask >> c) & 1) em[c] += x0[c].x / (double)ctx->V;
    }
    for (int c = 0; c < 6; ++c) {
        ctx->eps_means[6 * icase + c] = em[c];
        inf->eps_mean[c] = (c >= 3) ? em[c] / r2 : em[c];
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    inf->time_ms = ms;
    inf->status = status;
    if (info) *info = *inf;
    return status;
}

// One load case.  sbar_t: prescribed mean stress (tensor components, same
// units as E) of the stress-controlled components in ctx->e64.g.mask0, or
// nullptr for pure strain control.
static int solve_case(hom_ctx *ctx, int icase, const double *mac_t, const double *sbar_t, double tol, int max_it,
                      const void *warm, hom_solve_info *info) {
    const long long nc = 6 * ctx->S;   // complex values per spectral vector
    cudaStream_t s = ctx->stream;
    const int mask = ctx->e64.g.mask0;
    double m[6], sbar_v[6] = {0, 0, 0, 0, 0, 0};
    macro_to_mandel(mac_t, m);
    if (mask) {
        double sb[6];
        macro_to_mandel(sbar_t, sb);
        for (int c = 0; c < 6; ++c) {
            if ((mask >> c) & 1) {
                m[c] = 0.0;                                   // an unknown, not a load
                sbar_v[c] = (double)ctx->V * sb[c] / ctx->E;  // F{sigma_bar} at xi = 0, units of E
            }
        }
    }
    for (int c = 0; c < 6; ++c) ctx->macros[6 * icase + c] = m[c];
    double2 *x = ctx->x64[icase];
    hom_solve_info inf{};
    CU(cudaEventRecord(ctx->ev0, s));
    if (ctx->solver == HOM_SOLVER_MODBFFT_CG) {
        if (warm) return fail(ctx, HOM_EINVAL, "warm starts are for the Galerkin solver");
        int status = HOM_OK;
        int rc = solve_case_modb(ctx, icase, m, tol, max_it, x, &inf, &status);
        if (rc) return rc;
        return finish_case(ctx, icase, m, x, &inf, status, info);
    }
    {
        // F{C : E_bar} = phi^ (C_m : E_bar): one point-wise FP64 pass
        double tau[6];
        const double tr = m[0] + m[1] + m[2];
        for (int c = 0; c < 6; ++c) tau[c] = (c < 3 ? ctx->lam * tr : 0.0) + 2.0 * ctx->mu * m[c];
        Launch<double>::rhs_phihat(ctx->e64.g, s, ctx->phihat, tau, mask ? sbar_v : nullptr, ctx->b64);
        ctx->launches += 1;
    }
    double b2 = 0.0;
    int rc = spec_norm2<double>(ctx, ctx->e64, ctx->b64, &b2);
    if (rc) return rc;
    const double bnorm = std::sqrt(b2);
    // scale of the right-hand side: ||C : E_bar|| over the grid (units of E);
    // Parseval: ||b||_real = ||b^||_w / sqrt(V)
    double ce2 = 0.0;
    for (int i = 0; i < 6; ++i) {
        double sv = 2.0 * ctx->mu * m[i] + (i < 3 ? ctx->lam * (m[0] + m[1] + m[2]) : 0.0);
        ce2 += sv * sv;
    }
    // plus ||sigma_bar_KL|| over the grid for stress-controlled components
    double s2 = 0.0;
    for (int c = 0; c < 6; ++c) s2 += sbar_v[c] * sbar_v[c];
    const double ntau = std::sqrt(ce2 * ctx->phi2_sum) + std::sqrt(s2 / (double)ctx->V);
    CU(cudaMemsetAsync(x, 0, sizeof(double2) * nc, s));
    int status = HOM_OK;
    if (!std::isfinite(bnorm)) {
        status = HOM_ENAN;
    } else if (bnorm / std::sqrt((double)ctx->V) <= kRhsZero * ntau) {
        // b vanishes up to round-off: zero fluctuation, 0 iterations
        inf.sweeps = 0;
    } else {
        double tres = 1.0;
        const long long n = 6 * ctx->V;
        if (warm && ctx->prec == HOM_PREC_FP64) {
            // x0 = G F (warm), tensor components -> Mandel, projected; FP64 residual
            double *st = (double *)ctx->r64;
            rc = stage_in(ctx, (const char *)warm + sizeof(double) * n * icase, sizeof(double) * n, st);
            if (rc) return rc;
            mandel_scale64(ctx->V, s, st, std::sqrt(2.0));
            real_to_spec<double>(ctx, ctx->e64, st, X3_MID_NONE, true, x);
            ctx->launches += 2;
            rc = true_residual(ctx, x, ctx->b64, ctx->r64, bnorm, &tres);
            if (rc) return rc;
        } else if (warm) {
            // FP32 fields: the projection and the residual that starts the
            // first FP32 sweep are FP32 operator applications (an FP64 pass is
            // many times slower on this part); the FP64 true residual after
            // the sweep still decides convergence.  An FP32 residual carries
            // round-off of about 1e-7 of b, so a start already that close is
            // measured with the FP64 operator instead.
            float *wr = (float *)ctx->xs;
            cpx<float> *x32 = (cpx<float> *)ctx->vbuf[0], *p32 = (cpx<float> *)ctx->vbuf[1];
            rc = stage_in(ctx, (const char *)warm + sizeof(float) * n * icase, sizeof(float) * n, wr);
            if (rc) return rc;
            Launch<float>::axpby(3 * ctx->V, s, std::sqrt(2.0), wr + 3 * ctx->V, 0.0, wr + 3 * ctx->V);
            real_to_spec<float>(ctx, ctx->e32, wr, X3_MID_NONE, true, x32);
            spec_f2d_acc(nc, s, x32, x);
            op_spec<float>(ctx, ctx->e32, x32, p32, false, nullptr, nullptr);
            spec_residual_mixed(ctx->e64.g, s, ctx->b64, p32, ctx->r64, ctx->partials);
            reduce_to(s, ctx->partials, ew_blocks(6 * ctx->S), ctx->d_scalar);
            ctx->launches += 5;
            CU(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            tres = std::sqrt(*ctx->h_scalar) / bnorm;
            if (tres < kWarmFp64Below) {
                rc = true_residual(ctx, x, ctx->b64, ctx->r64, bnorm, &tres);
                if (rc) return rc;
            }
        } else {   // x = 0: r = b
            CU(cudaMemcpyAsync(ctx->r64, ctx->b64, sizeof(double2) * nc, cudaMemcpyDeviceToDevice, s));
        }
        const int sweeps_max = (ctx->prec == HOM_PREC_FP64) ? 1 : 1 + ctx->refine;
        for (int sw = 0; sw < sweeps_max && tres > tol; ++sw) {
            // relative reduction this sweep must reach; FP32 fields cannot
            // resolve residuals much below 1e-6 of their right-hand side, so a
            // sweep never asks for less and the next sweep refines further
            double sweep_tol = (ctx->prec == HOM_PREC_FP32_FIELDS ? kSweepTarget : 1.0) * tol / tres;
            if (sweep_tol > 0.5) sweep_tol = 0.5;
            double floor = (sw == 0 && !warm && ctx->sweep_floor == kFp32SweepFloor)
                               ? kFp32FirstSweepFloor : ctx->sweep_floor;
            if (mask && ctx->sweep_floor == kFp32SweepFloor)
                floor = sw == 0 ? kFp32MixedSweepFloor : kFp32MixedLaterSweepFloor;
            if (ctx->prec == HOM_PREC_FP32_FIELDS && sweep_tol < floor) sweep_tol = floor;
            int it = 0, st = 0;
            double est = 0.0;
            if (ctx->prec == HOM_PREC_FP64) {
                CU(cudaMemcpyAsync(ctx->rhs, ctx->r64, sizeof(double2) * nc, cudaMemcpyDeviceToDevice, s));
                rc = run_krylov<double>(ctx, ctx->e64, sweep_tol, max_it, &it, &est, &st);
                if (rc) return rc;
                Launch<double>::axpby(2 * nc, s, 1.0, (const double *)ctx->xs, 1.0, (double *)x);
            } else {
                spec_d2f(nc, s, ctx->r64, (float2 *)ctx->rhs);
                rc = run_krylov<float>(ctx, ctx->e32, sweep_tol, max_it, &it, &est, &st);
                if (rc) return rc;
                spec_f2d_acc(nc, s, (const float2 *)ctx->xs, x);
            }
            ctx->launches += 2;
            inf.iterations += it;
            inf.est_residual = est * tres;     // relative to ||b||
            inf.sweeps = sw + 1;
            const double prev = tres;
            rc = true_residual(ctx, x, ctx->b64, ctx->r64, bnorm, &tres);
            if (rc) return rc;
            if (st == HOM_ENAN) { status = HOM_ENAN; break; }
            if (ctx->prec == HOM_PREC_FP32_FIELDS && !(tres < prev)) {
                // an FP32 sweep past the accuracy FP32 fields can carry (seen
                // under stress control): take it back and stop
                spec_f2d_acc(nc, s, (const float2 *)ctx->xs, x, -1.0);
                ctx->launches += 1;
                rc = true_residual(ctx, x, ctx->b64, ctx->r64, bnorm, &tres);
                if (rc) return rc;
                status = HOM_NOT_CONVERGED;
                break;
            }
            if (st == HOM_NOT_CONVERGED && tres > tol) { status = HOM_NOT_CONVERGED; break; }
        }
        inf.true_residual = tres;
        if (status == HOM_OK && tres > tol) status = HOM_NOT_CONVERGED;
    }
    return finish_case(ctx, icase, m, x, &inf, status, info);
}

// Galerkin-MINRES of the load cases [c0, c0 + nb) of one cell as one stacked
// batch: per case the FP64 right-hand side (from the DFT of phi) and, for a
// warm start, the projected start and its residual; then refinement sweeps
// in which every case still above tol runs MINRES in the same stacked
// launches on its FP64 residual (converted to the field precision), and the
// FP64 true residual of each case decides whether it needs another sweep.
// The sweep rules are those of a single case (solve_case).  In phases, so
// that hom_solve_batch can run the sweeps of several cells in one graph
// launch.  info[].time_ms is the device time of the whole batch.
struct Chunk {
    hom_ctx *ctx = nullptr;
    int c0 = 0, nb = 0;
    const double *macro_strain = nullptr, *macro_stress = nullptr;
    double tol = 0.0;
    int max_it = 0;
    const void *warm = nullptr;
    hom_solve_info *info = nullptr;
    int sw = 0;             // sweeps begun
    bool ran = false;       // the current sweep has a case that runs
    std::vector<double> M, bnorm, tres, stol, est;
    std::vector<int> status, live, solvable, mi, its, sts;
    std::vector<hom_solve_info> inf;
    // per case: the mean of phi C_m : eps~ at the last true residual (tau_ok:
    // taken on the current x)
    std::vector<double> tau;
    std::vector<int> tau_ok;
};

static int chunk_prepare(Chunk &ch) {
    hom_ctx *ctx = ch.ctx;
    const int nb = ch.nb;
    const long long nc = 6 * ctx->S;
    cudaStream_t s = ctx->stream;
    const int mask = ctx->e64.g.mask0;
    const bool f32 = ctx->prec == HOM_PREC_FP32_FIELDS;
    int rc = batch_reserve(ctx, nb);
    if (rc) return rc;
    ch.M.assign(6 * nb, 0.0);
    ch.bnorm.assign(nb, 0.0);
    ch.tres.assign(nb, 1.0);
    ch.stol.assign(nb, 0.5);
    ch.est.assign(nb, 0.0);
    ch.status.assign(nb, HOM_OK);
    ch.live.assign(nb, 0);
    ch.solvable.assign(nb, 0);
    ch.mi.assign(nb, 0);
    ch.its.assign(nb, 0);
    ch.sts.assign(nb, 0);
    ch.inf.assign(nb, hom_solve_info{});
    ch.tau.assign(6 * nb, 0.0);
    ch.tau_ok.assign(nb, 0);
    ch.sw = 0;
    CU(cudaEventRecord(ctx->ev0, s));
    for (int j = 0; j < nb; ++j) {
        const int k = ch.c0 + j;
        double *m = &ch.M[6 * j];
        double sbar_v[6] = {0, 0, 0, 0, 0, 0};
        macro_to_mandel(ch.macro_strain + 6 * k, m);
        if (mask) {
            double sb[6];
            macro_to_mandel(ch.macro_stress + 6 * k, sb);
            for (int c = 0; c < 6; ++c) {
                if ((mask >> c) & 1) {
                    m[c] = 0.0;                                   // an unknown, not a load
                    sbar_v[c] = (double)ctx->V * sb[c] / ctx->E;  // F{sigma_bar} at xi = 0, units of E
                }
            }
        }
        for (int c = 0; c < 6; ++c) ctx->macros[6 * k + c] = m[c];
        double2 *b = ctx->bb64 + j * nc, *r = ctx->br64 + j * nc, *x = ctx->x64[k];
        {   // F{C : E_bar} = phi^ (C_m : E_bar): one point-wise FP64 pass
            double tau[6];
            const double tr = m[0] + m[1] + m[2];
            for (int c = 0; c < 6; ++c) tau[c] = (c < 3 ? ctx->lam * tr : 0.0) + 2.0 * ctx->mu * m[c];
            Launch<double>::rhs_phihat(ctx->e64.g, s, ctx->phihat, tau, mask ? sbar_v : nullptr, b);
            ctx->launches += 1;
        }
        double b2 = 0.0;
        rc = spec_norm2<double>(ctx, ctx->e64, b, &b2);
        if (rc) return rc;
        ch.bnorm[j] = std::sqrt(b2);
        double ce2 = 0.0;
        for (int i = 0; i < 6; ++i) {
            const double sv = 2.0 * ctx->mu * m[i] + (i < 3 ? ctx->lam * (m[0] + m[1] + m[2]) : 0.0);
            ce2 += sv * sv;
        }
        double s2 = 0.0;
        for (int c = 0; c < 6; ++c) s2 += sbar_v[c] * sbar_v[c];
        const double ntau = std::sqrt(ce2 * ctx->phi2_sum) + std::sqrt(s2 / (double)ctx->V);
        CU(cudaMemsetAsync(x, 0, sizeof(double2) * nc, s));
        if (!std::isfinite(ch.bnorm[j])) {
            ch.status[j] = HOM_ENAN;
            continue;
        }
        if (ch.bnorm[j] / std::sqrt((double)ctx->V) <= kRhsZero * ntau) {
            ch.inf[j].sweeps = 0;   // b vanishes up to round-off: zero fluctuation, 0 iterations
            ch.tau_ok[j] = 1;       // x = 0: no fluctuation stress
            continue;
        }
        ch.live[j] = 1;
        ch.solvable[j] = 1;
        const long long n = 6 * ctx->V;
        if (ch.warm && !f32) {
            // x0 = G F (warm), tensor components -> Mandel, projected; FP64 residual
            double *st = (double *)ctx->r64;
            rc = stage_in(ctx, (const char *)ch.warm + sizeof(double) * n * k, sizeof(double) * n, st);
            if (rc) return rc;
            mandel_scale64(ctx->V, s, st, std::sqrt(2.0));
            real_to_spec<double>(ctx, ctx->e64, st, X3_MID_NONE, true, x);
            ctx->launches += 2;
            rc = true_residual(ctx, x, b, r, ch.bnorm[j], &ch.tres[j], &ch.tau[6 * j]);
            if (rc) return rc;
            ch.tau_ok[j] = 1;
        } else if (ch.warm) {
            // FP32 fields: projection and starting residual with the FP32
            // operator; a start already within kWarmFp64Below gets the FP64 one
            float *wr = (float *)ctx->xs;
            cpx<float> *x32 = (cpx<float> *)ctx->vbuf[0], *p32 = (cpx<float> *)ctx->vbuf[1];
            rc = stage_in(ctx, (const char *)ch.warm + sizeof(float) * n * k, sizeof(float) * n, wr);
            if (rc) return rc;
            Launch<float>::axpby(3 * ctx->V, s, std::sqrt(2.0), wr + 3 * ctx->V, 0.0, wr + 3 * ctx->V);
            real_to_spec<float>(ctx, ctx->e32, wr, X3_MID_NONE, true, x32);
            spec_f2d_acc(nc, s, x32, x);
            op_spec<float>(ctx, ctx->e32, x32, p32, false, nullptr, nullptr);
            spec_residual_mixed(ctx->e64.g, s, b, p32, r, ctx->partials);
            reduce_to(s, ctx->partials, ew_blocks(6 * ctx->S), ctx->d_scalar);
            ctx->launches += 5;
            CU(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            ch.tres[j] = std::sqrt(*ctx->h_scalar) / ch.bnorm[j];
            if (ch.tres[j] < kWarmFp64Below) {
                rc = true_residual(ctx, x, b, r, ch.bnorm[j], &ch.tres[j], &ch.tau[6 * j]);
                if (rc) return rc;
                ch.tau_ok[j] = 1;
            }
        } else {   // x = 0: r = b
            CU(cudaMemcpyAsync(r, b, sizeof(double2) * nc, cudaMemcpyDeviceToDevice, s));
        }
    }
    return HOM_OK;
}

// the next sweep's tolerances and right-hand sides and the start of its
// stacked MINRES; *more = false when no case needs a sweep (or the sweeps
// ran out)
static int chunk_sweep_begin(Chunk &ch, bool *more) {
    hom_ctx *ctx = ch.ctx;
    const long long nc = 6 * ctx->S;
    cudaStream_t s = ctx->stream;
    const int mask = ctx->e64.g.mask0;
    const bool f32 = ctx->prec == HOM_PREC_FP32_FIELDS;
    const int sweeps_max = f32 ? 1 + ctx->refine : 1;
    *more = false;
    ch.ran = false;
    if (ch.sw >= sweeps_max) return HOM_OK;
    const int sw = ch.sw;
    double floor = (sw == 0 && !ch.warm && ctx->sweep_floor == kFp32SweepFloor) ? kFp32FirstSweepFloor : ctx->sweep_floor;
    if (mask && ctx->sweep_floor == kFp32SweepFloor) floor = sw == 0 ? kFp32MixedSweepFloor : kFp32MixedLaterSweepFloor;
    bool any = false;
    for (int j = 0; j < ch.nb; ++j) {
        ch.mi[j] = 0;
        ch.stol[j] = 0.5;
        if (!ch.live[j] || !(ch.tres[j] > ch.tol)) continue;
        double sweep_tol = (f32 ? kSweepTarget : 1.0) * ch.tol / ch.tres[j];
        if (sweep_tol > 0.5) sweep_tol = 0.5;
        if (f32 && sweep_tol < floor) sweep_tol = floor;
        ch.stol[j] = sweep_tol;
        ch.mi[j] = ch.max_it;
        any = true;
        const double2 *r = ctx->br64 + j * nc;
        if (f32) spec_d2f(nc, s, r, (float2 *)ctx->brhs + j * nc);
        else CU(cudaMemcpyAsync((double2 *)ctx->brhs + j * nc, r, sizeof(double2) * nc, cudaMemcpyDeviceToDevice, s));
        ctx->launches += f32 ? 1 : 0;
    }
    if (!any) return HOM_OK;
    ch.sw += 1;
    const int mb = max_bodies_for(ctx, ch.max_it);
    int rc = f32 ? batch_begin<float>(ctx, ctx->e32, ch.nb, ch.stol.data(), ch.mi.data(), mb, &ch.ran)
                 : batch_begin<double>(ctx, ctx->e64, ch.nb, ch.stol.data(), ch.mi.data(), mb, &ch.ran);
    if (rc) return rc;
    if (f32) set_bgeom<float>(ctx, ctx->e32, ch.nb);
    else set_bgeom<double>(ctx, ctx->e64, ch.nb);
    *more = true;
    return HOM_OK;
}

// after the sweep's MINRES: the iterates into the FP64 solutions, the FP64
// true residuals, and the per-case decisions (stop, take back, continue)
static int chunk_sweep_end(Chunk &ch) {
    hom_ctx *ctx = ch.ctx;
    const long long nc = 6 * ctx->S;
    cudaStream_t s = ctx->stream;
    const bool f32 = ctx->prec == HOM_PREC_FP32_FIELDS;
    int rc = f32 ? batch_end<float>(ctx, ctx->e32, ch.nb, ch.mi.data(), ch.ran, ch.its.data(), ch.est.data(), ch.sts.data())
                 : batch_end<double>(ctx, ctx->e64, ch.nb, ch.mi.data(), ch.ran, ch.its.data(), ch.est.data(), ch.sts.data());
    if (rc) return rc;
    for (int j = 0; j < ch.nb; ++j) {
        if (ch.mi[j] == 0) continue;
        const int k = ch.c0 + j;
        double2 *x = ctx->x64[k], *b = ctx->bb64 + j * nc, *r = ctx->br64 + j * nc;
        if (f32) spec_f2d_acc(nc, s, (const float2 *)ctx->brhs + j * nc, x);
        else Launch<double>::axpby(2 * nc, s, 1.0, (const double *)((double2 *)ctx->brhs + j * nc), 1.0, (double *)x);
        ctx->launches += 1;
        ch.inf[j].iterations += ch.its[j];
        ch.inf[j].est_residual = ch.est[j] * ch.tres[j];   // relative to ||b||
        ch.inf[j].sweeps = ch.sw;
        const double prev = ch.tres[j];
        rc = true_residual(ctx, x, b, r, ch.bnorm[j], &ch.tres[j], &ch.tau[6 * j]);
        if (rc) return rc;
        ch.tau_ok[j] = 1;
        if (ch.sts[j] == HOM_ENAN) {
            ch.status[j] = HOM_ENAN;
            ch.live[j] = 0;
            continue;
        }
        if (f32 && !(ch.tres[j] < prev)) {
            // an FP32 sweep past the accuracy FP32 fields can carry: take it back and stop
            spec_f2d_acc(nc, s, (const float2 *)ctx->brhs + j * nc, x, -1.0);
            ctx->launches += 1;
            rc = true_residual(ctx, x, b, r, ch.bnorm[j], &ch.tres[j], &ch.tau[6 * j]);
            if (rc) return rc;
            ch.status[j] = HOM_NOT_CONVERGED;
            ch.live[j] = 0;
            continue;
        }
        if (ch.sts[j] == HOM_NOT_CONVERGED && ch.tres[j] > ch.tol) {
            ch.status[j] = HOM_NOT_CONVERGED;
            ch.live[j] = 0;
        }
    }
    return HOM_OK;
}

static int chunk_finish(Chunk &ch, int *worst) {
    hom_ctx *ctx = ch.ctx;
    for (int j = 0; j < ch.nb; ++j) {
        const int k = ch.c0 + j;
        if (ch.solvable[j]) {
            ch.inf[j].true_residual = ch.tres[j];
            if (ch.status[j] == HOM_OK && ch.tres[j] > ch.tol) ch.status[j] = HOM_NOT_CONVERGED;
        }
        int rc = finish_case(ctx, k, &ch.M[6 * j], ctx->x64[k], &ch.inf[j], ch.status[j], ch.info ? ch.info + k : nullptr,
                             ch.tau_ok[j] ? &ch.tau[6 * j] : nullptr);
        if (rc < 0) return rc;
        if (rc > *worst) *worst = rc;
    }
    return HOM_OK;
}

static int solve_chunk(hom_ctx *ctx, int c0, int nb, const double *macro_strain, const double *macro_stress,
                       double tol, int max_it, const void *warm, hom_solve_info *info) {
    Chunk ch;
    ch.ctx = ctx;
    ch.c0 = c0;
    ch.nb = nb;
    ch.macro_strain = macro_strain;
    ch.macro_stress = macro_stress;
    ch.tol = tol;
    ch.max_it = max_it;
    ch.warm = warm;
    ch.info = info;
    int rc = chunk_prepare(ch);
    if (rc) return rc;
    while (true) {
        bool more = false;
        rc = chunk_sweep_begin(ch, &more);
        if (rc) return rc;
        if (!more) break;
        if (ch.ran) {
            const int mb = max_bodies_for(ctx, max_it);
            rc = ctx->prec == HOM_PREC_FP32_FIELDS ? batch_launch<float>(ctx, ctx->e32, nb, mb)
                                                   : batch_launch<double>(ctx, ctx->e64, nb, mb);
            if (rc) return rc;
        }
        rc = chunk_sweep_end(ch);
        if (rc) return rc;
    }
    int worst = HOM_OK;
    rc = chunk_finish(ch, &worst);
    return rc ? rc : worst;
}

// ----- many cells, one graph per sweep -------------------------------------------
// Loop condition of the multi-cell graph: count the body (ctl[0]) and go on
// while some case of some cell is not done and the cap ctl[1] is not reached.
__global__ void k_loop_cond_cells(cudaGraphConditionalHandle h, MinresState *const *sts, const int *nbs, int ncell,
                                  int *ctl) {
    if (threadIdx.x != 0) return;
    ctl[0] += 1;
    int active = 0;
    for (int i = 0; i < ncell; ++i)
        for (int c = 0; c < nbs[i]; ++c) active |= !sts[i][c].done;
    cudaGraphSetConditional(h, (active && ctl[0] < ctl[1]) ? 1u : 0u);
}

// One sweep's MINRES of several cells (each a stacked batch begun by
// batch_begin) from one graph: the cells' steps are parallel branches of the
// graph's body, forked from and joined to the root stream, and the body
// repeats on the device until every case of every cell is done.  Where
// conditional nodes are unavailable, or cells[0] asked for the host loop,
// the host replays the body and polls the states.
static int launch_cells(std::vector<hom_ctx *> &cells, std::vector<int> &nbs, int max_bodies) {
    hom_ctx *c0 = cells[0];
    const int ncell = (int)cells.size();
    cudaStream_t root = nullptr;
    std::vector<cudaEvent_t> ev(ncell + 1, nullptr);
    MinresState **d_sts = nullptr;
    int *d_nbs = nullptr, *d_ctl = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> before(ncell), per_body(ncell);
    int rc = HOM_OK;
    bool loops = false;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        cudaFree(d_sts);
        cudaFree(d_nbs);
        cudaFree(d_ctl);
        if (root) cudaStreamDestroy(root);
    };
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        for (hom_ctx *c : cells) c->err = std::string(what) + ": " + cudaGetErrorString(e);
        hom_set_error((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
        cleanup();
        return e == cudaErrorMemoryAllocation ? HOM_ENOMEM : HOM_ECUDA;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking);
    for (int i = 0; i <= ncell && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&d_sts, sizeof(MinresState *) * ncell);
    if (e == cudaSuccess) e = cudaMalloc(&d_nbs, sizeof(int) * ncell);
    if (e == cudaSuccess) e = cudaMalloc(&d_ctl, sizeof(int) * 2);
    if (e != cudaSuccess) return cuda_fail(e, "multi-cell graph set-up");
    {
        std::vector<MinresState *> h_sts(ncell);
        for (int i = 0; i < ncell; ++i) h_sts[i] = cells[i]->d_bst;
        const int ctl[2] = {0, max_bodies};
        e = cudaMemcpy(d_sts, h_sts.data(), sizeof(MinresState *) * ncell, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_nbs, nbs.data(), sizeof(int) * ncell, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "multi-cell graph set-up");
    }
    // the work each cell enqueued so far (batch_begin) precedes the graph
    for (int i = 0; i < ncell && e == cudaSuccess; ++i) {
        e = cudaEventRecord(ev[i + 1], cells[i]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(root, ev[i + 1], 0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "multi-cell graph set-up");
    auto capture_branches = [&](cudaGraphConditionalHandle *h) -> cudaError_t {
        cudaError_t er = cudaEventRecord(ev[0], root);
        for (int i = 0; i < ncell && er == cudaSuccess; ++i) {
            hom_ctx *c = cells[i];
            er = cudaStreamWaitEvent(c->stream, ev[0], 0);
            if (er != cudaSuccess) break;
            before[i] = c->launches;
            if (c->prec == HOM_PREC_FP32_FIELDS) capture_bbody<float>(c, c->e32);
            else capture_bbody<double>(c, c->e64);
            per_body[i] = c->launches - before[i];
            c->launches = before[i];
            er = cudaEventRecord(ev[i + 1], c->stream);
            if (er == cudaSuccess) er = cudaStreamWaitEvent(root, ev[i + 1], 0);
        }
        if (er == cudaSuccess && h) k_loop_cond_cells<<<1, 32, 0, root>>>(*h, d_sts, d_nbs, ncell, d_ctl);
        return er;
    };
    if (!c0->host_loop && cudaGraphCreate(&graph, 0) == cudaSuccess) {
        cudaGraphConditionalHandle h;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        cudaGraphNode_t node;
        if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess) {
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess) {
                cudaGraph_t body = np.conditional.phGraph_out[0];
                e = cudaStreamBeginCaptureToGraph(root, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t ce = capture_branches(&h);
                    e = cudaStreamEndCapture(root, &body);
                    if (ce != cudaSuccess) e = ce;
                }
                if (e != cudaSuccess) return cuda_fail(e, "multi-cell graph capture");
                loops = true;
            }
        }
        if (!loops) {
            cudaGetLastError();
            cudaGraphDestroy(graph);
            graph = nullptr;
        }
    }
    if (!loops) {
        e = cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t ce = capture_branches(nullptr);
            e = cudaStreamEndCapture(root, &graph);
            if (ce != cudaSuccess) e = ce;
        }
        if (e != cudaSuccess) return cuda_fail(e, "multi-cell graph capture");
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "multi-cell graph instantiate");
    int bodies = 0;
    if (loops) {
        e = cudaGraphLaunch(exec, root);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bodies, d_ctl, sizeof(int), cudaMemcpyDeviceToHost, root);
        if (e == cudaSuccess) e = cudaStreamSynchronize(root);
    } else {
        while (e == cudaSuccess) {
            for (int r = 0; r < 4 && bodies < max_bodies && e == cudaSuccess; ++r, ++bodies) e = cudaGraphLaunch(exec, root);
            if (e == cudaSuccess) e = cudaStreamSynchronize(root);
            bool live = false;
            for (int i = 0; i < ncell && e == cudaSuccess; ++i) {
                e = cudaMemcpy(cells[i]->h_bst, cells[i]->d_bst, sizeof(MinresState) * nbs[i], cudaMemcpyDeviceToHost);
                for (int c = 0; c < nbs[i]; ++c) live = live || !cells[i]->h_bst[c].done;
            }
            if (!live || bodies >= max_bodies) break;
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "multi-cell graph launch");
    for (int i = 0; i < ncell; ++i) cells[i]->launches += (long long)bodies * per_body[i] + (loops ? bodies : 0);
    cleanup();
    return rc;
}

// hom_solve_batch with every cell's load cases in one stacked batch and the
// sweeps of all cells from one graph launch each (all cells Galerkin-MINRES
// of one precision on the current device, every cell's cases fitting in one
// stacked batch); returns 1 (not taken) when these conditions do not hold.
int solve_cells_one_graph(hom_ctx *const *ctxs, int ncell, const double *macro_strain, int ncase, double tol,
                          int max_it, hom_solve_info *info, int *worst_out) {
    if (ncase > kNbMax) return 1;
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < ncell; ++i) {
        const hom_ctx *c = ctxs[i];
        if (c->solver != HOM_SOLVER_GALERKIN_MINRES || c->prec != ctxs[0]->prec || c->device != dev) return 1;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return 1;
    }
    std::vector<Chunk> ch(ncell);
    for (int i = 0; i < ncell; ++i) {
        hom_ctx *ctx = ctxs[i];
        if (batch_width(ctx, ncase) < ncase) return 1;
        set_stress_mask(ctx, 0);
        while ((int)ctx->x64.size() < ncase) {
            double2 *p = nullptr;
            CU(cudaMalloc(&p, sizeof(double2) * 6 * ctx->S));
            ctx->x64.push_back(p);
        }
        ctx->ncase = 0;
        ctx->macros.assign(6 * ncase, 0.0);
        ctx->eps_means.assign(6 * ncase, 0.0);
        ctx->sig_mean.assign(6 * ncase, 0.0);
        ch[i].ctx = ctx;
        ch[i].c0 = 0;
        ch[i].nb = ncase;
        ch[i].macro_strain = macro_strain;
        ch[i].tol = tol;
        ch[i].max_it = max_it;
        ch[i].info = info ? info + (size_t)i * ncase : nullptr;
        int rc = chunk_prepare(ch[i]);
        if (rc) return rc;
    }
    while (true) {
        std::vector<hom_ctx *> cells;
        std::vector<int> nbs;
        std::vector<int> in_sweep(ncell, 0);
        for (int i = 0; i < ncell; ++i) {
            bool more = false;
            int rc = chunk_sweep_begin(ch[i], &more);
            if (rc) return rc;
            in_sweep[i] = more;
            if (more && ch[i].ran) {
                cells.push_back(ch[i].ctx);
                nbs.push_back(ncase);
            }
        }
        bool any = false;
        for (int v : in_sweep) any = any || v;
        if (!any) break;
        if (!cells.empty()) {
            int rc = launch_cells(cells, nbs, max_bodies_for(ctxs[0], max_it));
            if (rc) return rc;
        }
        for (int i = 0; i < ncell; ++i) {
            if (!in_sweep[i]) continue;
            int rc = chunk_sweep_end(ch[i]);
            if (rc) return rc;
        }
    }
    int worst = HOM_OK;
    for (int i = 0; i < ncell; ++i) {
        int w = HOM_OK;
        int rc = chunk_finish(ch[i], &w);
        if (rc) return rc;
        ch[i].ctx->ncase = ncase;
        rc = finish(ch[i].ctx);
        if (rc) return rc;
        worst = std::max(worst, w);
    }
    *worst_out = worst;
    return 0;
}

// the projector's stress-controlled components at xi = 0; a change rebuilds
// the captured solve graph, whose kernels take the geometry by value
static void set_stress_mask(hom_ctx *ctx, int mask) {
    if (ctx->e64.g.mask0 == mask && ctx->e32.g.mask0 == mask) return;
    ctx->e64.g.mask0 = mask;
    ctx->e32.g.mask0 = mask;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    if (ctx->bgraph) {
        cudaGraphExecDestroy(ctx->bgraph);
        ctx->bgraph = nullptr;
        ctx->bgraph_nb = 0;
    }
    if (ctx->cg_graph && ctx->solver == HOM_SOLVER_GALERKIN_CG) {
        cudaGraphExecDestroy(ctx->cg_graph);
        ctx->cg_graph = nullptr;
    }
}

static int solve_cases(hom_ctx *ctx, const double *macro_strain, const double *macro_stress, int mask, int ncase,
                       double tol, int max_it, const void *warm_start, hom_solve_info *info) {
    cudaSetDevice(ctx->device);
    set_stress_mask(ctx, mask);
    while ((int)ctx->x64.size() < ncase) {
        double2 *p = nullptr;
        CU(cudaMalloc(&p, sizeof(double2) * 6 * ctx->S));
        ctx->x64.push_back(p);
    }
    ctx->ncase = 0;
    ctx->macros.assign(6 * ncase, 0.0);
    ctx->eps_means.assign(6 * ncase, 0.0);
    ctx->sig_mean.assign(6 * ncase, 0.0);
    int worst = HOM_OK;
    if (ctx->solver == HOM_SOLVER_GALERKIN_MINRES) {
        // the load cases in stacked batches (as many per batch as fit)
        for (int c0 = 0; c0 < ncase;) {
            const int nb = batch_width(ctx, ncase - c0);
            int rc = solve_chunk(ctx, c0, nb, macro_strain, macro_stress, tol, max_it, warm_start, info);
            if (rc < 0) {
                if (info)
                    for (int k = c0; k < c0 + nb; ++k) info[k].status = rc;
                return rc;
            }
            if (rc > worst) worst = rc;
            c0 += nb;
        }
        ctx->ncase = ncase;
        int rc = finish(ctx);
        return rc ? rc : worst;
    }
    for (int k = 0; k < ncase; ++k) {
        int rc = solve_case(ctx, k, macro_strain + 6 * k, macro_stress ? macro_stress + 6 * k : nullptr, tol, max_it,
                            warm_start, info ? info + k : nullptr);
        if (rc < 0) {
            if (info) info[k].status = rc;
            return rc;
        }
        if (rc > worst) worst = rc;
    }
    ctx->ncase = ncase;
    int rc = finish(ctx);
    return rc ? rc : worst;
}

int hom_solve(hom_ctx *ctx, const double *macro_strain, int ncase, double tol, int max_it, const void *warm_start,
              hom_solve_info *info) {
    if (!ctx || !macro_strain || ncase <= 0) return fail(ctx, HOM_EINVAL, "null argument or ncase <= 0");
    if (!(tol > 0.0) || max_it < 0) return fail(ctx, HOM_EINVAL, "need tol > 0 and max_it >= 0");
    for (int i = 0; i < 6 * ncase; ++i)
        if (!std::isfinite(macro_strain[i])) return fail(ctx, HOM_ENAN, "macro strain not finite");
    return solve_cases(ctx, macro_strain, nullptr, 0, ncase, tol, max_it, warm_start, info);
}

int hom_solve_mixed(hom_ctx *ctx, const double *macro_strain, const double *macro_stress, int stress_mask,
                    int ncase, double tol, int max_it, const void *warm_start, hom_solve_info *info) {
    if (!ctx || !macro_strain || !macro_stress || ncase <= 0)
        return fail(ctx, HOM_EINVAL, "null argument or ncase <= 0");
    if (!(tol > 0.0) || max_it < 0) return fail(ctx, HOM_EINVAL, "need tol > 0 and max_it >= 0");
    if (stress_mask < 0 || stress_mask > 63) return fail(ctx, HOM_EINVAL, "stress_mask must be in 0..63");
    if (ctx->solver == HOM_SOLVER_MODBFFT_CG)
        return fail(ctx, HOM_EINVAL, "mixed control is for the Galerkin solvers");
    if (stress_mask && warm_start) return fail(ctx, HOM_EINVAL, "warm starts need pure strain control");
    for (int i = 0; i < 6 * ncase; ++i)
        if (!std::isfinite(macro_strain[i]) || !std::isfinite(macro_stress[i]))
            return fail(ctx, HOM_ENAN, "macro strain or stress not finite");
    return solve_cases(ctx, macro_strain, macro_stress, stress_mask, ncase, tol, max_it, warm_start, info);
}

int hom_effective_stiffness(hom_ctx *ctx, double C[36]) {
    if (!ctx || !C) return fail(ctx, HOM_EINVAL, "null argument");
    const int nc = ctx->ncase;
    if (nc < 6) return fail(ctx, HOM_EINVAL, "needs a prior hom_solve with >= 6 cases");
    // Voigt strains G (6 x nc) and mean stresses S (6 x nc); C = S G^T (G G^T)^-1
    std::vector<double> G(6 * nc), Sg(6 * nc);
    const double r2 = std::sqrt(2.0);
    for (int k = 0; k < nc; ++k)
        for (int c = 0; c < 6; ++c) {
            const double mm = ctx->eps_means[6 * k + c];
            G[c * nc + k] = (c < 3) ? mm : mm * r2;   // Mandel sqrt2 e -> engineering 2e
            Sg[c * nc + k] = ctx->sig_mean[6 * k + c];
        }
    double A[6][12];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double s = 0;
            for (int k = 0; k < nc; ++k) s += G[i * nc + k] * G[j * nc + k];
            A[i][j] = s;
            A[i][6 + j] = (i == j);
        }
    for (int c = 0; c < 6; ++c) {   // Gauss-Jordan with partial pivoting
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (fabs(A[piv][c]) < 1e-300) return fail(ctx, HOM_EINVAL, "solved cases do not span six strain directions");
        for (int j = 0; j < 12; ++j) std::swap(A[c][j], A[piv][j]);
        const double d = A[c][c];
        for (int j = 0; j < 12; ++j) A[c][j] /= d;
        for (int r = 0; r < 6; ++r)
            if (r != c) {
                const double f = A[r][c];
                for (int j = 0; j < 12; ++j) A[r][j] -= f * A[c][j];
            }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double s = 0;
            for (int k = 0; k < 6; ++k) {
                double sg = 0;
                for (int q = 0; q < nc; ++q) sg += Sg[i * nc + q] * G[k * nc + q];
                s += sg * A[k][6 + j];
            }
            C[i * 6 + j] = s;
        }
    return HOM_OK;
}

int hom_fields(hom_ctx *ctx, int icase, void *strain, void *stress) {
    if (!ctx) return HOM_EINVAL;
    if (icase < 0 || icase >= ctx->ncase) return fail(ctx, HOM_EINVAL, "icase out of range of the last solve");
    cudaSetDevice(ctx->device);
    const long long n = 6 * ctx->V;
    cudaStream_t s = ctx->stream;
    const double *m = &ctx->macros[6 * icase];
    const double *eps = fluctuation64(ctx, icase);
    if (ctx->prec == HOM_PREC_FP64) {
        double *de = (double *)ctx->vbuf[0], *ds = (double *)ctx->vbuf[1];
        fields_from64<double>(ctx->V, s, eps, ctx->e64.phi, ctx->lam, ctx->mu, ctx->E, m, strain ? de : nullptr,
                              stress ? ds : nullptr);
        ctx->launches += 1;
        if (strain) { int rc = stage_out(ctx, strain, sizeof(double) * n, de); if (rc) return rc; }
        if (stress) { int rc = stage_out(ctx, stress, sizeof(double) * n, ds); if (rc) return rc; }
    } else {
        float *de = (float *)ctx->vbuf[0], *ds = (float *)ctx->vbuf[1];
        fields_from64<float>(ctx->V, s, eps, ctx->e64.phi, ctx->lam, ctx->mu, ctx->E, m, strain ? de : nullptr,
                             stress ? ds : nullptr);
        ctx->launches += 1;
        if (strain) { int rc = stage_out(ctx, strain, sizeof(float) * n, de); if (rc) return rc; }
        if (stress) { int rc = stage_out(ctx, stress, sizeof(float) * n, ds); if (rc) return rc; }
    }
    return finish(ctx);
}

// ----- elastoplastic cells (section 2.1.1) ---------------------------------------
// device bytes of the history and Newton work fields
static long long j2_bytes(const hom_ctx *ctx) {
    const long long V = ctx->V;
    return (long long)sizeof(double) * 37 * V +
           (ctx->prec == HOM_PREC_FP64 ? (long long)sizeof(double) * 36 * V
                                        : (long long)sizeof(float) * 48 * V + (long long)sizeof(double2) * 6 * ctx->S);
}

static int j2_alloc(hom_ctx *ctx) {
    J2State &j = ctx->j2;
    const long long n6 = 6 * ctx->V;
    double **f6[] = {&j.eps, &j.eps_t, &j.etry, &j.epsp, &j.sig, &j.de};
    for (double **p : f6) CU(cudaMalloc(p, sizeof(double) * n6));
    CU(cudaMalloc(&j.alpha, sizeof(double) * ctx->V));
    if (ctx->prec == HOM_PREC_FP64) {
        CU(cudaMalloc(&j.Ct, sizeof(double) * 36 * ctx->V));
    } else {
        CU(cudaMalloc(&j.Ct32, sizeof(float) * 36 * ctx->V));
        CU(cudaMalloc(&j.sig32, sizeof(float) * n6));
        CU(cudaMalloc(&j.de32, sizeof(float) * n6));
        CU(cudaMalloc(&j.x64, sizeof(double2) * 6 * ctx->S));
    }
    CU(cudaMalloc(&j.partials, sizeof(double) * 6 * kJ2Blocks));
    CU(cudaMallocHost(&j.h_partials, sizeof(double) * 6 * kJ2Blocks));
    return HOM_OK;
}

int hom_j2_begin(hom_ctx *ctx, double yield_stress, double hardening) {
    if (!ctx) return fail(nullptr, HOM_EINVAL, "null context");
    if (ctx->solver != HOM_SOLVER_GALERKIN_MINRES)
        return fail(ctx, HOM_EINVAL, "elastoplastic cells need a Galerkin-MINRES context");
    if (!(yield_stress > 0.0) || !(hardening >= 0.0) || !std::isfinite(yield_stress) || !std::isfinite(hardening))
        return fail(ctx, HOM_EINVAL, "need yield_stress > 0 and hardening >= 0, finite");
    cudaSetDevice(ctx->device);
    J2State &j = ctx->j2;
    const long long n6 = 6 * ctx->V;
    if (!j.active) {
        const int rc = j2_alloc(ctx);
        if (rc) {
            j2_free(ctx);
            return rc;
        }
        ctx->workspace += j2_bytes(ctx);
        j.active = true;
    }
    CU(cudaMemsetAsync(j.eps, 0, sizeof(double) * n6, ctx->stream));
    CU(cudaMemsetAsync(j.epsp, 0, sizeof(double) * n6, ctx->stream));
    CU(cudaMemsetAsync(j.alpha, 0, sizeof(double) * ctx->V, ctx->stream));
    j.mat = J2Material{1.0, ctx->nu, yield_stress / ctx->E, hardening / ctx->E};
    for (int c = 0; c < 6; ++c) j.Ebar[c] = 0.0;
    return finish(ctx);
}

int hom_j2_end(hom_ctx *ctx) {
    if (!ctx) return fail(nullptr, HOM_EINVAL, "null context");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->j2.active) ctx->workspace -= j2_bytes(ctx);
    j2_free(ctx);
    return HOM_OK;
}

// stress and tangent at eps (history at t), b^ = -G F{sigma - S_bar} (the
// right-hand side of eq. galnonlin, S_bar on the stress-controlled
// components through xi = 0) into b64; returns ||b^||_w
static int j2_residual(hom_ctx *ctx, const double *eps, const double sbar_v[6], double *nb) {
    J2State &j = ctx->j2;
    if (ctx->prec == HOM_PREC_FP64)
        j2_return<double>(ctx->V, j.mat, ctx->e64.phi, eps, j.epsp, j.alpha, j.sig, j.Ct, 0, ctx->stream);
    else
        j2_return<float>(ctx->V, j.mat, ctx->e64.phi, eps, j.epsp, j.alpha, j.sig, j.Ct32, 0, ctx->stream);
    real_to_spec<double>(ctx, ctx->e64, j.sig, X3_MID_NONE, true, ctx->b64);
    j2_negate_add_dc(6 * ctx->S, ctx->b64, sbar_v, ctx->stream);
    ctx->launches += 2;
    double b2 = 0.0;
    int rc = spec_norm2<double>(ctx, ctx->e64, ctx->b64, &b2);
    if (rc) return rc;
    *nb = std::sqrt(b2);
    return HOM_OK;
}

static int j2_increment_impl(hom_ctx *ctx, const double *mac_t, const double *sbar_t, int mask, double tol_lin,
                             double tol_newton, int max_newton, int max_lin, hom_j2_info *inf) {
    J2State &j = ctx->j2;
    cudaStream_t s = ctx->stream;
    const long long n6 = 6 * ctx->V, nc = 6 * ctx->S;
    const bool fp64 = ctx->prec == HOM_PREC_FP64;
    double En[6], Sn[6], sbar_v[6], d[6];
    macro_to_mandel(mac_t, En);
    macro_to_mandel(sbar_t, Sn);
    for (int c = 0; c < 6; ++c) {
        const bool kl = (mask >> c) & 1;
        sbar_v[c] = kl ? (double)ctx->V * Sn[c] / ctx->E : 0.0;   // F{S_bar} at xi = 0, units of E
        d[c] = kl ? 0.0 : En[c] - j.Ebar[c];
    }
    j.moved = false;
    CU(cudaEventRecord(ctx->ev0, s));
    CU(cudaMemcpyAsync(j.eps_t, j.eps, sizeof(double) * n6, cudaMemcpyDeviceToDevice, s));
    // predictor: the macro strain change added uniformly
    j.moved = true;
    j2_add_uniform(ctx->V, j.eps, d, s);
    ctx->launches += 1;
    double nb = 0.0;
    int rc = j2_residual(ctx, j.eps, sbar_v, &nb);
    if (rc) return rc;
    if (!std::isfinite(nb)) return fail(ctx, HOM_ENAN, "J2 residual not finite");
    const double b0 = nb;
    double rn = 0.0;
    int it = 0, lin = 0, back = 0;
    bool done = (nb == 0.0);
    while (!done && it < max_newton) {
        ++it;
        // A_i dE = b_i (eq. galnonlin) to ||A dE - b_i|| <= tol_lin ||b_0|| (eq. galrlin)
        const double tol_i = tol_lin * b0 / nb;
        const double tol_k = std::min(0.5, tol_i);
        int k = 0, st = 0;
        double est = 0.0;
        ctx->tangent_op = true;
        const double2 *dx = (const double2 *)ctx->xs;
        if (fp64) {
            CU(cudaMemcpyAsync(ctx->rhs, ctx->b64, sizeof(double2) * nc, cudaMemcpyDeviceToDevice, s));
            rc = run_minres<double>(ctx, ctx->e64, tol_k, max_lin, &k, &est, &st);
            if (rc) return rc;
            if (st == HOM_ENAN) return fail(ctx, HOM_ENAN, "J2 Newton system: MINRES breakdown");
        } else {
            // FP32 sweeps on the FP64 residual of the tangent system, whose
            // FP64 value (not the FP32 recurrence's estimate, which on cells
            // with void keeps falling below about 1e-5 while the true residual
            // stalls) measures the solve; a sweep that raises it is taken back
            CU(cudaMemsetAsync(j.x64, 0, sizeof(double2) * nc, s));
            CU(cudaMemcpyAsync(ctx->r64, ctx->b64, sizeof(double2) * nc, cudaMemcpyDeviceToDevice, s));
            double tres = 1.0;
            bool retried = false;
            for (int sweep = 0; sweep <= ctx->refine && k < max_lin; ++sweep) {
                const double floor_s = (sweep == 0 && !retried) ? kFp32MixedSweepFloor : kFp32MixedLaterSweepFloor;
                const double tol_s = std::min(0.5, std::max(kSweepTarget * tol_i / tres, floor_s));
                spec_d2f(nc, s, ctx->r64, (float2 *)ctx->rhs);
                ctx->launches += 1;
                int ks = 0;
                rc = run_minres<float>(ctx, ctx->e32, tol_s, max_lin - k, &ks, &est, &st);
                if (rc) return rc;
                if (st == HOM_ENAN) return fail(ctx, HOM_ENAN, "J2 Newton system: MINRES breakdown");
                k += ks;
                spec_f2d_acc(nc, s, (const float2 *)ctx->xs, j.x64);
                ctx->launches += 1;
                double tnew = 0.0;
                rc = true_residual(ctx, j.x64, ctx->b64, ctx->r64, nb, &tnew);
                if (rc) return rc;
                if (!(tnew < tres)) {
                    spec_f2d_acc(nc, s, (const float2 *)ctx->xs, j.x64, -1.0);
                    ctx->launches += 1;
                    // nothing gained yet: once more with the reduction of a
                    // later sweep, where the FP32 estimate still holds
                    if (sweep == 0 && !retried) {
                        retried = true;
                        sweep = -1;
                        // the step is zero again: its residual is b
                        CU(cudaMemcpyAsync(ctx->r64, ctx->b64, sizeof(double2) * nc, cudaMemcpyDeviceToDevice, s));
                        continue;
                    }
                    break;
                }
                tres = tnew;
                if (tres <= tol_i) break;
            }
            est = tres;
            dx = j.x64;
        }
        ctx->tangent_op = false;
        lin += k;
        const bool lin_ok = est * nb <= tol_lin * b0 * (1.0 + 1e-9) || tol_i >= 0.5;
        spec_to_real<double>(ctx, ctx->e64, dx, true, 1.0, j.de);
        // damped step: halve until ||b|| falls
        double t = 1.0, nt = 0.0;
        for (int tries = 0; tries < 8; ++tries) {
            CU(cudaMemcpyAsync(j.etry, j.eps, sizeof(double) * n6, cudaMemcpyDeviceToDevice, s));
            Launch<double>::axpby(n6, s, t, j.de, 1.0, j.etry);
            ctx->launches += 1;
            rc = j2_residual(ctx, j.etry, sbar_v, &nt);
            if (rc) return rc;
            if (nt < (1.0 - 1e-4 * t) * nb || tries == 7) break;
            t *= 0.5;
            ++back;
        }
        if (!std::isfinite(nt)) return fail(ctx, HOM_ENAN, "J2 residual not finite");
        // eq. (galrnewton): ||eps^{i+1} - eps^i||_inf against ||eps^{i+1} - eps^t||_inf
        const double dmax = j2_absmax(n6, j.etry, j.eps, j.partials, j.h_partials, s);
        const double emax = j2_absmax(n6, j.etry, j.eps_t, j.partials, j.h_partials, s);
        ctx->launches += 2;
        std::swap(j.eps, j.etry);
        nb = nt;
        rn = emax > 0.0 ? dmax / emax : 0.0;
        if (lin_ok && rn <= tol_newton) done = true;
    }
    // history to t + dt, mean stress and strain at the accepted iterate
    j2_return<double>(ctx->V, j.mat, ctx->e64.phi, j.eps, j.epsp, j.alpha, j.sig, nullptr, 1, s);
    double sm[6], em[6];
    j2_means(ctx->V, j.sig, j.partials, j.h_partials, sm, s);
    j2_means(ctx->V, j.eps, j.partials, j.h_partials, em, s);
    ctx->launches += 3;
    CU(cudaEventRecord(ctx->ev1, s));
    CU(cudaEventSynchronize(ctx->ev1));
    for (int c = 0; c < 6; ++c) j.Ebar[c] = En[c];
    const double r2 = std::sqrt(2.0);
    for (int c = 0; c < 6; ++c) {
        inf->sigma_mean[c] = sm[c] * ctx->E / (c >= 3 ? r2 : 1.0);
        inf->eps_mean[c] = em[c] / (c >= 3 ? r2 : 1.0);
    }
    inf->newton = it;
    inf->linear = lin;
    inf->backtracks = back;
    inf->r_newton = rn;
    inf->residual = b0 > 0.0 ? nb / b0 : 0.0;
    inf->status = done ? HOM_OK : HOM_NOT_CONVERGED;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    inf->time_ms = ms;
    return HOM_OK;
}

int hom_j2_increment(hom_ctx *ctx, const double macro_strain[6], const double macro_stress[6], int stress_mask,
                     double tol_lin, double tol_newton, int max_newton, int max_lin, hom_j2_info *info) {
    if (!ctx || !macro_strain || !macro_stress) return fail(ctx, HOM_EINVAL, "null argument");
    if (!ctx->j2.active) return fail(ctx, HOM_EINVAL, "hom_j2_begin first");
    if (stress_mask < 0 || stress_mask > 63) return fail(ctx, HOM_EINVAL, "stress_mask must be in 0..63");
    if (!(tol_lin > 0.0) || !(tol_newton > 0.0) || max_newton < 1 || max_lin < 1)
        return fail(ctx, HOM_EINVAL, "need tol_lin, tol_newton > 0 and max_newton, max_lin >= 1");
    for (int c = 0; c < 6; ++c)
        if (!std::isfinite(macro_strain[c]) || !std::isfinite(macro_stress[c]))
            return fail(ctx, HOM_ENAN, "macro strain or stress not finite");
    cudaSetDevice(ctx->device);
    set_stress_mask(ctx, stress_mask);
    ctx->ncase = 0;   // the linear solutions are not kept
    hom_j2_info inf{};
    int rc = j2_increment_impl(ctx, macro_strain, macro_stress, stress_mask, tol_lin, tol_newton, max_newton,
                               max_lin, &inf);
    ctx->tangent_op = false;
    if (rc) {
        // the history is written only at the end of an increment: putting
        // the strain at t back leaves the cell as it was
        if (ctx->j2.moved) {
            cudaMemcpyAsync(ctx->j2.eps, ctx->j2.eps_t, sizeof(double) * 6 * ctx->V, cudaMemcpyDeviceToDevice,
                            ctx->stream);
            cudaStreamSynchronize(ctx->stream);
        }
        inf.status = rc;
        if (info) *info = inf;
        return rc;
    }
    rc = finish(ctx);
    if (rc) inf.status = rc;
    if (info) *info = inf;
    return rc ? rc : inf.status;
}

int hom_j2_state(hom_ctx *ctx, double *strain, double *plastic_strain, double *alpha) {
    if (!ctx) return fail(nullptr, HOM_EINVAL, "null context");
    if (!ctx->j2.active) return fail(ctx, HOM_EINVAL, "hom_j2_begin first");
    cudaSetDevice(ctx->device);
    const long long n6 = 6 * ctx->V;
    double *tmp = (double *)ctx->r64;   // >= 6 V doubles
    const double *src[2] = {ctx->j2.eps, ctx->j2.epsp};
    double *dst[2] = {strain, plastic_strain};
    for (int f = 0; f < 2; ++f) {
        if (!dst[f]) continue;
        CU(cudaMemcpyAsync(tmp, src[f], sizeof(double) * n6, cudaMemcpyDeviceToDevice, ctx->stream));
        mandel_scale64(ctx->V, ctx->stream, tmp, 1.0 / std::sqrt(2.0));   // Mandel -> tensor components
        ctx->launches += 1;
        int rc = stage_out(ctx, dst[f], sizeof(double) * n6, tmp);
        if (rc) return rc;
    }
    if (alpha) {
        int rc = stage_out(ctx, alpha, sizeof(double) * ctx->V, ctx->j2.alpha);
        if (rc) return rc;
    }
    return finish(ctx);
}

// ----- instrumentation ----------------------------------------------------------
template <typename R>
static int time_kernels_impl(hom_ctx *ctx, Engine<R> &E, int reps, double *ms, int nmax) {
    const long long nr = 12 * ctx->S;
    cudaStream_t s = ctx->stream;
    cpx<R> *v0 = (cpx<R> *)ctx->vbuf[0], *v1 = (cpx<R> *)ctx->vbuf[1];
    cpx<R> *w1 = (cpx<R> *)ctx->wbuf[0], *w2 = (cpx<R> *)ctx->wbuf[1], *x = (cpx<R> *)ctx->xs;
    // a private state that never stops, unit-size coefficients
    MinresState h{};
    h.beta1 = 1.0; h.beta = 0.5; h.beta_prev = 0.5; h.alpha = 0.25; h.c = -1.0; h.s = 0.0; h.phibar = 1.0;
    h.tol = 0.0;
    h.u_delta = 0.1; h.u_eps = 0.1; h.u_inv_gamma = 1.0; h.u_tau = 0.0; h.u_inv_beta = 1.0;
    h.k = 1;                  // the lagged w / x update runs
    h.max_it = 1 << 30;
    // and copies at k = 1, 2, 3 for the fused n1 pass, which updates x on
    // one step in three: its launches cycle through them
    MinresState *d = nullptr;
    CU(cudaMalloc(&d, 4 * sizeof(MinresState)));
    CU(cudaMemcpy(d, &h, sizeof(h), cudaMemcpyHostToDevice));
    for (int q = 1; q <= 3; ++q) {
        MinresState hq = h;
        hq.k = q;
        CU(cudaMemcpy(d + q, &hq, sizeof(hq), cudaMemcpyHostToDevice));
    }
    for (void *b : {ctx->vbuf[0], ctx->vbuf[1], ctx->vbuf[2], ctx->wbuf[0], ctx->wbuf[1], ctx->xs})
        CU(cudaMemsetAsync(b, 0, sizeof(R) * ctx->krylov_reals, s));
    const int np3 = Launch<R>::x3_epart_grid(E.g), npl = Launch<R>::x1_lanczos_grid(E.g);
    const int nk = 6;
    Launch<R>::x1(E.g, s, X1_GAMMA_IN, v1, E.spec, nullptr, nullptr, d);
    for (int k = 0; k < nk && k < nmax; ++k) {
        // the fused n1 pass: a multiple of 3 launches (x steps in proportion)
        const int rk = k == 4 ? (reps + 2) / 3 * 3 : reps;
        for (int pass = 0; pass < 2; ++pass) {       // pass 0 warms up
            const int r = pass ? rk : 1;
            CU(cudaEventRecord(ctx->ev0, s));
            for (int i = 0; i < r; ++i) {
                switch (k) {
                    case 0: Launch<R>::x2(E.g, s, 1, E.spec, d); break;
                    case 1: Launch<R>::x3(E.g, s, X3_IN_SPEC, E.spec, X3_MID_MATERIAL, ctx->lam, ctx->mu, nullptr, 1.0,
                                          X3_OUT_SPEC, E.spec, E.phi, d, ctx->partials); break;
                    case 2: scalar_alpha(s, d, ctx->partials, np3, (double)ctx->V);
                            CU(cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, s)); break;
                    case 3: Launch<R>::x2(E.g, s, 0, E.spec, d); break;
                    case 4: Launch<R>::x1_lanczos(E.g, s, E.spec, v1, v0, (cpx<R> *)ctx->vbuf[2], w1, w2, x,
                                                  d + 1 + i % 3, ctx->partials); break;
                    default: scalar_givens(s, d, ctx->partials, npl);
                             CU(cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, s)); break;
                }
            }
            CU(cudaEventRecord(ctx->ev1, s));
            CU(cudaEventSynchronize(ctx->ev1));
            float t = 0.f;
            CU(cudaEventElapsedTime(&t, ctx->ev0, ctx->ev1));
            ms[k] = (double)t / r;
        }
        ctx->launches += rk + 1;
    }
    cudaFree(d);
    return nk < nmax ? nk : nmax;
}

int hom_time_kernels(hom_ctx *ctx, int reps, double *ms, int nmax) {
    if (!ctx || !ms || reps <= 0 || nmax <= 0) return fail(ctx, HOM_EINVAL, "bad argument");
    cudaSetDevice(ctx->device);
    int r = (ctx->prec == HOM_PREC_FP64) ? time_kernels_impl<double>(ctx, ctx->e64, reps, ms, nmax)
                                         : time_kernels_impl<float>(ctx, ctx->e32, reps, ms, nmax);
    if (r < 0) return r;
    int rc = finish(ctx);
    return rc ? rc : r;
}

// Average device time of the J2 kernels of one Newton iteration and one
// tangent-operator application, each launched `reps` times back to back on
// the context's stream between two CUDA events, at the current iterate:
// ms[0] radial return with the consistent tangent (k_j2_return, tangent in
// the operator's precision), ms[1] tangent application y = C_t : x
// (k_j2_tangent_apply, in the operator's precision), ms[2] the tangent
// operator's n3 C2R pass to a real field, ms[3] its n3 R2C pass from one.
template <typename R>
static int j2_time_impl(hom_ctx *ctx, Engine<R> &E, int reps, double *ms, int nmax) {
    J2State &j = ctx->j2;
    cudaStream_t s = ctx->stream;
    R *tin, *tout;
    if constexpr (std::is_same<R, double>::value) {
        tin = j.sig; tout = j.de;
    } else {
        tin = j.sig32; tout = j.de32;
    }
    const int nk = 4;
    for (int k = 0; k < nk && k < nmax; ++k) {
        for (int pass = 0; pass < 2; ++pass) {       // pass 0 warms up
            const int r = pass ? reps : 1;
            CU(cudaEventRecord(ctx->ev0, s));
            for (int i = 0; i < r; ++i) {
                switch (k) {
                    case 0:
                        if (j.Ct) j2_return<double>(ctx->V, j.mat, ctx->e64.phi, j.eps, j.epsp, j.alpha, j.sig, j.Ct, 0, s);
                        else j2_return<float>(ctx->V, j.mat, ctx->e64.phi, j.eps, j.epsp, j.alpha, j.sig, j.Ct32, 0, s);
                        break;
                    case 1:
                        if constexpr (std::is_same<R, double>::value) j2_tangent_apply<double, double>(ctx->V, j.Ct, tin, tout, s);
                        else j2_tangent_apply<float, float>(ctx->V, j.Ct32, tin, tout, s);
                        break;
                    case 2:
                        Launch<R>::x3(E.g, s, X3_IN_SPEC, E.spec, X3_MID_NONE, ctx->lam, ctx->mu, nullptr, 1.0, X3_OUT_REAL,
                                      tin, E.phi, nullptr);
                        break;
                    default:
                        Launch<R>::x3(E.g, s, X3_IN_REAL, tout, X3_MID_NONE, ctx->lam, ctx->mu, nullptr, 1.0, X3_OUT_SPEC,
                                      E.spec, E.phi, nullptr);
                        break;
                }
            }
            CU(cudaEventRecord(ctx->ev1, s));
            CU(cudaEventSynchronize(ctx->ev1));
            float t = 0.f;
            CU(cudaEventElapsedTime(&t, ctx->ev0, ctx->ev1));
            ms[k] = (double)t / r;
        }
        ctx->launches += reps + 1;
    }
    return nk < nmax ? nk : nmax;
}

int hom_j2_time_kernels(hom_ctx *ctx, int reps, double *ms, int nmax) {
    if (!ctx || !ms || reps <= 0 || nmax <= 0) return fail(ctx, HOM_EINVAL, "bad argument");
    if (!ctx->j2.active) return fail(ctx, HOM_EINVAL, "hom_j2_begin first");
    cudaSetDevice(ctx->device);
    int r = (ctx->prec == HOM_PREC_FP64) ? j2_time_impl<double>(ctx, ctx->e64, reps, ms, nmax)
                                         : j2_time_impl<float>(ctx, ctx->e32, reps, ms, nmax);
    if (r < 0) return r;
    int rc = finish(ctx);
    return rc ? rc : r;
}
