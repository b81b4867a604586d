// hom_batch.cu -- many cells at once (hom_solve_batch) and the launch-shape
// autotuner (hom_autotune).
//
// Batch: every cell has its own context (stream and workspace) and its load
// cases stacked in one batch; each refinement sweep of all cells is one
// graph launch whose body holds every cell's MINRES step as a parallel
// branch, repeated on the device until every case has converged.  Small
// grids (64^3 or 96^3) leave most of the GPU idle on their own; the cells'
// branches run concurrently and fill it.
//
// Autotuner: the three FFT passes are independent, so each pass's tile is
// chosen separately.  For each candidate the kernels of one MINRES iteration
// are timed with CUDA events (hom_time_kernels) on a scratch context with a
// random phase map; the fastest shape per pass wins.  Results are cached in
// memory per (grid, precision) and, when HOM_TUNE_CACHE names a file, in that
// text file ("n1 n2 n3 precision rows3 tile2 tile1" per line).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <random>
#include <tuple>
#include <vector>

#include "../../include/hom.h"
#include "hom_internal.h"

// defined in hom_api.cu: every cell's load cases stacked, the sweeps of all
// cells from one graph launch each; returns 1 when it does not apply
int solve_cells_one_graph(hom_ctx *const *ctxs, int ncell, const double *macro_strain, int ncase, double tol,
                          int max_it, hom_solve_info *info, int *worst_out);

namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::tuple<int, int, int>> g_tuned;

void load_cache_file() {
    const char *path = std::getenv("HOM_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    int a, b, c, p, r, t2, t1;
    while (std::fscanf(f, "%d %d %d %d %d %d %d", &a, &b, &c, &p, &r, &t2, &t1) == 7)
        g_tuned[std::make_tuple(a, b, c, p)] = std::make_tuple(r, t2, t1);
    std::fclose(f);
}

void append_cache_file(const int g[3], int p, int r, int t2, int t1) {
    const char *path = std::getenv("HOM_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%d %d %d %d %d %d %d\n", g[0], g[1], g[2], p, r, t2, t1);
    std::fclose(f);
}

// per-pass time of one MINRES iteration for a launch shape; < 0 if the shape
// is rejected.  Index: 0 n1 passes, 1 n2 passes, 2 n3 pass.
int time_shape(const int grid[3], int precision, const std::vector<float> &phi, int r, int t2, int t1,
               double out[3]) {
    hom_options o;
    hom_default_options(&o);
    o.precision = precision;
    o.rows3 = r;
    o.tile2 = t2;
    o.tile1 = t1;
    hom_ctx *ctx = nullptr;
    int rc = hom_create(&ctx, grid, phi.data(), HOM_INPUT_FRACTION_F32, 1.0, 0.3, HOM_SMOOTH_NONE,
                        HOM_DERIV_ROTATED, &o);
    if (rc != HOM_OK) return rc;
    double ms[16] = {0};
    rc = hom_time_kernels(ctx, 5, ms, 16);
    hom_destroy(ctx);
    if (rc < 6) return rc < 0 ? rc : HOM_ECUDA;
    out[0] = ms[4];           // fused n1 pass
    out[1] = ms[0] + ms[3];   // n2 inverse and forward
    out[2] = ms[1];           // n3 pass
    return HOM_OK;
}

}  // namespace

int hom_autotune(const int grid[3], int precision, int shape[3]) {
    if (!grid || !shape) return HOM_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    static bool loaded = false;
    if (!loaded) {
        load_cache_file();
        loaded = true;
    }
    const auto key = std::make_tuple(grid[0], grid[1], grid[2], precision);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
        shape[0] = std::get<0>(it->second);
        shape[1] = std::get<1>(it->second);
        shape[2] = std::get<2>(it->second);
        return HOM_OK;
    }
    const long long V = (long long)grid[0] * grid[1] * grid[2];
    std::vector<float> phi(V);
    std::mt19937 rng(1234);
    std::uniform_real_distribution<float> u(0.f, 1.f);
    for (long long i = 0; i < V; ++i) phi[i] = u(rng) < 0.3f ? 0.f : u(rng);
    // start from the defaults, then sweep each pass's tile with the others fixed
    double base[3];
    int rc = time_shape(grid, precision, phi, 0, 0, 0, base);
    if (rc) return rc;
    int best[3] = {0, 0, 0};
    double best_ms[3] = {base[0], base[1], base[2]};
    const int rows_c[] = {1, 2, 4, 8};
    const int t2_c[] = {8, 16, 32};
    const int t1_c[] = {1, 2, 4, 8};
    double t[3];
    for (int r : rows_c)
        if (time_shape(grid, precision, phi, r, 0, 0, t) == HOM_OK && t[2] < best_ms[2]) {
            best_ms[2] = t[2];
            best[0] = r;
        }
    for (int t2 : t2_c)
        if (time_shape(grid, precision, phi, 0, t2, 0, t) == HOM_OK && t[1] < best_ms[1]) {
            best_ms[1] = t[1];
            best[1] = t2;
        }
    for (int t1 : t1_c)
        if (time_shape(grid, precision, phi, 0, 0, t1, t) == HOM_OK && t[0] < best_ms[0]) {
            best_ms[0] = t[0];
            best[2] = t1;
        }
    g_tuned[key] = std::make_tuple(best[0], best[1], best[2]);
    append_cache_file(grid, precision, best[0], best[1], best[2]);
    shape[0] = best[0];
    shape[1] = best[1];
    shape[2] = best[2];
    return HOM_OK;
}

int hom_solve_batch(hom_ctx *const *ctxs, int ncell, const double *macro_strain, int ncase, double tol, int max_it,
                    hom_solve_info *info) {
    if (!ctxs || ncell <= 0 || !macro_strain || ncase <= 0) return HOM_EINVAL;
    if (!(tol > 0.0) || max_it < 0) return HOM_EINVAL;
    for (int i = 0; i < ncell; ++i)
        if (!ctxs[i]) return HOM_EINVAL;
    for (int i = 0; i < 6 * ncase; ++i)
        if (!std::isfinite(macro_strain[i])) return HOM_ENAN;
    int worst = HOM_OK;
    const int rc = solve_cells_one_graph(ctxs, ncell, macro_strain, ncase, tol, max_it, info, &worst);
    if (rc <= 0) return rc < 0 ? rc : worst;
    // otherwise (other solvers, mixed precisions, too many cases for one
    // stacked batch): the cells one after another
    for (int i = 0; i < ncell; ++i) {
        const int r = hom_solve(ctxs[i], macro_strain, ncase, tol, max_it, nullptr, info ? info + (size_t)i * ncase : nullptr);
        if (r < 0) return r;
        if (r > worst) worst = r;
    }
    return worst;
}
