// Autotuner for the multigrid preconditioner of the batched form: the tile
// shape of each fused V-cycle kernel is chosen per level by timing every
// compiled shape on the grid's own level buffers with the caller's batch
// size, and the smoother counts (nu1, nu2) by time to solution on the
// caller's right-hand sides. Tile shapes do not change the arithmetic (every
// shape gives bitwise identical results); smoother counts change the
// preconditioner, so they are judged by complete solves to the caller's
// tolerance. The paper fixes neither: it applies P^-1 without saying how.
#include <cfloat>
#include <cstring>
#include <functional>
#include <vector>

#include "vcycle.cuh"

namespace helm {

namespace {

constexpr int kTileReps = 20;

// Average device microseconds of `launch` (one kernel) over kTileReps
// back-to-back launches captured in a CUDA graph on the grid's capture
// stream, replayed once to warm up and once between CUDA events.
helm_status time_launches(helm_grid *g, const std::function<void()> &launch, double *us) {
    if (!g->cap_st && cudaStreamCreateWithFlags(&g->cap_st, cudaStreamNonBlocking) != cudaSuccess)
        return fail(HELM_ERR_CUDA, "capture stream");
    cudaStream_t keep = g->st;
    g->st = g->cap_st;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const uint64_t l0 = launch_count();
    cudaError_t e = cudaStreamBeginCapture(g->cap_st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < kTileReps; ++k) launch();
        e = cudaStreamEndCapture(g->cap_st, &graph);
    }
    const uint64_t per = launch_count() - l0;
    uncount_launch(per);
    g->st = keep;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "tuning graph: %s", cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaGraphLaunch(exec, g->st);
    cudaEventRecord(e0, g->st);
    cudaGraphLaunch(exec, g->st);
    cudaEventRecord(e1, g->st);
    count_launch(2 * per);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "tuning run: %s", cudaGetErrorString(e));
    *us = ms * 1e3 / kTileReps;
    return HELM_OK;
}

// Times every down and up shape on each fine level l (pair l, l+1) with the
// same argument types the solve uses (CB0: the level-0 right-hand side is a
// basis vector) and keeps the fastest in g->tile_dn / g->tile_up.
template <typename T, typename CB0>
helm_status tune_tiles(helm_grid *g, int nrhs, helm_tune_report *rep) {
    using C = cplx_t<T>;
    const int L = (int)g->lv.size();
    const int ns = num_tile_shapes(g->dim);
    const T wj = (T)g->opt.omega_jacobi;
    const size_t sV = (size_t)(g->opt.restart + 1) * g->N;
    const CB0 *b0 = g->V.as<CB0>();
    cudaStream_t st = g->st;
    // defined contents for the timed kernels (values do not affect timing)
    cudaMemsetAsync(g->V.p, 0, (size_t)nrhs * sV * sizeof(CB0), st);
    for (int l = 0; l < L; ++l) {
        const size_t b = g->lv[l].N * sizeof(C) * (size_t)nrhs;
        cudaMemsetAsync(g->lv[l].u.p, 0, b, st);
        cudaMemsetAsync(g->lv[l].t.p, 0, b, st);
        cudaMemsetAsync(g->lv[l].b.p, 0, b, st);
    }
    std::vector<int> dn(L, -1), up(L, -1);
    helm_status s;
    rep->levels = L - 1;
    for (int l = 0; l + 1 < L && l < HELM_TUNE_MAX_LEVELS; ++l) {
        const LevelView<T> F = level_view<T>(g, l), Cv = level_view<T>(g, l + 1);
        MGLevel &Lf = g->lv[l], &Lc = g->lv[l + 1];
        double best = DBL_MAX;
        for (int sh = 0; sh < ns; ++sh) {
            auto down = [&]() {
                if (l == 0)
                    launch_vdown<T, CB0>(F, Cv, wj, b0, sV, Lf.t.template as<C>(), Lf.N,
                                         Lc.b.template as<C>(), Lc.N, nrhs, nullptr, g->st, sh);
                else
                    launch_vdown<T, C>(F, Cv, wj, Lf.b.template as<C>(), Lf.N, Lf.t.template as<C>(),
                                       Lf.N, Lc.b.template as<C>(), Lc.N, nrhs, nullptr, g->st, sh);
            };
            double us = 0.0;
            if ((s = time_launches(g, down, &us))) return s;
            if (sh == auto_tile_shape(g->dim, 0, Lf.n, nrhs)) rep->down_default_us[l] = us;
            if (us < best) {
                best = us;
                dn[l] = sh;
            }
        }
        rep->down_shape[l] = dn[l];
        rep->down_us[l] = best;
        best = DBL_MAX;
        for (int sh = 0; sh < ns; ++sh) {
            auto upk = [&]() {
                if (l == 0)
                    launch_vup<T, CB0>(F, Cv, wj, Lf.t.template as<C>(), Lf.N, Lc.u.template as<C>(),
                                       Lc.N, b0, sV, Lf.u.template as<C>(), Lf.N, nrhs, nullptr,
                                       g->st, sh);
                else
                    launch_vup<T, C>(F, Cv, wj, Lf.t.template as<C>(), Lf.N, Lc.u.template as<C>(),
                                     Lc.N, Lf.b.template as<C>(), Lf.N, Lf.u.template as<C>(), Lf.N,
                                     nrhs, nullptr, g->st, sh);
            };
            double us = 0.0;
            if ((s = time_launches(g, upk, &us))) return s;
            if (sh == auto_tile_shape(g->dim, 1, Lf.n, nrhs)) rep->up_default_us[l] = us;
            if (us < best) {
                best = us;
                up[l] = sh;
            }
        }
        rep->up_shape[l] = up[l];
        rep->up_us[l] = best;
    }
    g->tile_dn = dn;
    g->tile_up = up;
    return check_cuda("tile tuning");
}

}  // namespace

}  // namespace helm

using namespace helm;

extern "C" {

int helm_num_tile_shapes(int dim) { return num_tile_shapes(dim); }

helm_status helm_tile_shape(int dim, int kernel, int shape, int extent[3], int *threads) {
    clear_error();
    if (!extent || !threads) return fail(HELM_ERR_ARG, "null argument");
    if (!tile_shape(dim, kernel, shape, extent, threads))
        return fail(HELM_ERR_ARG, "no tile shape %d for dim %d, kernel %d", shape, dim, kernel);
    return HELM_OK;
}

helm_status helm_tile_rhs_per_block(int dim, int kernel, int shape, int *rb) {
    clear_error();
    if (!rb) return fail(HELM_ERR_ARG, "null argument");
    int ext[3], threads;
    if (!tile_shape(dim, kernel, shape, ext, &threads, rb))
        return fail(HELM_ERR_ARG, "no tile shape %d for dim %d, kernel %d", shape, dim, kernel);
    return HELM_OK;
}

helm_status helm_set_tiles(helm_grid *g, int level, int down_shape, int up_shape) {
    clear_error();
    if (!g) return fail(HELM_ERR_ARG, "null grid");
    const int ns = num_tile_shapes(g->dim);
    if (ns == 0) return fail(HELM_ERR_UNSUPPORTED, "tile shapes exist for 2D and 3D grids only");
    if (level < 0 || level >= HELM_TUNE_MAX_LEVELS) return fail(HELM_ERR_ARG, "level out of range");
    if (down_shape < -1 || down_shape >= ns || up_shape < -1 || up_shape >= ns)
        return fail(HELM_ERR_ARG, "shape index must be -1 (automatic) or in [0, %d)", ns);
    if ((int)g->tile_dn.size() <= level) {
        g->tile_dn.resize(level + 1, -1);
        g->tile_up.resize(level + 1, -1);
    }
    g->tile_dn[level] = down_shape;
    g->tile_up[level] = up_shape;
    return HELM_OK;
}

helm_status helm_get_tiles(const helm_grid *g, int level, int *down_shape, int *up_shape) {
    clear_error();
    if (!g || !down_shape || !up_shape) return fail(HELM_ERR_ARG, "null argument");
    if (level < 0 || level >= HELM_TUNE_MAX_LEVELS) return fail(HELM_ERR_ARG, "level out of range");
    *down_shape = tile_setting(g->tile_dn, level);
    *up_shape = tile_setting(g->tile_up, level);
    return HELM_OK;
}

helm_status helm_autotune(helm_grid *g, int nrhs, const helm_c128 *f, double tol, int flags,
                          helm_tune_report *rep) {
    clear_error();
    if (!g || !rep) return fail(HELM_ERR_ARG, "null argument");
    if (nrhs < 1 || nrhs > 65535) return fail(HELM_ERR_ARG, "nrhs must be 1..65535");
    if ((flags & ~(HELM_TUNE_TILES | HELM_TUNE_SMOOTHER)) || !flags)
        return fail(HELM_ERR_ARG, "flags must combine HELM_TUNE_TILES and HELM_TUNE_SMOOTHER");
    if ((flags & HELM_TUNE_SMOOTHER) && (!f || !(tol > 0.0) || !(tol < 1.0)))
        return fail(HELM_ERR_ARG, "smoother tuning needs right-hand sides and tol in (0, 1)");
    if (!g->has_model) return fail(HELM_ERR_STATE, "helm_set_model has not been called");
    if (g->opt.precond != HELM_PRECOND_MG)
        return fail(HELM_ERR_UNSUPPORTED, "tuning applies to the multigrid preconditioner");
    memset(rep, 0, sizeof(*rep));
    rep->nu1 = g->opt.nu1;
    rep->nu2 = g->opt.nu2;
    helm_status s;
    if ((s = ensure_ready(g)) || (s = workspace_for(g, nrhs)) || (s = ensure_level_work(g, nrhs)))
        return s;
    // with a variable density the V-cycle runs the general kernels: no tiles to tune
    if ((flags & HELM_TUNE_TILES) && g->dim >= 2 && g->lv.size() > 1 && !g->has_rho) {
        if (g->opt.precision == HELM_PREC_F64) s = tune_tiles<double, double2>(g, nrhs, rep);
        else if (g->opt.precision == HELM_PREC_MIXED) s = tune_tiles<float, double2>(g, nrhs, rep);
        else if (g->opt.precision == HELM_PREC_MIXED_C64) s = tune_tiles<float, float2>(g, nrhs, rep);
        else s = tune_tiles<float, float4>(g, nrhs, rep);
        if (s) return s;
    }
    if (flags & HELM_TUNE_SMOOTHER) {
        const size_t bytes = (size_t)nrhs * g->N * sizeof(double2);
        DevBuf fb, ub;
        const double2 *fd = (const double2 *)f;
        if (!is_device_ptr(f)) {
            if ((s = fb.ensure(bytes))) return s;
            cudaMemcpyAsync(fb.p, f, bytes, cudaMemcpyHostToDevice, g->st);
            fd = fb.as<double2>();
        }
        if ((s = ub.ensure(bytes))) return s;
        static const int cand[HELM_TUNE_MAX_NU][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}};
        const helm_options keep = g->opt;
        std::vector<int> its(nrhs);
        std::vector<double> rel(nrhs);
        double best = DBL_MAX;
        int bi = -1;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int c = 0; c < HELM_TUNE_MAX_NU; ++c) {
            g->opt.nu1 = cand[c][0];
            g->opt.nu2 = cand[c][1];
            rep->nu[c][0] = cand[c][0];
            rep->nu[c][1] = cand[c][1];
            // first solve captures this option set's step graphs; the second is timed
            helm_status r = solve_device(g, nrhs, fd, tol, ub.as<double2>(), its.data(), rel.data());
            if (r == HELM_OK) {
                cudaEventRecord(e0, g->st);
                r = solve_device(g, nrhs, fd, tol, ub.as<double2>(), its.data(), rel.data());
                cudaEventRecord(e1, g->st);
                cudaEventSynchronize(e1);
            }
            float ms = 0.f;
            if (r == HELM_OK) cudaEventElapsedTime(&ms, e0, e1);
            int imax = 0;
            for (int k = 0; k < nrhs; ++k) imax = its[k] > imax ? its[k] : imax;
            rep->nu_ms[c] = (r == HELM_OK) ? ms : -1.0;
            rep->nu_iterations[c] = imax;
            rep->n_nu = c + 1;
            if (r == HELM_OK && ms < best) {
                best = ms;
                bi = c;
            }
            if (r != HELM_OK && r != HELM_ERR_NOT_CONVERGED && r != HELM_ERR_BREAKDOWN) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                g->opt = keep;
                return r;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        g->opt = keep;
        if (bi < 0) return fail(HELM_ERR_NOT_CONVERGED, "no smoother candidate converged");
        g->opt.nu1 = cand[bi][0];
        g->opt.nu2 = cand[bi][1];
        rep->nu1 = g->opt.nu1;
        rep->nu2 = g->opt.nu2;
    }
    return check_cuda("helm_autotune");
}

}  // extern "C"
