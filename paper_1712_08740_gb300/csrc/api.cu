// C ABI of libhelm: grid life cycle, model and shift set-up (Eq. 2, Eq. 6),
// the multigrid hierarchy, the V-cycle that applies M^-1 inside Eq. 7, and
// the single-operator entry points used to check each step.
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "grid.cuh"
#include "vcycle.cuh"

namespace helm {

namespace {
thread_local std::string t_err;
}

helm_status fail(helm_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}
void clear_error() { t_err.clear(); }
const char *last_error() { return t_err.c_str(); }

helm_status DevBuf::ensure(size_t b) {
    if (b <= bytes) return HELM_OK;
    release();
    if (b == 0) return HELM_OK;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? HELM_ERR_NOMEM : HELM_ERR_CUDA,
                    "cudaMalloc(%zu bytes): %s", b, cudaGetErrorString(e));
    }
    bytes = b;
    return HELM_OK;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

helm_status check_cuda(const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
    return HELM_OK;
}

helm_status sync_stream(helm_grid *g, const char *where) {
    cudaError_t e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
    return check_cuda(where);
}

// ------------------------------------------------------------ hierarchy
static bool can_coarsen(const int n[3], int dim) {
    for (int a = 0; a < dim; ++a)
        if (n[a] < 3 || (n[a] % 2) == 0) return false;
    return true;
}

// Builds levels, coefficients and the coarse inverse for the current model,
// shift, options and precision.
helm_status build_hierarchy(helm_grid *g) {
    if (!g->has_model) return fail(HELM_ERR_STATE, "helm_set_model has not been called");
    prepare_vfused();
    const int prec = g->opt.precision;
    const int pc = g->opt.precond;
    // level dimensions
    std::vector<std::array<int, 3>> dims;
    std::array<int, 3> cur = {g->n[0], g->n[1], g->n[2]};
    dims.push_back(cur);
    if (pc == HELM_PRECOND_MG) {
        while (true) {
            size_t Nl = (size_t)cur[0] * cur[1] * cur[2];
            if (Nl <= (size_t)g->opt.coarse_max || !can_coarsen(cur.data(), g->dim)) break;
            for (int a = 0; a < g->dim; ++a) cur[a] = (cur[a] + 1) / 2;
            dims.push_back(cur);
        }
    }
    const size_t Nc = (size_t)dims.back()[0] * dims.back()[1] * dims.back()[2];
    if (pc != HELM_PRECOND_NONE && Nc > 4096)
        return fail(HELM_ERR_UNSUPPORTED,
                    "coarsest level has %zu nodes (> 4096): grid axes must be odd so that "
                    "(n+1)/2 coarsening reaches coarse_max",
                    Nc);
    // keep level 0 (its m/w were set by helm_set_model); coarser levels keep their
    // buffers when the level count is unchanged (no cudaFree, which would
    // synchronise the whole device and stall other grids' streams)
    if (g->lv.size() > dims.size()) g->lv.resize(dims.size());
    while (g->lv.size() < dims.size()) g->lv.emplace_back();
    for (size_t l = 0; l < dims.size(); ++l) {
        MGLevel &L = g->lv[l];
        for (int a = 0; a < 3; ++a) L.n[a] = dims[l][a];
        L.dim = g->dim;
        L.h = g->h * (double)(1u << l);
        L.N = (size_t)L.n[0] * L.n[1] * L.n[2];
    }
    helm_status s;
    for (size_t l = 1; l < g->lv.size(); ++l) {
        MGLevel &F = g->lv[l - 1], &C = g->lv[l];
        if ((s = C.m.ensure(C.N * sizeof(double)))) return s;
        if ((s = C.w64.ensure(C.N * sizeof(double)))) return s;
        if ((s = C.w32.ensure(C.N * sizeof(float)))) return s;
        launch_inject<double>(F.m.as<double>(), F.n[0], F.n[1], C.m.as<double>(), C.n[0], C.n[1],
                              C.n[2], g->st);
        launch_make_w(C.m.as<double>(), C.N, g->omega, C.w64.as<double>(), C.w32.as<float>(),
                      g->flag.as<int>(), g->st);
        if (g->has_rho) {
            // rho of Eq. 1 injected like the slowness
            if ((s = C.rho64.ensure(C.N * sizeof(double))) || (s = C.rho32.ensure(C.N * sizeof(float))))
                return s;
            launch_inject<double>(F.rho64.as<double>(), F.n[0], F.n[1], C.rho64.as<double>(), C.n[0],
                                  C.n[1], C.n[2], g->st);
            launch_make_rho(C.rho64.as<double>(), C.N, C.rho32.as<float>(), nullptr, g->st);
        }
    }
    // inverse diagonal of M per level, in the V-cycle's precision (fused
    // kernels, which run with a constant density only)
    for (size_t l = 0; l < g->lv.size() && !g->has_rho; ++l) {
        MGLevel &L = g->lv[l];
        const size_t esz = (prec == HELM_PREC_F64) ? sizeof(double2) : sizeof(float2);
        if ((s = L.dinv.ensure(L.N * esz))) return s;
        LevelView<double> v = level_view<double>(g, (int)l);
        if (prec == HELM_PREC_F64)
            launch_make_dinv<double2>(v, shift_M<double>(g), L.dinv.as<double2>(), g->st);
        else
            launch_make_dinv<float2>(v, shift_M<double>(g), L.dinv.as<float2>(), g->st);
    }
    // coarse inverse
    g->nc = 0;
    if (pc != HELM_PRECOND_NONE) {
        const MGLevel &C = g->lv.back();
        const int nc = (int)C.N;
        const size_t esz = (prec == HELM_PREC_F64) ? sizeof(double2) : sizeof(float2);
        if ((s = g->Ainv.ensure((size_t)nc * nc * esz))) return s;
        if ((s = g->colbuf.ensure((size_t)nc * esz))) return s;
        if (prec == HELM_PREC_F64) {
            LevelView<double> v = level_view<double>(g, (int)g->lv.size() - 1);
            launch_assemble_dense<double>(v, shift_M<double>(g), g->Ainv.as<double2>(), g->st);
            launch_gauss_jordan<double>(g->Ainv.as<double2>(), g->colbuf.as<double2>(), nc, g->st);
            launch_transpose_square<double>(g->Ainv.as<double2>(), nc, g->st);
        } else {
            LevelView<float> v = level_view<float>(g, (int)g->lv.size() - 1);
            launch_assemble_dense<float>(v, shift_M<float>(g), g->Ainv.as<float2>(), g->st);
            launch_gauss_jordan<float>(g->Ainv.as<float2>(), g->colbuf.as<float2>(), nc, g->st);
            launch_transpose_square<float>(g->Ainv.as<float2>(), nc, g->st);
            if ((s = g->Atc.ensure(coarse_tc_tile_floats(nc) * sizeof(float)))) return s;
            launch_coarse_tc_tiles(g->Ainv.as<float2>(), nc, g->Atc.as<float>(), g->st);
        }
        g->nc = nc;
    }
    prepare_coarse_kernels();
    if ((s = check_cuda("build_hierarchy"))) return s;
    g->vc_prec = prec;
    g->cap_rhs = 0;   // level work vectors must be re-sized for the new hierarchy
    g->cpart_rhs = 0;
    g->ready = true;
    return HELM_OK;
}

helm_status ensure_ready(helm_grid *g) {
    if (!g->has_model) return fail(HELM_ERR_STATE, "helm_set_model has not been called");
    if (!g->ready) return build_hierarchy(g);
    return HELM_OK;
}

// V-cycle work vectors for nrhs right-hand sides (precision of the hierarchy).
helm_status ensure_level_work(helm_grid *g, int nrhs) {
    const size_t esz = (g->vc_prec == HELM_PREC_F64) ? sizeof(double2) : sizeof(float2);
    helm_status s;
    for (size_t l = 0; l < g->lv.size(); ++l) {
        MGLevel &L = g->lv[l];
        const size_t b = L.N * esz * (size_t)nrhs;
        if ((s = L.t.ensure(b)) || (s = L.r.ensure(b))) return s;
        if (l > 0 && ((s = L.u.ensure(b)) || (s = L.b.ensure(b)))) return s;
        if (l == 0 && ((s = L.u.ensure(b)) || (s = L.b.ensure(b)))) return s;
    }
    if (g->nc > 0 && g->cpart_rhs < nrhs) {
        size_t pb = coarse_part_elems(g->nc, nrhs) * esz;
        if (g->vc_prec != HELM_PREC_F64)
            pb = std::max(pb, coarse_tc_part_floats(g->nc, nrhs) * sizeof(float));
        if ((s = g->cpart.ensure(pb)) ||
            (s = g->cticket.ensure(coarse_tickets(g->nc, nrhs) * sizeof(unsigned))))
            return s;
        cudaMemsetAsync(g->cticket.p, 0, coarse_tickets(g->nc, nrhs) * sizeof(unsigned), g->st);
        g->cpart_rhs = nrhs;
    }
    return HELM_OK;
}

}  // namespace helm

using namespace helm;

// ------------------------------------------------------------ C ABI
extern "C" {

void helm_default_options(helm_options *o) {
    if (!o) return;
    o->restart = 30;
    o->max_iters = 5000;
    o->precond = HELM_PRECOND_MG;
    o->precision = HELM_PREC_F64;
    o->nu1 = 1;
    o->nu2 = 1;
    o->omega_jacobi = 0.8;
    o->coarse_max = 1500;
    o->reorth = 0;
    o->graphs = 1;
    o->side = HELM_SIDE_RIGHT;
    o->block = 0;
    o->recycle = 0;
}

const char *helm_last_error(void) { return helm::last_error(); }

uint64_t helm_kernel_launches(void) { return helm::launch_count(); }

helm_status helm_set_wait_limit_ns(uint64_t ns) {
    clear_error();
    const unsigned long long v = ns ? (unsigned long long)ns : 500ull * 1000 * 1000;
    cudaError_t e = set_consumer_wait_ns(v);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HELM_ERR_CUDA, "setting the wait limit: %s", cudaGetErrorString(e));
    }
    return HELM_OK;
}

helm_status helm_create_grid(int dim, const int64_t n[3], double h, helm_grid **out) {
    clear_error();
    if (!out) return fail(HELM_ERR_ARG, "out is null");
    *out = nullptr;
    if (dim < 1 || dim > 3 || !n) return fail(HELM_ERR_ARG, "dim must be 1, 2 or 3");
    if (!(h > 0.0) || !std::isfinite(h)) return fail(HELM_ERR_ARG, "h must be > 0");
    size_t N = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < dim && (n[a] < 2 || n[a] > (1 << 24)))
            return fail(HELM_ERR_ARG, "axis %d has %lld nodes (need 2..2^24)", a, (long long)n[a]);
        if (a >= dim && n[a] != 1 && n[a] != 0)
            return fail(HELM_ERR_ARG, "unused axis %d must have 1 node", a);
        N *= (a < dim) ? (size_t)n[a] : 1;
    }
    if (N > ((size_t)1 << 31)) return fail(HELM_ERR_ARG, "more than 2^31 nodes");
    helm_grid *g = new helm_grid();
    g->dim = dim;
    for (int a = 0; a < 3; ++a) g->n[a] = (a < dim) ? (int)n[a] : 1;
    g->h = h;
    g->N = N;
    helm_default_options(&g->opt);
    g->lv.emplace_back();
    MGLevel &L = g->lv[0];
    for (int a = 0; a < 3; ++a) L.n[a] = g->n[a];
    L.dim = dim;
    L.h = h;
    L.N = N;
    helm_status s;
    if ((s = L.m.ensure(N * sizeof(double))) || (s = L.w64.ensure(N * sizeof(double))) ||
        (s = L.w32.ensure(N * sizeof(float))) || (s = g->flag.ensure(64))) {
        delete g;
        return s;
    }
    *out = g;
    return HELM_OK;
}

void helm_destroy_grid(helm_grid *g) {
    if (!g) return;
    cudaStreamSynchronize(g->st);
    for (auto e : g->step_graphs)
        if (e) cudaGraphExecDestroy(e);
    for (auto e : g->ring) cudaEventDestroy(e);
    if (g->cap_st) cudaStreamDestroy(g->cap_st);
    if (g->hflag) cudaFreeHost(g->hflag);
    if (g->bhflag) cudaFreeHost(g->bhflag);
    delete g;
}

helm_status helm_set_stream(helm_grid *g, void *stream) {
    clear_error();
    if (!g) return fail(HELM_ERR_ARG, "grid is null");
    g->st = (cudaStream_t)stream;
    return HELM_OK;
}

helm_status helm_set_options(helm_grid *g, const helm_options *o) {
    clear_error();
    if (!g || !o) return fail(HELM_ERR_ARG, "null argument");
    if (o->restart < 1 || o->restart > 256) return fail(HELM_ERR_ARG, "restart must be 1..256");
    if (o->max_iters < 1) return fail(HELM_ERR_ARG, "max_iters must be >= 1");
    if (o->precond < 0 || o->precond > 2) return fail(HELM_ERR_ARG, "bad precond");
    if (o->precision < 0 || o->precision > 3) return fail(HELM_ERR_ARG, "bad precision");
    if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 > 16 || o->nu2 > 16)
        return fail(HELM_ERR_ARG, "nu1, nu2 must be 0..16");
    if (!(o->omega_jacobi > 0.0 && o->omega_jacobi <= 1.0))
        return fail(HELM_ERR_ARG, "omega_jacobi must be in (0, 1]");
    if (o->coarse_max < 1) return fail(HELM_ERR_ARG, "coarse_max must be >= 1");
    if (o->reorth < 0 || o->reorth > 2) return fail(HELM_ERR_ARG, "reorth must be 0, 1 or 2");
    if (o->side < 0 || o->side > 2) return fail(HELM_ERR_ARG, "side must be 0, 1 or 2");
    if (o->block < 0 || o->block > 1) return fail(HELM_ERR_ARG, "block must be 0 or 1");
    if (o->recycle < 0 || o->recycle > 16) return fail(HELM_ERR_ARG, "recycle must be 0..16");
    if (o->recycle &&
        ((o->precision != HELM_PREC_F64 && o->precision != HELM_PREC_MIXED) || o->precond == HELM_PRECOND_NONE ||
         o->side != HELM_SIDE_RIGHT || o->reorth != 0 || o->block || o->restart > 40 || o->restart < o->recycle))
        return fail(HELM_ERR_UNSUPPORTED,
                    "recycling needs precision HELM_PREC_F64 or HELM_PREC_MIXED, a preconditioner, side RIGHT, "
                    "reorth 0, block 0 and recycle <= restart <= 40");
    if (o->block &&
        (o->precision != HELM_PREC_MIXED || o->precond == HELM_PRECOND_NONE || o->side != HELM_SIDE_RIGHT ||
         o->restart > 32))
        return fail(HELM_ERR_UNSUPPORTED,
                    "block FGMRES needs precision HELM_PREC_MIXED, a preconditioner, side RIGHT and "
                    "restart <= 32");
    if (o->precision == HELM_PREC_MIXED_C64 &&
        (o->side != HELM_SIDE_RIGHT || o->reorth != 0 || o->precond == HELM_PRECOND_NONE))
        return fail(HELM_ERR_UNSUPPORTED,
                    "a complex64 Arnoldi basis needs side RIGHT, reorth 0 and a preconditioner");
    if (g->has_rho && o->precision == HELM_PREC_MIXED_C64)
        return fail(HELM_ERR_UNSUPPORTED, "a variable density needs precision HELM_PREC_F64 or HELM_PREC_MIXED");
    if (g->has_rho && o->precision == HELM_PREC_MIXED_DS)
        return fail(HELM_ERR_UNSUPPORTED, "a variable density needs precision HELM_PREC_F64 or HELM_PREC_MIXED");
    if (o->side != HELM_SIDE_RIGHT && o->precond != HELM_PRECOND_NONE &&
        o->precision == HELM_PREC_MIXED_DS)
        return fail(HELM_ERR_UNSUPPORTED,
                    "left and two-sided preconditioning need a complex128 Arnoldi basis "
                    "(precision HELM_PREC_F64 or HELM_PREC_MIXED)");
    if (o->precond == HELM_PRECOND_EXACT && g->N > 4096)
        return fail(HELM_ERR_UNSUPPORTED, "exact preconditioner needs <= 4096 nodes");
    const bool rebuild = o->precond != g->opt.precond || o->precision != g->opt.precision ||
                         o->coarse_max != g->opt.coarse_max;
    g->opt = *o;
    g->use_graphs = o->graphs != 0;
    if (rebuild) g->ready = false;
    return HELM_OK;
}

helm_status helm_get_options(const helm_grid *g, helm_options *o) {
    clear_error();
    if (!g || !o) return fail(HELM_ERR_ARG, "null argument");
    *o = g->opt;
    return HELM_OK;
}

helm_status helm_set_model(helm_grid *g, const double *m, double omega, double alpha) {
    clear_error();
    if (!g || !m) return fail(HELM_ERR_ARG, "null argument");
    if (!(omega > 0.0) || !std::isfinite(omega)) return fail(HELM_ERR_ARG, "omega must be > 0");
    if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(HELM_ERR_ARG, "alpha must be >= 0");
    MGLevel &L = g->lv[0];
    cudaError_t e = cudaMemcpyAsync(L.m.p, m, g->N * sizeof(double), cudaMemcpyDefault, g->st);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "copy of m: %s", cudaGetErrorString(e));
    cudaMemsetAsync(g->flag.p, 0, sizeof(int), g->st);
    launch_make_w(L.m.as<double>(), g->N, omega, L.w64.as<double>(), L.w32.as<float>(),
                  g->flag.as<int>(), g->st);
    int bad = 0;
    cudaMemcpyAsync(&bad, g->flag.p, sizeof(int), cudaMemcpyDeviceToHost, g->st);
    helm_status s = sync_stream(g, "helm_set_model");
    if (s) return s;
    g->has_model = false;
    g->ready = false;
    g->hdiag_ok = false;
    g->rec_stale = true;
    if (bad) return fail(HELM_ERR_NONFINITE, "slowness must be finite and > 0 at every node");
    g->omega = omega;
    g->alpha = alpha;
    g->has_model = true;
    return HELM_OK;
}

helm_status helm_set_density(helm_grid *g, const double *rho) {
    clear_error();
    if (!g) return fail(HELM_ERR_ARG, "grid is null");
    if (!rho) {
        g->has_rho = false;
        g->ready = false;
        g->rec_stale = true;
        return HELM_OK;
    }
    if (g->opt.precision == HELM_PREC_MIXED_DS || g->opt.precision == HELM_PREC_MIXED_C64)
        return fail(HELM_ERR_UNSUPPORTED, "a variable density needs precision HELM_PREC_F64 or HELM_PREC_MIXED");
    MGLevel &L = g->lv[0];
    helm_status s;
    if ((s = L.rho64.ensure(g->N * sizeof(double))) || (s = L.rho32.ensure(g->N * sizeof(float)))) return s;
    cudaError_t e = cudaMemcpyAsync(L.rho64.p, rho, g->N * sizeof(double), cudaMemcpyDefault, g->st);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "copy of rho: %s", cudaGetErrorString(e));
    cudaMemsetAsync(g->flag.p, 0, sizeof(int), g->st);
    launch_make_rho(L.rho64.as<double>(), g->N, L.rho32.as<float>(), g->flag.as<int>(), g->st);
    int bad = 0;
    cudaMemcpyAsync(&bad, g->flag.p, sizeof(int), cudaMemcpyDeviceToHost, g->st);
    if ((s = sync_stream(g, "helm_set_density"))) return s;
    g->ready = false;
    g->rec_stale = true;
    if (bad) {
        g->has_rho = false;
        return fail(HELM_ERR_NONFINITE, "rho must be finite and > 0 at every node");
    }
    g->has_rho = true;
    return HELM_OK;
}

helm_status helm_set_shift(helm_grid *g, double beta1, double beta2) {
    clear_error();
    if (!g) return fail(HELM_ERR_ARG, "grid is null");
    if (!std::isfinite(beta1) || !std::isfinite(beta2)) return fail(HELM_ERR_ARG, "beta not finite");
    if (!g->has_model) return fail(HELM_ERR_STATE, "helm_set_model has not been called");
    g->beta1 = beta1;
    g->beta2 = beta2;
    g->ready = false;
    g->rec_stale = true;
    helm_status s = build_hierarchy(g);
    if (s) return s;
    return sync_stream(g, "helm_set_shift");
}

int helm_num_levels(const helm_grid *g) {
    if (!g || !g->ready) return 0;
    return (int)g->lv.size();
}

helm_status helm_level_info(const helm_grid *g, int level, int64_t n_out[3], double *h_out) {
    clear_error();
    if (!g || !n_out) return fail(HELM_ERR_ARG, "null argument");
    if (!g->ready) return fail(HELM_ERR_STATE, "hierarchy not built (call helm_set_shift)");
    if (level < 0 || level >= (int)g->lv.size()) return fail(HELM_ERR_ARG, "no level %d", level);
    for (int a = 0; a < 3; ++a) n_out[a] = g->lv[level].n[a];
    if (h_out) *h_out = g->lv[level].h;
    return HELM_OK;
}

}  // extern "C"
