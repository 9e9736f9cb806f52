// The V-cycle that applies M^-1 (Eq. 6) inside the Krylov loop (Eq. 7), and
// the operator views it and the solver share.
//
// One V(nu1, nu2) cycle from a zero initial guess on every level:
//   nu1 damped-Jacobi sweeps (the first one is wj D^-1 b), residual,
//   full-weighting restriction, recursion, multilinear prolongation added to
//   the iterate, nu2 damped-Jacobi sweeps. The coarsest level is solved by
//   its dense inverse. Sweeps ping-pong between the level's iterate and a
//   scratch vector; the order is chosen so that the last sweep lands in the
//   iterate without a copy.
#pragma once

#include <array>
#include <type_traits>
#include <complex>
#include <vector>

#include "grid.cuh"

namespace helm {

bool is_device_ptr(const void *p);
helm_status check_cuda(const char *where);
helm_status sync_stream(helm_grid *g, const char *where);
helm_status ensure_ready(helm_grid *g);
helm_status ensure_level_work(helm_grid *g, int nrhs);
helm_status workspace_for(helm_grid *g, int nrhs);
// warm: u holds the initial guess x0 on entry (else x0 = 0)
helm_status solve_device(helm_grid *g, int nrhs, const double2 *f, double tol, double2 *u,
                         int *iterations, double *relres_out, bool warm = false);
const char *last_error();
// GCRO-DR with a recycled subspace kept across restarts and solves (helm_options.recycle)
helm_status solve_recycle_device(helm_grid *g, int nrhs, const double2 *f, double tol, double2 *u,
                                 int *iterations, double *relres_out, bool warm);
// block FGMRES (helm_options.block): nrhs sources in blocks of at most 64
helm_status solve_block_device(helm_grid *g, int nrhs, const double2 *f, double tol, double2 *u,
                               int *iterations, double *relres_out, bool warm);

template <typename T> inline LevelView<T> level_view(const helm_grid *g, int l) {
    const MGLevel &L = g->lv[l];
    LevelView<T> v;
    v.nx = L.n[0];
    v.ny = L.n[1];
    v.nz = L.n[2];
    v.dim = L.dim;
    v.inv_h2 = (T)(1.0 / (L.h * L.h));
    v.two_over_h = (T)(2.0 / L.h);
    v.w = (sizeof(T) == sizeof(double)) ? (const T *)L.w64.p : (const T *)L.w32.p;
    // the inverse diagonal exists in the V-cycle's own precision only
    const bool match = (sizeof(T) == sizeof(double)) == (g->vc_prec == HELM_PREC_F64);
    v.dinv = match ? (const cplx_t<T> *)L.dinv.p : nullptr;
    v.rho = !g->has_rho ? nullptr
                        : (sizeof(T) == sizeof(double)) ? (const T *)L.rho64.p : (const T *)L.rho32.p;
    return v;
}

// tile shape of the fused kernels on fine level l: the one set by
// helm_set_tiles / helm_autotune, else (-1) the automatic choice for nb
// right-hand sides
inline int tile_setting(const std::vector<int> &v, int l) {
    return l < (int)v.size() ? v[l] : -1;
}
inline int tile_down(const helm_grid *g, int l, int nb) {
    const int t = tile_setting(g->tile_dn, l);
    return t >= 0 ? t : auto_tile_shape(g->dim, 0, g->lv[l].n, nb);
}
inline int tile_up(const helm_grid *g, int l, int nb) {
    const int t = tile_setting(g->tile_up, l);
    return t >= 0 ? t : auto_tile_shape(g->dim, 1, g->lv[l].n, nb);
}

inline std::complex<double> q_of(double alpha) {
    return std::sqrt(std::complex<double>(1.0, -alpha));
}

// M = -Lap_bc - (beta1 - j beta2) w
template <typename T> inline OpShift<T> shift_M(const helm_grid *g) {
    const std::complex<double> q = q_of(g->alpha);
    return OpShift<T>{(T)g->beta1, (T)(-g->beta2), (T)q.real(), (T)q.imag()};
}

// H = -Lap_bc - (1 - j alpha) w
inline OpShift<double> shift_H(const helm_grid *g) {
    const std::complex<double> q = q_of(g->alpha);
    return OpShift<double>{1.0, -g->alpha, q.real(), q.imag()};
}

// u0 = V-cycle(b0) for nb right-hand sides; b0/u0 with per-rhs strides sb0/su0.
// CB0 is the type of b0: complex128 basis vectors feed a complex64 V-cycle
// directly in the mixed form (the fused kernels convert on load).
// Coarsest-level product z = Ainv r (Eq. 6's coarse solve): complex128 on the
// CUDA cores, complex64 on the tensor cores.
template <typename T>
inline void coarse_product(helm_grid *g, const cplx_t<T> *r, size_t sr, cplx_t<T> *z, size_t sz, int nb,
                           const int *act, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value)
        launch_coarse_tc(g->Atc.as<float>(), g->nc, r, sr, z, sz, nb, act, g->cpart.as<float>(), st);
    else
        launch_dense_gemv<T>((const cplx_t<T> *)g->Ainv.p, g->nc, r, sr, z, sz, nb, act, g->cpart.p,
                             g->cticket.template as<unsigned>(), st);
}

// With w0 (complex64 basis only: T = float, CB0 = float2) the level-0
// right-hand side is not yet in b0: it is v = w0 / ||w0|| rounded to
// complex64 (sc0: the scale as float hi + lo, nrm0: ||w0||^2), which the
// level-0 down kernel forms as it loads w0 and writes to b0 (a basis slot);
// kernels that cannot take w0 get v from launch_scale_c64 first.
template <typename T, typename CB0>
void vcycle(helm_grid *g, const CB0 *b0, size_t sb0, cplx_t<T> *u0, size_t su0, int nb,
            const int *act, const float4 *w0 = nullptr, size_t sw0 = 0, const float2 *sc0 = nullptr,
            const double *nrm0 = nullptr) {
    using C = cplx_t<T>;
    constexpr bool kC64 = std::is_same<T, float>::value && std::is_same<CB0, float2>::value;
    const int L = (int)g->lv.size();
    const OpShift<T> sM = shift_M<T>(g);
    const T wj = (T)g->opt.omega_jacobi;
    const int nu1 = g->opt.nu1, nu2 = g->opt.nu2;
    cudaStream_t st = g->st;
    // the fused level kernels carry the constant-density stencil only
    const bool fused = L > 1 && g->dim >= 2 && nu1 == 1 && nu2 == 1 && !g->has_rho;
    bool v_done = w0 == nullptr;
    auto make_v = [&] {
        if constexpr (kC64) {
            if (!v_done) launch_scale_c64(w0, sw0, nrm0, const_cast<float2 *>(b0), sb0, g->lv[0].N, nb, act, st);
        }
        v_done = true;
    };
    if (fused) {
        // down: u_l (pre-smoothed, into the level's scratch) and b_{l+1}
        for (int l = 0; l < L - 1; ++l) {
            const LevelView<T> F = level_view<T>(g, l), Cv = level_view<T>(g, l + 1);
            C *bc = g->lv[l + 1].b.template as<C>();
            if (l == 0) {
                if constexpr (kC64) {
                    if (!v_done) {
                        if (launch_vdown_c64w(F, Cv, wj, w0, sw0, sc0, const_cast<float2 *>(b0), sb0,
                                              g->lv[0].t.template as<C>(), g->lv[0].N, bc, g->lv[1].N, nb, act, st,
                                              tile_down(g, 0, nb))) {
                            v_done = true;
                            continue;
                        }
                        make_v();
                    }
                }
                launch_vdown<T, CB0>(F, Cv, wj, b0, sb0, g->lv[0].t.template as<C>(), g->lv[0].N,
                                     bc, g->lv[1].N, nb, act, st, tile_down(g, 0, nb), true);
            } else
                launch_vdown<T, C>(F, Cv, wj, g->lv[l].b.template as<C>(), g->lv[l].N,
                                   g->lv[l].t.template as<C>(), g->lv[l].N, bc, g->lv[l + 1].N, nb,
                                   act, st, tile_down(g, l, nb));
        }
        C *uc = (L - 1 == 0) ? u0 : g->lv[L - 1].u.template as<C>();
        coarse_product<T>(g, g->lv[L - 1].b.template as<C>(), g->lv[L - 1].N, uc, g->lv[L - 1].N, nb,
                          act, st);
        // up: u_l = Jacobi(u_pre + P e_{l+1})
        for (int l = L - 2; l >= 0; --l) {
            const LevelView<T> F = level_view<T>(g, l), Cv = level_view<T>(g, l + 1);
            const C *ec = g->lv[l + 1].u.template as<C>();
            if (l == 0)
                launch_vup<T, CB0>(F, Cv, wj, g->lv[0].t.template as<C>(), g->lv[0].N, ec,
                                   g->lv[1].N, b0, sb0, u0, su0, nb, act, st, tile_up(g, 0, nb), true);
            else
                launch_vup<T, C>(F, Cv, wj, g->lv[l].t.template as<C>(), g->lv[l].N, ec,
                                 g->lv[l + 1].N, g->lv[l].b.template as<C>(), g->lv[l].N,
                                 g->lv[l].u.template as<C>(), g->lv[l].N, nb, act, st, tile_up(g, l, nb));
        }
        return;
    }
    // general path: level-0 right-hand side in the V-cycle's own type
    make_v();
    const C *b0c;
    size_t sb0c;
    if constexpr (std::is_same<CB0, C>::value) {
        b0c = b0;
        sb0c = sb0;
    } else {
        launch_convert<CB0, C>(b0, sb0, g->lv[0].b.template as<C>(), g->lv[0].N, g->lv[0].N, nb, st);
        b0c = g->lv[0].b.template as<C>();
        sb0c = g->lv[0].N;
    }
    if (L == 1) {
        coarse_product<T>(g, b0c, sb0c, u0, su0, nb, act, st);
        return;
    }
    std::vector<const C *> B(L);
    std::vector<C *> U(L);
    std::vector<size_t> SB(L), SU(L);
    B[0] = b0c;
    SB[0] = sb0c;
    U[0] = u0;
    SU[0] = su0;
    for (int l = 1; l < L; ++l) {
        B[l] = g->lv[l].b.template as<C>();
        U[l] = g->lv[l].u.template as<C>();
        SB[l] = SU[l] = g->lv[l].N;
    }
    for (int l = 0; l < L - 1; ++l) {
        const LevelView<T> Lv = level_view<T>(g, l);
        const size_t N = g->lv[l].N;
        C *tmp = g->lv[l].t.template as<C>();
        if (nu1 == 0) {
            cudaMemset2DAsync(U[l], SU[l] * sizeof(C), 0, N * sizeof(C), nb, st);
            launch_restrict<T>(Lv, level_view<T>(g, l + 1), B[l], SB[l], g->lv[l + 1].b.template as<C>(),
                               g->lv[l + 1].N, nb, act, st);
            continue;
        }
        // sweep k (1-based) writes U[l] when nu1 - k is even, tmp otherwise
        const C *prev = nullptr;
        size_t sprev = 0;
        for (int k = 1; k <= nu1; ++k) {
            C *dst = ((nu1 - k) % 2 == 0) ? U[l] : tmp;
            const size_t sdst = ((nu1 - k) % 2 == 0) ? SU[l] : N;
            if (k == 1)
                launch_stencil<T, C, C>(ST_JACOBI0, Lv, sM, (const C *)nullptr, 0, B[l], SB[l], dst,
                                        sdst, nb, wj, act, st);
            else
                launch_stencil<T, C, C>(ST_JACOBI, Lv, sM, prev, sprev, B[l], SB[l], dst, sdst, nb,
                                        wj, act, st);
            prev = dst;
            sprev = sdst;
        }
        C *res = g->lv[l].r.template as<C>();
        launch_stencil<T, C, C>(ST_RESID, Lv, sM, U[l], SU[l], B[l], SB[l], res, N, nb, wj, act,
                                st);
        launch_restrict<T>(Lv, level_view<T>(g, l + 1), res, N, g->lv[l + 1].b.template as<C>(),
                           g->lv[l + 1].N, nb, act, st);
    }
    coarse_product<T>(g, B[L - 1], SB[L - 1], U[L - 1], SU[L - 1], nb, act, st);
    for (int l = L - 2; l >= 0; --l) {
        const LevelView<T> Lv = level_view<T>(g, l);
        const LevelView<T> Cv = level_view<T>(g, l + 1);
        const size_t N = g->lv[l].N;
        C *tmp = g->lv[l].t.template as<C>();
        // corrected iterate goes to U when nu2 is even, to tmp when odd
        C *cur = (nu2 % 2 == 0) ? U[l] : tmp;
        size_t scur = (nu2 % 2 == 0) ? SU[l] : N;
        launch_prolong_add<T>(Lv, Cv, U[l + 1], SU[l + 1], U[l], SU[l], cur, scur, nb, act, st);
        for (int k = 1; k <= nu2; ++k) {
            C *dst = (cur == U[l]) ? tmp : U[l];
            const size_t sdst = (cur == U[l]) ? N : SU[l];
            launch_stencil<T, C, C>(ST_JACOBI, Lv, sM, cur, scur, B[l], SB[l], dst, sdst, nb, wj,
                                    act, st);
            cur = dst;
            scur = sdst;
        }
    }
}

}  // namespace helm
