// Restarted flexible GMRES for H M^-1 z = f, u = M^-1 z (Eq. 7), for one or
// many right-hand sides that share H and M.
//
// Device side (complex128 unless noted): V-cycle z_j = M^-1 v_j (complex64 in
// the mixed form), w = H z_j written straight into the basis slot v_{j+1},
// classical Gram-Schmidt (twice by default) as fused multi-dot and
// multi-axpy kernels, the norm fused into the last axpy, scaling, and at the
// end of a cycle x += Z y and the true residual f - H x.
// Host side: the (m+1) x m Hessenberg least-squares problem per right-hand
// side with complex Givens rotations (real cosine), which costs O(m) flops
// per step and needs one small device-to-host copy per Arnoldi step.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "vcycle.cuh"

namespace helm {

using cd = std::complex<double>;

namespace {

struct RhsState {
    double fnorm = 0.0;
    std::vector<cd> R, g, sn;
    std::vector<double> cs;
    int k = 0;             // steps in the current cycle
    int its = 0;
    bool done = false;      // converged or given up
    bool iter = false;      // still stepping in this cycle
    bool converged = false;
    bool broke = false;
    double relres = 0.0;
};

helm_status ensure_workspace(helm_grid *g, int nrhs) {
    const int m = g->opt.restart;
    const int prec = g->opt.precision;
    const int pc = g->opt.precond;
    if (g->cap_rhs >= nrhs && g->cap_m == m && g->cap_prec == prec) return HELM_OK;
    const size_t N = g->N;
    helm_status s;
    const size_t zsz = (prec == HELM_PREC_F64) ? sizeof(double2) : sizeof(float2);
    if ((s = g->V.ensure((size_t)nrhs * (m + 1) * N * sizeof(double2)))) return s;
    if (pc != HELM_PRECOND_NONE) {
        if ((s = g->Z.ensure((size_t)nrhs * m * N * zsz))) return s;
        if (prec == HELM_PREC_MIXED && (s = g->Zin.ensure((size_t)nrhs * N * sizeof(float2))))
            return s;
    }
    const int nv = m + 1;
    if ((s = g->hbuf.ensure((size_t)nrhs * 2 * nv * sizeof(double2)))) return s;
    if ((s = g->nrm.ensure((size_t)nrhs * sizeof(double)))) return s;
    if ((s = g->yv.ensure((size_t)nrhs * m * sizeof(double2)))) return s;
    const int max_blocks = 4 * 152;
    if ((s = g->partial.ensure((size_t)nrhs * max_blocks * nv * sizeof(double2)))) return s;
    if ((s = g->counter.ensure((size_t)nrhs * sizeof(unsigned)))) return s;
    cudaMemsetAsync(g->counter.p, 0, (size_t)nrhs * sizeof(unsigned), g->st);
    if ((s = g->act_it.ensure((size_t)nrhs * sizeof(int)))) return s;
    if ((s = g->act_cy.ensure((size_t)nrhs * sizeof(int)))) return s;
    const size_t pin_need = (size_t)nrhs * 2 * nv * sizeof(double2) + (size_t)nrhs * sizeof(double);
    if (g->pin_bytes < pin_need) {
        if (g->pin) cudaFreeHost(g->pin);
        g->pin = nullptr;
        g->pin_bytes = 0;
        if (cudaMallocHost(&g->pin, pin_need) != cudaSuccess) {
            cudaGetLastError();
            return fail(HELM_ERR_NOMEM, "pinned host buffer of %zu bytes", pin_need);
        }
        g->pin_bytes = pin_need;
    }
    if ((s = ensure_level_work(g, nrhs))) return s;
    g->cap_rhs = nrhs;
    g->cap_m = m;
    g->cap_prec = prec;
    return HELM_OK;
}

KrylovScratch scratch(helm_grid *g) {
    KrylovScratch ks;
    ks.partial = g->partial.as<double2>();
    ks.counter = g->counter.as<unsigned>();
    ks.max_blocks = 4 * 152;
    ks.nvec_max = g->opt.restart + 1;
    return ks;
}

// z_j = M^-1 v_j for all flagged right-hand sides
void apply_precond_j(helm_grid *g, int j, int nrhs, const int *act) {
    const size_t N = g->N;
    const int m = g->opt.restart;
    const size_t sV = (size_t)(m + 1) * N, sZ = (size_t)m * N;
    const double2 *vj = g->V.as<double2>() + (size_t)j * N;
    if (g->opt.precision == HELM_PREC_F64) {
        vcycle<double>(g, vj, sV, g->Z.as<double2>() + (size_t)j * N, sZ, nrhs, act);
    } else {
        launch_convert<double2, float2>(vj, sV, g->Zin.as<float2>(), N, N, nrhs, g->st);
        vcycle<float>(g, g->Zin.as<float2>(), N, g->Z.as<float2>() + (size_t)j * N, sZ, nrhs, act);
    }
}

// w = H z_j into basis slot j+1
void apply_H_j(helm_grid *g, int j, int nrhs, const int *act) {
    const size_t N = g->N;
    const int m = g->opt.restart;
    const size_t sV = (size_t)(m + 1) * N, sZ = (size_t)m * N;
    double2 *w = g->V.as<double2>() + (size_t)(j + 1) * N;
    const LevelView<double> Lv = level_view<double>(g, 0);
    if (g->opt.precond == HELM_PRECOND_NONE) {
        const double2 *z = g->V.as<double2>() + (size_t)j * N;
        launch_stencil<double, double2, double2>(ST_APPLY, Lv, shift_H(g), z, sV,
                                                 (const double2 *)nullptr, 0, w, sV, nrhs, 0.0,
                                                 act, g->st);
    } else if (g->opt.precision == HELM_PREC_F64) {
        const double2 *z = g->Z.as<double2>() + (size_t)j * N;
        launch_stencil<double, double2, double2>(ST_APPLY, Lv, shift_H(g), z, sZ,
                                                 (const double2 *)nullptr, 0, w, sV, nrhs, 0.0,
                                                 act, g->st);
    } else {
        const float2 *z = g->Z.as<float2>() + (size_t)j * N;
        launch_stencil<double, float2, double2>(ST_APPLY, Lv, shift_H(g), z, sZ,
                                                (const double2 *)nullptr, 0, w, sV, nrhs, 0.0,
                                                act, g->st);
    }
}

// Givens rotation with real cosine that maps (a, b) to (r, 0)
inline void givens(cd a, cd b, double &c, cd &s, cd &r) {
    const double aa = std::abs(a), bb = std::abs(b);
    if (aa == 0.0) {
        c = 0.0;
        s = cd(1.0, 0.0);
        r = b;
        return;
    }
    const double rho = std::hypot(aa, bb);
    c = aa / rho;
    s = (a / aa) * std::conj(b) / rho;
    r = (a / aa) * rho;
}

}  // namespace

// Core solver on device arrays f (nrhs x N) and u (nrhs x N), stride N.
helm_status solve_device(helm_grid *g, int nrhs, const double2 *f, double tol, double2 *u,
                         int *iterations, double *relres_out) {
    helm_status s;
    if ((s = ensure_ready(g))) return s;
    if ((s = ensure_workspace(g, nrhs))) return s;
    const size_t N = g->N;
    const int m = g->opt.restart;
    const int nv = m + 1;
    const size_t sV = (size_t)(m + 1) * N;
    cudaStream_t st = g->st;
    KrylovScratch ks = scratch(g);
    double2 *V = g->V.as<double2>();
    double2 *hb = g->hbuf.as<double2>();
    double *nrm = g->nrm.as<double>();
    int *act_it = g->act_it.as<int>(), *act_cy = g->act_cy.as<int>();
    double2 *hpin = (double2 *)g->pin;
    double *npin = (double *)((char *)g->pin + (size_t)nrhs * 2 * nv * sizeof(double2));
    const LevelView<double> L0 = level_view<double>(g, 0);

    // non-finite input check
    cudaMemsetAsync(g->flag.p, 0, sizeof(int), st);
    launch_finite_check((const double *)f, 2 * N * (size_t)nrhs, g->flag.as<int>(), st);
    int bad = 0;
    cudaMemcpyAsync(&bad, g->flag.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    // x = 0, v_0 = f, ||f||
    cudaMemsetAsync(u, 0, (size_t)nrhs * N * sizeof(double2), st);
    launch_convert<double2, double2>(f, N, V, sV, N, nrhs, st);
    launch_norm2(f, N, N, nrm, nrhs, nullptr, ks, st);
    cudaMemcpyAsync(npin, nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st);
    if ((s = sync_stream(g, "solve start"))) return s;
    if (bad) return fail(HELM_ERR_NONFINITE, "right-hand side contains NaN or Inf");

    std::vector<RhsState> S(nrhs);
    std::vector<int> h_act(nrhs);
    for (int k = 0; k < nrhs; ++k) {
        RhsState &R = S[k];
        R.R.assign((size_t)(m + 1) * m, 0.0);
        R.g.assign(m + 1, 0.0);
        R.sn.assign(m, 0.0);
        R.cs.assign(m, 0.0);
        R.fnorm = std::sqrt(npin[k]);
        if (R.fnorm == 0.0) {
            R.done = R.converged = true;
            R.relres = 0.0;
        }
    }
    std::vector<double> beta(nrhs);
    for (int k = 0; k < nrhs; ++k) beta[k] = S[k].fnorm;
    std::vector<double2> ypin((size_t)nrhs * m);

    while (true) {
        // ---- start a cycle: v_0 = r / ||r|| (r already in slot 0, ||r||^2 in nrm)
        int ncy = 0;
        for (int k = 0; k < nrhs; ++k) {
            RhsState &R = S[k];
            R.iter = !R.done;
            R.k = 0;
            h_act[k] = R.iter ? 1 : 0;
            ncy += h_act[k];
            if (R.iter) {
                std::fill(R.g.begin(), R.g.end(), cd(0.0));
                R.g[0] = beta[k];
            }
        }
        if (ncy == 0) break;
        cudaMemcpyAsync(act_cy, h_act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(act_it, h_act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st);
        launch_scale<double2>(V, sV, nrm, V, sV, N, nrhs, act_cy, st);

        for (int j = 0; j < m; ++j) {
            if (g->opt.precond != HELM_PRECOND_NONE) apply_precond_j(g, j, nrhs, act_it);
            apply_H_j(g, j, nrhs, act_it);
            double2 *w = V + (size_t)(j + 1) * N;
            const int nvec = j + 1;
            const bool two = g->opt.reorth != 0;
            launch_multidot(V, sV, nvec, w, sV, N, hb, 2 * nv, nrhs, act_it, ks, st);
            launch_multiaxpy(V, sV, nvec, hb, 2 * nv, w, sV, N, two ? nullptr : nrm, nrhs, act_it,
                             ks, st);
            if (two) {
                launch_multidot(V, sV, nvec, w, sV, N, hb + nv, 2 * nv, nrhs, act_it, ks, st);
                launch_multiaxpy(V, sV, nvec, hb + nv, 2 * nv, w, sV, N, nrm, nrhs, act_it, ks, st);
            }
            cudaMemcpyAsync(hpin, hb, (size_t)nrhs * 2 * nv * sizeof(double2),
                            cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(npin, nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st);
            if ((s = sync_stream(g, "arnoldi step"))) return s;
            bool changed = false;
            int still = 0;
            for (int k = 0; k < nrhs; ++k) {
                RhsState &R = S[k];
                if (!R.iter) continue;
                cd *col = &R.R[(size_t)j];   // column j, row stride m
                auto Rij = [&](int i) -> cd & { return R.R[(size_t)i * m + j]; };
                for (int i = 0; i <= j; ++i) {
                    const double2 a = hpin[(size_t)k * 2 * nv + i];
                    cd v(a.x, a.y);
                    if (two) {
                        const double2 b2 = hpin[(size_t)k * 2 * nv + nv + i];
                        v += cd(b2.x, b2.y);
                    }
                    Rij(i) = v;
                }
                (void)col;
                const double hn = std::sqrt(npin[k]);
                Rij(j + 1) = hn;
                bool finite = std::isfinite(hn);
                for (int i = 0; i <= j; ++i) finite = finite && std::isfinite(Rij(i).real()) &&
                                                      std::isfinite(Rij(i).imag());
                if (!finite) {
                    R.iter = false;
                    R.done = true;
                    R.broke = true;
                    changed = true;
                    continue;
                }
                for (int i = 0; i < j; ++i) {
                    const cd a = Rij(i), b = Rij(i + 1);
                    Rij(i) = R.cs[i] * a + R.sn[i] * b;
                    Rij(i + 1) = -std::conj(R.sn[i]) * a + R.cs[i] * b;
                }
                cd rr;
                givens(Rij(j), Rij(j + 1), R.cs[j], R.sn[j], rr);
                Rij(j) = rr;
                Rij(j + 1) = 0.0;
                R.g[j + 1] = -std::conj(R.sn[j]) * R.g[j];
                R.g[j] = R.cs[j] * R.g[j];
                R.k = j + 1;
                R.its += 1;
                const double est = std::abs(R.g[j + 1]);
                if (est <= tol * R.fnorm || hn <= 1e-300 || R.its >= g->opt.max_iters) {
                    R.iter = false;
                    changed = true;
                } else {
                    ++still;
                }
            }
            if (still == 0 || j == m - 1) break;
            if (changed) {
                for (int k = 0; k < nrhs; ++k) h_act[k] = S[k].iter ? 1 : 0;
                cudaMemcpyAsync(act_it, h_act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice,
                                st);
            }
            launch_scale<double2>(w, sV, nrm, w, sV, N, nrhs, act_it, st);
        }

        // ---- end of cycle: y = R^-1 g, x += Z y, r = f - H x
        int kmax = 0;
        for (int k = 0; k < nrhs; ++k) {
            RhsState &R = S[k];
            double2 *y = &ypin[(size_t)k * m];
            for (int i = 0; i < m; ++i) y[i] = make_double2(0.0, 0.0);
            if (R.done && !R.broke) continue;
            if (R.broke || R.k == 0) continue;
            std::vector<cd> yy(R.k);
            for (int i = R.k - 1; i >= 0; --i) {
                cd acc = R.g[i];
                for (int q = i + 1; q < R.k; ++q) acc -= R.R[(size_t)i * m + q] * yy[q];
                yy[i] = acc / R.R[(size_t)i * m + i];
            }
            for (int i = 0; i < R.k; ++i) y[i] = make_double2(yy[i].real(), yy[i].imag());
            if (R.k > kmax) kmax = R.k;
        }
        for (int k = 0; k < nrhs; ++k) h_act[k] = (!S[k].done || S[k].broke) && S[k].k > 0 ? 1 : 0;
        for (int k = 0; k < nrhs; ++k)
            if (S[k].broke) h_act[k] = 0;
        cudaMemcpyAsync(act_cy, h_act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(g->yv.p, ypin.data(), (size_t)nrhs * m * sizeof(double2),
                        cudaMemcpyHostToDevice, st);
        if (kmax > 0) {
            if (g->opt.precond == HELM_PRECOND_NONE)
                launch_update<double2>(V, sV, kmax, g->yv.as<double2>(), m, u, N, N, nrhs, act_cy,
                                       st);
            else if (g->opt.precision == HELM_PREC_F64)
                launch_update<double2>(g->Z.as<double2>(), (size_t)m * N, kmax,
                                       g->yv.as<double2>(), m, u, N, N, nrhs, act_cy, st);
            else
                launch_update<float2>(g->Z.as<float2>(), (size_t)m * N, kmax, g->yv.as<double2>(),
                                      m, u, N, N, nrhs, act_cy, st);
        }
        // true residual into slot 0
        launch_stencil<double, double2, double2>(ST_RESID, L0, shift_H(g), u, N, f, N, V, sV, nrhs,
                                                 0.0, act_cy, st);
        launch_norm2(V, sV, N, nrm, nrhs, act_cy, ks, st);
        cudaMemcpyAsync(npin, nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st);
        if ((s = sync_stream(g, "cycle end"))) return s;
        for (int k = 0; k < nrhs; ++k) {
            RhsState &R = S[k];
            if (!h_act[k]) continue;
            beta[k] = std::sqrt(npin[k]);
            R.relres = beta[k] / R.fnorm;
            if (R.relres <= tol) {
                R.done = R.converged = true;
            } else if (R.its >= g->opt.max_iters) {
                R.done = true;
            }
        }
    }
    bool all_conv = true, any_broke = false;
    for (int k = 0; k < nrhs; ++k) {
        if (iterations) iterations[k] = S[k].its;
        if (relres_out) relres_out[k] = S[k].relres;
        all_conv = all_conv && S[k].converged;
        any_broke = any_broke || S[k].broke;
    }
    if (any_broke) return fail(HELM_ERR_BREAKDOWN, "Arnoldi produced a non-finite value");
    if (!all_conv)
        return fail(HELM_ERR_NOT_CONVERGED, "not converged within %d iterations", g->opt.max_iters);
    return HELM_OK;
}

}  // namespace helm

using namespace helm;

namespace {

// Stages a (possibly host) input array onto the device.
helm_status stage_in(helm_grid *g, const void *src, size_t bytes, DevBuf &buf, const void **dev) {
    if (is_device_ptr(src)) {
        *dev = src;
        return HELM_OK;
    }
    helm_status s = buf.ensure(bytes);
    if (s) return s;
    cudaError_t e = cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, g->st);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "host-to-device copy: %s", cudaGetErrorString(e));
    *dev = buf.p;
    return HELM_OK;
}

helm_status out_buf(helm_grid *g, void *dst, size_t bytes, DevBuf &buf, void **dev) {
    if (is_device_ptr(dst)) {
        *dev = dst;
        return HELM_OK;
    }
    helm_status s = buf.ensure(bytes);
    if (s) return s;
    *dev = buf.p;
    return HELM_OK;
}

helm_status copy_out(helm_grid *g, void *dst, const void *dev, size_t bytes) {
    if (dst == dev) return HELM_OK;
    cudaError_t e = cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, g->st);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "device-to-host copy: %s", cudaGetErrorString(e));
    return sync_stream(g, "copy out");
}

}  // namespace

extern "C" {

helm_status helm_solve_batch(helm_grid *g, int nrhs, const helm_c128 *f, double tol, helm_c128 *u,
                             int *iterations, double *true_rel_residual) {
    clear_error();
    if (!g || !f || !u) return fail(HELM_ERR_ARG, "null argument");
    if (nrhs < 1 || nrhs > 65535) return fail(HELM_ERR_ARG, "nrhs must be 1..65535");
    if (!(tol > 0.0) || !(tol < 1.0)) return fail(HELM_ERR_ARG, "tol must be in (0, 1)");
    if (!g->has_model) return fail(HELM_ERR_STATE, "helm_set_model has not been called");
    const size_t bytes = (size_t)nrhs * g->N * sizeof(double2);
    const void *fd;
    void *ud;
    helm_status s;
    if ((s = stage_in(g, f, bytes, g->fst, &fd))) return s;
    if ((s = out_buf(g, u, bytes, g->ust, &ud))) return s;
    helm_status rs = solve_device(g, nrhs, (const double2 *)fd, tol, (double2 *)ud, iterations,
                                  true_rel_residual);
    if (rs != HELM_OK && rs != HELM_ERR_NOT_CONVERGED && rs != HELM_ERR_BREAKDOWN) return rs;
    std::string keep = last_error();
    if ((s = copy_out(g, u, ud, bytes))) return s;
    if (rs != HELM_OK) return fail(rs, "%s", keep.c_str());
    return HELM_OK;
}

helm_status helm_solve(helm_grid *g, const helm_c128 *f, double tol, helm_c128 *u, int *iterations,
                       double *true_rel_residual) {
    return helm_solve_batch(g, 1, f, tol, u, iterations, true_rel_residual);
}

helm_status helm_apply_H(helm_grid *g, const helm_c128 *x, helm_c128 *y) {
    clear_error();
    if (!g || !x || !y) return fail(HELM_ERR_ARG, "null argument");
    if (!g->has_model) return fail(HELM_ERR_STATE, "helm_set_model has not been called");
    const size_t bytes = g->N * sizeof(double2);
    const void *xd;
    void *yd;
    helm_status s;
    if ((s = stage_in(g, x, bytes, g->fst, &xd)) || (s = out_buf(g, y, bytes, g->ust, &yd))) return s;
    launch_stencil<double, double2, double2>(ST_APPLY, level_view<double>(g, 0), shift_H(g),
                                             (const double2 *)xd, 0, (const double2 *)nullptr, 0,
                                             (double2 *)yd, 0, 1, 0.0, nullptr, g->st);
    if ((s = check_cuda("helm_apply_H"))) return s;
    if ((s = copy_out(g, y, yd, bytes))) return s;
    return sync_stream(g, "helm_apply_H");
}

helm_status helm_apply_M(helm_grid *g, int level, const helm_c128 *x, helm_c128 *y) {
    clear_error();
    if (!g || !x || !y) return fail(HELM_ERR_ARG, "null argument");
    helm_status s;
    if ((s = ensure_ready(g))) return s;
    if (level < 0 || level >= (int)g->lv.size()) return fail(HELM_ERR_ARG, "no level %d", level);
    if ((s = ensure_level_work(g, 1))) return s;
    const size_t Nl = g->lv[level].N;
    const size_t bytes = Nl * sizeof(double2);
    const void *xd;
    void *yd;
    if ((s = stage_in(g, x, bytes, g->fst, &xd)) || (s = out_buf(g, y, bytes, g->ust, &yd))) return s;
    if (g->vc_prec == HELM_PREC_F64) {
        launch_stencil<double, double2, double2>(ST_APPLY, level_view<double>(g, level),
                                                 shift_M<double>(g), (const double2 *)xd, 0,
                                                 (const double2 *)nullptr, 0, (double2 *)yd, 0, 1,
                                                 0.0, nullptr, g->st);
    } else {
        float2 *xf = g->lv[level].t.as<float2>(), *yf = g->lv[level].r.as<float2>();
        launch_convert<double2, float2>((const double2 *)xd, 0, xf, 0, Nl, 1, g->st);
        launch_stencil<float, float2, float2>(ST_APPLY, level_view<float>(g, level),
                                              shift_M<float>(g), xf, 0, (const float2 *)nullptr, 0,
                                              yf, 0, 1, 0.0f, nullptr, g->st);
        launch_convert<float2, double2>(yf, 0, (double2 *)yd, 0, Nl, 1, g->st);
    }
    if ((s = check_cuda("helm_apply_M"))) return s;
    if ((s = copy_out(g, y, yd, bytes))) return s;
    return sync_stream(g, "helm_apply_M");
}

helm_status helm_apply_precond(helm_grid *g, const helm_c128 *r, helm_c128 *z) {
    clear_error();
    if (!g || !r || !z) return fail(HELM_ERR_ARG, "null argument");
    helm_status s;
    if ((s = ensure_ready(g))) return s;
    if ((s = ensure_level_work(g, 1))) return s;
    const size_t N = g->N;
    const size_t bytes = N * sizeof(double2);
    const void *rd;
    void *zd;
    if ((s = stage_in(g, r, bytes, g->fst, &rd)) || (s = out_buf(g, z, bytes, g->ust, &zd))) return s;
    if (g->opt.precond == HELM_PRECOND_NONE) {
        cudaMemcpyAsync(zd, rd, bytes, cudaMemcpyDeviceToDevice, g->st);
    } else if (g->vc_prec == HELM_PREC_F64) {
        vcycle<double>(g, (const double2 *)rd, N, (double2 *)zd, N, 1, nullptr);
    } else {
        float2 *bf = g->lv[0].b.as<float2>(), *uf = g->lv[0].u.as<float2>();
        launch_convert<double2, float2>((const double2 *)rd, 0, bf, 0, N, 1, g->st);
        vcycle<float>(g, bf, N, uf, N, 1, nullptr);
        launch_convert<float2, double2>(uf, 0, (double2 *)zd, 0, N, 1, g->st);
    }
    if ((s = check_cuda("helm_apply_precond"))) return s;
    if ((s = copy_out(g, z, zd, bytes))) return s;
    return sync_stream(g, "helm_apply_precond");
}

helm_status helm_true_residual(helm_grid *g, const helm_c128 *f, const helm_c128 *u, double *rel) {
    clear_error();
    if (!g || !f || !u || !rel) return fail(HELM_ERR_ARG, "null argument");
    if (!g->has_model) return fail(HELM_ERR_STATE, "helm_set_model has not been called");
    helm_status s;
    const size_t N = g->N;
    const size_t bytes = N * sizeof(double2);
    const void *fd, *ud;
    if ((s = stage_in(g, f, bytes, g->fst, &fd)) || (s = stage_in(g, u, bytes, g->xst, &ud))) return s;
    if ((s = g->yst.ensure(bytes)) || (s = g->nrm.ensure(2 * sizeof(double))) ||
        (s = g->partial.ensure((size_t)4 * 152 * sizeof(double2))) ||
        (s = g->counter.ensure(sizeof(unsigned))))
        return s;
    if (g->cap_rhs == 0) cudaMemsetAsync(g->counter.p, 0, sizeof(unsigned), g->st);
    KrylovScratch ks;
    ks.partial = g->partial.as<double2>();
    ks.counter = g->counter.as<unsigned>();
    ks.max_blocks = 4 * 152;
    ks.nvec_max = 1;
    double2 *r = g->yst.as<double2>();
    launch_stencil<double, double2, double2>(ST_RESID, level_view<double>(g, 0), shift_H(g),
                                             (const double2 *)ud, 0, (const double2 *)fd, 0, r, 0,
                                             1, 0.0, nullptr, g->st);
    double *nd = g->nrm.as<double>();
    launch_norm2(r, 0, N, nd, 1, nullptr, ks, g->st);
    launch_norm2((const double2 *)fd, 0, N, nd + 1, 1, nullptr, ks, g->st);
    double hn[2];
    cudaMemcpyAsync(hn, nd, 2 * sizeof(double), cudaMemcpyDeviceToHost, g->st);
    if ((s = sync_stream(g, "helm_true_residual"))) return s;
    *rel = (hn[1] > 0.0) ? std::sqrt(hn[0] / hn[1]) : 0.0;
    return HELM_OK;
}

}  // extern "C"
