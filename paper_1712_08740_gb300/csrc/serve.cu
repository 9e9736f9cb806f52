// Serving front end: a request loop that solves Helmholtz problems of
// different grid sizes, frequencies, media and source counts as they arrive.
//
// Design. A dispatcher thread takes requests from a FIFO queue and hands each
// to an idle worker. Every worker owns a CUDA stream and keeps one grid (model
// buffers, multigrid hierarchy, Krylov basis, captured step graphs) resident
// between requests of the same size, so a request only pays for its own model
// upload and coarse-grid factorisation. Admission is by device memory: a
// request's footprint (Krylov basis x restart length, multigrid work vectors,
// coefficients, coarse inverse, staging) is computed up front, and the head of
// the queue is admitted only when the footprints held by all workers plus its
// own fit the budget; idle workers drop their cached grids when that makes
// room. Requests that arrive while others are on the GPU start as soon as a
// worker and memory free up, and their kernels overlap on the device with the
// others' (independent streams). All right-hand sides of a request are solved
// together by the batched solver.
#include <atomic>
#include <chrono>
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "vcycle.cuh"

namespace helm {

namespace {

using clk = std::chrono::steady_clock;

struct Req {
    uint64_t id = 0;
    int dim = 2;
    int n[3] = {1, 1, 1};
    double h = 0.0;
    std::vector<double> m;
    double omega = 0.0, alpha = 0.0;
    int nrhs = 0;
    std::vector<double2> f;
    double tol = 0.0;
    helm_c128 *u_out = nullptr;
    uint64_t key = 0;           // hash of grid, slowness, omega, alpha and tol (coalescing)
    size_t footprint = 0;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    helm_status status = HELM_OK;
    int its_max = 0;
    double rel_max = 0.0;
    bool done = false;
    std::string err;
};

struct Worker {
    std::thread th;
    cudaStream_t st = nullptr;
    helm_grid *grid = nullptr;
    int gdim = 0, gn[3] = {0, 0, 0};
    double gh = 0.0;
    size_t held = 0;            // bytes held by the cached grid (or the running job)
    std::vector<std::shared_ptr<Req>> jobs;   // requests solved together (one lock-step batch)
    bool busy = false;
};

// FNV-1a over bytes
uint64_t fnv(uint64_t h, const void *p, size_t n) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

// requests that one lock-step batch may serve together: the same operator and tolerance
bool same_problem(const Req &a, const Req &b) {
    return a.key == b.key && a.dim == b.dim && a.n[0] == b.n[0] && a.n[1] == b.n[1] && a.n[2] == b.n[2] &&
           a.h == b.h && a.omega == b.omega && a.alpha == b.alpha && a.tol == b.tol && a.m == b.m;
}

bool same_grid(const Worker &w, const Req &r) {
    return w.grid && w.gdim == r.dim && w.gn[0] == r.n[0] && w.gn[1] == r.n[1] && w.gn[2] == r.n[2] &&
           w.gh == r.h;
}

}  // namespace

// Device bytes a solve of nrhs right-hand sides on this grid holds (upper estimate).
size_t solve_footprint(int dim, const int n[3], int nrhs, const helm_options &o) {
    const double N = (double)n[0] * n[1] * n[2];
    const int m = o.restart;
    const double zsz = (o.precond == HELM_PRECOND_NONE) ? 0.0 : (o.precision == HELM_PREC_F64 ? 16.0 : 8.0);
    const double csz = (o.precision == HELM_PREC_F64) ? 16.0 : 8.0;
    // level sizes by the same rule as the hierarchy
    int c[3] = {n[0], n[1], n[2]};
    double level_N[32];
    int nlev = 0;
    while (nlev < 32) {
        const double Nl = (double)c[0] * c[1] * c[2];
        level_N[nlev++] = Nl;
        bool odd = true;
        for (int a = 0; a < dim; ++a) odd = odd && c[a] >= 3 && (c[a] % 2) == 1;
        if (o.precond != HELM_PRECOND_MG || Nl <= o.coarse_max || !odd) break;
        for (int a = 0; a < dim; ++a) c[a] = (c[a] + 1) / 2;
    }
    const double nc = (double)c[0] * c[1] * c[2];
    // every device buffer as the solver allocates it; the driver hands out
    // large allocations in whole 2 MiB pages
    double b = 0.0;
    auto add = [&](double bytes) {
        const double page = 2.0 * 1024 * 1024;
        b += bytes > page / 2 ? std::ceil(bytes / page) * page : bytes;
    };
    if (o.block) {
        // block FGMRES: complex64 basis, Z and new block for 64 sources with
        // a padded stride, tensor-core scratch, block Hessenberg and reflectors
        const double Np = std::ceil(N / 8.0) * 8.0, S = 64.0, nv = m * S, ldh = (m + 1.0) * S;
        add((m + 1.0) * S * Np * 8.0);
        add(m * S * Np * 8.0);
        add(S * Np * 8.0);
        add((double)block_gram_part_floats((int)nv, (size_t)Np) * 4.0);
        add((double)block_image_floats((int)nv) * 4.0);
        add(ldh * nv * 16.0);                            // block Hessenberg
        add(ldh * S * 16.0 + nv * (S + 1) * 16.0 + 2.0 * nv * S * 16.0);
        add(S * N * 16.0);                               // complex128 residual block
    } else {
        add(nrhs * (m + 1.0) * N * (o.precision == HELM_PREC_MIXED_C64 ? 8.0 : 16.0));   // basis V
        if (zsz > 0.0) add(nrhs * (double)m * N * zsz);  // preconditioned vectors Z
    }
    for (int l = 0; l < nlev; ++l) {                     // per level of the hierarchy
        const double Nl = level_N[l];
        for (int k = 0; k < 4; ++k) add(nrhs * Nl * csz);  // V-cycle work vectors
        add(Nl * 8.0);                                   // slowness
        add(Nl * 8.0);                                   // coefficient (FP64)
        add(Nl * 4.0);                                   // coefficient (FP32)
        add(Nl * csz);                                   // 1/diag(M)
    }
    if (o.precond != HELM_PRECOND_NONE) {
        add(nc * nc * csz);                              // coarse inverse
        add(nc * csz);                                   // Gauss-Jordan column
        double part = (double)coarse_part_elems((int)nc, nrhs) * csz;
        if (csz == 8.0) {
            // complex64: TF32 tensor-core tiles of the inverse and their partial products
            add((double)coarse_tc_tile_floats((int)nc) * 4.0);
            part = std::max(part, (double)coarse_tc_part_floats((int)nc, nrhs) * 4.0);
        }
        add(part);
        add(coarse_tickets((int)nc, nrhs) * 4.0);
    }
    add(nrhs * N * 16.0);                                // staging of host f
    add(nrhs * N * 16.0);                                // staging of host u
    if (o.precision == HELM_PREC_MIXED_DS || o.precision == HELM_PREC_MIXED_C64) {
        add(nrhs * N * 16.0);                            // complex128 residuals
        add(N * 16.0);                                   // diagonal of H, double-single
    } else if (o.side != HELM_SIDE_RIGHT && o.precond != HELM_PRECOND_NONE) {
        add(nrhs * N * 16.0);                            // H x before M^-1
    }
    add((double)nrhs * (m + 1.0) * m * 16.0);            // rotated Hessenberg R
    add((double)nrhs * (m + 1.0) * (m + 1.0) * 16.0);    // rotation product Q
    add((double)nrhs * 2.0 * (m + 1.0) * 16.0);          // Hessenberg column buffer
    {
        double per_rhs = (m + 1.0) * kMaxBlocks;         // reduction partials
        if (o.precision == HELM_PREC_MIXED_DS)
            per_rhs = std::max(per_rhs, (double)ds_partial_per_rhs((size_t)N, m + 1));
        add((double)nrhs * per_rhs * 16.0);
    }
    b += 4.0 * 1024 * 1024;                              // small buffers and captured graphs
    return (size_t)b;
}

}  // namespace helm

struct helm_server {
    std::mutex mu;
    std::condition_variable cv_disp, cv_done, cv_work;
    std::deque<std::shared_ptr<helm::Req>> queue;
    std::map<uint64_t, std::shared_ptr<helm::Req>> reqs;
    std::vector<std::unique_ptr<helm::Worker>> workers;
    size_t budget = 0;
    int coalesce = 0;           // most right-hand sides of one merged batch (<= 1: off)
    helm_options opt{};
    double beta1 = 1.0, beta2 = 0.5;
    bool stop = false;
    uint64_t next_id = 1;
    int device = 0;
    std::thread dispatcher;
    helm::clk::time_point t0;
    double now() const { return std::chrono::duration<double>(helm::clk::now() - t0).count(); }
};

namespace helm {
namespace {

// Solves a group of requests with the same operator as one lock-step batch
// (a single request directly into its output).
void run_group(helm_server *S, Worker &w, std::vector<std::shared_ptr<Req>> &grp) {
    Req &r = *grp[0];
    helm_status s = HELM_OK;
    if (!same_grid(w, r)) {
        if (w.grid) helm_destroy_grid(w.grid);
        w.grid = nullptr;
        int64_t n64[3] = {r.n[0], r.n[1], r.n[2]};
        s = helm_create_grid(r.dim, n64, r.h, &w.grid);
        if (s == HELM_OK) {
            w.gdim = r.dim;
            for (int a = 0; a < 3; ++a) w.gn[a] = r.n[a];
            w.gh = r.h;
            s = helm_set_stream(w.grid, w.st);
        }
    }
    if (s == HELM_OK) s = helm_set_options(w.grid, &S->opt);
    if (s == HELM_OK) s = helm_set_model(w.grid, r.m.data(), r.omega, r.alpha);
    if (s == HELM_OK) s = helm_set_shift(w.grid, S->beta1, S->beta2);
    const size_t N = r.m.size();
    int tot = 0;
    for (auto &q : grp) tot += q->nrhs;
    std::vector<int> its(tot, 0);
    std::vector<double> rel(tot, 0.0);
    if (s == HELM_OK) {
        if (grp.size() == 1) {
            s = helm_solve_batch(w.grid, r.nrhs, reinterpret_cast<const helm_c128 *>(r.f.data()), r.tol,
                                 r.u_out, its.data(), rel.data());
        } else {
            // the members' right-hand sides in order, one solve, the solutions back
            std::vector<double2> f((size_t)tot * N), u((size_t)tot * N);
            size_t off = 0;
            for (auto &q : grp) {
                memcpy(f.data() + off, q->f.data(), q->f.size() * sizeof(double2));
                off += q->f.size();
            }
            s = helm_solve_batch(w.grid, tot, reinterpret_cast<const helm_c128 *>(f.data()), r.tol,
                                 reinterpret_cast<helm_c128 *>(u.data()), its.data(), rel.data());
            off = 0;
            for (auto &q : grp) {
                const size_t bytes = (size_t)q->nrhs * N * sizeof(double2);
                if (cudaMemcpy(q->u_out, u.data() + off, bytes, cudaMemcpyDefault) != cudaSuccess && s == HELM_OK) {
                    cudaGetLastError();
                    s = fail(HELM_ERR_CUDA, "copy of a merged request's solution");
                }
                off += (size_t)q->nrhs * N;
            }
        }
    }
    const std::string err = s != HELM_OK ? std::string(helm_last_error()) : std::string();
    int k0 = 0;
    for (auto &q : grp) {
        q->status = s;
        q->err = err;
        bool all_met = true;
        for (int k = 0; k < q->nrhs; ++k) {
            q->its_max = std::max(q->its_max, its[k0 + k]);
            q->rel_max = std::max(q->rel_max, rel[k0 + k]);
            all_met = all_met && rel[k0 + k] <= q->tol;
        }
        // in a merged batch that did not converge as a whole, a member whose
        // own right-hand sides all met the tolerance gets the status of its
        // solve alone (right preconditioning stops on this true residual)
        if (s == HELM_ERR_NOT_CONVERGED && grp.size() > 1 && all_met && S->opt.side == HELM_SIDE_RIGHT) {
            q->status = HELM_OK;
            q->err.clear();
        }
        k0 += q->nrhs;
        q->f.clear();
        q->f.shrink_to_fit();
    }
    if (s != HELM_OK && s != HELM_ERR_NOT_CONVERGED && w.grid) {   // do not keep a grid in a bad state
        helm_destroy_grid(w.grid);
        w.grid = nullptr;
    }
}

void worker_loop(helm_server *S, Worker *w) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_work.wait(lk, [&] { return S->stop || !w->jobs.empty(); });
        if (w->jobs.empty()) break;
        std::vector<std::shared_ptr<Req>> grp = w->jobs;
        lk.unlock();
        run_group(S, *w, grp);
        lk.lock();
        const double t = S->now();
        for (auto &q : grp) {
            q->t_done = t;
            q->done = true;
        }
        w->jobs.clear();
        w->busy = false;
        w->held = w->grid ? std::max(w->held, grp[0]->footprint) : 0;
        S->cv_done.notify_all();
        S->cv_disp.notify_all();
    }
    if (w->grid) helm_destroy_grid(w->grid);
    w->grid = nullptr;
}

void dispatch_loop(helm_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        if (S->queue.empty()) {
            S->cv_disp.wait(lk);
            continue;
        }
        std::shared_ptr<Req> r = S->queue.front();
        // the group it leads: queued requests of the same problem, in arrival
        // order, up to `coalesce` right-hand sides and within the budget
        std::vector<std::shared_ptr<Req>> grp{r};
        size_t gfp = r->footprint;
        if (S->coalesce > 1) {
            int tot = r->nrhs;
            for (auto &q : S->queue) {
                if (q == r || tot + q->nrhs > S->coalesce || !same_problem(*q, *r)) continue;
                const size_t fp = solve_footprint(r->dim, r->n, tot + q->nrhs, S->opt);
                if (fp > S->budget) break;
                grp.push_back(q);
                tot += q->nrhs;
                gfp = fp;
            }
        }
        // idle worker, preferring one whose resident grid has this size
        Worker *pick = nullptr;
        for (auto &w : S->workers)
            if (!w->busy && same_grid(*w, *r)) { pick = w.get(); break; }
        if (!pick)
            for (auto &w : S->workers)
                if (!w->busy && (!pick || w->held < pick->held)) pick = w.get();
        if (!pick) {
            S->cv_disp.wait(lk);
            continue;
        }
        const bool reuse = same_grid(*pick, *r);
        const size_t need = reuse ? std::max(pick->held, gfp) : gfp;
        size_t others = 0;
        for (auto &w : S->workers)
            if (w.get() != pick) others += w->held;
        // grids dropped here are freed after the lock is released: freeing
        // device memory synchronises the device, and the workers' completions
        // must not wait for that behind the server lock
        std::vector<helm_grid *> doomed;
        auto release = [&] {
            if (doomed.empty()) return;
            lk.unlock();
            for (helm_grid *dg : doomed) helm_destroy_grid(dg);
            lk.lock();
            doomed.clear();
        };
        if (others + need > S->budget) {
            // make room by dropping grids cached by idle workers
            for (auto &w : S->workers) {
                if (w.get() == pick || w->busy || !w->grid) continue;
                doomed.push_back(w->grid);
                w->grid = nullptr;
                others -= w->held;
                w->held = 0;
                if (others + need <= S->budget) break;
            }
        }
        if (others + need > S->budget) {
            if (others == 0) {   // can never fit: reject instead of waiting forever
                S->queue.pop_front();
                r->status = HELM_ERR_NOMEM;
                r->err = "request footprint exceeds the server's memory budget";
                r->t_admit = r->t_done = S->now();
                r->done = true;
                S->cv_done.notify_all();
                release();
                continue;
            }
            if (!doomed.empty()) {
                release();   // state may have changed meanwhile: decide again
                continue;
            }
            S->cv_disp.wait(lk);   // wait for a running request to release memory
            continue;
        }
        if (!reuse && pick->grid) {
            doomed.push_back(pick->grid);
            pick->grid = nullptr;
        }
        const double ta = S->now();
        for (auto &q : grp) {
            S->queue.erase(std::find(S->queue.begin(), S->queue.end(), q));
            q->t_admit = ta;
            q->footprint = gfp;
        }
        pick->held = need;
        pick->busy = true;
        pick->jobs = grp;
        S->cv_work.notify_all();
        release();
    }
}

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" {

helm_status helm_server_create(const helm_server_config *cfg, helm_server **out) {
    clear_error();
    if (!cfg || !out) return fail(HELM_ERR_ARG, "null argument");
    *out = nullptr;
    if (cfg->workers < 1 || cfg->workers > 64) return fail(HELM_ERR_ARG, "workers must be 1..64");
    if (cfg->memory_budget == 0) return fail(HELM_ERR_ARG, "memory_budget must be > 0");
    auto *S = new helm_server();
    S->budget = cfg->memory_budget;
    S->opt = cfg->options;
    S->beta1 = cfg->beta1;
    S->beta2 = cfg->beta2;
    S->coalesce = cfg->options.block ? 0 : cfg->coalesce;
    S->t0 = clk::now();
    cudaGetDevice(&S->device);
    for (int i = 0; i < cfg->workers; ++i) {
        auto w = std::make_unique<Worker>();
        if (cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto &x : S->workers) cudaStreamDestroy(x->st);
            delete S;
            return fail(HELM_ERR_CUDA, "stream creation");
        }
        S->workers.push_back(std::move(w));
    }
    for (auto &w : S->workers) w->th = std::thread(worker_loop, S, w.get());
    S->dispatcher = std::thread(dispatch_loop, S);
    *out = S;
    return HELM_OK;
}

void helm_server_destroy(helm_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_disp.notify_all();
    S->cv_work.notify_all();
    S->dispatcher.join();
    for (auto &w : S->workers) w->th.join();
    for (auto &w : S->workers) cudaStreamDestroy(w->st);
    delete S;
}

double helm_server_clock(const helm_server *S) { return S ? S->now() : 0.0; }

size_t helm_solve_footprint(int dim, const int64_t n[3], int nrhs, const helm_options *opt) {
    if (!n || !opt || dim < 1 || dim > 3 || nrhs < 1) return 0;
    int nn[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) nn[a] = (int)n[a];
    return solve_footprint(dim, nn, nrhs, *opt);
}

helm_status helm_server_submit(helm_server *S, const helm_request *q, helm_c128 *u, uint64_t *id) {
    clear_error();
    if (!S || !q || !u || !id || !q->m || !q->f) return fail(HELM_ERR_ARG, "null argument");
    if (q->dim < 1 || q->dim > 3 || q->nrhs < 1 || !(q->h > 0.0) || !(q->tol > 0.0 && q->tol < 1.0))
        return fail(HELM_ERR_ARG, "bad request");
    auto r = std::make_shared<Req>();
    r->dim = q->dim;
    size_t N = 1;
    for (int a = 0; a < 3; ++a) {
        r->n[a] = a < q->dim ? (int)q->n[a] : 1;
        if (r->n[a] < (a < q->dim ? 2 : 1)) return fail(HELM_ERR_ARG, "bad grid");
        N *= (size_t)r->n[a];
    }
    r->h = q->h;
    r->m.assign(q->m, q->m + N);
    r->omega = q->omega;
    r->alpha = q->alpha;
    r->nrhs = q->nrhs;
    r->f.resize((size_t)q->nrhs * N);
    memcpy(r->f.data(), q->f, (size_t)q->nrhs * N * sizeof(double2));
    r->tol = q->tol;
    r->u_out = u;
    r->footprint = solve_footprint(r->dim, r->n, r->nrhs, S->opt);
    uint64_t k = 1469598103934665603ull;
    k = fnv(k, r->n, sizeof r->n);
    k = fnv(k, &r->h, sizeof r->h);
    k = fnv(k, &r->omega, sizeof r->omega);
    k = fnv(k, &r->alpha, sizeof r->alpha);
    k = fnv(k, &r->tol, sizeof r->tol);
    r->key = fnv(k, r->m.data(), r->m.size() * sizeof(double));
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = S->next_id++;
        r->t_submit = S->now();
        S->reqs[r->id] = r;
        S->queue.push_back(r);
        *id = r->id;
    }
    S->cv_disp.notify_all();
    return HELM_OK;
}

static void fill_result(const Req &r, helm_result *res) {
    res->id = r.id;
    res->status = r.status;
    res->nrhs = r.nrhs;
    res->iterations_max = r.its_max;
    res->true_rel_residual_max = r.rel_max;
    res->t_submit = r.t_submit;
    res->t_admit = r.t_admit;
    res->t_done = r.t_done;
    res->footprint_bytes = r.footprint;
}

helm_status helm_server_wait(helm_server *S, uint64_t id, helm_result *res) {
    clear_error();
    if (!S || !res) return fail(HELM_ERR_ARG, "null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return fail(HELM_ERR_ARG, "unknown request %llu", (unsigned long long)id);
    std::shared_ptr<Req> r = it->second;
    S->cv_done.wait(lk, [&] { return r->done; });
    fill_result(*r, res);
    S->reqs.erase(id);
    if (r->status != HELM_OK) return fail(r->status, "request %llu: %s", (unsigned long long)id, r->err.c_str());
    return HELM_OK;
}

helm_status helm_server_poll(helm_server *S, uint64_t id, int *done) {
    clear_error();
    if (!S || !done) return fail(HELM_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return fail(HELM_ERR_ARG, "unknown request %llu", (unsigned long long)id);
    *done = it->second->done ? 1 : 0;
    return HELM_OK;
}

}  // extern "C"
