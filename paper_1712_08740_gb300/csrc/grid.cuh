// Library-side state of one helm_grid: model, multigrid hierarchy, coarse
// inverse and the Krylov workspace, all resident in device memory.
#pragma once

#include <string>
#include <vector>

#include "../../include/helm.h"
#include "helm_internal.cuh"

namespace helm {

helm_status fail(helm_status s, const char *fmt, ...);
void clear_error();

// A device allocation that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    helm_status ensure(size_t b);
    void release();
    template <typename P> P *as() const { return static_cast<P *>(p); }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
};

struct MGLevel {
    int n[3] = {1, 1, 1};
    int dim = 1;
    double h = 0.0;
    size_t N = 0;
    DevBuf m;                  // slowness on this level (injected)
    DevBuf rho64, rho32;       // rho of Eq. 1 (variable density only; injected)
    DevBuf w64, w32;           // omega^2 m^2
    DevBuf dinv;               // 1 / diagonal of M, V-cycle precision (complex)
    DevBuf u, t, b, r;         // V-cycle work vectors, [cap_rhs][N] in the V-cycle type
};

}  // namespace helm

struct helm_grid {
    int dim = 0;
    int n[3] = {1, 1, 1};
    double h = 0.0;
    size_t N = 0;
    cudaStream_t st = 0;
    helm_options opt{};
    bool has_model = false;
    bool has_rho = false;      // a variable density (Eq. 1) is set
    bool ready = false;        // hierarchy + coarse inverse match model/shift/options
    double omega = 0.0, alpha = 0.0, beta1 = 1.0, beta2 = 0.5;

    std::vector<helm::MGLevel> lv;      // lv[0] is the fine grid
    std::vector<int> tile_dn, tile_up;  // fused-kernel tile shape per fine level (helm_autotune)
    int vc_prec = -1;                   // precision the hierarchy was built for
    int nc = 0;                         // coarse inverse order
    helm::DevBuf Ainv, colbuf;          // coarse inverse (transposed) and Gauss-Jordan column
    helm::DevBuf Atc;                   // complex64 inverse as TF32 hi/lo tensor-core tiles
    helm::DevBuf cpart, cticket;        // coarse product scratch: group sums, tickets
    int cpart_rhs = 0;                  // right-hand sides cpart/cticket are sized for

    // Krylov workspace
    int cap_rhs = 0, cap_m = 0, cap_prec = -1, cap_side = -1;
    helm::DevBuf V, Z, hbuf, nrm, yv, partial, counter, act_it, act_cy, act2, flag;
    helm::DevBuf cR, cg, ccs, csn, cfn, cbeta, crel, ck, cits, cstat, cany, cQ;   // FGMRES state
    helm::DevBuf fst, ust, xst, yst;    // staging for host pointers / helper vectors
    helm::DevBuf rbuf;                  // residuals in complex128 (double-single basis), or H x
                                        // before M^-1 (left and two-sided preconditioning)
    helm::DevBuf tnrm;                  // true-residual norms of the left/two-sided sides
    helm::DevBuf hdiag;                 // diagonal of H as double-single pairs
    helm::DevBuf c64sc;                 // complex64 basis: 1/||w|| per right-hand side, float hi + lo
    bool hdiag_ok = false;              // hdiag matches the current model
    int *hflag = nullptr;               // host-mapped "any right-hand side active" flag
    std::vector<cudaEvent_t> ring;      // look-ahead events of the Arnoldi loop

    // block FGMRES workspace (helm_options.block): complex64 basis, Z and the
    // new block with a padded per-vector stride; tensor-core scratch; the
    // block Hessenberg, its reflectors and the least-squares right-hand sides
    helm::DevBuf bV, bZ, bW, bpart, bimg, bG, bR, bRinv, bHb, bg, bVh, btau, bpub, bticket;
    helm::DevBuf best, bflags, bY, bfn, bnp, bncnt, bnrm;
    int bcap_m = 0;
    int bls_epoch = 0;
    int *bhflag = nullptr;              // host-mapped "cycle goes on" flag

    // Krylov recycling (helm_options.recycle): [C | V] per right-hand side,
    // U and Ut, Z, Ritz scratch; kept across solves while the shape stays
    helm::DevBuf rCV, rU, rUt, rZ, rNew, rRes, rH, rB, rWt, rcC, rcU, rScr, rhb, rc, rpart, rcnt, rbad;
    helm::DevBuf rupd, rhas;            // per right-hand side: update now / holds a recycled space
    int rec_nrhs = 0, rec_k = 0, rec_m = 0, rec_prec = -1;
    bool rec_any = false;               // some right-hand side holds a recycled space
    bool rec_stale = false;             // the operator changed: rebuild U and C from Ut

    // CUDA graphs of one Arnoldi step per j, valid for graph_key
    std::vector<cudaGraphExec_t> step_graphs;
    std::vector<uint64_t> step_launches;                           // kernels per step graph
    std::vector<std::vector<helm::ProfRecPublic>> step_prof;       // timing nodes per graph
    long long graph_key = -1;
    cudaStream_t cap_st = nullptr;      // private stream used only for capture
    bool use_graphs = true;
    int last_nrhs = 0;                  // batch size of the last solve (kernel timing)
};
