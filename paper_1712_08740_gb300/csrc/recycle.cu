// Krylov-subspace recycling across restarts and across the solves of a
// frequency sweep: GCRO-DR (Parks, de Sturler et al.) with the right
// preconditioning of Eq. 7, for every right-hand side of a batch in
// lock-step (helm_options.recycle = k > 0).
//
// Each right-hand side keeps k recycled vectors: Ut in the preconditioned
// variable, U = M^-1 Ut in the solution space and C = H U with orthonormal
// columns. Arnoldi runs on (I - C C^H) H M^-1: the basis is stored as
// [C_0..C_{k-1} | V_0..V_m] per right-hand side, so the fused H z_j + multi-dot
// and the multi-axpy of the ordinary step orthogonalise the new vector against
// C and V in one pass each; the coefficients against C form B_m. A right-hand
// side without a recycled space yet (its first cycle) holds zero C, U and Ut:
// its coefficients against C are exact zeros and every kernel does the same
// arithmetic for it as for the others, so a right-hand side's result does not
// depend on the rest of its batch. With
// H [U, Z_m] = [C, V_{m+1}] Ghat, Ghat = [[I, B_m], [0, Hbar_m]], a cycle
// takes y_z from the usual least squares (Givens, device) and y_u = -B_m y_z.
// A cycle that ends unconverged replaces the recycled space by the k
// harmonic Ritz vectors of the k smallest |theta| over span([Ut, V_m]):
// Ghat^H Ghat p = theta Ghat^H (What^H [Ut, V_m]) p, solved per right-hand
// side by subspace iteration through the thin QR of Ghat (k_rec_ritz, FP64),
// then recombined through the thin QR of Ghat P so that C stays orthonormal
// (What = [C, V_{m+1}] is orthonormal). A new
// solve on a new H and M (the next frequency) keeps Ut: U = M^-1 Ut, C = H U,
// orthonormalised with the same column operations on U and Ut, and the
// initial guess gains U C^H r0.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cycle.cuh"
#include "vcycle.cuh"

namespace helm {

namespace {

constexpr int kRecMax = 16;     // recycled vectors per right-hand side
constexpr int kRecRestart = 40; // largest restart with recycling (Ritz problem size)
constexpr int kRitzThreads = 256;
constexpr int kRitzIters = 24;  // subspace iterations for the harmonic Ritz space

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {   // conj(a) b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cscal(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// After the multi-dot of step j: hb[r][0 .. kc) = C^H w (column j of B),
// hb[r][kc .. kc + j] = V^H w (column j of Hbar), ||w||^2 in nrm[r]. The
// whole column of Hbar is written, zeros below the subdiagonal included.
__global__ void k_rec_store(const double2 *__restrict__ hb, int hstride, int kc, int j,
                            const double *__restrict__ nrm, double2 *__restrict__ Hraw,
                            double2 *__restrict__ B, int m, int k, const int *__restrict__ act) {
    const int r = blockIdx.x;
    if (act && !act[r]) return;
    const double2 *h = hb + (size_t)r * hstride;
    double2 *hr = Hraw + (size_t)r * (m + 1) * m + (size_t)j * (m + 1);
    double2 *br = B + (size_t)r * k * m + (size_t)j * k;
    for (int i = threadIdx.x; i < kc; i += blockDim.x) br[i] = h[i];
    for (int i = threadIdx.x; i <= m; i += blockDim.x)
        hr[i] = i <= j ? h[kc + i] : (i == j + 1 ? make_double2(sqrt(nrm[r]), 0.0) : make_double2(0.0, 0.0));
}

// c[r][i] = -sum_{l < k_r} B[r][i][l] y[r][l] (i < kc): the recycled part
// of the cycle's update, x += U c
__global__ void k_rec_by(const double2 *__restrict__ B, const double2 *__restrict__ y, int ystride,
                         const int *__restrict__ kcount, int kc, int m, int k, double2 *__restrict__ c,
                         const int *__restrict__ act) {
    const int r = blockIdx.x, i = threadIdx.x;
    if ((act && !act[r]) || i >= kc) return;
    const int kr = kcount[r];
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < kr; ++l) acc = cadd(acc, cmul(B[(size_t)r * k * m + (size_t)l * k + i], y[(size_t)r * ystride + l]));
    c[(size_t)r * k + i] = make_double2(-acc.x, -acc.y);
}

// beta = ||r|| after the projection r -= C C^H r; the next cycle starts from it
__global__ void k_rec_beta(CycleState S, const double *__restrict__ nrm, int nrhs) {
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
        if (!S.act_cy[r]) continue;
        const double b = sqrt(nrm[r]);
        S.beta[r] = b;
        S.g[(size_t)r * (S.m + 1)] = make_double2(b, 0.0);
    }
}

// Harmonic Ritz subspace per right-hand side (one block each, FP64).
// In: Hraw ((m+1) x m), B (kc x m), Wt ((kc+m+1) x kc) = [C, V_{m+1}]^H Ut.
// Out: coefC ((kc+m+1) x kn) and coefU ((kc+m) x kn), column-major, with
//   C_new = [C, V_0..V_m] coefC,  Ut_new = [Ut, V_0..V_{m-1}] coefU,
//   U_new = [U, Z_0..Z_{m-1}] coefU.
// With the thin QR Ghat = Qg Rg, Ghat^H Ghat p = theta Ghat^H Wtil p becomes
// Rg p = theta (Qg^H Wtil) p, so the wanted p are the dominant eigenvectors
// of Mr = Rg^-1 Qg^H Wtil (eigenvalues 1 / theta), taken by subspace
// iteration; no normal-equations matrix is formed. Then Ghat P = Q2 R2 (thin
// QR): coefC = Q2 and coefU = P R2^-1, so C_new has orthonormal columns as far
// as [C, V] has. Every QR is classical Gram-Schmidt twice, the dot products
// of one column taken by all warps at once.
// Scratch per right-hand side: Ghat -> Qg ((n+1) x n), Rg (n x n),
// X -> Mr (n x n, later Ghat P), P and T (n x kn).
struct RitzArgs {
    const double2 *Hraw, *B, *Wt;
    double2 *coefC, *coefU;
    double2 *scratch;
    size_t scratch_per_rhs;
    int *act;                   // cleared where the QR lost a direction: no update there
    int m, kc, k, kn, iters;
    int *bad;
};

constexpr int kRitzWarps = kRitzThreads / 32;
constexpr int kRitzMaxN = kRecMax + kRecRestart + 1;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// In-place thin QR of A (rows x cols, column-major, leading dimension ld) by
// classical Gram-Schmidt twice. R (upper, leading dimension ldr) is written
// when given. d: shared scratch of kRitzMaxN values. Clears *ok on a zero
// column.
__device__ void cgs2_qr(double2 *A, int ld, int rows, int cols, double2 *R, int ldr, double2 *d, double *nr_sh,
                        int *ok) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int c = 0; c < cols; ++c) {
        double2 *ac = A + (size_t)c * ld;
        if (R)
            for (int i = tid; i < cols; i += kRitzThreads) R[(size_t)c * ldr + i] = make_double2(0.0, 0.0);
        for (int pass = 0; pass < 2 && c > 0; ++pass) {
            for (int l = warp; l < c; l += kRitzWarps) {
                const double2 *al = A + (size_t)l * ld;
                double sx = 0.0, sy = 0.0;
                for (int i = lane; i < rows; i += 32) {
                    const double2 t = cconjmul(al[i], ac[i]);
                    sx += t.x;
                    sy += t.y;
                }
                sx = wsum(sx);
                sy = wsum(sy);
                if (lane == 0) d[l] = make_double2(sx, sy);
            }
            __syncthreads();
            for (int i = tid; i < rows; i += kRitzThreads) {
                double2 acc = ac[i];
                for (int l = 0; l < c; ++l) acc = csub(acc, cmul(A[(size_t)l * ld + i], d[l]));
                ac[i] = acc;
            }
            if (R)
                for (int l = tid; l < c; l += kRitzThreads) R[(size_t)c * ldr + l] = cadd(R[(size_t)c * ldr + l], d[l]);
            __syncthreads();
        }
        if (warp == 0) {
            double s = 0.0;
            for (int i = lane; i < rows; i += 32) s += ac[i].x * ac[i].x + ac[i].y * ac[i].y;
            s = wsum(s);
            if (lane == 0) *nr_sh = sqrt(s);
        }
        __syncthreads();
        const double nr = *nr_sh;
        if (tid == 0 && !(nr > 0.0)) *ok = 0;
        const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
        for (int i = tid; i < rows; i += kRitzThreads) ac[i] = cscal(inv, ac[i]);
        if (R && tid == 0) R[(size_t)c * ldr + c] = make_double2(nr, 0.0);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kRitzThreads) k_rec_ritz(RitzArgs a) {
    const int r = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (a.act && !a.act[r]) return;
    const int m = a.m, kc = a.kc, n = kc + m, kn = a.kn, ld1 = n + 1;
    double2 *G = a.scratch + (size_t)r * a.scratch_per_rhs;   // (n+1) x n: Ghat, then Qg
    double2 *Rg = G + (size_t)ld1 * n;                          // n x n, upper
    double2 *X = Rg + (size_t)n * n;                            // n x n: Mr, later Ghat P
    double2 *P = X + (size_t)n * n;                             // n x kn
    double2 *T = P + (size_t)n * kn;                            // n x kn
    const double2 *Hr = a.Hraw + (size_t)r * (m + 1) * m;
    const double2 *Br = a.B + (size_t)r * a.k * m;
    const double2 *Wr = a.Wt + (size_t)r * a.k * (a.k + m + 1);
    const double2 zero = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0);
    __shared__ double2 d[kRitzMaxN];
    __shared__ double2 R2[kRecMax * kRecMax];
    __shared__ double nr_sh;
    __shared__ int ok;
    if (tid == 0) ok = 1;
    // Ghat = [[I_kc, B], [0, Hbar]]
    for (int e = tid; e < ld1 * n; e += kRitzThreads) {
        const int i = e % ld1, c = e / ld1;
        double2 v = zero;
        if (c < kc) v = (i == c) ? one : zero;
        else if (i < kc) v = Br[(size_t)(c - kc) * a.k + i];
        else v = Hr[(size_t)(c - kc) * (m + 1) + (i - kc)];
        G[e] = v;
    }
    __syncthreads();
    cgs2_qr(G, ld1, ld1, n, Rg, n, d, &nr_sh, &ok);
    // X = Qg^H Wtil: column c < kc from Wt, column c >= kc is the unit vector e_c
    for (int e = tid; e < n * n; e += kRitzThreads) {
        const int i = e % n, c = e / n;
        double2 s = zero;
        if (c < kc) {
            for (int l = 0; l < ld1; ++l) s = cadd(s, cconjmul(G[(size_t)i * ld1 + l], Wr[(size_t)c * (a.k + m + 1) + l]));
        } else {
            const double2 q = G[(size_t)i * ld1 + c];
            s = make_double2(q.x, -q.y);
        }
        X[e] = s;
    }
    __syncthreads();
    // Mr = Rg^-1 X: one warp per column, back substitution with the lanes over rows
    for (int c = warp; c < n; c += kRitzWarps) {
        double2 *x = X + (size_t)c * n;
        for (int i = n - 1; i >= 0; --i) {
            const double2 rii = Rg[(size_t)i * n + i];
            const double2 xi = cscal(rii.x > 0.0 ? 1.0 / rii.x : 0.0, x[i]);
            __syncwarp();
            for (int q = lane; q < i; q += 32) x[q] = csub(x[q], cmul(Rg[(size_t)i * n + q], xi));
            if (lane == 0) x[i] = xi;
            __syncwarp();
        }
    }
    // subspace iteration on Mr from the last kn unit vectors (the newest
    // Krylov directions); its dominant eigenvalues are 1 / theta of the
    // smallest |theta|
    for (int e = tid; e < n * kn; e += kRitzThreads) {
        const int i = e % n, c = e / n;
        P[e] = (i == n - kn + c) ? one : zero;
    }
    __syncthreads();
    for (int it = 0; it < a.iters; ++it) {
        for (int e = tid; e < n * kn; e += kRitzThreads) {
            const int i = e % n, c = e / n;
            double2 s = zero;
            for (int l = 0; l < n; ++l) s = cadd(s, cmul(X[(size_t)l * n + i], P[(size_t)c * n + l]));
            T[e] = s;
        }
        __syncthreads();
        cgs2_qr(T, n, n, kn, nullptr, 0, d, &nr_sh, &ok);
        for (int e = tid; e < n * kn; e += kRitzThreads) P[e] = T[e];
        __syncthreads();
    }
    // Ghat P = Qg (Rg P): Y = Rg P into T, then Qg Y into X ((n+1) x kn)
    for (int e = tid; e < n * kn; e += kRitzThreads) {
        const int i = e % n, c = e / n;
        double2 s = zero;
        for (int l = i; l < n; ++l) s = cadd(s, cmul(Rg[(size_t)l * n + i], P[(size_t)c * n + l]));
        T[e] = s;
    }
    __syncthreads();
    double2 *Qp = X;
    for (int e = tid; e < ld1 * kn; e += kRitzThreads) {
        const int i = e % ld1, c = e / ld1;
        double2 s = zero;
        for (int l = 0; l < n; ++l) s = cadd(s, cmul(G[(size_t)l * ld1 + i], T[(size_t)c * n + l]));
        Qp[e] = s;
    }
    __syncthreads();
    cgs2_qr(Qp, ld1, ld1, kn, R2, kn, d, &nr_sh, &ok);
    // coefC = Q2; coefU = P R2^-1 (x_c = (p_c - sum_{l<c} x_l R2(l, c)) / R2(c, c), one thread per row)
    double2 *cC = a.coefC + (size_t)r * (a.k + m + 1) * a.k;
    double2 *cU = a.coefU + (size_t)r * (a.k + m) * a.k;
    for (int e = tid; e < ld1 * kn; e += kRitzThreads) {
        const int i = e % ld1, c = e / ld1;
        cC[(size_t)c * ld1 + i] = Qp[e];
    }
    for (int i = tid; i < n; i += kRitzThreads) {
        for (int c = 0; c < kn; ++c) {
            double2 s = P[(size_t)c * n + i];
            for (int l = 0; l < c; ++l) s = csub(s, cmul(cU[(size_t)l * n + i], R2[c * kn + l]));
            const double rcc = R2[c * kn + c].x;
            cU[(size_t)c * n + i] = cscal(rcc > 0.0 ? 1.0 / rcc : 0.0, s);
        }
    }
    if (tid == 0 && !ok) {
        a.bad[r] = 1;
        a.act[r] = 0;
    }
}

// out[r][i] = sum_l A_l coef[l][i] + sum_l Bv_l coef[na + l][i] (i < kn):
// na vectors A (complex128) and nb vectors Bv (CB) per right-hand side;
// coef column-major with leading dimension ldc, per right-hand side stride cs
template <typename CB>
__global__ void __launch_bounds__(256)
k_rec_combine(const double2 *__restrict__ A, size_t sa, int na, const CB *__restrict__ Bv, size_t sb, int nb,
              const double2 *__restrict__ coef, int ldc, size_t cs, int kn, double2 *__restrict__ out, size_t so,
              size_t N, const int *__restrict__ act) {
    const int r = blockIdx.y;
    if (act && !act[r]) return;
    __shared__ double2 cf[(kRecMax + kRecRestart + 1) * kRecMax];
    const double2 *cr = coef + (size_t)r * cs;
    for (int e = threadIdx.x; e < (na + nb) * kn; e += blockDim.x) {
        const int l = e % (na + nb), i = e / (na + nb);
        cf[i * (na + nb) + l] = cr[(size_t)i * ldc + l];
    }
    __syncthreads();
    const double2 *Ar = A + (size_t)r * sa;
    const CB *Br = Bv + (size_t)r * sb;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        double2 acc[kRecMax];
#pragma unroll
        for (int i = 0; i < kRecMax; ++i) acc[i] = make_double2(0.0, 0.0);
        for (int l = 0; l < na + nb; ++l) {
            const double2 v = l < na ? Ar[(size_t)l * N + p] : cvt<double2>(Br[(size_t)(l - na) * N + p]);
#pragma unroll
            for (int i = 0; i < kRecMax; ++i)
                if (i < kn) acc[i] = cadd(acc[i], cmul(v, cf[i * (na + nb) + l]));
        }
#pragma unroll
        for (int i = 0; i < kRecMax; ++i)
            if (i < kn) out[(size_t)r * so + (size_t)i * N + p] = acc[i];
    }
}

template <typename CB>
void launch_rec_combine(const double2 *A, size_t sa, int na, const CB *Bv, size_t sb, int nb, const double2 *coef,
                        int ldc, size_t cs, int kn, double2 *out, size_t so, size_t N, int nrhs, const int *act,
                        cudaStream_t st) {
    const size_t bx = std::min<size_t>((N + 255) / 256, 1024);
    prof_begin(st);
    k_rec_combine<CB><<<dim3((unsigned)bx, nrhs), 256, 0, st>>>(A, sa, na, Bv, sb, nb, coef, ldc, cs, kn, out, so, N,
                                                              act);
    count_launch();
    if (prof_on())
        prof_end("rec_combine", st, ((double)na * 16.0 + nb * sizeof(CB) + kn * 16.0) * N * nrhs,
                 8.0 * (na + nb) * kn * N * nrhs);
}

// phase 0 (before the cycle-end test): upd[r] = this cycle took all m steps;
// phase 1 (after it): upd[r] &= the right-hand side goes on
__global__ void k_rec_mark(CycleState S, int *__restrict__ upd, int nrhs, int phase) {
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
        if (phase == 0) upd[r] = S.act_cy[r] && S.k[r] == S.m;
        else upd[r] = upd[r] && S.act_cy[r];
    }
}

// the new recycled space into place: nw = [C_new | Ut_new | U_new] (k vectors
// each) per right-hand side; has[r] = 1 from now on
__global__ void k_rec_place(const double2 *__restrict__ nw, size_t snw, double2 *__restrict__ C, size_t sC,
                            double2 *__restrict__ Ut, double2 *__restrict__ U, size_t sU, size_t kN,
                            const int *__restrict__ upd, int *__restrict__ has) {
    const int r = blockIdx.y;
    if (!upd[r]) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) has[r] = 1;
    const double2 *src = nw + (size_t)r * snw;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < kN; p += (size_t)gridDim.x * blockDim.x) {
        C[(size_t)r * sC + p] = src[p];
        Ut[(size_t)r * sU + p] = src[kN + p];
        U[(size_t)r * sU + p] = src[2 * kN + p];
    }
}

}  // namespace

// ------------------------------------------------------------------ solver
helm_status solve_recycle_device(helm_grid *g, int nrhs, const double2 *f, double tol, double2 *u,
                                 int *iterations, double *relres_out, bool warm) {
    helm_status s;
    if ((s = ensure_ready(g))) return s;
    if ((s = workspace_for(g, nrhs))) return s;   // cycle state, level work, scratch sizes
    cudaStream_t st = g->st;
    const size_t N = g->N;
    const int m = g->opt.restart, k = g->opt.recycle;
    const bool f64 = g->opt.precision == HELM_PREC_F64;
    const int nv = k + m + 1;                 // [C | V] vectors per right-hand side
    const size_t sCV = (size_t)nv * N, sU = (size_t)k * N, sZ = (size_t)m * N;
    const int hstride = 2 * nv;
    // workspace (kept across solves while shape, k and m stay)
    const bool fresh = g->rec_nrhs != nrhs || g->rec_k != k || g->rec_m != m || g->rec_prec != g->opt.precision;
    const size_t zsz = f64 ? sizeof(double2) : sizeof(float2);
    const size_t n_r = (size_t)k + m;
    const size_t scratch_per = (n_r + 1) * n_r + 2 * n_r * n_r + 2 * n_r * k;
    const size_t R = nrhs;
    if ((s = g->rCV.ensure(R * sCV * sizeof(double2))) || (s = g->rU.ensure(R * sU * sizeof(double2))) ||
        (s = g->rUt.ensure(R * sU * sizeof(double2))) || (s = g->rZ.ensure(R * sZ * zsz)) ||
        (s = g->rNew.ensure(R * 3 * sU * sizeof(double2))) || (s = g->rRes.ensure(R * N * sizeof(double2))) ||
        (s = g->rH.ensure(R * (m + 1) * m * sizeof(double2))) || (s = g->rB.ensure(R * k * m * sizeof(double2))) ||
        (s = g->rWt.ensure(R * k * nv * sizeof(double2))) || (s = g->rcC.ensure(R * k * nv * sizeof(double2))) ||
        (s = g->rcU.ensure(R * k * (k + m) * sizeof(double2))) ||
        (s = g->rScr.ensure(R * scratch_per * sizeof(double2))) || (s = g->rhb.ensure(R * hstride * sizeof(double2))) ||
        (s = g->rc.ensure(R * k * sizeof(double2))) || (s = g->rpart.ensure(R * kMaxBlocks * nv * sizeof(double2))) ||
        (s = g->rcnt.ensure(R * sizeof(unsigned))) || (s = g->rupd.ensure(R * sizeof(int))) ||
        (s = g->rhas.ensure(R * sizeof(int))) || (s = g->rbad.ensure(R * sizeof(int))))
        return s;
    double2 *CV = g->rCV.as<double2>();
    double2 *V = CV + (size_t)k * N;          // V_i at V + i N, C_i at CV + i N
    double2 *U = g->rU.as<double2>(), *Ut = g->rUt.as<double2>();
    int *upd = g->rupd.as<int>(), *has = g->rhas.as<int>();
    if (fresh) {
        // no recycled space: zero C, U and Ut
        cudaMemset2DAsync(CV, sCV * sizeof(double2), 0, sU * sizeof(double2), R, st);
        cudaMemsetAsync(U, 0, R * sU * sizeof(double2), st);
        cudaMemsetAsync(Ut, 0, R * sU * sizeof(double2), st);
        cudaMemsetAsync(has, 0, R * sizeof(int), st);
        cudaMemsetAsync(g->rcnt.p, 0, R * sizeof(unsigned), st);
        g->rec_any = false;
        g->rec_nrhs = nrhs;
        g->rec_k = k;
        g->rec_m = m;
        g->rec_prec = g->opt.precision;
    }
    cudaMemsetAsync(g->rbad.p, 0, R * sizeof(int), st);
    KrylovScratch ks;
    ks.partial = g->rpart.as<double2>();
    ks.counter = g->rcnt.as<unsigned>();
    ks.max_blocks = kMaxBlocks;
    ks.nvec_max = nv;
    double2 *hb = g->rhb.as<double2>();
    double *nrm = g->nrm.as<double>();
    double2 *rc = g->rc.as<double2>();
    double2 *res = g->rRes.as<double2>();
    const CycleState S = [&] {
        CycleState q;
        q.m = m;
        q.R = g->cR.as<double2>();
        q.g = g->cg.as<double2>();
        q.cs = g->ccs.as<double>();
        q.sn = g->csn.as<double2>();
        q.Q = g->cQ.as<double2>();
        q.fnorm = g->cfn.as<double>();
        q.beta = g->cbeta.as<double>();
        q.relres = g->crel.as<double>();
        q.k = g->ck.as<int>();
        q.its = g->cits.as<int>();
        q.status = g->cstat.as<int>();
        q.act_it = g->act_it.as<int>();
        q.act_cy = g->act_cy.as<int>();
        q.any_dev = g->cany.as<int>();
        q.ticket = reinterpret_cast<unsigned *>(g->cany.as<int>() + 8);
        return q;
    }();
    const LevelView<double> L0 = level_view<double>(g, 0);
    const OpShift<double> sH = shift_H(g);
    // r -= C C^H r and x += U C^H r (r in V_0), ||r||^2 into nrm
    auto project = [&](const int *act) {
        launch_multidot(CV, sCV, k, V, sCV, N, rc, k, nrhs, act, ks, st);
        launch_update<double2>(U, sU, k, rc, k, u, N, N, nrhs, act, st);
        launch_multiaxpy(CV, sCV, k, rc, k, V, sCV, N, nrm, nrhs, act, ks, st);
    };
    // z = M^-1 x (x complex128), complex128 output
    auto precond = [&](const double2 *x, size_t sx, double2 *z, size_t sz, const int *act) {
        if (f64) {
            vcycle<double, double2>(g, x, sx, z, sz, nrhs, act);
        } else {
            float2 *t = g->lv[0].u.as<float2>();
            vcycle<float, double2>(g, x, sx, t, N, nrhs, act);
            launch_convert<float2, double2>(t, N, z, sz, N, nrhs, st);
        }
    };
    // a new operator (frequency) for the right-hand sides that hold a
    // recycled space: U = M^-1 Ut, C = H U, orthonormalised (modified
    // Gram-Schmidt twice) with the same column operations on U and Ut
    if (g->rec_any && g->rec_stale) {
        for (int i = 0; i < k; ++i) {
            // every right-hand side (Ut = 0 gives U = 0 where there is no space)
            precond(Ut + (size_t)i * N, sU, U + (size_t)i * N, sU, nullptr);
            launch_stencil<double, double2, double2>(ST_APPLY, L0, sH, U + (size_t)i * N, sU,
                                                     (const double2 *)nullptr, 0, CV + (size_t)i * N, sCV, nrhs,
                                                     0.0, has, st);
        }
        for (int i = 0; i < k; ++i) {
            for (int pass = 0; pass < 2 && i > 0; ++pass) {
                launch_multidot(CV, sCV, i, CV + (size_t)i * N, sCV, N, rc, k, nrhs, has, ks, st);
                launch_multiaxpy(CV, sCV, i, rc, k, CV + (size_t)i * N, sCV, N, nullptr, nrhs, has, ks, st);
                launch_multiaxpy(U, sU, i, rc, k, U + (size_t)i * N, sU, N, nullptr, nrhs, has, ks, st);
                launch_multiaxpy(Ut, sU, i, rc, k, Ut + (size_t)i * N, sU, N, nullptr, nrhs, has, ks, st);
            }
            launch_norm2(CV + (size_t)i * N, sCV, N, nrm, nrhs, has, ks, st);
            launch_scale<double2>(CV + (size_t)i * N, sCV, nrm, CV + (size_t)i * N, sCV, N, nrhs, has, st);
            launch_scale<double2>(U + (size_t)i * N, sU, nrm, U + (size_t)i * N, sU, N, nrhs, has, st);
            launch_scale<double2>(Ut + (size_t)i * N, sU, nrm, Ut + (size_t)i * N, sU, N, nrhs, has, st);
        }
    }
    g->rec_stale = false;
    // start: x = x0 (or 0), ||f||, r_0 = f - H x0 into V_0, projected on C-perp
    int *flag = g->flag.as<int>();
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    launch_finite_check((const double *)f, 2 * N * (size_t)nrhs, flag, st);
    if (warm) launch_finite_check((const double *)u, 2 * N * (size_t)nrhs, flag, st);
    else cudaMemsetAsync(u, 0, (size_t)nrhs * N * sizeof(double2), st);
    launch_norm2(f, N, N, nrm, nrhs, nullptr, ks, st);
    launch_cycle_init(S, nrm, nrhs, g->hflag, st);
    launch_zero_inactive(u, N, S.act_cy, nrhs, st);
    launch_stencil<double, double2, double2>(ST_RESID, L0, sH, u, N, f, N, V, sCV, nrhs, 0.0, S.act_cy, st);
    launch_norm2(V, sCV, N, nrm, nrhs, S.act_cy, ks, st);
    launch_cycle_check(S, nrm, nrhs, tol, g->opt.max_iters, g->hflag, st);
    project(S.act_cy);
    k_rec_beta<<<1, 256, 0, st>>>(S, nrm, nrhs);
    count_launch();
    int bad = 0;
    cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if ((s = sync_stream(g, "recycling solve start"))) return s;
    if (bad) return fail(HELM_ERR_NONFINITE, "right-hand side or initial guess contains NaN or Inf");
    std::vector<int> hupd(nrhs);
    while (*(volatile int *)g->hflag) {
        launch_scale<double2>(V, sCV, nrm, V, sCV, N, nrhs, S.act_cy, st);
        for (int j = 0; j < m; ++j) {
            const int *act = S.act_it;
            double2 *Zj = nullptr;
            float2 *Zf = nullptr;
            if (f64) {
                Zj = g->rZ.as<double2>() + (size_t)j * N;
                vcycle<double, double2>(g, V + (size_t)j * N, sCV, Zj, sZ, nrhs, act);
            } else {
                Zf = g->rZ.as<float2>() + (size_t)j * N;
                vcycle<float, double2>(g, V + (size_t)j * N, sCV, Zf, sZ, nrhs, act);
            }
            double2 *w = V + (size_t)(j + 1) * N;
            // against [C_0 .. C_{k-1} | V_0 .. V_j]
            if (f64)
                launch_multidot_h<double2>(CV, sCV, k + j + 1, w, sCV, N, hb, hstride, nrhs, act, ks, L0, sH, Zj, sZ,
                                           st);
            else
                launch_multidot_h<float2>(CV, sCV, k + j + 1, w, sCV, N, hb, hstride, nrhs, act, ks, L0, sH, Zf, sZ,
                                          st);
            launch_multiaxpy(CV, sCV, k + j + 1, hb, hstride, w, sCV, N, nrm, nrhs, act, ks, st);
            k_rec_store<<<nrhs, 64, 0, st>>>(hb, hstride, k, j, nrm, g->rH.as<double2>(), g->rB.as<double2>(), m, k,
                                           act);
            count_launch();
            // v_{j+1} = w / ||w|| for every right-hand side of this step (the
            // recycled-space update reads V_m even where the cycle stops),
            // then the least-squares update alone
            launch_scale<double2>(w, sCV, nrm, w, sCV, N, nrhs, act, st);
            launch_givens_scale<double2>(S, j, hb + k, hstride, 0, nrm, nrhs, tol, g->opt.max_iters, g->hflag,
                                         (double2 *)nullptr, sCV, N, st);
            if ((s = sync_stream(g, "recycling step"))) return s;
            if (!*(volatile int *)g->hflag) break;
        }
        // end of cycle: y_z, x += Z y_z + U (-B y_z), the true residual (into
        // its own buffer: the recycled-space update still reads V_0)
        launch_backsolve(S, g->yv.as<double2>(), nrhs, st);
        if (f64)
            launch_update<double2>(g->rZ.as<double2>(), sZ, m, g->yv.as<double2>(), m, u, N, N, nrhs, S.act_cy, st, S.k);
        else
            launch_update<float2>(g->rZ.as<float2>(), sZ, m, g->yv.as<double2>(), m, u, N, N, nrhs, S.act_cy, st, S.k);
        k_rec_by<<<nrhs, kRecMax, 0, st>>>(g->rB.as<double2>(), g->yv.as<double2>(), m, S.k, k, m, k, rc, S.act_cy);
        count_launch();
        launch_update<double2>(U, sU, k, rc, k, u, N, N, nrhs, S.act_cy, st);
        launch_stencil<double, double2, double2>(ST_RESID, L0, sH, u, N, f, N, res, N, nrhs, 0.0, S.act_cy, st);
        launch_norm2(res, N, N, nrm, nrhs, S.act_cy, ks, st);
        k_rec_mark<<<1, 256, 0, st>>>(S, upd, nrhs, 0);
        count_launch();
        launch_cycle_check(S, nrm, nrhs, tol, g->opt.max_iters, g->hflag, st);
        k_rec_mark<<<1, 256, 0, st>>>(S, upd, nrhs, 1);
        count_launch();
        cudaMemcpyAsync(hupd.data(), upd, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st);
        if ((s = sync_stream(g, "recycling cycle end"))) return s;
        if (!*(volatile int *)g->hflag) break;
        // a new recycled space for every right-hand side that goes on after a
        // cycle of all m steps (the full Arnoldi relation)
        bool any = false;
        for (int q = 0; q < nrhs; ++q) any = any || hupd[q];
        if (any) {
            // What^H Ut ((k + m + 1) x k per right-hand side), column i from a multi-dot
            for (int i = 0; i < k; ++i)
                launch_multidot(CV, sCV, k + m + 1, Ut + (size_t)i * N, sU, N,
                                g->rWt.as<double2>() + (size_t)i * (k + m + 1), (size_t)k * (k + m + 1), nrhs, upd,
                                ks, st);
            RitzArgs ra;
            ra.Hraw = g->rH.as<double2>();
            ra.B = g->rB.as<double2>();
            ra.Wt = g->rWt.as<double2>();
            ra.coefC = g->rcC.as<double2>();
            ra.coefU = g->rcU.as<double2>();
            ra.scratch = g->rScr.as<double2>();
            ra.scratch_per_rhs = scratch_per;
            ra.act = upd;
            ra.m = m;
            ra.kc = k;
            ra.k = k;
            ra.kn = k;
            ra.iters = kRitzIters;
            ra.bad = g->rbad.as<int>();
            prof_begin(st);
            k_rec_ritz<<<nrhs, kRitzThreads, 0, st>>>(ra);
            count_launch();
            if (prof_on()) prof_end("rec_ritz", st, 0.0, 0.0);
            double2 *nw = g->rNew.as<double2>();
            const size_t sNew = 3 * sU;
            // C_new = [C, V_0..V_m] coefC; Ut_new = [Ut, V_0..V_{m-1}] coefU; U_new = [U, Z] coefU
            launch_rec_combine<double2>(CV, sCV, k, V, sCV, m + 1, g->rcC.as<double2>(), k + m + 1,
                                        (size_t)(k + m + 1) * k, k, nw, sNew, N, nrhs, upd, st);
            launch_rec_combine<double2>(Ut, sU, k, V, sCV, m, g->rcU.as<double2>(), k + m, (size_t)(k + m) * k, k,
                                        nw + sU, sNew, N, nrhs, upd, st);
            if (f64)
                launch_rec_combine<double2>(U, sU, k, g->rZ.as<double2>(), sZ, m, g->rcU.as<double2>(), k + m,
                                            (size_t)(k + m) * k, k, nw + 2 * sU, sNew, N, nrhs, upd, st);
            else
                launch_rec_combine<float2>(U, sU, k, g->rZ.as<float2>(), sZ, m, g->rcU.as<double2>(), k + m,
                                           (size_t)(k + m) * k, k, nw + 2 * sU, sNew, N, nrhs, upd, st);
            const size_t bx = std::min<size_t>((sU + 255) / 256, 1024);
            k_rec_place<<<dim3((unsigned)bx, nrhs), 256, 0, st>>>(nw, sNew, CV, sCV, Ut, U, sU, sU, upd, has);
            count_launch();
            g->rec_any = true;
        }
        // the next cycle starts from the true residual, made orthogonal to C
        cudaMemcpy2DAsync(V, sCV * sizeof(double2), res, N * sizeof(double2), N * sizeof(double2), nrhs,
                          cudaMemcpyDeviceToDevice, st);
        project(S.act_cy);
        k_rec_beta<<<1, 256, 0, st>>>(S, nrm, nrhs);
        count_launch();
    }
    std::vector<int> its(nrhs), stat(nrhs);
    std::vector<double> rel(nrhs);
    std::vector<int> rb(nrhs);
    cudaMemcpyAsync(its.data(), S.its, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(stat.data(), S.status, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(rel.data(), S.relres, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(rb.data(), g->rbad.p, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st);
    if ((s = sync_stream(g, "recycling solve end"))) return s;
    bool all_conv = true;
    int ritz_bad = -1, broke = -1;
    for (int q = 0; q < nrhs; ++q) {
        if (iterations) iterations[q] = its[q];
        if (relres_out) relres_out[q] = rel[q];
        all_conv = all_conv && stat[q] == ST_CONVERGED;
        if (stat[q] == ST_BROKE && broke < 0) broke = q;
        if (rb[q] && ritz_bad < 0) ritz_bad = q;
    }
    if (broke >= 0)
        return fail(HELM_ERR_BREAKDOWN, "right-hand side %d: a non-finite value after %d iterations%s", broke,
                    its[broke], rb[broke] ? " (its recycled-space QR had lost a direction)" : "");
    if (ritz_bad >= 0)
        return fail(HELM_ERR_BREAKDOWN, "right-hand side %d: the QR of its recycled space lost a direction",
                    ritz_bad);
    if (!all_conv) return fail(HELM_ERR_NOT_CONVERGED, "not converged within %d iterations", g->opt.max_iters);
    return HELM_OK;
}

}  // namespace helm
