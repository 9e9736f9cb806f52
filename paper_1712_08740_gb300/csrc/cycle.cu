// Device-side bookkeeping of restarted flexible GMRES (Eq. 7), so that a whole
// Arnoldi cycle runs without a host round trip:
//   k_cycle_init   ||f|| and the first cycle's beta, flags
//   k_givens       after each Arnoldi step: new Hessenberg column (from the
//                  two Gram-Schmidt passes and the norm), earlier rotations,
//                  a new complex Givens rotation (real cosine), the residual
//                  estimate |g_{j+1}|, and the stop decision
//   k_backsolve    y = R^-1 g for the steps taken in the cycle
//   k_cycle_check  true residual -> converged / give up / next cycle
// Each kernel publishes "any right-hand side still active" to a host-mapped
// flag that the host polls without synchronising the stream.
#include "helm_internal.cuh"
#include "cycle.cuh"

namespace helm {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }

__global__ void k_cycle_init(CycleState S, const double *__restrict__ nrm2, int nrhs, int *host_flag) {
    int any = 0;
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
        const double fn = sqrt(nrm2[r]);
        S.fnorm[r] = fn;
        S.beta[r] = fn;
        S.its[r] = 0;
        S.k[r] = 0;
        S.relres[r] = 0.0;
        const int live = fn > 0.0;
        S.status[r] = live ? ST_LIVE : ST_CONVERGED;
        S.act_cy[r] = live;
        S.act_it[r] = live;
        S.g[(size_t)r * (S.m + 1)] = make_double2(fn, 0.0);
        S.Q[(size_t)r * (S.m + 1) * (S.m + 1)] = make_double2(1.0, 0.0);
        any |= live;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0 && host_flag) *(volatile int *)host_flag = any;
}

// One warp per right-hand side. The product of the rotations so far is kept
// explicitly, Q_j = G_{j-1} ... G_0 (lower Hessenberg, column-major per
// right-hand side), so rotating the new Hessenberg column is a lane-parallel
// product Q_j h instead of a serial chain of j rotations: on GB300 every FP64
// warp instruction holds the SM's FP64 pipe for ~16 cycles whatever the lane
// mask, so short dependent chains matter. Lane 0 builds the new complex
// rotation (real cosine) from the last two entries; the warp then writes the
// rotated column into R and the two new rows of Q. Entries of Q outside the
// Hessenberg profile are never read, so Q needs no clearing between cycles:
// only Q[0][0] = 1 is set when a cycle starts. "Any right-hand side still
// stepping" is combined across blocks with an atomic and a last-block ticket,
// whose block publishes it to the host-mapped flag.
__global__ void k_givens(CycleState S, int j, const double2 *__restrict__ hb, int hstride, int two,
                         const double *__restrict__ nrm2, int nrhs, double tol, int max_iters,
                         int *host_flag, int *any_dev, unsigned *ticket, int q_in_smem) {
    extern __shared__ unsigned char smem_raw[];
    const int m = S.m;
    const int ld = m + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + warp;
    double2 *h = reinterpret_cast<double2 *>(smem_raw) + (size_t)warp * (2 * ld);
    double2 *rot = h + ld;
    // with one warp per block, Q_j (its Hessenberg profile) is staged in shared memory
    double2 *Qs = (blockDim.x == 32 && q_in_smem) ? rot + ld : nullptr;
    int live = 0;
    if (r < nrhs && S.act_it[r]) {
        double2 *R = S.R + (size_t)r * ld * m + (size_t)j * ld;
        double2 *Q = S.Q + (size_t)r * ld * ld;
        double2 *g = S.g + (size_t)r * ld;
        bool finite = true;
        for (int i = lane; i <= j; i += 32) {
            double2 v = hb[(size_t)r * hstride + i];
            if (two) v = cadd(v, hb[(size_t)r * hstride + ld + i]);
            finite = finite && isfinite(v.x) && isfinite(v.y);
            h[i] = v;
        }
        const double hn = sqrt(nrm2[r]);
        finite = __all_sync(0xffffffffu, finite) && isfinite(hn);
        if (Qs) {
            // columns c <= j of Q_j copied as one contiguous block of (j+1) * ld
            // values (column-major), eight independent loads in flight per lane
            const int nq = (j + 1) * ld;
            for (int t0 = lane; t0 < nq; t0 += 32 * 8) {
                double2 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int t = t0 + 32 * u;
                    if (t < nq) v[u] = Q[t];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int t = t0 + 32 * u;
                    if (t < nq) Qs[t] = v[u];
                }
            }
        }
        __syncwarp();
        const double2 *Qr = Qs ? Qs : Q;
        if (!finite) {
            if (lane == 0) {
                S.status[r] = ST_BROKE;
                S.act_it[r] = 0;
                S.act_cy[r] = 0;
            }
        } else {
            // rotated h: rot[i] = sum_{c <= min(i+1, j)} Q[i][c] h[c]
            for (int i = lane; i <= j; i += 32) {
                const int cmax = min(i + 1, j);
                double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
                int c = 0;
                for (; c + 1 <= cmax; c += 2) {
                    a0 = cadd(a0, cmul(Qr[i + (size_t)c * ld], h[c]));
                    a1 = cadd(a1, cmul(Qr[i + (size_t)(c + 1) * ld], h[c + 1]));
                }
                if (c <= cmax) a0 = cadd(a0, cmul(Qr[i + (size_t)c * ld], h[c]));
                rot[i] = cadd(a0, a1);
            }
            __syncwarp();
            int stop = 0;
            double cs = 0.0;
            double2 sv = make_double2(0.0, 0.0);
            if (lane == 0) {
                const double2 a = rot[j];
                const double2 b = make_double2(hn, 0.0);
                const double aa = cabs2(a), bb = hn;
                double2 rr;
                if (aa == 0.0) {
                    cs = 0.0;
                    sv = make_double2(1.0, 0.0);
                    rr = b;
                } else {
                    const double rho = hypot(aa, bb);
                    const double2 ph = cscale(1.0 / aa, a);
                    cs = aa / rho;
                    sv = cscale(bb / rho, ph);                     // (a/|a|) conj(b) / rho, b real
                    rr = cscale(rho, ph);
                }
                rot[j] = rr;
                S.cs[(size_t)r * m + j] = cs;
                S.sn[(size_t)r * m + j] = sv;
                const double2 gj = g[j];
                g[j + 1] = cscale(-1.0, cconjmul(sv, gj));
                g[j] = cscale(cs, gj);
                S.k[r] = j + 1;
                const int its = S.its[r] + 1;
                S.its[r] = its;
                const double est = cabs2(g[j + 1]);
                stop = (est <= tol * S.fnorm[r] || hn <= 1e-300 || its >= max_iters || j + 1 >= m);
                if (stop) S.act_it[r] = 0;
            }
            cs = __shfl_sync(0xffffffffu, cs, 0);
            sv.x = __shfl_sync(0xffffffffu, sv.x, 0);
            sv.y = __shfl_sync(0xffffffffu, sv.y, 0);
            __syncwarp();
            // rotated column into R (R[j+1][j] = 0)
            for (int i = lane; i <= j + 1; i += 32) R[i] = (i <= j) ? rot[i] : make_double2(0.0, 0.0);
            // rows j and j+1 of Q_{j+1} = G_j diag(Q_j, 1)
            for (int c = lane; c <= j + 1; c += 32) {
                const double2 qj = (c <= j) ? Qr[j + (size_t)c * ld] : make_double2(0.0, 0.0);
                const double2 e = (c == j + 1) ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
                Q[j + (size_t)c * ld] = cadd(cscale(cs, qj), cmul(sv, e));
                Q[j + 1 + (size_t)c * ld] = cadd(cscale(-1.0, cconjmul(sv, qj)), cscale(cs, e));
            }
            live = __shfl_sync(0xffffffffu, stop, 0) ? 0 : 1;
        }
    }
    // any right-hand side still stepping, over all blocks
    const int blk_any = __syncthreads_or(live);
    if (threadIdx.x == 0) {
        if (blk_any) atomicOr(any_dev, 1);
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        if (t == gridDim.x - 1) {
            const int a = atomicExch(any_dev, 0);
            if (host_flag) *(volatile int *)host_flag = a;
            *ticket = 0;
        }
    }
}

// One block per right-hand side: y = R^-1 g for the k steps of the cycle.
// R and g are staged in shared memory when they fit; warp 0 then runs a
// column-oriented substitution (lane-parallel updates after each pivot).
__global__ void k_backsolve(CycleState S, double2 *__restrict__ y, int nrhs, int use_smem) {
    extern __shared__ unsigned char smem_raw[];
    const int m = S.m;
    const int r = blockIdx.x;
    if (r >= nrhs) return;
    double2 *yr = y + (size_t)r * m;
    const int k = S.act_cy[r] ? S.k[r] : 0;
    const double2 *Rg = S.R + (size_t)r * (m + 1) * m;
    double2 *Rs = reinterpret_cast<double2 *>(smem_raw);
    double2 *acc = Rs + (use_smem ? (size_t)(m + 1) * m : 0);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        yr[i] = make_double2(0.0, 0.0);
        acc[i] = i < k ? S.g[(size_t)r * (m + 1) + i] : make_double2(0.0, 0.0);
    }
    if (use_smem)
        for (int t = threadIdx.x; t < (m + 1) * k; t += blockDim.x) Rs[t] = Rg[t];
    const double2 *R = use_smem ? Rs : Rg;
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    for (int i = k - 1; i >= 0; --i) {
        const double2 d = R[i + (size_t)i * (m + 1)];
        const double2 a = acc[i];
        const double den = d.x * d.x + d.y * d.y;
        const double2 yi = make_double2((a.x * d.x + a.y * d.y) / den, (a.y * d.x - a.x * d.y) / den);
        __syncwarp();
        if (lane == 0) yr[i] = yi;
        for (int q = lane; q < i; q += 32) {
            const double2 t = cmul(R[q + (size_t)i * (m + 1)], yi);
            acc[q] = make_double2(acc[q].x - t.x, acc[q].y - t.y);
        }
        __syncwarp();
    }
}

__global__ void k_cycle_check(CycleState S, const double *__restrict__ nrm2, int nrhs, double tol,
                              int max_iters, int *host_flag) {
    int any = 0;
    const int m = S.m;
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
        if (S.act_cy[r]) {
            const double b = sqrt(nrm2[r]);
            S.beta[r] = b;
            S.relres[r] = b / S.fnorm[r];
            if (S.relres[r] <= tol) {
                S.status[r] = ST_CONVERGED;
            } else if (S.its[r] >= max_iters || !isfinite(b)) {
                S.status[r] = isfinite(b) ? ST_MAXIT : ST_BROKE;
            }
        }
        const int live = S.status[r] == ST_LIVE;
        S.act_cy[r] = live;
        S.act_it[r] = live;
        S.k[r] = 0;
        double2 *g = S.g + (size_t)r * (m + 1);
        g[0] = make_double2(live ? S.beta[r] : 0.0, 0.0);
        S.Q[(size_t)r * (m + 1) * (m + 1)] = make_double2(1.0, 0.0);
        any |= live;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0 && host_flag) *(volatile int *)host_flag = any;
}

constexpr int kCycleThreads = 256;

}  // namespace

void launch_cycle_init(const CycleState &S, const double *nrm2, int nrhs, int *host_flag,
                       cudaStream_t st) {
    k_cycle_init<<<1, kCycleThreads, 0, st>>>(S, nrm2, nrhs, host_flag);
    count_launch();
}

void launch_givens(const CycleState &S, int j, const double2 *hb, int hstride, int two,
                   const double *nrm2, int nrhs, double tol, int max_iters, int *host_flag,
                   cudaStream_t st) {
    // small batches: one warp per block with Q_j staged in shared memory
    const size_t ld = S.m + 1;
    const size_t qsm = (2 * ld + ld * ld) * sizeof(double2);
    const bool qs = nrhs <= 2 * 152 && qsm <= 96 * 1024;
    const int warps = qs ? 1 : 4;
    const size_t sm = qs ? qsm : (size_t)warps * 2 * ld * sizeof(double2);
    prof_begin(st);
    k_givens<<<(nrhs + warps - 1) / warps, warps * 32, sm, st>>>(
        S, j, hb, hstride, two, nrm2, nrhs, tol, max_iters, host_flag, S.any_dev, S.ticket, qs ? 1 : 0);
    count_launch();
    if (prof_on()) prof_end("givens", st, 0.0, 0.0);
}

void launch_backsolve(const CycleState &S, double2 *y, int nrhs, cudaStream_t st) {
    const size_t full = ((size_t)(S.m + 1) * S.m + S.m) * sizeof(double2);
    const int use_smem = full <= 96 * 1024;
    const size_t sm = use_smem ? full : S.m * sizeof(double2);
    prof_begin(st);
    k_backsolve<<<nrhs, 128, sm, st>>>(S, y, nrhs, use_smem);
    count_launch();
    if (prof_on()) prof_end("backsolve", st, 0.0, 0.0);
}

void prepare_cycle_kernels() {
    cudaFuncSetAttribute(k_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024 + 8192);
    cudaFuncSetAttribute(k_givens, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024 + 8192);
}

void launch_cycle_check(const CycleState &S, const double *nrm2, int nrhs, double tol,
                        int max_iters, int *host_flag, cudaStream_t st) {
    k_cycle_check<<<1, kCycleThreads, 0, st>>>(S, nrm2, nrhs, tol, max_iters, host_flag);
    count_launch();
}

}  // namespace helm
