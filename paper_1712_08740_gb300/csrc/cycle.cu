// Device-side bookkeeping of restarted flexible GMRES (Eq. 7), so that a whole
// Arnoldi cycle runs without a host round trip:
//   k_cycle_init   ||f|| and the first cycle's beta, flags
//   k_givens_scale after each Arnoldi step: new Hessenberg column (from the
//                  Gram-Schmidt passes and the norm), earlier rotations, a
//                  new complex Givens rotation (real cosine), the residual
//                  estimate |g_{j+1}| and the stop decision, side by side
//                  with the scaling of the new basis vector
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

// Scaling of the new basis vector v_{j+1} = w / ||w|| in the basis type.
template <typename SV> struct ScaleOp;
template <> struct ScaleOp<double2> {
    __device__ static double2 apply(double2 x, double s, float, float) {
        return make_double2(x.x * s, x.y * s);
    }
};
template <> struct ScaleOp<float4> {       // double-single x times double-single s
    __device__ static float4 apply(float4 x, double, float sh, float sl) {
        float4 o;
        {
            const float p = x.x * sh;
            float e = fmaf(x.x, sh, -p);
            e = fmaf(x.x, sl, fmaf(x.y, sh, e));
            o.x = p + e;
            o.y = e - (o.x - p);
        }
        {
            const float p = x.z * sh;
            float e = fmaf(x.z, sh, -p);
            e = fmaf(x.z, sl, fmaf(x.w, sh, e));
            o.z = p + e;
            o.w = e - (o.z - p);
        }
        return o;
    }
};

constexpr int kGivensThreads = 256;

// The end of an Arnoldi step, one launch: one block per right-hand side
// updates its least-squares problem, the other blocks scale w = slot j+1 into
// v_{j+1} = w / ||w||. The two parts only read what the
// Gram-Schmidt kernels wrote, so they run side by side.
//
// Least-squares update. The product of the rotations so far is kept
// explicitly, Q_j = G_{j-1} ... G_0 (lower Hessenberg, column-major per
// right-hand side), so rotating the new Hessenberg column h is the product
// Q_j h rather than a serial chain of j rotations: on GB300 the FP64 pipe
// takes ~16 cycles per warp instruction, so long dependent chains are slow.
// The block stages Q_j in shared memory with every load in flight, forms
// Q_j h with 8 threads per row, and thread 0 builds the new complex rotation
// (real cosine) from the last two entries; the block then writes the rotated
// column into R and the two new rows of Q. Entries of Q outside the
// Hessenberg profile are never read, so Q needs no clearing between cycles:
// only Q[0][0] = 1 is set when a cycle starts. "Any right-hand side still
// stepping" is combined over the right-hand sides with an atomic and a ticket;
// the last least-squares block publishes it to the host-mapped flag.
//
// A scaling block that reads the stop decision of its right-hand side before
// or after block 0 writes it produces the same result for every vector that
// is ever used again: a stopped right-hand side's v_{j+1} is never read.
template <typename SV>
__global__ void __launch_bounds__(kGivensThreads)
k_givens_scale(CycleState S, int j, const double2 *__restrict__ hb, int hstride, int two,
               const double *__restrict__ nrm2, int nrhs, double tol, int max_iters,
               int *host_flag, int q_in_smem, SV *__restrict__ w, size_t sw, size_t N) {
    // blocks in launch order: the nrhs least-squares blocks first (their
    // latency then overlaps the scaling), then nbs scaling blocks per
    // right-hand side
    const int nbs = gridDim.x - 1;
    const long long lin = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    const int tid = threadIdx.x;
    if (lin >= nrhs) {
        const long long ls = lin - nrhs;
        const int r = (int)(ls / nbs);
        const int bx = (int)(ls % nbs);
        if (!S.act_it[r]) return;
        __shared__ double s_sh;
        __shared__ float2 s_ds;
        if (tid == 0) {
            s_sh = 1.0 / sqrt(nrm2[r]);
            s_ds = ds_split(s_sh);
        }
        __syncthreads();
        const double s = s_sh;
        const float2 sd = s_ds;
        SV *wr = w + (size_t)r * sw;
        // four nodes per round, all loads issued first
        const size_t stride = (size_t)nbs * kGivensThreads;
        size_t p = (size_t)bx * kGivensThreads + tid;
        for (; p + 3 * stride < N; p += 4 * stride) {
            const SV a0 = wr[p], a1 = wr[p + stride], a2 = wr[p + 2 * stride], a3 = wr[p + 3 * stride];
            wr[p] = ScaleOp<SV>::apply(a0, s, sd.x, sd.y);
            wr[p + stride] = ScaleOp<SV>::apply(a1, s, sd.x, sd.y);
            wr[p + 2 * stride] = ScaleOp<SV>::apply(a2, s, sd.x, sd.y);
            wr[p + 3 * stride] = ScaleOp<SV>::apply(a3, s, sd.x, sd.y);
        }
        for (; p < N; p += stride) wr[p] = ScaleOp<SV>::apply(wr[p], s, sd.x, sd.y);
        return;
    }
    const int r = (int)lin;
    extern __shared__ unsigned char smem_raw[];
    const int m = S.m;
    const int ld = m + 1;
    double2 *h = reinterpret_cast<double2 *>(smem_raw);
    double2 *rot = h + ld;
    double2 *Qs = q_in_smem ? rot + ld : nullptr;
    __shared__ double sh_cs;
    __shared__ double2 sh_sv;
    __shared__ int sh_stop;
    int live = 0;
    if (S.act_it[r]) {                       // block-uniform
        double2 *R = S.R + (size_t)r * ld * m + (size_t)j * ld;
        double2 *Q = S.Q + (size_t)r * ld * ld;
        double2 *g = S.g + (size_t)r * ld;
        int fin = 1;
        for (int i = tid; i <= j; i += kGivensThreads) {
            double2 v = hb[(size_t)r * hstride + i];
            if (two) v = cadd(v, hb[(size_t)r * hstride + ld + i]);
            fin &= isfinite(v.x) && isfinite(v.y);
            h[i] = v;
        }
        if (Qs) {
            // columns c <= j of Q_j, one contiguous block of (j + 1) * ld values
            const int nq = (j + 1) * ld;
            for (int t = tid; t < nq; t += kGivensThreads) Qs[t] = Q[t];
        }
        const double hn = sqrt(nrm2[r]);
        const int finite = __syncthreads_and(fin) && isfinite(hn);
        const double2 *Qr = Qs ? Qs : Q;
        if (!finite) {
            if (tid == 0) {
                S.status[r] = ST_BROKE;
                S.act_it[r] = 0;
                S.act_cy[r] = 0;
            }
        } else {
            // rot[i] = sum_{c <= min(i+1, j)} Q[i][c] h[c]; a group of 8 lanes per
            // row, every lane of a warp takes the same number of rounds
            const int sub = tid & 7;
            for (int base = 0; base <= j; base += kGivensThreads / 8) {
                const int i = base + (tid >> 3);
                double2 a = make_double2(0.0, 0.0);
                if (i <= j) {
                    const int cmax = min(i + 1, j);
                    for (int c = sub; c <= cmax; c += 8) a = cadd(a, cmul(Qr[i + (size_t)c * ld], h[c]));
                }
                for (int o = 4; o; o >>= 1) {
                    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
                    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
                }
                if (sub == 0 && i <= j) rot[i] = a;
            }
            __syncthreads();
            if (tid == 0) {
                const double2 a = rot[j];
                const double2 b = make_double2(hn, 0.0);
                const double aa = cabs2(a), bb = hn;
                double cs;
                double2 sv, rr;
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
                const int stop = (est <= tol * S.fnorm[r] || hn <= 1e-300 || its >= max_iters || j + 1 >= m);
                if (stop) S.act_it[r] = 0;
                sh_cs = cs;
                sh_sv = sv;
                sh_stop = stop;
            }
            __syncthreads();
            const double cs = sh_cs;
            const double2 sv = sh_sv;
            // rotated column into R (R[j+1][j] = 0)
            for (int i = tid; i <= j + 1; i += kGivensThreads) R[i] = (i <= j) ? rot[i] : make_double2(0.0, 0.0);
            // rows j and j+1 of Q_{j+1} = G_j diag(Q_j, 1)
            for (int c = tid; c <= j + 1; c += kGivensThreads) {
                const double2 qj = (c <= j) ? Qr[j + (size_t)c * ld] : make_double2(0.0, 0.0);
                const double2 e = (c == j + 1) ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
                Q[j + (size_t)c * ld] = cadd(cscale(cs, qj), cmul(sv, e));
                Q[j + 1 + (size_t)c * ld] = cadd(cscale(-1.0, cconjmul(sv, qj)), cscale(cs, e));
            }
            live = !sh_stop;
        }
    }
    // any right-hand side still stepping, over the least-squares blocks
    if (tid == 0) {
        if (live) atomicOr(S.any_dev, 1);
        __threadfence();
        const unsigned t = atomicAdd(S.ticket, 1u);
        if (t == (unsigned)nrhs - 1) {
            const int a = atomicExch(S.any_dev, 0);
            if (host_flag) *(volatile int *)host_flag = a;
            *S.ticket = 0;
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

template <typename SV>
void launch_givens_scale(const CycleState &S, int j, const double2 *hb, int hstride, int two,
                         const double *nrm2, int nrhs, double tol, int max_iters, int *host_flag,
                         SV *w, size_t sw, size_t N, cudaStream_t st) {
    const size_t ld = S.m + 1;
    const size_t qsm = (2 * ld + ld * ld) * sizeof(double2);
    const bool qs = qsm <= 96 * 1024;
    const size_t sm = qs ? qsm : 2 * ld * sizeof(double2);
    // scaling blocks per right-hand side: one node per thread for a single
    // right-hand side; for batches about 1216 blocks in all, so each block's
    // set-up (1/||w|| in FP64) is spread over many nodes
    size_t nbs = (N + kGivensThreads - 1) / kGivensThreads;
    const size_t cap = (size_t)((1216 + nrhs - 1) / nrhs);
    if (nrhs > 1 && nbs > cap) nbs = cap;
    if (nbs < 1) nbs = 1;
    if (nbs > 65535) nbs = 65535;
    if (!w) nbs = 0;   // least-squares blocks only: the caller scales w itself
    prof_begin(st);
    k_givens_scale<SV><<<dim3(1 + (unsigned)nbs, nrhs), kGivensThreads, sm, st>>>(
        S, j, hb, hstride, two, nrm2, nrhs, tol, max_iters, host_flag, qs ? 1 : 0, w, sw, N);
    count_launch();
    if (prof_on()) prof_end("givens_scale", st, 32.0 * N * nrhs, 0.0);
}
template void launch_givens_scale<double2>(const CycleState &, int, const double2 *, int, int,
                                           const double *, int, double, int, int *, double2 *,
                                           size_t, size_t, cudaStream_t);
template void launch_givens_scale<float4>(const CycleState &, int, const double2 *, int, int,
                                          const double *, int, double, int, int *, float4 *,
                                          size_t, size_t, cudaStream_t);

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
    cudaFuncSetAttribute(k_givens_scale<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024 + 8192);
    cudaFuncSetAttribute(k_givens_scale<float4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024 + 8192);
}

void launch_cycle_check(const CycleState &S, const double *nrm2, int nrhs, double tol,
                        int max_iters, int *host_flag, cudaStream_t st) {
    k_cycle_check<<<1, kCycleThreads, 0, st>>>(S, nrm2, nrhs, tol, max_iters, host_flag);
    count_launch();
}

}  // namespace helm
