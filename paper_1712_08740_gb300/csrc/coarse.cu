// Coarsest-level solve of the shifted Laplacian (Eq. 6): the level's matrix is
// assembled densely on the device, inverted once per (model, omega, shift) by
// Gauss-Jordan elimination, stored transposed, and applied in every V-cycle
// as a dense product with the level's right-hand sides.
//
// Gauss-Jordan runs without pivoting. D M (D halves boundary rows per face)
// is complex symmetric with a positive-definite imaginary part (beta2 > 0 and
// the outgoing boundary term), so every leading block is non-singular and no
// zero pivot can occur; row scaling by D does not change that.
#include "helm_internal.cuh"

namespace helm {

namespace {

template <typename T> __device__ __forceinline__ T dsqrt(T v);
template <> __device__ __forceinline__ float dsqrt<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double dsqrt<double>(double v) { return sqrt(v); }

template <typename T>
__global__ void k_assemble_dense(LevelView<T> L, OpShift<T> s, cplx_t<T> *__restrict__ A) {
    const int N = L.nx * L.ny * L.nz;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int ix = p % L.nx;
    const int iy = (p / L.nx) % L.ny;
    const int iz = p / (L.nx * L.ny);
    const int coord[3] = {ix, iy, iz};
    const int n[3] = {L.nx, L.ny, L.nz};
    const int stride[3] = {1, L.nx, L.nx * L.ny};
    cplx_t<T> *row = A + (size_t)p * N;
    // neighbour weights c (times the face coefficient of Eq. 1 when rho is
    // set), their sum (Laplacian part of the diagonal) and the boundary factor
    const T rp = L.rho ? L.rho[p] : T(1);
    T dsum = 0, bsum = 0;
    for (int a = 0; a < L.dim; ++a) {
        const int i = coord[a];
        if (i > 0) {
            const T face = L.rho ? T(0.5) * (rp + L.rho[p - stride[a]]) : T(1);
            T c = ((i == n[a] - 1) ? T(2) : T(1)) * face;
            row[p - stride[a]].x += -c * L.inv_h2;
            dsum += c;
            if (i == n[a] - 1) bsum += face;
        }
        if (i < n[a] - 1) {
            const T face = L.rho ? T(0.5) * (rp + L.rho[p + stride[a]]) : T(1);
            T c = ((i == 0) ? T(2) : T(1)) * face;
            row[p + stride[a]].x += -c * L.inv_h2;
            dsum += c;
            if (i == 0) bsum += face;
        }
    }
    if (L.rho) bsum /= dsqrt<T>(rp);
    const T wp = L.w[p];
    T dre = dsum * L.inv_h2 - s.s_re * wp;
    T dim_ = -s.s_im * wp;
    if (bsum != T(0)) {
        const T f = bsum * L.two_over_h * dsqrt<T>(wp);
        dre -= f * s.q_im;
        dim_ += f * s.q_re;
    }
    row[p].x = dre;
    row[p].y = dim_;
}

// Step k, part 1: save column k, then scale row k by 1/a_kk (a_kk <- 1/a_kk).
template <typename T>
__global__ void k_gj_pivot(cplx_t<T> *__restrict__ A, cplx_t<T> *__restrict__ col, int n, int k) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = A[(size_t)i * n + k];
    __syncthreads();
    const cplx_t<T> p = col[k];
    const T den = p.x * p.x + p.y * p.y;
    const T ir = p.x / den, ii = -p.y / den;       // 1 / p
    cplx_t<T> *rk = A + (size_t)k * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        cplx_t<T> v = (j == k) ? mk<cplx_t<T>>(1.0, 0.0) : rk[j];
        cplx_t<T> o;
        o.x = v.x * ir - v.y * ii;
        o.y = v.x * ii + v.y * ir;
        rk[j] = o;
    }
}

// Step k, part 2: every other row i: a_ij -= a_ik_old * a_kj_new (a_ik_old from col).
template <typename T>
__global__ void k_gj_elim(cplx_t<T> *__restrict__ A, const cplx_t<T> *__restrict__ col, int n,
                          int k) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= n || i == k) return;
    const cplx_t<T> f = col[i];
    const cplx_t<T> rkj = A[(size_t)k * n + j];
    cplx_t<T> a = (j == k) ? mk<cplx_t<T>>(0.0, 0.0) : A[(size_t)i * n + j];
    a.x -= f.x * rkj.x - f.y * rkj.y;
    a.y -= f.x * rkj.y + f.y * rkj.x;
    A[(size_t)i * n + j] = a;
}

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// (re, im) += a v as two FMA chains: four FMA instructions per complex
// multiply-add (the form "re += a.x v.x - a.y v.y" compiles to a multiply, an
// FMA and an add, 1.5x the issue time on GB300's narrow FP64 pipe)
template <typename T>
__device__ __forceinline__ void cmac(T &re, T &im, cplx_t<T> a, cplx_t<T> v) {
    re = fmaT(a.x, v.x, re);
    re = fmaT(-a.y, v.y, re);
    im = fmaT(a.x, v.y, im);
    im = fmaT(a.y, v.x, im);
}

// In-place transpose of the n x n inverse (row-major -> column-major), so
// that consecutive rows of one column are contiguous for the product below.
template <typename T>
__global__ void k_transpose_square(cplx_t<T> *__restrict__ A, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= n || j <= i) return;
    const cplx_t<T> a = A[(size_t)i * n + j];
    A[(size_t)i * n + j] = A[(size_t)j * n + i];
    A[(size_t)j * n + i] = a;
}

// Z_k = Ainv R_k for nb right-hand sides, Ainv stored column-major (At).
//
// The arithmetic per (row i, right-hand side k) depends only on n: the
// columns are split into G(n) groups of width cw = ceil(n / G); in a group
// one lane forms sum_c Ainv[i][c] R_k[c] in column order with two
// accumulators (columns at even and odd offsets from the group start, added
// at the end of the group); the G group sums are then added in group order.
// So batched and single solves agree bitwise whatever tile of right-hand
// sides a warp takes.
//
// Work: a warp owns 32 consecutive rows (one per lane, so each column read is
// one coalesced row of At), one column group and a tile of RT (1 or 4) right-hand
// sides, whose slice of R it stages in shared memory. G is chosen so that
// the single-right-hand-side grid is about one wave of (SMs) x 8 warps with
// every SM given the same number of warps up to one (contiguous task ranges
// per block). Each warp writes its group sums to `part`; the last of the G
// warps of a (row group, right-hand-side tile) to finish (atomic ticket)
// adds them in group order and writes Z.
constexpr int kGemmWarps = 8;

inline int gemm_groups(int n) {
    const int rgs = (n + 31) / 32;
    int G = (device_sms() * kGemmWarps) / rgs;
    if (G < 1) G = 1;
    if (G > 64) G = 64;
    const int gmin = (n + 127) / 128;      // groups of at most 128 columns (shared-memory slice)
    if (G < gmin) G = gmin;
    if (G > n) G = n;
    return G;
}

template <typename T, int RT>
__global__ void __launch_bounds__(kGemmWarps * 32, 1)
k_coarse_gemm(const cplx_t<T> *__restrict__ At, int n, const cplx_t<T> *__restrict__ R, size_t sr,
              cplx_t<T> *__restrict__ Z, size_t sz, int nb, const int *__restrict__ active,
              cplx_t<T> *__restrict__ part, unsigned *__restrict__ ticket, int ntask, int G) {
    using C = cplx_t<T>;
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cw = (n + G - 1) / G;
    const int rgs = (n + 31) / 32;
    // contiguous task range of this block: every SM gets the same count up to one
    const int t0 = (int)((long long)blockIdx.x * ntask / gridDim.x);
    const int t1 = (int)((long long)(blockIdx.x + 1) * ntask / gridDim.x);
    const int task = t0 + warp;
    if (task >= t1) return;                                  // warp-uniform
    const int cg = task % G;
    const int rg = (task / G) % rgs;
    const int kt = task / (G * rgs);
    const int c0 = min(cg * cw, n), c1 = min(c0 + cw, n);
    const int len = c1 - c0;
    const int i = rg * 32 + lane;
    bool use[RT];
#pragma unroll
    for (int k = 0; k < RT; ++k) {
        const int rhs = kt * RT + k;
        use[k] = rhs < nb && (!active || active[rhs]);
    }
    // this warp's slice of the right-hand sides: xs[k * cw + (c - c0)]
    C *xs = reinterpret_cast<C *>(smem_raw) + (size_t)warp * RT * cw;
#pragma unroll
    for (int k = 0; k < RT; ++k) {
        const C *rk = R + (size_t)(kt * RT + k) * sr + c0;
        for (int c = lane; c < len; c += 32) {
            C v;
            v.x = T(0);
            v.y = T(0);
            if (use[k]) v = rk[c];
            xs[k * cw + c] = v;
        }
    }
    __syncwarp();
    T er[RT], ei[RT], orr[RT], oi[RT];
#pragma unroll
    for (int k = 0; k < RT; ++k) er[k] = ei[k] = orr[k] = oi[k] = T(0);
    if (i < n) {
        const C *col = At + (size_t)c0 * n + i;
        const int full = len & ~7;
        // the next chunk of 8 columns is loaded while the current one is used
        C an[8];
        if (full > 0) {
#pragma unroll
            for (int u = 0; u < 8; ++u) an[u] = col[(size_t)u * n];
        }
        int c = 0;
        for (; c < full; c += 8) {
            C a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = an[u];
            if (c + 8 < full) {
#pragma unroll
                for (int u = 0; u < 8; ++u) an[u] = col[(size_t)(c + 8 + u) * n];
            }
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    cmac(er[k], ei[k], a[u], xs[k * cw + c + u]);
                    cmac(orr[k], oi[k], a[u + 1], xs[k * cw + c + u + 1]);
                }
            }
        }
        for (; c < len; ++c) {
            const C a = col[(size_t)c * n];
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                if (c & 1) cmac(orr[k], oi[k], a, xs[k * cw + c]);
                else cmac(er[k], ei[k], a, xs[k * cw + c]);
            }
        }
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            if (!use[k]) continue;
            C v;
            v.x = er[k] + orr[k];
            v.y = ei[k] + oi[k];
            part[((size_t)(kt * RT + k) * G + cg) * n + i] = v;
        }
    }
    // the last warp of this (row group, tile) adds the G group sums in order
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&ticket[kt * rgs + rg], 1u);
        last = (t == (unsigned)G - 1);
        if (last) ticket[kt * rgs + rg] = 0;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    if (i >= n) return;
#pragma unroll
    for (int k = 0; k < RT; ++k) {
        if (!use[k]) continue;
        const C *pk = part + (size_t)(kt * RT + k) * G * n + i;
        C s = __ldcg(pk);
        int q = 1;
        // eight group sums in flight at a time, added in group order
        for (; q + 8 <= G; q += 8) {
            C v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(pk + (size_t)(q + u) * n);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                s.x += v[u].x;
                s.y += v[u].y;
            }
        }
        for (; q < G; ++q) {
            const C v = __ldcg(pk + (size_t)q * n);
            s.x += v.x;
            s.y += v.y;
        }
        Z[(size_t)(kt * RT + k) * sz + i] = s;
    }
}

}  // namespace

template <typename T>
void launch_assemble_dense(const LevelView<T> &L, OpShift<T> s, cplx_t<T> *A, cudaStream_t st) {
    const int N = L.nx * L.ny * L.nz;
    cudaMemsetAsync(A, 0, sizeof(cplx_t<T>) * (size_t)N * N, st);
    k_assemble_dense<T><<<(N + 127) / 128, 128, 0, st>>>(L, s, A);
    count_launch();
}

template <typename T>
void launch_gauss_jordan(cplx_t<T> *A, cplx_t<T> *colbuf, int n, cudaStream_t st) {
    const dim3 blk(32, 8);
    const dim3 grd((n + 31) / 32, (n + 7) / 8);
    prof_begin(st);
    for (int k = 0; k < n; ++k) {
        k_gj_pivot<T><<<1, 1024, 0, st>>>(A, colbuf, n, k);
        k_gj_elim<T><<<grd, blk, 0, st>>>(A, colbuf, n, k);
    }
    count_launch(2ull * n);
    if (prof_on())
        prof_end(sizeof(T) == 8 ? "gauss_jordan_f64" : "gauss_jordan_f32", st,
                 2.0 * n * (double)n * n * sizeof(cplx_t<T>), sizeof(T) == 8 ? 8.0 * n * n * (double)n : 0.0);
}

namespace {

template <typename T, int RT>
void gemm_impl(const cplx_t<T> *At, int n, const cplx_t<T> *r, size_t sr, cplx_t<T> *z, size_t sz,
               int nb, const int *active, cplx_t<T> *part, unsigned *ticket, cudaStream_t st) {
    const int G = gemm_groups(n);
    const int cw = (n + G - 1) / G;
    const int ntask = ((n + 31) / 32) * G * ((nb + RT - 1) / RT);
    const int sms = device_sms();
    const int per_sm = (ntask + sms - 1) / sms;
    // up to 8 warps (tasks) per block; when one wave suffices, one block per SM
    const int blocks = per_sm <= kGemmWarps ? (ntask < sms ? ntask : sms)
                                            : (ntask + kGemmWarps - 1) / kGemmWarps;
    const size_t sm = (size_t)kGemmWarps * RT * cw * sizeof(cplx_t<T>);
    k_coarse_gemm<T, RT><<<blocks, kGemmWarps * 32, sm, st>>>(At, n, r, sr, z, sz, nb, active, part,
                                                              ticket, ntask, G);
}

}  // namespace

void prepare_coarse_kernels() {
    static const int once = [] {   // thread-safe once per process
        const int big = 100 * 1024;
        cudaFuncSetAttribute(k_coarse_gemm<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        cudaFuncSetAttribute(k_coarse_gemm<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        return 1;
    }();
    (void)once;
}

size_t coarse_part_elems(int n, int nb) { return (size_t)nb * gemm_groups(n) * n; }
size_t coarse_tickets(int n, int nb) { return (size_t)((n + 31) / 32) * (size_t)nb; }

template <typename T>
void launch_transpose_square(cplx_t<T> *A, int n, cudaStream_t st) {
    const dim3 blk(32, 8);
    const dim3 grd((n + 31) / 32, (n + 7) / 8);
    k_transpose_square<T><<<grd, blk, 0, st>>>(A, n);
    count_launch();
}

template <typename T>
void launch_dense_gemv(const cplx_t<T> *At, int n, const cplx_t<T> *r, size_t sr,
                       cplx_t<T> *z, size_t sz, int nb, const int *active, void *part,
                       unsigned *ticket, cudaStream_t st) {
    prof_begin(st);
    cplx_t<T> *pp = static_cast<cplx_t<T> *>(part);
    if (nb == 1) gemm_impl<T, 1>(At, n, r, sr, z, sz, nb, active, pp, ticket, st);
    else gemm_impl<T, 4>(At, n, r, sr, z, sz, nb, active, pp, ticket, st);
    count_launch();
    if (prof_on())
        prof_end(sizeof(T) == 8 ? "coarse_gemv_f64" : "coarse_gemv_f32", st,
                 ((double)n * n + 2.0 * n * nb) * sizeof(cplx_t<T>),
                 sizeof(T) == 8 ? 8.0 * n * n * nb : 0.0);
}

template void launch_assemble_dense<float>(const LevelView<float> &, OpShift<float>, float2 *,
                                           cudaStream_t);
template void launch_assemble_dense<double>(const LevelView<double> &, OpShift<double>, double2 *,
                                            cudaStream_t);
template void launch_gauss_jordan<float>(float2 *, float2 *, int, cudaStream_t);
template void launch_gauss_jordan<double>(double2 *, double2 *, int, cudaStream_t);
template void launch_dense_gemv<double>(const double2 *, int, const double2 *, size_t, double2 *,
                                        size_t, int, const int *, void *, unsigned *, cudaStream_t);
template void launch_transpose_square<float>(float2 *, int, cudaStream_t);
template void launch_transpose_square<double>(double2 *, int, cudaStream_t);

}  // namespace helm
