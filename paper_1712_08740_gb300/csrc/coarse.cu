// Coarsest-level solve of the shifted Laplacian (Eq. 6): the level's matrix is
// assembled densely on the device, inverted once per (model, omega, shift) by
// Gauss-Jordan elimination, and applied in every V-cycle as a dense
// matrix-vector product (one warp per row).
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
    int nf = 0;
    for (int a = 0; a < L.dim; ++a) {
        const int i = coord[a];
        if (i > 0) {
            T c = (i == n[a] - 1) ? T(2) : T(1);
            row[p - stride[a]].x += -c * L.inv_h2;
        } else {
            ++nf;
        }
        if (i < n[a] - 1) {
            T c = (i == 0) ? T(2) : T(1);
            row[p + stride[a]].x += -c * L.inv_h2;
        } else {
            ++nf;
        }
    }
    const T wp = L.w[p];
    T dre = T(2 * L.dim) * L.inv_h2 - s.s_re * wp;
    T dim_ = -s.s_im * wp;
    if (nf) {
        const T f = T(nf) * L.two_over_h * dsqrt<T>(wp);
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

// One quarter of one row of Ainv times one vector, by one warp: columns
// [c0, c1), eight independent accumulators per lane (column j + 32q) keep
// eight row loads in flight, then a fixed combination and shuffle tree.
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// (re, im) += a v as two FMA chains: four FP64 instructions per complex
// multiply-add (the form "re += a.x v.x - a.y v.y" compiles to a multiply, an
// FMA and an add, 1.5x the issue time on GB300's narrow FP64 pipe)
template <typename T>
__device__ __forceinline__ void cmac(T &re, T &im, cplx_t<T> a, cplx_t<T> v) {
    re = fmaT(a.x, v.x, re);
    re = fmaT(-a.y, v.y, re);
    im = fmaT(a.x, v.y, im);
    im = fmaT(a.y, v.x, im);
}

template <typename T>
__device__ __forceinline__ cplx_t<T> quarter_dot(const cplx_t<T> *__restrict__ row,
                                                 const cplx_t<T> *__restrict__ r, int c0, int c1,
                                                 int lane) {
    T are[8] = {0, 0, 0, 0, 0, 0, 0, 0}, aim[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int j = c0 + lane;
    for (; j + 224 < c1; j += 256) {
        cplx_t<T> a[8], v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            a[q] = row[j + 32 * q];
            v[q] = r[j + 32 * q];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            cmac(are[q], aim[q], a[q], v[q]);
        }
    }
    for (; j < c1; j += 32) {
        const cplx_t<T> a = row[j];
        const cplx_t<T> v = r[j];
        cmac(are[0], aim[0], a, v);
    }
    T sre = ((are[0] + are[1]) + (are[2] + are[3])) + ((are[4] + are[5]) + (are[6] + are[7]));
    T sim = ((aim[0] + aim[1]) + (aim[2] + aim[3])) + ((aim[4] + aim[5]) + (aim[6] + aim[7]));
    for (int o = 16; o; o >>= 1) {
        sre += __shfl_xor_sync(0xffffffffu, sre, o);
        sim += __shfl_xor_sync(0xffffffffu, sim, o);
    }
    cplx_t<T> out;
    out.x = sre;
    out.y = sim;
    return out;
}

// Arithmetic per row shared by both GEMV kernels: each row is split into four
// quarters (starting on multiples of 32 columns), a warp forms each quarter's
// dot product (quarter_dot), and the four quarter sums are added in order
// 0..3. The kernels differ only in which warps and blocks handle which rows,
// so batched and single solves agree bitwise.
__device__ __forceinline__ void quarter_range(int n, int q, int &c0, int &c1) {
    const int Q = ((n + 127) / 128) * 32;
    c0 = min(q * Q, n);
    c1 = min((q + 1) * Q, n);
}

// z = Ainv r for one right-hand side. The rows are split into one contiguous
// range per block (one block per SM, 152 blocks), so every SM gets the same
// number of rows up to one; a block of 16 warps runs four rows at a time,
// warp w taking quarter (w % 4) of row slot (w / 4), so each SM sub-partition
// (warp w runs on sub-partition w % 4) gets the same share of the FP64 work
// and four warps per sub-partition hide the load latency.
constexpr int kG1Warps = 16;

template <typename T>
__global__ void __launch_bounds__(kG1Warps * 32, 1)
k_dense_gemv1(const cplx_t<T> *__restrict__ Ainv, int n, const cplx_t<T> *__restrict__ r,
              cplx_t<T> *__restrict__ z, const int *__restrict__ active) {
    if (active && !active[0]) return;
    extern __shared__ unsigned char smem_raw[];
    cplx_t<T> *part = reinterpret_cast<cplx_t<T> *>(smem_raw);   // [row of the block][quarter]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3, slot = warp >> 2;
    const int r0 = (int)((long long)blockIdx.x * n / gridDim.x);
    const int r1 = (int)((long long)(blockIdx.x + 1) * n / gridDim.x);
    int c0, c1;
    quarter_range(n, q, c0, c1);
    for (int i = r0 + slot; i < r1; i += kG1Warps / 4) {
        const cplx_t<T> v = quarter_dot<T>(Ainv + (size_t)i * n, r, c0, c1, lane);
        if (lane == 0) part[(i - r0) * 4 + q] = v;
    }
    __syncthreads();
    // quarters added in order 0..3, as in k_dense_gemv
    for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
        const cplx_t<T> *pq = part + (size_t)(i - r0) * 4;
        cplx_t<T> s = pq[0];
        for (int k = 1; k < 4; ++k) {
            s.x += pq[k].x;
            s.y += pq[k].y;
        }
        z[i] = s;
    }
}

// z_k = Ainv r_k for a tile of up to kRT right-hand sides per block (one row pair)
constexpr int kRT = 4;

template <typename T>
__global__ void __launch_bounds__(256)
k_dense_gemv(const cplx_t<T> *__restrict__ Ainv, int n, const cplx_t<T> *__restrict__ r, size_t sr,
             cplx_t<T> *__restrict__ z, size_t sz, int nb, const int *__restrict__ active) {
    __shared__ cplx_t<T> part[kRT][2][4];
    const int rhs0 = blockIdx.y * kRT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3, half = warp >> 2;
    const int i = 2 * blockIdx.x + half;
    int c0, c1;
    quarter_range(n, q, c0, c1);
    for (int t = 0; t < kRT; ++t) {
        const int k = rhs0 + t;
        if (k >= nb || (active && !active[k]) || i >= n) continue;
        const cplx_t<T> v = quarter_dot<T>(Ainv + (size_t)i * n, r + (size_t)k * sr, c0, c1, lane);
        if (lane == 0) part[t][half][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * kRT) {
        const int t = threadIdx.x >> 1, hh = threadIdx.x & 1;
        const int k = rhs0 + t, row = 2 * blockIdx.x + hh;
        if (k < nb && (!active || active[k]) && row < n) {
            cplx_t<T> s = part[t][hh][0];
            for (int m = 1; m < 4; ++m) {
                s.x += part[t][hh][m].x;
                s.y += part[t][hh][m].y;
            }
            z[(size_t)k * sz + row] = s;
        }
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

template <typename T>
void launch_dense_gemv(const cplx_t<T> *Ainv, int n, const cplx_t<T> *r, size_t sr,
                       cplx_t<T> *z, size_t sz, int nb, const int *active, cudaStream_t st) {
    const int npairs = (n + 1) / 2;
    prof_begin(st);
    if (nb == 1) {
        const int blocks = n < 152 ? n : 152;
        const size_t sm = (size_t)((n + blocks - 1) / blocks) * 4 * sizeof(cplx_t<T>);
        k_dense_gemv1<T><<<blocks, kG1Warps * 32, sm, st>>>(Ainv, n, r, z, active);
    } else
        k_dense_gemv<T><<<dim3(npairs, (nb + kRT - 1) / kRT), 256, 0, st>>>(Ainv, n, r, sr, z, sz, nb,
                                                                             active);
    count_launch();
    if (prof_on())
        prof_end(sizeof(T) == 8 ? "coarse_gemv_f64" : "coarse_gemv_f32", st,
                 ((double)n * n * ((nb + kRT - 1) / kRT) + 2.0 * n * nb) * sizeof(cplx_t<T>),
                 sizeof(T) == 8 ? 8.0 * n * n * nb : 0.0);
}

template void launch_assemble_dense<float>(const LevelView<float> &, OpShift<float>, float2 *,
                                           cudaStream_t);
template void launch_assemble_dense<double>(const LevelView<double> &, OpShift<double>, double2 *,
                                            cudaStream_t);
template void launch_gauss_jordan<float>(float2 *, float2 *, int, cudaStream_t);
template void launch_gauss_jordan<double>(double2 *, double2 *, int, cudaStream_t);
template void launch_dense_gemv<float>(const float2 *, int, const float2 *, size_t, float2 *,
                                       size_t, int, const int *, cudaStream_t);
template void launch_dense_gemv<double>(const double2 *, int, const double2 *, size_t, double2 *,
                                        size_t, int, const int *, cudaStream_t);

}  // namespace helm
