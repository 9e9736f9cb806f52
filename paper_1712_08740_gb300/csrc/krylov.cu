// Complex128 kernels of the flexible GMRES outer loop (Eq. 7): the Arnoldi
// inner products (classical Gram-Schmidt as one fused multi-dot), the basis
// update, norms, scaling and the solution update x += Z y.
//
// Reductions are two-level and deterministic: warp shuffles, then a block
// sum in shared memory into a per-block partial; the last block to finish
// (found with a threadfence + atomic ticket) adds the partials in block order.
// The result does not depend on scheduling, so reruns are bit-identical.
//
// Every kernel takes a right-hand-side index from blockIdx.y and skips
// right-hand sides whose `active` flag is zero (converged members of a batch).
#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 4;                 // points per thread per chunk
constexpr int kMaxVec = 257;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Last-block reduction of partial[b * nv + i] over b < nblk into out[i * ostride] / norm.
// Returns true in the block that did it.
__device__ bool last_block(unsigned *counter) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

__global__ void __launch_bounds__(kThreads)
k_multidot(const double2 *__restrict__ V, size_t sV, int nvec, const double2 *__restrict__ w,
           size_t sw, size_t N, double2 *__restrict__ out, size_t ostride,
           double2 *__restrict__ partial, unsigned *__restrict__ counter, int nvec_max,
           const int *__restrict__ active) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    V += r * sV;
    w += r * sw;
    double2 *part = partial + ((size_t)r * gridDim.x + blockIdx.x) * nvec_max;
    __shared__ double2 red[kWarps][kMaxVec];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t chunk = (size_t)kThreads * kItems;
    const size_t step = chunk * gridDim.x;
    for (int i = 0; i < nvec; ++i) {
        const double2 *Vi = V + (size_t)i * N;
        double are = 0.0, aim = 0.0;
        for (size_t base = blockIdx.x * chunk; base < N; base += step) {
#pragma unroll
            for (int t = 0; t < kItems; ++t) {
                const size_t p = base + (size_t)t * kThreads + threadIdx.x;
                if (p < N) {
                    const double2 v = Vi[p];
                    const double2 x = w[p];
                    are = fma(v.x, x.x, are);
                    are = fma(v.y, x.y, are);
                    aim = fma(v.x, x.y, aim);
                    aim = fma(-v.y, x.x, aim);
                }
            }
        }
        are = warp_sum(are);
        aim = warp_sum(aim);
        if (lane == 0) red[warp][i] = make_double2(are, aim);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nvec; i += kThreads) {
        double2 s = red[0][i];
        for (int q = 1; q < kWarps; ++q) {
            s.x += red[q][i].x;
            s.y += red[q][i].y;
        }
        part[i] = s;
    }
    if (last_block(counter + r)) {
        const double2 *pr = partial + (size_t)r * gridDim.x * nvec_max;
        for (int i = threadIdx.x; i < nvec; i += kThreads) {
            double2 s = make_double2(0.0, 0.0);
            for (unsigned b = 0; b < gridDim.x; ++b) {
                s.x += pr[(size_t)b * nvec_max + i].x;
                s.y += pr[(size_t)b * nvec_max + i].y;
            }
            out[r * ostride + i] = s;
        }
        if (threadIdx.x == 0) counter[r] = 0;
    }
}

// Block-sum of one double into a partial, then the last block finishes norm2[r].
__device__ void reduce_norm(double v, double *partial_d, unsigned *counter, double *norm2, int r) {
    __shared__ double red[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = warp_sum(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kWarps; ++q) s += red[q];
        partial_d[(size_t)r * gridDim.x + blockIdx.x] = s;
    }
    if (last_block(counter + r)) {
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) s += partial_d[(size_t)r * gridDim.x + b];
            norm2[r] = s;
            counter[r] = 0;
        }
    }
}

__global__ void __launch_bounds__(kThreads)
k_multiaxpy(const double2 *__restrict__ V, size_t sV, int nvec, const double2 *__restrict__ c,
            size_t cstride, double2 *__restrict__ w, size_t sw, size_t N,
            double *__restrict__ norm2, double *__restrict__ partial_d,
            unsigned *__restrict__ counter, const int *__restrict__ active) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    V += r * sV;
    w += r * sw;
    __shared__ double2 cs[kMaxVec];
    for (int i = threadIdx.x; i < nvec; i += kThreads) cs[i] = c[r * cstride + i];
    __syncthreads();
    double n2 = 0.0;
    for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N;
         p += (size_t)gridDim.x * kThreads) {
        double2 acc = w[p];
        for (int i = 0; i < nvec; ++i) {
            const double2 v = V[(size_t)i * N + p];
            const double2 h = cs[i];
            acc.x = fma(-v.x, h.x, acc.x);
            acc.x = fma(v.y, h.y, acc.x);
            acc.y = fma(-v.x, h.y, acc.y);
            acc.y = fma(-v.y, h.x, acc.y);
        }
        w[p] = acc;
        n2 = fma(acc.x, acc.x, n2);
        n2 = fma(acc.y, acc.y, n2);
    }
    if (norm2) reduce_norm(n2, partial_d, counter, norm2, r);
}

__global__ void __launch_bounds__(kThreads)
k_norm2(const double2 *__restrict__ x, size_t sx, size_t N, double *__restrict__ norm2,
        double *__restrict__ partial_d, unsigned *__restrict__ counter,
        const int *__restrict__ active) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    x += r * sx;
    double n2 = 0.0;
    for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N;
         p += (size_t)gridDim.x * kThreads) {
        const double2 v = x[p];
        n2 = fma(v.x, v.x, n2);
        n2 = fma(v.y, v.y, n2);
    }
    reduce_norm(n2, partial_d, counter, norm2, r);
}

template <typename COut>
__global__ void __launch_bounds__(kThreads)
k_scale(const double2 *x, size_t sx, const double *__restrict__ norm2, COut *y, size_t sy,
        size_t N, const int *__restrict__ active) {
    // x and y may alias (in-place normalisation of a basis vector)
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    x += r * sx;
    y += r * sy;
    const double s = 1.0 / sqrt(norm2[r]);
    for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N;
         p += (size_t)gridDim.x * kThreads) {
        const double2 v = x[p];
        y[p] = cvt<COut>(make_double2(v.x * s, v.y * s));
    }
}

template <typename CZ>
__global__ void __launch_bounds__(kThreads)
k_update(const CZ *__restrict__ Z, size_t sZ, int nvec, const double2 *__restrict__ yv,
         size_t ystride, double2 *__restrict__ x, size_t sx, size_t N,
         const int *__restrict__ active) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    Z += r * sZ;
    x += r * sx;
    __shared__ double2 ys[kMaxVec];
    for (int i = threadIdx.x; i < nvec; i += kThreads) ys[i] = yv[r * ystride + i];
    __syncthreads();
    for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N;
         p += (size_t)gridDim.x * kThreads) {
        double2 acc = x[p];
        for (int i = 0; i < nvec; ++i) {
            const double2 z = cvt<double2>(Z[(size_t)i * N + p]);
            const double2 h = ys[i];
            acc.x = fma(z.x, h.x, acc.x);
            acc.x = fma(-z.y, h.y, acc.x);
            acc.y = fma(z.x, h.y, acc.y);
            acc.y = fma(z.y, h.x, acc.y);
        }
        x[p] = acc;
    }
}

template <typename CIn, typename COut>
__global__ void __launch_bounds__(kThreads)
k_convert(const CIn *__restrict__ x, size_t sx, COut *__restrict__ y, size_t sy, size_t N) {
    const int r = blockIdx.y;
    x += r * sx;
    y += r * sy;
    for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N;
         p += (size_t)gridDim.x * kThreads)
        y[p] = cvt<COut>(x[p]);
}

__global__ void k_finite(const double *__restrict__ x, size_t n, int *__restrict__ flag) {
    int bad = 0;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (size_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[p]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

inline int blocks_for(size_t N, int per_block, int cap) {
    size_t b = (N + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)(b < (size_t)cap ? b : cap);
}

}  // namespace

void launch_multidot(const double2 *V, size_t sV, int nvec, const double2 *w, size_t sw,
                     size_t N, double2 *out, size_t out_stride, int nrhs, const int *active,
                     KrylovScratch &ks, cudaStream_t st) {
    const int nb = blocks_for(N, kThreads * kItems, ks.max_blocks);
    prof_begin(st);
    k_multidot<<<dim3(nb, nrhs), kThreads, 0, st>>>(V, sV, nvec, w, sw, N, out, out_stride,
                                                    ks.partial, ks.counter, ks.nvec_max, active);
    count_launch();
    if (prof_on())
        prof_end("multidot_f64", st, (nvec + 1.0) * N * 16.0 * nrhs, 8.0 * nvec * N * nrhs);
}

void launch_multiaxpy(const double2 *V, size_t sV, int nvec, const double2 *c, size_t c_stride,
                      double2 *w, size_t sw, size_t N, double *norm2, int nrhs,
                      const int *active, KrylovScratch &ks, cudaStream_t st) {
    const int nb = blocks_for(N, kThreads * kItems, ks.max_blocks);
    prof_begin(st);
    k_multiaxpy<<<dim3(nb, nrhs), kThreads, 0, st>>>(V, sV, nvec, c, c_stride, w, sw, N, norm2,
                                                     (double *)ks.partial, ks.counter, active);
    count_launch();
    if (prof_on())
        prof_end("multiaxpy_f64", st, (nvec + 2.0) * N * 16.0 * nrhs,
                 (8.0 * nvec + (norm2 ? 4.0 : 0.0)) * N * nrhs);
}

void launch_norm2(const double2 *x, size_t sx, size_t N, double *norm2, int nrhs,
                  const int *active, KrylovScratch &ks, cudaStream_t st) {
    const int nb = blocks_for(N, kThreads * kItems, ks.max_blocks);
    prof_begin(st);
    k_norm2<<<dim3(nb, nrhs), kThreads, 0, st>>>(x, sx, N, norm2, (double *)ks.partial,
                                                 ks.counter, active);
    count_launch();
    if (prof_on()) prof_end("norm2_f64", st, 16.0 * N * nrhs, 4.0 * N * nrhs);
}

template <typename COut>
void launch_scale(const double2 *x, size_t sx, const double *norm2, COut *y, size_t sy, size_t N,
                  int nrhs, const int *active, cudaStream_t st) {
    const int nb = blocks_for(N, kThreads * kItems, 1 << 16);
    prof_begin(st);
    k_scale<COut><<<dim3(nb, nrhs), kThreads, 0, st>>>(x, sx, norm2, y, sy, N, active);
    count_launch();
    if (prof_on()) prof_end("scale_f64", st, (16.0 + sizeof(COut)) * N * nrhs, 2.0 * N * nrhs);
}

template <typename CZ>
void launch_update(const CZ *Z, size_t sZ, int nvec, const double2 *y, size_t y_stride,
                   double2 *x, size_t sx, size_t N, int nrhs, const int *active, cudaStream_t st) {
    const int nb = blocks_for(N, kThreads * kItems, 1 << 16);
    prof_begin(st);
    k_update<CZ><<<dim3(nb, nrhs), kThreads, 0, st>>>(Z, sZ, nvec, y, y_stride, x, sx, N, active);
    count_launch();
    if (prof_on())
        prof_end("update_f64", st, ((double)nvec * sizeof(CZ) + 32.0) * N * nrhs,
                 8.0 * nvec * N * nrhs);
}

template <typename CIn, typename COut>
void launch_convert(const CIn *x, size_t sx, COut *y, size_t sy, size_t N, int nrhs,
                    cudaStream_t st) {
    const int nb = blocks_for(N, kThreads * kItems, 1 << 16);
    prof_begin(st);
    k_convert<CIn, COut><<<dim3(nb, nrhs), kThreads, 0, st>>>(x, sx, y, sy, N);
    count_launch();
    if (prof_on()) prof_end("convert", st, (double)(sizeof(CIn) + sizeof(COut)) * N * nrhs, 0.0);
}

void launch_finite_check(const double *x, size_t n, int *flag, cudaStream_t st) {
    const int nb = blocks_for(n, kThreads * kItems, 1024);
    k_finite<<<nb, kThreads, 0, st>>>(x, n, flag);
    count_launch();
}

template void launch_scale<double2>(const double2 *, size_t, const double *, double2 *, size_t,
                                    size_t, int, const int *, cudaStream_t);
template void launch_scale<float2>(const double2 *, size_t, const double *, float2 *, size_t,
                                   size_t, int, const int *, cudaStream_t);
template void launch_update<double2>(const double2 *, size_t, int, const double2 *, size_t,
                                     double2 *, size_t, size_t, int, const int *, cudaStream_t);
template void launch_update<float2>(const float2 *, size_t, int, const double2 *, size_t,
                                    double2 *, size_t, size_t, int, const int *, cudaStream_t);
template void launch_convert<double2, float2>(const double2 *, size_t, float2 *, size_t, size_t,
                                              int, cudaStream_t);
template void launch_convert<float2, double2>(const float2 *, size_t, double2 *, size_t, size_t,
                                              int, cudaStream_t);
template void launch_convert<double2, double2>(const double2 *, size_t, double2 *, size_t,
                                               size_t, int, cudaStream_t);

}  // namespace helm
