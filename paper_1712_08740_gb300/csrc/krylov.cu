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

// Reduce-scatter of 16 doubles across a warp: afterwards lanes 2i and 2i+1 both
// hold the warp sum of v[i]. Costs 16 additions instead of 5 per value.
__device__ __forceinline__ double warp_reduce16(double v[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int half = 8, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
        const bool up = (lane & bit) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const double send = up ? v[k] : v[k + half];
            const double keep = up ? v[k + half] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
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

// Multi-dot: out[i] = sum_p conj(V_i[p]) w[p], i < nvec.
// Basis vectors are taken in groups of kGroup: for each group a thread walks
// its points once (w in a register, kGroup complex accumulators), so V is read
// once and w nvec/kGroup times (from L1/L2). Every block then writes one
// partial per vector; the last block adds the partials in block order, one
// warp per vector (lane-strided over blocks, fixed shuffle tree).
constexpr int kGroup = 8;

__global__ void __launch_bounds__(kThreads)
k_multidot(const double2 *__restrict__ V, size_t sV, int nvec, const double2 *__restrict__ w,
           size_t sw, size_t N, double2 *__restrict__ out, size_t ostride,
           double2 *__restrict__ partial, unsigned *__restrict__ counter, int nvec_max,
           const int *__restrict__ active) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    V += r * sV;
    w += r * sw;
    // partials transposed, [rhs][vector][block], so the last block reads them coalesced
    double2 *part = partial + (size_t)r * nvec_max * gridDim.x + blockIdx.x;
    __shared__ double2 red[kWarps][kMaxVec];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t step = (size_t)gridDim.x * kThreads;
    for (int i0 = 0; i0 < nvec; i0 += kGroup) {
        double are[kGroup], aim[kGroup];
#pragma unroll
        for (int q = 0; q < kGroup; ++q) are[q] = aim[q] = 0.0;
        for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N; p += step) {
            const double2 x = w[p];
#pragma unroll
            for (int q = 0; q < kGroup; ++q) {
                if (i0 + q < nvec) {
                    const double2 v = V[(size_t)(i0 + q) * N + p];
                    are[q] = fma(v.x, x.x, are[q]);
                    are[q] = fma(v.y, x.y, are[q]);
                    aim[q] = fma(v.x, x.y, aim[q]);
                    aim[q] = fma(-v.y, x.x, aim[q]);
                }
            }
        }
        double v[16];
#pragma unroll
        for (int q = 0; q < kGroup; ++q) {
            v[2 * q] = are[q];
            v[2 * q + 1] = aim[q];
        }
        const double tot = warp_reduce16(v);
        // lane 2i holds component i = 2q + (0 re | 1 im)
        const int comp = (lane >> 1) & 15;
        if ((lane & 1) == 0 && i0 + (comp >> 1) < nvec) {
            double *dst = reinterpret_cast<double *>(&red[warp][i0 + (comp >> 1)]);
            dst[comp & 1] = tot;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nvec; i += kThreads) {
        double2 s = red[0][i];
        for (int q = 1; q < kWarps; ++q) {
            s.x += red[q][i].x;
            s.y += red[q][i].y;
        }
        part[(size_t)i * gridDim.x] = s;
    }
    if (last_block(counter + r)) {
        const double2 *pr = partial + (size_t)r * nvec_max * gridDim.x;
        for (int i = warp; i < nvec; i += kWarps) {
            double sx, sy;
            lane_sum(pr + (size_t)i * gridDim.x, gridDim.x, lane, sx, sy);
            sx = warp_sum(sx);
            sy = warp_sum(sy);
            if (lane == 0) out[r * ostride + i] = make_double2(sx, sy);
        }
        if (threadIdx.x == 0) counter[r] = 0;
    }
}

// (H z)_p of Eq. 2-3 at one node (the same formulas as k_stencil's APPLY
// mode): d_p z_p - (1/h^2) sum_nbr c z_nbr, c = 2 at a mirrored boundary
// neighbour, d_p with the absorbing boundary term at boundary nodes.
template <int DIM, typename CZ>
__device__ __forceinline__ double2 h_at(const LevelView<double> &L, const OpShift<double> &s,
                                        const CZ *__restrict__ z, size_t p) {
    const unsigned nx = (unsigned)L.nx, ny = (unsigned)L.ny, nz = (unsigned)L.nz;
    const unsigned up = (unsigned)p;
    const unsigned ix = up % nx, row = up / nx;
    const unsigned iy = DIM == 3 ? row % ny : row, iz = DIM == 3 ? row / ny : 0;
    double sre = 0.0, sim = 0.0;
    int nf = 0;
    auto axis = [&](unsigned i, unsigned n, size_t stride) {
        if (i > 0) {
            const double2 v = cvt<double2>(z[p - stride]);
            const double c = (i == n - 1) ? 2.0 : 1.0;
            sre += c * v.x;
            sim += c * v.y;
        } else {
            ++nf;
        }
        if (i < n - 1) {
            const double2 v = cvt<double2>(z[p + stride]);
            const double c = (i == 0) ? 2.0 : 1.0;
            sre += c * v.x;
            sim += c * v.y;
        } else {
            ++nf;
        }
    };
    axis(ix, nx, 1);
    if (DIM >= 2) axis(iy, ny, (size_t)nx);
    if (DIM == 3) axis(iz, nz, (size_t)nx * ny);
    const double wp = L.w[p];
    double dre = 2.0 * DIM * L.inv_h2 - s.s_re * wp;
    double dim_ = -s.s_im * wp;
    if (nf) {
        const double f = nf * L.two_over_h * sqrt(wp);
        dre -= f * s.q_im;
        dim_ += f * s.q_re;
    }
    const double2 zp = cvt<double2>(z[p]);
    return make_double2(dre * zp.x - dim_ * zp.y - L.inv_h2 * sre,
                        dre * zp.y + dim_ * zp.x - L.inv_h2 * sim);
}

// w = H z_j (written into basis slot j+1) fused with the multi-dot
// out[i] = sum_p conj(V_i[p]) w[p], i < nvec: the first group of basis vectors
// forms w at each node from z and stores it, later groups read it back (the
// thread's own writes). Saves the separate H z launch and one pass over w.
template <int DIM, typename CZ>
__global__ void __launch_bounds__(kThreads)
k_multidot_h(const double2 *__restrict__ V, size_t sV, int nvec, double2 *__restrict__ w,
             size_t sw, size_t N, double2 *__restrict__ out, size_t ostride,
             double2 *__restrict__ partial, unsigned *__restrict__ counter, int nvec_max,
             const int *__restrict__ active, LevelView<double> L, OpShift<double> sH,
             const CZ *__restrict__ z, size_t sz) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    V += r * sV;
    w += r * sw;
    z += r * sz;
    double2 *part = partial + (size_t)r * nvec_max * gridDim.x + blockIdx.x;
    __shared__ double2 red[kWarps][kMaxVec];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t step = (size_t)gridDim.x * kThreads;
    for (int i0 = 0; i0 < nvec; i0 += kGroup) {
        double are[kGroup], aim[kGroup];
#pragma unroll
        for (int q = 0; q < kGroup; ++q) are[q] = aim[q] = 0.0;
        for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N; p += step) {
            double2 x;
            if (i0 == 0) {
                x = h_at<DIM>(L, sH, z, p);
                w[p] = x;
            } else {
                x = w[p];
            }
#pragma unroll
            for (int q = 0; q < kGroup; ++q) {
                if (i0 + q < nvec) {
                    const double2 v = V[(size_t)(i0 + q) * N + p];
                    are[q] = fma(v.x, x.x, are[q]);
                    are[q] = fma(v.y, x.y, are[q]);
                    aim[q] = fma(v.x, x.y, aim[q]);
                    aim[q] = fma(-v.y, x.x, aim[q]);
                }
            }
        }
        double v[16];
#pragma unroll
        for (int q = 0; q < kGroup; ++q) {
            v[2 * q] = are[q];
            v[2 * q + 1] = aim[q];
        }
        const double tot = warp_reduce16(v);
        const int comp = (lane >> 1) & 15;
        if ((lane & 1) == 0 && i0 + (comp >> 1) < nvec) {
            double *dst = reinterpret_cast<double *>(&red[warp][i0 + (comp >> 1)]);
            dst[comp & 1] = tot;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nvec; i += kThreads) {
        double2 s = red[0][i];
        for (int q = 1; q < kWarps; ++q) {
            s.x += red[q][i].x;
            s.y += red[q][i].y;
        }
        part[(size_t)i * gridDim.x] = s;
    }
    if (last_block(counter + r)) {
        const double2 *pr = partial + (size_t)r * nvec_max * gridDim.x;
        for (int i = warp; i < nvec; i += kWarps) {
            double sx, sy;
            lane_sum(pr + (size_t)i * gridDim.x, gridDim.x, lane, sx, sy);
            sx = warp_sum(sx);
            sy = warp_sum(sy);
            if (lane == 0) out[r * ostride + i] = make_double2(sx, sy);
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
        if (warp == 0) {
            double s = lane_sum(partial_d + (size_t)r * gridDim.x, gridDim.x, lane);
            s = warp_sum(s);
            if (lane == 0) {
                norm2[r] = s;
                counter[r] = 0;
            }
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
        int i = 0;
        for (; i + 4 <= nvec; i += 4) {
            double2 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = V[(size_t)(i + q) * N + p];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double2 h = cs[i + q];
                acc.x = fma(-v[q].x, h.x, acc.x);
                acc.x = fma(v[q].y, h.y, acc.x);
                acc.y = fma(-v[q].x, h.y, acc.y);
                acc.y = fma(-v[q].y, h.x, acc.y);
            }
        }
        for (; i < nvec; ++i) {
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
    __shared__ double s_sh;
    if (threadIdx.x == 0) s_sh = 1.0 / sqrt(norm2[r]);
    __syncthreads();
    const double s = s_sh;
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
         const int *__restrict__ active, const int *__restrict__ kcount) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    // only the columns this right-hand side filled in the cycle: the others may
    // hold stale or uninitialised values (NaN * 0 would poison x)
    if (kcount) nvec = min(nvec, kcount[r]);
    Z += r * sZ;
    x += r * sx;
    __shared__ double2 ys[kMaxVec];
    for (int i = threadIdx.x; i < nvec; i += kThreads) ys[i] = yv[r * ystride + i];
    __syncthreads();
    for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N;
         p += (size_t)gridDim.x * kThreads) {
        double2 acc = x[p];
#pragma unroll 4
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

// Selective reorthogonalisation test (Daniel-Gragg-Kaufman-Stewart): a second
// Gram-Schmidt pass is needed when the first pass cancelled most of w,
// ||w'||^2 < eta2 ||w||^2. ||w||^2 is the last entry of the first multi-dot
// (w itself taken as an extra vector). Right-hand sides that skip the second
// pass get zero second-pass coefficients.
__global__ void k_reorth_flags(const int *__restrict__ act, const double2 *__restrict__ h1,
                               double2 *__restrict__ h2, int hstride, int wslot,
                               const double *__restrict__ n1, double eta2, int *__restrict__ act2,
                               int nvec, int nrhs) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrhs; r += gridDim.x * blockDim.x) {
        const int a = act ? act[r] : 1;
        const int need = a && (n1[r] < eta2 * h1[(size_t)r * hstride + wslot].x);
        act2[r] = need;
        if (a && !need)
            for (int i = 0; i < nvec; ++i) h2[(size_t)r * hstride + i] = make_double2(0.0, 0.0);
    }
}

__global__ void k_finite(const double *__restrict__ x, size_t n, int *__restrict__ flag) {
    int bad = 0;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (size_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[p]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// x_r = 0 for every right-hand side r with active[r] == 0
__global__ void k_zero_inactive(double2 *__restrict__ x, size_t N, const int *__restrict__ active,
                                int nrhs) {
    const int r = blockIdx.y;
    if (active[r]) return;
    double2 *xr = x + (size_t)r * N;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (size_t)gridDim.x * blockDim.x)
        xr[p] = make_double2(0.0, 0.0);
}

// Reduction grids are whole multiples of the SM count (152 on GB300): one,
// two, four or eight blocks per SM, so that no SM runs an extra block while
// the others idle, with roughly `per_thread` points per thread.
inline int sm_blocks_for(size_t N, int per_thread, int cap) {
    const int sms = device_sms();
    const size_t per_wave = (size_t)sms * kThreads * per_thread;
    int k = 1;
    while (k < 8 && (size_t)k * per_wave < N && sms * 2 * k <= cap) k *= 2;
    return sms * k <= cap ? sms * k : cap;
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
    const int nb = sm_blocks_for(N, 4, ks.max_blocks);
    prof_begin(st);
    k_multidot<<<dim3(nb, nrhs), kThreads, 0, st>>>(V, sV, nvec, w, sw, N, out, out_stride,
                                                    ks.partial, ks.counter, ks.nvec_max, active);
    count_launch();
    if (prof_on())
        prof_end("multidot_f64", st, (nvec + 1.0) * N * 16.0 * nrhs, 8.0 * nvec * N * nrhs);
}

template <typename CZ>
void launch_multidot_h(const double2 *V, size_t sV, int nvec, double2 *w, size_t sw, size_t N,
                       double2 *out, size_t out_stride, int nrhs, const int *active,
                       KrylovScratch &ks, const LevelView<double> &L, OpShift<double> sH,
                       const CZ *z, size_t sz, cudaStream_t st) {
    const int nb = sm_blocks_for(N, 4, ks.max_blocks);
    prof_begin(st);
    const dim3 g(nb, nrhs);
    if (L.dim == 1)
        k_multidot_h<1, CZ><<<g, kThreads, 0, st>>>(V, sV, nvec, w, sw, N, out, out_stride, ks.partial,
                                                    ks.counter, ks.nvec_max, active, L, sH, z, sz);
    else if (L.dim == 2)
        k_multidot_h<2, CZ><<<g, kThreads, 0, st>>>(V, sV, nvec, w, sw, N, out, out_stride, ks.partial,
                                                    ks.counter, ks.nvec_max, active, L, sH, z, sz);
    else
        k_multidot_h<3, CZ><<<g, kThreads, 0, st>>>(V, sV, nvec, w, sw, N, out, out_stride, ks.partial,
                                                    ks.counter, ks.nvec_max, active, L, sH, z, sz);
    count_launch();
    if (prof_on())
        prof_end("multidot_h_f64", st, ((nvec + 1.0) * 16.0 + sizeof(CZ) + 8.0) * N * nrhs,
                 (8.0 * nvec + 4.0 * L.dim + 12.0) * N * nrhs);
}
template void launch_multidot_h<double2>(const double2 *, size_t, int, double2 *, size_t, size_t,
                                         double2 *, size_t, int, const int *, KrylovScratch &,
                                         const LevelView<double> &, OpShift<double>,
                                         const double2 *, size_t, cudaStream_t);
template void launch_multidot_h<float2>(const double2 *, size_t, int, double2 *, size_t, size_t,
                                        double2 *, size_t, int, const int *, KrylovScratch &,
                                        const LevelView<double> &, OpShift<double>,
                                        const float2 *, size_t, cudaStream_t);

void launch_multiaxpy(const double2 *V, size_t sV, int nvec, const double2 *c, size_t c_stride,
                      double2 *w, size_t sw, size_t N, double *norm2, int nrhs,
                      const int *active, KrylovScratch &ks, cudaStream_t st) {
    const int nb = sm_blocks_for(N, 4, ks.max_blocks);
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
    const int nb = sm_blocks_for(N, 4, ks.max_blocks);
    prof_begin(st);
    k_norm2<<<dim3(nb, nrhs), kThreads, 0, st>>>(x, sx, N, norm2, (double *)ks.partial,
                                                 ks.counter, active);
    count_launch();
    if (prof_on()) prof_end("norm2_f64", st, 16.0 * N * nrhs, 4.0 * N * nrhs);
}

template <typename COut>
void launch_scale(const double2 *x, size_t sx, const double *norm2, COut *y, size_t sy, size_t N,
                  int nrhs, const int *active, cudaStream_t st) {
    const int nb = blocks_for(N, kThreads, 1 << 16);
    prof_begin(st);
    k_scale<COut><<<dim3(nb, nrhs), kThreads, 0, st>>>(x, sx, norm2, y, sy, N, active);
    count_launch();
    if (prof_on()) prof_end("scale_f64", st, (16.0 + sizeof(COut)) * N * nrhs, 2.0 * N * nrhs);
}

template <typename CZ>
void launch_update(const CZ *Z, size_t sZ, int nvec, const double2 *y, size_t y_stride,
                   double2 *x, size_t sx, size_t N, int nrhs, const int *active, cudaStream_t st,
                   const int *kcount) {
    const int nb = blocks_for(N, kThreads, 1 << 16);
    prof_begin(st);
    k_update<CZ><<<dim3(nb, nrhs), kThreads, 0, st>>>(Z, sZ, nvec, y, y_stride, x, sx, N, active,
                                                      kcount);
    count_launch();
    if (prof_on())
        prof_end("update_f64", st, ((double)nvec * sizeof(CZ) + 32.0) * N * nrhs,
                 8.0 * nvec * N * nrhs);
}

template <typename CIn, typename COut>
void launch_convert(const CIn *x, size_t sx, COut *y, size_t sy, size_t N, int nrhs,
                    cudaStream_t st) {
    const int nb = blocks_for(N, kThreads, 1 << 16);
    prof_begin(st);
    k_convert<CIn, COut><<<dim3(nb, nrhs), kThreads, 0, st>>>(x, sx, y, sy, N);
    count_launch();
    if (prof_on()) prof_end("convert", st, (double)(sizeof(CIn) + sizeof(COut)) * N * nrhs, 0.0);
}

void launch_reorth_flags(const int *act, const double2 *h1, double2 *h2, int hstride, int wslot,
                         const double *n1, double eta2, int *act2, int nvec, int nrhs,
                         cudaStream_t st) {
    k_reorth_flags<<<(nrhs + 127) / 128, 128, 0, st>>>(act, h1, h2, hstride, wslot, n1, eta2, act2,
                                                       nvec, nrhs);
    count_launch();
}

void launch_finite_check(const double *x, size_t n, int *flag, cudaStream_t st) {
    const int nb = blocks_for(n, kThreads * kItems, 1024);
    k_finite<<<nb, kThreads, 0, st>>>(x, n, flag);
    count_launch();
}

void launch_zero_inactive(double2 *x, size_t N, const int *active, int nrhs, cudaStream_t st) {
    const int nb = blocks_for(N, kThreads * kItems, 1024);
    k_zero_inactive<<<dim3(nb, nrhs), kThreads, 0, st>>>(x, N, active, nrhs);
    count_launch();
}

template void launch_scale<double2>(const double2 *, size_t, const double *, double2 *, size_t,
                                    size_t, int, const int *, cudaStream_t);
template void launch_scale<float2>(const double2 *, size_t, const double *, float2 *, size_t,
                                   size_t, int, const int *, cudaStream_t);
template void launch_update<double2>(const double2 *, size_t, int, const double2 *, size_t,
                                     double2 *, size_t, size_t, int, const int *, cudaStream_t,
                                     const int *);
template void launch_update<float2>(const float2 *, size_t, int, const double2 *, size_t,
                                    double2 *, size_t, size_t, int, const int *, cudaStream_t,
                                    const int *);
template void launch_convert<double2, float2>(const double2 *, size_t, float2 *, size_t, size_t,
                                              int, cudaStream_t);
template void launch_convert<float2, double2>(const float2 *, size_t, double2 *, size_t, size_t,
                                              int, cudaStream_t);
template void launch_convert<double2, double2>(const double2 *, size_t, double2 *, size_t,
                                               size_t, int, cudaStream_t);
template void launch_convert<float4, double2>(const float4 *, size_t, double2 *, size_t, size_t, int,
                                               cudaStream_t);
template void launch_convert<float4, float2>(const float4 *, size_t, float2 *, size_t, size_t, int,
                                             cudaStream_t);

}  // namespace helm
