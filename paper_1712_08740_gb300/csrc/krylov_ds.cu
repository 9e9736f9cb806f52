// Arnoldi kernels on a double-single basis (precision HELM_PREC_MIXED_DS).
//
// GB300 issues FP64 at about 2 lanes per clock per SM and FP32 at 128: the
// complex128 multi-dot and multi-axpy of the Arnoldi step are bound by the
// FP64 pipe. Here the basis vectors are stored as float4 (re_hi, re_lo,
// im_hi, im_lo), each part an unevaluated sum hi + lo of two floats (about 48
// significant bits), and the products and sums run on the FP32 pipe with
// error-free transformations:
//   product   p = a_hi * b_hi exactly as p + e, e = fma(a_hi, b_hi, -p),
//             plus the cross terms a_hi*b_lo + a_lo*b_hi in FP32;
//   sum       two-sum of the high parts, low parts accumulated in FP32.
// A complex multiply-add costs 44 FP32 instructions instead of 4 FP64 ones,
// about six times less issue time. The Hessenberg coefficients, norms and
// everything outside these kernels stay complex128; partial sums are joined
// into doubles before the block and grid reductions, which are the same
// deterministic two-level reductions as in krylov.cu.
#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxVec = 257;
constexpr int kGroup = 8;

// acc += a * b, all double-single (acc unnormalised: h carries the leading part)
__device__ __forceinline__ void ds_fma(float &h, float &l, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = h + p;
    const float bb = s - h;
    const float err = (h - (s - bb)) + (p - bb);
    h = s;
    l += err + e;
}

// (h, l) = a * b for a fresh accumulator: the same bits as ds_fma into (0, 0)
__device__ __forceinline__ void ds_init(float &h, float &l, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    h = p;
    l = e;
}

// (h, l) += (bh, bl), renormalised
__device__ __forceinline__ void ds_add(float &h, float &l, float bh, float bl) {
    const float s = h + bh;
    const float bb = s - h;
    float e = (h - (s - bb)) + (bh - bb);
    e += l + bl;
    h = s + e;
    l = e - (h - s);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduce-scatter of 16 double-single values across a warp (FP32 adds only):
// afterwards lanes 2i and 2i+1 hold the warp sum of value i.
__device__ __forceinline__ void warp_reduce16_ds(float h[16], float l[16], float &oh, float &ol) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int half = 8, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
        const bool up = (lane & bit) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const float sh = up ? h[k] : h[k + half], sl = up ? l[k] : l[k + half];
            float kh = up ? h[k + half] : h[k], kl = up ? l[k + half] : l[k];
            ds_add(kh, kl, __shfl_xor_sync(0xffffffffu, sh, bit), __shfl_xor_sync(0xffffffffu, sl, bit));
            h[k] = kh;
            l[k] = kl;
        }
    }
    oh = h[0];
    ol = l[0];
    ds_add(oh, ol, __shfl_xor_sync(0xffffffffu, h[0], 1), __shfl_xor_sync(0xffffffffu, l[0], 1));
}

__device__ bool last_block(unsigned *counter) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

__global__ void __launch_bounds__(kThreads)
k_multidot_ds(const float4 *__restrict__ V, size_t sV, int nvec, const float4 *__restrict__ w,
              size_t sw, size_t N, double2 *__restrict__ out, size_t ostride,
              double2 *__restrict__ partial, unsigned *__restrict__ counter, int nvec_max,
              const int *__restrict__ active) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    V += r * sV;
    w += r * sw;
    double2 *part = partial + (size_t)r * nvec_max * gridDim.x + blockIdx.x;
    __shared__ double2 red[kWarps][kMaxVec];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t step = (size_t)gridDim.x * kThreads;
    for (int i0 = 0; i0 < nvec; i0 += kGroup) {
        float h[16], l[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) h[q] = l[q] = 0.f;
        // two of the thread's nodes per round, all their loads issued before
        // use; each accumulator still sums the thread's nodes in index order
        // (a missing second node adds an exact zero). In the thread's first
        // round the first product into each accumulator initialises it
        // (the same bits as adding it to zero, without the two-sum).
        bool first = true;
        for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N; p += 2 * step) {
            const size_t p2 = p + step;
            const bool two = p2 < N;
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 x0 = w[p], x1 = two ? w[p2] : zero;
            float4 va[kGroup], vb[kGroup];
#pragma unroll
            for (int q = 0; q < kGroup; ++q) {
                if (i0 + q < nvec) {
                    va[q] = V[(size_t)(i0 + q) * N + p];
                    vb[q] = two ? V[(size_t)(i0 + q) * N + p2] : zero;
                }
            }
#pragma unroll
            for (int q = 0; q < kGroup; ++q) {
                if (i0 + q < nvec) {
                    // conj(v) x: re = vr xr + vi xi, im = vr xi - vi xr
                    const float4 v = va[q];
                    if (first) {
                        ds_init(h[2 * q], l[2 * q], v.x, v.y, x0.x, x0.y);
                        ds_init(h[2 * q + 1], l[2 * q + 1], v.x, v.y, x0.z, x0.w);
                    } else {
                        ds_fma(h[2 * q], l[2 * q], v.x, v.y, x0.x, x0.y);
                        ds_fma(h[2 * q + 1], l[2 * q + 1], v.x, v.y, x0.z, x0.w);
                    }
                    ds_fma(h[2 * q], l[2 * q], v.z, v.w, x0.z, x0.w);
                    ds_fma(h[2 * q + 1], l[2 * q + 1], -v.z, -v.w, x0.x, x0.y);
                    const float4 u = vb[q];
                    ds_fma(h[2 * q], l[2 * q], u.x, u.y, x1.x, x1.y);
                    ds_fma(h[2 * q], l[2 * q], u.z, u.w, x1.z, x1.w);
                    ds_fma(h[2 * q + 1], l[2 * q + 1], u.x, u.y, x1.z, x1.w);
                    ds_fma(h[2 * q + 1], l[2 * q + 1], -u.z, -u.w, x1.x, x1.y);
                }
            }
            first = false;
        }
        float oh, ol;
        warp_reduce16_ds(h, l, oh, ol);
        const int comp = (lane >> 1) & 15;
        if ((lane & 1) == 0 && i0 + (comp >> 1) < nvec) {
            double *dst = reinterpret_cast<double *>(&red[warp][i0 + (comp >> 1)]);
            dst[comp & 1] = ds_join(oh, ol);
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

// w -= sum_i V_i c_i (c complex128, split once per block), optional ||w||^2
__global__ void __launch_bounds__(kThreads)
k_multiaxpy_ds(const float4 *__restrict__ V, size_t sV, int nvec, const double2 *__restrict__ c,
               size_t cstride, float4 *__restrict__ w, size_t sw, size_t N, double *__restrict__ norm2,
               double *__restrict__ partial_d, unsigned *__restrict__ counter,
               const int *__restrict__ active) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    V += r * sV;
    w += r * sw;
    __shared__ float4 cs[kMaxVec];   // (re_hi, re_lo, im_hi, im_lo) of -c_i
    for (int i = threadIdx.x; i < nvec; i += kThreads) {
        const double2 ci = c[r * cstride + i];
        cs[i] = cvt<float4>(make_double2(-ci.x, -ci.y));
    }
    __syncthreads();
    // ||w||^2 accumulates in double-single as well (the FP64 pipe would spend
    // four instructions per node on it); it is joined into a double once per
    // thread, before the deterministic block and grid reductions.
    float nh = 0.f, nl = 0.f;
    const size_t step = (size_t)gridDim.x * kThreads;
    // two of the thread's nodes per round (p and p + step), all basis loads of
    // a group of eight vectors issued for both before use; each node's update
    // and the norm keep the order of a one-node loop
    for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N; p += 2 * step) {
        const size_t p2 = p + step;
        const bool two = p2 < N;
        const float4 xa = w[p];
        const float4 xb = two ? w[p2] : make_float4(0.f, 0.f, 0.f, 0.f);
        float rh = xa.x, rl = xa.y, ih = xa.z, il = xa.w;
        float sh = xb.x, sl = xb.y, jh = xb.z, jl = xb.w;
        for (int i0 = 0; i0 < nvec; i0 += kGroup) {
            float4 v[kGroup], u[kGroup];
#pragma unroll
            for (int q = 0; q < kGroup; ++q) {
                if (i0 + q < nvec) {
                    v[q] = V[(size_t)(i0 + q) * N + p];
                    if (two) u[q] = V[(size_t)(i0 + q) * N + p2];
                }
            }
#pragma unroll
            for (int q = 0; q < kGroup; ++q) {
                if (i0 + q < nvec) {
                    const float4 m = cs[i0 + q];   // -c_i
                    // w += v * (-c): re = vr mr - vi mi, im = vr mi + vi mr
                    ds_fma(rh, rl, v[q].x, v[q].y, m.x, m.y);
                    ds_fma(rh, rl, -v[q].z, -v[q].w, m.z, m.w);
                    ds_fma(ih, il, v[q].x, v[q].y, m.z, m.w);
                    ds_fma(ih, il, v[q].z, v[q].w, m.x, m.y);
                    if (two) {
                        ds_fma(sh, sl, u[q].x, u[q].y, m.x, m.y);
                        ds_fma(sh, sl, -u[q].z, -u[q].w, m.z, m.w);
                        ds_fma(jh, jl, u[q].x, u[q].y, m.z, m.w);
                        ds_fma(jh, jl, u[q].z, u[q].w, m.x, m.y);
                    }
                }
            }
        }
        // renormalise (h, l) and store, node p then node p2
        auto fin = [&](size_t pp, float &ah, float &al, float &bh, float &bl) {
            float th = ah + al;
            al = al - (th - ah);
            ah = th;
            th = bh + bl;
            bl = bl - (th - bh);
            bh = th;
            w[pp] = make_float4(ah, al, bh, bl);
            if (norm2) {
                ds_fma(nh, nl, ah, al, ah, al);
                ds_fma(nh, nl, bh, bl, bh, bl);
            }
        };
        fin(p, rh, rl, ih, il);
        if (two) fin(p2, sh, sl, jh, jl);
    }
    if (norm2) reduce_norm(ds_join(nh, nl), partial_d, counter, norm2, r);
}

template <typename CIn> __device__ __forceinline__ float4 ds_scaled(CIn x, float sh, float sl, double s);
template <>
__device__ __forceinline__ float4 ds_scaled<double2>(double2 x, float, float, double s) {
    return cvt<float4>(make_double2(x.x * s, x.y * s));
}
template <>
__device__ __forceinline__ float4 ds_scaled<float4>(float4 x, float sh, float sl, double) {
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

template <typename CIn>
__global__ void __launch_bounds__(kThreads)
k_scale_ds(const CIn *x, size_t sx, const double *__restrict__ norm2, float4 *y, size_t sy, size_t N,
           const int *__restrict__ active) {
    // x and y may alias (in-place normalisation of a basis vector)
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    x += r * sx;
    y += r * sy;
    __shared__ double s_sh;
    __shared__ float2 s_ds;
    if (threadIdx.x == 0) {
        s_sh = 1.0 / sqrt(norm2[r]);
        s_ds = ds_split(s_sh);
    }
    __syncthreads();
    const double s = s_sh;
    const float2 sd = s_ds;
    for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N;
         p += (size_t)gridDim.x * kThreads)
        y[p] = ds_scaled<CIn>(x[p], sd.x, sd.y, s);
}

__global__ void __launch_bounds__(kThreads)
k_update_ds(const float4 *__restrict__ Z, size_t sZ, int nvec, const double2 *__restrict__ yv,
            size_t ystride, double2 *__restrict__ x, size_t sx, size_t N,
            const int *__restrict__ active, const int *__restrict__ kcount) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    if (kcount) nvec = min(nvec, kcount[r]);
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

// acc += a * b with a exact in FP32 and b double-single (acc unnormalised)
__device__ __forceinline__ void ds_fma1(float &h, float &l, float a, float bh, float bl) {
    const float p = a * bh;
    float e = fmaf(a, bh, -p);
    e = fmaf(a, bl, e);
    const float s = h + p;
    const float bb = s - h;
    const float err = (h - (s - bb)) + (p - bb);
    h = s;
    l += err + e;
}

// x += sum_i Z_i y_i for complex64 z_i (exact in FP32): the sum is formed in
// double-single on the FP32 pipe and added to the complex128 x once per node
// (two FP64 additions per component instead of 4 FMAs per basis vector).
__global__ void __launch_bounds__(kThreads)
k_update_zds(const float2 *__restrict__ Z, size_t sZ, int nvec, const double2 *__restrict__ yv,
             size_t ystride, double2 *__restrict__ x, size_t sx, size_t N,
             const int *__restrict__ active, const int *__restrict__ kcount) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    if (kcount) nvec = min(nvec, kcount[r]);
    Z += r * sZ;
    x += r * sx;
    __shared__ float4 ys[kMaxVec];   // (re_hi, re_lo, im_hi, im_lo) of y_i
    for (int i = threadIdx.x; i < nvec; i += kThreads) ys[i] = cvt<float4>(yv[r * ystride + i]);
    __syncthreads();
    for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < N;
         p += (size_t)gridDim.x * kThreads) {
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        for (int i0 = 0; i0 < nvec; i0 += kGroup) {
            float2 z[kGroup];
#pragma unroll
            for (int q = 0; q < kGroup; ++q)
                if (i0 + q < nvec) z[q] = Z[(size_t)(i0 + q) * N + p];
#pragma unroll
            for (int q = 0; q < kGroup; ++q) {
                if (i0 + q < nvec) {
                    const float4 y = ys[i0 + q];
                    // re += zr yr - zi yi, im += zr yi + zi yr
                    ds_fma1(rh, rl, z[q].x, y.x, y.y);
                    ds_fma1(rh, rl, -z[q].y, y.z, y.w);
                    ds_fma1(ih, il, z[q].x, y.z, y.w);
                    ds_fma1(ih, il, z[q].y, y.x, y.y);
                }
            }
        }
        double2 acc = x[p];
        acc.x += ds_join(rh, rl);
        acc.y += ds_join(ih, il);
        x[p] = acc;
    }
}

inline int sm_blocks_for(size_t N, int per_thread, int cap) {
    const size_t per_wave = (size_t)152 * kThreads * per_thread;
    int k = 1;
    while (k < 8 && (size_t)k * per_wave < N && 152 * 2 * k <= cap) k *= 2;
    return 152 * k <= cap ? 152 * k : cap;
}

inline int blocks_for(size_t N, int cap) {
    size_t b = (N + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    return (int)(b < (size_t)cap ? b : cap);
}

}  // namespace

void launch_multidot_ds(const float4 *V, size_t sV, int nvec, const float4 *w, size_t sw, size_t N,
                        double2 *out, size_t out_stride, int nrhs, const int *active,
                        KrylovScratch &ks, cudaStream_t st) {
    const int nb = sm_blocks_for(N, 4, ks.max_blocks);
    prof_begin(st);
    k_multidot_ds<<<dim3(nb, nrhs), kThreads, 0, st>>>(V, sV, nvec, w, sw, N, out, out_stride,
                                                       ks.partial, ks.counter, ks.nvec_max, active);
    count_launch();
    if (prof_on())
        prof_end("multidot_ds", st, (nvec + 1.0) * N * 16.0 * nrhs, 0.0);
}

void launch_multiaxpy_ds(const float4 *V, size_t sV, int nvec, const double2 *c, size_t c_stride,
                         float4 *w, size_t sw, size_t N, double *norm2, int nrhs, const int *active,
                         KrylovScratch &ks, cudaStream_t st) {
    const int nb = sm_blocks_for(N, 4, ks.max_blocks);
    prof_begin(st);
    k_multiaxpy_ds<<<dim3(nb, nrhs), kThreads, 0, st>>>(V, sV, nvec, c, c_stride, w, sw, N, norm2,
                                                        (double *)ks.partial, ks.counter, active);
    count_launch();
    if (prof_on())
        prof_end("multiaxpy_ds", st, (nvec + 2.0) * N * 16.0 * nrhs, norm2 ? 4.0 * N * nrhs : 0.0);
}

template <typename CIn>
void launch_scale_ds(const CIn *x, size_t sx, const double *norm2, float4 *y, size_t sy, size_t N,
                     int nrhs, const int *active, cudaStream_t st) {
    const int nb = blocks_for(N, 1 << 16);
    prof_begin(st);
    k_scale_ds<CIn><<<dim3(nb, nrhs), kThreads, 0, st>>>(x, sx, norm2, y, sy, N, active);
    count_launch();
    if (prof_on()) prof_end("scale_ds", st, (16.0 + sizeof(CIn)) * N * nrhs, 0.0);
}

void launch_update_ds(const float4 *Z, size_t sZ, int nvec, const double2 *y, size_t y_stride,
                      double2 *x, size_t sx, size_t N, int nrhs, const int *active, cudaStream_t st,
                      const int *kcount) {
    const int nb = blocks_for(N, 1 << 16);
    prof_begin(st);
    k_update_ds<<<dim3(nb, nrhs), kThreads, 0, st>>>(Z, sZ, nvec, y, y_stride, x, sx, N, active,
                                                     kcount);
    count_launch();
    if (prof_on()) prof_end("update_ds", st, (16.0 * nvec + 32.0) * N * nrhs, 8.0 * nvec * N * nrhs);
}

void launch_update_zds(const float2 *Z, size_t sZ, int nvec, const double2 *y, size_t y_stride,
                       double2 *x, size_t sx, size_t N, int nrhs, const int *active, cudaStream_t st,
                       const int *kcount) {
    const int nb = blocks_for(N, 1 << 16);
    prof_begin(st);
    k_update_zds<<<dim3(nb, nrhs), kThreads, 0, st>>>(Z, sZ, nvec, y, y_stride, x, sx, N, active,
                                                      kcount);
    count_launch();
    if (prof_on()) prof_end("update_zds", st, (8.0 * nvec + 32.0) * N * nrhs, 4.0 * N * nrhs);
}

template void launch_scale_ds<double2>(const double2 *, size_t, const double *, float4 *, size_t,
                                       size_t, int, const int *, cudaStream_t);
template void launch_scale_ds<float4>(const float4 *, size_t, const double *, float4 *, size_t,
                                      size_t, int, const int *, cudaStream_t);

}  // namespace helm
