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
#include "pipe.cuh"

namespace helm {

namespace {

constexpr int kThreads = 256;
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

// acc += a * b with a exact in FP32 and b double-single (acc unnormalised):
// the product a * b_hi is exact as p + e
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


// ---------------------------------------------------------------- streamed Arnoldi kernels
// The multi-dot and multi-axpy read every basis vector V_0..V_{n-1} of every
// right-hand side once per call: about 1.3 GB for a 64-source batch of the
// 401 x 201 grid at n = 16. Both run as persistent blocks of 8 consumer warps
// and one producer warp. One lane of the producer streams tiles of the
// vectors through a ring of shared-memory stages with cp.async.bulk, each
// stage completing on its "full" mbarrier; the consumer warps release a stage
// with one arrive each on its "empty" mbarrier. The consumer warps never
// synchronise with one another: every warp writes its own partial results,
// and a small finalize kernel adds them in a fixed order. All sums thus have
// an order fixed by N alone (the same for a batch as for one right-hand side).
constexpr int kCons = 256;                  // consumer threads (8 warps)
constexpr int kConsWarps = kCons / 32;
constexpr int kPipeThreads = kCons + 32;    // + the producer warp

// multi-dot: a stage is one tile of kDotTile nodes of w and of up to kGroup
// vectors (9 x 4 KB); the accumulators of a group run over a chunk of
// dot_tpi consecutive tiles (one node per thread and tile) before the warp
// reduction, which costs about as much as the chunk's products.
constexpr int kDotTile = 256;
constexpr int kDotStages = 3;
constexpr int kDotBlocksPerSM = 2;

// Tiles per chunk, a function of the tile count alone, so that a batch sums
// in the same order as one right-hand side. Measured on 64-source 2D batches
// and a 4-source 3D batch: 8 tiles beat 4 by 1-11 % (the warp reduction runs
// half as often); 16 beat 8 only on the 3D grid (12.7 M nodes, 4 %) and lost
// on 801 x 401, so 16 is kept for grids of 2 M nodes and more.
__host__ __device__ __forceinline__ int dot_tpi(int ntiles) { return ntiles >= 8192 ? 16 : 8; }

struct DotSmem {
    float4 slot[kDotStages][kGroup + 1][kDotTile];
    uint64_t full[kDotStages], empty[kDotStages];
    int abort;
};

// multi-axpy: a stage is one tile of kAxpyTile nodes (16 KB) of w or of one
// vector; 4 nodes per consumer thread.
constexpr int kAxpyTile = 1024;
constexpr int kAxpyStages = 6;
constexpr int kAxpyBlocksPerSM = 2;

struct alignas(16) AxpySmem {
    float4 slot[kAxpyStages][kAxpyTile];
    uint64_t full[kAxpyStages], empty[kAxpyStages];
    int abort;
    // followed by float4 cs[kConsWarps][nvec]: each warp's copy of -c split
};

__host__ __device__ constexpr int ceil_div(size_t a, size_t b) { return (int)((a + b - 1) / b); }

template <int S> __device__ __forceinline__ void ring_init(uint64_t (&full)[S], uint64_t (&empty)[S], int &abort) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            pipe::mbar_init(&full[s], 1);
            pipe::mbar_init(&empty[s], kConsWarps);
        }
        abort = 0;
        pipe::mbar_init_fence();
    }
    __syncthreads();
}

// Producer teardown: wait (bounded) for the copies of the last stages issued
// (the stages issued always form a prefix 0 .. issued - 1; a slot is reused
// only after its previous copy was consumed, so earlier stages have landed).
// Each stage gets its own bounded wait, so one late copy does not cut the
// wait for the others short.
template <int S> __device__ __forceinline__ void ring_drain(uint64_t (&full)[S], unsigned issued) {
    const unsigned k0 = issued > (unsigned)S ? issued - S : 0u;
    for (unsigned k = k0; k < issued; ++k) pipe::mbar_wait_drain(&full[k % S], (k / S) & 1u);
}

// Time limit of the consumers' waits for a copy to land. The default is the
// pipeline's own bound; helm_set_wait_limit_ns lowers it to make those waits
// run out on purpose (tests of the timeout path). Producer and teardown waits
// keep the default, so no block exits with a copy in flight.
__device__ unsigned long long g_cons_wait_ns = pipe::kWaitNs;

__device__ __forceinline__ bool aborted(const int &abort) { return *(volatile const int *)&abort != 0; }

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7ff8000000000000ll); }

// partial[((r * nvec_max + i) * nch + c) * 8 + warp] = warp's part of
// sum_p conj(V_i[p]) w[p] over chunk c of right-hand side r
__global__ void __launch_bounds__(kPipeThreads, kDotBlocksPerSM)
k_multidot_ds(const float4 *__restrict__ V, size_t sV, int nvec, const float4 *__restrict__ w,
              size_t sw, size_t N, double2 *__restrict__ partial, int nvec_max, int nrhs,
              const int *__restrict__ active) {
    extern __shared__ __align__(128) unsigned char pipe_raw[];
    DotSmem &S = *reinterpret_cast<DotSmem *>(pipe_raw);
    ring_init(S.full, S.empty, S.abort);
    const int ntiles = ceil_div(N, kDotTile), nch = ceil_div(ntiles, dot_tpi(ntiles));
    const int items = nrhs * nch;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned k = 0;
    if (warp == kConsWarps) {
        // producer: per item (r, c), per group, per tile: one stage
        if (lane == 0) {
            unsigned issued = 0;
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int r = it / nch, c = it % nch;
                if (active && !active[r]) continue;
                const int t0 = c * dot_tpi(ntiles), t1 = min(t0 + dot_tpi(ntiles), ntiles);
                const float4 *Vr = V + r * sV, *wr = w + r * sw;
                for (int i0 = 0; i0 < nvec; i0 += kGroup) {
                    const int nq = min(kGroup, nvec - i0);
                    for (int tl = t0; tl < t1; ++tl, ++k) {
                        const size_t p0 = (size_t)tl * kDotTile;
                        const unsigned bytes = (unsigned)min((size_t)kDotTile, N - p0) * 16u;
                        const int s = (int)(k % kDotStages);
                        if (!pipe::mbar_wait(&S.empty[s], ((k / kDotStages) & 1u) ^ 1u, &S.abort) ||
                            aborted(S.abort))
                            continue;
                        pipe::mbar_arrive_expect_tx(&S.full[s], bytes * (nq + 1));
                        pipe::bulk_load(&S.slot[s][0][0], wr + p0, bytes, &S.full[s]);
                        for (int q = 0; q < nq; ++q)
                            pipe::bulk_load(&S.slot[s][1 + q][0], Vr + (size_t)(i0 + q) * N + p0, bytes, &S.full[s]);
                        issued = k + 1;
                    }
                }
            }
            ring_drain(S.full, issued);
        }
        __syncwarp();
        __syncthreads();
        return;
    }
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const int t = threadIdx.x;
    const unsigned long long wait_ns = g_cons_wait_ns;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int r = it / nch, c = it % nch;
        if (active && !active[r]) continue;
        const int t0 = c * dot_tpi(ntiles), t1 = min(t0 + dot_tpi(ntiles), ntiles);
        for (int i0 = 0; i0 < nvec; i0 += kGroup) {
            const int nq = min(kGroup, nvec - i0);
            float h[16], l[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) h[q] = l[q] = 0.f;
            // each accumulator sums the thread's nodes of the chunk in index
            // order; the first product into it initialises it (the same bits
            // as adding it to zero, without the two-sum)
            bool first = true;
            for (int tl = t0; tl < t1; ++tl, ++k) {
                const int nodes = (int)min((size_t)kDotTile, N - (size_t)tl * kDotTile);
                const int s = (int)(k % kDotStages);
                const bool ok = pipe::mbar_wait(&S.full[s], (k / kDotStages) & 1u, &S.abort, wait_ns);
                const bool in = ok && t < nodes;
                const float4 x = in ? S.slot[s][0][t] : zero;
                float4 v[kGroup];
#pragma unroll
                for (int q = 0; q < kGroup; ++q) v[q] = (in && q < nq) ? S.slot[s][1 + q][t] : zero;
                __syncwarp();
                if (lane == 0) pipe::mbar_arrive(&S.empty[s]);
#pragma unroll
                for (int q = 0; q < kGroup; ++q) {
                    if (q < nq) {
                        // conj(v) x: re = vr xr + vi xi, im = vr xi - vi xr
                        if (first) {
                            ds_init(h[2 * q], l[2 * q], v[q].x, v[q].y, x.x, x.y);
                            ds_init(h[2 * q + 1], l[2 * q + 1], v[q].x, v[q].y, x.z, x.w);
                        } else {
                            ds_fma(h[2 * q], l[2 * q], v[q].x, v[q].y, x.x, x.y);
                            ds_fma(h[2 * q + 1], l[2 * q + 1], v[q].x, v[q].y, x.z, x.w);
                        }
                        ds_fma(h[2 * q], l[2 * q], v[q].z, v[q].w, x.z, x.w);
                        ds_fma(h[2 * q + 1], l[2 * q + 1], -v[q].z, -v[q].w, x.x, x.y);
                    }
                }
                first = false;
            }
            float oh, ol;
            warp_reduce16_ds(h, l, oh, ol);
            const int comp = (lane >> 1) & 15;
            if ((lane & 1) == 0 && (comp >> 1) < nq) {
                double *dst = reinterpret_cast<double *>(
                    partial + (((size_t)r * nvec_max + i0 + (comp >> 1)) * nch + c) * kConsWarps + warp);
                dst[comp & 1] = S.abort ? qnan() : ds_join(oh, ol);
            }
        }
    }
    __syncthreads();
}

// out[r * ostride + i] = sum of the n partials of (r, i), in index order per
// thread, then warps and threads in a fixed tree
__global__ void __launch_bounds__(256)
k_dot_finalize(const double2 *__restrict__ partial, int nvec_max, int n, double2 *__restrict__ out,
               size_t ostride, const int *__restrict__ active) {
    const int i = blockIdx.x, r = blockIdx.y;
    if (active && !active[r]) return;
    const double2 *p = partial + ((size_t)r * nvec_max + i) * n;
    __shared__ double2 red[8];
    double sx = 0.0, sy = 0.0;
    for (int t = threadIdx.x; t < n; t += 256) {
        const double2 v = p[t];
        sx += v.x;
        sy += v.y;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(sx, sy);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = red[0];
        for (int q = 1; q < 8; ++q) {
            s.x += red[q].x;
            s.y += red[q].y;
        }
        out[r * ostride + i] = s;
    }
}

// w -= sum_i V_i c_i (c complex128, split into double-single by each warp per
// item); partial_d[(r * ntiles + tile) * 8 + warp] = warp's part of ||w||^2.
// Stages of item (r, tile): w, then V_0..V_{n-1}; the updated tile of w is
// stored from registers.
__global__ void __launch_bounds__(kPipeThreads, kAxpyBlocksPerSM)
k_multiaxpy_ds(const float4 *__restrict__ V, size_t sV, int nvec, const double2 *__restrict__ c,
               size_t cstride, float4 *__restrict__ w, size_t sw, size_t N, double *__restrict__ partial_d,
               int nrhs, const int *__restrict__ active) {
    constexpr int NPT = kAxpyTile / kCons;
    extern __shared__ __align__(128) unsigned char pipe_raw[];
    AxpySmem &S = *reinterpret_cast<AxpySmem *>(pipe_raw);
    float4 *cs = reinterpret_cast<float4 *>(pipe_raw + sizeof(AxpySmem)) + (threadIdx.x >> 5) * nvec;
    ring_init(S.full, S.empty, S.abort);
    const int ntiles = ceil_div(N, kAxpyTile);
    const int items = nrhs * ntiles;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned k = 0;
    if (warp == kConsWarps) {
        if (lane == 0) {
            unsigned issued = 0;
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int r = it / ntiles, tl = it % ntiles;
                if (active && !active[r]) continue;
                const size_t p0 = (size_t)tl * kAxpyTile;
                const unsigned bytes = (unsigned)min((size_t)kAxpyTile, N - p0) * 16u;
                const float4 *Vr = V + r * sV, *wr = w + r * sw;
                for (int i = -1; i < nvec; ++i, ++k) {
                    const int s = (int)(k % kAxpyStages);
                    if (!pipe::mbar_wait(&S.empty[s], ((k / kAxpyStages) & 1u) ^ 1u, &S.abort) ||
                        aborted(S.abort))
                        continue;
                    pipe::mbar_arrive_expect_tx(&S.full[s], bytes);
                    pipe::bulk_load(&S.slot[s][0], i < 0 ? wr + p0 : Vr + (size_t)i * N + p0, bytes, &S.full[s]);
                    issued = k + 1;
                }
            }
            ring_drain(S.full, issued);
        }
        __syncwarp();
        __syncthreads();
        return;
    }
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const int t = threadIdx.x;
    const unsigned long long wait_ns = g_cons_wait_ns;
    auto take = [&](int nodes, float4 (&a)[NPT]) {
        const int s = (int)(k % kAxpyStages);
        const bool ok = pipe::mbar_wait(&S.full[s], (k / kAxpyStages) & 1u, &S.abort, wait_ns);
#pragma unroll
        for (int m = 0; m < NPT; ++m) a[m] = (ok && t + m * kCons < nodes) ? S.slot[s][t + m * kCons] : zero;
        __syncwarp();
        if (lane == 0) pipe::mbar_arrive(&S.empty[s]);
        ++k;
    };
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int r = it / ntiles, tl = it % ntiles;
        if (active && !active[r]) continue;
        const size_t p0 = (size_t)tl * kAxpyTile;
        const int nodes = (int)min((size_t)kAxpyTile, N - p0);
        float4 *wr = w + r * sw;
        for (int i = lane; i < nvec; i += 32) {
            const double2 ci = c[r * cstride + i];
            cs[i] = cvt<float4>(make_double2(-ci.x, -ci.y));   // (re_hi, re_lo, im_hi, im_lo) of -c_i
        }
        __syncwarp();
        float4 xa[NPT];
        take(nodes, xa);
        float rh[NPT], rl[NPT], ih[NPT], il[NPT];
#pragma unroll
        for (int m = 0; m < NPT; ++m) {
            rh[m] = xa[m].x;
            rl[m] = xa[m].y;
            ih[m] = xa[m].z;
            il[m] = xa[m].w;
        }
        for (int i = 0; i < nvec; ++i) {
            float4 v[NPT];
            take(nodes, v);
            const float4 mc = cs[i];   // -c_i
#pragma unroll
            for (int m = 0; m < NPT; ++m) {
                // w += v * (-c): re = vr mr - vi mi, im = vr mi + vi mr
                ds_fma(rh[m], rl[m], v[m].x, v[m].y, mc.x, mc.y);
                ds_fma(rh[m], rl[m], -v[m].z, -v[m].w, mc.z, mc.w);
                ds_fma(ih[m], il[m], v[m].x, v[m].y, mc.z, mc.w);
                ds_fma(ih[m], il[m], v[m].z, v[m].w, mc.x, mc.y);
            }
        }
        // renormalise (h, l), store, and add to the thread's norm, node by node
        float nh = 0.f, nl = 0.f;
#pragma unroll
        for (int m = 0; m < NPT; ++m) {
            float th = rh[m] + rl[m];
            rl[m] = rl[m] - (th - rh[m]);
            rh[m] = th;
            th = ih[m] + il[m];
            il[m] = il[m] - (th - ih[m]);
            ih[m] = th;
            if (t + m * kCons < nodes) {
                wr[p0 + t + m * kCons] = make_float4(rh[m], rl[m], ih[m], il[m]);
                ds_fma(nh, nl, rh[m], rl[m], rh[m], rl[m]);
                ds_fma(nh, nl, ih[m], il[m], ih[m], il[m]);
            }
        }
        if (partial_d) {
            const double v = warp_sum(ds_join(nh, nl));
            if (lane == 0) partial_d[((size_t)r * ntiles + tl) * kConsWarps + warp] = S.abort ? qnan() : v;
        }
        __syncwarp();   // this warp's cs is rewritten by the next item
    }
    __syncthreads();
}

// ---------------------------------------------------------------- complex64 basis
// The same streamed multi-dot and multi-axpy for a basis stored in complex64
// (precision HELM_PREC_MIXED_C64): the vector w being orthogonalised is still
// double-single, the basis tiles are float2 and half the bytes. Each basis
// vector starts at a multiple of Nv elements, Nv = N rounded up to even, so
// every bulk copy starts on a 16-byte boundary and moves a multiple of 16
// bytes (a ragged last tile copies one padding element, which no consumer
// reads).
// half-size stages, so the ring is deeper than the double-single one (more
// bytes in flight per block)
constexpr int kDotStagesSB = 5;

struct DotSmemSB {
    float4 w[kDotStagesSB][kDotTile];
    float2 v[kDotStagesSB][kGroup][kDotTile];
    uint64_t full[kDotStagesSB], empty[kDotStagesSB];
    int abort;
};

// as k_multidot_ds; the products and each thread's sums over its nodes are
// plain FP32 against the high part of w (the coefficients only set how
// orthogonal the new vector comes out: the update below subtracts the same h
// that enter the Hessenberg, in double-single), the warp, block and chunk
// sums double-single and FP64
__global__ void __launch_bounds__(kPipeThreads, kDotBlocksPerSM)
k_multidot_sb(const float2 *__restrict__ V, size_t sV, size_t Nv, int nvec, const float4 *__restrict__ w,
              size_t sw, size_t N, double2 *__restrict__ partial, int nvec_max, int nrhs,
              const int *__restrict__ active) {
    extern __shared__ __align__(128) unsigned char pipe_raw[];
    DotSmemSB &S = *reinterpret_cast<DotSmemSB *>(pipe_raw);
    ring_init(S.full, S.empty, S.abort);
    const int ntiles = ceil_div(N, kDotTile), nch = ceil_div(ntiles, dot_tpi(ntiles));
    const int items = nrhs * nch;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned k = 0;
    if (warp == kConsWarps) {
        if (lane == 0) {
            unsigned issued = 0;
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int r = it / nch, c = it % nch;
                if (active && !active[r]) continue;
                const int t0 = c * dot_tpi(ntiles), t1 = min(t0 + dot_tpi(ntiles), ntiles);
                const float2 *Vr = V + r * sV;
                const float4 *wr = w + r * sw;
                for (int i0 = 0; i0 < nvec; i0 += kGroup) {
                    const int nq = min(kGroup, nvec - i0);
                    for (int tl = t0; tl < t1; ++tl, ++k) {
                        const size_t p0 = (size_t)tl * kDotTile;
                        const unsigned nodes = (unsigned)min((size_t)kDotTile, N - p0);
                        const unsigned bw = nodes * 16u, bv = ((nodes + 1u) & ~1u) * 8u;
                        const int s = (int)(k % kDotStagesSB);
                        if (!pipe::mbar_wait(&S.empty[s], ((k / kDotStagesSB) & 1u) ^ 1u, &S.abort) ||
                            aborted(S.abort))
                            continue;
                        pipe::mbar_arrive_expect_tx(&S.full[s], bw + bv * nq);
                        pipe::bulk_load(&S.w[s][0], wr + p0, bw, &S.full[s]);
                        for (int q = 0; q < nq; ++q)
                            pipe::bulk_load(&S.v[s][q][0], Vr + (size_t)(i0 + q) * Nv + p0, bv, &S.full[s]);
                        issued = k + 1;
                    }
                }
            }
            ring_drain(S.full, issued);
        }
        __syncwarp();
        __syncthreads();
        return;
    }
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 zero2 = make_float2(0.f, 0.f);
    const int t = threadIdx.x;
    const unsigned long long wait_ns = g_cons_wait_ns;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int r = it / nch, c = it % nch;
        if (active && !active[r]) continue;
        const int t0 = c * dot_tpi(ntiles), t1 = min(t0 + dot_tpi(ntiles), ntiles);
        for (int i0 = 0; i0 < nvec; i0 += kGroup) {
            const int nq = min(kGroup, nvec - i0);
            float h[16], l[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) h[q] = l[q] = 0.f;
            for (int tl = t0; tl < t1; ++tl, ++k) {
                const int nodes = (int)min((size_t)kDotTile, N - (size_t)tl * kDotTile);
                const int s = (int)(k % kDotStagesSB);
                const bool ok = pipe::mbar_wait(&S.full[s], (k / kDotStagesSB) & 1u, &S.abort, wait_ns);
                const bool in = ok && t < nodes;
                const float4 x = in ? S.w[s][t] : zero4;
                float2 v[kGroup];
#pragma unroll
                for (int q = 0; q < kGroup; ++q) v[q] = (in && q < nq) ? S.v[s][q][t] : zero2;
                __syncwarp();
                if (lane == 0) pipe::mbar_arrive(&S.empty[s]);
#pragma unroll
                for (int q = 0; q < kGroup; ++q) {
                    // conj(v) x: re = vr xr + vi xi, im = vr xi - vi xr
                    h[2 * q] = fmaf(v[q].x, x.x, h[2 * q]);
                    h[2 * q] = fmaf(v[q].y, x.z, h[2 * q]);
                    h[2 * q + 1] = fmaf(v[q].x, x.z, h[2 * q + 1]);
                    h[2 * q + 1] = fmaf(-v[q].y, x.x, h[2 * q + 1]);
                }
            }
            float oh, ol;
            warp_reduce16_ds(h, l, oh, ol);
            const int comp = (lane >> 1) & 15;
            if ((lane & 1) == 0 && (comp >> 1) < nq) {
                double *dst = reinterpret_cast<double *>(
                    partial + (((size_t)r * nvec_max + i0 + (comp >> 1)) * nch + c) * kConsWarps + warp);
                dst[comp & 1] = S.abort ? qnan() : ds_join(oh, ol);
            }
        }
    }
    __syncthreads();
}

// as k_multiaxpy_ds with complex64 basis tiles (in the same ring slots): w
// stays double-single, each product of a basis entry with the double-single
// coefficient is exact as p + e
__global__ void __launch_bounds__(kPipeThreads, kAxpyBlocksPerSM)
k_multiaxpy_sb(const float2 *__restrict__ V, size_t sV, size_t Nv, int nvec, const double2 *__restrict__ c,
               size_t cstride, float4 *__restrict__ w, size_t sw, size_t N, double *__restrict__ partial_d,
               int nrhs, const int *__restrict__ active) {
    constexpr int NPT = kAxpyTile / kCons;
    extern __shared__ __align__(128) unsigned char pipe_raw[];
    AxpySmem &S = *reinterpret_cast<AxpySmem *>(pipe_raw);
    float4 *cs = reinterpret_cast<float4 *>(pipe_raw + sizeof(AxpySmem)) + (threadIdx.x >> 5) * nvec;
    ring_init(S.full, S.empty, S.abort);
    const int ntiles = ceil_div(N, kAxpyTile);
    const int items = nrhs * ntiles;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned k = 0;
    if (warp == kConsWarps) {
        if (lane == 0) {
            unsigned issued = 0;
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int r = it / ntiles, tl = it % ntiles;
                if (active && !active[r]) continue;
                const size_t p0 = (size_t)tl * kAxpyTile;
                const unsigned nodes = (unsigned)min((size_t)kAxpyTile, N - p0);
                const float2 *Vr = V + r * sV;
                const float4 *wr = w + r * sw;
                for (int i = -1; i < nvec; ++i, ++k) {
                    const int s = (int)(k % kAxpyStages);
                    if (!pipe::mbar_wait(&S.empty[s], ((k / kAxpyStages) & 1u) ^ 1u, &S.abort) ||
                        aborted(S.abort))
                        continue;
                    const unsigned bytes = i < 0 ? nodes * 16u : ((nodes + 1u) & ~1u) * 8u;
                    pipe::mbar_arrive_expect_tx(&S.full[s], bytes);
                    if (i < 0)
                        pipe::bulk_load(&S.slot[s][0], wr + p0, bytes, &S.full[s]);
                    else
                        pipe::bulk_load(&S.slot[s][0], Vr + (size_t)i * Nv + p0, bytes, &S.full[s]);
                    issued = k + 1;
                }
            }
            ring_drain(S.full, issued);
        }
        __syncwarp();
        __syncthreads();
        return;
    }
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 zero2 = make_float2(0.f, 0.f);
    const int t = threadIdx.x;
    const unsigned long long wait_ns = g_cons_wait_ns;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int r = it / ntiles, tl = it % ntiles;
        if (active && !active[r]) continue;
        const size_t p0 = (size_t)tl * kAxpyTile;
        const int nodes = (int)min((size_t)kAxpyTile, N - p0);
        float4 *wr = w + r * sw;
        for (int i = lane; i < nvec; i += 32) {
            const double2 ci = c[r * cstride + i];
            cs[i] = cvt<float4>(make_double2(-ci.x, -ci.y));   // (re_hi, re_lo, im_hi, im_lo) of -c_i
        }
        __syncwarp();
        float rh[NPT], rl[NPT], ih[NPT], il[NPT];
        {
            const int s = (int)(k % kAxpyStages);
            const bool ok = pipe::mbar_wait(&S.full[s], (k / kAxpyStages) & 1u, &S.abort, wait_ns);
#pragma unroll
            for (int m = 0; m < NPT; ++m) {
                const float4 a = (ok && t + m * kCons < nodes) ? S.slot[s][t + m * kCons] : zero4;
                rh[m] = a.x;
                rl[m] = a.y;
                ih[m] = a.z;
                il[m] = a.w;
            }
            __syncwarp();
            if (lane == 0) pipe::mbar_arrive(&S.empty[s]);
            ++k;
        }
        for (int i = 0; i < nvec; ++i) {
            const int s = (int)(k % kAxpyStages);
            const bool ok = pipe::mbar_wait(&S.full[s], (k / kAxpyStages) & 1u, &S.abort, wait_ns);
            const float2 *vs = reinterpret_cast<const float2 *>(&S.slot[s][0]);
            float2 v[NPT];
#pragma unroll
            for (int m = 0; m < NPT; ++m) v[m] = (ok && t + m * kCons < nodes) ? vs[t + m * kCons] : zero2;
            __syncwarp();
            if (lane == 0) pipe::mbar_arrive(&S.empty[s]);
            ++k;
            const float4 mc = cs[i];   // -c_i
#pragma unroll
            for (int m = 0; m < NPT; ++m) {
                // w += v * (-c): re = vr mr - vi mi, im = vr mi + vi mr
                ds_fma1(rh[m], rl[m], v[m].x, mc.x, mc.y);
                ds_fma1(rh[m], rl[m], -v[m].y, mc.z, mc.w);
                ds_fma1(ih[m], il[m], v[m].x, mc.z, mc.w);
                ds_fma1(ih[m], il[m], v[m].y, mc.x, mc.y);
            }
        }
        float nh = 0.f, nl = 0.f;
#pragma unroll
        for (int m = 0; m < NPT; ++m) {
            float th = rh[m] + rl[m];
            rl[m] = rl[m] - (th - rh[m]);
            rh[m] = th;
            th = ih[m] + il[m];
            il[m] = il[m] - (th - ih[m]);
            ih[m] = th;
            if (t + m * kCons < nodes) {
                wr[p0 + t + m * kCons] = make_float4(rh[m], rl[m], ih[m], il[m]);
                ds_fma(nh, nl, rh[m], rl[m], rh[m], rl[m]);
                ds_fma(nh, nl, ih[m], il[m], ih[m], il[m]);
            }
        }
        if (partial_d) {
            const double v = warp_sum(ds_join(nh, nl));
            if (lane == 0) partial_d[((size_t)r * ntiles + tl) * kConsWarps + warp] = S.abort ? qnan() : v;
        }
        __syncwarp();   // this warp's cs is rewritten by the next item
    }
    __syncthreads();
}

// norm2[r] = sum of the n partials of r (fixed order, as k_dot_finalize);
// with sc, also the scale 1/sqrt(norm2[r]) split into float hi + lo parts
// (the complex64 basis's v = w / ||w||, formed by the next level-0 V-cycle
// kernel)
__global__ void __launch_bounds__(256)
k_norm_finalize(const double *__restrict__ partial_d, int n, double *__restrict__ norm2,
                float2 *__restrict__ sc, const int *__restrict__ active) {
    const int r = blockIdx.x;
    if (active && !active[r]) return;
    const double *p = partial_d + (size_t)r * n;
    __shared__ double red[8];
    double s = 0.0;
    for (int t = threadIdx.x; t < n; t += 256) s += p[t];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = red[0];
        for (int q = 1; q < 8; ++q) a += red[q];
        norm2[r] = a;
        if (sc) {
            const double t = 1.0 / sqrt(a);
            const float th = (float)t;
            sc[r] = make_float2(th, (float)(t - (double)th));
        }
    }
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


inline int blocks_for(size_t N, int cap) {
    size_t b = (N + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    return (int)(b < (size_t)cap ? b : cap);
}

}  // namespace

namespace {
void set_pipe_attrs() {
    static const int once = [] {
        cudaFuncSetAttribute(k_multidot_ds, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DotSmem));
        cudaFuncSetAttribute(k_multiaxpy_ds, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(AxpySmem) + kConsWarps * kMaxVec * sizeof(float4)));
        cudaFuncSetAttribute(k_multidot_sb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DotSmemSB));
        cudaFuncSetAttribute(k_multiaxpy_sb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(AxpySmem) + kConsWarps * kMaxVec * sizeof(float4)));
        return 1;
    }();
    (void)once;
}
int pipe_grid(int items, int per_sm) {
    const int cap = device_sms() * per_sm;
    return items < cap ? (items > 0 ? items : 1) : cap;
}
}  // namespace

cudaError_t set_consumer_wait_ns(unsigned long long ns) {
    return cudaMemcpyToSymbol(g_cons_wait_ns, &ns, sizeof ns);
}

size_t ds_partial_per_rhs(size_t N, int nvec_max) {
    const size_t dot = (size_t)nvec_max * ceil_div(ceil_div(N, kDotTile), dot_tpi(ceil_div(N, kDotTile))) * kConsWarps;
    const size_t axpy = ((size_t)ceil_div(N, kAxpyTile) * kConsWarps + 1) / 2;   // doubles, in double2 units
    return dot > axpy ? dot : axpy;
}

void launch_multidot_ds(const float4 *V, size_t sV, int nvec, const float4 *w, size_t sw, size_t N,
                        double2 *out, size_t out_stride, int nrhs, const int *active,
                        KrylovScratch &ks, cudaStream_t st) {
    set_pipe_attrs();
    const int nch = ceil_div(ceil_div(N, kDotTile), dot_tpi(ceil_div(N, kDotTile)));
    const int nb = pipe_grid(nrhs * nch, kDotBlocksPerSM);
    prof_begin(st);
    k_multidot_ds<<<nb, kPipeThreads, sizeof(DotSmem), st>>>(V, sV, nvec, w, sw, N, ks.partial,
                                                             ks.nvec_max, nrhs, active);
    k_dot_finalize<<<dim3(nvec, nrhs), 256, 0, st>>>(ks.partial, ks.nvec_max, nch * kConsWarps, out,
                                                     out_stride, active);
    count_launch(2);
    if (prof_on())
        prof_end("multidot_ds", st, (nvec + 1.0) * N * 16.0 * nrhs, 0.0);
}

void launch_multiaxpy_ds(const float4 *V, size_t sV, int nvec, const double2 *c, size_t c_stride,
                         float4 *w, size_t sw, size_t N, double *norm2, int nrhs, const int *active,
                         KrylovScratch &ks, cudaStream_t st) {
    set_pipe_attrs();
    const int ntiles = ceil_div(N, kAxpyTile);
    const int nb = pipe_grid(nrhs * ntiles, kAxpyBlocksPerSM);
    double *pd = norm2 ? (double *)ks.partial : nullptr;
    prof_begin(st);
    k_multiaxpy_ds<<<nb, kPipeThreads, sizeof(AxpySmem) + kConsWarps * nvec * sizeof(float4), st>>>(
        V, sV, nvec, c, c_stride, w, sw, N, pd, nrhs, active);
    count_launch();
    if (norm2) {
        k_norm_finalize<<<nrhs, 256, 0, st>>>(pd, ntiles * kConsWarps, norm2, nullptr, active);
        count_launch();
    }
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

void launch_multidot_sb(const float2 *V, size_t sV, size_t Nv, int nvec, const float4 *w, size_t sw, size_t N,
                        double2 *out, size_t out_stride, int nrhs, const int *active, KrylovScratch &ks,
                        cudaStream_t st) {
    set_pipe_attrs();
    const int nch = ceil_div(ceil_div(N, kDotTile), dot_tpi(ceil_div(N, kDotTile)));
    const int nb = pipe_grid(nrhs * nch, kDotBlocksPerSM);
    prof_begin(st);
    k_multidot_sb<<<nb, kPipeThreads, sizeof(DotSmemSB), st>>>(V, sV, Nv, nvec, w, sw, N, ks.partial, ks.nvec_max,
                                                              nrhs, active);
    k_dot_finalize<<<dim3(nvec, nrhs), 256, 0, st>>>(ks.partial, ks.nvec_max, nch * kConsWarps, out, out_stride,
                                                     active);
    count_launch(2);
    if (prof_on()) prof_end("multidot_c64", st, (nvec * 8.0 + 16.0) * N * nrhs, 0.0);
}

void launch_multiaxpy_sb(const float2 *V, size_t sV, size_t Nv, int nvec, const double2 *c, size_t c_stride,
                         float4 *w, size_t sw, size_t N, double *norm2, int nrhs, const int *active,
                         KrylovScratch &ks, cudaStream_t st, float2 *scale) {
    set_pipe_attrs();
    const int ntiles = ceil_div(N, kAxpyTile);
    const int nb = pipe_grid(nrhs * ntiles, kAxpyBlocksPerSM);
    double *pd = norm2 ? (double *)ks.partial : nullptr;
    prof_begin(st);
    k_multiaxpy_sb<<<nb, kPipeThreads, sizeof(AxpySmem) + kConsWarps * nvec * sizeof(float4), st>>>(
        V, sV, Nv, nvec, c, c_stride, w, sw, N, pd, nrhs, active);
    count_launch();
    if (norm2) {
        k_norm_finalize<<<nrhs, 256, 0, st>>>(pd, ntiles * kConsWarps, norm2, scale, active);
        count_launch();
    }
    if (prof_on()) prof_end("multiaxpy_c64", st, (nvec * 8.0 + 32.0) * N * nrhs, 0.0);
}

}  // namespace helm
