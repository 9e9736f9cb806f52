// Block flexible GMRES (Eq. 7, right-preconditioned by the shifted Laplacian
// of Eq. 6) for up to 64 sources that share H and M: the sources share one
// block Krylov space, so every block step widens the space by one vector per
// source and each source minimises its residual over all of it.
//
// One block step j (V_0..V_j orthonormal blocks of s vectors):
//   Z_j = M^-1 V_j            complex64 V-cycle on the s vectors
//   W   = H Z_j               complex128 stencil, stored in complex64
//   two passes of block classical Gram-Schmidt:
//     G = [V_0..V_j]^H W      tensor cores (k_bgram + k_bgram_sum)
//     W = W - [V_0..V_j] G    tensor cores (k_bcomb)
//   W = V_{j+1} R             two passes of Cholesky QR: G = W^H W on the
//                             tensor cores, R^H R = G (+ shift on the first
//                             pass) in FP64 (k_bchol), W = W R^-1 on the
//                             tensor cores
//   block Hessenberg QR       Householder reflectors, one per column, FP64
//                             (k_bls: s co-resident blocks, one per column)
//   stop when every source's least-squares residual is <= tol ||f||
// A cycle ends with Y = R^-1 g (k_bbacksolve), x += Z Y (tensor cores, then
// widened into complex128) and the true residual in complex128; a source
// whose true residual is above tol restarts the whole block from
// R = F - H X = V_0 B.
//
// Tensor-core contractions. Both run tcgen05.mma kind::tf32 with FP32
// accumulators in TMEM on operands split into TF32 hi + lo (three MMAs per
// product, FP32 accuracy). Complex values stay interleaved (re, im) along K:
//   Gram: A = basis vectors (rows, K = 2 floats per node), B = [W | W'] with
//         W' = (im, -re) per node, so one real MMA of N = 128 columns gives
//         Re G (columns 0..63) and Im G (64..127). A CTA owns a range of
//         nodes and up to four 128-row tiles (512 TMEM columns); partial sums
//         per node range are added in FP64 in a fixed order.
//   Combine: out = alpha W + V C with A = nodes x (2 floats per basis
//         vector), B = the real image of C (columns: Re out, Im out), built
//         once per call in the operand layout and streamed by cp.async.bulk.
// The basis, Z and W are complex64 with a per-vector stride Np (N rounded up
// to 8 nodes, zero padded) so that every vector starts 64-byte aligned.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cycle.cuh"
#include "tc.cuh"
#include "vcycle.cuh"

namespace helm {

namespace {

constexpr int kBS = 64;            // sources per block (MMA N = 128 real columns)
constexpr int kTM = 128;           // rows per MMA tile
constexpr int kTiles = 4;          // tiles per CTA (4 x 128 TMEM columns)
constexpr int kKS = 16;            // K floats per pipeline stage
constexpr int kPlane = kTM * kKS;  // floats per operand plane of a stage
constexpr int kBT = 256;           // threads of the tensor-core kernels
constexpr uint32_t kTmemCols = 512;
constexpr int kGramNodes = kKS / 2;   // Gram: nodes per stage
constexpr int kCombVecs = kKS / 2;    // combine: basis vectors per stage
constexpr int kCombNodes = kTiles * kTM;

__device__ __forceinline__ float qnanf() { return __int_as_float(0x7fc00000); }
__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7ff8000000000000ll); }

struct alignas(1024) TcStages {
    float a[2][kTiles][2][kPlane];   // stage, tile, plane (hi, lo)
    float b[2][2][kPlane];           // stage, plane
    uint64_t bbar[2], mbar[2];       // B landed (combine); the stage's MMAs complete
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ void split4(float4 x, float4 &hi, float4 &lo) {
    hi = make_float4(tc::tf32_hi(x.x), tc::tf32_hi(x.y), tc::tf32_hi(x.z), tc::tf32_hi(x.w));
    lo = make_float4(x.x - hi.x, x.y - hi.y, x.z - hi.z, x.w - hi.w);
}

// Issue the 2 x 3 MMAs of one stage for tile t (K = 16 = two steps of 8):
// D += A_hi B_hi + A_hi B_lo + A_lo B_hi.
__device__ __forceinline__ void stage_mmas(const TcStages &S, int st, int t, uint32_t d, bool first) {
    constexpr uint32_t idesc = tc::idesc_tf32(kTM, 128);
    constexpr unsigned lbo = 128, sbo = (kKS / 4) * 128;
#pragma unroll
    for (int kk = 0; kk < kKS / 8; ++kk) {
        const uint64_t ah = tc::smem_desc(&S.a[st][t][0][kk * 64], lbo, sbo);
        const uint64_t al = tc::smem_desc(&S.a[st][t][1][kk * 64], lbo, sbo);
        const uint64_t bh = tc::smem_desc(&S.b[st][0][kk * 64], lbo, sbo);
        const uint64_t bl = tc::smem_desc(&S.b[st][1][kk * 64], lbo, sbo);
        tc::mma_tf32(d, ah, bh, idesc, (first && kk == 0) ? 0u : 1u);
        tc::mma_tf32(d, ah, bl, idesc, 1u);
        tc::mma_tf32(d, al, bh, idesc, 1u);
    }
}

// Last MMAs of the CTA: wait (bounded, retried) before reading TMEM.
__device__ __forceinline__ void wait_last(TcStages &S, int n) {
    if (n <= 0) return;
    const int il = n - 1;
    bool done = false;
    for (int a = 0; a < 4 && !done; ++a) done = pipe::mbar_wait_drain(&S.mbar[il & 1], (unsigned)(il >> 1) & 1u);
    if (!done) S.abort = 1;
}

// ------------------------------------------------------------------ Gram
// part[((kc * nv) + i) * 128 + col]: node range kc's share of
//   sum_p Re/Im conj(V_i[p]) W_c[p]   (col = c: real part, col = 64 + c: imaginary part)
__global__ void __launch_bounds__(kBT, 1)
k_bgram(const float2 *__restrict__ V, size_t sv, int nv, const float2 *__restrict__ W, size_t sw, int s,
        size_t Np, int chunk, float *__restrict__ part) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    TcStages &S = *reinterpret_cast<TcStages *>(tc_raw);
    const int kc = blockIdx.x, mg = blockIdx.y;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int row0 = mg * kTiles * kTM;
    const int ntile = min(kTiles, (nv - row0 + kTM - 1) / kTM);
    const size_t p0 = (size_t)kc * chunk;
    const size_t p1 = min(p0 + (size_t)chunk, Np);
    const int nsub = p1 > p0 ? (int)((p1 - p0) / kGramNodes) : 0;   // Np, chunk: multiples of 8
    if (t == 0) {
        for (int st = 0; st < 2; ++st) pipe::mbar_init(&S.mbar[st], 1);
        S.abort = 0;
        pipe::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&S.tmem, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    // thread t loads rows (t + 256 u) / 4, node pair (t % 4) of the stage, and
    // source t / 4 of W (complex values interleaved: one float4 = two nodes)
    auto load = [&](int it, float4 (&a)[8], float4 &b) {
        const size_t pn = p0 + (size_t)it * kGramNodes + 2 * (t & 3);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int row = (t >> 2) + 64 * u;
            a[u] = (row < ntile * kTM && row0 + row < nv)
                       ? *reinterpret_cast<const float4 *>(V + (size_t)(row0 + row) * sv + pn)
                       : zero;
        }
        const int c = t >> 2;
        b = c < s ? *reinterpret_cast<const float4 *>(W + (size_t)c * sw + pn) : zero;
    };
    float4 ra[8], rb;
    if (nsub > 0) load(0, ra, rb);
    for (int it = 0; it < nsub; ++it) {
        const int st = it & 1;
        float4 na[8], nb = zero;
#pragma unroll
        for (int u = 0; u < 8; ++u) na[u] = zero;
        if (it + 1 < nsub) load(it + 1, na, nb);
        // stage st was last read by the MMAs of step it - 2
        if (it >= 2 && !pipe::mbar_wait_drain(&S.mbar[st], (unsigned)((it - 2) >> 1) & 1u)) S.abort = 1;
        tc::fence_after();
        if (!*(volatile int *)&S.abort) {
            const int k0 = 4 * (t & 3);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int row = (t >> 2) + 64 * u;
                float4 hi, lo;
                split4(ra[u], hi, lo);
                const int o = tc::cm_off<kKS>(row & (kTM - 1), k0);
                *reinterpret_cast<float4 *>(&S.a[st][row >> 7][0][o]) = hi;
                *reinterpret_cast<float4 *>(&S.a[st][row >> 7][1][o]) = lo;
            }
            const int c = t >> 2;
            float4 hi, lo;
            split4(rb, hi, lo);                         // (re0, im0, re1, im1): column c
            *reinterpret_cast<float4 *>(&S.b[st][0][tc::cm_off<kKS>(c, k0)]) = hi;
            *reinterpret_cast<float4 *>(&S.b[st][1][tc::cm_off<kKS>(c, k0)]) = lo;
            split4(make_float4(rb.y, -rb.x, rb.w, -rb.z), hi, lo);   // (im, -re): column 64 + c
            *reinterpret_cast<float4 *>(&S.b[st][0][tc::cm_off<kKS>(64 + c, k0)]) = hi;
            *reinterpret_cast<float4 *>(&S.b[st][1][tc::cm_off<kKS>(64 + c, k0)]) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> MMA reads
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (t == 0) {
            if (!*(volatile int *)&S.abort)
                for (int tl = 0; tl < ntile; ++tl) stage_mmas(S, st, tl, tmem + (uint32_t)(tl * 128), it == 0);
            tc::mma_commit(&S.mbar[st]);
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 8; ++u) ra[u] = na[u];
        rb = nb;
    }
    if (t == 0) wait_last(S, nsub);
    __syncthreads();
    tc::fence_after();
    const bool bad = S.abort != 0;
    // warp w reads TMEM lanes 32 (w % 4).. (rows of a tile), columns 64 (w / 4)..
    for (int tl = 0; tl < ntile; ++tl) {
        uint32_t v[64];
        tc::tmem_ld64(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(tl * 128 + 64 * (warp >> 2)), v);
        const int row = row0 + tl * kTM + 32 * (warp & 3) + lane;
        if (row < nv) {
            float4 *dst = reinterpret_cast<float4 *>(part + ((size_t)kc * nv + row) * 128 + 64 * (warp >> 2));
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                float4 o;
                o.x = nsub == 0 ? 0.f : bad ? qnanf() : __uint_as_float(v[4 * q]);
                o.y = nsub == 0 ? 0.f : bad ? qnanf() : __uint_as_float(v[4 * q + 1]);
                o.z = nsub == 0 ? 0.f : bad ? qnanf() : __uint_as_float(v[4 * q + 2]);
                o.w = nsub == 0 ? 0.f : bad ? qnanf() : __uint_as_float(v[4 * q + 3]);
                dst[q] = o;
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tmem, kTmemCols);
}

// G[i * ldg + c] = sum over node ranges (in order) of the partials; with
// hacc, also Hacc[c * ldh + i] = G (add = 0) or += G (add = 1): the block
// Hessenberg column, column-major
__global__ void k_bgram_sum(const float *__restrict__ part, int nkc, int nv, int s, double2 *__restrict__ G,
                            int ldg, double2 *__restrict__ hacc, size_t ldh, int add) {
    const int i = blockIdx.x, c = threadIdx.x;
    if (c >= s) return;
    double re = 0.0, im = 0.0;
    for (int kc = 0; kc < nkc; ++kc) {
        const float *p = part + ((size_t)kc * nv + i) * 128;
        re += (double)p[c];
        im += (double)p[64 + c];
    }
    const double2 gv = make_double2(re, im);
    if (G) G[(size_t)i * ldg + c] = gv;
    if (hacc) {
        double2 &h = hacc[(size_t)c * ldh + i];
        h = add ? make_double2(h.x + re, h.y + im) : gv;
    }
}

// ------------------------------------------------------------------ combine
// Real image of sign * C (nv x s complex, C[i * ldc + c]) in the B-operand
// layout: chunk kc (basis vectors 8 kc .. 8 kc + 7), planes hi / lo of a
// 128-column x 16-K tile; K = 2 i + comp, columns c (real part of out) and
// 64 + c (imaginary part).
__global__ void k_bcomb_image(const double2 *__restrict__ C, int ldc, int nv, int s, double sign,
                              float *__restrict__ img) {
    const int kc = blockIdx.x;
    for (int e = threadIdx.x; e < 128 * kKS; e += blockDim.x) {
        const int n = e / kKS, k = e % kKS;
        const int i = kc * kCombVecs + (k >> 1), comp = k & 1, c = n & 63, part = n >> 6;
        double v = 0.0;
        if (i < nv && c < s) {
            const double2 z = C[(size_t)i * ldc + c];
            const double zr = sign * z.x, zi = sign * z.y;
            // out_re = sum vr zr - vi zi; out_im = sum vr zi + vi zr
            v = part == 0 ? (comp == 0 ? zr : -zi) : (comp == 0 ? zi : zr);
        }
        const float f = (float)v;
        const float hi = tc::tf32_hi(f);
        const int o = tc::cm_off<kKS>(n, k);
        img[((size_t)kc * 2 + 0) * kPlane + o] = hi;
        img[((size_t)kc * 2 + 1) * kPlane + o] = f - hi;
    }
}

// out[c * so + p] = alpha * win[c * sw + p] + sum_i V_i[p] C_ic for nodes p of
// this CTA's 512-node tile (c < s). out may be win, and V may be win too
// (each CTA reads only its own nodes, all before its epilogue writes).
__global__ void __launch_bounds__(kBT, 1)
k_bcomb(const float2 *__restrict__ V, size_t sv, int nv, const float *__restrict__ img,
        const float2 *win, size_t sw, float alpha, float2 *out, size_t so, int s, size_t N,
        size_t Np) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    TcStages &S = *reinterpret_cast<TcStages *>(tc_raw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const size_t p0 = (size_t)blockIdx.x * kCombNodes;
    const int nch = (nv + kCombVecs - 1) / kCombVecs;
    const unsigned bbytes = 2u * kPlane * sizeof(float);
    unsigned issued[2] = {0u, 0u};
    auto copy_b = [&](int it) {
        const int st = it & 1;
        pipe::mbar_arrive_expect_tx(&S.bbar[st], bbytes);
        pipe::bulk_load(&S.b[st][0][0], img + (size_t)it * 2 * kPlane, bbytes, &S.bbar[st]);
        ++issued[st];
    };
    if (t == 0) {
        for (int st = 0; st < 2; ++st) {
            pipe::mbar_init(&S.bbar[st], 1);
            pipe::mbar_init(&S.mbar[st], 1);
        }
        S.abort = 0;
        pipe::mbar_init_fence();
        if (nch > 0) copy_b(0);
        if (nch > 1) copy_b(1);
    }
    if (warp == 0) tc::tmem_alloc(&S.tmem, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    // thread t loads vector (t + 256 u) / 256 = u of the stage, nodes 2 (t % 256), +1
    auto load = [&](int it, float4 (&a)[8]) {
        const size_t pn = p0 + 2 * (size_t)t;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = it * kCombVecs + u;
            a[u] = (i < nv && pn < Np) ? *reinterpret_cast<const float4 *>(V + (size_t)i * sv + pn) : zero;
        }
    };
    float4 ra[8];
    if (nch > 0) load(0, ra);
    for (int it = 0; it < nch; ++it) {
        const int st = it & 1;
        const unsigned ph = (unsigned)(it >> 1) & 1u;
        float4 na[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) na[u] = zero;
        if (it + 1 < nch) load(it + 1, na);
        if (it >= 2 && !pipe::mbar_wait_drain(&S.mbar[st], ph ^ 1u)) S.abort = 1;
        tc::fence_after();
        if (!*(volatile int *)&S.abort) {
            // node pair (2t, 2t + 1) of the 512-node tile: tile 2t / 128, rows r, r + 1
            const int nl = 2 * t, tl = nl >> 7, r = nl & (kTM - 1);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float4 hi, lo;
                split4(ra[u], hi, lo);
                const int o0 = tc::cm_off<kKS>(r, 2 * u), o1 = tc::cm_off<kKS>(r + 1, 2 * u);
                *reinterpret_cast<float2 *>(&S.a[st][tl][0][o0]) = make_float2(hi.x, hi.y);
                *reinterpret_cast<float2 *>(&S.a[st][tl][1][o0]) = make_float2(lo.x, lo.y);
                *reinterpret_cast<float2 *>(&S.a[st][tl][0][o1]) = make_float2(hi.z, hi.w);
                *reinterpret_cast<float2 *>(&S.a[st][tl][1][o1]) = make_float2(lo.z, lo.w);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (t == 0) {
            if (pipe::mbar_wait(&S.bbar[st], ph, &S.abort))
                for (int tl = 0; tl < kTiles; ++tl) stage_mmas(S, st, tl, tmem + (uint32_t)(tl * 128), it == 0);
            tc::mma_commit(&S.mbar[st]);
            // refill the other stage's B with chunk it + 1 once chunk it - 1's MMAs read it
            if (it >= 1 && it + 1 < nch) {
                const int so2 = st ^ 1;
                if (pipe::mbar_wait(&S.mbar[so2], (unsigned)((it - 1) >> 1) & 1u, &S.abort)) copy_b(it + 1);
            }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 8; ++u) ra[u] = na[u];
    }
    if (t == 0) wait_last(S, nch);
    __syncthreads();
    tc::fence_after();
    const bool bad = S.abort != 0;
    // warps 0-3: tiles 0, 1; warps 4-7: tiles 2, 3; lanes = nodes
    for (int q = 0; q < 2; ++q) {
        const int tl = 2 * (warp >> 2) + q;
        uint32_t vr[64], vi[64];
        const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(tl * 128);
        tc::tmem_ld64(ta, vr);
        tc::tmem_ld64(ta + 64, vi);
        const size_t p = p0 + (size_t)tl * kTM + 32 * (warp & 3) + lane;
        if (p < N) {
#pragma unroll
            for (int c = 0; c < kBS; ++c) {
                if (c < s) {
                    float2 o = make_float2(0.f, 0.f);
                    if (alpha != 0.f) {
                        const float2 w = win[(size_t)c * sw + p];
                        o = make_float2(alpha * w.x, alpha * w.y);
                    }
                    if (nch > 0) {
                        o.x += bad ? qnanf() : __uint_as_float(vr[c]);
                        o.y += bad ? qnanf() : __uint_as_float(vi[c]);
                    }
                    out[(size_t)c * so + p] = o;
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tmem, kTmemCols);
    if (t == 0 && bad)
        for (int st = 0; st < 2; ++st)
            if (issued[st]) pipe::mbar_wait_drain(&S.bbar[st], (issued[st] - 1) & 1u);
}

// ------------------------------------------------------------------ small dense FP64 kernels
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {   // conj(a) b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscal(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

constexpr int kCh = 256;   // threads of the Cholesky kernel

__device__ __forceinline__ float2 fmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 fconjmulc(float2 a, float2 b) {   // conj(a) b
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// Cholesky QR step on the s x s Gram G = W^H W (row-major, Hermitian):
// R^H R = G + shift_rel * max(diag G) I with R upper triangular, in FP32 (the
// Gram itself is FP32-accurate). A pivot at or below 1e-7 max(diag G) marks
// a direction W has lost: its row of R and column of R^-1 are zero. Writes
// Rinv (row-major, upper) for W <- W R^-1, and Racc <- R Racc (upper,
// row-major: the accumulated R of the passes), both as complex128.
__global__ void __launch_bounds__(kCh)
k_bchol(const double2 *__restrict__ G, int s, double shift_rel, double2 *__restrict__ Rinv,
        double2 *__restrict__ Racc, int first) {
    extern __shared__ float2 chol_raw[];
    float2 *A = chol_raw;                 // working copy, then R
    float2 *X = chol_raw + kBS * kBS;     // R^-1
    __shared__ float maxd;
    const int tid = threadIdx.x;
    for (int e = tid; e < s * s; e += kCh) A[e] = make_float2((float)G[e].x, (float)G[e].y);
    __syncthreads();
    if (tid == 0) {
        float mx = 0.f;
        for (int k = 0; k < s; ++k) mx = fmaxf(mx, A[k * s + k].x);
        maxd = mx;
    }
    __syncthreads();
    const float floor_ = 1e-7f * maxd, shift = (float)shift_rel * maxd;
    for (int k = tid; k < s; k += kCh) A[k * s + k].x += shift;
    __syncthreads();
    for (int k = 0; k < s; ++k) {
        const float d = A[k * s + k].x;
        const bool dead = !(d > floor_);
        const float rk = dead ? 0.f : sqrtf(d);
        __syncthreads();
        for (int jj = tid; jj < s; jj += kCh) {
            if (jj < k) A[k * s + jj] = make_float2(0.f, 0.f);
            else if (jj == k) A[k * s + jj] = make_float2(rk, 0.f);
            else A[k * s + jj] = dead ? make_float2(0.f, 0.f) : make_float2(A[k * s + jj].x / rk, A[k * s + jj].y / rk);
        }
        __syncthreads();
        if (!dead)
            for (int e = tid; e < (s - k - 1) * (s - k - 1); e += kCh) {
                const int i = k + 1 + e / (s - k - 1), jj = k + 1 + e % (s - k - 1);
                if (i <= jj) {
                    const float2 t = fconjmulc(A[k * s + i], A[k * s + jj]);
                    A[i * s + jj] = make_float2(A[i * s + jj].x - t.x, A[i * s + jj].y - t.y);
                }
            }
        __syncthreads();
    }
    // X = R^-1 by rows from the bottom: X_ij = (delta_ij - sum_{i<l<=j} R_il X_lj) / R_ii
    for (int e = tid; e < s * s; e += kCh) X[e] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int i = s - 1; i >= 0; --i) {
        const float rii = A[i * s + i].x;
        for (int jj = i + tid; jj < s; jj += kCh) {
            float2 acc = make_float2(jj == i ? 1.f : 0.f, 0.f);
            for (int l = i + 1; l <= jj; ++l) {
                const float2 t = fmulc(A[i * s + l], X[l * s + jj]);
                acc = make_float2(acc.x - t.x, acc.y - t.y);
            }
            X[i * s + jj] = rii > 0.f ? make_float2(acc.x / rii, acc.y / rii) : make_float2(0.f, 0.f);
        }
        __syncthreads();
    }
    for (int e = tid; e < s * s; e += kCh) Rinv[e] = make_double2((double)X[e].x, (double)X[e].y);
    // Racc <- R Racc (first pass: Racc <- R), in FP32 like the factors: one
    // thread per output, the previous Racc staged in shared memory (A's
    // buffer is free once X is formed)
    __syncthreads();
    if (first) {
        for (int e = tid; e < s * s; e += kCh) Racc[e] = make_double2((double)A[e].x, (double)A[e].y);
        return;
    }
    float2 *P = X;                         // X was written out above
    for (int e = tid; e < s * s; e += kCh) P[e] = make_float2((float)Racc[e].x, (float)Racc[e].y);
    __syncthreads();
    for (int e = tid; e < s * s; e += kCh) {
        const int i = e / s, jj = e % s;
        float2 acc = make_float2(0.f, 0.f);
        for (int l = i; l <= jj; ++l) {
            const float2 t = fmulc(A[i * s + l], P[l * s + jj]);
            acc = make_float2(acc.x + t.x, acc.y + t.y);
        }
        Racc[e] = make_double2((double)acc.x, (double)acc.y);
    }
}

// R (row-major s x s) into the block Hessenberg rows r0 .. r0 + s - 1 of block
// column j (column-major, leading dimension ldh); the block above is left as is
__global__ void k_bput_r(const double2 *__restrict__ R, int s, double2 *__restrict__ Hb, size_t ldh, int r0,
                         int c0) {
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
        const int i = e / s, c = e % s;
        Hb[(size_t)(c0 + c) * ldh + r0 + i] = R[e];
    }
}

// least-squares right-hand side of a cycle: g[:, c] = (B[:, c]; 0)
__global__ void k_brhs_init(const double2 *__restrict__ B, int s, double2 *__restrict__ g, size_t ldh, int rows) {
    const int c = blockIdx.x;
    for (int i = threadIdx.x; i < rows; i += blockDim.x)
        g[(size_t)c * ldh + i] = i < s ? B[i * s + c] : make_double2(0.0, 0.0);
}

constexpr unsigned long long kLsWaitNs = 500ull * 1000 * 1000;
constexpr int kLsThreads = 32;       // one warp per column of the new block
constexpr int kMaxRows = 64 * 33;    // rows of the block Hessenberg kept in shared memory
constexpr int kLsDepth = 4;          // reflectors of earlier blocks loaded ahead

__device__ __forceinline__ double2 warp_csum(double2 a) {
    for (int o = 16; o; o >>= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
        a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
    }
    return a;
}

// lane l's share v[l], v[l + 32], v[l + 64] of a reflector (k <= s; zeros beyond)
__device__ __forceinline__ void load_refl(const double2 *v, int s, bool l2only, double2 (&r)[3]) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int k = lane + 32 * q;
        r[q] = k <= s ? (l2only ? __ldcg(v + k) : __ldg(v + k)) : make_double2(0.0, 0.0);
    }
}

// x[0 .. s] (shared memory) -= tau v (v^H x), one warp
__device__ __forceinline__ void warp_refl(const double2 (&v)[3], double tau, double2 *x, int s) {
    const int lane = threadIdx.x;
    double2 xs[3], a = make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int k = lane + 32 * q;
        xs[q] = k <= s ? x[k] : make_double2(0.0, 0.0);
        a = cadd(a, cconjmul(v[q], xs[q]));
    }
    a = warp_csum(a);
    const double2 f = cscal(tau, a);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int k = lane + 32 * q;
        if (k <= s) x[k] = csub(xs[q], cmul(v[q], f));
    }
    __syncwarp();
}

// bounded wait until flag == epoch (another block publishes it)
__device__ __forceinline__ bool wait_flag(const int *flag, int epoch) {
    pipe::WaitClock clk;
    for (unsigned n = 0;; ++n) {
        if (*(volatile const int *)flag == epoch) {
            __threadfence();
            return true;
        }
        if ((n & 15) == 15 && (clk.over(kLsWaitNs) || n > (1u << 28))) return false;
        __nanosleep(64);
    }
}

// all lanes: lane 0 waits, the result is broadcast
__device__ __forceinline__ bool warp_wait_flag(const int *flag, int epoch) {
    int ok = 1;
    if (threadIdx.x == 0) ok = wait_flag(flag, epoch) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// QR update of the block Hessenberg after block step j, one warp-sized block
// per new column q = j s + c (s co-resident blocks, cooperative launch): the
// column takes every earlier reflector (earlier blocks: stored, loaded a few
// ahead; this block: as the blocks of the earlier columns publish them), then
// yields its own reflector (Householder, v[0] = 1, real tau, so that
// H x = beta e1 with conj(alpha) beta real) and its column of the triangular
// factor. Then block c applies this block's s reflectors to source c's
// least-squares right-hand side, whose rows (j+1) s .. (j+2) s - 1 give the
// source's residual estimate. The last block to finish decides whether the
// cycle stops.
struct LsArgs {
    double2 *Hb;        // (m+1) s x m s, column-major, ldh
    size_t ldh;
    double2 *Vh;        // reflectors [q][s + 1]
    double *tau;        // [q]
    double2 *g;         // right-hand sides, column-major, ldh
    int *pub;           // [q] = epoch once reflector q is stored
    unsigned *ticket;   // zero at rest
    const double *fnorm;  // [s]
    double *est;        // [s] residual estimates
    int *stop;          // device flag: 1 = the cycle stops after this step
    int *bad;           // device flag: a wait ran out or a value is not finite
    int *host_flag;     // host-mapped copy of !stop (nullable)
    int j, s, m, epoch, last_step;
    double tol;
};

__global__ void __launch_bounds__(kLsThreads) k_bls(LsArgs a) {
    extern __shared__ double2 ls_raw[];
    double2 *col = ls_raw;                 // rows 0 .. (j+2) s - 1 of the column / right-hand side
    const int lane = threadIdx.x, c = blockIdx.x, s = a.s;
    const int q = a.j * s + c, rows = (a.j + 2) * s;
    double2 *hcol = a.Hb + (size_t)q * a.ldh;
    for (int i = lane; i < rows; i += kLsThreads) col[i] = hcol[i];
    __syncwarp();
    bool ok = true;
    // reflectors of the earlier blocks, kLsDepth loads in flight
    const int nprev = a.j * s;
    {
        double2 vr[kLsDepth][3];
        double tr[kLsDepth];
#pragma unroll
        for (int d = 0; d < kLsDepth; ++d) {
            if (d < nprev) {
                load_refl(a.Vh + (size_t)d * (s + 1), s, false, vr[d]);
                tr[d] = __ldg(a.tau + d);
            }
        }
        for (int q0 = 0; q0 < nprev; q0 += kLsDepth) {
#pragma unroll
            for (int d = 0; d < kLsDepth; ++d) {
                const int qq = q0 + d;
                if (qq < nprev) {
                    warp_refl(vr[d], tr[d], col + qq, s);
                    const int qn = qq + kLsDepth;
                    if (qn < nprev) {
                        load_refl(a.Vh + (size_t)qn * (s + 1), s, false, vr[d]);
                        tr[d] = __ldg(a.tau + qn);
                    }
                }
            }
        }
    }
    // reflectors of this block, as they are published
    for (int cc = 0; cc < c && ok; ++cc) {
        const int qq = a.j * s + cc;
        ok = warp_wait_flag(a.pub + qq, a.epoch);
        if (!ok) break;
        double2 vr[3];
        load_refl(a.Vh + (size_t)qq * (s + 1), s, true, vr);
        warp_refl(vr, __ldcg(a.tau + qq), col + qq, s);
    }
    // own reflector from rows q .. q + s
    {
        const double2 alpha = col[q];
        double2 xs[3];
        double sg = 0.0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int k = lane + 32 * r;
            xs[r] = (k >= 1 && k <= s) ? col[q + k] : make_double2(0.0, 0.0);
            sg += xs[r].x * xs[r].x + xs[r].y * xs[r].y;
        }
        for (int o = 16; o; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
        const double aa = hypot(alpha.x, alpha.y);
        double2 beta = alpha, v0 = make_double2(1.0, 0.0);
        double t = 0.0;
        if (sg > 0.0) {
            const double nrm = sqrt(aa * aa + sg);
            const double2 ph = aa > 0.0 ? cscal(1.0 / aa, alpha) : make_double2(1.0, 0.0);
            beta = cscal(-nrm, ph);
            v0 = csub(alpha, beta);          // = ph (aa + nrm)
        }
        double vv = 0.0;
        double2 vk[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            vk[r] = sg > 0.0 ? cdiv(xs[r], v0) : make_double2(0.0, 0.0);
            vv += vk[r].x * vk[r].x + vk[r].y * vk[r].y;
        }
        for (int o = 16; o; o >>= 1) vv += __shfl_xor_sync(0xffffffffu, vv, o);
        if (sg > 0.0) t = 2.0 / (1.0 + vv);
        if (!(isfinite(beta.x) && isfinite(beta.y) && isfinite(t))) ok = false;
        double2 *v = a.Vh + (size_t)q * (s + 1);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int k = lane + 32 * r;
            if (k == 0) v[0] = make_double2(1.0, 0.0);
            else if (k <= s) v[k] = vk[r];
        }
        if (lane == 0) {
            a.tau[q] = t;
            col[q] = beta;
        }
        __syncwarp();
        // the column of the triangular factor: rows 0 .. q
        for (int i = lane; i < rows; i += kLsThreads) hcol[i] = i <= q ? col[i] : make_double2(0.0, 0.0);
        __threadfence();
        __syncwarp();
        if (lane == 0) *(volatile int *)(a.pub + q) = a.epoch;
    }
    // source c: this block's reflectors on its right-hand side
    double2 *gcol = a.g + (size_t)c * a.ldh;
    for (int i = lane; i < rows; i += kLsThreads) col[i] = gcol[i];
    __syncwarp();
    for (int cc = 0; cc < s && ok; ++cc) {
        const int qq = a.j * s + cc;
        if (cc != c) ok = warp_wait_flag(a.pub + qq, a.epoch);
        if (!ok) break;
        double2 vr[3];
        load_refl(a.Vh + (size_t)qq * (s + 1), s, true, vr);
        warp_refl(vr, __ldcg(a.tau + qq), col + qq, s);
    }
    for (int i = lane; i < rows; i += kLsThreads) gcol[i] = col[i];
    double e = 0.0;
    for (int i = (a.j + 1) * s + lane; i < rows; i += kLsThreads) e += col[i].x * col[i].x + col[i].y * col[i].y;
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) {
        e = sqrt(e);
        if (!ok || !isfinite(e)) {
            e = qnan();
            atomicOr(a.bad, 1);
        }
        a.est[c] = e;
        __threadfence();
        const unsigned tk = atomicAdd(a.ticket, 1u);
        if (tk == (unsigned)s - 1) {
            __threadfence();
            int done = 1;
            for (int k = 0; k < s; ++k) {
                const double ek = *(volatile double *)(a.est + k);
                if (a.fnorm[k] > 0.0 && !(ek <= a.tol * a.fnorm[k])) done = 0;
            }
            if (*(volatile int *)a.bad) done = 1;
            if (a.last_step) done = 1;
            *a.stop = done;
            if (a.host_flag) *(volatile int *)a.host_flag = !done;
            *a.ticket = 0;
        }
    }
}

// y[:, c] = R^-1 g[:, c] over the first K rows (R: the triangular factor in
// Hb, column-major); a zero diagonal (a direction the basis lost) gives 0.
// Y is written row-major [i][c] (ldy = s) as the combine's coefficients.
__global__ void __launch_bounds__(256) k_bbacksolve(const double2 *__restrict__ Hb, size_t ldh,
                                                    const double2 *__restrict__ g, int K, int s,
                                                    double2 *__restrict__ Y) {
    extern __shared__ double2 bs_raw[];
    double2 *y = bs_raw;
    const int c = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < K; i += blockDim.x) y[i] = g[(size_t)c * ldh + i];
    __syncthreads();
    __shared__ double2 yr_sh;
    for (int r = K - 1; r >= 0; --r) {
        if (tid == 0) {
            const double2 d = Hb[(size_t)r * ldh + r];
            const double2 yr = (d.x != 0.0 || d.y != 0.0) ? cdiv(y[r], d) : make_double2(0.0, 0.0);
            y[r] = yr;
            yr_sh = yr;
        }
        __syncthreads();
        const double2 yr = yr_sh;
        const double2 *hc = Hb + (size_t)r * ldh;
        for (int i = tid; i < r; i += blockDim.x) y[i] = csub(y[i], cmul(hc[i], yr));
        __syncthreads();
    }
    for (int i = tid; i < K; i += blockDim.x) Y[(size_t)i * s + c] = y[i];
}

// u[c * N + p] += t[c * Np + p] (complex64 widened exactly), c < s
__global__ void k_badd(const float2 *__restrict__ t, size_t Np, double2 *__restrict__ u, size_t N, int s) {
    const int c = blockIdx.y;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        const double2 d = cvt<double2>(t[(size_t)c * Np + p]);
        double2 x = u[(size_t)c * N + p];
        x.x += d.x;
        x.y += d.y;
        u[(size_t)c * N + p] = x;
    }
}

void set_attrs() {
    static const int once = [] {
        cudaFuncSetAttribute(k_bgram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcStages));
        cudaFuncSetAttribute(k_bcomb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcStages));
        cudaFuncSetAttribute(k_bchol, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * kBS * kBS * sizeof(float2)));
        cudaFuncSetAttribute(k_bls, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kMaxRows * sizeof(double2)));
        cudaFuncSetAttribute(k_bbacksolve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kMaxRows * sizeof(double2)));
        return 1;
    }();
    (void)once;
}

// node-range chunking of the Gram: about one CTA per SM over all row groups
void gram_geometry(int nv, size_t Np, int *nkc, int *chunk, int *ngroups) {
    const int ng = (nv + kTiles * kTM - 1) / (kTiles * kTM);
    int kcs = std::max(1, device_sms() / ng);
    size_t ch = (Np + kcs - 1) / kcs;
    ch = (ch + kGramNodes - 1) / kGramNodes * kGramNodes;
    kcs = (int)((Np + ch - 1) / ch);
    *nkc = kcs;
    *chunk = (int)ch;
    *ngroups = ng;
}

}  // namespace

size_t block_gram_part_floats(int nv_max, size_t Np) {
    size_t best = 0;
    for (int nv = 1; nv <= nv_max; ++nv) {
        int nkc, chunk, ng;
        gram_geometry(nv, Np, &nkc, &chunk, &ng);
        best = std::max(best, (size_t)nkc * nv * 128);
    }
    return best;
}

// G = V^H W (nv rows) in complex128: G row-major [i][c] (ldg), and added into
// the block Hessenberg column (hacc, column-major ldh) when hacc is non-null
void launch_bgram(const float2 *V, size_t sv, int nv, const float2 *W, size_t sw, int s, size_t Np,
                  float *part, double2 *G, int ldg, double2 *hacc, size_t ldh, int add, cudaStream_t st) {
    set_attrs();
    int nkc, chunk, ng;
    gram_geometry(nv, Np, &nkc, &chunk, &ng);
    prof_begin(st);
    k_bgram<<<dim3(nkc, ng), kBT, sizeof(TcStages), st>>>(V, sv, nv, W, sw, s, Np, chunk, part);
    count_launch();
    if (prof_on())
        prof_end("block_gram_tc", st, ((double)nv + s) * Np * 8.0 + (double)nkc * nv * 512.0, 0.0);
    prof_begin(st);
    k_bgram_sum<<<nv, kBS, 0, st>>>(part, nkc, nv, s, G, ldg, hacc, ldh, add);
    count_launch();
    prof_end("block_gram_sum", st, (double)nkc * nv * 512.0, 0.0);
}

// out = alpha win + V (sign C), C: nv x s complex128 row-major (ldc)
void launch_bcomb(const float2 *V, size_t sv, int nv, const double2 *C, int ldc, double sign, float *img,
                  const float2 *win, size_t sw, float alpha, float2 *out, size_t so, int s, size_t N,
                  size_t Np, cudaStream_t st) {
    set_attrs();
    const int nch = (nv + kCombVecs - 1) / kCombVecs;
    k_bcomb_image<<<nch, 256, 0, st>>>(C, ldc, nv, s, sign, img);
    count_launch();
    const int blocks = (int)((N + kCombNodes - 1) / kCombNodes);
    prof_begin(st);
    k_bcomb<<<blocks, kBT, sizeof(TcStages), st>>>(V, sv, nv, img, win, sw, alpha, out, so, s, N, Np);
    count_launch();
    if (prof_on())
        prof_end("block_combine_tc", st, ((double)nv + (alpha != 0.f ? 2.0 : 1.0) * s) * N * 8.0, 0.0);
}

size_t block_image_floats(int nv_max) { return (size_t)((nv_max + kCombVecs - 1) / kCombVecs) * 2 * kPlane; }


// ------------------------------------------------------------------ solver
namespace {

helm_status ensure_block_ws(helm_grid *g) {
    const int m = g->opt.restart;
    if (g->bcap_m == m) return HELM_OK;
    const size_t N = g->N, Np = (N + 7) / 8 * 8;
    const size_t S = kBS, nv_max = (size_t)m * kBS, ldh = (size_t)(m + 1) * kBS;
    helm_status s;
    if ((s = g->bV.ensure((size_t)(m + 1) * S * Np * sizeof(float2))) ||
        (s = g->bZ.ensure((size_t)m * S * Np * sizeof(float2))) || (s = g->bW.ensure(S * Np * sizeof(float2))) ||
        (s = g->bpart.ensure(block_gram_part_floats((int)nv_max, Np) * sizeof(float))) ||
        (s = g->bimg.ensure(block_image_floats((int)nv_max) * sizeof(float))) ||
        (s = g->bG.ensure(nv_max * S * sizeof(double2))) || (s = g->bR.ensure(S * S * sizeof(double2))) ||
        (s = g->bRinv.ensure(S * S * sizeof(double2))) || (s = g->bHb.ensure(ldh * nv_max * sizeof(double2))) ||
        (s = g->bg.ensure(ldh * S * sizeof(double2))) || (s = g->bVh.ensure(nv_max * (S + 1) * sizeof(double2))) ||
        (s = g->btau.ensure(nv_max * sizeof(double))) || (s = g->bpub.ensure(nv_max * sizeof(int))) ||
        (s = g->bticket.ensure(64)) || (s = g->best.ensure(S * sizeof(double))) || (s = g->bflags.ensure(64)) ||
        (s = g->bY.ensure(nv_max * S * sizeof(double2))) || (s = g->bfn.ensure(S * sizeof(double))) ||
        (s = g->bnp.ensure(S * kMaxBlocks * sizeof(double))) || (s = g->bncnt.ensure(S * sizeof(unsigned))) ||
        (s = g->bnrm.ensure(S * sizeof(double))) || (s = g->rbuf.ensure(S * N * sizeof(double2))))
        return s;
    // zero padding between N and Np must stay zero: it is read, never written
    cudaMemsetAsync(g->bV.p, 0, g->bV.bytes, g->st);
    cudaMemsetAsync(g->bZ.p, 0, g->bZ.bytes, g->st);
    cudaMemsetAsync(g->bW.p, 0, g->bW.bytes, g->st);
    cudaMemsetAsync(g->bpub.p, 0, g->bpub.bytes, g->st);
    cudaMemsetAsync(g->bticket.p, 0, 64, g->st);
    cudaMemsetAsync(g->bncnt.p, 0, g->bncnt.bytes, g->st);
    g->bls_epoch = 0;
    if (!g->bhflag) {
        if (cudaHostAlloc((void **)&g->bhflag, 64, cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            g->bhflag = nullptr;
            return fail(HELM_ERR_NOMEM, "host-mapped flag");
        }
    }
    g->bcap_m = m;
    return HELM_OK;
}

// W (s vectors, stride Np) = out R with out orthonormal (two Cholesky QR
// passes, the first shifted); the accumulated R (row-major s x s) in g->bR
void block_cholqr(helm_grid *g, float2 *W, float2 *out, int s, size_t Np) {
    cudaStream_t st = g->st;
    const size_t N = g->N;
    for (int pass = 0; pass < 2; ++pass) {
        launch_bgram(W, Np, s, W, Np, s, Np, g->bpart.as<float>(), g->bG.as<double2>(), s, nullptr, 0, 0, st);
        prof_begin(st);
        k_bchol<<<1, kCh, 2 * kBS * kBS * sizeof(float2), st>>>(g->bG.as<double2>(), s, pass == 0 ? 1e-5 : 0.0,
                                                                 g->bRinv.as<double2>(), g->bR.as<double2>(),
                                                                 pass == 0);
        count_launch();
        prof_end("block_cholesky", st, 0.0, 0.0);
        launch_bcomb(W, Np, s, g->bRinv.as<double2>(), s, 1.0, g->bimg.as<float>(), W, Np, 0.f,
                     pass == 0 ? W : out, Np, s, N, Np, st);
    }
}

helm_status block_norms(helm_grid *g, const double2 *x, int s, std::vector<double> &out) {
    KrylovScratch ks;
    ks.partial = g->bnp.as<double2>();
    ks.counter = g->bncnt.as<unsigned>();
    ks.max_blocks = kMaxBlocks;
    ks.nvec_max = 1;
    launch_norm2(x, g->N, g->N, g->bnrm.as<double>(), s, nullptr, ks, g->st);
    out.resize(s);
    cudaMemcpyAsync(out.data(), g->bnrm.p, s * sizeof(double), cudaMemcpyDeviceToHost, g->st);
    return sync_stream(g, "block norms");
}

// One block of s <= 64 sources: f, u (device, stride N).
helm_status solve_block_group(helm_grid *g, int s, const double2 *f, double tol, double2 *u, int *its_out,
                              double *rel_out, bool warm) {
    cudaStream_t st = g->st;
    const size_t N = g->N, Np = (N + 7) / 8 * 8;
    const int m = g->opt.restart;
    const size_t ldh = (size_t)(m + 1) * kBS;
    const LevelView<double> L0 = level_view<double>(g, 0);
    float2 *V = g->bV.as<float2>(), *Z = g->bZ.as<float2>(), *W = g->bW.as<float2>();
    double2 *Hb = g->bHb.as<double2>(), *gl = g->bg.as<double2>();
    double2 *rb = g->rbuf.as<double2>();
    int *dflags = g->bflags.as<int>();
    helm_status s_;
    // ||f|| per source
    std::vector<double> fn2;
    if ((s_ = block_norms(g, f, s, fn2))) return s_;
    std::vector<double> fn(s);
    for (int c = 0; c < s; ++c) fn[c] = std::sqrt(fn2[c]);
    cudaMemcpyAsync(g->bfn.p, fn.data(), s * sizeof(double), cudaMemcpyHostToDevice, st);
    if (!warm) cudaMemsetAsync(u, 0, (size_t)s * N * sizeof(double2), st);
    cudaMemsetAsync(dflags, 0, 64, st);
    int steps = 0;
    std::vector<double> rel(s, 0.0), r2;
    bool converged = false, broke = false;
    while (true) {
        // true residual R = F - H U (complex128) and its norms
        launch_stencil<double, double2, double2>(ST_RESID, L0, shift_H(g), u, N, f, N, rb, N, s, 0.0, nullptr, st);
        if ((s_ = block_norms(g, rb, s, r2))) return s_;
        bool all = true;
        for (int c = 0; c < s; ++c) {
            rel[c] = fn[c] > 0.0 ? std::sqrt(r2[c]) / fn[c] : 0.0;
            if (!std::isfinite(rel[c])) broke = true;
            if (fn[c] > 0.0 && !(rel[c] <= tol)) all = false;
        }
        if (all || broke || steps >= g->opt.max_iters) {
            converged = all && !broke;
            break;
        }
        // V_0 B = R
        launch_convert<double2, float2>(rb, N, W, Np, N, s, st);
        block_cholqr(g, W, V, s, Np);
        k_brhs_init<<<s, 256, 0, st>>>(g->bR.as<double2>(), s, gl, ldh, (int)ldh);
        count_launch();
        int k = 0;
        for (int j = 0; j < m; ++j) {
            const int nv = (j + 1) * s;
            float2 *Vj = V + (size_t)j * s * Np, *Zj = Z + (size_t)j * s * Np;
            vcycle<float, float2>(g, Vj, Np, Zj, Np, s, nullptr);
            launch_stencil<double, float2, float2>(ST_APPLY, L0, shift_H(g), Zj, Np, (const float2 *)nullptr, 0, W,
                                                   Np, s, 0.0, nullptr, st);
            double2 *hcol = Hb + (size_t)j * s * ldh;
            // block classical Gram-Schmidt twice (one pass loses orthogonality
            // in the complex64 basis: about 1.7x the block steps, measured)
            const int passes = 2;
            for (int pass = 0; pass < passes; ++pass) {
                launch_bgram(V, Np, nv, W, Np, s, Np, g->bpart.as<float>(), g->bG.as<double2>(), s, hcol, ldh,
                             pass, st);
                launch_bcomb(V, Np, nv, g->bG.as<double2>(), s, -1.0, g->bimg.as<float>(), W, Np, 1.f, W, Np, s, N,
                             Np, st);
            }
            block_cholqr(g, W, V + (size_t)(j + 1) * s * Np, s, Np);
            k_bput_r<<<1, 256, 0, st>>>(g->bR.as<double2>(), s, Hb, ldh, (j + 1) * s, j * s);
            count_launch();
            // least-squares update (co-resident blocks, one per new column)
            LsArgs a;
            a.Hb = Hb;
            a.ldh = ldh;
            a.Vh = g->bVh.as<double2>();
            a.tau = g->btau.as<double>();
            a.g = gl;
            a.pub = g->bpub.as<int>();
            a.ticket = g->bticket.as<unsigned>();
            a.fnorm = g->bfn.as<double>();
            a.est = g->best.as<double>();
            a.stop = dflags;
            a.bad = dflags + 1;
            a.host_flag = g->bhflag;
            a.j = j;
            a.s = s;
            a.m = m;
            a.epoch = ++g->bls_epoch;
            a.last_step = (j + 1 == m || steps + 1 >= g->opt.max_iters) ? 1 : 0;
            a.tol = tol;
            *(volatile int *)g->bhflag = 1;
            void *args[] = {&a};
            prof_begin(st);
            cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_bls, dim3(s), dim3(kLsThreads), args,
                                                        (size_t)(j + 2) * s * sizeof(double2), st);
            if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "least-squares update: %s", cudaGetErrorString(e));
            count_launch();
            prof_end("block_least_squares", st, 0.0, 0.0);
            ++steps;
            k = j + 1;
            if ((s_ = sync_stream(g, "block step"))) return s_;
            if (!*(volatile int *)g->bhflag) break;
        }
        // u += Z Y, Y = R^-1 g over the k block steps of the cycle
        const int K = k * s;
        prof_begin(st);
        k_bbacksolve<<<s, 256, (size_t)K * sizeof(double2), st>>>(Hb, ldh, gl, K, s, g->bY.as<double2>());
        count_launch();
        prof_end("block_backsolve", st, 0.0, 0.0);
        launch_bcomb(Z, Np, K, g->bY.as<double2>(), s, 1.0, g->bimg.as<float>(), W, Np, 0.f, W, Np, s, N, Np, st);
        k_badd<<<dim3((unsigned)std::min<size_t>((N + 255) / 256, 4096), s), 256, 0, st>>>(W, Np, u, N, s);
        count_launch();
        int hb[2] = {0, 0};
        cudaMemcpyAsync(hb, dflags, sizeof hb, cudaMemcpyDeviceToHost, st);
        if ((s_ = sync_stream(g, "block cycle end"))) return s_;
        if (hb[1]) broke = true;
    }
    for (int c = 0; c < s; ++c) {
        if (its_out) its_out[c] = fn[c] > 0.0 ? steps : 0;
        if (rel_out) rel_out[c] = rel[c];
    }
    if (broke) return fail(HELM_ERR_BREAKDOWN, "block Arnoldi produced a non-finite value");
    if (!converged) return fail(HELM_ERR_NOT_CONVERGED, "not converged within %d block steps", g->opt.max_iters);
    return HELM_OK;
}

}  // namespace

helm_status solve_block_device(helm_grid *g, int nrhs, const double2 *f, double tol, double2 *u,
                               int *iterations, double *relres_out, bool warm) {
    helm_status s;
    if ((s = ensure_ready(g))) return s;
    if ((s = ensure_block_ws(g)) || (s = ensure_level_work(g, kBS))) return s;
    int flag = 0;
    int *dflag = g->flag.as<int>();
    cudaMemsetAsync(dflag, 0, sizeof(int), g->st);
    launch_finite_check((const double *)f, 2 * g->N * (size_t)nrhs, dflag, g->st);
    if (warm) launch_finite_check((const double *)u, 2 * g->N * (size_t)nrhs, dflag, g->st);
    cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, g->st);
    if ((s = sync_stream(g, "block solve start"))) return s;
    if (flag) return fail(HELM_ERR_NONFINITE, "right-hand side or initial guess contains NaN or Inf");
    helm_status worst = HELM_OK;
    for (int k0 = 0; k0 < nrhs; k0 += kBS) {
        const int sb = std::min(kBS, nrhs - k0);
        s = solve_block_group(g, sb, f + (size_t)k0 * g->N, tol, u + (size_t)k0 * g->N,
                              iterations ? iterations + k0 : nullptr, relres_out ? relres_out + k0 : nullptr, warm);
        if (s != HELM_OK && s != HELM_ERR_NOT_CONVERGED && s != HELM_ERR_BREAKDOWN) return s;
        if (s == HELM_ERR_BREAKDOWN || (s == HELM_ERR_NOT_CONVERGED && worst == HELM_OK)) worst = s;
    }
    if (worst == HELM_ERR_BREAKDOWN) return fail(worst, "block Arnoldi produced a non-finite value");
    if (worst == HELM_ERR_NOT_CONVERGED)
        return fail(worst, "not converged within %d block steps", g->opt.max_iters);
    return HELM_OK;
}

}  // namespace helm

using namespace helm;

namespace {
helm_status check_block_args(int nv, int s, size_t N, size_t ld) {
    if (nv < 1 || nv > 32 * 64 || s < 1 || s > 64) return fail(HELM_ERR_ARG, "need 1 <= nv <= 2048 and 1 <= s <= 64");
    if (N < 1 || ld < N || ld % 8) return fail(HELM_ERR_ARG, "ld must be >= N and a multiple of 8");
    return HELM_OK;
}
}  // namespace

extern "C" helm_status helm_block_gram(int nv, int s, size_t N, size_t ld, const void *V, const void *W,
                                       helm_c128 *G) {
    clear_error();
    helm_status st;
    if (!V || !W || !G) return fail(HELM_ERR_ARG, "null argument");
    if ((st = check_block_args(nv, s, N, ld))) return st;
    if (!is_device_ptr(V) || !is_device_ptr(W)) return fail(HELM_ERR_ARG, "V and W must be device pointers");
    DevBuf part, gd;
    if ((st = part.ensure(block_gram_part_floats(nv, ld) * sizeof(float))) ||
        (st = gd.ensure((size_t)nv * s * sizeof(double2))))
        return st;
    launch_bgram((const float2 *)V, ld, nv, (const float2 *)W, ld, s, ld, part.as<float>(), gd.as<double2>(), s,
                 nullptr, 0, 0, 0);
    cudaError_t e = cudaMemcpy(G, gd.p, (size_t)nv * s * sizeof(double2), cudaMemcpyDefault);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "helm_block_gram: %s", cudaGetErrorString(e));
    return check_cuda("helm_block_gram");
}

extern "C" helm_status helm_block_combine(int nv, int s, size_t N, size_t ld, const void *V, const helm_c128 *C,
                                          float alpha, void *W) {
    clear_error();
    helm_status st;
    if (!V || !C || !W) return fail(HELM_ERR_ARG, "null argument");
    if ((st = check_block_args(nv, s, N, ld))) return st;
    if (!is_device_ptr(V) || !is_device_ptr(W)) return fail(HELM_ERR_ARG, "V and W must be device pointers");
    DevBuf img, cd;
    if ((st = img.ensure(block_image_floats(nv) * sizeof(float))) || (st = cd.ensure((size_t)nv * s * sizeof(double2))))
        return st;
    cudaError_t e = cudaMemcpy(cd.p, C, (size_t)nv * s * sizeof(double2), cudaMemcpyDefault);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "helm_block_combine: %s", cudaGetErrorString(e));
    launch_bcomb((const float2 *)V, ld, nv, cd.as<double2>(), s, 1.0, img.as<float>(), (const float2 *)W, ld, alpha,
                 (float2 *)W, ld, s, N, ld, 0);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "helm_block_combine: %s", cudaGetErrorString(e));
    return check_cuda("helm_block_combine");
}
