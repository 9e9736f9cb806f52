// w = H z in double-single arithmetic, for the double-single Arnoldi basis
// (precision HELM_PREC_MIXED_DS).
//
// z comes from the complex64 V-cycle and is exact in FP32; the neighbour sum
// of the 5/7-point stencil is accumulated with two-sums (no rounding loss),
// the diagonal d_p of H (Eq. 2-3: 2 dim/h^2 - omega^2 m^2 (1 - j alpha) plus
// the absorbing boundary term) is precomputed once per model as a double-
// single pair, and d_p z_p - (1/h^2) sum is formed with error-free products.
// The result (about 48 significant bits) is written straight into the
// double-single basis slot. Roughly 120 FP32 instructions per node replace
// about 14 FP64 ones, so the kernel is bound by memory instead of the FP64
// pipe.
#include "helm_internal.cuh"

namespace helm {

namespace {

struct dsf {
    float h, l;
};

__device__ __forceinline__ dsf ds_norm(dsf a) {
    const float s = a.h + a.l;
    return {s, a.l - (s - a.h)};
}
__device__ __forceinline__ dsf ds_mul_f(dsf a, float b) {      // unnormalised
    const float p = a.h * b;
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    return {p, e};
}
__device__ __forceinline__ dsf ds_mul(dsf a, dsf b) {          // unnormalised
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return {p, e};
}
__device__ __forceinline__ dsf ds_add(dsf a, dsf b) {
    const float s = a.h + b.h;
    const float bb = s - a.h;
    float e = (a.h - (s - bb)) + (b.h - bb);
    e += a.l + b.l;
    return ds_norm({s, e});
}

template <typename T> __device__ __forceinline__ T dsqrt(T v);
template <> __device__ __forceinline__ double dsqrt<double>(double v) { return sqrt(v); }

__global__ void k_make_hdiag_ds(LevelView<double> L, OpShift<double> s, float4 *__restrict__ hd) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(p % L.nx);
        const int iy = (int)((p / L.nx) % L.ny);
        const int iz = (int)(p / ((size_t)L.nx * L.ny));
        int nf = (ix == 0) + (ix == L.nx - 1);
        if (L.dim >= 2) nf += (iy == 0) + (iy == L.ny - 1);
        if (L.dim == 3) nf += (iz == 0) + (iz == L.nz - 1);
        const double wp = L.w[p];
        double dre = 2.0 * L.dim * L.inv_h2 - s.s_re * wp;
        double dim_ = -s.s_im * wp;
        if (nf) {
            const double f = nf * L.two_over_h * dsqrt<double>(wp);
            dre -= f * s.q_im;
            dim_ += f * s.q_re;
        }
        hd[p] = cvt<float4>(make_double2(dre, dim_));
    }
}

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ dsf two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
// (s.h, s.l) + (t.h, t.l) for two exact pair sums; renormalised
__device__ __forceinline__ dsf add_pairs(dsf s, dsf t) {
    const dsf u = two_sum(s.h, t.h);
    return ds_norm({u.h, (s.l + t.l) + u.l});
}

// Neighbour of node p along one axis, scaled by the boundary factor: the
// mirrored ghost of the absorbing boundary doubles the inner neighbour at
// the first and last node, and the missing outer neighbour contributes 0.
__device__ __forceinline__ float2 nbr(const float2 *__restrict__ z, size_t q, bool exists, bool twice) {
    if (!exists) return make_float2(0.f, 0.f);
    const float2 v = z[q];
    return twice ? make_float2(2.f * v.x, 2.f * v.y) : v;
}

// One block covers (part of) a row of the grid with one node per thread; the
// grid's y dimension strides over rows (y, z), its z dimension over
// right-hand sides.
template <int DIM>
__global__ void __launch_bounds__(512)
k_apply_H_ds(LevelView<double> L, const float4 *__restrict__ hd, float ihh, float ihl,
             const float2 *__restrict__ z, size_t sz, float4 *__restrict__ w, size_t sw,
             const int *__restrict__ active) {
    const int r = blockIdx.z;
    if (active && !active[r]) return;
    z += r * sz;
    w += r * sw;
    const int nx = L.nx, ny = L.ny;
    const int rows = L.ny * L.nz;
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    if (ix >= nx) return;
    const dsf ih = {ihh, ihl};
    const bool xw = ix > 0, xe = ix < nx - 1;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const size_t p = (size_t)row * nx + ix;
        const float2 zp = z[p];
        // neighbour sums, exact as unevaluated pairs: x pair + y pair (+ z pair)
        dsf sr, si;
        {
            const float2 a = nbr(z, p - 1, xw, !xe), b = nbr(z, p + 1, xe, !xw);
            sr = two_sum(a.x, b.x);
            si = two_sum(a.y, b.y);
        }
        if (DIM >= 2) {
            const int iy = DIM == 3 ? row % ny : row;
            const bool ys = iy > 0, yn = iy < ny - 1;
            const float2 a = nbr(z, p - nx, ys, !yn), b = nbr(z, p + nx, yn, !ys);
            sr = add_pairs(sr, two_sum(a.x, b.x));
            si = add_pairs(si, two_sum(a.y, b.y));
        } else {
            sr = ds_norm(sr);
            si = ds_norm(si);
        }
        if (DIM == 3) {
            const int iz = row / ny;
            const size_t sl = (size_t)nx * ny;
            const bool zb = iz > 0, zf = iz < L.nz - 1;
            const float2 a = nbr(z, p - sl, zb, !zf), b = nbr(z, p + sl, zf, !zb);
            sr = add_pairs(sr, ds_norm(two_sum(a.x, b.x)));
            si = add_pairs(si, ds_norm(two_sum(a.y, b.y)));
        }
        const float4 d = hd[p];
        const dsf dre = {d.x, d.y}, dim_ = {d.z, d.w};
        // d z
        const dsf ar = ds_add(ds_mul_f(dre, zp.x), ds_mul_f(dim_, -zp.y));
        const dsf ai = ds_add(ds_mul_f(dre, zp.y), ds_mul_f(dim_, zp.x));
        // (1/h^2) sum
        const dsf br = ds_mul(ih, sr), bi = ds_mul(ih, si);
        const dsf wr = ds_add(ar, {-br.h, -br.l});
        const dsf wi = ds_add(ai, {-bi.h, -bi.l});
        w[p] = make_float4(wr.h, wr.l, wi.h, wi.l);
    }
}

}  // namespace

void launch_make_hdiag_ds(const LevelView<double> &L, OpShift<double> s, float4 *hd, cudaStream_t st) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    size_t b = (N + 255) / 256;
    const int nb = (int)(b < 4096 ? (b ? b : 1) : 4096);
    k_make_hdiag_ds<<<nb, 256, 0, st>>>(L, s, hd);
    count_launch();
}

void launch_apply_H_ds(const LevelView<double> &L, const float4 *hd, const float2 *z, size_t sz,
                       float4 *w, size_t sw, int nb, const int *active, cudaStream_t st) {
    const double ih = L.inv_h2;
    const float ihh = (float)ih;                    // nearest float; ih - ihh is exact in FP64
    const float ihl = (float)(ih - (double)ihh);
    const int rows = L.ny * L.nz;
    // blocks of whole warps spanning a row: 401 nodes -> 416 threads
    const int wpr = (L.nx + 31) / 32, bpr = (wpr + 15) / 16;
    const int bx = 32 * ((wpr + bpr - 1) / bpr);
    const dim3 g(bpr, rows < 65535 ? rows : 65535, nb);
    prof_begin(st);
    if (L.dim == 1) k_apply_H_ds<1><<<g, bx, 0, st>>>(L, hd, ihh, ihl, z, sz, w, sw, active);
    else if (L.dim == 2) k_apply_H_ds<2><<<g, bx, 0, st>>>(L, hd, ihh, ihl, z, sz, w, sw, active);
    else k_apply_H_ds<3><<<g, bx, 0, st>>>(L, hd, ihh, ihl, z, sz, w, sw, active);
    count_launch();
    if (prof_on()) {
        // per right-hand side: z in, w out; the diagonal once per launch
        const double n1 = (double)L.nx * L.ny * L.nz, n = n1 * nb;
        prof_end("stencil_apply_ds", st, n * (8.0 + 16.0) + n1 * 16.0, 0.0);
    }
}

}  // namespace helm
