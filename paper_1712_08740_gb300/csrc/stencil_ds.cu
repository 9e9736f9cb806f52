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

// Scaled neighbour values: the mirrored ghost of the absorbing boundary
// doubles the inner neighbour at the first and last node of an axis, and the
// missing outer neighbour contributes 0.
__device__ __forceinline__ float2 scaled(float2 v, bool exists, bool twice) {
    if (!exists) return make_float2(0.f, 0.f);
    return twice ? make_float2(2.f * v.x, 2.f * v.y) : v;
}

// w_p = d_p z_p - (1/h^2) sum_nbr, double-single; the neighbour sums are exact
// as unevaluated pairs: x pair + y pair (+ z pair)
template <int DIM>
__device__ __forceinline__ float4 node_out(float2 zp, float2 xa, float2 xb, float2 ya, float2 yb, float2 za,
                                           float2 zb, float4 d, dsf ih) {
    // cascade of two-sums over the neighbours (x-, x+, y-, y+, z-, z+): the
    // leading part is exact, the errors are added once at the end; the pair
    // is left unnormalised (the product with 1/h^2 below takes it as it is)
    dsf sr = two_sum(xa.x, xb.x), si = two_sum(xa.y, xb.y);
    if (DIM >= 2) {
        const dsf r2 = two_sum(sr.h, ya.x), i2 = two_sum(si.h, ya.y);
        const dsf r3 = two_sum(r2.h, yb.x), i3 = two_sum(i2.h, yb.y);
        float lr = (sr.l + r2.l) + r3.l, li = (si.l + i2.l) + i3.l;
        float hr = r3.h, hi = i3.h;
        if (DIM == 3) {
            const dsf r4 = two_sum(hr, za.x), i4 = two_sum(hi, za.y);
            const dsf r5 = two_sum(r4.h, zb.x), i5 = two_sum(i4.h, zb.y);
            lr = (lr + r4.l) + r5.l;
            li = (li + i4.l) + i5.l;
            hr = r5.h;
            hi = i5.h;
        }
        sr = {hr, lr};
        si = {hi, li};
    }
    const dsf dre = {d.x, d.y}, dim_ = {d.z, d.w};
    // w = (d z) - (1/h^2) sum as one three-term sum per part: the products
    // d_re z_re, -d_im z_im (error-free, unnormalised) and -(1/h^2) sum; the
    // leading parts are added with two two-sums, the rest folded in once
    const dsf pr1 = ds_mul_f(dre, zp.x), pr2 = ds_mul_f(dim_, -zp.y);
    const dsf pi1 = ds_mul_f(dre, zp.y), pi2 = ds_mul_f(dim_, zp.x);
    const dsf br = ds_mul(ih, sr), bi = ds_mul(ih, si);
    auto sum3 = [](dsf a, dsf b, dsf c) {
        const dsf s1 = two_sum(a.h, b.h);
        const dsf s2 = two_sum(s1.h, -c.h);
        return ds_norm({s2.h, ((a.l + b.l) - c.l) + (s1.l + s2.l)});
    };
    const dsf wr = sum3(pr1, pr2, br);
    const dsf wi = sum3(pi1, pi2, bi);
    return make_float4(wr.h, wr.l, wi.h, wi.l);
}

// One thread per pair of x-adjacent nodes (ix0, ix0 + 1) of a row: the pair
// shares its x-neighbour loads (four for two nodes) and index arithmetic.
// Blocks of whole warps span a row's pairs; the grid's y dimension strides
// over rows (y, z), its z dimension over right-hand sides. Indices are 32-bit
// (a right-hand side has fewer than 2^31 nodes).
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
    const int ix0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (ix0 >= nx) return;
    const int ix1 = ix0 + 1;
    const bool two = ix1 < nx;
    const dsf ih = {ihh, ihl};
    const float2 zero = make_float2(0.f, 0.f);
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const unsigned p = (unsigned)row * (unsigned)nx + (unsigned)ix0;
        // x: z[p-1], z[p], z[p+1], z[p+2]
        const float2 zl = ix0 > 0 ? z[p - 1] : zero;
        const float2 za_ = z[p];
        const float2 zb_ = two ? z[p + 1] : zero;
        const float2 zr = ix1 + 1 < nx ? z[p + 2] : zero;
        float2 ya0 = zero, yb0 = zero, ya1 = zero, yb1 = zero;
        if (DIM >= 2) {
            const int iy = DIM == 3 ? row % ny : row;
            const bool ys = iy > 0, yn = iy < ny - 1;
            if (ys) {
                ya0 = z[p - nx];
                if (two) ya1 = z[p + 1 - nx];
            }
            if (yn) {
                yb0 = z[p + nx];
                if (two) yb1 = z[p + 1 + nx];
            }
            ya0 = scaled(ya0, ys, !yn);
            yb0 = scaled(yb0, yn, !ys);
            ya1 = scaled(ya1, ys, !yn);
            yb1 = scaled(yb1, yn, !ys);
        }
        float2 za0 = zero, zb0 = zero, za1 = zero, zb1 = zero;
        if (DIM == 3) {
            const int iz = row / ny;
            const unsigned sl = (unsigned)nx * (unsigned)ny;
            const bool zbk = iz > 0, zfw = iz < L.nz - 1;
            if (zbk) {
                za0 = z[p - sl];
                if (two) za1 = z[p + 1 - sl];
            }
            if (zfw) {
                zb0 = z[p + sl];
                if (two) zb1 = z[p + 1 + sl];
            }
            za0 = scaled(za0, zbk, !zfw);
            zb0 = scaled(zb0, zfw, !zbk);
            za1 = scaled(za1, zbk, !zfw);
            zb1 = scaled(zb1, zfw, !zbk);
        }
        const float4 d0 = hd[p];
        const float4 d1 = two ? hd[p + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        // node ix0: left z[p-1], right z[p+1]
        w[p] = node_out<DIM>(za_, scaled(zl, ix0 > 0, ix0 == nx - 1), scaled(zb_, two, ix0 == 0), ya0, yb0,
                             za0, zb0, d0, ih);
        // node ix1: left z[p], right z[p+2]
        if (two)
            w[p + 1] = node_out<DIM>(zb_, scaled(za_, true, ix1 == nx - 1), scaled(zr, ix1 + 1 < nx, false),
                                     ya1, yb1, za1, zb1, d1, ih);
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
    // blocks of whole warps spanning a row's node pairs: 401 nodes -> 201 pairs -> 224 threads
    const int wpr = ((L.nx + 1) / 2 + 31) / 32, bpr = (wpr + 15) / 16;
    const int bx = 32 * ((wpr + bpr - 1) / bpr);
    // a block takes four rows (its y-stride loop); fewer, longer-lived blocks
    const int ry = (rows + 3) / 4;
    const dim3 g(bpr, ry < 65535 ? ry : 65535, nb);
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
