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

constexpr int kBX = 128;

struct dsf {
    float h, l;
};

__device__ __forceinline__ dsf ds_add_f(dsf a, float b) {      // unnormalised
    const float s = a.h + b;
    const float bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b - bb);
    return {s, a.l + e};
}
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

template <int DIM, typename CIn>
__device__ __forceinline__ void nbr_terms(const CIn *__restrict__ z, size_t p, int i, int n,
                                          size_t stride, dsf &sr, dsf &si) {
    if (i > 0) {
        const float2 v = cvt<float2>(z[p - stride]);
        const float c = (i == n - 1) ? 2.f : 1.f;
        sr = ds_add_f(sr, c * v.x);
        si = ds_add_f(si, c * v.y);
    }
    if (i < n - 1) {
        const float2 v = cvt<float2>(z[p + stride]);
        const float c = (i == 0) ? 2.f : 1.f;
        sr = ds_add_f(sr, c * v.x);
        si = ds_add_f(si, c * v.y);
    }
}

template <int DIM>
__global__ void __launch_bounds__(kBX)
k_apply_H_ds(LevelView<double> L, const float4 *__restrict__ hd, float ihh, float ihl,
             const float2 *__restrict__ z, size_t sz, float4 *__restrict__ w, size_t sw,
             const int *__restrict__ active) {
    const int r = blockIdx.z;
    if (active && !active[r]) return;
    z += r * sz;
    w += r * sw;
    const int nx = L.nx;
    const int rows = L.ny * L.nz;
    const int ix = blockIdx.x * kBX + threadIdx.x;
    if (ix >= nx) return;
    const dsf ih = {ihh, ihl};
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const size_t p = (size_t)row * nx + ix;
        dsf sr = {0.f, 0.f}, si = {0.f, 0.f};
        nbr_terms<DIM>(z, p, ix, nx, 1, sr, si);
        if (DIM >= 2) nbr_terms<DIM>(z, p, (DIM == 3) ? row % L.ny : row, L.ny, (size_t)nx, sr, si);
        if (DIM == 3) nbr_terms<DIM>(z, p, row / L.ny, L.nz, (size_t)nx * L.ny, sr, si);
        sr = ds_norm(sr);
        si = ds_norm(si);
        const float4 d = hd[p];
        const float2 zp = z[p];
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
    const dim3 g((L.nx + kBX - 1) / kBX, rows < 65535 ? rows : 65535, nb);
    prof_begin(st);
    if (L.dim == 1) k_apply_H_ds<1><<<g, kBX, 0, st>>>(L, hd, ihh, ihl, z, sz, w, sw, active);
    else if (L.dim == 2) k_apply_H_ds<2><<<g, kBX, 0, st>>>(L, hd, ihh, ihl, z, sz, w, sw, active);
    else k_apply_H_ds<3><<<g, kBX, 0, st>>>(L, hd, ihh, ihl, z, sz, w, sw, active);
    count_launch();
    if (prof_on()) {
        // per right-hand side: z in, w out; the diagonal once per launch
        const double n1 = (double)L.nx * L.ny * L.nz, n = n1 * nb;
        prof_end("stencil_apply_ds", st, n * (8.0 + 16.0) + n1 * 16.0, 0.0);
    }
}

}  // namespace helm
