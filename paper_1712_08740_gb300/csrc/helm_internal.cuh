// Internal declarations shared by the libhelm translation units.
//
// Operators. On a level with spacing h and node coefficient w = omega^2 m^2
// (real, per node) the library applies
//     (A u)_p = d_p u_p - (1/h^2) sum_axes (c_lo u_lo + c_hi u_hi)
//     d_p     = 2 dim / h^2 - s w_p + nfaces_p (2/h) j kappa_p
//     kappa_p = sqrt(w_p) * q,   q = sqrt(1 - j alpha) (principal root)
// with neighbour weights c = 1 inside, c = 2 for the inward neighbour of a
// boundary node (centred ghost node of the absorbing condition) and c = 0
// for the missing outer neighbour. s = 1 - j alpha gives H (Eq. 2-3);
// s = beta1 - j beta2 gives the shifted Laplacian M (Eq. 6).
//
// Variable density (Eq. 1, -div(rho grad u) in place of -Lap u): each
// neighbour weight is multiplied by the face coefficient, the mean of rho at
// the node and at that neighbour (the inward weight of a boundary node stays
// doubled), the Laplacian part of d_p is the sum of those weights over h^2,
// and a boundary face adds (2/h) j (kappa_p / sqrt(rho_p)) times the face
// coefficient of the inner face instead of (2/h) j kappa_p.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <vector>

namespace helm {

// ------------------------------------------------------------ complex helpers
template <typename T> struct cplx;
template <> struct cplx<float>  { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im);
template <> __host__ __device__ __forceinline__ float2 mk<float2>(double re, double im) {
    return make_float2((float)re, (float)im);
}
template <> __host__ __device__ __forceinline__ double2 mk<double2>(double re, double im) {
    return make_double2(re, im);
}

// widen/narrow between complex types
template <typename To, typename From> __device__ __forceinline__ To cvt(From a) {
    return mk<To>((double)a.x, (double)a.y);
}
template <> __device__ __forceinline__ float2 cvt<float2, float2>(float2 a) { return a; }
template <> __device__ __forceinline__ double2 cvt<double2, double2>(double2 a) { return a; }
// Precision changes go through the integer pipe: GB300 runs F2F conversions
// at its (low) FP64 rate, while these bit manipulations use INT32 lanes.
// f2d_exact widens exactly (zero, normal, inf/NaN; denormals fall back to the
// hardware conversion). d2f_trunc narrows by truncating the mantissa (error
// below one float ulp), flushing |x| < 2^-126 to zero: it feeds the complex64
// preconditioner only, where rounding mode does not matter.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u) return (u & 0x7fffffu) ? (double)f : __hiloint2double((int)(u & 0x80000000u), 0);
    const unsigned hi = (u & 0x80000000u) | ((e == 255u ? 2047u : e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)((u & 0x7u) << 29));
}
__device__ __forceinline__ float d2f_trunc(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned e = (hi >> 20) & 0x7ffu;
    const unsigned sign = hi & 0x80000000u;
    if (e < 897u) return __uint_as_float(sign);
    if (e > 1150u) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
template <> __device__ __forceinline__ double2 cvt<double2, float2>(float2 a) {
    return make_double2(f2d_exact(a.x), f2d_exact(a.y));
}

// Double-single ("DS") complex numbers: float4 = (re_hi, re_lo, im_hi, im_lo),
// value = hi + lo per part, |lo| <= ulp(hi); about 48 significant bits.
// Splitting a double costs one FP64 subtraction (the rest is integer work):
// hi is the mantissa truncated to 24 bits, so x - hi is exact in FP64.
__device__ __forceinline__ float2 ds_split(double x) {
    const float hi = d2f_trunc(x);
    const float lo = d2f_trunc(x - f2d_exact(hi));
    return make_float2(hi, lo);
}
__device__ __forceinline__ double ds_join(float hi, float lo) { return f2d_exact(hi) + f2d_exact(lo); }
template <> __device__ __forceinline__ float4 cvt<float4, double2>(double2 a) {
    const float2 r = ds_split(a.x), i = ds_split(a.y);
    return make_float4(r.x, r.y, i.x, i.y);
}
template <> __device__ __forceinline__ double2 cvt<double2, float4>(float4 a) {
    return make_double2(ds_join(a.x, a.y), ds_join(a.z, a.w));
}
template <> __device__ __forceinline__ float2 cvt<float2, float4>(float4 a) {
    return make_float2(a.x + a.y, a.z + a.w);
}
template <> __device__ __forceinline__ float4 cvt<float4, float4>(float4 a) { return a; }
template <> __device__ __forceinline__ float2 cvt<float2, double2>(double2 a) {
    return make_float2(d2f_trunc(a.x), d2f_trunc(a.y));
}

// ------------------------------------------------------------ level geometry
// One multigrid level (or the fine grid) as the kernels see it.
template <typename T> struct LevelView {
    int nx, ny, nz;          // node counts (1 on unused axes)
    int dim;
    T inv_h2;                // 1 / h^2
    T two_over_h;            // 2 / h
    const T *w;              // omega^2 m^2 per node
    const cplx_t<T> *dinv;   // 1 / diagonal of M per node (fused V-cycle), or null
    const T *rho;            // rho of Eq. 1 per node (variable density), or null (rho = 1)
};

// Shift of the zero-order term and the boundary factor q = sqrt(1 - j alpha).
template <typename T> struct OpShift {
    T s_re, s_im;            // s
    T q_re, q_im;            // q
};

// ------------------------------------------------------------ last-block reductions
// Sum of p[lane], p[lane + 32], p[lane + 64], ... (n values in all, in this
// order), as one lane's share of a cross-block reduction: four loads are in
// flight at a time instead of one per dependent add.
__device__ __forceinline__ void lane_sum(const double2 *p, unsigned n, unsigned lane, double &sx,
                                         double &sy) {
    sx = 0.0;
    sy = 0.0;
    unsigned b = lane;
    for (; b + 96 < n; b += 128) {
        const double2 v0 = p[b], v1 = p[b + 32], v2 = p[b + 64], v3 = p[b + 96];
        sx += v0.x;
        sy += v0.y;
        sx += v1.x;
        sy += v1.y;
        sx += v2.x;
        sy += v2.y;
        sx += v3.x;
        sy += v3.y;
    }
    for (; b < n; b += 32) {
        const double2 v = p[b];
        sx += v.x;
        sy += v.y;
    }
}
__device__ __forceinline__ double lane_sum(const double *p, unsigned n, unsigned lane) {
    double s = 0.0;
    unsigned b = lane;
    for (; b + 96 < n; b += 128) {
        const double v0 = p[b], v1 = p[b + 32], v2 = p[b + 64], v3 = p[b + 96];
        s += v0;
        s += v1;
        s += v2;
        s += v3;
    }
    for (; b < n; b += 32) s += p[b];
    return s;
}

// ------------------------------------------------------------ launch counter + profiler
void count_launch(uint64_t k = 1);
void uncount_launch(uint64_t k);     // kernels that were captured into a graph, not run
uint64_t launch_count();

// Optional per-launch timing (off by default). prof_begin records a start
// event on the launch stream; prof_end records the stop event and the
// launch's algorithmic bytes and FP64 flops under `name`.
bool prof_on();
void prof_begin(cudaStream_t st);
void prof_end(const char *name, cudaStream_t st, double bytes, double flops64);
// During graph capture the timing events become event-record nodes of the
// graph; prof_graph_replayed() reads them after each replay of that graph.
struct ProfRecPublic {
    const char *name;
    cudaEvent_t e0, e1;
    double bytes, flops;
};
void prof_capture_begin();
std::vector<ProfRecPublic> prof_capture_end();
void prof_graph_replayed(const std::vector<ProfRecPublic> &recs);

// ------------------------------------------------------------ stencil family
enum StencilMode { ST_APPLY = 0, ST_RESID = 1, ST_JACOBI = 2, ST_JACOBI0 = 3 };

// mode APPLY : y = A x
// mode RESID : y = b - A x
// mode JACOBI: y = x + wj (b - A x) / d
// mode JACOBI0: y = wj b / d        (x ignored: first sweep from zero)
// nb right-hand sides at strides sx, sb, sy (elements); blockIdx.z walks them.
template <typename T, typename CIn, typename COut>
void launch_stencil(int mode, const LevelView<T> &L, OpShift<T> s, const CIn *x, size_t sx,
                    const COut *b, size_t sb, COut *y, size_t sy, int nb, T wj,
                    const int *active, cudaStream_t st);

template <typename T>
void launch_restrict(const LevelView<T> &fine, const LevelView<T> &coarse, const cplx_t<T> *rf,
                     size_t sf, cplx_t<T> *rc, size_t sc, int nb, const int *active,
                     cudaStream_t st);

template <typename T>
void launch_prolong_add(const LevelView<T> &fine, const LevelView<T> &coarse,
                        const cplx_t<T> *ec, size_t sc, const cplx_t<T> *uin, size_t sin,
                        cplx_t<T> *uf, size_t sf, int nb, const int *active, cudaStream_t st);

// dinv = 1 / diag(M) on a level (diagonal from Eq. 6 with the absorbing
// boundary term), computed in FP64 and stored as C (double2 or float2).
template <typename C>
void launch_make_dinv(const LevelView<double> &L, OpShift<double> s, C *dinv, cudaStream_t st);

// Fused V(1,1) level kernels for 2D/3D (templates in vfused.cuh, instantiated
// per type pair in vfused_*.cu). CB: type of the level's right-hand side
// (complex128 basis vector at level 0 of the mixed form).
// `finest` only names the launch for the profiler (level 0 is reported apart
// from the coarser levels).
template <typename T, typename CB>
void launch_vdown(const LevelView<T> &F, const LevelView<T> &Cv, T wj, const CB *b,
                  size_t sb, cplx_t<T> *u, size_t su, cplx_t<T> *bc, size_t sbc, int nb,
                  const int *active, cudaStream_t st, int shape, bool finest = false);
template <typename T, typename CB>
void launch_vup(const LevelView<T> &F, const LevelView<T> &Cv, T wj,
                const cplx_t<T> *uin, size_t sin, const cplx_t<T> *ec, size_t sec, const CB *b,
                size_t sb, cplx_t<T> *uout, size_t sout, int nb, const int *active,
                cudaStream_t st, int shape, bool finest = false);
// tile shapes of the fused kernels: count per dimension (down and up lists
// have equal length) and the extents/threads of one (kernel 0 down, 1 up)
int num_tile_shapes(int dim);
bool tile_shape(int dim, int kernel, int shape, int ext[3], int *threads, int *rb = nullptr);
// automatic shape for a fine level of `fine` nodes and nb right-hand sides:
// the first shape in list order whose grid has at least 2 blocks per SM, else
// the shape with the most blocks (small levels need every SM)
int auto_tile_shape(int dim, int kernel, const int fine[3], int nb);
void prepare_vfused();   // sets shared-memory attributes; call outside graph capture

// ------------------------------------------------------------ set-up kernels
// w64 = omega^2 m^2 (and w32 = float(w64) if non-null); flag |= 1 where m is
// not finite or not > 0
void launch_make_w(const double *m, size_t n, double omega, double *w64, float *w32, int *flag,
                   cudaStream_t st);
// rho32 = float(rho64); flag |= 1 where rho is not finite or not > 0
void launch_make_rho(const double *rho64, size_t n, float *rho32, int *flag, cudaStream_t st);
// coarse[I] = fine[2 I] (injection) on an nx x ny x nz coarse grid
template <typename T>
void launch_inject(const T *fine, int fnx, int fny, T *coarse, int cnx, int cny, int cnz,
                   cudaStream_t st);

// ------------------------------------------------------------ coarse solve
template <typename T>
void launch_assemble_dense(const LevelView<T> &L, OpShift<T> s, cplx_t<T> *A, cudaStream_t st);
template <typename T>
void launch_gauss_jordan(cplx_t<T> *A, cplx_t<T> *colbuf, int n, cudaStream_t st);
// z = Ainv r for nb right-hand sides (complex128; the complex64 product is launch_coarse_tc)
template <typename T>
void launch_dense_gemv(const cplx_t<T> *At, int n, const cplx_t<T> *r, size_t sr,
                       cplx_t<T> *z, size_t sz, int nb, const int *active, void *part,
                       unsigned *ticket, cudaStream_t st);
// the inverse is stored transposed (column-major) for launch_dense_gemv
template <typename T>
void launch_transpose_square(cplx_t<T> *A, int n, cudaStream_t st);
// complex64 coarse product on the tensor cores (tcgen05 kind::tf32, FP32
// operands split into TF32 hi + lo): Ainv (given column-major, as stored for
// launch_dense_gemv) is laid out once into coarse_tc_tile_floats(n) floats;
// z = Ainv r for nb right-hand sides uses coarse_tc_part_floats(n, nb) floats
// of scratch
size_t coarse_tc_tile_floats(int n);
size_t coarse_tc_part_floats(int n, int nb);
void launch_coarse_tc_tiles(const float2 *At, int n, float *tiles, cudaStream_t st);
void launch_coarse_tc(const float *tiles, int n, const float2 *r, size_t sr, float2 *z, size_t sz,
                      int nb, const int *active, float *part, cudaStream_t st);
// scratch of launch_dense_gemv for nb right-hand sides: group sums (complex
// elements of the V-cycle type) and tickets (unsigned, zero at rest)
size_t coarse_part_elems(int n, int nb);
size_t coarse_tickets(int n, int nb);
void prepare_coarse_kernels();   // shared-memory attributes; call outside graph capture

// ------------------------------------------------------------ Krylov (complex128 outer)
// All vectors of right-hand side k sit at base + k * stride_rhs; basis vector i
// of right-hand side k at V + k * stride_rhs + i * N.
constexpr int kMaxBlocks = 8 * 152;   // reduction grids: at most this many blocks (scratch size)

// Number of SMs of the current device (read once per device and cached).
// Grid shapes derive from it, so every sum's order is fixed per device.
int device_sms();

struct KrylovScratch {
    double2 *partial;        // [nrhs][max_blocks][nvec_max] block partial sums
    unsigned *counter;       // [nrhs] last-block counters (zero between launches)
    int max_blocks;
    int nvec_max;
};

// out[k * out_stride + i] = sum_p conj(V_i[p]) w[p], i < nvec
void launch_multidot(const double2 *V, size_t sV, int nvec, const double2 *w, size_t sw,
                     size_t N, double2 *out, size_t out_stride, int nrhs, const int *active,
                     KrylovScratch &ks, cudaStream_t st);
// w[p] -= sum_i V_i[p] c[k * c_stride + i]; if norm2 != null, norm2[k] = ||w_new||^2
// w = H z (basis slot j+1) fused with the multi-dot of w against V_0..V_{nvec-1}
template <typename CZ>
void launch_multidot_h(const double2 *V, size_t sV, int nvec, double2 *w, size_t sw, size_t N,
                       double2 *out, size_t out_stride, int nrhs, const int *active,
                       KrylovScratch &ks, const LevelView<double> &L, OpShift<double> sH,
                       const CZ *z, size_t sz, cudaStream_t st);
void launch_multiaxpy(const double2 *V, size_t sV, int nvec, const double2 *c, size_t c_stride,
                      double2 *w, size_t sw, size_t N, double *norm2, int nrhs,
                      const int *active, KrylovScratch &ks, cudaStream_t st);
// norm2[k] = ||x||^2
void launch_norm2(const double2 *x, size_t sx, size_t N, double *norm2, int nrhs,
                  const int *active, KrylovScratch &ks, cudaStream_t st);
// y = x * scale[k] (real per right-hand side); COut may be float2 for the mixed V-cycle input
template <typename COut>
void launch_scale(const double2 *x, size_t sx, const double *scale, COut *y, size_t sy, size_t N,
                  int nrhs, const int *active, cudaStream_t st);
// x += sum_{i < min(nvec, kcount[k])} Z_i y[k * y_stride + i]   (Z complex128 or complex64;
// kcount nullable: all nvec columns)
template <typename CZ>
void launch_update(const CZ *Z, size_t sZ, int nvec, const double2 *y, size_t y_stride,
                   double2 *x, size_t sx, size_t N, int nrhs, const int *active, cudaStream_t st,
                   const int *kcount = nullptr);
template <typename CIn, typename COut>
void launch_convert(const CIn *x, size_t sx, COut *y, size_t sy, size_t N, int nrhs,
                    cudaStream_t st);
// act2[r] = act[r] && n1[r] < eta2 * Re h1[r][wslot]; zero h2[r][0..nvec) where no second pass
void launch_reorth_flags(const int *act, const double2 *h1, double2 *h2, int hstride, int wslot,
                         const double *n1, double eta2, int *act2, int nvec, int nrhs,
                         cudaStream_t st);
// ---- double-single basis (precision HELM_PREC_MIXED_DS): the same operations on
// a basis stored as float4 (re_hi, re_lo, im_hi, im_lo), computed with FP32
// error-free products and two-sums; results and coefficients stay complex128.
// double2 elements of KrylovScratch::partial that the double-single multi-dot
// and multi-axpy need per right-hand side (nvec_max = restart + 1)
size_t ds_partial_per_rhs(size_t N, int nvec_max);
void launch_multidot_ds(const float4 *V, size_t sV, int nvec, const float4 *w, size_t sw, size_t N,
                        double2 *out, size_t out_stride, int nrhs, const int *active,
                        KrylovScratch &ks, cudaStream_t st);
void launch_multiaxpy_ds(const float4 *V, size_t sV, int nvec, const double2 *c, size_t c_stride,
                         float4 *w, size_t sw, size_t N, double *norm2, int nrhs, const int *active,
                         KrylovScratch &ks, cudaStream_t st);
// time limit (ns) of the consumer waits of the streamed double-single kernels
// on the current device (synchronous copy to a device variable)
cudaError_t set_consumer_wait_ns(unsigned long long ns);
// y = x / sqrt(norm2[k]) with x complex128 or DS, y DS
template <typename CIn>
void launch_scale_ds(const CIn *x, size_t sx, const double *norm2, float4 *y, size_t sy, size_t N,
                     int nrhs, const int *active, cudaStream_t st);
// x += sum_i Z_i y_i where the basis is DS (no preconditioner: Z = V)
// x += Z y for complex64 Z, the sum formed in double-single (HELM_PREC_MIXED_DS)
void launch_update_zds(const float2 *Z, size_t sZ, int nvec, const double2 *y, size_t y_stride,
                       double2 *x, size_t sx, size_t N, int nrhs, const int *active, cudaStream_t st,
                       const int *kcount);
void launch_update_ds(const float4 *Z, size_t sZ, int nvec, const double2 *y, size_t y_stride,
                      double2 *x, size_t sx, size_t N, int nrhs, const int *active, cudaStream_t st,
                      const int *kcount = nullptr);

// ---- complex64 basis (precision HELM_PREC_MIXED_C64): v_i stored as float2 at
// a per-vector stride Nv = c64_stride(N) (N rounded up to even, so that every
// vector starts on a 16-byte boundary), the vector being orthogonalised as
// double-single float4 (stride sw), coefficients complex128; partial sums as
// the double-single kernels (ds_partial_per_rhs)
inline size_t c64_stride(size_t N) { return (N + 1) & ~(size_t)1; }
void launch_multidot_sb(const float2 *V, size_t sV, size_t Nv, int nvec, const float4 *w, size_t sw, size_t N,
                        double2 *out, size_t out_stride, int nrhs, const int *active, KrylovScratch &ks,
                        cudaStream_t st);
// scale (nullable, with norm2): per right-hand side 1/sqrt(norm2) as float hi + lo
void launch_multiaxpy_sb(const float2 *V, size_t sV, size_t Nv, int nvec, const double2 *c, size_t c_stride,
                         float4 *w, size_t sw, size_t N, double *norm2, int nrhs, const int *active,
                         KrylovScratch &ks, cudaStream_t st, float2 *scale = nullptr);
// v = w / sqrt(norm2[k]) rounded to complex64
void launch_scale_c64(const float4 *w, size_t sw, const double *norm2, float2 *v, size_t sv, size_t N, int nrhs,
                      const int *active, cudaStream_t st);
// The level-0 down kernel of the complex64-basis form that takes w (double-
// single) and the scale pair sc of launch_multiaxpy_sb instead of v: it forms
// v = w * (sc.x + sc.y) rounded to complex64 with the arithmetic of
// launch_scale_c64, writes v of its own nodes to vout (stride svout), and
// goes on as launch_vdown. 2D levels only: returns false, launching nothing,
// for a 3D level (the caller then scales w on its own first).
bool launch_vdown_c64w(const LevelView<float> &F, const LevelView<float> &Cv, float wj, const float4 *w,
                       size_t sw, const float2 *sc, float2 *vout, size_t svout, float2 *u, size_t su, float2 *bc,
                       size_t sbc, int nb, const int *active, cudaStream_t st, int shape);

// diagonal of H on the fine grid as double-single pairs, and w = H z in
// double-single arithmetic (z complex64, w double-single)
void launch_make_hdiag_ds(const LevelView<double> &L, OpShift<double> s, float4 *hd, cudaStream_t st);
void launch_apply_H_ds(const LevelView<double> &L, const float4 *hd, const float2 *z, size_t sz,
                       float4 *w, size_t sw, int nb, const int *active, cudaStream_t st);

// ---- block FGMRES tensor-core contractions (block.cu), complex64 vectors with
// per-vector stride, padded to Np nodes (a multiple of 8, zeros beyond N)
// G = V^H W for nv basis vectors and s <= 64 sources, complex128 G[i * ldg + c];
// with hacc non-null also hacc[c * ldh + i] = G (add = 0) or += G (add = 1)
void launch_bgram(const float2 *V, size_t sv, int nv, const float2 *W, size_t sw, int s, size_t Np,
                  float *part, double2 *G, int ldg, double2 *hacc, size_t ldh, int add, cudaStream_t st);
// out = alpha win + V (sign C), C[i * ldc + c] complex128 (nv x s); out may be win or V
void launch_bcomb(const float2 *V, size_t sv, int nv, const double2 *C, int ldc, double sign, float *img,
                  const float2 *win, size_t sw, float alpha, float2 *out, size_t so, int s, size_t N,
                  size_t Np, cudaStream_t st);
size_t block_gram_part_floats(int nv_max, size_t Np);
size_t block_image_floats(int nv_max);

// finite check: flag[0] |= 1 if any entry is NaN/Inf
void launch_finite_check(const double *x, size_t n, int *flag, cudaStream_t st);
// x_r = 0 (N complex128 values) for each right-hand side r with active[r] == 0
void launch_zero_inactive(double2 *x, size_t N, const int *active, int nrhs, cudaStream_t st);

}  // namespace helm
