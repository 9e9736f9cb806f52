// The scaling step of the complex64-basis form (precision
// HELM_PREC_MIXED_C64): v_{j+1} = w / ||w|| from the double-single w,
// rounded once to complex64. On 2D grids the next step's level-0 down kernel
// forms v_{j+1} itself with the same arithmetic (launch_vdown_c64w); this
// kernel serves 3D grids and the V-cycles that cannot take w. The streamed
// multi-dot and multi-axpy of that form sit beside their double-single
// counterparts in krylov_ds.cu.
#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int kThreads = 256;

// v = w / sqrt(norm2[r]) rounded to complex64: the double-single product with
// the scale (sh + sl) in FP32, rounded once
__global__ void __launch_bounds__(kThreads)
k_scale_c64(const float4 *__restrict__ w, size_t sw, const double *__restrict__ norm2, float2 *__restrict__ v,
            size_t sv, size_t N, const int *__restrict__ active) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    w += r * sw;
    v += r * sv;
    __shared__ float2 s_sh;
    if (threadIdx.x == 0) {
        const double s = 1.0 / sqrt(norm2[r]);
        const float sh = (float)s;
        s_sh = make_float2(sh, (float)(s - (double)sh));
    }
    __syncthreads();
    const float sh = s_sh.x, sl = s_sh.y;
    // four nodes per thread and round, all loads issued first
    const size_t stride = (size_t)gridDim.x * kThreads;
    size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x;
    for (; p + 3 * stride < N; p += 4 * stride) {
        float4 x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = w[p + q * stride];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            v[p + q * stride] = make_float2(fmaf(x[q].x, sh, fmaf(x[q].x, sl, x[q].y * sh)),
                                            fmaf(x[q].z, sh, fmaf(x[q].z, sl, x[q].w * sh)));
    }
    for (; p < N; p += stride) {
        const float4 x = w[p];
        v[p] = make_float2(fmaf(x.x, sh, fmaf(x.x, sl, x.y * sh)), fmaf(x.z, sh, fmaf(x.z, sl, x.w * sh)));
    }
}

}  // namespace

void launch_scale_c64(const float4 *w, size_t sw, const double *norm2, float2 *v, size_t sv, size_t N, int nrhs,
                      const int *active, cudaStream_t st) {
    // about four nodes per thread; a whole number of blocks per SM over the batch
    const size_t want = (N + 4 * kThreads - 1) / (4 * kThreads);
    const int nb = (int)(want < (size_t)(1 << 16) ? (want ? want : 1) : (1 << 16));
    prof_begin(st);
    k_scale_c64<<<dim3(nb, nrhs), kThreads, 0, st>>>(w, sw, norm2, v, sv, N, active);
    count_launch();
    if (prof_on()) prof_end("scale_c64", st, 24.0 * N * nrhs, 0.0);
}

}  // namespace helm
