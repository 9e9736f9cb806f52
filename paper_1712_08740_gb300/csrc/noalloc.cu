// True relative residual ||f - H u|| / ||f|| without any device allocation.
//
// Some callers cannot call cudaMalloc: a serving process that reserves the
// GPU's memory up front and hands it out from its own pool leaves nothing for
// cudaMalloc to take, and a caller that must not stall other streams cannot
// afford cudaMalloc/cudaFree, which may synchronise the device.
// helm_true_residual may allocate staging and reduction buffers on its first
// use; this variant never does. Its scratch is one file-scope device array of
// a fixed size, so it serves at most kNaMaxRhs right-hand sides per call.
//
// The residual and the norms are fused into one kernel: each thread forms
// r_p = f_p - (H u)_p in registers and accumulates |r_p|^2 and |f_p|^2, so
// no residual vector is stored. Blocks write their partial sums into the
// static array; the last block to finish (threadfence + atomic ticket) adds
// them in block order, so the result is deterministic.
#include <cmath>
#include <mutex>

#include "vcycle.cuh"

namespace helm {

namespace {

constexpr int kNaMaxRhs = 64;       // right-hand sides per call
constexpr int kNaBlocks = 304;      // reduction grid (fixed, so the summation order is too)
constexpr int kNaThreads = 256;
// layout of the scratch: partial sums [rhs][2][block], results [rhs][2],
// then one ticket counter per right-hand side
constexpr size_t kNaPartials = (size_t)kNaMaxRhs * 2 * kNaBlocks;
constexpr size_t kNaResults = (size_t)kNaMaxRhs * 2;
constexpr size_t kNaBytes = (kNaPartials + kNaResults) * sizeof(double) + kNaMaxRhs * sizeof(unsigned);

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

__device__ __forceinline__ double na_warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int DIM>
__global__ void __launch_bounds__(kNaThreads)
k_resid_norms(LevelView<double> L, OpShift<double> s, const double2 *__restrict__ f,
              const double2 *__restrict__ u, size_t N, unsigned char *__restrict__ scratch) {
    const int r = blockIdx.y;
    f += r * N;
    u += r * N;
    double *part = reinterpret_cast<double *>(scratch);
    double *res = part + kNaPartials;
    unsigned *ticket = reinterpret_cast<unsigned *>(res + kNaResults);
    const size_t nxy = (size_t)L.nx * L.ny;
    double rr = 0.0, ff = 0.0;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(p % L.nx);
        const int iy = (int)((p / L.nx) % L.ny);
        const int iz = (int)(p / nxy);
        const int c[3] = {ix, iy, iz};
        const int n[3] = {L.nx, L.ny, L.nz};
        const size_t st[3] = {1, (size_t)L.nx, nxy};
        double sx = 0.0, sy = 0.0;
        int nf = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            if (c[a] > 0) {
                const double w = (c[a] == n[a] - 1) ? 2.0 : 1.0;
                const double2 v = u[p - st[a]];
                sx += w * v.x;
                sy += w * v.y;
            } else {
                ++nf;
            }
            if (c[a] < n[a] - 1) {
                const double w = (c[a] == 0) ? 2.0 : 1.0;
                const double2 v = u[p + st[a]];
                sx += w * v.x;
                sy += w * v.y;
            } else {
                ++nf;
            }
        }
        const double wp = L.w[p];
        double dre = 2.0 * DIM * L.inv_h2 - s.s_re * wp;
        double dim_ = -s.s_im * wp;
        if (nf) {
            const double fb = nf * L.two_over_h * sqrt(wp);
            dre -= fb * s.q_im;
            dim_ += fb * s.q_re;
        }
        const double2 up = u[p], fp = f[p];
        const double ax = dre * up.x - dim_ * up.y - L.inv_h2 * sx;
        const double ay = dre * up.y + dim_ * up.x - L.inv_h2 * sy;
        const double ex = fp.x - ax, ey = fp.y - ay;
        rr = fma(ex, ex, fma(ey, ey, rr));
        ff = fma(fp.x, fp.x, fma(fp.y, fp.y, ff));
    }
    __shared__ double red[2][kNaThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    rr = na_warp_sum(rr);
    ff = na_warp_sum(ff);
    if (lane == 0) {
        red[0][warp] = rr;
        red[1][warp] = ff;
    }
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < kNaThreads / 32; ++q) {
            a += red[0][q];
            b += red[1][q];
        }
        part[((size_t)r * 2 + 0) * kNaBlocks + blockIdx.x] = a;
        part[((size_t)r * 2 + 1) * kNaBlocks + blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(&ticket[r], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && warp < 2) {
        __threadfence();
        double v = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) v += part[((size_t)r * 2 + warp) * kNaBlocks + b];
        v = na_warp_sum(v);
        if (lane == 0) res[(size_t)r * 2 + warp] = v;
    }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_na_mu;
void *g_na_ptr[64] = {};

helm_status na_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(HELM_ERR_UNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(HELM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s",
                        cudaGetErrorString(e));
        }
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return HELM_OK;
}

}  // namespace

}  // namespace helm

using namespace helm;

extern "C" helm_status helm_true_residual_noalloc(helm_grid *g, int nrhs, const helm_c128 *f,
                                                  const helm_c128 *u, double *rel) {
    clear_error();
    if (!g || !f || !u || !rel) return fail(HELM_ERR_ARG, "null argument");
    if (nrhs < 1 || nrhs > kNaMaxRhs)
        return fail(HELM_ERR_ARG, "nrhs = %d is outside 1..%d, the size of the static scratch", nrhs,
                    kNaMaxRhs);
    if (!g->has_model) return fail(HELM_ERR_STATE, "helm_set_model has not been called");
    if (g->has_rho) return fail(HELM_ERR_UNSUPPORTED, "variable density is not served by this entry point");
    if (!is_device_ptr(f) || !is_device_ptr(u))
        return fail(HELM_ERR_ARG, "f and u must be device pointers (this entry point stages nothing)");
    {
        // both arrays must live on the current device: another device's
        // memory would be read through the wrong address space
        int cur = -1;
        cudaPointerAttributes af, au;
        if (cudaGetDevice(&cur) != cudaSuccess || cudaPointerGetAttributes(&af, f) != cudaSuccess ||
            cudaPointerGetAttributes(&au, u) != cudaSuccess) {
            cudaGetLastError();
            return fail(HELM_ERR_CUDA, "pointer attributes");
        }
        if ((af.type == cudaMemoryTypeDevice && af.device != cur) ||
            (au.type == cudaMemoryTypeDevice && au.device != cur))
            return fail(HELM_ERR_ARG, "f and u must be device pointers of the current device %d", cur);
    }
    void *scr = nullptr;
    helm_status s = na_scratch(&scr);
    if (s) return s;
    unsigned char *base = static_cast<unsigned char *>(scr);
    unsigned *ticket = reinterpret_cast<unsigned *>(base + (kNaPartials + kNaResults) * sizeof(double));
    // the tickets must start at zero; the array keeps whatever the last call left
    cudaError_t e = cudaMemsetAsync(ticket, 0, nrhs * sizeof(unsigned), g->st);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "clearing the scratch: %s", cudaGetErrorString(e));
    const LevelView<double> L = level_view<double>(g, 0);
    const dim3 grid(kNaBlocks, nrhs);
    if (g->dim == 1)
        k_resid_norms<1><<<grid, kNaThreads, 0, g->st>>>(L, shift_H(g), (const double2 *)f, (const double2 *)u, g->N, base);
    else if (g->dim == 2)
        k_resid_norms<2><<<grid, kNaThreads, 0, g->st>>>(L, shift_H(g), (const double2 *)f, (const double2 *)u, g->N, base);
    else
        k_resid_norms<3><<<grid, kNaThreads, 0, g->st>>>(L, shift_H(g), (const double2 *)f, (const double2 *)u, g->N, base);
    count_launch();
    double out[2 * kNaMaxRhs];
    e = cudaMemcpyAsync(out, base + kNaPartials * sizeof(double), (size_t)nrhs * 2 * sizeof(double),
                        cudaMemcpyDeviceToHost, g->st);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, "reading the result: %s", cudaGetErrorString(e));
    if ((s = sync_stream(g, "helm_true_residual_noalloc"))) return s;
    for (int k = 0; k < nrhs; ++k)
        rel[k] = out[2 * k + 1] > 0.0 ? std::sqrt(out[2 * k] / out[2 * k + 1]) : 0.0;
    return HELM_OK;
}
