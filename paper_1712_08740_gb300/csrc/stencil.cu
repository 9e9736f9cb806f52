// Matrix-free stencil kernels: H and M application (Eq. 2-3, Eq. 6), residual,
// damped Jacobi, full-weighting restriction and multilinear prolongation.
//
// Thread mapping: one thread per node; threadIdx.x / blockIdx.x run along x
// (the contiguous axis, so every load and store of a warp is one coalesced
// segment of float2/double2), blockIdx.y walks the (y, z) rows, blockIdx.z the
// right-hand sides. Neighbour reuse across rows comes from L1/L2: a 2D row of
// a 1601-node grid is 13 KB in complex64, so the three rows a block touches
// stay on chip.
#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int kBX = 128;

template <typename T> __device__ __forceinline__ T dsqrt(T v);
template <> __device__ __forceinline__ float dsqrt<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double dsqrt<double>(double v) { return sqrt(v); }

// Accumulates the weighted neighbours along one axis and counts boundary faces.
template <typename T, typename CIn>
__device__ __forceinline__ void axis_terms(const CIn *__restrict__ x, size_t p, int i, int n,
                                           size_t stride, T &sre, T &sim, int &nf) {
    if (i > 0) {
        auto v = cvt<cplx_t<T>>(x[p - stride]);
        T c = (i == n - 1) ? T(2) : T(1);
        sre += c * v.x;
        sim += c * v.y;
    } else {
        ++nf;
    }
    if (i < n - 1) {
        auto v = cvt<cplx_t<T>>(x[p + stride]);
        T c = (i == 0) ? T(2) : T(1);
        sre += c * v.x;
        sim += c * v.y;
    } else {
        ++nf;
    }
}

// The same with the face coefficients of Eq. 1: each neighbour weight is
// c times the mean of rho at the node and the neighbour; dsum collects the
// weights (the Laplacian part of the diagonal) and bsum, per boundary face,
// the coefficient of the inner face (the absorbing term's factor). With
// LOADX false only the weights are formed (the first Jacobi sweep).
template <typename T, bool LOADX, typename CIn>
__device__ __forceinline__ void axis_terms_rho(const CIn *__restrict__ x, const T *__restrict__ rho, T rp,
                                               size_t p, int i, int n, size_t stride, T &sre, T &sim,
                                               T &dsum, T &bsum) {
    if (i > 0) {
        const T face = T(0.5) * (rp + rho[p - stride]);
        const T c = (i == n - 1) ? T(2) * face : face;
        if (LOADX) {
            auto v = cvt<cplx_t<T>>(x[p - stride]);
            sre += c * v.x;
            sim += c * v.y;
        }
        dsum += c;
        if (i == n - 1) bsum += face;
    }
    if (i < n - 1) {
        const T face = T(0.5) * (rp + rho[p + stride]);
        const T c = (i == 0) ? T(2) * face : face;
        if (LOADX) {
            auto v = cvt<cplx_t<T>>(x[p + stride]);
            sre += c * v.x;
            sim += c * v.y;
        }
        dsum += c;
        if (i == 0) bsum += face;
    }
}

template <typename T, int DIM, int MODE, bool RHO, typename CIn, typename COut>
__global__ void __launch_bounds__(kBX)
k_stencil(LevelView<T> L, OpShift<T> s, const CIn *__restrict__ x, size_t sx,
          const COut *__restrict__ b, size_t sb, COut *__restrict__ y, size_t sy, T wj,
          const int *__restrict__ active) {
    const int r = blockIdx.z;
    if (active && !active[r]) return;
    x += r * sx;
    b += r * sb;
    y += r * sy;
    const int nx = L.nx;
    const int rows = L.ny * L.nz;
    const int ix = blockIdx.x * kBX + threadIdx.x;
    if (ix >= nx) return;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const size_t p = (size_t)row * nx + ix;
        T sre = 0, sim = 0;
        int nf = 0;
        T dsum = 0, bsum = 0;
        if (RHO) {
            constexpr bool LX = MODE != ST_JACOBI0;
            const T rp = L.rho[p];
            axis_terms_rho<T, LX>(x, L.rho, rp, p, ix, nx, 1, sre, sim, dsum, bsum);
            if (DIM >= 2) {
                const int iy = (DIM == 3) ? row % L.ny : row;
                axis_terms_rho<T, LX>(x, L.rho, rp, p, iy, L.ny, (size_t)nx, sre, sim, dsum, bsum);
            }
            if (DIM == 3) {
                const int iz = row / L.ny;
                axis_terms_rho<T, LX>(x, L.rho, rp, p, iz, L.nz, (size_t)nx * L.ny, sre, sim, dsum, bsum);
            }
            // kappa_p / sqrt(rho_p) on the boundary faces, weighted by their inner faces
            bsum /= dsqrt<T>(rp);
        } else if (MODE != ST_JACOBI0) {
            axis_terms<T>(x, p, ix, nx, 1, sre, sim, nf);
            if (DIM >= 2) {
                const int iy = (DIM == 3) ? row % L.ny : row;
                axis_terms<T>(x, p, iy, L.ny, (size_t)nx, sre, sim, nf);
            }
            if (DIM == 3) {
                const int iz = row / L.ny;
                axis_terms<T>(x, p, iz, L.nz, (size_t)nx * L.ny, sre, sim, nf);
            }
        } else {
            nf = (ix == 0) + (ix == nx - 1);
            if (DIM >= 2) {
                const int iy = (DIM == 3) ? row % L.ny : row;
                nf += (iy == 0) + (iy == L.ny - 1);
            }
            if (DIM == 3) {
                const int iz = row / L.ny;
                nf += (iz == 0) + (iz == L.nz - 1);
            }
        }
        const T wp = L.w[p];
        T dre = (RHO ? dsum : T(2 * DIM)) * L.inv_h2 - s.s_re * wp;
        T dim_ = -s.s_im * wp;
        if (RHO ? bsum != T(0) : nf != 0) {
            const T f = (RHO ? bsum : T(nf)) * L.two_over_h * dsqrt<T>(wp);
            dre -= f * s.q_im;     // j * kappa = sqrt(w) (-q_im + j q_re)
            dim_ += f * s.q_re;
        }
        using C = cplx_t<T>;
        if (MODE == ST_JACOBI0) {
            C bp = cvt<C>(b[p]);
            T inv = wj / (dre * dre + dim_ * dim_);
            C o;
            o.x = (bp.x * dre + bp.y * dim_) * inv;
            o.y = (bp.y * dre - bp.x * dim_) * inv;
            y[p] = cvt<COut>(o);
            continue;
        }
        C xp = cvt<C>(x[p]);
        C ax;
        ax.x = dre * xp.x - dim_ * xp.y - L.inv_h2 * sre;
        ax.y = dre * xp.y + dim_ * xp.x - L.inv_h2 * sim;
        if (MODE == ST_APPLY) {
            y[p] = cvt<COut>(ax);
        } else {
            C bp = cvt<C>(b[p]);
            C rr;
            rr.x = bp.x - ax.x;
            rr.y = bp.y - ax.y;
            if (MODE == ST_RESID) {
                y[p] = cvt<COut>(rr);
            } else {  // ST_JACOBI
                T inv = wj / (dre * dre + dim_ * dim_);
                C o;
                o.x = xp.x + (rr.x * dre + rr.y * dim_) * inv;
                o.y = xp.y + (rr.y * dre - rr.x * dim_) * inv;
                y[p] = cvt<COut>(o);
            }
        }
    }
}

inline dim3 grid_for(int nx, int rows, int nb) {
    int gy = rows < 65535 ? rows : 65535;
    return dim3((nx + kBX - 1) / kBX, gy, nb);
}

template <typename T, int MODE, typename CIn, typename COut>
void dispatch_dim(const LevelView<T> &L, OpShift<T> s, const CIn *x, size_t sx, const COut *b,
                  size_t sb, COut *y, size_t sy, int nb, T wj, const int *active,
                  cudaStream_t st) {
    dim3 g = grid_for(L.nx, L.ny * L.nz, nb);
    prof_begin(st);
    if (L.rho) {
        if (L.dim == 1)
            k_stencil<T, 1, MODE, true><<<g, kBX, 0, st>>>(L, s, x, sx, b, sb, y, sy, wj, active);
        else if (L.dim == 2)
            k_stencil<T, 2, MODE, true><<<g, kBX, 0, st>>>(L, s, x, sx, b, sb, y, sy, wj, active);
        else
            k_stencil<T, 3, MODE, true><<<g, kBX, 0, st>>>(L, s, x, sx, b, sb, y, sy, wj, active);
    } else if (L.dim == 1)
        k_stencil<T, 1, MODE, false><<<g, kBX, 0, st>>>(L, s, x, sx, b, sb, y, sy, wj, active);
    else if (L.dim == 2)
        k_stencil<T, 2, MODE, false><<<g, kBX, 0, st>>>(L, s, x, sx, b, sb, y, sy, wj, active);
    else
        k_stencil<T, 3, MODE, false><<<g, kBX, 0, st>>>(L, s, x, sx, b, sb, y, sy, wj, active);
    count_launch();
    if (prof_on()) {
        // algorithmic traffic per node: x (except JACOBI0), b (RESID/JACOBI*), y, w
        const double n = (double)L.nx * L.ny * L.nz * nb;
        double per = sizeof(COut) + sizeof(T) * (L.rho ? 2 : 1);
        if (MODE != ST_JACOBI0) per += sizeof(CIn);
        if (MODE != ST_APPLY) per += sizeof(COut);
        // flops: neighbour sums, diagonal, d*x - S/h^2, plus residual / damped update
        double fl = (MODE == ST_JACOBI0) ? 14.0 : 4.0 * L.dim + 12.0;
        if (MODE == ST_RESID) fl += 2.0;
        if (MODE == ST_JACOBI) fl += 14.0;
        static const char *names[2][4] = {
            {"stencil_apply_f32", "stencil_resid_f32", "jacobi_f32", "jacobi0_f32"},
            {"stencil_apply_f64", "stencil_resid_f64", "jacobi_f64", "jacobi0_f64"}};
        prof_end(names[sizeof(T) == 8][MODE], st, n * per, sizeof(T) == 8 ? n * fl : 0.0);
    }
}

// ------------------------------------------------------------ restriction
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX)
k_restrict(LevelView<T> F, LevelView<T> Cv, const cplx_t<T> *__restrict__ rf, size_t sf,
           cplx_t<T> *__restrict__ rc, size_t sc, const int *__restrict__ active) {
    const int r = blockIdx.z;
    if (active && !active[r]) return;
    rf += r * sf;
    rc += r * sc;
    const int I = blockIdx.x * kBX + threadIdx.x;
    if (I >= Cv.nx) return;
    const int rows = Cv.ny * Cv.nz;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int J = (DIM >= 2) ? ((DIM == 3) ? row % Cv.ny : row) : 0;
        const int K = (DIM == 3) ? row / Cv.ny : 0;
        T are = 0, aim = 0;
        for (int oz = (DIM == 3 ? -1 : 0); oz <= (DIM == 3 ? 1 : 0); ++oz) {
            int fz = 2 * K + oz;
            if (fz < 0) fz = 1;
            if (fz > F.nz - 1) fz = F.nz - 2;
            const T wz = (DIM == 3) ? (oz == 0 ? T(0.5) : T(0.25)) : T(1);
            for (int oy = (DIM >= 2 ? -1 : 0); oy <= (DIM >= 2 ? 1 : 0); ++oy) {
                int fy = 2 * J + oy;
                if (fy < 0) fy = 1;
                if (fy > F.ny - 1) fy = F.ny - 2;
                const T wy = (DIM >= 2) ? (oy == 0 ? T(0.5) : T(0.25)) : T(1);
                const size_t rowbase = ((size_t)fz * F.ny + fy) * F.nx;
                for (int ox = -1; ox <= 1; ++ox) {
                    int fx = 2 * I + ox;
                    if (fx < 0) fx = 1;
                    if (fx > F.nx - 1) fx = F.nx - 2;
                    const T wx = (ox == 0) ? T(0.5) : T(0.25);
                    const cplx_t<T> v = rf[rowbase + fx];
                    const T wgt = wx * wy * wz;
                    are += wgt * v.x;
                    aim += wgt * v.y;
                }
            }
        }
        cplx_t<T> o;
        o.x = are;
        o.y = aim;
        rc[(size_t)row * Cv.nx + I] = o;
    }
}

// ------------------------------------------------------------ prolongation + correction
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX)
k_prolong_add(LevelView<T> F, LevelView<T> Cv, const cplx_t<T> *__restrict__ ec, size_t sc,
              const cplx_t<T> *uin, size_t sin, cplx_t<T> *uf, size_t sf,
              const int *__restrict__ active) {
    // uf = uin + P ec; uin may alias uf (in-place correction)
    const int r = blockIdx.z;
    if (active && !active[r]) return;
    ec += r * sc;
    uin += r * sin;
    uf += r * sf;
    const int i = blockIdx.x * kBX + threadIdx.x;
    if (i >= F.nx) return;
    const int rows = F.ny * F.nz;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int j = (DIM >= 2) ? ((DIM == 3) ? row % F.ny : row) : 0;
        const int k = (DIM == 3) ? row / F.ny : 0;
        // per axis: even -> one coarse node (weight 1); odd -> two (1/2 each)
        const int x0 = i >> 1, x1 = (i & 1) ? x0 + 1 : x0;
        const int y0 = j >> 1, y1 = (j & 1) ? y0 + 1 : y0;
        const int z0 = k >> 1, z1 = (k & 1) ? z0 + 1 : z0;
        const T wx = (i & 1) ? T(0.5) : T(1);
        const T wy = (j & 1) ? T(0.5) : T(1);
        const T wz = (k & 1) ? T(0.5) : T(1);
        T are = 0, aim = 0;
        const int nzc = (DIM == 3) ? 2 : 1, nyc = (DIM >= 2) ? 2 : 1;
        for (int a = 0; a < nzc; ++a) {
            const int zz = a ? z1 : z0;
            if (a && z1 == z0) break;
            for (int bq = 0; bq < nyc; ++bq) {
                const int yy = bq ? y1 : y0;
                if (bq && y1 == y0) break;
                const size_t base = ((size_t)zz * Cv.ny + yy) * Cv.nx;
                cplx_t<T> v0 = ec[base + x0];
                are += v0.x;
                aim += v0.y;
                if (x1 != x0) {
                    cplx_t<T> v1 = ec[base + x1];
                    are += v1.x;
                    aim += v1.y;
                }
            }
        }
        const T wgt = wx * wy * wz;
        const size_t p = (size_t)row * F.nx + i;
        cplx_t<T> u = uin[p];
        u.x += wgt * are;
        u.y += wgt * aim;
        uf[p] = u;
    }
}

}  // namespace

template <typename T, typename CIn, typename COut>
void launch_stencil(int mode, const LevelView<T> &L, OpShift<T> s, const CIn *x, size_t sx,
                    const COut *b, size_t sb, COut *y, size_t sy, int nb, T wj,
                    const int *active, cudaStream_t st) {
    switch (mode) {
        case ST_APPLY: dispatch_dim<T, ST_APPLY>(L, s, x, sx, b, sb, y, sy, nb, wj, active, st); break;
        case ST_RESID: dispatch_dim<T, ST_RESID>(L, s, x, sx, b, sb, y, sy, nb, wj, active, st); break;
        case ST_JACOBI: dispatch_dim<T, ST_JACOBI>(L, s, x, sx, b, sb, y, sy, nb, wj, active, st); break;
        default: dispatch_dim<T, ST_JACOBI0>(L, s, x, sx, b, sb, y, sy, nb, wj, active, st); break;
    }
}

template <typename T>
void launch_restrict(const LevelView<T> &fine, const LevelView<T> &coarse, const cplx_t<T> *rf,
                     size_t sf, cplx_t<T> *rc, size_t sc, int nb, const int *active,
                     cudaStream_t st) {
    dim3 g = grid_for(coarse.nx, coarse.ny * coarse.nz, nb);
    prof_begin(st);
    if (fine.dim == 1) k_restrict<T, 1><<<g, kBX, 0, st>>>(fine, coarse, rf, sf, rc, sc, active);
    else if (fine.dim == 2) k_restrict<T, 2><<<g, kBX, 0, st>>>(fine, coarse, rf, sf, rc, sc, active);
    else k_restrict<T, 3><<<g, kBX, 0, st>>>(fine, coarse, rf, sf, rc, sc, active);
    count_launch();
    if (prof_on()) {
        const double nf = (double)fine.nx * fine.ny * fine.nz * nb;
        const double nc = (double)coarse.nx * coarse.ny * coarse.nz * nb;
        prof_end(sizeof(T) == 8 ? "restrict_f64" : "restrict_f32", st,
                 (nf + nc) * sizeof(cplx_t<T>), 0.0);
    }
}

template <typename T>
void launch_prolong_add(const LevelView<T> &fine, const LevelView<T> &coarse,
                        const cplx_t<T> *ec, size_t sc, const cplx_t<T> *uin, size_t sin,
                        cplx_t<T> *uf, size_t sf, int nb, const int *active, cudaStream_t st) {
    dim3 g = grid_for(fine.nx, fine.ny * fine.nz, nb);
    prof_begin(st);
    if (fine.dim == 1)
        k_prolong_add<T, 1><<<g, kBX, 0, st>>>(fine, coarse, ec, sc, uin, sin, uf, sf, active);
    else if (fine.dim == 2)
        k_prolong_add<T, 2><<<g, kBX, 0, st>>>(fine, coarse, ec, sc, uin, sin, uf, sf, active);
    else
        k_prolong_add<T, 3><<<g, kBX, 0, st>>>(fine, coarse, ec, sc, uin, sin, uf, sf, active);
    count_launch();
    if (prof_on()) {
        const double nf = (double)fine.nx * fine.ny * fine.nz * nb;
        const double nc = (double)coarse.nx * coarse.ny * coarse.nz * nb;
        prof_end(sizeof(T) == 8 ? "prolong_f64" : "prolong_f32", st,
                 (2.0 * nf + nc) * sizeof(cplx_t<T>), 0.0);
    }
}

// explicit instantiations
#define HELM_INST_ST(T, CI, CO)                                                              \
    template void launch_stencil<T, CI, CO>(int, const LevelView<T> &, OpShift<T>, const CI *, \
                                            size_t, const CO *, size_t, CO *, size_t, int, T,  \
                                            const int *, cudaStream_t);
HELM_INST_ST(double, double2, double2)
HELM_INST_ST(double, float2, double2)
HELM_INST_ST(double, float2, float2)
HELM_INST_ST(float, float2, float2)
HELM_INST_ST(double, float2, float4)
HELM_INST_ST(double, float4, float4)
#undef HELM_INST_ST

template void launch_restrict<float>(const LevelView<float> &, const LevelView<float> &,
                                     const float2 *, size_t, float2 *, size_t, int, const int *,
                                     cudaStream_t);
template void launch_restrict<double>(const LevelView<double> &, const LevelView<double> &,
                                      const double2 *, size_t, double2 *, size_t, int,
                                      const int *, cudaStream_t);
template void launch_prolong_add<float>(const LevelView<float> &, const LevelView<float> &,
                                        const float2 *, size_t, const float2 *, size_t, float2 *,
                                        size_t, int, const int *, cudaStream_t);
template void launch_prolong_add<double>(const LevelView<double> &, const LevelView<double> &,
                                         const double2 *, size_t, const double2 *, size_t,
                                         double2 *, size_t, int, const int *, cudaStream_t);

}  // namespace helm
