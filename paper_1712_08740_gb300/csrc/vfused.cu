// Fused V(1,1) multigrid kernels for 2D and 3D levels (Eq. 6 operator M).
//
// down: from the level's right-hand side b, one kernel computes
//         u  = wj D^-1 b                          (first Jacobi sweep from 0)
//         r  = b - M u = (1 - wj) b + (1/h^2) sum_nbr c u_nbr
//         bc = full-weighting restriction of r    (mirrored outside nodes)
//       and writes u (the pre-smoothed iterate) and bc (the coarse
//       right-hand side). A block owns a tile of coarse nodes; it stages b
//       and u for the tile's fine footprint plus a halo of two fine nodes in
//       shared memory, so each fine u and r is computed once.
// up:   from the pre-smoothed u, the coarse correction e and b, one kernel
//       computes v = u + P e (multilinear prolongation) on a fine tile plus a
//       halo of one node in shared memory and writes one damped-Jacobi sweep
//       of v. Up and down never read what they write (u comes from the
//       level's scratch vector, the result goes to the iterate).
//
// The right-hand side type CB may be wider than the level's arithmetic
// (complex128 basis vector feeding a complex64 V-cycle): the conversion is
// fused into the loads.
#include "helm_internal.cuh"

namespace helm {

namespace {

template <typename T> __device__ __forceinline__ T dsqrt(T v);
template <> __device__ __forceinline__ float dsqrt<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double dsqrt<double>(double v) { return sqrt(v); }

// diagonal d_p of M at a node with `nf` boundary faces
template <typename T>
__device__ __forceinline__ void diag_of(const LevelView<T> &L, const OpShift<T> &s, T wp, int nf,
                                        int dim, T &dre, T &dim_) {
    dre = T(2 * dim) * L.inv_h2 - s.s_re * wp;
    dim_ = -s.s_im * wp;
    if (nf) {
        const T f = T(nf) * L.two_over_h * dsqrt<T>(wp);
        dre -= f * s.q_im;
        dim_ += f * s.q_re;
    }
}

__device__ __forceinline__ int mirror(int i, int n) {
    return i < 0 ? -i : (i > n - 1 ? 2 * (n - 1) - i : i);
}

template <int DIM> struct Tile;
template <> struct Tile<2> { static constexpr int CX = 16, CY = 8, CZ = 1, FX = 32, FY = 8, FZ = 1; };
template <> struct Tile<3> { static constexpr int CX = 8, CY = 4, CZ = 4, FX = 32, FY = 4, FZ = 4; };

template <typename T, typename CB, int DIM>
__global__ void __launch_bounds__(256)
k_down(LevelView<T> F, LevelView<T> Cv, OpShift<T> s, T wj, const CB *__restrict__ b, size_t sb,
       cplx_t<T> *__restrict__ u, size_t su, cplx_t<T> *__restrict__ bc, size_t sbc,
       const int *__restrict__ active) {
    using C = cplx_t<T>;
    using TL = Tile<DIM>;
    const int r = blockIdx.z / ((Cv.nz + TL::CZ - 1) / TL::CZ);
    const int bz = blockIdx.z % ((Cv.nz + TL::CZ - 1) / TL::CZ);
    if (active && !active[r]) return;
    b += r * sb;
    u += r * su;
    bc += r * sbc;
    const int I0 = blockIdx.x * TL::CX, J0 = blockIdx.y * TL::CY, K0 = bz * TL::CZ;
    // u region: fine [2*I0-2, 2*I0+2*CX] per axis (2*CX+3 nodes); r region one node inside
    constexpr int UX = 2 * TL::CX + 3, UY = 2 * TL::CY + 3, UZ = DIM == 3 ? 2 * TL::CZ + 3 : 1;
    constexpr int RX = UX - 2, RY = UY - 2, RZ = DIM == 3 ? UZ - 2 : 1;
    extern __shared__ unsigned char smem_raw[];
    C *su_ = reinterpret_cast<C *>(smem_raw);
    C *sb_ = su_ + UX * UY * UZ;
    C *sr_ = sb_ + UX * UY * UZ;
    const int X0 = 2 * I0 - 2, Y0 = 2 * J0 - 2, Z0 = DIM == 3 ? 2 * K0 - 2 : 0;
    const size_t fxy = (size_t)F.nx * F.ny;
    // phase 1: b and u = wj b / d on the u region (in-range nodes)
    for (int t = threadIdx.x; t < UX * UY * UZ; t += blockDim.x) {
        const int lx = t % UX, ly = (t / UX) % UY, lz = t / (UX * UY);
        const int x = X0 + lx, y = Y0 + ly, z = Z0 + lz;
        if (x < 0 || x >= F.nx || y < 0 || y >= F.ny || (DIM == 3 && (z < 0 || z >= F.nz))) continue;
        const size_t p = (size_t)z * fxy + (size_t)y * F.nx + x;
        const C bp = cvt<C>(b[p]);
        const int nf = (x == 0) + (x == F.nx - 1) + (y == 0) + (y == F.ny - 1) +
                       (DIM == 3 ? (z == 0) + (z == F.nz - 1) : 0);
        T dre, dim_;
        diag_of<T>(F, s, F.w[p], nf, DIM, dre, dim_);
        const T inv = wj / (dre * dre + dim_ * dim_);
        C up;
        up.x = (bp.x * dre + bp.y * dim_) * inv;
        up.y = (bp.y * dre - bp.x * dim_) * inv;
        su_[t] = up;
        sb_[t] = bp;
        // owned fine nodes: [2*I0, 2*I0 + 2*CX) per axis
        if (lx >= 2 && lx < 2 + 2 * TL::CX && ly >= 2 && ly < 2 + 2 * TL::CY &&
            (DIM == 2 || (lz >= 2 && lz < 2 + 2 * TL::CZ)))
            u[p] = up;
    }
    __syncthreads();
    // phase 2: r = (1 - wj) b + (1/h^2) sum c u_nbr on the r region (in-range nodes)
    for (int t = threadIdx.x; t < RX * RY * RZ; t += blockDim.x) {
        const int lx = t % RX + 1, ly = (t / RX) % RY + 1, lz = DIM == 3 ? t / (RX * RY) + 1 : 0;
        const int x = X0 + lx, y = Y0 + ly, z = Z0 + lz;
        if (x < 0 || x >= F.nx || y < 0 || y >= F.ny || (DIM == 3 && (z < 0 || z >= F.nz))) continue;
        const int q = (lz * UY + ly) * UX + lx;
        T sx = 0, sy = 0;
        // x axis
        if (x > 0) { const T c = (x == F.nx - 1) ? T(2) : T(1); sx += c * su_[q - 1].x; sy += c * su_[q - 1].y; }
        if (x < F.nx - 1) { const T c = (x == 0) ? T(2) : T(1); sx += c * su_[q + 1].x; sy += c * su_[q + 1].y; }
        if (y > 0) { const T c = (y == F.ny - 1) ? T(2) : T(1); sx += c * su_[q - UX].x; sy += c * su_[q - UX].y; }
        if (y < F.ny - 1) { const T c = (y == 0) ? T(2) : T(1); sx += c * su_[q + UX].x; sy += c * su_[q + UX].y; }
        if (DIM == 3) {
            if (z > 0) { const T c = (z == F.nz - 1) ? T(2) : T(1); sx += c * su_[q - UX * UY].x; sy += c * su_[q - UX * UY].y; }
            if (z < F.nz - 1) { const T c = (z == 0) ? T(2) : T(1); sx += c * su_[q + UX * UY].x; sy += c * su_[q + UX * UY].y; }
        }
        const C bp = sb_[q];
        C rr;
        rr.x = (T(1) - wj) * bp.x + F.inv_h2 * sx;
        rr.y = (T(1) - wj) * bp.y + F.inv_h2 * sy;
        sr_[t] = rr;
    }
    __syncthreads();
    // phase 3: full weighting onto the tile's coarse nodes
    const size_t cxy = (size_t)Cv.nx * Cv.ny;
    for (int t = threadIdx.x; t < TL::CX * TL::CY * TL::CZ; t += blockDim.x) {
        const int I = I0 + t % TL::CX, J = J0 + (t / TL::CX) % TL::CY,
                  K = K0 + (DIM == 3 ? t / (TL::CX * TL::CY) : 0);
        if (I >= Cv.nx || J >= Cv.ny || (DIM == 3 && K >= Cv.nz)) continue;
        T ax = 0, ay = 0;
#pragma unroll
        for (int oz = (DIM == 3 ? -1 : 0); oz <= (DIM == 3 ? 1 : 0); ++oz) {
            const int fz = DIM == 3 ? mirror(2 * K + oz, F.nz) : 0;
            const T wz = DIM == 3 ? (oz == 0 ? T(0.5) : T(0.25)) : T(1);
            const int rz = DIM == 3 ? fz - (Z0 + 1) : 0;
#pragma unroll
            for (int oy = -1; oy <= 1; ++oy) {
                const int fy = mirror(2 * J + oy, F.ny);
                const T wy = oy == 0 ? T(0.5) : T(0.25);
                const int ry = fy - (Y0 + 1);
#pragma unroll
                for (int ox = -1; ox <= 1; ++ox) {
                    const int fx = mirror(2 * I + ox, F.nx);
                    const T wgt = (ox == 0 ? T(0.5) : T(0.25)) * wy * wz;
                    const C v = sr_[(rz * RY + ry) * RX + (fx - (X0 + 1))];
                    ax += wgt * v.x;
                    ay += wgt * v.y;
                }
            }
        }
        C o;
        o.x = ax;
        o.y = ay;
        bc[(size_t)K * cxy + (size_t)J * Cv.nx + I] = o;
    }
}

template <typename T, typename CB, int DIM>
__global__ void __launch_bounds__(256)
k_up(LevelView<T> F, LevelView<T> Cv, OpShift<T> s, T wj, const cplx_t<T> *__restrict__ uin,
     size_t sin, const cplx_t<T> *__restrict__ ec, size_t sec, const CB *__restrict__ b, size_t sb,
     cplx_t<T> *__restrict__ uout, size_t sout, const int *__restrict__ active) {
    using C = cplx_t<T>;
    using TL = Tile<DIM>;
    const int nzb = (F.nz + TL::FZ - 1) / TL::FZ;
    const int r = blockIdx.z / nzb;
    const int bz = blockIdx.z % nzb;
    if (active && !active[r]) return;
    uin += r * sin;
    ec += r * sec;
    b += r * sb;
    uout += r * sout;
    const int x0 = blockIdx.x * TL::FX, y0 = blockIdx.y * TL::FY, z0 = bz * TL::FZ;
    constexpr int VX = TL::FX + 2, VY = TL::FY + 2, VZ = DIM == 3 ? TL::FZ + 2 : 1;
    constexpr int EX = TL::FX / 2 + 2, EY = TL::FY / 2 + 2, EZ = DIM == 3 ? TL::FZ / 2 + 2 : 1;
    extern __shared__ unsigned char smem_raw[];
    C *sv_ = reinterpret_cast<C *>(smem_raw);
    C *se_ = sv_ + VX * VY * VZ;
    const int cx0 = x0 / 2 - 1, cy0 = y0 / 2 - 1, cz0 = DIM == 3 ? z0 / 2 - 1 : 0;
    const size_t cxy = (size_t)Cv.nx * Cv.ny, fxy = (size_t)F.nx * F.ny;
    // phase 1: coarse correction around the tile
    for (int t = threadIdx.x; t < EX * EY * EZ; t += blockDim.x) {
        const int X = cx0 + t % EX, Y = cy0 + (t / EX) % EY, Z = cz0 + (DIM == 3 ? t / (EX * EY) : 0);
        if (X < 0 || X >= Cv.nx || Y < 0 || Y >= Cv.ny || (DIM == 3 && (Z < 0 || Z >= Cv.nz))) continue;
        se_[t] = ec[(size_t)Z * cxy + (size_t)Y * Cv.nx + X];
    }
    __syncthreads();
    // phase 2: v = u + P e on the tile plus a one-node halo
    for (int t = threadIdx.x; t < VX * VY * VZ; t += blockDim.x) {
        const int x = x0 - 1 + t % VX, y = y0 - 1 + (t / VX) % VY,
                  z = DIM == 3 ? z0 - 1 + t / (VX * VY) : 0;
        if (x < 0 || x >= F.nx || y < 0 || y >= F.ny || (DIM == 3 && (z < 0 || z >= F.nz))) continue;
        const int ax = (x >> 1) - cx0, bxp = ((x + 1) >> 1) - cx0;
        const int ay = (y >> 1) - cy0, byp = ((y + 1) >> 1) - cy0;
        const int az = DIM == 3 ? (z >> 1) - cz0 : 0, bzp = DIM == 3 ? ((z + 1) >> 1) - cz0 : 0;
        const T wx = (x & 1) ? T(0.5) : T(1), wy = (y & 1) ? T(0.5) : T(1),
                wz = (DIM == 3 && (z & 1)) ? T(0.5) : T(1);
        T px = 0, py = 0;
#pragma unroll
        for (int kz = 0; kz < (DIM == 3 ? 2 : 1); ++kz) {
            const int zz = kz ? bzp : az;
            if (kz && bzp == az) break;
#pragma unroll
            for (int ky = 0; ky < 2; ++ky) {
                const int yy = ky ? byp : ay;
                if (ky && byp == ay) break;
                const C e0 = se_[(zz * EY + yy) * EX + ax];
                px += e0.x;
                py += e0.y;
                if (bxp != ax) {
                    const C e1 = se_[(zz * EY + yy) * EX + bxp];
                    px += e1.x;
                    py += e1.y;
                }
            }
        }
        const T wgt = wx * wy * wz;
        C v = uin[(size_t)z * fxy + (size_t)y * F.nx + x];
        v.x += wgt * px;
        v.y += wgt * py;
        sv_[t] = v;
    }
    __syncthreads();
    // phase 3: one damped-Jacobi sweep on the tile
    for (int t = threadIdx.x; t < TL::FX * TL::FY * TL::FZ; t += blockDim.x) {
        const int lx = t % TL::FX, ly = (t / TL::FX) % TL::FY, lz = DIM == 3 ? t / (TL::FX * TL::FY) : 0;
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        if (x >= F.nx || y >= F.ny || (DIM == 3 && z >= F.nz)) continue;
        const int q = ((DIM == 3 ? lz + 1 : 0) * VY + ly + 1) * VX + lx + 1;
        T sx = 0, sy = 0;
        int nf = 0;
        if (x > 0) { const T c = (x == F.nx - 1) ? T(2) : T(1); sx += c * sv_[q - 1].x; sy += c * sv_[q - 1].y; } else ++nf;
        if (x < F.nx - 1) { const T c = (x == 0) ? T(2) : T(1); sx += c * sv_[q + 1].x; sy += c * sv_[q + 1].y; } else ++nf;
        if (y > 0) { const T c = (y == F.ny - 1) ? T(2) : T(1); sx += c * sv_[q - VX].x; sy += c * sv_[q - VX].y; } else ++nf;
        if (y < F.ny - 1) { const T c = (y == 0) ? T(2) : T(1); sx += c * sv_[q + VX].x; sy += c * sv_[q + VX].y; } else ++nf;
        if (DIM == 3) {
            if (z > 0) { const T c = (z == F.nz - 1) ? T(2) : T(1); sx += c * sv_[q - VX * VY].x; sy += c * sv_[q - VX * VY].y; } else ++nf;
            if (z < F.nz - 1) { const T c = (z == 0) ? T(2) : T(1); sx += c * sv_[q + VX * VY].x; sy += c * sv_[q + VX * VY].y; } else ++nf;
        }
        const size_t p = (size_t)z * fxy + (size_t)y * F.nx + x;
        T dre, dim_;
        diag_of<T>(F, s, F.w[p], nf, DIM, dre, dim_);
        const C vp = sv_[q];
        const C bp = cvt<C>(b[p]);
        const T rx = bp.x - (dre * vp.x - dim_ * vp.y - F.inv_h2 * sx);
        const T ry = bp.y - (dre * vp.y + dim_ * vp.x - F.inv_h2 * sy);
        const T inv = wj / (dre * dre + dim_ * dim_);
        C o;
        o.x = vp.x + (rx * dre + ry * dim_) * inv;
        o.y = vp.y + (ry * dre - rx * dim_) * inv;
        uout[p] = o;
    }
}

template <int DIM> constexpr size_t down_smem(size_t csz) {
    using TL = Tile<DIM>;
    constexpr int UX = 2 * TL::CX + 3, UY = 2 * TL::CY + 3, UZ = DIM == 3 ? 2 * TL::CZ + 3 : 1;
    constexpr int RX = UX - 2, RY = UY - 2, RZ = DIM == 3 ? UZ - 2 : 1;
    return csz * (2 * UX * UY * UZ + RX * RY * RZ);
}
template <int DIM> constexpr size_t up_smem(size_t csz) {
    using TL = Tile<DIM>;
    constexpr int VX = TL::FX + 2, VY = TL::FY + 2, VZ = DIM == 3 ? TL::FZ + 2 : 1;
    constexpr int EX = TL::FX / 2 + 2, EY = TL::FY / 2 + 2, EZ = DIM == 3 ? TL::FZ / 2 + 2 : 1;
    return csz * (VX * VY * VZ + EX * EY * EZ);
}

template <typename T, typename CB, int DIM>
void down_impl(const LevelView<T> &F, const LevelView<T> &Cv, OpShift<T> s, T wj, const CB *b,
               size_t sb, cplx_t<T> *u, size_t su, cplx_t<T> *bc, size_t sbc, int nb,
               const int *active, cudaStream_t st) {
    using TL = Tile<DIM>;
    const size_t sm = down_smem<DIM>(sizeof(cplx_t<T>));
    const int gz = (Cv.nz + TL::CZ - 1) / TL::CZ;
    dim3 g((Cv.nx + TL::CX - 1) / TL::CX, (Cv.ny + TL::CY - 1) / TL::CY, gz * nb);
    k_down<T, CB, DIM><<<g, 256, sm, st>>>(F, Cv, s, wj, b, sb, u, su, bc, sbc, active);
}

template <typename T, typename CB, int DIM>
void up_impl(const LevelView<T> &F, const LevelView<T> &Cv, OpShift<T> s, T wj,
             const cplx_t<T> *uin, size_t sin, const cplx_t<T> *ec, size_t sec, const CB *b,
             size_t sb, cplx_t<T> *uout, size_t sout, int nb, const int *active, cudaStream_t st) {
    using TL = Tile<DIM>;
    const size_t sm = up_smem<DIM>(sizeof(cplx_t<T>));
    const int gz = (F.nz + TL::FZ - 1) / TL::FZ;
    dim3 g((F.nx + TL::FX - 1) / TL::FX, (F.ny + TL::FY - 1) / TL::FY, gz * nb);
    k_up<T, CB, DIM><<<g, 256, sm, st>>>(F, Cv, s, wj, uin, sin, ec, sec, b, sb, uout, sout, active);
}

template <typename T, typename CB, int DIM> void set_attr() {
    cudaFuncSetAttribute(k_down<T, CB, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)down_smem<DIM>(sizeof(cplx_t<T>)));
    cudaFuncSetAttribute(k_up<T, CB, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)up_smem<DIM>(sizeof(cplx_t<T>)));
}

}  // namespace

void prepare_vfused() {
    static bool done = false;
    if (done) return;
    set_attr<double, double2, 2>();
    set_attr<double, double2, 3>();
    set_attr<float, float2, 2>();
    set_attr<float, float2, 3>();
    set_attr<float, double2, 2>();
    set_attr<float, double2, 3>();
    set_attr<float, float4, 2>();
    set_attr<float, float4, 3>();
    done = true;
}

template <typename T, typename CB>
void launch_vdown(const LevelView<T> &F, const LevelView<T> &Cv, OpShift<T> s, T wj, const CB *b,
                  size_t sb, cplx_t<T> *u, size_t su, cplx_t<T> *bc, size_t sbc, int nb,
                  const int *active, cudaStream_t st) {
    prof_begin(st);
    if (F.dim == 2) down_impl<T, CB, 2>(F, Cv, s, wj, b, sb, u, su, bc, sbc, nb, active, st);
    else down_impl<T, CB, 3>(F, Cv, s, wj, b, sb, u, su, bc, sbc, nb, active, st);
    count_launch();
    if (prof_on()) {
        const double nf = (double)F.nx * F.ny * F.nz * nb, nc = (double)Cv.nx * Cv.ny * Cv.nz * nb;
        prof_end(sizeof(T) == 8 ? "vdown_f64" : "vdown_f32", st,
                 nf * (sizeof(CB) + sizeof(T) + sizeof(cplx_t<T>)) + nc * sizeof(cplx_t<T>),
                 sizeof(T) == 8 ? nf * 40.0 : 0.0);
    }
}

template <typename T, typename CB>
void launch_vup(const LevelView<T> &F, const LevelView<T> &Cv, OpShift<T> s, T wj,
                const cplx_t<T> *uin, size_t sin, const cplx_t<T> *ec, size_t sec, const CB *b,
                size_t sb, cplx_t<T> *uout, size_t sout, int nb, const int *active,
                cudaStream_t st) {
    prof_begin(st);
    if (F.dim == 2) up_impl<T, CB, 2>(F, Cv, s, wj, uin, sin, ec, sec, b, sb, uout, sout, nb, active, st);
    else up_impl<T, CB, 3>(F, Cv, s, wj, uin, sin, ec, sec, b, sb, uout, sout, nb, active, st);
    count_launch();
    if (prof_on()) {
        const double nf = (double)F.nx * F.ny * F.nz * nb, nc = (double)Cv.nx * Cv.ny * Cv.nz * nb;
        prof_end(sizeof(T) == 8 ? "vup_f64" : "vup_f32", st,
                 nf * (2.0 * sizeof(cplx_t<T>) + sizeof(CB) + sizeof(T)) + nc * sizeof(cplx_t<T>),
                 sizeof(T) == 8 ? nf * 44.0 : 0.0);
    }
}

#define HELM_INST_V(T, CB)                                                                      \
    template void launch_vdown<T, CB>(const LevelView<T> &, const LevelView<T> &, OpShift<T>, T, \
                                      const CB *, size_t, cplx_t<T> *, size_t, cplx_t<T> *,     \
                                      size_t, int, const int *, cudaStream_t);                  \
    template void launch_vup<T, CB>(const LevelView<T> &, const LevelView<T> &, OpShift<T>, T,   \
                                    const cplx_t<T> *, size_t, const cplx_t<T> *, size_t,       \
                                    const CB *, size_t, cplx_t<T> *, size_t, int, const int *,  \
                                    cudaStream_t);
HELM_INST_V(double, double2)
HELM_INST_V(float, float2)
HELM_INST_V(float, double2)
HELM_INST_V(float, float4)
#undef HELM_INST_V

}  // namespace helm
