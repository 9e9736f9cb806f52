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
// Both sweeps are written with the inverse diagonal alone, precomputed per
// level (no division, square root or boundary test per node):
//   first sweep from 0:  u  = wj D^-1 b,   r = (1 - wj) b + (1/h^2) sum c u_nbr
//   sweep from v:        v' = (1 - wj) v + wj D^-1 (b + (1/h^2) sum c v_nbr)
// (M = D - (1/h^2) sum c (.)_nbr, so b - M v = b + (1/h^2) sum c v_nbr - D v.)
//
// The right-hand side type CB may be wider than the level's arithmetic
// (complex128 basis vector feeding a complex64 V-cycle): the conversion is
// fused into the loads.
#include "helm_internal.cuh"

#include <tuple>
#include <utility>

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

template <typename C> __device__ __forceinline__ C from_d2(double2 a);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 a) {
    return make_float2(__double2float_rn(a.x), __double2float_rn(a.y));
}

template <typename C>
__global__ void k_make_dinv(LevelView<double> L, OpShift<double> s, C *__restrict__ dinv) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(p % L.nx), y = (int)((p / L.nx) % L.ny), z = (int)(p / ((size_t)L.nx * L.ny));
        int nf = (x == 0) + (x == L.nx - 1);
        if (L.dim >= 2) nf += (y == 0) + (y == L.ny - 1);
        if (L.dim == 3) nf += (z == 0) + (z == L.nz - 1);
        double dre, dim_;
        diag_of<double>(L, s, L.w[p], nf, L.dim, dre, dim_);
        const double den = dre * dre + dim_ * dim_;
        dinv[p] = from_d2<C>(make_double2(dre / den, -dim_ / den));
    }
}

// Tile shapes. A down shape is the block's tile of coarse nodes (SX x SY x SZ;
// the block covers twice that on the fine level plus a halo), an up shape the
// block's tile of fine nodes (even extents); NT is the block size. Index 0 of
// each list is the default; helm_autotune times every shape on each level and
// keeps the fastest. The arithmetic per node does not depend on the shape, so
// all shapes give bitwise identical results.
template <int X, int Y, int Z, int NT_> struct Shape {
    static constexpr int SX = X, SY = Y, SZ = Z, NT = NT_;
};
template <int DIM> struct Shapes;
template <> struct Shapes<2> {
    using Down = std::tuple<Shape<16, 8, 1, 256>, Shape<8, 8, 1, 128>, Shape<8, 4, 1, 128>,
                            Shape<32, 4, 1, 256>>;
    using Up = std::tuple<Shape<32, 8, 1, 256>, Shape<16, 16, 1, 256>, Shape<16, 8, 1, 128>,
                          Shape<64, 4, 1, 256>>;
};
template <> struct Shapes<3> {
    using Down = std::tuple<Shape<8, 4, 4, 256>, Shape<8, 4, 2, 128>, Shape<16, 4, 2, 256>>;
    using Up = std::tuple<Shape<32, 4, 4, 256>, Shape<16, 4, 4, 128>, Shape<32, 8, 2, 256>>;
};

template <typename T, typename CB, int DIM, typename TL>
__global__ void __launch_bounds__(TL::NT)
k_down(LevelView<T> F, LevelView<T> Cv, T wj, const CB *__restrict__ b, size_t sb,
       cplx_t<T> *__restrict__ u, size_t su, cplx_t<T> *__restrict__ bc, size_t sbc,
       const int *__restrict__ active) {
    using C = cplx_t<T>;
    const int r = blockIdx.z / ((Cv.nz + TL::SZ - 1) / TL::SZ);
    const int bz = blockIdx.z % ((Cv.nz + TL::SZ - 1) / TL::SZ);
    if (active && !active[r]) return;
    b += r * sb;
    u += r * su;
    bc += r * sbc;
    const int I0 = blockIdx.x * TL::SX, J0 = blockIdx.y * TL::SY, K0 = bz * TL::SZ;
    // u region: fine [2*I0-2, 2*I0+2*CX] per axis (2*CX+3 nodes); r region one node inside
    constexpr int UX = 2 * TL::SX + 3, UY = 2 * TL::SY + 3, UZ = DIM == 3 ? 2 * TL::SZ + 3 : 1;
    constexpr int RX = UX - 2, RY = UY - 2, RZ = DIM == 3 ? UZ - 2 : 1;
    extern __shared__ unsigned char smem_raw[];
    C *su_ = reinterpret_cast<C *>(smem_raw);
    C *sb_ = su_ + UX * UY * UZ;
    C *sr_ = sb_ + UX * UY * UZ;
    const int X0 = 2 * I0 - 2, Y0 = 2 * J0 - 2, Z0 = DIM == 3 ? 2 * K0 - 2 : 0;
    const size_t fxy = (size_t)F.nx * F.ny;
    // phase 1: b and u = wj b / d on the u region (in-range nodes). All of a
    // thread's loads are issued before any of them is used, so a block waits
    // on one memory latency, not one per node it owns.
    constexpr int NU = (UX * UY * UZ + TL::NT - 1) / TL::NT;
    CB bq[NU];
    C dq[NU];
#pragma unroll
    for (int k = 0; k < NU; ++k) {
        const int t = threadIdx.x + k * TL::NT;
        const int lx = t % UX, ly = (t / UX) % UY, lz = t / (UX * UY);
        const int x = X0 + lx, y = Y0 + ly, z = Z0 + lz;
        if (t < UX * UY * UZ && x >= 0 && x < F.nx && y >= 0 && y < F.ny &&
            (DIM != 3 || (z >= 0 && z < F.nz))) {
            const size_t p = (size_t)z * fxy + (size_t)y * F.nx + x;
            bq[k] = b[p];
            dq[k] = F.dinv[p];
        }
    }
#pragma unroll
    for (int k = 0; k < NU; ++k) {
        const int t = threadIdx.x + k * TL::NT;
        const int lx = t % UX, ly = (t / UX) % UY, lz = t / (UX * UY);
        const int x = X0 + lx, y = Y0 + ly, z = Z0 + lz;
        if (t >= UX * UY * UZ || x < 0 || x >= F.nx || y < 0 || y >= F.ny ||
            (DIM == 3 && (z < 0 || z >= F.nz)))
            continue;
        const C bp = cvt<C>(bq[k]);
        const C di = dq[k];
        C up;
        up.x = wj * (di.x * bp.x - di.y * bp.y);
        up.y = wj * (di.x * bp.y + di.y * bp.x);
        su_[t] = up;
        sb_[t] = bp;
        // owned fine nodes: [2*I0, 2*I0 + 2*CX) per axis
        if (lx >= 2 && lx < 2 + 2 * TL::SX && ly >= 2 && ly < 2 + 2 * TL::SY &&
            (DIM == 2 || (lz >= 2 && lz < 2 + 2 * TL::SZ)))
            u[(size_t)z * fxy + (size_t)y * F.nx + x] = up;
    }
    __syncthreads();
    // phase 2: r = (1 - wj) b + (1/h^2) sum c u_nbr on the r region (in-range nodes)
    for (int t = threadIdx.x; t < RX * RY * RZ; t += TL::NT) {
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
    for (int t = threadIdx.x; t < TL::SX * TL::SY * TL::SZ; t += TL::NT) {
        const int I = I0 + t % TL::SX, J = J0 + (t / TL::SX) % TL::SY,
                  K = K0 + (DIM == 3 ? t / (TL::SX * TL::SY) : 0);
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

template <typename T, typename CB, int DIM, typename TL>
__global__ void __launch_bounds__(TL::NT)
k_up(LevelView<T> F, LevelView<T> Cv, T wj, const cplx_t<T> *__restrict__ uin,
     size_t sin, const cplx_t<T> *__restrict__ ec, size_t sec, const CB *__restrict__ b, size_t sb,
     cplx_t<T> *__restrict__ uout, size_t sout, const int *__restrict__ active) {
    using C = cplx_t<T>;
    const int nzb = (F.nz + TL::SZ - 1) / TL::SZ;
    const int r = blockIdx.z / nzb;
    const int bz = blockIdx.z % nzb;
    if (active && !active[r]) return;
    uin += r * sin;
    ec += r * sec;
    b += r * sb;
    uout += r * sout;
    const int x0 = blockIdx.x * TL::SX, y0 = blockIdx.y * TL::SY, z0 = bz * TL::SZ;
    constexpr int VX = TL::SX + 2, VY = TL::SY + 2, VZ = DIM == 3 ? TL::SZ + 2 : 1;
    constexpr int EX = TL::SX / 2 + 2, EY = TL::SY / 2 + 2, EZ = DIM == 3 ? TL::SZ / 2 + 2 : 1;
    extern __shared__ unsigned char smem_raw[];
    C *sv_ = reinterpret_cast<C *>(smem_raw);
    C *se_ = sv_ + VX * VY * VZ;
    const int cx0 = x0 / 2 - 1, cy0 = y0 / 2 - 1, cz0 = DIM == 3 ? z0 / 2 - 1 : 0;
    const size_t cxy = (size_t)Cv.nx * Cv.ny, fxy = (size_t)F.nx * F.ny;
    // All global loads of the three phases are issued up front (coarse
    // correction, pre-smoothed iterate with its halo, and b and w of the owned
    // nodes), so a block waits on one memory latency instead of three.
    constexpr int NE = (EX * EY * EZ + TL::NT - 1) / TL::NT;
    constexpr int NV = (VX * VY * VZ + TL::NT - 1) / TL::NT;
    constexpr int NO = (TL::SX * TL::SY * TL::SZ + TL::NT - 1) / TL::NT;
    C eq[NE], uq[NV];
    CB bq[NO];
    C dq[NO];
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        const int t = threadIdx.x + k * TL::NT;
        const int X = cx0 + t % EX, Y = cy0 + (t / EX) % EY, Z = cz0 + (DIM == 3 ? t / (EX * EY) : 0);
        if (t < EX * EY * EZ && X >= 0 && X < Cv.nx && Y >= 0 && Y < Cv.ny &&
            (DIM != 3 || (Z >= 0 && Z < Cv.nz)))
            eq[k] = ec[(size_t)Z * cxy + (size_t)Y * Cv.nx + X];
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int t = threadIdx.x + k * TL::NT;
        const int x = x0 - 1 + t % VX, y = y0 - 1 + (t / VX) % VY,
                  z = DIM == 3 ? z0 - 1 + t / (VX * VY) : 0;
        if (t < VX * VY * VZ && x >= 0 && x < F.nx && y >= 0 && y < F.ny &&
            (DIM != 3 || (z >= 0 && z < F.nz)))
            uq[k] = uin[(size_t)z * fxy + (size_t)y * F.nx + x];
    }
#pragma unroll
    for (int k = 0; k < NO; ++k) {
        const int t = threadIdx.x + k * TL::NT;
        const int x = x0 + t % TL::SX, y = y0 + (t / TL::SX) % TL::SY,
                  z = DIM == 3 ? z0 + t / (TL::SX * TL::SY) : 0;
        if (t < TL::SX * TL::SY * TL::SZ && x < F.nx && y < F.ny && (DIM != 3 || z < F.nz)) {
            const size_t p = (size_t)z * fxy + (size_t)y * F.nx + x;
            bq[k] = b[p];
            dq[k] = F.dinv[p];
        }
    }
    // phase 1: coarse correction around the tile
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        const int t = threadIdx.x + k * TL::NT;
        if (t < EX * EY * EZ) se_[t] = eq[k];
    }
    __syncthreads();
    // phase 2: v = u + P e on the tile plus a one-node halo
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int t = threadIdx.x + k * TL::NT;
        const int x = x0 - 1 + t % VX, y = y0 - 1 + (t / VX) % VY,
                  z = DIM == 3 ? z0 - 1 + t / (VX * VY) : 0;
        if (t >= VX * VY * VZ || x < 0 || x >= F.nx || y < 0 || y >= F.ny ||
            (DIM == 3 && (z < 0 || z >= F.nz)))
            continue;
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
        C v = uq[k];
        v.x += wgt * px;
        v.y += wgt * py;
        sv_[t] = v;
    }
    __syncthreads();
    // phase 3: one damped-Jacobi sweep on the tile
#pragma unroll
    for (int k = 0; k < NO; ++k) {
        const int t = threadIdx.x + k * TL::NT;
        const int lx = t % TL::SX, ly = (t / TL::SX) % TL::SY, lz = DIM == 3 ? t / (TL::SX * TL::SY) : 0;
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        if (t >= TL::SX * TL::SY * TL::SZ || x >= F.nx || y >= F.ny || (DIM == 3 && z >= F.nz)) continue;
        const int q = ((DIM == 3 ? lz + 1 : 0) * VY + ly + 1) * VX + lx + 1;
        T sx = 0, sy = 0;
        if (x > 0) { const T c = (x == F.nx - 1) ? T(2) : T(1); sx += c * sv_[q - 1].x; sy += c * sv_[q - 1].y; }
        if (x < F.nx - 1) { const T c = (x == 0) ? T(2) : T(1); sx += c * sv_[q + 1].x; sy += c * sv_[q + 1].y; }
        if (y > 0) { const T c = (y == F.ny - 1) ? T(2) : T(1); sx += c * sv_[q - VX].x; sy += c * sv_[q - VX].y; }
        if (y < F.ny - 1) { const T c = (y == 0) ? T(2) : T(1); sx += c * sv_[q + VX].x; sy += c * sv_[q + VX].y; }
        if (DIM == 3) {
            if (z > 0) { const T c = (z == F.nz - 1) ? T(2) : T(1); sx += c * sv_[q - VX * VY].x; sy += c * sv_[q - VX * VY].y; }
            if (z < F.nz - 1) { const T c = (z == 0) ? T(2) : T(1); sx += c * sv_[q + VX * VY].x; sy += c * sv_[q + VX * VY].y; }
        }
        const size_t p = (size_t)z * fxy + (size_t)y * F.nx + x;
        const C vp = sv_[q];
        const C bp = cvt<C>(bq[k]);
        const C di = dq[k];
        const T gx = bp.x + F.inv_h2 * sx, gy = bp.y + F.inv_h2 * sy;
        const T omw = T(1) - wj;
        C o;
        o.x = omw * vp.x + wj * (di.x * gx - di.y * gy);
        o.y = omw * vp.y + wj * (di.x * gy + di.y * gx);
        uout[p] = o;
    }
}

template <int DIM, typename TL> constexpr size_t down_smem(size_t csz) {
    constexpr int UX = 2 * TL::SX + 3, UY = 2 * TL::SY + 3, UZ = DIM == 3 ? 2 * TL::SZ + 3 : 1;
    constexpr int RX = UX - 2, RY = UY - 2, RZ = DIM == 3 ? UZ - 2 : 1;
    return csz * (2 * UX * UY * UZ + RX * RY * RZ);
}
template <int DIM, typename TL> constexpr size_t up_smem(size_t csz) {
    constexpr int VX = TL::SX + 2, VY = TL::SY + 2, VZ = DIM == 3 ? TL::SZ + 2 : 1;
    constexpr int EX = TL::SX / 2 + 2, EY = TL::SY / 2 + 2, EZ = DIM == 3 ? TL::SZ / 2 + 2 : 1;
    return csz * (VX * VY * VZ + EX * EY * EZ);
}

template <typename T, typename CB, int DIM, typename TL>
void down_impl(const LevelView<T> &F, const LevelView<T> &Cv, T wj, const CB *b,
               size_t sb, cplx_t<T> *u, size_t su, cplx_t<T> *bc, size_t sbc, int nb,
               const int *active, cudaStream_t st) {
    const size_t sm = down_smem<DIM, TL>(sizeof(cplx_t<T>));
    const int gz = (Cv.nz + TL::SZ - 1) / TL::SZ;
    dim3 g((Cv.nx + TL::SX - 1) / TL::SX, (Cv.ny + TL::SY - 1) / TL::SY, gz * nb);
    k_down<T, CB, DIM, TL><<<g, TL::NT, sm, st>>>(F, Cv, wj, b, sb, u, su, bc, sbc, active);
}

template <typename T, typename CB, int DIM, typename TL>
void up_impl(const LevelView<T> &F, const LevelView<T> &Cv, T wj,
             const cplx_t<T> *uin, size_t sin, const cplx_t<T> *ec, size_t sec, const CB *b,
             size_t sb, cplx_t<T> *uout, size_t sout, int nb, const int *active, cudaStream_t st) {
    const size_t sm = up_smem<DIM, TL>(sizeof(cplx_t<T>));
    const int gz = (F.nz + TL::SZ - 1) / TL::SZ;
    dim3 g((F.nx + TL::SX - 1) / TL::SX, (F.ny + TL::SY - 1) / TL::SY, gz * nb);
    k_up<T, CB, DIM, TL><<<g, TL::NT, sm, st>>>(F, Cv, wj, uin, sin, ec, sec, b, sb, uout, sout, active);
}

// shape index -> instantiation
template <typename T, typename CB, int DIM, size_t... I>
void down_sel(int shape, std::index_sequence<I...>, const LevelView<T> &F, const LevelView<T> &Cv,
              T wj, const CB *b, size_t sb, cplx_t<T> *u, size_t su, cplx_t<T> *bc, size_t sbc,
              int nb, const int *active, cudaStream_t st) {
    ((shape == (int)I
          ? down_impl<T, CB, DIM, std::tuple_element_t<I, typename Shapes<DIM>::Down>>(
                F, Cv, wj, b, sb, u, su, bc, sbc, nb, active, st)
          : void()),
     ...);
}
template <typename T, typename CB, int DIM, size_t... I>
void up_sel(int shape, std::index_sequence<I...>, const LevelView<T> &F, const LevelView<T> &Cv,
            T wj, const cplx_t<T> *uin, size_t sin, const cplx_t<T> *ec, size_t sec, const CB *b,
            size_t sb, cplx_t<T> *uout, size_t sout, int nb, const int *active, cudaStream_t st) {
    ((shape == (int)I
          ? up_impl<T, CB, DIM, std::tuple_element_t<I, typename Shapes<DIM>::Up>>(
                F, Cv, wj, uin, sin, ec, sec, b, sb, uout, sout, nb, active, st)
          : void()),
     ...);
}

template <typename T, typename CB, int DIM, size_t... I>
void set_attr_all(std::index_sequence<I...>) {
    (cudaFuncSetAttribute(k_down<T, CB, DIM, std::tuple_element_t<I, typename Shapes<DIM>::Down>>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)down_smem<DIM, std::tuple_element_t<I, typename Shapes<DIM>::Down>>(
                              sizeof(cplx_t<T>))),
     ...);
    (cudaFuncSetAttribute(k_up<T, CB, DIM, std::tuple_element_t<I, typename Shapes<DIM>::Up>>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)up_smem<DIM, std::tuple_element_t<I, typename Shapes<DIM>::Up>>(
                              sizeof(cplx_t<T>))),
     ...);
}

template <int DIM> constexpr size_t n_down() { return std::tuple_size<typename Shapes<DIM>::Down>::value; }
template <int DIM> constexpr size_t n_up() { return std::tuple_size<typename Shapes<DIM>::Up>::value; }

template <typename T, typename CB> void set_attr() {
    static_assert(n_down<2>() == n_up<2>() && n_down<3>() == n_up<3>(), "paired shape lists");
    set_attr_all<T, CB, 2>(std::make_index_sequence<n_down<2>()>{});
    set_attr_all<T, CB, 3>(std::make_index_sequence<n_down<3>()>{});
}

template <int DIM, size_t... I>
void shape_info(bool up, int shape, int ext[3], int *threads, std::index_sequence<I...>) {
    auto one = [&](auto tag) {
        using S = decltype(tag);
        ext[0] = S::SX;
        ext[1] = S::SY;
        ext[2] = S::SZ;
        *threads = S::NT;
    };
    if (up)
        ((shape == (int)I ? one(std::tuple_element_t<I, typename Shapes<DIM>::Up>{}) : void()), ...);
    else
        ((shape == (int)I ? one(std::tuple_element_t<I, typename Shapes<DIM>::Down>{}) : void()), ...);
}

}  // namespace

template <typename C>
void launch_make_dinv(const LevelView<double> &L, OpShift<double> s, C *dinv, cudaStream_t st) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    const size_t b = (N + 255) / 256;
    const int nb = (int)(b < 4096 ? (b ? b : 1) : 4096);
    k_make_dinv<C><<<nb, 256, 0, st>>>(L, s, dinv);
    count_launch();
}
template void launch_make_dinv<double2>(const LevelView<double> &, OpShift<double>, double2 *, cudaStream_t);
template void launch_make_dinv<float2>(const LevelView<double> &, OpShift<double>, float2 *, cudaStream_t);

int num_tile_shapes(int dim) {
    return dim == 2 ? (int)n_down<2>() : dim == 3 ? (int)n_down<3>() : 0;
}

bool tile_shape(int dim, int kernel, int shape, int ext[3], int *threads) {
    if (shape < 0 || shape >= num_tile_shapes(dim) || (kernel != 0 && kernel != 1)) return false;
    if (dim == 2) shape_info<2>(kernel == 1, shape, ext, threads, std::make_index_sequence<n_down<2>()>{});
    else shape_info<3>(kernel == 1, shape, ext, threads, std::make_index_sequence<n_down<3>()>{});
    return true;
}

int auto_tile_shape(int dim, int kernel, const int fine[3], int nb) {
    const int ns = num_tile_shapes(dim);
    const int cn[3] = {(fine[0] + 1) / 2, (fine[1] + 1) / 2, (fine[2] + 1) / 2};
    const int *ext_of = kernel == 0 ? cn : fine;   // down tiles cover coarse nodes, up tiles fine
    long long best_blocks = -1;
    int best = 0;
    for (int sh = 0; sh < ns; ++sh) {
        int e[3], nt;
        tile_shape(dim, kernel, sh, e, &nt);
        long long blocks = (long long)nb * ((ext_of[0] + e[0] - 1) / e[0]) * ((ext_of[1] + e[1] - 1) / e[1]);
        if (dim == 3) blocks *= (ext_of[2] + e[2] - 1) / e[2];
        if (blocks >= 2 * 152) return sh;
        if (blocks > best_blocks) {
            best_blocks = blocks;
            best = sh;
        }
    }
    return best;
}

void prepare_vfused() {
    static bool done = false;
    if (done) return;
    set_attr<double, double2>();
    set_attr<float, float2>();
    set_attr<float, double2>();
    set_attr<float, float4>();
    done = true;
}

template <typename T, typename CB>
void launch_vdown(const LevelView<T> &F, const LevelView<T> &Cv, T wj, const CB *b,
                  size_t sb, cplx_t<T> *u, size_t su, cplx_t<T> *bc, size_t sbc, int nb,
                  const int *active, cudaStream_t st, int shape) {
    prof_begin(st);
    if (F.dim == 2)
        down_sel<T, CB, 2>(shape, std::make_index_sequence<n_down<2>()>{}, F, Cv, wj, b, sb, u, su,
                           bc, sbc, nb, active, st);
    else
        down_sel<T, CB, 3>(shape, std::make_index_sequence<n_down<3>()>{}, F, Cv, wj, b, sb, u, su,
                           bc, sbc, nb, active, st);
    count_launch();
    if (prof_on()) {
        const double nf = (double)F.nx * F.ny * F.nz * nb, nc = (double)Cv.nx * Cv.ny * Cv.nz * nb;
        prof_end(sizeof(T) == 8 ? "vdown_f64" : "vdown_f32", st,
                 nf * (sizeof(CB) + 2.0 * sizeof(cplx_t<T>)) + nc * sizeof(cplx_t<T>),
                 sizeof(T) == 8 ? nf * 40.0 : 0.0);
    }
}

template <typename T, typename CB>
void launch_vup(const LevelView<T> &F, const LevelView<T> &Cv, T wj,
                const cplx_t<T> *uin, size_t sin, const cplx_t<T> *ec, size_t sec, const CB *b,
                size_t sb, cplx_t<T> *uout, size_t sout, int nb, const int *active,
                cudaStream_t st, int shape) {
    prof_begin(st);
    if (F.dim == 2)
        up_sel<T, CB, 2>(shape, std::make_index_sequence<n_up<2>()>{}, F, Cv, wj, uin, sin, ec, sec, b,
                         sb, uout, sout, nb, active, st);
    else
        up_sel<T, CB, 3>(shape, std::make_index_sequence<n_up<3>()>{}, F, Cv, wj, uin, sin, ec, sec, b,
                         sb, uout, sout, nb, active, st);
    count_launch();
    if (prof_on()) {
        const double nf = (double)F.nx * F.ny * F.nz * nb, nc = (double)Cv.nx * Cv.ny * Cv.nz * nb;
        prof_end(sizeof(T) == 8 ? "vup_f64" : "vup_f32", st,
                 nf * (3.0 * sizeof(cplx_t<T>) + sizeof(CB)) + nc * sizeof(cplx_t<T>),
                 sizeof(T) == 8 ? nf * 44.0 : 0.0);
    }
}

#define HELM_INST_V(T, CB)                                                                      \
    template void launch_vdown<T, CB>(const LevelView<T> &, const LevelView<T> &, T,             \
                                      const CB *, size_t, cplx_t<T> *, size_t, cplx_t<T> *,     \
                                      size_t, int, const int *, cudaStream_t, int);             \
    template void launch_vup<T, CB>(const LevelView<T> &, const LevelView<T> &, T,               \
                                    const cplx_t<T> *, size_t, const cplx_t<T> *, size_t,       \
                                    const CB *, size_t, cplx_t<T> *, size_t, int, const int *,  \
                                    cudaStream_t, int);
HELM_INST_V(double, double2)
HELM_INST_V(float, float2)
HELM_INST_V(float, double2)
HELM_INST_V(float, float4)
#undef HELM_INST_V

}  // namespace helm
