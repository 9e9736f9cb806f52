// Fused V(1,1) multigrid kernels for 2D and 3D levels (Eq. 6 operator M):
// the templates. vfused.cu holds the shape queries, the inverse diagonal and
// the one-time set-up; vfused_*.cu instantiate the kernels for one
// (arithmetic, right-hand side) type pair each, so the pairs compile in
// parallel.
//
// down: from the level's right-hand side b, one kernel computes
//         u  = wj D^-1 b                          (first Jacobi sweep from 0)
//         r  = b - M u = (1 - wj) b + (1/h^2) sum_nbr c u_nbr
//         bc = full-weighting restriction of r    (mirrored outside nodes)
//       and writes u (the pre-smoothed iterate) and bc (the coarse
//       right-hand side).
// up:   from the pre-smoothed u, the coarse correction e and b, one kernel
//       computes v = u + P e (multilinear prolongation) and writes one
//       damped-Jacobi sweep of v. Up and down never read what they write (u
//       comes from the level's scratch vector, the result goes to the
//       iterate).
//
// In both kernels a block owns a tile of coarse nodes, one thread per coarse
// node, and each thread computes the values of that node's 2^d fine
// children; the tile's fine footprint plus a halo (two fine nodes below,
// one above for down; one on each side for up) is staged in shared memory,
// and the halo nodes are shared out among the block's threads, so every fine
// value is computed once per block with no per-node index search.
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
#pragma once
#include "helm_internal.cuh"

#include <tuple>
#include <type_traits>
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

// Explicit fused multiply-adds: a node's value is computed in the block that
// owns it and again as halo in a neighbouring block, so the arithmetic must
// not depend on how the compiler contracts a*b + c at each site.
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ int mirror(int i, int n) {
    return i < 0 ? -i : (i > n - 1 ? 2 * (n - 1) - i : i);
}
template <bool INT> __device__ __forceinline__ int mirror_if(int i, int n) {
    return INT ? i : mirror(i, n);
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

// Tile shapes: a block owns a tile of SX x SY x SZ coarse nodes, one thread
// per coarse node (NT = SX SY SZ threads), and each thread owns the node's
// fine children (2I + {0,1}, 2J + {0,1}, 2K + {0,1}), so a tile covers twice
// its extent on the fine level. Index 0 of each list is the first candidate
// of the automatic choice; helm_autotune times every shape on each level and
// keeps the fastest. The arithmetic per node does not depend on the shape, so
// all shapes give bitwise identical results.
// QP threads share a coarse node's children (QP = 1: one thread computes all
// 2^d children; QP = 2^d: one thread per fine node, for small levels where
// latency rather than issue rate bounds the kernel).
// RB right-hand sides per block: the block's threads keep the positions,
// boundary tests and D^-1 of their nodes once and apply them to RB
// right-hand sides (RB boxes in shared memory); a batch's last block may
// hold fewer.
template <int X, int Y, int Z, int NT_, int QP_, int RB_ = 1> struct Shape {
    static constexpr int SX = X, SY = Y, SZ = Z, NT = NT_, QP = QP_, RB = RB_;
    static constexpr bool MARCH = false;
    static_assert(X * Y * Z * QP_ == NT_, "QP threads per coarse node");
};
// 3D down kernel that marches along z: a block takes X x Y coarse nodes in x, y
// and KC consecutive coarse planes, one thread per coarse (x, y) node, and
// walks the fine planes in order with rings of planes in shared memory.
template <int X, int Y, int KC> struct ZShape {
    static constexpr int SX = X, SY = Y, SZ = KC, NT = X * Y, QP = 1, RB = 1;
    static constexpr bool MARCH = true;
};
template <int DIM> struct Shapes;
template <> struct Shapes<2> {
    using Down = std::tuple<Shape<16, 16, 1, 256, 1>, Shape<32, 8, 1, 256, 1>, Shape<16, 8, 1, 128, 1>,
                            Shape<8, 8, 1, 256, 4>, Shape<8, 4, 1, 128, 4>, Shape<4, 4, 1, 64, 4>,
                            Shape<8, 4, 1, 128, 4, 2>, Shape<8, 4, 1, 128, 4, 4>, Shape<16, 8, 1, 128, 1, 2>,
                            Shape<4, 4, 1, 64, 4, 4>>;
    using Up = Down;
};
template <> struct Shapes<3> {
    using Down = std::tuple<Shape<8, 4, 4, 128, 1>, Shape<8, 8, 2, 128, 1>, Shape<4, 4, 4, 64, 1>,
                            Shape<4, 4, 2, 256, 8>, Shape<8, 4, 4, 256, 2>, Shape<8, 8, 2, 256, 2>,
                            Shape<8, 4, 4, 512, 4>, Shape<8, 8, 4, 512, 2>, ZShape<16, 8, 16>>;
    using Up = std::tuple<Shape<8, 4, 4, 128, 1>, Shape<8, 8, 2, 128, 1>, Shape<4, 4, 4, 64, 1>,
                          Shape<4, 4, 2, 256, 8>, Shape<8, 4, 4, 256, 2>, Shape<8, 8, 2, 256, 2>,
                          Shape<8, 4, 4, 512, 4>, Shape<8, 8, 4, 512, 2>, Shape<4, 4, 4, 128, 2>>;
};

// Halo shells. A block's local box has U = (UX, UY, UZ) nodes per axis; its
// threads own the interior [L, U - H) of every axis, and the shell (the
// first L and last H nodes of any axis) is shared out round-robin. shell_pos
// maps a shell index to local coordinates: whole z-planes first (3D), then
// y-rows, then x-columns of the remaining rows.
template <int DIM, int UX, int UY, int UZ, int L, int H> __host__ __device__ constexpr int shell_count() {
    return DIM == 3 ? UX * UY * UZ - (UX - L - H) * (UY - L - H) * (UZ - L - H)
                    : UX * UY - (UX - L - H) * (UY - L - H);
}

template <int DIM, int UX, int UY, int UZ, int L, int H>
__device__ __forceinline__ void shell_pos(int h, int &lx, int &ly, int &lz) {
    constexpr int S = L + H;
    int zlo = 0, zn = 1;
    if (DIM == 3) {
        constexpr int A = S * UX * UY;
        if (h < A) {
            const int s = h / (UX * UY), rem = h % (UX * UY);
            lz = s < L ? s : UZ - H + (s - L);
            ly = rem / UX;
            lx = rem % UX;
            return;
        }
        h -= A;
        zlo = L;
        zn = UZ - S;
    } else {
        lz = 0;
    }
    const int B = S * UX * zn;
    if (h < B) {
        const int s = h / (UX * zn), rem = h % (UX * zn);
        ly = s < L ? s : UY - H + (s - L);
        lz = zlo + rem / UX;
        lx = rem % UX;
        return;
    }
    h -= B;
    constexpr int NYI = UY - S;
    const int s = h / (NYI * zn), rem = h % (NYI * zn);
    lx = s < L ? s : UX - H + (s - L);
    ly = L + rem % NYI;
    lz = zlo + rem / NYI;
}

// INT: the block's whole box lies strictly inside the level, so no node of it
// needs a boundary test, a doubled neighbour or a mirrored restriction point
// (the same arithmetic as the general body on those nodes).
// SC (complex64 basis, level 0): b is the double-single w of the Arnoldi
// step (CB = float4) and sc the per-right-hand-side scale 1/||w|| as float
// hi + lo; the kernel uses v = w (sc.x + sc.y) rounded to complex64 (the
// arithmetic of k_scale_c64) and writes v of its own nodes to vout.
__device__ __forceinline__ float2 scaled_c64(float4 x, float2 s) {
    return make_float2(fmaf(x.x, s.x, fmaf(x.x, s.y, x.y * s.x)), fmaf(x.z, s.x, fmaf(x.z, s.y, x.w * s.x)));
}

template <typename T, typename CB, int DIM, typename TL, bool INT, bool SC = false>
__device__ __forceinline__ void down_tile(const LevelView<T> &F, const LevelView<T> &Cv, T wj,
                                          const CB *__restrict__ b, size_t sb,
                                          cplx_t<T> *__restrict__ u, size_t su,
                                          cplx_t<T> *__restrict__ bc, size_t sbc, int nb,
                                          const int *__restrict__ active, const float2 *__restrict__ sc = nullptr,
                                          float2 *__restrict__ vout = nullptr, size_t svout = 0) {
    using C = cplx_t<T>;
    static_assert(!SC || (std::is_same<CB, float4>::value && std::is_same<C, float2>::value),
                  "the scaled input is the double-single w of the complex64 basis");
    constexpr int SX = TL::SX, SY = TL::SY, SZ = DIM == 3 ? TL::SZ : 1;
    // local box of u: fine [2 I0 - 2, 2 I0 + 2 SX] per axis; own children at [2, U - 1)
    constexpr int UX = 2 * SX + 3, UY = 2 * SY + 3, UZ = DIM == 3 ? 2 * SZ + 3 : 1;
    constexpr int BOX = UX * UY * UZ;
    constexpr int NQ = DIM == 3 ? 8 : 4;
    constexpr int NH = shell_count<DIM, UX, UY, UZ, 2, 1>();
    // r is needed on [2 I0 - 1, 2 I0 + 2 SX - 1]: local [1, U - 1), own part [2, U - 1)
    constexpr int RX = UX - 2, RY = UY - 2, RZ = DIM == 3 ? UZ - 2 : 1;
    constexpr int NR = shell_count<DIM, RX, RY, RZ, 1, 0>();
    constexpr int HP = (NH + TL::NT - 1) / TL::NT;
    constexpr int RB = TL::RB;                   // right-hand sides per block
    const int gz = DIM == 3 ? (Cv.nz + SZ - 1) / SZ : 1;
    const int r0 = (blockIdx.z / gz) * RB, bz = blockIdx.z % gz;
    bool on[RB];
    bool any = false;
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        on[k] = r0 + k < nb && (!active || active[r0 + k]);
        any = any || on[k];
    }
    if (!any) return;
    b += r0 * sb;
    u += r0 * su;
    bc += r0 * sbc;
    float2 scr[RB];
    if constexpr (SC) {
        vout += r0 * svout;
#pragma unroll
        for (int r = 0; r < RB; ++r) scr[r] = on[r] ? sc[r0 + r] : make_float2(0.f, 0.f);
    }
    // the right-hand side value of right-hand side r in the level's type
    auto cv = [&](int r, CB braw) -> C {
        if constexpr (SC) return scaled_c64(braw, scr[r]);
        else return cvt<C>(braw);
    };
    const int I0 = blockIdx.x * SX, J0 = blockIdx.y * SY, K0 = bz * SZ;
    const int X0 = 2 * I0 - 2, Y0 = 2 * J0 - 2, Z0 = DIM == 3 ? 2 * K0 - 2 : 0;
    constexpr int QP = TL::QP;
    constexpr int NQL = NQ / QP;                 // children per thread
    const int cn = threadIdx.x / QP, q0 = threadIdx.x % QP;
    const int tx = cn % SX, ty = (cn / SX) % SY, tz = DIM == 3 ? cn / (SX * SY) : 0;
    const size_t fxy = (size_t)F.nx * F.ny;
    extern __shared__ unsigned char smem_raw[];
    // per right-hand side k: u, b and r boxes at su_ + k BOX, sb_ + k BOX, sr_ + k BOX
    C *su_ = reinterpret_cast<C *>(smem_raw);
    C *sb_ = su_ + RB * BOX;
    C *sr_ = sb_ + RB * BOX;
    auto in_f = [&](int x, int y, int z) {
        return INT || (x >= 0 && x < F.nx && y >= 0 && y < F.ny && (DIM != 3 || (z >= 0 && z < F.nz)));
    };
    // loads first: own children, then this thread's share of the halo shell
    // (D^-1 once, b for every right-hand side)
    CB bq[RB][NQL], bh[RB][HP];
    C dq[NQL], dh[HP];
    size_t pq[NQL];
    bool iq[NQL];
#pragma unroll
    for (int k = 0; k < NQL; ++k) {
        const int q = q0 + k * QP;
        const int x = 2 * (I0 + tx) + (q & 1), y = 2 * (J0 + ty) + ((q >> 1) & 1),
                  z = DIM == 3 ? 2 * (K0 + tz) + (q >> 2) : 0;
        iq[k] = in_f(x, y, z);
        pq[k] = (size_t)z * fxy + (size_t)y * F.nx + x;
        if (iq[k]) {
            dq[k] = F.dinv[pq[k]];
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (on[r]) bq[r][k] = b[r * sb + pq[k]];
        }
    }
    int th[HP];   // local index of the thread's halo node, -1 if none
#pragma unroll
    for (int k = 0; k < HP; ++k) {
        const int hidx = threadIdx.x + k * TL::NT;
        th[k] = -1;
        if (hidx < NH) {
            int lx, ly, lz;
            shell_pos<DIM, UX, UY, UZ, 2, 1>(hidx, lx, ly, lz);
            const int x = X0 + lx, y = Y0 + ly, z = Z0 + lz;
            if (in_f(x, y, z)) {
                th[k] = (lz * UY + ly) * UX + lx;
                const size_t p = (size_t)z * fxy + (size_t)y * F.nx + x;
                dh[k] = F.dinv[p];
#pragma unroll
                for (int r = 0; r < RB; ++r)
                    if (on[r]) bh[r][k] = b[r * sb + p];
            }
        }
    }
    // u = wj D^-1 b (first Jacobi sweep from zero) on the whole box; b goes to
    // shared memory only for the halo (own children keep it in registers)
    auto put_u = [&](int r, int t, CB braw, C di, bool keep_b) {
        const C bp = cv(r, braw);
        C up;
        up.x = wj * fmaT(di.x, bp.x, -(di.y * bp.y));
        up.y = wj * fmaT(di.x, bp.y, di.y * bp.x);
        su_[r * BOX + t] = up;
        if (keep_b) sb_[r * BOX + t] = bp;
        return up;
    };
#pragma unroll
    for (int k = 0; k < HP; ++k)
        if (th[k] >= 0) {
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (on[r]) put_u(r, th[k], bh[r][k], dh[k], true);
        }
    // in interior 2D blocks with one thread per coarse node the thread keeps
    // its four children's u and r in registers: two of each child's four u
    // neighbours and four of the coarse node's nine restriction taps
    constexpr bool RREG = DIM == 2 && QP == 1 && INT;
    C uo[RB][RREG ? NQL : 1];
#pragma unroll
    for (int k = 0; k < NQL; ++k) {
        const int q = q0 + k * QP;
        const int x = 2 * (I0 + tx) + (q & 1), y = 2 * (J0 + ty) + ((q >> 1) & 1),
                  z = DIM == 3 ? 2 * (K0 + tz) + (q >> 2) : 0;
        if (iq[k]) {
            const int t = ((z - Z0) * UY + (y - Y0)) * UX + (x - X0);
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (on[r]) {
                    const C up = put_u(r, t, bq[r][k], dq[k], false);
                    u[r * su + pq[k]] = up;
                    if constexpr (SC) vout[r * svout + pq[k]] = cv(r, bq[r][k]);
                    if constexpr (RREG) uo[r][k] = up;
                }
        }
    }
    __syncthreads();
    // r = (1 - wj) b + (1/h^2) sum_nbr c u_nbr on the r box
    auto put_r = [&](int r, int lx, int ly, int lz, C bp) {
        const int x = X0 + lx, y = Y0 + ly, z = Z0 + lz;
        const C *sur = su_ + r * BOX;
        const int q = (lz * UY + ly) * UX + lx;
        T sx = 0, sy = 0;
        if (INT || x > 0) { const T c = (!INT && x == F.nx - 1) ? T(2) : T(1); sx = fmaT(c, sur[q - 1].x, sx); sy = fmaT(c, sur[q - 1].y, sy); }
        if (INT || x < F.nx - 1) { const T c = (!INT && x == 0) ? T(2) : T(1); sx = fmaT(c, sur[q + 1].x, sx); sy = fmaT(c, sur[q + 1].y, sy); }
        if (INT || y > 0) { const T c = (!INT && y == F.ny - 1) ? T(2) : T(1); sx = fmaT(c, sur[q - UX].x, sx); sy = fmaT(c, sur[q - UX].y, sy); }
        if (INT || y < F.ny - 1) { const T c = (!INT && y == 0) ? T(2) : T(1); sx = fmaT(c, sur[q + UX].x, sx); sy = fmaT(c, sur[q + UX].y, sy); }
        if (DIM == 3) {
            if (INT || z > 0) { const T c = (!INT && z == F.nz - 1) ? T(2) : T(1); sx = fmaT(c, sur[q - UX * UY].x, sx); sy = fmaT(c, sur[q - UX * UY].y, sy); }
            if (INT || z < F.nz - 1) { const T c = (!INT && z == 0) ? T(2) : T(1); sx = fmaT(c, sur[q + UX * UY].x, sx); sy = fmaT(c, sur[q + UX * UY].y, sy); }
        }
        const T omw = T(1) - wj;
        C o;
        o.x = fmaT(F.inv_h2, sx, omw * bp.x);
        o.y = fmaT(F.inv_h2, sy, omw * bp.y);
        sr_[r * BOX + q] = o;
        return o;
    };
    for (int hidx = threadIdx.x; hidx < NR; hidx += TL::NT) {
        int lx, ly, lz;
        shell_pos<DIM, RX, RY, RZ, 1, 0>(hidx, lx, ly, lz);
        ++lx;
        ++ly;
        if (DIM == 3) ++lz;
        if (in_f(X0 + lx, Y0 + ly, Z0 + lz)) {
            const int t = (lz * UY + ly) * UX + lx;
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (on[r]) put_r(r, lx, ly, lz, sb_[r * BOX + t]);
        }
    }
    C ro[RB][RREG ? NQL : 1];
#pragma unroll
    for (int k = 0; k < NQL; ++k) {
        const int q = q0 + k * QP;
        const int x = 2 * (I0 + tx) + (q & 1), y = 2 * (J0 + ty) + ((q >> 1) & 1),
                  z = DIM == 3 ? 2 * (K0 + tz) + (q >> 2) : 0;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            if (!on[r]) continue;
            if constexpr (RREG) {
                // child (cx, cy) = (k & 1, k >> 1); the same multiply-adds in the
                // same order as put_r (interior: every factor 1)
                const int cx = k & 1, cy = k >> 1;
                const int t = (y - Y0) * UX + (x - X0);
                const C *sur = su_ + r * BOX;
                const C wv = cx ? uo[r][k - 1] : sur[t - 1];
                const C ev = cx ? sur[t + 1] : uo[r][k + 1];
                const C sv = cy ? uo[r][k - 2] : sur[t - UX];
                const C nv = cy ? sur[t + UX] : uo[r][k + 2];
                T sx = 0, sy = 0;
                sx = fmaT(T(1), wv.x, sx); sy = fmaT(T(1), wv.y, sy);
                sx = fmaT(T(1), ev.x, sx); sy = fmaT(T(1), ev.y, sy);
                sx = fmaT(T(1), sv.x, sx); sy = fmaT(T(1), sv.y, sy);
                sx = fmaT(T(1), nv.x, sx); sy = fmaT(T(1), nv.y, sy);
                const C bp = cv(r, bq[r][k]);
                const T omw = T(1) - wj;
                C o;
                o.x = fmaT(F.inv_h2, sx, omw * bp.x);
                o.y = fmaT(F.inv_h2, sy, omw * bp.y);
                sr_[r * BOX + t] = o;
                ro[r][k] = o;
            } else if (iq[k]) {
                put_r(r, x - X0, y - Y0, z - Z0, cv(r, bq[r][k]));
            }
        }
    }
    __syncthreads();
    // full weighting, one coarse node per thread: threads 0 .. SX SY SZ - 1
    // (whole warps; r is in shared memory), outside nodes mirrored
    if (threadIdx.x >= SX * SY * SZ) return;
    const int rx = threadIdx.x % SX, ry = (threadIdx.x / SX) % SY, rz = DIM == 3 ? threadIdx.x / (SX * SY) : 0;
    const int I = I0 + rx, J = J0 + ry, K = K0 + rz;
    if (I >= Cv.nx || J >= Cv.ny || (DIM == 3 && K >= Cv.nz)) return;
    T ax[RB], ay[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) ax[r] = ay[r] = 0;
#pragma unroll
    for (int oz = (DIM == 3 ? -1 : 0); oz <= (DIM == 3 ? 1 : 0); ++oz) {
        const int lz = DIM == 3 ? mirror_if<INT>(2 * K + oz, F.nz) - Z0 : 0;
        const T wz = DIM == 3 ? (oz == 0 ? T(0.5) : T(0.25)) : T(1);
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy) {
            const int ly = mirror_if<INT>(2 * J + oy, F.ny) - Y0;
            const T wy = oy == 0 ? T(0.5) : T(0.25);
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
                const int lx = mirror_if<INT>(2 * I + ox, F.nx) - X0;
                const T wgt = (ox == 0 ? T(0.5) : T(0.25)) * wy * wz;
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    if (!on[r]) continue;
                    C v;
                    if constexpr (RREG) {
                        if (ox >= 0 && oy >= 0) v = ro[r][ox + 2 * oy];   // own child (2I + ox, 2J + oy)
                        else v = sr_[r * BOX + (lz * UY + ly) * UX + lx];
                    } else {
                        v = sr_[r * BOX + (lz * UY + ly) * UX + lx];
                    }
                    ax[r] = fmaT(wgt, v.x, ax[r]);
                    ay[r] = fmaT(wgt, v.y, ay[r]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
        if (on[r]) {
            C o;
            o.x = ax[r];
            o.y = ay[r];
            bc[r * sbc + (size_t)K * Cv.nx * Cv.ny + (size_t)J * Cv.nx + I] = o;
        }
}

template <typename T, typename CB, int DIM, typename TL, bool INT>
__device__ __forceinline__ void up_tile(const LevelView<T> &F, const LevelView<T> &Cv, T wj,
                                        const cplx_t<T> *__restrict__ uin, size_t sin,
                                        const cplx_t<T> *__restrict__ ec, size_t sec,
                                        const CB *__restrict__ b, size_t sb,
                                        cplx_t<T> *__restrict__ uout, size_t sout, int nb,
                                        const int *__restrict__ active) {
    using C = cplx_t<T>;
    constexpr int SX = TL::SX, SY = TL::SY, SZ = DIM == 3 ? TL::SZ : 1;
    // local box of v: fine [2 I0 - 1, 2 I0 + 2 SX] per axis; own children at [1, V - 1)
    constexpr int VX = 2 * SX + 2, VY = 2 * SY + 2, VZ = DIM == 3 ? 2 * SZ + 2 : 1;
    // coarse correction needed on [I0 - 1, I0 + SX]
    constexpr int EX = SX + 2, EY = SY + 2, EZ = DIM == 3 ? SZ + 2 : 1;
    constexpr int VBOX = VX * VY * VZ, EBOX = EX * EY * EZ;
    constexpr int NQ = DIM == 3 ? 8 : 4;
    constexpr int NH = shell_count<DIM, VX, VY, VZ, 1, 1>();
    constexpr int HP = (NH + TL::NT - 1) / TL::NT;
    constexpr int EP = (EBOX + TL::NT - 1) / TL::NT;
    constexpr int RB = TL::RB;                   // right-hand sides per block
    const int gz = DIM == 3 ? (Cv.nz + SZ - 1) / SZ : 1;
    const int r0 = (blockIdx.z / gz) * RB, bz = blockIdx.z % gz;
    bool on[RB];
    bool any = false;
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        on[k] = r0 + k < nb && (!active || active[r0 + k]);
        any = any || on[k];
    }
    if (!any) return;
    uin += r0 * sin;
    ec += r0 * sec;
    b += r0 * sb;
    uout += r0 * sout;
    const int I0 = blockIdx.x * SX, J0 = blockIdx.y * SY, K0 = bz * SZ;
    const int X0 = 2 * I0 - 1, Y0 = 2 * J0 - 1, Z0 = DIM == 3 ? 2 * K0 - 1 : 0;
    const int CX0 = I0 - 1, CY0 = J0 - 1, CZ0 = DIM == 3 ? K0 - 1 : 0;
    constexpr int QP = TL::QP;
    constexpr int NQL = NQ / QP;                 // children per thread
    const int cn = threadIdx.x / QP, q0 = threadIdx.x % QP;
    const int tx = cn % SX, ty = (cn / SX) % SY, tz = DIM == 3 ? cn / (SX * SY) : 0;
    const size_t fxy = (size_t)F.nx * F.ny, cxy = (size_t)Cv.nx * Cv.ny;
    extern __shared__ unsigned char smem_raw[];
    // per right-hand side r: the v box at sv_ + r VBOX, the coarse tile at se_ + r EBOX
    C *sv_ = reinterpret_cast<C *>(smem_raw);
    C *se_ = sv_ + RB * VBOX;
    auto in_f = [&](int x, int y, int z) {
        return INT || (x >= 0 && x < F.nx && y >= 0 && y < F.ny && (DIM != 3 || (z >= 0 && z < F.nz)));
    };
    // loads first: coarse correction tile, own children (u, b, D^-1 once), halo u
    C eq[RB][EP], uq[RB][NQL], dq[NQL], uh[RB][HP];
    CB bq[RB][NQL];
    size_t pq[NQL];
    bool iq[NQL];
#pragma unroll
    for (int k = 0; k < EP; ++k) {
        const int t = threadIdx.x + k * TL::NT;
        const int X = CX0 + t % EX, Y = CY0 + (t / EX) % EY, Z = CZ0 + (DIM == 3 ? t / (EX * EY) : 0);
        if (t < EBOX && X >= 0 && X < Cv.nx && Y >= 0 && Y < Cv.ny && (DIM != 3 || (Z >= 0 && Z < Cv.nz))) {
            const size_t pc = (size_t)Z * cxy + (size_t)Y * Cv.nx + X;
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (on[r]) eq[r][k] = ec[r * sec + pc];
        }
    }
#pragma unroll
    for (int k = 0; k < NQL; ++k) {
        const int q = q0 + k * QP;
        const int x = 2 * (I0 + tx) + (q & 1), y = 2 * (J0 + ty) + ((q >> 1) & 1),
                  z = DIM == 3 ? 2 * (K0 + tz) + (q >> 2) : 0;
        iq[k] = in_f(x, y, z);
        pq[k] = (size_t)z * fxy + (size_t)y * F.nx + x;
        if (iq[k]) {
            dq[k] = F.dinv[pq[k]];
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (on[r]) {
                    uq[r][k] = uin[r * sin + pq[k]];
                    bq[r][k] = b[r * sb + pq[k]];
                }
        }
    }
    int lh[HP][3];   // local coordinates of the thread's halo nodes (lh[k][0] = -1: none)
#pragma unroll
    for (int k = 0; k < HP; ++k) {
        const int hidx = threadIdx.x + k * TL::NT;
        lh[k][0] = -1;
        if (hidx < NH) {
            int lx, ly, lz;
            shell_pos<DIM, VX, VY, VZ, 1, 1>(hidx, lx, ly, lz);
            const int x = X0 + lx, y = Y0 + ly, z = Z0 + lz;
            if (in_f(x, y, z)) {
                lh[k][0] = lx;
                lh[k][1] = ly;
                lh[k][2] = lz;
                const size_t p = (size_t)z * fxy + (size_t)y * F.nx + x;
#pragma unroll
                for (int r = 0; r < RB; ++r)
                    if (on[r]) uh[r][k] = uin[r * sin + p];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < EP; ++k) {
        const int t = threadIdx.x + k * TL::NT;
        if (t < EBOX) {
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (on[r]) se_[r * EBOX + t] = eq[r][k];
        }
    }
    __syncthreads();
    // v = u + P e (multilinear prolongation) on the whole box
    auto put_v = [&](int lx, int ly, int lz, const C *uv) {
        const int x = X0 + lx, y = Y0 + ly, z = Z0 + lz;
        const int ax = (x >> 1) - CX0, bxp = ((x + 1) >> 1) - CX0;
        const int ay = (y >> 1) - CY0, byp = ((y + 1) >> 1) - CY0;
        const int az = DIM == 3 ? (z >> 1) - CZ0 : 0, bzp = DIM == 3 ? ((z + 1) >> 1) - CZ0 : 0;
        const T wx = (x & 1) ? T(0.5) : T(1), wy = (y & 1) ? T(0.5) : T(1),
                wz = (DIM == 3 && (z & 1)) ? T(0.5) : T(1);
        const T wgt = wx * wy * wz;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            if (!on[r]) continue;
            const C *ser = se_ + r * EBOX;
            T px = 0, py = 0;
#pragma unroll
            for (int kz = 0; kz < (DIM == 3 ? 2 : 1); ++kz) {
                const int zz = kz ? bzp : az;
                if (kz && bzp == az) break;
#pragma unroll
                for (int ky = 0; ky < 2; ++ky) {
                    const int yy = ky ? byp : ay;
                    if (ky && byp == ay) break;
                    const C e0 = ser[(zz * EY + yy) * EX + ax];
                    px += e0.x;
                    py += e0.y;
                    if (bxp != ax) {
                        const C e1 = ser[(zz * EY + yy) * EX + bxp];
                        px += e1.x;
                        py += e1.y;
                    }
                }
            }
            C o = uv[r];
            o.x = fmaT(wgt, px, o.x);
            o.y = fmaT(wgt, py, o.y);
            sv_[r * VBOX + (lz * VY + ly) * VX + lx] = o;
        }
    };
#pragma unroll
    for (int k = 0; k < HP; ++k)
        if (lh[k][0] >= 0) {
            C hv[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) hv[r] = uh[r][k];
            put_v(lh[k][0], lh[k][1], lh[k][2], hv);
        }
#pragma unroll
    for (int k = 0; k < NQL; ++k) {
        const int q = q0 + k * QP;
        const int x = 2 * (I0 + tx) + (q & 1), y = 2 * (J0 + ty) + ((q >> 1) & 1),
                  z = DIM == 3 ? 2 * (K0 + tz) + (q >> 2) : 0;
        if (iq[k]) {
            C ov[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) ov[r] = uq[r][k];
            put_v(x - X0, y - Y0, z - Z0, ov);
        }
    }
    __syncthreads();
    // one damped-Jacobi sweep on the own children
#pragma unroll
    for (int k = 0; k < NQL; ++k) {
        const int q = q0 + k * QP;
        const int x = 2 * (I0 + tx) + (q & 1), y = 2 * (J0 + ty) + ((q >> 1) & 1),
                  z = DIM == 3 ? 2 * (K0 + tz) + (q >> 2) : 0;
        if (!iq[k]) continue;
        const int qq = ((z - Z0) * VY + (y - Y0)) * VX + (x - X0);
        const C di = dq[k];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            if (!on[r]) continue;
            const C *svr = sv_ + r * VBOX;
            T sx = 0, sy = 0;
            if (INT || x > 0) { const T c = (!INT && x == F.nx - 1) ? T(2) : T(1); sx = fmaT(c, svr[qq - 1].x, sx); sy = fmaT(c, svr[qq - 1].y, sy); }
            if (INT || x < F.nx - 1) { const T c = (!INT && x == 0) ? T(2) : T(1); sx = fmaT(c, svr[qq + 1].x, sx); sy = fmaT(c, svr[qq + 1].y, sy); }
            if (INT || y > 0) { const T c = (!INT && y == F.ny - 1) ? T(2) : T(1); sx = fmaT(c, svr[qq - VX].x, sx); sy = fmaT(c, svr[qq - VX].y, sy); }
            if (INT || y < F.ny - 1) { const T c = (!INT && y == 0) ? T(2) : T(1); sx = fmaT(c, svr[qq + VX].x, sx); sy = fmaT(c, svr[qq + VX].y, sy); }
            if (DIM == 3) {
                if (INT || z > 0) { const T c = (!INT && z == F.nz - 1) ? T(2) : T(1); sx = fmaT(c, svr[qq - VX * VY].x, sx); sy = fmaT(c, svr[qq - VX * VY].y, sy); }
                if (INT || z < F.nz - 1) { const T c = (!INT && z == 0) ? T(2) : T(1); sx = fmaT(c, svr[qq + VX * VY].x, sx); sy = fmaT(c, svr[qq + VX * VY].y, sy); }
            }
            const C vp = svr[qq];
            const C bp = cvt<C>(bq[r][k]);
            const T gx = fmaT(F.inv_h2, sx, bp.x), gy = fmaT(F.inv_h2, sy, bp.y);
            const T omw = T(1) - wj;
            C o;
            o.x = fmaT(omw, vp.x, wj * fmaT(di.x, gx, -(di.y * gy)));
            o.y = fmaT(omw, vp.y, wj * fmaT(di.x, gy, di.y * gx));
            uout[r * sout + pq[k]] = o;
        }
    }
}

template <typename T, typename CB, int DIM, typename TL, bool SC = false>
__global__ void __launch_bounds__(TL::NT)
k_down(LevelView<T> F, LevelView<T> Cv, T wj, const CB *__restrict__ b, size_t sb,
       cplx_t<T> *__restrict__ u, size_t su, cplx_t<T> *__restrict__ bc, size_t sbc, int nb,
       const int *__restrict__ active, const float2 *__restrict__ sc, float2 *__restrict__ vout, size_t svout) {
    // the box of u spans fine [2 I0 - 2, 2 I0 + 2 S] per axis
    const int gz = DIM == 3 ? (Cv.nz + TL::SZ - 1) / TL::SZ : 1;
    const int bz = blockIdx.z % gz;
    const int x0 = 2 * (int)blockIdx.x * TL::SX - 2, y0 = 2 * (int)blockIdx.y * TL::SY - 2,
              z0 = 2 * bz * TL::SZ - 2;
    const bool inside = x0 >= 0 && x0 + 2 * TL::SX + 2 <= F.nx - 1 && y0 >= 0 &&
                        y0 + 2 * TL::SY + 2 <= F.ny - 1 &&
                        (DIM != 3 || (z0 >= 0 && z0 + 2 * TL::SZ + 2 <= F.nz - 1));
    if (inside)
        down_tile<T, CB, DIM, TL, true, SC>(F, Cv, wj, b, sb, u, su, bc, sbc, nb, active, sc, vout, svout);
    else
        down_tile<T, CB, DIM, TL, false, SC>(F, Cv, wj, b, sb, u, su, bc, sbc, nb, active, sc, vout, svout);
}

template <typename T, typename CB, int DIM, typename TL>
__global__ void __launch_bounds__(TL::NT)
k_up(LevelView<T> F, LevelView<T> Cv, T wj, const cplx_t<T> *__restrict__ uin,
     size_t sin, const cplx_t<T> *__restrict__ ec, size_t sec, const CB *__restrict__ b, size_t sb,
     cplx_t<T> *__restrict__ uout, size_t sout, int nb, const int *__restrict__ active) {
    // the box of v spans fine [2 I0 - 1, 2 I0 + 2 S] per axis (coarse [I0 - 1, I0 + S])
    const int gz = DIM == 3 ? (Cv.nz + TL::SZ - 1) / TL::SZ : 1;
    const int bz = blockIdx.z % gz;
    const int x0 = 2 * (int)blockIdx.x * TL::SX - 1, y0 = 2 * (int)blockIdx.y * TL::SY - 1,
              z0 = 2 * bz * TL::SZ - 1;
    const bool inside = x0 >= 0 && x0 + 2 * TL::SX + 1 <= F.nx - 1 && y0 >= 0 &&
                        y0 + 2 * TL::SY + 1 <= F.ny - 1 &&
                        (DIM != 3 || (z0 >= 0 && z0 + 2 * TL::SZ + 1 <= F.nz - 1));
    if (inside) up_tile<T, CB, DIM, TL, true>(F, Cv, wj, uin, sin, ec, sec, b, sb, uout, sout, nb, active);
    else up_tile<T, CB, DIM, TL, false>(F, Cv, wj, uin, sin, ec, sec, b, sb, uout, sout, nb, active);
}

// ---------------------------------------------------------------- 3D down, marching along z
// The same arithmetic as the 3D k_down (u = wj D^-1 b, r with the neighbours
// in the order x-, x+, y-, y+, z-, z+, full weighting with the 27 taps in the
// order z, y, x), so its results equal every other 3D shape's bit for bit.
// The block keeps three planes of u, two of b and three of r (its x, y box of
// (2 SX + 3) x (2 SY + 3) fine nodes) in shared memory and walks the fine
// planes 2 K0 - 2 .. 2 K1 in order: u of plane z, then r of plane z - 1, then
// the restriction of coarse plane K once r of 2K - 1, 2K and 2K + 1 exist.
// The loads of the next plane are issued before the current plane is used.
template <typename T, typename CB, typename TL, bool INT>
__device__ __forceinline__ void down_zm_tile(const LevelView<T> &F, const LevelView<T> &Cv, T wj,
                                             const CB *__restrict__ b, size_t sb,
                                             cplx_t<T> *__restrict__ u, size_t su,
                                             cplx_t<T> *__restrict__ bc, size_t sbc) {
    using C = cplx_t<T>;
    constexpr int SX = TL::SX, SY = TL::SY, KC = TL::SZ, NT = TL::NT;
    constexpr int UX = 2 * SX + 3, UY = 2 * SY + 3, UP = UX * UY;
    constexpr int NH = shell_count<2, UX, UY, 1, 2, 1>();
    constexpr int HP = (NH + NT - 1) / NT;
    constexpr int RX = UX - 2, RY = UY - 2;
    constexpr int NR = shell_count<2, RX, RY, 1, 1, 0>();
    const int gz = (Cv.nz + KC - 1) / KC;
    const int bz = blockIdx.z % gz;
    const int I0 = blockIdx.x * SX, J0 = blockIdx.y * SY, K0 = bz * KC, K1 = min(K0 + KC, Cv.nz);
    const int X0 = 2 * I0 - 2, Y0 = 2 * J0 - 2;
    const int tx = threadIdx.x % SX, ty = threadIdx.x / SX;
    const int nz = F.nz;
    const size_t fxy = (size_t)F.nx * F.ny;
    extern __shared__ unsigned char smem_raw[];
    C *su_ = reinterpret_cast<C *>(smem_raw);   // u, planes z mod 3
    C *sb_ = su_ + 3 * UP;                        // b, planes z mod 2
    C *sr_ = sb_ + 2 * UP;                        // r, planes z mod 3
    auto in_xy = [&](int x, int y) { return INT || (x >= 0 && x < F.nx && y >= 0 && y < F.ny); };
    const int zs = max(0, 2 * K0 - 2), ze = min(nz - 1, 2 * K1);
    const int zr_lo = max(0, 2 * K0 - 1), zr_hi = min(nz - 1, 2 * K1 - 1);
    CB bq[4], bh[HP], bq2[4], bh2[HP];
    C dq[4], dh[HP], dq2[4], dh2[HP];
    auto load_plane = [&](int z, CB (&pb)[4], C (&pd)[4], CB (&hb)[HP], C (&hd)[HP]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = 2 * (I0 + tx) + (k & 1), y = 2 * (J0 + ty) + (k >> 1);
            if (in_xy(x, y)) {
                const size_t p = (size_t)z * fxy + (size_t)y * F.nx + x;
                pb[k] = b[p];
                pd[k] = F.dinv[p];
            }
        }
#pragma unroll
        for (int k = 0; k < HP; ++k) {
            const int hidx = threadIdx.x + k * NT;
            if (hidx < NH) {
                int lx, ly, lz;
                shell_pos<2, UX, UY, 1, 2, 1>(hidx, lx, ly, lz);
                const int x = X0 + lx, y = Y0 + ly;
                if (in_xy(x, y)) {
                    const size_t p = (size_t)z * fxy + (size_t)y * F.nx + x;
                    hb[k] = b[p];
                    hd[k] = F.dinv[p];
                }
            }
        }
    };
    auto put_u = [&](C *sup, C *sbp, int t, CB braw, C di) {
        const C bp = cvt<C>(braw);
        C up;
        up.x = wj * fmaT(di.x, bp.x, -(di.y * bp.y));
        up.y = wj * fmaT(di.x, bp.y, di.y * bp.x);
        sup[t] = up;
        sbp[t] = bp;
        return up;
    };
    auto put_r = [&](int lx, int ly, int zr, const C *um, const C *uc, const C *upl, const C *sbp, C *srp) {
        const int x = X0 + lx, y = Y0 + ly;
        const int q = ly * UX + lx;
        T sx = 0, sy = 0;
        if (INT || x > 0) { const T c = (!INT && x == F.nx - 1) ? T(2) : T(1); sx = fmaT(c, uc[q - 1].x, sx); sy = fmaT(c, uc[q - 1].y, sy); }
        if (INT || x < F.nx - 1) { const T c = (!INT && x == 0) ? T(2) : T(1); sx = fmaT(c, uc[q + 1].x, sx); sy = fmaT(c, uc[q + 1].y, sy); }
        if (INT || y > 0) { const T c = (!INT && y == F.ny - 1) ? T(2) : T(1); sx = fmaT(c, uc[q - UX].x, sx); sy = fmaT(c, uc[q - UX].y, sy); }
        if (INT || y < F.ny - 1) { const T c = (!INT && y == 0) ? T(2) : T(1); sx = fmaT(c, uc[q + UX].x, sx); sy = fmaT(c, uc[q + UX].y, sy); }
        if (zr > 0) { const T c = (zr == nz - 1) ? T(2) : T(1); sx = fmaT(c, um[q].x, sx); sy = fmaT(c, um[q].y, sy); }
        if (zr < nz - 1) { const T c = (zr == 0) ? T(2) : T(1); sx = fmaT(c, upl[q].x, sx); sy = fmaT(c, upl[q].y, sy); }
        const C bp = sbp[q];
        const T omw = T(1) - wj;
        C o;
        o.x = fmaT(F.inv_h2, sx, omw * bp.x);
        o.y = fmaT(F.inv_h2, sy, omw * bp.y);
        srp[q] = o;
    };
    load_plane(zs, bq, dq, bh, dh);
    for (int zu = zs; zu <= ze + 1; ++zu) {
        // the next plane's loads go out before this plane is used
        const bool more = zu + 1 <= ze;
        if (more) load_plane(zu + 1, bq2, dq2, bh2, dh2);
        if (zu <= ze) {
            C *sup = su_ + (zu % 3) * UP, *sbp = sb_ + (zu & 1) * UP;
#pragma unroll
            for (int k = 0; k < HP; ++k) {
                const int hidx = threadIdx.x + k * NT;
                if (hidx < NH) {
                    int lx, ly, lz;
                    shell_pos<2, UX, UY, 1, 2, 1>(hidx, lx, ly, lz);
                    if (in_xy(X0 + lx, Y0 + ly)) put_u(sup, sbp, ly * UX + lx, bh[k], dh[k]);
                }
            }
            const bool own = zu >= 2 * K0 && zu < 2 * K1;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int x = 2 * (I0 + tx) + (k & 1), y = 2 * (J0 + ty) + (k >> 1);
                if (in_xy(x, y)) {
                    const C up = put_u(sup, sbp, (y - Y0) * UX + (x - X0), bq[k], dq[k]);
                    if (own) u[(size_t)zu * fxy + (size_t)y * F.nx + x] = up;
                }
            }
        }
        __syncthreads();
        const int zr = zu - 1;
        if (zr >= zr_lo && zr <= zr_hi) {
            const C *um = su_ + ((zr + 2) % 3) * UP, *uc = su_ + (zr % 3) * UP, *upl = su_ + ((zr + 1) % 3) * UP;
            const C *sbp = sb_ + (zr & 1) * UP;
            C *srp = sr_ + (zr % 3) * UP;
            for (int hidx = threadIdx.x; hidx < NR; hidx += NT) {
                int lx, ly, lz;
                shell_pos<2, RX, RY, 1, 1, 0>(hidx, lx, ly, lz);
                ++lx;
                ++ly;
                if (in_xy(X0 + lx, Y0 + ly)) put_r(lx, ly, zr, um, uc, upl, sbp, srp);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int x = 2 * (I0 + tx) + (k & 1), y = 2 * (J0 + ty) + (k >> 1);
                if (in_xy(x, y)) put_r(x - X0, y - Y0, zr, um, uc, upl, sbp, srp);
            }
        }
        __syncthreads();
        // coarse plane K once r of 2K - 1, 2K, 2K + 1 (mirrored at the ends) exists
        int K = -1;
        if (zr >= 1 && (zr & 1) && zr <= zr_hi) K = (zr - 1) >> 1;
        else if (zr == nz - 1 && !(zr & 1)) K = zr >> 1;
        if (K >= K0 && K < K1) {
            const int I = I0 + tx, J = J0 + ty;
            if (I < Cv.nx && J < Cv.ny) {
                T ax = 0, ay = 0;
#pragma unroll
                for (int oz = -1; oz <= 1; ++oz) {
                    const C *srp = sr_ + (mirror(2 * K + oz, nz) % 3) * UP;
                    const T wz = oz == 0 ? T(0.5) : T(0.25);
#pragma unroll
                    for (int oy = -1; oy <= 1; ++oy) {
                        const int ly = mirror_if<INT>(2 * J + oy, F.ny) - Y0;
                        const T wy = oy == 0 ? T(0.5) : T(0.25);
#pragma unroll
                        for (int ox = -1; ox <= 1; ++ox) {
                            const int lx = mirror_if<INT>(2 * I + ox, F.nx) - X0;
                            const T wgt = (ox == 0 ? T(0.5) : T(0.25)) * wy * wz;
                            const C v = srp[ly * UX + lx];
                            ax = fmaT(wgt, v.x, ax);
                            ay = fmaT(wgt, v.y, ay);
                        }
                    }
                }
                C o;
                o.x = ax;
                o.y = ay;
                bc[(size_t)K * Cv.nx * Cv.ny + (size_t)J * Cv.nx + I] = o;
            }
        }
        if (more) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                bq[k] = bq2[k];
                dq[k] = dq2[k];
            }
#pragma unroll
            for (int k = 0; k < HP; ++k) {
                bh[k] = bh2[k];
                dh[k] = dh2[k];
            }
        }
    }
}

template <typename T, typename CB, typename TL>
__global__ void __launch_bounds__(TL::NT)
k_down_zm(LevelView<T> F, LevelView<T> Cv, T wj, const CB *__restrict__ b, size_t sb,
          cplx_t<T> *__restrict__ u, size_t su, cplx_t<T> *__restrict__ bc, size_t sbc,
          const int *__restrict__ active) {
    const int gz = (Cv.nz + TL::SZ - 1) / TL::SZ;
    const int rr = blockIdx.z / gz;
    if (active && !active[rr]) return;
    b += rr * sb;
    u += rr * su;
    bc += rr * sbc;
    // the x, y box spans fine [2 I0 - 2, 2 I0 + 2 S] (as k_down)
    const int x0 = 2 * (int)blockIdx.x * TL::SX - 2, y0 = 2 * (int)blockIdx.y * TL::SY - 2;
    const bool inside = x0 >= 0 && x0 + 2 * TL::SX + 2 <= F.nx - 1 && y0 >= 0 && y0 + 2 * TL::SY + 2 <= F.ny - 1;
    if (inside) down_zm_tile<T, CB, TL, true>(F, Cv, wj, b, sb, u, su, bc, sbc);
    else down_zm_tile<T, CB, TL, false>(F, Cv, wj, b, sb, u, su, bc, sbc);
}

template <int DIM, typename TL> constexpr size_t down_smem(size_t csz) {
    constexpr int UX = 2 * TL::SX + 3, UY = 2 * TL::SY + 3, UZ = DIM == 3 ? 2 * TL::SZ + 3 : 1;
    if constexpr (TL::MARCH) return csz * 8 * UX * UY;   // u: 3 planes, b: 2, r: 3
    else return csz * 3 * UX * UY * UZ * TL::RB;
}
template <int DIM, typename TL> constexpr size_t up_smem(size_t csz) {
    constexpr int VX = 2 * TL::SX + 2, VY = 2 * TL::SY + 2, VZ = DIM == 3 ? 2 * TL::SZ + 2 : 1;
    constexpr int EX = TL::SX + 2, EY = TL::SY + 2, EZ = DIM == 3 ? TL::SZ + 2 : 1;
    return csz * (VX * VY * VZ + EX * EY * EZ) * TL::RB;
}

// right-hand sides one launch can take when each group of rb needs gz blocks along z
inline int rhs_per_launch(int gz, int rb, int nb) {
    const int cap = (65535 / gz) * rb;
    return nb < cap ? nb : cap;
}

template <typename T, typename CB, int DIM, typename TL>
void down_impl(const LevelView<T> &F, const LevelView<T> &Cv, T wj, const CB *b,
               size_t sb, cplx_t<T> *u, size_t su, cplx_t<T> *bc, size_t sbc, int nb,
               const int *active, cudaStream_t st) {
    const size_t sm = down_smem<DIM, TL>(sizeof(cplx_t<T>));
    const int gz = DIM == 3 ? (Cv.nz + TL::SZ - 1) / TL::SZ : 1;
    // gridDim.z = z tiles x right-hand sides; a batch beyond its 65535 limit
    // runs as several launches over consecutive right-hand sides
    const int chunk = rhs_per_launch(gz, TL::RB, nb);
    for (int r0 = 0; r0 < nb; r0 += chunk) {
        const int n = nb - r0 < chunk ? nb - r0 : chunk;
        dim3 g((Cv.nx + TL::SX - 1) / TL::SX, (Cv.ny + TL::SY - 1) / TL::SY,
               gz * ((n + TL::RB - 1) / TL::RB));
        const int *act = active ? active + r0 : nullptr;
        if constexpr (TL::MARCH) {
            static_assert(DIM == 3, "marching tiles are 3D");
            k_down_zm<T, CB, TL><<<g, TL::NT, sm, st>>>(F, Cv, wj, b + r0 * sb, sb, u + r0 * su, su,
                                                        bc + r0 * sbc, sbc, act);
        } else {
            k_down<T, CB, DIM, TL><<<g, TL::NT, sm, st>>>(F, Cv, wj, b + r0 * sb, sb, u + r0 * su,
                                                          su, bc + r0 * sbc, sbc, n, act, nullptr, nullptr, 0);
        }
        count_launch();
    }
}

template <typename T, typename CB, int DIM, typename TL>
void up_impl(const LevelView<T> &F, const LevelView<T> &Cv, T wj,
             const cplx_t<T> *uin, size_t sin, const cplx_t<T> *ec, size_t sec, const CB *b,
             size_t sb, cplx_t<T> *uout, size_t sout, int nb, const int *active, cudaStream_t st) {
    const size_t sm = up_smem<DIM, TL>(sizeof(cplx_t<T>));
    const int gz = DIM == 3 ? (Cv.nz + TL::SZ - 1) / TL::SZ : 1;
    const int chunk = rhs_per_launch(gz, TL::RB, nb);
    for (int r0 = 0; r0 < nb; r0 += chunk) {
        const int n = nb - r0 < chunk ? nb - r0 : chunk;
        dim3 g((Cv.nx + TL::SX - 1) / TL::SX, (Cv.ny + TL::SY - 1) / TL::SY,
               gz * ((n + TL::RB - 1) / TL::RB));
        k_up<T, CB, DIM, TL><<<g, TL::NT, sm, st>>>(F, Cv, wj, uin + r0 * sin, sin, ec + r0 * sec,
                                                    sec, b + r0 * sb, sb, uout + r0 * sout, sout, n,
                                                    active ? active + r0 : nullptr);
        count_launch();
    }
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
// the level-0 down kernel of the complex64 basis taking w and the scale pair
// (the z-marching 3D kernel cannot take w)
template <int DIM, typename TL>
bool down_c64w_impl(const LevelView<float> &F, const LevelView<float> &Cv, float wj, const float4 *w, size_t sw,
                    const float2 *sc, float2 *vout, size_t svout, float2 *u, size_t su, float2 *bc, size_t sbc,
                    int nb, const int *active, cudaStream_t st) {
    if constexpr (TL::MARCH) {
        return false;
    } else {
        const size_t sm = down_smem<DIM, TL>(sizeof(float2));
        const int gz = DIM == 3 ? (Cv.nz + TL::SZ - 1) / TL::SZ : 1;
        const int chunk = rhs_per_launch(gz, TL::RB, nb);
        for (int r0 = 0; r0 < nb; r0 += chunk) {
            const int n = nb - r0 < chunk ? nb - r0 : chunk;
            dim3 g((Cv.nx + TL::SX - 1) / TL::SX, (Cv.ny + TL::SY - 1) / TL::SY,
                   gz * ((n + TL::RB - 1) / TL::RB));
            k_down<float, float4, DIM, TL, true><<<g, TL::NT, sm, st>>>(
                F, Cv, wj, w + r0 * sw, sw, u + r0 * su, su, bc + r0 * sbc, sbc, n, active ? active + r0 : nullptr,
                sc + r0, vout + r0 * svout, svout);
            count_launch();
        }
        return true;
    }
}

template <int DIM, size_t... I>
bool down_c64w_sel(int shape, std::index_sequence<I...>, const LevelView<float> &F, const LevelView<float> &Cv,
                   float wj, const float4 *w, size_t sw, const float2 *sc, float2 *vout, size_t svout, float2 *u,
                   size_t su, float2 *bc, size_t sbc, int nb, const int *active, cudaStream_t st) {
    bool ok = false;
    ((shape == (int)I
          ? (void)(ok = down_c64w_impl<DIM, std::tuple_element_t<I, typename Shapes<DIM>::Down>>(
                       F, Cv, wj, w, sw, sc, vout, svout, u, su, bc, sbc, nb, active, st))
          : void()),
     ...);
    return ok;
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

template <int DIM, typename TL> void set_attr_down_c64w() {
    if constexpr (!TL::MARCH)
        cudaFuncSetAttribute(k_down<float, float4, DIM, TL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)down_smem<DIM, TL>(sizeof(float2)));
}

template <int DIM, size_t... I> void set_attr_all_c64w(std::index_sequence<I...>) {
    (set_attr_down_c64w<DIM, std::tuple_element_t<I, typename Shapes<DIM>::Down>>(), ...);
}

template <typename T, typename CB, int DIM, typename TL> void set_attr_down() {
    const int sm = (int)down_smem<DIM, TL>(sizeof(cplx_t<T>));
    if constexpr (TL::MARCH)
        cudaFuncSetAttribute(k_down_zm<T, CB, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    else
        cudaFuncSetAttribute(k_down<T, CB, DIM, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

template <typename T, typename CB, int DIM, size_t... I>
void set_attr_all(std::index_sequence<I...>) {
    (set_attr_down<T, CB, DIM, std::tuple_element_t<I, typename Shapes<DIM>::Down>>(), ...);
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
void shape_info(bool up, int shape, int ext[3], int *threads, int *rb, std::index_sequence<I...>) {
    auto one = [&](auto tag) {
        using S = decltype(tag);
        ext[0] = S::SX;
        ext[1] = S::SY;
        ext[2] = S::SZ;
        *threads = S::NT;
        *rb = S::RB;
    };
    if (up)
        ((shape == (int)I ? one(std::tuple_element_t<I, typename Shapes<DIM>::Up>{}) : void()), ...);
    else
        ((shape == (int)I ? one(std::tuple_element_t<I, typename Shapes<DIM>::Down>{}) : void()), ...);
}

}  // namespace

template <typename T, typename CB>
void launch_vdown(const LevelView<T> &F, const LevelView<T> &Cv, T wj, const CB *b,
                  size_t sb, cplx_t<T> *u, size_t su, cplx_t<T> *bc, size_t sbc, int nb,
                  const int *active, cudaStream_t st, int shape, bool finest) {
    prof_begin(st);
    if (F.dim == 2)
        down_sel<T, CB, 2>(shape, std::make_index_sequence<n_down<2>()>{}, F, Cv, wj, b, sb, u, su,
                           bc, sbc, nb, active, st);
    else
        down_sel<T, CB, 3>(shape, std::make_index_sequence<n_down<3>()>{}, F, Cv, wj, b, sb, u, su,
                           bc, sbc, nb, active, st);
    if (prof_on()) {
        // per right-hand side: b in, u and the coarse right-hand side out;
        // D^-1 once per launch (shared by the right-hand sides)
        const double n1 = (double)F.nx * F.ny * F.nz;
        const double nf = n1 * nb, nc = (double)Cv.nx * Cv.ny * Cv.nz * nb;
        prof_end(sizeof(T) == 8 ? (finest ? "vdown_l0_f64" : "vdown_f64") : (finest ? "vdown_l0_f32" : "vdown_f32"), st,
                 nf * (sizeof(CB) + sizeof(cplx_t<T>)) + n1 * sizeof(cplx_t<T>) + nc * sizeof(cplx_t<T>),
                 sizeof(T) == 8 ? nf * 26.0 : 0.0);
    }
}

template <typename T, typename CB>
void launch_vup(const LevelView<T> &F, const LevelView<T> &Cv, T wj,
                const cplx_t<T> *uin, size_t sin, const cplx_t<T> *ec, size_t sec, const CB *b,
                size_t sb, cplx_t<T> *uout, size_t sout, int nb, const int *active,
                cudaStream_t st, int shape, bool finest) {
    prof_begin(st);
    if (F.dim == 2)
        up_sel<T, CB, 2>(shape, std::make_index_sequence<n_up<2>()>{}, F, Cv, wj, uin, sin, ec, sec, b,
                         sb, uout, sout, nb, active, st);
    else
        up_sel<T, CB, 3>(shape, std::make_index_sequence<n_up<3>()>{}, F, Cv, wj, uin, sin, ec, sec, b,
                         sb, uout, sout, nb, active, st);
    if (prof_on()) {
        // per right-hand side: u and b in, the sweep out, the coarse
        // correction in; D^-1 once per launch
        const double n1 = (double)F.nx * F.ny * F.nz;
        const double nf = n1 * nb, nc = (double)Cv.nx * Cv.ny * Cv.nz * nb;
        prof_end(sizeof(T) == 8 ? (finest ? "vup_l0_f64" : "vup_f64") : (finest ? "vup_l0_f32" : "vup_f32"), st,
                 nf * (2.0 * sizeof(cplx_t<T>) + sizeof(CB)) + n1 * sizeof(cplx_t<T>) + nc * sizeof(cplx_t<T>),
                 sizeof(T) == 8 ? nf * 24.0 : 0.0);
    }
}

#define HELM_INST_V(T, CB)                                                                      \
    template void launch_vdown<T, CB>(const LevelView<T> &, const LevelView<T> &, T,             \
                                      const CB *, size_t, cplx_t<T> *, size_t, cplx_t<T> *,     \
                                      size_t, int, const int *, cudaStream_t, int, bool);       \
    template void launch_vup<T, CB>(const LevelView<T> &, const LevelView<T> &, T,               \
                                    const cplx_t<T> *, size_t, const cplx_t<T> *, size_t,       \
                                    const CB *, size_t, cplx_t<T> *, size_t, int, const int *,  \
                                    cudaStream_t, int, bool);

// each type pair's translation unit sets its kernels' shared-memory limits
void vfused_attr_f64();
void vfused_attr_mixed();
void vfused_attr_c64();
void vfused_attr_ds();

}  // namespace helm
