// Coarsest-level product of the complex64 V-cycle on the tensor cores:
// Z = Ainv R, Ainv the dense inverse of the coarsest shifted Laplacian (Eq. 6;
// n x n complex, about 1300 x 1300 on the 401 x 201 grid) and R the coarse
// right-hand sides of up to 64 sources at once.
//
// The complex product is split into real ones, Zr = Ar Rr - Ai Ri and
// Zi = Ai Rr + Ar Ri, each formed with tcgen05.mma kind::tf32 (M = 128 rows,
// N = 64 right-hand sides, K = 8 per instruction; the minus sign is the
// instruction's negate-B bit). TF32 keeps 10 mantissa bits, so every FP32
// operand x is split into x_hi = x with its low 13 bits cleared (exact in
// TF32) and x_lo = x - x_hi, and a b = a_hi b_hi + a_hi b_lo + a_lo b_hi
// (the dropped a_lo b_lo is ~2^-22 relative): the product keeps FP32
// accuracy, as the rest of the complex64 V-cycle.
//
// Ainv is split and laid out once per model (launch_coarse_tc_tiles) in
// blocks of 128 rows x 32 columns, four planes (re_hi, re_lo, im_hi, im_lo)
// in the K-major core-matrix order the MMA reads, so one cp.async.bulk copy
// stages 64 KB of Ainv. For chunk kc a CTA takes rows 128 rt.., columns
// 32 kc.. and sources 64 jt..; it splits its slice of R into shared memory,
// issues 48 MMAs into two TMEM accumulators (real, imaginary: 128 lanes x 64
// columns each). A CTA walks a group of consecutive chunks (about one CTA per
// SM), accumulating in TMEM, and writes its partial product;
// k_coarse_tc_sum adds the partials in group order. Each output element's arithmetic depends on
// n only (one source's column never mixes with another's), so batched and
// single solves agree bitwise.
#include "helm_internal.cuh"
#include "pipe.cuh"
#include "tc.cuh"

namespace helm {

namespace {

constexpr int kM = 128;               // rows of Ainv per CTA (MMA M)
constexpr int kN = 64;                // right-hand sides per CTA (MMA N)
constexpr int kK = 32;                // columns of Ainv per CTA
constexpr int kThreads = 256;
constexpr int kAPlane = kM * kK;      // floats per plane of an Ainv block
constexpr int kBPlane = kN * kK;
constexpr unsigned kTmemCols = 128;   // two accumulators of kN columns

// element (row, k) of a block with kK columns, K-major core-matrix order:
// core matrices of 8 rows x 4 floats (128 contiguous bytes), kK / 4 of them
// along K for each group of 8 rows
__host__ __device__ constexpr int cm_off(int row, int k) {
    return ((row >> 3) * (kK / 4) + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3);
}

using tc::tf32_hi;

// two stages: the Ainv copy of the next chunk lands while this chunk's MMAs run
struct alignas(1024) TcSmem {
    float a[2][4][kAPlane];    // re_hi, re_lo, im_hi, im_lo of an Ainv block, per stage
    float b[2][4][kBPlane];    // re_hi, re_lo, im_hi, im_lo of an R slice (row = source), per stage
    uint64_t abar[2], mbar[2]; // per stage: Ainv block landed; the stage's MMAs complete
    uint32_t tmem;             // TMEM base address
    int abort;
};

using tc::smem_desc;
using tc::mma_tf32;
using tc::tmem_ld64;
__device__ __forceinline__ void tc_fence_before() { tc::fence_before(); }
__device__ __forceinline__ void tc_fence_after() { tc::fence_after(); }

struct TcGeom {
    int n, nrt, nkc, Mp, nsb;   // order, row blocks, column chunks, padded rows, source blocks
    int kch, nkg;               // chunks per CTA (accumulated in TMEM), CTA column groups
};

inline TcGeom tc_geom(int n, int nb) {
    TcGeom g;
    g.n = n;
    g.nrt = (n + kM - 1) / kM;
    g.nkc = (n + kK - 1) / kK;
    g.Mp = g.nrt * kM;
    g.nsb = (nb + kN - 1) / kN;
    // about one CTA per SM per block of sources; depends on n and the SM
    // count only, so the order of every sum is fixed by n on a device
    const int sms = device_sms();
    g.kch = (g.nrt * g.nkc + sms - 1) / sms;
    g.nkg = (g.nkc + g.kch - 1) / g.kch;
    return g;
}

// tiles[((rt * nkc + kc) * 4 + plane) * kAPlane + cm_off(m % kM, k % kK)],
// m = row, k = column of Ainv (At is Ainv column-major); zero padding
__global__ void k_coarse_tc_tiles(const float2 *__restrict__ At, TcGeom G, float *__restrict__ tiles) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (m >= G.Mp) return;
    float2 v = make_float2(0.f, 0.f);
    if (m < G.n && k < G.n) v = At[(size_t)k * G.n + m];
    float *blk = tiles + (size_t)((m / kM) * G.nkc + k / kK) * 4 * kAPlane;
    const int o = cm_off(m % kM, k % kK);
    const float rh = tf32_hi(v.x), ih = tf32_hi(v.y);
    blk[o] = rh;
    blk[kAPlane + o] = v.x - rh;
    blk[2 * kAPlane + o] = ih;
    blk[3 * kAPlane + o] = v.y - ih;
}

// part[((kg * 2 + plane) * nb + source) * Mp + row]: the share of Z of
// column group kg (chunks kg * kch .. kg * kch + kch - 1, accumulated in TMEM).
//
// Chunk i of the group uses stage i % 2. Each stage has its own "landed" and
// "MMAs done" barriers, completing once per use of the stage (phase i / 2),
// and each phase is waited for before the next use of that stage is issued,
// so no wait can find its barrier two phases ahead.
__global__ void __launch_bounds__(kThreads, 1)
k_coarse_tc(const float *__restrict__ tiles, TcGeom G, const float2 *__restrict__ R, size_t sr,
            float *__restrict__ part, int nb, const int *__restrict__ active) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(tc_raw);
    const int kg = blockIdx.x, rt = blockIdx.y, jt = blockIdx.z;
    const int c0 = kg * G.kch, c1 = min(c0 + G.kch, G.nkc);
    const int nch = c1 - c0;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const unsigned abytes = 4u * kAPlane * sizeof(float);
    unsigned issued[2] = {0u, 0u};   // Ainv copies issued per stage (thread 0)
    auto copy_a = [&](int i) {       // thread 0: Ainv block of chunk c0 + i into stage i % 2
        const int st = i & 1;
        pipe::mbar_arrive_expect_tx(&S.abar[st], abytes);
        pipe::bulk_load(&S.a[st][0][0], tiles + (size_t)(rt * G.nkc + c0 + i) * 4 * kAPlane, abytes,
                        &S.abar[st]);
        ++issued[st];
    };
    if (t == 0) {
        for (int st = 0; st < 2; ++st) {
            pipe::mbar_init(&S.abar[st], 1);
            pipe::mbar_init(&S.mbar[st], 1);
        }
        S.abort = 0;
        pipe::mbar_init_fence();
        copy_a(0);
        if (nch > 1) copy_a(1);
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         pipe::smem_addr(&S.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // every warp reads the abort word (and later the barriers and the TMEM
    // address) that thread 0 and warp 0 have just written: without this
    // barrier a warp could read the word before it is cleared, i.e. whatever
    // an earlier block, of any kernel, left at that shared-memory address,
    // and skip staging its sources' slice
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    static_assert(kN == 8 * (kThreads / 32) && kK == 32, "one source per four lanes, eight groups of four columns");
    const int src_j = jt * kN + 8 * warp + (lane >> 2);
    const bool use_j = src_j < nb && (!active || active[src_j]);
    for (int i = 0; i < nch; ++i) {
        const int st = i & 1, kc = c0 + i;
        const unsigned ph = (unsigned)(i >> 1) & 1u;
        // stage st was last read by the MMAs of chunk i - 2; after an abort the
        // stage is no longer written (those MMAs may not have finished)
        if (i >= 2 && !pipe::mbar_wait_drain(&S.mbar[st], ph ^ 1u)) S.abort = 1;
        tc_fence_after();
        // this chunk's slice of R, split into TF32 hi and lo planes. Thread
        // (warp w, lane l) owns source j = 8 w + l / 4 and columns 4 g + l % 4,
        // g = 0..7: all eight loads are issued first, and each warp's stores
        // cover 32 consecutive floats of a plane (one core-matrix row group)
        if (!*(volatile int *)&S.abort) {
            float2 v[kK / 4];
            const size_t base = (size_t)src_j * sr + (size_t)kc * kK + (lane & 3);
#pragma unroll
            for (int g = 0; g < kK / 4; ++g) {
                v[g] = make_float2(0.f, 0.f);
                if (use_j && kc * kK + 4 * g + (lane & 3) < G.n) v[g] = R[base + 4 * g];
            }
#pragma unroll
            for (int g = 0; g < kK / 4; ++g) {
                const int o = (warp * (kK / 4) + g) * 32 + lane;   // = cm_off(8 w + l / 4, 4 g + l % 4)
                const float rh = tf32_hi(v[g].x), ih = tf32_hi(v[g].y);
                S.b[st][0][o] = rh;
                S.b[st][1][o] = v[g].x - rh;
                S.b[st][2][o] = ih;
                S.b[st][3][o] = v[g].y - ih;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> MMA reads
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0) {
            const uint32_t tmem = S.tmem;
            if (pipe::mbar_wait(&S.abar[st], ph, &S.abort)) {
                // D f32, A and B tf32, both K-major, N = 64, M = 128; bit 14 negates B
                const uint32_t idp = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                                     ((uint32_t)(kM >> 4) << 24);
                const uint32_t idn = idp | (1u << 14);
                const uint32_t dr = tmem, di = tmem + kN;
                constexpr unsigned lbo = 128, sbo = (kK / 4) * 128;
#pragma unroll
                for (int s = 0; s < kK / 8; ++s) {
                    uint64_t a[4], b[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        a[q] = smem_desc(&S.a[st][q][s * 64], lbo, sbo);
                        b[q] = smem_desc(&S.b[st][q][s * 64], lbo, sbo);
                    }
                    const uint32_t acc = (i > 0 || s > 0) ? 1u : 0u;
                    // Zr += Ar Rr - Ai Ri
                    mma_tf32(dr, a[0], b[0], idp, acc);
                    mma_tf32(dr, a[0], b[1], idp, 1);
                    mma_tf32(dr, a[1], b[0], idp, 1);
                    mma_tf32(dr, a[2], b[2], idn, 1);
                    mma_tf32(dr, a[2], b[3], idn, 1);
                    mma_tf32(dr, a[3], b[2], idn, 1);
                    // Zi += Ai Rr + Ar Ri
                    mma_tf32(di, a[2], b[0], idp, acc);
                    mma_tf32(di, a[2], b[1], idp, 1);
                    mma_tf32(di, a[3], b[0], idp, 1);
                    mma_tf32(di, a[0], b[2], idp, 1);
                    mma_tf32(di, a[0], b[3], idp, 1);
                    mma_tf32(di, a[1], b[2], idp, 1);
                }
            }
            // arrives once the MMAs issued so far (if any) have completed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             pipe::smem_addr(&S.mbar[st]))
                         : "memory");
            // refill the other stage with chunk i + 1 once chunk i - 1's MMAs
            // have read it (chunk 1 was issued up front)
            if (i >= 1 && i + 1 < nch) {
                const int so = st ^ 1;
                if (pipe::mbar_wait(&S.mbar[so], (unsigned)((i - 1) >> 1) & 1u, &S.abort)) copy_a(i + 1);
            }
        }
        __syncwarp();
    }
    const uint32_t tmem = S.tmem;
    {
        // the accumulators are read and TMEM is freed only after the last
        // MMAs have completed: a wait that runs out is retried (each bounded)
        // before the block gives up on them
        const int il = nch - 1;
        bool done = false;
        for (int a = 0; a < 4 && !done; ++a) done = pipe::mbar_wait_drain(&S.mbar[il & 1], (unsigned)(il >> 1) & 1u);
        if (!done) S.abort = 1;
    }
    __syncthreads();   // every thread sees the same abort word
    tc_fence_after();
    // warps 0-3 read the real accumulator, 4-7 the imaginary one; warp w sees
    // TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 = rows of the block
    const int qtr = warp & 3, plane = warp >> 2;
    uint32_t v[64];
    tmem_ld64(tmem + ((uint32_t)(32 * qtr) << 16) + (uint32_t)(plane * kN), v);
    const int row = rt * kM + 32 * qtr + lane;
    const bool bad = S.abort != 0;
    float *dst = part + ((size_t)(kg * 2 + plane) * nb + (size_t)jt * kN) * G.Mp + row;
    const int ncol = min(kN, nb - jt * kN);   // padding columns are not stored
#pragma unroll
    for (int c = 0; c < kN; ++c)
        if (c < ncol) dst[(size_t)c * G.Mp] = bad ? __int_as_float(0x7fc00000) : __uint_as_float(v[c]);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    // after an abort, wait (bounded) for the last Ainv copy of each stage before the CTA exits
    if (t == 0 && bad)
        for (int st = 0; st < 2; ++st)
            if (issued[st]) pipe::mbar_wait_drain(&S.abar[st], (issued[st] - 1) & 1u);
}

// Z[source][row] = sum over column groups kg, in group order, of the partials
// (eight groups' loads in flight at a time)
__global__ void __launch_bounds__(256)
k_coarse_tc_sum(const float *__restrict__ part, TcGeom G, float2 *__restrict__ Z, size_t sz, int nb,
                const int *__restrict__ active) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x, src = blockIdx.y;
    if (row >= G.n || src >= nb || (active && !active[src])) return;
    const size_t plane = (size_t)nb * G.Mp;
    const float *p = part + (size_t)src * G.Mp + row;
    float re = 0.f, im = 0.f;
    int kg = 0;
    for (; kg + 8 <= G.nkg; kg += 8) {
        float a[8], b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            a[u] = p[(size_t)(2 * (kg + u)) * plane];
            b[u] = p[(size_t)(2 * (kg + u) + 1) * plane];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            re += a[u];
            im += b[u];
        }
    }
    for (; kg < G.nkg; ++kg) {
        re += p[(size_t)(2 * kg) * plane];
        im += p[(size_t)(2 * kg + 1) * plane];
    }
    Z[(size_t)src * sz + row] = make_float2(re, im);
}

}  // namespace

size_t coarse_tc_tile_floats(int n) {
    const TcGeom g = tc_geom(n, 1);
    return (size_t)g.nrt * g.nkc * 4 * kAPlane;
}

size_t coarse_tc_part_floats(int n, int nb) {
    const TcGeom g = tc_geom(n, nb);
    return (size_t)g.nkg * 2 * nb * g.Mp;
}

void launch_coarse_tc_tiles(const float2 *At, int n, float *tiles, cudaStream_t st) {
    const TcGeom g = tc_geom(n, 1);
    k_coarse_tc_tiles<<<dim3((g.Mp + 255) / 256, g.nkc * kK), 256, 0, st>>>(At, g, tiles);
    count_launch();
}

void launch_coarse_tc(const float *tiles, int n, const float2 *r, size_t sr, float2 *z, size_t sz,
                      int nb, const int *active, float *part, cudaStream_t st) {
    static const int once = [] {
        cudaFuncSetAttribute(k_coarse_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
        return 1;
    }();
    (void)once;
    const TcGeom g = tc_geom(n, nb);
    prof_begin(st);
    k_coarse_tc<<<dim3(g.nkg, g.nrt, g.nsb), kThreads, sizeof(TcSmem), st>>>(tiles, g, r, sr, part,
                                                                                   nb, active);
    k_coarse_tc_sum<<<dim3((n + 255) / 256, nb), 256, 0, st>>>(part, g, z, sz, nb, active);
    count_launch(2);
    if (prof_on()) {
        // Ainv planes once per source block, R and Z once
        const double ab = (double)g.nrt * g.nkc * 4 * kAPlane * 4.0 * g.nsb;
        prof_end("coarse_tc", st, ab + 16.0 * n * (double)nb, 0.0);
    }
}

}  // namespace helm
