// wave_pass.cuh -- the pipelined pass kernel of libwave.so (instantiated per
// stencil radius in wave_pass_r*.cu).
//
// The kernel advances the damped acoustic wave equation
//     u^{n+1} = ((dt d - 2m) u^{n-1} + 4m u^n + 2dt^2 (L_h u^n + q^n)) / (dt d + 2m)
// (McCormick 2017, Fig. acoustic_devito).  Dividing by 2m and writing the
// increment v^{n+1/2} = u^{n+1} - u^n gives the same recurrence as
//     v^{n+1/2} = ((1 - g) v^{n-1/2} + kappa (L_h u^n + q^n)) / (1 + g),
//     u^{n+1}   = u^n + v^{n+1/2},
//     kappa = dt^2 / m,  g = dt d / (2m) = d kappa / (2 dt),
// which the kernel steps with the state (u^n, v^{n-1/2}).  In exact
// arithmetic the two are identical; in float32 carrying v keeps the rounding
// of u^{n+1} out of the velocity, where leapfrog would amplify it by
// 1 / sin(omega dt) at every step.
//
// One pass advances T time steps over HBM (Chapter "Time-Tiling").  Each
// thread block owns an output tile by x bz in the y-z plane and streams
// through a slab of x planes.  The T steps form a pipeline along x: step k
// works on plane x_k = x_0 - k r (r = SO/2), r planes behind step k-1 -- the
// skew by r per time step that makes tiling through time legal (Section
// "Skewing Dependencies").  In the y-z plane the tile carries an overlapped
// halo of r (T - k) points at step k, so no block depends on another within a
// pass; outputs go to a second buffer set, so no write-after-read hazard
// crosses blocks (the paper's rolling time buffer bounds the time tile by its
// modulus instead, Section "Time Dimension Buffering").
//
// Data movement per iteration (one x plane per step):
//   * TMA (cp.async.bulk.tensor) stages the plane of u^n with its halo, and
//     the planes of v^{n-1/2} and kappa, into a shared-memory ring completed
//     on mbarriers; out-of-range boxes are zero-filled by the TMA unit, which
//     is the zero Dirichlet ghost layer.
//   * Every thread owns a column of 4 consecutive z points (128-bit loads and
//     stores) and keeps, per step, a register queue of the 2r + 1 planes of
//     its column along x: the x neighbours never touch shared memory.
//   * In-plane (y, z) neighbours of step k come from shared memory: step 1
//     reads the TMA ring, step k >= 2 a plane buffer that the threads fill
//     from the centres of their queues once per iteration.
//   * The increment of step k-1 at plane x_k, produced r iterations earlier,
//     waits in a thread-private shared-memory ring until step k needs it.
//   * One __syncthreads per iteration.
//
// Every arithmetic operation of the point update is an explicit
// round-to-nearest intrinsic in one fixed order (per-axis partial sums of the
// Laplacian, sources, increment, field; the k = 1 pairs as differences from
// the centre), so a pass with T = 1 and passes with
// T > 1 produce bit-identical fields: tiling only reorders independent
// updates.
#pragma once
#include "wave_kernels.cuh"

#include <climits>
#include <type_traits>
#include <utility>

namespace wave {
namespace detail {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // bound on any wait: 2 s

template <int R, int T>
struct Cfg {
    static constexpr int D = (R == 8) ? 2 : 3;    // iterations loaded ahead
    static constexpr int P = 2 * R + 1;           // queue length along x
    static constexpr int ZH = (R + 3) & ~3;       // z halo of the staged box, rounded to 4
    static constexpr int NQ = ZH / 4;             // halo quads on each side
    static constexpr int NA = D + R + 1;          // ring slots of u^n planes
    static constexpr int NB = D + 1;              // ring slots of (v^{n-1/2}, kappa) planes
    static constexpr int NV = R + 1;              // delay slots of the increments (steps >= 2)
};

// Compile-time geometry of a thread block: RY rows of QZ z quads; the staged
// u^n box adds r rows and ZH columns on each side.
template <int R, int T, int QZ, int RY>
struct Geo {
    static constexpr int ZH = Cfg<R, T>::ZH;
    static constexpr int NTHR = QZ * RY;
    static constexpr int B_COLS = 4 * QZ, B_ROWS = RY;
    static constexpr int A_COLS = B_COLS + 2 * ZH, A_ROWS = RY + 2 * R;
    static constexpr int AFL = (A_ROWS * A_COLS + 31) & ~31;  // floats per u^n slot (128-byte aligned)
    static constexpr int BFL = (B_ROWS * B_COLS + 31) & ~31;  // floats per v or kappa plane
    static_assert(NTHR % 32 == 0, "whole warps");
    static_assert(A_COLS <= 256 && A_ROWS <= 256, "TMA box limit");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier, giving up after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitLimitNs)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Tensor memory (TMEM, 512 columns x 128 lanes of 32 bits per SM).  A warp
// reaches only the 32 lanes of its quarter (warp index % 4 within the CTA):
// lane l of the quarter belongs to thread l of the warp, so each thread has a
// private row of columns.  Every tcgen05 instruction here is executed by all
// 32 threads of a warp together (.sync.aligned), always outside divergent
// branches.
__device__ __forceinline__ void tmem_alloc(uint32_t smem_dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_dst), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const float4& v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
                 "r"(__float_as_uint(v.w)));
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;"); }
// tmem_ld_xN starts a load of N consecutive columns of the thread's lane into
// r; tmem_wait_ld(r) waits for every load the thread has started and makes r
// usable (the registers are its operands, so no use of r can move above it).
// The tcgen05 loads, stores and waits touch no memory the compiler sees: they
// carry no memory clobber, so shared-memory loads and stores may be scheduled
// across them; their order among themselves is kept (asm volatile).
__device__ __forceinline__ void tmem_ld_x4(uint32_t taddr, uint32_t (&r)[4])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {"
        "%0, %1, %2, %3}, [%4];"
        :
          "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[4])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 :
                   "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]));
}
__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {"
        "%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        :
          "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 :
                   "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]));
}
__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {"
        "%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, "
        "%20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        :
          "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 :
                   "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]),
                   "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]),
                   "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}
__device__ __forceinline__ void tmem_ld_x64(uint32_t taddr, uint32_t (&r)[64])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {"
        "%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, "
        "%20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, "
        "%38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, "
        "%56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
        :
          "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]),
          "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]),
          "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]),
          "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]),
          "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[64])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 :
                   "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]),
                   "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]),
                   "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]), "+r"(r[32]), "+r"(r[33]), "+r"(r[34]),
                   "+r"(r[35]), "+r"(r[36]), "+r"(r[37]), "+r"(r[38]), "+r"(r[39]), "+r"(r[40]), "+r"(r[41]),
                   "+r"(r[42]), "+r"(r[43]), "+r"(r[44]), "+r"(r[45]), "+r"(r[46]), "+r"(r[47]), "+r"(r[48]),
                   "+r"(r[49]), "+r"(r[50]), "+r"(r[51]), "+r"(r[52]), "+r"(r[53]), "+r"(r[54]), "+r"(r[55]),
                   "+r"(r[56]), "+r"(r[57]), "+r"(r[58]), "+r"(r[59]), "+r"(r[60]), "+r"(r[61]), "+r"(r[62]),
                   "+r"(r[63]));
}


template <int... Is, class F>
__device__ __forceinline__ void static_for_impl(std::integer_sequence<int, Is...>, F& f)
{
    (f(std::integral_constant<int, Is>{}), ...);
}

// f(std::integral_constant<int, S>) for S = 0 .. N-1, fully unrolled.
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f)
{
    static_for_impl(std::make_integer_sequence<int, N>{}, f);
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float lane_of(const float4& v, int l)
{
    return l == 0 ? v.x : (l == 1 ? v.y : (l == 2 ? v.z : v.w));
}

// Packed float32 pairs (sm_100+: one instruction, two IEEE round-to-nearest
// operations, each bit-identical to its scalar counterpart).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 c, float2 x, float2 acc) { return __ffma2_rn(c, x, acc); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// L_h u at the 4 points of a column quad, in the one fixed order every kernel
// uses: three partial sums, Ly = centre + y pairs k = 1..r, Lz = z pairs,
// Lx = x pairs (each accumulated in k order), then L = (Ly + Lz) + Lx.  The
// k = 1 pairs enter as exact differences (u(+1) - u) + (u(-1) - u); their
// share of the centre weight is left out of c0.  For a smooth field the
// centre term and the neighbour sums nearly cancel, and summing the dominant
// k = 1 pair as differences keeps float32 rounding from swamping L_h u (the
// differences of neighbouring values are exact).  Lanes 0-1 and 2-3 are
// computed as packed pairs.

// L += coef * s (the first term of a chain is a plain product)
__device__ __forceinline__ void acc2(float2& L, float2 coef, float2 s, bool first)
{
    L = first ? __fmul2_rn(coef, s) : fma2(coef, s, L);
}

// One neighbour pair (m, p) of the centre quad c into both halves of a chain.
__device__ __forceinline__ void pair2(float2& Ll, float2& Lh, float2 coef, const float4& m, const float4& p,
                                      const float4& c, bool diff, bool first)
{
    if (diff) {
        const float2 ncl = neg2(lo2(c)), nch = neg2(hi2(c));
        acc2(Ll, coef, add2(add2(lo2(m), ncl), add2(lo2(p), ncl)), first);
        acc2(Lh, coef, add2(add2(hi2(m), nch), add2(hi2(p), nch)), first);
    } else {
        acc2(Ll, coef, add2(lo2(m), lo2(p)), first);
        acc2(Lh, coef, add2(hi2(m), hi2(p)), first);
    }
}

// Ly of the quad with centre c (the centre term and the y pairs);
// yq(k) is the quad k rows away, k = -r .. r, called with compile-time k.
template <int R, class YQ>
__device__ __forceinline__ void laplacian_y(const float4& c, const YQ& yq, const PassArgs& a, float2& yl, float2& yh)
{
    yl = __fmul2_rn(a.c0, lo2(c));
    yh = __fmul2_rn(a.c0, hi2(c));
    static_for<R>([&](auto kc) {
        constexpr int k = decltype(kc)::value + 1;
        pair2(yl, yh, a.cy[k - 1], yq(std::integral_constant<int, -k>{}), yq(std::integral_constant<int, k>{}), c,
              k == 1, false);
    });
}

// Lz of the quad with centre c.  plane: shared-memory plane holding u of
// this step's input level at the current x with a halo of ZH columns; pos:
// the quad's own index.
template <int R>
__device__ __forceinline__ void laplacian_z(const float* plane, int pos, const float4& c, const PassArgs& a,
                                            float2& zl, float2& zh)
{
    constexpr int NQ = ((R + 3) & ~3) / 4;
    // z window: the centre quad and NQ quads on each side, one float per point
    float w[4 * (2 * NQ + 1)];
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        const float4 lft = lds4(plane + pos - 4 * (NQ - j));
        const float4 rgt = lds4(plane + pos + 4 * (j + 1));
        w[4 * j + 0] = lft.x; w[4 * j + 1] = lft.y; w[4 * j + 2] = lft.z; w[4 * j + 3] = lft.w;
        w[4 * (NQ + 1 + j) + 0] = rgt.x; w[4 * (NQ + 1 + j) + 1] = rgt.y;
        w[4 * (NQ + 1 + j) + 2] = rgt.z; w[4 * (NQ + 1 + j) + 3] = rgt.w;
    }
    w[4 * NQ + 0] = c.x; w[4 * NQ + 1] = c.y; w[4 * NQ + 2] = c.z; w[4 * NQ + 3] = c.w;
    constexpr int o = 4 * NQ;
    static_for<R>([&](auto kc) {
        constexpr int k = decltype(kc)::value + 1;
        if constexpr (k == 1) {
            // (m - c) + (p - c) per lane from the neighbour differences
            // e_j = w[o+j] - w[o+j-1]: m - c = -e_j and p - c = e_{j+1} exactly,
            // so the pair is e_{j+1} - e_j, shared between adjacent lanes
            float e[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) e[j] = __fsub_rn(w[o + j], w[o + j - 1]);
            acc2(zl, a.cz[0], f2(__fsub_rn(e[1], e[0]), __fsub_rn(e[2], e[1])), true);
            acc2(zh, a.cz[0], f2(__fsub_rn(e[3], e[2]), __fsub_rn(e[4], e[3])), true);
        } else if constexpr (k % 2 == 1) {
            // odd shift: the lane pairs of m and p straddle register pairs, so
            // the sums are formed lane by lane into aligned pairs
            acc2(zl, a.cz[k - 1], f2(__fadd_rn(w[o - k], w[o + k]), __fadd_rn(w[o + 1 - k], w[o + 1 + k])), false);
            acc2(zh, a.cz[k - 1], f2(__fadd_rn(w[o + 2 - k], w[o + 2 + k]), __fadd_rn(w[o + 3 - k], w[o + 3 + k])),
                 false);
        } else {
            const float4 m = make_float4(w[o - k], w[o + 1 - k], w[o + 2 - k], w[o + 3 - k]);
            const float4 p = make_float4(w[o + k], w[o + 1 + k], w[o + 2 + k], w[o + 3 + k]);
            pair2(zl, zh, a.cz[k - 1], m, p, c, false, false);
        }
    });
}

// Ly and Lz of the quad with centre c.  plane: shared-memory plane holding u
// of this step's input level at the current x with a halo of r rows and ZH
// columns; pos: the quad's own index.
template <int R>
__device__ __forceinline__ void laplacian_yz(const float* plane, int pos, int pitch, const float4& c,
                                             const PassArgs& a, float2& yl, float2& yh, float2& zl, float2& zh)
{
    laplacian_y<R>(c, [&](auto kc) { return lds4(plane + pos + decltype(kc)::value * pitch); }, a, yl, yh);
    laplacian_z<R>(plane, pos, c, a, zl, zh);
}

// Lx of the quad with centre c; xq(j) is the quad's u at logical plane j of
// 0 .. 2r along x (centre r), called with compile-time j.
template <int R, class XQ>
__device__ __forceinline__ void laplacian_x(const float4& c, const XQ& xq, const PassArgs& a, float2& xl, float2& xh)
{
    static_for<R>([&](auto kc) {
        constexpr int k = decltype(kc)::value + 1;
        pair2(xl, xh, a.cx[k - 1], xq(std::integral_constant<int, R - k>{}), xq(std::integral_constant<int, R + k>{}),
              c, k == 1, k == 1);
    });
}

__device__ __forceinline__ float4 combine(float2 yl, float2 yh, float2 zl, float2 zh, float2 xl, float2 xh)
{
    const float2 Ll = add2(add2(yl, zl), xl);
    const float2 Lh = add2(add2(yh, zh), xh);
    return make_float4(Ll.x, Ll.y, Lh.x, Lh.y);
}

// New increment of the 4 points of a quad, ((1 - g) v + kappa L) / (1 + g)
// with g = d kappa / (2 dt), and the field u + v.  Where g == 0 the increment
// is fma(kappa, L, v) on both paths ((1 - 0) v is v), so whether a warp takes
// the damped or the undamped branch never changes a result; where g > 0 the
// quotient is formed with the fast reciprocal (__fdividef, 2 ulp), the same
// instructions in every kernel.
__device__ __forceinline__ void update4(const float4& L, float4& u, float4& v, const float4& kap, float dx,
                                        const float4& dyz, bool dyz_zero, float inv2dt)
{
    const float2 kl = lo2(kap), kh = hi2(kap);
    float2 vl, vh;
    // warp-uniform: the damped path only where some lane of the warp is in the sponge
    if (!__any_sync(0xffffffffu, !(dx == 0.f && dyz_zero))) {
        vl = __ffma2_rn(kl, lo2(L), lo2(v));
        vh = __ffma2_rn(kh, hi2(L), hi2(v));
    } else {
        const float2 dx2 = f2(dx, dx), i2 = f2(inv2dt, inv2dt), one = f2(1.f, 1.f);
        const float2 gl = __fmul2_rn(__fmul2_rn(__fadd2_rn(dx2, lo2(dyz)), kl), i2);
        const float2 gh = __fmul2_rn(__fmul2_rn(__fadd2_rn(dx2, hi2(dyz)), kh), i2);
        const float2 nl = __ffma2_rn(kl, lo2(L), __ffma2_rn(neg2(gl), lo2(v), lo2(v)));
        const float2 nh = __ffma2_rn(kh, hi2(L), __ffma2_rn(neg2(gh), hi2(v), hi2(v)));
        const float2 dl = __fadd2_rn(one, gl), dh = __fadd2_rn(one, gh);
        vl = f2(gl.x == 0.f ? nl.x : __fdividef(nl.x, dl.x), gl.y == 0.f ? nl.y : __fdividef(nl.y, dl.y));
        vh = f2(gh.x == 0.f ? nh.x : __fdividef(nh.x, dh.x), gh.y == 0.f ? nh.y : __fdividef(nh.y, dh.y));
    }
    v = make_float4(vl.x, vl.y, vh.x, vh.y);
    const float2 ul = __fadd2_rn(lo2(u), vl);
    const float2 uh = __fadd2_rn(hi2(u), vh);
    u = make_float4(ul.x, ul.y, uh.x, uh.y);
}

// First CSR entry of [lo, hi) whose x is >= x0.
template <class E>
__device__ __forceinline__ int first_at_or_after(const E* ent, int lo, int hi, int x0)
{
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ent[mid].x < x0) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Storage of the per-step x queues (template parameter QM):
//   0: registers, moved down one slot per iteration;
//   1: registers, the loop unrolled over the queue length so that the slot
//      of a plane rotates instead of moving;
//   2: tensor memory.  Each warp keeps, per step, a ring of the 2r previous
//      planes of its threads' column quads, every plane written twice (slots
//      s and s + 2r), so that the window of any iteration is 2r consecutive
//      columns: one tcgen05.ld brings it into registers, which the stencil
//      reads in place, and the newest plane stays in registers.  Nothing
//      moves, and the queues hold no registers between iterations.
template <int R, int T, int QZ, int RY>
struct TmemGeo {
    static constexpr int NW = QZ * RY / 32;         // warps of the block
    static constexpr int WPQ = (NW + 3) / 4;        // warps sharing a lane quarter
    static constexpr int CPS = 16 * R;              // columns per step and warp: 2 x 2r planes x 4
    static constexpr int CPW = T * CPS;             // columns per warp
    static constexpr int NEED = WPQ * CPW;
    static constexpr int COLS = NEED <= 32 ? 32 : NEED <= 64 ? 64 : NEED <= 128 ? 128 : NEED <= 256 ? 256 : 512;
    static constexpr bool fits = NEED <= 512;
};

template <int R, int T, int QZ, int RY, int QM>
constexpr int min_blocks()
{
    // one-step kernels keep 512 threads resident per SM (128 registers), or
    // 256 at radius 8 when the queue lives in registers (its 17 planes do
    // not fit in 128); T > 1 kernels may use the whole register file.
    return (T == 1 && QZ * RY < 512) ? ((R == 8 && QM != 2) ? (256 / (QZ * RY) > 0 ? 256 / (QZ * RY) : 1)
                                                             : 512 / (QZ * RY))
                                     : 1;
}

// Programmatic dependent launch of consecutive passes in a stream: a pass
// lets the next one be scheduled once every one of its blocks has left its
// plane loop (grid_dep_launch), and the next one runs its prologue (tensor
// memory, mbarriers, tap lookups) on SMs that free up, then waits in
// grid_dep_wait until the previous pass has completed and its writes are
// visible, before it touches the fields.  Without the launch attribute both
// are no-ops.
__device__ __forceinline__ void grid_dep_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void grid_dep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch a pass kernel with programmatic stream serialisation allowed.
template <class... P, class... A>
cudaError_t launch_dependent(void (*fn)(P...), long long blocks, int threads, size_t smem, cudaStream_t st,
                             A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, std::forward<A>(args)...);
}

__device__ __forceinline__ void mbar_inval(uint32_t bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// Imaging condition of the FWI gradient at the four points of a z quad
// (element offset off of the padded layout): g += -(scale mu) (v_new - v_old),
// the adjoint field mu times dt^2 D_tt u of the forward, where
// dt^2 D_tt u^{j-1} = v^{j-1/2} - v^{j-3/2}.  Each point is written by the
// one thread that owns it in a one-step pass.
// The operands are loaded where the point is written: loading them earlier
// keeps their registers live through the stencil of every pass, which cost
// the radius-8 pass registers and speed, and did not make the gradient faster.
__device__ __forceinline__ void image4(const PassArgs& a, long long off, const float4& mu)
{
    float4 g = *reinterpret_cast<const float4*>(a.gacc + off);
    const float4 vn = __ldg(reinterpret_cast<const float4*>(a.img_vn + off));
    const float4 vo = __ldg(reinterpret_cast<const float4*>(a.img_vo + off));
    const float s = a.img_scale;
    g.x = __fmaf_rn(-__fmul_rn(s, mu.x), __fsub_rn(vn.x, vo.x), g.x);
    g.y = __fmaf_rn(-__fmul_rn(s, mu.y), __fsub_rn(vn.y, vo.y), g.y);
    g.z = __fmaf_rn(-__fmul_rn(s, mu.z), __fsub_rn(vn.z, vo.z), g.z);
    g.w = __fmaf_rn(-__fmul_rn(s, mu.w), __fsub_rn(vn.w, vo.w), g.w);
    *reinterpret_cast<float4*>(a.gacc + off) = g;
}

// The threads that run one tile: the whole block (bar = 0), or one of
// several teams of a block, each with a named barrier of its own.  tid is the
// thread's index within the team.
struct Team {
    int tid;
    int bar;
    int nthreads;
};

__device__ __forceinline__ void team_sync(const Team& t)
{
    if (t.bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(t.bar), "r"(t.nthreads) : "memory");
}

// One output tile (thread block `blk` of the pass's grid) of a pass: the
// body of pass_kernel, and the work item of the persistent batched kernel.
// mapA, mapV, mapK: tensor maps (kernel parameters or global memory); a:
// the pass arguments (kernel parameter or constant memory), with n0 the time
// level at the start of the pass (in place of a.n0); tmem_base: the block's
// tensor-memory allocation (QM = 2; at least TmemGeo::COLS columns); reuse:
// the block runs another tile after this one, so the tile's mbarriers are
// invalidated at its end.
template <int R, int T, int QZ, int RY, int QM>
__device__ __forceinline__ void pass_tile(const CUtensorMap* mapA, const CUtensorMap* mapV, const CUtensorMap* mapK,
                                          const PassArgs& a, int n0, long long blk, unsigned char* smem,
                                          uint32_t tmem_base, bool reuse, const Team& team)
{
    using C = Cfg<R, T>;
    using G = Geo<R, T, QZ, RY>;
    using TG = TmemGeo<R, T, QZ, RY>;
    constexpr bool TQ = QM == 2;
    static_assert(!TQ || TG::fits, "tensor-memory queues exceed 512 columns");
    constexpr int P = C::P, NA = C::NA, NB = C::NB, NV = C::NV, ZH = C::ZH, kPrefetch = C::D;
    constexpr int afl = G::AFL, bfl = G::BFL, pitch = G::A_COLS, NTHR = G::NTHR;
    constexpr int R2 = 2 * R;
    constexpr uint32_t hdr = (8u * (NA + NB) + 8u + 127u) & ~127u;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    volatile int* s_abort = reinterpret_cast<volatile int*>(smem + 8 * (NA + NB));
    // disjoint regions: the TMA rings, the published planes, the increment ring
    float* __restrict__ ringA = reinterpret_cast<float*>(smem + hdr);
    float* __restrict__ ringB = ringA + NA * afl;
    float* __restrict__ planes = ringB + NB * 2 * bfl;
    float4* __restrict__ vring = reinterpret_cast<float4*>(planes + 2 * (T - 1) * afl);
    constexpr uint32_t txA = static_cast<uint32_t>(G::A_ROWS * G::A_COLS * 4);
    constexpr uint32_t txB = static_cast<uint32_t>(2 * G::B_ROWS * G::B_COLS * 4);

    // thread block -> tile (z fastest, then y, then x slab)
    const int tzi = static_cast<int>(blk % a.ntz);
    blk /= a.ntz;
    const int tyi = static_cast<int>(blk % a.nty);
    const int xsi = static_cast<int>(blk / a.nty);
    const int y0 = tyi * a.by, z0 = tzi * a.bz;
    const int X0 = xsi * a.xc, X1 = min(X0 + a.xc, a.nx);
    const int NIT = (X1 - X0) + 2 * R * T;
    const int xbase = X0 - R * T;  // x_0 of iteration 0
    const int ylo = y0 - R * (T - 1), zlo = z0 + a.zlead;

    // thread -> column quad.  Columns and planes outside the grid need no
    // special case: kappa is zero there (TMA zero fill, zero z padding), so
    // the update keeps u = v = 0 on them -- the zero ghost layer.
    const int tid = team.tid;
    const int ty = tid / QZ, tq = tid % QZ;
    const int gy = ylo + ty, gz = zlo + 4 * tq;
    const bool colv = gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nzp;
    const bool own = colv && gy >= y0 && gy < y0 + a.by && gz >= z0 && gz < z0 + a.bz;
    const int posA = (ty + R) * pitch + ZH + 4 * tq;
    const int posB = ty * G::B_COLS + 4 * tq;
    const long long colofs = static_cast<long long>(colv ? gy : 0) * a.nzp + (colv ? gz : 0);
    const int col = colv ? gy * (a.nzp >> 2) + (gz >> 2) : 0;

    float4 dyz = make_float4(0.f, 0.f, 0.f, 0.f);
    bool dyz_zero = true;
    if (colv) {
        const float dyv = a.damp_y[gy];
        dyz = make_float4(__fadd_rn(dyv, a.damp_z[gz]), __fadd_rn(dyv, a.damp_z[gz + 1]),
                          __fadd_rn(dyv, a.damp_z[gz + 2]), __fadd_rn(dyv, a.damp_z[gz + 3]));
        dyz_zero = dyz.x == 0.f && dyz.y == 0.f && dyz.z == 0.f && dyz.w == 0.f;
    }

    // Steps this warp computes.  Step k is needed on thread rows
    // [k R, RY - k R) (the output tile plus the halo of the later steps); a
    // warp whose rows all lie outside skips step k and every later one, and
    // keeps only the queue of step k (the outputs of step k - 1) that its
    // neighbours read.  Uniform over the warp.
    int wsteps = 0;
    {
        const int wr_lo = (tid & ~31) / QZ, wr_hi = ((tid & ~31) + 31) / QZ;
#pragma unroll
        for (int k = 0; k < T; ++k)
            if (wr_hi >= k * R && wr_lo < RY - k * R) wsteps = k + 1;
    }

    // sparse events per step: next x with a source or receiver tap in this column
    int scur[T], rcur[T], nxt[T], send = 0, rend = 0;
#pragma unroll
    for (int k = 0; k < T; ++k) { scur[k] = 0; rcur[k] = 0; nxt[k] = INT_MAX; }
    // (cursors always start inside the column's own CSR range [lo, end))
    if (colv && a.src_ptr != nullptr) {
        const int lo = a.src_ptr[col];
        send = a.src_ptr[col + 1];
#pragma unroll
        for (int k = 0; k < T; ++k) {
            scur[k] = lo < send ? first_at_or_after(a.src_ent, lo, send, X0 - R * (T - 1 - k)) : send;
            if (scur[k] < send) nxt[k] = a.src_ent[scur[k]].x;
        }
    }
    if (own && a.rec_ptr != nullptr) {
        const int lo = a.rec_ptr[col];
        rend = a.rec_ptr[col + 1];
        const int c0 = lo < rend ? first_at_or_after(a.rec_ent, lo, rend, X0) : rend;
#pragma unroll
        for (int k = 0; k < T; ++k) {
            rcur[k] = c0;
            if (c0 < rend) nxt[k] = min(nxt[k], a.rec_ent[c0].x);
        }
    }

    if (tid == 0) {
        for (int s = 0; s < NA + NB; ++s) mbar_init(smem_u32(&bars[s]), 1);
        *s_abort = 0;
        fence_mbar_init();
    }
    team_sync(team);
    // this warp's columns: lane quarter (warp % 4), column block (warp / 4)
    uint32_t twarp = 0;
    if constexpr (TQ) {
        const int warp = tid >> 5;
        twarp = tmem_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                static_cast<uint32_t>((warp >> 2) * TG::CPW);
    }
    // column of slot s (0 .. 4r - 1) of the ring of step k
    auto tcol = [&](int k, int s) { return twarp + static_cast<uint32_t>(k * TG::CPS + 4 * s); };

    auto issue = [&](int j) {
        const int x0 = xbase + j;
        const uint32_t ba = smem_u32(&bars[j % NA]);
        mbar_expect_tx(ba, txA);
        tma_load3(smem_u32(ringA + (j % NA) * afl), mapA, ba, zlo - ZH, ylo - R, x0);
        const uint32_t bb = smem_u32(&bars[NA + j % NB]);
        float* bs = ringB + (j % NB) * 2 * bfl;
        mbar_expect_tx(bb, txB);
        tma_load3(smem_u32(bs), mapV, bb, zlo, ylo, x0 - R);
        tma_load3(smem_u32(bs + bfl), mapK, bb, zlo, ylo, x0 - R);
    };
    int issued = 0;
    if (tid == 0) {
        for (int j = 0; j < kPrefetch && j < NIT; ++j) issue(j);
        issued = kPrefetch < NIT ? kPrefetch : NIT;
    }

    constexpr int QL = TQ ? 1 : P;  // register queue length
    float4 q[T][QL];
#pragma unroll
    for (int k = 0; k < T; ++k)
#pragma unroll
        for (int j = 0; j < QL; ++j) q[k][j] = make_float4(0.f, 0.f, 0.f, 0.f);

    // ring positions of iteration i, advanced incrementally
    int sA = 0, sAc = NA - R, sB = 0, vslot = 0;  // i % NA, (i - R) % NA, i % NB, i % NV
    int phA = 0, phB = 0;                         // (i / NA) & 1, (i / NB) & 1
    int ts = 0;                                   // i % 2r (tensor-memory ring slot)
    const long long sx = a.sx;
    bool abort = false;

    // One iteration with NACT active steps (compile time) and, if OUTP, the
    // write of the pass outputs.  Steps k >= NACT are not active yet: their
    // queues are filled (k == NACT) or untouched (k > NACT).
    // rot_c (register queues): -1 = the queues move down one slot per
    // iteration; S >= 0 = logical slot j lives at register (S + j) % P.
    auto body = [&](int i, auto nact_c, auto out_c, auto rot_c) {
        constexpr int NACT = decltype(nact_c)::value;
        constexpr bool OUTP = decltype(out_c)::value;
        constexpr int SR = decltype(rot_c)::value;
        constexpr int S = SR < 0 ? 0 : SR;
        constexpr bool MOVE = !TQ && SR < 0;
        (void)S;
        (void)MOVE;
        // kappa of steps k >= 1 at their planes, fetched early (cache hits)
        float4 kpre[T];
#pragma unroll
        for (int k = 1; k < T; ++k) {
            kpre[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < NACT && k < wsteps) {
                const int xk = xbase + i - (k + 1) * R;
                if (colv && xk >= 0 && xk < a.nx)
                    kpre[k] = __ldg(reinterpret_cast<const float4*>(a.kap + xk * sx + colofs));
            }
        }
        bool ok = mbar_wait(smem_u32(&bars[sA]), phA);
        ok = mbar_wait(smem_u32(&bars[NA + sB]), phB) && ok;
        if (!ok) {
            *s_abort = 1;
            atomicOr(a.err, 1);
        }
        // publish the centre planes x_k of active steps k >= 1 (the plane
        // their queue took r iterations ago)
        float4 ctr[T];
        if constexpr (TQ) {
            __syncwarp();
            tmem_wait_st();  // the previous iteration's ring writes
        }
#pragma unroll
        for (int k = 1; k < T; ++k) {
            ctr[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < NACT && k <= wsteps) {
                if constexpr (TQ) {
                    uint32_t r4[4];
                    tmem_ld_x4(tcol(k, ts + R < R2 ? ts + R : ts - R), r4);
                    tmem_wait_ld(r4);
                    ctr[k] = make_float4(__uint_as_float(r4[0]), __uint_as_float(r4[1]), __uint_as_float(r4[2]),
                                         __uint_as_float(r4[3]));
                } else {
                    ctr[k] = q[k][MOVE ? R + 1 : (S + R) % P];
                }
                sts4(planes + ((k - 1) * 2 + (i & 1)) * afl + posA, ctr[k]);
            }
        }
        team_sync(team);
        if (*s_abort) {
            if (tid == 0)
                for (int j = i; j < issued; ++j) {
                    mbar_wait(smem_u32(&bars[j % NA]), (j / NA) & 1);
                    mbar_wait(smem_u32(&bars[NA + j % NB]), (j / NB) & 1);
                }
            abort = true;
            return;
        }
        if (tid == 0 && i + kPrefetch < NIT) {
            issue(i + kPrefetch);
            issued = i + kPrefetch + 1;
        }
        const float* pnew = ringA + sA * afl;
        const float* pctr = ringA + sAc * afl;
        const float* pb = ringB + sB * 2 * bfl;
        const int vread = vslot == NV - 1 ? 0 : vslot + 1;  // slot of iteration i - R
        float4 prev_u = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 prev_v = prev_u;
#pragma unroll
        for (int k = 0; k < T; ++k) {
            if (k <= NACT && (k == 0 || k <= wsteps)) {
                // the newest plane of step k's queue: u^n from the TMA ring, or
                // the plane step k - 1 produced in this iteration
                const float4 newest = (k == 0) ? lds4(pnew + posA) : prev_u;
                if constexpr (!TQ) {
                    if (MOVE) {
#pragma unroll
                        for (int j = 0; j + 1 < P; ++j) q[k][j] = q[k][j + 1];
                    }
                    q[k][(S + 2 * R) % P] = newest;
                }
                if (k >= 1) vring[((k - 1) * NV + vslot) * NTHR + tid] = prev_v;
                if (k < NACT && k < wsteps) {
                    // step k+1 of the pass: u^{n0+k+1}, v^{n0+k+1/2} at plane xk
                    const int xk = xbase + i - (k + 1) * R;
                    const float* plane = (k == 0) ? pctr : planes + (((k - 1) * 2 + (i & 1)) * afl);
                    float2 yl, yh, zl, zh, xl, xh;
                    float4 u;
                    if constexpr (TQ) {
                        // window: the 2r planes before the newest, oldest first
                        uint32_t r[4 * R2];
                        if constexpr (R == 2) tmem_ld_x16(tcol(k, ts), r);
                        if constexpr (R == 4) tmem_ld_x32(tcol(k, ts), r);
                        if constexpr (R == 8) tmem_ld_x64(tcol(k, ts), r);
                        u = (k == 0) ? lds4(pctr + posA) : ctr[k];
                        laplacian_yz<R>(plane, posA, pitch, u, a, yl, yh, zl, zh);
                        tmem_wait_ld(r);
                        auto xq = [&](auto jc) -> float4 {
                            constexpr int j = decltype(jc)::value;
                            if constexpr (j == R2) {
                                return newest;
                            } else {
                                return make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                                   __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                            }
                        };
                        laplacian_x<R>(u, xq, a, xl, xh);
                    } else {
                        u = q[k][(S + R) % P];
                        laplacian_yz<R>(plane, posA, pitch, u, a, yl, yh, zl, zh);
                        auto xq = [&](auto jc) -> float4 { return q[k][(S + decltype(jc)::value) % P]; };
                        laplacian_x<R>(u, xq, a, xl, xh);
                    }
                    float4 L = combine(yl, yh, zl, zh, xl, xh);
                    if (xk == nxt[k]) {
                        // sources of this plane (before the update) ...
                        int c = scur[k];
                        while (c < send) {
                            const int4 e = a.src_ent[c];
                            if (e.x != xk) break;
                            const float w = __int_as_float(e.w);
                            const float qv = a.wavelet[static_cast<long long>(n0 + k) * a.nsrc + e.z];
                            if (e.y == 0) L.x = __fmaf_rn(w, qv, L.x);
                            else if (e.y == 1) L.y = __fmaf_rn(w, qv, L.y);
                            else if (e.y == 2) L.z = __fmaf_rn(w, qv, L.z);
                            else L.w = __fmaf_rn(w, qv, L.w);
                            ++c;
                        }
                        scur[k] = c;
                    }
                    float4 v = (k == 0) ? lds4(pb + posB) : vring[((k - 1) * NV + vread) * NTHR + tid];
                    const float4 kp = (k == 0) ? lds4(pb + bfl + posB) : kpre[k];
                    const float dx = (xk < a.dxlo || xk >= a.dxhi) ? a.damp_x[min(max(xk, 0), a.nx - 1)] : 0.f;
                    update4(L, u, v, kp, dx, dyz, dyz_zero, a.inv2dt);
                    if (xk == nxt[k]) {
                        // ... and receivers (after it); then the next event of this step
                        int c = rcur[k];
                        while (c < rend) {
                            const int2 e = a.rec_ent[c];
                            if (e.x != xk) break;
                            if (xk < X1)
                                a.slots[static_cast<long long>(n0 + k - a.slot_row0) * a.ntaps + (e.y >> 2)] =
                                    lane_of(u, e.y & 3);
                            ++c;
                        }
                        rcur[k] = c;
                        int nx2 = INT_MAX;
                        if (scur[k] < send) nx2 = a.src_ent[scur[k]].x;
                        if (rcur[k] < rend) nx2 = min(nx2, a.rec_ent[rcur[k]].x);
                        nxt[k] = nx2;
                    }
                    prev_u = u;
                    prev_v = v;
                }
                if constexpr (TQ) {
                    // the newest plane into the ring (slot i % 2r and its
                    // mirror), after this iteration's window was read
                    __syncwarp();
                    tmem_st4(tcol(k, ts), newest);
                    tmem_st4(tcol(k, ts + R2), newest);
                }
            }
        }
        if (OUTP && own) {
            // write u^{n+T} and v^{n+T-1/2} of plane x_T
            const long long off = (xbase + i - T * R) * sx + colofs;
            *reinterpret_cast<float4*>(a.out_u + off) = prev_u;
            *reinterpret_cast<float4*>(a.out_v + off) = prev_v;
            if constexpr (T == 1)
                if (a.gacc != nullptr) image4(a, off, prev_u);
        }
        // advance the ring positions
        vslot = vslot == NV - 1 ? 0 : vslot + 1;
        ts = ts == R2 - 1 ? 0 : ts + 1;
        if (++sA == NA) { sA = 0; phA ^= 1; }
        if (++sAc == NA) sAc = 0;
        if (++sB == NB) { sB = 0; phB ^= 1; }
    };

    using NoRot = std::integral_constant<int, -1>;
    int i = 0;
    static_for<T>([&](auto kc) {
        constexpr int k = decltype(kc)::value;  // steps 0 .. k-1 active in this phase
        const int end = 2 * (k + 1) * R;
        for (; i < end && !abort; ++i) body(i, std::integral_constant<int, k>{}, std::false_type{}, NoRot{});
    });
    if constexpr (QM == 1) {
        // steady state unrolled over the queue length.  After a moving
        // iteration logical slot j sits at register j and the newest plane at
        // 2r; the next iteration sees that plane as slot 2r - 1, which is
        // register (S + 2r - 1) % P for S = 1: the unrolled loop starts at
        // rotation 1 and writes its first new plane over register 0 (the
        // oldest, no longer read).
        for (int i0 = i; i0 < NIT && !abort; i0 += P)
            static_for<P>([&](auto sc) {
                constexpr int S = (decltype(sc)::value + 1) % P;
                if (i0 + decltype(sc)::value < NIT && !abort)
                    body(i0 + decltype(sc)::value, std::integral_constant<int, T>{}, std::true_type{},
                         std::integral_constant<int, S>{});
            });
    } else {
        for (; i < NIT && !abort; ++i) body(i, std::integral_constant<int, T>{}, std::true_type{}, NoRot{});
    }
    if constexpr (TQ) {
        // every warp is done with the tensor memory before it is freed or reused
        tmem_wait_st();
        tmem_fence_before();
    }
    if (TQ || reuse) team_sync(team);
    if constexpr (TQ) tmem_fence_after();
    if (reuse && tid == 0)
        for (int s = 0; s < NA + NB; ++s) mbar_inval(smem_u32(&bars[s]));
}

template <int R, int T, int QZ, int RY, int QM>
__global__ void __launch_bounds__(QZ * RY, min_blocks<R, T, QZ, RY, QM>())
    pass_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV,
                const __grid_constant__ CUtensorMap mapK, const PassArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    using TG = TmemGeo<R, T, QZ, RY>;
    constexpr bool TQ = QM == 2;
    // the tensor-memory address lives in the header word after the abort flag
    volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(smem + 8 * (Cfg<R, T>::NA + Cfg<R, T>::NB) + 4);
    uint32_t tbase = 0;
    if constexpr (TQ) {
        // warp 0 allocates the block's tensor memory (all 32 threads)
        if (threadIdx.x < 32) {
            tmem_alloc(smem_u32(const_cast<uint32_t*>(s_tmem)), TG::COLS);
            tmem_relinquish();
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        tbase = *s_tmem;
    }
    grid_dep_wait();
    pass_tile<R, T, QZ, RY, QM>(&mapA, &mapV, &mapK, a, a.n0, blockIdx.x, smem, tbase, false,
                                Team{static_cast<int>(threadIdx.x), 0, static_cast<int>(blockDim.x)});
    grid_dep_launch();
    if constexpr (TQ) {
        if (threadIdx.x < 32) tmem_dealloc(tbase, TG::COLS);
    }
}

// Shared memory of the (R, T, QZ, RY) instantiation.
template <int R, int T, int QZ, int RY>
constexpr size_t smem_bytes()
{
    using C = Cfg<R, T>;
    using G = Geo<R, T, QZ, RY>;
    return ((8u * (C::NA + C::NB) + 8u + 127u) & ~127u) +
           4u * (static_cast<size_t>(C::NA) * G::AFL + 2u * C::NB * G::BFL + 2u * (T - 1) * G::AFL) +
           16u * static_cast<size_t>(T - 1) * C::NV * G::NTHR;
}

template <int R, int T, int QZ, int RY, int QM>
cudaError_t launch_impl(const CUtensorMap& mapA, const CUtensorMap& mapV, const CUtensorMap& mapK,
                        const PassArgs& a, int threads, size_t smem, long long blocks, cudaStream_t st)
{
    auto fn = pass_kernel<R, T, QZ, RY, QM>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return launch_dependent(fn, blocks, threads, smem, st, mapA, mapV, mapK, a);
}

}  // namespace detail
}  // namespace wave
