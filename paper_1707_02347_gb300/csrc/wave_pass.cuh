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
// round-to-nearest intrinsic in one fixed order (centre, y pairs, z pairs,
// x pairs, sources, increment, field; the k = 1 pairs as differences from the
// centre), so a pass with T = 1 and passes with
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
__device__ __forceinline__ float2 fma2(float c, float2 x, float2 acc) { return __ffma2_rn(make_float2(c, c), x, acc); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// L_h u at the 4 points of a column quad, in the one fixed order every kernel
// uses: centre, then y pairs k = 1..r, then z pairs, then x pairs.  The
// k = 1 pairs enter as exact differences (u(+1) - u) + (u(-1) - u); their
// share of the centre weight is left out of c0.  For a smooth field the
// centre term and the neighbour sums nearly cancel, and summing the dominant
// k = 1 pair as differences keeps float32 rounding from swamping L_h u (the
// differences of neighbouring values are exact).  Lanes 0-1 and 2-3 are
// computed as packed pairs.
// plane: shared-memory plane holding u of this step's input level at the
// current x with a halo of r rows and ZH columns; pos: the quad's own index;
// q: the x queue, logical index j at physical (S + j) % P.
template <int R, int S>
__device__ __forceinline__ float4 laplacian4(const float* plane, int pos, int pitch, const float4 (&q)[2 * R + 1],
                                             const PassArgs& a)
{
    constexpr int P = 2 * R + 1;
    constexpr int NQ = ((R + 3) & ~3) / 4;
    const float4 c = q[(S + R) % P];
    const float2 cl = lo2(c), ch = hi2(c);
    const float2 ncl = neg2(cl), nch = neg2(ch);
    float2 Ll = __fmul2_rn(make_float2(a.c0, a.c0), cl);
    float2 Lh = __fmul2_rn(make_float2(a.c0, a.c0), ch);
    // one neighbour pair (m, p) of coefficient coef into both halves
    auto pair = [&](float coef, const float4& m, const float4& p, bool diff) {
        if (diff) {
            Ll = fma2(coef, add2(add2(lo2(m), ncl), add2(lo2(p), ncl)), Ll);
            Lh = fma2(coef, add2(add2(hi2(m), nch), add2(hi2(p), nch)), Lh);
        } else {
            Ll = fma2(coef, add2(lo2(m), lo2(p)), Ll);
            Lh = fma2(coef, add2(hi2(m), hi2(p)), Lh);
        }
    };
#pragma unroll
    for (int k = 1; k <= R; ++k) {
        const float4 m = lds4(plane + pos - k * pitch);
        const float4 p = lds4(plane + pos + k * pitch);
        pair(a.cy[k - 1], m, p, k == 1);
    }
    float v[4 * (2 * NQ + 1)];
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        const float4 lft = lds4(plane + pos - 4 * (NQ - j));
        const float4 rgt = lds4(plane + pos + 4 * (j + 1));
        v[4 * j + 0] = lft.x; v[4 * j + 1] = lft.y; v[4 * j + 2] = lft.z; v[4 * j + 3] = lft.w;
        v[4 * (NQ + 1 + j) + 0] = rgt.x; v[4 * (NQ + 1 + j) + 1] = rgt.y;
        v[4 * (NQ + 1 + j) + 2] = rgt.z; v[4 * (NQ + 1 + j) + 3] = rgt.w;
    }
    v[4 * NQ + 0] = c.x; v[4 * NQ + 1] = c.y; v[4 * NQ + 2] = c.z; v[4 * NQ + 3] = c.w;
#pragma unroll
    for (int k = 1; k <= R; ++k) {
        constexpr int o = 4 * NQ;
        const float4 m = make_float4(v[o - k], v[o + 1 - k], v[o + 2 - k], v[o + 3 - k]);
        const float4 p = make_float4(v[o + k], v[o + 1 + k], v[o + 2 + k], v[o + 3 + k]);
        pair(a.cz[k - 1], m, p, k == 1);
    }
#pragma unroll
    for (int k = 1; k <= R; ++k) pair(a.cx[k - 1], q[(S + R - k) % P], q[(S + R + k) % P], k == 1);
    return make_float4(Ll.x, Ll.y, Lh.x, Lh.y);
}

// New increment of one point: ((1 - g) v + kappa L) / (1 + g), g = d kappa / (2 dt).
// With g == 0 this is bit-identical to fma(kappa, L, v): (1 - 0) v is v and
// x / 1 is x, so whether a warp takes the damped or the undamped branch never
// changes a result.
__device__ __forceinline__ float increment(float L, float v, float kap, float g)
{
    return __fdiv_rn(__fmaf_rn(kap, L, __fmaf_rn(-g, v, v)), __fadd_rn(1.f, g));
}

__device__ __forceinline__ void update4(const float4& L, float4& u, float4& v, const float4& kap, float dx,
                                        const float (&dyz)[4], bool dyz_zero, float inv2dt)
{
    // warp-uniform: the damped path only where some lane of the warp is in the sponge
    if (!__any_sync(0xffffffffu, !(dx == 0.f && dyz_zero))) {
        const float2 vl = __ffma2_rn(lo2(kap), lo2(L), lo2(v));
        const float2 vh = __ffma2_rn(hi2(kap), hi2(L), hi2(v));
        v = make_float4(vl.x, vl.y, vh.x, vh.y);
    } else {
        v.x = increment(L.x, v.x, kap.x, __fmul_rn(__fmul_rn(__fadd_rn(dx, dyz[0]), kap.x), inv2dt));
        v.y = increment(L.y, v.y, kap.y, __fmul_rn(__fmul_rn(__fadd_rn(dx, dyz[1]), kap.y), inv2dt));
        v.z = increment(L.z, v.z, kap.z, __fmul_rn(__fmul_rn(__fadd_rn(dx, dyz[2]), kap.z), inv2dt));
        v.w = increment(L.w, v.w, kap.w, __fmul_rn(__fmul_rn(__fadd_rn(dx, dyz[3]), kap.w), inv2dt));
    }
    const float2 ul = __fadd2_rn(lo2(u), lo2(v));
    const float2 uh = __fadd2_rn(hi2(u), hi2(v));
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

// One-step kernels keep at least 512 threads resident per SM (their single
// x-queue fits in 128 registers); T > 1 kernels may use the whole register
// file for their queues.
template <int R, int T, int QZ, int RY, bool ROT>
__global__ void __launch_bounds__(QZ * RY, (T == 1 && QZ * RY < 512) ? 512 / (QZ * RY) : 1)
    pass_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV,
                const __grid_constant__ CUtensorMap mapK, const PassArgs a)
{
    using C = Cfg<R, T>;
    using G = Geo<R, T, QZ, RY>;
    constexpr int P = C::P, NA = C::NA, NB = C::NB, NV = C::NV, ZH = C::ZH, kPrefetch = C::D;
    constexpr int afl = G::AFL, bfl = G::BFL, pitch = G::A_COLS, NTHR = G::NTHR;
    constexpr uint32_t hdr = (8u * (NA + NB) + 4u + 127u) & ~127u;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    volatile int* s_abort = reinterpret_cast<volatile int*>(smem + 8 * (NA + NB));
    float* ringA = reinterpret_cast<float*>(smem + hdr);
    float* ringB = ringA + NA * afl;
    float* planes = ringB + NB * 2 * bfl;
    float4* vring = reinterpret_cast<float4*>(planes + 2 * (T - 1) * afl);
    constexpr uint32_t txA = static_cast<uint32_t>(G::A_ROWS * G::A_COLS * 4);
    constexpr uint32_t txB = static_cast<uint32_t>(2 * G::B_ROWS * G::B_COLS * 4);

    // thread block -> tile (z fastest, then y, then x slab)
    long long blk = blockIdx.x;
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
    const int tid = threadIdx.x;
    constexpr bool act = true;  // every thread of the block owns a column quad
    const int ty = tid / QZ, tq = tid % QZ;
    const int gy = ylo + ty, gz = zlo + 4 * tq;
    const bool colv = gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nzp;
    const bool own = colv && gy >= y0 && gy < y0 + a.by && gz >= z0 && gz < z0 + a.bz;
    const int posA = (ty + R) * pitch + ZH + 4 * tq;
    const int posB = ty * G::B_COLS + 4 * tq;
    const long long colofs = static_cast<long long>(colv ? gy : 0) * a.nzp + (colv ? gz : 0);
    const int col = colv ? gy * (a.nzp >> 2) + (gz >> 2) : 0;

    float dyz[4] = {0.f, 0.f, 0.f, 0.f};
    bool dyz_zero = true;
    if (colv) {
        const float dyv = a.damp_y[gy];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            dyz[l] = __fadd_rn(dyv, a.damp_z[gz + l]);
            dyz_zero = dyz_zero && (dyz[l] == 0.f);
        }
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
    __syncthreads();

    auto issue = [&](int j) {
        const int x0 = xbase + j;
        const uint32_t ba = smem_u32(&bars[j % NA]);
        mbar_expect_tx(ba, txA);
        tma_load3(smem_u32(ringA + (j % NA) * afl), &mapA, ba, zlo - ZH, ylo - R, x0);
        const uint32_t bb = smem_u32(&bars[NA + j % NB]);
        float* bs = ringB + (j % NB) * 2 * bfl;
        mbar_expect_tx(bb, txB);
        tma_load3(smem_u32(bs), &mapV, bb, zlo, ylo, x0 - R);
        tma_load3(smem_u32(bs + bfl), &mapK, bb, zlo, ylo, x0 - R);
    };
    int issued = 0;
    if (tid == 0) {
        for (int j = 0; j < kPrefetch && j < NIT; ++j) issue(j);
        issued = kPrefetch < NIT ? kPrefetch : NIT;
    }

    float4 q[T][P];
#pragma unroll
    for (int k = 0; k < T; ++k)
#pragma unroll
        for (int j = 0; j < P; ++j) q[k][j] = make_float4(0.f, 0.f, 0.f, 0.f);

    // ring positions of iteration i, advanced incrementally
    int sA = 0, sAc = NA - R, sB = 0, ph = 0, vslot = 0;  // i % NA, (i - R) % NA, i % NB, parities, i % NV
    int phA = 0, phB = 0;                                 // (i / NA) & 1, (i / NB) & 1
    // x of step 0 at iteration 0 is xbase - R; kappa rows of steps >= 1 and the output row follow it
    const long long sx = a.sx;
    bool abort = false;

    // One iteration with NACT active steps (compile time) and, if OUTP, the
    // write of the pass outputs.  Steps k >= NACT are not active yet: their
    // queues are filled (k == NACT) or untouched (k > NACT).
    // rot_c: -1 = the queues move down one slot per iteration (register moves);
    // S >= 0 = the loop is unrolled over the queue length and logical slot j
    // lives at register (S + j) % P, so the rotation costs nothing.
    auto body = [&](int i, auto nact_c, auto out_c, auto rot_c) {
        constexpr int NACT = decltype(nact_c)::value;
        constexpr bool OUTP = decltype(out_c)::value;
        constexpr int SR = decltype(rot_c)::value;
        constexpr int S = SR < 0 ? 0 : SR;
        constexpr bool MOVE = SR < 0;
        // kappa of steps k >= 1 at their planes, fetched early (cache hits)
        float4 kpre[T];
#pragma unroll
        for (int k = 1; k < T; ++k) {
            kpre[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < NACT) {
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
        // publish the centre planes x_k of active steps k >= 1
        if (act) {
#pragma unroll
            for (int k = 1; k < T; ++k)
                if (k < NACT) sts4(planes + ((k - 1) * 2 + (i & 1)) * afl + posA, q[k][MOVE ? R + 1 : (S + R) % P]);
        }
        __syncthreads();
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
        if (act) {
            const float* pnew = ringA + sA * afl;
            const float* pctr = ringA + sAc * afl;
            const float* pb = ringB + sB * 2 * bfl;
            const int vread = vslot == NV - 1 ? 0 : vslot + 1;  // slot of iteration i - R
            float4 prev_u = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 prev_v = prev_u;
#pragma unroll
            for (int k = 0; k < T; ++k) {
                if (k <= NACT) {
                    // the x queue of step k moves down one plane and takes its newest
                    if (MOVE) {
#pragma unroll
                        for (int j = 0; j + 1 < P; ++j) q[k][j] = q[k][j + 1];
                    }
                    q[k][(S + 2 * R) % P] = (k == 0) ? lds4(pnew + posA) : prev_u;
                    if (k >= 1) vring[((k - 1) * NV + vslot) * NTHR + tid] = prev_v;
                }
                if (k < NACT) {
                    // step k+1 of the pass: u^{n0+k+1}, v^{n0+k+1/2} at plane xk
                    const int xk = xbase + i - (k + 1) * R;
                    const float* plane = (k == 0) ? pctr : planes + (((k - 1) * 2 + (i & 1)) * afl);
                    float4 L = laplacian4<R, S>(plane, posA, pitch, q[k], a);
                    float4 u = q[k][(S + R) % P];
                    if (xk == nxt[k]) {
                        // sources of this plane (before the update) ...
                        int c = scur[k];
                        while (c < send) {
                            const int4 e = a.src_ent[c];
                            if (e.x != xk) break;
                            const float w = __int_as_float(e.w);
                            const float qv = a.wavelet[static_cast<long long>(a.n0 + k) * a.nsrc + e.z];
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
                                a.slots[static_cast<long long>(a.n0 + k - a.slot_row0) * a.ntaps + (e.y >> 2)] =
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
            }
            if (OUTP && own) {
                // write u^{n+T} and v^{n+T-1/2} of plane x_T
                const long long off = (xbase + i - T * R) * sx + colofs;
                *reinterpret_cast<float4*>(a.out_u + off) = prev_u;
                *reinterpret_cast<float4*>(a.out_v + off) = prev_v;
            }
        }
        // advance the ring positions
        vslot = vslot == NV - 1 ? 0 : vslot + 1;
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
    if (ROT) {
        // steady state unrolled over the queue length; the queues enter it in
        // the moved layout, which is rotation 0
        for (int i0 = i; i0 < NIT && !abort; i0 += P)
            static_for<P>([&](auto sc) {
                constexpr int S = decltype(sc)::value;
                if (i0 + S < NIT && !abort)
                    body(i0 + S, std::integral_constant<int, T>{}, std::true_type{}, std::integral_constant<int, S>{});
            });
    } else {
        for (; i < NIT && !abort; ++i) body(i, std::integral_constant<int, T>{}, std::true_type{}, NoRot{});
    }
    (void)ph;
}

// Shared memory of the (R, T, QZ, RY) instantiation.
template <int R, int T, int QZ, int RY>
constexpr size_t smem_bytes()
{
    using C = Cfg<R, T>;
    using G = Geo<R, T, QZ, RY>;
    return ((8u * (C::NA + C::NB) + 4u + 127u) & ~127u) +
           4u * (static_cast<size_t>(C::NA) * G::AFL + 2u * C::NB * G::BFL + 2u * (T - 1) * G::AFL) +
           16u * static_cast<size_t>(T - 1) * C::NV * G::NTHR;
}

template <int R, int T, int QZ, int RY, bool ROT>
cudaError_t launch_impl(const CUtensorMap& mapA, const CUtensorMap& mapV, const CUtensorMap& mapK,
                        const PassArgs& a, int threads, size_t smem, long long blocks, cudaStream_t st)
{
    auto fn = pass_kernel<R, T, QZ, RY, ROT>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    fn<<<static_cast<unsigned>(blocks), threads, smem, st>>>(mapA, mapV, mapK, a);
    return cudaGetLastError();
}

}  // namespace detail
}  // namespace wave
