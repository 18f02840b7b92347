// wave_lean.cuh -- warp-specialised pass kernel of libwave.so (variants 5 and 6,
// instantiated per stencil radius in wave_pass_r*.cu).
//
// It computes what pass_kernel (wave_pass.cuh) computes, with the same float32
// operations in the same order, on the same schedule: a pass of T steps
// streams a slab of x planes, step k works r planes behind step k-1 (the skew
// by r per time step of Section "Skewing Dependencies"), and the y-z tile
// carries an overlapped halo of r (T - k) points at step k.  Two things differ.
//
// Synchronisation.  One producer warp issues the TMA copies.  The compute
// warps wait for a plane on its "full" mbarrier and, once every read of a
// ring slot is done, release the slot on its "empty" mbarrier; the producer
// refills a slot when all compute warps have released it.  The planes that
// step k >= 1 reads from neighbouring threads are handed over on a "full"
// mbarrier per plane buffer.  No block-wide barrier separates two planes:
// the warps that skip the last steps (the halo rows) and the warps waiting
// for shared memory do not hold the others back, and a warp may start the
// first step of a plane while others finish the last step of the one before.
//
// Work per thread.  A compute thread owns NY consecutive rows of one z quad
// (variant 5: NY = 1, variants 6 and 7: NY = 2).  The y neighbours of its rows
// form one column of 2r + NY quads, loaded once for all NY rows, and the
// per-plane bookkeeping of the thread is shared by its NY quads.
//
// x queues (SH).  Variants 5 and 6 keep each queue as a mirrored ring in
// tensor memory: every plane is stored twice, so that the window of 2r
// planes is always 8r consecutive columns.  Variant 7 (SH) keeps it as a
// shift register of 2r planes: the window is loaded, used, and stored back
// one plane further on (the oldest plane dropped, the newest appended) with
// one tcgen05.st of the same registers.  That halves the tensor memory of a
// queue, which lets two rows per thread run with 12 compute warps; the
// delay line of the previous level (steps k >= 1) moves from shared memory
// into tensor memory too, and the copies run two iterations ahead instead of
// three, which frees the shared memory of a taller tile.
#pragma once
#include "wave_pass.cuh"

namespace wave {
namespace detail {

// Shared memory of a warp-specialised pass that copies D iterations ahead:
// the mbarrier header, the ring of NA = D + r + 1 halo boxes of u^n, the
// ring of NB = D + 1 (v, kappa) planes, the planes of steps k >= 1 and, unless
// SH, their delay lines (previous increment and kappa).
template <int R, int T, int QZ, int RY, int NY, bool SH>
constexpr size_t lean_smem_for(int D)
{
    using G = Geo<R, T, QZ, RY>;
    const size_t NA = D + R + 1, NB = D + 1, NC = QZ * RY / NY;
    const size_t nbar = 2 * (NA + NB) + 2 * (T - 1);
    const size_t hdr = (8 * nbar + 8 + 127) & ~static_cast<size_t>(127);
    return hdr + 4 * (NA * G::AFL + 2 * NB * G::BFL + 2 * (T - 1) * G::AFL) +
           (SH ? 0 : 2 * 16 * static_cast<size_t>(T - 1) * R * NY * NC);
}

template <int R, int T, int QZ, int RY, int NY, bool SH = false>
struct LeanGeo {
    static_assert(RY % NY == 0, "whole row groups");
    static constexpr int NC = QZ * RY / NY;  // compute threads
    static_assert(NC % 32 == 0, "whole compute warps");
    static constexpr int NW = NC / 32;       // compute warps
    static constexpr int NTHR = NC + 32;     // and one producer warp
    // iterations copied ahead: the radius's default (three, or two at radius
    // 8) where the shared memory holds it, else two; two for SH
    static constexpr int D = (SH || lean_smem_for<R, T, QZ, RY, NY, SH>(Cfg<R, T>::D) > 227u * 1024u)
                                 ? 2 : Cfg<R, T>::D;
    static constexpr int NA = D + R + 1, NB = D + 1;
    static constexpr int NPF = 2 * (T - 1);  // plane buffers of the steps k >= 1, two per step
    // mbarriers: full A [NA], full B [NB], empty A [NA], empty B [NB], planes full [NPF]
    static constexpr int NBAR = 2 * (NA + NB) + NPF;
    static constexpr uint32_t HDR = (8u * NBAR + 8u + 127u) & ~127u;
    // tensor memory per quad and step: a mirrored ring of 2r planes (16 r
    // columns) or (SH) a shift register of 2r planes (8 r columns); SH also
    // keeps the previous-level delay line of the steps k >= 1 (r slots of 4
    // columns per row) after the queues
    static constexpr int CPQ = SH ? 8 * R : 16 * R;
    static constexpr int VCOL = T * NY * CPQ;                  // first delay-line column of a warp
    static constexpr int CPW = VCOL + (SH ? (T - 1) * NY * R * 4 : 0);  // columns of one warp's lanes
    static constexpr int WPQ = (NW + 3) / 4;  // warps sharing a lane quarter
    static constexpr int NEED = WPQ * CPW;
    static constexpr int COLS = NEED <= 32 ? 32 : NEED <= 64 ? 64 : NEED <= 128 ? 128 : NEED <= 256 ? 256 : 512;
    static_assert(NEED <= 512, "tensor-memory queues exceed 512 columns");
};

template <int R, int T, int QZ, int RY, int NY>
constexpr int lean_min_blocks()
{
    // one-step kernels keep 512 column quads resident per SM; T > 1 kernels
    // run one block per SM with the whole register file
    return (T == 1 && QZ * RY < 512) ? 512 / (QZ * RY) : 1;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// try_wait with a suspend-time hint: a waiting warp sleeps until the phase
// completes (or the hint runs out) instead of spinning on issue slots that
// the working warps of the SM need.
constexpr uint32_t kSuspendHintNs = 20000;
__device__ __forceinline__ bool mbar_try_sleep(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "n"(kSuspendHintNs)
        : "memory");
    return ok != 0;
}

// mbar_wait that also gives up as soon as another warp has set the block's
// abort word.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort_word)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 8; ++k)
            if (mbar_try_sleep(bar, parity)) return true;
        if (*abort_word) return false;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
}

__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[4], uint32_t (&s)[4])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]));
}

// the 2r-plane window of an x queue (8 r columns) into w
template <int R>
__device__ __forceinline__ void tmem_ld_window(uint32_t taddr, uint32_t (&w)[8 * R])
{
    if constexpr (R == 2) tmem_ld_x16(taddr, w);
    if constexpr (R == 4) tmem_ld_x32(taddr, w);
    if constexpr (R == 8) tmem_ld_x64(taddr, w);
}

// the window of an x queue (8 r columns) stored from w, shifted by one plane:
// columns [0, 8r - 4) take w[4 ..], the last 4 take the newest plane
template <int R>
__device__ __forceinline__ void tmem_st_shift(uint32_t taddr, const uint32_t (&w)[8 * R], const float4& nw)
{
    if constexpr (R == 2) {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15, %16};" ::"r"(taddr),
            "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[9]), "r"(w[10]), "r"(w[11]), "r"(w[12]),
            "r"(w[13]), "r"(w[14]), "r"(w[15]), "r"(__float_as_uint(nw.x)), "r"(__float_as_uint(nw.y)),
            "r"(__float_as_uint(nw.z)), "r"(__float_as_uint(nw.w)));
    }
    if constexpr (R == 4) {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::
                "r"(taddr),
            "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[9]), "r"(w[10]), "r"(w[11]), "r"(w[12]),
            "r"(w[13]), "r"(w[14]), "r"(w[15]), "r"(w[16]), "r"(w[17]), "r"(w[18]), "r"(w[19]), "r"(w[20]),
            "r"(w[21]), "r"(w[22]), "r"(w[23]), "r"(w[24]), "r"(w[25]), "r"(w[26]), "r"(w[27]), "r"(w[28]),
            "r"(w[29]), "r"(w[30]), "r"(w[31]), "r"(__float_as_uint(nw.x)), "r"(__float_as_uint(nw.y)),
            "r"(__float_as_uint(nw.z)), "r"(__float_as_uint(nw.w)));
    }
    static_assert(R == 2 || R == 4, "shift-register queues are compiled for radius 2 and 4");
}

template <int R, int T, int QZ, int RY, int NY, bool SH = false>
__global__ void __launch_bounds__(LeanGeo<R, T, QZ, RY, NY, SH>::NTHR, lean_min_blocks<R, T, QZ, RY, NY>())
    lean_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV,
                const __grid_constant__ CUtensorMap mapK, const PassArgs a)
{
    using C = Cfg<R, T>;
    using G = Geo<R, T, QZ, RY>;
    using L = LeanGeo<R, T, QZ, RY, NY, SH>;
    constexpr int NA = L::NA, NB = L::NB, NW = L::NW, NC = L::NC, ZH = C::ZH, R2 = 2 * R;
    constexpr int afl = G::AFL, bfl = G::BFL, pitch = G::A_COLS;
    extern __shared__ __align__(128) unsigned char smem[];
    volatile int* s_abort = reinterpret_cast<volatile int*>(smem + 8 * L::NBAR);
    volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(smem + 8 * L::NBAR + 4);
    // disjoint regions: the TMA rings, the published planes, the increment ring
    float* __restrict__ ringA = reinterpret_cast<float*>(smem + L::HDR);
    float* __restrict__ ringB = ringA + NA * afl;
    float* __restrict__ planes = ringB + NB * 2 * bfl;
    // (not SH) the delay lines of steps k >= 1: the previous level's
    // increment and kappa of the plane, r iterations from step k-1 to step k
    float4* __restrict__ vring = reinterpret_cast<float4*>(planes + 2 * (T - 1) * afl);
    float4* __restrict__ kring = vring + (T - 1) * R * NY * L::NC;
    const uint32_t fullA = smem_u32(smem), fullB = fullA + 8 * NA, emptyA = fullB + 8 * NB,
                   emptyB = emptyA + 8 * NA, fullP = emptyB + 8 * NB;
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
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        // warp 0 allocates the block's tensor memory (all 32 threads)
        tmem_alloc(smem_u32(const_cast<uint32_t*>(s_tmem)), L::COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < NA; ++s) {
            mbar_init(fullA + 8 * s, 1);
            mbar_init(emptyA + 8 * s, NW);
        }
        for (int s = 0; s < NB; ++s) {
            mbar_init(fullB + 8 * s, 1);
            mbar_init(emptyB + 8 * s, NW);
        }
        for (int s = 0; s < L::NPF; ++s) mbar_init(fullP + 8 * s, NW);
        *s_abort = 0;
        fence_mbar_init();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();

    if (warp == NW) {
        // Producer: one thread issues the copies of every iteration j in
        // order, each into a slot the compute warps have released.  The
        // slot of iteration j of ring A is free once every compute warp has
        // finished iteration j - NA + r (its last read, as the centre plane);
        // the slot of ring B once iteration j - NB is done.  The fields are
        // the previous pass's outputs: copies start once it has completed.
        grid_dep_wait();
        if (lane == 0) {
            int sa = 0, sb = 0, issued = 0;
            for (int j = 0; j < NIT; ++j) {
                bool ok = true;
                if (j >= NA) ok = mbar_wait_or_abort(emptyA + 8 * sa, ((j / NA) - 1) & 1, s_abort);
                if (ok && j >= NB) ok = mbar_wait_or_abort(emptyB + 8 * sb, ((j / NB) - 1) & 1, s_abort);
                if (!ok) {
                    *s_abort = 1;
                    atomicOr(a.err, 1);
                    break;
                }
                const int x0 = xbase + j;
                mbar_expect_tx(fullA + 8 * sa, txA);
                tma_load3(smem_u32(ringA + sa * afl), &mapA, fullA + 8 * sa, zlo - ZH, ylo - R, x0);
                float* bs = ringB + sb * 2 * bfl;
                mbar_expect_tx(fullB + 8 * sb, txB);
                tma_load3(smem_u32(bs), &mapV, fullB + 8 * sb, zlo, ylo, x0 - R);
                tma_load3(smem_u32(bs + bfl), &mapK, fullB + 8 * sb, zlo, ylo, x0 - R);
                issued = j + 1;
                if (++sa == NA) sa = 0;
                if (++sb == NB) sb = 0;
            }
            // no copy may still be in flight when the block exits
            for (int j = max(0, issued - NA); j < issued; ++j) mbar_wait(fullA + 8 * (j % NA), (j / NA) & 1);
            for (int j = max(0, issued - NB); j < issued; ++j) mbar_wait(fullB + 8 * (j % NB), (j / NB) & 1);
        }
        __syncwarp();
    } else {
        // compute thread -> z quad tq, thread rows ty0 .. ty0 + NY - 1.
        // Columns and planes outside the grid need no special case: kappa is
        // zero there (TMA zero fill, zero z padding), so the update keeps
        // u = v = 0 on them -- the zero ghost layer.
        const int tq = tid % QZ, ty0 = (tid / QZ) * NY;
        const int gz = zlo + 4 * tq;
        const int posA0 = (ty0 + R) * pitch + ZH + 4 * tq;
        bool colv[NY], own[NY], dyz_zero[NY];
        long long colofs[NY];
        float4 dyz[NY];
        bool all_zero = true;
#pragma unroll
        for (int r = 0; r < NY; ++r) {
            const int gy = ylo + ty0 + r;
            colv[r] = gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nzp;
            own[r] = colv[r] && gy >= y0 && gy < y0 + a.by && gz >= z0 && gz < z0 + a.bz;
            colofs[r] = static_cast<long long>(colv[r] ? gy : 0) * a.nzp + (colv[r] ? gz : 0);
            dyz[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            dyz_zero[r] = true;
            if (colv[r]) {
                const float dyv = a.damp_y[gy];
                dyz[r] = make_float4(__fadd_rn(dyv, a.damp_z[gz]), __fadd_rn(dyv, a.damp_z[gz + 1]),
                                     __fadd_rn(dyv, a.damp_z[gz + 2]), __fadd_rn(dyv, a.damp_z[gz + 3]));
                dyz_zero[r] = dyz[r].x == 0.f && dyz[r].y == 0.f && dyz[r].z == 0.f && dyz[r].w == 0.f;
            }
            all_zero = all_zero && dyz_zero[r];
        }
        // no y-z sponge anywhere in the warp: where dx is zero too, the
        // increment is fma(kappa, L, v), the fast path of update4
        const bool wint = __all_sync(0xffffffffu, all_zero);

        // Steps this warp computes: step k is needed on thread rows
        // [k R, RY - k R); a warp whose rows all lie outside skips step k and
        // every later one, and keeps only the queue of step k that its
        // neighbours read.  Uniform over the warp.
        int wsteps = 0;
        {
            const int wr_lo = ((tid & ~31) / QZ) * NY, wr_hi = (((tid & ~31) + 31) / QZ) * NY + NY - 1;
#pragma unroll
            for (int k = 0; k < T; ++k)
                if (wr_hi >= k * R && wr_lo < RY - k * R) wsteps = k + 1;
        }

        // sparse events per row and step: next x with a source or receiver tap
        // in the row's column (cursors start inside the column's own CSR range)
        int scur[T][NY], rcur[T][NY], nxt[T][NY], send[NY], rend[NY];
#pragma unroll
        for (int r = 0; r < NY; ++r) {
            send[r] = 0;
            rend[r] = 0;
#pragma unroll
            for (int k = 0; k < T; ++k) {
                scur[k][r] = 0;
                rcur[k][r] = 0;
                nxt[k][r] = INT_MAX;
            }
            const int gy = ylo + ty0 + r;
            const int col = colv[r] ? gy * (a.nzp >> 2) + (gz >> 2) : 0;
            if (colv[r] && a.src_ptr != nullptr) {
                const int lo = a.src_ptr[col];
                send[r] = a.src_ptr[col + 1];
#pragma unroll
                for (int k = 0; k < T; ++k) {
                    scur[k][r] = lo < send[r] ? first_at_or_after(a.src_ent, lo, send[r], X0 - R * (T - 1 - k)) : send[r];
                    if (scur[k][r] < send[r]) nxt[k][r] = a.src_ent[scur[k][r]].x;
                }
            }
            if (own[r] && a.rec_ptr != nullptr) {
                const int lo = a.rec_ptr[col];
                rend[r] = a.rec_ptr[col + 1];
                const int c0 = lo < rend[r] ? first_at_or_after(a.rec_ent, lo, rend[r], X0) : rend[r];
#pragma unroll
                for (int k = 0; k < T; ++k) {
                    rcur[k][r] = c0;
                    if (c0 < rend[r]) nxt[k][r] = min(nxt[k][r], a.rec_ent[c0].x);
                }
            }
        }

        // this warp's tensor-memory columns: lane quarter (warp % 4), column block (warp / 4)
        const uint32_t twarp =
            *s_tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + static_cast<uint32_t>((warp >> 2) * L::CPW);
        // column of slot s (0 .. 4r - 1, or 0 .. 2r - 1 for SH) of the queue of step k, row r
        auto tcol = [&](int k, int r, int s) { return twarp + static_cast<uint32_t>((k * NY + r) * L::CPQ + 4 * s); };
        // (SH) column of slot s (0 .. r - 1) of the previous-level delay line of step k >= 1, row r
        auto vcol = [&](int k, int r, int s) {
            return twarp + static_cast<uint32_t>(L::VCOL + (((k - 1) * NY + r) * R + s) * 4);
        };

        // ring positions of iteration i, advanced incrementally
        int sA = 0, sAc = NA - R, sB = 0;  // i % NA, (i - R) % NA, i % NB
        int phA = 0, phB = 0;              // (i / NA) & 1, (i / NB) & 1
        int ts = 0, vs = 0;                // i % 2r (tensor-memory slot), i % r (increment delay slot)
        const long long sx = a.sx;
        bool abort = false;

        // One iteration with NACT active steps (compile time) and, if OUTP,
        // the write of the pass outputs.  Steps k >= NACT are not active yet:
        // their queues are filled (k == NACT) or untouched (k > NACT).
        auto body = [&](int i, auto nact_c, auto out_c) {
            constexpr int NACT = decltype(nact_c)::value;
            constexpr bool OUTP = decltype(out_c)::value;
            // (SH) kappa of steps k >= 1 at their planes, fetched early (cache
            // hits); otherwise it comes down the delay line from step k-1
            float4 kpre[T][NY];
#pragma unroll
            for (int k = 1; k < T; ++k) {
                const int xk = xbase + i - (k + 1) * R;
#pragma unroll
                for (int r = 0; r < NY; ++r) {
                    kpre[k][r] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (SH && k < NACT && k < wsteps && colv[r] && xk >= 0 && xk < a.nx)
                        kpre[k][r] = __ldg(reinterpret_cast<const float4*>(a.kap + xk * sx + colofs[r]));
                }
            }
            __syncwarp();
            tmem_wait_st();  // the previous iteration's ring writes
            // publish the centre planes x_k of steps k >= 1 (the plane their
            // queue took r iterations ago) and hand them over
            float4 ctr[T][NY];
#pragma unroll
            for (int k = 1; k < T; ++k) {
                float* pl = planes + ((k - 1) * 2 + (i & 1)) * afl + posA0;
                if (k < NACT && k <= wsteps) {
                    // (uniform over the warp, as every tcgen05 access)
                    const int sc = SH ? R : (ts + R < R2 ? ts + R : ts - R);
                    uint32_t c4[NY][4];
#pragma unroll
                    for (int r = 0; r < NY; ++r) tmem_ld_x4(tcol(k, r, sc), c4[r]);
                    if constexpr (NY == 1) tmem_wait_ld(c4[0]);
                    else tmem_wait_ld(c4[0], c4[NY - 1]);
#pragma unroll
                    for (int r = 0; r < NY; ++r) {
                        ctr[k][r] = make_float4(__uint_as_float(c4[r][0]), __uint_as_float(c4[r][1]),
                                                __uint_as_float(c4[r][2]), __uint_as_float(c4[r][3]));
                        sts4(pl + r * pitch, ctr[k][r]);
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < NY; ++r) ctr[k][r] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            if constexpr (T > 1) {
                __syncwarp();
                if (lane == 0)
#pragma unroll
                    for (int k = 1; k < T; ++k) mbar_arrive(fullP + 8 * ((k - 1) * 2 + (i & 1)));
            }
            // this iteration's planes of u^n and of (v^{n-1/2}, kappa)
            bool ok = mbar_wait_or_abort(fullA + 8 * sA, phA, s_abort);
            ok = mbar_wait_or_abort(fullB + 8 * sB, phB, s_abort) && ok;
            if (!__all_sync(0xffffffffu, ok)) {
                *s_abort = 1;
                atomicOr(a.err, 1);
                abort = true;
                return;
            }
            const float* pnew = ringA + sA * afl;
            const float* pctr = ringA + sAc * afl;
            const float* pb = ringB + sB * 2 * bfl;
            float4 pu[NY], pv[NY], pk[NY];  // u, v and kappa of the latest step computed in this iteration

            // Step k of the pass at plane x_k = x_0 - k r for the NY rows:
            // plane holds its input level with the y-z halo; newest[r] is the
            // plane after x_k + r - 1 of row r's queue.
            auto run_step = [&](auto kc, const float* plane, const float4 (&newest)[NY]) {
                constexpr int k = decltype(kc)::value;
                const int xk = xbase + i - (k + 1) * R;
                // row j of the thread's y column (j = -r .. NY - 1 + r); the
                // thread's own rows of a step k >= 1 are its published centres
                auto ycol = [&](auto jc) -> float4 {
                    constexpr int j = decltype(jc)::value;
                    if constexpr (k >= 1 && j >= 0 && j < NY) return ctr[k][j];
                    else return lds4(plane + posA0 + j * pitch);
                };
                float4 cen[NY];
                static_for<NY>([&](auto rc) { cen[decltype(rc)::value] = ycol(rc); });
                // the first window load overlaps the y sums
                __syncwarp();
                uint32_t w[4 * R2];
                tmem_ld_window<R>(tcol(k, 0, SH ? 0 : ts), w);
                // Ly of every row, the pairs k' = 1 .. r taken in order for each
                // row (the same operations as laplacian_y), rows interleaved so
                // that only a sliding part of the y column is live
                float2 yl[NY], yh[NY];
#pragma unroll
                for (int r = 0; r < NY; ++r) {
                    yl[r] = __fmul2_rn(a.c0, lo2(cen[r]));
                    yh[r] = __fmul2_rn(a.c0, hi2(cen[r]));
                }
                static_for<R>([&](auto kc2) {
                    constexpr int kk = decltype(kc2)::value + 1;
                    static_for<NY>([&](auto rc) {
                        constexpr int r = decltype(rc)::value;
                        pair2(yl[r], yh[r], a.cy[kk - 1], ycol(std::integral_constant<int, r - kk>{}),
                              ycol(std::integral_constant<int, r + kk>{}), cen[r], kk == 1, false);
                    });
                });
                const float dx = (xk < a.dxlo || xk >= a.dxhi) ? a.damp_x[min(max(xk, 0), a.nx - 1)] : 0.f;
                const bool fast = wint && dx == 0.f;
                static_for<NY>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    // window: the 2r planes before the newest, oldest first
                    // (the warp may have diverged on the previous row's events)
                    if constexpr (r > 0) {
                        __syncwarp();
                        tmem_ld_window<R>(tcol(k, r, SH ? 0 : ts), w);
                    }
                    // (SH, steps k >= 1) the previous level of this row, from the delay line
                    uint32_t pv4[4] = {0u, 0u, 0u, 0u};
                    if constexpr (SH && k >= 1) tmem_ld_x4(vcol(k, r, vs), pv4);
                    const float4 c = cen[r];
                    float2 zl, zh, xl, xh;
                    laplacian_z<R>(plane, posA0 + r * pitch, c, a, zl, zh);
                    tmem_wait_ld(w);
                    if constexpr (SH && k >= 1) tmem_wait_ld(pv4);
                    auto xq = [&](auto jc) -> float4 {
                        constexpr int j = decltype(jc)::value;
                        if constexpr (j == R2) {
                            return newest[r];
                        } else {
                            return make_float4(__uint_as_float(w[4 * j]), __uint_as_float(w[4 * j + 1]),
                                               __uint_as_float(w[4 * j + 2]), __uint_as_float(w[4 * j + 3]));
                        }
                    };
                    laplacian_x<R>(c, xq, a, xl, xh);
                    // (SH) the queue advances: the window shifted by one plane, the newest appended
                    if constexpr (SH) tmem_st_shift<R>(tcol(k, r, 0), w, newest[r]);
                    float4 Lq = combine(yl[r], yh[r], zl, zh, xl, xh);
                    if (xk == nxt[k][r]) {
                        // sources of this plane (before the update) ...
                        int e0 = scur[k][r];
                        while (e0 < send[r]) {
                            const int4 e = a.src_ent[e0];
                            if (e.x != xk) break;
                            const float wgt = __int_as_float(e.w);
                            const float qv = a.wavelet[static_cast<long long>(a.n0 + k) * a.nsrc + e.z];
                            if (e.y == 0) Lq.x = __fmaf_rn(wgt, qv, Lq.x);
                            else if (e.y == 1) Lq.y = __fmaf_rn(wgt, qv, Lq.y);
                            else if (e.y == 2) Lq.z = __fmaf_rn(wgt, qv, Lq.z);
                            else Lq.w = __fmaf_rn(wgt, qv, Lq.w);
                            ++e0;
                        }
                        scur[k][r] = e0;
                    }
                    float4 u = c;
                    float4 v;
                    if constexpr (k == 0) {
                        v = lds4(pb + (ty0 + r) * G::B_COLS + 4 * tq);
                    } else if constexpr (SH) {
                        v = make_float4(__uint_as_float(pv4[0]), __uint_as_float(pv4[1]), __uint_as_float(pv4[2]),
                                        __uint_as_float(pv4[3]));
                    } else {
                        v = vring[(((k - 1) * R + vs) * NY + r) * NC + tid];
                    }
                    float4 kp;
                    if constexpr (k == 0) kp = lds4(pb + bfl + (ty0 + r) * G::B_COLS + 4 * tq);
                    else if constexpr (SH) kp = kpre[k][r];
                    else kp = kring[(((k - 1) * R + vs) * NY + r) * NC + tid];
                    if (fast) {
                        const float2 vl = __ffma2_rn(lo2(kp), lo2(Lq), lo2(v));
                        const float2 vh = __ffma2_rn(hi2(kp), hi2(Lq), hi2(v));
                        v = make_float4(vl.x, vl.y, vh.x, vh.y);
                        const float2 ul = __fadd2_rn(lo2(u), vl);
                        const float2 uh = __fadd2_rn(hi2(u), vh);
                        u = make_float4(ul.x, ul.y, uh.x, uh.y);
                    } else {
                        update4(Lq, u, v, kp, dx, dyz[r], dyz_zero[r], a.inv2dt);
                    }
                    if (xk == nxt[k][r]) {
                        // ... and receivers (after it); then the next event of this step
                        int e0 = rcur[k][r];
                        while (e0 < rend[r]) {
                            const int2 e = a.rec_ent[e0];
                            if (e.x != xk) break;
                            if (xk < X1)
                                a.slots[static_cast<long long>(a.n0 + k - a.slot_row0) * a.ntaps + (e.y >> 2)] =
                                    lane_of(u, e.y & 3);
                            ++e0;
                        }
                        rcur[k][r] = e0;
                        int nx2 = INT_MAX;
                        if (scur[k][r] < send[r]) nx2 = a.src_ent[scur[k][r]].x;
                        if (rcur[k][r] < rend[r]) nx2 = min(nx2, a.rec_ent[rcur[k][r]].x);
                        nxt[k][r] = nx2;
                    }
                    pu[r] = u;
                    pv[r] = v;
                    pk[r] = kp;
                });
            };

            // step 1 of the pass (k = 0): newest plane from the TMA ring
            {
                float4 nw[NY];
#pragma unroll
                for (int r = 0; r < NY; ++r) nw[r] = lds4(pnew + posA0 + r * pitch);
                if constexpr (NACT >= 1) run_step(std::integral_constant<int, 0>{}, pctr, nw);
                // the newest plane into the ring (slot i % 2r and its mirror),
                // after this iteration's window was read; (SH) run_step
                // advanced the shift register, else it is advanced here
                __syncwarp();
                if constexpr (SH) {
                    if constexpr (NACT < 1) {
#pragma unroll
                        for (int r = 0; r < NY; ++r) {
                            uint32_t w[4 * R2];
                            tmem_ld_window<R>(tcol(0, r, 0), w);
                            tmem_wait_ld(w);
                            tmem_st_shift<R>(tcol(0, r, 0), w, nw[r]);
                        }
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < NY; ++r) {
                        tmem_st4(tcol(0, r, ts), nw[r]);
                        tmem_st4(tcol(0, r, ts + R2), nw[r]);
                    }
                }
            }
            // step 1 is done with ring B's slot and with ring A's centre plane
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(emptyB + 8 * sB);
                if (i >= R) mbar_arrive(emptyA + 8 * sAc);
            }
            // steps k >= 1: newest plane = what step k-1 produced in this iteration
            static_for<T - 1>([&](auto kc1) {
                constexpr int k = decltype(kc1)::value + 1;
                if (abort) return;
                const bool okp =
                    mbar_wait_or_abort(fullP + 8 * ((k - 1) * 2 + (i & 1)), (i >> 1) & 1, s_abort);
                if (!__all_sync(0xffffffffu, okp)) {
                    *s_abort = 1;
                    atomicOr(a.err, 1);
                    abort = true;
                    return;
                }
                if (k <= NACT && k <= wsteps) {
                    float4 nw[NY], vin[NY], kin[NY];
#pragma unroll
                    for (int r = 0; r < NY; ++r) {
                        nw[r] = pu[r];
                        vin[r] = pv[r];
                        kin[r] = pk[r];
                    }
                    const bool comp = k < NACT && k < wsteps;
                    if (comp) run_step(std::integral_constant<int, k>{}, planes + ((k - 1) * 2 + (i & 1)) * afl, nw);
                    // the increment of step k-1 waits r iterations for step k
                    // (its slot was read above, by the step r iterations later)
                    __syncwarp();
                    if constexpr (SH) {
#pragma unroll
                        for (int r = 0; r < NY; ++r) tmem_st4(vcol(k, r, vs), vin[r]);
                        if (!comp) {
                            // the queue of a step this warp does not compute still advances
#pragma unroll
                            for (int r = 0; r < NY; ++r) {
                                uint32_t w[4 * R2];
                                tmem_ld_window<R>(tcol(k, r, 0), w);
                                tmem_wait_ld(w);
                                tmem_st_shift<R>(tcol(k, r, 0), w, nw[r]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < NY; ++r) {
                            vring[(((k - 1) * R + vs) * NY + r) * NC + tid] = vin[r];
                            kring[(((k - 1) * R + vs) * NY + r) * NC + tid] = kin[r];
                        }
                        __syncwarp();
#pragma unroll
                        for (int r = 0; r < NY; ++r) {
                            tmem_st4(tcol(k, r, ts), nw[r]);
                            tmem_st4(tcol(k, r, ts + R2), nw[r]);
                        }
                    }
                }
            });
            if (abort) return;
            if (OUTP) {
                // write u^{n+T} and v^{n+T-1/2} of plane x_T
                const long long xo = static_cast<long long>(xbase + i - T * R) * sx;
#pragma unroll
                for (int r = 0; r < NY; ++r)
                    if (own[r]) {
                        *reinterpret_cast<float4*>(a.out_u + xo + colofs[r]) = pu[r];
                        *reinterpret_cast<float4*>(a.out_v + xo + colofs[r]) = pv[r];
                        if constexpr (T == 1)
                            if (a.gacc != nullptr) image4(a, xo + colofs[r], pu[r]);
                    }
            }
            // advance the ring positions
            vs = vs == R - 1 ? 0 : vs + 1;
            ts = ts == R2 - 1 ? 0 : ts + 1;
            if (++sA == NA) { sA = 0; phA ^= 1; }
            if (++sAc == NA) sAc = 0;
            if (++sB == NB) { sB = 0; phB ^= 1; }
        };

        // the outputs overwrite what the previous pass read: wait for it
        grid_dep_wait();
        int i = 0;
        static_for<T>([&](auto kc) {
            constexpr int k = decltype(kc)::value;  // steps 0 .. k-1 active in this phase
            const int end = 2 * (k + 1) * R;
            for (; i < end && !abort; ++i) body(i, std::integral_constant<int, k>{}, std::false_type{});
        });
        for (; i < NIT && !abort; ++i) body(i, std::integral_constant<int, T>{}, std::true_type{});
        __syncwarp();
        tmem_wait_st();
    }
    grid_dep_launch();
    // every warp is done with the tensor memory (and the producer with its
    // copies) before warp 0 frees it
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc(*s_tmem, L::COLS);
}

// Shared memory of the (R, T, QZ, RY, NY, SH) instantiation.
template <int R, int T, int QZ, int RY, int NY, bool SH = false>
constexpr size_t lean_smem_bytes()
{
    return lean_smem_for<R, T, QZ, RY, NY, SH>(LeanGeo<R, T, QZ, RY, NY, SH>::D);
}

template <int R, int T, int QZ, int RY, int NY, bool SH = false>
cudaError_t launch_lean(const CUtensorMap& mapA, const CUtensorMap& mapV, const CUtensorMap& mapK, const PassArgs& a,
                        int /*threads: fixed by the instantiation*/, size_t smem, long long blocks, cudaStream_t st)
{
    auto fn = lean_kernel<R, T, QZ, RY, NY, SH>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return launch_dependent(fn, blocks, LeanGeo<R, T, QZ, RY, NY, SH>::NTHR, smem, st, mapA, mapV, mapK, a);
}

}  // namespace detail
}  // namespace wave
