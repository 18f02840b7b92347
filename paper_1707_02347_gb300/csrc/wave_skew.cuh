// wave_skew.cuh -- the skewed wavefront variant of the two-step pass
// (instantiated per stencil radius in wave_pass_r*.cu, variant 4).
//
// Section "Skewing Dependencies" tiles the space loops with parallelograms
// skewed by r per time step, so that no point-step is computed twice, and
// runs the tiles in an order that respects their dependences (Fig.
// tiled_256).  This kernel applies that to the y tiles of a pass of T = 2
// steps (x stays the streamed, pipelined axis and z keeps its overlapped
// halo):
//
//   * tile j computes step 1 (u^{n+1}) on rows [j by, (j+1) by) and step 2
//     (u^{n+2}) on rows [j by - r, (j+1) by - r): the tile boundary moves by
//     -r per step, the skew;
//   * step 2 of tile j reads step-1 values on rows [j by - 2r, (j+1) by):
//     its own, plus the top 2r rows of tile j-1, which are the only values a
//     tile takes from another (u of those 2r rows and, for the r rows whose
//     step 2 it computes, their increments v);
//   * tile j-1 writes those rows, plane by plane, to an exchange buffer and
//     publishes how many of its iterations are complete; tile j waits for
//     the plane it needs (a wavefront along y).
//
// Thread blocks are persistent: each takes the next tile from an atomic
// counter, in wavefront order (y level j, then slab, then z tile), so a tile
// only ever waits for a tile that a running block has already taken, and
// every wait is bounded (on timeout the block flags an error and stops).
// The release store of a tile's progress comes after the block barrier that
// ends the iteration, so every thread's exchange writes are ordered before it
// (release is cumulative over what the barrier ordered before it).  The
// producer never waits for its consumer: the exchange buffer holds every
// plane of a tile's slab.  Results are bit-identical to the one-step pass:
// each point-step is computed once, by the same arithmetic.
#pragma once
#include "wave_pass.cuh"

namespace wave {
namespace detail {

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// 16-byte asynchronous copy global -> shared through L2 only (the exchange
// rows are written by another block); cp_async_wait_all waits for the
// thread's own copies.
__device__ __forceinline__ void cp_async16(void* dst, const float* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Sources of plane xk of step k (entries of this column at xk) added to L in
// the pass kernel's order; advances the cursor.
__device__ __forceinline__ void inject(const PassArgs& a, float4& L, int xk, int& scur, int send, int k)
{
    int c = scur;
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
    scur = c;
}

// Receivers of plane xk of step k (rows whose values this tile owns), then
// the next event of the step.
__device__ __forceinline__ void record(const PassArgs& a, const float4& u, int xk, int X1, bool own, int scur, int send,
                                       int& rcur, int rend, int& nxt, int k)
{
    int c = rcur;
    if (own) {
        while (c < rend) {
            const int2 e = a.rec_ent[c];
            if (e.x != xk) break;
            if (xk < X1)
                a.slots[static_cast<long long>(a.n0 + k - a.slot_row0) * a.ntaps + (e.y >> 2)] = lane_of(u, e.y & 3);
            ++c;
        }
    }
    rcur = c;
    int nx2 = INT_MAX;
    if (scur < send) nx2 = a.src_ent[scur].x;
    if (own && rcur < rend) nx2 = min(nx2, a.rec_ent[rcur].x);
    nxt = nx2;
}

// Shared memory of the skewed (R, QZ, RY) instantiation: the two-step pass's
// layout plus two slots per thread of the bottom r rows (tile j-1's u and v
// of the step-2 queue row), double-buffered.
template <int R, int QZ, int RY>
constexpr size_t skew_smem_bytes()
{
    return smem_bytes<R, 2, QZ, RY>() + 2u * 2u * 16u * R * QZ;
}

template <int R, int QZ, int RY>
__global__ void __launch_bounds__(QZ * RY, 1)
    skew_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV,
                const __grid_constant__ CUtensorMap mapK, const PassArgs a)
{
    constexpr int T = 2;
    using C = Cfg<R, T>;
    using G = Geo<R, T, QZ, RY>;
    using TG = TmemGeo<R, T, QZ, RY>;
    static_assert(TG::fits, "tensor-memory queues exceed 512 columns");
    constexpr int NA = C::NA, NB = C::NB, NV = C::NV, ZH = C::ZH, kPrefetch = C::D;
    constexpr int afl = G::AFL, bfl = G::BFL, pitch = G::A_COLS, NTHR = G::NTHR;
    constexpr int R2 = 2 * R;
    constexpr int BY = RY - R;          // rows of a tile per step
    constexpr int XR = 3 * R;           // exchange rows per plane: u of 2r rows, v of r rows
    constexpr int XC = 4 * QZ;          // exchange columns
    static_assert(BY >= 2 * R, "a tile must be at least 2r rows high");
    constexpr uint32_t hdr = (8u * (NA + NB) + 8u + 127u) & ~127u;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    volatile int* s_abort = reinterpret_cast<volatile int*>(smem + 8 * (NA + NB));
    volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(smem + 8 * (NA + NB) + 4);
    float* __restrict__ ringA = reinterpret_cast<float*>(smem + hdr);
    float* __restrict__ ringB = ringA + NA * afl;
    float* __restrict__ plane1 = ringB + NB * 2 * bfl;  // step-1 values published for step 2 (two buffers)
    float4* __restrict__ vring = reinterpret_cast<float4*>(plane1 + 2 * afl);
    float4* __restrict__ xslot = vring + NV * NTHR;  // [2][u, v][r rows x QZ]
    __shared__ int s_item;
    constexpr uint32_t txA = static_cast<uint32_t>(G::A_ROWS * G::A_COLS * 4);
    constexpr uint32_t txB = static_cast<uint32_t>(2 * G::B_ROWS * G::B_COLS * 4);

    const int tid = threadIdx.x;
    const int ty = tid / QZ, tq = tid % QZ;
    // warp roles: step 1 on region rows [r, RY), step 2 on rows [0, BY)
    const int wr_lo = (tid & ~31) / QZ, wr_hi = ((tid & ~31) + 31) / QZ;
    const bool wstep1 = wr_hi >= R;
    const bool wstep2 = wr_lo < BY;

    if (tid < 32) {
        __syncwarp();
        tmem_alloc(smem_u32(const_cast<uint32_t*>(s_tmem)), TG::COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < NA + NB; ++s) mbar_init(smem_u32(&bars[s]), 1);
        *s_abort = 0;
        fence_mbar_init();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const int warp = tid >> 5;
    const uint32_t twarp =
        *s_tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + static_cast<uint32_t>((warp >> 2) * TG::CPW);
    auto tcol = [&](int k, int s) { return twarp + static_cast<uint32_t>(k * TG::CPS + 4 * s); };

    int* const progress = a.sync;
    int* const work = a.sync + a.nitems;
    const long long sx = a.sx;
    const long long exch_item = static_cast<long long>(a.exch_nit) * XR * XC;
    // ring positions, continued from tile to tile (g = iterations done by this block)
    long long g = 0;
    int sA = 0, sAc = NA - R, sB = 0, vslot = 0, ts = 0, phA = 0, phB = 0;
    bool abort = false;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(work, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();  // everyone has read s_item before it is written again
        if (item >= a.nitems || *s_abort) break;
        // tiles in wavefront order: y level j slowest, then slab, then z tile,
        // so that a tile's producer was taken a whole level earlier
        const int nxs = (a.nx + a.xc - 1) / a.xc;
        const int tzi = item % a.ntz;
        const int xsi = (item / a.ntz) % nxs;
        const int tyi = item / (a.ntz * nxs);
        const int prod = tyi > 0 ? item - a.ntz * nxs : -1;  // tile j-1 of the same slab and z column
        const int y0 = tyi * BY, z0 = tzi * a.bz;
        const int ylo = y0 - R, zlo = z0 + a.zlead;  // region: rows [y0 - r, y0 + BY)
        const int X0 = xsi * a.xc, X1 = min(X0 + a.xc, a.nx);
        const int NIT = (X1 - X0) + 2 * R * T;
        const int xbase = X0 - R * T;
        const int gy = ylo + ty, gz = zlo + 4 * tq;
        const bool colv = gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nzp;
        const bool ztile = gz >= z0 && gz < z0 + a.bz;
        const bool step1 = ty >= R, step2 = ty < BY;  // rows whose step 1 / step 2 this tile computes
        const bool own1 = colv && ztile && step1, own2 = colv && ztile && step2;
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
        // sparse events of the two steps (rows that compute the step; receivers
        // on the rows whose values of that step this tile owns)
        int scur[T], rcur[T], nxt[T], send = 0, rend = 0;
#pragma unroll
        for (int k = 0; k < T; ++k) { scur[k] = 0; rcur[k] = 0; nxt[k] = INT_MAX; }
        if (colv && a.src_ptr != nullptr) {
            const int lo = a.src_ptr[col];
            send = a.src_ptr[col + 1];
#pragma unroll
            for (int k = 0; k < T; ++k) {
                scur[k] = lo < send ? first_at_or_after(a.src_ent, lo, send, X0 - R * (T - 1 - k)) : send;
                if (scur[k] < send && (k == 0 ? step1 : step2)) nxt[k] = a.src_ent[scur[k]].x;
            }
        }
        if (colv && ztile && a.rec_ptr != nullptr) {
            const int lo = a.rec_ptr[col];
            rend = a.rec_ptr[col + 1];
            const int c0 = lo < rend ? first_at_or_after(a.rec_ent, lo, rend, X0) : rend;
#pragma unroll
            for (int k = 0; k < T; ++k) {
                rcur[k] = c0;
                if (c0 < rend && (k == 0 ? step1 : step2)) nxt[k] = min(nxt[k], a.rec_ent[c0].x);
            }
        }
        float* const xout = a.exch + item * exch_item;                           // this tile's exchange planes
        const float* const xin = prod >= 0 ? a.exch + prod * exch_item : nullptr;  // tile j-1's

        auto issue = [&](long long gi, int j) {
            const int x0 = xbase + j;
            const int slA = static_cast<int>(gi % NA), slB = static_cast<int>(gi % NB);
            const uint32_t ba = smem_u32(&bars[slA]);
            mbar_expect_tx(ba, txA);
            tma_load3(smem_u32(ringA + slA * afl), &mapA, ba, zlo - ZH, ylo - R, x0);
            const uint32_t bb = smem_u32(&bars[NA + slB]);
            float* bs = ringB + slB * 2 * bfl;
            mbar_expect_tx(bb, txB);
            tma_load3(smem_u32(bs), &mapV, bb, zlo, ylo, x0 - R);
            tma_load3(smem_u32(bs + bfl), &mapK, bb, zlo, ylo, x0 - R);
        };
        int issued = 0, seen = 0;
        // the bottom tile of a column has nothing below: zero halo rows in both plane buffers
        if (xin == nullptr && ty < R) {
            sts4(plane1 + posA - R * pitch, make_float4(0.f, 0.f, 0.f, 0.f));
            sts4(plane1 + afl + posA - R * pitch, make_float4(0.f, 0.f, 0.f, 0.f));
        }
        if (tid == 0) {
            for (int j = 0; j < kPrefetch && j < NIT; ++j) issue(g + j, j);
            issued = kPrefetch < NIT ? kPrefetch : NIT;
        }

        for (int i = 0; i < NIT && !abort; ++i) {
            const int nact = i < 2 * R ? 0 : (i < 4 * R ? 1 : 2);  // steps active in this iteration
            const bool outp = i >= 4 * R;
            const int x1 = xbase + i - R, x2 = xbase + i - 2 * R;  // planes of step 1 and step 2
            float4 kp2 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (nact > 1 && step2 && colv && x2 >= 0 && x2 < a.nx)
                kp2 = __ldg(reinterpret_cast<const float4*>(a.kap + x2 * sx + colofs));
            bool ok = mbar_wait(smem_u32(&bars[sA]), phA);
            ok = mbar_wait(smem_u32(&bars[NA + sB]), phB) && ok;
            // tile j-1 must have finished iteration i+1, whose rows this block
            // starts copying during this iteration (seen: the last progress
            // value read; an acquire that returned at least `need` already
            // orders everything up to that iteration)
            const bool pre = xin != nullptr && i + 1 < NIT && i + 1 >= 2 * R;  // rows of iteration i+1 needed
            if (tid == 0 && pre && ok && seen < i + 2) {
                const int need = i + 2;
                seen = ld_acquire(progress + prod);
                if (seen < need) {
                    const unsigned long long t0 = global_ns();
                    while ((seen = ld_acquire(progress + prod)) < need) {
                        if (global_ns() - t0 > kWaitLimitNs) {
                            ok = false;
                            atomicOr(a.err, 2);
                            break;
                        }
                    }
                }
            }
            if (!ok) {
                *s_abort = 1;
                atomicOr(a.err, 1);
            }
            // step-2 plane x2: own step-1 values (queue centres); the rows below,
            // tile j-1's, were copied into it during the previous iteration
            if (ty < R) cp_async_wait_all();
            __syncwarp();
            tmem_wait_st();
            float4 ctr = make_float4(0.f, 0.f, 0.f, 0.f);
            float* pl = plane1 + (i & 1) * afl;
            if (nact >= 2) {
                uint32_t r4[4];
                tmem_ld_x4(tcol(1, ts + R < R2 ? ts + R : ts - R), r4);
                tmem_wait_ld(r4);
                ctr = make_float4(__uint_as_float(r4[0]), __uint_as_float(r4[1]), __uint_as_float(r4[2]),
                                  __uint_as_float(r4[3]));
                sts4(pl + posA, ctr);
            }
            __syncthreads();
            // every thread is past iteration i-1: publish it (with its exchange writes)
            if (tid == 0 && i > 0) st_release(progress + item, i);
            if (*s_abort) {
                if (tid == 0)
                    for (long long j = g; j < g - i + issued; ++j) {
                        mbar_wait(smem_u32(&bars[j % NA]), static_cast<uint32_t>((j / NA) & 1));
                        mbar_wait(smem_u32(&bars[NA + j % NB]), static_cast<uint32_t>((j / NB) & 1));
                    }
                abort = true;
                break;
            }
            if (tid == 0 && i + kPrefetch < NIT) {
                issue(g + kPrefetch, i + kPrefetch);
                issued = i + kPrefetch + 1;
            }
            // copy tile j-1's rows for iteration i+1: the step-2 queue row (plane
            // x1 + 1) and its increment and the halo row (plane x2 + 1)
            if (pre && ty < R) {
                float4* slot = xslot + ((i + 1) & 1) * 2 * R * QZ + ty * QZ + tq;
                cp_async16(slot, xin + (static_cast<long long>(i + 1) * XR + R + ty) * XC + 4 * tq);
                if (i + 1 >= 4 * R) {
                    const long long row = static_cast<long long>(i + 1 - R) * XR;
                    cp_async16(slot + R * QZ, xin + (row + 2 * R + ty) * XC + 4 * tq);
                    cp_async16(plane1 + ((i + 1) & 1) * afl + posA - R * pitch, xin + (row + ty) * XC + 4 * tq);
                }
            }
            const float* pnew = ringA + sA * afl;
            const float* pctr = ringA + sAc * afl;
            const float* pb = ringB + sB * 2 * bfl;
            const int vread = vslot == NV - 1 ? 0 : vslot + 1;
            float4 u1 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = u1;

            // ---- step 1 (u^{n+1}) at plane x1, rows [r, RY)
            {
                const float4 newest = lds4(pnew + posA);
                if (nact >= 1 && wstep1) {
                    uint32_t r[4 * R2];
                    if constexpr (R == 2) tmem_ld_x16(tcol(0, ts), r);
                    if constexpr (R == 4) tmem_ld_x32(tcol(0, ts), r);
                    float4 u = lds4(pctr + posA);
                    float2 yl, yh, zl, zh, xl, xh;
                    laplacian_yz<R>(pctr, posA, pitch, u, a, yl, yh, zl, zh);
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
                    float4 L = combine(yl, yh, zl, zh, xl, xh);
                    if (x1 == nxt[0]) inject(a, L, x1, scur[0], send, 0);
                    float4 v = lds4(pb + posB);
                    const float4 kp = lds4(pb + bfl + posB);
                    const float dx = (x1 < a.dxlo || x1 >= a.dxhi) ? a.damp_x[min(max(x1, 0), a.nx - 1)] : 0.f;
                    update4(L, u, v, kp, dx, dyz, dyz_zero, a.inv2dt);
                    if (x1 == nxt[0]) record(a, u, x1, X1, own1, scur[0], send, rcur[0], rend, nxt[0], 0);
                    u1 = u;
                    v1 = v;
                }
                __syncwarp();
                tmem_st4(tcol(0, ts), newest);
                tmem_st4(tcol(0, ts + R2), newest);
            }
            // tile j's top rows to the exchange (for tile j+1): u of rows [BY - r, RY), v of rows [BY, RY)
            if (nact >= 1 && ty >= BY - R) {
                float* xo = xout + static_cast<long long>(i) * XR * XC + 4 * tq;
                *reinterpret_cast<float4*>(xo + (ty - (BY - R)) * XC) = u1;
                if (ty >= BY) *reinterpret_cast<float4*>(xo + (2 * R + ty - BY) * XC) = v1;
            }

            // ---- step 2 (u^{n+2}) at plane x2, rows [0, BY)
            {
                // the newest plane of the step-2 queue: this tile's step-1 value,
                // or, on rows [0, r), tile j-1's (zero below the grid)
                const float4* slot = xslot + (i & 1) * 2 * R * QZ + (ty < R ? ty : 0) * QZ + tq;
                float4 newest = u1;
                if (ty < R) newest = (xin != nullptr && nact >= 1) ? slot[0] : make_float4(0.f, 0.f, 0.f, 0.f);
                if (nact >= 1 && ty >= R) vring[vslot * NTHR + tid] = v1;
                if (nact >= 2 && wstep2) {
                    uint32_t r[4 * R2];
                    if constexpr (R == 2) tmem_ld_x16(tcol(1, ts), r);
                    if constexpr (R == 4) tmem_ld_x32(tcol(1, ts), r);
                    float4 u = ctr;
                    float2 yl, yh, zl, zh, xl, xh;
                    laplacian_yz<R>(pl, posA, pitch, u, a, yl, yh, zl, zh);
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
                    float4 L = combine(yl, yh, zl, zh, xl, xh);
                    if (x2 == nxt[1]) inject(a, L, x2, scur[1], send, 1);
                    // the increment of step 1 at x2: own (delayed r planes), or tile j-1's
                    float4 v = vring[vread * NTHR + tid];
                    if (ty < R) v = xin != nullptr ? slot[R * QZ] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float dx = (x2 < a.dxlo || x2 >= a.dxhi) ? a.damp_x[min(max(x2, 0), a.nx - 1)] : 0.f;
                    update4(L, u, v, kp2, dx, dyz, dyz_zero, a.inv2dt);
                    if (x2 == nxt[1]) record(a, u, x2, X1, own2, scur[1], send, rcur[1], rend, nxt[1], 1);
                    if (outp && own2) {
                        const long long off = x2 * sx + colofs;
                        *reinterpret_cast<float4*>(a.out_u + off) = u;
                        *reinterpret_cast<float4*>(a.out_v + off) = v;
                    }
                }
                __syncwarp();
                tmem_st4(tcol(1, ts), newest);
                tmem_st4(tcol(1, ts + R2), newest);
            }
            vslot = vslot == NV - 1 ? 0 : vslot + 1;
            ts = ts == R2 - 1 ? 0 : ts + 1;
            if (++sA == NA) { sA = 0; phA ^= 1; }
            if (++sAc == NA) sAc = 0;
            if (++sB == NB) { sB = 0; phB ^= 1; }
            ++g;
        }
        // the tile's last iterations: published once the block is past them
        __syncthreads();
        if (tid == 0 && !abort) st_release(progress + item, NIT);
        if (abort) break;
    }
    tmem_wait_st();
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (tid < 32) tmem_dealloc(*s_tmem, TG::COLS);
}

template <int R, int QZ, int RY>
cudaError_t launch_skew(const CUtensorMap& mapA, const CUtensorMap& mapV, const CUtensorMap& mapK, const PassArgs& a,
                        int threads, size_t smem, long long blocks, cudaStream_t st)
{
    auto fn = skew_kernel<R, QZ, RY>;
    if (threads != QZ * RY) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    fn<<<static_cast<unsigned>(blocks), threads, smem, st>>>(mapA, mapV, mapK, a);
    return cudaGetLastError();
}

}  // namespace detail
}  // namespace wave
