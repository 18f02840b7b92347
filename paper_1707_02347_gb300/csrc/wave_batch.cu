// wave_batch.cu -- the persistent kernel of batched shots (wave_batch_forward).
//
// Many independent shots, each with its own grid, space order and tiling, are
// advanced by one launch: a work queue in device memory lists every (shot,
// pass, tile) item, and each thread block (one per SM) takes the next item
// from an atomic counter, runs that output tile of that pass (pass_tile, the
// same code and arithmetic as the standalone pass kernel) and then publishes
// the tile on the shot's completion counter.  An item of a one-step team
// shape covers four consecutive tiles, run side by side by the block's four
// teams of 128 threads (the occupancy a one-step tile has on its own).  A pass of a shot may start
// only once every tile of the shot's previous pass is done: it reads their
// outputs, with halos, and may overwrite their inputs.  The per-problem
// tiling is the autotuner's pick for each shot (the paper's per-problem
// tiling configuration, Section "Future Work", "Automating time-tiling in
// Devito"); the items of all shots are interleaved pass level by pass level,
// so a block that waits for one shot's previous pass is rare and short.
//
// No deadlock: the queue lists every item of a shot's pass before any item
// of its next pass, so an item only waits for items that running blocks have
// already taken, and those wait only for items taken before them.  No hang:
// every wait gives up after a time limit, sets the queue's abort word (the
// other blocks stop at their next item) and error bit 1; the tile's own
// bounded TMA waits report through error bit 0.
//
// Memory ordering: a finished tile's stores are generic-proxy writes that
// the next pass reads with TMA (the async proxy) from other SMs.  Every
// writer fences its stores (proxy fence, then a GPU-scope fence) before the
// block barrier, one thread publishes with a release add, and the consumer
// acquires the counter and issues a proxy fence before its first TMA copy.
#include "wave_pass.cuh"

namespace wave {
namespace detail {

// Pass arguments of the batch's descriptors.  Constant memory, like the
// kernel parameters of a standalone pass, so the tile's coefficient and
// argument reads stay uniform constant-cache loads.  One array per device,
// written by the batch's graph before its persistent launch.
__constant__ PassArgs c_batch_args[kMaxBatchArgs];

// The compiled shapes of the persistent kernel, all with the x queues in
// tensor memory (variant 2): radius, T, z quads per row, rows.  Block shapes
// use all 512 threads of a block for one tile; team shapes (one-step, 128
// threads) run four tiles at once, one per team of four warps, each team
// with its own named barrier, shared memory and tensor-memory columns.
#define WAVE_BATCH_SHAPES(X) \
    X(0, 2, 1, 16, 32)       \
    X(1, 2, 2, 16, 32)       \
    X(2, 2, 2, 8, 64)        \
    X(3, 2, 3, 16, 32)       \
    X(4, 4, 1, 16, 32)       \
    X(5, 4, 2, 16, 32)       \
    X(6, 4, 2, 8, 64)
#define WAVE_BATCH_TEAM_SHAPES(X) \
    X(7, 2, 1, 16, 8)             \
    X(8, 4, 1, 16, 8)

constexpr int kTeams = 4, kTeamThreads = 128;

// shared memory and tensor-memory columns of one team (the largest team shape)
constexpr size_t team_smem()
{
    size_t m = 0;
#define WAVE_TEAM_SMEM(I, R, T, QZ, RY) m = smem_bytes<R, T, QZ, RY>() > m ? smem_bytes<R, T, QZ, RY>() : m;
    WAVE_BATCH_TEAM_SHAPES(WAVE_TEAM_SMEM)
#undef WAVE_TEAM_SMEM
    return (m + 127) & ~static_cast<size_t>(127);
}
constexpr uint32_t team_cols()
{
    uint32_t m = 0;
#define WAVE_TEAM_COLS(I, R, T, QZ, RY) \
    m = TmemGeo<R, T, QZ, RY>::COLS > static_cast<int>(m) ? static_cast<uint32_t>(TmemGeo<R, T, QZ, RY>::COLS) : m;
    WAVE_BATCH_TEAM_SHAPES(WAVE_TEAM_COLS)
#undef WAVE_TEAM_COLS
    return m;
}
constexpr size_t kTeamSmem = team_smem();
constexpr uint32_t kTeamCols = team_cols();
static_assert(kTeams * kTeamThreads == 512, "four teams fill a block");
static_assert(kTeams * kTeamCols <= 512, "team tensor memory");

constexpr size_t batch_smem_max()
{
    size_t m = kTeams * kTeamSmem;
#define WAVE_SMEM_MAX(I, R, T, QZ, RY) m = smem_bytes<R, T, QZ, RY>() > m ? smem_bytes<R, T, QZ, RY>() : m;
    WAVE_BATCH_SHAPES(WAVE_SMEM_MAX)
#undef WAVE_SMEM_MAX
    return m;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int* p, int v)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Wait until *done >= need, giving up after limit_ns or once *abort is set.
__device__ __forceinline__ bool wait_done(const int* done, int need, const int* abort, unsigned long long limit_ns)
{
    if (ld_acquire_gpu(done) >= need) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 16; ++k)
            if (ld_acquire_gpu(done) >= need) return true;
        if (ld_acquire_gpu(abort) != 0) return false;
        if (global_ns() - t0 > limit_ns) return false;
        __nanosleep(256);
    }
}

__global__ void __launch_bounds__(512, 1) batch_kernel(const __grid_constant__ BatchQueue q)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ int4 s_item;
    __shared__ int s_go, s_shot, s_shape, s_count;
    const int tid = threadIdx.x;
    // the block's tensor memory, for every tile it runs (512 columns cover every shape)
    if (tid < 32) {
        tmem_alloc(smem_u32(&s_tmem), 512);
        tmem_relinquish();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tbase = s_tmem;
    for (;;) {
        if (tid == 0) {
            s_go = 0;
            const int k = atomicAdd(q.next, 1);
            if (k < q.nitems && ld_acquire_gpu(q.abort) == 0 && (ld_acquire_gpu(q.err) & 1) == 0) {
                const int4 it = q.items[k];
                const int shot = q.desc[it.x].shot;
                if (wait_done(q.done + shot, it.z, q.abort, q.limit_ns)) {
                    // the previous pass's outputs are read by TMA (async proxy)
                    fence_proxy_async_global();
                    s_item = it;
                    s_shot = shot;
                    s_shape = q.desc[it.x].shape;
                    // tiles this item covers: one, or (team shapes) up to one per team
                    s_count = q.desc[it.x].team ? min(kTeams, q.desc[it.x].ntiles - it.y) : 1;
                    s_go = 1;
                } else {
                    atomicOr(q.err, 2);
                    atomicExch(q.abort, 1);
                }
            }
        }
        __syncthreads();
        if (!s_go) break;
        const int4 it = s_item;
        const CUtensorMap* m = q.maps + 3 * it.x;
        const PassArgs& a = c_batch_args[it.x];
        switch (s_shape) {
#define WAVE_CASE(I, R, T, QZ, RY)                                                          \
    case I:                                                                                 \
        pass_tile<R, T, QZ, RY, 2>(m, m + 1, m + 2, a, it.w, it.y, smem, tbase, true, Team{tid, 0, 512}); \
        break;
            WAVE_BATCH_SHAPES(WAVE_CASE)
#undef WAVE_CASE
#define WAVE_TEAM_CASE(I, R, T, QZ, RY)                                                                      \
    case I: {                                                                                                \
        const int g = tid / kTeamThreads;                                                                    \
        if (g < s_count)                                                                                     \
            pass_tile<R, T, QZ, RY, 2>(m, m + 1, m + 2, a, it.w, it.y + g, smem + g * kTeamSmem,              \
                                       tbase + g * kTeamCols, true, Team{tid % kTeamThreads, 1 + g, kTeamThreads}); \
        break;                                                                                               \
    }
            WAVE_BATCH_TEAM_SHAPES(WAVE_TEAM_CASE)
#undef WAVE_TEAM_CASE
            default: break;
        }
        // publish the tiles: their stores before the release of the shot's counter
        fence_proxy_async_global();
        __threadfence();
        __syncthreads();
        if (tid == 0) red_release_add(q.done + s_shot, s_count);
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (tid < 32) tmem_dealloc(tbase, 512);
}

}  // namespace detail

int batch_shape_index(int R, int T, int qz, int ry, int unroll)
{
    if (unroll != 2) return -1;
#define WAVE_FIND(I, R_, T_, QZ, RY) \
    if (R == R_ && T == T_ && qz == QZ && ry == RY) return I;
    WAVE_BATCH_SHAPES(WAVE_FIND)
    WAVE_BATCH_TEAM_SHAPES(WAVE_FIND)
#undef WAVE_FIND
    return -1;
}

bool batch_shape_is_team(int shape)
{
#define WAVE_IS_TEAM(I, R, T, QZ, RY) \
    if (shape == I) return true;
    WAVE_BATCH_TEAM_SHAPES(WAVE_IS_TEAM)
#undef WAVE_IS_TEAM
    return false;
}

size_t batch_smem_bytes() { return detail::batch_smem_max(); }

cudaError_t batch_copy_args(const PassArgs* dev_args, int n, cudaStream_t st)
{
    if (n < 0 || n > kMaxBatchArgs) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    return cudaMemcpyToSymbolAsync(detail::c_batch_args, dev_args, sizeof(PassArgs) * static_cast<size_t>(n), 0,
                                   cudaMemcpyDeviceToDevice, st);
}

cudaError_t launch_batch(const BatchQueue& q, int blocks, cudaStream_t st)
{
    const size_t smem = detail::batch_smem_max();
    cudaError_t e = cudaFuncSetAttribute(detail::batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    detail::batch_kernel<<<blocks, 512, smem, st>>>(q);
    return cudaGetLastError();
}

}  // namespace wave
