// wave_noalloc.cu -- receiver sampling that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they need a
// trace: code running inside a memory pool that must not grow, a host
// application whose allocator owns the whole device, or a real-time loop that
// forbids cudaMalloc because it may synchronise the device.  This file gives
// them one entry point, wave_sample_noalloc, with the same receiver sampling
// as the plan's forward pass (trilinear taps gathered into slots, then summed
// in fixed corner order) but with its slots in a fixed static device array
// instead of plan-owned memory.  Nothing here calls cudaMalloc, cudaFree or an
// allocating library routine.
//
// The static array is shared by every call in the process: calls that run on
// the GPU at the same time (different streams, or several host threads) race
// on it.  Each call writes every slot it later reads, so nothing has to start
// at zero and stale contents from an earlier call are never used.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "wave_host.h"

namespace {

// Capacity: receivers per call.  Per receiver: its position (3 doubles),
// 8 tap values, 8 tap weights (floats) and a tap count (int) = 92 bytes, so
// 65536 receivers take 5.75 MiB of device memory on every GPU that loads the
// library, held until the process exits.
constexpr int kMaxReceivers = 65536;
constexpr size_t kPosBytes = sizeof(double) * 3 * kMaxReceivers;
constexpr size_t kValBytes = sizeof(float) * 8 * kMaxReceivers;
constexpr size_t kCntBytes = sizeof(int) * kMaxReceivers;
constexpr size_t kScratchBytes = kPosBytes + 2 * kValBytes + kCntBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Grid {
    int nx, ny, nz;
    double hx, hy, hz;
};

// One thread per receiver: its trilinear taps (corner c = 4 dx + 2 dy + dz,
// corners with zero weight or outside the grid dropped, as in the plan's tap
// lists) and the field values there, written to the slots.
__global__ void noalloc_gather_kernel(unsigned char* scratch, Grid g, const float* __restrict__ u, int nrec)
{
    const double* pos = reinterpret_cast<const double*>(scratch);
    float* val = reinterpret_cast<float*>(scratch + kPosBytes);
    float* wgt = reinterpret_cast<float*>(scratch + kPosBytes + kValBytes);
    int* cnt = reinterpret_cast<int*>(scratch + kPosBytes + 2 * kValBytes);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    const double h[3] = {g.hx, g.hy, g.hz};
    const int n[3] = {g.nx, g.ny, g.nz};
    int i0[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        const double x = pos[3 * r + a] / h[a];
        const double fl = floor(x);
        i0[a] = static_cast<int>(fl);
        fr[a] = x - fl;
    }
    int c = 0;
    for (int corner = 0; corner < 8; ++corner) {
        const int d[3] = {(corner >> 2) & 1, (corner >> 1) & 1, corner & 1};
        double w = 1.0;
        bool inside = true;
        long long idx = 0;
        for (int a = 0; a < 3; ++a) {
            w *= d[a] ? fr[a] : 1.0 - fr[a];
            const int k = i0[a] + d[a];
            inside = inside && k >= 0 && k < n[a];
            idx = idx * n[a] + k;
        }
        if (w == 0.0 || !inside) continue;
        val[8 * r + c] = u[idx];
        wgt[8 * r + c] = static_cast<float>(w);
        ++c;
    }
    cnt[r] = c;
}

// One thread per receiver: sum of weight x value over its taps in corner order.
__global__ void noalloc_reduce_kernel(const unsigned char* scratch, float* __restrict__ rec, int nrec)
{
    const float* val = reinterpret_cast<const float*>(scratch + kPosBytes);
    const float* wgt = reinterpret_cast<const float*>(scratch + kPosBytes + kValBytes);
    const int* cnt = reinterpret_cast<const int*>(scratch + kPosBytes + 2 * kValBytes);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    float acc = 0.f;
    for (int t = 0; t < cnt[r]; ++t) acc = __fmaf_rn(wgt[8 * r + t], val[8 * r + t], acc);
    rec[r] = acc;
}

// Device address of the static array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

wave_status scratch_address(int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices) return wave::fail(WAVE_ERR_ARG, "wave_sample_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return wave::fail(WAVE_ERR_CUDA, std::string("wave_sample_noalloc: cudaGetSymbolAddress failed: ") +
                                                 cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return WAVE_OK;
}

}  // namespace

extern "C" wave_status wave_sample_noalloc(const int grid[3], const double spacing[3], const float* u, int nrec,
                                           const double* xyz, float* rec, void* stream)
{
    if (!grid || !spacing || !u || (nrec > 0 && (!xyz || !rec)))
        return wave::fail(WAVE_ERR_ARG, "wave_sample_noalloc: null argument");
    if (nrec < 0 || nrec > kMaxReceivers)
        return wave::fail(WAVE_ERR_ARG, "wave_sample_noalloc: nrec must be in [0, " + std::to_string(kMaxReceivers) +
                                            "] (the static slot array holds that many receivers)");
    for (int a = 0; a < 3; ++a)
        if (grid[a] < 1 || !(spacing[a] > 0.0) || !std::isfinite(spacing[a]))
            return wave::fail(WAVE_ERR_ARG, "wave_sample_noalloc: grid extents and spacing must be positive");
    if (nrec == 0) return WAVE_OK;
    // the kernel turns xyz / h into cell indices: only finite positions inside the grid get there
    std::string why;
    if (!wave::positions_valid(nrec, xyz, spacing, grid, &why))
        return wave::fail(WAVE_ERR_ARG, "wave_sample_noalloc: " + why);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return wave::fail(WAVE_ERR_CUDA, "wave_sample_noalloc: no current device");
    void* base = nullptr;
    wave_status s = scratch_address(dev, &base);
    if (s) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(base, xyz, sizeof(double) * 3 * static_cast<size_t>(nrec), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return wave::fail(WAVE_ERR_CUDA, std::string("wave_sample_noalloc: ") + cudaGetErrorString(e));
    const Grid g{grid[0], grid[1], grid[2], spacing[0], spacing[1], spacing[2]};
    const int blocks = (nrec + 255) / 256;
    noalloc_gather_kernel<<<blocks, 256, 0, st>>>(static_cast<unsigned char*>(base), g, u, nrec);
    noalloc_reduce_kernel<<<blocks, 256, 0, st>>>(static_cast<const unsigned char*>(base), rec, nrec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return wave::fail(WAVE_ERR_CUDA, std::string("wave_sample_noalloc: ") + cudaGetErrorString(e));
    return WAVE_OK;
}
