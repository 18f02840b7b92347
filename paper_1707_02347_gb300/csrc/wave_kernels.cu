// wave_kernels.cu -- the elementwise and reduction kernels of libwave.so and
// the dispatcher of the pipelined pass kernel (wave_pass.cuh).
#include "wave_kernels.cuh"

#include <mutex>
#include <vector>

namespace wave {

const PassShape* pass_shapes_r2(int* n);
const PassShape* pass_shapes_r4(int* n);
const PassShape* pass_shapes_r8(int* n);

namespace {
// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

__global__ void kappa_kernel(const float* __restrict__ m, float* __restrict__ kap, int nx, int ny, int nz, int nzp,
                             float dt2)
{
    const long long n = static_cast<long long>(nx) * ny * nzp;
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int z = static_cast<int>(p % nzp);
        const long long xy = p / nzp;
        kap[p] = z < nz ? __fdiv_rn(dt2, m[xy * nz + z]) : 0.f;
    }
}

__global__ void pad_kernel(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny, int nz, int nzp)
{
    const long long n = static_cast<long long>(nx) * ny * nzp;
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int z = static_cast<int>(p % nzp);
        const long long xy = p / nzp;
        dst[p] = z < nz ? src[xy * nz + z] : 0.f;
    }
}

__global__ void unpad_kernel(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny, int nz, int nzp)
{
    const long long n = static_cast<long long>(nx) * ny * nz;
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int z = static_cast<int>(p % nz);
        const long long xy = p / nz;
        dst[p] = src[xy * nzp + z];
    }
}

// rec[row][j] = sum over the taps of receiver j, in tap order, of w * value.
__global__ void rec_reduce_kernel(const float* __restrict__ slots, const int* __restrict__ tptr,
                                  const float* __restrict__ tw, float* __restrict__ rec, int rows, int nrec, int ntaps)
{
    const long long n = static_cast<long long>(rows) * nrec;
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int j = static_cast<int>(p % nrec);
        const long long row = p / nrec;
        float acc = 0.f;
        for (int t = tptr[j]; t < tptr[j + 1]; ++t) acc = __fmaf_rn(tw[t], slots[row * ntaps + t], acc);
        rec[p] = acc;
    }
}

// One trace row gathered from a field after a one-step pass: the taps of
// each receiver in the order (and with the arithmetic) of rec_reduce_kernel.
__global__ void rec_gather_kernel(const float* __restrict__ u, const int* __restrict__ gidx,
                                  const int* __restrict__ tptr, const float* __restrict__ tw, float* __restrict__ rec,
                                  int nrec)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nrec; j += gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int t = tptr[j]; t < tptr[j + 1]; ++t) acc = __fmaf_rn(tw[t], u[gidx[t]], acc);
        rec[j] = acc;
    }
}

// grad -= scale * mu * (v_new - v_old), scale = 1/dt^2: the imaging condition
// mu^{n+1} (u^{n+1} - 2u^n + u^{n-1}) / dt^2 with u^{n+1} - u^n = v^{n+1/2}.
__global__ void init_state_kernel(const float* __restrict__ u2, float* __restrict__ u, float* __restrict__ v, int nx,
                                  int ny, int nz, int nzp)
{
    const long long n = static_cast<long long>(nx) * ny * nzp;
    const long long dense = static_cast<long long>(nx) * ny * nz;
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int z = static_cast<int>(p % nzp);
        const long long xy = p / nzp;
        float a = 0.f, b = 0.f;
        if (z < nz) {
            a = u2[xy * nz + z];           // u^{-1}
            b = u2[dense + xy * nz + z];   // u^0
        }
        u[p] = b;
        v[p] = __fsub_rn(b, a);
    }
}

__global__ void final_state_kernel(const float* __restrict__ u, const float* __restrict__ v, float* __restrict__ u2,
                                   int nx, int ny, int nz, int nzp)
{
    const long long dense = static_cast<long long>(nx) * ny * nz;
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < dense;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int z = static_cast<int>(p % nz);
        const long long q = (p / nz) * nzp + z;
        u2[p] = __fsub_rn(u[q], v[q]);
        u2[dense + p] = u[q];
    }
}

// resid_rev[nt-1-n][j] = rec[n][j] - dobs[n][j]; partial[b] = per-block sum of squares (FP64).
__global__ void residual_kernel(const float* __restrict__ rec, const float* __restrict__ dobs,
                                float* __restrict__ resid_rev, double* __restrict__ partial, int nt, int nrec)
{
    __shared__ double red[256];
    const long long n = static_cast<long long>(nt) * nrec;
    double acc = 0.0;
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long row = p / nrec;
        const int j = static_cast<int>(p % nrec);
        const float e = __fsub_rn(rec[p], dobs[p]);
        resid_rev[(nt - 1 - row) * nrec + j] = e;
        acc += static_cast<double>(e) * static_cast<double>(e);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void reverse_rows_kernel(const float* __restrict__ src, float* __restrict__ dst, int nt, int ncol)
{
    const long long n = static_cast<long long>(nt) * ncol;
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long row = p / ncol;
        const int j = static_cast<int>(p % ncol);
        dst[(nt - 1 - row) * ncol + j] = src[p];
    }
}

unsigned grid_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152LL * 32) b = 152LL * 32;
    return static_cast<unsigned>(b);
}

}  // namespace

const PassShape* pass_shapes(int* count)
{
    static std::vector<PassShape> all;
    static std::once_flag once;
    std::call_once(once, [] {
        for (auto fn : {pass_shapes_r2, pass_shapes_r4, pass_shapes_r8}) {
            int n = 0;
            const PassShape* s = fn(&n);
            all.insert(all.end(), s, s + n);
        }
    });
    *count = static_cast<int>(all.size());
    return all.data();
}

const PassShape* find_pass_shape(int R, int T, int qz, int ry, int unroll)
{
    int n = 0;
    const PassShape* s = pass_shapes(&n);
    for (int i = 0; i < n; ++i)
        if (s[i].R == R && s[i].T == T && s[i].qz == qz && s[i].ry == ry && s[i].unroll == unroll) return &s[i];
    return nullptr;
}

cudaError_t launch_rec_gather(const float* u, const int* gidx, const int* tptr, const float* tw, float* rec, int nrec,
                              cudaStream_t st)
{
    rec_gather_kernel<<<grid_for(nrec, 256), 256, 0, st>>>(u, gidx, tptr, tw, rec, nrec);
    return cudaGetLastError();
}

cudaError_t launch_kappa(const float* m, float* kap, int nx, int ny, int nz, int nzp, float dt2, cudaStream_t st)
{
    kappa_kernel<<<grid_for(static_cast<long long>(nx) * ny * nzp, 256), 256, 0, st>>>(m, kap, nx, ny, nz, nzp, dt2);
    return cudaGetLastError();
}

cudaError_t launch_pad_copy(const float* src, float* dst, int nx, int ny, int nz, int nzp, cudaStream_t st)
{
    pad_kernel<<<grid_for(static_cast<long long>(nx) * ny * nzp, 256), 256, 0, st>>>(src, dst, nx, ny, nz, nzp);
    return cudaGetLastError();
}

cudaError_t launch_unpad_copy(const float* src, float* dst, int nx, int ny, int nz, int nzp, cudaStream_t st)
{
    unpad_kernel<<<grid_for(static_cast<long long>(nx) * ny * nz, 256), 256, 0, st>>>(src, dst, nx, ny, nz, nzp);
    return cudaGetLastError();
}

cudaError_t launch_unpad_grad(const float* src, float* dst, int nx, int ny, int nz, int nzp, cudaStream_t st)
{
    return launch_unpad_copy(src, dst, nx, ny, nz, nzp, st);
}

cudaError_t launch_rec_reduce(const float* slots, const int* tptr, const float* tw, float* rec, int rows, int nrec,
                              int ntaps, cudaStream_t st)
{
    if (rows <= 0 || nrec <= 0) return cudaSuccess;
    rec_reduce_kernel<<<grid_for(static_cast<long long>(rows) * nrec, 256), 256, 0, st>>>(slots, tptr, tw, rec, rows,
                                                                                          nrec, ntaps);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const float* u2, float* u, float* v, int nx, int ny, int nz, int nzp, cudaStream_t st)
{
    init_state_kernel<<<grid_for(static_cast<long long>(nx) * ny * nzp, 256), 256, 0, st>>>(u2, u, v, nx, ny, nz,
                                                                                           nzp);
    return cudaGetLastError();
}

cudaError_t launch_final_state(const float* u, const float* v, float* u2, int nx, int ny, int nz, int nzp,
                               cudaStream_t st)
{
    final_state_kernel<<<grid_for(static_cast<long long>(nx) * ny * nz, 256), 256, 0, st>>>(u, v, u2, nx, ny, nz,
                                                                                           nzp);
    return cudaGetLastError();
}

cudaError_t launch_residual(const float* rec, const float* dobs, float* resid_rev, double* partial, int nt, int nrec,
                            cudaStream_t st)
{
    residual_kernel<<<256, 256, 0, st>>>(rec, dobs, resid_rev, partial, nt, nrec);
    return cudaGetLastError();
}

cudaError_t launch_reverse_rows(const float* src, float* dst, int nt, int ncol, cudaStream_t st)
{
    if (nt <= 0 || ncol <= 0) return cudaSuccess;
    reverse_rows_kernel<<<grid_for(static_cast<long long>(nt) * ncol, 256), 256, 0, st>>>(src, dst, nt, ncol);
    return cudaGetLastError();
}

}  // namespace wave
