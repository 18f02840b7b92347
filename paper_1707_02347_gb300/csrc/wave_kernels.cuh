// wave_kernels.cuh -- device-side interface shared by the kernels and the
// host code of libwave.so.  Nothing here is visible through the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wave {

constexpr int kMaxR = 8;

// Geometry and inputs of one pass of the pipelined kernel (see wave_kernels.cu).
struct PassArgs {
    int nx, ny, nz, nzp;    // grid; nzp = z extent of the padded device layout
    long long sx;           // elements per x plane of the padded layout (ny * nzp)
    int by, bz, xc;         // output tile along y, z and x-slab length
    int nty, ntz;           // tiles along y and z
    int qz, r1y;            // threads per row (z quads) and rows of the thread region
    int zlead;              // z of the thread region relative to the tile's z0 (<= 0, multiple of 4)
    int a_rows, a_cols;     // staged box of u^n (thread region plus the stencil halo)
    int b_rows, b_cols;     // staged box of v^{n-1/2} and kappa (the thread region)
    float* out_u;           // receives u^{n+T}
    float* out_v;           // receives v^{n+T-1/2} = u^{n+T} - u^{n+T-1} (may alias the input for T = 1)
    const float* kap;       // kappa = dt^2 / m, padded layout
    const float* damp_x;    // sponge profile per axis: d(x,y,z) = dx[x] + (dy[y] + dz[z])
    const float* damp_y;
    const float* damp_z;
    int dxlo, dxhi;         // planes x in [dxlo, dxhi) have dx[x] == 0
    float inv2dt;           // 1 / (2 dt)
    float2 c0;              // (a_0 + 2 a_1) (1/hx^2 + 1/hy^2 + 1/hz^2), twice: centre weight of the k >= 2 pairs
    float2 cx[kMaxR], cy[kMaxR], cz[kMaxR];  // a_k / h^2 per axis, each twice (operands of packed pair ops)
    int n0;                 // time level n at the start of the pass
    // sources: per z-quad column CSR of {x, lane, source, weight bits}, sorted by x
    const int* src_ptr;
    const int4* src_ent;
    const float* wavelet;   // [nt][nsrc]
    int nsrc;
    // receivers: per column CSR of {x, (tap << 2) | lane}; values go to slots
    const int* rec_ptr;
    const int2* rec_ent;
    float* slots;           // [rows][ntaps]
    int ntaps;
    int slot_row0;          // rec row stored in slot row 0
    // skewed wavefront tiling (variant 4): tile j of a column of y tiles
    // takes the top rows of tile j-1's first step from `exch` once tile j-1's
    // progress word says the plane is there.  sync: [nitems] progress words
    // (iterations completed) then the work counter; exch: [nitems][exch_nit]
    // [3 r][4 qz] floats per tile.
    float* exch;
    int* sync;
    int nitems;
    int exch_nit;
    int* err;               // device error word (bit 0: a bounded wait gave up; bit 1: a tile waited too long for its neighbour)
    // imaging condition of the FWI gradient, fused into a one-step adjoint
    // pass (gacc == nullptr: none): at every point the pass writes,
    // gacc += -(img_scale * mu) * (img_vn - img_vo), mu the adjoint field it
    // wrote and img_vn - img_vo = v^{j-1/2} - v^{j-3/2} of the forward
    float* gacc;
    const float* img_vn;
    const float* img_vo;
    float img_scale;
};

// One compiled instantiation of the pass kernel: radius R, T steps, thread
// blocks of `ry` rows by `qz` z quads, its shared memory and its launcher.
struct PassShape {
    int R, T, qz, ry;
    int unroll;  // variant: x-queue storage 0 = registers (moved), 1 = registers (loop unrolled),
                 // 2 = tensor memory; 4 = skewed wavefront tiling in y (T = 2, tensor memory);
                 // 5, 6 = warp-specialised pass (tensor memory), 1 or 2 rows per thread;
                 // 7 = warp-specialised pass, 2 rows per thread, tensor-memory shift registers
    size_t smem;
    cudaError_t (*launch)(const CUtensorMap& mapA, const CUtensorMap& mapV, const CUtensorMap& mapK,
                          const PassArgs& a, int threads, size_t smem, long long blocks, cudaStream_t st);
};

// Every compiled shape (wave_pass_r*.cu), and the one matching (R, T, qz, ry)
// or nullptr.  A pass runs from the state (u^n, v^{n-1/2}): mapA over u^n,
// mapV over v^{n-1/2}, mapK over kappa.
const PassShape* pass_shapes(int* count);
const PassShape* find_pass_shape(int R, int T, int qz, int ry, int unroll);

// Persistent kernel of batched shots (wave_batch.cu).  One descriptor per
// (shot, pass kind): the shot's index and the index of its compiled batch
// shape; its pass arguments (n0 set per item) are entry d of the kernel's
// constant array (batch_copy_args), its three tensor maps (u^n with the
// stencil halo, v^{n-1/2}, kappa) maps[3 d .. 3 d + 2].  Items are int4
// {descriptor, tile, tiles of the shot that must be done first, n0}, in
// queue order; an item of a team shape covers tiles [tile, tile + 4) of its
// pass (those below ntiles).
constexpr int kMaxBatchArgs = 112;
struct BatchDesc {
    int shot;
    int shape;
    int team;    // 1: a one-step team shape (four tiles per item)
    int ntiles;  // tiles of the pass
};
struct BatchQueue {
    const BatchDesc* desc;
    const CUtensorMap* maps;  // 64-byte aligned
    const int4* items;
    int nitems;
    int* next;                // work counter (starts at 0)
    int* done;                // finished tiles per shot (start at 0)
    int* abort;               // set when a dependency wait gave up
    int* err;                 // bit 0: a tile's TMA wait gave up; bit 1: a dependency wait gave up
    unsigned long long limit_ns;  // bound on a dependency wait
};
// Index of the compiled batch shape (radius, T, z quads per row, rows,
// variant) or -1; the dynamic shared memory of the kernel; its launch.
int batch_shape_index(int R, int T, int qz, int ry, int unroll);
bool batch_shape_is_team(int shape);
size_t batch_smem_bytes();
// Copy n <= kMaxBatchArgs pass arguments (device memory) into the constant
// array the persistent kernel reads; stream-ordered (capturable).
cudaError_t batch_copy_args(const PassArgs* dev_args, int n, cudaStream_t st);
cudaError_t launch_batch(const BatchQueue& q, int blocks, cudaStream_t st);

// Elementwise helpers.
cudaError_t launch_kappa(const float* m, float* kap, int nx, int ny, int nz, int nzp, float dt2, cudaStream_t st);
cudaError_t launch_pad_copy(const float* src, float* dst, int nx, int ny, int nz, int nzp, cudaStream_t st);
cudaError_t launch_unpad_copy(const float* src, float* dst, int nx, int ny, int nz, int nzp, cudaStream_t st);
// (u^{-1}, u^0) dense -> state u = u^0, v = u^0 - u^{-1} (padded)
cudaError_t launch_init_state(const float* u2, float* u, float* v, int nx, int ny, int nz, int nzp, cudaStream_t st);
// state (u, v) padded -> dense (u - v, u)
cudaError_t launch_final_state(const float* u, const float* v, float* u2, int nx, int ny, int nz, int nzp,
                               cudaStream_t st);
cudaError_t launch_rec_reduce(const float* slots, const int* tptr, const float* tw, float* rec, int rows,
                              int nrec, int ntaps, cudaStream_t st);
// rec[j] = sum over the taps t of receiver j (in order) of tw[t] * u[gidx[t]]: one trace row
// gathered from a field in the padded layout, the same sums in the same order as
// launch_rec_reduce.
cudaError_t launch_rec_gather(const float* u, const int* gidx, const int* tptr, const float* tw, float* rec, int nrec,
                              cudaStream_t st);
cudaError_t launch_unpad_grad(const float* src, float* dst, int nx, int ny, int nz, int nzp, cudaStream_t st);
cudaError_t launch_residual(const float* rec, const float* dobs, float* resid_rev, double* partial, int nt,
                            int nrec, cudaStream_t st);
cudaError_t launch_reverse_rows(const float* src, float* dst, int nt, int ncol, cudaStream_t st);

}  // namespace wave
