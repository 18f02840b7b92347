// wave_host.h -- host-side internals of libwave.so (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/wave.h"

namespace wave {

// Thread-local message behind wave_last_error().
void set_error(const std::string& msg);
wave_status fail(wave_status s, const std::string& msg);

// FD weights a_0..a_r as exact rationals rounded to double (fd_weights.cpp).
bool fd_weights_exact(int so, double* a);
// rho = |a_0| + 2 sum_k |a_k| (the stencil's spectral radius on unit spacing).
double fd_spectral_radius(int so);

// Geometry of one pass of the pipelined kernel for a grid, radius and tiling
// (schedule.cpp).  See wave_kernels.cuh for the meaning of the fields.
struct PassGeom {
    int R = 0, T = 0, by = 0, bz = 0, xc = 0;
    int nty = 0, ntz = 0, nxs = 0;
    int qz = 0, r1y = 0, zlead = 0;
    int a_rows = 0, a_cols = 0, b_rows = 0, b_cols = 0;
    int threads = 0;         // threads of a block (qz * r1y, whole warps)
    int block = 0;           // launched block size (= threads)
    const struct PassShape* shape = nullptr;  // the compiled instantiation
    long long blocks = 0;
    size_t smem = 0;
};

int padded_nz(int nz);
// Fill g for (grid, R, tiling); false with a reason if the tiling is not legal
// for the kernel (limits, alignment, TMA box sizes, shared memory).
// need_kernel = false checks the schedule geometry only (no compiled shape needed).
bool make_geom(const int grid[3], int R, const wave_tiling& t, PassGeom* g, std::string* why,
               bool need_kernel = true);
// Built-in default tiling for a grid, radius and T.
wave_tiling default_tiling(const int grid[3], int R, int T);
// Candidate tilings for the autotuner.
std::vector<wave_tiling> tiling_candidates(const int grid[3], int R);

// Trilinear taps of a point (schedule-independent, taps.cpp).
struct Tap {
    int i, j, k;
    double w;
};
// True if every coordinate of the count points is finite and inside
// [0, (n_a - 1) h_a] (the grid's extent), else false with the first offender
// in *why.  Checked before any position reaches trilinear_taps.
bool positions_valid(int count, const double* xyz, const double h[3], const int n[3], std::string* why);
// Corners of the cell containing xyz with non-zero weight and inside the grid,
// in corner order c = 4 dx + 2 dy + dz.
int trilinear_taps(const double xyz[3], const double h[3], const int n[3], Tap out[8]);

// Per z-quad column CSR of sparse entries sorted by (column, x, lane, id).
struct ColumnCsr {
    std::vector<int> ptr;      // ncols + 1
    std::vector<int> ent;      // 4 ints per source entry or 2 per receiver entry
};
// Sources: entry {x, lane, source index, weight as float bits}.
void build_source_csr(int nsrc, const double* xyz, const double h[3], const int n[3], int nzp, ColumnCsr* out);
// Receivers: entry {x, (tap << 2) | lane}; taps numbered receiver by receiver;
// tptr [nrec + 1] and tw [ntaps] describe each receiver's taps and weights.
void build_receiver_csr(int nrec, const double* xyz, const double h[3], const int n[3], int nzp, ColumnCsr* out,
                        std::vector<int>* tptr, std::vector<float>* tw);

// Gather plan of a dense receiver surface (taps in at most two adjacent z
// quads, at least min_rec receivers): per tap its index in the padded layout.
bool receiver_gather_plan(int nrec, const double* xyz, const double h[3], const int n[3], int nzp, int min_rec,
                          std::vector<int>* idx);

// Sponge profile of one axis (1/ms), in double, rounded to float by the caller.
void sponge_profile(int n, int width, bool lo, bool hi, double dmax, std::vector<float>* out, int padded_n);

}  // namespace wave
