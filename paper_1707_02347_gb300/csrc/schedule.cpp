// schedule.cpp -- tile-legality scheduler of libwave.so.
//
// McCormick 2017, Section "Skewing Dependencies": the acoustic stencil reads
// u[time] at offsets +-r (r = SO/2) along every axis, i.e. the dependence
// distance vectors (1, 0, 0, +-r), (1, 0, +-r, 0), (1, +-r, 0, 0).  A tiling
// through time is legal when every dependence distance, after skewing each
// tiled space loop by r per time step, is lexicographically non-negative
// (Section "Legality of Tiling").
//
// The GPU schedule (wave_pass.cuh) applies this once per pass of T steps:
//   * along x, the streamed axis, step k of the pass works r planes behind
//     step k-1 (skew factor r), so every value a step reads along x has
//     already been produced by the previous step of the same thread block;
//   * across y and z each thread block recomputes an overlapped halo of
//     r (T - k) points at step k, so blocks never wait for each other
//     inside a pass (the overlap replaces the paper's skewed tile shapes
//     in the two tiled dimensions, and needs no inter-block ordering);
//   * reads come only from the pass's input buffer set and writes go to the
//     other set, so no write-after-read hazard crosses blocks (the paper's
//     rolling "time dimension buffering" bounds the time tile by the buffer
//     modulus instead).
// make_geom() checks the kernel's limits for a tiling; verify_schedule()
// enumerates the schedule on a small grid and checks every dependence.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "wave_host.h"
#include "wave_kernels.cuh"

namespace wave {

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

int padded_nz(int nz) { return round_up(nz, 4); }

bool make_geom(const int grid[3], int R, const wave_tiling& t, PassGeom* g, std::string* why, bool need_kernel)
{
    auto no = [&](const std::string& s) {
        if (why) *why = s;
        return false;
    };
    if (R != 2 && R != 4 && R != 8) return no("space order must be 4, 8 or 16");
    if (t.T < 1) return no("T must be >= 1");
    if (t.by < 1) return no("tile by must be >= 1");
    if (t.bz < 4 || t.bz % 4) return no("tile bz must be a positive multiple of 4");
    if (t.xc < 1) return no("slab xc must be >= 1");
    const int nx = grid[0], ny = grid[1], nzp = padded_nz(grid[2]);
    PassGeom G;
    G.R = R;
    G.T = t.T;
    G.by = t.by;
    G.bz = t.bz;
    G.xc = std::min(t.xc, nx);
    const int halo = R * (t.T - 1);  // overlapped halo of step 1
    const bool skew = t.unroll == 4;  // skewed wavefront tiling in y (T = 2 only)
    if (skew && t.T != 2) return no("the skewed wavefront variant has T = 2");
    if (skew && t.by < 2 * R) return no("the skewed wavefront variant needs by >= SO");
    G.zlead = -round_up(halo, 4);
    G.b_cols = round_up(t.bz + halo, 4) - G.zlead;
    G.qz = G.b_cols / 4;
    G.r1y = skew ? t.by + halo : t.by + 2 * halo;  // skewed: the tile shifts by r per step
    G.b_rows = G.r1y;
    const int ZH = round_up(R, 4);
    G.a_rows = G.r1y + 2 * R;
    G.a_cols = G.b_cols + 2 * ZH;
    G.threads = G.qz * G.r1y;
    // variants 5, 6, 7: one compute thread per 1 or 2 rows of a quad, plus the producer warp
    G.block = (t.unroll == 5) ? G.threads + 32 : (t.unroll == 6 || t.unroll == 7) ? G.threads / 2 + 32 : G.threads;
    G.shape = find_pass_shape(R, t.T, G.qz, G.r1y, t.unroll);
    if (!G.shape && need_kernel)
        return no("no compiled kernel for SO " + std::to_string(2 * R) + ", T = " + std::to_string(t.T) +
                  " with " + std::to_string(G.r1y) + " thread rows of " + std::to_string(G.qz) + " z quads" +
                  (t.unroll ? " (unrolled)" : ""));
    G.smem = G.shape ? G.shape->smem : 0;
    if (G.smem > 227 * 1024) return no("tile needs " + std::to_string(G.smem) + " bytes of shared memory");
    G.nty = skew ? (ny + R + t.by - 1) / t.by : (ny + t.by - 1) / t.by;
    G.ntz = (nzp + t.bz - 1) / t.bz;
    G.nxs = (nx + G.xc - 1) / G.xc;
    G.blocks = static_cast<long long>(G.nty) * G.ntz * G.nxs;
    if (G.blocks > 0x7fffffffLL) return no("too many thread blocks");
    *g = G;
    return true;
}

// The compiled shape (qz, r1y) of a variant as an output tile (by, bz) for radius R and T.
static bool shape_tile(int R, int T, int qz, int ry, int variant, int* by, int* bz)
{
    const int halo = R * (T - 1);
    *by = variant == 4 ? ry - halo : ry - 2 * halo;
    // largest bz (multiple of 4) with round_up(bz + halo, 4) + round_up(halo, 4) == 4 qz
    *bz = 0;
    for (int b = 4; b <= 4 * qz; b += 4)
        if (round_up(b + halo, 4) + round_up(halo, 4) == 4 * qz) *bz = b;
    return *by >= 1 && *bz >= 4;
}

wave_tiling default_tiling(const int grid[3], int R, int T)
{
    // the first compiled shape of (R, T) (bank-conflict-free: rows of 8, 16 or 32 quads)
    wave_tiling t{T, 0, 0, std::min(grid[0], 128), 0};
    int n = 0;
    const PassShape* s = pass_shapes(&n);
    for (int i = 0; i < n; ++i)
        if (s[i].R == R && s[i].T == T && s[i].unroll == 0 &&
            shape_tile(R, T, s[i].qz, s[i].ry, 0, &t.by, &t.bz))
            return t;
    return wave_tiling{T, 0, 0, 0, 0};
}

std::vector<wave_tiling> tiling_candidates(const int grid[3], int R)
{
    // every compiled shape of radius R, with four slab lengths (short slabs
    // give small grids more thread blocks than the SMs hold at once)
    std::vector<wave_tiling> out;
    int n = 0;
    const PassShape* s = pass_shapes(&n);
    const int slabs[] = {32, 64, 128, 256};
    for (int i = 0; i < n; ++i) {
        if (s[i].R != R) continue;
        int by, bz;
        if (!shape_tile(R, s[i].T, s[i].qz, s[i].ry, s[i].unroll, &by, &bz)) continue;
        for (int xc : slabs) {
            wave_tiling t{s[i].T, by, bz, std::min(xc, grid[0]), s[i].unroll};
            PassGeom g;
            if (!make_geom(grid, R, t, &g, nullptr)) continue;
            bool dup = false;
            for (auto& o : out)
                dup = dup || (o.T == t.T && o.by == t.by && o.bz == t.bz && o.xc == t.xc && o.unroll == t.unroll);
            if (!dup) out.push_back(t);
        }
    }
    return out;
}

// ---------------------------------------------------------------------------
// Brute-force verification of the pass schedule.
//
// Model: one pass of T steps from levels (n-1, n).  For each thread block,
// step k (1..T) at loop iteration i computes plane x_k = xbase + i - lag k for
// every column of the block's thread region, when i >= 2 lag k.  A computed
// value is valid when every value it reads is valid:
//   u^{n+k-1} at (x_k +- j, y, z), (x_k, y +- j, z), (x_k, y, z +- j), j <= r,
//   u^{n+k-2} at (x_k, y, z);
// levels n-1 and n are the pass input (valid everywhere, zero outside the
// grid); points outside the grid are forced to zero and count as valid.
// Every output point of levels n+T-1 and n+T must be written exactly once,
// by its owning block, with a valid value.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Brute-force verification of the skewed wavefront variant (T = 2).
//
// Model (wave_skew.cuh): tiles of BY rows along y, x slabs and z tiles, taken
// in wavefront order (y level, slab, z tile).  Tile j computes step 1 (level
// n+1) on rows [y0, y0 + BY) and step 2 (level n+2) on rows [y0 - r, y0 +
// BY - r), both over the z columns of its region (z carries an overlapped
// halo), step k at plane x_k = xbase + i - r k of iteration i (i >= 2 r k).
// The only values a tile takes from another are level n+1 on the
// `exchange_rows` rows below y0, produced by tile j-1 of the same slab and z
// tile; a value tile j-1 produced in its iteration p may be read by tile j
// in its iteration i only if p <= i + wait_lead - 1 (the kernel waits, before
// iteration i copies the rows it needs at i+1, until tile j-1 has completed
// iteration i+1: exchange_rows = 2r, wait_lead = 1).  Rows outside the grid
// are zero.  Every output point (levels n+1 and n+2, the v form's (u, v))
// must be written exactly once, by the tile that owns it, with a valid value.
// ---------------------------------------------------------------------------
static bool verify_skew_schedule(const int grid[3], int R, const wave_tiling& t, int exchange_rows, int wait_lead,
                                 std::string* why)
{
    PassGeom g;
    if (!make_geom(grid, R, t, &g, why, false)) return false;
    if (t.unroll != 4 || t.T != 2) {
        if (why) *why = "not a skewed wavefront tiling";
        return false;
    }
    const int nx = grid[0], ny = grid[1], nz = grid[2];
    const int BY = t.by, RY = g.r1y, bcols = g.b_cols;
    const int nxs = g.nxs;
    auto in_grid = [&](int x, int y, int z) { return x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz; };
    auto pidx = [&](int x, int y, int z) { return (static_cast<size_t>(x) * ny + y) * nz + z; };
    std::vector<int> writes(static_cast<size_t>(nx) * ny * nz, 0);
    // level n+1 of tile j-1 (same slab and z tile): iteration that produced
    // it (-1: not produced) and validity, over its box
    struct Box {
        int x0 = 0, y0 = 0, z0 = 0, nxb = 0, nyb = 0, nzb = 0;
        std::vector<int> iter;
        std::vector<char> ok;
        size_t at(int x, int y, int z) const
        {
            return (static_cast<size_t>(x - x0) * nyb + (y - y0)) * nzb + (z - z0);
        }
        bool inside(int x, int y, int z) const
        {
            return x >= x0 && x < x0 + nxb && y >= y0 && y < y0 + nyb && z >= z0 && z < z0 + nzb;
        }
    };
    std::vector<Box> prev(static_cast<size_t>(nxs) * g.ntz);  // per (slab, z tile): the tile below
    for (int tyi = 0; tyi < g.nty; ++tyi)
        for (int xsi = 0; xsi < nxs; ++xsi)
            for (int tzi = 0; tzi < g.ntz; ++tzi) {
                const int y0 = tyi * BY, z0 = tzi * t.bz;
                const int ylo = y0 - R, zlo = z0 + g.zlead;
                const int X0 = xsi * g.xc, X1 = std::min(X0 + g.xc, nx);
                const int NIT = (X1 - X0) + 4 * R, xbase = X0 - 2 * R;
                Box cur;  // this tile's levels n+1 (index 0) and n+2 (index 1) over its region
                cur.x0 = xbase - 2 * R;
                cur.y0 = ylo;
                cur.z0 = zlo;
                cur.nxb = NIT + 2 * R;
                cur.nyb = RY;
                cur.nzb = bcols;
                const size_t nb = static_cast<size_t>(cur.nxb) * cur.nyb * cur.nzb;
                std::vector<int> it1(nb, -1);
                std::vector<char> ok1(nb, 0), ok2(nb, 0), done2(nb, 0);
                const Box& below = prev[static_cast<size_t>(xsi) * g.ntz + tzi];
                // level n+1 at (x, y, z) as read by this tile in iteration i
                auto lev1 = [&](int x, int y, int z, int i) -> bool {
                    if (!in_grid(x, y, z)) return true;  // zero ghost
                    if (y >= y0 && y < y0 + BY) {
                        if (!cur.inside(x, y, z)) return false;
                        const size_t a = cur.at(x, y, z);
                        return it1[a] >= 0 && it1[a] <= i && ok1[a];
                    }
                    if (y < y0 && y >= y0 - exchange_rows && tyi > 0) {
                        if (!below.inside(x, y, z)) return false;
                        const size_t a = below.at(x, y, z);
                        return below.iter[a] >= 0 && below.iter[a] <= i + wait_lead - 1 && below.ok[a];
                    }
                    return false;  // neither computed here nor exchanged
                };
                for (int i = 0; i < NIT; ++i) {
                    // step 1 at plane x1, rows [y0, y0 + BY): reads the pass input only
                    if (i >= 2 * R) {
                        const int x = xbase + i - R;
                        for (int y = y0; y < y0 + BY; ++y)
                            for (int z = zlo; z < zlo + bcols; ++z) {
                                const size_t a = cur.at(x, y, z);
                                it1[a] = i;
                                ok1[a] = 1;
                            }
                    }
                    // step 2 at plane x2, rows [y0 - r, y0 + BY - r)
                    if (i >= 4 * R) {
                        const int x = xbase + i - 2 * R;
                        for (int y = y0 - R; y < y0 + BY - R; ++y)
                            for (int z = zlo; z < zlo + bcols; ++z) {
                                bool ok = true;
                                if (in_grid(x, y, z)) {
                                    for (int j = -R; j <= R && ok; ++j) {
                                        ok = ok && lev1(x + j, y, z, i);
                                        ok = ok && lev1(x, y + j, z, i);
                                        ok = ok && lev1(x, y, z + j, i);
                                    }
                                }
                                const size_t a = cur.at(x, y, z);
                                ok2[a] = ok;
                                done2[a] = 1;
                                // outputs: u^{n+2} and v^{n+3/2} of the owned points
                                if (x >= X0 && x < X1 && z >= z0 && z < std::min(z0 + t.bz, nz) && y >= 0 &&
                                    y < ny) {
                                    if (!ok || !lev1(x, y, z, i)) {
                                        if (why)
                                            *why = "tile (" + std::to_string(tyi) + "," + std::to_string(xsi) + "," +
                                                   std::to_string(tzi) + ") writes an invalid value at (" +
                                                   std::to_string(x) + "," + std::to_string(y) + "," +
                                                   std::to_string(z) + ")";
                                        return false;
                                    }
                                    writes[pidx(x, y, z)]++;
                                }
                            }
                    }
                }
                Box& keep = prev[static_cast<size_t>(xsi) * g.ntz + tzi];
                keep = cur;
                keep.iter = std::move(it1);
                keep.ok = std::move(ok1);
            }
    for (size_t p = 0; p < writes.size(); ++p)
        if (writes[p] != 1) {
            if (why) *why = "point " + std::to_string(p) + " written " + std::to_string(writes[p]) + " times";
            return false;
        }
    return true;
}

static bool verify_schedule(const int grid[3], int R, const wave_tiling& t, int lag, int halo_per_step,
                            std::string* why)
{
    PassGeom g;
    if (!make_geom(grid, R, t, &g, why, false)) return false;
    if (t.unroll == 4) {
        // the skewed variant has no lag or halo parameters of its own: its
        // model checks the exchange between tiles instead
        if (lag != R || halo_per_step != R) {
            if (why) *why = "the skewed wavefront variant has no lag or halo parameters";
            return false;
        }
        return verify_skew_schedule(grid, R, t, 2 * R, 1, why);
    }
    const int nx = grid[0], ny = grid[1], nz = grid[2];
    const int T = t.T;
    // geometry under test: the thread region carries halo_per_step (T-1) rows
    const int halo = halo_per_step * (T - 1);
    const int zlead = -round_up(halo, 4);
    const int b_cols = round_up(t.bz + halo, 4) - zlead;
    const int r1y = t.by + 2 * halo;
    auto pidx = [&](int x, int y, int z) { return (static_cast<size_t>(x) * ny + y) * nz + z; };
    const size_t npts = static_cast<size_t>(nx) * ny * nz;
    std::vector<int> writes_cur(npts, 0), writes_prev(npts, 0);
    // valid[k][x][y][z] per block: levels n+k, k = 1..T (index k-1)
    const int xs_len = g.xc;
    for (long long b = 0; b < g.blocks; ++b) {
        long long bb = b;
        const int tzi = static_cast<int>(bb % g.ntz);
        bb /= g.ntz;
        const int tyi = static_cast<int>(bb % g.nty);
        const int xsi = static_cast<int>(bb / g.nty);
        const int y0 = tyi * t.by, z0 = tzi * t.bz;
        const int X0 = xsi * xs_len, X1 = std::min(X0 + xs_len, nx);
        const int NIT = (X1 - X0) + 2 * lag * T;
        const int xbase = X0 - lag * T;
        const int ylo = y0 - halo, zlo = z0 + zlead;
        // computed[k] over the block's box: x in [xbase - lag T, X1 + lag T), y rows, z cols
        const int bx0 = xbase - lag * T - 1, bxn = NIT + 2 * lag * T + 2;
        auto in_region = [&](int y, int z) { return y >= ylo && y < ylo + r1y && z >= zlo && z < zlo + b_cols; };
        // state: 0 = not computed, 1 = valid, 2 = invalid
        std::vector<std::vector<char>> st(T + 1,
                                          std::vector<char>(static_cast<size_t>(bxn) * r1y * b_cols, 0));
        auto sidx = [&](int x, int y, int z) {
            return (static_cast<size_t>(x - bx0) * r1y + (y - ylo)) * b_cols + (z - zlo);
        };
        auto in_grid = [&](int x, int y, int z) {
            return x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz;
        };
        // value of level n+k (k >= 1) at a point, as seen by this block
        auto level_valid = [&](int k, int x, int y, int z) -> bool {
            if (k <= 0) return true;  // pass input (or its zero ghosts)
            if (!in_grid(x, y, z)) {
                // ghost: the block forces zero wherever it computes; outside its
                // region the value is only read if some computed point needs it
                if (!in_region(y, z) || x - bx0 < 0 || x - bx0 >= bxn) return false;
                return st[k][sidx(x, y, z)] != 0;
            }
            if (!in_region(y, z) || x - bx0 < 0 || x - bx0 >= bxn) return false;
            return st[k][sidx(x, y, z)] == 1;
        };
        for (int i = 0; i < NIT; ++i) {
            for (int k = 1; k <= T; ++k) {
                if (i < 2 * lag * k) continue;
                const int x = xbase + i - lag * k;
                for (int y = ylo; y < ylo + r1y; ++y)
                    for (int z = zlo; z < zlo + b_cols; ++z) {
                        bool ok = true;
                        if (in_grid(x, y, z)) {
                            for (int j = -R; j <= R && ok; ++j) {
                                ok = ok && level_valid(k - 1, x + j, y, z);
                                ok = ok && level_valid(k - 1, x, y + j, z);
                                ok = ok && level_valid(k - 1, x, y, z + j);
                            }
                            ok = ok && level_valid(k - 2, x, y, z);
                        }
                        if (x - bx0 >= 0 && x - bx0 < bxn) st[k][sidx(x, y, z)] = ok ? 1 : 2;
                    }
            }
            // outputs of plane x_T
            if (i >= 2 * lag * T) {
                const int x = xbase + i - lag * T;
                for (int y = y0; y < std::min(y0 + t.by, ny); ++y)
                    for (int z = z0; z < std::min(z0 + t.bz, nz); ++z) {
                        if (x < X0 || x >= X1) continue;
                        if (!level_valid(T, x, y, z) || !level_valid(T - 1, x, y, z)) {
                            if (why)
                                *why = "block " + std::to_string(b) + " writes an invalid value at (" +
                                       std::to_string(x) + "," + std::to_string(y) + "," + std::to_string(z) + ")";
                            return false;
                        }
                        writes_cur[pidx(x, y, z)]++;
                        writes_prev[pidx(x, y, z)]++;
                    }
            }
        }
    }
    for (size_t p = 0; p < npts; ++p)
        if (writes_cur[p] != 1 || writes_prev[p] != 1) {
            if (why) *why = "point " + std::to_string(p) + " written " + std::to_string(writes_cur[p]) + " times";
            return false;
        }
    return true;
}

// Paper's loop order in 1D + t (Fig. tiled_skew_snippet): skewed coordinate
// x' = x + skew t; tiles of tt steps by ts skewed points, executed in the
// lexicographic order (time tile, space tile, t, x').  Checks every read of
// u[t-1][x +- j] (j <= r) and u[t-2][x] happens after its write.
static bool skewed_order_legal(int n, int nt, int r, int skew, int tt, int ts)
{
    if (n <= 2 * r || nt < 1 || tt < 1 || ts < 1 || skew < 0) return false;
    struct Pt { long long key[4]; int t, x; };
    std::vector<Pt> pts;
    for (int t = 1; t <= nt; ++t)
        for (int x = r; x < n - r; ++x) {
            const int xs = x + skew * t;
            pts.push_back({{(t - 1) / tt, xs / ts, t, xs}, t, x});
        }
    std::sort(pts.begin(), pts.end(), [](const Pt& a, const Pt& b) {
        return std::lexicographical_compare(a.key, a.key + 4, b.key, b.key + 4);
    });
    std::vector<long long> when(static_cast<size_t>(nt + 1) * n, -1);
    for (size_t o = 0; o < pts.size(); ++o) when[static_cast<size_t>(pts[o].t) * n + pts[o].x] = static_cast<long long>(o);
    for (size_t o = 0; o < pts.size(); ++o) {
        const int t = pts[o].t, x = pts[o].x;
        for (int j = -r; j <= r; ++j) {
            const int xx = x + j;
            if (t - 1 >= 1 && xx >= r && xx < n - r && when[static_cast<size_t>(t - 1) * n + xx] > static_cast<long long>(o))
                return false;
        }
        if (t - 2 >= 1 && when[static_cast<size_t>(t - 2) * n + x] > static_cast<long long>(o)) return false;
    }
    return true;
}

}  // namespace wave

extern "C" int wave_skew_factor(int so) { return so / 2; }

extern "C" wave_status wave_tiling_check(const int grid[3], int so, const wave_tiling* tiling)
{
    if (!grid || !tiling) return wave::fail(WAVE_ERR_ARG, "wave_tiling_check: null argument");
    wave::PassGeom g;
    std::string why;
    if (!wave::make_geom(grid, so / 2, *tiling, &g, &why)) return wave::fail(WAVE_ERR_ARG, why);
    return WAVE_OK;
}

extern "C" wave_status wave_schedule_verify(const int grid[3], int so, const wave_tiling* tiling)
{
    if (!grid || !tiling) return wave::fail(WAVE_ERR_ARG, "wave_schedule_verify: null argument");
    std::string why;
    if (!wave::verify_schedule(grid, so / 2, *tiling, so / 2, so / 2, &why)) return wave::fail(WAVE_ERR_ARG, why);
    return WAVE_OK;
}

extern "C" wave_status wave_schedule_verify_custom(const int grid[3], int so, const wave_tiling* tiling, int lag,
                                                   int halo_per_step)
{
    if (!grid || !tiling) return wave::fail(WAVE_ERR_ARG, "wave_schedule_verify_custom: null argument");
    std::string why;
    if (!wave::verify_schedule(grid, so / 2, *tiling, lag, halo_per_step, &why))
        return wave::fail(WAVE_ERR_ARG, why);
    return WAVE_OK;
}

extern "C" wave_status wave_schedule_verify_skew(const int grid[3], int so, const wave_tiling* tiling,
                                                 int exchange_rows, int wait_lead)
{
    if (!grid || !tiling) return wave::fail(WAVE_ERR_ARG, "wave_schedule_verify_skew: null argument");
    std::string why;
    if (!wave::verify_skew_schedule(grid, so / 2, *tiling, exchange_rows, wait_lead, &why))
        return wave::fail(WAVE_ERR_ARG, why);
    return WAVE_OK;
}

extern "C" int wave_skewed_order_legal(int n, int nt, int r, int skew, int tt, int ts)
{
    return wave::skewed_order_legal(n, nt, r, skew, tt, ts) ? 1 : 0;
}
