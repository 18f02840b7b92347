// taps.cpp -- sparse source and receiver taps, sponge profile (host side).
//
// The paper injects its source and samples its 101 receivers in separate
// loops around the stencil (McCormick 2017, Section "Testing environment":
// loop_p_src and loop_p_rec) and removes the source before tiling because its
// sparse, non-uniform dependences do not fit the tiled loop (Section
// "Functional Correctness"; tiling the source and receiver loops is left as
// future work).  Here both are fused into every pass: each trilinear tap of a
// source or receiver is binned into the CSR list of its z-quad column, sorted
// by x, so the thread that owns the column meets it while it streams along x.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>

#include "wave_host.h"

namespace wave {

bool positions_valid(int count, const double* xyz, const double h[3], const int n[3], std::string* why)
{
    for (int p = 0; p < count; ++p)
        for (int a = 0; a < 3; ++a) {
            const double c = xyz[3 * p + a];
            if (!std::isfinite(c) || c < 0.0 || c > (n[a] - 1) * h[a]) {
                if (why)
                    *why = "position " + std::to_string(p) + " axis " + std::to_string(a) + " = " +
                           std::to_string(c) + " m is not finite or lies outside [0, (n-1) h] = [0, " +
                           std::to_string((n[a] - 1) * h[a]) + "]";
                return false;
            }
        }
    return true;
}

int trilinear_taps(const double xyz[3], const double h[3], const int n[3], Tap out[8])
{
    int i0[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        const double g = xyz[a] / h[a];
        const double fl = std::floor(g);
        i0[a] = static_cast<int>(fl);
        fr[a] = g - fl;
    }
    int cnt = 0;
    for (int c = 0; c < 8; ++c) {
        const int d[3] = {(c >> 2) & 1, (c >> 1) & 1, c & 1};
        double w = 1.0;
        bool inside = true;
        int idx[3];
        for (int a = 0; a < 3; ++a) {
            w *= d[a] ? fr[a] : 1.0 - fr[a];
            idx[a] = i0[a] + d[a];
            inside = inside && idx[a] >= 0 && idx[a] < n[a];
        }
        if (w == 0.0 || !inside) continue;
        out[cnt++] = {idx[0], idx[1], idx[2], w};
    }
    return cnt;
}

namespace {

struct SrcEnt {
    int col, x, lane, id;
    float w;
};

struct RecEnt {
    int col, x, lane, tap;
};

}  // namespace

void build_source_csr(int nsrc, const double* xyz, const double h[3], const int n[3], int nzp, ColumnCsr* out)
{
    const int ncols = n[1] * (nzp / 4);
    std::vector<SrcEnt> e;
    for (int s = 0; s < nsrc; ++s) {
        Tap t[8];
        const int c = trilinear_taps(xyz + 3 * s, h, n, t);
        for (int j = 0; j < c; ++j)
            e.push_back({t[j].j * (nzp / 4) + t[j].k / 4, t[j].i, t[j].k % 4, s, static_cast<float>(t[j].w)});
    }
    std::stable_sort(e.begin(), e.end(), [](const SrcEnt& a, const SrcEnt& b) {
        if (a.col != b.col) return a.col < b.col;
        if (a.x != b.x) return a.x < b.x;
        if (a.lane != b.lane) return a.lane < b.lane;
        return a.id < b.id;
    });
    out->ptr.assign(ncols + 1, 0);
    out->ent.resize(4 * e.size());
    for (size_t i = 0; i < e.size(); ++i) {
        out->ptr[e[i].col + 1]++;
        int wbits;
        std::memcpy(&wbits, &e[i].w, 4);
        out->ent[4 * i + 0] = e[i].x;
        out->ent[4 * i + 1] = e[i].lane;
        out->ent[4 * i + 2] = e[i].id;
        out->ent[4 * i + 3] = wbits;
    }
    for (int c = 0; c < ncols; ++c) out->ptr[c + 1] += out->ptr[c];
}

void build_receiver_csr(int nrec, const double* xyz, const double h[3], const int n[3], int nzp, ColumnCsr* out,
                        std::vector<int>* tptr, std::vector<float>* tw)
{
    const int ncols = n[1] * (nzp / 4);
    std::vector<RecEnt> e;
    tptr->assign(nrec + 1, 0);
    tw->clear();
    for (int r = 0; r < nrec; ++r) {
        Tap t[8];
        const int c = trilinear_taps(xyz + 3 * r, h, n, t);
        for (int j = 0; j < c; ++j) {
            const int tap = static_cast<int>(tw->size());
            tw->push_back(static_cast<float>(t[j].w));
            e.push_back({t[j].j * (nzp / 4) + t[j].k / 4, t[j].i, t[j].k % 4, tap});
        }
        (*tptr)[r + 1] = static_cast<int>(tw->size());
    }
    std::stable_sort(e.begin(), e.end(), [](const RecEnt& a, const RecEnt& b) {
        if (a.col != b.col) return a.col < b.col;
        if (a.x != b.x) return a.x < b.x;
        if (a.lane != b.lane) return a.lane < b.lane;
        return a.tap < b.tap;
    });
    out->ptr.assign(ncols + 1, 0);
    out->ent.resize(2 * e.size());
    for (size_t i = 0; i < e.size(); ++i) {
        out->ptr[e[i].col + 1]++;
        out->ent[2 * i + 0] = e[i].x;
        out->ent[2 * i + 1] = (e[i].tap << 2) | e[i].lane;
    }
    for (int c = 0; c < ncols; ++c) out->ptr[c + 1] += out->ptr[c];
}

// Gather plan of a dense receiver surface: when every tap of every receiver
// lies in at most two adjacent z quads (a surface or a line of receivers at
// one depth), each column quad holding taps has them on almost every plane,
// and recording them tap by tap inside the pass stalls every warp on the same
// planes; one-step passes gather the traces from the field after the pass
// instead.  idx[t] is the padded-layout index of tap t (receiver order, as
// tw).  False for fewer than min_rec receivers, taps in more than two quads,
// or a padded grid of 2^31 points or more.
bool receiver_gather_plan(int nrec, const double* xyz, const double h[3], const int n[3], int nzp, int min_rec,
                          std::vector<int>* idx)
{
    if (nrec < min_rec) return false;
    if (static_cast<long long>(n[0]) * n[1] * nzp >= 0x7fffffffLL) return false;
    int qlo = INT_MAX, qhi = -1;
    idx->clear();
    for (int r = 0; r < nrec; ++r) {
        Tap t[8];
        const int c = trilinear_taps(xyz + 3 * r, h, n, t);
        for (int j = 0; j < c; ++j) {
            idx->push_back((t[j].i * n[1] + t[j].j) * nzp + t[j].k);
            qlo = std::min(qlo, t[j].k / 4);
            qhi = std::max(qhi, t[j].k / 4);
        }
    }
    return !idx->empty() && qhi - qlo <= 1;
}

// Sponge (the paper's `damp` array, whose profile it does not give): for a
// point delta < W cells from an absorbing face, dmax ((W - delta) / W)^2,
// summed over the two faces of the axis; padded entries are zero.
void sponge_profile(int n, int width, bool lo, bool hi, double dmax, std::vector<float>* out, int padded_n)
{
    out->assign(std::max(n, padded_n), 0.f);
    if (width <= 0) return;
    for (int g = 0; g < n; ++g) {
        double d = 0.0;
        if (lo && g < width) {
            const double s = static_cast<double>(width - g) / width;
            d += dmax * s * s;
        }
        const int dh = n - 1 - g;
        if (hi && dh < width) {
            const double s = static_cast<double>(width - dh) / width;
            d += dmax * s * s;
        }
        (*out)[g] = static_cast<float>(d);
    }
}

}  // namespace wave
