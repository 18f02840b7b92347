/*
 * oracle.c -- plain FP64 reference for the 3D acoustic wave path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py (plus `bench.py --impl reference`) may load liboracle.so.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (McCormick 2017, "Applying the Polyhedral Model to Tile
 * Loops in Devito"):
 *   - Section "Acoustic wave equation", Fig. acoustic_devito: the untiled
 *     damped update of the 3D acoustic wave equation m u_tt + d u_t = Lap u + q
 *     stepped with second-order leapfrog,
 *        u[t+1] = ((dt*d - 2m) u[t-1] + 4m u[t] + 2dt^2 (L_h u[t] + q)) / (dt*d + 2m)
 *     where the printed coefficients are the centred second-derivative FD
 *     weights of space order SO times 2dt^2/h^2 (SO = 8 in the figure, with
 *     tcse0 = dt*damp, dt = 3.04).
 *   - Section "Simulation", Figs. acoustic_devito / tiled_256: the stencil
 *     reads u[time] at offsets +-1..+-SO/2 along each axis and u[time-1] at
 *     the centre; the loops run over the interior, the ghost layer of width
 *     SO/2 is never written (zero Dirichlet).
 *   - The source term that the paper removes before tiling (Section
 *     "Functional Correctness") is kept here as a term q of the same discrete
 *     equation, injected through trilinear taps; receivers sample u with the
 *     same trilinear taps after every update.
 *
 * The loop nest below is the definition written out: no blocking, no fusion,
 * no reordering.  The only concession to speed is an OpenMP "parallel for"
 * on the outermost space loop, which does not change any result (every
 * point is computed independently from the previous two levels).
 *
 * Readings where the paper is silent (the same readings the library takes):
 *   - the damping profile d: a sponge of `sponge_width` cells on the faces in
 *     `sponge_faces`, d = dmax_a ((W - delta)/W)^2 for a point delta < W cells
 *     from a face on axis a, summed over faces and axes, with
 *     dmax_a = 3 vmax ln(1000) / (2 W h_a);
 *   - q enters as a point source through trilinear weights w of the source
 *     position (no 1/h^3 factor), i.e. L_h u -> L_h u + sum_s w_s q_s;
 *   - receivers: rec[n][j] = trilinear interpolation of u^{n+1} (the field
 *     produced by update n); update n injects wavelet row n.
 *
 * Parity: every function here is pinned by tests/test_oracle_*.py (printed
 * SO8 coefficients, exactness on polynomials, periodic dispersion relation,
 * leapfrog energy, dense-matrix brute force, reciprocity, central finite
 * differences and the dot-product test for the adjoint and gradient).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EARG 1
#define OR_ENOMEM 2

/* ------------------------------------------------------------------------ */
/* FD weights: Fornberg's 1988 recursion ("Generation of finite difference   */
/* formulas on arbitrarily spaced grids", Math. Comp. 51).  Weights of the   */
/* derivatives 0..mmax at x0 on the nodes x[0..n-1].                         */
/* c is [n][mmax+1], row-major.                                              */
/* ------------------------------------------------------------------------ */
static void fornberg(int n, const double* x, double x0, int mmax, double* c)
{
    int M = mmax + 1;
    memset(c, 0, sizeof(double) * (size_t)n * (size_t)M);
    double c1 = 1.0;
    double c4 = x[0] - x0;
    c[0] = 1.0;
    for (int i = 1; i < n; ++i) {
        int mn = i < mmax ? i : mmax;
        double c2 = 1.0;
        double c5 = c4;
        c4 = x[i] - x0;
        for (int j = 0; j < i; ++j) {
            double c3 = x[i] - x[j];
            c2 *= c3;
            if (j == i - 1) {
                for (int k = mn; k >= 1; --k)
                    c[i * M + k] = c1 * (k * c[(i - 1) * M + k - 1] - c5 * c[(i - 1) * M + k]) / c2;
                c[i * M + 0] = -c1 * c5 * c[(i - 1) * M + 0] / c2;
            }
            for (int k = mn; k >= 1; --k)
                c[j * M + k] = (c4 * c[j * M + k] - k * c[j * M + k - 1]) / c3;
            c[j * M + 0] = c4 * c[j * M + 0] / c3;
        }
        c1 = c2;
    }
}

/* Centred second-derivative weights of accuracy order `so` on unit spacing:
 * a[0] is the centre weight, a[k] (k = 1..so/2) the weight of the points at
 * +-k.  Fig. acoustic_devito prints these for so = 8 multiplied by 2dt^2/h^2. */
int oracle_fd_weights(int so, double* a)
{
    if (so < 2 || so > 32 || (so & 1)) return OR_EARG;
    int r = so / 2, n = 2 * r + 1;
    double* x = (double*)malloc(sizeof(double) * n);
    double* c = (double*)malloc(sizeof(double) * n * 3);
    if (!x || !c) { free(x); free(c); return OR_ENOMEM; }
    for (int j = 0; j < n; ++j) x[j] = (double)(j - r);
    fornberg(n, x, 0.0, 2, c);
    for (int k = 0; k <= r; ++k) a[k] = c[(r + k) * 3 + 2];
    free(x);
    free(c);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Problem description shared by the entry points below.                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;       /* extents of the grid (or of a window of it)        */
    int ox, oy, oz;       /* global index of the window's first point          */
    int gnx, gny, gnz;    /* extents of the global grid (sponge faces)          */
    double hx, hy, hz;    /* spacing in metres                                  */
    int so;               /* space order                                        */
    double dt;            /* time step in ms                                    */
    int nt;               /* number of updates                                  */
    int boundary;         /* 0: zero ghosts outside the box, 1: periodic        */
    int sponge_width;     /* W in cells, 0 = no damping                         */
    int sponge_faces;     /* bit f set = face f absorbs: x-,x+,y-,y+,z-,z+      */
    double vmax;          /* km/s, sets dmax                                    */
    const double* m;      /* [nx][ny][nz] squared slowness                      */
    int nsrc;
    const double* src_xyz;   /* [nsrc][3] metres, global frame                  */
    const double* wavelet;   /* [nt][nsrc]                                      */
    int nrec;
    const double* rec_xyz;   /* [nrec][3] metres, global frame                  */
} oracle_problem;

#define IDX(p, i, j, k) (((size_t)(i) * (size_t)(p)->ny + (size_t)(j)) * (size_t)(p)->nz + (size_t)(k))

/* Sponge profile of one axis at global index g of n points. */
static double sponge_axis(int g, int n, int W, int lo_on, int hi_on, double dmax)
{
    double d = 0.0;
    if (W <= 0) return 0.0;
    if (lo_on && g < W) {
        double s = (double)(W - g) / (double)W;
        d += dmax * s * s;
    }
    int dh = n - 1 - g;
    if (hi_on && dh < W) {
        double s = (double)(W - dh) / (double)W;
        d += dmax * s * s;
    }
    return d;
}

/* Damping d at every point of the box (1/ms). */
int oracle_damping(const oracle_problem* p, double* d)
{
    int W = p->sponge_width;
    double lnr = log(1000.0);
    double dmx = W > 0 ? 3.0 * p->vmax * lnr / (2.0 * W * p->hx) : 0.0;
    double dmy = W > 0 ? 3.0 * p->vmax * lnr / (2.0 * W * p->hy) : 0.0;
    double dmz = W > 0 ? 3.0 * p->vmax * lnr / (2.0 * W * p->hz) : 0.0;
    int f = p->sponge_faces;
    for (int i = 0; i < p->nx; ++i)
        for (int j = 0; j < p->ny; ++j)
            for (int k = 0; k < p->nz; ++k) {
                double dx = sponge_axis(i + p->ox, p->gnx, W, f & 1, f & 2, dmx);
                double dy = sponge_axis(j + p->oy, p->gny, W, f & 4, f & 8, dmy);
                double dz = sponge_axis(k + p->oz, p->gnz, W, f & 16, f & 32, dmz);
                d[IDX(p, i, j, k)] = dx + dy + dz;
            }
    return OR_OK;
}

/* Value of u at (i, j, k), with the box's boundary rule. */
static double at(const oracle_problem* p, const double* u, int i, int j, int k)
{
    if (p->boundary == 1) {
        i = ((i % p->nx) + p->nx) % p->nx;
        j = ((j % p->ny) + p->ny) % p->ny;
        k = ((k % p->nz) + p->nz) % p->nz;
        return u[IDX(p, i, j, k)];
    }
    if (i < 0 || i >= p->nx || j < 0 || j >= p->ny || k < 0 || k >= p->nz) return 0.0;
    return u[IDX(p, i, j, k)];
}

/* L_h u at one point: sum over axes of (a0 u + sum_k a_k (u(+k) + u(-k))) / h^2. */
static double lap_point(const oracle_problem* p, const double* a, const double* u, int i, int j, int k)
{
    int r = p->so / 2;
    double c = at(p, u, i, j, k);
    double lx = a[0] * c, ly = a[0] * c, lz = a[0] * c;
    for (int q = 1; q <= r; ++q) {
        lx += a[q] * (at(p, u, i + q, j, k) + at(p, u, i - q, j, k));
        ly += a[q] * (at(p, u, i, j + q, k) + at(p, u, i, j - q, k));
        lz += a[q] * (at(p, u, i, j, k + q) + at(p, u, i, j, k - q));
    }
    return lx / (p->hx * p->hx) + ly / (p->hy * p->hy) + lz / (p->hz * p->hz);
}

int oracle_laplacian(const oracle_problem* p, const double* u, double* out)
{
    double a[17];
    int rc = oracle_fd_weights(p->so, a);
    if (rc) return rc;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < p->nx; ++i)
        for (int j = 0; j < p->ny; ++j)
            for (int k = 0; k < p->nz; ++k)
                out[IDX(p, i, j, k)] = lap_point(p, a, u, i, j, k);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Trilinear taps of a position (global metres) inside the box.              */
/* Corner c = 4*dx + 2*dy + dz of the cell whose low corner is floor(pos/h). */
/* Corners with zero weight or outside the box are dropped.                  */
/* ------------------------------------------------------------------------ */
typedef struct { size_t idx; double w; } tap;

static int trilinear(const oracle_problem* p, const double* xyz, tap* t)
{
    double g[3] = { xyz[0] / p->hx, xyz[1] / p->hy, xyz[2] / p->hz };
    int o[3] = { p->ox, p->oy, p->oz };
    int n[3] = { p->nx, p->ny, p->nz };
    int i0[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(g[a]);
        i0[a] = (int)fl;
        fr[a] = g[a] - fl;
    }
    int cnt = 0;
    for (int c = 0; c < 8; ++c) {
        int d[3] = { (c >> 2) & 1, (c >> 1) & 1, c & 1 };
        double w = 1.0;
        int li[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            w *= d[a] ? fr[a] : 1.0 - fr[a];
            li[a] = i0[a] + d[a] - o[a];
            if (li[a] < 0 || li[a] >= n[a]) inside = 0;
        }
        if (w == 0.0 || !inside) continue;
        t[cnt].idx = IDX(p, li[0], li[1], li[2]);
        t[cnt].w = w;
        ++cnt;
    }
    return cnt;
}

static int check_problem(const oracle_problem* p)
{
    if (!p || p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return OR_EARG;
    if (p->so < 2 || p->so > 32 || (p->so & 1)) return OR_EARG;
    if (p->nt < 0 || !(p->dt > 0.0) || !p->m) return OR_EARG;
    if (p->nsrc > 0 && (!p->src_xyz || !p->wavelet)) return OR_EARG;
    if (p->nrec > 0 && !p->rec_xyz) return OR_EARG;
    return OR_OK;
}

/* One leapfrog update of the whole box:
 *   next = ((dt d - 2m) prev + 4m cur + 2dt^2 (L_h cur + q)) / (dt d + 2m)
 * with q a dense array holding the injected source term of this update. */
static void leapfrog(const oracle_problem* p, const double* a, const double* dmp, const double* q,
                     const double* prev, const double* cur, double* next)
{
    double dt = p->dt;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < p->nx; ++i)
        for (int j = 0; j < p->ny; ++j)
            for (int k = 0; k < p->nz; ++k) {
                size_t s = IDX(p, i, j, k);
                double m = p->m[s], d = dmp[s];
                double lap = lap_point(p, a, cur, i, j, k);
                double num = (dt * d - 2.0 * m) * prev[s] + 4.0 * m * cur[s] + 2.0 * dt * dt * (lap + q[s]);
                next[s] = num / (dt * d + 2.0 * m);
            }
}

typedef struct {
    size_t n;
    double a[17];
    double *dmp, *q;
    tap* stap;  /* [nsrc][8] */
    int* scnt;
    tap* rtap;  /* [nrec][8] */
    int* rcnt;
} oracle_ws;

static void ws_free(oracle_ws* w)
{
    free(w->dmp); free(w->q); free(w->stap); free(w->scnt); free(w->rtap); free(w->rcnt);
}

static int ws_init(const oracle_problem* p, oracle_ws* w)
{
    memset(w, 0, sizeof(*w));
    w->n = (size_t)p->nx * p->ny * p->nz;
    int rc = oracle_fd_weights(p->so, w->a);
    if (rc) return rc;
    w->dmp = (double*)malloc(sizeof(double) * w->n);
    w->q = (double*)calloc(w->n, sizeof(double));
    w->stap = (tap*)malloc(sizeof(tap) * 8 * (size_t)(p->nsrc > 0 ? p->nsrc : 1));
    w->scnt = (int*)malloc(sizeof(int) * (size_t)(p->nsrc > 0 ? p->nsrc : 1));
    w->rtap = (tap*)malloc(sizeof(tap) * 8 * (size_t)(p->nrec > 0 ? p->nrec : 1));
    w->rcnt = (int*)malloc(sizeof(int) * (size_t)(p->nrec > 0 ? p->nrec : 1));
    if (!w->dmp || !w->q || !w->stap || !w->scnt || !w->rtap || !w->rcnt) { ws_free(w); return OR_ENOMEM; }
    oracle_damping(p, w->dmp);
    for (int s = 0; s < p->nsrc; ++s) w->scnt[s] = trilinear(p, p->src_xyz + 3 * s, w->stap + 8 * s);
    for (int r = 0; r < p->nrec; ++r) w->rcnt[r] = trilinear(p, p->rec_xyz + 3 * r, w->rtap + 8 * r);
    return OR_OK;
}

/* Dense source term of update n: q[p] = sum_s sum_taps w * wavelet[n][s]. */
static void set_sources(const oracle_problem* p, oracle_ws* w, int n, double sign)
{
    for (int s = 0; s < p->nsrc; ++s)
        for (int c = 0; c < w->scnt[s]; ++c)
            w->q[w->stap[8 * s + c].idx] += sign * w->stap[8 * s + c].w * p->wavelet[(size_t)n * p->nsrc + s];
}

static void clear_sources(const oracle_problem* p, oracle_ws* w)
{
    for (int s = 0; s < p->nsrc; ++s)
        for (int c = 0; c < w->scnt[s]; ++c) w->q[w->stap[8 * s + c].idx] = 0.0;
}

static double sample(const tap* t, int cnt, const double* u)
{
    double v = 0.0;
    for (int c = 0; c < cnt; ++c) v += t[c].w * u[t[c].idx];
    return v;
}

/* Forward modelling.
 * u_prev0 / u_cur0: u^{-1}, u^0 (NULL = zero).  rec: [nt][nrec] (may be NULL).
 * u_prev_out / u_cur_out: u^{nt-1}, u^{nt} (may be NULL). */
int oracle_forward(const oracle_problem* p, const double* u_prev0, const double* u_cur0,
                   double* rec, double* u_prev_out, double* u_cur_out)
{
    int rc = check_problem(p);
    if (rc) return rc;
    oracle_ws w;
    rc = ws_init(p, &w);
    if (rc) return rc;
    double* b0 = (double*)calloc(w.n, sizeof(double));
    double* b1 = (double*)calloc(w.n, sizeof(double));
    double* b2 = (double*)calloc(w.n, sizeof(double));
    if (!b0 || !b1 || !b2) { free(b0); free(b1); free(b2); ws_free(&w); return OR_ENOMEM; }
    if (u_prev0) memcpy(b0, u_prev0, sizeof(double) * w.n);
    if (u_cur0) memcpy(b1, u_cur0, sizeof(double) * w.n);
    double *prev = b0, *cur = b1, *next = b2;
    for (int n = 0; n < p->nt; ++n) {
        set_sources(p, &w, n, 1.0);
        leapfrog(p, w.a, w.dmp, w.q, prev, cur, next);
        clear_sources(p, &w);
        if (rec)
            for (int r = 0; r < p->nrec; ++r) rec[(size_t)n * p->nrec + r] = sample(w.rtap + 8 * r, w.rcnt[r], next);
        double* t = prev; prev = cur; cur = next; next = t;
    }
    if (u_prev_out) memcpy(u_prev_out, prev, sizeof(double) * w.n);
    if (u_cur_out) memcpy(u_cur_out, cur, sizeof(double) * w.n);
    free(b0); free(b1); free(b2);
    ws_free(&w);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjoint and gradient (extensions of the forward path; the paper's         */
/* equation written as F_n(u) = A+ u^{n+1} - (2m/dt^2 + L_h) u^n             */
/*                               + A- u^{n-1} - S q^n = 0,                    */
/* A+- = m/dt^2 +- d/(2dt), which is the printed update divided by 2dt^2).   */
/*                                                                          */
/* The adjoint field mu solves the transposed recurrence backwards in time,  */
/*   A+ mu^j = (2m/dt^2 + L_h) mu^{j+1} - A- mu^{j+2} + R^T r^{j-1},          */
/* mu^{N+1} = mu^{N+2} = 0, which is the same update with the receiver taps  */
/* acting as sources of the time-reversed r (L_h is symmetric, A+- diagonal). */
/* ------------------------------------------------------------------------ */

/* Adjoint modelling: resid [nt][nrec] is injected at the receiver taps,
 * out [nt][nsrc] receives (S^T mu^{n+1})_s, i.e. the adjoint of the map
 * wavelet -> rec computed by oracle_forward with zero initial fields. */
int oracle_adjoint(const oracle_problem* p, const double* resid, double* out)
{
    int rc = check_problem(p);
    if (rc) return rc;
    oracle_ws w;
    rc = ws_init(p, &w);
    if (rc) return rc;
    double* b0 = (double*)calloc(w.n, sizeof(double));
    double* b1 = (double*)calloc(w.n, sizeof(double));
    double* b2 = (double*)calloc(w.n, sizeof(double));
    if (!b0 || !b1 || !b2) { free(b0); free(b1); free(b2); ws_free(&w); return OR_ENOMEM; }
    /* later = mu^{j+2}, cur = mu^{j+1}, next = mu^j */
    double *later = b0, *cur = b1, *next = b2;
    for (int j = p->nt; j >= 1; --j) {
        for (int r = 0; r < p->nrec; ++r)
            for (int c = 0; c < w.rcnt[r]; ++c)
                w.q[w.rtap[8 * r + c].idx] += w.rtap[8 * r + c].w * resid[(size_t)(j - 1) * p->nrec + r];
        leapfrog(p, w.a, w.dmp, w.q, later, cur, next);
        for (int r = 0; r < p->nrec; ++r)
            for (int c = 0; c < w.rcnt[r]; ++c) w.q[w.rtap[8 * r + c].idx] = 0.0;
        if (out)
            for (int s = 0; s < p->nsrc; ++s) out[(size_t)(j - 1) * p->nsrc + s] = sample(w.stap + 8 * s, w.scnt[s], next);
        double* t = later; later = cur; cur = next; next = t;
    }
    free(b0); free(b1); free(b2);
    ws_free(&w);
    return OR_OK;
}

/* Misfit J = 1/2 sum (rec - d_obs)^2 and its gradient with respect to m:
 *   dJ/dm = - sum_{n=0}^{nt-1} mu^{n+1} (u^{n+1} - 2u^n + u^{n-1}) / dt^2,
 * with mu the adjoint field driven by r = rec - d_obs.  Zero initial fields.
 * All nt+2 levels of u are kept (small grids only). */
int oracle_gradient(const oracle_problem* p, const double* d_obs, double* grad, double* misfit)
{
    int rc = check_problem(p);
    if (rc) return rc;
    oracle_ws w;
    rc = ws_init(p, &w);
    if (rc) return rc;
    size_t n = w.n;
    int nt = p->nt;
    /* levels[l] = u^{l-1}, l = 0..nt+1 */
    double* lev = (double*)calloc(n * (size_t)(nt + 2), sizeof(double));
    double* rres = (double*)malloc(sizeof(double) * (size_t)(nt > 0 ? nt : 1) * (size_t)(p->nrec > 0 ? p->nrec : 1));
    double* b0 = (double*)calloc(n, sizeof(double));
    double* b1 = (double*)calloc(n, sizeof(double));
    double* b2 = (double*)calloc(n, sizeof(double));
    if (!lev || !rres || !b0 || !b1 || !b2) {
        free(lev); free(rres); free(b0); free(b1); free(b2); ws_free(&w);
        return OR_ENOMEM;
    }
    double J = 0.0;
    for (int t = 0; t < nt; ++t) {
        set_sources(p, &w, t, 1.0);
        leapfrog(p, w.a, w.dmp, w.q, lev + n * (size_t)t, lev + n * (size_t)(t + 1), lev + n * (size_t)(t + 2));
        clear_sources(p, &w);
        for (int r = 0; r < p->nrec; ++r) {
            double v = sample(w.rtap + 8 * r, w.rcnt[r], lev + n * (size_t)(t + 2));
            double e = v - d_obs[(size_t)t * p->nrec + r];
            rres[(size_t)t * p->nrec + r] = e;
            J += 0.5 * e * e;
        }
    }
    memset(grad, 0, sizeof(double) * n);
    double *later = b0, *cur = b1, *next = b2;
    double idt2 = 1.0 / (p->dt * p->dt);
    for (int j = nt; j >= 1; --j) {
        for (int r = 0; r < p->nrec; ++r)
            for (int c = 0; c < w.rcnt[r]; ++c)
                w.q[w.rtap[8 * r + c].idx] += w.rtap[8 * r + c].w * rres[(size_t)(j - 1) * p->nrec + r];
        leapfrog(p, w.a, w.dmp, w.q, later, cur, next);
        for (int r = 0; r < p->nrec; ++r)
            for (int c = 0; c < w.rcnt[r]; ++c) w.q[w.rtap[8 * r + c].idx] = 0.0;
        /* next = mu^j pairs with equation n = j-1: D_tt u^{j-1} = (u^j - 2u^{j-1} + u^{j-2}) / dt^2 */
        const double* up = lev + n * (size_t)(j + 1);   /* u^j     */
        const double* uc = lev + n * (size_t)j;         /* u^{j-1} */
        const double* um = lev + n * (size_t)(j - 1);   /* u^{j-2} */
        for (size_t s = 0; s < n; ++s) grad[s] -= next[s] * (up[s] - 2.0 * uc[s] + um[s]) * idt2;
        double* t = later; later = cur; cur = next; next = t;
    }
    if (misfit) *misfit = J;
    free(lev); free(rres); free(b0); free(b1); free(b2);
    ws_free(&w);
    return OR_OK;
}
