"""Pins of the FP64 oracle against facts other than itself.

Each test checks the oracle against what the paper prints or what the
mathematics fixes, chosen so that a dropped term, a wrong sign, a wrong index
or a transposed operand in oracle.c fails at least one of them:

* printed SO8 coefficients (Fig. acoustic_devito / Fig. tiled_256);
* closed-form weights vs the oracle's Fornberg recursion, and exactness on
  monomials up to degree SO + 1;
* L_h exact on polynomials of degree <= SO (interior points);
* the discrete dispersion relation of a periodic standing wave;
* conservation of the discrete leapfrog energy with zero ghosts;
* a dense-matrix brute force of the printed damped update on tiny grids;
* the sponge profile's closed form at chosen cells;
* source/receiver reciprocity;
* finite speed of propagation (window == full grid inside the cone);
* dot-product test of the adjoint and central finite differences of the
  gradient.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "so8_printed_coefficients.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _closed_form(so):
    r = so // 2
    ak = [Fraction(2 * (-1) ** (k + 1) * math.factorial(r) ** 2,
                   k * k * math.factorial(r - k) * math.factorial(r + k)) for k in range(1, r + 1)]
    return [-2 * sum(ak)] + ak


# ---------------------------------------------------------------------------
# FD weights
# ---------------------------------------------------------------------------

def test_so8_weights_reproduce_printed_coefficients(oracle):
    g = _golden()
    a = oracle.fd_weights(8)
    scale = 2.0 * g["dt"] ** 2 / g["h"] ** 2
    assert scale == pytest.approx(0.046208, rel=1e-15)
    for k in range(1, 5):
        assert a[k] * scale == pytest.approx(g["k%d" % k], rel=1e-12, abs=0)
    # three axes' centre weights
    assert 3 * a[0] * scale == pytest.approx(g["centre"], rel=1e-12, abs=0)


@pytest.mark.parametrize("so", [2, 4, 6, 8, 12, 16])
def test_weights_match_closed_form(oracle, so):
    a = oracle.fd_weights(so)
    exact = _closed_form(so)
    for k, e in enumerate(exact):
        assert a[k] == pytest.approx(float(e), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("so", [4, 8, 16])
def test_weights_exact_on_monomials(oracle, so):
    r = so // 2
    a = oracle.fd_weights(so)
    for j in range(0, so + 2):
        # second derivative of x^j at 0 is 2 for j == 2, else 0
        s = a[0] * (1.0 if j == 0 else 0.0) + sum(a[k] * (k ** j + (-k) ** j) for k in range(1, r + 1))
        want = 2.0 if j == 2 else 0.0
        assert s == pytest.approx(want, abs=1e-9 * max(1.0, float(r) ** j)), (so, j, s)
    # and not on x^(so+2): the truncation term is non-zero (order is exactly so)
    j = so + 2
    s = sum(a[k] * (k ** j + (-k) ** j) for k in range(1, r + 1))
    assert abs(s) > 1e-6


# ---------------------------------------------------------------------------
# Spatial operator
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("so", [4, 8])
def test_laplacian_exact_on_polynomials(oracle, so):
    r = so // 2
    n = (2 * r + 6, 2 * r + 5, 2 * r + 7)
    h = (7.0, 5.0, 3.0)
    x = np.arange(n[0])[:, None, None] * h[0]
    y = np.arange(n[1])[None, :, None] * h[1]
    z = np.arange(n[2])[None, None, :] * h[2]
    # centre the coordinates so the monomials stay well scaled
    xc, yc, zc = x - x.mean(), y - y.mean(), z - z.mean()
    rng = np.random.default_rng(0)
    cx, cy, cz = rng.standard_normal(so + 1), rng.standard_normal(so + 1), rng.standard_normal(3)
    u = (sum(cx[j] * (xc / 10) ** j for j in range(so + 1))
         + sum(cy[j] * (yc / 10) ** j for j in range(so + 1))
         + cz[0] * (xc / 10) * (yc / 10) * (zc / 10) + cz[1] * (xc / 10) ** 2 * (zc / 10) ** 2)
    u = np.broadcast_to(u, n).copy()
    d2x = sum(cx[j] * j * (j - 1) * (xc / 10) ** (j - 2) / 100 for j in range(2, so + 1))
    d2y = sum(cy[j] * j * (j - 1) * (yc / 10) ** (j - 2) / 100 for j in range(2, so + 1))
    lap = d2x + d2y + cz[1] * (2 * (zc / 10) ** 2 / 100 + 2 * (xc / 10) ** 2 / 100)
    lap = np.broadcast_to(lap, n)
    got = oracle.laplacian(u, h, so)
    inner = (slice(r, n[0] - r), slice(r, n[1] - r), slice(r, n[2] - r))
    np.testing.assert_allclose(got[inner], lap[inner], rtol=1e-9, atol=1e-9 * np.abs(lap).max())
    # at the boundary the zero ghosts make it inexact (the ghost ring is real)
    assert np.abs(got[0] - lap[0]).max() > 1e-6


# ---------------------------------------------------------------------------
# Time stepping
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("so", [4, 8])
def test_periodic_standing_wave_dispersion(oracle, so):
    n = (12, 10, 8)
    h = (10.0, 12.0, 9.0)
    v = 2.0
    modes = (1, 2, 3)
    a = [float(f) for f in _closed_form(so)]
    lam = 0.0
    for ax in range(3):
        th = 2 * math.pi * modes[ax] / n[ax]
        lam -= (a[0] + 2 * sum(a[k] * math.cos(k * th) for k in range(1, so // 2 + 1))) / h[ax] ** 2
    rho = abs(a[0]) + 2 * sum(abs(x) for x in a[1:])
    dt = 0.8 * 2.0 / (v * math.sqrt(sum(rho / hh ** 2 for hh in h)))
    cwdt = 1.0 - 0.5 * dt * dt * v * v * lam  # cos(omega dt)
    wdt = math.acos(cwdt)
    i, j, k = np.meshgrid(*[np.arange(s) for s in n], indexing="ij")
    u0 = (np.cos(2 * math.pi * modes[0] * i / n[0]) * np.cos(2 * math.pi * modes[1] * j / n[1])
          * np.cos(2 * math.pi * modes[2] * k / n[2]))
    um1 = math.cos(wdt) * u0
    m = np.full(n, 1.0 / v ** 2)
    nt = 60
    _, up, uc = oracle.forward(n, h, so, dt, nt, m, u_prev0=um1, u_cur0=u0, periodic=True)
    np.testing.assert_allclose(uc, math.cos(nt * wdt) * u0, atol=1e-11)
    np.testing.assert_allclose(up, math.cos((nt - 1) * wdt) * u0, atol=1e-11)


def test_leapfrog_energy_conserved(oracle):
    n, h, so = (14, 12, 10), (10.0, 10.0, 10.0), 8
    rng = np.random.default_rng(1)
    v = 1.5 + rng.random(n)
    m = 1.0 / v ** 2
    dt = 0.9 * 2.0 / (v.max() * math.sqrt(3 * (2048 / 315) / 100.0))
    um = rng.standard_normal(n)
    uc = um + 0.1 * rng.standard_normal(n)

    def energy(a, b):  # E^{n+1/2} with a = u^n, b = u^{n+1}
        return float(np.sum(m * ((b - a) / dt) ** 2) - np.sum(b * oracle.laplacian(a, h, so)))

    e0 = energy(um, uc)
    es = []
    for _ in range(10):
        _, um, uc = oracle.forward(n, h, so, dt, 20, m, u_prev0=um, u_cur0=uc)
        es.append(energy(um, uc))
    assert max(abs(e - e0) for e in es) <= 1e-11 * abs(e0)
    # a sanity check that energy is not trivially constant: damping must decrease it
    _, a2, b2 = oracle.forward(n, h, so, dt, 200, m, u_prev0=um, u_cur0=uc, sponge_width=3,
                               sponge_faces=0b111111, vmax=float(v.max()))
    assert energy(a2, b2) < 0.9 * e0


def _dense_laplacian(n, h, so, weights):
    mats = []
    r = so // 2
    for ax in range(3):
        D = np.zeros((n[ax], n[ax]))
        for i in range(n[ax]):
            D[i, i] = weights[0]
            for k in range(1, r + 1):
                if i + k < n[ax]:
                    D[i, i + k] = weights[k]
                if i - k >= 0:
                    D[i, i - k] = weights[k]
        mats.append(D / h[ax] ** 2)
    I = [np.eye(s) for s in n]
    return (np.kron(np.kron(mats[0], I[1]), I[2]) + np.kron(np.kron(I[0], mats[1]), I[2])
            + np.kron(np.kron(I[0], I[1]), mats[2]))


def _trilinear_dense(pos, n, h):
    """Independent trilinear weights of one position as a dense vector."""
    w = np.zeros(n)
    g = [pos[a] / h[a] for a in range(3)]
    i0 = [int(math.floor(x)) for x in g]
    fr = [g[a] - i0[a] for a in range(3)]
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                idx = (i0[0] + dx, i0[1] + dy, i0[2] + dz)
                if all(0 <= idx[a] < n[a] for a in range(3)):
                    w[idx] += ((fr[0] if dx else 1 - fr[0]) * (fr[1] if dy else 1 - fr[1])
                               * (fr[2] if dz else 1 - fr[2]))
    return w.ravel()


@pytest.mark.parametrize("so,n", [(4, (8, 8, 8)), (8, (9, 8, 10))])
def test_dense_bruteforce_matches_loop_nest(oracle, so, n):
    h = (10.0, 11.0, 12.0)
    rng = np.random.default_rng(2 + so)
    v = 1.5 + 1.5 * rng.random(n)
    m = 1.0 / v ** 2
    vmax = float(v.max())
    dt = 0.5 * 2.0 / (vmax * math.sqrt(sum(8.0 / hh ** 2 for hh in h)))
    nt = 12
    src = np.array([[3.3 * h[0], 4.0 * h[1], 2.5 * h[2]], [5.0 * h[0], 2.0 * h[1], 6.0 * h[2]]])
    wav = rng.standard_normal((nt, 2))
    rec = np.array([[2.2 * h[0], 5.7 * h[1], 3.1 * h[2]], [6.0 * h[0], 6.0 * h[1], 1.0 * h[2]],
                    [0.0, 0.0, 0.0]])
    um0 = 0.1 * rng.standard_normal(n)
    uc0 = 0.1 * rng.standard_normal(n)
    sponge = dict(sponge_width=3, sponge_faces=0b101111, vmax=vmax)
    rec_o, up_o, uc_o = oracle.forward(n, h, so, dt, nt, m, src_xyz=src, wavelet=wav, rec_xyz=rec,
                                       u_prev0=um0, u_cur0=uc0, **sponge)
    # brute force: the printed update with dense matrices, in long double
    weights = [float(f) for f in _closed_form(so)]
    A = _dense_laplacian(n, h, so, weights).astype(np.longdouble)
    d = oracle.damping(n, h, **sponge).ravel().astype(np.longdouble)
    mm = m.ravel().astype(np.longdouble)
    S = np.stack([_trilinear_dense(s, n, h) for s in src], axis=1).astype(np.longdouble)
    R = np.stack([_trilinear_dense(r, n, h) for r in rec], axis=0).astype(np.longdouble)
    prev = um0.ravel().astype(np.longdouble)
    cur = uc0.ravel().astype(np.longdouble)
    dtl = np.longdouble(dt)
    recs = []
    for t in range(nt):
        q = S @ wav[t].astype(np.longdouble)
        nxt = ((dtl * d - 2 * mm) * prev + 4 * mm * cur + 2 * dtl * dtl * (A @ cur + q)) / (dtl * d + 2 * mm)
        recs.append(R @ nxt)
        prev, cur = cur, nxt
    scale = float(np.abs(cur).max())
    np.testing.assert_allclose(uc_o.ravel(), cur.astype(np.float64), atol=1e-13 * scale, rtol=0)
    np.testing.assert_allclose(up_o.ravel(), prev.astype(np.float64), atol=1e-13 * scale, rtol=0)
    np.testing.assert_allclose(rec_o, np.array(recs, dtype=np.float64), atol=1e-13 * scale, rtol=0)


def test_sponge_profile_closed_form(oracle):
    n, h, W, vmax = (30, 26, 24), (10.0, 5.0, 20.0), 10, 3.0
    d = oracle.damping(n, h, sponge_width=W, sponge_faces=0b101111, vmax=vmax)
    dmax = [3 * vmax * math.log(1000.0) / (2 * W * hh) for hh in h]
    # centre-ish point away from every face: no damping
    assert d[15, 13, 12] == 0.0
    # on the x- face, mid y, deep z: dmax_x
    assert d[0, 13, 12] == pytest.approx(dmax[0], rel=1e-14)
    # 3 cells from the x+ face: ((W-3)/W)^2
    assert d[n[0] - 1 - 3, 13, 12] == pytest.approx(dmax[0] * (7 / 10) ** 2, rel=1e-14)
    # z = 0 is the free surface (face bit 4 off); z+ absorbs
    assert d[15, 13, 0] == 0.0
    assert d[15, 13, n[2] - 1] == pytest.approx(dmax[2], rel=1e-14)
    # W cells from a face: outside the sponge
    assert d[W, 13, 12] == 0.0
    # a corner sums the axes
    assert d[1, 2, n[2] - 1] == pytest.approx(dmax[0] * 0.81 + dmax[1] * 0.64 + dmax[2], rel=1e-14)


def test_source_receiver_reciprocity(oracle):
    n, h, so = (20, 18, 16), (10.0, 10.0, 10.0), 8
    rng = np.random.default_rng(5)
    v = 1.5 + rng.random(n)
    m = 1.0 / v ** 2
    vmax = float(v.max())
    dt = 0.8 * 2.0 / (vmax * math.sqrt(3 * (2048 / 315) / 100.0))
    nt = 80
    a = np.array([[52.5, 61.0, 47.3]])
    b = np.array([[121.0, 97.7, 88.8]])
    wav = rng.standard_normal((nt, 1))
    kw = dict(sponge_width=4, sponge_faces=0b111111, vmax=vmax)
    rab, _, _ = oracle.forward(n, h, so, dt, nt, m, src_xyz=a, wavelet=wav, rec_xyz=b, **kw)
    rba, _, _ = oracle.forward(n, h, so, dt, nt, m, src_xyz=b, wavelet=wav, rec_xyz=a, **kw)
    assert np.abs(rab).max() > 1e-8
    np.testing.assert_allclose(rab, rba, atol=1e-12 * np.abs(rab).max(), rtol=0)
    # linearity in the wavelet
    r2, _, _ = oracle.forward(n, h, so, dt, nt, m, src_xyz=a, wavelet=2.5 * wav, rec_xyz=b, **kw)
    np.testing.assert_allclose(r2, 2.5 * rab, atol=1e-13 * np.abs(rab).max(), rtol=0)


def test_on_grid_receiver_samples_the_point(oracle):
    n, h = (10, 10, 10), (10.0, 10.0, 10.0)
    rng = np.random.default_rng(6)
    um, uc = rng.standard_normal(n), rng.standard_normal(n)
    m = np.full(n, 0.4)
    rec, up, u1 = oracle.forward(n, h, 4, 1.0, 1, m, u_prev0=um, u_cur0=uc,
                                 rec_xyz=np.array([[30.0, 40.0, 50.0], [35.0, 40.0, 50.0]]))
    assert rec[0, 0] == u1[3, 4, 5]
    assert rec[0, 1] == pytest.approx(0.5 * (u1[3, 4, 5] + u1[4, 4, 5]), rel=1e-15)
    np.testing.assert_array_equal(up, uc)


def test_window_matches_full_grid_inside_cone(oracle):
    n, h, so = (40, 36, 32), (10.0, 10.0, 10.0), 8
    r = so // 2
    rng = np.random.default_rng(7)
    v = 1.5 + rng.random(n)
    m = 1.0 / v ** 2
    vmax = float(v.max())
    dt = 0.8 * 2.0 / (vmax * math.sqrt(3 * (2048 / 315) / 100.0))
    nt = 3
    src = np.array([[20 * h[0], 18 * h[1], 3 * h[2]]])
    wav = rng.standard_normal((nt, 1))
    um, uc = rng.standard_normal(n), rng.standard_normal(n)
    kw = dict(sponge_width=6, sponge_faces=0b101111, vmax=vmax)
    _, _, full = oracle.forward(n, h, so, dt, nt, m, src_xyz=src, wavelet=wav, u_prev0=um, u_cur0=uc, **kw)
    o = (10, 8, 0)
    s = (24, 22, 20)
    sl = tuple(slice(o[a], o[a] + s[a]) for a in range(3))
    _, _, win = oracle.forward(s, h, so, dt, nt, m[sl], src_xyz=src, wavelet=wav, u_prev0=um[sl], u_cur0=uc[sl],
                               origin=o, global_shape=n, **kw)
    c = r * nt
    # x and y window edges are interior cuts: exact only c cells inside; z starts at the real boundary
    inner = (slice(c, s[0] - c), slice(c, s[1] - c), slice(0, s[2] - c))
    np.testing.assert_array_equal(win[inner], full[sl][inner])
    assert np.abs(win[0] - full[sl][0]).max() > 0  # the cut is visible outside the cone


# ---------------------------------------------------------------------------
# Adjoint and gradient
# ---------------------------------------------------------------------------

def _small_problem(seed=8, n=(14, 13, 12), so=4, nt=40):
    h = (10.0, 10.0, 10.0)
    rng = np.random.default_rng(seed)
    v = 1.5 + rng.random(n)
    m = 1.0 / v ** 2
    vmax = float(v.max())
    dt = 0.8 * 2.0 / (vmax * math.sqrt(3 * (16 / 3) / 100.0)) if so == 4 else \
        0.8 * 2.0 / (vmax * math.sqrt(3 * (2048 / 315) / 100.0))
    src = np.array([[61.0, 55.5, 23.3], [30.0, 70.0, 50.0]])
    rec = np.array([[20.0, 30.0, 20.0], [90.0, 40.0, 20.0], [70.7, 91.2, 44.4]])
    kw = dict(sponge_width=3, sponge_faces=0b101111, vmax=vmax)
    return n, h, so, dt, nt, m, src, rec, kw, rng


def test_adjoint_dot_product(oracle):
    n, h, so, dt, nt, m, src, rec, kw, rng = _small_problem()
    q = rng.standard_normal((nt, 2))
    d = rng.standard_normal((nt, 3))
    Pq, _, _ = oracle.forward(n, h, so, dt, nt, m, src_xyz=src, wavelet=q, rec_xyz=rec, **kw)
    PTd = oracle.adjoint(n, h, so, dt, nt, m, src_xyz=src, rec_xyz=rec, resid=d, **kw)
    lhs = float(np.sum(Pq * d))
    rhs = float(np.sum(q * PTd))
    assert abs(lhs) > 1e-10
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gradient_central_differences(oracle):
    n, h, so, dt, nt, m, src, rec, kw, rng = _small_problem(nt=50)
    wav = rng.standard_normal((nt, 2))
    m_true = m * (1.0 + 0.05 * rng.standard_normal(n))
    d_obs, _, _ = oracle.forward(n, h, so, dt, nt, m_true, src_xyz=src, wavelet=wav, rec_xyz=rec, **kw)
    J, g = oracle.gradient(n, h, so, dt, nt, m, src_xyz=src, wavelet=wav, rec_xyz=rec, d_obs=d_obs, **kw)
    assert J > 0
    cells = [(3, 4, 2), (7, 6, 5), (10, 2, 9), (6, 9, 3)]
    for c in cells:
        eps = 1e-6 * m[c]
        mp, mn = m.copy(), m.copy()
        mp[c] += eps
        mn[c] -= eps
        rp, _, _ = oracle.forward(n, h, so, dt, nt, mp, src_xyz=src, wavelet=wav, rec_xyz=rec, **kw)
        rn, _, _ = oracle.forward(n, h, so, dt, nt, mn, src_xyz=src, wavelet=wav, rec_xyz=rec, **kw)
        fd = (0.5 * np.sum((rp - d_obs) ** 2) - 0.5 * np.sum((rn - d_obs) ** 2)) / (2 * eps)
        assert g[c] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(g).max()), c
