"""CPU tests of libwave.so's host side: the library loads and exports every
symbol include/wave.h declares, the FD-coefficient generator reproduces the
paper's printed SO8 coefficients, the CFL limit, and the tile-legality
scheduler (brute force on tiny grids).  No GPU is touched."""
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def W():
    import paper_1707_02347_gb300 as W

    W.load()
    return W


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(wave_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(W):
    lib = W.load()
    names = _declared()
    assert "wave_forward" in names and "wave_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_fd_weights_match_printed_so8_coefficients(W):
    vals = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "so8_printed_coefficients.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    a = W.fd_weights(8)
    s = 2 * vals["dt"] ** 2 / vals["h"] ** 2
    for k in range(1, 5):
        assert a[k] * s == pytest.approx(vals["k%d" % k], rel=1e-12)
    assert 3 * a[0] * s == pytest.approx(vals["centre"], rel=1e-12)


@pytest.mark.parametrize("so", [2, 4, 6, 8, 10, 12, 14, 16])
def test_fd_weights_are_exactness_conditions(W, so):
    # the weights solve the moment conditions sum_k a_k (k^{2j}) = delta_{j1}, j = 0..r,
    # which the test solves independently in exact arithmetic
    r = so // 2
    A = [[Fraction(1 if j == 0 else 0)] + [Fraction(2 * k ** (2 * j)) for k in range(1, r + 1)] for j in range(r + 1)]
    b = [Fraction(0), Fraction(2)] + [Fraction(0)] * (r - 1)
    # Gaussian elimination in fractions
    n = r + 1
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for c in range(n):
        p = next(i for i in range(c, n) if M[i][c] != 0)
        M[c], M[p] = M[p], M[c]
        for i in range(n):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [x - f * y for x, y in zip(M[i], M[c])]
    sol = [M[i][n] / M[i][i] for i in range(n)]
    got = W.fd_weights(so)
    for k in range(n):
        assert got[k] == float(sol[k]), (so, k, got[k], sol[k])


def test_cfl_limit(W):
    # SO4, h = 10 m, v = 1.5 km/s: rho = 16/3 -> dt_max = 2h / (v sqrt(3 rho)) = 20/6 ms
    assert W.cfl_limit(4, (10.0, 10.0, 10.0), 1.5) == pytest.approx(10.0 / 3.0, rel=1e-14)
    dt8 = W.cfl_limit(8, (10.0, 10.0, 10.0), 4.725)
    assert 0.9 * dt8 == pytest.approx(0.8625819, rel=1e-6)


def test_skew_factor(W):
    assert [W.skew_factor(s) for s in (4, 8, 16)] == [2, 4, 8]


@pytest.mark.parametrize("so,tiling", [
    (4, (1, 8, 8, 5)), (4, (2, 8, 8, 7)), (4, (3, 6, 8, 9)), (4, (4, 8, 12, 6)),
    (8, (1, 8, 8, 7)), (8, (2, 8, 8, 7)), (8, (2, 5, 12, 100)), (8, (3, 8, 8, 9)),
    (16, (1, 8, 8, 9)), (16, (2, 8, 8, 11)),
])
def test_pass_schedule_is_legal(W, so, tiling):
    grid = (19, 17, 15)
    ok, msg = W.schedule_verify(grid, so, tiling)
    assert ok, msg


@pytest.mark.parametrize("so,T", [(4, 2), (8, 2), (8, 3), (4, 4)])
def test_short_skew_or_halo_is_rejected(W, so, T):
    grid = (19, 17, 15)
    r = so // 2
    tiling = (T, 8, 8, 9)
    assert W.schedule_verify_custom(grid, so, tiling, r, r)[0]
    assert not W.schedule_verify_custom(grid, so, tiling, r - 1, r)[0]   # x skew too small
    assert not W.schedule_verify_custom(grid, so, tiling, r, r - 1)[0]   # overlapped halo too small


def test_paper_skewed_schedule_order(W):
    # Fig. tiled_256 reduced to one axis: time tile 8, space tile 16, skew 4, SO8
    assert W.skewed_order_legal(120, 24, 4, 4, 8, 16)
    # any smaller skew leaves a negative dependence distance and breaks the order
    for skew in range(0, 4):
        assert not W.skewed_order_legal(120, 24, 4, skew, 8, 16), skew
    # Fig. skew_snippet: radius 1 needs skew >= 1 (the paper skews by 2)
    assert W.skewed_order_legal(40, 12, 1, 2, 4, 3)
    assert W.skewed_order_legal(40, 12, 1, 1, 4, 3)
    assert not W.skewed_order_legal(40, 12, 1, 0, 4, 3)


@pytest.mark.parametrize("tiling,ok", [
    ((2, 16, 56, 128), True), ((2, 32, 32, 128), False), ((2, 64, 64, 128), False), ((2, 32, 30, 128), False),
    ((9, 32, 32, 64), False), ((1, 16, 64, 128), True), ((3, 16, 16, 128), True), ((3, 24, 24, 128), False),
])
def test_tiling_check_limits(W, tiling, ok):
    assert W.tiling_check((512, 512, 512), 8, tiling) == ok


@pytest.mark.parametrize("so,tiling,ok", [
    # skewed wavefront variant: T = 2 only; a tile is by = rows - r high (one
    # halo side instead of two), so 32 rows give by = 32 - r
    (8, (2, 28, 56, 128, 4), True), (8, (2, 60, 24, 128, 4), True), (4, (2, 30, 56, 128, 4), True),
    (8, (2, 24, 56, 128, 4), False),  # the overlapped shape's by: no compiled skewed kernel
    (8, (3, 24, 16, 128, 4), False),  # T = 3
    (16, (2, 24, 16, 128, 4), False),  # no radius-8 skewed kernel
])
def test_tiling_check_skewed_variant(W, so, tiling, ok):
    assert W.tiling_check((512, 512, 512), so, tiling) == ok


@pytest.mark.parametrize("so,tiling,ok", [
    # warp-specialised variants: 5 = one row per thread, 6 = two rows per thread
    # (a compute thread per 2 rows of a z quad); compiled for the listed shapes only
    (8, (2, 24, 56, 128, 5), True), (8, (2, 24, 56, 128, 6), False), (8, (1, 32, 64, 128, 5), False),
    (8, (1, 8, 64, 128, 5), True), (8, (1, 16, 64, 128, 5), True),
    (4, (2, 28, 56, 128, 5), True), (4, (3, 24, 56, 128, 5), True), (4, (2, 28, 56, 128, 6), False),
    (16, (1, 64, 32, 128, 6), True), (16, (1, 32, 64, 256, 6), True), (16, (1, 32, 64, 256, 5), False),
    # variant 7: two rows per thread, shift-register queues (11 compute warps: 44 thread rows)
    (8, (2, 36, 56, 128, 7), True), (4, (2, 40, 56, 128, 7), True), (4, (3, 36, 56, 128, 7), True),
    (8, (2, 24, 56, 128, 7), False), (16, (1, 64, 32, 128, 7), False),
])
def test_tiling_check_warp_specialised_variants(W, so, tiling, ok):
    assert W.tiling_check((512, 512, 512), so, tiling) == ok


@pytest.mark.parametrize("so,tiling", [(8, (2, 24, 56, 16, 5)), (4, (3, 24, 56, 9, 5)), (16, (1, 64, 32, 8, 6)),
                                       (8, (2, 36, 56, 16, 7)), (4, (3, 36, 56, 9, 7))])
def test_warp_specialised_schedule_is_legal(W, so, tiling):
    # same tiles and skew as the overlapped pass; only the synchronisation differs
    ok, msg = W.schedule_verify((40, 36, 44), so, tiling)
    assert ok, msg


@pytest.mark.parametrize("so,grid,tiling", [
    (8, (40, 90, 44), (2, 28, 56, 16, 4)),  # several y levels and z tiles, two slabs
    (8, (25, 130, 70), (2, 60, 24, 9, 4)),  # the other compiled shape, three slabs
    (4, (31, 95, 30), (2, 30, 56, 11, 4)),
    (8, (20, 17, 9), (2, 28, 56, 20, 4)),  # one y tile taller than the grid
])
def test_skewed_wavefront_schedule_is_legal(W, so, grid, tiling):
    """The skewed wavefront variant in the brute-force model: every step-2
    value reads either its own tile's step-1 values or the 2r rows tile j-1
    exchanged, published no later than the iteration that reads them."""
    ok, msg = W.schedule_verify(grid, so, tiling)
    assert ok, msg
    ok, msg = W.schedule_verify_skew(grid, so, tiling, so, 1)
    assert ok, msg


@pytest.mark.parametrize("so,grid,tiling", [(8, (40, 90, 44), (2, 28, 56, 16, 4)), (4, (31, 95, 30), (2, 30, 56, 11, 4))])
def test_skewed_wavefront_short_exchange_or_missing_wait_is_rejected(W, so, grid, tiling):
    r = so // 2
    # fewer than 2r exchanged rows: the lowest step-2 rows lack a y neighbour
    ok, why = W.schedule_verify_skew(grid, so, tiling, 2 * r - 1, 1)
    assert not ok and "invalid" in why
    # no progress wait: tile j would read a plane tile j-1 has not published yet
    ok, why = W.schedule_verify_skew(grid, so, tiling, 2 * r, 0)
    assert not ok and "invalid" in why
