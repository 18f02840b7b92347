"""GPU parity of the forward path (CUDA through the C ABI vs the FP64 oracle).

Bars (FP32 on the GPU, FP64 in the oracle):
* relative L2 error <= 1e-5 of the final field and of the traces after nt
  steps, on the same seeded inputs, and every element within 2e-5 of the
  oracle's largest magnitude (tests/parity.py);
* the time-tiled passes (T > 1) are bit-identical to the one-step kernel
  (T = 1) -- tiling only reorders independent updates;
* edge cases: ragged tiles in every axis, nz not a multiple of 4, minimum
  grids, nt = 0, nt not a multiple of T, several sources on one point,
  receivers on the grid boundary, no sources, paper's Gaussian initial field.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from parity import TOL, assert_close


def close(got, ref):
    """Relative L2 and per-element bound against the oracle, both <= TOL."""
    assert_close(got, ref, TOL)
    return True


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W

    W.load()
    return W


def run_gpu(W, w, tiling, u_init=None, want_final=True):
    dev = torch.device("cuda")
    m = torch.from_numpy(np.ascontiguousarray(w.m, dtype=np.float32)).to(dev)
    plan = W.WavePlan(w.shape, w.spacing, w.so, w.dt, w.nt, m, sponge_width=w.sponge_width,
                      sponge_faces=w.sponge_faces, vmax=w.vmax, tiling=tiling)
    if len(w.src_xyz):
        wav = torch.from_numpy(np.ascontiguousarray(w.wavelet, dtype=np.float32)).to(dev)
        plan.set_sources(w.src_xyz, wav)
    if len(w.rec_xyz):
        plan.set_receivers(w.rec_xyz)
    ui = None if u_init is None else torch.from_numpy(np.ascontiguousarray(u_init, dtype=np.float32)).to(dev)
    rec, uf = plan.forward(u_init=ui, want_final=want_final)
    torch.cuda.synchronize()
    out = (None if rec is None else rec.cpu().numpy(), None if uf is None else uf.cpu().numpy())
    plan.close()
    return out


def run_oracle(oracle, w, u_init=None):
    up0 = uc0 = None
    if u_init is not None:
        up0, uc0 = (np.asarray(u_init[0], np.float64), np.asarray(u_init[1], np.float64))
    return oracle.forward(w.shape, w.spacing, w.so, w.dt, w.nt, np.asarray(w.m, np.float64),
                          src_xyz=w.src_xyz if len(w.src_xyz) else None,
                          wavelet=w.wavelet if len(w.src_xyz) else None,
                          rec_xyz=w.rec_xyz if len(w.rec_xyz) else None, u_prev0=up0, u_cur0=uc0,
                          sponge_width=w.sponge_width, sponge_faces=w.sponge_faces, vmax=w.vmax)


def small_layered(shape, so, nt, seed, nrec=9, f=25.0, sponge=6):
    from paper_1707_02347_gb300 import inputs

    w = inputs.layered_forward(shape, so, nt, seed=seed, f=f, h=10.0, sponge_width=sponge, nrec_line=nrec)
    # an off-grid second source and a receiver on the far corner face
    w.src_xyz = np.vstack([w.src_xyz, [[(shape[0] / 3 + 0.37) * 10.0, (shape[1] / 2 - 0.81) * 10.0, 55.5]]])
    w.wavelet = np.stack([w.wavelet[:, 0], 0.7 * np.roll(w.wavelet[:, 0], 5)], axis=1)
    w.rec_xyz = np.vstack([w.rec_xyz, [[(shape[0] - 1) * 10.0, (shape[1] - 1) * 10.0, (shape[2] - 1) * 10.0]]])
    return w


def test_plain_forward_64_so4_vs_oracle(W, oracle):
    from paper_1707_02347_gb300 import inputs

    w = inputs.plain_forward_64(50)
    rec_o, up_o, uc_o = run_oracle(oracle, w)
    for tiling in [(1, 16, 64, 64), (2, 12, 56, 64), (4, 20, 16, 64)]:
        rec, uf = run_gpu(W, w, tiling)
        assert close(uf[1], uc_o), tiling
        assert close(uf[0], up_o), tiling
        assert close(rec, rec_o), tiling


@pytest.mark.parametrize("so,shape,tilings", [
    (4, (37, 34, 30), [(1, 16, 64, 11), (2, 28, 24, 9), (3, 24, 24, 40), (4, 12, 48, 13), (1, 16, 64, 37, 1),
                       (2, 12, 56, 30, 1), (3, 24, 24, 19, 1), (1, 16, 64, 37, 2), (2, 28, 56, 30, 2),
                       (3, 24, 56, 19, 2), (2, 20, 56, 20, 2), (4, 20, 16, 13, 2), (2, 30, 56, 30, 4),
                       (2, 28, 56, 13, 5), (3, 24, 56, 19, 5), (1, 8, 64, 37, 5), (1, 16, 64, 11, 5),
                       (2, 40, 56, 30, 7), (3, 36, 56, 19, 7), (3, 36, 56, 37, 7), (2, 36, 56, 30, 5),
                       (2, 40, 56, 13, 5)]),
    (8, (41, 35, 38), [(1, 32, 32, 40), (2, 24, 24, 10), (2, 16, 56, 41), (3, 16, 16, 17), (1, 32, 32, 41, 1),
                       (1, 16, 64, 23, 1), (2, 16, 56, 41, 1), (2, 24, 24, 29, 1), (3, 16, 16, 40, 1),
                       (1, 8, 64, 41, 2), (1, 16, 64, 23, 2), (2, 16, 56, 41, 2), (2, 24, 56, 29, 2),
                       (2, 56, 24, 17, 2), (3, 16, 16, 40, 2), (1, 32, 64, 41, 2), (2, 28, 56, 41, 4),
                       (2, 60, 24, 13, 4), (2, 24, 56, 29, 5), (2, 24, 56, 17, 5), (1, 8, 64, 41, 5),
                       (1, 16, 64, 23, 5), (2, 36, 56, 41, 7), (2, 36, 56, 17, 7)]),
    (16, (36, 33, 34), [(1, 16, 64, 12), (2, 16, 16, 12), (2, 16, 16, 40), (1, 32, 32, 7), (1, 16, 64, 36, 1),
                        (2, 16, 16, 36, 1), (1, 8, 64, 36, 2), (1, 16, 64, 12, 2), (2, 16, 16, 36, 2),
                        (1, 32, 64, 36, 2), (1, 32, 64, 36, 6), (1, 64, 32, 12, 6)]),
])
def test_tiled_bit_identical_to_one_step(W, oracle, so, shape, tilings):
    nt = 23
    w = small_layered(shape, so, nt, seed=3 + so)
    ref_rec, ref_u = run_gpu(W, w, tilings[0])
    rec_o, up_o, uc_o = run_oracle(oracle, w)
    assert close(ref_u[1], uc_o)
    assert close(ref_u[0], up_o)
    assert close(ref_rec, rec_o)
    for t in tilings[1:]:
        rec, uf = run_gpu(W, w, t)
        assert np.array_equal(rec, ref_rec), t
        assert np.array_equal(uf, ref_u), t


def test_layered_so8_long_run_vs_oracle(W, oracle):
    w = small_layered((64, 56, 60), 8, 300, seed=21, f=20.0, sponge=8)
    rec_o, up_o, uc_o = run_oracle(oracle, w)
    rec, uf = run_gpu(W, w, (2, 24, 24, 64))
    assert close(uf[1], uc_o)
    assert close(rec, rec_o)


@pytest.mark.parametrize("so,shape,tilings", [
    # SO16: the two-row warp-specialised one-step pass the SO16 bench picks, and the one-row pass
    (16, (56, 52, 48), [(1, 64, 32, 40, 6), (1, 32, 64, 56, 2)]),
    # SO4: the three-step warp-specialised passes (one row, two rows per thread) and the one-step pass
    (4, (64, 60, 56), [(3, 24, 56, 40, 5), (1, 16, 64, 64, 0), (3, 36, 56, 40, 7)]),
])
def test_layered_long_run_vs_oracle(W, oracle, so, shape, tilings):
    """400 steps (the accumulated float32 rounding of a long run) against the
    FP64 oracle, through the sponge and the free surface; the variants agree
    bit for bit."""
    w = small_layered(shape, so, 400, seed=30 + so, f=20.0, sponge=8)
    rec_o, up_o, uc_o = run_oracle(oracle, w)
    rec, uf = run_gpu(W, w, tilings[0])
    assert close(uf[1], uc_o)
    assert close(uf[0], up_o)
    assert close(rec, rec_o)
    for t in tilings[1:]:
        rec2, uf2 = run_gpu(W, w, t)
        assert np.array_equal(rec2, rec), t
        assert np.array_equal(uf2, uf), t


def test_gaussian_initial_field_source_free(W, oracle):
    """Section "Functional Correctness": source removed, u initialised with a
    3D Gaussian (sigma 0.4 on [-1, 1]^3); tiled vs untiled and vs the oracle."""
    from paper_1707_02347_gb300 import inputs

    shape = (44, 40, 36)
    g = inputs.gaussian_field(shape, 0.4)
    w = inputs.layered_forward(shape, 8, 40, seed=5, f=20.0, h=20.0, sponge_width=0)
    w.src_xyz = np.zeros((0, 3))
    w.rec_xyz = np.zeros((0, 3))
    u0 = np.stack([g, g])
    _, ref = run_gpu(W, w, (1, 8, 64, 44), u_init=u0)
    _, up_o, uc_o = run_oracle(oracle, w, u_init=u0)
    assert close(ref[1], uc_o)
    for t in [(2, 16, 56, 44), (3, 16, 16, 20), (2, 24, 56, 44, 5)]:
        _, uf = run_gpu(W, w, t, u_init=u0)
        assert np.array_equal(uf, ref), t


def test_edge_cases(W, oracle):
    from paper_1707_02347_gb300 import inputs

    # minimum grid (so + 1 per axis), nz not a multiple of 4
    w = small_layered((9, 9, 9), 8, 7, seed=2, nrec=3, sponge=2)
    rec_o, up_o, uc_o = run_oracle(oracle, w)
    for t in [(1, 8, 64, 9), (2, 8, 56, 5), (3, 16, 16, 9), (2, 24, 56, 5, 5)]:
        rec, uf = run_gpu(W, w, t)
        assert close(uf[1], uc_o) and close(rec, rec_o), t
    # minimum SO16 grid, the two-row warp-specialised pass (tile larger than the grid)
    w = small_layered((17, 17, 17), 16, 5, seed=3, nrec=3, sponge=2)
    rec_o, _, uc_o = run_oracle(oracle, w)
    rec, uf = run_gpu(W, w, (1, 64, 32, 17, 6))
    assert close(uf[1], uc_o) and close(rec, rec_o)
    # nt = 0: the initial fields come back (u^0 exactly, u^{-1} through one
    # rounding of the stored increment u^0 - u^{-1}) and there are no traces
    w0 = small_layered((20, 18, 17), 4, 0, seed=4)
    rng = np.random.default_rng(0)
    u0 = rng.standard_normal((2,) + w0.shape).astype(np.float32)
    for t in [(2, 12, 56, 20), (2, 28, 56, 20, 5)]:
        rec, uf = run_gpu(W, w0, t, u_init=u0)
        assert rec.shape == (0, w0.rec_xyz.shape[0])
        assert np.array_equal(uf[1], u0[1])
        np.testing.assert_allclose(uf[0], u0[0], rtol=0, atol=2.5e-7 * np.abs(u0).max())
    # nt not a multiple of T; two sources on the same grid point
    w = small_layered((30, 28, 26), 4, 11, seed=7)
    w.src_xyz = np.vstack([w.src_xyz, w.src_xyz[:1]])
    w.wavelet = np.concatenate([w.wavelet, -0.5 * w.wavelet[:, :1]], axis=1)
    rec_o, _, uc_o = run_oracle(oracle, w)
    r1, u1 = run_gpu(W, w, (1, 16, 64, 30))
    r3, u3 = run_gpu(W, w, (3, 24, 24, 30))
    r4, u4 = run_gpu(W, w, (4, 20, 16, 30))
    r5, u5 = run_gpu(W, w, (3, 24, 56, 30, 5))
    assert close(u1[1], uc_o) and close(r1, rec_o)
    assert np.array_equal(u1, u3) and np.array_equal(r1, r3)
    assert np.array_equal(u1, u4) and np.array_equal(r1, r4)
    assert np.array_equal(u1, u5) and np.array_equal(r1, r5)


def test_invalid_arguments(W):
    dev = torch.device("cuda")
    m = torch.full((20, 20, 20), 1.0 / 2.25, device=dev)
    h = (10.0, 10.0, 10.0)
    dt_max = W.cfl_limit(8, h, 1.5)
    with pytest.raises(W.WaveError) as e:
        W.WavePlan((20, 20, 20), h, 8, 1.01 * dt_max, 10, m)
    assert e.value.status == 2  # WAVE_ERR_CFL
    with pytest.raises(W.WaveError) as e:
        W.WavePlan((20, 20, 20), h, 6, 0.5 * dt_max, 10, m)
    assert e.value.status == 1
    with pytest.raises(W.WaveError) as e:
        W.WavePlan((8, 20, 20), h, 8, 0.5 * dt_max, 10, m)
    assert e.value.status == 1
    bad = m.clone()
    bad[3, 4, 5] = -1.0
    with pytest.raises(W.WaveError) as e:
        W.WavePlan((20, 20, 20), h, 8, 0.5 * dt_max, 10, bad)
    assert e.value.status == 1
    plan = W.WavePlan((20, 20, 20), h, 8, 0.5 * dt_max, 10, m)
    with pytest.raises(W.WaveError):
        plan.set_tiling((2, 64, 64, 20))
    with pytest.raises(W.WaveError):
        plan.set_tiling((2, 16, 30, 20))
    plan.set_tiling((2, 24, 24, 20))
    assert plan.get_tiling() == (2, 24, 24, 20, 0)
    plan.close()


def test_bounded_wait_reports_timeout_and_device_stays_usable(W, oracle):
    """Failure detection without a fault: a wait that nothing satisfies gives
    up after 50 ms and is reported as WAVE_ERR_TIMEOUT; the context keeps
    working (a forward run afterwards still matches the oracle)."""
    import ctypes

    lib = W.load()
    lib.wave_selftest_timeout.restype = ctypes.c_int
    lib.wave_selftest_timeout.argtypes = [ctypes.c_double]
    assert lib.wave_selftest_timeout(50.0) == 5  # WAVE_ERR_TIMEOUT
    assert lib.wave_selftest_timeout(0.0) == 1
    w = small_layered((20, 18, 17), 4, 9, seed=12)
    rec_o, _, uc_o = run_oracle(oracle, w)
    rec, uf = run_gpu(W, w, (2, 12, 56, 20))
    assert close(uf[1], uc_o) and close(rec, rec_o)


@pytest.mark.parametrize("so", [8, 16])
def test_dense_receiver_surface_gather(W, oracle, so):
    """64 x 64 surface receivers at 25 m (all taps in the first z quad): with
    one-step passes the traces are gathered from the field after each pass;
    they equal, bit for bit, the per-tap path (forced by one extra receiver
    deeper down, and used by the T = 2 pass), and match the oracle."""
    from paper_1707_02347_gb300 import inputs

    shape = (40, 37, 30)
    w = small_layered(shape, so, 21, seed=31, nrec=0)
    surf = inputs.surface_receivers(shape, w.spacing, 64, 25.0)
    deep = np.vstack([surf, [[150.0, 160.0, 215.0]]])  # taps in a third z quad: per-tap path
    tilings = [(1, 16, 64, 40, 2), (2, 16, 56, 40, 2) if so == 8 else (2, 16, 16, 40, 2), (1, 16, 64, 40, 0)]
    w.rec_xyz = surf
    cap = [run_gpu(W, w, t)[0] for t in tilings]
    w.rec_xyz = deep
    csr = [run_gpu(W, w, t)[0] for t in tilings]
    for a, b in zip(cap, csr):
        assert np.array_equal(a, cap[0])
        assert np.array_equal(b[:, :-1], cap[0])
    w.rec_xyz = surf
    rec_o, _, _ = run_oracle(oracle, w)
    assert close(cap[0], rec_o)


@pytest.mark.parametrize("so,tiling", [(8, (2, 28, 56, 12, 4)), (8, (2, 60, 24, 9, 4)), (4, (2, 30, 56, 11, 4))])
def test_skewed_wavefront_tiles(W, oracle, so, tiling):
    """Skewed wavefront variant (y tiles shifted by r per step, each tile
    taking the top rows of the tile below through the exchange buffer) on a
    grid of several y tiles, x slabs and z tiles: bit-identical to the
    one-step kernel, fields and traces, and within the parity bar of the
    oracle."""
    shape = (31, 95, 130)
    w = small_layered(shape, so, 19, seed=61 + so, nrec=11)
    ref_rec, ref_u = run_gpu(W, w, (1, 16, 64, 31))
    rec, uf = run_gpu(W, w, tiling)
    assert np.array_equal(rec, ref_rec)
    assert np.array_equal(uf, ref_u)
    rec_o, up_o, uc_o = run_oracle(oracle, w)
    assert close(uf[1], uc_o)
    assert close(rec, rec_o)


@pytest.mark.parametrize("so", [4, 8, 16])
def test_autotune_then_forward(W, oracle, so):
    """The autotuner times every compiled candidate on the plan's grid (all
    variants, including the skewed wavefront one, whose buffers it sizes on
    the way), keeps the fastest, and the tuned plan still matches the
    one-step kernel bit for bit."""
    shape = (44, 60, 52)
    w = small_layered(shape, so, 17, seed=71 + so, nrec=7)
    ref_rec, ref_u = run_gpu(W, w, (1, 16, 64, 44))
    dev = torch.device("cuda")
    m = torch.from_numpy(np.ascontiguousarray(w.m, dtype=np.float32)).to(dev)
    plan = W.WavePlan(w.shape, w.spacing, w.so, w.dt, w.nt, m, sponge_width=w.sponge_width,
                      sponge_faces=w.sponge_faces, vmax=w.vmax)
    plan.set_sources(w.src_xyz, torch.from_numpy(np.ascontiguousarray(w.wavelet, dtype=np.float32)).to(dev))
    plan.set_receivers(w.rec_xyz)
    tuned = plan.autotune(passes=1)
    assert len(tuned) > 3
    assert any(t[0][4] == 4 for t in tuned) == (so in (4, 8))  # skewed candidates timed where compiled
    rec, uf = plan.forward(want_final=True)
    torch.cuda.synchronize()
    assert np.array_equal(rec.cpu().numpy(), ref_rec)
    assert np.array_equal(uf.cpu().numpy(), ref_u)
    plan.close()


def test_autotune_cache(W, tmp_path, monkeypatch):
    """wave_autotune_cached: the first plan of a key times the candidates, a
    second plan of the same key takes the stored tilings (the overall pick and
    the one-step sweep tiling) without timing, and with WAVE_AUTOTUNE_CACHE
    both persist to a fresh process."""
    import os
    import subprocess
    import sys

    path = tmp_path / "tune.txt"
    monkeypatch.setenv("WAVE_AUTOTUNE_CACHE", str(path))
    script = """
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import paper_1707_02347_gb300 as W
from paper_1707_02347_gb300 import inputs
w = inputs.layered_forward((40, 44, 36), 8, 9, seed=5, f=25.0, h=10.0, sponge_width=4)
m = torch.from_numpy(np.ascontiguousarray(w.m)).cuda()
p = W.WavePlan(w.shape, w.spacing, 8, w.dt, w.nt, m, sponge_width=w.sponge_width, vmax=w.vmax)
t, hit = p.autotune_cached(passes=1)
print(int(hit), *t, *p.get_sweep_tiling())
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

    def run_here():
        from paper_1707_02347_gb300 import inputs

        w = inputs.layered_forward((40, 44, 36), 8, 9, seed=5, f=25.0, h=10.0, sponge_width=4)
        m = torch.from_numpy(np.ascontiguousarray(w.m)).cuda()
        p = W.WavePlan(w.shape, w.spacing, 8, w.dt, w.nt, m, sponge_width=w.sponge_width, vmax=w.vmax)
        t, hit = p.autotune_cached(passes=1)
        sweep = p.get_sweep_tiling()
        p.close()
        return t, hit, sweep

    t1, hit1, s1 = run_here()
    assert not hit1
    assert s1[0] == 1  # the fastest one-step candidate runs the one-step sweeps
    t2, hit2, s2 = run_here()
    assert hit2 and t2 == t1
    assert s2 == s1  # a cache hit restores the one-step sweep tiling too
    lines = path.read_text().splitlines()
    assert any(line.split()[1:] == [str(v) for v in t1 + s1] for line in lines)
    out = subprocess.run([sys.executable, "-c", script.format(root=root)], capture_output=True, text=True,
                         env=dict(os.environ), timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    fields = out.stdout.split()
    assert fields[0] == "1" and tuple(int(v) for v in fields[1:]) == tuple(t1) + tuple(s1)
