"""Parity at the full sizes, in the launch configurations the benchmark
times: the 512^3 SO8 workload (the warp-specialised one-step pass the
autotuner picks, and the T = 2 pass with the x queues in tensor memory), the
same grid at SO4 (the warp-specialised two-step pass the autotuner picks
there), and the 768 x 768 x 384 SO16 workload with its 501 x 501 receiver
surface (the warp-specialised one-step pass with two rows per thread).

The other variants (the block-barrier one-step pass, the skewed wavefront
and warp-specialised two-step passes, the one-row SO16 pass) are checked
against the same passes bit for bit.

The FP64 oracle cannot run the whole grid, so outputs are checked one by one:
the GPU runs the workload for n1 steps and keeps the state (u^{n1-1}, u^{n1});
then it advances one more pass (T steps) from that state.  For each sampled
point p the oracle advances the same T steps on a window around p that
reaches r T points past p on every side (clipped at the grid, where its zero
ghosts are the grid's), starting from the GPU's state in FP64.  After T steps
the oracle's value at p depends only on the window, so it is the exact result
of the paper's update at p.  Sampled points: near the source, at the free
surface, in the sponge, on the receiver line, and at random.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N = 512
SO = 8
R = SO // 2
N1 = 110  # steps before the checked pass (the 15 Hz Ricker peaks near step 77)


@pytest.fixture(scope="module")
def state(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W
    from paper_1707_02347_gb300 import inputs

    W.load()
    dev = torch.device("cuda")
    w = inputs.layered_forward((N, N, N), SO, N1 + 2, seed=1, f=15.0, h=10.0, sponge_width=10, nrec_line=512)
    m = torch.from_numpy(np.ascontiguousarray(w.m)).to(dev)
    wav = np.ascontiguousarray(w.wavelet.astype(np.float32))
    plan = W.WavePlan(w.shape, w.spacing, SO, w.dt, N1, m, sponge_width=w.sponge_width, vmax=w.vmax,
                      tiling=(1, 8, 64, 64, 2))
    plan.set_sources(w.src_xyz, torch.from_numpy(wav[:N1]).to(dev))
    plan.set_receivers(w.rec_xyz)
    _, uA = plan.forward(want_final=True)
    plan.close()
    out = {}
    for T, tiling in ((1, (1, 8, 64, 64, 5)), ("T1v2", (1, 8, 64, 64, 2)), (2, (2, 24, 56, 128, 2)),
                      ("skew", (2, 28, 56, 128, 4)), ("lean", (2, 24, 56, 256, 5)), ("v7", (2, 36, 56, 256, 7))):
        nT = 2 if T in (2, "skew", "lean", "v7") else 1
        p = W.WavePlan(w.shape, w.spacing, SO, w.dt, nT, m, sponge_width=w.sponge_width, vmax=w.vmax, tiling=tiling)
        p.set_sources(w.src_xyz, torch.from_numpy(wav[N1:N1 + nT].copy()).to(dev))
        _, uB = p.forward(u_init=uA, want_final=True)
        torch.cuda.synchronize()
        out[T] = uB[1].cpu().numpy()
        p.close()
    # two one-step passes from the same state: bit-identical to the T = 2 pass
    p = W.WavePlan(w.shape, w.spacing, SO, w.dt, 2, m, sponge_width=w.sponge_width, vmax=w.vmax,
                   tiling=(1, 8, 64, 64, 2))
    p.set_sources(w.src_xyz, torch.from_numpy(wav[N1:N1 + 2].copy()).to(dev))
    _, uC = p.forward(u_init=uA, want_final=True)
    torch.cuda.synchronize()
    out["T1x2"] = uC[1].cpu().numpy()
    p.close()
    A = uA.cpu().numpy()
    return w, A, out


def _samples(w, rng):
    n = np.asarray(w.shape)
    src = np.round(w.src_xyz[0] / np.asarray(w.spacing)).astype(int)
    pts = []
    for _ in range(24):  # around the source, where the wavefield is
        pts.append(np.clip(src + rng.integers(-14, 15, 3), 0, n - 1))
    for _ in range(8):  # free surface z = 0 .. 3
        pts.append(np.array([src[0] + rng.integers(-12, 13), src[1] + rng.integers(-12, 13), rng.integers(0, 4)]))
    for _ in range(8):  # sponge layers, every face
        a = rng.integers(0, 3)
        p = np.array([rng.integers(0, c) for c in n])
        p[a] = rng.integers(0, 10) if rng.integers(0, 2) else n[a] - 1 - rng.integers(0, 10)
        pts.append(p)
    for _ in range(8):  # grid corners and edges
        pts.append(np.array([rng.choice([0, 1, c - 2, c - 1]) for c in n]))
    for _ in range(8):  # anywhere
        pts.append(np.array([rng.integers(0, c) for c in n]))
    return [tuple(int(c) for c in p) for p in pts]


def _oracle_at(oracle, w, A, p, T, n1=N1):
    r = w.so // 2
    lo = [max(0, c - r * T) for c in p]
    hi = [min(n, c + r * T + 1) for c, n in zip(p, w.shape)]
    sl = tuple(slice(a, b) for a, b in zip(lo, hi))
    shape = tuple(b - a for a, b in zip(lo, hi))
    _, _, uc = oracle.forward(shape, w.spacing, w.so, w.dt, T, w.m[sl].astype(np.float64), src_xyz=w.src_xyz,
                              wavelet=w.wavelet[n1:n1 + T].astype(np.float32).astype(np.float64),
                              u_prev0=A[0][sl].astype(np.float64), u_cur0=A[1][sl].astype(np.float64),
                              sponge_width=w.sponge_width, sponge_faces=w.sponge_faces, vmax=w.vmax,
                              origin=tuple(lo), global_shape=tuple(w.shape))
    return uc[tuple(c - a for c, a in zip(p, lo))], float(np.abs(uc).max())


def _check_sampled(oracle, w, A, out, T, seed, n1=N1):
    rng = np.random.default_rng(seed)
    got, ref, scale = [], [], []
    for p in _samples(w, rng):
        o, s = _oracle_at(oracle, w, A, p, T, n1)
        got.append(float(out[p]))
        ref.append(o)
        scale.append(s)
    got, ref, scale = np.array(got), np.array(ref), np.array(scale)
    assert np.abs(ref).max() > 0.0  # the checked pass carries a wavefield
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    assert np.all(np.abs(got - ref) <= 1e-5 * np.maximum(scale, 1e-30))


@pytest.mark.parametrize("T", [1, 2])
def test_full_size_pass_vs_oracle_at_sampled_points(state, oracle, T):
    w, A, out = state
    _check_sampled(oracle, w, A, out[T], T, 40 + T)


def test_full_size_two_one_step_passes_equal_one_t2_pass(state):
    _, _, out = state
    assert np.array_equal(out["T1x2"], out[2])
    assert np.array_equal(out["T1x2"], out["skew"])  # the skewed wavefront variant of the two-step pass
    assert np.array_equal(out["T1x2"], out["lean"])  # the warp-specialised two-step pass
    assert np.array_equal(out["T1x2"], out["v7"])  # two rows per thread, shift-register queues


def test_full_size_one_step_variants_bit_identical(state):
    _, _, out = state
    assert np.array_equal(out[1], out["T1v2"])  # warp-specialised vs block-barrier one-step pass


@pytest.fixture(scope="module")
def state4(oracle):
    """512^3 SO4: N1 steps, then two more steps from that state as one
    two-step pass in the launch configuration the SO4 bench picks (40 x 56
    tile, 64-plane slabs, warp-specialised pass) and as two one-step passes."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W
    from paper_1707_02347_gb300 import inputs

    W.load()
    dev = torch.device("cuda")
    w = inputs.layered_forward((N, N, N), 4, N1 + 2, seed=1, f=15.0, h=10.0, sponge_width=10, nrec_line=512)
    m = torch.from_numpy(np.ascontiguousarray(w.m)).to(dev)
    wav = np.ascontiguousarray(w.wavelet.astype(np.float32))
    kw = dict(sponge_width=w.sponge_width, vmax=w.vmax)
    plan = W.WavePlan(w.shape, w.spacing, 4, w.dt, N1, m, tiling=(1, 8, 64, 64, 5), **kw)
    plan.set_sources(w.src_xyz, torch.from_numpy(wav[:N1]).to(dev))
    plan.set_receivers(w.rec_xyz)
    _, uA = plan.forward(want_final=True)
    plan.close()
    out = {}
    for name, tiling in (("T2", (2, 40, 56, 64, 5)), ("T1x2", (1, 8, 64, 64, 5))):
        p = W.WavePlan(w.shape, w.spacing, 4, w.dt, 2, m, tiling=tiling, **kw)
        p.set_sources(w.src_xyz, torch.from_numpy(wav[N1:N1 + 2].copy()).to(dev))
        _, uB = p.forward(u_init=uA, want_final=True)
        torch.cuda.synchronize()
        out[name] = uB[1].cpu().numpy()
        p.close()
    return w, uA.cpu().numpy(), out


def test_full_size_so4_two_step_pass_vs_oracle_at_sampled_points(state4, oracle):
    w, A, out = state4
    _check_sampled(oracle, w, A, out["T2"], 2, 44)


def test_full_size_so4_two_step_pass_equals_two_one_step_passes(state4):
    _, _, out = state4
    assert np.array_equal(out["T2"], out["T1x2"])


N1_16 = 100  # SO16 steps before the checked pass (the Ricker peaks near step 66)


@pytest.fixture(scope="module")
def state16(oracle):
    """768 x 768 x 384 SO16 with the 501 x 501 surface: N1_16 steps, then one
    more pass in the bench's launch configuration (64 x 32 tile, 128-plane
    slabs, variant 6) and in the one-row tensor-memory pass."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W
    from paper_1707_02347_gb300 import inputs

    W.load()
    dev = torch.device("cuda")
    w = inputs.high_order_forward(N1_16 + 1)
    m = torch.from_numpy(np.ascontiguousarray(w.m)).to(dev)
    wav = np.ascontiguousarray(w.wavelet.astype(np.float32))
    kw = dict(sponge_width=w.sponge_width, vmax=w.vmax)
    plan = W.WavePlan(w.shape, w.spacing, w.so, w.dt, N1_16, m, tiling=(1, 64, 32, 128, 6), **kw)
    plan.set_sources(w.src_xyz, torch.from_numpy(wav[:N1_16]).to(dev))
    plan.set_receivers(w.rec_xyz)
    _, uA = plan.forward(want_final=True)
    plan.close()
    out = {}
    for name, tiling in (("v6", (1, 64, 32, 128, 6)), ("v2", (1, 32, 64, 256, 2))):
        p = W.WavePlan(w.shape, w.spacing, w.so, w.dt, 1, m, tiling=tiling, **kw)
        p.set_sources(w.src_xyz, torch.from_numpy(wav[N1_16:N1_16 + 1].copy()).to(dev))
        p.set_receivers(w.rec_xyz)
        rec, uB = p.forward(u_init=uA, want_final=True)
        torch.cuda.synchronize()
        out[name] = uB[1].cpu().numpy()
        out[name + "_rec"] = rec.cpu().numpy()
        p.close()
    A = uA.cpu().numpy()
    return w, A, out


def test_full_size_so16_pass_vs_oracle_at_sampled_points(state16, oracle):
    w, A, out = state16
    _check_sampled(oracle, w, A, out["v6"], 1, 61, n1=N1_16)


def test_full_size_so16_variants_bit_identical(state16):
    _, _, out = state16
    assert np.array_equal(out["v6"], out["v2"])
    assert np.array_equal(out["v6_rec"], out["v2_rec"])
    assert np.abs(out["v6_rec"]).max() > 0.0
