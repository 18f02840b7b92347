"""Batched shots: uneven grids, SO 4 and 8 mixed, per-shot tilings, all
advanced by one CUDA graph launch -- bit-identical to running each plan's
wave_forward on its own, and correct against the FP64 oracle."""
import numpy as np
import pytest
from parity import assert_close

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _shots(n, seed):
    from paper_1707_02347_gb300 import inputs

    rng = np.random.default_rng(seed)
    out = []
    for s in range(n):
        shape = (int(rng.integers(20, 41)), int(rng.integers(20, 41)), int(rng.integers(16, 33)))
        so = 4 if s % 2 == 0 else 8
        nt = 20 + int(rng.integers(0, 9))
        f = float(rng.uniform(20.0, 35.0))
        w = inputs.layered_forward(shape, so, nt, seed=100 + s, f=f, h=10.0, sponge_width=4, nrec_line=6)
        out.append(w)
    return out


def test_batched_shots_match_single_plans_and_oracle(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W

    W.load()
    dev = torch.device("cuda")
    shots = _shots(6, 7)
    plans = []
    for i, w in enumerate(shots):
        m = torch.from_numpy(np.ascontiguousarray(w.m)).to(dev)
        tiling = ((2, 12, 56, 32) if w.so == 4 else (2, 24, 24, 32)) if i % 3 else (1, 16, 64, 32)
        p = W.WavePlan(w.shape, w.spacing, w.so, w.dt, w.nt, m, sponge_width=w.sponge_width, vmax=w.vmax,
                       tiling=tiling)
        p.set_sources(w.src_xyz, torch.from_numpy(w.wavelet.astype(np.float32)).to(dev))
        p.set_receivers(w.rec_xyz)
        plans.append(p)
    single = []
    for p in plans:
        rec, _ = p.forward()
        single.append(rec.clone())
    batch = W.WaveBatch(plans)
    for rep in range(2):  # the second call replays the captured graph
        recs = batch.forward()
        torch.cuda.synchronize()
        for a, b in zip(recs, single):
            assert torch.equal(a, b)
    for w, r in zip(shots, single):
        ref, _, _ = oracle.forward(w.shape, w.spacing, w.so, w.dt, w.nt, w.m.astype(np.float64), src_xyz=w.src_xyz,
                                   wavelet=w.wavelet, rec_xyz=w.rec_xyz, sponge_width=w.sponge_width,
                                   sponge_faces=w.sponge_faces, vmax=w.vmax)
        assert_close(r.cpu().numpy(), ref, 1e-5, "batched traces")
    batch.close()
    for p in plans:
        p.close()


def test_batched_gradients_match_single_plans(oracle):
    """wave_batch_gradient: every shot's checkpointed forward, adjoint sweep
    and imaging in one graph launch, bit-identical to wave_gradient per plan;
    a buffer replaced between calls (a changed tiling) triggers a recapture
    and the forward graph keeps working."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W

    W.load()
    dev = torch.device("cuda")
    shots = _shots(4, 11)
    plans, dobs = [], []
    for i, w in enumerate(shots):
        m_true = torch.from_numpy(np.ascontiguousarray(w.m)).to(dev)
        tiling = ((2, 28, 56, 32, 2) if w.so == 4 else (2, 24, 56, 32, 2)) if i % 2 else (1, 16, 64, 32)
        p = W.WavePlan(w.shape, w.spacing, w.so, w.dt, w.nt, m_true, sponge_width=w.sponge_width, vmax=w.vmax,
                       tiling=tiling)
        p.set_sources(w.src_xyz, torch.from_numpy(w.wavelet.astype(np.float32)).to(dev))
        p.set_receivers(w.rec_xyz)
        d, _ = p.forward()
        dobs.append(d.clone())
        # start model: 3 % slower everywhere
        p.set_model(m_true * 1.03 ** 2)
        plans.append(p)
    single = []
    for p, d in zip(plans, dobs):
        J, g = p.gradient(d, checkpoint_every=7)
        single.append((J, g.clone()))
    batch = W.WaveBatch(plans)
    for rep in range(2):
        mis, grads = batch.gradient(dobs, checkpoint_every=7)
        torch.cuda.synchronize()
        for (J, g), j2, g2 in zip(single, mis, grads):
            assert j2 == J
            assert torch.equal(g2, g)
    # a new tiling replaces the plan's geometry: both graphs are captured again
    plans[0].set_tiling((2, 12, 56, 32) if shots[0].so == 4 else (2, 24, 24, 32))
    recs = batch.forward()
    mis, grads = batch.gradient(dobs, checkpoint_every=7)
    torch.cuda.synchronize()
    J0, g0 = plans[0].gradient(dobs[0], checkpoint_every=7)
    assert mis[0] == J0 and torch.equal(grads[0], g0)
    r0, _ = plans[0].forward()
    assert torch.equal(recs[0], r0)
    batch.close()
    for p in plans:
        p.close()


def test_full_size_batched_shots(oracle):
    """Four shots of the 24-shot workload at their full sizes (the same draws
    of seed 5: grids U[128, 320] x U[128, 320] x U[128, 256], SO 4/8, 600 steps,
    Ricker 8-15 Hz, 64 receivers at 20 m), each with a tiling the autotuner
    picks for it (variants 0 and 5, T = 1 and 2): the batched forward and
    the batched gradient (checkpoints every 40 steps) equal the single plans
    bit for bit, and the smallest shot's traces match the FP64 oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W
    from paper_1707_02347_gb300 import inputs

    W.load()
    dev = torch.device("cuda")
    nt = 600
    rng = np.random.default_rng(5)
    draws = []
    for s in range(24):
        shape = (int(rng.integers(128, 321)), int(rng.integers(128, 321)), int(rng.integers(128, 257)))
        draws.append((shape, 4 if s % 2 == 0 else 8, float(rng.uniform(8.0, 15.0))))
    picked = {0: (2, 28, 56, 64, 5), 2: (2, 28, 24, 64, 0), 3: (1, 8, 64, 64, 5), 21: (1, 8, 64, 64, 5)}
    plans, works, m_true = [], [], []
    for s, tiling in picked.items():
        shape, so, f = draws[s]
        w = inputs.layered_forward(shape, so, nt, seed=500 + s, f=f, h=10.0, sponge_width=10, nrec_line=64)
        m = torch.from_numpy(np.ascontiguousarray(w.m)).to(dev)
        p = W.WavePlan(w.shape, w.spacing, so, w.dt, nt, m, sponge_width=w.sponge_width, vmax=w.vmax, tiling=tiling)
        p.set_sources(w.src_xyz, torch.from_numpy(w.wavelet.astype(np.float32)).to(dev))
        p.set_receivers(w.rec_xyz)
        plans.append(p)
        works.append(w)
        m_true.append(m)
    single = [p.forward()[0].clone() for p in plans]
    batch = W.WaveBatch(plans)
    recs = batch.forward()
    torch.cuda.synchronize()
    for r, r1 in zip(recs, single):
        assert torch.equal(r, r1)
    # the smallest shot (206 x 128 x 134, SO8) against the oracle
    k = list(picked).index(3)
    w = works[k]
    rec_o, _, _ = oracle.forward(w.shape, w.spacing, w.so, w.dt, nt, w.m.astype(np.float64), src_xyz=w.src_xyz,
                                 wavelet=w.wavelet.astype(np.float32).astype(np.float64), rec_xyz=w.rec_xyz,
                                 sponge_width=w.sponge_width, sponge_faces=w.sponge_faces, vmax=w.vmax)
    got = recs[k].cpu().numpy().astype(np.float64)
    assert np.abs(rec_o).max() > 0.0
    assert_close(got, rec_o, 1e-5, "smallest full-size shot")
    # gradients on a start model 3 % slower
    d_obs = [r.clone() for r in recs]
    for p, m in zip(plans, m_true):
        p.set_model(m * 1.03 ** 2)
    single_g = []
    for p, d in zip(plans, d_obs):
        J, g = p.gradient(d, checkpoint_every=40)
        single_g.append((J, g.clone()))
    mis, grads = batch.gradient(d_obs, checkpoint_every=40)
    torch.cuda.synchronize()
    for (J, g), j2, g2 in zip(single_g, mis, grads):
        assert np.isfinite(J) and J > 0.0
        assert j2 == J
        assert torch.equal(g2, g)
        assert bool(torch.isfinite(g2).all())
    batch.close()
    for p in plans:
        p.close()


# tilings of the persistent batched kernel (tensor-memory queues): 512-thread
# tiles for SO4 and SO8, T = 1, 2, 3, both tile orientations, and the
# one-step 128-thread tile that four teams of a block run side by side
_PERSISTENT = {4: [(1, 32, 64, 32, 2), (2, 28, 56, 32, 2), (1, 8, 64, 32, 2), (2, 60, 24, 32, 2),
                   (3, 24, 56, 32, 2)],
               8: [(1, 8, 64, 32, 2), (2, 24, 56, 32, 2), (1, 32, 64, 32, 2), (2, 56, 24, 32, 2)]}


def test_persistent_batch_matches_single_plans_and_recovers_from_timeout(oracle):
    """Every shot's tiling has a shape in the persistent kernel, so the batch
    runs as one persistent launch fed by the device work queue: its traces
    equal each plan's own wave_forward bit for bit (nt not a multiple of T:
    the remainder passes run one-step tiles in the same queue) and match the
    FP64 oracle.  Then a dependency is withheld on the host side: the waiting
    work items give up after 50 ms with WAVE_ERR_TIMEOUT, and the next
    batched forward runs normally with the same bits."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W

    W.load()
    dev = torch.device("cuda")
    shots = _shots(9, 17)
    plans = []
    for i, w in enumerate(shots):
        m = torch.from_numpy(np.ascontiguousarray(w.m)).to(dev)
        opts = _PERSISTENT[w.so]
        p = W.WavePlan(w.shape, w.spacing, w.so, w.dt, w.nt, m, sponge_width=w.sponge_width, vmax=w.vmax,
                       tiling=opts[(i // 2) % len(opts)])
        p.set_sources(w.src_xyz, torch.from_numpy(w.wavelet.astype(np.float32)).to(dev))
        p.set_receivers(w.rec_xyz)
        plans.append(p)
    assert any(w.nt % p.get_tiling()[0] for w, p in zip(shots, plans))  # some remainder passes
    single = []
    for p in plans:
        rec, _ = p.forward()
        single.append(rec.clone())
    batch = W.WaveBatch(plans)
    for rep in range(2):
        recs = batch.forward()
        torch.cuda.synchronize()
        persistent, items, blocks = batch.mode()
        assert persistent and items > 0 and blocks > 0
        for a, b in zip(recs, single):
            assert torch.equal(a, b)
    w = shots[1]
    ref, _, _ = oracle.forward(w.shape, w.spacing, w.so, w.dt, w.nt, w.m.astype(np.float64), src_xyz=w.src_xyz,
                               wavelet=w.wavelet.astype(np.float32).astype(np.float64), rec_xyz=w.rec_xyz,
                               sponge_width=w.sponge_width, sponge_faces=w.sponge_faces, vmax=w.vmax)
    assert_close(recs[1].cpu().numpy(), ref, 1e-5, "persistent batch traces")
    # failure detection: a withheld dependency times out, the device stays usable
    assert batch.selftest_withhold(50.0) == 5  # WAVE_ERR_TIMEOUT
    recs = batch.forward()
    torch.cuda.synchronize()
    assert batch.mode()[0]
    for a, b in zip(recs, single):
        assert torch.equal(a, b)
    batch.close()
    for p in plans:
        p.close()


def test_full_size_persistent_batch_autotuned(oracle):
    """Four shots of the 24-shot workload at their full sizes (the same draws
    of seed 5, 600 steps), each autotuned over the persistent kernel's
    tilings: one persistent launch gives every plan's own wave_forward traces
    bit for bit, and the smallest shot matches the FP64 oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W
    from paper_1707_02347_gb300 import inputs

    W.load()
    dev = torch.device("cuda")
    nt = 600
    rng = np.random.default_rng(5)
    draws = []
    for s in range(24):
        shape = (int(rng.integers(128, 321)), int(rng.integers(128, 321)), int(rng.integers(128, 257)))
        draws.append((shape, 4 if s % 2 == 0 else 8, float(rng.uniform(8.0, 15.0))))
    plans, works = [], []
    for s in (0, 2, 3, 21):
        shape, so, f = draws[s]
        w = inputs.layered_forward(shape, so, nt, seed=500 + s, f=f, h=10.0, sponge_width=10, nrec_line=64)
        m = torch.from_numpy(np.ascontiguousarray(w.m)).to(dev)
        p = W.WavePlan(w.shape, w.spacing, so, w.dt, nt, m, sponge_width=w.sponge_width, vmax=w.vmax)
        p.set_sources(w.src_xyz, torch.from_numpy(w.wavelet.astype(np.float32)).to(dev))
        p.set_receivers(w.rec_xyz)
        plans.append(p)
        works.append(w)
    batch = W.WaveBatch(plans)
    tilings = batch.autotune(passes=1)
    assert all(t[4] == 2 for t in tilings), tilings
    single = [p.forward()[0].clone() for p in plans]
    recs = batch.forward()
    torch.cuda.synchronize()
    assert batch.mode()[0]
    for r, r1 in zip(recs, single):
        assert torch.equal(r, r1)
    k = 2  # draw 3: 206 x 128 x 134, SO8
    w = works[k]
    rec_o, _, _ = oracle.forward(w.shape, w.spacing, w.so, w.dt, nt, w.m.astype(np.float64), src_xyz=w.src_xyz,
                                 wavelet=w.wavelet.astype(np.float32).astype(np.float64), rec_xyz=w.rec_xyz,
                                 sponge_width=w.sponge_width, sponge_faces=w.sponge_faces, vmax=w.vmax)
    assert_close(recs[k].cpu().numpy(), rec_o, 1e-5, "smallest full-size shot, persistent")
    batch.close()
    for p in plans:
        p.close()
