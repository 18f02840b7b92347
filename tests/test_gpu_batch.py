"""Batched shots: uneven grids, SO 4 and 8 mixed, per-shot tilings, all
advanced by one CUDA graph launch -- bit-identical to running each plan's
wave_forward on its own, and correct against the FP64 oracle."""
import numpy as np
import pytest

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
        got = r.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    batch.close()
    for p in plans:
        p.close()
