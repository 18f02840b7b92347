"""Parity after a workload's whole time loop, at a size where the tiles, x
slabs and sponge look like the benchmark's.

The 512^3 headline recipe (layered 1.5-4.5 km/s model with the seeded 5 %
blurred perturbation of seed 1, 15 Hz Ricker at 20 m depth, 10-cell sponge on
every face but the free surface, SO8, h = 10 m, 1000 steps) on a 256^3 grid,
with 256 receivers on a line at 20 m.  The GPU runs the tiling the autotuner
picks for this grid; the FP64 oracle runs the same 1000 steps on the whole
grid.  Compared element by element (tests/parity.py: relative L2 and the
per-element bound, both 1e-5): the last two fields u^{999}, u^{1000} and all
1000 trace rows.  The fastest one-step and the fastest time-tiled candidate
of the same sweep give the same bits (tiling only reorders independent
updates).
"""
import numpy as np
import pytest
from parity import assert_close

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N, NT = 256, 1000


def test_headline_recipe_full_nt_vs_oracle(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W
    from paper_1707_02347_gb300 import inputs

    W.load()
    dev = torch.device("cuda")
    w = inputs.layered_forward((N, N, N), 8, NT, seed=1, f=15.0, h=10.0, sponge_width=10, nrec_line=256)
    m = torch.from_numpy(np.ascontiguousarray(w.m)).to(dev)
    wav = torch.from_numpy(w.wavelet.astype(np.float32)).to(dev)
    plan = W.WavePlan(w.shape, w.spacing, 8, w.dt, NT, m, sponge_width=w.sponge_width,
                      sponge_faces=w.sponge_faces, vmax=w.vmax)
    plan.set_sources(w.src_xyz, wav)
    plan.set_receivers(w.rec_xyz)
    tuned = plan.autotune(passes=2)
    best = plan.get_tiling()
    rec, uf = plan.forward(want_final=True)
    torch.cuda.synchronize()
    rec, uf = rec.cpu().numpy(), uf.cpu().numpy()
    # the fastest candidate of the other kind (one-step vs time-tiled) gives the same bits
    others = [t for t, _ in sorted(tuned, key=lambda c: c[1]) if (t[0] >= 2) != (best[0] >= 2)]
    assert others, "the sweep timed no candidate of the other kind"
    plan.set_tiling(others[0])
    rec2, uf2 = plan.forward(want_final=True)
    torch.cuda.synchronize()
    assert np.array_equal(rec2.cpu().numpy(), rec), (best, others[0])
    assert np.array_equal(uf2.cpu().numpy(), uf), (best, others[0])
    plan.close()

    rec_o, up_o, uc_o = oracle.forward(w.shape, w.spacing, 8, w.dt, NT, w.m.astype(np.float64), src_xyz=w.src_xyz,
                                       wavelet=w.wavelet.astype(np.float32).astype(np.float64), rec_xyz=w.rec_xyz,
                                       sponge_width=w.sponge_width, sponge_faces=w.sponge_faces, vmax=w.vmax)
    assert np.abs(uc_o).max() > 0.0 and np.abs(rec_o).max() > 0.0
    assert_close(uf[1], uc_o, 1e-5, "u^1000 in tiling %s" % (best,))
    assert_close(uf[0], up_o, 1e-5, "u^999 in tiling %s" % (best,))
    assert_close(rec, rec_o, 1e-5, "traces in tiling %s" % (best,))
