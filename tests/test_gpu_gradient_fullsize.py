"""The FWI gradient at its full size (256^3, SO8, 800 steps, 10 Hz Ricker,
256 receivers on a line at 20 m, observed data from the true model of seed
3, start model = true velocity blurred with sigma = 10 cells, checkpoints
every 40 steps), in the tiling the benchmark's autotuner picks for it.

Central finite differences of the float32 misfit along a smooth model
perturbation agree with the adjoint-state gradient's directional derivative
<g, dm>, and the gradient does not depend on the checkpoint interval.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N, NT = 256, 800


def test_full_size_gradient_fd_check_and_checkpoint_invariance():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W
    from paper_1707_02347_gb300 import inputs

    W.load()
    dev = torch.device("cuda")
    w = inputs.layered_forward((N, N, N), 8, NT, seed=3, f=10.0, h=10.0, sponge_width=10, nrec_line=256)
    v_true = 1.0 / np.sqrt(w.m.astype(np.float64))
    v0 = inputs.gaussian_blur(v_true.astype(np.float32), 10.0) / inputs.gaussian_blur(np.ones(w.shape, np.float32), 10.0)
    m_true = torch.from_numpy(w.m).to(dev)
    m0_h = inputs.slowness2(v0).astype(np.float32)
    m0 = torch.from_numpy(m0_h).to(dev)
    plan = W.WavePlan(w.shape, w.spacing, 8, w.dt, NT, m_true, sponge_width=w.sponge_width, vmax=w.vmax,
                      tiling=(1, 16, 64, 64, 5))
    plan.set_sources(w.src_xyz, torch.from_numpy(w.wavelet.astype(np.float32)).to(dev))
    plan.set_receivers(w.rec_xyz)
    d_obs, _ = plan.forward()
    d_obs = d_obs.clone()
    plan.set_model(m0)
    J, g = plan.gradient(d_obs, checkpoint_every=40)
    g = g.clone()
    assert np.isfinite(J) and J > 0.0 and bool(torch.isfinite(g).all())
    # the checkpoint interval only changes what is recomputed
    J2, g2 = plan.gradient(d_obs, checkpoint_every=100)
    assert J2 == J and torch.equal(g2, g)
    # a smooth bump of 1 % in m, 400 m below the source and the receiver line
    x = np.arange(N, dtype=np.float64)
    c, s = (128.0, 128.0, 40.0), 12.0
    bump = (np.exp(-(x - c[0]) ** 2 / (2 * s * s))[:, None, None] *
            np.exp(-(x - c[1]) ** 2 / (2 * s * s))[None, :, None] *
            np.exp(-(x - c[2]) ** 2 / (2 * s * s))[None, None, :])
    dm = (0.01 * m0_h.astype(np.float64) * bump).astype(np.float32)
    dJ = float(np.sum(g.cpu().numpy().astype(np.float64) * dm.astype(np.float64)))
    dm_d = torch.from_numpy(dm).to(dev)
    plan.set_model(m0 + dm_d)
    Jp, _ = plan.gradient(d_obs, checkpoint_every=40)
    plan.set_model(m0 - dm_d)
    Jm, _ = plan.gradient(d_obs, checkpoint_every=40)
    fd = (Jp - Jm) / 2.0
    assert abs(dJ) > 1e-4 * J, (dJ, J)  # the bump moves the misfit
    rel = abs(fd - dJ) / abs(dJ)
    assert rel <= 1e-3, (fd, dJ, rel)  # measured: 1.6e-4
    plan.close()
