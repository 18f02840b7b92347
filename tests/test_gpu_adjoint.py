"""GPU adjoint and FWI gradient (through the C ABI) against the FP64 oracle.

* dot-product test <P q, d> = <q, P^T d> with FP64 inner products of the FP32
  traces, relative mismatch <= 1e-6, for random q and d and for d = P q;
* the final adjoint field equals the forward field of the swapped problem
  (receivers as sources, time-reversed residual) and matches the oracle;
* adjoint traces and gradient vs the oracle's (relative L2);
* the gradient does not depend on the checkpoint interval (bit-identical:
  the recompute uses the one-step kernel, bit-identical to the tiled one),
  nor on the schedule (the recompute overlapped with the adjoint sweep, or
  serial);
* the gradient matches central finite differences of the FP64 oracle misfit
  at 16 seeded cells;
* FWIGradient (torch.autograd.Function) returns the same gradient.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W

    W.load()
    return W


from parity import assert_close


def problem(seed=3, shape=(34, 30, 28), so=8, nt=90):
    from paper_1707_02347_gb300 import inputs

    h = (10.0, 10.0, 10.0)
    rng = np.random.default_rng(seed)
    v = inputs.velocity_model(shape, seed, vmin=1.5, vmax=3.0, sigma=3.0)
    m_true = inputs.slowness2(v)
    vs = inputs.gaussian_blur(v, 4.0) / inputs.gaussian_blur(np.ones(shape, np.float32), 4.0)
    m0 = inputs.slowness2(vs)
    vmax = 3.2
    dt = inputs.cfl_dt(so, h, vmax, 0.8)
    src = np.array([[120.0, 145.5, 40.0], [200.0, 100.0, 60.0]])
    wav = np.stack([inputs.ricker(nt, dt, 30.0), 0.5 * inputs.ricker(nt, dt, 25.0, 60.0)], axis=1)
    rec = inputs.line_receivers(shape, h, 12, 30.0)
    return dict(shape=shape, h=h, so=so, nt=nt, dt=dt, m_true=m_true, m0=m0, src=src, wav=wav, rec=rec, vmax=vmax,
                sponge=dict(sponge_width=5, sponge_faces=0b101111), rng=rng)


def plan_for(W, P, m, tiling=(2, 24, 24, 34)):
    dev = torch.device("cuda")
    mt = torch.from_numpy(np.ascontiguousarray(m, np.float32)).to(dev)
    plan = W.WavePlan(P["shape"], P["h"], P["so"], P["dt"], P["nt"], mt, vmax=P["vmax"], tiling=tiling,
                      **P["sponge"])
    plan.set_sources(P["src"], torch.from_numpy(P["wav"].astype(np.float32)).to(dev))
    plan.set_receivers(P["rec"])
    return plan


def oracle_kw(P):
    return dict(sponge_width=P["sponge"]["sponge_width"], sponge_faces=P["sponge"]["sponge_faces"], vmax=P["vmax"])


def test_adjoint_dot_product_and_oracle(W, oracle):
    P = problem()
    plan = plan_for(W, P, P["m0"])
    rng = np.random.default_rng(11)
    q = rng.standard_normal((P["nt"], 2)).astype(np.float32)
    d = rng.standard_normal((P["nt"], P["rec"].shape[0])).astype(np.float32)
    dev = torch.device("cuda")
    plan.set_sources(P["src"], torch.from_numpy(q).to(dev))
    Pq, _ = plan.forward()
    PTd = plan.adjoint(torch.from_numpy(d).to(dev))
    torch.cuda.synchronize()
    Pq, PTd = Pq.cpu().numpy().astype(np.float64), PTd.cpu().numpy().astype(np.float64)
    lhs = float(np.sum(Pq * d))
    rhs = float(np.sum(q.astype(np.float64) * PTd))
    # random q and d: the relative mismatch of the two inner products
    rel = abs(lhs - rhs) / abs(lhs)
    assert rel <= 1e-6, ("random-vector dot-product test", lhs, rhs, rel)
    # correlated data d = P q: no cancellation, plain relative mismatch
    d2 = Pq.astype(np.float32)
    PTd2 = plan.adjoint(torch.from_numpy(d2).to(dev))
    torch.cuda.synchronize()
    PTd2 = PTd2.cpu().numpy().astype(np.float64)
    lhs2 = float(np.sum(Pq * d2))
    rhs2 = float(np.sum(q.astype(np.float64) * PTd2))
    assert abs(lhs2 - rhs2) <= 1e-6 * abs(lhs2), (lhs2, rhs2)
    ref = oracle.adjoint(P["shape"], P["h"], P["so"], P["dt"], P["nt"], P["m0"].astype(np.float64), src_xyz=P["src"],
                         rec_xyz=P["rec"], resid=d.astype(np.float64), **oracle_kw(P))
    assert_close(PTd, ref, 1e-5, "adjoint traces")
    plan.close()


def test_adjoint_final_field(W, oracle):
    """v_final of wave_adjoint: the adjoint sweep is the forward update run on
    the time-reversed residual with receivers and sources swapping roles, so
    its last two levels equal, bit for bit, u_final of a forward plan of that
    swapped problem in the same tiling, and match the FP64 oracle's forward
    run of it."""
    P = problem()
    dev = torch.device("cuda")
    rng = np.random.default_rng(13)
    d = rng.standard_normal((P["nt"], P["rec"].shape[0])).astype(np.float32)
    for tiling in ((2, 24, 24, 34), (1, 16, 64, 34, 5)):
        plan = plan_for(W, P, P["m0"], tiling=tiling)
        src_a, vf = plan.adjoint(torch.from_numpy(d).to(dev), want_final=True)
        torch.cuda.synchronize()
        vf = vf.cpu().numpy()
        plan.close()
        swapped = dict(P, src=P["rec"], rec=P["src"], wav=d[::-1].astype(np.float64))
        sp = plan_for(W, swapped, P["m0"], tiling=tiling)
        _, uf = sp.forward(want_final=True)
        torch.cuda.synchronize()
        uf = uf.cpu().numpy()
        sp.close()
        assert np.array_equal(vf, uf), tiling
        assert np.abs(vf[1]).max() > 0.0
    _, up_o, uc_o = oracle.forward(P["shape"], P["h"], P["so"], P["dt"], P["nt"], P["m0"].astype(np.float64),
                                   src_xyz=P["rec"], wavelet=d[::-1].astype(np.float64), **oracle_kw(P))
    assert_close(vf[1], uc_o, 1e-5, "final adjoint level")
    assert_close(vf[0], up_o, 1e-5, "level before the final adjoint level")


def test_gradient_vs_oracle_and_checkpointing(W, oracle):
    P = problem()
    ok = oracle_kw(P)
    d_obs, _, _ = oracle.forward(P["shape"], P["h"], P["so"], P["dt"], P["nt"], P["m_true"].astype(np.float64),
                                 src_xyz=P["src"], wavelet=P["wav"], rec_xyz=P["rec"], **ok)
    J_o, g_o = oracle.gradient(P["shape"], P["h"], P["so"], P["dt"], P["nt"], P["m0"].astype(np.float64),
                               src_xyz=P["src"], wavelet=P["wav"], rec_xyz=P["rec"], d_obs=d_obs, **ok)
    plan = plan_for(W, P, P["m0"])
    dobs_t = torch.from_numpy(d_obs.astype(np.float32)).cuda()
    J, g = plan.gradient(dobs_t, checkpoint_every=0)
    g = g.cpu().numpy()
    assert J == pytest.approx(J_o, rel=1e-4)
    assert_close(g, g_o, 1e-4, "gradient")
    for K in (7, 40, P["nt"]):
        J2, g2 = plan.gradient(dobs_t, checkpoint_every=K)
        assert J2 == J
        assert np.array_equal(g2.cpu().numpy(), g), K
    plan.close()


def test_gradient_overlapped_schedule_bit_identical(W, oracle, monkeypatch):
    """The recompute of one segment on the plan's second stream, overlapped
    with the adjoint sweep of the next (two segment buffers), gives the
    serial schedule's misfit and gradient bit for bit, single and batched."""
    P = problem(nt=50)
    ok = oracle_kw(P)
    d_obs, _, _ = oracle.forward(P["shape"], P["h"], P["so"], P["dt"], P["nt"], P["m_true"].astype(np.float64),
                                 src_xyz=P["src"], wavelet=P["wav"], rec_xyz=P["rec"], **ok)
    dobs_t = torch.from_numpy(d_obs.astype(np.float32)).cuda()
    out = {}
    for serial in ("1", "0"):
        monkeypatch.setenv("WAVE_GRADIENT_SERIAL", serial)
        plan = plan_for(W, P, P["m0"])
        J, g = plan.gradient(dobs_t, checkpoint_every=6)
        b = W.WaveBatch([plan])
        Jb, gb = b.gradient([dobs_t], checkpoint_every=6)
        out[serial] = (J, g.clone(), Jb[0], gb[0].clone())
        b.close()
        plan.close()
    assert out["0"][0] == out["1"][0] == out["0"][2] == out["1"][2]
    assert torch.equal(out["0"][1], out["1"][1])
    assert torch.equal(out["0"][1], out["0"][3])
    assert torch.equal(out["1"][1], out["1"][3])


def test_gradient_central_differences_16_cells(W, oracle):
    P = problem(nt=70)
    ok = oracle_kw(P)
    d_obs, _, _ = oracle.forward(P["shape"], P["h"], P["so"], P["dt"], P["nt"], P["m_true"].astype(np.float64),
                                 src_xyz=P["src"], wavelet=P["wav"], rec_xyz=P["rec"], **ok)
    plan = plan_for(W, P, P["m0"])
    J, g = plan.gradient(torch.from_numpy(d_obs.astype(np.float32)).cuda(), checkpoint_every=10)
    g = g.cpu().numpy()
    plan.close()
    # 16 seeded interior cells inside the illuminated region
    rng = np.random.default_rng(4)
    cells = set()
    while len(cells) < 16:
        c = (int(rng.integers(6, 28)), int(rng.integers(6, 24)), int(rng.integers(2, 12)))
        cells.add(c)
    m0 = P["m0"].astype(np.float64)
    scale = np.abs(g).max()
    for c in sorted(cells):
        eps = 1e-4 * m0[c]
        mp, mn = m0.copy(), m0.copy()
        mp[c] += eps
        mn[c] -= eps
        rp, _, _ = oracle.forward(P["shape"], P["h"], P["so"], P["dt"], P["nt"], mp, src_xyz=P["src"],
                                  wavelet=P["wav"], rec_xyz=P["rec"], **ok)
        rn, _, _ = oracle.forward(P["shape"], P["h"], P["so"], P["dt"], P["nt"], mn, src_xyz=P["src"],
                                  wavelet=P["wav"], rec_xyz=P["rec"], **ok)
        fd = (0.5 * np.sum((rp - d_obs) ** 2) - 0.5 * np.sum((rn - d_obs) ** 2)) / (2 * eps)
        assert abs(g[c] - fd) <= 1e-3 * abs(fd) + 1e-4 * scale, (c, g[c], fd)


def test_fwi_autograd_function(W, oracle):
    P = problem(nt=50)
    ok = oracle_kw(P)
    d_obs, _, _ = oracle.forward(P["shape"], P["h"], P["so"], P["dt"], P["nt"], P["m_true"].astype(np.float64),
                                 src_xyz=P["src"], wavelet=P["wav"], rec_xyz=P["rec"], **ok)
    plan = plan_for(W, P, P["m0"])
    dobs_t = torch.from_numpy(d_obs.astype(np.float32)).cuda()
    J_ref, g_ref = plan.gradient(dobs_t)
    g_ref = g_ref.clone()
    m = torch.from_numpy(P["m0"].astype(np.float32)).cuda().requires_grad_(True)
    J = W.FWIGradient.apply(m, plan, dobs_t, 0)
    J.backward()
    assert float(J.detach()) == pytest.approx(J_ref, rel=1e-7)
    assert torch.equal(m.grad, g_ref)
    plan.close()


@pytest.mark.parametrize("tiling", [(2, 28, 56, 34, 4), (2, 24, 56, 34, 2), (1, 8, 64, 34, 2), (2, 24, 56, 34, 5),
                                    (2, 36, 56, 34, 7)])
def test_gradient_independent_of_pass_variant(W, oracle, tiling):
    """The gradient runs its forward and adjoint sweeps with the plan's
    tiling: the skewed wavefront variant, the tensor-memory T = 2 pass, the
    warp-specialised T = 2 pass and the one-step pass all give the register
    one-step plan's gradient bit for bit."""
    P = problem(nt=40)
    ok = oracle_kw(P)
    d_obs, _, _ = oracle.forward(P["shape"], P["h"], P["so"], P["dt"], P["nt"], P["m_true"].astype(np.float64),
                                 src_xyz=P["src"], wavelet=P["wav"], rec_xyz=P["rec"], **ok)
    dobs_t = torch.from_numpy(d_obs.astype(np.float32)).cuda()
    ref = plan_for(W, P, P["m0"], tiling=(1, 16, 64, 34))
    J_ref, g_ref = ref.gradient(dobs_t, checkpoint_every=9)
    g_ref = g_ref.clone()
    rec_a = ref.adjoint(dobs_t).clone()
    ref.close()
    plan = plan_for(W, P, P["m0"], tiling=tiling)
    J, g = plan.gradient(dobs_t, checkpoint_every=9)
    assert J == J_ref
    assert torch.equal(g, g_ref)
    assert torch.equal(plan.adjoint(dobs_t), rec_a)
    plan.close()
