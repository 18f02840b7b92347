"""The allocation-free receiver sampling entry point (wave_sample_noalloc).

Called straight through the C ABI (ctypes), twice in a row on different
fields and receiver sets, and compared bit for bit with the traces the
plan's wave_forward records for the same fields.  Its slots live in a static device
array shared by all calls, so the second call also checks that nothing from
the first one leaks into it.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu



def _run_forward(W, shape, nt, seed, nrec):
    from paper_1707_02347_gb300 import inputs

    w = inputs.layered_forward(shape, 8, nt, seed=seed, f=25.0, h=10.0, sponge_width=4, nrec_line=nrec)
    # receivers off the grid points, one on the far corner
    rng = np.random.default_rng(seed)
    extra = rng.uniform(0.0, 1.0, (5, 3)) * (np.array(shape) - 1) * 10.0
    w.rec_xyz = np.vstack([w.rec_xyz, extra, [[(shape[0] - 1) * 10.0, (shape[1] - 1) * 10.0, (shape[2] - 1) * 10.0]]])
    dev = torch.device("cuda")
    m = torch.from_numpy(np.ascontiguousarray(w.m)).to(dev)
    plan = W.WavePlan(shape, w.spacing, 8, w.dt, nt, m, sponge_width=w.sponge_width, vmax=w.vmax,
                      tiling=(2, 16, 56, 40))
    plan.set_sources(w.src_xyz, torch.from_numpy(w.wavelet.astype(np.float32)).to(dev))
    plan.set_receivers(w.rec_xyz)
    rec, uf = plan.forward(want_final=True)
    torch.cuda.synchronize()
    plan.close()
    return w, rec, uf


def _noalloc(lib, shape, spacing, u, xyz):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    out = torch.full((xyz.shape[0],), float("nan"), dtype=torch.float32, device=u.device)
    rc = lib.wave_sample_noalloc((ctypes.c_int * 3)(*shape), (ctypes.c_double * 3)(*spacing),
                                 ctypes.c_void_p(u.data_ptr()), xyz.shape[0],
                                 xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.c_void_p(out.data_ptr()), None)
    torch.cuda.synchronize()
    return rc, out.cpu().numpy()


def test_noalloc_sampling_matches_forward_traces_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W

    lib = W.load()
    lib.wave_sample_noalloc.restype = ctypes.c_int
    lib.wave_sample_noalloc.argtypes = [ctypes.c_int * 3, ctypes.c_double * 3, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p]
    # two different problems, the second with fewer receivers than the first
    for shape, nt, seed, nrec in (((36, 30, 28), 24, 5, 40), ((30, 34, 26), 17, 6, 9)):
        w, rec, uf = _run_forward(W, shape, nt, seed, nrec)
        rc, got = _noalloc(lib, shape, w.spacing, uf[1].contiguous(), w.rec_xyz)
        assert rc == 0, lib.wave_last_error()
        want = rec[-1].cpu().numpy()  # trace row nt-1 samples u^{nt}
        assert np.all(np.isfinite(got))
        assert np.abs(want).max() > 0.0
        # the same taps, weights and summation order as the forward traces
        assert np.array_equal(got, want)


def test_noalloc_rejects_positions_outside_the_grid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W

    lib = W.load()
    lib.wave_sample_noalloc.restype = ctypes.c_int
    u = torch.zeros((6, 5, 4), dtype=torch.float32, device="cuda")
    for bad in ([float("nan"), 1.0, 1.0], [1.0, float("inf"), 1.0], [-0.5, 1.0, 1.0], [1.0, 1.0, 3.5]):
        rc, _ = _noalloc(lib, (6, 5, 4), (1.0, 1.0, 1.0), u, np.array([[1.0, 1.0, 1.0], bad]))
        assert rc == 1, bad  # WAVE_ERR_ARG
        assert b"position 1" in lib.wave_last_error()


def test_noalloc_rejects_too_many_receivers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1707_02347_gb300 as W

    lib = W.load()
    lib.wave_sample_noalloc.restype = ctypes.c_int
    u = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    xyz = np.zeros((65537, 3))
    rc, _ = _noalloc(lib, (4, 4, 4), (1.0, 1.0, 1.0), u, xyz)
    assert rc == 1  # WAVE_ERR_ARG
    assert b"65536" in lib.wave_last_error()
