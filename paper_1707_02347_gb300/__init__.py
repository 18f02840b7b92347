"""Time-tiled 3D acoustic wave propagation on GB300 (sm_103a).

Thin Python binding of libwave.so (include/wave.h): argument marshalling only.
Every step of the wave path runs in the library's CUDA kernels; PyTorch
provides device memory and the current stream.  There is no CPU fallback: if
the library is not built, or no CUDA device is present, calls raise.

The method is the one of McCormick 2017, "Applying the Polyhedral Model to
Tile Loops in Devito": the damped acoustic update of Fig. acoustic_devito,
time-tiled with spatial skew SO/2 per step (Chapter "Time-Tiling").
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = [
    "WaveError", "load", "fd_weights", "cfl_limit", "skew_factor", "tiling_check", "schedule_verify",
    "schedule_verify_custom", "schedule_verify_skew", "skewed_order_legal", "WavePlan", "WaveBatch", "FWIGradient", "STATUS",
]

STATUS = {0: "WAVE_OK", 1: "WAVE_ERR_ARG", 2: "WAVE_ERR_CFL", 3: "WAVE_ERR_OOM", 4: "WAVE_ERR_CUDA",
          5: "WAVE_ERR_TIMEOUT", 6: "WAVE_ERR_STATE"}


class WaveError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), message))
        self.status = status


class Tiling(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("by", ctypes.c_int), ("bz", ctypes.c_int), ("xc", ctypes.c_int),
                ("unroll", ctypes.c_int)]

    def as_tuple(self):
        return (self.T, self.by, self.bz, self.xc, self.unroll)


class Options(ctypes.Structure):
    _fields_ = [("sponge_width", ctypes.c_int), ("sponge_faces", ctypes.c_int), ("vmax", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("tiling", Tiling), ("autotune", ctypes.c_int), ("device", ctypes.c_int)]


_lock = threading.Lock()
_lib = None
_I3 = ctypes.c_int * 3
_D3 = ctypes.c_double * 3
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)


def load(build_if_missing: bool = True):
    """Load libwave.so from the package's _lib/ directory (building it first if
    it is missing and ``build_if_missing``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise WaveError(4, "libwave.so is not built (run __graft_entry__.build())")
            _build.build()
        lib = ctypes.CDLL(path)
        st = ctypes.c_int
        sig = {
            "wave_options_default": (st, [ctypes.POINTER(Options)]),
            "wave_fd_weights": (st, [ctypes.c_int, _DP]),
            "wave_cfl_limit": (st, [ctypes.c_int, _D3, ctypes.c_double, _DP]),
            "wave_plan_create": (st, [ctypes.POINTER(_VP), _I3, _D3, ctypes.c_int, ctypes.c_double, ctypes.c_int, _VP,
                                      ctypes.POINTER(Options)]),
            "wave_set_model": (st, [_VP, _VP]),
            "wave_set_sources": (st, [_VP, ctypes.c_int, _DP, _VP]),
            "wave_set_receivers": (st, [_VP, ctypes.c_int, _DP]),
            "wave_set_tiling": (st, [_VP, ctypes.POINTER(Tiling)]),
            "wave_get_tiling": (st, [_VP, ctypes.POINTER(Tiling)]),
            "wave_get_sweep_tiling": (st, [_VP, ctypes.POINTER(Tiling)]),
            "wave_autotune": (st, [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Tiling), _DP, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int)]),
            "wave_forward": (st, [_VP, _VP, _VP, _VP]),
            "wave_forward_host": (st, [_VP, _VP, _VP, _VP]),
            "wave_adjoint": (st, [_VP, _VP, _VP, _VP]),
            "wave_gradient": (st, [_VP, _VP, _VP, _DP, ctypes.c_int]),
            "wave_plan_destroy": (st, [_VP]),
            "wave_last_error": (ctypes.c_char_p, []),
            "wave_skew_factor": (ctypes.c_int, [ctypes.c_int]),
            "wave_tiling_check": (st, [_I3, ctypes.c_int, ctypes.POINTER(Tiling)]),
            "wave_schedule_verify": (st, [_I3, ctypes.c_int, ctypes.POINTER(Tiling)]),
            "wave_schedule_verify_custom": (st, [_I3, ctypes.c_int, ctypes.POINTER(Tiling), ctypes.c_int,
                                                 ctypes.c_int]),
            "wave_skewed_order_legal": (ctypes.c_int, [ctypes.c_int] * 6),
            "wave_schedule_verify_skew": (st, [_I3, ctypes.c_int, ctypes.POINTER(Tiling), ctypes.c_int,
                                               ctypes.c_int]),
            "wave_batch_create": (st, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP)]),
            "wave_autotune_cached": (st, [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
            "wave_batch_forward": (st, [_VP, ctypes.POINTER(_VP), _VP]),
            "wave_batch_gradient": (st, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _DP, ctypes.c_int, _VP]),
            "wave_batch_destroy": (st, [_VP]),
            "wave_batch_autotune": (st, [_VP, ctypes.c_int]),
            "wave_batch_get_mode": (st, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
            "wave_batch_selftest_withhold": (st, [_VP, ctypes.c_double]),
            "wave_selftest_timeout": (st, [ctypes.c_double]),
            "wave_profile_enable": (st, [_VP, ctypes.c_int]),
            "wave_profile_read": (st, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_longlong)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        msg = load().wave_last_error()
        raise WaveError(rc, msg.decode() if msg else "")


def fd_weights(so: int) -> np.ndarray:
    """Centred 2nd-derivative weights a_0..a_r of order ``so`` (exact rationals
    rounded to double; Fig. acoustic_devito prints SO 8 times 2dt^2/h^2)."""
    out = np.zeros(so // 2 + 1)
    _check(load().wave_fd_weights(int(so), out.ctypes.data_as(_DP)))
    return out


def cfl_limit(so: int, spacing, vmax: float) -> float:
    """Largest stable leapfrog dt (ms) for velocity vmax (km/s)."""
    out = ctypes.c_double(0.0)
    _check(load().wave_cfl_limit(int(so), _D3(*spacing), float(vmax), ctypes.byref(out)))
    return out.value


def skew_factor(so: int) -> int:
    return load().wave_skew_factor(int(so))


def _tiling(t) -> Tiling:
    if isinstance(t, Tiling):
        return t
    T, by, bz, xc, unroll = (tuple(t) + (0, 0, 0, 0, 0))[:5]
    return Tiling(int(T), int(by), int(bz), int(xc), int(unroll))


def tiling_check(grid, so: int, tiling) -> bool:
    return load().wave_tiling_check(_I3(*grid), int(so), ctypes.byref(_tiling(tiling))) == 0


def schedule_verify(grid, so: int, tiling):
    """(ok, message) of the brute-force legality check of the pass schedule."""
    lib = load()
    rc = lib.wave_schedule_verify(_I3(*grid), int(so), ctypes.byref(_tiling(tiling)))
    return rc == 0, (lib.wave_last_error() or b"").decode() if rc else ""


def schedule_verify_custom(grid, so: int, tiling, lag: int, halo_per_step: int):
    lib = load()
    rc = lib.wave_schedule_verify_custom(_I3(*grid), int(so), ctypes.byref(_tiling(tiling)), int(lag),
                                         int(halo_per_step))
    return rc == 0, (lib.wave_last_error() or b"").decode() if rc else ""


def schedule_verify_skew(grid, so: int, tiling, exchange_rows: int, wait_lead: int):
    """(ok, message) of the brute-force check of the skewed wavefront variant
    with its exchange rows and its progress wait overridden."""
    lib = load()
    rc = lib.wave_schedule_verify_skew(_I3(*grid), int(so), ctypes.byref(_tiling(tiling)), int(exchange_rows),
                                       int(wait_lead))
    return rc == 0, (lib.wave_last_error() or b"").decode() if rc else ""


def skewed_order_legal(n: int, nt: int, r: int, skew: int, tt: int, ts: int) -> bool:
    return bool(load().wave_skewed_order_legal(n, nt, r, skew, tt, ts))


def _torch():
    import torch

    return torch


def _dev_ptr(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float32 tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


class WavePlan:
    """A plan of libwave.so bound to the current CUDA device and stream.

    shape (nx, ny, nz), spacing (m), so in {4, 8, 16}, dt (ms), nt steps,
    m: CUDA float32 tensor [nx, ny, nz] of squared slowness (copied)."""

    def __init__(self, shape, spacing, so, dt, nt, m, *, sponge_width=10, sponge_faces=0x2F, vmax=0.0,
                 tiling=None, autotune=False, stream=None):
        torch = _torch()
        lib = load()
        self._lib = lib
        self.shape = tuple(int(s) for s in shape)
        self.spacing = tuple(float(h) for h in spacing)
        self.so, self.dt, self.nt = int(so), float(dt), int(nt)
        opt = Options()
        _check(lib.wave_options_default(ctypes.byref(opt)))
        opt.sponge_width = int(sponge_width)
        opt.sponge_faces = int(sponge_faces)
        opt.vmax = float(vmax)
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        opt.stream = ctypes.c_void_p(st.cuda_stream)
        opt.device = int(m.device.index if m.device.index is not None else torch.cuda.current_device())
        if tiling is not None:
            opt.tiling = _tiling(tiling)
        opt.autotune = 1 if autotune else 0
        self._m = m
        h = _VP()
        _check(lib.wave_plan_create(ctypes.byref(h), _I3(*self.shape), _D3(*self.spacing), self.so, self.dt, self.nt,
                                    _dev_ptr(m, "m"), ctypes.byref(opt)))
        self._h = h
        self.device = m.device
        self.nsrc = 0
        self.nrec = 0

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.wave_plan_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_model(self, m):
        _check(self._lib.wave_set_model(self._h, _dev_ptr(m, "m")))

    def set_sources(self, xyz, wavelet):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        if xyz.shape[0] == 0:
            _check(self._lib.wave_set_sources(self._h, 0, None, None))
        else:
            _check(self._lib.wave_set_sources(self._h, xyz.shape[0], xyz.ctypes.data_as(_DP),
                                              _dev_ptr(wavelet, "wavelet")))
        self.nsrc = xyz.shape[0]
        self._src = xyz

    def set_receivers(self, xyz):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        _check(self._lib.wave_set_receivers(self._h, xyz.shape[0], xyz.ctypes.data_as(_DP) if xyz.shape[0] else None))
        self.nrec = xyz.shape[0]
        self._rec = xyz

    def set_tiling(self, tiling):
        _check(self._lib.wave_set_tiling(self._h, ctypes.byref(_tiling(tiling))))

    def get_tiling(self):
        t = Tiling()
        _check(self._lib.wave_get_tiling(self._h, ctypes.byref(t)))
        return t.as_tuple()

    def get_sweep_tiling(self):
        """The one-step tiling of the plan's one-step sweeps (gradient recompute
        and adjoint sweeps, remainder steps)."""
        t = Tiling()
        _check(self._lib.wave_get_sweep_tiling(self._h, ctypes.byref(t)))
        return t.as_tuple()

    def autotune(self, passes=3, T_only=0, cap=256):
        cands = (Tiling * cap)()
        ms = (ctypes.c_double * cap)()
        n = ctypes.c_int(0)
        _check(self._lib.wave_autotune(self._h, int(passes), int(T_only), cands, ms, cap, ctypes.byref(n)))
        return [(cands[i].as_tuple(), ms[i]) for i in range(min(n.value, cap))]

    def autotune_cached(self, passes=3, T_only=0):
        """Autotune through the result cache (see wave_autotune_cached):
        returns (tiling, from_cache)."""
        hit = ctypes.c_int(0)
        _check(self._lib.wave_autotune_cached(self._h, int(passes), int(T_only), ctypes.byref(hit)))
        return self.get_tiling(), bool(hit.value)

    def forward(self, u_init=None, want_final=False, rec_out=None, u_final=None):
        """Run nt steps; returns (rec [nt, nrec], u_final [2, nx, ny, nz] or None)."""
        torch = _torch()
        if rec_out is None and self.nrec:
            rec_out = torch.empty((self.nt, self.nrec), dtype=torch.float32, device=self.device)
        if want_final and u_final is None:
            u_final = torch.empty((2,) + self.shape, dtype=torch.float32, device=self.device)
        _check(self._lib.wave_forward(self._h, _dev_ptr(u_init, "u_init") if u_init is not None else None,
                                      _dev_ptr(rec_out, "rec_out") if rec_out is not None else None,
                                      _dev_ptr(u_final, "u_final") if u_final is not None else None))
        return rec_out, u_final

    def forward_host(self, m_host, wavelet_host, rec_host):
        """The same as forward with numpy (ideally pinned) host arrays; copies inside."""
        def hp(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return ctypes.c_void_p(a.data_ptr())
            return a.ctypes.data_as(ctypes.c_void_p)
        _check(self._lib.wave_forward_host(self._h, hp(m_host), hp(wavelet_host), hp(rec_host)))
        return rec_host

    def adjoint(self, rec_resid, src_out=None, want_final=False, v_final=None):
        """Adjoint traces at the sources [nt, nsrc]; with want_final (or a
        given v_final) also the last two adjoint levels [2, nx, ny, nz]:
        returns src_out, or (src_out, v_final) when a final field is asked."""
        torch = _torch()
        if src_out is None:
            src_out = torch.empty((self.nt, self.nsrc), dtype=torch.float32, device=self.device)
        if want_final and v_final is None:
            v_final = torch.empty((2,) + self.shape, dtype=torch.float32, device=self.device)
        _check(self._lib.wave_adjoint(self._h, _dev_ptr(rec_resid, "rec_resid"), _dev_ptr(src_out, "src_out"),
                                      _dev_ptr(v_final, "v_final") if v_final is not None else None))
        return (src_out, v_final) if v_final is not None else src_out

    def gradient(self, d_obs, checkpoint_every=0, grad_out=None):
        """(misfit J, dJ/dm [nx, ny, nz]) for observed traces d_obs [nt, nrec]."""
        torch = _torch()
        if grad_out is None:
            grad_out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        J = ctypes.c_double(0.0)
        _check(self._lib.wave_gradient(self._h, _dev_ptr(d_obs, "d_obs"), _dev_ptr(grad_out, "grad_m"),
                                       ctypes.byref(J), int(checkpoint_every)))
        return J.value, grad_out


class WaveBatch:
    """Several plans (shots) advanced together, one graph launch per call: the
    forward of every shot in one persistent kernel fed by a device work queue
    (when every plan's tiling has a shape in it; else one stream per shot),
    the gradient as every shot's launches, one stream per shot."""

    def __init__(self, plans):
        self._lib = load()
        self.plans = list(plans)
        arr = (_VP * len(self.plans))(*[p._h for p in self.plans])
        h = _VP()
        _check(self._lib.wave_batch_create(ctypes.byref(h), len(self.plans), arr))
        self._h = h

    def autotune(self, passes=2):
        """Tune every plan over the tilings the persistent batched kernel runs."""
        _check(self._lib.wave_batch_autotune(self._h, int(passes)))
        return [p.get_tiling() for p in self.plans]

    def mode(self):
        """(persistent, work items, thread blocks) of the captured forward."""
        a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(self._lib.wave_batch_get_mode(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return bool(a.value), b.value, c.value

    def selftest_withhold(self, limit_ms=100.0):
        """Status code of wave_batch_selftest_withhold (5 = WAVE_ERR_TIMEOUT, the expected one)."""
        return int(self._lib.wave_batch_selftest_withhold(self._h, float(limit_ms)))

    def forward(self, recs=None):
        """recs: one CUDA tensor [nt, nrec] per plan (allocated if None)."""
        torch = _torch()
        if recs is None:
            recs = [torch.empty((p.nt, p.nrec), dtype=torch.float32, device=p.device) if p.nrec else None
                    for p in self.plans]
        ptrs = (_VP * len(self.plans))(*[None if r is None else r.data_ptr() for r in recs])
        _check(self._lib.wave_batch_forward(self._h, ptrs, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
        return recs

    def gradient(self, d_obs, checkpoint_every=0, grads=None):
        """FWI gradient of every shot in one graph launch.  d_obs: one CUDA
        tensor [nt, nrec] per plan; returns (misfits, grads), grads one CUDA
        tensor of the grid shape per plan (allocated if None)."""
        torch = _torch()
        n = len(self.plans)
        if len(d_obs) != n:
            raise ValueError("one d_obs per plan")
        for p, d in zip(self.plans, d_obs):
            _dev_ptr(d, "d_obs")
            if tuple(d.shape) != (p.nt, p.nrec):
                raise ValueError("d_obs shape %s, expected %s" % (tuple(d.shape), (p.nt, p.nrec)))
        if grads is None:
            grads = [torch.empty(p.shape, dtype=torch.float32, device=p.device) for p in self.plans]
        obs = (_VP * n)(*[d.data_ptr() for d in d_obs])
        gp = (_VP * n)(*[_dev_ptr(g, "grad") for g in grads])
        mis = (ctypes.c_double * n)()
        _check(self._lib.wave_batch_gradient(self._h, obs, gp, mis, int(checkpoint_every),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
        return list(mis), grads

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.wave_batch_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_fwi_function():
    torch = _torch()

    class FWIGradient(torch.autograd.Function):
        """J(m) = 1/2 |rec(m) - d_obs|^2 with the adjoint-state gradient of
        libwave.so as its backward: FWIGradient.apply(m, plan, d_obs, K)."""

        @staticmethod
        def forward(ctx, m, plan, d_obs, checkpoint_every=0):
            plan.set_model(m.detach().contiguous())
            J, g = plan.gradient(d_obs, checkpoint_every)
            ctx.save_for_backward(g)
            return m.new_tensor(J)

        @staticmethod
        def backward(ctx, gJ):
            (g,) = ctx.saved_tensors
            return gJ * g, None, None, None

    return FWIGradient


class _LazyFWI:
    _cls = None

    def __getattr__(self, item):
        if _LazyFWI._cls is None:
            _LazyFWI._cls = _make_fwi_function()
        return getattr(_LazyFWI._cls, item)


FWIGradient = _LazyFWI()
