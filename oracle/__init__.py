"""FP64 oracle for the 3D acoustic wave path (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py`` (its cpu_baseline leg
and ``--impl reference``) may import this package.  The product package never
does, and this package never imports the product package.

The arithmetic lives in ``oracle.c`` (plain C, double precision); this module
only builds it and marshals numpy arrays through ctypes.  Each wrapper cites
the passage of McCormick 2017 ("Applying the Polyhedral Model to Tile Loops in
Devito") that the C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP on the outer loop only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("ox", ctypes.c_int), ("oy", ctypes.c_int), ("oz", ctypes.c_int),
        ("gnx", ctypes.c_int), ("gny", ctypes.c_int), ("gnz", ctypes.c_int),
        ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
        ("so", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("nt", ctypes.c_int),
        ("boundary", ctypes.c_int),
        ("sponge_width", ctypes.c_int),
        ("sponge_faces", ctypes.c_int),
        ("vmax", ctypes.c_double),
        ("m", ctypes.POINTER(ctypes.c_double)),
        ("nsrc", ctypes.c_int),
        ("src_xyz", ctypes.POINTER(ctypes.c_double)),
        ("wavelet", ctypes.POINTER(ctypes.c_double)),
        ("nrec", ctypes.c_int),
        ("rec_xyz", ctypes.POINTER(ctypes.c_double)),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_fd_weights.argtypes = [ctypes.c_int, _DP]
            lib.oracle_fd_weights.restype = ctypes.c_int
            for name, args in (
                ("oracle_damping", [ctypes.POINTER(Problem), _DP]),
                ("oracle_laplacian", [ctypes.POINTER(Problem), _DP, _DP]),
                ("oracle_forward", [ctypes.POINTER(Problem), _DP, _DP, _DP, _DP, _DP]),
                ("oracle_adjoint", [ctypes.POINTER(Problem), _DP, _DP]),
                ("oracle_gradient", [ctypes.POINTER(Problem), _DP, _DP, _DP]),
            ):
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_DP)


def _f64(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


class _Spec:
    """Keeps the numpy buffers alive while the C struct points at them."""

    def __init__(self, shape, spacing, so, dt, nt, m, *, src_xyz=None, wavelet=None, rec_xyz=None,
                 sponge_width=0, sponge_faces=0b101111, vmax=None, boundary=0,
                 origin=(0, 0, 0), global_shape=None):
        nx, ny, nz = (int(s) for s in shape)
        self.m = _f64(m).reshape(nx, ny, nz)
        self.src = _f64(np.zeros((0, 3)) if src_xyz is None else src_xyz).reshape(-1, 3)
        nsrc = self.src.shape[0]
        self.wav = _f64(np.zeros((max(nt, 0), nsrc)) if wavelet is None else wavelet).reshape(nt, nsrc) if nsrc else _f64(np.zeros(1))
        self.rec = _f64(np.zeros((0, 3)) if rec_xyz is None else rec_xyz).reshape(-1, 3)
        nrec = self.rec.shape[0]
        if vmax is None:
            vmax = float(np.max(1.0 / np.sqrt(self.m)))
        g = global_shape if global_shape is not None else (nx, ny, nz)
        self.s = Problem(nx, ny, nz, int(origin[0]), int(origin[1]), int(origin[2]),
                         int(g[0]), int(g[1]), int(g[2]),
                         float(spacing[0]), float(spacing[1]), float(spacing[2]),
                         int(so), float(dt), int(nt), int(boundary), int(sponge_width), int(sponge_faces),
                         float(vmax), _ptr(self.m), nsrc, _ptr(self.src) if nsrc else None,
                         _ptr(self.wav) if nsrc else None, nrec, _ptr(self.rec) if nrec else None)
        self.shape = (nx, ny, nz)
        self.nt, self.nsrc, self.nrec = nt, nsrc, nrec


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("%s failed with code %d" % (what, rc))


def fd_weights(so: int) -> np.ndarray:
    """Centred 2nd-derivative weights a_0..a_r of accuracy order ``so`` on unit
    spacing (Fornberg's recursion).  Fig. acoustic_devito prints them for SO=8
    scaled by 2dt^2/h^2."""
    lib = _load()
    out = np.zeros(so // 2 + 1)
    _check(lib.oracle_fd_weights(int(so), _ptr(out)), "oracle_fd_weights")
    return out


def damping(shape, spacing, *, sponge_width, sponge_faces=0b101111, vmax, origin=(0, 0, 0), global_shape=None):
    """Sponge damping d (1/ms) of every point (reading of the paper's ``damp``
    array, Fig. acoustic_devito, whose profile the paper does not give)."""
    lib = _load()
    spec = _Spec(shape, spacing, 8, 1.0, 0, np.ones(shape), sponge_width=sponge_width,
                 sponge_faces=sponge_faces, vmax=vmax, origin=origin, global_shape=global_shape)
    out = np.zeros(shape)
    _check(lib.oracle_damping(ctypes.byref(spec.s), _ptr(out)), "oracle_damping")
    return out


def laplacian(u, spacing, so, *, periodic=False):
    """L_h u with zero ghosts (or periodic wrap): the spatial part of the
    update in Fig. acoustic_devito."""
    lib = _load()
    u = _f64(u)
    spec = _Spec(u.shape, spacing, so, 1.0, 0, np.ones(u.shape), boundary=1 if periodic else 0)
    out = np.zeros(u.shape)
    _check(lib.oracle_laplacian(ctypes.byref(spec.s), _ptr(u), _ptr(out)), "oracle_laplacian")
    return out


def forward(shape, spacing, so, dt, nt, m, *, src_xyz=None, wavelet=None, rec_xyz=None,
            u_prev0=None, u_cur0=None, sponge_width=0, sponge_faces=0b101111, vmax=None,
            periodic=False, origin=(0, 0, 0), global_shape=None):
    """Leapfrog modelling, Fig. acoustic_devito's update applied nt times.

    Returns (rec [nt][nrec], u^{nt-1}, u^{nt})."""
    lib = _load()
    spec = _Spec(shape, spacing, so, dt, nt, m, src_xyz=src_xyz, wavelet=wavelet, rec_xyz=rec_xyz,
                 sponge_width=sponge_width, sponge_faces=sponge_faces, vmax=vmax,
                 boundary=1 if periodic else 0, origin=origin, global_shape=global_shape)
    up0 = _f64(u_prev0)
    uc0 = _f64(u_cur0)
    rec = np.zeros((nt, spec.nrec))
    up = np.zeros(spec.shape)
    uc = np.zeros(spec.shape)
    _check(lib.oracle_forward(ctypes.byref(spec.s), _ptr(up0), _ptr(uc0), _ptr(rec) if spec.nrec else None,
                              _ptr(up), _ptr(uc)), "oracle_forward")
    return rec, up, uc


def adjoint(shape, spacing, so, dt, nt, m, *, src_xyz, rec_xyz, resid, sponge_width=0,
            sponge_faces=0b101111, vmax=None):
    """Adjoint of wavelet -> receivers: injects ``resid`` [nt][nrec] at the
    receivers backwards in time and samples at the sources ([nt][nsrc])."""
    lib = _load()
    nsrc = np.asarray(src_xyz).reshape(-1, 3).shape[0]
    spec = _Spec(shape, spacing, so, dt, nt, m, src_xyz=src_xyz, wavelet=np.zeros((nt, nsrc)),
                 rec_xyz=rec_xyz, sponge_width=sponge_width, sponge_faces=sponge_faces, vmax=vmax)
    r = _f64(resid).reshape(nt, spec.nrec)
    out = np.zeros((nt, nsrc))
    _check(lib.oracle_adjoint(ctypes.byref(spec.s), _ptr(r), _ptr(out)), "oracle_adjoint")
    return out


def gradient(shape, spacing, so, dt, nt, m, *, src_xyz, wavelet, rec_xyz, d_obs, sponge_width=0,
             sponge_faces=0b101111, vmax=None):
    """Misfit J = 1/2 |rec - d_obs|^2 and dJ/dm (adjoint-state gradient)."""
    lib = _load()
    spec = _Spec(shape, spacing, so, dt, nt, m, src_xyz=src_xyz, wavelet=wavelet, rec_xyz=rec_xyz,
                 sponge_width=sponge_width, sponge_faces=sponge_faces, vmax=vmax)
    d = _f64(d_obs).reshape(nt, spec.nrec)
    g = np.zeros(spec.shape)
    J = ctypes.c_double(0.0)
    _check(lib.oracle_gradient(ctypes.byref(spec.s), _ptr(d), _ptr(g), ctypes.byref(J)), "oracle_gradient")
    return J.value, g
