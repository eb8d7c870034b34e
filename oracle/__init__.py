"""CPU oracle for the sparse D3Q19 TRT path: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library
(``paper_1111_1129_gb300``) never imports, links or calls it, and the two
share no code.

The arithmetic lives in ``lbm_oracle.c`` (plain FP64 C, OpenMP over
cells), compiled with gcc on first use; this module only marshals numpy
arrays.  Dense arrays are laid out like the flags, ``[nz, ny, nx]`` with x
fastest, and PDFs as ``[19, nz, ny, nx]``.

Every function is pinned by a ``-m "not gpu"`` test against closed forms
or brute force (Poiseuille channel and duct, conservation in a collision,
equilibrium moments, uniform acceleration, mirror symmetry, Morton order
by octant recursion, blocking invariants, adjoint vs finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

ORDER_LEX, ORDER_BLOCKED, ORDER_MORTON1, ORDER_MORTON2, ORDER_HILBERT = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile ``liblbm_oracle.so`` (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32, i64, u32, d = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                    ctypes.c_uint32, ctypes.c_double)
            lib.oracle_velocity_set.argtypes = [vp, vp, vp]
            lib.oracle_velocity_set.restype = None
            lib.oracle_keys.argtypes = [i32, vp, vp, vp]
            lib.oracle_keys.restype = None
            lib.oracle_count_fluid.argtypes = [vp, vp]
            lib.oracle_count_fluid.restype = i64
            lib.oracle_build_sparse.argtypes = [vp, vp, i32, vp, u32, vp, vp, vp]
            lib.oracle_build_sparse.restype = i64
            lib.oracle_collide.argtypes = [vp, vp, d, d, d, vp, vp, vp]
            lib.oracle_collide.restype = None
            lib.oracle_rest_state.argtypes = [vp, vp, vp]
            lib.oracle_rest_state.restype = None
            lib.oracle_run.argtypes = [vp, vp, u32, d, d, vp, vp, i32, vp, vp, vp, vp]
            lib.oracle_run.restype = ctypes.c_int
            lib.oracle_adjoint.argtypes = [vp, vp, u32, d, d, vp, vp, i32, i32, vp, vp, vp, vp,
                                           vp]
            lib.oracle_adjoint.restype = ctypes.c_int
            lib.oracle_sparse_step.argtypes = [vp, vp, vp, i64, vp, vp, d, d]
            lib.oracle_sparse_step.restype = None
            _lib = lib
    return _lib


def _dims(flags):
    nz, ny, nx = flags.shape
    return np.array([nx, ny, nz], dtype=np.int32)


def _flags(flags):
    return np.ascontiguousarray(flags, dtype=np.uint8)


def velocity_set():
    """(c [19,3] int32, w [19] float64, opp [19] int32)."""
    c = np.empty((19, 3), np.int32)
    w = np.empty(19, np.float64)
    opp = np.empty(19, np.int32)
    _load().oracle_velocity_set(_p(c), _p(w), _p(opp))
    return c, w, opp


def keys(kind: int, dims, block=(1, 1, 1)) -> np.ndarray:
    """Numbering-scheme key I(x,y,z) of every box cell, shape [nz, ny, nx]."""
    d = np.array(dims, np.int32)
    b = np.array(block, np.int32)
    out = np.empty(int(d[2]) * int(d[1]) * int(d[0]), np.uint64)
    _load().oracle_keys(int(kind), _p(d), _p(b), _p(out))
    return out.reshape(int(d[2]), int(d[1]), int(d[0]))


def build_sparse(flags, kind: int = ORDER_LEX, block=(1, 1, 1), periodic: int = 0):
    """(cells [N] int32, inv [nz,ny,nx] int32, adj [18,N] int32)."""
    flags = _flags(flags)
    d = _dims(flags)
    b = np.array(block, np.int32)
    lib = _load()
    n = lib.oracle_count_fluid(_p(flags), _p(d))
    cells = np.empty(max(n, 1), np.int32)
    inv = np.empty(flags.shape, np.int32)
    adj = np.empty((18, max(n, 1)), np.int32)
    got = lib.oracle_build_sparse(_p(flags), _p(d), int(kind), _p(b), int(periodic), _p(cells),
                                  _p(inv), _p(adj))
    if got != n:
        raise RuntimeError("oracle_build_sparse failed")
    return cells[:n].copy(), inv, np.ascontiguousarray(adj[:, :n])


def collide(g, F, alpha: float, omega_p: float, omega_m: float):
    """One TRT collision: (f* [19], rho, u [3])."""
    g = np.ascontiguousarray(g, np.float64)
    F = np.ascontiguousarray(F, np.float64)
    fo = np.empty(19)
    rho = ctypes.c_double(0.0)
    u = np.empty(3)
    _load().oracle_collide(_p(g), _p(F), float(alpha), float(omega_p), float(omega_m), _p(fo),
                           ctypes.byref(rho), _p(u))
    return fo, rho.value, u


def rest_state(flags) -> np.ndarray:
    flags = _flags(flags)
    f = np.empty((19,) + flags.shape)
    _load().oracle_rest_state(_p(flags), _p(_dims(flags)), _p(f))
    return f


def run(flags, periodic: int, omega_p: float, omega_m: float, F, n_steps: int, alpha=None,
        f=None):
    """``n_steps`` steps from ``f`` (dense [19,nz,ny,nx], default rest).

    Returns (f, obs [n_steps, 4] = (sum rho, sum u_x, sum u_y, sum u_z) per
    step, rho [nz,ny,nx] and u [3,nz,ny,nx] of the last step's collision)."""
    flags = _flags(flags)
    f = rest_state(flags) if f is None else np.array(f, np.float64, copy=True, order="C")
    F = np.ascontiguousarray(F, np.float64)
    a = None if alpha is None else np.ascontiguousarray(alpha, np.float64)
    obs = np.zeros((max(n_steps, 1), 4))
    rho = np.zeros(flags.shape)
    u = np.zeros((3,) + flags.shape)
    rc = _load().oracle_run(_p(flags), _p(_dims(flags)), int(periodic), float(omega_p),
                            float(omega_m), _p(F), _p(a), int(n_steps), _p(f), _p(obs), _p(rho),
                            _p(u))
    if rc != 0:
        raise RuntimeError("oracle_run failed")
    return f, obs[:n_steps], rho, u


def adjoint(flags, periodic: int, omega_p: float, omega_m: float, F, n_steps: int, axis: int,
            alpha=None, f0=None):
    """J = mean u_axis of step ``n_steps`` and its gradients:
    (J, dJ/dF [3], dJ/dalpha [nz,ny,nx], dJ/df0 [19,nz,ny,nx])."""
    flags = _flags(flags)
    f0 = rest_state(flags) if f0 is None else np.ascontiguousarray(f0, np.float64)
    F = np.ascontiguousarray(F, np.float64)
    a = None if alpha is None else np.ascontiguousarray(alpha, np.float64)
    J = ctypes.c_double(0.0)
    dF = np.zeros(3)
    da = np.zeros(flags.shape)
    lam0 = np.zeros((19,) + flags.shape)
    rc = _load().oracle_adjoint(_p(flags), _p(_dims(flags)), int(periodic), float(omega_p),
                                float(omega_m), _p(F), _p(a), int(n_steps), int(axis), _p(f0),
                                ctypes.byref(J), _p(dF), _p(da), _p(lam0))
    if rc != 0:
        raise RuntimeError("oracle_adjoint failed")
    return J.value, dF, da, lam0


def omega_minus(omega_p: float, magic: float = 3.0 / 16.0) -> float:
    """omega- from omega+ and the TRT magic parameter
    Lambda = (1/omega+ - 1/2)(1/omega- - 1/2)."""
    return 1.0 / (0.5 + magic / (1.0 / omega_p - 0.5))


def to_sparse(dense, cells) -> np.ndarray:
    """Gather a dense [..., nz, ny, nx] field onto the fluid-cell list."""
    lead = dense.shape[:-3]
    return dense.reshape(lead + (-1,))[..., cells]


def sparse_step(f_src, adj, n: int, F, omega_p: float, omega_m: float, alpha=None):
    """One step on a sparse list: f_src is 1-D (19 n own PDFs, possibly
    followed by ghosts), adj [18, n] indexes it; returns f_dst [19 * n]."""
    f_src = np.ascontiguousarray(f_src, np.float64).ravel()
    adj = np.ascontiguousarray(adj, np.int32)
    F = np.ascontiguousarray(F, np.float64)
    a = None if alpha is None else np.ascontiguousarray(alpha, np.float64)
    out = np.empty(19 * int(n))
    _load().oracle_sparse_step(_p(f_src), _p(out), _p(adj), int(n), _p(F), _p(a),
                               float(omega_p), float(omega_m))
    return out
