"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module only generates inputs (voxel flags of packed beds, uniform random
fields, batch parameters).  It contains none of the lattice Boltzmann
arithmetic.  The geometries stand in for the paper's benchmark geometries,
the empty "channel" and the sphere "packing" in a tube of size (5d) x d x d
(Sec. 6, Fig. 2), which are not available; only their shape family and fluid
fractions are reproduced (the paper quotes ~0.96 and ~0.42 fluid fraction
for 500x100x100, Sec. 7).

The generator is plain C (``packed_bed.c``), compiled on first use with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "packed_bed.c")
_LIB = os.path.join(_HERE, "libpacked_bed.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator into ``libpacked_bed.so`` next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.pb_uniform.restype = ctypes.c_double
            lib.pb_uniform.argtypes = [ctypes.c_uint64] * 3
            lib.pb_uniform_field.restype = None
            lib.pb_uniform_field.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
            lib.pb_packed_bed.restype = ctypes.c_int
            lib.pb_packed_bed.argtypes = [ctypes.c_int32] * 4 + [ctypes.c_double] * 3 + [
                ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            _lib = lib
    return _lib


def uniform(n: int, seed: int, stream: int = 0, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``n`` uniform doubles in [lo, hi) from the counter-based generator."""
    out = np.empty(int(n), dtype=np.float64)
    _load().pb_uniform_field(int(n), int(seed), int(stream), float(lo), float(hi),
                             out.ctypes.data)
    return out


@dataclass
class Bed:
    flags: np.ndarray          # uint8 [nz, ny, nx], 0 fluid, 1 solid
    dims: tuple                # (nx, ny, nz)
    axis: int                  # tube / flow axis, 0=x 1=y 2=z
    periodic: int              # bit mask, bit0 x, bit1 y, bit2 z
    n_spheres: int
    n_fluid: int

    @property
    def porosity(self) -> float:
        return self.n_fluid / self.flags.size


def packed_bed(dims, axis: int, tube_d: float, radius: float, porosity: float, seed: int,
               max_rejects: int = 20000) -> Bed:
    """Tube of diameter ``tube_d`` along ``axis`` packed by random sequential
    addition of spheres of radius ``radius`` until the box porosity is at or
    below ``porosity`` or ``max_rejects`` consecutive candidates were
    rejected.  Periodic along ``axis`` only."""
    nx, ny, nz = (int(d) for d in dims)
    flags = np.empty((nz, ny, nx), dtype=np.uint8)
    ns = ctypes.c_int64(0)
    nf = ctypes.c_int64(0)
    rc = _load().pb_packed_bed(nx, ny, nz, int(axis), float(tube_d), float(radius),
                               float(porosity), int(max_rejects), int(seed), flags.ctypes.data,
                               ctypes.byref(ns), ctypes.byref(nf))
    if rc != 0:
        raise RuntimeError(f"pb_packed_bed failed with status {rc}")
    return Bed(flags, (nx, ny, nz), int(axis), 1 << int(axis), int(ns.value), int(nf.value))


def alpha_field(dims, seed: int, lo: float = 0.0, hi: float = 0.05) -> np.ndarray:
    """Per box cell Brinkman damping drawn uniform in [lo, hi), laid out like
    the flags ([nz, ny, nx]); independent of any cell ordering."""
    nx, ny, nz = (int(d) for d in dims)
    return uniform(nx * ny * nz, seed, stream=7, lo=lo, hi=hi).reshape(nz, ny, nx)


# ---------------------------------------------------------------------------
# The workloads.  Each is seeded; the primary seed is 0.

def bed_small(seed: int = 0) -> Bed:
    """32x32x64 box, tube of diameter 30 along z, spheres of radius 4,
    porosity ~0.45 (random sequential addition saturates near 0.43 here)."""
    return packed_bed((32, 32, 64), 2, 30.0, 4.0, 0.45, seed)


def bed_large(seed: int = 0) -> Bed:
    """1024x256x256 box, tube of diameter 250 along x, spheres of radius 8,
    porosity target 0.40, which random sequential addition does not reach
    in this tube: it jams near 0.49 (~33 M fluid cells)."""
    return packed_bed((1024, 256, 256), 0, 250.0, 8.0, 0.40, seed)


def bed_medium(seed: int = 0) -> Bed:
    """256x128x128 bed of the large family: tube of diameter 122 along x,
    spheres of radius 8, periodic in x."""
    return packed_bed((256, 128, 128), 0, 122.0, 8.0, 0.40, seed)


def bed_cube128(seed: int = 0) -> Bed:
    """128^3 box, tube of diameter 126 along z, spheres of radius 6,
    porosity target 0.45."""
    return packed_bed((128, 128, 128), 2, 126.0, 6.0, 0.45, seed)


def batch_params(n_beds: int = 256, seed: int = 0):
    """Per-bed (side, radius, force) for the batched workload: cubic sides
    uniform in {24..96}, radii uniform in [3, 8], forces uniform in
    [1e-7, 1e-5] along z."""
    u = uniform(3 * n_beds, seed, stream=11).reshape(n_beds, 3)
    sides = 24 + np.minimum((u[:, 0] * 73).astype(np.int64), 72)
    radii = 3.0 + 5.0 * u[:, 1]
    forces = 1e-7 + (1e-5 - 1e-7) * u[:, 2]
    return sides, radii, forces


def batch_beds(n_beds: int = 256, seed: int = 0):
    """The beds of the batched workload: cube of side s, tube of diameter
    s - 2 along z, random sequential addition to saturation."""
    sides, radii, forces = batch_params(n_beds, seed)
    beds = []
    for b in range(n_beds):
        s = int(sides[b])
        beds.append(packed_bed((s, s, s), 2, float(s - 2), float(radii[b]), 0.0,
                               seed * 100003 + b))
    return beds, forces
