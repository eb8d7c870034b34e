"""Choosing the numbering scheme by simulating a sample of the geometry.

The best blocking factor depends on the machine and the geometry, so the
paper proposes to pick it by running only samples of the geometry (Sec. 8,
future work).  This does exactly that on the GPU: cut a slab from the
domain along the chosen axis, build its sparse representation under each
candidate ordering, time a few sweeps, and rank the candidates.  The slab
is made periodic along the cut axis so that it keeps the flow structure of
a tube section.
"""
from __future__ import annotations

import numpy as np
import torch

from .lbm import LBMState, SparseLattice, omega_minus

DEFAULT_CANDIDATES = [("lex", (1, 1, 1))] + [("blocked", (b, b, b)) for b in (4, 8, 16, 32, 64)] + [
    ("morton1", (1, 1, 1)), ("morton2", (1, 1, 1)), ("hilbert", (1, 1, 1))]


def sample_slab(flags: np.ndarray, axis: int, length: int) -> np.ndarray:
    """The first ``length`` cells of ``flags`` ([nz, ny, nx]) along ``axis``
    (0 = x)."""
    sl = [slice(None)] * 3
    sl[2 - axis] = slice(0, min(length, flags.shape[2 - axis]))
    return np.ascontiguousarray(flags[tuple(sl)])


def tune_ordering(flags: np.ndarray, axis: int, periodic: int, precision: str = "f64x",
                  candidates=None, sample_length: int = 128, steps: int = 30,
                  omega_plus: float = 1.25, force: float = 1e-6):
    """Rank ``candidates`` ((name, block) pairs) by MFLUP/s on a slab of
    ``sample_length`` cells along ``axis``.  Returns (best, table) with
    table a list of (name, block, mflups) sorted fastest first."""
    candidates = candidates or DEFAULT_CANDIDATES
    slab = sample_slab(flags, axis, sample_length)
    per = int(periodic) | (1 << axis)
    F = [0.0, 0.0, 0.0]
    F[axis] = force
    wm = omega_minus(omega_plus)
    flags_dev = torch.from_numpy(slab).cuda()
    table = []
    for name, block in candidates:
        lat = SparseLattice(flags_dev, name, block, per)
        st = LBMState(lat, precision)
        st.step(3, omega_plus, wm, F)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        st.step(steps, omega_plus, wm, F)
        e1.record()
        torch.cuda.synchronize()
        table.append((name, tuple(block), lat.n * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6))
        st.close()
        lat.close()
    table.sort(key=lambda r: -r[2])
    return table[0][:2], table
