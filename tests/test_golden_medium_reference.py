"""The stored FP64 oracle field of the 256x128x128 packed bed (written by
tests/golden/make_medium_bed_reference.py) is consistent with the oracle
and with itself, checked on the CPU:

* its cell list is the oracle's lexicographic list of the seeded bed;
* the run conserved mass exactly (sum rho = N: the collision conserves mass
  and the bed's walls bounce back);
* the stored FP32 velocities reproduce the FP64 sums (mean u_x, the
  permeability reference) and the FP64 norm to FP32 resolution;
* the parameters are the steady-state precision configuration (F = 1e-6
  along x, omega+ = 1/0.8, Lambda = 3/16, 20,000 steps);
* the flow runs along +x and is, on average, axial: the mean transverse
  velocities are below 1e-6 of the axial one.
"""
import hashlib
import os

import numpy as np

import oracle
from paper_1111_1129_gb300 import inputs

REF = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                   "medium_bed_u_fp64_oracle.npz")


def test_medium_bed_reference_is_consistent():
    with np.load(REF) as z:
        ref = {k: z[k] for k in z.files}
    bed = inputs.bed_medium(0)
    cells, _, _ = oracle.build_sparse(bed.flags, oracle.ORDER_LEX, periodic=bed.periodic)
    n = int(ref["n_fluid"])
    assert n == cells.size == bed.n_fluid
    assert hashlib.sha256(cells.astype(np.int32).tobytes()).hexdigest() == str(ref["cells_sha256"])
    assert int(ref["steps"]) == 20000
    assert tuple(ref["force"]) == (1e-6, 0.0, 0.0)
    assert float(ref["omega_plus"]) == 1.0 / 0.8
    assert abs(float(ref["omega_minus"]) - oracle.omega_minus(1.0 / 0.8)) < 1e-15
    sums = ref["sums"]
    assert abs(sums[0] - n) <= 1e-9 * n                       # mass conserved
    u = ref["u"].astype(np.float64)
    assert u.shape == (3, n) and np.isfinite(u).all()
    mean = u.sum(axis=1) / n
    assert abs(mean[0] - sums[1] / n) <= 1e-6 * abs(sums[1] / n)   # FP32 resolution
    assert sums[1] > 0                                          # flow along +x
    assert abs(sums[2]) < 1e-6 * sums[1] and abs(sums[3]) < 1e-6 * sums[1]
    assert abs(np.linalg.norm(u) - float(ref["u_norm"])) <= 1e-6 * float(ref["u_norm"])
