"""Storage precision forms on the 256x128x128 packed bed against the FP64
oracle at steady state.

The reference is the FP64 oracle's own run of this bed (tube of diameter 122
along x, spheres of radius 8, seed 0, periodic in x; F = 1e-6 along x,
omega+ = 1/0.8, Lambda = 3/16, 20,000 steps from rest), written by
tests/golden/make_medium_bed_reference.py: the velocity field of the last
step's collision (FP32) and its FP64 sums.  Each form runs the same 20,000
steps on the GPU in lexicographic order; the velocity-field L2 error
||u - u_ref|| / ||u_ref|| and the permeability error (the mean axial velocity
at fixed force; the Darcy normalisation cancels) are measured against it.

Bounds, from the arithmetic of each form:
  f64x  : FP64 storage: L2(u) at the FP32 resolution of the stored field
          (<= 1e-7); permeability from the FP64 sums <= 1e-10.
  f32s  : FP32 deviations: L2(u) <= 1e-4, permeability <= 1e-5.
  f16s  : 11-bit significand of the scaled deviation: the permeability
          target, <= 1e-3; L2(u) <= 1e-2.
  bf16s : 8-bit significand: reported; permeability <= 1e-2, L2(u) <= 1e-1.
Set LBM_REPORT_DIR to also write the measured errors as JSON.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

from paper_1111_1129_gb300 import (LBMState, SparseLattice, build, capi, deviation_bound, inputs,
                                   omega_minus, shifted_scale_exp)

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
REF = os.path.join(HERE, "golden", "medium_bed_u_fp64_oracle.npz")
BOUNDS = {"f64x": (1e-7, 1e-10), "f32s": (1e-4, 1e-5), "f16s": (1e-2, 1e-3),
          "bf16s": (1e-1, 1e-2)}


def load_reference(path: str = REF) -> dict:
    """The stored oracle field: u [3, N] (FP64 from its stored FP32), the FP64
    sums, its FP64 norm and the run's parameters."""
    from golden.make_medium_bed_reference import load
    return load(path)


@pytest.fixture(scope="module")
def reference():
    build.build()
    capi.load()
    ref = load_reference()
    bed = inputs.bed_medium(0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", periodic=bed.periodic)
    cells = lat.cells().cpu().numpy().astype(np.int32)
    assert lat.n == int(ref["n_fluid"])
    assert hashlib.sha256(cells.tobytes()).hexdigest() == str(ref["cells_sha256"])
    yield ref, lat
    lat.close()


@pytest.mark.parametrize("precision", ["f64x", "f32s", "f16s", "bf16s"])
def test_medium_bed_precision_against_the_oracle(reference, precision):
    ref, lat = reference
    wp, F = float(ref["omega_plus"]), tuple(float(v) for v in ref["force"])
    assert abs(float(ref["omega_minus"]) - omega_minus(wp)) < 1e-15
    steps = int(ref["steps"])
    k = shifted_scale_exp(deviation_bound(F[0], 61.0, wp))
    st = LBMState(lat, precision, k)
    st.step(steps, wp, omega_minus(wp), F)
    mass, flux = st.reduce_flux(0)
    _, u = st.moments()
    u = u.cpu().numpy()
    st.close()
    n = lat.n
    l2 = float(np.linalg.norm(u - ref["u"]) / ref["u_norm"])
    flux_ref = float(ref["sums"][1]) / n
    k_err = abs(flux - flux_ref) / abs(flux_ref)
    report = {"precision": precision, "scale_exp": k if precision in ("f16s", "bf16s") else None,
              "steps": steps, "n_fluid": n, "u_l2_rel": l2, "permeability_rel": k_err,
              "mass_drift_rel": abs(mass - n) / n, "reference": "FP64 oracle"}
    print(json.dumps(report))
    out = os.environ.get("LBM_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, f"precision_medium_{precision}.json"), "w") as fh:
            json.dump(report, fh)
    assert np.isfinite(u).all() and np.isfinite(mass)
    tol_u, tol_k = BOUNDS[precision]
    assert l2 <= tol_u, report
    assert k_err <= tol_k, report
