"""Error measures of an FP64 GPU field against the FP64 oracle.

Reading of the FP64 tolerance.  The FP64 forms store the PDFs f themselves,
and f_q sits near its weight w_q <= 1/3.  Every FP64 operation on such a
value rounds by up to half an ulp of 1/3 (ulp 2^-54 = 5.6e-17) in
absolute terms, however small the deviation f - w that carries the flow.  The GPU
and the oracle sum in different orders, so their difference after K steps
is a sum of such roundings: the FP64 tolerance "1e-12 relative" is read
relative to the stored PDFs, max|f_gpu - f_oracle| <= 1e-12 max|f_oracle|.

Relative to the deviation max|f - w| (about 1e-6 in a flow driven by
F = 1e-6) the same absolute rounding is a larger fraction, so that measure
and the velocity measure are reported next to it and bounded by the
absolute round-off they follow from:
  max|df| <= 16 K 2^-54  per step at most 16 ulps of 1/3: the rest
                         population takes the rounding of rho, a sum of 19
                         values near 1 (ulp 2^-52) formed in a different
                         order on each side, times w+/3 < 2/3;
  max|du| <= 11 K 16 2^-54  u = j + F/2 sums 10 pulled values, each off by
                         at most max|df|, plus its own rounding.
Each test prints all three measures.
"""
from __future__ import annotations

import json
import os

import numpy as np

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
ULP_THIRD = 2.0 ** -54      # ulp of values in [1/4, 1/2)
PER_STEP = 16 * ULP_THIRD
TOL_REL_F = 1e-12


def measures(got, ref, steps: int, u_got=None, u_ref=None, label: str = "") -> dict:
    """The error measures of PDFs [19, N] (and optionally velocities
    [3, N]) and their round-off bounds; prints one JSON line, also written
    to $LBM_REPORT_DIR/fp64_errors.jsonl when that is set."""
    got = np.asarray(got, np.float64).reshape(19, -1)
    ref = np.asarray(ref, np.float64).reshape(19, -1)
    df = float(np.max(np.abs(got - ref))) if ref.size else 0.0
    fmax = float(np.max(np.abs(ref))) if ref.size else 1.0
    dev = float(np.max(np.abs(ref - W[:, None]))) if ref.size else 1.0
    bound_abs = PER_STEP * max(steps, 1)
    out = {"label": label, "steps": int(steps), "n": int(ref.shape[1]),
           "max_abs_df": df, "rel_to_max_f": df / fmax,
           "rel_to_max_dev": df / dev if dev > 0 else 0.0, "max_dev": dev,
           "bound_abs_df": bound_abs}
    if u_ref is not None:
        u_got = np.asarray(u_got, np.float64)
        u_ref = np.asarray(u_ref, np.float64)
        du = float(np.max(np.abs(u_got - u_ref))) if u_ref.size else 0.0
        umax = float(np.max(np.abs(u_ref))) if u_ref.size else 0.0
        out.update({"max_abs_du": du, "rel_to_max_u": du / umax if umax > 0 else 0.0,
                    "max_u": umax, "bound_abs_du": 11.0 * bound_abs})
    print("fp64 errors " + json.dumps(out))
    rep = os.environ.get("LBM_REPORT_DIR")
    if rep:
        os.makedirs(rep, exist_ok=True)
        with open(os.path.join(rep, "fp64_errors.jsonl"), "a") as fh:
            fh.write(json.dumps(out) + "\n")
    return out


def check(got, ref, steps: int, u_got=None, u_ref=None, label: str = "") -> dict:
    """measures() plus the asserts: 1e-12 of max|f|, and the absolute
    round-off bounds on f and u."""
    m = measures(got, ref, steps, u_got, u_ref, label)
    assert m["rel_to_max_f"] <= TOL_REL_F, m
    assert m["max_abs_df"] <= m["bound_abs_df"], m
    if u_ref is not None:
        assert m["max_abs_du"] <= m["bound_abs_du"], m
    return m
