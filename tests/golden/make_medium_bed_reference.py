"""Writes the FP64 oracle's steady-state velocity field of the 256x128x128
packed bed, the reference of the storage-precision study.

Workload: the 256x128x128 bed of the large-bed family (tube of diameter 122
along x, spheres of radius 8, seeded random sequential addition, seed 0,
periodic in x), omega+ = 1/0.8, Lambda = 3/16, body force 1e-6 along x,
20,000 steps from the rest state (the steady-state precision configuration;
the numbering scheme does not change the field).

Only ``oracle/`` computes anything here; the seeded geometry comes from the
shared input generator.  The oracle's dense full-array solver runs the steps
in chunks (``--chunk``), handing the PDFs from one call to the next, which
leaves every PDF bit-identical to one long call; ``--resume`` continues from
the PDFs a killed run saved.

Stored (``medium_bed_u_fp64_oracle.npz``):
  u          float32 [3, N]  velocity of the last step's collision, fluid
                             cells in lexicographic order (x fastest)
  sums       float64 [4]     (sum rho, sum u_x, sum u_y, sum u_z) of that step
  u_norm     float64         ||u||_2 over fluid cells, in FP64
  n_fluid, steps, force, omega_plus, omega_minus, cells_sha256

FP32 storage of u keeps 2^-24 relative resolution per value: enough to
measure the FP32, FP16 and BF16 storage forms (errors >= 1e-7); the FP64
forms are held to the oracle at 1e-12 by their own parity tests.  The
permeability reference is sums[1] / N, kept in FP64.

Usage: python tests/golden/make_medium_bed_reference.py [--steps 20000]
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "medium_bed_u_fp64_oracle.npz")
WP = 1.0 / 0.8
FORCE = (1e-6, 0.0, 0.0)


def load(path: str = OUT) -> dict:
    """The stored reference as a dict; u as FP64 [3, N] (from its FP32)."""
    with np.load(path) as z:
        ref = {k: z[k] for k in z.files}
    ref["u"] = ref["u"].astype(np.float64)
    return ref


def main() -> int:
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1111_1129_gb300 import inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--chunk", type=int, default=500)
    ap.add_argument("--out", default=OUT)
    ap.add_argument("--resume", default="", help="PDF checkpoint (.npz) to continue from")
    ap.add_argument("--checkpoint", default="", help="where to save the PDFs after each chunk")
    args = ap.parse_args()
    wm = oracle.omega_minus(WP)
    bed = inputs.bed_medium(0)
    cells, _, _ = oracle.build_sparse(bed.flags, oracle.ORDER_LEX, periodic=bed.periodic)
    assert cells.size == bed.n_fluid
    f, done = None, 0
    if args.resume:
        ck = np.load(args.resume)
        f, done = ck["f"], int(ck["done"])
    t0 = time.time()
    obs = u = None
    while done < args.steps:
        k = min(args.chunk, args.steps - done)
        f, obs, _, u = oracle.run(bed.flags, bed.periodic, WP, wm, FORCE, k, f=f)
        done += k
        if args.checkpoint:
            np.savez(args.checkpoint + ".tmp.npz", f=f, done=done)
            os.replace(args.checkpoint + ".tmp.npz", args.checkpoint)
        el = time.time() - t0
        print(f"{done}/{args.steps} steps, {el:.0f} s, mean u_x {obs[-1, 1] / cells.size:.6e}",
              flush=True)
    u_s = oracle.to_sparse(u, cells)
    np.savez_compressed(
        args.out, u=u_s.astype(np.float32), sums=obs[-1].astype(np.float64),
        u_norm=np.float64(np.linalg.norm(u_s)), n_fluid=np.int64(cells.size),
        steps=np.int64(args.steps), force=np.array(FORCE), omega_plus=np.float64(WP),
        omega_minus=np.float64(wm),
        cells_sha256=np.array(hashlib.sha256(cells.astype(np.int32).tobytes()).hexdigest()))
    print(f"wrote {args.out}", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
