"""Benchmark: MFLUP/s of the sparse D3Q19 TRT sweep on one GB300.

Workload: the 1024x256x256 packed bed (tube of diameter 250 along x,
spheres of radius 8 by seeded random sequential addition, periodic in x,
~33 M fluid cells), body force 1e-6 along x, omega+ = 1/0.8, Lambda = 3/16,
rest initial state, FP64 PDFs, lexicographic order (--ordering picks
another).  The default form is f64x: FP64 storage with the update computed
in exact 64-bit fixed point (results equal IEEE FP64 to round-off);
--precision f64 times the IEEE-FP64-arithmetic kernel, which GB300's FP64
rate caps near 4.3 GLUP/s.

One "step" is one time step of the hot path: pull through the adjacency
list, TRT collision, streaming store (one kernel launch per step), with the
FP64 mass/flux reduction fused into the last step and finished by
lbm_reduce_flux.  MFLUP/s counts fluid cells only (Sec. 7).

The JSON line carries: value (device-resident inputs), e2e (the same metric
through the C ABI from pinned host flags to a host result, the copies inside
the library's calls), roofline of the sweep kernel, the CPU oracle timed on
a bounded sample, the SM clocks sampled during the timed region, the rates
of the IEEE-FP64 and FP16-shifted forms beside the headline with their
ratios, and extra measurements (orderings, storage forms) each labelled
with its own step count.

--impl reference times the CPU oracle instead (the only reference this
method has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WP = 1.0 / 0.8
FORCE = (1e-6, 0.0, 0.0)
AXIS = 0
BYTES_PER_LUP = {"f64": 19 * 8 * 2 + 18 * 4, "f64x": 19 * 8 * 2 + 18 * 4,
                 "f32": 19 * 4 * 2 + 18 * 4,
                 "f32s": 19 * 4 * 2 + 18 * 4, "f16s": 19 * 2 * 2 + 18 * 4,
                 "bf16s": 19 * 2 * 2 + 18 * 4}
# DRAM bytes (read + write) per fluid update of one sweep launch, measured by
# ncu (dram__bytes_read.sum + dram__bytes_write.sum of one launch, after
# three warm-up steps) per (workload, form, ordering).  The roofline's
# `traffic` multiplies them by the benchmark's cells.  Drop an entry when its
# kernel changes.
MEASURED_DRAM_BYTES_PER_LUP = {
    ("large", "f64x", "lex"): 379.9, ("large", "f32s", "lex"): 223.4,
    ("large", "f16s", "lex"): 147.2,
}
STORAGE = {"f64": "f64", "f64x": "f64", "f32": "f32", "f32s": "f32 (f - w)",
           "f16s": "f16 ((f - w) 2^k)", "bf16s": "bf16 ((f - w) 2^k)"}
ARITHMETIC = {"f64": "f64", "f64x": "int64", "f32": "f32", "f32s": "f32", "f16s": "f32",
              "bf16s": "f32"}
ARITHMETIC_NOTE = {
    "f64": "IEEE FP64",
    "f64x": "FP64 storage; update exact to FP64 round-off (int64 fixed point on f - w, unit "
            "2^-58): results agree with IEEE FP64 to round-off (parity 1e-12 of max|f| vs the "
            "oracle) and conserve the stored mass exactly; cells outside the fast range use "
            "IEEE FP64",
    "f32": "FP32", "f32s": "FP32", "f16s": "FP32", "bf16s": "FP32"}
# name: (label, input generator, flow axis, tube radius).  The body force,
# 1e-6, points along the tube.
WORKLOADS = {
    "large": ("packed bed 1024x256x256, tube D=250 along x, spheres r=8, seed 0", "bed_large",
              0, 125.0),
    "medium": ("packed bed 256x128x128, tube D=122 along x, spheres r=8, seed 0", "bed_medium",
               0, 61.0),
    "small": ("packed bed 32x32x64, tube D=30 along z, spheres r=4, seed 0", "bed_small", 2,
              15.0),
}


def _flow(workload):
    """(force, axis) of a workload."""
    axis = WORKLOADS[workload][2]
    return tuple(1e-6 if d == axis else 0.0 for d in range(3)), axis


def _scale_exp(workload):
    """Scale exponent of the 16-bit shifted forms for a workload's flow."""
    from paper_1111_1129_gb300 import deviation_bound, shifted_scale_exp
    return shifted_scale_exp(deviation_bound(1e-6, WORKLOADS[workload][3], WP))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples go to $LBM_CLOCKS_DIR (default: a temporary folder);
        # the JSON line carries their summary
        out_dir = os.environ.get("LBM_CLOCKS_DIR") or os.path.join(tempfile.gettempdir(),
                                                                   "lbm_clocks")
        self.path = os.path.join(out_dir, f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _oracle_slab(bed):
    """What the CPU oracle runs: a bed up to 64 cells long in x whole, with
    its own boundaries, else the slab x in [0, 64), periodic in x (the tube
    of the larger beds runs along x).  Returns (flags, periodic, label)."""
    import numpy as np

    nz, ny, nx = bed.flags.shape
    if nx <= 64:
        return bed.flags, bed.periodic, f"the whole {nx}x{ny}x{nz} bed"
    slab = np.ascontiguousarray(bed.flags[:, :, :64])
    return slab, 1, f"64x{ny}x{nz} slab of the bed (x in [0,64), periodic x)"


def _oracle_sample(bed, budget_s: float, force, max_steps: int | None = None):
    """The CPU oracle on a bounded sample of the bed (_oracle_slab): returns
    (MFLUP/s, steps, fluid cells, cores, seconds, label)."""
    import oracle

    slab, periodic, label = _oracle_slab(bed)
    n_fluid = int((slab == 0).sum())
    wm = oracle.omega_minus(WP)
    f = oracle.rest_state(slab)
    t0 = time.perf_counter()
    f, _, _, _ = oracle.run(slab, periodic, WP, wm, force, 1, f=f)
    one = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(one, 1e-6)))
    if max_steps is not None:
        steps = min(steps, max_steps)
    t0 = time.perf_counter()
    oracle.run(slab, periodic, WP, wm, force, steps, f=f)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n_fluid * steps / dt / 1e6, steps, n_fluid, cores, dt, label


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_1111_1129_gb300 import inputs
    bed = getattr(inputs, WORKLOADS[args.workload][1])(0)
    force, _ = _flow(args.workload)
    for _ in range(args.warmup):
        _oracle_sample(bed, 0.5, force, max_steps=1)
    lups = 0.0
    dt = 0.0          # the oracle's own time steps; its per-sample set-up is not counted
    samples = []
    # each step is a sample of ~3 s of oracle time, less when many steps are
    # asked for, so that the whole run stays within about two and a half
    # minutes
    budget = min(3.0, 150.0 / max(args.steps, 1))
    for _ in range(args.steps):
        mflups, steps, n_fluid, cores, t, label = _oracle_sample(bed, budget, force)
        lups += n_fluid * steps
        dt += t
        samples.append(steps)
    value = lups / dt / 1e6
    line = {
        "impl": "reference", "metric": "MFLUP/s", "value": value, "unit": "MFLUP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0], "ordering": "dense full-array oracle",
                   "precision": "f64", "fluid_cells_per_sample": n_fluid},
        "cpu_baseline": {"value": value, "unit": "MFLUP/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step: {label} ({n_fluid} fluid cells), ~{budget:.2f} s "
                                   f"of oracle time steps ({samples[0]} steps in the first)"},
        "e2e": {"value": value, "unit": "MFLUP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_1111_1129_gb300 import (LBMState, SparseLattice, capi, inputs, omega_minus,
                                       use_torch_allocator)
    from paper_1111_1129_gb300 import lbm as lbm_mod

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    capi.load()
    # the library's device memory comes from PyTorch's caching allocator
    # (lbm_set_allocator), as in any PyTorch program that uses it
    use_torch_allocator(True)
    wm = omega_minus(WP)
    # weak scaling: each rank owns an independent bed (seed = rank)
    bed = getattr(inputs, WORKLOADS[args.workload][1])(rank)
    force, axis = _flow(args.workload)
    flags_host = torch.from_numpy(bed.flags).pin_memory()
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    lat = SparseLattice(flags_host.cuda(), args.ordering, (8, 8, 8), bed.periodic)
    n = lat.n
    k16 = _scale_exp(args.workload)
    st = LBMState(lat, args.precision, k16)
    st.step(args.warmup, WP, wm, force)
    st.reduce_flux(axis)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier()
        ev0.record(stream)
        st.step(args.steps, WP, wm, force)
        mass, flux = st.reduce_flux(axis)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        tot = torch.tensor([float(n)], device="cuda", dtype=torch.float64)
        dist.all_reduce(tot)
        total_cells = float(tot.item())
    else:
        total_cells = float(n)
    value = total_cells * args.steps / (ms * 1e-3) / 1e6
    launch_ms = ms / args.steps
    st.close()

    # ---- e2e: pinned host flags -> C ABI -> host result -------------------
    # lbm_build_sparse copies the host flags to the device itself, and
    # lbm_reduce_flux returns the sums in host memory; the handles' device
    # memory comes from PyTorch's cache, which holds the blocks the run
    # above released
    # three independent calls, each host flags -> host sums; the median is
    # reported (one call of ~40 ms varies by several percent)
    e2e_times = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h_lat = capi.lbm_build_sparse(flags_host.data_ptr(), bed.dims,
                                      capi.make_ordering(lbm_mod.ORDERINGS[args.ordering],
                                                         (8, 8, 8), bed.periodic),
                                      int(stream.cuda_stream))
        h_st = capi.lbm_state_create(h_lat, lbm_mod.PRECISIONS[args.precision], k16)
        capi.lbm_step(h_st, args.steps, WP, wm, force)
        e2e_mass, e2e_flux = capi.lbm_reduce_flux(h_st, axis)
        e2e_times.append(time.perf_counter() - t0)
        capi.lbm_free(h_st)
        capi.lbm_free(h_lat)
    e2e_s = statistics.median(e2e_times)
    e2e_value = n * args.steps / e2e_s / 1e6
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_value = total_cells * args.steps / float(t.item()) / 1e6

    extra = {}
    cpu = None
    if rank == 0 and world == 1 and not args.no_extra:
        extra = _extras(lat, bed, wm, args, force, k16)
    forms = None
    if extra:
        # the FP64-storage, IEEE-FP64 and FP16-shifted rates from runs of the
        # same step count, and the ratios of the FP16-shifted form to each
        rate = dict(extra["by_storage_mflups"])
        forms = {f"{p}_mflups": rate[p] for p in ("f64x", "f64", "f32s", "f16s") if p in rate}
        if "f16s" in rate:
            for p in ("f64x", "f64"):
                if p in rate:
                    forms[f"f16s_over_{p}"] = rate["f16s"] / rate[p]
        forms["note"] = ("f64x: FP64 storage, int64 fixed-point update; f64: IEEE FP64 "
                         f"arithmetic; every rate from a {args.extra_steps}-step call "
                         "(one reducing step)")
    if rank == 0 and world == 1 and not args.no_cpu:
        mflups, steps_c, n_c, cores, dt, label = _oracle_sample(bed, args.cpu_seconds, force)
        cpu = {"value": mflups, "unit": "MFLUP/s", "cores": cores, "kind": "oracle",
               "sample": f"{label} ({n_c} fluid cells), {steps_c} FP64 steps of the dense "
                         f"full-array oracle ({dt:.1f} s)"}
    lat.close()
    peak, peak_kind = _peaks()
    bpl = BYTES_PER_LUP[args.precision]
    ws = (2 * 19 * (bpl - 72) / 38 + 72) * n   # two PDF grids + adjacency, bytes
    achieved = bpl * n / (launch_ms * 1e-3) / 1e9
    line = {
        "metric": "MFLUP/s", "value": value, "unit": "MFLUP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ARITHMETIC[args.precision], "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0], "fluid_cells_per_gpu": n, "ordering": f"{args.ordering}"
                   + (" 8^3" if args.ordering == "blocked" else ""),
                   "precision": args.precision, "storage": STORAGE[args.precision],
                   "scale_exp": k16 if args.precision in ("f16s", "bf16s") else None,
                   "arithmetic": ARITHMETIC_NOTE[args.precision], "force": list(force),
                   "omega_plus": WP, "omega_minus": wm,
                   "l2": ("inputs larger than L2 (PDFs+adjacency ~%.1f GB)" if ws > 129e6 else
                          "inputs fit in L2 (PDFs+adjacency ~%.3f GB): an L2-bound rate, not an "
                          "HBM one") % (ws / 1e9),
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (MEASURED_DRAM_BYTES_PER_LUP[key] * n
                                 if (key := (args.workload, args.precision, args.ordering))
                                 in MEASURED_DRAM_BYTES_PER_LUP else None),
                     "bytes_per_lup": bpl, "peak_kind": peak_kind,
                     "kernel": "sweep_fx_kernel" if args.precision == "f64x"
                     else (f"sweep_pair_kernel<{args.precision}>"
                           if args.precision in ("f16s", "bf16s") else
                           f"sweep_kernel<{args.precision}>")},
        "e2e": {"value": e2e_value, "unit": "MFLUP/s",
                "h2d_bytes_per_step": (bed.flags.nbytes + 24) / args.steps,
                "d2h_bytes_per_step": 32 / args.steps,
                "calls": "lbm_build_sparse (pinned host flags) + lbm_state_create + lbm_step "
                         "+ lbm_reduce_flux (host sums); device memory from PyTorch's caching "
                         "allocator (lbm_set_allocator), warm from the device-timed run; median "
                         "of 3 independent calls",
                "samples_mflups": [n * args.steps / t / 1e6 for t in e2e_times]},
        "gpu_launches": args.steps + 2,
        "clocks": clocks.summary(),
        "result": {"mass": mass, "flux": flux, "e2e_flux": e2e_flux},
    }
    if forms is not None:
        line["forms"] = forms
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if extra:
        line["extra"] = extra
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _extras(lat, bed, wm, args, force, k16):
    """Short labelled runs: the other orderings (in the benchmark's form) and
    the other storage forms (in the benchmark's ordering)."""
    import torch

    from paper_1111_1129_gb300 import LBMState, SparseLattice

    def timed(lattice, precision, steps, scale_exp=0):
        st = LBMState(lattice, precision, scale_exp)
        st.step(3, WP, wm, force)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st.step(steps, WP, wm, force)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st.close()
        return lattice.n * steps / (ms * 1e-3) / 1e6

    out = {"steps_each": args.extra_steps}
    orders = {}
    for name in ("lex", "blocked", "morton1", "morton2"):
        if name == args.ordering:
            l2 = lat
        else:
            l2 = SparseLattice(torch.from_numpy(bed.flags).cuda(), name, (8, 8, 8), bed.periodic)
        orders[name + (" 8^3" if name == "blocked" else "")] = timed(l2, args.precision,
                                                                    args.extra_steps, k16)
        if l2 is not lat:
            l2.close()
    out[f"{args.precision}_by_ordering_mflups"] = orders
    forms = {}
    for prec, k in (("f64", 0), ("f64x", 0), ("f32", 0), ("f32s", 0), ("f16s", k16),
                    ("bf16s", k16)):
        # every form, the headline's included, at the same step count
        forms[prec] = timed(lat, prec, args.extra_steps, k)
    out["by_storage_mflups"] = forms
    return out


def run_precision_study(args):
    """Storage forms against the FP64 oracle on the 256x128x128 bed at
    steady state: velocity-field L2 error, permeability (mean axial
    velocity) error, mass drift and MFLUP/s.  The reference is the oracle's
    own 20,000-step run of this bed, stored by
    tests/golden/make_medium_bed_reference.py (velocity field in FP32, sums
    in FP64); the GPU FP64 forms are listed against it too.  Prints one JSON
    line."""
    import hashlib

    import numpy as np
    import torch

    from paper_1111_1129_gb300 import (LBMState, SparseLattice, capi, deviation_bound, inputs,
                                       omega_minus, shifted_scale_exp)

    ref_path = os.path.join(ROOT, "tests", "golden", "medium_bed_u_fp64_oracle.npz")
    if not os.path.exists(ref_path):
        raise SystemExit(f"{ref_path} is missing: run tests/golden/make_medium_bed_reference.py")
    with np.load(ref_path) as z:
        ref = {k: z[k] for k in z.files}
    if args.study_steps != int(ref["steps"]):
        raise SystemExit(f"the oracle reference is for {int(ref['steps'])} steps")
    ref_u = ref["u"].astype(np.float64)
    capi.load()
    wm = omega_minus(WP)
    bed = inputs.bed_medium(0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", (8, 8, 8), bed.periodic)
    cells = lat.cells().cpu().numpy().astype(np.int32)
    if hashlib.sha256(cells.tobytes()).hexdigest() != str(ref["cells_sha256"]):
        raise SystemExit("the stored oracle field is for another cell list")
    flux_ref = float(ref["sums"][1]) / lat.n
    k16 = shifted_scale_exp(deviation_bound(FORCE[0], 61.0, WP))
    rows = {}
    for prec in ("f64", "f64x", "f32s", "f16s", "f32", "bf16s"):
        st = LBMState(lat, prec, k16)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st.step(args.study_steps, WP, wm, FORCE)
        e1.record()
        mass, flux = st.reduce_flux(AXIS)
        ms = e0.elapsed_time(e1)
        _, u = st.moments()
        u = u.cpu().numpy()
        st.close()
        rows[prec] = {
            "mflups": lat.n * args.study_steps / (ms * 1e-3) / 1e6,
            "u_l2_rel": float(np.linalg.norm(u - ref_u) / ref["u_norm"]),
            "permeability_rel": abs(flux - flux_ref) / abs(flux_ref),
            "mass_drift_rel": abs(mass - lat.n) / lat.n,
            "finite": bool(np.isfinite(u).all()),
        }
    line = {"study": "storage precision at steady state",
            "workload": WORKLOADS["medium"][0], "fluid_cells": lat.n,
            "steps": args.study_steps, "force": list(FORCE), "ordering": "lex",
            "scale_exp_16bit": k16,
            "reference": "FP64 oracle (dense full-array solver), same bed and steps; stored "
                         "velocity field in FP32 (L2 errors below ~3e-8 are its resolution), "
                         "sums in FP64",
            "forms": rows}
    lat.close()
    print(json.dumps(line), flush=True)
    return 0


def run_adjoint_study(args):
    """The 128^3 bed with per-cell Brinkman damping (uniform in [0, 0.05)),
    FP32 shifted storage, K = 2000 steps, checkpoints every 45 steps: time
    of a plain forward run, of the checkpointed forward pass and of the
    reverse pass, and the memory the adjoint holds."""
    import torch

    from paper_1111_1129_gb300 import Adjoint, LBMState, SparseLattice, capi, inputs, omega_minus

    capi.load()
    wm = omega_minus(WP)
    bed = inputs.bed_cube128(0)
    alpha_dense = inputs.alpha_field(bed.dims, seed=0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), args.ordering, (8, 8, 8), bed.periodic)
    alpha = torch.from_numpy(alpha_dense.reshape(-1)[lat.cells().cpu().numpy()].copy()).cuda()
    K, stride, F = args.adjoint_steps, 45, (0.0, 0.0, 1e-6)
    out = {}
    ref_f64 = None
    for prec in args.adjoint_forms.split(","):
        st = LBMState(lat, prec)
        st.set_damping(alpha)

        def timed(fn):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            return r, time.perf_counter() - t0

        st.step(3, WP, wm, F)
        st.reset()
        _, t_fwd = timed(lambda: (st.step(K, WP, wm, F), st.reduce_flux(2)))
        st.reset()
        torch.cuda.reset_peak_memory_stats()
        free0 = torch.cuda.mem_get_info()[0]
        adj = Adjoint(st, K, stride)
        held = free0 - torch.cuda.mem_get_info()[0]
        J, t_af = timed(lambda: adj.forward(WP, wm, F, 2))
        (dF, da, _), t_ab = timed(lambda: adj.backward())
        state_bytes = lat.n * 19 * (4 if prec == "f32s" else 8)
        # the FP64 forms' gradients against each other (f64: IEEE FP64
        # arithmetic; f64x: fixed-point steps, double-single reverse steps)
        if prec == "f64":
            ref_f64 = (dF, da.clone())
        if prec == "f64x" and ref_f64 is not None:
            rel_dF = max(abs(a - b) for a, b in zip(dF, ref_f64[0])) / max(abs(v) for v in ref_f64[0])
            rel_da = float(torch.linalg.norm(da - ref_f64[1]) / torch.linalg.norm(ref_f64[1]))
        out[prec] = {"forward_s": t_fwd, "adjoint_forward_s": t_af, "adjoint_backward_s": t_ab,
                     "adjoint_total_over_forward": (t_af + t_ab) / t_fwd,
                     "adjoint_device_bytes": held,
                     "adjoint_bytes_over_one_state": held / state_bytes,
                     "J": J, "dJdFz": dF[2]}
        if prec == "f64x" and ref_f64 is not None:
            out[prec]["vs_f64"] = {"dJdF_rel": rel_dF, "dJdalpha_norm_rel": rel_da}
        adj.close()
        st.close()
    line = {"study": "adjoint", "workload": "packed bed 128^3, tube D=126 along z, spheres r=6, "
            "damping U[0,0.05)", "fluid_cells": lat.n, "ordering": args.ordering, "steps": K,
            "checkpoint_stride": stride, "forms": out}
    lat.close()
    print(json.dumps(line), flush=True)
    return 0


def _l2_copy_ceiling(frac: float = 0.6, copies: int = 50, seconds: float = 1.5):
    """Copy bandwidth of data resident in L2: two FP32 buffers holding
    `frac` of the L2 together, copied back and forth `copies` times in one
    CUDA graph, best of the replays of `seconds`, each timed with CUDA
    events on the launching stream (the clocks are sampled meanwhile).
    Counts read + write bytes.  Returns (GB/s, bytes per buffer, clocks)."""
    import torch

    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    nbytes = int(frac * l2 / 2) // 4096 * 4096
    a = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):
            b.copy_(a)
            a.copy_(b)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for i in range(copies):
                (b if i % 2 == 0 else a).copy_(a if i % 2 == 0 else b)
        best = None
        with ClockSampler(torch.cuda.current_device()) as clocks:
            t_end = time.perf_counter() + seconds
            while time.perf_counter() < t_end:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                g.replay()
                e1.record(s)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
    s.synchronize()
    return 2 * nbytes * copies / (best * 1e-3) / 1e9, nbytes, clocks.summary()


def run_batch_study(args):
    """256 packed beds (cube sides uniform in {24..96}, sphere radii in
    [3, 8], forces in [1e-7, 1e-5] along z), in the storage form of
    --batch-precision (FP32 shifted by default): the autotuned batched
    launch in L2 groups, with resident steps (one cooperative launch per
    group that keeps the links in shared memory), and as one group under a
    CUDA graph, against the same beds stepped one by one; per-bed fluxes are
    compared bit for bit."""
    import torch

    from paper_1111_1129_gb300 import (BatchedState, LBMState, SparseLattice, capi,
                                       deviation_bound, inputs, omega_minus, shifted_scale_exp)

    capi.load()
    wm = omega_minus(WP)
    prec = args.batch_precision
    beds, fz = inputs.batch_beds(256, 0)
    forces = [(0.0, 0.0, float(f)) for f in fz]
    # 16-bit forms: one scale for all beds, from the largest force and the
    # widest bed (tube radius at most half the largest cube side, 48)
    k = shifted_scale_exp(deviation_bound(float(max(abs(fz))), 48.0, WP)) \
        if prec in ("f16s", "bf16s") else 0
    lats = [SparseLattice(torch.from_numpy(b.flags).cuda(), args.ordering, (8, 8, 8), b.periodic)
            for b in beds]
    n_fluid = sum(l.n for l in lats)
    K = args.batch_steps
    tuner = BatchedState(lats, prec, k)
    block, cpt, cand = tuner.tune(20, WP, wm, forces)
    tuner.close()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    out = {}
    resident_cells = None
    for label, graph, group_bytes, resident in (("batched_l2_groups", True, -1, 0),
                                                ("batched_resident", True, -1, 1),
                                                ("batched_graph", True, 0, 0),
                                                ("batched_no_graph", False, 0, 0)):
        bs = BatchedState(lats, prec, k)
        bs.configure(block, cpt, graph)
        n_groups = bs.groups(group_bytes)
        if resident:
            n_groups, resident_cells = bs.resident(1)
        bs.step(K, WP, wm, forces)          # warm-up; captures the graph
        bs.reset()                          # back to rest, same grid parity
        ms = timed(lambda: bs.step(K, WP, wm, forces))
        mass, flux = bs.reduce_flux(2)
        out[label] = {"mflups": n_fluid * K / (ms * 1e-3) / 1e6, "ms": ms, "groups": n_groups}
        if label == "batched_l2_groups":
            batched_flux = flux
        else:
            assert list(flux) == list(batched_flux), "grouping changed a bed's flux"
        bs.close()
    states = [LBMState(l, prec, k) for l in lats]

    def separate():
        for st, F in zip(states, forces):
            st.step(K, WP, wm, F)

    ms = timed(separate)
    same = sum(1 for st, q in zip(states, batched_flux) if st.reduce_flux(2)[1] == q)
    out["separate_loops"] = {"mflups": n_fluid * K / (ms * 1e-3) / 1e6, "ms": ms}
    for st in states:
        st.close()
    for l in lats:
        l.close()
    # L2 groups stream from L2: their roofline is an L2 copy ceiling
    # measured here; the form's algorithmic bytes per update (19 loads, 19
    # stores, 18 int32 links; 224 for FP32), plus the per-block bed-table
    # reads (chunk's bed, begin, count, force: 52 bytes per block of block x
    # cells/thread)
    l2_gbs, l2_buf, l2_clocks = _l2_copy_ceiling()
    bpl = BYTES_PER_LUP[prec] + 52 / (block * cpt)
    achieved = bpl * n_fluid * K / (out["batched_l2_groups"]["ms"] * 1e-3) / 1e9
    roofline = {"bound": "l2", "achieved": achieved, "peak": l2_gbs, "unit": "GB/s",
                "frac": achieved / l2_gbs, "bytes_per_lup": bpl,
                "peak_kind": f"measured here: L2-resident copy, 2 x {l2_buf / 1e6:.1f} MB "
                             "FP32 buffers, 50 copies per CUDA graph, best replay of 1.5 s",
                "peak_clocks": l2_clocks, "kernel": f"batch_sweep_kernel<{prec}> (L2 groups)"}
    # resident steps read the links once per call: 19 loads and 19 stores per
    # update, plus 72 bytes of links per cell and call
    bpl_res = BYTES_PER_LUP[prec] - 72 + 72 / K
    achieved_res = bpl_res * n_fluid * K / (out["batched_resident"]["ms"] * 1e-3) / 1e9
    roofline_res = {"bound": "l2", "achieved": achieved_res, "peak": l2_gbs, "unit": "GB/s",
                    "frac": achieved_res / l2_gbs, "bytes_per_lup": bpl_res,
                    "kernel": f"batch_resident_kernel<{prec}> (groups of <= "
                              f"{resident_cells} cells)"}
    line = {"study": "batched beds", "n_beds": 256, "fluid_cells": n_fluid, "steps": K,
            "roofline": roofline, "roofline_resident": roofline_res,
            "ordering": args.ordering, "precision": prec,
            "scale_exp": k if prec in ("f16s", "bf16s") else None,
            "tuned": {"block": block, "cells_per_thread": cpt,
                                           "candidate_ms_block_major": cand},
            **out, "speedup_vs_separate": out["batched_l2_groups"]["mflups"] /
            out["separate_loops"]["mflups"],
            "resident_speedup_vs_l2_groups": out["batched_resident"]["mflups"] /
            out["batched_l2_groups"]["mflups"],
            "per_bed_flux_bit_identical": f"{same}/256"}
    print(json.dumps(line), flush=True)
    return 0


def _interface_metrics_gpu(adj, n, p):
    """Neighbour partitions and remote links per chunk of p equal chunks
    (Fig. 7 metrics), on the GPU for large lists."""
    import torch

    q, r = divmod(n, p)
    k = torch.arange(p + 1, device="cuda", dtype=torch.int64)
    bounds = k * q + torch.minimum(k, torch.tensor(r, device="cuda"))
    cell_owner = torch.searchsorted(bounds, torch.arange(n, device="cuda"), right=True) - 1
    links = torch.zeros(p, dtype=torch.int64, device="cuda")
    pairs = []
    for i in range(18):
        m = adj[i].to(torch.int64) % n
        so = torch.searchsorted(bounds, m, right=True) - 1
        remote = so != cell_owner
        links += torch.bincount(cell_owner[remote], minlength=p)
        pairs.append(torch.unique(cell_owner[remote] * p + so[remote]))
    uniq = torch.unique(torch.cat(pairs))
    nb = torch.bincount(uniq // p, minlength=p)
    return nb.float(), links.float()


def run_ordering_study(args):
    """MFLUP/s of the HBM-bound storage forms and the chunk-interface
    metrics as functions of the numbering scheme (lexicographic with
    blocking factor b = 1..128, Z curve 1-bit and 2-bit) on the
    1024x256x256 bed: the GB300 counterpart of Sec. 7's Fig. 4 and Fig. 7."""
    import torch

    from paper_1111_1129_gb300 import LBMState, SparseLattice, capi, inputs, omega_minus

    capi.load()
    wm = omega_minus(WP)
    bed = inputs.bed_large(0)
    flags = torch.from_numpy(bed.flags).cuda()
    rows = []
    orders = [("lex", (1, 1, 1))] + [("blocked", (b, b, b)) for b in (2, 4, 8, 16, 32, 64, 128)] + [
        ("morton1", (1, 1, 1)), ("morton2", (1, 1, 1)), ("hilbert", (1, 1, 1))]
    for name, block in orders:
        lat = SparseLattice(flags, name, block, bed.periodic)
        row = {"ordering": name if name != "blocked" else f"blocked {block[0]}"}
        for prec in args.study_forms.split(","):
            st = LBMState(lat, prec, _scale_exp("large"))
            st.step(3, WP, wm, FORCE)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st.step(args.extra_steps, WP, wm, FORCE)
            e1.record()
            torch.cuda.synchronize()
            row[f"{prec}_mflups"] = lat.n * args.extra_steps / (e0.elapsed_time(e1) * 1e-3) / 1e6
            st.close()
        adj = torch.as_tensor(lat.adjacency())
        for p in (64, 1024):
            nb, links = _interface_metrics_gpu(adj, lat.n, p)
            row[f"P{p}_neighbours_mean"] = nb.mean().item()
            row[f"P{p}_neighbours_max"] = nb.max().item()
            row[f"P{p}_remote_links_mean"] = links.mean().item()
        del adj
        rows.append(row)
        lat.close()
    # the tuner's pick from a 128-cell slab, and where it ranks at full size
    from paper_1111_1129_gb300.autotune import tune_ordering
    form = args.study_forms.split(",")[0] if "f64x" not in args.study_forms else "f64x"
    best, table = tune_ordering(bed.flags, AXIS, bed.periodic, precision=form)
    label = best[0] if best[0] != "blocked" else f"blocked {best[1][0]}"
    full = sorted(((r[f"{form}_mflups"], r["ordering"]) for r in rows if f"{form}_mflups" in r),
                  reverse=True)
    rank = next((i + 1 for i, (_, o) in enumerate(full) if o == label), None)
    tuned = {"form": form, "sample": "x in [0,128), periodic x", "pick": label,
             "sample_table": [(n if n != "blocked" else f"blocked {b[0]}", v) for n, b, v in table],
             "pick_full_size_rank": rank,
             "pick_full_size_mflups": next((v for v, o in full if o == label), None),
             "best_full_size": full[0] if full else None}
    print(json.dumps({"study": "ordering", "workload": WORKLOADS["large"][0],
                      "steps_each": args.extra_steps, "rows": rows, "tuner": tuned}), flush=True)
    return 0


def run_seed_study(args):
    """MFLUP/s and fraction of the copy ceiling of the storage forms on the
    1024x256x256 bed drawn with seeds 0-4 (lexicographic order): how much the
    rate depends on the particular packing."""
    import torch

    from paper_1111_1129_gb300 import LBMState, SparseLattice, capi, inputs, omega_minus

    capi.load()
    wm = omega_minus(WP)
    peak, peak_kind = _peaks()
    forms = args.study_forms.split(",")
    rows = []
    for seed in range(5):
        bed = inputs.bed_large(seed)
        lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", (1, 1, 1), bed.periodic)
        row = {"seed": seed, "fluid_cells": lat.n, "porosity": lat.n / bed.flags.size}
        for prec in forms:
            st = LBMState(lat, prec, _scale_exp("large"))
            st.step(3, WP, wm, FORCE)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st.step(args.extra_steps, WP, wm, FORCE)
            e1.record()
            torch.cuda.synchronize()
            rate = lat.n * args.extra_steps / (e0.elapsed_time(e1) * 1e-3) / 1e6
            row[f"{prec}_mflups"] = rate
            row[f"{prec}_frac"] = rate * 1e6 * BYTES_PER_LUP[prec] / 1e9 / peak
            st.close()
        rows.append(row)
        lat.close()
    summary = {}
    for prec in forms:
        v = [r[f"{prec}_mflups"] for r in rows]
        summary[prec] = {"mean_mflups": statistics.mean(v), "min": min(v), "max": max(v),
                         "spread": (max(v) - min(v)) / statistics.mean(v),
                         "mean_frac": statistics.mean(r[f"{prec}_frac"] for r in rows)}
    print(json.dumps({"study": "seeds", "workload": "packed bed 1024x256x256, tube D=250 along "
                      "x, spheres r=8, seeds 0-4", "ordering": "lex",
                      "steps_each": args.extra_steps, "peak_gbs": peak, "peak_kind": peak_kind,
                      "rows": rows, "summary": summary}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=list(WORKLOADS))
    ap.add_argument("--ordering", default="lex", choices=["lex", "blocked", "morton1",
                                                               "morton2", "hilbert"])
    ap.add_argument("--precision", default="f64x", choices=list(BYTES_PER_LUP))
    ap.add_argument("--extra-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--precision-study", action="store_true",
                    help="run the storage-precision study instead of the benchmark")
    ap.add_argument("--study-steps", type=int, default=20000)
    ap.add_argument("--batch-study", action="store_true",
                    help="run the 256-bed batching study instead of the benchmark")
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--batch-precision", default="f32s", choices=list(BYTES_PER_LUP))
    ap.add_argument("--ordering-study", action="store_true",
                    help="run the numbering-scheme study instead of the benchmark")
    ap.add_argument("--study-forms", default="f64x,f32s,f16s")
    ap.add_argument("--seed-study", action="store_true",
                    help="the storage forms on the large bed drawn with seeds 0-4")
    ap.add_argument("--adjoint-study", action="store_true",
                    help="time the checkpointed adjoint against the forward run")
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--adjoint-forms", default="f32s,f64,f64x")
    args = ap.parse_args()
    if args.adjoint_study:
        return run_adjoint_study(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.precision_study:
        return run_precision_study(args)
    if args.batch_study:
        return run_batch_study(args)
    if args.ordering_study:
        return run_ordering_study(args)
    if args.seed_study:
        return run_seed_study(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
