"""Storage units of the reduced-precision forms, for one-step comparisons
with the FP64 oracle.

The GPU computes a step in FP32 and rounds once into storage, so each
output lies within one storage unit of the FP64 result, plus the FP32
rounding of the collision.  The forms: FP32 of f itself; FP32, FP16 and
BF16 of the deviation d = f - w (the 16-bit forms scaled by 2^k).
"""
from __future__ import annotations

import numpy as np

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
EPS32 = 2.0 ** -24


def ulp_f16(v):
    """Spacing of FP16 at |v| (v already scaled), from numpy's float16."""
    return np.spacing(np.abs(v).astype(np.float16)).astype(np.float64)


def ulp_bf16(v):
    """Spacing of BF16 (8-bit significand, FP32 exponent range) at |v|."""
    a = np.abs(v)
    e = np.floor(np.log2(np.where(a > 0, a, 2.0 ** -126)))
    return 2.0 ** (np.maximum(e, -126) - 7)


def ulp_f32(v):
    return np.spacing(np.abs(v).astype(np.float32)).astype(np.float64)


def rn_bf16(v):
    """Round FP64 to BF16 (via FP32, nearest even), returned as FP64."""
    u = np.asarray(v, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def one_step_tolerance(precision: str, f_ref, dev_rep_max: float, k: int):
    """Per-output bound on |f_gpu - f_ref| after one step from a state whose
    largest stored deviation is dev_rep_max: one storage unit at the
    result, plus the FP32 rounding of the collision (4 x 2^-24 of the
    largest intermediate deviation sum, 19 dev_rep_max, for the shifted
    forms; 64 x for the 16-bit forms, whose unit dwarfs it anyway; 6 x 2^-24
    of rho ~ 1 for FP32 of f itself)."""
    big = 19.0 * dev_rep_max
    scale = 2.0 ** k
    d_ref = (f_ref - W[:, None]) * scale     # exact: the subtraction cancels w's bits
    if precision == "f16s":
        return ulp_f16(d_ref) / scale + 64 * EPS32 * big
    if precision == "bf16s":
        return ulp_bf16(d_ref) / scale + 64 * EPS32 * big
    if precision == "f32s":
        return ulp_f32(f_ref - W[:, None]) + 4 * EPS32 * big
    if precision == "f32":
        return ulp_f32(f_ref) + 6 * EPS32
    raise ValueError(precision)


def codes_equal_fraction(precision: str, f_gpu, f_ref, k: int) -> float:
    """Fraction of 16-bit codes equal to the FP64 result rounded to nearest
    even at the same scale."""
    scale = 2.0 ** k
    d_ref = (f_ref - W[:, None]) * scale
    code_gpu = (f_gpu - W[:, None]) * scale
    code_ref = d_ref.astype(np.float16).astype(np.float64) if precision == "f16s" else rn_bf16(d_ref)
    return float(np.mean(code_gpu == code_ref))
