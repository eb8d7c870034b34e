"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of oracle/lbm_oracle.c (a dropped term, a swapped rate, a wrong
weight, sign, coefficient, slot or key bit), builds it on the side, and
runs every pin of tests/test_oracle_pins.py (and the sparse-stepper pin of
tests/test_partition.py) against it: at least one pin must fail.  Every mistake keeps all memory accesses in bounds.  The oracle
itself is not modified."""
import itertools
import os
import subprocess

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")

# (name, text in the oracle, planted text)
MISTAKES = [
    ("half force dropped from u",
     "u[k] = (j[k] + 0.5 * F[k]) / (1.0 + 0.5 * alpha);",
     "u[k] = j[k] / (1.0 + 0.5 * alpha);"),
    ("relaxation rates swapped",
     "fout[q] = g[q] - omega_p * (gp - ep) - omega_m * (gm - em) +",
     "fout[q] = g[q] - omega_m * (gp - ep) - omega_p * (gm - em) +"),
    ("axis weight 1/36",
     "if (q <= 6) return 1.0 / 18.0;",
     "if (q <= 6) return 1.0 / 36.0;"),
    ("quadratic coefficient 3 instead of 9/2",
     "e[q] = weight(q) * (rho + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);",
     "e[q] = weight(q) * (rho + 3.0 * cu + 3.0 * cu * cu - 1.5 * usq);"),
    ("sign of the u.u term",
     "e[q] = weight(q) * (rho + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);",
     "e[q] = weight(q) * (rho + 3.0 * cu + 4.5 * cu * cu + 1.5 * usq);"),
    ("forcing prefactor with the even rate",
     "(1.0 - 0.5 * omega_m) * 3.0 * weight(q) * cF;",
     "(1.0 - 0.5 * omega_p) * 3.0 * weight(q) * cF;"),
    ("Brinkman drag dropped from the force",
     "for (int k = 0; k < 3; ++k) Fn[k] = F[k] - alpha * u[k];",
     "for (int k = 0; k < 3; ++k) Fn[k] = F[k];"),
    ("dense bounce back into the same direction",
     "g[q] = f[(int64_t)opposite(q) * box + c];",
     "g[q] = f[(int64_t)q * box + c];"),
    ("sparse bounce back into the same direction",
     "slot = (int64_t)opposite(q) * n + i;",
     "slot = (int64_t)q * n + i;"),
    ("periodic wrap off by one",
     "s[k] = (s[k] % dims[k] + dims[k]) % dims[k];",
     "s[k] = (s[k] + 1 + dims[k]) % dims[k];"),
    ("Morton bit of the wrong axis",
     "key |= ((p[k] >> bit) & 1ull) << (3 * bit + k);",
     "key |= ((p[k] >> bit) & 1ull) << (3 * bit + (2 - k));"),
    ("block stride without its depth",
     "return (uint64_t)(blk * (bx * by * bz) + loc);",
     "return (uint64_t)(blk * (bx * by) + loc);"),
    ("Jacobian of the quadratic term halved",
     "de_du[q][k] = weight(q) * (3.0 * CQ[q][k] + 9.0 * cu * CQ[q][k] - 3.0 * u[k]);",
     "de_du[q][k] = weight(q) * (3.0 * CQ[q][k] + 4.5 * cu * CQ[q][k] - 3.0 * u[k]);"),
    ("transposed bounce back into the same direction",
     "lam_f[(int64_t)opposite(q) * box + c] += lam_g[(int64_t)q * box + c];",
     "lam_f[(int64_t)q * box + c] += lam_g[(int64_t)q * box + c];"),
    ("direct dJ/dF term dropped",
     "dJdF[axis] += 0.5 * s / (double)nf;",
     "dJdF[axis] += 0.0 * s / (double)nf;"),
    ("sparse stepper reads the rest value from the wrong row",
     "g[0] = f_src[i];",
     "g[0] = f_src[n + i];"),
    ("sparse stepper stores the pulled values uncollided",
     "for (int q = 0; q < 19; ++q) f_dst[(int64_t)q * n + i] = fo[q];",
     "for (int q = 0; q < 19; ++q) f_dst[(int64_t)q * n + i] = g[q];"),
]


def _pin_calls():
    """Every pin of test_oracle_pins.py, its parametrisations expanded, and
    the sparse-stepper pin of test_partition.py."""
    from tests import test_oracle_pins as pins
    from tests import test_partition as part
    fns = [(name, getattr(pins, name)) for name in sorted(dir(pins))]
    fns.append(("test_sparse_step_matches_dense_pull", part.test_sparse_step_matches_dense_pull))
    calls = []
    for name, fn in fns:
        if not (name.startswith("test_") and callable(fn)):
            continue
        grids = []
        for mark in getattr(fn, "pytestmark", []):
            if mark.name != "parametrize":
                continue
            names = [a.strip() for a in mark.args[0].split(",")]
            grids.append([dict(zip(names, v if len(names) > 1 else (v,))) for v in mark.args[1]])
        for combo in itertools.product(*grids) if grids else [()]:
            kwargs = {}
            for part in combo:
                kwargs.update(part)
            calls.append((name, fn, kwargs))
    return calls


def test_every_pin_passes_on_the_oracle_as_it_is():
    failed = []
    for name, fn, kwargs in _pin_calls():
        try:
            fn(**kwargs)
        except AssertionError:
            failed.append(name)
    assert not failed, failed


@pytest.mark.parametrize("label,before,after", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_a_planted_mistake_fails_a_pin(label, before, after, tmp_path, monkeypatch):
    text = open(SRC).read()
    assert text.count(before) == 1, label
    src = tmp_path / "lbm_oracle.c"
    src.write_text(text.replace(before, after))
    lib = tmp_path / "liblbm_oracle.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(lib), str(src), "-lm"])
    monkeypatch.setattr(oracle, "_SRC", str(src))
    monkeypatch.setattr(oracle, "_LIB", str(lib))
    monkeypatch.setattr(oracle, "_lib", None)
    caught = []
    for name, fn, kwargs in _pin_calls():
        try:
            fn(**kwargs)
        except (AssertionError, RuntimeError, ValueError, FloatingPointError):
            caught.append(name)
            break
    assert caught, f"no pin fails with the mistake: {label}"
