"""Reading the FP64 oracle's multipoles of the full-size workloads (written by
``make_oracle_golden.py`` beside this file) and comparing an estimate with
them.  Plain numpy; no estimator arithmetic and no oracle code runs here.

Comparison metric (the tests' tolerance): per moment (l, m), the largest
over bins of |B - B_ref| / max(|B_ref|, 1e-2 max_bins |B_ref|) -- moments
that change sign pass through zero, so the error is floored at 1e-2 of the
moment's largest value -- with identical empty-bin (NaN) patterns.
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def path(name: str) -> str:
    return os.path.join(HERE, f"{name}_oracle_B.npz")


def load(name: str):
    """The stored result as a dict, or None if the file is absent."""
    p = path(name)
    if not os.path.exists(p):
        return None
    with np.load(p) as z:
        return {k: z[k] for k in z.files}


def moment_labels(l_max: int):
    return [f"B{l}{m}" for l in range(0, l_max + 1, 2) for m in range(l + 1)]


def field_check(sample_val, total_sum, total_sumsq, g, max_ulp=2):
    """Compare a regenerated float32 field with the stored fingerprint: the
    values at the stored positions within ``max_ulp`` units in the last place
    and the sum of squares to 1e-9.  Returns (ok, detail).  A field made by
    another FFT library agrees to float32 rounding (a few values one unit in
    the last place apart), which moves B by far less than the tolerance."""
    want = np.asarray(g["field_sample_val"], dtype=np.float32)
    got = np.asarray(sample_val, dtype=np.float32)
    ulp = np.abs(got.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64)).max()
    rel_sq = abs(total_sumsq - float(g["field_sumsq"])) / float(g["field_sumsq"])
    scale = np.sqrt(float(g["field_sumsq"]))
    abs_sum = abs(total_sum - float(g["field_sum"]))
    ok = ulp <= max_ulp and rel_sq <= 1e-9 and abs_sum <= 1e-6 * scale
    return ok, f"sample ulp {int(ulp)}, sum of squares rel {rel_sq:.2e}, sum diff {abs_sum:.2e}"


def floored_rel_err(got, ref):
    """Per-moment floored relative error (see the module docstring); raises
    if the empty-bin patterns differ."""
    fin = np.isfinite(ref)
    if not np.array_equal(fin, np.isfinite(got)):
        raise AssertionError("empty-bin pattern differs")
    g = np.where(fin, got, 0.0).reshape(-1, ref.shape[-1])
    r = np.where(fin, ref, 0.0).reshape(-1, ref.shape[-1])
    floor = 1e-2 * np.abs(r).max(axis=0, keepdims=True)
    return (np.abs(g - r) / np.maximum(np.abs(r), np.maximum(floor, 1e-300))).max(axis=0)


def raw_rel_err(got, ref):
    """Per-moment median of |B - B_ref| / |B_ref| over populated bins (no floor)."""
    fin = np.isfinite(ref) & (ref != 0)
    out = []
    for j in range(ref.shape[-1]):
        f = fin[..., j]
        out.append(float(np.median(np.abs(got[..., j][f] - ref[..., j][f]) / np.abs(ref[..., j][f]))))
    return np.array(out)
