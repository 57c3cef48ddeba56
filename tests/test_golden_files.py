"""The stored FP64 oracle results of the full-size workloads (``tests/golden/``)
hold what the oracle's own symmetries fix, and their field fingerprints
describe the seeded recipe's field.

For a real field the odd-l moments of Eq. bs_lm2_1 and the imaginary parts of
the even-l numerators cancel between the members of each +-n pair (the
oracle sums both), so a stored run that did not cover every ordered
combination, or mixed two fields, would show up here.
"""
import hashlib
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import golden_io  # noqa: E402

from paper_2405_14513_gb300 import synth  # noqa: E402


@pytest.mark.parametrize("name,ng,bins,populated", [("c2", 256, 8000, 5280), ("c3", 512, 12000, 7920)])
def test_stored_estimates_cancel_and_fill(name, ng, bins, populated):
    g = golden_io.load(name)
    assert g is not None
    B = g["B"]
    assert int(g["ng"]) == ng and B.shape[:3] == (len(g["k1_edges"]) - 1, int(g["n_mu"]), int(g["n_t"]))
    assert B.shape[-1] == 16 and B[..., 0].size == bins
    fin = np.isfinite(B)
    assert np.array_equal(fin, np.broadcast_to(fin[..., :1], fin.shape))        # a bin is empty for all moments
    assert int(fin[..., 0].sum()) == populated
    top = np.nanmax(np.abs(B))
    assert float(g["odd_l_max_abs_B"]) < 1e-12 * top
    assert float(g["even_l_max_abs_num_im"]) < 1e-12 * float(g["even_l_max_abs_num_re"])
    assert int(g["n_combos"]) > 0 and float(g["oracle_wall_s"]) > 0


def test_stored_fingerprint_is_the_recipes_field():
    """The 256^3 field regenerated here (numpy, float32) has the stored
    sha256; its sampled values and sum of squares pass the check the GPU
    test applies to a field made on the device."""
    g = golden_io.load("c2")
    f32 = synth.make_field(int(g["ng"]), float(g["box_len"]), int(g["seed"])).astype(np.float32)
    assert hashlib.sha256(f32.tobytes()).hexdigest() == str(g["field_sha256"])
    flat = f32.reshape(-1)
    f64 = flat.astype(np.float64)
    ok, detail = golden_io.field_check(flat[g["field_sample_pos"]], float(f64.sum()), float(f64 @ f64), g)
    assert ok, detail
    other = synth.make_field(int(g["ng"]), float(g["box_len"]), int(g["seed"]) + 1).astype(np.float32).reshape(-1)
    o64 = other.astype(np.float64)
    ok2, _ = golden_io.field_check(other[g["field_sample_pos"]], float(o64.sum()), float(o64 @ o64), g)
    assert not ok2


def test_validation_models():
    """The stored models of the paper's validation setup: the discrete and
    continuum monopoles are positive where populated and w = [B]_d/[B]_c."""
    g = golden_io.load("val384")
    assert g is not None
    d, c, w = g["B_d"], g["B_c"], g["w"]
    fin = np.isfinite(d[..., 0])
    assert fin.sum() > 50
    assert (d[..., 0][fin] > 0).all() and (c[..., 0][fin] > 0).all()
    assert np.allclose(w[..., 0][fin], d[..., 0][fin] / c[..., 0][fin], rtol=1e-12)
