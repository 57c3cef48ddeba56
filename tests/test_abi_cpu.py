"""CPU checks of the C ABI: the library builds and loads, exports every
entry point that include/bisp.h declares, and rejects bad plans before any
device work (no GPU is touched here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2405_14513_gb300 import api, build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "bisp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(estimator_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings():
    assert api.status_string(0) == "ok"
    assert api.status_string(1) == "invalid argument"
    assert api.status_string(2) == "unsupported grid size"
    assert api.status_string(99) == "unknown status"


@pytest.mark.parametrize("kw,code", [
    (dict(n_g=40), 2),
    (dict(n_g=4), 2),
    (dict(n_g=1536), 2),
    (dict(n_g=2048), 2),
    (dict(l_max=3), 1),
    (dict(l_max=10), 1),
    (dict(n_mu=0), 1),
    (dict(n_t=-1), 1),
    (dict(precision=7), 1),
    (dict(precision=-1), 1),
    (dict(max_batch=0), 1),
    (dict(box_len=0.0), 1),
    (dict(box_len=float("nan")), 1),
    (dict(edges="beyond"), 1),
    (dict(edges="descending"), 1),
    (dict(n_mu_l=[12, 12, 8, 6]), 1),                         # per-l mu bins without t bins
    (dict(n_mu_l=[12, 12, 8, 0], n_t_l=[12, 12, 8, 6]), 1),   # an empty grid
    (dict(n_mu_l=[12, 12, 8, 6], n_t_l=[12, 12, 8, 5000]), 1),
])
def test_plan_rejects_bad_arguments(kw, code):
    ng = kw.get("n_g", 32)
    L = kw.get("box_len", 500.0)
    e = synth.default_k1_edges(32, 500.0, 3)
    if kw.get("edges") == "beyond":
        e = e.copy()
        e[-1] *= 1.01
    elif kw.get("edges") == "descending":
        e = e[::-1].copy()
    st, msg = api.try_plan(ng, L, e, kw.get("n_mu", 4), kw.get("n_t", 4), kw.get("l_max", 6),
                           kw.get("precision", "mixed"), kw.get("max_batch", 1), kw.get("n_mu_l"), kw.get("n_t_l"))
    assert st == code, msg
    assert msg


def test_workspace_query_rejects_null_plan():
    lib = api.load()
    assert lib.estimator_workspace_bytes(None, 1) == 0
    assert lib.estimator_combo_table(None, 0, None, None, None, None) < 0
    lib.estimator_destroy(None)
