"""The host part of the plan (csrc/plan.cpp) on the CPU: the library's
combination enumeration, reduction-grid choice, tensor-core tiling and D-store
layout, built from the oracle's triangle counts by a small C++ driver
(tests/plan_host_check.cpp, compiled here with g++), checked against the
oracle's combination set and against the rules they must obey:

- every combination is summed on a grid of F x 2^q points (F = 1, 3, 5, 7, a
  multiple of 4) above its aliasing bound maxc1 + maxc2 + maxc3, on which the
  reduced triple sum is exact (the oracle pins that identity);
- the CUDA-core plan takes each combination's smallest such grid; the
  tensor-core plan sums all r3 of one (n1, n2, r1, r2) row on one grid, the
  smallest above the largest bound among them;
- every field a combination reads is stored on its grid;
- the tensor-core tiles cover every combination's partial sum exactly once,
  within the tile limits (128 rows, windows of 16-64 columns, at most 250
  staged fields, at least two shared-memory ring buffers)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2405_14513_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# (N_g, L, k1 bins, (mu, t) bins): a 2^k and a 3 x 2^k grid
CASES = {64: (64, 1000.0, 6, 5), 48: (48, 800.0, 6, 5)}


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("plan_host")
    exe = str(d / "plan_host_check")
    src = os.path.join(ROOT, "paper_2405_14513_gb300", "csrc")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-I", src,
                    os.path.join(ROOT, "tests", "plan_host_check.cpp"), os.path.join(src, "plan.cpp"), "-o", exe,
                    "-lpthread"], check=True)
    return d, exe


@pytest.fixture(scope="module", params=sorted(CASES))
def plans(request, driver):
    d, exe = driver
    NG, L, NK1, NMU = CASES[request.param]
    d = d / f"ng{NG}"
    d.mkdir()
    ntri, _ = O.ntri(NG)
    ntri.astype(np.int64).tofile(str(d / "ntri.bin"))
    edges = synth.default_k1_edges(NG, L, NK1)
    np.asarray(edges, dtype=np.float64).tofile(str(d / "edges.bin"))
    out = {}
    for tensor in (0, 1):
        pre = str(d / f"plan{tensor}")
        r = subprocess.run([exe, str(NG), repr(L), str(NK1), str(NMU), str(tensor), str(d / "ntri.bin"),
                            str(d / "edges.bin"), pre], check=True, capture_output=True, text=True)
        nc, ng_, nt, missing = map(int, r.stdout.split())
        out[tensor] = {
            "combos": np.fromfile(pre + ".combos", dtype=np.int32).reshape(nc, 7),
            "groups": np.fromfile(pre + ".groups", dtype=np.int64).reshape(ng_, 2),
            "tcrows": np.fromfile(pre + ".tcrows", dtype=np.int64).reshape(nt, 7),
            "missing": missing,
        }
    out.update(edges=edges, ng=NG, L=L, nmu=NMU)
    return out


def _ring_maxc(ng):
    edges, _, _ = O.rings(ng)
    i = np.arange(-(ng // 2), ng // 2)
    ux, uy = np.meshgrid(i, i, indexing="ij")
    rad = np.hypot(ux, uy)
    return np.array([np.abs(ux[(rad >= edges[r]) & (rad < edges[r + 1])]).max() for r in range(len(edges) - 1)])


def test_combinations_match_the_oracle(plans):
    ref = O.combos(plans["ng"], plans["L"], plans["edges"], plans["nmu"], plans["nmu"], half_space=True)
    want = {tuple(map(int, r)) for r in ref["ints"]}
    for tensor in (0, 1):
        got = [tuple(map(int, r)) for r in plans[tensor]["combos"][:, :6]]
        assert len(got) == len(set(got)) == len(want)
        assert set(got) == want


def test_grids_are_exact_and_chosen_by_the_rules(plans):
    NG = plans["ng"]
    grids = np.array(sorted({f * 2 ** q for f in (1, 3, 5, 7) for q in range(2, 10) if 8 <= f * 2 ** q <= NG}))
    maxc = _ring_maxc(NG)
    for tensor in (0, 1):
        c = plans[tensor]["combos"]
        M = c[:, 6].astype(np.int64)
        bound = maxc[c[:, 3]] + maxc[c[:, 4]] + maxc[c[:, 5]]
        assert np.all(np.isin(M, grids)) and np.all(M > bound)
        smallest = grids[np.searchsorted(grids, bound + 1)]
        if not tensor:
            assert np.array_equal(M, smallest)
            continue
        keys = c[:, [0, 1, 3, 4]].astype(np.int64)
        _, row = np.unique(keys, axis=0, return_inverse=True)
        row = row.ravel()
        top = np.zeros(row.max() + 1, dtype=np.int64)
        np.maximum.at(top, row, smallest)
        assert np.array_equal(M, top[row])
        assert np.any(M > smallest)            # some rows were merged onto a larger grid
        assert plans[tensor]["missing"] == 0
    assert plans[0]["missing"] == 0


def test_tensor_core_tiles_cover_every_sum_once(plans):
    g, t = plans[1]["groups"], plans[1]["tcrows"]
    want = np.concatenate([np.arange(p0, p0 + n) for p0, n in g])
    p0, n, col0, ncol, nrow, nslot, ring = t.T
    got = np.concatenate([np.arange(a, a + b) for a, b in zip(p0, n)])
    assert got.size == want.size and np.array_equal(np.sort(got), np.sort(want))
    assert np.all(nrow <= 128) and np.all(np.isin(ncol, (16, 32, 48, 64)))
    assert np.all(col0 + n <= ncol) and np.all(n >= 1)
    assert np.all(nslot <= 250) and np.all(ring >= 2)
