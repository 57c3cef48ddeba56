#!/usr/bin/env python3
"""Write the FP64 oracle's multipoles of the full-size workloads to
``tests/golden/<name>_oracle_B.npz``.

Calls only the oracle (``oracle/``) and the seeded input generator
(``paper_2405_14513_gb300/synth.py``, which holds none of the estimator's
arithmetic).  The oracle runs in slabs of n1 with a checkpoint after each
slab (``oracle.estimate_stream``), so an interrupted run resumes.

val384 holds no estimate: the oracle's discrete model [B]_d, the continuum
[B]_c of Eq. bs_lm at each bin's mean triangle and the discreteness weights
w = [B]_d / [B]_c for the paper's validation setup (Sec. III.B-C).

Workloads (seeded synthetic field: P = A k^-2, sigma_G = 0.1, f_NG = 0.5,
Kaiser beta = 0.5, seed 1, cast to float32 as the estimator reads it):

  c3  N_g = 512, L = 2000, 30 linear k1 bins over [N_g/12, N_g/3] k_f,
      (mu, t) step 0.025 (20 x 20 bins), l <= 6
  c2  N_g = 256, L = 1000, 20 linear k1 bins, (mu, t) step 0.025, l <= 6

The file holds B_l^m for even l (the estimator's 16 moments, NaN in empty
bins), the largest |B| of the odd-l moments and of the even-l imaginary
numerators (both cancel for a real field), the configuration, and a
fingerprint of the float32 field: its sha256, its sum and sum of squares in
float64, and 4096 values at fixed positions.  A test that regenerates the
field on another host checks the fingerprint before it compares.

  python tests/golden/make_oracle_golden.py c3|c2|val384 [--threads N] [--ckpt PATH]
"""
from __future__ import annotations

import argparse
import hashlib
import os
import platform
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O                      # noqa: E402
from paper_2405_14513_gb300 import synth            # noqa: E402

CONFIGS = {
    "c3": {"ng": 512, "box": 2000.0, "nk1": 30, "nmu": 20, "l_max": 6, "seed": 1},
    "c2": {"ng": 256, "box": 1000.0, "nk1": 20, "nmu": 20, "l_max": 6, "seed": 1},
}
# the paper's validation setup (Sec. III.B): N_g = 384, L = 215 Mpc, P = A k^-2
# with sigma_G = 0.1, f_NG = 0.5, beta = 1, k1 = 2.1 +- 0.1 Mpc^-1, (mu, t)
# step 0.05; its models, not an estimate
MODELS = {
    "val384": {"ng": 384, "box": 215.0, "edges": [2.0, 2.2], "nmu": 10, "l_max": 6, "sigma_g": 0.1,
               "f_ng": 0.5, "beta": 1.0, "index": -2.0},
}
N_SAMPLES = 4096


def make_input(cfg):
    """The float32 field the estimator reads, and its k1 edges."""
    f32 = synth.make_field(cfg["ng"], cfg["box"], cfg["seed"]).astype(np.float32)
    edges = synth.default_k1_edges(cfg["ng"], cfg["box"], cfg["nk1"])
    return f32, edges


def sample_positions(n_total):
    """4096 fixed positions spread over the flattened cube."""
    return (np.arange(N_SAMPLES, dtype=np.int64) * 2654435761) % n_total


def fingerprint(f32):
    flat = f32.reshape(-1)
    pos = sample_positions(flat.size)
    f64 = flat.astype(np.float64)
    return {"sha256": hashlib.sha256(f32.tobytes()).hexdigest(),
            "sum": float(np.sum(f64)), "sumsq": float(np.dot(f64, f64)),
            "sample_pos": pos, "sample_val": flat[pos].copy()}


def golden_path(name):
    return os.path.join(HERE, f"{name}_oracle_B.npz")


def write_models(name, threads):
    """The discrete model [B]_d, the continuum [B]_c at each bin's mean
    triangle and the discreteness weights w = [B]_d / [B]_c (even l)."""
    m = MODELS[name]
    A = synth.power_amplitude(m["ng"], m["box"], m["sigma_g"], m["index"])
    edges = np.asarray(m["edges"], dtype=np.float64)
    t0 = time.time()
    r = O.discreteness_weights(m["ng"], m["box"], edges, m["nmu"], m["nmu"], m["l_max"], A, m["index"],
                               m["f_ng"], m["beta"], nthreads=threads)
    ev = lambda a: O.select_even(a, m["l_max"])
    np.savez_compressed(golden_path(name), B_d=ev(r["d"]), B_c=ev(r["c"]), w=ev(r["w"]), k1_mu_t=r["k1_mu_t"],
                        k1_edges=edges, ng=m["ng"], box_len=m["box"], n_mu=m["nmu"], n_t=m["nmu"],
                        l_max=m["l_max"], A=A, index=m["index"], f_ng=m["f_ng"], beta=m["beta"],
                        sigma_g=m["sigma_g"], oracle_wall_s=time.time() - t0)
    print(f"{name}: wrote {golden_path(name)} ({time.time() - t0:.0f} s)", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(CONFIGS) + sorted(MODELS))
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--ckpt", default=None)
    args = ap.parse_args()
    if args.name in MODELS:
        return write_models(args.name, args.threads)
    cfg = CONFIGS[args.name]
    ckpt = args.ckpt or os.path.join(tempfile.gettempdir(), f"bisp_oracle_{args.name}.ckpt")
    t0 = time.time()
    f32, edges = make_input(cfg)
    fp = fingerprint(f32)
    print(f"field ready ({time.time() - t0:.1f} s), sha256 {fp['sha256']}", flush=True)
    t1 = time.time()
    res = O.estimate_stream(f32.astype(np.float64), cfg["box"], edges, cfg["nmu"], cfg["nmu"], cfg["l_max"],
                            ckpt=ckpt, verbose=True, nthreads=args.threads)
    wall = time.time() - t1
    l_max = cfg["l_max"]
    B = O.select_even(res["B"], l_max)
    odd = [O.lm_index(l, m) for l in range(1, l_max + 1, 2) for m in range(l + 1)]
    odd_max = float(np.nanmax(np.abs(res["B"][..., odd]))) if odd else 0.0
    im_even = float(np.abs(O.select_even(res["num_im"], l_max)).max())
    re_even = float(np.abs(O.select_even(res["num_re"], l_max)).max())
    np.savez_compressed(
        golden_path(args.name), B=B, k1_edges=edges,
        ng=cfg["ng"], box_len=cfg["box"], n_mu=cfg["nmu"], n_t=cfg["nmu"], l_max=l_max, seed=cfg["seed"],
        n_combos=res["n_combos"], oracle_wall_s=wall, threads=args.threads or os.cpu_count(),
        host=f"{platform.machine()} {os.cpu_count()} cores", odd_l_max_abs_B=odd_max,
        even_l_max_abs_num_im=im_even, even_l_max_abs_num_re=re_even,
        field_sha256=fp["sha256"], field_sum=fp["sum"], field_sumsq=fp["sumsq"],
        field_sample_pos=fp["sample_pos"], field_sample_val=fp["sample_val"])
    print(f"{args.name}: {res['n_combos']} combinations, {wall:.0f} s; wrote {golden_path(args.name)}", flush=True)


if __name__ == "__main__":
    main()
