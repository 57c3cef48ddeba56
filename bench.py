#!/usr/bin/env python3
"""Benchmark of the GB300 estimator of the redshift-space bispectrum
multipoles B_l^m(k1, mu, t) on its headline workload.

Workload: N_g = 512, L = 2000 Mpc/h, 30 linear k1 bins over
[(N_g/12) k_f, (N_g/3) k_f], (mu, t) step 0.025 on [0.5, 1] (20 x 20 bins),
l <= 6 (16 moments).  Default precision "mixed_tc": FP32 transforms, the
Step-II triple sums on the tcgen05 tensor cores with each FP32 operand split
into TF32 high and low parts (FP32 accuracy), FP64 across chunks and in the
binning; --precision mixed runs Step II on the FP32 CUDA cores instead.
The input is the seeded synthetic non-Gaussian redshift-space field (P(k) =
A k^-2, sigma_G = 0.1, f_NG = 0.5, Kaiser beta = 0.5).

One step = one full estimate of one field (forward transform, Step I,
Step II, binning).  The metric is output (k1, mu, t) bins per second, each
bin carrying all 16 moments ("configs/s"; the line also gives the rate of
populated bins).  On N > 1 GPUs (one rank each; started by this script when
no launcher did) the default splits one field's Step II over the ranks with
one sum all-reduce of the output ("scaling": "strong"); --split replicas
gives each rank its own field instead (no collective, "scaling": "weak").
At N = 1 the 512^3 line also carries the batched-mock (c4) and served (c5)
results, the per-moment error against the stored FP64 oracle result, and
the CPU oracle baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--precision P]

--impl reference times the FP64 CPU oracle (the only other implementation
of the method; the paper publishes no code) on a bounded sample of the same
workload, on the host cores, and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LMAX = 6
# the workloads of the paper's method at three sizes (c3 is the headline);
# (mu, t) bins of step 0.025 (20 x 20) or 0.1 (5 x 5) on [0.5, 1]
WORKLOADS = {
    "c3": {"ng": 512, "box": 2000.0, "nk1": 30, "nmu": 20},
    "c2": {"ng": 256, "box": 1000.0, "nk1": 20, "nmu": 20},
    "c1": {"ng": 64, "box": 1000.0, "nk1": 6, "nmu": 5},
    # batched mocks: 256 seeded realisations, one plan, batches of 16 fields
    # per launch, each batch a captured CUDA graph
    "c4": {"ng": 128, "box": 500.0, "nk1": 12, "nmu": 10, "mocks": 256, "batch": 16},
    # serving: a Poisson trace (20 requests/s) of mixed N_g, k1-bin runs and l_max
    "c5": {"ng": 512, "box": 2000.0, "nk1": 30, "nmu": 10, "requests": 300, "rate": 20.0},
    # the spherical-shell m = 0 estimator against the ring/plane estimator on c1's workload
    "m0": {"ng": 64, "box": 1000.0, "nk1": 6, "nmu": 5, "shells": True},
    # the paper's validation (Sec. III.B): 50 realisations at N_g = 384, L = 215 Mpc,
    # beta = 1, k1 = 2.1 +- 0.1 Mpc^-1, against the stored discrete model [B]_d
    "val": {"ng": 384, "box": 215.0, "nk1": 1, "nmu": 10, "realisations": 50, "batch": 10},
}
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
TF32_PER_BF16 = 1.1 / 2.25          # nominal dense tensor rates of GB300
METRIC = "B_l^m(k1,mu,t) configs/s at N_g={ng}"


PRECISION_TEXT = {
    "mixed_tc": "FP32 transforms; Step-II products on tcgen05 tensor cores (TF32 high/low split, 3 passes, FP32 accuracy); FP32 sums per 16384-point chunk, FP64 across chunks and in the binning",
    "mixed": "FP32 transforms and products on CUDA cores, FP64 sums",
    "fp32": "FP32 throughout",
    "fp64": "FP64 throughout",
}


def workload(W, precision="mixed_tc"):
    from paper_2405_14513_gb300 import synth
    ng, box, nk1, nmu = W["ng"], W["box"], W["nk1"], W["nmu"]
    return {"workload": f"redshift-space bispectrum multipoles, N_g={ng}^3, L={box:g} Mpc/h, "
                        f"{nk1} linear k1 bins, (mu,t) step {0.5 / nmu:g} ({nmu}x{nmu}), l<=6 (16 moments)",
            "n_g": ng, "box_len": box, "n_k1": nk1, "n_mu": nmu, "n_t": nmu, "l_max": LMAX,
            "precision": f"{precision}: {PRECISION_TEXT[precision]}",
            "field": "seeded synthetic: P=A k^-2, sigma_G=0.1, f_NG=0.5, Kaiser beta=0.5",
            "l2": "inputs and D-field store larger than L2 (no flush needed)"}, \
        synth.default_k1_edges(ng, box, nk1)


# ----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=None):
        self.rows, self.proc = [], None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if index is not None:
            cmd += ["-i", str(index)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest x over all ranks (the slowest rank's time); x itself when
    no process group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank processes its own units (weak
    scaling), the job ends with the slowest rank."""
    return world * units_per_rank / seconds


# source that decides the Step-II kernel's DRAM traffic, per precision mode:
# (file, first line, end marker) regions; None = the file's start / end
STEP2_SOURCE = {
    "mixed_tc": [("step2_tc.cu", None, "template <int NC>\ncudaError_t launch_class"),
                 ("plan.hpp", "constexpr int kTcRows", "struct TcUnit"),
                 ("plan.cpp", "bool build_rings(", "int half_unit_bin("),
                 ("plan.cpp", "std::string build_tc(", "void build_views(")],
    "mixed": [("kernels.cu", None, None)], "fp32": [("kernels.cu", None, None)],
    "fp64": [("kernels.cu", None, None)],
}


def _traffic(ng, precision):
    """DRAM bytes of Step II per estimate from the committed ncu summary, if
    one was taken at this grid size on the kernel source as it is now.
    Returns (bytes, how) or (None, why)."""
    p = os.path.join(ROOT, "profiles", f"step2_dram_{precision}.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        if d.get("kernel_digest") != _kernel_digest(precision):
            return None, "the kernel changed since the DRAM capture"
        for c in d["captures"]:
            if int(c["n_g"]) == ng:
                return float(c["bytes_per_estimate"]), f"ncu capture at {ng}^3 ({c.get('source', '')})"
        # another grid size is not scaled: its L2 hit rate differs (the D
        # store of 256^3 is 1.8 GB, that of 512^3 17.9 GB)
        return None, f"no capture at {ng}^3"
    except (OSError, ValueError, KeyError, TypeError):
        return None, "no capture"


def _kernel_digest(precision):
    """Digest of the Step-II kernel source regions of a precision mode (the
    kernel and the tiling that decides what it reads)."""
    import hashlib
    h = hashlib.sha256()
    for name, start, end in STEP2_SOURCE[precision]:
        with open(os.path.join(ROOT, "paper_2405_14513_gb300", "csrc", name)) as fh:
            text = fh.read()
        a = text.index(start) if start else 0
        b = text.index(end, a) if end else len(text)
        h.update(text[a:b].encode())
    return h.hexdigest()[:16]


def fft_crosscheck(plan, field, ws, box):
    """Our forward transform against cuFFT: largest |ours - ref| / max |ref|
    over planes 0, 1 and N_g/3 of Delta = (V/N^3) DFT(delta), Delta(0) = 0,
    ours the FP32 planes the last estimate left in the workspace, ref
    torch.fft.fftn (cuFFT) in FP64.  Not timed."""
    import torch
    ng = plan.n_g
    ref = torch.fft.fftn(field.double()) * (box ** 3 / ng ** 3)
    ref[0, 0, 0] = 0
    err = 0.0
    for n in (0, 1, ng // 3):
        got = plan.delta_plane(ws, n)
        want = ref[:, :, n].cpu().numpy()
        err = max(err, float(np.abs(got - want).max() / np.abs(want).max()))
    del ref
    torch.cuda.empty_cache()
    return {"ref": "cuFFT via torch.fft.fftn, FP64", "planes": [0, 1, ng // 3], "max_rel_err": err}


def _peaks():
    """Measured peaks of this GPU type (written by the harness), or the
    fallback: bf16 dense TFLOP/s as a burst and sustained over a seconds-long
    loop, HBM copy GB/s, and which of the two sources."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        burst = float(d["bf16_tflops"])
        return burst, float(d.get("bf16_tflops_sustained", burst)), float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, 1700.0, 6800.0, "fallback"


def golden_errors(workload_name, field, out, W):
    """Per-moment error of this estimate against the FP64 oracle's stored
    multipoles of the same workload (tests/golden, written by the oracle
    alone), when the file exists and its field fingerprint matches the
    benchmark's field (the same seeded recipe: sampled values to float32
    rounding, sum of squares to 1e-9).  None otherwise."""
    import torch
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    try:
        import golden_io
    finally:
        sys.path.pop(0)
    g = golden_io.load(workload_name)
    if g is None or int(g["ng"]) != W["ng"] or float(g["box_len"]) != W["box"]:
        return None
    flat = field.reshape(-1)
    pos = torch.from_numpy(np.asarray(g["field_sample_pos"], dtype=np.int64)).to(flat.device)
    f64 = flat.double()
    ok, detail = golden_io.field_check(flat[pos].cpu().numpy(), float(f64.sum()), float((f64 * f64).sum()), g)
    del f64
    if not ok:
        return {"field_matches": False, "detail": detail}
    B = out.cpu().numpy()[0]
    ref = g["B"]
    err = golden_io.floored_rel_err(B, ref)
    raw = golden_io.raw_rel_err(B, ref)
    labels = golden_io.moment_labels(LMAX)
    return {"field_matches": True, "oracle": f"FP64 oracle, all {int(g['n_combos'])} ordered combinations "
                                            f"({float(g['oracle_wall_s']):.0f} s on {g['host']})",
            "max_err": float(err.max()), "max_err_per_lm": dict(zip(labels, map(float, err))),
            "median_raw_rel_err_per_lm": dict(zip(labels, map(float, raw))),
            "metric": "per moment: max over bins of |B - B_oracle| / max(|B_oracle|, 1e-2 max|B_oracle|)",
            "bins_compared": int(np.isfinite(ref[..., 0]).sum()), "tolerance": 1e-4}


# ----------------------------------------------------------------------------
def oracle_table(W, edges):
    """The oracle's combination table (its own triangle counts, Eq. Ntri2) and its wall time."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    c = O.combos(W["ng"], W["box"], edges, W["nmu"], W["nmu"], half_space=True, nthreads=os.cpu_count() or 1)
    return c, time.perf_counter() - t0


def cpu_baseline(W, edges, field64, n_bins, sample_pairs=2, seed=0, table=None):
    """The FP64 oracle, as it stands, on a bounded sample of the workload.

    The oracle enumerates the combinations (its own triangle counts, Eq.
    Ntri2), then computes the plane transforms, D fields and triple sums of
    every combination of `sample_pairs` random plane pairs.  Its full-workload
    time is extrapolated stage by stage: table time + plane time + per-field
    time x all (plane, ring) fields + per-combination time x all
    combinations of both signs of n (the oracle enumerates both)."""
    from oracle import oracle as O
    nthreads = os.cpu_count() or 1
    ng = W["ng"]
    t0 = time.perf_counter()
    c, t_tab = table if table is not None else oracle_table(W, edges)
    ints = c["ints"]
    n_half = len(ints)
    n_self = int(np.sum((ints[:, 0] == 0) & (ints[:, 1] == 0)))
    n_full = 2 * n_half - n_self
    key = ints[:, 0].astype(np.int64) * 4096 + ints[:, 1]      # combinations come grouped by pair
    starts = np.flatnonzero(np.r_[True, key[1:] != key[:-1]])
    pairs = ints[starts, :2]
    rng = np.random.default_rng(seed)
    pick = pairs[rng.choice(len(pairs), size=min(sample_pairs, len(pairs)), replace=False)]
    pk = set(int(p[0]) * 4096 + int(p[1]) for p in pick)
    sample = np.concatenate([ints[a:b] for a, b in zip(starts, np.r_[starts[1:], n_half])
                             if int(key[a]) in pk])
    times = []
    O.combo_sums(field64, W["box"], sample, nthreads=nthreads, times=times)
    t_planes, t_fields, t_sums = times
    nr = len(O.rings(ng)[1])
    nz = ng // 3
    fields = {(int(n), int(r)) for row in sample for n, r in zip(row[:3], row[3:])}
    t_full = (t_tab + t_planes + t_fields / len(fields) * (2 * nz + 1) * nr
              + t_sums / len(sample) * n_full)
    return {"value": n_bins / t_full, "unit": "configs/s", "cores": nthreads, "kind": "oracle",
            "sample": f"oracle table of all {n_half} combinations ({t_tab:.1f} s), then plane transforms, "
                      f"{len(fields)} D fields and {len(sample)} triple sums of {len(pick)} random plane "
                      f"pairs; full time extrapolated per stage to {(2 * nz + 1) * nr} fields and "
                      f"{n_full} combinations: {t_full:.0f} s",
            "wall_s": time.perf_counter() - t0 + (t_tab if table is None else 0.0), "extrapolated_s": t_full}


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return 0
    from paper_2405_14513_gb300 import synth
    W = WORKLOADS[args.workload]
    cfg, edges = workload(W, args.precision)
    cfg["precision"] = "fp64: the FP64 CPU oracle (plain definitions on the full N_g^2 plane, every ordered combination)"
    cfg["split"] = "replicas"
    n_bins = W["nk1"] * W["nmu"] * W["nmu"]
    field64 = synth.make_field(W["ng"], W["box"], 1).astype(np.float32).astype(np.float64)
    vals, walls = [], []
    table = oracle_table(W, edges)
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(W, edges, field64, n_bins, sample_pairs=1, seed=i, table=table)
        if i >= args.warmup:
            vals.append(r["value"])
            walls.append(r["wall_s"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC.format(ng=W["ng"]), "value": value, "unit": "configs/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": n_bins / value * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"kind": "oracle", "cores": r["cores"], "value": value, "unit": "configs/s",
                             "sample": "each step: " + r["sample"]},
            "e2e": {"value": value, "unit": "configs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_wall_s_per_step": statistics.median(walls)}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
def systems_summary(args):
    """The batched-mocks (c4) and served-trace (c5) workloads on this GPU,
    summarised for the headline line (each is also its own workload)."""
    import copy
    import torch
    a4 = copy.copy(args)
    a4.workload, a4.steps, a4.warmup = "c4", 2, 3
    l4 = run_batched(a4, emit=False)
    torch.cuda.empty_cache()
    a5 = copy.copy(args)
    a5.workload = "c5"
    l5 = run_serving(a5, emit=False)
    torch.cuda.empty_cache()
    keep4 = ("metric", "value", "unit", "ms_per_step", "single_job", "batched_over_single",
             "results_identical_to_single_job", "device_status", "e2e")
    keep5 = ("metric", "value", "unit", "ms_per_step", "served", "one_by_one", "served_over_one_by_one",
             "launch_batch_sizes", "device_status")
    return {"c4": dict({k: l4[k] for k in keep4}, workload=l4["config"]["workload"], mocks=l4["config"]["mocks"],
                       batch_per_launch=l4["config"]["batch_per_launch"]),
            "c5": dict({k: l5[k] for k in keep5}, workload=l5["config"]["workload"], server=l5["config"]["server"])}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2405_14513_gb300 import api, shard, synth

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    shares = args.split == "shares" and world > 1
    W = WORKLOADS[args.workload]
    ng = W["ng"]
    cfg, edges = workload(W, args.precision)
    cfg["split"] = "shares" if shares else "replicas"
    plan = api.Plan(ng, W["box"], edges, W["nmu"], W["nmu"], LMAX, precision=args.precision, max_batch=1)
    # replicas: one field per rank; shares: every rank holds the same field
    field = synth.make_field_torch(ng, W["box"], 1 if shares else 1 + rank, device=dev).to(torch.float32).contiguous()
    ws = plan.workspace(1, device=dev)
    out = torch.empty(plan.out_shape(1), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def step():
        if shares:
            shard.estimate_sharded(plan, field, ws, out=out)
        else:
            plan.estimate(field, ws, out=out, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    plan.set_timing(True)
    clocks = ClockSampler(index=local) if rank == 0 else None
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    clk = clocks.stop() if clocks else None
    ms = t0.elapsed_time(t1) / args.steps
    st_ms, st_n = plan.stage_times()
    plan.set_timing(False)
    flops = plan.stage_flops()
    ms = max_over_ranks(ms, device=dev)
    fields_per_step = 1 if shares else world
    value = job_rate(plan.n_bins, fields_per_step, ms / 1e3)
    finite = bool(torch.isfinite(out).any().item())
    populated = int(torch.isfinite(out[0, ..., 0]).sum().item())
    golden = golden_errors(args.workload, field, out, W) if rank == 0 else None
    fft_check = fft_crosscheck(plan, field, ws, W["box"])

    # end to end through the host side: every step copies a field in from
    # pinned host memory and its B out, copies timed.  Replicas stream the
    # fields through estimator_host_submit / _wait (the copy of one field in
    # overlaps the estimate of the one before); shares copy, estimate their
    # share and all-reduce.
    host = field.cpu().pin_memory()
    host_np = host.numpy()
    outs = [torch.empty(plan.out_shape(1), dtype=torch.float64).pin_memory().numpy() for _ in range(2)]
    out_pin = torch.from_numpy(outs[0])

    def step_host():
        field.copy_(host, non_blocking=True)
        shard.estimate_sharded(plan, field, ws, out=out)
        out_pin.copy_(out, non_blocking=True)
        stream.synchronize()

    if shares:
        step_host()
        barrier()
        te = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        te = (time.perf_counter() - te) / args.steps
        e2e_form = "copy in, shares of the estimate, one all-reduce, copy out"
    else:
        plan.host_submit(host_np, outs[0], stream)
        plan.host_wait(stream)
        barrier()
        te = time.perf_counter()
        plan.host_submit(host_np, outs[0], stream)
        for k in range(1, args.steps):
            plan.host_submit(host_np, outs[k % 2], stream)
            plan.host_wait(stream)
        plan.host_wait(stream)
        te = (time.perf_counter() - te) / args.steps
        e2e_form = "estimator_host_submit / estimator_host_wait (two fields in flight)"
    te = max_over_ranks(te, device=dev)
    e2e = {"value": job_rate(plan.n_bins, fields_per_step, te), "unit": "configs/s",
           "h2d_bytes_per_step": int(host.numel() * host.element_size()),
           "d2h_bytes_per_step": int(outs[0].size * 8), "form": e2e_form}

    # roofline of the dominant kernel (Step II), from its own events
    # Step II runs as one launch per block class; its time per estimate is the
    # sum of those launches, timed by events on the launching stream.  The
    # algorithmic flops are the method's real arithmetic: 4 per grid point of
    # each combination (Re of a complex product) + 6 per grid point of each
    # distinct pair product.
    s2_ms = st_ms["step2"] / args.steps
    achieved = flops["step2"] / (s2_ms / 1e3) / 1e12
    bf16, bf16_sus, _, src = _peaks()
    if args.precision == "mixed_tc":
        # Step II runs for most of every step, back to back over the timed
        # region: the peak sustained over a seconds-long loop applies
        peak = bf16_sus * TF32_PER_BF16
        roof = {"kernel": "k_step2_tc (Step II triple sums, tcgen05 kind::tf32)", "bound": "tensor",
                "peak_source": f"tf32 dense: bf16 sustained (seconds-long loop) of {src} x {TF32_PER_BF16:.4f} "
                               f"(nominal 1.1 / 2.25 PFLOP/s)",
                "frac_of_burst_peak": achieved / (bf16 * TF32_PER_BF16)}
    else:
        peak = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
        roof = {"kernel": "k_step2 (Step II triple sums, FP32 FMA)", "bound": "alu",
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (nominal max clock)"}
    traffic, traffic_how = _traffic(ng, args.precision)
    n2 = st_n["step2"] / args.steps          # Step-II launches per estimate; traffic is per launch, averaged
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": None if traffic is None else traffic / n2,
                 "traffic_per_estimate": traffic, "traffic_source": traffic_how,
                 "flops_per_estimate": flops["step2"], "ms_per_estimate": s2_ms, "launches_per_estimate": n2})
    # Step I (HBM-bound transforms): algorithmic bytes = the D store written
    # once + the kept planes of Delta read once, over its own event time
    _, _, hbm, src_ = _peaks()
    s1_ms = st_ms["step1"] / args.steps
    s1_bytes = plan.info["dstore_bytes"] + (ng // 3 + 1) * ng * ng * (16 if args.precision == "fp64" else 8)
    roof1 = {"kernels": "k_ring_gather + k_fft_rows_T (Step I, per reduction grid)", "bound": "hbm",
             "achieved": s1_bytes / (s1_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
             "frac": s1_bytes / (s1_ms / 1e3) / 1e9 / hbm, "bytes_per_estimate": s1_bytes,
             "ms_per_estimate": s1_ms, "peak_source": f"{src_} HBM copy bandwidth"}
    stage_share = {k: st_ms[k] / max(sum(st_ms.values()), 1e-9) for k in st_ms}
    launches = int(sum(st_n.values()))

    line = {"metric": METRIC.format(ng=ng), "value": value, "unit": "configs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if shares else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "e2e": e2e, "roofline": roof, "roofline_step1": roof1, "fft_crosscheck": fft_check,
            "gpu_launches": launches, "clocks": clk,
            "stage_ms_per_step": {k: v / args.steps for k, v in st_ms.items()},
            "stage_share": stage_share, "output_finite": finite,
            "bins": {"grid": int(plan.n_bins), "populated": populated,
                     "value_counts": "grid bins: every (k1, mu, t) bin of the output, each with 16 moments; "
                                     "empty bins (NaN) cost nothing",
                     "value_populated_bins": job_rate(populated, fields_per_step, ms / 1e3)},
            "vs_oracle": golden,
            "plan": {k: plan.info[k] for k in ("n_combos", "n_pairs", "n_items", "n_levels",
                                                "triple_products", "pair_products", "tc_row_points",
                                                "tc_lane_points", "tc_mma_products", "tc_staged_bytes",
                                                "dstore_bytes",
                                                "workspace_bytes")}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        f64 = field.double().cpu().numpy()
        del ws
        torch.cuda.empty_cache()
        line["cpu_baseline"] = cpu_baseline(W, edges, f64, plan.n_bins)
        if golden and golden.get("field_matches"):
            line["cpu_baseline"]["full_run"] = golden["oracle"] + " (the streamed oracle of the same definitions)"
    if rank == 0 and world == 1 and args.workload == "c3" and not args.no_systems:
        plan.close()
        del out, field
        torch.cuda.empty_cache()
        line["systems"] = systems_summary(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batched(args, emit=True):
    """Batched mocks (c4): every mock of the workload through one plan, in
    batches of W["batch"] fields per launch, each batch a captured CUDA graph;
    beside it, the same mocks one by one through estimator_estimate (the
    plain single-job form).  One step = all mocks."""
    import torch

    from paper_2405_14513_gb300 import api, synth

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = WORKLOADS[args.workload]
    ng, nm, G = W["ng"], W["mocks"], W["batch"]
    cfg, edges = workload(W, args.precision)
    cfg.update({"mocks": nm, "batch_per_launch": G, "graphs": nm // G,
                "l2": "fields (2.1 GB) and D stores larger than L2 (no flush needed)"})
    fields = torch.empty((nm, ng, ng, ng), dtype=torch.float32, device=dev)
    for i in range(nm):
        fields[i] = synth.make_field_torch(ng, W["box"], 1000 * rank + i + 1, device=dev).float()
    plan = api.Plan(ng, W["box"], edges, W["nmu"], W["nmu"], LMAX, precision=args.precision, max_batch=G)
    ws = plan.workspace(G, device=dev)
    out = torch.empty(plan.out_shape(nm), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(dev)
    graphs = [plan.graph(fields[j:j + G], ws, out[j:j + G], stream=stream) for j in range(0, nm, G)]

    def step():
        for g in graphs:
            g.launch(stream=stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    clocks = ClockSampler(index=local) if rank == 0 else None
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    stream.synchronize()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, device=dev)
    value = job_rate(nm * plan.n_bins, world, ms / 1e3)
    status = plan.workspace_status(ws, G, stream)

    # the plain single-job form: the same mocks one by one, no graph
    plan1 = api.Plan(ng, W["box"], edges, W["nmu"], W["nmu"], LMAX, precision=args.precision, max_batch=1)
    ws1 = plan1.workspace(1, device=dev)
    out1 = torch.empty(plan1.out_shape(nm), dtype=torch.float64, device=dev)
    for i in range(min(nm, 8)):
        plan1.estimate(fields[i:i + 1], ws1, out=out1[i:i + 1], stream=stream)
    stream.synchronize()
    t0.record(stream)
    for i in range(nm):
        plan1.estimate(fields[i:i + 1], ws1, out=out1[i:i + 1], stream=stream)
    t1.record(stream)
    stream.synchronize()
    ms1 = max_over_ranks(t0.elapsed_time(t1), device=dev)
    same = bool(torch.equal(torch.nan_to_num(out, nan=-1.0), torch.nan_to_num(out1, nan=-1.0)))

    # end to end: pinned host fields in, results out, copies timed
    host = fields.cpu().pin_memory()
    out_h = torch.empty(out.shape, dtype=torch.float64).pin_memory()
    te = time.perf_counter()
    for _ in range(args.steps):
        fields.copy_(host, non_blocking=True)
        step()
        out_h.copy_(out, non_blocking=True)
        stream.synchronize()
    te = max_over_ranks((time.perf_counter() - te) / args.steps, device=dev)
    line = {"metric": f"B_l^m(k1,mu,t) configs/s, {nm} mocks at N_g={ng} (batched, CUDA graphs)",
            "value": value, "unit": "configs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": cfg,
            "e2e": {"value": job_rate(nm * plan.n_bins, world, te), "unit": "configs/s",
                    "h2d_bytes_per_step": int(host.numel() * 4), "d2h_bytes_per_step": int(out_h.numel() * 8)},
            "single_job": {"value": job_rate(nm * plan.n_bins, world, ms1 / 1e3), "unit": "configs/s",
                           "ms_per_step": ms1, "form": "estimator_estimate, one mock per call, no graph"},
            "batched_over_single": ms1 / ms, "results_identical_to_single_job": same,
            "device_status": status, "clocks": clk,
            "gpu_launches": len(graphs) * (3 + 2 * plan.info["n_levels"] + 3 + 3)}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    for g in graphs:
        g.close()
    plan.close()
    plan1.close()
    return line if not emit else 0


def run_shells(args):
    """The spherical-shell estimator of the m = 0 multipoles (B_l^0 only)
    against the ring/plane estimator (all 16 moments) on the same field and
    bins: device time per estimate of each, and how their B_l^0 compare (the
    two bin triangles differently, so they agree in expectation, not bin by
    bin; on a point field both give a^3/V exactly)."""
    import torch

    from paper_2405_14513_gb300 import api, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    W = WORKLOADS[args.workload]
    ng = W["ng"]
    cfg, edges = workload(W, "mixed_tc")
    cfg["workload"] = cfg["workload"] + "; spherical shells (ring edges), m = 0"
    shell = api.ShellPlan(ng, W["box"], edges, W["nmu"], W["nmu"], LMAX)
    ring = api.Plan(ng, W["box"], edges, W["nmu"], W["nmu"], LMAX, precision="mixed_tc")
    field = synth.make_field_torch(ng, W["box"], 1, device=dev).to(torch.float32).contiguous()
    wss, wsr = shell.workspace(device=dev), ring.workspace(1, device=dev)
    outs = torch.empty(shell.out_shape(), dtype=torch.float64, device=dev)
    outr = torch.empty(ring.out_shape(1), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize(dev)
        return t0.elapsed_time(t1) / args.steps

    clocks = ClockSampler(index=0)
    ms_s = timed(lambda: shell.estimate(field, wss, out=outs, stream=stream))
    ms_r = timed(lambda: ring.estimate(field[None], wsr, out=outr, stream=stream))
    clk = clocks.stop()
    Bs = outs.cpu().numpy()
    Br = outr.cpu().numpy()[0][..., [0, 1, 4, 9][: LMAX // 2 + 1]]      # the m = 0 moments, l = 0, 2, 4, 6
    both = np.isfinite(Bs) & np.isfinite(Br)
    agree = {}
    for li in range(LMAX // 2 + 1):
        a, b = Bs[..., li][both[..., li]], Br[..., li][both[..., li]]
        scale = np.abs(b).max() if b.size else 1.0
        agree[f"l={2 * li}"] = {"bins": int(b.size), "median_abs_diff_over_max": float(np.median(np.abs(a - b)) / scale),
                                "correlation": float(np.corrcoef(a, b)[0, 1]) if b.size > 2 else None}
    # point field: both give a^3/V
    c = torch.zeros((ng, ng, ng), dtype=torch.float32, device=dev)
    c[3, 5, 7] = 1.0
    c -= 1.0 / ng ** 3
    a3v = (W["box"] ** 3 / ng ** 3) ** 3 / W["box"] ** 3
    ps = shell.estimate(c, wss).cpu().numpy()[..., 0]
    pr = ring.estimate(c[None].contiguous(), wsr).cpu().numpy()[0][..., 0]
    point = {"shell_max_rel_err": float(np.nanmax(np.abs(ps / a3v - 1))),
             "ring_plane_max_rel_err": float(np.nanmax(np.abs(pr / a3v - 1)))}
    n_bins = shell.n_k1 * shell.n_mu * shell.n_t
    line = {"metric": f"B_l^0(k1,mu,t) configs/s at N_g={ng}, spherical shells (m = 0 only)",
            "value": n_bins / (ms_s / 1e3), "unit": "configs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg, "clocks": clk,
            "shells": {"n_shells": shell.n_shells, "n_triples": shell.n_triples, "moments": LMAX // 2 + 1},
            "ring_plane": {"configs_per_s": n_bins / (ms_r / 1e3), "ms_per_step": ms_r, "moments": ring.n_lm},
            "agreement_B_l0": agree, "point_field": point}
    print(json.dumps(line), flush=True)
    shell.close()
    ring.close()
    return 0


def run_serving(args, emit=True):
    """Serving (c5): the seeded 300-request Poisson trace through the serving
    loop (resident plans, continuous batching on 4 streams, HBM budget), then
    the same trace one request at a time on one stream (the plain
    single-job form).  Latency = completion - arrival, queueing included."""
    import torch

    from paper_2405_14513_gb300 import serve

    rank, world, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    W = WORKLOADS[args.workload]
    trace = serve.make_trace(W["requests"], rate=W["rate"], seed=0)
    srv = serve.Server(precision=args.precision, budget_gb=160.0, streams=4)
    warm = serve.make_trace(24, rate=200.0, seed=99)
    srv.run(warm)
    clocks = ClockSampler(index=local)
    lat, span, _ = srv.run(trace)
    clk = clocks.stop()
    served = serve.summary(trace, lat, span)
    batches = collections.Counter(k for _, k in srv.log)
    srv.sched.slots = []
    torch.cuda.empty_cache()
    lat1, span1, _ = srv.run(trace, one_by_one=True)
    single = serve.summary(trace, lat1, span1)
    status = max(srv.status.values(), default=0)
    cfg = {"workload": "served estimator requests: Poisson arrivals 20/s, N_g in {64,128,256,512} "
                       "(weights 0.4/0.3/0.2/0.1, L 1000/500/1000/2000 Mpc/h), runs of 4-30 of 30 default "
                       "k1 bins, (mu,t) step 0.05, l_max in {2,4,6}; seeded trace of 300 requests",
           "precision": f"{args.precision}: {PRECISION_TEXT[args.precision]}",
           "server": "one resident plan per N_g (30 bins, l<=6; answers are slices); up to 16/8/4/1 "
                     "fields per launch for N_g 64/128/256/512; 4 streams; 160 GB budget",
           "field": "seeded synthetic, generated on the device per request (part of the latency)"}
    line = {"metric": "served B_l^m configs/s and p50/p99 latency (s)", "value": served["configs_per_s"],
            "unit": "configs/s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": span * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg, "served": served, "one_by_one": single,
            "served_over_one_by_one": served["configs_per_s"] / single["configs_per_s"],
            "launch_batch_sizes": dict(sorted(batches.items())), "device_status": status, "clocks": clk}
    if emit:
        print(json.dumps(line), flush=True)
    srv.close()
    return line if not emit else 0


def launch_decision(gpus: int, env) -> tuple:
    """How this process runs for --gpus N: ("run", None) as one rank of an
    existing launch (or alone for N = 1), ("spawn", None) to start N ranks
    itself with torch.distributed.run on this node, or ("error", why) when
    the launch it is part of has another world size."""
    world = env.get("WORLD_SIZE")
    if world is None:
        return ("spawn", None) if gpus > 1 else ("run", None)
    if int(world) != gpus:
        return ("error", f"--gpus {gpus} but WORLD_SIZE={world}: launch one rank per GPU")
    return ("run", None)


def rank_command(gpus: int, argv, port: int) -> list:
    """The torch.distributed.run command line that runs this script as `gpus`
    ranks of one node (rendezvous on 127.0.0.1:port) with the same arguments."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
            "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + list(argv)


def spawn_ranks(gpus: int, argv) -> int:
    """Run this script as `gpus` ranks of one node; returns their exit status."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    return subprocess.call(rank_command(gpus, argv, port))


def run_validation(args):
    """The paper's statistical validation (Sec. III.B): the mean over 50
    seeded realisations against the discrete model [B]_d (stored by the
    oracle in tests/golden/val384_oracle_B.npz), per moment and bin:
    Delta = |mean - [B]_d| / sigma, sigma the standard error of the mean over
    the realisations, and the discreteness weights w = [B]_d / [B]_c the
    oracle stored beside it.  One step = all realisations."""
    import torch

    from paper_2405_14513_gb300 import api, synth

    rank, world, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import golden_io
    sys.path.pop(0)
    g = golden_io.load("val384")
    if g is None:
        print(json.dumps({"error": "tests/golden/val384_oracle_B.npz missing"}), flush=True)
        return 1
    W = WORKLOADS["val"]
    ng, L, nr, G = W["ng"], W["box"], W["realisations"], W["batch"]
    edges = np.asarray(g["k1_edges"])
    plan = api.Plan(ng, L, edges, W["nmu"], W["nmu"], LMAX, precision=args.precision, max_batch=G)
    ws = plan.workspace(G, device=dev)
    stream = torch.cuda.current_stream(dev)
    kw = dict(sigma_g=float(g["sigma_g"]), f_ng=float(g["f_ng"]), beta=float(g["beta"]), device=dev)
    fields = torch.empty((G, ng, ng, ng), dtype=torch.float32, device=dev)
    B = []
    status = 0
    t_est = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for s0 in range(0, nr, G):
        for i in range(G):
            fields[i] = synth.make_field_torch(ng, L, 1 + s0 + i, **kw).float()
        e0.record(stream)
        out = plan.estimate(fields, ws, stream=stream)
        e1.record(stream)
        status = max(status, plan.workspace_status(ws, G, stream))
        t_est += e0.elapsed_time(e1)
        B.append(out.cpu().numpy()[:, 0])                # [field][mu][t][lm]
    B = np.concatenate(B)
    mean, sem = B.mean(0), B.std(0, ddof=1) / np.sqrt(nr)
    Bd = g["B_d"][0]
    labels = golden_io.moment_labels(LMAX)
    fin = np.isfinite(Bd[..., 0]) & np.isfinite(mean[..., 0])
    per = {}
    for j, lab in enumerate(labels):
        with np.errstate(invalid="ignore", divide="ignore"):
            d = np.abs(mean[..., j] - Bd[..., j]) / sem[..., j]
        dv = d[fin]
        w = g["w"][0][..., j][fin]
        per[lab] = {"chi2_per_bin": float(np.mean(dv ** 2)), "frac_le_3": float(np.mean(dv <= 3)),
                    "n_3_to_5": int(np.sum((dv > 3) & (dv <= 5))), "n_5_to_7": int(np.sum((dv > 5) & (dv <= 7))),
                    "n_gt_7": int(np.sum(dv > 7)), "max": float(dv.max()),
                    "delta_map": np.round(np.where(fin, d, np.nan), 2).tolist(),
                    "w_median_abs_dev_from_1": float(np.nanmedian(np.abs(w - 1))) if np.isfinite(w).any() else None}
    frac = (mean[..., 0] - Bd[..., 0]) / Bd[..., 0]
    line = {"metric": "validation: Delta_l^m = |mean - [B]_d| / sigma over 50 realisations (paper Sec. III.B)",
            "value": float(np.mean([p["frac_le_3"] for p in per.values()])), "unit": "fraction of bins with Delta<=3",
            "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": t_est, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"N_g={ng}^3, L={L:g} Mpc, P=A k^-2 (sigma_G={float(g['sigma_g'])}), "
                                   f"f_NG={float(g['f_ng'])}, beta={float(g['beta'])}, k1 in [{edges[0]}, {edges[1]}) "
                                   f"Mpc^-1, (mu,t) step 0.05, l<=6, {nr} realisations",
                       "precision": f"{args.precision}: {PRECISION_TEXT[args.precision]}",
                       "model": "[B]_d of the FP64 oracle (tests/golden/val384_oracle_B.npz)"},
            "bins": int(fin.sum()), "monopole_fractional_deviation": [float(np.nanmin(frac[fin])),
                                                                      float(np.nanmax(frac[fin]))],
            "per_moment": per, "device_status": status}
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS),
                    help="c3: 512^3 headline (default); c2: 256^3, L=1000, 20 k1 bins; c1: 64^3, L=1000, "
                         "6 bins; c4: 256 mocks of 128^3 in batched graphs; c5: served request trace; "
                         "m0: the spherical-shell m = 0 estimator against the ring/plane one at 64^3; "
                         "val: the paper's validation, 50 realisations at 384^3 against [B]_d")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-systems", action="store_true",
                    help="c3 at N = 1: skip the batched (c4) and served (c5) summaries added to the line")
    ap.add_argument("--split", default="shares", choices=["replicas", "shares"],
                    help="N > 1: shares (one field's Step II split over the ranks, one all-reduce of the "
                         "output; strong scaling; the default) or replicas (a field per rank, weak scaling)")
    ap.add_argument("--precision", default="mixed_tc", choices=["mixed_tc", "mixed", "fp32", "fp64"],
                    help="mixed_tc: Step II on tcgen05 (the default); mixed: on FP32 CUDA cores")
    args = ap.parse_args(argv)
    what, why = launch_decision(args.gpus, os.environ)
    if what == "error":
        print(json.dumps({"error": why}), flush=True)
        return 2
    if what == "spawn":
        return spawn_ranks(args.gpus, argv)
    if args.impl == "reference":
        return run_reference(args)
    if "mocks" in WORKLOADS[args.workload]:
        return run_batched(args)
    if "requests" in WORKLOADS[args.workload]:
        return run_serving(args)
    if "shells" in WORKLOADS[args.workload]:
        return run_shells(args)
    if "realisations" in WORKLOADS[args.workload]:
        return run_validation(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
