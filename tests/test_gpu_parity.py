"""GPU parity of the CUDA estimator against the FP64 oracle.

Every check calls the CUDA library through its C ABI (``paper_2405_14513_gb300.api``)
on seeded synthetic fields and compares with the oracle on the same input:
the transformed planes (forward transform), the D fields of Step I on each
reduction grid (Eq. iFT), the combination table and its triangle counts
(Eqs. Ntri1/Ntri2), the per-combination sums (Eq. fftbs), the denominators
and the multipoles of Eq. bs_lm2_1.

Tolerances: relative error of B_l^m per bin, floored at 1e-2 of the largest
|B_l^m| of that moment (moments that change sign pass through zero), is at
most 1e-4 for the FP32-transform paths and 1e-10 for the FP64 path.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2405_14513_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_14513_gb300 import api  # noqa: E402

TOL = {"fp32": 1e-4, "mixed": 1e-4, "mixed_tc": 1e-4, "fp64": 1e-10}


def floored_rel_err(got, ref):
    """max over bins of |got - ref| / max(|ref|, 1e-2 max_bins |ref|), per moment."""
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got)), "empty-bin pattern differs"
    g = np.where(fin, got, 0.0).reshape(-1, ref.shape[-1])
    r = np.where(fin, ref, 0.0).reshape(-1, ref.shape[-1])
    floor = 1e-2 * np.abs(r).max(axis=0, keepdims=True)
    return (np.abs(g - r) / np.maximum(np.abs(r), np.maximum(floor, 1e-300))).max(axis=0)


class Case:
    def __init__(self, ng, L, n_k1, nmu, nt, l_max, seed=1, precision="mixed", edges=None):
        self.ng, self.L, self.nmu, self.nt, self.l_max = ng, L, nmu, nt, l_max
        self.edges = synth.default_k1_edges(ng, L, n_k1) if edges is None else np.asarray(edges)
        self.precision = precision
        field = synth.make_field(ng, L, seed)
        dt = np.float64 if precision == "fp64" else np.float32
        self.field = field.astype(dt)                     # what the GPU sees
        self.field64 = self.field.astype(np.float64)      # the same values for the oracle
        self.plan = api.Plan(ng, L, self.edges, nmu, nt, l_max, precision=precision, max_batch=2)
        self.ws = self.plan.workspace(2)
        d = torch.from_numpy(self.field).cuda()
        self.B = self.plan.estimate(d, self.ws).cpu().numpy()[0]
        torch.cuda.synchronize()
        self._oracle = None

    @property
    def oracle(self):
        if self._oracle is None:
            self._oracle = O.estimate(self.field64, self.L, self.edges, self.nmu, self.nt, self.l_max)
        return self._oracle


@pytest.fixture(scope="module")
def c64():
    # 64^3, L = 1000 Mpc/h, 6 linear k1 bins, (mu, t) step 0.1, l <= 6
    return Case(64, 1000.0, 6, 5, 5, 6)


@pytest.fixture(scope="module")
def c64_fp64():
    return Case(64, 1000.0, 6, 5, 5, 6, precision="fp64")


def test_forward_transform_planes(c64):
    cube = O.forward(c64.field64, c64.L)
    nz = c64.ng // 3
    for n in (0, 1, 7, nz):
        got = c64.plan.delta_plane(c64.ws, n)
        want = cube[:, :, n]
        assert np.abs(got - want).max() < 2e-6 * np.abs(want).max()


def test_step1_dfields_on_every_grid(c64):
    """Stored D fields of sampled combinations of every reduction grid in use
    (sides F x 2^q, F = 1, 3, 5, 7) against the oracle's direct evaluation."""
    tab = c64.plan.combo_table()
    rng = np.random.default_rng(3)
    seen = set()
    pick = np.concatenate([rng.choice(np.flatnonzero(tab["grid"] == M), size=min(6, int((tab["grid"] == M).sum())),
                                      replace=False) for M in np.unique(tab["grid"])])
    for k in pick:
        n1, n2, n3, r1, r2, r3 = tab["ints"][k]
        M = int(tab["grid"][k])
        for n, r in ((n1, r1), (n2, r2), (n3, r3)):
            key = (M, abs(int(n)), int(r))
            if key in seen:
                continue
            seen.add(key)
            got = c64.plan.dfield(c64.ws, M, abs(int(n)), int(r))
            want = O.dfield_at(c64.field64, c64.L, int(r), abs(int(n)), M)
            assert np.abs(got - want).max() < 2e-6 * max(np.abs(want).max(), 1e-30), key
    grids = {int(M) for M, _, _ in seen}
    assert grids == {int(M) for M in np.unique(tab["grid"])}
    for f in (3, 5, 7):
        assert any(M % f == 0 for M in grids), (f, grids)
    assert any(M & (M - 1) == 0 for M in grids), grids


def test_combination_table_matches_oracle(c64):
    """The product computes each combination's shape, orientation and bin on a
    route of its own (half-angle cosine law, the line of sight from the
    closing side, a search over bin edges); the oracle takes the cosine law
    and inverts Eq. orient.  The same combinations and triangle counts, the
    same shape and orientation to rounding, and the same bins except where the
    oracle's mu, t or K1 lies within 1e-12 of a bin edge (counted; at most one
    bin apart along that axis)."""
    tab = c64.plan.combo_table()
    geo = c64.plan.combo_geometry()
    ref = O.combos(c64.ng, c64.L, c64.edges, c64.nmu, c64.nt, half_space=True)
    key = lambda ints: [tuple(r) for r in ints]
    g = dict(zip(key(tab["ints"]), range(len(tab["ints"]))))
    o = dict(zip(key(ref["ints"]), range(len(ref["ints"]))))
    assert set(g) == set(o)
    gi = np.array([g[k] for k in o])
    oi = np.array(list(o.values()))
    assert np.array_equal(tab["ntri"][gi], ref["ntri"][oi])
    rg, ro = geo[gi], ref["geo"][oi]                  # product: mu, t, pz, cphi; oracle: K1, t, mu, pz, cphi, deg
    assert np.abs(rg[:, 0] - ro[:, 2]).max() < 1e-13
    assert np.abs(rg[:, 1] - ro[:, 1]).max() < 1e-15
    assert np.abs(rg[:, 2] - ro[:, 3]).max() < 1e-15
    sin_g = np.sqrt(np.maximum(0.0, 1.0 - rg[:, 2] ** 2))
    sin_o = np.sqrt(np.maximum(0.0, 1.0 - ro[:, 3] ** 2))
    assert np.abs(sin_g * rg[:, 3] - sin_o * ro[:, 4]).max() < 1e-11
    # bins: exact away from the edges
    def near(x, edges):
        return np.abs(x[:, None] - edges[None, :]).min(axis=1) < 1e-12 * np.maximum(1.0, np.abs(x))
    mu_e = 0.5 + np.arange(1, c64.nmu) / (2.0 * c64.nmu)
    t_e = 0.5 + np.arange(1, c64.nt) / (2.0 * c64.nt)
    edge = near(ro[:, 2], mu_e) | near(ro[:, 1], t_e) | near(ro[:, 0], c64.edges[1:-1])
    diff = tab["bin"][gi] != ref["bin"][oi]
    assert not np.any(diff & ~edge)
    assert diff.sum() <= max(1, 1e-4 * len(diff)), (int(diff.sum()), int(edge.sum()))
    nb = c64.nmu * c64.nt
    a, b = tab["bin"][gi][diff], ref["bin"][oi][diff]
    assert np.all(a // nb == b // nb) and np.all(np.abs(a % nb - b % nb) <= c64.nt)


def test_denominators_match_oracle(c64):
    den = c64.plan.denominator()
    ref = O.select_even(c64.oracle["den"], c64.l_max)
    assert np.abs(den - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("which", ["mixed", "fp64"])
def test_per_combination_sums(which, c64, c64_fp64):
    """Re S of Eq. fftbs per combination.  FP32 transforms carry about 1e-6
    relative error per field value, so the FP32-path bound is 1e-4 of the
    rms sum; the FP64 path is held to 1e-10."""
    c = c64 if which == "mixed" else c64_fp64
    tab = c.plan.combo_table()
    S = c.plan.combo_sums(c.ws)
    rng = np.random.default_rng(5)
    pick = rng.choice(len(S), size=400, replace=False)
    want = O.combo_sums(c.field64, c.L, tab["ints"][pick]).real
    scale = np.sqrt(np.mean(want ** 2))
    assert np.abs(S[pick] - want).max() < TOL[which] * scale


@pytest.mark.parametrize("which", ["mixed", "fp64"])
def test_multipoles_match_oracle(which, c64, c64_fp64):
    c = c64 if which == "mixed" else c64_fp64
    ref = O.select_even(c.oracle["B"], c.l_max)
    err = floored_rel_err(c.B, ref)
    assert err.max() < TOL[which], err


def _ring_maxc(ng):
    """Largest |u_x| of the lattice members of each ring (edges from the oracle)."""
    edges, _, _ = O.rings(ng)
    i = np.arange(-(ng // 2), ng // 2)
    ux, uy = np.meshgrid(i, i, indexing="ij")
    rad = np.hypot(ux, uy)
    return np.array([np.abs(ux[(rad >= edges[r]) & (rad < edges[r + 1])]).max() for r in range(len(edges) - 1)])


@pytest.mark.parametrize("prec", ["mixed", "mixed_tc"])
def test_reduction_grids_are_exact_and_rows_share_one(prec):
    """Every combination is summed on a grid of F x 2^q points (F = 1, 3, 5,
    7; a multiple of 4) above its aliasing bound maxc1 + maxc2 + maxc3.  The
    CUDA-core path takes the smallest such grid; the tensor-core path sums
    every r3 of one (n1, n2, r1, r2) row on one grid, the smallest above the
    largest bound among them."""
    ng, L = 64, 1000.0
    plan = api.Plan(ng, L, synth.default_k1_edges(ng, L, 6), 5, 5, 6, precision=prec)
    tab = plan.combo_table()
    plan.close()
    grids = np.array(sorted({f * 2 ** q for f in (1, 3, 5, 7) for q in range(2, 10)
                             if 8 <= f * 2 ** q <= ng}))
    maxc = _ring_maxc(ng)
    ints, M = tab["ints"], tab["grid"].astype(np.int64)
    bound = maxc[ints[:, 3]] + maxc[ints[:, 4]] + maxc[ints[:, 5]]
    assert np.all(np.isin(M, grids)) and np.all(M > bound)
    smallest = grids[np.searchsorted(grids, bound + 1)]
    if prec == "mixed":
        assert np.array_equal(M, smallest)
        return
    rows = {}
    for k, key in enumerate(map(tuple, ints[:, [0, 1, 3, 4]])):
        rows.setdefault(key, []).append(k)
    merged = 0
    for idx in rows.values():
        assert len(set(M[idx])) == 1
        assert M[idx[0]] == smallest[idx].max()
        merged += int(np.any(M[idx] > smallest[idx]))
    assert merged > 0


@pytest.mark.parametrize("prec", ["fp32", "mixed_tc"])
def test_fp32_plain_and_tensor_core_paths(prec):
    c = Case(64, 1000.0, 6, 5, 5, 6, precision=prec, seed=2)
    ref = O.select_even(c.oracle["B"], c.l_max)
    err = floored_rel_err(c.B, ref)
    assert err.max() < TOL[prec], err
    tab = c.plan.combo_table()
    S = c.plan.combo_sums(c.ws)
    pick = np.random.default_rng(8).choice(len(S), size=300, replace=False)
    want = O.combo_sums(c.field64, c.L, tab["ints"][pick]).real
    assert np.abs(S[pick] - want).max() < TOL[prec] * np.sqrt(np.mean(want ** 2))


def test_brute_force_16():
    """N_g = 16 against the direct triangle sums of Eq. binbs / Eq. Ntri1."""
    c = Case(16, 1000.0, 2, 5, 5, 6, precision="fp64", seed=4)
    ref = O.estimate(c.field64, c.L, c.edges, c.nmu, c.nt, c.l_max, direct=True)
    err = floored_rel_err(c.B, O.select_even(ref["B"], c.l_max))
    assert err.max() < TOL["fp64"], err


def test_batch_equals_single_calls(c64):
    f2 = synth.make_field(64, 1000.0, 9).astype(np.float32)
    d = torch.from_numpy(np.stack([c64.field, f2])).cuda()
    both = c64.plan.estimate(d, c64.ws).cpu().numpy()
    one = c64.plan.estimate(torch.from_numpy(f2).cuda()[None], c64.ws).cpu().numpy()[0]
    assert np.array_equal(both[0], c64.B, equal_nan=True)
    assert np.array_equal(both[1], one, equal_nan=True)


def test_host_entry_point_matches_device(c64):
    host = c64.plan.estimate_host(c64.field)[0]
    assert np.array_equal(host, c64.B, equal_nan=True)


def test_ragged_and_degenerate_configurations():
    """Smallest grid, a single k1 bin, l_max = 0, one (mu, t) bin and k1
    edges that leave bins empty."""
    for ng, L, edges, nmu, nt, lmax in [
        (8, 100.0, None, 1, 1, 0),
        (32, 500.0, np.array([0.03, 0.1, 0.12]), 3, 7, 2),
        (32, 500.0, synth.default_k1_edges(32, 500.0, 1), 16, 16, 8),
    ]:
        if edges is None:
            edges = synth.default_k1_edges(ng, L, 1)
        c = Case(ng, L, len(edges) - 1, nmu, nt, lmax, precision="fp64", edges=edges, seed=6)
        ref = O.select_even(c.oracle["B"], lmax)
        if np.isfinite(ref).any():
            assert floored_rel_err(c.B, ref).max() < TOL["fp64"]
        else:
            assert not np.isfinite(c.B).any()


# --------------------------------------------------------------------------
# Step II on tcgen05 (precision "mixed_tc", the benchmark's path)
# --------------------------------------------------------------------------
def test_tensor_core_ragged_and_degenerate_configurations():
    """The tcgen05 path on the smallest grid, one k1 bin, l_max = 0, one
    (mu, t) bin, empty bins, and a grid whose tiles hold few rows."""
    for ng, L, edges, nmu, nt, lmax in [
        (8, 100.0, None, 1, 1, 0),
        (32, 500.0, np.array([0.03, 0.1, 0.12]), 3, 7, 2),
        (32, 500.0, synth.default_k1_edges(32, 500.0, 1), 16, 16, 8),
        (16, 300.0, None, 4, 4, 4),
    ]:
        if edges is None:
            edges = synth.default_k1_edges(ng, L, 1)
        c = Case(ng, L, len(edges) - 1, nmu, nt, lmax, precision="mixed_tc", edges=edges, seed=7)
        assert c.plan.workspace_status(c.ws, 1) == 0
        ref = O.select_even(c.oracle["B"], lmax)
        if np.isfinite(ref).any():
            assert floored_rel_err(c.B, ref).max() < TOL["mixed_tc"]
        else:
            assert not np.isfinite(c.B).any()


def test_tensor_core_128_sampled_sums_and_cuda_core_agreement():
    """128^3 with 20 x 20 (mu, t) bins, several tiles per window class and
    every reduction grid: sampled Re S against the oracle, and B against the
    CUDA-core FP32 path."""
    ng, L = 128, 500.0
    tc = Case(ng, L, 12, 20, 20, 6, precision="mixed_tc", seed=11)
    assert tc.plan.workspace_status(tc.ws, 1) == 0
    tab = tc.plan.combo_table()
    S = tc.plan.combo_sums(tc.ws)
    pick = np.random.default_rng(12).choice(len(S), size=300, replace=False)
    want = O.combo_sums(tc.field64, L, tab["ints"][pick]).real
    assert np.abs(S[pick] - want).max() < TOL["mixed_tc"] * np.sqrt(np.mean(want ** 2))
    cc = Case(ng, L, 12, 20, 20, 6, precision="mixed", seed=11)
    assert floored_rel_err(tc.B, cc.B).max() < 2 * TOL["mixed_tc"]


@pytest.mark.slow
def test_tensor_core_full_size_512_sampled():
    """The benchmark's workload and launch configuration (512^3, L = 2000,
    30 k1 bins, 20 x 20 (mu, t), l <= 6, mixed_tc): Re S of sampled
    combinations, spread over the reduction grids, against the oracle."""
    ng, L = 512, 2000.0
    edges = synth.default_k1_edges(ng, L, 30)
    plan = api.Plan(ng, L, edges, 20, 20, 6, precision="mixed_tc")
    ws = plan.workspace(1)
    fd = synth.make_field_torch(ng, L, 1, device="cuda").float().contiguous()
    field = fd.cpu().numpy()                      # the values the GPU sees, for the oracle
    B = plan.estimate(fd[None], ws).cpu().numpy()[0]
    assert plan.workspace_status(ws, 1) == 0
    assert np.isfinite(B).any() and not np.isnan(B[np.isfinite(B)]).any()
    tab = plan.combo_table()
    S = plan.combo_sums(ws)
    rng = np.random.default_rng(13)
    pick = []
    for M in np.unique(tab["grid"]):
        idx = np.flatnonzero(tab["grid"] == M)
        pick.extend(rng.choice(idx, size=min(3, len(idx)), replace=False))
    pick = np.array(pick)
    want = O.combo_sums(field.astype(np.float64), L, tab["ints"][pick]).real
    # error relative to the magnitude a sum of M^2 terms of this size reaches
    scale = np.sqrt(np.mean(want ** 2))
    assert np.abs(S[pick] - want).max() < TOL["mixed_tc"] * scale
    plan.close()


# --------------------------------------------------------------------------
# Batched launches and captured estimates
# --------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["mixed_tc", "mixed", "fp64"])
def test_batched_launch_equals_single_fields(precision):
    """All fields of a batch go through each stage in one launch, each in its
    own workspace region; every field's result must equal its own estimate."""
    ng, L = 32, 500.0
    edges = synth.default_k1_edges(ng, L, 3)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = api.Plan(ng, L, edges, 4, 4, 6, precision=precision, max_batch=3)
    ws = plan.workspace(3)
    fields = torch.stack([torch.from_numpy(synth.make_field(ng, L, s)) for s in (21, 22, 23)]).to(dt).cuda()
    both = plan.estimate(fields.contiguous(), ws).cpu().numpy()
    for i in range(3):
        one = plan.estimate(fields[i:i + 1].contiguous(), ws).cpu().numpy()[0]
        assert np.array_equal(both[i], one, equal_nan=True), i
    assert plan.workspace_bytes(3) == 3 * plan.workspace_bytes(1)
    plan.close()


def test_captured_estimate_replays_exactly():
    """estimator_graph_create captures a batched estimate; launching the graph
    gives the estimate's result, and again after the inputs change in place."""
    ng, L = 64, 1000.0
    edges = synth.default_k1_edges(ng, L, 6)
    plan = api.Plan(ng, L, edges, 5, 5, 6, precision="mixed_tc", max_batch=2)
    ws = plan.workspace(2)
    fields = torch.stack([torch.from_numpy(synth.make_field(ng, L, s).astype(np.float32)) for s in (31, 32)]).cuda()
    want = plan.estimate(fields, ws).cpu().numpy()
    out = torch.full(plan.out_shape(2), float("nan"), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    g = plan.graph(fields, ws, out, stream=side)
    g.launch(stream=side)
    side.synchronize()
    assert np.array_equal(out.cpu().numpy(), want, equal_nan=True)
    fields[0].copy_(torch.from_numpy(synth.make_field(ng, L, 33).astype(np.float32)))
    want2 = plan.estimate(fields, ws).cpu().numpy()
    g.launch(stream=side)
    side.synchronize()
    assert np.array_equal(out.cpu().numpy(), want2, equal_nan=True)
    assert plan.workspace_status(ws, fields.shape[0]) == 0
    g.close()
    plan.close()


# --------------------------------------------------------------------------
# Grids of 3 x 2^k points (the paper's N_g = 384 study)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["mixed_tc", "fp64"])
def test_grid_of_3_times_2k_matches_oracle(precision):
    """N_g = 48 = 3 x 16: every transform length has a radix-3 stage."""
    c = Case(48, 700.0, 4, 5, 5, 6, precision=precision, seed=17)
    ref = O.select_even(c.oracle["B"], c.l_max)
    assert floored_rel_err(c.B, ref).max() < TOL[precision]


def test_grid_384_sampled_sums():
    """N_g = 384, L = 215 (the paper's validation grid): Re S of sampled
    combinations on every reduction grid against the oracle."""
    ng, L = 384, 215.0
    kf = 2 * np.pi / L
    edges = np.array([2.0, 2.2])                      # k1 = 2.1 +- 0.1
    assert edges[-1] <= ng / 3 * kf
    plan = api.Plan(ng, L, edges, 10, 10, 6, precision="mixed_tc")
    ws = plan.workspace(1)
    fd = synth.make_field_torch(ng, L, 3, beta=1.0, device="cuda").float().contiguous()
    field = fd.cpu().numpy()
    plan.estimate(fd[None], ws)
    assert plan.workspace_status(ws, 1) == 0
    tab = plan.combo_table()
    S = plan.combo_sums(ws)
    rng = np.random.default_rng(19)
    pick = []
    for M in np.unique(tab["grid"]):
        idx = np.flatnonzero(tab["grid"] == M)
        pick.extend(rng.choice(idx, size=min(4, len(idx)), replace=False))
    want = O.combo_sums(field.astype(np.float64), L, tab["ints"][np.array(pick)]).real
    assert np.abs(S[np.array(pick)] - want).max() < TOL["mixed_tc"] * np.sqrt(np.mean(want ** 2))
    plan.close()


def test_transform_tiles_do_not_change_results():
    """The plan's autotuner picks transform tiles by timing; rows are
    transformed independently, so two plans of one configuration (tuned
    separately) must give bit-identical estimates."""
    ng, L = 64, 1000.0
    edges = synth.default_k1_edges(ng, L, 6)
    f = torch.from_numpy(synth.make_field(ng, L, 41).astype(np.float32)).cuda()[None].contiguous()
    outs = []
    for _ in range(2):
        plan = api.Plan(ng, L, edges, 5, 5, 6, precision="mixed_tc")
        outs.append(plan.estimate(f, plan.workspace(1)).cpu().numpy())
        plan.close()
    assert np.array_equal(outs[0], outs[1], equal_nan=True)


# --------------------------------------------------------------------------
# One estimate split into shares (estimator_estimate_part)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["mixed_tc", "mixed", "fp64"])
def test_shares_sum_to_whole_estimate(precision):
    """The Step-II work of an estimate split into nparts shares: the shares'
    outputs add up to the whole estimate to FP64 rounding, for every field of
    a batch, whatever ran in the workspace before (each share clears the
    other shares' partial sums)."""
    ng, L = 64, 1000.0
    edges = synth.default_k1_edges(ng, L, 6)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = api.Plan(ng, L, edges, 5, 5, 6, precision=precision, max_batch=2)
    ws = plan.workspace(2)
    fields = torch.stack([torch.from_numpy(synth.make_field(ng, L, s)) for s in (51, 52)]).to(dt).cuda()
    whole = plan.estimate(fields, ws).cpu().numpy()
    for nparts in (2, 3, 7, 50):
        shares = [plan.estimate_part(fields, ws, p, nparts).cpu().numpy() for p in range(nparts)]
        total = np.sum(shares, axis=0)
        for i in range(2):
            assert floored_rel_err(total[i], whole[i]).max() < 1e-12, (nparts, i)
        if nparts == 2:
            fin = np.isfinite(whole)
            for s in shares:
                assert np.abs(s[fin]).max() > 0 and np.abs(s[fin] - whole[fin]).max() > 0
    assert np.array_equal(plan.estimate_part(fields, ws, 0, 1).cpu().numpy(), whole, equal_nan=True)
    for part, nparts in ((3, 3), (-1, 2), (0, 0)):
        with pytest.raises(api.BispError):
            plan.estimate_part(fields, ws, part, nparts)
    plan.close()


# --------------------------------------------------------------------------
# Per-l (mu, t) grids and logarithmic k1 bins
# --------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["mixed_tc", "fp64"])
def test_per_l_grids_and_log_k1_bins(precision):
    """The paper's binning: k1 bins of equal logarithmic width and (mu, t) grids
    of 12, 12, 8 and 6 bins per axis for l = 0, 2, 4, 6.  Each view's block
    matches the oracle estimate on that view's grid, and equals bit for bit
    the same moments of a plan that bins every l on that grid (Step II and
    the combination order do not depend on the (mu, t) grid)."""
    ng, L = 48, 500.0
    edges = synth.log_k1_edges(ng, L, 4)
    dt = np.float64 if precision == "fp64" else np.float32
    field = synth.make_field(ng, L, 61).astype(dt)
    plan = api.Plan(ng, L, edges, 1, 1, 6, precision=precision, mu_t_bins_l=[12, 12, 8, 6])
    assert [(v["l_lo"], v["l_hi"], v["n_mu"], v["n_t"], v["n_lm"]) for v in plan.views] == \
        [(0, 2, 12, 12, 4), (4, 4, 8, 8, 5), (6, 6, 6, 6, 7)]
    assert plan.out_shape(1) == (1, plan.out_doubles)
    assert plan.out_doubles == sum(v["n_bins"] * v["n_lm"] for v in plan.views)
    d = torch.from_numpy(field).cuda()[None].contiguous()
    blocks = plan.split(plan.estimate(d, plan.workspace(1)).cpu().numpy())
    dens = plan.split(plan.denominator()[None])
    for v, blk, den in zip(plan.views, blocks, dens):
        lm = slice((v["l_lo"] // 2) ** 2, (v["l_lo"] // 2) ** 2 + v["n_lm"])
        ref = O.estimate(field.astype(np.float64), L, edges, v["n_mu"], v["n_t"], 6)
        want = O.select_even(ref["B"], 6)[..., lm]
        assert floored_rel_err(blk[0], want).max() < TOL[precision], v
        dref = O.select_even(ref["den"], 6)[..., lm]
        assert np.abs(den[0] - dref).max() <= 1e-12 * np.abs(dref).max()
        one = api.Plan(ng, L, edges, v["n_mu"], v["n_t"], 6, precision=precision)
        same = one.estimate(d, one.workspace(1)).cpu().numpy()[0][..., lm]
        assert np.array_equal(blk[0], same, equal_nan=True), v
        one.close()
    plan.close()


# --------------------------------------------------------------------------
# Statistics over many mocks (estimator_stats_update, mocks.run_mocks)
# --------------------------------------------------------------------------
def test_mock_statistics_match_per_field_estimates():
    """Ten seeded mocks, four per captured launch (two graph replays and a
    partial batch of two): the device-side running count, mean and standard
    deviation of B equal those of the ten estimates made one by one."""
    from paper_2405_14513_gb300 import mocks
    ng, L = 32, 500.0
    edges = synth.default_k1_edges(ng, L, 3)
    plan = api.Plan(ng, L, edges, 4, 4, 6, precision="mixed_tc", max_batch=4)
    seeds = list(range(100, 110))
    c, mean, std = mocks.run_mocks(plan, seeds, 4).numpy()
    ws = plan.workspace(1)
    one = np.stack([plan.estimate(synth.make_field_torch(ng, L, s, device="cuda").float()[None].contiguous(),
                                  ws).cpu().numpy()[0] for s in seeds])
    fin = np.isfinite(one)
    assert np.array_equal(c, fin.sum(axis=0))
    ok = c > 1
    assert ok.any()
    scale = np.nanmax(np.abs(one))
    ref_mean = np.nanmean(np.where(fin, one, np.nan), axis=0)
    ref_std = np.nanstd(np.where(fin, one, np.nan), axis=0, ddof=1)
    assert np.abs(mean[ok] - ref_mean[ok]).max() <= 1e-12 * scale
    assert np.abs(std[ok] - ref_std[ok]).max() <= 1e-10 * scale
    assert np.isnan(mean[c == 0]).all()
    plan.close()


def test_tensor_core_waits_give_up_and_the_plan_recovers():
    """The tcgen05 Step II bounds every wait.  With the limit cut to one poll
    (a poll that reports at once; the producers' first copies cannot have
    landed by then), its blocks give up: they write NaN sums, and the
    workspace status reports BISP_TIMEOUT for that estimate only; every
    populated bin is then NaN.  With the default limit restored, the next
    estimate on the same plan and workspace is the normal one again, bit for
    bit, and reports success."""
    ng, L = 16, 1000.0
    edges = synth.default_k1_edges(ng, L, 3)
    field = torch.from_numpy(synth.make_field(ng, L, 2).astype(np.float32)).cuda()[None].contiguous()
    plan = api.Plan(ng, L, edges, 5, 5, 6, precision="mixed_tc")
    ws, other = plan.workspace(1), plan.workspace(1)
    ref = plan.estimate(field, ws).cpu().numpy()
    assert plan.workspace_status(ws, 1) == 0
    fin = np.isfinite(ref)
    assert fin.any()
    plan.set_wait_limit(1)
    bad = plan.estimate(field, ws).cpu().numpy()
    assert plan.workspace_status(ws, 1) == 5                  # BISP_TIMEOUT
    assert plan.workspace_status(ws, 1) == 0                  # reading it cleared it
    assert np.isnan(bad[fin]).all()
    plan.set_wait_limit(0)
    good = plan.estimate(field, other).cpu().numpy()
    assert plan.workspace_status(other, 1) == 0
    again = plan.estimate(field, ws).cpu().numpy()
    assert plan.workspace_status(ws, 1) == 0
    assert np.array_equal(again, ref, equal_nan=True) and np.array_equal(good, ref, equal_nan=True)
    plan.close()


def test_host_streaming_equals_host_estimates():
    """estimator_host_submit / estimator_host_wait: fields from host memory,
    the copy of one overlapping the estimate of the other, give the bits of
    estimator_estimate_host for each field; a third submission in flight and
    a wait with none are refused."""
    ng, L = 32, 600.0
    plan = api.Plan(ng, L, synth.default_k1_edges(ng, L, 3), 5, 5, 6, precision="mixed_tc", max_batch=2)
    fields = [torch.from_numpy(synth.make_field(ng, L, s).astype(np.float32)).pin_memory().numpy()
              for s in (5, 6, 7)]
    want = [plan.estimate_host(f) for f in fields]
    outs = [torch.empty(int(np.prod(plan.out_shape(1))), dtype=torch.float64).pin_memory().numpy()
            for _ in fields]
    stream = torch.cuda.current_stream()
    plan.host_submit(fields[0], outs[0], stream)
    plan.host_submit(fields[1], outs[1], stream)
    with pytest.raises(api.BispError):
        plan.host_submit(fields[2], outs[2], stream)
    got0 = plan.host_wait(stream)
    plan.host_submit(fields[2], outs[2], stream)
    got1 = plan.host_wait(stream)
    got2 = plan.host_wait(stream)
    with pytest.raises(api.BispError):
        plan.host_wait(stream)
    for g, w in zip((got0, got1, got2), want):
        assert np.array_equal(g.reshape(w.shape), w, equal_nan=True)
    plan.close()
