"""GPU parity of the spherical-shell m = 0 estimator (``estimator_shell_*``)
against the oracle's shell estimator: the shell triples, their bins,
triangle counts and denominators (plan time, FP64), the per-triple sums and
B_l^0 (FP32 fields, FP64 sums), and the point-field closed form shared with
the ring/plane estimator."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2405_14513_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_14513_gb300 import api  # noqa: E402

L_MAX = 6


def floored_rel_err(got, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got)), "empty-bin pattern differs"
    g = np.where(fin, got, 0.0).reshape(-1, ref.shape[-1])
    r = np.where(fin, ref, 0.0).reshape(-1, ref.shape[-1])
    floor = 1e-2 * np.abs(r).max(axis=0, keepdims=True)
    return (np.abs(g - r) / np.maximum(np.abs(r), np.maximum(floor, 1e-300))).max(axis=0)


@pytest.mark.parametrize("ng,L,nk", [(24, 500.0, 2), (32, 500.0, 3)])
def test_shell_estimator_matches_oracle(ng, L, nk):
    edges = synth.default_k1_edges(ng, L, nk)
    field = synth.make_field(ng, L, 17).astype(np.float32)
    plan = api.ShellPlan(ng, L, edges, 4, 4, L_MAX)
    ref = O.shell_triples(field.astype(np.float64), ng, L, edges, 4, 4, L_MAX)
    tab = plan.triples()
    assert plan.n_triples == len(ref["tri"]) > 0
    assert np.array_equal(tab["tri"], ref["tri"])
    assert np.array_equal(tab["ntri"], ref["ntri"])
    assert np.abs(tab["den"] - ref["den"]).max() <= 1e-10 * np.abs(ref["den"]).max()
    ws = plan.workspace()
    d = torch.from_numpy(field).cuda().contiguous()
    B = plan.estimate(d, ws).cpu().numpy()
    num = plan.sums(ws)
    for li in range(L_MAX // 2 + 1):
        rms = np.sqrt(np.mean(ref["num"][:, li] ** 2))
        assert np.abs(num[:, li] - ref["num"][:, li]).max() < 1e-4 * rms, li
    want = O.shell_estimate(field.astype(np.float64), L, edges, 4, 4, L_MAX)
    assert floored_rel_err(B, want).max() < 1e-4
    plan.close()


def test_shell_point_field_equals_ring_plane_monopole():
    """delta = delta_x0 - N^-3: both estimators give B_0^0 = a^3/V in every bin."""
    ng, L = 32, 500.0
    edges = synth.default_k1_edges(ng, L, 3)
    c = np.zeros((ng, ng, ng), dtype=np.float32)
    c[5, 9, 2] = 1.0
    c -= np.float32(1.0 / ng ** 3)
    a3v = (L ** 3 / ng ** 3) ** 3 / L ** 3
    d = torch.from_numpy(c).cuda().contiguous()
    shell = api.ShellPlan(ng, L, edges, 4, 4, L_MAX)
    Bs = shell.estimate(d, shell.workspace()).cpu().numpy()
    ring = api.Plan(ng, L, edges, 4, 4, L_MAX, precision="mixed_tc")
    Br = ring.estimate(d[None], ring.workspace(1)).cpu().numpy()[0]
    for B in (Bs[..., 0], Br[..., 0]):
        fin = np.isfinite(B)
        assert fin.sum() > 5
        np.testing.assert_allclose(B[fin], a3v, rtol=1e-4)
    shell.close()
    ring.close()


def test_shell_plan_rejects_unsupported():
    e = synth.default_k1_edges(256, 1000.0, 4)
    with pytest.raises(api.BispError):
        api.ShellPlan(256, 1000.0, e, 4, 4, 6)          # N_g above 128
    e = synth.default_k1_edges(32, 500.0, 3)
    with pytest.raises(api.BispError):
        api.ShellPlan(32, 500.0, e, 4, 4, 8)            # l_max above 6
