"""The served form: a burst of requests of two grid sizes through the
serving loop (continuous batching on several streams).  Each request's
answer must equal the same request estimated alone, and the loop must have
batched and overlapped work."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_14513_gb300 import serve, synth  # noqa: E402


def test_each_result_is_the_same_alone_and_in_the_mix():
    trace = serve.make_trace(24, rate=400.0, seed=5, grids=(32, 64), weights=(0.5, 0.5))
    srv = serve.Server(grids=(32, 64), precision="mixed_tc", max_batch={32: 4, 64: 4}, budget_gb=8.0, streams=3)
    lat, makespan, res = srv.run(trace, keep_results=True)
    assert sorted(res) == [r.rid for r in trace]
    assert any(k > 1 for _, k in srv.log), srv.log          # batched launches happened
    # every request's own launch reported success (each slot's workspace holds its status)
    assert sorted(srv.status) == [r.rid for r in trace] and not any(srv.status.values())
    for r in trace:
        p = srv.plans[r.ng]
        f = synth.make_field_torch(r.ng, serve.BOXES[r.ng], r.seed, device="cuda").float()[None].contiguous()
        alone = p.estimate(f, p.workspace(1)).cpu().numpy()[0]
        want = alone[r.k1_lo:r.k1_lo + r.n_k1, :, :, :r.n_lm()]
        assert np.array_equal(res[r.rid], want, equal_nan=True), r
    s = serve.summary(trace, lat, makespan)
    assert s["p50_s"] <= s["p99_s"] <= s["max_s"]
    srv.close()
