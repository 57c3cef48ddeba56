"""Splitting one field's estimate over ranks (CPU; gloo, world size 2).

The numerator of Eq. bs_lm2_1 is a sum over combinations, so estimates over
disjoint shares of the combinations, each divided by the whole denominator,
add up to the whole estimate.  The oracle's shares pin that on the CPU; the
sharded driver (`shard.estimate_sharded`: one share per rank, then a SUM
all-reduce) runs here on two gloo ranks whose plans compute their shares
with the oracle.  The GPU shares themselves are checked in
test_gpu_parity.py.
"""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_2405_14513_gb300 import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

NG, L, N_K1, NMU, NT, LMAX = 16, 1000.0, 2, 4, 4, 6


def _case():
    return synth.make_field(NG, L, 7), synth.default_k1_edges(NG, L, N_K1)


def _close(a, b, rtol=1e-12):
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(b)
    scale = np.abs(b[ok]).max()
    assert np.abs(a[ok] - b[ok]).max() <= rtol * scale


@pytest.mark.parametrize("nparts", [2, 3])
def test_oracle_shares_sum_to_whole(nparts):
    d, e = _case()
    whole = O.estimate(d, L, e, NMU, NT, LMAX)["B"]
    shares = [O.estimate_part(d, L, e, NMU, NT, LMAX, p, nparts) for p in range(nparts)]
    _close(sum(shares), whole)
    for s in shares:          # every share holds some of the sum, none all of it
        ok = ~np.isnan(whole)
        assert np.abs(s[ok]).max() > 0 and np.abs(s[ok] - whole[ok]).max() > 0
    with pytest.raises(ValueError):
        O.estimate_part(d, L, e, NMU, NT, LMAX, nparts, nparts)


class _OraclePlan:
    """Stands in for api.Plan on a CPU rank: its shares come from the oracle."""

    def __init__(self, d, e):
        self.d, self.e = d, e

    def estimate_part(self, delta, workspace, part, nparts, out=None, stream=None):
        B = O.select_even(O.estimate_part(self.d, L, self.e, NMU, NT, LMAX, part, nparts), LMAX)
        t = torch.from_numpy(np.ascontiguousarray(B))[None]
        if out is None:
            return t.clone()
        out.copy_(t)
        return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2405_14513_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d, e = _case()
        out = shard.estimate_sharded(_OraclePlan(d, e), None, None)
        q.put((rank, out.numpy()))
    finally:
        dist.destroy_process_group()


def test_sharded_estimate_on_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    d, e = _case()
    whole = O.select_even(O.estimate(d, L, e, NMU, NT, LMAX)["B"], LMAX)[None]
    for r in range(world):
        _close(got[r], whole)
    assert np.array_equal(got[0], got[1], equal_nan=True)
