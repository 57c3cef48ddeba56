"""estimator_estimate_static: the estimate for callers that cannot allocate
device memory (code under a memory manager that owns the device heap, plugins
handed a device and a stream but no allocator) keeps its workspace in a
static device array of the library.  Its results must equal those of
estimator_estimate with a caller workspace on calls in a row, whatever an
earlier call (of another plan, precision or field) left in the array, and
plans too large for the array must be refused with a clear error.

This file is collected last on purpose: the first call of the entry point
on a device loads the array, and the test must pass both on its own in a
fresh process and after every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_14513_gb300 import api, synth  # noqa: E402

TOL = 1e-4   # the FP32-transform tolerance of the GPU parity tests


def _lib():
    lib = api.load()
    lib.estimator_estimate_static.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    lib.estimator_estimate_static.restype = C.c_int
    lib.estimator_static_scratch_bytes.argtypes = []
    lib.estimator_static_scratch_bytes.restype = C.c_size_t
    return lib


def _floored_rel_err(got, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got)), "empty-bin pattern differs"
    g = np.where(fin, got, 0.0).reshape(-1, ref.shape[-1])
    r = np.where(fin, ref, 0.0).reshape(-1, ref.shape[-1])
    floor = 1e-2 * np.abs(r).max(axis=0, keepdims=True)
    return (np.abs(g - r) / np.maximum(np.abs(r), np.maximum(floor, 1e-300))).max()


def _fields(ng, L, seeds, dtype=np.float32):
    return torch.from_numpy(np.stack([synth.make_field(ng, L, s).astype(dtype) for s in seeds])).cuda().contiguous()


def _static(lib, plan, field, stream):
    out = torch.full(plan.out_shape(field.shape[0]), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.estimator_estimate_static(plan._h, C.c_void_p(field.data_ptr()), field.shape[0],
                                       C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert st == 0, lib.estimator_last_error().decode()
    assert plan.workspace_status(None, field.shape[0], stream) == 0
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", ["mixed", "mixed_tc"])
@pytest.mark.parametrize("batch", [1, 2])
def test_static_scratch_matches_caller_workspace(precision, batch):
    lib = _lib()
    stream = torch.cuda.current_stream()
    ng, L = (64, 1000.0) if batch == 1 else (48, 800.0)
    plan = api.Plan(ng, L, synth.default_k1_edges(ng, L, 6), 5, 5, 6, precision=precision, max_batch=batch)
    assert 0 < plan.workspace_bytes(batch) <= lib.estimator_static_scratch_bytes()
    # leave another plan's data (FP64 values, other layout) in the array first
    other = api.Plan(32, 600.0, synth.default_k1_edges(32, 600.0, 3), 5, 5, 6, precision="fp64")
    _static(lib, other, _fields(32, 600.0, [7], np.float64), stream)
    other.close()
    fa, fb = _fields(ng, L, range(3, 3 + batch)), _fields(ng, L, range(20, 20 + batch))
    ref_b = plan.estimate(fb, plan.workspace(batch)).cpu().numpy()
    for call, (f, tag) in enumerate([(fa, "A"), (fb, "B")]):
        got = _static(lib, plan, f, stream)
        if tag == "B":
            err = _floored_rel_err(got, ref_b)
            assert err <= TOL, f"call {call}: relative error {err:.3e}"


@pytest.mark.parametrize("precision", ["mixed", "mixed_tc"])
def test_workspace_contents_are_scratch(precision):
    """Nothing of a workspace is read before the estimate writes it: a
    workspace filled with NaN gives the bits of a zeroed one."""
    ng, L = 48, 800.0
    plan = api.Plan(ng, L, synth.default_k1_edges(ng, L, 6), 5, 5, 6, precision=precision)
    f = _fields(ng, L, [4])
    ws0 = torch.zeros(plan.workspace_bytes(1), dtype=torch.uint8, device="cuda")
    wsn = torch.full((plan.workspace_bytes(1) // 8,), float("nan"), dtype=torch.float64, device="cuda")
    a = plan.estimate(f, ws0).cpu().numpy()
    b = plan.estimate(f, wsn).cpu().numpy()
    assert np.array_equal(a, b, equal_nan=True)
    assert plan.workspace_status(wsn, 1) == 0


def test_static_scratch_refuses_large_plans():
    lib = _lib()
    ng, L = 128, 500.0
    plan = api.Plan(ng, L, synth.default_k1_edges(ng, L, 12), 10, 10, 6, precision="mixed")
    assert plan.workspace_bytes(1) > lib.estimator_static_scratch_bytes()
    field = torch.zeros((1, ng, ng, ng), dtype=torch.float32, device="cuda")
    out = torch.empty(plan.out_shape(1), dtype=torch.float64, device="cuda")
    st = lib.estimator_estimate_static(plan._h, C.c_void_p(field.data_ptr()), 1, C.c_void_p(out.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1
    assert "static scratch" in lib.estimator_last_error().decode()
