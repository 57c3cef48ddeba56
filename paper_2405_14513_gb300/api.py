"""Thin Python binding of the C ABI in ``include/bisp.h`` (argument
marshalling only; every step of the estimator runs in ``libbisp.so``).

Device buffers are torch CUDA tensors (PyTorch supplies memory and
streams); host buffers are numpy arrays.  There is no CPU fallback: if the
CUDA library cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import build as _build

PRECISIONS = {"fp32": 0, "mixed": 1, "fp64": 2, "mixed_tc": 3}
STATUS = {0: "BISP_OK", 1: "BISP_INVALID_ARG", 2: "BISP_UNSUPPORTED_SIZE", 3: "BISP_OUT_OF_MEMORY",
          4: "BISP_CUDA_ERROR", 5: "BISP_TIMEOUT", 6: "BISP_INTERNAL"}

_lock = threading.Lock()
_lib = None


class BispError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")


class Desc(C.Structure):
    _fields_ = [("n_g", C.c_int), ("box_len", C.c_double), ("n_k1", C.c_int),
                ("k1_edges", C.POINTER(C.c_double)), ("n_mu", C.c_int), ("n_t", C.c_int),
                ("l_max", C.c_int), ("precision", C.c_int), ("max_batch", C.c_int),
                ("n_mu_l", C.POINTER(C.c_int)), ("n_t_l", C.POINTER(C.c_int))]


class PlanInfo(C.Structure):
    _fields_ = [("n_g", C.c_int), ("n_rings", C.c_int), ("n_planes", C.c_int), ("l_max", C.c_int),
                ("n_lm", C.c_int), ("n_k1", C.c_int), ("n_mu", C.c_int), ("n_t", C.c_int),
                ("n_levels", C.c_int), ("n_bins", C.c_int64), ("n_combos", C.c_int64),
                ("n_pairs", C.c_int64), ("n_items", C.c_int64), ("triple_products", C.c_double),
                ("dstore_bytes", C.c_size_t), ("workspace_bytes", C.c_size_t),
                ("resident_bytes", C.c_size_t), ("n_views", C.c_int), ("out_doubles", C.c_int64),
                ("pair_products", C.c_double), ("tc_row_points", C.c_double), ("tc_lane_points", C.c_double),
                ("tc_mma_products", C.c_double), ("tc_staged_bytes", C.c_double)]


class ViewInfo(C.Structure):
    _fields_ = [("l_lo", C.c_int), ("l_hi", C.c_int), ("n_mu", C.c_int), ("n_t", C.c_int), ("n_lm", C.c_int),
                ("n_bins", C.c_int64), ("offset", C.c_int64)]


def load():
    """Build (if needed) and load libbisp.so; raises on failure."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(_build.build())
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        lib.estimator_plan.argtypes = [C.POINTER(vp), C.POINTER(Desc), vp]
        lib.estimator_plan.restype = C.c_int
        lib.estimator_plan_info.argtypes = [vp, C.POINTER(PlanInfo)]
        lib.estimator_plan_info.restype = C.c_int
        lib.estimator_view_info.argtypes = [vp, C.c_int, C.POINTER(ViewInfo)]
        lib.estimator_view_info.restype = C.c_int
        lib.estimator_workspace_bytes.argtypes = [vp, C.c_int]
        lib.estimator_workspace_bytes.restype = C.c_size_t
        lib.estimator_estimate.argtypes = [vp, vp, C.c_int, vp, vp, vp]
        lib.estimator_estimate.restype = C.c_int
        lib.estimator_estimate_host.argtypes = [vp, vp, C.c_int, vp, vp]
        lib.estimator_estimate_host.restype = C.c_int
        lib.estimator_host_submit.argtypes = [vp, vp, C.c_int, vp, vp]
        lib.estimator_host_submit.restype = C.c_int
        lib.estimator_host_wait.argtypes = [vp, vp]
        lib.estimator_host_wait.restype = C.c_int
        lib.estimator_estimate_part.argtypes = [vp, vp, C.c_int, vp, vp, C.c_int, C.c_int, vp]
        lib.estimator_estimate_part.restype = C.c_int
        lib.estimator_stats_update.argtypes = [vp, C.c_int, C.c_int64, vp, vp, vp, vp]
        lib.estimator_stats_update.restype = C.c_int
        lib.estimator_shell_plan.argtypes = [C.POINTER(vp), C.POINTER(Desc), vp]
        lib.estimator_shell_plan.restype = C.c_int
        lib.estimator_shell_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_size_t)]
        lib.estimator_shell_info.restype = C.c_int
        lib.estimator_shell_estimate.argtypes = [vp, vp, vp, vp, vp]
        lib.estimator_shell_estimate.restype = C.c_int
        lib.estimator_shell_triples.argtypes = [vp, vp, vp, vp]
        lib.estimator_shell_triples.restype = C.c_int
        lib.estimator_shell_sums.argtypes = [vp, vp, vp, vp]
        lib.estimator_shell_sums.restype = C.c_int
        lib.estimator_shell_destroy.argtypes = [vp]
        lib.estimator_shell_destroy.restype = None
        lib.estimator_destroy.argtypes = [vp]
        lib.estimator_destroy.restype = None
        lib.estimator_status_string.argtypes = [C.c_int]
        lib.estimator_status_string.restype = C.c_char_p
        lib.estimator_last_error.argtypes = []
        lib.estimator_last_error.restype = C.c_char_p
        lib.estimator_denominator.argtypes = [vp, dp]
        lib.estimator_denominator.restype = C.c_int
        lib.estimator_combo_table.argtypes = [vp, C.c_int64, vp, vp, vp, vp]
        lib.estimator_combo_table.restype = C.c_int64
        lib.estimator_combo_geometry.argtypes = [vp, C.c_int64, dp]
        lib.estimator_combo_geometry.restype = C.c_int64
        lib.estimator_combo_sums.argtypes = [vp, vp, dp, vp]
        lib.estimator_combo_sums.restype = C.c_int
        lib.estimator_dfield.argtypes = [vp, vp, C.c_int, C.c_int, C.c_int, dp, vp]
        lib.estimator_dfield.restype = C.c_int
        lib.estimator_delta_plane.argtypes = [vp, vp, C.c_int, dp, vp]
        lib.estimator_delta_plane.restype = C.c_int
        lib.estimator_graph_create.argtypes = [C.POINTER(vp), vp, vp, C.c_int, vp, vp, vp]
        lib.estimator_graph_create.restype = C.c_int
        lib.estimator_graph_launch.argtypes = [vp, vp]
        lib.estimator_graph_launch.restype = C.c_int
        lib.estimator_graph_destroy.argtypes = [vp]
        lib.estimator_graph_destroy.restype = None
        lib.estimator_workspace_status.argtypes = [vp, vp, C.c_int, vp]
        lib.estimator_workspace_status.restype = C.c_int
        lib.estimator_set_wait_limit.argtypes = [vp, C.c_int]
        lib.estimator_set_wait_limit.restype = C.c_int
        lib.estimator_set_timing.argtypes = [vp, C.c_int]
        lib.estimator_set_timing.restype = C.c_int
        lib.estimator_stage_times.argtypes = [vp, dp, vp]
        lib.estimator_stage_times.restype = C.c_int
        lib.estimator_stage_flops.argtypes = [vp, dp]
        lib.estimator_stage_flops.restype = C.c_int
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != 0:
        raise BispError(status, where, load().estimator_last_error().decode())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def even_moments(l_max: int):
    """(l, m) of the moment axis of B: even l, 0 <= m <= l."""
    return [(l, m) for l in range(0, l_max + 1, 2) for m in range(l + 1)]


class Graph:
    """A captured estimate (``estimator_graph_*``); keeps its tensors alive."""

    def __init__(self, handle, keep):
        self._h, self._keep = handle, keep

    def launch(self, stream=None):
        _check(load().estimator_graph_launch(self._h, _stream_handle(stream)), "estimator_graph_launch")

    def close(self):
        if getattr(self, "_h", None):
            load().estimator_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """An estimator plan (``estimator_plan``) and its calls."""

    def __init__(self, n_g: int, box_len: float, k1_edges, n_mu: int, n_t: int, l_max: int,
                 precision: str = "mixed", max_batch: int = 1, stream=None, mu_t_bins_l=None):
        """mu_t_bins_l: optional per-l (mu, t) grids, one entry per even l <= l_max,
        each n (an n x n grid) or (n_mu, n_t); n_mu and n_t are then ignored and
        the output is laid out by view (``views``, ``split``)."""
        lib = load()
        self._edges = np.ascontiguousarray(k1_edges, dtype=np.float64)
        self.n_g, self.box_len, self.n_mu, self.n_t, self.l_max = n_g, box_len, n_mu, n_t, l_max
        self.n_k1 = len(self._edges) - 1
        self.precision = precision
        self.max_batch = max_batch
        self._inflight = []              # host arrays of estimator_host_submit calls not yet waited for
        d = Desc(n_g, box_len, self.n_k1, _dp(self._edges), n_mu, n_t, l_max,
                 PRECISIONS[precision], max_batch)
        if mu_t_bins_l is not None:
            g = [(int(x), int(x)) if np.isscalar(x) else (int(x[0]), int(x[1])) for x in mu_t_bins_l]
            if len(g) != l_max // 2 + 1:
                raise ValueError("mu_t_bins_l needs one entry per even l <= l_max")
            mu_l = (C.c_int * len(g))(*[a for a, _ in g])
            t_l = (C.c_int * len(g))(*[b for _, b in g])
            d.n_mu_l = C.cast(mu_l, C.POINTER(C.c_int))
            d.n_t_l = C.cast(t_l, C.POINTER(C.c_int))
        h = C.c_void_p()
        st = lib.estimator_plan(C.byref(h), C.byref(d), _stream_handle(stream) if stream is not None
                                else C.c_void_p(0))
        _check(st, "estimator_plan")
        self._h = h
        inf = PlanInfo()
        _check(lib.estimator_plan_info(h, C.byref(inf)), "estimator_plan_info")
        self.info = {k: getattr(inf, k) for k, _ in PlanInfo._fields_}
        self.n_lm = inf.n_lm
        self.n_bins = inf.n_bins
        self.n_combos = inf.n_combos
        self.n_mu, self.n_t = inf.n_mu, inf.n_t
        self.out_doubles = inf.out_doubles
        self.views = []
        for v in range(inf.n_views):
            vi = ViewInfo()
            _check(lib.estimator_view_info(h, v, C.byref(vi)), "estimator_view_info")
            self.views.append({k: getattr(vi, k) for k, _ in ViewInfo._fields_})
        self.field_dtype = np.float64 if precision == "fp64" else np.float32

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().estimator_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def out_shape(self, batch: int = 1):
        """[batch][n_k1][n_mu][n_t][n_lm] with one view, else [batch][out_doubles]."""
        if len(self.views) == 1:
            return (batch, self.n_k1, self.n_mu, self.n_t, self.n_lm)
        return (batch, self.out_doubles)

    def split(self, out):
        """The views' blocks of an output (torch tensor or numpy array, first
        axis the batch): a list of [batch][n_k1][n_mu][n_t][n_lm] arrays, one
        per view, moments of orders view["l_lo"] .. view["l_hi"]."""
        flat = out.reshape(out.shape[0], self.out_doubles)
        return [flat[:, v["offset"]:v["offset"] + v["n_bins"] * v["n_lm"]].reshape(
                    out.shape[0], self.n_k1, v["n_mu"], v["n_t"], v["n_lm"]) for v in self.views]

    def workspace_bytes(self, batch: int = 1) -> int:
        return int(load().estimator_workspace_bytes(self._h, batch))

    def workspace(self, batch: int = 1, device="cuda"):
        import torch
        return torch.empty(max(self.workspace_bytes(batch), 256), dtype=torch.uint8, device=device)

    def _check_field(self, delta):
        import torch
        want = torch.float64 if self.precision == "fp64" else torch.float32
        if delta.dtype != want or not delta.is_cuda or not delta.is_contiguous():
            raise ValueError(f"delta must be a contiguous CUDA {want} tensor")
        if delta.dim() != 4 or tuple(delta.shape[1:]) != (self.n_g,) * 3:
            raise ValueError("delta must be [batch][N][N][N] of the plan's grid size")

    def estimate(self, delta, workspace, out=None, stream=None):
        """delta: CUDA tensor [batch][N][N][N] (float32, or float64 for fp64);
        returns (or fills) a CUDA float64 tensor [batch][n_k1][n_mu][n_t][n_lm]."""
        import torch
        if delta.dim() == 3:
            delta = delta.unsqueeze(0)
        batch = delta.shape[0]
        self._check_field(delta)
        if out is None:
            out = torch.empty(self.out_shape(batch), dtype=torch.float64, device=delta.device)
        st = load().estimator_estimate(self._h, C.c_void_p(delta.data_ptr()), batch,
                                       C.c_void_p(workspace.data_ptr()), C.c_void_p(out.data_ptr()),
                                       _stream_handle(stream))
        _check(st, "estimator_estimate")
        return out

    def estimate_part(self, delta, workspace, part: int, nparts: int, out=None, stream=None):
        """Share `part` of `nparts` of estimate(delta) (``estimator_estimate_part``):
        the shares' outputs sum to the whole estimate."""
        import torch
        if delta.dim() == 3:
            delta = delta.unsqueeze(0)
        batch = delta.shape[0]
        self._check_field(delta)
        if out is None:
            out = torch.empty(self.out_shape(batch), dtype=torch.float64, device=delta.device)
        st = load().estimator_estimate_part(self._h, C.c_void_p(delta.data_ptr()), batch,
                                            C.c_void_p(workspace.data_ptr()), C.c_void_p(out.data_ptr()),
                                            int(part), int(nparts), _stream_handle(stream))
        _check(st, "estimator_estimate_part")
        return out

    def graph(self, delta, workspace, out, stream=None) -> "Graph":
        """Capture estimate(delta, workspace, out) into a CUDA graph
        (``estimator_graph_create``); the tensors must outlive the graph."""
        self._check_field(delta)
        h = C.c_void_p()
        st = load().estimator_graph_create(C.byref(h), self._h, C.c_void_p(delta.data_ptr()), delta.shape[0],
                                           C.c_void_p(workspace.data_ptr()), C.c_void_p(out.data_ptr()),
                                           _stream_handle(stream))
        _check(st, "estimator_graph_create")
        return Graph(h, (delta, workspace, out))

    def host_submit(self, delta: np.ndarray, out: np.ndarray, stream=None):
        """Queue the estimate of a host field (see estimator_host_submit):
        delta [batch][N][N][N] (float32, or float64 for fp64; page-locked for
        overlap), out float64 [batch][out_doubles]; both stay referenced until
        the matching host_wait."""
        d = np.asarray(delta)
        if d.ndim == 3:
            d = d[None]
        dt = np.float64 if self.precision == "fp64" else np.float32
        if d.dtype != dt or not d.flags.c_contiguous or d.shape[1:] != (self.n_g,) * 3:
            raise ValueError(f"delta must be a contiguous {np.dtype(dt).name} [batch][N][N][N] array")
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size < d.shape[0] * self.info["out_doubles"]:
            raise ValueError("out must be a contiguous float64 array of batch x out_doubles")
        _check(load().estimator_host_submit(self._h, C.c_void_p(d.ctypes.data), d.shape[0],
                                            C.c_void_p(out.ctypes.data), _stream_handle(stream)),
               "estimator_host_submit")
        self._inflight.append((d, out))

    def host_wait(self, stream=None):
        """Wait for the oldest host submission; returns its output array."""
        st = load().estimator_host_wait(self._h, _stream_handle(stream))
        d, out = self._inflight.pop(0) if self._inflight else (None, None)
        _check(st, "estimator_host_wait")
        return out

    def estimate_host(self, delta: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """Host-memory variant: numpy in, numpy out (copies inside the call)."""
        d = np.ascontiguousarray(delta, dtype=self.field_dtype)
        if d.ndim == 3:
            d = d[None]
        if out is None:
            out = np.empty(self.out_shape(d.shape[0]), dtype=np.float64)
        st = load().estimator_estimate_host(self._h, C.c_void_p(d.ctypes.data), d.shape[0],
                                            C.c_void_p(out.ctypes.data),
                                            _stream_handle(stream) if stream is not None else C.c_void_p(0))
        _check(st, "estimator_estimate_host")
        return out

    # ------------------------------------------------------------------
    def denominator(self) -> np.ndarray:
        """Denominators laid out as one field's output (out_shape(1)[1:])."""
        den = np.zeros(self.out_doubles)
        _check(load().estimator_denominator(self._h, _dp(den)), "estimator_denominator")
        return den.reshape(self.out_shape(1)[1:])

    def combo_table(self):
        n = self.n_combos
        ints = np.zeros((max(n, 1), 6), dtype=np.int32)
        ntri = np.zeros(max(n, 1), dtype=np.int64)
        binv = np.zeros(max(n, 1), dtype=np.int32)
        grid = np.zeros(max(n, 1), dtype=np.int32)
        got = load().estimator_combo_table(self._h, n, C.c_void_p(ints.ctypes.data),
                                           C.c_void_p(ntri.ctypes.data), C.c_void_p(binv.ctypes.data),
                                           C.c_void_p(grid.ctypes.data))
        if got != n:
            raise BispError(6, "estimator_combo_table", "count mismatch")
        return {"ints": ints[:n], "ntri": ntri[:n], "bin": binv[:n], "grid": grid[:n]}

    def combo_geometry(self) -> np.ndarray:
        """[n_combos][4]: mu, t, p_z, cos phi of each combination (combo_table order)."""
        n = self.n_combos
        geo = np.zeros((max(n, 1), 4))
        got = load().estimator_combo_geometry(self._h, n, _dp(geo))
        if got != n:
            raise BispError(6, "estimator_combo_geometry", "count mismatch")
        return geo[:n]

    def workspace_status(self, workspace=None, batch: int = 1, stream=None) -> int:
        """Status code of the last estimate run in `workspace` (None: the
        array of estimator_estimate_static): BISP_TIMEOUT (5) if a
        tensor-core Step-II block gave up a bounded wait for one of its
        `batch` fields, else 0.  Synchronises the stream; clears the status."""
        ws = C.c_void_p(None) if workspace is None else C.c_void_p(workspace.data_ptr())
        return int(load().estimator_workspace_status(self._h, ws, int(batch), _stream_handle(stream)))

    def set_wait_limit(self, spins: int):
        """Polls after which the tensor-core Step II's waits give up (0: default)."""
        _check(load().estimator_set_wait_limit(self._h, int(spins)), "estimator_set_wait_limit")

    def combo_sums(self, workspace, stream=None) -> np.ndarray:
        S = np.zeros(max(self.n_combos, 1))
        _check(load().estimator_combo_sums(self._h, C.c_void_p(workspace.data_ptr()), _dp(S),
                                           _stream_handle(stream)), "estimator_combo_sums")
        return S[: self.n_combos]

    def dfield(self, workspace, M: int, n: int, r: int, stream=None) -> np.ndarray:
        out = np.zeros((M, M, 2))
        _check(load().estimator_dfield(self._h, C.c_void_p(workspace.data_ptr()), M, n, r, _dp(out),
                                       _stream_handle(stream)), "estimator_dfield")
        return out[..., 0] + 1j * out[..., 1]

    def delta_plane(self, workspace, n: int, stream=None) -> np.ndarray:
        out = np.zeros((self.n_g, self.n_g, 2))
        _check(load().estimator_delta_plane(self._h, C.c_void_p(workspace.data_ptr()), n, _dp(out),
                                            _stream_handle(stream)), "estimator_delta_plane")
        return out[..., 0] + 1j * out[..., 1]


    # ------------------------------------------------------------------
    def set_timing(self, on: bool):
        _check(load().estimator_set_timing(self._h, 1 if on else 0), "estimator_set_timing")

    def stage_times(self):
        """(ms, launches) per stage since timing was switched on."""
        ms = np.zeros(len(STAGES))
        n = np.zeros(len(STAGES), dtype=np.int64)
        _check(load().estimator_stage_times(self._h, _dp(ms), C.c_void_p(n.ctypes.data)),
               "estimator_stage_times")
        return dict(zip(STAGES, ms.tolist())), dict(zip(STAGES, n.tolist()))

    def stage_flops(self):
        f = np.zeros(len(STAGES))
        _check(load().estimator_stage_flops(self._h, _dp(f)), "estimator_stage_flops")
        return dict(zip(STAGES, f.tolist()))


class ShellPlan:
    """The spherical-shell estimator of the m = 0 multipoles
    (``estimator_shell_*``): B_l^0 [n_k1][n_mu][n_t][l_max/2 + 1]."""

    def __init__(self, n_g: int, box_len: float, k1_edges, n_mu: int, n_t: int, l_max: int, stream=None):
        lib = load()
        self._edges = np.ascontiguousarray(k1_edges, dtype=np.float64)
        self.n_g, self.box_len, self.n_mu, self.n_t, self.l_max = n_g, box_len, n_mu, n_t, l_max
        self.n_k1 = len(self._edges) - 1
        self.nl = l_max // 2 + 1
        d = Desc(n_g, box_len, self.n_k1, _dp(self._edges), n_mu, n_t, l_max, PRECISIONS["mixed"], 1)
        h = C.c_void_p()
        _check(lib.estimator_shell_plan(C.byref(h), C.byref(d), _stream_handle(stream) if stream is not None
                                        else C.c_void_p(0)), "estimator_shell_plan")
        self._h = h
        ns, nt, wb = C.c_int(), C.c_int64(), C.c_size_t()
        _check(lib.estimator_shell_info(h, C.byref(ns), C.byref(nt), C.byref(wb)), "estimator_shell_info")
        self.n_shells, self.n_triples, self._ws_bytes = ns.value, nt.value, wb.value

    def close(self):
        if getattr(self, "_h", None):
            load().estimator_shell_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def out_shape(self):
        return (self.n_k1, self.n_mu, self.n_t, self.nl)

    def workspace(self, device="cuda"):
        import torch
        return torch.empty(max(self._ws_bytes, 256), dtype=torch.uint8, device=device)

    def estimate(self, delta, workspace, out=None, stream=None):
        """delta: contiguous CUDA float32 [N][N][N]; returns CUDA float64 B_l^0."""
        import torch
        if delta.dtype != torch.float32 or not delta.is_cuda or not delta.is_contiguous() or \
                tuple(delta.shape) != (self.n_g,) * 3:
            raise ValueError("delta must be a contiguous CUDA float32 [N][N][N] of the plan's grid")
        if out is None:
            out = torch.empty(self.out_shape(), dtype=torch.float64, device=delta.device)
        _check(load().estimator_shell_estimate(self._h, C.c_void_p(delta.data_ptr()), C.c_void_p(workspace.data_ptr()),
                                               C.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "estimator_shell_estimate")
        return out

    def triples(self):
        n = self.n_triples
        tri = np.zeros((max(n, 1), 4), dtype=np.int32)
        nt = np.zeros(max(n, 1))
        den = np.zeros((max(n, 1), self.nl))
        _check(load().estimator_shell_triples(self._h, C.c_void_p(tri.ctypes.data), C.c_void_p(nt.ctypes.data),
                                              C.c_void_p(den.ctypes.data)), "estimator_shell_triples")
        return {"tri": tri[:n], "ntri": nt[:n], "den": den[:n]}

    def sums(self, workspace, stream=None):
        num = np.zeros((max(self.n_triples, 1), self.nl))
        _check(load().estimator_shell_sums(self._h, C.c_void_p(workspace.data_ptr()), C.c_void_p(num.ctypes.data),
                                           _stream_handle(stream)), "estimator_shell_sums")
        return num[: self.n_triples]


STAGES = ["forward", "step1", "step2", "reduce", "bin"]


def stats_update(B, count, mean, m2, stream=None):
    """estimator_stats_update: Welford update of (count, mean, m2) [n] with the
    fields of B [batch][n] (CUDA float64 / int64 tensors)."""
    n = mean.numel()
    if B.dtype.itemsize != 8 or not (B.is_cuda and B.is_contiguous()) or B.numel() % max(n, 1):
        raise ValueError("B must be a contiguous CUDA float64 tensor [batch][n]")
    st = load().estimator_stats_update(C.c_void_p(B.data_ptr()), B.numel() // max(n, 1), n,
                                       C.c_void_p(count.data_ptr()), C.c_void_p(mean.data_ptr()),
                                       C.c_void_p(m2.data_ptr()), _stream_handle(stream))
    _check(st, "estimator_stats_update")


def status_string(status: int) -> str:
    return load().estimator_status_string(status).decode()


def try_plan(n_g, box_len, k1_edges, n_mu, n_t, l_max, precision="mixed", max_batch=1, n_mu_l=None, n_t_l=None):
    """Call estimator_plan and return (status, last_error); destroys any plan.
    Used to check argument validation (n_mu_l, n_t_l: raw per-l lists)."""
    lib = load()
    e = np.ascontiguousarray(k1_edges, dtype=np.float64)
    d = Desc(n_g, box_len, len(e) - 1, _dp(e), n_mu, n_t, l_max, PRECISIONS.get(precision, precision),
             max_batch)
    keep = []
    for name, vals in (("n_mu_l", n_mu_l), ("n_t_l", n_t_l)):
        if vals is not None:
            arr = (C.c_int * len(vals))(*vals)
            keep.append(arr)
            setattr(d, name, C.cast(arr, C.POINTER(C.c_int)))
    h = C.c_void_p()
    st = lib.estimator_plan(C.byref(h), C.byref(d), C.c_void_p(0))
    if h.value:
        lib.estimator_destroy(h)
    return st, lib.estimator_last_error().decode()
