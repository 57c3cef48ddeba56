"""ctypes front end of the FP64 CPU oracle (``bisp_oracle.c``).

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it to check the CUDA estimator.  The
product package never imports this module, and this module imports nothing
from the product package.

Every function here marshals numpy arrays into the C library and back; the
arithmetic lives in ``bisp_oracle.c`` (plain double precision, one definition
per equation of Gill & Bharadwaj, arXiv:2405.14513, Sec. II).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bisp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no floating-point contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Desc(C.Structure):
    _fields_ = [("ng", C.c_int), ("box_len", C.c_double), ("n_k1", C.c_int),
                ("k1_edges", C.POINTER(C.c_double)), ("n_mu", C.c_int), ("n_t", C.c_int),
                ("l_max", C.c_int), ("mode", C.c_int), ("nthreads", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            lp = C.POINTER(C.c_long)
            ip = C.POINTER(C.c_int)
            lib.bo_dft.argtypes = [dp, C.c_int]
            lib.bo_rings.argtypes = [C.c_int, lp, dp, lp]
            lib.bo_rings.restype = C.c_int
            lib.bo_forward.argtypes = [C.c_int, C.c_double, dp, dp]
            lib.bo_dfield.argtypes = [C.c_int, C.c_double, dp, C.c_int, C.c_int, dp]
            lib.bo_dfield_at.argtypes = [C.c_int, C.c_double, dp, C.c_int, C.c_int, C.c_int, dp]
            lib.bo_ntri.argtypes = [C.c_int, C.c_int, C.c_int, lp]
            lib.bo_ntri.restype = C.c_double
            lib.bo_ylm.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, dp]
            lib.bo_estimate.argtypes = [C.POINTER(Desc), dp, dp, dp, dp, dp]
            lib.bo_estimate.restype = C.c_long
            lib.bo_estimate_part.argtypes = [C.POINTER(Desc), dp, C.c_int, C.c_int, dp]
            lib.bo_estimate_part.restype = C.c_long
            lib.bo_estimate_stream.argtypes = [C.POINTER(Desc), dp, C.c_char_p, C.c_int, C.c_int, dp, dp, dp, dp]
            lib.bo_estimate_stream.restype = C.c_long
            lib.bo_combos.argtypes = [C.POINTER(Desc), C.c_int, C.c_long, ip, lp, ip, dp]
            lib.bo_combos.restype = C.c_long
            lib.bo_combo_sums.argtypes = [C.c_int, C.c_double, dp, C.c_long, ip, C.c_int, dp, dp]
            lib.bo_combo_sums.restype = C.c_int
            lib.bo_gauss_legendre.argtypes = [C.c_int, dp, dp]
            lib.bo_continuum.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                         C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                         C.c_int, dp]
            lib.bo_discrete_model.argtypes = [C.POINTER(Desc), C.c_double, C.c_double, C.c_double,
                                              C.c_double, dp]
            lib.bo_discrete_model.restype = C.c_long
            lib.bo_orientation.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp]
            lib.bo_shell_triples.argtypes = [C.POINTER(Desc), dp, C.c_long, ip, dp, dp, dp]
            lib.bo_shell_triples.restype = C.c_long
            lib.bo_shell_estimate.argtypes = [C.POINTER(Desc), dp, dp]
            lib.bo_shell_estimate.restype = C.c_long
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _lp(a):
    return a.ctypes.data_as(C.POINTER(C.c_long))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def n_moments_all(l_max: int) -> int:
    return (l_max + 1) * (l_max + 2) // 2


def lm_index(l: int, m: int) -> int:
    return l * (l + 1) // 2 + m


def even_moments(l_max: int):
    """(l, m) pairs of the estimator output: even l, 0 <= m <= l."""
    return [(l, m) for l in range(0, l_max + 1, 2) for m in range(l + 1)]


# ----------------------------------------------------------------------------
def dft(x: np.ndarray) -> np.ndarray:
    """Forward DFT of one line, X_k = sum_j x_j exp(-2 pi i jk/n)."""
    x = np.ascontiguousarray(x, dtype=np.complex128).copy()
    buf = x.view(np.float64)
    _load().bo_dft(_dp(buf), len(x))
    return x


def rings(ng: int):
    """Ring table: (edges in grid units [nr+1], mean radii [nr], mode counts [nr])."""
    e3 = np.zeros(300, dtype=np.int64)
    kp = np.zeros(300)
    cnt = np.zeros(300, dtype=np.int64)
    nr = _load().bo_rings(ng, _lp(e3), _dp(kp), _lp(cnt))
    if nr < 0:
        raise ValueError("bad grid size")
    return e3[: nr + 1] / 3.0, kp[:nr].copy(), cnt[:nr].copy()


def forward(delta: np.ndarray, box_len: float) -> np.ndarray:
    """Delta(k) = (V/N^3) DFT3(delta), Delta(0) = 0; complex [ng][ng][ng]."""
    d = np.ascontiguousarray(delta, dtype=np.float64)
    ng = d.shape[0]
    out = np.zeros(d.shape + (2,))
    if _load().bo_forward(ng, box_len, _dp(d), _dp(out)):
        raise RuntimeError("bo_forward failed")
    return out[..., 0] + 1j * out[..., 1]


def dfield(delta: np.ndarray, box_len: float, r: int, n: int) -> np.ndarray:
    """D(r, n, x) of Eq. iFT on the full grid, complex [ng][ng]."""
    d = np.ascontiguousarray(delta, dtype=np.float64)
    ng = d.shape[0]
    out = np.zeros((ng, ng, 2))
    if _load().bo_dfield(ng, box_len, _dp(d), r, n, _dp(out)):
        raise RuntimeError("bo_dfield failed")
    return out[..., 0] + 1j * out[..., 1]


def dfield_at(delta: np.ndarray, box_len: float, r: int, n: int, M: int) -> np.ndarray:
    """D(r, n, x) of Eq. iFT at x = (N_g/M) y for integer y on an M x M grid,
    summed directly over the ring's modes; complex [M][M]."""
    d = np.ascontiguousarray(delta, dtype=np.float64)
    ng = d.shape[0]
    out = np.zeros((M, M, 2))
    if _load().bo_dfield_at(ng, box_len, _dp(d), r, n, M, _dp(out)):
        raise RuntimeError("bo_dfield_at failed")
    return out[..., 0] + 1j * out[..., 1]


def ntri(ng: int, direct: bool = False, nthreads: int = 0):
    """Triangle-count table [nr][nr][nr] by Eq. Ntri2 (default) or Eq. Ntri1,
    and the largest distance of an Eq. Ntri2 value from its integer."""
    nr = len(rings(ng)[1])
    t = np.zeros(nr ** 3, dtype=np.int64)
    worst = _load().bo_ntri(ng, 1 if direct else 0, nthreads, _lp(t))
    return t.reshape(nr, nr, nr), worst


def ylm(l: int, m: int, z: float, cphi: float, sphi: float) -> complex:
    out = np.zeros(2)
    _load().bo_ylm(l, m, z, cphi, sphi, _dp(out))
    return complex(out[0], out[1])


def _desc(ng, box_len, k1_edges, n_mu, n_t, l_max, direct=False, nthreads=0):
    e = np.ascontiguousarray(k1_edges, dtype=np.float64)
    d = Desc(ng, box_len, len(e) - 1, _dp(e), n_mu, n_t, l_max, 1 if direct else 0, nthreads)
    return d, e


def estimate(delta, box_len, k1_edges, n_mu, n_t, l_max, direct=False, nthreads=0):
    """Run the oracle estimator.  Returns a dict with B, num_re, num_im, den
    (arrays [n_k1][n_mu][n_t][n_lm_all], all l <= l_max) and the combination
    count."""
    d_arr = np.ascontiguousarray(delta, dtype=np.float64)
    ng = d_arr.shape[0]
    desc, keep = _desc(ng, box_len, k1_edges, n_mu, n_t, l_max, direct, nthreads)
    shape = (len(keep) - 1, n_mu, n_t, n_moments_all(l_max))
    B = np.zeros(shape)
    nr_, ni_, dn_ = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    nc = _load().bo_estimate(C.byref(desc), _dp(d_arr), _dp(B), _dp(nr_), _dp(ni_), _dp(dn_))
    if nc < 0:
        raise ValueError("invalid estimator parameters")
    return {"B": B, "num_re": nr_, "num_im": ni_, "den": dn_, "n_combos": int(nc)}


def estimate_part(delta, box_len, k1_edges, n_mu, n_t, l_max, part, nparts, direct=False, nthreads=0):
    """Share `part` of `nparts` of estimate(...)["B"]: the numerator over the
    combinations whose ordered plane pair (n1, n2) has index
    (n1 + nz)(2 nz + 1) + (n2 + nz) = part (mod nparts), divided by the whole
    denominator.  The shares sum to the whole B."""
    d_arr = np.ascontiguousarray(delta, dtype=np.float64)
    ng = d_arr.shape[0]
    desc, keep = _desc(ng, box_len, k1_edges, n_mu, n_t, l_max, direct, nthreads)
    B = np.zeros((len(keep) - 1, n_mu, n_t, n_moments_all(l_max)))
    if _load().bo_estimate_part(C.byref(desc), _dp(d_arr), int(part), int(nparts), _dp(B)) < 0:
        raise ValueError("invalid estimator parameters")
    return B


def estimate_stream(delta, box_len, k1_edges, n_mu, n_t, l_max, ckpt=None, max_slabs=0, verbose=False,
                    nthreads=0):
    """estimate(...) in slabs of n1 with the D fields of the planes n >= 0 only
    (D(r, -n) = conj D(r, n) for a real field) and, if ``ckpt`` is a path, a
    checkpoint after each slab from which a later call resumes.  With
    ``max_slabs`` > 0 it stops after that many slabs and returns None."""
    d_arr = np.ascontiguousarray(delta, dtype=np.float64)
    ng = d_arr.shape[0]
    desc, keep = _desc(ng, box_len, k1_edges, n_mu, n_t, l_max, False, nthreads)
    shape = (len(keep) - 1, n_mu, n_t, n_moments_all(l_max))
    B = np.zeros(shape)
    nr_, ni_, dn_ = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    path = None if ckpt is None else os.fsencode(ckpt)
    nc = _load().bo_estimate_stream(C.byref(desc), _dp(d_arr), path, int(max_slabs), 1 if verbose else 0,
                                    _dp(B), _dp(nr_), _dp(ni_), _dp(dn_))
    if nc == -2:
        return None
    if nc < 0:
        raise ValueError("invalid estimator parameters, no memory, or a checkpoint of another run")
    return {"B": B, "num_re": nr_, "num_im": ni_, "den": dn_, "n_combos": int(nc)}


def select_even(arr: np.ndarray, l_max: int) -> np.ndarray:
    """Keep the estimator's moments (even l) from an all-l moment axis."""
    idx = [lm_index(l, m) for (l, m) in even_moments(l_max)]
    return arr[..., idx]


def combos(ng, box_len, k1_edges, n_mu, n_t, l_max=0, half_space=True, direct=False, nthreads=0):
    """Accepted combinations: dict of ints [n][6] (n1,n2,n3,r1,r2,r3), ntri [n],
    bin [n], geo [n][6] (K1, t, mu, p_z, cos phi, degenerate)."""
    desc, keep = _desc(ng, box_len, k1_edges, n_mu, n_t, l_max, direct, nthreads)
    lib = _load()
    z = np.zeros(1, dtype=np.int32)
    n = lib.bo_combos(C.byref(desc), 1 if half_space else 0, 0, _ip(z), _lp(np.zeros(1, np.int64)),
                      _ip(z), _dp(np.zeros(6)))
    if n < 0:
        raise ValueError("invalid estimator parameters")
    ints = np.zeros((max(n, 1), 6), dtype=np.int32)
    nt = np.zeros(max(n, 1), dtype=np.int64)
    bins = np.zeros(max(n, 1), dtype=np.int32)
    geo = np.zeros((max(n, 1), 6))
    lib.bo_combos(C.byref(desc), 1 if half_space else 0, n, _ip(ints), _lp(nt), _ip(bins), _dp(geo))
    return {"ints": ints[:n], "ntri": nt[:n], "bin": bins[:n], "geo": geo[:n]}


def combo_sums(delta, box_len, ints, nthreads=0, times=None) -> np.ndarray:
    """S = sum_x D1 D2 D3 (Eq. fftbs numerator) for listed combinations.
    If ``times`` is a list, the wall seconds of the plane transforms, the D
    fields and the triple sums are appended to it."""
    d_arr = np.ascontiguousarray(delta, dtype=np.float64)
    ng = d_arr.shape[0]
    q = np.ascontiguousarray(ints, dtype=np.int32)
    out = np.zeros((len(q), 2))
    t = np.zeros(3)
    if _load().bo_combo_sums(ng, box_len, _dp(d_arr), len(q), _ip(q), nthreads, _dp(out), _dp(t)):
        raise ValueError("bad combination list")
    if times is not None:
        times.extend(t.tolist())
    return out[:, 0] + 1j * out[:, 1]


def gauss_legendre(n: int):
    x, w = np.zeros(n), np.zeros(n)
    _load().bo_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def continuum(A, index, f_ng, beta, k1, mu, t, l_max, n_gl=16, n_phi=32, factor_mask=7, axis=0):
    """[B_l^m]_c of Eq. bs_lm for the model of Eqs. mod_bs/rsd_bs, complex [n_lm_all].
    axis 0: polar axis along k1 (the estimator's reading); 1: in-plane, perpendicular to k1."""
    out = np.zeros((n_moments_all(l_max), 2))
    _load().bo_continuum(A, index, f_ng, beta, factor_mask, axis, k1, mu, t, l_max, n_gl, n_phi, _dp(out))
    return out[:, 0] + 1j * out[:, 1]


def discrete_model(ng, box_len, k1_edges, n_mu, n_t, l_max, A, index, f_ng, beta, nthreads=0):
    """[B_l^m]_d: the model at each combination's mean values, binned as the estimator."""
    desc, keep = _desc(ng, box_len, k1_edges, n_mu, n_t, l_max, False, nthreads)
    B = np.zeros((len(keep) - 1, n_mu, n_t, n_moments_all(l_max)))
    if _load().bo_discrete_model(C.byref(desc), A, index, f_ng, beta, _dp(B)) < 0:
        raise ValueError("invalid estimator parameters")
    return B


def orientation(mu1, mu2, mu):
    pz, px = C.c_double(), C.c_double()
    _load().bo_orientation(mu1, mu2, mu, C.byref(pz), C.byref(px))
    return pz.value, px.value


def shell_triples(delta, ng, box_len, k1_edges, n_mu, n_t, l_max, direct=False, nthreads=0):
    """Spherical-shell m = 0 estimator: accepted shell triples (s1 >= s2 >= s3)
    with their bin, N_tri, num_l and den_l (l = 0, 2, .., l_max).  delta may
    be None (counts and denominators only)."""
    desc, keep = _desc(ng, box_len, k1_edges, n_mu, n_t, l_max, direct, nthreads)
    lib = _load()
    d_arr = None if delta is None else np.ascontiguousarray(delta, dtype=np.float64)
    dptr = _dp(d_arr) if d_arr is not None else C.cast(None, C.POINTER(C.c_double))
    z = np.zeros(1)
    n = lib.bo_shell_triples(C.byref(desc), dptr, 0, _ip(np.zeros(4, np.int32)), _dp(z), _dp(z), _dp(z))
    if n < 0:
        raise ValueError("invalid estimator parameters")
    nl = l_max // 2 + 1
    tri = np.zeros((max(n, 1), 4), dtype=np.int32)
    nt = np.zeros(max(n, 1))
    num = np.zeros((max(n, 1), nl))
    den = np.zeros((max(n, 1), nl))
    lib.bo_shell_triples(C.byref(desc), dptr, n, _ip(tri), _dp(nt), _dp(num), _dp(den))
    return {"tri": tri[:n], "ntri": nt[:n], "num": num[:n], "den": den[:n]}


def shell_estimate(delta, box_len, k1_edges, n_mu, n_t, l_max, direct=False, nthreads=0):
    """B_l^0 [n_k1][n_mu][n_t][l_max/2 + 1] of the spherical-shell estimator."""
    d_arr = np.ascontiguousarray(delta, dtype=np.float64)
    ng = d_arr.shape[0]
    desc, keep = _desc(ng, box_len, k1_edges, n_mu, n_t, l_max, direct, nthreads)
    B = np.zeros((len(keep) - 1, n_mu, n_t, l_max // 2 + 1))
    if _load().bo_shell_estimate(C.byref(desc), _dp(d_arr), _dp(B)) < 0:
        raise ValueError("invalid estimator parameters")
    return B


def discreteness_weights(ng, box_len, k1_edges, n_mu, n_t, l_max, A, index, f_ng, beta, nthreads=0):
    """Discreteness weights w_l^m = [B_l^m]_d / [B_l^m]_c (Sec. III.C): the
    discrete model binned as the estimator, over the continuum integral of
    Eq. bs_lm at each bin's mean triangle (K1, mu, t averaged over the bin's
    combinations with their triangle counts as weights).  Returns a dict of
    arrays [n_k1][n_mu][n_t][n_lm_all]: "d", "c" and "w" (NaN for empty bins
    and where |[B]_c| is below 1e-12 of the bin's monopole), and the mean
    shape "k1_mu_t" [n_k1][n_mu][n_t][3]."""
    d = discrete_model(ng, box_len, k1_edges, n_mu, n_t, l_max, A, index, f_ng, beta, nthreads)
    c = combos(ng, box_len, k1_edges, n_mu, n_t, half_space=False, nthreads=nthreads)
    nb = d.shape[0] * n_mu * n_t
    w = c["ntri"].astype(np.float64)
    wsum = np.bincount(c["bin"], weights=w, minlength=nb)
    shape = np.full((nb, 3), np.nan)
    for j, col in enumerate((0, 2, 1)):           # geo: K1, t, mu -> (k1, mu, t)
        s = np.bincount(c["bin"], weights=w * c["geo"][:, col], minlength=nb)
        with np.errstate(invalid="ignore", divide="ignore"):
            shape[:, j] = np.where(wsum > 0, s / wsum, np.nan)
    cont = np.full((nb, n_moments_all(l_max)), np.nan)
    for b in range(nb):
        if wsum[b] > 0:
            k1, mu, t = shape[b]
            cont[b] = continuum(A, index, f_ng, beta, k1, mu, t, l_max).real
    cont = cont.reshape(d.shape)
    with np.errstate(invalid="ignore", divide="ignore"):
        big = np.abs(cont) > 1e-12 * np.abs(cont[..., :1])
        ratio = np.where(big, d / np.where(big, cont, 1.0), np.nan)
    return {"d": d, "c": cont, "w": ratio, "k1_mu_t": shape.reshape(d.shape[:3] + (3,))}
