"""Seeded synthetic input fields (the validation field of Sec. III).

This module is shared, unchanged, by the CUDA estimator's tests and benchmark
and by the CPU oracle's tests.  It holds no arithmetic of the estimator
itself: it only draws the input cube.

Recipe, per seed (all in float64):

1. white noise w(x) ~ N(0, 1): SplitMix64 of the counter (seed, 2i) and
   (seed, 2i+1), turned into two uniforms of 53 bits, then Box-Muller
   (cosine branch);
2. Gaussian field delta_G with power spectrum P(k) = A k^index (index = -2):
   its transform is W(k) sqrt(P(k) N^3 / V), W = DFT(w), with the zero mode
   removed, and A = sigma_G^2 V / sum_{k != 0} k^index so that the ensemble
   variance on the grid is sigma_G^2 (Sec. III.B uses P = k^-2);
3. local quadratic non-Gaussianity delta = delta_G + f_NG (delta_G^2 -
   <delta_G^2>) (Eq. nG), <.> the mean over the cube;
4. linear Kaiser redshift-space distortion Delta^s = (1 + beta mu_k^2) Delta
   (Eq. RSD) with the line of sight along z (the last, contiguous axis);
5. delta^s = inverse DFT (real).

Defaults follow the estimator's validation workloads: sigma_G = 0.1,
f_NG = 0.5, beta = 0.5.  The paper's own run used beta = 1 (Sec. III.B).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to counter values (uint64 array)."""
    with np.errstate(over="ignore"):
        z = state + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def white_noise(n: int, seed: int, chunk: int = 1 << 22) -> np.ndarray:
    """n standard normal deviates of the stream ``seed`` (float64)."""
    out = np.empty(n, dtype=np.float64)
    base = np.uint64(seed) * np.uint64(0x100000000)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        i = np.arange(s, e, dtype=np.uint64)
        with np.errstate(over="ignore"):
            a = splitmix64(base + np.uint64(2) * i)
            b = splitmix64(base + np.uint64(2) * i + np.uint64(1))
        u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)
        u2 = (b >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        out[s:e] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return out


def _kgrid(ng: int, box_len: float):
    kf = 2.0 * np.pi / box_len
    k = np.fft.fftfreq(ng, d=1.0 / ng) * kf
    kz = np.fft.rfftfreq(ng, d=1.0 / ng) * kf
    return k[:, None, None], k[None, :, None], kz[None, None, :]


def power_amplitude(ng: int, box_len: float, sigma_g: float, index: float = -2.0) -> float:
    """A such that sum_{k != 0} A k^index / V = sigma_g^2 over the full grid."""
    kf = 2.0 * np.pi / box_len
    k = np.fft.fftfreq(ng, d=1.0 / ng) * kf
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    kk = kk.ravel()[1:]
    return float(sigma_g ** 2 * box_len ** 3 / np.sum(kk ** index))


def make_field(ng: int, box_len: float, seed: int, sigma_g: float = 0.1, f_ng: float = 0.5,
               beta: float = 0.5, index: float = -2.0, gaussian_only: bool = False) -> np.ndarray:
    """Redshift-space field delta^s[x][y][z] (float64, z = line of sight)."""
    V = box_len ** 3
    w = white_noise(ng ** 3, seed).reshape(ng, ng, ng)
    W = np.fft.rfftn(w)
    kx, ky, kz = _kgrid(ng, box_len)
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    A = power_amplitude(ng, box_len, sigma_g, index)
    with np.errstate(divide="ignore"):
        amp = np.sqrt(A * np.where(k > 0, k, 1.0) ** index * ng ** 3 / V)
    amp[0, 0, 0] = 0.0
    dG = np.fft.irfftn(W * amp, s=(ng, ng, ng), axes=(0, 1, 2))
    if gaussian_only:
        d = dG
    else:
        d = dG + f_ng * (dG * dG - np.mean(dG * dG))
    D = np.fft.rfftn(d)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu2 = np.where(k > 0, (kz / np.where(k > 0, k, 1.0)) ** 2, 0.0)
    D *= 1.0 + beta * mu2
    return np.fft.irfftn(D, s=(ng, ng, ng), axes=(0, 1, 2))


def default_k1_edges(ng: int, box_len: float, n_k1: int) -> np.ndarray:
    """Linear k1 edges from (N_g/12) k_f to (N_g/3) k_f."""
    kf = 2.0 * np.pi / box_len
    e = np.linspace(ng / 12.0, ng / 3.0, n_k1 + 1) * kf
    e[-1] = (ng / 3.0) * kf
    return e


def log_k1_edges(ng: int, box_len: float, n_k1: int, lo: float | None = None) -> np.ndarray:
    """k1 edges of equal logarithmic width (the paper's k1 binning) from `lo`
    (default (N_g/12) k_f) to (N_g/3) k_f."""
    kf = 2.0 * np.pi / box_len
    hi = (ng / 3.0) * kf
    e = np.geomspace(lo if lo is not None else (ng / 12.0) * kf, hi, n_k1 + 1)
    e[-1] = hi
    return e


# ---------------------------------------------------------------------------
# The same recipe with torch (for large grids on a GPU): the noise stream is
# bit-identical to white_noise(); the transforms run in float64 with torch.fft.
def _splitmix64_torch(x):
    import torch

    def srl(v, k):   # logical right shift of int64 bit patterns
        return torch.bitwise_and(torch.bitwise_right_shift(v, k), (1 << (64 - k)) - 1)

    g = 0x9E3779B97F4A7C15 - (1 << 64)
    m1 = 0xBF58476D1CE4E5B9 - (1 << 64)
    m2 = 0x94D049BB133111EB - (1 << 64)
    z = x + g
    z = torch.bitwise_xor(z, srl(z, 30)) * m1
    z = torch.bitwise_xor(z, srl(z, 27)) * m2
    return torch.bitwise_xor(z, srl(z, 31))


def white_noise_torch(n: int, seed: int, device="cpu", chunk: int = 1 << 24):
    import torch
    out = torch.empty(n, dtype=torch.float64, device=device)
    base = seed * 0x100000000
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        i = torch.arange(s, e, dtype=torch.int64, device=device)
        a = _splitmix64_torch(base + 2 * i)
        b = _splitmix64_torch(base + 2 * i + 1)
        ua = torch.bitwise_and(torch.bitwise_right_shift(a, 11), (1 << 53) - 1).to(torch.float64)
        ub = torch.bitwise_and(torch.bitwise_right_shift(b, 11), (1 << 53) - 1).to(torch.float64)
        u1 = (ua + 1.0) * (1.0 / 9007199254740992.0)
        u2 = ub * (1.0 / 9007199254740992.0)
        out[s:e] = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
    return out


def make_field_torch(ng: int, box_len: float, seed: int, device="cpu", sigma_g: float = 0.1,
                     f_ng: float = 0.5, beta: float = 0.5, index: float = -2.0):
    """make_field() computed with torch on `device`; float64 [ng][ng][ng]."""
    import torch
    V = box_len ** 3
    w = white_noise_torch(ng ** 3, seed, device).reshape(ng, ng, ng)
    W = torch.fft.rfftn(w)
    del w
    kf = 2.0 * math.pi / box_len
    k1 = torch.fft.fftfreq(ng, d=1.0 / ng, dtype=torch.float64, device=device) * kf
    kz = torch.fft.rfftfreq(ng, d=1.0 / ng, dtype=torch.float64, device=device) * kf
    k = torch.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2)
    kfull = torch.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k1[None, None, :] ** 2)
    kfull = kfull.reshape(-1)[1:]
    A = float(sigma_g ** 2 * V / torch.sum(kfull ** index))
    del kfull
    kk = torch.where(k > 0, k, torch.ones_like(k))
    amp = torch.sqrt(A * kk ** index * ng ** 3 / V)
    amp[0, 0, 0] = 0.0
    dG = torch.fft.irfftn(W * amp, s=(ng, ng, ng), dim=(0, 1, 2))
    del W, amp
    d = dG + f_ng * (dG * dG - torch.mean(dG * dG))
    del dG
    D = torch.fft.rfftn(d)
    del d
    mu2 = torch.where(k > 0, (kz[None, None, :] / kk) ** 2, torch.zeros_like(k))
    D *= 1.0 + beta * mu2
    return torch.fft.irfftn(D, s=(ng, ng, ng), dim=(0, 1, 2))
