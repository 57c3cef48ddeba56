"""Pins of the FP64 oracle against things other than itself.

Each test checks one part of the oracle against a textbook definition,
a library routine, a closed form, a brute-force count or an exact invariant,
chosen so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.  Paper references are to
Gill & Bharadwaj, arXiv:2405.14513.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2405_14513_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Transforms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 8, 12, 16, 24, 32])
def test_dft_matches_defining_sum_and_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    j = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(j, j) / n)          # textbook DFT matrix
    got = O.dft(x)
    assert np.allclose(got, F @ x, rtol=0, atol=1e-12 * np.abs(x).sum())
    assert np.allclose(got, np.fft.fft(x), rtol=0, atol=1e-12 * np.abs(x).sum())


def test_forward_cube_normalisation_and_zero_mode():
    ng, L = 8, 300.0
    d = np.random.default_rng(1).normal(size=(ng, ng, ng))
    got = O.forward(d, L)
    want = np.fft.fftn(d) * (L ** 3 / ng ** 3)            # continuous-FT convention V/N^3
    want[0, 0, 0] = 0.0
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_dfield_is_the_ring_sum_of_eq_iFT():
    """D(r,n,x) = sum_{u in r} Delta(u,n) exp(-i u.x), evaluated term by term."""
    ng, L = 16, 500.0
    d = synth.make_field(ng, L, 3)
    cube = np.fft.fftn(d) * (L ** 3 / ng ** 3)
    cube[0, 0, 0] = 0
    edges, kp, cnt = O.rings(ng)
    x = np.arange(ng)
    for r, n in [(0, 1), (2, 0), (3, -2), (5, 4)]:
        got = O.dfield(d, L, r, n)
        want = np.zeros((ng, ng), complex)
        for i in range(-ng // 2, ng // 2):
            for j in range(-ng // 2, ng // 2):
                rad = math.hypot(i, j)
                if not (edges[r] <= rad < edges[r + 1]):
                    continue
                ph = np.exp(-2j * np.pi * (i * x[:, None] + j * x[None, :]) / ng)
                want += cube[i % ng, j % ng, n % ng] * ph
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_dfield_on_reduced_grids():
    """D(r,n,x) at x = (N_g/M) y on M x M grids, M = 2^q or 3 x 2^q, against
    the term-by-term ring sum; M = N_g reproduces the FFT-based field, and the
    triple sum of Eq. fftbs on a grid with M > maxc1 + maxc2 + maxc3 times
    (N_g/M)^2 equals the full-grid sum (no wrapped triangle u1+u2+u3 = M e)."""
    ng, L = 16, 500.0
    d = synth.make_field(ng, L, 5)
    cube = np.fft.fftn(d) * (L ** 3 / ng ** 3)
    cube[0, 0, 0] = 0
    edges, kp, cnt = O.rings(ng)
    for M in (8, 12, 16):
        y = np.arange(M)
        for r, n in [(0, 1), (1, 0), (2, -2)]:
            got = O.dfield_at(d, L, r, n, M)
            want = np.zeros((M, M), complex)
            for i in range(-ng // 2, ng // 2):
                for j in range(-ng // 2, ng // 2):
                    if not (edges[r] <= math.hypot(i, j) < edges[r + 1]):
                        continue
                    want += cube[i % ng, j % ng, n % ng] * np.exp(-2j * np.pi * (i * y[:, None] + j * y[None, :]) / M)
            assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max()), (M, r, n)
    assert np.abs(O.dfield_at(d, L, 2, 1, ng) - O.dfield(d, L, 2, 1)).max() <= 1e-12 * np.abs(O.dfield(d, L, 2, 1)).max()
    # rings 1, 2, 2 reach |u_x|, |u_y| <= 1, 2, 2, so M = 8 and 12 hold the sum exactly
    trip = [(1, 1), (2, 1), (2, -2)]
    full = np.sum(np.prod([O.dfield(d, L, r, n) for r, n in trip], axis=0))
    for M in (8, 12):
        red = np.sum(np.prod([O.dfield_at(d, L, r, n, M) for r, n in trip], axis=0)) * (ng / M) ** 2
        assert abs(red - full) <= 1e-10 * abs(full), M
    # too small a grid wraps triangles in: the identity must fail at M = 4
    red4 = np.sum(np.prod([O.dfield_at(d, L, r, n, 4) for r, n in trip], axis=0)) * (ng / 4) ** 2
    assert abs(red4 - full) > 1e-6 * abs(full)


def test_dfield_on_5x2q_and_7x2q_grids():
    """The same on grids of 5 x 2^q and 7 x 2^q points (M = 20 and 28 at
    N_g = 32, which neither divides): D at x = (N_g/M) y against the
    term-by-term ring sum, and the reduced triple sum of rings 3, 5, 6
    (|u_x| <= 3, 5, 6: the bound is 14) exact on M = 16, 20 and 28, wrong on
    M = 12."""
    ng, L = 32, 500.0
    d = synth.make_field(ng, L, 5)
    cube = np.fft.fftn(d) * (L ** 3 / ng ** 3)
    cube[0, 0, 0] = 0
    edges, kp, cnt = O.rings(ng)
    for M in (20, 28):
        y = np.arange(M)
        for r, n in [(3, 1), (5, -2)]:
            got = O.dfield_at(d, L, r, n, M)
            want = np.zeros((M, M), complex)
            for i in range(-ng // 2, ng // 2):
                for j in range(-ng // 2, ng // 2):
                    if not (edges[r] <= math.hypot(i, j) < edges[r + 1]):
                        continue
                    want += cube[i % ng, j % ng, n % ng] * np.exp(-2j * np.pi * (i * y[:, None] + j * y[None, :]) / M)
            assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), (M, r, n)
    trip = [(3, 1), (5, 1), (6, -2)]
    full = np.sum(np.prod([O.dfield(d, L, r, n) for r, n in trip], axis=0))
    for M in (16, 20, 28):
        red = np.sum(np.prod([O.dfield_at(d, L, r, n, M) for r, n in trip], axis=0)) * (ng / M) ** 2
        assert abs(red - full) <= 1e-12 * abs(full), M
    red12 = np.sum(np.prod([O.dfield_at(d, L, r, n, 12) for r, n in trip], axis=0)) * (ng / 12) ** 2
    assert abs(red12 - full) > 1e-6 * abs(full)


# --------------------------------------------------------------------------
# Rings (Sec. II)
# --------------------------------------------------------------------------
def _golden_edges():
    out = {}
    for line in open(os.path.join(GOLD, "ring_edges.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        ng, nr = int(line[0]), int(line[1])
        out[ng] = (nr, [float(Fraction(t)) for t in line[2:]])
    return out


@pytest.mark.parametrize("ng", [16, 24, 64, 384, 512])
def test_ring_edges_match_paper_rule(ng):
    nr, edges = _golden_edges()[ng]
    got_edges, kp, cnt = O.rings(ng)
    assert len(kp) == nr
    assert np.allclose(got_edges, edges, rtol=0, atol=1e-12)


@pytest.mark.parametrize("ng", [16, 24, 64])
def test_ring_membership_and_mean_radius_by_counting(ng):
    edges, kp, cnt = O.rings(ng)
    h = ng // 2
    i = np.arange(-h, h)
    rad = np.hypot(i[:, None], i[None, :]).ravel()
    for r in range(len(kp)):
        sel = rad[(rad >= edges[r] - 1e-12) & (rad < edges[r + 1] - 1e-12)]
        assert len(sel) == cnt[r]
        assert abs(sel.mean() - kp[r]) < 1e-12
    assert cnt.sum() == (rad < ng / 3.0).sum()


# --------------------------------------------------------------------------
# Triangle counts (Eqs. Ntri1, Ntri2)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ng", [16, 24])
def test_ntri_fft_equals_direct_count(ng):
    t_fft, worst = O.ntri(ng)
    t_dir, _ = O.ntri(ng, direct=True)
    assert worst < 1e-6
    assert np.array_equal(t_fft, t_dir)


def test_ntri_closed_forms_and_symmetry():
    ng = 24
    t, _ = O.ntri(ng)
    _, _, cnt = O.rings(ng)
    nr = len(cnt)
    # ring 0 is the single mode u = 0, so a triangle (0, v, -v) needs v and -v
    # in the other two rings: N_tri(0, r, r') = count(r) delta_{r r'}
    for r in range(nr):
        for q in range(nr):
            assert t[0, r, q] == (cnt[r] if r == q else 0)
    # the count does not depend on which side is called 1, 2 or 3
    for p in [(0, 1, 2), (1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0), (2, 0, 1)]:
        assert np.array_equal(t, np.transpose(t, p))


def test_ntri_brute_force_in_python():
    ng = 16
    t, _ = O.ntri(ng)
    edges, kp, cnt = O.rings(ng)
    h = ng // 2
    modes = {}
    for i in range(-h, h):
        for j in range(-h, h):
            rad = math.hypot(i, j)
            for r in range(len(kp)):
                if edges[r] <= rad < edges[r + 1]:
                    modes[(i, j)] = r
    want = np.zeros_like(t)
    for u, ru in modes.items():
        for v, rv in modes.items():
            w = (-u[0] - v[0], -u[1] - v[1])
            if w in modes:
                want[ru, rv, modes[w]] += 1
    assert np.array_equal(t, want)


# --------------------------------------------------------------------------
# Spherical harmonics and quadrature
# --------------------------------------------------------------------------
def _closed_forms(th, ph):
    s, c = math.sin(th), math.cos(th)
    e = lambda m: complex(math.cos(m * ph), math.sin(m * ph))
    return {
        (0, 0): 0.5 / math.sqrt(math.pi),
        (1, 0): math.sqrt(3 / (4 * math.pi)) * c,
        (1, 1): -math.sqrt(3 / (8 * math.pi)) * s * e(1),
        (2, 0): math.sqrt(5 / (16 * math.pi)) * (3 * c * c - 1),
        (2, 1): -math.sqrt(15 / (8 * math.pi)) * s * c * e(1),
        (2, 2): math.sqrt(15 / (32 * math.pi)) * s * s * e(2),
        (3, 3): -math.sqrt(35 / (64 * math.pi)) * s ** 3 * e(3),
        (4, 0): 3 / (16 * math.sqrt(math.pi)) * (35 * c ** 4 - 30 * c * c + 3),
        (4, 4): 3 / 16 * math.sqrt(35 / (2 * math.pi)) * s ** 4 * e(4),
        (6, 6): 1 / 64 * math.sqrt(3003 / math.pi) * s ** 6 * e(6),
    }


def test_ylm_closed_forms():
    for th, ph in [(0.3, 0.2), (1.1, -2.0), (2.5, 3.0), (math.pi / 2, 1.0)]:
        for (l, m), want in _closed_forms(th, ph).items():
            got = O.ylm(l, m, math.cos(th), math.cos(ph), math.sin(ph))
            assert abs(got - want) < 1e-13, (l, m)


def test_ylm_matches_scipy():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(0)
    for _ in range(20):
        th, ph = rng.uniform(0, np.pi), rng.uniform(-np.pi, np.pi)
        for l in range(7):
            for m in range(l + 1):
                got = O.ylm(l, m, math.cos(th), math.cos(ph), math.sin(ph))
                assert abs(got - complex(sp.sph_harm_y(l, m, th, ph))) < 1e-13


def test_gauss_legendre_and_ylm_orthonormality():
    x, w = O.gauss_legendre(12)
    xr, wr = np.polynomial.legendre.leggauss(12)
    assert np.allclose(np.sort(x), xr, atol=1e-14) and np.allclose(w[np.argsort(x)], wr, atol=1e-14)
    nphi = 16
    lm = [(l, m) for l in range(7) for m in range(-l, l + 1)]
    G = np.zeros((len(lm), len(lm)), complex)
    for xi, wi in zip(x, w):
        for k in range(nphi):
            ph = 2 * np.pi * k / nphi
            y = []
            for l, m in lm:
                v = O.ylm(l, abs(m), xi, math.cos(ph), math.sin(ph))
                y.append(v if m >= 0 else (-1) ** m * np.conj(v))
            y = np.array(y)
            G += np.outer(np.conj(y), y) * wi * 2 * np.pi / nphi
    assert np.abs(G - np.eye(len(lm))).max() < 1e-12


# --------------------------------------------------------------------------
# Triangle shape and orientation (Eqs. shape, orient)
# --------------------------------------------------------------------------
def test_orientation_inverse_against_explicit_triangles():
    """Eq. orient written from explicit 3D triangles: the line of sight seen
    from the frame (z' along k1, x' in the k1-k2 plane) is p."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        k1 = rng.normal(size=3)
        k2 = rng.normal(size=3)
        k3 = -k1 - k2
        a, b = np.linalg.norm(k1), np.linalg.norm(k2)
        mu = -k1 @ k2 / (a * b)
        t = b / a
        zp = k1 / a
        xp = (k2 / b + mu * zp)
        xp /= np.linalg.norm(xp)
        yp = np.cross(zp, xp)
        los = np.array([0.0, 0.0, 1.0])
        p = np.array([los @ xp, los @ yp, los @ zp])
        mus = [k @ los / np.linalg.norm(k) for k in (k1, k2, k3)]
        pz, px = O.orientation(mus[0], mus[1], mu)
        assert abs(pz - p[2]) < 1e-12 and abs(px - p[0]) < 1e-10
        # Eq. orient's third cosine follows from closure with t = k2/k1
        mu3 = -((1 - t * mu) * p[2] + t * math.sqrt(1 - mu * mu) * p[0]) / math.sqrt(1 - 2 * t * mu + t * t)
        assert abs(mu3 - mus[2]) < 1e-12


# --------------------------------------------------------------------------
# Continuum multipoles (Eqs. bs_lm, mod_bs, rsd_bs)
# --------------------------------------------------------------------------
def _gold_setup():
    out = {}
    for line in open(os.path.join(GOLD, "paper_setup.txt")):
        line = line.split("#")[0].split()
        if line:
            out[line[0]] = float(line[1])
    return out


def test_continuum_special_cases():
    A, idx, f, beta = 2.0, -2.0, 0.5, 0.7
    k1, mu, t = 0.3, 0.7, 0.8
    k2, k3 = t * k1, k1 * math.sqrt(1 - 2 * t * mu + t * t)
    P = lambda k: A * k ** idx
    Br = 2 * f * (P(k1) * P(k2) + P(k2) * P(k3) + P(k3) * P(k1))
    # beta = 0: isotropic, only the monopole survives and equals B^r
    c = O.continuum(A, idx, f, 0.0, k1, mu, t, 8)
    assert abs(c[0] - Br) < 1e-12 * Br
    assert np.abs(c[1:]).max() < 1e-12 * Br
    # one factor (1 + beta p_z^2): p_z^2 = 1/3 + (2/3) P_2 gives
    # B_0^0 = (1 + beta/3) B^r, B_2^0 = (2 beta / 3) B^r, nothing else
    c = O.continuum(A, idx, f, beta, k1, mu, t, 8, factor_mask=1)
    want = np.zeros_like(c)
    want[O.lm_index(0, 0)] = (1 + beta / 3) * Br
    want[O.lm_index(2, 0)] = (2 * beta / 3) * Br
    assert np.abs(c - want).max() < 1e-12 * Br


def _nonzero_moments(axis):
    A, idx, f, beta = 1.0, -2.0, 0.5, 1.0
    out = []
    for k1, mu, t in [(0.5, 0.62, 0.77), (1.0, 0.9, 0.55), (2.1, 0.55, 0.95)]:
        c = O.continuum(A, idx, f, beta, k1, mu, t, 8, n_gl=16, n_phi=40, axis=axis)
        scale = np.abs(c).max()
        assert np.abs(c.imag).max() < 1e-12 * scale
        out.append([(l, m) for l in range(9) for m in range(l + 1) if abs(c[O.lm_index(l, m)]) > 1e-10 * scale])
    return out


def test_continuum_moment_content():
    """Eq. rsd_bs is even in p and of degree six, so only even l <= 6
    survive; the paper counts four with m = 0 and sixteen in all (Sec. IV).
    Sixteen needs the polar axis of Y_l^m in the triangle plane: with the
    axis along k1 (p_z = mu_1, the estimator's reading of Eq. orient) p_x
    enters at most to the fourth power and l = 6, m = 5, 6 vanish."""
    g = _gold_setup()
    for nz in _nonzero_moments(axis=1):
        assert len(nz) == g["nonzero_all"]
        assert sum(1 for (l, m) in nz if m == 0) == g["nonzero_m0"]
        assert all(l % 2 == 0 and l <= 6 for (l, m) in nz)
    for nz in _nonzero_moments(axis=0):
        assert sum(1 for (l, m) in nz if m == 0) == g["nonzero_m0"]
        assert all(l % 2 == 0 and l <= 6 for (l, m) in nz)
        assert sorted(nz) == sorted((l, m) for l in (0, 2, 4, 6) for m in range(min(l, 4) + 1))


def test_paper_units():
    g = _gold_setup()
    assert abs(2 * math.pi / g["box_len"] - g["k_min"]) < 0.0005
    assert abs(g["box_len"] / g["n_g"] - g["spacing"]) < 0.005
    assert len(O.rings(int(g["n_g"]))[1]) == 38


# --------------------------------------------------------------------------
# Discrete model [B]_d (Sec. III.C: Eqs. mod_bs and rsd_bs at each
# combination, binned as the estimator)
# --------------------------------------------------------------------------
def _discrete_model_numpy(ng, L, edges, nmu, nt, l_max, A, index, f_ng, beta):
    """[B]_d rebuilt without the oracle's model code: sides K_i from the ring
    radii and planes, side cosines from Eq. orient's three lines applied to the
    oracle's orientation p (checked against n_i / K_i), Y_l^m from scipy."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    c = O.combos(ng, L, edges, nmu, nt, half_space=False)
    _, kp, _ = O.rings(ng)
    kf = 2 * np.pi / L
    n = c["ints"][:, :3].astype(float)
    K = kf * np.sqrt(kp[c["ints"][:, 3:]] ** 2 + n ** 2)
    K1, t, mu, pz, cphi, deg = c["geo"].T
    deg = deg > 0
    # Eq. orient, all three lines, from p = (sin th cos phi, sin th sin phi, p_z)
    px = np.sqrt(np.maximum(0.0, 1 - pz ** 2)) * cphi
    sm = np.sqrt(np.maximum(0.0, 1 - mu ** 2))
    m1 = pz
    m2 = -mu * pz + sm * px
    m3 = -((1 - t * mu) * pz + t * sm * px) / np.sqrt(1 - 2 * t * mu + t * t)
    # where the mean radii close a triangle (mu not clamped), Eq. orient gives
    # back the cosines n_i / K_i of the combination's own sides
    # back the cosines n_i / K_i of the combination's own sides; where they do
    # not (mu clamped, or p_y clamped to 0 because the mean radii and planes
    # admit no unit p), the model takes n_i / K_i as the oracle's reading says
    direct = n * kf / K
    closed = np.abs(K[:, 2] - K1 * np.sqrt(1 - 2 * t * mu + t * t)) < 1e-9 * K1
    consistent = closed & ~deg & (np.abs(cphi) < 1.0)
    got = np.stack([m1, m2, m3], 1)
    assert np.abs(got - direct)[consistent].max() < 1e-9
    assert consistent.mean() > 0.8
    mui = np.where(consistent[:, None], got, direct)
    P = A * K ** index
    Br = 2 * f_ng * (P[:, 0] * P[:, 1] + P[:, 1] * P[:, 2] + P[:, 2] * P[:, 0])
    Bs = np.prod(1 + beta * mui ** 2, axis=1) * Br
    nbin = len(edges) - 1
    nlm = (l_max + 1) * (l_max + 2) // 2
    num = np.zeros((nbin * nmu * nt, nlm))
    den = np.zeros_like(num)
    th = np.arccos(np.clip(pz, -1, 1))
    ph = np.arccos(np.clip(cphi, -1, 1))
    for l in range(l_max + 1):
        for m in range(l + 1):
            y = sp.sph_harm_y(l, m, th, ph)                 # mean of Y* over p_y = +-: Re Y
            w = np.where(deg, y.real if m == 0 else 0.0, y.real)
            a2 = np.abs(y) ** 2
            j = O.lm_index(l, m)
            np.add.at(num[:, j], c["bin"], w * Bs * c["ntri"])
            np.add.at(den[:, j], c["bin"], a2 * c["ntri"])
    pref = np.array([np.sqrt((2 * l + 1) / (4 * np.pi)) for l in range(l_max + 1) for m in range(l + 1)])
    with np.errstate(invalid="ignore", divide="ignore"):
        B = np.where(den > 0, pref * num / den, np.nan)
    return B.reshape(nbin, nmu, nt, nlm)


def test_discrete_model_matches_an_independent_evaluation():
    ng, L, l_max = 32, 1000.0, 6
    edges = synth.default_k1_edges(ng, L, 4)
    A, index, f_ng, beta = 3.0, -2.0, 0.5, 0.8
    want = _discrete_model_numpy(ng, L, edges, 5, 5, l_max, A, index, f_ng, beta)
    got = O.discrete_model(ng, L, edges, 5, 5, l_max, A, index, f_ng, beta)
    fin = np.isfinite(want)
    assert np.array_equal(fin, np.isfinite(got))
    scale = np.abs(want[fin]).max()
    assert np.abs(got[fin] - want[fin]).max() < 1e-10 * scale


def test_discreteness_weights():
    """w_l^m = [B]_d / [B]_c (Sec. III.C).  With an isotropic model and a
    constant P every triangle has the same bispectrum, so the discrete and
    continuum monopoles are both B^r and w_0^0 = 1 in every bin, whatever the
    sampling; with beta != 0 the weights are the ratio of the two models at
    each bin's mean triangle."""
    ng, L = 32, 1000.0
    edges = synth.default_k1_edges(ng, L, 3)
    A, f_ng = 2.0, 0.5
    r = O.discreteness_weights(ng, L, edges, 5, 5, 2, A, 0.0, f_ng, 0.0)
    fin = np.isfinite(r["d"][..., 0])
    assert fin.sum() > 10
    assert np.abs(r["w"][..., 0][fin] - 1.0).max() < 1e-12
    assert np.abs(r["d"][..., 0][fin] - 6 * f_ng * A * A).max() < 1e-12 * 6 * f_ng * A * A
    r = O.discreteness_weights(ng, L, edges, 5, 5, 2, A, -2.0, f_ng, 1.0)
    i = np.argwhere(fin)[0]
    k1, mu, t = r["k1_mu_t"][tuple(i)]
    c = O.continuum(A, -2.0, f_ng, 1.0, k1, mu, t, 2).real
    assert np.allclose(r["c"][tuple(i)], c, rtol=1e-12)
    assert np.allclose(r["w"][tuple(i)][0], r["d"][tuple(i)][0] / c[0], rtol=1e-12)
