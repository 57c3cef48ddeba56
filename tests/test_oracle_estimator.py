"""Pins of the oracle's estimator (Eqs. binbs/fftbs, Ntri1/Ntri2, bs_lm2_1).

The FFT form of the oracle is checked against the direct triangle sums on
small grids for every combination (an exact identity, Sec. II), against a
field whose bispectrum is known in closed form, and against exact symmetries
of the estimator: translation, rotation by 90 degrees and mirrors.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2405_14513_gb300 import synth

L_MAX = 6


def _case(ng, n_k1, nmu, nt, seed=1, L=1000.0):
    d = synth.make_field(ng, L, seed)
    e = synth.default_k1_edges(ng, L, n_k1)
    return d, L, e, nmu, nt


@pytest.mark.parametrize("ng,n_k1", [(16, 2), (24, 3)])
def test_fft_form_equals_direct_triangle_sum(ng, n_k1):
    d, L, e, nmu, nt = _case(ng, n_k1, 5, 5)
    a = O.estimate(d, L, e, nmu, nt, L_MAX)
    b = O.estimate(d, L, e, nmu, nt, L_MAX, direct=True)
    assert a["n_combos"] == b["n_combos"] > 0
    scale = np.abs(b["num_re"]).max()
    for key in ("num_re", "num_im"):
        assert np.abs(a[key] - b[key]).max() < 1e-12 * scale
    assert np.array_equal(a["den"], b["den"])
    fin = np.isfinite(b["B"])
    assert np.array_equal(fin, np.isfinite(a["B"]))
    assert np.abs(a["B"][fin] - b["B"][fin]).max() < 1e-12 * np.abs(b["B"][fin]).max()


def test_per_combination_sums_fft_vs_direct():
    ng, L = 24, 700.0
    d = synth.make_field(ng, L, 5)
    e = synth.default_k1_edges(ng, L, 3)
    c = O.combos(ng, L, e, 5, 5, half_space=False)
    S = O.combo_sums(d, L, c["ints"])
    # direct Eq. binbs in numpy: N_g^2 sum over closed triangles
    cube = O.forward(d, L)
    edges, kp, cnt = O.rings(ng)
    h = ng // 2
    ii = np.arange(-h, h)
    rad = np.hypot(ii[:, None], ii[None, :])
    ring = np.full(rad.shape, -1)
    for r in range(len(kp)):
        ring[(rad >= edges[r]) & (rad < edges[r + 1])] = r
    rng = np.random.default_rng(0)
    pick = rng.choice(len(S), size=min(150, len(S)), replace=False)
    for k in pick:
        n1, n2, n3, r1, r2, r3 = c["ints"][k]
        U = np.argwhere(ring == r1) - h
        Vv = np.argwhere(ring == r2) - h
        W = -(U[:, None, :] + Vv[None, :, :])
        ok = (np.abs(W) < h).all(-1)
        ok &= ring[np.clip(W[..., 0] + h, 0, ng - 1), np.clip(W[..., 1] + h, 0, ng - 1)] == r3
        a = cube[U[:, 0] % ng, U[:, 1] % ng, n1 % ng][:, None]
        b = cube[Vv[:, 0] % ng, Vv[:, 1] % ng, n2 % ng][None, :]
        w = cube[W[..., 0] % ng, W[..., 1] % ng, n3 % ng]
        want = ng * ng * np.sum(np.where(ok, a * b * w, 0))
        assert ok.sum() == c["ntri"][k]
        assert abs(S[k] - want) <= 1e-11 * max(abs(want), 1e-300) + 1e-300


def test_point_field_gives_constant_bispectrum():
    """delta = c (delta_{x,0} - N^-3) has Delta(k) = a = c V/N^3 for every
    k != 0, so every closed triangle carries a^3 and Bhat = a^3/V for every
    combination: B_0^0 = a^3 / V in every populated bin, and every moment
    equals the discrete-model prediction for a constant bispectrum."""
    ng, L, c0 = 24, 500.0, 3.0
    d = np.full((ng, ng, ng), -c0 / ng ** 3)
    d[0, 0, 0] += c0
    e = synth.default_k1_edges(ng, L, 3)
    out = O.estimate(d, L, e, 5, 5, L_MAX)
    a = c0 * L ** 3 / ng ** 3
    B00 = out["B"][..., 0]
    fin = np.isfinite(B00)
    assert fin.sum() > 10
    assert np.abs(B00[fin] / (a ** 3 / L ** 3) - 1).max() < 1e-12
    # constant model: A = 1, index 0 gives B^r = 6 f_NG; f_NG chosen so B^r = a^3/V
    Bd = O.discrete_model(ng, L, e, 5, 5, L_MAX, 1.0, 0.0, (a ** 3 / L ** 3) / 6.0, 0.0)
    ev = O.select_even(out["B"], L_MAX)
    evd = O.select_even(Bd, L_MAX)
    assert np.array_equal(np.isfinite(ev), np.isfinite(evd))
    f = np.isfinite(ev)
    assert np.abs(ev[f] - evd[f]).max() < 1e-10 * np.abs(evd[f]).max()


def _rel_close(x, y, tol):
    f = np.isfinite(y)
    assert np.array_equal(f, np.isfinite(x))
    scale = np.abs(y[f]).max()
    return np.abs(x[f] - y[f]).max() <= tol * scale


@pytest.fixture(scope="module")
def base32():
    ng, L = 32, 800.0
    d = synth.make_field(ng, L, 11)
    e = synth.default_k1_edges(ng, L, 3)
    return d, L, e, O.estimate(d, L, e, 4, 4, L_MAX)


def test_translation_invariance(base32):
    """A shifted field multiplies Delta(k) by exp(-i k.s); the phases cancel
    only on closed triangles (u+v+w = 0, n1+n2+n3 = 0)."""
    d, L, e, ref = base32
    sh = np.roll(d, shift=(3, -5, 7), axis=(0, 1, 2))
    out = O.estimate(sh, L, e, 4, 4, L_MAX)
    assert _rel_close(O.select_even(out["B"], L_MAX), O.select_even(ref["B"], L_MAX), 1e-10)


def test_rotation_and_mirror_invariance(base32):
    """A 90-degree rotation about the line of sight and a mirror x -> -x map
    rings onto themselves (the mirror swaps the two chiralities); a mirror
    z -> -z maps n -> -n and p -> (-p_x, p_y, -p_z), which leaves every even-l
    weight unchanged."""
    d, L, e, ref = base32
    want = O.select_even(ref["B"], L_MAX)
    rot = np.ascontiguousarray(np.rot90(d, k=1, axes=(0, 1)))
    mx = np.ascontiguousarray(d[::-1, :, :])
    mz = np.ascontiguousarray(d[:, :, ::-1])
    for f in (rot, mx, mz):
        out = O.estimate(f, L, e, 4, 4, L_MAX)
        assert _rel_close(O.select_even(out["B"], L_MAX), want, 1e-10)


def test_odd_l_and_imaginary_parts_cancel(base32):
    """Summed over n and -n, Re Y* S is real for even l and imaginary for odd
    l (D(r,-n) = conj D(r,n) for a real field)."""
    d, L, e, ref = base32
    scale = np.abs(ref["num_re"]).max()
    for l in range(L_MAX + 1):
        for m in range(l + 1):
            i = O.lm_index(l, m)
            if l % 2 == 0:
                assert np.abs(ref["num_im"][..., i]).max() < 1e-12 * scale
            else:
                assert np.abs(ref["num_re"][..., i]).max() < 1e-12 * scale


def test_ntri_and_combination_counts_scale():
    """Total triangles grow as N_g^6 at fixed k-range fraction (Sec. II,
    computational complexity paragraph): doubling N_g multiplies the sum of
    N_tri over accepted combinations by about 2^6."""
    tot = []
    for ng in (16, 32):
        L = float(ng)
        e = synth.default_k1_edges(ng, L, 1)
        c = O.combos(ng, L, e, 2, 2, half_space=False)
        tot.append(c["ntri"].sum())
    ratio = tot[1] / tot[0]
    assert 40 < ratio < 100


def test_combination_geometry_against_explicit_triangles():
    """For combinations whose mean radii close a perpendicular triangle, build
    the 3D sides (k_perp, n) explicitly and read p off the frame of Eq. orient
    (z' along k1, x' in the k1-k2 plane): the oracle's t, mu, p_z and cos phi
    must be those of the explicit triangle."""
    ng, L = 32, 640.0
    e = synth.default_k1_edges(ng, L, 3)
    c = O.combos(ng, L, e, 4, 4, half_space=False)
    _, kp, _ = O.rings(ng)
    checked = 0
    for (n1, n2, n3, r1, r2, r3), geo in zip(c["ints"], c["geo"]):
        a, b, cc = kp[r1], kp[r2], kp[r3]
        cg = (cc * cc - a * a - b * b) / (2 * a * b) if a > 0 and b > 0 else 2.0
        if abs(cg) >= 0.999:
            continue
        sg = np.sqrt(1 - cg * cg)
        k1 = np.array([a, 0.0, n1])
        k2 = np.array([b * cg, b * sg, n2])
        k3 = -k1 - k2
        assert abs(np.hypot(k3[0], k3[1]) - cc) < 1e-9 and k3[2] == n3
        K = [np.linalg.norm(k) for k in (k1, k2, k3)]
        mu = -k1 @ k2 / (K[0] * K[1])
        if mu > 1 - 1e-9:
            continue
        zp = k1 / K[0]
        xp = k2 / K[1] + mu * zp
        xp /= np.linalg.norm(xp)
        yp = np.cross(zp, xp)
        p = np.array([xp[2], yp[2], zp[2]])
        Kt, t, mu_o, pz, cphi, degen = geo
        assert abs(t - K[1] / K[0]) < 1e-12 and abs(mu_o - mu) < 1e-12
        assert abs(pz - p[2]) < 1e-12
        assert abs(cphi - p[0] / np.hypot(p[0], p[1])) < 1e-8
        checked += 1
    assert checked > 100


@pytest.mark.parametrize("ng,n_k1,nmu", [(16, 3, 4), (32, 5, 5), (48, 6, 5)])
def test_streamed_estimate_equals_plain_estimate(ng, n_k1, nmu):
    """The slab-streamed oracle (planes n >= 0 stored, D(r,-n) = conj D(r,n),
    mirrored combinations from conj S) gives the plain estimate of every
    ordered combination to FP64 rounding."""
    d, L, e, _, _ = _case(ng, n_k1, nmu, nmu, seed=4)
    a = O.estimate(d, L, e, nmu, nmu, L_MAX)
    b = O.estimate_stream(d, L, e, nmu, nmu, L_MAX)
    assert a["n_combos"] == b["n_combos"] > 0
    for key in ("num_re", "num_im", "den"):
        assert np.abs(a[key] - b[key]).max() <= 1e-13 * np.abs(a[key]).max(), key
    fin = np.isfinite(a["B"])
    assert np.array_equal(fin, np.isfinite(b["B"]))
    assert np.abs(a["B"][fin] - b["B"][fin]).max() <= 1e-13 * np.abs(a["B"][fin]).max()


def test_streamed_estimate_resumes_from_checkpoint(tmp_path):
    """Stopped after some slabs and resumed from its checkpoint, the streamed
    oracle ends with the result of one uninterrupted run; a checkpoint of
    another field is refused."""
    d, L, e, nmu, nt = _case(32, 4, 5, 5, seed=6)
    whole = O.estimate_stream(d, L, e, nmu, nt, L_MAX, nthreads=2)
    ck = str(tmp_path / "run.ckpt")
    assert O.estimate_stream(d, L, e, nmu, nt, L_MAX, ckpt=ck, max_slabs=3, nthreads=2) is None
    assert O.estimate_stream(d, L, e, nmu, nt, L_MAX, ckpt=ck, max_slabs=4, nthreads=2) is None
    part = O.estimate_stream(d, L, e, nmu, nt, L_MAX, ckpt=ck, nthreads=2)
    assert part["n_combos"] == whole["n_combos"]
    for key in ("num_re", "num_im", "den"):
        assert np.array_equal(part[key], whole[key]), key
    with pytest.raises(ValueError):
        O.estimate_stream(d * 1.5, L, e, nmu, nt, L_MAX, ckpt=ck, nthreads=2)
