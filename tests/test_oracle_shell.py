"""Pins of the oracle's spherical-shell m = 0 estimator (the comparison
estimator of the shell-based FFT methods the paper cites, Sec. I).

The FFT form equals the direct sum over mode pairs (the Kronecker identity
that Eq. fftbs rests on, in 3D), the triangle counts and denominators equal
an independent numpy enumeration with numpy's Legendre polynomials, a point
field gives B_0^0 = a^3/V in every bin (as for the ring/plane estimator), and
B is invariant under the symmetries of a plane-parallel line of sight."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import oracle as O
from paper_2405_14513_gb300 import synth

L_MAX = 6


def _case(ng, nk, seed=3, L=1000.0):
    return synth.make_field(ng, L, seed), L, synth.default_k1_edges(ng, L, nk)


@pytest.mark.parametrize("ng,nk", [(12, 2), (16, 2), (24, 3)])
def test_fft_form_equals_direct_sums(ng, nk):
    d, L, e = _case(ng, nk)
    a = O.shell_triples(d, ng, L, e, 4, 4, L_MAX)
    b = O.shell_triples(d, ng, L, e, 4, 4, L_MAX, direct=True)
    assert len(a["tri"]) > 0
    assert np.array_equal(a["tri"], b["tri"])
    assert np.array_equal(a["ntri"], b["ntri"])
    assert np.abs(a["den"] - b["den"]).max() <= 1e-10 * np.abs(b["den"]).max()
    assert np.abs(a["num"] - b["num"]).max() <= 1e-10 * np.abs(b["num"]).max()


def _edges3(ng):
    e = [0]
    r = 0
    while e[-1] < ng:
        r += 1
        e.append(min(e[-1] + (3 << ((r - 1) // 10)), ng))
    return np.array(e)


def test_counts_and_denominators_against_numpy_enumeration():
    """N_tri and den_l per shell triple from an enumeration of every mode
    pair in numpy, Y_l0 from numpy's Legendre series."""
    ng, L = 12, 1000.0
    e = synth.default_k1_edges(ng, L, 2)
    got = O.shell_triples(None, ng, L, e, 4, 4, L_MAX)
    e3 = _edges3(ng)
    f = np.fft.fftfreq(ng, 1.0 / ng).astype(int)
    I, J, N = np.meshgrid(f, f, f, indexing="ij")
    k = np.stack([I.ravel(), J.ravel(), N.ravel()], axis=1)
    q9 = 9 * (k ** 2).sum(axis=1)
    shell = np.full(len(k), -1)
    for s in range(len(e3) - 1):
        shell[(q9 >= e3[s] ** 2) & (q9 < e3[s + 1] ** 2)] = s
    keep = shell >= 1
    k, shell = k[keep], shell[keep]
    mu = k[:, 2] / np.sqrt((k ** 2).sum(axis=1))
    y = np.stack([np.sqrt((2 * l + 1) / (4 * np.pi)) * npleg.legval(mu, [0] * l + [1])
                  for l in range(0, L_MAX + 1, 2)], axis=1)
    index = {tuple(v): i for i, v in enumerate(k)}
    cnt, den = {}, {}
    for a in range(len(k)):
        for b in range(len(k)):
            c = index.get(tuple(-k[a] - k[b]))
            if c is None:
                continue
            t = (shell[a], shell[b], shell[c])
            if not (t[0] >= t[1] >= t[2]):
                continue
            cnt[t] = cnt.get(t, 0) + 1
            den[t] = den.get(t, 0) + y[a] ** 2
    for row, nt, dn in zip(got["tri"], got["ntri"], got["den"]):
        t = tuple(int(v) for v in row[:3])
        assert cnt[t] == nt
        np.testing.assert_allclose(dn, den[t], rtol=1e-12)


@pytest.mark.parametrize("direct", [False, True])
def test_point_field_gives_constant_monopole(direct):
    ng, L = 16, 1000.0
    e = synth.default_k1_edges(ng, L, 2)
    c = np.zeros((ng, ng, ng))
    c[3, 5, 7] = 1.0
    c -= 1.0 / ng ** 3
    a = L ** 3 / ng ** 3
    B = O.shell_estimate(c, L, e, 4, 4, L_MAX, direct=direct)
    fin = np.isfinite(B[..., 0])
    assert fin.sum() > 5
    np.testing.assert_allclose(B[..., 0][fin], a ** 3 / L ** 3, rtol=1e-10)


def test_line_of_sight_symmetries():
    """A z mirror maps k_z -> -k_z (even l unchanged); a 90-degree rotation
    about the line of sight and a translation keep every shell and k_z."""
    d, L, e = _case(16, 2, seed=5)
    B = O.shell_estimate(d, L, e, 4, 4, L_MAX)
    fin = np.isfinite(B)
    scale = np.abs(B[fin]).max()
    for t in (d[:, :, ::-1].copy(), np.rot90(d, axes=(0, 1)).copy(), np.roll(d, (3, -2, 5), axis=(0, 1, 2))):
        Bt = O.shell_estimate(t, L, e, 4, 4, L_MAX)
        assert np.array_equal(np.isfinite(Bt), fin)
        assert np.abs(Bt[fin] - B[fin]).max() <= 1e-10 * scale
