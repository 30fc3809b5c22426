"""Pins of the oracle's random numbers, lattices and moment basis (CPU only).

The generator is pinned to the published Philox4x32-10 known answers; the
velocity sets to the lattice isotropy conditions; the Gram-Schmidt basis to
norms derived by hand from the monomial list and to the hydrodynamic moments."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_gaussian_moments():
    # 2^17 normals from stream 0 of consecutive sites: mean 0, variance 1, kurtosis 3 (5 sigma)
    g = np.concatenate([O.gaussians(7, 3, s, 0, 2) for s in range(8192)])
    n = g.size
    assert abs(g.mean()) < 5 / np.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(g ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)
    # the pairs of one Box-Muller draw are uncorrelated
    gg = g.reshape(-1, 2)
    assert abs(np.mean(gg[:, 0] * gg[:, 1])) < 5 / np.sqrt(gg.shape[0])


def test_gaussian_pairs_sit_on_the_uniform_grids():
    # each pair (g0, g1) is r (cos, sin)(2 pi v) of one 32-bit word: its radius
    # uniform u = exp(-r^2/2) lies on the 20-bit grid (k + 1/2) 2^-20 and its
    # angle v on the 12-bit grid (m + 1/2) 2^-12; both grids are filled, and
    # the drawn radius never passes the grid's bound sqrt(-2 ln 2^-21)
    gg = np.concatenate([O.gaussians(3, 11, s, 1, 2) for s in range(16384)]).reshape(-1, 2)
    r2 = (gg ** 2).sum(axis=1)
    ku = np.exp(-r2 / 2) * 2.0 ** 20 - 0.5
    assert np.abs(ku - np.round(ku)).max() < 1e-4
    v = np.mod(np.arctan2(gg[:, 1], gg[:, 0]) / (2 * np.pi), 1.0)
    km = v * 4096 - 0.5
    assert np.abs(km - np.round(km)).max() < 1e-6
    assert len(np.unique(np.round(km))) == 4096
    assert np.sqrt(r2.max()) <= np.sqrt(42 * np.log(2)) + 1e-12
    # the 4096 angles make (cos, sin) moments below order 4096 the continuous ones
    th = 2 * np.pi * (np.arange(4096) + 0.5) / 4096
    assert abs(np.mean(np.cos(th) ** 4) - 3 / 8) < 1e-15 and abs(np.mean(np.cos(th) ** 2 * np.sin(th) ** 2) - 1 / 8) < 1e-15


def test_gaussians_depend_on_every_counter_word():
    base = O.gaussians(1, 5, 10, 0, 1)
    for other in (O.gaussians(2, 5, 10, 0, 1), O.gaussians(1, 6, 10, 0, 1), O.gaussians(1, 5, 11, 0, 1),
                  O.gaussians(1, 5, 10, 1, 1), O.gaussians(1, 5 + (1 << 32), 10, 0, 1),
                  O.gaussians(1, 5, 10, 0, 2)[8:]):
        assert not np.allclose(base, other)
    assert np.array_equal(O.gaussians(1, 5, 10, 0, 2)[:8], base)


@pytest.mark.parametrize("dim,q", [(2, 9), (3, 19), (3, 15)])
def test_lattice_isotropy(dim, q):
    c, w = O.lattice(dim, q)
    cs2 = 1.0 / 3.0
    d = np.eye(3)[:dim, :dim]
    cc = c[:, :dim].astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, cc), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, cc, cc), cs2 * d, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, cc, cc, cc), 0, atol=1e-16)
    iso4 = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, cc, cc, cc, cc), iso4, atol=1e-15)
    # opposite pairs (i, i+1)
    for i in range(1, q, 2):
        assert np.array_equal(c[i], -c[i + 1])


# Norms of the Gram-Schmidt vectors, derived by hand from the monomials:
# e.g. c^2 - 1 on D3Q19 has norm sum w c^4 - 1 = 2/3; c_x (c^2 - 5/3) has 2/27;
# c^4 - 2 c^2 + 1/3 has 2/9; (3c_x^2 - c^2)(c^2 - 3/2) has 1/3.
NORMS = {
    (3, 19): "1 1/3 1/3 1/3 2/3 4/3 4/9 1/9 1/9 1/9 2/27 2/27 2/27 2/9 2/9 2/9 2/9 1/3 1/9",
    (2, 9): "1 1/3 1/3 4/9 4/9 1/9 2/27 2/27 16/81",
    # D3Q15 (w 2/9, 1/9, 1/72): c_x(c^2 - 5/3) has 8/27, c_x c_y c_z 1/9, c^4 - 3c^2 + 4/3 has 8/9
    (3, 15): "1 1/3 1/3 1/3 2/3 4/3 4/9 1/9 1/9 1/9 8/27 8/27 8/27 1/9 8/9",
}


@pytest.mark.parametrize("dim,q", [(2, 9), (3, 19), (3, 15)])
def test_moment_basis(dim, q):
    E, b = O.moment_basis(dim, q)
    c, w = O.lattice(dim, q)
    G = np.einsum("ki,i,li->kl", E, w, E)
    assert np.allclose(G, np.diag(b), atol=1e-15)
    assert np.allclose(b, [float(Fraction(x)) for x in NORMS[(dim, q)].split()], rtol=1e-14)
    # mass and momentum modes are 1 and c
    assert np.allclose(E[0], 1.0)
    for a in range(dim):
        assert np.allclose(E[1 + a], c[:, a])
    # stress modes span exactly the Q_ab = c_a c_b - c_s^2 delta_ab rows
    ns = dim * (dim + 1) // 2
    Q = np.array([c[:, a] * c[:, bb] - (a == bb) / 3.0 for a in range(dim) for bb in range(a, dim)])
    St = E[1 + dim:1 + dim + ns]
    assert np.linalg.matrix_rank(np.vstack([St, Q]), tol=1e-12) == ns
    assert np.linalg.matrix_rank(E, tol=1e-12) == q
    # ghost modes are orthogonal (under w) to every polynomial of degree <= 2
    polys = [np.ones(q)] + [c[:, a] for a in range(dim)] + [c[:, a] * c[:, bb] for a in range(dim) for bb in range(a, dim)]
    for k in range(1 + dim + ns, q):
        for pv in polys:
            assert abs(np.sum(w * E[k] * pv)) < 1e-15
