"""Pins of the oracle's reference-triangle numerics against facts fixed by the
mathematics: orthonormality, closed-form low-order members, finite differences,
monomial integrals, interpolation identities."""
import math

import numpy as np
import pytest

from oracle import koornwinder as kw
from oracle import rules
from paper_2006_02545_gb300 import workloads


def monomial_integral(a, b):
    """int_T0 u^a v^b du dv = a! b! / (a+b+2)!"""
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


@pytest.mark.parametrize("d", range(0, 11))
def test_koornwinder_orthonormal(d):
    # a rule exact to degree 2d+1 makes the Gram matrix exact
    u, v, w = rules.conical_rule(d + 1)
    K = kw.basis(d, u, v)
    G = (K * w[None, :]) @ K.T
    assert np.abs(G - np.eye(kw.n_basis(d))).max() < 1e-12


def test_koornwinder_closed_forms(rng):
    u = rng.uniform(0, 0.5, 50)
    v = rng.uniform(0, 0.5, 50)
    K = kw.basis(2, u, v)
    assert np.allclose(K[kw.index(0, 0)], math.sqrt(2.0), rtol=0, atol=1e-14)
    # K_10 = 2 (1 - 3v); K_11 = 2 sqrt(3) (2u + v - 1) (worked by hand from the definition)
    assert np.allclose(K[kw.index(1, 0)], 2.0 * (1.0 - 3.0 * v), atol=1e-13)
    assert np.allclose(K[kw.index(1, 1)], 2.0 * math.sqrt(3.0) * (2 * u + v - 1), atol=1e-13)


def test_koornwinder_total_degree():
    # K_nm has total degree n: it is orthogonal to every monomial of degree < n
    d = 6
    u, v, w = rules.conical_rule(d + 2)
    K = kw.basis(d, u, v)
    for n in range(d + 1):
        for m in range(n + 1):
            for a in range(n):
                for b in range(n - a):
                    assert abs((K[kw.index(n, m)] * w * u ** a * v ** b).sum()) < 1e-13


@pytest.mark.parametrize("d", [1, 4, 8, 10])
def test_koornwinder_derivatives_fd(d, rng):
    u = rng.uniform(0.05, 0.45, 20)
    v = rng.uniform(0.05, 0.45, 20)
    K, Ku, Kv = kw.basis(d, u, v, derivs=True)
    h = 1e-6
    fu = (kw.basis(d, u + h, v) - kw.basis(d, u - h, v)) / (2 * h)
    fv = (kw.basis(d, u, v + h) - kw.basis(d, u, v - h)) / (2 * h)
    scale = np.abs(K).max()
    assert np.abs(Ku - fu).max() < 1e-6 * scale
    assert np.abs(Kv - fv).max() < 1e-6 * scale


def test_koornwinder_vertex_values_finite():
    K, Ku, Kv = kw.basis(8, np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]), derivs=True)
    assert np.isfinite(K).all() and np.isfinite(Ku).all() and np.isfinite(Kv).all()


@pytest.mark.parametrize("m", [1, 2, 3, 5, 8, 12, 20])
def test_conical_rule_exactness(m):
    u, v, w = rules.conical_rule(m)
    assert len(w) == m * m and (w > 0).all()
    assert (u > 0).all() and (v > 0).all() and (u + v < 1).all()
    for a in range(2 * m):
        for b in range(2 * m - a):
            got = (w * u ** a * v ** b).sum()
            assert abs(got - monomial_integral(a, b)) < 1e-14 + 1e-12 * monomial_integral(a, b)
    # not exact one degree higher (the claimed order is sharp)
    errs = [abs((w * u ** a * v ** (2 * m - a)).sum() / monomial_integral(a, 2 * m - a) - 1.0)
            for a in range(2 * m + 1)]
    assert max(errs) > 1e-13


@pytest.mark.parametrize("d", range(1, 11))
def test_interp_nodes(d):
    u, v = rules.interp_nodes(d)
    n = kw.n_basis(d)
    assert len(u) == n
    assert (u > 0).all() and (v > 0).all() and (1 - u - v > 0).all()
    # invariant under the symmetries of T0 (permutations of barycentric coordinates)
    bary = np.stack([u, v, 1 - u - v], axis=1)
    key = lambda B: np.round(B, 12)[np.lexsort(np.round(B, 12).T[::-1])]  # noqa: E731
    for perm in ([1, 0, 2], [2, 1, 0], [0, 2, 1], [1, 2, 0]):
        assert np.allclose(key(bary), key(bary[:, perm]), atol=1e-12)
    # same points as the input module's independent construction
    wu, wv = workloads.ref_nodes(d)
    assert np.abs(wu - u).max() < 1e-14 and np.abs(wv - v).max() < 1e-14


@pytest.mark.parametrize("d", range(1, 11))
def test_vals_to_coefs(d, rng):
    V = rules.vals_to_coefs(d)
    u, v = rules.interp_nodes(d)
    U = kw.basis(d, u, v).T
    assert np.abs(U @ V - np.eye(len(u))).max() < 1e-12
    # interpolation reproduces a random polynomial of total degree <= d at other points
    c = rng.standard_normal((d + 1, d + 1))
    poly = lambda x, y: sum(c[a, b] * x ** a * y ** b for a in range(d + 1)  # noqa: E731
                            for b in range(d + 1 - a))
    coef = V @ poly(u, v)
    xu, xv = rng.uniform(0, 0.5, 30), rng.uniform(0, 0.5, 30)
    assert np.abs(kw.basis(d, xu, xv).T @ coef - poly(xu, xv)).max() < 1e-10 * np.abs(c).sum()
    w = rules.interp_weights(d)
    assert (w > 0).all()
    for a in range(d + 1):
        for b in range(d + 1 - a):
            assert abs((w * u ** a * v ** b).sum() - monomial_integral(a, b)) < 1e-14


@pytest.mark.parametrize("d,i", [(2, 0), (4, 3), (6, 0), (6, 17), (8, 44)])
def test_self_rule_smooth_exactness(d, i):
    # the Duffy/sinh rule integrates smooth polynomials exactly-in-the-limit
    u, v, w = rules.self_rule(d, i, 16, 16)
    assert (w > 0).all() and (u >= 0).all() and (v >= 0).all() and (u + v <= 1 + 1e-15).all()
    assert abs(w.sum() - 0.5) < 1e-14
    for a in range(7):
        for b in range(7 - a):
            assert abs((w * u ** a * v ** b).sum() - monomial_integral(a, b)) < 1e-11


def test_subdivide_children_cover_parent():
    kids = rules.subdivide(rules.T0)
    areas = [abs((b - a)[0] * (c - a)[1] - (b - a)[1] * (c - a)[0]) / 2 for a, b, c in kids]
    assert np.allclose(areas, 0.125)
    # child vertex order as stated: (a, ab, ca), (ab, b, bc), (ca, bc, c), (bc, ca, ab)
    a, b, c = rules.T0
    assert np.allclose(kids[1][1], b) and np.allclose(kids[2][2], c) and np.allclose(kids[0][0], a)
    assert np.allclose(kids[3][0], (b + c) / 2)
    # a mapped rule integrates over the child exactly
    u, v, w = rules.map_rule(kids[3], *rules.conical_rule(4))
    assert abs(w.sum() - 0.125) < 1e-15
