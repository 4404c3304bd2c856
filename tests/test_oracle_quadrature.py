"""Pins of the oracle's geometry, kernels and local quadratures against closed forms,
finite differences and the independent truth integrators."""
import numpy as np
import pytest

from oracle import geometry, quadrature, rules, truth
from oracle.kernels import kernel_jac
from paper_2006_02545_gb300 import workloads


def flat_patch(d, A, B, C):
    u, v = rules.interp_nodes(d)
    y = A[:, None] + u[None, :] * (B - A)[:, None] + v[None, :] * (C - A)[:, None]
    return geometry.make_patch(d, y)


A0 = np.array([0.1, -0.2, 0.3])
B0 = np.array([1.2, 0.1, 0.25])
C0 = np.array([0.3, 0.9, 0.5])


def test_flat_patch_geometry():
    pt = flat_patch(5, A0, B0, C0)
    area2 = np.linalg.norm(np.cross(B0 - A0, C0 - A0))
    assert np.allclose(pt.J, area2, rtol=1e-13)
    assert np.allclose(pt.c, (A0 + B0 + C0) / 3, atol=1e-14)
    # the vertices are in the sample set, and for a flat triangle the farthest point is a vertex
    assert abs(pt.R - max(np.linalg.norm(P - pt.c) for P in (A0, B0, C0))) < 1e-13
    X, N, _ = pt.eval(np.array([0.2]), np.array([0.3]))
    assert np.allclose(X[:, 0], A0 + 0.2 * (B0 - A0) + 0.3 * (C0 - A0), atol=1e-14)
    assert np.allclose(N[:, 0], np.cross(B0 - A0, C0 - A0), atol=1e-13)
    assert abs(pt.dj - np.sqrt(area2 * rules.interp_weights(5).min())) < 1e-14


def test_curved_patch_interpolation_converges():
    errs = []
    for d in (2, 4, 6, 8):
        s = workloads.ellipsoid(2, d)
        pt = geometry.make_patch(d, s.xyz[:, s.node_off[0]:s.node_off[1]])
        tri = s.meta["triangles"][0]
        u = np.array([0.13, 0.61, 0.3])
        v = np.array([0.22, 0.05, 0.41])
        p = tri[0][:, None] + u * (tri[1] - tri[0])[:, None] + v * (tri[2] - tri[0])[:, None]
        exact = p / np.linalg.norm(p, axis=0)
        X, N, _ = pt.eval(u, v)
        errs.append(np.abs(X - exact).max())
        # outward orientation
        assert (np.einsum("ip,ip->p", N, X) > 0).all()
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < 1e-6


def test_kernels_match_finite_differences(rng):
    x = np.array([0.3, -0.2, 0.5])
    X = rng.standard_normal((3, 5))
    N = rng.standard_normal((3, 5))
    k = 2.5 + 0.1j
    G = lambda y: np.exp(1j * k * np.linalg.norm(x - y)) / (4 * np.pi * np.linalg.norm(x - y))  # noqa
    h = 1e-6
    for p in range(5):
        grad = np.array([(G(X[:, p] + h * e) - G(X[:, p] - h * e)) / (2 * h) for e in np.eye(3)])
        d = kernel_jac(x, X[:, p:p + 1], N[:, p:p + 1], k, "D")[0]
        assert abs(d - N[:, p] @ grad) < 1e-7 * abs(d) + 1e-12
        s = kernel_jac(x, X[:, p:p + 1], N[:, p:p + 1], k, "S")[0]
        assert abs(s - G(X[:, p]) * np.linalg.norm(N[:, p])) < 1e-14
    a, b = 0.7 - 0.2j, 1.3j
    cf = kernel_jac(x, X, N, k, "CFIE", a, b)
    assert np.allclose(cf, a * kernel_jac(x, X, N, k, "D") + b * kernel_jac(x, X, N, k, "S"))
    # r = 0 contributes nothing
    assert kernel_jac(x, x[:, None], N[:, :1], k, "CFIE", a, b)[0] == 0


def test_truth_closed_forms_vs_brute_force():
    # the closed forms used as pins agree with plain high-order quadrature at a distance
    u, v, w = rules.conical_rule(30)
    y = A0[:, None] + u * (B0 - A0)[:, None] + v * (C0 - A0)[:, None]
    area2 = np.linalg.norm(np.cross(B0 - A0, C0 - A0))
    nrm = np.cross(B0 - A0, C0 - A0) / area2
    for x in (np.array([0.5, 0.3, 1.5]), np.array([0.4, 0.2, -0.9]), np.array([2.0, 2.0, 0.4])):
        r = np.linalg.norm(x[:, None] - y, axis=0)
        sl = (w * area2 / (4 * np.pi * r)).sum()
        dl = (w * area2 * (nrm @ (x[:, None] - y)) / (4 * np.pi * r ** 3)).sum()
        assert abs(truth.flat_single_layer(x, A0, B0, C0) - sl) < 1e-12
        assert abs(truth.laplace_dl_flat(x, A0, B0, C0) - dl) < 1e-12


@pytest.mark.parametrize("d", [3, 6])
def test_self_flat_closed_form(d):
    """S_0 self weights on a flat triangle sum to the in-plane closed form; D_0 self is 0."""
    pt = flat_patch(d, A0, B0, C0)
    for i in (0, 3, pt.n - 1):
        x = pt.y[:, i]
        exact = truth.flat_single_layer(x, A0, B0, C0)
        for order, tol in ((11, 1e-8), (16, 1e-12)):
            a = quadrature.self_weights(pt, i, x, quadrature.Kern("S", 0.0), order)
            assert abs(a.sum() - exact) < tol * abs(exact)
        a = quadrature.self_weights(pt, i, x, quadrature.Kern("D", 0.0), 14)
        assert np.abs(a).max() < 1e-12


@pytest.mark.parametrize("kind", ["S", "D", "CFIE"])
def test_self_curved_vs_truth(kind):
    s = workloads.ellipsoid(2, 6, axes=(1.0, 2.0, 3.0))
    pt = geometry.make_patch(6, s.xyz[:, s.node_off[7]:s.node_off[8]])
    k = 2 * np.pi
    kern = quadrature.Kern(kind, k, 1.0, -1j * k)
    sc = np.sqrt(pt.w * pt.J)
    for i in (0, 10, 27):
        x = pt.y[:, i]
        at = pt.V.T @ truth.moments_self(pt, i, x, kern)
        for eps in (1e-6, 1e-9):
            a = quadrature.self_weights(pt, i, x, kern, rules.default_self_order(eps))
            # per-target bound of Eq. errestself in the L2(Gamma_j) sense
            assert np.linalg.norm((a - at) / sc) < eps


def test_adaptive_flat_closed_forms():
    """Adaptive near integration of sigma = 1 over a flat triangle reproduces the Laplace
    double and single layer closed forms within the eps scaling of Eq. errestnear."""
    d = 4
    pt = flat_patch(d, A0, B0, C0)
    nrm = np.cross(B0 - A0, C0 - A0)
    nrm /= np.linalg.norm(nrm)
    eps = 1e-8
    tol0 = eps * pt.dj / pt.normV
    cache = quadrature.LeafCache(pt, 6)
    l2 = np.sqrt(pt.J[0] * 0.5)           # ||1||_{L2(Gamma_j)}
    cen = (A0 + B0 + C0) / 3
    pts = [cen + 0.01 * nrm, cen - 0.003 * nrm, A0 + 0.02 * (B0 - A0) + 0.01 * nrm,
           0.5 * (A0 + B0) + 0.002 * nrm - 0.01 * (C0 - A0)]
    for x in pts:
        for kind, exact in (("D", truth.laplace_dl_flat(x, A0, B0, C0)),
                            ("S", truth.flat_single_layer(x, A0, B0, C0))):
            I, st = quadrature.adaptive_moments(cache, x, quadrature.Kern(kind, 0.0), tol0, 24)
            got = (pt.V.T @ I).sum()
            assert abs(got - exact) < 4 * eps * l2, (kind, x, got, exact, st)
            assert st["leaves"] > 4 and not st["depth_hit"]


def test_adaptive_curved_vs_truth():
    s = workloads.ellipsoid(6, 6, axes=(1.0, 2.0, 3.0))
    pt = geometry.make_patch(6, s.xyz[:, s.node_off[3]:s.node_off[4]])
    k = 2 * np.pi
    kern = quadrature.Kern("CFIE", k, 1.0, -1j * k)
    X, N, _ = pt.eval(np.array([0.3, 0.02, 0.45]), np.array([0.3, 0.5, 0.53]))
    nh = N / np.linalg.norm(N, axis=0)
    eps = 1e-9
    tol0 = eps * pt.dj / pt.normV
    cache = quadrature.LeafCache(pt, 8)
    for p, h in ((0, 0.01), (1, -0.003), (2, 0.03)):
        x = X[:, p] + h * nh[:, p]
        I, st = quadrature.adaptive_moments(cache, x, kern, tol0, 24)
        It = truth.moments_adaptive(pt, x, kern)
        assert np.linalg.norm(I - It) < 2 * eps * pt.dj / pt.normV, st


def test_far_order_definition_and_far_accuracy():
    """q_j meets Eq. qj and the rule q_j integrates targets outside N_eta to eps d_j/||V||."""
    s = workloads.ellipsoid(2, 4)
    pt = geometry.make_patch(4, s.xyz[:, s.node_off[0]:s.node_off[1]])
    kern = quadrature.Kern("S", 1.0)
    eta = 2.0
    dirs = workloads.test_directions(3)
    F = [pt.c + eta * pt.R * dv for dv in dirs]
    for eps in (1e-6, 1e-9):
        q, sat, _ = quadrature.far_order(pt, F, kern, eps, 3, 24)
        assert not sat
        tol = eps * pt.dj / pt.normV
        for dv in workloads.test_directions(11)[:5]:
            x = pt.c + 1.05 * eta * pt.R * dv
            Iq = quadrature.rule_moments(pt, x, *rules.conical_rule(q), kern)
            assert np.linalg.norm(Iq - truth.moments_adaptive(pt, x, kern)) < 5 * tol
