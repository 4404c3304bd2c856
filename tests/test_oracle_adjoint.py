"""Pins of the oracle's adjoint (oracle/adjoint.py) against what fixes it independently:
central finite differences of the kernel and of the whole forward method, and the
adjoint identity <A sigma, g> = <sigma, A^H g>."""
import numpy as np
import pytest

from oracle import adjoint as OA
from oracle import corrections as C
from oracle.kernels import kernel_jac
from paper_2006_02545_gb300 import workloads as W


@pytest.mark.parametrize("kind,k", [("S", 1.3), ("D", 2.0 + 0.4j), ("CFIE", 3.1)])
def test_kernel_derivatives_match_central_differences(kind, k):
    rng = np.random.default_rng(5)
    x = rng.standard_normal(3)
    X = x[:, None] + rng.uniform(0.2, 1.5, 6)[None, :] * rng.standard_normal((3, 6))
    N = rng.standard_normal((3, 6))
    a, b = 0.7 - 0.2j, -1j * k
    dX, dN = OA.kernel_jac_grad(x, X, N, k, kind, a, b)
    h = 1e-6
    for c in range(3):
        e = np.zeros((3, 1))
        e[c] = h
        fdX = (kernel_jac(x, X + e, N, k, kind, a, b) - kernel_jac(x, X - e, N, k, kind, a, b)) / (2 * h)
        fdN = (kernel_jac(x, X, N + e, k, kind, a, b) - kernel_jac(x, X, N - e, k, kind, a, b)) / (2 * h)
        scale = np.abs(kernel_jac(x, X, N, k, kind, a, b)).max()
        assert np.abs(fdX - dX[c]).max() <= 1e-7 * scale
        assert np.abs(fdN - dN[c]).max() <= 1e-7 * scale


def _case():
    s = W.ellipsoid(1, 2, axes=(1.0, 1.2, 0.9))
    xo = W.radial_targets(s, 5, 4, 0.03, 0.6, True)
    return s, xo


def test_apply_adjoint_identity():
    """<A sigma, g> = <sigma, A^H g> for on- and off-surface targets (self, near, far)."""
    s = W.ellipsoid(1, 2)
    xs, tns = W.onsurface_targets(s)
    xo = W.radial_targets(s, 6, 2, 0.02, 0.5, True)
    x = np.concatenate([xs[:, ::7], xo], axis=1)
    tn = np.concatenate([tns[::7], -np.ones(xo.shape[1], np.int64)])
    p = C.Params(eps=1e-6, test_dirs=W.test_directions(3))
    kind, k, a, b = "CFIE", 2.0 + 0.1j, 1.0, -2j
    corr = C.gen_corrections(s.deg, s.node_off, s.xyz, x, tn, kind, k, a, b, params=p)
    rng = np.random.default_rng(1)
    for _ in range(2):
        sig = rng.standard_normal(s.n_points) + 1j * rng.standard_normal(s.n_points)
        g = rng.standard_normal(x.shape[1]) + 1j * rng.standard_normal(x.shape[1])
        u = C.apply_corrected(corr, s.node_off, sig, x, kind, k, a, b)
        ah = OA.apply_adjoint(corr, s.node_off, g, x, kind, k, a, b)
        lhs, rhs = np.vdot(g, u), np.vdot(ah, sig)
        assert abs(lhs - rhs) <= 1e-12 * np.abs(g).sum() * np.abs(u).max() * 10


@pytest.mark.parametrize("kind,k", [("S", 1.3), ("CFIE", 2.2)])
def test_shape_gradient_matches_finite_differences(kind, k):
    """dL/dy of L = Re sum conj(g) u with every discrete choice frozen, against central
    differences (step 1e-6) of the full forward method (near lists, far orders and
    refinement rerun at each perturbed geometry) on sampled coordinates."""
    s, x = _case()
    tn = -np.ones(x.shape[1], np.int64)
    a, b = 1.0, -1j * k
    p = C.Params(eps=1e-7, test_dirs=W.test_directions(3))
    rng = np.random.default_rng(2)
    sig = W.density(s.n_points, 3)
    g = rng.standard_normal(x.shape[1]) + 1j * rng.standard_normal(x.shape[1])
    grad, corr = OA.shape_gradient(s.deg, s.node_off, s.xyz, x, tn, kind, k, a, b, p, sig, g)
    assert any(ad.any() for _, ad, _ in corr.near)       # adaptive pairs are exercised
    assert any((~ad).any() for _, ad, _ in corr.near)    # and annulus pairs

    def L(xyz):
        c = C.gen_corrections(s.deg, s.node_off, xyz, x, tn, kind, k, a, b, params=p)
        return float(np.real(np.vdot(g, C.apply_corrected(c, s.node_off, sig, x, kind, k, a, b))))

    # the coordinates with the largest gradients plus random ones
    flat = np.abs(grad).ravel()
    pick = list(np.argsort(flat)[-3:]) + list(rng.choice(flat.size, 3, replace=False))
    h = 1e-6
    for idx in pick:
        c, i = divmod(int(idx), s.n_points)
        xp, xm = s.xyz.copy(), s.xyz.copy()
        xp[c, i] += h
        xm[c, i] -= h
        fd = (L(xp) - L(xm)) / (2 * h)
        assert abs(fd - grad[c, i]) <= 1e-6 * max(abs(grad[c, i]), 1e-2 * flat.max()), (c, i, fd, grad[c, i])
