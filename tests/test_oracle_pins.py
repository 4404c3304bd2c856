"""Pins of the oracle's parts that the other pins reach only indirectly:

  * koornwinder.basis_delta (K_nm(P + delta) - K_nm(P) by difference recurrences, used by
    every self weight) against the two values evaluated in 50-digit arithmetic from the
    Legendre and Jacobi polynomials of mpmath, for every degree and offsets 1e-1 .. 1e-9;
  * kernels.kernel_jac at k = 0 against the Laplace closed forms;
  * kernels.kernel_envelope (the rounding floor of the adaptive test): for S it is the
    kernel value's magnitude; for D, S' and the CFIE's double-layer part it is exactly the
    change of the kernel per unit coordinate error along the normal times R, in the tangent
    plane where that change is largest; and it bounds the FP64 rounding error of kernel_jac
    (against the 50-digit kernel at the same inputs) over near-singular configurations;
  * truth.sphere_eigen_S / sphere_eigen_D (the Bessel-function eigenvalues the pipeline is
    checked against) against the defining surface integrals over the exact unit sphere,
    by Gauss-Legendre quadrature in geodesic polar coordinates about the target.
"""
import numpy as np
import pytest

from oracle import koornwinder as kw
from oracle import truth
from oracle.kernels import kernel_envelope, kernel_jac

mp = pytest.importorskip("mpmath")

U = 2.0 ** -53   # unit roundoff of FP64


def basis_mp(d, u, v):
    """K_nm(u, v) in mpmath: c_nm (1-v)^m P^{(0,2m+1)}_{n-m}(1-2v) P_m((2u+v-1)/(1-v))."""
    out = []
    q = 1 - v
    for n in range(d + 1):
        for m in range(n + 1):
            c = mp.sqrt(2 * (2 * m + 1) * (n + 1))
            out.append(c * q ** m * mp.legendre(m, (2 * u + v - 1) / q) *
                       mp.jacobi(n - m, 0, 2 * m + 1, 1 - 2 * v))
    return out


@pytest.mark.parametrize("d", range(1, 11))
def test_basis_delta_matches_extended_precision(d):
    rng = np.random.default_rng(100 + d)
    points = [tuple(rng.dirichlet([2.0, 2.0, 2.0])[:2]), (0.04, 0.9)]
    with mp.workdps(50):
        for P in points:
            K0 = basis_mp(d, mp.mpf(P[0]), mp.mpf(P[1]))
            for e in (1, 3, 5, 7, 9):
                ang = rng.uniform(0.0, 2.0 * np.pi)
                du, dv = 10.0 ** -e * np.cos(ang), 10.0 ** -e * np.sin(ang)
                if P[1] + dv >= 1.0 or P[0] + du < 0.0:
                    du, dv = -du, -dv
                got = kw.basis_delta(d, P, np.array([du]), np.array([dv]))[:, 0]
                K1 = basis_mp(d, mp.mpf(P[0]) + mp.mpf(du), mp.mpf(P[1]) + mp.mpf(dv))
                ex = np.array([float(a - b) for a, b in zip(K1, K0)])
                scale = np.abs(ex).max()
                assert np.linalg.norm(got - ex) <= 1e-13 * np.linalg.norm(ex), (d, P, e)
                assert (np.abs(got - ex) <= 1e-12 * np.abs(ex) + 1e-14 * scale).all(), (d, P, e)


def _configs(rng, n=40, R=0.3):
    """Near-singular source/target pairs relative to a patch centroid: sources at |X| ~ R,
    targets at distance 1e-4 R .. R, some exactly in the source's tangent plane."""
    X = R * rng.uniform(-1.0, 1.0, (3, n))
    N = rng.standard_normal((3, n))
    N *= rng.uniform(0.05, 2.0, n) / np.linalg.norm(N, axis=0)
    dirs = rng.standard_normal((3, n))
    half = n // 2
    # first half: x - X orthogonal to N (tangent plane), second half: arbitrary directions
    nh = N[:, :half] / np.linalg.norm(N[:, :half], axis=0)
    dirs[:, :half] -= nh * (nh * dirs[:, :half]).sum(axis=0)
    dirs /= np.linalg.norm(dirs, axis=0)
    dist = R * 10.0 ** rng.uniform(-4.0, 0.0, n)
    return X, N, X + dist * dirs


@pytest.mark.parametrize("k", [0.0, 1.3, 2.0 * np.pi, 3.0 + 0.7j])
def test_kernel_envelope_bounds_fp64_rounding(k):
    """|kernel_jac (FP64) - kernel (50 digits, same FP64 inputs)| <= 8 u envelope."""
    rng = np.random.default_rng(7)
    R = 0.3
    X, N, x = _configs(rng, R=R)
    kk = mp.mpc(complex(k))
    for kind, al, be in (("S", 1.0, 0.0), ("D", 1.0, 0.0), ("CFIE", 1.0, -1j * complex(k) - 0.3)):
        worst = 0.0
        with mp.workdps(50):
            for p in range(X.shape[1]):
                got = kernel_jac(x[:, p], X[:, p:p + 1], N[:, p:p + 1], k, kind, al, be)[0]
                env = kernel_envelope(x[:, p], X[:, p:p + 1], N[:, p:p + 1], k, kind, al, be, R)[0]
                dv = [mp.mpf(float(x[c, p])) - mp.mpf(float(X[c, p])) for c in range(3)]
                nv = [mp.mpf(float(N[c, p])) for c in range(3)]
                r = mp.sqrt(sum(t * t for t in dv))
                e = mp.exp(1j * kk * r) / (4 * mp.pi * r)
                S = e * mp.sqrt(sum(t * t for t in nv))
                D = sum(a * b for a, b in zip(nv, dv)) * (1 - 1j * kk * r) * e / (r * r)
                exact = {"S": S, "D": D, "CFIE": mp.mpc(al) * D + mp.mpc(be) * S}[kind]
                err = abs(complex(exact) - got)
                worst = max(worst, err / (U * env))
        assert worst <= 8.0, (kind, k, worst)


def test_kernel_envelope_is_the_tangent_plane_sensitivity():
    """In the source's tangent plane, R |dK/dx_n| equals the double-layer envelope for D and
    S' (and the CFIE's envelope is |beta| |S| + |alpha| of that); for S the envelope is |S|."""
    rng = np.random.default_rng(9)
    R = 0.4
    X, N, x = _configs(rng, n=20, R=R)
    for k in (0.0, 1.7, 2.5 + 0.4j):
        for p in range(10):   # tangent-plane configurations
            Xp, Np, xp = X[:, p:p + 1], N[:, p:p + 1], x[:, p]
            nh = Np[:, 0] / np.linalg.norm(Np[:, 0])
            h = 1e-7 * np.linalg.norm(xp - Xp[:, 0])
            dK = (kernel_jac(xp + h * nh, Xp, Np, k, "D")[0] -
                  kernel_jac(xp - h * nh, Xp, Np, k, "D")[0]) / (2 * h)
            envD = kernel_envelope(xp, Xp, Np, k, "D", R=R)[0]
            assert abs(R * abs(dK) / envD - 1.0) < 1e-6
            # S' with the target normal along the source normal: same envelope form
            envSp = kernel_envelope(xp, Xp, Np, k, "Sp", R=R, nx=nh)[0]
            assert abs(envSp / envD - 1.0) < 1e-14
            envS = kernel_envelope(xp, Xp, Np, k, "S", R=R)[0]
            assert abs(envS / abs(kernel_jac(xp, Xp, Np, k, "S")[0]) - 1.0) < 1e-14
            al, be = 0.7 - 0.2j, 1.1 + 0.5j
            envC = kernel_envelope(xp, Xp, Np, k, "CFIE", al, be, R=R)[0]
            assert abs(envC / (abs(be) * envS + abs(al) * envD) - 1.0) < 1e-14


def test_kernels_reduce_to_laplace_closed_forms_at_k0():
    """k = 0: S J = |N| / (4 pi r), D J = N.(x - X) / (4 pi r^3), CFIE = alpha D + beta S,
    S' = -n_x.(x - X) |N| / (4 pi r^3); all real."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(3)
    X = x[:, None] + rng.standard_normal((3, 6))
    N = rng.standard_normal((3, 6))
    nx = rng.standard_normal(3)
    nx /= np.linalg.norm(nx)
    d = x[:, None] - X
    r = np.linalg.norm(d, axis=0)
    nN = np.linalg.norm(N, axis=0)
    S = nN / (4 * np.pi * r)
    D = (N * d).sum(axis=0) / (4 * np.pi * r ** 3)
    Sp = -(nx[:, None] * d).sum(axis=0) * nN / (4 * np.pi * r ** 3)
    assert np.allclose(kernel_jac(x, X, N, 0.0, "S"), S, rtol=1e-14, atol=0)
    assert np.allclose(kernel_jac(x, X, N, 0.0, "D"), D, rtol=1e-13, atol=0)
    assert np.allclose(kernel_jac(x, X, N, 0.0, "CFIE", 2.0, -0.5), 2.0 * D - 0.5 * S,
                       rtol=1e-13, atol=0)
    assert np.allclose(kernel_jac(x, X, N, 0.0, "Sp", nx=nx), Sp, rtol=1e-13, atol=0)
    # a source exactly at the target contributes 0
    assert kernel_jac(x, x[:, None], N[:, :1], 1.0, "CFIE", 1.0, -1j)[0] == 0.0


def _sphere_polar_integral(f, n, k):
    """int over the unit sphere of f(r, k) P_n(cos theta) dA, in geodesic polar coordinates
    about the target at the north pole (r = 2 sin(theta/2), dA = 2 pi sin(theta) dtheta,
    sin(theta)/r = cos(theta/2): the integrand is smooth for f ~ 1/r).  The target value
    of Y_n = P_n(cos theta) there is 1, so the integral is the eigenvalue."""
    from scipy.special import eval_legendre, roots_legendre
    t, w = roots_legendre(400)
    th = 0.5 * np.pi * (t + 1.0)
    w = 0.5 * np.pi * w
    r = 2.0 * np.sin(th / 2)
    return np.sum(w * f(r, k) * r * np.cos(th / 2) * 2.0 * np.pi * eval_legendre(n, np.cos(th)))


@pytest.mark.parametrize("n", [0, 1, 2, 3])
@pytest.mark.parametrize("k", [0.5, 1.0, 2.0 * np.pi])
def test_sphere_eigenvalues_match_the_surface_integrals(n, k):
    """S_k Y_n = int G_k Y_n dA and D_k Y_n = PV int n(y).grad_y G_k Y_n dA on the unit
    sphere (outward n: n(y).(x - y) = -r^2/2, so the double-layer kernel is
    -(1 - ikr) e^{ikr} / (8 pi r), integrable) against truth.sphere_eigen_S / _D."""
    S = _sphere_polar_integral(lambda r, k: np.exp(1j * k * r) / (4 * np.pi * r), n, k)
    D = _sphere_polar_integral(lambda r, k: -(1 - 1j * k * r) * np.exp(1j * k * r) / (8 * np.pi * r),
                               n, k)
    assert abs(S - truth.sphere_eigen_S(n, k)) <= 1e-13 * max(1.0, abs(S))
    assert abs(D - truth.sphere_eigen_D(n, k)) <= 1e-13 * max(1.0, abs(D))


def test_every_oracle_function_cites_what_it_follows():
    """Each public function and class of oracle/ states the passage of the paper it follows
    (section, equation, table, remark or figure), or that it is a closed form or textbook
    construction used as a pin, or that the paper has no counterpart."""
    import ast
    import os
    import re
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
    missing = []
    for fn in sorted(os.listdir(root)):
        if not fn.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(root, fn)).read())
        for node in tree.body:   # module-level definitions only (nested helpers excluded)
            if isinstance(node, (ast.FunctionDef, ast.ClassDef)) and not node.name.startswith("_"):
                doc = ast.get_docstring(node) or ""
                if not re.search(r"Sec\.|Eq\.|Table|Remark|Fig\.|closed form|textbook|counterpart",
                                 doc):
                    missing.append(f"{fn}:{node.name}")
    assert not missing, missing
