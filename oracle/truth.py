"""Truth oracle: near machine-precision integrals by rules and formulas independent of
the scheme oracle, used only to pin it.

  * solid_angle: Van Oosterom & Strackee (IEEE TBME 30, 1983) signed solid angle of a
    flat triangle; the Laplace double layer of sigma = 1 over it is -Omega/(4 pi).
  * flat_single_layer: Laplace single layer of sigma = 1 over a flat triangle at any
    point: split at the foot point in the plane, integrate the radial part in closed
    form (sqrt(rho^2 + z^2) - |z|) and the angle numerically (adaptive Gauss-Kronrod).
  * moments_adaptive: I_nm(x) for an off-patch target by adaptive subdivision with a
    collapsed Gauss-Legendre x Gauss-Legendre rule and a relative tolerance near 1e-14.
  * moments_self: I_nm(x_i) for the target at node i: conformal affine change of
    variables, Duffy splitting at the node, Gauss-Legendre in s and geometrically
    graded Gauss-Legendre panels in t (no sinh map).
  * sphere_eigen_S / sphere_eigen_D: eigenvalues of S_k and D_k on the unit sphere for
    spherical harmonics of degree n: S: i k j_n(k) h_n(k); D (principal value, outward
    normal): i k^2 j_n(k) h_n'(k) + 1/2.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate
from scipy.special import roots_legendre, spherical_jn, spherical_yn

from . import rules


def solid_angle(x, A, B, C):
    """Signed solid angle of the flat triangle (A, B, C) seen from x, in closed form (Van
    Oosterom and Strackee): a pin of the Laplace double layer, not a step of the paper."""
    R1, R2, R3 = A - x, B - x, C - x
    r1, r2, r3 = np.linalg.norm(R1), np.linalg.norm(R2), np.linalg.norm(R3)
    num = np.dot(R1, np.cross(R2, R3))
    den = r1 * r2 * r3 + np.dot(R1, R2) * r3 + np.dot(R1, R3) * r2 + np.dot(R2, R3) * r1
    return 2.0 * np.arctan2(num, den)


def laplace_dl_flat(x, A, B, C):
    """int_T n.grad_y (1/(4 pi |x-y|)) dA, n oriented by (B-A) x (C-A): the k = 0 double
    layer of Sec. 3 over a flat triangle, in closed form from the solid angle."""
    return -solid_angle(np.asarray(x, float), A, B, C) / (4.0 * np.pi)


def flat_single_layer(x, A, B, C):
    """int_T 1/(4 pi |x-y|) dA for a flat triangle T = (A, B, C) and any point x: the k = 0
    single layer of Sec. 3, radial part in closed form (module docstring)."""
    x = np.asarray(x, float)
    n = np.cross(B - A, C - A)
    n = n / np.linalg.norm(n)
    z = float(np.dot(x - A, n))
    F = x - z * n                       # foot point in the plane
    e1 = (B - A) / np.linalg.norm(B - A)
    e2 = np.cross(n, e1)
    to2 = lambda P: np.array([np.dot(P - F, e1), np.dot(P - F, e2)])  # noqa: E731
    verts = [to2(A), to2(B), to2(C)]
    total = 0.0
    az = abs(z)
    for k in range(3):
        P0, P1 = verts[k], verts[(k + 1) % 3]
        D = P1 - P0
        Lk = np.linalg.norm(D)
        # signed distance from the origin (foot point) to the edge line; positive inside
        h = (P0[0] * D[1] - P0[1] * D[0]) / Lk
        if abs(h) < 1e-300:
            continue
        s0 = np.dot(P0, D) / Lk
        s1 = np.dot(P1, D) / Lk
        th0, th1 = np.arctan2(s0, abs(h)), np.arctan2(s1, abs(h))
        f = lambda th: np.sqrt((h / np.cos(th)) ** 2 + z * z) - az  # noqa: E731
        val, _ = integrate.quad(f, th0, th1, epsabs=1e-16, epsrel=1e-14, limit=200)
        total += np.sign(h) * val
    return total / (4.0 * np.pi)


def _collapsed_gl(m):
    """Collapsed (Duffy) Gauss-Legendre product rule on T0, independent of the scheme
    oracle's conical rules (a textbook construction)."""
    a, wa = roots_legendre(m)
    a = (a + 1) / 2
    wa = wa / 2
    u = (a[None, :] * (1 - a[:, None])).ravel()
    v = np.repeat(a, m)
    w = (wa[:, None] * wa[None, :] * (1 - a[:, None])).ravel()
    return u, v, w


def moments_adaptive(patch, x, kern, rtol=1e-15, m=14, max_level=14):
    """I_nm(x) (the Sec. 4.2 moments) for a target off the patch, to near machine
    precision, by adaptive midpoint subdivision (depth first) with an independent rule.

    A triangle is accepted when its children agree with it to rtol * |I_T0| (absolute,
    independent of the level), so the total error is below (#leaves) rtol |I_T0|."""
    rule = _collapsed_gl(m)

    def mom(T):
        u, v, w = rules.map_rule(T, *rule)
        X, N, K = patch.eval(u, v)
        return K @ (w * kern(x, X, N))

    I0 = mom(rules.T0)
    scale = max(np.linalg.norm(I0), 1e-300)

    def rec(T, I_T, level):
        kids = rules.subdivide(T)
        Ic = [mom(c) for c in kids]
        S = sum(Ic)
        if np.linalg.norm(S - I_T) <= rtol * scale or level >= max_level:
            return S
        return sum(rec(c, i, level + 1) for c, i in zip(kids, Ic))

    return rec(rules.T0, I0, 0)


def _graded_panels(length, mu, ratio=0.2):
    """Panels of [0, length] graded geometrically toward 0, finest ~ mu*1e-2 (textbook
    graded quadrature for the near-singular direction of the self integrals of Sec. 4)."""
    edges = [length]
    while edges[-1] > max(mu * 1e-2, 1e-14 * length):
        edges.append(edges[-1] * ratio)
    edges.append(0.0)
    return edges[::-1]


def moments_self(patch, i, x, kern, ns=40, nt=24):
    """I_nm (Sec. 4.2 moments) at node i, the self integral, to near machine precision:
    affine-conformal change of variables at the node (G^{-1/2} from
    the closed-form 2x2 square root), Duffy split at the node, Gauss-Legendre in s and
    geometrically graded Gauss-Legendre panels in t."""
    from . import koornwinder as kw
    from . import rules as R
    un, vn = R.interp_nodes(patch.d)
    P = np.array([un[i], vn[i]])
    _, Ku, Kv = kw.basis(patch.d, un[i:i + 1], vn[i:i + 1], derivs=True)
    A = np.stack([patch.coefs.T @ Ku[:, 0], patch.coefs.T @ Kv[:, 0]], axis=1)
    G = A.T @ A
    sq = np.sqrt(np.linalg.det(G))
    root = (G + sq * np.eye(2)) / np.sqrt(np.trace(G) + 2.0 * sq)   # sqrt(G)
    M = np.linalg.inv(root)
    detM = abs(np.linalg.det(M))
    verts = [root @ (np.array(vx) - P) for vx in ((0.0, 0.0), (1.0, 0.0), (0.0, 1.0))]
    s, ws = R.gauss_legendre01(ns)
    g, wg = R.gauss_legendre01(nt)
    I = 0.0
    for e in range(3):
        E0, E1 = verts[e], verts[(e + 1) % 3]
        D = E1 - E0
        L = np.hypot(*D)
        t0 = float(np.clip(np.dot(-E0, D) / (L * L), 0.0, 1.0))
        area2 = abs(E0[0] * D[1] - E0[1] * D[0])
        mu = area2 / (L * L)
        ts, wts = [], []
        for side, length in ((1.0, 1.0 - t0), (-1.0, t0)):
            if length <= 0:
                continue
            ed = _graded_panels(length, mu)
            for a, b in zip(ed[:-1], ed[1:]):
                ts.append(t0 + side * (a + (b - a) * g))
                wts.append((b - a) * wg)
        t = np.concatenate(ts)
        wt = np.concatenate(wts)
        E = E0[None, :] + t[:, None] * D[None, :]
        Z = (s[:, None, None] * E[None, :, :]).reshape(-1, 2)
        UV = P[None, :] + Z @ M.T
        ww = (ws[:, None] * wt[None, :] * s[:, None] * area2 * detM).ravel()
        X, N, K = patch.eval(UV[:, 0], UV[:, 1])
        I = I + K @ (ww * kern(x, X, N))
    return I


def sphere_eigen_S(n, k):
    """Eigenvalue of the single layer S_k of Sec. 3 on the unit sphere for spherical
    harmonics of degree n, in closed form: i k j_n(k) h_n(k)."""
    h = spherical_jn(n, k) + 1j * spherical_yn(n, k)
    return 1j * k * spherical_jn(n, k) * h


def sphere_eigen_D(n, k):
    """Eigenvalue of the double layer D_k of Sec. 3 (principal value, outward normal) on the
    unit sphere for degree-n harmonics, in closed form: i k^2 j_n(k) h_n'(k) + 1/2."""
    hp = spherical_jn(n, k, derivative=True) + 1j * spherical_yn(n, k, derivative=True)
    return 1j * k * k * spherical_jn(n, k) * hp + 0.5
