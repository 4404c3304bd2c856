"""Reference-triangle rules on T0: discretization nodes, V = U^{-1}, smooth rules,
self (singular) rules.  Sec. 2.1-2.2 and Sec. 4 (self interaction, Eq. errestself).

Readings (the paper's tables are not in the paper):
  * Discretization nodes (stand-in for Vioreanu-Rokhlin, Sec. 2.2): the
    Blyth-Pozrikidis construction on the d+1 interior Gauss-Lobatto points of
    [0,1] (roots of P^{(1,1)}_{d+1}).  Interior, positive interpolatory weights.
  * Smooth rule family (stand-in for Xiao-Gimbutas / VR rules of order q,
    Sec. 2.2 and 4.2): Stroud conical products, rule m has m^2 nodes
    (u, v) = (b (1-a), a), a ~ Gauss-Jacobi (weight 1-a), b ~ Gauss-Legendre,
    exact for total degree <= 2m-1.
  * Self rule for node i (stand-in for the generalized Gaussian rules of
    Bremer-Gimbutas): after an affine change of variables that makes the chart
    conformal at the node, T0 is split at the node into three triangles, each
    Duffy-mapped (s radial from the node, t along the opposite edge).  s uses
    n_s-point Gauss-Legendre; t is split at the foot of the perpendicular from the
    node and each side uses the sinh substitution t - t0 = mu sinh(xi), mu = h/L
    (Johnston & Elliott 2005), which removes the near-singular peak of flat
    sub-triangles, with [0, xi_max] cut into panels of length <= 1.5 carrying
    n_t-point Gauss-Legendre each.
"""
from __future__ import annotations

import numpy as np
from scipy.special import roots_jacobi, roots_legendre

from . import koornwinder as kw


def gauss_legendre01(n: int):
    """Textbook n-point Gauss-Legendre rule moved to [0, 1] (a building block of the smooth
    and self rules that stand in for the tables of Sec. 2.2)."""
    x, w = roots_legendre(n)
    return (x + 1.0) / 2.0, w / 2.0


def interp_nodes(d: int):
    """Discretization nodes (u_l, v_l) of degree d (Sec. 2.1), BP on interior Lobatto points.

    Node order: i = 0..d, j = 0..d-i, k = d-i-j;
    u = (1 + 2 t_i - t_j - t_k)/3, v = (1 + 2 t_j - t_i - t_k)/3.
    """
    x, _ = roots_jacobi(d + 1, 1.0, 1.0)
    t = np.sort((x + 1.0) / 2.0)
    u, v = [], []
    for i in range(d + 1):
        for j in range(d + 1 - i):
            k = d - i - j
            u.append((1.0 + 2.0 * t[i] - t[j] - t[k]) / 3.0)
            v.append((1.0 + 2.0 * t[j] - t[i] - t[k]) / 3.0)
    return np.array(u), np.array(v)


def vals_to_coefs(d: int) -> np.ndarray:
    """V[(nm), l] with c_nm = sum_l V[(nm), l] f_l (Eq. v2c); U[l, (nm)] = K_nm(u_l, v_l)."""
    u, v = interp_nodes(d)
    U = kw.basis(d, u, v).T
    return np.linalg.inv(U)


def interp_weights(d: int) -> np.ndarray:
    """Interpolatory weights w_l of the node set (the quadrature use of the nodes, Sec. 2.2):
    w = V^T m, m_(nm) = integral of K_nm = delta/sqrt(2)."""
    V = vals_to_coefs(d)
    mom = np.zeros(V.shape[0])
    mom[0] = 1.0 / np.sqrt(2.0)
    return V.T @ mom


def norm_V(d: int) -> float:
    """Operator 2-norm ||V|| used in the tolerance eps d_j / ||V|| (Eq. qj)."""
    return float(np.linalg.norm(vals_to_coefs(d), 2))


def conical_rule(m: int):
    """Smooth rule of the family, m^2 nodes, exact to total degree 2m-1: the stand-in for
    the order-q rules of Sec. 2.2 and 4.2 (their tables are not printed), a Stroud
    conical product.

    Integral over T0 of f = int_0^1 int_0^1 f(b(1-a), a) (1-a) db da.
    """
    x, wj = roots_jacobi(m, 1.0, 0.0)       # weight (1-x) on [-1,1]
    a = (1.0 + x) / 2.0
    wa = wj / 4.0                           # (1-x) dx = 4 (1-a) da
    b, wb = gauss_legendre01(m)
    u = (b[None, :] * (1.0 - a[:, None])).ravel()
    v = np.repeat(a, m)
    w = (wa[:, None] * wb[None, :]).ravel()
    return u, v, w


def self_rule(d: int, i: int, ns: int, nt: int, M=None, offsets: bool = False):
    """Singular rule on T0 for the target at node i (reading of Sec. 4, Eq. errestself).

    M is a 2x2 matrix mapping local coordinates zeta to reference offsets
    (u, v) - P = M zeta; the caller chooses M = G^{-1/2}, G = DX^T DX at the node, so
    that the chart is conformal at the node in zeta (the affine normalization used by
    generalized Gaussian self rules).  M = None means the identity.  In zeta
    coordinates the image of T0 is split at the node into three triangles, each
    Duffy-mapped (s radial, t along the opposite edge); s uses ns-point
    Gauss-Legendre, t is split at the foot of the perpendicular from the node and each
    side uses t - t0 = mu sinh(xi), mu = h/L, with [0, xi_max] cut into
    ceil(xi_max / 1.5) equal panels of nt-point Gauss-Legendre.
    Returns (u, v, w) on T0 (and the offsets (u - u_i, v - v_i) computed directly
    when offsets=True); the weights carry all Jacobians.
    """
    un, vn = interp_nodes(d)
    P = np.array([un[i], vn[i]])
    M = np.eye(2) if M is None else np.asarray(M, dtype=np.float64)
    Minv = np.linalg.inv(M)
    detM = abs(np.linalg.det(M))
    verts = [Minv @ (np.array(vx) - P) for vx in ((0.0, 0.0), (1.0, 0.0), (0.0, 1.0))]
    s, ws = gauss_legendre01(ns)
    xg, wg = gauss_legendre01(nt)
    out_z, out_w = [], []
    for e in range(3):
        E0, E1 = verts[e], verts[(e + 1) % 3]
        D = E1 - E0
        L = float(np.hypot(D[0], D[1]))
        t0 = float(np.clip(np.dot(-E0, D) / (L * L), 0.0, 1.0))
        area2 = abs(E0[0] * D[1] - E0[1] * D[0])   # = L h, apex at the origin
        mu = area2 / (L * L)                       # h / L
        for side, length in ((+1.0, 1.0 - t0), (-1.0, t0)):
            if length <= 0.0:
                continue
            xi_max = float(np.arcsinh(length / mu))
            npan = max(1, int(np.ceil(xi_max / SELF_XI_PANEL)))
            for pnl in range(npan):
                lo = xi_max * pnl / npan
                hi = xi_max * (pnl + 1) / npan
                xi = lo + (hi - lo) * xg
                t = t0 + side * mu * np.sinh(xi)
                wt = wg * (hi - lo) * mu * np.cosh(xi)
                E = E0[None, :] + t[:, None] * D[None, :]
                for a in range(ns):
                    out_z.append(s[a] * E)
                    out_w.append(ws[a] * wt * s[a] * area2 * detM)
    Z = np.concatenate(out_z)
    W = np.concatenate(out_w)
    dUV = Z @ M.T
    UV = P[None, :] + dUV
    if offsets:
        return UV[:, 0], UV[:, 1], W, dUV[:, 0], dUV[:, 1]
    return UV[:, 0], UV[:, 1], W


SELF_XI_PANEL = 1.5


def default_self_order(eps: float) -> int:
    """n_s = n_t of the self rule for precision eps: ceil(1.2 digits) + 3, within [6, 24]
    (the self rules of Sec. 4 come from tables the paper does not print; this order is
    this oracle's choice, shared with the library)."""
    digits = -np.log10(min(max(eps, 1e-15), 1e-1))
    return int(min(24, max(6, int(np.ceil(1.2 * digits - 1e-9)) + 3)))


def subdivide(T):
    """Midpoint split of a triangle (a, b, c) into 4 children (Sec. 4.3 steps 1-2).

    Child order: (a, ab, ca), (ab, b, bc), (ca, bc, c), (bc, ca, ab).
    """
    a, b, c = T
    ab, bc, ca = (a + b) / 2.0, (b + c) / 2.0, (c + a) / 2.0
    return [(a, ab, ca), (ab, b, bc), (ca, bc, c), (bc, ca, ab)]


def map_rule(T, ru, rv, rw):
    """Push a T0 rule onto the sub-triangle T = (a, b, c) of T0: y = a + s(b-a) + t(c-a)
    (the rules on the descendants of Sec. 4.3)."""
    a, b, c = T
    e1, e2 = b - a, c - a
    det = abs(e1[0] * e2[1] - e1[1] * e2[0])
    u = a[0] + ru * e1[0] + rv * e2[0]
    v = a[1] + ru * e1[1] + rv * e2[1]
    return u, v, rw * det


T0 = (np.array([0.0, 0.0]), np.array([1.0, 0.0]), np.array([0.0, 1.0]))
