"""Local quadratures on one patch: smooth-rule moments, far order q_j, self weights,
adaptive near moments (Sec. 4.2-4.3, Eq. qj, errestself, errestnear).

I^j_nm(x) = int_T0 K(x, X(u,v)) K_nm(u,v) J(u,v) du dv; point weights
a_l(x) = sum_nm V[(nm), l] I_nm(x) (Sec. 4.3).
"""
from __future__ import annotations

from collections import deque

import numpy as np

from . import koornwinder as kw
from . import rules
from .kernels import kernel_envelope, kernel_jac


class Kern:
    """A kernel of Sec. 3 (S, D, CFIE or S') with its wavenumber and CFIE coefficients."""

    def __init__(self, kind, k, alpha=1.0, beta=0.0):
        self.kind, self.k, self.alpha, self.beta = kind, complex(k), complex(alpha), complex(beta)

    def __call__(self, x, X, N, nx=None):
        return kernel_jac(x, X, N, self.k, self.kind, self.alpha, self.beta, nx)

    def envelope(self, x, X, N, R):
        return kernel_envelope(x, X, N, self.k, self.kind, self.alpha, self.beta, R)


def rule_moments(patch, x, ru, rv, rw, kern, nx=None):
    """I_nm(x) of Sec. 4.2 by one rule (u_q, v_q, w_q) on T0: sum_q w_q K(x, X_q) J_q K_nm(u_q, v_q).
    Positions are taken relative to the patch centroid (x - c_j against X - c_j); nx is
    the target normal of S'."""
    X, N, K = patch.eval_rel(ru, rv)
    return K @ (rw * kern(np.asarray(x) - patch.c, X, N, nx))


def radial_normal(patch, x):
    """Target normal given to S' (Sec. 3) at a far-order test point of Sec. 4.2: the unit
    vector from c_j to x (a reading: the paper's test points carry no normal)."""
    d = np.asarray(x, dtype=np.float64) - patch.c
    r = np.linalg.norm(d)
    return d / r if r > 0.0 else np.array([0.0, 0.0, 1.0])


def far_order(patch, test_pts, kern, eps, m_min, m_max):
    """q_j of Eq. qj: smallest m with max_x ||I_m(x) - I_{m+1}(x)||_2 <= eps d_j/||V||.

    Returns (m, saturated, margin) with margin = |err - tol|/tol at the deciding step.
    """
    tol = eps * patch.dj / patch.normV

    def mom(m):
        ru, rv, rw = rules.conical_rule(m)
        X, N, K = patch.eval_rel(ru, rv)
        return [K @ (rw * kern(np.asarray(x) - patch.c, X, N, radial_normal(patch, x)))
                for x in test_pts]

    prev = mom(m_min)
    margin = np.inf
    for m in range(m_min, m_max):
        nxt = mom(m + 1)
        err = max((np.linalg.norm(a - b) for a, b in zip(prev, nxt)), default=0.0)
        margin = min(margin, abs(err - tol) / tol)
        if err <= tol:
            return m, False, margin
        prev = nxt
    return m_max, True, margin


def smooth_weights(patch, x, m, kern, nx=None):
    """Weights the smooth rule m puts on the nodes: s_l(x) = sum_q w_q K J (K(u_q) V)_l (Sec. 4.2 Remark)."""
    ru, rv, rw = rules.conical_rule(m)
    return patch.V.T @ rule_moments(patch, x, ru, rv, rw, kern, nx)


def conformal_map(patch, i):
    """M = G^{-1/2}, G = DX^T DX at node i (first fundamental form), by eigendecomposition:
    the change of variables that makes the chart conformal at the node, used by the self
    rules of Sec. 4 (whose printed tables are not available)."""
    un, vn = rules.interp_nodes(patch.d)
    _, Ku, Kv = kw.basis(patch.d, un[i:i + 1], vn[i:i + 1], derivs=True)
    A = np.stack([patch.coefs.T @ Ku[:, 0], patch.coefs.T @ Kv[:, 0]], axis=1)
    lam, Q = np.linalg.eigh(A.T @ A)
    return Q @ np.diag(lam ** -0.5) @ Q.T


def node_normal(patch, i):
    """Unit normal of the chart at node i (Sec. 3.2; the target normal of S', Sec. 3, for
    on-surface targets)."""
    un, vn = rules.interp_nodes(patch.d)
    _, N, _ = patch.eval(un[i:i + 1], vn[i:i + 1])
    return N[:, 0] / np.linalg.norm(N[:, 0])


def self_weights(patch, i, x, kern, order):
    """Self point weights a_l(x_i) for the target at node i (Sec. 4, Eq. errestself).

    The target is the chart's value at the node, X(P); the chord x - X(P + delta) is
    formed as -(X(P + delta) - X(P)) from Koornwinder differences (koornwinder.
    basis_delta), so that the near-singular double-layer factor n.(x - X) keeps its
    relative precision as delta -> 0.  (x itself is not used beyond that.)"""
    ru, rv, rw, du, dv = rules.self_rule(patch.d, i, order, order, conformal_map(patch, i),
                                         offsets=True)
    un, vn = rules.interp_nodes(patch.d)
    _, N, K = patch.eval_rel(ru, rv)
    dX = patch.coefs.T @ kw.basis_delta(patch.d, (un[i], vn[i]), du, dv)
    g = kern(np.zeros(3), dX, N, node_normal(patch, i) if kern.kind == "Sp" else None)
    return patch.V.T @ (K @ (rw * g))


class LeafCache:
    """Geometry at the leaf-rule nodes of sub-triangles, shared by all targets of a patch
    (reuse of X, K_nm and J across targets, Sec. 4.3 and Fig. multipletargpot)."""

    def __init__(self, patch, m):
        self.patch = patch
        self.rule = rules.conical_rule(m)
        self.memo = {}

    def get(self, path, T):
        """Leaf-rule geometry of sub-triangle T (path: its position in the Sec. 4.3 tree)."""
        if path not in self.memo:
            u, v, w = rules.map_rule(T, *self.rule)
            X, N, K = self.patch.eval_rel(u, v)
            self.memo[path] = (X, N, K, w)
        return self.memo[path]


ROUNDING_FLOOR = 2e-13


def adaptive_moments(cache: LeafCache, x, kern, tol0, max_depth, record=None, nx=None):
    """Adaptive integration of I_nm(x) over T0 by midpoint subdivision (Sec. 4.3).

    A triangle T at level L (|T|/|T0| = 4^-L) is compared with its 4 children;
    if ||I_T - sum_c I_c||_2 <= max(tol0 4^-L, 2e-13 sum_c E_c) the children's sum is
    accepted, otherwise each child is tested in turn (breadth first).  E_c is the
    rounding envelope of the kernel summed over child c's nodes (kernels.
    kernel_envelope): the second term is a rounding floor (a reading: the paper's
    absolute tolerance can fall below what FP64 resolves for near-singular
    integrands, and the double-layer integrand loses digits to cancellation for
    targets near the tangent plane).  Children at level max_depth are not tested
    further: their sum is accepted and the depth flag set.
    Returns (I [n], stats dict).  With `record` (a list), the accepted leaf triangles
    (the children of every accepted triangle) are appended to it.  nx: target normal (S').
    """
    patch = cache.patch
    xr = np.asarray(x) - patch.c

    def moments(path, T):
        X, N, K, w = cache.get(path, T)
        return K @ (w * kern(xr, X, N, nx))

    def envelope(path, T):
        X, N, K, w = cache.get(path, T)
        return float((w * kern.envelope(xr, X, N, patch.R)).sum())

    I_root = moments((), rules.T0)
    queue = deque([((), rules.T0, I_root)])
    total = np.zeros_like(I_root)
    leaves, tests, min_margin, depth_hit, max_level = 0, 0, np.inf, False, 0
    floor_sum = 0.0   # sum of the tolerances of tests decided by the rounding floor
    close_sum = 0.0   # sum of the tolerances of tests decided within 1e-3 of the threshold
    while queue:
        path, T, I_T = queue.popleft()
        L = len(path)
        kids = rules.subdivide(T)
        I_c = [moments(path + (c,), kids[c]) for c in range(4)]
        S = I_c[0] + I_c[1] + I_c[2] + I_c[3]
        E = sum(envelope(path + (c,), kids[c]) for c in range(4))
        err = float(np.linalg.norm(I_T - S))
        tauL = tol0 * 0.25 ** L
        tau = max(tauL, ROUNDING_FLOOR * E)
        if tau > tauL:
            floor_sum += tau
        tests += 1
        min_margin = min(min_margin, abs(err - tau) / tau)
        if abs(err - tau) < 1e-3 * tau:
            close_sum += tau
        if err <= tau or L + 1 >= max_depth:
            if err > tau:
                depth_hit = True
            total = total + S
            leaves += 4
            if record is not None:
                record.extend(kids)
            max_level = max(max_level, L + 1)
        else:
            for c in range(4):
                queue.append((path + (c,), kids[c], I_c[c]))
    return total, dict(leaves=leaves, tests=tests, margin=min_margin, depth_hit=depth_hit,
                       max_level=max_level, floor_sum=floor_sum, close_sum=close_sum, tol0=tol0)
