"""Patch geometry from node samples (Sec. 3.1-3.2, Sec. 4 centroid and radius).

x_nm = sum_l V[(nm), l] y_l (chart expansion, Sec. 3.2); X, X_u, X_v from the
Koornwinder series; n = X_u x X_v (unnormalized), J = |n| (Eq. loc).

Readings:
  * Centroid c_j (Sec. 4, printed as the unnormalized, unweighted integral of X
    over T0): the area-weighted centroid on the node rule,
    c_j = sum_l w_l J_l y_l / sum_l w_l J_l.
  * Radius R_j (Eq. rjdef, the minimal ball about c_j containing the patch): the
    largest |X - c_j| over the nodes and the 153 vertices of the level-4 uniform
    subdivision of T0, i.e. (a/16, b/16), a+b <= 16.
  * d_j = min_l sqrt(J_l w_l) (Sec. 4.2).
  * Local quadratures evaluate X - c_j (the series with x_00 shifted by c_j/K_00)
    against x - c_j: the same differences x - X, with rounding proportional to the
    patch size instead of the distance from the origin.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import koornwinder as kw
from . import rules


@dataclass
class Patch:
    """One patch's chart (Sec. 3.2) and the quantities of Sec. 4 built from it: V, ||V||,
    node weights and Jacobians, centroid c_j, radius R_j and d_j."""
    d: int
    y: np.ndarray          # [3, n] node coordinates
    coefs: np.ndarray      # [n, 3] Koornwinder coefficients x_nm
    V: np.ndarray          # [n, n]
    normV: float
    w: np.ndarray          # [n] node weights
    J: np.ndarray          # [n] Jacobian at the nodes
    c: np.ndarray          # [3] centroid
    R: float               # radius
    dj: float              # min sqrt(J w)
    coefs_rel: np.ndarray = None   # [n, 3] coefficients of X - c_j

    @property
    def n(self) -> int:
        """Nodes of the patch, n = (d+1)(d+2)/2 (Sec. 2.1)."""
        return kw.n_basis(self.d)

    def eval(self, u, v):
        """The chart X(u, v) = sum x_nm K_nm(u, v) and its normal N = X_u x X_v (Sec. 3.1-3.2)
        at reference points; returns (X [3,P], N [3,P], K [n,P])."""
        return self._eval(self.coefs, u, v)

    def eval_rel(self, u, v):
        """As eval (Sec. 3.2), with X measured from the centroid c_j of Sec. 4: X - c_j
        (the series with shifted x_00)."""
        return self._eval(self.coefs_rel, u, v)

    def _eval(self, coefs, u, v):
        """Chart series sum coefs_nm K_nm and its u, v derivatives (Sec. 3.2)."""
        K, Ku, Kv = kw.basis(self.d, u, v, derivs=True)
        X = coefs.T @ K
        Xu = coefs.T @ Ku
        Xv = coefs.T @ Kv
        N = np.cross(Xu, Xv, axis=0)
        return X, N, K


_TABLES: dict = {}


def tables(d: int):
    """Per degree: V = U^{-1} (Eq. v2c), ||V||_2 (the scale of Eq. qj), the node weights and
    the nodes (Sec. 2.1-2.2)."""
    if d not in _TABLES:
        V = rules.vals_to_coefs(d)
        _TABLES[d] = (V, float(np.linalg.norm(V, 2)), rules.interp_weights(d), rules.interp_nodes(d))
    return _TABLES[d]


def sample_points_level4():
    """The 153 vertices of the level-4 uniform subdivision of T0, the sample over which the
    radius R_j of Sec. 4 (Eq. rjdef) is taken (the paper does not say how R_j is found)."""
    a, b = np.meshgrid(np.arange(17), np.arange(17), indexing="ij")
    keep = (a + b) <= 16
    return a[keep] / 16.0, b[keep] / 16.0


def make_patch(d: int, y: np.ndarray) -> Patch:
    """One patch from its node coordinates y [3, n]: chart coefficients x_nm = V y (Sec. 3.2,
    Eq. v2c), Jacobian at the nodes, the area-weighted centroid c_j and radius R_j of Sec. 4
    (printed garbled: the centroid is read as sum w J y / sum w J), and d_j = min sqrt(J w)
    of Sec. 4.2."""
    V, nV, w, (un, vn) = tables(d)
    coefs = V @ y.T
    K, Ku, Kv = kw.basis(d, un, vn, derivs=True)
    Xu = coefs.T @ Ku
    Xv = coefs.T @ Kv
    J = np.linalg.norm(np.cross(Xu, Xv, axis=0), axis=0)
    wJ = w * J
    c = (y * wJ[None, :]).sum(axis=1) / wJ.sum()
    su, sv = sample_points_level4()
    Xs = coefs.T @ kw.basis(d, su, sv)
    R = max(np.linalg.norm(Xs - c[:, None], axis=0).max(),
            np.linalg.norm(y - c[:, None], axis=0).max())
    dj = float(np.sqrt(J * w).min())
    # X - c_j = sum x_nm K_nm - c_j, and K_00 = sqrt(2) is constant
    coefs_rel = coefs.copy()
    coefs_rel[0] -= c / np.sqrt(2.0)
    return Patch(d, y, coefs, V, nV, w, J, c, float(R), dj, coefs_rel)


def make_patches(deg, node_off, xyz):
    """make_patch (Sec. 3.2, Sec. 4) for every patch of a surface."""
    return [make_patch(int(deg[j]), xyz[:, node_off[j]:node_off[j + 1]]) for j in range(len(deg))]


def default_eta(d: int) -> float:
    """eta by the paper's order p = d+1: 2.75 (p <= 4), 2 (4 < p <= 8), 1.25 (p > 8) (Sec. 4.1, 5.2)."""
    p = d + 1
    if p <= 4:
        return 2.75
    if p <= 8:
        return 2.0
    return 1.25
