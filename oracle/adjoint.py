"""Adjoint of the corrected layer potential (an extension: the paper has no gradients).

Test infrastructure only, like the rest of this package.

The corrected potential at the targets is linear in the density, u = A(y) sigma, and
depends on the node coordinates y through the charts.  For a real functional L of u
with upstream gradient g = dL/d(conj u) (PyTorch's convention for complex tensors, so
that dL = Re sum_t conj(g_t) du_t):
  * the density gradient is A^H g (apply_adjoint);
  * the coordinate gradient (shape_gradient) differentiates the discrete method with
    every discrete choice frozen: near lists, far orders q_j, annulus orders and the
    adaptive refinement trees.  Then for an off-surface target
        u_t = sum_j sum_{nodes (u, w) of the rule used for (t, j)} w K~(x_t, X(u), N(u)) sigma_j(u),
    where the rule is q_j on T0 for a far pair, the annulus rule for an annulus pair
    and the leaf rule on the accepted leaves for an adaptive pair (for a near pair the
    stored correction a - s plus the smooth-rule far term leaves exactly the near rule,
    Sec. 5.3).  sigma_j(u) = sum_l phi_l(u) sigma_l does not depend on y; X = sum_nm
    x_nm K_nm(u) and N = X_u x X_v do, through x = V y (Sec. 3.2).
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import koornwinder as kw
from . import rules
from .corrections import gen_corrections
from .quadrature import Kern

FOUR_PI = 4.0 * np.pi


def kernel_jac_grad(x, X, N, k, kind: str, alpha=1.0, beta=0.0):
    """Derivatives of kernels.kernel_jac (the Sec. 3 kernels; the gradient itself has no
    counterpart in the paper) with respect to the source position X and the
    unnormalized normal N: (dX [3,P], dN [3,P]), complex.  With r = |x - X|:
      S~ = G(r) |N|, G = e^{ikr}/(4 pi r):
          dS~/dX = G (ik - 1/r) |N| (X - x)/r,      dS~/dN = G N/|N|
      D~ = h(r) (x - X).N, h = (1 - ikr) e^{ikr}/(4 pi r^3):
          dD~/dX = -h N + (x - X).N h'(r) (X - x)/r,  dD~/dN = h (x - X),
          h'(r) = e^{ikr} (k^2 r^2 + 3ikr - 3)/(4 pi r^4)
      CFIE = alpha D~ + beta S~.  A source at r = 0 gives 0 (as in kernel_jac)."""
    if kind not in ("S", "D", "CFIE"):
        raise ValueError(f"no source-geometry derivative for kernel {kind}")
    x = np.asarray(x, dtype=np.float64)
    k = complex(k)
    dvec = x[:, None] - X                       # x - X
    r = np.sqrt((dvec * dvec).sum(axis=0))
    zero = r == 0.0
    rs = np.where(zero, 1.0, r)
    e = np.exp(1j * k * rs)
    unit = -dvec / rs                           # (X - x)/r
    dX = np.zeros(X.shape, dtype=np.complex128)
    dN = np.zeros(X.shape, dtype=np.complex128)
    if kind in ("S", "CFIE"):
        c = 1.0 if kind == "S" else complex(beta)
        G = e / (FOUR_PI * rs)
        nN = np.sqrt((N * N).sum(axis=0))
        dX += c * (G * (1j * k - 1.0 / rs) * nN) * unit
        dN += c * (G / np.where(nN == 0.0, 1.0, nN)) * N
    if kind in ("D", "CFIE"):
        c = 1.0 if kind == "D" else complex(alpha)
        h = (1.0 - 1j * k * rs) * e / (FOUR_PI * rs ** 3)
        hp = e * (k * k * rs * rs + 3j * k * rs - 3.0) / (FOUR_PI * rs ** 4)
        ndx = (N * dvec).sum(axis=0)
        dX += c * (-h * N + (ndx * hp) * unit)
        dN += c * (h * dvec)
    dX[:, zero] = 0.0
    dN[:, zero] = 0.0
    return dX, dN


def apply_adjoint(corr, node_off, g, tgt_xyz, kind, k, alpha=1.0, beta=0.0):
    """A^H g for the corrected potential of corrections.apply_corrected (the adjoint of the
    Sec. 5.3 apply; no counterpart in the paper).

    Far part: u_t = sum_{q, patch(q) != own(t)} K~(x_t, X_q) (B_j sigma_j)_q with the real
    matrix B_j = diag(w) K^T V (interpolation to the rule q_j times its weights), so
    (A^H g)_j = B_j^T z with z_q = sum_t conj(K~(x_t, X_q)) g_t.  CSR part: conj(c) g."""
    kern = Kern(kind, k, alpha, beta)
    node_off = np.asarray(node_off)
    g = np.asarray(g, dtype=np.complex128)
    out = np.zeros(int(node_off[-1]), dtype=np.complex128)
    for t in range(tgt_xyz.shape[1]):
        a, b = corr.row_ptr[t], corr.row_ptr[t + 1]
        np.add.at(out, corr.col[a:b], np.conj(corr.val[a:b]) * g[t])
    for j, pt in enumerate(corr.patches):
        ru, rv, rw = rules.conical_rule(int(corr.q[j]))
        X, N, K = pt.eval(ru, rv)
        z = np.zeros(len(rw), dtype=np.complex128)
        for t in np.nonzero(corr.tgt_patch != j)[0]:
            z += np.conj(kern(tgt_xyz[:, t], X, N)) * g[t]
        B = (rw[:, None] * K.T) @ pt.V
        out[node_off[j]:node_off[j + 1]] += B.T @ z
    return out


def _rule_grad(pt, s_hat, ru, rv, rw, targets, tgt_xyz, g, k, kind, alpha, beta):
    """sum over the rule's nodes and the targets of dL/dx_nm (x the chart coefficients of
    Sec. 3.2; one rule of Sec. 4.2-4.3 with the rule frozen):
    per node a_X = Re(sum_t conj(g_t) w sigma(u) dK~/dX), a_N likewise with dK~/dN; since
    dN = dX_u x X_v + X_u x dX_v, a_N.dN = dX_u.(X_v x a_N) + dX_v.(a_N x X_u), so
        dL/dx_nm = sum_nodes K_nm a_X + dK_nm/du (X_v x a_N) + dK_nm/dv (a_N x X_u)."""
    K, Ku, Kv = kw.basis(pt.d, ru, rv, derivs=True)
    X, Xu, Xv = pt.coefs.T @ K, pt.coefs.T @ Ku, pt.coefs.T @ Kv
    N = np.cross(Xu, Xv, axis=0)
    sig = K.T @ s_hat
    aX = np.zeros(X.shape)
    aN = np.zeros(X.shape)
    for t in targets:
        dX, dN = kernel_jac_grad(tgt_xyz[:, t], X, N, k, kind, alpha, beta)
        c = np.conj(g[t]) * rw * sig
        aX += np.real(c * dX)
        aN += np.real(c * dN)
    bu = np.cross(Xv, aN, axis=0)
    bv = np.cross(aN, Xu, axis=0)
    return K @ aX.T + Ku @ bu.T + Kv @ bv.T


def shape_gradient(deg, node_off, xyz, tgt_xyz, tgt_node, kind, k, alpha, beta, params, sigma,
                   g):
    """dL/dy [3, N] for dL = Re sum_t conj(g_t) du_t at off-surface targets, with the
    discrete choices of gen_corrections (Sec. 4.2-4.3) frozen (module docstring; no
    counterpart in the paper).  Returns (grad, corr)."""
    tgt_node = np.asarray(tgt_node)
    if (tgt_node >= 0).any():
        raise ValueError("shape gradient: off-surface targets only")
    p = replace(params, record_leaves=True)
    corr = gen_corrections(deg, node_off, xyz, tgt_xyz, tgt_node, kind, k, alpha, beta, params=p)
    node_off = np.asarray(node_off)
    g = np.asarray(g, dtype=np.complex128)
    sigma = np.asarray(sigma, dtype=np.complex128)
    nt = tgt_xyz.shape[1]
    grad = np.zeros((3, int(node_off[-1])))
    for j, pt in enumerate(corr.patches):
        s_hat = pt.V @ sigma[node_off[j]:node_off[j + 1]]
        ids, adaptive, _ = corr.near[j]
        near = set(int(t) for t in ids)
        far_t = [t for t in range(nt) if t not in near]
        args = (tgt_xyz, g, k, kind, alpha, beta)
        M = _rule_grad(pt, s_hat, *rules.conical_rule(int(corr.q[j])), far_t, *args)
        leaf_m = p.leaf_order if p.leaf_order > 0 else int(corr.q[j])
        leaf_rule = rules.conical_rule(leaf_m)
        for t, ad in zip(ids, adaptive):
            if ad:
                for T in corr.pair_stats[(int(t), j)]["leaf_tris"]:
                    M += _rule_grad(pt, s_hat, *rules.map_rule(T, *leaf_rule), [int(t)], *args)
            else:
                M += _rule_grad(pt, s_hat, *rules.conical_rule(int(corr.q_near[j])), [int(t)],
                                *args)
        grad[:, node_off[j]:node_off[j + 1]] += (pt.V.T @ M).T
    return grad, corr
