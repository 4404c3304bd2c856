"""Precomputation of all near and self corrections and the corrected layer potential
(Sec. 5.2 Precomputation, Sec. 5.3 subtract-and-add, Sec. 4.4 Eq. for I(x)).

Order of steps (Sec. 5.2): geometry -> near lists -> far order q_j (Eq. qj) and the
annulus rule order -> self weights S_j -> near weights N_j (adaptive inside
eta_1 R_j, one oversampled rule in the annulus) -> net corrections.

Net correction (subtract-and-add, Sec. 5.3, folded into the stored entry):
    c_{t,l} = a^j_l(x_t) - s^j_l(x_t)   for near pairs,
    c_{t,l} = a^j_l(x_t)                for the target's own patch (self pair),
where a is the self or near point weight and s the weight the smooth rule q_j puts
on node l for the same target.  Apply then computes
    u(x_t) = sum_{j != own(t)} sum_{q in rule q_j} K(x_t, X_q) J_q w_q sigma~_q
             + sum_row c_{t,col} sigma_col,
i.e. the own patch of an on-surface target is masked out of the far sum instead of
being subtracted (the masked variant of Sec. 5.3; equal in exact arithmetic).  A
smooth-rule node can fall very close to a node of the same patch, and subtracting
its large spurious contribution loses digits; masking avoids that cancellation.
Rows are targets; within a row, patches ascend, and each patch contributes its n
nodes in node order.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import geometry, nearlist, quadrature, rules
from .quadrature import Kern


@dataclass
class Params:
    """Parameters of the generation (Sec. 4.1-4.3): tolerance, near-field cutoffs eta and
    eta_1, the termination loosening, depth cap, rule orders and test directions."""
    eps: float
    eta: float = -1.0            # <= 0: default by degree (Sec. 4.1)
    eta1: float = 1.25           # Remark on eta_1
    eps_loosen: float = 1.0      # termination loosening of Sec. 4.3 Remark (unstated there)
    max_depth: int = 24
    m_max: int = 24              # largest smooth rule of the family
    self_order: int = 0          # 0: rules.default_self_order(eps)
    leaf_order: int = 0          # 0: the patch's far order q_j
    test_dirs: np.ndarray | None = None
    record_leaves: bool = False  # keep each adaptive pair's leaf triangles (adjoint)


def fibonacci_dirs(n: int = 15) -> np.ndarray:
    """Default test directions for the points on the sphere of radius eta R_j that the far
    test set of Sec. 4.2 adds when a near list is short (the paper draws 15 at random; a
    fixed set lets both implementations see the same points): z_k = 1 - (2k+1)/n, azimuth
    k pi (3 - sqrt 5)."""
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    r = np.sqrt(1.0 - z * z)
    phi = k * np.pi * (3.0 - np.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


@dataclass
class Corrections:
    """The corrections of Sec. 5.3 as a CSR by target (row_ptr, col, val), with the far and
    annulus orders of Sec. 4.2-4.3, the cutoffs and near lists used and per-pair records."""
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    q: np.ndarray                 # far order per patch
    q_near: np.ndarray            # annulus order per patch (0: no annulus targets)
    q_saturated: np.ndarray
    eta: np.ndarray
    eta1: np.ndarray
    near: list
    patches: list
    pair_stats: dict = field(default_factory=dict)   # (t, j) -> dict
    depth_hit: bool = False
    tgt_patch: np.ndarray = None                       # own patch of each target (-1: off surface)


class LazyPatches:
    """Patches (Sec. 3.2, Sec. 4 geometry) built on first use, for runs restricted to a few
    patches of a large surface."""

    def __init__(self, deg, node_off, xyz):
        self.deg, self.node_off, self.xyz = deg, node_off, xyz
        self.memo = {}

    def __len__(self):
        return len(self.deg)

    def __getitem__(self, j):
        if j not in self.memo:
            a, b = self.node_off[j], self.node_off[j + 1]
            self.memo[j] = geometry.make_patch(int(self.deg[j]), self.xyz[:, a:b])
        return self.memo[j]


def patch_of_node(node_off, tgt_node):
    """Own patch of each target (-1 off the surface): the patch whose nodes hold the
    target's node id, which makes the pair a self pair (Sec. 4, Sec. 5.2)."""
    tp = np.full(tgt_node.shape, -1, dtype=np.int64)
    on = tgt_node >= 0
    tp[on] = np.searchsorted(node_off, tgt_node[on], side="right") - 1
    return tp


def target_normals(patches, node_off, tgt_node, tgt_normal):
    """Unit target normals n(x) for S' (Sec. 3): the chart normal at the node for an on-surface target
    (so that n_x.(x - y) vanishes to second order on its own patch), the caller's
    tgt_normal [3, NT] (normalized) for an off-surface target."""
    tgt_node = np.asarray(tgt_node)
    tp = patch_of_node(node_off, tgt_node)
    out = np.zeros((3, len(tgt_node)))
    for t in range(len(tgt_node)):
        if tp[t] >= 0:
            out[:, t] = quadrature.node_normal(patches[tp[t]], int(tgt_node[t] - node_off[tp[t]]))
        else:
            if tgt_normal is None:
                raise ValueError("S' needs the normals of off-surface targets")
            v = np.asarray(tgt_normal[:, t], dtype=np.float64)
            out[:, t] = v / np.linalg.norm(v)
    return out


def gen_corrections(deg, node_off, xyz, tgt_xyz, tgt_node, kind, k, alpha=1.0, beta=0.0,
                    params: Params = None, patches=None, only_patches=None, tgt_normal=None):
    """All corrections for the targets, in the order of Sec. 4.2-4.3 and 5.2: geometry,
    near lists, far order q_j (Eq. qj), then per near pair the adaptive or annulus moments
    and per self pair the self weights, each contracted with V and stored net of the smooth
    rule's weights.  `only_patches` restricts the work to some patches (rows then hold only
    those patches' entries).  kind "Sp" (S') uses target normals (target_normals)."""
    p = params
    kern = Kern(kind, k, alpha, beta)
    deg = np.asarray(deg)
    node_off = np.asarray(node_off)
    tgt_node = np.asarray(tgt_node)
    if patches is None:
        patches = (geometry.make_patches(deg, node_off, xyz) if only_patches is None
                   else LazyPatches(deg, node_off, xyz))
    npat = len(patches)
    tgt_patch = patch_of_node(node_off, tgt_node)
    eta = np.array([p.eta if p.eta > 0 else geometry.default_eta(int(d)) for d in deg])
    eta1 = np.minimum(p.eta1, eta)
    listed = range(npat) if only_patches is None else only_patches
    centers = np.zeros((npat, 3))
    radii = np.zeros(npat)
    for j in listed:
        centers[j], radii[j] = patches[j].c, patches[j].R
    near = nearlist.near_lists(centers, radii, eta, eta1, tgt_xyz, tgt_patch, only_patches)
    nrm = target_normals(patches, node_off, tgt_node, tgt_normal) if kind == "Sp" else None
    dirs = fibonacci_dirs() if p.test_dirs is None else np.asarray(p.test_dirs)
    self_order = p.self_order if p.self_order > 0 else rules.default_self_order(p.eps)

    work = range(npat) if only_patches is None else only_patches
    q = np.zeros(npat, dtype=np.int64)
    q_near = np.zeros(npat, dtype=np.int64)
    q_sat = np.zeros(npat, dtype=bool)
    entries = {}          # (t, j) -> values [n]
    stats = {}
    depth_hit = False
    for j in work:
        pt = patches[j]
        ids, adaptive, d2 = near[j]
        m_min = (pt.d + 2) // 2
        # far order q_j (Sec. 4.2, Eq. qj)
        far_t, add_sphere = nearlist.far_test_targets(ids, d2)
        F = [tgt_xyz[:, t] for t in far_t]
        if add_sphere:
            F += [pt.c + eta[j] * pt.R * dvec for dvec in dirs]
        q[j], q_sat[j], _ = quadrature.far_order(pt, F, kern, p.eps, m_min, p.m_max)
        # annulus rule order (reading): 15 points on the eta_1 sphere + 10 nearest annulus targets
        if (~adaptive).any():
            F1 = [pt.c + eta1[j] * pt.R * dvec for dvec in dirs]
            F1 += [tgt_xyz[:, t] for t in nearlist.annulus_test_targets(ids, adaptive, d2)]
            q_near[j], sat, _ = quadrature.far_order(pt, F1, kern, p.eps, m_min, p.m_max)
            q_sat[j] |= sat
        # near weights
        leaf_m = p.leaf_order if p.leaf_order > 0 else int(q[j])
        cache = quadrature.LeafCache(pt, leaf_m)
        tol0 = p.eps * p.eps_loosen * pt.dj / pt.normV
        an_rule = rules.conical_rule(int(q_near[j])) if q_near[j] > 0 else None
        for t, ad in zip(ids, adaptive):
            x = tgt_xyz[:, t]
            nx = nrm[:, t] if nrm is not None else None
            if ad:
                rec = [] if p.record_leaves else None
                I, st = quadrature.adaptive_moments(cache, x, kern, tol0, p.max_depth, rec, nx)
                depth_hit |= st["depth_hit"]
                st["kind"] = "adaptive"
                if rec is not None:
                    st["leaf_tris"] = rec
            else:
                I = quadrature.rule_moments(pt, x, *an_rule, kern, nx)
                st = {"kind": "annulus"}
            a = pt.V.T @ I
            s = quadrature.smooth_weights(pt, x, int(q[j]), kern, nx)
            entries[(int(t), j)] = a - s
            stats[(int(t), j)] = st
        # self weights (the own patch is masked out of the far sum, nothing to subtract)
        for t in np.nonzero(tgt_patch == j)[0]:
            i = int(tgt_node[t] - node_off[j])
            x = tgt_xyz[:, t]
            entries[(int(t), j)] = quadrature.self_weights(pt, i, x, kern, self_order)
            stats[(int(t), j)] = {"kind": "self"}

    nt = tgt_xyz.shape[1]
    keys = sorted(entries.keys())
    counts = np.zeros(nt + 1, dtype=np.int64)
    for (t, j) in keys:
        counts[t + 1] += patches[j].n
    row_ptr = np.cumsum(counts)
    col = np.empty(int(row_ptr[-1]), dtype=np.int64)
    val = np.empty(int(row_ptr[-1]), dtype=np.complex128)
    pos = 0
    for (t, j) in keys:
        n = patches[j].n
        col[pos:pos + n] = node_off[j] + np.arange(n)
        val[pos:pos + n] = entries[(t, j)]
        pos += n
    return Corrections(row_ptr, col, val, q, q_near, q_sat, eta, eta1, near, patches, stats,
                       depth_hit, tgt_patch)


def far_sources(patches, q, sigma, node_off):
    """Oversampled sources of the smooth rules q_j: positions, normals, w_q sigma~_q (Sec. 4.2
    Remark: sigma~_q = sum_nm s_nm K_nm(u_q, v_q), s = V sigma), and their patch ids."""
    Xs, Ns, str_, pid = [], [], [], []
    for j, pt in enumerate(patches):
        ru, rv, rw = rules.conical_rule(int(q[j]))
        X, N, K = pt.eval(ru, rv)
        s = pt.V @ sigma[node_off[j]:node_off[j + 1]]
        Xs.append(X)
        Ns.append(N)
        str_.append(rw * (K.T @ s))
        pid.append(np.full(len(rw), j))
    return (np.concatenate(Xs, axis=1), np.concatenate(Ns, axis=1), np.concatenate(str_),
            np.concatenate(pid))


def apply_corrected(corr: Corrections, node_off, sigma, tgt_xyz, kind, k, alpha=1.0, beta=0.0,
                    tgt_node=None, tgt_normal=None):
    """u(x_t) = far sum over the oversampled sources of every patch but the target's own
    + CSR correction (Sec. 5.3).  S' (kind "Sp") needs tgt_node (and tgt_normal for
    off-surface targets) for the target normals."""
    kern = Kern(kind, k, alpha, beta)
    X, N, strength, pid = far_sources(corr.patches, corr.q, sigma, node_off)
    nt = tgt_xyz.shape[1]
    nrm = (target_normals(corr.patches, node_off, tgt_node, tgt_normal) if kind == "Sp"
           else np.zeros((3, nt)))
    u = np.zeros(nt, dtype=np.complex128)
    for t in range(nt):
        keep = pid != corr.tgt_patch[t]
        u[t] = (kern(tgt_xyz[:, t], X[:, keep], N[:, keep], nrm[:, t]) * strength[keep]).sum()
        a, b = corr.row_ptr[t], corr.row_ptr[t + 1]
        u[t] += (corr.val[a:b] * sigma[corr.col[a:b]]).sum()
    return u
