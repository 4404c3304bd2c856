"""Near field of each patch (Sec. 4, definition of N_eta(Gamma_j); Sec. 5.2; Remark on eta_1).

N_eta(Gamma_j) = { targets x not on Gamma_j : |x - c_j| <= eta R_j }.
(Sec. 4 writes <=, Sec. 5.2 writes <; this project reads <=, tested as
|x - c_j|^2 <= (eta R_j)^2.)  A near target is adaptive iff |x - c_j|^2 <= (eta_1 R_j)^2
(Remark: adaptive integration only inside N_eta1, one oversampled rule in between).
"""
from __future__ import annotations

import numpy as np


def near_lists(centers, radii, eta, eta1, tgt_xyz, tgt_patch, only=None):
    """The near lists N_eta(Gamma_j) of Sec. 4 with the N_eta1 flag of the Sec. 4.3 remark.
    Per patch: (ascending target ids, adaptive flags, squared distances).  With `only`,
    the lists of the other patches are left empty (their centers and radii are unused)."""
    out = []
    keep = None if only is None else set(int(j) for j in only)
    for j in range(len(radii)):
        if keep is not None and j not in keep:
            out.append((np.zeros(0, np.int64), np.zeros(0, bool), np.zeros(0)))
            continue
        c = centers[j]
        d2 = ((tgt_xyz - c[:, None]) ** 2).sum(axis=0)
        near = (d2 <= (eta[j] * radii[j]) ** 2) & (tgt_patch != j)
        ids = np.nonzero(near)[0]
        adaptive = d2[ids] <= (eta1[j] * radii[j]) ** 2
        out.append((ids, adaptive, d2[ids]))
    return out


def far_test_targets(ids, d2):
    """Target part of the test set F(Gamma_j) (Sec. 4.2): the 10 farthest near targets if
    |N_eta| >= 20, else the floor(|N_eta|/2) farthest.  Ties: lower target id first."""
    cnt = 10 if len(ids) >= 20 else len(ids) // 2
    order = np.lexsort((ids, -d2))
    return ids[order[:cnt]], len(ids) < 20


def annulus_test_targets(ids, adaptive, d2, count=10):
    """The `count` nearest annulus targets, ties by id: test points for the order of the
    single rule the Sec. 4.3 remark uses between N_eta1 and N_eta (an order it leaves
    unstated; chosen like q_j of Sec. 4.2)."""
    sel = ~adaptive
    a_ids, a_d2 = ids[sel], d2[sel]
    order = np.lexsort((a_ids, a_d2))
    return a_ids[order[:count]]
