"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and the oracle on
the same seeded inputs, and compare per (target, patch) pair."""
import numpy as np

from oracle import corrections as C
from paper_2006_02545_gb300 import workloads as W


def run_gpu(ctx, surf, x, tn, kind, k, eps, eta=-1.0, alpha=1.0, beta=0.0, dirs_seed=3, sigma_seed=0,
            precision="fp64", tgt_normal=None, **kw):
    import torch
    from paper_2006_02545_gb300 import lcq
    dev = ctx.torch_device
    ds = lcq.DeviceSurface(surf.deg, surf.node_off, torch.from_numpy(surf.xyz).to(dev))
    prm = lcq.params(eps, eta=eta, test_dirs=W.test_directions(dirs_seed), **kw)
    near = lcq.build_near_lists(ctx, ds, torch.from_numpy(np.ascontiguousarray(x)).to(dev),
                                torch.from_numpy(tn).to(dev), prm)
    if tgt_normal is not None:
        near.set_target_normals(torch.from_numpy(np.ascontiguousarray(tgt_normal)).to(dev))
    corr = lcq.gen_corrections(ctx, ds, near, kind, k, prm, alpha, beta, precision=precision)
    st = ctx.sync(120000)
    rp, col, val = corr.export(x.shape[1])
    q, qn, leaves = corr.stats(surf.n_patches)
    sig = W.density(surf.n_points, sigma_seed)
    fn = {"S": lcq.apply_corrected_S, "D": lcq.apply_corrected_D, "CFIE": lcq.apply_corrected_CFIE,
          "Sp": lcq.apply_corrected_Sp}
    u = fn[kind](ctx, ds, near, corr, torch.from_numpy(sig).to(dev), x.shape[1]).cpu().numpy()
    st2 = ctx.sync(120000)
    pp, tgt, ad, cen, rad = near.export(surf.n_patches)
    out = dict(status=st, status_apply=st2, row_ptr=rp, col=col, val=val, q=q, q_near=qn,
               leaves=leaves, u=u, sigma=sig, pair_ptr=pp, pair_tgt=tgt, pair_ad=ad, cen=cen,
               rad=rad, near=near, corr=corr, ds=ds)
    return out


def run_oracle(surf, x, tn, kind, k, eps, eta=-1.0, alpha=1.0, beta=0.0, dirs_seed=3, sigma=None,
               only_patches=None, apply=True, tgt_normal=None, **kw):
    p = C.Params(eps=eps, eta=eta, test_dirs=W.test_directions(dirs_seed), **kw)
    oc = C.gen_corrections(surf.deg, surf.node_off, surf.xyz, x, tn, kind, k, alpha, beta, params=p,
                           only_patches=only_patches, tgt_normal=tgt_normal)
    u = (C.apply_corrected(oc, surf.node_off, sigma, x, kind, k, alpha, beta, tgt_node=tn,
                           tgt_normal=tgt_normal) if apply else None)
    return oc, u


def pair_entries(row_ptr, col, val, node_off, t, j):
    a, b = row_ptr[t], row_ptr[t + 1]
    c = col[a:b]
    lo = np.searchsorted(c, node_off[j])
    hi = np.searchsorted(c, node_off[j + 1])
    return val[a + lo:a + hi]


def pair_tolerance(oc, t, j, c_pair_norm, c_max):
    """Allowed ||c_gpu - c_oracle||_2 for the pair (t, j), derived from the arithmetic:
    1e-10 relative to the pair, 1e-12 of the largest pair, plus what refinement decisions
    that rounding can flip may move: tests decided by the rounding floor or within 1e-3
    of the threshold change the accepted moments by at most twice their tolerance each,
    and V^T scales moments by at most ||V||_2."""
    st = oc.pair_stats[(t, j)]
    slack = 0.0
    if st.get("kind") == "adaptive":
        slack = 2.0 * (st["floor_sum"] + st["close_sum"])
    return 1e-10 * c_pair_norm + 1e-12 * c_max + oc.patches[j].normV * slack


def compare_pairs(g, oc, node_off, pairs=None):
    """Check every oracle pair against its tolerance; returns (worst ratio, npairs)."""
    keys = list(oc.pair_stats.keys() if pairs is None else pairs)
    vals = {}
    c_max = 0.0
    for (t, j) in keys:
        vo = pair_entries(oc.row_ptr, oc.col, oc.val, node_off, t, j)
        vg = pair_entries(g["row_ptr"], g["col"], g["val"], node_off, t, j)
        assert len(vo) == len(vg) == node_off[j + 1] - node_off[j], (t, j)
        vals[(t, j)] = (vo, vg)
        c_max = max(c_max, np.linalg.norm(vo))
    worst, where = 0.0, None
    used_slack = 0      # pairs within tolerance only thanks to the decision slack
    for (t, j), (vo, vg) in vals.items():
        nv = np.linalg.norm(vo)
        tol = pair_tolerance(oc, t, j, nv, c_max)
        err = np.linalg.norm(vo - vg)
        if err > 1e-10 * nv + 1e-12 * c_max:
            used_slack += 1
        r = err / tol
        if r > worst:
            worst, where = r, (t, j)
    compare_pairs.used_slack = used_slack
    return worst, len(keys), where


def leaves_by_pair(g, oc):
    """(gpu leaves, oracle leaves, oracle margin) for every adaptive pair of the oracle."""
    out = []
    pp, tg = g["pair_ptr"], g["pair_tgt"]
    for (t, j), st in oc.pair_stats.items():
        if st.get("kind") != "adaptive":
            continue
        seg = tg[pp[j]:pp[j + 1]]
        idx = pp[j] + np.searchsorted(seg, t)
        out.append((int(g["leaves"][idx]), st["leaves"], st["margin"]))
    return out
