"""The allocation-free entry point lcq_adaptive_corrections_noalloc, for callers that cannot
allocate device memory (no cudaMalloc in their context): called twice in a row through the
C ABI, it must reproduce the adaptive near corrections lcq_gen_corrections stores for the
same patch and targets.  Kept in its own file, collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the FP64 parity bar of the other GPU tests


def test_noalloc_matches_gen_corrections():
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2006_02545_gb300 import lcq
    from paper_2006_02545_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    s = W.ellipsoid(8, 6, axes=(1.0, 2.0, 3.0))
    j = 517
    y = np.ascontiguousarray(s.xyz[:, s.node_off[j]:s.node_off[j + 1]])
    one = W.Surface("one_patch", s.deg[j:j + 1], np.array([0, 28], np.int64), y)
    c = y.mean(axis=1, keepdims=True)
    # candidate targets: nodes pulled toward the middle and pushed off the surface
    cand = []
    for i in range(28):
        for f, h in ((0.9, 0.004), (0.7, -0.01), (1.0, 0.02)):
            p = c + f * (y[:, i:i + 1] - c)
            cand.append(p[:, 0] * (1.0 + h / np.linalg.norm(p)))
    cand = np.ascontiguousarray(np.array(cand).T)

    ctx = lcq.Context(0)
    ds = lcq.DeviceSurface(one.deg, one.node_off, torch.from_numpy(y).to(dev))
    k = 2.0 * np.pi
    prm = lcq.params(1e-9, test_dirs=W.test_directions(7))

    def existing(x):
        tn = torch.full((x.shape[1],), -1, dtype=torch.int64, device=dev)
        near = lcq.build_near_lists(ctx, ds, torch.from_numpy(x).to(dev), tn, prm)
        corr = lcq.gen_corrections(ctx, ds, near, "CFIE", k, prm, 1.0, -1j * k)
        assert ctx.sync(60000) == 0
        rp, col, val = corr.export(x.shape[1])
        q, _, _ = corr.stats(1)
        pp, tg, ad, cen, rad = near.export(1)
        return rp, val, int(q[0]), tg, ad

    # keep the candidates inside eta_1 R of the patch: every pair adaptive
    _, _, _, tg, ad = existing(cand)
    x = np.ascontiguousarray(cand[:, tg[ad]])
    assert 20 <= x.shape[1] <= 128
    rp, val, q, tg, ad = existing(x)
    nt = x.shape[1]
    assert ad.all() and len(tg) == nt and np.array_equal(np.diff(rp), np.full(nt, 28))
    ref = val.reshape(nt, 28)

    y_d = torch.from_numpy(y).to(dev)
    x_d = torch.from_numpy(x).to(dev)
    for _ in range(2):
        out = torch.full((nt, 28), complex("nan"), dtype=torch.complex128, device=dev)
        st = lcq.adaptive_corrections_noalloc(6, y_d, x_d, "CFIE", k, q, 1e-9, out, 1.0, -1j * k,
                                              max_depth=16)
        assert st == 0
        got = out.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= TOL, err

    # sizes beyond the stated maximum are refused before any work
    big = torch.zeros((3, 129), dtype=torch.float64, device=dev)
    out = torch.zeros((129, 28), dtype=torch.complex128, device=dev)
    assert lcq.adaptive_corrections_noalloc(6, y_d, big, "CFIE", k, q, 1e-9, out) == 5
    ctx.close()
