"""Adjoint on the GPU through the C ABI: A^H g and the frozen-rule shape gradient against
the oracle's (oracle/adjoint.py, pinned by finite differences), the adjoint identity with
the jump term, and the autograd wrapper against central finite differences of the GPU
forward on the 2000-patch ellipsoid gradient workload."""
import numpy as np
import pytest

from oracle import adjoint as OA
from oracle import corrections as C
from paper_2006_02545_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    from paper_2006_02545_gb300 import lcq
    c = lcq.Context(0)
    yield c
    c.close()


def _gpu(ctx, s, x, tn, kind, k, eps, a, b):
    import torch
    from paper_2006_02545_gb300 import lcq
    dev = ctx.torch_device
    ds = lcq.DeviceSurface(s.deg, s.node_off, torch.from_numpy(s.xyz).to(dev))
    prm = lcq.params(eps, test_dirs=W.test_directions(3))
    near = lcq.build_near_lists(ctx, ds, torch.from_numpy(x).to(dev), torch.from_numpy(tn).to(dev),
                                prm)
    corr = lcq.gen_corrections(ctx, ds, near, kind, k, prm, a, b)
    assert ctx.sync(60000) == 0
    return ds, near, corr


def test_apply_adjoint_matches_oracle(ctx):
    import torch
    from paper_2006_02545_gb300 import lcq
    s = W.ellipsoid(1, 3)
    xs, tns = W.onsurface_targets(s)
    xo = W.radial_targets(s, 40, 2, 0.02, 0.5, True)
    x = np.ascontiguousarray(np.concatenate([xs, xo], axis=1))
    tn = np.concatenate([tns, -np.ones(xo.shape[1], np.int64)])
    kind, k, a, b = "CFIE", 2.0 + 0.1j, 1.0, -2j
    ds, near, corr = _gpu(ctx, s, x, tn, kind, k, 1e-7, a, b)
    rng = np.random.default_rng(4)
    g = rng.standard_normal(x.shape[1]) + 1j * rng.standard_normal(x.shape[1])
    gd = torch.from_numpy(g).to(ctx.torch_device)
    ah = lcq.apply_adjoint(ctx, ds, near, corr, gd).cpu().numpy()
    assert ctx.sync(60000) == 0
    p = C.Params(eps=1e-7, test_dirs=W.test_directions(3))
    oc = C.gen_corrections(s.deg, s.node_off, s.xyz, x, tn, kind, k, a, b, params=p)
    ref = OA.apply_adjoint(oc, s.node_off, g, x, kind, k, a, b)
    rel = np.linalg.norm(ah - ref) / np.linalg.norm(ref)
    assert rel <= 1e-10, rel
    # the adjoint identity holds with the jump term too (D, exterior limit 1/2)
    ds, near, corr = _gpu(ctx, s, x, tn, "D", k, 1e-7, 1.0, 0.0)
    sig = W.density(s.n_points, 1)
    u = lcq.apply_corrected_D(ctx, ds, near, corr, torch.from_numpy(sig).to(ctx.torch_device),
                              x.shape[1], jump=0.5).cpu().numpy()
    ah = lcq.apply_adjoint(ctx, ds, near, corr, gd, jump=0.5).cpu().numpy()
    lhs, rhs = np.vdot(g, u), np.vdot(ah, sig)
    assert abs(lhs - rhs) <= 1e-12 * np.abs(g).sum() * np.abs(u).max() * 10


@pytest.mark.parametrize("kind,k", [("S", 1.3), ("CFIE", 2.2 + 0.3j)])
def test_shape_gradient_matches_oracle(ctx, kind, k):
    import torch
    from paper_2006_02545_gb300 import lcq
    s = W.ellipsoid(1, 3, axes=(1.0, 1.2, 0.9))
    x = W.radial_targets(s, 30, 4, 0.02, 0.6, True)
    tn = -np.ones(x.shape[1], np.int64)
    a, b = 1.0, -1j * k
    ds, near, corr = _gpu(ctx, s, x, tn, kind, k, 1e-8, a, b)
    assert near.n_adaptive > 0
    rng = np.random.default_rng(6)
    sig = W.density(s.n_points, 2)
    g = rng.standard_normal(x.shape[1]) + 1j * rng.standard_normal(x.shape[1])
    dev = ctx.torch_device
    gy = lcq.shape_gradient(ctx, ds, near, corr, torch.from_numpy(sig).to(dev),
                            torch.from_numpy(g).to(dev)).cpu().numpy()
    assert ctx.sync(60000) == 0
    p = C.Params(eps=1e-8, test_dirs=W.test_directions(3))
    ref, _ = OA.shape_gradient(s.deg, s.node_off, s.xyz, x, tn, kind, k, a, b, p, sig, g)
    err = np.abs(gy - ref).max() / np.abs(ref).max()
    assert err <= 1e-9, err


def test_autograd_matches_finite_differences():
    """Gradient of sum |S_k sigma|^2 (k = 5, eps = 1e-8) at 1000 exterior targets of the
    ellipsoid (1, 1.5, 2.5) with 2000 degree-5 patches, w.r.t. the density and all node
    coordinates; 50 coordinates (step 1e-6) and 10 density entries against central
    differences of the GPU forward.  The loss is a quadratic form in sigma, so the central
    difference in a density entry has no truncation error at any step; its rounding noise,
    about u L / h = 2e-11 at h = 1e-6 against density gradients of 1e-5, would alone be
    1e-6 relative, so the density step is 1e-2 (noise 1e-10)."""
    import torch
    import __graft_entry__ as gr
    gr.build()
    from paper_2006_02545_gb300 import lcq
    from paper_2006_02545_gb300.autograd import corrected_potential
    dev = torch.device("cuda", 0)
    ctx = lcq.Context(0)
    s, x = W.ellipsoid_adjoint_s_k5(10)
    assert s.n_patches == 2000 and x.shape[1] == 1000
    tx = torch.from_numpy(x).to(dev)
    tn = torch.full((x.shape[1],), -1, dtype=torch.int64, device=dev)
    prm = lcq.params(1e-8, test_dirs=W.test_directions(3))
    k = 5.0
    xyz0 = torch.from_numpy(s.xyz).to(dev)
    sig0 = torch.from_numpy(W.density(s.n_points, 0)).to(dev)

    def L(xyz, sig):
        u = corrected_potential(ctx, s.deg, s.node_off, xyz, sig, tx, tn, "S", k, prm)
        return (u.abs() ** 2).sum()

    xyz = xyz0.clone().requires_grad_(True)
    sig = sig0.clone().requires_grad_(True)
    loss = L(xyz, sig)
    loss.backward()
    assert ctx.sync(120000) == 0
    gy = xyz.grad.cpu().numpy()
    gs = sig.grad.cpu().numpy()
    rng = np.random.default_rng(0)
    h = 1e-6
    worst = 0.0
    with torch.no_grad():
        for idx in rng.choice(3 * s.n_points, 50, replace=False):
            c, i = divmod(int(idx), s.n_points)
            xp, xm = xyz0.clone(), xyz0.clone()
            xp[c, i] += h
            xm[c, i] -= h
            fd = (L(xp, sig0).item() - L(xm, sig0).item()) / (2 * h)
            worst = max(worst, abs(fd - gy[c, i]) / max(abs(gy[c, i]), 1e-3 * np.abs(gy).max()))
        for i in rng.choice(s.n_points, 10, replace=False):
            for dz in (1.0, 1j):     # dL = Re(conj(grad) dsigma) for complex sigma
                hs = 1e-2
                sp, sm = sig0.clone(), sig0.clone()
                sp[i] += hs * dz
                sm[i] -= hs * dz
                fd = (L(xyz0, sp).item() - L(xyz0, sm).item()) / (2 * hs)
                an = float(np.real(np.conj(gs[i]) * dz))
                worst = max(worst, abs(fd - an) / max(abs(an), 1e-3 * np.abs(gs).max()))
    assert worst <= 1e-6, worst
    ctx.close()


def test_adjoint_of_a_batch_matches_oracle_per_surface(ctx):
    """A^H g and the shape gradient of a two-surface batch (different k, CFIE coefficients
    and eps, overlapping in space) equal the oracle's for each surface alone: nothing of
    either gradient crosses surfaces."""
    import torch
    from paper_2006_02545_gb300 import lcq
    dev = ctx.torch_device
    parts = [W.ellipsoid(1, 3, axes=(1.0, 1.2, 0.9)), W.ellipsoid(1, 2, axes=(0.8, 0.7, 1.1))]
    phys = [(2.0, 1.0, -2j, 1e-7), (3.5 + 0.2j, 0.5, -3.5j, 1e-6)]
    s, poff = W.concat_surfaces(parts)
    xs = [W.radial_targets(p, 20, 5 + i, 0.02, 0.6, True) for i, p in enumerate(parts)]
    x = np.ascontiguousarray(np.concatenate(xs, axis=1))
    tn = -np.ones(x.shape[1], np.int64)
    tsurf = np.concatenate([np.full(xi.shape[1], i, np.int32) for i, xi in enumerate(xs)])
    ds = lcq.DeviceSurface(s.deg, s.node_off, torch.from_numpy(s.xyz).to(dev))
    prm = lcq.params(1e-6, test_dirs=W.test_directions(3))
    near = lcq.build_near_lists_batched(ctx, ds, poff, torch.from_numpy(x).to(dev),
                                        torch.from_numpy(tn).to(dev), prm,
                                        torch.from_numpy(tsurf).to(dev))
    corr = lcq.gen_corrections_batched(ctx, ds, near, "CFIE", phys, prm)
    rng = np.random.default_rng(9)
    g = rng.standard_normal(x.shape[1]) + 1j * rng.standard_normal(x.shape[1])
    sig = W.density(s.n_points, 4)
    gd, sd = torch.from_numpy(g).to(dev), torch.from_numpy(sig).to(dev)
    ah = lcq.apply_adjoint(ctx, ds, near, corr, gd).cpu().numpy()
    gy = lcq.shape_gradient(ctx, ds, near, corr, sd, gd).cpu().numpy()
    assert ctx.sync(60000) == 0
    t0 = 0
    for i, (p, (k, a, b, eps)) in enumerate(zip(parts, phys)):
        n0, n1 = s.node_off[poff[i]], s.node_off[poff[i + 1]]
        t1 = t0 + xs[i].shape[1]
        xi, ti, gi = xs[i], tn[t0:t1], g[t0:t1]
        pp = C.Params(eps=eps, test_dirs=W.test_directions(3))
        oc = C.gen_corrections(p.deg, p.node_off, p.xyz, xi, ti, "CFIE", k, a, b, params=pp)
        ref = OA.apply_adjoint(oc, p.node_off, gi, xi, "CFIE", k, a, b)
        assert np.linalg.norm(ah[n0:n1] - ref) <= 1e-10 * np.linalg.norm(ref), i
        rg, _ = OA.shape_gradient(p.deg, p.node_off, p.xyz, xi, ti, "CFIE", k, a, b, pp,
                                  sig[n0:n1], gi)
        assert np.abs(gy[:, n0:n1] - rg).max() <= 1e-9 * np.abs(rg).max(), i
        t0 = t1
