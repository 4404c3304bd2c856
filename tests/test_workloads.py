"""The seeded input generators against the recipes they state (CPU): the 64-torus draw and
its lattice, the benchmark ellipsoid, the large torus, the gradient workload's exterior
targets and the density and test-direction draws."""
import math

import numpy as np

from paper_2006_02545_gb300 import workloads as W


def test_batched_tori_draws():
    a = W.batched_tori(64, 0)
    assert a == W.batched_tori(64, 0) and a != W.batched_tori(64, 1) and len(a) == 64
    for sp in a:
        assert 200 <= sp["n_patches"] <= 5000
        assert 3 <= sp["deg"] <= 8
        assert 1.0 <= sp["k"] <= 20.0
        assert sp["eps"] in (1e-6, 1e-9)
        assert sp["dtype"] in ("complex64", "complex128")
    # every value the recipe allows occurs among 64 draws
    assert {sp["deg"] for sp in a} == set(range(3, 9))
    assert {sp["eps"] for sp in a} == {1e-6, 1e-9}
    assert {sp["dtype"] for sp in a} == {"complex64", "complex128"}


def test_torus_patch_count_nearest_on_its_grid():
    # n_phi = 2 n_theta cells of two triangles: 4 n_theta^2 patches, the nearest to the ask
    for want in (200, 777, 1000, 5000):
        got = W.torus_with_patches(want, 3).n_patches
        nt = math.isqrt(got // 4)
        assert got == 4 * nt * nt
        assert all(abs(got - want) <= abs(4 * m * m - want) for m in (nt - 1, nt + 1))


def test_batched_tori_lattice_keeps_surfaces_apart():
    surf, poff, phys, dtypes = W.batched_tori_batch(16, 0, scale=0.05)
    assert len(poff) == 17 and poff[0] == 0 and poff[-1] == surf.n_patches
    assert len(phys) == 16 and len(dtypes) == 16
    boxes = []
    for i in range(16):
        n0, n1 = surf.node_off[poff[i]], surf.node_off[poff[i + 1]]
        x = surf.xyz[:, n0:n1]
        boxes.append((x.min(axis=1), x.max(axis=1)))
    for i in range(16):
        for j in range(i + 1, 16):
            (lo_i, hi_i), (lo_j, hi_j) = boxes[i], boxes[j]
            assert not (np.all(lo_i <= hi_j) and np.all(lo_j <= hi_i)), (i, j)
    for k, alpha, beta, _ in phys:   # CFIE alpha = 1, beta = -ik
        assert alpha == 1.0 and beta == -1j * k


def test_benchmark_ellipsoid():
    wl = W.ellipsoid_cfie_k2pi(8)
    s = wl.surface
    assert s.n_patches == 1280 and s.n_points == 35840 and set(s.deg.tolist()) == {6}
    assert wl.tgt_xyz.shape == (3, 35840) and np.array_equal(wl.tgt_node, np.arange(35840))
    assert wl.kernel == "CFIE" and wl.k == 2 * math.pi and wl.eps == 1e-9
    assert wl.alpha == 1.0 and wl.beta == -1j * wl.k
    assert wl.eta == -1.0   # the paper's cutoff by order: 2 at p = 7
    # nodes on the ellipsoid (1, 2, 3)
    q = (s.xyz[0] / 1.0) ** 2 + (s.xyz[1] / 2.0) ** 2 + (s.xyz[2] / 3.0) ** 2
    assert np.abs(q - 1.0).max() < 1e-12


def test_large_torus_recipe():
    wl = W.torus_cfie_k20(5)   # 4 n_theta^2 degree-6 patches; the benchmark uses n_theta = 100
    assert wl.surface.n_patches == 100 and wl.surface.n_points == 2800
    assert wl.kernel == "CFIE" and wl.k == 20.0 and wl.eps == 1e-9 and wl.beta == -20j


def test_gradient_workload_targets_are_exterior():
    s, x = W.ellipsoid_adjoint_s_k5(10)
    assert s.n_patches == 2000 and set(s.deg.tolist()) == {5} and x.shape == (3, 1000)
    q = (x[0] / 1.0) ** 2 + (x[1] / 1.5) ** 2 + (x[2] / 2.5) ** 2
    assert q.min() > 1.0


def test_density_and_directions():
    d = W.density(10000, 3)
    assert np.array_equal(d, W.density(10000, 3)) and d.dtype == np.complex128
    assert abs(d.real.mean()) < 0.05 and abs(d.real.std() - 1.0) < 0.05
    assert abs(d.imag.std() - 1.0) < 0.05
    t = W.test_directions(7)
    assert t.shape == (15, 3) and np.allclose(np.linalg.norm(t, axis=1), 1.0, atol=1e-15)
