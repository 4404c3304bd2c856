"""Pins of the oracle's whole pipeline (near lists, far order, self, adaptive and annulus
weights, CSR assembly, subtract-and-add apply) against identities fixed by potential
theory."""
import numpy as np
import pytest

from oracle import corrections as C
from oracle import nearlist, truth
from paper_2006_02545_gb300 import workloads


@pytest.fixture(scope="module")
def flat_icosa_D0():
    s = workloads.ellipsoid(1, 3, flat=True)
    x_on, t_on = workloads.onsurface_targets(s)
    inner = workloads.radial_targets(s, 6, 5, 0.02, 0.3, outside=False)
    outer = workloads.radial_targets(s, 6, 6, 0.02, 0.3, outside=True)
    x = np.concatenate([x_on, inner, outer], axis=1)
    tn = np.concatenate([t_on, -np.ones(12, np.int64)])
    p = C.Params(eps=1e-7, test_dirs=workloads.test_directions(2))
    corr = C.gen_corrections(s.deg, s.node_off, s.xyz, x, tn, "D", 0.0, params=p)
    u = C.apply_corrected(corr, s.node_off, np.ones(s.n_points, complex), x, "D", 0.0)
    return s, corr, u


def test_gauss_identity_flat_polyhedron(flat_icosa_D0):
    """D_0[1] = -1/2 on the surface, -1 inside, 0 outside, for a closed flat polyhedron
    (charts match along edges, so the identity is exact up to quadrature error)."""
    s, corr, u = flat_icosa_D0
    n = s.n_points
    assert np.abs(u[:n] + 0.5).max() < 2e-7
    assert np.abs(u[n:n + 6] + 1.0).max() < 2e-7
    assert np.abs(u[n + 6:]).max() < 2e-7
    assert not corr.depth_hit


def test_csr_structure(flat_icosa_D0):
    s, corr, _ = flat_icosa_D0
    nt = len(corr.row_ptr) - 1
    for t in range(nt):
        cols = corr.col[corr.row_ptr[t]:corr.row_ptr[t + 1]]
        patches = np.searchsorted(s.node_off, cols, side="right") - 1
        # patches ascend, each contributes its n nodes in order
        assert (np.diff(patches) >= 0).all()
        for j in np.unique(patches):
            cj = cols[patches == j]
            assert (cj == s.node_off[j] + np.arange(len(cj))).all() and len(cj) == s.node_off[j + 1] - s.node_off[j]


def test_near_list_definition_tiny():
    """Hand-placed targets around one patch: the <= boundary, self exclusion, eta_1 flag."""
    c = np.array([[0.0, 0.0, 0.0]])
    R = np.array([1.0])
    tx = np.array([[0.5, 0, 0], [2.0, 0, 0], [2.0000001, 0, 0], [1.2, 0, 0], [0.1, 0, 0]]).T
    tp = np.array([-1, -1, -1, -1, 0])
    ids, ad, _ = nearlist.near_lists(c, R, np.array([2.0]), np.array([1.25]), tx, tp)[0]
    assert list(ids) == [0, 1, 3] and list(ad) == [True, False, True]


@pytest.mark.parametrize("kind", ["S", "D"])
def test_sphere_eigenvalues_converge(kind):
    """S_k Y_n = i k j_n(k) h_n(k) Y_n and D_k Y_n = (i k^2 j_n(k) h_n'(k) + 1/2) Y_n (principal
    value, outward normal) on the unit sphere for n = 0, 1, 2, through the full pipeline with
    the densities Y_0 = 1, Y_1 = z and Y_2 = (3 z^2 - 1)/2 sampled at the nodes; the error
    falls with the patch size as the chart approximation improves (the eigenvalue formulas
    themselves are pinned against the surface integrals in test_oracle_pins.py)."""
    k = 1.0
    lam = {n: (truth.sphere_eigen_S if kind == "S" else truth.sphere_eigen_D)(n, k)
           for n in range(3)}
    errs = {n: [] for n in range(3)}
    for sdiv, d in ((1, 2), (1, 4), (1, 6)):
        s = workloads.ellipsoid(sdiv, d)
        x, tn = workloads.onsurface_targets(s)
        z = s.xyz[2] / np.linalg.norm(s.xyz, axis=0)
        p = C.Params(eps=1e-7, eta=1.25, test_dirs=workloads.test_directions(4))
        corr = C.gen_corrections(s.deg, s.node_off, s.xyz, x, tn, kind, k, params=p)
        for n, Y in enumerate((np.ones_like(z), z, 0.5 * (3 * z * z - 1))):
            u = C.apply_corrected(corr, s.node_off, Y.astype(complex), x, kind, k)
            errs[n].append(np.abs(u - lam[n] * Y).max() / abs(lam[n]))
    for n in range(3):
        e = errs[n]
        assert e[1] < 0.2 * e[0] and e[2] < 0.2 * e[1] and e[2] < 3e-3, (n, e)


def test_sphere_adjoint_double_layer_eigenvalue_converges():
    """S' (normal derivative of S at the target) on the unit sphere with outward normals:
    S'_k Y_n = (i k^2 / 2)(j_n h_n' + j_n' h_n) Y_n, which the Wronskian j_n h_n' - j_n' h_n
    = i / k^2 makes the same eigenvalue as D's (truth.sphere_eigen_D), for n = 0, 1, 2 with
    the densities Y_0 = 1, Y_1 = z, Y_2 = (3 z^2 - 1)/2; the error of the full pipeline
    falls with the chart error.  For n >= 1 the potential has a tangential gradient, which
    the error of the target normal (a derivative of the interpolated chart) multiplies at
    first order, so those errors fall more slowly than D's (measured: 0.115, 0.034, 0.0078
    for n = 1 at degrees 2, 4, 6, and 2.9e-4 on 80 degree-6 patches)."""
    k = 1.0
    lam = {n: truth.sphere_eigen_D(n, k) for n in range(3)}
    errs = {n: [] for n in range(3)}
    for sdiv, d in ((1, 2), (1, 4), (1, 6)):
        s = workloads.ellipsoid(sdiv, d)
        x, tn = workloads.onsurface_targets(s)
        z = s.xyz[2] / np.linalg.norm(s.xyz, axis=0)
        p = C.Params(eps=1e-7, eta=1.25, test_dirs=workloads.test_directions(4))
        corr = C.gen_corrections(s.deg, s.node_off, s.xyz, x, tn, "Sp", k, params=p)
        for n, Y in enumerate((np.ones_like(z), z, 0.5 * (3 * z * z - 1))):
            u = C.apply_corrected(corr, s.node_off, Y.astype(complex), x, "Sp", k, tgt_node=tn)
            errs[n].append(np.abs(u - lam[n] * Y).max() / abs(lam[n]))
    e = errs[0]
    assert e[1] < 0.2 * e[0] and e[2] < 0.2 * e[1] and e[2] < 3e-3, (0, e)
    for n in (1, 2):
        e = errs[n]
        assert e[1] < 0.4 * e[0] and e[2] < 0.3 * e[1] and e[2] < 1.5e-2, (n, e)


def test_adjoint_double_layer_kernel_is_normal_derivative_of_single_layer():
    """kernel_jac "Sp" equals the central difference of the S kernel along the target
    normal (x + h n_x)."""
    from oracle.kernels import kernel_jac
    rng = np.random.default_rng(8)
    x = rng.standard_normal(3)
    X = x[:, None] + rng.uniform(0.3, 2.0, 5) * rng.standard_normal((3, 5))
    N = rng.standard_normal((3, 5))
    nx = rng.standard_normal(3)
    nx /= np.linalg.norm(nx)
    for k in (0.0, 1.7, 2.0 + 0.5j):
        h = 1e-6
        fd = (kernel_jac(x + h * nx, X, N, k, "S") - kernel_jac(x - h * nx, X, N, k, "S")) / (2 * h)
        got = kernel_jac(x, X, N, k, "Sp", nx=nx)
        assert np.abs(fd - got).max() <= 1e-7 * np.abs(got).max()
