"""The parameters and rules the paper states in its text or tables
(tests/golden/paper_parameters.txt, each value with its section or table) against the
oracle, the input generators, and the library's host-side defaults and node tables where
the library exposes them without a GPU."""
import ctypes as C
import os

import numpy as np
import pytest

from oracle import corrections, geometry, nearlist, rules

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "paper_parameters.txt")


def load_golden():
    """name -> (value, printed text of the value)"""
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, cite = line.split(None, 2)
            assert cite.startswith(("Sec. ", "Table ")), f"{name} has no citation"
            out[name] = (float(value), value)
    return out


G = {k: v for k, (v, _) in load_golden().items()}
PRINTED = {k: t for k, (_, t) in load_golden().items()}


def paper_eta(p):
    if p <= 4:
        return G["eta.p_le_4"]
    if p <= 8:
        return G["eta.p_le_8"]
    return G["eta.p_gt_8"]


def test_golden_file_complete():
    assert set(G) == {"eta.p_le_4", "eta.p_le_8", "eta.p_gt_8", "eta1", "far_test.count",
                      "far_test.small_list", "far_test.sphere_pts", "subdivision.children",
                      "nodes.p16"} | {f"table2.{q}.{c}" for q in ("npat", "a_avg")
                                      for c in range(1, 6)}


@pytest.mark.parametrize("d", range(0, 13))
def test_default_eta_by_order(d):
    # the degree-d patch has the paper's order p = d + 1
    assert geometry.default_eta(d) == paper_eta(d + 1)


def test_eta1_defaults():
    assert corrections.Params(eps=1e-6).eta1 == G["eta1"]


@pytest.mark.parametrize("size", [0, 1, 2, 3, 9, 18, 19, 20, 21, 37, 250])
def test_far_test_set_sizes(size):
    rng = np.random.default_rng(size)
    ids = np.sort(rng.choice(10 * size + 5, size=size, replace=False)).astype(np.int64)
    d2 = rng.uniform(0.1, 4.0, size)
    far_t, add_sphere = nearlist.far_test_targets(ids, d2)
    small = size < G["far_test.small_list"]
    want = size // 2 if small else int(G["far_test.count"])
    assert len(far_t) == want and add_sphere == small
    # the farthest ones: every chosen target is at least as far as every other one
    if 0 < want < size:
        rest = np.setdiff1d(ids, far_t)
        chosen_d2 = d2[np.searchsorted(ids, far_t)]
        rest_d2 = d2[np.searchsorted(ids, rest)]
        assert chosen_d2.min() >= rest_d2.max()


def test_sphere_points_of_the_small_list_rule():
    dirs = corrections.fibonacci_dirs()
    assert dirs.shape == (int(G["far_test.sphere_pts"]), 3)
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-15)
    assert len({tuple(np.round(x, 12)) for x in dirs}) == dirs.shape[0]


def test_midpoint_subdivision():
    T0 = (np.array([0.0, 0.0]), np.array([1.0, 0.0]), np.array([0.0, 1.0]))
    kids = rules.subdivide(T0)
    assert len(kids) == G["subdivision.children"]

    def area(T):
        a, b, c = T
        return 0.5 * abs((b[0] - a[0]) * (c[1] - a[1]) - (c[0] - a[0]) * (b[1] - a[1]))

    for T in kids:
        assert area(T) == area(T0) / G["subdivision.children"]
    # the children's vertices are T0's corners and edge midpoints, each corner in one child
    verts = {tuple(x) for T in kids for x in T}
    assert verts == {(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (0.5, 0.0), (0.5, 0.5), (0.0, 0.5)}
    for corner in [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0)]:
        assert sum(corner in {tuple(x) for x in T} for T in kids) == 1


def test_nodes_per_patch():
    # order p = 16 is degree 15
    u, v = rules.interp_nodes(15)
    assert len(u) == len(v) == G["nodes.p16"]
    for d in range(1, 11):
        assert len(rules.interp_nodes(d)[0]) == (d + 1) * (d + 2) // 2


def test_aspect_ratio_closed_form():
    # the chart A + u(B - A) + v(C - A) of an equilateral triangle has DX = [B - A, C - A]
    # with singular values in the ratio sqrt(3) everywhere, so a_j = sqrt(3) exactly
    # (Sec. 6.1 definition, sigma read as the singular values of DX)
    from paper_2006_02545_gb300 import workloads as W
    a = W.aspect_ratios(W.ellipsoid(2, 3, flat=True))   # flat icosahedron, 80 equilateral faces
    assert len(a) == 80 and np.abs(a - np.sqrt(3.0)).max() < 1e-12


@pytest.mark.parametrize("col", range(1, 6))
def test_twisted_torus_aspect_ratio_row_of_table2(col):
    # the paper's twisted torus (Sec. 6) at p = 4 (degree 3) on the input generator's grid
    # for column `col` of Table 2: its patch count, and its average aspect ratio (Sec. 6.1
    # definition) within one unit of the last printed digit
    from paper_2006_02545_gb300 import workloads as W
    n_u, n_v = W.TABLE2_GRIDS[col - 1]
    s = W.stellarator(n_u, n_v, 3)
    assert s.n_patches == G[f"table2.npat.{col}"]
    text = PRINTED[f"table2.a_avg.{col}"]
    unit = 10.0 ** -(len(text.split(".")[1]) if "." in text else 0)
    assert abs(float(W.aspect_ratios(s).mean()) - G[f"table2.a_avg.{col}"]) <= unit


@pytest.fixture(scope="module")
def lcq():
    import __graft_entry__ as g
    g.build()
    from paper_2006_02545_gb300 import lcq as mod
    return mod


def test_library_host_defaults(lcq):
    # the C default, before the binding applies its own keyword defaults
    p = lcq.Params_t()
    lcq._lib.lcq_params_default(C.byref(p))
    assert p.eta == -1.0          # -1: the paper's cutoff by order, applied per patch
    assert p.eta1 == G["eta1"]
    assert p.n_test_dirs == 0     # 0: the library's own sphere directions


def test_library_node_count(lcq):
    for d in range(1, 11):
        u, v, w = lcq.ref_nodes(d)
        assert len(u) == (d + 1) * (d + 2) // 2
