"""Seeded synthetic inputs: patch surfaces, targets, densities, test directions.

A surface is a collection of curved triangular charts X^j : T0 -> R^3 (Sec. 3.1),
each sampled at the discretization nodes of its degree (Sec. 5.2).  This module
describes inputs only; it holds no step of the correction method.  Both the CUDA
path and the CPU oracle consume what it returns.

Degrees follow the "total degree <= d" convention: a degree-d patch carries
n_d = (d+1)(d+2)/2 nodes, which is the paper's order p = d+1 (n_p = p(p+1)/2).

Discretization nodes.  The paper samples each chart at Vioreanu-Rokhlin nodes
(Sec. 2.2), whose tables are not published in the paper.  The stand-in used
throughout this project is the Blyth-Pozrikidis construction (IMA J. Appl. Math.
71, 2006) applied to the d+1 interior Gauss-Lobatto points of [0,1] (the roots
of the Jacobi polynomial P^{(1,1)}_{d+1}): every node is strictly interior,
and the interpolatory weights are positive for d = 1..10.  Each consumer of the
node set implements this closed form on its own; here the 1-D roots come from
the Golub-Welsch eigenvalue problem.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MAX_DEG = 10


def n_nodes(deg: int) -> int:
    return (deg + 1) * (deg + 2) // 2


def _interior_lobatto(n: int) -> np.ndarray:
    """Roots of P^{(1,1)}_n mapped to (0,1), ascending (Golub-Welsch)."""
    if n == 1:
        return np.array([0.5])
    k = np.arange(1, n, dtype=np.float64)
    off = np.sqrt(k * (k + 2.0) / ((2.0 * k + 1.0) * (2.0 * k + 3.0)))
    jac = np.diag(off, 1) + np.diag(off, -1)
    x = np.linalg.eigvalsh(jac)
    x = 0.5 * (x - x[::-1])  # exact antisymmetry of the root set
    return np.sort((1.0 + x) / 2.0)


def ref_nodes(deg: int) -> tuple[np.ndarray, np.ndarray]:
    """Discretization nodes (u_l, v_l) on T0 for degree `deg`.

    Order: i = 0..d outer, j = 0..d-i inner, k = d-i-j, with barycentric
    coordinates l1 = (1 + 2 t_i - t_j - t_k)/3 -> u and l2 = (1 + 2 t_j - t_i - t_k)/3 -> v.
    """
    if not 1 <= deg <= MAX_DEG:
        raise ValueError(f"degree {deg} outside 1..{MAX_DEG}")
    t = _interior_lobatto(deg + 1)
    u, v = [], []
    for i in range(deg + 1):
        for j in range(deg + 1 - i):
            k = deg - i - j
            u.append((1.0 + 2.0 * t[i] - t[j] - t[k]) / 3.0)
            v.append((1.0 + 2.0 * t[j] - t[i] - t[k]) / 3.0)
    return np.array(u), np.array(v)


# ----------------------------------------------------------------------------- charts
@dataclass
class Surface:
    """Patch surface: degrees, node offsets, SoA node coordinates [3][N]."""

    name: str
    deg: np.ndarray            # int32 [n_patches]
    node_off: np.ndarray       # int64 [n_patches + 1]
    xyz: np.ndarray            # float64 [3, N] (C-contiguous)
    meta: dict = field(default_factory=dict)

    @property
    def n_patches(self) -> int:
        return int(self.deg.shape[0])

    @property
    def n_points(self) -> int:
        return int(self.node_off[-1])


def _icosahedron() -> tuple[np.ndarray, np.ndarray]:
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-1.0, 1.0):
            v += [(0.0, a, b * g), (a, b * g, 0.0), (b * g, 0.0, a)]
    v = np.array(v)
    v /= np.linalg.norm(v, axis=1)[:, None]
    edge = min(np.linalg.norm(v[0] - v[i]) for i in range(1, 12))
    faces = []
    for i in range(12):
        for j in range(i + 1, 12):
            for k in range(j + 1, 12):
                if all(abs(np.linalg.norm(v[a] - v[b]) - edge) < 1e-9
                       for a, b in ((i, j), (j, k), (i, k))):
                    f = [i, j, k]
                    n = np.cross(v[j] - v[i], v[k] - v[i])
                    if np.dot(n, v[i] + v[j] + v[k]) < 0:
                        f = [i, k, j]
                    faces.append(f)
    return v, np.array(faces)


def _subdivided_faces(s: int) -> np.ndarray:
    """Flat icosahedron faces, each split into s*s triangles: [n_tri, 3 vertices, 3]."""
    v, faces = _icosahedron()
    tris = []
    for f in faces:
        A, B, C = v[f[0]], v[f[1]], v[f[2]]
        P = lambda i, j: A + (i / s) * (B - A) + (j / s) * (C - A)  # noqa: E731
        for i in range(s):
            for j in range(s - i):
                tris.append((P(i, j), P(i + 1, j), P(i, j + 1)))
                if i + j < s - 1:
                    tris.append((P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)))
    return np.array(tris)


def _sample(charts, degs) -> tuple[np.ndarray, np.ndarray]:
    degs = np.asarray(degs, dtype=np.int32)
    off = np.zeros(len(degs) + 1, dtype=np.int64)
    off[1:] = np.cumsum([n_nodes(int(d)) for d in degs])
    xyz = np.empty((3, int(off[-1])))
    cache = {}
    for j, (chart, d) in enumerate(zip(charts, degs)):
        d = int(d)
        if d not in cache:
            cache[d] = ref_nodes(d)
        u, v = cache[d]
        xyz[:, off[j]:off[j + 1]] = chart(u, v)
    return off, np.ascontiguousarray(xyz)


def ellipsoid(s: int, deg: int, axes=(1.0, 1.0, 1.0), flat: bool = False) -> Surface:
    """Icosahedron refined s*s per face, radially projected and scaled by `axes`.

    Chart of a sub-triangle (A, B, C): X(u,v) = diag(axes) * normalize(A + u(B-A) + v(C-A)).
    With flat=True the chart is the affine map itself (a polyhedron, not projected).
    Patches are oriented so that X_u x X_v points outward.
    """
    tris = _subdivided_faces(s)
    ax = np.asarray(axes, dtype=np.float64)[:, None]

    def make(t):
        A, B, C = (t[0][:, None], t[1][:, None], t[2][:, None])

        def chart(u, v):
            p = A + u[None, :] * (B - A) + v[None, :] * (C - A)
            if flat:
                return p
            return ax * (p / np.linalg.norm(p, axis=0)[None, :])
        return chart

    charts = [make(t) for t in tris]
    off, xyz = _sample(charts, [deg] * len(tris))
    name = ("icosahedron" if flat else "ellipsoid") + f"_s{s}_d{deg}"
    return Surface(name, np.full(len(tris), deg, np.int32), off, xyz,
                   {"kind": "flat" if flat else "ellipsoid", "s": s, "axes": tuple(axes),
                    "triangles": tris})


def torus_radius(theta, phi, amp=0.2):
    return 1.0 + amp * np.sin(3.0 * theta) * np.cos(5.0 * phi)


def torus_point(theta, phi, R=2.0, amp=0.2):
    r = torus_radius(theta, phi, amp)
    return np.stack([(R + r * np.cos(theta)) * np.cos(phi),
                     (R + r * np.cos(theta)) * np.sin(phi),
                     r * np.sin(theta)])


def torus(n_theta: int, n_phi: int, deg: int, R: float = 2.0, amp: float = 0.2) -> Surface:
    """Perturbed torus r(theta,phi) = 1 + amp*sin(3 theta)cos(5 phi) (theta poloidal).

    Two triangles per (phi, theta) grid cell, counter-clockwise in the (phi, theta)
    plane, which orients X_u x X_v outward.
    """
    charts = []
    dphi, dth = 2 * math.pi / n_phi, 2 * math.pi / n_theta
    for i in range(n_theta):
        for j in range(n_phi):
            p0 = np.array([j * dphi, i * dth])
            for (a, b, c) in (((0, 0), (1, 0), (1, 1)), ((0, 0), (1, 1), (0, 1))):
                P0 = p0 + np.array(a) * [dphi, dth]
                P1 = p0 + np.array(b) * [dphi, dth]
                P2 = p0 + np.array(c) * [dphi, dth]

                def chart(u, v, P0=P0, P1=P1, P2=P2):
                    q = P0[:, None] + u[None, :] * (P1 - P0)[:, None] + v[None, :] * (P2 - P0)[:, None]
                    return torus_point(q[1], q[0], R, amp)
                charts.append(chart)
    off, xyz = _sample(charts, [deg] * len(charts))
    return Surface(f"torus_{n_theta}x{n_phi}_d{deg}", np.full(len(charts), deg, np.int32), off, xyz,
                   {"kind": "torus", "n_theta": n_theta, "n_phi": n_phi, "R": R, "amp": amp})


# Twisted torus of the paper's numerical examples (Sec. 6): nonzero delta_{i,j} of
# X(u, v) = sum_{i,j} delta_{i,j} (cos v cos t, sin v cos t, sin t), t = (1 - i) u + j v.
STELLARATOR_DELTA = {(-1, -1): 0.17, (-1, 0): 0.11, (0, 0): 1.0, (1, 0): 4.5, (2, 0): -0.25,
                     (0, 1): 0.07, (2, 1): -0.45}


def stellarator_point(u, v):
    u, v = np.asarray(u, dtype=np.float64), np.asarray(v, dtype=np.float64)
    out = np.zeros((3,) + u.shape)
    for (i, j), dl in STELLARATOR_DELTA.items():
        t = (1 - i) * u + j * v
        out += dl * np.stack([np.cos(v) * np.cos(t), np.sin(v) * np.cos(t), np.sin(t)])
    return out


def stellarator(n_u: int, n_v: int, deg) -> Surface:
    """The paper's twisted torus on an n_u x n_v grid of (u, v) in [0, 2 pi]^2 (u poloidal,
    v toroidal), two triangles per cell with the right angle at the chart origin (so that
    a cell of equal physical sides gives aspect ratio 1); deg is one degree or one per
    patch.  Triangles are oriented so that X_u x X_v points away from the tube's centre circle 4.5 (cos v,
    sin v, 0) (outward)."""
    du, dv = 2 * math.pi / n_u, 2 * math.pi / n_v
    charts = []
    for a in range(n_u):
        for b in range(n_v):
            p0 = np.array([a * du, b * dv])
            for tri in (((0, 0), (1, 0), (0, 1)), ((1, 1), (0, 1), (1, 0))):
                P = [p0 + np.array(c) * [du, dv] for c in tri]
                # orientation from the chart's normal at the centroid
                cu, cv = (P[0] + P[1] + P[2]) / 3.0
                h = 1e-6
                e1, e2 = P[1] - P[0], P[2] - P[0]
                Xa = stellarator_point(np.array([cu + h * e1[0]]), np.array([cv + h * e1[1]]))[:, 0]
                Xb = stellarator_point(np.array([cu + h * e2[0]]), np.array([cv + h * e2[1]]))[:, 0]
                X0 = stellarator_point(np.array([cu]), np.array([cv]))[:, 0]
                nrm = np.cross(Xa - X0, Xb - X0)
                ctr = 4.5 * np.array([math.cos(cv), math.sin(cv), 0.0])
                if nrm @ (X0 - ctr) < 0:
                    P = [P[0], P[2], P[1]]

                def chart(uu, vv, P0=P[0], P1=P[1], P2=P[2]):
                    q = P0[:, None] + uu[None, :] * (P1 - P0)[:, None] + vv[None, :] * (P2 - P0)[:, None]
                    return stellarator_point(q[0], q[1])
                charts.append(chart)
    degs = np.full(len(charts), deg, np.int32) if np.isscalar(deg) else np.asarray(deg, np.int32)
    off, xyz = _sample(charts, degs)
    return Surface(f"stellarator_{n_u}x{n_v}_d{int(degs[0])}", degs, off, xyz,
                   {"kind": "stellarator", "n_u": n_u, "n_v": n_v})


def aspect_ratios(surf: Surface) -> np.ndarray:
    """Per-patch aspect ratio of Sec. 6: a_j = sqrt(int (s1/s2)^2 da / int da), s1 >= s2 the
    singular values of the chart's Jacobian DX, on the patch's node rule."""
    out = np.empty(surf.n_patches)
    cache = {}
    for j in range(surf.n_patches):
        d = int(surf.deg[j])
        if d not in cache:
            u, v = ref_nodes(d)
            cache[d] = (u, v, _vander_derivs(d, u, v))
        u, v, (Vm, Du, Dv) = cache[d]
        y = surf.xyz[:, surf.node_off[j]:surf.node_off[j + 1]]
        c = np.linalg.solve(Vm, y.T)          # monomial coefficients of the interpolant
        Xu, Xv = (Du @ c).T, (Dv @ c).T       # [3, n]
        G11, G12, G22 = (Xu * Xu).sum(0), (Xu * Xv).sum(0), (Xv * Xv).sum(0)
        tr, det = G11 + G22, G11 * G22 - G12 * G12
        disc = np.sqrt(np.maximum(tr * tr / 4 - det, 0.0))
        s1, s2 = np.sqrt(tr / 2 + disc), np.sqrt(np.maximum(tr / 2 - disc, 0.0))
        J = s1 * s2
        w = _node_weights(d)
        out[j] = math.sqrt(((s1 / s2) ** 2 * J * w).sum() / (J * w).sum())
    return out


def _vander_derivs(d, u, v):
    """Monomial Vandermonde u^a v^b (a + b <= d) at the nodes and its u, v derivatives."""
    ex = [(a, b) for a in range(d + 1) for b in range(d + 1 - a)]
    Vm = np.stack([u ** a * v ** b for a, b in ex], axis=1)
    Du = np.stack([a * u ** max(a - 1, 0) * v ** b if a else 0 * u for a, b in ex], axis=1)
    Dv = np.stack([b * u ** a * v ** max(b - 1, 0) if b else 0 * u for a, b in ex], axis=1)
    return Vm, Du, Dv


def _node_weights(d):
    """Interpolatory weights of the node set (monomial moments over T0)."""
    u, v = ref_nodes(d)
    ex = [(a, b) for a in range(d + 1) for b in range(d + 1 - a)]
    Vm = np.stack([u ** a * v ** b for a, b in ex], axis=0)
    mom = np.array([math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2) for a, b in ex])
    return np.linalg.solve(Vm, mom)


def torus_with_patches(n_patches: int, deg: int) -> Surface:
    """Torus with n_phi = 2 n_theta cells and the achievable count nearest n_patches."""
    nt = max(2, int(round(math.sqrt(n_patches / 4.0))))
    return torus(nt, 2 * nt, deg)


# ----------------------------------------------------------------------------- targets etc.
def onsurface_targets(surf: Surface) -> tuple[np.ndarray, np.ndarray]:
    """All discretization nodes as targets: xyz [3][N] and their node ids."""
    return surf.xyz.copy(), np.arange(surf.n_points, dtype=np.int64)


def radial_targets(surf: Surface, n: int, seed: int, lo: float, hi: float,
                   outside: bool = True) -> np.ndarray:
    """Off-surface points X(u,v)*(1 +/- delta), delta ~ U[lo,hi], at random nodes.

    For the sphere/ellipsoid family the radial direction points out of the body.
    """
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, surf.n_points, size=n)
    delta = rng.uniform(lo, hi, size=n)
    s = (1.0 + delta) if outside else (1.0 - delta)
    return np.ascontiguousarray(surf.xyz[:, idx] * s[None, :])


def density(n: int, seed: int) -> np.ndarray:
    """Complex normal density sigma = re + i im, re/im ~ N(0,1) from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(n)
    im = rng.standard_normal(n)
    return re + 1j * im


def test_directions(seed: int, count: int = 15) -> np.ndarray:
    """Random unit vectors [count][3] for the far-order test points of Sec. 4.2."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((count, 3))
    return np.ascontiguousarray(g / np.linalg.norm(g, axis=1)[:, None])


# ----------------------------------------------------------------------------- named configs
@dataclass
class Workload:
    name: str
    surface: Surface
    tgt_xyz: np.ndarray
    tgt_node: np.ndarray
    kernel: str                 # "S" | "D" | "CFIE"
    k: complex
    eps: float
    eta: float                  # <= 0: default by order
    alpha: complex = 1.0        # CFIE: alpha*D + beta*S
    beta: complex = 0.0
    sigma_seed: int = 0

    @property
    def n_points(self) -> int:
        return self.surface.n_points


def sphere_s_k1() -> Workload:
    """Single layer, k=1, unit sphere as 20 flat-to-sphere degree-4 patches (300 points),
    eps=1e-6, eta=1.25."""
    s = ellipsoid(1, 4)
    x, t = onsurface_targets(s)
    return Workload("sphere20_d4_S_k1_eps1e-6", s, x, t, "S", 1.0, 1e-6, 1.25)


def ellipsoid_cfie_k2pi(s: int = 8) -> Workload:
    """CFIE D - ik S, k=2 pi, ellipsoid (1,2,3) with 20 s^2 degree-6 patches, eps=1e-9."""
    surf = ellipsoid(s, 6, axes=(1.0, 2.0, 3.0))
    x, t = onsurface_targets(surf)
    k = 2.0 * math.pi
    return Workload(f"ellipsoid123_{20*s*s}p_d6_CFIE_k2pi_eps1e-9", surf, x, t, "CFIE", k, 1e-9,
                    -1.0, alpha=1.0, beta=-1j * k)


def torus_cfie_k20(n_theta: int = 100) -> Workload:
    """CFIE, k=20, perturbed torus with 2*n_theta*2n_theta degree-6 patches, eps=1e-9."""
    surf = torus(n_theta, 2 * n_theta, 6)
    x, t = onsurface_targets(surf)
    return Workload(f"torus_{surf.n_patches}p_d6_CFIE_k20_eps1e-9", surf, x, t, "CFIE", 20.0, 1e-9,
                    -1.0, alpha=1.0, beta=-20j)


def batched_tori(count: int = 64, seed: int = 0, scale: float = 1.0):
    """Independent tori: patches ~ U[200,5000]*scale, degree ~ U{3..8}, k ~ U[1,20],
    eps ~ U{1e-6,1e-9}, density dtype ~ U{c64,c128}, drawn in that order per surface."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        npat = int(rng.integers(200, 5001))
        deg = int(rng.integers(3, 9))
        k = float(rng.uniform(1.0, 20.0))
        eps = float(rng.choice([1e-6, 1e-9]))
        dt = str(rng.choice(["complex64", "complex128"]))
        out.append(dict(n_patches=max(8, int(npat * scale)), deg=deg, k=k, eps=eps, dtype=dt))
    return out


def concat_surfaces(parts, shifts=None, name: str = "batch"):
    """Several surfaces as one Surface, one after another (part i translated by shifts[i]),
    and the patch range of each part ([n_parts + 1], starting at 0)."""
    shifts = shifts if shifts is not None else [(0.0, 0.0, 0.0)] * len(parts)
    deg = np.concatenate([p.deg for p in parts]).astype(np.int32)
    off = [np.zeros(1, np.int64)]
    xyz = []
    for p, sh in zip(parts, shifts):
        off.append(off[-1][-1] + p.node_off[1:])
        xyz.append(p.xyz + np.asarray(sh, dtype=np.float64)[:, None])
    patch_off = np.concatenate([[0], np.cumsum([p.n_patches for p in parts])]).astype(np.int64)
    return Surface(name, deg, np.concatenate(off), np.ascontiguousarray(np.concatenate(xyz, 1)),
                   {"kind": "batch", "parts": [p.name for p in parts]}), patch_off


def batched_tori_batch(count: int = 64, seed: int = 0, scale: float = 1.0, spacing: float = 8.0):
    """The batched-tori workload as one concatenated surface: the tori drawn by
    batched_tori (n_phi = 2 n_theta cells nearest the drawn patch count) on a square
    lattice `spacing` apart (the tori, of outer radius 3.2, do not touch), their patch
    ranges, and per torus the CFIE physics (k, alpha=1, beta=-ik, eps) and density dtype."""
    specs = batched_tori(count, seed, scale)
    side = int(math.ceil(math.sqrt(count)))
    parts, shifts, phys = [], [], []
    for i, sp in enumerate(specs):
        parts.append(torus_with_patches(sp["n_patches"], sp["deg"]))
        shifts.append((spacing * (i % side), spacing * (i // side), 0.0))
        phys.append((sp["k"], 1.0, -1j * sp["k"], sp["eps"]))
    surf, patch_off = concat_surfaces(parts, shifts, f"tori{count}_seed{seed}_x{scale:g}")
    return surf, patch_off, phys, [sp["dtype"] for sp in specs]


def exterior_targets(surf: Surface, n: int, seed: int, lo: float = 0.05, hi: float = 0.5):
    """Off-surface points p (1 + delta), delta ~ U[lo, hi], where p is a random convex
    combination (Dirichlet weights) of the nodes of a random patch: a point on or just
    inside the patch, pushed outward along the radius (the ellipsoid family is star-shaped
    about the origin)."""
    rng = np.random.default_rng(seed)
    pts = []
    for _ in range(n):
        j = int(rng.integers(0, surf.n_patches))
        y = surf.xyz[:, surf.node_off[j]:surf.node_off[j + 1]]
        p = y @ rng.dirichlet(np.ones(y.shape[1]))
        pts.append(p * (1.0 + rng.uniform(lo, hi)))
    return np.ascontiguousarray(np.array(pts).T)


def ellipsoid_adjoint_s_k5(s: int = 10):
    """Gradient workload: single layer k=5 on the ellipsoid (1, 1.5, 2.5) with 20 s^2
    degree-5 patches, eps=1e-8, 1000 exterior targets."""
    surf = ellipsoid(s, 5, axes=(1.0, 1.5, 2.5))
    x = exterior_targets(surf, 1000, 0)
    return surf, x


# (n_u, n_v) cell grids of the twisted torus for the five columns of the paper's Table 2
# (aspect-ratio sweep at about 2400 patches): 2 n_u n_v patches, average aspect ratios
# 1.610, 2.333, 4.658, 9.314, 13.97 at degree 3 (printed: 1.61, 2.33, 4.66, 9.32, 14).
TABLE2_GRIDS = ((20, 60), (24, 48), (35, 35), (48, 24), (60, 20))


def stellarator_s_k1(deg: int = 3) -> Workload:
    """Single layer, k=1, on the paper's twisted torus with 2400 patches (20 x 60 cells,
    average aspect ratio 1.61 as in the paper's Table 2 first column); eps=5e-7."""
    surf = stellarator(20, 60, deg)
    x, t = onsurface_targets(surf)
    return Workload(f"stellarator2400_d{deg}_S_k1", surf, x, t, "S", 1.0, 5e-7, -1.0)
