"""Layer-potential kernels times the area element (Sec. 3, Eq. greenfunhelm, sldef, dldef).

G_k(x,y) = e^{ik|x-y|} / (4 pi |x-y|).
Single layer: K_S J = G_k(x, X) |n|.
Double layer: n(y).grad_y G_k J; with n = X_u x X_v unnormalized this is
    n.(x-y) (1 - ik r) e^{ikr} / (4 pi r^3).
Combined field (Eq. urep, inteq): alpha D + beta S, default alpha = 1, beta = -ik.
Adjoint double layer S' (Sec. 3, the normal derivative of S at the target, used for
Neumann problems): n_x.grad_x G_k J = -n_x.(x-y) (1 - ik r) e^{ikr} / (4 pi r^3) |n|, with
n_x the target's unit normal.
A source point at r = 0 contributes 0 (it only occurs when a rule node meets a target).
"""
from __future__ import annotations

import numpy as np

FOUR_PI = 4.0 * np.pi


def kernel_jac(x, X, N, k, kind: str, alpha=1.0, beta=0.0, nx=None):
    """Kernel values times J at sources X [3,P] with normals N [3,P] for target x [3]:
    G_k = e^{ikr}/(4 pi r) for S, n(y) . grad_y G_k for D, alpha D + beta S for the CFIE,
    and n(x) . grad_x G_k for S' (Sec. 3, the single- and double-layer definitions).

    kind: "S", "D", "CFIE" (alpha D + beta S) or "Sp" (S', needs the target's unit
    normal nx [3]).  Returns complex [P].
    """
    x = np.asarray(x, dtype=np.float64)
    dvec = x[:, None] - X
    r = np.sqrt((dvec * dvec).sum(axis=0))
    zero = r == 0.0
    rs = np.where(zero, 1.0, r)
    e = np.exp(1j * k * rs) / (FOUR_PI * rs)
    out = np.zeros(X.shape[1], dtype=np.complex128)
    if kind in ("S", "CFIE"):
        s = e * np.sqrt((N * N).sum(axis=0))
        out = out + (s if kind == "S" else beta * s)
    if kind in ("D", "CFIE"):
        ndx = (N * dvec).sum(axis=0)
        dd = ndx * (1.0 - 1j * k * rs) * e / (rs * rs)
        out = out + (dd if kind == "D" else alpha * dd)
    if kind == "Sp":
        nxd = (np.asarray(nx, dtype=np.float64)[:, None] * dvec).sum(axis=0)
        out = -nxd * (1.0 - 1j * k * rs) * e / (rs * rs) * np.sqrt((N * N).sum(axis=0))
    out[zero] = 0.0
    return out


def kernel_envelope(x, X, N, k, kind: str, alpha=1.0, beta=0.0, R=1.0, nx=None):
    """Rounding envelope of kernel_jac at each source, which sets the floor of the adaptive
    test of Sec. 4.3 (a reading; the paper is silent on finite precision): |G| J (b + a |1 - ik r| R / r^2), with b = 1, 0, |beta|, 0 and
    a = 0, 1, |alpha|, 1 for S, D, CFIE, S' (the target-normal factor of S' rounds like the
    source-normal factor of D).  The double-layer term is the size of
    |n| |delta(x - X)| / r^2 for a coordinate rounding error delta ~ u R (charts and
    targets are taken relative to the patch centroid), which bounds the noise of
    n.(x - X) when x is nearly in the tangent plane."""
    x = np.asarray(x, dtype=np.float64)
    dvec = x[:, None] - X
    r = np.sqrt((dvec * dvec).sum(axis=0))
    zero = r == 0.0
    rs = np.where(zero, 1.0, r)
    k = complex(k)
    g = np.exp(-k.imag * rs) / (FOUR_PI * rs) * np.sqrt((N * N).sum(axis=0))
    b = {"S": 1.0, "D": 0.0, "CFIE": abs(beta), "Sp": 0.0}[kind]
    a = {"S": 0.0, "D": 1.0, "CFIE": abs(alpha), "Sp": 1.0}[kind]
    f = np.sqrt((1.0 + k.imag * rs) ** 2 + (k.real * rs) ** 2)
    out = g * (b + a * f * R / (rs * rs))
    out[zero] = 0.0
    return out
