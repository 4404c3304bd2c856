"""Koornwinder orthonormal basis on T0 = {u,v >= 0, u+v <= 1} (Sec. 2, Eq. for K_nm).

K_nm(u,v) = c_nm (1-v)^m P^{(0,2m+1)}_{n-m}(1-2v) P_m((2u+v-1)/(1-v)),  0 <= m <= n <= d,
with c_nm chosen so that the integral of K_nm^2 over T0 is 1.  Working the
integral through the substitution x = (2u+v-1)/(1-v), y = 1-2v and the Legendre
and Jacobi norms gives c_nm = sqrt(2 (2m+1)(n+1)).

Basis order: n-major, then m ascending: index(n, m) = n(n+1)/2 + m.  (The paper
writes both "n+m < p" and "0 <= m <= n"; the total degree of K_nm is n, so the
degree-d space is n <= d.)

The factor (1-v)^m P_m((2u+v-1)/(1-v)) is evaluated by the Legendre three-term
recurrence multiplied through by (1-v)^{m+1}, which never divides by 1-v.
Parity unpinned: none (pinned by orthonormality, closed-form low-order members
and finite differences in tests/test_oracle_koornwinder.py).
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_jacobi


def n_basis(d: int) -> int:
    """Number of Koornwinder polynomials of total degree <= d: the paper's n_p = p(p+1)/2
    with p = d + 1 (Sec. 2.1)."""
    return (d + 1) * (d + 2) // 2


def index(n: int, m: int) -> int:
    """Position of K_nm in the basis, n-major with m ascending (Sec. 2.1 indexes the
    basis by (n, m) without fixing an order; this one is used throughout)."""
    return n * (n + 1) // 2 + m


def c_nm(n: int, m: int) -> float:
    """Normalization of K_nm (Sec. 2.1 leaves it to the cited basis): sqrt(2(2m+1)(n+1)),
    the constant that makes the integral of K_nm^2 over T0 equal to 1."""
    return float(np.sqrt(2.0 * (2 * m + 1) * (n + 1)))


def scaled_legendre(mmax: int, u, v):
    """L_m = (1-v)^m P_m((2u+v-1)/(1-v)) for m = 0..mmax with d/du and d/dv: the Legendre
    factor of the Koornwinder polynomials of Sec. 2.1.

    Legendre: (m+1) P_{m+1}(x) = (2m+1) x P_m(x) - m P_{m-1}(x); with s = 2u+v-1 and
    q = 1-v this becomes (m+1) L_{m+1} = (2m+1) s L_m - m q^2 L_{m-1}.
    """
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    s = 2.0 * u + v - 1.0
    q = 1.0 - v
    L = [np.ones_like(u), s]
    Lu = [np.zeros_like(u), np.full_like(u, 2.0)]
    Lv = [np.zeros_like(u), np.ones_like(u)]
    for m in range(1, mmax):
        L.append(((2 * m + 1) * s * L[m] - m * q * q * L[m - 1]) / (m + 1))
        Lu.append(((2 * m + 1) * (2.0 * L[m] + s * Lu[m]) - m * q * q * Lu[m - 1]) / (m + 1))
        Lv.append(((2 * m + 1) * (L[m] + s * Lv[m])
                   - m * (-2.0 * q * L[m - 1] + q * q * Lv[m - 1])) / (m + 1))
    return L[:mmax + 1], Lu[:mmax + 1], Lv[:mmax + 1]


def basis(d: int, u, v, derivs: bool = False):
    """K[nm, point] for all 0 <= m <= n <= d (the Koornwinder basis of Sec. 2.1,
    K_nm = c_nm L_m P^{(0,2m+1)}_{n-m}(1-2v)); with derivs also dK/du and dK/dv."""
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    v = np.atleast_1d(np.asarray(v, dtype=np.float64))
    L, Lu, Lv = scaled_legendre(d, u, v)
    y = 1.0 - 2.0 * v
    nb = n_basis(d)
    K = np.empty((nb, u.size))
    Ku = np.empty((nb, u.size))
    Kv = np.empty((nb, u.size))
    for n in range(d + 1):
        for m in range(n + 1):
            a, beta = n - m, 2 * m + 1
            P = eval_jacobi(a, 0.0, beta, y)
            # d/dy P_a^{(0,b)}(y) = (a+b+1)/2 P_{a-1}^{(1,b+1)}(y)
            dP = 0.5 * (a + beta + 1) * eval_jacobi(a - 1, 1.0, beta + 1, y) if a > 0 else 0.0 * y
            c = c_nm(n, m)
            i = index(n, m)
            K[i] = c * L[m] * P
            Ku[i] = c * Lu[m] * P
            Kv[i] = c * (Lv[m] * P + L[m] * (-2.0) * dP)
    if derivs:
        return K, Ku, Kv
    return K


def jacobi_recurrence(a: int, b: int):
    """P^{(0,b)}_{a+1}(y) = (c1 y + c0) P_a(y) - c2 P_{a-1}(y): the textbook three-term
    recurrence of the Jacobi factor of the Sec. 2.1 basis."""
    den = 2.0 * (a + 1) * (a + b + 1) * (2 * a + b)
    c1 = (2 * a + b + 1) * (2 * a + b + 2) * (2 * a + b) / den
    c0 = -(2 * a + b + 1) * b * b / den
    c2 = 2.0 * a * (a + b) * (2 * a + b + 2) / den
    return c1, c0, c2


def basis_delta(d: int, P, du, dv):
    """K_nm(P + delta) - K_nm(P) (the Sec. 2.1 basis) for offsets delta = (du, dv), as the
    self rules of Sec. 4 need them near the target node, computed without forming
    the two values: the differences obey the same recurrences, e.g. for the scaled
    Legendre factor
        (m) dL_m = (2m-1)(s_Q dL_{m-1} + ds L_{m-1}(P)) - (m-1)(q_Q^2 dL_{m-2} + d(q^2) L_{m-2}(P)),
    with ds = 2 du + dv and d(q^2) = -dv (q_Q + q_P), and for the Jacobi factor
        dP_{a+1} = (c1 y_Q + c0) dP_a + c1 dy P_a(P) - c2 dP_{a-1},  dy = -2 dv.
    The result keeps full relative precision as delta -> 0 (used by the self rules, where
    x - X(P + delta) = -(X(P + delta) - X(P)) sets the near-singular behaviour)."""
    du = np.atleast_1d(np.asarray(du, dtype=np.float64))
    dv = np.atleast_1d(np.asarray(dv, dtype=np.float64))
    pu, pv = float(P[0]), float(P[1])
    uq, vq = pu + du, pv + dv
    sP, qP, yP = 2 * pu + pv - 1.0, 1.0 - pv, 1.0 - 2.0 * pv
    sQ, qQ, yQ = 2 * uq + vq - 1.0, 1.0 - vq, 1.0 - 2.0 * vq
    ds = 2.0 * du + dv
    dq2 = -dv * (qQ + qP)
    dy = -2.0 * dv
    nb = n_basis(d)
    out = np.empty((nb, du.size))
    LP = [1.0, sP]
    LQ = [np.ones_like(du), sQ]
    dL = [np.zeros_like(du), ds]
    for m in range(1, d):
        LP.append(((2 * m + 1) * sP * LP[m] - m * qP * qP * LP[m - 1]) / (m + 1))
        LQ.append(((2 * m + 1) * sQ * LQ[m] - m * qQ * qQ * LQ[m - 1]) / (m + 1))
        dL.append(((2 * m + 1) * (sQ * dL[m] + ds * LP[m])
                   - m * (qQ * qQ * dL[m - 1] + dq2 * LP[m - 1])) / (m + 1))
    for m in range(d + 1):
        b = 2 * m + 1
        PP, PQ, dP = 1.0, np.ones_like(du), np.zeros_like(du)
        PPm, PQm, dPm = 0.0, np.zeros_like(du), np.zeros_like(du)
        for a in range(d - m + 1):
            n = m + a
            out[index(n, m)] = c_nm(n, m) * (dL[m] * PQ + LP[m] * dP)
            c1, c0, c2 = jacobi_recurrence(a, b)
            PPn = (c1 * yP + c0) * PP - c2 * PPm
            PQn = (c1 * yQ + c0) * PQ - c2 * PQm
            dPn = (c1 * yQ + c0) * dP + c1 * dy * PP - c2 * dPm
            PPm, PP = PP, PPn
            PQm, PQ = PQ, PQn
            dPm, dP = dP, dPn
    return out
