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
    return (d + 1) * (d + 2) // 2


def index(n: int, m: int) -> int:
    return n * (n + 1) // 2 + m


def c_nm(n: int, m: int) -> float:
    return float(np.sqrt(2.0 * (2 * m + 1) * (n + 1)))


def scaled_legendre(mmax: int, u, v):
    """L_m = (1-v)^m P_m((2u+v-1)/(1-v)) for m = 0..mmax with d/du and d/dv.

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
    """K[nm, point] for all 0 <= m <= n <= d; with derivs also dK/du and dK/dv."""
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
