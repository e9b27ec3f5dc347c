"""Butcher tableaux of the fully implicit families of Section 5: RadauIIA(s)
(order 2s-1), Gauss(s) (order 2s) and LobattoIIIC(s) (order 2s-2), all of
stage order s in the sense used there; Section 2 fixes the consistency
conditions sum_j b_j = 1 and sum_j a_ij = c_i and the stability function r(z).

The nodes c are the s roots of P_s(2x-1) - P_{s-1}(2x-1) (Radau right points,
so c_s = 1).  A follows from the simplifying condition C(s):
    sum_j a_ij c_j^(k-1) = c_i^k / k,  k = 1..s,
and b from B(s): sum_i b_i c_i^(k-1) = 1/k, k = 1..s.
"""
import numpy as np
from numpy.polynomial import legendre as L


def radau_nodes(s):
    # coefficients of P_s - P_{s-1} in the Legendre basis, as a function of xi = 2x-1
    coef = np.zeros(s + 1)
    coef[s] = 1.0
    coef[s - 1] = -1.0
    xi = np.sort(np.real(L.legroots(coef)))
    return (xi + 1.0) / 2.0


def radau_iia(s):
    """Return (A, b, c) for the s-stage Radau IIA method in FP64."""
    if s < 1:
        raise ValueError("s >= 1")
    c = radau_nodes(s)
    c[-1] = 1.0
    V = np.vander(c, s, increasing=True)           # V[j, k] = c_j^k
    rhs = np.array([[ci ** (k + 1) / (k + 1) for k in range(s)] for ci in c])
    A = np.linalg.solve(V.T, rhs.T).T               # A V = rhs  (C(s))
    b = np.linalg.solve(V.T, np.array([1.0 / (k + 1) for k in range(s)]))
    return A, b, c


def stability_function(A, b, z):
    """r(z) = 1 + z b^T (I - z A)^{-1} 1  (Section 2, Dahlquist test problem)."""
    s = len(b)
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))


def check_consistency(A, b, c, tol=1e-12):
    """The two consistency conditions of Section 2."""
    return abs(b.sum() - 1.0) <= tol and np.all(np.abs(A.sum(axis=1) - c) <= tol)


def gauss_nodes(s):
    """Roots of P_s(2x-1) (Gauss-Legendre points on [0, 1])."""
    coef = np.zeros(s + 1)
    coef[s] = 1.0
    return (np.sort(np.real(L.legroots(coef))) + 1.0) / 2.0


def lobatto_nodes(s):
    """0, 1 and the roots of P'_{s-1}(2x-1) (Lobatto points on [0, 1])."""
    if s == 2:
        return np.array([0.0, 1.0])
    coef = np.zeros(s)
    coef[s - 1] = 1.0
    inner = np.sort(np.real(L.legroots(L.legder(coef))))
    return np.concatenate([[0.0], (inner + 1.0) / 2.0, [1.0]])


def _quadrature_weights(c):
    s = len(c)
    V = np.vander(c, s, increasing=True)
    return np.linalg.solve(V.T, np.array([1.0 / (k + 1) for k in range(s)]))


def gauss(s):
    """Gauss(s): collocation at the Gauss points, i.e. C(s) with those nodes."""
    c = gauss_nodes(s)
    V = np.vander(c, s, increasing=True)
    rhs = np.array([[ci ** (k + 1) / (k + 1) for k in range(s)] for ci in c])
    A = np.linalg.solve(V.T, rhs.T).T
    return A, _quadrature_weights(c), c


def lobatto_iiic(s):
    """LobattoIIIC(s): Lobatto nodes and weights, first column a_i1 = b_1 and
    the simplifying condition C(s-1): sum_j a_ij c_j^(k-1) = c_i^k / k for
    k = 1..s-1 (s-1 equations for the remaining s-1 entries of each row)."""
    c = lobatto_nodes(s)
    b = _quadrature_weights(c)
    A = np.zeros((s, s))
    A[:, 0] = b[0]
    # unknowns a_i2..a_is: sum_{j>=2} a_ij c_j^(k-1) = c_i^k/k - b_1 c_1^(k-1)
    Vr = np.array([[c[j] ** k for j in range(1, s)] for k in range(s - 1)])
    for i in range(s):
        rhs = np.array([c[i] ** (k + 1) / (k + 1) - b[0] * c[0] ** k for k in range(s - 1)])
        A[i, 1:] = np.linalg.solve(Vr, rhs)
    return A, b, c
