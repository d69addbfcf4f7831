"""Pins of the oracle's method coefficients by the order conditions.

Tsit5 (paper Sec. 2.1, Tsitouras 2011): all 17 rooted trees up to order 5 for b,
all 8 up to order 4 for bhat. Rodas5P (paper Sec. 3.2, Steinebach 2023): the
Rosenbrock order conditions (Hairer & Wanner II, Sec. IV.7) after converting the
transformed (a, C, m) form back to (alpha, Gamma, b). The elementary weights
are computed here from the trees, independently of the oracle's step code.
"""
import numpy as np
import pytest

import oracle

TOL = 5e-14  # the published tables carry ~16 significant digits


def _trees(n, memo={}):
    if n in memo:
        return memo[n]
    if n == 1:
        memo[1] = [()]
        return memo[1]
    out = set()

    def rec(rem, acc):
        if rem == 0:
            out.add(tuple(sorted(acc)))
            return
        for m in range(1, rem + 1):
            for t in _trees(m):
                rec(rem - m, acc + [(m, t)])

    rec(n - 1, [])
    memo[n] = sorted(out)
    return memo[n]


def _order(t):
    return 1 + sum(m for m, _ in t)


def _density(t):
    return _order(t) * np.prod([_density(c) for _, c in t]) if t else 1.0


def _phi(t, alpha, B):
    """Elementary weight of tree t. Single-child nodes couple through B = alpha + Gamma
    (the Rosenbrock Jacobian term), multi-child nodes through alpha alone."""
    s = alpha.shape[0]
    if not t:
        return np.ones(s)
    if len(t) == 1:
        return B @ _phi(t[0][1], alpha, B)
    out = np.ones(s)
    for _, c in t:
        out = out * (alpha @ _phi(c, alpha, B))
    return out


def residuals(alpha, Gam, b, p):
    B = alpha + Gam
    return [(t, float(b @ _phi(t, alpha, B) - 1.0 / _density(t))) for n in range(1, p + 1) for t in _trees(n)]


def rodas_standard(tab):
    """(a, C, m, gamma) transformed form -> (alpha, Gamma, b):
    Gamma^{-1} = diag(1/gamma) - C, alpha = a Gamma, b = m Gamma."""
    g = tab["gamma"]
    Ginv = np.diag(np.full(8, 1.0 / g)) - tab["C"]
    G = np.linalg.inv(Ginv)
    return tab["a"] @ G, G, tab["m"] @ G


def test_tree_counts():
    # 1, 1, 2, 4, 9, 20, 48 rooted trees of orders 1..7 (Butcher).
    assert [len(_trees(n)) for n in range(1, 8)] == [1, 1, 2, 4, 9, 20, 48]


def test_tsit5_order_conditions():
    tab = oracle.tableau(oracle.METHOD_TSIT5)
    A, b, bh, c = tab["A"], tab["b"], tab["bhat"], tab["c"]
    Z = np.zeros_like(A)
    r5 = residuals(A, Z, b, 5)
    r4 = residuals(A, Z, bh, 4)
    assert len(r5) == 17 and len(r4) == 8
    assert max(abs(r) for _, r in r5) < TOL
    assert max(abs(r) for _, r in r4) < TOL
    # bhat is a genuinely lower-order solution: some order-5 condition fails for it
    assert max(abs(r) for _, r in residuals(A, Z, bh, 5)) > 1e-4
    np.testing.assert_allclose(A.sum(1), c, atol=1e-15)
    # FSAL: the last stage is evaluated at y_new (row 7 of A equals b, b_7 = 0)
    np.testing.assert_array_equal(A[6], b)
    assert b[6] == 0.0
    assert np.allclose(np.tril(A, -1), A)  # explicit


def test_rodas5p_order_conditions():
    tab = oracle.tableau(oracle.METHOD_RODAS5P)
    alpha, G, b = rodas_standard(tab)
    mh = tab["m"].copy()
    mh[7] = 0.0  # embedded solution: y_new - U_8
    bh = mh @ G
    r5 = residuals(alpha, G, b, 5)
    r4 = residuals(alpha, G, bh, 4)
    assert max(abs(r) for _, r in r5) < TOL
    assert max(abs(r) for _, r in r4) < TOL
    assert max(abs(r) for _, r in residuals(alpha, G, bh, 5)) > 1e-6
    assert np.allclose(np.diag(G), tab["gamma"])


def _rosenbrock_R(alpha, G, b, z):
    # Scalar stability function: R(z) = 1 + z b^T (I - z (alpha + Gamma))^{-1} 1
    B = alpha + G
    s = B.shape[0]
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * B, np.ones(s))


def test_rodas5p_stiffly_accurate():
    tab = oracle.tableau(oracle.METHOD_RODAS5P)
    alpha, G, b = rodas_standard(tab)
    mh = tab["m"].copy()
    mh[7] = 0.0
    bh = mh @ G
    for z in (-1e8, -1e12):
        assert abs(_rosenbrock_R(alpha, G, b, z)) < 1e-6
        assert abs(_rosenbrock_R(alpha, G, bh, z)) < 1e-6
    # A-stability spot check on the negative real axis and the imaginary axis
    for z in np.concatenate([-np.logspace(-3, 6, 60), 1j * np.logspace(-3, 6, 60)]):
        assert abs(_rosenbrock_R(alpha, G, b, z)) <= 1.0 + 1e-12


def test_verner7_order_conditions():
    """Verner's 7(6) pair: all 85 trees to order 7 for b, all 37 to order 6 for
    bhat, bhat not of order 7; Verner's structure: explicit, row sums c,
    c_9 = c_10 = 1, stages 2 and 3 unweighted and stage 2 used only by stage 3,
    stage 10 feeding only the embedded formula. The table's entries reach 187,
    whose double has an ulp of 2.8e-14: the residuals of the rounded table are
    ~4e-15 (row sums ~1e-14), against ~1e-8 for a coefficient changed in its
    ninth digit (test_planted_coefficient_error_is_detected)."""
    tab = oracle.tableau(oracle.METHOD_VERNER7)
    A, b, bh, c = tab["A"], tab["b"], tab["bhat"], tab["c"]
    Z = np.zeros_like(A)
    r7 = residuals(A, Z, b, 7)
    r6 = residuals(A, Z, bh, 6)
    assert len(r7) == 85 and len(r6) == 37
    assert max(abs(r) for _, r in r7) < 1e-14
    assert max(abs(r) for _, r in r6) < 1e-14
    assert max(abs(r) for _, r in residuals(A, Z, bh, 7)) > 1e-5
    np.testing.assert_allclose(A.sum(1), c, atol=3e-14)
    assert c[8] == 1.0 and c[9] == 1.0
    assert np.allclose(np.tril(A, -1), A)
    assert b[1] == b[2] == bh[1] == bh[2] == 0.0 and b[9] == 0.0 and bh[9] != 0.0
    assert (A[3:, 1] == 0.0).all() and (A[:9, 9] == 0.0).all()


def _quadrature_weights(c, cols, p):
    """The unique weights w on the nodes c[cols] with sum_j w_j c_j^k = 1/(k+1),
    k = 0..p-1 (a Vandermonde system), in exact rational arithmetic on the
    doubles c."""
    from fractions import Fraction
    import sympy
    M = sympy.Matrix([[Fraction(float(c[j])) ** k for j in cols] for k in range(p)])
    rhs = sympy.Matrix([sympy.Rational(1, k + 1) for k in range(p)])
    return [float(x) for x in M.LUsolve(rhs)]


def test_verner7_weights_are_the_quadrature_weights_of_its_nodes():
    """With seven nonzero 7th-order weights (stages 1, 4..9) and six nonzero
    6th-order weights (stages 1, 4..7, 10), the bushy-tree conditions
    sum_j b_j c_j^k = 1/(k+1) alone fix b and bhat from the nodes: the pair's
    weights must be those quadrature weights (to the rounding of the nodes)."""
    tab = oracle.tableau(oracle.METHOD_VERNER7)
    b, bh, c = tab["b"], tab["bhat"], tab["c"]
    wb = _quadrature_weights(c, [0, 3, 4, 5, 6, 7, 8], 7)
    wh = _quadrature_weights(c, [0, 3, 4, 5, 6, 9], 6)
    np.testing.assert_allclose(b[[0, 3, 4, 5, 6, 7, 8]], wb, rtol=0, atol=1e-15)
    np.testing.assert_allclose(bh[[0, 3, 4, 5, 6, 9]], wh, rtol=0, atol=1e-15)


def test_planted_coefficient_error_is_detected():
    # A perturbation in the 9th digit of one coefficient must break a condition.
    tab = oracle.tableau(oracle.METHOD_TSIT5)
    A = tab["A"].copy()
    A[4, 2] *= 1 + 1e-9
    bad = residuals(A, np.zeros_like(A), A[6], 5)
    assert max(abs(r) for _, r in bad) > 10 * TOL
    rt = oracle.tableau(oracle.METHOD_RODAS5P)
    rt["C"] = rt["C"].copy()
    rt["C"][5, 2] *= 1 + 1e-9
    alpha, G, b = rodas_standard(rt)
    assert max(abs(r) for _, r in residuals(alpha, G, b, 5)) > 10 * TOL
    vt = oracle.tableau(oracle.METHOD_VERNER7)
    A = vt["A"].copy()
    A[6, 3] *= 1 + 1e-9
    assert max(abs(r) for _, r in residuals(A, np.zeros_like(A), vt["b"], 7)) > 1e-12
