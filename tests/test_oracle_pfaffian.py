"""Pins of the oracle's Pfaffian (Parlett-Reid with pivoting) against definitions that do
not use it: the sum over perfect matchings, Pf^2 = det, Pf(B A B^T) = det(B) Pf(A)."""
import numpy as np
import pytest

from oracle import native
from paper_2410_04204_gb300 import inputs


def pf_matchings(a):
    """Pf(A) = sum_j (-1)^(j+1) A[0, j] Pf(A without rows/cols 0, j)  (expansion over matchings)."""
    n = a.shape[0]
    if n == 0:
        return 1.0 + 0j
    if n % 2:
        return 0j
    tot = 0j
    for j in range(1, n):
        keep = [x for x in range(n) if x not in (0, j)]
        tot += (-1) ** (j + 1) * a[0, j] * pf_matchings(a[np.ix_(keep, keep)])
    return tot


@pytest.mark.parametrize("n", [2, 4, 6, 8, 10])
@pytest.mark.parametrize("cplx", [False, True])
def test_pfaffian_matches_perfect_matchings(n, cplx):
    for a in inputs.random_skew(n, 3, tag=n, complex_=cplx):
        assert abs(native.pfaffian(a) - pf_matchings(a)) <= 1e-12 * max(1.0, abs(pf_matchings(a)))


@pytest.mark.parametrize("n", [2, 6, 12, 20, 32, 40])
def test_pfaffian_squared_is_determinant(n):
    for a in inputs.random_skew(n, 2, tag=100 + n, complex_=True):
        pf = native.pfaffian(a)
        det = np.linalg.det(a)
        assert abs(pf * pf - det) <= 1e-10 * max(1.0, abs(det))


def test_pfaffian_odd_is_zero():
    for n in (1, 3, 9):
        assert native.pfaffian(inputs.random_skew(n, 1, tag=n, complex_=True)[0]) == 0


def test_pfaffian_congruence():
    g = inputs.rng(7)
    for n in (4, 8, 14):
        a = inputs.random_skew(n, 1, tag=n, complex_=True)[0]
        b = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
        lhs = native.pfaffian(b @ a @ b.T)
        rhs = np.linalg.det(b) * native.pfaffian(a)
        assert abs(lhs - rhs) <= 1e-9 * abs(rhs)


def test_pfaffian_special_cases():
    # Pf of the canonical block diag(J, J, ...) with J = [[0, x], [-x, 0]] is prod x
    xs = [1.5, -2.0, 0.25j]
    a = np.zeros((6, 6), complex)
    for i, x in enumerate(xs):
        a[2 * i, 2 * i + 1], a[2 * i + 1, 2 * i] = x, -x
    assert abs(native.pfaffian(a) - np.prod(xs)) < 1e-15
    assert native.pfaffian(np.zeros((0, 0))) == 1.0
    assert native.pfaffian(np.zeros((4, 4))) == 0.0
    # a row permutation that needs pivoting (zero in the natural pivot slot)
    p = np.zeros((4, 4))
    p[0, 2], p[1, 3] = 1.0, 1.0
    p = p - p.T
    assert abs(native.pfaffian(p) - pf_matchings(p)) < 1e-15
